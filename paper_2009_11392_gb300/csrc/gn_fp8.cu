// e4m3 operand preparation for the block-scaled tensor-core sketch: one
// power-of-two scale per 128 x 128 tile, codes in both orientations (the
// tensor cores read every e4m3 operand K-major), the 512-byte scale-factor
// images the sketch kernel copies into tensor memory, and an exact BF16
// expansion of an e4m3 operand for the split-precision core product.
#include "gn_internal.cuh"

#include <cuda_fp8.h>

namespace gn {
namespace {

constexpr int QT = 128;          // tile edge
constexpr int Q_THREADS = 256;
constexpr int QLD = QT + 1;      // padded smem row (floats)

// Smallest e with amax <= 448 * 2^e, within [-127, 127]; 0 for amax == 0.
// amax = 1.f * 2^(F-127) for a normal FP32 (F = biased exponent field): in
// frexp form (m in [0.5, 1)) the exponent is F - 126 and m <= 0.875 iff the
// fraction field is at most 0.75 * 2^23.  Subnormal maxima clamp to -127.
__device__ __forceinline__ int tile_exponent(float amax) {
    const uint32_t b = __float_as_uint(amax);
    const int F = static_cast<int>((b >> 23) & 0xFF);
    if (amax == 0.0f) return 0;
    if (F == 0) return -127;
    const int E = F - 126;
    const int e = (b & 0x7FFFFF) <= 0x600000u ? E - 9 : E - 8;
    return e < -127 ? -127 : (e > 127 ? 127 : e);
}

// 2^k as an FP32 for k in [-127, 127] (2^-127 is subnormal).
__device__ __forceinline__ float exp2i(int k) {
    return k >= -126 ? __uint_as_float(static_cast<uint32_t>(k + 127) << 23) : __uint_as_float(0x00400000u);
}

// Two FP32 values -> two e4m3 codes (round to nearest even, saturating);
// lo lands in the low byte (the lower address).
__device__ __forceinline__ uint32_t cvt_e4m3x2(float lo, float hi) {
    uint16_t d;
    asm("{\n\t.reg .b16 t;\n\tcvt.rn.satfinite.e4m3x2.f32 t, %1, %2;\n\tmov.b16 %0, t;\n\t}"
        : "=h"(d)
        : "f"(hi), "f"(lo));
    return d;
}

__global__ void __launch_bounds__(Q_THREADS) quantize_e4m3_kernel(const void* __restrict__ src, int src_f64,
                                                                  long long rows, long long cols, long long lds,
                                                                  uint8_t* __restrict__ dst, long long ld,
                                                                  uint8_t* __restrict__ dst_t, long long ld_t,
                                                                  uint8_t* __restrict__ scale) {
    extern __shared__ float tile[];   // [QT][QLD]
    __shared__ float red[Q_THREADS / 32];
    __shared__ float s_scale;
    const long long r0 = static_cast<long long>(blockIdx.y) * QT, c0 = static_cast<long long>(blockIdx.x) * QT;
    const int tid = threadIdx.x;
    float amax = 0.0f;
    for (int e = tid; e < QT * QT; e += Q_THREADS) {
        const int i = e >> 7, j = e & (QT - 1);
        const long long gi = r0 + i, gj = c0 + j;
        float v = 0.0f;
        if (gi < rows && gj < cols) {
            v = src_f64 ? static_cast<float>(static_cast<const double*>(src)[gi * lds + gj])
                        : static_cast<const float*>(src)[gi * lds + gj];
        }
        tile[i * QLD + j] = v;
        amax = fmaxf(amax, fabsf(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((tid & 31) == 0) red[tid >> 5] = amax;
    __syncthreads();
    if (tid == 0) {
        float a = 0.0f;
        for (int w = 0; w < Q_THREADS / 32; ++w) a = fmaxf(a, red[w]);
        const int e = tile_exponent(a);
        s_scale = exp2i(-e);
        scale[static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x] = static_cast<uint8_t>(e + 127);
    }
    __syncthreads();
    const float sc = s_scale;
    // 16-byte chunks: 128 rows x 8 chunks per orientation
    for (int ch = tid; ch < QT * (QT / 16); ch += Q_THREADS) {
        const int i = ch >> 3, j0 = (ch & 7) * 16;
        uint32_t w[4];
        if (dst) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float* t = tile + i * QLD + j0 + 4 * q;
                w[q] = cvt_e4m3x2(t[0] * sc, t[1] * sc) | (cvt_e4m3x2(t[2] * sc, t[3] * sc) << 16);
            }
            const long long gi = r0 + i, gj = c0 + j0;
            if (gi < rows) {
                uint8_t* d = dst + gi * ld + gj;
                if (gj + 16 <= cols) {
                    *reinterpret_cast<uint4*>(d) = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
                    for (int b = 0; b < 16 && gj + b < cols; ++b) d[b] = static_cast<uint8_t>(w[b >> 2] >> (8 * (b & 3)));
                }
            }
        }
        if (dst_t) {   // row j of the transposed tile = column j of this tile
            const int jt = i, it0 = j0;   // reuse the chunk index: column jt, rows it0 .. it0 + 15
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float* t = tile + (it0 + 4 * q) * QLD + jt;
                w[q] = cvt_e4m3x2(t[0] * sc, t[QLD] * sc) | (cvt_e4m3x2(t[2 * QLD] * sc, t[3 * QLD] * sc) << 16);
            }
            const long long gr = c0 + jt, gc = r0 + it0;   // position in the transpose
            if (gr < cols) {
                uint8_t* d = dst_t + gr * ld_t + gc;
                if (gc + 16 <= rows) {
                    *reinterpret_cast<uint4*>(d) = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
                    for (int b = 0; b < 16 && gc + b < rows; ++b) d[b] = static_cast<uint8_t>(w[b >> 2] >> (8 * (b & 3)));
                }
            }
        }
    }
}

__global__ void sf_image_kernel(const uint8_t* __restrict__ scale, long long tiles, uint4* __restrict__ image) {
    const long long total = tiles * 32;   // 32 x 16 bytes per tile
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const uint32_t b = scale[e >> 5];
        const uint32_t w = b * 0x01010101u;
        image[e] = make_uint4(w, w, w, w);
    }
}

// out (cols x rows of the original, BF16) from data_t (cols x rows, e4m3): the
// element at (i, j) of the transpose belongs to original tile (j/128, i/128).
__global__ void e4m3_t_to_bf16_kernel(const uint8_t* __restrict__ data_t, long long ld_t,
                                      const uint8_t* __restrict__ scale, long long rows, long long cols,
                                      __nv_bfloat16* __restrict__ out, long long ldo) {
    const long long tc = (cols + QT - 1) / QT;   // tile columns of the original
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / rows, j = e % rows;   // transpose row i (original column), column j
        __nv_fp8_e4m3 c;
        c.__x = data_t[i * ld_t + j];
        const int ex = static_cast<int>(scale[(j / QT) * tc + i / QT]) - 127;
        out[i * ldo + j] = __float2bfloat16_rn(static_cast<float>(c) * exp2i(ex));
    }
}

int grid_for(gn_handle h, long long work) {
    const long long b = (work + 255) / 256;
    const long long cap = static_cast<long long>(h->sm_count) * 8;
    return static_cast<int>(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

gn_status quantize_e4m3(gn_handle h, const void* src, int src_f64, long long rows, long long cols, long long lds,
                        uint8_t* dst, long long ld, uint8_t* dst_t, long long ld_t, uint8_t* scale) {
    if (!src || !scale || rows <= 0 || cols <= 0) return GN_ERR_INVALID_ARG;
    if ((dst && ((reinterpret_cast<uintptr_t>(dst) & 15) || ld % 16 || ld < cols)) ||
        (dst_t && ((reinterpret_cast<uintptr_t>(dst_t) & 15) || ld_t % 16 || ld_t < rows)))
        return GN_ERR_ALIGNMENT;
    static bool attr = false;
    const int smem = QT * QLD * static_cast<int>(sizeof(float));
    if (!attr) {
        GN_CUDA_TRY(cudaFuncSetAttribute(quantize_e4m3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    const dim3 grid(static_cast<unsigned>((cols + QT - 1) / QT), static_cast<unsigned>((rows + QT - 1) / QT));
    quantize_e4m3_kernel<<<grid, Q_THREADS, smem, h->stream>>>(src, src_f64, rows, cols, lds, dst, ld, dst_t, ld_t,
                                                              scale);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status e4m3_sf_image(gn_handle h, const uint8_t* scale, long long tiles, uint8_t* image) {
    if ((reinterpret_cast<uintptr_t>(image) & 15) != 0) return GN_ERR_ALIGNMENT;
    sf_image_kernel<<<grid_for(h, tiles * 32), 256, 0, h->stream>>>(scale, tiles, reinterpret_cast<uint4*>(image));
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status e4m3_t_to_bf16(gn_handle h, const uint8_t* data_t, long long ld_t, const uint8_t* scale,
                         long long rows, long long cols, __nv_bfloat16* out, long long ldo) {
    e4m3_t_to_bf16_kernel<<<grid_for(h, rows * cols), 256, 0, h->stream>>>(data_t, ld_t, scale, rows, cols, out,
                                                                           ldo);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

}  // namespace gn

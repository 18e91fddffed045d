// FP64 matrix products on the BF16 tensor cores by exact digit slicing.
//
// The splitting is the error-free transformation of matrix products of Ozaki,
// Ogita, Oishi and Rump (Numer. Algorithms 59, 2012), here with BF16 digits and
// the FP32 accumulators of tcgen05:
//   * every row i of A (over the K range of one pass) is scaled by 2^-ea_i so that
//     its entries lie in (-1/2, 1/2), and written as sum_s d_s 2^{-7(s+1)} with
//     signed integer digits |d_s| <= 64 (round to nearest at each step, so every
//     remainder stays in [-1/2, 1/2]); slice s holds d_s 2^{-7(s+1)}, exact in
//     BF16.  Columns of B the same with 2^-eb_j.
//   * the slice products of one order o = s + t carry the unit 2^{-7(o+2)}; each
//     term is at most 2^12 units, so the FP32 accumulation of the (o+1) products
//     of order o over K terms is exact while (o+1) K 2^12 <= 2^24.  A pass covers
//     at most 1024 of K: orders 0..3 are exact; orders 4..6 are rounded, their
//     rounding sits below 2^-52 of the leading term.
//   * one launch of the multi-GEMM engine computes D_o = sum_{s+t=o} A_s B_t for
//     every kept order; C = beta C + alpha 2^{ea_i + eb_j} sum_o D_o in FP64.
// Orders above 6 are dropped: with 7 digits per operand the error per element is
// about 2^-46 K max_k|a_ik| max_k|b_kj|, the size of an FP64 product's own
// worst-case rounding error.  FP32 operands take 7 digits too: the digits cover
// a window below the row's largest entry, not each entry's own 24 bits.
#include "gn_internal.cuh"

#include <algorithm>

namespace gn {
namespace {

constexpr int OZ_KPASS = 1024;   // K per pass (exactness of the orders <= 3)
constexpr int OZ_NPANEL = 256;   // least N per GEMM launch (oz_npanel bounds the FP32 outputs)
constexpr int OZ_MAX_DIGITS = 7;

size_t al256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

// Columns of C per GEMM launch: at least 256, more while the FP32 outputs of all
// orders stay within 64 MB (short, wide products in one launch).
long long oz_npanel(long long M, long long N) {
    long long np = (64LL << 20) / (4LL * OZ_MAX_DIGITS * std::max<long long>(M, 1));
    np = std::max<long long>(np, OZ_NPANEL) / 16 * 16;
    return std::min<long long>(N, np);
}
long long r8(long long x) { return (x + 7) / 8 * 8; }
long long r4(long long x) { return (x + 3) / 4 * 4; }

// ---- digit extraction in integer arithmetic (the FP64 pipe is the slow one)
//
// |x| as an unsigned integer orders like |x| itself; the row exponent e comes
// from the largest one: |x| < 2^(e-1) for every entry of the row.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long abs_bits(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }

template <typename T>
__device__ __forceinline__ int row_exponent(unsigned long long mx);
template <>
__device__ __forceinline__ int row_exponent<double>(unsigned long long mx) {
    if (mx == 0) return 0;
    const int E = static_cast<int>(mx >> 52);
    return E == 0 ? -1021 : E - 1021;   // |x| < 2^(E-1022) = 2^(e-1)
}
template <>
__device__ __forceinline__ int row_exponent<float>(unsigned long long mx) {
    if (mx == 0) return 0;
    const int E = static_cast<int>(mx >> 23);
    return E == 0 ? -125 : E - 125;
}

// round(x 2^(49-e)) as a signed integer, |result| <= 2^48.
__device__ __forceinline__ long long fixed49(double x, int e) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const int E = static_cast<int>((b >> 52) & 0x7FF);
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
    const int sh = (E ? E : 1) - 1075 + 49 - e;   // x = mant 2^(E-1075); always < 0 for |x| < 2^(e-1) normal
    long long v;
    if (sh >= 0) v = static_cast<long long>(mant << sh);
    else if (sh > -64) v = static_cast<long long>((mant + (1ull << (-sh - 1))) >> (-sh));
    else v = 0;
    return (b >> 63) ? -v : v;
}
__device__ __forceinline__ long long fixed49(float x, int e) {
    const uint32_t b = __float_as_uint(x);
    const int E = static_cast<int>((b >> 23) & 0xFF);
    const unsigned long long mant = (b & 0x7FFFFFu) | (E ? 0x800000u : 0u);
    const int sh = (E ? E : 1) - 150 + 49 - e;
    long long v;
    if (sh >= 0) v = static_cast<long long>(mant << sh);
    else if (sh > -64) v = static_cast<long long>((mant + (1ull << (-sh - 1))) >> (-sh));
    else v = 0;
    return (b >> 31) ? -v : v;
}

// Signed base-2^7 digits of Y (round to nearest at each step): slice s holds
// d_s 2^{-7(s+1)}, Y 2^-49 = sum_s d_s 2^{-7(s+1)}, |d_s| <= 64.
__device__ __forceinline__ void write_digits(long long Y, int S, __nv_bfloat16* out, long long slice_stride) {
#pragma unroll
    for (int s = 0; s < OZ_MAX_DIGITS; ++s) {
        if (s >= S) break;
        const int sh = 7 * (OZ_MAX_DIGITS - 1 - s);
        const long long d = sh ? (Y + (1ll << (sh - 1))) >> sh : Y;
        Y -= d * (1ll << sh);
        out[s * slice_stride] = __float2bfloat16_rn(static_cast<float>(static_cast<int>(d)) *
                                                    __int_as_float((127 - 7 * (s + 1)) << 23));
    }
}

// Largest |entry| of every operand row, as the bits of |x|.  Rows contiguous
// along K (s_k == 1): a warp per row.
template <typename T>
__global__ void oz_rowmax_rows_kernel(const T* __restrict__ src, long long s_row, int rows, int K,
                                      unsigned long long* __restrict__ mx) {
    const long long w = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= rows) return;   // warp-uniform
    const T* row = src + w * s_row;
    unsigned long long m = 0;
    for (int k = lane; k < K; k += 32) m = max(m, abs_bits(row[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) mx[w] = m;
}

// Rows contiguous across rows (s_row == 1): blocks of 32 rows x one chunk of K,
// the 8 warps striding the chunk; atomicMax into mx (zeroed before).
template <typename T>
__global__ void oz_rowmax_cols_kernel(const T* __restrict__ src, long long s_k, int rows, int K, int kchunk,
                                      unsigned long long* __restrict__ mx) {
    __shared__ unsigned long long part[8][32];
    const int lane = threadIdx.x & 31, kg = threadIdx.x >> 5;
    const long long i = static_cast<long long>(blockIdx.x) * 32 + lane;
    const int k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
    unsigned long long m = 0;
    if (i < rows)
        for (int k = k0 + kg; k < k1; k += 8) m = max(m, abs_bits(src[i + k * s_k]));
    part[kg][lane] = m;
    __syncthreads();
    if (kg == 0 && i < rows) {
#pragma unroll
        for (int g = 1; g < 8; ++g) m = max(m, part[g][lane]);
        if (m) atomicMax(mx + i, m);
    }
}

// Digits, rows contiguous along K: one thread per entry, k fastest.
template <typename T>
__global__ void oz_digits_rows_kernel(const T* __restrict__ src, long long s_row, int rows, int K, int S,
                                      const unsigned long long* __restrict__ mx, __nv_bfloat16* __restrict__ out,
                                      long long ldk, long long slice_stride) {
    const long long total = static_cast<long long>(rows) * K;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / K, k = e - i * K;
        write_digits(fixed49(src[i * s_row + k], row_exponent<T>(mx[i])), S, out + i * ldk + k, slice_stride);
    }
}

// Digits, rows contiguous across rows: 32 x 32 tiles through shared memory,
// read along the rows, written along K.
template <typename T>
__global__ void oz_digits_cols_kernel(const T* __restrict__ src, long long s_k, int rows, int K, int S,
                                      const unsigned long long* __restrict__ mx, __nv_bfloat16* __restrict__ out,
                                      long long ldk, long long slice_stride) {
    __shared__ long long ys[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 256 threads
    const long long i0 = static_cast<long long>(blockIdx.x) * 32, k0 = static_cast<long long>(blockIdx.y) * 32;
    const long long i = i0 + tx;
    const int e = i < rows ? row_exponent<T>(mx[i]) : 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long k = k0 + ty + 8 * q;
        ys[ty + 8 * q][tx] = (i < rows && k < K) ? fixed49(src[i + k * s_k], e) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long ii = i0 + ty + 8 * q, kk = k0 + tx;
        if (ii < rows && kk < K) write_digits(ys[tx][ty + 8 * q], S, out + ii * ldk + kk, slice_stride);
    }
}

// C[i, j] = beta C[i, j] + alpha 2^{ea_i + eb_j} sum_o D_o[i, j].  The exact
// orders 0..3 are summed as integers in units of 2^-35 (one rounding), the
// rounded orders 4.. in FP32 below them.  A thread per column, rows across
// blockIdx.y (no division per element); each exact order is an integer below
// 2^24 units, so it converts through a 32-bit integer.
__global__ void oz_combine_kernel(const float* __restrict__ D, long long d_stride, long long ldd, int norders,
                                  int M, int N, const unsigned long long* __restrict__ mxa, int a_f32,
                                  const unsigned long long* __restrict__ mxb, double alpha, double beta,
                                  double* __restrict__ C, long long ldc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int eb = row_exponent<double>(mxb[j]);
    const int nexact = norders < 4 ? norders : 4;
    for (int i = blockIdx.y; i < M; i += gridDim.y) {
        const float* d = D + static_cast<long long>(i) * ldd + j;
        long long acc = 0;
        for (int o = 0; o < nexact; ++o)   // D_o is an integer number of units 2^{-7(o+2)}
            acc += static_cast<long long>(__float2int_rn(d[o * d_stride] * __int_as_float((127 + 7 * (o + 2)) << 23)))
                   << (7 * (3 - o));
        float low = 0.0f;
        for (int o = norders - 1; o >= 4; --o) low += d[o * d_stride];
        // times 2^(ea + eb - 35): a power of two built from its bits when normal
        const int ea = a_f32 ? row_exponent<float>(mxa[i]) : row_exponent<double>(mxa[i]);
        const int p = ea + eb - 35;
        const double x = fma(static_cast<double>(low), 34359738368.0, static_cast<double>(acc));
        const double v = (p >= -1022 && p <= 1023)
                             ? x * (alpha * __longlong_as_double(static_cast<long long>(p + 1023) << 52))
                             : alpha * ldexp(x, p);
        double* c = C + static_cast<long long>(i) * ldc + j;
        *c = beta == 0.0 ? v : fma(beta, *c, v);
    }
}

template <typename T>
gn_status slice(gn_handle h, const T* src, long long s_row, long long s_k, long long rows, long long K, int S,
                __nv_bfloat16* out, long long ldk, long long slice_stride, unsigned long long* mx) {
    if (s_k == 1) {
        oz_rowmax_rows_kernel<T><<<static_cast<unsigned>((rows * 32 + 255) / 256), 256, 0, h->stream>>>(
            src, s_row, static_cast<int>(rows), static_cast<int>(K), mx);
        count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        const long long total = rows * K;
        const long long blocks = std::min<long long>((total + 255) / 256, static_cast<long long>(h->sm_count) * 16);
        oz_digits_rows_kernel<T><<<static_cast<unsigned>(blocks), 256, 0, h->stream>>>(
            src, s_row, static_cast<int>(rows), static_cast<int>(K), S, mx, out, ldk, slice_stride);
    } else if (s_row == 1) {
        constexpr int KCHUNK = 64;
        GN_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * rows, h->stream));
        const dim3 g1(static_cast<unsigned>((rows + 31) / 32), static_cast<unsigned>((K + KCHUNK - 1) / KCHUNK));
        oz_rowmax_cols_kernel<T><<<g1, 256, 0, h->stream>>>(src, s_k, static_cast<int>(rows), static_cast<int>(K),
                                                            KCHUNK, mx);
        count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        const dim3 g2(static_cast<unsigned>((rows + 31) / 32), static_cast<unsigned>((K + 31) / 32));
        oz_digits_cols_kernel<T><<<g2, 256, 0, h->stream>>>(src, s_k, static_cast<int>(rows), static_cast<int>(K), S,
                                                            mx, out, ldk, slice_stride);
    } else {
        return GN_ERR_INVALID_ARG;
    }
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

struct OzWs {
    __nv_bfloat16 *as, *bs;
    float* d;
    unsigned long long *mxa, *mxb;
    long long ldk, ldd;
};

bool oz_carve(long long M, long long N, long long K, int sa, int sb, void* ws, size_t ws_bytes, OzWs* o) {
    const long long kp = std::min<long long>(K, OZ_KPASS), np = oz_npanel(M, N);
    o->ldk = r8(kp);
    o->ldd = r4(np);
    char* p = static_cast<char*>(ws);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* q = p + off;
        off += al256(bytes);
        return q;
    };
    o->as = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * sa * M * o->ldk));
    o->bs = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * sb * N * o->ldk));
    o->d = reinterpret_cast<float*>(take(sizeof(float) * OZ_MAX_DIGITS * M * o->ldd));
    o->mxa = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * M));
    o->mxb = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * N));
    return off <= ws_bytes;
}

}  // namespace

size_t oz_ws_bytes(long long M, long long N, long long K, int a_f32) {
    (void)a_f32;
    const int sa = OZ_MAX_DIGITS, sb = OZ_MAX_DIGITS;
    const long long kp = std::min<long long>(std::max<long long>(K, 1), OZ_KPASS);
    const long long np = oz_npanel(M, std::max<long long>(N, 1));
    return al256(sizeof(__nv_bfloat16) * sa * M * r8(kp)) + al256(sizeof(__nv_bfloat16) * sb * N * r8(kp)) +
           al256(sizeof(float) * OZ_MAX_DIGITS * M * r4(np)) + al256(8 * M) + al256(8 * N) + 256;
}

gn_status oz_dgemm(gn_handle h, long long M, long long N, long long K, double alpha, const void* A, int a_f32,
                   long long lda, int ta, const double* B, long long ldb, int tb, double beta, double* C,
                   long long ldc, void* ws, size_t ws_bytes, int digits) {
    if (M <= 0 || N <= 0) return GN_OK;
    if (K <= 0 || !A || !B || !C || !ws || digits < 2 || digits > OZ_MAX_DIGITS) return GN_ERR_INVALID_ARG;
    const int sa = digits, sb = digits;
    if (M > (1LL << 30) || N > (1LL << 30)) return GN_ERR_SHAPE;
    OzWs o;
    if (!oz_carve(M, N, K, sa, sb, ws, ws_bytes, &o)) return GN_ERR_WORKSPACE;
    const int omax = std::max(sa, sb) - 1;   // kept orders 0 .. omax
    int norders = 0, pairs[OZ_MAX_DIGITS][2 * OZ_MAX_DIGITS][2], npairs[OZ_MAX_DIGITS];
    for (int ord = 0; ord <= omax; ++ord) {
        npairs[ord] = 0;
        for (int s = 0; s < sa; ++s) {
            const int t = ord - s;
            if (t < 0 || t >= sb) continue;
            pairs[ord][npairs[ord]][0] = s;
            pairs[ord][npairs[ord]][1] = t;
            ++npairs[ord];
        }
        if (npairs[ord] > 0) norders = ord + 1;
    }
    // every order 0 .. omax has the pair (0, ord): no order is empty
    if (norders > TC_MAX_GEMMS || sa + sb > TC_MAX_MAPS || npairs[omax] > TC_MAX_SRC) return GN_ERR_UNSUPPORTED;
    const long long as_stride = M * o.ldk, bs_stride = N * o.ldk, d_stride = M * o.ldd;
    for (long long k0 = 0; k0 < K; k0 += OZ_KPASS) {
        const long long kc = std::min<long long>(OZ_KPASS, K - k0);
        // A rows (i over M, k along the pass) and B "rows" (j over N)
        const long long a_row = ta ? 1 : lda, a_k = ta ? lda : 1;
        const long long a_off = ta ? k0 * lda : k0;
        if (a_f32)
            GN_TRY(slice(h, static_cast<const float*>(A) + a_off, a_row, a_k, M, kc, sa, o.as, o.ldk, as_stride, o.mxa));
        else
            GN_TRY(slice(h, static_cast<const double*>(A) + a_off, a_row, a_k, M, kc, sa, o.as, o.ldk, as_stride,
                         o.mxa));
        const long long b_row = tb ? ldb : 1, b_k = tb ? 1 : ldb;
        const long long b_off = tb ? k0 : k0 * ldb;
        GN_TRY(slice(h, B + b_off, b_row, b_k, N, kc, sb, o.bs, o.ldk, bs_stride, o.mxb));
        const double beta_pass = k0 == 0 ? beta : 1.0;
        const long long npanel = oz_npanel(M, N);
        for (long long j0 = 0; j0 < N; j0 += npanel) {
            const long long nb = std::min<long long>(npanel, N - j0);
            // N tile: the widest of 256 / 128 / 64 that still gives the GPU about
            // two tiles per SM over the orders (small products are latency-bound)
            int bn = static_cast<int>(std::min<long long>(256, (nb + 31) / 32 * 32));
            while (bn > 64 && ((M + 127) / 128) * ((nb + bn - 1) / bn) * norders < 2LL * h->sm_count)
                bn = (bn / 2 + 31) / 32 * 32;
            TcParams p;
            memset(&p, 0, sizeof(p));
            for (int s = 0; s < sa; ++s)
                GN_TRY(tc_make_map_bf16(&p.maps[s], o.as + s * as_stride, M, kc, o.ldk, 64, 128));
            for (int t = 0; t < sb; ++t)
                GN_TRY(tc_make_map_bf16(&p.maps[sa + t], o.bs + t * bs_stride + j0 * o.ldk, nb, kc, o.ldk, 64, bn));
            // the orders with the most slice products first (the longest tiles)
            int order_of[OZ_MAX_DIGITS];
            for (int i = 0; i < norders; ++i) order_of[i] = i;
            std::stable_sort(order_of, order_of + norders, [&](int a, int b) { return npairs[a] > npairs[b]; });
            for (int gi = 0; gi < norders; ++gi) {
                const int ord = order_of[gi];
                TcGemm& g = p.g[gi];
                g.M = static_cast<int>(M);
                g.N = static_cast<int>(nb);
                g.K = static_cast<int>(kc);
                g.bn = bn;
                g.a_mn = 0;
                g.b_mn = 0;
                g.nsrc = npairs[ord];
                for (int q = 0; q < npairs[ord]; ++q) {
                    g.a_map[q] = pairs[ord][q][0];
                    g.b_map[q] = sa + pairs[ord][q][1];
                }
                g.D = o.d + ord * d_stride;
                g.ldd = o.ldd;
            }
            p.ngemm = norders;
            GN_TRY(tc_launch(h, &p));
            const unsigned gx = static_cast<unsigned>((nb + 255) / 256);
            const unsigned gy = static_cast<unsigned>(
                std::max<long long>(1, std::min<long long>(M, static_cast<long long>(h->sm_count) * 16 / gx)));
            oz_combine_kernel<<<dim3(gx, gy), 256, 0, h->stream>>>(
                o.d, d_stride, o.ldd, norders, static_cast<int>(M), static_cast<int>(nb), o.mxa, a_f32, o.mxb + j0,
                alpha, beta_pass, C + j0, ldc);
            count_launch();
            GN_CUDA_TRY(cudaGetLastError());
        }
    }
    return GN_OK;
}

}  // namespace gn

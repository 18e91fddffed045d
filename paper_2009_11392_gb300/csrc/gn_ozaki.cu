// FP64 matrix products on the BF16 tensor cores by exact digit slicing.
//
// The splitting is the error-free transformation of matrix products of Ozaki,
// Ogita, Oishi and Rump (Numer. Algorithms 59, 2012), here with BF16 digits and
// the FP32 accumulators of tcgen05:
//   * every row i of A (over the K range of one pass) is scaled by 2^-ea_i so that
//     its entries lie in (-1/2, 1/2), rounded to 49 fractional bits and written
//     as sum_s d_s 2^{-7(s+1)} with balanced base-128 digits |d_s| <= 64 (the
//     plain digits of the value plus a bias of 64 per position, less 64); slice
//     s holds d_s 2^{-7(s+1)}, exact in BF16.  Columns of B the same with 2^-eb_j.
//     Both operands of up to four passes are sliced in one launch.
//   * the slice products of one order o = s + t carry the unit 2^{-7(o+2)}; each
//     term is at most 2^12 units, so the FP32 accumulation of the (o+1) products
//     of order o over K terms is exact while (o+1) K 2^12 <= 2^24.  A pass covers
//     at most 1024 of K: orders 0..3 are exact; orders 4..6 are rounded, their
//     rounding sits below 2^-52 of the leading term.
//   * one launch of the multi-GEMM engine computes D_o = sum_{s+t=o} A_s B_t for
//     every kept order and every pass of the group (the passes as K-aligned
//     parts stored apart; the orders of 7, 6, ..., 1 slice products paired on
//     the CTAs by the boustrophedon tile order); C = beta C + sum over the
//     passes of alpha 2^{ea_i + eb_j} sum_o D_o in FP64, the passes in order.
// Orders above 6 are dropped: with 7 digits per operand the error per element is
// about 2^-46 K max_k|a_ik| max_k|b_kj|, the size of an FP64 product's own
// worst-case rounding error.  FP32 operands take 7 digits too: the digits cover
// a window below the row's largest entry, not each entry's own 24 bits.
#include "gn_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace gn {
namespace {

constexpr int OZ_KPASS = 1024;   // K per pass (exactness of the orders <= 3)
constexpr int OZ_NPANEL = 256;   // least N per GEMM launch (oz_npanel bounds the FP32 outputs)
constexpr int OZ_MAX_DIGITS = 7;
constexpr int OZ_PGRP = 4;       // passes per group of launches (slicing, products, combination)

size_t al256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

// Columns of C per GEMM launch: at least 256, more while the FP32 outputs of all
// orders and K parts stay within 64 MB (short, wide products in one launch).
long long oz_npanel(long long M, long long N, long long parts) {
    long long np = (64LL << 20) / (4LL * OZ_MAX_DIGITS * std::max<long long>(M, 1) * std::max<long long>(parts, 1));
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

// Signed base-2^7 digits of Y (|Y| <= 2^48): slice s holds d_s 2^{-7(s+1)},
// |d_s| <= 64.  With a bias of 64 in each kept digit position (plus half of the
// last kept unit when S < 7), U = Y + bias >= 0 has plain base-128 digits u_s,
// and d_s = u_s - 64: the S digits sum to Y exactly for S = 7 and to Y rounded
// to the last kept unit (nearest, ties up) for S < 7.  Bit fields of one 64-bit
// integer, no carries to propagate.
__device__ __forceinline__ unsigned long long digit_bias(int S) {
    unsigned long long b = 0;
#pragma unroll
    for (int s = 0; s < OZ_MAX_DIGITS; ++s)
        if (s < S) b += 64ull << (7 * (OZ_MAX_DIGITS - 1 - s));
    if (S < OZ_MAX_DIGITS) b += 1ull << (7 * (OZ_MAX_DIGITS - S) - 1);
    return b;
}

// Digits of two entries adjacent along K, stored as one bf16 pair per slice
// (out 4-byte aligned, slice_stride even).
__device__ __forceinline__ void write_digits2(long long Y0, long long Y1, int S, unsigned long long bias,
                                              __nv_bfloat16* out, long long slice_stride) {
    const unsigned long long U0 = static_cast<unsigned long long>(Y0) + bias;
    const unsigned long long U1 = static_cast<unsigned long long>(Y1) + bias;
#pragma unroll
    for (int s = 0; s < OZ_MAX_DIGITS; ++s) {
        if (s >= S) break;
        const int sh = 7 * (OZ_MAX_DIGITS - 1 - s);
        const unsigned u0 = s ? static_cast<unsigned>(U0 >> sh) & 127u : static_cast<unsigned>(U0 >> sh);
        const unsigned u1 = s ? static_cast<unsigned>(U1 >> sh) & 127u : static_cast<unsigned>(U1 >> sh);
        const float sc = __int_as_float((127 - 7 * (s + 1)) << 23);   // 2^{-7(s+1)}
        const float2 f = make_float2(fmaf(__uint2float_rn(u0), sc, -64.0f * sc), fmaf(__uint2float_rn(u1), sc, -64.0f * sc));
        *reinterpret_cast<__nv_bfloat162*>(out + s * slice_stride) = __float22bfloat162_rn(f);
    }
}

// ---- slicing of both operands of one pass in one launch
//
// An operand is `rows` rows of K entries (row i, entry k at src[i s_row + k s_k];
// one of the strides is 1).  Its slices go to out[s slice_stride + i ldk + k] and
// the bits of max_k |x_ik| to mx[i].  FP32 sources are widened to FP64 on load
// (exact), so mx always holds FP64 bits.
struct OzOperand {
    const void* src;   // FP32 for operand 0 of the FP32-A instance, FP64 otherwise
    long long s_row, s_k, ldk, slice_stride;
    __nv_bfloat16* out;
    unsigned long long* mx;   // [passes][rows]
    int rows, K, S;
    int passes;     // ceil(K / OZ_KPASS): pass p is K range [p OZ_KPASS, min(K, (p + 1) OZ_KPASS))
    int tpr;        // K contiguous: threads per row, 32 (K <= 256) or 128
    int rpc;        // rows per cluster: OZ_CS OZ_ST / tpr (K contiguous) or 32 (rows contiguous)
    int clusters;   // passes x ceil(rows / rpc): one cluster of OZ_CS CTAs per pass and rpc rows
};
struct OzSliceArgs {
    OzOperand op[2];
};

constexpr int OZ_CS = 8;                      // CTAs per cluster (the K split of a strided operand)
constexpr int OZ_ST = 512;                    // threads per CTA
constexpr int OZ_NW = OZ_ST / 32;
constexpr int OZ_KC_MAX = OZ_KPASS / OZ_CS;   // K per CTA of a strided operand (<= 128)

struct OzSmem {
    long long ys[OZ_KC_MAX][33];
    unsigned long long part[OZ_NW][32];
    unsigned long long lmax[32], rmax[32];
};

// mx[i] in FP64 form for the combine: the largest |entry| itself for FP64 rows;
// for FP32 rows an FP64 power of two with the same row exponent.
__device__ __forceinline__ unsigned long long mx_word(unsigned long long m, double*) { return m; }
__device__ __forceinline__ unsigned long long mx_word(unsigned long long m, float*) {
    return m ? static_cast<unsigned long long>(row_exponent<float>(m) + 1021) << 52 : 0ull;
}

// K contiguous (s_k == 1): tpr threads per row (a warp when K <= 256, else four
// warps), OZ_ST / tpr rows per CTA, pairs of entries along K (8 entries per
// thread); the row maximum is a shuffle, plus an exchange between the row's
// warps when there are four.
template <typename T>
__device__ __forceinline__ void slice_kcontig(const OzOperand& o, int pass, int q, int rank, OzSmem& sm) {
    const long long koff = static_cast<long long>(pass) * OZ_KPASS;
    const T* src = static_cast<const T*>(o.src) + koff;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tpr = o.tpr;   // uniform over the cluster
    const int r = tid / tpr, l = tid - r * tpr;
    const long long i = static_cast<long long>(q) * o.rpc + rank * (OZ_ST / tpr) + r;
    const bool live = i < o.rows;
    const int K = min(OZ_KPASS, o.K - pass * OZ_KPASS);   // <= 8 tpr
    T v[8];
    unsigned long long m = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int k = 2 * l + 2 * tpr * u;
        v[2 * u] = live && k < K ? src[i * o.s_row + k] : T(0);
        v[2 * u + 1] = live && k + 1 < K ? src[i * o.s_row + k + 1] : T(0);
        m = max(m, max(abs_bits(v[2 * u]), abs_bits(v[2 * u + 1])));
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, s));
    if (tpr > 32) {   // four warps per row
        if (lane == 0) sm.part[warp][0] = m;
        __syncthreads();
        m = max(max(sm.part[4 * r][0], sm.part[4 * r + 1][0]), max(sm.part[4 * r + 2][0], sm.part[4 * r + 3][0]));
    }
    if (!live) return;   // no barrier follows in this path
    if (l == 0) o.mx[static_cast<long long>(pass) * o.rows + i] = mx_word(m, static_cast<T*>(nullptr));
    const int e = row_exponent<T>(m);
    const unsigned long long bias = digit_bias(o.S);
    __nv_bfloat16* out = o.out + i * o.ldk + koff;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int k = 2 * l + 2 * tpr * u;   // k + 1 < ldk: ldk is K rounded up to 8
        if (k < K) write_digits2(fixed49(v[2 * u], e), fixed49(v[2 * u + 1], e), o.S, bias, out + k, o.slice_stride);
    }
}

// Rows contiguous (s_row == 1): the cluster's 8 CTAs split K into chunks of
// <= 128; a CTA reads its 32 x chunk block along the rows (coalesced, 8
// entries per thread), the partial row maxima go through distributed shared
// memory, and the digits are written along K after a transpose in shared memory.
template <typename T>
__device__ __forceinline__ void slice_strided(const OzOperand& o, int pass, int q, int rank, OzSmem& sm) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const long long koff = static_cast<long long>(pass) * OZ_KPASS;
    const T* src = static_cast<const T*>(o.src) + koff * o.s_k;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = min(OZ_KPASS, o.K - pass * OZ_KPASS);
    const int kc = ((K + OZ_CS - 1) / OZ_CS + 7) / 8 * 8;   // <= 128, a multiple of 8
    const int k0 = rank * kc, k1 = min(K, k0 + kc);
    const long long i = static_cast<long long>(q) * 32 + lane;
    const bool live = i < o.rows;
    T v[8];
    unsigned long long m = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int k = k0 + warp + OZ_NW * u;
        v[u] = live && k < k1 ? src[i + static_cast<long long>(k) * o.s_k] : T(0);
        m = max(m, abs_bits(v[u]));
    }
    sm.part[warp][lane] = m;
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int g = 1; g < OZ_NW; ++g) m = max(m, sm.part[g][lane]);
        sm.lmax[lane] = m;
    }
    cluster.sync();   // every CTA's partial maxima written
    if (warp == 0) {
        unsigned long long mr = 0;
#pragma unroll
        for (int c = 0; c < OZ_CS; ++c) mr = max(mr, cluster.map_shared_rank(sm.lmax, c)[lane]);
        sm.rmax[lane] = mr;
        if (rank == 0 && live) o.mx[static_cast<long long>(pass) * o.rows + i] = mx_word(mr, static_cast<T*>(nullptr));
    }
    cluster.sync();   // peers' reads of lmax done before any CTA moves on or exits
    const int e = row_exponent<T>(sm.rmax[lane]);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int kk = warp + OZ_NW * u;
        if (kk < kc) sm.ys[kk][lane] = fixed49(v[u], e);
    }
    __syncthreads();
    const int w = k1 - k0;
    if (w <= 0) return;
    // pairs along K: w is a multiple of 8 except in the last chunk, where an odd
    // w pairs the last entry with the zero row kk = w < kc (column K < ldk).
    // Thread: pair kp = tid % 64, rows tid / 64 + 8 j.
    const int wp = (w + 1) / 2, kp = tid & 63;
    if (kp >= wp) return;
    const unsigned long long bias = digit_bias(o.S);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int ii = (tid >> 6) + 8 * j;
        const long long row = static_cast<long long>(q) * 32 + ii;
        if (row < o.rows)
            write_digits2(sm.ys[2 * kp][ii], sm.ys[2 * kp + 1][ii], o.S, bias, o.out + row * o.ldk + koff + k0 + 2 * kp,
                          o.slice_stride);
    }
}

// Cluster q of the grid slices pass p, rows [rpc q', rpc q' + rpc) of operand 0
// (FP32 when A32) for q < op[0].clusters, else of operand 1 (FP64), with
// q - (operand base) = p ceil(rows / rpc) + q'.
template <bool A32>
__global__ void __launch_bounds__(OZ_ST) oz_slice_kernel(const __grid_constant__ OzSliceArgs args) {
    __shared__ OzSmem sm;
    const int rank = static_cast<int>(cooperative_groups::this_cluster().block_rank());
    int q = static_cast<int>(blockIdx.x) / OZ_CS;
    const int which = q < args.op[0].clusters ? 0 : 1;
    const OzOperand& o = args.op[which];
    if (which) q -= args.op[0].clusters;
    const int rq = (o.rows + o.rpc - 1) / o.rpc;
    const int pass = q / rq;
    q -= pass * rq;
    if (which == 0 && A32) {
        if (o.s_k == 1) slice_kcontig<float>(o, pass, q, rank, sm);
        else slice_strided<float>(o, pass, q, rank, sm);
    } else {
        if (o.s_k == 1) slice_kcontig<double>(o, pass, q, rank, sm);
        else slice_strided<double>(o, pass, q, rank, sm);
    }
}

OzOperand oz_operand(const void* src, long long s_row, long long s_k, long long rows, long long K, int S,
                     __nv_bfloat16* out, long long ldk, long long slice_stride, unsigned long long* mx) {
    OzOperand o;
    o.src = src;
    o.s_row = s_row;
    o.s_k = s_k;
    o.rows = static_cast<int>(rows);
    o.K = static_cast<int>(K);
    o.S = S;
    o.out = out;
    o.ldk = ldk;
    o.slice_stride = slice_stride;
    o.mx = mx;
    o.passes = static_cast<int>((K + OZ_KPASS - 1) / OZ_KPASS);
    o.tpr = s_k == 1 ? (K <= 256 ? 32 : 128) : 0;
    o.rpc = s_k == 1 ? OZ_CS * (OZ_ST / o.tpr) : 32;
    o.clusters = o.passes * static_cast<int>((rows + o.rpc - 1) / o.rpc);
    return o;
}

// Both operands, every pass of their K range (at most OZ_PGRP passes), in one launch.
gn_status slice_pair(gn_handle h, const OzOperand& a, int a_f32, const OzOperand& b) {
    OzSliceArgs args;
    args.op[0] = a;
    args.op[1] = b;
    for (const OzOperand& o : args.op)
        if ((o.s_k != 1 && o.s_row != 1) || o.K < 1 || o.passes > OZ_PGRP || o.rows < 1) return GN_ERR_INVALID_ARG;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(OZ_CS * (static_cast<long long>(a.clusters) + b.clusters)));
    cfg.blockDim = dim3(OZ_ST);
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = OZ_CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (a_f32) GN_CUDA_TRY(cudaLaunchKernelEx(&cfg, oz_slice_kernel<true>, args));
    else GN_CUDA_TRY(cudaLaunchKernelEx(&cfg, oz_slice_kernel<false>, args));
    count_launch();
    return GN_OK;
}

// C[i, j] = beta C[i, j] + sum_q alpha 2^{ea_qi + eb_qj} sum_o D_qo[i, j] over
// the K parts q (passes, each with its own row exponents), added in part
// order with one rounding each.  Within a part the exact orders 0..3 are
// summed as integers in units of 2^-35 (one rounding), the rounded orders 4..
// in FP32 below them.  A thread per column and row group (no division per
// element; narrow products fill a block with more rows); each exact order is
// an integer below 2^24 units, so it converts through a 32-bit integer.
__global__ void oz_combine_kernel(const float* __restrict__ D, long long d_stride, long long part_stride,
                                  long long ldd, int norders, int nparts, int M, int N,
                                  const unsigned long long* __restrict__ mxa,
                                  const unsigned long long* __restrict__ mxb, long long mxb_part, double alpha,
                                  double beta, double* __restrict__ C, long long ldc, int cw) {
    // a block is cw columns by blockDim.x / cw rows (cw: a power of two >= min(N, 256), >= 32)
    const int j = blockIdx.x * cw + static_cast<int>(threadIdx.x) % cw;
    const int rb = static_cast<int>(blockDim.x) / cw;
    if (j >= N) return;
    const int nexact = norders < 4 ? norders : 4;
    for (int i = blockIdx.y * rb + static_cast<int>(threadIdx.x) / cw; i < M; i += gridDim.y * rb) {
        double* c = C + static_cast<long long>(i) * ldc + j;
        double out = 0.0;
        for (int q = 0; q < nparts; ++q) {   // K parts (passes) in order, as separate passes would add them
            const float* d = D + q * part_stride + static_cast<long long>(i) * ldd + j;
            long long acc = 0;
            for (int o = 0; o < nexact; ++o)   // D_o is an integer number of units 2^{-7(o+2)}
                acc += static_cast<long long>(__float2int_rn(d[o * d_stride] * __int_as_float((127 + 7 * (o + 2)) << 23)))
                       << (7 * (3 - o));
            float low = 0.0f;
            for (int o = norders - 1; o >= 4; --o) low += d[o * d_stride];
            // times 2^(ea + eb - 35): a power of two built from its bits when normal
            const int ea = row_exponent<double>(mxa[static_cast<long long>(q) * M + i]);
            const int eb = row_exponent<double>(mxb[q * mxb_part + j]);
            const int p = ea + eb - 35;
            const double x = fma(static_cast<double>(low), 34359738368.0, static_cast<double>(acc));
            const double v = (p >= -1022 && p <= 1023)
                                 ? x * (alpha * __longlong_as_double(static_cast<long long>(p + 1023) << 52))
                                 : alpha * ldexp(x, p);
            out = q ? out + v : (beta == 0.0 ? v : fma(beta, *c, v));
        }
        *c = out;
    }
}

struct OzWs {
    __nv_bfloat16 *as, *bs;
    float* d;
    unsigned long long *mxa, *mxb;
    long long ldk, ldd;
};

// K per group of passes, its passes, and the workspace carve for them.
long long oz_kgroup(long long K) { return std::min<long long>(std::max<long long>(K, 1), OZ_PGRP * OZ_KPASS); }
long long oz_parts(long long kg) { return (kg + OZ_KPASS - 1) / OZ_KPASS; }

bool oz_carve(long long M, long long N, long long K, int sa, int sb, void* ws, size_t ws_bytes, OzWs* o) {
    const long long kg = oz_kgroup(K), S = oz_parts(kg), np = oz_npanel(M, N, S);
    o->ldk = r8(kg);
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
    o->d = reinterpret_cast<float*>(take(sizeof(float) * S * OZ_MAX_DIGITS * M * o->ldd));
    o->mxa = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * S * M));
    o->mxb = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * S * N));
    return off <= ws_bytes;
}

}  // namespace

size_t oz_ws_bytes(long long M, long long N, long long K, int a_f32) {
    (void)a_f32;
    const int sa = OZ_MAX_DIGITS, sb = OZ_MAX_DIGITS;
    const long long kg = oz_kgroup(K), S = oz_parts(kg);
    // the FP32 outputs of s parts at the panel for s parts, largest over s <= S:
    // the panel narrows as the parts grow, and the size must not shrink with K
    size_t d = 0;
    for (long long s = 1; s <= S; ++s)
        d = std::max(d, al256(sizeof(float) * s * OZ_MAX_DIGITS * M * r4(oz_npanel(M, std::max<long long>(N, 1), s))));
    return al256(sizeof(__nv_bfloat16) * sa * M * r8(kg)) + al256(sizeof(__nv_bfloat16) * sb * N * r8(kg)) + d +
           al256(8 * S * M) + al256(8 * S * N) + 256;
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
    // groups of at most OZ_PGRP passes: one slicing launch for all of them, the
    // passes as K-aligned parts of one multi-GEMM launch (stored apart), one
    // combination adding them in order
    const long long part_stride = OZ_MAX_DIGITS * d_stride;
    const long long npanel = oz_npanel(M, N, oz_parts(oz_kgroup(K)));   // the carve's panel (largest group)
    for (long long k0 = 0; k0 < K; k0 += OZ_PGRP * OZ_KPASS) {
        const long long kc = std::min<long long>(OZ_PGRP * OZ_KPASS, K - k0);
        const int S = static_cast<int>(oz_parts(kc));
        // A rows (i over M, k along the group) and B "rows" (j over N)
        const long long a_row = ta ? 1 : lda, a_k = ta ? lda : 1;
        const long long a_off = ta ? k0 * lda : k0;
        const long long b_row = tb ? ldb : 1, b_k = tb ? 1 : ldb;
        const long long b_off = tb ? k0 : k0 * ldb;
        const size_t esz = a_f32 ? sizeof(float) : sizeof(double);
        GN_TRY(slice_pair(h,
                          oz_operand(static_cast<const char*>(A) + esz * a_off, a_row, a_k, M, kc, sa, o.as, o.ldk,
                                     as_stride, o.mxa),
                          a_f32, oz_operand(B + b_off, b_row, b_k, N, kc, sb, o.bs, o.ldk, bs_stride, o.mxb)));
        const double beta_grp = k0 == 0 ? beta : 1.0;
        for (long long j0 = 0; j0 < N; j0 += npanel) {
            const long long nb = std::min<long long>(npanel, N - j0);
            // N tile: the widest of 256 / 128 / 64 that still gives the GPU about
            // two work items per SM over the orders and parts (small products are latency-bound)
            int bn = static_cast<int>(std::min<long long>(256, (nb + 31) / 32 * 32));
            while (bn > 64 && ((M + 127) / 128) * ((nb + bn - 1) / bn) * norders * S < 2LL * h->sm_count)
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
                if (S >= 2) {   // pass q of the group: its own row scaling, stored at D + q part_stride
                    g.ksplit = S;
                    g.part_stride = part_stride;
                    g.kpart = OZ_KPASS / TC_BK;
                }
            }
            p.ngemm = norders;
            // orders of 7, 6, ..., 1 slice products: the boustrophedon order on
            // 4 groups of CTAs gives every CTA 7 (order 6; 5 + 0; 4 + 1; 3 + 2)
            p.snake_groups = (norders + 1) / 2;
            GN_TRY(tc_launch(h, &p));
            int cw = 32;   // a power of two, so that it divides the block's 256 threads
            while (cw < nb && cw < 256) cw *= 2;
            const long long rows_per_block = 256 / cw;
            const unsigned gx = static_cast<unsigned>((nb + cw - 1) / cw);
            const unsigned gy = static_cast<unsigned>(std::max<long long>(
                1, std::min<long long>((M + rows_per_block - 1) / rows_per_block,
                                       static_cast<long long>(h->sm_count) * 16 / gx)));
            oz_combine_kernel<<<dim3(gx, gy), 256, 0, h->stream>>>(
                o.d, d_stride, part_stride, o.ldd, norders, S, static_cast<int>(M), static_cast<int>(nb), o.mxa,
                o.mxb + j0, N, alpha, beta_grp, C + j0, ldc, cw);
            count_launch();
            GN_CUDA_TRY(cudaGetLastError());
        }
    }
    return GN_OK;
}

}  // namespace gn

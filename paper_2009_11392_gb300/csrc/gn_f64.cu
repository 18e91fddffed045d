// FP64 kernels of the stable core of generalized Nystrom (Section 5.1) and of
// the plain FP64 GN path:
//   * a tiled FP64 GEMM (DFMA) with optional split-K, used for the FP64
//     sketches, the core product C = (Y^T A) X, the WY updates of the QR and
//     the factor products;
//   * blocked Householder QR with compact-WY trailing updates (Algorithm 2
//     step 2, "Y^T A X = QR"), diag(R) made non-negative;
//   * blocked right triangular solves F R = B and F R^T = B (eq. 5.1's AX/R
//     and Section 5.1.1's Q_2 R_2^{-T});
//   * the truncation rank and the power-method estimate of ||R^{-1}||_2
//     (Sections 5.1.1 and 5.1.2);
//   * operand quantisation (FP64/FP32 -> BF16, split BF16) and the fused
//     ||A - F G||_F^2 accumulation.
// On GB300 FP64 runs on the CUDA cores at a small fraction of the FP32 rate,
// so these kernels aim at keeping the DFMA pipes busy (enough CTAs, split-K for
// skinny products) rather than at data movement.
#include "gn_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace gn {
namespace {

constexpr int GT = 64;    // GEMM tile (M and N)
constexpr int GK = 16;    // GEMM K step
constexpr int GTHREADS = 256;

template <typename TA>
__device__ __forceinline__ double ld_a(const TA* p) { return static_cast<double>(*p); }
template <>
__device__ __forceinline__ double ld_a<__nv_bfloat16>(const __nv_bfloat16* p) {
    return static_cast<double>(__bfloat162float(*p));
}

// Epilogue modes of the tiled FP64 product.
enum { EPI_STORE = 0, EPI_PARTIAL = 1, EPI_ERR = 2 };

struct ErrArgs {
    const void* A;     // reference matrix of ||A - F G||
    const void* A_lo;  // low part for split bf16
    int a_dtype;
    long long lda;
    double* partial;   // one double per CTA
};

__device__ __forceinline__ double load_ref(const ErrArgs& e, long long i, long long j) {
    const long long off = i * e.lda + j;
    switch (e.a_dtype) {
        case GN_F64: return static_cast<const double*>(e.A)[off];
        case GN_F32: return static_cast<double>(static_cast<const float*>(e.A)[off]);
        case GN_BF16:
            return static_cast<double>(__bfloat162float(static_cast<const __nv_bfloat16*>(e.A)[off]));
        default:
            return static_cast<double>(__bfloat162float(static_cast<const __nv_bfloat16*>(e.A)[off])) +
                   static_cast<double>(__bfloat162float(static_cast<const __nv_bfloat16*>(e.A_lo)[off]));
    }
}

// C tile = alpha * op(A) op(B) (+ beta C); BM x BN tile, 256 threads as a
// 16 x 16 grid, each thread a (BM/16) x (BN/16) block of outputs at rows
// ty + 16 i and columns tx + 16 j.  BM = 16 serves the skinny (panel-width)
// products of the WY updates without padding waste.
template <int BM, int BN, typename TA, typename TB_, int EPI>
__global__ void __launch_bounds__(GTHREADS) dgemm_kernel(
    int M, int N, int K, double alpha, const TA* __restrict__ A, long long lda, int ta,
    const TB_* __restrict__ B, long long ldb, int tb, double beta, double* C, long long ldc,
    double* part, int kchunk, ErrArgs err) {
    constexpr int RI = BM / 16, RJ = BN / 16;
    __shared__ double As[GK][BM + 1];
    __shared__ double Bs[GK][BN + 1];
    __shared__ double red[GTHREADS / 32];
    const int m0 = blockIdx.y * BM;
    const int n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int tx = threadIdx.x & 15;
    const int ty = threadIdx.x >> 4;
    double acc[RI][RJ];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < RJ; ++j) acc[i][j] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += GK) {
#pragma unroll
        for (int e = threadIdx.x; e < BM * GK; e += GTHREADS) {
            int mm, kk;
            if (ta) { mm = e % BM; kk = e / BM; } else { kk = e & 15; mm = e >> 4; }
            const int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < kend)
                v = ta ? ld_a(A + static_cast<long long>(gk) * lda + gm)
                       : ld_a(A + static_cast<long long>(gm) * lda + gk);
            As[kk][mm] = v;
        }
#pragma unroll
        for (int e = threadIdx.x; e < BN * GK; e += GTHREADS) {
            int nn, kk;
            if (tb) { kk = e & 15; nn = e >> 4; } else { nn = e % BN; kk = e / BN; }
            const int gn_ = n0 + nn, gk = k0 + kk;
            double v = 0.0;
            if (gn_ < N && gk < kend)
                v = tb ? ld_a(B + static_cast<long long>(gn_) * ldb + gk)
                       : ld_a(B + static_cast<long long>(gk) * ldb + gn_);
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[RI], b[RJ];
#pragma unroll
            for (int i = 0; i < RI; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < RJ; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < RI; ++i)
#pragma unroll
                for (int j = 0; j < RJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    if (EPI == EPI_ERR) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < RI; ++i)
#pragma unroll
            for (int j = 0; j < RJ; ++j) {
                const int gm = m0 + ty + 16 * i, gn_ = n0 + tx + 16 * j;
                if (gm < M && gn_ < N) {
                    const double d = load_ref(err, gm, gn_) - acc[i][j];
                    s = fma(d, d, s);
                }
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < GTHREADS / 32; ++w) t += red[w];
            err.partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < RJ; ++j) {
            const int gm = m0 + ty + 16 * i, gn_ = n0 + tx + 16 * j;
            if (gm < M && gn_ < N) {
                if (EPI == EPI_PARTIAL) {
                    part[(static_cast<long long>(blockIdx.z) * M + gm) * N + gn_] = alpha * acc[i][j];
                } else {
                    double* c = C + static_cast<long long>(gm) * ldc + gn_;
                    *c = beta == 0.0 ? alpha * acc[i][j] : fma(beta, *c, alpha * acc[i][j]);
                }
            }
        }
}

__global__ void splitk_reduce_kernel(int M, int N, int splits, const double* __restrict__ part,
                                     double beta, double* C, long long ldc) {
    const long long total = static_cast<long long>(M) * N;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < splits; ++z) s += part[z * total + e];
        const long long i = e / N, j = e % N;
        double* c = C + i * ldc + j;
        *c = beta == 0.0 ? s : fma(beta, *c, s);
    }
}

__global__ void reduce_sum_kernel(const double* __restrict__ part, long long n, double* out) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) t += red[w];
        *out = t;
    }
}

// Tile shape: 16 x 128 or 32 x 128 for panel-width products (M <= 32), else 64 x 64.
inline int tile_m(long long M) { return M <= 16 ? 16 : (M <= 32 ? 32 : GT); }

int choose_splits(long long M, long long N, long long K, int sm_count) {
    const long long bm = tile_m(M), bn = bm < GT ? 128 : GT;
    const long long tiles = ((M + bm - 1) / bm) * ((N + bn - 1) / bn);
    if (tiles >= sm_count || K < 256) return 1;
    long long s = (2LL * sm_count + tiles - 1) / tiles;
    s = std::min(s, K / 64);
    s = std::min<long long>(s, 64);
    return static_cast<int>(std::max<long long>(s, 1));
}

template <int BM, int BN, typename TA, typename TB_>
gn_status dgemm_launch(gn_handle h, long long M, long long N, long long K, double alpha, const TA* A,
                       long long lda, int ta, const TB_* B, long long ldb, int tb, double beta, double* C,
                       long long ldc, double* ws, size_t ws_bytes) {
    ErrArgs e{};
    if (K <= 0) {
        dim3 grid(static_cast<unsigned>((N + BN - 1) / BN), static_cast<unsigned>((M + BM - 1) / BM), 1);
        dgemm_kernel<BM, BN, TA, TB_, EPI_STORE><<<grid, GTHREADS, 0, h->stream>>>(
            (int)M, (int)N, 0, 0.0, A, lda, ta, B, ldb, tb, beta, C, ldc, nullptr, 1, e); count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        return GN_OK;
    }
    int splits = choose_splits(M, N, K, h->sm_count);
    while (splits > 1 && static_cast<size_t>(splits) * M * N * sizeof(double) > ws_bytes) --splits;
    if (ws == nullptr) splits = 1;
    int kchunk = static_cast<int>(((K + splits - 1) / splits + GK - 1) / GK * GK);
    splits = static_cast<int>((K + kchunk - 1) / kchunk);
    dim3 grid(static_cast<unsigned>((N + BN - 1) / BN), static_cast<unsigned>((M + BM - 1) / BM),
              static_cast<unsigned>(splits));
    if (splits == 1) {
        dgemm_kernel<BM, BN, TA, TB_, EPI_STORE><<<grid, GTHREADS, 0, h->stream>>>(
            (int)M, (int)N, (int)K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, nullptr, kchunk, e); count_launch();
    } else {
        dgemm_kernel<BM, BN, TA, TB_, EPI_PARTIAL><<<grid, GTHREADS, 0, h->stream>>>(
            (int)M, (int)N, (int)K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, ws, kchunk, e); count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        const long long total = M * N;
        const int blocks = static_cast<int>(std::min<long long>((total + 255) / 256, 4LL * h->sm_count));
        splitk_reduce_kernel<<<blocks, 256, 0, h->stream>>>((int)M, (int)N, splits, ws, beta, C, ldc); count_launch();
    }
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

template <typename TA, typename TB_>
gn_status dgemm_impl(gn_handle h, long long M, long long N, long long K, double alpha, const TA* A,
                     long long lda, int ta, const TB_* B, long long ldb, int tb, double beta,
                     double* C, long long ldc, double* ws, size_t ws_bytes) {
    if (M <= 0 || N <= 0) return GN_OK;
    if (K <= 0 && beta == 0.0) return set_zero_f64(h, C, M, N, ldc);
    if (tile_m(M) == 16)
        return dgemm_launch<16, 128, TA, TB_>(h, M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, ws, ws_bytes);
    if (tile_m(M) == 32)
        return dgemm_launch<32, 128, TA, TB_>(h, M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, ws, ws_bytes);
    return dgemm_launch<GT, GT, TA, TB_>(h, M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, ws, ws_bytes);
}

// --------------------------------------------------------------------------
// Householder QR
// --------------------------------------------------------------------------
constexpr int QR_THREADS = 512;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr int QR_JB = 16;                 // panel width of the single-CTA panel kernel
constexpr int QR_NB = 32;                 // widest panel (cluster kernel); sizes the T / Z storage
constexpr size_t QR_SMEM_PANEL_MAX = 208 * 1024;

// Sum of `n` per-thread values across the CTA; results in out[0..n).
template <int NV>
__device__ void block_sum_vec(double (&v)[NV], int n, double* red /* [QR_WARPS][NV] */, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        if (c >= n) break;
        double s = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp * NV + c] = s;
    }
    __syncthreads();
    if (threadIdx.x < n) {
        double s = 0.0;
        for (int w = 0; w < QR_WARPS; ++w) s += red[w * NV + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Factor the panel W[j0:M, j0:j0+jb] in place: R above the diagonal, the
// Householder vectors (unit leading entry) below it.  Writes the explicit
// vectors into V (column j0+c holds v in rows j0+c..M-1, zeros above), tau,
// and the upper-triangular T of the compact WY form H_0...H_{jb-1} = I - V T V^T.
__global__ void __launch_bounds__(QR_THREADS) qr_panel_kernel(double* W, long long ld, int M, int j0,
                                                              int jb, double* V, long long ldv,
                                                              double* tau, double* T, int use_smem) {
    extern __shared__ double sh[];
    __shared__ double red[QR_WARPS * QR_JB];
    __shared__ double wsum[QR_JB];
    __shared__ double s_tau, s_beta, s_scale;
    __shared__ double tloc[QR_JB * QR_JB];
    __shared__ double tauloc[QR_JB];
    const int Mp = M - j0;
    const int tid = threadIdx.x;
    double* P;
    long long ldp;
    if (use_smem) {
        P = sh;
        ldp = jb + 1;   // odd stride: column walks across rows avoid bank conflicts
        for (long long e = tid; e < static_cast<long long>(Mp) * jb; e += QR_THREADS) {
            const long long i = e / jb;
            const int c = static_cast<int>(e % jb);
            P[i * ldp + c] = W[(j0 + i) * ld + j0 + c];
        }
        __syncthreads();
    } else {
        P = W + static_cast<long long>(j0) * ld + j0;
        ldp = ld;
    }

    for (int c = 0; c < jb; ++c) {
        double acc1[1] = {0.0};
        for (int i = c + 1 + tid; i < Mp; i += QR_THREADS) {
            const double x = P[i * ldp + c];
            acc1[0] = fma(x, x, acc1[0]);
        }
        block_sum_vec<1>(acc1, 1, red, wsum);
        if (tid == 0) {
            const double alpha = P[static_cast<long long>(c) * ldp + c];
            const double tail = wsum[0];
            if (tail == 0.0) {
                s_tau = 0.0;
                s_beta = alpha;
                s_scale = 0.0;
            } else {
                const double nx = sqrt(fma(alpha, alpha, tail));
                const double beta = alpha >= 0.0 ? -nx : nx;
                s_tau = (beta - alpha) / beta;
                s_beta = beta;
                s_scale = 1.0 / (alpha - beta);
            }
        }
        __syncthreads();
        const double t = s_tau;
        if (t != 0.0) {
            const double sc = s_scale;
            for (int i = c + 1 + tid; i < Mp; i += QR_THREADS) P[i * ldp + c] *= sc;
            __syncthreads();
            const int nrem = jb - c - 1;
            if (nrem > 0) {
                double w[QR_JB];
#pragma unroll
                for (int q = 0; q < QR_JB; ++q) w[q] = 0.0;
                for (int i = c + tid; i < Mp; i += QR_THREADS) {
                    const double vi = (i == c) ? 1.0 : P[i * ldp + c];
                    const double* row = P + i * ldp + c + 1;
#pragma unroll
                    for (int q = 0; q < QR_JB; ++q)
                        if (q < nrem) w[q] = fma(vi, row[q], w[q]);
                }
                block_sum_vec<QR_JB>(w, nrem, red, wsum);
                for (int i = c + tid; i < Mp; i += QR_THREADS) {
                    const double vi = (i == c) ? 1.0 : P[i * ldp + c];
                    double* row = P + i * ldp + c + 1;
#pragma unroll
                    for (int q = 0; q < QR_JB; ++q)
                        if (q < nrem) row[q] = fma(-t * vi, wsum[q], row[q]);
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            P[static_cast<long long>(c) * ldp + c] = s_beta;
            tauloc[c] = t;
            tau[j0 + c] = t;
        }
        __syncthreads();
    }

    // Explicit V and the write-back of the panel.
    for (long long e = tid; e < static_cast<long long>(Mp) * jb; e += QR_THREADS) {
        const long long i = e / jb;
        const int c = static_cast<int>(e % jb);
        const double pv = P[i * ldp + c];
        double v;
        if (i < c) v = 0.0;
        else if (i == c) v = 1.0;
        else v = tauloc[c] == 0.0 ? 0.0 : pv;
        V[(j0 + i) * ldv + j0 + c] = v;
        if (use_smem) W[(j0 + i) * ld + j0 + c] = pv;
    }
    __syncthreads();

    // Gram products g_c[q] = v_q^T v_c (q < c) and T (forward, columnwise).
    for (int c = 1; c < jb; ++c) {
        double g[QR_JB];
#pragma unroll
        for (int q = 0; q < QR_JB; ++q) g[q] = 0.0;
        for (int i = c + tid; i < Mp; i += QR_THREADS) {   // v_c is zero above row c
            const double vc = (i == c) ? 1.0 : (tauloc[c] == 0.0 ? 0.0 : P[i * ldp + c]);
#pragma unroll
            for (int q = 0; q < QR_JB; ++q) {
                if (q < c) {
                    const double vq = (i == q) ? 1.0 : (tauloc[q] == 0.0 ? 0.0 : P[i * ldp + q]);
                    g[q] = fma(vq, vc, g[q]);
                }
            }
        }
        block_sum_vec<QR_JB>(g, c, red, tloc + c * QR_JB);   // row c of tloc holds g for column c
    }
    if (tid == 0) {
        double Tm[QR_JB][QR_JB];
        for (int a = 0; a < QR_JB; ++a)
            for (int b = 0; b < QR_JB; ++b) Tm[a][b] = 0.0;
        for (int c = 0; c < jb; ++c) {
            const double tc = tauloc[c];
            Tm[c][c] = tc;
            for (int a = 0; a < c; ++a) {
                double s = 0.0;
                for (int b = a; b < c; ++b) s = fma(Tm[a][b], tloc[c * QR_JB + b], s);
                Tm[a][c] = -tc * s;
            }
        }
        for (int a = 0; a < jb; ++a)
            for (int b = 0; b < jb; ++b) T[a * jb + b] = Tm[a][b];
    }
}

// ---------------------------------------------------------------------------
// Cluster panel factorization.  The panel rows are split across the CTAs of a
// thread-block cluster (each CTA keeps its rows in shared memory); the two
// reductions per column (the norm of the column below the diagonal and the
// vector w = v^T P of the rank-1 update) combine per-CTA partials read through
// distributed shared memory, summed in rank order so every CTA derives the same
// reflector.  Partials are double-buffered by column parity, so two cluster
// barriers per column suffice.  Same outputs as qr_panel_kernel.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;
constexpr int CP_THREADS = 256;
constexpr int CP_WARPS = CP_THREADS / 32;

__device__ __forceinline__ double warp_sum(double s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

template <int JB>
__host__ __device__ constexpr size_t cluster_panel_smem(int rows_per) {
    // P + exchange slots [2][2+2JB] + tv[max(rows_per, 256)] + dsum/prow/g [3][JB] + gram, T [2][JB*JB]
    // + per-warp Gram partials [7][JB(JB-1)/2]
    return sizeof(double) * (static_cast<size_t>(rows_per) * (JB + 1) + 2 * (2 + 2 * JB) +
                             (rows_per > 256 ? rows_per : 256) + 3 * JB + 2 * JB * JB + 7 * (JB * (JB - 1) / 2));
}

// One exchange per column: with x = P[c:, c], alpha = x_0, beta = -sign(alpha)||x||
// and v = x / (alpha - beta) (v_0 = 1), the update vector is
//     w_q = v^T P_q = (x^T P_q - beta P_cq) / (alpha - beta),
// so ||x[1:]||^2, the dot products x^T P_q and the owner's row c are all the
// per-CTA partials a column needs, and they are exchanged in one cluster round.
// With d = 1 / (beta (alpha - beta)) the update P_q -= tau v w_q is
//     P_iq += xt_i g_q,   g_q = d (x^T P_q - beta P_cq),
// where xt = x below row c and xt_c = alpha - beta: it uses the column as it
// stands, so the reflectors are normalised (v = xt / (alpha - beta)) once,
// after the last column.  The Gram V^T V that T needs is formed column by
// column by warps 1-7 while warp 0 computes the next reflector's scalars.
template <int JB>
__global__ void __launch_bounds__(CP_THREADS) qr_panel_cluster_kernel(double* W, long long ld, int M, int j0,
                                                                     int jb, double* V, long long ldv,
                                                                     double* tau, double* T, int rows_per) {
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = static_cast<int>(cluster.num_blocks());
    const int rank = static_cast<int>(cluster.block_rank());
    extern __shared__ double sm[];
    constexpr int LDP = JB + 1;
    constexpr int SLOT = 2 + 2 * JB;   // [tail, alpha, dots[JB], row_c[JB]]
    double* P = sm;
    double* xch = P + static_cast<size_t>(rows_per) * LDP;   // [2][SLOT]
    double* tv = xch + 2 * SLOT;                             // [max(rows_per, 256)] tau * v_i
    double* dsum = tv + (rows_per > 256 ? rows_per : 256);   // [JB] x^T P_q summed over ranks
    double* prow = dsum + JB;                                // [JB] row c of the panel
    double* wv = prow + JB;                                  // [JB] g_q
    double* gram = wv + JB;                                  // [JB][JB] partial V^T V
    double* Ts = gram + JB * JB;                             // [JB][JB]
    constexpr int NPAIR = JB * (JB - 1) / 2;
    double* gpart = Ts + JB * JB;                            // [7][NPAIR] Gram partials of warps 1-7
    __shared__ double taus[JB], sc_col[JB], amb_col[JB];
    __shared__ double s_tau, s_beta, s_amb;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Mp = M - j0;
    const int r0 = rank * rows_per;
    const int nr = max(0, min(rows_per, Mp - r0));

    for (int e = tid; e < nr * jb; e += CP_THREADS) {
        const int i = e / jb, c = e - i * jb;
        P[i * LDP + c] = W[static_cast<long long>(j0 + r0 + i) * ld + j0 + c];
    }
    __syncthreads();

    for (int e = tid; e < JB; e += CP_THREADS) {
        taus[e] = 0.0;
        sc_col[e] = 0.0;
        amb_col[e] = 0.0;
    }
    // Warps 1-7: partial Gram of reflector a with reflectors q < a over this CTA's
    // rows below row a, from the unnormalised columns (xt_a = alpha - beta at row a).
    auto gram_partial = [&](int a) {
        const int np = a > 16 ? 32 : a > 8 ? 16 : a > 4 ? 8 : a > 2 ? 4 : a > 1 ? 2 : 1;
        const int q = lane & (np - 1), sub = lane / np, nsub = 32 / np;
        const int cla = a - r0;
        // two partial sums: the loads of one overlap the other's FMA (~64 cycles each on GB300)
        double acc = 0.0, acc1 = 0.0;
        if (q < a) {
            const int step = (CP_WARPS - 1) * nsub;
            int li = max(0, cla) + (warp - 1) * nsub + sub;
            for (; li + step < nr; li += 2 * step) {
                const double xa = li == cla ? amb_col[a] : P[li * LDP + a];
                const double xb = li + step == cla ? amb_col[a] : P[(li + step) * LDP + a];
                acc = fma(xa, P[li * LDP + q], acc);
                acc1 = fma(xb, P[(li + step) * LDP + q], acc1);
            }
            if (li < nr) {
                const double xa = li == cla ? amb_col[a] : P[li * LDP + a];
                acc = fma(xa, P[li * LDP + q], acc);
            }
        }
        acc += acc1;
        for (int o = np; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (sub == 0 && q < a) gpart[(warp - 1) * NPAIR + a * (a - 1) / 2 + q] = acc;
    };
    // Per-column thread tiles cover only the live columns: with na live columns
    // (padded to np, a power of two), lane = sub * np + column offset and the
    // 8 * 32 / np row chunks split the rows.  On GB300 each FP64 warp
    // instruction holds its sub-partition's FP64 unit for ~64 cycles whatever
    // its mask, so idle lanes are what this avoids.
    for (int c = 0; c < jb; ++c) {
        double* slot = xch + (c & 1) * SLOT;
        const int cl = c - r0;                       // local index of row c (owner iff 0 <= cl < nr)
        const bool owner = cl >= 0 && cl < nr;
        const int lo = max(0, cl);                   // first local row with panel row >= c
        // ---- per-CTA partials: tail = sum_{rows > c} x_i^2 (column c),
        //      dots_j = sum_{rows >= c} x_i P_ij (columns j > c)
        {
            const int na = jb - c;
            const int np = na > 16 ? 32 : na > 8 ? 16 : na > 4 ? 8 : na > 2 ? 4 : na > 1 ? 2 : 1;
            const int off = lane & (np - 1), sub = lane / np;
            const int nchunk = CP_WARPS * (32 / np);
            const int chunk = warp * (32 / np) + sub;
            const int j = c + off;
            double acc = 0.0, acc1 = 0.0;   // two partial sums: half the FMA chain
            if (off < na) {
                const int jj = off == 0 ? c : j;
                int li = (off == 0 ? max(0, cl + 1) : lo) + chunk;
                for (; li + nchunk < nr; li += 2 * nchunk) {
                    acc = fma(P[li * LDP + c], P[li * LDP + jj], acc);
                    acc1 = fma(P[(li + nchunk) * LDP + c], P[(li + nchunk) * LDP + jj], acc1);
                }
                if (li < nr) acc = fma(P[li * LDP + c], P[li * LDP + jj], acc);
            }
            acc += acc1;
            for (int o = np; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (sub == 0) tv[warp * 32 + off] = acc;   // tv doubles as the 8 x 32 partial table here
        }
        __syncthreads();
        if (warp == 0) {
            const int j = c + lane;
            if (j < jb) {
                const double t8 = ((tv[lane] + tv[32 + lane]) + (tv[64 + lane] + tv[96 + lane])) +
                                  ((tv[128 + lane] + tv[160 + lane]) + (tv[192 + lane] + tv[224 + lane]));
                if (lane == 0) {
                    slot[0] = t8;
                    slot[1] = owner ? P[cl * LDP + c] : 0.0;
                } else {
                    slot[2 + j] = t8;
                    slot[2 + JB + j] = owner ? P[cl * LDP + j] : 0.0;
                }
            }
        }
        cluster.sync();
        // ---- combine over ranks (the same order in every CTA): warps 0-3 each sum
        //      four ranks' partials for every column, warp 0 adds the four sums
        const int cj = lane;
        if (warp < 4 && cj >= c && cj < jb) {
            const int o0 = cj == c ? 0 : 2 + cj, o1 = cj == c ? 1 : 2 + JB + cj;
            double p0[4], p1[4];   // all four loads first, then a tree (short FP64 chain)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int k = 4 * warp + kk;
                p0[kk] = 0.0;
                p1[kk] = 0.0;
                if (k < cs) {
                    const double* rs = cluster.map_shared_rank(slot, k);
                    p0[kk] = rs[o0];
                    p1[kk] = rs[o1];
                }
            }
            tv[warp * 64 + cj] = (p0[0] + p0[1]) + (p0[2] + p0[3]);   // tv is free here: 4 x 2 x 32 partial sums
            tv[warp * 64 + 32 + cj] = (p1[0] + p1[1]) + (p1[2] + p1[3]);
        }
        __syncthreads();
        if (warp == 0) {
            double a0 = 0.0, a1 = 0.0, beta_l = 0.0, d_l = 0.0;
            if (cj >= c && cj < jb) {
                a0 = (tv[cj] + tv[64 + cj]) + (tv[128 + cj] + tv[192 + cj]);
                a1 = (tv[32 + cj] + tv[96 + cj]) + (tv[160 + cj] + tv[224 + cj]);
            }
            if (cj == c) {
                const double tail = a0, alpha = a1;
                if (tail == 0.0) {
                    s_tau = 0.0;
                    s_beta = alpha;
                    s_amb = 0.0;
                } else {
                    const double nx = sqrt(fma(alpha, alpha, tail));
                    const double beta = alpha >= 0.0 ? -nx : nx;
                    // one division: d = 1 / (beta (alpha - beta)) gives both 1/beta and 1/(alpha - beta)
                    const double amb = alpha - beta;
                    const double d = 1.0 / (beta * amb);
                    s_tau = (beta - alpha) * (amb * d);
                    s_beta = beta;
                    s_amb = amb;
                    sc_col[c] = beta * d;   // 1 / (alpha - beta)
                    amb_col[c] = amb;
                    beta_l = beta;
                    d_l = d;
                }
            }
            const double beta = __shfl_sync(0xffffffffu, beta_l, c);
            const double d = __shfl_sync(0xffffffffu, d_l, c);
            if (cj > c && cj < jb) wv[cj] = d * fma(-beta, a1, a0);
        } else if (c >= 2) {
            // Gram of reflector a = c - 1 with reflectors q < a over this CTA's rows
            // (unnormalised columns; scaled by both normalisations at the end).
            // Lanes cover only the live pairs: lane = sub * np + q.
            gram_partial(c - 1);
        }
        __syncthreads();
        const double t = s_tau;
        if (tid == 0) {
            if (owner) P[cl * LDP + c] = s_beta;
            taus[c] = t;
            if (rank == 0) tau[j0 + c] = t;
        }
        if (t != 0.0) {
            const double amb = s_amb;
            const int na = jb - c - 1;   // columns c+1 .. jb-1
            if (na > 0) {
                const int np = na > 16 ? 32 : na > 8 ? 16 : na > 4 ? 8 : na > 2 ? 4 : na > 1 ? 2 : 1;
                const int off = lane & (np - 1);
                const int nchunk = CP_WARPS * (32 / np);
                const int chunk = warp * (32 / np) + lane / np;
                if (off < na) {
                    const int j = c + 1 + off;
                    const double gj = wv[j];
                    for (int li = lo + chunk; li < nr; li += nchunk) {
                        const double x = li == cl ? amb : P[li * LDP + c];
                        P[li * LDP + j] = fma(x, gj, P[li * LDP + j]);
                    }
                }
            }
        }
        __syncthreads();
    }

    // Gram of the last reflector (raw columns), then every partial scaled by the
    // two normalisations: g(a, q) = sc_a sc_q xt_a^T xt_q
    if (jb >= 2 && warp >= 1) gram_partial(jb - 1);
    __syncthreads();
    for (int e = tid; e < NPAIR; e += CP_THREADS) {
        int q = 1, q2 = e;
        while (q2 >= q) {
            q2 -= q;
            ++q;
        }
        double g = 0.0;
        if (q < jb) {
#pragma unroll
            for (int w = 0; w < CP_WARPS - 1; ++w) g += gpart[w * NPAIR + e];
            g *= sc_col[q] * sc_col[q2];
        }
        gram[e] = g;
    }
    // normalise the reflectors below the diagonal: v = xt / (alpha - beta)
    for (int e = tid; e < nr * jb; e += CP_THREADS) {
        const int li = e / jb, c = e - li * jb;
        if (r0 + li > c) P[li * LDP + c] *= sc_col[c];
    }
    __syncthreads();

    // write back the panel and the explicit reflectors
    for (int e = tid; e < nr * jb; e += CP_THREADS) {
        const int li = e / jb, c = e - li * jb;
        const int gi = r0 + li;
        const double pv = P[li * LDP + c];
        const bool live = taus[c] != 0.0;
        const double v = gi < c ? 0.0 : (gi == c ? 1.0 : (live ? pv : 0.0));
        V[static_cast<long long>(j0 + gi) * ldv + j0 + c] = v;
        W[static_cast<long long>(j0 + gi) * ld + j0 + c] = pv;
    }
    cluster.sync();
    if (rank == 0) {
        // Ts: the Gram in the strict lower triangle (zero for dropped reflectors and
        // padding), tau on the diagonal; T is built in the upper triangle.
        for (int e = tid; e < JB * JB; e += CP_THREADS) {
            const int q = e / JB, q2 = e - q * JB;
            double g = 0.0;
            if (q2 < q) {
                const int pe = q * (q - 1) / 2 + q2;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < cs) g += cluster.map_shared_rank(gram, k)[pe];
                if (taus[q] == 0.0 || taus[q2] == 0.0) g = 0.0;
            } else if (q2 == q) {
                g = taus[q];
            }
            Ts[e] = g;
        }
        __syncthreads();
        // T by recursive doubling: for adjacent diagonal blocks T1 (rows o..o+s) and
        // T2 (o+s..o+2s), the off-diagonal block is -T1 (V1^T V2) T2, where
        // (V1^T V2)[a][b] = g(o+s+b, o+a).  Mt holds (V1^T V2) T2 for every pair.
        double* Mt = tv;
        for (int sz = 1; sz < JB; sz <<= 1) {
            const int items = (JB / (2 * sz)) * sz * sz;
            for (int e = tid; e < items; e += CP_THREADS) {
                const int pr = e / (sz * sz), rem = e - pr * sz * sz, a = rem / sz, b = rem - a * sz;
                const int o = pr * 2 * sz;
                double m = 0.0;
                for (int k = 0; k <= b; ++k) m = fma(Ts[(o + sz + k) * JB + o + a], Ts[(o + sz + k) * JB + o + sz + b], m);
                Mt[e] = m;
            }
            __syncthreads();
            for (int e = tid; e < items; e += CP_THREADS) {
                const int pr = e / (sz * sz), rem = e - pr * sz * sz, a = rem / sz, b = rem - a * sz;
                const int o = pr * 2 * sz;
                double v = 0.0;
                for (int k = a; k < sz; ++k) v = fma(Ts[(o + a) * JB + o + k], Mt[pr * sz * sz + k * sz + b], v);
                Ts[(o + a) * JB + o + sz + b] = -v;
            }
            __syncthreads();
        }
        for (int e = tid; e < jb * jb; e += CP_THREADS) {
            const int a = e / jb, b = e - a * jb;
            T[e] = b >= a ? Ts[a * JB + b] : 0.0;
        }
    }
    cluster.sync();
}

// ---------------------------------------------------------------------------
// Compact-WY application W <- W - V op(T) (V^T W) for one panel, in one launch:
// clusters of CS CTAs, one cluster per 64-column block of W, each CTA owning a
// slice of rows (its rows of V and of the W block stay in shared memory for
// both products).  Z = V^T W_blk is reduced over the cluster through DSMEM
// (reduce-scatter by rows, all-gather), each CTA forms its share of
// op(T) Z, and the shares are gathered again.  op(T) = T^T for the trailing
// update of the factorization, T for the formation of Q.
// ---------------------------------------------------------------------------
constexpr int WY_THREADS = 256;
constexpr int WY_JB = 32;
constexpr int WY_MAX_ROWS = 188;   // rows per CTA that fit in shared memory (BN = 64)

__host__ __device__ inline size_t wy_smem(int rp, int bn) {
    return sizeof(double) * (static_cast<size_t>(rp) * (WY_JB + 1 + bn + 1) + 3 * WY_JB * bn + WY_JB * WY_JB);
}

// BN: columns of W per block (8, 16, 32 or 64).  The grid holds one wave of
// clusters; cluster c takes column blocks c, c + ncl, ... (its rows of V and
// op(T) are loaded once).  The kernel is bound by each SM's FP64 rate.
template <int BN>
__global__ void __launch_bounds__(WY_THREADS) qr_wy_apply_kernel(double* W, long long ldw, int Mp, int Nw,
                                                                const double* V, long long ldv, int jb,
                                                                const double* T, int transT, int rp) {
    constexpr int G = WY_THREADS / BN;    // thread groups per column
    constexpr int AU = WY_JB / G;         // rows of Z per thread
    static_assert(AU >= 1 && AU * G == WY_JB, "BN must be 8, 16, 32 or 64");
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = static_cast<int>(cluster.num_blocks());
    const int rank = static_cast<int>(cluster.block_rank());
    const int cid = blockIdx.x / cs, ncl = gridDim.x / cs;
    const int nblk = (Nw + BN - 1) / BN;
    const int r0 = rank * rp;
    const int nr = max(0, min(rp, Mp - r0));
    extern __shared__ double sm[];
    double* Vs = sm;                                   // [rp][JB+1]
    double* Ws = Vs + static_cast<size_t>(rp) * (WY_JB + 1);   // [rp][BN+1]
    double* Zp = Ws + static_cast<size_t>(rp) * (BN + 1);      // [JB][BN] partial V^T W (read remotely)
    double* Z = Zp + WY_JB * BN;                       // [JB][BN] reduced Z, then op(T) Z
    double* Zt = Z + WY_JB * BN;                       // [JB][BN] own rows of op(T) Z (read remotely)
    double* Ts = Zt + WY_JB * BN;                      // [JB][JB] op(T)
    const int tid = threadIdx.x;

    for (int e = tid; e < nr * WY_JB; e += WY_THREADS) {
        const int i = e >> 5, a = e & 31;
        Vs[i * (WY_JB + 1) + a] = a < jb ? V[static_cast<long long>(r0 + i) * ldv + a] : 0.0;
    }
    for (int e = tid; e < WY_JB * WY_JB; e += WY_THREADS) {
        const int a = e >> 5, c = e & 31;
        double v = 0.0;
        if (a < jb && c < jb) v = transT ? T[c * jb + a] : T[a * jb + c];
        Ts[e] = v;
    }
    const int b = tid % BN, ag = tid / BN;
    const int rows_per_rank = (WY_JB + cs - 1) / cs;
    const int a0 = rank * rows_per_rank, a1 = min(WY_JB, a0 + rows_per_rank);
    for (int blk = cid; blk < nblk; blk += ncl) {
        const int c0 = blk * BN;
        const int nbw = min(BN, Nw - c0);
        for (int e = tid; e < nr * BN; e += WY_THREADS) {
            const int i = e / BN, bb = e % BN;
            Ws[i * (BN + 1) + bb] = bb < nbw ? W[static_cast<long long>(r0 + i) * ldw + c0 + bb] : 0.0;
        }
        __syncthreads();
        // ---- Zp = V_rows^T W_rows,blk: thread -> column b, AU consecutive a
        {
            double acc[AU];
#pragma unroll
            for (int u = 0; u < AU; ++u) acc[u] = 0.0;
            for (int i = 0; i < nr; ++i) {
                const double w = Ws[i * (BN + 1) + b];
#pragma unroll
                for (int u = 0; u < AU; ++u) acc[u] = fma(Vs[i * (WY_JB + 1) + ag * AU + u], w, acc[u]);
            }
#pragma unroll
            for (int u = 0; u < AU; ++u) Zp[(ag * AU + u) * BN + b] = acc[u];
        }
        cluster.sync();
        // ---- reduce-scatter: rank k sums rows a in its share of Z over all ranks (rank order)
        for (int e = tid; e < (a1 - a0) * BN; e += WY_THREADS) {
            const int a = a0 + e / BN, bb = e % BN;
            double z = 0.0;
            for (int k = 0; k < cs; ++k) z += cluster.map_shared_rank(Zp, k)[a * BN + bb];
            Z[a * BN + bb] = z;
        }
        cluster.sync();
        // ---- all-gather Z
        for (int e = tid; e < WY_JB * BN; e += WY_THREADS) {
            const int a = e / BN;
            const int owner = a / rows_per_rank;
            if (owner != rank) Z[e] = cluster.map_shared_rank(Z, owner)[e];
        }
        __syncthreads();
        // ---- own rows of op(T) Z
        for (int e = tid; e < (a1 - a0) * BN; e += WY_THREADS) {
            const int a = a0 + e / BN, bb = e % BN;
            double z = 0.0;
            for (int c = 0; c < WY_JB; ++c) z = fma(Ts[a * WY_JB + c], Z[c * BN + bb], z);
            Zt[a * BN + bb] = z;
        }
        cluster.sync();
        // ---- all-gather op(T) Z into Z (Z itself is no longer read by anyone after the sync)
        for (int e = tid; e < WY_JB * BN; e += WY_THREADS) {
            const int a = e / BN;
            const int owner = a / rows_per_rank;
            Z[e] = owner == rank ? Zt[e] : cluster.map_shared_rank(Zt, owner)[e];
        }
        __syncthreads();
        // ---- W_rows,blk -= V_rows (op(T) Z): thread -> column b, rows ag, ag + G, ...
        {
            double zc[WY_JB];
#pragma unroll
            for (int a = 0; a < WY_JB; ++a) zc[a] = Z[a * BN + b];
            for (int i = ag; i < nr; i += G) {
                double w = Ws[i * (BN + 1) + b];
#pragma unroll
                for (int a = 0; a < WY_JB; ++a) w = fma(-Vs[i * (WY_JB + 1) + a], zc[a], w);
                if (b < nbw) W[static_cast<long long>(r0 + i) * ldw + c0 + b] = w;
            }
        }
        cluster.sync();   // peers may still read this CTA's Zt / Z slices; Ws / Zp are reused next
    }
}

__global__ void qr_init_q_kernel(double* Q, long long ldq, int M, int N) {
    const long long total = static_cast<long long>(M) * N;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / N, j = e % N;
        Q[i * ldq + j] = (i == j) ? 1.0 : 0.0;
    }
}

// R = sign-normalised upper triangle of W[0:N, 0:N] (row i flipped when W_ii < 0).
__global__ void qr_write_r_kernel(const double* W, long long ld, int N, double* R, long long ldr) {
    const long long total = static_cast<long long>(N) * N;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / N, j = e % N;
        const double s = W[i * ld + i] < 0.0 ? -1.0 : 1.0;
        R[i * ldr + j] = (j >= i) ? s * W[i * ld + j] : 0.0;
    }
}

// Flip column j of Q where W_jj < 0 (the matching sign normalisation of Q).
__global__ void qr_flip_q_kernel(const double* W, long long ld, int M, int N, double* Q, long long ldq) {
    const long long total = static_cast<long long>(M) * N;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / N, j = e % N;
        if (W[j * ld + j] < 0.0) Q[i * ldq + j] = -Q[i * ldq + j];
    }
}

// --------------------------------------------------------------------------
// Triangular solves on 32-column diagonal blocks, one thread per row of F.
// --------------------------------------------------------------------------
constexpr int TB = 32;

// trans == 0: F[:, J] <- F[:, J] R_JJ^{-1}   (forward over columns)
// trans == 1: F[:, J] <- F[:, J] R_JJ^{-T}   (backward over columns)
__global__ void trsm_diag_kernel(double* F, long long m, long long ldf, int j0, int jb,
                                 const double* R, long long ldr, int trans) {
    __shared__ double Rs[TB][TB + 1];
    __shared__ double rdiag[TB];   // 1 / R_jj: one division per column and block, not per row
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
        const int a = e / TB, b = e % TB;
        Rs[a][b] = (a < jb && b < jb) ? R[static_cast<long long>(j0 + a) * ldr + j0 + b] : 0.0;
    }
    if (threadIdx.x < TB)
        rdiag[threadIdx.x] = threadIdx.x < jb ? 1.0 / R[static_cast<long long>(j0 + threadIdx.x) * (ldr + 1)] : 0.0;
    __syncthreads();
    const long long row = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (row >= m) return;
    double* f = F + row * ldf + j0;
    double x[TB];
#pragma unroll
    for (int j = 0; j < TB; ++j) x[j] = (j < jb) ? f[j] : 0.0;
    if (!trans) {
#pragma unroll
        for (int j = 0; j < TB; ++j) {
            if (j < jb) {
                double s = x[j];
#pragma unroll
                for (int i = 0; i < TB; ++i)
                    if (i < j) s = fma(-x[i], Rs[i][j], s);
                x[j] = s * rdiag[j];
            }
        }
    } else {
#pragma unroll
        for (int j = TB - 1; j >= 0; --j) {
            if (j < jb) {
                double s = x[j];
#pragma unroll
                for (int i = 0; i < TB; ++i)
                    if (i > j && i < jb) s = fma(-x[i], Rs[j][i], s);
                x[j] = s * rdiag[j];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < TB; ++j)
        if (j < jb) f[j] = x[j];
}

// --------------------------------------------------------------------------
// Core diagnostics: truncation rank and est ||R^{-1}||_2 (one CTA).
// --------------------------------------------------------------------------
constexpr int DG_THREADS = 1024;

__device__ double dg_block_sum(double s, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if (lane == 0) red[warp] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < DG_THREADS / 32; ++w) t += red[w];
    return t;
}

// Solves in place on vector z (length r, in global scratch):
//   lower == 1: R^T y = z (forward);  lower == 0: R w = z (backward).
// Each 32 x 32 diagonal block is staged in shared memory and solved by warp 0;
// the rest of the CTA applies the block's contribution to the remaining entries.
__device__ void dg_tri_solve(const double* R, long long ldr, int r, double* z, int lower,
                             double (*Rb)[33]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = (r + 31) / 32;
    for (int bi = 0; bi < nb; ++bi) {
        const int b = lower ? bi : nb - 1 - bi;
        const int j0 = b * 32;
        const int jb = min(32, r - j0);
        {
            const int a = threadIdx.x >> 5, c = threadIdx.x & 31;   // 1024 threads = 32 x 32
            Rb[a][c] = (a < jb && c < jb) ? R[(j0 + a) * ldr + j0 + c] : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            double zl = lane < jb ? z[j0 + lane] : 0.0;
            if (lower) {
                for (int i = 0; i < jb; ++i) {
                    double yi = __shfl_sync(0xffffffffu, zl, i);
                    yi = yi / Rb[i][i];
                    if (lane == i) zl = yi;
                    if (lane > i && lane < jb) zl = fma(-Rb[i][lane], yi, zl);
                }
            } else {
                for (int i = jb - 1; i >= 0; --i) {
                    double wi = __shfl_sync(0xffffffffu, zl, i);
                    wi = wi / Rb[i][i];
                    if (lane == i) zl = wi;
                    if (lane < i) zl = fma(-Rb[lane][i], wi, zl);
                }
            }
            if (lane < jb) z[j0 + lane] = zl;
        }
        __syncthreads();
        if (lower) {   // z_j -= sum_{i in block} R[i][j] y_i for j after the block
            for (int j = j0 + jb + threadIdx.x; j < r; j += DG_THREADS) {
                double s = z[j];
                for (int i = 0; i < jb; ++i) s = fma(-R[(j0 + i) * ldr + j], z[j0 + i], s);
                z[j] = s;
            }
        } else {       // z_j -= sum_{i in block} R[j][i] w_i for j before the block
            for (int j = threadIdx.x; j < j0; j += DG_THREADS) {
                double s = z[j];
                const double* rr = R + j * ldr + j0;
                for (int i = 0; i < jb; ++i) s = fma(-rr[i], z[j0 + i], s);
                z[j] = s;
            }
        }
        __syncthreads();
    }
}

// out[0] = est ||R^{-1}||_2, out[1] = est ||R||_2, out[2] = eps used; *k_out = truncation rank.
__global__ void __launch_bounds__(DG_THREADS) core_diag_kernel(const double* R, long long ldr, int r,
                                                               double eps, int eps_relative, int want_est,
                                                               int iters, double* z, double* out,
                                                               int* k_out) {
    __shared__ double red[32];
    __shared__ double Rb[32][33];
    __shared__ int kmin;
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const double inv = 1.0 / sqrt(static_cast<double>(r));
    double* y = z + r;
    // ||R||_2 by power iteration on R^T R from the all-ones vector
    double rn = 0.0;
    if (eps_relative) {
        for (int i = threadIdx.x; i < r; i += DG_THREADS) z[i] = inv;
        __syncthreads();
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int it = 0; it < iters; ++it) {
            for (int i = warp; i < r; i += DG_THREADS / 32) {   // y = R z, one warp per row
                double s = 0.0;
                for (int j = i + lane; j < r; j += 32) s = fma(R[static_cast<long long>(i) * ldr + j], z[j], s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) y[i] = s;
            }
            __syncthreads();
            double ss = 0.0;
            for (int j = threadIdx.x; j < r; j += DG_THREADS) {   // w = R^T y
                double s = 0.0;
                for (int i = 0; i <= j; ++i) s = fma(R[static_cast<long long>(i) * ldr + j], y[i], s);
                z[j] = s;   // each thread owns its j
                ss = fma(s, s, ss);
            }
            const double nw = sqrt(dg_block_sum(ss, red));
            if (nw == 0.0 || !isfinite(nw)) {
                rn = nw;
                break;
            }
            rn = sqrt(nw);
            const double sc = 1.0 / nw;
            for (int j = threadIdx.x; j < r; j += DG_THREADS) z[j] *= sc;
            __syncthreads();
        }
        eps = eps * rn;
    }
    if (threadIdx.x == 0) kmin = r;
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += DG_THREADS)
        if (fabs(R[static_cast<long long>(i) * ldr + i]) <= eps) atomicMin(&kmin, i);
    __syncthreads();
    if (threadIdx.x == 0) {
        *k_out = kmin;
        out[1] = rn;
        out[2] = eps;
        out[0] = 0.0;
    }
    if (!want_est) return;
    int has_zero = 0;
    for (int i = threadIdx.x; i < r; i += DG_THREADS)
        if (R[static_cast<long long>(i) * ldr + i] == 0.0) has_zero = 1;
    has_zero = __syncthreads_or(has_zero);
    if (has_zero) {
        if (threadIdx.x == 0) out[0] = inf;
        return;
    }
    for (int i = threadIdx.x; i < r; i += DG_THREADS) z[i] = inv;
    __syncthreads();
    double est = 0.0;
    for (int it = 0; it < iters; ++it) {
        dg_tri_solve(R, ldr, r, z, 1, Rb);
        dg_tri_solve(R, ldr, r, z, 0, Rb);
        double s = 0.0;
        for (int i = threadIdx.x; i < r; i += DG_THREADS) s = fma(z[i], z[i], s);
        const double nw = sqrt(dg_block_sum(s, red));
        if (!isfinite(nw)) {
            est = inf;
            break;
        }
        est = sqrt(nw);
        if (nw == 0.0) break;
        const double sc = 1.0 / nw;
        __syncthreads();
        for (int i = threadIdx.x; i < r; i += DG_THREADS) z[i] *= sc;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = est;
}

// Cluster version of the core diagnostics: rows of R are split over the CTAs of
// a cluster.  The power iteration for ||R||_2 exchanges the matrix-vector
// products through distributed shared memory; the blocked triangular solves of
// the ||R^{-1}||_2 iteration are right-looking: the CTA owning a 32-row block
// solves it with one warp, the block's solution is read by every CTA through
// DSMEM (double-buffered by block parity, one cluster barrier per block), and
// each CTA updates its own rows.  Same results as core_diag_kernel.
constexpr int CD_THREADS = 512;
constexpr int CD_WARPS = CD_THREADS / 32;
constexpr int CD_MAX_R = 4096;

__host__ __device__ inline int cd_rows_per(int r, int cs) { return ((r + cs - 1) / cs + 31) / 32 * 32; }
__host__ __device__ inline size_t cd_smem(int r, int cs) {
    const size_t rp = cd_rows_per(r, cs);
    return sizeof(double) * (2 * static_cast<size_t>(r) + rp + 64 + 32 + 32 * 33 + 8 + (rp / 32) * 32 * 33);
}

__global__ void __launch_bounds__(CD_THREADS) core_diag_cluster_kernel(const double* R, long long ldr, int r,
                                                                      double eps, int eps_relative,
                                                                      int want_est, int iters, double* out,
                                                                      int* k_out) {
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = static_cast<int>(cluster.num_blocks());
    const int rank = static_cast<int>(cluster.block_rank());
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    extern __shared__ double sm[];
    const int rp = cd_rows_per(r, cs);
    double* v = sm;              // [r]  full iterate (identical in every CTA)
    double* u = v + r;           // [r]  gathered R v
    double* loc = u + r;         // [rp] own slice of the vector being solved
    double* blk = loc + rp;      // [2][32] solved block, read by the other CTAs
    double* ybuf = blk + 64;     // [32] local copy of the solved block
    double* Rb = ybuf + 32;      // [32][33] diagonal block (owner)
    double* part = Rb + 32 * 33; // [8] partial norms, double-buffered
    double* Xinv = part + 8;     // [rp/32][32][33] inverses of the owned diagonal blocks
    __shared__ int s_kmin;
    const int s0 = rank * rp;
    const int s1 = min(r, s0 + rp);
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const double inv = 1.0 / sqrt(static_cast<double>(r));

    // ---- ||R||_2 (power iteration on R^T R from the all-ones vector)
    double rn = 0.0;
    if (eps_relative) {
        for (int i = tid; i < r; i += CD_THREADS) v[i] = inv;
        __syncthreads();
        for (int it = 0; it < iters; ++it) {
            const int par = it & 1;
            for (int i = s0 + warp; i < s1; i += CD_WARPS) {   // u_i = (R v)_i, own rows
                double acc = 0.0;
                for (int j = i + lane; j < r; j += 32) acc = fma(R[static_cast<long long>(i) * ldr + j], v[j], acc);
                acc = warp_sum(acc);
                if (lane == 0) u[i] = acc;
            }
            cluster.sync();
            for (int k = 0; k < cs; ++k) {   // gather the other slices of u
                if (k == rank) continue;
                const double* ru = cluster.map_shared_rank(u, k);
                const int a = k * rp, b = min(r, a + rp);
                for (int i = a + tid; i < b; i += CD_THREADS) u[i] = ru[i];
            }
            cluster.sync();
            double ss = 0.0;
            for (int j = s0 + tid; j < s1; j += CD_THREADS) {   // w_j = (R^T u)_j, own columns
                double acc = 0.0;
                for (int i = 0; i <= j; ++i) acc = fma(R[static_cast<long long>(i) * ldr + j], u[i], acc);
                v[j] = acc;
                ss = fma(acc, acc, ss);
            }
            ss = warp_sum(ss);
            if (lane == 0) Rb[warp] = ss;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < CD_WARPS; ++w) t += Rb[w];
                part[par] = t;
            }
            cluster.sync();
            double nw2 = 0.0;
            for (int k = 0; k < cs; ++k) nw2 += cluster.map_shared_rank(part, k)[par];
            for (int k = 0; k < cs; ++k) {   // gather the other slices of w into v
                if (k == rank) continue;
                const double* rv = cluster.map_shared_rank(v, k);
                const int a = k * rp, b = min(r, a + rp);
                for (int i = a + tid; i < b; i += CD_THREADS) v[i] = rv[i];
            }
            const double nw = sqrt(nw2);
            cluster.sync();   // every CTA has read my slice of v before it is rescaled
            if (nw == 0.0 || !isfinite(nw)) {
                rn = nw;
                break;
            }
            rn = sqrt(nw);
            const double sc = 1.0 / nw;
            for (int i = tid; i < r; i += CD_THREADS) v[i] *= sc;
            __syncthreads();
        }
        eps = eps * rn;
    }

    // ---- truncation rank (every CTA scans the diagonal; rank 0 reports)
    if (tid == 0) s_kmin = r;
    __syncthreads();
    int zero_diag = 0;
    for (int i = tid; i < r; i += CD_THREADS) {
        const double d = R[static_cast<long long>(i) * ldr + i];
        if (fabs(d) <= eps) atomicMin(&s_kmin, i);
        if (d == 0.0) zero_diag = 1;
    }
    zero_diag = __syncthreads_or(zero_diag);
    if (rank == 0 && tid == 0) {
        *k_out = s_kmin;
        out[1] = rn;
        out[2] = eps;
        out[0] = 0.0;
    }
    if (!want_est) {
        cluster.sync();
        return;
    }
    if (zero_diag) {
        if (rank == 0 && tid == 0) out[0] = inf;
        cluster.sync();
        return;
    }

    // ---- ||R^{-1}||_2 (power iteration on R^{-1} R^{-T} from the all-ones vector)
    // Blocked substitution over 32-row blocks.  Each CTA first inverts the
    // diagonal blocks it owns (once, in shared memory), so a block step is a
    // 32 x 32 matrix-vector product instead of a 32-step dependent chain.
    const int nb = (r + 31) / 32;
    for (int ob = warp; ob * 32 < s1 - s0; ob += CD_WARPS) {
        const int j0 = s0 + ob * 32, jb = min(32, r - j0);
        double* X = Xinv + ob * 32 * 33;
        // load D (identity padding beyond jb), then invert in place: rows from the
        // bottom, X[i][j] = (delta_ij - sum_{i<k<=j} D[i][k] X[k][j]) / D[i][i]
#pragma unroll 4
        for (int a = 0; a < 32; ++a)
            X[a * 33 + lane] = (a < jb && lane < jb) ? (lane >= a ? R[static_cast<long long>(j0 + a) * ldr + j0 + lane] : 0.0)
                                                     : (a == lane ? 1.0 : 0.0);
        __syncwarp();
        const double rdl = 1.0 / X[lane * 33 + lane];
        for (int i = 31; i >= 0; --i) {
            double acc = lane == i ? 1.0 : 0.0;
            for (int k = i + 1; k <= lane; ++k) acc = fma(-X[i * 33 + k], X[k * 33 + lane], acc);
            const double rdi = __shfl_sync(0xffffffffu, rdl, i);   // every lane takes part
            const double xi = lane >= i ? acc * rdi : 0.0;
            __syncwarp();
            X[i * 33 + lane] = xi;
            __syncwarp();
        }
    }
    for (int i = s0 + tid; i < s1; i += CD_THREADS) loc[i - s0] = inv;
    __syncthreads();
    double est = 0.0;
    const int ra = tid >> 4, rpart = tid & 15;   // block product: row ra, k = rpart, rpart + 16
    const int urow = tid >> 2, uq = tid & 3;      // updates: 4 lanes per row, 8 terms each
    for (int it = 0; it < iters; ++it) {
        for (int pass = 0; pass < 2; ++pass) {   // pass 0: R^T y = z; pass 1: R w = y
            for (int bi = 0; bi < nb; ++bi) {
                const int b = pass == 0 ? bi : nb - 1 - bi;
                const int j0 = b * 32, jb = min(32, r - j0);
                const int owner = j0 / rp;
                if (rank == owner) {
                    const double* X = Xinv + ((j0 - s0) >> 5) * 32 * 33;
                    const int k0 = rpart, k1 = rpart + 16;
                    const double z0 = k0 < jb ? loc[j0 - s0 + k0] : 0.0;
                    const double z1 = k1 < jb ? loc[j0 - s0 + k1] : 0.0;
                    // pass 0: y = X^T z (X upper); pass 1: w = X y
                    double acc = pass == 0 ? fma(X[k0 * 33 + ra], z0, X[k1 * 33 + ra] * z1)
                                           : fma(X[ra * 33 + k0], z0, X[ra * 33 + k1] * z1);
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    __syncthreads();   // every block-product read of loc is done
                    // buffer alternates with (b + pass): consecutive blocks, including the
                    // last block of one pass and the first of the next, never share a slot
                    if (rpart == 0 && ra < jb) {
                        loc[j0 - s0 + ra] = acc;
                        blk[((b + pass) & 1) * 32 + ra] = acc;
                    }
                }
                cluster.sync();
                if (tid < jb) ybuf[tid] = cluster.map_shared_rank(blk, owner)[((b + pass) & 1) * 32 + tid];
                __syncthreads();
                if (pass == 0) {   // z_j -= sum_{i in block} R[i][j] y_i, own rows j after the block
                    const int jlo = max(s0, j0 + jb);
                    for (int base = jlo; base < s1; base += CD_THREADS / 4) {
                        const int j = base + urow;
                        double acc = 0.0;
                        if (j < s1) {
#pragma unroll
                            for (int t = 0; t < 8; ++t) {
                                const int i = uq * 8 + t;
                                if (i < jb) acc = fma(R[static_cast<long long>(j0 + i) * ldr + j], ybuf[i], acc);
                            }
                        }
                        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                        if (j < s1 && uq == 0) loc[j - s0] -= acc;
                    }
                } else {           // y_i -= sum_{j in block} R[i][j] w_j, own rows i before the block
                    const int ihi = min(s1, j0);
                    for (int base = s0; base < ihi; base += CD_THREADS / 4) {
                        const int i = base + urow;
                        double acc = 0.0;
                        if (i < ihi) {
                            const double* rr = R + static_cast<long long>(i) * ldr + j0;
#pragma unroll
                            for (int t = 0; t < 8; ++t) {
                                const int j = uq * 8 + t;
                                if (j < jb) acc = fma(rr[j], ybuf[j], acc);
                            }
                        }
                        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                        if (i < ihi && uq == 0) loc[i - s0] -= acc;
                    }
                }
                __syncthreads();
            }
        }
        const int par = it & 1;
        double ss = 0.0;
        for (int i = s0 + tid; i < s1; i += CD_THREADS) ss = fma(loc[i - s0], loc[i - s0], ss);
        ss = warp_sum(ss);
        if (lane == 0) Rb[warp] = ss;   // Rb is free here (owner warps are done)
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < CD_WARPS; ++w) t += Rb[w];
            part[2 + par] = t;
        }
        cluster.sync();
        double nw2 = 0.0;
        for (int k = 0; k < cs; ++k) nw2 += cluster.map_shared_rank(part, k)[2 + par];
        const double nw = sqrt(nw2);
        if (!isfinite(nw)) {
            est = inf;
            break;
        }
        est = sqrt(nw);
        if (nw == 0.0) break;
        const double sc = 1.0 / nw;
        for (int i = s0 + tid; i < s1; i += CD_THREADS) loc[i - s0] *= sc;
        __syncthreads();
    }
    if (rank == 0 && tid == 0) out[0] = est;
    cluster.sync();
}

// --------------------------------------------------------------------------
// Elementwise helpers
// --------------------------------------------------------------------------
__global__ void copy_f32_f64_kernel(const float* __restrict__ s, long long rows, long long cols,
                                    long long lds, double* d, long long ldd) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e % cols;
        d[i * ldd + j] = static_cast<double>(s[i * lds + j]);
    }
}

__global__ void split3_kernel(const float* __restrict__ s, long long rows, long long cols, long long lds,
                              __nv_bfloat16* hi, __nv_bfloat16* mid, __nv_bfloat16* lo, long long ldd) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e % cols;
        const float x = s[i * lds + j];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(m);
        hi[i * ldd + j] = h;
        mid[i * ldd + j] = m;
        lo[i * ldd + j] = __float2bfloat16_rn(r2);
    }
}

__global__ void sum3_kernel(const float* __restrict__ a, const float* __restrict__ b,
                            const float* __restrict__ c, long long rows, long long cols, long long lds,
                            double* d, long long ldd) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e % cols;
        const long long o = i * lds + j;
        d[i * ldd + j] = static_cast<double>(a[o]) + static_cast<double>(b[o]) + static_cast<double>(c[o]);
    }
}

// FP64 / FP32 -> BF16 (round to nearest even through FP32); optional low part.
__global__ void quantize_kernel(const void* __restrict__ src, int src_f64, long long rows, long long cols,
                                long long lds, __nv_bfloat16* hi, __nv_bfloat16* lo, long long ldd) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e % cols;
        const float x = src_f64 ? static_cast<float>(static_cast<const double*>(src)[i * lds + j])
                                : static_cast<const float*>(src)[i * lds + j];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[i * ldd + j] = h;
        if (lo) lo[i * ldd + j] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

__global__ void transpose_rows_kernel(const double* __restrict__ s, long long rows, long long cols,
                                      long long lds, long long keep, double* d, long long ldd) {
    // d (cols x rows) = [s[0:keep, :]^T | 0]
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long j = e / rows, i = e % rows;   // d[j][i]
        d[j * ldd + i] = (i < keep) ? s[i * lds + j] : 0.0;
    }
}

// Latch GN_ERR_NONFINITE when the upper triangle of R (r x r) holds a NaN or an
// infinity: a non-finite entry anywhere in the core reaches R's last columns.
__global__ void nonfinite_upper_kernel(const double* __restrict__ R, long long r, long long ldr,
                                       int32_t* status) {
    const long long total = r * r;
    bool bad = false;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / r, j = e - i * r;
        if (j >= i && !isfinite(R[i * ldr + j])) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
        if (atomicCAS(&status[GN_DEV_STATUS], 0, GN_ERR_NONFINITE) == 0) status[GN_DEV_WHERE] = 20;
    }
}

__global__ void zero_kernel(double* p, long long rows, long long cols, long long ld) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        p[(e / cols) * ld + e % cols] = 0.0;
}

int ew_blocks(gn_handle h, long long total) {
    return static_cast<int>(std::max<long long>(1, std::min<long long>((total + 255) / 256, 8LL * h->sm_count)));
}

}  // namespace

// ============================================================================ host
size_t dgemm_ws_bytes(long long M, long long N, long long K, int sm_count) {
    return static_cast<size_t>(choose_splits(M, N, K, sm_count)) * M * N * sizeof(double);
}

gn_status dgemm(gn_handle h, long long M, long long N, long long K, double alpha, const double* A,
                long long lda, int ta, const double* B, long long ldb, int tb, double beta, double* C,
                long long ldc, double* ws, size_t ws_bytes) {
    return dgemm_impl<double, double>(h, M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, ws, ws_bytes);
}

gn_status dgemm_a32(gn_handle h, long long M, long long N, long long K, double alpha, const float* A,
                    long long lda, int ta, const double* B, long long ldb, int tb, double beta, double* C,
                    long long ldc, double* ws, size_t ws_bytes) {
    return dgemm_impl<float, double>(h, M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, ws, ws_bytes);
}

gn_status dgemm_b32(gn_handle h, long long M, long long N, long long K, double alpha, const double* A,
                    long long lda, int ta, const float* B, long long ldb, int tb, double beta, double* C,
                    long long ldc, double* ws, size_t ws_bytes) {
    return dgemm_impl<double, float>(h, M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, ws, ws_bytes);
}

gn_status latch_nonfinite_upper(gn_handle h, const double* R, long long r, long long ldr) {
    nonfinite_upper_kernel<<<ew_blocks(h, r * r), 256, 0, h->stream>>>(R, r, ldr, h->dstatus); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status set_zero_f64(gn_handle h, double* p, long long rows, long long cols, long long ld) {
    if (rows <= 0 || cols <= 0) return GN_OK;
    zero_kernel<<<ew_blocks(h, rows * cols), 256, 0, h->stream>>>(p, rows, cols, ld); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

// QR workspace: V (M x N), tau (N), T per panel (jb x jb), Z1, Z2 (jb x N), GEMM split-K.
size_t qr_ws_bytes(long long M, long long N, int sm_count) {
    const long long panels = (N + QR_JB - 1) / QR_JB;
    size_t b = sizeof(double) * (M * N + N + panels * QR_NB * QR_NB + 2 * QR_NB * N);
    b += std::max(dgemm_ws_bytes(QR_NB, N, M, sm_count), dgemm_ws_bytes(QR_JB, N, M, sm_count));
    return b + 256;
}

namespace {
struct QrWs {
    double *V, *tau, *Tall, *Z1, *Z2, *gws;
    size_t gws_bytes;
};

QrWs qr_carve(long long M, long long N, double* ws, size_t ws_bytes) {
    const long long panels = (N + QR_JB - 1) / QR_JB;
    QrWs q;
    q.V = ws;
    q.tau = q.V + M * N;
    q.Tall = q.tau + N;
    q.Z1 = q.Tall + panels * QR_NB * QR_NB;
    q.Z2 = q.Z1 + QR_NB * N;
    q.gws = q.Z2 + QR_NB * N;
    q.gws_bytes = ws_bytes - sizeof(double) * (q.gws - ws);
    return q;
}

constexpr size_t CP_SMEM_MAX = 200 * 1024;

// Panel scheme for an M x N factorization: the cluster kernel with 32- or
// 16-wide panels when a panel's rows fit the cluster's shared memory, else the
// single-CTA kernel (global-memory panel for tall inputs).
struct PanelCfg {
    int nb;
    int cluster;
    int cs;
};

int cluster_size(gn_handle h) {
    static int cached = -1;
    if (cached >= 0) return cached;
    cached = 0;
    cudaFuncSetAttribute(qr_panel_cluster_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(CP_SMEM_MAX));
    cudaFuncSetAttribute(qr_panel_cluster_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(CP_SMEM_MAX));
    cudaFuncSetAttribute(qr_panel_cluster_kernel<32>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(qr_panel_cluster_kernel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int cs : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(CP_THREADS);
        cfg.dynamicSmemBytes = CP_SMEM_MAX;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, qr_panel_cluster_kernel<32>, &cfg) == cudaSuccess && n >= 1 &&
            cudaOccupancyMaxActiveClusters(&n, qr_panel_cluster_kernel<16>, &cfg) == cudaSuccess && n >= 1) {
            cached = cs;
            break;
        }
    }
    cudaGetLastError();
    (void)h;
    return cached;
}

PanelCfg panel_cfg(gn_handle h, long long M) {
    const int cs = cluster_size(h);
    if (cs > 0) {
        const int rp = static_cast<int>((M + cs - 1) / cs);
        if (cluster_panel_smem<32>(rp) <= CP_SMEM_MAX) return {32, 1, cs};
        if (cluster_panel_smem<16>(rp) <= CP_SMEM_MAX) return {16, 1, cs};
    }
    return {QR_JB, 0, 0};
}

gn_status launch_cluster_panel(gn_handle h, const PanelCfg& pc, double* W, long long ld, long long M,
                               long long j0, int jb, double* V, long long ldv, double* tau, double* T) {
    const long long Mp = M - j0;
    const int rows_per = static_cast<int>((Mp + pc.cs - 1) / pc.cs);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pc.cs);
    cfg.blockDim = dim3(CP_THREADS);
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pc.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int Mi = static_cast<int>(M), j0i = static_cast<int>(j0);
    if (pc.nb == 32) {
        cfg.dynamicSmemBytes = cluster_panel_smem<32>(rows_per);
        GN_CUDA_TRY(cudaLaunchKernelEx(&cfg, qr_panel_cluster_kernel<32>, W, ld, Mi, j0i, jb, V, ldv, tau, T,
                                       rows_per));
    } else {
        cfg.dynamicSmemBytes = cluster_panel_smem<16>(rows_per);
        GN_CUDA_TRY(cudaLaunchKernelEx(&cfg, qr_panel_cluster_kernel<16>, W, ld, Mi, j0i, jb, V, ldv, tau, T,
                                       rows_per));
    }
    count_launch();
    return GN_OK;
}
}  // namespace

template <int BN>
bool wy_attrs() {
    return cudaFuncSetAttribute(qr_wy_apply_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(wy_smem(WY_MAX_ROWS, BN))) == cudaSuccess &&
           cudaFuncSetAttribute(qr_wy_apply_kernel<BN>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
               cudaSuccess;
}

// Largest cluster size the WY kernel can launch with (0: none).
int wy_cluster_max() {
    static int cs_max = -1;
    if (cs_max < 0) {
        cs_max = 0;
        if (wy_attrs<64>() && wy_attrs<32>() && wy_attrs<16>() && wy_attrs<8>()) {
            for (int cs : {16, 8}) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(cs);
                cfg.blockDim = dim3(WY_THREADS);
                cfg.dynamicSmemBytes = wy_smem(WY_MAX_ROWS, 64);
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = cs;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int n = 0;
                if (cudaOccupancyMaxActiveClusters(&n, qr_wy_apply_kernel<64>, &cfg) == cudaSuccess && n >= 1) {
                    cs_max = cs;
                    break;
                }
            }
        }
        cudaGetLastError();
    }
    return cs_max;
}

// Clusters of cs CTAs that fit at once with one CTA per SM (cached per size).
int wy_cluster_capacity(int cs, int sm_count) {
    static int cap[17] = {0};
    if (cs < 1 || cs > 16) return 1;
    if (cap[cs] == 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(WY_THREADS);
        cfg.dynamicSmemBytes = wy_smem(WY_MAX_ROWS, 64);   // > half an SM's shared memory
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, qr_wy_apply_kernel<64>, &cfg) != cudaSuccess || n < 1)
            n = sm_count / cs > 0 ? sm_count / cs : 1;
        cudaGetLastError();
        cap[cs] = n;
    }
    return cap[cs];
}

// Whether wy_apply can handle panels with up to Mp rows.
bool wy_usable(long long Mp) {
    const int cm = wy_cluster_max();
    return cm > 0 && (Mp + cm - 1) / cm <= WY_MAX_ROWS;
}

// One-launch compact-WY application when a row slice of the panel fits a CTA's
// shared memory; returns GN_ERR_UNSUPPORTED otherwise (the caller then uses the
// GEMM sequence).  reserve: another 16-CTA cluster runs alongside (a panel or
// the diagnostics), so one cluster slot of 16 SMs is left free.
gn_status wy_apply(gn_handle h, double* W, long long ldw, long long Mp, long long Nw, const double* V, long long ldv,
                   int jb, const double* T, int transT, int reserve) {
    const int cs_max = wy_cluster_max();
    if (cs_max == 0 || jb > WY_JB || Mp <= 0 || Nw <= 0) return GN_ERR_UNSUPPORTED;
    // Cluster size (rows per CTA) and column block width: the kernel is bound by
    // each SM's FP64 rate and its clusters loop over the blocks, so its time is
    // ~ ceil(blocks / clusters) x rows per CTA x (bn + a fixed cost of about 8
    // columns' work per block).
    int cs = 0, bn = 64;
    long long rp = 0, best = -1, ncl = 1;
    for (int c : {8, 16}) {
        if (c > cs_max) continue;
        const long long rpc = (Mp + c - 1) / c;
        if (rpc > WY_MAX_ROWS) continue;
        const long long capc = std::max<long long>(1, wy_cluster_capacity(c, h->sm_count) - (reserve ? 16 / c : 0));
        for (int cand : {64, 32, 16, 8}) {
            const long long nb = (Nw + cand - 1) / cand;
            const long long per = (nb + capc - 1) / capc;   // blocks per cluster
            const long long cost = per * rpc * (cand + 8);
            if (best < 0 || cost < best) {
                best = cost;
                cs = c;
                bn = cand;
                rp = rpc;
                ncl = std::min<long long>(nb, capc);
            }
        }
    }
    if (cs == 0) return GN_ERR_UNSUPPORTED;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(ncl * cs));
    cfg.blockDim = dim3(WY_THREADS);
    cfg.dynamicSmemBytes = wy_smem(static_cast<int>(rp), bn);
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int mpi = static_cast<int>(Mp), nwi = static_cast<int>(Nw), rpi = static_cast<int>(rp);
    switch (bn) {
        case 64: GN_CUDA_TRY(cudaLaunchKernelEx(&cfg, qr_wy_apply_kernel<64>, W, ldw, mpi, nwi, V, ldv, jb, T, transT, rpi)); break;
        case 32: GN_CUDA_TRY(cudaLaunchKernelEx(&cfg, qr_wy_apply_kernel<32>, W, ldw, mpi, nwi, V, ldv, jb, T, transT, rpi)); break;
        case 16: GN_CUDA_TRY(cudaLaunchKernelEx(&cfg, qr_wy_apply_kernel<16>, W, ldw, mpi, nwi, V, ldv, jb, T, transT, rpi)); break;
        default: GN_CUDA_TRY(cudaLaunchKernelEx(&cfg, qr_wy_apply_kernel<8>, W, ldw, mpi, nwi, V, ldv, jb, T, transT, rpi)); break;
    }
    count_launch();
    return GN_OK;
}

namespace {

// T = S^{-1} for S = striu(G) + diag(1 / tau) (n x n upper triangular, n <=
// QR_SB): the UT transform of a block of reflectors, H_0 ... H_{n-1} = I - V T V^T
// with G = V^T V (Puglisi 1992; Joffrain et al. 2006).  Column w of T solves
// S x = e_w by back substitution x_i = tau_i (x_i - sum_{k>i} G_ik x_k), from
// i = w up (x_i = 0 below w); a dropped reflector (tau_i = 0) gets x_i = 0.
// One warp per column.
constexpr int QR_SB = 256;   // reflectors per block of the tensor-core Q formation

// Four warps per CTA, one per SM sub-partition (each warp's FP64 instructions
// then have a sub-partition's FP64 unit to themselves); CTA b takes columns b,
// b + G, b + 2G, b + 3G (G = gridDim.x), one from each quarter, so the CTAs
// carry equal work.  No CTA-wide barrier: a warp past n just returns.
__global__ void __launch_bounds__(128) ut_inverse_kernel(const double* __restrict__ G, long long ldg,
                                                         const double* __restrict__ tau, int n,
                                                         double* __restrict__ X, long long ldx) {
    const int w = blockIdx.x + gridDim.x * (threadIdx.x >> 5);   // the column of T this warp solves for
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    constexpr int NT = QR_SB / 32;
    // lane l holds x_{32 t + l}; blocks of 32 rows from the one holding row w up.
    // Inside a block: back substitution, one row per step (the row's final value
    // broadcast from its lane, the rows below it in the block updated in their
    // lanes).  After a block: its contribution removed from the blocks above
    // with G_{k, 32m + l} = G_{32m + l, k} (G is symmetric), read along rows.
    double x[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) x[t] = (32 * t + lane == w) ? 1.0 : 0.0;
    const int qb = w >> 5;
#pragma unroll
    for (int p = NT - 1; p >= 0; --p) {
        if (p > qb) continue;   // warp-uniform
        // the block's coefficients in registers first (loads off the chain):
        // G rows 32p .. 32p + 31 of this lane's column (G is ldg x ldg, ldg >=
        // QR_SB, so every row read exists; rows past w are never used) and tau
        double gcol[32];
#pragma unroll
        for (int sr = 0; sr < 32; ++sr) gcol[sr] = G[static_cast<long long>(32 * p + sr) * ldg + 32 * p + lane];
        const double tl = 32 * p + lane < n ? tau[32 * p + lane] : 0.0;
#pragma unroll
        for (int sr = 31; sr >= 0; --sr) {
            const int i = 32 * p + sr;
            if (i > w) continue;   // rows past w stay zero
            // the chain per row is one shuffle and one FMA: tau_i scales the
            // coefficients (off the chain), not the broadcast value
            const double ti = __shfl_sync(0xffffffffu, tl, sr);
            const double cik = lane < sr ? gcol[sr] * ti : 0.0;
            const double xu = __shfl_sync(0xffffffffu, x[p], sr);
            x[p] = lane == sr ? xu * ti : fma(-cik, xu, x[p]);
        }
        if (p == 0) break;
        // two partial sums per block row: half the FMA chain; rows past w
        // contribute nothing (their coefficient is taken as 0, not their value)
        double y[NT];
#pragma unroll
        for (int m = 0; m < NT; ++m) y[m] = 0.0;
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const int k = 32 * p + kk;
            const bool on = k <= w;
            const double xk = __shfl_sync(0xffffffffu, x[p], kk);
            const double* gk = G + static_cast<long long>(k) * ldg + lane;
#pragma unroll
            for (int m = 0; m < NT; ++m) {
                if (m >= p) continue;
                const double g = on ? gk[32 * m] : 0.0;
                if (kk & 1) y[m] = fma(-g, xk, y[m]);
                else x[m] = fma(-g, xk, x[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < NT; ++m)
            if (m < p) x[m] += y[m];
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int k = lane + 32 * t;
        if (k < n) X[k * ldx + w] = x[t];
    }
}

void launch_ut_inverse(gn_handle h, const double* G, long long ldg, const double* tau, int n, double* X,
                       long long ldx) {
    ut_inverse_kernel<<<static_cast<unsigned>((n + 3) / 4), 128, 0, h->stream>>>(G, ldg, tau, n, X, ldx);
    count_launch();
}

// Zero V above the diagonal inside each block of QR_SB reflectors: a panel
// writes its reflectors from its own first row down, so rows of the block's
// earlier panels are left unwritten in its columns.
__global__ void v_zero_upper_kernel(double* V, long long ldv, int N) {
    const long long total = static_cast<long long>(N) * QR_SB;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(e / QR_SB), i = (c / QR_SB) * QR_SB + static_cast<int>(e % QR_SB);
        if (i < c) V[static_cast<long long>(i) * ldv + c] = 0.0;
    }
}

}  // namespace

// Two-level blocking of the look-ahead factorization (tensor-core trailing
// updates): blocks of QR_BB columns, each factored as nb-wide panels whose
// FP64 updates stay inside the block; after a block, its QR_BB reflectors
// update the next block on the high-priority chain and everything further
// right on the side stream (one block behind), as three digit-sliced products
// with the block's T from its Gram matrix (ut_inverse).  The trailing matrix is
// sliced and combined once per block instead of once per panel.
constexpr int QR_BB = 256;

size_t qr_oz_side_bytes(long long M, long long N) {
    return oz_ws_bytes(std::max<long long>(M, QR_SB), std::max<long long>(N, QR_SB), M, 0);
}
size_t qr_oz_crit_bytes(long long M) { return oz_ws_bytes(std::max<long long>(M, QR_BB), QR_BB, M, 0); }
size_t al256d(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }
size_t qr_blk_bytes(long long M, long long N) {
    const long long nblk = (N + QR_BB - 1) / QR_BB;
    return al256d(qr_oz_crit_bytes(M)) + al256d(sizeof(double) * nblk * QR_BB * QR_BB) +
           al256d(sizeof(double) * QR_BB * QR_BB) + 2 * al256d(sizeof(double) * QR_BB * N) +
           al256d(sizeof(double) * QR_BB * QR_BB) + al256d(sizeof(double) * nblk * M * QR_BB) + 1024;
}

struct QrBlk {
    void* oz_side;
    size_t oz_side_bytes;
    void* oz_crit;
    size_t oz_crit_bytes;
    double *TB, *GB, *Z1s, *Z2s, *Z1c;
    double* UB;   // U_b = V_b T_b (M_p x b_w, ld QR_BB) of every block but the last, at UB + b M QR_BB
};

bool qr_blk_carve(long long M, long long N, void* oz, size_t oz_bytes, QrBlk* b) {
    if (!oz || (reinterpret_cast<uintptr_t>(oz) & 255)) return false;
    char* p = static_cast<char*>(oz);
    size_t off = 0;
    auto take = [&](size_t n) {
        char* q = p + off;
        off += al256d(n);
        return q;
    };
    const long long nblk = (N + QR_BB - 1) / QR_BB;
    b->oz_side_bytes = qr_oz_side_bytes(M, N);
    b->oz_side = take(b->oz_side_bytes);
    b->oz_crit_bytes = qr_oz_crit_bytes(M);
    b->oz_crit = take(b->oz_crit_bytes);
    b->TB = reinterpret_cast<double*>(take(sizeof(double) * nblk * QR_BB * QR_BB));
    b->GB = reinterpret_cast<double*>(take(sizeof(double) * QR_BB * QR_BB));
    b->Z1s = reinterpret_cast<double*>(take(sizeof(double) * QR_BB * N));
    b->Z2s = reinterpret_cast<double*>(take(sizeof(double) * QR_BB * N));
    b->Z1c = reinterpret_cast<double*>(take(sizeof(double) * QR_BB * QR_BB));
    b->UB = reinterpret_cast<double*>(take(sizeof(double) * nblk * M * QR_BB));
    return off <= oz_bytes;
}

// C (Mp x nc at ldc) <- (I - V T V^T)^T C = C - V (T^T V^T C), V: Mp x bw at
// ldv, T bw x bw upper triangular, given as U = V T (Mp x bw at ldu, formed once
// per block): Z = U^T C, C -= V Z, both digit-sliced.
gn_status block_apply_u(gn_handle h, double* C, long long ldc, long long Mp, long long nc, const double* V,
                        long long ldv, int bw, const double* U, long long ldu, double* Z, void* oz, size_t oz_bytes) {
    GN_TRY(oz_dgemm(h, bw, nc, Mp, 1.0, U, 0, ldu, 1, C, ldc, 0, 0.0, Z, nc, oz, oz_bytes));
    return oz_dgemm(h, Mp, nc, bw, -1.0, V, 0, ldv, 0, Z, nc, 0, 1.0, C, ldc, oz, oz_bytes);
}

// Whether qr_factor takes the blocked path for this shape and workspace (and,
// when it does, the workspace's regions): the look-ahead (cluster panels, side
// and high-priority streams, one-launch WY) and at least two blocks.
bool qr_blocked_path(gn_handle h, long long M, long long N, void* oz, size_t oz_bytes, QrBlk* bk) {
    const PanelCfg pc = panel_cfg(h, M);
    const bool lookahead = pc.cluster && h->side != nullptr && h->crit != nullptr && wy_usable(M);
    return lookahead && N >= 2 * QR_BB && QR_BB % pc.nb == 0 && qr_blk_carve(M, N, oz, oz_bytes, bk);
}

gn_status qr_factor(gn_handle h, double* W, long long M, long long N, long long ld, double* R, long long ldr,
                    double* ws, size_t ws_bytes, void* oz, size_t oz_bytes) {
    if (M < N || N <= 0) return GN_ERR_SHAPE;
    if (ws_bytes < qr_ws_bytes(M, N, h->sm_count)) return GN_ERR_WORKSPACE;
    QrWs q = qr_carve(M, N, ws, ws_bytes);
    static bool attr = false;
    if (!attr) {
        GN_CUDA_TRY(cudaFuncSetAttribute(qr_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(QR_SMEM_PANEL_MAX)));
        attr = true;
    }
    const PanelCfg pc = panel_cfg(h, M);
    const int nb = pc.nb;
    auto factor_panel = [&](long long j0) -> gn_status {
        const int jb = static_cast<int>(std::min<long long>(nb, N - j0));
        const long long Mp = M - j0;
        double* T = q.Tall + (j0 / nb) * QR_NB * QR_NB;
        if (pc.cluster) return launch_cluster_panel(h, pc, W, ld, M, j0, jb, q.V, N, q.tau, T);
        const size_t panel_bytes = static_cast<size_t>(Mp) * (jb + 1) * sizeof(double);
        const int use_smem = panel_bytes <= QR_SMEM_PANEL_MAX ? 1 : 0;
        qr_panel_kernel<<<1, QR_THREADS, use_smem ? panel_bytes : 0, h->stream>>>(
            W, ld, static_cast<int>(M), static_cast<int>(j0), jb, q.V, N, q.tau, T, use_smem); count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        return GN_OK;
    };
    // Look-ahead: after panel j only panel j+1's columns are updated on the main
    // stream; panel j+1 is then factored (16-SM cluster) while the rest of the
    // trailing update runs on the side stream.  Requires the one-launch WY path.
    const bool lookahead = pc.cluster && h->side != nullptr && h->crit != nullptr && wy_usable(M);
    // The look-ahead chain (next-block updates and panels) runs on a
    // high-priority stream so the block scheduler places its clusters ahead of
    // the trailing updates queued on the side stream.
    const gn_handle h0 = h;
    gn_handle_s crit = *h;
    if (lookahead) {
        crit.stream = h->crit;
        GN_CUDA_TRY(cudaEventRecord(h->ev_crit0, h->stream));
        GN_CUDA_TRY(cudaStreamWaitEvent(h->crit, h->ev_crit0, 0));
        h = &crit;
    }
    bool had_second = false, side_used = false;
    QrBlk bk;
    const bool blocked = lookahead && qr_blocked_path(h0, M, N, oz, oz_bytes, &bk);
    if (blocked) {
        // rows above a panel inside its block are part of V_B and must read zero
        GN_CUDA_TRY(cudaMemsetAsync(q.V, 0, sizeof(double) * M * N, h->stream));
        bool pending = false;   // the previous block's side update of the next block's columns is queued
        const long long nblk = (N + QR_BB - 1) / QR_BB;
        for (long long bi = 0; bi < nblk; ++bi) {
            const long long b0 = bi * QR_BB, bw = std::min<long long>(QR_BB, N - b0);
            for (long long j0 = b0; j0 < b0 + bw; j0 += nb) {
                GN_TRY(factor_panel(j0));
                const int jb = static_cast<int>(std::min<long long>(nb, b0 + bw - j0));
                const long long rest = b0 + bw - j0 - jb;
                if (rest > 0)
                    GN_TRY(wy_apply(h, W + j0 * ld + j0 + jb, ld, M - j0, rest, q.V + j0 * N + j0, N, jb,
                                    q.Tall + (j0 / nb) * QR_NB * QR_NB, 1, 0));
            }
            const long long N2 = N - b0 - bw;
            if (N2 <= 0) break;
            const long long Mp = M - b0;
            const double* VB = q.V + b0 * N + b0;
            double* TB = bk.TB + bi * QR_BB * QR_BB;
            GN_TRY(oz_dgemm(h, bw, bw, Mp, 1.0, VB, 0, N, 1, VB, N, 0, 0.0, bk.GB, QR_BB, bk.oz_crit,
                            bk.oz_crit_bytes));
            launch_ut_inverse(h, bk.GB, QR_BB, q.tau + b0, static_cast<int>(bw), TB, QR_BB);
            GN_CUDA_TRY(cudaGetLastError());
            // the next block's columns already have the block before this one (side stream)
            if (pending) GN_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
            // U_b = V_b T_b (kept for the formation of Q): each update below is then two
            // products, Z = U_b^T C and C -= V_b Z
            double* UB = bk.UB + bi * M * QR_BB;
            GN_TRY(oz_dgemm(h, Mp, bw, bw, 1.0, VB, 0, N, 0, TB, QR_BB, 0, 0.0, UB, QR_BB, bk.oz_crit,
                            bk.oz_crit_bytes));
            const long long nnext = std::min<long long>(QR_BB, N2);
            const long long nsec = std::min<long long>(QR_BB, N2 - nnext);
            const long long nrest = N2 - nnext - nsec;
            if (nsec > 0) {   // everything right of the next block, on the side stream, in one update: the
                              // chain waits for it only after the next block's panels
                GN_CUDA_TRY(cudaEventRecord(h->ev_fork, h->stream));
                GN_CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
                gn_handle_s side = *h;
                side.stream = h->side;
                GN_TRY(block_apply_u(&side, W + b0 * ld + b0 + bw + nnext, ld, Mp, nsec + nrest, VB, N,
                                     static_cast<int>(bw), UB, QR_BB, bk.Z1s, bk.oz_side, bk.oz_side_bytes));
                GN_CUDA_TRY(cudaEventRecord(h->ev_join, h->side));
                side_used = true;
            }
            pending = nsec > 0;
            GN_TRY(block_apply_u(h, W + b0 * ld + b0 + bw, ld, Mp, nnext, VB, N, static_cast<int>(bw), UB, QR_BB,
                                 bk.Z1c, bk.oz_crit, bk.oz_crit_bytes));
        }
    } else {
        GN_TRY(factor_panel(0));
    }
    for (long long j0 = 0; j0 < N && !blocked; j0 += nb) {
        const int jb = static_cast<int>(std::min<long long>(nb, N - j0));
        const long long Mp = M - j0;
        const long long N2 = N - j0 - jb;
        if (N2 <= 0) break;
        double* T = q.Tall + (j0 / nb) * QR_NB * QR_NB;
        double* W2 = W + j0 * ld + j0 + jb;
        const double* Vb = q.V + j0 * N + j0;
        if (lookahead) {
            // W2 <- (I - V T V^T)^T W2 = W2 - V T^T (V^T W2), in three column ranges:
            //   next panel (main stream, before it is factored);
            //   the panel after it (side stream, then ev_join marks it done);
            //   everything further right (side stream, may lag behind the panels).
            // Each column range receives the panels' updates in order: the side
            // stream is in order, and the main stream's next-panel update waits for
            // the side stream's update of the same columns by the previous panel.
            const long long nnext = std::min<long long>(nb, N2);
            const long long nsec = std::min<long long>(nb, N2 - nnext);
            const long long nrest = N2 - nnext - nsec;
            if (j0 > 0 && had_second) GN_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
            if (nsec > 0) {
                GN_CUDA_TRY(cudaEventRecord(h->ev_fork, h->stream));   // panel j0 factored
                GN_CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
                gn_handle_s side = *h;
                side.stream = h->side;
                GN_TRY(wy_apply(&side, W2 + nnext, ld, Mp, nsec, Vb, N, jb, T, 1, 1));
                GN_CUDA_TRY(cudaEventRecord(h->ev_join, h->side));
                if (nrest >= 128 && oz) {
                    // W3 <- W3 - V (T^T (V^T W3)) with the two large products digit-sliced
                    double* W3 = W2 + nnext + nsec;
                    GN_TRY(oz_dgemm(&side, jb, nrest, Mp, 1.0, Vb, 0, N, 1, W3, ld, 0, 0.0, q.Z1, nrest, oz,
                                    oz_bytes));
                    GN_TRY(dgemm(&side, jb, nrest, jb, 1.0, T, jb, 1, q.Z1, nrest, 0, 0.0, q.Z2, nrest, q.gws,
                                 q.gws_bytes));
                    GN_TRY(oz_dgemm(&side, Mp, nrest, jb, -1.0, Vb, 0, N, 0, q.Z2, nrest, 0, 1.0, W3, ld, oz,
                                    oz_bytes));
                } else if (nrest > 0) {
                    GN_TRY(wy_apply(&side, W2 + nnext + nsec, ld, Mp, nrest, Vb, N, jb, T, 1, 1));
                }
                side_used = true;
            }
            had_second = nsec > 0;
            GN_TRY(wy_apply(h, W2, ld, Mp, nnext, Vb, N, jb, T, 1, 0));
            GN_TRY(factor_panel(j0 + jb));
            continue;
        }
        const gn_status st = wy_apply(h, W2, ld, Mp, N2, Vb, N, jb, T, 1, 0);
        if (st == GN_ERR_UNSUPPORTED) {
            GN_TRY(dgemm(h, jb, N2, Mp, 1.0, Vb, N, 1, W2, ld, 0, 0.0, q.Z1, N2, q.gws, q.gws_bytes));
            GN_TRY(dgemm(h, jb, N2, jb, 1.0, T, jb, 1, q.Z1, N2, 0, 0.0, q.Z2, N2, q.gws, q.gws_bytes));
            GN_TRY(dgemm(h, Mp, N2, jb, -1.0, Vb, N, 0, q.Z2, N2, 0, 1.0, W2, ld, q.gws, q.gws_bytes));
        } else {
            GN_TRY(st);
        }
        GN_TRY(factor_panel(j0 + jb));
    }
    if (side_used) {   // every lagging update is done before R and the reflectors are used
        GN_CUDA_TRY(cudaEventRecord(h->ev_join, h->side));
        GN_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    }
    qr_write_r_kernel<<<ew_blocks(h, N * N), 256, 0, h->stream>>>(W, ld, static_cast<int>(N), R, ldr); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    if (h != h0) {   // join the high-priority chain back into the caller's stream
        GN_CUDA_TRY(cudaEventRecord(h0->ev_crit1, h->stream));
        GN_CUDA_TRY(cudaStreamWaitEvent(h0->stream, h0->ev_crit1, 0));
    }
    return GN_OK;
}

size_t qr_oz_ws_bytes(long long M, long long N) {
    // the Q formation's buffers, or the blocked factorization's, after the side stream's products' scratch
    return qr_oz_side_bytes(M, N) +
           std::max<size_t>(sizeof(double) * (2 * QR_SB * QR_SB + 2 * QR_SB * N) + 2048, qr_blk_bytes(M, N));
}

namespace {

// Q = H_0 ... H_{N-1} [I; 0] in blocks of QR_SB reflectors from the last block:
// Q_s <- Q_s - V_b T_b (V_b^T Q_s), with G_b = V_b^T V_b, V_b^T Q_s, T_b (.) and the
// update on the tensor cores (oz_dgemm, FP64 accuracy); T_b from G_b by
// ut_inverse.
// Z[c][j] = V[j][c] for c, j < nb.  When block b's reflectors are applied to Q
// (from the last block back), Q's columns j0 .. j0 + nb - 1 below row j0 are
// still [I; 0], so that part of V_b^T Q is the transpose of V_b's top nb rows:
// copied, not multiplied.
__global__ void vtop_t_kernel(const double* __restrict__ V, long long ldv, int nb, double* __restrict__ Z,
                              long long ldz) {
    const int total = nb * nb;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int c = e / nb, j = e - c * nb;
        Z[c * ldz + j] = V[j * ldv + c];
    }
}

// Z (nb x Nq, ld Nq) = V_b^T Q_s for the block of reflectors at column j0: the
// first nb columns by the copy above, the rest as a digit-sliced product.
gn_status block_vtq(gn_handle h, const double* Vb, long long ldv, long long Mp, long long nbb, const double* Qs,
                    long long ldq, long long Nq, double* Z, void* oz, size_t oz_bytes) {
    vtop_t_kernel<<<ew_blocks(h, nbb * nbb), 256, 0, h->stream>>>(Vb, ldv, static_cast<int>(nbb), Z, Nq);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    if (Nq > nbb)
        GN_TRY(oz_dgemm(h, nbb, Nq - nbb, Mp, 1.0, Vb, 0, ldv, 1, Qs + nbb, ldq, 0, 0.0, Z + nbb, Nq, oz, oz_bytes));
    return GN_OK;
}

gn_status form_q_tc(gn_handle h, const QrWs& q, long long M, long long N, double* Q, long long ldq, void* oz,
                    size_t oz_bytes) {
    static_assert(QR_BB == QR_SB, "the blocked factorization's T_b serve the Q formation's blocks");
    QrBlk bk;
    if (qr_blocked_path(h, M, N, oz, oz_bytes, &bk)) {
        // the factorization left V zero above each block's diagonal, and T_b and
        // U_b = V_b T_b of every block but the last in bk.TB and bk.UB
        const long long nblk = (N + QR_BB - 1) / QR_BB;
        for (long long bi = nblk - 1; bi >= 0; --bi) {
            const long long j0 = bi * QR_BB;
            const long long nbb = std::min<long long>(QR_BB, N - j0), Mp = M - j0, Nq = N - j0;
            const double* Vb = q.V + j0 * N + j0;
            double* Qs = Q + j0 * ldq + j0;
            double* Tb = bk.TB + bi * QR_BB * QR_BB;
            GN_TRY(block_vtq(h, Vb, N, Mp, nbb, Qs, ldq, Nq, bk.Z1s, bk.oz_side, bk.oz_side_bytes));
            if (bi < nblk - 1) {   // Q_s -= U_b (V_b^T Q_s) with the factorization's U_b = V_b T_b
                GN_TRY(oz_dgemm(h, Mp, Nq, nbb, -1.0, bk.UB + bi * M * QR_BB, 0, QR_BB, 0, bk.Z1s, Nq, 0, 1.0, Qs,
                                ldq, bk.oz_side, bk.oz_side_bytes));
                continue;
            }
            // the last block: its T here, then Q_s -= V_b (T_b (V_b^T Q_s))
            GN_TRY(oz_dgemm(h, nbb, nbb, Mp, 1.0, Vb, 0, N, 1, Vb, N, 0, 0.0, bk.GB, QR_BB, bk.oz_side,
                            bk.oz_side_bytes));
            launch_ut_inverse(h, bk.GB, QR_BB, q.tau + j0, static_cast<int>(nbb), Tb, QR_BB);
            GN_CUDA_TRY(cudaGetLastError());
            GN_TRY(oz_dgemm(h, nbb, Nq, nbb, 1.0, Tb, 0, QR_BB, 0, bk.Z1s, Nq, 0, 0.0, bk.Z2s, Nq, bk.oz_side,
                            bk.oz_side_bytes));
            GN_TRY(oz_dgemm(h, Mp, Nq, nbb, -1.0, Vb, 0, N, 0, bk.Z2s, Nq, 0, 1.0, Qs, ldq, bk.oz_side,
                            bk.oz_side_bytes));
        }
        return GN_OK;
    }
    char* base = static_cast<char*>(oz);
    const size_t g_bytes = (sizeof(double) * QR_SB * QR_SB + 255) & ~static_cast<size_t>(255);
    const size_t w_bytes = (sizeof(double) * QR_SB * N + 255) & ~static_cast<size_t>(255);
    double* G = reinterpret_cast<double*>(base);
    double* Tb = reinterpret_cast<double*>(base + g_bytes);
    double* Wb = reinterpret_cast<double*>(base + 2 * g_bytes);
    double* Wb2 = reinterpret_cast<double*>(base + 2 * g_bytes + w_bytes);
    if (2 * (g_bytes + w_bytes) >= oz_bytes) return GN_ERR_WORKSPACE;
    void* ozw = base + 2 * (g_bytes + w_bytes);
    const size_t ozw_bytes = oz_bytes - 2 * (g_bytes + w_bytes);
    v_zero_upper_kernel<<<ew_blocks(h, N * QR_SB), 256, 0, h->stream>>>(q.V, N, static_cast<int>(N)); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    for (long long j0 = ((N - 1) / QR_SB) * QR_SB; j0 >= 0; j0 -= QR_SB) {
        const long long nbb = std::min<long long>(QR_SB, N - j0), Mp = M - j0, Nq = N - j0;
        const double* Vb = q.V + j0 * N + j0;   // Mp x nbb, ld N (explicit unit diagonal, zeros above)
        double* Qs = Q + j0 * ldq + j0;
        GN_TRY(oz_dgemm(h, nbb, nbb, Mp, 1.0, Vb, 0, N, 1, Vb, N, 0, 0.0, G, QR_SB, ozw, ozw_bytes));
        launch_ut_inverse(h, G, QR_SB, q.tau + j0, static_cast<int>(nbb), Tb, QR_SB);
        GN_CUDA_TRY(cudaGetLastError());
        GN_TRY(block_vtq(h, Vb, N, Mp, nbb, Qs, ldq, Nq, Wb, ozw, ozw_bytes));
        GN_TRY(oz_dgemm(h, nbb, Nq, nbb, 1.0, Tb, 0, QR_SB, 0, Wb, Nq, 0, 0.0, Wb2, Nq, ozw, ozw_bytes));
        GN_TRY(oz_dgemm(h, Mp, Nq, nbb, -1.0, Vb, 0, N, 0, Wb2, Nq, 0, 1.0, Qs, ldq, ozw, ozw_bytes));
    }
    return GN_OK;
}

}  // namespace

gn_status qr_form_q(gn_handle h, const double* W, long long M, long long N, long long ld, double* Q,
                    long long ldq, double* ws, size_t ws_bytes, void* oz, size_t oz_bytes) {
    QrWs q = qr_carve(M, N, ws, ws_bytes);
    if (oz) {
        qr_init_q_kernel<<<ew_blocks(h, M * N), 256, 0, h->stream>>>(Q, ldq, static_cast<int>(M),
                                                                      static_cast<int>(N)); count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        GN_TRY(form_q_tc(h, q, M, N, Q, ldq, oz, oz_bytes));
        qr_flip_q_kernel<<<ew_blocks(h, M * N), 256, 0, h->stream>>>(W, ld, static_cast<int>(M),
                                                                      static_cast<int>(N), Q, ldq); count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        return GN_OK;
    }
    const int nb = panel_cfg(h, M).nb;   // the factorization's panel width
    // Q = H_0 ... H_{N-1} [I; 0], applied block by block from the last panel.
    qr_init_q_kernel<<<ew_blocks(h, M * N), 256, 0, h->stream>>>(Q, ldq, static_cast<int>(M),
                                                                  static_cast<int>(N)); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    for (long long j0 = ((N - 1) / nb) * nb; j0 >= 0; j0 -= nb) {
        const int jb = static_cast<int>(std::min<long long>(nb, N - j0));
        const long long Mp = M - j0;
        const long long Nq = N - j0;
        double* Qs = Q + j0 * ldq + j0;
        const double* Vb = q.V + j0 * N + j0;
        const double* T = q.Tall + (j0 / nb) * QR_NB * QR_NB;
        // Q_s <- (I - V T V^T) Q_s
        const gn_status st = wy_apply(h, Qs, ldq, Mp, Nq, Vb, N, jb, T, 0, 1);
        if (st == GN_ERR_UNSUPPORTED) {
            GN_TRY(dgemm(h, jb, Nq, Mp, 1.0, Vb, N, 1, Qs, ldq, 0, 0.0, q.Z1, Nq, q.gws, q.gws_bytes));
            GN_TRY(dgemm(h, jb, Nq, jb, 1.0, T, jb, 0, q.Z1, Nq, 0, 0.0, q.Z2, Nq, q.gws, q.gws_bytes));
            GN_TRY(dgemm(h, Mp, Nq, jb, -1.0, Vb, N, 0, q.Z2, Nq, 0, 1.0, Qs, ldq, q.gws, q.gws_bytes));
        } else {
            GN_TRY(st);
        }
    }
    qr_flip_q_kernel<<<ew_blocks(h, M * N), 256, 0, h->stream>>>(W, ld, static_cast<int>(M),
                                                                  static_cast<int>(N), Q, ldq); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status householder_qr(gn_handle h, double* W, long long M, long long N, long long ld, double* Q,
                         long long ldq, double* R, long long ldr, double* ws, size_t ws_bytes) {
    GN_TRY(qr_factor(h, W, M, N, ld, R, ldr, ws, ws_bytes));
    return qr_form_q(h, W, M, N, ld, Q, ldq, ws, ws_bytes);
}

size_t trsm_ws_bytes(long long m, long long k, int sm_count) {
    return dgemm_ws_bytes(m, TB, k, sm_count) + 256;
}

gn_status trsm_right_upper(gn_handle h, double* F, long long m, long long k, long long ldf,
                           const double* R, long long ldr, int trans, double* ws, size_t ws_bytes, void* oz,
                           size_t oz_bytes) {
    if (m <= 0 || k <= 0) return GN_OK;
    // Two levels of blocking: 128-column outer blocks take the bulk of the
    // update as one wide FP64 GEMM each; inside, 32-column blocks take a narrow
    // GEMM over the outer block and the per-row triangular solve.
    constexpr long long OB = 128;
    const long long nob = (k + OB - 1) / OB;
    const int blocks = static_cast<int>((m + 127) / 128);
    for (long long obi = 0; obi < nob; ++obi) {
        const long long ob = trans ? nob - 1 - obi : obi;
        const long long J0 = ob * OB, JB = std::min<long long>(OB, k - J0);
        // (oz: these and the inner updates below on the tensor cores by exact digit slicing)
        if (!trans && J0 > 0) {   // F[:, J] -= F[:, 0:J0] R[0:J0, J]
            if (oz)
                GN_TRY(oz_dgemm(h, m, JB, J0, -1.0, F, 0, ldf, 0, R + J0, ldr, 0, 1.0, F + J0, ldf, oz, oz_bytes));
            else
                GN_TRY(dgemm(h, m, JB, J0, -1.0, F, ldf, 0, R + J0, ldr, 0, 1.0, F + J0, ldf, ws, ws_bytes));
        }
        if (trans && J0 + JB < k) {   // F[:, J] -= F[:, J+] R[J, J+]^T
            const long long kk = k - J0 - JB;
            if (oz)
                GN_TRY(oz_dgemm(h, m, JB, kk, -1.0, F + J0 + JB, 0, ldf, 0, R + J0 * ldr + J0 + JB, ldr, 1, 1.0,
                                F + J0, ldf, oz, oz_bytes));
            else
                GN_TRY(dgemm(h, m, JB, kk, -1.0, F + J0 + JB, ldf, 0, R + J0 * ldr + J0 + JB, ldr, 1, 1.0, F + J0,
                             ldf, ws, ws_bytes));
        }
        const long long nb = (JB + TB - 1) / TB;
        for (long long bi = 0; bi < nb; ++bi) {
            const long long b = trans ? nb - 1 - bi : bi;
            const long long j0 = J0 + b * TB;
            const int jb = static_cast<int>(std::min<long long>(TB, J0 + JB - j0));
            if (!trans && j0 > J0) {
                // F[:, j] -= F[:, J0:j0] R[J0:j0, j]
                if (oz)
                    GN_TRY(oz_dgemm(h, m, jb, j0 - J0, -1.0, F + J0, 0, ldf, 0, R + J0 * ldr + j0, ldr, 0, 1.0,
                                    F + j0, ldf, oz, oz_bytes));
                else
                    GN_TRY(dgemm(h, m, jb, j0 - J0, -1.0, F + J0, ldf, 0, R + J0 * ldr + j0, ldr, 0, 1.0, F + j0, ldf,
                                 ws, ws_bytes));
            }
            if (trans && j0 + jb < J0 + JB) {
                // F[:, j] -= F[:, j+ .. J0+JB] R[j, j+ ..]^T
                const long long kk = J0 + JB - j0 - jb;
                if (oz)
                    GN_TRY(oz_dgemm(h, m, jb, kk, -1.0, F + j0 + jb, 0, ldf, 0, R + j0 * ldr + j0 + jb, ldr, 1, 1.0,
                                    F + j0, ldf, oz, oz_bytes));
                else
                    GN_TRY(dgemm(h, m, jb, kk, -1.0, F + j0 + jb, ldf, 0, R + j0 * ldr + j0 + jb, ldr, 1, 1.0, F + j0,
                                 ldf, ws, ws_bytes));
            }
            trsm_diag_kernel<<<blocks, 128, 0, h->stream>>>(F, m, ldf, static_cast<int>(j0), jb, R, ldr, trans); count_launch();
            GN_CUDA_TRY(cudaGetLastError());
        }
    }
    return GN_OK;
}

gn_status core_diagnostics(gn_handle h, const double* R, long long r, long long ldr, double eps,
                           int eps_relative, int want_estimate, int iters, double* out3, int* k_out,
                           double* ws, size_t ws_bytes) {
    static int cd_cs = -1;
    if (cd_cs < 0) {
        cd_cs = 0;
        const size_t smax = cd_smem(CD_MAX_R, 8);
        if (cudaFuncSetAttribute(core_diag_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smax)) == cudaSuccess &&
            cudaFuncSetAttribute(core_diag_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess) {
            for (int cs : {16, 8}) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(cs);
                cfg.blockDim = dim3(CD_THREADS);
                cfg.dynamicSmemBytes = smax;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = cs;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int n = 0;
                if (cudaOccupancyMaxActiveClusters(&n, core_diag_cluster_kernel, &cfg) == cudaSuccess && n >= 1) {
                    cd_cs = cs;
                    break;
                }
            }
        }
        cudaGetLastError();
    }
    if (cd_cs > 0 && r <= CD_MAX_R && r >= 64) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cd_cs);
        cfg.blockDim = dim3(CD_THREADS);
        cfg.dynamicSmemBytes = cd_smem(static_cast<int>(r), cd_cs);
        cfg.stream = h->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cd_cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        GN_CUDA_TRY(cudaLaunchKernelEx(&cfg, core_diag_cluster_kernel, R, ldr, static_cast<int>(r), eps,
                                       eps_relative, want_estimate, iters, out3, k_out));
        count_launch();
        return GN_OK;
    }
    if (ws_bytes < 2 * static_cast<size_t>(r) * sizeof(double)) return GN_ERR_WORKSPACE;
    core_diag_kernel<<<1, DG_THREADS, 0, h->stream>>>(R, ldr, static_cast<int>(r), eps, eps_relative,
                                                      want_estimate, iters, ws, out3, k_out); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status copy_f32_to_f64(gn_handle h, const float* src, long long rows, long long cols, long long lds,
                          double* dst, long long ldd) {
    if (rows * cols == 0) return GN_OK;
    copy_f32_f64_kernel<<<ew_blocks(h, rows * cols), 256, 0, h->stream>>>(src, rows, cols, lds, dst, ldd); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

__global__ void split3_f64_kernel(const double* __restrict__ s, long long rows, long long cols, long long lds,
                                  __nv_bfloat16* hi, __nv_bfloat16* mid, __nv_bfloat16* lo, long long ldd) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e % cols;
        const double x = s[i * lds + j];
        const __nv_bfloat16 h = __double2bfloat16(x);
        const double r1 = x - static_cast<double>(__bfloat162float(h));
        const __nv_bfloat16 m = __double2bfloat16(r1);
        const double r2 = r1 - static_cast<double>(__bfloat162float(m));
        hi[i * ldd + j] = h;
        mid[i * ldd + j] = m;
        lo[i * ldd + j] = __double2bfloat16(r2);
    }
}

gn_status split3_f64_bf16(gn_handle h, const double* src, long long rows, long long cols, long long lds,
                          __nv_bfloat16* hi, __nv_bfloat16* mid, __nv_bfloat16* lo, long long ldd) {
    if (rows * cols == 0) return GN_OK;
    split3_f64_kernel<<<ew_blocks(h, rows * cols), 256, 0, h->stream>>>(src, rows, cols, lds, hi, mid, lo, ldd); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status split3_bf16(gn_handle h, const float* src, long long rows, long long cols, long long lds,
                      __nv_bfloat16* hi, __nv_bfloat16* mid, __nv_bfloat16* lo, long long ldd) {
    if (rows * cols == 0) return GN_OK;
    split3_kernel<<<ew_blocks(h, rows * cols), 256, 0, h->stream>>>(src, rows, cols, lds, hi, mid, lo, ldd); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status sum3_f32_to_f64(gn_handle h, const float* a, const float* b, const float* c, long long rows,
                          long long cols, long long lds, double* dst, long long ldd) {
    if (rows * cols == 0) return GN_OK;
    sum3_kernel<<<ew_blocks(h, rows * cols), 256, 0, h->stream>>>(a, b, c, rows, cols, lds, dst, ldd); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status quantize_bf16(gn_handle h, const void* src, int src_f64, long long rows, long long cols,
                        long long lds, __nv_bfloat16* hi, __nv_bfloat16* lo, long long ldd) {
    if (rows * cols == 0) return GN_OK;
    quantize_kernel<<<ew_blocks(h, rows * cols), 256, 0, h->stream>>>(src, src_f64, rows, cols, lds, hi, lo,
                                                                      ldd); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status transpose_rows_f64(gn_handle h, const double* src, long long rows, long long cols,
                             long long lds, long long keep_rows, double* dst, long long ldd) {
    if (rows * cols == 0) return GN_OK;
    transpose_rows_kernel<<<ew_blocks(h, rows * cols), 256, 0, h->stream>>>(src, rows, cols, lds, keep_rows,
                                                                            dst, ldd); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

size_t error_ws_bytes(long long m, long long n, int) {
    return static_cast<size_t>(((m + GT - 1) / GT) * ((n + GT - 1) / GT)) * sizeof(double) + 256;
}

gn_status error_fro2(gn_handle h, const void* A, int a_dtype, const void* A_lo, long long m, long long n,
                     long long lda, const double* F, long long ldf, const double* G, long long ldg,
                     long long k, double* out, double* ws, size_t ws_bytes) {
    if (ws_bytes < error_ws_bytes(m, n, h->sm_count)) return GN_ERR_WORKSPACE;
    dim3 grid(static_cast<unsigned>((n + GT - 1) / GT), static_cast<unsigned>((m + GT - 1) / GT), 1);
    ErrArgs e{A, A_lo, a_dtype, lda, ws};
    const int kk = static_cast<int>(k);
    dgemm_kernel<GT, GT, double, double, EPI_ERR><<<grid, GTHREADS, 0, h->stream>>>(
        (int)m, (int)n, kk, 1.0, F, ldf, 0, G, ldg, 0, 0.0, nullptr, 0, nullptr, kk > 0 ? kk : 1, e); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    reduce_sum_kernel<<<1, 1024, 0, h->stream>>>(ws, static_cast<long long>(grid.x) * grid.y, out); count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

}  // namespace gn

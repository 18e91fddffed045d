// Section 5.1.1's alternatives to truncating R, and SGN with the SVD-based
// epsilon-pseudoinverse of eq. 2.2, on the GPU:
//
//   SVD_TRUNCATE: C = U S V^T, keep s_i > eps:  F = AX V_k S_k^{-1}, G = U_k^T (Y^T A)
//   SVD_RAISE   : s_i -> max(s_i, eps):         F = AX V S~^{-1},   G = U^T (Y^T A)
//   RRQR_RAISE  : C P = Q R (column pivoting), |R_ii| -> max(|R_ii|, eps), sign kept:
//                 F = (AX P) R~^{-1} (triangular solve), G = Q^T (Y^T A)
//   DIAG_RAISE  : C = Q R (no pivoting), |R_ii| raised the same way: F = AX R~^{-1}
//
// The SVD and pivoted variants factor C in one CTA's shared memory (r <= 128,
// r + l <= 192, the batched path's limits): the pivoted QR by Householder
// reflectors with the column of largest remaining norm moved forward at each
// step; the SVD from it, preconditioned as Drmac and Veselic (2008) do, by
// one-sided (Hestenes) Jacobi rotations of the rows of R in round-robin order
// (C P = Q R, G^T R = T with orthogonal rows, so U = Q G and V = P T^T S^-1),
// run over a thread-block cluster whose CTAs each hold a slice of the columns
// of T and of the accumulated rotations.  DIAG_RAISE
// takes the library's blocked Householder QR for any r.  The products that
// form F and G and the triangular solves are the FP64 routines of gn_f64.cu.
#include "gn_internal.cuh"
#include "gn_smem_core.cuh"

#include <cooperative_groups.h>

#include <string.h>

#include <algorithm>

namespace gn {
namespace {
using namespace smemcore;

constexpr int JACOBI_MAX_SWEEPS = 40;

// C (M x N, global, ld N) -> the core's pivoted QR, C P = Q R.
//   SVD variants: Q to Qg (M x N), R to Rg (N x N); jacobi_cluster_kernel follows.
//   RRQR_RAISE: Q with diag(R) >= 0 to Ul (M x N, ld N), R~ (|R_ii| raised to
//     eps) to Wr (N x N, upper triangular), diag(R) to sv, out[0] = N, out[1] = 0.
//   perm (N): the column order.
__global__ void __launch_bounds__(BT, 1) variant_core_kernel(const double* __restrict__ C, int M, int N, int variant,
                                                          double eps, double* Ul, double* Wr, int* perm, double* sv,
                                                          int* out, double* Qg, double* Rg) {
    extern __shared__ double shm[];
    const int tid = threadIdx.x;
    if (variant != GN_VARIANT_RRQR_RAISE) {
        // SVD variants, preconditioned (Drmac and Veselic): C P = Q R by the
        // pivoted QR, R to Rg and the explicit Q to Qg; the Jacobi below then
        // runs on the rows of R (N x N), which the pivoting leaves nearly
        // orthogonal, instead of on the columns of C.
        Smem sm;
        sm.ld = N + 1;
        sm.S = shm;
        sm.red = sm.S + static_cast<size_t>(MMAX) * (NMAX + 1);
        sm.tau = sm.red + BW * NMAX;
        sm.dsum = sm.tau + NMAX;
        sm.wv = sm.dsum + NMAX;
        sm.scal = sm.wv + NMAX;
        const int ld = sm.ld;
        for (int e = tid; e < M * N; e += BT) sm.S[(e / N) * ld + e % N] = C[e];
        for (int j = tid; j < N; j += BT) perm[j] = j;
        __syncthreads();
        smem_qr(sm, M, N, perm);
        for (int e = tid; e < N * N; e += BT) {
            const int i = e / N, j = e - i * N;
            Rg[e] = j >= i ? sm.S[i * ld + j] : 0.0;
        }
        __syncthreads();
        smem_form_q(sm, M, N);
        for (int e = tid; e < M * N; e += BT) Qg[e] = sm.S[(e / N) * ld + e % N];
    } else {
        Smem sm;
        sm.ld = N + 1;
        sm.S = shm;
        sm.red = sm.S + static_cast<size_t>(MMAX) * (NMAX + 1);
        sm.tau = sm.red + BW * NMAX;
        sm.dsum = sm.tau + NMAX;
        sm.wv = sm.dsum + NMAX;
        sm.scal = sm.wv + NMAX;
        double* sgnv = sm.scal + 8;
        const int ld = sm.ld;
        for (int e = tid; e < M * N; e += BT) sm.S[(e / N) * ld + e % N] = C[e];
        for (int j = tid; j < N; j += BT) perm[j] = j;
        __syncthreads();
        smem_qr(sm, M, N, perm);
        // diag(R) >= 0 (rows flipped, Q's columns below), then |R_ii| raised to eps
        for (int i = tid; i < N; i += BT) sgnv[i] = sm.S[i * ld + i] < 0.0 ? -1.0 : 1.0;
        __syncthreads();
        for (int e = tid; e < N * N; e += BT) {
            const int i = e / N, j = e - i * N;
            double v = j >= i ? sgnv[i] * sm.S[i * ld + j] : 0.0;
            if (i == j) {
                sv[i] = v;
                v = fmax(v, eps);
            }
            Wr[e] = v;
        }
        __syncthreads();
        smem_form_q(sm, M, N);
        for (int e = tid; e < M * N; e += BT) {
            const int i = e / N, j = e - i * N;
            Ul[e] = sgnv[j] * sm.S[i * ld + j];
        }
        if (tid == 0) {
            out[0] = N;
            out[1] = 0;
        }
    }
}

// ---- one-sided Jacobi on the rows of T = R (N x N) over a cluster: CTA c holds
// columns [c w, c w + w) of T and of G^T (the accumulated rotations), w =
// ceil(N / JC_CS).  A round's pairs are disjoint: every CTA forms the pairs'
// partial dot products over its columns, the partials go through distributed
// shared memory (double-buffered by round parity, one cluster barrier per
// round), every CTA adds them in rank order (so all CTAs take the same
// decisions and run the same number of barriers) and rotates its own columns.
constexpr int JC_CS = 8;                    // CTAs per cluster
constexpr int JC_T = 256;                   // threads per CTA
constexpr int JC_W = NMAX / JC_CS;          // columns per CTA (at most)
constexpr int JC_PAIRS = NMAX / 2;          // pairs per round (at most)
constexpr int JC_G = JC_T / JC_PAIRS;       // threads per pair

struct JcSmem {
    double T[NMAX][JC_W + 1];
    double V[NMAX][JC_W + 1];
    double part[2][JC_PAIRS][4];   // alpha, beta, gamma of every pair, by round parity
    double normp[NMAX];            // partial squared row norms (after the sweeps)
    double s[NMAX];
    int rank[NMAX];
    int k;
};

// Rg (N x N): R on entry, G with columns by decreasing s on exit (U = Q Rg,
// formed by the caller); Wr (N x N): V S~^{-1}, rows permuted back by perm;
// sv: s in decreasing order; out[0] = k, out[1] = sweeps.
__global__ void __cluster_dims__(JC_CS, 1, 1) __launch_bounds__(JC_T)
    jacobi_cluster_kernel(int N, int variant, double eps, double* Rg, double* Wr, const int* __restrict__ perm,
                          double* sv, int* out) {
    namespace cg = cooperative_groups;
    __shared__ JcSmem sm;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = static_cast<int>(cluster.block_rank());
    const int tid = threadIdx.x;
    const int wc = (N + JC_CS - 1) / JC_CS;
    const int c0 = rank * wc, ncol = max(0, min(N, c0 + wc) - c0);   // this CTA's columns
    for (int e = tid; e < N * wc; e += JC_T) {
        const int j = e / wc, i = e - j * wc;
        sm.T[j][i] = i < ncol ? Rg[j * N + c0 + i] : 0.0;
        sm.V[j][i] = i < ncol && j == c0 + i ? 1.0 : 0.0;
    }
    __syncthreads();
    const int n2 = (N + 1) & ~1;
    const int npairs = n2 / 2;
    const int pair = tid / JC_G, gl = tid % JC_G;
    const double tol = 2.0 * static_cast<double>(N) * 1.1102230246251565e-16;
    int sweeps = 0, parity = 0;
    for (; sweeps < JACOBI_MAX_SWEEPS; ++sweeps) {
        int rotated = 0;
        for (int round = 0; round < n2 - 1; ++round, parity ^= 1) {
            int p = 0, q = N;   // q = N: no pair, or the dummy player
            if (pair < npairs) {
                const int a = (round + pair) % (n2 - 1);
                const int b = pair == 0 ? n2 - 1 : (round - pair + n2 - 1) % (n2 - 1);
                p = min(a, b);
                q = max(a, b);
            }
            const bool act = q < N;
            double al = 0.0, be = 0.0, ga = 0.0;
            if (act)
                for (int i = gl; i < ncol; i += JC_G) {
                    const double tp = sm.T[p][i], tq = sm.T[q][i];
                    al = fma(tp, tp, al);
                    be = fma(tq, tq, be);
                    ga = fma(tp, tq, ga);
                }
#pragma unroll
            for (int o = 1; o < JC_G; o <<= 1) {   // the pair's JC_G lanes are adjacent in one warp
                al += __shfl_xor_sync(0xffffffffu, al, o);
                be += __shfl_xor_sync(0xffffffffu, be, o);
                ga += __shfl_xor_sync(0xffffffffu, ga, o);
            }
            if (gl == 0 && pair < JC_PAIRS) {
                sm.part[parity][pair][0] = al;
                sm.part[parity][pair][1] = be;
                sm.part[parity][pair][2] = ga;
            }
            cluster.sync();   // every CTA's partials of this round written
            if (act) {
                al = be = ga = 0.0;
                for (int c = 0; c < JC_CS; ++c) {   // rank order: the same sums in every CTA
                    const double* pc = cluster.map_shared_rank(&sm.part[parity][pair][0], c);
                    al += pc[0];
                    be += pc[1];
                    ga += pc[2];
                }
                if (fabs(ga) > tol * sqrt(al * be) && ga != 0.0) {
                    const double zeta = (be - al) / (2.0 * ga);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                    for (int i = gl; i < ncol; i += JC_G) {
                        const double tp = sm.T[p][i], tq = sm.T[q][i];
                        sm.T[p][i] = cs * tp - sn * tq;
                        sm.T[q][i] = sn * tp + cs * tq;
                        const double vp = sm.V[p][i], vq = sm.V[q][i];
                        sm.V[p][i] = cs * vp - sn * vq;
                        sm.V[q][i] = sn * vp + cs * vq;
                    }
                    rotated = 1;
                }
            }
            __syncthreads();   // the round's rotations in place before the next round's partials
        }
        // the same decisions in every CTA: the same answer here, the same number of barriers
        if (!__syncthreads_or(rotated)) break;
    }
    // singular values = row norms of T (partials over the CTAs' columns, added in rank order)
    for (int j = tid; j < N; j += JC_T) {
        double a = 0.0;
        for (int i = 0; i < ncol; ++i) a = fma(sm.T[j][i], sm.T[j][i], a);
        sm.normp[j] = a;
    }
    cluster.sync();
    for (int j = tid; j < N; j += JC_T) {
        double a = 0.0;
        for (int c = 0; c < JC_CS; ++c) a += cluster.map_shared_rank(sm.normp, c)[j];
        sm.s[j] = sqrt(a);
    }
    __syncthreads();
    for (int j = tid; j < N; j += JC_T) {
        int rk = 0;
        const double sj = sm.s[j];
        for (int i = 0; i < N; ++i) rk += (sm.s[i] > sj || (sm.s[i] == sj && i < j)) ? 1 : 0;
        sm.rank[j] = rk;
        if (rank == 0) sv[rk] = sj;
    }
    if (tid == 0) {
        int k = 0;
        if (variant == GN_VARIANT_SVD_TRUNCATE) {
            for (int j = 0; j < N; ++j) k += sm.s[j] > eps ? 1 : 0;
        } else {
            k = N;
        }
        sm.k = k;
        if (rank == 0) {
            out[0] = k;
            out[1] = sweeps;
        }
    }
    __syncthreads();
    // R = G T with T_j = s_j W_j (W orthonormal rows), so C P = (Q G) diag(s) W:
    //   U = Q G: Rg[i][rank_j] = G[i][j] = V[j][i] (this CTA's rows i of G);
    //   V = P W^T: V[perm[i]][rank_j] = T[j][i] / s_j, stored as Wr = V S~^{-1}.
    const int k = sm.k;
    for (int e = tid; e < N * ncol; e += JC_T) {
        const int j = e / ncol, i = e - j * ncol;
        const int gi = c0 + i, pos = sm.rank[j];
        Rg[gi * N + pos] = sm.V[j][i];
        const double sj = sm.s[j];
        double w;
        if (variant == GN_VARIANT_SVD_TRUNCATE) w = pos < k && sj > 0.0 ? sm.T[j][i] / (sj * sj) : 0.0;
        else w = sj > 0.0 ? sm.T[j][i] / (sj * fmax(sj, eps)) : 0.0;
        Wr[perm[gi] * N + pos] = w;
    }
    cluster.sync();   // peers' reads of normp done before any CTA exits
}

size_t variant_smem_bytes() {
    return sizeof(double) * (static_cast<size_t>(MMAX) * (NMAX + 1) + BW * NMAX + 3 * NMAX + 8 + 2 * NMAX);
}

// |R_ii| -> max(|R_ii|, eps) with the sign kept (sign(0) = +1); sv_i = R_ii before.
__global__ void raise_diag_kernel(double* R, long long r, long long ldr, double eps, double* sv) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < r;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double d = R[i * ldr + i];
        if (sv) sv[i] = d;
        R[i * ldr + i] = (d < 0.0 ? -1.0 : 1.0) * fmax(fabs(d), eps);
    }
}

// F[:, j] = AX[:, perm[j]] (FP64 or FP32 AX) into FP64
template <typename T>
__global__ void gather_cols_kernel(const T* __restrict__ AX, long long m, long long r, long long ldx,
                                   const int* __restrict__ perm, double* F, long long ldf) {
    const long long total = m * r;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / r, j = e - i * r;
        const int c = perm ? perm[j] : static_cast<int>(j);
        F[i * ldf + j] = static_cast<double>(AX[i * ldx + c]);
    }
}

__global__ void bf16_f64_kernel(const __nv_bfloat16* __restrict__ s, long long rows, long long cols, long long lds,
                                double* d) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        d[e] = static_cast<double>(__bfloat162float(s[(e / cols) * lds + e % cols]));
}

int grid_for(gn_handle h, long long work) {
    return static_cast<int>(std::max<long long>(1, std::min<long long>((work + 255) / 256, 16LL * h->sm_count)));
}

size_t al256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

struct VarWs {
    double *C, *X64, *Ul, *Wr, *VT, *Q, *R, *Wq;
    int* perm;
    int* out;
    double* inner;
    size_t inner_bytes;
};

size_t var_carve(long long m, long long n, long long r, long long l, int sms, char* base, VarWs* w) {
    const long long rl = r + l;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* q = base ? base + off : nullptr;
        off += al256(bytes);
        return q;
    };
    VarWs v;
    v.C = reinterpret_cast<double*>(take(8 * rl * r));
    v.X64 = reinterpret_cast<double*>(take(8 * n * r));
    v.Ul = reinterpret_cast<double*>(take(8 * rl * r));
    v.Wr = reinterpret_cast<double*>(take(8 * r * r));
    v.VT = reinterpret_cast<double*>(take(8 * r * r));
    v.Q = reinterpret_cast<double*>(take(8 * rl * r));
    v.R = reinterpret_cast<double*>(take(8 * r * r));
    v.Wq = reinterpret_cast<double*>(take(8 * rl * r));
    v.perm = reinterpret_cast<int*>(take(4 * r));
    v.out = reinterpret_cast<int*>(take(64));
    v.inner_bytes = std::max({qr_ws_bytes(rl, r, sms), trsm_ws_bytes(m, r, sms), dgemm_ws_bytes(rl, r, n, sms),
                              dgemm_ws_bytes(m, r, r, sms), dgemm_ws_bytes(r, n, rl, sms)});
    v.inner = reinterpret_cast<double*>(take(v.inner_bytes));
    if (w) *w = v;
    return off + 256;
}

}  // namespace
}  // namespace gn

using namespace gn;

extern "C" gn_status gn_variant_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l, size_t* bytes) {
    if (!bytes) return GN_ERR_INVALID_ARG;
    if (m < 1 || n < 1 || r < 1 || l < 1 || r > std::min(m, n) || r + l > m) return GN_ERR_SHAPE;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *bytes = var_carve(m, n, r, l, sms, nullptr, nullptr);
    return GN_OK;
}

extern "C" gn_status gn_factors_variant(gn_handle h, const gn_mat* AX, const gn_mat* YtA, const gn_mat* X, double eps,
                                        int32_t variant, gn_mat* F, gn_mat* G, int64_t* k_out, double* sv, void* ws,
                                        size_t ws_bytes) {
    if (!h || !AX || !YtA || !X || !F || !G || !k_out || !ws) return GN_ERR_INVALID_ARG;
    if (!AX->data || !YtA->data || !X->data || !F->data || !G->data) return GN_ERR_INVALID_ARG;
    if (variant < GN_VARIANT_SVD_TRUNCATE || variant > GN_VARIANT_DIAG_RAISE || !(eps >= 0.0)) return GN_ERR_INVALID_ARG;
    if ((variant == GN_VARIANT_SVD_RAISE || variant == GN_VARIANT_RRQR_RAISE || variant == GN_VARIANT_DIAG_RAISE) &&
        !(eps > 0.0))
        return GN_ERR_INVALID_ARG;   // the raised floor must be positive
    const long long m = AX->rows, r = AX->cols, rl = YtA->rows, n = YtA->cols, l = rl - r;
    if (r < 1 || l < 1 || X->rows != n || X->cols != r || r > std::min(m, n) || rl > m) return GN_ERR_SHAPE;
    if (AX->ld < r || YtA->ld < n || X->ld < r) return GN_ERR_SHAPE;
    if (F->rows != m || F->cols < r || G->rows < r || G->cols != n || F->ld < F->cols || G->ld < n) return GN_ERR_SHAPE;
    if ((AX->dtype != GN_F64 && AX->dtype != GN_F32) || AX->dtype != YtA->dtype) return GN_ERR_DTYPE;
    if (X->dtype != GN_F64 && X->dtype != GN_BF16) return GN_ERR_DTYPE;
    if (F->dtype != GN_F64 || G->dtype != GN_F64) return GN_ERR_DTYPE;
    const bool small = r <= NMAX && rl <= MMAX;
    if (variant != GN_VARIANT_DIAG_RAISE && !small) return GN_ERR_UNSUPPORTED;
    VarWs v;
    if (var_carve(m, n, r, l, h->sm_count, static_cast<char*>(ws), &v) > ws_bytes) return GN_ERR_WORKSPACE;
    const bool f32 = AX->dtype == GN_F32;
    // X in FP64 (a BF16 sketch is exact in FP64)
    const double* X64 = static_cast<const double*>(X->data);
    long long ldx = X->ld;
    if (X->dtype == GN_BF16) {
        bf16_f64_kernel<<<grid_for(h, n * r), 256, 0, h->stream>>>(static_cast<const __nv_bfloat16*>(X->data), n, r,
                                                                   X->ld, v.X64);
        count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        X64 = v.X64;
        ldx = r;
    }
    // C = (Y^T A) X in FP64
    if (f32)
        GN_TRY(dgemm_a32(h, rl, r, n, 1.0, static_cast<const float*>(YtA->data), YtA->ld, 0, X64, ldx, 0, 0.0, v.C, r,
                         v.inner, v.inner_bytes));
    else
        GN_TRY(dgemm(h, rl, r, n, 1.0, static_cast<const double*>(YtA->data), YtA->ld, 0, X64, ldx, 0, 0.0, v.C, r,
                     v.inner, v.inner_bytes));
    double* Fd = static_cast<double*>(F->data);
    double* Gd = static_cast<double*>(G->data);
    long long k = r;
    const double* Left = nullptr;   // (r+l) x r, ld r: U or Q
    if (variant == GN_VARIANT_DIAG_RAISE) {
        GN_CUDA_TRY(cudaMemcpyAsync(v.Wq, v.C, sizeof(double) * rl * r, cudaMemcpyDeviceToDevice, h->stream));
        GN_TRY(householder_qr(h, v.Wq, rl, r, r, v.Q, r, v.R, r, v.inner, v.inner_bytes));
        raise_diag_kernel<<<grid_for(h, r), 256, 0, h->stream>>>(v.R, r, r, eps, sv);
        count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        Left = v.Q;
    } else {
        static bool attr = false;
        if (!attr) {
            GN_CUDA_TRY(cudaFuncSetAttribute(variant_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(variant_smem_bytes())));
            attr = true;
        }
        double* svd = sv ? sv : v.VT;   // sv optional: any N doubles of scratch otherwise
        variant_core_kernel<<<1, BT, variant_smem_bytes(), h->stream>>>(
            v.C, static_cast<int>(rl), static_cast<int>(r), variant, eps, v.Ul, v.Wr, v.perm, svd, v.out, v.Q, v.R);
        count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        if (variant != GN_VARIANT_RRQR_RAISE) {
            // Jacobi on the rows of R over one cluster; G (columns by rank) left in v.R, then U = Q G
            jacobi_cluster_kernel<<<JC_CS, JC_T, 0, h->stream>>>(static_cast<int>(r), variant, eps, v.R, v.Wr, v.perm,
                                                                 svd, v.out);
            count_launch();
            GN_CUDA_TRY(cudaGetLastError());
            GN_TRY(dgemm(h, rl, r, r, 1.0, v.Q, r, 0, v.R, r, 0, 0.0, v.Ul, r, v.inner, v.inner_bytes));
        }
        int out_h[2] = {0, 0};
        GN_CUDA_TRY(cudaMemcpyAsync(out_h, v.out, sizeof(out_h), cudaMemcpyDeviceToHost, h->stream));
        GN_CUDA_TRY(cudaStreamSynchronize(h->stream));
        k = out_h[0];
        Left = v.Ul;
    }
    *k_out = k;
    if (k < 1) return GN_ERR_NONFINITE;   // nothing of the core is above eps
    // F (m x k)
    if (variant == GN_VARIANT_SVD_TRUNCATE || variant == GN_VARIANT_SVD_RAISE) {
        if (f32)
            GN_TRY(dgemm_a32(h, m, k, r, 1.0, static_cast<const float*>(AX->data), AX->ld, 0, v.Wr, r, 0, 0.0, Fd,
                             F->ld, v.inner, v.inner_bytes));
        else
            GN_TRY(dgemm(h, m, k, r, 1.0, static_cast<const double*>(AX->data), AX->ld, 0, v.Wr, r, 0, 0.0, Fd, F->ld,
                         v.inner, v.inner_bytes));
    } else {
        const int* perm = variant == GN_VARIANT_RRQR_RAISE ? v.perm : nullptr;
        const double* Rt = variant == GN_VARIANT_RRQR_RAISE ? v.Wr : v.R;
        if (f32)
            gather_cols_kernel<float><<<grid_for(h, m * r), 256, 0, h->stream>>>(
                static_cast<const float*>(AX->data), m, r, AX->ld, perm, Fd, F->ld);
        else
            gather_cols_kernel<double><<<grid_for(h, m * r), 256, 0, h->stream>>>(
                static_cast<const double*>(AX->data), m, r, AX->ld, perm, Fd, F->ld);
        count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        GN_TRY(trsm_right_upper(h, Fd, m, r, F->ld, Rt, r, 0, v.inner, v.inner_bytes));
    }
    // G = Left_k^T (Y^T A)   (k x n)
    if (f32)
        GN_TRY(dgemm_b32(h, k, n, rl, 1.0, Left, r, 1, static_cast<const float*>(YtA->data), YtA->ld, 0, 0.0, Gd, G->ld,
                         v.inner, v.inner_bytes));
    else
        GN_TRY(dgemm(h, k, n, rl, 1.0, Left, r, 1, static_cast<const double*>(YtA->data), YtA->ld, 0, 0.0, Gd, G->ld,
                     v.inner, v.inner_bytes));
    return GN_OK;
}

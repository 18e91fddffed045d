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
// with the rotations accumulated in global memory.  DIAG_RAISE
// takes the library's blocked Householder QR for any r.  The products that
// form F and G and the triangular solves are the FP64 routines of gn_f64.cu.
#include "gn_internal.cuh"
#include "gn_smem_core.cuh"

#include <string.h>

#include <algorithm>

namespace gn {
namespace {
using namespace smemcore;

constexpr int JACOBI_MAX_SWEEPS = 40;

__device__ inline double group_sum(double v, int g) {
    for (int o = g >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// C (M x N, global, ld N) -> one of the small-core factorizations.
//   Ul (M x N, ld N): Q (RRQR); unused by the SVD variants
//   Wr (N x N, ld N): V S~^{-1} (SVD variants, columns by decreasing s) or R~ (RRQR, upper triangular)
//   VT (N x N, ld N): scratch for the rotations G^T
//   Qg (M x N), Rg (N x N): SVD variants: the pivoted QR's Q and R; Rg then
//     receives G with columns by decreasing s (U = Qg Rg, formed by the caller)
//   perm (N): RRQR column order; sv (N): s (SVD) or diag(R) after pivoting
//   out[0] = k, out[1] = Jacobi sweeps
__global__ void __launch_bounds__(BT) variant_core_kernel(const double* __restrict__ C, int M, int N, int variant,
                                                          double eps, double* Ul, double* Wr, double* VT, int* perm,
                                                          double* sv, int* out, double* Qg, double* Rg) {
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
        __syncthreads();   // R and Q written (block-wide visibility) before shared memory is reused
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
        return;
    }

    // ---- one-sided Jacobi on the rows of T = R (N x N, ld N + 1): plane
    // rotations of row pairs in round-robin order until every pair is
    // orthogonal to tol; G^T (the product of the rotations) accumulates in VT.
    const int MJ = N;                       // row length
    const int ldt = MJ + 1;
    double* T = shm;
    double* s_norm = T + static_cast<size_t>(N) * ldt;   // [NMAX]
    int* s_rank = reinterpret_cast<int*>(s_norm + NMAX);  // [NMAX]
    __shared__ int s_rot;
    for (int e = tid; e < N * N; e += BT) {
        const int j = e / N, i = e - j * N;
        T[j * ldt + i] = Rg[e];
    }
    for (int e = tid; e < N * N; e += BT) VT[e] = (e / N == e % N) ? 1.0 : 0.0;
    __syncthreads();
    const int n2 = (N + 1) & ~1;          // even player count (a dummy when N is odd)
    const int npairs = n2 / 2;
    int g = 32;
    while (g > 1 && g * npairs > BT) g >>= 1;   // threads per pair (a power of two <= 32)
    const int pair = tid / g, gl = tid % g;
    const double tol = 2.0 * static_cast<double>(MJ) * 1.1102230246251565e-16;
    int sweeps = 0;
    for (; sweeps < JACOBI_MAX_SWEEPS; ++sweeps) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        int rotated = 0;
        for (int round = 0; round < n2 - 1; ++round) {
            int p = 0, q = N;   // q = N: an idle group (no pair, or the dummy player)
            if (pair < npairs) {
                const int a = (round + pair) % (n2 - 1);
                const int b = pair == 0 ? n2 - 1 : (round - pair + n2 - 1) % (n2 - 1);
                p = min(a, b);
                q = max(a, b);
            }
            const bool act = q < N;
            double al = 0.0, be = 0.0, ga = 0.0;
            if (act)
                for (int i = gl; i < MJ; i += g) {
                    const double tp = T[p * ldt + i], tq = T[q * ldt + i];
                    al = fma(tp, tp, al);
                    be = fma(tq, tq, be);
                    ga = fma(tp, tq, ga);
                }
            // every lane of every warp takes part in the shuffles
            al = group_sum(al, g);
            be = group_sum(be, g);
            ga = group_sum(ga, g);
            if (act && fabs(ga) > tol * sqrt(al * be) && ga != 0.0) {
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = gl; i < MJ; i += g) {
                    const double tp = T[p * ldt + i], tq = T[q * ldt + i];
                    T[p * ldt + i] = c * tp - s * tq;
                    T[q * ldt + i] = s * tp + c * tq;
                }
                for (int i = gl; i < N; i += g) {
                    const double vp = VT[p * N + i], vq = VT[q * N + i];
                    VT[p * N + i] = c * vp - s * vq;
                    VT[q * N + i] = s * vp + c * vq;
                }
                rotated = 1;
            }
            __syncthreads();
        }
        if (rotated) s_rot = 1;
        __syncthreads();
        if (!s_rot) break;
        __syncthreads();
    }
    // singular values = row norms of T; ranks by decreasing value (index order on ties)
    for (int j = tid / 32; j < N; j += BW) {
        double a = 0.0;
        for (int i = tid % 32; i < MJ; i += 32) a = fma(T[j * ldt + i], T[j * ldt + i], a);
        a = group_sum(a, 32);
        if (tid % 32 == 0) s_norm[j] = sqrt(a);
    }
    __syncthreads();
    for (int j = tid; j < N; j += BT) {
        int rk = 0;
        const double sj = s_norm[j];
        for (int i = 0; i < N; ++i) rk += (s_norm[i] > sj || (s_norm[i] == sj && i < j)) ? 1 : 0;
        s_rank[j] = rk;
        sv[rk] = sj;
    }
    __syncthreads();
    __shared__ int s_k;
    if (tid == 0) {
        int k = 0;
        if (variant == GN_VARIANT_SVD_TRUNCATE) {
            for (int j = 0; j < N; ++j) k += s_norm[j] > eps ? 1 : 0;
        } else {
            k = N;
        }
        s_k = k;
        out[0] = k;
        out[1] = sweeps;
    }
    __syncthreads();
    const int k = s_k;
    // R = G T with T_j = s_j W_j (W orthonormal rows), so C P = (Q G) diag(s) W:
    //   U = Q G, column rank_j = Q G_j  (G_j = row j of VT): Rg[:, rank_j] = VT[j, :]^T,
    //     multiplied by Q outside the kernel;
    //   V = P W^T: V[perm[i]][rank_j] = T[j][i] / s_j, stored as Wr = V S~^{-1}.
    for (int e = tid; e < N * N; e += BT) {
        const int j = e / N, i = e - j * N;   // Rg[i][rank_j] = G[i][j] = VT[j][i]
        Rg[i * N + s_rank[j]] = VT[e];
    }
    for (int e = tid; e < N * N; e += BT) {
        const int j = e / N, i = e - j * N;
        const double sj = s_norm[j];
        const int pos = s_rank[j];
        double w;
        if (variant == GN_VARIANT_SVD_TRUNCATE) w = pos < k && sj > 0.0 ? T[j * ldt + i] / (sj * sj) : 0.0;
        else w = sj > 0.0 ? T[j * ldt + i] / (sj * fmax(sj, eps)) : 0.0;
        Wr[perm[i] * N + pos] = w;
    }
    (void)Ul;
}

size_t variant_smem_bytes() {
    const size_t qr = sizeof(double) * (static_cast<size_t>(MMAX) * (NMAX + 1) + BW * NMAX + 3 * NMAX + 8 + 2 * NMAX);
    const size_t jac = sizeof(double) * (static_cast<size_t>(NMAX) * (MMAX + 1) + NMAX) + sizeof(int) * NMAX;
    return std::max(qr, jac);
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
        double* vt = sv ? v.VT : v.Wq;
        variant_core_kernel<<<1, BT, variant_smem_bytes(), h->stream>>>(
            v.C, static_cast<int>(rl), static_cast<int>(r), variant, eps, v.Ul, v.Wr, vt, v.perm, svd, v.out, v.Q,
            v.R);
        count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        if (variant != GN_VARIANT_RRQR_RAISE)   // U = Q G (the kernel left G, columns by rank, in v.R)
            GN_TRY(dgemm(h, rl, r, r, 1.0, v.Q, r, 0, v.R, r, 0, 0.0, v.Ul, r, v.inner, v.inner_bytes));
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

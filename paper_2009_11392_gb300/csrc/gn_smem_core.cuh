// Shared-memory Householder routines for one core per CTA (512 threads): the
// batched path's per-problem core and the single-core variants of Section
// 5.1.1.  A core of up to MMAX x NMAX doubles lives in shared memory (ld N + 1).
#pragma once

#include "gn_internal.cuh"

namespace gn {
namespace smemcore {

constexpr int BT = 512;          // threads of a core CTA
constexpr int BW = BT / 32;
constexpr int NMAX = 128;        // widest core handled in shared memory
constexpr int MMAX = 192;        // (r + l) <= 192 rows

// S is M x N in shared memory (ld = N + 1).
//    Partial sums are formed per (row chunk, column) and combined once: on GB300
//    a warp's FP64 instruction occupies its sub-partition's FP64 unit for ~64
//    cycles whatever its mask, so work is spread over all 16 warps rather than
//    reduced by butterflies.
struct Smem {
    double* S;
    int ld;
    double* red;    // [BW][NMAX]
    double* tau;    // [NMAX]
    double* dsum;   // [NMAX]
    double* wv;     // [NMAX]
    double* scal;   // [4]
};

// Householder QR in place: R on and above the diagonal, v below (v_j = 1 implicit),
// tau[j]; the diagonal holds beta_j (sign not normalised).
// perm (optional): column pivoting -- before column j, the column of largest
// remaining norm (rows j..M-1; the first on ties) is swapped into place and
// perm records the original column of every position (perm[j] = j on entry).
__device__ inline void smem_qr(const Smem& sm, int M, int N, int* perm = nullptr) {
    double* S = sm.S;
    const int ld = sm.ld;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int j = 0; j < N; ++j) {
        if (perm) {
            // squared norms of the trailing columns over rows j..M-1
            for (int q0 = j; q0 < N; q0 += 32) {
                const int q = q0 + lane;
                double a0 = 0.0, a1 = 0.0;
                if (q < N) {
                    int i = j + warp;
                    for (; i + BW < M; i += 2 * BW) {
                        a0 = fma(S[i * ld + q], S[i * ld + q], a0);
                        a1 = fma(S[(i + BW) * ld + q], S[(i + BW) * ld + q], a1);
                    }
                    if (i < M) a0 = fma(S[i * ld + q], S[i * ld + q], a0);
                    sm.red[warp * NMAX + (q - j)] = a0 + a1;
                }
            }
            __syncthreads();
            if (tid < N - j) {
                double s0 = 0.0, s1 = 0.0;
                for (int w = 0; w < BW; w += 2) {
                    s0 += sm.red[w * NMAX + tid];
                    s1 += sm.red[(w + 1) * NMAX + tid];
                }
                sm.dsum[tid] = s0 + s1;
            }
            __syncthreads();
            __shared__ int s_piv;
            if (tid == 0) {
                int p = 0;
                double best = sm.dsum[0];
                for (int q = 1; q < N - j; ++q)
                    if (sm.dsum[q] > best) {
                        best = sm.dsum[q];
                        p = q;
                    }
                s_piv = j + p;
                if (p != 0) {
                    const int t = perm[j];
                    perm[j] = perm[j + p];
                    perm[j + p] = t;
                }
            }
            __syncthreads();
            const int pv = s_piv;
            if (pv != j)
                for (int i = tid; i < M; i += BT) {
                    const double t = S[i * ld + j];
                    S[i * ld + j] = S[i * ld + pv];
                    S[i * ld + pv] = t;
                }
            __syncthreads();
        }
        for (int q0 = j; q0 < N; q0 += 32) {
            const int q = q0 + lane;
            // two partial sums: the loads of one overlap the other's FMA (~64 cycles)
            double a0 = 0.0, a1 = 0.0;
            if (q < N) {
                const int q2 = q == j ? j : q;
                int i = (q == j ? j + 1 : j) + warp;
                for (; i + BW < M; i += 2 * BW) {
                    a0 = fma(S[i * ld + j], S[i * ld + q2], a0);
                    a1 = fma(S[(i + BW) * ld + j], S[(i + BW) * ld + q2], a1);
                }
                if (i < M) a0 = fma(S[i * ld + j], S[i * ld + q2], a0);
            }
            if (q < N) sm.red[warp * NMAX + (q - j)] = a0 + a1;
        }
        __syncthreads();
        if (tid < N - j) {
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int w = 0; w < BW; w += 2) {
                s0 += sm.red[w * NMAX + tid];
                s1 += sm.red[(w + 1) * NMAX + tid];
            }
            const double s = s0 + s1;
            if (tid == 0) {
                const double alpha = S[j * ld + j];
                if (s == 0.0) {
                    sm.scal[0] = 0.0;
                    sm.scal[1] = alpha;
                    sm.scal[2] = 0.0;
                } else {
                    const double nx = sqrt(fma(alpha, alpha, s));
                    const double beta = alpha >= 0.0 ? -nx : nx;
                    sm.scal[0] = (beta - alpha) / beta;
                    sm.scal[1] = beta;
                    sm.scal[2] = 1.0 / (alpha - beta);
                }
            } else {
                sm.dsum[tid] = s;
            }
        }
        __syncthreads();
        const double t = sm.scal[0], beta = sm.scal[1], sc = sm.scal[2];
        if (t != 0.0) {
            for (int i = j + 1 + tid; i < M; i += BT) S[i * ld + j] *= sc;
            if (tid > 0 && tid < N - j) sm.wv[tid] = fma(-beta, S[j * ld + j + tid], sm.dsum[tid]) * sc;
            __syncthreads();
            for (int q0 = j + 1; q0 < N; q0 += 32) {
                const int q = q0 + lane;
                if (q < N) {
                    const double wq = t * sm.wv[q - j];
                    for (int i = j + warp; i < M; i += BW) {
                        const double vi = (i == j) ? 1.0 : S[i * ld + j];
                        S[i * ld + q] = fma(-vi, wq, S[i * ld + q]);
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            S[j * ld + j] = beta;
            sm.tau[j] = t;
        }
        __syncthreads();
    }
}

// Q formed in place from the reflectors (backward accumulation): afterwards
// S[0:M, 0:N] holds the thin Q (before sign normalisation).
__device__ inline void smem_form_q(const Smem& sm, int M, int N) {
    double* S = sm.S;
    const int ld = sm.ld;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int j = N - 1; j >= 0; --j) {
        const double t = sm.tau[j];
        if (j < N - 1 && t != 0.0) {
            // w_q = v^T S[j:, q] for q > j (v_j = 1), then S[j:, q] -= t v w_q
            for (int q0 = j + 1; q0 < N; q0 += 32) {
                const int q = q0 + lane;
                double a0 = 0.0, a1 = 0.0;
                if (q < N) {
                    int i = j + warp;
                    for (; i + BW < M; i += 2 * BW) {
                        const double vi = (i == j) ? 1.0 : S[i * ld + j];
                        a0 = fma(vi, S[i * ld + q], a0);
                        a1 = fma(S[(i + BW) * ld + j], S[(i + BW) * ld + q], a1);
                    }
                    if (i < M) a0 = fma((i == j) ? 1.0 : S[i * ld + j], S[i * ld + q], a0);
                }
                if (q < N) sm.red[warp * NMAX + (q - j)] = a0 + a1;
            }
            __syncthreads();
            if (tid > 0 && tid < N - j) {
                double s0 = 0.0, s1 = 0.0;
#pragma unroll
                for (int w = 0; w < BW; w += 2) {
                    s0 += sm.red[w * NMAX + tid];
                    s1 += sm.red[(w + 1) * NMAX + tid];
                }
                sm.wv[tid] = t * (s0 + s1);
            }
            __syncthreads();
            for (int q0 = j + 1; q0 < N; q0 += 32) {
                const int q = q0 + lane;
                if (q < N) {
                    const double wq = sm.wv[q - j];
                    for (int i = j + warp; i < M; i += BW) {
                        const double vi = (i == j) ? 1.0 : S[i * ld + j];
                        S[i * ld + q] = fma(-vi, wq, S[i * ld + q]);
                    }
                }
            }
            __syncthreads();
        }
        // column j of Q: e_j - t v
        for (int i = tid; i < M; i += BT) {
            double v;
            if (i < j) v = 0.0;
            else if (i == j) v = 1.0 - t;
            else v = -t * S[i * ld + j];
            S[i * ld + j] = v;
        }
        __syncthreads();
    }
}

// Triangular solves on R (N x N upper, global, ld) for the power method,
// lower: R^T y = z (forward); else R w = z (backward); z in shared memory.
// 32 x 32 diagonal blocks are solved by warp 0 from a shared-memory copy with
// reciprocal diagonals; the other rows are updated by the whole CTA.
__device__ inline void smem_tri_solve(const double* R, int ld, int N, double* z, int lower, double* Rb /*[32*33]*/) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = (N + 31) / 32;
    for (int bi = 0; bi < nb; ++bi) {
        const int b = lower ? bi : nb - 1 - bi;
        const int j0 = b * 32, jb = min(32, N - j0);
        for (int e = tid; e < 32 * 32; e += BT) {
            const int a = e >> 5, c = e & 31;
            Rb[a * 33 + c] = (a < jb && c < jb) ? R[(j0 + a) * ld + j0 + c] : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            const double rd = lane < jb ? 1.0 / Rb[lane * 33 + lane] : 0.0;
            double zl = lane < jb ? z[j0 + lane] : 0.0;
            if (lower) {
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (i < jb) {
                        const double yi = __shfl_sync(0xffffffffu, zl, i) * __shfl_sync(0xffffffffu, rd, i);
                        if (lane == i) zl = yi;
                        if (lane > i && lane < jb) zl = fma(-Rb[i * 33 + lane], yi, zl);
                    }
            } else {
#pragma unroll
                for (int i = 31; i >= 0; --i)
                    if (i < jb) {
                        const double wi = __shfl_sync(0xffffffffu, zl, i) * __shfl_sync(0xffffffffu, rd, i);
                        if (lane == i) zl = wi;
                        if (lane < i) zl = fma(-Rb[lane * 33 + i], wi, zl);
                    }
            }
            if (lane < jb) z[j0 + lane] = zl;
        }
        __syncthreads();
        // four partial sums per update (short FP64 dependency chains)
        if (lower) {
            for (int jj = j0 + jb + tid; jj < N; jj += BT) {
                double a[4] = {z[jj], 0.0, 0.0, 0.0};
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (i < jb) a[i & 3] = fma(-R[(j0 + i) * ld + jj], z[j0 + i], a[i & 3]);
                z[jj] = (a[0] + a[1]) + (a[2] + a[3]);
            }
        } else {
            for (int i = tid; i < j0; i += BT) {
                double a[4] = {z[i], 0.0, 0.0, 0.0};
                const double* rr = R + i * ld + j0;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj)
                    if (jj < jb) a[jj & 3] = fma(-rr[jj], z[j0 + jj], a[jj & 3]);
                z[i] = (a[0] + a[1]) + (a[2] + a[3]);
            }
        }
        __syncthreads();
    }
}

__device__ inline double block_sum512(double s, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if (lane == 0) red[warp] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < BW; ++w) t += red[w];
    return t;
}

}  // namespace smemcore
}  // namespace gn

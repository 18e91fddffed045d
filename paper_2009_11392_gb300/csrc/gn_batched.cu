// Batched generalized Nystrom: the sketches (Algorithm 2, step 2) and the core
// (C = Y^T A X, Householder QR, Section 5.1.1/5.1.2) of many independent
// problems of uneven m, n, r, in a fixed sequence of four launches:
//
//   1. one grouped tcgen05 launch computing AX and Y^T A of every problem (the
//      two products of a problem are adjacent in the tile order, so its A is
//      still in L2 when the second product streams it);
//   2. one launch splitting every Y^T A into three BF16 slices;
//   3. one grouped tcgen05 launch for the three slice products of every core;
//   4. one launch with a CTA per problem: C = sum of the slice products in FP64,
//      Householder QR in shared memory, R and Q (formed in place), the
//      detector / truncation, and the second QR when the core is truncated.
//
// gn_batched_prepare builds every descriptor and TMA tensor map on the host and
// uploads them into the caller's workspace once; gn_batched_run only launches
// kernels on the handle's stream (no host synchronisation, no allocation).
#include "gn_internal.cuh"
#include "gn_smem_core.cuh"

#include <cooperative_groups.h>
#include <string.h>

#include <algorithm>
#include <vector>

namespace gn {
namespace {
using namespace smemcore;

constexpr int DIAG_ITERS_B = 6;

struct ProblemDev {
    int m, n, r, l;
    const float* YtA;
    long long ld_yta;
    __nv_bfloat16* s[3];     // slices of Y^T A, (r+l) x lds
    long long lds;
    float* cpart[3];         // slice products, (r+l) x r
    double* Q;
    double* R;
    double* Q2;
    double* R2;
    int* k;
    double* diag;            // [3]: est ||R^{-1}||, est ||C||, eps used
    int* sgn;
};

size_t al(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }
long long r8(long long x) { return (x + 7) / 8 * 8; }

// ----------------------------------------------------------------------------
// 2. split every Y^T A into hi / mid / lo BF16 slices (blockIdx.y = problem)
__global__ void batched_split3_kernel(const ProblemDev* __restrict__ P) {
    const ProblemDev& p = P[blockIdx.y];
    const long long rows = p.r + p.l, cols = p.n, total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e % cols;
        const float x = p.YtA[i * p.ld_yta + j];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(m);
        p.s[0][i * p.lds + j] = h;
        p.s[1][i * p.lds + j] = m;
        p.s[2][i * p.lds + j] = __float2bfloat16_rn(r2);
    }
}

// ----------------------------------------------------------------------------
// 4. per-problem core (shared-memory Householder routines: gn_smem_core.cuh).
__global__ void __launch_bounds__(BT) batched_core_kernel(const ProblemDev* __restrict__ PP, const int* __restrict__ order,
                                                         double eps, int eps_rel, int mode) {
    const ProblemDev& p = PP[order[blockIdx.x]];   // largest cores first (longest-processing-time order)
    extern __shared__ double shm[];
    const int N = p.r, M = p.r + p.l, tid = threadIdx.x;
    Smem sm;
    sm.ld = N + 1;
    sm.S = shm;
    sm.red = sm.S + static_cast<size_t>(MMAX) * (NMAX + 1);
    sm.tau = sm.red + BW * NMAX;
    sm.dsum = sm.tau + NMAX;
    sm.wv = sm.dsum + NMAX;
    sm.scal = sm.wv + NMAX;
    double* z = sm.scal + 8;          // [NMAX]
    double* sgnv = z + NMAX;          // [NMAX]
    const int ld = sm.ld;

    // C = sum of the three slice products, promoted to FP64
    for (int e = tid; e < M * N; e += BT) {
        const int i = e / N, j = e - i * N;
        const long long o = static_cast<long long>(i) * N + j;
        sm.S[i * ld + j] = static_cast<double>(p.cpart[0][o]) + static_cast<double>(p.cpart[1][o]) +
                           static_cast<double>(p.cpart[2][o]);
    }
    __syncthreads();
    smem_qr(sm, M, N);
    // R with diag(R) >= 0 (rows flipped), then Q in place with matching column flips
    for (int i = tid; i < N; i += BT) sgnv[i] = sm.S[i * ld + i] < 0.0 ? -1.0 : 1.0;
    __syncthreads();
    for (int e = tid; e < N * N; e += BT) {
        const int i = e / N, j = e - i * N;
        p.R[e] = j >= i ? sgnv[i] * sm.S[i * ld + j] : 0.0;
    }
    __syncthreads();
    smem_form_q(sm, M, N);
    for (int e = tid; e < M * N; e += BT) {
        const int i = e / N, j = e - i * N;
        p.Q[e] = sgnv[j] * sm.S[i * ld + j];
    }
    __threadfence_block();
    __syncthreads();

    // ---- Section 5.1.2 / 5.1.1 diagnostics (mode SGN / AUTO)
    int k = N, sgn = 0;
    double est = 0.0, rn = 0.0;
    if (mode != GN_MODE_PLAIN) {
        const double inv = 1.0 / sqrt(static_cast<double>(N));
        if (eps_rel) {   // ||R||_2 by power iteration on R^T R
            for (int i = tid; i < N; i += BT) z[i] = inv;
            __syncthreads();
            for (int it = 0; it < DIAG_ITERS_B; ++it) {
                double* y = sm.dsum;
                // y = R z: a warp per row, lanes over its columns
                const int warp = tid >> 5, lane = tid & 31;
                for (int i = warp; i < N; i += BW) {
                    double a = 0.0;
                    for (int jj = i + lane; jj < N; jj += 32) a = fma(p.R[i * N + jj], z[jj], a);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                    if (lane == 0) y[i] = a;
                }
                __syncthreads();
                // w = R^T y: every column split into BT / N row parts, partials combined
                const int parts = min(BT / N, BW);   // sm.red holds BW rows of NMAX
                {
                    const int jj = tid % N, part = tid / N;
                    double a = 0.0;
                    if (part < parts)
                        for (int i = part; i <= jj; i += parts) a = fma(p.R[i * N + jj], y[i], a);
                    if (part < parts) sm.red[part * NMAX + jj] = a;
                }
                __syncthreads();
                double ss = 0.0;
                for (int jj = tid; jj < N; jj += BT) {
                    double a = 0.0;
                    for (int part = 0; part < parts; ++part) a += sm.red[part * NMAX + jj];
                    sm.wv[jj] = a;
                    ss = fma(a, a, ss);
                }
                const double nw = sqrt(block_sum512(ss, sm.red));
                if (nw == 0.0 || !isfinite(nw)) {
                    rn = nw;
                    break;
                }
                rn = sqrt(nw);
                for (int i = tid; i < N; i += BT) z[i] = sm.wv[i] / nw;
                __syncthreads();
            }
            eps = eps * rn;
        }
        // truncation rank: first |R_ii| <= eps
        int kl = N, zero = 0;
        for (int i = tid; i < N; i += BT) {
            const double d = p.R[i * N + i];
            if (fabs(d) <= eps) kl = min(kl, i);
            if (d == 0.0) zero = 1;
        }
        __shared__ int s_k;
        if (tid == 0) s_k = N;
        __syncthreads();
        atomicMin(&s_k, kl);
        zero = __syncthreads_or(zero);
        const int kt = s_k;
        if (zero) {
            est = __longlong_as_double(0x7ff0000000000000LL);
        } else {
            for (int i = tid; i < N; i += BT) z[i] = inv;
            __syncthreads();
            for (int it = 0; it < DIAG_ITERS_B; ++it) {
                smem_tri_solve(p.R, N, N, z, 1, sm.red);
                smem_tri_solve(p.R, N, N, z, 0, sm.red);
                double ss = 0.0;
                for (int i = tid; i < N; i += BT) ss = fma(z[i], z[i], ss);
                const double nw = sqrt(block_sum512(ss, sm.red));
                if (!isfinite(nw)) {
                    est = __longlong_as_double(0x7ff0000000000000LL);
                    break;
                }
                est = sqrt(nw);
                if (nw == 0.0) break;
                for (int i = tid; i < N; i += BT) z[i] /= nw;
                __syncthreads();
            }
        }
        sgn = (mode == GN_MODE_SGN) || (eps > 0.0 && est * eps >= 100.0);
        if (sgn) k = kt;
    }
    if (tid == 0) {
        *p.k = k;
        *p.sgn = sgn;
        p.diag[0] = est;
        p.diag[1] = rn;
        p.diag[2] = eps;
    }
    if (sgn && k > 0 && k < N) {
        // second QR: R_1^T (N x k) = Q2 R2
        __syncthreads();
        sm.ld = k + 1;
        const int ld2 = sm.ld;
        for (int e = tid; e < N * k; e += BT) {
            const int i = e / k, j = e - i * k;   // (R_1^T)[i][j] = R[j][i]
            sm.S[i * ld2 + j] = p.R[j * N + i];
        }
        __syncthreads();
        smem_qr(sm, N, k);
        for (int i = tid; i < k; i += BT) sgnv[i] = sm.S[i * ld2 + i] < 0.0 ? -1.0 : 1.0;
        __syncthreads();
        for (int e = tid; e < k * k; e += BT) {
            const int i = e / k, j = e - i * k;
            p.R2[i * N + j] = j >= i ? sgnv[i] * sm.S[i * ld2 + j] : 0.0;
        }
        __syncthreads();
        smem_form_q(sm, N, k);
        for (int e = tid; e < N * k; e += BT) {
            const int i = e / k, j = e - i * k;
            p.Q2[i * N + j] = sgnv[j] * sm.S[i * ld2 + j];
        }
    }
}

size_t core_smem_bytes() {
    return sizeof(double) * (static_cast<size_t>(MMAX) * (NMAX + 1) + BW * NMAX + 3 * NMAX + 8 + 2 * NMAX);
}

// Layout of the prepared tables at the start of the workspace.
struct Layout {
    size_t maps, sk_gemms, c_gemms, probs, scratch, total;
    int n_maps, sk_tiles, c_tiles;
};

}  // namespace
}  // namespace gn

using namespace gn;

extern "C" {

gn_status gn_batched_workspace_size(int32_t count, const gn_problem* probs, size_t* bytes) {
    if (count <= 0 || !probs || !bytes) return GN_ERR_INVALID_ARG;
    size_t b = 4096;
    b += al(sizeof(CUtensorMap) * 7 * count);
    b += al(sizeof(TcGemm) * 2 * count) + al(sizeof(TcGemm) * 3 * count) + al(sizeof(ProblemDev) * count);
    b += al(sizeof(int) * count);
    for (int i = 0; i < count; ++i) {
        const long long n = probs[i].A.cols, r = probs[i].X.cols, rl = probs[i].Y.cols;
        b += 3 * al(sizeof(__nv_bfloat16) * rl * r8(n)) + 3 * al(sizeof(float) * rl * r) + al(8 * 4);
    }
    *bytes = b;
    return GN_OK;
}

gn_status gn_batched_prepare(gn_handle h, int32_t count, const gn_problem* probs, void* ws, size_t ws_bytes) {
    if (!h || count <= 0 || !probs || !ws) return GN_ERR_INVALID_ARG;
    size_t need = 0;
    GN_TRY(gn_batched_workspace_size(count, probs, &need));
    if (ws_bytes < need) return GN_ERR_WORKSPACE;
    char* base = static_cast<char*>(ws);
    size_t off = 256;   // header: counts
    const size_t o_maps = off;
    off += al(sizeof(CUtensorMap) * 7 * count);
    const size_t o_sk = off;
    off += al(sizeof(TcGemm) * 2 * count);
    const size_t o_c = off;
    off += al(sizeof(TcGemm) * 3 * count);
    const size_t o_p = off;
    off += al(sizeof(ProblemDev) * count);
    const size_t o_ord = off;
    off += al(sizeof(int) * count);

    std::vector<CUtensorMap> maps(7 * static_cast<size_t>(count));
    std::vector<TcGemm> sk(2 * static_cast<size_t>(count)), cg(3 * static_cast<size_t>(count));
    std::vector<ProblemDev> pd(count);
    int sk_tiles = 0, c_tiles = 0;
    const int policy = h->batched_policy;
    const int sk_mt = (policy & 16) ? 2 : 1;
    const int bn_yta = (policy & 3) == 1 ? 64 : ((policy & 3) == 2 ? 256 : 128);
    // position of each problem's two sketch GEMMs in the tile list
    std::vector<int> slot(count);
    {
        std::vector<int> ord(count);
        for (int i = 0; i < count; ++i) ord[i] = i;
        if (policy & 8) {
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b2) {
                const auto w = [&](int i) {
                    return double(probs[i].A.rows) * probs[i].A.cols * (2.0 * probs[i].X.cols + probs[i].Y.cols);
                };
                return w(a) > w(b2);
            });
        }
        for (int pos = 0; pos < count; ++pos) slot[ord[pos]] = pos;
    }
    for (int i = 0; i < count; ++i) {
        const gn_problem& q = probs[i];
        const long long m = q.A.rows, n = q.A.cols, r = q.X.cols, rl = q.Y.cols, l = rl - r;
        if (m <= 0 || n <= 0 || r < 1 || l < 1 || r > std::min(m, n) || rl > m) return GN_ERR_SHAPE;
        if (r > NMAX || rl > MMAX) return GN_ERR_UNSUPPORTED;   // the core must fit in shared memory
        if (q.X.rows != n || q.Y.rows != m || q.AX.rows != m || q.AX.cols != r || q.YtA.rows != rl ||
            q.YtA.cols != n)
            return GN_ERR_SHAPE;
        if (q.A.dtype != GN_BF16 || q.X.dtype != GN_BF16 || q.Y.dtype != GN_BF16 || q.AX.dtype != GN_F32 ||
            q.YtA.dtype != GN_F32)
            return GN_ERR_DTYPE;
        if (!q.A.data || !q.X.data || !q.Y.data || !q.AX.data || !q.YtA.data || !q.Q || !q.R || !q.Q2 ||
            !q.R2 || !q.k)
            return GN_ERR_INVALID_ARG;
        for (const gn_mat* mm : {&q.A, &q.X, &q.Y})
            if ((reinterpret_cast<uintptr_t>(mm->data) & 15) || mm->ld % 8) return GN_ERR_ALIGNMENT;
        CUtensorMap* mp = &maps[7 * static_cast<size_t>(i)];
        GN_TRY(tc_make_map_bf16(&mp[0], q.A.data, m, n, q.A.ld, 64, 128));
        GN_TRY(tc_make_map_bf16(&mp[1], q.A.data, m, n, q.A.ld, 64, 64));
        GN_TRY(tc_make_map_bf16(&mp[2], q.X.data, n, r, q.X.ld, 64, 64));
        GN_TRY(tc_make_map_bf16(&mp[3], q.Y.data, m, rl, q.Y.ld, 64, 64));
        // per-problem scratch
        ProblemDev& d = pd[i];
        d.m = static_cast<int>(m);
        d.n = static_cast<int>(n);
        d.r = static_cast<int>(r);
        d.l = static_cast<int>(l);
        d.YtA = static_cast<const float*>(q.YtA.data);
        d.ld_yta = q.YtA.ld;
        d.lds = r8(n);
        for (int s = 0; s < 3; ++s) {
            d.s[s] = reinterpret_cast<__nv_bfloat16*>(base + off);
            off += al(sizeof(__nv_bfloat16) * rl * d.lds);
        }
        for (int s = 0; s < 3; ++s) {
            d.cpart[s] = reinterpret_cast<float*>(base + off);
            off += al(sizeof(float) * rl * r);
        }
        d.diag = reinterpret_cast<double*>(base + off);
        d.sgn = reinterpret_cast<int*>(base + off + 24);
        off += al(8 * 4);
        d.Q = q.Q;
        d.R = q.R;
        d.Q2 = q.Q2;
        d.R2 = q.R2;
        d.k = q.k;
        for (int s = 0; s < 3; ++s) GN_TRY(tc_make_map_bf16(&mp[4 + s], d.s[s], rl, n, d.lds, 64, 128));
        // sketch GEMMs: AX (A K-major, X MN-major), Y^T A (Y MN-major, A MN-major)
        const int mi = 7 * i;
        TcGemm& g0 = sk[2 * slot[i]];
        memset(&g0, 0, sizeof(g0));
        g0.M = static_cast<int>(m);
        g0.N = static_cast<int>(r);
        g0.K = static_cast<int>(n);
        g0.bn = (policy & 4) && r > 64 ? 64 : static_cast<int>(std::min<long long>(256, (r + 63) / 64 * 64));
        g0.b_mn = 1;
        g0.nsrc = 1;
        g0.a_map[0] = mi + 0;
        g0.b_map[0] = mi + 2;
        g0.D = static_cast<float*>(q.AX.data);
        g0.ldd = q.AX.ld;
        TcGemm& g1 = sk[2 * slot[i] + 1];
        memset(&g1, 0, sizeof(g1));
        g1.M = static_cast<int>(rl);
        g1.N = static_cast<int>(n);
        g1.K = static_cast<int>(m);
        g1.bn = bn_yta;
        g1.a_mn = 1;
        g1.b_mn = 1;
        g1.nsrc = 1;
        g1.a_map[0] = mi + 3;
        g1.b_map[0] = mi + 1;
        g1.D = static_cast<float*>(q.YtA.data);
        g1.ldd = q.YtA.ld;
        for (int s = 0; s < 3; ++s) {
            TcGemm& g = cg[3 * i + s];
            memset(&g, 0, sizeof(g));
            g.M = static_cast<int>(rl);
            g.N = static_cast<int>(r);
            g.K = static_cast<int>(n);
            g.bn = static_cast<int>(std::min<long long>(256, (r + 63) / 64 * 64));
            g.b_mn = 1;
            g.nsrc = 1;
            g.a_map[0] = mi + 4 + s;
            g.b_map[0] = mi + 2;
            g.D = d.cpart[s];
            g.ldd = r;
            GN_TRY(tc_prepare_gemm(&g, c_tiles));
            c_tiles += g.tiles_m * g.tiles_n;
        }
    }
    for (int pos = 0; pos < 2 * count; ++pos) {   // tile bases in list order
        GN_TRY(tc_prepare_gemm(&sk[pos], sk_tiles, sk_mt));
        sk_tiles += sk[pos].tiles_m * sk[pos].tiles_n;
    }
    if (off > ws_bytes) return GN_ERR_WORKSPACE;
    int header[4] = {count, sk_tiles, c_tiles, 0};
    GN_CUDA_TRY(cudaMemcpy(base, header, sizeof(header), cudaMemcpyHostToDevice));
    GN_CUDA_TRY(cudaMemcpy(base + o_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
    GN_CUDA_TRY(cudaMemcpy(base + o_sk, sk.data(), sizeof(TcGemm) * sk.size(), cudaMemcpyHostToDevice));
    GN_CUDA_TRY(cudaMemcpy(base + o_c, cg.data(), sizeof(TcGemm) * cg.size(), cudaMemcpyHostToDevice));
    GN_CUDA_TRY(cudaMemcpy(base + o_p, pd.data(), sizeof(ProblemDev) * pd.size(), cudaMemcpyHostToDevice));
    // core kernel order: decreasing (r + l) r^2, the FP64 work of a core
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b2) {
        const double wa = double(pd[a].r + pd[a].l) * pd[a].r * pd[a].r;
        const double wb = double(pd[b2].r + pd[b2].l) * pd[b2].r * pd[b2].r;
        return wa > wb;
    });
    GN_CUDA_TRY(cudaMemcpy(base + o_ord, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
    // keep the host-side counts in the header's host mirror (the run call re-reads them)
    h->batched_count = count;
    h->batched_sk_tiles = sk_tiles;
    h->batched_mt = sk_mt;
    h->batched_c_tiles = c_tiles;
    h->batched_ws = ws;
    return GN_OK;
}

gn_status gn_batched_set_policy(gn_handle h, int32_t policy) {
    if (!h || policy < 0 || policy >= 32 || (policy & 3) == 3) return GN_ERR_INVALID_ARG;
    h->batched_policy = policy;
    return GN_OK;
}

gn_status gn_batched_tune(gn_handle h, int32_t count, const gn_problem* probs, void* ws, size_t ws_bytes,
                          double eps, int32_t mode, int32_t* best, double* best_ms) {
    if (!h || !best) return GN_ERR_INVALID_ARG;
    static const int kPolicies[GN_BATCHED_POLICIES] = {0,  1,  2,  4,  5,  6,  8,  9,  10, 12, 13, 14,
                                                       16, 17, 18, 20, 21, 22, 24, 25, 26, 28, 29, 30};
    cudaEvent_t e0, e1;
    GN_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GN_ERR_CUDA;
    }
    int best_p = -1;
    float best_t = 0.0f;
    gn_status st = GN_OK;
    for (int c = 0; c < GN_BATCHED_POLICIES && st == GN_OK; ++c) {
        h->batched_policy = kPolicies[c];
        st = gn_batched_prepare(h, count, probs, ws, ws_bytes);
        if (st == GN_OK) st = gn_batched_run(h, eps, mode, ws, ws_bytes);   // warm-up
        if (st != GN_OK) break;
        if (cudaEventRecord(e0, h->stream) != cudaSuccess) { st = GN_ERR_CUDA; break; }
        for (int rep = 0; rep < 3 && st == GN_OK; ++rep) st = gn_batched_run(h, eps, mode, ws, ws_bytes);
        if (st != GN_OK) break;
        float ms = 0.0f;
        if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = GN_ERR_CUDA;
            break;
        }
        if (best_p < 0 || ms < best_t) {
            best_p = kPolicies[c];
            best_t = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GN_OK) return st;
    h->batched_policy = best_p;
    GN_TRY(gn_batched_prepare(h, count, probs, ws, ws_bytes));
    *best = best_p;
    if (best_ms) *best_ms = best_t / 3.0;
    return GN_OK;
}

gn_status gn_batched_run(gn_handle h, double eps, int32_t mode, void* ws, size_t ws_bytes) {
    if (!h || !ws) return GN_ERR_INVALID_ARG;
    const int eps_rel = (mode & GN_EPS_RELATIVE) ? 1 : 0;
    mode &= ~GN_EPS_RELATIVE;
    if (mode < GN_MODE_PLAIN || mode > GN_MODE_AUTO || !(eps >= 0.0)) return GN_ERR_INVALID_ARG;
    if (ws != h->batched_ws || h->batched_count <= 0) return GN_ERR_INVALID_ARG;   // prepare first
    const int count = h->batched_count;
    char* base = static_cast<char*>(ws);
    const size_t o_maps = 256;
    const size_t o_sk = o_maps + al(sizeof(CUtensorMap) * 7 * count);
    const size_t o_c = o_sk + al(sizeof(TcGemm) * 2 * count);
    const size_t o_p = o_c + al(sizeof(TcGemm) * 3 * count);
    const size_t o_ord = o_p + al(sizeof(ProblemDev) * count);
    (void)ws_bytes;
    const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(base + o_maps);
    GN_TRY(tc_launch_grouped(h, reinterpret_cast<const TcGemm*>(base + o_sk), 2 * count, maps, h->batched_sk_tiles,
                             h->batched_mt));
    const ProblemDev* pd = reinterpret_cast<const ProblemDev*>(base + o_p);
    batched_split3_kernel<<<dim3(16, count), 256, 0, h->stream>>>(pd);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    GN_TRY(tc_launch_grouped(h, reinterpret_cast<const TcGemm*>(base + o_c), 3 * count, maps, h->batched_c_tiles));
    static bool attr = false;
    if (!attr) {
        GN_CUDA_TRY(cudaFuncSetAttribute(batched_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(core_smem_bytes())));
        attr = true;
    }
    batched_core_kernel<<<count, BT, core_smem_bytes(), h->stream>>>(
        pd, reinterpret_cast<const int*>(base + o_ord), eps, eps_rel, mode);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

}  // extern "C"

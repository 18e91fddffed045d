// Adjoint of the generalized Nystrom map A -> A_hat (plain GN, full-rank core).
//
// For L(A) = <G, A_hat(A)> with X, Y fixed and C = Y^T A X = QR of full column
// rank, differentiating A_hat = AX C^+ Y^T A (d(C^+) = -C^+ dC C^+ +
// (C^T C)^{-1} dC^T (I - C C^+)) gives
//
//     dL/dA = (S1 Q R^{-T} + Y K) X^T + Y (Q S2),
//     S1 = G (Y^T A)^T,  F = AX R^{-1},  S2 = F^T G,  W = F^T S1,
//     K  = (I - Q Q^T) W^T R^{-T} - Q (W Q) R^{-T}.
//
// Every C^+ enters through Q and triangular solves with R (the paper's
// Section 5.1 rule: never form the core's inverse).  FP64 inputs: every step
// in FP64 on the FP64 units.  FP32 inputs, all on the tcgen05 tensor cores
// except the QR, the two triangular solves and the r x r algebra (FP64): the
// sketches AX, Y^T A, the core C = (Y^T A) X and the contractions over G (S1,
// S2, W), whose errors the core's conditioning and the projection I - Q Q^T
// amplify, as FP64-accurate digit-sliced products; the products after those
// (P, Q S2 and the two rank-r products that form the gradient) as three-slice
// BF16 products (x = s0 + s1 + s2, the six slice products of order <= 2, FP32
// accumulation: FP32-level accuracy).  With K R^T = (I - Q Q^T) W^T - Q W Q,
// the two m x r terms share one solve: P = (S1 Q + Y (K R^T)) R^{-T}.
// gn_forward_dense and gn_backward form the shared front (the sketches, C's QR
// and F) in the workspace and leave it there; gn_backward_saved starts from it,
// as an autograd backward starts from what its forward saved.
#include "gn_internal.cuh"

#include <algorithm>
#include <string.h>

namespace gn {
namespace {

__global__ void copy_t_kernel(const double* __restrict__ s, long long rows, long long cols, long long lds, double* d,
                              long long ldd) {
    // d (cols x rows) = s^T
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e % cols;
        d[j * ldd + i] = s[i * lds + j];
    }
}

int ew(gn_handle h, long long total) {
    return static_cast<int>(std::max<long long>(1, std::min<long long>((total + 255) / 256, 8LL * h->sm_count)));
}

gn_status transpose_f64(gn_handle h, const double* s, long long rows, long long cols, long long lds, double* d,
                        long long ldd) {
    if (rows * cols == 0) return GN_OK;
    copy_t_kernel<<<ew(h, rows * cols), 256, 0, h->stream>>>(s, rows, cols, lds, d, ldd);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }
long long rnd8(long long x) { return (x + 7) / 8 * 8; }

// ---------------------------------------------------------------- three-slice BF16 products
// Three BF16 slices of a row-major FP32 or FP64 matrix: s0 = bf16(x), s1 =
// bf16(x - s0), s2 = bf16(x - s0 - s1) (residuals in the source precision), so
// s0 + s1 + s2 holds the 24 significant bits of an FP32 x.
__global__ void split3s_kernel(const void* __restrict__ src, int f64, long long rows, long long cols, long long lds,
                               __nv_bfloat16* __restrict__ s0, __nv_bfloat16* __restrict__ s1,
                               __nv_bfloat16* __restrict__ s2, long long ldd) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e - i * cols;
        __nv_bfloat16 a, b, c;
        if (f64) {
            const double x = static_cast<const double*>(src)[i * lds + j];
            a = __float2bfloat16_rn(static_cast<float>(x));
            const double r1 = x - static_cast<double>(__bfloat162float(a));
            b = __float2bfloat16_rn(static_cast<float>(r1));
            c = __float2bfloat16_rn(static_cast<float>(r1 - static_cast<double>(__bfloat162float(b))));
        } else {
            const float x = static_cast<const float*>(src)[i * lds + j];
            a = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(a);
            b = __float2bfloat16_rn(r1);
            c = __float2bfloat16_rn(r1 - __bfloat162float(b));
        }
        s0[i * ldd + j] = a;
        s1[i * ldd + j] = b;
        s2[i * ldd + j] = c;
    }
}

// A matrix held as three BF16 planes (row-major, ld a multiple of 8: the TMA rule).
struct Plane {
    __nv_bfloat16* s[3];
    long long rows, cols, ld;
};

gn_status split3s(gn_handle h, const void* src, int f64, long long lds, const Plane& p) {
    const long long total = p.rows * p.cols;
    if (total == 0) return GN_OK;
    split3s_kernel<<<ew(h, total), 256, 0, h->stream>>>(src, f64, p.rows, p.cols, lds, p.s[0], p.s[1], p.s[2], p.ld);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

// One product of a launch: D (M x N, FP32) = sum over pairs of op(A_p) op(B_p),
// each pair as the six slice products of order <= 2 (FP32-level accuracy,
// FP32 accumulation).  a_mn = 0: A plane is M x K (K-major); a_mn = 1: A plane
// is K x M.  b_mn = 0: B plane is N x K; b_mn = 1: K x N.  A plane narrower than
// K reads zeros beyond its width (TMA fill), so pairs with different K share
// the launch's K.
struct X6 {
    int M, N, K;
    int a_mn, b_mn;
    int npair;
    const Plane* A[2];
    const Plane* B[2];
    float* D;
    long long ldd;
};

gn_status x6_launch(gn_handle h, X6* gs, int ng) {
    static const int ord[6][2] = {{0, 0}, {0, 1}, {1, 0}, {0, 2}, {1, 1}, {2, 0}};
    TcParams p;
    memset(&p, 0, sizeof(p));
    int nm = 0;
    for (int g = 0; g < ng; ++g) {
        X6& x = gs[g];
        TcGemm& G = p.g[g];
        G.M = x.M;
        G.N = x.N;
        G.K = x.K;
        G.a_mn = x.a_mn;
        G.b_mn = x.b_mn;
        // N tile: the widest that keeps about two tiles per SM (MN-major B: a multiple of 64)
        const int q = x.b_mn ? 64 : 16;
        int bn = static_cast<int>(std::min<long long>(256, (x.N + q - 1) / q * q));
        while (bn > 64 && static_cast<long long>((x.M + 127) / 128) * ((x.N + bn - 1) / bn) < 2LL * h->sm_count)
            bn = std::max(64, (bn / 2 + q - 1) / q * q);
        G.bn = bn;
        G.nsrc = 6 * x.npair;
        if (G.nsrc > TC_MAX_SRC || nm + 6 * x.npair > TC_MAX_MAPS) return GN_ERR_UNSUPPORTED;
        for (int pi = 0; pi < x.npair; ++pi) {
            const Plane& A = *x.A[pi];
            const Plane& B = *x.B[pi];
            const int ma = nm, mb = nm + 3;
            for (int t = 0; t < 3; ++t) {
                if (x.a_mn) GN_TRY(tc_make_map_bf16(&p.maps[ma + t], A.s[t], A.rows, A.cols, A.ld, 64, 64));
                else GN_TRY(tc_make_map_bf16(&p.maps[ma + t], A.s[t], A.rows, A.cols, A.ld, 64, 128));
                if (x.b_mn) GN_TRY(tc_make_map_bf16(&p.maps[mb + t], B.s[t], B.rows, B.cols, B.ld, 64, 64));
                else GN_TRY(tc_make_map_bf16(&p.maps[mb + t], B.s[t], B.rows, B.cols, B.ld, 64, bn));
            }
            nm += 6;
            for (int o = 0; o < 6; ++o) {
                G.a_map[6 * pi + o] = ma + ord[o][0];
                G.b_map[6 * pi + o] = mb + ord[o][1];
            }
        }
        G.D = x.D;
        G.ldd = x.ldd;
    }
    p.ngemm = ng;
    return tc_launch(h, &p);
}

struct Bump {
    char* base;
    size_t cap, off;
    bool ok;
    template <typename T>
    T* take(size_t n) {
        const size_t b = align256(n * sizeof(T));
        if (off + b > cap) {
            ok = false;
            return nullptr;
        }
        T* p = reinterpret_cast<T*>(base + off);
        off += b;
        return p;
    }
};

// Scratch of the adjoint; the QR / GEMM scratch is the tail after these.
size_t backward_fixed(long long m, long long n, long long r, long long l) {
    const long long rl = r + l;
    size_t b = 0;
    b += align256(8 * m * r) * 3;     // AX (f64), F, P
    b += align256(8 * rl * n) * 2;    // Y^T A (f64), Q' = Q S2
    b += align256(8 * rl * r) * 5;    // C, W (QR copy), Q, K1, scratch
    b += align256(8 * r * r) * 3;     // R, QtZ, WQ
    b += align256(8 * m * rl);        // S1
    b += align256(8 * r * n);         // S2
    b += align256(8 * r * rl) * 2;    // W, W^T
    return b + 4096;
}

// ---------------------------------------------------------------- FP32 inputs on the tensor cores
// Workspace of the FP32 path (forward and backward share the layout).
struct TcWs {
    Plane Xs, Ys, YtATs, Fs, S1s, S2Ts, Qs, Kts, Ps, QpTs, Ahs;
    float *S2, *P32, *QpT;
    double *X64, *Y64, *AX, *YtAT, *C, *Wq, *Q, *R, *W64, *Wt, *M1, *P64, *S1, *S2T;
    double* inner;
    size_t inner_bytes;
    void* oz;
    size_t oz_bytes;
};

size_t tc_inner_bytes(long long m, long long n, long long r, long long l, int sms) {
    const long long rl = r + l;
    return std::max({qr_ws_bytes(rl, r, sms), trsm_ws_bytes(m, r, sms), dgemm_ws_bytes(r, r, rl, sms),
                     dgemm_ws_bytes(rl, r, r, sms)});
}
size_t tc_oz_bytes(long long m, long long n, long long r, long long l) {
    return std::max({oz_ws_bytes(m, r, n, 1), oz_ws_bytes(n, r + l, m, 1), oz_ws_bytes(r + l, r, n, 0),
                     oz_ws_bytes(m, 128, r, 0), oz_ws_bytes(m, r + l, n, 1), oz_ws_bytes(n, r, m, 1),
                     oz_ws_bytes(r, r + l, m, 0)});
}

// Carves (or, with base == nullptr, sizes) the FP32 path's workspace.
size_t tc_carve(long long m, long long n, long long r, long long l, int sms, char* base, TcWs* w) {
    const long long rl = r + l;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* q = base ? base + off : nullptr;
        off += align256(bytes);
        return q;
    };
    auto plane = [&](long long rows, long long cols) {
        Plane p;
        p.rows = rows;
        p.cols = cols;
        p.ld = rnd8(cols);
        for (int t = 0; t < 3; ++t) p.s[t] = reinterpret_cast<__nv_bfloat16*>(take(2 * rows * p.ld));
        return p;
    };
    TcWs t;
    t.Xs = plane(n, r);
    t.Ys = plane(m, rl);
    t.YtATs = plane(n, rl);
    t.Fs = plane(m, r);
    t.S1s = plane(m, rl);
    t.S2Ts = plane(n, r);
    t.Qs = plane(rl, r);
    t.Kts = plane(rl, r);
    t.Ps = plane(m, r);
    t.QpTs = plane(n, rl);
    t.Ahs = plane(r, n);
    auto f32 = [&](long long rows, long long cols) { return reinterpret_cast<float*>(take(4 * rows * rnd8(cols))); };
    auto f64 = [&](long long count) { return reinterpret_cast<double*>(take(8 * count)); };
    t.S2 = f32(r, n);
    t.P32 = f32(m, r);
    t.QpT = f32(n, rl);
    t.X64 = f64(n * r);
    t.Y64 = f64(m * rl);
    t.AX = f64(m * r);
    t.YtAT = f64(n * rl);
    t.C = f64(rl * r);
    t.Wq = f64(rl * r);
    t.Q = f64(rl * r);
    t.R = f64(r * r);
    t.W64 = f64(r * rl);
    t.Wt = f64(rl * r);
    t.M1 = f64(r * r);
    t.P64 = f64(m * r);
    t.S1 = f64(m * rl);
    t.S2T = f64(n * r);
    t.oz_bytes = tc_oz_bytes(m, n, r, l);
    t.oz = take(t.oz_bytes);
    t.inner_bytes = tc_inner_bytes(m, n, r, l, sms);
    t.inner = reinterpret_cast<double*>(take(t.inner_bytes));
    if (w) *w = t;
    return off + 256;
}

// BF16 digits per operand of the FP32 adjoint's digit-sliced products: every
// term within about 2^-27 of max|a_i.| max|b_.j| (orders 0..3, all exact in the
// FP32 accumulators), far inside the FP32 gradient's 1e-3.
constexpr int ADJ_DIGITS = 4;

// The steps both directions share.  The sketches of the FP32 A feed the core,
// whose conditioning amplifies their errors, so they are formed to FP64
// accuracy by digit slicing on the tensor cores: AX (m x r) and (Y^T A)^T =
// A^T Y (n x (r+l), kept transposed), then C = (Y^T A) X, Householder C = QR,
// F = (AX) R^{-1}.
gn_status tc_front(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, long long m, long long n,
                   long long r, long long rl, TcWs& t) {
    GN_TRY(copy_f32_to_f64(h, static_cast<const float*>(X->data), n, r, X->ld, t.X64, r));
    GN_TRY(copy_f32_to_f64(h, static_cast<const float*>(Y->data), m, rl, Y->ld, t.Y64, rl));
    GN_TRY(oz_dgemm(h, m, r, n, 1.0, A->data, 1, A->ld, 0, t.X64, r, 0, 0.0, t.AX, r, t.oz, t.oz_bytes, ADJ_DIGITS));
    GN_TRY(oz_dgemm(h, n, rl, m, 1.0, A->data, 1, A->ld, 1, t.Y64, rl, 0, 0.0, t.YtAT, rl, t.oz, t.oz_bytes, ADJ_DIGITS));
    GN_TRY(oz_dgemm(h, rl, r, n, 1.0, t.YtAT, 0, rl, 1, t.X64, r, 0, 0.0, t.C, r, t.oz, t.oz_bytes, ADJ_DIGITS));
    GN_CUDA_TRY(cudaMemcpyAsync(t.Wq, t.C, sizeof(double) * rl * r, cudaMemcpyDeviceToDevice, h->stream));
    GN_TRY(householder_qr(h, t.Wq, rl, r, r, t.Q, r, t.R, r, t.inner, t.inner_bytes));
    GN_TRY(trsm_right_upper(h, t.AX, m, r, r, t.R, r, 0, t.inner, t.inner_bytes, t.oz, t.oz_bytes));   // F in AX
    GN_TRY(split3s(h, t.AX, 1, r, t.Fs));
    GN_TRY(split3s(h, t.YtAT, 1, rl, t.YtATs));
    GN_TRY(split3s(h, t.Q, 1, r, t.Qs));
    return GN_OK;
}

// The backward's own part, from the front in t (F in t.AX, (Y^T A)^T, Q, R and
// their BF16 slices); reads nothing of A and leaves the front as it was.
gn_status tc_back(gn_handle h, const gn_mat* X, const gn_mat* Y, const gn_mat* Gup, gn_mat* dA, long long m,
                  long long n, long long r, long long rl, TcWs& t) {
    const double* F = t.AX;
    // The contractions over G feed W and K, where the projection (I - Q Q^T)
    // cancels most of W^T: FP64-accurate digit-sliced products.
    //   S1 = G (Y^T A)^T (m x (r+l)),  S2^T = G^T F (n x r),  W = F^T S1 (r x (r+l))
    GN_TRY(oz_dgemm(h, m, rl, n, 1.0, Gup->data, 1, Gup->ld, 0, t.YtAT, rl, 0, 0.0, t.S1, rl, t.oz, t.oz_bytes, ADJ_DIGITS));
    GN_TRY(oz_dgemm(h, n, r, m, 1.0, Gup->data, 1, Gup->ld, 1, F, r, 0, 0.0, t.S2T, r, t.oz, t.oz_bytes, ADJ_DIGITS));
    GN_TRY(oz_dgemm(h, r, rl, m, 1.0, F, 0, r, 1, t.S1, rl, 0, 0.0, t.W64, rl, t.oz, t.oz_bytes, ADJ_DIGITS));
    // K R^T = W^T - Q (Q^T W^T + W Q)   ((r+l) x r, FP64)
    GN_TRY(transpose_f64(h, t.W64, r, rl, rl, t.Wt, r));
    GN_TRY(dgemm(h, r, r, rl, 1.0, t.Q, r, 1, t.Wt, r, 0, 0.0, t.M1, r, t.inner, t.inner_bytes));
    GN_TRY(dgemm(h, r, r, rl, 1.0, t.W64, rl, 0, t.Q, r, 0, 1.0, t.M1, r, t.inner, t.inner_bytes));
    GN_TRY(dgemm(h, rl, r, r, -1.0, t.Q, r, 0, t.M1, r, 0, 1.0, t.Wt, r, t.inner, t.inner_bytes));
    // P = (S1 Q + Y (K R^T)) R^{-T} (m x r);  Q'^T = S2^T Q^T (n x (r+l))
    GN_TRY(split3s(h, t.S1, 1, rl, t.S1s));
    GN_TRY(split3s(h, t.Wt, 1, r, t.Kts));
    GN_TRY(split3s(h, Y->data, 0, Y->ld, t.Ys));
    GN_TRY(split3s(h, t.S2T, 1, r, t.S2Ts));
    X6 g[1];
    g[0] = X6{static_cast<int>(m), static_cast<int>(r), static_cast<int>(rl), 0, 1, 2, {&t.S1s, &t.Ys},
              {&t.Qs, &t.Kts}, t.P32, rnd8(r)};
    GN_TRY(x6_launch(h, g, 1));   // 12 tensor maps: the launch's limit
    g[0] = X6{static_cast<int>(n), static_cast<int>(rl), static_cast<int>(r), 0, 0, 1, {&t.S2Ts}, {&t.Qs},
              t.QpT, rnd8(rl)};
    GN_TRY(x6_launch(h, g, 1));
    GN_TRY(copy_f32_to_f64(h, t.P32, m, r, rnd8(r), t.P64, r));
    GN_TRY(trsm_right_upper(h, t.P64, m, r, r, t.R, r, 1, t.inner, t.inner_bytes, t.oz, t.oz_bytes));
    // dA = P X^T + Y Q'
    GN_TRY(split3s(h, t.P64, 1, r, t.Ps));
    GN_TRY(split3s(h, t.QpT, 0, rnd8(rl), t.QpTs));
    GN_TRY(split3s(h, X->data, 0, X->ld, t.Xs));
    g[0] = X6{static_cast<int>(m), static_cast<int>(n), static_cast<int>(rl), 0, 0, 2, {&t.Ps, &t.Ys},
              {&t.Xs, &t.QpTs}, static_cast<float*>(dA->data), dA->ld};
    return x6_launch(h, g, 1);
}

// The forward's own part: G = Q^T (Y^T A) (r x n), then A_hat = F G; the front
// stays in t for a later backward.
gn_status tc_forward_rest(gn_handle h, gn_mat* Ahat, long long m, long long n, long long r, long long rl, TcWs& t) {
    X6 g[1];
    g[0] = X6{static_cast<int>(r), static_cast<int>(n), static_cast<int>(rl), 1, 0, 1, {&t.Qs}, {&t.YtATs},
              t.S2, rnd8(n)};
    GN_TRY(x6_launch(h, g, 1));
    GN_TRY(split3s(h, t.S2, 0, rnd8(n), t.Ahs));
    g[0] = X6{static_cast<int>(m), static_cast<int>(n), static_cast<int>(r), 0, 1, 1, {&t.Fs}, {&t.Ahs},
              static_cast<float*>(Ahat->data), Ahat->ld};
    return x6_launch(h, g, 1);
}

// ---------------------------------------------------------------- FP64 inputs
// Workspace of the FP64 path (forward and backward share the layout), the QR /
// GEMM scratch in the tail.
struct F64Ws {
    double *AX, *F, *P, *YtA, *Qp, *C, *Wq, *Q, *K1, *Wt, *R, *QtZ, *WQ, *S1, *S2, *W;
    double* inner;
    size_t inner_bytes;
};

bool f64_carve(void* ws, size_t ws_bytes, long long m, long long n, long long r, long long rl, F64Ws* w) {
    Bump b{static_cast<char*>(ws), ws_bytes, 0, true};
    w->AX = b.take<double>(m * r);
    w->F = b.take<double>(m * r);
    w->P = b.take<double>(m * r);
    w->YtA = b.take<double>(rl * n);
    w->Qp = b.take<double>(rl * n);   // Q' = Q S2 (backward) or G = Q^T (Y^T A) (forward)
    w->C = b.take<double>(rl * r);
    w->Wq = b.take<double>(rl * r);
    w->Q = b.take<double>(rl * r);
    w->K1 = b.take<double>(rl * r);
    w->Wt = b.take<double>(rl * r);
    w->R = b.take<double>(r * r);
    w->QtZ = b.take<double>(r * r);
    w->WQ = b.take<double>(r * r);
    w->S1 = b.take<double>(m * rl);
    w->S2 = b.take<double>(r * n);
    w->W = b.take<double>(r * rl);
    if (!b.ok) return false;
    const size_t o = align256(b.off);
    w->inner = reinterpret_cast<double*>(static_cast<char*>(ws) + o);
    w->inner_bytes = ws_bytes > o ? ws_bytes - o : 0;
    return true;
}

// Sketches and the core (Algorithm 2 step 2), then F = AX R^{-1}.
gn_status f64_front(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, long long m, long long n,
                    long long r, long long rl, F64Ws& w) {
    const double* A64 = static_cast<const double*>(A->data);
    const double* X64 = static_cast<const double*>(X->data);
    GN_TRY(dgemm(h, m, r, n, 1.0, A64, A->ld, 0, X64, X->ld, 0, 0.0, w.AX, r, w.inner, w.inner_bytes));
    GN_TRY(dgemm(h, rl, n, m, 1.0, static_cast<const double*>(Y->data), Y->ld, 1, A64, A->ld, 0, 0.0, w.YtA, n,
                 w.inner, w.inner_bytes));
    GN_TRY(dgemm(h, rl, r, n, 1.0, w.YtA, n, 0, X64, X->ld, 0, 0.0, w.C, r, w.inner, w.inner_bytes));
    GN_CUDA_TRY(cudaMemcpyAsync(w.Wq, w.C, sizeof(double) * rl * r, cudaMemcpyDeviceToDevice, h->stream));
    GN_TRY(householder_qr(h, w.Wq, rl, r, r, w.Q, r, w.R, r, w.inner, w.inner_bytes));
    GN_CUDA_TRY(cudaMemcpyAsync(w.F, w.AX, sizeof(double) * m * r, cudaMemcpyDeviceToDevice, h->stream));
    return trsm_right_upper(h, w.F, m, r, r, w.R, r, 0, w.inner, w.inner_bytes);
}

// The backward's own part from the front (F, Y^T A, Q, R), which it leaves as it was.
gn_status f64_back(gn_handle h, const gn_mat* X, const gn_mat* Y, const gn_mat* Gup, gn_mat* dA, long long m,
                   long long n, long long r, long long rl, F64Ws& w) {
    const double* G64 = static_cast<const double*>(Gup->data);
    const double* X64 = static_cast<const double*>(X->data);
    const double* Y64 = static_cast<const double*>(Y->data);
    double* inner = w.inner;
    const size_t ib = w.inner_bytes;
    // S1 = G (Y^T A)^T (m x (r+l)), S2 = F^T G (r x n): the two contractions over G
    GN_TRY(dgemm(h, m, rl, n, 1.0, G64, Gup->ld, 0, w.YtA, n, 1, 0.0, w.S1, rl, inner, ib));
    GN_TRY(dgemm(h, r, n, m, 1.0, w.F, r, 1, G64, Gup->ld, 0, 0.0, w.S2, n, inner, ib));
    // W = F^T S1 (r x (r+l)); K1 = W^T R^{-T}; K1 -= Q (Q^T K1)
    GN_TRY(dgemm(h, r, rl, m, 1.0, w.F, r, 1, w.S1, rl, 0, 0.0, w.W, rl, inner, ib));
    GN_TRY(transpose_f64(h, w.W, r, rl, rl, w.K1, r));
    GN_TRY(trsm_right_upper(h, w.K1, rl, r, r, w.R, r, 1, inner, ib));
    GN_TRY(dgemm(h, r, r, rl, 1.0, w.Q, r, 1, w.K1, r, 0, 0.0, w.QtZ, r, inner, ib));
    GN_TRY(dgemm(h, rl, r, r, -1.0, w.Q, r, 0, w.QtZ, r, 0, 1.0, w.K1, r, inner, ib));
    // WQ = (W Q) R^{-T};  K = K1 - Q WQ   (stored in K1)
    GN_TRY(dgemm(h, r, r, rl, 1.0, w.W, rl, 0, w.Q, r, 0, 0.0, w.WQ, r, inner, ib));
    GN_TRY(trsm_right_upper(h, w.WQ, r, r, r, w.R, r, 1, inner, ib));
    GN_TRY(dgemm(h, rl, r, r, -1.0, w.Q, r, 0, w.WQ, r, 0, 1.0, w.K1, r, inner, ib));
    // P = (S1 Q) R^{-T} + Y K  (m x r);  Q' = Q S2 ((r+l) x n)
    GN_TRY(dgemm(h, m, r, rl, 1.0, w.S1, rl, 0, w.Q, r, 0, 0.0, w.P, r, inner, ib));
    GN_TRY(trsm_right_upper(h, w.P, m, r, r, w.R, r, 1, inner, ib));
    GN_TRY(dgemm(h, m, r, rl, 1.0, Y64, Y->ld, 0, w.K1, r, 0, 1.0, w.P, r, inner, ib));
    GN_TRY(dgemm(h, rl, n, r, 1.0, w.Q, r, 0, w.S2, n, 0, 0.0, w.Qp, n, inner, ib));
    // dA = P X^T + Y Q'
    double* dA64 = static_cast<double*>(dA->data);
    GN_TRY(dgemm(h, m, n, r, 1.0, w.P, r, 0, X64, X->ld, 1, 0.0, dA64, dA->ld, inner, ib));
    return dgemm(h, m, n, rl, 1.0, Y64, Y->ld, 0, w.Qp, n, 0, 1.0, dA64, dA->ld, inner, ib);
}

// The forward's own part: G = Q^T (Y^T A) (first r rows, in Qp), A_hat = F G.
gn_status f64_forward_rest(gn_handle h, gn_mat* Ahat, long long m, long long n, long long r, long long rl,
                           F64Ws& w) {
    GN_TRY(dgemm(h, r, n, rl, 1.0, w.Q, r, 1, w.YtA, n, 0, 0.0, w.Qp, n, w.inner, w.inner_bytes));
    return dgemm(h, m, n, r, 1.0, w.F, r, 0, w.Qp, n, 0, 0.0, static_cast<double*>(Ahat->data), Ahat->ld, w.inner,
                 w.inner_bytes);
}

}  // namespace
}  // namespace gn

using namespace gn;

extern "C" gn_status gn_backward_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l, int32_t dtype,
                                                size_t* bytes) {
    if (!bytes) return GN_ERR_INVALID_ARG;
    if (m <= 0 || n <= 0 || r < 1 || l < 1 || r > std::min(m, n) || r + l > m) return GN_ERR_SHAPE;
    if (dtype != GN_F64 && dtype != GN_F32) return GN_ERR_DTYPE;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dtype == GN_F32) {
        *bytes = tc_carve(m, n, r, l, sms, nullptr, nullptr);
        return GN_OK;
    }
    const size_t inner = std::max({qr_ws_bytes(r + l, r, sms), dgemm_ws_bytes(r + l, r, n, sms),
                                   dgemm_ws_bytes(r, r + l, m, sms), trsm_ws_bytes(m, r, sms),
                                   dgemm_ws_bytes(m, r, r + l, sms)});
    *bytes = backward_fixed(m, n, r, l) + inner;
    return GN_OK;
}

namespace {

// Shapes, leading dimensions and one shared dtype (FP64 or FP32) of the adjoint's
// matrices; FP32 operands also need 16-byte aligned data and ld % 4 == 0
// (tensor maps), except the last (an output written row by row).
gn_status check_adj(const gn_mat* const* mats, const long long (*shp)[2], int count, int dtype) {
    for (int i = 0; i < count; ++i) {
        if (!mats[i]->data) return GN_ERR_INVALID_ARG;
        if (mats[i]->rows != shp[i][0] || mats[i]->cols != shp[i][1]) return GN_ERR_SHAPE;
        if (mats[i]->ld < mats[i]->cols) return GN_ERR_INVALID_ARG;
        if (mats[i]->dtype != dtype) return GN_ERR_DTYPE;
    }
    if (dtype != GN_F32 && dtype != GN_F64) return GN_ERR_DTYPE;
    if (dtype == GN_F32)
        for (int i = 0; i < count; ++i)
            if ((reinterpret_cast<uintptr_t>(mats[i]->data) & 15) || (i < count - 1 && mats[i]->ld % 4))
                return GN_ERR_ALIGNMENT;
    return GN_OK;
}

void adj_record(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, const void* ws, size_t ws_bytes,
                long long m, long long n, long long r, long long l) {
    h->adj.valid = 1;
    h->adj.ws = ws;
    h->adj.ws_bytes = ws_bytes;
    h->adj.A = A->data;
    h->adj.X = X->data;
    h->adj.Y = Y->data;
    h->adj.m = m;
    h->adj.n = n;
    h->adj.r = r;
    h->adj.l = l;
    h->adj.lda = A->ld;
    h->adj.ldx = X->ld;
    h->adj.ldy = Y->ld;
    h->adj.dtype = A->dtype;
}

}  // namespace

extern "C" gn_status gn_backward(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, const gn_mat* Gup,
                                 gn_mat* dA, void* ws, size_t ws_bytes) {
    if (!h || !A || !X || !Y || !Gup || !dA || !ws) return GN_ERR_INVALID_ARG;
    const long long m = A->rows, n = A->cols, r = X->cols, rl = Y->cols, l = rl - r;
    if (m <= 0 || n <= 0 || r < 1 || l < 1 || r > std::min(m, n) || rl > m) return GN_ERR_SHAPE;
    const gn_mat* mats[5] = {A, X, Y, Gup, dA};
    const long long shp[5][2] = {{m, n}, {n, r}, {m, rl}, {m, n}, {m, n}};
    GN_TRY(check_adj(mats, shp, 5, A->dtype));
    size_t need = 0;
    GN_TRY(gn_backward_workspace_size(m, n, r, l, A->dtype, &need));
    if (ws_bytes < need) return GN_ERR_WORKSPACE;
    h->adj.valid = 0;
    if (A->dtype == GN_F32) {
        TcWs t;
        if (tc_carve(m, n, r, l, h->sm_count, static_cast<char*>(ws), &t) > ws_bytes) return GN_ERR_WORKSPACE;
        GN_TRY(tc_front(h, A, X, Y, m, n, r, rl, t));
        adj_record(h, A, X, Y, ws, ws_bytes, m, n, r, l);
        return tc_back(h, X, Y, Gup, dA, m, n, r, rl, t);
    }
    F64Ws w;
    if (!f64_carve(ws, ws_bytes, m, n, r, rl, &w)) return GN_ERR_WORKSPACE;
    GN_TRY(f64_front(h, A, X, Y, m, n, r, rl, w));
    adj_record(h, A, X, Y, ws, ws_bytes, m, n, r, l);
    return f64_back(h, X, Y, Gup, dA, m, n, r, rl, w);
}

// Forward value A_hat = F G of plain GN in the precision of A (for the autograd
// wrapper): A_hat (m x n) from A, X, Y.  The front stays in ws for
// gn_backward_saved.
extern "C" gn_status gn_forward_dense(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, gn_mat* Ahat,
                                      void* ws, size_t ws_bytes) {
    if (!h || !A || !X || !Y || !Ahat || !ws) return GN_ERR_INVALID_ARG;
    const long long m = A->rows, n = A->cols, r = X->cols, rl = Y->cols, l = rl - r;
    if (m <= 0 || n <= 0 || r < 1 || l < 1 || r > std::min(m, n) || rl > m) return GN_ERR_SHAPE;
    const gn_mat* mats[4] = {A, X, Y, Ahat};
    const long long shp[4][2] = {{m, n}, {n, r}, {m, rl}, {m, n}};
    GN_TRY(check_adj(mats, shp, 4, A->dtype));
    size_t need = 0;
    GN_TRY(gn_backward_workspace_size(m, n, r, l, A->dtype, &need));
    if (ws_bytes < need) return GN_ERR_WORKSPACE;
    h->adj.valid = 0;
    if (A->dtype == GN_F32) {
        TcWs t;
        if (tc_carve(m, n, r, l, h->sm_count, static_cast<char*>(ws), &t) > ws_bytes) return GN_ERR_WORKSPACE;
        GN_TRY(tc_front(h, A, X, Y, m, n, r, rl, t));
        adj_record(h, A, X, Y, ws, ws_bytes, m, n, r, l);
        return tc_forward_rest(h, Ahat, m, n, r, rl, t);
    }
    F64Ws w;
    if (!f64_carve(ws, ws_bytes, m, n, r, rl, &w)) return GN_ERR_WORKSPACE;
    GN_TRY(f64_front(h, A, X, Y, m, n, r, rl, w));
    adj_record(h, A, X, Y, ws, ws_bytes, m, n, r, l);
    return f64_forward_rest(h, Ahat, m, n, r, rl, w);
}

extern "C" gn_status gn_backward_saved(gn_handle h, const gn_mat* X, const gn_mat* Y, const gn_mat* Gup, gn_mat* dA,
                                       void* ws, size_t ws_bytes) {
    if (!h || !X || !Y || !Gup || !dA || !ws) return GN_ERR_INVALID_ARG;
    const long long m = Gup->rows, n = Gup->cols, r = X->cols, rl = Y->cols, l = rl - r;
    if (!h->adj.valid || h->adj.ws != ws || h->adj.ws_bytes != ws_bytes || h->adj.X != X->data ||
        h->adj.Y != Y->data || h->adj.ldx != X->ld || h->adj.ldy != Y->ld || h->adj.m != m || h->adj.n != n ||
        h->adj.r != r || h->adj.l != l || h->adj.dtype != Gup->dtype)
        return GN_ERR_INVALID_ARG;
    const gn_mat* mats[4] = {X, Y, Gup, dA};
    const long long shp[4][2] = {{n, r}, {m, rl}, {m, n}, {m, n}};
    GN_TRY(check_adj(mats, shp, 4, Gup->dtype));
    if (Gup->dtype == GN_F32) {
        TcWs t;
        if (tc_carve(m, n, r, l, h->sm_count, static_cast<char*>(ws), &t) > ws_bytes) return GN_ERR_WORKSPACE;
        return tc_back(h, X, Y, Gup, dA, m, n, r, rl, t);
    }
    F64Ws w;
    if (!f64_carve(ws, ws_bytes, m, n, r, rl, &w)) return GN_ERR_WORKSPACE;
    return f64_back(h, X, Y, Gup, dA, m, n, r, rl, w);
}

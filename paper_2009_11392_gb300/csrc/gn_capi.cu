// The C ABI of the library (include/gn.h): argument checks on the host, then
// the stream-ordered launch sequence of each call.  Nothing here computes: every
// step runs in the kernels of gn_tc.cu (tensor cores) and gn_f64.cu (FP64).
#include "gn_internal.cuh"

#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>

#include <atomic>

using namespace gn;

namespace gn {
static std::atomic<unsigned long long> g_launches{0};
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace gn

namespace {

constexpr int DIAG_ITERS = 6;

bool valid_dtype(int32_t d) { return d >= GN_F64 && d <= GN_BF16X2; }

long long tiles128(long long x) { return (x + 127) / 128; }

size_t elem_size(int32_t d) {
    switch (d) {
        case GN_F64: return 8;
        case GN_F32: return 4;
        default: return 2;
    }
}

// An e4m3 operand: scales and at least one orientation, TMA-aligned.
gn_status check_e4m3(const gn_mat* a, long long rows, long long cols, bool need_data, bool need_t) {
    if (!a) return GN_ERR_INVALID_ARG;
    if (a->dtype != GN_E4M3) return GN_ERR_DTYPE;
    if (a->rows != rows || a->cols != cols) return GN_ERR_SHAPE;
    if (!a->scale || (need_data && !a->data) || (need_t && !a->data_t) || (!a->data && !a->data_t))
        return GN_ERR_INVALID_ARG;
    if (a->data && ((reinterpret_cast<uintptr_t>(a->data) & 15) || a->ld < cols || a->ld % 16)) return GN_ERR_ALIGNMENT;
    if (a->data_t && ((reinterpret_cast<uintptr_t>(a->data_t) & 15) || a->ld_t < rows || a->ld_t % 16))
        return GN_ERR_ALIGNMENT;
    return GN_OK;
}

gn_status check_mat(const gn_mat* a, long long rows, long long cols) {
    if (!a || !a->data) return GN_ERR_INVALID_ARG;
    if (!valid_dtype(a->dtype)) return GN_ERR_DTYPE;
    if (a->rows != rows || a->cols != cols) return GN_ERR_SHAPE;
    if (a->ld < a->cols || a->ld <= 0) return GN_ERR_INVALID_ARG;
    if (a->dtype == GN_BF16X2 && !a->lo) return GN_ERR_INVALID_ARG;
    return GN_OK;
}

gn_status check_tma_operand(const gn_mat* a) {
    if ((reinterpret_cast<uintptr_t>(a->data) & 15) || (a->ld % 8)) return GN_ERR_ALIGNMENT;
    if (a->dtype == GN_BF16X2 && (reinterpret_cast<uintptr_t>(a->lo) & 15)) return GN_ERR_ALIGNMENT;
    return GN_OK;
}

gn_status check_sizes(long long m, long long n, long long r, long long l) {
    if (m <= 0 || n <= 0) return GN_ERR_SHAPE;
    if (r < 1 || r > std::min(m, n) || l < 1 || r + l > m) return GN_ERR_SHAPE;
    if (m > (1LL << 31) - 1 || n > (1LL << 31) - 1) return GN_ERR_SHAPE;
    return GN_OK;
}

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

// Bump allocator over the caller's workspace.
struct Carve {
    char* base;
    size_t cap;
    size_t off;
    bool ok;
    template <typename T>
    T* take(size_t count) {
        const size_t bytes = align256(count * sizeof(T));
        if (off + bytes > cap) {
            ok = false;
            return nullptr;
        }
        T* p = reinterpret_cast<T*>(base + off);
        off += bytes;
        return p;
    }
    double* rest(size_t* bytes) {
        const size_t o = align256(off);
        *bytes = o < cap ? cap - o : 0;
        return reinterpret_cast<double*>(base + o);
    }
};

long long round8(long long x) { return (x + 7) / 8 * 8; }

// ---------------------------------------------------------------- sizing helpers
size_t core_ws(long long n, long long r, long long l, int mixed, int sms) {
    const long long rl = r + l;
    size_t b = 0;
    b += align256(sizeof(double) * rl * r);            // W for the QR of C
    b += align256(sizeof(double) * r * r);             // W2 for the QR of R_1^T
    b += align256(sizeof(double) * 2 * std::max<long long>(r, 64));   // diag scratch
    b += 256;                                          // k, est
    if (mixed) {
        b += 3 * align256(sizeof(__nv_bfloat16) * rl * round8(n));
        b += 3 * align256(sizeof(float) * rl * r);
        b += align256(qr_oz_ws_bytes(rl, r));          // tensor-core formation of Q
    }
    size_t inner = std::max(qr_ws_bytes(rl, r, sms), dgemm_ws_bytes(rl, r, n, sms));
    if (mixed)   // FP64-level C (gn_set_fp64_accum): X in FP64 and the digit-sliced product's scratch
        inner = std::max(inner, align256(sizeof(double) * n * r) + oz_ws_bytes(rl, r, n, 1));
    return b + inner + 1024;
}

__global__ void bf16_to_f64_kernel(const __nv_bfloat16* __restrict__ s, long long rows, long long cols,
                                   long long lds, double* __restrict__ d, long long ldd) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e - i * cols;
        d[i * ldd + j] = static_cast<double>(__bfloat162float(s[i * lds + j]));
    }
}

// e4m3 sketch: the scale-factor images of A, X and Y (512 bytes per tile).
size_t sketch_e4m3_ws(long long m, long long n, long long r, long long l) {
    return align256(512 * static_cast<size_t>(tiles128(m) * tiles128(n))) +
           align256(512 * static_cast<size_t>(tiles128(n) * tiles128(r))) +
           align256(512 * static_cast<size_t>(tiles128(m) * tiles128(r + l))) + 1024;
}

// e4m3 X in the core product: an exact BF16 copy of X^T (r x n) ahead of the core workspace.
size_t core_e4m3_ws(long long n, long long r) { return align256(sizeof(__nv_bfloat16) * r * round8(n)) + 256; }

// Digit-sliced tensor-core FP64 products of the factors (FP32 AX): the solve's
// outer-block updates (N = 128, K < r) and AX Q_2 (FP32 A, N = k <= r, K = r).
size_t factors_oz_ws(long long m, long long r) {
    return std::max(oz_ws_bytes(m, 128, r, 0), oz_ws_bytes(m, r, r, 1));
}

// Factors: the FP64 solves' scratch, plus (FP32 Y^T A) the BF16 slices of Y^T A
// and Q_1 and the FP32 product G.
size_t factors_ws(long long m, long long n, long long r, long long l, int mixed, int sms) {
    size_t b = trsm_ws_bytes(m, r, sms) + dgemm_ws_bytes(m, r, r, sms) + 1024;
    if (mixed)
        b += 3 * align256(sizeof(__nv_bfloat16) * (r + l) * round8(n)) +
             3 * align256(sizeof(__nv_bfloat16) * (r + l) * round8(r)) + align256(sizeof(float) * r * round8(n)) +
             factors_oz_ws(m, r);
    return b;
}

size_t hmt_ws(long long m, long long n, long long r, int sms) {
    return align256(sizeof(double) * m * r) + align256(sizeof(double) * r * r) + qr_ws_bytes(m, r, sms) +
           dgemm_ws_bytes(r, n, m, sms) + 1024;
}

// FP64-level accumulation of split-BF16 sketches (gn_set_fp64_accum): the K
// range of each product runs as parts of about part_k elements, each
// accumulated in FP32 in tensor memory and stored, then summed in FP64.
int acc_parts(long long K, int nsrc, long long part_k) {
    const long long kel = nsrc * ((K + 63) / 64) * 64;
    return static_cast<int>(std::max<long long>(1, (kel + part_k - 1) / part_k));
}
long long round4(long long x) { return (x + 3) / 4 * 4; }
size_t split_parts_ws(long long m, long long n, long long r, long long rl, long long part_k) {
    return align256(4 * static_cast<size_t>(acc_parts(n, 2, part_k)) * m * round4(r)) +
           align256(4 * static_cast<size_t>(acc_parts(m, 2, part_k)) * rl * round4(n)) + 512;
}

__global__ void sum_parts_kernel(const float* __restrict__ parts, int nparts, long long stride, long long rows,
                                 long long cols, long long ldp, float* __restrict__ out, long long ldo) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e - i * cols;
        double s = 0.0;
        for (int c = 0; c < nparts; ++c) s += static_cast<double>(parts[c * stride + i * ldp + j]);
        out[i * ldo + j] = static_cast<float>(s);
    }
}

gn_status sum_parts(gn_handle h, const float* parts, int nparts, long long stride, long long rows, long long cols,
                    long long ldp, float* out, long long ldo) {
    const long long total = rows * cols;
    const int blocks = static_cast<int>(std::min<long long>((total + 255) / 256, 16LL * h->sm_count));
    sum_parts_kernel<<<blocks, 256, 0, h->stream>>>(parts, nparts, stride, rows, cols, ldp, out, ldo);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

gn_status launch_sketch_tc(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, gn_mat* AX,
                           gn_mat* YtA, void* ws, size_t ws_bytes) {
    const long long m = A->rows, n = A->cols, r = X->cols, rl = Y->cols;
    TcParams p;
    memset(&p, 0, sizeof(p));
    int nm = 0;
    const int mAk = nm++, mAmn = nm++;
    GN_TRY(tc_make_map_bf16(&p.maps[mAk], A->data, m, n, A->ld, 64, 128));
    GN_TRY(tc_make_map_bf16(&p.maps[mAmn], A->data, m, n, A->ld, 64, 64));
    int mLk = -1, mLmn = -1;
    const int nsrc = A->dtype == GN_BF16X2 ? 2 : 1;
    if (nsrc == 2) {
        mLk = nm++;
        mLmn = nm++;
        GN_TRY(tc_make_map_bf16(&p.maps[mLk], A->lo, m, n, A->ld, 64, 128));
        GN_TRY(tc_make_map_bf16(&p.maps[mLmn], A->lo, m, n, A->ld, 64, 64));
    }
    const int mX = nm++, mY = nm++;
    if (r > 0) GN_TRY(tc_make_map_bf16(&p.maps[mX], X->data, n, r, X->ld, 64, 64));
    if (rl > 0) GN_TRY(tc_make_map_bf16(&p.maps[mY], Y->data, m, rl, Y->ld, 64, 64));

    // GEMM 0: AX (m x r) = A (K-major) . X (MN-major), K = n
    TcGemm& g0 = p.g[0];
    g0.M = static_cast<int>(m);
    g0.N = static_cast<int>(r);
    g0.K = static_cast<int>(n);
    g0.bn = static_cast<int>(std::min<long long>(256, std::max<long long>(64, (r + 63) / 64 * 64)));
    g0.a_mn = 0;
    g0.b_mn = 1;
    g0.nsrc = nsrc;
    g0.a_map[0] = mAk;
    g0.b_map[0] = mX;
    if (nsrc == 2) {
        g0.a_map[1] = mLk;
        g0.b_map[1] = mX;
    }
    g0.D = static_cast<float*>(AX->data);
    g0.ldd = AX->ld;
    // GEMM 1: Y^T A ((r+l) x n) = Y^T (MN-major A operand) . A (MN-major B), K = m
    TcGemm& g1 = p.g[1];
    g1.M = static_cast<int>(rl);
    g1.N = static_cast<int>(n);
    g1.K = static_cast<int>(m);
    // Per-tile cost ~ bn * K.  When K = m is much longer than the other GEMM's,
    // the tiles keep bn = 256 (the fewest L2 bytes per flop) and run as two
    // half-K items each, so that every item costs about the same.
    g1.bn = 256;
    g1.ksplit = (2 * 256LL * m >= 3LL * g0.bn * n) ? 2 : 1;
    g1.a_mn = 1;
    g1.b_mn = 1;
    g1.nsrc = nsrc;
    g1.a_map[0] = mY;
    g1.b_map[0] = mAmn;
    if (nsrc == 2) {
        g1.a_map[1] = mY;
        g1.b_map[1] = mLmn;
    }
    g1.D = static_cast<float*>(YtA->data);
    g1.ldd = YtA->ld;
    // split-BF16 operands with FP64-level accumulation: stored K parts, summed in FP64
    float *pax = nullptr, *pyta = nullptr;
    int sax = 1, syta = 1;
    const long long ldpx = round4(r), ldpy = round4(n);
    if (nsrc == 2 && h->fp64_accum > 0) {
        const long long pk = h->fp64_accum;
        sax = acc_parts(n, 2, pk);
        syta = acc_parts(m, 2, pk);
        if (!ws || ws_bytes < split_parts_ws(m, n, r, rl, pk)) return GN_ERR_WORKSPACE;
        pax = static_cast<float*>(ws);
        pyta = reinterpret_cast<float*>(static_cast<char*>(ws) + align256(4 * static_cast<size_t>(sax) * m * ldpx));
        g0.D = pax;
        g0.ldd = ldpx;
        g0.ksplit = sax;
        g0.part_stride = m * ldpx;
        g1.D = pyta;
        g1.ldd = ldpy;
        g1.ksplit = syta;
        g1.part_stride = rl * ldpy;
        if (sax < 2) g0.ksplit = 0, g0.part_stride = 0;
        if (syta < 2) g1.ksplit = 0, g1.part_stride = 0;
    }
    auto finish = [&]() -> gn_status {
        if (!pax) return GN_OK;
        if (r > 0) GN_TRY(sum_parts(h, pax, sax, m * ldpx, m, r, ldpx, static_cast<float*>(AX->data), AX->ld));
        if (rl > 0) GN_TRY(sum_parts(h, pyta, syta, rl * ldpy, rl, n, ldpy, static_cast<float*>(YtA->data), YtA->ld));
        return GN_OK;
    };
    if (r == 0 || rl == 0) {   // a block sketch that needs one product only
        if (r == 0) p.g[0] = p.g[1];
        if (!pax) p.g[0].ksplit = 0;
        p.ngemm = 1;
        GN_TRY(tc_launch(h, &p));
        return finish();
    }
    // Order: the longer-K GEMM first (its tiles are the expensive ones).
    if (m >= n) {
        TcGemm t = p.g[0];
        p.g[0] = p.g[1];
        p.g[1] = t;
    }
    p.ngemm = 2;
    GN_TRY(tc_launch(h, &p));
    return finish();
}

// e4m3 sketch: both products from K-major operands in one block-scaled launch.
//   AX   = A (m x n) . (X^T)^T     : A operand A.data, B operand X.data_t (r x n)
//   Y^T A = (Y^T) . (A^T)^T        : A operand Y.data_t ((r+l) x m), B operand A.data_t (n x m)
gn_status launch_sketch_e4m3(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, gn_mat* AX,
                             gn_mat* YtA, void* ws, size_t ws_bytes) {
    const long long m = A->rows, n = A->cols, r = X->cols, rl = Y->cols;
    Carve cv{static_cast<char*>(ws), ws_bytes, 0, true};
    const long long tA = tiles128(m) * tiles128(n), tX = tiles128(n) * tiles128(r), tY = tiles128(m) * tiles128(rl);
    uint8_t* imA = cv.take<uint8_t>(512 * tA);
    uint8_t* imX = cv.take<uint8_t>(512 * tX);
    uint8_t* imY = cv.take<uint8_t>(512 * tY);
    if (!cv.ok) return GN_ERR_WORKSPACE;
    GN_TRY(e4m3_sf_image(h, A->scale, tA, imA));
    if (r > 0) GN_TRY(e4m3_sf_image(h, X->scale, tX, imX));
    if (rl > 0) GN_TRY(e4m3_sf_image(h, Y->scale, tY, imY));
    TcParams p;
    memset(&p, 0, sizeof(p));
    if (r > 0) {
        GN_TRY(tc_make_map_e4m3(&p.maps[0], A->data, m, n, A->ld, 128));
        GN_TRY(tc_make_map_e4m3(&p.maps[1], X->data_t, r, n, X->ld_t, 128));
    }
    if (rl > 0) {
        GN_TRY(tc_make_map_e4m3(&p.maps[2], Y->data_t, rl, m, Y->ld_t, 128));
        GN_TRY(tc_make_map_e4m3(&p.maps[3], A->data_t, n, m, A->ld_t, 128));
    }
    TcGemm& g0 = p.g[0];
    g0.M = static_cast<int>(m);
    g0.N = static_cast<int>(r);
    g0.K = static_cast<int>(n);
    g0.bn = 128;
    g0.nsrc = 1;
    g0.a_map[0] = 0;
    g0.b_map[0] = 1;
    g0.D = static_cast<float*>(AX->data);
    g0.ldd = AX->ld;
    g0.sfa = imA;                               // A tile (rb, kb): image (rb, kb)
    g0.sfa_ld = static_cast<int>(tiles128(n));
    g0.sfa_tr = 0;
    g0.sfa_rows = static_cast<int>(tiles128(m));
    g0.sfb = imX;                               // X^T tile (rb, kb) is X tile (kb, rb)
    g0.sfb_ld = static_cast<int>(tiles128(r));
    g0.sfb_tr = 1;
    g0.sfb_rows = static_cast<int>(tiles128(r));
    TcGemm& g1 = p.g[1];
    g1.M = static_cast<int>(rl);
    g1.N = static_cast<int>(n);
    g1.K = static_cast<int>(m);
    g1.bn = 128;
    g1.nsrc = 1;
    g1.a_map[0] = 2;
    g1.b_map[0] = 3;
    g1.D = static_cast<float*>(YtA->data);
    g1.ldd = YtA->ld;
    g1.sfa = imY;                               // Y^T tile (rb, kb) is Y tile (kb, rb)
    g1.sfa_ld = static_cast<int>(tiles128(rl));
    g1.sfa_tr = 1;
    g1.sfa_rows = static_cast<int>(tiles128(rl));
    g1.sfb = imA;                               // A^T tile (rb, kb) is A tile (kb, rb)
    g1.sfb_ld = static_cast<int>(tiles128(n));
    g1.sfb_tr = 1;
    g1.sfb_rows = static_cast<int>(tiles128(n));
    if (r == 0 || rl == 0) {   // a block sketch that needs one product only
        if (r == 0) p.g[0] = p.g[1];
        p.ngemm = 1;
        p.f8 = 1;
        return tc_launch(h, &p);
    }
    if (m >= n) {   // the longer-K GEMM first
        TcGemm t = p.g[0];
        p.g[0] = p.g[1];
        p.g[1] = t;
    }
    p.ngemm = 2;
    p.f8 = 1;
    return tc_launch(h, &p);
}

// dst (rows x cols, ldd) += src (rows x cols, lds), FP32 or FP64.
template <typename T>
__global__ void add_into_kernel(T* __restrict__ dst, long long ldd, const T* __restrict__ src, long long lds,
                                long long rows, long long cols) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / cols, j = e - i * cols;
        dst[i * ldd + j] += src[i * lds + j];
    }
}

gn_status add_into(gn_handle h, gn_mat* dst, const void* src, long long lds) {
    const long long total = dst->rows * dst->cols;
    const int blocks = static_cast<int>(std::min<long long>((total + 255) / 256, 16LL * h->sm_count));
    if (dst->dtype == GN_F32)
        add_into_kernel<float><<<blocks, 256, 0, h->stream>>>(static_cast<float*>(dst->data), dst->ld,
                                                              static_cast<const float*>(src), lds, dst->rows,
                                                              dst->cols);
    else
        add_into_kernel<double><<<blocks, 256, 0, h->stream>>>(static_cast<double*>(dst->data), dst->ld,
                                                               static_cast<const double*>(src), lds, dst->rows,
                                                               dst->cols);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

size_t update_scratch(long long m, long long n, long long r, long long l, int op_dtype) {
    const size_t es = op_dtype == GN_F64 ? sizeof(double) : sizeof(float);
    return align256(es * m * round8(r)) + align256(es * (r + l) * round8(n)) + 512;
}

// Scratch of sketch_block for an m x n block with rx = X's and ry = Y's columns.
size_t block_sketch_ws(long long m, long long n, long long rx, long long ry, int op_dtype, int sms) {
    if (op_dtype == GN_E4M3) return sketch_e4m3_ws(m, n, rx, ry - rx);
    if (op_dtype == GN_F64) return std::max(dgemm_ws_bytes(m, rx, n, sms), dgemm_ws_bytes(ry, n, m, sms)) + 1024;
    return 1024;
}

// The sketch products A X (m x rx) and Y^T A (ry x n) of any block A (m, n >= 1);
// either product may be absent (rx == 0 or ry == 0: that operand and its output
// are not read).  gn_sketch adds GN's own size rules on top (r <= min(m, n),
// l >= 1); the sketch-state calls of Section 6 sketch blocks of any size.
gn_status sketch_block(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, gn_mat* AX, gn_mat* YtA,
                       void* ws, size_t ws_bytes) {
    if (!h || !A || !X || !Y || !AX || !YtA) return GN_ERR_INVALID_ARG;
    const long long m = A->rows, n = A->cols, r = X->cols, rl = Y->cols;
    if (m < 1 || n < 1 || r < 0 || rl < 0 || r + rl < 1) return GN_ERR_SHAPE;
    if (m > (1LL << 31) - 1 || n > (1LL << 31) - 1 || r > (1LL << 31) - 1 || rl > (1LL << 31) - 1)
        return GN_ERR_SHAPE;
    if (X->rows != n || Y->rows != m) return GN_ERR_SHAPE;
    if (A->dtype == GN_E4M3) {
        GN_TRY(check_e4m3(A, m, n, r > 0, rl > 0));
        if (r > 0) {
            GN_TRY(check_e4m3(X, n, r, false, true));
            GN_TRY(check_mat(AX, m, r));
            if (AX->dtype != GN_F32) return GN_ERR_DTYPE;
        }
        if (rl > 0) {
            GN_TRY(check_e4m3(Y, m, rl, false, true));
            GN_TRY(check_mat(YtA, rl, n));
            if (YtA->dtype != GN_F32) return GN_ERR_DTYPE;
        }
        if (!ws || ws_bytes < sketch_e4m3_ws(m, n, r, rl - r)) return GN_ERR_WORKSPACE;
        return launch_sketch_e4m3(h, A, X, Y, AX, YtA, ws, ws_bytes);
    }
    GN_TRY(check_mat(A, m, n));
    if (r > 0) {
        GN_TRY(check_mat(X, n, r));
        GN_TRY(check_mat(AX, m, r));
    }
    if (rl > 0) {
        GN_TRY(check_mat(Y, m, rl));
        GN_TRY(check_mat(YtA, rl, n));
    }
    if (A->dtype == GN_F64) {
        if ((r > 0 && (X->dtype != GN_F64 || AX->dtype != GN_F64)) ||
            (rl > 0 && (Y->dtype != GN_F64 || YtA->dtype != GN_F64)))
            return GN_ERR_DTYPE;
        double* gws = static_cast<double*>(ws);
        if (r > 0)
            GN_TRY(dgemm(h, m, r, n, 1.0, static_cast<const double*>(A->data), A->ld, 0,
                         static_cast<const double*>(X->data), X->ld, 0, 0.0, static_cast<double*>(AX->data),
                         AX->ld, gws, ws_bytes));
        if (rl > 0)
            GN_TRY(dgemm(h, rl, n, m, 1.0, static_cast<const double*>(Y->data), Y->ld, 1,
                         static_cast<const double*>(A->data), A->ld, 0, 0.0, static_cast<double*>(YtA->data),
                         YtA->ld, gws, ws_bytes));
        return GN_OK;
    }
    if (A->dtype == GN_BF16 || A->dtype == GN_BF16X2) {
        if ((r > 0 && (X->dtype != GN_BF16 || AX->dtype != GN_F32)) ||
            (rl > 0 && (Y->dtype != GN_BF16 || YtA->dtype != GN_F32)))
            return GN_ERR_DTYPE;
        GN_TRY(check_tma_operand(A));
        if (r > 0) GN_TRY(check_tma_operand(X));
        if (rl > 0) GN_TRY(check_tma_operand(Y));
        return launch_sketch_tc(h, A, X, Y, AX, YtA, ws, ws_bytes);
    }
    return GN_ERR_DTYPE;
}

}  // namespace

// ============================================================================ API
extern "C" {

const char* gn_status_string(gn_status s) {
    switch (s) {
        case GN_OK: return "ok";
        case GN_ERR_INVALID_ARG: return "invalid argument";
        case GN_ERR_SHAPE: return "invalid shape";
        case GN_ERR_DTYPE: return "unsupported dtype combination";
        case GN_ERR_WORKSPACE: return "workspace too small";
        case GN_ERR_CUDA: return "CUDA error";
        case GN_ERR_NONFINITE: return "non-finite value in the core";
        case GN_ERR_TIMEOUT: return "device-side wait timed out";
        case GN_ERR_UNSUPPORTED: return "unsupported request";
        case GN_ERR_ALIGNMENT: return "operand breaks a TMA alignment rule";
    }
    return "unknown status";
}

gn_status gn_create(gn_handle* out, void* stream) {
    if (!out) return GN_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GN_ERR_CUDA;
    int sms = 0;
    GN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    gn_handle h = new (std::nothrow) gn_handle_s;
    if (!h) return GN_ERR_INVALID_ARG;
    h->device = dev;
    h->sm_count = sms;
    h->stream = static_cast<cudaStream_t>(stream);
    h->wait_limit_ns = 2000000000ULL;
    h->batched_ws = nullptr;
    h->batched_count = h->batched_sk_tiles = h->batched_c_tiles = 0;
    h->batched_mt = 1;
    h->batched_policy = 0;
    h->fp64_g = 0;
    h->fp64_tc = 1;
    h->fp64_accum = 0;
    h->stall_test = 0;
    h->adj.valid = 0;
    if (cudaMalloc(&h->dstatus, 64) != cudaSuccess) {
        delete h;
        return GN_ERR_CUDA;
    }
    if (cudaMemsetAsync(h->dstatus, 0, 64, h->stream) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(h->dstatus);
        delete h;
        return GN_ERR_CUDA;
    }
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->crit, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
        cudaStreamDestroy(h->side);
        cudaFree(h->dstatus);
        delete h;
        return GN_ERR_CUDA;
    }
    h->pend.active = 0;
    void* pin = nullptr;
    if (cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_crit0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_crit1, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_defer, cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc(&pin, 64, cudaHostAllocDefault) != cudaSuccess) {
        cudaStreamDestroy(h->crit);
        cudaStreamDestroy(h->side);
        cudaFree(h->dstatus);
        delete h;
        return GN_ERR_CUDA;
    }
    h->pin_diag = static_cast<double*>(pin);
    h->pin_k = reinterpret_cast<int32_t*>(h->pin_diag + 4);
    *out = h;
    return GN_OK;
}

gn_status gn_destroy(gn_handle h) {
    if (!h) return GN_ERR_INVALID_ARG;
    cudaStreamSynchronize(h->stream);
    cudaStreamSynchronize(h->side);
    cudaStreamSynchronize(h->crit);
    cudaEventDestroy(h->ev_fork);
    cudaEventDestroy(h->ev_join);
    cudaEventDestroy(h->ev_crit0);
    cudaEventDestroy(h->ev_crit1);
    cudaEventDestroy(h->ev_defer);
    cudaFreeHost(h->pin_diag);
    cudaStreamDestroy(h->crit);
    cudaStreamDestroy(h->side);
    cudaFree(h->dstatus);
    delete h;
    return GN_OK;
}

gn_status gn_set_stream(gn_handle h, void* stream) {
    if (!h) return GN_ERR_INVALID_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return GN_OK;
}

gn_status gn_set_fp64_g(gn_handle h, int32_t fp64_g) {
    if (!h || (fp64_g != 0 && fp64_g != 1)) return GN_ERR_INVALID_ARG;
    h->fp64_g = fp64_g;
    return GN_OK;
}

gn_status gn_set_fp64_accum(gn_handle h, int64_t part_k) {
    if (!h || (part_k != 0 && (part_k < 4096 || part_k % 64))) return GN_ERR_INVALID_ARG;
    h->fp64_accum = part_k;
    return GN_OK;
}

gn_status gn_set_fp64_tc(gn_handle h, int32_t on) {
    if (!h || (on != 0 && on != 1)) return GN_ERR_INVALID_ARG;
    h->fp64_tc = on;
    return GN_OK;
}

gn_status gn_dgemm_tc_workspace_size(int64_t M, int64_t N, int64_t K, int32_t a_f32, size_t* bytes) {
    if (!bytes || M < 0 || N < 0 || K < 1) return GN_ERR_INVALID_ARG;
    *bytes = oz_ws_bytes(M, N, K, a_f32 ? 1 : 0);
    return GN_OK;
}

gn_status gn_dgemm_tc(gn_handle h, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int32_t a_f32,
                      int64_t lda, int32_t ta, const double* B, int64_t ldb, int32_t tb, double beta, double* C,
                      int64_t ldc, void* ws, size_t ws_bytes) {
    if (!h || M < 0 || N < 0 || K < 1 || !A || !B || !C || !ws) return GN_ERR_INVALID_ARG;
    if (lda < (ta ? M : K) || ldb < (tb ? K : N) || ldc < N) return GN_ERR_SHAPE;
    if (reinterpret_cast<uintptr_t>(ws) & 255) return GN_ERR_ALIGNMENT;
    if (ws_bytes < oz_ws_bytes(M, N, K, a_f32 ? 1 : 0)) return GN_ERR_WORKSPACE;
    return oz_dgemm(h, M, N, K, alpha, A, a_f32 ? 1 : 0, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, beta, C, ldc, ws,
                    ws_bytes);
}

gn_status gn_set_wait_limit(gn_handle h, uint64_t ns) {
    if (!h || ns == 0) return GN_ERR_INVALID_ARG;
    h->wait_limit_ns = ns;
    return GN_OK;
}

gn_status gn_set_stall_test(gn_handle h, int32_t on) {
    if (!h || (on != 0 && on != 1)) return GN_ERR_INVALID_ARG;
    h->stall_test = on;
    return GN_OK;
}

int gn_device_sm_count(gn_handle h) { return h ? h->sm_count : 0; }

uint64_t gn_kernel_launches(void) { return launch_count(); }

gn_status gn_sync_status(gn_handle h) {
    if (!h) return GN_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return GN_ERR_CUDA;
    int32_t st[2] = {0, 0};
    GN_CUDA_TRY(cudaMemcpy(st, h->dstatus, sizeof(st), cudaMemcpyDeviceToHost));
    if (st[0] != 0) GN_CUDA_TRY(cudaMemset(h->dstatus, 0, 64));
    return static_cast<gn_status>(st[0]);
}

gn_status gn_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l, int32_t op_dtype, size_t* bytes) {
    if (!bytes) return GN_ERR_INVALID_ARG;
    GN_TRY(check_sizes(m, n, r, l));
    if (op_dtype != GN_F64 && op_dtype != GN_BF16 && op_dtype != GN_BF16X2 && op_dtype != GN_E4M3)
        return GN_ERR_DTYPE;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int mixed = op_dtype != GN_F64;
    size_t b = core_ws(n, r, l, mixed, sms) + (op_dtype == GN_E4M3 ? core_e4m3_ws(n, r) : 0);
    if (op_dtype == GN_BF16X2) b = std::max(b, split_parts_ws(m, n, r, r + l, 4096));
    if (op_dtype == GN_E4M3) b = std::max(b, sketch_e4m3_ws(m, n, r, l));
    b = std::max(b, factors_ws(m, n, r, l, mixed, sms));
    b = std::max(b, hmt_ws(m, n, r, sms));
    b = std::max(b, error_ws_bytes(m, n, sms));
    *bytes = b;
    return GN_OK;
}

gn_status gn_quantize(gn_handle h, const gn_mat* src, gn_mat* dst) {
    if (!h || !src || !dst) return GN_ERR_INVALID_ARG;
    GN_TRY(check_mat(src, src->rows, src->cols));
    if (dst->dtype == GN_E4M3) {
        if (src->dtype != GN_F64 && src->dtype != GN_F32) return GN_ERR_DTYPE;
        GN_TRY(check_e4m3(dst, src->rows, src->cols, false, false));
        return quantize_e4m3(h, src->data, src->dtype == GN_F64, src->rows, src->cols, src->ld,
                             static_cast<uint8_t*>(dst->data), dst->ld, static_cast<uint8_t*>(dst->data_t),
                             dst->ld_t, dst->scale);
    }
    GN_TRY(check_mat(dst, src->rows, src->cols));
    if (src->dtype != GN_F64 && src->dtype != GN_F32) return GN_ERR_DTYPE;
    if (dst->dtype != GN_BF16 && dst->dtype != GN_BF16X2) return GN_ERR_DTYPE;
    GN_TRY(check_tma_operand(dst));
    return quantize_bf16(h, src->data, src->dtype == GN_F64, src->rows, src->cols, src->ld,
                         static_cast<__nv_bfloat16*>(dst->data),
                         dst->dtype == GN_BF16X2 ? static_cast<__nv_bfloat16*>(dst->lo) : nullptr, dst->ld);
}

gn_status gn_sketch(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, gn_mat* AX,
                    gn_mat* YtA, void* ws, size_t ws_bytes) {
    if (!h || !A || !X || !Y || !AX || !YtA) return GN_ERR_INVALID_ARG;
    GN_TRY(check_sizes(A->rows, A->cols, X->cols, Y->cols - X->cols));
    return sketch_block(h, A, X, Y, AX, YtA, ws, ws_bytes);
}

gn_status gn_core(gn_handle h, const gn_mat* YtA, const gn_mat* X, double eps, int32_t mode,
                  gn_core_t* core, void* ws, size_t ws_bytes) {
    if (!h || !YtA || !X || !core || !ws) return GN_ERR_INVALID_ARG;
    const int eps_rel = (mode & GN_EPS_RELATIVE) ? 1 : 0;
    const int defer = (mode & GN_CORE_DEFER) ? 1 : 0;
    const int c_given = (mode & GN_CORE_C_GIVEN) ? 1 : 0;
    mode &= ~(GN_EPS_RELATIVE | GN_CORE_DEFER | GN_CORE_C_GIVEN);
    if (mode < GN_MODE_PLAIN || mode > GN_MODE_AUTO || !(eps >= 0.0)) return GN_ERR_INVALID_ARG;
    if (defer && h->pend.active) return GN_ERR_INVALID_ARG;   // finish the pending core first
    const long long n = X->rows, r = X->cols, rl = YtA->rows, l = rl - r;
    if (r < 1 || l < 1 || n < r) return GN_ERR_SHAPE;
    GN_TRY(check_mat(YtA, rl, n));
    const int x8 = X->dtype == GN_E4M3;
    if (c_given) {   // X gives the shapes and the path only; its data is not read
        if (X->dtype != YtA->dtype && !(YtA->dtype == GN_F32 && X->dtype == GN_BF16) && !x8) return GN_ERR_DTYPE;
    } else if (x8) {
        GN_TRY(check_e4m3(X, n, r, false, true));
    } else {
        GN_TRY(check_mat(X, n, r));
    }
    if (!core->Q || !core->R || !core->C || ((mode != GN_MODE_PLAIN) && (!core->Q2 || !core->R2)))
        return GN_ERR_INVALID_ARG;
    const int mixed = (YtA->dtype == GN_F32 && (X->dtype == GN_BF16 || x8));
    const int fp64 = (YtA->dtype == GN_F64 && X->dtype == GN_F64);
    if (!mixed && !fp64) return GN_ERR_DTYPE;
    // e4m3 X: its exact BF16 transpose (r x n) takes the front of the workspace
    __nv_bfloat16* xt16 = nullptr;
    const long long ldx16 = round8(n);
    if (x8) {
        const size_t front = core_e4m3_ws(n, r);
        if (ws_bytes < front) return GN_ERR_WORKSPACE;
        xt16 = static_cast<__nv_bfloat16*>(ws);
        ws = static_cast<char*>(ws) + front;
        ws_bytes -= front;
    }
    if (ws_bytes < core_ws(n, r, l, mixed, h->sm_count)) return GN_ERR_WORKSPACE;
    core->r = r;
    core->l = l;

    Carve cv{static_cast<char*>(ws), ws_bytes, 0, true};
    double* W = cv.take<double>(rl * r);
    double* W2 = cv.take<double>(r * r);
    double* zscr = cv.take<double>(2 * std::max<long long>(r, 64));
    double* diag_d = cv.take<double>(3);
    int* k_d = cv.take<int>(1);
    __nv_bfloat16 *s_hi = nullptr, *s_mid = nullptr, *s_lo = nullptr;
    float *c_hi = nullptr, *c_mid = nullptr, *c_lo = nullptr;
    const long long lds = round8(n);
    if (mixed) {
        s_hi = cv.take<__nv_bfloat16>(rl * lds);
        s_mid = cv.take<__nv_bfloat16>(rl * lds);
        s_lo = cv.take<__nv_bfloat16>(rl * lds);
        c_hi = cv.take<float>(rl * r);
        c_mid = cv.take<float>(rl * r);
        c_lo = cv.take<float>(rl * r);
    }
    // FP32 sketches: Q formed with its large products on the tensor cores
    void* qoz = nullptr;
    size_t qoz_bytes = 0;
    if (mixed && h->fp64_tc) {
        qoz_bytes = qr_oz_ws_bytes(rl, r);
        qoz = cv.take<char>(qoz_bytes);
    }
    size_t inner_bytes = 0;
    double* inner = cv.rest(&inner_bytes);
    if (!cv.ok) return GN_ERR_WORKSPACE;

    // C = (Y^T A) X  ((r+l) x r, FP64, ld = r)
    if (c_given) {
        // the caller formed C (for a structured X, e.g. gn_countsketch_apply)
    } else if (fp64) {
        GN_TRY(dgemm(h, rl, r, n, 1.0, static_cast<const double*>(YtA->data), YtA->ld, 0,
                     static_cast<const double*>(X->data), X->ld, 0, 0.0, core->C, r, inner, inner_bytes));
    } else if (h->fp64_accum && !x8) {
        // FP64-level C: (Y^T A) X by exact digit slicing on the tensor cores
        double* X64 = inner;
        const size_t xb = align256(sizeof(double) * n * r);
        const long long total = n * r;
        bf16_to_f64_kernel<<<static_cast<int>(std::min<long long>((total + 255) / 256, 16LL * h->sm_count)), 256, 0,
                             h->stream>>>(static_cast<const __nv_bfloat16*>(X->data), n, r, X->ld, X64, r);
        count_launch();
        GN_CUDA_TRY(cudaGetLastError());
        GN_TRY(oz_dgemm(h, rl, r, n, 1.0, YtA->data, 1, YtA->ld, 0, X64, r, 0, 0.0, core->C, r,
                        reinterpret_cast<char*>(inner) + xb, inner_bytes - xb));
    } else {
        if (!x8) GN_TRY(check_tma_operand(X));
        GN_TRY(split3_bf16(h, static_cast<const float*>(YtA->data), rl, n, YtA->ld, s_hi, s_mid, s_lo, lds));
        TcParams p;
        memset(&p, 0, sizeof(p));
        __nv_bfloat16* sl[3] = {s_hi, s_mid, s_lo};
        float* cl[3] = {c_hi, c_mid, c_lo};
        for (int s = 0; s < 3; ++s) GN_TRY(tc_make_map_bf16(&p.maps[s], sl[s], rl, n, lds, 64, 128));
        if (x8) {   // X^T in BF16 as a K-major B operand
            GN_TRY(e4m3_t_to_bf16(h, static_cast<const uint8_t*>(X->data_t), X->ld_t, X->scale, n, r, xt16, ldx16));
            GN_TRY(tc_make_map_bf16(&p.maps[3], xt16, r, n, ldx16, 64, static_cast<int>(std::min<long long>(256, (r + 63) / 64 * 64))));
        } else {
            GN_TRY(tc_make_map_bf16(&p.maps[3], X->data, n, r, X->ld, 64, 64));
        }
        for (int s = 0; s < 3; ++s) {
            TcGemm& g = p.g[s];
            g.M = static_cast<int>(rl);
            g.N = static_cast<int>(r);
            g.K = static_cast<int>(n);
            g.bn = static_cast<int>(std::min<long long>(256, (r + 63) / 64 * 64));
            g.a_mn = 0;
            g.b_mn = x8 ? 0 : 1;
            g.nsrc = 1;
            g.a_map[0] = s;
            g.b_map[0] = 3;
            g.D = cl[s];
            g.ldd = r;
        }
        p.ngemm = 3;
        GN_TRY(tc_launch(h, &p));
        GN_TRY(sum3_f32_to_f64(h, c_hi, c_mid, c_lo, rl, r, r, core->C, r));
    }
    // Householder QR of a copy of C: factor (R), then the thin Q.  In SGN / AUTO
    // mode the Section 5.1.1/5.1.2 diagnostics on R run on the side stream
    // while the main stream forms Q.
    GN_CUDA_TRY(cudaMemcpy2DAsync(W, r * sizeof(double), core->C, r * sizeof(double), r * sizeof(double), rl,
                                  cudaMemcpyDeviceToDevice, h->stream));
    GN_TRY(qr_factor(h, W, rl, r, r, core->R, r, inner, inner_bytes, qoz, qoz_bytes));
    core->k = r;
    core->sgn = 0;
    core->rinv_est = 0.0;
    core->c_norm_est = 0.0;
    core->eps_abs = eps;
    if (mode == GN_MODE_PLAIN) {
        GN_TRY(latch_nonfinite_upper(h, core->R, r, r));
        return qr_form_q(h, W, rl, r, r, core->Q, r, inner, inner_bytes, qoz, qoz_bytes);
    }

    GN_CUDA_TRY(cudaEventRecord(h->ev_fork, h->stream));
    GN_CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    {
        gn_handle_s side = *h;
        side.stream = h->side;
        GN_TRY(latch_nonfinite_upper(&side, core->R, r, r));
        GN_TRY(core_diagnostics(&side, core->R, r, r, eps, eps_rel, 1, DIAG_ITERS, diag_d, k_d, zscr,
                                sizeof(double) * 2 * std::max<long long>(r, 64)));
        // k and the three diagnostics to the pinned host words as soon as they exist
        GN_CUDA_TRY(cudaMemcpyAsync(h->pin_k, k_d, sizeof(int32_t), cudaMemcpyDeviceToHost, h->side));
        GN_CUDA_TRY(cudaMemcpyAsync(h->pin_diag, diag_d, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->side));
        GN_CUDA_TRY(cudaEventRecord(h->ev_defer, h->side));
    }
    GN_CUDA_TRY(cudaEventRecord(h->ev_join, h->side));
    GN_TRY(qr_form_q(h, W, rl, r, r, core->Q, r, inner, inner_bytes, qoz, qoz_bytes));
    GN_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    h->pend.active = 1;
    h->pend.mode = mode;
    h->pend.r = r;
    h->pend.R = core->R;
    h->pend.Q2 = core->Q2;
    h->pend.R2 = core->R2;
    h->pend.W2 = W2;
    h->pend.inner = inner;
    h->pend.inner_bytes = inner_bytes;
    if (defer) {   // the host fields arrive with gn_core_finish
        core->k = -1;
        core->sgn = -1;
        return GN_OK;
    }
    return gn_core_finish(h, core);
}

gn_status gn_core_finish(gn_handle h, gn_core_t* core) {
    if (!h || !core) return GN_ERR_INVALID_ARG;
    if (!h->pend.active) return core->k >= 1 ? GN_OK : GN_ERR_INVALID_ARG;   // nothing pending
    if (core->R != h->pend.R) return GN_ERR_INVALID_ARG;                     // another core is pending
    h->pend.active = 0;
    // Waits for the diagnostics only (the side stream), not for the formation of Q.
    GN_CUDA_TRY(cudaEventSynchronize(h->ev_defer));
    const long long r = h->pend.r;
    const int mode = h->pend.mode;
    const long long k_h = *h->pin_k;
    const double diag_h[3] = {h->pin_diag[0], h->pin_diag[1], h->pin_diag[2]};
    core->k = r;
    core->sgn = 0;
    core->rinv_est = diag_h[0];
    core->c_norm_est = diag_h[1];
    core->eps_abs = diag_h[2];
    // A NaN in the core makes the estimates NaN (an exactly zero pivot makes the
    // estimate of ||R^{-1}|| infinite, which is the SGN branch, not an error).
    if (std::isnan(diag_h[0]) || std::isnan(diag_h[1]) || std::isnan(diag_h[2])) return GN_ERR_NONFINITE;
    // Section 5.1.2: switch when ||R^{-1}|| >> 1/u in the paper's normalisation,
    // where eps = 10u; ">>" read as a factor 10, i.e. est * eps >= 100.
    const int use_sgn = (mode == GN_MODE_SGN) || (diag_h[2] > 0.0 && diag_h[0] * diag_h[2] >= 100.0);
    core->sgn = use_sgn;
    if (!use_sgn) return GN_OK;
    core->k = k_h;
    if (k_h >= r) return GN_OK;
    if (k_h == 0) return GN_ERR_NONFINITE;   // every |R_ii| <= eps: nothing left of the core
    // Section 5.1.1: QR of R_1^T (r x k), R_1 = R[0:k, :].
    GN_TRY(transpose_rows_f64(h, core->R, k_h, r, r, k_h, h->pend.W2, k_h));
    GN_TRY(householder_qr(h, h->pend.W2, r, k_h, k_h, core->Q2, r, core->R2, r, h->pend.inner,
                          h->pend.inner_bytes));
    return GN_OK;
}

gn_status gn_factors(gn_handle h, const gn_mat* AX, const gn_mat* YtA, const gn_core_t* core, gn_mat* F,
                     gn_mat* G, void* ws, size_t ws_bytes) {
    if (!h || !AX || !YtA || !core || !F || !G || !ws) return GN_ERR_INVALID_ARG;
    const long long m = AX->rows, r = core->r, l = core->l, k = core->k, n = YtA->cols;
    if (k < 1 || k > r) return GN_ERR_INVALID_ARG;
    GN_TRY(check_mat(AX, m, r));
    GN_TRY(check_mat(YtA, r + l, n));
    if (!F->data || !G->data || F->dtype != GN_F64 || G->dtype != GN_F64) return GN_ERR_DTYPE;
    if (F->rows != m || F->cols < k || G->rows < k || G->cols != n || F->ld < F->cols || G->ld < n)
        return GN_ERR_SHAPE;
    if (AX->dtype != GN_F64 && AX->dtype != GN_F32) return GN_ERR_DTYPE;
    if (YtA->dtype != GN_F64 && YtA->dtype != GN_F32) return GN_ERR_DTYPE;
    const int tc_g = YtA->dtype == GN_F32 && !h->fp64_g && !h->fp64_accum;
    const int mixed = AX->dtype == GN_F32 || YtA->dtype == GN_F32;
    if (ws_bytes < factors_ws(m, n, r, l, mixed, h->sm_count)) return GN_ERR_WORKSPACE;
    double* Fd = static_cast<double*>(F->data);
    double* Gd = static_cast<double*>(G->data);
    // FP32 Y^T A: G = Q_1^T (Y^T A) on the tensor cores from three BF16 slices of
    // each factor (the six slice products of order <= 2: FP32-level accuracy,
    // below the sketch's own error); the FP64 path keeps an FP64 product.
    Carve cv{static_cast<char*>(ws), ws_bytes, 0, true};
    const long long rl = r + l, lds = round8(n), ldq = round8(k);
    __nv_bfloat16 *sl[3] = {nullptr, nullptr, nullptr}, *ql[3] = {nullptr, nullptr, nullptr};
    float* g32 = nullptr;
    // FP32 AX: the solve's large products on the tensor cores (digit slicing)
    const bool oz_on = AX->dtype == GN_F32 && h->fp64_tc && m >= 1024;
    void* oz = nullptr;
    const size_t oz_bytes = oz_on ? factors_oz_ws(m, r) : 0;
    if (tc_g) {
        for (int i = 0; i < 3; ++i) sl[i] = cv.take<__nv_bfloat16>(rl * lds);
        for (int i = 0; i < 3; ++i) ql[i] = cv.take<__nv_bfloat16>(rl * ldq);
        g32 = cv.take<float>(k * lds);
        if (!cv.ok) return GN_ERR_WORKSPACE;
    }
    if (oz_on) {
        oz = cv.take<char>(oz_bytes);
        if (!cv.ok) return GN_ERR_WORKSPACE;
    }
    size_t gws_bytes = 0;
    double* gws = cv.rest(&gws_bytes);
    ws_bytes = gws_bytes;
    const bool truncated = core->sgn && k < r;
    if (!truncated) {
        // F = AX R^{-1}
        if (AX->dtype == GN_F32) {
            GN_TRY(copy_f32_to_f64(h, static_cast<const float*>(AX->data), m, r, AX->ld, Fd, F->ld));
        } else {
            GN_CUDA_TRY(cudaMemcpy2DAsync(Fd, F->ld * 8, AX->data, AX->ld * 8, r * 8, m, cudaMemcpyDeviceToDevice,
                                          h->stream));
        }
        GN_TRY(trsm_right_upper(h, Fd, m, r, F->ld, core->R, r, 0, gws, ws_bytes, oz, oz_bytes));
    } else {
        // F = (AX Q_2) R_2^{-T}
        if (oz)
            GN_TRY(oz_dgemm(h, m, k, r, 1.0, AX->data, 1, AX->ld, 0, core->Q2, r, 0, 0.0, Fd, F->ld, oz, oz_bytes));
        else if (AX->dtype == GN_F32)
            GN_TRY(dgemm_a32(h, m, k, r, 1.0, static_cast<const float*>(AX->data), AX->ld, 0, core->Q2, r, 0,
                             0.0, Fd, F->ld, gws, ws_bytes));
        else
            GN_TRY(dgemm(h, m, k, r, 1.0, static_cast<const double*>(AX->data), AX->ld, 0, core->Q2, r, 0, 0.0,
                         Fd, F->ld, gws, ws_bytes));
        GN_TRY(trsm_right_upper(h, Fd, m, k, F->ld, core->R2, r, 1, gws, ws_bytes, oz, oz_bytes));
    }
    // G = Q_1^T (Y^T A)
    if (YtA->dtype == GN_F32 && !tc_g) {
        GN_TRY(dgemm_b32(h, k, n, r + l, 1.0, core->Q, r, 1, static_cast<const float*>(YtA->data), YtA->ld, 0,
                         0.0, Gd, G->ld, gws, ws_bytes));
    } else if (tc_g) {
        GN_TRY(split3_bf16(h, static_cast<const float*>(YtA->data), rl, n, YtA->ld, sl[0], sl[1], sl[2], lds));
        GN_TRY(split3_f64_bf16(h, core->Q, rl, k, r, ql[0], ql[1], ql[2], ldq));
        TcParams p;
        memset(&p, 0, sizeof(p));
        for (int i = 0; i < 3; ++i) {
            GN_TRY(tc_make_map_bf16(&p.maps[i], ql[i], rl, k, ldq, 64, 64));       // Q_1^T: MN-major A operand
            GN_TRY(tc_make_map_bf16(&p.maps[3 + i], sl[i], rl, n, lds, 64, 64));   // slices: MN-major B operand
        }
        TcGemm& g = p.g[0];
        g.M = static_cast<int>(k);
        g.N = static_cast<int>(n);
        g.K = static_cast<int>(rl);
        g.bn = 256;
        g.a_mn = 1;
        g.b_mn = 1;
        g.nsrc = 6;
        const int am[6] = {0, 0, 1, 0, 1, 2}, bm[6] = {3, 4, 3, 5, 4, 3};   // slice orders 0, 1, 1, 2, 2, 2
        for (int i = 0; i < 6; ++i) {
            g.a_map[i] = am[i];
            g.b_map[i] = bm[i];
        }
        g.D = g32;
        g.ldd = lds;
        p.ngemm = 1;
        GN_TRY(tc_launch(h, &p));
        GN_TRY(copy_f32_to_f64(h, g32, k, n, lds, Gd, G->ld));
    } else
        GN_TRY(dgemm(h, k, n, r + l, 1.0, core->Q, r, 1, static_cast<const double*>(YtA->data), YtA->ld, 0, 0.0,
                     Gd, G->ld, gws, ws_bytes));
    return GN_OK;
}

gn_status gn_approx(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y, double eps, int32_t mode,
                    gn_mat* AX, gn_mat* YtA, gn_core_t* core, gn_mat* F, gn_mat* G, void* ws, size_t ws_bytes) {
    GN_TRY(gn_sketch(h, A, X, Y, AX, YtA, ws, ws_bytes));
    GN_TRY(gn_core(h, YtA, X, eps, mode, core, ws, ws_bytes));
    return gn_factors(h, AX, YtA, core, F, G, ws, ws_bytes);
}

gn_status gn_error_fro2(gn_handle h, const gn_mat* A, const gn_mat* F, const gn_mat* G, double* out, void* ws,
                        size_t ws_bytes) {
    if (!h || !A || !F || !G || !out || !ws) return GN_ERR_INVALID_ARG;
    const long long m = A->rows, n = A->cols, k = F->cols;
    GN_TRY(check_mat(A, m, n));
    GN_TRY(check_mat(F, m, k));
    GN_TRY(check_mat(G, k, n));
    if (F->dtype != GN_F64 || G->dtype != GN_F64) return GN_ERR_DTYPE;
    return error_fro2(h, A->data, A->dtype, A->lo, m, n, A->ld, static_cast<const double*>(F->data), F->ld,
                      static_cast<const double*>(G->data), G->ld, k, out, static_cast<double*>(ws), ws_bytes);
}

gn_status gn_update_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l, int32_t op_dtype, size_t* bytes) {
    if (!bytes) return GN_ERR_INVALID_ARG;
    if (m < 1 || n < 1 || r < 1 || l < 0) return GN_ERR_SHAPE;
    if (op_dtype != GN_F64 && op_dtype != GN_BF16 && op_dtype != GN_BF16X2 && op_dtype != GN_E4M3)
        return GN_ERR_DTYPE;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *bytes = update_scratch(m, n, r, l, op_dtype) + block_sketch_ws(m, n, r, r + l, op_dtype, sms);
    return GN_OK;
}

gn_status gn_resample_workspace_size(int64_t m, int64_t n, int64_t dr, int64_t dl, int32_t op_dtype, size_t* bytes) {
    if (!bytes) return GN_ERR_INVALID_ARG;
    if (m < 1 || n < 1 || dr < 0 || dl < 0 || dr + dl < 1) return GN_ERR_SHAPE;
    if (op_dtype != GN_F64 && op_dtype != GN_BF16 && op_dtype != GN_BF16X2 && op_dtype != GN_E4M3)
        return GN_ERR_DTYPE;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *bytes = block_sketch_ws(m, n, dr, dr + dl, op_dtype, sms);
    return GN_OK;
}

gn_status gn_update(gn_handle h, const gn_mat* E, const gn_mat* X, const gn_mat* Y, gn_mat* AX, gn_mat* YtA,
                    void* ws, size_t ws_bytes) {
    if (!h || !E || !X || !Y || !AX || !YtA || !ws) return GN_ERR_INVALID_ARG;
    const long long m = E->rows, n = E->cols, r = X->cols, rl = Y->cols;
    if (rl <= r) return GN_ERR_SHAPE;
    GN_TRY(check_mat(AX, m, r));
    GN_TRY(check_mat(YtA, rl, n));
    if (AX->dtype != YtA->dtype || (AX->dtype != GN_F32 && AX->dtype != GN_F64)) return GN_ERR_DTYPE;
    const size_t scratch = update_scratch(m, n, r, rl - r, E->dtype);
    if (ws_bytes <= scratch) return GN_ERR_WORKSPACE;
    // E's sketches into the front of ws (the layout gn_sketch writes), the rest is gn_sketch's own scratch
    const size_t es = AX->dtype == GN_F64 ? sizeof(double) : sizeof(float);
    char* base = static_cast<char*>(ws);
    const long long ldx = round8(r), ldy = round8(n);
    gn_mat dAX = *AX, dYtA = *YtA;
    dAX.data = base;
    dAX.ld = ldx;
    dYtA.data = base + align256(es * m * ldx);
    dYtA.ld = ldy;
    if (align256(es * m * ldx) + align256(es * rl * ldy) > scratch) return GN_ERR_WORKSPACE;
    GN_TRY(sketch_block(h, E, X, Y, &dAX, &dYtA, base + scratch, ws_bytes - scratch));
    GN_TRY(add_into(h, AX, dAX.data, ldx));
    GN_TRY(add_into(h, YtA, dYtA.data, ldy));
    return GN_OK;
}

// Copy rows x cols elements of a sketch matrix (FP32 or FP64) between two
// strided buffers on the handle's stream.
static gn_status copy_block(gn_handle h, void* dst, long long ldd, const void* src, long long lds, long long rows,
                     long long cols, size_t es) {
    GN_CUDA_TRY(cudaMemcpy2DAsync(dst, es * ldd, src, es * lds, es * cols, rows, cudaMemcpyDeviceToDevice,
                                  h->stream));
    return GN_OK;
}

static size_t sketch_es(const gn_mat* a) { return a->dtype == GN_F64 ? sizeof(double) : sizeof(float); }

gn_status gn_resample(gn_handle h, const gn_mat* A, const gn_mat* Xd, const gn_mat* Yd, const gn_mat* AX,
                      const gn_mat* YtA, gn_mat* AXn, gn_mat* YtAn, void* ws, size_t ws_bytes) {
    if (!h || !A || !Xd || !Yd || !AX || !YtA || !AXn || !YtAn || !ws) return GN_ERR_INVALID_ARG;
    const long long m = A->rows, n = A->cols, r = AX->cols, rl = YtA->rows, dr = Xd->cols, drl = Yd->cols;
    // dr >= 0 new columns of X, dl = drl - dr >= 0 extra oversampling, dr + dl >= 1
    if (dr < 0 || drl < dr || drl < 1) return GN_ERR_SHAPE;
    GN_TRY(check_mat(AX, m, r));
    GN_TRY(check_mat(YtA, rl, n));
    GN_TRY(check_mat(AXn, m, r + dr));
    GN_TRY(check_mat(YtAn, rl + drl, n));
    if (AXn->dtype != AX->dtype || YtAn->dtype != YtA->dtype || AX->dtype != YtA->dtype) return GN_ERR_DTYPE;
    const size_t es = sketch_es(AX);
    GN_TRY(copy_block(h, AXn->data, AXn->ld, AX->data, AX->ld, m, r, es));
    GN_TRY(copy_block(h, YtAn->data, YtAn->ld, YtA->data, YtA->ld, rl, n, es));
    gn_mat ax = *AXn, yta = *YtAn;   // the new columns / rows, written in place by the sketch
    ax.data = static_cast<char*>(AXn->data) + es * r;
    ax.cols = dr;
    yta.data = static_cast<char*>(YtAn->data) + es * rl * YtAn->ld;
    yta.rows = drl;
    return sketch_block(h, A, Xd, Yd, &ax, &yta, ws, ws_bytes);
}

gn_status gn_append_rows(gn_handle h, const gn_mat* B, const gn_mat* X, const gn_mat* Yb, const gn_mat* AX,
                         gn_mat* YtA, gn_mat* AXn, void* ws, size_t ws_bytes) {
    if (!h || !B || !X || !Yb || !AX || !YtA || !AXn || !ws) return GN_ERR_INVALID_ARG;
    const long long mb = B->rows, n = B->cols, r = X->cols, rl = Yb->cols, m = AX->rows;
    GN_TRY(check_mat(AX, m, r));
    GN_TRY(check_mat(YtA, rl, n));
    GN_TRY(check_mat(AXn, m + mb, r));
    if (AXn->dtype != AX->dtype || YtA->dtype != AX->dtype) return GN_ERR_DTYPE;
    const size_t es = sketch_es(AX);
    const size_t scratch = update_scratch(mb, n, r, rl - r, B->dtype);
    if (ws_bytes <= scratch) return GN_ERR_WORKSPACE;
    GN_TRY(copy_block(h, AXn->data, AXn->ld, AX->data, AX->ld, m, r, es));
    gn_mat bx = *AXn, dyta = *YtA;   // B X straight into the new rows; Yb^T B into scratch
    bx.data = static_cast<char*>(AXn->data) + es * m * AXn->ld;
    bx.rows = mb;
    const long long ldy = round8(n);
    dyta.data = ws;
    dyta.ld = ldy;
    if (align256(es * rl * ldy) > scratch) return GN_ERR_WORKSPACE;
    GN_TRY(sketch_block(h, B, X, Yb, &bx, &dyta, static_cast<char*>(ws) + scratch, ws_bytes - scratch));
    return add_into(h, YtA, dyta.data, ldy);
}

gn_status gn_append_cols(gn_handle h, const gn_mat* B, const gn_mat* Xb, const gn_mat* Y, gn_mat* AX,
                         const gn_mat* YtA, gn_mat* YtAn, void* ws, size_t ws_bytes) {
    if (!h || !B || !Xb || !Y || !AX || !YtA || !YtAn || !ws) return GN_ERR_INVALID_ARG;
    const long long m = B->rows, nb = B->cols, r = Xb->cols, rl = Y->cols, n = YtA->cols;
    GN_TRY(check_mat(AX, m, r));
    GN_TRY(check_mat(YtA, rl, n));
    GN_TRY(check_mat(YtAn, rl, n + nb));
    if (YtAn->dtype != YtA->dtype || YtA->dtype != AX->dtype) return GN_ERR_DTYPE;
    const size_t es = sketch_es(AX);
    const size_t scratch = update_scratch(m, nb, r, rl - r, B->dtype);
    if (ws_bytes <= scratch) return GN_ERR_WORKSPACE;
    GN_TRY(copy_block(h, YtAn->data, YtAn->ld, YtA->data, YtA->ld, rl, n, es));
    gn_mat dax = *AX, ytb = *YtAn;   // B Xb into scratch; Y^T B straight into the new columns
    const long long ldx = round8(r);
    dax.data = ws;
    dax.ld = ldx;
    ytb.data = static_cast<char*>(YtAn->data) + es * n;
    ytb.cols = nb;
    if (align256(es * m * ldx) > scratch) return GN_ERR_WORKSPACE;
    GN_TRY(sketch_block(h, B, Xb, Y, &dax, &ytb, static_cast<char*>(ws) + scratch, ws_bytes - scratch));
    return add_into(h, AX, dax.data, ldx);
}

// Scratch of gn_apply: two FP64 blocks of at most max(r + l, r) x kw, the
// triangular solve's and the GEMMs' split-K partials; for FP32 sketches the
// transposed products (r x kw, n x kw) and the digit-sliced products' scratch.
size_t apply_oz_ws(long long m, long long n, long long r, long long l, long long kw) {
    const long long rl = r + l;
    return align256(sizeof(double) * r * kw) + align256(sizeof(double) * n * kw) +
           std::max({oz_ws_bytes(rl, kw, n, 1), oz_ws_bytes(m, kw, r, 1), oz_ws_bytes(r, kw, m, 1),
                     oz_ws_bytes(n, kw, rl, 1)}) + 512;
}
size_t apply_ws(long long m, long long n, long long r, long long l, long long kw, int sms) {
    const long long rl = r + l;
    return 2 * align256(sizeof(double) * rl * kw) + trsm_ws_bytes(kw, r, sms) +
           std::max({dgemm_ws_bytes(rl, kw, n, sms), dgemm_ws_bytes(m, kw, r, sms), dgemm_ws_bytes(kw, r, m, sms),
                     dgemm_ws_bytes(kw, n, rl, sms), dgemm_ws_bytes(kw, rl, r, sms)}) +
           apply_oz_ws(m, n, r, l, kw) + 1024;
}

gn_status gn_apply_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l, int64_t kw, int32_t side,
                                  size_t* bytes) {
    if (!bytes || m < 1 || n < 1 || r < 1 || l < 0 || kw < 1 || (side != 0 && side != 1)) return GN_ERR_INVALID_ARG;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *bytes = apply_ws(m, n, r, l, kw, sms);
    return GN_OK;
}

gn_status gn_apply(gn_handle h, const gn_mat* AX, const gn_mat* YtA, const gn_core_t* core, const gn_mat* W,
                   gn_mat* out, int32_t side, void* ws, size_t ws_bytes) {
    if (!h || !AX || !YtA || !core || !W || !out || !ws || (side != 0 && side != 1)) return GN_ERR_INVALID_ARG;
    const long long m = AX->rows, n = YtA->cols, r = core->r, l = core->l, k = core->k, rl = r + l;
    if (k < 1 || k > r || !core->Q || !core->R) return GN_ERR_INVALID_ARG;
    const bool trunc = core->sgn && k < r;
    if (trunc && (!core->Q2 || !core->R2)) return GN_ERR_INVALID_ARG;
    GN_TRY(check_mat(AX, m, r));
    GN_TRY(check_mat(YtA, rl, n));
    if (AX->dtype != GN_F64 && AX->dtype != GN_F32) return GN_ERR_DTYPE;
    if (YtA->dtype != GN_F64 && YtA->dtype != GN_F32) return GN_ERR_DTYPE;
    if (W->dtype != GN_F64 || out->dtype != GN_F64 || !W->data || !out->data) return GN_ERR_DTYPE;
    const long long kw = side == 0 ? W->cols : W->rows;
    if (kw < 1) return GN_ERR_SHAPE;
    if (side == 0 && (W->rows != n || out->rows != m || out->cols != kw)) return GN_ERR_SHAPE;
    if (side == 1 && (W->cols != m || out->rows != kw || out->cols != n)) return GN_ERR_SHAPE;
    if (W->ld < W->cols || out->ld < out->cols) return GN_ERR_SHAPE;
    if (ws_bytes < apply_ws(m, n, r, l, kw, h->sm_count)) return GN_ERR_WORKSPACE;
    Carve cv{static_cast<char*>(ws), ws_bytes, 0, true};
    double* B1 = cv.take<double>(rl * kw);
    double* B2 = cv.take<double>(rl * kw);
    // FP32 sketches: the m- and n-sized products by exact digit slicing on the tensor cores
    const bool ax32 = AX->dtype == GN_F32, yta32 = YtA->dtype == GN_F32;
    const bool oz = h->fp64_tc && (ax32 || yta32);
    double* T1 = cv.take<double>(r * kw);   // (W AX)^T
    double* T2 = cv.take<double>(n * kw);   // (B Y^T A)^T
    const size_t ozb = std::max({oz_ws_bytes(rl, kw, n, 1), oz_ws_bytes(m, kw, r, 1), oz_ws_bytes(r, kw, m, 1),
                                 oz_ws_bytes(n, kw, rl, 1)});
    void* ozw = cv.take<char>(ozb);
    if (!cv.ok) return GN_ERR_WORKSPACE;
    size_t gws_bytes = 0;
    double* gws = cv.rest(&gws_bytes);
    const double* Wd = static_cast<const double*>(W->data);
    double* Od = static_cast<double*>(out->data);
    if (side == 0) {
        // B1 = Y^T A W   ((r+l) x kw)
        if (yta32 && oz)
            GN_TRY(oz_dgemm(h, rl, kw, n, 1.0, YtA->data, 1, YtA->ld, 0, Wd, W->ld, 0, 0.0, B1, kw, ozw, ozb));
        else if (yta32)
            GN_TRY(dgemm_a32(h, rl, kw, n, 1.0, static_cast<const float*>(YtA->data), YtA->ld, 0, Wd, W->ld, 0, 0.0,
                             B1, kw, gws, gws_bytes));
        else
            GN_TRY(dgemm(h, rl, kw, n, 1.0, static_cast<const double*>(YtA->data), YtA->ld, 0, Wd, W->ld, 0, 0.0, B1,
                         kw, gws, gws_bytes));
        // B2 = (Q_1^T B1)^T = B1^T Q_1   (kw x k)
        GN_TRY(dgemm(h, kw, k, rl, 1.0, B1, kw, 1, core->Q, r, 0, 0.0, B2, k, gws, gws_bytes));
        const double* Zt = B2;   // Z^T (kw x r) with Z the core pseudoinverse applied to Y^T A W
        if (!trunc) {
            // (R^{-1} Q^T B1)^T = B2 R^{-T}
            GN_TRY(trsm_right_upper(h, B2, kw, r, k, core->R, r, 1, gws, gws_bytes));
        } else {
            // (R_2^{-T} Q_1^T B1)^T = B2 R_2^{-1}, then Z^T = that Q_2^T (kw x r)
            GN_TRY(trsm_right_upper(h, B2, kw, k, k, core->R2, r, 0, gws, gws_bytes));
            GN_TRY(dgemm(h, kw, r, k, 1.0, B2, k, 0, core->Q2, r, 1, 0.0, B1, r, gws, gws_bytes));
            Zt = B1;
        }
        // out = AX Z = AX (Z^T)^T   (m x kw)
        if (ax32 && oz)
            GN_TRY(oz_dgemm(h, m, kw, r, 1.0, AX->data, 1, AX->ld, 0, Zt, r, 1, 0.0, Od, out->ld, ozw, ozb));
        else if (ax32)
            GN_TRY(dgemm_a32(h, m, kw, r, 1.0, static_cast<const float*>(AX->data), AX->ld, 0, Zt, r, 1, 0.0, Od,
                             out->ld, gws, gws_bytes));
        else
            GN_TRY(dgemm(h, m, kw, r, 1.0, static_cast<const double*>(AX->data), AX->ld, 0, Zt, r, 1, 0.0, Od, out->ld,
                         gws, gws_bytes));
        return GN_OK;
    }
    // side 1: B1 = W AX   (kw x r)
    if (ax32 && oz) {   // (W AX)^T = AX^T W^T, then transposed
        GN_TRY(oz_dgemm(h, r, kw, m, 1.0, AX->data, 1, AX->ld, 1, Wd, W->ld, 1, 0.0, T1, kw, ozw, ozb));
        GN_TRY(transpose_rows_f64(h, T1, r, kw, kw, r, B1, r));
    } else if (ax32)
        GN_TRY(dgemm_b32(h, kw, r, m, 1.0, Wd, W->ld, 0, static_cast<const float*>(AX->data), AX->ld, 0, 0.0, B1, r,
                         gws, gws_bytes));
    else
        GN_TRY(dgemm(h, kw, r, m, 1.0, Wd, W->ld, 0, static_cast<const double*>(AX->data), AX->ld, 0, 0.0, B1, r,
                     gws, gws_bytes));
    const double* P = B1;   // (kw x k): (W AX) times the core pseudoinverse's left part
    if (!trunc) {
        GN_TRY(trsm_right_upper(h, B1, kw, r, r, core->R, r, 0, gws, gws_bytes));
    } else {
        GN_TRY(dgemm(h, kw, k, r, 1.0, B1, r, 0, core->Q2, r, 0, 0.0, B2, k, gws, gws_bytes));
        GN_TRY(trsm_right_upper(h, B2, kw, k, k, core->R2, r, 1, gws, gws_bytes));
        P = B2;
    }
    const long long ldp = trunc ? k : r;
    // B = P Q_1^T   (kw x (r+l)), into the buffer P does not occupy
    double* Bq = trunc ? B1 : B2;
    GN_TRY(dgemm(h, kw, rl, k, 1.0, P, ldp, 0, core->Q, r, 1, 0.0, Bq, rl, gws, gws_bytes));
    // out = B Y^T A   (kw x n)
    if (yta32 && oz) {   // (B Y^T A)^T = (Y^T A)^T B^T, then transposed
        GN_TRY(oz_dgemm(h, n, kw, rl, 1.0, YtA->data, 1, YtA->ld, 1, Bq, rl, 1, 0.0, T2, kw, ozw, ozb));
        GN_TRY(transpose_rows_f64(h, T2, n, kw, kw, n, Od, out->ld));
    } else if (yta32)
        GN_TRY(dgemm_b32(h, kw, n, rl, 1.0, Bq, rl, 0, static_cast<const float*>(YtA->data), YtA->ld, 0, 0.0, Od,
                         out->ld, gws, gws_bytes));
    else
        GN_TRY(dgemm(h, kw, n, rl, 1.0, Bq, rl, 0, static_cast<const double*>(YtA->data), YtA->ld, 0, 0.0, Od, out->ld,
                     gws, gws_bytes));
    return GN_OK;
}

gn_status gn_hmt(gn_handle h, const gn_mat* A, const gn_mat* X, gn_mat* Q, gn_mat* B, void* ws, size_t ws_bytes) {
    if (!h || !A || !X || !Q || !B || !ws) return GN_ERR_INVALID_ARG;
    const long long m = A->rows, n = A->cols, r = X->cols;
    if (r < 1 || r > std::min(m, n)) return GN_ERR_SHAPE;
    GN_TRY(check_mat(A, m, n));
    GN_TRY(check_mat(X, n, r));
    GN_TRY(check_mat(Q, m, r));
    GN_TRY(check_mat(B, r, n));
    if (A->dtype != GN_F64 || X->dtype != GN_F64 || Q->dtype != GN_F64 || B->dtype != GN_F64) return GN_ERR_DTYPE;
    if (ws_bytes < hmt_ws(m, n, r, h->sm_count)) return GN_ERR_WORKSPACE;
    Carve cv{static_cast<char*>(ws), ws_bytes, 0, true};
    double* W = cv.take<double>(m * r);
    double* Rx = cv.take<double>(r * r);
    size_t inner_bytes = 0;
    double* inner = cv.rest(&inner_bytes);
    if (!cv.ok) return GN_ERR_WORKSPACE;
    // AX (Algorithm 1, step 2), then its Householder QR (step 3)
    GN_TRY(dgemm(h, m, r, n, 1.0, static_cast<const double*>(A->data), A->ld, 0,
                 static_cast<const double*>(X->data), X->ld, 0, 0.0, W, r, inner, inner_bytes));
    GN_TRY(householder_qr(h, W, m, r, r, static_cast<double*>(Q->data), Q->ld, Rx, r, inner, inner_bytes));
    // B = Q^T A (step 4; a second pass over A)
    return dgemm(h, r, n, m, 1.0, static_cast<const double*>(Q->data), Q->ld, 1,
                 static_cast<const double*>(A->data), A->ld, 0, 0.0, static_cast<double*>(B->data), B->ld, inner,
                 inner_bytes);
}

}  // extern "C"

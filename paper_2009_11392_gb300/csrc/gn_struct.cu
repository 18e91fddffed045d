// Structured sketches of Section 7's experiments and Section 2.5's fast
// sketches, made on the device from their random draws.
//
// Subsampled DCT: X = D C^T S (n x r) with D = diag(signs), C the orthonormal
// DCT-II matrix, C[k, i] = a_k cos(pi (2 i + 1) k / (2 n)) (a_0 = sqrt(1/n),
// a_k = sqrt(2/n)), S the columns `cols` of the identity; the sqrt(n/r) scale
// is left out (GN is invariant under X -> X c).  The matrix is written
// explicitly and the sketches then run on the tensor cores like Gaussian ones:
// on GB300 the 2 m n r flops of the dense product at the BF16 tensor rate take
// about as long as an O(m n log n) FFT on the FP32 CUDA cores at r ~ 10^3 (and
// the dense product needs no transposed transform for Y^T A).
//
// The angle is reduced exactly in integers, (2 i + 1) k mod 4n, before cospi,
// so every entry is the cosine of an exactly known multiple of pi / (2 n).
#include "gn_internal.cuh"

#include <algorithm>

namespace gn {
namespace {

template <typename T>
__device__ __forceinline__ void put(T* p, double v);
template <>
__device__ __forceinline__ void put<double>(double* p, double v) { *p = v; }
template <>
__device__ __forceinline__ void put<float>(float* p, double v) { *p = static_cast<float>(v); }
template <>
__device__ __forceinline__ void put<__nv_bfloat16>(__nv_bfloat16* p, double v) {
    *p = __float2bfloat16_rn(static_cast<float>(v));   // through FP32, as gn_quantize rounds
}

template <typename T>
__global__ void dct_sketch_kernel(long long n, long long r, const double* __restrict__ signs,
                                  const long long* __restrict__ cols, T* __restrict__ X, long long ldx) {
    const long long total = n * r;
    const double a0 = sqrt(1.0 / static_cast<double>(n)), a1 = sqrt(2.0 / static_cast<double>(n));
    const long long four_n = 4 * n;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / r, j = e - i * r;
        const long long k = cols[j];
        // (2 i + 1) k < 2 n^2 <= 2^63 for n <= 2^31 (k < n): exact in 64 bits
        const unsigned long long t = (static_cast<unsigned long long>(2 * i + 1) * static_cast<unsigned long long>(k)) %
                                     static_cast<unsigned long long>(four_n);
        const double c = cospi(static_cast<double>(t) / static_cast<double>(2 * n));
        put<T>(X + i * ldx + j, signs[i] * ((k == 0 ? a0 : a1) * c));
    }
}

}  // namespace
}  // namespace gn

using namespace gn;

extern "C" gn_status gn_dct_sketch(gn_handle h, int64_t n, int64_t r, const double* signs, const int64_t* cols,
                                   gn_mat* X) {
    if (!h || !signs || !cols || !X || !X->data) return GN_ERR_INVALID_ARG;
    if (n < 1 || r < 1 || r > n || n > (1LL << 31)) return GN_ERR_SHAPE;
    if (X->rows != n || X->cols != r || X->ld < r) return GN_ERR_SHAPE;
    const long long total = static_cast<long long>(n) * r;
    const int blocks = static_cast<int>(std::max<long long>(1, std::min<long long>((total + 255) / 256,
                                                                                     16LL * h->sm_count)));
    const long long* c = reinterpret_cast<const long long*>(cols);
    switch (X->dtype) {
        case GN_F64:
            dct_sketch_kernel<double><<<blocks, 256, 0, h->stream>>>(n, r, signs, c, static_cast<double*>(X->data),
                                                                     X->ld);
            break;
        case GN_F32:
            dct_sketch_kernel<float><<<blocks, 256, 0, h->stream>>>(n, r, signs, c, static_cast<float*>(X->data),
                                                                    X->ld);
            break;
        case GN_BF16:
            if ((reinterpret_cast<uintptr_t>(X->data) & 15) || X->ld % 8) return GN_ERR_ALIGNMENT;
            dct_sketch_kernel<__nv_bfloat16><<<blocks, 256, 0, h->stream>>>(
                n, r, signs, c, static_cast<__nv_bfloat16*>(X->data), X->ld);
            break;
        default:
            return GN_ERR_DTYPE;
    }
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

// ---------------------------------------------------------------------------
// Sparse A (CSR) with CountSketch sketches: Section 2.5's input-sparsity route.
// A CountSketch X (n x r) has one +-1 per row: X[j, bx[j]] = sx[j]; likewise Y
// (m x (r + l)) with by, sy.  Then every nonzero a_ij adds sx[j] a_ij to
// AX[i, bx[j]] and sy[i] a_ij to (Y^T A)[by[i], j]: O(nnz) work, one thread per
// nonzero (its row found by binary search in row_ptr), FP64 or FP32 atomic adds
// into the zeroed outputs (the summation order is not fixed).  Indices are
// checked on the device: a column index outside [0, n) or a bucket outside the
// output skips that nonzero and latches GN_ERR_INVALID_ARG in the status word.
namespace gn {
namespace {

template <typename T>
__global__ void zero2d_kernel(T* p, long long rows, long long cols, long long ld) {
    const long long total = rows * cols;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        p[(e / cols) * ld + e % cols] = T(0);
}

template <typename T>
__global__ void countsketch_csr_kernel(const long long* __restrict__ row_ptr, const int* __restrict__ col_idx,
                                       const T* __restrict__ vals, long long m, long long nnz,
                                       long long n, const long long* __restrict__ bx,
                                       const double* __restrict__ sx, T* AX, long long ldx, long long rx,
                                       const long long* __restrict__ by, const double* __restrict__ sy, T* YtA,
                                       long long ldy, long long ry, int32_t* status) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < nnz;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        // row i: the last row whose first nonzero is at or before e
        long long lo = 0, hi = m - 1;
        while (lo < hi) {
            const long long mid = (lo + hi + 1) >> 1;
            if (row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const long long i = lo;
        const long long j = col_idx[e];
        if (j < 0 || j >= n) {
            atomicCAS(&status[GN_DEV_STATUS], 0, GN_ERR_INVALID_ARG);
            continue;
        }
        const T v = vals[e];
        if (AX) {
            const long long c = bx[j];
            if (c >= 0 && c < rx) atomicAdd(AX + i * ldx + c, static_cast<T>(sx[j]) * v);
            else atomicCAS(&status[GN_DEV_STATUS], 0, GN_ERR_INVALID_ARG);
        }
        if (YtA) {
            const long long c = by[i];
            if (c >= 0 && c < ry) atomicAdd(YtA + c * ldy + j, static_cast<T>(sy[i]) * v);
            else atomicCAS(&status[GN_DEV_STATUS], 0, GN_ERR_INVALID_ARG);
        }
    }
}

template <typename T>
__global__ void countsketch_matrix_kernel(long long n, long long r, const long long* __restrict__ b,
                                          const double* __restrict__ s, T* X, long long ldx) {
    const long long total = n * r;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / r, j = e - i * r;
        X[i * ldx + j] = b[i] == j ? static_cast<T>(s[i]) : T(0);
    }
}

int grid_of(gn_handle h, long long work) {
    return static_cast<int>(std::max<long long>(1, std::min<long long>((work + 255) / 256, 16LL * h->sm_count)));
}

}  // namespace
}  // namespace gn

extern "C" gn_status gn_sketch_csr_countsketch(gn_handle h, const gn_csr* A, const int64_t* bx, const double* sx,
                                               const int64_t* by, const double* sy, gn_mat* AX, gn_mat* YtA) {
    if (!h || !A || !A->row_ptr || !A->col_idx || (!A->vals && A->nnz > 0)) return GN_ERR_INVALID_ARG;
    const long long m = A->rows, n = A->cols, nnz = A->nnz;
    if (m < 1 || n < 1 || nnz < 0 || n > (1LL << 31) - 1) return GN_ERR_SHAPE;
    if (A->dtype != GN_F64 && A->dtype != GN_F32) return GN_ERR_DTYPE;
    if (!AX && !YtA) return GN_ERR_INVALID_ARG;
    if (AX) {
        if (!AX->data || !bx || !sx) return GN_ERR_INVALID_ARG;
        if (AX->rows != m || AX->cols < 1 || AX->ld < AX->cols) return GN_ERR_SHAPE;
        if (AX->dtype != A->dtype) return GN_ERR_DTYPE;
    }
    if (YtA) {
        if (!YtA->data || !by || !sy) return GN_ERR_INVALID_ARG;
        if (YtA->cols != n || YtA->rows < 1 || YtA->ld < n) return GN_ERR_SHAPE;
        if (YtA->dtype != A->dtype) return GN_ERR_DTYPE;
    }
    const long long* rp = reinterpret_cast<const long long*>(A->row_ptr);
    const long long* bxl = reinterpret_cast<const long long*>(bx);
    const long long* byl = reinterpret_cast<const long long*>(by);
    if (A->dtype == GN_F64) {
        double* ax = AX ? static_cast<double*>(AX->data) : nullptr;
        double* yta = YtA ? static_cast<double*>(YtA->data) : nullptr;
        if (ax) { zero2d_kernel<double><<<grid_of(h, m * AX->cols), 256, 0, h->stream>>>(ax, m, AX->cols, AX->ld); count_launch(); }
        if (yta) { zero2d_kernel<double><<<grid_of(h, YtA->rows * n), 256, 0, h->stream>>>(yta, YtA->rows, n, YtA->ld); count_launch(); }
        if (nnz > 0) {
            countsketch_csr_kernel<double><<<grid_of(h, nnz), 256, 0, h->stream>>>(
                rp, A->col_idx, static_cast<const double*>(A->vals), m, nnz, n, bxl, sx, ax, AX ? AX->ld : 0,
                AX ? AX->cols : 0, byl, sy, yta, YtA ? YtA->ld : 0, YtA ? YtA->rows : 0, h->dstatus);
            count_launch();
        }
    } else {
        float* ax = AX ? static_cast<float*>(AX->data) : nullptr;
        float* yta = YtA ? static_cast<float*>(YtA->data) : nullptr;
        if (ax) { zero2d_kernel<float><<<grid_of(h, m * AX->cols), 256, 0, h->stream>>>(ax, m, AX->cols, AX->ld); count_launch(); }
        if (yta) { zero2d_kernel<float><<<grid_of(h, YtA->rows * n), 256, 0, h->stream>>>(yta, YtA->rows, n, YtA->ld); count_launch(); }
        if (nnz > 0) {
            countsketch_csr_kernel<float><<<grid_of(h, nnz), 256, 0, h->stream>>>(
                rp, A->col_idx, static_cast<const float*>(A->vals), m, nnz, n, bxl, sx, ax, AX ? AX->ld : 0,
                AX ? AX->cols : 0, byl, sy, yta, YtA ? YtA->ld : 0, YtA ? YtA->rows : 0, h->dstatus);
            count_launch();
        }
    }
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

extern "C" gn_status gn_countsketch_matrix(gn_handle h, int64_t n, int64_t r, const int64_t* buckets,
                                           const double* signs, gn_mat* X) {
    if (!h || !buckets || !signs || !X || !X->data) return GN_ERR_INVALID_ARG;
    if (n < 1 || r < 1 || X->rows != n || X->cols != r || X->ld < r) return GN_ERR_SHAPE;
    const long long* b = reinterpret_cast<const long long*>(buckets);
    if (X->dtype == GN_F64)
        countsketch_matrix_kernel<double><<<grid_of(h, n * r), 256, 0, h->stream>>>(n, r, b, signs,
                                                                                   static_cast<double*>(X->data), X->ld);
    else if (X->dtype == GN_F32)
        countsketch_matrix_kernel<float><<<grid_of(h, n * r), 256, 0, h->stream>>>(n, r, b, signs,
                                                                                  static_cast<float*>(X->data), X->ld);
    else
        return GN_ERR_DTYPE;
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

// B X for a dense B (rows x n) and a CountSketch X (n x r): column c of the
// result is the signed sum of the columns j of B with bx[j] = c (O(rows n)
// work; one thread per entry of B, FP64 atomic adds into the zeroed output).
namespace gn {
namespace {
template <typename TB>
__global__ void countsketch_dense_kernel(const TB* __restrict__ B, long long rows, long long n, long long ldb,
                                         const long long* __restrict__ bx, const double* __restrict__ sx,
                                         double* out, long long ldo, long long r, int32_t* status) {
    const long long total = rows * n;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = e / n, j = e - i * n;
        const long long c = bx[j];
        if (c < 0 || c >= r) {
            atomicCAS(&status[GN_DEV_STATUS], 0, GN_ERR_INVALID_ARG);
            continue;
        }
        atomicAdd(out + i * ldo + c, sx[j] * static_cast<double>(B[i * ldb + j]));
    }
}
}  // namespace
}  // namespace gn

extern "C" gn_status gn_countsketch_apply(gn_handle h, const gn_mat* B, const int64_t* bx, const double* sx,
                                          gn_mat* out) {
    if (!h || !B || !B->data || !bx || !sx || !out || !out->data) return GN_ERR_INVALID_ARG;
    const long long rows = B->rows, n = B->cols, r = out->cols;
    if (rows < 1 || n < 1 || r < 1 || out->rows != rows || B->ld < n || out->ld < r) return GN_ERR_SHAPE;
    if (out->dtype != GN_F64 || (B->dtype != GN_F64 && B->dtype != GN_F32)) return GN_ERR_DTYPE;
    double* o = static_cast<double*>(out->data);
    zero2d_kernel<double><<<grid_of(h, rows * r), 256, 0, h->stream>>>(o, rows, r, out->ld);
    count_launch();
    const long long* b = reinterpret_cast<const long long*>(bx);
    if (B->dtype == GN_F64)
        countsketch_dense_kernel<double><<<grid_of(h, rows * n), 256, 0, h->stream>>>(
            static_cast<const double*>(B->data), rows, n, B->ld, b, sx, o, out->ld, r, h->dstatus);
    else
        countsketch_dense_kernel<float><<<grid_of(h, rows * n), 256, 0, h->stream>>>(
            static_cast<const float*>(B->data), rows, n, B->ld, b, sx, o, out->ld, r, h->dstatus);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

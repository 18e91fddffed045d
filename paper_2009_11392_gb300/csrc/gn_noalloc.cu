// Allocation-free variant of gn_error_fro2 (see include/gn.h).
//
// gn_error_fro2 reduces ||A - F G||_F^2 in two launches: one partial sum per
// 64 x 64 output tile, then a fixed-order sum of the partials.  The partials
// normally live in the caller's workspace.  Here they live in a file-scope
// device array instead, so a caller that cannot allocate device memory still
// gets the fused error without a workspace.
#include "gn_internal.cuh"

#include <mutex>

namespace {

// Capacity: one double per 64 x 64 tile of A, i.e. up to 16384 tiles
// (m x n <= 67,108,864 elements, e.g. 8192 x 8192).  Every GPU that loads the
// library holds these 128 KB (plus slack) until the process exits.
constexpr long long kMaxTiles = 16384;
constexpr long long kSlots = kMaxTiles + 64;   // gn::error_fro2 checks a little slack

static __device__ __align__(256) double g_err_partials[kSlots];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};

// Device address of g_err_partials on `device`, looked up once per device with
// that device current (host code cannot use the symbol's name as an address).
gn_status partials_for(int device, double** out) {
    if (device < 0 || device >= kMaxDevices) return GN_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[device]) {
        int prev = 0;
        if (cudaGetDevice(&prev) != cudaSuccess) return GN_ERR_CUDA;
        if (prev != device && cudaSetDevice(device) != cudaSuccess) return GN_ERR_CUDA;
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_err_partials);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess || p == nullptr) return GN_ERR_CUDA;
        g_ptr[device] = static_cast<double*>(p);
    }
    *out = g_ptr[device];
    return GN_OK;
}

}  // namespace

extern "C" gn_status gn_error_fro2_noalloc(gn_handle h, const gn_mat* A, const gn_mat* F, const gn_mat* G,
                                          double* out) {
    if (!h || !A || !F || !G || !out || !A->data || !F->data || !G->data) return GN_ERR_INVALID_ARG;
    const long long m = A->rows, n = A->cols, k = F->cols;
    if (m <= 0 || n <= 0 || k < 0) return GN_ERR_SHAPE;
    if (F->rows != m || G->rows != k || G->cols != n) return GN_ERR_SHAPE;
    if (A->ld < n || F->ld < k || G->ld < n) return GN_ERR_INVALID_ARG;
    if (A->dtype < GN_F64 || A->dtype > GN_BF16X2 || (A->dtype == GN_BF16X2 && !A->lo)) return GN_ERR_DTYPE;
    if (F->dtype != GN_F64 || G->dtype != GN_F64) return GN_ERR_DTYPE;
    const long long tiles = ((m + 63) / 64) * ((n + 63) / 64);
    if (tiles > kMaxTiles) return GN_ERR_SHAPE;   // beyond the static array's capacity
    double* partials = nullptr;
    GN_TRY(partials_for(h->device, &partials));
    // Every slot this call reads is written by this call first: nothing to clear.
    return gn::error_fro2(h, A->data, A->dtype, A->lo, m, n, A->ld, static_cast<const double*>(F->data), F->ld,
                          static_cast<const double*>(G->data), G->ld, k, out, partials,
                          static_cast<size_t>(kSlots) * sizeof(double));
}

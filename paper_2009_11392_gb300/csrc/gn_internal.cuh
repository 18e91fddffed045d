// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/gn.h"

// Device status word layout (int32 slots of the handle's 64-byte status block).
enum { GN_DEV_STATUS = 0, GN_DEV_WHERE = 1 };

struct gn_handle_s {
    int device;
    int sm_count;
    cudaStream_t stream;
    cudaStream_t side;         // second stream: work that overlaps the main sequence
    cudaEvent_t ev_fork, ev_join;
    cudaStream_t crit;         // high-priority stream for the QR's panel chain
    cudaEvent_t ev_crit0, ev_crit1;
    int32_t* dstatus;          // device: [0] latched gn_status, [1] where
    uint64_t wait_limit_ns;
    // batched path: the tables gn_batched_prepare uploaded into batched_ws
    void* batched_ws;
    int batched_count, batched_sk_tiles, batched_c_tiles, batched_mt;
    int batched_policy;        // tile policy of the next gn_batched_prepare
    int fp64_g;                // gn_factors: FP64 G even for FP32 Y^T A
    int fp64_tc;               // gn_factors: digit-sliced tensor-core FP64 products (FP32 AX)
    long long fp64_accum;      // gn_set_fp64_accum: K per stored part of split sketches (0: off); C, G in FP64
    int stall_test;            // gn_set_stall_test: the next sketch launches wait on a barrier nothing completes
    // gn_core with GN_CORE_DEFER: the core whose k and diagnostics are still on
    // their way to the pinned host words; gn_core_finish completes it.
    cudaEvent_t ev_defer;
    int32_t* pin_k;            // pinned host: k
    double* pin_diag;          // pinned host: est ||R^-1||, est ||C||, eps_abs
    struct {
        int active;
        int mode;
        long long r;
        double *R, *Q2, *R2, *W2, *inner;
        size_t inner_bytes;
    } pend;
    // gn_forward_dense / gn_backward: the workspace whose shared front (sketches,
    // core QR, F) was formed last, and from which inputs; gn_backward_saved
    // requires a match
    struct {
        int valid;
        const void *ws, *A, *X, *Y;
        size_t ws_bytes;
        long long m, n, r, l, lda, ldx, ldy;
        int dtype;
    } adj;
};

#define GN_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return GN_ERR_CUDA;          \
    } while (0)

#define GN_TRY(expr)                                        \
    do {                                                    \
        gn_status _s = (expr);                              \
        if (_s != GN_OK) return _s;                         \
    } while (0)

// --------------------------------------------------------------------------
// Tensor-core (tcgen05) multi-GEMM engine: D_g = sum_s A_{g,s} B_{g,s}
// --------------------------------------------------------------------------
namespace gn {

// Number of kernels this library has launched (all threads, all handles).
unsigned long long launch_count();
void count_launch();

constexpr int TC_MAX_MAPS = 14;
constexpr int TC_MAX_GEMMS = 7;
constexpr int TC_MAX_SRC = 12;

constexpr int TC_BK = 64;   // K elements per stage of the BF16 multi-GEMM (one K block)

struct TcGemm {
    int M, N, K;             // D is M x N, contraction length K
    int bn;                  // N tile: multiple of 64 (MN-major B) or 16 (K-major B), <= 256
    int a_mn, b_mn;          // 0: K-major operand, 1: MN-major operand
    int nsrc;                // number of (A, B) pairs summed into D
    int a_map[TC_MAX_SRC];   // tensor-map indices
    int b_map[TC_MAX_SRC];
    int tiles_m, tiles_n, kblocks;
    int tile_base;           // first global tile index of this GEMM
    float* D;
    long long ldd;
    int vec4;                // D rows 16-byte aligned -> float4 stores
    int ksplit;              // S >= 2: every tile runs as S items over equal parts of its K range
                             // (single launches only; 0 or 1: whole K)
    long long part_stride;   // 0: the S parts add into a pre-zeroed D; > 0: part c is stored
                             // (not added) at D + c * part_stride, to be summed by the caller
    int kpart;               // > 0 (stored parts only): part c covers K blocks [c kpart, (c + 1) kpart)
                             // of every source (K-aligned); 0: parts of the sources' joint K sequence
    // e4m3 launches (TcParams::f8): scale-factor images, 512 bytes of the tile's
    // UE8M0 byte per 128 x 128 tile of the original matrix, row-major over tiles.
    const uint8_t* sfa;
    const uint8_t* sfb;
    int sfa_ld, sfb_ld;      // tiles per row of the image's tile grid
    int sfa_tr, sfb_tr;      // 1: operand tile (row block rb, k block kb) is image tile (kb, rb)
    int sfa_rows, sfb_rows;  // operand row blocks (ragged tiles clamp to the last)
};

struct TcParams {
    CUtensorMap maps[TC_MAX_MAPS];
    TcGemm g[TC_MAX_GEMMS];
    const TcGemm* gg;          // grouped mode: descriptors in device memory
    const CUtensorMap* gmaps;  // grouped mode: tensor maps in device memory (64-B aligned)
    int ngemm;
    int total_tiles;
    int32_t* status;
    unsigned long long wait_limit_ns;
    int f8;                    // 1: e4m3 operands (K-major, block-scaled MMA, bn = 128)
    int stall_test;            // 1: the epilogue first waits on a barrier nothing completes (tests the timeout path)
    // Balanced last round: cluster tiles [split_base, split_base + nsplit) run
    // as two halves of their K range each (work items split_base + 2u, + 2u + 1),
    // adding into a pre-zeroed D.
    int split_base, nsplit;
    // snake_groups > 0: CTA c takes tile k ncl + c in even rounds k and
    // k ncl + ncl - 1 - c in odd ones, on snake_groups x (tiles of GEMM 0) CTAs
    // at most.  With the GEMMs in decreasing cost order this pairs the longest
    // with the shortest (GEMMs of n, n-1, ..., 1 units on ceil(n/2) groups: n
    // units per CTA); the last-round split is off.
    int snake_groups;
    int snake;   // set by tc_launch from snake_groups
    int max_ctas;
};

// Host helpers (gn_tc.cu).
gn_status tc_make_map_bf16(CUtensorMap* map, const void* base, long long rows, long long cols,
                           long long ld, int box_cols, int box_rows);
// e4m3 operand: rows x cols bytes, leading dimension ld bytes, 128-byte boxes.
gn_status tc_make_map_e4m3(CUtensorMap* map, const void* base, long long rows, long long cols,
                           long long ld, int box_rows);
gn_status tc_launch(gn_handle h, TcParams* p);
// Fill tiles_m / tiles_n / kblocks / tile_base / vec4 of one GEMM descriptor.
gn_status tc_prepare_gemm(TcGemm* G, int tile_base, int mt = 1, int f8 = 0);

// e4m3 helpers (gn_fp8.cu).
// Per 128 x 128 tile of src (FP64 or FP32, rows x cols): scale byte, and the
// codes row-major (dst, ld) and / or transposed (dst_t, ld_t); either may be null.
gn_status quantize_e4m3(gn_handle h, const void* src, int src_f64, long long rows, long long cols, long long lds,
                        uint8_t* dst, long long ld, uint8_t* dst_t, long long ld_t, uint8_t* scale);
// 512-byte scale-factor image of every tile from its scale byte.
gn_status e4m3_sf_image(gn_handle h, const uint8_t* scale, long long tiles, uint8_t* image);
// BF16 copy of the transposed e4m3 operand data_t (cols x rows of the original
// rows x cols matrix) with the scales applied: exact (3 mantissa bits fit in 8).
gn_status e4m3_t_to_bf16(gn_handle h, const uint8_t* data_t, long long ld_t, const uint8_t* scale,
                         long long rows, long long cols, __nv_bfloat16* out, long long ldo);
// Grouped launch: descriptors (tile_base ascending) and tensor maps already in
// device memory; any number of GEMMs.
gn_status tc_launch_grouped(gn_handle h, const TcGemm* dev_gemms, int ngemm, const CUtensorMap* dev_maps,
                            int total_tiles, int mt = 1);

// --------------------------------------------------------------------------
// FP64 / FP32 helper kernels (gn_f64.cu)
// --------------------------------------------------------------------------
// C = alpha * op(A) op(B) + beta * C  (row-major, FP64).  ta / tb: operand is
// stored transposed (op(A)[i][k] = A[k*lda + i]).  ws (may be null) enables
// split-K for skinny outputs: bytes needed = dgemm_ws_bytes(M, N, K).
size_t dgemm_ws_bytes(long long M, long long N, long long K, int sm_count);
gn_status dgemm(gn_handle h, long long M, long long N, long long K, double alpha,
                const double* A, long long lda, int ta, const double* B, long long ldb, int tb,
                double beta, double* C, long long ldc, double* ws, size_t ws_bytes);

// Same product with an FP32 A operand (promoted to FP64 on load).
gn_status dgemm_a32(gn_handle h, long long M, long long N, long long K, double alpha,
                    const float* A, long long lda, int ta, const double* B, long long ldb, int tb,
                    double beta, double* C, long long ldc, double* ws, size_t ws_bytes);

// Same product with an FP32 B operand.
gn_status dgemm_b32(gn_handle h, long long M, long long N, long long K, double alpha,
                    const double* A, long long lda, int ta, const float* B, long long ldb, int tb,
                    double beta, double* C, long long ldc, double* ws, size_t ws_bytes);

// Householder QR (blocked, compact WY).  W (M x N, ld) is overwritten; Q (M x N,
// ldq) and R (N x N, ldr) receive the thin factors with diag(R) >= 0.
size_t qr_ws_bytes(long long M, long long N, int sm_count);
gn_status householder_qr(gn_handle h, double* W, long long M, long long N, long long ld,
                         double* Q, long long ldq, double* R, long long ldr,
                         double* ws, size_t ws_bytes);
// The two halves of householder_qr: the factorization (R written, reflectors
// kept in ws) and the formation of the thin Q from them (same W and ws).
// oz (optional, >= qr_oz_ws_bytes(M, N)): with the look-ahead and at least two
// 256-column blocks, the factorization is blocked and each block's update of the
// columns to its right runs as digit-sliced products on the tensor cores (for
// cores of FP32 sketches); the blocks' T stay in oz for qr_form_q; null: FP64
// units only.
gn_status qr_factor(gn_handle h, double* W, long long M, long long N, long long ld, double* R,
                    long long ldr, double* ws, size_t ws_bytes, void* oz = nullptr, size_t oz_bytes = 0);
// oz (optional, >= qr_oz_ws_bytes(M, N)): form Q in blocks of 256 reflectors with
// the large products on the tensor cores (oz_dgemm); null: FP64 units only.
gn_status qr_form_q(gn_handle h, const double* W, long long M, long long N, long long ld, double* Q,
                    long long ldq, double* ws, size_t ws_bytes, void* oz = nullptr, size_t oz_bytes = 0);
size_t qr_oz_ws_bytes(long long M, long long N);

// Right triangular solves, FP64, in place on F (m x k):
//   upper == 1, trans == 0: F <- F R^{-1}   (R upper, k x k)
//   upper == 1, trans == 1: F <- F R^{-T}
// oz (optional): workspace of oz_dgemm for the outer-block updates (>= oz_ws_bytes(m,
// 128, k, 0)); null keeps every update on the FP64 units.
size_t trsm_ws_bytes(long long m, long long k, int sm_count);
gn_status trsm_right_upper(gn_handle h, double* F, long long m, long long k, long long ldf,
                           const double* R, long long ldr, int trans, double* ws, size_t ws_bytes,
                           void* oz = nullptr, size_t oz_bytes = 0);

// FP64 product on the BF16 tensor cores by exact digit slicing (gn_ozaki.cu);
// same operand conventions as dgemm, A FP64 or (a_f32) FP32.  digits: BF16
// digits per operand row / column (7: FP64 accuracy; d < 7: every term carries
// an error of about 2^(1 - 7d) max|a_i.| max|b_.j|).
size_t oz_ws_bytes(long long M, long long N, long long K, int a_f32);
gn_status oz_dgemm(gn_handle h, long long M, long long N, long long K, double alpha, const void* A, int a_f32,
                   long long lda, int ta, const double* B, long long ldb, int tb, double beta, double* C,
                   long long ldc, void* ws, size_t ws_bytes, int digits = 7);

// Core diagnostics (one CTA): out3[0] = est ||R^{-1}||_2 (if want_estimate),
// out3[1] = est ||R||_2 (if eps_relative), out3[2] = the absolute threshold
// used (eps, or eps * est ||R||_2); *k_out = first i with |R_ii| <= threshold.
// ws: 2 r doubles.
gn_status core_diagnostics(gn_handle h, const double* R, long long r, long long ldr, double eps,
                           int eps_relative, int want_estimate, int iters, double* out3, int* k_out,
                           double* ws, size_t ws_bytes);

gn_status copy_f32_to_f64(gn_handle h, const float* src, long long rows, long long cols,
                          long long lds, double* dst, long long ldd);
// FP64 -> three BF16 slices hi + mid + lo (residuals taken in FP64).
gn_status split3_f64_bf16(gn_handle h, const double* src, long long rows, long long cols, long long lds,
                          __nv_bfloat16* hi, __nv_bfloat16* mid, __nv_bfloat16* lo, long long ldd);
gn_status split3_bf16(gn_handle h, const float* src, long long rows, long long cols, long long lds,
                      __nv_bfloat16* hi, __nv_bfloat16* mid, __nv_bfloat16* lo, long long ldd);
gn_status sum3_f32_to_f64(gn_handle h, const float* a, const float* b, const float* c,
                          long long rows, long long cols, long long lds, double* dst, long long ldd);
gn_status quantize_bf16(gn_handle h, const void* src, int src_f64, long long rows, long long cols,
                        long long lds, __nv_bfloat16* hi, __nv_bfloat16* lo, long long ldd);
gn_status transpose_rows_f64(gn_handle h, const double* src, long long rows, long long cols,
                             long long lds, long long keep_rows, double* dst, long long ldd);
gn_status error_fro2(gn_handle h, const void* A, int a_dtype, const void* A_lo, long long m,
                     long long n, long long lda, const double* F, long long ldf, const double* G,
                     long long ldg, long long k, double* out, double* ws, size_t ws_bytes);
size_t error_ws_bytes(long long m, long long n, int sm_count);
gn_status set_zero_f64(gn_handle h, double* p, long long rows, long long cols, long long ld);
// Latch GN_ERR_NONFINITE in the handle's status word if R's upper triangle
// (r x r, FP64) holds a NaN or an infinity.
gn_status latch_nonfinite_upper(gn_handle h, const double* R, long long r, long long ldr);

}  // namespace gn

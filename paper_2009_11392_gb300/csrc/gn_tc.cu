// Tensor-core engine for the sketch products of generalized Nystrom
// (Algorithm 2, step 2: AX and Y^T A) and for the split-precision core product
// C = (Y^T A) X, and for the digit-sliced FP64 products (one GEMM per digit
// order).  One persistent, warp-specialised sm_103a kernel computes up to
// TC_MAX_GEMMS independent GEMMs D_g = sum_s A_{g,s} B_{g,s} in a single launch
// (any number in grouped mode), tiles in round-robin or boustrophedon order,
// optionally as K parts (added into D, or stored apart, K-aligned or not):
//
//   warp 0      : TMA producer -- cp.async.bulk.tensor tiles of both operands
//                 into a shared-memory ring (128B swizzle; 4 stages of 48 KB
//                 for 128-row tiles, 3 of 64 KB for 256-row tiles), one
//                 mbarrier with a transaction count per stage;
//   warp 1      : tcgen05.mma issuer (one thread) -- 128 x bn x 16 BF16 MMAs
//                 with FP32 accumulators in tensor memory, two accumulator
//                 buffers of 256 columns so the epilogue of one tile overlaps
//                 the main loop of the next; also owns the TMEM allocation;
//   warps 2..5  : epilogue -- tcgen05.ld 32 lanes x 32 columns per warp,
//                 FP32 stores to global memory.
//
// Operands are used in their natural row-major layout: the A operand of a
// GEMM may be K-major (rows of A contiguous along K) or MN-major, likewise B.
// For AX, A is K-major and X (n x r, r contiguous) is an MN-major B; for
// Y^T A, Y (m x (r+l)) is an MN-major A and the data matrix A an MN-major B.
// Every wait on an mbarrier is bounded by a time limit; on expiry the kernel
// latches GN_ERR_TIMEOUT in the status word, drains its copies and MMAs,
// frees its tensor memory and returns.
#include "gn_internal.cuh"

#include <string.h>

namespace gn {
namespace {

constexpr int BM = 128;                          // M of one tcgen05 MMA
constexpr int BK = TC_BK;                        // K per stage: 64 bf16 = one 128B swizzle row
constexpr int B_STAGE_BYTES = 256 * BK * 2;      // 32 KB (bn <= 256)
constexpr int TMEM_COLS = 512;
constexpr int NUM_THREADS = 192;

// MT = number of 128-row M halves per tile.  MT = 1: 128 x bn tiles, 4 stages of
// 48 KB, two TMEM accumulator buffers (the epilogue of a tile overlaps the next
// main loop).  MT = 2: 256 x bn tiles whose two MMAs share each B stage (a third
// fewer operand bytes per flop), 3 stages of 64 KB, one accumulator buffer of
// 2 x 256 columns.
//
// F8: e4m3 operands, both K-major, 128 elements (128 bytes) per stage row; the
// MMAs are block-scaled (kind::mxf8f6f4, one UE8M0 scale per 32 K-elements of a
// row or column), bn = 128 so that every MMA covers whole 128 x 128 scale
// tiles.  Each stage also carries the scale-factor images of its operand tiles
// (512 bytes each: the A tile of every M half, then the B tile), copied into
// tensor memory with tcgen05.cp before the stage's MMAs.  Because each image
// holds one byte value, every scale-factor cell an MMA reads holds the tile's
// scale whatever cell it reads.  Accumulators use columns [0, 128) and
// [256, 384); the scale factors of stage s sit at columns 384 + 16 s.
template <int MT, bool F8 = false>
struct Cfg {
    // e4m3 tiles are 128 columns wide (16 KB of B per stage), so their stages
    // are smaller and the ring deeper: 4 (256-row tiles) or 6 (128-row tiles)
    // stages keep more operand bytes in flight at the doubled MMA rate.
    static constexpr int STG = F8 ? (MT == 2 ? 4 : 6) : (MT == 2 ? 3 : 4);
    static constexpr int A_BYTES = MT * BM * BK * 2;
    static constexpr int STAGE = A_BYTES + (F8 ? 128 * BK * 2 : B_STAGE_BYTES);
    static constexpr int NACC = MT == 2 ? 1 : 2;
    static constexpr int TM = BM * MT;
    static constexpr int SF_STAGE = F8 ? (MT + 1) * 512 : 0;
    static constexpr int SMEM = STG * STAGE + 1024 + (F8 ? 1024 + STG * SF_STAGE : 256);
};
constexpr uint32_t SF_TMEM_COL = 384;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait.  Returns false when the limit expired or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit,
                                          volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
#pragma unroll 1
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Block-scaled e4m3 MMA: scale factors (UE8M0) for A rows and B columns in
// tensor memory at sfa / sfb.
__device__ __forceinline__ void tc_mma_mxf8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%5], [%6], p;\n\t}" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(sfa), "r"(sfb)
        : "memory");
}

// 32 rows x 16 bytes of shared memory (no swizzle) into tensor-memory columns
// [taddr, taddr + 4) of all four 32-lane groups.
__device__ __forceinline__ void tc_cp_32x128b_x4(uint32_t taddr, uint64_t sdesc) {
    asm volatile("tcgen05.cp.cta_group::1.32x128b.warpx4 [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}

// Non-tensor bulk copy global -> shared, completing bytes on an mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor for tcgen05 (128B swizzle, version 1).
//   start: shared address; lbo / sbo: leading / stride byte offsets.
__device__ __forceinline__ uint64_t smem_desc(uint32_t start, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((start & 0x3FFFF) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32;
    d |= static_cast<uint64_t>(1) << 46;   // descriptor version for tcgen05
    d |= static_cast<uint64_t>(2) << 61;   // SWIZZLE_128B
    return d;
}

// No-swizzle descriptor of a 32-row x 16-byte block (8-row core matrices of
// 128 contiguous bytes, 128 bytes apart).
__device__ __forceinline__ uint64_t smem_desc_plain(uint32_t start) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((start & 0x3FFFF) >> 4);
    d |= static_cast<uint64_t>(128 >> 4) << 16;
    d |= static_cast<uint64_t>(128 >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;   // layout type 0: no swizzle
}

// Instruction descriptor, kind::mxf8f6f4 (block-scaled): e4m3 A and B (format
// code 0), K-major, FP32 accumulator, UE8M0 scale factors; sf ids pick the
// byte of each 32-bit scale-factor cell.
__device__ __forceinline__ uint32_t instr_desc_mxf8(int m, int n, int sfa_id, int sfb_id) {
    return (static_cast<uint32_t>(sfb_id) << 4)     // B scale-factor id
           | (static_cast<uint32_t>(n >> 3) << 17)   // N / 8
           | (1u << 23)                              // scale type UE8M0
           | (static_cast<uint32_t>(m >> 4) << 24)   // M / 16
           | (static_cast<uint32_t>(sfa_id) << 29);  // A scale-factor id
}

// Instruction descriptor, kind::f16 with BF16 inputs and an FP32 accumulator.
__device__ __forceinline__ uint32_t instr_desc_bf16(int m, int n, int a_mn, int b_mn) {
    return (1u << 4)                                   // D format: F32
           | (1u << 7)                                 // A format: BF16
           | (1u << 10)                                // B format: BF16
           | (static_cast<uint32_t>(a_mn) << 15)       // A major-ness
           | (static_cast<uint32_t>(b_mn) << 16)       // B major-ness
           | (static_cast<uint32_t>(n >> 3) << 17)     // N / 8
           | (static_cast<uint32_t>(m >> 4) << 24);    // M / 16
}

struct TileCoord {
    int g, tm, tn;
    int half;   // 0: whole K range; c >= 1: part c of the K range (of ksplit parts, or of 2)
};

// GEMM descriptors and tensor maps live in the kernel parameters (up to
// TC_MAX_GEMMS GEMMs) or, in grouped mode, in device memory (any number of
// GEMMs; the batched path).  Tiles are numbered GEMM after GEMM (tile_base
// ascending).
template <bool GROUPED>
__device__ __forceinline__ const TcGemm* gemm_of(const TcParams& p, int i) {
    return GROUPED ? p.gg + i : p.g + i;
}
template <bool GROUPED>
__device__ __forceinline__ const CUtensorMap* map_of(const TcParams& p, int i) {
    return GROUPED ? p.gmaps + i : p.maps + i;
}

template <bool GROUPED>
__device__ __forceinline__ TileCoord decode_tile(const TcParams& p, int t) {
    // tiles_m / tiles_n / tile_base are in units of this launch's tile shape
    TileCoord c;
    c.half = 0;
    if (!GROUPED && p.nsplit > 0 && t >= p.split_base) {
        const int u = t - p.split_base;
        c.half = 1 + (u & 1);
        t = p.split_base + (u >> 1);
    }
    if (GROUPED) {   // last GEMM whose tile_base <= t
        int lo = 0, hi = p.ngemm - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.gg[mid].tile_base <= t) lo = mid; else hi = mid - 1;
        }
        c.g = lo;
    } else {
        c.g = 0;
#pragma unroll 1
        for (int i = 1; i < p.ngemm; ++i)
            if (t >= p.g[i].tile_base) c.g = i;
    }
    const TcGemm& G = *gemm_of<GROUPED>(p, c.g);
    const int local = t - G.tile_base;
    const int ctm_n = G.tiles_m;
    int ctm;
    if (!GROUPED && G.ksplit >= 2) {
        // the K parts of a tile are separate items; the items that share an
        // operand panel (same part) stay consecutive
        const int S = G.ksplit;
        if (G.a_mn) {
            ctm = local % ctm_n;
            const int v = local / ctm_n;
            c.half = 1 + v % S;
            c.tn = v / S;
        } else {
            c.tn = local % G.tiles_n;
            const int v = local / G.tiles_n;
            c.half = 1 + v % S;
            ctm = v / S;
        }
    } else if (G.a_mn) {   // A operand is the small sketch (Y^T): walk M fastest so the big B is shared
        ctm = local % ctm_n;
        c.tn = local / ctm_n;
    } else {        // walk N fastest so the big A row panel is shared
        ctm = local / G.tiles_n;
        c.tn = local % G.tiles_n;
    }
    c.tm = ctm;
    return c;
}

// K blocks of one work item: sequence positions [kb0, kb1), position j being
// K block kk0 + j % nk of source j / nk.  Whole tiles and parts of the joint
// sequence (ksplit without kpart) have nk = kblocks, kk0 = 0; a K-aligned part
// runs its K range for every source.
struct KRange {
    int kb0, kb1, nk, kk0;
};
__device__ __forceinline__ KRange k_range(const TcGemm& G, int half) {
    KRange r;
    if (half && G.kpart > 0) {
        r.kk0 = (half - 1) * G.kpart;
        r.nk = min(G.kpart, G.kblocks - r.kk0);
        r.kb0 = 0;
        r.kb1 = G.nsrc * r.nk;
    } else {
        const int nkb = G.nsrc * G.kblocks;
        const int S = G.ksplit >= 2 ? G.ksplit : 2;
        r.kb0 = half ? (half - 1) * nkb / S : 0;
        r.kb1 = half ? half * nkb / S : nkb;
        r.nk = G.kblocks;
        r.kk0 = 0;
    }
    return r;
}

// Tile of round k for CTA cid (boustrophedon order when snake).  Once a CTA's
// tile is past the end, so are all its later ones.
__device__ __forceinline__ int sched_tile(int k, int cid, int ncl, int snake) {
    return k * ncl + ((snake && (k & 1)) ? ncl - 1 - cid : cid);
}

__device__ void latch(int32_t* status, int code, int where, volatile int* abort_flag) {
    *abort_flag = 1;
    if (atomicCAS(&status[GN_DEV_STATUS], 0, code) == 0) status[GN_DEV_WHERE] = where;
}

// Every CTA loads its own operand tiles; CTAs exchange nothing.
template <bool GROUPED, int MT, bool F8>
__global__ void __launch_bounds__(NUM_THREADS, 1) tc_multigemm_kernel(const __grid_constant__ TcParams p) {
    using K = Cfg<MT, F8>;
    constexpr int KE = F8 ? 128 : BK;                     // K elements per stage (128 bytes per row)
    constexpr int STAGES = K::STG;
    constexpr int STAGE_BYTES = K::STAGE;
    constexpr int A_STAGE_BYTES = K::A_BYTES;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;            // 1024-aligned stage ring
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t bars = base + STAGES * STAGE_BYTES;        // barrier block
    const uint32_t sfs = bars + 1024;                         // F8: scale-factor images per stage
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
    auto tfull_bar = [&](int a) { return bars + 8u * (2 * STAGES + a); };
    auto tempty_bar = [&](int a) { return bars + 8u * (2 * STAGES + 2 + a); };
    const uint32_t final_bar = bars + 8u * (2 * STAGES + 4);
    const uint32_t stall_bar = bars + 8u * (2 * STAGES + 6);   // never completed (timeout-path test)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + STAGES * STAGE_BYTES + 8 * (2 * STAGES + 5));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const unsigned long long limit = p.wait_limit_ns;
    // Draining the CTA's own copies and MMAs (which always complete) before its
    // shared and tensor memory are released keeps at least a second, however
    // short the limit on waits for other roles.
    const unsigned long long drain = limit > 1000000000ULL ? limit : 1000000000ULL;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < K::NACC; ++a) {
            mbar_init(tfull_bar(a), 1);
            mbar_init(tempty_bar(a), 128);
        }
        mbar_init(final_bar, 1);
        mbar_init(stall_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int cid = blockIdx.x, ncl = gridDim.x;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int stage = 0;
            uint32_t ephase = 0;
            uint32_t issued_mask = 0;            // stages that ever received a load
            uint32_t last_parity = 0;            // parity of the last armed phase per stage
            bool ok = true;
            for (int k = 0, t = sched_tile(0, cid, ncl, p.snake); t < p.total_tiles && ok; t = sched_tile(++k, cid, ncl, p.snake)) {
                const TileCoord c = decode_tile<GROUPED>(p, t);
                const TcGemm& G = *gemm_of<GROUPED>(p, c.g);
                const KRange kr = k_range(G, c.half);
                const uint32_t bytes = A_STAGE_BYTES + G.bn * BK * 2 + K::SF_STAGE;
                for (int kb = kr.kb0; kb < kr.kb1; ++kb) {
                    if (!mbar_wait(empty_bar(stage), ephase ^ 1u, limit, abort_flag)) {
                        latch(p.status, GN_ERR_TIMEOUT, 1, abort_flag);
                        ok = false;
                        break;
                    }
                    const int src = kb / kr.nk;
                    const int kk = kr.kk0 + (kb - src * kr.nk);
                    const CUtensorMap* ma = map_of<GROUPED>(p, G.a_map[src]);
                    const CUtensorMap* mb = map_of<GROUPED>(p, G.b_map[src]);
                    if (GROUPED && kk == 0) {   // maps written to device memory before the launch
                        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                                         reinterpret_cast<uint64_t>(ma))
                                     : "memory");
                        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                                         reinterpret_cast<uint64_t>(mb))
                                     : "memory");
                    }
                    const uint32_t sa = base + stage * STAGE_BYTES;
                    const uint32_t sb = sa + A_STAGE_BYTES;
                    const uint32_t fb = full_bar(stage);
                    mbar_arrive_expect_tx(fb, bytes);
                    issued_mask |= 1u << stage;
                    last_parity = (last_parity & ~(1u << stage)) | (ephase << stage);
#pragma unroll
                    for (int hh = 0; hh < MT; ++hh) {
                        const int m0 = c.tm * K::TM + hh * BM;
                        if (!F8 && G.a_mn) {
                            tma_load_2d(sa + hh * 16384, ma, fb, m0, kk * BK);
                            tma_load_2d(sa + hh * 16384 + 8192, ma, fb, m0 + 64, kk * BK);
                        } else {
                            tma_load_2d(sa + hh * 16384, ma, fb, kk * KE, m0);
                        }
                        if (F8) {   // scale-factor image of this A tile
                            const int rb = min(m0 / BM, G.sfa_rows - 1);
                            const long long ti = G.sfa_tr ? static_cast<long long>(kk) * G.sfa_ld + rb
                                                          : static_cast<long long>(rb) * G.sfa_ld + kk;
                            bulk_load(sfs + stage * K::SF_STAGE + hh * 512, G.sfa + ti * 512, 512, fb);
                        }
                    }
                    if (F8) {       // and of the B tile (bn = 128: one tile)
                        const int rb = min(c.tn * G.bn / BM, G.sfb_rows - 1);
                        const long long ti = G.sfb_tr ? static_cast<long long>(kk) * G.sfb_ld + rb
                                                      : static_cast<long long>(rb) * G.sfb_ld + kk;
                        bulk_load(sfs + stage * K::SF_STAGE + MT * 512, G.sfb + ti * 512, 512, fb);
                    }
                    if (G.b_mn) {
                        for (int j = 0; j < G.bn / 64; ++j)
                            tma_load_2d(sb + 8192 * j, mb, fb, c.tn * G.bn + 64 * j, kk * BK);
                    } else {
                        tma_load_2d(sb, mb, fb, kk * KE, c.tn * G.bn);
                    }
                    if (++stage == STAGES) {
                        stage = 0;
                        ephase ^= 1u;
                    }
                }
            }
            // Drain: every armed stage must have landed before shared memory is released.
            for (int s = 0; s < STAGES; ++s)
                if (issued_mask & (1u << s)) {
                    volatile int no_abort = 0;
                    if (!mbar_wait(full_bar(s), (last_parity >> s) & 1u, drain, &no_abort))
                        latch(p.status, GN_ERR_TIMEOUT, 2, abort_flag);
                }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t fphase = 0;
            int acc = 0;
            uint32_t aphase = 0;
            bool ok = true;
            bool issued_any = false;
            for (int k = 0, t = sched_tile(0, cid, ncl, p.snake); t < p.total_tiles && ok; t = sched_tile(++k, cid, ncl, p.snake)) {
                const TileCoord c = decode_tile<GROUPED>(p, t);
                const TcGemm& G = *gemm_of<GROUPED>(p, c.g);
                const KRange kr = k_range(G, c.half);
                const int kb0 = kr.kb0, kb1 = kr.kb1;
                const uint32_t idesc = F8 ? 0u : instr_desc_bf16(BM, G.bn, G.a_mn, G.b_mn);
                if (!mbar_wait(tempty_bar(acc), aphase ^ 1u, limit, abort_flag)) {
                    latch(p.status, GN_ERR_TIMEOUT, 3, abort_flag);
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + acc * MT * 256;
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(full_bar(stage), fphase, limit, abort_flag)) {
                        latch(p.status, GN_ERR_TIMEOUT, 4, abort_flag);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + stage * STAGE_BYTES;
                    const uint32_t sb = sa + A_STAGE_BYTES;
                    if (F8) {
                        // scale factors of this stage into tensor memory (ordered
                        // before the MMAs below: same issuing thread), then
                        // 4 K-steps of 32 e4m3 (32 bytes) per M half
                        const uint32_t sfs_s = sfs + stage * K::SF_STAGE;
                        const uint32_t tsf = tmem_base + SF_TMEM_COL + 16u * stage;
#pragma unroll
                        for (int hh = 0; hh < MT; ++hh) tc_cp_32x128b_x4(tsf + 4u * hh, smem_desc_plain(sfs_s + 512u * hh));
                        tc_cp_32x128b_x4(tsf + 8u, smem_desc_plain(sfs_s + 512u * MT));
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint64_t bd = smem_desc(sb + 32u * k, 16u, 1024u);
                            const uint32_t id = instr_desc_mxf8(BM, G.bn, k, k);
#pragma unroll
                            for (int hh = 0; hh < MT; ++hh)
                                tc_mma_mxf8(d_tmem + 256u * hh, smem_desc(sa + 16384u * hh + 32u * k, 16u, 1024u), bd, id,
                                            tsf + 4u * hh, tsf + 8u, (kb != kb0 || k != 0) ? 1u : 0u);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k) {
                            const uint64_t bd = G.b_mn ? smem_desc(sb + 2048u * k, 8192u, 1024u)
                                                       : smem_desc(sb + 32u * k, 16u, 1024u);
#pragma unroll
                            for (int hh = 0; hh < MT; ++hh) {
                                const uint32_t sah = sa + 16384u * hh;
                                const uint64_t ad = G.a_mn ? smem_desc(sah + 2048u * k, 8192u, 1024u)
                                                           : smem_desc(sah + 32u * k, 16u, 1024u);
                                tc_mma_bf16(d_tmem + 256u * hh, ad, bd, idesc, (kb != kb0 || k != 0) ? 1u : 0u);
                            }
                        }
                    }
                    issued_any = true;
                    tc_commit(empty_bar(stage));
                    if (++stage == STAGES) {
                        stage = 0;
                        fphase ^= 1u;
                    }
                }
                if (!ok) break;
                tc_commit(tfull_bar(acc));
                if (++acc == K::NACC) {
                    acc = 0;
                    aphase ^= 1u;
                }
            }
            if (issued_any) {   // all MMAs complete before tensor memory is released
                tc_commit(final_bar);
                volatile int no_abort = 0;
                if (!mbar_wait(final_bar, 0, drain, &no_abort))
                    latch(p.status, GN_ERR_TIMEOUT, 5, abort_flag);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;   // TMEM lane quarter this warp may access
        int acc = 0;
        uint32_t aphase = 0;
        bool stalled = false;
        if (p.stall_test) {   // a wait that nothing can satisfy: runs out at the limit
            stalled = !mbar_wait(stall_bar, 0, limit, abort_flag);
            if (stalled && lane == 0) latch(p.status, GN_ERR_TIMEOUT, 7, abort_flag);
        }
        for (int k = 0, t = sched_tile(0, cid, ncl, p.snake); t < p.total_tiles && !stalled; t = sched_tile(++k, cid, ncl, p.snake)) {
            const TileCoord c = decode_tile<GROUPED>(p, t);
            const TcGemm& G = *gemm_of<GROUPED>(p, c.g);
            const bool got = mbar_wait(tfull_bar(acc), aphase, limit, abort_flag);
            if (!__all_sync(0xffffffffu, got)) {   // warp-uniform exit: tcgen05.ld is .sync.aligned
                if (lane == 0) latch(p.status, GN_ERR_TIMEOUT, 6, abort_flag);
                break;
            }
            tc_fence_after();
#pragma unroll 1
            // part c of a K range split into stored parts goes to its own copy of D
            const bool stored_part = c.half && G.ksplit >= 2 && G.part_stride > 0;
            float* Dbase = stored_part ? G.D + (c.half - 1) * G.part_stride : G.D;
            for (int hh = 0; hh < MT; ++hh) {
                const int row = c.tm * K::TM + hh * BM + q * 32 + lane;
                const bool row_ok = row < G.M;
                float* drow = Dbase + static_cast<long long>(row_ok ? row : 0) * G.ldd;
                for (int c0 = 0; c0 < G.bn; c0 += 32) {
                    uint32_t v[32];
                    tmem_ld32(tmem_base + (static_cast<uint32_t>(q * 32) << 16) + (acc * MT + hh) * 256 + c0, v);
                    const int col0 = c.tn * G.bn + c0;
                    if (!row_ok || col0 >= G.N) continue;
                    // columns of this chunk inside both the tile and D
                    const int ncol = min(min(32, G.bn - c0), G.N - col0);
                    if (c.half && !stored_part) {   // part of the K range: add into the pre-zeroed D
                        if (G.vec4 && ncol == 32) {
                            float4* dst = reinterpret_cast<float4*>(drow + col0);
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                atomicAdd(dst + j, make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                                               __uint_as_float(v[4 * j + 2]),
                                                               __uint_as_float(v[4 * j + 3])));
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (j < ncol) atomicAdd(drow + col0 + j, __uint_as_float(v[j]));
                        }
                    } else if (G.vec4 && ncol == 32) {
                        float4* dst = reinterpret_cast<float4*>(drow + col0);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                                 __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < ncol) drow[col0 + j] = __uint_as_float(v[j]);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(tempty_bar(acc));
            if (++acc == K::NACC) {
                acc = 0;
                aphase ^= 1u;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

}  // namespace

gn_status tc_make_map_bf16(CUtensorMap* map, const void* base, long long rows, long long cols,
                           long long ld, int box_cols, int box_rows) {
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 2) % 16 != 0) return GN_ERR_ALIGNMENT;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return GN_ERR_CUDA;
    memset(map, 0, sizeof(*map));
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * 2)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GN_OK : GN_ERR_CUDA;
}

gn_status tc_make_map_e4m3(CUtensorMap* map, const void* base, long long rows, long long cols, long long ld,
                           int box_rows) {
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || ld % 16 != 0) return GN_ERR_ALIGNMENT;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return GN_ERR_CUDA;
    memset(map, 0, sizeof(*map));
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld)};
    cuuint32_t box[2] = {128u, static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GN_OK : GN_ERR_CUDA;
}

template <bool GROUPED, int MT, bool F8 = false>
gn_status launch_cfg(gn_handle h, const TcParams& p, int total_tiles) {
    static bool attr_set = false;
    if (!attr_set) {
        GN_CUDA_TRY(cudaFuncSetAttribute(tc_multigemm_kernel<GROUPED, MT, F8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<MT, F8>::SMEM));
        attr_set = true;
    }
    int ctas = total_tiles < h->sm_count ? total_tiles : h->sm_count;
    if (p.max_ctas > 0 && p.max_ctas < ctas) ctas = p.max_ctas;
    tc_multigemm_kernel<GROUPED, MT, F8><<<ctas, NUM_THREADS, Cfg<MT, F8>::SMEM, h->stream>>>(p);
    count_launch();
    GN_CUDA_TRY(cudaGetLastError());
    return GN_OK;
}

// Tile shape: 256-row tiles (two MMAs sharing each B stage) when every GEMM has
// at least 256 rows and the launch keeps enough tiles, else 128-row tiles.
int pick_mt(const TcGemm* g, int ngemm, int sm_count) {
    long long tiles2 = 0;   // work items with 256-row tiles (a K-split tile counts twice)
    for (int i = 0; i < ngemm; ++i) {
        if (g[i].M < 2 * BM) return 1;
        tiles2 += ((g[i].M + 2 * BM - 1) / (2 * BM)) * ((g[i].N + g[i].bn - 1) / g[i].bn) * (g[i].ksplit >= 2 ? g[i].ksplit : 1);
    }
    return tiles2 >= 4LL * sm_count ? 2 : 1;   // keep enough tiles to fill the GPU
}

gn_status tc_launch(gn_handle h, TcParams* p) {
    const int MT = pick_mt(p->g, p->ngemm, h->sm_count);
    for (int i = 0; i < p->ngemm; ++i) {
        if (p->f8 && (p->g[i].a_mn || p->g[i].b_mn || p->g[i].bn != 128 || p->g[i].nsrc != 1 || !p->g[i].sfa ||
                      !p->g[i].sfb || p->g[i].sfa_rows < 1 || p->g[i].sfb_rows < 1))
            return GN_ERR_INVALID_ARG;
        GN_TRY(tc_prepare_gemm(&p->g[i], 0, MT, p->f8));
    }
    int total = 0;
    for (int i = 0; i < p->ngemm; ++i) {
        TcGemm& G = p->g[i];
        // parts that add into D need enough K to pay; stored parts are the caller's layout
        if (G.ksplit >= 2 && G.part_stride == 0 && (p->f8 || G.nsrc * G.kblocks < 4 * G.ksplit)) G.ksplit = 1;
        if (G.ksplit >= 2 && G.part_stride > 0 && G.nsrc * G.kblocks < G.ksplit) return GN_ERR_INVALID_ARG;
        G.tile_base = total;
        total += G.tiles_m * G.tiles_n * (G.ksplit >= 2 ? G.ksplit : 1);
        if (G.ksplit >= 2 && G.part_stride == 0)   // the parts add into D
            GN_CUDA_TRY(cudaMemset2DAsync(G.D, sizeof(float) * G.ldd, 0, sizeof(float) * G.N, G.M, h->stream));
    }
    // Balance the last round: when the tiles leave a partial round of R tiles
    // (R <= half the CTAs) that are whole rows of tiles of the last GEMM with A
    // K-major (a contiguous row range of its D), those R tiles run as 2R half-K
    // items adding into D, zeroed first; the last round then costs half a tile.
    p->split_base = 0;
    p->nsplit = 0;
    p->snake = p->snake_groups > 0 ? 1 : 0;
    p->max_ctas = p->snake ? p->snake_groups * p->g[0].tiles_m * p->g[0].tiles_n * std::max(1, p->g[0].ksplit) : 0;
    if (!p->f8 && !p->snake && total > 0) {
        const int ncl = std::min(total, h->sm_count);
        const int R = total % ncl;
        const TcGemm& G = p->g[p->ngemm - 1];
        if (total > ncl && R > 0 && 2 * R <= ncl && !G.a_mn && G.ksplit < 2 && R % G.tiles_n == 0 &&
            G.nsrc * G.kblocks >= 8) {
            const long long row0 = static_cast<long long>(G.tiles_m - R / G.tiles_n) * BM * MT;
            if (row0 >= 0 && row0 < G.M) {
                GN_CUDA_TRY(cudaMemset2DAsync(G.D + row0 * G.ldd, sizeof(float) * G.ldd, 0, sizeof(float) * G.N,
                                              G.M - row0, h->stream));
                p->split_base = total - R;
                p->nsplit = R;
                total += R;
            }
        }
    }
    p->total_tiles = total;
    p->gg = nullptr;
    p->gmaps = nullptr;
    p->status = h->dstatus;
    p->wait_limit_ns = h->wait_limit_ns;
    p->stall_test = h->stall_test;
    if (total == 0) return GN_OK;
    if (p->f8) return MT == 2 ? launch_cfg<false, 2, true>(h, *p, total) : launch_cfg<false, 1, true>(h, *p, total);
    return MT == 2 ? launch_cfg<false, 2>(h, *p, total) : launch_cfg<false, 1>(h, *p, total);
}

gn_status tc_prepare_gemm(TcGemm* G, int tile_base, int mt, int f8) {
    if (G->bn < 16 || G->bn > 256 || (G->b_mn && G->bn % 64) || G->bn % 16) return GN_ERR_INVALID_ARG;
    const int ke = f8 ? 128 : BK;
    G->tiles_m = static_cast<int>((G->M + BM * mt - 1) / (BM * mt));
    G->tiles_n = static_cast<int>((G->N + G->bn - 1) / G->bn);
    G->kblocks = static_cast<int>((G->K + ke - 1) / ke);
    G->tile_base = tile_base;
    G->vec4 = ((reinterpret_cast<uintptr_t>(G->D) & 15) == 0 && G->ldd % 4 == 0) ? 1 : 0;
    return GN_OK;
}

gn_status tc_launch_grouped(gn_handle h, const TcGemm* dev_gemms, int ngemm, const CUtensorMap* dev_maps,
                            int total_tiles, int mt) {
    if (total_tiles <= 0 || ngemm <= 0) return GN_OK;
    TcParams p;
    memset(&p, 0, sizeof(p));
    p.gg = dev_gemms;
    p.gmaps = dev_maps;
    p.ngemm = ngemm;
    p.total_tiles = total_tiles;
    p.status = h->dstatus;
    p.wait_limit_ns = h->wait_limit_ns;
    return mt == 2 ? launch_cfg<true, 2>(h, p, total_tiles) : launch_cfg<true, 1>(h, p, total_tiles);
}

}  // namespace gn

// Shared pieces of the tcgen05 complex-as-real GEMM (Sec. 3.3, Eq. 5-6):
// PTX wrappers (mbarriers with bounded waits, TMA, tcgen05.mma / commit /
// ld, shared-memory descriptors), the per-launch argument block, the tile
// walk, and the epilogue's store of one 16-column accumulator chunk.  Used by
// the stand-alone GEMM launches (tc_gemm.cu) and by the work-queue kernel
// (queue.cu), so both compute the same values with the same roundings.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.cuh"

namespace tn {

// Host: 3-D tiled tensor map over [depth][rows][inner] elements of esz bytes
// (2: FP16/BF16 by dtype, 1: E4M3) with a box_inner x box_rows box and the
// swizzle that matches box_inner * esz (32, 64 or 128 bytes); false on failure.
bool tc_encode_3d(CUtensorMap *m, int dtype, int esz, const void *base, uint64_t inner, uint64_t rows,
                  uint64_t depth, uint32_t box_inner, uint32_t box_rows);
// Host: the raster group (m tiles) the launcher picks for an N tile of bn.
int tc_default_gm(int bn);


constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait
constexpr int kEpiThreads = 256;                  // warps 2..9
constexpr int kTcThreads = 64 + kEpiThreads;      // producer, MMA, epilogue

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// CL: cluster-scope acquire (barriers that CTA-pair peers arrive on).
// The thread may be suspended in the instruction until the phase completes,
// for at most kSuspendNs (it resumes as soon as the phase completes), so a
// waiting warp issues few instructions.
constexpr uint32_t kSuspendNs = 20000;

template <bool CL = false>
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    if constexpr (CL)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
            : "memory");
    return ok != 0;
}

// bounded wait: returns false (and raises the CTA abort flag) on timeout or
// when another role already aborted
template <bool CL = false>
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait<CL>(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait<CL>(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            return false;
        }
    }
}

// ---- CTA pairs (cluster of 2): one tcgen05.mma with M = 256 spans both SMs
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the same shared variable in CTA `rank`
__device__ __forceinline__ uint32_t mapa_rank(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// CTA pair: the tile lands in this CTA's shared memory, its byte count on the
// leader CTA's barrier (bar_cluster: a shared::cluster address)
__device__ __forceinline__ void tma_load_3d_pair(void *dst, const CUtensorMap *map, uint32_t bar_cluster,
                                                 int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar_cluster)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// completion of this thread's earlier tcgen05 ops arrives on `bar`; a CTA
// pair arrives on the barrier at the same offset in both CTAs
template <bool PAIR = false>
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    if constexpr (PAIR)
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
            " [%0], %1;" ::"r"(smem_u32(bar)),
            "h"((uint16_t)3)
            : "memory");
    else
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(bar))
                     : "memory");
}

// the same, on this CTA's barrier only
__device__ __forceinline__ void tc_commit_pair_local(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

template <bool F8, bool PAIR>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
    if constexpr (F8 && PAIR)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else if constexpr (F8)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else if constexpr (PAIR)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
}

// kind::tf32 (FP32 words read as TF32, FP32 accumulation), one CTA
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// K-major shared-memory matrix descriptor (tcgen05): start address, leading
// byte offset (unused for swizzled K-major), stride byte offset = 8 rows,
// descriptor version 1, swizzle mode.  BKB: bytes of one K chunk row.
template <int BKB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    constexpr uint32_t row_bytes = BKB;                // one swizzle row
    constexpr uint32_t sbo = 8 * row_bytes;            // 8-row core-matrix group
    constexpr uint64_t layout = BKB == 128 ? 2 : (BKB == 64 ? 4 : 6);  // 128B / 64B / 32B
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                            // LBO (16 B, ignored)
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;                            // version
    d |= layout << 61;
    return d;
}

template <int N>
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ int scale_exp_tc(float maxa, float maxb, int lk) {
    const float t = 2.0f * maxa * maxb;
    if (!(t > 0.0f) || !isfinite(t)) return 0;
    int x;
    const float f = frexpf(t, &x);
    const int c = (f == 0.5f) ? x - 1 : x;
    int e = 14 - lk - c;
    return max(-120, min(120, e));
}

struct TcArgs {
    void *C;
    int64_t M;
    int64_t n_mt;          // m tiles per batch
    int n_nt;              // n tiles
    int64_t batch;
    int64_t tiles;
    int N;                 // complex columns
    int lk;
    int nk;                // K chunks
    int dtype;
    int batch_a, batch_b;
    int gm;                // m tiles per raster group
    int withhold;          // self-test: issue no loads, so consumers' waits run out
    int out_c64;           // C stored complex64 (no rounding, e = 0)
    int split;             // K parts (split-K); tiles of part p cover K chunks [p*nk, (p+1)*nk)
    float *partial;        // split > 1: FP32 partial sums [part][batch][M][N] complex
    int64_t tiles_per_part;
    // sparse-state gathers (Sec. 3.4.2): per batch entry b the A chunk za[b],
    // the B' chunk zb[b] and the output chunk zc[b] (< 0: not stored); NULL:
    // the batch entry itself
    const int32_t *za, *zb, *zc;
    int gather_r;          // > 0: B' tile = gather_r chunks (padded 2-D index), zb/zc [batch][m_r]
    int m_r, np_chunk;
    // > 0: C stored in a permuted mode order: bit i of the natural element
    // index goes to bit out_dpos[i] (bits 0..2 stay)
    int out_rank;
    int8_t out_dpos[40];
    int ln;                // log2 N (bit position of the row part of an element index)
    int staged;            // 1: complex-half results by tc_store_block (where tc_staged_ok)
    ScaleRef sr;
    int32_t *err;
};

// Tile t -> (batch, m tile, n tile).  Tiles go in groups of `gm` m-tiles:
// inside a group the m index runs fastest, so the tiles in flight at once
// cover about gm m-tiles x (SMs / gm) n-tiles, whose A rows and B' columns
// fit in L2 together; A and B' are then read from DRAM about once per group
// instead of once per m-tile.
// Bits lo..hi-1 of a C element index moved to the consumer's mode order
// (the fused permutation is a bit permutation, so the parts OR together).
// Host: tensor maps and argument block of one tensor-core step exactly as
// launch_gemm_tc runs it (one_cta: never on CTA pairs); bn, bk: the N tile
// (real columns) and the K chunk (elements) the tensor maps were encoded for.
// cudaErrorInvalidValue for shapes the kernel does not take.
cudaError_t tc_setup(const TcGemmDesc &d, const ScaleRef &sr, int32_t *d_err, bool one_cta, CUtensorMap *ma,
                     CUtensorMap *mb, TcArgs *a, int *bn, int *bk, bool *pair);

__device__ __forceinline__ int64_t permute_bits(const TcArgs &a, int64_t e, int lo, int hi) {
    int64_t d = 0;
    for (int i = lo; i < hi; ++i) d |= ((e >> i) & 1) << a.out_dpos[i];
    return d;
}

__device__ __forceinline__ void tile_coords(const TcArgs &a, int64_t t, int64_t &b, int64_t &mt,
                                            int &nt) {
    t %= a.tiles_per_part;          // the K part is t / tiles_per_part
    const int64_t per_batch = a.n_mt * a.n_nt;
    b = t / per_batch;
    const int64_t r = t - b * per_batch;
    const int64_t span = (int64_t)a.gm * a.n_nt;
    const int64_t g = r / span;
    const int64_t in = r - g * span;
    const int64_t gm = min((int64_t)a.gm, a.n_mt - g * a.gm);
    mt = g * a.gm + in % gm;
    nt = (int)(in / gm);
}

// BROWS: rows of the B' tile this CTA holds (BN, or BN / 2 in a CTA pair)
template <int BROWS, int BKB, int STAGES>
struct TcSmem {
    static constexpr int a_bytes = 128 * BKB;
    static constexpr int b_bytes = BROWS * BKB;
    static constexpr int stage_bytes = (a_bytes + b_bytes + 1023) / 1024 * 1024;
    static constexpr int ring = STAGES * stage_bytes;
    static constexpr int bars = (2 * STAGES + 5) * 8;
    // epilogue staging (tc_store_block): 8 warps x 32 rows x 128 bytes, after
    // the barriers
    static constexpr int stg = ring + 1024;
    static constexpr int total = 1024 + stg + 8 * 4096;   // + alignment slack
    static_assert(bars + 16 <= 1024, "barriers overflow their kilobyte");
    static_assert(total <= 232448, "over the 227 KiB of shared memory a CTA may have");
};

// One tcgen05.ld of the epilogue: 16 accumulator columns of this thread's
// row m (real columns col0 + c .. col0 + c + 15 of the output tile; col_end
// bounds the tile's real columns), scaled by sc (an exact 2^e), rounded to
// the plan's complex-half type (or kept FP32 for a complex64 result or a
// split-K partial) and stored interleaved; mx tracks max |stored value|.
// cb: output chunk of the tile's batch entry; prow: the row part of the
// fused output permutation (out_rank > 0); t: the tile (its K part).
__device__ __forceinline__ void tc_store16(const TcArgs &args, const uint32_t (&r)[16], int64_t b, int64_t m,
                                           int64_t t, int col0, int c, int col_end, int64_t cb, int64_t prow,
                                           const int64_t (&lowtab)[8], bool low_kept, float sc, float &mx) {
    int64_t cbk = cb;              // output chunk of these 16 columns
    int colr = col0 + c;           // their first real column in that chunk
    int nreal = min(16, col_end - c);
    if (args.gather_r) {
        const int gcol = col0 + c, rr = gcol / args.np_chunk;
        colr = gcol - rr * args.np_chunk;
        cbk = rr < args.m_r ? (int64_t)args.zc[b * args.m_r + rr] : -1;
        nreal = min(16, 2 * args.N - colr);
    }
    if (cbk < 0 || nreal <= 0) {
        // padded place of the 2-D index (or padding of B'): computed, not stored
    } else if (m < args.M && (args.out_c64 || args.partial)) {
        // complex64 result (or split-K partial): the FP32 accumulators as they are
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            v[j] = __uint_as_float(r[j]);
            if (j < nreal) mx = fmaxf(mx, fabsf(v[j]));
        }
        const int64_t part = t / args.tiles_per_part;
        const int64_t ei = (cbk * args.M + m) * (int64_t)args.N + colr / 2;
        float *dst = args.partial
                         ? args.partial + (((part * args.batch + b) * args.M + m) * (int64_t)args.N +
                                           colr / 2) * 2
                         : reinterpret_cast<float *>(args.C) + ei * 2;
        if (args.out_rank) {
            // 8 complex values, each to its permuted place
            const int64_t base = prow | permute_bits(args, colr / 2, 3, args.ln);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                reinterpret_cast<float2 *>(args.C)[base | lowtab[j]] = make_float2(v[2 * j], v[2 * j + 1]);
        } else if (nreal >= 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (4 * q < nreal)
                    reinterpret_cast<float4 *>(dst)[q] =
                        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
            reinterpret_cast<float2 *>(dst)[0] = make_float2(v[0], v[1]);
        }
    } else if (m < args.M) {
        // nreal: 2, 4, 8 or 16
        uint32_t packed[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float re = __uint_as_float(r[2 * j]) * sc;
            const float im = __uint_as_float(r[2 * j + 1]) * sc;
            float2 back;
            if (args.dtype == TN_BF16) {
                __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
                packed[j] = *reinterpret_cast<uint32_t *>(&h);
                back = __bfloat1622float2(h);
            } else {
                __half2 h = __floats2half2_rn(re, im);
                packed[j] = *reinterpret_cast<uint32_t *>(&h);
                back = __half22float2(h);
            }
            if (2 * j < nreal) mx = fmaxf(mx, fmaxf(fabsf(back.x), fabsf(back.y)));
        }
        const int64_t ei = (cbk * args.M + m) * (int64_t)args.N + colr / 2;
        uint32_t *dst = reinterpret_cast<uint32_t *>(args.C) + ei;
        if (args.out_rank) {
            const int64_t base = prow | permute_bits(args, colr / 2, 3, args.ln);
            if (low_kept) {
                uint4 *d4 = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(args.C) + base);
                d4[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                d4[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    reinterpret_cast<uint32_t *>(args.C)[base | lowtab[j]] = packed[j];
            }
        } else if (nreal == 16) {
            reinterpret_cast<uint4 *>(dst)[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            reinterpret_cast<uint4 *>(dst)[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        } else if (nreal == 8) {
            reinterpret_cast<uint4 *>(dst)[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        } else if (nreal == 4) {
            reinterpret_cast<uint2 *>(dst)[0] = make_uint2(packed[0], packed[1]);
        } else {
            dst[0] = packed[0];
        }
    }
}

// Staged stores of complex-half results (no complex64 result, no split-K
// partial, no 2-D gather index, a fused permutation that keeps the low 3
// bits).  tc_store16 has each thread store its own row, so a warp's 16-byte
// stores land in 32 different rows: every store instruction becomes 32
// partial-sector requests to L2.  Here a warp rounds the w real columns (16,
// 32 or 64) of block c of its 32 rows into a 32 x 128-byte staging area of
// its own (16-byte unit u of row r at unit u ^ (r & 7): conflict-free both
// ways), then writes them row segment by row segment: one instruction covers
// 32 / (w / 8) rows x 2w bytes, whole 32-byte sectors.  Values, rounding and
// the running max are tc_store16's.  taddr: the warp's TMEM lane quadrant and
// accumulator; m: this lane's row; prow: its row part of the fused
// permutation; cb: output chunk (>= 0).  Which of the two store paths wins
// depends on the step: the autotuner times both (tile bit 12).
__device__ __forceinline__ bool tc_staged_ok(const TcArgs &a, bool low_kept) {
    return !a.out_c64 && !a.partial && !a.gather_r && a.ln >= 3 && (a.out_rank == 0 || low_kept);
}

__device__ __forceinline__ void tc_store_block(const TcArgs &args, uint32_t taddr, int c, int w, int64_t m,
                                               int lane, int col0, int64_t cb, int64_t prow, float sc, float &mx,
                                               uint8_t *stg) {
    uint8_t *line = stg + lane * 128;
    for (int cc = 0; cc < w; cc += 16) {
        uint32_t r[16];
        tmem_ld16<16>(taddr + (uint32_t)(c + cc), r);
        tmem_wait_ld();
        uint32_t packed[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float re = __uint_as_float(r[2 * j]) * sc;
            const float im = __uint_as_float(r[2 * j + 1]) * sc;
            float2 back;
            if (args.dtype == TN_BF16) {
                __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
                packed[j] = *reinterpret_cast<uint32_t *>(&h);
                back = __bfloat1622float2(h);
            } else {
                __half2 h = __floats2half2_rn(re, im);
                packed[j] = *reinterpret_cast<uint32_t *>(&h);
                back = __half22float2(h);
            }
            if (m < args.M) mx = fmaxf(mx, fmaxf(fabsf(back.x), fabsf(back.y)));
        }
        const int u = cc >> 3;
        *reinterpret_cast<uint4 *>(line + ((u ^ (lane & 7)) << 4)) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        *reinterpret_cast<uint4 *>(line + (((u + 1) ^ (lane & 7)) << 4)) =
            make_uint4(packed[4], packed[5], packed[6], packed[7]);
    }
    __syncwarp();
    const int lu = w == 64 ? 3 : (w == 32 ? 2 : 1);     // log2 of 16-byte units per row
    const int u = lane & ((1 << lu) - 1);
    const int64_t m0 = m - lane;
    const int64_t jc = (int64_t)((col0 + c) >> 1) + 4 * u;   // first complex column of this unit
    const int64_t colpart = args.out_rank ? (permute_bits(args, jc, 3, args.ln) | (jc & 7)) : 0;
    uint32_t *C = reinterpret_cast<uint32_t *>(args.C);
    for (int i = 0; i < 32; i += 32 >> lu) {
        const int rr = i + (lane >> lu);
        const uint4 v = *reinterpret_cast<const uint4 *>(stg + rr * 128 + ((u ^ (rr & 7)) << 4));
        const int64_t pr = __shfl_sync(0xffffffffu, prow, rr);
        const int64_t mr = m0 + rr;
        if (mr < args.M) {
            const int64_t ei = args.out_rank ? (pr | colpart) : (cb * args.M + mr) * (int64_t)args.N + jc;
            *reinterpret_cast<uint4 *>(C + ei) = v;
        }
    }
    __syncwarp();
}

}  // namespace tn

// Complex-half contraction step on the 5th-generation tensor cores.
//
// Paper Sec. 3.3 (Eq. 5-6): the large operand A keeps its interleaved
// real/imag mode as an extra reduced mode, so A[M][K] complex is read as a
// real [M][2K] matrix with no copy; the small operand is padded to
// B'[(n,co)][(k,ci)] = [[Re, -Im], [Im, Re]] (bprep), and ONE real GEMM
// C'[M][2N] = A'[M][2K] B'^T gives C[M][N] complex, interleaved, exactly the
// four real products of the complex multiply (8 M N K real flops).
//
// Blackwell mapping (sm_103a):
//   * warp 0      : TMA producer -- cp.async.bulk.tensor tiles of A' and B'
//                   into a STAGES-deep shared-memory ring (K-major, swizzled),
//                   completion counted on mbarriers;
//   * warp 1      : allocates TMEM and issues tcgen05.mma kind::f16
//                   (M=128, N=BN, K=16 per instruction, FP32 accumulate in
//                   TMEM), double-buffered accumulators, tcgen05.commit frees
//                   ring stages and publishes finished tiles; the FP8
//                   variant issues kind::f8f6f4 with E4M3 operands (K=32);
//   * warps 2..9  : epilogue, two warps per TMEM lane quadrant taking
//                   alternate 16-column chunks (one warp per scheduler left
//                   short-K steps bound by the epilogue's own latency) --
//                   tcgen05.ld rows out of TMEM, exact 2^e scale,
//                   round to FP16/BF16, record max |C| for the next step's
//                   exponent, store interleaved complex-half rows.
// Persistent: one CTA per SM walks tiles (batch, m-tile, n-tile).
// Every mbarrier wait is bounded by wall time (globaltimer); on expiry the
// CTA records an error, drains, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "tc_common.cuh"

namespace tn {

namespace {

// BKB: bytes of a K chunk per row (32, 64 or 128); F8: E4M3 operands.
// PAIR: the kernel runs as clusters of 2 CTAs on 2 SMs; a pair computes a
// 256 x BN tile with one tcgen05.mma (M = 256, cta_group::2) issued by the
// leader (rank 0): each CTA loads its 128 rows of A and its BN/2 rows of B'
// and holds its 128 rows of the accumulator in its own TMEM, so each SM
// streams half the B' bytes of a 1-CTA tile through shared memory.
template <int BN, int BKB, int STAGES, bool F8, bool PAIR>
__global__ void __launch_bounds__(kTcThreads, 1) gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB,
                                                         const TcArgs args) {
    using S = TcSmem<PAIR ? BN / 2 : BN, BKB, STAGES>;
    constexpr int BK = F8 ? BKB : BKB / 2;             // K chunk in operand elements
    constexpr int TM = PAIR ? 256 : 128;               // rows of a tile
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + S::ring);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    uint64_t *acce = accf + 2;
    uint64_t *drain = acce + 2;
    volatile uint32_t *tmem_slot = (volatile uint32_t *)(drain + 1);
    __shared__ int abort_flag;
    __shared__ int peer_abort;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr uint32_t tmem_cols = (2 * BN < 32) ? 32 : 2 * BN;
    const uint32_t rank = PAIR ? cluster_rank() : 0;
    const bool leader = rank == 0;
    // tile walker: the CTA, or the CTA pair
    const int64_t walker = PAIR ? blockIdx.x >> 1 : blockIdx.x;
    const int64_t walkers = PAIR ? gridDim.x >> 1 : gridDim.x;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        peer_abort = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], PAIR ? 2 * kEpiThreads : kEpiThreads);   // pair: both CTAs' epilogues
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
    }
    if (warp == 1) {
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32((const void *)tmem_slot)),
                         "r"(tmem_cols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32((const void *)tmem_slot)),
                         "r"(tmem_cols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();     // the peer's barriers exist before any arrive on them
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer --
        if (lane == 0 && !args.withhold) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            int8_t armed[STAGES];   // phase parity of the last load issued per stage
            for (int s = 0; s < STAGES; ++s) armed[s] = -1;
            const uint32_t full_leader = PAIR ? mapa_rank(&full[0], 0) : 0;
            for (int64_t t = walker; t < args.tiles && ok; t += walkers) {
                int64_t b, mt;
                int nt;
                tile_coords(args, t, b, mt, nt);
                const int kbase = (int)(t / args.tiles_per_part) * args.nk * BK;
                for (int kc = 0; kc < args.nk; ++kc) {
                    if (!mbar_wait<PAIR>(&empty[stage], phase ^ 1, &abort_flag)) { ok = false; break; }
                    uint8_t *sa = smem + stage * S::stage_bytes;
                    uint8_t *sb = sa + S::a_bytes;
                    const int zA = args.za ? args.za[b] : (args.batch_a ? (int)b : 0);
                    if constexpr (PAIR) {
                        // the leader's barrier counts both CTAs' bytes
                        if (leader) mbar_expect_tx(&full[stage], 2 * (S::a_bytes + S::b_bytes));
                        const int zB = args.batch_b ? (int)b : 0;
                        const uint32_t fb = full_leader + (uint32_t)(stage * 8);
                        tma_load_3d_pair(sa, &tmA, fb, kbase + kc * BK, (int)(mt * 256 + rank * 128), zA);
                        tma_load_3d_pair(sb, &tmB, fb, kbase + kc * BK, nt * BN + (int)rank * (BN / 2), zB);
                        armed[stage] = (int8_t)phase;
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                        continue;
                    }
                    mbar_expect_tx(&full[stage], S::a_bytes + S::b_bytes);
                    tma_load_3d(sa, &tmA, &full[stage], kbase + kc * BK, (int)(mt * 128), zA);
                    if (args.gather_r) {
                        // B_P: one whole B' chunk (np_chunk rows) per r of this tile
                        for (int rr = 0; rr < args.gather_r; ++rr) {
                            const int r = nt * args.gather_r + rr;
                            const int zB = r < args.m_r ? max(0, args.zb[b * args.m_r + r]) : 0;
                            tma_load_3d(sb + rr * args.np_chunk * BKB, &tmB, &full[stage], kbase + kc * BK,
                                        0, zB);
                        }
                    } else {
                        const int zB = args.zb ? max(0, args.zb[b]) : (args.batch_b ? (int)b : 0);
                        tma_load_3d(sb, &tmB, &full[stage], kbase + kc * BK, nt * BN, zB);
                    }
                    armed[stage] = (int8_t)phase;
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
            }
            if (!ok && (!PAIR || leader)) {
                // drain: only the last STAGES loads can still be in flight;
                // wait (bounded) until each has landed before shared memory goes
                // (a pair's peer sees its loads land on the leader's barriers
                // only: it waits out the teardown delay instead)
                for (int s = 0; s < STAGES; ++s) {
                    if (armed[s] < 0) continue;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try_wait(&full[s], (uint32_t)armed[s]) &&
                           globaltimer() - t0 < kWaitLimitNs / 4) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // --------------------------------------------------- MMA issue --
        if (lane == 0 && (!PAIR || leader)) {
            uint32_t idesc = 0;
            idesc |= 1u << 4;                                  // D = F32
            // kind::f16: 0 F16, 1 BF16; kind::f8f6f4: 0 E4M3
            const uint32_t fmt = (!F8 && args.dtype == TN_BF16) ? 1u : 0u;
            idesc |= fmt << 7;                                 // A format
            idesc |= fmt << 10;                                // B format
            idesc |= (uint32_t)(BN >> 3) << 17;                // N
            idesc |= (uint32_t)(TM >> 4) << 24;                // M
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            bool issued = false;
            for (int64_t t = walker; t < args.tiles && ok; t += walkers) {
                if (!mbar_wait<PAIR>(&acce[acc], acc_phase ^ 1, &abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
                for (int kc = 0; kc < args.nk; ++kc) {
                    if (!mbar_wait<PAIR>(&full[stage], phase, &abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(smem + stage * S::stage_bytes);
                    const uint32_t b_addr = a_addr + S::a_bytes;
#pragma unroll
                    for (int kk = 0; kk < BKB / 32; ++kk) {     // 32 bytes of K per MMA
                        const uint64_t ad = smem_desc<BKB>(a_addr + kk * 32);
                        const uint64_t bd = smem_desc<BKB>(b_addr + kk * 32);
                        tc_mma<F8, PAIR>(d_tmem, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                    }
                    issued = true;
                    tc_commit<PAIR>(&empty[stage]);
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                tc_commit<PAIR>(&accf[acc]);
                if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            }
            if (!ok && issued) {
                // aborted: MMAs issued may still run; let them finish
                // (bounded) before TMEM and shared memory are released
                if constexpr (PAIR) tc_commit_pair_local(drain);
                else tc_commit(drain);
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kWaitLimitNs / 4) {
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- epilogue --
        const int q = warp & 3;                 // TMEM lane quadrant of this warp
        const int half = (warp - 2) >> 2;       // which alternate 16-column chunks
        const int row = q * 32 + lane;
        int e;
        if (args.out_c64 || args.sr.scale_off)
            e = 0;
        else if (args.sr.tmax)
            e = min(120, scale_exp_tc(args.sr.tmax[args.sr.meta_a], args.sr.tmax[args.sr.meta_b], args.lk) +
                             args.sr.headroom);
        else
            e = args.sr.fixed_exp;
        if (args.sr.texp && !args.partial && blockIdx.x == 0 && threadIdx.x == 64)
            args.sr.texp[args.sr.meta_c] = args.sr.texp[args.sr.meta_a] + args.sr.texp[args.sr.meta_b] + e;
        const float sc = __int_as_float((127 + e) << 23);
        // fused permutation: where the 8 values of one chunk go (low 3 bits)
        int64_t lowtab[8];
        bool low_kept = true;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            lowtab[j] = args.out_rank ? permute_bits(args, j, 0, 3) : j;
            low_kept = low_kept && lowtab[j] == j;
        }
        const bool staged = args.staged && tc_staged_ok(args, low_kept);
        uint8_t *stg = smem + S::stg + (warp - 2) * 4096;
        // staged stores: blocks of WB real columns, alternating between the
        // quadrant's two warps
        constexpr int WB = BN >= 128 ? 64 : (BN >= 32 ? BN / 2 : 16);
        float mx = 0.f;
        int acc = 0;
        uint32_t acc_phase = 0;
        const uint32_t acce_leader = PAIR ? mapa_rank(&acce[0], 0) : 0;
        for (int64_t t = walker; t < args.tiles; t += walkers) {
            int64_t b, mt;
            int nt;
            tile_coords(args, t, b, mt, nt);
            if (!mbar_wait<PAIR>(&accf[acc], acc_phase, &abort_flag)) break;
            tc_fence_after();
            const int64_t m = mt * TM + rank * 128 + row;
            const int col0 = nt * BN;                          // real column of this tile
            const int64_t cb = args.zc ? (int64_t)args.zc[b] : b;   // output chunk (< 0: skip)
            // fused permutation: destination = row part | column part | low 3 bits
            int64_t prow = 0;
            if (args.out_rank) prow = permute_bits(args, (cb * args.M + m) * (int64_t)args.N, args.ln, args.out_rank);
            // gather_r: the tile's columns are gather_r chunks of np_chunk real
            // columns, chunk r of row b going to output chunk zc[b m_r + r]
            const int col_end = args.gather_r ? BN : min(BN, 2 * args.N - col0);   // warp-uniform
            if (staged) {
                if (cb >= 0)
                    for (int c = WB * half; c < col_end; c += 2 * WB)
                        tc_store_block(args, tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN), c,
                                       min(WB, col_end - c), m, lane, col0, cb, prow, sc, mx, stg);
            } else {
                for (int c = 16 * half; c < col_end; c += 32) {
                    uint32_t r[16];
                    tmem_ld16<16>(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c), r);
                    tmem_wait_ld();
                    tc_store16(args, r, b, m, t, col0, c, col_end, cb, prow, lowtab, low_kept, sc, mx);
                }
            }
            tc_fence_before();
            if constexpr (PAIR) mbar_arrive_cluster(acce_leader + (uint32_t)(acc * 8));
            else mbar_arrive(&acce[acc]);
            if (++acc == 2) { acc = 0; acc_phase ^= 1; }
        }
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        if (lane == 0 && args.sr.out_max && !args.partial)
            atomicMax(reinterpret_cast<int *>(args.sr.out_max), __float_as_int(mx));
        if (lane == 0 && args.sr.err && args.dtype == TN_F16 && !args.out_c64 && !args.partial &&
            !(mx <= 65504.0f))
            atomicOr(args.sr.err, 2);
    }

    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) {
        // Neither CTA leaves while the other may still use its shared memory
        // or TMEM.  After an abort, loads the peer issued may still be landing
        // here (their completion counts on the leader's barriers only): wait
        // a bounded 2 ms before either CTA releases anything.
        if (threadIdx.x == 0 && abort_flag)
            asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(mapa_rank(&peer_abort, rank ^ 1)), "r"(1)
                         : "memory");
        cluster_sync();
        if (abort_flag || peer_abort) {
            const uint64_t t0 = globaltimer();
            while (globaltimer() - t0 < 2000000ull) {
            }
        }
        cluster_sync();
    }
    if (abort_flag && threadIdx.x == 0 && args.err) atomicOr(args.err, 1);
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"(tmem_cols)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"(tmem_cols)
                         : "memory");
    }
}

// ------------------------------------------------ B'-resident variant --
// Short-K steps (the whole K of a B' tile fits in shared memory) are bound
// by L2 rather than by the tensor pipe: the kernel above reloads each tile's
// B' slice (BN rows x 2K) with every tile, while only the A tile and the C
// tile are new.  Here each walker keeps its B' slice resident in one of two
// shared-memory slots and reloads it only when the tile's (n tile, B batch
// entry) changes; the ring carries A alone (more stages).  Tiles are walked
// n-fastest (t -> b, m tile, n tile) and the grid is a multiple of the number
// of n tiles, so a walker's n tile never changes and consecutive walkers
// share the same A tile in L2.  Same MMA, same epilogue (same bits).
// Barriers: bfull[s] -- the B' slice in slot s landed (TMA bytes);
// bfree[s] -- the MMAs that read slot s finished (tcgen05.commit when the
// MMA warp moves to the other slot).  1-CTA, FP16/BF16, no gathers, one K
// part.
struct BresCfg {
    int bn;                 // N tile (real columns), 16..256
    int stages;             // A stages in the ring
    uint32_t chunk_bytes;   // one K chunk of the slice (bn x BKB), rounded up to 1 KiB
    uint32_t slot_bytes;    // nk chunks, <= 64 KiB
    int tma_store;          // 1: C tiles staged in shared memory and written by TMA stores
    uint32_t stage_c_bytes; // one staged C tile: bn / 64 panels of 128 rows x 128 bytes
};

// AND of a predicate over the 256 epilogue threads (named barrier 2): the
// epilogue's decisions to stop must agree before any of them waits on a
// named barrier the others would never reach
__device__ __forceinline__ bool epi_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 2, 256, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// TMA store of one staged 128-row panel of C (bulk group of this thread)
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(map),
                 "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}

__device__ __forceinline__ void bres_coords(const TcArgs &a, int64_t t, int64_t &b, int64_t &mt, int &nt) {
    nt = (int)(t % a.n_nt);
    const int64_t r = t / a.n_nt;
    mt = r % a.n_mt;
    b = r / a.n_mt;
}

constexpr int kBresMaxStages = 12;

template <int BKB>
__global__ void __launch_bounds__(kTcThreads, 1) gemm_tc_bres_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB,
                                                              const __grid_constant__ CUtensorMap tmC,
                                                              const TcArgs args, const BresCfg cfg) {
    constexpr int BK = BKB / 2;
    constexpr uint32_t a_bytes = 128 * BKB;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int bn = cfg.bn, stages = cfg.stages;
    uint8_t *bslot0 = smem + (size_t)stages * a_bytes;           // B' slots after the A ring
    uint8_t *cstage = bslot0 + 2 * (size_t)cfg.slot_bytes;       // staged C tiles (two)
    uint64_t *full = (uint64_t *)(cstage + (cfg.tma_store ? 2 * (size_t)cfg.stage_c_bytes : 0));
    uint64_t *empty = full + kBresMaxStages;
    uint64_t *accf = empty + kBresMaxStages;
    uint64_t *acce = accf + 2;
    uint64_t *bfull = acce + 2;
    uint64_t *bfree = bfull + 2;
    uint64_t *drain = bfree + 2;
    volatile uint32_t *tmem_slot = (volatile uint32_t *)(drain + 1);
    __shared__ int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = 2 * bn < 32 ? 32 : 2 * bn;
    const int64_t walker = blockIdx.x, walkers = gridDim.x;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], kEpiThreads);
            mbar_init(&bfull[i], 1);
            mbar_init(&bfree[i], 1);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer --
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            int8_t armed[kBresMaxStages];
            for (int s = 0; s < kBresMaxStages; ++s) armed[s] = -1;
            int8_t barmed[2] = {-1, -1};
            uint32_t bfree_bits = 0;       // parity of the next load into slot s
            int slot = 1;
            int64_t cur_key = -1;
            for (int64_t t = walker; t < args.tiles && ok; t += walkers) {
                int64_t b, mt;
                int nt;
                bres_coords(args, t, b, mt, nt);
                const int zA = args.batch_a ? (int)b : 0;
                const int zB = args.batch_b ? (int)b : 0;
                const int64_t key = (int64_t)zB * args.n_nt + nt;
                if (key != cur_key) {
                    // the whole K of this tile's B' slice into the next slot,
                    // once the MMAs that read that slot before have finished
                    slot ^= 1;
                    const uint32_t par = (bfree_bits >> slot) & 1u;
                    if (!mbar_wait(&bfree[slot], par ^ 1u, &abort_flag)) { ok = false; break; }
                    bfree_bits ^= 1u << slot;
                    uint8_t *sb = bslot0 + (size_t)slot * cfg.slot_bytes;
                    mbar_expect_tx(&bfull[slot], (uint32_t)args.nk * (uint32_t)bn * BKB);
                    for (int kc = 0; kc < args.nk; ++kc)
                        tma_load_3d(sb + (size_t)kc * cfg.chunk_bytes, &tmB, &bfull[slot], kc * BK, nt * bn, zB);
                    barmed[slot] = (int8_t)par;
                    cur_key = key;
                }
                for (int kc = 0; kc < args.nk; ++kc) {
                    if (!mbar_wait(&empty[stage], phase ^ 1, &abort_flag)) { ok = false; break; }
                    uint8_t *sa = smem + (size_t)stage * a_bytes;
                    mbar_expect_tx(&full[stage], a_bytes);
                    tma_load_3d(sa, &tmA, &full[stage], kc * BK, (int)(mt * 128), zA);
                    armed[stage] = (int8_t)phase;
                    if (++stage == stages) { stage = 0; phase ^= 1; }
                }
            }
            if (!ok) {
                // drain (bounded): loads still in flight land before shared memory goes
                for (int s = 0; s < stages; ++s) {
                    if (armed[s] < 0) continue;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try_wait(&full[s], (uint32_t)armed[s]) && globaltimer() - t0 < kWaitLimitNs / 4) {
                    }
                }
                for (int s = 0; s < 2; ++s) {
                    if (barmed[s] < 0) continue;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try_wait(&bfull[s], (uint32_t)barmed[s]) && globaltimer() - t0 < kWaitLimitNs / 4) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // --------------------------------------------------- MMA issue --
        if (lane == 0) {
            uint32_t idesc = 0;
            idesc |= 1u << 4;                                  // D = F32
            const uint32_t fmt = args.dtype == TN_BF16 ? 1u : 0u;
            idesc |= fmt << 7;                                 // A format
            idesc |= fmt << 10;                                // B format
            idesc |= (uint32_t)(bn >> 3) << 17;                // N
            idesc |= (uint32_t)(128 >> 4) << 24;               // M
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            uint32_t bfull_bits = 0;       // parity of the next use of slot s
            int slot = 1;
            int64_t cur_key = -1;
            bool ok = true;
            bool issued = false;
            for (int64_t t = walker; t < args.tiles && ok; t += walkers) {
                int64_t b, mt;
                int nt;
                bres_coords(args, t, b, mt, nt);
                const int zB = args.batch_b ? (int)b : 0;
                const int64_t key = (int64_t)zB * args.n_nt + nt;
                if (key != cur_key) {
                    // the MMAs issued so far read the old slot: release it
                    // when they finish, then wait for the new slice
                    if (cur_key >= 0) tc_commit(&bfree[slot]);
                    slot ^= 1;
                    if (!mbar_wait(&bfull[slot], (bfull_bits >> slot) & 1u, &abort_flag)) { ok = false; break; }
                    bfull_bits ^= 1u << slot;
                    tc_fence_after();
                    cur_key = key;
                }
                if (!mbar_wait(&acce[acc], acc_phase ^ 1, &abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * bn);
                const uint32_t b_base = smem_u32(bslot0 + (size_t)slot * cfg.slot_bytes);
                for (int kc = 0; kc < args.nk; ++kc) {
                    if (!mbar_wait(&full[stage], phase, &abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(smem + (size_t)stage * a_bytes);
                    const uint32_t b_addr = b_base + (uint32_t)kc * cfg.chunk_bytes;
#pragma unroll
                    for (int kk = 0; kk < BKB / 32; ++kk) {     // 32 bytes of K per MMA
                        const uint64_t ad = smem_desc<BKB>(a_addr + kk * 32);
                        const uint64_t bd = smem_desc<BKB>(b_addr + kk * 32);
                        tc_mma<false, false>(d_tmem, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                    }
                    issued = true;
                    tc_commit(&empty[stage]);
                    if (++stage == stages) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                tc_commit(&accf[acc]);
                if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            }
            if (!ok && issued) {
                tc_commit(drain);
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kWaitLimitNs / 4) {
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- epilogue --
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        int e;
        if (args.out_c64 || args.sr.scale_off) e = 0;
        else if (args.sr.tmax)
            e = min(120, scale_exp_tc(args.sr.tmax[args.sr.meta_a], args.sr.tmax[args.sr.meta_b], args.lk) +
                             args.sr.headroom);
        else e = args.sr.fixed_exp;
        if (args.sr.texp && blockIdx.x == 0 && threadIdx.x == 64)
            args.sr.texp[args.sr.meta_c] = args.sr.texp[args.sr.meta_a] + args.sr.texp[args.sr.meta_b] + e;
        const float sc = __int_as_float((127 + e) << 23);
        int64_t lowtab[8];
        bool low_kept = true;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            lowtab[j] = args.out_rank ? permute_bits(args, j, 0, 3) : j;
            low_kept = low_kept && lowtab[j] == j;
        }
        float mx = 0.f;
        int acc = 0;
        uint32_t acc_phase = 0;
        int64_t ntile = 0;
        for (int64_t t = walker; t < args.tiles; t += walkers) {
            int64_t b, mt;
            int nt;
            bres_coords(args, t, b, mt, nt);
            const bool got = mbar_wait(&accf[acc], acc_phase, &abort_flag);
            if (cfg.tma_store ? !epi_all(got) : !got) break;
            tc_fence_after();
            const int64_t m = mt * 128 + row;
            const int col0 = nt * bn;
            const int64_t cb = b;
            int64_t prow = 0;
            if (args.out_rank) prow = permute_bits(args, (cb * args.M + m) * (int64_t)args.N, args.ln, args.out_rank);
            const int col_end = min(bn, 2 * args.N - col0);
            if (cfg.tma_store) {
                // the tile's rounded values go to a staged C tile in shared
                // memory (128-byte swizzle: 16-byte unit u of row r at unit
                // u ^ (r & 7) of its 128-byte line), then one thread writes
                // the bn / 64 panels with TMA stores -- full lines, no
                // row-per-thread global stores.  Two staged tiles alternate;
                // before one is rewritten its stores must have read it.
                uint8_t *stg = cstage + (size_t)(ntile & 1) * cfg.stage_c_bytes;
                if (threadIdx.x == 64 && ntile >= 2)
                    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
                for (int c = 16 * half; c < col_end; c += 32) {
                    uint32_t r[16];
                    tmem_ld16<16>(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * bn + c), r);
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
                    const int p = c >> 6, u = (c & 63) >> 3;
                    uint8_t *line = stg + (size_t)p * 16384 + (size_t)row * 128;
                    *reinterpret_cast<uint4 *>(line + (((u) ^ (row & 7)) << 4)) =
                        make_uint4(packed[0], packed[1], packed[2], packed[3]);
                    *reinterpret_cast<uint4 *>(line + (((u + 1) ^ (row & 7)) << 4)) =
                        make_uint4(packed[4], packed[5], packed[6], packed[7]);
                }
                tc_fence_before();
                mbar_arrive(&acce[acc]);          // TMEM is read: the MMA may reuse it
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
                if (threadIdx.x == 64) {
                    for (int p = 0; p < bn / 64; ++p)
                        tma_store_3d(&tmC, stg + (size_t)p * 16384, col0 + 64 * p, (int)(mt * 128), (int)cb);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
                ++ntile;
                if (++acc == 2) { acc = 0; acc_phase ^= 1; }
                continue;
            }
            for (int c = 16 * half; c < col_end; c += 32) {
                uint32_t r[16];
                tmem_ld16<16>(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * bn + c), r);
                tmem_wait_ld();
                tc_store16(args, r, b, m, t, col0, c, col_end, cb, prow, lowtab, low_kept, sc, mx);
            }
            tc_fence_before();
            mbar_arrive(&acce[acc]);
            if (++acc == 2) { acc = 0; acc_phase ^= 1; }
        }
        // every TMA store written out before the kernel ends
        if (cfg.tma_store && threadIdx.x == 64) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && args.sr.out_max)
            atomicMax(reinterpret_cast<int *>(args.sr.out_max), __float_as_int(mx));
        if (lane == 0 && args.sr.err && args.dtype == TN_F16 && !args.out_c64 && !(mx <= 65504.0f))
            atomicOr(args.sr.err, 2);
    }

    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0 && args.err) atomicOr(args.err, 1);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols)
                     : "memory");
    }
}

// ------------------------------------------- complex64 on TF32 (x3) --
// Complex64 steps on the tensor cores: the real GEMM of Eq. 6 with FP32
// operands, each split as x ~ hi + lo, both exactly TF32 values (hi = x
// rounded to 11 significant bits, lo = the rounded remainder); then
// A B'^T ~ A_hi B'_hi + A_hi B'_lo + A_lo B'_hi (A_lo B'_lo is about 2^-22
// of the product), three kind::tf32 MMAs per 8-element K slice, each part of
// kX3Part K chunks in a fresh TMEM accumulator whose values the epilogue adds
// in FP32 registers.  The four operands come from hi / lo arrays built beforehand
// (split_tf32, bprep_x3).  Same roles as gemm_tc_kernel (1-CTA, 320
// threads, bounded waits, double-buffered accumulators); the result is
// complex64 (the epilogue's FP32 path: no rounding, no scale).
// K chunks per accumulation part of the x3 kernel (the epilogue adds the
// parts in FP32 registers): 2 chunks of 128 bytes = 64 real K terms.  The
// tensor cores' own FP32 accumulation loses bits with every MMA it adds up:
// measured against FP64 per GEMM, one accumulator over all of K: 8e-6;
// 256-term parts: 1.9e-6; 64-term parts: 5.3e-7 (253 TFLOP/s); 32-term
// parts: 3.2e-7 (222 TFLOP/s); the CUDA cores: 0.4-1.6e-6
constexpr int kX3Part = 2;

template <int BN, int BKB>
struct X3Smem {
    static constexpr int a_bytes = 128 * BKB;
    static constexpr int b_bytes = BN * BKB;
    // a stage: A_hi | B'_hi | A_lo | B'_lo (each a whole number of KiB)
    static constexpr int stage_bytes = (2 * (a_bytes + b_bytes) + 1023) / 1024 * 1024;
    static constexpr int stages0 = (192 * 1024) / stage_bytes;
    static constexpr int STAGES = stages0 > 8 ? 8 : (stages0 < 2 ? 2 : stages0);
    static constexpr int ring = STAGES * stage_bytes;
    static constexpr int total = 1024 + ring + 1024;
    static_assert(total <= 232448, "over the 227 KiB of shared memory a CTA may have");
    static_assert((2 * STAGES + 5) * 8 + 16 <= 1024, "barriers overflow their kilobyte");
};

template <int BN, int BKB>
__global__ void __launch_bounds__(kTcThreads, 1) gemm_tc_x3_kernel(const __grid_constant__ CUtensorMap tmAh,
                                                            const __grid_constant__ CUtensorMap tmAl,
                                                            const __grid_constant__ CUtensorMap tmBh,
                                                            const __grid_constant__ CUtensorMap tmBl,
                                                            const TcArgs args) {
    using S = X3Smem<BN, BKB>;
    constexpr int STAGES = S::STAGES;
    constexpr int BK = BKB / 4;                        // FP32 elements per K chunk
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + S::ring);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    uint64_t *acce = accf + 2;
    uint64_t *drain = acce + 2;
    volatile uint32_t *tmem_slot = (volatile uint32_t *)(drain + 1);
    __shared__ int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr uint32_t tmem_cols = (2 * BN < 32) ? 32 : 2 * BN;
    const int64_t walker = blockIdx.x, walkers = gridDim.x;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], kEpiThreads);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmAh) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmAl) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmBh) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmBl) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer --
        if (lane == 0 && !args.withhold) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            int8_t armed[STAGES];
            for (int st = 0; st < STAGES; ++st) armed[st] = -1;
            for (int64_t t = walker; t < args.tiles && ok; t += walkers) {
                int64_t b, mt;
                int nt;
                tile_coords(args, t, b, mt, nt);
                const int kbase = (int)(t / args.tiles_per_part) * args.nk * BK;
                const int zA = args.batch_a ? (int)b : 0, zB = args.batch_b ? (int)b : 0;
                for (int kc = 0; kc < args.nk; ++kc) {
                    if (!mbar_wait(&empty[stage], phase ^ 1, &abort_flag)) { ok = false; break; }
                    uint8_t *sa = smem + stage * S::stage_bytes;
                    uint8_t *sb = sa + S::a_bytes;
                    uint8_t *sa2 = sb + S::b_bytes;
                    uint8_t *sb2 = sa2 + S::a_bytes;
                    mbar_expect_tx(&full[stage], 2 * (S::a_bytes + S::b_bytes));
                    const int x = kbase + kc * BK;
                    tma_load_3d(sa, &tmAh, &full[stage], x, (int)(mt * 128), zA);
                    tma_load_3d(sb, &tmBh, &full[stage], x, nt * BN, zB);
                    tma_load_3d(sa2, &tmAl, &full[stage], x, (int)(mt * 128), zA);
                    tma_load_3d(sb2, &tmBl, &full[stage], x, nt * BN, zB);
                    armed[stage] = (int8_t)phase;
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
            }
            if (!ok) {
                // drain: only the last STAGES loads can still be in flight
                for (int st = 0; st < STAGES; ++st) {
                    if (armed[st] < 0) continue;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try_wait(&full[st], (uint32_t)armed[st]) && globaltimer() - t0 < kWaitLimitNs / 4) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // --------------------------------------------------- MMA issue --
        // each tile's K range in parts of kX3Part chunks, each part into a
        // fresh TMEM accumulator (the epilogue sums the parts in registers)
        if (lane == 0) {
            uint32_t idesc = 0;
            idesc |= 1u << 4;                                  // D = F32
            idesc |= 2u << 7;                                  // A = TF32
            idesc |= 2u << 10;                                 // B = TF32
            idesc |= (uint32_t)(BN >> 3) << 17;                // N
            idesc |= (uint32_t)(128 >> 4) << 24;               // M
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            bool issued = false;
            for (int64_t t = walker; t < args.tiles && ok; t += walkers) {
                for (int k0 = 0; k0 < args.nk && ok; k0 += kX3Part) {
                    const int k1 = min(args.nk, k0 + kX3Part);
                    if (!mbar_wait(&acce[acc], acc_phase ^ 1, &abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
                    for (int kc = k0; kc < k1; ++kc) {
                        if (!mbar_wait(&full[stage], phase, &abort_flag)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t a_addr = smem_u32(smem + stage * S::stage_bytes);
                        const uint32_t b_addr = a_addr + S::a_bytes;
                        const uint32_t a2_addr = b_addr + S::b_bytes;
                        const uint32_t b2_addr = a2_addr + S::a_bytes;
#pragma unroll
                        for (int kk = 0; kk < BKB / 32; ++kk) {     // 8 FP32 of K per MMA
                            const uint64_t ah = smem_desc<BKB>(a_addr + kk * 32);
                            const uint64_t bh = smem_desc<BKB>(b_addr + kk * 32);
                            const uint64_t al = smem_desc<BKB>(a2_addr + kk * 32);
                            const uint64_t bl = smem_desc<BKB>(b2_addr + kk * 32);
                            tc_mma_tf32(d_tmem, ah, bh, idesc, (kc > k0 || kk > 0) ? 1u : 0u);
                            tc_mma_tf32(d_tmem, ah, bl, idesc, 1u);
                            tc_mma_tf32(d_tmem, al, bh, idesc, 1u);
                        }
                        issued = true;
                        tc_commit(&empty[stage]);
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                    }
                    if (!ok) break;
                    tc_commit(&accf[acc]);
                    if (++acc == 2) { acc = 0; acc_phase ^= 1; }
                }
            }
            if (!ok && issued) {
                tc_commit(drain);
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kWaitLimitNs / 4) {
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- epilogue --
        // per tile: the K parts' accumulators added in FP32 registers (IEEE
        // adds; the tensor cores' own accumulation drifts over long K), then
        // stored as complex64 (or as a split-K partial)
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        constexpr int NCH = (BN + 31) / 32;                // this warp's 16-column chunks
        int64_t lowtab[8];
        bool low_kept = true;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            lowtab[j] = args.out_rank ? permute_bits(args, j, 0, 3) : j;
            low_kept = low_kept && lowtab[j] == j;
        }
        float mx = 0.f;
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int64_t t = walker; t < args.tiles && ok; t += walkers) {
            int64_t b, mt;
            int nt;
            tile_coords(args, t, b, mt, nt);
            const int col0 = nt * BN;
            const int col_end = min(BN, 2 * args.N - col0);
            float sum[NCH][16];
#pragma unroll
            for (int i = 0; i < NCH; ++i)
#pragma unroll
                for (int j = 0; j < 16; ++j) sum[i][j] = 0.f;
            for (int k0 = 0; k0 < args.nk; k0 += kX3Part) {
                if (!mbar_wait(&accf[acc], acc_phase, &abort_flag)) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int i = 0; i < NCH; ++i) {
                    const int c = 16 * half + 32 * i;
                    if (c < col_end) {
                        uint32_t r[16];
                        tmem_ld16<16>(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c), r);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; ++j) sum[i][j] += __uint_as_float(r[j]);
                    }
                }
                tc_fence_before();
                mbar_arrive(&acce[acc]);
                if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            }
            if (!ok) break;
            const int64_t m = mt * 128 + row;
            const int64_t cb = b;
            int64_t prow = 0;
            if (args.out_rank) prow = permute_bits(args, (cb * args.M + m) * (int64_t)args.N, args.ln, args.out_rank);
#pragma unroll
            for (int i = 0; i < NCH; ++i) {
                const int c = 16 * half + 32 * i;
                if (c < col_end) {
                    uint32_t r[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(sum[i][j]);
                    tc_store16(args, r, b, m, t, col0, c, col_end, cb, prow, lowtab, low_kept, 1.0f, mx);
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && args.sr.out_max && !args.partial)
            atomicMax(reinterpret_cast<int *>(args.sr.out_max), __float_as_int(mx));
    }

    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0 && args.err) atomicOr(args.err, 1);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols)
                     : "memory");
    }
}

// shared memory of the B'-resident kernel: A ring + two B' slots + barriers
constexpr int kBresSmemBudget = 196 * 1024;
constexpr int kBresSmemTotal = 1024 + kBresSmemBudget + (2 * kBresMaxStages + 9) * 8 + 16;

// ------------------------------------------------------------ host side --
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    });
    return fn;
}

// esz 2: FP16/BF16 elements (dtype), esz 1: E4M3 bytes
bool encode_3d(CUtensorMap *m, int dtype, int esz, const void *base, uint64_t inner, uint64_t rows,
               uint64_t depth, uint32_t box_inner, uint32_t box_rows) {
    EncodeFn enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[3] = {inner, rows, depth};
    const cuuint64_t strides[2] = {inner * esz, inner * rows * esz};
    const cuuint32_t box[3] = {box_inner, box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const uint32_t row_bytes = box_inner * esz;
    const CUtensorMapSwizzle sw = row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                    : CU_TENSOR_MAP_SWIZZLE_32B;
    const CUtensorMapDataType dt = esz == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dtype == TN_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    return enc(m, dt, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int BKB, bool PAIR = false>
struct TcCfg {
    static constexpr int brows = PAIR ? BN / 2 : BN;
    static constexpr int stage_bytes = (128 * BKB + brows * BKB + 1023) / 1024 * 1024;
    static constexpr int stages0 = (192 * 1024) / stage_bytes;
    static constexpr int STAGES = stages0 > 12 ? 12 : (stages0 < 2 ? 2 : stages0);
};

template <int BN, int BKB, bool F8, bool PAIR = false>
cudaError_t set_attr() {
    constexpr int ST = TcCfg<BN, BKB, PAIR>::STAGES;
    using S = TcSmem<TcCfg<BN, BKB, PAIR>::brows, BKB, ST>;
    return cudaFuncSetAttribute(gemm_tc_kernel<BN, BKB, ST, F8, PAIR>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, S::total);
}

// CTA-pair kernel (BN = 256, 128-byte K chunks): launch configuration with a
// cluster of 2, and how many pairs the GPU holds at once
template <bool F8>
cudaLaunchConfig_t pair_config(int64_t grid, cudaStream_t s, cudaLaunchAttribute *attr) {
    constexpr int ST = TcCfg<256, 128, true>::STAGES;
    using S = TcSmem<128, 128, ST>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(kTcThreads, 1, 1);
    cfg.dynamicSmemBytes = S::total;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

int g_pair_clusters[2] = {0, 0};   // [F8]: resident CTA pairs (0: not known yet)

template <bool F8>
cudaError_t prepare_pair() {
    constexpr int ST = TcCfg<256, 128, true>::STAGES;
    cudaError_t e = set_attr<256, 128, F8, true>();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config<F8>(2 * 76, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, gemm_tc_kernel<256, 128, ST, F8, true>, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = tc_num_sms() / 2;
    }
    g_pair_clusters[F8 ? 1 : 0] = n;
    return cudaSuccess;
}

template <int BKB, bool F8>
cudaError_t set_attr_bn() {
    cudaError_t e = set_attr<16, BKB, F8>();
    if (e == cudaSuccess) e = set_attr<32, BKB, F8>();
    if (e == cudaSuccess) e = set_attr<64, BKB, F8>();
    if (e == cudaSuccess) e = set_attr<128, BKB, F8>();
    if (e == cudaSuccess) e = set_attr<256, BKB, F8>();
    return e;
}

template <int BN, int BKB, bool F8>
cudaError_t run_tc(const CUtensorMap &ma, const CUtensorMap &mb, const TcArgs &a, cudaStream_t s) {
    constexpr int ST = TcCfg<BN, BKB>::STAGES;
    using S = TcSmem<BN, BKB, ST>;
    auto kern = gemm_tc_kernel<BN, BKB, ST, F8, false>;
    const int64_t grid = std::min<int64_t>(a.tiles, tc_num_sms());
    kern<<<(unsigned)grid, kTcThreads, S::total, s>>>(ma, mb, a);
    return cudaGetLastError();
}

template <bool F8>
cudaError_t run_tc_pair(const CUtensorMap &ma, const CUtensorMap &mb, const TcArgs &a, cudaStream_t s) {
    constexpr int ST = TcCfg<256, 128, true>::STAGES;
    const int pairs = g_pair_clusters[F8 ? 1 : 0] > 0 ? g_pair_clusters[F8 ? 1 : 0] : tc_num_sms() / 2;
    const int64_t grid = 2 * std::min<int64_t>(a.tiles, pairs);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config<F8>(grid, s, attr);
    return cudaLaunchKernelEx(&cfg, gemm_tc_kernel<256, 128, ST, F8, true>, ma, mb, a);
}

template <int BKB, bool F8>
cudaError_t run_tc_bn(int bn, const CUtensorMap &ma, const CUtensorMap &mb, const TcArgs &a,
                      cudaStream_t s) {
    switch (bn) {
        case 16: return run_tc<16, BKB, F8>(ma, mb, a, s);
        case 32: return run_tc<32, BKB, F8>(ma, mb, a, s);
        case 64: return run_tc<64, BKB, F8>(ma, mb, a, s);
        case 128: return run_tc<128, BKB, F8>(ma, mb, a, s);
        case 256: return run_tc<256, BKB, F8>(ma, mb, a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int BN, int BKB>
cudaError_t set_attr_x3() {
    return cudaFuncSetAttribute(gemm_tc_x3_kernel<BN, BKB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                X3Smem<BN, BKB>::total);
}

template <int BKB>
cudaError_t set_attr_x3_bn() {
    cudaError_t e = set_attr_x3<16, BKB>();
    if (e == cudaSuccess) e = set_attr_x3<32, BKB>();
    if (e == cudaSuccess) e = set_attr_x3<64, BKB>();
    if (e == cudaSuccess) e = set_attr_x3<128, BKB>();
    return e;
}

template <int BKB>
cudaError_t run_tc_x3(int bn, const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh,
                      const CUtensorMap &bl, const TcArgs &a, cudaStream_t s) {
    const int64_t grid = std::min<int64_t>(a.tiles, tc_num_sms());
#define TN_X3_CASE(BNV)                                                                              \
    gemm_tc_x3_kernel<BNV, BKB><<<(unsigned)grid, kTcThreads, X3Smem<BNV, BKB>::total, s>>>(ah, al, bh, bl, a); \
    break;
    switch (bn) {
        case 16: TN_X3_CASE(16)
        case 32: TN_X3_CASE(32)
        case 64: TN_X3_CASE(64)
        case 128: TN_X3_CASE(128)
        default: return cudaErrorInvalidValue;
    }
#undef TN_X3_CASE
    return cudaGetLastError();
}

}  // namespace

int tc_num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 152;     // no device (host-side planning and features): GB300's count
    }
    return n;
}

// Raster group the launcher picks when none is given (see launch_gemm_tc).
static int default_gm(int bn) {
    const int target = tc_num_sms() * bn / 128;
    int g = 1;
    while (4 * g * g <= target && g < 64) g *= 2;
    return g;
}

int tc_effective_tile(int tile, int ln) {
    const int np = std::max(16, 2 << ln);
    const int bn_max = np >= 256 ? 256 : np;
    int bn = bn_max;
    const int bq = tc_tile_bn(tile);
    if (bq > 0 && bq < bn) bn = bq;
    const int gq = tc_tile_gm(tile);
    const int gm = gq > 0 ? gq : default_gm(bn);
    int bc = 0, gc = 0;
    for (int c = 1; c < 5; ++c)
        if (kTcBn[c] == bn) bc = c;
    for (int c = 1; c < 6; ++c)
        if (kTcGm[c] == gm) gc = c;
    return bc | (gc << 4);
}

// Set the dynamic shared-memory limit of every tensor-core GEMM variant on
// the current device (must happen outside any stream capture).
cudaError_t tc_prepare() {
    static int done_mask = 0;  // one bit per device (first 31)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 31 && ((done_mask >> dev) & 1)) return cudaSuccess;
    cudaError_t e = set_attr_bn<32, false>();
    if (e == cudaSuccess) e = set_attr_bn<64, false>();
    if (e == cudaSuccess) e = set_attr_bn<128, false>();
    if (e == cudaSuccess) e = set_attr_bn<128, true>();
    if (e == cudaSuccess) e = prepare_pair<false>();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_tc_bres_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBresSmemTotal);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_tc_bres_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBresSmemTotal);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_tc_bres_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBresSmemTotal);
    if (e == cudaSuccess) e = set_attr_x3_bn<32>();
    if (e == cudaSuccess) e = set_attr_x3_bn<64>();
    if (e == cudaSuccess) e = set_attr_x3_bn<128>();
    if (e == cudaSuccess && dev < 31) done_mask |= 1 << dev;
    return e;
}

bool tc_encode_3d(CUtensorMap *m, int dtype, int esz, const void *base, uint64_t inner, uint64_t rows,
                  uint64_t depth, uint32_t box_inner, uint32_t box_rows) {
    return encode_3d(m, dtype, esz, base, inner, rows, depth, box_inner, box_rows);
}

int tc_default_gm(int bn) { return default_gm(bn); }

bool tc_bres_eligible(int lm, int ln, int lk, int64_t batch, int bn, int fp8, int gathered) {
    if (fp8 || gathered || !tc_gemm_supported(lk, ln) || lk > kSplitLog2K) return false;
    if (tc_split(lm, ln, lk, batch) != 1) return false;
    const int kreal = 2 << lk;
    const int bk = kreal >= 64 ? 64 : kreal;
    const uint32_t chunk = ((uint32_t)bn * 2 * bk + 1023u) / 1024u * 1024u;
    return (uint64_t)(kreal / bk) * chunk <= 65536;
}

bool tc_bres_store_eligible(int lm, int ln, int lk, int64_t batch, int bn) {
    if (!tc_bres_eligible(lm, ln, lk, batch, bn, 0, 0) || bn < 64 || bn % 64) return false;
    const int kreal = 2 << lk;
    const int bk = kreal >= 64 ? 64 : kreal;
    const uint64_t chunk = ((uint64_t)bn * 2 * bk + 1023u) / 1024u * 1024u;
    const uint64_t slot = (uint64_t)(kreal / bk) * chunk, stage_c = (uint64_t)(bn / 64) * 16384;
    return 2 * slot + 2 * stage_c + 2 * 128u * 2 * bk <= (uint64_t)kBresSmemBudget;
}

bool tc_gemm_supported(int lk, int ln) { return lk >= 3 && lk <= 24 && ln <= 24; }

// A step runs on CTA pairs when asked and when its tiles are the pair
// kernel's: FP16/BF16, N tile 256 real columns, 128-byte K chunks (K >= 32
// complex), M a multiple of 256.
bool tc_pair_eligible(int want, int fp8, int lm, int ln, int lk, int bn) {
    return want && !fp8 && bn == 256 && (2 << ln) >= 256 && lk >= 5 && lm >= 8;
}
bool tc_gemm_supported_fp8(int lk, int ln) { return lk >= 6 && lk <= 24 && ln <= 24; }

// K parts of one tensor-core GEMM.  Each part accumulates at most
// 2^kSplitLog2K complex terms in TMEM (the tensor cores' FP32 accumulation
// drifts with K: 2.6e-4 relative at K = 2^16, 2e-2 at 2^23 against 2e-4 for
// the output rounding alone); a step with few output tiles is cut further so
// that its parts fill the GPU, down to 512 complex terms per part and within
// 256 MB of FP32 partials.  Depends on the shape only, so a plan sizes its
// partial buffer once.
int tc_split(int lm, int ln, int lk, int64_t batch) {
    if (lk < 9) return 1;
    int split = lk > kSplitLog2K ? 1 << (lk - kSplitLog2K) : 1;
    const int np = std::max(16, 2 << ln);
    const int64_t tiles = (((int64_t)1 << lm) + 127) / 128 * (np / std::min(np, 256)) * batch;
    const int64_t part_bytes = (batch << (lm + ln)) * 8;
    const int max_split = 1 << (lk - 9);                 // parts of >= 512 complex terms
    while (split < max_split && tiles * split < tc_num_sms() &&
           part_bytes * split * 2 <= ((int64_t)256 << 20))
        split *= 2;
    return split;
}

size_t tc_split_bytes(int lm, int ln, int lk, int64_t batch) {
    const int split = tc_split(lm, ln, lk, batch);
    return split > 1 ? (size_t)split * (size_t)(batch << (lm + ln)) * 8 : 0;
}

cudaError_t tc_setup(const TcGemmDesc &d, const ScaleRef &sr, int32_t *d_err, bool one_cta, CUtensorMap *ma_out,
                     CUtensorMap *mb_out, TcArgs *a_out, int *bn_out, int *bk_out, bool *pair_out) {
    if (d.fp8 ? !tc_gemm_supported_fp8(d.lk, d.ln) : !tc_gemm_supported(d.lk, d.ln))
        return cudaErrorInvalidValue;
    if (d.x3 && (d.fp8 || d.pair || d.za || d.zb || d.zc || d.gather_r || !d.out_c64 || !d.A2 || !d.Bp2))
        return cudaErrorInvalidValue;
    const int esz = d.x3 ? 4 : d.fp8 ? 1 : 2;
    const int kreal = 2 << d.lk;                 // 2K elements
    // K chunk: 128-byte rows where K allows (FP8: always, K >= 64)
    int bk = d.x3 ? (kreal >= 32 ? 32 : kreal) : d.fp8 ? 128 : (kreal >= 64 ? 64 : kreal);
    int bn = d.np >= (d.x3 ? 128 : 256) ? (d.x3 ? 128 : 256) : d.np;   // 16 .. 256 (x3: 128)
    if (d.bn > 0) {
        if ((d.bn & (d.bn - 1)) != 0 || d.bn < 16 || d.bn > 256) return cudaErrorInvalidValue;
        bn = (d.bn < bn || d.gather_r > 0) ? d.bn : bn;   // B_P tiles span several chunks
    }
    if (d.x3 && bn > 128) bn = 128;
    const int64_t M = (int64_t)1 << d.lm;
    const bool gathered = d.za || d.zb || d.zc;
    // CTA pairs: 256 x 256 tiles of FP16/BF16 with 128-byte K chunks
    const bool pair = !one_cta && tc_pair_eligible(d.pair, d.fp8, d.lm, d.ln, d.lk, bn) && !gathered &&
                      d.gather_r == 0;
    if (d.half_k && !pair && !d.fp8 && bk == 64) bk = 32;
    CUtensorMap &ma = *ma_out, &mb = *mb_out;
    const int64_t depth_a = d.depth_a > 0 ? d.depth_a : (d.batch_a ? d.batch : 1);
    const int64_t depth_b = d.depth_b > 0 ? d.depth_b : (d.batch_b ? d.batch : 1);
    if (!encode_3d(&ma, d.dtype, esz, d.A, (uint64_t)kreal, (uint64_t)M, (uint64_t)depth_a, bk, 128))
        return cudaErrorInvalidValue;
    if (d.gather_r > 0 && (bn % d.np != 0 || bn / d.np != d.gather_r)) return cudaErrorInvalidValue;
    if (!encode_3d(&mb, d.dtype, esz, d.Bp, (uint64_t)kreal, (uint64_t)d.np, (uint64_t)depth_b, bk,
                   d.gather_r > 0 ? d.np : (pair ? bn / 2 : bn)))
        return cudaErrorInvalidValue;
    TcArgs &a = *a_out;
    a = TcArgs{};
    a.C = d.C;
    a.M = M;
    a.n_mt = pair ? M / 256 : (M + 127) / 128;
    a.n_nt = d.gather_r > 0 ? ((int64_t)d.m_r * d.np + bn - 1) / bn : d.np / bn;
    a.batch = d.batch;
    a.tiles = a.n_mt * a.n_nt * d.batch;
    a.N = 1 << d.ln;
    a.lk = d.lk;
    a.nk = kreal / bk;
    if (gathered && d.lk > kSplitLog2K) return cudaErrorInvalidValue;   // one K part only
    if (d.out_rank > 0 && d.lk > kSplitLog2K) return cudaErrorInvalidValue;
    // a permuted C is written by this kernel's epilogue, so no K parts
    a.split = (d.withhold || gathered || d.out_rank > 0) ? 1 : tc_split(d.lm, d.ln, d.lk, d.batch);
    a.partial = a.split > 1 ? d.partial : nullptr;
    if (a.split > 1) {
        if (!d.partial || a.nk % a.split != 0) return cudaErrorInvalidValue;
        a.nk /= a.split;
    }
    a.tiles_per_part = a.tiles;
    a.tiles *= a.split;
    a.dtype = d.dtype;
    a.batch_a = d.batch_a;
    a.batch_b = d.batch_b;
    a.withhold = d.withhold;
    a.za = d.za;
    a.zb = d.zb;
    a.zc = d.zc;
    a.gather_r = d.gather_r;
    a.m_r = d.m_r;
    a.np_chunk = d.np;
    a.out_rank = d.out_rank;
    a.ln = d.ln;
    a.staged = d.staged;
    for (int i = 0; i < 40; ++i) a.out_dpos[i] = i < d.out_rank ? d.out_dpos[i] : 0;
    if (a.out_rank > 0 && (a.N < 8 || a.out_rank > 40)) return cudaErrorInvalidValue;
    a.out_c64 = d.out_c64;
    if (d.gm > 0) {
        a.gm = d.gm;
    } else {
        // A wave of one tile per SM covers gm m-tiles x (SMs / gm) n-tiles, and
        // its CTAs walk K roughly in step, so L2 only has to hold the current
        // K chunk of the wave's operands while DRAM delivers each of its
        // gm A tiles (128 rows) and SMs/gm B' tiles (BN rows) once: fewest
        // bytes at gm^2 = SMs * BN / 128 (power of two at or below).
        a.gm = default_gm(bn);
    }
    if (pair) a.gm = std::max(1, a.gm / 2);   // gm counts 128-row m tiles
    a.sr = sr;
    a.err = d_err;
    *bn_out = bn;
    *bk_out = bk;
    *pair_out = pair;
    return cudaSuccess;
}

// B'-resident launch (gemm_tc_bres_kernel) when the step allows it: one K
// part, no gathers, 1-CTA FP16/BF16 tiles, the whole K of a B' slice within
// 64 KiB.  Returns false when it does not apply.
bool bres_config(const TcArgs &a, int bn, int bkb, bool pair, int fp8, bool tma_store, BresCfg &cfg) {
    if (pair || fp8 || a.split != 1 || a.za || a.zb || a.zc || a.gather_r || a.withhold) return false;
    const uint32_t chunk = ((uint32_t)bn * bkb + 1023u) / 1024u * 1024u;
    const uint64_t slot = (uint64_t)a.nk * chunk;
    if (slot > 65536) return false;
    // TMA stores of staged C tiles: complex-half C in natural order, N tiles
    // of whole 64-column panels
    const bool st = tma_store && !a.out_c64 && a.out_rank == 0 && !a.partial && bn >= 64 && bn % 64 == 0;
    const uint64_t stage_c = st ? (uint64_t)(bn / 64) * 16384 : 0;
    if (2 * slot + 2 * stage_c >= (uint64_t)kBresSmemBudget) return false;
    const int stages = (int)std::min<uint64_t>(kBresMaxStages, (kBresSmemBudget - 2 * slot - 2 * stage_c) / (128u * bkb));
    if (stages < 2) return false;
    cfg.bn = bn;
    cfg.stages = stages;
    cfg.chunk_bytes = chunk;
    cfg.slot_bytes = (uint32_t)slot;
    cfg.tma_store = st ? 1 : 0;
    cfg.stage_c_bytes = (uint32_t)stage_c;
    return true;
}

template <int BKB>
cudaError_t run_tc_bres(const CUtensorMap &ma, const CUtensorMap &mb, const TcArgs &a, const BresCfg &cfg,
                        cudaStream_t s) {
    // a grid that is a multiple of the n tiles keeps each walker on one n tile
    int64_t grid = std::min<int64_t>(a.tiles, tc_num_sms());
    if (a.n_nt > 1 && a.n_nt <= grid) grid = grid / a.n_nt * a.n_nt;
    CUtensorMap mc;
    std::memset(&mc, 0, sizeof(mc));
    if (cfg.tma_store &&
        !encode_3d(&mc, a.dtype, 2, a.C, (uint64_t)(2 * a.N), (uint64_t)a.M, (uint64_t)a.batch, 64, 128))
        return cudaErrorInvalidValue;
    gemm_tc_bres_kernel<BKB><<<(unsigned)grid, kTcThreads, kBresSmemTotal, s>>>(ma, mb, mc, a, cfg);
    return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const TcGemmDesc &d, const ScaleRef &sr, int32_t *d_err, cudaStream_t s) {
    {
        const cudaError_t e = tc_prepare();
        if (e != cudaSuccess) return e;
    }
    CUtensorMap ma, mb;
    TcArgs a;
    int bn = 0, bk = 0;
    bool pair = false;
    {
        const cudaError_t e = tc_setup(d, sr, d_err, false, &ma, &mb, &a, &bn, &bk, &pair);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e;
    if (d.x3) {
        // the remainder maps: the same shapes and boxes over A2 and Bp2
        CUtensorMap ma2, mb2;
        const int kreal = 2 << d.lk;
        const uint64_t M = (uint64_t)1 << d.lm;
        if (!encode_3d(&ma2, d.dtype, 4, d.A2, (uint64_t)kreal, M, (uint64_t)(d.batch_a ? d.batch : 1), bk, 128) ||
            !encode_3d(&mb2, d.dtype, 4, d.Bp2, (uint64_t)kreal, (uint64_t)d.np, (uint64_t)(d.batch_b ? d.batch : 1),
                       bk, bn))
            return cudaErrorInvalidValue;
        switch (bk) {
            case 8: e = run_tc_x3<32>(bn, ma, ma2, mb, mb2, a, s); break;
            case 16: e = run_tc_x3<64>(bn, ma, ma2, mb, mb2, a, s); break;
            default: e = run_tc_x3<128>(bn, ma, ma2, mb, mb2, a, s); break;
        }
        if (e == cudaSuccess && a.split > 1)
            e = launch_splitk_reduce(a.partial, a.split, d.C, 1, d.dtype, d.batch, d.lm, d.ln, d.lk, sr, s);
        return e;
    }
    BresCfg bc;
    if (d.bres && bres_config(a, bn, 2 * bk, pair, d.fp8, d.tma_store != 0, bc)) {
        switch (bk) {
            case 16: return run_tc_bres<32>(ma, mb, a, bc, s);
            case 32: return run_tc_bres<64>(ma, mb, a, bc, s);
            default: return run_tc_bres<128>(ma, mb, a, bc, s);
        }
    }
    if (pair) {
        e = run_tc_pair<false>(ma, mb, a, s);
    } else if (d.fp8) {
        e = run_tc_bn<128, true>(bn, ma, mb, a, s);
    } else {
        switch (bk) {
            case 16: e = run_tc_bn<32, false>(bn, ma, mb, a, s); break;
            case 32: e = run_tc_bn<64, false>(bn, ma, mb, a, s); break;
            default: e = run_tc_bn<128, false>(bn, ma, mb, a, s); break;
        }
    }
    if (e == cudaSuccess && a.split > 1)
        e = launch_splitk_reduce(a.partial, a.split, d.C, d.out_c64, d.dtype, d.batch, d.lm, d.ln, d.lk, sr, s);
    return e;
}

}  // namespace tn

// Persistent work-queue executor: the whole contraction of one or many plans
// (every pass of every slice range, every step) in ONE kernel launch.
//
// The paper's slices -- and the independent circuits of a batch -- are
// independent sub-tasks (Sec. 3.1, global level); inside one slice pass the
// steps form a chain (each step's operands are earlier steps' results, and
// the workspace is reused between steps).  The host compiles the ops of all
// plans into a table of ops (leaf preparation with slice decoding,
// permutations, B' builds, CUDA-core GEMMs, tensor-core GEMM tiles, split-K
// reductions, FP64 slice sums, clears); every op is cut into tiles that any
// CTA can run, and each op depends on the op before it in its chain.
//
// One CTA of 320 threads per SM takes items from a list (see queue_kernel):
// an op's tiles are listed only when its predecessor's last tile is done
// (release: fence + atomic), so a claimed tile never waits on another and
// no CTA holds its SM while a dependency runs elsewhere.  The tiles of the
// chains' first ops are listed at launch, longest chain first.  The queue
// always progresses whether or not every CTA is resident: a CTA whose entry
// is not listed yet only waits for tiles that CTAs are running.  That wait is
// bounded (%globaltimer); when it runs out, every CTA returns and the host
// reports TN_ETIMEOUT.
//
// Tensor-core items run the same tcgen05 pipeline as the stand-alone GEMM
// (tc_gemm.cu: warp 0 TMA producer, warp 1 MMA issuer, warps 2..9 epilogue,
// accumulators in TMEM allocated once per CTA for the kernel's lifetime);
// one item is one walker of the persistent tile loop (tiles w, w + W, ...),
// so a large GEMM's tiles spread over all SMs in the usual raster order.
// SIMT items run the device bodies of kernels.cu (bodies.cuh) on warps
// 0..7 with named barriers, their shared memory aliasing the TMA ring, so
// the queue computes the same bits as the stream of stand-alone launches.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bodies.cuh"
#include "plan.h"
#include "tc_common.cuh"

namespace tn {
namespace {

constexpr int kQThreads = kTcThreads;            // 320: producer, MMA, 8 epilogue warps
constexpr int kQSimt = 256;                      // SIMT items: warps 0..7
constexpr int kQRing = 4 * (128 * 128 + 256 * 128);  // 192 KiB: 4 stages at BN = 256, 128-byte K chunks
constexpr int kQStages = 12;                     // most stages of a ring of smaller tiles
constexpr int kQBars = 2 * kQStages + 5;
constexpr int kQSmem = 1024 + kQRing + kQBars * 8 + 16;
constexpr uint32_t kQTmemCols = 512;             // two accumulators of up to 256 columns
constexpr int kQAccStride = 256;

enum QKind : int32_t {
    Q_ZERO = 1,         // clear n 32-bit words
    Q_LEAF = 2,         // leaf preparation (slice decoding), 8 leaves per item
    Q_PERM = 3,         // generic bit permutation, per_item tiles per item
    Q_PERM_TILED = 4,   // tiled permutation or B' expansion, per_item tiles per item
    Q_BPREP_GATHER = 5, // B' by direct gather
    Q_BPREP_C64 = 6,    // B' from a complex64 B (one item)
    Q_ROWS = 7,         // CUDA-core GEMM, two 128-row blocks per item
    Q_TILED_C64 = 8,    // complex64 tiled GEMM, one 64x64 tile per item
    Q_TC = 9,           // tensor-core GEMM, one tile walker per item
    Q_SPLITK = 10,      // FP64 sum of split-K parts
    Q_SUM = 11,         // FP64 slice sum into the amplitudes
};

struct QOp {
    int32_t kind, sub;
    int32_t ntiles;     // items of this op
    int32_t next;       // the op after this one in its chain (-1: last)
    int32_t chain, pad_;
    int64_t prm;        // byte offset of the parameter record in the blob
};

constexpr int kQKinds = 12;
struct QState {
    int32_t head;       // next ticket: the list entry the next claiming CTA takes
    int32_t tail;       // list entries reserved by the ops listed so far
    int32_t abort;      // 1: a wait ran out; every CTA returns
    int32_t err;        // bit 0: a listed entry did not appear within the wait limit
    int32_t idle_at;    // list entry whose wait ran out
    int32_t pad_;
    // profiling (tn_queue_profile): per op kind, items run, ns spent waiting
    // for the list entry, ns running (summed over CTAs)
    unsigned long long items[kQKinds], wait_ns[kQKinds], busy_ns[kQKinds];
};

struct QZero { uint32_t *p; int64_t n, per_item; };
struct QLeaf {
    const LeafJob *jobs;
    const double2 *store;
    char *ws;
    float *tmax;
    int32_t *texp;
    int64_t slice_base;
    int32_t count, pad_;
};
struct QPerm {
    const void *in;
    void *out;
    int64_t ntiles;
    int32_t per_item, esz, expand, pad_;
    ExpandArgs ex;
    int32_t pad2_;
    PermParams pp;
};
struct QBprepGather {
    const uint32_t *B;
    uint32_t *Bp;
    int64_t total, per_item;
    int32_t lk, ln, np, rank;
    PermParams g;
};
struct QBprepC64 {
    const float2 *B;
    uint32_t *Bp;
    double2 *corr;
    float *tmax;
    int32_t *texp;
    int32_t lk, ln, lb, np, rank, meta_src, meta_dst, scale_off;
    PermParams g;
};
struct QRows {
    const void *A, *B;
    void *C;
    const int32_t *za, *zb;
    int64_t sa, sb, sc;
    int64_t gx, gx2;    // 128-row blocks, pairs of them
    int32_t gy, lm, ln, lk;
    ScaleRef sr;
};
struct QTiled {
    const float2 *A, *B;
    float2 *C;
    const int32_t *za, *zb;
    int64_t sa, sb, sc, gx;
    int32_t gy, lm, ln, lk;
};
struct QTc {
    CUtensorMap ma, mb;   // 64-byte aligned (records are 256-byte aligned)
    TcArgs a;
    int32_t bn, bkb;      // N tile (real columns), K chunk (bytes per row)
};
struct QSplitK {
    const float2 *partial;
    void *C;
    int64_t n, per_item;
    int32_t split, lk;
    ScaleRef sr;
};
struct QSum {
    const void *F;
    double2 *amps;
    const int32_t *texp;
    const double2 *stepcorr;
    uint64_t split_mask, split_val;
    int32_t n_open, t_lo, t_hi, overwrite, n_steps, pad_;
    SumOp op;
};

// sub codes
//   Q_PERM / Q_PERM_TILED: element bytes (4 or 8); expand flag in the record
//   Q_BPREP_C64: dtype
//   Q_ROWS: dt (0 complex64, 1 FP16, 2 BF16) | ta << 2 | tb << 3 | tc << 4 | nc_log2 << 5
//   Q_TILED_C64: 1 = long K (FP64 partial sums)
//   Q_SPLITK: dtype | out_c64 << 4
//   Q_SUM: dtype | tf << 4

__device__ __forceinline__ int32_t ld_acquire(const int32_t *p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void nanosleep_ns(uint32_t ns) { asm volatile("nanosleep.u32 %0;" ::"r"(ns)); }

// ------------------------------------------------------------ SIMT items --
template <typename T>
__device__ __noinline__ void q_perm(const QPerm &r, int64_t tile, int tid, uint8_t *scratch) {
    const int64_t t0 = tile * r.per_item, t1 = min(r.ntiles, t0 + r.per_item);
    T *sm = reinterpret_cast<T *>(scratch);
    for (int64_t t = t0; t < t1; ++t) {
        permute_tile_body<T, SyncNamed<1, kQSimt>>(reinterpret_cast<const T *>(r.in), reinterpret_cast<T *>(r.out),
                                                   r.pp, t, tid, kQSimt, sm);
        SyncNamed<1, kQSimt>::sync();
    }
}

template <typename T, bool EXPAND>
__device__ __noinline__ void q_perm_tiled(const QPerm &r, int64_t tile, int tid, uint8_t *scratch) {
    const int64_t t0 = tile * r.per_item, t1 = min(r.ntiles, t0 + r.per_item);
    permute_tiled_body<T, EXPAND, SyncNamed<1, kQSimt>>(reinterpret_cast<const T *>(r.in), r.out, r.pp, t0, t1, 1,
                                                        r.ex, tid, *reinterpret_cast<PermTiledSmem<T> *>(scratch));
}

__device__ __noinline__ void q_bprep_gather(const QBprepGather &r, int64_t tile, int tid) {
    const int64_t i0 = tile * r.per_item, i1 = min(r.total, i0 + r.per_item);
    bprep_gather_body(r.B, r.Bp, r.lk, r.ln, r.np, r.g, r.rank, i0 + tid, i1, kQSimt);
}

// B already in [batch][N][K] order: per_item 16-byte units of B' row pairs
__device__ __noinline__ void q_bprep_stream(const QBprepGather &r, int64_t tile, int tid) {
    const int64_t i0 = tile * r.per_item, i1 = min(r.total, i0 + r.per_item);
    bprep_stream_body<4>(reinterpret_cast<const uint4 *>(r.B), reinterpret_cast<uint4 *>(r.Bp), r.lk, r.ln, r.np,
                         i0 + tid, i1, kQSimt);
}

template <int DT>
__device__ __noinline__ void q_bprep_c64(const QBprepC64 &r, int tid, uint8_t *scratch) {
    // the stand-alone kernel's 1024-thread summation order, played by 256 threads
    bprep_c64_body<DT, kQSimt, 1024, SyncNamed<1, kQSimt>>(r.B, r.Bp, r.lk, r.ln, r.lb, r.np, r.g, r.rank, r.corr,
                                                           r.tmax, r.texp, r.meta_src, r.meta_dst, r.scale_off, tid,
                                                           *reinterpret_cast<BprepC64Smem<1024> *>(scratch));
}

// two 128-row blocks per item, one per group of 4 warps (named barriers 2, 3)
template <typename TA, typename TB, typename TC, int NC, int DT>
__device__ __noinline__ void q_rows(const QRows &r, int64_t tile, int tid, uint8_t *scratch) {
    const int64_t px = tile % r.gx2;
    const int64_t rest = tile / r.gx2;
    const int by = (int)(rest % r.gy);
    const int64_t bz = rest / r.gy;
    const int g = tid >> 7;
    const int64_t bx = 2 * px + g;
    if (bx >= r.gx) return;
    auto *sm = reinterpret_cast<RowsSmem<TA, NC> *>(scratch + (size_t)g * ((sizeof(RowsSmem<TA, NC>) + 255) / 256 * 256));
    const TA *A = reinterpret_cast<const TA *>(r.A);
    const TB *B = reinterpret_cast<const TB *>(r.B);
    TC *C = reinterpret_cast<TC *>(r.C);
    float mx = 0.f;
    if (g == 0)
        rows_body<TA, TB, TC, NC, DT, SyncNamed<2, 128>>(A, B, C, r.lm, r.ln, r.lk, r.sa, r.sb, r.sc, r.sr, r.za, r.zb,
                                                         bx, by, bz, tid & 127, *sm, mx);
    else
        rows_body<TA, TB, TC, NC, DT, SyncNamed<3, 128>>(A, B, C, r.lm, r.ln, r.lk, r.sa, r.sb, r.sc, r.sr, r.za, r.zb,
                                                         bx, by, bz, tid & 127, *sm, mx);
    rows_flush<TC, DT>(r.sr, mx, tid);
}

template <typename TA, typename TB, typename TC, int DT>
__device__ __forceinline__ void q_rows_nc(const QRows &r, int ncl, int64_t tile, int tid, uint8_t *scratch) {
    switch (ncl) {
        case 0: q_rows<TA, TB, TC, 1, DT>(r, tile, tid, scratch); break;
        case 1: q_rows<TA, TB, TC, 2, DT>(r, tile, tid, scratch); break;
        case 2: q_rows<TA, TB, TC, 4, DT>(r, tile, tid, scratch); break;
        case 3: q_rows<TA, TB, TC, 8, DT>(r, tile, tid, scratch); break;
        default: q_rows<TA, TB, TC, 16, DT>(r, tile, tid, scratch); break;
    }
}

template <int DT, typename H>
__device__ __forceinline__ void q_rows_mixed(const QRows &r, int code, int ncl, int64_t tile, int tid,
                                             uint8_t *scratch) {
    switch (code) {
        case 0: q_rows_nc<float2, float2, float2, DT>(r, ncl, tile, tid, scratch); break;
        case 1: q_rows_nc<float2, float2, H, DT>(r, ncl, tile, tid, scratch); break;
        case 4: q_rows_nc<H, float2, float2, DT>(r, ncl, tile, tid, scratch); break;
        case 5: q_rows_nc<H, float2, H, DT>(r, ncl, tile, tid, scratch); break;
        case 6: q_rows_nc<H, H, float2, DT>(r, ncl, tile, tid, scratch); break;
        default: q_rows_nc<H, H, H, DT>(r, ncl, tile, tid, scratch); break;
    }
}

__device__ __noinline__ void q_rows_dispatch(const QRows &r, int sub, int64_t tile, int tid, uint8_t *scratch) {
    const int dt = sub & 3, ncl = (sub >> 5) & 7;
    const int code = ((sub >> 2) & 1) * 4 + ((sub >> 3) & 1) * 2 + ((sub >> 4) & 1);
    if (dt == 0) q_rows_nc<float2, float2, float2, TN_C64>(r, ncl, tile, tid, scratch);
    else if (dt == 1) q_rows_mixed<TN_F16, __half2>(r, code, ncl, tile, tid, scratch);
    else q_rows_mixed<TN_BF16, __nv_bfloat162>(r, code, ncl, tile, tid, scratch);
}

template <bool LONGK>
__device__ __noinline__ void q_tiled(const QTiled &r, int64_t tile, int tid, uint8_t *scratch) {
    const int64_t bx = tile % r.gx;
    const int64_t rest = tile / r.gx;
    const int by = (int)(rest % r.gy);
    const int64_t bz = rest / r.gy;
    tiled_c64_body<64, 64, 16, LONGK, SyncNamed<1, kQSimt>>(r.A, r.B, r.C, r.lm, r.ln, r.lk, r.sa, r.sb, r.sc, r.za,
                                                           r.zb, bx, by, bz, tid,
                                                           *reinterpret_cast<TiledC64Smem<64, 64, 16> *>(scratch));
}

template <int DT, bool OUT_C64>
__device__ __noinline__ void q_splitk(const QSplitK &r, int64_t tile, int tid) {
    const int64_t i0 = tile * r.per_item, i1 = min(r.n, i0 + r.per_item);
    splitk_body<DT, OUT_C64>(r.partial, r.split, r.C, r.n, r.lk, r.sr, i0 + tid, i1, kQSimt, tile == 0, tid);
}

template <typename TF, int DT>
__device__ __noinline__ void q_sum(const QSum &r, int64_t tile, int tid, uint8_t *scratch) {
    double2 *corr = reinterpret_cast<double2 *>(scratch);
    if (tid == 0) *corr = slice_corr(r.stepcorr, r.n_steps);
    SyncNamed<1, kQSimt>::sync();
    slice_sum_body<TF, DT>(reinterpret_cast<const TF *>(r.F), r.op, r.amps, r.n_open, r.t_lo, r.t_hi, r.overwrite,
                           r.texp, *corr, r.n_steps, r.split_mask, r.split_val, tile * kQSimt + tid);
}

__device__ __noinline__ void q_simt(const QOp &op, const uint8_t *blob, int64_t tile, int tid, uint8_t *scratch) {
    const uint8_t *rec = blob + op.prm;
    switch (op.kind) {
        case Q_ZERO: {
            const QZero &r = *reinterpret_cast<const QZero *>(rec);
            const int64_t i0 = tile * r.per_item, i1 = min(r.n, i0 + r.per_item);
            for (int64_t i = i0 + tid; i < i1; i += kQSimt) r.p[i] = 0u;
            break;
        }
        case Q_LEAF: {
            const QLeaf &r = *reinterpret_cast<const QLeaf *>(rec);
            const int64_t l = tile * 8 + (tid >> 5);
            if (l < r.count) leaf_warp_body(r.jobs[l], r.store, r.ws, r.slice_base, r.tmax, r.texp, tid & 31);
            break;
        }
        case Q_PERM: {
            const QPerm &r = *reinterpret_cast<const QPerm *>(rec);
            if (op.sub == 4) q_perm<uint32_t>(r, tile, tid, scratch);
            else q_perm<uint2>(r, tile, tid, scratch);
            break;
        }
        case Q_PERM_TILED: {
            const QPerm &r = *reinterpret_cast<const QPerm *>(rec);
            if (r.expand) q_perm_tiled<uint32_t, true>(r, tile, tid, scratch);
            else if (op.sub == 4) q_perm_tiled<uint32_t, false>(r, tile, tid, scratch);
            else q_perm_tiled<uint2, false>(r, tile, tid, scratch);
            break;
        }
        case Q_BPREP_GATHER:
            if (op.sub == 1) q_bprep_stream(*reinterpret_cast<const QBprepGather *>(rec), tile, tid);
            else q_bprep_gather(*reinterpret_cast<const QBprepGather *>(rec), tile, tid);
            break;
        case Q_BPREP_C64:
            if (op.sub == TN_F16) q_bprep_c64<TN_F16>(*reinterpret_cast<const QBprepC64 *>(rec), tid, scratch);
            else q_bprep_c64<TN_BF16>(*reinterpret_cast<const QBprepC64 *>(rec), tid, scratch);
            break;
        case Q_ROWS: q_rows_dispatch(*reinterpret_cast<const QRows *>(rec), op.sub, tile, tid, scratch); break;
        case Q_TILED_C64:
            if (op.sub) q_tiled<true>(*reinterpret_cast<const QTiled *>(rec), tile, tid, scratch);
            else q_tiled<false>(*reinterpret_cast<const QTiled *>(rec), tile, tid, scratch);
            break;
        case Q_SPLITK: {
            const QSplitK &r = *reinterpret_cast<const QSplitK *>(rec);
            const int dt = op.sub & 15, oc = op.sub >> 4;
            if (dt == TN_F16) {
                if (oc) q_splitk<TN_F16, true>(r, tile, tid);
                else q_splitk<TN_F16, false>(r, tile, tid);
            } else {
                if (oc) q_splitk<TN_BF16, true>(r, tile, tid);
                else q_splitk<TN_BF16, false>(r, tile, tid);
            }
            break;
        }
        case Q_SUM: {
            const QSum &r = *reinterpret_cast<const QSum *>(rec);
            const int dt = op.sub & 15, tf = op.sub >> 4;
            if (dt == TN_C64) q_sum<float2, TN_C64>(r, tile, tid, scratch);
            else if (tf == 0 && dt == TN_F16) q_sum<float2, TN_F16>(r, tile, tid, scratch);
            else if (tf == 0) q_sum<float2, TN_BF16>(r, tile, tid, scratch);
            else if (dt == TN_F16) q_sum<__half2, TN_F16>(r, tile, tid, scratch);
            else q_sum<__nv_bfloat162, TN_BF16>(r, tile, tid, scratch);
            break;
        }
        default: break;
    }
}

// ----------------------------------------------------- tensor-core items --
template <int BKB>
__device__ __forceinline__ void q_mma_chunk(uint32_t d_tmem, uint32_t a_addr, uint32_t b_addr, uint32_t idesc,
                                            bool first) {
#pragma unroll
    for (int kk = 0; kk < BKB / 32; ++kk) {     // 32 bytes of K per MMA
        const uint64_t ad = smem_desc<BKB>(a_addr + kk * 32);
        const uint64_t bd = smem_desc<BKB>(b_addr + kk * 32);
        tc_mma<false, false>(d_tmem, ad, bd, idesc, (!first || kk > 0) ? 1u : 0u);
    }
}

// Ring and accumulator state kept across items.  A tensor-core item cuts
// the ring into as many stages as its tile size allows (up to kQStages) and
// walks them from stage 0; each stage barrier's phase parity is tracked per
// stage (bit s of the masks), so items with different stage counts follow
// one another.
struct TcPipe {
    uint32_t p_bits;     // producer: parity of the next fill of stage s
    uint32_t m_bits;     // MMA: parity of the next consumption of stage s
    int m_acc, e_acc;
    uint32_t m_acc_phase, e_acc_phase;
};

// One walker (tiles w, w + W, ...) of a tensor-core GEMM.  Returns false
// when a bounded wait ran out (abort_flag set; in-flight loads and MMAs
// drained).
__device__ __forceinline__ bool q_tc(const QTc &R, int64_t walker, int64_t walkers, uint8_t *ring, uint64_t *full,
                                     uint64_t *empty, uint64_t *accf, uint64_t *acce, uint64_t *drain,
                                     uint32_t tmem_base, volatile int *abort_flag, TcPipe &st) {
    // a private copy: the epilogue's stores to global memory cannot alias it,
    // so its fields stay in registers across them
    const TcArgs args = R.a;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int bn = R.bn, bkb = R.bkb;
    const int bk = bkb / 2;                 // K chunk in FP16/BF16 elements
    const uint32_t a_bytes = 128u * bkb, b_bytes = (uint32_t)bn * bkb;
    const uint32_t stage_bytes = (a_bytes + b_bytes + 1023u) / 1024u * 1024u;
    const int n_st = min(kQStages, (int)(kQRing / stage_bytes));
    const int64_t tiles = args.tiles;
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            // generic-proxy writes (earlier SIMT items in this CTA's ring,
            // other CTAs' results in global memory) before async-proxy reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("fence.proxy.async.global;" ::: "memory");
            int8_t armed[kQStages];
            for (int s = 0; s < kQStages; ++s) armed[s] = -1;
            int stage = 0;
            for (int64_t t = walker; t < tiles && ok; t += walkers) {
                int64_t b, mt;
                int nt;
                tile_coords(args, t, b, mt, nt);
                const int kbase = (int)(t / args.tiles_per_part) * args.nk * bk;
                // the tile's batch coordinates, once per tile
                const int zA = args.za ? args.za[b] : (args.batch_a ? (int)b : 0);
                const int zB = args.zb ? max(0, args.zb[b]) : (args.batch_b ? (int)b : 0);
                for (int kc = 0; kc < args.nk; ++kc) {
                    const uint32_t par = (st.p_bits >> stage) & 1u;
                    if (!mbar_wait(&empty[stage], par ^ 1u, abort_flag)) { ok = false; break; }
                    uint8_t *sa = ring + stage * stage_bytes;
                    uint8_t *sb = sa + a_bytes;
                    mbar_expect_tx(&full[stage], a_bytes + b_bytes);
                    tma_load_3d(sa, &R.ma, &full[stage], kbase + kc * bk, (int)(mt * 128), zA);
                    tma_load_3d(sb, &R.mb, &full[stage], kbase + kc * bk, nt * bn, zB);
                    armed[stage] = (int8_t)par;
                    st.p_bits ^= 1u << stage;
                    if (++stage == n_st) stage = 0;
                }
            }
            if (!ok) {
                for (int s = 0; s < kQStages; ++s) {
                    if (armed[s] < 0) continue;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try_wait(&full[s], (uint32_t)armed[s]) && globaltimer() - t0 < kWaitLimitNs / 4) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t idesc = 0;
            idesc |= 1u << 4;                                  // D = F32
            const uint32_t fmt = args.dtype == TN_BF16 ? 1u : 0u;
            idesc |= fmt << 7;                                 // A format
            idesc |= fmt << 10;                                // B format
            idesc |= (uint32_t)(bn >> 3) << 17;                // N
            idesc |= (uint32_t)(128 >> 4) << 24;               // M
            bool issued = false;
            int stage = 0;
            for (int64_t t = walker; t < tiles && ok; t += walkers) {
                if (!mbar_wait(&acce[st.m_acc], st.m_acc_phase ^ 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(st.m_acc * kQAccStride);
                for (int kc = 0; kc < args.nk; ++kc) {
                    if (!mbar_wait(&full[stage], (st.m_bits >> stage) & 1u, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(ring + stage * stage_bytes);
                    const uint32_t b_addr = a_addr + a_bytes;
                    if (bkb == 128) q_mma_chunk<128>(d_tmem, a_addr, b_addr, idesc, kc == 0);
                    else if (bkb == 64) q_mma_chunk<64>(d_tmem, a_addr, b_addr, idesc, kc == 0);
                    else q_mma_chunk<32>(d_tmem, a_addr, b_addr, idesc, kc == 0);
                    issued = true;
                    tc_commit(&empty[stage]);
                    st.m_bits ^= 1u << stage;
                    if (++stage == n_st) stage = 0;
                }
                if (!ok) break;
                tc_commit(&accf[st.m_acc]);
                if (++st.m_acc == 2) { st.m_acc = 0; st.m_acc_phase ^= 1; }
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
        // epilogue: two warps per TMEM lane quadrant, alternate 16-column chunks
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        int e;
        if (args.out_c64 || args.sr.scale_off) e = 0;
        else if (args.sr.tmax)
            e = min(120, scale_exp_tc(args.sr.tmax[args.sr.meta_a], args.sr.tmax[args.sr.meta_b], args.lk) +
                             args.sr.headroom);
        else e = args.sr.fixed_exp;
        if (args.sr.texp && !args.partial && walker == 0 && threadIdx.x == 64)
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
        for (int64_t t = walker; t < tiles; t += walkers) {
            int64_t b, mt;
            int nt;
            tile_coords(args, t, b, mt, nt);
            if (!mbar_wait(&accf[st.e_acc], st.e_acc_phase, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const int64_t m = mt * 128 + row;
            const int col0 = nt * bn;
            const int64_t cb = args.zc ? (int64_t)args.zc[b] : b;
            int64_t prow = 0;
            if (args.out_rank) prow = permute_bits(args, (cb * args.M + m) * (int64_t)args.N, args.ln, args.out_rank);
            const int col_end = min(bn, 2 * args.N - col0);
            for (int c = 16 * half; c < col_end; c += 32) {
                uint32_t r[16];
                tmem_ld16<16>(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(st.e_acc * kQAccStride + c), r);
                tmem_wait_ld();
                tc_store16(args, r, b, m, t, col0, c, col_end, cb, prow, lowtab, low_kept, sc, mx);
            }
            tc_fence_before();
            mbar_arrive(&acce[st.e_acc]);
            if (++st.e_acc == 2) { st.e_acc = 0; st.e_acc_phase ^= 1; }
        }
        mx = warp_max(mx);
        if (lane == 0 && args.sr.out_max && !args.partial)
            atomicMax(reinterpret_cast<int *>(args.sr.out_max), __float_as_int(mx));
        if (lane == 0 && args.sr.err && args.dtype == TN_F16 && !args.out_c64 && !args.partial && !(mx <= 65504.0f))
            atomicOr(args.sr.err, 2);
    }
    return ok;
}

// ------------------------------------------------------------------ kernel --
// Scheduling: a list of items (op << 32 | tile), one entry per tile of every
// op.  The tiles of the chains' first ops are listed at launch; when the
// last tile of an op is counted done, the CTA that counted it reserves
// entries for every tile of the op's successor (one atomic on the tail) and
// writes them with all its threads.  A CTA claims the next entry with one
// atomic on the head (a ticket) and runs it as soon as it is written -- so a
// tile is only run when everything it depends on has finished, and an entry
// is taken by the first CTA free.  Only a CTA whose ticket is not yet listed
// waits, for tiles that other CTAs are running; that wait is bounded.
__device__ __forceinline__ long long ld_acquire64(const long long *p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kQThreads, 1)
    queue_kernel(const QOp *ops, int32_t n_items, const uint8_t *blob, int32_t *done, long long *list, QState *st,
                 uint64_t idle_limit_ns, int profile) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *ring = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(ring + kQRing);
    uint64_t *empty = full + kQStages;
    uint64_t *accf = empty + kQStages;
    uint64_t *acce = accf + 2;
    uint64_t *drain = acce + 2;
    volatile uint32_t *tmem_slot = (volatile uint32_t *)(drain + 1);
    __shared__ int s_op, s_tile;
    __shared__ int s_push_op, s_push_n, s_push_at;
    __shared__ int abort_flag;

    const int warp = threadIdx.x / 32;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < kQStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], kEpiThreads);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)tmem_slot)),
                     "r"(kQTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    TcPipe pipe{0u, 0u, 0, 0, 0u, 0u};
    uint64_t t_claim = 0, t_ready = 0;

    while (true) {
        if (threadIdx.x == 0) {
            t_claim = globaltimer();
            int op_id = -1, tile = 0;
            const int32_t h = *(volatile int32_t *)&st->abort ? n_items : atomicAdd(&st->head, 1);
            if (h < n_items) {
                long long e = ld_acquire64(list + h);
                uint32_t ns = 32;
                while (e < 0) {
                    if (*(volatile int32_t *)&st->abort) break;
                    if (globaltimer() - t_claim > idle_limit_ns) {
                        atomicOr(&st->err, 1);
                        atomicExch(&st->idle_at, h);
                        atomicExch(&st->abort, 1);
                        break;
                    }
                    nanosleep_ns(ns);
                    if (ns < 256) ns *= 2;
                    e = ld_acquire64(list + h);
                }
                if (e >= 0) {
                    op_id = (int)(e >> 32);
                    tile = (int)(e & 0xffffffffll);
                }
            }
            // the op's inputs, written by other CTAs through the generic
            // proxy, before any load here
            __threadfence();
            s_op = op_id;
            s_tile = tile;
            t_ready = globaltimer();
        }
        __syncthreads();
        const int op_id = s_op;
        if (op_id < 0) break;
        const int tile = s_tile;
        const QOp &op = ops[op_id];
        if (op.kind == Q_TC) {
            const QTc &R = *reinterpret_cast<const QTc *>(blob + op.prm);
            const bool ok = q_tc(R, tile, op.ntiles, ring, full, empty, accf, acce, drain, tmem_base, &abort_flag, pipe);
            (void)ok;
            tc_fence_before();
        } else if (threadIdx.x < kQSimt) {
            q_simt(op, blob, tile, threadIdx.x, ring);
            // generic writes to the ring before later TMA loads into it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (abort_flag) {
            if (threadIdx.x == 0) {
                atomicOr(&st->err, 1);
                atomicExch(&st->abort, 1);
            }
            break;
        }
        if (threadIdx.x == 0) {
            __threadfence();
            const int32_t d = atomicAdd(done + op_id, 1) + 1;
            s_push_n = 0;
            if (d == op.ntiles && op.next >= 0) {
                // every tile of this op is done (the other tiles' writes are
                // ordered before their counts): list the successor's tiles
                __threadfence();
                const int32_t n = ops[op.next].ntiles;
                s_push_op = op.next;
                s_push_n = n;
                s_push_at = atomicAdd(&st->tail, n);
            }
            if (profile) {
                const int kind = op.kind < kQKinds ? op.kind : 0;
                atomicAdd(&st->items[kind], 1ull);
                atomicAdd(&st->wait_ns[kind], (unsigned long long)(t_ready - t_claim));
                atomicAdd(&st->busy_ns[kind], (unsigned long long)(globaltimer() - t_ready));
            }
        }
        __syncthreads();
        if (s_push_n > 0) {
            __threadfence();
            const long long hi = (long long)s_push_op << 32;
            for (int t = threadIdx.x; t < s_push_n; t += kQThreads)
                *(volatile long long *)(list + s_push_at + t) = hi | (long long)t;
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kQTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------- builder --
struct Builder {
    std::vector<QOp> ops;
    std::vector<uint8_t> blob;
    std::vector<std::vector<int>> chains;

    template <class R>
    int64_t rec(const R &r) {
        const size_t off = (blob.size() + 255) / 256 * 256;
        blob.resize(off + sizeof(R));
        std::memcpy(blob.data() + off, &r, sizeof(R));
        return (int64_t)off;
    }
    int add(int chain, int kind, int sub, int64_t ntiles, int64_t prm) {
        QOp o{};
        o.kind = kind;
        o.sub = sub;
        o.ntiles = (int32_t)std::max<int64_t>(1, ntiles);
        o.next = -1;
        o.chain = chain;
        o.prm = prm;
        ops.push_back(o);
        chains[chain].push_back((int)ops.size() - 1);
        return (int)ops.size() - 1;
    }
    void zero(int chain, void *p, int64_t words) {
        if (words <= 0) return;
        QZero r{(uint32_t *)p, words, 4096};
        add(chain, Q_ZERO, 0, (words + 4095) / 4096, rec(r));
    }
};

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// One plan op (as run_op_raw launches it) -> queue ops on `chain`.
int emit_op(Builder &Bd, int chain, tn_plan_s *P, const Op &op, int64_t slice_base, double2 *amps, int t_lo,
            int t_hi, int overwrite, int walkers) {
    const int dtype = P->opts.dtype;
    char *ws = P->d_ws;
    switch (op.kind) {
        case OP_LEAF: {
            QLeaf r{};
            r.jobs = P->d_jobs + op.leaf_first;
            r.store = P->d_store;
            r.ws = ws;
            r.tmax = dtype == TN_C64 ? nullptr : P->d_tmax;
            r.texp = P->d_texp;
            r.slice_base = slice_base;
            r.count = op.leaf_count;
            if (op.leaf_count > 0) Bd.add(chain, Q_LEAF, 0, cdiv(op.leaf_count, 8), Bd.rec(r));
            return TN_OK;
        }
        case OP_PERM: {
            QPerm r{};
            r.pp = make_perm_params(op.perm.rank, op.perm.perm);
            r.in = ws + op.perm.src;
            r.out = ws + op.perm.dst;
            r.esz = op.perm.esz;
            r.ntiles = (int64_t)1 << r.pp.n_outer;
            if (r.pp.tile_bits == 10 && r.pp.lin == 5 && r.pp.lout == 5 && r.pp.n_outer <= 32) {
                r.per_item = 16;
                Bd.add(chain, Q_PERM_TILED, op.perm.esz, cdiv(r.ntiles, r.per_item), Bd.rec(r));
            } else {
                r.per_item = 8;
                Bd.add(chain, Q_PERM, op.perm.esz, cdiv(r.ntiles, r.per_item), Bd.rec(r));
            }
            return TN_OK;
        }
        case OP_BPREP: {
            const BprepOp &b = op.bprep;
            PermParams g;
            std::memset(&g, 0, sizeof(g));
            for (int i = 0; i < b.rank; ++i) g.outer_in[b.rank - 1 - i] = (int8_t)(b.rank - 1 - b.perm[i]);
            if (b.tb == 0) {
                QBprepC64 r{};
                r.B = (const float2 *)(ws + b.src);
                r.Bp = (uint32_t *)(ws + b.dst);
                r.corr = P->d_stepcorr + b.step;
                r.tmax = P->d_tmax;
                r.texp = P->d_texp;
                r.lk = b.lk; r.ln = b.ln; r.lb = b.lb; r.np = b.np; r.rank = b.rank;
                r.meta_src = b.meta_src;
                r.meta_dst = b.meta_dst;
                r.scale_off = P->opts.no_scaling ? 1 : 0;
                r.g = g;
                Bd.add(chain, Q_BPREP_C64, dtype, 1, Bd.rec(r));
                return TN_OK;
            }
            bool ident = true;
            for (int i = 0; i < b.rank; ++i) ident = ident && b.perm[i] == i;
            if (ident && b.lk >= 2 && b.rank == b.lk + b.ln + b.lb && ((b.src | b.dst) & 15) == 0) {
                // B in [batch][N][K] order already: the streaming expansion
                QBprepGather r{};
                r.B = (const uint32_t *)(ws + b.src);
                r.Bp = (uint32_t *)(ws + b.dst);
                r.total = ((int64_t)(b.np >> 1) << (b.lk - 2)) << b.lb;   // 16-byte units
                r.per_item = 8 * kQSimt * 4;
                r.lk = b.lk; r.ln = b.ln; r.np = b.np; r.rank = b.rank;
                Bd.add(chain, Q_BPREP_GATHER, 1, cdiv(r.total, r.per_item), Bd.rec(r));
                return TN_OK;
            }
            if (b.rank >= 10 && b.lk >= 2 && b.np == 2 << b.ln) {
                const PermParams pp = make_perm_params(b.rank, b.perm);
                if (pp.tile_bits == 10 && pp.lin == 5 && pp.lout == 5 && pp.n_outer <= 32) {
                    QPerm r{};
                    r.pp = pp;
                    r.in = ws + b.src;
                    r.out = ws + b.dst;
                    r.esz = 4;
                    r.expand = 1;
                    r.ex = ExpandArgs{b.lk, b.ln, b.np};
                    r.ntiles = (int64_t)1 << pp.n_outer;
                    r.per_item = 16;
                    Bd.add(chain, Q_PERM_TILED, 4, cdiv(r.ntiles, r.per_item), Bd.rec(r));
                    return TN_OK;
                }
            }
            QBprepGather r{};
            r.B = (const uint32_t *)(ws + b.src);
            r.Bp = (uint32_t *)(ws + b.dst);
            r.total = ((int64_t)b.np << b.lk) << b.lb;
            r.per_item = 4096;
            r.lk = b.lk; r.ln = b.ln; r.np = b.np; r.rank = b.rank;
            r.g = g;
            Bd.add(chain, Q_BPREP_GATHER, 0, cdiv(r.total, r.per_item), Bd.rec(r));
            return TN_OK;
        }
        case OP_GEMM: {
            const GemmOp &g = op.gemm;
            const int64_t batch = (int64_t)1 << g.lb;
            const int64_t sa = g.bcast_a ? 0 : (int64_t)1 << (g.lm + g.lk),
                          sb = g.bcast_b ? 0 : (int64_t)1 << (g.lk + g.ln), sc = (int64_t)1 << (g.lm + g.ln);
            const int32_t *za = g.idx_a >= 0 ? P->d_gidx + g.idx_a : nullptr;
            const int32_t *zb = g.idx_b >= 0 ? P->d_gidx + g.idx_b : nullptr;
            ScaleRef sr{};
            sr.tmax = P->d_tmax;
            sr.texp = P->d_texp;
            sr.meta_a = g.meta_a;
            sr.meta_b = g.meta_b;
            sr.meta_c = g.meta_c;
            sr.out_max = P->d_tmax + g.meta_c;
            sr.headroom = g.headroom;
            sr.err = P->d_err;
            sr.scale_off = P->opts.no_scaling ? 1 : 0;
            if (g.kernel == GK_C64_ROWS || g.kernel == GK_LP_ROWS) {
                QRows r{};
                r.A = ws + g.a;
                r.B = ws + g.b;
                r.C = ws + g.c;
                r.za = za;
                r.zb = zb;
                r.sa = sa; r.sb = sb; r.sc = sc;
                r.lm = g.lm; r.ln = g.ln; r.lk = g.lk;
                const int N = 1 << g.ln;
                const int nc = N >= 16 ? 16 : N;
                int ncl = 0;
                while ((1 << ncl) < nc) ++ncl;
                r.gx = cdiv((int64_t)1 << g.lm, kRows);
                r.gx2 = cdiv(r.gx, 2);
                r.gy = (int)cdiv(N, nc);
                int sub;
                if (g.kernel == GK_C64_ROWS || dtype == TN_C64) {
                    r.sr = ScaleRef{};
                    sub = 0;
                } else {
                    r.sr = sr;
                    const int code = g.ta * 4 + g.tb * 2 + g.tc;
                    if (code == 2 || code == 3) return record_error(TN_EUNSUPPORTED, "queue: operand storage");
                    sub = (dtype == TN_F16 ? 1 : 2) | (g.ta << 2) | (g.tb << 3) | (g.tc << 4);
                }
                sub |= ncl << 5;
                Bd.add(chain, Q_ROWS, sub, r.gx2 * r.gy * batch, Bd.rec(r));
                return TN_OK;
            }
            if (g.kernel == GK_C64_TILED) {
                if (g.lm < 6 || g.ln < 6 || g.lk < 4) return record_error(TN_EINVAL, "queue: tiled c64 shape");
                QTiled r{};
                r.A = (const float2 *)(ws + g.a);
                r.B = (const float2 *)(ws + g.b);
                r.C = (float2 *)(ws + g.c);
                r.za = za;
                r.zb = zb;
                r.sa = sa; r.sb = sb; r.sc = sc;
                r.lm = g.lm; r.ln = g.ln; r.lk = g.lk;
                r.gx = ((int64_t)1 << g.lm) / 64;
                r.gy = (1 << g.ln) / 64;
                Bd.add(chain, Q_TILED_C64, g.lk > 12 ? 1 : 0, r.gx * r.gy * batch, Bd.rec(r));
                return TN_OK;
            }
            // tensor cores (1-CTA tiles)
            if (g.fp8) return record_error(TN_EUNSUPPORTED, "queue: FP8 steps are not queued");
            if (g.kernel == GK_C64_TC)
                return record_error(TN_EUNSUPPORTED, "queue: complex64 tensor-core steps are not queued");
            TcGemmDesc d;
            d.dtype = dtype;
            d.A = ws + g.a;
            d.Bp = ws + g.b;
            d.C = ws + g.c;
            d.lm = g.lm; d.ln = g.ln; d.lk = g.lk;
            d.batch = batch;
            d.batch_a = g.lb > 0 && !g.bcast_a;
            d.batch_b = g.lb > 0 && !g.bcast_b;
            d.za = za;
            d.zb = zb;
            if (za) d.depth_a = (int64_t)1 << g.gather_a_log2;
            if (zb) d.depth_b = (int64_t)1 << g.gather_b_log2;
            d.np = std::max(16, 2 << g.ln);
            d.bn = tc_tile_bn(g.tile);
            d.gm = tc_tile_gm(g.tile);
            d.pair = 0;
            d.half_k = (g.tile & kTcHalfKTile) ? 1 : 0;
            d.out_c64 = g.tc == 0;
            d.partial = P->d_splitk;
            d.out_rank = g.out_rank;
            for (int i = 0; i < g.out_rank && i < 40; ++i) d.out_dpos[i] = g.out_dpos[i];
            QTc r;
            std::memset(&r, 0, sizeof(r));
            int bn = 0, bk = 0;
            bool pair = false;
            if (!tc_gemm_supported(d.lk, d.ln) ||
                tc_setup(d, sr, P->d_err, true, &r.ma, &r.mb, &r.a, &bn, &bk, &pair) != cudaSuccess || pair)
                return record_error(TN_EUNSUPPORTED, "queue: tensor-core step shape");
            r.bn = bn;
            r.bkb = 2 * bk;
            if (r.bkb != 32 && r.bkb != 64 && r.bkb != 128) return record_error(TN_EUNSUPPORTED, "queue: K chunk");
            Bd.add(chain, Q_TC, 0, std::min<int64_t>(r.a.tiles, walkers), Bd.rec(r));
            if (r.a.split > 1) {
                QSplitK s{};
                s.partial = reinterpret_cast<const float2 *>(r.a.partial);
                s.C = d.C;
                s.n = batch << (g.lm + g.ln);
                s.per_item = 8192;
                s.split = r.a.split;
                s.lk = g.lk;
                s.sr = sr;
                Bd.add(chain, Q_SPLITK, dtype | (d.out_c64 ? 16 : 0), cdiv(s.n, s.per_item), Bd.rec(s));
            }
            return TN_OK;
        }
        case OP_SUM: {
            if (op.sum.n_split < 0 || op.sum.n_split > 8 || op.sum.n_split > P->net.n_open)
                return record_error(TN_EINVAL, "queue: split outputs");
            uint64_t split_val = 0, split_mask = 0;
            for (int i = 0; i < op.sum.n_split; ++i) {
                split_mask |= 1ull << op.sum.split_t[i];
                if ((slice_base >> op.sum.split_bit[i]) & 1) split_val |= 1ull << op.sum.split_t[i];
            }
            QSum r{};
            r.F = ws + op.sum.src;
            r.amps = amps;
            r.texp = dtype == TN_C64 ? nullptr : P->d_texp;
            r.stepcorr = dtype == TN_C64 ? nullptr : P->d_stepcorr;
            r.n_steps = dtype == TN_C64 ? 0 : (int)P->sched.steps.size();
            r.split_mask = split_mask;
            r.split_val = split_val;
            r.n_open = P->net.n_open;
            r.t_lo = t_lo;
            r.t_hi = t_hi;
            r.overwrite = overwrite;
            r.op = op.sum;
            const int64_t n = (int64_t)1 << (P->net.n_open - op.sum.n_split);
            Bd.add(chain, Q_SUM, dtype | (op.sum.tf << 4), cdiv(n, kQSimt), Bd.rec(r));
            return TN_OK;
        }
        case OP_QUANT: return record_error(TN_EUNSUPPORTED, "queue: FP8 steps are not queued");
        default: return record_error(TN_EINVAL, "queue: unknown op");
    }
}

// The ops of one tn_contract(P, begin, count, amps, accumulate) call, in the
// order enqueue_contract issues them, as one chain.
int emit_plan(Builder &Bd, int chain, tn_plan_s *P, int64_t slice_begin, int64_t slice_count, double *d_amps,
              int accumulate, int walkers) {
    const Schedule &S = P->sched;
    const bool lp = P->opts.dtype != TN_C64;
    const int64_t n_amps = (int64_t)1 << P->net.n_open;
    if (slice_count == 0) {
        if (!accumulate) Bd.zero(chain, d_amps, n_amps * 4);
        return TN_OK;
    }
    Bd.zero(chain, P->d_err, 1);
    if (lp) {
        Bd.zero(chain, P->d_tmax, S.n_meta);
        Bd.zero(chain, P->d_texp, S.n_meta);
    }
    int rc;
    for (const Op &op : S.ops)
        if (op.phase == 0) {
            rc = emit_op(Bd, chain, P, op, 0, nullptr, 0, 0, 0, walkers);
            if (rc != TN_OK) return rc;
        }
    const int64_t bsize = (int64_t)1 << P->batch_log2;
    const int64_t first = slice_begin / bsize * bsize;
    const int64_t last = (slice_begin + slice_count - 1) / bsize * bsize;
    const bool parts = P->n_recompute > 0;
    if (parts && !accumulate) Bd.zero(chain, d_amps, n_amps * 4);
    for (int64_t base = first; base <= last; base += bsize) {
        if (lp && S.n_meta > S.n_meta_inv) Bd.zero(chain, P->d_tmax + S.n_meta_inv, S.n_meta - S.n_meta_inv);
        const int t_lo = (int)std::max<int64_t>(0, slice_begin - base);
        const int t_hi = (int)std::min<int64_t>(bsize, slice_begin + slice_count - base);
        const int overwrite = (!accumulate && !parts && base == first) ? 1 : 0;
        for (const Op &op : S.ops)
            if (op.phase == 1) {
                rc = emit_op(Bd, chain, P, op, base, (double2 *)d_amps, t_lo, t_hi, overwrite, walkers);
                if (rc != TN_OK) return rc;
            }
    }
    return TN_OK;
}

int g_queue_sms = 0;

cudaError_t queue_prepare() {
    static int done_mask = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 31 && ((done_mask >> dev) & 1)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(queue_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kQSmem);
    if (e != cudaSuccess) return e;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, queue_kernel, kQThreads, kQSmem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return cudaErrorInvalidConfiguration;
    }
    g_queue_sms = tc_num_sms() * std::min(n, 1);
    if (dev < 31) done_mask |= 1 << dev;
    return cudaSuccess;
}

}  // namespace
}  // namespace tn

using namespace tn;

struct tn_queue_s {
    int device = -1;
    std::vector<tn_plan_s *> plans;
    void *d_mem = nullptr;      // ops | blob | run state | its initial copy
    QOp *d_ops = nullptr;
    uint8_t *d_blob = nullptr;
    // run state: done[n_ops] | list[n_items] | QState, reset from d_init
    // before every run
    char *d_run = nullptr, *d_init = nullptr;
    int32_t *d_done = nullptr;
    long long *d_list = nullptr;
    QState *d_state = nullptr;
    int32_t n_ops = 0, n_items = 0, max_chain = 0, grid = 0;
    size_t run_bytes = 0;
    int64_t blob_bytes = 0;
    int32_t n_heads = 0;
    double flops = 0;
    int64_t slices = 0;
    uint64_t idle_limit_ns = 10000000000ull;
    int profile = 0;
};

namespace {

int qfail(int code, const std::string &msg) { return record_error(code, msg); }

// heads: the chains whose first op is listed at launch (all, normally).
int queue_finish(tn_queue_s *Q, Builder &Bd, const std::vector<int> *heads = nullptr) {
    // successors along each chain; the chains' first ops listed longest
    // chain first (the longest chains bound the run)
    std::vector<int> order(Bd.chains.size());
    for (size_t c = 0; c < order.size(); ++c) order[c] = (int)c;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return Bd.chains[a].size() > Bd.chains[b].size(); });
    size_t maxd = 0;
    for (auto &ch : Bd.chains) maxd = std::max(maxd, ch.size());
    for (auto &ch : Bd.chains)
        for (size_t d = 0; d + 1 < ch.size(); ++d) Bd.ops[ch[d]].next = ch[d + 1];
    const int n_ops = (int)Bd.ops.size();
    int64_t n_items = 0;
    for (const QOp &o : Bd.ops) n_items += o.ntiles;
    if (n_items > 0x7fffffff) return qfail(TN_EUNSUPPORTED, "queue: too many items");
    // the list: every tile of the listed first ops, the rest empty (-1)
    std::vector<long long> list((size_t)std::max<int64_t>(1, n_items), -1ll);
    int64_t n_listed = 0;
    int n_heads = 0;
    auto list_op = [&](int op) {
        for (int t = 0; t < Bd.ops[op].ntiles; ++t) list[n_listed++] = ((long long)op << 32) | t;
        ++n_heads;
    };
    if (heads) {
        for (int op : *heads) list_op(op);
    } else {
        for (int c : order)
            if (!Bd.chains[c].empty()) list_op(Bd.chains[c][0]);
    }
    Q->n_ops = n_ops;
    Q->n_items = (int32_t)n_items;
    Q->n_heads = n_heads;
    Q->max_chain = (int32_t)maxd;
    Q->grid = (int)std::max<int64_t>(1, std::min<int64_t>(g_queue_sms, n_items));
    const size_t ops_b = ((size_t)std::max(1, n_ops) * sizeof(QOp) + 255) / 256 * 256;
    const size_t blob_b = (Bd.blob.size() + 255) / 256 * 256;
    const size_t done_b = ((size_t)std::max(1, n_ops) * 4 + 255) / 256 * 256;
    const size_t list_b = (list.size() * 8 + 255) / 256 * 256;
    const size_t state_b = (sizeof(QState) + 255) / 256 * 256;
    Q->run_bytes = done_b + list_b + state_b;
    const size_t total = ops_b + blob_b + 2 * Q->run_bytes;
    cudaError_t e = cudaMalloc(&Q->d_mem, total);
    if (e != cudaSuccess) return qfail(TN_ENOMEM, std::string("queue tables: ") + cudaGetErrorString(e));
    char *m = (char *)Q->d_mem;
    Q->d_ops = (QOp *)m;
    Q->d_blob = (uint8_t *)(m + ops_b);
    Q->d_run = m + ops_b + blob_b;
    Q->d_init = Q->d_run + Q->run_bytes;
    Q->d_done = (int32_t *)Q->d_run;
    Q->d_list = (long long *)(Q->d_run + done_b);
    Q->d_state = (QState *)(Q->d_run + done_b + list_b);
    Q->blob_bytes = (int64_t)Bd.blob.size();
    std::vector<char> init(Q->run_bytes, 0);
    std::memcpy(init.data() + done_b, list.data(), list.size() * 8);
    QState s0{};
    s0.head = 0;
    s0.tail = (int32_t)n_listed;
    std::memcpy(init.data() + done_b + list_b, &s0, sizeof(s0));
    e = cudaMemcpy(Q->d_ops, Bd.ops.data(), (size_t)n_ops * sizeof(QOp), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !Bd.blob.empty())
        e = cudaMemcpy(Q->d_blob, Bd.blob.data(), Bd.blob.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(Q->d_init, init.data(), Q->run_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return qfail(TN_ECUDA, std::string("queue upload: ") + cudaGetErrorString(e));
    return TN_OK;
}

}  // namespace

extern "C" {

int tn_queue_create(tn_plan_t *const *plans, int32_t n, const int64_t *slice_begin, const int64_t *slice_count,
                    double *const *d_amps, tn_queue_t **out) {
    if (!out || n < 1 || !plans || !d_amps) return qfail(TN_EINVAL, "bad queue arguments");
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!plans[i] || !d_amps[i]) return qfail(TN_EINVAL, "plans and outputs must be non-NULL");
    cudaError_t e = tc_prepare();
    if (e == cudaSuccess) e = queue_prepare();
    if (e != cudaSuccess) return qfail(TN_ECUDA, std::string("queue kernel set-up: ") + cudaGetErrorString(e));
    int dev = 0;
    cudaGetDevice(&dev);
    Builder Bd;
    Bd.chains.resize(n);
    tn_queue_s *Q = new tn_queue_s();
    Q->device = dev;
    for (int i = 0; i < n; ++i) {
        tn_plan_s *P = plans[i];
        if (P->prof_mask) { delete Q; return qfail(TN_EINVAL, "profiling must be off for a queue"); }
        int rc = prepare_for_contract(P, nullptr);
        if (rc == TN_OK) {
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) rc = qfail(TN_ECUDA, std::string("plan set-up: ") + cudaGetErrorString(e));
        }
        if (rc != TN_OK) { delete Q; return rc; }
        const int64_t ns = (int64_t)1 << P->sliced.size();
        const int64_t b0 = slice_begin ? slice_begin[i] : 0;
        const int64_t cnt = slice_count ? slice_count[i] : ns;
        if (b0 < 0 || cnt < 0 || b0 + cnt > ns) { delete Q; return qfail(TN_EINVAL, "slice range outside [0, n_slices)"); }
        rc = emit_plan(Bd, i, P, b0, cnt, d_amps[i], 0, g_queue_sms);
        if (rc != TN_OK) { delete Q; return rc; }
        if (cnt > 0) {
            const int64_t bsize = (int64_t)1 << P->batch_log2;
            const int64_t passes = (b0 + cnt - 1) / bsize - b0 / bsize + 1;
            Q->flops += P->sched.flops_inv + P->sched.flops_per_pass * (double)passes;
        }
        Q->slices += cnt;
        Q->plans.push_back(P);
    }
    const int rc = queue_finish(Q, Bd);
    if (rc != TN_OK) {
        if (Q->d_mem) cudaFree(Q->d_mem);
        delete Q;
        return rc;
    }
    *out = Q;
    return TN_OK;
}

int tn_queue_run(tn_queue_t *Q, void *stream, tn_contract_report *rep) {
    if (!Q || !Q->d_mem) return qfail(TN_EINVAL, "NULL queue");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != Q->device) return qfail(TN_EINVAL, "queue was created on another device");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (rep) {
        if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess)
            return qfail(TN_ECUDA, "event");
        cudaEventRecord(ev0, s);
    }
    cudaError_t e = cudaMemcpyAsync(Q->d_run, Q->d_init, Q->run_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        queue_kernel<<<Q->grid, kQThreads, kQSmem, s>>>(Q->d_ops, Q->n_items, Q->d_blob, Q->d_done, Q->d_list,
                                                       Q->d_state, Q->idle_limit_ns, Q->profile);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return qfail(TN_ECUDA, std::string("queue launch: ") + cudaGetErrorString(e));
    if (rep) {
        cudaEventRecord(ev1, s);
        e = cudaEventSynchronize(ev1);
        float ms = 0;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        if (e != cudaSuccess) return qfail(TN_ECUDA, std::string("queue run: ") + cudaGetErrorString(e));
        std::memset(rep, 0, sizeof(*rep));
        rep->ms = ms;
        rep->flops = Q->flops;
        rep->slices = Q->slices;
        rep->kernels = 1;
        QState h{};
        e = cudaMemcpy(&h, Q->d_state, sizeof(h), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return qfail(TN_ECUDA, "read queue state");
        if (h.err & 1)
            return qfail(TN_ETIMEOUT, "a bounded device wait of the work queue gave up (list entry " +
                                          std::to_string(h.idle_at) + " was never written)");
        for (tn_plan_s *P : Q->plans) {
            int32_t herr = 0;
            e = cudaMemcpy(&herr, P->d_err, 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return qfail(TN_ECUDA, "read error flag");
            if (herr & 1) return qfail(TN_ETIMEOUT, "a bounded device wait gave up");
            if (herr & 2) return qfail(TN_EUNSUPPORTED, "a complex-half value overflowed its power-of-two scale");
        }
    }
    return TN_OK;
}

int tn_queue_info(const tn_queue_t *Q, tn_queue_stats *out) {
    if (!Q || !out) return qfail(TN_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->n_plans = (int32_t)Q->plans.size();
    out->n_ops = Q->n_ops;
    out->n_items = Q->n_items;
    out->max_chain = Q->max_chain;
    out->ctas = Q->grid;
    out->table_bytes = Q->blob_bytes;
    out->flops = Q->flops;
    out->slices = Q->slices;
    return TN_OK;
}

int tn_queue_set_wait_limit(tn_queue_t *Q, int64_t limit_us) {
    if (!Q || limit_us < 1) return qfail(TN_EINVAL, "bad wait limit");
    Q->idle_limit_ns = (uint64_t)limit_us * 1000ull;
    return TN_OK;
}

int tn_queue_profile(tn_queue_t *Q, int enable) {
    if (!Q) return qfail(TN_EINVAL, "NULL queue");
    Q->profile = enable ? 1 : 0;
    return TN_OK;
}

int tn_queue_profile_read(const tn_queue_t *Q, tn_queue_kind_stats *out, int32_t capacity) {
    if (!Q || !out || capacity < 1) return qfail(TN_EINVAL, "bad argument");
    QState h{};
    const cudaError_t e = cudaMemcpy(&h, Q->d_state, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return qfail(TN_ECUDA, std::string("read queue state: ") + cudaGetErrorString(e));
    for (int k = 0; k < capacity; ++k) {
        out[k].items = k < kQKinds ? (int64_t)h.items[k] : 0;
        out[k].wait_ms = k < kQKinds ? (double)h.wait_ns[k] * 1e-6 : 0.0;
        out[k].busy_ms = k < kQKinds ? (double)h.busy_ns[k] * 1e-6 : 0.0;
    }
    return TN_OK;
}

void tn_queue_destroy(tn_queue_t *Q) {
    if (!Q) return;
    if (Q->d_mem) cudaFree(Q->d_mem);
    delete Q;
}

// A queue with an op that nothing ever lists: the wait of the CTA holding its
// list entry
// runs out after limit_ms and the call returns TN_ETIMEOUT with the context
// intact.
int tn_selftest_queue_timeout(int32_t limit_ms, void *stream) {
    if (limit_ms < 1 || limit_ms > 10000) return qfail(TN_EINVAL, "limit_ms must be in 1..10000");
    cudaError_t e = queue_prepare();
    if (e != cudaSuccess) return qfail(TN_ECUDA, std::string("queue kernel set-up: ") + cudaGetErrorString(e));
    int dev = 0;
    cudaGetDevice(&dev);
    void *scratch = nullptr;
    e = cudaMalloc(&scratch, 4096);
    if (e != cudaSuccess) return qfail(TN_ENOMEM, "self-test buffer");
    // two one-op chains, only the first of which is listed: after it runs,
    // the second is never listed by anything ("a flag nothing sets"), so the
    // wait for that list entry runs out
    Builder Bd;
    Bd.chains.resize(2);
    Bd.zero(0, scratch, 16);
    Bd.zero(1, (char *)scratch + 64, 16);
    tn_queue_s *Q = new tn_queue_s();
    Q->device = dev;
    const std::vector<int> heads = {0};
    int rc = queue_finish(Q, Bd, &heads);
    if (rc == TN_OK) {
        Q->idle_limit_ns = (uint64_t)limit_ms * 1000000ull;
        tn_contract_report rep;
        rc = tn_queue_run(Q, stream, &rep);
    }
    if (Q->d_mem) cudaFree(Q->d_mem);
    delete Q;
    cudaFree(scratch);
    return rc;
}

}  // extern "C"

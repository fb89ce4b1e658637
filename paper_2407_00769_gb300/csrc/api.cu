// C ABI of the contraction library (declared in include/tn.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "kernels.cuh"
#include "plan.h"

using namespace tn;

namespace {

thread_local std::string g_err;

// complex64 step that the tensor cores can run (tn_plan_opts.c64_tensor_cores)
// (one K part only: split-K steps, K > 2^15 or cut for few tiles, stay on
// the CUDA cores)
bool x3_eligible(const tn_plan_s *P, const GemmOp &g) {
    return P->opts.dtype == TN_C64 && P->opts.c64_tensor_cores && tc_gemm_supported(g.lk, g.ln) &&
           g.idx_a < 0 && g.idx_b < 0 && g.out_rank == 0 && g.lm <= 30 && g.lk <= kSplitLog2KHost &&
           tc_split(g.lm, g.ln, g.lk, (int64_t)1 << g.lb) == 1;
}

// scratch of such a step: hi and lo parts of A ([batch][M][2K] FP32) and of
// B' ([batch][np][2K] FP32)
int64_t x3_bytes(const GemmOp &g) {
    const int64_t ba = (g.lb > 0 && !g.bcast_a) ? (int64_t)1 << g.lb : 1;
    const int64_t bb = (g.lb > 0 && !g.bcast_b) ? (int64_t)1 << g.lb : 1;
    const int64_t np = std::max(16, 2 << g.ln);
    return 2 * (ba << (g.lm + g.lk)) * 8 + 2 * ((bb * np) << g.lk) * 8;
}


int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(TN_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define TN_CUDA(call, where)                         \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

void *plan_dev_alloc(tn_plan_s *P, size_t bytes) {
    void *p = nullptr;
    if (P->opts.dev_alloc) p = P->opts.dev_alloc(bytes, P->opts.alloc_ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) P->owned.push_back(p);
    return p;
}

void plan_dev_free_all(tn_plan_s *P) {
    for (void *p : P->owned) {
        if (P->opts.dev_free) P->opts.dev_free(p, P->opts.alloc_ctx);
        else cudaFree(p);
    }
    P->owned.clear();
}

int ensure_device(tn_plan_s *P) {
    int dev = 0;
    TN_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (P->dev_ready) {
        if (dev != P->device) return fail(TN_EINVAL, "plan was set up on another device");
        return TN_OK;
    }
    P->device = dev;
    const Schedule &S = P->sched;
    P->d_ws = (char *)plan_dev_alloc(P, (size_t)S.ws_bytes);
    P->d_store = (double2 *)plan_dev_alloc(P, std::max<size_t>(16, P->leaf_store.size() * 16));
    P->d_jobs = (LeafJob *)plan_dev_alloc(P, std::max<size_t>(64, S.leaf_jobs.size() * sizeof(LeafJob)));
    P->d_tmax = (float *)plan_dev_alloc(P, std::max<size_t>(64, (size_t)(S.n_meta + S.n_meta_extra) * 4));
    P->d_texp = (int32_t *)plan_dev_alloc(P, std::max<size_t>(64, (size_t)(S.n_meta + S.n_meta_extra) * 4));
    P->d_err = (int32_t *)plan_dev_alloc(P, 64);
    P->d_stepcorr = (double2 *)plan_dev_alloc(P, std::max<size_t>(64, S.steps.size() * sizeof(double2)));
    size_t split_bytes = 64;
    int64_t x3b = 0;
    for (const Op &op : S.ops)
        if (op.kind == OP_GEMM && (op.gemm.kernel == GK_LP_TC || x3_eligible(P, op.gemm))) {
            split_bytes = std::max(split_bytes, tc_split_bytes(op.gemm.lm, op.gemm.ln, op.gemm.lk,
                                                               (int64_t)1 << op.gemm.lb));
            if (op.gemm.kernel != GK_LP_TC) x3b = std::max(x3b, x3_bytes(op.gemm));
        }
    P->d_splitk = (float *)plan_dev_alloc(P, split_bytes);
    P->d_gidx = (int32_t *)plan_dev_alloc(P, std::max<size_t>(64, S.gidx.size() * 4));
    P->d_bpart = plan_dev_alloc(P, bprep_c64_scratch_bytes());
    if (x3b > 0) {
        P->d_x3 = (float *)plan_dev_alloc(P, (size_t)x3b);
        if (!P->d_x3) {
            plan_dev_free_all(P);
            return fail(TN_ENOMEM, "device allocation of the complex64 tensor-core scratch (" + std::to_string(x3b) +
                                       " bytes) failed");
        }
    }
    if (!P->d_ws || !P->d_store || !P->d_jobs || !P->d_tmax || !P->d_texp || !P->d_err || !P->d_stepcorr ||
        !P->d_splitk || !P->d_gidx || !P->d_bpart) {
        plan_dev_free_all(P);
        return fail(TN_ENOMEM, "device allocation of the plan workspace (" +
                                   std::to_string(S.ws_bytes) + " bytes) failed");
    }
    const size_t store_bytes = P->leaf_store.size() * 16;
    if (cudaMallocHost(&P->h_store_pinned, std::max<size_t>(16, store_bytes)) != cudaSuccess) {
        plan_dev_free_all(P);
        return fail(TN_ENOMEM, "pinned host allocation failed");
    }
    std::memcpy(P->h_store_pinned, P->leaf_store.data(), store_bytes);
    TN_CUDA(cudaMemcpy(P->d_store, P->h_store_pinned, store_bytes, cudaMemcpyHostToDevice), "upload leaves");
    if (!S.leaf_jobs.empty())
        TN_CUDA(cudaMemcpy(P->d_jobs, S.leaf_jobs.data(), S.leaf_jobs.size() * sizeof(LeafJob),
                           cudaMemcpyHostToDevice),
                "upload leaf jobs");
    if (!S.gidx.empty())
        TN_CUDA(cudaMemcpy(P->d_gidx, S.gidx.data(), S.gidx.size() * 4, cudaMemcpyHostToDevice),
                "upload gather indices");
    {
        // per-step rounding compensation: 1 until a step measures its own
        std::vector<double2> ones(std::max<size_t>(1, S.steps.size()), make_double2(1.0, 0.0));
        TN_CUDA(cudaMemcpy(P->d_stepcorr, ones.data(), ones.size() * sizeof(double2), cudaMemcpyHostToDevice),
                "init step corrections");
    }
    TN_CUDA(tc_prepare(), "tensor-core kernel attributes");
    tc_num_sms();
    P->dev_ready = true;
    return TN_OK;
}

// kernel class and algorithmic flops / bytes of one op
int op_class(const tn_plan_s *P, const Op &op, double &flops, double &bytes) {
    const int dtype = P->opts.dtype;
    const double esz = dtype == TN_C64 ? 8 : 4;
    flops = 0;
    bytes = 0;
    switch (op.kind) {
        case OP_LEAF: {
            for (int k = 0; k < op.leaf_count; ++k) {
                const LeafJob &j = P->sched.leaf_jobs[op.leaf_first + k];
                bytes += std::ldexp(16.0, j.rank_out) + std::ldexp(esz, j.rank_out);
            }
            return TN_KC_LEAF;
        }
        case OP_PERM: bytes = 2 * std::ldexp((double)op.perm.esz, op.perm.rank); return TN_KC_PERMUTE;
        case OP_BPREP: {
            const double b = std::ldexp(1.0, op.bprep.lb);
            bytes = b * (std::ldexp(esz, op.bprep.lk + op.bprep.ln) + (double)op.bprep.np * std::ldexp(4.0, op.bprep.lk));
            return TN_KC_BPREP;
        }
        case OP_GEMM: {
            const GemmOp &g = op.gemm;
            flops = 8.0 * std::ldexp(1.0, g.lm + g.ln + g.lk + g.lb);
            const double ea = dtype == TN_C64 ? 8 : g.fp8 ? 2 : (g.ta ? 4 : 8),
                         eb = dtype == TN_C64 ? 8 : (g.tb ? 4 : 8), ec = dtype == TN_C64 ? 8 : (g.tc ? 4 : 8);
            const double bsz = g.kernel == GK_LP_TC
                                   ? std::max(16.0, std::ldexp(2.0, g.ln)) * std::ldexp(g.fp8 ? 2.0 : 4.0, g.lk)
                                   : std::ldexp(eb, g.lk + g.ln);
            bytes = std::ldexp(1.0, g.lb) * (std::ldexp(ea, g.lm + g.lk) + bsz + std::ldexp(ec, g.lm + g.ln));
            if (g.kernel == GK_LP_TC) return TN_KC_GEMM_TC;
            if (g.kernel == GK_LP_ROWS) return TN_KC_GEMM_LP;
            return TN_KC_GEMM_C64;
        }
        case OP_SUM: bytes = std::ldexp(esz, op.sum.rank); return TN_KC_SUM;
        case OP_QUANT: bytes = 6.0 * (double)op.quant.n_pairs; return TN_KC_QUANT;
    }
    return -1;
}

cudaEvent_t take_event(tn_plan_s *P) {
    if (!P->ev_pool.empty()) {
        cudaEvent_t e = P->ev_pool.back();
        P->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int run_op_raw(tn_plan_s *P, const Op &op, int64_t slice_base, double2 *amps, int t_lo, int t_hi,
               int overwrite, cudaStream_t s, int &launches);

int run_op(tn_plan_s *P, const Op &op, int64_t slice_base, double2 *amps, int t_lo, int t_hi,
           int overwrite, cudaStream_t s, int &launches) {
    if (!P->prof_mask) return run_op_raw(P, op, slice_base, amps, t_lo, t_hi, overwrite, s, launches);
    double fl, by;
    const int cls = op_class(P, op, fl, by);
    if (cls < 0 || !((P->prof_mask >> cls) & 1))
        return run_op_raw(P, op, slice_base, amps, t_lo, t_hi, overwrite, s, launches);
    tn_plan_s::ProfRec r{cls, take_event(P), take_event(P), fl, by, 0};
    cudaEventRecord(r.e0, s);
    const int before = launches;
    const int rc = run_op_raw(P, op, slice_base, amps, t_lo, t_hi, overwrite, s, launches);
    r.kernels = launches - before;
    cudaEventRecord(r.e1, s);
    P->prof.push_back(r);
    return rc;
}

int run_op_raw(tn_plan_s *P, const Op &op, int64_t slice_base, double2 *amps, int t_lo, int t_hi,
               int overwrite, cudaStream_t s, int &launches) {
    const int dtype = P->opts.dtype;
    const int esz = dtype == TN_C64 ? 8 : 4;
    char *ws = P->d_ws;
    cudaError_t e = cudaSuccess;
    switch (op.kind) {
        case OP_LEAF:
            e = launch_leaf_prep(P->d_jobs + op.leaf_first, op.leaf_count, P->d_store, ws, dtype,
                                 slice_base, P->d_tmax, P->d_texp, s);
            ++launches;
            break;
        case OP_PERM: {
            const PermParams pp = make_perm_params(op.perm.rank, op.perm.perm);
            e = launch_permute(ws + op.perm.src, ws + op.perm.dst, pp, op.perm.esz, s);
            ++launches;
            break;
        }
        case OP_BPREP:
            e = launch_bprep_perm(ws + op.bprep.src, ws + op.bprep.dst, op.bprep.rank, op.bprep.perm,
                                  op.bprep.lk, op.bprep.ln, op.bprep.lb, op.bprep.np, op.bprep.tb, dtype,
                                  P->d_stepcorr + op.bprep.step, P->d_tmax, P->d_texp, op.bprep.meta_src,
                                  op.bprep.meta_dst, s, P->opts.no_scaling ? 1 : 0, P->d_bpart);
            launches += (op.bprep.tb == 0 && P->d_bpart) ? 2 : 1;   // complex64 B: partial sums, then the tree
            break;
        case OP_GEMM: {
            const GemmOp &g = op.gemm;
            const int64_t batch = (int64_t)1 << g.lb;
            const int64_t sa = g.bcast_a ? 0 : (int64_t)1 << (g.lm + g.lk),
                          sb = g.bcast_b ? 0 : (int64_t)1 << (g.lk + g.ln), sc = (int64_t)1 << (g.lm + g.ln);
            // sparse-state gathers: the operand chunk of each batch entry
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
            switch (g.kernel) {
                case GK_C64_ROWS:
                    e = launch_gemm_rows_c64((const float2 *)(ws + g.a), (const float2 *)(ws + g.b),
                                             (float2 *)(ws + g.c), g.lm, g.ln, g.lk, batch, sa, sb, sc, s, za,
                                             zb);
                    break;
                case GK_C64_TILED:
                    e = launch_gemm_tiled_c64((const float2 *)(ws + g.a), (const float2 *)(ws + g.b),
                                              (float2 *)(ws + g.c), g.lm, g.ln, g.lk, batch, sa, sb,
                                              sc, g.tile, s, za, zb);
                    break;
                case GK_LP_ROWS:
                    e = launch_gemm_rows_mixed(dtype, g.ta, g.tb, g.tc, ws + g.a, ws + g.b, ws + g.c, g.lm,
                                               g.ln, g.lk, batch, sa, sb, sc, sr, s, za, zb);
                    break;
                case GK_C64_TC: {
                    // TF32 parts of A and of B' (from B [batch][K][N]), then
                    // three kind::tf32 MMAs per K slice
                    if (!P->d_x3 || !x3_eligible(P, g)) return fail(TN_EINVAL, "complex64 tensor-core step not set up");
                    const int np = std::max(16, 2 << g.ln);
                    const int64_t ba = g.bcast_a ? 1 : batch, bb = g.bcast_b ? 1 : batch;
                    const int64_t na = (ba << (g.lm + g.lk)) * 2, nb = ((bb * np) << g.lk) * 2;   // FP32 values
                    float *ah = P->d_x3, *al = ah + na, *bh = al + na, *bl = bh + nb;
                    e = launch_split_tf32(ws + g.a, ah, al, na, s);
                    if (e == cudaSuccess) e = launch_bprep_x3(ws + g.b, bh, bl, g.lk, g.ln, bb, np, s);
                    launches += 2;
                    if (e != cudaSuccess) break;
                    TcGemmDesc d;
                    d.dtype = TN_C64;
                    d.A = ah; d.A2 = al;
                    d.Bp = bh; d.Bp2 = bl;
                    d.C = ws + g.c;
                    d.lm = g.lm; d.ln = g.ln; d.lk = g.lk;
                    d.batch = batch;
                    d.batch_a = g.lb > 0 && !g.bcast_a;
                    d.batch_b = g.lb > 0 && !g.bcast_b;
                    d.np = np;
                    d.bn = tc_tile_bn(g.tile);
                    d.gm = tc_tile_gm(g.tile);
                    d.x3 = 1;
                    d.out_c64 = 1;
                    d.partial = P->d_splitk;
                    e = launch_gemm_tc(d, ScaleRef{}, P->d_err, s);
                    if (tc_split(g.lm, g.ln, g.lk, batch) > 1) ++launches;
                    break;
                }
                case GK_LP_TC: {
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
                    d.pair = (g.tile & kTcPairTile) ? 1 : 0;
                    d.half_k = (g.tile & kTcHalfKTile) ? 1 : 0;
                    d.bres = (g.tile & kTcBresTile) ? 1 : 0;
                    d.tma_store = (g.tile & kTcStoreTile) ? 1 : 0;
                    d.staged = (g.tile & kTcStagedTile) ? 1 : 0;
                    d.out_c64 = g.tc == 0;
                    d.partial = P->d_splitk;
                    d.fp8 = g.fp8;
                    d.out_rank = g.out_rank;
                    for (int i = 0; i < g.out_rank && i < 40; ++i) d.out_dpos[i] = g.out_dpos[i];
                    e = launch_gemm_tc(d, sr, P->d_err, s);
                    // split K: the parts' FP64 sum is a second kernel
                    if (!(za || zb) && g.out_rank == 0 && tc_split(g.lm, g.ln, g.lk, batch) > 1) ++launches;
                    break;
                }
                default:
                    return fail(TN_EINVAL, "unknown kernel");
            }
            ++launches;
            break;
        }
        case OP_QUANT:
            // the destination's max is an atomic max over the quantized values
            e = cudaMemsetAsync(P->d_tmax + op.quant.meta_dst, 0, 4, s);
            if (e == cudaSuccess)
                e = launch_quant_e4m3(ws + op.quant.src, ws + op.quant.dst, op.quant.n_pairs, dtype, P->d_tmax,
                                  P->d_texp, op.quant.meta_src, op.quant.meta_dst, s);
            ++launches;
            break;
        case OP_SUM: {
            // recomputation: this pass fills the part of the output its
            // split legs' values (slice-id bits) select
            uint64_t split_val = 0;
            for (int i = 0; i < op.sum.n_split; ++i)
                if ((slice_base >> op.sum.split_bit[i]) & 1) split_val |= 1ull << op.sum.split_t[i];
            e = launch_slice_sum(ws + op.sum.src, dtype, op.sum, amps, P->net.n_open, t_lo, t_hi,
                                 overwrite, P->d_texp, P->d_stepcorr, (int)P->sched.steps.size(), split_val, s);
            ++launches;
            break;
        }
        default:
            return fail(TN_EINVAL, "unknown op");
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return TN_OK;
}

// Legal (kernel, tile) configurations of a GEMM op: N tile x raster group,
// each also on CTA pairs where the shape allows.
std::vector<std::pair<int, int>> gemm_candidates(const GemmOp &g, bool x3 = false) {
    std::vector<std::pair<int, int>> c;
    if (g.kernel == GK_C64_ROWS || g.kernel == GK_C64_TILED || g.kernel == GK_C64_TC) {
        c.push_back({GK_C64_ROWS, 0});
        if (g.lm >= 6 && g.ln >= 6 && g.lk >= 4) c.push_back({GK_C64_TILED, 0});
        if (x3) c.push_back({GK_C64_TC, 0});
    } else if (g.kernel == GK_LP_ROWS) {
        c.push_back({GK_LP_ROWS, 0});
    } else {
        const int np = std::max(16, 2 << g.ln);
        const int bn_max = std::min(np, 256);
        std::vector<int> bn_codes;
        for (int code = 1; code <= 4; ++code)
            if (kTcBn[code] <= bn_max && (int)bn_codes.size() < 3) bn_codes.push_back(code);
        if (bn_codes.empty()) bn_codes.push_back(0);
        const int64_t n_mt = std::max<int64_t>(1, ((int64_t)1 << g.lm) / 128);
        std::vector<int> gm_codes;
        if (n_mt > 4) {
            for (int code = 1; code <= 4; ++code)
                if (kTcGm[code] <= 2 * n_mt) gm_codes.push_back(code);
        }
        if (gm_codes.empty()) gm_codes.push_back(0);
        std::vector<int> codes = {0};   // 0: the fixed heuristic's N tile and raster group
        std::vector<int> seen = {tc_effective_tile(0, g.ln)};
        for (int b : bn_codes)
            for (int m : gm_codes) {
                const int code = b | (m << 4);
                const int eff = tc_effective_tile(code, g.ln);
                if (code == 0 || std::find(seen.begin(), seen.end(), eff) != seen.end()) continue;
                seen.push_back(eff);
                codes.push_back(code);
            }
        const bool gathered = g.idx_a >= 0 || g.idx_b >= 0;
        auto pair_ok = [&](int code) {
            const int bn = tc_tile_bn(tc_effective_tile(code, g.ln));
            return !gathered && tc_pair_eligible(1, g.fp8, g.lm, g.ln, g.lk, bn);
        };
        auto bres_ok = [&](int code) {
            const int bn = tc_tile_bn(tc_effective_tile(code, g.ln));
            return !g.fp8 && tc_bres_eligible(g.lm, g.ln, g.lk, (int64_t)1 << g.lb, bn, 0, gathered ? 1 : 0);
        };
        // the staged-store epilogue where the C write matters: short K, a
        // complex-half result, no split, no 2-D gather
        const bool staged_ok = g.lk <= 9 && g.tc == 1 && !gathered && g.ln >= 3 &&
                               tc_split(g.lm, g.ln, g.lk, (int64_t)1 << g.lb) == 1;
        for (int code : codes) {
            c.push_back({GK_LP_TC, code});
            if (staged_ok) c.push_back({GK_LP_TC, code | kTcStagedTile});
            if (pair_ok(code)) c.push_back({GK_LP_TC, code | kTcPairTile});
            if (bres_ok(code)) {
                c.push_back({GK_LP_TC, code | kTcBresTile});
                const int bn = tc_tile_bn(tc_effective_tile(code, g.ln));
                if (g.tc != 0 && g.out_rank == 0 && tc_bres_store_eligible(g.lm, g.ln, g.lk, (int64_t)1 << g.lb, bn))
                    c.push_back({GK_LP_TC, code | kTcBresTile | kTcStoreTile});
            }
            // (64-byte K chunks, tile bit 9, lost to 128-byte chunks on
            // every step of the 30-qubit workload: not a candidate)
        }
    }
    return c;
}

int perm_stride_class(const PermOp &p) {
    // how many of the 5 lowest output bits come from the 5 lowest input bits
    const int r = p.rank;
    int cls = 0;
    for (int ob = 0; ob < std::min(5, r); ++ob) {
        const int i = r - 1 - ob;              // output mode index
        const int in_bit = r - 1 - p.perm[i];
        if (in_bit < 5) ++cls;
    }
    return cls;
}

// Time one launch of an op (events around it on stream s).
int time_op(tn_plan_s *P, const Op &op, int64_t slice_base, cudaStream_t s, double &ms) {
    cudaEvent_t e0 = take_event(P), e1 = take_event(P);
    int launches = 0;
    TN_CUDA(cudaEventRecord(e0, s), "event");
    const int rc = run_op_raw(P, op, slice_base, nullptr, 0, 0, 0, s, launches);
    TN_CUDA(cudaEventRecord(e1, s), "event");
    if (rc != TN_OK) return rc;
    TN_CUDA(cudaEventSynchronize(e1), "event sync");
    float f = 0;
    cudaEventElapsedTime(&f, e0, e1);
    P->ev_pool.push_back(e0);
    P->ev_pool.push_back(e1);
    ms = f;
    return TN_OK;
}

// Power-of-two scale calibration (complex-half plans).  Each GEMM's output
// exponent comes from a bound, 2 K max|A| max|B|, that assumes the K terms add
// coherently; random-phase sums grow like sqrt(K), so large-K outputs land far
// below the top of the FP16 range and their small entries lose precision.
// Run slice 0's pass once: after each GEMM read the stored maximum and, if it
// is below 2^12, raise that step's exponent by the largest headroom h that
// keeps it at or below 2^12 (so it lands in (2^11, 2^12], 16x below the FP16
// limit), re-run it, and go on.  Outputs already at or above 2^12 keep the
// bound's exponent, which caps them at 2^14.  So on the calibration pass every
// complex-half GEMM output's stored maximum lies in (2^11, 2^14].  The
// headrooms are then fixed, so later calls stay deterministic.
int calibrate_plan(tn_plan_s *P, cudaStream_t s) {
    Schedule &S = P->sched;
    TN_CUDA(cudaMemsetAsync(P->d_err, 0, 4, s), "memset");
    TN_CUDA(cudaMemsetAsync(P->d_tmax, 0, (size_t)S.n_meta * 4, s), "memset");
    TN_CUDA(cudaMemsetAsync(P->d_texp, 0, (size_t)S.n_meta * 4, s), "memset");
    for (int phase = 0; phase < 2; ++phase)
        for (Op &op : S.ops) {
            if (op.phase != phase || op.kind == OP_SUM) continue;
            int launches = 0;
            int rc = run_op_raw(P, op, 0, nullptr, 0, 0, 0, s, launches);
            if (rc != TN_OK) return rc;
            if (op.kind != OP_GEMM || op.gemm.tc == 0) continue;   // complex64 outputs keep e = 0
            float mx = 0.0f;
            TN_CUDA(cudaMemcpyAsync(&mx, P->d_tmax + op.gemm.meta_c, 4, cudaMemcpyDeviceToHost, s), "read max");
            TN_CUDA(cudaStreamSynchronize(s), "sync");
            if (!(mx > 0.0f) || !std::isfinite(mx) || mx >= 4096.0f) continue;
            const int hr = std::min(100, (int)std::floor(std::log2(4096.0 / (double)mx)));
            if (hr <= 0) continue;
            op.gemm.headroom = hr;
            rc = run_op_raw(P, op, 0, nullptr, 0, 0, 0, s, launches);
            if (rc != TN_OK) return rc;
        }
    P->calibrated = true;
    if (P->graph_exec) {
        cudaGraphExecDestroy(P->graph_exec);
        P->graph_exec = nullptr;
    }
    int32_t herr = 0;
    TN_CUDA(cudaMemcpy(&herr, P->d_err, 4, cudaMemcpyDeviceToHost), "read error flag");
    if (herr & 1) return fail(TN_ETIMEOUT, "a bounded device wait gave up while calibrating");
    return TN_OK;
}

int tune_plan(tn_plan_s *P, cudaStream_t s) {
    Schedule &S = P->sched;
    const int dtype = P->opts.dtype;
    TN_CUDA(cudaMemsetAsync(P->d_err, 0, 4, s), "memset");
    if (dtype != TN_C64) {
        TN_CUDA(cudaMemsetAsync(P->d_tmax, 0, (size_t)S.n_meta * 4, s), "memset");
        TN_CUDA(cudaMemsetAsync(P->d_texp, 0, (size_t)S.n_meta * 4, s), "memset");
    }
    for (int phase = 0; phase < 2; ++phase)
        for (Op &op : S.ops) {
            if (op.phase != phase || op.kind == OP_SUM) continue;
            if (op.kind == OP_GEMM) {
                GemmOp &g = op.gemm;
                double best = 1e30;
                std::pair<int, int> pick{g.kernel, g.tile};
                for (const auto &cand : gemm_candidates(g, x3_eligible(P, g))) {
                    Op trial = op;
                    trial.gemm.kernel = cand.first;
                    trial.gemm.tile = cand.second;
                    double ms = 0, ms2 = 0;
                    int rc = time_op(P, trial, 0, s, ms);       // warm
                    if (rc == TN_OK) rc = time_op(P, trial, 0, s, ms2);
                    if (rc != TN_OK) return rc;
                    ms = std::min(ms, ms2);
                    P->tune_recs.push_back(tn_tune_record{0, g.lm, g.ln, g.lk, g.lb, dtype, cand.first,
                                                          cand.second, g.step, 0, ms});
                    if (ms < best) { best = ms; pick = cand; }
                }
                g.kernel = pick.first;
                g.tile = pick.second;
                // leave C as the chosen configuration writes it
                double ms = 0;
                const int rc = time_op(P, op, 0, s, ms);
                if (rc != TN_OK) return rc;
            } else {
                double ms = 0;
                const int rc = time_op(P, op, 0, s, ms);
                if (rc != TN_OK) return rc;
                if (op.kind == OP_PERM)
                    P->tune_recs.push_back(tn_tune_record{1, op.perm.rank, 0, 0, 0, dtype, -1,
                                                          perm_stride_class(op.perm), -1, 0, ms});
            }
        }
    // keep the per-step records (tn_plan_step) in line with the choices
    for (const Op &op : S.ops)
        if (op.kind == OP_GEMM && op.gemm.step >= 0 && op.gemm.step < (int)S.steps.size()) {
            S.steps[op.gemm.step].kernel = op.gemm.kernel;
            S.steps[op.gemm.step].tile = op.gemm.tile;
        }
    P->tuned = true;
    if (P->graph_exec) {
        cudaGraphExecDestroy(P->graph_exec);
        P->graph_exec = nullptr;
    }
    int32_t herr = 0;
    TN_CUDA(cudaMemcpy(&herr, P->d_err, 4, cudaMemcpyDeviceToHost), "read error flag");
    if (herr & 1) return fail(TN_ETIMEOUT, "a bounded device wait gave up while tuning");
    return TN_OK;
}

void cost_features(const tn_tune_record &r, float *f) {
    for (int i = 0; i < TN_COST_NFEAT; ++i) f[i] = 0.0f;
    const double esz = r.dtype == TN_C64 ? 8.0 : 4.0;
    if (r.dtype >= 0 && r.dtype <= 2) f[6 + r.dtype] = 1.0f;
    if (r.kind == 0) {
        f[0] = r.lm / 32.0f;
        f[1] = r.ln / 32.0f;
        f[2] = r.lk / 32.0f;
        f[3] = r.lb / 16.0f;
        f[4] = (r.lm + r.ln + r.lk + r.lb) / 64.0f;
        const double bytes = esz * (std::ldexp(1.0, r.lm + r.lk + r.lb) + std::ldexp(1.0, r.lk + r.ln + r.lb) +
                                    std::ldexp(1.0, r.lm + r.ln + r.lb));
        f[5] = (float)(std::log2(bytes) / 40.0);
        if (r.kernel >= 0 && r.kernel <= 3) f[10 + r.kernel] = 1.0f;
        if (r.kernel == GK_LP_TC) {
            // the configuration the launch really uses (tile 0 = the fixed
            // heuristic's choice for this shape)
            const int eff = tc_effective_tile(r.tile, r.ln);
            const int bc = eff & 15, gc = (eff >> 4) & 15;
            if (bc < 5) f[14 + bc] = 1.0f;
            if (gc < 5) f[19 + gc] = 1.0f;
            // CTA pairs (slot 25 is the permutation size in permute records)
            if ((r.tile & kTcPairTile) && tc_pair_eligible(1, 0, r.lm, r.ln, r.lk, tc_tile_bn(eff))) f[25] = 1.0f;
            // the B'-resident kernel (slot 24 is the stride class in permute records)
            if ((r.tile & kTcBresTile) &&
                tc_bres_eligible(r.lm, r.ln, r.lk, (int64_t)1 << r.lb, tc_tile_bn(eff), 0, 0))
                f[24] = (r.tile & kTcStoreTile) ? 2.0f : 1.0f;
        }
    } else {
        f[9] = 1.0f;
        f[5] = (float)(std::log2(2.0 * esz * std::ldexp(1.0, r.lm)) / 40.0);
        f[24] = r.tile / 5.0f;
        f[25] = r.lm / 40.0f;
    }
}

int predict_records(tn_cost_model_t *M, const std::vector<tn_tune_record> &recs, std::vector<float> &ms,
                    cudaStream_t s) {
    std::vector<float> x(recs.size() * TN_COST_NFEAT), y(recs.size());
    for (size_t i = 0; i < recs.size(); ++i) cost_features(recs[i], &x[i * TN_COST_NFEAT]);
    const int rc = tn_cost_model_predict(M, x.data(), (int64_t)recs.size(), y.data(), s);
    if (rc != TN_OK) return rc;
    ms.resize(recs.size());
    for (size_t i = 0; i < recs.size(); ++i) ms[i] = std::exp2(y[i]) * 1e-3f;   // log2 us -> ms
    return TN_OK;
}

int choose_by_model(tn_plan_s *P, tn_cost_model_t *M, cudaStream_t s) {
    Schedule &S = P->sched;
    std::vector<tn_tune_record> recs;
    std::vector<std::pair<int, std::pair<int, int>>> who;   // op index, candidate
    for (int i = 0; i < (int)S.ops.size(); ++i) {
        const Op &op = S.ops[i];
        if (op.kind != OP_GEMM) continue;
        const GemmOp &g = op.gemm;
        for (const auto &cand : gemm_candidates(g, x3_eligible(P, g))) {
            // the kernel variants of tile bits 10-12 (B'-resident, TMA
            // stores, staged stores) are left to exhaustive tuning: the
            // bundled training timings hold none of them, so the model would
            // extrapolate
            if (cand.second & (kTcBresTile | kTcStoreTile | kTcStagedTile)) continue;
            if (cand.first == GK_C64_TC) continue;
            recs.push_back(tn_tune_record{0, g.lm, g.ln, g.lk, g.lb, P->opts.dtype, cand.first, cand.second,
                                          g.step, 0, 0});
            who.push_back({i, cand});
        }
    }
    std::vector<float> ms;
    if (!recs.empty()) {
        const int rc = predict_records(M, recs, ms, s);
        if (rc != TN_OK) return rc;
    }
    // per op: the predicted time of the fixed heuristic's own choice and of
    // the best candidate.  The model moves away from the default only for a
    // predicted gain beyond its own error: 8% on steps predicted under
    // kSmallStepMs (launch-latency bound, where the timings it learned from
    // are mostly noise), 10% on larger ones (held-out steps of 0.2 s were
    // mispredicted by that much in relative terms).
    constexpr float kLearnedMargin = 0.92f, kLargeStepMargin = 0.90f;
    constexpr float kSmallStepMs = 0.05f;
    std::vector<float> best(S.ops.size(), 1e30f), dflt(S.ops.size(), -1.0f);
    std::vector<std::pair<int, int>> pick(S.ops.size());
    for (size_t k = 0; k < recs.size(); ++k) {
        const int i = who[k].first;
        const GemmOp &g = S.ops[i].gemm;
        if (who[k].second.first == g.kernel && who[k].second.second == g.tile) dflt[i] = ms[k];
        if (ms[k] < best[i]) {
            best[i] = ms[k];
            pick[i] = who[k].second;
        }
    }
    for (size_t i = 0; i < S.ops.size(); ++i) {
        if (S.ops[i].kind != OP_GEMM || best[i] >= 1e29f) continue;
        const float margin = dflt[i] < kSmallStepMs ? kLearnedMargin : kLargeStepMargin;
        if (dflt[i] < 0 || best[i] < margin * dflt[i]) {
            S.ops[i].gemm.kernel = pick[i].first;
            S.ops[i].gemm.tile = pick[i].second;
        }
    }
    for (const Op &op : S.ops)
        if (op.kind == OP_GEMM && op.gemm.step >= 0 && op.gemm.step < (int)S.steps.size()) {
            S.steps[op.gemm.step].kernel = op.gemm.kernel;
            S.steps[op.gemm.step].tile = op.gemm.tile;
        }
    P->tuned = true;
    if (P->graph_exec) {
        cudaGraphExecDestroy(P->graph_exec);
        P->graph_exec = nullptr;
    }
    return TN_OK;
}

}  // namespace

int tn::record_error(int code, const std::string &msg) { return fail(code, msg); }

// Device state, scale calibration and tile choice of a plan, as the first
// tn_contract call does them (each once).
int tn::prepare_for_contract(tn_plan_s *P, cudaStream_t s) {
    int rc = ensure_device(P);
    if (rc != TN_OK) return rc;
    if (!P->calibrated && P->opts.dtype != TN_C64 && P->prof_mask == 0 && !P->opts.no_scaling) {
        rc = calibrate_plan(P, s);
        if (rc != TN_OK) return rc;
    }
    if (!P->tuned && P->opts.tile_policy == TN_TILE_EXHAUSTIVE && P->prof_mask == 0) {
        rc = tune_plan(P, s);
        if (rc != TN_OK) return rc;
    }
    if (!P->tuned && P->opts.tile_policy == TN_TILE_LEARNED && P->cost_model) {
        rc = choose_by_model(P, P->cost_model, s);
        if (rc != TN_OK) return rc;
    }
    return TN_OK;
}

extern "C" {

void tn_plan_opts_default(tn_plan_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->dtype = TN_F16;
    o->max_log2_elems = 0;
    o->n_slice_edges = 0;
    o->path_seed = 1;
    o->path_trials = 1;
    o->slice_batch_log2 = 0;
    o->tile_policy = TN_TILE_FIXED;
}

}  // extern "C"

namespace {

int check_opts(const tn_plan_opts &o) {
    if (o.dtype != TN_C64 && o.dtype != TN_F16 && o.dtype != TN_BF16) return fail(TN_EINVAL, "bad dtype");
    if (o.path_trials < 1 || o.path_trials > 4096) return fail(TN_EINVAL, "path_trials must be in 1..4096");
    if (o.n_slice_edges < -1 || o.n_slice_edges > 40) return fail(TN_EINVAL, "n_slice_edges must be in -1..40");
    if (o.max_log2_elems > 40) return fail(TN_EINVAL, "max_log2_elems must be <= 40");
    if (o.anneal_kappa < 0) return fail(TN_EINVAL, "anneal_kappa must be >= 0");
    if (o.slice_batch_log2 < 0 || o.slice_batch_log2 > 16) return fail(TN_EINVAL, "slice_batch_log2 must be in 0..16");
    if (o.tile_policy < 0 || o.tile_policy > 2) return fail(TN_EINVAL, "bad tile_policy");
    if (o.small_log2 < 0) return fail(TN_EINVAL, "small_log2 must be >= 0");
    if (o.path_anneal_iters < 0) return fail(TN_EINVAL, "path_anneal_iters must be >= 0");
    if (o.recompute_log2 < 0 || o.recompute_log2 > 8) return fail(TN_EINVAL, "recompute_log2 must be in 0..8");
    if (o.no_scaling != 0 && o.no_scaling != 1) return fail(TN_EINVAL, "no_scaling must be 0 or 1");
    if (o.c64_tensor_cores != 0 && o.c64_tensor_cores != 1) return fail(TN_EINVAL, "c64_tensor_cores must be 0 or 1");
    if (o.no_scaling && o.fp8_min_log2_flops > 0)
        return fail(TN_EINVAL, "no_scaling does not apply to E4M3 steps (their scale is their range)");
    if (o.n_slice_edges < 0 && o.max_log2_elems <= 0)
        return fail(TN_EINVAL, "n_slice_edges = -1 needs max_log2_elems > 0");
    if (o.workspace_budget < 0) return fail(TN_EINVAL, "workspace_budget must be >= 0");
    return TN_OK;
}

// Path and slices on `plan_net` (the network the planner sees), refined by
// annealing when asked; checks the cap and the slice batch.
int plan_path(tn_plan_s *P, const Network &plan_net_in, std::string &err) {
    const tn_plan_opts &o = P->opts;
    const int n_target = o.n_slice_edges >= 0 ? o.n_slice_edges : -1;
    const int cap = o.max_log2_elems;
    int rc;
    // recomputation first: the open legs that shrink the unsliced path's
    // largest intermediate most are split off, and the path and the summed
    // slices are planned without them
    std::vector<int> split;
    Network split_net;
    if (o.recompute_log2 > 0) {
        Path p0;
        std::vector<int> none;
        rc = choose_slices(plan_net_in, o.path_seed, o.path_trials, 0, 0, p0, none, err);
        if (rc != TN_OK) return rc;
        rc = choose_recompute(plan_net_in, o.recompute_log2, p0, split, err);
        if (rc != TN_OK) return rc;
        split_net = plan_net_in;
        fix_legs(split_net, split);
    }
    const Network &plan_net = o.recompute_log2 > 0 ? split_net : plan_net_in;
    rc = choose_slices(plan_net, o.path_seed, o.path_trials, n_target, cap, P->path, P->sliced, err);
    if (rc != TN_OK) return rc;
    if (o.path_anneal_iters > 0) {
        // kappa: flops one element of HBM traffic is worth at the ridge
        // (complex-half 4 B x ~250 flop/B on the tensor cores; complex64
        // 8 B x ~12 flop/B on the CUDA cores)
        const double kappa =
            o.anneal_kappa > 0 ? (double)o.anneal_kappa : (o.dtype == TN_C64 ? 100.0 : 1000.0);
        // which edges are sliced is fixed by the greedy start (with a fixed
        // slice count annealing does not change it) and decides much of what
        // annealing can reach: anneal from path_trials starts (greedy
        // slicings under different seeds), two chains each, and keep the
        // cheapest job
        const int starts = std::max(1, o.path_trials);
        // slices per pass: as given, or (a workspace budget picks it later)
        // assumed all of them.  With recomputation the split output legs,
        // fixed while the path is planned, loop over every pass too: the
        // steps they reach are not known here, so no step is weighted
        const int bl = o.recompute_log2 > 0 ? -1 : o.workspace_budget > 0 ? 64 : std::max(0, o.slice_batch_log2);
        // the starts run on threads of their own (they share no mutable
        // state); the cheapest wins, ties to the lower start, as in order
        std::vector<Path> ps(starts);
        std::vector<std::vector<int>> ss(starts);
        std::vector<double> cost(starts, 0.0);
        std::vector<char> ok(starts, 0);
        ps[0] = P->path;
        ss[0] = P->sliced;
        run_parallel(starts, [&](int st) {
            const uint64_t sd = st == 0 ? o.path_seed : o.path_seed + 0xD1B54A32D192ED03ull * (uint64_t)st;
            std::string e2;
            if (st > 0 && choose_slices(plan_net, sd, o.path_trials, n_target, cap, ps[st], ss[st], e2) != TN_OK)
                return;
            refine_plan(plan_net, n_target, cap, sd, o.path_anneal_iters, kappa, bl, 2, ps[st], ss[st], &cost[st]);
            ok[st] = 1;
        });
        int best = 0;
        for (int st = 1; st < starts; ++st)
            if (ok[st] && cost[st] < cost[best]) best = st;
        P->path = std::move(ps[best]);
        P->sliced = std::move(ss[best]);
    }
    if (cap > 0 && P->path.max_log2 > cap) {
        err = "the slicing does not reach the cap (largest intermediate 2^" + std::to_string(P->path.max_log2) + ")";
        return TN_EINVAL;
    }
    if (o.slice_batch_log2 > (int)P->sliced.size()) {
        if (n_target >= 0) {
            err = "slice_batch_log2 exceeds the number of sliced edges";
            return TN_EINVAL;
        }
        // slicing to a cap: the planner decides how many slices there are
        P->opts.slice_batch_log2 = (int)P->sliced.size();
    }
    if (o.recompute_log2 > 0) {
        // the split legs after the summed slices: a pass's part of the
        // output is fixed by its highest slice-id bits
        P->sliced.insert(P->sliced.end(), split.begin(), split.end());
        P->n_recompute = o.recompute_log2;
    }
    P->batch_log2 = P->opts.slice_batch_log2;
    return TN_OK;
}

// Schedule and leaf store of a planned network.
int finish_plan(tn_plan_s *P, const SampleSpec *spec, std::string &err) {
    const tn_plan_opts &o = P->opts;
    auto schedule = [&](int b, Schedule &out) {
        return build_schedule(P->net, P->path, P->sliced, b, o.dtype, o.small_log2 > 0 ? o.small_log2 : kSmallLog2,
                              o.no_tensor_cores == 0, o.dtype == TN_C64 ? 0 : o.fp8_min_log2_flops, out, err, spec);
    };
    int rc;
    if (o.workspace_budget > 0) {
        // as many slices per pass as the workspace budget allows (one path,
        // several schedules): the largest fitting batch, else none
        const int summed = (int)P->sliced.size() - P->n_recompute;
        int b = std::min(16, summed);
        for (; b >= 0; --b) {
            Schedule S;
            rc = schedule(b, S);
            if (rc != TN_OK) return rc;
            if (S.ws_bytes <= o.workspace_budget || b == 0) {
                P->sched = std::move(S);
                break;
            }
        }
        P->batch_log2 = std::max(b, 0);
        P->opts.slice_batch_log2 = P->batch_log2;
    } else {
        rc = schedule(P->batch_log2, P->sched);
        if (rc != TN_OK) return rc;
    }
    int64_t offs = 0;
    for (const Leaf &L : P->net.leaves) {
        P->leaf_offset.push_back(offs);
        P->leaf_store.insert(P->leaf_store.end(), L.data.begin(), L.data.end());
        offs += (int64_t)L.data.size();
    }
    for (LeafJob &j : P->sched.leaf_jobs) j.src = P->leaf_offset[j.src];
    // complex64 on the tensor cores (opt-in): the fixed choice for the large
    // steps, where the split passes are small against the GEMM
    for (Op &op : P->sched.ops)
        if (op.kind == OP_GEMM && x3_eligible(P, op.gemm) &&
            op.gemm.lm + op.gemm.ln + op.gemm.lk + op.gemm.lb + 3 >= 36) {
            op.gemm.kernel = GK_C64_TC;
            op.gemm.tile = 0;
            if (op.gemm.step >= 0 && op.gemm.step < (int)P->sched.steps.size()) {
                P->sched.steps[op.gemm.step].kernel = GK_C64_TC;
                P->sched.steps[op.gemm.step].tile = 0;
            }
        }
    return TN_OK;
}

}  // namespace

extern "C" {

int tn_plan(const tn_circuit *circuit, const tn_query *query, const tn_plan_opts *opts,
            tn_plan_t **out) {
    if (!out) return fail(TN_EINVAL, "out is NULL");
    *out = nullptr;
    tn_plan_opts o;
    if (opts) o = *opts;
    else tn_plan_opts_default(&o);
    int rc = check_opts(o);
    if (rc != TN_OK) return rc;
    try {
        tn_plan_s *P = new tn_plan_s();
        P->opts = o;
        std::string err;
        rc = build_network(circuit, query, P->net, err);
        if (rc == TN_OK) rc = plan_path(P, P->net, err);
        if (rc == TN_OK) rc = finish_plan(P, nullptr, err);  // correlated query
        if (rc != TN_OK) { delete P; return fail(rc, err); }
        *out = P;
        return TN_OK;
    } catch (const std::bad_alloc &) {
        return fail(TN_ENOMEM, "host allocation failed");
    } catch (const std::exception &ex) {
        return fail(TN_EINVAL, ex.what());
    }
}

int tn_plan_samples(const tn_circuit *circuit, const uint8_t *samples, int32_t n_samples,
                    const tn_plan_opts *opts, tn_plan_t **out) {
    if (!out || !circuit || !samples) return fail(TN_EINVAL, "NULL argument");
    *out = nullptr;
    if (n_samples < 1 || n_samples > (1 << 20)) return fail(TN_EINVAL, "n_samples must be in 1..2^20");
    tn_plan_opts o;
    if (opts) o = *opts;
    else tn_plan_opts_default(&o);
    int rc = check_opts(o);
    if (rc != TN_OK) return rc;
    const int n = circuit->n_qubits;
    if (n < 1 || n > 64) return fail(TN_EINVAL, "n_qubits must be in 1..64");
    int k = 0;
    while ((1 << k) < n_samples) ++k;
    if (k > 24) return fail(TN_EINVAL, "too many samples");
    if (o.recompute_log2 != 0) return fail(TN_EINVAL, "recompute_log2 applies to correlated plans only");
    try {
        std::vector<uint64_t> bits((size_t)1 << k);
        for (int64_t s = 0; s < ((int64_t)1 << k); ++s) {
            const int64_t src = s < n_samples ? s : n_samples - 1;     // padding repeats the last
            uint64_t b = 0;
            for (int q = 0; q < n; ++q) {
                const uint8_t v = samples[src * n + q];
                if (v > 1) return fail(TN_EINVAL, "sample bits must be 0 or 1");
                b |= (uint64_t)v << q;
            }
            bits[(size_t)s] = b;
        }
        std::vector<int32_t> all(n);
        for (int q = 0; q < n; ++q) all[q] = q;
        std::vector<uint8_t> zeros(n, 0);
        tn_query query{n, all.data(), zeros.data()};
        // Two planning views, the cheaper schedule kept: output legs visible
        // as legs (the planner merges the tensors that carry them late, where
        // few rows per sample remain; best for many samples), or fixed (the
        // path of one closed network; best for few samples).  A view whose
        // hybrid schedule holds a tensor above the cap is dropped.
        tn_plan_s *P = nullptr;
        double best = 0;
        std::string err, first_err;
        rc = TN_OK;
        int first_rc = TN_OK;
        for (int view = 0; view < 2; ++view) {
            tn_plan_s *Q = new tn_plan_s();
            Q->opts = o;
            // the all-open network defeats the noiseless greedy pass (30-qubit
            // circuit, 4096 bitstrings: 1.6e18 flops against 1.6e15 with
            // randomized restarts): at least 4 restarts per view
            Q->opts.path_trials = std::max(o.path_trials, 4);
            std::string e;
            int r = build_network_open(circuit, &query, 64, Q->net, e);
            Network plan_net;
            if (r == TN_OK) {
                plan_net = Q->net;
                if (view == 1) fix_open_legs(plan_net);
                r = plan_path(Q, plan_net, e);
            }
            if (r == TN_OK) {
                SampleSpec spec;
                spec.k = k;
                spec.bits = bits;
                for (int j = 0; j < k; ++j) {
                    spec.sample_edges.push_back((int)Q->net.edges.size());
                    Q->net.edges.push_back(Edge{-1, -1, -1, -1, j});   // output bit j = sample index bit j
                }
                for (Edge &ed : Q->net.edges)
                    if (ed.qubit >= 0) ed.open_t = ed.open_t >= 0 ? n + ed.open_t : -1;   // dense outputs: not amplitude bits
                Q->net.n_open = k;
                r = finish_plan(Q, &spec, e);
            }
            if (r == TN_OK) {
                int real_max = 0;
                for (const StepRec &st : Q->sched.steps) real_max = std::max(real_max, st.lm + st.ln + st.lb);
                Q->path.max_log2 = real_max;
                if (view > 0 && o.max_log2_elems > 0 && real_max > o.max_log2_elems) {
                    r = TN_EINVAL;
                    e = "hybrid schedule above the cap";
                }
            }
            if (r != TN_OK) {
                if (first_rc == TN_OK) { first_rc = r; first_err = e; }
                delete Q;
                continue;
            }
            const double flops = Q->sched.flops_per_pass * (double)((int64_t)1 << Q->sliced.size()) + Q->sched.flops_inv;
            if (!P || flops < best) {
                delete P;
                P = Q;
                best = flops;
            } else {
                delete Q;
            }
        }
        if (!P) return fail(first_rc, first_err);
        *out = P;
        return TN_OK;
    } catch (const std::bad_alloc &) {
        return fail(TN_ENOMEM, "host allocation failed");
    } catch (const std::exception &ex) {
        return fail(TN_EINVAL, ex.what());
    }
}

int tn_plan_info(const tn_plan_t *P, tn_plan_stats *s) {
    if (!P || !s) return fail(TN_EINVAL, "NULL argument");
    std::memset(s, 0, sizeof(*s));
    s->n_qubits = P->net.n_qubits;
    s->n_open = P->net.n_open;
    s->n_leaves = (int32_t)P->net.leaves.size();
    int internal = 0;
    for (const Edge &e : P->net.edges) internal += e.v >= 0;
    s->n_edges = internal;
    s->n_slice_edges = (int32_t)P->sliced.size();
    s->n_slices = (int64_t)1 << P->sliced.size();
    s->n_steps = (int32_t)P->sched.steps.size();
    s->n_steps_invariant = P->sched.n_steps_inv;
    s->max_log2_elems = P->path.max_log2;
    s->slice_batch_log2 = P->batch_log2;
    const double passes_per_slice = std::ldexp(1.0, -P->batch_log2);
    s->flops_per_slice = P->sched.flops_per_pass * passes_per_slice;
    s->flops_invariant = P->sched.flops_inv;
    s->bytes_per_slice = P->sched.bytes_per_pass * passes_per_slice;
    s->workspace_bytes = P->sched.ws_bytes;
    s->n_permutes = P->sched.n_permutes;
    s->dtype = P->opts.dtype;
    s->leaf_bytes = (int64_t)P->leaf_store.size() * 16;
    s->n_recompute_edges = P->n_recompute;
    return TN_OK;
}

int tn_plan_sliced_edges(const tn_plan_t *P, int32_t *qubit, int32_t *after_gate, int32_t capacity) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    for (int j = 0; j < (int)P->sliced.size() && j < capacity; ++j) {
        const Edge &e = P->net.edges[P->sliced[j]];
        if (qubit) qubit[j] = e.qubit;
        if (after_gate) after_gate[j] = e.after_gate;
    }
    return TN_OK;
}

int tn_plan_leaf_source(const tn_plan_t *P, int32_t i, int32_t *gate, int32_t *qubit) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    if (i < 0 || i >= (int)P->net.leaves.size()) return fail(TN_EINVAL, "leaf index out of range");
    if (gate) *gate = P->net.leaves[i].gate;
    if (qubit) *qubit = P->net.leaves[i].qubit;
    return TN_OK;
}

int tn_plan_step(const tn_plan_t *P, int32_t i, tn_step_info *out) {
    if (!P || !out) return fail(TN_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)P->sched.steps.size()) return fail(TN_EINVAL, "step index out of range");
    const StepRec &r = P->sched.steps[i];
    out->a = r.a; out->b = r.b; out->c = r.c;
    out->log2_m = r.lm; out->log2_n = r.ln; out->log2_k = r.lk; out->log2_batch = r.lb;
    out->permute_a = r.permute_a;
    out->permute_b = r.permute_b;
    out->storage = r.storage;
    out->scale_headroom = 0;
    for (const Op &op : P->sched.ops)
        if (op.kind == OP_GEMM && op.gemm.step == i) out->scale_headroom = op.gemm.headroom;
    out->slice_invariant = r.invariant;
    out->kernel = r.kernel;
    out->tile = r.tile;
    return TN_OK;
}

int tn_plan_step_scale(tn_plan_t *P, int32_t i, int32_t *exp, float *stored_max) {
    if (!P || (!exp && !stored_max)) return fail(TN_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)P->sched.steps.size()) return fail(TN_EINVAL, "step index out of range");
    if (P->opts.dtype == TN_C64) return fail(TN_EINVAL, "complex64 plans keep no scale state");
    if (!P->dev_ready) return fail(TN_EINVAL, "no tn_contract call has run on this plan");
    int dev = 0;
    TN_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != P->device) return fail(TN_EINVAL, "plan was set up on another device");
    int meta = -1;
    for (const Op &op : P->sched.ops)
        if (op.kind == OP_GEMM && op.gemm.step == i) meta = op.gemm.meta_c;
    if (meta < 0) return fail(TN_EINVAL, "step has no GEMM");
    TN_CUDA(cudaDeviceSynchronize(), "sync");
    if (exp) TN_CUDA(cudaMemcpy(exp, P->d_texp + meta, 4, cudaMemcpyDeviceToHost), "read exponent");
    if (stored_max) TN_CUDA(cudaMemcpy(stored_max, P->d_tmax + meta, 4, cudaMemcpyDeviceToHost), "read max");
    return TN_OK;
}

int tn_plan_leaf_tensor(const tn_plan_t *P, int32_t i, int32_t capacity, int32_t *rank, int32_t *qubit,
                        int32_t *after_gate, double *data) {
    if (!P || !rank) return fail(TN_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)P->net.leaves.size()) return fail(TN_EINVAL, "leaf index out of range");
    const Leaf &lf = P->net.leaves[i];
    *rank = (int32_t)lf.legs.size();
    for (int p = 0; p < (int)lf.legs.size() && p < capacity; ++p) {
        const Edge &e = P->net.edges[lf.legs[p]];
        if (qubit) qubit[p] = e.qubit;
        if (after_gate) after_gate[p] = e.after_gate;
    }
    if (data)
        for (size_t x = 0; x < lf.data.size(); ++x) {
            data[2 * x] = lf.data[x].real();
            data[2 * x + 1] = lf.data[x].imag();
        }
    return TN_OK;
}

int tn_plan_decode_leaf(tn_plan_t *P, int64_t slice_id, int32_t i, int32_t capacity, int32_t *rank,
                        int32_t *qubit, int32_t *after_gate, float *data, void *stream) {
    if (!P || !rank) return fail(TN_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)P->net.leaves.size()) return fail(TN_EINVAL, "leaf index out of range");
    const int64_t n_slices = (int64_t)1 << P->sliced.size();
    const int64_t bsize = (int64_t)1 << P->batch_log2;
    if (slice_id < 0 || slice_id >= n_slices || slice_id % bsize != 0)
        return fail(TN_EINVAL, "slice_id must be a pass base (a multiple of 2^slice_batch_log2) below n_slices");
    int k = -1;
    for (size_t j = 0; j < P->sched.leaf_jobs.size(); ++j)
        if (P->sched.leaf_jobs[j].src == P->leaf_offset[i]) k = (int)j;
    if (k < 0) return fail(TN_EINVAL, "leaf has no preparation job");
    const LeafJob &job = P->sched.leaf_jobs[k];
    const Leaf &lf = P->net.leaves[i];
    *rank = job.rank_out;
    for (int q = 0; q < job.rank_out && q < capacity; ++q) {
        // leg q (outermost first) is output bit rank_out-1-q; keep_pos gives
        // its bit in the full leaf, whose leg p sits at bit rank_in-1-p
        const int p = job.rank_in - 1 - job.keep_pos[job.rank_out - 1 - q];
        const Edge &e = P->net.edges[lf.legs[p]];
        if (qubit) qubit[q] = e.qubit;
        if (after_gate) after_gate[q] = e.after_gate;
    }
    if (!data) return TN_OK;
    int rc = ensure_device(P);
    if (rc != TN_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    TN_CUDA(launch_leaf_prep(P->d_jobs + k, 1, P->d_store, P->d_ws, P->opts.dtype, slice_id, P->d_tmax,
                             P->d_texp, s),
            "leaf preparation");
    TN_CUDA(cudaMemcpyAsync(data, P->d_ws + job.dst, (size_t)8 << job.rank_out, cudaMemcpyDeviceToHost, s),
            "read prepared leaf");
    TN_CUDA(cudaStreamSynchronize(s), "sync");
    return TN_OK;
}

}  // extern "C"

namespace {

// Issue every op of one tn_contract call on stream s (no synchronization).
int enqueue_contract(tn_plan_s *P, int64_t slice_begin, int64_t slice_count, double *d_amps,
                     int accumulate, cudaStream_t s, int &launches) {
    const Schedule &S = P->sched;
    const bool lp = P->opts.dtype != TN_C64;
    int rc;
    TN_CUDA(cudaMemsetAsync(P->d_err, 0, 4, s), "memset");
    if (lp) {
        TN_CUDA(cudaMemsetAsync(P->d_tmax, 0, (size_t)S.n_meta * 4, s), "memset");
        TN_CUDA(cudaMemsetAsync(P->d_texp, 0, (size_t)S.n_meta * 4, s), "memset");
    }
    for (const Op &op : S.ops)
        if (op.phase == 0) {
            rc = run_op(P, op, 0, nullptr, 0, 0, 0, s, launches);
            if (rc != TN_OK) return rc;
        }
    const int64_t bsize = (int64_t)1 << P->batch_log2;
    const int64_t first = slice_begin / bsize * bsize;
    const int64_t last = (slice_begin + slice_count - 1) / bsize * bsize;
    // recomputation: passes fill disjoint parts of the output, so it is
    // cleared once and every pass adds
    const bool parts = P->n_recompute > 0;
    if (parts && !accumulate)
        TN_CUDA(cudaMemsetAsync(d_amps, 0, ((size_t)16) << P->net.n_open, s), "memset");
    for (int64_t base = first; base <= last; base += bsize) {
        if (lp && S.n_meta > S.n_meta_inv)
            TN_CUDA(cudaMemsetAsync(P->d_tmax + S.n_meta_inv, 0, (size_t)(S.n_meta - S.n_meta_inv) * 4, s),
                    "memset");
        const int t_lo = (int)std::max<int64_t>(0, slice_begin - base);
        const int t_hi = (int)std::min<int64_t>(bsize, slice_begin + slice_count - base);
        const int overwrite = (!accumulate && !parts && base == first) ? 1 : 0;
        for (const Op &op : S.ops)
            if (op.phase == 1) {
                rc = run_op(P, op, base, (double2 *)d_amps, t_lo, t_hi, overwrite, s, launches);
                if (rc != TN_OK) return rc;
            }
    }
    return TN_OK;
}

int64_t plan_passes(const tn_plan_s *P, int64_t slice_begin, int64_t slice_count) {
    const int64_t bsize = (int64_t)1 << P->batch_log2;
    const int64_t first = slice_begin / bsize * bsize;
    const int64_t last = (slice_begin + slice_count - 1) / bsize * bsize;
    return (last - first) / bsize + 1;
}

}  // namespace

extern "C" {

int tn_plan_tune(tn_plan_t *P, void *stream) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    if (P->prof_mask) return fail(TN_EINVAL, "profiling must be off while tuning");
    int rc = ensure_device(P);
    if (rc != TN_OK) return rc;
    return tune_plan(P, (cudaStream_t)stream);
}

int tn_plan_apply_tuning(tn_plan_t *P, const tn_tune_record *recs, int32_t n) {
    if (!P || n < 0 || (n > 0 && !recs)) return fail(TN_EINVAL, "bad argument");
    auto family = [](int k) {
        return (k == GK_C64_ROWS || k == GK_C64_TILED || k == GK_C64_TC) ? 0 : (k == GK_LP_ROWS ? 1 : 2);
    };
    Schedule &S = P->sched;
    for (Op &op : S.ops) {
        if (op.kind != OP_GEMM) continue;
        GemmOp &g = op.gemm;
        double best = 1e300;
        for (int i = 0; i < n; ++i) {
            const tn_tune_record &r = recs[i];
            if (r.kind != 0 || r.dtype != P->opts.dtype || r.lm != g.lm || r.ln != g.ln || r.lk != g.lk ||
                r.lb != g.lb || family(r.kernel) != family(g.kernel))
                continue;
            if (r.ms < best) {
                best = r.ms;
                g.kernel = r.kernel;
                g.tile = r.tile;
            }
        }
        if (g.step >= 0 && g.step < (int)S.steps.size()) {
            S.steps[g.step].kernel = g.kernel;
            S.steps[g.step].tile = g.tile;
        }
    }
    P->tuned = true;
    if (P->graph_exec) {
        cudaGraphExecDestroy(P->graph_exec);
        P->graph_exec = nullptr;
    }
    return TN_OK;
}

int tn_tune_records(const tn_plan_t *P, tn_tune_record *out, int32_t capacity, int32_t *n_total) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    if (n_total) *n_total = (int32_t)P->tune_recs.size();
    for (int i = 0; i < (int)P->tune_recs.size() && i < capacity && out; ++i) out[i] = P->tune_recs[i];
    return TN_OK;
}

int tn_cost_features(const tn_tune_record *recs, int32_t n, float *out) {
    if (n < 0 || (n > 0 && (!recs || !out))) return fail(TN_EINVAL, "bad argument");
    for (int i = 0; i < n; ++i) cost_features(recs[i], out + (size_t)i * TN_COST_NFEAT);
    return TN_OK;
}

int tn_cost_targets(const tn_tune_record *recs, int32_t n, float *out) {
    if (n < 0 || (n > 0 && (!recs || !out))) return fail(TN_EINVAL, "bad argument");
    for (int i = 0; i < n; ++i) out[i] = (float)std::log2(std::max(recs[i].ms, 1e-6) * 1e3);
    return TN_OK;
}

int tn_plan_set_cost_model(tn_plan_t *P, tn_cost_model_t *M) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    P->cost_model = M;
    return TN_OK;
}

int tn_plan_predict_ms(tn_plan_t *P, tn_cost_model_t *M, double *out_ms, void *stream) {
    if (!P || !M || !out_ms) return fail(TN_EINVAL, "NULL argument");
    const Schedule &S = P->sched;
    std::vector<tn_tune_record> recs;
    std::vector<int> phase;
    for (const Op &op : S.ops) {
        if (op.kind == OP_GEMM)
            recs.push_back(tn_tune_record{0, op.gemm.lm, op.gemm.ln, op.gemm.lk, op.gemm.lb, P->opts.dtype,
                                          op.gemm.kernel, op.gemm.tile, op.gemm.step, 0, 0});
        else if (op.kind == OP_PERM)
            recs.push_back(tn_tune_record{1, op.perm.rank, 0, 0, 0, P->opts.dtype, -1,
                                          perm_stride_class(op.perm), -1, 0, 0});
        else
            continue;
        phase.push_back(op.phase);
    }
    std::vector<float> ms;
    if (!recs.empty()) {
        const int rc = predict_records(M, recs, ms, (cudaStream_t)stream);
        if (rc != TN_OK) return rc;
    }
    const double passes = (double)plan_passes(P, 0, (int64_t)1 << P->sliced.size());
    double t = 0;
    for (size_t i = 0; i < recs.size(); ++i) t += phase[i] ? passes * ms[i] : ms[i];
    *out_ms = t;
    return TN_OK;
}

int tn_plan_set_queue(tn_plan_t *P, int enable) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    P->use_queue = enable != 0;
    if (!P->use_queue && P->queue) {
        tn_queue_destroy(P->queue);
        P->queue = nullptr;
    }
    return TN_OK;
}

int tn_plan_set_graph(tn_plan_t *P, int enable) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    P->use_graph = enable != 0;
    if (!P->use_graph && P->graph_exec) {
        cudaGraphExecDestroy(P->graph_exec);
        P->graph_exec = nullptr;
    }
    return TN_OK;
}

int tn_contract(tn_plan_t *P, int64_t slice_begin, int64_t slice_count, double *d_amps,
                int accumulate, void *stream, tn_contract_report *rep) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    const int64_t n_slices = (int64_t)1 << P->sliced.size();
    if (slice_begin < 0 || slice_count < 0 || slice_begin + slice_count > n_slices)
        return fail(TN_EINVAL, "slice range outside [0, n_slices)");
    if (!d_amps) return fail(TN_EINVAL, "d_amps is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = prepare_for_contract(P, s);
    if (rc != TN_OK) return rc;
    const int64_t n_amps = (int64_t)1 << P->net.n_open;
    if (slice_count == 0) {
        if (!accumulate) TN_CUDA(cudaMemsetAsync(d_amps, 0, n_amps * 16, s), "memset");
        if (rep) std::memset(rep, 0, sizeof(*rep));
        return TN_OK;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (rep) {
        TN_CUDA(cudaEventCreate(&ev0), "event");
        TN_CUDA(cudaEventCreate(&ev1), "event");
        TN_CUDA(cudaEventRecord(ev0, s), "event");
    }
    const Schedule &S = P->sched;
    int launches = 0;
    const bool graph = P->use_graph && s != nullptr && s != cudaStreamLegacy &&
                       s != cudaStreamPerThread && P->prof_mask == 0;
    if (P->use_queue && P->prof_mask == 0 && !accumulate) {
        const tn_plan_s::GraphKey key{slice_begin, slice_count, d_amps, accumulate, nullptr};
        if (!P->queue || !(P->queue_key == key)) {
            if (P->queue) {
                tn_queue_destroy(P->queue);
                P->queue = nullptr;
            }
            tn_plan_t *pl[1] = {P};
            double *am[1] = {d_amps};
            const int64_t b0[1] = {slice_begin}, c0[1] = {slice_count};
            rc = tn_queue_create(pl, 1, b0, c0, am, &P->queue);
            if (rc != TN_OK) return rc;
            P->queue_key = key;
        }
        // with a report requested the run is synchronized and its waits checked
        tn_contract_report qrep;
        rc = tn_queue_run(P->queue, stream, rep ? &qrep : nullptr);
        if (rc != TN_OK) return rc;
        launches = 1;
    } else if (graph) {
        const tn_plan_s::GraphKey key{slice_begin, slice_count, d_amps, accumulate, s};
        if (!P->graph_exec || !(P->graph_key == key)) {
            if (P->graph_exec) {
                cudaGraphExecDestroy(P->graph_exec);
                P->graph_exec = nullptr;
            }
            TN_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
            rc = enqueue_contract(P, slice_begin, slice_count, d_amps, accumulate, s, launches);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(s, &g);
            if (rc != TN_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ec != cudaSuccess) return cuda_fail(ec, "end capture");
            const cudaError_t ei = cudaGraphInstantiate(&P->graph_exec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                P->graph_exec = nullptr;
                return cuda_fail(ei, "graph instantiate");
            }
            P->graph_key = key;
            P->graph_launches = launches;
        }
        TN_CUDA(cudaGraphLaunch(P->graph_exec, s), "graph launch");
        launches = P->graph_launches;
    } else {
        rc = enqueue_contract(P, slice_begin, slice_count, d_amps, accumulate, s, launches);
        if (rc != TN_OK) return rc;
    }
    if (rep) {
        TN_CUDA(cudaEventRecord(ev1, s), "event");
        TN_CUDA(cudaEventSynchronize(ev1), "sync");
        float ms = 0;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        std::memset(rep, 0, sizeof(*rep));
        rep->ms = ms;
        rep->flops = S.flops_inv + S.flops_per_pass * (double)plan_passes(P, slice_begin, slice_count);
        rep->slices = slice_count;
        rep->kernels = launches;
        int32_t herr = 0;
        TN_CUDA(cudaMemcpy(&herr, P->d_err, 4, cudaMemcpyDeviceToHost), "read error flag");
        if (herr & 1) return fail(TN_ETIMEOUT, "a bounded device wait gave up");
        if (herr & 2)
            return fail(TN_EUNSUPPORTED, "a complex-half value overflowed its power-of-two scale");
    }
    return TN_OK;
}

int tn_contract_host(tn_plan_t *P, int64_t slice_begin, int64_t slice_count, double *h_amps,
                     void *stream, tn_contract_report *rep) {
    if (!P || !h_amps) return fail(TN_EINVAL, "NULL argument");
    int rc = ensure_device(P);
    if (rc != TN_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t amp_bytes = ((size_t)1 << P->net.n_open) * 16;
    double *d_amps = nullptr;
    TN_CUDA(cudaMallocAsync((void **)&d_amps, amp_bytes, s), "cudaMallocAsync");
    TN_CUDA(cudaMemcpyAsync(P->d_store, P->h_store_pinned, P->leaf_store.size() * 16,
                            cudaMemcpyHostToDevice, s),
            "upload leaves");
    rc = tn_contract(P, slice_begin, slice_count, d_amps, 0, stream, rep);
    if (rc == TN_OK) {
        cudaError_t e = cudaMemcpyAsync(h_amps, d_amps, amp_bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "download amplitudes");
    }
    cudaFreeAsync(d_amps, s);
    return rc;
}

struct tn_batch_s {
    std::vector<tn_plan_s *> plans;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
    double flops = 0;
    int64_t slices = 0;
};

int tn_batch_create(tn_plan_t *const *plans, int32_t n, double *const *d_amps, int32_t n_streams,
                    tn_batch_t **out) {
    if (!out || n < 1 || !plans || !d_amps) return fail(TN_EINVAL, "bad batch");
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!plans[i] || !d_amps[i] || plans[i]->opts.dtype != plans[0]->opts.dtype)
            return fail(TN_EINVAL, "plans and outputs must be non-NULL; plans must share dtype");
    if (n_streams < 1) n_streams = 1;
    n_streams = std::min(n_streams, std::min(n, 64));
    for (int i = 0; i < n; ++i) {
        if (plans[i]->prof_mask) return fail(TN_EINVAL, "profiling must be off for a batch");
        // device state, scale calibration and tile choice, as a first
        // tn_contract would do them (outside the capture below)
        int rc = prepare_for_contract(plans[i], nullptr);
        if (rc == TN_OK) {
            const cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) rc = cuda_fail(e, "plan set-up");
        }
        if (rc != TN_OK) return rc;
    }
    // longest-processing-time assignment of plans to side streams: by the
    // cost model's predicted time when every plan has a model attached,
    // else by flops
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    bool all_models = true;
    for (int i = 0; i < n; ++i) all_models = all_models && plans[i]->cost_model != nullptr;
    std::vector<double> w(n);
    for (int i = 0; i < n; ++i) {
        const tn_plan_s *P = plans[i];
        w[i] = P->sched.flops_inv + P->sched.flops_per_pass * (double)plan_passes(P, 0, (int64_t)1 << P->sliced.size()) + 1.0;
    }
    if (all_models)
        for (int i = 0; i < n; ++i) {
            double ms = 0;
            const int rc = tn_plan_predict_ms(plans[i], plans[i]->cost_model, &ms, nullptr);
            if (rc != TN_OK) return rc;
            w[i] = ms;
        }
    auto work = [&](int i) { return w[i]; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    std::vector<double> load(n_streams, 0.0);
    std::vector<std::vector<int>> assign(n_streams);
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        assign[k].push_back(i);
        load[k] += work(i);
    }
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> side(n_streams, nullptr);
    std::vector<cudaEvent_t> ev(n_streams + 1, nullptr);
    auto cleanup = [&]() {
        for (auto x : side) if (x) cudaStreamDestroy(x);
        for (auto e : ev) if (e) cudaEventDestroy(e);
        if (origin) cudaStreamDestroy(origin);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
    for (int k = 0; k < n_streams && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking);
    for (int k = 0; k <= n_streams && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "batch streams"); }
    tn_batch_s *B = new tn_batch_s();
    e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { delete B; cleanup(); return cuda_fail(e, "begin capture"); }
    cudaEventRecord(ev[n_streams], origin);
    int rc = TN_OK;
    for (int k = 0; k < n_streams && rc == TN_OK; ++k) {
        cudaStreamWaitEvent(side[k], ev[n_streams], 0);
        for (int i : assign[k]) {
            tn_plan_s *P = plans[i];
            const int64_t ns = (int64_t)1 << P->sliced.size();
            rc = enqueue_contract(P, 0, ns, d_amps[i], 0, side[k], B->launches);
            if (rc != TN_OK) break;
            B->flops += P->sched.flops_inv + P->sched.flops_per_pass * (double)plan_passes(P, 0, ns);
            B->slices += ns;
        }
        cudaEventRecord(ev[k], side[k]);
        cudaStreamWaitEvent(origin, ev[k], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(origin, &g);
    if (rc == TN_OK && e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cleanup();
    if (rc != TN_OK) { delete B; return rc; }
    if (e != cudaSuccess) { delete B; return cuda_fail(e, "batch graph"); }
    B->plans.assign(plans, plans + n);
    *out = B;
    return TN_OK;
}

int tn_batch_run(tn_batch_t *B, void *stream, tn_contract_report *rep) {
    if (!B || !B->exec) return fail(TN_EINVAL, "NULL batch");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (rep) {
        TN_CUDA(cudaEventCreate(&ev0), "event");
        TN_CUDA(cudaEventCreate(&ev1), "event");
        TN_CUDA(cudaEventRecord(ev0, s), "event");
    }
    TN_CUDA(cudaGraphLaunch(B->exec, s), "graph launch");
    if (rep) {
        TN_CUDA(cudaEventRecord(ev1, s), "event");
        TN_CUDA(cudaEventSynchronize(ev1), "sync");
        float ms = 0;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        std::memset(rep, 0, sizeof(*rep));
        rep->ms = ms;
        rep->flops = B->flops;
        rep->slices = B->slices;
        rep->kernels = B->launches;
        for (tn_plan_s *P : B->plans) {
            int32_t herr = 0;
            TN_CUDA(cudaMemcpy(&herr, P->d_err, 4, cudaMemcpyDeviceToHost), "read error flag");
            if (herr & 1) return fail(TN_ETIMEOUT, "a bounded device wait gave up");
            if (herr & 2)
                return fail(TN_EUNSUPPORTED, "a complex-half value overflowed its power-of-two scale");
        }
    }
    return TN_OK;
}

void tn_batch_destroy(tn_batch_t *B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    delete B;
}

int tn_contract_batch(tn_plan_t *const *plans, int32_t n, double *const *d_amps, void *stream) {
    if (n == 0) return TN_OK;
    tn_batch_t *B = nullptr;
    int rc = tn_batch_create(plans, n, d_amps, 16, &B);
    if (rc != TN_OK) return rc;
    rc = tn_batch_run(B, stream, nullptr);
    if (rc == TN_OK) {
        const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "batch sync");
    }
    tn_batch_destroy(B);
    return rc;
}

int tn_sample(const double *d_amps, int32_t n_open, int32_t k, int64_t *out_idx, double *out_prob,
              void *stream) {
    if (!d_amps || !out_idx || !out_prob) return fail(TN_EINVAL, "NULL argument");
    if (n_open < 0 || n_open > 30) return fail(TN_EINVAL, "n_open must be in 0..30");
    const int64_t n = (int64_t)1 << n_open;
    if (k < 1 || k > n) return fail(TN_EINVAL, "k must be in 1..2^n_open");
    cudaStream_t s = (cudaStream_t)stream;
    // one allocation: the k results, then the selection's scratch
    const size_t scratch = topk_scratch_bytes(n, k);
    const size_t res = ((size_t)k * 16 + 255) / 256 * 256;
    char *d_buf = nullptr;
    TN_CUDA(cudaMallocAsync((void **)&d_buf, res + scratch, s), "cudaMallocAsync");
    int64_t *d_idx = (int64_t *)d_buf;
    double *d_prob = (double *)(d_buf + (size_t)k * 8);
    cudaError_t e = launch_topk_select((const double2 *)d_amps, n, k, scratch ? d_buf + res : nullptr, d_idx,
                                       d_prob, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_idx, d_idx, (size_t)k * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_prob, d_prob, (size_t)k * 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_buf, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "tn_sample");
    return TN_OK;
}

int tn_metrics(const double *d_amps, const double *d_ref, int64_t n, int32_t n_qubits, double *out,
               void *stream) {
    if (!d_amps || !out || n < 1) return fail(TN_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int n_blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
    double *d_part = nullptr;
    TN_CUDA(cudaMallocAsync((void **)&d_part, (size_t)(n_blocks * 5 + 5) * 8, s), "cudaMallocAsync");
    double h[5];
    cudaError_t e = launch_metrics((const double2 *)d_amps, (const double2 *)d_ref, n,
                                   d_part + n_blocks * 5, d_part, n_blocks, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_part + n_blocks * 5, 40, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_part, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "tn_metrics");
    out[0] = h[0];
    if (d_ref) {
        out[1] = std::sqrt(h[2]) / std::sqrt(h[1]);
        out[2] = (h[3] * h[3] + h[4] * h[4]) / (h[1] * h[0]);
    } else {
        out[1] = out[2] = NAN;
    }
    out[3] = std::ldexp(h[0] / (double)n, n_qubits) - 1.0;
    return TN_OK;
}

int tn_profile(tn_plan_t *P, uint32_t class_mask) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    for (auto &r : P->prof) {
        P->ev_pool.push_back(r.e0);
        P->ev_pool.push_back(r.e1);
    }
    P->prof.clear();
    P->prof_mask = class_mask & ((1u << TN_KC_COUNT) - 1);
    return TN_OK;
}

int tn_profile_read(tn_plan_t *P, tn_kernel_stats *out) {
    if (!P || !out) return fail(TN_EINVAL, "NULL argument");
    for (int c = 0; c < TN_KC_COUNT; ++c) out[c] = tn_kernel_stats{0, 0.0, 0.0, 0.0};
    for (auto &r : P->prof) {
        TN_CUDA(cudaEventSynchronize(r.e1), "event sync");
        float ms = 0;
        TN_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1), "event time");
        out[r.cls].launches += r.kernels;
        out[r.cls].ms += ms;
        out[r.cls].flops += r.flops;
        out[r.cls].bytes += r.bytes;
    }
    return TN_OK;
}

void tn_plan_destroy(tn_plan_t *P) {
    if (!P) return;
    if (P->dev_ready) cudaDeviceSynchronize();
    if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
    if (P->queue) tn_queue_destroy(P->queue);
    for (auto &r : P->prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    for (auto e : P->ev_pool) cudaEventDestroy(e);
    plan_dev_free_all(P);
    if (P->h_store_pinned) cudaFreeHost(P->h_store_pinned);
    delete P;
}

const char *tn_strerror(int code) {
    switch (code) {
        case TN_OK: return "ok";
        case TN_EINVAL: return "invalid argument";
        case TN_ENOMEM: return "out of memory";
        case TN_ECUDA: return "CUDA error";
        case TN_ETIMEOUT: return "device wait timed out";
        case TN_EUNSUPPORTED: return "unsupported";
        default: return "unknown error";
    }
}

const char *tn_last_error(void) { return g_err.c_str(); }

}  // extern "C"

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
    P->d_tmax = (float *)plan_dev_alloc(P, std::max<size_t>(64, (size_t)S.n_meta * 4));
    P->d_texp = (int32_t *)plan_dev_alloc(P, std::max<size_t>(64, (size_t)S.n_meta * 4));
    P->d_err = (int32_t *)plan_dev_alloc(P, 64);
    if (!P->d_ws || !P->d_store || !P->d_jobs || !P->d_tmax || !P->d_texp || !P->d_err) {
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
        case OP_PERM: bytes = 2 * std::ldexp(esz, op.perm.rank); return TN_KC_PERMUTE;
        case OP_BPREP: {
            const double b = std::ldexp(1.0, op.bprep.lb);
            bytes = b * (std::ldexp(esz, op.bprep.lk + op.bprep.ln) + (double)op.bprep.np * std::ldexp(4.0, op.bprep.lk));
            return TN_KC_BPREP;
        }
        case OP_GEMM: {
            const GemmOp &g = op.gemm;
            flops = 8.0 * std::ldexp(1.0, g.lm + g.ln + g.lk + g.lb);
            const double bsz = g.kernel == GK_LP_TC
                                   ? std::max(16.0, std::ldexp(2.0, g.ln)) * std::ldexp(4.0, g.lk)
                                   : std::ldexp(esz, g.lk + g.ln);
            bytes = std::ldexp(1.0, g.lb) * (std::ldexp(esz, g.lm + g.lk) + bsz + std::ldexp(esz, g.lm + g.ln));
            if (g.kernel == GK_LP_TC) return TN_KC_GEMM_TC;
            if (g.kernel == GK_LP_ROWS) return TN_KC_GEMM_LP;
            return TN_KC_GEMM_C64;
        }
        case OP_SUM: bytes = std::ldexp(esz, op.sum.rank); return TN_KC_SUM;
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
    tn_plan_s::ProfRec r{cls, take_event(P), take_event(P), fl, by};
    cudaEventRecord(r.e0, s);
    const int rc = run_op_raw(P, op, slice_base, amps, t_lo, t_hi, overwrite, s, launches);
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
            e = launch_permute(ws + op.perm.src, ws + op.perm.dst, pp, esz, s);
            ++launches;
            break;
        }
        case OP_BPREP:
            e = launch_bprep_perm(ws + op.bprep.src, ws + op.bprep.dst, op.bprep.rank, op.bprep.perm,
                                  op.bprep.lk, op.bprep.ln, op.bprep.lb, op.bprep.np, s);
            ++launches;
            break;
        case OP_GEMM: {
            const GemmOp &g = op.gemm;
            const int64_t batch = (int64_t)1 << g.lb;
            const int64_t sa = (int64_t)1 << (g.lm + g.lk), sb = (int64_t)1 << (g.lk + g.ln),
                          sc = (int64_t)1 << (g.lm + g.ln);
            ScaleRef sr{};
            sr.tmax = P->d_tmax;
            sr.texp = P->d_texp;
            sr.meta_a = g.meta_a;
            sr.meta_b = g.meta_b;
            sr.meta_c = g.meta_c;
            sr.out_max = P->d_tmax + g.meta_c;
            switch (g.kernel) {
                case GK_C64_ROWS:
                    e = launch_gemm_rows_c64((const float2 *)(ws + g.a), (const float2 *)(ws + g.b),
                                             (float2 *)(ws + g.c), g.lm, g.ln, g.lk, batch, sa, sb, sc, s);
                    break;
                case GK_C64_TILED:
                    e = launch_gemm_tiled_c64((const float2 *)(ws + g.a), (const float2 *)(ws + g.b),
                                              (float2 *)(ws + g.c), g.lm, g.ln, g.lk, batch, sa, sb,
                                              sc, g.tile, s);
                    break;
                case GK_LP_ROWS:
                    e = launch_gemm_rows_lp(dtype, ws + g.a, ws + g.b, ws + g.c, g.lm, g.ln, g.lk,
                                            batch, sa, sb, sc, sr, s);
                    break;
                case GK_LP_TC: {
                    TcGemmDesc d;
                    d.dtype = dtype;
                    d.A = ws + g.a;
                    d.Bp = ws + g.b;
                    d.C = ws + g.c;
                    d.lm = g.lm; d.ln = g.ln; d.lk = g.lk;
                    d.batch = batch;
                    d.batch_a = g.lb > 0;
                    d.batch_b = g.lb > 0;
                    d.np = std::max(16, 2 << g.ln);
                    e = launch_gemm_tc(d, sr, P->d_err, s);
                    break;
                }
                default:
                    return fail(TN_EINVAL, "unknown kernel");
            }
            ++launches;
            break;
        }
        case OP_SUM:
            e = launch_slice_sum(ws + op.sum.src, dtype, op.sum, amps, P->net.n_open, t_lo, t_hi,
                                 overwrite, P->d_texp, s);
            ++launches;
            break;
        default:
            return fail(TN_EINVAL, "unknown op");
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return TN_OK;
}

}  // namespace

int tn::record_error(int code, const std::string &msg) { return fail(code, msg); }

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

int tn_plan(const tn_circuit *circuit, const tn_query *query, const tn_plan_opts *opts,
            tn_plan_t **out) {
    if (!out) return fail(TN_EINVAL, "out is NULL");
    *out = nullptr;
    tn_plan_opts o;
    if (opts) o = *opts;
    else tn_plan_opts_default(&o);
    if (o.dtype != TN_C64 && o.dtype != TN_F16 && o.dtype != TN_BF16) return fail(TN_EINVAL, "bad dtype");
    if (o.path_trials < 1 || o.path_trials > 4096) return fail(TN_EINVAL, "path_trials must be in 1..4096");
    if (o.n_slice_edges < -1 || o.n_slice_edges > 40) return fail(TN_EINVAL, "n_slice_edges must be in -1..40");
    if (o.max_log2_elems > 40) return fail(TN_EINVAL, "max_log2_elems must be <= 40");
    if (o.slice_batch_log2 < 0 || o.slice_batch_log2 > 16) return fail(TN_EINVAL, "slice_batch_log2 must be in 0..16");
    if (o.tile_policy < 0 || o.tile_policy > 2) return fail(TN_EINVAL, "bad tile_policy");
    try {
        tn_plan_s *P = new tn_plan_s();
        P->opts = o;
        std::string err;
        int rc = build_network(circuit, query, P->net, err);
        if (rc != TN_OK) { delete P; return fail(rc, err); }
        const int n_target = o.n_slice_edges >= 0 ? o.n_slice_edges : -1;
        const int cap = o.max_log2_elems;
        if (n_target < 0 && cap <= 0) { delete P; return fail(TN_EINVAL, "n_slice_edges = -1 needs max_log2_elems > 0"); }
        rc = choose_slices(P->net, o.path_seed, o.path_trials, n_target, cap, P->path, P->sliced, err);
        if (rc != TN_OK) { delete P; return fail(rc, err); }
        if (cap > 0 && P->path.max_log2 > cap) {
            delete P;
            return fail(TN_EINVAL, "the slicing does not reach the cap (largest intermediate 2^" +
                                       std::to_string(P->path.max_log2) + ")");
        }
        if (o.slice_batch_log2 > (int)P->sliced.size()) {
            delete P;
            return fail(TN_EINVAL, "slice_batch_log2 exceeds the number of sliced edges");
        }
        P->batch_log2 = o.slice_batch_log2;
        rc = build_schedule(P->net, P->path, P->sliced, P->batch_log2, o.dtype, P->sched, err);
        if (rc != TN_OK) { delete P; return fail(rc, err); }
        // leaf store
        int64_t offs = 0;
        for (const Leaf &L : P->net.leaves) {
            P->leaf_offset.push_back(offs);
            P->leaf_store.insert(P->leaf_store.end(), L.data.begin(), L.data.end());
            offs += (int64_t)L.data.size();
        }
        for (LeafJob &j : P->sched.leaf_jobs) j.src = P->leaf_offset[j.src];
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

int tn_plan_step(const tn_plan_t *P, int32_t i, tn_step_info *out) {
    if (!P || !out) return fail(TN_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)P->sched.steps.size()) return fail(TN_EINVAL, "step index out of range");
    const StepRec &r = P->sched.steps[i];
    out->a = r.a; out->b = r.b; out->c = r.c;
    out->log2_m = r.lm; out->log2_n = r.ln; out->log2_k = r.lk; out->log2_batch = r.lb;
    out->permute_a = r.permute_a;
    out->permute_b = r.permute_b;
    out->slice_invariant = r.invariant;
    out->kernel = r.kernel;
    out->tile = r.tile;
    return TN_OK;
}

int tn_contract(tn_plan_t *P, int64_t slice_begin, int64_t slice_count, double *d_amps,
                int accumulate, void *stream, tn_contract_report *rep) {
    if (!P) return fail(TN_EINVAL, "NULL plan");
    const int64_t n_slices = (int64_t)1 << P->sliced.size();
    if (slice_begin < 0 || slice_count < 0 || slice_begin + slice_count > n_slices)
        return fail(TN_EINVAL, "slice range outside [0, n_slices)");
    if (!d_amps) return fail(TN_EINVAL, "d_amps is NULL");
    int rc = ensure_device(P);
    if (rc != TN_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
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
    const bool lp = P->opts.dtype != TN_C64;
    int launches = 0;
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
    for (int64_t base = first; base <= last; base += bsize) {
        if (lp && S.n_meta > S.n_meta_inv)
            TN_CUDA(cudaMemsetAsync(P->d_tmax + S.n_meta_inv, 0, (size_t)(S.n_meta - S.n_meta_inv) * 4, s),
                    "memset");
        const int t_lo = (int)std::max<int64_t>(0, slice_begin - base);
        const int t_hi = (int)std::min<int64_t>(bsize, slice_begin + slice_count - base);
        const int overwrite = (!accumulate && base == first) ? 1 : 0;
        for (const Op &op : S.ops)
            if (op.phase == 1) {
                rc = run_op(P, op, base, (double2 *)d_amps, t_lo, t_hi, overwrite, s, launches);
                if (rc != TN_OK) return rc;
            }
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
        const int64_t passes = (last - first) / bsize + 1;
        rep->flops = S.flops_inv + S.flops_per_pass * (double)passes;
        rep->slices = slice_count;
        rep->kernels = launches;
        int32_t herr = 0;
        TN_CUDA(cudaMemcpy(&herr, P->d_err, 4, cudaMemcpyDeviceToHost), "read error flag");
        if (herr) return fail(TN_ETIMEOUT, "a bounded device wait gave up");
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

int tn_contract_batch(tn_plan_t *const *plans, int32_t n, double *const *d_amps, void *stream) {
    if (n < 0 || (n > 0 && (!plans || !d_amps))) return fail(TN_EINVAL, "bad batch");
    for (int i = 0; i < n; ++i)
        if (!plans[i] || plans[i]->opts.dtype != plans[0]->opts.dtype)
            return fail(TN_EINVAL, "plans must be non-NULL and share dtype");
    for (int i = 0; i < n; ++i) {
        const int64_t ns = (int64_t)1 << plans[i]->sliced.size();
        const int rc = tn_contract(plans[i], 0, ns, d_amps[i], 0, stream, nullptr);
        if (rc != TN_OK) return rc;
    }
    return TN_OK;
}

int tn_sample(const double *d_amps, int32_t n_open, int32_t k, int64_t *out_idx, double *out_prob,
              void *stream) {
    if (!d_amps || !out_idx || !out_prob) return fail(TN_EINVAL, "NULL argument");
    if (n_open < 0 || n_open > 30) return fail(TN_EINVAL, "n_open must be in 0..30");
    const int64_t n = (int64_t)1 << n_open;
    if (k < 1 || k > n) return fail(TN_EINVAL, "k must be in 1..2^n_open");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t *d_idx = nullptr;
    double *d_prob = nullptr;
    TN_CUDA(cudaMallocAsync((void **)&d_idx, (size_t)k * 8, s), "cudaMallocAsync");
    TN_CUDA(cudaMallocAsync((void **)&d_prob, (size_t)k * 8, s), "cudaMallocAsync");
    cudaError_t e = launch_topk((const double2 *)d_amps, n, k, d_idx, d_prob, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_idx, d_idx, (size_t)k * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_prob, d_prob, (size_t)k * 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_idx, s);
    cudaFreeAsync(d_prob, s);
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
        out[r.cls].launches += 1;
        out[r.cls].ms += ms;
        out[r.cls].flops += r.flops;
        out[r.cls].bytes += r.bytes;
    }
    return TN_OK;
}

void tn_plan_destroy(tn_plan_t *P) {
    if (!P) return;
    if (P->dev_ready) cudaDeviceSynchronize();
    for (auto &r : P->prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    for (auto e : P->ev_pool) cudaEventDestroy(e);
    plan_dev_free_all(P);
    if (P->h_store_pinned) cudaFreeHost(P->h_store_pinned);
    delete P;
}

int tn_permute(const void *in, void *out, int32_t rank, const int32_t *perm, int32_t elem_bytes,
               void *stream) {
    if (!in || !out || !perm) return fail(TN_EINVAL, "NULL argument");
    if (rank < 0 || rank > 34) return fail(TN_EINVAL, "rank must be in 0..34");
    if (elem_bytes != 4 && elem_bytes != 8) return fail(TN_EINVAL, "elem_bytes must be 4 or 8");
    bool seen[kMaxRank] = {false};
    for (int i = 0; i < rank; ++i) {
        if (perm[i] < 0 || perm[i] >= rank || seen[perm[i]]) return fail(TN_EINVAL, "perm is not a permutation");
        seen[perm[i]] = true;
    }
    const PermParams pp = make_perm_params(rank, perm);
    cudaError_t e = launch_permute(in, out, pp, elem_bytes, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "tn_permute");
    return TN_OK;
}

int tn_gemm(int32_t dtype, const void *A, const void *B, void *C, int64_t M, int64_t N, int64_t K,
            int64_t batch, int32_t batch_a, int32_t batch_b, int32_t scale_exp, int32_t kernel,
            float *out_max, void *stream) {
    if (!A || !B || !C) return fail(TN_EINVAL, "NULL operand");
    auto lg = [](int64_t v) {
        int l = 0;
        while (((int64_t)1 << l) < v) ++l;
        return (((int64_t)1 << l) == v) ? l : -1;
    };
    const int lm = lg(M), ln = lg(N), lk = lg(K);
    if (lm < 0 || ln < 0 || lk < 0 || lm > 34 || ln > 24 || lk > 24)
        return fail(TN_EINVAL, "M, N, K must be powers of two (M <= 2^34, N, K <= 2^24)");
    if (batch < 1 || batch > 65535) return fail(TN_EINVAL, "batch must be in 1..65535");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t sa = batch_a ? M * K : 0, sb = batch_b ? K * N : 0, sc = M * N;
    cudaError_t e;
    if (dtype == TN_C64) {
        int kk = kernel;
        if (kk < 0) kk = (lm >= 6 && ln >= 6 && lk >= 4) ? GK_C64_TILED : GK_C64_ROWS;
        if (kk == GK_C64_TILED)
            e = launch_gemm_tiled_c64((const float2 *)A, (const float2 *)B, (float2 *)C, lm, ln, lk,
                                      batch, sa, sb, sc, 0, s);
        else if (kk == GK_C64_ROWS)
            e = launch_gemm_rows_c64((const float2 *)A, (const float2 *)B, (float2 *)C, lm, ln, lk,
                                     batch, sa, sb, sc, s);
        else
            return fail(TN_EINVAL, "kernel variant not valid for TN_C64");
    } else if (dtype == TN_F16 || dtype == TN_BF16) {
        ScaleRef sr{};
        sr.fixed_exp = scale_exp;
        sr.out_max = out_max;
        int kk = kernel;
        if (kk < 0) kk = tc_gemm_supported(lk, ln) ? GK_LP_TC : GK_LP_ROWS;
        if (kk == GK_LP_ROWS) {
            e = launch_gemm_rows_lp(dtype, A, B, C, lm, ln, lk, batch, sa, sb, sc, sr, s);
        } else if (kk == GK_LP_TC) {
            if (!tc_gemm_supported(lk, ln)) return fail(TN_EUNSUPPORTED, "tensor-core path needs K >= 8");
            const int np = std::max(16, (int)(2 * N));
            const int64_t bbatch = batch_b ? batch : 1;
            void *bp = nullptr;
            TN_CUDA(cudaMallocAsync(&bp, (size_t)np * 2 * K * 2 * bbatch, s), "cudaMallocAsync");
            e = launch_bprep(dtype, B, bp, lk, ln, bbatch, np, s);
            if (e == cudaSuccess) {
                TcGemmDesc d;
                d.dtype = dtype;
                d.A = A; d.Bp = bp; d.C = C;
                d.lm = lm; d.ln = ln; d.lk = lk;
                d.batch = batch;
                d.batch_a = batch_a ? 1 : 0;
                d.batch_b = batch_b ? 1 : 0;
                d.np = np;
                e = launch_gemm_tc(d, sr, nullptr, s);
            }
            cudaFreeAsync(bp, s);
        } else {
            return fail(TN_EINVAL, "kernel variant not valid for complex-half");
        }
    } else {
        return fail(TN_EINVAL, "bad dtype");
    }
    if (e != cudaSuccess) return cuda_fail(e, "tn_gemm");
    return TN_OK;
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

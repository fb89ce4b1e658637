// Device schedule of a plan: for every pairwise step, the GEMM form of the
// einsum (paper Sec. 3.3, Eq. 3-4: reduced modes = the modes both operands
// share; result modes = the union minus those), the operand layouts and the
// explicit permutations they need, the workspace buffers, and the kernel.
//
// Layout rule.  Each device tensor is stored row-major over an ordered mode
// list.  The larger operand A must be [batch][M][K] (K innermost, so it is
// read as a K-major GEMM operand with no copy); if its K modes are not
// already its innermost modes it is permuted once.  The smaller operand B is
// brought to [batch][K][N] (same K order as A), and for the tensor-core path
// padded to B' (Eq. 6).  C is written as [batch][M][N].  When A must be
// permuted anyway, and for B's N modes, the order is chosen so that the modes
// the next step will contract end up innermost (fewer permutations later).
//
// Slices: bit j of a slice id fixes sliced edge j.  The low `batch_log2`
// sliced edges are not fixed but carried as batch modes (hyperedges that are
// never reduced) so 2^batch_log2 slices run in one pass; their sum is taken
// by the final FP64 kernel.  Steps whose inputs do not depend on the looped
// slice bits run once per contract call (phase 0).
#include <algorithm>
#include <cmath>
#include <map>
#include <set>

#include "plan.h"

namespace tn {

namespace {

bool contains(const std::vector<int> &v, int e) { return std::find(v.begin(), v.end(), e) != v.end(); }

std::vector<int> sorted_copy(std::vector<int> v) {
    std::sort(v.begin(), v.end());
    return v;
}

// first-fit arena on byte offsets
struct Arena {
    std::map<int64_t, int64_t> free_;  // offset -> size
    int64_t top = 0;
    static int64_t align(int64_t x) { return (x + 1023) / 1024 * 1024; }
    int64_t alloc(int64_t bytes) {
        bytes = align(std::max<int64_t>(bytes, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const int64_t off = it->first, rem = it->second - bytes;
                free_.erase(it);
                if (rem > 0) free_[off + bytes] = rem;
                return off;
            }
        }
        const int64_t off = top;
        top += bytes;
        return off;
    }
    void release(int64_t off, int64_t bytes) {
        bytes = align(std::max<int64_t>(bytes, 1));
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct BufReq {
    int64_t bytes = 0;
    int create = -1;     // op index of first write
    int last = -1;       // op index of last read
    bool pinned = false; // survives to the end of the call
    int64_t off = -1;
};

}  // namespace

int build_schedule(const Network &net, const Path &path, const std::vector<int> &sliced,
                   int batch_log2, int dtype, int small_log2, bool allow_tc, int fp8_min_log2_flops,
                   Schedule &S, std::string &err, const SampleSpec *spec) {
    S = Schedule();
    const int L = (int)net.leaves.size();
    const int NS = (int)path.steps.size();
    const int T = L + NS;
    const int E = (int)net.edges.size();
    if (L == 0) { err = "empty network"; return TN_EINVAL; }
    if (NS != L - 1) { err = "path does not merge every tensor"; return TN_EINVAL; }
    if (batch_log2 < 0 || batch_log2 > (int)sliced.size() || batch_log2 > 16) {
        err = "slice_batch_log2 must be in 0..min(16, n_slice_edges)";
        return TN_EINVAL;
    }
    std::vector<int> sbit(E, -1);
    for (int j = 0; j < (int)sliced.size(); ++j) sbit[sliced[j]] = j;
    // sample edges (uncorrelated bitstrings): batch modes of the tensors that
    // hold one row per sample, read out at the end as the amplitude index
    std::vector<char> is_sample(E, 0);
    if (spec)
        for (int e : spec->sample_edges) is_sample[e] = 1;
    // dense output legs (sample mode: a qubit's output leg before its tensor
    // switches to rows per sample)
    auto is_open = [&](int e) { return net.edges[e].open_t >= 0 && !is_sample[e]; };
    auto n_open_in = [&](const std::vector<int> &v) {
        int n = 0;
        for (int e : v) n += is_open(e);
        return n;
    };
    auto looped = [&](int e) { return sbit[e] >= batch_log2; };
    auto batched = [&](int e) { return (sbit[e] >= 0 && sbit[e] < batch_log2) || is_sample[e]; };
    // ---- leg orders, invariance, sets
    std::vector<std::vector<int>> legs(T), sets(T);
    std::vector<char> inv(T, 1);
    for (int l = 0; l < L; ++l) {
        for (int e : net.leaves[l].legs) {
            if (looped(e)) inv[l] = 0;
            else legs[l].push_back(e);
        }
        sets[l] = sorted_copy(legs[l]);
    }
    std::vector<int> consumer(T, -1);
    std::vector<char> samp(T, 0);   // sample mode: the tensor holds one row per sample
    for (int s = 0; s < NS; ++s) {
        const int a = path.steps[s].first, b = path.steps[s].second;
        if (a < 0 || b < 0 || a >= L + s || b >= L + s || a == b || consumer[a] >= 0 || consumer[b] >= 0) {
            err = "malformed path";
            return TN_EINVAL;
        }
        consumer[a] = consumer[b] = s;
        std::vector<int> sh, out;
        std::set_intersection(sets[a].begin(), sets[a].end(), sets[b].begin(), sets[b].end(),
                              std::back_inserter(sh));
        std::vector<int> un;
        std::set_union(sets[a].begin(), sets[a].end(), sets[b].begin(), sets[b].end(),
                       std::back_inserter(un));
        bool to_rows = false;
        if (spec) {
            const int oa = n_open_in(sets[a]), ob = n_open_in(sets[b]);
            to_rows = samp[a] || samp[b] || oa + ob > spec->k || (s == NS - 1 && oa + ob > 0);
        }
        samp[L + s] = to_rows;
        for (int e : un)
            if (!(std::binary_search(sh.begin(), sh.end(), e) && !batched(e)) && !(to_rows && is_open(e)))
                out.push_back(e);
        if (to_rows)
            for (int e : spec->sample_edges)
                if (!std::binary_search(out.begin(), out.end(), e)) out.insert(std::lower_bound(out.begin(), out.end(), e), e);
        sets[L + s] = out;
        inv[L + s] = inv[a] && inv[b];
    }
    const int final_t = NS > 0 ? T - 1 : 0;
    S.final_tensor = final_t;
    // storage of each tensor: complex64 for complex64 plans; in complex-half
    // plans, complex64 for leaves and tensors of <= 2^kSmallLog2 elements
    std::vector<int> tdt(T, 0);
    for (int t = 0; t < T; ++t)
        tdt[t] = (dtype != TN_C64 && t >= L && (int)sets[t].size() > small_log2) ? 1 : 0;
    auto esz_of = [&](int t) { return tdt[t] ? 4 : 8; };

    // role of each step: A = operand with more legs (ties: the first)
    auto a_side = [&](int s) {
        const int a = path.steps[s].first, b = path.steps[s].second;
        return sets[b].size() > sets[a].size() ? b : a;
    };
    // order `v` so that modes the consumer of tensor t batches come first and
    // modes it contracts come last (only when t is that step's large operand)
    auto for_consumer = [&](int t, std::vector<int> v) {
        const int c = consumer[t];
        if (c < 0 || a_side(c) != t) return v;
        const int p = path.steps[c].first == t ? path.steps[c].second : path.steps[c].first;
        auto key = [&](int e) {
            const bool sh = std::binary_search(sets[p].begin(), sets[p].end(), e);
            if (sh && batched(e)) return 0;
            if (sh) return 2;
            return 1;
        };
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return key(x) < key(y); });
        return v;
    };

    // ---- meta slots: invariant tensors first
    std::vector<int> meta(T, -1);
    int nm = 0;
    for (int t = 0; t < T; ++t)
        if (inv[t]) meta[t] = nm++;
    S.n_meta_inv = nm;
    for (int t = 0; t < T; ++t)
        if (!inv[t]) meta[t] = nm++;
    S.n_meta = nm;

    int n_extra_meta = 0;   // scale slots of complex64 B operands rounded for tensor cores

    // ---- ops with symbolic buffers: buffer id t for tensor t, temps after
    std::vector<BufReq> bufs(T);
    auto tensor_bytes = [&](int t) { return (int64_t)esz_of(t) << legs[t].size(); };
    std::vector<Op> ph[2];
    auto new_temp = [&](int64_t bytes) {
        BufReq r;
        r.bytes = bytes;
        bufs.push_back(r);
        return (int)bufs.size() - 1;
    };
    // leaf ops
    for (int phase = 0; phase < 2; ++phase) {
        Op op;
        op.kind = OP_LEAF;
        op.phase = phase;
        op.leaf_first = (int)S.leaf_jobs.size();
        for (int l = 0; l < L; ++l) {
            if ((inv[l] != 0) != (phase == 0)) continue;
            const Leaf &lf = net.leaves[l];
            LeafJob j{};
            const int rin = (int)lf.legs.size();
            if ((int)legs[l].size() > 31 || rin > 40) {
                err = "a leaf has too many legs";
                return TN_EINVAL;
            }
            j.rank_in = rin;
            j.rank_out = (int)legs[l].size();
            int nf = 0;
            for (int p = 0; p < rin; ++p) {
                const int e = lf.legs[p];
                if (looped(e)) {
                    j.fixed_pos[nf] = rin - 1 - p;
                    j.fixed_bit[nf] = sbit[e];
                    ++nf;
                }
            }
            j.n_fixed = nf;
            for (int i = 0; i < j.rank_out; ++i) {
                const int e = legs[l][j.rank_out - 1 - i];
                const int p = (int)(std::find(lf.legs.begin(), lf.legs.end(), e) - lf.legs.begin());
                j.keep_pos[i] = rin - 1 - p;
            }
            j.src = l;     // fixed up to an element offset by the caller
            j.dst = l;     // buffer id, replaced by its offset below
            j.meta = meta[l];
            bufs[l].bytes = tensor_bytes(l);
            S.leaf_jobs.push_back(j);
        }
        op.leaf_count = (int)S.leaf_jobs.size() - op.leaf_first;
        if (op.leaf_count > 0) ph[phase].push_back(op);
    }

    for (int s = 0; s < NS; ++s) {
        const int a0 = path.steps[s].first, b0 = path.steps[s].second;
        const int ia = a_side(s), ib = ia == a0 ? b0 : a0;
        const int c = L + s;
        const int phase = inv[c] ? 0 : 1;
        auto &ops = ph[phase];
        const std::vector<int> &LA = legs[ia], &LB = legs[ib];
        std::set<int> shared, bset, kset;
        for (int e : LA)
            if (contains(LB, e)) {
                shared.insert(e);
                if (batched(e)) bset.insert(e);
                else kset.insert(e);
            }
        const int nb = (int)bset.size(), nk = (int)kset.size();
        bool okA = true;
        for (int i = 0; i < nb; ++i) okA = okA && bset.count(LA[i]);
        for (int i = 0; i < nk; ++i) okA = okA && kset.count(LA[LA.size() - 1 - i]);
        std::vector<int> bo, mo, ko, no;
        if (okA) {
            bo.assign(LA.begin(), LA.begin() + nb);
            mo.assign(LA.begin() + nb, LA.end() - nk);
            ko.assign(LA.end() - nk, LA.end());
        } else {
            for (int e : LA) {
                if (bset.count(e)) bo.push_back(e);
                else if (kset.count(e)) ko.push_back(e);
                else mo.push_back(e);
            }
            mo = for_consumer(c, mo);
        }
        for (int e : LB)
            if (!shared.count(e)) no.push_back(e);
        no = for_consumer(c, no);

        // sparse-state gather step: C switches to (or stays in) one row per
        // sample while an operand still holds dense output legs.  Operand
        // roles: rows per sample (its batch dims: the sample edges), dense
        // outputs (batch dims: those legs, gathered by each sample's bits),
        // or neither (broadcast).
        enum { R_NONE = 0, R_ROWS = 1, R_GATHER = 2 };
        auto role = [&](int x) {
            if (samp[x]) return (int)R_ROWS;
            return (samp[c] && n_open_in(legs[x]) > 0) ? (int)R_GATHER : (int)R_NONE;
        };
        const bool gstep = spec && samp[c] && (role(ia) == R_GATHER || role(ib) == R_GATHER);
        std::vector<int> abat, bbat;
        int role_a = R_NONE, role_b = R_NONE;
        int nsb = 0;     // slices run together: shared batch modes outside the sample index
        if (gstep) {
            role_a = role(ia);
            role_b = role(ib);
            std::vector<int> sord;                       // sample bit k-1 outermost
            for (int j = spec->k - 1; j >= 0; --j) sord.push_back(spec->sample_edges[j]);
            auto bat_of = [&](int x, int r) {
                std::vector<int> v;
                if (r == R_ROWS) return sord;
                if (r == R_GATHER) {
                    for (int e : legs[x])
                        if (is_open(e)) v.push_back(e);
                    std::sort(v.begin(), v.end(), [&](int p, int q) { return net.edges[p].qubit < net.edges[q].qubit; });
                }
                return v;
            };
            // slice-batch modes both operands hold stay batch modes, outermost
            std::vector<int> sbs;
            for (int e : LA)
                if (shared.count(e) && batched(e) && !is_sample[e]) sbs.push_back(e);
            nsb = (int)sbs.size();
            abat = sbs;
            bbat = sbs;
            const std::vector<int> ga = bat_of(ia, role_a), gb = bat_of(ib, role_b);
            abat.insert(abat.end(), ga.begin(), ga.end());
            bbat.insert(bbat.end(), gb.begin(), gb.end());
            if (nsb + spec->k > 24) {
                err = "slices run together x samples exceed 2^24 rows";
                return TN_EINVAL;
            }
            bo = sbs;
            bo.insert(bo.end(), sord.begin(), sord.end());
            ko.clear();
            mo.clear();
            no.clear();
            for (int e : LA)
                if (!contains(abat, e) && shared.count(e) && !batched(e)) ko.push_back(e);
            for (int e : LA)
                if (!contains(abat, e) && !contains(ko, e)) mo.push_back(e);
            for (int e : LB)
                if (!contains(bbat, e) && !contains(ko, e)) no.push_back(e);
            std::vector<int> want(abat);
            want.insert(want.end(), mo.begin(), mo.end());
            want.insert(want.end(), ko.begin(), ko.end());
            okA = want == LA;
        }

        int meta_b_override = -1, meta_a_override = -1, fp8 = 0;
        StepRec rec{};
        rec.a = ia; rec.b = ib; rec.c = c;
        rec.lm = (int)mo.size(); rec.ln = (int)no.size(); rec.lk = gstep ? (int)ko.size() : nk;
        rec.lb = gstep ? nsb + spec->k : nb;
        rec.invariant = inv[c];

        int64_t abuf = ia, bbuf = ib;
        auto permute_to = [&](int src_t, const std::vector<int> &from, const std::vector<int> &to) {
            const int esz = esz_of(src_t);
            Op op;
            op.kind = OP_PERM;
            op.phase = phase;
            op.perm.esz = esz;
            op.perm.rank = (int)to.size();
            for (int i = 0; i < (int)to.size(); ++i)
                op.perm.perm[i] = (int)(std::find(from.begin(), from.end(), to[i]) - from.begin());
            const int tmp = new_temp((int64_t)esz << to.size());
            op.perm.src = src_t;
            op.perm.dst = tmp;
            ops.push_back(op);
            ++S.n_permutes;
            const double bytes = 2.0 * (double)((int64_t)esz << to.size());
            if (phase) S.bytes_per_pass += bytes;
            return tmp;
        };
        if (!okA) {
            std::vector<int> tgt(gstep ? abat : bo);
            tgt.insert(tgt.end(), mo.begin(), mo.end());
            tgt.insert(tgt.end(), ko.begin(), ko.end());
            abuf = permute_to(ia, LA, tgt);
            rec.permute_a = 1;
        }
        const int ta = tdt[ia], tb = tdt[ib], tc = tdt[c];
        rec.storage = ta | (tb << 1) | (tc << 2);
        int kernel;
        if (dtype == TN_C64) kernel = (rec.lm >= 6 && rec.ln >= 6 && rec.lk >= 4) ? GK_C64_TILED : GK_C64_ROWS;
        else kernel = (allow_tc && ta == 1 && rec.lk >= 3 && rec.lk <= 24 && rec.ln <= 24) ? GK_LP_TC : GK_LP_ROWS;
        rec.kernel = kernel;
        rec.tile = 0;
        if (kernel == GK_LP_TC) {
            // B goes straight from its stored order to the padded B' of
            // Eq. 6 ([batch][N][K] complex expanded to real rows) in one pass
            std::vector<int> tgt(gstep ? bbat : bo);
            tgt.insert(tgt.end(), no.begin(), no.end());
            tgt.insert(tgt.end(), ko.begin(), ko.end());
            const int blb = gstep ? (int)bbat.size() : rec.lb;    // B' chunks: 2^blb
            Op op;
            op.kind = OP_BPREP;
            op.phase = phase;
            const int np = std::max(16, 2 << rec.ln);
            op.bprep.src = bbuf;
            op.bprep.lk = rec.lk;
            op.bprep.ln = rec.ln;
            op.bprep.lb = blb;
            op.bprep.np = np;
            op.bprep.step = s;
            op.bprep.rank = (int)tgt.size();
            op.bprep.tb = tb;
            op.bprep.meta_src = meta[ib];
            op.bprep.meta_dst = meta[ib];
            if (tb == 0) {
                // complex64 B: B' = B 2^s gets a scale slot of its own
                op.bprep.meta_dst = S.n_meta + n_extra_meta++;
                meta_b_override = op.bprep.meta_dst;
            }
            for (int i = 0; i < (int)tgt.size(); ++i)
                op.bprep.perm[i] = (int)(std::find(LB.begin(), LB.end(), tgt[i]) - LB.begin());
            const int64_t bpbytes = ((int64_t)np * (2LL << rec.lk) * 2) << blb;
            const int tmp = new_temp(bpbytes);
            op.bprep.dst = tmp;
            ops.push_back(op);
            if (phase) S.bytes_per_pass += (double)(((int64_t)esz_of(ib) << (rec.lk + rec.ln + rec.lb)) + bpbytes);
            bbuf = tmp;
            // FP8 step: E4M3 copies of B' and A, each with its own scale slot
            if (!gstep && fp8_min_log2_flops > 0 && rec.lk >= 6 &&
                rec.lm + rec.ln + rec.lk + rec.lb + 3 >= fp8_min_log2_flops) {
                auto quant = [&](int64_t src, int64_t pairs, int meta_src) {
                    Op q;
                    q.kind = OP_QUANT;
                    q.phase = phase;
                    q.quant.src = src;
                    q.quant.n_pairs = pairs;
                    q.quant.meta_src = meta_src;
                    q.quant.meta_dst = S.n_meta + n_extra_meta++;
                    const int t = new_temp(2 * pairs);
                    q.quant.dst = t;
                    ops.push_back(q);
                    if (phase) S.bytes_per_pass += 6.0 * (double)pairs;
                    return std::make_pair(t, q.quant.meta_dst);
                };
                const auto qb = quant(bbuf, bpbytes / 4, op.bprep.meta_dst);
                bbuf = qb.first;
                meta_b_override = qb.second;
                const auto qa = quant(abuf, (int64_t)1 << (rec.lm + rec.lk + rec.lb), meta[ia]);
                abuf = qa.first;
                meta_a_override = qa.second;
                fp8 = 1;
                rec.storage |= 8;
            }
        } else {
            std::vector<int> tgt(gstep ? bbat : bo);
            tgt.insert(tgt.end(), ko.begin(), ko.end());
            tgt.insert(tgt.end(), no.begin(), no.end());
            if (tgt != LB) {
                bbuf = permute_to(ib, LB, tgt);
                rec.permute_b = 1;
            }
        }
        legs[c] = bo;
        legs[c].insert(legs[c].end(), mo.begin(), mo.end());
        legs[c].insert(legs[c].end(), no.begin(), no.end());
        bufs[c].bytes = tensor_bytes(c);
        Op op;
        op.kind = OP_GEMM;
        op.phase = phase;
        op.gemm.a = abuf;
        op.gemm.b = bbuf;
        op.gemm.c = c;
        op.gemm.lm = rec.lm; op.gemm.ln = rec.ln; op.gemm.lk = rec.lk; op.gemm.lb = rec.lb;
        op.gemm.a_batched = rec.lb > 0;
        op.gemm.b_batched = rec.lb > 0;
        op.gemm.meta_a = meta_a_override >= 0 ? meta_a_override : meta[ia];
        op.gemm.meta_b = meta_b_override >= 0 ? meta_b_override : meta[ib];
        op.gemm.meta_c = meta[c];
        op.gemm.step = s;
        op.gemm.kernel = kernel;
        // the fixed heuristic's tile (1-CTA); CTA pairs are an autotuner
        // candidate: they lose on some long-K steps
        op.gemm.tile = 0;
        op.gemm.ta = ta;
        op.gemm.tb = tb;
        op.gemm.tc = tc;
        op.gemm.fp8 = fp8;
        if (gstep) {
            // per operand: rows per sample (chunk z), gathered (chunk = the
            // slice-batch index, then the sample's bits on its output legs,
            // outermost first), or broadcast over the samples (chunk = the
            // slice-batch index; no table without one).  Output batch entry
            // z = slice-batch index x 2^k + sample.
            auto gather_table = [&](const std::vector<int> &gat) {
                const int64_t off = (int64_t)S.gidx.size();
                const int m = (int)gat.size();
                for (int64_t zs = 0; zs < ((int64_t)1 << nsb); ++zs)
                    for (uint64_t bits : spec->bits) {
                        int64_t z = zs << m;
                        for (int i = 0; i < m; ++i)
                            z |= (int64_t)((bits >> net.edges[gat[i]].qubit) & 1) << (m - 1 - i);
                        S.gidx.push_back((int32_t)z);
                    }
                return off;
            };
            auto setup = [&](int r, const std::vector<int> &bat, int64_t &idx, int32_t &glog2,
                             int32_t &is_batched, int32_t &bcast) {
                is_batched = 1;
                bcast = 0;
                if (r == R_ROWS) return;
                if (r == R_NONE && nsb == 0) {
                    is_batched = 0;
                    bcast = 1;
                    return;
                }
                idx = gather_table(std::vector<int>(bat.begin() + nsb, bat.end()));
                glog2 = (int)bat.size();
            };
            setup(role_a, abat, op.gemm.idx_a, op.gemm.gather_a_log2, op.gemm.a_batched, op.gemm.bcast_a);
            setup(role_b, bbat, op.gemm.idx_b, op.gemm.gather_b_log2, op.gemm.b_batched, op.gemm.bcast_b);
        }
        ops.push_back(op);
        ++S.n_gemm_steps;
        const double fl = 8.0 * std::ldexp(1.0, rec.lm + rec.ln + rec.lk + rec.lb);
        const double by = (double)(((int64_t)esz_of(ia) << (rec.lm + rec.lk + rec.lb)) +
                                   ((int64_t)esz_of(ib) << (rec.lk + rec.ln + rec.lb)) +
                                   ((int64_t)esz_of(c) << (rec.lm + rec.ln + rec.lb)));
        if (phase) { S.flops_per_pass += fl; S.bytes_per_pass += by; }
        else { S.flops_inv += fl; ++S.n_steps_inv; }
        S.steps.push_back(rec);
    }
    // final sum
    {
        Op op;
        op.kind = OP_SUM;
        op.phase = 1;
        const auto &F = legs[final_t];
        const int r = (int)F.size();
        op.sum.src = final_t;
        op.sum.rank = r;
        op.sum.meta = meta[final_t];
        for (int p = 0; p < r; ++p) {
            const Edge &ed = net.edges[F[p]];
            if (ed.open_t >= 0) op.sum.open_pos[ed.open_t] = r - 1 - p;
            else if (batched(F[p])) op.sum.batch_pos[sbit[F[p]]] = r - 1 - p;
            else { err = "final tensor has a non-output mode"; return TN_EINVAL; }
        }
        // recomputation: open outputs sliced (looped) are fixed per pass
        op.sum.n_split = 0;
        for (int j = 0; j < (int)sliced.size(); ++j) {
            const Edge &ed = net.edges[sliced[j]];
            if (ed.open_t < 0) continue;
            if (j < batch_log2 || op.sum.n_split >= 8) {
                err = "an open leg can be split only outside the slice batch (at most 8)";
                return TN_EINVAL;
            }
            op.sum.split_t[op.sum.n_split] = ed.open_t;
            op.sum.split_bit[op.sum.n_split] = j;
            ++op.sum.n_split;
        }
        if (r != net.n_open - op.sum.n_split + batch_log2) {
            err = "final tensor misses output modes";
            return TN_EINVAL;
        }
        op.sum.n_batch = batch_log2;
        op.sum.tf = tdt[final_t];
        ph[1].push_back(op);
    }

    S.n_meta_extra = n_extra_meta;

    // ---- a permutation of a tensor-core GEMM's result (its only reader) is
    // written by that GEMM's epilogue instead: each thread holds 8
    // consecutive complex values of one row of C (C must hold >= 8 columns)
    // and a warp 32 consecutive rows
    for (auto &ops_p : ph) {
        std::vector<int> readers;
        auto count_reads = [&](int64_t id) {
            int n = 0;
            for (const auto &pv : ph)
                for (const Op &o : pv) {
                    if (o.kind == OP_PERM && o.perm.src == id) ++n;
                    if (o.kind == OP_BPREP && o.bprep.src == id) ++n;
                    if (o.kind == OP_QUANT && o.quant.src == id) ++n;
                    if (o.kind == OP_SUM && o.sum.src == id) ++n;
                    if (o.kind == OP_GEMM && (o.gemm.a == id || o.gemm.b == id)) ++n;
                }
            return n;
        };
        for (size_t i = 1; i < ops_p.size(); ++i) {
            Op &pm = ops_p[i];
            if (pm.kind != OP_PERM) continue;
            size_t gi = i;                       // the op that made the permuted tensor
            while (gi > 0 && !(ops_p[gi - 1].kind == OP_GEMM && ops_p[gi - 1].gemm.c == pm.perm.src)) --gi;
            if (gi == 0) continue;
            Op &g = ops_p[gi - 1];
            if (g.gemm.kernel != GK_LP_TC || g.gemm.ln < 3) continue;
            const int r = pm.perm.rank;
            if (r != g.gemm.lb + g.gemm.lm + g.gemm.ln || r < 3) continue;
            // the destination's lowest 3 bits must come from the 8 columns a
            // thread holds or from the 32 rows of a warp, so that a warp's
            // stores still fill whole 32-byte sectors
            bool coalesced = true;
            for (int k = r - 3; k < r; ++k) {
                const int src = r - 1 - pm.perm.perm[k];      // source bit of destination bit r-1-k
                const bool thread_col = src < 3;
                const bool warp_row = src >= g.gemm.ln && src < g.gemm.ln + std::min(5, g.gemm.lm);
                coalesced = coalesced && (thread_col || warp_row);
            }
            if (!coalesced) continue;
            if (g.gemm.lk > kSplitLog2KHost ||
                tc_split(g.gemm.lm, g.gemm.ln, g.gemm.lk, (int64_t)1 << g.gemm.lb) != 1)
                continue;
            if (count_reads(g.gemm.c) != 1) continue;
            g.gemm.out_rank = r;
            for (int k = 0; k < r; ++k) g.gemm.out_dpos[r - 1 - pm.perm.perm[k]] = (int8_t)(r - 1 - k);
            g.gemm.c = pm.perm.dst;
            --S.n_permutes;
            if (pm.phase) S.bytes_per_pass -= 2.0 * (double)((int64_t)pm.perm.esz << r);
            ops_p.erase(ops_p.begin() + (long)i);
            --i;
        }
    }

    // ---- lifetimes over the op sequence (phase 0 then phase 1)
    S.ops = ph[0];
    S.ops.insert(S.ops.end(), ph[1].begin(), ph[1].end());
    const int n_ops = (int)S.ops.size();
    auto touch_create = [&](int64_t id, int i) {
        if (bufs[id].create < 0) bufs[id].create = i;
    };
    auto touch_read = [&](int64_t id, int i) {
        bufs[id].last = std::max(bufs[id].last, i);
        if (S.ops[i].phase == 1 && bufs[id].create >= 0 && S.ops[bufs[id].create].phase == 0)
            bufs[id].pinned = true;
    };
    for (int i = 0; i < n_ops; ++i) {
        const Op &op = S.ops[i];
        switch (op.kind) {
            case OP_LEAF:
                for (int k = 0; k < op.leaf_count; ++k) touch_create(S.leaf_jobs[op.leaf_first + k].dst, i);
                break;
            case OP_PERM: touch_read(op.perm.src, i); touch_create(op.perm.dst, i); break;
            case OP_BPREP: touch_read(op.bprep.src, i); touch_create(op.bprep.dst, i); break;
            case OP_QUANT: touch_read(op.quant.src, i); touch_create(op.quant.dst, i); break;
            case OP_GEMM:
                touch_read(op.gemm.a, i); touch_read(op.gemm.b, i); touch_create(op.gemm.c, i);
                break;
            case OP_SUM: touch_read(op.sum.src, i); break;
        }
    }
    Arena arena;
    std::vector<std::vector<int>> created_at(n_ops), freed_at(n_ops);
    for (int id = 0; id < (int)bufs.size(); ++id) {
        if (bufs[id].create < 0) continue;
        created_at[bufs[id].create].push_back(id);
        if (!bufs[id].pinned) freed_at[std::max(bufs[id].last, bufs[id].create)].push_back(id);
    }
    for (int i = 0; i < n_ops; ++i) {
        for (int id : created_at[i]) bufs[id].off = arena.alloc(bufs[id].bytes);
        for (int id : freed_at[i]) arena.release(bufs[id].off, bufs[id].bytes);
    }
    S.ws_bytes = std::max<int64_t>(arena.top, 1024);
    auto off = [&](int64_t id) { return bufs[id].off; };
    for (LeafJob &j : S.leaf_jobs) j.dst = off(j.dst);
    for (Op &op : S.ops) {
        switch (op.kind) {
            case OP_PERM: op.perm.src = off(op.perm.src); op.perm.dst = off(op.perm.dst); break;
            case OP_BPREP: op.bprep.src = off(op.bprep.src); op.bprep.dst = off(op.bprep.dst); break;
            case OP_QUANT: op.quant.src = off(op.quant.src); op.quant.dst = off(op.quant.dst); break;
            case OP_GEMM:
                op.gemm.a = off(op.gemm.a); op.gemm.b = off(op.gemm.b); op.gemm.c = off(op.gemm.c);
                break;
            case OP_SUM: op.sum.src = off(op.sum.src); break;
            default: break;
        }
        if (op.phase == 1) ++S.kernels_per_pass;
        else ++S.kernels_inv;
    }
    return TN_OK;
}

}  // namespace tn

// Contraction-tree refinement by simulated annealing (paper Sec. 3: the path
// is searched by simulated annealing under a memory cap, taking the lowest
// time complexity per cap).
//
// The path is read as a binary tree whose leaves are the network's tensors
// (sliced edges removed).  A move rotates one internal node X = (P, (Q1, Q2))
// into ((P, Q1), Q2) or ((P, Q2), Q1): only the inner node's legs change, so
// the cost difference is local (two steps).  The objective is a step time in
// flop units: 8 2^(|A|+|B|-|A&B|) flops plus kappa (2^|A| + 2^|B| + 2^|C|)
// for the elements the step moves through HBM (kappa = bytes per element x
// the GPU's flop-per-byte ridge), so that a cheap-in-flops but huge-in-bytes
// order does not win.  The library runs the slices of a pass as one batch,
// each tensor carrying as batch modes only the sliced edges below it, and a
// step that no looped sliced edge reaches runs once per call: a step's cost
// is weighted by how many times it really runs (slice_weight), so the search
// may move work to where fewer slices reach it.
// A move whose new intermediate would exceed the width cap is rejected; a
// worse move is accepted with probability exp(-d / T), d the change of
// log2(cost), T falling geometrically.  The best tree seen is returned as a
// post-order path.
#include <algorithm>
#include <array>
#include <cmath>
#include <exception>
#include <functional>
#include <random>
#include <system_error>
#include <thread>

#include "internal.h"
#include "plan.h"

namespace tn {

namespace {

int shared_count(const std::vector<int> &a, const std::vector<int> &b) {
    int n = 0;
    size_t i = 0, j = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] == b[j]) { ++n; ++i; ++j; }
        else if (a[i] < b[j]) ++i;
        else ++j;
    }
    return n;
}

std::vector<int> sym_diff(const std::vector<int> &a, const std::vector<int> &b) {
    std::vector<int> out;
    std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
    return out;
}

// Weight of a step against its per-slice cost, for a call that contracts
// all 2^S slices, 2^b per pass (sliced edges 0..b-1 batched, the others
// looped over passes; m: the sliced edges below the step).  Its tensors carry
// as batch modes only the batched edges below it, so a pass runs it
// 2^|m & batch| times; it runs in every pass if a looped edge reaches it,
// else once per call.  Relative to 2^S per-slice runs:
// 2^(|m & batch| - b) x (looped edge below ? 1 : 2^(b - S)).  b < 0: no
// weighting (every step once per slice).
double slice_weight(uint64_t m, int S, int b) {
    if (b < 0) return 1.0;     // every step counted once per slice
    S = std::min(S, 64);
    b = std::min(b, S);
    const uint64_t batch = b >= 64 ? ~0ull : ((1ull << b) - 1);
    const int e = __builtin_popcountll(m & batch) - b + ((m & ~batch) ? 0 : b - S);
    return std::ldexp(1.0, e);
}

struct Tree {
    int L = 0;                                  // leaves 0..L-1, internal L..2L-2
    std::vector<std::array<int, 2>> kid;        // children of internal nodes (index - L)
    std::vector<int> parent;                    // parent of every node (-1: root)
    std::vector<std::vector<int>> legs;         // open legs of every node
    int root = -1;

    std::vector<uint64_t> smask;                // sliced edges (bit j: edge j of the list) below a node

    double kappa = 0;
    int S = 0;                                  // sliced edges
    int B = 0;                                  // of them batched in a pass

    double step_cost(int x) const {
        const auto &k = kid[x - L];
        return cost_of(legs[k[0]], legs[k[1]], legs[x], smask[x]);
    }
    double cost_of(const std::vector<int> &a, const std::vector<int> &b, const std::vector<int> &c,
                   uint64_t m) const {
        return (8.0 * std::ldexp(1.0, (int)(a.size() + b.size()) - shared_count(a, b)) +
                kappa * (std::ldexp(1.0, (int)a.size()) + std::ldexp(1.0, (int)b.size()) +
                         std::ldexp(1.0, (int)c.size()))) *
               slice_weight(m, S, B);
    }
};

}  // namespace

int anneal_path(const Network &net, const std::vector<int> &sliced, int width_cap, uint64_t seed,
                int iters, double kappa, int batch_log2, Path &path) {
    const int L = (int)net.leaves.size();
    if (L < 3 || iters <= 0 || (int)path.steps.size() != L - 1) return TN_OK;
    std::vector<int> slot(net.edges.size(), -1);
    for (int j = 0; j < (int)sliced.size(); ++j) slot[sliced[j]] = j;
    Tree t;
    t.L = L;
    t.kappa = kappa;
    t.S = (int)sliced.size();
    t.B = batch_log2;
    t.legs.resize(2 * L - 1);
    t.parent.assign(2 * L - 1, -1);
    t.kid.resize(L - 1);
    t.smask.assign(2 * L - 1, 0);
    for (int i = 0; i < L; ++i) {
        for (int e : net.leaves[i].legs) {
            if (slot[e] < 0) t.legs[i].push_back(e);
            else if (slot[e] < 64) t.smask[i] |= 1ull << slot[e];
        }
        std::sort(t.legs[i].begin(), t.legs[i].end());
    }
    int width = 0;
    for (int i = 0; i < L; ++i) width = std::max(width, (int)t.legs[i].size());
    double total = 0;
    for (int s = 0; s < L - 1; ++s) {
        const int x = L + s, a = path.steps[s].first, b = path.steps[s].second;
        t.kid[s] = {a, b};
        t.parent[a] = t.parent[b] = x;
        t.legs[x] = sym_diff(t.legs[a], t.legs[b]);
        t.smask[x] = t.smask[a] | t.smask[b];
        width = std::max(width, (int)t.legs[x].size());
        total += t.step_cost(x);
    }
    t.root = 2 * L - 2;
    const int cap = std::max(width_cap, width);
    const double start_total = total;

    std::mt19937_64 rng(seed);
    std::uniform_int_distribution<int> pick_node(L, 2 * L - 2);
    std::uniform_real_distribution<double> unif(0.0, 1.0);
    const double T0 = 0.02, T1 = 1e-4;
    double best_total = total;
    std::vector<std::array<int, 2>> best_kid = t.kid;
    for (int it = 0; it < iters; ++it) {
        const double T = T0 * std::pow(T1 / T0, (double)it / iters);
        const int x = pick_node(rng);
        const auto kx = t.kid[x - L];
        // an internal child Q of X to rotate through; P is the other child
        int qi = (int)(rng() & 1);
        if (kx[qi] < L) qi ^= 1;
        const int q = kx[qi], p = kx[qi ^ 1];
        if (q < L) continue;
        const int keep = (int)(rng() & 1);          // Q's child that joins P
        const int q1 = t.kid[q - L][keep], q2 = t.kid[q - L][keep ^ 1];
        std::vector<int> nq = sym_diff(t.legs[p], t.legs[q1]);
        if ((int)nq.size() > cap) continue;
        const uint64_t dq = t.smask[p] | t.smask[q1];
        const double old_f = t.step_cost(x) + t.step_cost(q);
        const double f_q = t.cost_of(t.legs[p], t.legs[q1], nq, dq);
        const double f_x = t.cost_of(nq, t.legs[q2], t.legs[x], t.smask[x]);
        const double nt = total - old_f + f_q + f_x;
        const double d = std::log2(nt) - std::log2(total);
        if (d > 0 && unif(rng) >= std::exp(-d / T)) continue;
        // apply: Q = (P, Q1), X = (Q, Q2)
        t.kid[q - L] = {p, q1};
        t.kid[x - L] = {q, q2};
        t.parent[p] = q;
        t.parent[q1] = q;
        t.parent[q] = x;
        t.parent[q2] = x;
        t.legs[q] = std::move(nq);
        t.smask[q] = dq;
        total = nt;
        if (total < best_total * (1.0 - 1e-12)) {
            best_total = total;
            best_kid = t.kid;
        }
    }
    if (!(best_total < start_total * (1.0 - 1e-9))) return TN_OK;   // no gain: keep the input
    // post-order emission of the best tree; leaves keep their ids
    std::vector<int> id(2 * L - 1, -1);
    for (int i = 0; i < L; ++i) id[i] = i;
    Path out;
    std::vector<std::pair<int, int>> stack = {{t.root, 0}};
    while (!stack.empty()) {
        auto &top = stack.back();
        const int n = top.first;
        if (n < L) { stack.pop_back(); continue; }
        const auto &k = best_kid[n - L];
        if (top.second < 2) {
            const int c = k[top.second++];
            if (c >= L && id[c] < 0) stack.push_back({c, 0});
            continue;
        }
        id[n] = L + (int)out.steps.size();
        out.steps.push_back({id[k[0]], id[k[1]]});
        stack.pop_back();
    }
    if ((int)out.steps.size() != L - 1) return TN_OK;     // defensive: keep the input path
    out.flops = 0;                      // the caller measures flops and width
    out.max_log2 = path.max_log2;
    path = std::move(out);
    return TN_OK;
}

// Per-slice flops, cost (steps weighted by slice_weight) and largest
// intermediate of `path` with `sliced` removed.
static void measure(const Network &net, const std::vector<int> &sliced, const Path &path, double kappa,
                    int batch_log2, int &max_log2, double &flops, double &cost, double *roof = nullptr) {
    std::vector<int> slot(net.edges.size(), -1);
    for (int j = 0; j < (int)sliced.size(); ++j) slot[sliced[j]] = j;
    const int S = (int)sliced.size();
    std::vector<std::vector<int>> legs;
    std::vector<uint64_t> mask;
    max_log2 = 0;
    for (const Leaf &lf : net.leaves) {
        std::vector<int> k;
        uint64_t m = 0;
        for (int e : lf.legs) {
            if (slot[e] < 0) k.push_back(e);
            else if (slot[e] < 64) m |= 1ull << slot[e];
        }
        std::sort(k.begin(), k.end());
        max_log2 = std::max(max_log2, (int)k.size());
        legs.push_back(std::move(k));
        mask.push_back(m);
    }
    flops = 0;
    cost = 0;
    if (roof) *roof = 0;
    for (const auto &st : path.steps) {
        const auto &a = legs[st.first], &b = legs[st.second];
        const double f = 8.0 * std::ldexp(1.0, (int)(a.size() + b.size()) - shared_count(a, b));
        flops += f;
        std::vector<int> c = sym_diff(a, b);
        const uint64_t m = mask[st.first] | mask[st.second];
        const double mv = kappa * (std::ldexp(1.0, (int)a.size()) + std::ldexp(1.0, (int)b.size()) +
                                   std::ldexp(1.0, (int)c.size()));
        const double w = slice_weight(m, S, batch_log2);
        cost += (f + mv) * w;
        // roofline time of the step (flop units): tensor work or traffic,
        // whichever is larger
        if (roof) *roof += std::max(f, mv) * w;
        max_log2 = std::max(max_log2, (int)c.size());
        legs.push_back(std::move(c));
        mask.push_back(m);
    }
}

// One annealing chain of 3 rounds from (path, sliced); returns its job's
// roofline cost (2^S x the weighted per-slice cost: all slices in one call,
// 2^batch_log2 per pass).
static double refine_chain(const Network &net, int n_target, int cap, uint64_t seed, int iters, double kappa,
                           int batch_log2, Path &path, std::vector<int> &sliced) {
    int mx;
    double fl, co;
    measure(net, sliced, path, kappa, batch_log2, mx, fl, co);
    const int width_cap = cap > 0 ? cap : mx;
    for (int round = 0; round < 3; ++round) {
        anneal_path(net, sliced, width_cap, seed + 0x5851F42D4C957F2Dull * (uint64_t)(round + 1), iters,
                    kappa, batch_log2, path);
        measure(net, sliced, path, kappa, batch_log2, mx, fl, co);
        if (n_target >= 0 || cap <= 0) continue;
        // fewer slices where the refined tree leaves room under the cap: the
        // job's cost is 2^S x the per-slice cost
        for (int j = (int)sliced.size() - 1; j >= 0; --j) {
            std::vector<int> trial(sliced);
            trial.erase(trial.begin() + j);
            int m2;
            double f2, c2;
            measure(net, trial, path, kappa, batch_log2, m2, f2, c2);
            if (m2 <= cap && c2 < 2.0 * co) {
                sliced.swap(trial);
                mx = m2;
                fl = f2;
                co = c2;
            }
        }
    }
    path.max_log2 = mx;
    path.flops = fl;
    // the chains are compared on the roofline form of the cost (a step takes
    // max(flops, traffic), not their sum): the sum steers the search better,
    // the maximum ranks finished paths closer to their measured times
    double roof = 0;
    measure(net, sliced, path, kappa, batch_log2, mx, fl, co, &roof);
    return std::ldexp(roof, (int)sliced.size());
}

void run_parallel(int n, const std::function<void(int)> &fn) {
    std::vector<std::exception_ptr> err(std::max(0, n));
    auto body = [&](int i) {
        try {
            fn(i);
        } catch (...) {
            err[i] = std::current_exception();
        }
    };
    std::vector<std::thread> th;
    th.reserve(std::max(0, n));  // no reallocation (and no throw) once threads run
    int spawned = 0;
    if (std::thread::hardware_concurrency() > 1) {
        for (int i = 1; i < n; ++i) {
            try {
                th.emplace_back(body, i);
                ++spawned;
            } catch (const std::system_error &) {
                break;  // no more threads: the rest run on this one
            }
        }
    }
    if (n > 0) body(0);
    for (int i = spawned + 1; i < n; ++i) body(i);
    for (auto &t : th) t.join();
    for (auto &e : err)
        if (e) std::rethrow_exception(e);
}

int refine_plan(const Network &net, int n_target, int cap, uint64_t seed, int iters, double kappa,
                int batch_log2, int chains, Path &path, std::vector<int> &sliced, double *cost_out) {
    // independent chains from the same start, one thread each; the cheapest
    // job wins (the lowest time complexity found under the cap), ties to the
    // lower chain index, so the result does not depend on the threads
    const int nc = std::max(1, chains);
    std::vector<Path> ps(nc, path);
    std::vector<std::vector<int>> ss(nc, sliced);
    std::vector<double> cost(nc, 0.0);
    run_parallel(nc, [&](int c) {
        cost[c] = refine_chain(net, n_target, cap, seed + 0x9E3779B97F4A7C15ull * (uint64_t)c, iters, kappa,
                               batch_log2, ps[c], ss[c]);
    });
    int best = 0;
    for (int c = 1; c < nc; ++c)
        if (cost[c] < cost[best]) best = c;
    path = std::move(ps[best]);
    sliced = std::move(ss[best]);
    if (cost_out) *cost_out = cost[best];
    return TN_OK;
}

}  // namespace tn

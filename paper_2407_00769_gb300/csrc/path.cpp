// Contraction path and slicing (paper Sec. 3, Innovations: the path search and
// edge breaking follow Pan et al.; Sec. 3.1: sub-networks from fixed edges).
//
// Path: greedy pairwise order -- repeatedly contract the pair of tensors that
// share an edge whose result grows the total size least (size(C) - size(A) -
// size(B)); trial 0 is deterministic, later trials add seeded noise to the
// score and the best (largest intermediate, then flops) is kept.  Tensors left
// without shared edges are then merged smallest first (outer products).
//
// Slicing: edges are chosen one at a time among the legs of the largest
// intermediates, each time the edge whose removal gives the smallest
// (largest intermediate, flops per slice); after each choice the greedy path
// is searched again on the sliced network and kept if better.
#include <algorithm>
#include <array>
#include <cmath>
#include <random>
#include <set>

#include "internal.h"

namespace tn {

namespace {

std::vector<int> symdiff(const std::vector<int> &a, const std::vector<int> &b) {
    std::vector<int> out;
    std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
    return out;
}

int count_shared(const std::vector<int> &a, const std::vector<int> &b) {
    int n = 0;
    size_t i = 0, j = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] == b[j]) { ++n; ++i; ++j; }
        else if (a[i] < b[j]) ++i;
        else ++j;
    }
    return n;
}

}  // namespace

// leaf_legs: sorted leg sets (sliced edges already removed).  Every edge is in
// at most two tensors.
Path greedy_path(const std::vector<std::vector<int>> &leaf_legs, int n_edges, uint64_t seed,
                 double noise) {
    const int L = (int)leaf_legs.size();
    std::vector<std::vector<int>> legs(leaf_legs);
    std::vector<char> alive(L, 1);
    std::vector<std::array<int, 2>> owner(n_edges, {-1, -1});
    for (int t = 0; t < L; ++t)
        for (int e : legs[t]) {
            if (owner[e][0] < 0) owner[e][0] = t;
            else owner[e][1] = t;
        }
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> gauss(0.0, 1.0);
    Path p;
    auto size_of = [](size_t r) { return std::ldexp(1.0, (int)r); };
    int n_alive = L;
    while (n_alive > 1) {
        int best_a = -1, best_b = -1;
        double best_key = 0;
        int best_rc = 0;
        for (int e = 0; e < n_edges; ++e) {
            int a = owner[e][0], b = owner[e][1];
            if (a < 0 || b < 0) continue;
            if (a > b) std::swap(a, b);
            const int sh = count_shared(legs[a], legs[b]);
            const int rc = (int)legs[a].size() + (int)legs[b].size() - 2 * sh;
            double key = size_of(rc) - size_of(legs[a].size()) - size_of(legs[b].size());
            if (noise > 0) {
                const double f = std::exp(noise * gauss(rng));
                key = key > 0 ? key * f : key / f;
            }
            const bool better = best_a < 0 || key < best_key ||
                                (key == best_key && (rc < best_rc || (rc == best_rc &&
                                 std::make_pair(a, b) < std::make_pair(best_a, best_b))));
            if (better) { best_a = a; best_b = b; best_key = key; best_rc = rc; }
        }
        if (best_a < 0) {
            // no shared edges left: merge the two smallest tensors
            int s1 = -1, s2 = -1;
            for (int t = 0; t < (int)legs.size(); ++t) {
                if (!alive[t]) continue;
                auto smaller = [&](int x, int y) {
                    return legs[x].size() < legs[y].size() ||
                           (legs[x].size() == legs[y].size() && x < y);
                };
                if (s1 < 0 || smaller(t, s1)) { s2 = s1; s1 = t; }
                else if (s2 < 0 || smaller(t, s2)) s2 = t;
            }
            best_a = std::min(s1, s2);
            best_b = std::max(s1, s2);
        }
        const int c = (int)legs.size();
        std::vector<int> lc = symdiff(legs[best_a], legs[best_b]);
        p.flops += 8.0 * std::ldexp(1.0, (int)(legs[best_a].size() + legs[best_b].size() -
                                               count_shared(legs[best_a], legs[best_b])));
        p.max_log2 = std::max(p.max_log2, (int)lc.size());
        std::vector<std::pair<int, int>> keep;  // (edge, its other owner)
        for (int e : lc) {
            const int self = std::binary_search(legs[best_a].begin(), legs[best_a].end(), e) ? best_a : best_b;
            keep.push_back({e, owner[e][0] == self ? owner[e][1] : owner[e][0]});
        }
        for (int e : legs[best_a]) owner[e] = {-1, -1};
        for (int e : legs[best_b]) owner[e] = {-1, -1};
        for (const auto &k : keep) owner[k.first] = {c, k.second};
        legs.push_back(lc);
        alive.push_back(1);
        alive[best_a] = alive[best_b] = 0;
        p.steps.push_back({best_a, best_b});
        --n_alive;
    }
    for (const auto &l : leaf_legs) p.max_log2 = std::max(p.max_log2, (int)l.size());
    return p;
}

// Replay a path with some edges removed: largest intermediate and flops.
void replay(const std::vector<std::vector<int>> &leaf_legs, const Path &p,
            const std::vector<char> &removed, int &max_log2, double &flops,
            std::vector<std::vector<int>> *inter) {
    std::vector<std::vector<int>> legs;
    legs.reserve(leaf_legs.size() + p.steps.size());
    max_log2 = 0;
    for (const auto &l : leaf_legs) {
        std::vector<int> k;
        for (int e : l)
            if (!removed[e]) k.push_back(e);
        max_log2 = std::max(max_log2, (int)k.size());
        legs.push_back(std::move(k));
    }
    flops = 0;
    for (const auto &st : p.steps) {
        const auto &a = legs[st.first];
        const auto &b = legs[st.second];
        const int sh = count_shared(a, b);
        flops += 8.0 * std::ldexp(1.0, (int)(a.size() + b.size() - sh));
        std::vector<int> c = symdiff(a, b);
        max_log2 = std::max(max_log2, (int)c.size());
        legs.push_back(std::move(c));
    }
    if (inter) *inter = std::move(legs);
}

static std::vector<std::vector<int>> sliced_leaf_legs(const Network &net, const std::vector<char> &removed) {
    std::vector<std::vector<int>> out;
    for (const Leaf &L : net.leaves) {
        std::vector<int> k;
        for (int e : L.legs)
            if (!removed[e]) k.push_back(e);
        std::sort(k.begin(), k.end());
        out.push_back(std::move(k));
    }
    return out;
}

Path best_greedy(const Network &net, const std::vector<char> &removed, uint64_t seed, int trials) {
    const auto ll = sliced_leaf_legs(net, removed);
    Path best;
    bool have = false;
    for (int t = 0; t < std::max(1, trials); ++t) {
        Path p = greedy_path(ll, (int)net.edges.size(), seed + 0x9E3779B97F4A7C15ull * (uint64_t)t,
                             t == 0 ? 0.0 : 0.6);
        if (!have || p.max_log2 < best.max_log2 ||
            (p.max_log2 == best.max_log2 && p.flops < best.flops)) {
            best = std::move(p);
            have = true;
        }
    }
    return best;
}

// Choose sliced edges.  n_target >= 0: exactly that many; else until the
// largest intermediate is <= cap (cap <= 0: none).  Returns TN_OK or TN_EINVAL.
int choose_slices(const Network &net, uint64_t seed, int trials, int n_target, int cap,
                  Path &path, std::vector<int> &sliced, std::string &err) {
    const int E = (int)net.edges.size();
    std::vector<char> removed(E, 0);
    sliced.clear();
    path = best_greedy(net, removed, seed, trials);
    std::vector<std::vector<int>> ll_full;
    for (const Leaf &L : net.leaves) {
        std::vector<int> k(L.legs);
        std::sort(k.begin(), k.end());
        ll_full.push_back(std::move(k));
    }
    auto need_more = [&](int cur_max) {
        if (n_target >= 0) return (int)sliced.size() < n_target;
        return cap > 0 && cur_max > cap;
    };
    int cur_max = path.max_log2;
    while (need_more(cur_max)) {
        std::vector<std::vector<int>> inter;
        int mx;
        double fl;
        replay(ll_full, path, removed, mx, fl, &inter);
        std::set<int> cand;
        for (const auto &t : inter)
            if ((int)t.size() >= mx - 1)
                for (int e : t)
                    if (net.edges[e].v >= 0 && !removed[e]) cand.insert(e);
        if (cand.empty()) {
            for (int e = 0; e < E; ++e)
                if (net.edges[e].v >= 0 && !removed[e]) cand.insert(e);
        }
        if (cand.empty()) {
            err = "no edge left to slice";
            return TN_EINVAL;
        }
        int best_e = -1, best_mx = 0;
        double best_fl = 0;
        for (int e : cand) {
            removed[e] = 1;
            int m2;
            double f2;
            replay(ll_full, path, removed, m2, f2, nullptr);
            removed[e] = 0;
            if (best_e < 0 || m2 < best_mx || (m2 == best_mx && f2 < best_fl)) {
                best_e = e; best_mx = m2; best_fl = f2;
            }
        }
        removed[best_e] = 1;
        sliced.push_back(best_e);
        Path p2 = best_greedy(net, removed, seed + 7919u * (uint64_t)sliced.size(), trials);
        int m3;
        double f3;
        replay(ll_full, path, removed, m3, f3, nullptr);
        if (p2.max_log2 < m3 || (p2.max_log2 == m3 && p2.flops < f3)) {
            path = std::move(p2);
            cur_max = path.max_log2;
        } else {
            path.max_log2 = m3;
            path.flops = f3;
            cur_max = m3;
        }
    }
    // final numbers of the chosen path on the sliced network
    int mx;
    double fl;
    replay(ll_full, path, removed, mx, fl, nullptr);
    path.max_log2 = mx;
    path.flops = fl;
    return TN_OK;
}

int choose_recompute(const Network &net, int r, Path &path, std::vector<int> &sliced, std::string &err) {
    const int E = (int)net.edges.size();
    std::vector<char> removed(E, 0);
    for (int e : sliced) removed[e] = 1;
    std::vector<std::vector<int>> ll_full;
    for (const Leaf &L : net.leaves) {
        std::vector<int> k(L.legs);
        std::sort(k.begin(), k.end());
        ll_full.push_back(std::move(k));
    }
    for (int i = 0; i < r; ++i) {
        int best_e = -1, best_mx = 0;
        double best_fl = 0;
        for (int e = 0; e < E; ++e) {
            if (net.edges[e].open_t < 0 || net.edges[e].u < 0 || removed[e]) continue;
            removed[e] = 1;
            int m2;
            double f2;
            replay(ll_full, path, removed, m2, f2, nullptr);
            removed[e] = 0;
            if (best_e < 0 || m2 < best_mx || (m2 == best_mx && f2 < best_fl)) {
                best_e = e; best_mx = m2; best_fl = f2;
            }
        }
        if (best_e < 0) {
            err = "recompute_log2 exceeds the number of open output legs";
            return TN_EINVAL;
        }
        removed[best_e] = 1;
        sliced.push_back(best_e);
    }
    int mx;
    double fl;
    replay(ll_full, path, removed, mx, fl, nullptr);
    path.max_log2 = mx;
    path.flops = fl;
    return TN_OK;
}

}  // namespace tn

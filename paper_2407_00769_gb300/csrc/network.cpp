// Circuit -> tensor network (paper Sec. 2: an n-qubit state is a rank-n
// tensor, a single-qubit gate a rank-2 tensor, a two-qubit gate a rank-4
// tensor; contracting the network yields chosen amplitudes).
//
// One leaf per two-qubit gate.  Everything else is absorbed exactly:
//   * the single-qubit gates between two two-qubit gates on a wire are
//     multiplied into the input leg of the later two-qubit gate;
//   * the initial |0> of a qubit (with the single-qubit gates before its
//     first two-qubit gate) is contracted into that gate's input leg;
//   * the single-qubit gates after a qubit's last two-qubit gate are
//     multiplied into that gate's output leg, and a fixed output bit x
//     selects component x of it (the leg disappears); an open qubit keeps
//     the leg as an output index.
// A qubit without any two-qubit gate becomes a rank-1 (open) or rank-0
// (fixed) leaf of its own.
// Edge e = (qubit, after_gate): the wire of `qubit` right after two-qubit
// gate `after_gate`, so fixing its value (slicing) is the projector |b><b|
// applied at that point of the circuit.
#include <algorithm>
#include <array>
#include <cmath>

#include "internal.h"

namespace tn {

namespace {

using M2 = std::array<cd, 4>;  // row-major 2x2

M2 ident2() { return {cd(1), cd(0), cd(0), cd(1)}; }

M2 mul2(const M2 &a, const M2 &b) {  // a * b
    return {a[0] * b[0] + a[1] * b[2], a[0] * b[1] + a[1] * b[3],
            a[2] * b[0] + a[3] * b[2], a[2] * b[1] + a[3] * b[3]};
}

// leaf.data[.., o, ..] <- sum_j P[o][j] leaf.data[.., j, ..]  on leg position li
void apply_on_leg(Leaf &L, int li, const M2 &P) {
    const int r = (int)L.legs.size();
    const int64_t bit = (int64_t)1 << (r - 1 - li);
    std::vector<cd> out(L.data.size());
    for (int64_t i = 0; i < (int64_t)L.data.size(); ++i) {
        const int o = (i & bit) ? 1 : 0;
        const int64_t i0 = i & ~bit, i1 = i | bit;
        out[i] = P[2 * o + 0] * L.data[i0] + P[2 * o + 1] * L.data[i1];
    }
    L.data.swap(out);
}

// drop leg position li by fixing its value x
void select_leg(Leaf &L, int li, int x) {
    const int r = (int)L.legs.size();
    const int low = r - 1 - li;  // bit position of the leg
    std::vector<cd> out((size_t)1 << (r - 1));
    for (int64_t i = 0; i < (int64_t)out.size(); ++i) {
        const int64_t lo = i & (((int64_t)1 << low) - 1);
        const int64_t hi = i >> low;
        out[i] = L.data[(hi << (low + 1)) | ((int64_t)x << low) | lo];
    }
    L.data.swap(out);
    L.legs.erase(L.legs.begin() + li);
}

}  // namespace

int build_network(const tn_circuit *c, const tn_query *q, Network &net, std::string &err) {
    return build_network_open(c, q, 30, net, err);
}

int build_network_open(const tn_circuit *c, const tn_query *q, int max_open, Network &net, std::string &err) {
    if (!c || !q) { err = "null circuit or query"; return TN_EINVAL; }
    const int n = c->n_qubits;
    if (n < 1 || n > 64) { err = "n_qubits must be in 1..64"; return TN_EINVAL; }
    if (c->n_gates < 0 || (c->n_gates > 0 && !c->gates)) { err = "bad gate list"; return TN_EINVAL; }
    if (q->n_open < 0 || q->n_open > max_open || q->n_open > n) {
        err = "n_open must be in 0..min(" + std::to_string(max_open) + ", n)";
        return TN_EINVAL;
    }
    if (q->n_open > 0 && !q->open_qubits) { err = "open_qubits is NULL"; return TN_EINVAL; }
    if (!q->fixed_bits && q->n_open < n) { err = "fixed_bits is NULL"; return TN_EINVAL; }
    std::vector<int> open_t(n, -1);
    for (int t = 0; t < q->n_open; ++t) {
        const int oq = q->open_qubits[t];
        if (oq < 0 || oq >= n) { err = "open qubit out of range"; return TN_EINVAL; }
        if (t > 0 && oq <= q->open_qubits[t - 1]) { err = "open qubits must be strictly ascending"; return TN_EINVAL; }
        open_t[oq] = t;
    }
    for (int g = 0; g < c->n_gates; ++g) {
        const tn_gate &G = c->gates[g];
        if (G.q0 < 0 || G.q0 >= n || G.q1 >= n || G.q1 == G.q0) {
            err = "gate " + std::to_string(g) + " has a bad qubit index";
            return TN_EINVAL;
        }
        for (int k = 0; k < 16; ++k)
            if (!std::isfinite(G.re[k]) || !std::isfinite(G.im[k])) {
                err = "gate " + std::to_string(g) + " has a non-finite entry";
                return TN_EINVAL;
            }
    }

    net = Network();
    net.n_qubits = n;
    net.n_open = q->n_open;
    std::vector<M2> pend(n, ident2());
    std::vector<int> last_edge(n, -1);

    for (int g = 0; g < c->n_gates; ++g) {
        const tn_gate &G = c->gates[g];
        if (G.q1 < 0) {
            const M2 m = {cd(G.re[0], G.im[0]), cd(G.re[1], G.im[1]),
                          cd(G.re[4], G.im[4]), cd(G.re[5], G.im[5])};
            pend[G.q0] = mul2(m, pend[G.q0]);
            continue;
        }
        const int a = G.q0, b = G.q1;
        Leaf L;
        L.gate = g;
        // legs (oa, ob, ia, ib); data[(oa ob ia ib)] = M[(oa ob), (ia ib)]
        const int ea = (int)net.edges.size();
        net.edges.push_back(Edge{a, g, (int)net.leaves.size(), -1, -1});
        const int eb = (int)net.edges.size();
        net.edges.push_back(Edge{b, g, (int)net.leaves.size(), -1, -1});
        L.legs = {ea, eb, -2, -3};  // placeholders for the inputs
        L.data.resize(16);
        for (int r = 0; r < 4; ++r)
            for (int cc = 0; cc < 4; ++cc) L.data[4 * r + cc] = cd(G.re[4 * r + cc], G.im[4 * r + cc]);
        // absorb pending single-qubit gates on the inputs: T = M (Pa x Pb)
        // leg of input a is position 2, of input b position 3; multiplying on
        // the right by P means data[.., j] <- sum_i data[.., i] P[i][j]
        for (int side = 0; side < 2; ++side) {
            const int qq = side == 0 ? a : b;
            M2 Pt = pend[qq];
            // right multiplication by P on an input leg == left application of P^T
            Pt = {pend[qq][0], pend[qq][2], pend[qq][1], pend[qq][3]};
            apply_on_leg(L, 2 + side, Pt);
            pend[qq] = ident2();
        }
        // connect or close the inputs (b first so positions stay valid)
        for (int side = 1; side >= 0; --side) {
            const int qq = side == 0 ? a : b;
            const int li = 2 + side;
            if (last_edge[qq] < 0) {
                select_leg(L, li, 0);  // contract with |0>
            } else {
                L.legs[li] = last_edge[qq];
                net.edges[last_edge[qq]].v = (int)net.leaves.size();
            }
        }
        last_edge[a] = ea;
        last_edge[b] = eb;
        net.leaves.push_back(std::move(L));
    }

    // outputs
    std::vector<char> dead(net.edges.size(), 0);
    for (int qq = 0; qq < n; ++qq) {
        const int t = open_t[qq];
        const int x = t < 0 ? (q->fixed_bits[qq] ? 1 : 0) : 0;
        if (last_edge[qq] < 0) {
            Leaf L;
            L.qubit = qq;
            const cd v0 = pend[qq][0], v1 = pend[qq][2];  // P|0>
            if (t >= 0) {
                const int e = (int)net.edges.size();
                net.edges.push_back(Edge{qq, -1, (int)net.leaves.size(), -1, t});
                dead.push_back(0);
                L.legs = {e};
                L.data = {v0, v1};
            } else {
                L.data = {x ? v1 : v0};
            }
            net.leaves.push_back(std::move(L));
            continue;
        }
        const int e = last_edge[qq];
        Leaf &L = net.leaves[net.edges[e].u];
        const int li = (int)(std::find(L.legs.begin(), L.legs.end(), e) - L.legs.begin());
        apply_on_leg(L, li, pend[qq]);
        if (t >= 0) {
            net.edges[e].open_t = t;
        } else {
            select_leg(L, li, x);
            dead[e] = 1;
        }
    }

    // renumber the live edges: internal (two endpoints) and open ones
    std::vector<int> remap(net.edges.size(), -1);
    std::vector<Edge> live;
    for (size_t e = 0; e < net.edges.size(); ++e) {
        if (dead[e]) continue;
        remap[e] = (int)live.size();
        live.push_back(net.edges[e]);
    }
    for (Leaf &L : net.leaves)
        for (int &lg : L.legs) lg = remap[lg];
    net.edges.swap(live);
    return TN_OK;
}

int fix_open_legs(Network &net) {
    // every open output leg at value 0: a planning view of a sample network
    for (Leaf &L : net.leaves)
        for (int i = (int)L.legs.size() - 1; i >= 0; --i)
            if (L.legs[i] >= 0 && net.edges[L.legs[i]].open_t >= 0) select_leg(L, i, 0);
    return TN_OK;
}

int fix_legs(Network &net, const std::vector<int> &edges) {
    std::vector<char> fix(net.edges.size(), 0);
    for (int e : edges) fix[e] = 1;
    for (Leaf &L : net.leaves)
        for (int i = (int)L.legs.size() - 1; i >= 0; --i)
            if (L.legs[i] >= 0 && fix[L.legs[i]]) select_leg(L, i, 0);
    return TN_OK;
}

}  // namespace tn

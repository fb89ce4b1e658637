// Internal structures of the contraction library: the tensor network, the
// contraction path, and the device schedule (ops) that tn_contract replays.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "tn.h"

namespace tn {

using cd = std::complex<double>;

constexpr int kMaxRank = 40;   // modes of any device tensor (incl. batch modes)

// ---------------------------------------------------------------- network --
// An edge is one wire segment between two two-qubit gates: the wire of
// `qubit` right after gate `after_gate`.  Open edges end at the output.
struct Edge {
    int qubit = -1, after_gate = -1;
    int u = -1, v = -1;   // endpoint leaves (v < 0 for an open edge)
    int open_t = -1;      // output bit position t for an open edge
};

// A leaf: one two-qubit gate tensor with its neighbouring single-qubit gates,
// initial states and fixed output bits absorbed.  legs: edge ids, outermost
// first; data: row-major over legs.
struct Leaf {
    std::vector<int> legs;
    std::vector<cd> data;
    int gate = -1;        // circuit gate index it came from (-1: isolated qubit)
    int qubit = -1;       // the isolated qubit (gate == -1)
};

struct Network {
    int n_qubits = 0, n_open = 0;
    std::vector<Edge> edges;
    std::vector<Leaf> leaves;
};

int build_network(const tn_circuit *c, const tn_query *q, Network &out, std::string &err);
// build_network allowing up to max_open open qubits (sample networks: all)
int build_network_open(const tn_circuit *c, const tn_query *q, int max_open, Network &out, std::string &err);
// Every open output leg fixed at 0: one planning view of an
// uncorrelated-bitstring network.
int fix_open_legs(Network &net);
// The given legs fixed at 0 (a planning view with those legs split off).
int fix_legs(Network &net, const std::vector<int> &edges);

// ------------------------------------------------------------------- path --
struct Path {
    std::vector<std::pair<int, int>> steps;  // tensor ids; step s makes id L+s
    double flops = 0;                         // per slice, 8*M*N*K summed
    int max_log2 = 0;                         // largest intermediate (log2)
};

// --------------------------------------------------------------- schedule --
enum OpKind : int32_t {
    OP_LEAF = 1,    // prepare leaves of one phase (slice bits fixed, dtype convert)
    OP_PERM = 2,    // bit-permute one tensor
    OP_BPREP = 3,   // B [batch][K][N] complex-half -> B' real [batch][N'][K'] + colsum
    OP_GEMM = 4,    // one contraction step
    OP_SUM = 5,     // final tensor -> FP64 amplitudes
    OP_QUANT = 6,   // complex-half -> E4M3 operand of an FP8 tensor-core step
};

enum GemmKernel : int32_t {
    GK_C64_ROWS = 0,   // complex64, thread per row, B in shared memory
    GK_C64_TILED = 1,  // complex64, 2-D shared-memory tiles
    GK_LP_ROWS = 2,    // complex-half, FP32 math, thread per row
    GK_LP_TC = 3,      // complex-half as real, tcgen05 + TMA, FP32 in TMEM
    GK_C64_TC = 4,     // complex64 as real, tcgen05 kind::tf32 on hi / lo parts
};

// Tensor-core tile code: bits 0-3 N-tile width code, bits 4-7 raster-group
// code, bit 8 CTA pairs (256-row tiles on a cluster of 2 SMs), bit 9 64-byte
// K chunks (twice the ring stages of 128-byte chunks in the same memory),
// bit 10 the B'-resident kernel (each walker keeps its B' slice in shared
// memory; short-K steps), bit 11 (with bit 10) its C tiles staged in shared
// memory and written by TMA stores.
constexpr int kTcPairTile = 0x100;
constexpr int kTcHalfKTile = 0x200;
constexpr int kTcBresTile = 0x400;   // bit 10: B' slice resident in shared memory (short K)
constexpr int kTcStoreTile = 0x800;  // bit 11 (with bit 10): C tiles written by TMA stores
constexpr int kTcStagedTile = 0x1000; // bit 12: complex-half C through per-warp staging, whole-sector stores
// whether a step of this shape runs on CTA pairs when asked (bn: the N tile
// in real columns the launch uses)
bool tc_pair_eligible(int want, int fp8, int lm, int ln, int lk, int bn);

struct LeafJob {          // one leaf to prepare (device-side struct)
    int64_t src;          // element offset into the leaf store (complex128)
    int64_t dst;          // byte offset into the workspace
    int32_t rank_in;      // legs of the full leaf
    int32_t rank_out;     // legs kept
    int32_t n_fixed;      // legs fixed by looped slice bits
    int32_t fixed_pos[4]; // bit position (from LSB) of each fixed leg in the input
    int32_t fixed_bit[4]; // slice-id bit that fixes it
    int32_t keep_pos[32]; // bit position (from LSB) in the input of output bit i
    int32_t meta;         // tensor meta slot (complex-half)
    int32_t pad_;
};

struct PermOp {
    int64_t src, dst;     // byte offsets
    int32_t esz;          // element bytes (8: complex64, 4: complex-half)
    int32_t rank;
    int32_t perm[kMaxRank];  // output mode i (outermost first) = input mode perm[i]
};

struct GemmOp {
    int64_t a, b, c;      // byte offsets; b is [batch][K][N] (c64 / lp rows) or B'
    int32_t lm, ln, lk, lb;        // log2 of M, N, K, batch
    int32_t a_batched, b_batched;  // operand carries the batch modes (else broadcast)
    int32_t meta_a, meta_b, meta_c, step;
    int32_t kernel, tile;
    int32_t headroom;     // extra power-of-two scale from calibration (complex-half)
    int32_t ta, tb, tc;   // storage of A, B, C: 0 complex64, 1 complex-half
    int32_t fp8;          // tensor-core step on E4M3 copies of A and B'
    // > 0: C is written straight in a permuted mode order (a permutation of
    // its out_rank modes fused into the epilogue): source bit i of the
    // element index goes to bit out_dpos[i]; the lowest 3 bits stay
    int32_t out_rank;
    int8_t out_dpos[kMaxRank];
    // sparse-state gather step (uncorrelated bitstrings): per operand, the
    // batch entry s reads chunk idx[s] (offset of an int32 array in the plan's
    // index table, -1: chunk s) out of 2^gather_log2 chunks; bcast: one chunk
    // for every entry
    int64_t idx_a = -1, idx_b = -1;
    int32_t gather_a_log2 = 0, gather_b_log2 = 0;
    int32_t bcast_a = 0, bcast_b = 0;
};

struct QuantOp {
    int64_t src, dst;     // byte offsets: complex-half (or B' real) -> E4M3
    int64_t n_pairs;      // 16-bit value pairs
    int32_t meta_src, meta_dst;
};

struct BprepOp {
    int64_t src, dst;     // B (stored mode order) -> B' [batch][N'][K'] real
    int32_t lk, ln, lb, step;
    int32_t np;           // padded N' (real columns, >= 16)
    int32_t rank;         // modes of B
    int32_t tb;           // storage of B: 0 complex64 (scaled and rounded here), 1 complex-half
    int32_t meta_src, meta_dst;  // tb = 0: scale slots of B and of B' (B' = B 2^s)
    int32_t perm[kMaxRank];  // [batch][N][K] order: output mode i = stored mode perm[i]
};

struct SumOp {
    int64_t src;          // final tensor (byte offset)
    int32_t rank;         // legs of the final tensor
    int32_t open_pos[32]; // bit position (from LSB) of open output t in the tensor
    int32_t n_batch;      // batched slice bits in the final tensor
    int32_t batch_pos[16];// bit position (from LSB) of batched slice bit j
    int32_t meta;
    int32_t tf;           // storage of the final tensor: 0 complex64, 1 complex-half
    // recomputation: open outputs split into passes (absent from the final
    // tensor): output bit split_t[i] = slice-id bit split_bit[i]
    int32_t n_split;
    int32_t split_t[8], split_bit[8];
};

// Storage rule of complex-half plans: tensors of at most 2^kSmallLog2
// elements (leaves and small intermediates, whose values come from a few
// gates and are far from random) stay complex64; larger ones are stored in
// complex-half.
constexpr int kSmallLog2 = 16;   // default of tn_plan_opts.small_log2

struct Op {
    int32_t kind = 0;
    int32_t phase = 0;    // 0: once per call (slice invariant), 1: every pass
    int32_t leaf_first = 0, leaf_count = 0;  // OP_LEAF: range in plan leaf jobs
    PermOp perm{};
    GemmOp gemm{};
    BprepOp bprep{};
    SumOp sum{};
    QuantOp quant{};
};

// Record `msg` as the calling thread's last error (tn_last_error) and
// return `code`.
int record_error(int code, const std::string &msg);

// Per-step record for inspection.
struct StepRec {
    int a, b, c;
    int lm, ln, lk, lb;
    int permute_a, permute_b;
    int storage;
    int invariant;
    int kernel, tile;
};

}  // namespace tn

// The plan object behind the opaque tn_plan_t.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "internal.h"

namespace tn {

// Tensor-core split-K rule (tc_gemm.cu): K parts of one step; steps with
// K above 2^kSplitLog2KHost are always split.
int tc_split(int lm, int ln, int lk, int64_t batch);
constexpr int kSplitLog2KHost = 15;

// Refine `path` (on the network with `sliced` removed) by simulated
// annealing over tree rotations; intermediates stay within
// max(width_cap, current width); a step's cost counts as often as the step
// runs when all slices are contracted, 2^batch_log2 per pass.  Keeps the
// input when nothing improves.
int anneal_path(const Network &net, const std::vector<int> &sliced, int width_cap, uint64_t seed,
                int iters, double kappa, int batch_log2, Path &path);
// `chains` independent annealing chains (3 rounds each) on the chosen path
// and slices, the cheapest job kept (*cost_out: its roofline cost); with a
// cap (n_target < 0) a sliced edge is given back whenever the refined path
// stays within the cap and the job's cost (2^S x per-slice) drops.
int refine_plan(const Network &net, int n_target, int cap, uint64_t seed, int iters, double kappa,
                int batch_log2, int chains, Path &path, std::vector<int> &sliced, double *cost_out = nullptr);
int choose_slices(const Network &net, uint64_t seed, int trials, int n_target, int cap, Path &path,
                  std::vector<int> &sliced, std::string &err);
// fn(0), ..., fn(n-1), each on a thread of its own (fn(0) on the caller's;
// all on the caller's with one hardware thread or when no thread can be
// started); returns when all have ended and rethrows the first exception
// (by index) that one of them threw.  The calls must share no mutable state.
void run_parallel(int n, const std::function<void(int)> &fn);
// Recomputation (Sec. 3.4.1): append r open output legs to `sliced`, each
// the one whose removal shrinks the largest intermediate of `path` most
// (then its flops); updates the path's size and flops.
int choose_recompute(const Network &net, int r, Path &path, std::vector<int> &sliced, std::string &err);

struct Schedule {
    std::vector<Op> ops;                // phase 0 ops first, then phase 1
    std::vector<LeafJob> leaf_jobs;
    std::vector<StepRec> steps;
    int64_t ws_bytes = 0;               // workspace bytes
    int n_meta = 0, n_meta_inv = 0;     // meta slots; [0, n_meta_inv) invariant
    int n_meta_extra = 0;               // B' slots after n_meta (always written before read)
    double flops_per_pass = 0, flops_inv = 0;
    double bytes_per_pass = 0;
    int n_permutes = 0;
    int n_steps_inv = 0;
    int final_tensor = -1;
    int kernels_per_pass = 0, kernels_inv = 0;
    int n_gemm_steps = 0;
    std::vector<int32_t> gidx;          // index table of sparse-state gather steps
};

// Uncorrelated bitstrings: k sample edges (output bit j of the amplitude
// index = bit j of the sample index) and the 2^k bitstrings (bit q = qubit q).
// Tensors keep their output legs dense while they hold at most k of them; the
// step that would hold more (or that meets a tensor already indexed by
// sample) switches to one row per sample, gathering each operand's row by the
// sample's bits on that operand's output legs (the paper's sparse state).
struct SampleSpec {
    int k = 0;
    std::vector<int> sample_edges;       // [j] = edge of sample bit j
    std::vector<uint64_t> bits;          // 2^k bitstrings
};

int build_schedule(const Network &net, const Path &path, const std::vector<int> &sliced,
                   int batch_log2, int dtype, int small_log2, bool allow_tc, int fp8_min_log2_flops,
                   Schedule &out, std::string &err, const SampleSpec *spec = nullptr);

}  // namespace tn

struct tn_plan_s;
namespace tn {
// Device state (workspace, leaf upload), scale calibration and tile choice
// of a plan, as the first tn_contract call does them (each once).
int prepare_for_contract(tn_plan_s *P, cudaStream_t s);
}  // namespace tn

struct tn_plan_s {
    tn::Network net;
    tn_plan_opts opts{};
    std::vector<int> sliced;   // edge ids; slice-id bit j <-> sliced[j]
    int batch_log2 = 0;
    int n_recompute = 0;       // the last n sliced edges are split open legs
    tn::Path path;
    tn::Schedule sched;
    std::vector<tn::cd> leaf_store;     // all leaves, full legs, complex128
    std::vector<int64_t> leaf_offset;   // element offset of each leaf in the store
    // device state (created on first contract)
    bool dev_ready = false;
    int device = -1;
    char *d_ws = nullptr;
    double2 *d_store = nullptr;
    tn::LeafJob *d_jobs = nullptr;
    float *d_tmax = nullptr;
    int32_t *d_texp = nullptr;
    int32_t *d_err = nullptr;
    double2 *d_stepcorr = nullptr;      // per step: 1/(1+alpha) of its B' rounding
    float *d_splitk = nullptr;          // FP32 partials of split-K tensor-core steps
    void *d_bpart = nullptr;            // partial sums of the multi-block complex64 B' build
    float *d_x3 = nullptr;              // complex64 on the tensor cores: TF32 parts of A and B'
    int32_t *d_gidx = nullptr;          // index table of sparse-state gather steps
    void *h_store_pinned = nullptr;     // pinned copy of the leaf store
    // per-kernel-class event timing (tn_profile)
    uint32_t prof_mask = 0;
    struct ProfRec { int cls; cudaEvent_t e0, e1; double flops, bytes; int kernels; };
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<void *> owned;          // allocations to free
    // CUDA graph of the last captured tn_contract call (tn_plan_set_graph)
    bool use_graph = false;
    struct GraphKey {
        int64_t begin, count;
        double *amps;
        int accumulate;
        cudaStream_t stream;
        bool operator==(const GraphKey &o) const {
            return begin == o.begin && count == o.count && amps == o.amps &&
                   accumulate == o.accumulate && stream == o.stream;
        }
    };
    GraphKey graph_key{};
    cudaGraphExec_t graph_exec = nullptr;
    int graph_launches = 0;
    // work queue of the last tn_contract call (tn_plan_set_queue)
    bool use_queue = false;
    struct tn_queue_s *queue = nullptr;
    GraphKey queue_key{};
    // autotuner: chosen (kernel, tile) per GEMM op live in sched.ops; every
    // timing taken is kept as a record (the cost model's training data)
    bool tuned = false;
    bool calibrated = false;
    std::vector<tn_tune_record> tune_recs;
    struct tn_cost_model_s *cost_model = nullptr;
};

/*
 * tn.h -- C ABI of the GB300 sliced tensor-network contraction library.
 *
 * The library computes amplitudes <x|U|0^n> of a random quantum circuit U for
 * a correlated set of bitstrings x (some qubits open, the rest fixed) by
 * contracting the circuit's tensor network (paper Sec. 2, "RQC simulation
 * methods": a circuit becomes a network of rank-2 and rank-4 gate tensors
 * whose contraction yields chosen amplitudes).  The network is cut into
 * independent sub-networks by fixing the values of chosen edges -- slicing,
 * "breaking edges" (Sec. 3, Innovations; Sec. 3.1) -- and each slice is
 * contracted as a sequence of pairwise steps, each one index permutation
 * followed by a matrix multiplication (Sec. 3.1, device level; Sec. 3.3,
 * Eq. 3-4: a pairwise einsum is a pure GEMM when its reduced modes are the
 * modes the two operands share).  Slice results are summed in FP64.  Low-
 * precision steps use the complex-as-real layout of Sec. 3.3 (Eq. 5-6): the
 * large operand keeps its interleaved real/imag mode as an extra reduced mode
 * and the small operand is padded to [[Re, -Im], [Im, Re]], so one real GEMM
 * with K -> 2K and N -> 2N does the complex product.  Post-selection keeps the
 * k most probable bitstrings of a correlated subspace (Sec. 1 and Sec. 2,
 * post-processing).  Arbitrary (uncorrelated) bitstrings are planned by
 * tn_plan_samples, whose last steps contract many gathered tensor pairs at
 * once (Sec. 3.4.2, sparse state); tn_plan_opts.recompute_log2 splits output
 * legs into sequential passes (Sec. 3.4.1, recomputation).
 *
 * Conventions
 *   - qubit q of a bitstring x is bit q of x;
 *   - a 2x2 gate is row-major (out, in); a 4x4 gate is row-major over
 *     |q0 q1>, q0 the high bit of the local index;
 *   - amplitude index j of an output: bit t of j is qubit open_qubits[t];
 *   - slice id s: bit j of s is the value of sliced edge j (LSB first).
 *   - amplitude buffers are complex128, interleaved (re, im) doubles.
 *
 * Errors: every int-returning call returns TN_OK (0) or a TN_E* code; no C++
 * exception crosses this boundary.  tn_strerror() names a code;
 * tn_last_error() gives a message for the calling thread's last failure.
 *
 * Streams: `stream` arguments are cudaStream_t values passed as void*
 * (NULL = the legacy default stream).  Device pointers must come from the
 * CUDA runtime of the calling process and belong to the current device.
 */
#ifndef TN_H_
#define TN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define TN_OK 0
#define TN_EINVAL 1        /* bad argument (indices, sizes, ranges)            */
#define TN_ENOMEM 2        /* host or device allocation failed                 */
#define TN_ECUDA 3         /* a CUDA runtime/driver call failed                */
#define TN_ETIMEOUT 4      /* a bounded device wait gave up (kernel returned)  */
#define TN_EUNSUPPORTED 5  /* valid request outside the supported range        */

/* ---- element types of the contraction ---- */
#define TN_C64 0    /* complex64: FP32 re/im, FP32 SIMT arithmetic           */
#define TN_F16 1    /* complex-half: FP16 re/im, tensor-core FP32 accumulate */
#define TN_BF16 2   /* BF16 re/im, tensor-core FP32 accumulate               */
#define TN_FP8 3    /* tn_gemm only: E4M3 re/im operands, FP16 result; in a
                       plan, see tn_plan_opts.fp8_min_log2_flops          */

/* ---- tile policies (which GEMM tile each step uses) ---- */
#define TN_TILE_FIXED 0       /* built-in heuristic                              */
#define TN_TILE_EXHAUSTIVE 1  /* time every legal tile on first contract         */
#define TN_TILE_LEARNED 2     /* rank tiles with the trained cost model          */

typedef struct {
    int32_t q0, q1;       /* q1 < 0: single-qubit gate on q0                     */
    double re[16], im[16];/* 2x2 in [0],[1],[4],[5] (row-major, 4-wide rows)    */
                          /* or 4x4 row-major over |q0 q1>                       */
} tn_gate;

typedef struct {
    int32_t n_qubits;     /* 1..64                                               */
    int32_t n_gates;
    const tn_gate *gates; /* host, length n_gates, in circuit order              */
} tn_circuit;

typedef struct {
    int32_t n_open;              /* 0..30                                        */
    const int32_t *open_qubits;  /* host, ascending, length n_open               */
    const uint8_t *fixed_bits;   /* host, length n_qubits; open entries ignored  */
} tn_query;

typedef struct {
    int32_t dtype;            /* TN_C64 | TN_F16 | TN_BF16                       */
    int32_t max_log2_elems;   /* slice until every per-slice intermediate has
                                 at most 2^this elements (<= 0: no cap)          */
    int32_t n_slice_edges;    /* >= 0: slice exactly this many edges;
                                 -1: as many as the cap needs                    */
    uint64_t path_seed;       /* seed of the randomized greedy path search       */
    int32_t path_trials;      /* greedy restarts (>= 1); trial 0 is noiseless    */
    int32_t path_anneal_iters;/* > 0: refine the path by simulated annealing
                                 (Sec. 3): path_trials starts (greedy
                                 slicings under different seeds), two chains
                                 each of 3 rounds of this many tree
                                 rotations; the job of lowest roofline cost
                                 is kept (ties to the lower start and chain:
                                 the starts and chains run on host threads of
                                 their own and the result does not depend on
                                 them); with a cap, sliced edges the refined
                                 path no longer needs are given back        */
    int32_t slice_batch_log2; /* run 2^this consecutive slices in one pass, the
                                 batch carried as an extra tensor mode (>= 0;
                                 slicing to a cap: lowered to the number of
                                 summed sliced edges if the planner keeps
                                 fewer)                                          */
    int32_t tile_policy;      /* TN_TILE_*                                       */
    int32_t small_log2;       /* complex-half plans: tensors of at most
                                 2^small_log2 elements are stored complex64
                                 (0: default 16; > 40: every tensor)            */
    int32_t no_tensor_cores;  /* 1: complex-half steps on CUDA cores only
                                 (validation of the tensor-core path)           */
    int32_t fp8_min_log2_flops; /* complex-half plans: tensor-core steps of at
                                 least 2^this real flops per pass (and K >= 64)
                                 take E4M3 operands (A and B' quantized with a
                                 power-of-two scale, FP32 accumulate, result in
                                 the plan's dtype); 0: never                    */
    int32_t recompute_log2;   /* recomputation (Sec. 3.4.1): split this many
                                 open output legs into sequential passes, each
                                 computing its part of the amplitude vector
                                 (concatenated, not summed); the planner picks
                                 the legs that shrink the largest intermediate
                                 most.  They become the highest slice-id bits:
                                 the slices of one part are contiguous.  The
                                 steps before the legs meet the path run once
                                 per call.  0: off; correlated plans only     */
    int32_t no_scaling;       /* validation only.  1: complex-half tensors are
                                 stored without their power-of-two scale (every
                                 exponent 0, no calibration pass), which shows
                                 what the scaling protects against: the small
                                 values of deep intermediates fall into FP16's
                                 subnormal range or flush to zero.  0: scaled
                                 (default).  Not with fp8_min_log2_flops.     */
    int32_t anneal_kappa;     /* path_anneal_iters > 0: the flops one element
                                 of a step's operands and result counts for in
                                 the annealer's cost (its HBM traffic against
                                 tensor work).  0: 1000 (complex-half), 100
                                 (complex64)                                  */
    int64_t workspace_budget; /* > 0: the library chooses slice_batch_log2 itself
                                 (the given value is ignored): the largest
                                 b <= min(16, summed sliced edges) whose device
                                 workspace fits in this many bytes, else 0 --
                                 as many slices per pass as memory allows, one
                                 path search.  0: slice_batch_log2 as given   */
    int32_t c64_tensor_cores; /* dtype TN_C64: 1 = complex64 steps of one K
                                 part (K <= 2^15, not split) may run on the
                                 tensor cores (tn_gemm kernel 9: TF32 parts
                                 and rounded remainders, three MMAs per K
                                 slice, 64-term K parts summed in FP32
                                 registers; ~5e-7 relative error per GEMM, as
                                 the CUDA cores; device scratch for the split
                                 operands of the largest such step).  The
                                 fixed policy takes it for steps of >= 2^36
                                 flops, the autotuner times it.  0 (default):
                                 CUDA cores only                            */
    int32_t pad_;
    /* Optional device allocator for the plan's workspace (e.g. PyTorch's
       caching allocator).  NULL: cudaMalloc/cudaFree. */
    void *(*dev_alloc)(size_t bytes, void *ctx);
    void (*dev_free)(void *ptr, void *ctx);
    void *alloc_ctx;
} tn_plan_opts;

typedef struct tn_plan_s tn_plan_t;  /* opaque */

typedef struct {
    int32_t n_qubits, n_open;
    int32_t n_leaves;             /* tensors after absorbing 1q gates/boundaries */
    int32_t n_edges;              /* internal (contracted) edges before slicing   */
    int32_t n_slice_edges;
    int64_t n_slices;             /* 2^n_slice_edges                             */
    int32_t n_steps;              /* pairwise contractions per slice             */
    int32_t n_steps_invariant;    /* of those, independent of the slice          */
    int32_t max_log2_elems;       /* largest intermediate of one slice (log2)    */
    int32_t slice_batch_log2;
    double flops_per_slice;       /* sum over steps of 8*M*N*K (real flops)      */
    double flops_invariant;       /* part of it done once per contract call      */
    double bytes_per_slice;       /* algorithmic bytes: per step, operands +
                                     result once, plus permuted copies          */
    int64_t workspace_bytes;      /* device workspace of the plan                */
    int32_t n_permutes;           /* explicit permutations per slice             */
    int32_t dtype;
    int64_t leaf_bytes;           /* host->device bytes of the leaf tensors      */
    int32_t n_recompute_edges;    /* open legs split by recomputation; they are
                                     the last n of the n_slice_edges           */
} tn_plan_stats;

typedef struct {
    double ms;                    /* device time of the call (CUDA events)       */
    double flops;                 /* real flops executed                         */
    int64_t slices;               /* slices summed                               */
    int32_t kernels;              /* kernel launches issued                      */
    int32_t min_exp, max_exp;     /* range of per-slice scale exponents (lp)     */
} tn_contract_report;

/* One step of a plan (for inspection and tests). */
typedef struct {
    int32_t a, b, c;              /* tensor ids: inputs, output                  */
    int32_t log2_m, log2_n, log2_k, log2_batch;
    int32_t permute_a;            /* 1 if A is permuted before the GEMM          */
    int32_t slice_invariant;
    int32_t kernel;               /* which GEMM kernel variant runs this step    */
    int32_t tile;                 /* tile configuration index                    */
    int32_t permute_b;            /* 1 if B is permuted before the GEMM          */
    int32_t scale_headroom;       /* calibrated extra 2^e of the step's output   */
    int32_t storage;              /* bit 0: A, bit 1: B, bit 2: C stored
                                     complex-half (else complex64); bit 3: the
                                     GEMM takes E4M3 copies of A and B'          */
} tn_step_info;

/*
 * tn_plan: build the tensor network of `circuit` for `query`, search a greedy
 * pairwise contraction path, choose sliced edges and lay out every step.
 * The circuit becomes one tensor per two-qubit gate; single-qubit gates, the
 * initial |0> states and the fixed output bits are absorbed into them
 * (exact).  Host work only; device memory is allocated on the first
 * tn_contract.  *out receives a plan the caller frees with tn_plan_destroy.
 * Errors: TN_EINVAL (bad qubit index, repeated/unsorted open qubits, n_open
 * > 30, bad dtype, a cap the slicing cannot reach), TN_ENOMEM.
 */
int tn_plan(const tn_circuit *circuit, const tn_query *query, const tn_plan_opts *opts,
            tn_plan_t **out);

/*
 * tn_plan_samples: a plan for the amplitudes of n_samples arbitrary
 * (uncorrelated) bitstrings of `circuit`: samples[s * n_qubits + q] is bit q
 * (0 or 1) of bitstring s.  The network keeps every qubit's output leg; a
 * tensor holds its output legs densely while it has at most
 * k = ceil(log2 n_samples) of them, and the step that would give it more (or
 * that meets a tensor already indexed by sample, or the last step) switches
 * to one row per sample: each operand still holding dense outputs is read at
 * the row the sample's bits select, through index arrays built here (the
 * sparse state of paper Sec. 3.4.2, on the gathering GEMMs).  The path is
 * planned twice, on the network with its output legs as legs and with them
 * fixed (each with at least 4 randomized greedy restarts), and the cheaper
 * resulting schedule is kept.  tn_contract fills 2^k
 * amplitudes, entry s for bitstring s (entries past n_samples repeat the
 * last bitstring); slicing, slice batching and dtypes as for tn_plan
 * (slices run together x 2^k must stay within 2^24 rows).
 * Errors: TN_EINVAL (NULL, n_samples outside 1..2^20, k > 24, a bit other
 * than 0/1), as tn_plan otherwise.
 */
int tn_plan_samples(const tn_circuit *circuit, const uint8_t *samples, int32_t n_samples,
                    const tn_plan_opts *opts, tn_plan_t **out);

/* Fill default options (TN_F16, no cap, no slicing, seed 1, 1 trial). */
void tn_plan_opts_default(tn_plan_opts *opts);

int tn_plan_info(const tn_plan_t *plan, tn_plan_stats *out);

/* Sliced edges as (qubit, after_gate) pairs: edge j is the wire of `qubit`
 * right after gate index `after_gate` of the circuit.  Writes
 * min(capacity, n_slice_edges) pairs; returns TN_OK. */
int tn_plan_sliced_edges(const tn_plan_t *plan, int32_t *qubit, int32_t *after_gate,
                         int32_t capacity);

/* Step i of the per-slice schedule (0 <= i < n_steps).  Tensor ids a, b, c:
 * ids below n_leaves are leaves (tn_plan_leaf_source), step s creates id
 * n_leaves + s; the steps in order are the contraction path. */
int tn_plan_step(const tn_plan_t *plan, int32_t i, tn_step_info *out);

/* Where leaf i (0 <= i < n_leaves) comes from: *gate = index in the circuit
 * of its two-qubit gate (the single-qubit gates, initial states and output
 * bits around it absorbed, Sec. 2 circuit-to-network), or -1 for a qubit
 * that no two-qubit gate touches, whose index is then written to *qubit
 * (else -1).  Errors: TN_EINVAL (NULL plan, i out of range). */
int tn_plan_leaf_source(const tn_plan_t *plan, int32_t i, int32_t *gate, int32_t *qubit);

/*
 * tn_plan_leaf_tensor: leaf i (0 <= i < n_leaves) as the plan holds it on the
 * host, before slicing: *rank legs, leg p (outermost first) being the wire of
 * qubit[p] right after circuit gate after_gate[p] (the first min(capacity,
 * rank) legs are written; qubit / after_gate may be NULL); data (host,
 * nullable) receives its 2^rank complex128 values (interleaved re, im),
 * row-major over the legs.  Errors: TN_EINVAL (NULL plan or rank, i out of
 * range).
 */
int tn_plan_leaf_tensor(const tn_plan_t *plan, int32_t i, int32_t capacity, int32_t *rank,
                        int32_t *qubit, int32_t *after_gate, double *data);

/*
 * tn_plan_decode_leaf: slice decoding of one leaf, as tn_contract does it on
 * the device (Sec. 3.1: a slice fixes the values of the sliced edges; bit j
 * of the slice id is the value of sliced edge j, LSB first).  Runs the plan's
 * leaf preparation of leaf i for the pass starting at slice_id (a multiple
 * of 2^slice_batch_log2 below n_slices) and copies the prepared sub-tensor to
 * `data` (host, 2^rank complex64, interleaved re, im; nullable: legs only).
 * Its legs are the leaf's legs minus the sliced edges the pass fixes (edges
 * run as slice-batch modes stay legs), in the order the schedule lays them
 * out: leg q (outermost first) is the wire of qubit[q] after gate
 * after_gate[q].  The values are the leaf's complex128 values rounded to
 * complex64 (round to nearest even).  Synchronizes `stream`; sets up the
 * plan's device state if no tn_contract has run.  Errors: TN_EINVAL (NULL
 * plan or rank, i or slice_id out of range), TN_ENOMEM, TN_ECUDA.
 */
int tn_plan_decode_leaf(tn_plan_t *plan, int64_t slice_id, int32_t i, int32_t capacity, int32_t *rank,
                        int32_t *qubit, int32_t *after_gate, float *data, void *stream);

/*
 * tn_contract: contract slices [slice_begin, slice_begin + slice_count) and
 * add (accumulate != 0) or write (accumulate == 0) their FP64 sum into d_amps
 * (device, 2^n_open complex128, caller-owned).  Slices are summed in
 * ascending order, each slice's amplitudes added one slice at a time, so
 * splitting a range into ordered sub-ranges with accumulate=1 gives
 * bit-identical sums (plans with slice_batch_log2 = 0).  Enqueued on
 * `stream`; returns after enqueueing unless `rep` is non-NULL (then it
 * synchronizes and fills the report).  A plan serves one stream at a time.
 * Errors: TN_EINVAL (range outside [0, n_slices)), TN_ENOMEM, TN_ECUDA,
 * TN_ETIMEOUT.
 */
int tn_contract(tn_plan_t *plan, int64_t slice_begin, int64_t slice_count, double *d_amps,
                int accumulate, void *stream, tn_contract_report *rep);

/* As tn_contract, end to end from host memory: the leaf tensors are copied
 * host->device from the plan's pinned host copy, the slices contracted, and
 * the 2^n_open amplitudes copied to h_amps (host).  Synchronizes. */
int tn_contract_host(tn_plan_t *plan, int64_t slice_begin, int64_t slice_count,
                     double *h_amps, void *stream, tn_contract_report *rep);

/*
 * tn_plan_set_graph: when enable != 0, tn_contract captures its launches
 * into a CUDA graph the first time it is called with a given (slice range,
 * d_amps, accumulate, stream) and replays the graph on later identical
 * calls.  Needs a non-default stream (on the legacy default stream the
 * launches are issued directly).  Off by default.
 */
int tn_plan_set_graph(tn_plan_t *plan, int enable);

/*
 * Batched launch of many independent plans (e.g. uneven circuits): every
 * slice of plans[i] is contracted into d_amps[i] (device, 2^n_open_i
 * complex128, overwritten).  tn_batch_create sets up each plan's device
 * state, spreads the plans over n_streams side streams (largest work first,
 * to the least loaded stream; work = the cost model's predicted time when
 * every plan has one attached, else flops) and captures all their launches into one CUDA
 * graph; tn_batch_run replays that graph on `stream` (rep: optional timing,
 * synchronizes).  Plans must share dtype, have profiling off, and not be
 * used elsewhere while the batch exists.
 */
typedef struct tn_batch_s tn_batch_t;
int tn_batch_create(tn_plan_t *const *plans, int32_t n, double *const *d_amps, int32_t n_streams,
                    tn_batch_t **out);
int tn_batch_run(tn_batch_t *batch, void *stream, tn_contract_report *rep);
void tn_batch_destroy(tn_batch_t *batch);

/* One-shot form: create (16 streams), run once, synchronize, destroy. */
int tn_contract_batch(tn_plan_t *const *plans, int32_t n, double *const *d_amps, void *stream);

/*
 * Persistent work queue: the contraction of many independent plans (uneven
 * circuits, or slice ranges of one plan) in ONE kernel launch.  Slices and
 * circuits are independent sub-tasks whose results are summed (Sec. 3.1,
 * global level); within one pass the steps form a chain.  tn_queue_create
 * sets up each plan's device state (calibration and tile choice included,
 * as a first tn_contract would), then compiles every op of the contraction
 * of slices [slice_begin[i], slice_begin[i] + slice_count[i]) of plans[i]
 * into d_amps[i] (device, 2^n_open_i complex128, overwritten; NULL range
 * arrays: every slice) into a device table of ops, each cut into tiles
 * (items) and chained to the op after it.  tn_queue_run launches one
 * persistent kernel (one 320-thread CTA per SM, the tensor-core tiles on
 * tcgen05/TMA/TMEM as in tn_contract, the other ops on the same kernels'
 * device code) whose CTAs claim tiles from a list, one atomic ticket each:
 * the tiles of the chains' first ops are listed at launch, and an op's
 * tiles are listed by the CTA that counts its predecessor's last tile done
 * (per-op counters), so a claimed tile never waits on another.  A CTA whose
 * ticket is not listed yet waits for running tiles to list more, a wait
 * bounded by the queue's limit (default 10 s, tn_queue_set_wait_limit),
 * after which every CTA returns and the run reports TN_ETIMEOUT
 * (rep != NULL).  Results equal tn_contract's bit for
 * bit.  rep: optional timing and error check (synchronizes `stream`).
 * Plans must have profiling off and must not be used elsewhere while the
 * queue exists; the queue owns its tables (device memory from cudaMalloc).
 * TN_EUNSUPPORTED: a plan with FP8 steps.
 */
typedef struct tn_queue_s tn_queue_t;
typedef struct {
    int32_t n_plans;
    int32_t n_ops;                /* ops in the table                             */
    int32_t n_items;              /* tiles (items) claimed by the CTAs, all ops   */
    int32_t max_chain;            /* longest dependency chain (ops)               */
    int32_t ctas;                 /* CTAs of the launch                           */
    int32_t pad_;
    int64_t table_bytes;          /* op parameter records                         */
    double flops;                 /* real flops of one run                        */
    int64_t slices;               /* slices summed in one run                     */
} tn_queue_stats;
int tn_queue_create(tn_plan_t *const *plans, int32_t n, const int64_t *slice_begin,
                    const int64_t *slice_count, double *const *d_amps, tn_queue_t **out);
int tn_queue_run(tn_queue_t *queue, void *stream, tn_contract_report *rep);
int tn_queue_info(const tn_queue_t *queue, tn_queue_stats *out);
int tn_queue_set_wait_limit(tn_queue_t *queue, int64_t limit_us);
/*
 * Queue profiling: when enabled, each run sums per op kind (index =
 * TN_QK_*) the items run, the time their CTAs spent waiting for the
 * item's list entry to be written and the time spent running them (CTA-milliseconds, from
 * %globaltimer); tn_queue_profile_read returns the last run's sums (after it
 * finished) for kinds 0..capacity-1.
 */
#define TN_QK_ZERO 1
#define TN_QK_LEAF 2
#define TN_QK_PERM 3
#define TN_QK_PERM_TILED 4
#define TN_QK_BPREP_GATHER 5
#define TN_QK_BPREP_C64 6
#define TN_QK_ROWS 7
#define TN_QK_TILED_C64 8
#define TN_QK_TC 9
#define TN_QK_SPLITK 10
#define TN_QK_SUM 11
#define TN_QK_COUNT 12
typedef struct {
    int64_t items;
    double wait_ms;
    double busy_ms;
} tn_queue_kind_stats;
int tn_queue_profile(tn_queue_t *queue, int enable);
int tn_queue_profile_read(const tn_queue_t *queue, tn_queue_kind_stats *out, int32_t capacity);
void tn_queue_destroy(tn_queue_t *queue);

/*
 * tn_plan_set_queue: when enable != 0, tn_contract runs the whole call as
 * one work-queue launch (above), built the first time it is called with a
 * given (slice range, d_amps, accumulate) and reused on later identical
 * calls.  Off by default.
 */
int tn_plan_set_queue(tn_plan_t *plan, int enable);

/*
 * tn_selftest_queue_timeout: runs a queue holding an op that nothing ever
 * lists, with a wait limit of limit_ms (1..10000); the wait of the CTA
 * holding that op's ticket runs out and the call returns TN_ETIMEOUT, the
 * context still usable.
 */
int tn_selftest_queue_timeout(int32_t limit_ms, void *stream);

/*
 * tn_sample: post-selection on one correlated subspace (Sec. 1/2,
 * post-processing): from d_amps (device, 2^n_open complex128) return the k
 * indices of largest |amp|^2 and their probabilities, ties to the lower index,
 * in descending order.  out_idx / out_prob: host, length k, caller-owned.
 * Small problems (k * 2^n_open <= 2^22) run one block that rescans the
 * amplitudes once per result; larger ones a multi-block radix select over
 * the bits of |amp|^2 (8 passes over the amplitudes), the collection of the
 * k kept entries (ties at the threshold to the lowest indices) and a bitonic
 * sort -- O(2^n_open) reads per pass at any k.  Allocates its results and
 * scratch on `stream` (stream-ordered allocator) and frees them.
 * Synchronizes `stream`.  Errors: TN_EINVAL (k < 1 or k > 2^n_open, n_open
 * > 30), TN_ENOMEM, TN_ECUDA.
 */
int tn_sample(const double *d_amps, int32_t n_open, int32_t k, int64_t *out_idx,
              double *out_prob, void *stream);

/*
 * tn_sample_noalloc: tn_sample for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a deployment variant.
 * tn_sample allocates a small device buffer for the k results (and the
 * selection's scratch) on every call; a caller inside a host application
 * that owns all device memory through its own pool, or a latency-critical
 * thread that must not enter the CUDA allocator (cudaMalloc/cudaFree can
 * synchronize the device), cannot.  This call allocates nothing: its
 * scratch is a fixed array in device global memory holding
 * TN_SAMPLE_NOALLOC_MAX_K indices and probabilities and the selection's
 * working space for that many results (44 KiB), present on every GPU that
 * loads the library until the process exits.  Same arguments, results,
 * ordering and kernels as tn_sample.
 *   - k > TN_SAMPLE_NOALLOC_MAX_K is rejected with TN_EINVAL (use tn_sample).
 *   - The first call on a device looks up the array's device address
 *     (set-up, once per device, with that device current).  The address is
 *     kept for the life of the process: after cudaDeviceReset on a device,
 *     do not call this on that device again.
 *   - All calls on a device share the one array and it keeps the last
 *     call's contents; calls that overlap on the GPU (different streams or
 *     threads without ordering between them) race and may return each
 *     other's results.  Each call writes every entry it reads back, so
 *     nothing has to start at zero.
 * Synchronizes `stream` (the results are copied to the host), so it cannot be
 * called on a stream that is being captured into a graph.
 */
#define TN_SAMPLE_NOALLOC_MAX_K 1024
int tn_sample_noalloc(const double *d_amps, int32_t n_open, int32_t k, int64_t *out_idx,
                      double *out_prob, void *stream);

/*
 * tn_metrics: FP64 reductions on the device over n complex128 amplitudes:
 * out[0] = sum |r|^2, out[1] = rel-L2 ||r - b|| / ||b||, out[2] = fidelity
 * |<b,r>|^2 / (||b||^2 ||r||^2) (Sec. 4.2, Eq. 8, conjugate-linear inner
 * product), out[3] = linear XEB 2^n_qubits * mean |r|^2 - 1 of the n entries.
 * d_ref may be NULL (then out[1], out[2] are NaN).  out: host, 4 doubles.
 */
int tn_metrics(const double *d_amps, const double *d_ref, int64_t n, int32_t n_qubits,
               double *out, void *stream);

/*
 * tn_plan_step_scale: the power-of-two scale state of step i's output after
 * the last tn_contract pass of a complex-half plan (validation of the
 * per-tensor scaling).  *exp (nullable) = the output's exponent E, stored
 * value = true value x 2^E (E adds the exponents of the operands and the
 * step's own e); *stored_max (nullable) = the largest |re| or |im| of the
 * values stored in that pass.  With scaling on, e is chosen on the device so
 * that 2 K max|A| max|B| 2^e <= 2^14, plus a headroom that the first call's
 * calibration pass fixes per step: on that pass every complex-half output's
 * stored_max lies in (2^11, 2^14], and in (2^11, 2^12] for steps given a
 * headroom.  Synchronizes the device.  Errors: TN_EINVAL (NULL, i out of
 * range, complex64 plan, no tn_contract yet), TN_ECUDA.
 */
int tn_plan_step_scale(tn_plan_t *plan, int32_t i, int32_t *exp, float *stored_max);

void tn_plan_destroy(tn_plan_t *plan);

/* ---- autotuner (tile choice per step) ---- */

/* One timing taken by the autotuner: a GEMM step under one (kernel, tile)
 * configuration, or a permutation. */
typedef struct {
    int32_t kind;          /* 0: GEMM step, 1: permutation                    */
    int32_t lm, ln, lk, lb;/* log2 M, N, K, batch (GEMM); lm = rank (perm)     */
    int32_t dtype;
    int32_t kernel;        /* GEMM kernel variant (perm: -1)                   */
    int32_t tile;          /* tile configuration (perm: stride class 0..5 =
                              low output bits that stay low input bits).
                              Tensor-core steps: bits 0-3 N-tile code, 4-7
                              raster-group code, 8 CTA pairs, 9 64-byte K
                              chunks, 10 B' resident in shared memory, 11
                              (with 10) TMA-store epilogue, 12 staged
                              whole-sector stores                             */
    int32_t step;          /* plan step of a GEMM record (perm: -1)            */
    int32_t pad_;
    double ms;             /* CUDA-event time of one launch                    */
} tn_tune_record;

/*
 * tn_plan_tune: exhaustive autotuning.  Runs the slice-invariant ops and one
 * pass of the per-slice ops on slice 0's data; every GEMM step is launched
 * under each legal (kernel, tile) configuration, timed with CUDA events, and
 * the fastest is kept for later tn_contract calls; every permutation is
 * timed once.  All timings are kept as records.  Synchronizes.  Plans with
 * tile_policy TN_TILE_EXHAUSTIVE tune themselves on their first tn_contract.
 */
int tn_plan_tune(tn_plan_t *plan, void *stream);

/* Autotuner cache: for every GEMM step of `plan`, pick the fastest
 * configuration among `recs` (records from tuning other plans) whose
 * signature -- (log2 M, N, K, batch), dtype and kernel family -- matches
 * the step; steps without a matching record keep their configuration. */
int tn_plan_apply_tuning(tn_plan_t *plan, const tn_tune_record *recs, int32_t n);

/* Copy up to `capacity` autotuner records; *n_total receives how many exist. */
int tn_tune_records(const tn_plan_t *plan, tn_tune_record *out, int32_t capacity, int32_t *n_total);

/* ---- learned cost model ----
 * A small MLP (TN_COST_NFEAT inputs -> 3 hidden ReLU layers -> 1) predicting
 * log2 of a step's time in microseconds from its shape features; trained on
 * the GPU by the library's own forward/backward/Adam kernels on autotuner
 * records; used by TN_TILE_LEARNED plans to pick each GEMM step's (kernel,
 * tile) without timing, and to compare plans by predicted time.  FP32. */
#define TN_COST_NFEAT 26
typedef struct tn_cost_model_s tn_cost_model_t;
int tn_cost_model_create(int32_t hidden, uint64_t seed, tn_cost_model_t **out);
void tn_cost_model_destroy(tn_cost_model_t *model);
/* Get (set = 0) or set (set = 1) the flat FP32 parameter vector
 * [W1, b1, W2, b2, W3, b3, W4, b4], each W row-major (inputs x outputs);
 * *n_params receives its length.  Setting resets the Adam state. */
int tn_cost_model_params(tn_cost_model_t *model, float *h_params, int64_t capacity, int64_t *n_params,
                         int32_t set);
/* Mean-squared-error loss of n samples (h_x: n x TN_COST_NFEAT, h_t: n) and
 * its gradient with respect to every parameter (h_grad, may be NULL). */
int tn_cost_model_grad(tn_cost_model_t *model, const float *h_x, const float *h_t, int32_t n,
                       float *h_grad, double *loss, void *stream);
/* Adam on shuffled minibatches (splitmix64(seed) order), `epochs` passes. */
int tn_cost_model_train(tn_cost_model_t *model, const float *h_x, const float *h_t, int64_t n,
                        int32_t epochs, int32_t batch, float lr, uint64_t seed, double *final_loss,
                        void *stream);
int tn_cost_model_predict(tn_cost_model_t *model, const float *h_x, int64_t n, float *h_y,
                          void *stream);
/* Feature rows (n x TN_COST_NFEAT) of autotuner records. */
int tn_cost_features(const tn_tune_record *recs, int32_t n, float *out);
/* Training targets of autotuner records: log2 of each record's time in
 * microseconds (times below 1 ns count as 1 ns), the quantity the model
 * predicts. */
int tn_cost_targets(const tn_tune_record *recs, int32_t n, float *out);
/* Attach a model to a plan: with tile_policy TN_TILE_LEARNED the first
 * tn_contract picks every GEMM step's configuration by predicted time. */
int tn_plan_set_cost_model(tn_plan_t *plan, tn_cost_model_t *model);
/* Predicted milliseconds of contracting every slice of the plan (GEMM
 * steps under their current configuration + permutations). */
int tn_plan_predict_ms(tn_plan_t *plan, tn_cost_model_t *model, double *ms, void *stream);

/* ---- per-kernel timing (measurement, not for production runs) ---- */
#define TN_KC_LEAF 0        /* leaf preparation / slice decoding            */
#define TN_KC_PERMUTE 1     /* bit-permute transposes                       */
#define TN_KC_BPREP 2       /* B' padding for the tensor-core path          */
#define TN_KC_GEMM_TC 3     /* tcgen05 complex-as-real GEMM                 */
#define TN_KC_GEMM_LP 4     /* complex-half GEMM on CUDA cores              */
#define TN_KC_GEMM_C64 5    /* complex64 GEMMs on CUDA cores                */
#define TN_KC_SUM 6         /* FP64 cross-slice sum                          */
#define TN_KC_QUANT 7       /* E4M3 operand quantization (FP8 steps)         */
#define TN_KC_COUNT 8

typedef struct {
    int64_t launches;
    double ms;        /* summed CUDA-event durations of those launches       */
    double flops;     /* algorithmic real flops (8 M N K per GEMM)            */
    double bytes;     /* algorithmic bytes: operands read + result written   */
} tn_kernel_stats;

/* Record a CUDA event pair around every later launch of the kernel classes
 * in class_mask (bit TN_KC_*) made by tn_contract on this plan; 0 turns it
 * off.  Resets the counters. */
int tn_profile(tn_plan_t *plan, uint32_t class_mask);
/* Synchronize on the recorded events and return TN_KC_COUNT entries. */
int tn_profile_read(tn_plan_t *plan, tn_kernel_stats *out);

/* ---- single-kernel entry points (used by tests; same kernels as above) ---- */

/*
 * tn_permute: out = in with its rank-r dim-2 modes reordered (Sec. 3.1,
 * "index permutation"): out index bit (r-1-i) = in index bit (r-1-perm[i]),
 * i.e. output mode i (outermost first) is input mode perm[i].  Bit-exact
 * data movement.  elem_bytes: 4 (complex-half) or 8 (complex64).  in, out:
 * device, 2^r elements, non-overlapping.  r <= 34.
 */
int tn_permute(const void *in, void *out, int32_t rank, const int32_t *perm,
               int32_t elem_bytes, void *stream);

/*
 * tn_gemm: one contraction step as a GEMM, C[b][M][N] = sum_k A[b][M][K] *
 * B[b][K][N] on interleaved complex data (row-major; batch stride 0 for a
 * broadcast operand: pass batch_a / batch_b = 0 for no batch mode).
 *   dtype TN_C64: A, B, C complex64, FP32 accumulation; scale ignored.
 *   dtype TN_F16/TN_BF16: A, B, C complex-half (B is padded on the device to
 *   the real 2K x 2N form of Eq. 6 for the tensor-core variant); FP32
 *   accumulation; C is multiplied by 2^scale_exp before rounding.
 * kernel: -1 = automatic; otherwise a variant index (tests): 0 complex64
 *   rows, 1 complex64 tiled, 2 complex-half rows, 3 complex-half tensor
 *   cores, 4 complex-half tensor cores on CTA pairs (clusters of 2 SMs,
 *   256-row tiles; shapes with M >= 256, N >= 128, K >= 32, else as 3),
 *   5 complex-half tensor cores with 64-byte K chunks (K >= 32, else as 3),
 *   6 complex-half tensor cores with each CTA's B' slice resident in shared
 *   memory across its tiles (short K: the whole K of a B' tile within
 *   64 KiB, one K part; else as 3), 7 as 6 with the C tiles staged in
 *   shared memory and written by TMA stores (N >= 32; else as 6), 8 as 3
 *   with each warp's results staged in shared memory and stored in whole
 *   32-byte sectors (N >= 8; else as 3); with dtype TN_C64, 9 = the
 *   complex64 GEMM on the tensor cores: each FP32 operand of Eq. 6's real
 *   form split into a TF32 part and its remainder, A B'^T = A_hi B'_hi +
 *   A_hi B'_lo + A_lo B'_hi by three kind::tf32 MMAs per K slice, FP32
 *   accumulation (K >= 8; the split arrays are allocated per call).
 * out_max: optional device float, receives max |component| of the stored C.
 */
int tn_gemm(int32_t dtype, const void *A, const void *B, void *C, int64_t M, int64_t N,
            int64_t K, int64_t batch, int32_t batch_a, int32_t batch_b, int32_t scale_exp,
            int32_t kernel, float *out_max, void *stream);

/*
 * tn_gemm_gather: contraction of many tensor pairs in the sparse state (paper
 * Sec. 3.4.2).  A holds m_a chunks [m_a][M][K], B holds m_b chunks
 * [m_b][K][N], C receives m_n chunks [m_n][M][N], all complex-half (dtype
 * TN_F16 or TN_BF16, interleaved re/im, device memory, caller-owned):
 *
 *     C[n] = 2^scale_exp A[index_a[n]] B[index_b[n]]      (0 <= n < m_n)
 *
 * index_a, index_b: HOST int32 arrays of m_n entries in [0, m_a) and
 * [0, m_b); m_a, m_n <= 2^30, m_b <= 65535.  The tensor-core GEMM reads the operand chunks where they are
 * (TMA coordinates from the indices, no gathered copy).  scheme:
 *   TN_GATHER_DIRECT  one output chunk per n;
 *   TN_GATHER_PADDED  index_a non-decreasing: the paper's padded 2-D index,
 *                     P[i][r] = the B chunk of the r-th n paired with A chunk
 *                     i, -1 past its count (m_r columns, m_r = the largest
 *                     repeat count, written to *out_m_r if non-NULL); tiles
 *                     walk (i, r) so one A chunk serves all its r in turn,
 *                     the -1 places are computed and not stored, and C is
 *                     written straight at the valid places (the extraction).
 * M, N, K powers of two, N <= 2^24, 8 <= K <= 2^15.  out_max (device,
 * nullable) receives max |C| (atomic max on a zeroed float).  The per-call
 * index table is uploaded from host memory, so the call synchronizes
 * `stream` once, before the B' build and the GEMM are enqueued; device
 * scratch is allocated stream-ordered and freed after.
 * Errors: TN_EINVAL (NULL pointers, sizes, index out of range, unsorted
 * index_a for TN_GATHER_PADDED), TN_EUNSUPPORTED (K outside the range).
 */
/*
 * Low-precision codec for tensors that cross a link (paper Sec. 3.2, Eq. 1,
 * Table 1).  Per group i of a real FP32 tensor x[n] (a complex64 tensor as
 * its 2n interleaved reals):
 *     Q([x]_i) = [x]_i^exp * scale + zero,
 *     scale = (q_max - q_min) / (max - min),
 *     zero  = (q_min max - q_max min) / (max - min),
 * max / min over the group's transformed values, x^exp = sign(x)|x|^exp.
 *   TN_CODEC_HALF  q in +-65504, exp 1, one group (group = 0), not rounded;
 *                  codes: FP16[n]
 *   TN_CODEC_INT8  q in -128..127, exp 0.2, one group (group = 0), rounded to
 *                  nearest even; codes: int8[n]
 *   TN_CODEC_INT4  q in 0..15, exp 1, groups of `group` values (a power of
 *                  two in 128..65536 dividing n), rounded; codes: uint8[n/2],
 *                  two per byte, even index in the low nibble
 * scale, zero: device FP32[n / group] (one entry for the whole-tensor kinds).
 * A group of equal values gets scale 1 and zero q_min - value.  tn_decode
 * inverts Eq. 1 into x[n] (FP32).  All pointers are device memory,
 * caller-owned; enqueued on `stream` (tn_encode of the whole-tensor kinds
 * allocates a small stream-ordered scratch).  Errors: TN_EINVAL (NULL, bad
 * kind, group or n), TN_ECUDA.
 */
#define TN_CODEC_HALF 0
#define TN_CODEC_INT8 1
#define TN_CODEC_INT4 2
int tn_encode(int32_t kind, const float *x, int64_t n, int32_t group, void *codes, float *scale,
              float *zero, void *stream);
int tn_decode(int32_t kind, const void *codes, const float *scale, const float *zero, int64_t n,
              int32_t group, float *x, void *stream);

#define TN_GATHER_DIRECT 0
#define TN_GATHER_PADDED 1
int tn_gemm_gather(int32_t dtype, const void *A, int64_t m_a, const void *B, int64_t m_b, void *C,
                   int64_t m_n, int64_t M, int64_t N, int64_t K, const int32_t *index_a,
                   const int32_t *index_b, int32_t scheme, int32_t scale_exp, float *out_max,
                   int32_t *out_m_r, void *stream);

/*
 * tn_selftest_wait_timeout: failure-detection self-test.  Launches one small
 * tensor-core GEMM whose TMA producer is told to issue nothing, so the MMA
 * warp's bounded mbarrier wait runs out (about 2 s); the kernel then records
 * an error word, frees its tensor memory and returns.  Returns TN_ETIMEOUT
 * when the timeout was detected and reported (the expected outcome; the CUDA
 * context stays usable), TN_OK if not, TN_ECUDA on a CUDA error.
 * Synchronizes `stream`; allocates a few KiB of device memory.
 */
int tn_selftest_wait_timeout(void *stream);
/* The same on the CTA-pair kernel (one 256 x 256 tile on a cluster of 2):
 * both CTAs' waits run out, the pair meets at its teardown barrier and
 * frees its tensor memory.  Same return codes. */
int tn_selftest_wait_timeout_pair(void *stream);

const char *tn_strerror(int code);
const char *tn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TN_H_ */

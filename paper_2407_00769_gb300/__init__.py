"""GB300 sliced tensor-network contraction of random quantum circuits.

Thin binding over the C ABI in include/tn.h (library: _build/libtn.so).  This
module only marshals arguments: every step of the contraction runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  There is
no CPU fallback: if the library cannot be built or loaded, every call raises.

    from paper_2407_00769_gb300 import Plan, F16
    plan = Plan(circuit, query, dtype=F16, n_slice_edges=8)
    amps = plan.contract()               # torch complex128 on the GPU
    idx, prob = sample(amps, k=1)        # post-selection (top-k)
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build_mod

C64, F16, BF16, FP8 = 0, 1, 2, 3
TILE_FIXED, TILE_EXHAUSTIVE, TILE_LEARNED = 0, 1, 2
DTYPE_NAMES = {C64: "c64", F16: "f16", BF16: "bf16"}
KERNEL_NAMES = {0: "c64_rows", 1: "c64_tiled", 2: "lp_rows", 3: "lp_tc"}
GEMM_TC_PAIR = 4   # tn_gemm kernel index: tensor cores on CTA pairs
GEMM_TC_HALF_K = 5  # tn_gemm kernel index: tensor cores, 64-byte K chunks
GEMM_TC_BRES = 6    # tn_gemm kernel index: tensor cores, B' slice resident in shared memory
GEMM_TC_BRES_STORE = 7  # ... and C tiles written by TMA stores
GEMM_TC_STAGED = 8      # tensor cores, results stored in whole 32-byte sectors via staging
GEMM_C64_TC = 9         # complex64 on the tensor cores: TF32 parts, three MMAs per K slice

TN_OK, TN_EINVAL, TN_ENOMEM, TN_ECUDA, TN_ETIMEOUT, TN_EUNSUPPORTED = range(6)

EXPORTED = [
    "tn_plan", "tn_plan_samples", "tn_plan_opts_default", "tn_plan_info", "tn_plan_sliced_edges",
    "tn_plan_step",
    "tn_plan_leaf_source", "tn_plan_leaf_tensor", "tn_plan_decode_leaf", "tn_plan_step_scale",
    "tn_contract", "tn_contract_host", "tn_contract_batch", "tn_sample", "tn_metrics",
    "tn_plan_destroy", "tn_permute", "tn_gemm", "tn_strerror", "tn_last_error",
    "tn_profile", "tn_profile_read", "tn_sample_noalloc", "tn_selftest_wait_timeout",
    "tn_selftest_wait_timeout_pair",
    "tn_plan_set_graph", "tn_batch_create", "tn_batch_run", "tn_batch_destroy",
    "tn_plan_tune", "tn_tune_records",
    "tn_cost_model_create", "tn_cost_model_destroy", "tn_cost_model_params", "tn_cost_model_grad",
    "tn_cost_model_train", "tn_cost_model_predict", "tn_cost_features", "tn_plan_set_cost_model",
    "tn_plan_predict_ms", "tn_plan_apply_tuning", "tn_gemm_gather", "tn_encode", "tn_decode",
    "tn_queue_create", "tn_queue_run", "tn_queue_info", "tn_queue_set_wait_limit", "tn_queue_destroy",
    "tn_plan_set_queue", "tn_selftest_queue_timeout", "tn_cost_targets", "tn_queue_profile",
    "tn_queue_profile_read",
]
QK_NAMES = ["", "zero", "leaf", "permute", "permute_tiled", "bprep_gather", "bprep_c64", "gemm_rows",
            "gemm_tiled_c64", "gemm_tc", "splitk", "slice_sum"]
COST_NFEAT = 26
KC_NAMES = ["leaf", "permute", "bprep", "gemm_tc", "gemm_lp_rows", "gemm_c64", "slice_sum", "quant"]


class TnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class Gate(ctypes.Structure):
    _fields_ = [("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("re", ctypes.c_double * 16), ("im", ctypes.c_double * 16)]


class CircuitC(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_gates", ctypes.c_int32),
                ("gates", ctypes.POINTER(Gate))]


class QueryC(ctypes.Structure):
    _fields_ = [("n_open", ctypes.c_int32), ("open_qubits", ctypes.POINTER(ctypes.c_int32)),
                ("fixed_bits", ctypes.POINTER(ctypes.c_uint8))]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class PlanOpts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("max_log2_elems", ctypes.c_int32),
                ("n_slice_edges", ctypes.c_int32), ("path_seed", ctypes.c_uint64),
                ("path_trials", ctypes.c_int32), ("path_anneal_iters", ctypes.c_int32),
                ("slice_batch_log2", ctypes.c_int32),
                ("tile_policy", ctypes.c_int32), ("small_log2", ctypes.c_int32),
                ("no_tensor_cores", ctypes.c_int32),
                ("fp8_min_log2_flops", ctypes.c_int32),
                ("recompute_log2", ctypes.c_int32),
                ("no_scaling", ctypes.c_int32), ("anneal_kappa", ctypes.c_int32),
                ("workspace_budget", ctypes.c_int64),
                ("c64_tensor_cores", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_open", ctypes.c_int32),
                ("n_leaves", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("n_slice_edges", ctypes.c_int32), ("n_slices", ctypes.c_int64),
                ("n_steps", ctypes.c_int32), ("n_steps_invariant", ctypes.c_int32),
                ("max_log2_elems", ctypes.c_int32), ("slice_batch_log2", ctypes.c_int32),
                ("flops_per_slice", ctypes.c_double), ("flops_invariant", ctypes.c_double),
                ("bytes_per_slice", ctypes.c_double), ("workspace_bytes", ctypes.c_int64),
                ("n_permutes", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("leaf_bytes", ctypes.c_int64), ("n_recompute_edges", ctypes.c_int32)]


class ContractReport(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("flops", ctypes.c_double), ("slices", ctypes.c_int64),
                ("kernels", ctypes.c_int32), ("min_exp", ctypes.c_int32),
                ("max_exp", ctypes.c_int32)]


class QueueStats(ctypes.Structure):
    _fields_ = [("n_plans", ctypes.c_int32), ("n_ops", ctypes.c_int32), ("n_items", ctypes.c_int32),
                ("max_chain", ctypes.c_int32), ("ctas", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("table_bytes", ctypes.c_int64), ("flops", ctypes.c_double), ("slices", ctypes.c_int64)]


class QueueKindStats(ctypes.Structure):
    _fields_ = [("items", ctypes.c_int64), ("wait_ms", ctypes.c_double), ("busy_ms", ctypes.c_double)]


class KernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class TuneRecord(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("lm", ctypes.c_int32), ("ln", ctypes.c_int32),
                ("lk", ctypes.c_int32), ("lb", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("tile", ctypes.c_int32), ("step", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("ms", ctypes.c_double)]


class StepInfo(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int32), ("b", ctypes.c_int32), ("c", ctypes.c_int32),
                ("log2_m", ctypes.c_int32), ("log2_n", ctypes.c_int32),
                ("log2_k", ctypes.c_int32), ("log2_batch", ctypes.c_int32),
                ("permute_a", ctypes.c_int32), ("slice_invariant", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("permute_b", ctypes.c_int32), ("scale_headroom", ctypes.c_int32),
                ("storage", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build_mod.LIB


def build(force: bool = False) -> str:
    return _build_mod.build(force=force)


def lib():
    """Load libtn.so (building it first if needed).  Raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build_mod.build()
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.tn_plan.argtypes = [ctypes.POINTER(CircuitC), ctypes.POINTER(QueryC),
                              ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
        L.tn_plan_opts_default.argtypes = [ctypes.POINTER(PlanOpts)]
        L.tn_plan_samples.argtypes = [ctypes.POINTER(CircuitC), ctypes.POINTER(ctypes.c_uint8), i32,
                                      ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
        L.tn_plan_opts_default.restype = None
        L.tn_plan_info.argtypes = [vp, ctypes.POINTER(PlanStats)]
        L.tn_plan_sliced_edges.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), i32]
        L.tn_plan_step.argtypes = [vp, i32, ctypes.POINTER(StepInfo)]
        L.tn_plan_leaf_source.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.tn_plan_leaf_tensor.argtypes = [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                          ctypes.POINTER(i32), vp]
        L.tn_plan_decode_leaf.argtypes = [vp, i64, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                          ctypes.POINTER(i32), vp, vp]
        L.tn_plan_step_scale.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]
        L.tn_contract.argtypes = [vp, i64, i64, vp, ctypes.c_int, vp, ctypes.POINTER(ContractReport)]
        L.tn_contract_host.argtypes = [vp, i64, i64, vp, vp, ctypes.POINTER(ContractReport)]
        L.tn_contract_batch.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), vp]
        L.tn_sample.argtypes = [vp, i32, i32, vp, vp, vp]
        L.tn_metrics.argtypes = [vp, vp, i64, i32, vp, vp]
        L.tn_sample_noalloc.argtypes = [vp, i32, i32, vp, vp, vp]
        L.tn_selftest_wait_timeout.argtypes = [vp]
        L.tn_selftest_wait_timeout_pair.argtypes = [vp]
        L.tn_plan_set_graph.argtypes = [vp, ctypes.c_int]
        L.tn_plan_tune.argtypes = [vp, vp]
        L.tn_plan_apply_tuning.argtypes = [vp, ctypes.POINTER(TuneRecord), i32]
        f32p = ctypes.POINTER(ctypes.c_float)
        L.tn_cost_model_create.argtypes = [i32, ctypes.c_uint64, ctypes.POINTER(vp)]
        L.tn_cost_model_destroy.argtypes = [vp]
        L.tn_cost_model_destroy.restype = None
        L.tn_cost_model_params.argtypes = [vp, f32p, i64, ctypes.POINTER(i64), i32]
        L.tn_cost_model_grad.argtypes = [vp, f32p, f32p, i32, f32p, ctypes.POINTER(ctypes.c_double), vp]
        L.tn_cost_model_train.argtypes = [vp, f32p, f32p, i64, i32, i32, ctypes.c_float,
                                          ctypes.c_uint64, ctypes.POINTER(ctypes.c_double), vp]
        L.tn_cost_model_predict.argtypes = [vp, f32p, i64, f32p, vp]
        L.tn_cost_features.argtypes = [ctypes.POINTER(TuneRecord), i32, f32p]
        L.tn_cost_targets.argtypes = [ctypes.POINTER(TuneRecord), i32, f32p]
        L.tn_plan_set_cost_model.argtypes = [vp, vp]
        L.tn_plan_predict_ms.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double), vp]
        L.tn_tune_records.argtypes = [vp, ctypes.POINTER(TuneRecord), i32, ctypes.POINTER(i32)]
        L.tn_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), i32,
                                      ctypes.POINTER(vp)]
        L.tn_batch_run.argtypes = [vp, vp, ctypes.POINTER(ContractReport)]
        L.tn_batch_destroy.argtypes = [vp]
        L.tn_batch_destroy.restype = None
        L.tn_queue_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.tn_queue_run.argtypes = [vp, vp, ctypes.POINTER(ContractReport)]
        L.tn_queue_info.argtypes = [vp, ctypes.POINTER(QueueStats)]
        L.tn_queue_set_wait_limit.argtypes = [vp, i64]
        L.tn_queue_destroy.argtypes = [vp]
        L.tn_queue_destroy.restype = None
        L.tn_plan_set_queue.argtypes = [vp, ctypes.c_int]
        L.tn_queue_profile.argtypes = [vp, ctypes.c_int]
        L.tn_queue_profile_read.argtypes = [vp, ctypes.POINTER(QueueKindStats), i32]
        L.tn_selftest_queue_timeout.argtypes = [i32, vp]
        L.tn_plan_destroy.argtypes = [vp]
        L.tn_plan_destroy.restype = None
        L.tn_permute.argtypes = [vp, vp, i32, ctypes.POINTER(i32), i32, vp]
        L.tn_gemm.argtypes = [i32, vp, vp, vp, i64, i64, i64, i64, i32, i32, i32, i32, vp, vp]
        L.tn_encode.argtypes = [i32, vp, i64, i32, vp, vp, vp, vp]
        L.tn_decode.argtypes = [i32, vp, vp, vp, i64, i32, vp, vp]
        L.tn_gemm_gather.argtypes = [i32, vp, i64, vp, i64, vp, i64, i64, i64, i64,
                                     ctypes.POINTER(i32), ctypes.POINTER(i32), i32, i32, vp,
                                     ctypes.POINTER(i32), vp]
        L.tn_profile.argtypes = [vp, ctypes.c_uint32]
        L.tn_profile_read.argtypes = [vp, ctypes.POINTER(KernelStats)]
        L.tn_strerror.argtypes = [ctypes.c_int]
        L.tn_strerror.restype = ctypes.c_char_p
        L.tn_last_error.argtypes = []
        L.tn_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name not in ("tn_plan_opts_default", "tn_plan_destroy", "tn_strerror", "tn_last_error",
                            "tn_batch_destroy", "tn_cost_model_destroy", "tn_queue_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(rc: int):
    if rc != TN_OK:
        L = lib()
        raise TnError(rc, f"{L.tn_strerror(rc).decode()}: {L.tn_last_error().decode()}")


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def circuit_struct(circuit):
    """Marshal an rqcgen.Circuit into the C structs (kept alive by the caller)."""
    n_g = int(circuit.n_gates)
    gates = (Gate * max(1, n_g))()
    mats = np.asarray(circuit.mats, dtype=np.complex128).reshape(n_g, 16)
    for g in range(n_g):
        gates[g].q0 = int(circuit.q0[g])
        gates[g].q1 = int(circuit.q1[g])
        ctypes.memmove(gates[g].re, np.ascontiguousarray(mats[g].real).ctypes.data, 128)
        ctypes.memmove(gates[g].im, np.ascontiguousarray(mats[g].imag).ctypes.data, 128)
    c = CircuitC(int(circuit.n_qubits), n_g, gates)
    return c, gates


def query_struct(query, n_qubits):
    oq = np.ascontiguousarray(query.open_qubits, dtype=np.int32)
    fb = np.ascontiguousarray(query.fixed_bits, dtype=np.uint8)
    if fb.shape[0] != n_qubits:
        raise ValueError("fixed_bits must have one entry per qubit")
    q = QueryC(int(oq.shape[0]), oq.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
               fb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return q, (oq, fb)


class _TorchAllocator:
    """Routes the plan's workspace through PyTorch's caching allocator."""

    def __init__(self):
        torch = _torch()
        self._live = {}

        def alloc(nbytes, ctx):
            # an exception must not leave this callback: ctypes would hand the
            # library an undefined pointer.  Out of memory: release PyTorch's
            # cached blocks and try once more, else NULL (the library then
            # returns TN_ENOMEM)
            try:
                t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            except Exception:
                try:
                    torch.cuda.empty_cache()
                    t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
                except Exception:
                    return None
            p = t.data_ptr()
            self._live[p] = t
            return p

        def free(ptr, ctx):
            self._live.pop(int(ptr or 0), None)

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


class Plan:
    """A contraction plan (tn_plan): network, path, slicing and schedule."""

    def __init__(self, circuit, query, dtype: int = F16, max_log2_elems: int = 0,
                 n_slice_edges: int = 0, seed: int = 1, trials: int = 1,
                 slice_batch_log2: int = 0, tile_policy: int = TILE_FIXED,
                 torch_allocator: bool = True, small_log2: int = 0,
                 no_tensor_cores: bool = False, fp8_min_log2_flops: int = 0, anneal_iters: int = 0,
                 recompute_log2: int = 0, no_scaling: bool = False, workspace_budget: int = 0,
                 anneal_kappa: int = 0, c64_tensor_cores: bool = False, _samples=None):
        L = lib()
        self._c, self._gates = circuit_struct(circuit)
        if _samples is None:
            self._q, self._qkeep = query_struct(query, int(circuit.n_qubits))
        opts = PlanOpts()
        L.tn_plan_opts_default(ctypes.byref(opts))
        opts.dtype = int(dtype)
        opts.max_log2_elems = int(max_log2_elems)
        opts.n_slice_edges = int(n_slice_edges)
        opts.path_seed = int(seed)
        opts.path_trials = int(trials)
        opts.path_anneal_iters = int(anneal_iters)
        opts.anneal_kappa = int(anneal_kappa)
        opts.c64_tensor_cores = 1 if c64_tensor_cores else 0
        opts.workspace_budget = int(workspace_budget)
        opts.slice_batch_log2 = int(slice_batch_log2)
        opts.tile_policy = int(tile_policy)
        opts.small_log2 = int(small_log2)
        opts.no_tensor_cores = 1 if no_tensor_cores else 0
        opts.fp8_min_log2_flops = int(fp8_min_log2_flops)
        opts.recompute_log2 = int(recompute_log2)
        opts.no_scaling = 1 if no_scaling else 0
        self._alloc = None
        if torch_allocator:
            self._alloc = _TorchAllocator()
            opts.dev_alloc = self._alloc.alloc
            opts.dev_free = self._alloc.free
        self._opts = opts
        h = ctypes.c_void_p()
        if _samples is None:
            _check(L.tn_plan(ctypes.byref(self._c), ctypes.byref(self._q), ctypes.byref(opts),
                             ctypes.byref(h)))
            self._h = h
            self.n_open = int(query.n_open) if hasattr(query, "n_open") else len(query.open_qubits)
        else:
            sm = np.ascontiguousarray(_samples, dtype=np.uint8)
            if sm.ndim != 2 or sm.shape[1] != int(circuit.n_qubits):
                raise ValueError("samples must be (n_samples, n_qubits) bits")
            _check(L.tn_plan_samples(ctypes.byref(self._c), sm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                     int(sm.shape[0]), ctypes.byref(opts), ctypes.byref(h)))
            self._h = h
            self.n_open = int(self.info()["n_open"])
            self.n_samples = int(sm.shape[0])
        self.n_qubits = int(circuit.n_qubits)
        self.dtype = int(dtype)

    @classmethod
    def from_samples(cls, circuit, samples, **kw):
        """A plan for the amplitudes of arbitrary bitstrings (tn_plan_samples):
        samples is (n_samples, n_qubits) of 0/1; contract() returns 2^k
        amplitudes, entry s for bitstring s (k = ceil(log2 n_samples))."""
        return cls(circuit, None, _samples=samples, **kw)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().tn_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        s = PlanStats()
        _check(lib().tn_plan_info(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in PlanStats._fields_}

    def sliced_edges(self):
        n = self.info()["n_slice_edges"]
        q = (ctypes.c_int32 * max(1, n))()
        g = (ctypes.c_int32 * max(1, n))()
        _check(lib().tn_plan_sliced_edges(self._h, q, g, n))
        return [(int(q[j]), int(g[j])) for j in range(n)]

    def leaf_sources(self):
        """(gate, qubit) of every leaf: the circuit index of its two-qubit gate,
        or (-1, q) for a qubit no two-qubit gate touches."""
        out = []
        g, q = ctypes.c_int32(), ctypes.c_int32()
        for i in range(self.info()["n_leaves"]):
            _check(lib().tn_plan_leaf_source(self._h, i, ctypes.byref(g), ctypes.byref(q)))
            out.append((g.value, q.value))
        return out

    def leaf_tensor(self, i: int):
        """Leaf i before slicing: ([(qubit, after_gate) per leg], complex128
        array of shape (2,) * rank)."""
        L = lib()
        r = ctypes.c_int32(0)
        _check(L.tn_plan_leaf_tensor(self._h, int(i), 0, ctypes.byref(r), None, None, None))
        n = r.value
        q = (ctypes.c_int32 * max(1, n))()
        g = (ctypes.c_int32 * max(1, n))()
        data = np.zeros(1 << n, dtype=np.complex128)
        _check(L.tn_plan_leaf_tensor(self._h, int(i), n, ctypes.byref(r), q, g, data.ctypes.data))
        return [(int(q[p]), int(g[p])) for p in range(n)], data.reshape((2,) * n)

    def decode_leaf(self, slice_id: int, i: int, stream=None):
        """Leaf i as the device prepares it for the pass at slice_id (slice
        decoding): ([(qubit, after_gate) per kept leg], complex64 array)."""
        L = lib()
        r = ctypes.c_int32(0)
        _check(L.tn_plan_decode_leaf(self._h, int(slice_id), int(i), 0, ctypes.byref(r), None, None,
                                     None, None))
        n = r.value
        q = (ctypes.c_int32 * max(1, n))()
        g = (ctypes.c_int32 * max(1, n))()
        data = np.zeros(1 << n, dtype=np.complex64)
        _check(L.tn_plan_decode_leaf(self._h, int(slice_id), int(i), n, ctypes.byref(r), q, g,
                                     data.ctypes.data, _stream_ptr(stream)))
        return [(int(q[p]), int(g[p])) for p in range(n)], data.reshape((2,) * n)

    def step_scale(self, i: int):
        """(exponent E, stored max) of step i's output after the last pass."""
        e = ctypes.c_int32(0)
        m = ctypes.c_float(0)
        _check(lib().tn_plan_step_scale(self._h, int(i), ctypes.byref(e), ctypes.byref(m)))
        return e.value, m.value

    def steps(self):
        out = []
        for i in range(self.info()["n_steps"]):
            st = StepInfo()
            _check(lib().tn_plan_step(self._h, i, ctypes.byref(st)))
            out.append({f: getattr(st, f) for f, _ in StepInfo._fields_})
        return out

    def contract(self, slice_begin: int = 0, slice_count: Optional[int] = None, out=None,
                 accumulate: bool = False, stream=None, report: bool = False):
        """Sum of slices [slice_begin, slice_begin+slice_count) into a complex128
        CUDA tensor of 2^n_open amplitudes (``out`` if given)."""
        torch = _torch()
        n_slices = self.info()["n_slices"]
        if slice_count is None:
            slice_count = n_slices - slice_begin
        if out is None:
            out = torch.zeros(1 << self.n_open, dtype=torch.complex128, device="cuda")
        if out.dtype != torch.complex128 or not out.is_cuda or not out.is_contiguous() \
                or out.numel() != (1 << self.n_open):
            raise ValueError("out must be a contiguous CUDA complex128 tensor of 2^n_open")
        rep = ContractReport() if report else None
        _check(lib().tn_contract(self._h, int(slice_begin), int(slice_count), out.data_ptr(),
                                 1 if accumulate else 0, _stream_ptr(stream),
                                 ctypes.byref(rep) if rep is not None else None))
        if report:
            return out, {f: getattr(rep, f) for f, _ in ContractReport._fields_}
        return out

    def tune(self, stream=None):
        """Exhaustive autotuning of every GEMM step's (kernel, tile)."""
        _check(lib().tn_plan_tune(self._h, _stream_ptr(stream)))

    def apply_tuning(self, records):
        """Reuse other plans' autotuner records (same step signatures)."""
        n = len(records)
        arr = (TuneRecord * max(1, n))()
        for i, r in enumerate(records):
            for f, _ in TuneRecord._fields_:
                setattr(arr[i], f, r.get(f, 0))
        _check(lib().tn_plan_apply_tuning(self._h, arr, n))

    def tune_records(self):
        """Every timing the autotuner took, as a list of dicts."""
        n = ctypes.c_int32(0)
        _check(lib().tn_tune_records(self._h, None, 0, ctypes.byref(n)))
        arr = (TuneRecord * max(1, n.value))()
        _check(lib().tn_tune_records(self._h, arr, n.value, ctypes.byref(n)))
        return [{f: getattr(arr[i], f) for f, _ in TuneRecord._fields_} for i in range(n.value)]

    def set_cost_model(self, model):
        """Attach a CostModel (used by tile_policy=TILE_LEARNED)."""
        _check(lib().tn_plan_set_cost_model(self._h, model.handle if model else None))
        self._model = model

    def predict_ms(self, model, stream=None) -> float:
        out = ctypes.c_double(0)
        _check(lib().tn_plan_predict_ms(self._h, model.handle, ctypes.byref(out), _stream_ptr(stream)))
        return out.value

    def set_graph(self, enable: bool = True):
        """Capture tn_contract calls into a CUDA graph and replay identical ones."""
        _check(lib().tn_plan_set_graph(self._h, 1 if enable else 0))

    def set_queue(self, enable: bool = True):
        """Run every contract() call as one work-queue launch (tn_plan_set_queue)."""
        _check(lib().tn_plan_set_queue(self._h, 1 if enable else 0))
        return self

    def profile(self, classes=None):
        """Start per-kernel-class event timing (names from KC_NAMES; None: off)."""
        mask = 0
        for c in classes or []:
            mask |= 1 << KC_NAMES.index(c)
        _check(lib().tn_profile(self._h, mask))

    def profile_read(self) -> dict:
        arr = (KernelStats * len(KC_NAMES))()
        _check(lib().tn_profile_read(self._h, arr))
        return {KC_NAMES[i]: {f: getattr(arr[i], f) for f, _ in KernelStats._fields_}
                for i in range(len(KC_NAMES)) if arr[i].launches}

    def contract_host(self, slice_begin: int = 0, slice_count: Optional[int] = None, stream=None,
                      report: bool = False):
        """End to end from host memory: leaves uploaded, amplitudes downloaded."""
        n_slices = self.info()["n_slices"]
        if slice_count is None:
            slice_count = n_slices - slice_begin
        h = np.zeros(1 << self.n_open, dtype=np.complex128)
        rep = ContractReport() if report else None
        _check(lib().tn_contract_host(self._h, int(slice_begin), int(slice_count),
                                      h.ctypes.data, _stream_ptr(stream),
                                      ctypes.byref(rep) if rep is not None else None))
        if report:
            return h, {f: getattr(rep, f) for f, _ in ContractReport._fields_}
        return h


def plan_within_budget(circuit, query, dtype=F16, max_log2_elems=24, trials=4,
                       workspace_budget=1 << 30, **kw):
    """Plan with automatic slicing under a width cap, running as many of the
    slices together (slice_batch_log2) as fit in ``workspace_budget`` bytes
    (tn_plan_opts.workspace_budget: the library picks the batch)."""
    return Plan(circuit, query, dtype=dtype, n_slice_edges=-1, max_log2_elems=max_log2_elems,
                trials=trials, workspace_budget=workspace_budget, **kw)


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def cost_features(records) -> np.ndarray:
    """Feature rows (n x COST_NFEAT) of autotuner records (dicts)."""
    n = len(records)
    arr = (TuneRecord * max(1, n))()
    for i, r in enumerate(records):
        for f, _ in TuneRecord._fields_:
            setattr(arr[i], f, r.get(f, 0))
    out = np.zeros((n, COST_NFEAT), dtype=np.float32)
    _check(lib().tn_cost_features(arr, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def load_timings(path=None):
    """Autotuner timings saved by paper_2407_00769_gb300.data.collect_timings
    (default: the bundled GB300 set), as record dicts for cost_features /
    cost_targets.  Returns [] when the file is absent."""
    import os
    if path is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "timings_gb300.npz")
    if not os.path.exists(path):
        return []
    z = np.load(path)
    n = int(z["ms"].shape[0])
    keys = ("kind", "lm", "ln", "lk", "lb", "dtype", "kernel", "tile")
    cols = {k: z[k].tolist() for k in keys}
    ms = z["ms"].tolist()
    return [dict({k: cols[k][i] for k in keys}, step=-1, pad_=0, ms=ms[i]) for i in range(n)]


def _records(records):
    n = len(records)
    arr = (TuneRecord * max(1, n))()
    for i, r in enumerate(records):
        for f, _ in TuneRecord._fields_:
            setattr(arr[i], f, r.get(f, 0))
    return arr, n


def cost_targets(records) -> np.ndarray:
    """Training targets (tn_cost_targets): log2 of each record's time in
    microseconds."""
    arr, n = _records(records)
    out = np.zeros(n, dtype=np.float32)
    _check(lib().tn_cost_targets(arr, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


class CostModel:
    """The learned cost model (tn_cost_model_*): MLP trained on the GPU."""

    def __init__(self, hidden: int = 128, seed: int = 1):
        h = ctypes.c_void_p()
        _check(lib().tn_cost_model_create(int(hidden), int(seed), ctypes.byref(h)))
        self._h = h
        self.hidden = hidden

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().tn_cost_model_destroy(h)
            except Exception:
                pass
            self._h = None

    def params(self) -> np.ndarray:
        n = ctypes.c_int64(0)
        _check(lib().tn_cost_model_params(self._h, None, 0, ctypes.byref(n), 0))
        out = np.zeros(n.value, dtype=np.float32)
        _check(lib().tn_cost_model_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          n.value, ctypes.byref(n), 0))
        return out

    def set_params(self, p):
        a, ptr = _f32(p)
        n = ctypes.c_int64(0)
        _check(lib().tn_cost_model_params(self._h, ptr, a.size, ctypes.byref(n), 1))

    def grad(self, x, t, stream=None):
        xa, xp = _f32(x)
        ta, tp = _f32(t)
        g = np.zeros(self.params().size, dtype=np.float32)
        loss = ctypes.c_double(0)
        _check(lib().tn_cost_model_grad(self._h, xp, tp, int(ta.size),
                                        g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value, g

    def train(self, x, t, epochs=20, batch=256, lr=1e-3, seed=1, stream=None) -> float:
        xa, xp = _f32(x)
        ta, tp = _f32(t)
        loss = ctypes.c_double(0)
        _check(lib().tn_cost_model_train(self._h, xp, tp, int(ta.size), int(epochs), int(batch),
                                         float(lr), int(seed), ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value

    def predict(self, x, stream=None) -> np.ndarray:
        xa, xp = _f32(x)
        y = np.zeros(xa.shape[0], dtype=np.float32)
        _check(lib().tn_cost_model_predict(self._h, xp, xa.shape[0],
                                           y.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           _stream_ptr(stream)))
        return y


def contract_batch(plans, outs, stream=None):
    """One-shot batched contraction of independent plans (one CUDA graph)."""
    n = len(plans)
    hs = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    ds = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    _check(lib().tn_contract_batch(hs, n, ds, _stream_ptr(stream)))
    return outs


class Batch:
    """Many independent plans captured into one CUDA graph (tn_batch_*);
    run() replays it.  Keeps the plans and output tensors alive."""

    def __init__(self, plans, outs, n_streams: int = 16):
        self.plans, self.outs = list(plans), list(outs)
        n = len(self.plans)
        hs = (ctypes.c_void_p * n)(*[p.handle.value for p in self.plans])
        ds = (ctypes.c_void_p * n)(*[o.data_ptr() for o in self.outs])
        h = ctypes.c_void_p()
        _check(lib().tn_batch_create(hs, n, ds, int(n_streams), ctypes.byref(h)))
        self._h = h

    def run(self, stream=None, report: bool = False):
        rep = ContractReport() if report else None
        _check(lib().tn_batch_run(self._h, _stream_ptr(stream),
                                  ctypes.byref(rep) if rep is not None else None))
        if report:
            return {f: getattr(rep, f) for f, _ in ContractReport._fields_}
        return None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().tn_batch_destroy(h)
            except Exception:
                pass
            self._h = None


class Queue:
    """Many independent plans (or slice ranges) contracted in ONE persistent
    kernel launch (tn_queue_*): a device table of (op, tile) items in
    dependency order, claimed by one CTA per SM.  ranges: optional list of
    (slice_begin, slice_count) per plan (default: every slice).  run()
    launches it.  Keeps the plans and output tensors alive."""

    def __init__(self, plans, outs, ranges=None):
        self.plans, self.outs = list(plans), list(outs)
        n = len(self.plans)
        if len(self.outs) != n:
            raise ValueError("one output tensor per plan")
        for o, p in zip(self.outs, self.plans):
            if _amps_log2(o, "outs") != p.info()["n_open"]:
                raise ValueError("each output must hold 2^n_open amplitudes of its plan")
        hs = (ctypes.c_void_p * n)(*[p.handle.value for p in self.plans])
        ds = (ctypes.c_void_p * n)(*[o.data_ptr() for o in self.outs])
        b = c = None
        if ranges is not None:
            b = (ctypes.c_int64 * n)(*[int(r[0]) for r in ranges])
            c = (ctypes.c_int64 * n)(*[int(r[1]) for r in ranges])
        h = ctypes.c_void_p()
        _check(lib().tn_queue_create(hs, n, b, c, ds, ctypes.byref(h)))
        self._h = h

    def run(self, stream=None, report: bool = False):
        rep = ContractReport() if report else None
        _check(lib().tn_queue_run(self._h, _stream_ptr(stream),
                                  ctypes.byref(rep) if rep is not None else None))
        if report:
            return {f: getattr(rep, f) for f, _ in ContractReport._fields_}
        return None

    def info(self) -> dict:
        st = QueueStats()
        _check(lib().tn_queue_info(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in QueueStats._fields_ if f != "pad_"}

    def set_wait_limit(self, limit_us: int):
        _check(lib().tn_queue_set_wait_limit(self._h, int(limit_us)))

    def profile(self, enable: bool = True):
        """Per op kind: items, CTA-ms waiting for dependencies, CTA-ms running."""
        _check(lib().tn_queue_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        arr = (QueueKindStats * len(QK_NAMES))()
        _check(lib().tn_queue_profile_read(self._h, arr, len(QK_NAMES)))
        return {QK_NAMES[k]: {"items": arr[k].items, "wait_ms": arr[k].wait_ms, "busy_ms": arr[k].busy_ms}
                for k in range(1, len(QK_NAMES)) if arr[k].items}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().tn_queue_destroy(h)
            except Exception:
                pass
            self._h = None


def selftest_queue_timeout(limit_ms: int = 200, stream=None) -> int:
    """Status of a work queue whose second op waits for a count that is never
    reached (tn_selftest_queue_timeout): TN_ETIMEOUT when the bounded wait
    works."""
    return int(lib().tn_selftest_queue_timeout(int(limit_ms), _stream_ptr(stream)))


def _amps_log2(amps, name="amps") -> int:
    """log2 of the length of a contiguous CUDA complex128 amplitude tensor
    (the kernels read it as 2^n double2 values at its device address)."""
    torch = _torch()
    if not isinstance(amps, torch.Tensor) or amps.dtype != torch.complex128 or not amps.is_cuda \
            or not amps.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA complex128 tensor")
    n = amps.numel()
    n_open = n.bit_length() - 1
    if n < 1 or (1 << n_open) != n:
        raise ValueError(f"{name}: amplitude count must be a power of two")
    return n_open


def sample(amps, k: int = 1, stream=None):
    """Top-k post-selection: (indices, probabilities) as numpy arrays."""
    n_open = _amps_log2(amps)
    idx = np.zeros(k, dtype=np.int64)
    prob = np.zeros(k, dtype=np.float64)
    _check(lib().tn_sample(amps.data_ptr(), n_open, int(k), idx.ctypes.data, prob.ctypes.data,
                           _stream_ptr(stream)))
    return idx, prob


def sample_noalloc(amps, k: int = 1, stream=None):
    """tn_sample without device allocation (k <= 1024; see include/tn.h)."""
    n_open = _amps_log2(amps)
    idx = np.zeros(k, dtype=np.int64)
    prob = np.zeros(k, dtype=np.float64)
    _check(lib().tn_sample_noalloc(amps.data_ptr(), n_open, int(k), idx.ctypes.data,
                                   prob.ctypes.data, _stream_ptr(stream)))
    return idx, prob


def metrics(amps, ref=None, n_qubits: int = 0, stream=None) -> dict:
    """FP64 norm, rel-L2, fidelity and linear XEB of amps against ref (tn_metrics)."""
    _amps_log2(amps)
    if ref is not None:
        _amps_log2(ref, "ref")
        if ref.numel() != amps.numel():
            raise ValueError("ref must have as many amplitudes as amps")
    out = np.zeros(4, dtype=np.float64)
    _check(lib().tn_metrics(amps.data_ptr(), ref.data_ptr() if ref is not None else None,
                            int(amps.numel()), int(n_qubits), out.ctypes.data,
                            _stream_ptr(stream)))
    return {"norm2": out[0], "rel_l2": out[1], "fidelity": out[2], "xeb": out[3]}


def permute(x, perm, out=None, elem_bytes=None, stream=None):
    """Bit-permute a tensor of 2^r elements (4- or 8-byte elements; complex64
    tensors are 8-byte, anything else is read as 4-byte elements)."""
    torch = _torch()
    r = len(perm)
    if out is None:
        out = torch.empty_like(x)
    if elem_bytes is None:
        elem_bytes = 8 if x.dtype in (torch.complex64, torch.int64, torch.float64) else 4
    if elem_bytes not in (4, 8):
        raise ValueError("elem_bytes must be 4 or 8")
    for t, name in ((x, "x"), (out, "out")):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if t.numel() * t.element_size() != elem_bytes << r:
            raise ValueError(f"{name} must hold exactly 2^rank elements of elem_bytes bytes")
    if sorted(int(v) for v in perm) != list(range(r)):
        raise ValueError("perm must be a permutation of 0..rank-1")
    p = (ctypes.c_int32 * max(1, r))(*[int(v) for v in perm])
    _check(lib().tn_permute(x.data_ptr(), out.data_ptr(), r, p, int(elem_bytes),
                            _stream_ptr(stream)))
    return out


CODEC_HALF, CODEC_INT8, CODEC_INT4 = 0, 1, 2


def encode(kind, x, group=0, stream=None):
    """Eq. 1 codec (tn_encode) of a float32 CUDA tensor (complex64: its
    reals).  Returns (codes, scale, zero) CUDA tensors."""
    torch = _torch()
    xf = x.contiguous().view(torch.float32).reshape(-1)
    n = xf.numel()
    ng = 1 if kind != CODEC_INT4 else n // group
    if kind == CODEC_HALF:
        codes = torch.empty(n, dtype=torch.float16, device=xf.device)
    elif kind == CODEC_INT8:
        codes = torch.empty(n, dtype=torch.int8, device=xf.device)
    else:
        codes = torch.empty(n // 2, dtype=torch.uint8, device=xf.device)
    scale = torch.empty(ng, dtype=torch.float32, device=xf.device)
    zero = torch.empty(ng, dtype=torch.float32, device=xf.device)
    _check(lib().tn_encode(int(kind), xf.data_ptr(), n, int(group), codes.data_ptr(), scale.data_ptr(),
                           zero.data_ptr(), _stream_ptr(stream)))
    return codes, scale, zero


def decode(kind, codes, scale, zero, n, group=0, stream=None):
    """Inverse of encode (tn_decode): float32 CUDA tensor of n values."""
    torch = _torch()
    x = torch.empty(n, dtype=torch.float32, device=codes.device)
    _check(lib().tn_decode(int(kind), codes.data_ptr(), scale.data_ptr(), zero.data_ptr(), int(n), int(group),
                           x.data_ptr(), _stream_ptr(stream)))
    return x


GATHER_DIRECT, GATHER_PADDED = 0, 1


def gemm_gather(dtype, A, B, C, index_a, index_b, scheme=GATHER_DIRECT, scale_exp=0, out_max=None,
                stream=None):
    """Sparse-state contraction of many tensor pairs (tn_gemm_gather):
    C[n] = 2^scale_exp A[index_a[n]] B[index_b[n]]; A [m_a][M][K][2],
    B [m_b][K][N][2], C [m_n][M][N][2] complex-half CUDA tensors; the index
    arrays are host sequences.  Returns m_r (the padded index's columns)."""
    ia = np.ascontiguousarray(index_a, dtype=np.int32)
    ib = np.ascontiguousarray(index_b, dtype=np.int32)
    m_a, M, K = int(A.shape[0]), int(A.shape[1]), int(A.shape[2])
    m_b, N = int(B.shape[0]), int(B.shape[2])
    m_r = ctypes.c_int32(0)
    _check(lib().tn_gemm_gather(int(dtype), A.data_ptr(), m_a, B.data_ptr(), m_b, C.data_ptr(),
                                int(ia.shape[0]), M, N, K,
                                ia.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                ib.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(scheme),
                                int(scale_exp), out_max.data_ptr() if out_max is not None else None,
                                ctypes.byref(m_r), _stream_ptr(stream)))
    return m_r.value


def gemm(dtype, A, B, C, M, N, K, batch=1, batch_a=False, batch_b=False, scale_exp=0,
         kernel=-1, out_max=None, stream=None):
    _check(lib().tn_gemm(int(dtype), A.data_ptr(), B.data_ptr(), C.data_ptr(), int(M), int(N),
                         int(K), int(batch), 1 if batch_a else 0, 1 if batch_b else 0,
                         int(scale_exp), int(kernel),
                         out_max.data_ptr() if out_max is not None else None,
                         _stream_ptr(stream)))
    return C

"""ctypes binding of the C ABI declared in include/tn.h.

Argument marshalling only: every step of the contraction runs in the library
(host planner in C++, slices in CUDA kernels).  Device buffers are torch CUDA
tensors, passed by data pointer; streams are torch CUDA streams.  There is no
CPU fallback: if the shared library is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_NAME = "libtn_gb300.so"
LIB_PATH = os.path.join(_HERE, LIB_NAME)

TN_OK = 0
TN_ERR_ARG = -1
TN_ERR_OOM = -2
TN_ERR_CUDA = -3
TN_ERR_PLAN = -4
TN_ERR_TIMEOUT = -5
TN_ERR_UNSUPPORTED = -6
TN_ERR_DEVICE = -7

TN_TUNING_INTS = 5   # int32 per step in tn_plan_get_tuning / tn_plan_set_tuning

PREC = {"fp32": 0, "tf32": 1, "bf16x3": 2, "fp16x3": 3}
PREC_NAME = {v: k for k, v in PREC.items()}


class TnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tn status {status}: {msg}")
        self.status = status


class tn_circuit(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_gates", ctypes.c_int32),
                ("gate_qubits", ctypes.POINTER(ctypes.c_int32)),
                ("gate_matrices", ctypes.POINTER(ctypes.c_double)),
                ("gate_layer", ctypes.POINTER(ctypes.c_int32))]


class tn_plan_opts(ctypes.Structure):
    _fields_ = [("open_mask", ctypes.c_uint64), ("max_log2_intermediate", ctypes.c_int32),
                ("min_log2_slices", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("trials", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("complex_mult", ctypes.c_int32), ("log2_batch_slices", ctypes.c_int32),
                ("max_arena_bytes", ctypes.c_int64), ("n_forced_slices", ctypes.c_int32),
                ("forced_slice_qubit", ctypes.POINTER(ctypes.c_int32)),
                ("forced_slice_t", ctypes.POINTER(ctypes.c_int32)),
                ("mem_weight", ctypes.c_double), ("sm_pairs", ctypes.c_int32)]


class tn_plan_stats(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_open", ctypes.c_int32),
                ("n_leaves", ctypes.c_int32), ("n_steps", ctypes.c_int32),
                ("log2_slices", ctypes.c_int32), ("log2_batch_slices", ctypes.c_int32),
                ("log2_max_intermediate", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("flops_per_slice", ctypes.c_double), ("bytes_per_slice", ctypes.c_double),
                ("flops_per_chunk", ctypes.c_double), ("bytes_per_chunk", ctypes.c_double),
                ("arena_bytes", ctypes.c_int64), ("k_histogram", ctypes.c_int32 * 40),
                ("complex_mult", ctypes.c_int32), ("n_kernel_launches_per_chunk", ctypes.c_int32)]


# name -> (restype, argtypes); every symbol include/tn.h declares
_SIGS = {
    "tn_last_error": (ctypes.c_char_p, []),
    "tn_network_from_circuit": (ctypes.c_int, [ctypes.POINTER(tn_circuit), ctypes.POINTER(ctypes.c_void_p)]),
    "tn_network_wire_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "tn_network_destroy": (None, [ctypes.c_void_p]),
    "tn_plan_default_opts": (ctypes.c_int, [ctypes.POINTER(tn_plan_opts)]),
    "tn_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tn_plan_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "tn_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tn_plan_stats)]),
    "tn_plan_sliced_wires": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32)]),
    "tn_plan_step_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int32)] * 4),
    "tn_frugal_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    "tn_plan_select": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tn_plan_opts), ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_double)]),
    "tn_plan_select_list": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tn_plan_opts), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_double)]),
    "tn_plan_rank": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tn_plan_opts), ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                                    ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "tn_plan_tree": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32)]),
    "tn_plan_chunk_launches": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "tn_plan_batch_launches": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "tn_plan_model_time": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_double)]),
    "tn_plan_step_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "tn_contract_slices": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "tn_plan_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "tn_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "tn_plan_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32)]),
    "tn_plan_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "tn_plan_step_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "tn_plan_destroy": (None, [ctypes.c_void_p]),
    "tn_xeb": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                              ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "tn_permute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_int32), ctypes.c_int64, ctypes.c_void_p]),
    "tn_contract_pair": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                        ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "tn_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "tn_device_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "tn_contract_pair_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
}

_lib = None


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load the shared library (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} not built: run __graft_entry__.build() first")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(status: int) -> None:
    if status != TN_OK:
        msg = load().tn_last_error()
        raise TnError(status, msg.decode() if msg else "")


def _i32(seq) -> ctypes.Array:
    arr = (ctypes.c_int32 * max(1, len(seq)))()
    for i, v in enumerate(seq):
        arr[i] = int(v)
    return arr


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class Network:
    """tn_network_from_circuit: a circuit (rqcgen.Circuit or arrays) as a tensor network."""

    def __init__(self, circuit):
        lib = load()
        qs = np.ascontiguousarray(circuit.gate_qubits, dtype=np.int32)
        mats = circuit.flat_matrices()
        layers = np.ascontiguousarray(circuit.gate_layer, dtype=np.int32)
        c = tn_circuit(circuit.n_qubits, circuit.n_gates,
                       qs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                       mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       layers.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        h = ctypes.c_void_p()
        _check(lib.tn_network_from_circuit(ctypes.byref(c), ctypes.byref(h)))
        self.handle = h
        self.n_qubits = circuit.n_qubits

    def gates_per_qubit(self) -> List[int]:
        arr = (ctypes.c_int32 * self.n_qubits)()
        _check(load().tn_network_wire_counts(self.handle, arr, self.n_qubits))
        return list(arr)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_network_destroy(self.handle)
            self.handle = None


def default_opts() -> tn_plan_opts:
    o = tn_plan_opts()
    _check(load().tn_plan_default_opts(ctypes.byref(o)))
    return o


def _make_opts(open_mask, max_log2_intermediate, min_log2_slices, precision, complex_mult, seed, trials,
               log2_batch_slices, max_arena_bytes, forced_slices, mem_weight, sm_pairs=1):
    o = default_opts()
    o.open_mask = open_mask
    o.max_log2_intermediate = max_log2_intermediate
    o.min_log2_slices = min_log2_slices
    o.seed = seed
    o.trials = trials
    o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    o.complex_mult = complex_mult
    o.log2_batch_slices = log2_batch_slices
    if max_arena_bytes:
        o.max_arena_bytes = max_arena_bytes
    fq = _i32([q for q, _ in forced_slices])
    ft = _i32([t for _, t in forced_slices])
    o.n_forced_slices = len(forced_slices)
    o.forced_slice_qubit = ctypes.cast(fq, ctypes.POINTER(ctypes.c_int32))
    o.forced_slice_t = ctypes.cast(ft, ctypes.POINTER(ctypes.c_int32))
    o.mem_weight = float(mem_weight)
    o.sm_pairs = int(sm_pairs)
    return o, (fq, ft)


class Plan:
    """tn_plan: contraction order + slice set + device step program (host only)."""

    def __init__(self, network: Network, open_mask: int = 0, max_log2_intermediate: int = 30,
                 min_log2_slices: int = 0, precision: str = "fp32", complex_mult: int = 4,
                 seed: int = 1, trials: int = 64, log2_batch_slices: int = 0,
                 max_arena_bytes: int = 0,
                 forced_slices: Sequence[Tuple[int, int]] = (), mem_weight: float = 0.0,
                 sm_pairs: int = 1, _handle=None):
        self.network = network
        self.open_mask = open_mask
        if _handle is not None:
            self.handle = _handle
            return
        o, keep = _make_opts(open_mask, max_log2_intermediate, min_log2_slices, precision, complex_mult, seed,
                             trials, log2_batch_slices, max_arena_bytes, forced_slices, mem_weight, sm_pairs)
        h = ctypes.c_void_p()
        _check(load().tn_plan(network.handle, ctypes.byref(o), ctypes.byref(h)))
        self.handle = h

    def info(self) -> dict:
        s = tn_plan_stats()
        _check(load().tn_plan_info(self.handle, ctypes.byref(s)))
        d = {name: getattr(s, name) for name, _ in tn_plan_stats._fields_}
        d["k_histogram"] = list(s.k_histogram)
        return d

    def sliced_wires(self) -> List[Tuple[int, int]]:
        cnt = ctypes.c_int32()
        q = (ctypes.c_int32 * 64)()
        t = (ctypes.c_int32 * 64)()
        _check(load().tn_plan_sliced_wires(self.handle, q, t, 64, ctypes.byref(cnt)))
        return [(q[j], t[j]) for j in range(cnt.value)]

    def step_shapes(self) -> List[Tuple[int, int, int, int]]:
        n = self.info()["n_steps"]
        out = []
        a, b, c, d = (ctypes.c_int32() for _ in range(4))
        for i in range(n):
            _check(load().tn_plan_step_shape(self.handle, i, ctypes.byref(a), ctypes.byref(b),
                                             ctypes.byref(c), ctypes.byref(d)))
            out.append((a.value, b.value, c.value, d.value))
        return out

    def step_layout(self, i: int) -> dict:
        """Bit positions of step i's operands (A streamed, B small, C result):
        keys a_m, a_k, b_k, b_n, c_m, c_n, a_b, b_b, c_b; dep_flags (bit 0:
        depends on the slice id, bit 1: on the closed output bits); group (steps
        with one id >= 0 run concurrently; -1: alone)."""
        buf = (ctypes.c_int32 * 256)()
        cnt = ctypes.c_int32()
        _check(load().tn_plan_step_layout(self.handle, i, buf, 256, ctypes.byref(cnt)))
        v = list(buf[:cnt.value])
        nm, nk, nn, nb = v[:4]
        out, pos = {}, 4
        for key, n in (("a_m", nm), ("a_k", nk), ("b_k", nk), ("b_n", nn), ("c_m", nm), ("c_n", nn),
                       ("a_b", nb), ("b_b", nb), ("c_b", nb)):
            out[key] = v[pos:pos + n]
            pos += n
        out["dep_flags"] = v[pos]
        out["group"] = v[pos + 1]
        return out

    def tree(self, n_gates: int) -> Tuple[List[int], List[Tuple[int, int]]]:
        """tn_plan_tree: (leaf of every circuit gate, the two node ids of every
        step in execution order; leaves first, step j creates node n_leaves + j)."""
        n_steps = self.info()["n_steps"]
        log = (ctypes.c_int32 * max(1, n_gates))()
        nodes = (ctypes.c_int32 * max(2, 2 * n_steps))()
        nl, ns = ctypes.c_int32(), ctypes.c_int32()
        _check(load().tn_plan_tree(self.handle, log, n_gates, nodes, n_steps, ctypes.byref(nl), ctypes.byref(ns)))
        return list(log[:n_gates]), [(nodes[2 * j], nodes[2 * j + 1]) for j in range(ns.value)]

    def model_time(self, peak_flops: float, peak_bytes: float) -> float:
        """tn_plan_model_time: modeled seconds of one chunk on a roofline
        (peak_flops in algorithmic flop/s, peak_bytes in B/s)."""
        s = ctypes.c_double()
        _check(load().tn_plan_model_time(self.handle, peak_flops, peak_bytes, ctypes.byref(s)))
        return s.value

    def chunk_launches(self) -> int:
        """Kernels one chunk launches with the kernels chosen so far (after the first contract call)."""
        n = ctypes.c_int32()
        _check(load().tn_plan_chunk_launches(self.handle, ctypes.byref(n)))
        return n.value

    def batch_launches(self) -> int:
        """Kernels the per-batch prologue launches for a new bitstring (after the first contract call)."""
        n = ctypes.c_int32()
        _check(load().tn_plan_batch_launches(self.handle, ctypes.byref(n)))
        return n.value

    def contract_slices(self, slice_first: int, slice_count: int, bitstrings: Sequence[int],
                        out, stream=None) -> None:
        """Add the slices' contribution to `out` (torch complex128 CUDA tensor of
        n_batches * 2^k amplitudes)."""
        bs = (ctypes.c_uint64 * len(bitstrings))(*[int(b) for b in bitstrings])
        _check(load().tn_contract_slices(self.handle, slice_first, slice_count, bs, len(bitstrings),
                                         ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))

    KERNELS = {0: "simt64x64", 1: "simt128x16", 2: "simt256x4", 3: "tc_tf32", 4: "tc_bf16x3",
               5: "tc_tf32_3m", 6: "tc_bf16x3_3m", 7: "tc_fp16x3", 8: "tc_fp16x3_3m"}

    def step_times(self, reps: int = 3, stream=None) -> List[Tuple[float, str]]:
        """(mean device milliseconds per launch, kernel name) of every step."""
        n = self.info()["n_steps"]
        arr = (ctypes.c_double * max(1, n))()
        kid = (ctypes.c_int32 * max(1, n))()
        _check(load().tn_plan_step_times(self.handle, reps, arr, kid, _stream_handle(stream)))
        return [(arr[i], self.KERNELS.get(kid[i], str(kid[i]))) for i in range(n)]

    def autotune(self, reps: int = 2, stream=None) -> None:
        """Pick the fastest kernel / tile for every step by timing (tn_plan_autotune)."""
        _check(load().tn_plan_autotune(self.handle, reps, _stream_handle(stream)))

    def get_tuning(self) -> List[List[int]]:
        """tn_plan_get_tuning: per step [kernel id, log2 tile width, write-back,
        B' slots, SM pair] of the kernels in use (after one contract call)."""
        n = self.info()["n_steps"]
        buf = (ctypes.c_int32 * max(1, n * TN_TUNING_INTS))()
        cnt = ctypes.c_int32()
        _check(load().tn_plan_get_tuning(self.handle, buf, n * TN_TUNING_INTS, ctypes.byref(cnt)))
        v = list(buf[:cnt.value])
        return [v[i:i + TN_TUNING_INTS] for i in range(0, len(v), TN_TUNING_INTS)]

    def set_tuning(self, tuning: Sequence[Sequence[int]]) -> None:
        """tn_plan_set_tuning: use the given per-step kernel choices (after one contract call)."""
        flat = [int(x) for row in tuning for x in row]
        _check(load().tn_plan_set_tuning(self.handle, _i32(flat), len(flat)))

    def sync(self, stream=None) -> None:
        _check(load().tn_plan_sync(self.handle, _stream_handle(stream)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_plan_destroy(self.handle)
            self.handle = None


def xeb(amplitudes, n_qubits: int, stream=None) -> float:
    """tn_xeb on a complex128 CUDA tensor."""
    f = ctypes.c_double()
    _check(load().tn_xeb(ctypes.c_void_p(amplitudes.data_ptr()), amplitudes.numel(), n_qubits,
                         ctypes.byref(f), _stream_handle(stream)))
    return f.value


def selftest_bounded_wait(wait_ms: int = 200, stream=None) -> int:
    """Run the bounded-wait self-test kernel; returns the device status word."""
    st = ctypes.c_int32()
    _check(load().tn_selftest_bounded_wait(wait_ms, ctypes.byref(st), _stream_handle(stream)))
    return st.value


def device_sync(stream=None) -> None:
    """tn_device_sync: wait for the stream and raise TnError if a kernel of a
    call without a plan reported an error since the last call (the word is
    cleared)."""
    _check(load().tn_device_sync(_stream_handle(stream)))


def contract_pair_noalloc(a, a_wires, b, b_wires, c, c_wires, batch: int = 1, precision: str = "fp32",
                          complex_mult: int = 4, stream=None) -> None:
    """tn_contract_pair_noalloc on complex64 CUDA tensors (scratch from the
    library's static device array; nothing is allocated)."""
    p = PREC[precision] if isinstance(precision, str) else int(precision)
    _check(load().tn_contract_pair_noalloc(ctypes.c_void_p(a.data_ptr()), _i32(a_wires), len(a_wires),
                                           ctypes.c_void_p(b.data_ptr()), _i32(b_wires), len(b_wires),
                                           ctypes.c_void_p(c.data_ptr()), _i32(c_wires), len(c_wires),
                                           batch, p, complex_mult, _stream_handle(stream)))


def permute(inp, out, rank: int, perm: Sequence[int], batch: int = 1, stream=None) -> None:
    """tn_permute on complex64 CUDA tensors."""
    _check(load().tn_permute(ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(out.data_ptr()), rank,
                             _i32(perm), batch, _stream_handle(stream)))


def contract_pair(a, a_wires, b, b_wires, c, c_wires, batch: int = 1, precision: str = "fp32",
                  complex_mult: int = 4, stream=None) -> None:
    """tn_contract_pair on complex64 CUDA tensors."""
    p = PREC[precision] if isinstance(precision, str) else int(precision)
    _check(load().tn_contract_pair(ctypes.c_void_p(a.data_ptr()), _i32(a_wires), len(a_wires),
                                   ctypes.c_void_p(b.data_ptr()), _i32(b_wires), len(b_wires),
                                   ctypes.c_void_p(c.data_ptr()), _i32(c_wires), len(c_wires),
                                   batch, p, complex_mult, _stream_handle(stream)))


def frugal_sample(amplitudes, n_qubits: int, m_bound: float, candidates, uniforms, stream=None) -> List[int]:
    """tn_frugal_sample: amplitudes complex128 CUDA tensor [count]; candidates
    int64 and uniforms float64 CUDA tensors [n_samples, n_draws]; returns the
    accepted draw of each sample (-1 if none)."""
    n_samples, n_draws = (int(candidates.shape[0]), int(candidates.shape[1])) if candidates.dim() == 2 \
        else (1, int(candidates.numel()))
    out = (ctypes.c_int64 * n_samples)()
    _check(load().tn_frugal_sample(ctypes.c_void_p(amplitudes.data_ptr()), amplitudes.numel(), n_qubits,
                                   float(m_bound), ctypes.c_void_p(candidates.data_ptr()),
                                   ctypes.c_void_p(uniforms.data_ptr()), n_draws, n_samples, out,
                                   _stream_handle(stream)))
    return list(out)


def select_plan(network: Network, n_candidates: int, bitstring: int, stream=None, open_mask: int = 0,
                max_log2_intermediate: int = 30, min_log2_slices: int = 0, precision: str = "fp32",
                complex_mult: int = 4, seed: int = 1, trials: int = 64, log2_batch_slices: int = 0,
                max_arena_bytes: int = 0, forced_slices: Sequence[Tuple[int, int]] = (),
                mem_weight: float = 0.0) -> Tuple["Plan", List[float]]:
    """tn_plan_select: the fastest of n_candidates plans by measured chunk time;
    returns the plan and every candidate's estimated seconds for all slices."""
    o, keep = _make_opts(open_mask, max_log2_intermediate, min_log2_slices, precision, complex_mult, seed, trials,
                         log2_batch_slices, max_arena_bytes, forced_slices, mem_weight)
    h = ctypes.c_void_p()
    est = (ctypes.c_double * n_candidates)()
    _check(load().tn_plan_select(network.handle, ctypes.byref(o), n_candidates, bitstring,
                                 _stream_handle(stream), ctypes.byref(h), est))
    return Plan(network, open_mask=open_mask, _handle=h), list(est)


def rank_plans(network: Network, seeds: Sequence[int], mem_weights: Sequence[float], peak_flops: float,
               peak_bytes: float, open_mask: int = 0, max_log2_intermediate: int = 30, min_log2_slices: int = 0,
               precision: str = "fp32", complex_mult: int = 4, trials: int = 64, log2_batch_slices: int = 0,
               max_arena_bytes: int = 0, forced_slices: Sequence[Tuple[int, int]] = ()) -> List[float]:
    """tn_plan_rank: modeled seconds for all slices of every candidate (seed,
    memory weight), -1 where a candidate cannot be planned (host only)."""
    n = len(seeds)
    if n != len(mem_weights):
        raise ValueError("seeds and mem_weights differ in length")
    o, keep = _make_opts(open_mask, max_log2_intermediate, min_log2_slices, precision, complex_mult, 1, trials,
                         log2_batch_slices, max_arena_bytes, forced_slices, 0.0)
    sd = (ctypes.c_uint64 * n)(*[int(x) for x in seeds])
    wt = (ctypes.c_double * n)(*[float(x) for x in mem_weights])
    out = (ctypes.c_double * n)()
    _check(load().tn_plan_rank(network.handle, ctypes.byref(o), n, sd, wt, float(peak_flops), float(peak_bytes),
                               out))
    return list(out)


def select_plan_list(network: Network, seeds: Sequence[int], mem_weights: Sequence[float], bitstring: int,
                     stream=None, open_mask: int = 0, max_log2_intermediate: int = 30, min_log2_slices: int = 0,
                     precision: str = "fp32", complex_mult: int = 4, trials: int = 64, log2_batch_slices: int = 0,
                     max_arena_bytes: int = 0, forced_slices: Sequence[Tuple[int, int]] = ()
                     ) -> Tuple["Plan", List[float]]:
    """tn_plan_select_list: the fastest of the given candidates (seed, memory
    weight) by measured chunk time; returns the plan and every candidate's
    estimated seconds for all slices (-1: could not run)."""
    n = len(seeds)
    if n != len(mem_weights):
        raise ValueError("seeds and mem_weights differ in length")
    o, keep = _make_opts(open_mask, max_log2_intermediate, min_log2_slices, precision, complex_mult, 1, trials,
                         log2_batch_slices, max_arena_bytes, forced_slices, 0.0)
    sd = (ctypes.c_uint64 * n)(*[int(x) for x in seeds])
    wt = (ctypes.c_double * n)(*[float(x) for x in mem_weights])
    est = (ctypes.c_double * n)()
    h = ctypes.c_void_p()
    _check(load().tn_plan_select_list(network.handle, ctypes.byref(o), n, sd, wt, bitstring,
                                      _stream_handle(stream), ctypes.byref(h), est))
    return Plan(network, open_mask=open_mask, _handle=h), list(est)

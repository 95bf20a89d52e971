"""Python binding of libsv.so: the same calls as ``include/sv.h``, argument
marshalling only.

Device memory and streams come from PyTorch: a state is a CUDA tensor of
dtype complex64 or complex128 with 2^n elements, owned by the caller (the
library borrows its pointer, as the paper's relaxed memory model has it,
Sec. II-A). Every step of the computation runs in the CUDA library; there is
no CPU or PyTorch fallback, and loading fails loudly when ``libsv.so`` is
missing.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "SvError", "lib", "sv_create", "sv_destroy", "sv_set_stream", "sv_set_state_pointer", "sv_set_state",
    "sv_set_basis_state", "sv_copy_from_host", "sv_copy_to_host", "sv_copy_from_host_async",
    "sv_copy_to_host_async", "sv_apply_matrix",
    "sv_apply_fused", "sv_fuse_plan", "sv_expectation_pauli", "sv_measure_probs", "sv_collapse",
    "sv_measure", "sv_norm2", "sv_check_device_status", "sv_launch_count", "sv_status_string",
    "SV_C64", "SV_C128", "SV_PREC_NATIVE", "SV_PREC_TF32", "SV_PREC_SPLIT_BF16", "StateVector",
    "EXPORTED",
]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsv.so")

SV_C64, SV_C128 = 0, 1
SV_PREC_NATIVE, SV_PREC_TF32, SV_PREC_SPLIT_BF16 = 0, 1, 2
SV_MAX_TARGETS, SV_MAX_CONTROLS = 6, 24
STATUS = {0: "SV_OK", 1: "SV_ERR_INVALID_ARGUMENT", 2: "SV_ERR_NOT_SUPPORTED",
          3: "SV_ERR_INSUFFICIENT_WORKSPACE", 4: "SV_ERR_CUDA", 5: "SV_ERR_TIMEOUT", 6: "SV_ERR_ALLOC"}

# every entry point declared in include/sv.h
EXPORTED = [
    "sv_create", "sv_destroy", "sv_set_stream", "sv_set_state_pointer", "sv_set_basis_state",
    "sv_copy_from_host", "sv_copy_to_host", "sv_apply_matrix", "sv_apply_fused", "sv_fuse_plan",
    "sv_expectation_pauli", "sv_measure_probs", "sv_collapse", "sv_measure", "sv_norm2",
    "sv_check_device_status", "sv_launch_count", "sv_status_string", "sv_expectation_pauli_noalloc",
    "sv_batch_create", "sv_batch_destroy", "sv_batch_compile", "sv_batch_info", "sv_batch_program_stats",
    "sv_batch_launch",
    "sv_batch_results", "sv_swap_index_bits", "sv_apply_pauli_rotation", "sv_sample",
    "sv_check_bounded_wait", "sv_apply_fused_ex", "sv_fuse_plan_ex", "sv_copy_from_host_async",
    "sv_copy_to_host_async", "sv_batch_compile_ex", "sv_set_state", "sv_pool_create", "sv_pool_destroy",
    "sv_pool_alloc", "sv_pool_free", "sv_pool_stats",
]


class SvError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


class sv_fusion_options_t(C.Structure):
    _fields_ = [("max_fused_qubits", C.c_int), ("max_fused_diagonal_qubits", C.c_int), ("precision", C.c_int)]


class sv_gate_t(C.Structure):
    _fields_ = [("n_targets", C.c_int), ("targets", C.c_int * SV_MAX_TARGETS),
                ("n_controls", C.c_int), ("controls", C.c_int * SV_MAX_CONTROLS),
                ("control_values", C.c_int * SV_MAX_CONTROLS), ("matrix", C.POINTER(C.c_double))]


_lib = None
_VP, _I, _D = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)


def lib():
    """Load libsv.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2308_01999_gb300._build` (no fallback exists)")
        L = C.CDLL(LIB_PATH)
        sig = {
            "sv_create": [C.c_int, C.c_int, _VP, _VP, C.POINTER(_VP)],
            "sv_destroy": [_VP], "sv_set_stream": [_VP, _VP], "sv_set_state_pointer": [_VP, _VP],
            "sv_set_state": [_VP, C.c_int, C.c_int, _VP], "sv_set_basis_state": [_VP, C.c_uint64],
            "sv_copy_from_host": [_VP, _VP], "sv_copy_to_host": [_VP, _VP],
            "sv_copy_from_host_async": [_VP, _VP], "sv_copy_to_host_async": [_VP, _VP],
            "sv_apply_matrix": [_VP, _I, C.c_int, _I, _I, C.c_int, _D, C.c_int],
            "sv_apply_fused": [_VP, C.POINTER(sv_gate_t), C.c_int, C.c_int, C.c_int, _I],
            "sv_fuse_plan": [C.POINTER(sv_gate_t), C.c_int, C.c_int, C.c_int, C.c_int, _I, _I, _I, _D],
            "sv_expectation_pauli": [_VP, _I, _I, C.c_int, C.c_int, _D],
            "sv_measure_probs": [_VP, _I, C.c_int, _D, _D],
            "sv_collapse": [_VP, _I, C.c_int, C.c_int, C.c_double],
            "sv_measure": [_VP, _I, C.c_int, C.c_double, C.c_int, _I],
            "sv_norm2": [_VP, _D], "sv_check_device_status": [_VP],
            "sv_launch_count": [_VP, C.POINTER(C.c_uint64)],
            "sv_expectation_pauli_noalloc": [C.c_int, C.c_int, _VP, _VP, _I, _I, C.c_int, C.c_int, _D],
            "sv_batch_create": [_VP, C.POINTER(_VP)], "sv_batch_destroy": [_VP],
            "sv_batch_compile": [_VP, _VP, C.c_int, _VP, C.c_int, _I, C.c_int],
            "sv_batch_compile_ex": [_VP, _VP, C.c_int, _VP, C.c_int, _I, _VP],
            "sv_batch_info": [_VP, _I, _I, _I, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)],
            "sv_batch_program_stats": [_VP, C.POINTER(C.c_uint64)],
            "sv_batch_launch": [_VP, C.c_int, _VP, C.c_int],
            "sv_batch_results": [_VP, _D, C.c_int],
            "sv_swap_index_bits": [_VP, _I, C.c_int],
            "sv_apply_pauli_rotation": [_VP, C.c_double, _I, _I, C.c_int],
            "sv_sample": [_VP, _D, C.c_int, C.POINTER(C.c_int64)],
            "sv_check_bounded_wait": [_VP, C.c_longlong],
            "sv_pool_create": [_VP, C.c_uint64, C.c_uint64, C.POINTER(_VP)], "sv_pool_destroy": [_VP],
            "sv_pool_alloc": [_VP, C.c_uint64, C.POINTER(_VP)], "sv_pool_free": [_VP, _VP],
            "sv_pool_stats": [_VP, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)],
            "sv_apply_fused_ex": [_VP, C.POINTER(sv_gate_t), C.c_int, C.POINTER(sv_fusion_options_t), _I],
            "sv_fuse_plan_ex": [C.POINTER(sv_gate_t), C.c_int, C.c_int, C.POINTER(sv_fusion_options_t), C.c_int, _I,
                                _I, _I, _D],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.sv_status_string.argtypes = [C.c_int]
        L.sv_status_string.restype = C.c_char_p
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise SvError(code, where)


def _ints(xs):
    a = np.ascontiguousarray(np.asarray(list(xs) if not isinstance(xs, np.ndarray) else xs,
                                        dtype=np.int32).reshape(-1))
    return a, (a.ctypes.data_as(_I) if a.size else None)


def _cmat(m):
    a = np.ascontiguousarray(np.asarray(m, dtype=np.complex128))
    return a, a.ctypes.data_as(_D)


# ---- thin wrappers with the ABI's names ----

def sv_status_string(code: int) -> str:
    return lib().sv_status_string(int(code)).decode()


def sv_create(n_qubits: int, dtype: int, d_state_ptr: int, stream_ptr: int = 0) -> int:
    h = _VP()
    _check(lib().sv_create(int(n_qubits), int(dtype), _VP(d_state_ptr), _VP(stream_ptr), C.byref(h)), "sv_create")
    return h.value


def sv_destroy(h: int):
    _check(lib().sv_destroy(_VP(h)), "sv_destroy")


def sv_set_stream(h: int, stream_ptr: int):
    _check(lib().sv_set_stream(_VP(h), _VP(stream_ptr)), "sv_set_stream")


def sv_set_state_pointer(h: int, d_state_ptr: int):
    _check(lib().sv_set_state_pointer(_VP(h), _VP(d_state_ptr)), "sv_set_state_pointer")


def sv_set_state(h: int, n_qubits: int, dtype: int, d_state_ptr: int):
    _check(lib().sv_set_state(_VP(h), int(n_qubits), int(dtype), _VP(d_state_ptr)), "sv_set_state")


def sv_set_basis_state(h: int, index: int):
    _check(lib().sv_set_basis_state(_VP(h), C.c_uint64(index)), "sv_set_basis_state")


def sv_copy_from_host(h: int, host_ptr: int):
    _check(lib().sv_copy_from_host(_VP(h), _VP(host_ptr)), "sv_copy_from_host")


def sv_copy_to_host(h: int, host_ptr: int):
    _check(lib().sv_copy_to_host(_VP(h), _VP(host_ptr)), "sv_copy_to_host")


def sv_copy_from_host_async(h: int, host_ptr: int):
    _check(lib().sv_copy_from_host_async(_VP(h), _VP(host_ptr)), "sv_copy_from_host_async")


def sv_copy_to_host_async(h: int, host_ptr: int):
    _check(lib().sv_copy_to_host_async(_VP(h), _VP(host_ptr)), "sv_copy_to_host_async")


def sv_apply_matrix(h: int, targets, matrix, controls=(), control_values=None, adjoint: bool = False):
    t, tp = _ints(targets)
    c, cp = _ints(controls)
    if control_values is not None and len(control_values):
        cv, cvp = _ints(control_values)
    else:
        cv, cvp = None, None
    m, mp = _cmat(matrix)
    if m.shape != (1 << t.size, 1 << t.size):
        raise ValueError("matrix shape does not match the number of targets")
    _check(lib().sv_apply_matrix(_VP(h), tp, int(t.size), cp, cvp, int(c.size), mp, int(bool(adjoint))),
           "sv_apply_matrix")


def _gate_array(gates):
    arr = (sv_gate_t * max(1, len(gates)))()
    keep = []
    for i, g in enumerate(gates):
        m, mp = _cmat(g.matrix)
        keep.append(m)
        s = arr[i]
        s.n_targets = len(g.targets)
        for j, q in enumerate(g.targets):
            s.targets[j] = int(q)
        s.n_controls = len(g.controls)
        cv = tuple(g.control_values) if g.control_values else (1,) * len(g.controls)
        for j, q in enumerate(g.controls):
            s.controls[j] = int(q)
            s.control_values[j] = int(cv[j])
        s.matrix = mp
    return arr, keep


def sv_apply_fused(h: int, gates, max_fused_qubits: int, prec: int = SV_PREC_NATIVE) -> int:
    """Apply ``gates`` (objects with targets/matrix/controls/control_values) fused; returns the block count."""
    arr, _keep = _gate_array(gates)
    nf = C.c_int(0)
    _check(lib().sv_apply_fused(_VP(h), arr, len(gates), int(max_fused_qubits), int(prec), C.byref(nf)),
           "sv_apply_fused")
    return nf.value


def sv_apply_fused_ex(h: int, gates, max_fused_qubits: int, max_fused_diagonal_qubits: int = 0,
                      prec: int = SV_PREC_NATIVE) -> int:
    """sv_apply_fused with a separate width for diagonal blocks; returns the block count."""
    arr, _keep = _gate_array(gates)
    opt = sv_fusion_options_t(int(max_fused_qubits), int(max_fused_diagonal_qubits), int(prec))
    nf = C.c_int(0)
    _check(lib().sv_apply_fused_ex(_VP(h), arr, len(gates), C.byref(opt), C.byref(nf)), "sv_apply_fused_ex")
    return nf.value


def sv_fuse_plan(gates, n_qubits: int, max_fused_qubits: int, max_blocks: int | None = None,
                 max_fused_diagonal_qubits: int = 0):
    """Host-only fusion plan: list of (targets tuple, matrix) in application order."""
    arr, _keep = _gate_array(gates)
    cap = max_blocks if max_blocks is not None else max(1, len(gates))
    nb = C.c_int(0)
    ks = np.zeros(cap, dtype=np.int32)
    ts = np.zeros(cap * SV_MAX_TARGETS, dtype=np.int32)
    ms = np.zeros(cap * 64 * 64 * 2, dtype=np.float64)
    opt = sv_fusion_options_t(int(max_fused_qubits), int(max_fused_diagonal_qubits), SV_PREC_NATIVE)
    _check(lib().sv_fuse_plan_ex(arr, len(gates), int(n_qubits), C.byref(opt), cap, C.byref(nb),
                                 ks.ctypes.data_as(_I), ts.ctypes.data_as(_I), ms.ctypes.data_as(_D)),
           "sv_fuse_plan_ex")
    out = []
    for b in range(nb.value):
        k = int(ks[b])
        d = 1 << k
        flat = ms[b * 8192: b * 8192 + 2 * d * d]
        out.append((tuple(int(x) for x in ts[b * SV_MAX_TARGETS: b * SV_MAX_TARGETS + k]),
                    (flat[0::2] + 1j * flat[1::2]).reshape(d, d)))
    return out


def sv_expectation_pauli(h: int, paulis, sites) -> np.ndarray:
    """paulis, sites: int arrays of shape (n_strings, n_sites). Returns float64 (n_strings,)."""
    p = np.ascontiguousarray(np.asarray(paulis, dtype=np.int32))
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32))
    if p.ndim == 1:
        p, s = p[None, :], s[None, :]
    if p.shape != s.shape:
        raise ValueError("paulis and sites must have the same shape")
    out = np.zeros(p.shape[0], dtype=np.float64)
    _check(lib().sv_expectation_pauli(_VP(h), p.ctypes.data_as(_I), s.ctypes.data_as(_I), int(p.shape[1]),
                                      int(p.shape[0]), out.ctypes.data_as(_D)), "sv_expectation_pauli")
    return out


def sv_expectation_pauli_noalloc(n_qubits: int, dtype: int, d_state_ptr: int, stream_ptr: int, paulis,
                                 sites) -> np.ndarray:
    """Allocation-free Pauli expectations on a caller-owned device state (no handle)."""
    p = np.ascontiguousarray(np.asarray(paulis, dtype=np.int32))
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32))
    if p.ndim == 1:
        p, s = p[None, :], s[None, :]
    if p.shape != s.shape:
        raise ValueError("paulis and sites must have the same shape")
    out = np.zeros(p.shape[0], dtype=np.float64)
    _check(lib().sv_expectation_pauli_noalloc(int(n_qubits), int(dtype), _VP(d_state_ptr), _VP(stream_ptr),
                                              p.ctypes.data_as(_I), s.ctypes.data_as(_I), int(p.shape[1]),
                                              int(p.shape[0]), out.ctypes.data_as(_D)),
           "sv_expectation_pauli_noalloc")
    return out


def sv_swap_index_bits(h: int, pairs):
    """Exchange index bits a <-> b for each (a, b) in `pairs` (disjoint)."""
    p, pp = _ints([q for ab in pairs for q in ab])
    _check(lib().sv_swap_index_bits(_VP(h), pp, len(pairs)), "sv_swap_index_bits")


def sv_apply_pauli_rotation(h: int, theta: float, paulis, sites):
    """psi <- exp(i theta P) psi for the Pauli string (paulis[i] on qubit sites[i])."""
    p, pp = _ints(paulis)
    s, sp = _ints(sites)
    if p.size != s.size:
        raise ValueError("paulis and sites must have the same length")
    _check(lib().sv_apply_pauli_rotation(_VP(h), float(theta), pp, sp, int(p.size)), "sv_apply_pauli_rotation")


def sv_sample(h: int, randnums) -> np.ndarray:
    """Basis indices sampled from |psi|^2 by inverting the cumulative distribution."""
    r = np.ascontiguousarray(np.asarray(randnums, dtype=np.float64).reshape(-1))
    out = np.zeros(r.size, dtype=np.int64)
    _check(lib().sv_sample(_VP(h), r.ctypes.data_as(_D), int(r.size), out.ctypes.data_as(C.POINTER(C.c_int64))),
           "sv_sample")
    return out


def sv_measure_probs(h: int, qubits):
    q, qp = _ints(qubits)
    a, b = C.c_double(), C.c_double()
    _check(lib().sv_measure_probs(_VP(h), qp, int(q.size), C.byref(a), C.byref(b)), "sv_measure_probs")
    return a.value, b.value


def sv_collapse(h: int, qubits, parity: int, prob: float):
    q, qp = _ints(qubits)
    _check(lib().sv_collapse(_VP(h), qp, int(q.size), int(parity), float(prob)), "sv_collapse")


def sv_measure(h: int, qubits, randnum: float, collapse: bool) -> int:
    q, qp = _ints(qubits)
    out = C.c_int(-1)
    _check(lib().sv_measure(_VP(h), qp, int(q.size), float(randnum), int(bool(collapse)), C.byref(out)),
           "sv_measure")
    return out.value


def sv_norm2(h: int) -> float:
    v = C.c_double()
    _check(lib().sv_norm2(_VP(h), C.byref(v)), "sv_norm2")
    return v.value


def sv_check_device_status(h: int) -> int:
    return int(lib().sv_check_device_status(_VP(h)))


def sv_check_bounded_wait(h: int, cycles: int) -> int:
    """Run the bounded-wait diagnostic; returns the status code (SV_ERR_TIMEOUT = 5 expected)."""
    return int(lib().sv_check_bounded_wait(_VP(h), C.c_longlong(cycles)))


def sv_launch_count(h: int) -> int:
    v = C.c_uint64()
    _check(lib().sv_launch_count(_VP(h), C.byref(v)), "sv_launch_count")
    return int(v.value)


# ---- convenience: a handle bound to a torch tensor ----

@dataclass
class StateVector:
    """A handle over a caller-owned CUDA tensor (complex64 / complex128, 2^n elements)."""

    state: object          # torch.Tensor
    stream: object = None  # torch.cuda.Stream (None = current stream)

    def __post_init__(self):
        import torch
        t = self.state
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("state must be a contiguous CUDA tensor")
        if t.dtype == torch.complex64:
            self.dtype = SV_C64
        elif t.dtype == torch.complex128:
            self.dtype = SV_C128
        else:
            raise ValueError("state dtype must be complex64 or complex128")
        self.n = int(t.numel()).bit_length() - 1
        if (1 << self.n) != t.numel():
            raise ValueError("state length must be a power of two")
        if self.stream is None:
            self.stream = torch.cuda.current_stream(t.device)
        with torch.cuda.device(t.device):
            self.handle = sv_create(self.n, self.dtype, t.data_ptr(), self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            sv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_basis_state(self, index: int = 0):
        sv_set_basis_state(self.handle, index)

    def apply(self, targets, matrix, controls=(), control_values=None, adjoint=False):
        sv_apply_matrix(self.handle, targets, matrix, controls, control_values, adjoint)

    def apply_gate(self, g, adjoint=False):
        sv_apply_matrix(self.handle, g.targets, g.matrix, g.controls, g.control_values or None, adjoint)

    def apply_circuit(self, gates):
        for g in gates:
            self.apply_gate(g)

    def apply_fused(self, gates, max_fused_qubits: int, prec: int = SV_PREC_NATIVE,
                    max_fused_diagonal_qubits: int = 0) -> int:
        if max_fused_diagonal_qubits:
            return sv_apply_fused_ex(self.handle, gates, max_fused_qubits, max_fused_diagonal_qubits, prec)
        return sv_apply_fused(self.handle, gates, max_fused_qubits, prec)

    def expectation_pauli(self, paulis, sites):
        return sv_expectation_pauli(self.handle, paulis, sites)

    def expectation_z_all(self):
        n = self.n
        return sv_expectation_pauli(self.handle, np.full((n, 1), 3, np.int32), np.arange(n, dtype=np.int32)[:, None])

    def pauli_rotation(self, theta, paulis, sites):
        sv_apply_pauli_rotation(self.handle, theta, paulis, sites)

    def sample(self, randnums):
        return sv_sample(self.handle, randnums)

    def swap_index_bits(self, pairs):
        sv_swap_index_bits(self.handle, pairs)

    def measure_probs(self, qubits):
        return sv_measure_probs(self.handle, qubits)

    def collapse(self, qubits, parity, prob):
        sv_collapse(self.handle, qubits, parity, prob)

    def measure(self, qubits, randnum, collapse=False):
        return sv_measure(self.handle, qubits, randnum, collapse)

    def norm2(self):
        return sv_norm2(self.handle)

    def check(self):
        code = sv_check_device_status(self.handle)
        if code != 0:
            raise SvError(code, "device status")

    def launches(self) -> int:
        return sv_launch_count(self.handle)


# ---- batched small states ----

SV_BATCH_KEEP_STATES = 1
SV_BATCH_CHECK_WAIT = 2
SV_BATCH_STATS = 9
SV_BATCH_MAX_QUBITS = 26
SV_BATCH_TILE_QUBITS = 14     # largest (and default) tile: local qubits of one pass
GATE_DTYPE = np.dtype([("n_targets", "<i4"), ("targets", "<i4", (SV_MAX_TARGETS,)), ("n_controls", "<i4"),
                       ("controls", "<i4", (SV_MAX_CONTROLS,)), ("control_values", "<i4", (SV_MAX_CONTROLS,)),
                       ("matrix", "<u8")])
ITEM_DTYPE = np.dtype([("n_qubits", "<i4"), ("gate_begin", "<i4"), ("n_gates", "<i4"), ("pauli_begin", "<i4"),
                       ("n_strings", "<i4"), ("out_begin", "<i4"), ("state_offset", "<u8")])


def pack_gates(gates):
    """sv_gate_t records for `gates` (a numpy structured array with the C layout)
    and the complex128 buffer their matrix pointers point into (keep both alive).
    Gates are grouped by target and control count so that each group fills its
    fields with one array assignment."""
    assert C.sizeof(sv_gate_t) == GATE_DTYPE.itemsize
    ng = len(gates)
    rec = np.zeros(ng, dtype=GATE_DTYPE)
    if ng == 0:
        return rec, np.empty(1, dtype=np.complex128)
    mats = [np.asarray(g.matrix, dtype=np.complex128).reshape(-1) for g in gates]
    sizes = np.fromiter((m.size for m in mats), dtype=np.int64, count=ng)
    buf = np.concatenate(mats)
    offs = np.zeros(ng, dtype=np.int64)
    np.cumsum(sizes[:-1], out=offs[1:])
    rec["matrix"] = np.uint64(buf.ctypes.data) + 16 * offs.astype(np.uint64)
    kt = np.fromiter((len(g.targets) for g in gates), dtype=np.int32, count=ng)
    kc = np.fromiter((len(g.controls) for g in gates), dtype=np.int32, count=ng)
    rec["n_targets"] = kt
    rec["n_controls"] = kc
    for k in np.unique(kt):
        idx = np.nonzero(kt == k)[0]
        rec["targets"][idx, :k] = np.array([gates[i].targets for i in idx], dtype=np.int32).reshape(-1, k)
    for c in np.unique(kc):
        if c == 0:
            continue
        idx = np.nonzero(kc == c)[0]
        rec["controls"][idx, :c] = np.array([gates[i].controls for i in idx], dtype=np.int32).reshape(-1, c)
        rec["control_values"][idx, :c] = np.array(
            [gates[i].control_values if gates[i].control_values else (1,) * c for i in idx],
            dtype=np.int32).reshape(-1, c)
    return rec, buf


def sv_batch_create(stream_ptr: int = 0) -> int:
    b = _VP()
    _check(lib().sv_batch_create(_VP(stream_ptr), C.byref(b)), "sv_batch_create")
    return b.value


def sv_batch_destroy(b: int):
    _check(lib().sv_batch_destroy(_VP(b)), "sv_batch_destroy")


def sv_batch_compile(b: int, items: np.ndarray, gate_rec: np.ndarray, paulis: np.ndarray, fusion_width: int):
    items = np.ascontiguousarray(items, dtype=ITEM_DTYPE)
    gate_rec = np.ascontiguousarray(gate_rec, dtype=GATE_DTYPE)
    paulis = np.ascontiguousarray(paulis, dtype=np.int32).reshape(-1)
    _check(lib().sv_batch_compile(_VP(b), _VP(items.ctypes.data), int(items.size), _VP(gate_rec.ctypes.data),
                                  int(gate_rec.size), paulis.ctypes.data_as(_I) if paulis.size else None,
                                  int(fusion_width)), "sv_batch_compile")


def sv_batch_compile_ex(b: int, items: np.ndarray, gate_rec: np.ndarray, paulis: np.ndarray, fusion_width: int,
                        window_qubits: int, keep_permutations: bool = False, tile_qubits: int = SV_BATCH_TILE_QUBITS):
    """sv_batch_compile with the register-window width (0, 2, 3 or 4), the
    keep-permutations fusion rule and the tile size (local qubits of a pass,
    10..14) as options."""
    items = np.ascontiguousarray(items, dtype=ITEM_DTYPE)
    gate_rec = np.ascontiguousarray(gate_rec, dtype=GATE_DTYPE)
    paulis = np.ascontiguousarray(paulis, dtype=np.int32).reshape(-1)
    opt = (C.c_int * 4)(int(fusion_width), int(window_qubits), int(bool(keep_permutations)), int(tile_qubits))
    _check(lib().sv_batch_compile_ex(_VP(b), _VP(items.ctypes.data), int(items.size), _VP(gate_rec.ctypes.data),
                                     int(gate_rec.size), paulis.ctypes.data_as(_I) if paulis.size else None,
                                     C.cast(opt, _VP)), "sv_batch_compile_ex")


def sv_batch_info(b: int) -> dict:
    ni, ns, no = C.c_int(), C.c_int(), C.c_int()
    amps, launches = C.c_uint64(), C.c_uint64()
    _check(lib().sv_batch_info(_VP(b), C.byref(ni), C.byref(ns), C.byref(no), C.byref(amps), C.byref(launches)),
           "sv_batch_info")
    return {"items": ni.value, "stages": ns.value, "ops": no.value, "state_amps": amps.value,
            "launches": launches.value}


BATCH_STATS = ("dense_ops", "diagonal_ops", "permutation_ops", "windows", "win_2x2", "win_2x2_with_exchange",
               "win_4x4", "win_exchanges", "win_diagonals")


def sv_batch_program_stats(b: int) -> dict:
    """What the compiled program does, by op and window sub-op kind."""
    out = (C.c_uint64 * len(BATCH_STATS))()
    _check(lib().sv_batch_program_stats(_VP(b), out), "sv_batch_program_stats")
    return {k: int(v) for k, v in zip(BATCH_STATS, out)}


def sv_batch_launch(b: int, d_states_ptr: int, keep_states: bool = False, dtype: int = SV_C64, flags: int = 0):
    flags |= SV_BATCH_KEEP_STATES if keep_states else 0
    _check(lib().sv_batch_launch(_VP(b), int(dtype), _VP(d_states_ptr), int(flags)), "sv_batch_launch")


def sv_batch_results(b: int, n_out: int) -> np.ndarray:
    out = np.zeros(max(1, n_out), dtype=np.float64)
    _check(lib().sv_batch_results(_VP(b), out.ctypes.data_as(_D), int(n_out)), "sv_batch_results")
    return out[:n_out]


@dataclass
class PackedBatch:
    """A batch's states in the C layout of sv_batch_compile_ex, packed once and
    compiled as often as needed (the autotuner compiles several options)."""
    items: np.ndarray
    gate_rec: np.ndarray
    matrices: np.ndarray
    paulis: np.ndarray
    n_out: int
    state_amps: int
    ns: list
    gate_counts: list

    @property
    def offsets(self):
        return [(int(it["state_offset"]), int(it["n_qubits"]), int(it["out_begin"]), int(it["n_strings"]))
                for it in self.items]


def pack_batch(states, state_offsets=None) -> PackedBatch:
    """states: list of (n_qubits, gates, paulis) with paulis an (S, n_qubits) int
    array of Pauli codes. state_offsets (amplitudes, optional): where each state
    lives relative to the d_states pointer given at launch; by default the
    states are laid out back to back."""
    items = np.zeros(len(states), dtype=ITEM_DTYPE)
    all_gates, pls = [], []
    g0 = p0 = o0 = 0
    a0 = 0
    amps = 0
    for i, (n, gates, paulis) in enumerate(states):
        paulis = np.asarray(paulis, dtype=np.int32).reshape(-1, n) if len(paulis) else np.zeros((0, n), np.int32)
        off = a0 if state_offsets is None else int(state_offsets[i])
        items[i] = (n, g0, len(gates), p0, paulis.shape[0], o0, off)
        all_gates.extend(gates)
        pls.append(paulis.reshape(-1))
        g0 += len(gates)
        p0 += paulis.size
        o0 += paulis.shape[0]
        a0 += 1 << n
        amps = max(amps, off + (1 << n))
    rec, buf = pack_gates(all_gates)
    pl = np.concatenate(pls) if pls else np.zeros(0, np.int32)
    return PackedBatch(items, rec, buf, pl, o0, amps, [int(n) for n, _, _ in states],
                       [len(g) for _, g, _ in states])


class Batch:
    """Many independent small circuits (from |0...0>) advanced in one launch.

    states: list of (n_qubits, gates, paulis) with paulis an (S, n_qubits) int
    array of Pauli codes (column q acts on qubit q), or a PackedBatch. Results
    come back in input order, S values per state. The engine can be compiled
    and launched again and again; its device program buffer only grows."""

    def __init__(self, stream=None):
        self.stream = stream
        ptr = stream.cuda_stream if stream is not None else 0
        self.handle = sv_batch_create(ptr)
        self._keep = None
        self.choice = None

    def compile(self, states, fusion_width: int = 2, window_qubits: int = 4, keep_permutations: bool = False,
                tile_qubits: int = SV_BATCH_TILE_QUBITS, autotune: bool = False, tuner=None, state_offsets=None):
        """Compile on the host. With autotune (or a tuner given), the fusion width,
        window width, fusion rule and tile size come from the tuner
        (``autotune.BatchTuner``), which times its candidates on a sample of
        these states once per workload signature."""
        packed = states if isinstance(states, PackedBatch) else pack_batch(states, state_offsets)
        if autotune or tuner is not None:
            from .autotune import default_tuner
            tuner = tuner or default_tuner(self.stream)
            fusion_width, window_qubits, keep_permutations, tile_qubits = tuner.choose(packed)
        sv_batch_compile_ex(self.handle, packed.items, packed.gate_rec, packed.paulis, fusion_width, window_qubits,
                            keep_permutations, tile_qubits)
        self._keep = packed
        self.n_out = packed.n_out
        self.state_amps = packed.state_amps
        self.offsets = packed.offsets
        self.choice = (int(fusion_width), int(window_qubits), int(bool(keep_permutations)), int(tile_qubits))
        return self.info()

    def info(self):
        return sv_batch_info(self.handle)

    def program_stats(self):
        return sv_batch_program_stats(self.handle)

    def launch(self, d_states, keep_states: bool = False, flags: int = 0):
        """d_states: a complex64 CUDA tensor of at least `state_amps` elements, or
        a device address (int) the caller vouches for."""
        if isinstance(d_states, int):
            sv_batch_launch(self.handle, d_states, keep_states, flags=flags)
            return
        if d_states.numel() < self.state_amps:
            raise ValueError("d_states is too small for this batch")
        sv_batch_launch(self.handle, d_states.data_ptr(), keep_states, flags=flags)

    def results(self):
        flat = sv_batch_results(self.handle, self.n_out)
        return [flat[o:o + s] for (_, _, o, s) in self.offsets]

    def close(self):
        if getattr(self, "handle", None):
            sv_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- state memory pool ----

def sv_pool_create(d_base_ptr: int, nbytes: int, min_block_bytes: int = 256) -> int:
    p = _VP()
    _check(lib().sv_pool_create(_VP(d_base_ptr), C.c_uint64(nbytes), C.c_uint64(min_block_bytes), C.byref(p)),
           "sv_pool_create")
    return p.value


def sv_pool_destroy(p: int):
    _check(lib().sv_pool_destroy(_VP(p)), "sv_pool_destroy")


def sv_pool_alloc(p: int, nbytes: int):
    """Device address of a block of at least nbytes, or None when none is free."""
    out = _VP()
    code = lib().sv_pool_alloc(_VP(p), C.c_uint64(nbytes), C.byref(out))
    if code == 3:
        return None
    _check(code, "sv_pool_alloc")
    return out.value


def sv_pool_free(p: int, d_ptr: int):
    _check(lib().sv_pool_free(_VP(p), _VP(d_ptr)), "sv_pool_free")


def sv_pool_stats(p: int) -> dict:
    a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
    _check(lib().sv_pool_stats(_VP(p), C.byref(a), C.byref(b), C.byref(c)), "sv_pool_stats")
    return {"in_use": a.value, "largest_free": b.value, "capacity": c.value}


class StatePool:
    """Buddy pool of state vectors in one device arena (``sv_pool_*``). The arena
    is a caller-owned allocation (a torch tensor here) made once; blocks are
    device addresses inside it."""

    def __init__(self, arena_ptr: int, nbytes: int, min_block_bytes: int = 256):
        self.base = int(arena_ptr)
        self.handle = sv_pool_create(self.base, nbytes, min_block_bytes)

    def alloc(self, nbytes: int):
        return sv_pool_alloc(self.handle, nbytes)

    def free(self, ptr: int):
        sv_pool_free(self.handle, ptr)

    def stats(self) -> dict:
        return sv_pool_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sv_pool_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

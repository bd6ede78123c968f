"""Python binding of libsg (include/sg.h): GB300 Metropolis aging dynamics for the Viana-Bray and
Sherrington-Kirkpatrick spin glasses (arXiv:1906.11195).

The functions below carry the C names and only marshal arguments; every step of the dynamics and
of the measurements runs in the CUDA kernels of libsg.  PyTorch supplies the device workspace and
the stream.  There is no CPU fallback: if the library is missing or no GPU is present the calls
raise.

Quick use::

    import paper_1906_11195_gb300 as sg
    run = sg.VBRun([graph], n_lanes=64, n_replicas=2, kernel=sg.SG_VB_PACKED, tw=[16], tm=[16, 32])
    run.sweep(32)
    C, q, E = run.results()
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libsg.so")

SG_OK, SG_EINVAL, SG_ENOMEM, SG_ECUDA, SG_ETIMEOUT, SG_ESTATE = 0, -1, -2, -3, -4, -5
SG_VB_PLAIN, SG_VB_PACKED, SG_SK_PLAIN, SG_SK_BLOCKED = 0, 1, 2, 3
SG_VB_MAX_DEGREE = 63

_ERRNAMES = {SG_EINVAL: "SG_EINVAL", SG_ENOMEM: "SG_ENOMEM", SG_ECUDA: "SG_ECUDA",
             SG_ETIMEOUT: "SG_ETIMEOUT", SG_ESTATE: "SG_ESTATE"}

EXPORTED = [
    "sg_last_error", "sg_create_vb", "sg_create_sk", "sg_create_sk_batch", "sg_workspace_bytes",
    "sg_attach",
    "sg_sweep", "sg_time", "sg_synchronize", "sg_result_shape", "sg_read_results", "sg_measure",
    "sg_get_spins", "sg_get_thresholds", "sg_state_bytes", "sg_save_state", "sg_load_state",
    "sg_destroy", "sg_launch_count", "sg_sk_fields_noalloc", "sg_set_windows", "sg_read_windows",
    "sg_set_schedule", "sg_transfer_bytes", "sg_sk_blocked_schedule", "sg_vb_colouring",
]


class SGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class sg_vb_graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("jbits", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("temps", ctypes.c_void_p)]


class sg_sk_sample(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("J", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("temps", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"libsg is not built ({_LIB_PATH} missing); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(_LIB_PATH)
            P, i32, i64, u64, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                         ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t)
            H = ctypes.c_void_p
            sig = {
                "sg_last_error": (ctypes.c_char_p, []),
                "sg_create_vb": (ctypes.c_int, [P, i32, i32, i32, i32, P, i32, P, i32, P]),
                "sg_create_sk": (ctypes.c_int, [i32, P, i32, P, u64, i32, i32, P, i32, P, i32, P]),
                "sg_create_sk_batch": (ctypes.c_int, [P, i32, i32, i32, i32, P, i32, P, i32, P]),
                "sg_workspace_bytes": (ctypes.c_int, [H, P]),
                "sg_attach": (ctypes.c_int, [H, P, sz, P]),
                "sg_sweep": (ctypes.c_int, [H, i64]),
                "sg_time": (ctypes.c_int, [H, P]),
                "sg_synchronize": (ctypes.c_int, [H]),
                "sg_result_shape": (ctypes.c_int, [H, P]),
                "sg_read_results": (ctypes.c_int, [H, P, sz, P, sz, P, sz]),
                "sg_measure": (ctypes.c_int, [H, P, sz, P, sz, P, sz]),
                "sg_get_spins": (ctypes.c_int, [H, P, sz]),
                "sg_get_thresholds": (ctypes.c_int, [H, P, sz]),
                "sg_vb_colouring": (ctypes.c_int, [H, i32, P, sz, P]),
                "sg_state_bytes": (ctypes.c_int, [H, P]),
                "sg_save_state": (ctypes.c_int, [H, P, sz]),
                "sg_load_state": (ctypes.c_int, [H, P, sz]),
                "sg_destroy": (ctypes.c_int, [H]),
                "sg_launch_count": (ctypes.c_int, [H, P]),
                "sg_sk_fields_noalloc": (ctypes.c_int, [P, P, i32, i32, P, P]),
                "sg_set_windows": (ctypes.c_int, [H, P, i32]),
                "sg_read_windows": (ctypes.c_int, [H, P, P, P, P]),
                "sg_set_schedule": (ctypes.c_int, [H, P, i32, P, i32]),
                "sg_transfer_bytes": (ctypes.c_int, [H, P, P]),
                "sg_sk_blocked_schedule": (ctypes.c_int, [i32, i32, P, i32, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc):
    if rc != SG_OK:
        msg = _load().sg_last_error().decode(errors="replace")
        raise SGError(rc, msg)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i64(a):
    return np.ascontiguousarray(np.asarray(a if a is not None else [], dtype=np.int64))


# ----------------------------------------------------------------------------------------------
# thin wrappers with the C names
# ----------------------------------------------------------------------------------------------
def sg_last_error() -> str:
    return _load().sg_last_error().decode(errors="replace")


def sg_create_vb(graphs, n_lanes, n_replicas, kernel, tw, tm):
    """graphs: list of dicts with n, row_ptr, col, jbits, seed, temps (numpy arrays)."""
    lib = _load()
    keep = []
    arr = (sg_vb_graph * len(graphs))()
    for b, g in enumerate(graphs):
        rp = np.ascontiguousarray(g["row_ptr"], dtype=np.int32)
        cl = np.ascontiguousarray(g["col"], dtype=np.int32)
        jb = np.ascontiguousarray(g["jbits"], dtype=np.uint64)
        T = np.ascontiguousarray(g["temps"], dtype=np.float64)
        keep += [rp, cl, jb, T]
        arr[b] = sg_vb_graph(int(rp.size - 1), _p(rp), _p(cl), _p(jb),
                             int(g["seed"]) & (2**64 - 1), _p(T))
    tw_a, tm_a = _i64(tw), _i64(tm)
    h = ctypes.c_void_p()
    _check(lib.sg_create_vb(ctypes.cast(arr, ctypes.c_void_p), len(graphs), int(n_lanes),
                            int(n_replicas), int(kernel), _p(tw_a), tw_a.size, _p(tm_a), tm_a.size,
                            ctypes.byref(h)))
    return h


def sg_create_sk(J, n_replicas, temps, seed, kernel, block, tw, tm):
    lib = _load()
    Jc = np.ascontiguousarray(J, dtype=np.int8)
    T = np.ascontiguousarray(temps, dtype=np.float64)
    tw_a, tm_a = _i64(tw), _i64(tm)
    h = ctypes.c_void_p()
    _check(lib.sg_create_sk(int(Jc.shape[0]), _p(Jc), int(n_replicas), _p(T),
                            int(seed) & (2**64 - 1), int(kernel), int(block), _p(tw_a), tw_a.size,
                            _p(tm_a), tm_a.size, ctypes.byref(h)))
    return h


def sg_create_sk_batch(samples, n_replicas, kernel, block, tw, tm):
    """samples: list of dicts with J (int8 n x n), seed, temps (n_replicas temperatures)."""
    lib = _load()
    keep = []
    arr = (sg_sk_sample * len(samples))()
    for b, x in enumerate(samples):
        Jc = np.ascontiguousarray(x["J"], dtype=np.int8)
        T = np.ascontiguousarray(x["temps"], dtype=np.float64)
        keep += [Jc, T]
        arr[b] = sg_sk_sample(int(Jc.shape[0]), _p(Jc), int(x["seed"]) & (2**64 - 1), _p(T))
    tw_a, tm_a = _i64(tw), _i64(tm)
    h = ctypes.c_void_p()
    _check(lib.sg_create_sk_batch(ctypes.cast(arr, ctypes.c_void_p), len(samples), int(n_replicas),
                                  int(kernel), int(block), _p(tw_a), tw_a.size, _p(tm_a),
                                  tm_a.size, ctypes.byref(h)))
    return h


def sg_workspace_bytes(h) -> int:
    v = ctypes.c_size_t()
    _check(_load().sg_workspace_bytes(h, ctypes.byref(v)))
    return int(v.value)


def sg_attach(h, dev_ptr: int, nbytes: int, stream_handle: int):
    _check(_load().sg_attach(h, ctypes.c_void_p(dev_ptr), nbytes, ctypes.c_void_p(stream_handle)))


def sg_sweep(h, n: int):
    _check(_load().sg_sweep(h, int(n)))


def sg_time(h) -> int:
    v = ctypes.c_int64()
    _check(_load().sg_time(h, ctypes.byref(v)))
    return int(v.value)


def sg_synchronize(h):
    _check(_load().sg_synchronize(h))


def sg_result_shape(h):
    s = np.zeros(5, dtype=np.int32)
    _check(_load().sg_result_shape(h, _p(s)))
    return tuple(int(x) for x in s)


def sg_read_results(h):
    n_inst, R, L, ntw, ntm = sg_result_shape(h)
    C = np.zeros((n_inst, R, L, ntw, ntm), dtype=np.int64)
    q = np.zeros((n_inst, R // 2, L, ntm), dtype=np.int64)
    E = np.zeros((n_inst, R, L, ntm), dtype=np.int64)
    _check(_load().sg_read_results(h, _p(C), C.size, _p(q), q.size, _p(E), E.size))
    return C, q, E


def sg_measure(h):
    n_inst, R, L, ntw, _ = sg_result_shape(h)
    C = np.zeros((n_inst, R, L, ntw), dtype=np.int64)
    q = np.zeros((n_inst, R // 2, L), dtype=np.int64)
    E = np.zeros((n_inst, R, L), dtype=np.int64)
    _check(_load().sg_measure(h, _p(C), C.size, _p(q), q.size, _p(E), E.size))
    return C, q, E


def sg_set_schedule(h, tw, tm):
    """Replace the snapshot times tw and measurement times tm (see sg.h for when this is allowed)."""
    tw_a, tm_a = _i64(tw), _i64(tm)
    _check(_load().sg_set_schedule(h, _p(tw_a), int(tw_a.size), _p(tm_a), int(tm_a.size)))


def sg_set_windows(h, bounds):
    b = _i64(bounds)
    _check(_load().sg_set_windows(h, _p(b), int(b.size)))


def sg_read_windows(h, n_bins: int):
    """Window sums C[n_inst][R][L][n_tw][n_bins], q, E and n_meas[n_tw + 1][n_bins]."""
    n_inst, R, L, ntw, _ = sg_result_shape(h)
    C = np.zeros((n_inst, R, L, ntw, n_bins), dtype=np.int64)
    q = np.zeros((n_inst, R // 2, L, n_bins), dtype=np.int64)
    E = np.zeros((n_inst, R, L, n_bins), dtype=np.int64)
    n = np.zeros((ntw + 1, n_bins), dtype=np.int64)
    _check(_load().sg_read_windows(h, _p(C), _p(q), _p(E), _p(n)))
    return C, q, E, n


def sg_get_spins(h, nbytes: int, dtype):
    out = np.zeros(nbytes // np.dtype(dtype).itemsize, dtype=dtype)
    _check(_load().sg_get_spins(h, _p(out), out.nbytes))
    return out


def sg_get_thresholds(h, n: int):
    out = np.zeros(n, dtype=np.uint32)
    _check(_load().sg_get_thresholds(h, _p(out), out.size))
    return out


def sg_vb_colouring(h, graph: int, n: int):
    """(colour int32[n] of graph `graph`, number of colour classes) of a VB handle."""
    out = np.zeros(n, dtype=np.int32)
    nc = ctypes.c_int32(0)
    _check(_load().sg_vb_colouring(h, int(graph), _p(out), out.size, ctypes.byref(nc)))
    return out, nc.value


def sg_save_state(h) -> bytes:
    n = ctypes.c_size_t()
    _check(_load().sg_state_bytes(h, ctypes.byref(n)))
    buf = np.zeros(n.value, dtype=np.uint8)
    _check(_load().sg_save_state(h, _p(buf), buf.size))
    return buf


def sg_load_state(h, blob):
    b = np.ascontiguousarray(blob, dtype=np.uint8)
    _check(_load().sg_load_state(h, _p(b), b.size))


def sg_destroy(h):
    _check(_load().sg_destroy(h))


def sg_launch_count(h) -> int:
    v = ctypes.c_int64()
    _check(_load().sg_launch_count(h, ctypes.byref(v)))
    return int(v.value)


def sg_transfer_bytes(h):
    """(host -> device, device -> host) bytes the handle has copied so far."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(_load().sg_transfer_bytes(h, ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def sg_sk_blocked_schedule(n, block):
    """The blocked SK sweep's operations in issue order: int32[n_ops][6] rows of
    (op, stream, block, skip0, skip1, event), as include/sg.h describes."""
    lib = _load()
    cnt = ctypes.c_int32(0)
    lib.sg_sk_blocked_schedule(int(n), int(block), None, 0, ctypes.byref(cnt))
    out = np.zeros((max(1, cnt.value), 6), dtype=np.int32)
    _check(lib.sg_sk_blocked_schedule(int(n), int(block), out.ctypes.data, cnt.value, ctypes.byref(cnt)))
    return out[:cnt.value]


def sg_sk_fields_noalloc(J_dev: int, s_dev: int, n: int, n_replicas: int, h_dev: int,
                         stream_handle: int):
    """Local fields h = J s for callers that cannot allocate device memory (device pointers in
    and out; the library's fixed static scratch holds the tensor-core operand images)."""
    _check(_load().sg_sk_fields_noalloc(ctypes.c_void_p(J_dev), ctypes.c_void_p(s_dev), int(n),
                                        int(n_replicas), ctypes.c_void_p(h_dev),
                                        ctypes.c_void_p(stream_handle)))


# ----------------------------------------------------------------------------------------------
# convenience owners: allocate the workspace with PyTorch and bind the current stream
# ----------------------------------------------------------------------------------------------
class _Run:
    def __init__(self, handle, device=None, stream=None, windows=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libsg needs a CUDA device")
        self.h = None
        self.device = torch.device(device or "cuda")
        self.n_bins = 0
        try:
            if windows is not None:
                sg_set_windows(handle, windows)
                self.n_bins = len(windows) - 1
            nbytes = sg_workspace_bytes(handle)
            # 256-byte alignment: PyTorch's caching allocator returns 512-byte aligned blocks
            self.workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.device)
            self.stream = stream or torch.cuda.current_stream(self.device)
            with torch.cuda.device(self.device):
                sg_attach(handle, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        except Exception:
            sg_destroy(handle)
            self.workspace = None
            raise
        self.h = handle

    def sweep(self, n):
        sg_sweep(self.h, n)

    @property
    def tau(self):
        return sg_time(self.h)

    def synchronize(self):
        sg_synchronize(self.h)

    def results(self):
        return sg_read_results(self.h)

    def measure(self):
        return sg_measure(self.h)

    def set_schedule(self, tw, tm):
        """Replace the schedule after attach (same sizes, no scheduled time reached yet)."""
        sg_set_schedule(self.h, tw, tm)

    def windows(self):
        """Window sums C, q, E and the measurement counts n_meas (see sg_read_windows)."""
        return sg_read_windows(self.h, self.n_bins)

    def save_state(self):
        return sg_save_state(self.h)

    def load_state(self, blob):
        sg_load_state(self.h, blob)

    @property
    def launches(self):
        return sg_launch_count(self.h)

    def close(self):
        if self.h is not None:
            sg_destroy(self.h)
            self.h = None
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VBRun(_Run):
    """A batch of Viana-Bray graphs (Eq. 3) evolving in lock-step under Metropolis dynamics."""

    def __init__(self, graphs, n_lanes=64, n_replicas=2, kernel=SG_VB_PACKED, tw=(), tm=(),
                 device=None, stream=None, windows=None):
        self.sizes = [int(np.asarray(g["row_ptr"]).size - 1) for g in graphs]
        self.n_replicas = n_replicas
        super().__init__(sg_create_vb(graphs, n_lanes, n_replicas, kernel, tw, tm), device, stream,
                         windows)

    def spins(self):
        """uint64 spins per graph: list of [R][n] arrays in the caller's vertex order."""
        total = sum(self.sizes) * self.n_replicas
        flat = sg_get_spins(self.h, total * 8, np.uint64)
        out, off = [], 0
        for n in self.sizes:
            out.append(flat[off:off + self.n_replicas * n].reshape(self.n_replicas, n))
            off += self.n_replicas * n
        return out

    def thresholds(self):
        return sg_get_thresholds(self.h, len(self.sizes) * self.n_replicas * 64).reshape(
            len(self.sizes), self.n_replicas, 64)


class SKBatchRun(_Run):
    """Independent SK samples of uneven size advancing in lock-step (one graph per sweep)."""

    def __init__(self, samples, n_replicas, kernel=SG_SK_BLOCKED, block=0, tw=(), tm=(),
                 device=None, stream=None, windows=None):
        self.sizes = [int(np.asarray(x["J"]).shape[0]) for x in samples]
        self.n_replicas = n_replicas
        super().__init__(sg_create_sk_batch(samples, n_replicas, kernel, block, tw, tm), device,
                         stream, windows)

    def spins(self):
        flat = sg_get_spins(self.h, sum(self.sizes) * self.n_replicas, np.int8)
        out, off = [], 0
        for n in self.sizes:
            out.append(flat[off:off + n * self.n_replicas].reshape(self.n_replicas, n))
            off += n * self.n_replicas
        return out


class SKRun(_Run):
    """A Sherrington-Kirkpatrick sample (Eq. 1, binary couplings) with R replicas sharing J."""

    def __init__(self, J, temps, seed, kernel=SG_SK_BLOCKED, block=128, tw=(), tm=(), device=None,
                 stream=None, windows=None):
        self.n = int(np.asarray(J).shape[0])
        self.n_replicas = len(temps)
        super().__init__(sg_create_sk(J, len(temps), temps, seed, kernel, block, tw, tm), device,
                         stream, windows)

    def spins(self):
        return sg_get_spins(self.h, self.n * self.n_replicas, np.int8).reshape(self.n_replicas, self.n)

    def thresholds(self):
        return sg_get_thresholds(self.h, self.n_replicas * self.n).reshape(self.n_replicas, self.n)

"""ctypes wrapper around the plain C oracle (sg_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use this package; the product path (``paper_1906_11195_gb300``) never
imports, links or runs it.  It shares no code with the CUDA library.

Functions follow the paper's definitions (arXiv:1906.11195): Metropolis dynamics for the
Viana-Bray model (Eq. 3, Methods, SI section 2) and the Sherrington-Kirkpatrick model with
binary couplings (Eq. 1, SI section 1); C(t_w+t, t_w) as in Eq. formula1.  The readings taken
where the paper is silent are listed in the header of sg_oracle.c.  Parity pins: see
tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsg_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sg_oracle.c with gcc into oracle/_build/libsg_oracle.so (plain -O2, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    P = ctypes.c_void_p
    i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    lib.orc_philox4x32_10.argtypes = [P, P, P]
    lib.orc_philox4x32_10.restype = None
    lib.orc_vb_thresholds.argtypes = [f64, i32, P]
    lib.orc_vb_thresholds.restype = None
    lib.orc_sk_thresholds.argtypes = [f64, i32, P]
    lib.orc_sk_thresholds.restype = None
    lib.orc_greedy_colour.argtypes = [i32, P, P, P]
    lib.orc_greedy_colour.restype = i32
    lib.orc_recolour.argtypes = [i32, P, P, P]
    lib.orc_recolour.restype = i32
    lib.orc_vb_run.argtypes = [i32, P, P, P, i32, i32, P, u64, i64,
                               P, i32, P, i32, P, P, P, P, P]
    lib.orc_vb_run.restype = i32
    lib.orc_sk_run.argtypes = [i32, P, i32, P, u64, i64, i32, i32,
                               P, i32, P, i32, P, P, P, P, P]
    lib.orc_sk_run.restype = i32
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def compile_variant(c_source: str, out_dir: str):
    """Compile an edited copy of the oracle (tests plant mistakes this way) and bind it.

    Returns an object whose vb_run / sk_run use that library instead of the real oracle.
    """
    src = os.path.join(out_dir, "variant.c")
    so = os.path.join(out_dir, "libvariant.so")
    with open(src, "w") as f:
        f.write(c_source)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", so, src, "-lm"], check=True)
    lib = _bind(ctypes.CDLL(so))

    class _Variant:
        def vb_run(self, *a, **k):
            return vb_run(*a, _lib_override=lib, **k)

        def sk_run(self, *a, **k):
            return sk_run(*a, _lib_override=lib, **k)
    return _Variant()


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 uint32 counter words, 2 uint32 key words -> 4 uint32 words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def vb_thresholds(T: float, dmax: int) -> np.ndarray:
    """uint32[dmax+1]: thr[m] = min(2^32-1, floor(2^32 exp(-2 m / T))), thr[0] = 2^32-1."""
    lib = _load()
    out = np.zeros(dmax + 1, dtype=np.uint32)
    lib.orc_vb_thresholds(float(T), int(dmax), _ptr(out))
    return out


def sk_thresholds(T: float, n: int) -> np.ndarray:
    """uint32[N]: thr[k] = min(2^32-1, floor(2^32 exp(-(2 k / T) / sqrt(N)))), thr[0] = 2^32-1."""
    lib = _load()
    out = np.zeros(n, dtype=np.uint32)
    lib.orc_sk_thresholds(float(T), int(n), _ptr(out))
    return out


def greedy_colour(row_ptr, col):
    """Greedy colouring in vertex order -> (colour int32[N], number of colours)."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    n = rp.size - 1
    colour = np.zeros(n, dtype=np.int32)
    nc = lib.orc_greedy_colour(n, _ptr(rp), _ptr(cl), _ptr(colour))
    if nc < 0:
        raise MemoryError("oracle colouring failed")
    return colour, int(nc)


def recolour(row_ptr, col, colour):
    """One recolouring pass: greedy again in the order (decreasing colour, increasing label)
    -> (colour int32[N], number of colours)."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    out = np.array(colour, dtype=np.int32, copy=True)
    nc = lib.orc_recolour(rp.size - 1, _ptr(rp), _ptr(cl), _ptr(out))
    if nc < 0:
        raise MemoryError("oracle recolouring failed")
    return out, int(nc)


def vb_colouring(row_ptr, col):
    """The colour classes a VB sweep visits in turn: greedy_colour, then one recolour pass."""
    colour, _ = greedy_colour(row_ptr, col)
    return recolour(row_ptr, col, colour)


def _sched(a):
    return np.ascontiguousarray(a if a is not None else [], dtype=np.int64)


def vb_run(row_ptr, col, jbits, n_lanes, temps, seed, n_sweeps, tw=(), tm=(), trajectory=False,
           _lib_override=None):
    """Run the Viana-Bray oracle for n_sweeps sweeps from tau = 0.

    Returns dict(spins uint64[R][N], C int64[R][L][n_tw][n_tm], q int64[R//2][L][n_tm],
    E int64[R][L][n_tm], n_colours, and traj uint64[n_sweeps+1][R][N] if trajectory).
    """
    lib = _lib_override or _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    jb = np.ascontiguousarray(jbits, dtype=np.uint64)
    T = np.ascontiguousarray(temps, dtype=np.float64)
    n, R, L = rp.size - 1, T.size, int(n_lanes)
    tw_a, tm_a = _sched(tw), _sched(tm)
    spins = np.zeros((R, n), dtype=np.uint64)
    C = np.zeros((R, L, tw_a.size, tm_a.size), dtype=np.int64)
    q = np.zeros((R // 2, L, tm_a.size), dtype=np.int64)
    E = np.zeros((R, L, tm_a.size), dtype=np.int64)
    traj = np.zeros((int(n_sweeps) + 1, R, n), dtype=np.uint64) if trajectory else None
    rc = lib.orc_vb_run(n, _ptr(rp), _ptr(cl), _ptr(jb), L, R, _ptr(T), int(seed) & (2**64 - 1),
                        int(n_sweeps), _ptr(tw_a), tw_a.size, _ptr(tm_a), tm_a.size,
                        _ptr(spins), _ptr(C), _ptr(q), _ptr(E), _ptr(traj))
    if rc < 0:
        raise RuntimeError(f"orc_vb_run failed ({rc})")
    out = dict(spins=spins, C=C, q=q, E=E, n_colours=int(rc))
    if trajectory:
        out["traj"] = traj
    return out


def sk_run(J, temps, seed, n_sweeps, tw=(), tm=(), r_first=0, r_count=None, trajectory=False,
           _lib_override=None):
    """Run the SK oracle (replicas [r_first, r_first + r_count) of a len(temps)-replica run).

    Returns dict(spins int8[rc][N], C int64[rc][n_tw][n_tm], q int64[rc//2][n_tm],
    E int64[rc][n_tm], and traj int8[n_sweeps+1][rc][N] if trajectory).
    """
    lib = _lib_override or _load()
    Jc = np.ascontiguousarray(J, dtype=np.int8)
    n = Jc.shape[0]
    T = np.ascontiguousarray(temps, dtype=np.float64)
    R = T.size
    rc_n = R - r_first if r_count is None else int(r_count)
    tw_a, tm_a = _sched(tw), _sched(tm)
    spins = np.zeros((rc_n, n), dtype=np.int8)
    C = np.zeros((rc_n, tw_a.size, tm_a.size), dtype=np.int64)
    q = np.zeros((rc_n // 2, tm_a.size), dtype=np.int64)
    E = np.zeros((rc_n, tm_a.size), dtype=np.int64)
    traj = np.zeros((int(n_sweeps) + 1, rc_n, n), dtype=np.int8) if trajectory else None
    rc = lib.orc_sk_run(n, _ptr(Jc), R, _ptr(T), int(seed) & (2**64 - 1), int(n_sweeps),
                        int(r_first), rc_n, _ptr(tw_a), tw_a.size, _ptr(tm_a), tm_a.size,
                        _ptr(spins), _ptr(C), _ptr(q), _ptr(E), _ptr(traj))
    if rc < 0:
        raise RuntimeError(f"orc_sk_run failed ({rc})")
    out = dict(spins=spins, C=C, q=q, E=E)
    if trajectory:
        out["traj"] = traj
    return out

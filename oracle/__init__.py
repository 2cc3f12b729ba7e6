"""CPU FP64 O(N^2) oracle for the short-range MD hot path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module, and this module never imports the product package;
the two share only the seeded inputs from ``synth``.

Every function is the plain definition (see ``oracle.c`` for the formulas and
the readings taken where the paper is silent):

* neighbour sets of the Verlet list (paper Sec. III.B),
* cut-off Lennard-Jones and Finnis-Sinclair EAM forces, energy and virial
  (paper App. A names both benchmark potentials),
* the LJ force vector-Jacobian product used by force matching,
* velocity-Verlet NVE (paper Sec. II, integration in double precision).

Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP). Returns the path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                   "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
            subprocess.check_call(cmd)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
    lib.oracle_neighbors.restype = _I64
    lib.oracle_neighbors.argtypes = [_I64, _d, _d, _D, _I64, _i64, _i32, _i32, _I64]
    lib.oracle_min_gap.restype = _D
    lib.oracle_min_gap.argtypes = [_I64, _d, _d, _D, _I64, _i64]
    lib.oracle_lj.restype = ctypes.c_int
    lib.oracle_lj.argtypes = [_I64, _d, _i32, _I32, _d, _d, _d, _D, _I32, _d, _d, _d]
    lib.oracle_lj_at.restype = ctypes.c_int
    lib.oracle_lj_at.argtypes = [_I64, _d, _i32, _I32, _d, _d, _d, _D, _I32, _I64, _i64, _d, _d, _i32]
    lib.oracle_lj_vjp.restype = ctypes.c_int
    lib.oracle_lj_vjp.argtypes = [_I64, _d, _i32, _I32, _d, _d, _d, _D, _d, _d, _d, _d]
    lib.oracle_eam.restype = ctypes.c_int
    lib.oracle_eam.argtypes = [_I64, _d, _d, _d, _d, _d, _d, _d, _d]
    lib.oracle_eam_at.restype = ctypes.c_int
    lib.oracle_eam_vjp.restype = ctypes.c_int
    lib.oracle_lj_cells.restype = ctypes.c_int
    lib.oracle_lj_cells.argtypes = [_I64, _d, _d, _D, _d]
    lib.oracle_nve_cells.restype = ctypes.c_int
    lib.oracle_nve_cells.argtypes = [_I64, _d, _d, _d, _D, _D, _D, _I64, _d, _I32]
    lib.oracle_eam_vjp.argtypes = [_I64, _d, _d, _d, _d, _d, _d]
    lib.oracle_eam_at.argtypes = [_I64, _d, _d, _d, _I64, _i64, _d, _d]
    lib.oracle_kinetic.restype = _D
    lib.oracle_kinetic.argtypes = [_I64, _d, _i32, _d, _D]
    lib.oracle_nve.restype = _I64
    lib.oracle_nve.argtypes = [_I64, _d, _d, _i32, _I32, _d, _D, _d, _I32, _d, _D, _I32, _D, _D,
                               _I64, _d, _d, _d]
    _lib = lib
    return lib


def _pd(a):
    return None if a is None else a.ctypes.data_as(_d)


def _pi32(a):
    return None if a is None else a.ctypes.data_as(_i32)


def _pi64(a):
    return None if a is None else a.ctypes.data_as(_i64)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _types(t, n):
    if t is None:
        return np.zeros(n, dtype=np.int32)
    return np.ascontiguousarray(t, dtype=np.int32)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed (status {rc}): box smaller than twice the cut-off?")


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def neighbors(x, box, rl, idx=None):
    """Full neighbour sets {j != i : |d_ij| < rl} (minimum image), ascending j.

    Returns a list of int32 arrays, one per atom (or per entry of ``idx``).
    """
    lib = _load()
    x = _f64(x, (-1, 3))
    box = _f64(box)
    n = x.shape[0]
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        m = idx.shape[0]
    else:
        m = n
    counts = np.zeros(m, dtype=np.int32)
    cap = 1
    nbr = np.zeros(cap, dtype=np.int32)
    tot = lib.oracle_neighbors(n, _pd(x), _pd(box), float(rl), m, _pi64(idx), _pi32(counts), _pi32(nbr), cap)
    if tot == -1:
        raise ValueError("oracle neighbors: invalid input")
    if tot == -2:
        cap = int(counts.sum())
        nbr = np.zeros(max(cap, 1), dtype=np.int32)
        tot = lib.oracle_neighbors(n, _pd(x), _pd(box), float(rl), m, _pi64(idx), _pi32(counts), _pi32(nbr), cap)
        if tot < 0:
            raise ValueError("oracle neighbors failed")
    offs = np.concatenate([[0], np.cumsum(counts, dtype=np.int64)])
    return [nbr[offs[k]:offs[k + 1]].copy() for k in range(m)]


def min_gap(x, box, rl, idx=None) -> float:
    """min over pairs (touching idx, or all) of | |d_ij| - rl |."""
    lib = _load()
    x = _f64(x, (-1, 3))
    box = _f64(box)
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        m = idx.shape[0]
    else:
        m = x.shape[0]
    return float(lib.oracle_min_gap(x.shape[0], _pd(x), _pd(box), float(rl), m, _pi64(idx)))


def _lj_params(eps, sig, nt):
    eps = _f64(eps).reshape(-1)
    sig = _f64(sig).reshape(-1)
    if eps.size != nt * nt or sig.size != nt * nt:
        raise ValueError("eps/sig must have n_types^2 entries")
    return eps, sig


def lj(x, box, rc, eps=1.0, sig=1.0, types=None, n_types=1, shift=False):
    """LJ forces (n,3), potential energy and virial (6: xx,yy,zz,xy,xz,yz)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    t = _types(types, n)
    eps, sig = _lj_params(np.broadcast_to(eps, (n_types, n_types)), np.broadcast_to(sig, (n_types, n_types)), n_types)
    f = np.zeros((n, 3))
    e = np.zeros(1)
    w = np.zeros(6)
    _check(lib.oracle_lj(n, _pd(x), _pi32(t), n_types, _pd(eps), _pd(sig), _pd(_f64(box)), float(rc),
                         int(bool(shift)), _pd(f), _pd(e), _pd(w)), "lj")
    return f, float(e[0]), w


def lj_at(x, box, rc, idx, eps=1.0, sig=1.0, types=None, n_types=1, shift=False):
    """LJ forces on atoms idx only: (forces (m,3), half pair energy (m,), partners (m,))."""
    lib = _load()
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    t = _types(types, n)
    eps, sig = _lj_params(np.broadcast_to(eps, (n_types, n_types)), np.broadcast_to(sig, (n_types, n_types)), n_types)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = idx.shape[0]
    f = np.zeros((m, 3))
    e = np.zeros(m)
    c = np.zeros(m, dtype=np.int32)
    _check(lib.oracle_lj_at(n, _pd(x), _pi32(t), n_types, _pd(eps), _pd(sig), _pd(_f64(box)), float(rc),
                            int(bool(shift)), m, _pi64(idx), _pd(f), _pd(e), _pi32(c)), "lj_at")
    return f, e, c


def lj_vjp(x, box, rc, g, eps, sig, types=None, n_types=1):
    """Backward of the LJ forces for L = sum_i g_i.F_i: (grad_x (n,3), grad_eps, grad_sig (nt,nt))."""
    lib = _load()
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    t = _types(types, n)
    eps, sig = _lj_params(np.broadcast_to(eps, (n_types, n_types)), np.broadcast_to(sig, (n_types, n_types)), n_types)
    g = _f64(g, (n, 3))
    gx = np.zeros((n, 3))
    ge = np.zeros(n_types * n_types)
    gs = np.zeros(n_types * n_types)
    _check(lib.oracle_lj_vjp(n, _pd(x), _pi32(t), n_types, _pd(eps), _pd(sig), _pd(_f64(box)), float(rc),
                             _pd(g), _pd(gx), _pd(ge), _pd(gs)), "lj_vjp")
    return gx, ge.reshape(n_types, n_types), gs.reshape(n_types, n_types)


def eam(x, box, p):
    """Finnis-Sinclair EAM, p = (rc, A, c0, c1, c2): (forces, energy, virial6, rho, F'(rho))."""
    lib = _load()
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    p = _f64(p)
    f = np.zeros((n, 3))
    e = np.zeros(1)
    w = np.zeros(6)
    rho = np.zeros(n)
    fp = np.zeros(n)
    _check(lib.oracle_eam(n, _pd(x), _pd(_f64(box)), _pd(p), _pd(f), _pd(e), _pd(w), _pd(rho), _pd(fp)), "eam")
    return f, float(e[0]), w, rho, fp


def eam_at(x, box, p, idx):
    """EAM forces and host densities on atoms idx only."""
    lib = _load()
    x = _f64(x, (-1, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = idx.shape[0]
    f = np.zeros((m, 3))
    rho = np.zeros(m)
    _check(lib.oracle_eam_at(x.shape[0], _pd(x), _pd(_f64(box)), _pd(_f64(p)), m, _pi64(idx), _pd(f), _pd(rho)),
           "eam_at")
    return f, rho


def eam_vjp(x, box, p, g):
    """Backward of the EAM forces for L = sum_i g_i.F_i: (grad_x (n,3), grad_p (5,)) with grad_p in the
    layout of p = (rc, A, c0, c1, c2); the cut-off slot is 0 (not differentiated)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    g = _f64(g, (n, 3))
    gx = np.zeros((n, 3))
    gp = np.zeros(5)
    _check(lib.oracle_eam_vjp(n, _pd(x), _pd(_f64(box)), _pd(_f64(p)), _pd(g), _pd(gx), _pd(gp)), "eam_vjp")
    return gx, gp


def lj_cells(x, box, rc):
    """Single-type LJ forces by cell lists (the O(N) CPU baseline; same sums as lj)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    f = np.zeros_like(x)
    _check(lib.oracle_lj_cells(x.shape[0], _pd(x), _pd(_f64(box)), float(rc), _pd(f)), "lj_cells")
    return f


def nve_cells(x, v, box, rc, dt, mass, nsteps, f=None):
    """Velocity-Verlet with cell-list LJ forces (O(N) CPU baseline): returns (x, v, f)."""
    lib = _load()
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    have = f is not None
    f = _f64(f, (-1, 3)).copy() if have else np.zeros_like(x)
    _check(lib.oracle_nve_cells(x.shape[0], _pd(x), _pd(v), _pd(_f64(box)), float(rc), float(dt), float(mass),
                                int(nsteps), _pd(f), 1 if have else 0), "nve_cells")
    return x, v, f


def kinetic(v, mass, types=None, ftm2v=1.0) -> float:
    lib = _load()
    v = _f64(v, (-1, 3))
    t = _types(types, v.shape[0])
    return float(lib.oracle_kinetic(v.shape[0], _pd(v), _pi32(t), _pd(_f64(mass)), float(ftm2v)))


def nve(x, v, box, nsteps, dt, rc, skin, pot="lj", eps=1.0, sig=1.0, eam_params=None, types=None,
        n_types=1, mass=(1.0,), ftm2v=1.0, shift=False):
    """Velocity-Verlet NVE. Returns dict(x, v, f, epot[nsteps+1], ekin[nsteps+1], rebuilds)."""
    lib = _load()
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    n = x.shape[0]
    t = _types(types, n)
    if pot == "lj":
        eps_, sig_ = _lj_params(np.broadcast_to(eps, (n_types, n_types)), np.broadcast_to(sig, (n_types, n_types)),
                                n_types)
        params = np.concatenate([eps_, sig_])
        ipot = 0
    elif pot == "eam":
        params = _f64(eam_params)
        rc = float(params[0])
        ipot = 1
    else:
        raise ValueError(pot)
    f = np.zeros((n, 3))
    ep = np.zeros(nsteps + 1)
    ek = np.zeros(nsteps + 1)
    nb = lib.oracle_nve(n, _pd(x), _pd(v), _pi32(t), n_types, _pd(_f64(mass)), float(ftm2v), _pd(_f64(box)),
                        ipot, _pd(params), float(rc), int(bool(shift)), float(skin), float(dt), int(nsteps),
                        _pd(f), _pd(ep), _pd(ek))
    if nb < 0:
        raise ValueError("oracle nve failed")
    return {"x": x, "v": v, "f": f, "epot": ep, "ekin": ek, "rebuilds": int(nb)}

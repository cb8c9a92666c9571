"""FP64 CPU oracle for the element volume term (Sec. 2, Eq. (2)).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
(``paper_1604_08501_gb300``) never imports it, and it imports nothing from the
GPU library: the two share only the seeded input generator, which holds none
of the method's arithmetic.

Python side of the C oracle in ``numa_oracle.c``: argument marshalling only.
Every number it returns is computed by the C code, in FP64 with
``-ffp-contract=off``.

Functions
---------
gll_nodes(N)            GLL nodes (Newton on x P_N - P_{N-1}).
diff_matrix(N)          D[i, n] = l_n'(xi_i) from the Lagrange definition.
pressure(Theta, c)      p0 (R Theta / p0)^gamma, gamma = cp / (cp - R).
vol_rhs_o1(prob, q)     brute force, one pass per reference direction.
vol_rhs_o2(prob, q)     fluxes once per node, then the D contractions.
vol_rhs_points(prob, q, ids)  Eq. (2) at selected nodes only.
vol_rhs_abs(prob, q)    running error bound |Jinv| sum |D| |F| per point.
condition_numbers(prob, q)  per field max(bound) / max|rhs|.
lsrk(prob, q, dt, n)    n steps of the 5-stage 4th-order 2N-storage Runge-Kutta
                        scheme (Carpenter-Kennedy 1994) on dq/dt = volume term.

``prob`` is a dict with keys N, Ne, g (9 x M), Jinv, rho_ref, rhotheta_ref
(each M = Ne*(N+1)^3 doubles, [e][k][j][i] order), constants p0, R, cp,
grav, and optionally ntracers (0..3, default 0).  ``q`` is a (5 + ntracers, M)
float64 array (rho, U1, U2, U3, Theta, Q1..).
"""
from __future__ import annotations

import contextlib
import ctypes as C

import numpy as np

from .build import LIB, build_oracle

_DP = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [
        ("N", C.c_int),
        ("Ne", C.c_int64),
        ("D", _DP),
        ("g", _DP * 9),
        ("Jinv", _DP),
        ("rho_ref", _DP),
        ("rhotheta_ref", _DP),
        ("p0", C.c_double),
        ("R", C.c_double),
        ("cp", C.c_double),
        ("grav", C.c_double),
        ("ntracers", C.c_int),
    ]


_lib = None


def _configure(lib):
    lib.oracle_gll_nodes.argtypes = [C.c_int, _DP]
    lib.oracle_diff_matrix.argtypes = [C.c_int, _DP, _DP]
    lib.oracle_pressure.argtypes = [C.c_double] * 4
    lib.oracle_pressure.restype = C.c_double
    lib.oracle_vol_rhs_o1.argtypes = [C.POINTER(_Problem), _DP, _DP]
    lib.oracle_vol_rhs_o2.argtypes = [C.POINTER(_Problem), _DP, _DP, C.c_int]
    lib.oracle_vol_rhs_points.argtypes = [C.POINTER(_Problem), _DP, C.c_int64,
                                          C.POINTER(C.c_int64), _DP]
    lib.oracle_vol_rhs_abs.argtypes = [C.POINTER(_Problem), _DP, _DP]
    lib.oracle_lsrk_coefficients.argtypes = [_DP, _DP, _DP]
    lib.oracle_lsrk.argtypes = [C.POINTER(_Problem), _DP, C.c_double, C.c_int, C.c_int]
    lib.oracle_lsrk_scalar.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
    lib.oracle_lsrk_scalar.restype = C.c_double
    lib.oracle_max_threads.restype = C.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        _lib = _configure(C.CDLL(LIB))
    return _lib


@contextlib.contextmanager
def variant(path: str):
    """Route every call to another build of the oracle source (a planted
    mistake, compiled by the mutation tests) for the duration of a block."""
    global _lib
    saved = _load()
    _lib = _configure(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def gll_nodes(N: int) -> np.ndarray:
    xi = np.zeros(N + 1)
    if _load().oracle_gll_nodes(N, _ptr(xi)) != 0:
        raise ValueError(f"N={N} out of range")
    return xi


def diff_matrix(N: int) -> np.ndarray:
    xi = gll_nodes(N)
    D = np.zeros((N + 1, N + 1))
    if _load().oracle_diff_matrix(N, _ptr(xi), _ptr(D)) != 0:
        raise ValueError(f"N={N} out of range")
    return D


def pressure(Theta: float, p0: float, R: float, cp: float) -> float:
    return _load().oracle_pressure(float(Theta), p0, R, cp)


def max_threads() -> int:
    return _load().oracle_max_threads()


class _Bound:
    """Keeps the numpy arrays alive while C holds pointers into them."""

    def __init__(self, prob: dict):
        N = int(prob["N"])
        self.N, self.Ne = N, int(prob["Ne"])
        self.nf = 5 + int(prob.get("ntracers", 0))
        self.M = self.Ne * (N + 1) ** 3
        self.D = np.ascontiguousarray(prob["D"] if "D" in prob else diff_matrix(N),
                                    dtype=np.float64)
        g = np.asarray(prob["g"])
        self.g = [np.ascontiguousarray(g[s], dtype=np.float64) for s in range(9)]
        self.Jinv = np.ascontiguousarray(prob["Jinv"], dtype=np.float64)
        self.rho_ref = np.ascontiguousarray(prob["rho_ref"], dtype=np.float64)
        self.rt_ref = np.ascontiguousarray(prob["rhotheta_ref"], dtype=np.float64)
        for a in self.g + [self.Jinv, self.rho_ref, self.rt_ref]:
            if a.shape != (self.M,):
                raise ValueError("per-node arrays must have Ne*(N+1)^3 entries")
        s = _Problem()
        s.N, s.Ne = N, self.Ne
        s.D = _ptr(self.D)
        for k in range(9):
            s.g[k] = _ptr(self.g[k])
        s.Jinv, s.rho_ref, s.rhotheta_ref = _ptr(self.Jinv), _ptr(self.rho_ref), _ptr(self.rt_ref)
        s.p0, s.R, s.cp, s.grav = (float(prob["p0"]), float(prob["R"]),
                                   float(prob["cp"]), float(prob["grav"]))
        s.ntracers = self.nf - 5
        self.s = s

    def state(self, q) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(self.nf, -1)
        if q.shape[1] != self.M:
            raise ValueError("q must be (5 + ntracers, Ne*(N+1)^3)")
        return q


def vol_rhs_o1(prob: dict, q) -> np.ndarray:
    b = _Bound(prob)
    q = b.state(q)
    out = np.empty((b.nf, b.M))
    if _load().oracle_vol_rhs_o1(C.byref(b.s), _ptr(q), _ptr(out)) != 0:
        raise RuntimeError("oracle O1 rejected its arguments")
    return out


def vol_rhs_o2(prob: dict, q, nthreads: int = 0) -> np.ndarray:
    b = _Bound(prob)
    q = b.state(q)
    out = np.empty((b.nf, b.M))
    if _load().oracle_vol_rhs_o2(C.byref(b.s), _ptr(q), _ptr(out), int(nthreads)) != 0:
        raise RuntimeError("oracle O2 failed")
    return out


def vol_rhs_abs(prob: dict, q) -> np.ndarray:
    """Running error bound: |Jinv| sum_d sum_n |D| |F| (+ |gravity term|) per point."""
    b = _Bound(prob)
    q = b.state(q)
    out = np.empty((b.nf, b.M))
    if _load().oracle_vol_rhs_abs(C.byref(b.s), _ptr(q), _ptr(out)) != 0:
        raise RuntimeError("oracle error bound rejected its arguments")
    return out


def lsrk_coefficients():
    """(A, B, C) of the five-stage fourth-order 2N-storage Runge-Kutta scheme."""
    A, B, Cc = np.zeros(5), np.zeros(5), np.zeros(5)
    _load().oracle_lsrk_coefficients(_ptr(A), _ptr(B), _ptr(Cc))
    return A, B, Cc


def lsrk(prob: dict, q, dt: float, nsteps: int, nthreads: int = 0) -> np.ndarray:
    """q advanced by nsteps low-storage RK steps of dq/dt = volume term (a copy)."""
    b = _Bound(prob)
    out = np.array(b.state(q), dtype=np.float64, copy=True)
    if _load().oracle_lsrk(C.byref(b.s), _ptr(out), float(dt), int(nsteps), int(nthreads)) != 0:
        raise RuntimeError("oracle LSRK failed")
    return out


def lsrk_scalar(lam: float, y0: float, dt: float, nsteps: int) -> float:
    return _load().oracle_lsrk_scalar(float(lam), float(y0), float(dt), int(nsteps))


def condition_numbers(prob: dict, q, rhs=None) -> np.ndarray:
    """Per field: max of the running error bound over max |rhs|."""
    ab = vol_rhs_abs(prob, q)
    rhs = vol_rhs_o2(prob, q) if rhs is None else np.asarray(rhs).reshape(ab.shape[0], -1)
    return np.array([ab[f].max() / max(np.abs(rhs[f]).max(), 1e-300) for f in range(ab.shape[0])])


def vol_rhs_points(prob: dict, q, node_ids) -> np.ndarray:
    b = _Bound(prob)
    q = b.state(q)
    ids = np.ascontiguousarray(node_ids, dtype=np.int64)
    out = np.empty((b.nf, ids.size))
    rc = _load().oracle_vol_rhs_points(C.byref(b.s), _ptr(q), ids.size,
                                       ids.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(out))
    if rc != 0:
        raise RuntimeError("oracle pointwise evaluation rejected its arguments")
    return out


__all__ = ["gll_nodes", "diff_matrix", "pressure", "vol_rhs_o1", "vol_rhs_o2",
           "vol_rhs_points", "vol_rhs_abs", "condition_numbers", "lsrk", "lsrk_coefficients",
           "lsrk_scalar", "max_threads", "build_oracle"]

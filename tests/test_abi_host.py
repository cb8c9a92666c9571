"""Host-side checks of the C ABI: no GPU needed.

* libnumavol.so builds for sm_103a, loads, and exports every function that
  include/*.h declares.
* The differentiation matrix the kernels apply (numa_vol_diff_matrix: closed
  Legendre form plus negative-sum diagonal) agrees with the oracle's
  (Lagrange definition).
* Invalid arguments are rejected on the host with NUMA_EINVAL, before any
  CUDA call.
"""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import _lib, build
from paper_1604_08501_gb300.numa_vol import diff_matrix

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(numa_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("numa_vol_create", "numa_vol_rhs", "numa_vol_destroy", "numa_vol_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("N", range(1, 16))
def test_library_diff_matrix_matches_oracle(N):
    D_lib = diff_matrix(N)
    D_or = oracle.diff_matrix(N)
    assert np.max(np.abs(D_lib - D_or)) <= 4e-15 * max(1.0, N * (N + 1) / 4)
    # negative-sum diagonal: rows sum to (almost exactly) zero
    assert np.max(np.abs(D_lib.sum(axis=1))) < 1e-14


def test_diff_matrix_rejects_bad_order(lib):
    D = np.zeros(256)
    p = D.ctypes.data_as(C.POINTER(C.c_double))
    assert lib.numa_vol_diff_matrix(0, p) == _lib.NUMA_EINVAL
    assert lib.numa_vol_diff_matrix(16, p) == _lib.NUMA_EINVAL
    assert b"N must be" in lib.numa_vol_last_error()
    assert lib.numa_vol_diff_matrix(3, None) == _lib.NUMA_EINVAL


def _geometry(M):
    arrays = [np.ones(M) for _ in range(12)]
    geo = _lib.numa_geometry()
    for s in range(9):
        geo.g[s] = arrays[s].ctypes.data
    geo.Jinv, geo.rho_ref, geo.rhotheta_ref = (arrays[9].ctypes.data, arrays[10].ctypes.data,
                                               arrays[11].ctypes.data)
    return geo, arrays


def test_create_rejects_invalid_arguments_without_a_gpu(lib):
    geo, keep = _geometry(8)
    consts = _lib.numa_constants(1e5, 287.0, 1004.0, 9.8)
    h = C.c_void_p()
    for N, Ne in ((0, 1), (16, 1), (-1, 1), (1, -1)):
        mesh = _lib.numa_mesh(Ne, N)
        assert lib.numa_vol_create(C.byref(mesh), C.byref(geo), C.byref(consts), 0,
                                   C.byref(h)) == _lib.NUMA_EINVAL
        assert h.value is None
    # tracers: 0..3 (checked before any device work)
    for T, prec, code in ((4, 0, _lib.NUMA_EINVAL), (-1, 0, _lib.NUMA_EINVAL),
                          (4, _lib.NUMA_DF64, _lib.NUMA_EINVAL)):
        mesh = _lib.numa_mesh(1, 7 if prec == _lib.NUMA_DF64 else 1, T)
        assert lib.numa_vol_create(C.byref(mesh), C.byref(geo), C.byref(consts), prec,
                                   C.byref(h)) == code
        assert h.value is None
    # orders above 7 do not exist in NUMA_DF64 (checked before any device work)
    for prec in (_lib.NUMA_DF64,):
        mesh = _lib.numa_mesh(1, 8)
        assert lib.numa_vol_create(C.byref(mesh), C.byref(geo), C.byref(consts), prec,
                                   C.byref(h)) == _lib.NUMA_EUNSUPPORTED
        assert h.value is None
    mesh = _lib.numa_mesh(1, 1)
    bad = _lib.numa_constants(1e5, 287.0, 200.0, 9.8)         # cp < R
    assert lib.numa_vol_create(C.byref(mesh), C.byref(geo), C.byref(bad), 0,
                               C.byref(h)) == _lib.NUMA_EINVAL
    geo.Jinv = None
    assert lib.numa_vol_create(C.byref(mesh), C.byref(geo), C.byref(consts), 0,
                               C.byref(h)) == _lib.NUMA_EINVAL
    assert b"NULL" in lib.numa_vol_last_error()
    assert lib.numa_vol_create(None, None, None, 0, C.byref(h)) == _lib.NUMA_EINVAL
    assert lib.numa_vol_create(C.byref(mesh), C.byref(geo), C.byref(consts), 0,
                               None) == _lib.NUMA_EINVAL


def test_rhs_rejects_null_handle(lib):
    assert lib.numa_vol_rhs(None, None, None, None) == _lib.NUMA_EINVAL
    assert lib.numa_vol_rhs_host(None, None, None) == _lib.NUMA_EINVAL
    lib.numa_vol_destroy(None)   # no-op


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_batch_engine_and_noalloc_reject_bad_arguments_without_a_gpu(lib):
    # Host-side validation returns status codes before any device work.
    vp = C.c_void_p
    assert lib.numa_batch_create(_lib.NUMA_DF64, C.byref(vp())) == _lib.NUMA_EUNSUPPORTED
    assert lib.numa_batch_create(_lib.NUMA_FP64, None) == _lib.NUMA_EINVAL
    assert lib.numa_batch_add(None, None, None, None) == _lib.NUMA_EINVAL
    assert lib.numa_batch_advance(None, 1, 0.01, None) == _lib.NUMA_EINVAL
    assert lib.numa_batch_tile(None, 8) == 0
    assert lib.numa_engine_create(_lib.NUMA_DF64, 1 << 20, 4, C.byref(vp())) == _lib.NUMA_EUNSUPPORTED
    assert lib.numa_engine_create(_lib.NUMA_FP64, 1 << 20, 0, C.byref(vp())) == _lib.NUMA_EINVAL
    assert lib.numa_engine_create(_lib.NUMA_FP64, 16, 4, C.byref(vp())) == _lib.NUMA_EINVAL
    rid = C.c_int64()
    assert lib.numa_engine_submit(None, None, None, None, 1, 0.01, C.byref(rid)) == _lib.NUMA_EINVAL
    assert lib.numa_engine_cancel(None, 1) == _lib.NUMA_EINVAL
    n = C.c_int()
    assert lib.numa_engine_progress(None, None, 0, C.byref(n)) == _lib.NUMA_EINVAL
    assert lib.numa_engine_query(None, 1, None) == _lib.NUMA_EINVAL
    assert lib.numa_engine_stats(None, None) == _lib.NUMA_EINVAL
    assert lib.numa_engine_checkpoint(None, 1, None, None) == _lib.NUMA_EINVAL
    assert lib.numa_engine_set_round_steps(None, 2) == _lib.NUMA_EINVAL
    assert lib.numa_engine_set_round_policy(None, 1) == _lib.NUMA_EINVAL
    assert b"NULL" in lib.numa_engine_last_error()
    lib.numa_engine_destroy(None)                        # no-op
    # the allocation-free advance: NULL arrays, counts out of range
    hs = (C.c_void_p * 65)()
    ss = (C.c_void_p * 65)()
    assert lib.numa_batch_advance_noalloc(None, None, 1, 1, 0.01, None) == _lib.NUMA_EINVAL
    assert lib.numa_batch_advance_noalloc(hs, ss, 0, 1, 0.01, None) == _lib.NUMA_EINVAL
    assert lib.numa_batch_advance_noalloc(hs, ss, 65, 1, 0.01, None) == _lib.NUMA_ELIMIT
    assert lib.numa_batch_advance_noalloc(hs, ss, 1, -1, 0.01, None) == _lib.NUMA_EINVAL

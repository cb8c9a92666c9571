"""The C ABI from a plain C program (tests/c_client/numa_client.c), compiled
with gcc as C11 with warnings as errors against include/numa_vol.h and linked
to libnumavol.so.

* CPU: the program builds, and its host-only checks pass (GLL D for N = 1, 2
  against the closed forms; invalid arguments rejected with a message).
* GPU: the program evaluates the volume term from host buffers for a problem
  written by the test; the result matches the oracle (FP64 <= 1e-12, mixed
  <= 1e-5, per-field normwise), with tracers and at a high order too.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from conftest import rel_err

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1604_08501_gb300")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    build.build()
    exe = str(tmp_path_factory.mktemp("c_client") / "numa_client")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_client", "numa_client.c"),
           "-L", PKG, "-lnumavol", f"-Wl,-rpath,{PKG}", "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_builds_and_passes_host_checks(client):
    r = subprocess.run([client, "check"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "ok"


def test_c_client_rejects_a_bad_command_line(client):
    r = subprocess.run([client, "rhs", "x", "y", "fp32"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 1


def write_problem(path, w, precision):
    p = w.problem()
    state = w.q_mixed().astype(np.float32) if precision == "mixed" else w.q.astype(np.float64)
    with open(path, "wb") as f:
        f.write(np.array([w.N, p["ntracers"]], dtype="<i4").tobytes())
        f.write(np.array([w.Ne], dtype="<i8").tobytes())
        f.write(np.array([p["p0"], p["R"], p["cp"], p["grav"]], dtype="<f8").tobytes())
        for a in list(p["g"]) + [p["Jinv"], p["rho_ref"], p["rhotheta_ref"]]:
            f.write(np.ascontiguousarray(a, dtype="<f8").tobytes())
        f.write(np.ascontiguousarray(state).astype(state.dtype.newbyteorder("<")).tobytes())


@pytest.mark.gpu
@pytest.mark.parametrize("precision,N,shape,tracers", [
    ("fp64", 4, (3, 2, 1), 0), ("fp64", 7, (5, 3, 2), 0), ("fp64", 11, (2, 1, 1), 3),
    ("mixed", 7, (5, 3, 2), 0), ("mixed", 3, (3, 2, 1), 2)])
def test_c_client_evaluates_the_volume_term(client, tmp_path, precision, N, shape, tracers):
    w = wl.make_workload(N, shape, seed=200 + N, tracers=tracers)
    src, out = str(tmp_path / "problem.bin"), str(tmp_path / "rhs.bin")
    write_problem(src, w, precision)
    r = subprocess.run([client, "rhs", src, out, precision], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    dtype = "<f4" if precision == "mixed" else "<f8"
    got = np.fromfile(out, dtype=dtype).reshape(w.q.shape).astype(np.float64)
    ref = oracle.vol_rhs_o2(w.problem(), w.q)
    tol = 1e-5 if precision == "mixed" else 1e-12
    for f0 in range(0, w.q.shape[0], 5):   # five fields at a time (rel_err takes five)
        g5, r5 = got[f0:f0 + 5], ref[f0:f0 + 5]
        pad = 5 - g5.shape[0]
        if pad:
            g5 = np.concatenate([g5, np.zeros((pad, g5.shape[1]))])
            r5 = np.concatenate([r5, np.zeros((pad, r5.shape[1]))])
        for b, (mx, _) in enumerate(rel_err(g5, r5)):
            assert mx <= tol, (precision, N, f0 + b, mx)

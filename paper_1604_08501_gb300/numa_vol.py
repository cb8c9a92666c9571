"""Python binding of the element volume term (argument marshalling only).

Every step of the computation runs in the CUDA kernels of ``libnumavol.so``.
This module passes pointers, sizes and a stream through the C ABI of
``include/numa_vol.h``.  PyTorch provides device memory and streams.

    vt = VolumeTerm.from_problem(prob)     # numa_vol_create
    rhs = vt.rhs(q)                        # numa_vol_rhs on the current stream
    rhs_host = vt.rhs_host(q_host)         # numa_vol_rhs_host (copies included)
    vt.close()                             # numa_vol_destroy
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (NUMA_DF64, NUMA_FP64, NUMA_MIXED, NUMA_SWEEP_AUTO, NUMA_SWEEP_CUDA_CORES,
                   NUMA_SWEEP_TENSOR_TF32, NumaError, check, check_batch,
                   check_engine)

NFIELDS = 5


def _host_or_device_ptr(a, M: int, keep: list) -> int:
    """Pointer to M contiguous doubles from a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64:
                raise TypeError("geometry tensors must be float64")
            a = a.contiguous()
            if a.numel() != M:
                raise ValueError(f"geometry array has {a.numel()} entries, expected {M}")
            keep.append(a)
            return a.data_ptr()
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if arr.size != M:
        raise ValueError(f"geometry array has {arr.size} entries, expected {M}")
    keep.append(arr)
    return arr.ctypes.data


def diff_matrix(N: int) -> np.ndarray:
    """The GLL differentiation matrix the kernels apply (numa_vol_diff_matrix)."""
    D = np.zeros((N + 1, N + 1))
    check(_lib.load().numa_vol_diff_matrix(int(N), D.ctypes.data_as(C.POINTER(C.c_double))))
    return D


class VolumeTerm:
    """One mesh on the current CUDA device (numa_vol_create ... numa_vol_destroy).

    precision: "fp64" (every operation on the FP64 pipe), "df64" (double-float
    arithmetic on the FP32 pipes, N = 7) or "mixed" (FP32 perturbation state,
    see workload.perturbation_state)."""

    def __init__(self, N: int, num_elements: int, g, Jinv, rho_ref, rhotheta_ref,
                 p0: float, R: float, cp: float, grav: float, precision: str = "fp64",
                 tracers: int = 0):
        lib = _lib.load()
        self.N = int(N)
        self.nf = NFIELDS + int(tracers)
        self.Ne = int(num_elements)
        self.Nq = self.N + 1
        self.M = self.Ne * self.Nq ** 3
        self.precision = precision
        self.dtype_name = "float32" if precision == "mixed" else "float64"
        keep: list = []
        geo = _lib.numa_geometry()
        g = list(g)
        if len(g) != 9:
            raise ValueError("g must hold 9 metric arrays")
        for s in range(9):
            geo.g[s] = _host_or_device_ptr(g[s], self.M, keep)
        geo.Jinv = _host_or_device_ptr(Jinv, self.M, keep)
        geo.rho_ref = _host_or_device_ptr(rho_ref, self.M, keep)
        geo.rhotheta_ref = _host_or_device_ptr(rhotheta_ref, self.M, keep)
        mesh = _lib.numa_mesh(self.Ne, self.N, int(tracers))
        consts = _lib.numa_constants(float(p0), float(R), float(cp), float(grav))
        prec = {"fp64": NUMA_FP64, "df64": NUMA_DF64, "mixed": NUMA_MIXED}[precision]
        h = C.c_void_p()
        check(lib.numa_vol_create(C.byref(mesh), C.byref(geo), C.byref(consts), prec, C.byref(h)))
        self._h = h

    @classmethod
    def from_problem(cls, prob: dict, precision: str = "fp64") -> "VolumeTerm":
        return cls(prob["N"], prob["Ne"], prob["g"], prob["Jinv"], prob["rho_ref"],
                   prob["rhotheta_ref"], prob["p0"], prob["R"], prob["cp"], prob["grav"],
                   precision=precision, tracers=prob.get("ntracers", 0))

    @property
    def handle(self) -> int:
        if self._h is None or not self._h.value:
            raise RuntimeError("VolumeTerm is closed")
        return self._h.value

    def set_sweep(self, sweep: str) -> None:
        """The D sums on the CUDA cores ("cuda_cores") or as TF32 split products
        on the tensor cores ("tensor_tf32": NUMA_MIXED handles of N = 7)."""
        code = {"cuda_cores": NUMA_SWEEP_CUDA_CORES, "tensor_tf32": NUMA_SWEEP_TENSOR_TF32}[sweep]
        check(_lib.load().numa_vol_set_sweep(C.c_void_p(self.handle), code))

    @property
    def kernel_name(self) -> str:
        """The kernel numa_vol_rhs launches for this handle."""
        return _lib.load().numa_vol_kernel_name(self.handle).decode()

    def _torch_dtype(self):
        import torch
        return torch.float32 if self.dtype_name == "float32" else torch.float64

    def rhs(self, q, out=None, stream=None):
        """Enqueue rhs = volume term of q on ``stream`` (default: torch's current
        stream).  q and out are (5 + tracers, M) CUDA tensors: float64 for "fp64" and
        "df64", float32 perturbation state (rho', U1, U2, U3, Theta') for "mixed"."""
        import torch
        dt = self._torch_dtype()
        if not (isinstance(q, torch.Tensor) and q.is_cuda and q.dtype == dt):
            raise TypeError(f"q must be a {dt} CUDA tensor")
        if q.numel() != self.nf * self.M or not q.is_contiguous():
            raise ValueError(f"q must be contiguous with {self.nf} x {self.M} entries")
        if out is None:
            out = torch.empty((self.nf, self.M), dtype=dt, device=q.device)
        elif not (out.is_cuda and out.dtype == dt and out.is_contiguous()
                  and out.numel() == self.nf * self.M):
            raise ValueError("out must be a contiguous CUDA tensor like q")
        if stream is None:
            stream = torch.cuda.current_stream(q.device)
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        check(_lib.load().numa_vol_rhs(self.handle, C.c_void_p(q.data_ptr()),
                                       C.c_void_p(out.data_ptr()), C.c_void_p(s)))
        return out

    def rhs_host(self, q, out=None):
        """Volume term of a host state through numa_vol_rhs_host (host-to-device
        copy, kernel, device-to-host copy; synchronous).  Accepts numpy arrays or
        CPU torch tensors of the handle's state type (pinned memory copies
        fastest) and returns ``out``."""
        import torch
        if isinstance(q, torch.Tensor):
            if q.is_cuda or q.dtype != self._torch_dtype() or not q.is_contiguous():
                raise TypeError("q must be a contiguous CPU tensor of the handle's type")
            qp = q.data_ptr()
            if out is None:
                out = torch.empty((self.nf, self.M), dtype=q.dtype, pin_memory=q.is_pinned())
            op = out.data_ptr()
        else:
            q = np.ascontiguousarray(q, dtype=self.dtype_name)
            qp = q.ctypes.data
            if out is None:
                out = np.empty((self.nf, self.M), dtype=self.dtype_name)
            op = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
        if int(np.prod(q.shape)) != self.nf * self.M:
            raise ValueError(f"q must have {self.nf} x {self.M} entries")
        check(_lib.load().numa_vol_rhs_host(self.handle, C.c_void_p(qp), C.c_void_p(op)))
        return out

    def status(self, stream=None) -> None:
        """numa_vol_status: raise NumaError(NUMA_ETIMEOUT) if a kernel enqueued on
        this handle gave up a bounded wait (reads and clears the status word)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        check(_lib.load().numa_vol_status(self.handle, C.c_void_p(s)))

    def selftest_wait(self, limit_us: int, stream=None) -> None:
        """numa_vol_selftest_wait: enqueue a bounded device wait that runs out
        after limit_us; the next status() on the stream raises NUMA_ETIMEOUT."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        check(_lib.load().numa_vol_selftest_wait(self.handle, int(limit_us), C.c_void_p(s)))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().numa_vol_destroy(self._h)
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched low-storage Runge-Kutta integration of many VolumeTerm instances
    (numa_batch_*).  States are CUDA tensors the batch updates in place."""

    SWEEPS = {"cuda_cores": NUMA_SWEEP_CUDA_CORES, "tensor_tf32": NUMA_SWEEP_TENSOR_TF32,
              "auto": NUMA_SWEEP_AUTO}

    def __init__(self, precision: str = "fp64", sweep: str = "cuda_cores"):
        self.precision = precision
        h = C.c_void_p()
        prec = {"fp64": NUMA_FP64, "mixed": NUMA_MIXED}[precision]
        check_batch(_lib.load().numa_batch_create(prec, C.byref(h)))
        self._h = h
        self._keep = []          # (VolumeTerm, state) pairs the device table points to
        if sweep != "cuda_cores":
            self.sweep = sweep

    @property
    def sweep(self) -> str:
        """How the D sums are evaluated: "cuda_cores", "tensor_tf32" (mixed only)
        or "auto" (the autotuner picks per order)."""
        v = _lib.load().numa_batch_sweep(self.handle)
        return {v2: k for k, v2 in self.SWEEPS.items()}[v]

    def sweep_of(self, nq: int) -> str:
        """The sweep order Nq uses now: "cuda_cores" or "tensor_tf32"."""
        v = _lib.load().numa_batch_sweep_of(self.handle, int(nq))
        return {NUMA_SWEEP_CUDA_CORES: "cuda_cores", NUMA_SWEEP_TENSOR_TF32: "tensor_tf32"}[v]

    @sweep.setter
    def sweep(self, name: str) -> None:
        check_batch(_lib.load().numa_batch_set_sweep(self.handle, self.SWEEPS[name]))

    def config(self) -> dict:
        """The launch configuration: tile (elements per work item) and sweep by
        Nq, CTAs per SM, item order, and the last autotune's ms per step and
        candidates timed."""
        c = _lib.numa_batch_config()
        check_batch(_lib.load().numa_batch_get_config(self.handle, C.byref(c)))
        names = {NUMA_SWEEP_CUDA_CORES: "cuda_cores", NUMA_SWEEP_TENSOR_TF32: "tensor_tf32"}
        return {"tile": {nq: c.tile[nq] for nq in range(2, 9)},
                "sweep": {nq: names[c.sweep[nq]] for nq in range(2, 9)},
                "ctas_per_sm": c.ctas_per_sm, "costliest_first": bool(c.costliest_first),
                "state_in_tmem": bool(c.state_in_tmem),
                "tuned_ms_per_step": c.tuned_ms_per_step,
                "tuned_candidates": c.tuned_candidates}

    def set_config(self, tile=None, sweep=None, ctas_per_sm=None, costliest_first=None,
                   state_in_tmem=None) -> None:
        """Set any of the configuration fields of config() (the others stay)."""
        cur = self.config()
        c = _lib.numa_batch_config()
        for nq in range(2, 9):
            c.tile[nq] = int((tile or {}).get(nq, cur["tile"][nq]))
            c.sweep[nq] = self.SWEEPS[(sweep or {}).get(nq, cur["sweep"][nq])]
        c.ctas_per_sm = int(cur["ctas_per_sm"] if ctas_per_sm is None else ctas_per_sm)
        c.costliest_first = int(cur["costliest_first"] if costliest_first is None
                                else bool(costliest_first))
        c.state_in_tmem = int(cur["state_in_tmem"] if state_in_tmem is None
                              else bool(state_in_tmem))
        check_batch(_lib.load().numa_batch_set_config(self.handle, C.byref(c)))

    def status(self, stream=None) -> None:
        """Raise NumaError(NUMA_ETIMEOUT) if a launch's bounded device wait ran out."""
        check_batch(_lib.load().numa_batch_status(self.handle, C.c_void_p(self._stream(stream))))

    @property
    def handle(self) -> int:
        if self._h is None or not self._h.value:
            raise RuntimeError("Batch is closed")
        return self._h.value

    def add(self, vt: "VolumeTerm", q) -> int:
        import torch
        if not (isinstance(q, torch.Tensor) and q.is_cuda and q.is_contiguous()
                and q.dtype == vt._torch_dtype() and q.numel() == vt.nf * vt.M):
            raise TypeError("q must be the instance's contiguous CUDA state tensor")
        idx = C.c_int()
        check_batch(_lib.load().numa_batch_add(self.handle, C.c_void_p(vt.handle),
                                               C.c_void_p(q.data_ptr()), C.byref(idx)))
        self._keep.append((vt, q))
        return idx.value

    def clear(self) -> None:
        check_batch(_lib.load().numa_batch_clear(self.handle))
        self._keep = []

    def __len__(self) -> int:
        return _lib.load().numa_batch_size(self.handle)

    def _stream(self, stream):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    def advance(self, nsteps: int, dt: float, stream=None) -> None:
        check_batch(_lib.load().numa_batch_advance(self.handle, int(nsteps), float(dt),
                                                   C.c_void_p(self._stream(stream))))

    def autotune(self, stream=None) -> None:
        check_batch(_lib.load().numa_batch_autotune(self.handle, C.c_void_p(self._stream(stream))))

    def tile(self, nq: int) -> int:
        return _lib.load().numa_batch_tile(self.handle, int(nq))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().numa_batch_destroy(self._h)
        self._h = None
        self._keep = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(a):
    """Address of a host buffer (numpy array or CPU torch tensor)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("host buffers must be contiguous")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor) and not a.is_cuda and a.is_contiguous():
        return a.data_ptr()
    raise TypeError("host buffers are numpy arrays or contiguous CPU tensors")


class Engine:
    """Serving engine (numa_engine_*): continuous batching of ensemble-member
    requests.  Each request advances a copy of an initial state on a resident
    mesh (a VolumeTerm) by nsteps low-storage RK steps; the final state lands
    in the request's host output buffer.  round_steps bounds the steps of one
    round; round_policy "lockstep" advances every resident by the same count
    (the smallest remaining), "per_member" each by its own (see
    numa_engine_set_round_policy)."""

    STATUS = {0: "queued", 1: "running", 2: "done", 3: "cancelled"}

    ROUND_POLICIES = {"lockstep": 0, "per_member": 1}   # NUMA_ROUND_*

    def __init__(self, precision: str = "fp64", budget_bytes: int = 1 << 30,
                 max_members: int = 256, round_steps: int = 1, round_policy: str = "lockstep"):
        self.precision = precision
        h = C.c_void_p()
        prec = {"fp64": NUMA_FP64, "mixed": NUMA_MIXED}[precision]
        check_engine(_lib.load().numa_engine_create(prec, int(budget_bytes), int(max_members),
                                                    C.byref(h)))
        self._h = h
        self._bufs = {}          # request id -> (mesh, q0, out) kept alive while in flight
        if round_steps != 1:
            check_engine(_lib.load().numa_engine_set_round_steps(self.handle, int(round_steps)))
        if round_policy != "lockstep":
            check_engine(_lib.load().numa_engine_set_round_policy(
                self.handle, self.ROUND_POLICIES[round_policy]))

    @property
    def handle(self) -> int:
        if self._h is None or not self._h.value:
            raise RuntimeError("Engine is closed")
        return self._h.value

    def submit(self, mesh: "VolumeTerm", q0, out, nsteps: int, dt: float) -> int:
        rid = C.c_int64()
        check_engine(_lib.load().numa_engine_submit(
            self.handle, C.c_void_p(mesh.handle), C.c_void_p(_host_ptr(q0)),
            C.c_void_p(_host_ptr(out)), int(nsteps), float(dt), C.byref(rid)))
        self._bufs[rid.value] = (mesh, q0, out)
        return rid.value

    def cancel(self, rid: int) -> None:
        check_engine(_lib.load().numa_engine_cancel(self.handle, C.c_int64(rid)))

    def progress(self, max_done: int = 4096):
        """Enqueue one round; returns the ids of requests whose final state has
        reached host memory since the last call."""
        ids = (C.c_int64 * max_done)()
        n = C.c_int()
        check_engine(_lib.load().numa_engine_progress(self.handle, ids, max_done, C.byref(n)))
        done = [ids[k] for k in range(n.value)]
        for rid in done:
            self._bufs.pop(rid, None)
        return done

    def drain(self, max_done: int = 4096):
        """Wait for everything enqueued; returns the ids of requests that finished."""
        ids = (C.c_int64 * max_done)()
        n = C.c_int()
        check_engine(_lib.load().numa_engine_drain(self.handle, ids, max_done, C.byref(n)))
        done = [ids[k] for k in range(n.value)]
        for rid in done:
            self._bufs.pop(rid, None)
        return done

    def query(self, rid: int) -> dict:
        info = _lib.numa_request_info()
        check_engine(_lib.load().numa_engine_query(self.handle, C.c_int64(rid), C.byref(info)))
        if info.status == 3:
            self._bufs.pop(rid, None)
        return {"id": info.id, "status": self.STATUS[info.status], "submit_s": info.submit_s,
                "admit_s": info.admit_s, "done_s": info.done_s}

    def checkpoint(self, rid: int, out=None):
        """numa_engine_checkpoint: (state after the request's last completed
        step, steps done).  Submit the state with the remaining steps to resume."""
        mesh, q0, _ = self._bufs[rid]
        if out is None:
            out = np.empty_like(np.asarray(q0))
        done = C.c_int()
        check_engine(_lib.load().numa_engine_checkpoint(self.handle, C.c_int64(rid),
                                                        C.c_void_p(_host_ptr(out)), C.byref(done)))
        return out, done.value

    def stats(self) -> dict:
        c = _lib.numa_engine_counters()
        check_engine(_lib.load().numa_engine_stats(self.handle, C.byref(c)))
        return {f: getattr(c, f) for f, _ in c._fields_}

    def run_until_idle(self, max_rounds: int = 1_000_000):
        done = []
        for _ in range(max_rounds):
            st = self.stats()
            if st["queued"] == 0 and st["resident"] == 0:
                break
            done += self.progress()
        return done

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().numa_engine_destroy(self._h)
        self._h = None
        self._bufs = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["VolumeTerm", "Batch", "Engine", "diff_matrix", "NumaError"]

"""Seeded synthetic inputs for the element volume term: mesh, metric terms,
hydrostatic reference state and perturbed state.

This module is shared by the tests, the benchmark and the oracle checks. It
holds none of the volume term's arithmetic: no differentiation matrix, no
equation of state of the model and no flux. It places GLL points (using
scipy's Gauss-Jacobi root finder) and evaluates closed-form geometry and
thermodynamics.

The workload follows the paper's setting (Sec. 2): a dry atmosphere on a
curvilinear hexahedral mesh of tensor-product elements with Nq^3 points each.
The benchmark adds a sine warp of a 10 km box, an isothermal hydrostatic
reference state and small seeded perturbations:

* Box [0, L]^3 split into nx*ny*nz elements. Element e = ex + nx*(ey + ny*ez).
  Within an element, point (i, j, k) sits at the GLL node (xi_i, xi_j, xi_k).
* Warp, applied to all three axes at once from the unwarped coordinates:
  x = xh + A s(yh) s(zh), y = yh + A s(zh) s(xh), z = zh + A s(xh) s(yh),
  where s(u) = sin(pi u / L) and A = warp * L. The box boundary stays fixed.
* Metric terms are analytic, g_{a,d} = J dxi_d/dx_a. With a_d = dx/dxi_d, the
  three vectors are J grad(xi_r) = a_s x a_t, J grad(xi_s) = a_t x a_r and
  J grad(xi_t) = a_r x a_s, and J = a_r . (a_s x a_t). They are stored as
  g[3*d + a].
* The reference state is isothermal (T = 300 K) and hydrostatic:
  p_h = p0 exp(-grav z / (R T)), rho_ref = p_h / (R T),
  theta_ref = T (p0 / p_h)^(R / cp) and Theta_ref = rho_ref * theta_ref.
  Here z is the warped height of the point.
* The state is rho = rho_ref (1 + eps B_rho), theta = theta_ref (1 + eps B_theta)
  and Theta = rho * theta. Velocities u, v and w are i.i.d. uniform(-vmax, vmax)
  at every point, and U_a = rho u_a. Each B is a sum of four Gaussian bumps
  a exp(-|x - c|^2 / w^2), with centres uniform in the box, widths uniform in
  [0.1 L, 0.3 L] and amplitudes uniform in [-1, 1]. The draws come from
  numpy's PCG64 in this order: the bumps of B_rho, the bumps of B_theta, then
  the velocities (3 x M values, field-major).
* Time-integration workloads (the batched integrator and the serving engine)
  take smooth velocities instead: u_a = vmax B_a / max|B_a|, with B_a a sum of
  four Gaussian bumps as above, drawn after B_theta.  Independent per-point
  velocities make the flow compress and expand at node scale: advanced ten
  0.01 s steps on the finest meshes of the batch (323 m elements), the density
  turns negative.  The smooth field keeps every state physical over the
  workloads' 20-step horizon.

Per-point arrays use [e][k][j][i] order with i fastest. State fields are
planes in the order (rho, U1, U2, U3, Theta).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import os

import numpy as np

NFIELDS = 5
FIELD_NAMES = ("rho", "U1", "U2", "U3", "Theta", "Q1", "Q2", "Q3")


@dataclass(frozen=True)
class Constants:
    """Dry-air constants of the benchmark (SI units)."""
    p0: float = 1.0e5
    R: float = 287.17
    cp: float = 1004.67
    grav: float = 9.80616

    def as_dict(self) -> dict:
        return {"p0": self.p0, "R": self.R, "cp": self.cp, "grav": self.grav}


DRY_AIR = Constants()
# The paper's nondimensional set (p_p0 = 1, p_Gamma = 1.4, p_R = 1), with cp
# chosen so that cp / (cp - R) = 1.4, and no gravity.
PAPER_UNITS = Constants(p0=1.0, R=1.0, cp=3.5, grav=0.0)


def gll_points(N: int) -> np.ndarray:
    """GLL points on [-1, 1]: the endpoints and the roots of P_N'.

    The interior points are the Gauss-Jacobi(1, 1) points of degree N - 1
    (P_N' is proportional to P^(1,1)_{N-1}). They come from scipy's
    ``roots_jacobi``, which is independent of the Newton iterations in the
    oracle and in the library."""
    if N < 1:
        raise ValueError("N must be >= 1")
    from scipy.special import roots_jacobi
    inner = roots_jacobi(N - 1, 1.0, 1.0)[0] if N > 1 else np.zeros(0)
    pts = np.concatenate(([-1.0], np.sort(inner), [1.0]))
    return pts


@dataclass
class Mesh:
    N: int
    shape: tuple            # (nx, ny, nz)
    L: float
    x: np.ndarray           # (3, M) physical coordinates
    g: np.ndarray           # (9, M) metric terms, g[3*d + a] = g_{a+1, d+1}
    Jinv: np.ndarray        # (M,)

    @property
    def Nq(self) -> int:
        return self.N + 1

    @property
    def Ne(self) -> int:
        return int(np.prod(self.shape))

    @property
    def M(self) -> int:
        return self.Ne * self.Nq ** 3


def _node_axes(N: int, shape, L: float, z_range=None):
    """Unwarped coordinates, broadcastable to (nz, ny, nx, Nq, Nq, Nq); with
    z_range = (z0, z1) only the element layers z0 <= ez < z1."""
    nx, ny, nz = shape
    z0, z1 = (0, nz) if z_range is None else z_range
    Nq = N + 1
    r = (gll_points(N) + 1.0) * 0.5
    hx, hy, hz = L / nx, L / ny, L / nz
    xh = (np.arange(nx)[:, None] + r[None, :]) * hx   # (nx, Nq)
    yh = (np.arange(ny)[:, None] + r[None, :]) * hy
    zh = (np.arange(z0, z1)[:, None] + r[None, :]) * hz
    xh = xh.reshape(1, 1, nx, 1, 1, Nq)
    yh = yh.reshape(1, ny, 1, 1, Nq, 1)
    zh = zh.reshape(z1 - z0, 1, 1, Nq, 1, 1)
    return xh, yh, zh, (hx, hy, hz)


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _finish(N, shape, L, X, a_r, a_s, a_t) -> Mesh:
    full = (shape[2], shape[1], shape[0], N + 1, N + 1, N + 1)
    M = int(np.prod(full))
    bc = lambda v: np.broadcast_to(v, full)
    a_r = [bc(c) for c in a_r]
    a_s = [bc(c) for c in a_s]
    a_t = [bc(c) for c in a_t]
    gr = _cross(a_s, a_t)
    gs = _cross(a_t, a_r)
    gt = _cross(a_r, a_s)
    J = a_r[0] * gr[0] + a_r[1] * gr[1] + a_r[2] * gr[2]
    if np.any(J <= 0):
        raise ValueError("mapping is not orientation preserving")
    g = np.empty((9, M))
    for d, gd in enumerate((gr, gs, gt)):
        for a in range(3):
            g[3 * d + a] = np.ascontiguousarray(gd[a]).reshape(M)
    x = np.empty((3, M))
    for a in range(3):
        x[a] = np.ascontiguousarray(bc(X[a])).reshape(M)
    return Mesh(N=N, shape=tuple(shape), L=L, x=x, g=g,
                Jinv=np.ascontiguousarray(1.0 / J).reshape(M))


def warped_box(N: int, shape=(8, 8, 8), L: float = 10_000.0, warp: float = 0.05,
               z_range=None) -> Mesh:
    """The benchmark mesh: the sine-warped box described in the module docstring.
    z_range = (z0, z1): only the element layers z0 <= ez < z1 (elements
    e = ex + nx (ey + ny ez), so a contiguous range of elements), point for
    point the same values as those elements of the whole mesh."""
    xh, yh, zh, (hx, hy, hz) = _node_axes(N, shape, L, z_range)
    if z_range is not None:
        shape = (shape[0], shape[1], z_range[1] - z_range[0])
    A = warp * L
    k = math.pi / L
    sx, sy, sz = np.sin(k * xh), np.sin(k * yh), np.sin(k * zh)
    cx, cy, cz = np.cos(k * xh), np.cos(k * yh), np.cos(k * zh)
    X = (xh + A * sy * sz, yh + A * sz * sx, zh + A * sx * sy)
    # a_d = dx/dxi_d. Each xi_d moves only its own unwarped coordinate, by h_d / 2.
    Ak = A * k
    a_r = (0.5 * hx + 0 * sx, 0.5 * hx * Ak * sz * cx, 0.5 * hx * Ak * cx * sy)
    a_s = (0.5 * hy * Ak * cy * sz, 0.5 * hy + 0 * sy, 0.5 * hy * Ak * sx * cy)
    a_t = (0.5 * hz * Ak * sy * cz, 0.5 * hz * Ak * cz * sx, 0.5 * hz + 0 * sz)
    return _finish(N, shape, L, X, a_r, a_s, a_t)


def affine_box(N: int, shape=(2, 2, 2), L: float = 1.0, B=None) -> Mesh:
    """An affine mesh x = B xh of the box (a constant, generally non-orthogonal
    map). Each element is affine, so the metric terms are constant."""
    if B is None:
        B = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])
    B = np.asarray(B, dtype=np.float64)
    xh, yh, zh, (hx, hy, hz) = _node_axes(N, shape, L)
    X = tuple(B[a, 0] * xh + B[a, 1] * yh + B[a, 2] * zh for a in range(3))
    a_r = tuple(np.float64(0.5 * hx * B[a, 0]) for a in range(3))
    a_s = tuple(np.float64(0.5 * hy * B[a, 1]) for a in range(3))
    a_t = tuple(np.float64(0.5 * hz * B[a, 2]) for a in range(3))
    return _finish(N, shape, L, X, a_r, a_s, a_t)


def hydrostatic_reference(z: np.ndarray, c: Constants = DRY_AIR, T: float = 300.0):
    """Isothermal hydrostatic reference state at heights z: (rho_ref, Theta_ref)."""
    p_h = c.p0 * np.exp(-c.grav * z / (c.R * T))
    rho = p_h / (c.R * T)
    theta = T * (c.p0 / p_h) ** (c.R / c.cp)
    return rho, rho * theta


def _bumps(rng: np.random.Generator, L: float, count: int = 4):
    centres = rng.uniform(0.0, L, size=(count, 3))
    widths = rng.uniform(0.1 * L, 0.3 * L, size=count)
    amps = rng.uniform(-1.0, 1.0, size=count)
    return centres, widths, amps


def _eval_bumps_into(out: np.ndarray, x: np.ndarray, bumps) -> None:
    centres, widths, amps = bumps
    for c, w, a in zip(centres, widths, amps):
        r2 = (x[0] - c[0]) ** 2 + (x[1] - c[1]) ** 2 + (x[2] - c[2]) ** 2
        out += a * np.exp(-r2 / (w * w))


def _eval_bumps(x: np.ndarray, bumps) -> np.ndarray:
    """Sum of the Gaussian bumps at the points x (3, M).  Large meshes are
    evaluated in chunks of points on a thread pool (NumPy releases the GIL in
    its element-wise loops); every point sees the same operations in the same
    order, so the result does not depend on the chunking."""
    out = np.zeros(x.shape[1])
    M = x.shape[1]
    chunk = 1 << 19
    if M <= 2 * chunk:
        _eval_bumps_into(out, x, bumps)
        return out
    from concurrent.futures import ThreadPoolExecutor
    starts = range(0, M, chunk)
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(lambda s0: _eval_bumps_into(out[s0:s0 + chunk], x[:, s0:s0 + chunk], bumps),
                    starts))
    return out


def perturbed_state(mesh: Mesh, rho_ref, rhotheta_ref, seed: int,
                    eps: float = 1e-3, vmax: float = 10.0,
                    smooth_velocity: bool = False, point_range=None) -> np.ndarray:
    """Seeded state (5, M): Gaussian-bump perturbations of rho and theta and
    per-point uniform random velocities, or smooth bump velocities of peak vmax
    (see module docstring).  point_range = (p0, M_all): the mesh is the points
    p0 .. p0 + M - 1 of a mesh of M_all points, and the state is those points'
    state in that mesh (the velocity draws are taken from the generator's
    stream at their positions; smooth velocities, normalised over the whole
    mesh, are not available then)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b_rho = _bumps(rng, mesh.L)
    b_theta = _bumps(rng, mesh.L)
    if smooth_velocity:
        if point_range is not None:
            raise ValueError("smooth velocities are normalised over the whole mesh")
        vel = np.empty((3, mesh.M))
        for a in range(3):
            B = _eval_bumps(mesh.x, _bumps(rng, mesh.L))
            vel[a] = vmax * B / max(np.max(np.abs(B)), 1e-300)
    elif point_range is not None:
        # the draws of the whole mesh are 40 for the bumps, then 3 M_all
        # uniforms (velocity a of point p at 40 + a M_all + p), one 64-bit
        # output each: jump the stream to this range's draws
        p0, m_all = point_range
        vel = np.empty((3, mesh.M))
        for a in range(3):
            bg = np.random.PCG64(seed)
            bg.advance(40 + a * m_all + p0)
            vel[a] = np.random.Generator(bg).uniform(-vmax, vmax, size=mesh.M)
    else:
        vel = rng.uniform(-vmax, vmax, size=(3, mesh.M))
    rho = rho_ref * (1.0 + eps * _eval_bumps(mesh.x, b_rho))
    theta = (rhotheta_ref / rho_ref) * (1.0 + eps * _eval_bumps(mesh.x, b_theta))
    q = np.empty((NFIELDS, mesh.M))
    q[0] = rho
    q[1:4] = rho[None, :] * vel
    q[4] = rho * theta
    return q


def perturbation_state(q: np.ndarray, rho_ref: np.ndarray, rhotheta_ref: np.ndarray) -> np.ndarray:
    """The FP32 state a mixed-precision handle takes: (rho - rho_ref, U1, U2, U3,
    Theta - Theta_ref, tracers...), differences formed in FP64 and then rounded
    once."""
    out = np.empty(q.shape, dtype=np.float32)
    out[0] = q[0] - rho_ref
    out[1:4] = q[1:4]
    out[4] = q[4] - rhotheta_ref
    out[5:] = q[5:]          # tracers, if any, as they are
    return out


@dataclass
class Workload:
    """Everything one evaluation of the volume term needs."""
    mesh: Mesh
    consts: Constants
    rho_ref: np.ndarray
    rhotheta_ref: np.ndarray
    q: np.ndarray
    seed: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.mesh.N

    @property
    def Ne(self):
        return self.mesh.Ne

    @property
    def M(self):
        return self.mesh.M

    def q_mixed(self) -> np.ndarray:
        """The state in the FP32 perturbation form of the mixed-precision mode."""
        return perturbation_state(self.q, self.rho_ref, self.rhotheta_ref)

    def problem(self) -> dict:
        """Geometry and constants in the dict form the oracle and the binding take."""
        d = {"N": self.mesh.N, "Ne": self.mesh.Ne, "g": self.mesh.g, "Jinv": self.mesh.Jinv,
             "rho_ref": self.rho_ref, "rhotheta_ref": self.rhotheta_ref,
             "ntracers": self.q.shape[0] - NFIELDS}
        d.update(self.consts.as_dict())
        return d


def tracer_state(mesh: Mesh, rho: np.ndarray, seed: int, count: int) -> np.ndarray:
    """Passive tracers Q_t = rho r_t, mixing ratios r_t = 0.01 (1 + 0.5 B_t)
    with B_t a sum of seeded Gaussian bumps as for the state, drawn from their
    own generator (seed, 1) so that the five base fields do not change."""
    rng = np.random.Generator(np.random.PCG64([seed, 1]))
    Q = np.empty((count, mesh.M))
    for t in range(count):
        Q[t] = rho * 0.01 * (1.0 + 0.5 * _eval_bumps(mesh.x, _bumps(rng, mesh.L)))
    return Q


def make_workload(N: int, n, seed: int, L: float = 10_000.0, warp: float = 0.05,
                  consts: Constants = DRY_AIR, T: float = 300.0, eps: float = 1e-3,
                  vmax: float = 10.0, name: str = "", tracers: int = 0,
                  smooth_velocity: bool = False, z_range=None) -> Workload:
    """Warped box of order N with the seeded perturbed hydrostatic state and
    ``tracers`` (0..3) passive tracers after Theta.
    ``n`` is the number of elements per axis, or a tuple (nx, ny, nz).
    z_range = (z0, z1): only the element layers z0 <= ez < z1, a contiguous
    range of elements, with the same geometry and state as those elements of
    the whole workload (rough velocities, no tracers)."""
    shape = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
    mesh = warped_box(N, shape, L=L, warp=warp, z_range=z_range)
    rho_ref, rt_ref = hydrostatic_reference(mesh.x[2], consts, T)
    point_range = None
    if z_range is not None:
        if tracers:
            raise ValueError("element ranges are generated without tracers")
        per_layer = shape[0] * shape[1] * (N + 1) ** 3
        point_range = (z_range[0] * per_layer, shape[2] * per_layer)
    q = perturbed_state(mesh, rho_ref, rt_ref, seed, eps=eps, vmax=vmax,
                        smooth_velocity=smooth_velocity, point_range=point_range)
    if tracers:
        q = np.concatenate([q, tracer_state(mesh, q[0], seed, tracers)])
    return Workload(mesh=mesh, consts=consts, rho_ref=rho_ref, rhotheta_ref=rt_ref,
                    q=q, seed=seed, name=name,
                    meta={"L": L, "warp": warp, "T": T, "eps": eps, "vmax": vmax, "n": n,
                          "tracers": tracers, "smooth_velocity": smooth_velocity})


def integration_workload(N: int, n, seed: int) -> Workload:
    """An instance of the time-integration workloads (batch, serving): the
    benchmark mesh and state with smooth velocities (module docstring)."""
    return make_workload(N, n, seed=seed, smooth_velocity=True)


def batch_plan(count: int = 64, seed: int = 99, orders=(3, 4, 5, 7),
               ne_range=(512, 32768)):
    """Orders and sizes of a batch of independent instances: N uniform from
    `orders`, element count log-uniform in `ne_range`, rounded to a cube
    n^3 with n = round(Ne^(1/3)).  Instance i uses state seed 100 + i.
    Returns a list of (N, n, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = rng.choice(np.asarray(orders), size=count)
    ne = np.exp(rng.uniform(np.log(ne_range[0]), np.log(ne_range[1]), size=count))
    ns = np.rint(np.cbrt(ne)).astype(int)
    return [(int(N), int(n), 100 + i) for i, (N, n) in enumerate(zip(Ns, ns))]


# The two single-GPU workloads: the small parity case and the timed case.
PARITY_SMALL = dict(N=4, n=8, seed=0, name="N=4 (Nq=5), 8^3=512 elements, warped 10 km box")
BENCH_FULL = dict(N=7, n=32, seed=1,
                  name="N=7 (Nq=8), 32^3=32768 elements (16.8M nodes), warped 10 km box")


def parity_small() -> Workload:
    return make_workload(**PARITY_SMALL)


def bench_full() -> Workload:
    return make_workload(**BENCH_FULL)

"""Plain FP64 CPU oracle for the SPH hot path of the FleCSPH paper (arXiv 2007.03097).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library in ``paper_2007_03097_gb300`` and never imports it.

The heavy loops (brute-force O(N^2) neighbour search, density, forces, Morton
and Hilbert keys) live in ``sph_oracle.c``; this module adds the parts that are plain array
arithmetic: the leapfrog step, conserved totals, leaf levels by definition and
the h-predictor MLP (numpy, FP64).

Parity pins: every function here is checked by ``tests/test_oracle_*.py``
against closed forms, invariants or brute force (see the docstrings there).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

M4, WC2, WC4 = 0, 1, 2
DONE, NOT_CONVERGED, H_BOUNDS = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_int), ("periodic", ctypes.c_int),
        ("box_lo", ctypes.c_double * 3), ("box_hi", ctypes.c_double * 3),
        ("gamma", ctypes.c_double), ("eta", ctypes.c_double),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("eps_visc", ctypes.c_double),
        ("fixed_h", ctypes.c_int), ("h_tol", ctypes.c_double), ("max_sweeps", ctypes.c_int),
        ("h_min", ctypes.c_double), ("h_max", ctypes.c_double), ("dim", ctypes.c_int),
    ]


@dataclass
class Params:
    """Physical and numerical parameters of one SPH evaluation (oracle side)."""
    kernel: int = M4
    periodic: bool = True
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_hi: tuple = (1.0, 1.0, 1.0)
    gamma: float = 5.0 / 3.0
    eta: float = 1.2
    alpha: float = 1.0
    beta: float = 2.0
    eps_visc: float = 0.01
    fixed_h: bool = False
    h_tol: float = 1e-6
    max_sweeps: int = 30
    h_min: float = 1e-6
    h_max: float = 0.25
    dim: int = 3

    def c(self) -> _Params:
        p = _Params()
        p.kernel = int(self.kernel)
        p.periodic = int(bool(self.periodic))
        p.box_lo = (ctypes.c_double * 3)(*self.box_lo)
        p.box_hi = (ctypes.c_double * 3)(*self.box_hi)
        p.gamma, p.eta = self.gamma, self.eta
        p.alpha, p.beta, p.eps_visc = self.alpha, self.beta, self.eps_visc
        p.fixed_h = int(bool(self.fixed_h))
        p.h_tol, p.max_sweeps = self.h_tol, int(self.max_sweeps)
        p.h_min, p.h_max = self.h_min, self.h_max
        p.dim = int(self.dim)
        return p


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        P = ctypes.c_void_p
        _lib.orc_W.restype = d
        _lib.orc_W.argtypes = [i32, i32, d, d]
        _lib.orc_dWdr.restype = d
        _lib.orc_dWdr.argtypes = [i32, i32, d, d]
        _lib.orc_dWdh.restype = d
        _lib.orc_dWdh.argtypes = [i32, i32, d, d]
        _lib.orc_kernel_eval.argtypes = [i32, i32, i64, P, P, P, P, P]
        _lib.orc_morton_keys.argtypes = [i64, P, P, P, P, d, P]
        _lib.orc_hilbert_keys.argtypes = [i64, P, P, P, P, d, P]
        _lib.orc_hilbert_index_many.argtypes = [i64, P, P, P, i32, P]
        _lib.orc_sort_perm.argtypes = [i64, P, P, P]
        _lib.orc_density.restype = i32
        _lib.orc_density.argtypes = [ctypes.POINTER(_Params), i64, P, P, P, P, P, i64, P,
                                     P, P, P, P, P, P, P]
        _lib.orc_neighbors.argtypes = [ctypes.POINTER(_Params), i32, i64, P, P, P, P, i64, P,
                                       P, P, P]
        _lib.orc_eos.argtypes = [i64, d, P, P, P, P]
        _lib.orc_forces.argtypes = [ctypes.POINTER(_Params), i64] + [P] * 11 + [i64, P] + [P] * 8 + [P]
        _lib.orc_energy_rate.argtypes = [ctypes.POINTER(_Params), i64] + [P] * 11 + [i64, P] + [P] * 2
        _lib.orc_num_threads.restype = i32
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# --------------------------------------------------------------------------- kernels
def kernel(kind: int, r, h, dim: int = 3):
    """W, dW/dr, dW/dh of the chosen smoothing kernel (support 2h) in D = dim
    dimensions, elementwise."""
    r = _f64(np.broadcast_to(r, np.broadcast(r, h).shape))
    h = _f64(np.broadcast_to(h, r.shape))
    W, dr, dh = np.empty_like(r), np.empty_like(r), np.empty_like(r)
    lib().orc_kernel_eval(kind, int(dim), r.size, _p(r), _p(h), _p(W), _p(dr), _p(dh))
    return W, dr, dh


# --------------------------------------------------------------------------- keys / sort
def domain(x, y, z, params: Params):
    """Cubic key domain: the periodic box, or for an open boundary the
    bounding-box minimum and L = (largest extent) * (1 + 2^-20)."""
    if params.periodic:
        lo = np.array(params.box_lo, dtype=np.float64)
        L = float(params.box_hi[0] - params.box_lo[0])
        return lo, L
    lo = np.array([x.min(), y.min(), z.min()], dtype=np.float64)
    ext = max(x.max() - x.min(), y.max() - y.min(), z.max() - z.min())
    L = float(ext * (1.0 + 2.0 ** -20))
    return lo, L


def morton_keys(x, y, z, lo, L):
    x, y, z = _f64(x), _f64(y), _f64(z)
    lo = _f64(lo)
    keys = np.empty(x.size, dtype=np.uint64)
    lib().orc_morton_keys(x.size, _p(x), _p(y), _p(z), _p(lo), float(L), _p(keys))
    return keys


def hilbert_keys(x, y, z, lo, L):
    """Hilbert keys (Sec. 2.1, Tree topology) on the Morton cells: 1 << 63 |
    the 63-bit Hilbert index of (ix, iy, iz) after Skilling (2004)."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    lo = _f64(lo)
    keys = np.empty(x.size, dtype=np.uint64)
    lib().orc_hilbert_keys(x.size, _p(x), _p(y), _p(z), _p(lo), float(L), _p(keys))
    return keys


def hilbert_index(ix, iy, iz, bits: int = 21):
    """Hilbert index of integer cells with ``bits`` bits per axis (1..21)."""
    assert 1 <= bits <= 21
    c = [np.ascontiguousarray(a, dtype=np.uint32) for a in (ix, iy, iz)]
    out = np.empty(c[0].size, dtype=np.uint64)
    lib().orc_hilbert_index_many(c[0].size, _p(c[0]), _p(c[1]), _p(c[2]), int(bits), _p(out))
    return out


def keys(x, y, z, lo, L, curve: str = "morton"):
    """Keys of the named curve ("morton" or "hilbert")."""
    return hilbert_keys(x, y, z, lo, L) if curve == "hilbert" else morton_keys(x, y, z, lo, L)


def sort_perm(keys, ids):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    perm = np.empty(keys.size, dtype=np.uint32)
    lib().orc_sort_perm(keys.size, _p(keys), _p(ids), _p(perm))
    return perm


def leaf_levels(sorted_keys, leaf_size: int = 32):
    """Level of the leaf cell holding each particle, by definition (Sec. 2.1,
    tree refinement): the shallowest octree cell containing the particle that
    holds at most ``leaf_size`` particles.  Level l keeps the top 3l key bits
    below the leading 1.  Returns -1 where even level 21 holds too many."""
    keys = np.asarray(sorted_keys, dtype=np.uint64)
    n = keys.size
    out = np.full(n, -1, dtype=np.int32)
    for lvl in range(0, 22):
        pref = keys >> np.uint64(63 - 3 * lvl)
        _, inv, cnt = np.unique(pref, return_inverse=True, return_counts=True)
        fits = (cnt[inv] <= leaf_size) & (out < 0)
        out[fits] = lvl
    return out


# --------------------------------------------------------------------------- density
@dataclass
class DensityResult:
    h: np.ndarray
    rho: np.ndarray
    drho_dh: np.ndarray
    nnb: np.ndarray
    sweeps: np.ndarray
    flags: np.ndarray
    pairs: np.ndarray = None     # neighbour pairs summed over the evaluations
    status: int = 0


def density(params: Params, x, y, z, m, h_seed, targets=None) -> DensityResult:
    """h-rho fixed point (Eqs. 7 and 9) for all particles or for ``targets``.
    Outputs are full-length arrays; entries outside ``targets`` are NaN/0."""
    x, y, z, m, h_seed = map(_f64, (x, y, z, m, h_seed))
    n = x.size
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.size
    h = np.full(n, np.nan)
    rho = np.full(n, np.nan)
    dr = np.full(n, np.nan)
    nnb = np.zeros(n, dtype=np.int32)
    sw = np.zeros(n, dtype=np.int32)
    fl = np.zeros(n, dtype=np.int32)
    pr = np.zeros(n, dtype=np.int64)
    pc = params.c()
    st = lib().orc_density(ctypes.byref(pc), n, _p(x), _p(y), _p(z), _p(m), _p(h_seed), nt, _p(tg),
                           _p(h), _p(rho), _p(dr), _p(nnb), _p(sw), _p(fl), _p(pr))
    return DensityResult(h, rho, dr, nnb, sw, fl, pr, int(st))


def neighbors(params: Params, kind: int, x, y, z, h, targets=None):
    """Sorted neighbour index sets by definition; kind 0 = density, 1 = force.
    Returns (counts, offsets, idx) in CSR form over the targets."""
    x, y, z, h = map(_f64, (x, y, z, h))
    n = x.size
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.size
    counts = np.zeros(nt, dtype=np.int64)
    pc = params.c()
    lib().orc_neighbors(ctypes.byref(pc), kind, n, _p(x), _p(y), _p(z), _p(h), nt, _p(tg),
                        _p(counts), None, None)
    offsets = np.zeros(nt + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    idx = np.empty(max(int(offsets[-1]), 1), dtype=np.int64)
    lib().orc_neighbors(ctypes.byref(pc), kind, n, _p(x), _p(y), _p(z), _p(h), nt, _p(tg),
                        _p(counts), _p(offsets), _p(idx))
    return counts, offsets, idx[: int(offsets[-1])]


def eos(gamma: float, rho, u):
    rho, u = _f64(rho), _f64(u)
    P, c = np.empty_like(rho), np.empty_like(rho)
    lib().orc_eos(rho.size, float(gamma), _p(rho), _p(u), _p(P), _p(c))
    return P, c


@dataclass
class ForceResult:
    ax: np.ndarray
    ay: np.ndarray
    az: np.ndarray
    dudt: np.ndarray
    divv: np.ndarray
    vsig: np.ndarray
    S_a: np.ndarray
    S_u: np.ndarray
    npairs: int = 0


def forces(params: Params, x, y, z, vx, vy, vz, m, h, rho, P, c, targets=None) -> ForceResult:
    """Eqs. 5-6 with Monaghan viscosity for all particles or for ``targets``."""
    arrs = list(map(_f64, (x, y, z, vx, vy, vz, m, h, rho, P, c)))
    n = arrs[0].size
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.size
    outs = [np.full(n, np.nan) for _ in range(8)]
    npairs = ctypes.c_int64(0)
    pc = params.c()
    lib().orc_forces(ctypes.byref(pc), n, *[_p(a) for a in arrs], nt, _p(tg),
                     *[_p(o) for o in outs], ctypes.cast(ctypes.byref(npairs), ctypes.c_void_p))
    return ForceResult(*outs, npairs=int(npairs.value))


def energy_rate(params: Params, x, y, z, vx, vy, vz, m, h, rho, P, c, targets=None):
    """Thermokinetic energy equation (Eq. thermo): de/dt of the specific total
    energy e = u + v^2/2 and its cancellation scale S_e, for all particles or
    for ``targets``."""
    arrs = list(map(_f64, (x, y, z, vx, vy, vz, m, h, rho, P, c)))
    n = arrs[0].size
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.size
    dedt, se = np.full(n, np.nan), np.full(n, np.nan)
    pc = params.c()
    lib().orc_energy_rate(ctypes.byref(pc), n, *[_p(a) for a in arrs], nt, _p(tg), _p(dedt), _p(se))
    return dedt, se


# --------------------------------------------------------------------------- leapfrog
@dataclass
class State:
    """SoA particle state in FP64 (oracle side)."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    m: np.ndarray
    h: np.ndarray
    u: np.ndarray
    ax: np.ndarray = None
    ay: np.ndarray = None
    az: np.ndarray = None
    dudt: np.ndarray = None
    dedt: np.ndarray = None
    rho: np.ndarray = None
    divv: np.ndarray = None
    vsig: np.ndarray = None
    nnb: np.ndarray = None
    extra: dict = field(default_factory=dict)

    def copy(self) -> "State":
        kw = {k: (None if v is None else (v.copy() if isinstance(v, np.ndarray) else v))
              for k, v in self.__dict__.items() if k != "extra"}
        return State(**kw, extra=dict(self.extra))


def evaluate(params: Params, s: State, vx=None, vy=None, vz=None, u=None, thermokinetic=False):
    """Density fixed point at the current positions (seeded by s.h), EOS with
    internal energy ``u`` and force pass with velocities ``v``; fills s (and
    s.dedt, the thermokinetic energy rate, when asked)."""
    vx = s.vx if vx is None else vx
    vy = s.vy if vy is None else vy
    vz = s.vz if vz is None else vz
    u = s.u if u is None else u
    d = density(params, s.x, s.y, s.z, s.m, s.h)
    s.h, s.rho, s.nnb = d.h, d.rho, d.nnb
    P, c = eos(params.gamma, d.rho, u)
    f = forces(params, s.x, s.y, s.z, vx, vy, vz, s.m, d.h, d.rho, P, c)
    s.ax, s.ay, s.az, s.dudt, s.divv, s.vsig = f.ax, f.ay, f.az, f.dudt, f.divv, f.vsig
    s.extra.update(P=P, c=c, sweeps=d.sweeps, flags=d.flags, S_a=f.S_a, S_u=f.S_u,
                   npairs=f.npairs, density_status=d.status)
    if thermokinetic:
        s.dedt, se = energy_rate(params, s.x, s.y, s.z, vx, vy, vz, s.m, d.h, d.rho, P, c)
        s.extra.update(S_e=se)
    return s


def wrap(params: Params, s: State):
    if not params.periodic:
        return
    for d, a in enumerate((s.x, s.y, s.z)):
        lo, hi = params.box_lo[d], params.box_hi[d]
        L = hi - lo
        a[a >= hi] -= L
        a[a < lo] += L


def kdk_step(params: Params, s: State, dt: float) -> State:
    """One kick-drift-kick leapfrog step (the paper names no integrator;
    reading): half kick of v and u with the old rates, drift x in FP64 and
    wrap, density at the new positions, forces evaluated with the predicted
    v_pred = v_half + a_old dt/2 and u_pred = u_half + du_old dt/2, closing
    half kick with the new rates."""
    hdt = 0.5 * dt
    s = s.copy()
    vxh = s.vx + s.ax * hdt
    vyh = s.vy + s.ay * hdt
    vzh = s.vz + s.az * hdt
    uh = s.u + s.dudt * hdt
    s.x = s.x + vxh * dt
    s.y = s.y + vyh * dt
    s.z = s.z + vzh * dt
    wrap(params, s)
    vxp, vyp, vzp = vxh + s.ax * hdt, vyh + s.ay * hdt, vzh + s.az * hdt
    up = uh + s.dudt * hdt
    evaluate(params, s, vxp, vyp, vzp, up)
    s.extra.update(vx_pred=vxp, vy_pred=vyp, vz_pred=vzp, u_pred=up)
    s.vx = vxh + s.ax * hdt
    s.vy = vyh + s.ay * hdt
    s.vz = vzh + s.az * hdt
    s.u = uh + s.dudt * hdt
    return s


def kdk_step_thermokinetic(params: Params, s: State, dt: float) -> State:
    """The kick-drift-kick step of kdk_step with the thermokinetic formulation
    (Eq. thermo): the kicks advance the specific total energy e = u + v^2/2
    with de/dt, and u = e - v^2/2 is recovered after each kick; forces and
    de/dt are evaluated at the predicted v_pred = v_half + a_old dt/2 and
    u_pred = e_pred - v_pred^2/2 with e_pred = e_half + de_old dt/2."""
    hdt = 0.5 * dt
    s = s.copy()
    ke = lambda vx, vy, vz: 0.5 * (vx * vx + vy * vy + vz * vz)
    e = s.u + ke(s.vx, s.vy, s.vz)
    eh = e + s.dedt * hdt
    vxh = s.vx + s.ax * hdt
    vyh = s.vy + s.ay * hdt
    vzh = s.vz + s.az * hdt
    s.x = s.x + vxh * dt
    s.y = s.y + vyh * dt
    s.z = s.z + vzh * dt
    wrap(params, s)
    vxp, vyp, vzp = vxh + s.ax * hdt, vyh + s.ay * hdt, vzh + s.az * hdt
    up = (eh + s.dedt * hdt) - ke(vxp, vyp, vzp)
    evaluate(params, s, vxp, vyp, vzp, up, thermokinetic=True)
    s.extra.update(vx_pred=vxp, vy_pred=vyp, vz_pred=vzp, u_pred=up)
    s.vx = vxh + s.ax * hdt
    s.vy = vyh + s.ay * hdt
    s.vz = vzh + s.az * hdt
    s.u = (eh + s.dedt * hdt) - ke(s.vx, s.vy, s.vz)
    return s


def totals(s: State, vx=None, vy=None, vz=None, u=None):
    """Conserved totals in FP64: momentum sum m v, force sum m a, energy
    sum m (v^2/2 + u), and its rate sum m (v . a + du/dt)."""
    vx = s.vx if vx is None else vx
    vy = s.vy if vy is None else vy
    vz = s.vz if vz is None else vz
    u = s.u if u is None else u
    m = s.m
    mom = np.array([math.fsum(m * vx), math.fsum(m * vy), math.fsum(m * vz)])
    force = np.array([math.fsum(m * s.ax), math.fsum(m * s.ay), math.fsum(m * s.az)])
    energy = math.fsum(m * (0.5 * (vx * vx + vy * vy + vz * vz) + u))
    power = math.fsum(m * (vx * s.ax + vy * s.ay + vz * s.az + s.dudt))
    return dict(momentum=mom, force=force, energy=energy, power=power)


def cfl_dt(s: State, cfl: float = 0.3) -> float:
    """dt = C_cfl min_a h_a / vsig_a (reading; the paper gives no step rule)."""
    return float(cfl * np.min(s.h / s.vsig))


# --------------------------------------------------------------------------- h-predictor MLP
# Not in the paper: a 5 -> 64 -> 64 -> 1 network with SiLU activations whose
# output y gives the predicted s = log(h_next / h_prev) = f3 * y.  Parameter layout (flat): W1[64,5], b1[64],
# W2[64,64], b2[64], W3[1,64], b3[1]; row-major, output index first.
HNET_SHAPES = [(64, 5), (64,), (64, 64), (64,), (1, 64), (1,)]
HNET_NPARAM = sum(int(np.prod(s)) for s in HNET_SHAPES)


def hnet_unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    for shp in HNET_SHAPES:
        k = int(np.prod(shp))
        out.append(theta[o:o + k].reshape(shp))
        o += k
    return out


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def hnet_forward(theta, feats):
    """y = W3 silu(W2 silu(W1 x + b1) + b2) + b3, FP64; returns (y, cache)."""
    W1, b1, W2, b2, W3, b3 = hnet_unpack(theta)
    X = np.asarray(feats, dtype=np.float64)
    z1 = X @ W1.T + b1
    a1 = z1 * _sigmoid(z1)
    z2 = a1 @ W2.T + b2
    a2 = z2 * _sigmoid(z2)
    y = (a2 @ W3.T + b3)[:, 0]
    return y, (X, z1, a1, z2, a2)


def hnet_predict(theta, feats):
    """Predicted log(h_next/h) of the h-predictor: s = f3 * y(f), the network
    output scaled by the feature f3 = div v * dt, so that a particle at rest
    keeps its h exactly and the network learns the gain of the continuity
    estimate (d ln h = div v dt / 3 for a uniform compression)."""
    y, _ = hnet_forward(theta, feats)
    return np.asarray(feats, dtype=np.float64)[:, 3] * y


def hnet_loss_grad(theta, feats, target):
    """Mean squared error L = mean((s - t)^2) of the prediction s = f3 y and
    its gradient with respect to the parameters by backprop."""
    W1, b1, W2, b2, W3, b3 = hnet_unpack(theta)
    y, (X, z1, a1, z2, a2) = hnet_forward(theta, feats)
    t = np.asarray(target, dtype=np.float64)
    B = X.shape[0]
    gain = X[:, 3]
    r = gain * y - t
    loss = float(np.mean(r * r))
    d3 = ((2.0 / B) * r * gain)[:, None]        # dL/dy
    gW3 = d3.T @ a2
    gb3 = d3.sum(axis=0)
    s2 = _sigmoid(z2)
    d2 = (d3 @ W3) * (s2 * (1.0 + z2 * (1.0 - s2)))
    gW2 = d2.T @ a1
    gb2 = d2.sum(axis=0)
    s1 = _sigmoid(z1)
    d1 = (d2 @ W2) * (s1 * (1.0 + z1 * (1.0 - s1)))
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_update(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction, step count t >= 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round FP32 values to bfloat16 (nearest, ties to even) and back to FP64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def hnet_features(h, hprev, nnb, rho, m, divv, dt, eta, rho_ref=1.0, dim=3):
    """Network inputs per particle: log(h/hbar) with hbar = eta (m/rho_ref)^(1/D),
    log(max(nnb, 1/2)/nbar) with nbar the neighbour count of a uniform medium
    inside 2h (32 pi eta^3/3 for D = 3, 4 eta for D = 1), log(rho h^D/(m eta^D))
    (the fixed-point ratio of Eq. 9), div v * dt, and log(h/hprev) (0 when
    hprev <= 0)."""
    h, hprev, rho, m, divv = map(lambda a: np.asarray(a, dtype=np.float64), (h, hprev, rho, m, divv))
    nnb = np.asarray(nnb, dtype=np.float64)
    etaD = eta ** dim
    hbar = eta * (m / rho_ref) ** (1.0 / dim) if dim != 3 else eta * np.cbrt(m / rho_ref)
    nbar = 4.0 * eta if dim == 1 else 32.0 * math.pi * etaD / 3.0
    f4 = np.where(hprev > 0, np.log(np.where(hprev > 0, h / np.where(hprev > 0, hprev, 1.0), 1.0)), 0.0)
    return np.stack([np.log(h / hbar), np.log(np.maximum(nnb, 0.5) / nbar), np.log(rho * h ** dim / (m * etaD)),
                     divv * dt, f4], axis=1)

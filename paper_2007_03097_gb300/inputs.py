"""Seeded synthetic particle sets for the five SPH workloads.

This module only places particles and assigns their initial fields; it holds
none of the SPH arithmetic and imports nothing else from the package, so the
CUDA path, the CPU oracle and the benchmark can all draw the same inputs from
it.  Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), one stream
per (workload, purpose), seed = 1000 * workload + purpose, converted to doubles
in [0, 1) as (z >> 11) * 2^-53.

Workloads (the paper's own runs use its initial-data generators, Sec. 2.1;
these are synthetic stand-ins with the paper's particle distributions):
  lattice   periodic jittered cubic lattice, uniform density, at rest
  sedov     jittered lattice with blast energy on the central particles
  polytrope n = 1 polytrope sampled radially (rho ~ sin(pi r)/(pi r))
  collision two polytropes approaching each other
  turbulence jittered lattice with a k^-4 solenoidal Gaussian velocity field
  sod       1D Sod shock tube (Sec. 3), particles on the x axis
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

M4, WC2, WC4 = 0, 1, 2

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Outputs 1..count of SplitMix64 started from state ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from SplitMix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Workload:
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    m: np.ndarray
    h: np.ndarray
    u: np.ndarray
    params: dict = field(default_factory=dict)
    dt: float | None = None
    steps: int = 1
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.size)

    @property
    def ids(self) -> np.ndarray:
        return np.arange(self.n, dtype=np.uint32)

    def subset(self, idx) -> "Workload":
        """Copy restricted to the given particle indices (same parameters)."""
        f = {k: getattr(self, k)[idx].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u")}
        return Workload(self.name, **f, params=dict(self.params), dt=self.dt, steps=self.steps,
                        info=dict(self.info))


def _base_params(**kw) -> dict:
    p = dict(kernel=M4, periodic=True, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0),
             gamma=5.0 / 3.0, eta=1.2, alpha=1.0, beta=2.0, eps_visc=0.01, cfl=0.3,
             fixed_h=False, h_tol=1e-6, max_sweeps=30, h_min=1e-6, h_max=0.25, rho_ref=1.0,
             precision="fp64")
    p.update(kw)
    # neighbour lists cover 2h (1 + skin); a particle whose h outgrows its
    # list within a step's iteration makes the iteration rebuild the lists
    p.setdefault("skin", 0.05)
    return p


def jittered_lattice(n_side: int, seed: int, jitter: float = 0.1):
    """Sites (i + 1/2)/n_side of the unit cube, x fastest, each component
    shifted by U(-jitter, jitter) lattice spacings."""
    g = (np.arange(n_side, dtype=np.float64) + 0.5) / n_side
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = xx.ravel().copy(), yy.ravel().copy(), zz.ravel().copy()
    n = x.size
    if jitter:
        r = uniform(seed, 3 * n).reshape(n, 3)
        d = (2.0 * r - 1.0) * (jitter / n_side)
        x += d[:, 0]
        y += d[:, 1]
        z += d[:, 2]
    return x, y, z


def lattice(n_side: int = 16, jitter: float = 0.1, kernel: int = M4, h_factor: float = 1.2,
            u0: float = 1.0, fixed_h: bool = True, seed: int = 1001, **kw) -> Workload:
    """Periodic unit box of n_side^3 equal-mass particles (total mass 1) on a
    jittered lattice, at rest, u = u0, h = h_factor lattice spacings."""
    x, y, z = jittered_lattice(n_side, seed, jitter)
    n = x.size
    dx = 1.0 / n_side
    zeros = np.zeros(n)
    params = _base_params(kernel=kernel, fixed_h=fixed_h, eta=h_factor, **kw)
    return Workload("lattice", x, y, z, zeros.copy(), zeros.copy(), zeros.copy(),
                    np.full(n, 1.0 / n), np.full(n, h_factor * dx), np.full(n, u0), params,
                    info=dict(n_side=n_side, jitter=jitter))


def sedov(n_side: int = 64, energy: float = 1.0, n_hot: int = 32, u_cold: float = 1e-5,
          seed: int = 2001, steps: int = 50, dt: float | None = None) -> Workload:
    """Sedov blast in the periodic unit box: rho0 = 1 jittered lattice,
    u = u_cold except the n_hot particles nearest the centre (ties by index)
    that share the blast energy.  Wendland C2, eta = 1.2, variable h."""
    x, y, z = jittered_lattice(n_side, seed, 0.1)
    n = x.size
    m = 1.0 / n
    d2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
    hot = np.lexsort((np.arange(n), d2))[:n_hot]
    u = np.full(n, u_cold)
    u[hot] = energy / (n_hot * m)
    zeros = np.zeros(n)
    eta = 1.2
    h0 = eta * (m / 1.0) ** (1.0 / 3.0)
    params = _base_params(kernel=WC2, eta=eta, fixed_h=False, h_tol=1e-6)
    if dt is None:
        # fixed step from the initial signal speed between two hot particles
        gamma = params["gamma"]
        c_hot = math.sqrt(gamma * (gamma - 1.0) * energy / (n_hot * m))
        dt = params["cfl"] * h0 / (2.0 * c_hot)
    return Workload("sedov", x, y, z, zeros.copy(), zeros.copy(), zeros.copy(), np.full(n, m),
                    np.full(n, h0), u, params, dt=dt, steps=steps,
                    info=dict(n_side=n_side, hot=hot))


def _polytrope_radius(uq: np.ndarray) -> np.ndarray:
    """Invert M(r) = (sin(pi r) - pi r cos(pi r)) / pi on [0, 1] by bisection."""
    lo = np.zeros_like(uq)
    hi = np.ones_like(uq)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        pm = math.pi * mid
        Mm = (np.sin(pm) - pm * np.cos(pm)) / math.pi
        below = Mm < uq
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def polytrope_particles(n: int, seed: int):
    """Positions and profile density of an n = 1 polytrope, R = 1, M = 1:
    rho(r) = rho_c sin(pi r)/(pi r), rho_c = pi/4."""
    r = _polytrope_radius(uniform(seed, n))
    cth = 2.0 * uniform(seed + 1, n) - 1.0
    phi = 2.0 * math.pi * uniform(seed + 2, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    x, y, z = r * sth * np.cos(phi), r * sth * np.sin(phi), r * cth
    pr = np.maximum(math.pi * r, 1e-300)
    rho = (math.pi / 4.0) * np.where(r > 0, np.sin(pr) / pr, 1.0)
    return x, y, z, rho


def polytrope(n: int = 1 << 20, seed: int = 3001, precision: str = "mixed") -> Workload:
    """n = 1 polytrope star (gamma = 2, K = 2/pi, u = K rho), open boundary,
    Wendland C2, eta = 1.2, at rest.  h seeded from the profile density."""
    x, y, z, rho = polytrope_particles(n, seed)
    K = 2.0 / math.pi
    m = 1.0 / n
    eta = 1.2
    rho_s = np.maximum(rho, 0.05 * (math.pi / 4.0))   # floor: a seed, not the SPH density
    h = eta * (m / rho_s) ** (1.0 / 3.0)
    zeros = np.zeros(n)
    params = _base_params(kernel=WC2, periodic=False, gamma=2.0, eta=eta, h_min=1e-6, h_max=20.0,
                          precision=precision)
    return Workload("polytrope", x, y, z, zeros.copy(), zeros.copy(), zeros.copy(), np.full(n, m),
                    h, K * rho, params, info=dict(K=K))


def collision(n_per_star: int = 1 << 21, seed: int = 4001, separation: float = 3.0,
              closing_speed: float = 1.0, precision: str = "mixed") -> Workload:
    """Two polytropes (different seeds) centred at (+-separation/2, 0, 0)
    moving towards each other with the given closing speed."""
    a = polytrope(n_per_star, seed, precision)
    b = polytrope(n_per_star, seed + 100, precision)
    s = 0.5 * separation
    v = 0.5 * closing_speed
    cat = np.concatenate
    n = 2 * n_per_star
    x = cat([a.x - s, b.x + s])
    vx = cat([np.full(n_per_star, v), np.full(n_per_star, -v)])
    m = np.full(n, 1.0 / n_per_star)
    params = dict(a.params)
    return Workload("collision", x, cat([a.y, b.y]), cat([a.z, b.z]), vx, np.zeros(n), np.zeros(n),
                    m, cat([a.h, b.h]), cat([a.u, b.u]), params, steps=100)


def turbulence(n_side: int = 256, seed: int = 5001, mach: float = 2.0, gamma: float = 1.01,
               n_max: int = 8, precision: str = "mixed") -> Workload:
    """Periodic jittered lattice with a Gaussian random solenoidal velocity
    field, |v(k)|^2 ~ k^-4 for integer wave vectors 1 <= |n| <= n_max,
    sampled at the unjittered sites and scaled to rms Mach number ``mach``
    (c_s = 1: u = 1/(gamma (gamma - 1))).  Wendland C4, ~100 neighbours."""
    x, y, z = jittered_lattice(n_side, seed, 0.1)
    n = x.size
    f = np.fft.fftfreq(n_side, d=1.0 / n_side)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    sel = (k2 >= 1.0) & (k2 <= n_max * n_max)
    idx = np.nonzero(sel)
    nm = idx[0].size
    amp = (2.0 * math.pi * np.sqrt(k2[idx])) ** -2.0
    comps = []
    for c in range(3):
        g = uniform(seed + 10 + c, 2 * nm).reshape(nm, 2)
        # Box-Muller from two uniforms
        rr = np.sqrt(-2.0 * np.log(np.maximum(g[:, 0], 1e-300)))
        comps.append(amp * rr * np.exp(2j * math.pi * g[:, 1]))
    vk = np.stack(comps)
    kv = np.stack([kx[idx], ky[idx], kz[idx]])
    vk = vk - kv * (np.sum(kv * vk, axis=0) / k2[idx])          # solenoidal projection
    vel = []
    for c in range(3):
        spec = np.zeros((n_side,) * 3, dtype=np.complex64)
        spec[idx] = vk[c].astype(np.complex64)
        vel.append(np.real(np.fft.ifftn(spec)).astype(np.float64).ravel())
        del spec
    vx, vy, vz = vel
    rms = math.sqrt(float(np.mean(vx * vx + vy * vy + vz * vz)))
    scale = mach / rms
    u0 = 1.0 / (gamma * (gamma - 1.0))
    eta = (300.0 / (32.0 * math.pi)) ** (1.0 / 3.0)
    m = 1.0 / n
    # a thin list skin: h moves by well under 2 % within a step's iteration
    # here (measured: one list build per step), and every list slot costs
    params = _base_params(kernel=WC4, gamma=gamma, eta=eta, precision=precision, skin=0.02)
    return Workload("turbulence", x, y, z, vx * scale, vy * scale, vz * scale, np.full(n, m),
                    np.full(n, eta / n_side), np.full(n, u0), params)


SOD_LEFT = (1.0, 0.0, 1.0)        # (rho, v, P) for 0 < x <= 0.5 (Sec. 3, Sod shock tube)
SOD_RIGHT = (0.125, 0.0, 0.1)     # (rho, v, P) for 0.5 < x < 1


def sod(n_tube: int = 10000, gamma: float = 1.4, kernel: int = M4, eta: float = 1.2,
        precision: str = "fp64") -> Workload:
    """One-dimensional Sod shock tube: the states of SOD_LEFT on x <= 0.5 and
    SOD_RIGHT beyond, equal-mass particles evenly spaced in each state, at
    rest, P = (gamma - 1) rho u.  The tube [0, 1) sits in a periodic box of
    length 2 with its mirror image on [1, 2) (the left state again on
    [1.5, 2)), so the box holds two Riemann problems, at x = 0.5 and at
    x = 1.5, whose waves do not reach each other before t = 0.28.  n_tube is
    the number of particles in [0, 1) (rounded so that the spacings are 1/8
    of each other); the box holds twice as many.  Every particle has
    y = z = 0 and the evaluation is one-dimensional (params dim = 1)."""
    rl, _, pl = SOD_LEFT
    rr, _, pr = SOD_RIGHT
    ratio = rl / rr                                  # 8: left spacing is 1/8 of the right one
    n_r = max(1, int(round(n_tube / (ratio + 1.0))))
    n_l = int(round(ratio * n_r))
    dl, dr = 0.5 / n_l, 0.5 / n_r
    xl = (np.arange(n_l) + 0.5) * dl                  # [0, 0.5)
    xr = 0.5 + (np.arange(2 * n_r) + 0.5) * dr        # [0.5, 1.5)
    xl2 = 1.5 + (np.arange(n_l) + 0.5) * dl           # [1.5, 2)
    x = np.concatenate([xl, xr, xl2])
    n = x.size
    m = rl * dl                                       # = rr * dr
    left = (x < 0.5) | (x >= 1.5)
    rho = np.where(left, rl, rr)
    u = np.where(left, pl, pr) / ((gamma - 1.0) * rho)
    h = eta * m / rho
    zeros = np.zeros(n)
    params = _base_params(kernel=kernel, gamma=gamma, eta=eta, fixed_h=False, h_tol=1e-6,
                          box_lo=(0.0, 0.0, 0.0), box_hi=(2.0, 2.0, 2.0), dim=1, precision=precision)
    return Workload("sod", x, zeros.copy(), zeros.copy(), zeros.copy(), zeros.copy(), zeros.copy(),
                    np.full(n, m), h, u, params, info=dict(n_left=n_l, n_right=n_r, n_tube=n_l + n_r))


def by_name(name: str, **kw) -> Workload:
    return {"lattice": lattice, "sedov": sedov, "polytrope": polytrope, "collision": collision,
            "turbulence": turbulence, "sod": sod}[name](**kw)

"""Seeded synthetic initial data for the paper's workloads.

This module holds no arithmetic of the method: it only builds initial conserved
states U(x, 0) (fields first, [p, ny, nx] or [p, nx], float64) and the seeded
request traces of the batched / served forms.  Both the CUDA path and the FP64
oracle are fed from here, so neither depends on the other.

Workloads (paper section in brackets):
  dam_break_1d        shallow-water dam break, h = 2 | 1, g = 9.81 on [0, 1]
                      (variant of the Sec. 5.1 / Table 1 dam-break problems)
  swe_riemann_1d      Table 1 rows (standard dam break, hydraulic, compression)
  swe_smooth_hump_1d  Eq. (53), characteristic-BC check (Sec. 5.1)
  euler_riemann_1d    Table 2 rows (Sod, Leblanc, sonic)
  entropy_wave_2d     Eq. (55) with exact solution Eq. (56)
  isentropic_vortex   Eq. (57), vortex strength eps, centre (xc, yc)
  orszag_tang         Orszag-Tang data (Eq. 60) in the [0, 2 pi]^2 normalisation
                      rho = gamma^2, p = gamma, v = (-sin y, sin x, 0),
                      B = (-sin y, sin 2x, 0), psi = 0
  swe_humps_batch     seeded Gaussian height humps on depth 1, sides 64..1024
  serving_trace       seeded Poisson arrivals of mixed SWE / Euler / MHD jobs
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def cell_centers(n, lo, hi):
    dx = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * dx


# ------------------------------------------------------------------------ 1D
def dam_break_1d(n=400, g=9.81, hl=2.0, hr=1.0, x0=0.5, lo=0.0, hi=1.0):
    x = cell_centers(n, lo, hi)
    h = np.where(x < x0, hl, hr).astype(np.float64)
    return np.stack([h, np.zeros_like(h)])


SWE_RIEMANN_TABLE1 = {
    # name: (domain, T, x0, (hl, hr), (hul, hur), g)
    "standard": ((-5.0, 5.0), 2.0, 0.0, (3.0, 1.0), (0.0, 0.0), 1.0),
    "hydraulic": ((-20.0, 20.0), 4.0, 0.0, (10.0, 1.0), (0.0, 0.0), 1.0),
    "compression": ((-2.0, 2.0), 0.5, 0.0, (1.0, 1.0), (1.0, -1.0), 1.0),
}


def swe_riemann_1d(name, n):
    (lo, hi), T, x0, (hl, hr), (ql, qr), g = SWE_RIEMANN_TABLE1[name]
    x = cell_centers(n, lo, hi)
    h = np.where(x < x0, hl, hr)
    q = np.where(x < x0, ql, qr)
    return np.stack([h, q]).astype(np.float64), dict(lo=lo, hi=hi, T=T, g=g, x0=x0)


def swe_smooth_hump_1d(n=512, lo=-5.0, hi=5.0):
    """Eq. (53): h = 1 + 0.3 ((1 - cos(pi (x + 1))) / 2)^2 on [-1, 1], else 1."""
    x = cell_centers(n, lo, hi)
    inside = np.abs(x) <= 1.0
    h = np.where(inside, 1.0 + 0.3 * ((1.0 - np.cos(np.pi * (x + 1.0))) / 2.0) ** 2, 1.0)
    return np.stack([h, np.zeros_like(h)])


EULER_RIEMANN_TABLE2 = {
    # name: (domain, T, x0, (rho l, r), (u l, r), (p l, r), gamma)
    "sod": ((-0.5, 0.5), 0.2, 0.0, (1.0, 0.125), (0.0, 0.0), (1.0, 0.1), 1.4),
    "leblanc": ((0.0, 9.0), 6.0, 3.0, (1.0, 1e-3), (0.0, 0.0), (6.667e-2, 6.667e-9), 5.0 / 3.0),
    "sonic": ((-1.0, 1.0), 0.5, -0.4, (1.0, 0.125), (0.75, 0.75), (1.0, 0.1), 1.4),
}


def euler_riemann_1d(name, n):
    (lo, hi), T, x0, rr, uu, pp, gamma = EULER_RIEMANN_TABLE2[name]
    x = cell_centers(n, lo, hi)
    left = x < x0
    rho = np.where(left, rr[0], rr[1])
    u = np.where(left, uu[0], uu[1])
    p = np.where(left, pp[0], pp[1])
    E = p / (gamma - 1.0) + 0.5 * rho * u * u
    return np.stack([rho, rho * u, E]).astype(np.float64), dict(lo=lo, hi=hi, T=T, gamma=gamma, x0=x0)


# ------------------------------------------------------------------------ 2D
def _grid(n, lo, hi):
    x = cell_centers(n, lo, hi)
    X, Y = np.meshgrid(x, x, indexing="xy")  # [ny, nx], x fastest
    return X, Y


def euler_conserved(rho, u, v, p, gamma):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E]).astype(np.float64)


def entropy_wave_2d(n, gamma=1.4, phase=0.0, lo=0.0, hi=1.0):
    """Eq. (55): rho = 1 + 0.1 sin(2 pi (x + y) + phase), u = v = p = 1."""
    X, Y = _grid(n, lo, hi)
    rho = 1.0 + 0.1 * np.sin(2.0 * np.pi * (X + Y) + phase)
    one = np.ones_like(rho)
    return euler_conserved(rho, one, one, one, gamma)


def entropy_wave_exact(n, t, gamma=1.4, phase=0.0, lo=0.0, hi=1.0):
    """Eq. (56): the density wave translates with (u, v) = (1, 1)."""
    X, Y = _grid(n, lo, hi)
    rho = 1.0 + 0.1 * np.sin(2.0 * np.pi * (X + Y - 2.0 * t) + phase)
    one = np.ones_like(rho)
    return euler_conserved(rho, one, one, one, gamma)


def isentropic_vortex(n, gamma=1.4, eps=5.0, lo=0.0, hi=10.0, center=(5.0, 5.0), shift=(0.0, 0.0)):
    """Eq. (57): T = 1 - (gamma-1) eps^2 / (8 gamma pi^2) e^{1 - r^2},
    rho = T^{1/(gamma-1)}, u = 1 - eps/(2 pi) e^{(1-r^2)/2} (y - yc),
    v = 1 + eps/(2 pi) e^{(1-r^2)/2} (x - xc), p = rho^gamma.
    ``shift`` translates the centre periodically (exact solution at time t is
    shift = (t, t))."""
    X, Y = _grid(n, lo, hi)
    L = hi - lo
    xc = center[0] + shift[0]
    yc = center[1] + shift[1]
    dxp = (X - xc + 0.5 * L) % L - 0.5 * L
    dyp = (Y - yc + 0.5 * L) % L - 0.5 * L
    r2 = dxp * dxp + dyp * dyp
    T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    e = eps / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = 1.0 - e * dyp
    v = 1.0 + e * dxp
    p = rho ** gamma
    return euler_conserved(rho, u, v, p, gamma)


def mhd_conserved(rho, u, v, w, p, bx, by, bz, psi, gamma):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w) + 0.5 * (bx * bx + by * by + bz * bz)
    return np.stack([rho, rho * u, rho * v, rho * w, E, bx, by, bz, psi]).astype(np.float64)


def orszag_tang(n, gamma=5.0 / 3.0, phase=(0.0, 0.0)):
    """Orszag-Tang on [0, 2 pi]^2: rho = gamma^2, p = gamma, v = (-sin y, sin x, 0),
    B = (-sin y, sin 2x, 0), psi = 0; ``phase`` shifts (x, y)."""
    X, Y = _grid(n, 0.0, 2.0 * np.pi)
    X = X + phase[0]
    Y = Y + phase[1]
    z = np.zeros_like(X)
    rho = np.full_like(X, gamma * gamma)
    p = np.full_like(X, gamma)
    return mhd_conserved(rho, -np.sin(Y), np.sin(X), z, p, -np.sin(Y), np.sin(2.0 * X), z, z, gamma)


def swe_sine_2d(n, g=9.81, phase=(0.0, 0.0)):
    """h = 1 + 0.1 sin(2 pi x + p1) + 0.1 sin(2 pi y + p2), zero velocity, [0,1]^2."""
    X, Y = _grid(n, 0.0, 1.0)
    h = 1.0 + 0.1 * np.sin(2.0 * np.pi * X + phase[0]) + 0.1 * np.sin(2.0 * np.pi * Y + phase[1])
    z = np.zeros_like(h)
    return np.stack([h, z, z]).astype(np.float64)


def swe_hump_2d(n, amp, x0, y0, sigma):
    """h = 1 + amp exp(-|x - x0|^2 / (2 sigma^2)) on [0,1]^2, hu = hv = 0."""
    X, Y = _grid(n, 0.0, 1.0)
    h = 1.0 + amp * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2.0 * sigma * sigma))
    z = np.zeros_like(h)
    return np.stack([h, z, z]).astype(np.float64)


@dataclass
class HumpSpec:
    n: int
    amp: float
    x0: float
    y0: float
    sigma: float


def swe_humps_batch(count=256, seed=0, nmin=64, nmax=1024):
    """Seeded batch of uneven SWE instances: side ~ U{nmin..nmax},
    amplitude ~ U[0.1, 1], centre ~ U[0.25, 0.75]^2, sigma ~ U[0.05, 0.1]."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        specs.append(HumpSpec(n=n, amp=float(rng.uniform(0.1, 1.0)),
                              x0=float(rng.uniform(0.25, 0.75)), y0=float(rng.uniform(0.25, 0.75)),
                              sigma=float(rng.uniform(0.05, 0.1))))
    return specs


@dataclass
class Request:
    rid: int
    arrival: float
    system: str       # "swe" | "euler" | "mhd_glm"
    n: int
    steps: int
    phase: tuple


def serving_trace(count=2000, rate=200.0, seed=0, nmin=128, nmax=2048, nstep=64,
                  smin=100, smax=2000):
    """Seeded Poisson arrivals (mean ``rate`` per second) of mixed jobs; side in
    steps of ``nstep`` between nmin and nmax, step counts uniform."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    sides = np.arange(nmin, nmax + 1, nstep)
    systems = ("swe", "euler", "mhd_glm")
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        out.append(Request(rid=i, arrival=t, system=systems[int(rng.integers(0, 3))],
                           n=int(rng.choice(sides)), steps=int(rng.integers(smin, smax + 1)),
                           phase=(float(rng.uniform(0, 2 * math.pi)), float(rng.uniform(0, 2 * math.pi)))))
    return out


def request_initial_state(req, gamma_euler=1.4, gamma_mhd=5.0 / 3.0):
    if req.system == "swe":
        return swe_sine_2d(req.n, phase=req.phase)
    if req.system == "euler":
        return entropy_wave_2d(req.n, gamma=gamma_euler, phase=req.phase[0])
    return orszag_tang(req.n, gamma=gamma_mhd, phase=req.phase)


def request_initial_state_torch(req, torch, device="cuda", gamma_euler=1.4, gamma_mhd=5.0 / 3.0):
    """request_initial_state evaluated by torch in float64 on ``device``: the
    server builds a request's analytic initial data (system, side, phases) where
    the state will live instead of copying it from the host."""
    n = req.n
    L = 2.0 * math.pi if req.system == "mhd_glm" else 1.0
    x = (torch.arange(n, dtype=torch.float64, device=device) + 0.5) * (L / n)
    Y, X = torch.meshgrid(x, x, indexing="ij")          # [ny, nx], x fastest
    two_pi = 2.0 * math.pi
    if req.system == "swe":
        h = 1.0 + 0.1 * torch.sin(two_pi * X + req.phase[0]) + 0.1 * torch.sin(two_pi * Y + req.phase[1])
        z = torch.zeros_like(h)
        return torch.stack([h, z, z]).contiguous()
    if req.system == "euler":
        g = gamma_euler
        rho = 1.0 + 0.1 * torch.sin(two_pi * (X + Y) + req.phase[0])
        E = 1.0 / (g - 1.0) + 0.5 * rho * 2.0
        return torch.stack([rho, rho, rho, E]).contiguous()
    g = gamma_mhd
    Xs, Ys = X + req.phase[0], Y + req.phase[1]
    rho = torch.full_like(X, g * g)
    u, v = -torch.sin(Ys), torch.sin(Xs)
    bx, by = -torch.sin(Ys), torch.sin(2.0 * Xs)
    z = torch.zeros_like(X)
    E = g / (g - 1.0) + 0.5 * rho * (u * u + v * v) + 0.5 * (bx * bx + by * by)
    return torch.stack([rho, rho * u, rho * v, z, E, bx, by, z, z]).contiguous()


def random_states(system, count, seed=0, dim=2, gamma=1.4, g=9.81):
    """Seeded random admissible states (positive depth / density / pressure),
    shape [p, count], for point-wise checks of fluxes and splittings."""
    rng = np.random.default_rng(seed)
    if system == "swe":
        h = rng.uniform(0.2, 3.0, count)
        vel = [rng.uniform(-3.0, 3.0, count) for _ in range(dim)]
        return np.stack([h] + [h * v for v in vel])
    if system == "euler":
        rho = rng.uniform(0.2, 3.0, count)
        p = rng.uniform(0.2, 3.0, count)
        vel = [rng.uniform(-2.5, 2.5, count) for _ in range(dim)]
        E = p / (gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel)
        return np.stack([rho] + [rho * v for v in vel] + [E])
    if system == "mhd_glm":
        rho = rng.uniform(0.3, 3.0, count)
        p = rng.uniform(0.2, 3.0, count)
        u, v, w = (rng.uniform(-2.0, 2.0, count) for _ in range(3))
        bx, by, bz = (rng.uniform(-1.5, 1.5, count) for _ in range(3))
        psi = rng.uniform(-0.2, 0.2, count)
        return mhd_conserved(rho, u, v, w, p, bx, by, bz, psi, gamma)
    if system == "advection":
        return rng.uniform(-1.0, 1.0, (1, count))
    raise ValueError(system)

"""Parity at the benchmark's full size and launch shape: the 1024^2 Euler
isentropic vortex (omega 2, CFL 0.3, c 0.05, k 2) in the launch shape bench.py
times (the autotuned tile and kernel variant), in FP32 and FP64; and the 2048^2
MHD-GLM Orszag-Tang vortex (omega 1, CFL 0.3, c_h factor 6) the same way.

The oracle cannot step 10^6 cells in seconds, but one step of the update at a
cell depends only on its 5-point neighbourhood and on the global lattice speed
xi_0 = max|lambda(U_0)| / nu (Eq. 29).  So xi_0 is taken from the oracle's
global maximum over the full grid, and each sampled cell is checked against an
oracle run on the 5 x 5 periodic patch around it with xi fixed at xi_0: its
centre after one step is exactly the full-grid result (pinned on the CPU by
test_one_step_is_local_given_global_xi).  The samples include the edges of
128-, 256- and 32-cell bricks and tiles, and of the periodic grid, where the
kernel's recomputed ring cells and index wrap act.  A property that holds at any size (Thm 4.3's
conservation on a periodic grid) is checked on the whole grid.
"""
import os
import sys

import numpy as np
import pytest

from oracle import systems, vklb as ovklb
from paper_2608_04283_b300 import inputs
from parity_util import max_rel, max_rel_mhd

pytestmark = pytest.mark.gpu

N = 1024
L = 10.0
GAMMA = 1.4
KW = dict(omega=2.0, cfl=0.3, c=0.05, k=2.0, gamma=GAMMA)


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


@pytest.fixture(scope="module")
def U0():
    return np.ascontiguousarray(inputs.isentropic_vortex(N))


def _bench():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    return bench


def _samples():
    rng = np.random.default_rng(20)
    edges = [0, 1, 31, 32, 127, 128, 129, 255, 256, 511, 512, N - 2, N - 1]
    rows = [0, 1, 7, 8, 9, 15, 16, 511, 512, N - 8, N - 1]
    pts = [(x, y) for x in edges[::2] for y in rows[::2]]
    pts += [(int(x), int(y)) for x, y in rng.integers(0, N, size=(24, 2))]
    pts += [(N // 2 + d, N // 2) for d in (-3, 0, 3)]     # through the vortex core
    return pts


def _oracle_at(U0, pts, xi0, lam0):
    """5 x 5 periodic patches with the full grid's xi_0 (fixed dt) and the full
    grid's max |lambda|, alpha's normaliser under the global reading."""
    dx = L / N
    sysm = systems.Euler(GAMMA, 2)
    out = np.empty((U0.shape[0], len(pts)))
    for i, (x, y) in enumerate(pts):
        xs = np.arange(x - 2, x + 3) % N
        ys = np.arange(y - 2, y + 3) % N
        patch = U0[:, ys][:, :, xs]
        ref = ovklb.Sim(sysm, (5, 5), (0.0, 0.0), (5 * dx, 5 * dx), omega=KW["omega"], nu=KW["cfl"], c=KW["c"],
                        k=KW["k"], dt=dx / xi0)
        ref.max_lambda = lambda U: lam0
        ref.set_state(patch)
        ref.step()
        out[:, i] = ref.moments()[:, 2, 2]
    return out


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-11)])
def test_fullsize_one_step_sampled(vk, U0, precision, tol):
    bench = _bench()
    shape = bench.launch_shape("euler", "fp32", (N, N))
    sim = vk.Sim("euler", (N, N), (0.0, 0.0), (L, L), precision=precision, **KW)
    bench.configure(sim, shape)
    sim.set_state(U0)
    sim.step(1)
    got = sim.moments()
    t, nsteps, _ = sim.time()
    sim.close()

    full = ovklb.Sim(systems.Euler(GAMMA, 2), (N, N), (0.0, 0.0), (L, L), omega=KW["omega"], nu=KW["cfl"])
    lam0 = full.max_lambda(U0)
    xi0 = lam0 / KW["cfl"]                                  # Eq. (29) over the full grid
    dx = L / N
    assert nsteps == 1
    assert abs(t - dx / xi0) <= (1e-6 if precision == "fp32" else 1e-13) * (dx / xi0)

    pts = _samples()
    want = _oracle_at(U0, pts, xi0, lam0)
    have = np.stack([got[:, y, x] for x, y in pts], axis=1)
    err = max_rel(have, want)
    assert err.max() <= tol, err


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-6), ("fp64", 1e-13)])
def test_fullsize_conservation(vk, U0, precision, tol):
    """Thm 4.3: on the periodic grid the totals of rho, m and E do not change;
    20 steps at the bench's launch shape, FP64 totals of the stored f."""
    sim = vk.Sim("euler", (N, N), (0.0, 0.0), (L, L), precision=precision, **KW)
    bench = _bench()
    bench.configure(sim, bench.launch_shape("euler", "fp32", (N, N)))
    sim.set_state(U0)
    t0 = sim.totals()
    sim.step(20)
    t1 = sim.totals()
    sim.close()
    scale = np.abs(t0).max()
    assert np.abs(t1 - t0).max() <= tol * scale, (t0, t1)


MN = 2048
ML = 2 * np.pi
MKW = dict(omega=1.0, cfl=0.3, c=0.05, k=2.0, gamma=5.0 / 3.0, ch_factor=6.0)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-11)])
def test_fullsize_mhd_one_step_sampled(vk, precision, tol):
    """As the Euler case, with c_h (reading R4: ch_factor x the largest fast
    speed of the full grid) also taken from the full grid for every patch.
    FP32: psi, B_z and m_z are zero or at rounding level, so they are measured
    against the terms that carry them (c_h |B|, |B|, |m|; max_rel_mhd), as in the
    whole-grid MHD-GLM parity tests."""
    bench = _bench()
    U0 = np.ascontiguousarray(inputs.orszag_tang(MN))
    shape = bench.launch_shape("mhd_glm", "fp32", (MN, MN))
    sim = vk.Sim("mhd_glm", (MN, MN), (0.0, 0.0), (ML, ML), precision=precision, **MKW)
    bench.configure(sim, shape)
    tx, ty = sim.info.tile_x, sim.info.tile_y
    sim.set_state(U0)
    sim.step(1)
    got = sim.moments()
    t, nsteps, _ = sim.time()
    sim.close()

    sysm = systems.MHDGLM(MKW["gamma"])
    full = ovklb.Sim(sysm, (MN, MN), (0.0, 0.0), (ML, ML), omega=1.0, nu=MKW["cfl"], ch_factor=MKW["ch_factor"])
    full.refresh_ch(U0)
    ch = full.sys.ch
    lam0 = full.max_lambda(U0)
    xi0 = lam0 / MKW["cfl"]
    dx = ML / MN
    assert nsteps == 1
    assert abs(t - dx / xi0) <= (1e-6 if precision == "fp32" else 1e-13) * (dx / xi0)

    rng = np.random.default_rng(21)
    xs = sorted({0, 1, tx - 1, tx, tx + 1, 2 * tx - 1, MN // 2, MN - 2, MN - 1})
    ys = sorted({0, 1, ty - 1, ty, ty + 1, 2 * ty - 1, 2 * ty, MN // 2, MN - 2, MN - 1})
    pts = [(x, y) for x in xs[::2] for y in ys[::2]]
    pts += [(int(x), int(y)) for x, y in rng.integers(0, MN, size=(16, 2))]
    want = np.empty((9, len(pts)))
    for i, (x, y) in enumerate(pts):
        patch = U0[:, np.arange(y - 2, y + 3) % MN][:, :, np.arange(x - 2, x + 3) % MN]
        ref = ovklb.Sim(systems.MHDGLM(MKW["gamma"]), (5, 5), (0.0, 0.0), (5 * dx, 5 * dx), omega=1.0,
                        nu=MKW["cfl"], c=MKW["c"], k=MKW["k"], dt=dx / xi0, ch_factor=MKW["ch_factor"])
        ref.refresh_ch = lambda U, r=ref: setattr(r.sys, "ch", ch)      # the full grid's c_h
        ref.max_lambda = lambda U: lam0                                  # and max |lambda|
        ref.set_state(patch)
        ref.step()
        want[:, i] = ref.moments()[:, 2, 2]
    have = np.stack([got[:, y, x] for x, y in pts], axis=1)
    err = max_rel_mhd(have, want, ch)
    assert err.max() <= tol, err

"""The paper's 1D verification suite on the GPU (Secs. 5.1, 5.2): the shallow-water
Riemann problems of Table 1 and the Euler problems of Table 2 with
characteristic boundaries (the paper's transmissive ones, reading R12; the
parity tests also run the zero-order extrapolation of reading R21), omega = 1,
c = 0.05, k = 2, and the smooth hump of Eq. (53).

* Parity with the FP64 oracle at the paper's CFL number 0.9 over 30 steps (the
  weighted set at rest is ill-conditioned at CFL 0.9 over long runs: its
  momentum diffusion at rest passes 1/2 above a local CFL number of about 0.67)
  and to the final time at CFL 0.6.
* Convergence against the exact Riemann solutions (oracle/riemann.py) at CFL 0.6
  for N = 256 .. 16384, sizes the oracle cannot reach: the L1 error falls at
  every refinement and its order at the finest pair is that of a first-order
  scheme on discontinuous data (slightly below one, Sec. 5.1)."""
import numpy as np
import pytest

from oracle import riemann, systems, vklb as ovklb
from paper_2608_04283_b300 import inputs
from parity_util import max_rel

pytestmark = pytest.mark.gpu

KW = dict(bc="characteristic", c=0.05, k=2.0, omega=1.0)


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


def _problem(table, name, n):
    if table == 1:
        U0, meta = inputs.swe_riemann_1d(name, n)
        return "swe", U0, meta, dict(g=meta["g"]), systems.ShallowWater(meta["g"], 1)
    U0, meta = inputs.euler_riemann_1d(name, n)
    return "euler", U0, meta, dict(gamma=meta["gamma"]), systems.Euler(meta["gamma"], 1)


def _exact(table, name, x, T):
    if table == 1:
        (lo, hi), _, x0, h, q, g = inputs.SWE_RIEMANN_TABLE1[name]
        return riemann.swe_sample(h[0], q[0] / h[0], h[1], q[1] / h[1], g, x, T, x0=x0)[0]
    (lo, hi), _, x0, r, u, p, gam = inputs.EULER_RIEMANN_TABLE2[name]
    return riemann.euler_sample(r[0], u[0], p[0], r[1], u[1], p[1], gam, x, T, x0=x0)[0]


PROBLEMS = [(1, "standard"), (1, "hydraulic"), (1, "compression"), (2, "sod"), (2, "sonic"), (2, "leblanc")]


@pytest.mark.parametrize("bc", ["characteristic", "transmissive"])
@pytest.mark.parametrize("table,name", PROBLEMS)
def test_tables_parity_paper_cfl(vk, table, name, bc):
    n = 128
    system, U0, meta, skw, sysm = _problem(table, name, n)
    kw = dict(KW, bc=bc)
    sim = vk.Sim(system, (n,), (meta["lo"],), (meta["hi"],), precision="fp64", cfl=0.9, **kw, **skw)
    sim.set_state(U0)
    sim.step(30)
    ref = ovklb.Sim(sysm, (n,), (meta["lo"],), (meta["hi"],), bc=bc, c=0.05, k=2.0, omega=1.0, nu=0.9)
    ref.set_state(U0)
    ref.run(30)
    assert max_rel(sim.moments(), ref.moments()).max() <= 1e-11
    t, nsteps, xi = sim.time()
    assert nsteps == 30 and abs(t - ref.t) <= 1e-12 * ref.t
    sim.close()


@pytest.mark.parametrize("bc", ["characteristic", "transmissive"])
@pytest.mark.parametrize("table,name", [(1, "standard"), (1, "compression"), (2, "sod")])
def test_tables_parity_to_final_time(vk, table, name, bc):
    n = 160
    system, U0, meta, skw, sysm = _problem(table, name, n)
    kw = dict(KW, bc=bc)
    sim = vk.Sim(system, (n,), (meta["lo"],), (meta["hi"],), precision="fp64", cfl=0.6, **kw, **skw)
    sim.set_state(U0)
    sim.step_to(meta["T"])
    ref = ovklb.Sim(sysm, (n,), (meta["lo"],), (meta["hi"],), bc=bc, c=0.05, k=2.0, omega=1.0, nu=0.6)
    ref.set_state(U0)
    ref.run_to(meta["T"])
    assert max_rel(sim.moments(), ref.moments()).max() <= 1e-10
    t, nsteps, _ = sim.time()
    assert nsteps == ref.steps and t == pytest.approx(meta["T"], abs=1e-13)
    sim.close()


@pytest.mark.parametrize("table,name", [(1, "standard"), (1, "hydraulic"), (1, "compression"), (2, "sod"),
                                        (2, "sonic")])
def test_tables_converge_to_exact(vk, table, name):
    errs = []
    for n in (256, 1024, 4096, 16384):
        system, U0, meta, skw, _ = _problem(table, name, n)
        sim = vk.Sim(system, (n,), (meta["lo"],), (meta["hi"],), precision="fp64", cfl=0.6, **KW, **skw)
        sim.set_state(U0)
        sim.step_to(meta["T"])
        dx = (meta["hi"] - meta["lo"]) / n
        x = meta["lo"] + (np.arange(n) + 0.5) * dx
        errs.append(float(np.sum(np.abs(sim.moments()[0] - _exact(table, name, x, meta["T"]))) * dx))
        sim.close()
    errs = np.array(errs)
    rates = np.log(errs[:-1] / errs[1:]) / np.log(4.0)
    assert np.all(rates > 0.3), (errs, rates)
    assert 0.5 < rates[-1] < 1.1, (errs, rates)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_smooth_hump_characteristic_bc(vk, precision, tol):
    """Eq. (53): the smooth hump leaves the domain through the characteristic
    boundaries (Eqs. 33-36).  CFL 0.6: at 0.9 the fluid at rest around the hump
    sits at a local CFL number near 0.8, where the weighted set amplifies
    rounding (at rest its momentum diffusion passes 1/2 above a local CFL
    number of about 0.67)."""
    n = 200
    U0 = inputs.swe_smooth_hump_1d(n)
    sim = vk.Sim("swe", (n,), (-5.0,), (5.0,), precision=precision, cfl=0.6, g=1.0, **KW)
    sim.set_state(U0)
    sim.step(60)
    ref = ovklb.Sim(systems.ShallowWater(1.0, 1), (n,), (-5.0,), (5.0,), bc="characteristic", c=0.05, k=2.0,
                    omega=1.0, nu=0.6)
    ref.set_state(U0)
    ref.run(60)
    got, want = sim.moments(), ref.moments()
    err = max_rel(got, want) if precision == "fp64" else np.abs(got - want).sum(axis=1) / np.abs(want).sum(axis=1).max()
    assert err.max() <= tol, err
    sim.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_smooth_hump_centered_subcharacteristic(vk, precision, tol):
    """The paper's first 1D check (Sec. 5.1, Eq. 53): the centered set (c = 1/3,
    F+- = F/2) with the characteristic boundaries, lattice speed from the
    subcharacteristic rule at eta = 0.9 (Sec. 2.3), omega = 1, to T = 8, when the
    hump has left the domain; N = 512."""
    n, T = 512, 8.0
    U0 = inputs.swe_smooth_hump_1d(n)
    sim = vk.Sim("swe", (n,), (-5.0,), (5.0,), precision=precision, g=1.0, bc="characteristic",
                 set_kind="centered", omega=1.0, eta=0.9)
    sim.set_state(U0)
    sim.step_to(T)
    ref = ovklb.Sim(systems.ShallowWater(1.0, 1), (n,), (-5.0,), (5.0,), bc="characteristic",
                    set_kind="centered", omega=1.0, eta=0.9)
    ref.set_state(U0)
    ref.run_to(T)
    got, want = sim.moments(), ref.moments()
    err = max_rel(got, want) if precision == "fp64" else np.abs(got - want).sum(axis=1) / np.abs(want).sum(axis=1).max()
    assert err.max() <= tol, err
    t, nsteps, _ = sim.time()
    assert nsteps == ref.steps and t == pytest.approx(T, abs=1e-12 if precision == "fp64" else 1e-5)
    sim.close()

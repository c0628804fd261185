"""GPU parity under the global reading of alpha's normaliser (Eq. 27 with the
grid-wide max |lambda| of the step, vklb_weight.alpha_norm = VKLB_ALPHA_GLOBAL)
against the FP64 oracle run with alpha_norm="global": FP64 <= 1e-11 max relative
per field, FP32 <= 1e-5 relative L1, in the 2D step kernels (plain and
bulk-copy variants, several tilings), the moment form, the batched form and the
1D step with characteristic boundaries."""
import numpy as np
import pytest

from oracle import systems, vklb as ovklb
from paper_2608_04283_b300 import inputs
from parity_util import max_rel, rel_l1, rel_l1_mhd

pytestmark = pytest.mark.gpu

G = "global"


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


def _vortex(nx, ny):
    return np.ascontiguousarray(inputs.isentropic_vortex(nx, lo=0.0, hi=10.0)[:, :ny, :])


def _oracle(sysm, n, lo, hi, U0, steps, **kw):
    ref = ovklb.Sim(sysm, n, lo, hi, alpha_norm=G, **kw)
    ref.set_state(U0)
    if isinstance(steps, float):
        ref.run_to(steps)
    else:
        ref.run(steps)
    return ref


@pytest.mark.parametrize("variant,tile", [((0, 0), None), ((0, 0), (32, 8)), ((1, 4), (64, 4)), ((1, 2), (32, 40))])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_euler_vortex(vk, variant, tile, precision):
    n = (48, 40)
    lo, hi = (0.0, 0.0), (10.0, 10.0 * 40 / 48)
    U0 = _vortex(*n)
    sim = vk.Sim("euler", n, lo, hi, precision=precision, omega=2.0, cfl=0.3, alpha_norm=G)
    if tile:
        sim.set_tiling(*tile)
    sim.set_variant(*variant)
    sim.set_state(U0)
    sim.step(30)
    ref = _oracle(systems.Euler(1.4, 2), n, lo, hi, U0, 30, omega=2.0, nu=0.3)
    got = sim.moments()
    if precision == "fp64":
        assert max_rel(got, ref.moments()).max() <= 1e-11
        t, steps, xi = sim.time()
        assert steps == 30 and abs(t - ref.t) <= 1e-12 * ref.t and abs(xi - ref.xi) <= 1e-11 * ref.xi
    else:
        assert rel_l1(got, ref.moments()).max() <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_swe_hump_to_time(vk, precision):
    n = (40, 36)
    U0 = np.ascontiguousarray(inputs.swe_hump_2d(40, 0.4, 0.5, 0.45, 0.08)[:, :36, :])
    lo, hi = (0.0, 0.0), (1.0, 36 / 40)
    sim = vk.Sim("swe", n, lo, hi, precision=precision, omega=1.0, cfl=0.3, alpha_norm=G)
    sim.set_state(U0)
    sim.step_to(0.02)
    ref = _oracle(systems.ShallowWater(9.81, 2), n, lo, hi, U0, 0.02, omega=1.0, nu=0.3)
    got = sim.moments()
    err = max_rel(got, ref.moments()) if precision == "fp64" else rel_l1(got, ref.moments())
    assert err.max() <= (1e-11 if precision == "fp64" else 1e-5), err
    assert sim.time()[1] == ref.steps


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mhd_orszag_tang(vk, precision):
    """c_h = 6 max c_f sits above every |u| + c_f, so the grid-wide maximum is
    c_h and the two readings agree here; the test pins that the global path
    through the MHD-GLM split normalises by it."""
    n = (36, 32)
    L = 2 * np.pi
    U0 = np.ascontiguousarray(inputs.orszag_tang(36)[:, :32, :])
    lo, hi = (0.0, 0.0), (L, L * 32 / 36)
    sim = vk.Sim("mhd_glm", n, lo, hi, precision=precision, omega=1.0, cfl=0.3, gamma=5 / 3, alpha_norm=G)
    sim.set_tiling(64, 8)
    sim.set_state(U0)
    sim.step(12)
    ref = _oracle(systems.MHDGLM(5 / 3), n, lo, hi, U0, 12, omega=1.0, nu=0.3)
    got = sim.moments()
    err = max_rel(got, ref.moments()) if precision == "fp64" else rel_l1_mhd(got, ref.moments())
    assert err.max() <= (1e-11 if precision == "fp64" else 1e-5), err


def test_moment_form(vk):
    """omega = 1 moment form (Thm 4.3) under the global reading."""
    n = (40, 36)
    U0 = np.ascontiguousarray(inputs.swe_hump_2d(40, 0.4, 0.5, 0.45, 0.08)[:, :36, :])
    lo, hi = (0.0, 0.0), (1.0, 36 / 40)
    sim = vk.Sim("swe", n, lo, hi, precision="fp64", omega=1.0, cfl=0.3, alpha_norm=G, form="moments")
    sim.set_state(U0)
    sim.step(25)
    ref = _oracle(systems.ShallowWater(9.81, 2), n, lo, hi, U0, 25, omega=1.0, nu=0.3)
    assert max_rel(sim.moments(), ref.moments()).max() <= 1e-11


def test_batched(vk):
    """A batch of uneven Euler grids under the global reading, each member with
    its own grid-wide maximum."""
    sizes = [(40, 40), (33, 33), (64, 64)]
    sims, refs = [], []
    for i, (nx, ny) in enumerate(sizes):
        U0 = np.ascontiguousarray(inputs.isentropic_vortex(nx, eps=3.0 + i)[:, :ny, :])
        s = vk.Sim("euler", (nx, ny), (0, 0), (10, 10 * ny / nx), precision="fp64", omega=2.0, cfl=0.3,
                   alpha_norm=G)
        s.set_state(U0)
        sims.append(s)
        refs.append(_oracle(systems.Euler(1.4, 2), (nx, ny), (0, 0), (10, 10 * ny / nx), U0, 12, omega=2.0,
                            nu=0.3))
    b = vk.Batch(sims)
    b.step(12)
    for s, r in zip(sims, refs):
        assert max_rel(s.moments(), r.moments()).max() <= 1e-11


@pytest.mark.parametrize("table,name", [(1, "standard"), (2, "sod")])
def test_1d_characteristic(vk, table, name):
    """1D step with characteristic boundaries: the boundary equilibria take the
    grid-wide maximum of U^{n+1} (Eq. 36 under the global reading)."""
    n = 96
    if table == 1:
        U0, meta = inputs.swe_riemann_1d(name, n)
        system, sysm, skw = "swe", systems.ShallowWater(meta["g"], 1), dict(g=meta["g"])
    else:
        U0, meta = inputs.euler_riemann_1d(name, n)
        system, sysm, skw = "euler", systems.Euler(meta["gamma"], 1), dict(gamma=meta["gamma"])
    sim = vk.Sim(system, (n,), (meta["lo"],), (meta["hi"],), precision="fp64", cfl=0.6, bc="characteristic",
                 omega=1.0, alpha_norm=G, **skw)
    sim.set_state(U0)
    sim.step_to(meta["T"])
    ref = _oracle(sysm, (n,), (meta["lo"],), (meta["hi"],), U0, float(meta["T"]), bc="characteristic",
                  omega=1.0, nu=0.6)
    assert max_rel(sim.moments(), ref.moments()).max() <= 1e-11
    assert sim.time()[1] == ref.steps


def test_alpha_norm_rejected(vk):
    with pytest.raises(KeyError):
        vk.Sim("euler", (32, 32), (0, 0), (1, 1), alpha_norm="per-direction")

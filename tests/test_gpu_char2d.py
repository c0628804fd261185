"""Non-periodic 2D faces on the GPU against the FP64 oracle: characteristic
(reading R19: the 1D construction of Eqs. 33-36 along each face's normal,
corners summing both faces) and transmissive (reading R21: the state of the
node one cell inwards); <= 1e-11 max relative per field in FP64, <= 1e-5
relative L1 in FP32, on ragged grids with all four faces open or one axis
periodic, several tilings; a uniform state is a fixed point; the smooth hump
leaves the box with small reflections at a size the oracle cannot reach;
MHD-GLM's nine-wave faces against the oracle in both precisions; and the
combinations not built are refused."""
import numpy as np
import pytest

from oracle import systems, vklb as ovklb
from paper_2608_04283_b300 import inputs
from parity_util import max_rel, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


def _hump(nx, ny, L):
    dx = 2 * L / nx
    x = -L + (np.arange(nx) + 0.5) * dx
    y = -L + (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y, indexing="xy")
    r = np.sqrt((X - 0.8) ** 2 + (Y + 0.4) ** 2)
    h = np.where(r <= 1.0, 1.0 + 0.3 * ((1.0 + np.cos(np.pi * r)) / 2.0) ** 2, 1.0)
    return np.stack([h, 0.2 * h, -0.1 * h])


@pytest.mark.parametrize("bc", ["characteristic", ("characteristic", "periodic"), ("periodic", "characteristic"),
                                "transmissive", ("transmissive", "periodic"), ("periodic", "transmissive")])
@pytest.mark.parametrize("tile", [(32, 8), (64, 5), None])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_swe_hump_against_oracle(vk, bc, tile, precision):
    nx, ny = 44, 36
    L = 3.0
    U0 = _hump(nx, ny, L)
    lo, hi = (-L, -L), (L, -L + ny * 2 * L / nx)
    sim = vk.Sim("swe", (nx, ny), lo, hi, precision=precision, g=1.0, omega=1.0, cfl=0.3, bc=bc)
    if tile:
        sim.set_tiling(*tile)
    sim.set_state(U0)
    sim.step(40)
    ref = ovklb.Sim(systems.ShallowWater(1.0, 2), (nx, ny), lo, hi, bc=bc, omega=1.0, nu=0.3)
    ref.set_state(U0)
    ref.run(40)
    got, want = sim.moments(), ref.moments()
    err = max_rel(got, want) if precision == "fp64" else rel_l1(got, want)
    assert err.max() <= (1e-11 if precision == "fp64" else 1e-5), err
    t, steps, xi = sim.time()
    assert steps == 40
    if precision == "fp64":
        assert abs(xi - ref.xi) <= 1e-11 * ref.xi and abs(t - ref.t) <= 1e-12 * ref.t
    sim.close()


@pytest.mark.parametrize("kind", ["characteristic", "transmissive"])
@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_euler_vortex_open_x(vk, omega, kind):
    """Euler, x faces characteristic, y periodic; the vortex placed off-centre so
    that its flow crosses the x faces; omega = 1.6 (relaxation, not f = f^eq)."""
    nx, ny = 40, 48
    U0 = np.ascontiguousarray(inputs.isentropic_vortex(48, center=(3.5, 5.0))[:, :, :40])
    lo, hi = (0.0, 0.0), (10.0 * 40 / 48, 10.0)
    sim = vk.Sim("euler", (nx, ny), lo, hi, precision="fp64", omega=omega, cfl=0.3, bc=(kind, "periodic"))
    sim.set_state(U0)
    sim.step_to(0.4)
    ref = ovklb.Sim(systems.Euler(1.4, 2), (nx, ny), lo, hi, bc=(kind, "periodic"), omega=omega, nu=0.3)
    ref.set_state(U0)
    ref.run_to(0.4)
    assert max_rel(sim.moments(), ref.moments()).max() <= 1e-11
    assert sim.time()[1] == ref.steps
    sim.close()


@pytest.mark.parametrize("kind", ["characteristic", "transmissive"])
def test_uniform_state_fixed(vk, kind):
    U = np.broadcast_to(inputs.euler_conserved(np.array(1.1), np.array(0.5), np.array(-0.3), np.array(0.8),
                                               1.4)[:, None, None], (4, 40, 72)).copy()
    sim = vk.Sim("euler", (72, 40), (0, 0), (1.8, 1.0), precision="fp64", omega=1.0, cfl=0.3, bc=kind)
    sim.set_state(U)
    sim.step(50)
    assert np.abs(sim.moments() - U).max() <= 1e-13
    sim.close()


@pytest.mark.parametrize("kind,frac,ratio", [("characteristic", 0.02, 0.35), ("transmissive", 0.01, 0.2)])
def test_hump_leaves_the_box(vk, kind, frac, ratio):
    """The radial Sec. 5.1 hump (Eq. 53) at N = 256 in [-5, 5]^2 to T = 8 against a
    periodic box three times as wide (which the waves do not cross before T).
    The characteristic construction applied per face is exact for waves
    leaving along the normal and reflects a part of obliquely incident ones,
    which numerical diffusion hides at coarse N (the oracle at N = 32 / 64:
    0.13 / 0.24 % of the amplitude) and which converges to a fixed level as N
    grows (measured here: 1.2 % of the amplitude, a quarter of what a periodic
    box of the same size is off by).  The transmissive faces reflect 0.45 % at
    N = 64 and 0.65 % at N = 256 (a seventh of the periodic box's error)."""
    def hump(n, L):
        x = inputs.cell_centers(n, -L, L)
        X, Y = np.meshgrid(x, x, indexing="xy")
        r = np.sqrt(X * X + Y * Y)
        h = np.where(r <= 1.0, 1.0 + 0.3 * ((1.0 + np.cos(np.pi * r)) / 2.0) ** 2, 1.0)
        z = np.zeros_like(h)
        return np.stack([h, z, z])
    n, T = 256, 8.0
    out = {}
    for bc in (kind, "periodic"):
        s = vk.Sim("swe", (n, n), (-5, -5), (5, 5), precision="fp64", g=1.0, omega=1.0, cfl=0.3, bc=bc)
        s.set_state(hump(n, 5.0))
        s.step_to(T)
        out[bc] = s.moments()
        s.close()
    big = vk.Sim("swe", (3 * n, 3 * n), (-15, -15), (15, 15), precision="fp64", g=1.0, omega=1.0, cfl=0.3)
    big.set_state(hump(3 * n, 15.0))
    big.step_to(T)
    ref = big.moments()[:, n:2 * n, n:2 * n]
    big.close()
    refl = np.abs(out[kind][0] - ref[0]).max()
    wrap = np.abs(out["periodic"][0] - ref[0]).max()
    assert refl < frac * 0.3 and refl < ratio * wrap, (refl, wrap)


def _mhd_pulse(nx, ny, L):
    dx = 2 * L / nx
    x = -L + (np.arange(nx) + 0.5) * dx
    y = -L + (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y, indexing="xy")
    r = np.sqrt((X - 2.4) ** 2 + (Y + 2.4) ** 2)
    b = np.where(r <= 1.4, ((1.0 + np.cos(np.pi * r / 1.4)) / 2.0) ** 2, 0.0)
    z = np.zeros_like(b)
    return inputs.mhd_conserved(1.0 + 0.2 * b, z + 0.3, z - 0.2, z, 1.0 + 0.3 * b, z + 0.5, z + 0.3, z, z, 5.0 / 3.0)


@pytest.mark.parametrize("bc", ["characteristic", ("characteristic", "periodic"), ("periodic", "characteristic"),
                                "transmissive"])
@pytest.mark.parametrize("tile", [(64, 5), None])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mhd_pulse_against_oracle(vk, bc, tile, precision):
    """MHD-GLM with non-periodic faces (the nine waves of the Jacobian along each
    face normal, c_h of step n): a pressure pulse in a uniform field over the
    x = hi / y = lo corner, on a ragged 44 x 34 grid, 30 steps; the default
    launch shape takes the 128-wide long-split march."""
    from parity_util import rel_l1_mhd
    nx, ny = 44, 34
    L = 3.0
    U0 = np.ascontiguousarray(_mhd_pulse(nx, ny, L))
    lo, hi = (-L, -L), (L, -L + ny * 2 * L / nx)
    sim = vk.Sim("mhd_glm", (nx, ny), lo, hi, precision=precision, omega=1.0, cfl=0.3, bc=bc, gamma=5.0 / 3.0)
    if tile:
        sim.set_tiling(*tile)
    sim.set_state(U0)
    sim.step(30)
    ref = ovklb.Sim(systems.MHDGLM(5.0 / 3.0), (nx, ny), lo, hi, bc=bc, omega=1.0, nu=0.3)
    ref.set_state(U0)
    ref.run(30)
    got, want = sim.moments(), ref.moments()
    if precision == "fp64":
        err = max_rel(got, want)
        assert err.max() <= 1e-11, err
        t, steps, xi = sim.time()
        assert steps == 30 and abs(xi - ref.xi) <= 1e-11 * ref.xi and abs(t - ref.t) <= 1e-12 * ref.t
    else:
        err = rel_l1_mhd(got, want)
        assert err.max() <= 1e-5, err
    if bc != "transmissive":
        assert np.abs(want[8]).max() > 1e-6     # the faces made a cleaning field: psi is compared, not zero
    sim.close()


@pytest.mark.parametrize("kind", ["characteristic", "transmissive"])
def test_uniform_mhd_state_fixed(vk, kind):
    u0 = inputs.mhd_conserved(np.array(1.3), np.array(0.2), np.array(-0.1), np.array(0.05), np.array(0.8),
                              np.array(0.6), np.array(-0.4), np.array(0.2), np.array(0.0), 5.0 / 3.0)
    U = np.broadcast_to(u0[:, None, None], (9, 30, 52)).copy()
    sim = vk.Sim("mhd_glm", (52, 30), (0, 0), (52 / 30, 1.0), precision="fp64", omega=1.0, cfl=0.3, bc=kind,
                 gamma=5.0 / 3.0)
    sim.set_state(U)
    sim.step(20)
    assert np.abs(sim.moments() - U).max() <= 1e-13 * np.abs(U).max()
    sim.close()


def test_refused_combinations(vk):
    s = vk.Sim("swe", (64, 64), (0, 0), (1, 1), bc="characteristic")
    with pytest.raises(vk.VKLBError) as e:
        s.set_variant(1, 4)
    assert e.value.status == vk.ERR_UNSUPPORTED
    with pytest.raises(vk.VKLBError) as e:
        s.set_form("moments")
    assert e.value.status == vk.ERR_UNSUPPORTED
    s.set_state(inputs.swe_sine_2d(64))
    with pytest.raises(vk.VKLBError) as e:
        vk.Batch([s])
    assert e.value.status == vk.ERR_UNSUPPORTED
    assert s.info.kernels_per_step == 3
    s.close()

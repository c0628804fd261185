"""The paired step kernel (vklb_set_variant 2: two neighbouring cells a thread,
packed two-lane FP32 arithmetic, 8-byte loads and stores) against the FP64
oracle (<= 1e-5 relative L1 per field) and against the plain FP32 kernel, on
ragged grids: odd widths (a tile whose last pair holds one cell), widths below
one tile, several tile shapes and both march directions; the global and the
per-cell normaliser; relaxation at omega != 1; characteristic faces; t_end
landing."""
import numpy as np
import pytest

from oracle import systems, vklb as ovklb
from paper_2608_04283_b300 import inputs
from parity_util import rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


def _vortex(nx, ny):
    return np.ascontiguousarray(inputs.isentropic_vortex(max(nx, ny), lo=0.0, hi=10.0)[:, :ny, :nx])


@pytest.mark.parametrize("n,tile", [((48, 40), (64, 8)), ((65, 37), (64, 5)), ((33, 30), (128, 7)),
                                    ((130, 50), (128, -1)), ((200, 24), (256, 6))])
@pytest.mark.parametrize("norm", ["global", "local"])
def test_euler_pair_against_oracle(vk, n, tile, norm):
    nx, ny = n
    L = 10.0 * nx / max(nx, ny)
    lo, hi = (0.0, 0.0), (L, L * ny / nx)
    U0 = _vortex(nx, ny)
    sim = vk.Sim("euler", n, lo, hi, precision="fp32", omega=2.0, cfl=0.3, alpha_norm=norm)
    sim.set_variant(2)
    sim.set_tiling(*tile)
    sim.set_state(U0)
    sim.step(20)
    ref = ovklb.Sim(systems.Euler(1.4, 2), n, lo, hi, omega=2.0, nu=0.3, alpha_norm=norm)
    ref.set_state(U0)
    ref.run(20)
    assert rel_l1(sim.moments(), ref.moments()).max() <= 1e-5
    plain = vk.Sim("euler", n, lo, hi, precision="fp32", omega=2.0, cfl=0.3, alpha_norm=norm)
    plain.set_state(U0)
    plain.step(20)
    assert rel_l1(sim.moments(), plain.moments()).max() <= 3e-6      # FP32 rounding of two kernels
    t, steps, xi = sim.time()
    assert steps == 20 and abs(xi - ref.xi) <= 1e-5 * ref.xi
    sim.close()
    plain.close()


@pytest.mark.parametrize("omega", [1.0, 1.4])
def test_swe_pair_to_time(vk, omega):
    n = (97, 64)
    U0 = np.ascontiguousarray(inputs.swe_hump_2d(97, 0.5, 0.5, 0.4, 0.08)[:, :64, :])
    lo, hi = (0.0, 0.0), (1.0, 64 / 97)
    sim = vk.Sim("swe", n, lo, hi, precision="fp32", omega=omega, cfl=0.3)
    sim.set_variant(2)
    sim.set_tiling(64, -1)
    sim.set_state(U0)
    sim.step_to(0.01)
    ref = ovklb.Sim(systems.ShallowWater(9.81, 2), n, lo, hi, omega=omega, nu=0.3)
    ref.set_state(U0)
    ref.run_to(0.01)
    assert rel_l1(sim.moments(), ref.moments()).max() <= 1e-5
    assert sim.time()[1] == ref.steps
    sim.close()


def test_pair_with_characteristic_faces(vk):
    nx, ny = 66, 40
    x = -3.0 + (np.arange(nx) + 0.5) * 6.0 / nx
    y = -3.0 + (np.arange(ny) + 0.5) * 6.0 / nx
    X, Y = np.meshgrid(x, y, indexing="xy")
    h = 1.0 + 0.3 * np.exp(-((X - 0.5) ** 2 + Y ** 2))
    U0 = np.stack([h, 0.2 * h, -0.1 * h])
    lo, hi = (-3.0, -3.0), (3.0, -3.0 + ny * 6.0 / nx)
    sim = vk.Sim("swe", (nx, ny), lo, hi, precision="fp32", g=1.0, omega=1.0, cfl=0.3, bc="characteristic")
    sim.set_variant(2)
    sim.set_tiling(64, 8)
    sim.set_state(U0)
    sim.step(30)
    ref = ovklb.Sim(systems.ShallowWater(1.0, 2), (nx, ny), lo, hi, bc="characteristic", omega=1.0, nu=0.3)
    ref.set_state(U0)
    ref.run(30)
    assert rel_l1(sim.moments(), ref.moments()).max() <= 1e-5
    sim.close()


def test_pair_refusals(vk):
    s = vk.Sim("euler", (64, 64), (0, 0), (1, 1), precision="fp64")
    with pytest.raises(vk.VKLBError) as e:
        s.set_variant(2)
    assert e.value.status == vk.ERR_UNSUPPORTED
    s.close()
    s = vk.Sim("mhd_glm", (64, 64), (0, 0), (1, 1), precision="fp32", gamma=5 / 3)
    with pytest.raises(vk.VKLBError) as e:
        s.set_variant(2)
    assert e.value.status == vk.ERR_UNSUPPORTED
    s.close()
    s = vk.Sim("euler", (64, 64), (0, 0), (1, 1), precision="fp32")
    s.set_tiling(96, 8)
    with pytest.raises(vk.VKLBError) as e:
        s.set_variant(2)                       # 96 cells = 48 threads: not whole warps
    assert e.value.status == vk.ERR_ARG
    s.set_tiling(128, 8)
    s.set_variant(2)
    with pytest.raises(vk.VKLBError):
        s.set_tiling(96, 8)
    s.set_state(inputs.entropy_wave_2d(64))
    with pytest.raises(vk.VKLBError) as e:
        vk.Batch([s])
    assert e.value.status == vk.ERR_UNSUPPORTED
    s.close()

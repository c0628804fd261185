"""Launch-shape rules on the GPU: the wave-fit tile height, the occupancy the
library reports, and parity at the extreme shapes it can pick (one-row tiles)."""
import numpy as np
import pytest

from oracle import systems, vklb as ovklb
from paper_2608_04283_b300 import inputs
from parity_util import max_rel, rel_l1_mhd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


@pytest.mark.parametrize("name,n,tx,prec", [("mhd_glm", 2048, 128, "fp32"), ("euler", 1024, 128, "fp32"),
                                             ("euler", 1000, 64, "fp64"), ("swe", 4096, 256, "fp32")])
def test_wave_fit_height(vk, name, n, tx, prec):
    """ty = -1 takes the smallest k whose height ceil(ny / (k floor(slots / gx)))
    fits 256 rows, slots = SMs x resident blocks per SM; the grid then fills at
    most k waves."""
    kw = dict(gamma=5 / 3) if name == "mhd_glm" else {}
    sim = vk.Sim(name, (n, n), (0, 0), (1, 1), precision=prec, **kw)
    sim.set_tiling(tx, -1)
    inf = sim.info
    assert inf.tile_x == tx and inf.blocks_per_sm >= 1 and inf.sms >= 1
    gx = -(-n // tx)
    rows = max(1, inf.blocks_per_sm * inf.sms // gx)
    k = 1
    while -(-n // (k * rows)) > 256:
        k += 1
    assert inf.tile_y == max(1, -(-n // (k * rows)))
    gy = -(-n // inf.tile_y)
    assert gx * gy <= k * inf.blocks_per_sm * inf.sms
    sim.close()


def test_occupancy_reports_register_bound(vk):
    """FP32 MHD-GLM runs the step with a 4-blocks-per-SM register bound when the
    block has at most 128 threads."""
    sim = vk.Sim("mhd_glm", (256, 256), (0, 0), (1, 1), precision="fp32", gamma=5 / 3)
    sim.set_tiling(128, 16)
    assert sim.info.blocks_per_sm >= 4
    sim.close()


@pytest.mark.parametrize("tile", [(32, -1), (32, 1), (64, 3)])
def test_short_tiles_fp64_parity(vk, tile):
    """One-row and three-row tiles (what the wave fit picks on small grids)."""
    n = (48, 40)
    U0 = np.ascontiguousarray(inputs.isentropic_vortex(48, lo=0.0, hi=10.0)[:, :40, :])
    lo, hi = (0.0, 0.0), (10.0, 10.0 * 40 / 48)
    sim = vk.Sim("euler", n, lo, hi, precision="fp64", omega=2.0, cfl=0.3)
    sim.set_tiling(*tile)
    sim.set_state(U0)
    sim.step(12)
    ref = ovklb.Sim(systems.Euler(1.4, 2), n, lo, hi, omega=2.0, nu=0.3)
    ref.set_state(U0)
    ref.run(12)
    assert max_rel(sim.moments(), ref.moments()).max() <= 1e-11
    sim.close()


def test_mhd_bounded_kernel_parity(vk):
    """The register-bounded FP32 MHD-GLM step against the oracle on a ragged grid
    (128-thread tiles take the bounded kernel, 256-thread tiles the unbounded one;
    both must agree with the oracle).  The strip of the Orszag-Tang state is not
    periodic in y, so the seam makes a small psi; the FP32 comparison measures
    psi against c_h |B| (rel_l1_mhd)."""
    n = (300, 36)
    L = 2 * np.pi
    U0 = np.ascontiguousarray(inputs.orszag_tang(300)[:, :36, :])
    lo, hi = (0.0, 0.0), (L, L * 36 / 300)
    ref = ovklb.Sim(systems.MHDGLM(5 / 3), n, lo, hi, omega=1.0, nu=0.3, ch_factor=6.0)
    ref.set_state(U0)
    ref.run(10)
    want = ref.moments()
    for tile in [(128, -1), (256, 8)]:
        sim = vk.Sim("mhd_glm", n, lo, hi, precision="fp32", omega=1.0, cfl=0.3, gamma=5 / 3)
        sim.set_tiling(*tile)
        sim.set_state(U0)
        sim.step(10)
        assert rel_l1_mhd(sim.moments(), want).max() <= 1e-5
        sim.close()

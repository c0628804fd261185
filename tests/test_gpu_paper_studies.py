"""The paper's verification studies on the GPU (FP64, sizes the oracle cannot
reach), under both readings of alpha's normaliser (Eq. 27; reading R1):

* Sec. 5.2 vortex (Eq. 57), CFL 0.3, omega = 2, T = 2, N = 64 .. 1024: second
  order with the grid-wide normaliser (the default); the per-cell one diverges
  from N = 512.
* Sec. 5.1 Table 1 at the paper's CFL numbers (0.9; 0.8 for the hydraulic jump),
  N = 64 .. 4096: the standard dam break converges with the grid-wide
  normaliser and degrades from N = 1024 with the per-cell one.
* Sec. 5.2 Table 2 at CFL 0.9 (Sod, Leblanc, sonic point) to N = 8192 / 16384:
  slightly below first order under both, the grid-wide one more accurate.
* Sec. 5.2 entropy wave (Eq. 55), omega = 2, T = 1: recorded as a finding --
  neither reading reaches the paper's N = 512 (the linearised scheme grows
  about 1.5 % a step at this uniform flow, so 3,840 steps amplify rounding
  beyond the physical range).
* The instability studies (E9): the discontinuous set fails on the vortex for
  every CFL number in 0.05 .. 0.30 (Sec. 5.2), where the weighted set
  converges; on the 1D problems with a sonic point (Leblanc, fixed sonic point)
  the weighted set is more accurate than the discontinuous one (Sec. 5.2).
The exact solutions are the translated initial data (vortex, entropy wave) and
the exact Riemann solvers of oracle/riemann.py."""
import numpy as np
import pytest

from oracle import riemann
from paper_2608_04283_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


def _vortex_err(vk, n, norm="global", set_kind="weighted", cfl=0.3, T=2.0, precision="fp64"):
    """L2 error per field at T against the translated vortex, or None when the
    run left the physical range (the library reports VKLB_ERR_NONPHYSICAL) or
    its wave speeds grew tenfold (an unstable run whose lattice speed, and so its
    step count to T, would grow without bound)."""
    s = vk.Sim("euler", (n, n), (0, 0), (10, 10), precision=precision, omega=2.0, cfl=cfl, alpha_norm=norm,
               set_kind=set_kind)
    s.set_state(inputs.isentropic_vortex(n))
    xi0 = s.time()[2]
    try:
        for i in range(1, 21):
            s.step_to(T * i / 20)
            if not s.time()[2] < 10 * xi0:
                return None
        U = s.moments()
    except vk.VKLBError as e:
        assert e.status == vk.ERR_NONPHYSICAL
        return None
    finally:
        s.close()
    err = np.sqrt(np.mean((U - inputs.isentropic_vortex(n, shift=(T, T))) ** 2, axis=(1, 2)))
    return err if np.all(np.isfinite(err)) else None


def test_vortex_convergence_study(vk):
    errs = np.array([_vortex_err(vk, n) for n in (64, 128, 256, 512, 1024)])
    rates = np.log2(errs[:-1] / errs[1:])
    # L2 per field (measured: 1.93-2.03 for rho, 1.95-2.10 for the others)
    assert np.all(rates[:, 0] > 1.9) and np.all(rates > 1.8) and np.all(rates < 2.2), (errs[:, 0], rates)
    assert errs[-1, 0] < 2.5e-6
    # the per-cell normaliser: second order at first, then the run diverges
    loc = [_vortex_err(vk, n, norm="local") for n in (64, 128, 256, 512)]
    assert np.log2(loc[0][0] / loc[1][0]) > 1.9
    assert loc[2][0] > 1.5 * errs[2, 0]
    assert loc[3] is None


def _riemann_l1(vk, table, name, n, cfl, norm="global", set_kind="weighted"):
    if table == 1:
        (lo, hi), T, x0, h, q, g = inputs.SWE_RIEMANN_TABLE1[name]
        U0, _ = inputs.swe_riemann_1d(name, n)
        sim = vk.Sim("swe", (n,), (lo,), (hi,), precision="fp64", cfl=cfl, bc="characteristic", omega=1.0, g=g,
                     alpha_norm=norm, set_kind=set_kind)
        x = inputs.cell_centers(n, lo, hi)
        ex = riemann.swe_sample(h[0], q[0] / h[0], h[1], q[1] / h[1], g, x, T, x0=x0)[0]
    else:
        (lo, hi), T, x0, r, u, p, gam = inputs.EULER_RIEMANN_TABLE2[name]
        U0, _ = inputs.euler_riemann_1d(name, n)
        sim = vk.Sim("euler", (n,), (lo,), (hi,), precision="fp64", cfl=cfl, bc="characteristic", omega=1.0,
                     gamma=gam, alpha_norm=norm, set_kind=set_kind)
        x = inputs.cell_centers(n, lo, hi)
        ex = riemann.euler_sample(r[0], u[0], p[0], r[1], u[1], p[1], gam, x, T, x0=x0)[0]
    sim.set_state(U0)
    try:
        sim.step_to(T)
        e = float(np.sum(np.abs(sim.moments()[0] - ex)) * (hi - lo) / n)
    except vk.VKLBError:
        e = float("inf")
    sim.close()
    return e


TABLE1 = [("standard", 0.9), ("hydraulic", 0.8), ("compression", 0.9)]


@pytest.mark.parametrize("name,cfl", TABLE1)
def test_table1_convergence_paper_cfl(vk, name, cfl):
    Ns = [64, 128, 256, 512, 1024, 2048, 4096]
    errs = np.array([_riemann_l1(vk, 1, name, n, cfl) for n in Ns])
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates > 0.55) and np.all(rates < 1.4), (errs, rates)
    if name == "standard":
        loc = [_riemann_l1(vk, 1, name, n, cfl, norm="local") for n in (512, 1024, 4096)]
        assert loc[1] > loc[0] and loc[2] > loc[0], loc      # the per-cell normaliser degrades
        assert errs[-1] < 0.1 * loc[2]


TABLE2 = [("sod", [128, 512, 2048, 8192]), ("leblanc", [512, 2048, 8192, 16384]),
          ("sonic", [128, 512, 2048, 8192])]


@pytest.mark.parametrize("name,Ns", TABLE2)
def test_table2_convergence_paper_cfl(vk, name, Ns):
    errs = np.array([_riemann_l1(vk, 2, name, n, 0.9) for n in Ns])
    rates = np.log2(errs[:-1] / errs[1:]) / np.log2(np.array(Ns[1:]) / np.array(Ns[:-1]))
    assert np.all(rates > 0.5) and np.all(rates < 1.1), (errs, rates)
    assert errs[-1] < _riemann_l1(vk, 2, name, Ns[-1], 0.9, norm="local")


@pytest.mark.parametrize("name", ["leblanc", "sonic"])
def test_weighted_beats_discontinuous_at_sonic_points(vk, name):
    """E9, 1D: where an eigenvalue changes sign in the rarefaction (Leblanc, the
    fixed sonic point) the discontinuous set forms a spurious jump; the weighted
    set is the more accurate of the two at every N."""
    for n in (1024, 4096):
        w = _riemann_l1(vk, 2, name, n, 0.9)
        d = _riemann_l1(vk, 2, name, n, 0.9, set_kind="discontinuous")
        assert w < d, (n, w, d)


@pytest.mark.parametrize("cfl", [0.05, 0.10, 0.15, 0.20, 0.25, 0.30])
def test_discontinuous_set_unstable_on_vortex(vk, cfl):
    """E9, 2D (Sec. 5.2): the discontinuous set is unstable on the vortex for
    every CFL number in 0.05 .. 0.30: it leaves the physical range or ends far
    from the exact solution, while the weighted set converges there."""
    n = 128
    d = _vortex_err(vk, n, set_kind="discontinuous", cfl=cfl)
    w = _vortex_err(vk, n, cfl=cfl)
    assert w is not None and w[0] < 3e-4
    assert d is None or d[0] > 100 * w[0], (cfl, d, w)


def test_entropy_wave_finding(vk):
    """Sec. 5.2 entropy wave (omega = 2, CFL 0.3, T = 1): second order from
    N = 32 to 64, but no reading reaches the paper's N = 512: the run leaves the
    physical range there under both (rounding grows about 1.5 % a step in this
    uniform flow under the grid-wide normaliser, 3.4 % under the per-cell one)."""
    def err(n, norm):
        s = vk.Sim("euler", (n, n), (0, 0), (1, 1), precision="fp64", omega=2.0, cfl=0.3, alpha_norm=norm)
        s.set_state(inputs.entropy_wave_2d(n))
        try:
            s.step_to(1.0)
            return float(np.sqrt(np.mean((s.moments()[0] - inputs.entropy_wave_exact(n, 1.0)[0]) ** 2)))
        except vk.VKLBError:
            return None
        finally:
            s.close()
    e32, e64 = err(32, "global"), err(64, "global")
    assert e64 < e32 / 3.0
    assert err(512, "global") is None and err(512, "local") is None

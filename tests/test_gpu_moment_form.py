"""The moment form (vklb_set_form(sim, 1)): at omega = 1 the collision leaves
f* = f^eq(U) (Eq. 42), so the step is the finite-volume update of Thm 4.3 and U
alone can be the state.  Checked against the FP64 oracle (the same oracle as the
distribution form, at omega = 1), and against the distribution form itself:
after every step the stored U equals ((((f1 + f2) + f3) + f4) + f5) of the
distribution form's stored f, summed in the store type, to rounding: the two
kernels share the arithmetic, but the compiler may fuse multiply-adds
differently in each, and in FP32 MHD-GLM a last-place difference can move a
cell across the switch to the FP64 eigenvector normalisation; so the bound is
the FP32 parity tolerance (FP64: 1e-13), not bit for bit."""
import numpy as np
import pytest

from oracle import systems, vklb as ovklb
from paper_2608_04283_b300 import inputs
from parity_util import max_rel, rel_l1, rel_l1_mhd

pytestmark = pytest.mark.gpu

HDR, CTL = 48, 112   # blob header and control words (vklb_get_state)


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


def _case(name, n):
    nx, ny = n
    if name == "swe":
        U0 = inputs.swe_hump_2d(nx, 0.4, 0.5, 0.45, 0.08)[:, :ny, :]
        return np.ascontiguousarray(U0), (0.0, 0.0), (1.0, ny / nx), {}, systems.ShallowWater(9.81, 2)
    if name == "euler":
        U0 = inputs.isentropic_vortex(nx, lo=0.0, hi=10.0)[:, :ny, :]
        return np.ascontiguousarray(U0), (0.0, 0.0), (10.0, 10.0 * ny / nx), {}, systems.Euler(1.4, 2)
    L = 2 * np.pi
    U0 = inputs.orszag_tang(nx)[:, :ny, :]
    return np.ascontiguousarray(U0), (0.0, 0.0), (L, L * ny / nx), dict(gamma=5 / 3), systems.MHDGLM(5 / 3)


def _cells(blob, p, q, nx, ny, dtype):
    """Blob payload in the brick layout -> [q][p][ny][nx] (q = 1: the moments)."""
    pitch = -(-nx // 32) * 32
    a = np.frombuffer(blob[HDR + CTL:].tobytes(), dtype=dtype).reshape(ny, pitch // 32, q * p, 32)
    a = a.transpose(2, 0, 1, 3).reshape(q * p, ny, pitch)[:, :, :nx]
    return a.reshape(q, p, ny, nx)


@pytest.mark.parametrize("name", ["swe", "euler", "mhd_glm"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("tile", [None, (32, 8), (64, 4), (32, 40)])
def test_moment_form_parity(vk, name, precision, tile):
    n = (44, 40)
    U0, lo, hi, kw, sysm = _case(name, n)
    sim = vk.Sim(name, n, lo, hi, precision=precision, omega=1.0, cfl=0.3, form="moments", **kw)
    assert sim.info.form == 1 and sim.info.bytes_per_lup == 2 * sim.p * (8 if precision == "fp64" else 4)
    if tile:
        sim.set_tiling(*tile)
    sim.set_state(U0)
    sim.step(15)
    got = sim.moments()
    t, nsteps, xi = sim.time()
    sim.close()
    ref = ovklb.Sim(sysm, n, lo, hi, omega=1.0, nu=0.3)
    ref.set_state(U0)
    ref.run(15)
    want = ref.moments()
    if precision == "fp64":
        assert max_rel(got, want).max() <= 1e-11
        assert abs(t - ref.t) <= 1e-12 * ref.t and abs(xi - ref.xi) <= 1e-11 * ref.xi
    else:
        err = rel_l1_mhd(got, want) if name == "mhd_glm" else rel_l1(got, want)
        assert err.max() <= 1e-5
    assert nsteps == 15


@pytest.mark.parametrize("name", ["swe", "euler", "mhd_glm"])
@pytest.mark.parametrize("precision,dtype,tol", [("fp32", np.float32, 1e-5), ("fp64", np.float64, 1e-13)])
def test_moment_form_equals_distribution_form(vk, name, precision, dtype, tol):
    n = (72, 44)
    U0, lo, hi, kw, _ = _case(name, n)
    sims = []
    for form in ("distributions", "moments"):
        s = vk.Sim(name, n, lo, hi, precision=precision, omega=1.0, cfl=0.3, form=form, **kw)
        s.set_tiling(64, 8)
        s.set_state(U0)
        sims.append(s)
    for steps in (0, 1, 6):
        for s in sims:
            s.step(steps)
        f = _cells(sims[0].get_state(), sims[0].p, 5, n[0], n[1], dtype)
        U = _cells(sims[1].get_state(), sims[1].p, 1, n[0], n[1], dtype)[0]
        fsum = (((f[0] + f[1]) + f[2]) + f[3]) + f[4]           # IEEE adds in the store type
        scale = np.abs(fsum).reshape(fsum.shape[0], -1).max(axis=1)
        # a small field (psi of Orszag-Tang) rounds with the c_h B terms its
        # components carry (Eq. 58), so its scale is at least 0.1 of the largest
        scale = np.maximum(scale, 0.1 * scale.max())
        err = np.abs(U.astype(np.float64) - fsum).reshape(fsum.shape[0], -1).max(axis=1) / scale
        assert err.max() <= tol, err
        (ta, na, xa), (tb, nb, xb) = sims[0].time(), sims[1].time()
        assert na == nb and abs(ta - tb) <= 4 * tol * ta and abs(xa - xb) <= 4 * tol * xa
    for s in sims:
        s.close()


def test_moment_form_bf16_storage(vk):
    """BF16 storage of U (FP32 arithmetic): the error is bounded by BF16 rounding
    of the stored moments (about 4e-3 relative a step), the same bound as the
    distribution form's BF16 experiment."""
    n = (44, 40)
    U0, lo, hi, kw, sysm = _case("euler", n)      # every field O(1), as in the distribution form's test
    sim = vk.Sim("euler", n, lo, hi, precision="bf16", omega=1.0, cfl=0.3, form="moments")
    assert sim.info.bytes_per_lup == 2 * 4 * 2
    sim.set_state(U0)
    sim.step(10)
    ref = ovklb.Sim(sysm, n, lo, hi, omega=1.0, nu=0.3)
    ref.set_state(U0)
    ref.run(10)
    assert rel_l1(sim.moments(), ref.moments()).max() <= 2e-2
    sim.close()


def test_moment_form_lands_on_t_and_conserves(vk):
    n = (40, 40)
    U0, lo, hi, kw, sysm = _case("swe", n)
    sim = vk.Sim("swe", n, lo, hi, precision="fp64", omega=1.0, cfl=0.3, form="moments")
    sim.set_state(U0)
    t0 = sim.totals()
    sim.step_to(0.02)
    t, nsteps, _ = sim.time()
    assert t == pytest.approx(0.02, abs=1e-15)
    ref = ovklb.Sim(sysm, n, lo, hi, omega=1.0, nu=0.3)
    ref.set_state(U0)
    ref.run_to(0.02)
    assert nsteps == ref.steps
    assert max_rel(sim.moments(), ref.moments()).max() <= 1e-11
    t1 = sim.totals()
    assert np.abs(t1 - t0).max() <= 1e-13 * np.abs(t0).max()      # Thm 4.3 on a periodic grid
    sim.close()


def test_moment_form_checkpoint_bitwise(vk):
    n = (48, 36)
    U0, lo, hi, kw, _ = _case("mhd_glm", n)
    a = vk.Sim("mhd_glm", n, lo, hi, precision="fp32", omega=1.0, cfl=0.3, form="moments", **kw)
    a.set_state(U0)
    a.step(10)
    blob = a.get_state()
    a.step(10)
    b = vk.Sim("mhd_glm", n, lo, hi, precision="fp32", omega=1.0, cfl=0.3, form="moments", **kw)
    b.put_state(blob)
    b.step(10)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.time() == b.time()
    c = vk.Sim("mhd_glm", n, lo, hi, precision="fp32", omega=1.0, cfl=0.3, **kw)   # distribution form
    with pytest.raises(vk.VKLBError) as e:
        c.put_state(blob)
    assert e.value.status == vk.ERR_ARG
    for s in (a, b, c):
        s.close()


def test_moment_form_batch(vk):
    """Batched moment-form steps: a batch of three uneven grids equals, member by
    member, a batch of one of the same member bit for bit (the same kernel), and
    the single-simulation kernel to FP32 rounding (two kernels may contract
    multiply-adds differently; measured 4e-7).  A member whose form changed
    behind the batch's back is refused."""
    sides = [64, 96, 40]
    sims, one, solo = [], [], []
    for i, m in enumerate(sides):
        U0 = inputs.swe_hump_2d(m, 0.3 + 0.1 * i, 0.5, 0.5, 0.08)
        for group in (sims, one, solo):
            s = vk.Sim("swe", (m, m), (0, 0), (1, 1), precision="fp32", omega=1.0, cfl=0.3, form="moments")
            s.set_tiling(64, 8)
            s.set_state(U0)
            group.append(s)
    b = vk.Batch(sims, tile=(64, 8))
    b.step(12, graph=True)
    sims[1].set_form("distributions")             # a member changed behind the batch's back
    with pytest.raises(vk.VKLBError) as e:
        b.step(1)
    assert e.value.status == vk.ERR_STATE
    b.close()
    sims[1].close()
    sims[1] = vk.Sim("swe", (96, 96), (0, 0), (1, 1), precision="fp32", omega=1.0, cfl=0.3, form="moments")
    sims[1].set_tiling(64, 8)
    sims[1].set_state(inputs.swe_hump_2d(96, 0.4, 0.5, 0.5, 0.08))
    b = vk.Batch(sims[1:2], tile=(64, 8))
    b.step(12, graph=True)
    b.close()
    for s in one:
        bo = vk.Batch([s], tile=(64, 8))
        bo.step(12, graph=True)
        bo.close()
    for s in solo:
        s.step(12)
    for x, y, z in zip(sims, one, solo):
        assert np.array_equal(x.get_state(), y.get_state())
        u, w = x.moments(), z.moments()
        for k in range(u.shape[0]):
            assert np.abs(u[k] - w[k]).max() <= 2e-6 * np.abs(w[k]).max()
        for s in (x, y, z):
            s.close()


def test_moment_form_rejections(vk):
    U0, lo, hi, kw, _ = _case("euler", (32, 32))
    s = vk.Sim("euler", (32, 32), lo, hi, precision="fp32", omega=2.0, cfl=0.3)
    with pytest.raises(vk.VKLBError) as e:
        s.set_form("moments")                        # omega != 1: f* is not f^eq
    assert e.value.status == vk.ERR_ARG
    s.close()
    s = vk.Sim("euler", (32, 32), lo, hi, precision="fp32", omega=1.0, cfl=0.3, form="moments")
    with pytest.raises(vk.VKLBError) as e:
        s.set_variant(1, 2)
    assert e.value.status == vk.ERR_UNSUPPORTED
    with pytest.raises(vk.VKLBError) as e:
        s.step(1)                                    # no state set after the form change
    assert e.value.status == vk.ERR_STATE
    s.close()
    s1 = vk.Sim("swe", (64,), (0.0,), (1.0,), precision="fp64", omega=1.0)
    with pytest.raises(vk.VKLBError) as e:
        s1.set_form("moments")
    assert e.value.status == vk.ERR_UNSUPPORTED
    s1.close()

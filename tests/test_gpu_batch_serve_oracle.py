"""The batched and served forms against the FP64 oracle, member by member.

Batched form: one launch per step over a tile work-list spanning uneven grids
(sides that are not multiples of 32, one smaller than a tile), both state forms,
with and without CUDA-graph replay; every member after the run equals its own
oracle run within 1e-11 (max relative per field), with the same step count, time
and lattice speed (each member keeps its own xi and c_h).
Served form: a small FP64 trace of mixed requests under a budget that forces
queueing; every result equals its own oracle run within 1e-11."""
import numpy as np
import pytest

from oracle import systems, vklb as ovklb
from paper_2608_04283_b300 import inputs
from parity_util import max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


def _oracle(sysm, n, side, U0, steps, **kw):
    ref = ovklb.Sim(sysm, n, (0.0, 0.0), (side, side * n[1] / n[0]), **kw)
    ref.set_state(U0)
    ref.run(steps)
    return ref


@pytest.mark.parametrize("form", ["distributions", "moments"])
def test_batched_swe_fp64_against_oracle(vk, form):
    sides = [(20, 20), (33, 33), (47, 40), (64, 64), (90, 71)]   # 20 < one 32-wide tile
    sims, refs = [], []
    for i, (nx, ny) in enumerate(sides):
        U0 = np.ascontiguousarray(inputs.swe_hump_2d(nx, 0.2 + 0.15 * i, 0.5, 0.45, 0.08)[:, :ny, :])
        s = vk.Sim("swe", (nx, ny), (0, 0), (1.0, ny / nx), precision="fp64", omega=1.0, cfl=0.3, form=form)
        s.set_state(U0)
        sims.append(s)
        refs.append(_oracle(systems.ShallowWater(9.81, 2), (nx, ny), 1.0, U0, 14, omega=1.0, nu=0.3))
    b = vk.Batch(sims, tile=(32, 8))
    b.step(6, graph=True)
    b.step(8, graph=False)
    b.close()
    for s, r in zip(sims, refs):
        assert max_rel(s.moments(), r.moments()).max() <= 1e-11
        t, steps, xi = s.time()
        assert steps == 14 and abs(t - r.t) <= 1e-12 * r.t and abs(xi - r.xi) <= 1e-11 * r.xi
        s.close()


def test_batched_mhd_fp64_against_oracle(vk):
    sides = [18, 40, 52]
    sims, refs = [], []
    L = 2 * np.pi
    for i, m in enumerate(sides):
        U0 = inputs.orszag_tang(m, phase=(0.4 * i, 0.2 * i))
        s = vk.Sim("mhd_glm", (m, m), (0, 0), (L, L), precision="fp64", omega=1.0, cfl=0.3, gamma=5 / 3)
        s.set_state(U0)
        sims.append(s)
        refs.append(_oracle(systems.MHDGLM(5 / 3), (m, m), L, U0, 10, omega=1.0, nu=0.3))
    b = vk.Batch(sims, tile=(64, 8))
    b.step(10, graph=True)
    b.close()
    for s, r in zip(sims, refs):
        assert max_rel(s.moments(), r.moments()).max() <= 1e-11
        t, steps, xi = s.time()
        assert steps == 10 and abs(xi - r.xi) <= 1e-11 * r.xi
        s.close()


def test_served_fp64_against_oracle(vk):
    from paper_2608_04283_b300 import serve
    trace = inputs.serving_trace(count=7, rate=1e6, seed=11, nmin=24, nmax=48, nstep=8, smin=6, smax=16)
    for r in trace:
        if r.system == "mhd_glm":        # keep the oracle's MHD-GLM runs short
            r.n, r.steps = 24, min(r.steps, 8)
    budget = 2.5 * max(serve.device_bytes(r.system, r.n, "fp64") for r in trace)
    server = serve.Server(budget_bytes=budget, tick_steps=5, precision="fp64", keep_results=True, max_side=64,
                          tiles={"swe": (32, 8), "euler": (32, 8), "mhd_glm": (64, 8)})
    rep = server.run(trace, realtime=False)
    assert rep.summary()["completed"] == len(trace)
    assert rep.peak_bytes <= budget
    mk = {"swe": lambda: systems.ShallowWater(9.81, 2), "euler": lambda: systems.Euler(1.4, 2),
          "mhd_glm": lambda: systems.MHDGLM(5 / 3)}
    for job in rep.jobs:
        r = job.req
        kw, side = serve.FAMILY[r.system]
        ref = _oracle(mk[r.system](), (r.n, r.n), side, inputs.request_initial_state(r), r.steps,
                      omega=kw["omega"], nu=kw["cfl"], alpha_norm=kw.get("alpha_norm", "global"))
        assert max_rel(job.result, ref.moments()).max() <= 1e-11, r

"""The allocation-free conservation totals (vklb_conservation_totals_noalloc).

Some callers cannot call cudaMalloc (they only receive device pointers from
another runtime, or run where allocation is not allowed).  This entry point
reduces a distribution buffer they own using a fixed device array inside the
library instead of an allocated scratch buffer.  Checked here through the C ABI
against the allocating vklb_conservation_totals on the same state, twice in a
row (the array keeps the previous call's contents), to host and to device
outputs: both reduce in the same fixed order (same blocks, chunks, shuffle tree
and final pass), so the totals must agree bit for bit.  This file is collected
last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2608_04283_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    fn = vklb.lib().vklb_conservation_totals_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_double,
                   C.c_void_p, C.c_int32, C.c_void_p]
    return vklb


def _noalloc(vk, sim, out, on_device, stream=None):
    info = sim.info
    vol = info.dx ** sim.dim
    ptr = out.data_ptr() if on_device else out.ctypes.data
    return vk.lib().vklb_conservation_totals_noalloc(
        C.c_void_p(sim.device_state()), info.precision, info.q, info.p, sim.n[0], sim.n[1] if sim.dim == 2 else 1,
        info.pitch, vol, C.c_void_p(ptr), 1 if on_device else 0, C.c_void_p(stream))


CASES = [
    ("euler", (48, 40), (0.0, 0.0), (10.0, 10.0 * 40 / 48), lambda: inputs.isentropic_vortex(48)[:, :40, :],
     dict(omega=2.0, cfl=0.3), "fp32"),
    ("mhd_glm", (36, 32), (0.0, 0.0), (2 * np.pi, 2 * np.pi * 32 / 36), lambda: inputs.orszag_tang(36)[:, :32, :],
     dict(omega=1.0, cfl=0.3, gamma=5 / 3), "fp64"),
    ("swe", (400,), (0.0,), (1.0,), lambda: inputs.dam_break_1d(400),
     dict(omega=1.0, cfl=0.6, bc="characteristic"), "fp64"),
    ("euler", (70, 64), (0.0, 0.0), (10.0, 10.0 * 64 / 70), lambda: inputs.isentropic_vortex(70)[:, :64, :],
     dict(omega=1.0, cfl=0.3), "bf16"),
]


@pytest.mark.parametrize("system,n,lo,hi,ic,kw,prec", CASES)
def test_noalloc_totals_match_allocating_entry_point(vk, system, n, lo, hi, ic, kw, prec):
    import torch
    sim = vk.Sim(system, n, lo, hi, precision=prec, **kw)
    sim.set_state(np.ascontiguousarray(ic()))
    sim.step(7)
    ref = sim.totals()
    for _ in range(2):                     # two calls in a row share the array
        host = np.full(sim.p, np.nan)
        assert _noalloc(vk, sim, host, False) == vk.OK
        assert np.array_equal(host, ref), (host, ref)
    dev = torch.full((sim.p,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        assert _noalloc(vk, sim, dev, True) == vk.OK
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), ref)
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_array(vk):
    sim = vk.Sim("euler", (16, 16), (0, 0), (1, 1), precision="fp32")
    sim.set_state(inputs.entropy_wave_2d(16))
    host = np.zeros(32)
    f = vk.lib().vklb_conservation_totals_noalloc
    st = f(C.c_void_p(sim.device_state()), 1, 5, 17, 16, 16, sim.info.pitch, 1.0, C.c_void_p(host.ctypes.data), 0,
           None)
    assert st == -9
    assert "fixed limits" in vk.lib().vklb_strerror(st).decode()
    sim.close()

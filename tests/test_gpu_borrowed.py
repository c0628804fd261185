"""Distribution buffers owned by the caller (vklb_create_borrowed): torch
tensors hold the state, the results equal those of a simulation that owns its
buffers bit for bit, the tensors hold the documented brick layout, and
destroying the simulation leaves them to their owner."""
import numpy as np
import pytest

from paper_2608_04283_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vk():
    from paper_2608_04283_b300 import build
    build.build()
    from paper_2608_04283_b300 import vklb
    return vklb


@pytest.mark.parametrize("system,precision", [("euler", "fp32"), ("euler", "fp64"), ("mhd_glm", "fp32")])
def test_borrowed_equals_owned(vk, system, precision):
    import torch
    n = (100, 37)
    if system == "euler":
        U0 = np.ascontiguousarray(inputs.isentropic_vortex(100, lo=0.0, hi=10.0)[:, :37, :])
        L, kw = 10.0, dict(omega=2.0, cfl=0.3)
    else:
        U0 = np.ascontiguousarray(inputs.orszag_tang(100)[:, :37, :])
        L, kw = 2 * np.pi, dict(omega=1.0, cfl=0.3, gamma=5 / 3)
    lo, hi = (0.0, 0.0), (L, L * 37 / 100)
    need = vk.buffer_bytes(system, n, precision)
    bufs = [torch.full((need + 512,), 7, dtype=torch.uint8, device="cuda") for _ in range(2)]
    a = vk.Sim(system, n, lo, hi, precision=precision, buffers=bufs, **kw)
    b = vk.Sim(system, n, lo, hi, precision=precision, **kw)
    for s in (a, b):
        s.set_state(U0)
        s.step(25)
    Ua = a.moments()
    assert np.array_equal(Ua, b.moments())
    # the state is in the caller's tensors, in the brick layout of vklb_device_state
    ptr = a.device_state()
    cur = [t.data_ptr() for t in bufs].index(ptr)
    p, nxb = a.p, a.info.pitch // 32
    dt = torch.float32 if precision == "fp32" else torch.float64
    f = bufs[cur][:need].view(dt).view(37, nxb, 5, p, 32)
    U = f.double().sum(dim=2).permute(2, 0, 1, 3).reshape(p, 37, nxb * 32)[:, :, :100].cpu().numpy()
    assert np.allclose(U, Ua, rtol=1e-6 if precision == "fp32" else 1e-13, atol=1e-6)
    with pytest.raises(vk.VKLBError) as e:
        a.set_form("moments")
    assert e.value.status == vk.ERR_UNSUPPORTED
    a.close()
    b.close()
    torch.cuda.synchronize()
    # the simulation freed nothing of the caller's: the tensors are still usable
    bufs[0].fill_(1)
    bufs[1].fill_(2)
    assert int(bufs[0].sum()) + int(bufs[1].sum()) == 3 * (need + 512)

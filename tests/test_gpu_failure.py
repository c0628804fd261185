"""Device-side failure detection without a GPU fault: the bounded mbarrier wait
that the bulk-copy step uses is made to run out (a barrier nothing arrives at,
a 1 ms limit); the device latches ERR_TIMEOUT in the error word, the host reads
VKLB_ERR_TIMEOUT, and the context stays usable for the next simulation.  (The
non-physical-state path is in test_gpu_parity.py.)"""
import time

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


def test_bounded_wait_times_out_and_context_survives(vk):
    t0 = time.perf_counter()
    assert vk.selftest_wait_timeout(1_000_000) == vk.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert vk.selftest_wait_timeout(100) == vk.ERR_ARG          # limit outside 1 us .. 100 ms
    sim = vk.Sim("swe", (64, 64), (0, 0), (1, 1), precision="fp32", omega=1.0, cfl=0.3)
    sim.set_state(inputs.swe_hump_2d(64, 0.5, 0.5, 0.5, 0.08))
    sim.step(5)
    U = sim.moments()
    assert np.isfinite(U).all()
    sim.close()


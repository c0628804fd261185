"""The seeded input generators (paper_2608_04283_b300/inputs.py): the device
(torch) evaluation of a served request's initial state equals the host one."""
import numpy as np
import torch

from paper_2608_04283_b300 import inputs


def test_request_initial_state_torch_matches_numpy():
    for r in inputs.serving_trace(count=12, seed=2, nmin=32, nmax=96, nstep=32):
        a = inputs.request_initial_state(r)
        b = inputs.request_initial_state_torch(r, torch, "cpu").numpy()
        assert a.shape == b.shape
        assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()

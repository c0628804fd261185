"""Pins of the oracle's bfloat16 storage model (reading R20): the rounding is
checked against closed-form ties and against torch's float32 -> bfloat16
conversion (a library routine); a simulation with bf16 storage keeps every
stored distribution representable, starts from the rounded f^eq, and departs
from the FP64 simulation by about the storage rounding, not more."""
import numpy as np
import pytest
import torch

from oracle import systems, vklb as ovklb
from paper_2608_04283_b300 import inputs

U8 = 2.0 ** -8


@pytest.mark.parametrize("x,want", [
    (1.0, 1.0),
    (1.0 + U8, 1.0),                          # tie between 1 and 1 + 2^-7: even significand
    (1.0 + 3 * U8, 1.0 + 2 ** -6),            # tie between 1 + 2^-7 and 1 + 2^-6: even
    (1.0 + U8 + 2 ** -30, 1.0 + 2 ** -7),     # just above the tie
    (1.0 + U8 - 2 ** -30, 1.0),               # just below
    (2.0 - 2 ** -9, 2.0),                     # rounds up into the next binade
    (-(1.0 + 3 * U8), -(1.0 + 2 ** -6)),      # symmetric in the sign
    (0.0, 0.0),
    (3.0e-5 * 2 ** -20, None),                # small normal value: only idempotence checked
    (1.0 / 3.0, 0.333984375),                 # 0.0101010101... -> 0.01010110 (8 bits)
])
def test_round_to_bf16_closed_forms(x, want):
    r = float(ovklb.round_to_bf16(x))
    if want is not None:
        assert r == want
    assert float(ovklb.round_to_bf16(r)) == r


def test_round_to_bf16_matches_torch():
    """On float32-representable values (one rounding on both sides) the result
    equals torch's round-to-nearest-even conversion bit for bit."""
    rng = np.random.default_rng(7)
    x = np.concatenate([
        rng.standard_normal(200000).astype(np.float32),
        (rng.uniform(-1, 1, 100000) * 10.0 ** rng.integers(-20, 20, 100000)).astype(np.float32),
        # exact ties and their float32 neighbours
        np.float32(1.0) + np.float32(U8) * np.arange(1, 512, 2, dtype=np.float32),
    ])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = ovklb.round_to_bf16(x.astype(np.float64))
    assert np.array_equal(got, want)


def test_rounded_values_have_eight_significant_bits():
    x = np.random.default_rng(3).standard_normal(10000) * 37.0
    r = ovklb.round_to_bf16(x)
    m, _ = np.frexp(r)
    assert np.array_equal(m * 256.0, np.round(m * 256.0))
    assert np.all(np.abs(r - x) <= U8 * np.abs(x) * (1 + 1e-15))   # unit roundoff 2^-8


@pytest.mark.parametrize("omega", [1.0, 2.0])
def test_bf16_storage_simulation(omega):
    n = (24, 20)
    U0 = np.ascontiguousarray(inputs.isentropic_vortex(24, lo=0.0, hi=10.0)[:, :20, :])
    lo, hi = (0.0, 0.0), (10.0, 10.0 * 20 / 24)
    sims = {}
    for st in ("fp64", "bf16"):
        s = ovklb.Sim(systems.Euler(1.4, 2), n, lo, hi, omega=omega, nu=0.3, storage=st)
        s.set_state(U0)
        sims[st] = s
    b, d = sims["bf16"], sims["fp64"]
    assert np.array_equal(b.f, ovklb.round_to_bf16(d.f))          # rounded f^eq of the same U0
    assert b.xi == d.xi                                            # xi_0 from U0 itself
    for s in sims.values():
        s.run(10)
    assert np.array_equal(ovklb.round_to_bf16(b.f), b.f)
    assert not np.array_equal(b.f, d.f)
    # ten steps of storage rounding: far below ten unit roundoffs of the state
    err = np.abs(b.moments() - d.moments()).reshape(4, -1).sum(axis=1)
    scale = np.abs(d.moments()).reshape(4, -1).sum(axis=1)
    rel = err / scale
    assert np.all(rel < 10 * U8) and np.all(rel > 1e-5), rel


def test_bf16_storage_rejects_unknown():
    with pytest.raises(ValueError):
        ovklb.Sim(systems.Euler(1.4, 2), (8, 8), (0, 0), (1, 1), storage="fp16")

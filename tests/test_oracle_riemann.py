"""Pins for oracle/riemann.py: jump conditions, Riemann invariants and the
textbook Sod star state (tests/golden/textbook_riemann.json)."""
import json
import os

import numpy as np

from oracle import riemann

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_sod_star_state_textbook():
    d = json.load(open(os.path.join(GOLD, "textbook_riemann.json")))["sod"]
    ps, us = riemann.euler_star(d["rho"][0], d["u"][0], d["p"][0], d["rho"][1], d["u"][1], d["p"][1], d["gamma"])
    assert round(ps, 5) == d["p_star"]
    assert round(us, 5) == d["u_star"]
    out = riemann.euler_sample(d["rho"][0], d["u"][0], d["p"][0], d["rho"][1], d["u"][1], d["p"][1],
                               d["gamma"], np.array([0.0, 0.25]), 0.2)
    assert round(out[0, 0], 5) == d["rho_star_left"]      # between rarefaction tail and contact
    assert round(out[0, 1], 5) == d["rho_star_right"]     # between contact and shock


def test_euler_rankine_hugoniot_right_shock():
    g = 1.4
    rL, uL, pL, rR, uR, pR = 1.0, 0.0, 1.0, 0.125, 0.0, 0.1
    ps, us = riemann.euler_star(rL, uL, pL, rR, uR, pR, g)
    g1 = (g - 1) / (g + 1)
    rs = rR * (ps / pR + g1) / (g1 * ps / pR + 1)
    S = (rs * us - rR * uR) / (rs - rR)                   # mass jump gives S
    E = lambda r, u, p: p / (g - 1) + 0.5 * r * u * u
    mom = lambda r, u, p: r * u * u + p
    en = lambda r, u, p: u * (E(r, u, p) + p)
    assert abs(S * (rs * us - rR * uR) - (mom(rs, us, ps) - mom(rR, uR, pR))) < 1e-12
    assert abs(S * (E(rs, us, ps) - E(rR, uR, pR)) - (en(rs, us, ps) - en(rR, uR, pR))) < 1e-12


def test_euler_rarefaction_isentropic_and_invariant():
    g = 1.4
    x = np.linspace(-0.5, 0.5, 2001)
    out = riemann.euler_sample(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g, x, 0.2)
    rho, u, p = out
    fan = (x > -0.5) & (x < -0.01) & (np.abs(np.gradient(rho)) > 0)
    s = p / rho ** g
    a = np.sqrt(g * p / rho)
    assert np.allclose(s[fan], 1.0, rtol=1e-12)
    assert np.allclose((u + 2 * a / (g - 1))[fan], 2 * np.sqrt(g) / (g - 1), rtol=1e-12)


def test_swe_dam_break_jump_and_invariant():
    g = 9.81
    hL, hR = 2.0, 1.0
    hs, us = riemann.swe_star(hL, 0.0, hR, 0.0, g)
    S = riemann.swe_shock_speed(hR, 0.0, hs, us, 1)
    # momentum jump: S [hu] = [h u^2 + g h^2 / 2]
    assert abs(S * (hs * us) - (hs * us * us + 0.5 * g * hs * hs - 0.5 * g * hR * hR)) < 1e-12
    # left rarefaction: u + 2 sqrt(g h) constant
    assert abs(us + 2 * np.sqrt(g * hs) - 2 * np.sqrt(g * hL)) < 1e-12
    x = np.linspace(0.0, 1.0, 4001)
    h, u = riemann.swe_sample(hL, 0.0, hR, 0.0, g, x, 0.1, x0=0.5)
    fan = (h < hL - 1e-9) & (h > hs + 1e-9)
    assert np.allclose(u[fan] + 2 * np.sqrt(g * h[fan]), 2 * np.sqrt(g * hL), rtol=1e-12)


def test_swe_two_shock_compression():
    """Table 1 compression data (hu = +-1, h = 1, g = 1): symmetric two-shock
    solution with u* = 0 and both momentum jumps satisfied."""
    hs, us = riemann.swe_star(1.0, 1.0, 1.0, -1.0, 1.0)
    assert abs(us) < 1e-14 and hs > 1.0
    S = riemann.swe_shock_speed(1.0, -1.0, hs, us, 1)
    assert abs(S * (hs * us - (-1.0)) - (hs * us * us + 0.5 * hs * hs - (1.0 + 0.5))) < 1e-12

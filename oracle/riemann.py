"""Exact Riemann solutions used to pin the oracle (Sec. 5.1 Table 1, Sec. 5.2
Table 2; the paper compares its Riemann runs with these exact solutions).

Shallow water: two-wave solution (shock or rarefaction on each side) found by
Newton iteration on the depth function  f_L(h) + f_R(h) + u_R - u_L = 0  with
  f_K(h) = 2 (sqrt(g h) - sqrt(g h_K))                          h <= h_K
         = (h - h_K) sqrt(g (h + h_K) / (2 h h_K))              h >  h_K.
Euler (ideal gas): the classical pressure-function solver, with
  f_K(p) = (p - p_K) sqrt(A_K / (p + B_K))                       p >  p_K
         = 2 a_K / (gamma - 1) ((p / p_K)^((gamma-1)/(2 gamma)) - 1)  p <= p_K
  A_K = 2 / ((gamma + 1) rho_K),  B_K = (gamma - 1) / (gamma + 1) p_K.
Both are sampled at x/t.  Test infrastructure only.

Pins (tests/test_oracle_riemann.py): Rankine-Hugoniot jump conditions across the
computed shocks, Riemann invariants across the rarefactions, and the textbook
star state of the Sod problem.
"""
import numpy as np


# ----------------------------------------------------------------- shallow water
def _swe_fK(h, hK, g):
    if h <= hK:
        return 2.0 * (np.sqrt(g * h) - np.sqrt(g * hK)), g / np.sqrt(g * h)
    s = np.sqrt(0.5 * g * (h + hK) / (h * hK))
    ds = 0.25 * g / (s * h * hK) * (1.0 - (h + hK) / h)
    return (h - hK) * s, s + (h - hK) * ds


def swe_star(hL, uL, hR, uR, g):
    h = 0.5 * (hL + hR)
    for _ in range(200):
        fl, dl = _swe_fK(h, hL, g)
        fr, dr = _swe_fK(h, hR, g)
        F = fl + fr + uR - uL
        hn = max(h - F / (dl + dr), 1e-12)
        if abs(hn - h) <= 1e-15 * h:
            h = hn
            break
        h = hn
    fl, _ = _swe_fK(h, hL, g)
    fr, _ = _swe_fK(h, hR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fr - fl)
    return h, u


def swe_sample(hL, uL, hR, uR, g, x, t, x0=0.0):
    """Exact (h, u) at positions x and time t > 0 for the dam-break data."""
    hs, us = swe_star(hL, uL, hR, uR, g)
    aL, aR, as_ = np.sqrt(g * hL), np.sqrt(g * hR), np.sqrt(g * hs)
    s = (np.asarray(x, float) - x0) / t
    h = np.empty_like(s)
    u = np.empty_like(s)
    for i, si in enumerate(s):
        if si <= us:  # left of contact
            if hs > hL:  # left shock
                SL = uL - aL * np.sqrt(0.5 * (hs + hL) * hs / hL ** 2)
                h[i], u[i] = (hL, uL) if si <= SL else (hs, us)
            else:
                head, tail = uL - aL, us - as_
                if si <= head:
                    h[i], u[i] = hL, uL
                elif si >= tail:
                    h[i], u[i] = hs, us
                else:
                    u[i] = (uL + 2.0 * aL + 2.0 * si) / 3.0
                    a = (uL + 2.0 * aL - si) / 3.0
                    h[i] = a * a / g
        else:
            if hs > hR:
                SR = uR + aR * np.sqrt(0.5 * (hs + hR) * hs / hR ** 2)
                h[i], u[i] = (hR, uR) if si >= SR else (hs, us)
            else:
                head, tail = uR + aR, us + as_
                if si >= head:
                    h[i], u[i] = hR, uR
                elif si <= tail:
                    h[i], u[i] = hs, us
                else:
                    u[i] = (uR - 2.0 * aR + 2.0 * si) / 3.0
                    a = (-uR + 2.0 * aR + si) / 3.0
                    h[i] = a * a / g
    return h, u


def swe_shock_speed(hK, uK, hs, us, side):
    """Shock speed from the mass jump: S = (h* u* - hK uK) / (h* - hK)."""
    return (hs * us - hK * uK) / (hs - hK)


# ------------------------------------------------------------------------ Euler
def _eul_fK(p, rhoK, pK, gamma):
    aK = np.sqrt(gamma * pK / rhoK)
    if p > pK:
        A = 2.0 / ((gamma + 1.0) * rhoK)
        B = (gamma - 1.0) / (gamma + 1.0) * pK
        s = np.sqrt(A / (p + B))
        return (p - pK) * s, s * (1.0 - 0.5 * (p - pK) / (p + B))
    e = (gamma - 1.0) / (2.0 * gamma)
    return 2.0 * aK / (gamma - 1.0) * ((p / pK) ** e - 1.0), (p / pK) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rhoK * aK)


def euler_star(rhoL, uL, pL, rhoR, uR, pR, gamma):
    p = max(0.5 * (pL + pR), 1e-12)
    for _ in range(500):
        fl, dl = _eul_fK(p, rhoL, pL, gamma)
        fr, dr = _eul_fK(p, rhoR, pR, gamma)
        F = fl + fr + uR - uL
        pn = p - F / (dl + dr)
        if pn <= 0:
            pn = 0.5 * p
        if abs(pn - p) <= 1e-15 * p:
            p = pn
            break
        p = pn
    fl, _ = _eul_fK(p, rhoL, pL, gamma)
    fr, _ = _eul_fK(p, rhoR, pR, gamma)
    return p, 0.5 * (uL + uR) + 0.5 * (fr - fl)


def euler_sample(rhoL, uL, pL, rhoR, uR, pR, gamma, x, t, x0=0.0):
    """Exact (rho, u, p) at x, t for 1D Euler Riemann data."""
    ps, us = euler_star(rhoL, uL, pL, rhoR, uR, pR, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    aL, aR = np.sqrt(gamma * pL / rhoL), np.sqrt(gamma * pR / rhoR)
    s = (np.asarray(x, float) - x0) / t
    out = np.empty((3, s.size))
    for i, si in enumerate(s):
        if si <= us:
            if ps > pL:
                rs = rhoL * (ps / pL + g1) / (g1 * ps / pL + 1.0)
                SL = uL - aL * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pL + (gamma - 1.0) / (2.0 * gamma))
                out[:, i] = (rhoL, uL, pL) if si <= SL else (rs, us, ps)
            else:
                rs = rhoL * (ps / pL) ** (1.0 / gamma)
                as_ = aL * (ps / pL) ** ((gamma - 1.0) / (2.0 * gamma))
                if si <= uL - aL:
                    out[:, i] = (rhoL, uL, pL)
                elif si >= us - as_:
                    out[:, i] = (rs, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) + g1 / aL * (uL - si)
                    out[:, i] = (rhoL * c ** (2.0 / (gamma - 1.0)),
                                 2.0 / (gamma + 1.0) * (aL + 0.5 * (gamma - 1.0) * uL + si),
                                 pL * c ** (2.0 * gamma / (gamma - 1.0)))
        else:
            if ps > pR:
                rs = rhoR * (ps / pR + g1) / (g1 * ps / pR + 1.0)
                SR = uR + aR * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pR + (gamma - 1.0) / (2.0 * gamma))
                out[:, i] = (rhoR, uR, pR) if si >= SR else (rs, us, ps)
            else:
                rs = rhoR * (ps / pR) ** (1.0 / gamma)
                as_ = aR * (ps / pR) ** ((gamma - 1.0) / (2.0 * gamma))
                if si >= uR + aR:
                    out[:, i] = (rhoR, uR, pR)
                elif si <= us + as_:
                    out[:, i] = (rs, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) - g1 / aR * (uR - si)
                    out[:, i] = (rhoR * c ** (2.0 / (gamma - 1.0)),
                                 2.0 / (gamma + 1.0) * (-aR + 0.5 * (gamma - 1.0) * uR + si),
                                 pR * c ** (2.0 * gamma / (gamma - 1.0)))
    return out

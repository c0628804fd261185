"""Pins for oracle/splitting.py (Sec. 2.2 Eqs. 11, 15-18; Sec. 3.1 Eqs. 25-27)."""
import numpy as np
import pytest

from oracle import systems, splitting
from paper_2608_04283_b300 import inputs

CASES = [("swe", 1, {"g": 9.81}), ("swe", 2, {"g": 9.81}), ("euler", 1, {"gamma": 1.4}),
         ("euler", 2, {"gamma": 1.4}), ("mhd_glm", 2, {"gamma": 5.0 / 3.0, "ch": 6.0}),
         ("mhd_glm", 2, {"gamma": 5.0 / 3.0, "ch": 1.0})]


def _states(kind, dim, kw, n=300, seed=11):
    return inputs.random_states(kind, n, seed=seed, dim=dim, gamma=kw.get("gamma", 1.4))


@pytest.mark.parametrize("kind,dim,kw", CASES)
@pytest.mark.parametrize("k", [0.5, 2.0, 7.0])
def test_matrix_function_equals_eig_route(kind, dim, kw, k):
    """alpha(A) F equals the literal sum_j alpha(lambda_j) phi_j r_j with
    phi = P^-1 F (Eqs. 16, 25, 26) and alpha of Eq. (27); F- is checked
    against sum_j (1 - alpha_j) phi_j r_j independently."""
    s = systems.make(kind, dim, **kw)
    U = _states(kind, dim, kw)
    for d in range(dim):
        Fp, Fm = splitting.split_weighted(s, U, d, k)
        Fp2, _ = splitting.split_eig(s, U, d, lambda lam, lm: splitting.sigmoid_weight(lam, lm, k))
        Fm2, _ = splitting.split_eig(s, U, d, lambda lam, lm: 1.0 - splitting.sigmoid_weight(lam, lm, k))
        scale = np.abs(s.flux(U, d)).max(axis=0) + 1.0
        assert np.max(np.abs(Fp - Fp2) / scale) < 1e-11
        assert np.max(np.abs(Fm - Fm2) / scale) < 1e-11


@pytest.mark.parametrize("kind,dim,kw", CASES)
def test_k_zero_is_half_flux(kind, dim, kw):
    """Sec. 3.1: alpha(0) = 1/2; with k = 0 every weight is 1/2, F+ = F- = F/2,
    which with c = 1/3 (1D) or 1/5 (2D) gives the centered set (Eqs. 8-10, 39)."""
    s = systems.make(kind, dim, **kw)
    U = _states(kind, dim, kw, n=50)
    for d in range(dim):
        Fp, Fm = splitting.split_eig(s, U, d, lambda lam, lm: splitting.sigmoid_weight(lam, lm, 0.0))
        F = s.flux(U, d)
        assert np.allclose(Fp, 0.5 * F, rtol=1e-11, atol=1e-11)
        assert np.allclose(Fm, 0.5 * F, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("kind,dim,kw", CASES[:4])
def test_large_k_tends_to_discontinuous(kind, dim, kw):
    """Sec. 3.1: F+- -> F^(+-) of Eqs. (17)-(18) as k -> infinity."""
    s = systems.make(kind, dim, **kw)
    U = _states(kind, dim, kw, n=400, seed=12)
    for d in range(dim):
        A = splitting.jacobian(s, U, d)
        lam = np.real(np.linalg.eigvals(A))
        gap = np.min(np.abs(lam), axis=1) / np.max(np.abs(lam), axis=1)
        ok = gap > 0.1
        # The matrix-function route is pinned to the eig route at moderate k;
        # at k = 300 E = expm(k A / max|lambda|) spans e^+-300 and (E + I) is
        # numerically singular, so the limit is taken on the eig route.
        Fw, _ = splitting.split_eig(s, U[:, ok], d,
                                    lambda lam, lm: splitting.sigmoid_weight(lam, lm, 300.0))
        Fd, _ = splitting.split_discontinuous(s, U[:, ok], d)
        scale = np.abs(s.flux(U[:, ok], d)).max(axis=0) + 1.0
        assert ok.sum() > 20
        assert np.max(np.abs(Fw - Fd) / scale) < 1e-9


def _steger_warming(U, gamma, d):
    """Textbook Steger-Warming (1981) split of the 2D Euler flux, written out:
    F+- = rho/(2 gamma) [ l1 (1, u-a, v, H-ua) + 2(gamma-1) l2 (1, u, v, |u|^2/2)
                          + l3 (1, u+a, v, H+ua) ]  with l = max/min(lambda, 0)
    (x direction; y by symmetry)."""
    rho = U[0]
    vel = [U[1] / rho, U[2] / rho]
    p = (gamma - 1) * (U[3] - 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2))
    a = np.sqrt(gamma * p / rho)
    H = (U[3] + p) / rho
    un, ut = vel[d], vel[1 - d]
    lam = [un - a, un, un + a]
    out = []
    for sgn in (1, -1):
        l = [np.maximum(x, 0) if sgn > 0 else np.minimum(x, 0) for x in lam]
        mass = l[0] + 2 * (gamma - 1) * l[1] + l[2]
        mn = l[0] * (un - a) + 2 * (gamma - 1) * l[1] * un + l[2] * (un + a)
        mt = ut * mass
        en = l[0] * (H - un * a) + (gamma - 1) * l[1] * (un * un + ut * ut) + l[2] * (H + un * a)
        comps = [mass, mn, mt, en] if d == 0 else [mass, mt, mn, en]
        out.append(rho / (2 * gamma) * np.stack(comps))
    return out


def test_euler_discontinuous_is_steger_warming():
    """Sec. 2.2 (after Eq. 18) and Thm 4.4: for Euler (homogeneous of degree one)
    the discontinuous split equals Steger-Warming P Lambda^+- P^-1 U."""
    g = 1.4
    e = systems.Euler(g, 2)
    U = inputs.random_states("euler", 300, seed=13, dim=2, gamma=g)
    for d in range(2):
        Fp, Fm = splitting.split_discontinuous(e, U, d)
        Sp, Sm = _steger_warming(U, g, d)
        scale = np.abs(e.flux(U, d)).max(axis=0) + 1.0
        assert np.max(np.abs(Fp - Sp) / scale) < 1e-11
        assert np.max(np.abs(Fm - Sm) / scale) < 1e-11


def test_advection_weight_is_scalar_sigmoid():
    """For F = a u the split is alpha(a) a u with alpha = 1/(1 + e^{-k sign(a)}) (Eq. 27)."""
    for a in (2.0, -0.7):
        s = systems.Advection(a=(a,), dim=1)
        U = inputs.random_states("advection", 20, seed=14)
        Fp, Fm = splitting.split_weighted(s, U, 0, 2.0)
        al = 1.0 / (1.0 + np.exp(-2.0 * np.sign(a)))
        assert np.allclose(Fp, al * a * U, rtol=1e-14, atol=1e-15)
        assert np.allclose(Fm, (1 - al) * a * U, rtol=1e-13, atol=1e-15)


def test_weighted_split_is_continuous_in_state():
    """Sec. 3.1: the weighted split varies continuously where an eigenvalue crosses
    zero (the discontinuous one jumps)."""
    s = systems.ShallowWater(9.81, 1)
    h = np.full(2, 1.0)
    c = np.sqrt(9.81)
    u = np.array([c - 1e-7, c + 1e-7])      # u - c crosses zero
    U = np.stack([h, h * u])
    Fw, _ = splitting.split_weighted(s, U, 0, 2.0)
    Fd, _ = splitting.split_discontinuous(s, U, 0)
    assert np.max(np.abs(Fw[:, 0] - Fw[:, 1])) < 1e-5
    assert np.max(np.abs(Fd[:, 0] - Fd[:, 1])) > 1e-3

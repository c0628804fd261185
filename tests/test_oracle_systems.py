"""Pins for oracle/systems.py: fluxes and wave speeds against properties the
paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

from oracle import systems, splitting
from paper_2608_04283_b300 import inputs


def _eig_max(sysm, U, d):
    A = splitting.jacobian(sysm, U, d)
    return np.max(np.abs(np.linalg.eigvals(A)), axis=1)


@pytest.mark.parametrize("kind,dim,kw", [
    ("swe", 1, {}), ("swe", 2, {}), ("euler", 1, {"gamma": 1.4}), ("euler", 2, {"gamma": 1.4}),
    ("mhd_glm", 2, {"gamma": 5.0 / 3.0, "ch": 0.5}), ("mhd_glm", 2, {"gamma": 5.0 / 3.0, "ch": 9.0}),
])
def test_wave_speed_is_spectral_radius(kind, dim, kw):
    """Closed-form max_j |lambda_j| (Sec. 5.1: u +- sqrt(gh); Sec. 5.2: u +- a;
    MHD fast speed and +-c_h) equals the spectral radius of dF/dU."""
    sysm = systems.make(kind, dim, **kw)
    U = inputs.random_states(kind, 200, seed=1, dim=dim, gamma=kw.get("gamma", 1.4))
    for d in range(dim):
        ref = _eig_max(sysm, U, d)
        got = sysm.max_speed(U, d)
        assert np.allclose(got, ref, rtol=1e-9, atol=0), (d, np.abs(got - ref).max())


def test_swe_eigenvalues_u_pm_c():
    """Sec. 5.1: the characteristic speeds of Eq. (52) are u -+ sqrt(g h)."""
    s = systems.ShallowWater(g=9.81, dim=1)
    U = inputs.random_states("swe", 50, seed=2, dim=1)
    A = splitting.jacobian(s, U, 0)
    lam = np.sort(np.real(np.linalg.eigvals(A)), axis=1)
    u = U[1] / U[0]
    c = np.sqrt(9.81 * U[0])
    assert np.allclose(lam[:, 0], u - c, rtol=1e-12, atol=1e-12)
    assert np.allclose(lam[:, 1], u + c, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_euler_homogeneous_degree_one(dim):
    """Remark after Eq. (18) and proof of Thm 4.4: the Euler flux satisfies F = (dF/dU) U."""
    e = systems.Euler(1.4, dim)
    U = inputs.random_states("euler", 300, seed=3, dim=dim)
    for d in range(dim):
        A = splitting.jacobian(e, U, d)
        AU = np.einsum("nij,jn->in", A, U)
        F = e.flux(U, d)
        assert np.allclose(AU, F, rtol=1e-13, atol=1e-13)


def test_swe_not_homogeneous():
    """Remark after Thm 4.4: the shallow-water flux is not homogeneous of degree one."""
    s = systems.ShallowWater(9.81, 1)
    U = inputs.random_states("swe", 20, seed=4, dim=1)
    A = splitting.jacobian(s, U, 0)
    AU = np.einsum("nij,jn->in", A, U)
    assert np.abs(AU - s.flux(U, 0)).max() > 1e-3


def test_mhd_reduces_to_euler_without_field():
    """Eq. (58) with B = 0 and psi = 0 is the Euler flux of Eq. (54) (plus a z-velocity)."""
    g = 5.0 / 3.0
    m = systems.MHDGLM(g, ch=3.0)
    e = systems.Euler(g, 2)
    Ue = inputs.random_states("euler", 100, seed=5, dim=2, gamma=g)
    z = np.zeros_like(Ue[0])
    Um = np.stack([Ue[0], Ue[1], Ue[2], z, Ue[3], z, z, z, z])
    for d in range(2):
        Fm = m.flux(Um, d)
        Fe = e.flux(Ue, d)
        assert np.allclose(Fm[[0, 1, 2, 4]], Fe, rtol=1e-14, atol=1e-14)
        assert np.all(Fm[[3, 5, 6, 7, 8]] == 0)


def test_mhd_flux_components_by_hand():
    """Eq. (58) spelled out for one state, x direction."""
    g = 5.0 / 3.0
    ch = 2.5
    rho, u, v, w, p, bx, by, bz, psi = 1.3, 0.4, -0.7, 0.2, 0.9, 0.6, -0.3, 0.8, 0.05
    U = inputs.mhd_conserved(*(np.array([t]) for t in (rho, u, v, w, p, bx, by, bz, psi)), g)
    F = systems.MHDGLM(g, ch).flux(U, 0)[:, 0]
    E = p / (g - 1) + 0.5 * rho * (u * u + v * v + w * w) + 0.5 * (bx * bx + by * by + bz * bz)
    pt = p + 0.5 * (bx * bx + by * by + bz * bz)
    bu = bx * u + by * v + bz * w
    want = [rho * u, rho * u * u + pt - bx * bx, rho * u * v - bx * by, rho * u * w - bx * bz,
            (E + pt) * u - bu * bx, psi, u * by - bx * v, u * bz - bx * w, ch * ch * bx]
    assert np.allclose(F, want, rtol=1e-14, atol=1e-14)


def test_mhd_xy_swap_symmetry():
    """Swapping x <-> y in the state maps F^(1) to F^(2) with the components swapped."""
    m = systems.MHDGLM(5.0 / 3.0, ch=4.0)
    U = inputs.random_states("mhd_glm", 50, seed=6, dim=2, gamma=5.0 / 3.0)
    perm = [0, 2, 1, 3, 4, 6, 5, 7, 8]
    Fy = m.flux(U, 1)
    Fx_sw = m.flux(U[perm], 0)[perm]
    assert np.allclose(Fy, Fx_sw, rtol=1e-14, atol=1e-14)

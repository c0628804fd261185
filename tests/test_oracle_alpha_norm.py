"""Pins for the two readings of alpha's normaliser max_j |lambda_j| (Eq. 27),
which the paper does not place (reading R1): per cell and direction ("local")
or one grid-wide number per step ("global", the maximum that Eq. 29 divides by
nu).  No GPU.

The global reading is pinned through what fixes it independently of the oracle's
own code path:
  * the eigen route (Eqs. 16, 25, 26) with alpha = sigma(k lambda / Lambda)
    equals the matrix-function route given the same Lambda;
  * sigma(k lambda / Lambda) = sigma((k lambda_max / Lambda) lambda / lambda_max),
    so a cell's global split equals its local split with k scaled by
    lambda_max(cell) / Lambda -- with the wave speeds written out here in closed
    form, so that a wrong Lambda (per direction, divided by nu, taken from the
    landed xi) fails;
  * on a uniform state both readings coincide; the moment constraints (Eqs. 3,
    5) and periodic conservation (Thm 4.3) hold under either.
The linear stability of each reading about a uniform state (the vortex's
background flow at omega = 2, a shallow-water state at rest at omega = 1) is
computed from the oracle's equilibria and recorded as findings.
"""
import numpy as np
import pytest

from oracle import riemann, splitting, systems, vklb
from paper_2608_04283_b300 import inputs

V2 = np.array([[1, 0], [-1, 0], [0, 0], [0, 1], [0, -1]])


def _euler_speed(U, d, gamma=1.4):
    """|u_d| + a, a = sqrt(gamma p / rho): the largest Euler wave speed along d."""
    rho = U[0]
    u = U[1 + d] / rho
    ke = sum(U[1 + i] ** 2 for i in range(U.shape[0] - 2)) / rho
    p = (gamma - 1.0) * (U[-1] - 0.5 * ke)
    return np.abs(u) + np.sqrt(gamma * p / rho)


def _swe_speed(U, d, g=9.81):
    """|u_d| + sqrt(g h)."""
    return np.abs(U[1 + d] / U[0]) + np.sqrt(g * U[0])


@pytest.mark.parametrize("kind,dim,kw", [("swe", 1, {"g": 9.81}), ("swe", 2, {"g": 9.81}),
                                         ("euler", 1, {"gamma": 1.4}), ("euler", 2, {"gamma": 1.4}),
                                         ("mhd_glm", 2, {"gamma": 5 / 3, "ch": 1.0})])
def test_global_normaliser_matrix_function_equals_eig_route(kind, dim, kw):
    s = systems.make(kind, dim, **kw)
    U = inputs.random_states(kind, 200, seed=41, dim=dim, gamma=kw.get("gamma", 1.4))
    lam = 1.3 * max(float(np.max(s.max_speed(U, d))) for d in range(dim))
    for d in range(dim):
        Fp, _ = splitting.split_weighted(s, U, d, 2.0, lam_norm=lam)
        Fe, _ = splitting.split_eig(s, U, d, lambda l, lm: splitting.sigmoid_weight(l, lm, 2.0), lam_norm=lam)
        scale = np.abs(s.flux(U, d)).max(axis=0) + 1.0
        assert np.max(np.abs(Fp - Fe) / scale) < 1e-11


@pytest.mark.parametrize("kind,speed", [("euler", _euler_speed), ("swe", _swe_speed)])
def test_global_equals_local_with_scaled_k(kind, speed):
    """Per cell: alpha(lambda / Lambda; k) = alpha(lambda / lambda_max; k lambda_max / Lambda).
    The Sim's global equilibria on a 2D grid equal Eq. (41) built from per-cell
    local splits with that scaled k, where Lambda = max over the grid and BOTH
    directions of the closed-form speed."""
    n = (6, 5)
    s = systems.make(kind, 2)
    U = inputs.random_states(kind, n[0] * n[1], seed=42, dim=2, gamma=1.4).reshape(-1, n[1], n[0])
    sim = vklb.Sim(s, n, (0, 0), (1.2, 1.0), set_kind="weighted", c=0.05, k=2.0, alpha_norm="global")
    xi = 7.3
    got = sim.equilibrium(U, xi)
    Lam = max(float(np.max(speed(U, 0))), float(np.max(speed(U, 1))))
    Uf = U.reshape(U.shape[0], -1)
    parts = []
    for d in range(2):
        lm = speed(Uf, d)
        Fp = np.empty_like(Uf)
        for i in range(Uf.shape[1]):
            Fp[:, i] = splitting.split_weighted(s, Uf[:, i:i + 1], d, 2.0 * lm[i] / Lam)[0][:, 0]
        F = np.real(s.flux(Uf, d))
        parts += [Fp, F - Fp]
    want = vklb.equilibrium_2d(Uf, *parts, xi, 0.05).reshape(got.shape)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
    # and the two readings differ on this grid
    loc = vklb.Sim(s, n, (0, 0), (1.2, 1.0), c=0.05, k=2.0, alpha_norm="local").equilibrium(U, xi)
    assert np.max(np.abs(loc - got)) > 1e-4


def test_uniform_state_both_readings_agree():
    """Where every cell's own maximum along each direction is the grid-wide one
    (a uniform state with |u| = |v|) the two readings are the same scheme (to
    rounding: after a step the two directions' maxima can differ by an ulp)."""
    s = systems.Euler(1.4, 2)
    U = np.broadcast_to(inputs.euler_conserved(np.array(1.0), np.array(0.6), np.array(-0.6), np.array(1.0),
                                               1.4)[:, None, None], (4, 8, 8)).copy()
    runs = []
    for norm in ("local", "global"):
        sim = vklb.Sim(s, (8, 8), (0, 0), (1, 1), omega=1.7, nu=0.5, alpha_norm=norm)
        sim.set_state(U)
        sim.run(3)
        runs.append(sim.f)
    assert np.allclose(runs[0], runs[1], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("kind,dim", [("swe", 1), ("euler", 2), ("mhd_glm", 2)])
def test_global_reading_moments_and_conservation(kind, dim):
    """Eqs. (3), (5) and Thm 4.3 hold under the global reading too."""
    if kind == "swe":
        s = systems.ShallowWater(9.81, 1)
        x = inputs.cell_centers(40, 0, 1)
        h = 1 + 0.3 * np.exp(-80 * (x - 0.4) ** 2)
        U = np.stack([h, 0.5 * h])
        sim = vklb.Sim(s, (40,), (0,), (1,), omega=1.0, nu=0.6, alpha_norm="global")
    elif kind == "euler":
        s = systems.Euler(1.4, 2)
        U = inputs.isentropic_vortex(16)
        sim = vklb.Sim(s, (16, 16), (0, 0), (10, 10), omega=2.0, nu=0.3, alpha_norm="global")
    else:
        s = systems.MHDGLM(5 / 3, dim=2)
        U = inputs.orszag_tang(12)
        sim = vklb.Sim(s, (12, 12), (0, 0), (2 * np.pi, 2 * np.pi), omega=1.0, nu=0.3, alpha_norm="global")
    sim.set_state(U)
    xi = sim.xi
    feq = sim.f
    assert np.allclose(feq.sum(0), U, rtol=1e-13, atol=1e-13)
    vel = np.array([[1], [0], [-1]]) if dim == 1 else V2
    for d in range(dim):
        mom = np.tensordot(vel[:, d] * xi, feq, axes=(0, 0))
        assert np.allclose(mom, np.real(s.flux(U, d)), rtol=1e-12, atol=1e-12)
    t0 = sim.totals()
    sim.run(10)
    t1 = sim.totals()
    scale = np.abs(U).sum(axis=tuple(range(1, U.ndim))) * sim.dx ** dim
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.maximum(scale, scale.max() * 1e-3))


def test_characteristic_boundary_uses_grid_normaliser():
    """1D characteristic boundaries (Eq. 36): the boundary nodes take
    f^eq(U_b^{n+1}) with alpha normalised by the whole grid's max |lambda| of
    U^{n+1}, not by the two boundary states' own."""
    s = systems.ShallowWater(9.81, 1)
    x = inputs.cell_centers(32, 0, 1)
    h = 1 + 0.8 * np.exp(-60 * (x - 0.5) ** 2)       # the fastest waves sit in the middle
    U0 = np.stack([h, 0.2 * h])
    sim = vklb.Sim(s, (32,), (0,), (1,), bc="characteristic", omega=1.0, nu=0.6, alpha_norm="global")
    sim.set_state(U0)
    sim.step()
    Un = sim.moments()
    Lam = float(np.max(_swe_speed(Un, 0)))
    assert Lam > 1.05 * max(_swe_speed(Un[:, [0]], 0)[0], _swe_speed(Un[:, [-1]], 0)[0])
    for b in (0, -1):
        ub = Un[:, b:b + 1] if b == 0 else Un[:, b:]
        Fp, Fm = splitting.split_weighted(s, ub, 0, 2.0, lam_norm=Lam)
        want = vklb.equilibrium_1d(ub, Fp, Fm, sim.xi, 0.05)[:, :, 0]
        assert np.allclose(sim.f[:, :, b], want, rtol=1e-13, atol=1e-14)


# ---------------------------------------------------------------- findings
def _amplification(s, U0, xi, omega, lam_norm, c=0.05, k=2.0, nth=13):
    """Largest |eigenvalue| over wave numbers of the D2Q5 scheme (Eqs. 41-43)
    linearised about the uniform state U0: per mode the 5p x 5p map
    f_q <- e^{-i theta.m_q} [(1 - omega) f_q + omega M_q sum_r f_r] with
    M_q = d f^eq_q / dU (central differences of the oracle's equilibria)."""
    p = len(U0)

    def feq(U):
        Uc = U.reshape(-1, 1)
        parts = []
        for d in range(2):
            Fp, Fm = splitting.split_weighted(s, Uc, d, k, lam_norm=lam_norm)
            parts += [Fp, Fm]
        return vklb.equilibrium_2d(Uc, *parts, xi, c)[:, :, 0]

    M = np.zeros((5, p, p))
    for j in range(p):
        e = np.zeros(p)
        e[j] = 1e-6 * max(1.0, abs(U0[j]))
        M[:, :, j] = (feq(U0 + e) - feq(U0 - e)) / (2 * e[j])
    worst = 0.0
    for tx in np.linspace(0, np.pi, nth):
        for ty in np.linspace(-np.pi, np.pi, 2 * nth - 1):
            G = np.zeros((5 * p, 5 * p), complex)
            for q in range(5):
                blk = np.tile(omega * M[q], (1, 5)).astype(complex)
                blk[:, q * p:(q + 1) * p] += (1 - omega) * np.eye(p)
                G[q * p:(q + 1) * p] = np.exp(-1j * (tx * V2[q][0] + ty * V2[q][1])) * blk
            worst = max(worst, float(np.abs(np.linalg.eigvals(G)).max()))
    return worst


def test_advection_neutral_at_omega2():
    """Scalar advection (both readings coincide) is neutrally stable at
    omega = 2: the amplification factor is 1 for every mode."""
    s = systems.Advection((1.0, 0.5), 2)
    g = _amplification(s, np.array([1.0]), 1.0 / 0.3, 2.0, None)
    assert abs(g - 1.0) < 1e-9


def test_vortex_background_growth_by_reading():
    """A finding: about the vortex's background flow (rho = 1, u = v = 1, p = 1)
    with the vortex's lattice speed xi = 2.928 / 0.3 (Sec. 5.2: CFL 0.3,
    omega = 2) the linearised scheme grows under both readings, but at about
    1.023 per step with the local normaliser (x 2e19 over the 2,000 steps of
    N = 1024, T = 2) against 1.005 with the global one (x 4e4).  omega = 1.9
    is stable under both."""
    s = systems.Euler(1.4, 2)
    U0 = inputs.euler_conserved(np.array(1.0), np.array(1.0), np.array(1.0), np.array(1.0), 1.4)
    xi = 2.928 / 0.3
    gl = _amplification(s, U0, xi, 2.0, None)
    gg = _amplification(s, U0, xi, 2.0, 2.928)
    assert 1.015 < gl < 1.03
    assert 1.0 < gg < 1.007
    assert _amplification(s, U0, xi, 1.9, None, nth=7) < 1 + 1e-8
    assert _amplification(s, U0, xi, 1.9, 2.928, nth=7) < 1 + 1e-8


def _rest_growth(g, h, xi, lam):
    """Largest amplification of the D1Q3 scheme at omega = 1 (Thm 4.2's form)
    linearised about the shallow-water state (h, 0) at rest, with the true
    Jacobian d(alpha(A) F)/dU of the oracle's split (central differences);
    lam = alpha's normaliser (None: the cell's own max |lambda|)."""
    s = systems.ShallowWater(g, 1)
    U0 = np.array([h, 0.0])

    def Fp(U):
        return splitting.split_weighted(s, U.reshape(2, 1), 0, 2.0, lam_norm=lam)[0][:, 0]
    J = np.zeros((2, 2))
    for j in range(2):
        e = np.zeros(2)
        e[j] = 1e-7
        J[:, j] = (Fp(U0 + e) - Fp(U0 - e)) / 2e-7
    A = splitting.jacobian(s, U0.reshape(2, 1), 0)[0]
    worst = 0.0
    for th in np.linspace(0.0, np.pi, 181):
        G = np.eye(2) * (1 - 0.1 * (1 - np.cos(th))) - (J * (1 - np.exp(-1j * th))
                                                         + (A - J) * (np.exp(1j * th) - 1)) / xi
        worst = max(worst, np.abs(np.linalg.eigvals(G)).max())
    return worst


def test_rest_state_growth_by_reading():
    """A finding: the checkerboard growth of the weighted set in a fluid at rest
    (tests/test_oracle_convergence.py) is the same under both readings where the
    resting state itself sets the grid-wide maximum (at rest
    d(lambda / lambda_max)/d(hu) = 1 / c either way), but where a faster state
    elsewhere sets it the global reading weakens it: Table 1's standard dam
    break (h = 3 | 1, g = 1, CFL 0.9; the star state's u + c = 2.104 sets the
    maximum) grows 1.20 a step at its left state with the per-cell normaliser
    and 1.034 with the grid-wide one -- the run that converges to N = 4096
    under the global reading and degrades from N = 1024 under the local one."""
    c = np.sqrt(9.81 * 2.0)
    xi = c / 0.785
    gl, gg = _rest_growth(9.81, 2.0, xi, None), _rest_growth(9.81, 2.0, xi, c)
    assert gl > 1.25 and abs(gl - gg) < 1e-6
    x = np.linspace(-5.0, 5.0, 4001)
    h, u = riemann.swe_sample(3.0, 0.0, 1.0, 0.0, 1.0, x, 2.0)
    Lam = float(np.max(np.abs(u) + np.sqrt(h)))
    assert abs(Lam - 2.1045) < 1e-3
    xi = Lam / 0.9
    gl, gg = _rest_growth(1.0, 3.0, xi, None), _rest_growth(1.0, 3.0, xi, Lam)
    assert 1.15 < gl < 1.25 and 1.0 < gg < 1.05


def _mode_amplification(M, tx, ty, omega=2.0):
    """|largest eigenvalue| of the linearised D2Q5 step for one wave vector,
    with M the equilibrium Jacobians of _amplification."""
    p = M.shape[1]
    G = np.zeros((5 * p, 5 * p), complex)
    for q in range(5):
        blk = np.tile(omega * M[q], (1, 5)).astype(complex)
        blk[:, q * p:(q + 1) * p] += (1 - omega) * np.eye(p)
        G[q * p:(q + 1) * p] = np.exp(-1j * (tx * V2[q][0] + ty * V2[q][1])) * blk
    return float(np.abs(np.linalg.eigvals(G)).max())


def _eq_jacobians(s, U0, xi, lam_norm, c=0.05, k=2.0):
    p = len(U0)

    def feq(U):
        Uc = U.reshape(-1, 1)
        parts = []
        for d in range(2):
            Fp, Fm = splitting.split_weighted(s, Uc, d, k, lam_norm=lam_norm)
            parts += [Fp, Fm]
        return vklb.equilibrium_2d(Uc, *parts, xi, c)[:, :, 0]
    M = np.zeros((5, p, p))
    for j in range(p):
        e = np.zeros(p)
        e[j] = 1e-6 * max(1.0, abs(U0[j]))
        M[:, :, j] = (feq(U0 + e) - feq(U0 - e)) / (2 * e[j])
    return M


def test_entropy_wave_unstable_mode():
    """A finding: the entropy wave's background flow (Sec. 5.2, Eq. 55: rho = 1,
    u = v = 1, p = 1; CFL 0.3, omega = 2, c = 0.05, k = 2, grid-wide normaliser
    2.247 = max |u| + c over the wave) is linearly unstable through one family
    of modes along the flow's diagonal, theta_x = theta_y near 0.68 pi (about
    three cells a wavelength), which grows about 1.7 % a step: x 1e14 over the
    1,918 steps of the paper's N = 256, T = 1.  The same state moving along x
    (v = 0) and the fluid at rest are neutral, as are the diagonal modes far
    from that band.  With d F+/dU taken as alpha(A) A (the weights'
    derivatives dropped) the same equilibria are neutral on the whole
    diagonal, so the growth comes from the derivative of the weighted split
    itself, not from a reading of the lattice speed or of c."""
    s = systems.Euler(1.4, 2)
    lam = 2.247
    diag = inputs.euler_conserved(np.array(1.0), np.array(1.0), np.array(1.0), np.array(1.0), 1.4)
    along = inputs.euler_conserved(np.array(1.0), np.array(1.0), np.array(0.0), np.array(1.0), 1.4)
    M = _eq_jacobians(s, diag, lam / 0.3, lam)
    th = np.linspace(0.0, np.pi, 91)
    a = np.array([_mode_amplification(M, t, t) for t in th])
    i = int(np.argmax(a))
    assert 1.012 < a[i] < 1.025, a[i]
    assert 0.6 < th[i] / np.pi < 0.75, th[i]
    assert a[th < 0.4 * np.pi].max() < 1 + 1e-8                 # long waves: neutral
    Ma = _eq_jacobians(s, along, lam / 0.3, lam)
    assert max(_mode_amplification(Ma, t, t) for t in th[::5]) < 1 + 1e-8
    assert max(_mode_amplification(Ma, t, 0.0) for t in th[::5]) < 1 + 1e-8
    # the same equilibria with d F+/dU taken as alpha(A) A (Eq. 41 with the
    # weights frozen): neutral on the whole diagonal
    import scipy.linalg as sla
    xi, c, I = lam / 0.3, 0.05, np.eye(4)
    Mf = np.zeros((5, 4, 4))
    for d in range(2):
        A = splitting.jacobian(s, diag.reshape(4, 1), d)[0]
        E = sla.expm(2.0 * A / lam)
        alA = np.linalg.solve((E + I).T, E.T).T @ A           # alpha(A) A, alpha = E (E + I)^-1
        Mf[3 * d] = c * I + alA / xi
        Mf[3 * d + 1] = c * I - (A - alA) / xi
    Mf[2] = I - Mf[0] - Mf[1] - Mf[3] - Mf[4]
    assert max(_mode_amplification(Mf, t, t) for t in th) < 1 + 1e-8

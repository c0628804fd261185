"""Flux splittings F = F+ + F- (Sec. 2.2, Eq. (11)) used by the equilibria.

weighted (the paper's method, Sec. 3.1):
    phi = P^-1 F (Eq. 16),  psi^{j,+} = alpha(lambda_j) phi_j,
    psi^{j,-} = (1 - alpha(lambda_j)) phi_j (Eq. 25),
    F+ = sum_j psi^{j,+} r_j, F- = sum_j psi^{j,-} r_j (Eq. 26),
    alpha = 1 / (1 + exp(-k lambda / max_j |lambda_j|)) (Eq. 27).
  Since sum_j alpha(lambda_j) phi_j r_j = P alpha(Lambda) P^-1 F = alpha(A) F with
  A = dF/dU (Eq. 15), the oracle evaluates the matrix function directly:
      alpha(A) = E (E + I)^-1,  E = expm(k A / max_j |lambda_j|).
  This is exact (up to rounding) whatever eigenbasis one would pick, including
  repeated eigenvalues.  The paper leaves open over what max_j |lambda_j| is
  taken (reading R1 of oracle/vklb.py): by default per cell and per direction,
  from the closed-form wave speeds; given ``lam_norm``, that one number for
  every cell (the grid-wide maximum of Eq. 29).

discontinuous (Sec. 2.2, Eqs. (17)-(18)): phi split by the sign of lambda,
  lambda >= 0 -> "+".  Evaluated literally by eigen-decomposition.

centered (Sec. 2.2, Eqs. (8)-(10)): F+ = F- = F/2 (the k = 0 weighted split).

Test infrastructure only.

Parity pins (tests/test_oracle_splitting.py): F+ + F- = F; matrix-function route
equals the literal eig route (Eqs. 16, 25, 26) on random states; k = 0 gives F/2;
large k tends to the discontinuous split; for Euler (homogeneous of degree one) the
discontinuous split equals Steger-Warming P Lambda^+- P^-1 U in its textbook closed
form.
"""
import numpy as np
import scipy.linalg as sla

COMPLEX_STEP = 1e-30


def jacobian(system, U, d):
    """A[n] = dF^(d)/dU at every cell n, by complex-step differentiation:
    column j = Im F(U + i h e_j) / h.  F is rational in U, so this is exact to
    rounding.  U: [p, N] real.  Returns [N, p, p]."""
    p, N = U.shape
    A = np.empty((N, p, p))
    for j in range(p):
        Uc = U.astype(np.complex128)
        Uc[j] = Uc[j] + 1j * COMPLEX_STEP
        A[:, :, j] = (np.imag(system.flux(Uc, d)) / COMPLEX_STEP).T
    return A


def sigmoid_weight(lam, lam_max, k):
    """Eq. (27): alpha = 1 / (1 + exp(-k lambda / max_j |lambda_j|)); alpha(0) = 1/2."""
    lam_max = np.where(lam_max > 0, lam_max, 1.0)
    return 1.0 / (1.0 + np.exp(-k * lam / lam_max))


def split_weighted(system, U, d, k, lam_norm=None):
    """Weighted upwind splitting (Eqs. 25-27) as alpha(A) F.  U: [p, N].
    alpha's normaliser max_j |lambda_j| is the cell's own along d, or
    ``lam_norm`` (a positive number) for every cell.  Returns (F+, F-), each
    [p, N]."""
    F = np.real(system.flux(U, d))
    if k == 0.0:
        return 0.5 * F, 0.5 * F
    p, N = U.shape
    A = jacobian(system, U, d)
    if lam_norm is None:
        lam_max = system.max_speed(U, d)
    else:
        lam_max = np.full(N, float(lam_norm))
    lam_max = np.where(lam_max > 0, lam_max, 1.0)
    E = sla.expm(k * A / lam_max[:, None, None])
    EF = np.einsum("nij,jn->ni", E, F)
    Fp = np.linalg.solve(E + np.eye(p)[None], EF[:, :, None])[:, :, 0].T
    return Fp, F - Fp


def split_eig(system, U, d, weight, lam_norm=None):
    """Literal eigen route (Eqs. 15, 16, 25, 26): A = P Lambda P^-1,
    phi = P^-1 F, F+ = sum_j weight(lambda_j, max|lambda|) phi_j r_j.
    ``weight(lam, lam_max)`` returns the "+" fraction per eigenvalue; lam_max is
    the largest |eigenvalue| of the cell, or ``lam_norm`` when given.
    Only meaningful where A has a well-conditioned eigenbasis."""
    F = np.real(system.flux(U, d))
    A = jacobian(system, U, d)
    w, P = np.linalg.eig(A)
    lam = np.real(w)                                   # [N, p]
    if lam_norm is None:
        lam_max = np.max(np.abs(lam), axis=1)          # [N]
    else:
        lam_max = np.full(lam.shape[0], float(lam_norm))
    phi = np.linalg.solve(P, F.T[:, :, None].astype(P.dtype))[:, :, 0]
    wts = weight(lam, lam_max[:, None])
    Fp = np.real(np.einsum("nij,nj->ni", P, wts * phi)).T
    return Fp, F - Fp


def split_discontinuous(system, U, d):
    """Eqs. (17)-(18): lambda_j >= 0 -> F+, lambda_j < 0 -> F-."""
    return split_eig(system, U, d, lambda lam, lm: (lam >= 0).astype(float))


def split_centered(system, U, d):
    """Centered flux set: F+ = F- = F/2 (Eqs. 8-10 written as a splitting)."""
    F = np.real(system.flux(U, d))
    return 0.5 * F, 0.5 * F


def split(system, U, d, set_kind, k, lam_norm=None):
    if set_kind == "weighted":
        return split_weighted(system, U, d, k, lam_norm)
    if set_kind == "centered":
        return split_centered(system, U, d)
    if set_kind == "discontinuous":
        return split_discontinuous(system, U, d)
    raise ValueError(set_kind)

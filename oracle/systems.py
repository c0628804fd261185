"""Hyperbolic systems dU/dt + sum_d dF^(d)(U)/dx_d = 0 (Sec. 2.1, Eq. (1)).

Each system gives the physical flux F^(d)(U) and the largest characteristic speed
max_j |lambda_j| along direction d.  Fluxes are written with plain arithmetic so
they accept complex arrays (needed by the complex-step Jacobian in
``splitting``).  U has shape [p, ...] (fields first).

Test infrastructure only (see the package docstring).

Parity pins (tests/test_oracle_systems.py):
  * wave speeds equal the eigenvalues of the complex-step Jacobian (numpy.eigvals);
  * Euler flux is homogeneous of degree one, A U = F (Sec. 2.2, remark after Eq. 18);
  * MHD-GLM with B = 0, psi = 0 reduces to the Euler flux (Eq. 58 vs Eq. 54);
  * shallow-water flux matches Eq. (52); wave speeds u +- sqrt(g h) (Sec. 5.1).
"""
import numpy as np


def _re(x):
    return np.real(x)


class Advection:
    """Scalar linear advection F^(d) = a_d u (p = 1); a test system whose
    exact solution is a shift."""

    name = "advection"

    def __init__(self, a=(1.0, 0.0), dim=1):
        self.a = tuple(float(v) for v in a)
        self.dim = dim
        self.p = 1

    def flux(self, U, d):
        return self.a[d] * U

    def max_speed(self, U, d):
        return np.full(np.shape(U)[1:], abs(self.a[d]))


class ShallowWater:
    """Shallow water, Eq. (52): U = (h, hu) in 1D, (h, hu, hv) in 2D.
    Wave speeds u_d +- sqrt(g h) (Sec. 5.1) and u_d (2D shear wave)."""

    name = "swe"

    def __init__(self, g=9.81, dim=1):
        self.g = float(g)
        self.dim = dim
        self.p = 2 if dim == 1 else 3

    def flux(self, U, d):
        g = self.g
        h = U[0]
        if self.dim == 1:
            hu = U[1]
            return np.stack([hu, hu * hu / h + 0.5 * g * h * h])
        hu, hv = U[1], U[2]
        if d == 0:
            return np.stack([hu, hu * hu / h + 0.5 * g * h * h, hu * hv / h])
        return np.stack([hv, hu * hv / h, hv * hv / h + 0.5 * g * h * h])

    def max_speed(self, U, d):
        h = _re(U[0])
        un = _re(U[1 + d]) / h
        return np.abs(un) + np.sqrt(self.g * h)

    def primitive(self, U):
        h = U[0]
        return (h,) + tuple(U[1 + i] / h for i in range(self.dim))


class Euler:
    """Compressible Euler, Eq. (54), ideal gas E = p/(gamma-1) + rho|u|^2/2.
    U = (rho, rho u, E) in 1D, (rho, rho u, rho v, E) in 2D.  Wave speeds
    u_d - a, u_d, u_d + a with a = sqrt(gamma p / rho) (Sec. 5.2)."""

    name = "euler"

    def __init__(self, gamma=1.4, dim=2):
        self.gamma = float(gamma)
        self.dim = dim
        self.p = dim + 2

    def pressure(self, U):
        rho = U[0]
        ke = 0.0
        for i in range(self.dim):
            ke = ke + U[1 + i] * U[1 + i]
        return (self.gamma - 1.0) * (U[-1] - 0.5 * ke / rho)

    def flux(self, U, d):
        rho = U[0]
        E = U[-1]
        p = self.pressure(U)
        un = U[1 + d] / rho
        out = [U[1 + d]]
        for i in range(self.dim):
            mom = U[1 + i] * un
            if i == d:
                mom = mom + p
            out.append(mom)
        out.append(un * (E + p))
        return np.stack(out)

    def sound_speed(self, U):
        return np.sqrt(self.gamma * _re(self.pressure(U)) / _re(U[0]))

    def max_speed(self, U, d):
        un = _re(U[1 + d]) / _re(U[0])
        return np.abs(un) + self.sound_speed(U)


class MHDGLM:
    """Ideal MHD with hyperbolic divergence cleaning, Eq. (58) (Sec. 5.3):
    U = (rho, rho u, rho v, rho w, E, Bx, By, Bz, psi)  (p = 9),
    E = p/(gamma-1) + rho|u|^2/2 + |B|^2/2,
    F^(d) = (rho u_d, rho u u_d + (p + |B|^2/2) e_d - B B_d,
             (E + p + |B|^2/2) u_d - (B.u) B_d,
             u_d B - B_d u + psi e_d,  c_h^2 B_d).
    c_h is a parameter of the flux (set by the time loop, reading R4 of
    oracle/vklb.py: c_h = 6 max c_f over the grid, refreshed every step).
    Wave speeds along d: u_d, u_d +- c_a, u_d +- c_s, u_d +- c_f and the two
    cleaning waves +- c_h."""

    name = "mhd_glm"

    def __init__(self, gamma=5.0 / 3.0, ch=1.0, dim=2):
        self.gamma = float(gamma)
        self.ch = float(ch)
        self.dim = dim
        self.p = 9

    def pressure(self, U):
        rho = U[0]
        ke = (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho
        bb = U[5] * U[5] + U[6] * U[6] + U[7] * U[7]
        return (self.gamma - 1.0) * (U[4] - 0.5 * ke - 0.5 * bb)

    def flux(self, U, d):
        rho, mx, my, mz, E, bx, by, bz, psi = (U[i] for i in range(9))
        p = self.pressure(U)
        bb = bx * bx + by * by + bz * bz
        pt = p + 0.5 * bb
        vel = (mx / rho, my / rho, mz / rho)
        B = (bx, by, bz)
        m = (mx, my, mz)
        un = vel[d]
        bn = B[d]
        bu = bx * vel[0] + by * vel[1] + bz * vel[2]
        out = [m[d]]
        for i in range(3):
            fi = m[i] * un - B[i] * bn
            if i == d:
                fi = fi + pt
            out.append(fi)
        out.append((E + pt) * un - bu * bn)
        for i in range(3):
            fi = un * B[i] - bn * vel[i]
            if i == d:
                fi = fi + psi
            out.append(fi)
        out.append(self.ch * self.ch * bn)
        return np.stack(out)

    def fast_speed(self, U, d):
        """Fast magnetosonic speed along d: c_f^2 = (a^2 + b^2 + sqrt((a^2 +
        b^2)^2 - 4 a^2 b_d^2)) / 2, a^2 = gamma p / rho, b^2 = |B|^2 / rho."""
        rho = _re(U[0])
        p = _re(self.pressure(U))
        a2 = self.gamma * p / rho
        b2 = (_re(U[5]) ** 2 + _re(U[6]) ** 2 + _re(U[7]) ** 2) / rho
        bn2 = _re(U[5 + d]) ** 2 / rho
        s = a2 + b2
        disc = np.sqrt(np.maximum(s * s - 4.0 * a2 * bn2, 0.0))
        return np.sqrt(0.5 * (s + disc))

    def max_speed(self, U, d):
        un = _re(U[1 + d]) / _re(U[0])
        return np.maximum(np.abs(un) + self.fast_speed(U, d), self.ch)


def make(kind, dim, **kw):
    if kind == "advection":
        return Advection(a=kw.get("a", (1.0, 0.0)), dim=dim)
    if kind == "swe":
        return ShallowWater(g=kw.get("g", 9.81), dim=dim)
    if kind == "euler":
        return Euler(gamma=kw.get("gamma", 1.4), dim=dim)
    if kind == "mhd_glm":
        return MHDGLM(gamma=kw.get("gamma", 5.0 / 3.0), ch=kw.get("ch", 1.0), dim=dim)
    raise ValueError(kind)

"""The VKLB time loop of Sec. 3.5 (Fig. 5), literally, in FP64.

One step, in the flow chart's order:
  1. Delta t = Delta x / xi                                  (Fig. 5, Sec. 3.2)
  2. collision  f*_q = f_q - omega (f_q - f_q^eq(U^n))       (Eq. 42)
  3. streaming  f_q(x + v_q Delta t) = f*_q(x); periodic wrap (Eq. 43, Eq. 37)
  4. moments    U^{n+1} = sum_q f_q                          (Eq. 3)
  5. characteristic boundary conditions (non-periodic axes)  (Eqs. 33-36)
  6. CFL        xi = max_j |lambda_j| / nu over the grid      (Eq. 29)
  7. equilibria f^eq(U^{n+1}) for the next step              (Eqs. 22-24 / 41)
Initialisation: xi from U(x,0), f_q(x,0) = f_q^eq(U(x,0)) (Eq. 2b, Fig. 5).

Lattices: D1Q3 v = (xi, 0, -xi) (Sec. 2.2, Fig. 1); D2Q5 v = (xi,0), (-xi,0),
(0,0), (0,xi), (0,-xi) (Eq. 38).  Distributions are stored f[q, field, (y,) x].

Readings of the paper taken here, where it is silent or ambiguous:
  R1  alpha normaliser max_j|lambda_j| (Eq. 27): ``alpha_norm="global"`` (the
      default) takes one number per step, the grid-wide maximum over cells,
      directions and eigenvalues of the state being split (the quantity Eq. 29
      divides by nu; MHD-GLM includes c_h); ``alpha_norm="local"`` takes it per
      cell and direction.  The paper's wording fits either; the two readings
      give different schemes wherever the wave speeds vary over the grid.  The
      global one reproduces the paper's omega = 2 vortex study (second order to
      N = 1024, Sec. 5.2) and its Table 1 dam break at CFL 0.9 to N = 4096
      (Sec. 5.1); the local one diverges at N >= 512 there and degrades from
      N = 1024 respectively.
  R2  xi is the max over all cells, both directions and all eigenvalues.
  R3  run_to(T) lands on T with evenly spread steps: every step takes
      xi_eff = m dx / (T - t), m = ceil((T - t) xi / dx) (the number of
      CFL-limited steps left), so xi_eff >= xi and the last step ends on T.
      (Clipping only the last step breaks second order at omega = 2.)
  R4  MHD-GLM: c_h = ch_factor * max over cells and directions of c_f(U^n),
      refreshed with xi every step; +-c_h are eigenvalues and enter xi.
  R9  1D nodes are cell centres x_i = lo + (i + 1/2) dx; nodes 0 and N-1 are the
      boundary nodes of the characteristic condition.
  R10 characteristic BC: W = P^-1 U with P frozen at x_b; one-sided difference
      towards the interior; incoming waves (lambda < 0 on the right, lambda > 0
      on the left) are dropped; Delta t = dx / xi_n.
  R11 boundary f = f^eq(U_b^{n+1}) uses xi_{n+1}.
  R19 2D characteristic boundaries (the paper writes Eqs. 33-36 for D1Q3 only):
      every node on a non-periodic face takes the 1D construction along the
      face normal d, U_b^{n+1} = U_b^n - (1/xi_n) P_d Lambda_d^out P_d^-1 D_d U^n
      with A_d = dF^(d)/dU frozen at the node, the one-sided difference D_d
      towards the interior and the waves leaving through that face kept; a
      corner node sums the terms of its two faces; tangential derivatives are
      not added (the construction of Sec. 3.3 applied per face).  Its
      distributions are f^eq(U_b^{n+1}) with xi_{n+1} (R11), and xi_{n+1}
      includes the boundary states.  Streaming wraps as on a periodic grid;
      what wraps lands only in boundary nodes, which are overwritten.
  R21 transmissive boundaries (zero-order extrapolation, the textbook outflow
      condition; the paper's own open boundary is the characteristic one):
      after streaming, a boundary node takes U_b^{n+1} = U^{n+1} of the node
      one cell inwards along every non-periodic face it lies on (a 2D corner
      takes its diagonal neighbour), and its distributions are f^eq(U_b^{n+1})
      with xi_{n+1} as in R11.  In 2D every non-periodic axis takes the same
      kind (characteristic or transmissive).
  R20 storage="bf16" models distributions kept in bfloat16 (the precision form
      of the GPU path; the paper computes in FP64 throughout): every stored f
      (the initial f^eq, and after each step the streamed f including the
      boundary nodes) is rounded to the nearest bfloat16, ties to even; U, the
      next lattice speed and the equilibria are formed from the rounded f, the
      arithmetic itself stays FP64.

Test infrastructure only.

Parity pins (tests/test_oracle_vklb.py, tests/test_oracle_convergence.py):
moment constraints (Eqs. 3, 5); Theorems 4.1-4.3 (finite-difference and
finite-volume forms); exact discrete conservation on periodic grids (Thm 4.3);
exact shift for advection; exact Riemann solutions (dam break, Sod); second-order
convergence for smooth problems at omega = 2 (Sec. 5.2); the printed Mach ranges
of the entropy wave and vortex initial data (Sec. 5.2).
"""
import numpy as np

from . import splitting
from .systems import MHDGLM

D1Q3_M = np.array([1, 0, -1])
D2Q5_M = np.array([[1, 0], [-1, 0], [0, 0], [0, 1], [0, -1]])


def equilibrium_1d(U, Fp, Fm, xi, c):
    """Weighted upwind set, Eqs. (22)-(24):
    f1 = c U + F+/xi,  f2 = (1 - 2c) U - (F+ - F-)/xi,  f3 = c U - F-/xi."""
    f1 = c * U + Fp / xi
    f2 = (1.0 - 2.0 * c) * U - (Fp - Fm) / xi
    f3 = c * U - Fm / xi
    return np.stack([f1, f2, f3])


def equilibrium_2d(U, Fp1, Fm1, Fp2, Fm2, xi, c):
    """2D weighted upwind set, Eq. (41):
    f1 = c U + F(1,+)/xi, f2 = c U - F(1,-)/xi, f4 = c U + F(2,+)/xi,
    f5 = c U - F(2,-)/xi,
    f3 = (1 - 4c) U - (F(1,+) + F(2,+) - F(1,-) - F(2,-))/xi."""
    f1 = c * U + Fp1 / xi
    f2 = c * U - Fm1 / xi
    f4 = c * U + Fp2 / xi
    f5 = c * U - Fm2 / xi
    f3 = (1.0 - 4.0 * c) * U - (Fp1 + Fp2 - Fm1 - Fm2) / xi
    return np.stack([f1, f2, f3, f4, f5])


def outgoing_part(A, v, side):
    """P Lambda^out P^-1 v for a diagonalisable A with real eigenvalues, the
    waves leaving through a low face (side 0: lambda < 0) or a high face
    (side 1: lambda > 0).  Basis-free and stable: an ordered real Schur form
    A = Z T Z^T puts the k outgoing eigenvalues first, T = [[T11, T12], [0, T22]];
    with Y solving T11 Y - Y T22 = -T12 (the block diagonalisation
    [[I, Y], [0, I]]^-1 T [[I, Y], [0, I]] = diag(T11, T22)) the outgoing part of
    T is [[T11, -T11 Y], [0, 0]], and A's is Z times that times Z^T.  (Sylvester's
    product formula over the distinct eigenvalues, used before, loses most of
    its digits on the nine close speeds of MHD-GLM.)"""
    import scipy.linalg as sla
    A = np.real(np.asarray(A, dtype=np.complex128))
    out_sel = (lambda x: np.real(x) < 0) if side == 0 else (lambda x: np.real(x) > 0)
    T, Z, k = sla.schur(A, output="real", sort=out_sel)
    if k == 0:
        return np.zeros_like(v)
    n = A.shape[0]
    w = Z.T @ v
    T11 = T[:k, :k]
    if k < n:
        Y = sla.solve_sylvester(T11, -T[k:, k:], -T[:k, k:])
        top = T11 @ (w[:k] - Y @ w[k:])
    else:
        top = T11 @ w
    return Z[:, :k] @ top


def round_to_bf16(x):
    """Nearest bfloat16 (8 significant bits, ties to even) of each FP64 value,
    returned as FP64; normal range (no overflow or subnormal handling): with
    x = m 2^e, 1/2 <= |m| < 1, the significand m 2^8 is rounded to an integer
    (numpy rounds halves to even) and scaled back."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0), e - 8)


class Sim:
    """One VKLB simulation on a uniform grid.

    system   : an ``oracle.systems`` object (its dim selects D1Q3 or D2Q5)
    n        : (nx,) or (nx, ny) cells;  lo, hi: domain corners
    bc       : "periodic", "characteristic" or "transmissive" (all sides), or
               in 2D a pair (x axis, y axis) of those (R19, R21)
    set_kind : "weighted" (c, k), "centered" (c = 1/Q, F/2), "discontinuous"
    omega    : relaxation parameter, 0 < omega <= 2 (Sec. 2.3)
    nu       : CFL number (Eq. 29);  dt > 0 fixes xi = dx / dt instead
    alpha_norm: "local" or "global", reading R1 of alpha's normaliser
    storage  : "fp64", or "bf16" to round every stored f to bfloat16 (R20)
    """

    def __init__(self, system, n, lo, hi, bc="periodic", set_kind="weighted",
                 c=0.05, k=2.0, omega=1.0, nu=0.9, dt=None, ch_factor=6.0, eta=None,
                 alpha_norm="global", storage="fp64"):
        self.sys = system
        self.dim = system.dim
        self.n = tuple(int(v) for v in n)
        assert len(self.n) == self.dim
        lo = np.atleast_1d(np.asarray(lo, float))
        hi = np.atleast_1d(np.asarray(hi, float))
        dxs = (hi - lo) / np.asarray(self.n, float)
        if self.dim == 2 and abs(dxs[0] - dxs[1]) > 1e-12 * dxs[0]:
            raise ValueError("D2Q5 needs dx == dy (Sec. 3.4)")
        self.dx = float(dxs[0])
        self.lo, self.hi = lo, hi
        axes = (bc,) * self.dim if isinstance(bc, str) else tuple(bc)
        if len(axes) != self.dim or any(b not in ("periodic", "characteristic", "transmissive") for b in axes):
            raise ValueError(bc)
        open_kinds = {b for b in axes if b != "periodic"}
        if len(open_kinds) > 1:
            raise ValueError("the non-periodic axes take one kind (R21)")
        self.bc_axes = axes
        self.bc = open_kinds.pop() if open_kinds else "periodic"
        self.set_kind = set_kind
        if set_kind == "centered":
            c = 1.0 / 3.0 if self.dim == 1 else 1.0 / 5.0
        elif set_kind == "discontinuous":
            c = 0.0
        self.c, self.k, self.omega, self.nu = float(c), float(k), float(omega), float(nu)
        if not (0.0 < self.omega <= 2.0):
            raise ValueError("omega must lie in (0, 2] (Sec. 2.3)")
        # eta: the subcharacteristic condition of the centered set (Sec. 2.3),
        # xi > sqrt(3/2) max_j |lambda_j|, taken as xi = sqrt(3/2) max|lambda| / eta
        # with eta < 1 (the paper runs the centered set at eta = 0.9, Sec. 5)
        if eta is not None and not (0.0 < eta < 1.0):
            raise ValueError("eta must lie in (0, 1) (Sec. 2.3)")
        self.eta = None if eta is None else float(eta)
        self.fixed_xi = None if dt is None or dt <= 0 else self.dx / float(dt)
        self.ch_factor = float(ch_factor)
        if alpha_norm not in ("local", "global"):
            raise ValueError(alpha_norm)
        self.alpha_norm = alpha_norm
        if storage not in ("fp64", "bf16"):
            raise ValueError(storage)
        self.store = round_to_bf16 if storage == "bf16" else (lambda f: f)
        self.f = None
        self.t = 0.0
        self.steps = 0
        self.xi = None

    # ----- pieces of one step -------------------------------------------------
    def _flat(self, U):
        return U.reshape(U.shape[0], -1)

    def split(self, U, d, lam_norm=None):
        Uf = self._flat(U)
        Fp, Fm = splitting.split(self.sys, Uf, d, self.set_kind, self.k, lam_norm)
        return Fp.reshape(U.shape), Fm.reshape(U.shape)

    def equilibrium(self, U, xi, lam_grid=None):
        """Equilibria of the states U.  With the global reading of R1, alpha is
        normalised by ``lam_grid``, the grid-wide max |lambda| (default: that of
        U itself; the boundary states of the characteristic condition pass the
        whole grid's)."""
        lam = None
        if self.alpha_norm == "global":
            lam = self.max_lambda(U) if lam_grid is None else float(lam_grid)
        if self.dim == 1:
            Fp, Fm = self.split(U, 0, lam)
            return equilibrium_1d(U, Fp, Fm, xi, self.c)
        Fp1, Fm1 = self.split(U, 0, lam)
        Fp2, Fm2 = self.split(U, 1, lam)
        return equilibrium_2d(U, Fp1, Fm1, Fp2, Fm2, xi, self.c)

    def refresh_ch(self, U):
        """R4: c_h = ch_factor * max_{x,d} c_f(U)."""
        if isinstance(self.sys, MHDGLM):
            Uf = self._flat(U)
            cf = max(np.max(self.sys.fast_speed(Uf, d)) for d in range(self.dim))
            self.sys.ch = self.ch_factor * float(cf)

    def max_lambda(self, U):
        """R2: global max over cells, directions and eigenvalues."""
        Uf = self._flat(U)
        return max(float(np.max(self.sys.max_speed(Uf, d))) for d in range(self.dim))

    def cfl_xi(self, U):
        """Eq. (29): xi = max_j |lambda_j| / nu (or the fixed dx/dt); with eta,
        the subcharacteristic rule xi = sqrt(3/2) max_j |lambda_j| / eta (Sec. 2.3)."""
        if self.fixed_xi is not None:
            return self.fixed_xi
        if self.eta is not None:
            return np.sqrt(1.5) * self.max_lambda(U) / self.eta
        return self.max_lambda(U) / self.nu

    def stream(self, fs):
        """Eq. (43) with periodic wrap (Eq. 37) or, for the characteristic BC, a
        plain shift whose boundary nodes are overwritten by the BC."""
        out = np.empty_like(fs)
        if self.dim == 1:
            for q, m in enumerate(D1Q3_M):
                if self.bc == "periodic":
                    out[q] = np.roll(fs[q], m, axis=-1)
                else:
                    out[q] = fs[q]
                    if m == 1:
                        out[q][..., 1:] = fs[q][..., :-1]
                    elif m == -1:
                        out[q][..., :-1] = fs[q][..., 1:]
            return out
        for q, (mx, my) in enumerate(D2Q5_M):
            out[q] = np.roll(np.roll(fs[q], mx, axis=-1), my, axis=-2)
        return out

    def char_bc(self, Uold, Unew, xi_n):
        """Eqs. (33)-(35) with R10: returns the boundary states U_b^{n+1}
        (left, right) computed from U^n."""
        res = []
        for side in (0, 1):
            if side == 0:
                ub, dU = Uold[:, 0], Uold[:, 1] - Uold[:, 0]
            else:
                ub, dU = Uold[:, -1], Uold[:, -1] - Uold[:, -2]
            A = splitting.jacobian(self.sys, ub[:, None], 0)[0]
            lam, P = np.linalg.eig(A)
            lam = np.real(lam)
            P = np.real(P)
            dW = np.linalg.solve(P, dU)          # dx * dW/dx, W = P^-1 U
            keep = (lam < 0) if side == 0 else (lam > 0)   # outgoing waves only
            rhs = P @ (np.where(keep, lam, 0.0) * dW)
            res.append(ub - rhs / xi_n)          # Delta t / dx = 1 / xi_n
        return res

    def boundary_mask(self):
        """2D: True at the nodes of the non-periodic faces ([ny, nx])."""
        ny, nx = self.n[1], self.n[0]
        m = np.zeros((ny, nx), dtype=bool)
        if self.bc_axes[0] != "periodic":
            m[:, 0] = m[:, -1] = True
        if self.bc_axes[1] != "periodic":
            m[0, :] = m[-1, :] = True
        return m

    def transmissive_2d(self, Unew):
        """R21: U_b^{n+1} = U^{n+1} of the node one cell inwards along every
        non-periodic face the node lies on ([p, ny, nx]; interior nodes keep
        their own value)."""
        ny, nx = self.n[1], self.n[0]
        xi = np.arange(nx)
        yi = np.arange(ny)
        if self.bc_axes[0] != "periodic":
            xi[0], xi[-1] = 1, nx - 2
        if self.bc_axes[1] != "periodic":
            yi[0], yi[-1] = 1, ny - 2
        return Unew[:, yi[:, None], xi[None, :]]

    def char_bc_2d(self, Uold, xi_n):
        """R19: Eqs. (33)-(35) along the normal of every non-periodic face, from
        U^n; a corner sums its two faces.  Returns U_b^{n+1} on the boundary
        nodes as a full [p, ny, nx] array (other nodes: U^n, unused)."""
        rhs = np.zeros_like(Uold)
        for d, axis in ((0, 2), (1, 1)):
            if self.bc_axes[d] != "characteristic":
                continue
            for side in (0, 1):
                take = [slice(None)] * 3
                inner = [slice(None)] * 3
                take[axis] = 0 if side == 0 else -1
                inner[axis] = 1 if side == 0 else -2
                ub = Uold[tuple(take)]                          # [p, face length]
                dU = (Uold[tuple(inner)] - ub) if side == 0 else (ub - Uold[tuple(inner)])
                A = splitting.jacobian(self.sys, ub, d)           # [m, p, p]
                for m in range(A.shape[0]):
                    rhs[tuple(take)][:, m] += outgoing_part(A[m], dU[:, m], side)
        return Uold - rhs / xi_n

    # ----- public API ---------------------------------------------------------
    def set_state(self, U0):
        U0 = np.array(U0, dtype=np.float64)
        assert U0.shape == (self.sys.p,) + tuple(reversed(self.n)), U0.shape
        self.refresh_ch(U0)
        self.xi = self.cfl_xi(U0)
        self.f = self.store(self.equilibrium(U0, self.xi))  # Eq. (2b), R20
        self.t = 0.0
        self.steps = 0

    def moments(self):
        return self.f.sum(axis=0)                             # Eq. (3)

    def step(self, t_end=None):
        """One step of Fig. 5.  With t_end, the lattice speed is raised to land
        on t_end with evenly spread steps (R3); returns False without stepping
        once t >= t_end."""
        xi = self.xi
        if t_end is not None:
            rem = t_end - self.t
            if rem <= 1e-14 * max(1.0, abs(t_end)):
                return False
            m = max(1.0, np.ceil(rem * xi / self.dx - 1e-9))
            xi = m * self.dx / rem
        U = self.f.sum(axis=0)
        feq = self.equilibrium(U, xi)                         # Eqs. (22)-(24)/(41)
        fs = self.f - self.omega * (self.f - feq)             # Eq. (42)
        fn = self.store(self.stream(fs))                      # Eq. (43), R20
        Un = fn.sum(axis=0)                                   # Eq. (3)
        if self.bc == "characteristic" and self.dim == 1:
            ubl, ubr = self.char_bc(U, Un, xi)                # Eqs. (33)-(35)
            Un[:, 0] = ubl
            Un[:, -1] = ubr
        elif self.bc == "transmissive" and self.dim == 1:
            Un[:, 0] = Un[:, 1]                               # R21
            Un[:, -1] = Un[:, -2]
        elif self.bc == "characteristic":
            mask = self.boundary_mask()
            Un[:, mask] = self.char_bc_2d(U, xi)[:, mask]     # R19
        elif self.bc == "transmissive":
            mask = self.boundary_mask()
            Un[:, mask] = self.transmissive_2d(Un)[:, mask]   # R21
        self.refresh_ch(Un)
        xin = self.cfl_xi(Un)                                 # Eq. (29)
        if self.bc != "periodic" and self.dim == 1:
            fb = self.equilibrium(np.stack([Un[:, 0], Un[:, -1]], axis=1), xin,
                                  self.max_lambda(Un))
            fn[:, :, 0] = fb[:, :, 0]                         # Eq. (36), R11
            fn[:, :, -1] = fb[:, :, 1]
        elif self.bc != "periodic":
            fb = self.equilibrium(Un[:, mask], xin, self.max_lambda(Un))
            fn[:, :, mask] = fb                               # Eq. (36), R11, R19
        self.f = self.store(fn)                               # R20 (boundary nodes)
        self.t = self.t + self.dx / xi
        if t_end is not None and abs(self.t - t_end) <= 1e-13 * max(1.0, abs(t_end)):
            self.t = float(t_end)
        self.xi = xin
        self.steps += 1
        return True

    def run(self, nsteps):
        for _ in range(int(nsteps)):
            self.step()

    def run_to(self, t_end, max_steps=10**7):
        for _ in range(max_steps):
            if not self.step(t_end):
                break

    def totals(self):
        """Conserved totals sum_x U(x) dx^D (Thm 4.3: conserved on periodic grids)."""
        U = self.moments()
        axes = tuple(range(1, U.ndim))
        return U.sum(axis=axes) * self.dx ** self.dim

    def cell_centers(self):
        cs = [self.lo[i] + (np.arange(self.n[i]) + 0.5) * self.dx for i in range(self.dim)]
        return cs

"""The closed-form eigen-structures of the CUDA path (vk_systems.cuh), evaluated
on the host through libvklb_hostcheck.so, against the FP64 oracle's matrix-function
split (no GPU).  This checks the device arithmetic itself before any kernel runs."""
import ctypes as C

import numpy as np
import pytest

from oracle import splitting, systems
from paper_2608_04283_b300 import build, inputs

build.build()
_lib = C.CDLL(build.HOSTCHECK)
_PD = C.POINTER(C.c_double)
KIND = {"advection": 0, "swe": 1, "euler": 2, "mhd_glm": 3}


def hc_split(kind, dim, d, prec, set_kind, k, ch, gamma, g, U, ax=1.0, ay=-0.5, lg=0.0):
    U = np.ascontiguousarray(U, dtype=np.float64)
    p, n = U.shape
    Fp, F = np.zeros_like(U), np.zeros_like(U)
    m1, m2 = np.zeros(n), np.zeros(n)
    st = _lib.vklb_hc_split(KIND[kind], dim, d, prec, set_kind, C.c_double(k), C.c_double(lg), C.c_double(ch),
                            C.c_double(gamma),
                            C.c_double(g), C.c_double(ax), C.c_double(ay), U.ctypes.data_as(_PD), C.c_int64(n),
                            Fp.ctypes.data_as(_PD), F.ctypes.data_as(_PD), m1.ctypes.data_as(_PD),
                            m2.ctypes.data_as(_PD))
    assert st == 0
    return Fp, F, m1, m2


CASES = [("swe", 1, {"g": 9.81}), ("swe", 2, {"g": 9.81}), ("euler", 1, {"gamma": 1.4}),
         ("euler", 2, {"gamma": 1.4}), ("mhd_glm", 2, {"gamma": 5 / 3, "ch": 6.0}),
         ("mhd_glm", 2, {"gamma": 5 / 3, "ch": 1.3})]


@pytest.mark.parametrize("name,dim,kw", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 2e-13), (1, 2e-5)])
def test_weighted_split_matches_oracle(name, dim, kw, prec, tol):
    s = systems.make(name, dim, **kw)
    gamma, g, ch = kw.get("gamma", 1.4), kw.get("g", 9.81), kw.get("ch", 0.0)
    U = inputs.random_states(name, 800, seed=31, dim=dim, gamma=gamma)
    for d in range(dim):
        Fp, F, m1, m2 = hc_split(name, dim, d, prec, 0, 2.0, ch, gamma, g, U)
        Fo, _ = splitting.split_weighted(s, U, d, 2.0)
        Fph = s.flux(U, d)
        scale = np.abs(Fph).max(axis=0) + 1.0
        assert np.max(np.abs(F - Fph) / scale) < tol
        assert np.max(np.abs(Fp - Fo) / scale) < tol
        lam = s.max_speed(U, d) if name != "mhd_glm" else np.abs(U[1 + d] / U[0]) + s.fast_speed(U, d)
        assert np.allclose(m1, lam, rtol=10 * tol)


@pytest.mark.parametrize("name,dim,kw", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 2e-13), (1, 2e-5)])
def test_weighted_split_global_normaliser_matches_oracle(name, dim, kw, prec, tol):
    """alpha normalised by one grid-wide max |lambda| (the global reading of the
    weight's normaliser): the device split given lg = that maximum equals the
    oracle's split with the same lam_norm, in both directions."""
    s = systems.make(name, dim, **kw)
    gamma, g, ch = kw.get("gamma", 1.4), kw.get("g", 9.81), kw.get("ch", 0.0)
    U = inputs.random_states(name, 600, seed=33, dim=dim, gamma=gamma)
    lam = max(float(np.max(s.max_speed(U, d))) for d in range(dim))
    for d in range(dim):
        Fp, F, _, _ = hc_split(name, dim, d, prec, 0, 2.0, ch, gamma, g, U, lg=lam)
        Fo, _ = splitting.split_weighted(s, U, d, 2.0, lam_norm=lam)
        scale = np.abs(s.flux(U, d)).max(axis=0) + 1.0
        assert np.max(np.abs(Fp - Fo) / scale) < tol
        # where the cells' own maxima differ it is not the per-cell split
        # (MHD-GLM with c_h above every fast speed normalises by c_h either way)
        Fl, _ = splitting.split_weighted(s, U, d, 2.0)
        if np.ptp(s.max_speed(U, d)) > 1e-3 * lam:
            assert np.max(np.abs(Fp - Fl) / scale) > 100 * tol
        else:
            assert np.max(np.abs(Fp - Fl) / scale) < tol


@pytest.mark.parametrize("name,dim,kw", CASES)
def test_discontinuous_and_centered_sets(name, dim, kw):
    s = systems.make(name, dim, **kw)
    gamma, g, ch = kw.get("gamma", 1.4), kw.get("g", 9.81), kw.get("ch", 0.0)
    U = inputs.random_states(name, 300, seed=32, dim=dim, gamma=gamma)
    for d in range(dim):
        Fp, F, _, _ = hc_split(name, dim, d, 0, 1, 2.0, ch, gamma, g, U)
        assert np.allclose(Fp, 0.5 * s.flux(U, d), rtol=1e-14, atol=1e-14)
        A = splitting.jacobian(s, U, d)
        lam = np.real(np.linalg.eigvals(A))
        ok = np.min(np.abs(lam), axis=1) > 1e-3 * np.max(np.abs(lam), axis=1)
        Fp, F, _, _ = hc_split(name, dim, d, 0, 2, 2.0, ch, gamma, g, U[:, ok])
        Fd, _ = splitting.split_discontinuous(s, U[:, ok], d)
        scale = np.abs(F).max(axis=0) + 1.0
        assert np.max(np.abs(Fp - Fd) / scale) < 1e-9


def test_mhd_degenerate_states():
    """Near and at the triple point (B_t = 0, a = c_a) and with B_x = 0 the
    closed-form split still equals the oracle's alpha(A) F."""
    g = 5 / 3
    rho = np.array([1.0, 1.0, 1.0, 2.0, 1.0, 1.0])
    p = np.array([0.6, 0.6, 0.6, 1.0, 0.6, 0.6])
    a = np.sqrt(g * p / rho)
    bx = np.array([1.0, 1.0, 0.0, 1.2, 1.0, 1.0]) * np.sqrt(rho) * a    # c_a = a in rows 0, 1
    by = np.array([0.0, 1e-9, 0.7, 0.0, 1e-4, 0.3])
    bz = np.array([0.0, 0.0, 0.0, 0.0, 0.0, -0.2])
    u = np.array([0.3, -0.2, 0.1, 0.0, 0.5, -0.4])
    U = inputs.mhd_conserved(rho, u, 0.2 * u, 0 * u, p, bx, by, bz, 0.01 + 0 * u, g)
    s = systems.MHDGLM(g, ch=5.0)
    for prec, tol in ((0, 1e-11), (1, 5e-5)):
        for d in range(2):
            Fp, F, _, _ = hc_split("mhd_glm", 2, d, prec, 0, 2.0, 5.0, g, 9.81, U)
            Fo, _ = splitting.split_weighted(s, U, d, 2.0)
            scale = np.abs(s.flux(U, d)).max(axis=0) + 1.0
            assert np.max(np.abs(Fp - Fo) / scale) < tol, (prec, d)


@pytest.mark.parametrize("name,kw", [("swe", {"g": 9.81}), ("euler", {"gamma": 1.4}), ("advection", {})])
@pytest.mark.parametrize("side", [0, 1])
def test_char_bc_rhs_matches_oracle_eig(name, kw, side):
    """Eqs. (33)-(35): P diag(lambda_j, outgoing) P^-1 dU against numpy.linalg.eig of
    the oracle's complex-step Jacobian."""
    s = systems.make(name, 1, **kw) if name != "advection" else systems.Advection(a=(0.7,), dim=1)
    U = inputs.random_states(name, 64, seed=33, dim=1, gamma=kw.get("gamma", 1.4))
    rng = np.random.default_rng(34)
    dU = rng.standard_normal(U.shape) * 0.1
    out = np.zeros_like(U)
    st = _lib.vklb_hc_char_rhs(KIND[name], 0, side, C.c_double(kw.get("gamma", 1.4)), C.c_double(kw.get("g", 9.81)),
                               C.c_double(0.7), np.ascontiguousarray(U).ctypes.data_as(_PD),
                               np.ascontiguousarray(dU).ctypes.data_as(_PD), C.c_int64(U.shape[1]),
                               out.ctypes.data_as(_PD))
    assert st == 0
    A = splitting.jacobian(s, U, 0)
    for i in range(U.shape[1]):
        lam, P = np.linalg.eig(A[i])
        lam, P = np.real(lam), np.real(P)
        keep = lam < 0 if side == 0 else lam > 0
        want = P @ (np.where(keep, lam, 0.0) * np.linalg.solve(P, dU[:, i]))
        assert np.allclose(out[:, i], want, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("name,kw", [("swe", {"g": 9.81}), ("euler", {"gamma": 1.4}),
                                     ("mhd_glm", {"gamma": 5 / 3, "ch": 6.0})])
@pytest.mark.parametrize("prec,tol", [(0, 2e-13), (1, 2e-5)])
@pytest.mark.parametrize("set_kind", [0, 1])
def test_split2_and_epilogue_match_oracle(name, kw, prec, tol, set_kind):
    """The both-direction split (shared primitives) and the step epilogue that the
    step kernels call: F(1,+-), F(2,+-) against the oracle; the epilogue maxima
    against the closed-form wave speeds; the physical test against p, rho > 0."""
    s = systems.make(name, 2, **kw)
    gamma, g, ch = kw.get("gamma", 1.4), kw.get("g", 9.81), kw.get("ch", 0.0)
    U = np.ascontiguousarray(inputs.random_states(name, 600, seed=35, dim=2, gamma=gamma))
    p, n = U.shape
    out = [np.zeros_like(U) for _ in range(4)]
    m1, m2 = np.zeros(n), np.zeros(n)
    ok = np.zeros(n, dtype=np.int32)
    st = _lib.vklb_hc_split2(KIND[name], prec, set_kind, C.c_double(2.0), C.c_double(0.0), C.c_double(ch),
                             C.c_double(gamma),
                             C.c_double(g), C.c_double(1.0), C.c_double(-0.5), U.ctypes.data_as(_PD), C.c_int64(n),
                             *[o.ctypes.data_as(_PD) for o in out], m1.ctypes.data_as(_PD), m2.ctypes.data_as(_PD),
                             ok.ctypes.data_as(C.POINTER(C.c_int)))
    assert st == 0
    for d in range(2):
        Fp, F = out[2 * d], out[2 * d + 1]
        Fph = s.flux(U, d)
        Fo = splitting.split_weighted(s, U, d, 2.0)[0] if set_kind == 0 else 0.5 * Fph
        scale = np.abs(Fph).max(axis=0) + 1.0
        assert np.max(np.abs(F - Fph) / scale) < tol
        assert np.max(np.abs(Fp - Fo) / scale) < tol
    if name == "mhd_glm":
        lam = np.maximum(*[np.abs(U[1 + d] / U[0]) + s.fast_speed(U, d) for d in range(2)])
        cf = np.maximum(s.fast_speed(U, 0), s.fast_speed(U, 1))
        assert np.allclose(m2, cf, rtol=10 * tol)
    else:
        lam = np.maximum(s.max_speed(U, 0), s.max_speed(U, 1))
    assert np.allclose(m1, lam, rtol=10 * tol)
    assert np.all(ok == 1)


@pytest.mark.parametrize("name,kw", [("swe", {"g": 9.81}), ("euler", {"gamma": 1.4}), ("advection", {}),
                                     ("mhd_glm", {"gamma": 5.0 / 3.0})])
@pytest.mark.parametrize("d,side", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_char_rhs_2d_matches_oracle(name, kw, d, side):
    """The 2D characteristic boundary's outgoing part along either face normal
    (closed-form eigenvectors, vk_systems.cuh) against the oracle's basis-free
    spectral projection (Sylvester's formula over the complex-step Jacobian).
    MHD-GLM: the 9-wave Jacobian with c_h = 6 max c_f of the states (R4)."""
    from oracle import vklb as ovklb
    s = systems.make(name, 2, a=(0.7, -0.4), **kw)
    U = np.ascontiguousarray(inputs.random_states(name, 150, seed=37 + 2 * d + side, dim=2,
                                                  gamma=kw.get("gamma", 1.4)))
    ch = 0.0
    if name == "mhd_glm":
        ch = 6.0 * float(max(s.fast_speed(U, 0).max(), s.fast_speed(U, 1).max()))
        s.ch = ch
    rng = np.random.default_rng(5)
    dU = np.ascontiguousarray(0.1 * rng.standard_normal(U.shape))
    out = np.zeros_like(U)
    st = _lib.vklb_hc_char_rhs2d(KIND[name], 0, d, side, C.c_double(kw.get("gamma", 1.4)),
                                 C.c_double(kw.get("g", 9.81)), C.c_double(0.7), C.c_double(-0.4), C.c_double(ch),
                                 U.ctypes.data_as(_PD), dU.ctypes.data_as(_PD), C.c_int64(U.shape[1]),
                                 out.ctypes.data_as(_PD))
    assert st == 0
    A = splitting.jacobian(s, U, d)
    for i in range(U.shape[1]):
        want = ovklb.outgoing_part(A[i], dU[:, i], side)
        scale = 1.0 if name != "mhd_glm" else max(1.0, float(np.abs(want).max()))
        assert np.allclose(out[:, i], want, rtol=1e-10, atol=1e-12 * scale), i


@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 7), (37, 5), (64, 64)])
@pytest.mark.parametrize("cbx,cby", [(1, 0), (0, 1), (1, 1)])
def test_char_face_enumeration(nx, ny, cbx, cby):
    """The boundary passes give one thread to each node of the characteristic
    faces: the enumeration covers exactly those nodes, each once, in range."""
    cap = 2 * (nx + ny)
    xs = np.zeros(cap, dtype=np.int32)
    ys = np.zeros(cap, dtype=np.int32)
    P = C.POINTER(C.c_int)
    nb = _lib.vklb_hc_char_faces(nx, ny, cbx, cby, xs.ctypes.data_as(P), ys.ctypes.data_as(P), cap)
    assert nb >= 0
    got = set(zip(xs[:nb].tolist(), ys[:nb].tolist()))
    assert len(got) == nb
    want = {(x, y) for x in range(nx) for y in range(ny)
            if (cbx and x in (0, nx - 1)) or (cby and y in (0, ny - 1))}
    assert got == want

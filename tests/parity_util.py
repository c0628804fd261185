"""Comparison helpers shared by the GPU parity tests.

max_rel:  per field max_x |a - b| / max_x |b| (the tolerance read per field); a
          field that is identically zero in the reference must be zero to the
          absolute tolerance scaled by the largest field.
rel_l1:   per field sum |a - b| / sum |b|, with the same rule for zero fields.
max_rel_mhd / rel_l1_mhd: max_rel / rel_l1 for the nine MHD-GLM fields, with
          the scale of the three fields that Orszag-Tang keeps at zero or at
          rounding level taken from the terms that carry them (Eq. 58):
            m_z   max(own norm, norm of |m|)      -- its distribution components
                  are momentum-flux terms mixed by the eigen-split;
            B_z   max(own norm, norm of |B|)      -- likewise for the induction;
            psi   max(own norm, c_h norm of |B|)  -- its components carry the
                  cleaning waves' c_h B_n / 2 (phi_+- = (psi +- c_h B_n) / 2), so
                  their FP32 rounding is of size c_h |B|, whatever psi is.
          Every other field is measured against its own norm.
"""
import numpy as np


def _per_field(a, b, norm, small=1e-12):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    p = b.shape[0]
    big = max(norm(b[k]) for k in range(p))
    out = []
    for k in range(p):
        d = a[k] - b[k]
        s = norm(b[k])
        if s <= small * big:
            s = big
        out.append(norm(d) / s)
    return np.array(out)


def max_rel(a, b):
    return _per_field(a, b, lambda x: np.max(np.abs(x)))


def rel_l1(a, b):
    return _per_field(a, b, lambda x: np.sum(np.abs(x)))


def _mhd(a, b, ch, norm):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    m = np.sqrt(b[1] ** 2 + b[2] ** 2 + b[3] ** 2)
    B = np.sqrt(b[5] ** 2 + b[6] ** 2 + b[7] ** 2)
    scale = [norm(b[k]) for k in range(9)]
    scale[3] = max(scale[3], norm(m))
    scale[7] = max(scale[7], norm(B))
    scale[8] = max(scale[8], ch * norm(B))
    return np.array([norm(a[k] - b[k]) / scale[k] for k in range(9)])


def mhd_ch(U, gamma=5.0 / 3.0, ch_factor=6.0):
    """c_h of the state U (the oracle's rule: ch_factor x max fast speed over the
    grid and both directions), the cleaning speed the scale of psi uses."""
    from oracle.systems import MHDGLM
    s = MHDGLM(gamma)
    Uf = np.asarray(U, float).reshape(9, -1)
    return ch_factor * max(float(np.max(s.fast_speed(Uf, d))) for d in range(2))


def rel_l1_mhd(a, b, ch=None):
    """ch defaults to mhd_ch(b) (gamma 5/3, factor 6)."""
    ch = mhd_ch(b) if ch is None else ch
    return _mhd(a, b, ch, lambda x: np.sum(np.abs(x)))


def max_rel_mhd(a, b, ch):
    return _mhd(a, b, ch, lambda x: np.max(np.abs(x)))

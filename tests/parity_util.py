"""Comparison helpers shared by the GPU parity tests.

max_rel:  per field max_x |a - b| / max_x |b| (the tolerance read per field); a
          field that is identically zero in the reference must be zero to the
          absolute tolerance scaled by the largest field.
rel_l1:   per field sum |a - b| / sum |b|, with the same rule for zero fields.
max_rel_coupled / rel_l1_coupled: max_rel / rel_l1, but a field below 1e-2 of
          the largest takes the
          largest field's norm as its scale.  For FP32 MHD-GLM: psi (and a weak
          B_z or m_z) is carried by distribution components dominated by the
          c_h B_x / B coupling terms of Eq. (58), so its rounding error scales
          with those, not with the field itself.
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


def rel_l1_coupled(a, b):
    return _per_field(a, b, lambda x: np.sum(np.abs(x)), small=1e-2)


def max_rel_coupled(a, b):
    return _per_field(a, b, lambda x: np.max(np.abs(x)), small=1e-2)

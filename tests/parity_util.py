"""Comparison helpers shared by the GPU parity tests.

max_rel:  per field max_x |a - b| / max_x |b| (reading R16 of the tolerance); a
          field that is identically zero in the reference must be zero to the
          absolute tolerance scaled by the largest field.
rel_l1:   per field sum |a - b| / sum |b|, with the same rule for zero fields.
"""
import numpy as np


def _per_field(a, b, norm):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    p = b.shape[0]
    big = max(norm(b[k]) for k in range(p))
    out = []
    for k in range(p):
        d = a[k] - b[k]
        s = norm(b[k])
        if s <= 1e-12 * big:
            s = big
        out.append(norm(d) / s)
    return np.array(out)


def max_rel(a, b):
    return _per_field(a, b, lambda x: np.max(np.abs(x)))


def rel_l1(a, b):
    return _per_field(a, b, lambda x: np.sum(np.abs(x)))

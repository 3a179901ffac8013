"""IPC smoothly clamped log barrier, Sec. 3.3, Eq. (IPC-barrier):

    b(d, c) = -(d - c)^2 ln(d / c)   for 0 < d < c,   0 for d >= c.

b is C^2 at d = c (b = b' = b'' = 0 there). c is dhat for the base barrier and
dhat + s_i for the augmentation barrier of Eq. (aug-lag). Closed-form
derivatives (differentiating the definition by hand):

    b'(d)  = -2 (d - c) ln(d/c) - (d - c)^2 / d
    b''(d) = -2 ln(d/c) - 4 (d - c)/d + (d - c)^2 / d^2
"""
import numpy as np


def b(d, c):
    d = np.asarray(d, dtype=np.float64)
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), d.shape)
    out = np.zeros_like(d)
    m = (d > 0) & (d < c)
    dm, cm = d[m], c[m]
    out[m] = -(dm - cm) ** 2 * np.log(dm / cm)
    out[(d <= 0)] = np.inf
    return out


def db(d, c):
    d = np.asarray(d, dtype=np.float64)
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), d.shape)
    out = np.zeros_like(d)
    m = (d > 0) & (d < c)
    dm, cm = d[m], c[m]
    out[m] = -2.0 * (dm - cm) * np.log(dm / cm) - (dm - cm) ** 2 / dm
    return out


def d2b(d, c):
    d = np.asarray(d, dtype=np.float64)
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), d.shape)
    out = np.zeros_like(d)
    m = (d > 0) & (d < c)
    dm, cm = d[m], c[m]
    out[m] = -2.0 * np.log(dm / cm) - 4.0 * (dm - cm) / dm + (dm - cm) ** 2 / dm ** 2
    return out

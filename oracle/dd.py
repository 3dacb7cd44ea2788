"""Double-double arithmetic on numpy float64 arrays (test infrastructure only).

Error-free transformations: Knuth's TwoSum and Dekker's splitting / TwoProduct
(Dekker 1971, "A floating-point technique for extending the available
precision").  A double-double value is a pair (hi, lo) with |lo| <= ulp(hi)/2.
Used by the oracle to form residuals f - A u to roughly 32 significant digits.
"""
import numpy as np

_SPLIT = 134217729.0  # 2^27 + 1


def two_sum(a, b):
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def fast_two_sum(a, b):
    s = a + b
    e = b - (s - a)
    return s, e


def split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def dd_add(x, y):
    """(hi, lo) + (hi, lo)."""
    s, e = two_sum(x[0], y[0])
    t, f = two_sum(x[1], y[1])
    e = e + t
    s, e = fast_two_sum(s, e)
    e = e + f
    return fast_two_sum(s, e)


def dd_neg(x):
    return (-x[0], -x[1])


def dd_mul_d(x, b):
    """(hi, lo) * double (b may be an array or scalar)."""
    p, e = two_prod(x[0], b)
    e = e + x[1] * b
    return fast_two_sum(p, e)


def dd_from(a):
    a = np.asarray(a, dtype=np.float64)
    return (a.copy(), np.zeros_like(a))


def dd_to_double(x):
    return x[0] + x[1]


class CDD:
    """Complex double-double array: re and im parts, each a (hi, lo) pair."""

    def __init__(self, re, im):
        self.re = re
        self.im = im

    @staticmethod
    def from_complex(z):
        z = np.asarray(z, dtype=np.complex128)
        return CDD(dd_from(z.real), dd_from(z.imag))

    def to_complex(self):
        return dd_to_double(self.re) + 1j * dd_to_double(self.im)

    def __add__(self, o):
        return CDD(dd_add(self.re, o.re), dd_add(self.im, o.im))

    def __sub__(self, o):
        return CDD(dd_add(self.re, dd_neg(o.re)), dd_add(self.im, dd_neg(o.im)))

    def mul_c(self, c):
        """Multiply by a complex double (scalar or broadcastable array)."""
        c = np.asarray(c, dtype=np.complex128)
        cr, ci = c.real, c.imag
        if np.all(ci == 0):
            return CDD(dd_mul_d(self.re, cr), dd_mul_d(self.im, cr))
        re = dd_add(dd_mul_d(self.re, cr), dd_neg(dd_mul_d(self.im, ci)))
        im = dd_add(dd_mul_d(self.im, cr), dd_mul_d(self.re, ci))
        return CDD(re, im)

    def map(self, fn):
        """Apply an index-only operation (slicing, padding) to every component."""
        return CDD((fn(self.re[0]), fn(self.re[1])), (fn(self.im[0]), fn(self.im[1])))

"""Forward-mode dual numbers over numpy arrays.  Test infrastructure only.

A Dual carries a value v (any shape, real or complex) and k tangents d of
shape (k,) + v.shape.  Arithmetic follows the product and chain rules, so a
function written with +, -, *, / and sqrt returns its exact (to rounding)
derivative along each tangent.  The oracle uses it to differentiate the
exterior velocity expansion in Cartesian coordinates for the traction
(Sec. 3.3, Eq. 3.18).
"""
import numpy as np


class Dual:
    __array_priority__ = 1000

    def __init__(self, v, d):
        self.v = np.asarray(v)
        self.d = np.asarray(d)

    @staticmethod
    def seed(x):
        """x of shape (3, ...) -> three Duals with unit tangents e_1, e_2, e_3."""
        x = np.asarray(x, float)
        out = []
        for i in range(3):
            d = np.zeros((3,) + x.shape[1:])
            d[i] = 1.0
            out.append(Dual(x[i], d))
        return out

    # --- helpers
    @staticmethod
    def _parts(o):
        if isinstance(o, Dual):
            return o.v, o.d
        return np.asarray(o), None

    def __add__(self, o):
        ov, od = Dual._parts(o)
        return Dual(self.v + ov, self.d + od if od is not None else self.d + 0 * ov)

    __radd__ = __add__

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        ov, od = Dual._parts(o)
        if od is None:
            return Dual(self.v * ov, self.d * ov)
        return Dual(self.v * ov, self.d * ov + self.v * od)

    __rmul__ = __mul__

    def __truediv__(self, o):
        ov, od = Dual._parts(o)
        if od is None:
            return Dual(self.v / ov, self.d / ov)
        return Dual(self.v / ov, (self.d * ov - self.v * od) / (ov * ov))

    def __rtruediv__(self, o):
        # o / self with o constant
        ov = np.asarray(o)
        return Dual(ov / self.v, -ov * self.d / (self.v * self.v))

    def __pow__(self, k):
        if not isinstance(k, (int, np.integer)) or k < 0:
            raise ValueError("non-negative integer powers only")
        out = Dual(np.ones_like(self.v), np.zeros_like(self.d))
        for _ in range(k):
            out = out * self
        return out

    def sqrt(self):
        s = np.sqrt(self.v)
        return Dual(s, self.d / (2.0 * s))

    @property
    def real(self):
        return Dual(np.real(self.v), np.real(self.d))

    def conj(self):
        return Dual(np.conj(self.v), np.conj(self.d))


def dsqrt(x):
    return x.sqrt() if isinstance(x, Dual) else np.sqrt(x)


def value(x):
    return x.v if isinstance(x, Dual) else np.asarray(x)


def tangents(x):
    return x.d

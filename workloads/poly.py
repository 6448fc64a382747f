"""A tiny sparse polynomial type used to *write down* problem data.

Polynomials are dictionaries from exponent tuples to coefficients. Only the
ring operations needed to type in dynamics and costs are provided.
"""
from __future__ import annotations

import numpy as np


class Poly:
    __slots__ = ("nv", "terms")

    def __init__(self, nv: int, terms: dict | None = None):
        self.nv = nv
        self.terms = {} if terms is None else {k: float(v) for k, v in terms.items() if v != 0.0}

    # constructors -------------------------------------------------------
    @staticmethod
    def const(nv: int, c: float) -> "Poly":
        return Poly(nv, {(0,) * nv: c})

    @staticmethod
    def var(nv: int, i: int, scale: float = 1.0) -> "Poly":
        e = [0] * nv
        e[i] = 1
        return Poly(nv, {tuple(e): scale})

    # ring operations ----------------------------------------------------
    def _coerce(self, o):
        return o if isinstance(o, Poly) else Poly.const(self.nv, float(o))

    def __add__(self, o):
        o = self._coerce(o)
        t = dict(self.terms)
        for k, v in o.terms.items():
            t[k] = t.get(k, 0.0) + v
        return Poly(self.nv, t)

    __radd__ = __add__

    def __neg__(self):
        return Poly(self.nv, {k: -v for k, v in self.terms.items()})

    def __sub__(self, o):
        return self + (-self._coerce(o))

    def __rsub__(self, o):
        return self._coerce(o) - self

    def __mul__(self, o):
        if not isinstance(o, Poly):
            return Poly(self.nv, {k: v * float(o) for k, v in self.terms.items()})
        t: dict = {}
        for k1, v1 in self.terms.items():
            for k2, v2 in o.terms.items():
                k = tuple(a + b for a, b in zip(k1, k2))
                t[k] = t.get(k, 0.0) + v1 * v2
        return Poly(self.nv, t)

    __rmul__ = __mul__

    def __pow__(self, p: int):
        r = Poly.const(self.nv, 1.0)
        for _ in range(p):
            r = r * self
        return r

    # queries ------------------------------------------------------------
    def degree(self) -> int:
        return max((sum(k) for k in self.terms), default=0)

    def max_abs_coef(self) -> float:
        return max((abs(v) for v in self.terms.values()), default=0.0)

    def scaled(self, s: float) -> "Poly":
        return self * s

    def normalized(self) -> "Poly":
        """Divide by the largest |coefficient| (the data rescaling of Sec. 5)."""
        m = self.max_abs_coef()
        return self if m == 0.0 else self * (1.0 / m)

    def evaluate(self, z) -> float:
        z = np.asarray(z, dtype=np.float64)
        s = 0.0
        for k, v in self.terms.items():
            t = v
            for i, e in enumerate(k):
                if e:
                    t *= z[i] ** e
            s += t
        return s

    def arrays(self):
        """(coef float64[T], expo uint8[T, nv]) in a deterministic term order."""
        keys = sorted(self.terms)
        coef = np.array([self.terms[k] for k in keys], dtype=np.float64)
        expo = np.array(keys, dtype=np.uint8).reshape(len(keys), self.nv)
        return coef, expo

    def __repr__(self):
        return "Poly(%d, %r)" % (self.nv, self.terms)

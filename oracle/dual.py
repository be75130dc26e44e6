"""Forward-mode dual numbers for the oracle (test infrastructure only).

A Dual holds a value array v (real or complex) and K tangent arrays stacked on
a trailing axis, d[..., k] = dv/dtheta_k; products of two infinitesimals
vanish, so every operation propagates first derivatives exactly (to
rounding).  The class speaks enough of numpy's protocols (ufuncs, einsum,
stack, where, sum, indexing, creation with like=) for the oracle's phase
space, PDF interpolation and Feynman-diagram code to run on it unchanged,
which gives the oracle's derivatives of the integrand with respect to the
unit-cube point and the top mass.

Root finds done by bisection on values are differentiated with one Newton
step taken in dual arithmetic from the converged root (the implicit function
theorem): newton_root.
"""
from __future__ import annotations

import numpy as np

_HANDLED = {}


def _implements(func):
    def deco(f):
        _HANDLED[func] = f
        return f
    return deco


def value(x):
    return x.v if isinstance(x, Dual) else x


def as_f64(x):
    """np.asarray(x, float64) for plain inputs; dual inputs pass through
    (np.asarray is not overridable)."""
    return x if isinstance(x, Dual) else np.asarray(x, dtype=np.float64)


def _d(x, K, shape=None):
    """Tangent array of x (zeros for plain arrays and scalars)."""
    if isinstance(x, Dual):
        return x.d
    a = np.asarray(x)
    return np.zeros(a.shape + (K,), dtype=a.dtype if np.iscomplexobj(a) else np.float64)


def _k(args):
    for a in args:
        if isinstance(a, Dual):
            return a.K
    raise TypeError("no dual operand")


def _ax(axis):
    """An axis of the value array as an axis of the tangent array."""
    return axis - 1 if axis is not None and axis < 0 else axis


class Dual:
    __array_priority__ = 100

    def __init__(self, v, d):
        self.v = np.asarray(v)
        self.d = np.asarray(d)
        if self.d.shape[:-1] != self.v.shape:
            self.d = np.broadcast_to(self.d, self.v.shape + self.d.shape[-1:]).copy()

    @property
    def K(self):
        return self.d.shape[-1]

    @classmethod
    def variables(cls, values):
        """Dual inputs: K arrays, the k-th with unit tangent in direction k."""
        K = len(values)
        out = []
        for k, v in enumerate(values):
            v = np.asarray(v, dtype=np.float64)
            d = np.zeros(v.shape + (K,))
            d[..., k] = 1.0
            out.append(cls(v, d))
        return out

    # ---------------------------------------------------------------- shape
    shape = property(lambda self: self.v.shape)
    ndim = property(lambda self: self.v.ndim)
    dtype = property(lambda self: self.v.dtype)
    real = property(lambda self: Dual(self.v.real, self.d.real))
    imag = property(lambda self: Dual(self.v.imag, self.d.imag))

    def __len__(self):
        return len(self.v)

    def __repr__(self):
        return f"Dual(v={self.v!r}, K={self.K})"

    def _idx(self, idx):
        return (idx if isinstance(idx, tuple) else (idx,)) + (slice(None),)

    def __getitem__(self, idx):
        if isinstance(idx, Dual):
            idx = idx.v
        return Dual(self.v[idx], self.d[self._idx(idx)])

    def __setitem__(self, idx, val):
        if isinstance(idx, Dual):
            idx = idx.v
        if isinstance(val, Dual):
            if np.iscomplexobj(val.v) and not np.iscomplexobj(self.v):
                self.v = self.v.astype(np.complex128)
                self.d = self.d.astype(np.complex128)
            self.v[idx] = val.v
            self.d[self._idx(idx)] = val.d
        else:
            self.v[idx] = val
            self.d[self._idx(idx)] = 0.0

    def astype(self, dtype):
        return Dual(self.v.astype(dtype), self.d.astype(dtype))

    def copy(self):
        return Dual(self.v.copy(), self.d.copy())

    def reshape(self, *shape):
        shape = shape[0] if len(shape) == 1 and isinstance(shape[0], tuple) else shape
        return Dual(self.v.reshape(shape), self.d.reshape(tuple(shape) + (self.K,)))

    def conj(self):
        return Dual(np.conj(self.v), np.conj(self.d))

    conjugate = conj

    def sum(self, axis=None):
        return np.sum(self, axis=axis)

    # ---------------------------------------------------------------- arithmetic
    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __pos__(self):
        return self

    def __add__(self, o):
        K = self.K
        return Dual(self.v + value(o), self.d + _expand(o, K))

    __radd__ = __add__

    def __sub__(self, o):
        return Dual(self.v - value(o), self.d - _expand(o, self.K))

    def __rsub__(self, o):
        return Dual(value(o) - self.v, _expand(o, self.K) - self.d)

    def __mul__(self, o):
        ov = value(o)
        return Dual(self.v * ov, self.d * np.asarray(ov)[..., None] + self.v[..., None] * _expand(o, self.K))

    __rmul__ = __mul__

    def __truediv__(self, o):
        ov = np.asarray(value(o))
        q = self.v / ov
        return Dual(q, (self.d - q[..., None] * _expand(o, self.K)) / ov[..., None])

    def __rtruediv__(self, o):
        q = value(o) / self.v
        return Dual(q, (_expand(o, self.K) - q[..., None] * self.d) / self.v[..., None])

    def __pow__(self, p):
        if isinstance(p, Dual):
            raise TypeError("dual exponents are not needed")
        if p == 0:
            return Dual(np.ones_like(self.v), np.zeros_like(self.d))
        return Dual(self.v ** p, (p * self.v ** (p - 1))[..., None] * self.d)

    # comparisons act on values
    def __lt__(self, o):
        return self.v < value(o)

    def __le__(self, o):
        return self.v <= value(o)

    def __gt__(self, o):
        return self.v > value(o)

    def __ge__(self, o):
        return self.v >= value(o)

    def __eq__(self, o):
        return self.v == value(o)

    def __ne__(self, o):
        return self.v != value(o)

    __hash__ = None

    # ---------------------------------------------------------------- numpy protocols
    def __array_ufunc__(self, ufunc, method, *inputs, **kwargs):
        if method != "__call__" or kwargs.get("out") is not None:
            return NotImplemented
        K = _k(inputs)
        if ufunc.nin == 1:
            x = inputs[0]
            v, d = x.v, x.d
            if ufunc is np.negative:
                return -x
            if ufunc is np.positive:
                return x
            if ufunc is np.sqrt:
                r = np.sqrt(v)
                return Dual(r, d * (0.5 / np.where(r != 0, r, np.inf))[..., None])
            if ufunc is np.exp:
                r = np.exp(v)
                return Dual(r, d * r[..., None])
            if ufunc is np.log:
                return Dual(np.log(v), d / v[..., None])
            if ufunc is np.log1p:
                return Dual(np.log1p(v), d / (1.0 + v)[..., None])
            if ufunc is np.expm1:
                return Dual(np.expm1(v), d * np.exp(v)[..., None])
            if ufunc is np.sin:
                return Dual(np.sin(v), d * np.cos(v)[..., None])
            if ufunc is np.cos:
                return Dual(np.cos(v), -d * np.sin(v)[..., None])
            if ufunc is np.sinh:
                return Dual(np.sinh(v), d * np.cosh(v)[..., None])
            if ufunc is np.cosh:
                return Dual(np.cosh(v), d * np.sinh(v)[..., None])
            if ufunc is np.conjugate:
                return x.conj()
            if ufunc is np.square:
                return x * x
            if ufunc is np.absolute:
                if np.iscomplexobj(v):
                    raise TypeError("|z| of a complex dual is not needed")
                return Dual(np.abs(v), d * np.sign(v)[..., None])
            if ufunc in (np.floor, np.isfinite, np.isnan, np.sign, np.rint, np.ceil):
                return ufunc(v)
            raise TypeError(f"ufunc {ufunc.__name__} not supported on dual numbers")
        a, b = inputs
        if ufunc is np.add:
            return a + b if isinstance(a, Dual) else b + a
        if ufunc is np.subtract:
            return a - b if isinstance(a, Dual) else -(b - a)
        if ufunc is np.multiply:
            return a * b if isinstance(a, Dual) else b * a
        if ufunc is np.true_divide:
            return a / b if isinstance(a, Dual) else b.__rtruediv__(a)
        if ufunc is np.power:
            return a ** value(b)
        if ufunc in (np.maximum, np.minimum):
            av, bv = value(a), value(b)
            take_a = (av >= bv) if ufunc is np.maximum else (av <= bv)
            return np.where(take_a, Dual(av, _expand(a, K)), Dual(bv, _expand(b, K)))
        if ufunc in (np.greater, np.greater_equal, np.less, np.less_equal, np.equal, np.not_equal, np.arctan2,
                     np.hypot, np.logical_and, np.logical_or):
            return ufunc(value(a), value(b))
        raise TypeError(f"ufunc {ufunc.__name__} not supported on dual numbers")

    def __array_function__(self, func, types, args, kwargs):
        if func is np.zeros:                  # np.zeros(shape, like=dual): numpy drops `like`
            kwargs = {**kwargs, "like": self}
        if func in _HANDLED:
            return _HANDLED[func](*args, **kwargs)
        raise TypeError(f"{func.__name__} not supported on dual numbers")


def _expand(o, K):
    """Tangent of o broadcastable against a value-shaped array with K axis."""
    if isinstance(o, Dual):
        return o.d
    return np.zeros((1,) * np.ndim(o) + (K,))


@_implements(np.asarray)
def _asarray(a, dtype=None, **kw):
    return a if dtype is None else a.astype(dtype)


@_implements(np.broadcast_to)
def _broadcast_to(a, shape, **kw):
    shape = tuple(np.atleast_1d(shape)) if not isinstance(shape, tuple) else shape
    return Dual(np.broadcast_to(a.v, shape), np.broadcast_to(a.d, shape + (a.K,)))


def _as_dual(x, K):
    return x if isinstance(x, Dual) else Dual(np.asarray(x), _d(x, K))


@_implements(np.stack)
def _stack(arrays, axis=0, **kw):
    K = _k(arrays)
    ds = [_as_dual(a, K) for a in arrays]
    return Dual(np.stack([x.v for x in ds], axis=axis), np.stack([x.d for x in ds], axis=_ax(axis)))


@_implements(np.concatenate)
def _concatenate(arrays, axis=0, **kw):
    K = _k(arrays)
    ds = [_as_dual(a, K) for a in arrays]
    return Dual(np.concatenate([x.v for x in ds], axis=axis), np.concatenate([x.d for x in ds], axis=_ax(axis)))


@_implements(np.where)
def _where(cond, a, b):
    K = _k([a, b])
    cond = value(cond)
    av, bv = value(a), value(b)
    return Dual(np.where(cond, av, bv), np.where(np.asarray(cond)[..., None], _expand(a, K), _expand(b, K)))


@_implements(np.sum)
def _sum(a, axis=None, **kw):
    if axis is None:
        return Dual(np.sum(a.v), a.d.reshape(-1, a.K).sum(axis=0))
    return Dual(np.sum(a.v, axis=axis), np.sum(a.d, axis=_ax(axis)))


@_implements(np.prod)
def _prod(a, axis=None, **kw):
    p = np.prod(a.v, axis=axis, keepdims=True)
    dp = np.sum((p / a.v)[..., None] * a.d, axis=_ax(axis), keepdims=False) if axis is not None else None
    return Dual(np.prod(a.v, axis=axis), dp)


@_implements(np.real)
def _real(a):
    return a.real


@_implements(np.imag)
def _imag(a):
    return a.imag


@_implements(np.conj)
def _conj(a):
    return a.conj()


@_implements(np.zeros_like)
def _zeros_like(a, dtype=None, **kw):
    v = np.zeros_like(a.v, dtype=dtype)
    return Dual(v, np.zeros(v.shape + (a.K,), dtype=v.dtype))


@_implements(np.empty_like)
def _empty_like(a, dtype=None, **kw):
    return _zeros_like(a, dtype=dtype)


@_implements(np.ones_like)
def _ones_like(a, dtype=None, **kw):
    v = np.ones_like(a.v, dtype=dtype)
    return Dual(v, np.zeros(v.shape + (a.K,), dtype=v.dtype))


@_implements(np.zeros)
def _zeros(shape, dtype=float, like=None, **kw):
    v = np.zeros(shape, dtype=dtype)
    return Dual(v, np.zeros(v.shape + (like.K,), dtype=v.dtype))


@_implements(np.full_like)
def _full_like(a, fill, dtype=None, **kw):
    v = np.full_like(a.v, value(fill), dtype=dtype)
    return Dual(v, np.broadcast_to(_expand(fill, a.K), v.shape + (a.K,)).astype(v.dtype))


@_implements(np.einsum)
def _einsum(subscripts, *operands, **kw):
    if not isinstance(subscripts, str) or "->" not in subscripts or "." in subscripts:
        raise TypeError("explicit einsum subscripts without ellipses are needed for dual numbers")
    ins, out = subscripts.split("->")
    ins = ins.split(",")
    K = _k(operands)
    vals = [value(o) for o in operands]
    v = np.einsum(subscripts, *vals)
    d = None
    for i, o in enumerate(operands):
        if not isinstance(o, Dual):
            continue
        sub = ",".join(s + "Z" if j == i else s for j, s in enumerate(ins)) + "->" + out + "Z"
        term = np.einsum(sub, *[o.d if j == i else vals[j] for j in range(len(operands))])
        d = term if d is None else d + term
    return Dual(v, d)


@_implements(np.nonzero)
def _nonzero(a):
    return np.nonzero(a.v)


@_implements(np.any)
def _any(a, **kw):
    return np.any(a.v, **kw)


@_implements(np.all)
def _all(a, **kw):
    return np.all(a.v, **kw)


@_implements(np.shape)
def _shape(a):
    return a.v.shape


@_implements(np.iscomplexobj)
def _iscomplexobj(a):
    return np.iscomplexobj(a.v)


@_implements(np.atleast_1d)
def _atleast_1d(a):
    return a if a.ndim >= 1 else a.reshape(1)


@_implements(np.searchsorted)
def _searchsorted(a, v, side="left", **kw):
    return np.searchsorted(value(a), value(v), side=side)


@_implements(np.choose)
def _choose(idx, choices, **kw):
    K = _k(choices)
    idx = value(idx)
    v = np.choose(idx, [value(c) for c in choices])
    d = np.choose(np.asarray(idx)[..., None], [_expand(c, K) * np.ones(np.shape(value(c)) + (1,))
                                                 for c in choices])
    return Dual(v, d)


@_implements(np.clip)
def _clip(a, lo, hi, **kw):
    inside = (a.v >= lo) & (a.v <= hi)
    return Dual(np.clip(a.v, lo, hi), np.where(inside[..., None], a.d, 0.0))


def newton_root(F, dF, x0):
    """Dual root of F(x) = 0 from its converged value x0 (an ndarray): one
    Newton step in dual arithmetic, x0 - F(x0) / F'(x0), whose tangent is the
    implicit derivative -F_theta / F_x."""
    f = F(x0)
    if not isinstance(f, Dual):
        return x0
    return x0 - f / value(dF(x0))

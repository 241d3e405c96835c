"""CPU reference evaluator of interaction-law systems ("oracle", test
infrastructure only: tests/, __graft_entry__.smoke() and bench.py's CPU leg).

It evaluates the same equation strings as the GPU law compiler, in FP64 and
independently of it: each right-hand side is evaluated by Python over numpy
arrays, with every field a per-particle array and, for pair expressions,
X_i / X_j / r_ij / d_ij / W_ij / gradW_ij arrays over all neighbour-image
pairs; sum_j and the SPH operators reduce pair arrays to particles.  The
neighbour images come from the C oracle (sph_oracle_bc.c, Section 3.2.1).

Operators, as the paper defines them (Section 5.1, Eq. diffop1 to
Eq. diffop3; grad W = grad_i W_ij of the Wendland kernel of Section 5.1.1):
  sph_S(A, m, rho) = sum_j A_j m_j/rho_j W_ij, i itself included
  sph_G(A, m, rho) = rho_i sum_j (A_i/rho_i^2 + A_j/rho_j^2) m_j grad W    (diffop1)
  sph_D(A, m, rho) = sum_j (A_j - A_i) m_j/rho_j grad W                    (diffop2)
                     (a vector A: the divergence, (A_j - A_i) . grad W)
  sph_L(A, m, rho) = sum_j 2 m_j/rho_j (A_i - A_j) (r_ij . grad W)/|r_ij|^2  (diffop3)
  sph_A(v, m, rho) = sum_j m_j min(v_ij . r_ij, 0)/(rho_i |r_ij|^2) grad W
                     (Appendix A's viscosity operator: 0.1 c h sph_A is the
                     -sum_j m_j Pi_ij grad W of Section 5.1.1)
The operators may also be written as in the paper's listings, op(A, m, rho,
Wp52220, 2*h) with sph_D00 = sph_D, sph_G11 = sph_G, sph_L0 = sph_L (the
kernel keyword must name the Wendland kernel and the radius must be 2h),
and ^ is the power operator.
Readings of the paper taken here: diffop3 as printed has no volume; the operator's
arguments (m, rho) supply m_j/rho_j, and r_ij = r_i - r_j so that a
minimum has a positive Laplacian; the kernel and radius are the context's
(Wendland, 2h) rather than an argument.
"""
from __future__ import annotations

import ast
import math

import numpy as np

from . import oracle as O


class Q:
    """A per-particle or per-pair value: shape (N,) scalar, (N, 3) vector;
    vector constants are (1, 3).  const marks values that hold for every
    particle (constants and expressions of constants only): they are neither
    gathered nor reflected at a neighbour's image, whatever N is."""

    __array_priority__ = 100

    def __init__(self, a, const=False):
        self.a = np.asarray(a, np.float64)
        self.const = const

    @staticmethod
    def _c(*xs):
        return all(x.const if isinstance(x, Q) else True for x in xs)

    @property
    def vec(self):
        return self.a.ndim == 2

    @staticmethod
    def _v(x):
        return x.a if isinstance(x, Q) else np.float64(x)

    def _pair(self, o):
        a, b = self.a, Q._v(o)
        isv_a = a.ndim == 2
        isv_b = np.ndim(b) == 2
        if isv_a and not isv_b and np.ndim(b) == 1:
            b = b[:, None]
        if isv_b and not isv_a and a.ndim == 1:
            a = a[:, None]
        return a, b

    def __add__(self, o):
        a, b = self._pair(o)
        return Q(a + b, Q._c(self, o))

    __radd__ = __add__

    def __sub__(self, o):
        a, b = self._pair(o)
        return Q(a - b, Q._c(self, o))

    def __rsub__(self, o):
        a, b = self._pair(o)
        return Q(b - a, Q._c(self, o))

    def __mul__(self, o):
        a, b = self._pair(o)
        return Q(a * b, Q._c(self, o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        a, b = self._pair(o)
        return Q(a / b, Q._c(self, o))

    def __rtruediv__(self, o):
        a, b = self._pair(o)
        return Q(b / a, Q._c(self, o))

    def __neg__(self):
        return Q(-self.a, self.const)

    def __pow__(self, e):
        return Q(self.a ** Q._v(e), Q._c(self, e))


_WENDLAND = object()  # the kernel keyword Wp52220 of the paper's listings


def _q(x):
    return x if isinstance(x, Q) else Q(x, True)


def _fn(f):
    return lambda x: Q(f(_q(x).a), Q._c(x))


class Pairs:
    """Neighbour images of the particles at r (input order)."""

    def __init__(self, p, case, r, ids):
        offs, nid, codes = O.bc_neighbours(p, r, ids)
        n = r.shape[0]
        inv = np.empty(int(ids.max()) + 1, np.int64)
        inv[ids] = np.arange(n)
        self.I = np.repeat(np.arange(n), np.diff(offs))
        self.J = inv[nid]
        D = case.dim
        rel = np.zeros((self.I.size, 3))
        vs = np.ones((self.I.size, 3))
        for k in range(D):
            t = (codes.astype(np.int64) // 3 ** k) % 3
            xi, xj = r[self.I, k], r[self.J, k]
            L = case.ncell[k] * case.cs
            lo = case.dom_min[k]
            hi = lo + L
            x = xi - xj
            if case.bc[k] == 2:      # periodic
                x = np.where(t == 1, (xi + L) - xj, np.where(t == 2, (xi - L) - xj, x))
            elif case.bc[k] == 1:    # symmetric
                x = np.where(t == 1, (xi - 2 * lo) + xj, np.where(t == 2, (xi - 2 * hi) + xj, x))
                vs[:, k] = np.where(t == 0, 1.0, -1.0)
            rel[:, k] = x
        self.rel = rel
        self.vs = vs
        self.mirror = (vs < 0).any(axis=1).astype(np.float64)   # j seen through a symmetric face
        self.d = np.sqrt((rel * rel).sum(1))
        h = case.h
        aD = O.alpha_D(D, h)
        q = self.d / h
        t = 1.0 - 0.5 * q
        self.W = aD * t ** 4 * (2.0 * q + 1.0)
        # grad_i W_ij = (dW/dr) r_ij / |r_ij|, dW/dr = -5 aD (q/h) t^3
        self.gW = (-5.0 * aD / (h * h) * t ** 3)[:, None] * rel
        self.W0 = aD
        self.n = n

    def reduce(self, x):
        x = _q(x).a
        if x.ndim == 0:
            x = np.full(self.I.size, float(x))
        if x.ndim == 1:
            return Q(np.bincount(self.I, weights=x, minlength=self.n))
        out = np.zeros((self.n, 3))
        for k in range(3):
            out[:, k] = np.bincount(self.I, weights=x[:, k], minlength=self.n)
        return Q(out)

    def at_i(self, x):
        q = _q(x)
        if q.const:
            return q
        return Q(q.a[self.I])

    def at_j(self, x):
        q = _q(x)
        if q.const:
            return q
        if q.a.ndim == 2:
            return Q(q.a[self.J] * self.vs)
        return Q(q.a[self.J])


def _dot(a, b):
    return Q((_q(a).a * _q(b).a).sum(-1), Q._c(a, b))


def _where(c, a, b):
    """where(c, a, b): a where c != 0, else b (per particle)."""
    c, a, b = _q(c).a, _q(a).a, _q(b).a
    if (a.ndim == 2 or b.ndim == 2) and c.ndim == 1:
        c = c[:, None]
    return Q(np.where(c != 0, a, b))


def _vec(*c):
    vals = [Q._v(x) for x in c]
    shape = np.broadcast_shapes(*[np.shape(v) for v in vals])
    comps = [np.broadcast_to(v, shape) for v in vals] + [np.zeros(shape)] * (3 - len(vals))
    out = np.stack(comps, -1)
    return Q(out.reshape(1, 3) if out.ndim == 1 else out, Q._c(*c))


class LawOracle:
    """The system on the CPU: fields in the case's particle order."""

    def __init__(self, case, fields, constants, equations, fp32_neighbours=False, variables=None):
        self.case = case
        # global scalars: an equation with one on its left-hand side gives a
        # single value; fmax / fmin / fsum reduce a per-particle value over
        # all particles
        self.vars = {k: float(v) for k, v in (variables or {}).items()}
        self.D = case.dim
        self.p = O.bc_params(case, fp32=fp32_neighbours)
        self.r = np.array(case.r, np.float64)
        self.ids = np.asarray(case.id, np.uint32)
        self.consts = {}
        for k, v in constants.items():
            if isinstance(v, (tuple, list, np.ndarray)):
                c = np.zeros((1, 3))
                c[0, :len(v)] = v
                self.consts[k] = Q(c, True)
            else:
                self.consts[k] = float(v)
        self.fields = {}
        self.kind = {}
        for name, (kind, vals) in fields.items():
            a = np.asarray(vals, np.float64)
            if kind == "vector":
                b = np.zeros((a.shape[0], 3))
                b[:, :self.D] = a.reshape(a.shape[0], -1)[:, :self.D]
                a = b
            self.fields[name] = Q(a)
            self.kind[name] = kind
        self.eqs = []
        for t in equations:
            lhs, rhs = (s.strip() for s in t.split("=", 1))
            rhs = rhs.replace("^", "**")       # the paper's power operator
            self.eqs.append((lhs, compile(ast.parse(rhs, mode="eval"), "<law>", "eval")))
        self.pairs = None

    def _pairs(self):
        if self.pairs is None:
            self.pairs = Pairs(self.p, self.case, self.r, self.ids)
        return self.pairs

    def _ops(self, P):
        def S_(A, m, rho):
            w = P.at_j(_q(A)) * (P.at_j(m) / P.at_j(rho)) * Q(P.W)
            return P.reduce(w) + _q(A) * (_q(m) / _q(rho)) * P.W0

        def G_(A, m, rho):
            Ai, Aj, ri, rj, mj = P.at_i(A), P.at_j(A), P.at_i(rho), P.at_j(rho), P.at_j(m)
            return _q(rho) * P.reduce(Q(P.gW) * ((Ai / (ri * ri) + Aj / (rj * rj)) * mj))

        def D_(A, m, rho):
            Ai, Aj, mj, rj = P.at_i(A), P.at_j(A), P.at_j(m), P.at_j(rho)
            if _q(A).vec:
                return P.reduce(_dot(Aj - Ai, Q(P.gW)) * (mj / rj))
            return P.reduce(Q(P.gW) * ((Aj - Ai) * (mj / rj)))

        def L_(A, m, rho):
            Ai, Aj, mj, rj = P.at_i(A), P.at_j(A), P.at_j(m), P.at_j(rho)
            return P.reduce(2.0 * (mj / rj) * (Ai - Aj) * _dot(Q(P.rel), Q(P.gW)) / Q(P.d * P.d))

        def A_(v, m, rho):
            vij = P.at_i(v) - P.at_j(v)
            vr = np.minimum(_dot(vij, Q(P.rel)).a, 0.0)
            return P.reduce(Q(P.gW) * (P.at_j(m) * Q(vr) / (P.at_i(rho) * Q(P.d * P.d))))

        h2 = 2.0 * float(self.case.h)

        def paper(fn, name):
            # the paper's form op(A, m, rho, Wp52220, 2*h): the kernel keyword
            # names the Wendland kernel, the radius must be the case's 2h
            def op(A, m, rho, kernel=None, radius=None):
                if kernel is not None or radius is not None:
                    if kernel is not _WENDLAND:
                        raise ValueError(f"{name}: unknown kernel")
                    if abs(float(radius) - h2) > 1e-12 * h2:
                        raise ValueError(f"{name}: radius {radius} is not 2h = {h2}")
                return fn(A, m, rho)
            return op

        ops = {"sph_S": S_, "sph_G": G_, "sph_D": D_, "sph_L": L_, "sph_A": A_}
        out = {k: paper(f, k) for k, f in ops.items()}
        out.update({"sph_D00": paper(D_, "sph_D00"), "sph_G11": paper(G_, "sph_G11"),
                    "sph_L0": paper(L_, "sph_L0"), "sum_j": P.reduce})
        return out

    def _namespace(self, code):
        ns = {"__builtins__": {}}
        ns.update(self.consts)
        ns["h"] = float(self.case.h)
        ns.update({"sqrt": _fn(np.sqrt), "exp": _fn(np.exp), "log": _fn(np.log), "abs": _fn(np.abs),
                   "sin": _fn(np.sin), "cos": _fn(np.cos), "tanh": _fn(np.tanh),
                   "min": lambda a, b: Q(np.minimum(Q._v(a), Q._v(b)), Q._c(a, b)),
                   "max": lambda a, b: Q(np.maximum(Q._v(a), Q._v(b)), Q._c(a, b)),
                   "pow": lambda a, b: Q(Q._v(a) ** Q._v(b), Q._c(a, b)), "dot": _dot,
                   "norm": lambda a: Q(np.sqrt((_q(a).a ** 2).sum(-1)), Q._c(a)),
                   "vec": _vec,
                   "euler": lambda x, xd, c: _q(x) + _q(xd) * c,
                   "where": _where})
        ns.update(self.vars)
        rr = np.zeros((self.r.shape[0], 3))
        rr[:, :self.D] = self.r
        ns["r"] = Q(rr)                      # the particle's own position
        ns.update({"fmax": lambda x: float(np.max(_q(x).a)), "fmin": lambda x: float(np.min(_q(x).a)),
                   "fsum": lambda x: float(np.sum(_q(x).a))})
        ns.update(self.fields)
        ns["Wp52220"] = _WENDLAND
        names = set(code.co_names)
        if names & {"sph_S", "sph_G", "sph_D", "sph_L", "sph_A", "sum_j", "sph_D00", "sph_G11", "sph_L0"}:
            P = self._pairs()
            ns.update(self._ops(P))
            ns["r_ij"], ns["d_ij"], ns["W_ij"], ns["gradW_ij"] = Q(P.rel), Q(P.d), Q(P.W), Q(P.gW)
            ns["mirror_ij"] = Q(P.mirror)
            for f, val in self.fields.items():
                ns[f + "_i"] = P.at_i(val)
                ns[f + "_j"] = P.at_j(val)
        return ns

    def step(self, nsteps=1):
        for _ in range(nsteps):
            for lhs, code in self.eqs:
                if lhs == "r":
                    # r = euler(r, V, c): evaluate the increment V c (V may
                    # read the current positions)
                    tree = code
                    ns = self._namespace(tree)
                    ns["euler"] = lambda x, xd, c: _q(xd) * c
                    dr = eval(tree, ns).a
                    for k in range(self.D):
                        x = self.r[:, k] + dr[:, k]
                        if self.case.bc[k] == 2:
                            lo = self.case.dom_min[k]
                            L = self.case.ncell[k] * self.case.cs
                            x = np.where(x < lo, x + L, np.where(x >= lo + L, x - L, x))
                        self.r[:, k] = x
                    self.pairs = None
                    continue
                val = eval(code, self._namespace(code))
                if lhs in self.vars:
                    self.vars[lhs] = float(np.asarray(_q(val).a).reshape(-1)[0])
                    continue
                val = _q(val)
                if self.kind[lhs] == "vector":
                    a = np.broadcast_to(val.a, (self.r.shape[0], 3)).copy()
                    a[:, self.D:] = 0.0
                else:
                    a = np.broadcast_to(val.a, (self.r.shape[0],)).copy()
                self.fields[lhs] = Q(a)

"""Interaction laws compiled to GB300 kernels.

The paper's general form (Section 2.1, Eq. general_interaction and
Eq. interaction_formula): a field update is a particle-wise expression plus
pair sums Psi_i = sum_j I(Phi_i, Phi_j) over the neighbours within an
influence radius.  Nauticle interprets such equations at run time through
its SFL expression tree (Section 3.1) and lists their "generation and runtime
compilation" as its first planned improvement (Section 7).  This module does
that for the GPU: a system of fields, constants and ordered equations written
in the style of Appendix A is parsed, typed, turned into CUDA source,
compiled with nvcc for sm_103a into a shared library (cached by content) and
launched through ctypes on the cells and sorted copy of a SPH_MODEL_FIELDS
context (sph_law_view).  Consecutive equations share one kernel
(group_equations): their pair sums run in one pass over the neighbour
images, and each later equation of the kernel takes the earlier results
from registers.

Language (one equation per string, "lhs = expr"):

* names: fields (scalar or vector), constants (numbers or vectors), h (the
  context's smoothing length), variables (global scalars), r (the
  particle's own position, outside pair sums; positions change only by
  "r = euler(r, V, c)");
* arithmetic + - * / and ** (constant exponent), functions sqrt exp log abs
  sin cos tanh min max pow, dot(a, b), norm(a), vec(x, y[, z]), euler(x, x',
  c) = x + c x', where(c, a, b) = a where c != 0 else b (when every pair
  equation of a kernel is where(c, <sums>, b), the neighbour walk is skipped
  for the particles whose c are all zero);
* interaction operators over the neighbour images of i within 2h (i itself
  excluded unless stated), kernel W = Wendland (Section 5.1.1) with the
  context's h, grad W = grad_i W_ij:
    sph_S(A, m, rho) = sum_j A_j m_j/rho_j W_ij + A_i m_i/rho_i W(0)   (sampling)
    sph_G(A, m, rho) = rho_i sum_j (A_i/rho_i^2 + A_j/rho_j^2) m_j grad W   (Eq. diffop1)
    sph_D(A, m, rho) = sum_j (A_j - A_i) m_j/rho_j grad W   (Eq. diffop2; a
                       vector A gives the divergence, (A_j - A_i) . grad W)
    sph_L(A, m, rho) = sum_j 2 m_j/rho_j (A_i - A_j) (r_ij . grad W) / |r_ij|^2
                       (Eq. diffop3 with the volumes m_j/rho_j, r_ij = r_i - r_j)
    sph_A(v, m, rho) = sum_j m_j min(v_ij . r_ij, 0) / (rho_i |r_ij|^2) grad W
                       (the viscosity sum of Appendix A: 0.1 c h sph_A is
                       -sum_j m_j Pi_ij grad W of Section 5.1.1)
    sum_j(body)      = sum over the images of any pair expression body, in
                       which X_i and X_j name field X at i and at the image
                       of j (vector fields reflected across symmetric faces),
                       and r_ij, d_ij = |r_ij|, W_ij, gradW_ij are the pair's;
                       mirror_ij = 1 when j is seen through a symmetric
                       face (a wall image), else 0.
The operators may also be written in the form of the paper's listings,
op(A, m, rho, Wp52220, 2*h) with sph_D00, sph_G11, sph_L0 and sph_A, and ^
is the power operator (PAPER_OPERATORS).
Equations run in order, each for all particles before the next (Section
3.3); fusion keeps that meaning, since a pair sum never joins a kernel that
has already written a field it reads.  A kernel writes second buffers,
swapped in after it.  After "r = euler(...)" the next pair equation rebuilds
the cells and reorders with the particles the fields read before they are
written again (live_at_rebuild).
"""
from __future__ import annotations

import ast
import ctypes as C
import hashlib
import os
import platform
import subprocess
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build
from . import sph as S

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")

SCALAR, VECTOR = "S", "V"
FUNCS1 = {"sqrt": "sqrt", "exp": "exp", "log": "log", "abs": "fabs", "sin": "sin", "cos": "cos", "tanh": "tanh"}
OPERATORS = ("sph_S", "sph_G", "sph_D", "sph_L", "sph_A", "sum_j")
# The operator names of the paper's equation listings (Appendix A, Example
# 1b), written with the kernel keyword and the influence radius as trailing
# arguments: op(A, m, rho, Wp52220, 2*h).  Wp52220 is read as the Wendland
# kernel of Section 5.1.1 and 2*h as the context's radius: the only kernel
# and radius the compiled operators take.
PAPER_OPERATORS = {"sph_D00": "sph_D", "sph_G11": "sph_G", "sph_L0": "sph_L", "sph_A": "sph_A"}
PAPER_KERNEL = "Wp52220"
# reductions over all particles, allowed in the equations of variables
REDUCTIONS = ("fmax", "fmin", "fsum")


def _is_two_h(node) -> bool:
    """2*h or h*2 (the context's influence radius)."""
    if not (isinstance(node, ast.BinOp) and isinstance(node.op, ast.Mult)):
        return False
    a, b = node.left, node.right
    two = lambda x: isinstance(x, ast.Constant) and x.value == 2
    hh = lambda x: isinstance(x, ast.Name) and x.id == "h"
    return (two(a) and hh(b)) or (hh(a) and two(b))


class _PaperForm(ast.NodeTransformer):
    """Rewrite op(A, m, rho, Wp52220, 2*h) of the paper's listings into the
    compiled operator op'(A, m, rho)."""

    def visit_Call(self, node):
        self.generic_visit(node)
        if isinstance(node.func, ast.Name) and len(node.args) == 5 and (
                node.func.id in PAPER_OPERATORS or node.func.id in OPERATORS):
            name = PAPER_OPERATORS.get(node.func.id, node.func.id)
            kern, rad = node.args[3], node.args[4]
            if not (isinstance(kern, ast.Name) and kern.id == PAPER_KERNEL):
                raise LawError(f"{node.func.id}: the only kernel is {PAPER_KERNEL} (Wendland, Section 5.1.1)")
            if not _is_two_h(rad):
                raise LawError(f"{node.func.id}: the influence radius must be 2*h (the context's)")
            return ast.copy_location(ast.Call(func=ast.Name(id=name, ctx=ast.Load()), args=node.args[:3],
                                              keywords=[]), node)
        return node


def _has_pair_sum(node) -> bool:
    """Whether an expression tree calls a pair operator."""
    return any(isinstance(x, ast.Call) and isinstance(x.func, ast.Name) and x.func.id in OPERATORS
               for x in ast.walk(node))


def _parse_rhs(rhs: str):
    """The right-hand side as an expression tree: the paper's power operator
    ^ is read as **, and its operator forms are rewritten (_PaperForm)."""
    tree = ast.parse(rhs.replace("^", "**"), mode="eval").body
    return _PaperForm().visit(tree)
# inside sum_j: the pair's separation, distance, kernel value and gradient,
# and mirror_ij = 1 when j is seen through a symmetric face (a wall image)
PAIR_NAMES = {"r_ij": VECTOR, "d_ij": SCALAR, "W_ij": SCALAR, "gradW_ij": VECTOR, "mirror_ij": SCALAR}


class LawError(ValueError):
    pass


@dataclass
class Acc:
    """One pair sum of an equation."""
    name: str
    kind: str        # SCALAR / VECTOR
    body: str        # per-pair increment (pair scope)
    result: str      # its value in the epilogue


@dataclass
class Eq:
    index: int
    lhs: str
    kind: str        # "pair", "local" or "move"
    accs: List[Acc]
    rhs: str         # epilogue expression (particle scope)
    rhs_kind: str
    reads: List[str]  # fields read
    tree: object = None           # the right-hand side (ast)
    pair_reads: List[str] = field(default_factory=list)   # fields read inside its pair sums
    reds: List[Tuple[str, str]] = field(default_factory=list)  # a variable's reductions


class _Emitter:
    """Typed code generation for one equation."""

    def __init__(self, fields: Dict[str, str], consts: Dict[str, object], dim: int,
                 locals_map: Optional[Dict[str, str]] = None, prefix: str = "acc",
                 variables: Optional[Dict[str, int]] = None, var_mode: bool = False):
        self.fields = fields
        self.consts = consts
        self.dim = dim
        self.accs: List[Acc] = []
        self.reads = set()        # fields read from memory
        self.pair_reads = set()   # fields read inside pair sums
        self.locals = locals_map or {}
        self.prefix = prefix
        self._in_pair = False
        # global scalar variables (name -> slot of the device array), and for
        # a variable's equation its reductions over the particles
        self.variables = variables or {}
        self.var_mode = var_mode
        self.reds: List[Tuple[str, str]] = []   # (fmax | fmin | fsum, particle expression)
        self._in_red = False
        self.reads_r = False      # the particle's own position is read

    # -- helpers -------------------------------------------------------------
    def _lit(self, x) -> Tuple[str, str]:
        if isinstance(x, (tuple, list, np.ndarray)):
            c = [float(v) for v in x] + [0.0] * (3 - len(x))
            return VECTOR, f"V3{{(T){c[0]!r}, (T){c[1]!r}, (T){c[2]!r}}}"
        return SCALAR, f"((T){float(x)!r})"

    def _field(self, name: str, side: str) -> Tuple[str, str]:
        kind = self.fields[name]
        if side == "i" and not self._in_pair and name in self.locals:
            return kind, self.locals[name]          # written earlier in the kernel
        self.reads.add(name)
        if self._in_pair:
            self.pair_reads.add(name)
        idx = "i" if side == "i" else "j"
        if kind == SCALAR:
            return SCALAR, f"a.f_{name}[{idx}]"      # (f_: clear of the generated code's names)
        comps = [f"a.f_{name}_{k}[{idx}]" if k < self.dim else "(T)0" for k in range(3)]
        if side == "j":
            comps = [f"msign(ic, {k}) * {c}" if k < self.dim else c for k, c in enumerate(comps)]
        return VECTOR, "V3{" + ", ".join(comps) + "}"

    @staticmethod
    def _bin(op, a, b):
        (ka, ca), (kb, cb) = a, b
        if op in ("+", "-"):
            if ka != kb:
                raise LawError(f"cannot {op} a scalar and a vector")
            return ka, f"({ca} {op} {cb})"
        if op == "*":
            if ka == VECTOR and kb == VECTOR:
                raise LawError("vector * vector: use dot()")
            return (VECTOR if VECTOR in (ka, kb) else SCALAR), f"({ca} * {cb})"
        if op == "/":
            if kb == VECTOR:
                raise LawError("division by a vector")
            if ka == VECTOR:
                return ka, f"({ca} * dv((T)1, {cb}))"
            return ka, f"dv({ca}, {cb})"
        raise LawError(f"operator {op}")

    # -- the walk ------------------------------------------------------------
    def emit(self, node, scope: str) -> Tuple[str, str]:
        """scope: 'p' (particle), 'i' / 'j' (an argument evaluated at i or at
        the image of j, inside a pair sum), 'pair' (a sum_j body).  Inside a
        pair sum every field is read from memory (a value written earlier in
        the same kernel is not visible to the other particles)."""
        if isinstance(node, ast.Constant) and isinstance(node.value, (int, float)):
            return self._lit(node.value)
        if isinstance(node, ast.Name):
            return self._name(node.id, scope)
        if isinstance(node, ast.UnaryOp) and isinstance(node.op, (ast.USub, ast.UAdd)):
            k, c = self.emit(node.operand, scope)
            return k, (f"(-{c})" if isinstance(node.op, ast.USub) else c)
        if isinstance(node, ast.BinOp):
            if isinstance(node.op, ast.Pow):
                k, c = self.emit(node.left, scope)
                if k != SCALAR:
                    raise LawError("power of a vector")
                e = node.right
                if isinstance(e, ast.Constant) and float(e.value).is_integer() and 1 <= e.value <= 4:
                    return SCALAR, "(" + " * ".join([c] * int(e.value)) + ")"
                ke, ce = self.emit(e, scope)
                if ke != SCALAR:
                    raise LawError("a vector exponent")
                return SCALAR, f"pow({c}, {ce})"
            ops = {ast.Add: "+", ast.Sub: "-", ast.Mult: "*", ast.Div: "/"}
            op = ops.get(type(node.op))
            if op is None:
                raise LawError("unsupported operator")
            return self._bin(op, self.emit(node.left, scope), self.emit(node.right, scope))
        if isinstance(node, ast.Call) and isinstance(node.func, ast.Name):
            return self._call(node.func.id, node.args, scope)
        raise LawError(f"unsupported expression: {ast.dump(node)[:80]}")

    def _name(self, name: str, scope: str) -> Tuple[str, str]:
        if name in self.consts:
            return self._lit(self.consts[name])
        if name == "h":
            return SCALAR, "((T)P.h)"
        if name in self.variables:
            return SCALAR, f"((T)vars[{self.variables[name]}])"
        if self.var_mode and not self._in_red and name in self.fields:
            raise LawError(f"{name}: a variable's equation reads fields only inside fmax / fmin / fsum")
        if scope in ("pair",):
            if name in PAIR_NAMES:
                return PAIR_NAMES[name], {"r_ij": "rij", "d_ij": "dij", "W_ij": "Wij", "gradW_ij": "gWij",
                                          "mirror_ij": "mirr"}[name]
            for side in ("i", "j"):
                if name.endswith("_" + side) and name[:-2] in self.fields:
                    return self._field(name[:-2], side)
            if name in self.fields:
                raise LawError(f"inside sum_j write {name}_i or {name}_j")
        if name in self.fields:
            return self._field(name, "i" if scope in ("p", "i") else "j")
        if name == "r" and scope in ("p", "i") and not self._in_pair and (self._in_red or not self.var_mode):
            # the particle's position (in the working precision; a periodic
            # axis gives the wrapped coordinate)
            self.reads_r = True
            comps = [f"(T)a.r_{k}[i]" if k < self.dim else "(T)0" for k in range(3)]
            return VECTOR, "V3{" + ", ".join(comps) + "}"
        if name in PAIR_NAMES or name == "r":
            raise LawError(f"{name} is only available inside sum_j" if name != "r" else
                           "r: the own position only, outside pair sums (r_ij inside them)")
        raise LawError(f"unknown name {name}")

    def _call(self, f: str, args, scope: str) -> Tuple[str, str]:
        if f in REDUCTIONS:
            if not self.var_mode or self._in_red:
                raise LawError(f"{f}: reductions over the particles belong in a variable's equation, unnested")
            if len(args) != 1:
                raise LawError(f"{f} takes one argument")
            self._in_red = True
            try:
                k, c = self.emit(args[0], "p")
            finally:
                self._in_red = False
            if k != SCALAR:
                raise LawError(f"{f} of a vector")
            self.reds.append((f, c))
            return SCALAR, f"red{len(self.reds) - 1}"
        if f in OPERATORS:
            if scope != "p":
                raise LawError(f"{f} cannot be nested in another pair sum")
            if self.var_mode:
                raise LawError(f"{f} in a variable's equation: compute it into a field first")
            return self._operator(f, args)
        if f in FUNCS1:
            k, c = self.emit(args[0], scope)
            if k != SCALAR:
                raise LawError(f"{f} of a vector")
            return SCALAR, f"{FUNCS1[f]}({c})"
        if f in ("min", "max", "pow"):
            (ka, ca), (kb, cb) = self.emit(args[0], scope), self.emit(args[1], scope)
            if ka != SCALAR or kb != SCALAR:
                raise LawError(f"{f} of a vector")
            return SCALAR, f"{ {'min': 'fmin', 'max': 'fmax', 'pow': 'pow'}[f] }({ca}, {cb})"
        if f == "dot":
            (ka, ca), (kb, cb) = self.emit(args[0], scope), self.emit(args[1], scope)
            if ka != VECTOR or kb != VECTOR:
                raise LawError("dot of scalars")
            return SCALAR, f"dot3({ca}, {cb})"
        if f == "norm":
            k, c = self.emit(args[0], scope)
            return SCALAR, f"sqrt(dot3({c}, {c}))"
        if f == "vec":
            comps = [self.emit(a, scope) for a in args]
            if any(k != SCALAR for k, _ in comps) or not 2 <= len(comps) <= 3:
                raise LawError("vec takes 2 or 3 scalars")
            cs = [c for _, c in comps] + ["(T)0"] * (3 - len(comps))
            return VECTOR, "V3{" + ", ".join(cs) + "}"
        if f == "euler":
            x, xd, c = (self.emit(a, scope) for a in args)
            if c[0] != SCALAR:
                raise LawError("euler: the step must be a scalar")
            return self._bin("+", x, self._bin("*", xd, c))
        if f == "where":
            if len(args) != 3:
                raise LawError("where(c, a, b) takes three arguments")
            (kc, cc), (ka, ca), (kb, cb) = (self.emit(a, scope) for a in args)
            if kc != SCALAR or ka != kb:
                raise LawError("where(c, a, b): a scalar condition and two values of one kind")
            return ka, f"(({cc}) != (T)0 ? ({ca}) : ({cb}))"
        raise LawError(f"unknown function {f}")

    def _operator(self, f: str, args) -> Tuple[str, str]:
        name = f"{self.prefix}{len(self.accs)}"
        self._in_pair = True
        try:
            return self._operator_body(f, args, name)
        finally:
            self._in_pair = False

    def _operator_body(self, f: str, args, name: str) -> Tuple[str, str]:
        if f == "sum_j":
            k, body = self.emit(args[0], "pair")
            self.accs.append(Acc(name, k, body, name))
            return k, name
        if len(args) != 3:
            raise LawError(f"{f}(A, m, rho) takes three arguments")
        Ai, mi, ri = (self.emit(a, "i") for a in args)
        Aj, mj, rj = (self.emit(a, "j") for a in args)
        if mi[0] != SCALAR or ri[0] != SCALAR:
            raise LawError(f"{f}: m and rho must be scalars")
        A_i, m_i, r_i, A_j, m_j, r_j = Ai[1], mi[1], ri[1], Aj[1], mj[1], rj[1]
        kA = Ai[0]
        if f == "sph_S":
            body = f"({A_j} * (dv({m_j}, {r_j}) * Wij))"
            self.accs.append(Acc(name, kA, body, f"({name} + {A_i} * (dv({m_i}, {r_i}) * (T)P.alphaD))"))
            return kA, self.accs[-1].result
        if f == "sph_G":
            if kA != SCALAR:
                raise LawError("sph_G of a vector")
            body = f"(gWij * ((dv({A_i}, {r_i} * {r_i}) + dv({A_j}, {r_j} * {r_j})) * {m_j}))"
            self.accs.append(Acc(name, VECTOR, body, f"({r_i} * {name})"))
            return VECTOR, self.accs[-1].result
        if f == "sph_D":
            if kA == SCALAR:
                body = f"(gWij * (({A_j} - {A_i}) * dv({m_j}, {r_j})))"
                self.accs.append(Acc(name, VECTOR, body, name))
                return VECTOR, name
            body = f"(dot3({A_j} - {A_i}, gWij) * dv({m_j}, {r_j}))"
            self.accs.append(Acc(name, SCALAR, body, name))
            return SCALAR, name
        if f == "sph_L":
            if kA != SCALAR:
                raise LawError("sph_L of a vector")
            body = f"dv((T)2 * dv({m_j}, {r_j}) * ({A_i} - {A_j}) * dot3(rij, gWij), dij * dij)"
            self.accs.append(Acc(name, SCALAR, body, name))
            return SCALAR, name
        if f == "sph_A":
            if kA != VECTOR:
                raise LawError("sph_A of a scalar")
            body = f"(gWij * dv({m_j} * fmin(dot3({A_i} - {A_j}, rij), (T)0), {r_i} * dij * dij))"
            self.accs.append(Acc(name, VECTOR, body, name))
            return VECTOR, name
        raise LawError(f)


def parse_equation(text: str, index: int, fields: Dict[str, str], consts: Dict[str, object], dim: int,
                   variables: Optional[Dict[str, int]] = None) -> Eq:
    """One equation.  variables: the system's global scalars (name -> slot);
    an equation whose left-hand side is one of them is evaluated once, its
    fields read only inside the reductions fmax / fmin / fsum over all
    particles (Section 3.3: a variable's equation runs on one thread)."""
    variables = variables or {}
    if "=" not in text:
        raise LawError(f"equation {index}: no '='")
    lhs, rhs = (s.strip() for s in text.split("=", 1))
    if not lhs.isidentifier():
        raise LawError(f"equation {index}: bad left-hand side {lhs!r}")
    tree = _parse_rhs(rhs)
    if lhs == "r":
        ok = (isinstance(tree, ast.Call) and isinstance(tree.func, ast.Name) and tree.func.id == "euler"
              and len(tree.args) == 3 and isinstance(tree.args[0], ast.Name) and tree.args[0].id == "r")
        if not ok:
            raise LawError(f"equation {index}: positions move only as r = euler(r, V, c)")
        em = _Emitter(fields, consts, dim, variables=variables)
        kv, cv = em.emit(tree.args[1], "p")
        kc, cc = em.emit(tree.args[2], "p")
        if kv != VECTOR or kc != SCALAR:
            raise LawError(f"equation {index}: r = euler(r, vector, scalar)")
        return Eq(index, "r", "move", [], f"(({cv}) * ({cc}))", VECTOR, sorted(em.reads), tree, [])
    if lhs in variables:
        em = _Emitter(fields, consts, dim, variables=variables, var_mode=True)
        kind, code = em.emit(tree, "p")
        if kind != SCALAR:
            raise LawError(f"equation {index}: the variable {lhs} is a scalar")
        return Eq(index, lhs, "var", [], code, SCALAR, sorted(em.reads), tree, [], list(em.reds))
    if lhs not in fields:
        raise LawError(f"equation {index}: {lhs} is neither a field nor a variable")
    em = _Emitter(fields, consts, dim, variables=variables)
    kind, code = em.emit(tree, "p")
    if kind != fields[lhs]:
        raise LawError(f"equation {index}: {lhs} is a {'vector' if fields[lhs] == VECTOR else 'scalar'} "
                       f"but the right-hand side is not")
    return Eq(index, lhs, "pair" if em.accs else "local", em.accs, code, kind, sorted(em.reads), tree,
              sorted(em.pair_reads))


# ---------------------------------------------------------------------------
# CUDA source

_PRELUDE = r"""
#include <cuda_runtime.h>
#include <cmath>
#include <cstring>
#include "sph_images.cuh"
using namespace sph;
using T = %(T)s;
constexpr int D = %(D)d;
// whether any face of the domain is symmetric (a mirror): without one every
// image's sign factor is 1 and drops out of the generated code
constexpr bool kMirror = %(M)s;
__device__ __forceinline__ T msign(const ImageCell<T> &ic, int k) { return kMirror ? ic.s[k] : (T)1; }
// cells of edge in [h, 2h) in a domain of cut-off faces: the neighbours are
// searched through the 5^D cells as rows (no images)
constexpr bool kRows = %(R)s;
// resident blocks of 128 threads per SM the particle kernels are compiled for
// (the library's FP32 pair passes: 12 in 2D, 9 in 3D)
constexpr int kLawMinBlocks = sizeof(T) == 4 ? (D == 2 ? 12 : 9) : 1;
struct V3 { T x, y, z; };
// division: the FP32 form divides as the library's pair kernels do
__device__ __forceinline__ T dv(T a, T b) { return Ar<T>::div_ftz(a, b); }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator-(V3 a) { return V3{-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V3 operator*(V3 a, T s) { return V3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ V3 operator*(T s, V3 a) { return V3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ V3 &operator+=(V3 &a, V3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
__device__ __forceinline__ T dot3(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
"""


@dataclass
class Group:
    """Consecutive equations fused into one kernel."""
    index: int
    eqs: List[Eq]
    reads: List[str] = field(default_factory=list)     # fields read from memory
    writes: List[str] = field(default_factory=list)    # fields written
    moves: bool = False
    pair: bool = False
    layout: list = field(default_factory=list)         # pointer order of the launcher
    var: bool = False                                  # a variable's equation (own kernels)


def group_equations(eqs: Sequence[Eq]) -> List[Group]:
    """Fusion rule: an equation joins the current kernel unless its pair sums
    read a field an earlier equation of that kernel writes (the others would
    not see the new values), or the kernel already moved the particles (its
    neighbour sets are then stale)."""
    groups: List[Group] = []
    cur: List[Eq] = []
    written = set()
    moved = False
    for eq in eqs:
        if eq.kind == "var":
            # a variable's equation is a reduction: a kernel (pair) of its own
            if cur:
                groups.append(Group(len(groups), cur))
            groups.append(Group(len(groups), [eq], var=True))
            cur, written, moved = [], set(), False
            continue
        if eq.kind == "pair" and cur and (moved or set(eq.pair_reads) & written):
            groups.append(Group(len(groups), cur))
            cur, written, moved = [], set(), False
        cur.append(eq)
        if eq.kind == "move":
            moved = True
        else:
            written.add(eq.lhs)
    if cur:
        groups.append(Group(len(groups), cur))
    return groups


def _group_source(g: Group, fields: Dict[str, str], consts: Dict[str, object], dim: int,
                  variables: Dict[str, int]) -> str:
    if g.var:
        return _var_source(g, fields, consts, dim, variables)
    locals_map: Dict[str, str] = {}
    accs: List[Acc] = []
    stmts: List[str] = []
    reads = set()
    last: Dict[str, str] = {}
    moves: List[str] = []
    reads_r = False
    # the pair loop may be skipped for a particle when every equation of the
    # kernel that has pair sums is where(c, a, b) with its sums in a only and
    # c read from memory, and every c is zero (the masks are still recorded)
    guards: List[str] = []
    guardable = True
    for eq in g.eqs:
        em = _Emitter(fields, consts, dim, dict(locals_map), prefix=f"acc{eq.index}_", variables=variables)
        if eq.kind == "pair":
            t = eq.tree
            ok = (isinstance(t, ast.Call) and isinstance(t.func, ast.Name) and t.func.id == "where"
                  and len(t.args) == 3 and not _has_pair_sum(t.args[0]) and not _has_pair_sum(t.args[2]))
            if ok:
                gem = _Emitter(fields, consts, dim, {}, prefix="guard_", variables=variables)
                kc, cc = gem.emit(t.args[0], "p")
                ok = kc == SCALAR and not (gem.reads & set(locals_map)) and not gem.accs
                if ok:
                    guards.append(cc)
                    reads |= gem.reads
                    reads_r = reads_r or gem.reads_r
            guardable = guardable and ok
        if eq.kind == "move":
            kv, cv = em.emit(eq.tree.args[1], "p")
            kc, cc = em.emit(eq.tree.args[2], "p")
            stmts.append(f"    const V3 dr{eq.index} = ({cv}) * ({cc});")
            moves.append(f"dr{eq.index}")
        else:
            k, c = em.emit(eq.tree, "p")
            lname = f"L{eq.index}"
            stmts.append(f"    const {'T' if k == SCALAR else 'V3'} {lname} = {c};")
            locals_map[eq.lhs] = lname
            last[eq.lhs] = lname
        accs += em.accs
        reads |= em.reads
        reads_r = reads_r or em.reads_r
    g.reads = sorted(reads)
    g.writes = sorted(last)
    g.moves = bool(moves)
    g.pair = bool(accs)
    # kernel arguments: fields read, outputs, positions
    members, layout = [], []
    for f in g.reads:
        if fields[f] == SCALAR:
            members.append(f"    const T *f_{f};")
            layout.append((f, None))
        else:
            for q in range(dim):
                members.append(f"    const T *f_{f}_{q};")
                layout.append((f, q))
    for f in g.writes:
        if fields[f] == SCALAR:
            members.append(f"    T *out_{f};")
            layout.append(("=" + f, None))
        else:
            for q in range(dim):
                members.append(f"    T *out_{f}_{q};")
                layout.append(("=" + f, q))
    if moves or reads_r:
        for q in range(dim):
            members.append(f"    double *r_{q};")
            layout.append(("r", q))
    g.layout = layout
    k = g.index
    loop = ""
    guard_open = guard_close = ""
    if accs and guardable and guards:
        guard_open = "if (" + " || ".join(f"(({c}) != (T)0)" for c in guards) + ") {\n        "
        guard_close = "\n        }"
    if accs:
        decl = "\n".join(
            f"    {'T' if ac.kind == SCALAR else 'V3'} {ac.name} = "
            f"{'(T)0' if ac.kind == SCALAR else 'V3{(T)0, (T)0, (T)0}'};" for ac in accs)
        incs = "\n".join(f"            {ac.name} += {ac.body};" for ac in accs)
        loop = f"""{decl}
    {{
        // neighbour images: candidate tests recorded as hit masks by the
        // first pair kernel after a cell build, walked by every pair kernel
        const vec4_t<T> pi = pos[i];
        const uint32_t clin = cell_s[i];
        const CellXYZ cc = decode_cell(P, clin);
        uint32_t *mbase = mask + (size_t)blockIdx.x * Stencil<D>::NC * 128 + threadIdx.x;
        bool over;
        int total;
        if (record) {{
            total = kRows ? row_image_masks<D, T>(P, pi, clin, pos, start, mbase, over)
                          : image_masks<D, T>(P, pi, cc, clin, pos, start, mbase, over);
            nnb[i] = (uint16_t)total;
            ovf[i] = over ? 1 : 0;
        }} else {{
            total = nnb[i];
            over = ovf[i] != 0;
        }}
        const T hih = (T)P.half_inv_h;
        const T gcoef = -(T)5 * (T)P.alphaD / ((T)P.h * (T)P.h);
        auto body = [&](uint32_t j, T xp, T yp, T zp, T d2, const ImageCell<T> &ic) {{
            if (j == (uint32_t)i && ic.code == 0) return;  // i itself
            const V3 rij{{msign(ic, 0) * xp, msign(ic, 1) * yp, D == 3 ? msign(ic, 2) * zp : (T)0}};
            const T dij = Ar<T>::dist_ftz(d2);
            const T u = dij * hih;
            const T t = (T)1 - u;
            const T t2 = t * t;
            const T Wij = (T)P.alphaD * t2 * t2 * ((T)4 * u + (T)1);
            const V3 gWij = rij * (gcoef * t2 * t);
            (void)Wij;
            (void)gWij;
            const T mirr = kMirror && (ic.s[0] < (T)0 || ic.s[1] < (T)0 || ic.s[2] < (T)0) ? (T)1 : (T)0;
            (void)mirr;
{incs}
        }};
        {guard_open}if (kRows) {{
            if (!over)
                walk_row_images<D, T>(P, pi, clin, pos, start, [&](int idx) {{ return mbase[idx * 128]; }}, total,
                                      body);
            else
                scan_row_images<D, T>(P, pi, clin, pos, start, body);
        }} else if (!over) {{
            walk_images<D, T>(P, pi, cc, clin, pos, start, [&](int idx) {{ return mbase[idx * 128]; }}, total, body);
        }} else {{
            scan_images<D, T>(P, pi, cc, clin, pos, start, body);
        }}{guard_close}
    }}"""
    stores = []
    for f, lname in last.items():
        if fields[f] == SCALAR:
            stores.append(f"    a.out_{f}[i] = {lname};")
        else:
            for q, comp in zip(range(dim), "xyz"):
                stores.append(f"    a.out_{f}_{q}[i] = {lname}.{comp};")
    for dr in moves:
        stores.append(f"""    {{
        const T d[3] = {{{dr}.x, {dr}.y, {dr}.z}};
#pragma unroll
        for (int q = 0; q < D; ++q) {{
            double *rq = q == 0 ? a.r_0 : {'(q == 1 ? a.r_1 : a.r_2)' if dim == 3 else 'a.r_1'};
            double x = rq[i] + (double)d[q];
            if (P.bc[q] == SPH_BC_PERIODIC) {{
                if (x < P.dom_min[q]) x = x + P.per[q];
                else if (x >= P.hi[q]) x = x - P.per[q];
            }}
            rq[i] = x;
        }}
    }}""")
    struct = f"struct Args{k} {{\n" + ("\n".join(members) if members else "    void *unused;") + "\n};\n"
    return f"""
{struct}
// equations {', '.join(str(e.index) for e in g.eqs)}
__global__ void __launch_bounds__(128, kLawMinBlocks) law_k{k}(DevParams P, int n, const vec4_t<T> *__restrict__ pos,
                                                 const uint32_t *__restrict__ cell_s,
                                                 const uint32_t *__restrict__ start, uint32_t *mask,
                                                 uint16_t *nnb, uint8_t *ovf, int record,
                                                 const double *__restrict__ vars, Args{k} a)
{{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    (void)pos; (void)cell_s; (void)start; (void)mask; (void)nnb; (void)ovf; (void)record; (void)vars;
{loop}
{chr(10).join(stmts)}
{chr(10).join(stores)}
}}

extern "C" int law_launch_{k}(const void *blob, long long bytes, int n, const void *pos, const void *cell_s,
                              const void *start, void *mask, void *nnb, void *ovf, int record,
                              void *vars, void *part, void *const *ptrs, void *stream)
{{
    (void)part;
    if (bytes != (long long)sizeof(DevParams)) return -1;
    if (n <= 0) return 0;
    DevParams P;
    std::memcpy(&P, blob, sizeof(P));
    Args{k} a;
    std::memcpy(&a, ptrs, sizeof(a));
    law_k{k}<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(P, n, static_cast<const vec4_t<T> *>(pos),
        static_cast<const uint32_t *>(cell_s), static_cast<const uint32_t *>(start),
        static_cast<uint32_t *>(mask), static_cast<uint16_t *>(nnb), static_cast<uint8_t *>(ovf), record,
        static_cast<const double *>(vars), a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}}
"""


_RED_OPS = {"fmax": ("fmax(x, y)", "-HUGE_VAL"), "fmin": ("fmin(x, y)", "HUGE_VAL"), "fsum": ("x + y", "0.0")}


def _var_source(g: Group, fields: Dict[str, str], consts: Dict[str, object], dim: int,
                variables: Dict[str, int]) -> str:
    """A variable's equation: one kernel reduces each fmax / fmin / fsum
    operand over the particles into per-block partials (in double, a fixed
    tree per block), a one-block kernel combines the partials in a fixed order
    and evaluates the right-hand side on one thread (deterministic)."""
    eq = g.eqs[0]
    em = _Emitter(fields, consts, dim, variables=variables, var_mode=True)
    kind, rhs = em.emit(eq.tree, "p")
    reds = em.reds
    g.reads = sorted(em.reads)
    g.writes = []
    g.moves = False
    g.pair = False
    members, layout = [], []
    for f in g.reads:
        if fields[f] == SCALAR:
            members.append(f"    const T *f_{f};")
            layout.append((f, None))
        else:
            for q in range(dim):
                members.append(f"    const T *f_{f}_{q};")
                layout.append((f, q))
    if em.reads_r:
        for q in range(dim):
            members.append(f"    const double *r_{q};")
            layout.append(("r", q))
    g.layout = layout
    k = g.index
    slot = variables[eq.lhs]
    nr = len(reds)
    struct = f"struct Args{k} {{\n" + ("\n".join(members) if members else "    void *unused;") + "\n};\n"
    # per-block reduction of every operand (identity for the threads past n)
    red_body = []
    for r, (op, code) in enumerate(reds):
        comb, ident = _RED_OPS[op]
        red_body.append(f"""    {{
        double x = i < n ? (double)({code}) : {ident};
        sh[threadIdx.x] = x;
        __syncthreads();
        for (int o = 64; o > 0; o >>= 1) {{
            if (threadIdx.x < o) {{
                const double y = sh[threadIdx.x + o];
                x = sh[threadIdx.x];
                sh[threadIdx.x] = {comb};
            }}
            __syncthreads();
        }}
        if (threadIdx.x == 0) part[{r} * gridDim.x + blockIdx.x] = sh[0];
        __syncthreads();
    }}""")
    fin = []
    for r, (op, code) in enumerate(reds):
        comb, ident = _RED_OPS[op]
        fin.append(f"""    {{
        double x = {ident};
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {{
            const double y = part[{r} * nb + b];
            x = {comb};
        }}
        sh[threadIdx.x] = x;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {{
            if (threadIdx.x < o) {{
                const double y = sh[threadIdx.x + o];
                x = sh[threadIdx.x];
                sh[threadIdx.x] = {comb};
            }}
            __syncthreads();
        }}
        if (threadIdx.x == 0) red[{r}] = sh[0];
        __syncthreads();
    }}""")
    decl = "\n".join(f"    const T red{r} = (T)red[{r}];" for r in range(nr))
    return f"""
{struct}
// equation {eq.index}: the variable {eq.lhs}
__global__ void __launch_bounds__(128) law_k{k}(DevParams P, int n, const double *__restrict__ vars,
                                                 double *__restrict__ part, Args{k} a)
{{
    __shared__ double sh[128];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    (void)P; (void)vars; (void)a;
{chr(10).join(red_body)}
}}

__global__ void __launch_bounds__(256) law_f{k}(DevParams P, int nb, const double *__restrict__ part, double *vars)
{{
    __shared__ double sh[256];
    __shared__ double red[{max(nr, 1)}];
    (void)P; (void)part; (void)nb; (void)sh;
{chr(10).join(fin)}
    if (threadIdx.x == 0) {{
{decl}
        vars[{slot}] = (double)({rhs});
    }}
}}

extern "C" int law_launch_{k}(const void *blob, long long bytes, int n, const void *pos, const void *cell_s,
                              const void *start, void *mask, void *nnb, void *ovf, int record,
                              void *vars, void *part, void *const *ptrs, void *stream)
{{
    (void)pos; (void)cell_s; (void)start; (void)mask; (void)nnb; (void)ovf; (void)record;
    if (bytes != (long long)sizeof(DevParams)) return -1;
    DevParams P;
    std::memcpy(&P, blob, sizeof(P));
    Args{k} a;
    std::memcpy(&a, ptrs, sizeof(a));
    const int nb = n > 0 ? (n + 127) / 128 : 0;
    if ({nr} > 0 && nb > 0)
        law_k{k}<<<nb, 128, 0, (cudaStream_t)stream>>>(P, n, static_cast<const double *>(vars),
                                                        static_cast<double *>(part), a);
    law_f{k}<<<1, 256, 0, (cudaStream_t)stream>>>(P, nb, static_cast<const double *>(part),
                                                   static_cast<double *>(vars));
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}}
"""


def generate(equations: Sequence[Eq], fields: Dict[str, str], consts: Dict[str, object], dim: int,
             f32: bool, variables: Optional[Dict[str, int]] = None, mirror: bool = True,
             rows: bool = False) -> Tuple[str, List[Group]]:
    """CUDA source and kernel groups of the equations.  mirror: whether any
    face of the domain is symmetric (False compiles the image sign factors
    out); rows: the cells have edge in [h, 2h) and every face is cut-off
    (the neighbours are searched through the 5^D cells as rows)."""
    groups = group_equations(equations)
    src = _PRELUDE % {"T": "float" if f32 else "double", "D": dim, "M": "true" if mirror else "false",
                      "R": "true" if rows else "false"}
    for g in groups:
        src += _group_source(g, fields, consts, dim, variables or {})
    return src, groups


def live_at_rebuild(groups: Sequence[Group], g0: int) -> List[str]:
    """Fields whose values are read (from memory) before being written when
    the kernels run from group g0 on, round the cycle of one step."""
    live, written = set(), set()
    order = list(range(g0, len(groups))) + list(range(0, g0))
    for k in order:
        live |= set(groups[k].reads) - written
        written |= set(groups[k].writes)
    return sorted(live)


def _cache_dir() -> str:
    """Where compiled laws are kept: SPH_LAW_CACHE, else _law_cache/ beside
    the library (in-tree, like the library itself)."""
    d = os.environ.get("SPH_LAW_CACHE") or os.path.join(HERE, "_law_cache")
    os.makedirs(d, exist_ok=True)
    return d


def compile_source(src: str) -> str:
    """nvcc -> shared library (cached by the source, the flags and the
    library headers); returns its path."""
    hdrs = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cuh")]
    hdrs.append(os.path.join(HERE, "..", "include", "sph.h"))
    hsh = hashlib.sha256(src.encode())
    for h in hdrs:
        with open(h, "rb") as f:
            hsh.update(f.read())
    flags = list(_build.ARCH) + list(_build.NVCC_FLAGS)
    hsh.update(" ".join(flags).encode())
    hsh.update(platform.machine().encode())      # a host-code library per host architecture
    key = hsh.hexdigest()[:20]
    d = _cache_dir()
    so = os.path.join(d, f"law_{key}.so")
    if os.path.exists(so):
        return so
    cu = os.path.join(d, f"law_{key}.cu")
    with open(cu, "w") as f:
        f.write(src)
    tmp = so + f".tmp{os.getpid()}"
    cmd = [_build.nvcc(), *flags, "-I", CSRC, "-shared", "-cudart=static", "-o", tmp, cu]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise LawError("nvcc failed on the generated laws:\n" + r.stderr[-4000:])
    os.replace(tmp, so)
    return so


# ---------------------------------------------------------------------------
# runtime

class LawSystem:
    """A particle system (a SPH_MODEL_FIELDS context over case's particles
    and cell grid) with fields, constants and compiled equations.

    fields: name -> (kind, initial values in the case's particle order),
    kind "scalar" or "vector" (values of shape (n,) or (n, dim)).
    Consecutive equations are fused into one kernel (group_equations); at a
    cell rebuild only the fields read before they are written again are
    reordered with the particles (live_at_rebuild), out of place into the
    second buffer of each field.

    variables: name -> initial value of global scalars (kept on the device
    in FP64): any equation may read them; an equation whose left-hand side
    is a variable is evaluated once per step, reading fields only through
    the reductions fmax / fmin / fsum over all particles (e.g. an adaptive
    time step, an elapsed time).
    """

    def __init__(self, case, fields: Dict[str, Tuple[str, np.ndarray]], constants: Dict[str, object],
                 equations: Sequence[str], precision=S.SPH_PREC_F32,
                 variables: Optional[Dict[str, float]] = None):
        import torch
        self.case = case
        self.dim = case.dim
        self.precision = precision
        self.f32 = precision == S.SPH_PREC_F32
        self.kinds = {k: (SCALAR if v[0] == "scalar" else VECTOR) for k, v in fields.items()}
        variables = dict(variables or {})
        names = list(self.kinds) + list(constants) + list(variables)
        if len(set(names)) != len(names):
            raise LawError("a name is used twice among fields, constants and variables")
        for name in names:
            if name in ("r", "h", PAPER_KERNEL) or name in OPERATORS or name in PAPER_OPERATORS or \
                    name in PAIR_NAMES or name in REDUCTIONS:
                raise LawError(f"{name} is reserved")
        self.consts = dict(constants)
        self.var_slot = {name: k for k, name in enumerate(variables)}
        self.eqs = [parse_equation(t, k, self.kinds, self.consts, self.dim, self.var_slot)
                    for k, t in enumerate(equations)]
        bc = tuple(getattr(case, "bc", (S.SPH_BC_CUTOFF,) * 3))[:self.dim]
        # cells smaller than the support radius (edge in [h, 2h)): the row
        # stencil, which has no images, so only in a domain of cut-off faces
        rows = case.cs < 2.0 * case.h
        if rows and any(b != S.SPH_BC_CUTOFF for b in bc):
            raise LawError("cells of edge below 2h need cut-off faces (the row stencil has no images)")
        src, self.groups = generate(self.eqs, self.kinds, self.consts, self.dim, self.f32, self.var_slot,
                                    mirror=S.SPH_BC_SYMMETRIC in bc, rows=rows)
        self.source = src
        self.lib = C.CDLL(compile_source(src))
        self.launch = []
        for g in self.groups:
            fn = getattr(self.lib, f"law_launch_{g.index}")
            fn.argtypes = [C.c_void_p, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            fn.restype = C.c_int
            self.launch.append(fn)
        self.live = [live_at_rebuild(self.groups, k) for k in range(len(self.groups))]
        p = S.params_from_case(case, precision=precision)
        p.model = S.SPH_MODEL_FIELDS
        self.params = p
        self.ctx = S.sph_create(p, case.n)
        n, D = case.n, self.dim
        self.n = n
        self.state = S.device_state(case.r, np.zeros((n, D)), case.kind, case.id, precision)
        self._view = self.state.view()
        # the state a build writes (the two alternate: a build reads one and
        # writes the other, the fields' canonical copies in the same pass)
        self.spare_state = S.device_state(case.r, np.zeros((n, D)), case.kind, case.id, precision)
        self._spare_view = self.spare_state.view()
        for k in range(3):
            self._view.v[k] = None       # positions only: the fields are the system's own
            self._spare_view.v[k] = None
        tdt = torch.float32 if self.f32 else torch.float64
        self.tdt = tdt
        self.data: Dict[str, List] = {}
        self.spare: Dict[str, List] = {}
        for name, (kind, vals) in fields.items():
            a = np.asarray(vals, np.float64)
            comps = [a] if self.kinds[name] == SCALAR else [a[:, k] for k in range(D)]
            self.data[name] = [torch.tensor(np.ascontiguousarray(c), dtype=tdt, device="cuda") for c in comps]
            self.spare[name] = [torch.empty_like(t) for t in self.data[name]]
        self.stale = set()
        self.builds = 0
        # the variables (FP64) and the per-block partials of the reductions
        self.vars = torch.tensor([float(v) for v in variables.values()] or [0.0], dtype=torch.float64,
                                 device="cuda")
        nred = max([len(e.reds) for e in self.eqs if e.kind == "var"] or [0])
        self.part = torch.empty(max(1, nred * ((n + 127) // 128)), dtype=torch.float64, device="cuda")
        # a first build: canonical order for the state and every field, and
        # the kernel constants (fixed for the context) for kernels without
        # pair sums
        self._rebuild(torch.cuda.current_stream(), list(self.data))
        v = S.sph_law_view(self.ctx)
        self._blob_bytes = v.params_bytes
        self._blob = C.create_string_buffer(C.string_at(v.params, v.params_bytes), v.params_bytes)
        self.dirty = False

    def close(self):
        if getattr(self, "ctx", None):
            S.sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _rebuild(self, stream, live):
        """Cell build into the spare state, with the live fields reordered
        in the same gather; the state and field buffers then swap roles."""
        eb = 4 if self.f32 else 8
        ins, outs = [], []
        for name in self.data:
            if name in live:
                for t, o in zip(self.data[name], self.spare[name]):
                    ins.append(t.data_ptr())
                    outs.append(o.data_ptr())
                self.data[name], self.spare[name] = self.spare[name], self.data[name]
                self.stale.discard(name)
            else:
                self.stale.add(name)   # not read again before it is written: no reorder
        S.sph_build_cells_into(self.ctx, self._view, self._spare_view, ins, outs, eb, stream)
        self.state, self.spare_state = self.spare_state, self.state
        self._view, self._spare_view = self._spare_view, self._view
        self.masks = False        # the next pair kernel records the hit masks
        self.dirty = False
        self.builds += 1

    def _ptrs(self, g: Group):
        ptrs = []
        for name, comp in g.layout:
            c = 0 if comp is None else comp
            if name == "r":
                ptrs.append(self.state.r[c].data_ptr())
            elif name.startswith("="):
                ptrs.append(self.spare[name[1:]][c].data_ptr())
            else:
                ptrs.append(self.data[name][c].data_ptr())
        return (C.c_void_p * max(1, len(ptrs)))(*ptrs)

    def step(self, nsteps: int = 1, stream=None, timing: Optional[dict] = None):
        """nsteps passes over the equations.  timing (a dict, optional)
        receives CUDA-event times in ms summed over the steps: "build" (cell
        build and field reorders) and "k<g>" per fused kernel g."""
        import torch
        st = stream or torch.cuda.current_stream()
        sv = C.c_void_p(st.cuda_stream)
        marks = []

        def mark(tag):
            if timing is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(st)
                marks.append((tag, e))
        for _ in range(int(nsteps)):
            for g, fn in zip(self.groups, self.launch):
                if g.pair and self.dirty:
                    mark("build")
                    self._rebuild(st, self.live[g.index])
                mark(f"k{g.index}")
                if g.pair:
                    v = S.sph_law_view(self.ctx)
                    record = 0 if self.masks else 1
                    rc = fn(C.c_void_p(v.params), v.params_bytes, v.n, C.c_void_p(v.pos), C.c_void_p(v.cell_s),
                            C.c_void_p(v.cell_start), C.c_void_p(v.mask), C.c_void_p(v.nnb), C.c_void_p(v.ovf),
                            record, C.c_void_p(self.vars.data_ptr()), C.c_void_p(self.part.data_ptr()),
                            self._ptrs(g), sv)
                    self.masks = True
                else:
                    rc = fn(C.c_void_p(C.addressof(self._blob)), self._blob_bytes, self.n, None, None, None, None,
                            None, None, 0, C.c_void_p(self.vars.data_ptr()), C.c_void_p(self.part.data_ptr()),
                            self._ptrs(g), sv)
                if rc != 0:
                    raise LawError(f"launch of kernel {g.index} failed ({rc})")
                for f in g.writes:
                    self.data[f], self.spare[f] = self.spare[f], self.data[f]
                    self.stale.discard(f)
                if g.moves:
                    self.dirty = True
        mark("end")
        if timing is not None and len(marks) > 1:
            marks[-1][1].synchronize()
            for (tag, a), (_, b) in zip(marks[:-1], marks[1:]):
                timing[tag] = timing.get(tag, 0.0) + a.elapsed_time(b)

    def variables(self) -> Dict[str, float]:
        """The current values of the variables."""
        vals = self.vars.cpu().numpy()
        return {name: float(vals[k]) for name, k in self.var_slot.items()}

    def host(self):
        """(r, {field: values}, ids) in the current particle order.  A field
        that a rebuild did not reorder because the equations overwrite it
        before reading it holds NaN until it is written."""
        r = np.stack([t.cpu().numpy() for t in self.state.r], axis=1)
        ids = self.state.id.cpu().numpy().astype(np.uint32)
        out = {}
        for name, comps in self.data.items():
            a = [t.cpu().double().numpy() for t in comps]
            v = a[0] if self.kinds[name] == SCALAR else np.stack(a, axis=1)
            if name in self.stale:
                v = np.full_like(v, np.nan)
            out[name] = v
        return r, out, ids

"""ctypes binding of the CPU FP64 SPH oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg import
this module.  The library is plain C compiled by `oracle.build.build()`;
nothing here computes SPH arithmetic, it only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))


class OrcParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("ncell", C.c_int * 3),
        ("dom_min", C.c_double * 3),
        ("cs", C.c_double),
        ("h", C.c_double),
        ("dx", C.c_double),
        ("mass", C.c_double),
        ("rho0", C.c_double),
        ("c0", C.c_double),
        ("gamma", C.c_double),
        ("alpha", C.c_double),
        ("visc_eps", C.c_double),
        ("dt", C.c_double),
        ("g", C.c_double * 3),
        ("rho_ref_lattice", C.c_int),
        ("clamp_neg_p", C.c_int),
        ("reaction_mode", C.c_int),
        ("fp32_neighbours", C.c_int),
        ("adaptive_dt", C.c_int),
        ("cfl", C.c_double),
    ]


class OrcBcParams(C.Structure):
    """orc_bc_params of sph_oracle_bc.c."""
    _fields_ = [
        ("dim", C.c_int),
        ("ncell", C.c_int * 3),
        ("dom_min", C.c_double * 3),
        ("cs", C.c_double),
        ("h", C.c_double),
        ("mass", C.c_double),
        ("rho0", C.c_double),
        ("c", C.c_double),
        ("visc", C.c_double),
        ("dt", C.c_double),
        ("g", C.c_double * 3),
        ("bc", C.c_int * 3),
        ("fp32", C.c_int),
    ]


class OrcBcDiag(C.Structure):
    _fields_ = [
        ("n_pairs", C.c_int64),
        ("vmax", C.c_double),
        ("amax", C.c_double),
        ("dt_cfl", C.c_double),
        ("out_of_domain", C.c_int),
    ]


class OrcDemParams(C.Structure):
    """orc_dem_params of sph_oracle_dem.c."""
    _fields_ = [
        ("dim", C.c_int),
        ("ncell", C.c_int * 3),
        ("dom_min", C.c_double * 3),
        ("cs", C.c_double),
        ("h", C.c_double),
        ("E", C.c_double),
        ("nu", C.c_double),
        ("cf", C.c_double),
        ("dt", C.c_double),
        ("g", C.c_double * 3),
        ("bc", C.c_int * 3),
        ("fp32", C.c_int),
        ("tank_M", C.c_double),
        ("tank_S", C.c_double),
    ]


class OrcDemDiag(C.Structure):
    _fields_ = [
        ("n_contacts", C.c_int64),
        ("vmax", C.c_double),
        ("amax", C.c_double),
        ("Fb", C.c_double * 3),
        ("Zddot", C.c_double),
        ("out_of_domain", C.c_int),
    ]


class OrcDiag(C.Structure):
    _fields_ = [
        ("n_pairs", C.c_int64),
        ("vmax", C.c_double),
        ("amax", C.c_double),
        ("dt_cfl", C.c_double),
        ("out_of_domain", C.c_int),
        ("dt", C.c_double),
        ("time", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        fp = C.POINTER(C.c_float)
        u32 = C.POINTER(C.c_uint32)
        i32 = C.POINTER(C.c_int32)
        i64 = C.POINTER(C.c_int64)
        u8 = C.POINTER(C.c_uint8)
        P = C.POINTER(OrcParams)
        L.orc_alpha_D.argtypes = [C.c_int, C.c_double]
        L.orc_alpha_D.restype = C.c_double
        L.orc_W.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_W.restype = C.c_double
        L.orc_dWdr.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_dWdr.restype = C.c_double
        L.orc_rho_ref.argtypes = [P]
        L.orc_rho_ref.restype = C.c_double
        L.orc_pressure.argtypes = [P, C.c_double, C.c_double]
        L.orc_pressure.restype = C.c_double
        L.orc_sort_cells.argtypes = [P, C.c_int, dp, u32, u32, u32, u32]
        L.orc_sort_cells.restype = C.c_int
        L.orc_cell_coords.argtypes = [P, C.c_int, dp, i32, fp]
        L.orc_cell_coords.restype = C.c_int
        L.orc_neighbours.argtypes = [P, C.c_int, dp, u32, C.c_int, C.c_int, i64, u32, C.c_int64]
        L.orc_neighbours.restype = C.c_int64
        L.orc_density.argtypes = [P, C.c_int, dp, u32, dp, dp]
        L.orc_density.restype = C.c_int64
        L.orc_accel.argtypes = [P, C.c_int, dp, dp, u8, u32, dp, dp, dp, dp, dp]
        L.orc_accel.restype = C.c_int
        L.orc_step.argtypes = [P, C.c_int, dp, dp, u8, u32, C.c_int, dp, dp, dp, C.POINTER(OrcDiag)]
        L.orc_step.restype = C.c_int
        L.orc_step_adjoint.argtypes = [P, C.c_int, dp, dp, u8, u32, dp, dp, dp, dp, dp]
        L.orc_step_adjoint.restype = C.c_int
        L.orc_step_adjoint_clamped.argtypes = [P, C.c_int, dp, dp, u8, u32, u8, dp, dp, dp, dp, dp]
        L.orc_step_adjoint_clamped.restype = C.c_int
        L.orc_step_cs.argtypes = [P, C.c_int, dp, dp, u8, u32, dp, dp, C.c_double, C.c_double, dp, dp, dp, dp]
        L.orc_step_cs.restype = C.c_int
        L.orc_sampled_forces.argtypes = [P, C.c_int, dp, dp, u8, u32, C.c_int, u32, dp, dp, dp, dp, dp]
        L.orc_sampled_forces.restype = C.c_int
        BP = C.POINTER(OrcBcParams)
        L.orc_bc_neighbours.argtypes = [BP, C.c_int, dp, u32, C.c_int, i64, u32, u8, C.c_int64]
        L.orc_bc_neighbours.restype = C.c_int64
        L.orc_bc_eval.argtypes = [BP, C.c_int, dp, dp, dp, u8, u32, dp, dp, dp, dp, dp, dp]
        L.orc_bc_eval.restype = C.c_int64
        L.orc_bc_step.argtypes = [BP, C.c_int, dp, dp, dp, u8, u32, C.c_int, dp, dp, C.POINTER(OrcBcDiag)]
        L.orc_bc_step.restype = C.c_int
        L.orc_bc_sample.argtypes = [BP, C.c_int, dp, u32, dp, dp, dp, dp, dp]
        L.orc_bc_sample.restype = C.c_int64
        DP = C.POINTER(OrcDemParams)
        L.orc_dem_forces.argtypes = [DP, C.c_int, dp, dp, dp, dp, u32, C.c_double, dp, dp, dp]
        L.orc_dem_forces.restype = C.c_int64
        L.orc_dem_step.argtypes = [DP, C.c_int, dp, dp, dp, dp, u8, u32, C.c_int, dp, dp, C.POINTER(OrcDemDiag)]
        L.orc_dem_step.restype = C.c_int
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        L.orc_set_num_threads.restype = None
        _lib = L
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def params(case, *, rho_ref_lattice=True, clamp_neg_p=True, reaction_mode=False,
           fp32_neighbours=False, g=None, adaptive_dt=False, cfl=1.0) -> OrcParams:
    p = OrcParams()
    p.dim = case.dim
    for k in range(3):
        p.ncell[k] = int(case.ncell[k])
        p.dom_min[k] = float(case.dom_min[k])
    p.cs = case.cs
    p.h = case.h
    p.dx = case.dx
    p.mass = case.mass
    p.rho0 = case.rho0
    p.c0 = case.c0
    p.gamma = case.gamma
    p.alpha = case.alpha
    p.visc_eps = case.visc_eps
    p.dt = case.dt
    gg = case.g if g is None else g
    for k in range(3):
        p.g[k] = float(gg[k])
    p.rho_ref_lattice = int(rho_ref_lattice)
    p.clamp_neg_p = int(clamp_neg_p)
    p.reaction_mode = int(reaction_mode)
    p.fp32_neighbours = int(fp32_neighbours)
    p.adaptive_dt = int(adaptive_dt)
    p.cfl = float(cfl)
    return p


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def W(dim, h, r):
    return lib().orc_W(dim, h, r)


def dWdr(dim, h, r):
    return lib().orc_dWdr(dim, h, r)


def alpha_D(dim, h):
    return lib().orc_alpha_D(dim, h)


def rho_ref(p: OrcParams) -> float:
    return lib().orc_rho_ref(C.byref(p))


def pressure(p: OrcParams, rho_ref_value: float, rho: float) -> float:
    return lib().orc_pressure(C.byref(p), rho_ref_value, rho)


def sort_cells(p: OrcParams, r, ids):
    r = _c64(r)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    n = r.shape[0]
    ncells = p.ncell[0] * p.ncell[1] * (p.ncell[2] if p.dim == 3 else 1)
    order = np.zeros(n, np.uint32)
    start = np.zeros(ncells + 1, np.uint32)
    cell_of = np.zeros(n, np.uint32)
    bad = lib().orc_sort_cells(C.byref(p), n, _ptr(r, C.c_double), _ptr(ids, C.c_uint32),
                               _ptr(order, C.c_uint32), _ptr(start, C.c_uint32),
                               _ptr(cell_of, C.c_uint32))
    return order, start, cell_of, bad


def cell_coords(p: OrcParams, r):
    r = _c64(r)
    n = r.shape[0]
    cc = np.zeros((n, 3), np.int32)
    off = np.zeros((n, 3), np.float32)
    bad = lib().orc_cell_coords(C.byref(p), n, _ptr(r, C.c_double), _ptr(cc, C.c_int32),
                                _ptr(off, C.c_float))
    return cc, off, bad


def neighbours(p: OrcParams, r, ids, *, method="cells", fp32=False):
    """CSR neighbour lists (persistent ids ascending) per input particle."""
    r = _c64(r)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    n = r.shape[0]
    m = 0 if method == "brute" else 1
    offs = np.zeros(n + 1, np.int64)
    tot = lib().orc_neighbours(C.byref(p), n, _ptr(r, C.c_double), _ptr(ids, C.c_uint32), m,
                               int(fp32), _ptr(offs, C.c_int64), None, 0)
    if tot < 0:
        raise RuntimeError(f"orc_neighbours failed ({tot})")
    nbr = np.zeros(max(tot, 1), np.uint32)
    tot2 = lib().orc_neighbours(C.byref(p), n, _ptr(r, C.c_double), _ptr(ids, C.c_uint32), m,
                                int(fp32), _ptr(offs, C.c_int64), _ptr(nbr, C.c_uint32), tot)
    assert tot2 == tot
    return offs, nbr[:tot]


def density(p: OrcParams, r, ids):
    r = _c64(r)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    n = r.shape[0]
    rho = np.zeros(n)
    pr = np.zeros(n)
    pairs = lib().orc_density(C.byref(p), n, _ptr(r, C.c_double), _ptr(ids, C.c_uint32),
                              _ptr(rho, C.c_double), _ptr(pr, C.c_double))
    if pairs < 0:
        raise RuntimeError("particle outside the cell grid")
    return rho, pr, int(pairs)


def accel(p: OrcParams, r, v, kind, ids, rho, pr, with_abs=False):
    """Accelerations; with_abs also returns (sum_j |pair term| + |g|, density
    sensitivity) per particle (see orc_accel)."""
    r = _c64(r)
    v = _c64(v)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    rho = _c64(rho)
    pr = _c64(pr)
    a = np.zeros_like(r)
    aabs = np.zeros(r.shape[0]) if with_abs else None
    asens = np.zeros(r.shape[0]) if with_abs else None
    rc = lib().orc_accel(C.byref(p), r.shape[0], _ptr(r, C.c_double), _ptr(v, C.c_double),
                         _ptr(kind, C.c_uint8), _ptr(ids, C.c_uint32), _ptr(rho, C.c_double),
                         _ptr(pr, C.c_double), _ptr(a, C.c_double), _ptr(aabs, C.c_double),
                         _ptr(asens, C.c_double))
    if rc:
        raise RuntimeError("particle outside the cell grid")
    return (a, aabs, asens) if with_abs else a


@dataclass
class StepResult:
    r: np.ndarray
    v: np.ndarray
    rho: np.ndarray
    p: np.ndarray
    a: np.ndarray
    n_pairs: int
    vmax: float
    amax: float
    dt_cfl: float
    rc: int
    dt: float = 0.0     # the step size of the last step
    time: float = 0.0   # the sum of the step sizes


def step(p: OrcParams, r, v, kind, ids, nsteps=1) -> StepResult:
    """nsteps oracle steps from (r, v); inputs are not modified."""
    r = _c64(r).copy()
    v = _c64(v).copy()
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    n = r.shape[0]
    rho = np.zeros(n)
    pr = np.zeros(n)
    a = np.zeros_like(r)
    d = OrcDiag()
    rc = lib().orc_step(C.byref(p), n, _ptr(r, C.c_double), _ptr(v, C.c_double),
                        _ptr(kind, C.c_uint8), _ptr(ids, C.c_uint32), int(nsteps),
                        _ptr(rho, C.c_double), _ptr(pr, C.c_double), _ptr(a, C.c_double),
                        C.byref(d))
    return StepResult(r, v, rho, pr, a, int(d.n_pairs), d.vmax, d.amax, d.dt_cfl, rc, d.dt, d.time)


def step_adjoint(p: OrcParams, r, v, kind, ids, rbar1, vbar1, clamped=None):
    """One reverse step: (rbar0, vbar0, alpha_bar) from the adjoint at n+1.
    clamped (n bools, optional): the pressure clamp's decision per particle
    in the forward step (orc_step_adjoint_clamped), else the step's own."""
    r = _c64(r)
    v = _c64(v)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    rbar1 = _c64(rbar1)
    vbar1 = _c64(vbar1)
    rbar0 = np.zeros_like(r)
    vbar0 = np.zeros_like(v)
    ab = np.zeros(1)
    if clamped is None:
        rc = lib().orc_step_adjoint(C.byref(p), r.shape[0], _ptr(r, C.c_double), _ptr(v, C.c_double),
                                    _ptr(kind, C.c_uint8), _ptr(ids, C.c_uint32), _ptr(rbar1, C.c_double),
                                    _ptr(vbar1, C.c_double), _ptr(rbar0, C.c_double), _ptr(vbar0, C.c_double),
                                    _ptr(ab, C.c_double))
    else:
        cl = np.ascontiguousarray(np.asarray(clamped).astype(np.uint8))
        rc = lib().orc_step_adjoint_clamped(C.byref(p), r.shape[0], _ptr(r, C.c_double), _ptr(v, C.c_double),
                                            _ptr(kind, C.c_uint8), _ptr(ids, C.c_uint32), _ptr(cl, C.c_uint8),
                                            _ptr(rbar1, C.c_double), _ptr(vbar1, C.c_double),
                                            _ptr(rbar0, C.c_double), _ptr(vbar0, C.c_double), _ptr(ab, C.c_double))
    if rc:
        raise RuntimeError("particle outside the cell grid")
    return rbar0, vbar0, float(ab[0])


def step_complex(p: OrcParams, r, v, kind, ids, dr, dv, dalpha, hcs=1e-30):
    """One step on complex inputs: (r', v', J_r (dr, dv, dalpha), J_v (...))."""
    r = _c64(r)
    v = _c64(v)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    dr = _c64(dr)
    dv = _c64(dv)
    ro, vo, dro, dvo = (np.zeros_like(r) for _ in range(4))
    rc = lib().orc_step_cs(C.byref(p), r.shape[0], _ptr(r, C.c_double), _ptr(v, C.c_double),
                           _ptr(kind, C.c_uint8), _ptr(ids, C.c_uint32), _ptr(dr, C.c_double),
                           _ptr(dv, C.c_double), float(dalpha), float(hcs), _ptr(ro, C.c_double),
                           _ptr(vo, C.c_double), _ptr(dro, C.c_double), _ptr(dvo, C.c_double))
    if rc:
        raise RuntimeError("particle outside the cell grid")
    return ro, vo, dro, dvo


def rollout_loss_grad(p: OrcParams, case, v0, target, nsteps):
    """FP64 loss L = mean over fluid of |r^T - target|^2 after nsteps from
    (case.r, v0), with dL/dv0 (n x dim) and dL/dalpha by the reverse sweep
    of orc_step_adjoint over the stored states."""
    r = _c64(case.r).copy()
    v = _c64(v0).copy()
    states = []
    for _ in range(nsteps):
        states.append((r, v))
        res = step(p, r, v, case.kind, case.id, 1)
        if res.rc:
            raise RuntimeError("particle left the grid")
        r, v = res.r, res.v
    nf = case.n_fluid
    fl = case.kind == 0
    diff = r[fl] - target
    L = float(np.mean(np.sum(diff * diff, axis=1)))
    rbar = np.zeros_like(r)
    rbar[fl] = 2.0 * diff / nf
    vbar = np.zeros_like(v)
    abar = 0.0
    for (rs, vs) in reversed(states):
        rbar, vbar, ab = step_adjoint(p, rs, vs, case.kind, case.id, rbar, vbar)
        abar += ab
    return L, vbar, abar, r


def rollout_loss(p: OrcParams, case, v0, target, nsteps):
    res = step(p, case.r, v0, case.kind, case.id, nsteps)
    if res.rc:
        raise RuntimeError("particle left the grid")
    fl = case.kind == 0
    diff = res.r[fl] - target
    return float(np.mean(np.sum(diff * diff, axis=1)))


def sampled_forces(p: OrcParams, r, v, kind, ids, idx):
    """(rho, p, a, A, G) at the sampled input indices idx (see orc_sampled_forces)."""
    r = _c64(r)
    v = _c64(v)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    m = idx.size
    rho, pr, A, G = (np.zeros(m) for _ in range(4))
    a = np.zeros((m, r.shape[1]))
    rc = lib().orc_sampled_forces(C.byref(p), r.shape[0], _ptr(r, C.c_double), _ptr(v, C.c_double),
                                  _ptr(kind, C.c_uint8), _ptr(ids, C.c_uint32), m, _ptr(idx, C.c_uint32),
                                  _ptr(rho, C.c_double), _ptr(pr, C.c_double), _ptr(a, C.c_double),
                                  _ptr(A, C.c_double), _ptr(G, C.c_double))
    if rc:
        raise RuntimeError("particle outside the cell grid")
    return rho, pr, a, A, G


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))


# ---------------------------------------------------------------------------
# Boundary treatments, Example 1a in the paper's form, sampling operator
# (sph_oracle_bc.c).

BC_CUTOFF, BC_SYMMETRIC, BC_PERIODIC = 0, 1, 2


def bc_params(case, *, fp32=False, g=None, bc=None, dt=None, visc=None) -> OrcBcParams:
    """orc_bc_params from a case: c = case.c0, visc = case.alpha, the
    boundary treatment of each axis from case.bc (overridable)."""
    p = OrcBcParams()
    p.dim = case.dim
    for k in range(3):
        p.ncell[k] = int(case.ncell[k])
        p.dom_min[k] = float(case.dom_min[k])
    p.cs = case.cs
    p.h = case.h
    p.mass = case.mass
    p.rho0 = case.rho0
    p.c = case.c0
    p.visc = case.alpha if visc is None else float(visc)
    p.dt = case.dt if dt is None else float(dt)
    gg = case.g if g is None else g
    bb = getattr(case, "bc", (0, 0, 0)) if bc is None else bc
    for k in range(3):
        p.g[k] = float(gg[k])
        p.bc[k] = int(bb[k])
    p.fp32 = int(fp32)
    return p


def bc_neighbours(p: OrcBcParams, r, ids, *, method="cells"):
    """CSR lists of neighbour images per input particle: (ids, image codes),
    sorted by id then code."""
    r = _c64(r)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    n = r.shape[0]
    m = 0 if method == "brute" else 1
    offs = np.zeros(n + 1, np.int64)
    tot = lib().orc_bc_neighbours(C.byref(p), n, _ptr(r, C.c_double), _ptr(ids, C.c_uint32), m,
                                  _ptr(offs, C.c_int64), None, None, 0)
    if tot < 0:
        raise RuntimeError(f"orc_bc_neighbours failed ({tot})")
    nbr = np.zeros(max(tot, 1), np.uint32)
    img = np.zeros(max(tot, 1), np.uint8)
    tot2 = lib().orc_bc_neighbours(C.byref(p), n, _ptr(r, C.c_double), _ptr(ids, C.c_uint32), m,
                                   _ptr(offs, C.c_int64), _ptr(nbr, C.c_uint32), _ptr(img, C.c_uint8), tot)
    assert tot2 == tot
    return offs, nbr[:tot], img[:tot]


@dataclass
class BcEval:
    rho: np.ndarray       # density after the continuity update (eq2)
    p: np.ndarray         # linear EOS pressure (eq3)
    a: np.ndarray         # acceleration (eq4, eq5)
    drho_abs: np.ndarray  # dt rho_i sum |continuity term|
    aabs: np.ndarray      # sum |momentum term| + |g|
    asens: np.ndarray     # change of |a| per unit relative density error
    n_pairs: int


def bc_eval(p: OrcBcParams, r, v, rho, kind, ids) -> BcEval:
    """eq1..eq5 of Example 1a at (r, v, rho) without integration."""
    r = _c64(r)
    v = _c64(v)
    rho = _c64(rho)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    n = r.shape[0]
    rho1, p1, dra, aabs, asens = (np.zeros(n) for _ in range(5))
    a = np.zeros_like(r)
    pairs = lib().orc_bc_eval(C.byref(p), n, _ptr(r, C.c_double), _ptr(v, C.c_double), _ptr(rho, C.c_double),
                              _ptr(kind, C.c_uint8), _ptr(ids, C.c_uint32), _ptr(rho1, C.c_double),
                              _ptr(p1, C.c_double), _ptr(a, C.c_double), _ptr(dra, C.c_double),
                              _ptr(aabs, C.c_double), _ptr(asens, C.c_double))
    if pairs < 0:
        raise RuntimeError("particle outside the cell grid")
    return BcEval(rho1, p1, a, dra, aabs, asens, int(pairs))


def bc_step(p: OrcBcParams, r, v, rho, kind, ids, nsteps=1) -> StepResult:
    """nsteps Example 1a steps from (r, v, rho); inputs are not modified."""
    r = _c64(r).copy()
    v = _c64(v).copy()
    rho = _c64(rho).copy()
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    n = r.shape[0]
    pr = np.zeros(n)
    a = np.zeros_like(r)
    d = OrcBcDiag()
    rc = lib().orc_bc_step(C.byref(p), n, _ptr(r, C.c_double), _ptr(v, C.c_double), _ptr(rho, C.c_double),
                           _ptr(kind, C.c_uint8), _ptr(ids, C.c_uint32), int(nsteps), _ptr(pr, C.c_double),
                           _ptr(a, C.c_double), C.byref(d))
    return StepResult(r, v, rho, pr, a, int(d.n_pairs), d.vmax, d.amax, d.dt_cfl, rc)


def bc_sample(p: OrcBcParams, r, ids, A, m, rho):
    """(S, sum of |terms|, neighbour images) of the sampling operator."""
    r = _c64(r)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    A, m, rho = _c64(A), _c64(m), _c64(rho)
    n = r.shape[0]
    S = np.zeros(n)
    Sabs = np.zeros(n)
    pairs = lib().orc_bc_sample(C.byref(p), n, _ptr(r, C.c_double), _ptr(ids, C.c_uint32), _ptr(A, C.c_double),
                                _ptr(m, C.c_double), _ptr(rho, C.c_double), _ptr(S, C.c_double),
                                _ptr(Sabs, C.c_double))
    if pairs < 0:
        raise RuntimeError("particle outside the cell grid")
    return S, Sabs, int(pairs)


# ---------------------------------------------------------------------------
# DEM particle damper of Example 2 (sph_oracle_dem.c).

def dem_params(case, *, fp32=False, g=None, bc=None, dt=None, tank=True) -> OrcDemParams:
    """orc_dem_params from a DEM case (case.extra: E, nu, cf, tank_M, tank_S)."""
    p = OrcDemParams()
    p.dim = case.dim
    for k in range(3):
        p.ncell[k] = int(case.ncell[k])
        p.dom_min[k] = float(case.dom_min[k])
    p.cs = case.cs
    p.h = case.h
    x = case.extra
    p.E, p.nu, p.cf = float(x["E"]), float(x["nu"]), float(x["cf"])
    p.dt = case.dt if dt is None else float(dt)
    gg = case.g if g is None else g
    bb = case.bc if bc is None else bc
    for k in range(3):
        p.g[k] = float(gg[k])
        p.bc[k] = int(bb[k])
    p.fp32 = int(fp32)
    p.tank_M = float(x["tank_M"]) if tank else 0.0
    p.tank_S = float(x["tank_S"]) if tank else 0.0
    return p


def dem_forces(p: OrcDemParams, r, v, R, m, ids, eps=0.0):
    """(F n x dim, F^b (3,), rounding bound per particle, contact count)."""
    r, v, R, m = _c64(r), _c64(v), _c64(R), _c64(m)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    n = r.shape[0]
    F = np.zeros_like(r)
    Fb = np.zeros(3)
    bound = np.zeros(n)
    c = lib().orc_dem_forces(C.byref(p), n, _ptr(r, C.c_double), _ptr(v, C.c_double), _ptr(R, C.c_double),
                             _ptr(m, C.c_double), _ptr(ids, C.c_uint32), float(eps), _ptr(F, C.c_double),
                             _ptr(Fb, C.c_double), _ptr(bound, C.c_double))
    if c < 0:
        raise RuntimeError("particle outside the cell grid")
    return F, Fb, bound, int(c)


@dataclass
class DemResult:
    r: np.ndarray
    v: np.ndarray
    tank: np.ndarray   # (Z, Zdot)
    F: np.ndarray      # last step's contact forces
    diag: OrcDemDiag
    rc: int


def dem_step(p: OrcDemParams, r, v, R, m, kind, ids, tank=(0.0, 0.0), nsteps=1) -> DemResult:
    """nsteps DEM steps from (r, v, tank); inputs are not modified."""
    r, v = _c64(r).copy(), _c64(v).copy()
    R, m = _c64(R), _c64(m)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    t = np.array(tank, np.float64)
    F = np.zeros_like(r)
    d = OrcDemDiag()
    rc = lib().orc_dem_step(C.byref(p), r.shape[0], _ptr(r, C.c_double), _ptr(v, C.c_double),
                            _ptr(R, C.c_double), _ptr(m, C.c_double), _ptr(kind, C.c_uint8),
                            _ptr(ids, C.c_uint32), int(nsteps), _ptr(t, C.c_double), _ptr(F, C.c_double),
                            C.byref(d))
    return DemResult(r, v, t, F, d, rc)

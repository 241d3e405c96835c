"""Thin ctypes binding of libsph_gb300.so (include/sph.h).

The functions carry the C names (sph_create, sph_build_cells, sph_step, ...)
and only marshal arguments: every step of the SPH path runs in the CUDA
kernels of the library.  Torch is used for device memory and streams.

If the compiled library is missing this module raises on first use; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# SPH_CHECKED=1 loads the bounds-checked build (build(check=True)) instead
LIB_PATH = os.path.join(HERE, "libsph_gb300_check.so" if os.environ.get("SPH_CHECKED") == "1"
                        else "libsph_gb300.so")

SPH_OK = 0
SPH_ERR_INVALID = -1
SPH_ERR_CUDA = -2
SPH_ERR_CAPACITY = -3
SPH_ERR_STATUS = -4

SPH_STATUS_OUT_OF_DOMAIN = 1
SPH_STATUS_CELL_OVERFLOW = 2
SPH_STATUS_NAN = 4
SPH_STATUS_CFL = 8
SPH_STATUS_BARRIER_TIMEOUT = 16
SPH_STATUS_DUPLICATE_ID = 32
SPH_STATUS_BOUNDS = 64
SPH_MAX_CELL = 4096

SPH_BATCH_PERSISTENT = 0
SPH_BATCH_PHASED = 1

SPH_PREC_F64 = 0
SPH_PREC_F32 = 1
SPH_RHO_REF_LATTICE = 0
SPH_RHO_REF_LITERAL = 1
SPH_MODEL_WCSPH = 0
SPH_MODEL_EXAMPLE_1A = 1
SPH_MODEL_DEM = 2
SPH_MODEL_FIELDS = 3
SPH_BC_CUTOFF = 0
SPH_BC_SYMMETRIC = 1
SPH_BC_PERIODIC = 2
SPH_FLUID = 0
SPH_BOUNDARY = 1
SPH_DT_FIXED = 0
SPH_DT_ADAPTIVE = 1
# limits of the allocation-free build (sph_build_cells_static)
SPH_STATIC_MAX_PARTICLES = 65536
SPH_STATIC_MAX_CELLS = 262144
SPH_STATIC_MAX_AXIS_CELLS = 16384
# phases of sph_profile_end
SPH_PROF_BUILD, SPH_PROF_DENSITY, SPH_PROF_FORCE, SPH_PROF_FINISH, SPH_PROF_NPHASE = 0, 1, 2, 3, 4


class SphParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("precision", C.c_int),
        ("rho_ref_mode", C.c_int),
        ("clamp_neg_p", C.c_int),
        ("ncell", C.c_int * 3),
        ("dom_min", C.c_double * 3),
        ("cs", C.c_double),
        ("dx", C.c_double),
        ("h", C.c_double),
        ("mass", C.c_double),
        ("rho0", C.c_double),
        ("c0", C.c_double),
        ("gamma", C.c_double),
        ("alpha", C.c_double),
        ("visc_eps", C.c_double),
        ("dt", C.c_double),
        ("g", C.c_double * 3),
        ("model", C.c_int),
        ("boundary", C.c_int * 3),
        ("young", C.c_double),
        ("poisson", C.c_double),
        ("friction", C.c_double),
        ("tank_mass", C.c_double),
        ("tank_stiffness", C.c_double),
        ("dt_mode", C.c_int),
        ("cfl", C.c_double),
    ]


class SphState(C.Structure):
    _fields_ = [
        ("n", C.c_int),
        ("r", C.c_void_p * 3),
        ("v", C.c_void_p * 3),
        ("rho", C.c_void_p),
        ("p", C.c_void_p),
        ("id", C.c_void_p),
        ("kind", C.c_void_p),
        ("radius", C.c_void_p),
        ("mass", C.c_void_p),
    ]


class SphDiag(C.Structure):
    _fields_ = [
        ("n_pairs", C.c_int64),
        ("n_pairs_fluid", C.c_int64),
        ("vmax", C.c_double),
        ("amax", C.c_double),
        ("dt_cfl", C.c_double),
        ("status", C.c_uint32),
        ("dt", C.c_double),
        ("time", C.c_double),
    ]


class SphLawViews(C.Structure):
    _fields_ = [
        ("pos", C.c_void_p),
        ("cell_s", C.c_void_p),
        ("cell_start", C.c_void_p),
        ("params", C.c_void_p),
        ("params_bytes", C.c_int64),
        ("n", C.c_int),
        ("precision", C.c_int),
        ("mask", C.c_void_p),
        ("nnb", C.c_void_p),
        ("ovf", C.c_void_p),
    ]


class SphCaseDesc(C.Structure):
    _fields_ = [("params", SphParams), ("n", C.c_int)]


class SphTune(C.Structure):
    _fields_ = [("block", C.c_int), ("blocks_per_sm", C.c_int), ("spin_limit", C.c_longlong), ("form", C.c_int)]


class SphGrad(C.Structure):
    _fields_ = [
        ("r_bar", C.c_void_p * 3),
        ("v_bar", C.c_void_p * 3),
    ]


_lib = None

# the exported C-ABI symbols (checked by the CPU tests against include/sph.h)
EXPORTS = ("sph_create", "sph_destroy", "sph_last_error", "sph_rho_ref", "sph_build_cells",
           "sph_cell_table", "sph_neighbor_counts", "sph_neighbor_list", "sph_forces", "sph_step",
           "sph_get_status", "sph_profile_begin", "sph_profile_end", "sph_step_adjoint", "sph_batch_create",
           "sph_batch_destroy", "sph_batch_last_error", "sph_batch_step", "sph_batch_get_status",
           "sph_batch_diag", "sph_batch_info", "sph_batch_selftest_barrier", "sph_build_cells_static",
           "sph_static_last_error", "sph_neighbor_images", "sph_sample", "sph_tank_set", "sph_tank_get",
           "sph_reorder_field", "sph_reorder_fields", "sph_law_view", "sph_step_host", "sph_build_save",
           "sph_build_load", "sph_adjoint_of_build", "sph_adjoint_of_saved", "sph_clock_get", "sph_clock_set", "sph_build_cells_into")

SPH_PROF_PHASES = ("build", "density", "force", "finish")


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.sph_create.argtypes = [C.POINTER(SphParams), C.c_int, C.POINTER(vp)]
        L.sph_create.restype = C.c_int
        L.sph_destroy.argtypes = [vp]
        L.sph_destroy.restype = C.c_int
        L.sph_last_error.argtypes = [vp]
        L.sph_last_error.restype = C.c_char_p
        L.sph_rho_ref.argtypes = [vp]
        L.sph_rho_ref.restype = C.c_double
        L.sph_build_cells.argtypes = [vp, C.POINTER(SphState), vp]
        L.sph_build_cells.restype = C.c_int
        L.sph_cell_table.argtypes = [vp, vp, C.POINTER(C.c_int64), vp]
        L.sph_cell_table.restype = C.c_int
        L.sph_neighbor_counts.argtypes = [vp, C.POINTER(SphState), vp, vp]
        L.sph_neighbor_counts.restype = C.c_int
        L.sph_neighbor_list.argtypes = [vp, C.POINTER(SphState), vp, vp, vp]
        L.sph_neighbor_list.restype = C.c_int
        L.sph_neighbor_images.argtypes = [vp, C.POINTER(SphState), vp, vp, vp, vp]
        L.sph_neighbor_images.restype = C.c_int
        L.sph_sample.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sph_sample.restype = C.c_int
        L.sph_reorder_field.argtypes = [vp, vp, vp, C.c_int, vp]
        L.sph_reorder_field.restype = C.c_int
        L.sph_reorder_fields.argtypes = [vp, C.c_int, vp, vp, C.c_int, vp]
        L.sph_reorder_fields.restype = C.c_int
        L.sph_law_view.argtypes = [vp, C.POINTER(SphLawViews)]
        L.sph_law_view.restype = C.c_int
        L.sph_tank_set.argtypes = [vp, C.c_double, C.c_double, vp]
        L.sph_tank_set.restype = C.c_int
        dpp = C.POINTER(C.c_double)
        L.sph_tank_get.argtypes = [vp, dpp, dpp, dpp, dpp, vp]
        L.sph_tank_get.restype = C.c_int
        L.sph_clock_get.argtypes = [vp, dpp, dpp, vp]
        L.sph_clock_get.restype = C.c_int
        L.sph_clock_set.argtypes = [vp, C.c_double, C.c_double, vp]
        L.sph_clock_set.restype = C.c_int
        L.sph_build_cells_into.argtypes = [vp, C.POINTER(SphState), C.POINTER(SphState), C.c_int, C.POINTER(vp),
                                           C.POINTER(vp), C.c_int, vp]
        L.sph_build_cells_into.restype = C.c_int
        L.sph_forces.argtypes = [vp, C.POINTER(SphState), C.POINTER(vp), vp]
        L.sph_forces.restype = C.c_int
        L.sph_step.argtypes = [vp, C.POINTER(SphState), C.c_int, C.POINTER(SphDiag), vp]
        L.sph_step.restype = C.c_int
        L.sph_step_host.argtypes = [vp, C.POINTER(SphState), C.c_int, C.POINTER(SphDiag), vp]
        L.sph_step_host.restype = C.c_int
        L.sph_get_status.argtypes = [vp, C.POINTER(C.c_uint32), C.c_int, vp]
        L.sph_get_status.restype = C.c_int
        L.sph_step_adjoint.argtypes = [vp, C.POINTER(SphState), C.POINTER(SphGrad), C.POINTER(SphGrad), vp, vp]
        L.sph_step_adjoint.restype = C.c_int
        L.sph_build_save.argtypes = [vp, vp, C.POINTER(C.c_int64), vp]
        L.sph_build_save.restype = C.c_int
        L.sph_build_load.argtypes = [vp, vp, C.c_int, vp]
        L.sph_build_load.restype = C.c_int
        L.sph_adjoint_of_build.argtypes = [vp, C.c_int, C.POINTER(SphGrad), C.POINTER(SphGrad), vp, vp]
        L.sph_adjoint_of_build.restype = C.c_int
        L.sph_adjoint_of_saved.argtypes = [vp, vp, C.c_int, C.POINTER(SphGrad), C.POINTER(SphGrad), vp, vp]
        L.sph_adjoint_of_saved.restype = C.c_int
        L.sph_batch_create.argtypes = [C.POINTER(SphCaseDesc), C.c_int, C.POINTER(SphTune), C.POINTER(vp)]
        L.sph_batch_create.restype = C.c_int
        L.sph_batch_destroy.argtypes = [vp]
        L.sph_batch_destroy.restype = C.c_int
        L.sph_batch_last_error.argtypes = [vp]
        L.sph_batch_last_error.restype = C.c_char_p
        L.sph_batch_step.argtypes = [vp, C.POINTER(SphState), C.c_int, vp]
        L.sph_batch_step.restype = C.c_int
        L.sph_batch_get_status.argtypes = [vp, C.POINTER(C.c_uint32), C.c_int, vp]
        L.sph_batch_get_status.restype = C.c_int
        L.sph_batch_diag.argtypes = [vp, C.POINTER(SphDiag), C.POINTER(C.c_int64)]
        L.sph_batch_diag.restype = C.c_int
        L.sph_batch_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_int)]
        L.sph_batch_info.restype = C.c_int
        L.sph_batch_selftest_barrier.argtypes = [vp, C.POINTER(SphState), C.c_longlong, C.POINTER(C.c_uint32), vp]
        L.sph_batch_selftest_barrier.restype = C.c_int
        L.sph_build_cells_static.argtypes = [C.POINTER(SphParams), C.POINTER(SphState), vp, vp, vp]
        L.sph_build_cells_static.restype = C.c_int
        L.sph_static_last_error.argtypes = []
        L.sph_static_last_error.restype = C.c_char_p
        L.sph_profile_begin.argtypes = [vp, C.c_int]
        L.sph_profile_begin.restype = C.c_int
        L.sph_profile_end.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.sph_profile_end.restype = C.c_int
        _lib = L
    return _lib


class SphError(RuntimeError):
    pass


def _check(rc, ctx=None, what=""):
    if rc != SPH_OK:
        msg = lib().sph_last_error(ctx).decode(errors="replace")
        raise SphError(f"{what} failed ({rc}): {msg}")


def params_from_case(case, precision=SPH_PREC_F32, rho_ref_mode=SPH_RHO_REF_LATTICE,
                     clamp_neg_p=True, dt=None, alpha=None, g=None, tank=True, dt_mode=SPH_DT_FIXED,
                     cfl=1.0) -> SphParams:
    p = SphParams()
    p.dim = case.dim
    p.precision = precision
    p.rho_ref_mode = rho_ref_mode
    p.clamp_neg_p = int(clamp_neg_p)
    for k in range(3):
        p.ncell[k] = int(case.ncell[k])
        p.dom_min[k] = float(case.dom_min[k])
    p.cs = case.cs
    p.dx = case.dx
    p.h = case.h
    p.mass = case.mass
    p.rho0 = case.rho0
    p.c0 = case.c0
    p.gamma = case.gamma
    p.alpha = case.alpha if alpha is None else alpha
    p.visc_eps = case.visc_eps
    p.dt = case.dt if dt is None else dt
    gg = case.g if g is None else g
    for k in range(3):
        p.g[k] = float(gg[k])
    p.model = int(getattr(case, "model", SPH_MODEL_WCSPH))
    bc = getattr(case, "bc", (SPH_BC_CUTOFF,) * 3)
    for k in range(3):
        p.boundary[k] = int(bc[k])
    if p.model == SPH_MODEL_DEM:
        x = case.extra
        p.young, p.poisson, p.friction = float(x["E"]), float(x["nu"]), float(x["cf"])
        p.tank_mass = float(x["tank_M"]) if tank else 0.0
        p.tank_stiffness = float(x["tank_S"]) if tank else 0.0
    p.dt_mode = int(dt_mode)
    p.cfl = float(cfl)
    return p


# ---- C-ABI wrappers (same names) -------------------------------------------

def sph_create(params: SphParams, n_capacity: int) -> int:
    out = C.c_void_p()
    rc = lib().sph_create(C.byref(params), int(n_capacity), C.byref(out))
    _check(rc, None, "sph_create")
    return out.value


def sph_destroy(ctx) -> None:
    lib().sph_destroy(ctx)


def sph_last_error(ctx=None) -> str:
    return lib().sph_last_error(ctx).decode(errors="replace")


def sph_rho_ref(ctx) -> float:
    return lib().sph_rho_ref(ctx)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def sph_build_cells(ctx, state: SphState, stream=None) -> None:
    _check(lib().sph_build_cells(ctx, C.byref(state), _stream(stream)), ctx, "sph_build_cells")


def sph_cell_table(ctx, cell_start_ptr: int = 0, stream=None) -> int:
    """Number of cells; copies the start table to cell_start_ptr if given."""
    n = C.c_int64()
    _check(lib().sph_cell_table(ctx, C.c_void_p(cell_start_ptr or None), C.byref(n), _stream(stream)),
           ctx, "sph_cell_table")
    return n.value


def sph_neighbor_counts(ctx, state: SphState, counts_ptr: int, stream=None) -> None:
    _check(lib().sph_neighbor_counts(ctx, C.byref(state), C.c_void_p(counts_ptr), _stream(stream)),
           ctx, "sph_neighbor_counts")


def sph_neighbor_list(ctx, state: SphState, offsets_ptr: int, ids_ptr: int, stream=None) -> None:
    _check(lib().sph_neighbor_list(ctx, C.byref(state), C.c_void_p(offsets_ptr), C.c_void_p(ids_ptr),
                                   _stream(stream)), ctx, "sph_neighbor_list")


def sph_neighbor_images(ctx, state: SphState, offsets_ptr: int, ids_ptr: int, images_ptr: int,
                        stream=None) -> None:
    _check(lib().sph_neighbor_images(ctx, C.byref(state), C.c_void_p(offsets_ptr), C.c_void_p(ids_ptr),
                                     C.c_void_p(images_ptr or None), _stream(stream)), ctx, "sph_neighbor_images")


def sph_sample(ctx, A_ptr: int, m_ptr: int, rho_ptr: int, S_ptr: int, stream=None) -> None:
    _check(lib().sph_sample(ctx, C.c_void_p(A_ptr), C.c_void_p(m_ptr), C.c_void_p(rho_ptr), C.c_void_p(S_ptr),
                            _stream(stream)), ctx, "sph_sample")


def sph_reorder_fields(ctx, in_ptrs, out_ptrs, elem_bytes: int, stream=None) -> None:
    """Reorder several device fields of one element size in one pass (see
    sph_reorder_field); in_ptrs / out_ptrs: equal-length lists of device
    pointers."""
    nf = len(in_ptrs)
    if len(out_ptrs) != nf:
        raise SphError("sph_reorder_fields: as many outputs as inputs")
    ins = (C.c_void_p * max(nf, 1))(*in_ptrs)
    outs = (C.c_void_p * max(nf, 1))(*out_ptrs)
    _check(lib().sph_reorder_fields(ctx, nf, ins, outs, int(elem_bytes), _stream(stream)), ctx,
           "sph_reorder_fields")


def sph_reorder_field(ctx, in_ptr: int, out_ptr: int, elem_bytes: int, stream=None) -> None:
    _check(lib().sph_reorder_field(ctx, C.c_void_p(in_ptr), C.c_void_p(out_ptr), int(elem_bytes),
                                   _stream(stream)), ctx, "sph_reorder_field")


def sph_law_view(ctx) -> SphLawViews:
    v = SphLawViews()
    _check(lib().sph_law_view(ctx, C.byref(v)), ctx, "sph_law_view")
    return v


def sph_tank_set(ctx, Z: float, Zdot: float, stream=None) -> None:
    _check(lib().sph_tank_set(ctx, float(Z), float(Zdot), _stream(stream)), ctx, "sph_tank_set")


def sph_tank_get(ctx, stream=None):
    """(Z, Zdot, Zddot, wall force (3,)) of the DEM tank."""
    z, zd, zdd = C.c_double(), C.c_double(), C.c_double()
    fb = (C.c_double * 3)()
    _check(lib().sph_tank_get(ctx, C.byref(z), C.byref(zd), C.byref(zdd), fb, _stream(stream)), ctx,
           "sph_tank_get")
    return z.value, zd.value, zdd.value, np.array(list(fb))


def sph_build_cells_into(ctx, state_in: SphState, state_out: SphState, ins, outs, elem_bytes: int,
                         stream=None) -> None:
    """Build of a field-model context into a second state, reordering the
    fields (device pointers ins -> outs) in the same gather."""
    n = len(ins)
    a = (C.c_void_p * max(1, n))(*[C.c_void_p(p) for p in ins])
    b = (C.c_void_p * max(1, n))(*[C.c_void_p(p) for p in outs])
    _check(lib().sph_build_cells_into(ctx, C.byref(state_in), C.byref(state_out), n, a, b, int(elem_bytes),
                                      _stream(stream)), ctx, "sph_build_cells_into")


def sph_clock_get(ctx, stream=None):
    """(step size of the next step, simulated time so far) of the context."""
    dt, t = C.c_double(), C.c_double()
    _check(lib().sph_clock_get(ctx, C.byref(dt), C.byref(t), _stream(stream)), ctx, "sph_clock_get")
    return dt.value, t.value


def sph_clock_set(ctx, dt_next: float, time: float, stream=None) -> None:
    _check(lib().sph_clock_set(ctx, float(dt_next), float(time), _stream(stream)), ctx, "sph_clock_set")


def sph_forces(ctx, state: SphState, a_ptrs, stream=None) -> None:
    arr = (C.c_void_p * 3)(*[C.c_void_p(p) if p else None for p in a_ptrs])
    _check(lib().sph_forces(ctx, C.byref(state), arr, _stream(stream)), ctx, "sph_forces")


def sph_step(ctx, state: SphState, nsteps: int, diag: Optional[SphDiag] = None, stream=None) -> None:
    d = C.byref(diag) if diag is not None else None
    _check(lib().sph_step(ctx, C.byref(state), int(nsteps), d, _stream(stream)), ctx, "sph_step")


def sph_step_host(ctx, state: SphState, nsteps: int, diag: Optional[SphDiag] = None, stream=None) -> None:
    """sph_step on a state whose arrays are HOST pointers (page-locked for full
    speed): copy in, step, copy back; returns when the host arrays hold the
    new state."""
    d = C.byref(diag) if diag is not None else None
    _check(lib().sph_step_host(ctx, C.byref(state), int(nsteps), d, _stream(stream)), ctx, "sph_step_host")


def host_state_view(arrays) -> SphState:
    """SphState over host tensors (dict with r, v: lists, rho, p, id, kind and
    optionally radius, mass)."""
    s = SphState()
    s.n = int(arrays["id"].numel())
    for k in range(3):
        s.r[k] = arrays["r"][k].data_ptr() if k < len(arrays["r"]) else None
        s.v[k] = arrays["v"][k].data_ptr() if k < len(arrays["v"]) else None
    s.rho = arrays["rho"].data_ptr() if arrays.get("rho") is not None else None
    s.p = arrays["p"].data_ptr() if arrays.get("p") is not None else None
    s.id = arrays["id"].data_ptr()
    s.kind = arrays["kind"].data_ptr()
    s.radius = arrays["radius"].data_ptr() if arrays.get("radius") is not None else None
    s.mass = arrays["mass"].data_ptr() if arrays.get("mass") is not None else None
    return s


def sph_get_status(ctx, sync=True, stream=None) -> int:
    v = C.c_uint32()
    _check(lib().sph_get_status(ctx, C.byref(v), int(sync), _stream(stream)), ctx, "sph_get_status")
    return int(v.value)


def sph_step_adjoint(ctx, state: SphState, g_np1: SphGrad, g_n: SphGrad, alpha_bar_ptr: int = 0,
                     stream=None) -> None:
    _check(lib().sph_step_adjoint(ctx, C.byref(state), C.byref(g_np1), C.byref(g_n),
                                  C.c_void_p(alpha_bar_ptr or None), _stream(stream)), ctx, "sph_step_adjoint")


def sph_build_save(ctx, dst_ptr: int = 0, stream=None) -> int:
    """Size in bytes of the last build + density products; with dst_ptr also
    enqueue their copy into that device buffer."""
    b = C.c_int64()
    _check(lib().sph_build_save(ctx, C.c_void_p(dst_ptr or None), C.byref(b), _stream(stream)), ctx,
           "sph_build_save")
    return int(b.value)


def sph_build_load(ctx, src_ptr: int, n: int, stream=None) -> None:
    _check(lib().sph_build_load(ctx, C.c_void_p(src_ptr), int(n), _stream(stream)), ctx, "sph_build_load")


def sph_adjoint_of_build(ctx, n: int, g_np1: SphGrad, g_n: SphGrad, alpha_bar_ptr: int = 0, stream=None) -> None:
    _check(lib().sph_adjoint_of_build(ctx, int(n), C.byref(g_np1), C.byref(g_n), C.c_void_p(alpha_bar_ptr or None),
                                      _stream(stream)), ctx, "sph_adjoint_of_build")


def sph_adjoint_of_saved(ctx, saved_ptr: int, n: int, g_np1: SphGrad, g_n: SphGrad, alpha_bar_ptr: int = 0,
                         stream=None) -> None:
    _check(lib().sph_adjoint_of_saved(ctx, C.c_void_p(saved_ptr), int(n), C.byref(g_np1), C.byref(g_n),
                                      C.c_void_p(alpha_bar_ptr or None), _stream(stream)), ctx,
           "sph_adjoint_of_saved")


def grad_view(r_bar, v_bar) -> SphGrad:
    """SphGrad over lists of device tensors (dim entries each)."""
    g = SphGrad()
    for k in range(3):
        g.r_bar[k] = r_bar[k].data_ptr() if k < len(r_bar) else None
        g.v_bar[k] = v_bar[k].data_ptr() if k < len(v_bar) else None
    return g


def sph_static_last_error() -> str:
    return lib().sph_static_last_error().decode(errors="replace")


def sph_build_cells_static(params: SphParams, state: SphState, cell_start_ptr: int = 0, status_ptr: int = 0,
                           stream=None) -> None:
    """The build without a context or any allocation (see include/sph.h):
    for callers that cannot allocate device memory where they need it."""
    rc = lib().sph_build_cells_static(C.byref(params), C.byref(state), C.c_void_p(cell_start_ptr or None),
                                      C.c_void_p(status_ptr or None), _stream(stream))
    if rc != SPH_OK:
        raise SphError(f"sph_build_cells_static failed ({rc}): {sph_static_last_error()}")


# ---- batched form ---------------------------------------------------------

def _bcheck(rc, b, what):
    if rc != SPH_OK:
        msg = lib().sph_batch_last_error(b).decode(errors="replace")
        raise SphError(f"{what} failed ({rc}): {msg}")


def sph_batch_create(descs, tune: Optional[SphTune] = None) -> int:
    arr = (SphCaseDesc * len(descs))(*descs)
    out = C.c_void_p()
    rc = lib().sph_batch_create(arr, len(descs), C.byref(tune) if tune is not None else None, C.byref(out))
    _bcheck(rc, None, "sph_batch_create")
    return out.value


def sph_batch_destroy(b) -> None:
    lib().sph_batch_destroy(b)


def sph_batch_last_error(b=None) -> str:
    return lib().sph_batch_last_error(b).decode(errors="replace")


def sph_batch_step(b, state: SphState, nsteps: int, stream=None) -> None:
    _bcheck(lib().sph_batch_step(b, C.byref(state), int(nsteps), _stream(stream)), b, "sph_batch_step")


def sph_batch_get_status(b, sync=True, stream=None) -> int:
    v = C.c_uint32()
    _bcheck(lib().sph_batch_get_status(b, C.byref(v), int(sync), _stream(stream)), b, "sph_batch_get_status")
    return int(v.value)


def sph_batch_diag(b, ncases: int):
    arr = (SphDiag * ncases)()
    npair = C.c_int64()
    _bcheck(lib().sph_batch_diag(b, arr, C.byref(npair)), b, "sph_batch_diag")
    return list(arr), int(npair.value)


def sph_batch_info(b):
    blk, grd, gr, nt = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _bcheck(lib().sph_batch_info(b, C.byref(blk), C.byref(grd), C.byref(gr), C.byref(nt)), b, "sph_batch_info")
    return {"block": blk.value, "grid": grd.value, "graph_used": gr.value, "n_total": nt.value}


def sph_batch_selftest_barrier(b, state: SphState, spin_limit: int, stream=None) -> int:
    v = C.c_uint32()
    _bcheck(lib().sph_batch_selftest_barrier(b, C.byref(state), int(spin_limit), C.byref(v), _stream(stream)), b,
            "sph_batch_selftest_barrier")
    return int(v.value)


def sph_profile_begin(ctx, max_steps: int) -> None:
    _check(lib().sph_profile_begin(ctx, int(max_steps)), ctx, "sph_profile_begin")


def sph_profile_end(ctx):
    """(dict phase -> summed device ms, number of recorded steps)."""
    ms = (C.c_double * len(SPH_PROF_PHASES))()
    n = C.c_int64()
    _check(lib().sph_profile_end(ctx, ms, C.byref(n)), ctx, "sph_profile_end")
    return {k: ms[i] for i, k in enumerate(SPH_PROF_PHASES)}, int(n.value)


# ---- torch-side convenience ---------------------------------------------------

@dataclass
class DeviceState:
    """Device SoA particle state held in torch tensors plus its SphState view."""
    r: list
    v: list
    rho: object
    p: object
    id: object
    kind: object
    n: int
    dim: int
    radius: object = None
    mass: object = None

    def view(self) -> SphState:
        s = SphState()
        s.n = self.n
        for k in range(3):
            s.r[k] = self.r[k].data_ptr() if k < self.dim else None
            s.v[k] = self.v[k].data_ptr() if k < self.dim else None
        s.rho = self.rho.data_ptr()
        s.p = self.p.data_ptr()
        s.id = self.id.data_ptr()
        s.kind = self.kind.data_ptr()
        s.radius = self.radius.data_ptr() if self.radius is not None else None
        s.mass = self.mass.data_ptr() if self.mass is not None else None
        return s

    def to_host(self):
        """(r (n,dim) f64, v (n,dim) f64, rho, p, id, kind) as numpy, in the
        current (canonical) order."""
        r = np.stack([t.cpu().numpy() for t in self.r], axis=1)
        v = np.stack([t.cpu().double().numpy() for t in self.v], axis=1)
        return (r, v, self.rho.cpu().double().numpy(), self.p.cpu().double().numpy(),
                self.id.cpu().numpy().astype(np.uint32), self.kind.cpu().numpy())


def device_state(r, v, kind, ids, precision=SPH_PREC_F32, device="cuda", rho=None, radius=None,
                 mass=None) -> DeviceState:
    """rho: the initial density field (SPH_MODEL_EXAMPLE_1A), else zeros;
    radius, mass: per-sphere arrays (SPH_MODEL_DEM)."""
    import torch
    r = np.asarray(r, np.float64)
    n, dim = r.shape
    tdt = torch.float32 if precision == SPH_PREC_F32 else torch.float64
    rr = [torch.tensor(np.ascontiguousarray(r[:, k]), dtype=torch.float64, device=device) for k in range(dim)]
    vv = [torch.tensor(np.ascontiguousarray(np.asarray(v)[:, k]), dtype=tdt, device=device) for k in range(dim)]
    return DeviceState(
        r=rr, v=vv,
        rho=(torch.zeros(n, dtype=tdt, device=device) if rho is None
             else torch.tensor(np.asarray(rho, np.float64), dtype=tdt, device=device)),
        p=torch.zeros(n, dtype=tdt, device=device),
        id=torch.tensor(np.asarray(ids, np.uint32).astype(np.int32), dtype=torch.int32, device=device),
        kind=torch.tensor(np.asarray(kind, np.uint8), dtype=torch.uint8, device=device),
        n=n, dim=dim,
        radius=None if radius is None else torch.tensor(np.asarray(radius, np.float64), dtype=tdt, device=device),
        mass=None if mass is None else torch.tensor(np.asarray(mass, np.float64), dtype=tdt, device=device))


class Simulation:
    """A context plus a device state for one case (the usual way to drive the ABI)."""

    def __init__(self, case, precision=SPH_PREC_F32, capacity=None, **kw):
        self.case = case
        self.precision = precision
        self.params = params_from_case(case, precision=precision, **kw)
        self.ctx = sph_create(self.params, capacity or case.n)
        dem = getattr(case, "model", 0) == SPH_MODEL_DEM
        self.state = device_state(case.r, case.v, case.kind, case.id, precision,
                                  rho=None if dem else getattr(case, "rho", None),
                                  radius=case.rho if dem else None, mass=case.extra["m"] if dem else None)
        self._view = self.state.view()
        if dem and self.params.tank_mass > 0.0:
            sph_tank_set(self.ctx, case.extra.get("z0", 0.0), 0.0)

    def close(self):
        if self.ctx:
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1, diag=False, stream=None):
        d = SphDiag() if diag else None
        sph_step(self.ctx, self._view, nsteps, d, stream)
        return d

    # ---- checkpoint / resume ------------------------------------------------
    def save(self, path):
        """Checkpoint to an .npz file: the context's parameters, the state's
        arrays exactly as they are on the device (canonical order, working
        precision), the clock (next step size, elapsed time) and, for the DEM
        model, the tank (Z, Zdot).  A simulation
        made by Simulation.restore(path) continues bit for bit."""
        st = self.state
        data = {"format": np.array([1]), "n": np.array([st.n]), "dim": np.array([st.dim])}
        for name, ctype in SphParams._fields_:
            val = getattr(self.params, name)
            data["param_" + name] = np.array(list(val) if hasattr(val, "__len__") else [val])
        for k in range(st.dim):
            data[f"r{k}"] = st.r[k].cpu().numpy()
            data[f"v{k}"] = st.v[k].cpu().numpy()
        for name in ("rho", "p", "id", "kind", "radius", "mass"):
            t = getattr(st, name)
            if t is not None:
                data[name] = t.cpu().numpy()
        if self.params.model == SPH_MODEL_DEM and self.params.tank_mass > 0.0:
            Z, Zd, _, _ = sph_tank_get(self.ctx)
            data["tank"] = np.array([Z, Zd])
        data["clock"] = np.array(sph_clock_get(self.ctx))   # next step size, elapsed time
        np.savez(path, **data)

    @classmethod
    def restore(cls, path, capacity=None):
        """A Simulation from a checkpoint written by save() (no case needed)."""
        import torch
        z = np.load(path)
        if int(z["format"][0]) != 1:
            raise SphError(f"{path}: unknown checkpoint format")
        p = SphParams()
        for name, ctype in SphParams._fields_:
            if "param_" + name not in z.files:
                continue                     # (a field added after the checkpoint: its default)
            vals = z["param_" + name]
            cur = getattr(p, name)
            if hasattr(cur, "__len__"):
                for k in range(len(cur)):
                    cur[k] = vals[k].item()
            else:
                setattr(p, name, vals[0].item())
        n, dim = int(z["n"][0]), int(z["dim"][0])
        self = cls.__new__(cls)
        self.case = None
        self.precision = p.precision
        self.params = p
        self.ctx = sph_create(p, capacity or n)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
        self.state = DeviceState(
            r=[dev(z[f"r{k}"]) for k in range(dim)], v=[dev(z[f"v{k}"]) for k in range(dim)],
            rho=dev(z["rho"]), p=dev(z["p"]), id=dev(z["id"]), kind=dev(z["kind"]), n=n, dim=dim,
            radius=dev(z["radius"]) if "radius" in z.files else None,
            mass=dev(z["mass"]) if "mass" in z.files else None)
        self._view = self.state.view()
        if "tank" in z.files:
            sph_tank_set(self.ctx, float(z["tank"][0]), float(z["tank"][1]))
        if "clock" in z.files:
            sph_clock_set(self.ctx, float(z["clock"][0]), float(z["clock"][1]))
        return self

    def build_cells(self, stream=None):
        sph_build_cells(self.ctx, self._view, stream)

    def forces(self):
        import torch
        tdt = torch.float32 if self.precision == SPH_PREC_F32 else torch.float64
        a = [torch.zeros(self.state.n, dtype=tdt, device="cuda") for _ in range(self.state.dim)]
        sph_forces(self.ctx, self._view, [t.data_ptr() for t in a] + [0] * (3 - self.state.dim))
        return a

    def neighbour_lists(self):
        import torch
        n = self.state.n
        counts = torch.zeros(n, dtype=torch.int32, device="cuda")
        sph_neighbor_counts(self.ctx, self._view, counts.data_ptr())
        offs = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        offs[1:] = torch.cumsum(counts.to(torch.int64), 0)
        tot = int(offs[-1].item())
        ids = torch.zeros(max(tot, 1), dtype=torch.int32, device="cuda")
        sph_neighbor_list(self.ctx, self._view, offs.data_ptr(), ids.data_ptr())
        return offs.cpu().numpy(), ids[:tot].cpu().numpy().astype(np.uint32), counts.cpu().numpy()

    def neighbour_images(self):
        """(offsets, ids, image codes, counts) of every particle's neighbour
        images, numpy, in the canonical order the call leaves."""
        import torch
        n = self.state.n
        counts = torch.zeros(n, dtype=torch.int32, device="cuda")
        sph_neighbor_counts(self.ctx, self._view, counts.data_ptr())
        offs = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        offs[1:] = torch.cumsum(counts.to(torch.int64), 0)
        tot = int(offs[-1].item())
        ids = torch.zeros(max(tot, 1), dtype=torch.int32, device="cuda")
        img = torch.zeros(max(tot, 1), dtype=torch.uint8, device="cuda")
        sph_neighbor_images(self.ctx, self._view, offs.data_ptr(), ids.data_ptr(), img.data_ptr())
        return (offs.cpu().numpy(), ids[:tot].cpu().numpy().astype(np.uint32), img[:tot].cpu().numpy(),
                counts.cpu().numpy())

    def sample(self, A, m, rho, stream=None):
        """The sampling operator on the cells of the last build: A, m, rho
        device tensors in the state's current order; returns S."""
        import torch
        S = torch.empty_like(A)
        sph_sample(self.ctx, A.data_ptr(), m.data_ptr(), rho.data_ptr(), S.data_ptr(), stream)
        return S

    def tank(self):
        """(Z, Zdot, Zddot, wall force) of the DEM tank."""
        return sph_tank_get(self.ctx)

    def cell_table(self):
        import torch
        ncells = sph_cell_table(self.ctx)
        out = torch.empty(ncells + 1, dtype=torch.int32, device="cuda")
        sph_cell_table(self.ctx, out.data_ptr())
        return out.cpu().numpy().astype(np.uint32)

    def status(self, sync=True):
        return sph_get_status(self.ctx, sync)


class Batch:
    """Packed device state of many cases plus a batched context."""

    def __init__(self, cases, precision=SPH_PREC_F32, tune: Optional[SphTune] = None, **kw):
        self.cases = cases
        self.precision = precision
        dim = cases[0].dim
        self.offsets = np.cumsum([0] + [c.n for c in cases])
        descs = []
        for c in cases:
            d = SphCaseDesc()
            d.params = params_from_case(c, precision=precision, **kw)
            d.n = c.n
            descs.append(d)
        self.handle = sph_batch_create(descs, tune)
        r = np.concatenate([c.r for c in cases], axis=0)
        v = np.concatenate([c.v for c in cases], axis=0)
        kind = np.concatenate([c.kind for c in cases])
        ids = np.concatenate([c.id for c in cases])
        self.state = device_state(r, v, kind, ids, precision)
        self._view = self.state.view()
        import torch
        # a stream of its own: the legacy default stream cannot be captured
        # into a CUDA graph
        self.stream = torch.cuda.Stream()

    def close(self):
        if self.handle:
            self.stream.synchronize()
            sph_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1):
        """nsteps steps of every case, ordered after the current stream's work."""
        import torch
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        sph_batch_step(self.handle, self._view, nsteps, self.stream)
        cur.wait_stream(self.stream)

    def status(self, sync=True):
        return sph_batch_get_status(self.handle, sync, self.stream)

    def info(self):
        return sph_batch_info(self.handle)

    def case_host(self, c):
        """(r, v, rho, p, id, kind) of case c, numpy, in its canonical order."""
        a, b = int(self.offsets[c]), int(self.offsets[c + 1])
        st = self.state
        r = np.stack([t[a:b].cpu().numpy() for t in st.r], axis=1)
        v = np.stack([t[a:b].cpu().double().numpy() for t in st.v], axis=1)
        return (r, v, st.rho[a:b].cpu().double().numpy(), st.p[a:b].cpu().double().numpy(),
                st.id[a:b].cpu().numpy().astype(np.uint32), st.kind[a:b].cpu().numpy())

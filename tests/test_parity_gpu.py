"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Integer work (cell sort, cell table, neighbour lists, pair counts) must match
bit for bit; floating point within the tolerances stated per field below.
Error metric (reading C12): max_i |f_i - f_i^ref| / max_i |f_i^ref| per field;
positions are compared by displacement over the step.
"""
import json
import os

import numpy as np
import pytest

from paper_1710_08259_gb300 import cases as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08259_gb300 import build as B
    B.build()
    from paper_1710_08259_gb300 import sph
    return sph


REPORT = []


def report(name, **vals):
    REPORT.append({"test": name, **{k: float(v) for k, v in vals.items()}})
    path = os.environ.get("SPH_ERR_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(REPORT, f, indent=1)
    print(name, vals)


def rel(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.abs(ref).max()
    if den == 0:
        return float(np.abs(got - ref).max())
    return float(np.abs(got - ref).max() / den)


def _inv(ids):
    inv = np.empty(int(ids.max()) + 1, np.int64)
    inv[ids] = np.arange(ids.size)
    return inv


def _cases_small():
    # cells of edge 2h (the 3^D stencil) and, suffix _h, of edge h (the 5^D
    # stencil walked as rows)
    out = []
    for k, sfx in ((1, ""), (2, "_h")):
        out += [
            ("cloud2" + sfx, C.random_cloud(2, 3000, seed=31, box=0.12, cells_per_radius=k)),
            ("cloud3" + sfx, C.random_cloud(3, 4000, seed=32, box=0.08, cells_per_radius=k)),
            ("dam2" + sfx, C.small_dam_break(2, 30, seed=33, cells_per_radius=k)),
            ("dam3" + sfx, C.small_dam_break(3, 12, seed=34, cells_per_radius=k)),
        ]
    return out


SMALL = _cases_small()
PRECS = ["f64", "f32"]


def _prec(S, name):
    return S.SPH_PREC_F64 if name == "f64" else S.SPH_PREC_F32


# --- cell build ---------------------------------------------------------------

@pytest.mark.parametrize("name,case", SMALL, ids=[c[0] for c in SMALL])
@pytest.mark.parametrize("prec", PRECS)
def test_cell_build_bitexact(S, orc, name, case, prec):
    sim = S.Simulation(case, precision=_prec(S, prec))
    sim.build_cells()
    r, v, _, _, ids, kind = sim.state.to_host()
    order, start, cell_of, bad = orc.sort_cells(orc.params(case), case.r, case.id)
    assert bad == 0
    assert np.array_equal(ids, case.id[order])
    assert np.array_equal(sim.cell_table(), start)
    inv = _inv(case.id)
    assert np.array_equal(r, case.r[inv[ids]])          # positions moved, not changed
    assert np.array_equal(kind, case.kind[inv[ids]])
    assert sim.status() == 0
    # rebuilding a sorted state is the identity
    sim.build_cells()
    r2, _, _, _, ids2, _ = sim.state.to_host()
    assert np.array_equal(ids2, ids) and np.array_equal(r2, r)


# --- neighbour lists and pair counts -------------------------------------------

@pytest.mark.parametrize("name,case", SMALL, ids=[c[0] for c in SMALL])
@pytest.mark.parametrize("prec", PRECS)
def test_neighbour_lists_bitexact(S, orc, name, case, prec):
    sim = S.Simulation(case, precision=_prec(S, prec))
    offs, nbr, counts = sim.neighbour_lists()
    _, _, _, _, ids, _ = sim.state.to_host()
    ro, rl = orc.neighbours(orc.params(case), case.r, case.id, method="cells", fp32=(prec == "f32"))
    inv = _inv(case.id)
    for i in range(case.n):
        k = inv[ids[i]]
        ref = rl[ro[k]:ro[k + 1]]
        got = nbr[offs[i]:offs[i + 1]]
        assert np.array_equal(got, ref), (i, int(ids[i]))
    assert int(counts.sum()) == int(ro[-1])


# --- density, pressure, accelerations --------------------------------------------

# Tolerances.  The raw metric (reading C12) max_i |f - f_ref| / max_i |f_ref|
# is reported for every field.  The bound that is asserted is a first-order
# error bound per particle for a relative error eps in the densities and in
# every arithmetic operation (eps = 1e-5, the per-step tolerance; FP64 is held
# to eps = 1e-12):
#   rho_i : eps |rho_i|
#   p_i   : eps gamma (|p_i| + B)            (dp = gamma (p + B) drho/rho)
#   a_i   : eps (G_i + A_i)                  G_i = density sensitivity of a_i,
#                                            A_i = sum_j |pair term| + |g|
#   v_i   : eps |v0_i| + dt * bound(a_i)
#   dr_i  : dt * bound(v_i)
# The assertion is max_i |err_i| / bound_i <= 1.  The reported "eq" numbers
# are the same ratio times eps: the equivalent relative error.
EPS = {"f64": 1e-12, "f32": 1e-5}


def bounded_errors(case, eps, got, ref, sens, k, kind):
    """Equivalent relative errors (|err| / first-order bound * eps)."""
    fl = kind == 0
    B = case.c0 ** 2 * case.rho0 / case.gamma
    out = {}
    if "rho" in got:
        out["rho"] = float((np.abs(got["rho"] - ref["rho"][k]) / np.abs(ref["rho"][k])).max())
    if "p" in got:
        bp = case.gamma * (np.abs(ref["p"][k]) + B)
        out["p"] = float((np.abs(got["p"] - ref["p"][k]) / bp).max())
    ba = (sens["G"][k] + sens["A"][k])[fl]
    if "a" in got:
        out["a"] = float((np.linalg.norm(got["a"][fl] - ref["a"][k][fl], axis=1) / ba).max())
    if "v" in got:
        v0 = np.linalg.norm(case.v[k][fl], axis=1)
        bv = v0 + case.dt * ba
        out["v"] = float((np.linalg.norm(got["v"][fl] - ref["v"][k][fl], axis=1) / bv).max())
        out["dr"] = float((np.linalg.norm(got["dr"][fl] - ref["dr"][fl], axis=1) / (case.dt * bv)).max())
    return out


def oracle_sensitivities(orc, P, case):
    orho, opr, _ = orc.density(P, case.r, case.id)
    oa, A, G = orc.accel(P, case.r, case.v, case.kind, case.id, orho, opr, with_abs=True)
    return {"rho": orho, "p": opr, "a": oa}, {"A": A, "G": G}


@pytest.mark.parametrize("name,case", SMALL, ids=[c[0] for c in SMALL])
@pytest.mark.parametrize("prec", PRECS)
def test_forces_parity(S, orc, name, case, prec):
    sim = S.Simulation(case, precision=_prec(S, prec))
    a = sim.forces()
    r, v, rho, p, ids, kind = sim.state.to_host()
    a = np.stack([t.cpu().double().numpy() for t in a], axis=1)
    k = _inv(case.id)[ids]
    ref, sens = oracle_sensitivities(orc, orc.params(case), case)
    e = bounded_errors(case, EPS[prec], {"rho": rho, "p": p, "a": a}, ref, sens, k, kind)
    report(f"forces[{name}-{prec}]", **e, raw_rho=rel(rho, ref["rho"][k]), raw_p=rel(p, ref["p"][k]),
           raw_a=rel(a, ref["a"][k]))
    for f in ("rho", "p", "a"):
        assert e[f] <= EPS[prec], (f, e[f])
    assert np.all(a[kind != 0] == 0)


@pytest.mark.parametrize("name,case", SMALL, ids=[c[0] for c in SMALL])
@pytest.mark.parametrize("prec", PRECS)
def test_step_parity(S, orc, name, case, prec):
    sim = S.Simulation(case, precision=_prec(S, prec))
    d = sim.step(1, diag=True)
    r, v, rho, p, ids, kind = sim.state.to_host()
    P = orc.params(case, fp32_neighbours=(prec == "f32"))
    res = orc.step(P, case.r, case.v, case.kind, case.id, 1)
    ref, sens = oracle_sensitivities(orc, P, case)
    k = _inv(case.id)[ids]
    dr_g = r - case.r[k]
    dr_o = res.r[k] - case.r[k]
    ref.update({"rho": res.rho, "p": res.p, "v": res.v, "dr": dr_o})
    e = bounded_errors(case, EPS[prec], {"rho": rho, "p": p, "v": v, "dr": dr_g}, ref, sens, k, kind)
    report(f"step[{name}-{prec}]", **e, raw_v=rel(v, res.v[k]), raw_dr=rel(dr_g, dr_o), raw_p=rel(p, res.p[k]))
    for f in ("dr", "v", "rho", "p"):
        assert e[f] <= EPS[prec], (f, e[f])
    assert d.n_pairs == res.n_pairs
    assert d.vmax == pytest.approx(res.vmax, rel=1e-3 if prec == "f32" else 1e-12)
    assert d.amax == pytest.approx(res.amax, rel=1e-2 if prec == "f32" else 1e-10)
    assert np.array_equal(r[kind == 1], case.r[k][kind == 1])


# --- the stated per-step tolerance, raw, on states away from rest -----------------
#
# Reading C12: per field, max_i |f_i - f_i^ref| / max_i |f_i^ref| (vectors by
# their Euclidean norm per particle, positions by the displacement over the
# step), one FP32 GPU step against one FP64 oracle step from the same state.
# From rest p is a jitter residue near zero and the metric means little, so
# these cases start where the flow is developed: the oracle's own state after
# thousands of steps of the 2D and 3D dam breaks, and a compressed, swirling
# state (hydrostatic-like pressure, |v| ~ 1 m/s) up to the full 1.44 M-particle
# workload.  rho, v and the displacement are held to the stated 1e-5.  p and
# a are functions of rho through the stiff EOS (reading C12b): an error e in
# rho moves p by gamma (p + B) e, so their raw error is bounded by the stated
# 1e-5 carried through that amplification, gamma (max p + B) / max p for p
# and max_i (G_i + A_i) / max_i |a_i| for a (G, A: the oracle's density
# sensitivity and absolute pair sum per particle).
C12_STEP = 1e-5


def _nrm(x):
    x = np.asarray(x, np.float64)
    return np.linalg.norm(x, axis=1) if x.ndim == 2 else np.abs(x)


def c12(got, ref):
    return float(_nrm(got - ref).max() / _nrm(ref).max())


def _one_step_c12(S, orc, case, name):
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    a = sim.forces()
    _, _, _, _, ids_a, kind_a = sim.state.to_host()
    a = np.stack([t.cpu().double().numpy() for t in a], axis=1)
    d = sim.step(1, diag=True)
    r, v, rho, p, ids, kind = sim.state.to_host()
    assert sim.status() == 0
    sim.close()
    P = orc.params(case, fp32_neighbours=True)
    res = orc.step(P, case.r, case.v, case.kind, case.id, 1)
    orho, opr, _ = orc.density(P, case.r, case.id)
    oa, A, G = orc.accel(P, case.r, case.v, case.kind, case.id, orho, opr, with_abs=True)
    inv = _inv(case.id)
    k, ka = inv[ids], inv[ids_a]
    fl, fla = kind == 0, kind_a == 0
    B = case.c0 ** 2 * case.rho0 / case.gamma
    e = {"rho": c12(rho, res.rho[k]), "p": c12(p, res.p[k]), "a": c12(a[fla], oa[ka][fla]),
         "v": c12(v[fl], res.v[k][fl]), "dr": c12((r - case.r[k])[fl], (res.r[k] - case.r[k])[fl])}
    amp = {"p": case.gamma * (np.abs(res.p).max() + B) / np.abs(res.p).max(),
           "a": float((G + A)[case.kind == 0].max() / _nrm(oa[case.kind == 0]).max())}
    report(f"c12_step[{name}]", **e, max_p=np.abs(res.p).max(), max_v=_nrm(res.v[case.kind == 0]).max(),
           max_a=_nrm(oa[case.kind == 0]).max(), amp_p=amp["p"], amp_a=amp["a"])
    assert d.n_pairs == res.n_pairs
    for f in ("rho", "v", "dr"):
        assert e[f] <= C12_STEP, (f, e[f])
    for f in ("p", "a"):
        assert e[f] <= C12_STEP * amp[f], (f, e[f], amp[f])
    return e


@pytest.fixture(scope="module")
def developed(orc):
    """Oracle FP64 states of the 2D (64 x 64, 3000 steps = 0.22 s: front at
    x = 1.07 m, |v| up to 3.5 m/s, p up to 10 kPa) and a 3D (12^3, 450 steps
    = 0.16 s: |v| up to 3 m/s, p up to 46 kPa, before the surge meets the end
    wall) dam break: the block has collapsed and the surge runs along the
    floor."""
    out = {}
    for name, case, steps in (("dam2d_3000", C.dam_break_2d(cells_per_radius=1), 3000),
                              ("dam3d_450", C.dam_break_3d(12, tank=(0.8, 0.55, 0.55), cells_per_radius=1), 450)):
        res = orc.step(orc.params(case), case.r, case.v, case.kind, case.id, steps)
        assert res.rc == 0
        c = case.copy()
        c.r, c.v = res.r, res.v
        out[name] = c
        # the same state on cells of edge h
        ch = (C.dam_break_2d(cells_per_radius=2) if case.dim == 2
              else C.dam_break_3d(12, tank=(0.8, 0.55, 0.55), cells_per_radius=2))
        ch.r, ch.v = res.r.copy(), res.v.copy()
        out[name + "_h"] = ch
    return out


@pytest.mark.parametrize("name", ["dam2d_3000", "dam3d_450", "dam2d_3000_h", "dam3d_450_h"])
def test_step_c12_developed_dam_break(S, orc, developed, name):
    """One FP32 step from the oracle's developed dam-break state: rho, v and
    the displacement within 1e-5 (raw C12), p and a within 1e-5 carried
    through the EOS (C12b)."""
    _one_step_c12(S, orc, developed[name], name)


@pytest.mark.parametrize("name,case",
                         [("swirl2d", C.compressed_swirl(C.dam_break_2d(cells_per_radius=1))),
                          ("swirl3d", C.compressed_swirl(C.small_dam_break(3, 12, seed=34, cells_per_radius=1))),
                          ("swirl2d_h", C.compressed_swirl(C.dam_break_2d(cells_per_radius=2))),
                          ("swirl3d_h", C.compressed_swirl(C.small_dam_break(3, 12, seed=34, cells_per_radius=2)))],
                         ids=["swirl2d", "swirl3d", "swirl2d_h", "swirl3d_h"])
def test_step_c12_compressed_swirl(S, orc, name, case):
    _one_step_c12(S, orc, case, name)


@pytest.mark.parametrize("k", [1, 2])
def test_step_c12_full_size_compressed_swirl(S, orc, k):
    """The 3D workload at full size (1M fluid + 444k boundary particles, the
    launch configuration of the benchmark) compressed with depth and swirling:
    one FP32 step against one oracle step, every particle, raw C12."""
    _one_step_c12(S, orc, C.compressed_swirl(C.dam_break_3d(cells_per_radius=k)), f"swirl3d_full_k{k}")


# --- multi-step -----------------------------------------------------------------

def test_dam_break_2d_fp64_100_steps(S, orc):
    """The 2D FP64 workload (64x64 fluid, 100 steps) against the oracle."""
    case = C.dam_break_2d()
    sim = S.Simulation(case, precision=S.SPH_PREC_F64)
    d = sim.step(100, diag=True)
    r, v, rho, p, ids, kind = sim.state.to_host()
    res = orc.step(orc.params(case), case.r, case.v, case.kind, case.id, 100)
    k = _inv(case.id)[ids]
    e = dict(dr=rel(r - case.r[k], res.r[k] - case.r[k]), v=rel(v, res.v[k]), rho=rel(rho, res.rho[k]),
             p=rel(p, res.p[k]))
    report("dam2d_fp64_100", **e)
    assert e["dr"] < 1e-8 and e["v"] < 1e-8 and e["rho"] < 1e-10 and e["p"] < 1e-7
    assert d.n_pairs == res.n_pairs
    assert sim.status() == 0


def _fp32_rounded_positions(orc, case):
    """Initial positions moved by the FP32 rounding of their offsets in cells
    of edge 2h (the paper's cell size, ~1e-7 dx whatever cell size the case
    is searched with): the size of perturbation the FP32 form starts from."""
    P = orc.params(case)
    P.cs = 2.0 * case.h
    D = case.dim
    for k in range(D):
        P.ncell[k] = int(np.ceil(case.ncell[k] * case.cs / P.cs))
    cc, off, bad = orc.cell_coords(P, case.r)
    assert bad == 0
    base = np.array(case.dom_min[:D]) + cc[:, :D] * P.cs
    return base + off[:, :D].astype(np.float64)


def test_dam_break_2d_fp32_1000_steps(S, orc):
    """FP32 form over 1000 steps of the 2D dam break.  Displacements stay
    within 1e-3 of the FP64 oracle (spec bound).  Velocity, density and
    pressure are bounded by the flow's own sensitivity: the FP32 error may not
    exceed 3x the divergence of two FP64 oracle runs whose initial positions
    differ only by FP32 offset rounding (that divergence is ~1e-2 for v: the
    jitter-driven acoustic field amplifies any 1e-7 perturbation)."""
    case = C.dam_break_2d()
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    sim.step(1000)
    r, v, rho, p, ids, kind = sim.state.to_host()
    P = orc.params(case)
    res = orc.step(P, case.r, case.v, case.kind, case.id, 1000)
    pert = orc.step(P, _fp32_rounded_positions(orc, case), case.v, case.kind, case.id, 1000)
    k = _inv(case.id)[ids]
    e = dict(dr=rel(r - case.r[k], res.r[k] - case.r[k]), v=rel(v, res.v[k]), rho=rel(rho, res.rho[k]),
             p=rel(p, res.p[k]))
    sens = dict(dr=rel(pert.r - case.r, res.r - case.r), v=rel(pert.v, res.v), rho=rel(pert.rho, res.rho),
                p=rel(pert.p, res.p))
    report("dam2d_fp32_1000", **e, **{"fp64_sens_" + f: x for f, x in sens.items()})
    assert e["dr"] < 1e-3
    for f in ("v", "rho", "p"):
        assert e[f] <= 3.0 * sens[f] + 1e-6, (f, e[f], sens[f])


def test_dam_break_3d_fp32_1000_steps(S, orc):
    """The same 1000-step bound in 3D (12^3 fluid in a 0.8 x 0.55 x 0.55 m
    tank, 6117 particles): displacements within 1e-3 of the FP64 oracle,
    velocity, density and pressure within 3x the oracle's own sensitivity to
    the FP32 rounding of the initial offsets."""
    case = C.dam_break_3d(12, tank=(0.8, 0.55, 0.55))
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    sim.step(1000)
    r, v, rho, p, ids, kind = sim.state.to_host()
    assert sim.status() == 0
    P = orc.params(case)
    res = orc.step(P, case.r, case.v, case.kind, case.id, 1000)
    pert = orc.step(P, _fp32_rounded_positions(orc, case), case.v, case.kind, case.id, 1000)
    k = _inv(case.id)[ids]
    e = dict(dr=rel(r - case.r[k], res.r[k] - case.r[k]), v=rel(v, res.v[k]), rho=rel(rho, res.rho[k]),
             p=rel(p, res.p[k]))
    sens = dict(dr=rel(pert.r - case.r, res.r - case.r), v=rel(pert.v, res.v), rho=rel(pert.rho, res.rho),
                p=rel(pert.p, res.p))
    report("dam3d_fp32_1000", **e, **{"fp64_sens_" + f: x for f, x in sens.items()})
    assert e["dr"] < 1e-3
    for f in ("v", "rho", "p"):
        assert e[f] <= 3.0 * sens[f] + 1e-6, (f, e[f], sens[f])


# --- full size ----------------------------------------------------------------------

def test_dam_break_3d_full_size_forces(S, orc):
    """The 3D workload at full size (1M fluid + 444k boundary), FP32 form, in
    the launch configuration the benchmark times: every particle's density,
    pressure and acceleration against the oracle."""
    case = C.dam_break_3d()
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    a = sim.forces()
    r, v, rho, p, ids, kind = sim.state.to_host()
    a = np.stack([t.cpu().double().numpy() for t in a], axis=1)
    P = orc.params(case)
    k = _inv(case.id)[ids]
    ref, sens = oracle_sensitivities(orc, P, case)
    e = bounded_errors(case, EPS["f32"], {"rho": rho, "p": p, "a": a}, ref, sens, k, kind)
    report("dam3d_full_forces_f32", **e, raw_rho=rel(rho, ref["rho"][k]), raw_p=rel(p, ref["p"][k]),
           raw_a=rel(a, ref["a"][k]))
    for f in ("rho", "p", "a"):
        assert e[f] <= EPS["f32"], (f, e[f])
    # bit-exact cell table at full size
    order, start, _, _ = orc.sort_cells(P, case.r, case.id)
    assert np.array_equal(ids, case.id[order])
    assert np.array_equal(sim.cell_table(), start)


# --- edge cases -------------------------------------------------------------------------

def test_empty_and_single(S):
    case = C.random_cloud(2, 1, seed=3)
    case.r = np.array([[0.05, 0.05]])
    case.v = np.array([[0.1, 0.0]])
    case.kind = np.zeros(1, np.uint8)
    case.id = np.zeros(1, np.uint32)
    for prec in (S.SPH_PREC_F64, S.SPH_PREC_F32):
        sim = S.Simulation(case, precision=prec)
        d = sim.step(3, diag=True)
        r, v, *_ = sim.state.to_host()
        g = np.array(case.g[:2])
        dt = case.dt
        v_ex = case.v[0] + 3 * dt * g
        r_ex = case.r[0] + 3 * dt * case.v[0] + dt * dt * g * 6
        tol = 1e-14 if prec == S.SPH_PREC_F64 else 1e-6
        assert np.allclose(v[0], v_ex, rtol=tol, atol=tol)
        assert np.allclose(r[0], r_ex, rtol=1e-12, atol=1e-12)
        assert d.n_pairs == 0
        # n = 0 is a no-op
        st = sim.state.view()
        st.n = 0
        S.sph_step(sim.ctx, st, 2)
        assert sim.status() == 0


def test_status_out_of_domain_and_nan(S):
    case = C.random_cloud(2, 200, seed=4)
    case.r[5, 0] = case.dom_min[0] - 1.0
    sim = S.Simulation(case)
    sim.step(1)
    assert sim.status() & S.SPH_STATUS_OUT_OF_DOMAIN
    assert sim.status() == 0  # cleared by the read
    case2 = C.random_cloud(2, 200, seed=4)
    case2.v[7, 1] = np.nan
    sim2 = S.Simulation(case2)
    sim2.step(1)
    assert sim2.status() & S.SPH_STATUS_NAN
    case3 = C.random_cloud(2, 200, seed=4)
    case3.r[10] = case3.r[11]          # same cell, same id
    case3.id[10] = case3.id[11]
    sim3 = S.Simulation(case3)
    sim3.build_cells()
    assert sim3.status() & S.SPH_STATUS_DUPLICATE_ID


def test_crowded_cell_at_and_over_the_cell_limit(S):
    """A cell holding SPH_MAX_CELL particles is still ordered canonically
    (by id) and steps without status; one particle more sets
    SPH_STATUS_CELL_OVERFLOW (the cell keeps its arrival order, every access
    stays in bounds) and the context stays usable."""
    for n, over in ((S.SPH_MAX_CELL, False), (S.SPH_MAX_CELL + 1, True)):
        case = C.random_cloud(2, n, seed=6, box=0.02)   # box < cs: one cell
        # (~400 times the rest density: a slow sound speed and a short step
        # keep the pressure forces and the motion finite)
        case.c0, case.dt = 1e-6, 1e-6
        sim = S.Simulation(case, precision=S.SPH_PREC_F32)
        sim.build_cells()
        st = sim.status()
        ids = sim.state.id.cpu().numpy().astype(np.int64)
        if over:
            assert st & S.SPH_STATUS_CELL_OVERFLOW
            assert np.array_equal(np.sort(ids), np.sort(case.id.astype(np.int64)))
        else:
            assert st == 0
            assert np.array_equal(ids, np.sort(case.id.astype(np.int64)))
        d = sim.step(1, diag=True)
        st = sim.status()
        assert bool(st & S.SPH_STATUS_CELL_OVERFLOW) == over
        assert st & ~(S.SPH_STATUS_CELL_OVERFLOW | S.SPH_STATUS_CFL) == 0
        assert d.n_pairs > 0
        r = sim.state.to_host()[0]
        assert np.isfinite(r).all()
        sim.close()


def test_capacity_error(S):
    case = C.random_cloud(2, 100, seed=5)
    sim = S.Simulation(case, capacity=100)
    st = sim.state.view()
    st.n = 101
    with pytest.raises(S.SphError) as e:
        S.sph_step(sim.ctx, st, 1)
    assert "(-3)" in str(e.value)


def test_dam_break_3d_large_sampled(S, orc):
    """The large 3D workload (256^3 fluid + 2.73 M boundary = 19.5 M
    particles) in the FP32 form at full size: densities, pressures and
    accelerations of 4000 sampled particles against the oracle evaluated at
    those particles (and their neighbours), with the first-order bounds of
    the small cases; the cell table bit for bit."""
    case = C.dam_break_3d_large()
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    a = sim.forces()
    r, v, rho, p, ids, kind = sim.state.to_host()
    a = np.stack([t.cpu().double().numpy() for t in a], axis=1)
    assert sim.status() == 0
    rng = np.random.default_rng(17)
    pick = np.concatenate([rng.choice(np.nonzero(kind == 0)[0], 3000, replace=False),
                           rng.choice(np.nonzero(kind == 1)[0], 1000, replace=False)])
    idx = _inv(case.id)[ids[pick]]
    P = orc.params(case)
    ors, ops, oas, A, G = orc.sampled_forces(P, case.r, case.v, case.kind, case.id, idx)
    B = case.c0 ** 2 * case.rho0 / case.gamma
    fl = kind[pick] == 0
    e = dict(rho=float((np.abs(rho[pick] - ors) / ors).max()),
             p=float((np.abs(p[pick] - ops) / (case.gamma * (np.abs(ops) + B))).max()),
             a=float((np.linalg.norm(a[pick][fl] - oas[fl], axis=1) / (A[fl] + G[fl])).max()))
    report("dam3d_large_sampled_f32", **e, raw_rho=rel(rho[pick], ors), raw_a=rel(a[pick][fl], oas[fl]))
    for f in ("rho", "p", "a"):
        assert e[f] <= 1e-5, (f, e[f])
    order, start, _, _ = orc.sort_cells(P, case.r, case.id)
    assert np.array_equal(ids, case.id[order])
    assert np.array_equal(sim.cell_table(), start)


@pytest.mark.parametrize("prec", PRECS)
def test_multi_step_graph_equals_single_steps(S, prec):
    """sph_step with nsteps >= 2 replays a recorded CUDA graph of one step;
    it must give the state that nsteps single-step calls give, bit for bit,
    also after the context records again for another state."""
    P = _prec(S, prec)
    for k in (1, 2):
        case = C.small_dam_break(2, 20, seed=81, cells_per_radius=k)
        case.v[: case.n_fluid] = np.random.default_rng(4).normal(0.0, 0.05, size=(case.n_fluid, 2))
        a = S.Simulation(case, precision=P)
        b = S.Simulation(case, precision=P)
        da = a.step(25, diag=True)                 # graph replay
        for _ in range(25):
            db = b.step(1, diag=True)              # one launch sequence per call
        for x, y in zip(a.state.to_host(), b.state.to_host()):
            assert np.array_equal(x, y)
        assert da.n_pairs == db.n_pairs and da.vmax == db.vmax
        # a second state on the same context: recorded again
        other = S.device_state(case.r, case.v, case.kind, case.id, P)
        view = other.view()
        S.sph_step(a.ctx, view, 10)
        for _ in range(10):
            b.step(1)
        ref = S.Simulation(case, precision=P)
        for _ in range(10):
            ref.step(1)
        for x, y in zip(other.to_host(), ref.state.to_host()):
            assert np.array_equal(x, y)
        assert a.status() == 0
        for sim in (a, b, ref):
            sim.close()

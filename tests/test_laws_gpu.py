"""GPU parity of compiled interaction laws (paper_1710_08259_gb300/laws.py)
against the CPU evaluators: the C Example 1a oracle for the equations of
Appendix A, the numpy law oracle (oracle/laws_oracle.py) for the other
systems, and the hand-written Example 1a kernels of the library.

FP64 runs are held to 1e-9 of the field's scale; FP32 runs to the
first-order per-step bounds of test_model_gpu.py for one step, and over
several steps to 1e-4 of the motion (well above FP32 rounding, far below any
wrong term)."""
import math

import numpy as np
import pytest

from paper_1710_08259_gb300 import cases as C

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SYM, PER, CUT = C.BC_SYMMETRIC, C.BC_PERIODIC, C.BC_CUTOFF

APPENDIX_A = ["rhodot = -rho*sph_D(v, mass, rho)",
              "rho = euler(rho, rhodot, dt)",
              "p = c**2*(rho - rho0)",
              "vdot = -1/rho*sph_G(p, mass, rho)",
              "vdot = vdot + 0.1*c*h*sph_A(v, mass, rho) + g",
              "v = euler(v, vdot, dt)",
              "r = euler(r, v, dt)"]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08259_gb300 import build as B
    B.build()
    from paper_1710_08259_gb300 import sph
    return sph


@pytest.fixture(scope="module")
def L(S):
    from paper_1710_08259_gb300 import laws
    return laws


def _prec(S, name):
    return S.SPH_PREC_F64 if name == "f64" else S.SPH_PREC_F32


def _inv(ids):
    inv = np.empty(int(ids.max()) + 1, np.int64)
    inv[ids] = np.arange(ids.size)
    return inv


def _appendix_a(case):
    n = case.n
    fields = {"rho": ("scalar", case.rho), "rhodot": ("scalar", np.zeros(n)), "p": ("scalar", np.zeros(n)),
              "v": ("vector", case.v), "vdot": ("vector", np.zeros((n, case.dim)))}
    consts = {"mass": case.mass, "c": case.c0, "rho0": case.rho0, "dt": case.dt, "g": tuple(case.g[:case.dim])}
    return fields, consts


def _box():
    c = C.paper_box(2, (24, 16), (11, 9), (SYM, SYM), seed=301, v_sigma=0.4, rho_sigma=0.004, jitter=0.08)
    c.alpha = 0.1
    return c


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_appendix_a_compiled_one_step(S, L, orc, prec):
    case = _box()
    fields, consts = _appendix_a(case)
    sysm = L.LawSystem(case, fields, consts, APPENDIX_A, precision=_prec(S, prec))
    sysm.step(1)
    r, f, ids = sysm.host()
    k = _inv(case.id)[ids]
    P = orc.bc_params(case, fp32=(prec == "f32"))
    res = orc.bc_step(P, case.r, case.v, case.rho, case.kind, case.id, 1)
    ev = orc.bc_eval(P, case.r, case.v, case.rho, case.kind, case.id)
    eps = 1e-12 if prec == "f64" else 1e-5
    rb = eps * (np.abs(ev.rho[k]) + ev.drho_abs[k])
    ab = eps * (ev.aabs[k] + ev.asens[k] * (1.0 + ev.drho_abs[k] / np.abs(ev.rho[k])))
    bv = eps * np.linalg.norm(case.v[k], axis=1) + case.dt * ab
    e = dict(rho=float((np.abs(f["rho"] - res.rho[k]) / rb).max()) * eps,
             p=float((np.abs(f["p"] - res.p[k]) / (case.c0 ** 2 * rb)).max()) * eps,
             v=float((np.linalg.norm(f["v"] - res.v[k], axis=1) / bv).max()) * eps,
             dr=float((np.linalg.norm((r - case.r[k]) - (res.r[k] - case.r[k]), axis=1) /
                       (case.dt * bv)).max()) * eps)
    print(f"laws_appendix_a[{prec}]", e)
    for name, x in e.items():
        assert x <= eps, (name, x)
    sysm.close()


def test_appendix_a_compiled_200_steps_fp64(S, L, orc):
    case = C.example_1a(1)
    fields, consts = _appendix_a(case)
    sysm = L.LawSystem(case, fields, consts, APPENDIX_A, precision=S.SPH_PREC_F64)
    sysm.step(200)
    r, f, ids = sysm.host()
    res = orc.bc_step(orc.bc_params(case), case.r, case.v, case.rho, case.kind, case.id, 200)
    assert res.rc == 0
    k = _inv(case.id)[ids]
    err = float(np.abs((r - case.r[k]) - (res.r[k] - case.r[k])).max() / np.abs(res.r - case.r).max())
    errv = float(np.abs(f["v"] - res.v[k]).max() / np.abs(res.v).max())
    print("laws_appendix_a_fp64_200", err, errv, "builds", sysm.builds)
    assert err < 1e-9 and errv < 1e-9
    assert sysm.builds == 200           # the first at construction, then one after each move
    sysm.close()


def test_compiled_equals_hand_written_example_1a(S, L):
    """The equations of Appendix A compiled, against the library's own
    Example 1a kernels, both FP32, 50 steps of the refined case."""
    case = C.example_1a(2)
    fields, consts = _appendix_a(case)
    sysm = L.LawSystem(case, fields, consts, APPENDIX_A, precision=S.SPH_PREC_F32)
    sysm.step(50)
    r, f, ids = sysm.host()
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    sim.step(50)
    r2, v2, rho2, p2, ids2, _ = sim.state.to_host()
    k = _inv(ids)[ids2]
    motion = np.abs(r2 - case.r[_inv(case.id)[ids2]]).max()
    e_r = float(np.abs(r[k] - r2).max() / motion)
    e_v = float(np.abs(f["v"][k] - v2).max() / np.abs(v2).max())
    print("laws_vs_hand_written", e_r, e_v)
    assert e_r < 1e-4 and e_v < 1e-4
    sysm.close()
    sim.close()


CAHN_HILLIARD = ["mu = c**3 - c - gam*sph_L(c, m, rho0)",
                 "cdot = Dm*sph_L(mu, m, rho0)",
                 "c = euler(c, cdot, dt)"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cahn_hilliard_on_a_periodic_sheet(S, L, prec):
    """Example 1b's model (Eq. cahnhilliard with the sph_L operator) on a
    flat periodic sheet of particles at rest."""
    from oracle import laws_oracle as LO
    case = C.paper_box(2, (40, 40), (18, 18), (PER, PER), seed=7, dx=0.01, cs_factor=40 * 0.01 / 18 / 0.022)
    rng = np.random.default_rng(3)
    c0 = 0.1 * rng.uniform(-1, 1, case.n)
    fields = {"c": ("scalar", c0), "mu": ("scalar", np.zeros(case.n)), "cdot": ("scalar", np.zeros(case.n))}
    consts = {"gam": 1e-4, "Dm": 1e-3, "m": case.mass, "rho0": case.rho0, "dt": 1e-2}
    sysm = L.LawSystem(case, fields, consts, CAHN_HILLIARD, precision=_prec(S, prec))
    sysm.step(20)
    _, f, ids = sysm.host()
    lo = LO.LawOracle(case, fields, consts, CAHN_HILLIARD, fp32_neighbours=(prec == "f32"))
    lo.step(20)
    k = _inv(case.id)[ids]
    ref = lo.fields["c"].a[k]
    err = float(np.abs(f["c"] - ref).max() / np.abs(ref - c0[k]).max())
    print(f"cahn_hilliard[{prec}]", err, "change", np.abs(ref - c0[k]).max())
    assert err < (1e-9 if prec == "f64" else 1e-4)
    assert sysm.builds == 1             # nothing moves: one build only
    sysm.close()


SOCIAL_FORCE = ["vdot = (v0*e0 - v)/tau + sum_j((A*exp((R_i + R_j - d_ij)/B) + k*max(R_i + R_j - d_ij, 0)"
                " - cA)*r_ij/d_ij)/m",
                "v = euler(v, vdot, dt)",
                "r = euler(r, v, dt)"]


def _crowd(seed=12, n=120):
    """A periodic corridor (x periodic, walls y symmetric) with people of
    radius R = 0.002 m + 0.15 (the law of Section 6, m ~ U[50, 100] kg)
    heading along +x."""
    rng = np.random.default_rng(seed)
    h = 0.6
    cs = 2 * h
    nc = (12, 5)
    Lx, Ly = nc[0] * cs, nc[1] * cs
    c = C.paper_box(2, (1, 1), nc, (PER, SYM), seed=seed, dx=h / 1.1)
    side = int(math.ceil(math.sqrt(n * Lx / Ly)))
    gx = (np.arange(n) % side + 0.5) * (Lx / side)
    gy = (np.arange(n) // side + 0.5) * (Ly / math.ceil(n / side))
    c.r = np.stack([gx + rng.uniform(-0.05, 0.05, n), gy + rng.uniform(-0.05, 0.05, n)], axis=1)
    c.r[:, 1] = np.clip(c.r[:, 1], 0.01, Ly - 0.01)
    m = rng.uniform(50.0, 100.0, n)
    R = 0.002 * m + 0.15
    ang = rng.normal(0.0, 0.2, n)
    e0 = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    v = 0.3 * e0
    c.v = v
    c.kind = np.zeros(n, np.uint8)
    c.id = rng.permutation(n).astype(np.uint32)
    c.n_fluid = n
    fields = {"v": ("vector", v), "vdot": ("vector", np.zeros((n, 2))), "e0": ("vector", e0),
              "R": ("scalar", R), "m": ("scalar", m)}
    consts = {"v0": 1.3, "tau": 0.5, "A": 2000.0, "B": 0.08, "k": 1.2e5, "cA": 0.0, "dt": 0.005}
    return c, fields, consts


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_social_force_crowd(S, L, prec):
    """The social force model of Section 6 (Eq. social_force_model) written
    as a user-defined pair law with sum_j."""
    from oracle import laws_oracle as LO
    case, fields, consts = _crowd()
    sysm = L.LawSystem(case, fields, consts, SOCIAL_FORCE, precision=_prec(S, prec))
    sysm.step(40)
    r, f, ids = sysm.host()
    lo = LO.LawOracle(case, fields, consts, SOCIAL_FORCE, fp32_neighbours=(prec == "f32"))
    lo.step(40)
    k = _inv(case.id)[ids]
    Lx = case.ncell[0] * case.cs
    d = r - lo.r[k]
    d[:, 0] -= Lx * np.round(d[:, 0] / Lx)
    motion = np.abs(f["v"]).max() * 40 * consts["dt"]
    err = float(np.abs(d).max() / motion)
    errv = float(np.abs(f["v"] - lo.fields["v"].a[k, :2]).max() / np.abs(lo.fields["v"].a).max())
    print(f"social_force[{prec}]", err, errv)
    assert err < (1e-9 if prec == "f64" else 1e-4)
    assert errv < (1e-9 if prec == "f64" else 1e-4)
    assert np.mean(f["v"][:, 0]) > 0.5          # the crowd walks along +x
    sysm.close()


def test_law_errors(S, L):
    case = _box()
    fields, consts = _appendix_a(case)
    for bad in (["rho = rho + q"],                      # unknown name
                ["rho = v"],                            # a vector into a scalar
                ["v = sum_j(rho)"],                     # bare field inside sum_j
                ["rho = sph_D(rho, mass, rho)"],        # sph_D of a scalar is a vector
                ["r = r + v"]):                         # positions move by euler only
        with pytest.raises(L.LawError):
            L.LawSystem(case, fields, consts, bad, precision=S.SPH_PREC_F32)


@pytest.mark.parametrize("eb", [4, 8, 12])
def test_reorder_fields_follow_the_build(S, eb):
    """sph_reorder_field / sph_reorder_fields gather caller fields into the
    order of the last build (out[k] = in[src[k]], src = the slot each
    particle came from), one field or several per call; overlapping outputs
    are rejected before any launch."""
    case = C.paper_box(2, (30, 20), (12, 10), (PER, SYM), seed=41, jitter=0.2, shuffle_ids=True)
    p = S.params_from_case(case, precision=S.SPH_PREC_F32)
    p.model = S.SPH_MODEL_FIELDS
    ctx = S.sph_create(p, case.n)
    st = S.device_state(case.r, np.zeros((case.n, 2)), case.kind, case.id, S.SPH_PREC_F32)
    ids0 = st.id.cpu().numpy().astype(np.int64)
    view = st.view()
    for k in range(3):
        view.v[k] = None                       # the field model keeps no velocity
    S.sph_build_cells(ctx, view)
    ids1 = st.id.cpu().numpy().astype(np.int64)
    inv0 = np.empty(ids0.max() + 1, np.int64)
    inv0[ids0] = np.arange(case.n)
    src = inv0[ids1]
    assert not np.array_equal(src, np.arange(case.n))   # the build did move particles
    w = eb // 4
    rng = np.random.default_rng(5)
    fields = [torch.tensor(rng.integers(0, 2 ** 31, (case.n, w)), dtype=torch.int32, device="cuda")
              for _ in range(11)]                  # more than one launch's worth (8)
    outs = [torch.empty_like(f) for f in fields]
    S.sph_reorder_fields(ctx, [f.data_ptr() for f in fields], [o.data_ptr() for o in outs], eb)
    one = torch.empty_like(fields[0])
    S.sph_reorder_field(ctx, fields[0].data_ptr(), one.data_ptr(), eb)
    torch.cuda.synchronize()
    for f, o in zip(fields, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), f.cpu().numpy()[src])
    np.testing.assert_array_equal(one.cpu().numpy(), outs[0].cpu().numpy())
    with pytest.raises(S.SphError):
        S.sph_reorder_fields(ctx, [fields[0].data_ptr(), fields[1].data_ptr()],
                             [outs[0].data_ptr(), outs[0].data_ptr()], eb)    # two outputs overlap
    with pytest.raises(S.SphError):
        S.sph_reorder_fields(ctx, [fields[0].data_ptr()], [fields[0].data_ptr()], eb)  # in place
    S.sph_reorder_fields(ctx, [], [], eb)            # nothing to do
    S.sph_destroy(ctx)


@pytest.mark.parametrize("eb", [4, 8])
def test_build_into_equals_build_then_reorder(S, eb):
    """sph_build_cells_into (the build writing a second state and reordering
    the fields in its gather) gives, bit for bit, the state and fields of
    sph_build_cells followed by sph_reorder_fields, and leaves its input
    state unchanged; more fields than one gather carries go through the
    permutation; overlaps and other models are rejected."""
    case = C.paper_box(2, (30, 20), (12, 10), (PER, SYM), seed=43, jitter=0.2, shuffle_ids=True)
    p = S.params_from_case(case, precision=S.SPH_PREC_F32)
    p.model = S.SPH_MODEL_FIELDS
    rng = np.random.default_rng(6)
    w = eb // 4
    fields = [torch.tensor(rng.integers(0, 2 ** 31, (case.n, w)), dtype=torch.int32, device="cuda")
              for _ in range(11)]

    def state():
        st = S.device_state(case.r, np.zeros((case.n, 2)), case.kind, case.id, S.SPH_PREC_F32)
        v = st.view()
        for k in range(3):
            v.v[k] = None
        return st, v

    ctx = S.sph_create(p, case.n)
    a, av = state()
    S.sph_build_cells(ctx, av)
    ref = [torch.empty_like(f) for f in fields]
    S.sph_reorder_fields(ctx, [f.data_ptr() for f in fields], [o.data_ptr() for o in ref], eb)
    S.sph_destroy(ctx)

    ctx = S.sph_create(p, case.n)
    b_in, biv = state()
    b_out, bov = state()
    got = [torch.empty_like(f) for f in fields]
    S.sph_build_cells_into(ctx, biv, bov, [f.data_ptr() for f in fields], [o.data_ptr() for o in got], eb)
    torch.cuda.synchronize()
    for x, y in zip(a.r + [a.id, a.kind], b_out.r + [b_out.id, b_out.kind]):
        assert torch.equal(x, y)
    for x, y in zip(ref, got):
        assert torch.equal(x, y)
    np.testing.assert_array_equal(b_in.id.cpu().numpy().astype(np.uint32), case.id)   # input untouched
    # the cells now belong to the output: a reorder follows its order
    one = torch.empty_like(fields[0])
    S.sph_reorder_field(ctx, fields[0].data_ptr(), one.data_ptr(), eb)
    assert torch.equal(one, got[0])
    with pytest.raises(S.SphError):                    # output state = input state
        S.sph_build_cells_into(ctx, biv, biv, [], [], eb)
    with pytest.raises(S.SphError):                    # a field output over an input
        S.sph_build_cells_into(ctx, biv, bov, [fields[0].data_ptr()], [fields[0].data_ptr()], eb)
    S.sph_destroy(ctx)
    q = S.params_from_case(case, precision=S.SPH_PREC_F32)
    q.model = S.SPH_MODEL_EXAMPLE_1A
    ctx = S.sph_create(q, case.n)
    c_in, civ = state()
    c_out, cov = state()
    with pytest.raises(S.SphError):
        S.sph_build_cells_into(ctx, civ, cov, [], [], eb)
    S.sph_destroy(ctx)


ADAPTIVE_CH = ["mu = c**3 - c - gam*sph_L(c, m, rho0)",
               "cdot = Dm*sph_L(mu, m, rho0)",
               "dt = 0.1*min(1/fmax(abs(cdot)), dtg)",
               "c = euler(c, cdot, dt)",
               "Time = Time + dt",
               "cmean = fsum(c)/np_",
               "cmin = fmin(c)"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cahn_hilliard_adaptive_time_step(S, L, prec):
    """Variables on the GPU: Example 1b's model with an adaptive time step
    dt = 0.1 min(1/max|c'|, dt_g) and an elapsed time (global variables,
    each a reduction kernel pair), plus a mean and a minimum, against the
    law oracle."""
    from oracle import laws_oracle as LO
    case = C.paper_box(2, (40, 40), (18, 18), (PER, PER), seed=7, dx=0.01, cs_factor=40 * 0.01 / 18 / 0.022)
    rng = np.random.default_rng(5)
    c0 = 0.1 * rng.uniform(-1, 1, case.n)
    fields = {"c": ("scalar", c0), "mu": ("scalar", np.zeros(case.n)), "cdot": ("scalar", np.zeros(case.n))}
    consts = {"gam": 1e-4, "Dm": 1e-3, "m": case.mass, "rho0": case.rho0, "dtg": 0.05, "np_": float(case.n)}
    vs = {"dt": 0.0, "Time": 0.0, "cmean": 0.0, "cmin": 0.0}
    sysm = L.LawSystem(case, fields, consts, ADAPTIVE_CH, precision=_prec(S, prec), variables=vs)
    sysm.step(20)
    _, f, ids = sysm.host()
    got = sysm.variables()
    lo = LO.LawOracle(case, fields, consts, ADAPTIVE_CH, fp32_neighbours=(prec == "f32"), variables=vs)
    lo.step(20)
    k = _inv(case.id)[ids]
    ref = lo.fields["c"].a[k]
    tol = 1e-9 if prec == "f64" else 1e-4
    err = float(np.abs(f["c"] - ref).max() / np.abs(ref - c0[k]).max())
    rel = {v: abs(got[v] - lo.vars[v]) / abs(lo.vars[v]) for v in vs}
    print(f"cahn_hilliard_adaptive[{prec}]", err, rel, lo.vars)
    assert err < tol
    for v in vs:
        assert rel[v] < tol, (v, got[v], lo.vars[v])
    assert lo.vars["dt"] < consts["dtg"]          # the adaptive bound is the active one
    sysm.close()


GOAL_SEEKING = ["vdot = (v0*(goal - r)/norm(goal - r) - v)/tau + sum_j((A*exp((R_i + R_j - d_ij)/B)"
                " + k*max(R_i + R_j - d_ij, 0) - cA)*r_ij/d_ij)/m",
                "v = euler(v, vdot, dt)",
                "r = euler(r, v, dt)"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_goal_seeking_crowd(S, L, prec):
    """The social force law with the desired direction toward a goal point
    (the paper's people head for exits): the law reads each person's own
    position r; against the law oracle."""
    from oracle import laws_oracle as LO
    case, fields, consts = _crowd(seed=21, n=100)
    consts = dict(consts, goal=(4.0, 1.5))
    fields = {k: v for k, v in fields.items() if k != "e0"}
    sysm = L.LawSystem(case, fields, consts, GOAL_SEEKING, precision=_prec(S, prec))
    sysm.step(40)
    r, f, ids = sysm.host()
    lo = LO.LawOracle(case, fields, consts, GOAL_SEEKING, fp32_neighbours=(prec == "f32"))
    lo.step(40)
    k = _inv(case.id)[ids]
    Lx = case.ncell[0] * case.cs
    d = r - lo.r[k]
    d[:, 0] -= Lx * np.round(d[:, 0] / Lx)
    motion = np.abs(f["v"]).max() * 40 * consts["dt"]
    err = float(np.abs(d).max() / motion)
    errv = float(np.abs(f["v"] - lo.fields["v"].a[k, :2]).max() / np.abs(lo.fields["v"].a).max())
    print(f"goal_seeking[{prec}]", err, errv)
    assert err < (1e-9 if prec == "f64" else 1e-4)
    assert errv < (1e-9 if prec == "f64" else 1e-4)
    sysm.close()


WCSPH_LAWS = ["rho = sph_S(1, m, 1)",
              "p = max(B*((rho/rho_ref)**7 - 1), 0)",
              "vdot = where(fl, g - sum_j(m*(p_i/rho_i**2 + p_j/rho_j**2"
              " - alpha*c0*h*min(dot(v_i - v_j, r_ij), 0)/(0.5*(rho_i + rho_j)*(d_ij**2 + eps*h**2)))*gradW_ij),"
              " 0*g)",
              "v = euler(v, vdot, dt)",
              "r = euler(r, v, dt)"]


def wcsph_law_system(S, case, precision):
    """The step of the hot path (summation density with the self term, Tait
    EOS against the lattice reference density with the p >= 0 clamp, the
    pressure gradient with the symmetric viscosity, semi-implicit Euler of
    the fluid particles only) written as equations."""
    probe = S.Simulation(case, precision=precision)
    rho_ref = S.sph_rho_ref(probe.ctx)
    probe.close()
    n = case.n
    fields = {"rho": ("scalar", np.full(n, case.rho0)), "p": ("scalar", np.zeros(n)),
              "v": ("vector", case.v), "vdot": ("vector", np.zeros((n, case.dim))),
              "fl": ("scalar", (case.kind == 0).astype(np.float64))}
    consts = {"m": case.mass, "c0": case.c0, "alpha": case.alpha, "eps": case.visc_eps, "dt": case.dt,
              "B": case.c0 ** 2 * case.rho0 / case.gamma, "rho_ref": rho_ref, "g": tuple(case.g[:case.dim])}
    return fields, consts


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_compiled_wcsph_equals_the_hand_written_step(S, L, prec, k):
    """The hot path's own model compiled from equations against sph_step
    (2D dam break with boundary particles, 30 steps).  FP64 to rounding.
    FP32: positions, velocities and densities to 2e-4; the pressure to 2e-3,
    because the compiled (rho/rho_ref)^7 - 1 cancels near rest, where the
    hand-written step evaluates d * poly(d), d = rho/rho_ref - 1 ~ 1e-3, and
    sums the density with Kahan compensation: a density rounding of 4e-7
    becomes ~ 4e-7 / d in the pressure.  k: cells per support radius (2:
    cells of edge h, the compiled kernels walk the rows as sph_step does)."""
    case = C.small_dam_break(2, 24, cells_per_radius=k)
    P = _prec(S, prec)
    fields, consts = wcsph_law_system(S, case, P)
    sysm = L.LawSystem(case, fields, consts, WCSPH_LAWS, precision=P)
    sysm.step(30)
    r, f, ids = sysm.host()
    sim = S.Simulation(case, precision=P)
    sim.step(30)
    r2, v2, rho2, p2, ids2, _ = sim.state.to_host()
    k = _inv(ids)[ids2]
    motion = np.abs(r2 - case.r[_inv(case.id)[ids2]]).max()
    e = dict(r=float(np.abs(r[k] - r2).max() / motion), v=float(np.abs(f["v"][k] - v2).max() / np.abs(v2).max()),
             rho=float(np.abs(f["rho"][k] - rho2).max() / np.abs(rho2).max()),
             p=float(np.abs(f["p"][k] - p2).max() / np.abs(p2).max()))
    print(f"compiled_wcsph[{prec}-k{k}]", e)
    for name, x in e.items():
        tol = 1e-9 if prec == "f64" else (2e-3 if name == "p" else 2e-4)
        assert x < tol, (name, x)
    sysm.close()
    sim.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_compiled_sampling_equals_sph_sample_3d(S, L, prec):
    """3D and periodic on every face: the sampling operator compiled from
    "Sv = sph_S(A, m, rho)" against the library's sph_sample (Section 6)."""
    case = C.periodic_cube(15, seed=71, rho_sigma=0.01, jitter=0.05)
    n = case.n
    fields = {"A": ("scalar", case.extra["A"]), "m": ("scalar", case.extra["m"]), "rho": ("scalar", case.rho),
              "Sv": ("scalar", np.zeros(n))}
    P = _prec(S, prec)
    sysm = L.LawSystem(case, fields, {}, ["Sv = sph_S(A, m, rho)"], precision=P)
    sysm.step(1)
    _, f, ids = sysm.host()
    sim = S.Simulation(case, precision=P)
    sim.build_cells()
    _, _, _, _, ids2, _ = sim.state.to_host()
    k = _inv(case.id)[ids2]
    tdt = torch.float32 if prec == "f32" else torch.float64
    t = lambda a: torch.tensor(a[k], dtype=tdt, device="cuda")
    Sg = sim.sample(t(case.extra["A"]), t(case.extra["m"]), t(case.rho)).cpu().double().numpy()
    kk = _inv(ids)[ids2]
    e = float(np.abs(f["Sv"][kk] - Sg).max() / np.abs(Sg).max())
    print(f"compiled_sample_3d[{prec}]", e)
    assert e < (1e-13 if prec == "f64" else 1e-6)
    sysm.close()
    sim.close()


@pytest.mark.parametrize("k", [1, 2])
def test_compiled_wcsph_3d_fp64(S, L, k):
    """The compiled WCSPH model in 3D (boundary particles, cut-off faces)
    against sph_step, FP64, 20 steps, on cells of edge 2h / k."""
    case = C.dam_break_3d(10, tank=(0.7, 0.5, 0.5), cells_per_radius=k)
    fields, consts = wcsph_law_system(S, case, S.SPH_PREC_F64)
    sysm = L.LawSystem(case, fields, consts, WCSPH_LAWS, precision=S.SPH_PREC_F64)
    sysm.step(20)
    r, f, ids = sysm.host()
    sim = S.Simulation(case, precision=S.SPH_PREC_F64)
    sim.step(20)
    r2, v2, rho2, p2, ids2, _ = sim.state.to_host()
    k = _inv(ids)[ids2]
    motion = np.abs(r2 - case.r[_inv(case.id)[ids2]]).max()
    e = dict(r=float(np.abs(r[k] - r2).max() / motion), v=float(np.abs(f["v"][k] - v2).max() / np.abs(v2).max()),
             rho=float(np.abs(f["rho"][k] - rho2).max() / np.abs(rho2).max()))
    print(f"compiled_wcsph_3d_f64[k{k}]", e)
    for name, x in e.items():
        assert x < 1e-9, (name, x)
    sysm.close()
    sim.close()


# The Hertz contact law of Example 2 (Eq. DEM_force with the effective
# quantities; friction only while sliding) written with sum_j; the tank's
# wall are the symmetric faces, seen as mirror images
_DL = "(R_i + R_j - d_ij)"
_VN = "(dot(v_i - v_j, r_ij)/d_ij)"
_KH = "(4/3*sqrt(R_i*R_j/(R_i + R_j))*Ep)"
_CH = f"(sqrt(m_i*m_j/(m_i + m_j)*{_KH})/8)"
_FN = f"({_KH}*{_DL}**1.5 - {_CH}*sqrt(sqrt({_DL}))*{_VN})"
_VT = f"((v_j - v_i) + {_VN}*r_ij/d_ij)"
_FT = f"where(max(dot({_VT}, {_VT}) - 1e-10*dot(v_i - v_j, v_i - v_j), 0), cf*abs({_FN})/norm({_VT}), 0)"
DEM_LAWS = [f"a = g + sum_j(where(max({_DL}, 0), {_FN}*r_ij/d_ij + {_FT}*{_VT}, 0*r_ij))/m",
            "v = euler(v, a, dt)",
            "r = euler(r, v, dt)"]


def test_compiled_dem_law_equals_the_hand_written_kernel(S, L):
    """Example 2's contact law compiled from one equation against the
    library's DEM kernel (the tank held fixed: its coupling needs the wall
    force summed over image pairs only), FP64, 5 steps of a packed damper."""
    case = C.dem_damper(7, 7, 6, spacing=0.0079, seed=5, v_sigma=0.2)
    n = case.n
    fields = {"v": ("vector", case.v), "a": ("vector", np.zeros((n, 3))), "R": ("scalar", case.rho),
              "m": ("scalar", case.extra["m"])}
    nu, E = case.extra["nu"], case.extra["E"]
    consts = {"Ep": E / (2.0 * (1.0 - nu * nu)), "cf": case.extra["cf"], "g": tuple(case.g), "dt": case.dt}
    sysm = L.LawSystem(case, fields, consts, DEM_LAWS, precision=S.SPH_PREC_F64)
    sysm.step(5)
    r, f, ids = sysm.host()
    sim = S.Simulation(case, precision=S.SPH_PREC_F64, tank=False)
    sim.step(5)
    r2, v2, _, _, ids2, _ = sim.state.to_host()
    k = _inv(ids)[ids2]
    motion = np.abs(r2 - case.r[_inv(case.id)[ids2]]).max()
    e = dict(r=float(np.abs(r[k] - r2).max() / motion), v=float(np.abs(f["v"][k] - v2).max() / np.abs(v2).max()))
    print("compiled_dem", e)
    for name, x in e.items():
        assert x < 1e-9, (name, x)
    sysm.close()
    sim.close()


_FORCE = f"({_FN}*r_ij/d_ij + {_FT}*{_VT})"
EXAMPLE_2_LAWS = [f"F = sum_j(where(max({_DL}, 0), {_FORCE}, 0*r_ij))",
                  f"fwz = sum_j(where(max({_DL}, 0)*mirror_ij, dot({_FORCE}, vec(0, 0, 1)), 0))",
                  "Fb = fsum(fwz)",
                  "Zdd = (-S*Z - Fb)/M",
                  "v = euler(v, F/m + g - Zdd*vec(0, 0, 1), dt)",
                  "r = euler(r, v, dt)",
                  "Zd = Zd + dt*Zdd",
                  "Z = Z + dt*Zd"]


def test_compiled_example_2_with_the_tank(S, L):
    """Example 2 entirely as equations, as the paper sets it up (the contact
    law as a pair law, the tank's state as variables): the wall force is the
    sum over particles of their contact forces with wall images
    (mirror_ij), the tank oscillator M Zdd + S Z = -F_z advances with the
    particles in the tank frame.  Against the library's DEM step with its
    tank, FP64, 20 steps."""
    case = C.dem_damper(7, 7, 6, spacing=0.0079, seed=5, v_sigma=0.2)
    n = case.n
    fields = {"v": ("vector", case.v), "F": ("vector", np.zeros((n, 3))), "fwz": ("scalar", np.zeros(n)),
              "R": ("scalar", case.rho), "m": ("scalar", case.extra["m"])}
    nu, E = case.extra["nu"], case.extra["E"]
    consts = {"Ep": E / (2.0 * (1.0 - nu * nu)), "cf": case.extra["cf"], "g": tuple(case.g), "dt": case.dt,
              "S": case.extra["tank_S"], "M": case.extra["tank_M"]}
    tank = {"Z": case.extra["z0"], "Zd": 0.0, "Zdd": 0.0, "Fb": 0.0}
    sysm = L.LawSystem(case, fields, consts, EXAMPLE_2_LAWS, precision=S.SPH_PREC_F64, variables=tank)
    sysm.step(20)
    r, f, ids = sysm.host()
    got = sysm.variables()
    sim = S.Simulation(case, precision=S.SPH_PREC_F64)
    sim.step(20)
    r2, v2, _, _, ids2, _ = sim.state.to_host()
    Z, Zd, Zdd, Fb = sim.tank()
    k = _inv(ids)[ids2]
    motion = np.abs(r2 - case.r[_inv(case.id)[ids2]]).max()
    e = dict(r=float(np.abs(r[k] - r2).max() / motion), v=float(np.abs(f["v"][k] - v2).max() / np.abs(v2).max()),
             Z=abs(got["Z"] - Z) / abs(Z), Zd=abs(got["Zd"] - Zd) / abs(Zd))
    print("compiled_example_2", e, got, (Z, Zd))
    for name, x in e.items():
        assert x < 1e-9, (name, x)
    sysm.close()
    sim.close()

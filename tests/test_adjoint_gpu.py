"""GPU adjoint (sph_step_adjoint and the checkpointed autograd rollout)
against the CPU FP64 oracle adjoint, the oracle's complex-step derivatives,
and central finite differences."""
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
    path = os.environ.get("SPH_ADJ_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(REPORT, f, indent=1)
    print(name, vals)


def nrel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def moving_case(orc, dim, n, seed, steps=15, k=1):
    case = C.small_dam_break(dim, n, seed=seed, alpha=0.05, cells_per_radius=k)
    rng = np.random.default_rng(seed)
    case.v[: case.n_fluid] = rng.normal(0.0, 0.3, size=(case.n_fluid, dim))
    res = orc.step(orc.params(case), case.r, case.v, case.kind, case.id, steps)
    case.r, case.v = res.r, res.v
    return case


def gpu_step_adjoint(S, case, prec, wr_by_id, wv_by_id):
    """GPU adjoint of one step from case's state; w given per particle id.
    Returns (rbar0, vbar0) in case order and alpha_bar."""
    tdt = torch.float32 if prec == S.SPH_PREC_F32 else torch.float64
    sim = S.Simulation(case, precision=prec)
    # the forward output order = canonical order of this state's cells
    probe = S.Simulation(case, precision=prec)
    probe.step(1)
    ids_out = probe.state.id.cpu().numpy().astype(np.int64)
    probe.close()
    dim = case.dim
    g1r = [torch.tensor(wr_by_id[ids_out, k], dtype=torch.float64, device="cuda") for k in range(dim)]
    g1v = [torch.tensor(wv_by_id[ids_out, k], dtype=tdt, device="cuda") for k in range(dim)]
    g0r = [torch.zeros(case.n, dtype=torch.float64, device="cuda") for _ in range(dim)]
    g0v = [torch.zeros(case.n, dtype=tdt, device="cuda") for _ in range(dim)]
    ab = torch.zeros(1, dtype=torch.float64, device="cuda")
    ids_before = sim.state.id.clone()
    S.sph_step_adjoint(sim.ctx, sim.state.view(), S.grad_view(g1r, g1v), S.grad_view(g0r, g0v), ab.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(sim.state.id, ids_before)  # s_n is not modified
    rb = np.stack([t.cpu().numpy() for t in g0r], 1)
    vb = np.stack([t.cpu().double().numpy() for t in g0v], 1)
    sim.close()
    return rb, vb, float(ab.item())


TOL_STEP = {"f64": 1e-10, "f32": 1e-4}


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 2])
def test_step_adjoint_vs_oracle(S, orc, dim, n, prec, k):
    """k: cells per support radius (2: cells of edge h, the row stencil)."""
    case = moving_case(orc, dim, n, seed=40 + dim, k=k)
    P = S.SPH_PREC_F64 if prec == "f64" else S.SPH_PREC_F32
    rng = np.random.default_rng(7)
    wr = rng.normal(size=case.r.shape)
    wv = rng.normal(size=case.v.shape)
    # oracle (input order; ids are positions here: case.id == arange)
    assert np.array_equal(case.id, np.arange(case.n))
    orb, ovb, oab = orc.step_adjoint(orc.params(case, fp32_neighbours=(prec == "f32")), case.r, case.v,
                                     case.kind, case.id, wr, wv)
    rb, vb, ab = gpu_step_adjoint(S, case, P, wr, wv)
    fl = case.kind == 0
    e = dict(r=nrel(rb[fl], orb[fl]), v=nrel(vb[fl], ovb[fl]), alpha=abs(ab - oab) / abs(oab))
    report(f"step_adjoint[{dim}d-{prec}-k{k}]", **e)
    for f, x in e.items():
        assert x <= TOL_STEP[prec], (f, x)


def test_step_adjoint_dot_product_gpu(S, orc):
    """<J u, w> with J u from the oracle's complex step, <u, J^T w> from the
    GPU FP64 adjoint: agreement to 1e-10."""
    case = moving_case(orc, 2, 16, seed=52)
    rng = np.random.default_rng(3)
    fl = (case.kind == 0)[:, None]
    ur = rng.normal(size=case.r.shape) * fl * case.dx * 1e-2
    uv = rng.normal(size=case.v.shape) * fl * 0.1
    ua = 0.01
    wr = rng.normal(size=case.r.shape)
    wv = rng.normal(size=case.v.shape)
    _, _, Jr, Jv = orc.step_complex(orc.params(case), case.r, case.v, case.kind, case.id, ur, uv, ua)
    lhs = np.sum(Jr * wr) + np.sum(Jv * wv)
    rb, vb, ab = gpu_step_adjoint(S, case, S.SPH_PREC_F64, wr, wv)
    rhs = np.sum(ur * rb) + np.sum(uv * vb) + ua * ab
    report("dot_product_gpu_f64", rel=abs(lhs - rhs) / abs(lhs))
    assert lhs == pytest.approx(rhs, rel=1e-10)


def _rollout_grad(case, prec, v0, target, nsteps, k, **kw):
    from paper_1710_08259_gb300 import autograd as AG
    v = torch.tensor(v0, dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(case.alpha, dtype=torch.float64, requires_grad=True)
    rf, ids = AG.rollout(v, a, case, prec, nsteps, k, **kw)
    L = AG.target_loss(rf, ids, case, target)
    L.backward()
    return float(L.item()), v.grad.cpu().numpy(), float(a.grad.item())


def _rollout_loss(case, prec, v0, target, nsteps, alpha=None):
    from paper_1710_08259_gb300 import autograd as AG
    from paper_1710_08259_gb300 import sph as S
    with torch.no_grad():
        v = torch.tensor(v0, dtype=torch.float64, device="cuda")
        a = torch.tensor(case.alpha if alpha is None else alpha, dtype=torch.float64)
        rf, ids = AG.SPHRollout.forward(_Ctx(), v, a, case, prec, nsteps, nsteps + 1)
        return float(AG.target_loss(rf, ids, case, target).item())


class _Ctx:
    def mark_non_differentiable(self, *a):
        pass


def _fp32_rounded(orc, case):
    """The case with its positions moved by the FP32 rounding of their
    offsets in cells of edge 2h (the paper's cell size; ~1e-7 dx)."""
    P = orc.params(case)
    P.cs = 2.0 * case.h
    D = case.dim
    for k in range(D):
        P.ncell[k] = int(np.ceil(case.ncell[k] * case.cs / P.cs))
    cc, off, bad = orc.cell_coords(P, case.r)
    assert bad == 0
    c2 = case.copy()
    c2.r = np.array(case.dom_min[:D]) + cc[:, :D] * P.cs + off[:, :D].astype(np.float64)
    return c2


@pytest.mark.parametrize("clamp", [True, False])
def test_rollout_gradient_diff_case(S, orc, clamp):
    """The differentiable workload: 128x128 fluid, 200 steps, checkpoints
    every 20, loss = mean |r_T - target|^2, gradients w.r.t. v0 and alpha.

    * FP64 GPU vs the FP64 CPU oracle adjoint: 1e-8 (exact adjoint).
    * FP32 GPU vs the FP64 oracle's gradient of its own FP64 trajectory:
      the two trajectories part (the acoustic field amplifies rounding, and
      particles within FP32 rounding of the p >= 0 kink take different
      sides), so this comparison measures the trajectory's sensitivity, not
      the adjoint (which test_fp32_gradient_against_the_fp64_adjoint_of_its_
      trajectory holds to 1e-4; reading A10b).  The bound is 5x the change
      of the FP64 oracle's own gradient when its initial positions move by
      their FP32 offset rounding in cells of 2h (~1e-7 dx), plus 1e-4.
    * FP64 GPU vs central differences (eps = 1e-3) of the FP64 GPU rollout,
      along alpha (relative) and 8 random v0 directions (error / |grad|)."""
    case = C.diff_case()
    nsteps, k = 200, 20
    v0, target = case.v, case.target
    fl = case.kind == 0
    P = orc.params(case, clamp_neg_p=clamp)
    L_o, gv_o, ga_o, _ = orc.rollout_loss_grad(P, case, v0, target, nsteps)
    _, gv_p, ga_p, _ = orc.rollout_loss_grad(P, _fp32_rounded(orc, case), v0, target, nsteps)
    sens_v, sens_a = nrel(gv_p[fl], gv_o[fl]), abs(ga_p - ga_o) / abs(ga_o)
    kw = {} if clamp else {"clamp_neg_p": False}
    L64, gv64, ga64 = _rollout_grad(case, S.SPH_PREC_F64, v0, target, nsteps, k, **kw)
    L32, gv32, ga32 = _rollout_grad(case, S.SPH_PREC_F32, v0, target, nsteps, k, **kw)
    e = dict(L64=abs(L64 - L_o) / L_o, v64=nrel(gv64[fl], gv_o[fl]), a64=abs(ga64 - ga_o) / abs(ga_o),
             L32=abs(L32 - L_o) / L_o, v32=nrel(gv32[fl], gv_o[fl]), a32=abs(ga32 - ga_o) / abs(ga_o),
             sens_v=sens_v, sens_a=sens_a)
    if clamp:
        eps = 1e-3 * case.alpha
        fda = (_rollout_loss(case, S.SPH_PREC_F64, v0, target, nsteps, case.alpha + eps) -
               _rollout_loss(case, S.SPH_PREC_F64, v0, target, nsteps, case.alpha - eps)) / (2 * eps)
        e["fd_alpha"] = abs(ga64 - fda) / abs(fda)
        rng = np.random.default_rng(8)
        worst = 0.0
        gnorm = np.linalg.norm(gv64)
        for _ in range(8):
            d = np.zeros_like(v0)
            d[fl] = rng.normal(size=(int(fl.sum()), 2))
            d /= np.linalg.norm(d)
            h = 1e-3 * 0.01
            fd = (_rollout_loss(case, S.SPH_PREC_F64, v0 + h * d, target, nsteps) -
                  _rollout_loss(case, S.SPH_PREC_F64, v0 - h * d, target, nsteps)) / (2 * h)
            worst = max(worst, abs(float(np.sum(gv64 * d)) - fd) / gnorm)
        e["fd_v0"] = worst
    report(f"rollout_diff_case[clamp={clamp}]", **e, L=L_o, ga=ga_o)
    assert e["L64"] < 1e-10 and e["v64"] < 1e-8 and e["a64"] < 1e-8
    assert e["v32"] <= 5 * sens_v + 1e-4 and e["a32"] <= 5 * sens_a + 1e-4
    if clamp:
        assert e["fd_alpha"] < 1e-3 and e["fd_v0"] < 1e-3


@pytest.mark.parametrize("clamp", [True, False])
def test_fp32_gradient_against_the_fp64_adjoint_of_its_trajectory(S, orc, clamp):
    """The FP32 gradient of the differentiable workload (128x128 fluid, 200
    steps, checkpoints every 20) against the FP64 oracle adjoint evaluated
    along the same FP32 trajectory, taking that trajectory's pressure-clamp
    decisions (reading A10b): the stated 1e-4 relative in dL/dv0 (norm) and
    dL/dalpha.  This separates the adjoint's own arithmetic from the
    trajectory's sensitivity: the FP32 and FP64 forward rollouts themselves
    part by more than 1e-4 (the acoustic field amplifies rounding, and
    particles within rounding of the p = 0 kink take different sides)."""
    case = C.diff_case()
    nsteps, k = 200, 20
    fl = case.kind == 0
    nf = int(fl.sum())
    kw = {} if clamp else {"clamp_neg_p": False}
    # the FP32 forward trajectory, state by state (the rollout's own kernels)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32, **kw)
    states = []
    for _ in range(nsteps):
        r, v, _, _, ids, _ = sim.state.to_host()
        o = np.argsort(ids)                   # id order (= case order: ids are 0..n-1)
        sim.step(1)
        _, _, _, p, ids2, _ = sim.state.to_host()
        cl = np.zeros(case.n, bool)
        cl[ids2] = p <= 0.0                   # clamped in this step (p = max(p, 0))
        states.append((r[o], v[o], cl))
    r, _, _, _, ids, _ = sim.state.to_host()
    rT = r[np.argsort(ids)]
    sim.close()
    diff = rT[fl] - case.target
    L_traj = float(np.mean(np.sum(diff * diff, axis=1)))
    P = orc.params(case, clamp_neg_p=clamp, fp32_neighbours=True)
    rbar = np.zeros_like(case.r)
    rbar[fl] = 2.0 * diff / nf
    vbar = np.zeros_like(case.v)
    abar = 0.0
    for (rn, vn, cl) in reversed(states):
        rbar, vbar, ab = orc.step_adjoint(P, rn, vn, case.kind, case.id, rbar, vbar, clamped=cl)
        abar += ab
    L32, gv32, ga32 = _rollout_grad(case, S.SPH_PREC_F32, case.v, case.target, nsteps, k, **kw)
    e = dict(L=abs(L32 - L_traj) / L_traj, v=nrel(gv32[fl], vbar[fl]), alpha=abs(ga32 - abar) / abs(abar),
             clamped_frac=float(np.mean([s[2][fl].mean() for s in states])))
    report(f"fp32_adjoint_on_its_trajectory[clamp={clamp}]", **e, ga=abar)
    assert e["L"] < 1e-12          # the same trajectory
    assert e["v"] <= 1e-4 and e["alpha"] <= 1e-4, e


@pytest.mark.parametrize("nsteps,k", [(60, 20), (50, 20), (30, 7)])
def test_rollout_graphs_equal_eager(S, nsteps, k):
    """The CUDA-graph replay of the repeated segments launches the same
    kernels in the same order as the eager sweep: loss and gradients agree
    bit for bit (full segments only, a partial last segment, odd k)."""
    from paper_1710_08259_gb300 import autograd as AG
    case = C.diff_case()
    out = []
    for graphs in (False, True):
        v = torch.tensor(case.v, dtype=torch.float64, device="cuda", requires_grad=True)
        a = torch.tensor(case.alpha, dtype=torch.float64, requires_grad=True)
        rf, ids = AG.rollout(v, a, case, S.SPH_PREC_F32, nsteps, k, graphs=graphs)
        L = AG.target_loss(rf, ids, case, case.target)
        L.backward()
        out.append((rf.detach().cpu().numpy(), ids.cpu().numpy(), float(L.item()), v.grad.cpu().numpy(),
                    float(a.grad.item())))
    (r0, i0, L0, g0, a0), (r1, i1, L1, g1, a1) = out
    np.testing.assert_array_equal(i0, i1)
    np.testing.assert_array_equal(r0, r1)
    assert L0 == L1 and a0 == a1
    np.testing.assert_array_equal(g0, g1)
    assert np.abs(g0).max() > 0 and a0 != 0.0


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_rollout_reusing_builds_equals_rebuilding(S, prec):
    """Reverse steps on the saved build + density products of their
    recomputed forward steps give, bit for bit, the gradients of reverse
    steps that rebuild from the stored states."""
    from paper_1710_08259_gb300 import autograd as AG
    case = C.diff_case()
    P = S.SPH_PREC_F32 if prec == "f32" else S.SPH_PREC_F64
    out = []
    for reuse in (False, True):
        v = torch.tensor(case.v, dtype=torch.float64, device="cuda", requires_grad=True)
        a = torch.tensor(case.alpha, dtype=torch.float64, requires_grad=True)
        rf, ids = AG.rollout(v, a, case, P, 50, 20, reuse_builds=reuse)
        L = AG.target_loss(rf, ids, case, case.target)
        L.backward()
        out.append((v.grad.cpu().numpy(), float(a.grad.item())))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_build_save_load_errors(S):
    case = C.small_dam_break(2, 10)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    sim.build_cells()
    with pytest.raises(S.SphError):
        S.sph_build_save(sim.ctx)                    # no density pass since the build
    sim.step(1)
    nb = S.sph_build_save(sim.ctx)
    assert nb > 0 and nb % 256 == 0
    g = [torch.zeros(case.n, dtype=torch.float64, device="cuda") for _ in range(4)]
    gv = [torch.zeros(case.n, dtype=torch.float32, device="cuda") for _ in range(4)]
    with pytest.raises(S.SphError):                  # products of another particle count
        S.sph_adjoint_of_build(sim.ctx, case.n - 1, S.grad_view(g[:2], gv[:2]), S.grad_view(g[2:], gv[2:]))
    sim.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_adjoint_of_saved_equals_load_then_adjoint(S, prec):
    """sph_adjoint_of_saved reads a saved block in place: the same gradients,
    bit for bit, as sph_build_load followed by sph_adjoint_of_build, and the
    context's own build products are left as they were (a later
    sph_build_save writes the same bytes)."""
    P = S.SPH_PREC_F32 if prec == "f32" else S.SPH_PREC_F64
    case = C.small_dam_break(2, 24)
    sim = S.Simulation(case, precision=P)
    sim.step(3)
    n = case.n
    nb = S.sph_build_save(sim.ctx)
    saved = torch.zeros(nb // 8, dtype=torch.float64, device="cuda")
    S.sph_build_save(sim.ctx, saved.data_ptr())
    sim.step(2)                                      # the context's products move on
    nb2 = S.sph_build_save(sim.ctx)
    # (zeroed: the 256-byte padding between the sections is not written)
    own = torch.zeros(nb2 // 8, dtype=torch.float64, device="cuda")
    S.sph_build_save(sim.ctx, own.data_ptr())
    rng = np.random.default_rng(5)
    gsrc = [torch.tensor(rng.standard_normal(n), device="cuda") for _ in range(4)]
    vdt = torch.float32 if prec == "f32" else torch.float64
    gsv = [torch.tensor(rng.standard_normal(n), dtype=vdt, device="cuda") for _ in range(4)]
    outs = []
    for way in ("saved", "load"):
        gr = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(2)]
        gv = [torch.zeros(n, dtype=vdt, device="cuda") for _ in range(2)]
        ab = torch.zeros(1, dtype=torch.float64, device="cuda")
        src, dst = S.grad_view(gsrc[:2], gsv[:2]), S.grad_view(gr, gv)
        if way == "saved":
            S.sph_adjoint_of_saved(sim.ctx, saved.data_ptr(), n, src, dst, ab.data_ptr())
            after = torch.zeros_like(own)
            S.sph_build_save(sim.ctx, after.data_ptr())
            assert torch.equal(after, own)
        else:
            S.sph_build_load(sim.ctx, saved.data_ptr(), n)
            S.sph_adjoint_of_build(sim.ctx, n, src, dst, ab.data_ptr())
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in gr + gv] + [ab.cpu().numpy()])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    assert np.abs(outs[0][0]).max() > 0 and outs[0][-1][0] != 0.0
    g = S.grad_view(gsrc[:2], gsv[:2])
    h = S.grad_view(gsrc[2:], gsv[2:])
    with pytest.raises(S.SphError):                  # more particles than the context holds
        S.sph_adjoint_of_saved(sim.ctx, saved.data_ptr(), 10 ** 9, g, h)
    with pytest.raises(S.SphError):                  # not 256-byte aligned
        S.sph_adjoint_of_saved(sim.ctx, saved.data_ptr() + 8, n, g, h)
    with pytest.raises(S.SphError):                  # g_n aliases g_np1
        S.sph_adjoint_of_saved(sim.ctx, saved.data_ptr(), n, g, g)
    sim.close()


def test_rollout_without_checkpoints_equals_checkpointed(S):
    """k = 0 keeps every step's build products instead of checkpoints: the
    reverse sweep recomputes nothing and gives the same gradients bit for
    bit."""
    from paper_1710_08259_gb300 import autograd as AG
    case = C.diff_case()
    out = []
    for k in (20, 0):
        v = torch.tensor(case.v, dtype=torch.float64, device="cuda", requires_grad=True)
        a = torch.tensor(case.alpha, dtype=torch.float64, requires_grad=True)
        rf, ids = AG.rollout(v, a, case, S.SPH_PREC_F32, 50, k)
        L = AG.target_loss(rf, ids, case, case.target)
        L.backward()
        out.append((rf.detach().cpu().numpy(), v.grad.cpu().numpy(), float(a.grad.item())))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]

"""Pins of the oracle adjoint (reverse mode of one step and of a rollout).

The adjoint is hand-derived; it is checked against derivatives that come
from the forward step alone:
  * complex-step differentiation (Im f(x + i h u) / h, h = 1e-30) of the
    same step written on complex numbers, exact to rounding: the dot-product
    test <J u, w> = <u, J^T w>;
  * central finite differences of a rollout loss.
"""
import numpy as np
import pytest

from paper_1710_08259_gb300 import cases as C


def _moving_case(dim, n, seed, steps=15):
    """A small dam break advanced a few oracle steps, with random velocities
    added so that viscosity and compression are active."""
    from oracle import oracle as O
    case = C.small_dam_break(dim, n, seed=seed, alpha=0.05)
    rng = np.random.default_rng(seed)
    case.v[: case.n_fluid] = rng.normal(0.0, 0.3, size=(case.n_fluid, dim))
    p = O.params(case)
    res = O.step(p, case.r, case.v, case.kind, case.id, steps)
    assert res.rc == 0
    case.r, case.v = res.r, res.v
    assert np.count_nonzero(res.p) > 10
    return case


@pytest.mark.parametrize("dim,n", [(2, 14), (3, 6)])
def test_complex_step_matches_real_step(orc, dim, n):
    case = _moving_case(dim, n, seed=3 + dim)
    p = orc.params(case)
    ref = orc.step(p, case.r, case.v, case.kind, case.id, 1)
    z = np.zeros_like(case.r)
    ro, vo, dro, dvo = orc.step_complex(p, case.r, case.v, case.kind, case.id, z, z, 0.0)
    assert np.allclose(ro, ref.r, rtol=0, atol=1e-15 * np.abs(ref.r).max())
    assert np.allclose(vo, ref.v, rtol=1e-12, atol=1e-14 * np.abs(ref.v).max())
    assert np.all(dro == 0) and np.all(dvo == 0)


@pytest.mark.parametrize("dim,n", [(2, 14), (3, 6)])
@pytest.mark.parametrize("fp32_nb", [False, True])
def test_adjoint_dot_product(orc, dim, n, fp32_nb):
    """<J u, w> (complex step) = <u, J^T w> (adjoint) to 1e-10 for one step."""
    case = _moving_case(dim, n, seed=11 + dim)
    p = orc.params(case, fp32_neighbours=fp32_nb)
    rng = np.random.default_rng(99 + dim)
    fl = (case.kind == 0)[:, None]
    scale_r = case.dx * 1e-2
    ur = rng.normal(size=case.r.shape) * fl * scale_r
    uv = rng.normal(size=case.v.shape) * fl * 0.1
    ua = 0.01
    wr = rng.normal(size=case.r.shape)
    wv = rng.normal(size=case.v.shape)
    _, _, Jr, Jv = orc.step_complex(p, case.r, case.v, case.kind, case.id, ur, uv, ua)
    lhs = np.sum(Jr * wr) + np.sum(Jv * wv)
    rb, vb, ab = orc.step_adjoint(p, case.r, case.v, case.kind, case.id, wr, wv)
    rhs = np.sum(ur * rb) + np.sum(uv * vb) + ua * ab
    assert lhs == pytest.approx(rhs, rel=1e-10)
    # each input block separately (a wrong sign in one block cannot cancel)
    for (dr, dv, da) in ((ur, 0 * uv, 0.0), (0 * ur, uv, 0.0), (0 * ur, 0 * uv, ua)):
        _, _, Jr, Jv = orc.step_complex(p, case.r, case.v, case.kind, case.id, dr, dv, da)
        l1 = np.sum(Jr * wr) + np.sum(Jv * wv)
        r1 = np.sum(dr * rb) + np.sum(dv * vb) + da * ab
        assert l1 == pytest.approx(r1, rel=1e-9, abs=1e-13 * abs(lhs))
    assert abs(ab) > 0


def test_rollout_gradient_finite_differences(orc):
    """dL/dalpha and dL/dv0 along 4 random directions of a 30-step rollout
    against central differences (eps = 1e-3 relative)."""
    case = C.small_dam_break(2, 16, seed=21, alpha=0.02)
    rng = np.random.default_rng(4)
    v0 = np.zeros_like(case.v)
    v0[: case.n_fluid] = rng.normal(0.0, 0.01, size=(case.n_fluid, 2))
    target = case.r[: case.n_fluid] + rng.normal(0.0, 0.5 * case.dx, size=(case.n_fluid, 2))
    nsteps = 30
    p = orc.params(case)
    L, gv, ga, _ = orc.rollout_loss_grad(p, case, v0, target, nsteps)
    # alpha
    eps = 1e-3 * case.alpha
    pp = orc.params(case)
    pp.alpha = case.alpha + eps
    pm = orc.params(case)
    pm.alpha = case.alpha - eps
    fd = (orc.rollout_loss(pp, case, v0, target, nsteps) - orc.rollout_loss(pm, case, v0, target, nsteps)) / (2 * eps)
    assert ga == pytest.approx(fd, rel=2e-4, abs=1e-6 * abs(L))
    # v0 directions (fluid only)
    for k in range(4):
        d = np.zeros_like(v0)
        d[: case.n_fluid] = rng.normal(size=(case.n_fluid, 2))
        d /= np.linalg.norm(d)
        e = 1e-3 * 0.01
        fd = (orc.rollout_loss(p, case, v0 + e * d, target, nsteps) -
              orc.rollout_loss(p, case, v0 - e * d, target, nsteps)) / (2 * e)
        an = float(np.sum(gv * d))
        assert an == pytest.approx(fd, rel=1e-4, abs=1e-8 * np.linalg.norm(gv))


@pytest.mark.parametrize("dim,n", [(2, 14), (3, 6)])
def test_adjoint_with_given_clamp_decisions(orc, dim, n):
    """The reverse step that takes the pressure clamp's decisions as an input
    (for differentiating a trajectory another computation produced): given
    the step's own decisions it is the plain reverse step, bit for bit; told
    that no particle was clamped it is the reverse step of the model without
    the clamp; and its decisions matter (some particles are clamped here)."""
    case = _moving_case(dim, n, seed=21 + dim)
    p = orc.params(case)
    rng = np.random.default_rng(5)
    wr = rng.normal(size=case.r.shape)
    wv = rng.normal(size=case.v.shape)
    rho, pr, _ = orc.density(p, case.r, case.id)
    B = case.c0 ** 2 * case.rho0 / case.gamma
    own = B * ((rho / orc.rho_ref(p)) ** case.gamma - 1.0) < 0.0
    assert own.any() and not own.all()
    a = orc.step_adjoint(p, case.r, case.v, case.kind, case.id, wr, wv)
    b = orc.step_adjoint(p, case.r, case.v, case.kind, case.id, wr, wv, clamped=own)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    none = np.zeros(case.n, bool)
    c = orc.step_adjoint(p, case.r, case.v, case.kind, case.id, wr, wv, clamped=none)
    p0 = orc.params(case, clamp_neg_p=False)
    d = orc.step_adjoint(p0, case.r, case.v, case.kind, case.id, wr, wv)
    assert np.array_equal(c[0], d[0]) and np.array_equal(c[1], d[1]) and c[2] == d[2]
    assert not np.array_equal(a[0], c[0])

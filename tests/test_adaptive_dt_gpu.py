"""The adaptive time step (SPH_DT_ADAPTIVE) of the WCSPH step: the step size
that the CFL bound of each step sets for the next one, kept on the device,
against the oracle's adaptive step (itself pinned to free-fall kinematics in
test_oracle_pins.py), and the context's clock through checkpoints."""
import math

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


def _lone_particle(c0, dt):
    case = C.random_cloud(2, 1, seed=1)
    case.r = np.array([[0.05, 0.09]])
    case.v = np.array([[0.3, 0.1]])
    case.kind = np.zeros(1, np.uint8)
    case.id = np.zeros(1, np.uint32)
    case.ncell = (case.ncell[0], case.ncell[1] + 400, 1)
    case.dom_min = (case.dom_min[0], case.dom_min[1] - 400 * case.cs, 0.0)
    case.c0 = c0
    case.dt = dt
    return case


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("c0,cfl,dt_max", [(0.05, 0.1, 5e-3), (20.0, 0.5, 1e-3)])
def test_adaptive_free_fall(S, orc, prec, c0, cfl, dt_max):
    """An isolated particle over 20 steps in two calls: the GPU's step sizes,
    velocity, position and clock against the oracle's adaptive step."""
    case = _lone_particle(c0, dt_max)
    P = S.SPH_PREC_F64 if prec == "f64" else S.SPH_PREC_F32
    sim = S.Simulation(case, precision=P, dt_mode=S.SPH_DT_ADAPTIVE, cfl=cfl)
    sim.step(10)
    d = sim.step(10, diag=True)
    r, v = sim.state.to_host()[:2]
    ref = orc.step(orc.params(case, adaptive_dt=True, cfl=cfl), case.r, case.v, case.kind, case.id, 20)
    tol = 1e-13 if prec == "f64" else 2e-6
    assert d.dt == pytest.approx(ref.dt, rel=tol) and d.dt < dt_max
    assert d.time == pytest.approx(ref.time, rel=tol)
    assert np.allclose(v[0], ref.v[0], rtol=tol, atol=0)
    disp = np.abs(ref.r[0] - case.r[0]).max()
    assert np.abs(r[0] - ref.r[0]).max() <= tol * disp + (1e-15 if prec == "f64" else 1e-9)
    dt_next, t = S.sph_clock_get(sim.ctx)
    g = float(np.linalg.norm(case.g[:2]))
    bound = min(0.25 * case.h / (c0 + float(np.linalg.norm(v[0]))), 0.25 * math.sqrt(case.h / g))
    assert dt_next == pytest.approx(min(dt_max, cfl * bound), rel=tol) and t == d.time
    # (the first step takes dt_max, above the sound-speed bound when c0 = 20:
    # that step, and only that kind of excess, raises the CFL bit)
    st = sim.status()
    assert st & ~S.SPH_STATUS_CFL == 0
    assert bool(st & S.SPH_STATUS_CFL) == (dt_max > 0.25 * case.h / (c0 + 0.33))
    sim.close()


@pytest.mark.parametrize("dim,n,prec", [(2, 24, "f64"), (3, 10, "f32")])
def test_adaptive_dam_break_against_the_oracle(S, orc, dim, n, prec):
    """A dam break whose cap dt (1.1 x 0.2 h/c0) lies between the CFL bound
    (0.25 h/(c0 + vmax)) and cfl = 0.8 times it: the first step takes the
    cap, the later ones the bound.  40 adaptive steps on the GPU and in the
    oracle give the same clock and positions (FP64 to rounding; FP32 within
    the displacement bound of the fixed-step parity tests), with no CFL
    status."""
    case = C.small_dam_break(dim, n, seed=21)
    case.dt = 1.1 * case.dt
    P = S.SPH_PREC_F64 if prec == "f64" else S.SPH_PREC_F32
    sim = S.Simulation(case, precision=P, dt_mode=S.SPH_DT_ADAPTIVE, cfl=0.8)
    d = sim.step(40, diag=True)
    r, v, rho, p, ids, kind = sim.state.to_host()
    ref = orc.step(orc.params(case, adaptive_dt=True, cfl=0.8), case.r, case.v, case.kind, case.id, 40)
    k = np.argsort(case.id)[ids]
    dr, dro = r - case.r[k], ref.r[k] - case.r[k]
    if prec == "f64":
        assert d.time == pytest.approx(ref.time, rel=1e-11)
        assert np.abs(dr - dro).max() <= 1e-9 * np.abs(dro).max()
    else:
        assert d.time == pytest.approx(ref.time, rel=1e-5)
        assert np.abs(dr - dro).max() <= 1e-3 * np.abs(dro).max() + 1e-7 * case.dx
    assert d.dt < case.dt                      # the bound set the last step
    assert not (sim.status() & S.SPH_STATUS_CFL)
    sim.close()


def test_adaptive_clock_through_a_checkpoint(S, tmp_path):
    """The next step size and the elapsed time travel with a checkpoint: the
    restored simulation continues bit for bit; the clock rejects a step
    above the configured one."""
    case = C.small_dam_break(2, 20, seed=22)
    case.dt = 1.1 * case.dt
    sim = S.Simulation(case, precision=S.SPH_PREC_F32, dt_mode=S.SPH_DT_ADAPTIVE, cfl=0.8)
    sim.step(15)
    path = str(tmp_path / "ck.npz")
    sim.save(path)
    back = S.Simulation.restore(path)
    assert S.sph_clock_get(back.ctx) == S.sph_clock_get(sim.ctx)
    a = sim.step(10, diag=True)
    b = back.step(10, diag=True)
    assert a.dt == b.dt and a.time == b.time
    for x, y in zip(sim.state.to_host(), back.state.to_host()):
        assert np.array_equal(x, y)
    with pytest.raises(S.SphError):
        S.sph_clock_set(sim.ctx, 2.0 * case.dt, 0.0)
    S.sph_clock_set(sim.ctx, 0.5 * case.dt, 1.25)
    assert S.sph_clock_get(sim.ctx) == (0.5 * case.dt, 1.25)
    d = sim.step(1, diag=True)
    assert d.dt == 0.5 * case.dt and d.time == pytest.approx(1.25 + 0.5 * case.dt, rel=1e-15)
    sim.close()
    back.close()


def test_fixed_step_clock(S):
    """A fixed step keeps params.dt and counts time."""
    case = C.small_dam_break(2, 12, seed=23)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    d = sim.step(7, diag=True)
    assert d.dt == case.dt and d.time == pytest.approx(7 * case.dt, rel=1e-14)
    assert S.sph_clock_get(sim.ctx)[0] == case.dt
    with pytest.raises(S.SphError):
        S.sph_clock_set(sim.ctx, 0.5 * case.dt, 0.0)
    sim.close()


def test_adaptive_step_not_in_the_adjoint_or_a_batch(S):
    case = C.small_dam_break(2, 10, seed=24)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32, dt_mode=S.SPH_DT_ADAPTIVE, cfl=0.5)
    n = case.n
    z = lambda dt: torch.zeros(n, dtype=dt, device="cuda")
    g1 = S.SphGrad()
    g0 = S.SphGrad()
    bufs = []
    for g in (g1, g0):
        for k in range(2):
            rb, vb = z(torch.float64), z(torch.float32)
            bufs += [rb, vb]
            g.r_bar[k], g.v_bar[k] = rb.data_ptr(), vb.data_ptr()
    ab = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SphError):
        S.sph_step_adjoint(sim.ctx, sim.state.view(), g1, g0, ab.data_ptr())
    sim.close()
    with pytest.raises(S.SphError):
        S.Batch([case], S.SPH_PREC_F32, dt_mode=S.SPH_DT_ADAPTIVE, cfl=0.5)

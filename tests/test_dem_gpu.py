"""GPU parity (through the C ABI) of the DEM particle damper of Example 2
(Section 5.2) against the CPU oracle (sph_oracle_dem.c).

Accelerations are held to the oracle's rounding bound: for relative
precision eps (FP32: 2^-23, FP64: 2^-52) every length the contact law sees
may carry 4 eps max(cs, R_i + R_j), and the law's terms are bounded through
their derivatives, the damping term delta^(1/4) through its Hoelder
continuity at 0, the friction direction through its turn (sph_oracle_dem.c).
The tank acceleration is held to the sum of those bounds / M.
"""
import math

import numpy as np
import pytest

from paper_1710_08259_gb300 import cases as C

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SYM, PER, CUT = C.BC_SYMMETRIC, C.BC_PERIODIC, C.BC_CUTOFF
EPS = {"f64": 2.0 ** -52, "f32": 2.0 ** -23}


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08259_gb300 import build as B
    B.build()
    from paper_1710_08259_gb300 import sph
    return sph


def _prec(S, name):
    return S.SPH_PREC_F64 if name == "f64" else S.SPH_PREC_F32


def _inv(ids):
    inv = np.empty(int(ids.max()) + 1, np.int64)
    inv[ids] = np.arange(ids.size)
    return inv


def _cloud(n, ncell, bc, seed, R=0.004, spread=0.3, v=0.3):
    """Random overlapping spheres (radii R (1 - U[0, spread])) in a box of
    ncell cells of edge 2R."""
    c = C.dem_damper(1, 1, 1)
    rng = np.random.default_rng(seed)
    c.cs = 2.0 * R
    c.h = R
    c.ncell = tuple(ncell)
    c.bc = tuple(bc)
    ext = np.asarray(ncell, float) * c.cs
    c.r = rng.uniform(0.0, 1.0, size=(n, 3)) * ext
    c.v = rng.normal(0.0, v, size=(n, 3))
    c.rho = R * (1.0 - rng.uniform(0.0, spread, n))
    c.extra["m"] = 7850.0 * 4.0 / 3.0 * math.pi * c.rho ** 3
    c.kind = np.zeros(n, np.uint8)
    c.id = rng.permutation(n).astype(np.uint32)
    c.n_fluid = n
    return c


CONFIGS = [
    ("walls3", lambda: _cloud(1500, (8, 7, 6), (SYM, SYM, SYM), 201)),
    ("per_walls", lambda: _cloud(1500, (8, 7, 6), (PER, SYM, SYM), 202)),
    ("cut_walls", lambda: _cloud(1200, (6, 6, 6), (CUT, SYM, SYM), 203)),
    ("damper_packed", lambda: C.dem_damper(9, 9, 7, spacing=0.00792, seed=204, v_sigma=0.2, jitter=0.01)),
]
IDS = [c[0] for c in CONFIGS]


def _reference(orc, case, prec, eps, tank):
    p = orc.dem_params(case, fp32=(prec == "f32"), tank=tank)
    F, Fb, bound, nc = orc.dem_forces(p, case.r, case.v, case.rho, case.extra["m"], case.id, eps=eps)
    M, Sk = case.extra["tank_M"], case.extra["tank_S"]
    Z0 = case.extra["z0"]
    Zdd = (-Sk * Z0 - Fb[2]) / M if tank else 0.0
    a = F / case.extra["m"][:, None] + np.asarray(case.g)[None, :] - np.array([0.0, 0.0, Zdd])[None, :]
    return a, F, Fb, bound, nc, Zdd, p


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name,make", CONFIGS, ids=IDS)
def test_dem_forces_within_the_rounding_bound(S, orc, name, make, prec):
    case = make()
    for k in range(3):
        assert case.r[:, k].min() >= 0.0 and case.r[:, k].max() < case.ncell[k] * case.cs
    sim = S.Simulation(case, precision=_prec(S, prec))
    a = sim.forces()
    r, v, _, _, ids, kind = sim.state.to_host()
    a = np.stack([t.cpu().double().numpy() for t in a], axis=1)
    Zg, Zdg, Zddg, Fbg = sim.tank()
    k = _inv(case.id)[ids]
    eps = EPS[prec]
    aref, F, Fb, bound, nc, Zdd, _ = _reference(orc, case, prec, eps, True)
    m = case.extra["m"][k]
    Zdd_bound = bound.sum() / case.extra["tank_M"] + 4 * eps * abs(Zdd)
    assert abs(Zddg - Zdd) <= Zdd_bound, (Zddg, Zdd, Zdd_bound)
    ab = bound[k] / m + 4 * eps * np.abs(aref[k]).max(1) + Zdd_bound
    err = np.linalg.norm(a - aref[k], axis=1)
    ratio = float((err / ab).max())
    print(f"dem_forces[{name}-{prec}] err/bound {ratio:.3g}, contacts {nc}, max|a| {np.abs(aref).max():.3g}")
    assert ratio <= 1.0
    assert nc > 0
    # radius and mass moved with their spheres
    np.testing.assert_array_equal(sim.state.radius.cpu().double().numpy(),
                                  case.rho[k].astype(np.float32 if prec == "f32" else np.float64))
    np.testing.assert_array_equal(r, case.r[k])
    assert (Zg, Zdg) == (case.extra["z0"], 0.0)           # sph_forces leaves the tank alone


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name,make", CONFIGS, ids=IDS)
def test_dem_step(S, orc, name, make, prec):
    case = make()
    sim = S.Simulation(case, precision=_prec(S, prec))
    d = sim.step(1, diag=True)
    r, v, _, _, ids, kind = sim.state.to_host()
    k = _inv(case.id)[ids]
    eps = EPS[prec]
    aref, F, Fb, bound, nc, Zdd, p = _reference(orc, case, prec, eps, True)
    res = orc.dem_step(p, case.r, case.v, case.rho, case.extra["m"], case.kind, case.id,
                       tank=(case.extra["z0"], 0.0), nsteps=1)
    assert res.rc == 0
    m = case.extra["m"][k]
    Zdd_bound = bound.sum() / case.extra["tank_M"] + 4 * eps * abs(Zdd)
    ab = bound[k] / m + 4 * eps * np.abs(aref[k]).max(1) + Zdd_bound
    bv = case.dt * ab + 4 * eps * np.abs(res.v[k]).max(1)
    ev = float((np.linalg.norm(v - res.v[k], axis=1) / bv).max())
    L = np.array([case.ncell[q] * case.cs for q in range(3)])
    dr_g, dr_o = r - case.r[k], res.r[k] - case.r[k]
    for q in range(3):
        if case.bc[q] == PER:
            dr_g[:, q] -= L[q] * np.round(dr_g[:, q] / L[q])
            dr_o[:, q] -= L[q] * np.round(dr_o[:, q] / L[q])
    er = float((np.linalg.norm(dr_g - dr_o, axis=1) / (case.dt * bv + 4 * eps * L.max())).max())
    Z, Zd, Zddg, Fbg = sim.tank()
    print(f"dem_step[{name}-{prec}] v {ev:.3g} dr {er:.3g}")
    assert ev <= 1.0 and er <= 1.0
    assert abs(Zd - res.tank[1]) <= case.dt * Zdd_bound + 4 * eps * abs(res.tank[1])
    if prec == "f64":
        assert d.n_pairs == res.diag.n_contacts
    else:
        assert abs(d.n_pairs - res.diag.n_contacts) <= 2
    assert sim.status() == 0


def _noisy_oracle(orc, case, p, nsteps, eps, seed):
    """The oracle stepped one step at a time with every position and velocity
    perturbed by a few units of rounding (eps) after each step: the spread a
    rounding difference at every step causes."""
    rng = np.random.default_rng(seed)
    r, v, tank = case.r.copy(), case.v.copy(), (case.extra["z0"], 0.0)
    for _ in range(nsteps):
        res = orc.dem_step(p, r, v, case.rho, case.extra["m"], case.kind, case.id, tank=tank, nsteps=1)
        assert res.rc == 0
        r = res.r * (1.0 + 4.0 * eps * rng.uniform(-1.0, 1.0, r.shape))
        v = res.v * (1.0 + 4.0 * eps * rng.uniform(-1.0, 1.0, v.shape))
        tank = tuple(res.tank)
    return r, v, np.array(tank)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_example_2_1000_steps(S, orc, prec):
    """Example 2 as tabulated (567 spheres, tank on its spring released from
    Z = -0.05 m), 1000 steps (50 ms: the spheres land and the tank swings),
    against the FP64 oracle.  The damping term delta^(1/4) has an infinite
    slope at contact onset, so rounding differences grow at every new
    contact: the trajectories are held to the oracle's own spread under a
    rounding-sized perturbation (4 units of the form's precision) at every
    step, within a factor 10."""
    case = C.dem_damper()
    n = 1000
    sim = S.Simulation(case, precision=_prec(S, prec))
    sim.step(n)
    r, v, _, _, ids, kind = sim.state.to_host()
    Z, Zd, Zdd, Fb = sim.tank()
    p = orc.dem_params(case)
    ref = orc.dem_step(p, case.r, case.v, case.rho, case.extra["m"], case.kind, case.id,
                       tank=(case.extra["z0"], 0.0), nsteps=n)
    assert ref.rc == 0 and ref.diag.n_contacts > 0      # the spheres are on the floor by now
    pr, pv, pt = _noisy_oracle(orc, case, p, n, EPS[prec], seed=9)
    k = _inv(case.id)[ids]
    sens = dict(r=np.abs(pr - ref.r).max(), v=np.abs(pv - ref.v).max(), Z=abs(pt[0] - ref.tank[0]),
                Zd=abs(pt[1] - ref.tank[1]))
    err = dict(r=np.abs(r - ref.r[k]).max(), v=np.abs(v - ref.v[k]).max(), Z=abs(Z - ref.tank[0]),
               Zd=abs(Zd - ref.tank[1]))
    print(f"example_2_{prec}_1000", {f: (float(err[f]), float(sens[f])) for f in err})
    for f in err:
        assert err[f] <= 10.0 * sens[f], (f, err[f], sens[f])
    if prec == "f64":
        # the same arithmetic up to rounding order: far inside the spread
        assert err["r"] <= 1e-10 * np.abs(ref.r - case.r).max()
        assert err["v"] <= 1e-10 * np.abs(ref.v).max()
    # the tank's motion itself agrees closely
    assert abs(Z - ref.tank[0]) <= 1e-3 * abs(ref.tank[0])
    assert sim.status() == 0


def test_dem_limits(S):
    case = C.dem_damper()
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    from paper_1710_08259_gb300.sph import SphGrad
    g = SphGrad()
    with pytest.raises(S.SphError):
        S.sph_step_adjoint(sim.ctx, sim._view, g, g)
    with pytest.raises(S.SphError):
        S.Batch([case])
    st = sim.state.view()
    st.radius = None
    with pytest.raises(S.SphError):
        S.sph_step(sim.ctx, st, 1)
    other = S.Simulation(C.small_dam_break(2, 10))
    with pytest.raises(S.SphError):
        S.sph_tank_get(other.ctx)

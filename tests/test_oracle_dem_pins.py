"""Pins of the DEM oracle (sph_oracle_dem.c: the contact law of Example 2,
Eq. DEM_force with Eq. effective_quantities, symmetric tank walls, the tank
oscillator of Eq. tank_ode), each against something other than the oracle:

* a sphere resting on a symmetric floor carries its weight at the overlap of
  Hertz's sphere-on-rigid-plane law (4/3) E/(1-nu^2) sqrt(R) d^(3/2) = m g
  (a mirror image reproduces that law exactly), with the 3/2 power;
* a head-on collision matches an independent integration (scipy) of the
  one-dimensional contact equation m' d'' = -(k d^(3/2) + c d^(1/4) d'):
  restitution coefficient and contact time; the damping model is
  self-similar, so the restitution does not depend on the impact speed and
  the contact time scales as v^(-1/5);
* pair forces (normal and friction) conserve momentum;
* friction has magnitude c_f |f_n|, is tangential and drags along the
  relative sliding velocity;
* walls equal explicit mirror copies in a larger cut-off domain, and the
  wall force F^b is the force those copies exert;
* the tank's symplectic-Euler oscillation has its discrete closed form, and
  a free particle stays at rest in the lab frame (tank frame acceleration).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1710_08259_gb300 import cases as C

SYM, PER, CUT = C.BC_SYMMETRIC, C.BC_PERIODIC, C.BC_CUTOFF


def _few(r, v, R=0.004, ncell=(6, 6, 6), bc=(CUT, CUT, CUT), dt=1e-6, g=(0.0, 0.0, 0.0), **kw):
    c = C.dem_damper(1, 1, 1, **kw)
    r = np.atleast_2d(np.asarray(r, float))
    n = r.shape[0]
    c.r = r
    c.v = np.atleast_2d(np.asarray(v, float))
    c.rho = np.full(n, R)
    c.extra["m"] = np.full(n, 7850.0 * 4.0 / 3.0 * math.pi * R ** 3)
    c.kind = np.zeros(n, np.uint8)
    c.id = np.arange(n, dtype=np.uint32)
    c.n_fluid = n
    c.h = R
    c.cs = 2.0 * R
    c.ncell = tuple(ncell)
    c.bc = tuple(bc)
    c.dt = dt
    c.g = tuple(g)
    return c


def _Ep(E, nu):
    return E / (2.0 * (1.0 - nu * nu))


def test_sphere_on_a_symmetric_floor_carries_its_weight():
    R, E, nu = 0.004, 2.06e6, 0.33
    c = _few([[0.024, 0.024, 0.0]], [[0, 0, 0]], R=R, bc=(CUT, CUT, SYM), g=(0.0, 0.0, -9.81))
    m = c.extra["m"][0]
    # Hertz, sphere on a rigid plane: (4/3) E/(1-nu^2) sqrt(R) d^(3/2) = m g
    dw = (m * 9.81 / (4.0 / 3.0 * E / (1.0 - nu * nu) * math.sqrt(R))) ** (2.0 / 3.0)
    c.r[0, 2] = R - dw
    p = O.dem_params(c, tank=False)
    F, Fb, _, n = O.dem_forces(p, c.r, c.v, c.rho, c.extra["m"], c.id)
    assert n == 1
    np.testing.assert_allclose(F[0], [0.0, 0.0, m * 9.81], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Fb, F[0], rtol=1e-15)          # the floor's force is the wall force
    # the 3/2 power: 21 % more overlap carries 1.21^1.5 the weight
    c.r[0, 2] = R - 1.21 * dw
    F2, _, _, _ = O.dem_forces(p, c.r, c.v, c.rho, c.extra["m"], c.id)
    np.testing.assert_allclose(F2[0, 2] / F[0, 2], 1.21 ** 1.5, rtol=1e-12)
    # at rest on the floor the next step leaves it at rest
    c.r[0, 2] = R - dw
    res = O.dem_step(p, c.r, c.v, c.rho, c.extra["m"], c.kind, c.id, nsteps=1)
    assert abs(res.v[0, 2]) < 1e-12


def _collide(v0, dt, R=0.004, E=2.06e6, nu=0.33, rho=7850.0):
    """Head-on collision of two equal spheres (relative speed 2 v0) in free
    space: (restitution coefficient, contact time) from the oracle."""
    x0 = 0.05
    gap = 1e-5
    c = _few([[x0 - R - gap / 2, 0.024, 0.024], [x0 + R + gap / 2, 0.024, 0.024]],
             [[v0, 0, 0], [-v0, 0, 0]], R=R, ncell=(13, 6, 6), dt=dt)
    p = O.dem_params(c, tank=False)
    r, v = c.r, c.v
    steps_in = 0
    seen = False
    for _ in range(200000):
        res = O.dem_step(p, r, v, c.rho, c.extra["m"], c.kind, c.id, nsteps=1)
        r, v = res.r, res.v
        if res.diag.n_contacts:
            seen = True
            steps_in += 1
        elif seen:
            break
    assert seen and res.diag.n_contacts == 0
    return (v[1, 0] - v[0, 0]) / (2.0 * v0), steps_in * dt


def _reference_collision(v0, R=0.004, E=2.06e6, nu=0.33, rho=7850.0):
    """The same contact as one ODE for the overlap d(t), integrated by scipy:
    m' d'' = -(k d^1.5 + c d^0.25 d'), d(0) = 0, d'(0) = 2 v0."""
    from scipy.integrate import solve_ivp
    m = rho * 4.0 / 3.0 * math.pi * R ** 3
    mp = m / 2.0
    Rp = R / 2.0
    k = 4.0 / 3.0 * math.sqrt(Rp) * _Ep(E, nu)
    cc = math.sqrt(mp * k) / 8.0

    def f(t, y):
        d, dd = y
        dp = max(d, 0.0)
        return [dd, -(k * dp ** 1.5 + cc * dp ** 0.25 * dd) / mp]

    def out(t, y):
        return y[0]
    out.terminal = True
    out.direction = -1
    sol = solve_ivp(f, [0.0, 1.0], [0.0, 2.0 * v0], events=out, rtol=1e-11, atol=1e-16, max_step=1e-6)
    te = sol.t_events[0][0]
    ve = sol.y_events[0][0][1]
    return -ve / (2.0 * v0), te


def test_collision_matches_the_contact_equation_and_is_self_similar():
    es, ts = [], []
    for v0 in (0.1, 0.5, 2.0):
        e, tc = _collide(v0, dt=2e-7 * (0.5 / v0) ** 0.2)
        e_ref, t_ref = _reference_collision(v0)
        assert abs(e / e_ref - 1.0) < 3e-3, (v0, e, e_ref)
        assert abs(tc / t_ref - 1.0) < 3e-3, (v0, tc, t_ref)
        es.append(e)
        ts.append(tc)
    assert 0.0 < es[0] < 1.0
    assert max(es) - min(es) < 3e-3 * es[0]                       # speed-independent restitution
    np.testing.assert_allclose(ts[0] / ts[2], (2.0 / 0.1) ** 0.2, rtol=3e-3)


def _cloud(n, ncell, bc, seed, R=0.004):
    rng = np.random.default_rng(seed)
    cs = 2.0 * R
    ext = np.asarray(ncell, float) * cs
    c = _few(rng.uniform(0.0, 1.0, size=(n, 3)) * ext, rng.normal(0, 0.3, size=(n, 3)), R=R, ncell=ncell, bc=bc)
    c.rho = R * (1.0 + rng.uniform(-0.3, 0.0, n))             # radii up to R: h = R
    c.extra["m"] = 7850.0 * 4.0 / 3.0 * math.pi * c.rho ** 3
    c.id = rng.permutation(n).astype(np.uint32)
    return c


def test_pair_forces_conserve_momentum():
    c = _cloud(600, (6, 6, 6), (CUT, CUT, CUT), seed=3)
    p = O.dem_params(c, tank=False)
    F, Fb, _, n = O.dem_forces(p, c.r, c.v, c.rho, c.extra["m"], c.id)
    assert n > 100
    assert np.all(np.abs(F.sum(0)) < 1e-12 * np.abs(F).sum())
    assert np.all(Fb == 0)


def test_friction_is_tangential_and_drags_along_the_sliding():
    R = 0.004
    c = _few([[0.02, 0.02, 0.02], [0.02 + 1.9 * R, 0.02, 0.02]], [[0.0, 0.3, 0.0], [-0.2, -0.1, 0.05]], R=R)
    p = O.dem_params(c, tank=False)
    F, _, _, n = O.dem_forces(p, c.r, c.v, c.rho, c.extra["m"], c.id)
    assert n == 2
    nrm = np.array([-1.0, 0.0, 0.0])                          # from 2 to 1
    fn = F[0] @ nrm
    ft = F[0] - fn * nrm
    vrel = c.v[1] - c.v[0]
    vt = vrel - (vrel @ nrm) * nrm                            # sliding of 2 relative to 1
    assert fn > 0                                             # repulsive (and approaching)
    np.testing.assert_allclose(np.linalg.norm(ft), c.extra["cf"] * abs(fn), rtol=1e-12)
    np.testing.assert_allclose(ft / np.linalg.norm(ft), vt / np.linalg.norm(vt), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(F[0], -F[1], rtol=1e-13, atol=1e-16)


def _explicit_copies(c):
    L = [c.ncell[k] * c.cs for k in range(3)]
    reps = []
    for code in range(27):
        t = [(code // 3 ** k) % 3 for k in range(3)]
        if any(t[k] and c.bc[k] == CUT for k in range(3)):
            continue
        r, v = c.r.copy(), c.v.copy()
        for k in range(3):
            if t[k] == 0:
                continue
            if c.bc[k] == PER:
                r[:, k] = r[:, k] - L[k] if t[k] == 1 else r[:, k] + L[k]
            else:
                w = 0.0 if t[k] == 1 else L[k]
                r[:, k] = 2.0 * w - r[:, k]
                v[:, k] = -v[:, k]
        reps.append((code, r, v))
    big = c.copy()
    big.r = np.concatenate([x[1] for x in reps])
    big.v = np.concatenate([x[2] for x in reps])
    big.rho = np.tile(c.rho, len(reps))
    big.extra["m"] = np.tile(c.extra["m"], len(reps))
    big.kind = np.tile(c.kind, len(reps))
    big.id = np.arange(big.r.shape[0], dtype=np.uint32)
    big.dom_min = tuple(-L[k] for k in range(3))
    big.ncell = tuple(3 * c.ncell[k] for k in range(3))
    big.bc = (CUT, CUT, CUT)
    real = [i for i, x in enumerate(reps) if x[0] == 0][0]
    return big, np.arange(real * c.n, (real + 1) * c.n)


@pytest.mark.parametrize("bc", [(SYM, SYM, SYM), (PER, SYM, SYM), (SYM, CUT, SYM)])
def test_walls_equal_explicit_mirror_copies(bc):
    c = _cloud(300, (4, 3, 3), bc, seed=5)
    p = O.dem_params(c, tank=False)
    F, Fb, _, n = O.dem_forces(p, c.r, c.v, c.rho, c.extra["m"], c.id)
    big, sel = _explicit_copies(c)
    Fbig, _, _, _ = O.dem_forces(O.dem_params(big, tank=False), big.r, big.v, big.rho, big.extra["m"], big.id)
    np.testing.assert_allclose(F, Fbig[sel], rtol=0, atol=1e-12 * np.abs(F).max())
    # F^b: what the mirror copies add (periodic copies are neighbours, not walls)
    only = c.copy()
    only.bc = tuple(PER if b == PER else CUT for b in c.bc)
    Fonly, _, _, _ = O.dem_forces(O.dem_params(only, tank=False), c.r, c.v, c.rho, c.extra["m"], c.id)
    np.testing.assert_allclose(Fb, (F - Fonly).sum(0), rtol=1e-10, atol=1e-12 * np.abs(F).sum())
    assert np.any(Fb != 0)


def test_tank_oscillation_and_the_tank_frame():
    c = C.dem_damper()                       # the 0.1 m tank of Example 2, one sphere left in it
    c.r = np.array([[0.05, 0.05, 0.05]])
    c.v = np.zeros((1, 3))
    c.rho = c.rho[:1]
    c.extra["m"] = c.extra["m"][:1]
    c.kind = c.kind[:1]
    c.id = np.zeros(1, np.uint32)
    c.n_fluid = 1
    c.g = (0.0, 0.0, 0.0)
    c.dt = 1e-4
    p = O.dem_params(c)
    M, S = c.extra["tank_M"], c.extra["tank_S"]
    Z0 = 0.2 * c.extra["z0"]                 # small enough that the sphere meets no wall
    n = 700
    res = O.dem_step(p, c.r, c.v, c.rho, c.extra["m"], c.kind, c.id, tank=(Z0, 0.0), nsteps=n)
    assert res.rc == 0 and res.diag.n_contacts == 0
    # symplectic Euler on M Z'' + S Z = 0: Z_n = Z0 cos(n th) + B sin(n th),
    # cos th = 1 - g2 dt^2 / 2, B = -Z0 g2 dt^2 / (2 sin th), g2 = S / M
    g2, dt = S / M, c.dt
    th = math.acos(1.0 - g2 * dt * dt / 2.0)
    B = -Z0 * g2 * dt * dt / (2.0 * math.sin(th))
    np.testing.assert_allclose(res.tank[0], Z0 * math.cos(n * th) + B * math.sin(n * th), rtol=1e-9, atol=1e-13)
    # a free particle stays at rest in the lab frame: it moves by -dZ in the tank's frame
    np.testing.assert_allclose(res.v[0], [0.0, 0.0, -res.tank[1]], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(res.r[0, 2] - 0.05, -(res.tank[0] - Z0), rtol=1e-9, atol=1e-15)


def test_a_resting_sphere_pushes_the_tank_down():
    """Newton's third law through the walls: the floor holds the sphere up
    with its weight m g, so the sphere pushes the tank (at Z = 0, no spring
    force) down: Zddot = -m g / M."""
    R, E, nu = 0.004, 2.06e6, 0.33
    c = C.dem_damper()
    m = c.extra["m"][0]
    dw = (m * 9.81 / (4.0 / 3.0 * E / (1.0 - nu * nu) * math.sqrt(R))) ** (2.0 / 3.0)
    c.r = np.array([[0.05, 0.05, R - dw]])
    c.v = np.zeros((1, 3))
    c.rho = c.rho[:1]
    c.extra["m"] = c.extra["m"][:1]
    c.kind = c.kind[:1]
    c.id = np.zeros(1, np.uint32)
    c.n_fluid = 1
    res = O.dem_step(O.dem_params(c), c.r, c.v, c.rho, c.extra["m"], c.kind, c.id, tank=(0.0, 0.0), nsteps=1)
    assert res.rc == 0 and res.diag.n_contacts == 1
    np.testing.assert_allclose(res.diag.Fb[2], m * 9.81, rtol=1e-12)
    np.testing.assert_allclose(res.diag.Zddot, -m * 9.81 / c.extra["tank_M"], rtol=1e-12)


def test_a_head_on_impact_has_no_friction():
    """Purely normal approach (and a sphere against its own wall image):
    no sliding, so no tangential force at all, whatever the rounding of the
    normal leaves in v_t."""
    R = 0.004
    rng = np.random.default_rng(4)
    for _ in range(20):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        x0 = np.array([0.024, 0.024, 0.024])
        c = _few([x0, x0 + 1.93 * R * u], [0.7 * u, -0.4 * u], R=R)
        F, _, _, n = O.dem_forces(O.dem_params(c, tank=False), c.r, c.v, c.rho, c.extra["m"], c.id)
        assert n == 2
        ft = F[0] - (F[0] @ u) * u
        assert np.linalg.norm(ft) <= 1e-12 * np.linalg.norm(F[0])
    c = _few([[0.024, 0.024, 0.6 * R]], [[0.0, 0.0, -1.3]], R=R, bc=(CUT, CUT, SYM))
    F, Fb, _, n = O.dem_forces(O.dem_params(c, tank=False), c.r, c.v, c.rho, c.extra["m"], c.id)
    assert n == 1 and F[0, 0] == 0.0 and F[0, 1] == 0.0 and F[0, 2] > 0

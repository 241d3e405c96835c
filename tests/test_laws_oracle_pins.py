"""Pins of the interaction-law oracle (oracle/laws_oracle.py), which
evaluates equation systems written for the GPU law compiler in FP64:

* the equations of Appendix A evaluated by it equal the Example 1a oracle
  written separately in C (sph_oracle_bc.c), step after step;
* on a uniform periodic lattice: sum_j(1) counts the 32 lattice neighbours,
  sph_S of a constant is the lattice sum, and a plane wave A = sin(k . x) is
  an eigenvector of sph_L, and sph_G / sph_D map it to cos(k . x) times a
  vector, with eigenvalues and coefficients from lattice sums over integer
  offsets (computed here, not by the oracle);
* sph_S written as sum_j(...) plus the self term equals sph_S;
* the social force model of Section 6 (Eq. social_force_model) written with
  sum_j: two people in and out of contact and beyond the radius against the
  equation written out by hand, Newton's third law, the semi-implicit Euler
  order, a person against their mirror image at a symmetric wall, the
  reflection of vector fields at that image (also for a single particle) and
  the distance across a periodic end.
"""
import math

import numpy as np
import pytest

from oracle import laws_oracle as LO
from oracle import oracle as O
from paper_1710_08259_gb300 import cases as C

APPENDIX_A = ["rhodot = -rho*sph_D(v, mass, rho)",
              "rho = euler(rho, rhodot, dt)",
              "p = c**2*(rho - rho0)",
              "vdot = -1/rho*sph_G(p, mass, rho)",
              "vdot = vdot + 0.1*c*h*sph_A(v, mass, rho) + g",
              "v = euler(v, vdot, dt)",
              "r = euler(r, v, dt)"]


def appendix_a_system(case):
    n = case.n
    fields = {"rho": ("scalar", case.rho), "rhodot": ("scalar", np.zeros(n)), "p": ("scalar", np.zeros(n)),
              "v": ("vector", case.v), "vdot": ("vector", np.zeros((n, case.dim)))}
    consts = {"mass": case.mass, "c": case.c0, "rho0": case.rho0, "dt": case.dt,
              "g": tuple(case.g[:case.dim])}
    return fields, consts


@pytest.mark.parametrize("fp32", [False, True])
def test_appendix_a_equations_equal_the_example_1a_oracle(fp32):
    case = C.paper_box(2, (20, 14), (10, 8), (C.BC_SYMMETRIC, C.BC_SYMMETRIC), seed=5, v_sigma=0.3,
                       rho_sigma=0.004, jitter=0.05)
    case.alpha = 0.1
    fields, consts = appendix_a_system(case)
    lo = LO.LawOracle(case, fields, consts, APPENDIX_A, fp32_neighbours=fp32)
    lo.step(4)
    ref = O.bc_step(O.bc_params(case, fp32=fp32), case.r, case.v, case.rho, case.kind, case.id, 4)
    assert ref.rc == 0
    np.testing.assert_allclose(lo.r, ref.r, rtol=0, atol=1e-12 * np.abs(ref.r).max())
    np.testing.assert_allclose(lo.fields["v"].a[:, :2], ref.v, rtol=0, atol=1e-10 * np.abs(ref.v).max())
    np.testing.assert_allclose(lo.fields["rho"].a, ref.rho, rtol=1e-13)
    np.testing.assert_allclose(lo.fields["p"].a, ref.p, rtol=0, atol=1e-9 * np.abs(ref.p).max())


def _offsets(R_over_dx):
    K = int(math.ceil(R_over_dx)) + 1
    ax = np.arange(-K, K + 1)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3).astype(float)
    d = np.sqrt((g * g).sum(1))
    keep = (d < R_over_dx) & (d > 0)
    return g[keep], d[keep]


def test_lattice_sums_and_plane_waves():
    n_side = 15
    case = C.periodic_cube(n_side, seed=2)
    dx, h = case.dx, case.h
    L = n_side * dx
    kv = 2.0 * math.pi * np.array([1.0, 1.0, 0.0]) / L     # |k| h = 0.65
    A = np.sin(case.r @ kv + 0.2)
    fields = {"A": ("scalar", A), "one": ("scalar", np.ones(case.n)), "cnt": ("scalar", np.zeros(case.n)),
              "Sv": ("scalar", np.zeros(case.n)), "S2": ("scalar", np.zeros(case.n)),
              "LA": ("scalar", np.zeros(case.n)), "GA": ("vector", np.zeros((case.n, 3))),
              "DA": ("vector", np.zeros((case.n, 3)))}
    consts = {"m": case.mass, "rho0": case.rho0}
    eqs = ["cnt = sum_j(1 + 0*d_ij)",
           "Sv = sph_S(one, m, rho0)",
           "S2 = sum_j(one_j*m/rho0*W_ij) + one*m/rho0*W0",
           "LA = sph_L(A, m, rho0)",
           "GA = sph_G(A, m, rho0)",
           "DA = sph_D(A, m, rho0)"]
    W0 = O.alpha_D(3, h)
    consts["W0"] = W0
    lo = LO.LawOracle(case, fields, consts, eqs)
    lo.step(1)
    f = lo.fields
    off, d = _offsets(2.0 * h / dx)
    assert off.shape[0] == 32
    np.testing.assert_array_equal(f["cnt"].a, 32.0)
    V = dx ** 3
    lat = (W0 + sum(O.W(3, h, x * dx) for x in d)) * V
    np.testing.assert_allclose(f["Sv"].a, lat, rtol=1e-13)
    np.testing.assert_allclose(f["S2"].a, f["Sv"].a, rtol=1e-13)
    # lattice coefficients (dW/dr from the pinned kernel derivative)
    dW = np.array([O.dWdr(3, h, x * dx) for x in d])
    kd = (off * dx) @ kv
    lam_L = float(np.sum(2.0 * V * (1.0 - np.cos(kd)) * dW / (d * dx)))
    np.testing.assert_allclose(f["LA"].a, lam_L * A, rtol=0, atol=1e-9 * abs(lam_L))
    assert lam_L < 0                                  # -|k|^2 in the continuum
    assert abs(lam_L / -(kv @ kv) - 1.0) < 0.1          # the continuum limit, to O((k h)^2)
    # gradient (both forms): with d = r_j - r_i and grad_i W = -W'(|d|) d/|d|,
    # cos(k.x + 0.2) times g = -V sum_d sin(k.d) W'(|d|) d/|d| (~ k: W' < 0)
    gvec = -V * np.sum((np.sin(kd) * dW / (d * dx))[:, None] * (off * dx), axis=0)
    cosx = np.cos(case.r @ kv + 0.2)
    for name in ("GA", "DA"):
        np.testing.assert_allclose(f[name].a, cosx[:, None] * gvec[None, :], rtol=0,
                                   atol=1e-9 * np.abs(gvec).max())
    np.testing.assert_allclose(gvec, kv, rtol=0.1, atol=0.1 * np.linalg.norm(kv))


SOCIAL_FORCE = ["vdot = (v0*e0 - v)/tau + sum_j((A*exp((R_i + R_j - d_ij)/B) + k*max(R_i + R_j - d_ij, 0)"
                " - cA)*r_ij/d_ij)/m",
                "v = euler(v, vdot, dt)",
                "r = euler(r, v, dt)"]
SF_CONSTS = {"v0": 1.3, "tau": 0.5, "A": 2000.0, "B": 0.08, "k": 1.2e5, "cA": 15.0, "dt": 0.005}


def _people(r, v, e0, m, bc, nc=(6, 4), h=0.6):
    """A few people in a 2D box of nc cells of edge 2h."""
    c = C.paper_box(2, (1, 1), nc, bc, seed=1, dx=h / 1.1)
    n = r.shape[0]
    c.r, c.v = np.asarray(r, float), np.asarray(v, float)
    c.kind = np.zeros(n, np.uint8)
    c.id = np.arange(n, dtype=np.uint32)[::-1].copy()
    c.n_fluid = n
    R = 0.002 * np.asarray(m, float) + 0.15
    fields = {"v": ("vector", c.v), "vdot": ("vector", np.zeros((n, 2))), "e0": ("vector", np.asarray(e0, float)),
              "R": ("scalar", R), "m": ("scalar", np.asarray(m, float))}
    return c, fields, R


def _sf_pair_force(Ri, Rj, d, c=SF_CONSTS):
    """Magnitude along r_ij/d_ij of the pair term of Eq. social_force_model:
    contact g(x) = max(x, 0) (Helbing's body force; the printed k(R_ij - d_ij)
    read as acting only in contact), minus the attraction c_ij."""
    x = Ri + Rj - d
    return c["A"] * math.exp(x / c["B"]) + c["k"] * max(x, 0.0) - c["cA"]


def test_social_force_two_people_closed_form():
    """Two people 0.55 m apart (in contact: R_i + R_j = 0.61 m) in an open
    box: the oracle's accelerations and one semi-implicit Euler step equal
    Eq. social_force_model written out by hand, and the pair forces are
    equal and opposite (different masses)."""
    CUT = C.BC_CUTOFF
    r = np.array([[3.0, 2.0], [3.0 + 0.55 * 0.8, 2.0 + 0.55 * 0.6]])
    v = np.array([[0.2, 0.1], [-0.3, 0.05]])
    e0 = np.array([[1.0, 0.0], [0.0, 1.0]])
    m = np.array([70.0, 90.0])
    case, fields, R = _people(r, v, e0, m, (CUT, CUT))
    lo = LO.LawOracle(case, fields, SF_CONSTS, SOCIAL_FORCE)
    lo.step(1)
    c = SF_CONSTS
    d = 0.55
    n01 = (r[0] - r[1]) / d                      # r_ij / d_ij for i = 0
    F = _sf_pair_force(R[0], R[1], d)
    assert F > 1000.0                            # contact: the body force dominates
    a0 = (c["v0"] * e0[0] - v[0]) / c["tau"] + F * n01 / m[0]
    a1 = (c["v0"] * e0[1] - v[1]) / c["tau"] - F * n01 / m[1]
    np.testing.assert_allclose(lo.fields["vdot"].a[:, :2], [a0, a1], rtol=1e-13)
    drive = (c["v0"] * e0 - v) / c["tau"]
    f = (lo.fields["vdot"].a[:, :2] - drive) * m[:, None]
    np.testing.assert_allclose(f[0], -f[1], rtol=1e-13)       # Newton's third law
    v1 = v + c["dt"] * np.array([a0, a1])
    np.testing.assert_allclose(lo.fields["v"].a[:, :2], v1, rtol=1e-13)
    np.testing.assert_allclose(lo.r, r + c["dt"] * v1, rtol=1e-14)   # moved with the new v


def test_social_force_out_of_contact_and_beyond_the_radius():
    """1.0 m apart (no contact): only the exponential and the attraction act;
    1.3 m apart (beyond 2h = 1.2 m): no pair term at all."""
    CUT = C.BC_CUTOFF
    for d, expect_pair in ((1.0, True), (1.3, False)):
        r = np.array([[3.0, 2.0], [3.0 + d, 2.0]])
        v = np.zeros((2, 2))
        e0 = np.array([[1.0, 0.0], [1.0, 0.0]])
        m = np.array([60.0, 80.0])
        case, fields, R = _people(r, v, e0, m, (CUT, CUT))
        lo = LO.LawOracle(case, fields, SF_CONSTS, SOCIAL_FORCE[:1])
        lo.step(1)
        F = _sf_pair_force(R[0], R[1], d) if expect_pair else 0.0
        a0 = np.array([SF_CONSTS["v0"] / SF_CONSTS["tau"] - F / m[0], 0.0])
        np.testing.assert_allclose(lo.fields["vdot"].a[0, :2], a0, rtol=1e-13, atol=1e-12)
        if expect_pair:
            assert F < 0.0                        # net attraction out of contact with cA = 15 N


def test_wall_mirror_image_and_periodic_wrap():
    """A person 0.2 m from a symmetric wall meets their own mirror image
    0.4 m away (same radius), pushed straight off the wall; vector fields of
    the image are reflected (sum_j(v_j) of a lone person near the wall is
    (vx, -vy)); two people 0.3 m from either periodic end interact across
    it at distance 0.6 m."""
    CUT, SYM, PER = C.BC_CUTOFF, C.BC_SYMMETRIC, C.BC_PERIODIC
    r = np.array([[3.0, 0.2]])
    v = np.array([[0.4, -0.25]])
    e0 = np.array([[1.0, 0.0]])
    m = np.array([75.0])
    case, fields, R = _people(r, v, e0, m, (CUT, SYM))
    fields["s"] = ("vector", np.zeros((1, 2)))
    fields["q"] = ("scalar", np.zeros(1))
    eqs = [SOCIAL_FORCE[0], "s = sum_j(v_j)", "q = sum_j(dot(r_ij, vec(0, 1))*m_j/m_i)"]
    lo = LO.LawOracle(case, fields, SF_CONSTS, eqs)
    lo.step(1)
    F = _sf_pair_force(R[0], R[0], 0.4)
    a = (SF_CONSTS["v0"] * e0[0] - v[0]) / SF_CONSTS["tau"] + np.array([0.0, F / m[0]])
    np.testing.assert_allclose(lo.fields["vdot"].a[0, :2], a, rtol=1e-13)
    np.testing.assert_allclose(lo.fields["s"].a[0, :2], [0.4, 0.25], rtol=1e-15)
    np.testing.assert_allclose(lo.fields["q"].a[0], 0.4, rtol=1e-14)     # r_ij = r_i - r_image points off the wall
    # periodic along x: ncell 6 of edge 1.2 -> L = 7.2
    L = 6 * 1.2
    r = np.array([[0.3, 2.0], [L - 0.3, 2.0]])
    case, fields, R = _people(r, np.zeros((2, 2)), np.array([[1.0, 0.0], [1.0, 0.0]]), np.array([70.0, 70.0]),
                              (PER, CUT))
    fields["q"] = ("scalar", np.zeros(2))
    lo = LO.LawOracle(case, fields, SF_CONSTS, ["q = sum_j(dot(r_ij, vec(1, 0)))"])
    lo.step(1)
    np.testing.assert_allclose(lo.fields["q"].a, [0.6, -0.6], rtol=1e-13)


def test_paper_operator_notation_in_the_oracle():
    """The oracle reads op(A, m, rho, Wp52220, 2*h), sph_D00 / sph_G11 /
    sph_L0 and ^ as the plain forms (identical values), and rejects a radius
    other than 2h."""
    case = C.paper_box(2, (16, 12), (8, 7), (C.BC_SYMMETRIC, C.BC_PERIODIC), seed=9, v_sigma=0.3,
                       rho_sigma=0.004, jitter=0.05)
    n = case.n
    base = {"rho": ("scalar", case.rho), "u": ("vector", case.v), "d": ("scalar", np.zeros(n)),
            "P": ("scalar", np.zeros(n)), "a": ("vector", np.zeros((n, 2))), "L": ("scalar", np.zeros(n))}
    consts = {"m0": case.mass, "c": case.c0, "rho0": case.rho0}
    paper = ["d = 2*sph_D00(u, m0, rho, Wp52220, 2*h) + rho", "P = c^3*d - rho0",
             "a = sph_G11(P, m0, rho, Wp52220, h*2) - 3*sph_A(u, m0, rho, Wp52220, 2*h)",
             "L = sph_L0(rho, m0, rho0, Wp52220, 2*h)"]
    plain = ["d = 2*sph_D(u, m0, rho) + rho", "P = c**3*d - rho0",
             "a = sph_G(P, m0, rho) - 3*sph_A(u, m0, rho)", "L = sph_L(rho, m0, rho0)"]
    x, y = LO.LawOracle(case, base, consts, paper), LO.LawOracle(case, base, consts, plain)
    x.step(1)
    y.step(1)
    for f in ("d", "P", "a", "L"):
        np.testing.assert_array_equal(x.fields[f].a, y.fields[f].a)
    assert np.abs(x.fields["a"].a).max() > 0
    z = LO.LawOracle(case, base, consts, ["d = sph_L0(rho, m0, rho0, Wp52220, 3*h)"])
    with pytest.raises(ValueError):
        z.step(1)


def test_oracle_variables_and_reductions():
    """Variables in the oracle: fmax / fmin / fsum are the numpy reductions
    of the per-particle values, a variable's equation gives one value, an
    elapsed time is the sum of the steps taken, and a field equation reads
    the variable's current value."""
    case = C.paper_box(2, (12, 10), (6, 6), (C.BC_PERIODIC, C.BC_PERIODIC), seed=4, dx=0.01,
                       cs_factor=1.0, jitter=0.1)
    n = case.n
    rng = np.random.default_rng(2)
    c0 = rng.uniform(-1, 1, n)
    fields = {"c": ("scalar", c0), "g": ("scalar", np.zeros(n))}
    consts = {"k": 0.5}
    vs = {"hi": 0.0, "lo": 0.0, "tot": 0.0, "dt": 0.0, "T": 0.0}
    eqs = ["hi = fmax(c*c)", "lo = fmin(c - 1)", "tot = fsum(2*c)", "dt = k/(1 + hi)", "g = c*dt",
           "c = c - dt*c", "T = T + dt"]
    lo = LO.LawOracle(case, fields, consts, eqs, variables=vs)
    lo.step(1)
    c = c0
    hi = float(np.max(c * c))
    assert lo.vars["hi"] == hi and lo.vars["lo"] == float(np.min(c - 1)) and lo.vars["tot"] == float(np.sum(2 * c))
    dt1 = 0.5 / (1 + hi)
    assert lo.vars["dt"] == dt1
    np.testing.assert_array_equal(lo.fields["g"].a, c * dt1)
    c1 = c - dt1 * c
    np.testing.assert_array_equal(lo.fields["c"].a, c1)
    lo.step(1)
    dt2 = 0.5 / (1 + float(np.max(c1 * c1)))
    assert lo.vars["dt"] == dt2 and lo.vars["T"] == dt1 + dt2


def test_oracle_reads_the_own_position():
    """r outside pair sums is the particle's own position: a projection
    equals the coordinate, and a move whose velocity reads r follows the
    closed form r' = r - dt k r."""
    case = C.paper_box(2, (10, 8), (6, 6), (C.BC_CUTOFF, C.BC_CUTOFF), seed=6, jitter=0.2)
    n = case.n
    fields = {"q": ("scalar", np.zeros(n)), "u": ("vector", np.zeros((n, 2)))}
    lo = LO.LawOracle(case, fields, {"k": 0.3, "dt": 0.01},
                      ["q = dot(r, vec(1, 0))", "u = vec(0, 0) - k*r", "r = euler(r, 0*u - k*r, dt)"])
    r0 = lo.r.copy()
    lo.step(1)
    np.testing.assert_array_equal(lo.fields["q"].a, r0[:, 0])
    np.testing.assert_allclose(lo.fields["u"].a[:, :2], -0.3 * r0, rtol=1e-15)
    np.testing.assert_allclose(lo.r, r0 + 0.01 * (-0.3 * r0), rtol=1e-14)


def test_oracle_where():
    """where(c, a, b) in the oracle: a where c != 0 else b, per particle, for
    scalars and vectors."""
    case = C.paper_box(2, (8, 6), (5, 5), (C.BC_CUTOFF, C.BC_CUTOFF), seed=8, jitter=0.2)
    n = case.n
    c = np.where(np.arange(n) % 3 == 0, 0.0, 2.0)
    fields = {"c": ("scalar", c), "x": ("scalar", np.zeros(n)), "u": ("vector", np.zeros((n, 2)))}
    lo = LO.LawOracle(case, fields, {}, ["x = where(c, c + 1, -1)", "u = where(c - 2, vec(1, 2), vec(3, 4))"])
    lo.step(1)
    np.testing.assert_array_equal(lo.fields["x"].a, np.where(c != 0, c + 1, -1))
    np.testing.assert_array_equal(lo.fields["u"].a[:, 0], np.where(c != 2, 1.0, 3.0))
    np.testing.assert_array_equal(lo.fields["u"].a[:, 1], np.where(c != 2, 2.0, 4.0))


def test_oracle_mirror_flag():
    """mirror_ij is 1 exactly for the images seen through a symmetric face:
    a lone person near a wall has one neighbour, its own mirror image."""
    case = C.paper_box(2, (1, 1), (6, 4), (C.BC_CUTOFF, C.BC_SYMMETRIC), seed=1, dx=0.6 / 1.1)
    case.r = np.array([[3.0, 0.2], [3.0, 2.4]])
    case.v = np.zeros((2, 2))
    case.kind = np.zeros(2, np.uint8)
    case.id = np.arange(2, dtype=np.uint32)
    case.n_fluid = 2
    fields = {"w": ("scalar", np.zeros(2)), "c": ("scalar", np.zeros(2))}
    lo = LO.LawOracle(case, fields, {}, ["w = sum_j(mirror_ij + 0*d_ij)", "c = sum_j(1 + 0*d_ij)"])
    lo.step(1)
    np.testing.assert_array_equal(lo.fields["w"].a, [1.0, 0.0])     # the first sees its image only
    np.testing.assert_array_equal(lo.fields["c"].a, [1.0, 0.0])

"""Pins of the oracle's domain boundary treatments (Section 3.2.1), its
Example 1a step in the paper's own form (Section 5.1.1: continuity equation,
linear EOS, viscosity with rho_i, symmetric walls) and its sampling operator
(Section 6), each against something other than the oracle's own formulas:

* brute force over every particle and image code equals the cell search;
* a symmetric or periodic face equals the same system with its images laid
  out as explicit particles in a larger cut-off domain;
* a uniform periodic lattice: neighbour counts and sums are lattice sums
  enumerated here over integer offsets; a plane wave is an eigenvector of
  the sampling operator with the lattice Fourier sum as eigenvalue;
* a linear velocity field: the continuity sum is the divergence times the
  lattice moment (close to 1, the continuum value), zero for a rotation;
* pressure-only forces conserve momentum; the viscosity is repulsive for
  approaching pairs only and carries 1/rho_i (ratio rho_j / rho_i);
* a wall-parallel translation feels nothing (free slip); an approach to a
  wall compresses and is repelled;
* free fall and the periodic shift of a particle leaving the domain;
* a settled hydrostatic column between symmetric walls has the pressure
  slope rho0 g / mu with mu the lattice gradient moment.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1710_08259_gb300 import cases as C

SYM, PER, CUT = C.BC_SYMMETRIC, C.BC_PERIODIC, C.BC_CUTOFF


def _cloud(dim, n, ncell, bc, seed, cs=0.022, h=0.011, margin=0.0):
    """Random particles filling a grid of `ncell` cells of edge cs."""
    rng = np.random.default_rng(seed)
    ext = np.asarray(ncell[:dim], float) * cs
    r = rng.uniform(margin, 1.0, size=(n, dim)) * (ext - margin)
    c = C.paper_box(dim, (1,) * dim, ncell, bc, seed=seed, dx=h / 1.1)
    c.r = r
    c.cs = cs
    c.h = h
    c.v = rng.normal(0.0, 0.3, size=(n, dim))
    c.rho = 1000.0 * (1.0 + rng.normal(0.0, 0.01, size=n))
    c.kind = np.zeros(n, np.uint8)
    c.id = rng.permutation(n).astype(np.uint32)
    c.n_fluid = n
    c.mass = 1000.0 * (h / 1.1) ** dim
    c.c0 = 20.0
    c.dt = 1e-4
    return c


def _same_lists(a, b):
    oa, na, ia = a
    ob, nb, ib = b
    assert np.array_equal(oa, ob)
    assert np.array_equal(na, nb)
    assert np.array_equal(ia, ib)


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("dim,ncell,bc", [
    (2, (4, 3, 1), (SYM, PER, CUT)),
    (2, (1, 2, 1), (PER, SYM, CUT)),
    (2, (3, 3, 1), (CUT, SYM, CUT)),
    (3, (3, 2, 1), (PER, SYM, SYM)),
    (3, (2, 3, 2), (SYM, CUT, PER)),
])
def test_brute_force_equals_cell_search(dim, ncell, bc, fp32):
    c = _cloud(dim, 300 if dim == 2 else 400, ncell, bc, seed=17 + dim)
    # adversarial: particles exactly on cell faces and on the domain faces
    c.r[:6, 0] = np.array([0.0, c.cs, 2 * c.cs, 0.0, c.cs * 0.5, 0.0])[:6] % (ncell[0] * c.cs)
    c.r[6:9, -1] = 0.0
    p = O.bc_params(c, fp32=fp32)
    brute = O.bc_neighbours(p, c.r, c.id, method="brute")
    cells = O.bc_neighbours(p, c.r, c.id, method="cells")
    _same_lists(brute, cells)
    assert brute[1].size > 0
    # images actually occur, and only on the axes that have them
    codes = brute[2]
    for k in range(dim):
        t = (codes // 3 ** k) % 3
        if bc[k] == CUT:
            assert not np.any(t)
        else:
            assert np.any(t == 1) and np.any(t == 2)


def _explicit_images(c, with_codes=False):
    """The system plus its images as explicit particles in a cut-off domain
    three times larger; returns (case, index of the real copy of each
    particle)."""
    dim = c.dim
    L = [c.ncell[k] * c.cs for k in range(3)]
    reps = []
    for code in range(3 ** dim):
        t = [(code // 3 ** k) % 3 for k in range(dim)]
        if any(t[k] and c.bc[k] == CUT for k in range(dim)):
            continue
        r = c.r.copy()
        v = c.v.copy()
        for k in range(dim):
            if t[k] == 0:
                continue
            if c.bc[k] == PER:
                r[:, k] = r[:, k] - L[k] if t[k] == 1 else r[:, k] + L[k]
            else:
                w = 0.0 if t[k] == 1 else L[k]
                r[:, k] = 2.0 * w - r[:, k]
                v[:, k] = -v[:, k]
        reps.append((code, r, v))
    n = c.n
    big = c.copy()
    big.r = np.concatenate([x[1] for x in reps])
    big.v = np.concatenate([x[2] for x in reps])
    big.rho = np.tile(c.rho, len(reps))
    big.kind = np.tile(c.kind, len(reps))
    big.id = np.arange(big.r.shape[0], dtype=np.uint32)
    big.n_fluid = big.r.shape[0]
    big.dom_min = tuple(-L[k] if k < dim else 0.0 for k in range(3))
    big.ncell = tuple(3 * c.ncell[k] if k < dim else 1 for k in range(3))
    big.bc = (CUT, CUT, CUT)
    real = [i for i, x in enumerate(reps) if x[0] == 0][0]
    return big, np.arange(real * n, (real + 1) * n)


@pytest.mark.parametrize("dim,ncell,bc", [
    (2, (4, 3, 1), (SYM, PER, CUT)),
    (2, (3, 3, 1), (SYM, SYM, CUT)),
    (3, (3, 2, 1), (PER, SYM, SYM)),
    (3, (2, 2, 2), (SYM, SYM, SYM)),
])
def test_faces_equal_explicit_images(dim, ncell, bc):
    c = _cloud(dim, 250 if dim == 2 else 300, ncell, bc, seed=31 + dim)
    big, sel = _explicit_images(c)
    # continuity (eq1, eq2): from the initial fields only
    p = O.bc_params(c)
    pb = O.bc_params(big)
    ev = O.bc_eval(p, c.r, c.v, c.rho, c.kind, c.id)
    eb = O.bc_eval(pb, big.r, big.v, big.rho, big.kind, big.id)
    np.testing.assert_allclose(ev.rho, eb.rho[sel], rtol=1e-12, atol=0)
    assert ev.n_pairs > 0
    # momentum (eq3..eq5) at dt = 0, where every explicit copy keeps the
    # density and pressure of its particle (with dt > 0 a copy at the edge
    # of the larger domain would miss images of its own)
    p0 = O.bc_params(c, dt=0.0)
    pb0 = O.bc_params(big, dt=0.0)
    ev = O.bc_eval(p0, c.r, c.v, c.rho, c.kind, c.id)
    eb = O.bc_eval(pb0, big.r, big.v, big.rho, big.kind, big.id)
    np.testing.assert_allclose(ev.p, eb.p[sel], rtol=0, atol=1e-9 * np.abs(eb.p[sel]).max())
    amax = np.abs(eb.a[sel]).max()
    np.testing.assert_allclose(ev.a, eb.a[sel], rtol=0, atol=1e-11 * amax)
    # the same for the sampling operator
    rng = np.random.default_rng(5)
    A = rng.uniform(-1, 1, c.n)
    m = rng.uniform(0.5, 1.5, c.n) * c.mass
    S, _, _ = O.bc_sample(p, c.r, c.id, A, m, c.rho)
    reps = big.r.shape[0] // c.n
    Sb, _, _ = O.bc_sample(pb, big.r, big.id, np.tile(A, reps), np.tile(m, reps), big.rho)
    np.testing.assert_allclose(S, Sb[sel], rtol=1e-12, atol=1e-12 * np.abs(Sb).max())


def _lattice_offsets(dim, R_over_dx):
    K = int(math.ceil(R_over_dx)) + 1
    ax = np.arange(-K, K + 1)
    g = np.stack(np.meshgrid(*([ax] * dim), indexing="ij"), -1).reshape(-1, dim)
    d = np.sqrt((g.astype(float) ** 2).sum(1))
    return g[d < R_over_dx], d[d < R_over_dx]


@pytest.mark.parametrize("n_side", [3, 6, 7])
@pytest.mark.parametrize("fp32", [False, True])
def test_periodic_lattice_counts_and_sums(n_side, fp32):
    c = C.periodic_cube(n_side, seed=3)
    p = O.bc_params(c, fp32=fp32)
    offs, ids, codes = O.bc_neighbours(p, c.r, c.id)
    off, d = _lattice_offsets(3, 2.0 * c.h / c.dx)
    nlat = off.shape[0] - 1  # offsets within the support, self excluded
    assert nlat == 32
    assert np.all(np.diff(offs) == nlat)
    # A = 1, m / rho = dx^3: every S_i is the lattice sum of dx^3 W
    lat = sum(O.W(3, c.h, float(x) * c.dx) for x in d) * c.dx ** 3
    S, _, pairs = O.bc_sample(p, c.r, c.id, np.ones(c.n), np.full(c.n, c.mass), np.full(c.n, c.rho0))
    np.testing.assert_allclose(S, lat, rtol=1e-13)
    assert pairs == nlat * c.n


@pytest.mark.parametrize("kvec", [(1, 0, 0), (0, 2, 1), (1, 1, 1)])
def test_plane_wave_is_an_eigenvector(kvec):
    n_side = 9
    c = C.periodic_cube(n_side, seed=4)
    L = n_side * c.dx
    k = 2.0 * math.pi * np.asarray(kvec, float) / L
    A = np.sin(c.r @ k + 0.3)
    p = O.bc_params(c)
    S, _, _ = O.bc_sample(p, c.r, c.id, A, np.full(c.n, c.mass), np.full(c.n, c.rho0))
    off, d = _lattice_offsets(3, 2.0 * c.h / c.dx)
    lam = sum(O.W(3, c.h, float(dd) * c.dx) * math.cos(float(np.dot(k, o)) * c.dx)
              for o, dd in zip(off, d)) * c.dx ** 3
    np.testing.assert_allclose(S, lam * A, rtol=0, atol=1e-12)
    assert 0.2 < lam < 1.0


def _lattice_moment(dim, h, dx):
    """mu = -(1/D) sum over lattice offsets of dx^D W'(|d|) |d|: the
    discrete counterpart of -(1/D) int W'(r) r dV = 1."""
    off, d = _lattice_offsets(dim, 2.0 * h / dx)
    s = sum(O.dWdr(dim, h, float(x) * dx) * float(x) * dx for x in d if x > 0)
    return -s * dx ** dim / dim


@pytest.mark.parametrize("G", [
    [[0.7, 0.2], [-0.5, -0.3]],    # general field, divergence 0.4
    [[0.0, 0.9], [-0.9, 0.0]],     # rotation, divergence 0
    [[-1.0, 0.0], [0.0, -0.6]],    # compression
])
def test_continuity_of_a_linear_field(G):
    G = np.asarray(G)
    c = C.paper_box(2, (26, 26), (12, 12), (CUT, CUT), seed=8, dx=0.01, shuffle_ids=True,
                    g=(0.0, 0.0))
    c.v = c.r @ G.T
    p = O.bc_params(c)
    ev = O.bc_eval(p, c.r, c.v, c.rho, c.kind, c.id)
    D = (c.rho - ev.rho) / (c.dt * c.rho)   # rho' = rho - dt rho D
    mu = _lattice_moment(2, c.h, c.dx)
    assert abs(mu - 1.0) < 0.05
    lo, hi = 0.5 * c.dx + 2 * c.h + 1e-9, (26 - 0.5) * c.dx - 2 * c.h - 1e-9
    inner = np.all((c.r > lo) & (c.r < hi), axis=1)
    assert inner.sum() > 100
    np.testing.assert_allclose(D[inner], mu * np.trace(G), rtol=0, atol=1e-9 * max(1.0, abs(np.trace(G))))
    # the sign: compression raises the density
    if np.trace(G) < 0:
        assert np.all(ev.rho[inner] > c.rho[inner])


def test_pressure_forces_conserve_momentum():
    c = _cloud(2, 400, (5, 5, 1), (CUT, CUT, CUT), seed=41)
    c.v[:] = 0.0
    p = O.bc_params(c, g=(0.0, 0.0, 0.0))
    ev = O.bc_eval(p, c.r, c.v, c.rho, c.kind, c.id)
    P = (c.mass * ev.a).sum(0)
    scale = (c.mass * np.abs(ev.a)).sum()
    assert scale > 0
    assert np.all(np.abs(P) < 1e-13 * scale)
    # and p is linear in rho with slope c^2 (p = 0 at rho0): eq3
    assert np.allclose(np.polyfit(ev.rho - c.rho0, ev.p, 1), [c.c0 ** 2, 0.0], rtol=1e-12, atol=1e-9)


def _pair(rho1, rho2, v1, v2, visc=0.1):
    c = C.paper_box(2, (1, 1), (6, 6), (CUT, CUT), seed=1, dx=0.01, g=(0.0, 0.0), visc=visc,
                    shuffle_ids=False)
    x0 = 2.5 * c.cs
    c.r = np.array([[x0, x0], [x0 + 1.3 * c.dx, x0 + 0.4 * c.dx]])
    c.v = np.array([v1, v2], float)
    c.rho = np.array([rho1, rho2], float)
    c.kind = np.zeros(2, np.uint8)
    c.id = np.arange(2, dtype=np.uint32)
    c.n_fluid = 2
    p = O.bc_params(c, dt=0.0)       # dt = 0: rho' = rho, only the momentum sum acts
    return c, O.bc_eval(p, c.r, c.v, c.rho, c.kind, c.id).a


def test_viscosity_of_the_paper():
    rho1, rho2 = 1003.0, 996.0
    c, a0 = _pair(rho1, rho2, [0, 0], [0, 0])
    r12 = c.r[0] - c.r[1]
    # approaching: 1 moves towards 2
    _, a = _pair(rho1, rho2, -r12 / np.linalg.norm(r12), [0, 0])
    av = a - a0
    assert np.dot(av[0], r12) > 0 and np.dot(av[1], -r12) > 0          # repulsive
    cross = av[0, 0] * r12[1] - av[0, 1] * r12[0]          # parallel to r_12
    assert abs(cross) < 1e-12 * np.abs(av).max() * np.linalg.norm(r12)
    # 1/rho_i in Pi_ij: the pair terms differ by rho_j / rho_i
    np.testing.assert_allclose(-av[0] / av[1], rho2 / rho1, rtol=1e-12)
    # linear in the coefficient
    _, a2 = _pair(rho1, rho2, -r12 / np.linalg.norm(r12), [0, 0], visc=0.2)
    c0_, a20 = _pair(rho1, rho2, [0, 0], [0, 0], visc=0.2)
    np.testing.assert_allclose(a2 - a20, 2.0 * av, rtol=1e-12)
    # separating: no viscosity
    _, a = _pair(rho1, rho2, r12 / np.linalg.norm(r12), [0, 0])
    np.testing.assert_allclose(a, a0, rtol=0, atol=0)


def test_continuity_weights_are_m_over_rho_j():
    # two particles: D_1 = (m/rho_2) X and D_2 = (m/rho_1) X with the same
    # X = (v_2 - v_1) . grad_1 W_12, so D_1 / D_2 = rho_1 / rho_2
    rho1, rho2 = 1020.0, 985.0
    c, _ = _pair(rho1, rho2, [0, 0], [0, 0])
    r12 = c.r[0] - c.r[1]
    c.v = np.array([-r12, r12]) / np.linalg.norm(r12)    # approaching
    ev = O.bc_eval(O.bc_params(c), c.r, c.v, c.rho, c.kind, c.id)
    D = (c.rho - ev.rho) / (c.dt * c.rho)
    assert D[0] < 0 and D[1] < 0                          # converging flow
    np.testing.assert_allclose(D[0] / D[1], rho1 / rho2, rtol=1e-12)


def test_sampling_weights_are_m_over_rho_j():
    # A_j = rho_j / m_j makes every weight 1: S_i = sum_j W_ij, the same
    # lattice sum for every particle of a periodic lattice whatever the
    # densities are
    c = C.periodic_cube(6, seed=12, rho_sigma=0.05)
    m = c.extra["m"] * (1.0 + 0.1 * np.random.default_rng(2).uniform(-1, 1, c.n))
    S, _, _ = O.bc_sample(O.bc_params(c), c.r, c.id, c.rho / m, m, c.rho)
    off, d = _lattice_offsets(3, 2.0 * c.h / c.dx)
    lat = sum(O.W(3, c.h, float(x) * c.dx) for x in d)
    np.testing.assert_allclose(S, lat, rtol=1e-13)


def test_wall_parallel_translation_is_free_slip():
    # a row of particles next to a symmetric floor, all moving along it
    c = C.paper_box(2, (12, 2), (8, 6), (CUT, SYM), seed=2, dx=0.01, g=(0.0, 0.0),
                    offset=(2.0, 0.0), v_sigma=0.0, shuffle_ids=False)
    c.v[:] = [1.5, 0.0]
    p = O.bc_params(c)
    ev = O.bc_eval(p, c.r, c.v, c.rho, c.kind, c.id)
    np.testing.assert_array_equal(ev.rho, c.rho)   # no compression at all
    res = O.bc_step(p, c.r, c.v, c.rho, c.kind, c.id, nsteps=20)
    assert res.rc == 0
    np.testing.assert_allclose(res.v[:, 0], 1.5, rtol=0, atol=1e-12)
    np.testing.assert_allclose(res.v[:, 1], 0.0, rtol=0, atol=1e-12)


def test_wall_approach_compresses_and_repels():
    c = C.paper_box(2, (1, 1), (6, 6), (CUT, SYM), seed=2, dx=0.01, g=(0.0, 0.0), shuffle_ids=False)
    c.r = np.array([[2.5 * c.cs, 0.6 * c.h]])
    c.v = np.array([[0.0, -1.0]])            # towards the floor
    p = O.bc_params(c)
    ev = O.bc_eval(p, c.r, c.v, c.rho, c.kind, c.id)
    assert ev.rho[0] > c.rho[0]               # compression by the own image
    assert ev.a[0, 1] > 0 and ev.a[0, 0] == 0.0
    # at rest with rho > rho0 the own image pushes the particle away
    c.v[:] = 0.0
    c.rho[:] = 1010.0
    ev = O.bc_eval(p, c.r, c.v, c.rho, c.kind, c.id)
    assert ev.a[0, 1] > 0 and ev.a[0, 0] == 0.0
    assert ev.n_pairs == 1                    # the image is the only neighbour


def test_free_fall_and_periodic_shift():
    c = C.paper_box(2, (1, 1), (10, 40), (PER, CUT), seed=2, dx=0.01, g=(0.0, -9.81), shuffle_ids=False)
    L = c.ncell[0] * c.cs
    # two isolated particles, one leaving through each periodic face
    r0 = np.array([[L - 0.3 * c.cs, 30.0 * c.cs], [0.3 * c.cs, 10.0 * c.cs]])
    v0 = np.array([[2.0, 0.5], [-2.0, 0.25]])
    c.r = r0.copy()
    c.v = v0.copy()
    c.rho = np.full(2, c.rho0)
    c.kind = np.zeros(2, np.uint8)
    c.id = np.arange(2, dtype=np.uint32)
    c.n_fluid = 2
    p = O.bc_params(c)
    n = 100
    res = O.bc_step(p, c.r, c.v, c.rho, c.kind, c.id, nsteps=n)
    assert res.rc == 0
    dt, g = c.dt, np.array([0.0, -9.81])
    np.testing.assert_allclose(res.v, v0 + n * dt * g, rtol=1e-13)
    rexp = r0 + n * dt * v0 + dt * dt * g * n * (n + 1) / 2
    assert rexp[0, 0] > L and rexp[1, 0] < 0.0   # each crossed a periodic face once
    np.testing.assert_allclose(res.r, [[rexp[0, 0] - L, rexp[0, 1]], [rexp[1, 0] + L, rexp[1, 1]]],
                               rtol=1e-12)
    np.testing.assert_array_equal(res.rho, c.rho)
    # leaving through a cut-off face is an error
    c2 = c.copy()
    c2.bc = (CUT, CUT, CUT)
    res2 = O.bc_step(O.bc_params(c2), c2.r, c2.v, c2.rho, c2.kind, c2.id, nsteps=n)
    assert res2.rc == -1


def test_hydrostatic_column_between_symmetric_walls():
    dx = 0.01
    nxp, nyp = 16, 24
    h = 1.1 * dx
    ncx = 7
    cs = nxp * dx / ncx
    c = C.paper_box(2, (nxp, nyp), (ncx, 21), (SYM, SYM), seed=9, dx=dx, cs_factor=cs / (2 * h),
                    visc=0.4, shuffle_ids=False)
    H = nyp * dx
    c.c0 = 10.0 * math.sqrt(2.0 * 9.81 * H)
    c.dt = 0.2 * c.h / c.c0
    p = O.bc_params(c)
    res = O.bc_step(p, c.r, c.v, c.rho, c.kind, c.id, nsteps=6000)
    assert res.rc == 0
    r, v, rho = res.r, res.v, res.rho
    slopes = []
    for _ in range(8):
        res = O.bc_step(p, r, v, rho, c.kind, c.id, nsteps=125)
        r, v, rho = res.r, res.v, res.rho
        top = r[:, 1].max()
        sel = (r[:, 1] > 2 * h) & (r[:, 1] < top - 3 * h)
        slopes.append(np.polyfit(top - r[sel, 1], res.p[sel], 1)[0])
    slope = float(np.mean(slopes))
    mu = _lattice_moment(2, h, dx)
    expect = c.rho0 * 9.81 / mu
    assert abs(slope / expect - 1.0) < 0.03, (slope, expect)
    assert np.abs(v).max() < 0.05 * math.sqrt(9.81 * H)

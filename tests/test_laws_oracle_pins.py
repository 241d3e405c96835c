"""Pins of the interaction-law oracle (oracle/laws_oracle.py), which
evaluates equation systems written for the GPU law compiler in FP64:

* the equations of Appendix A evaluated by it equal the Example 1a oracle
  written separately in C (sph_oracle_bc.c), step after step;
* on a uniform periodic lattice: sum_j(1) counts the 32 lattice neighbours,
  sph_S of a constant is the lattice sum, and a plane wave A = sin(k . x) is
  an eigenvector of sph_L, and sph_G / sph_D map it to cos(k . x) times a
  vector, with eigenvalues and coefficients from lattice sums over integer
  offsets (computed here, not by the oracle);
* sph_S written as sum_j(...) plus the self term equals sph_S.
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

"""Pins against the values the paper prints (tests/golden/*.txt, each file
citing its passage): the Wendland normalisation of Section 5.1.1, the
constants, domain and particle grid of Example 1a (Section 5.1.1, Appendix
A), the particle damper of Example 2 (Section 5.2, its parameter table), the
person size law of the social force example and the benchmark sizes of
Section 6.  The oracle and the input generators must reproduce them."""
import math
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1710_08259_gb300 import cases as C

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name, **env):
    """key = value lines ('#' comments); values are numbers, expressions in
    the paper's notation (juxtaposition multiplies, ^ raises, pi) over
    earlier keys and env, tuples, or bare words."""
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, expr = (s.strip() for s in line.split("=", 1))
        py = expr.replace("^", "**")
        py = re.sub(r"(\d)\s*(?![eE][-+]?\d)([A-Za-z(])", r"\1*\2", py)   # (not 2.06e6)
        py = re.sub(r"([A-Za-z0-9_)])\s+([A-Za-z(])", r"\1*\2", py)
        ns = {"pi": math.pi, **env, **vals}
        try:
            vals[key] = eval(py, {"__builtins__": {}}, ns)
        except NameError:
            vals[key] = tuple(w.strip() for w in expr.split(","))
    return vals


def test_wendland_normalisation():
    g = _load("wendland_kernel.txt")
    h = 0.37
    assert O.alpha_D(1, h) * h == pytest.approx(g["alpha_1_h1"], rel=1e-15)
    assert O.alpha_D(2, h) * h ** 2 == pytest.approx(g["alpha_2_h2"], rel=1e-15)
    assert O.alpha_D(3, h) * h ** 3 == pytest.approx(g["alpha_3_h3"], rel=1e-15)


def test_example_1a_case():
    g = _load("example_1a.txt")
    case = C.example_1a(1)
    assert case.rho0 == g["rho0"] and case.h == g["h"] and case.c0 == g["c"] and case.dt == g["dt"]
    assert case.dx == pytest.approx(g["dx"], rel=1e-15)
    assert case.mass == pytest.approx(g["mass"], rel=1e-15)
    assert tuple(case.g[:2]) == g["g"]
    assert case.cs == g["cell_size"]
    assert tuple(case.ncell[:2]) == tuple(int(round(x)) for x in g["cells"])
    assert g["boundary"] == ("symmetric", "symmetric") and tuple(case.bc[:2]) == (C.BC_SYMMETRIC,) * 2
    assert case.alpha == g["viscosity"]
    # the fluid grid: spacing dx inside the 7 m x 4 m block from the origin
    bx, by = g["fluid_block"]
    x, y = case.r[:, 0], case.r[:, 1]
    assert x.min() > 0 and x.max() < bx and y.min() > 0 and y.max() < by
    assert case.n_fluid == int(bx // case.dx) * int(by // case.dx)
    xs = np.unique(np.round(x, 9))
    assert np.allclose(np.diff(xs), case.dx)


def test_example_2_case():
    g = _load("example_2.txt")
    case = C.dem_damper()
    assert case.n == g["N"]
    np.testing.assert_array_equal(case.rho, g["R"])          # radii
    np.testing.assert_allclose(case.extra["m"], g["rho"] * 4.0 / 3.0 * math.pi * g["R"] ** 3, rtol=1e-15)
    ex = case.extra
    assert (ex["E"], ex["nu"], ex["tank_M"], ex["tank_S"], ex["z0"]) == (g["E"], g["nu"], g["M"], g["S"], g["z0"])
    assert tuple(case.g) == (0.0, 0.0, g["g"])
    for k in range(3):
        assert case.ncell[k] * case.cs == pytest.approx(g["L"], rel=1e-12)   # the domain is the tank's interior
    # the oracle's tank oscillator has the printed frequency: gamma^2 = S / M
    p = O.dem_params(case)
    assert p.tank_S / p.tank_M == pytest.approx(g["S"] / g["M"], rel=1e-15)


def test_social_force_sizes():
    g = _load("social_force.txt")
    case, fields, consts = C.social_force_crowd(400, seed=3)
    m = fields["m"][1]
    R = fields["R"][1]
    assert m.min() >= g["mass_min"] and m.max() <= g["mass_max"]
    np.testing.assert_allclose(R, g["radius_per_kg"] * m + g["radius_offset"], rtol=1e-15)


def test_sampling_benchmark_sizes():
    g = _load("sampling_benchmark.txt")
    side = round(g["peak_n"] ** (1 / 3))
    case = C.periodic_cube(side, seed=1)
    assert case.n == g["peak_n"] and side ** 3 == g["peak_n"]
    assert tuple(case.bc) == (C.BC_PERIODIC,) * 3

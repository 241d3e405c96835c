"""The interaction-law compiler on the CPU: parsing, typing and code
generation, and that nvcc compiles the generated source (no GPU needed)."""
import os

import pytest

from paper_1710_08259_gb300 import laws as L

KINDS = {"rho": "S", "rhodot": "S", "p": "S", "v": "V", "vdot": "V", "R": "S", "m": "S", "e0": "V"}
CONSTS = {"mass": 0.05, "c": 50.0, "rho0": 1000.0, "dt": 1e-3, "g": (0.0, -9.81), "A": 2000.0, "B": 0.08}


def _eq(t, k=0, dim=2):
    return L.parse_equation(t, k, KINDS, CONSTS, dim)


def test_kinds_and_fusion():
    e = _eq("vdot = -1/rho*sph_G(p, mass, rho) + 0.1*c*h*sph_A(v, mass, rho) + g")
    assert e.kind == "pair" and e.rhs_kind == "V" and len(e.accs) == 2   # two sums, one kernel
    assert _eq("rho = euler(rho, rhodot, dt)").kind == "local"
    assert _eq("r = euler(r, v, dt)").kind == "move"
    assert _eq("rhodot = -rho*sph_D(v, mass, rho)").rhs_kind == "S"      # divergence of a vector
    assert _eq("vdot = sph_D(p, mass, rho)").rhs_kind == "V"             # gradient of a scalar
    e = _eq("vdot = sum_j(A*exp((R_i + R_j - d_ij)/B)*r_ij/d_ij)/m")
    assert e.kind == "pair" and "R" in e.reads and "m" in e.reads


@pytest.mark.parametrize("bad", ["rho = rho + q", "rho = v", "v = sum_j(rho)", "rho = sph_D(rho, mass, rho)",
                                 "r = r + v", "rho = sum_j(sum_j(W_ij))", "rho = r_ij", "x = 1",
                                 "v = v*v", "rho = rho**v"])
def test_rejected(bad):
    with pytest.raises((L.LawError, SyntaxError)):
        _eq(bad)


def test_generated_source_compiles(tmp_path):
    os.environ["SPH_LAW_CACHE"] = str(tmp_path)
    try:
        eqs = [_eq(t, k) for k, t in enumerate([
            "rhodot = -rho*sph_D(v, mass, rho)", "rho = euler(rho, rhodot, dt)", "p = c**2*(rho - rho0)",
            "vdot = -1/rho*sph_G(p, mass, rho)", "vdot = vdot + 0.1*c*h*sph_A(v, mass, rho) + g",
            "v = euler(v, vdot, dt)", "r = euler(r, v, dt)"])]
        src, layouts = L.generate(eqs, KINDS, 2, True)
        assert src.count("__global__") == 7 and src.count('extern "C"') == 7
        so = L.compile_source(src)
        assert os.path.exists(so)
        assert L.compile_source(src) == so                    # cached
    finally:
        del os.environ["SPH_LAW_CACHE"]

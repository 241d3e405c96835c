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
                                 "v = v*v", "rho = rho**v", "rho = sum_j(dot(r, r_ij))",
                                 "rho = sph_S(r, mass, rho)"])
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
        src, groups = L.generate(eqs, KINDS, CONSTS, 2, True)
        assert src.count("__global__") == 2 and src.count('extern "C"') == 2
        so = L.compile_source(src)
        assert os.path.exists(so)
        assert L.compile_source(src) == so                    # cached
    finally:
        del os.environ["SPH_LAW_CACHE"]


APPENDIX_A = ["rhodot = -rho*sph_D(v, mass, rho)", "rho = euler(rho, rhodot, dt)", "p = c**2*(rho - rho0)",
              "vdot = -1/rho*sph_G(p, mass, rho)", "vdot = vdot + 0.1*c*h*sph_A(v, mass, rho) + g",
              "v = euler(v, vdot, dt)", "r = euler(r, v, dt)"]


def test_fusion_groups_and_liveness():
    """Appendix A fuses into two kernels: the continuity sum with the density
    update and the EOS, then (the pressure sums read the new rho and p) the
    momentum sums with the velocity update and the move.  At the rebuild
    before the first kernel only rho and v are read before written."""
    eqs = [_eq(t, k) for k, t in enumerate(APPENDIX_A)]
    g = L.group_equations(eqs)
    assert [[e.index for e in x.eqs] for x in g] == [[0, 1, 2], [3, 4, 5, 6]]
    src, g = L.generate(eqs, KINDS, CONSTS, 2, True)
    assert g[0].writes == ["p", "rho", "rhodot"] and g[0].reads == ["rho", "v"]
    assert g[1].writes == ["v", "vdot"] and g[1].reads == ["p", "rho", "v"] and g[1].moves
    assert L.live_at_rebuild(g, 0) == ["rho", "v"]
    # a pair sum over a field written earlier in the kernel splits it
    e2 = [_eq(t, k) for k, t in enumerate(["p = c**2*(rho - rho0)", "vdot = sph_G(p, mass, rho)",
                                            "rho = rho + dt*sph_L(rho, mass, rho)"])]
    assert [[e.index for e in x.eqs] for x in L.group_equations(e2)] == [[0], [1, 2]]
    # a pair sum after a move splits it too (the neighbour sets are stale)
    e3 = [_eq(t, k) for k, t in enumerate(["r = euler(r, v, dt)", "vdot = sph_G(p, mass, rho)"])]
    assert len(L.group_equations(e3)) == 2
    # a local equation reading a field written earlier in the kernel takes the
    # register value, not memory
    line = [x for x in src.splitlines() if "const T L1 =" in x][0]
    assert "L0" in line and "a.f_rhodot" not in line
    line = [x for x in src.splitlines() if "const V3 dr6 =" in x][0]
    assert "L5" in line and "a.f_v_0" not in line


def test_paper_operator_notation():
    """The operator forms of the paper's listings -- op(A, m, rho, Wp52220,
    2*h) with sph_D00 / sph_G11 / sph_L0 / sph_A, and ^ for powers -- compile
    to exactly the kernels of the plain forms; another kernel keyword or
    radius is rejected."""
    kinds = {"d": "S", "rho": "S", "P": "S", "u": "V", "a": "V", "cc": "S", "mu": "S"}
    consts = {"m0": 0.05, "c": 50.0, "rho0": 1000.0, "dt": 1e-3, "g": (0.0, -9.81), "gam": 1e-4}
    paper = ["d = 2*sph_D00(u, m0, rho, Wp52220, 2*h) + rho",
             "P = c^3*d - rho0",
             "a = sph_G11(P, m0, rho, Wp52220, h*2) - 3*sph_A(u, m0, rho, Wp52220, 2*h) + g*d",
             "mu = gam*sph_L0(cc, m0, rho0, Wp52220, 2*h) + cc^2"]
    plain = ["d = 2*sph_D(u, m0, rho) + rho",
             "P = c**3*d - rho0",
             "a = sph_G(P, m0, rho) - 3*sph_A(u, m0, rho) + g*d",
             "mu = gam*sph_L(cc, m0, rho0) + cc**2"]
    for dim in (2, 3):
        ep = [L.parse_equation(t, k, kinds, consts, dim) for k, t in enumerate(paper)]
        eq = [L.parse_equation(t, k, kinds, consts, dim) for k, t in enumerate(plain)]
        assert L.generate(ep, kinds, consts, dim, True)[0] == L.generate(eq, kinds, consts, dim, True)[0]
    for bad in ("d = sph_D00(u, m0, rho, Wq2, 2*h)", "d = sph_D00(u, m0, rho, Wp52220, 3*h)",
                "d = sph_D00(u, m0, rho, Wp52220, h)", "d = sph_D00(u, m0, rho)"):
        with pytest.raises(L.LawError):
            L.parse_equation(bad, 0, kinds, consts, 2)


def test_variables_and_reductions():
    """Global variables: read anywhere; an equation for a variable reads
    fields only inside fmax / fmin / fsum and runs as its own reduction
    kernel pair; misuse is rejected."""
    kinds = {"c": "S", "cdot": "S", "u": "V"}
    consts = {"dtg": 1e-2, "m": 0.01, "rho0": 1.0}
    vs = {"dt": 0, "Time": 1}
    eqs = ["cdot = sph_L(c, m, rho0)", "dt = 0.1*min(1/fmax(abs(cdot)), dtg)", "c = euler(c, cdot, dt)",
           "Time = Time + dt"]
    E = [L.parse_equation(t, k, kinds, consts, 2, vs) for k, t in enumerate(eqs)]
    assert [e.kind for e in E] == ["pair", "var", "local", "var"]
    assert E[1].reds and E[1].reds[0][0] == "fmax" and not E[3].reds
    src, G = L.generate(E, kinds, consts, 2, True, vs)
    assert [g.var for g in G] == [False, True, False, True]
    assert "vars[0]" in src and "vars[1]" in src
    for bad in ("dt = c", "c = fmax(c)", "dt = fmax(sph_L(c, m, rho0))", "dt = fmax(fmin(c))",
                "dt = fmax(u)", "dt = sph_L(c, m, rho0)"):
        with pytest.raises(L.LawError):
            L.parse_equation(bad, 0, kinds, consts, 2, vs)


def test_field_names_clear_of_generated_code(tmp_path):
    """Fields named like the generated code's own identifiers (T, D, P, n,
    i, a, pos, vars) still compile."""
    os.environ["SPH_LAW_CACHE"] = str(tmp_path)
    try:
        kinds = {"T": "S", "D": "S", "P": "V", "n": "S", "i": "S", "a": "S", "pos": "S"}
        consts = {"m": 0.01, "rho0": 1.0}
        vs = {"vars": 0}          # name -> slot
        eqs = ["D = sph_L(T, m, rho0) + n*i", "P = sph_G(T, m, rho0)*a", "vars = fmax(pos + T)",
               "T = T + vars*D"]
        E = [L.parse_equation(t, k, kinds, consts, 3, vs) for k, t in enumerate(eqs)]
        src, G = L.generate(E, kinds, consts, 3, True, vs)
        assert os.path.exists(L.compile_source(src))
    finally:
        del os.environ["SPH_LAW_CACHE"]


def test_where_and_the_pair_loop_guard():
    """where(c, a, b) selects per particle; when every pair equation of a
    kernel is where(c, sums..., b) with c read from memory, the neighbour
    walk runs only where some c is non-zero (the masks are still recorded);
    a condition computed in the same kernel disables the guard."""
    kinds = {"fl": "S", "q": "S", "s": "S", "w": "S"}
    consts = {"m": 0.01, "rho0": 1.0}
    g1 = [L.parse_equation(t, k, kinds, consts, 2) for k, t in
          enumerate(["q = where(fl, sph_L(s, m, rho0), 0)", "w = where(fl - 1, sph_S(s, m, rho0), 1)"])]
    src, _ = L.generate(g1, kinds, consts, 2, True)
    assert "if (((a.f_fl[i]) != (T)0) || (((a.f_fl[i] - ((T)1.0))) != (T)0))" in src
    g3 = [L.parse_equation(t, k, kinds, consts, 2) for k, t in      # a sum outside the guarded branch
          enumerate(["q = where(fl, sph_L(s, m, rho0), 0)", "w = where(fl, 1, sph_S(s, m, rho0))"])]
    assert "if (((a.f_fl" not in L.generate(g3, kinds, consts, 2, True)[0]
    g2 = [L.parse_equation(t, k, kinds, consts, 2) for k, t in
          enumerate(["fl = s*2", "q = where(fl, sph_L(s, m, rho0), 0)"])]
    src2, _ = L.generate(g2, kinds, consts, 2, True)
    assert "if (((a.f_fl" not in src2
    with pytest.raises(L.LawError):
        L.parse_equation("q = where(fl, s)", 0, kinds, consts, 2)


def test_mirror_sign_factors_compile_out():
    """Without a symmetric face every image sign factor is 1: the generated
    source says so at compile time."""
    kinds = {"v": L.VECTOR, "a": L.VECTOR}
    eqs = [L.parse_equation("a = sum_j(v_j*W_ij)", 0, kinds, {}, 3)]
    src_m, _ = L.generate(eqs, kinds, {}, 3, True, mirror=True)
    src_n, _ = L.generate(eqs, kinds, {}, 3, True, mirror=False)
    assert "constexpr bool kMirror = true;" in src_m
    assert "constexpr bool kMirror = false;" in src_n
    assert "msign(ic, 0) * a.f_v_0[j]" in src_n


def test_row_stencil_needs_cut_off_faces():
    """Cells of edge below 2h are searched as rows, which have no images: a
    law system on such cells with a periodic (or symmetric) face is refused
    before anything is compiled or allocated."""
    import numpy as np
    from paper_1710_08259_gb300 import cases as C
    from paper_1710_08259_gb300 import laws as L
    case = C.periodic_cube(6, seed=3)
    case.cs = case.h                      # cells of edge h in a periodic cube
    n = case.n
    fields = {"A": ("scalar", np.ones(n)), "m": ("scalar", np.ones(n)), "rho": ("scalar", np.ones(n)),
              "Sv": ("scalar", np.zeros(n))}
    with pytest.raises(L.LawError):
        L.LawSystem(case, fields, {}, ["Sv = sph_S(A, m, rho)"])

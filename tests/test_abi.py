"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every function include/sph.h declares; argument validation that
happens before any CUDA call."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(sph_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1710_08259_gb300 import build as B
    return B.build()


def test_header_symbols_exported(libpath):
    names = _declared("sph.h")
    assert "sph_step" in names and "sph_build_cells" in names
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sph_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = C.CDLL(libpath)
    for n in names:
        getattr(L, n)


def test_binding_covers_header():
    from paper_1710_08259_gb300 import sph
    names = _declared("sph.h")
    for n in names:
        assert hasattr(sph, n), n


def test_create_rejects_bad_params(libpath):
    from paper_1710_08259_gb300 import cases, sph
    case = cases.dam_break_2d()
    bad = []
    p = sph.params_from_case(case); p.dim = 4; bad.append(p)
    p = sph.params_from_case(case); p.cs = 0.999 * case.h; bad.append(p)  # cs < h
    ex = cases.example_1a(1)
    p = sph.params_from_case(ex); p.cs = 1.5 * ex.h; bad.append(p)        # cs < 2h outside the WCSPH step
    p = sph.params_from_case(case); p.gamma = 7.5; bad.append(p)
    p = sph.params_from_case(case); p.h = -1.0; bad.append(p)
    p = sph.params_from_case(case); p.dt = 0.0; bad.append(p)
    p = sph.params_from_case(case); p.precision = 5; bad.append(p)
    p = sph.params_from_case(case); p.dt_mode = 2; bad.append(p)
    p = sph.params_from_case(case, dt_mode=sph.SPH_DT_ADAPTIVE, cfl=0.0); bad.append(p)
    p = sph.params_from_case(case, dt_mode=sph.SPH_DT_ADAPTIVE, cfl=1.5); bad.append(p)
    p = sph.params_from_case(cases.example_1a(1), dt_mode=sph.SPH_DT_ADAPTIVE); bad.append(p)  # WCSPH only
    for p in bad:
        with pytest.raises(sph.SphError) as e:
            sph.sph_create(p, 100)
        assert "(-1)" in str(e.value)
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.params_from_case(case), 0)


def test_product_path_does_not_import_oracle():
    """The library package never reaches the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_1710_08259_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                for bad in ("import oracle", "from oracle", "liboracle", "sph_oracle", "orc_"):
                    assert bad not in txt, (f, bad)


def test_binding_struct_layouts_match_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the header's struct (gcc on this host)."""
    import shutil
    from paper_1710_08259_gb300 import sph
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    pairs = {"sph_params": sph.SphParams, "sph_state": sph.SphState, "sph_diag": sph.SphDiag,
             "sph_law_views": sph.SphLawViews, "sph_case_desc": sph.SphCaseDesc, "sph_tune": sph.SphTune,
             "sph_grad": sph.SphGrad}
    lines = ['#include <stdio.h>', '#include "sph.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        *key, val = ln.split()
        got[tuple(key)] = int(val)
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_binding_constants_match_header():
    """Every integer constant the header defines has the same value in the
    binding."""
    from paper_1710_08259_gb300 import sph
    txt = open(os.path.join(ROOT, "include", "sph.h")).read()
    defs = re.findall(r"^#define (SPH_\w+) \(?(-?\d+)u?\)?", txt, flags=re.M)
    assert len(defs) > 30
    for name, val in defs:
        assert hasattr(sph, name), name
        assert getattr(sph, name) == int(val), name

"""Checkpoint / resume: Simulation.save writes the context's parameters and
the exact device state (and the DEM tank); Simulation.restore continues bit
for bit, as if the run had never stopped."""
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


CASES = {
    "wcsph_3d_f32": (lambda: C.small_dam_break(3, 10), "f32"),
    "wcsph_2d_f64": (lambda: C.small_dam_break(2, 24), "f64"),
    "example_1a_f32": (lambda: C.example_1a(1), "f32"),
    "dem_f32": (lambda: C.dem_damper(6, 6, 5, seed=3, v_sigma=0.2), "f32"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_restore_continues_bit_for_bit(S, name, tmp_path):
    make, prec = CASES[name]
    P = S.SPH_PREC_F32 if prec == "f32" else S.SPH_PREC_F64
    a = S.Simulation(make(), precision=P)
    a.step(7)
    path = str(tmp_path / "ckpt.npz")
    a.save(path)
    a.step(9)
    b = S.Simulation.restore(path)
    b.step(9)
    for x, y in zip(a.state.to_host(), b.state.to_host()):
        np.testing.assert_array_equal(x, y)
    if name == "dem_f32":
        ta, tb = a.tank(), b.tank()
        assert ta[:3] == tb[:3]
        np.testing.assert_array_equal(np.asarray(ta[3]), np.asarray(tb[3]))
        np.testing.assert_array_equal(a.state.radius.cpu().numpy(), b.state.radius.cpu().numpy())
    assert b.status() == 0
    a.close()
    b.close()

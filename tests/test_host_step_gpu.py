"""sph_step_host: the end-to-end call on a state held in host memory (copy
in over the context's copy streams, step, write or copy back) gives, bit for
bit, the state that sph_step gives on device arrays, for one step per call
(the step reads the staged copy and writes the host state) and several (the
earlier steps run on the staged copy)."""
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


def _host(st, pinned):
    """Host copies of a device state: all page-locked (copied in by kernels
    over their device mapping, the last step writes them through it), none
    (driver copies both ways), or mixed (copy kernels for the page-locked
    ones, driver copies for the rest)."""
    def h(t, lock):
        t = t.cpu()
        return t.pin_memory() if lock else t.clone()
    lock_rv = pinned in ("all", "mixed")
    lock_rest = pinned == "all"
    a = {"r": [h(t, lock_rv) for t in st.r], "v": [h(t, lock_rv) for t in st.v], "rho": h(st.rho, lock_rest),
         "p": h(st.p, lock_rest), "id": h(st.id, lock_rest), "kind": h(st.kind, lock_rest)}
    if st.radius is not None:
        a["radius"], a["mass"] = h(st.radius, lock_rest), h(st.mass, lock_rest)
    return a


CASES = {
    "wcsph_3d_f32": (lambda: C.small_dam_break(3, 10), "f32"),
    "wcsph_2d_f64": (lambda: C.small_dam_break(2, 24), "f64"),
    "example_1a_f32": (lambda: C.example_1a(1), "f32"),
    "dem_f32": (lambda: C.dem_damper(6, 6, 5, seed=3, v_sigma=0.2), "f32"),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("pinned", ["all", "none", "mixed"])
def test_host_step_equals_device_step(S, name, pinned):
    make, prec = CASES[name]
    case = make()
    P = S.SPH_PREC_F32 if prec == "f32" else S.SPH_PREC_F64
    dev = S.Simulation(case, precision=P)
    ref = S.Simulation(case, precision=P)
    host = _host(dev.state, pinned)
    view = S.host_state_view(host)
    d = S.SphDiag()
    for k in (1, 2, 3, 0):
        S.sph_step_host(dev.ctx, view, k, d)
    ref.step(6)
    r, v, rho, p, ids, kind = ref.state.to_host()
    np.testing.assert_array_equal(np.stack([t.numpy() for t in host["r"]], 1), r)
    np.testing.assert_array_equal(np.stack([t.double().numpy() for t in host["v"]], 1), v)
    np.testing.assert_array_equal(host["id"].numpy().astype(np.uint32), ids)
    np.testing.assert_array_equal(host["kind"].numpy(), kind)
    if name != "dem_f32":
        np.testing.assert_array_equal(host["rho"].double().numpy(), rho)
        np.testing.assert_array_equal(host["p"].double().numpy(), p)
    assert dev.status() == 0
    if name != "dem_f32":             # (the damper's spheres start apart: no contact yet)
        assert d.n_pairs > 0
    dev.close()
    ref.close()


def test_host_step_rejects(S):
    case = C.small_dam_break(2, 10)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    host = _host(sim.state, "all")
    view = S.host_state_view(host)
    view.rho = None
    with pytest.raises(S.SphError):
        S.sph_step_host(sim.ctx, view, 1)
    view = S.host_state_view(host)
    with pytest.raises(S.SphError):
        S.sph_step_host(sim.ctx, view, -1)
    sim.close()

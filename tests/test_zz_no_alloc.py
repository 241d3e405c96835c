"""sph_build_cells_static: the neighbour-search build for callers that cannot
allocate device memory where they need it (code under another component's
allocator, loops that must not stall on cudaMalloc/cudaFree, plug-ins handed
only the particle arrays).  It must give exactly what sph_build_cells gives
(the sort and the cell table are integer work: bit for bit), call after call,
although every call reuses the same fixed scratch array."""
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


def _static_build(S, case, prec):
    """Sort a fresh device copy of the case with the no-allocation entry
    point; returns (host state, cell table, status)."""
    P = S.params_from_case(case, precision=prec)
    st = S.device_state(case.r, case.v, case.kind, case.id, prec)
    cells = torch.zeros(case.n_cells + 1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    S.sph_build_cells_static(P, st.view(), cells.data_ptr(), status.data_ptr())
    torch.cuda.synchronize()
    return st.to_host(), cells.cpu().numpy().astype(np.uint32), int(status.item())


def _context_build(S, case, prec):
    sim = S.Simulation(case, precision=prec)
    sim.build_cells()
    out = sim.state.to_host(), sim.cell_table(), sim.status()
    sim.close()
    return out


def _same(a, b):
    (ha, ca, sa), (hb, cb, sb) = a, b
    for x, y in zip(ha, hb):
        assert np.array_equal(x, y)
    assert np.array_equal(ca, cb)
    assert sa == sb == 0


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_static_build_matches_context_build_twice(S, prec):
    P = S.SPH_PREC_F32 if prec == "f32" else S.SPH_PREC_F64
    first = C.random_cloud(3, 5000, seed=61, box=0.09)
    second = C.small_dam_break(2, 40, seed=62)          # different grid and size
    # two calls in a row on different cases: the second must not see the
    # first one's leftovers in the shared scratch
    _same(_static_build(S, first, P), _context_build(S, first, P))
    _same(_static_build(S, second, P), _context_build(S, second, P))
    # and once more on the first case
    _same(_static_build(S, first, P), _context_build(S, first, P))


def test_static_build_of_a_field_model_without_velocity(S):
    """The field model carries no velocity (its fields belong to the
    caller): a state with NULL v is accepted, as sph_build_cells accepts it,
    and sorted exactly as the context build sorts it."""
    case = C.random_cloud(2, 3000, seed=63, box=0.1)
    case.model = S.SPH_MODEL_FIELDS
    P = S.params_from_case(case)
    st = S.device_state(case.r, case.v, case.kind, case.id)
    view = st.view()
    for k in range(3):
        view.v[k] = None
    S.sph_build_cells_static(P, view)
    torch.cuda.synchronize()
    sim = S.Simulation(case)
    sv = sim.state.view()
    for k in range(3):
        sv.v[k] = None
    S.sph_build_cells(sim.ctx, sv)
    torch.cuda.synchronize()
    for a, b in zip(st.r + [st.id, st.kind], sim.state.r + [sim.state.id, sim.state.kind]):
        assert torch.equal(a, b)
    sim.close()


def test_static_build_rejects_oversize(S):
    case = C.random_cloud(2, S_MAX + 1, seed=3)
    P = S.params_from_case(case)
    st = S.device_state(case.r, case.v, case.kind, case.id)
    with pytest.raises(S.SphError) as e:
        S.sph_build_cells_static(P, st.view())
    assert "(-3)" in str(e.value) and "static limit" in str(e.value)


def test_static_build_rejects_too_many_cells(S):
    """Grids beyond SPH_STATIC_MAX_CELLS in total, or beyond
    SPH_STATIC_MAX_AXIS_CELLS along one axis, are refused before any launch."""
    case = C.random_cloud(2, 100, seed=4)
    st = S.device_state(case.r, case.v, case.kind, case.id)
    for ncell in ((600, 600), (S.SPH_STATIC_MAX_AXIS_CELLS + 1, 2)):
        P = S.params_from_case(case)
        P.ncell[0], P.ncell[1] = ncell
        with pytest.raises(S.SphError) as e:
            S.sph_build_cells_static(P, st.view())
        assert "(-3)" in str(e.value) and "static limit" in str(e.value), str(e.value)


def test_static_build_allocates_no_device_memory(S):
    """After a first call (the set-up), further calls leave the device's free
    memory unchanged."""
    case = C.random_cloud(3, 5000, seed=64, box=0.09)
    P = S.params_from_case(case)
    st = S.device_state(case.r, case.v, case.kind, case.id)
    S.sph_build_cells_static(P, st.view())
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        S.sph_build_cells_static(P, st.view())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


S_MAX = 65536

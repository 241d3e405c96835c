"""Batched form: many uneven cases in one persistent cooperative launch, or
in one ordinary launch per phase (the phased form).

Every batched case must evolve bit for bit like the same case stepped alone
through sph_step (the paths run the same phase bodies), which ties the
batched forms to the single-case parity against the oracle."""
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


def _mixed_cases(dim, sizes, seed, k=1):
    out = []
    rng = np.random.default_rng(seed)
    for i, n in enumerate(sizes):
        c = C.small_dam_break(dim, n, seed=seed + i, alpha=float(rng.uniform(0.01, 0.05)), cells_per_radius=k)
        c.v[: c.n_fluid] = rng.normal(0.0, 0.05, size=(c.n_fluid, dim))
        out.append(c)
    return out


@pytest.mark.parametrize("dim,sizes,prec,k", [
    (2, [7, 23, 40, 12, 31, 5], "f32", 1),
    (2, [18, 9, 27], "f64", 1),
    (3, [6, 10, 4], "f32", 1),
    (2, [7, 23, 40, 12, 31, 5], "f32", 2),
    (2, [18, 9, 27], "f64", 2),
    (3, [6, 10, 4], "f32", 2),
])
@pytest.mark.parametrize("form,block", [("persistent", 64), ("persistent", 128), ("persistent", 256),
                                        ("phased", 128)])
def test_batch_matches_single_bitwise(S, dim, sizes, prec, k, form, block):
    """k: cells per support radius (2: cells of edge h, the row stencil)."""
    P = S.SPH_PREC_F32 if prec == "f32" else S.SPH_PREC_F64
    cases = _mixed_cases(dim, sizes, seed=100 + dim, k=k)
    t = S.SphTune()
    t.block, t.blocks_per_sm, t.spin_limit = block, 0, 0
    t.form = S.SPH_BATCH_PHASED if form == "phased" else S.SPH_BATCH_PERSISTENT
    b = S.Batch(cases, P, tune=t)
    nsteps = 25
    b.step(10)
    b.step(nsteps - 10)
    assert b.status() == 0
    for ci, c in enumerate(cases):
        sim = S.Simulation(c, precision=P)
        sim.step(nsteps)
        r1, v1, rho1, p1, id1, k1 = sim.state.to_host()
        r2, v2, rho2, p2, id2, k2 = b.case_host(ci)
        assert np.array_equal(id1, id2), ci
        assert np.array_equal(r1, r2) and np.array_equal(v1, v2), ci
        assert np.array_equal(rho1, rho2) and np.array_equal(p1, p2), ci
        sim.close()
    info = b.info()
    assert info["block"] == block and info["grid"] > 0
    assert info["graph_used"] in (0, 1)
    b.close()


def test_batch_rejects_mixed_cell_sizes(S):
    """Every case of a batch walks the same stencil: cells of edge >= 2h and
    cells of edge h cannot be mixed."""
    cases = _mixed_cases(2, [8], seed=5, k=1) + _mixed_cases(2, [9], seed=6, k=2)
    with pytest.raises(S.SphError):
        S.Batch(cases, S.SPH_PREC_F32)


def test_batch_vs_oracle(S, orc):
    """Two batched FP32 cases after 10 steps against the FP64 oracle (the
    single-case FP32 bounds: positions by displacement)."""
    cases = _mixed_cases(2, [20, 33], seed=7)
    b = S.Batch(cases, S.SPH_PREC_F32)
    b.step(10)
    for ci, c in enumerate(cases):
        r, v, rho, p, ids, kind = b.case_host(ci)
        res = orc.step(orc.params(c), c.r, c.v, c.kind, c.id, 10)
        k = np.argsort(c.id)[ids]
        dr, dro = r - c.r[k], res.r[k] - c.r[k]
        assert np.abs(dr - dro).max() <= 1e-4 * np.abs(dro).max()
        assert np.abs(rho - res.rho[k]).max() <= 1e-5 * np.abs(res.rho).max()
    b.close()


def test_batch_barrier_timeout_selftest(S):
    """The barrier's bounded wait: with one block absent, the others give up
    after the spin limit and report SPH_STATUS_BARRIER_TIMEOUT; the context
    stays usable and the next normal step is correct."""
    cases = _mixed_cases(2, [15, 22], seed=9)
    b = S.Batch(cases, S.SPH_PREC_F32)
    st = S.sph_batch_selftest_barrier(b.handle, b._view, 20000)
    assert st & S.SPH_STATUS_BARRIER_TIMEOUT
    b.step(5)
    assert b.status() == 0
    sim = S.Simulation(cases[1], precision=S.SPH_PREC_F32)
    sim.step(5)
    assert np.array_equal(sim.state.to_host()[0], b.case_host(1)[0])
    b.close()


def test_batched_workload_256_cases(S, orc):
    """The batched workload (256 cases, 1k-64k fluid each, log-uniform) at
    full size, in the benchmark's launch: a few steps in one launch, no
    status bits; three sampled cases bit-exact against single-case stepping,
    and the largest of the three against the FP64 oracle."""
    cases = C.batched_cases()
    b = S.Batch(cases, S.SPH_PREC_F32)
    b.step(3)
    assert b.status() == 0
    diag, npairs = S.sph_batch_diag(b.handle, len(cases))
    assert npairs > 0 and all(d.vmax > 0 for d in diag)
    for ci in (0, 77, 255):
        sim = S.Simulation(cases[ci], precision=S.SPH_PREC_F32)
        sim.step(3)
        r1 = sim.state.to_host()[0]
        assert np.array_equal(r1, b.case_host(ci)[0]), ci
        sim.close()
    big = max((0, 77, 255), key=lambda c: cases[c].n)
    c = cases[big]
    r, v, rho, p, ids, kind = b.case_host(big)
    res = orc.step(orc.params(c), c.r, c.v, c.kind, c.id, 3)
    k = np.argsort(c.id)[ids]
    dr, dro = r - c.r[k], res.r[k] - c.r[k]
    # three steps from rest move ~1e-4 dx: FP32 rounding of the accelerations
    # (~1e-7 relative) and of the cell-relative offsets (~1e-7 dx) bound it
    assert np.abs(dr - dro).max() <= 1e-4 * np.abs(dro).max() + 1e-7 * c.dx
    assert np.abs(rho - res.rho[k]).max() <= 1e-5 * np.abs(res.rho).max()
    b.close()


def test_phased_equals_persistent_256_cases(S):
    """The batched workload at full size: the phased form (one launch per
    phase) and the persistent kernel give the same packed state bit for bit
    after 3 steps, and the same pair count."""
    cases = C.batched_cases()
    out = []
    for form in (S.SPH_BATCH_PERSISTENT, S.SPH_BATCH_PHASED):
        t = S.SphTune()
        t.block, t.blocks_per_sm, t.spin_limit, t.form = 128, 0, 0, form
        b = S.Batch(cases, S.SPH_PREC_F32, tune=t)
        b.step(3)
        assert b.status() == 0
        _, npairs = S.sph_batch_diag(b.handle, len(cases))
        st = b.state
        out.append(([t.cpu() for t in st.r + st.v] + [st.rho.cpu(), st.p.cpu(), st.id.cpu()], npairs))
        b.close()
    (a, na), (b_, nb) = out
    assert na == nb > 0
    for x, y in zip(a, b_):
        assert torch.equal(x, y)


def test_batch_form_rejects(S):
    cases = _mixed_cases(2, [10, 12], seed=13)
    t = S.SphTune()
    t.block, t.form = 64, S.SPH_BATCH_PHASED
    with pytest.raises(S.SphError):
        S.Batch(cases, S.SPH_PREC_F32, tune=t)
    t.block, t.form = 128, 7
    with pytest.raises(S.SphError):
        S.Batch(cases, S.SPH_PREC_F32, tune=t)
    t.form = S.SPH_BATCH_PHASED
    b = S.Batch(cases, S.SPH_PREC_F32, tune=t)
    with pytest.raises(S.SphError):   # no grid barrier to test
        S.sph_batch_selftest_barrier(b.handle, b._view, 1000)
    b.close()


def test_autotuner(S, tmp_path, monkeypatch):
    from paper_1710_08259_gb300 import tune
    monkeypatch.setenv("SPH_TUNE_CACHE", str(tmp_path / "tune.json"))
    cases = _mixed_cases(2, [30, 45, 20, 60], seed=11)
    best = tune.autotune(cases, S.SPH_PREC_F32, steps=2)
    assert best["block"] in (64, 128, 256) and best["ms_per_step"] > 0
    assert {r["form"] for r in best["tried"]} == {"persistent", "phased"}
    again = tune.autotune(cases, S.SPH_PREC_F32, steps=2)
    assert again["block"] == best["block"]  # served from the cache
    assert (tmp_path / "tune.json").exists()


@pytest.mark.parametrize("dim,n,prec", [
    (2, 40, "f32"),     # 2,218 particles: 8 lanes per particle
    (2, 120, "f32"),    # 16,218: 8
    (2, 150, "f64"),    # 24,771: density 4 lanes, force one (FP64 force teams are of 8)
    (2, 200, "f32"),    # 43,018: density 2 lanes, force one (force teams are of 4 or 8)
    (3, 14, "f32"),     # 12,761: 8
    (3, 20, "f32"),     # 26,948: 4
    (3, 20, "f64"),     # 26,948: density 4, force one
])
def test_team_kernels_match_one_lane_bitwise(S, dim, n, prec):
    """Small cases step with teams of lanes per particle (sph_step picks the
    team from the particle count); the batched form runs the same case with
    one lane per particle.  The teams join their sums in the one-lane order,
    so the states agree bit for bit at every team size."""
    P = S.SPH_PREC_F32 if prec == "f32" else S.SPH_PREC_F64
    c = C.small_dam_break(dim, n, seed=300 + n, alpha=0.03, cells_per_radius=2)
    rng = np.random.default_rng(n)
    c.v[: c.n_fluid] = rng.normal(0.0, 0.05, size=(c.n_fluid, dim))
    t = S.SphTune()
    t.block, t.blocks_per_sm, t.spin_limit, t.form = 128, 0, 0, S.SPH_BATCH_PHASED
    b = S.Batch([c], P, tune=t)
    b.step(12)
    assert b.status() == 0
    sim = S.Simulation(c, precision=P)
    sim.step(12)
    assert sim.status() == 0
    r1, v1, rho1, p1, id1, _ = b.case_host(0)
    r2, v2, rho2, p2, id2, _ = sim.state.to_host()
    np.testing.assert_array_equal(id1, id2)
    np.testing.assert_array_equal(r1, r2)
    np.testing.assert_array_equal(v1, v2)
    np.testing.assert_array_equal(rho1, rho2)
    np.testing.assert_array_equal(p1, p2)
    sim.close()
    b.close()

"""Workloads run by test_checked_gpu.py, once through the normal library and
once (in a child process, SPH_CHECKED=1) through the bounds-checked build:
every model's step, the adjoint, the batched form, the sampling operator and
the neighbour images.  run() returns {name: array} including each
context's status word."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run():
    import torch
    from paper_1710_08259_gb300 import cases as C
    from paper_1710_08259_gb300 import sph as S
    out = {}

    def keep(name, sim):
        r, v, rho, p, ids, kind = sim.state.to_host()
        out[name + "/r"], out[name + "/v"], out[name + "/rho"], out[name + "/ids"] = r, v, rho, ids
        out[name + "/status"] = np.array([sim.status()])

    for name, case, prec, steps in (
            ("wcsph3d_f32", C.small_dam_break(3, 12), S.SPH_PREC_F32, 5),
            ("wcsph2d_f64", C.small_dam_break(2, 30), S.SPH_PREC_F64, 5),
            ("example1a_f32", C.example_1a(1), S.SPH_PREC_F32, 5),
            ("dem_f32", C.dem_damper(7, 7, 6, spacing=0.0079, seed=5, v_sigma=0.2), S.SPH_PREC_F32, 5)):
        sim = S.Simulation(case, precision=prec)
        sim.step(steps)
        keep(name, sim)
        if name == "example1a_f32":
            counts = torch.zeros(sim.state.n, dtype=torch.int32, device="cuda")
            S.sph_neighbor_counts(sim.ctx, sim._view, counts.data_ptr())
            out[name + "/counts"] = counts.cpu().numpy()
        sim.close()
    # the adjoint of one step
    case = C.small_dam_break(2, 20)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    sim.step(2)
    n = case.n
    g1r = [torch.ones(n, dtype=torch.float64, device="cuda") for _ in range(2)]
    g1v = [torch.ones(n, dtype=torch.float32, device="cuda") for _ in range(2)]
    g0r = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(2)]
    g0v = [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(2)]
    ab = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.sph_step_adjoint(sim.ctx, sim.state.view(), S.grad_view(g1r, g1v), S.grad_view(g0r, g0v), ab.data_ptr())
    out["adjoint/r"] = np.stack([t.cpu().numpy() for t in g0r], 1)
    out["adjoint/v"] = np.stack([t.cpu().double().numpy() for t in g0v], 1)
    out["adjoint/status"] = np.array([sim.status()])
    sim.close()
    # the batched form
    cases = [C.small_dam_break(2, k, seed=20 + k) for k in (8, 13, 21)]
    b = S.Batch(cases, S.SPH_PREC_F32)
    b.step(4)
    for c in range(len(cases)):
        r, v, rho, p, ids, kind = b.case_host(c)
        out[f"batch{c}/r"], out[f"batch{c}/v"] = r, v
    out["batch/status"] = np.array([b.status()])
    b.close()
    # the sampling operator on a periodic cube
    case = C.periodic_cube(12, seed=3)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    sim.build_cells()
    A = torch.linspace(0.5, 1.5, case.n, dtype=torch.float32, device="cuda")
    m = torch.full((case.n,), case.mass, dtype=torch.float32, device="cuda")
    rho = torch.full((case.n,), case.rho0, dtype=torch.float32, device="cuda")
    out["sample/S"] = sim.sample(A, m, rho).cpu().numpy()
    out["sample/status"] = np.array([sim.status()])
    sim.close()
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run())

#!/usr/bin/env python
"""Benchmark of the GB300 WCSPH step.

Headline workload (default --case large): the large 3D dam break, 256^3 =
16,777,216 fluid + 2,730,708 boundary particles, dx = 0.002 m, 1.6 x 0.6 x
0.6 m tank, FP32 pair sums (Kahan density) with FP64 positions; one "step" =
one sph_step (cell build, density + EOS, forces + integration, CFL
reduction).  Beside it: the plain FP64 GPU path on the same workload, the
end-to-end rate through sph_step_host, the CPU oracle on a bounded sample,
and secondary keys (the 100^3 dam break with its own roofline, the 2D FP64
64 x 64 x 100-step configuration, the adjoint, batched, Example 1a,
sampling, DEM and compiled-law legs).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--case large|3d|2d|3d_small]

--impl reference times the CPU FP64 oracle (the only reference this method
has: the paper ships no code) on the host cores, full oracle steps of the
same workload.  Under torchrun with N > 1 every rank runs an independent
replica (the step does not shard); value sums all ranks.
"""
from __future__ import annotations

import argparse
import copy
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH fluid particle-steps/s (3D dam break, FP32 pair sums)"
UNIT = "particle-steps/s"

# Algorithmic FP32 operations (FMA = 2), counted from the kernel bodies:
# a candidate test is the pair geometry (D subtractions, 1 mul, D-1 FMA);
# a density pair (self included) is |r| (max, rsqrt, mul), q/2, 1 - q/2,
# (1-q/2)^4 (2q+1) and the Kahan update; a force pair is the pair geometry
# plus its body (|r|, t^3, v_ij . r_ij, viscosity with one division, the
# coefficient and the D accumulations).  The force pass tests no candidate:
# it reuses the density pass's neighbour masks.
FLOPS_CAND = {2: 5, 3: 8}
FLOPS_PAIR_DENSITY = {2: 14, 3: 14}
FLOPS_PAIR_FORCE = {2: 32, 3: 40}
# Example 1a form: a continuity pair (self included) is |r|, t^3, the image's
# v_ij . r_ij, one division by rho_j and the accumulation; a momentum pair is
# the same geometry and v_ij . r_ij, the viscosity (one division), the
# coefficient and the D signed accumulations.
FLOPS_PAIR_CONT = {2: 18, 3: 22}
FLOPS_PAIR_MOM = {2: 28, 3: 35}
# sampling operator: candidate test as above; a hit is |r|, (1-q/2)^4 (2q+1)
# and the weighted accumulation
FLOPS_HIT_SAMPLE = 13
# DEM contact (3D, sqrt and division counted 1): |r| 3, overlap 2, 1/|r| 1,
# frame-space relative velocity 6, v_ij . n 6, R' 3, m' 3, k 3, c 3,
# sqrt(delta) 1, f_n 6, tangential velocity and its norm 14, friction 3,
# signed accumulation of the force 18
FLOPS_CONTACT_DEM = 72
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# secondary workloads' top kernels, from one-pass ncu launch lists of the
# named workload, labelled with the commit of the captured kernels and the
# summary that holds them: the Example 1a passes and the compiled Appendix A
# kernels (2,219,346 particles, x64 case), k_dem_force (100^3 spheres) and
# k_sample (200^3 = 8e6 particles; its traffic grows with the particle count,
# so other cube sizes scale it).
SECONDARY_CAPTURES = {
    "k_cont": {"dram_bytes": 148.3e6, "workload": "example_1a_x64", "commit": "2ae4da8",
               "summary": "profiles/k_cont_k_mom_example_1a_x64.md"},
    "k_mom": {"dram_bytes": 277.3e6, "workload": "example_1a_x64", "commit": "2ae4da8",
              "summary": "profiles/k_cont_k_mom_example_1a_x64.md"},
    "law_k0": {"dram_bytes": 137.3e6, "workload": "appendix_a_x64", "commit": "2ae4da8",
               "summary": "profiles/law_k0_law_k1_appendix_a_x64.md"},
    "law_k1": {"dram_bytes": 249.5e6, "workload": "appendix_a_x64", "commit": "2ae4da8",
               "summary": "profiles/law_k0_law_k1_appendix_a_x64.md"},
    "k_dem_force": {"dram_bytes": 40.0e6, "workload": "dem_damper_100^3", "commit": "2ae4da8",
                    "summary": "profiles/k_dem_force_dem_damper_100cubed.md"},
    "k_sample": {"dram_bytes": 186.6e6, "n": 8.0e6, "workload": "periodic_cube_200^3", "commit": "2b4756f",
                 "summary": "profiles/k_sample_periodic_cube_200cubed.md"},
}


def secondary_traffic(kernel, scale_n=None):
    """(DRAM bytes per launch, how the figure was obtained) of a secondary
    kernel's capture; scale_n: scale it to this particle count."""
    cap = SECONDARY_CAPTURES[kernel]
    if scale_n is None:
        return cap["dram_bytes"], f"ncu capture of {cap['workload']} (commit {cap['commit']}, {cap['summary']})"
    return (cap["dram_bytes"] * scale_n / cap["n"],
            f"ncu capture of {cap['workload']} (commit {cap['commit']}, {cap['summary']}) scaled by the particle count")


def aggregate_replicas(elapsed_ms: float, units: float, world: int, device=None):
    """Replicas: the job's time is the slowest rank's, its work the sum of all
    ranks' units (each rank runs its own copy of the workload)."""
    if world <= 1:
        return elapsed_ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms, units], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t[1:].clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax.item()), float(tsum.item())


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz=2070.0, sms=152):
    """FP32 ALU roofline: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index=0, period_ms=100):
        self.samples = []
        self.proc = None
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        self.cmd = ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                    "-lms", str(period_ms)]

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        if not self.samples:
            return None

        def f(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [f(s[0]) for s in self.samples]
        mx = [f(s[1]) for s in self.samples]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(np.nanmax(mx)), "reasons": reasons,
                "samples": len(sm)}


def candidates_from_table(start, kind_sorted, dim, ncell):
    """Candidate pairs tested by the fluid particles (force pass) and by all
    particles (density pass): sum over cells of (particles in cell) x
    (particles in its 3^D stencil)."""
    start = start.astype(np.int64)
    cnt = np.diff(start)
    cf = np.concatenate([[0], np.cumsum(kind_sorted == 0)])
    nf = cf[start[1:]] - cf[start[:-1]]
    shape = (ncell[2], ncell[1], ncell[0]) if dim == 3 else (ncell[1], ncell[0])
    c = cnt.reshape(shape)
    pad = np.pad(c, 1)
    st = np.zeros_like(c)
    if dim == 3:
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    st += pad[1 + dz:1 + dz + shape[0], 1 + dy:1 + dy + shape[1], 1 + dx:1 + dx + shape[2]]
    else:
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                st += pad[1 + dy:1 + dy + shape[0], 1 + dx:1 + dx + shape[1]]
    st = st.reshape(-1)
    return int((nf * st).sum()), int((cnt * st).sum())


def candidates_method(r, kind, dom_min, h, dim):
    """Candidate pairs of the paper's cell-list search (cells of edge 2h, the
    3^D adjacent cells; Section 3.2.1 with the cell size of Section 5.1.1)
    for the positions r: (tested by fluid particles, tested by all).  This is
    the algorithmic unit of the candidate tests whatever cell size the
    library searches with: a finer grid that tests fewer candidates counts as
    a faster search."""
    cs2 = 2.0 * h
    c = np.floor((np.asarray(r)[:, :dim] - np.asarray(dom_min[:dim])) / cs2).astype(np.int64)
    c -= c.min(axis=0)
    nc = c.max(axis=0) + 1
    lin = c[:, 0] + nc[0] * (c[:, 1] + (nc[1] * c[:, 2] if dim == 3 else 0))
    ncell = [int(x) for x in nc] + [1] * (3 - dim)
    cnt = np.bincount(lin, minlength=int(np.prod(nc)))
    nfc = np.bincount(lin, weights=(np.asarray(kind) == 0).astype(np.float64),
                      minlength=int(np.prod(nc))).astype(np.int64)
    start = np.concatenate([[0], np.cumsum(cnt)])
    # (candidates_from_table with the fluid counts per cell given directly)
    shape = (ncell[2], ncell[1], ncell[0]) if dim == 3 else (ncell[1], ncell[0])
    cc = cnt.reshape(shape)
    pad = np.pad(cc, 1)
    st = np.zeros_like(cc)
    import itertools
    for off in itertools.product((-1, 0, 1), repeat=dim):
        sl = tuple(slice(1 + o, 1 + o + shape[a]) for a, o in enumerate(off))
        st += pad[sl]
    st = st.reshape(-1)
    del start
    return int((nfc * st).sum()), int((cnt * st).sum())


def candidates_bc(start, dim, ncell, bc):
    """Candidate tests of the image stencil: sum over cells of (particles in
    cell) x (particles in its 3^D stencil), out-of-grid stencil cells mapped
    by the face treatment (cut-off: none, symmetric: the cell itself,
    periodic: the cell on the other side)."""
    cnt = np.diff(start.astype(np.int64))
    shape = tuple(int(ncell[k]) for k in range(dim))[::-1]   # (z,) y, x
    c = cnt.reshape(shape)
    pad = c
    for ax in range(dim):
        k = dim - 1 - ax                  # numpy axis ax holds grid axis k
        mode = {0: "constant", 1: "edge", 2: "wrap"}[int(bc[k])]
        widths = [(0, 0)] * dim
        widths[ax] = (1, 1)
        pad = np.pad(pad, widths, mode=mode)
    st = np.zeros_like(c)
    import itertools
    for off in itertools.product((-1, 0, 1), repeat=dim):
        sl = tuple(slice(1 + o, 1 + o + shape[a]) for a, o in enumerate(off))
        st += pad[sl]
    return int((c * st).sum())


def example_1a_rate(S, torch, scale=64, steps=200, cpu=True):
    """Example 1a in the paper's form (continuity, linear EOS, symmetric
    walls) at 64 x the resolution of Appendix A: 1971 x 1126 = 2,219,346
    particles, FP32 pair sums; one step = build, continuity pass, momentum +
    integration pass, CFL epilogue."""
    from paper_1710_08259_gb300 import cases as CS
    case = CS.example_1a(scale)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    sim.step(3)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    S.sph_profile_begin(sim.ctx, steps)
    e0.record(st)
    sim.step(steps - 1)
    d = sim.step(1, diag=True)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    prof, nprof = S.sph_profile_end(sim.ctx)
    start = sim.cell_table()
    cand = candidates_bc(start, 2, case.ncell, case.bc)
    n = case.n
    pairs = int(d.n_pairs)
    cont_ms = prof["density"] / max(nprof, 1)
    mom_ms = prof["force"] / max(nprof, 1)
    cont_flops = cand * FLOPS_CAND[2] + (pairs + n) * FLOPS_PAIR_CONT[2]
    mom_flops = (int(d.n_pairs_fluid) + case.n_fluid) * FLOPS_PAIR_MOM[2]
    status = sim.status()
    out = {"value": case.n_fluid * steps / (ms * 1e-3), "unit": "fluid particle-steps/s",
           "ms_per_step": ms / steps, "steps": steps, "workload": f"example_1a_x{scale}_fp32",
           "n_particles": n, "boundaries": "symmetric x symmetric", "n_pairs_per_step": pairs,
           "phase_ms_per_step": {k: v / max(nprof, 1) for k, v in prof.items()},
           "kernels": {"k_cont": {"launch_ms": cont_ms, "flops_per_launch": cont_flops,
                                  "candidates_per_launch": cand,
                                  "achieved_tflops": cont_flops / (cont_ms * 1e-3) / 1e12},
                       "k_mom": {"launch_ms": mom_ms, "flops_per_launch": mom_flops,
                                 "achieved_tflops": mom_flops / (mom_ms * 1e-3) / 1e12}},
           "vmax": d.vmax, "status": status}
    peaks, _ = _peaks()
    alu = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    top = max(("k_cont", "k_mom"), key=lambda k: out["kernels"][k]["launch_ms"])
    kt = out["kernels"][top]
    out["roofline"] = {"bound": "alu", "kernel": f"{top}<2,float>", "achieved": kt["achieved_tflops"], "peak": alu,
                       "unit": "TFLOP/s", "frac": kt["achieved_tflops"] / alu,
                       "traffic": secondary_traffic(top)[0] if scale == 64 else None,
                       "traffic_note": secondary_traffic(top)[1] if scale == 64 else None}
    sim.close()
    if cpu:
        from oracle import oracle as O
        p = O.bc_params(case, fp32=True)
        t0 = time.perf_counter()
        res = O.bc_step(p, case.r, case.v, case.rho, case.kind, case.id, 1)
        sec = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": case.n_fluid / sec, "unit": "fluid particle-steps/s",
                               "cores": O.num_threads(), "kind": "oracle",
                               "sample": f"1 oracle step of the full case ({n} particles)", "rc": res.rc}
    return out


def dem_rate(S, torch, n_side=100, steps=100, cpu=True):
    """The particle damper of Example 2 scaled to n_side^3 spheres (R = 4 mm,
    E = 2.06 MPa, tank on its spring, symmetric walls), FP32, from a
    compressed simple-cubic packing (spacing 7.96 mm < 2R: six contacts per
    sphere).  One step = build, contact forces, tank, integration."""
    from paper_1710_08259_gb300 import cases as CS
    case = CS.dem_damper(n_side, n_side, n_side, spacing=0.00796)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    sim.step(3)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    S.sph_profile_begin(sim.ctx, steps)
    e0.record(st)
    sim.step(steps - 1)
    d = sim.step(1, diag=True)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    prof, nprof = S.sph_profile_end(sim.ctx)
    cand = candidates_bc(sim.cell_table(), 3, case.ncell, case.bc)
    contacts = int(d.n_pairs)
    f_ms = prof["density"] / max(nprof, 1)
    flops = cand * FLOPS_CAND[3] + contacts * FLOPS_CONTACT_DEM
    peaks, _ = _peaks()
    alu = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    tf = flops / (f_ms * 1e-3) / 1e12
    Z, Zd, Zdd, Fb = sim.tank()
    out = {"value": case.n * steps / (ms * 1e-3), "unit": "sphere-steps/s", "ms_per_step": ms / steps,
           "steps": steps, "workload": f"dem_damper_{n_side}^3_fp32", "n_spheres": case.n,
           "contacts_per_step": contacts, "candidates_per_step": cand,
           "phase_ms_per_step": {"build": prof["build"] / max(nprof, 1), "contact_forces": f_ms,
                                 "tank_integrate": prof["force"] / max(nprof, 1),
                                 "finish": prof["finish"] / max(nprof, 1)},
           "roofline": {"bound": "alu", "kernel": "k_dem_force<3,float>", "achieved": tf, "peak": alu,
                        "unit": "TFLOP/s", "frac": tf / alu,
                        "traffic": secondary_traffic("k_dem_force")[0] if n_side == 100 else None,
                        "traffic_note": secondary_traffic("k_dem_force")[1] if n_side == 100 else None,
                        "flops_per_launch": flops,
                        "launch_ms": f_ms},
           "tank": {"Z": Z, "Zdot": Zd, "Zddot": Zdd, "F_wall": [float(x) for x in Fb]},
           "status": sim.status()}
    sim.close()
    if cpu:
        from oracle import oracle as O
        p = O.dem_params(case, fp32=True)
        t0 = time.perf_counter()
        res = O.dem_step(p, case.r, case.v, case.rho, case.extra["m"], case.kind, case.id,
                         tank=(case.extra["z0"], 0.0), nsteps=1)
        sec = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": case.n / sec, "unit": "sphere-steps/s", "cores": O.num_threads(),
                               "kind": "oracle", "sample": f"1 oracle step of the full case ({case.n} spheres)",
                               "rc": res.rc}
    return out


APPENDIX_A_LAWS = ["rhodot = -rho*sph_D(v, mass, rho)",
                   "rho = euler(rho, rhodot, dt)",
                   "p = c**2*(rho - rho0)",
                   "vdot = -1/rho*sph_G(p, mass, rho)",
                   "vdot = vdot + 0.1*c*h*sph_A(v, mass, rho) + g",
                   "v = euler(v, vdot, dt)",
                   "r = euler(r, v, dt)"]
SOCIAL_FORCE_LAWS = ["vdot = (v0*e0 - v)/tau + sum_j((A*exp((R_i + R_j - d_ij)/B) + k*max(R_i + R_j - d_ij, 0)"
                     " - cA)*r_ij/d_ij)/m",
                     "v = euler(v, vdot, dt)",
                     "r = euler(r, v, dt)"]


# the hot path's own model written as equations (summation density, Tait EOS
# with the clamp, pressure gradient with the symmetric viscosity, fluid-only
# semi-implicit Euler)
WCSPH_LAWS = ["rho = sph_S(1, m, 1)",
              "p = max(B*((rho/rho_ref)**7 - 1), 0)",
              "vdot = where(fl, g - sum_j(m*(p_i/rho_i**2 + p_j/rho_j**2"
              " - alpha*c0*h*min(dot(v_i - v_j, r_ij), 0)/(0.5*(rho_i + rho_j)*(d_ij**2 + eps*h**2)))*gradW_ij),"
              " 0*g)",
              "v = euler(v, vdot, dt)",
              "r = euler(r, v, dt)"]


# Example 2 as equations: the Hertz contact law as a pair law (walls as
# mirror images), the tank's state as variables, the wall force as a reduction
_DL = "(R_i + R_j - d_ij)"
_VN = "(dot(v_i - v_j, r_ij)/d_ij)"
_KH = "(4/3*sqrt(R_i*R_j/(R_i + R_j))*Ep)"
_CH = f"(sqrt(m_i*m_j/(m_i + m_j)*{_KH})/8)"
_FN = f"({_KH}*{_DL}**1.5 - {_CH}*sqrt(sqrt({_DL}))*{_VN})"
_VT = f"((v_j - v_i) + {_VN}*r_ij/d_ij)"
_FT = f"where(max(dot({_VT}, {_VT}) - 1e-10*dot(v_i - v_j, v_i - v_j), 0), cf*abs({_FN})/norm({_VT}), 0)"
_FORCE = f"({_FN}*r_ij/d_ij + {_FT}*{_VT})"
EXAMPLE_2_LAWS = [f"F = sum_j(where(max({_DL}, 0), {_FORCE}, 0*r_ij))",
                  f"fwz = sum_j(where(max({_DL}, 0)*mirror_ij, dot({_FORCE}, vec(0, 0, 1)), 0))",
                  "Fb = fsum(fwz)",
                  "Zdd = (-S*Z - Fb)/M",
                  "v = euler(v, F/m + g - Zdd*vec(0, 0, 1), dt)",
                  "r = euler(r, v, dt)",
                  "Zd = Zd + dt*Zdd",
                  "Z = Z + dt*Zd"]


def _example_2_system(case):
    n = case.n
    fields = {"v": ("vector", case.v), "F": ("vector", np.zeros((n, 3))), "fwz": ("scalar", np.zeros(n)),
              "R": ("scalar", case.rho), "m": ("scalar", case.extra["m"])}
    nu, E = case.extra["nu"], case.extra["E"]
    consts = {"Ep": E / (2.0 * (1.0 - nu * nu)), "cf": case.extra["cf"], "g": tuple(case.g), "dt": case.dt,
              "S": case.extra["tank_S"], "M": case.extra["tank_M"]}
    variables = {"Z": case.extra["z0"], "Zd": 0.0, "Zdd": 0.0, "Fb": 0.0}
    return case, fields, consts, variables


def _wcsph_system(S, case):
    probe = S.Simulation(case, precision=S.SPH_PREC_F32)
    rho_ref = S.sph_rho_ref(probe.ctx)
    probe.close()
    n = case.n
    fields = {"rho": ("scalar", np.full(n, case.rho0)), "p": ("scalar", np.zeros(n)),
              "v": ("vector", case.v), "vdot": ("vector", np.zeros((n, case.dim))),
              "fl": ("scalar", (case.kind == 0).astype(np.float64))}
    consts = {"m": case.mass, "c0": case.c0, "alpha": case.alpha, "eps": case.visc_eps, "dt": case.dt,
              "B": case.c0 ** 2 * case.rho0 / case.gamma, "rho_ref": rho_ref, "g": tuple(case.g[:case.dim])}
    return case, fields, consts


def laws_rates(S, torch, scale=64, crowd=1_000_000, steps=50):
    """Compiled interaction laws: the equations of Appendix A at 64 x its
    resolution (the workload of the example_1a leg, which runs the same
    model through the hand-written kernels), the social force model of
    Section 6 written with sum_j on a corridor of 1M people, the hot path's
    own WCSPH model on the 3D 100^3 dam break (the headline workload of the
    hand-written step), and Example 2 with its tank on the 100^3-sphere
    damper of the dem leg; FP32.  Per phase: CUDA events around the cell
    build (+ field reorders) and each compiled kernel."""
    from paper_1710_08259_gb300 import cases as CS
    from paper_1710_08259_gb300 import laws as LW
    out = {}
    case = CS.example_1a(scale)
    n = case.n
    fields = {"rho": ("scalar", case.rho), "rhodot": ("scalar", np.zeros(n)), "p": ("scalar", np.zeros(n)),
              "v": ("vector", case.v), "vdot": ("vector", np.zeros((n, 2)))}
    consts = {"mass": case.mass, "c": case.c0, "rho0": case.rho0, "dt": case.dt, "g": (0.0, -9.81)}
    for name, (cs_, fl, cn, vs, eqs) in {
            "appendix_a": (case, fields, consts, None, APPENDIX_A_LAWS),
            "social_force": CS.social_force_crowd(crowd, seed=13) + (None, SOCIAL_FORCE_LAWS),
            "wcsph_3d_100cubed": _wcsph_system(S, CS.dam_break_3d()) + (None, WCSPH_LAWS),
            "example_2_100cubed": _example_2_system(CS.dem_damper(100, 100, 100, spacing=0.00796))
            + (EXAMPLE_2_LAWS,)}.items():
        sysm = LW.LawSystem(cs_, fl, cn, eqs, precision=S.SPH_PREC_F32, variables=vs)
        sysm.step(3)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sysm.step(steps)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        tm = {}
        sysm.step(steps, timing=tm)
        out[name] = {"value": cs_.n / (ms * 1e-3), "unit": "particle-steps/s", "ms_per_step": ms,
                     "n_particles": cs_.n, "steps": steps, "equations": len(eqs), "kernels": len(sysm.groups),
                     "phase_ms_per_step": {k: v / steps for k, v in tm.items()}}
        if name == "appendix_a":
            out[name].update(_compiled_appendix_a_roofline(S, torch, sysm, case, tm, steps))
        sysm.close()
    return out


def _compiled_appendix_a_roofline(S, torch, sysm, case, tm, steps):
    """Algorithmic FLOPs of the two compiled Appendix A kernels: the same
    arithmetic as the hand-written Example 1a passes (k0: candidate tests
    recorded as hit masks, continuity pairs, density update and EOS; k1:
    momentum pairs over the masks, integration), counted on the system's
    last cell table and pair count (the pairs of its current state, counted
    by the hand-written pass)."""
    ncells = S.sph_cell_table(sysm.ctx)
    t = torch.empty(ncells + 1, dtype=torch.int32, device="cuda")
    S.sph_cell_table(sysm.ctx, t.data_ptr())
    start = t.cpu().numpy().astype(np.uint32)
    cand = candidates_bc(start, 2, case.ncell, case.bc)
    r, f, ids = sysm.host()
    inv = np.empty(int(case.id.max()) + 1, np.int64)
    inv[case.id] = np.arange(case.n)
    c2 = copy.copy(case)
    c2.r, c2.v, c2.rho, c2.id = r, f["v"], f["rho"], ids
    c2.kind = case.kind[inv[ids]]
    sim = S.Simulation(c2, precision=S.SPH_PREC_F32)
    pairs = int(sim.step(1, diag=True).n_pairs)
    sim.close()
    n = case.n
    k0 = cand * FLOPS_CAND[2] + (pairs + n) * FLOPS_PAIR_CONT[2]
    k1 = (pairs + n) * FLOPS_PAIR_MOM[2]          # walks k0's hit masks: no candidate test
    ker = {}
    for k, fl in (("k0", k0), ("k1", k1)):
        ms = tm[k] / steps
        ker[k] = {"launch_ms": ms, "flops_per_launch": fl, "achieved_tflops": fl / (ms * 1e-3) / 1e12}
    peaks, _ = _peaks()
    alu = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    top = max(ker, key=lambda k: ker[k]["launch_ms"])
    return {"n_pairs_per_step": pairs, "candidates_per_step": cand, "compiled_kernels": ker,
            "roofline": {"bound": "alu", "kernel": f"law_{top}", "achieved": ker[top]["achieved_tflops"],
                         "peak": alu, "unit": "TFLOP/s", "frac": ker[top]["achieved_tflops"] / alu,
                         "traffic": secondary_traffic(f"law_{top}")[0] if case.n == 2219346 else None,
                         "traffic_note": secondary_traffic(f"law_{top}")[1] if case.n == 2219346 else None}}


def sampling_rates(S, torch, sides=(15, 46, 100, 252), cpu_side=100):
    """The benchmark of Section 6: the SPH sampling operator S_i = sum_j A_j
    m_j/rho_j W_ij on n_side^3 particles of a uniform grid in a periodic
    cube (h = 1.1 dx: 32 neighbours), FP32.  Per size: processed particles
    per second of the operator on cells built once (the paper's static
    layout) and with a rebuild per evaluation.  The largest size carries the
    roofline of the call (k_sample_prep + k_sample)."""
    from paper_1710_08259_gb300 import cases as CS
    out = {"unit": "particles/s", "sizes": []}
    st = torch.cuda.current_stream()
    for side in sides:
        case = CS.periodic_cube(side, seed=7)
        n = case.n
        sim = S.Simulation(case, precision=S.SPH_PREC_F32)
        sim.build_cells()
        A = torch.rand(n, device="cuda")
        m = torch.full((n,), case.mass, device="cuda")
        rho = torch.full((n,), case.rho0, device="cuda")
        Sbuf = torch.empty(n, device="cuda")
        reps = max(20, min(2000, int(4e8 // n)))

        def op():
            S.sph_sample(sim.ctx, A.data_ptr(), m.data_ptr(), rho.data_ptr(), Sbuf.data_ptr())

        for _ in range(3):
            op()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            op()
        e1.record(st)
        e1.synchronize()
        ms_eager = e0.elapsed_time(e1) / reps
        # the same calls captured in a CUDA graph (the library call allocates
        # and synchronises nothing): small sizes are otherwise bound by the
        # host's launch rate, not by the GPU
        per_graph = 50
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(st)
        with torch.cuda.stream(cap):
            op()
        st.wait_stream(cap)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            for _ in range(per_graph):
                op()
        g.replay()
        torch.cuda.synchronize()
        nrep = max(1, reps // per_graph)
        e0.record(st)
        for _ in range(nrep):
            g.replay()
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / (nrep * per_graph)
        del g
        rb = max(5, reps // 10)
        e0.record(st)
        for _ in range(rb):
            sim.build_cells()
            op()
        e1.record(st)
        e1.synchronize()
        ms_b = e0.elapsed_time(e1) / rb
        row = {"n": n, "n_side": side, "op_ms": ms, "op_particles_per_s": n / (ms * 1e-3),
               "op_ms_eager": ms_eager, "with_build_ms": ms_b,
               "with_build_particles_per_s": n / (ms_b * 1e-3), "reps": reps}
        if side == max(sides):
            counts = torch.zeros(n, dtype=torch.int32, device="cuda")
            S.sph_neighbor_counts(sim.ctx, sim._view, counts.data_ptr())
            hits = int(counts.sum().item()) + n
            cand = candidates_bc(sim.cell_table(), 3, case.ncell, case.bc)
            flops = cand * FLOPS_CAND[3] + hits * FLOPS_HIT_SAMPLE
            row.update({"candidates": cand, "hits": hits, "flops_per_call": flops,
                        "achieved_tflops": flops / (ms * 1e-3) / 1e12})
            peaks, _ = _peaks()
            alu = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
            out["roofline"] = {"bound": "alu", "kernel": "k_sample<3,float> (+ k_sample_prep)",
                               "achieved": row["achieved_tflops"], "peak": alu, "unit": "TFLOP/s",
                               "frac": row["achieved_tflops"] / alu,
                               "traffic": secondary_traffic("k_sample", n)[0],
                               "traffic_note": secondary_traffic("k_sample", n)[1],
                               "n": n}
        out["sizes"].append(row)
        sim.close()
    # the paper's benchmark size and its published peak (12 CPU threads,
    # other hardware): context only
    out["paper"] = {"n": 3375, "particles_per_s": 1.05e3, "threads": 12, "code": "Nauticle (interpreted SFL)"}
    if cpu_side:
        from oracle import oracle as O
        case = CS.periodic_cube(cpu_side, seed=7)
        p = O.bc_params(case, fp32=True)
        t0 = time.perf_counter()
        O.bc_sample(p, case.r, case.id, case.extra["A"], case.extra["m"], case.rho)
        sec = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": case.n / sec, "unit": "particles/s", "cores": O.num_threads(),
                               "kind": "oracle", "sample": f"1 oracle evaluation, {case.n} particles "
                               "(cell build included)"}
    return out


def adjoint_forward_ratio(S, torch, steps=200, k=20):
    """Differentiable 2D workload (128x128 fluid, FP32 form): time of the
    backward pass (segment recompute + adjoint kernels) over the forward
    rollout (with checkpoint copies), CUDA events on the current stream."""
    from paper_1710_08259_gb300 import autograd as AG
    from paper_1710_08259_gb300 import cases as CS
    case = CS.diff_case(steps=steps)
    st = torch.cuda.current_stream()
    res = {}
    for graphs in (True, False):
        out = []
        for rep in range(2):  # the first repetition warms up
            v = torch.tensor(case.v, dtype=torch.float64, device="cuda", requires_grad=True)
            a = torch.tensor(case.alpha, dtype=torch.float64, requires_grad=True)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize()
            e[0].record(st)
            rf, ids = AG.rollout(v, a, case, S.SPH_PREC_F32, steps, k, graphs=graphs)
            e[1].record(st)
            L = AG.target_loss(rf, ids, case, case.target)
            L.backward()
            e[2].record(st)
            e[2].synchronize()
            out = [e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])]
        res[graphs] = out
    # no checkpoints: every step's build products kept (memory for recompute)
    for rep in range(2):
        v = torch.tensor(case.v, dtype=torch.float64, device="cuda", requires_grad=True)
        a = torch.tensor(case.alpha, dtype=torch.float64, requires_grad=True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record(st)
        rf, ids = AG.rollout(v, a, case, S.SPH_PREC_F32, steps, 0)
        e[1].record(st)
        L = AG.target_loss(rf, ids, case, case.target)
        L.backward()
        e[2].record(st)
        e[2].synchronize()
        keep = [e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])]
    out = res[True]
    return {"ratio": out[1] / out[0], "forward_ms": out[0], "backward_ms": out[1], "steps": steps,
            "checkpoint_every": k, "workload": "diff_2d_128x128_fp32", "segments_as_cuda_graphs": True,
            "eager": {"ratio": res[False][1] / res[False][0], "forward_ms": res[False][0],
                      "backward_ms": res[False][1]},
            "no_checkpoints": {"ratio": keep[1] / keep[0], "forward_ms": keep[0], "backward_ms": keep[1],
                               "note": "every step's build products kept: no recompute"}}


def _time_batch(S, torch, cases, tune, steps):
    """(ms for `steps` steps in one call, info, status) of one batched form."""
    b = S.Batch(cases, S.SPH_PREC_F32, tune=tune)
    b.step(steps)  # capture + warm-up with the same step count
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(steps)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    info = b.info()
    status = b.status()
    b.close()
    return ms, info, status


def batched_rate(S, torch, steps=50, seq_steps=3):
    """Batched workload: 256 dam breaks of 1k-64k fluid (log-uniform), FP32,
    all advanced together, steps per call through one CUDA graph: in the
    form and launch shape the autotuner picks, and in the persistent form
    (one cooperative launch per call) with its best shape.  Also the same
    cases stepped one after another through sph_step, for the
    launch-overhead comparison."""
    from paper_1710_08259_gb300 import cases as CS
    from paper_1710_08259_gb300 import tune as TU
    cases = CS.batched_cases()
    nf = sum(c.n_fluid for c in cases)
    best = TU.autotune(cases, S.SPH_PREC_F32, steps=3)
    ms, info, status = _time_batch(S, torch, cases, TU.tune_struct(best), steps)
    pers = [r for r in best.get("tried", []) if r.get("form", "persistent") == "persistent"]
    if best.get("form", "persistent") == "persistent" or not pers:
        ms_p, info_p, status_p = ms, info, status
        best_p = best
    else:
        best_p = min(pers, key=lambda r: r["ms_per_step"])
        ms_p, info_p, status_p = _time_batch(S, torch, cases, TU.tune_struct(best_p), steps)
    # the same cases, one sph_step call per case and step (seq_steps 0: not run)
    seq = None
    if seq_steps > 0:
        sims = [S.Simulation(c, precision=S.SPH_PREC_F32) for c in cases]
        for sm in sims:
            sm.step(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(seq_steps):
            for sm in sims:
                sm.step(1)
        e1.record()
        e1.synchronize()
        ms_seq = e0.elapsed_time(e1)
        for sm in sims:
            sm.close()
        seq = {"value": nf * seq_steps / (ms_seq * 1e-3), "ms_per_step": ms_seq / seq_steps}
    return {"value": nf * steps / (ms * 1e-3), "unit": "fluid particle-steps/s", "ms_per_step": ms / steps,
            "steps_per_launch": steps, "ncases": len(cases), "n_fluid": nf,
            "n_particles": sum(c.n for c in cases),
            "tune": {k: best.get(k, "persistent") for k in ("form", "block", "blocks_per_sm")},
            "graph_used": info["graph_used"], "grid": info["grid"], "status": status | status_p,
            "persistent": {"value": nf * steps / (ms_p * 1e-3), "ms_per_step": ms_p / steps,
                           "block": best_p["block"], "blocks_per_sm": best_p["blocks_per_sm"],
                           "grid": info_p["grid"], "graph_used": info_p["graph_used"],
                           "note": "one cooperative launch per call, 8 grid barriers per step"},
            "sequential_sph_step": seq}


def run_reference(case, steps, warmup):
    """The CPU FP64 oracle on the host cores: `warmup` untimed then `steps`
    timed oracle steps of the full workload, each from the state the last one
    left (the oracle as it stands, all host cores through OpenMP)."""
    from oracle import oracle as O
    O.lib()
    cores = O.num_threads()
    p = O.params(case)
    r, v = case.r, case.v
    for _ in range(max(0, warmup)):
        res = O.step(p, r, v, case.kind, case.id, 1)
        r, v = res.r, res.v
    times = []
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        res = O.step(p, r, v, case.kind, case.id, 1)
        times.append(time.perf_counter() - t0)
        r, v = res.r, res.v
    tot = sum(times)
    value = case.n_fluid * len(times) / tot
    return {"value": value, "cores": cores, "steps": len(times), "warmup": max(0, warmup),
            "sample": f"{len(times)} timed oracle step(s) of the full case ({case.n} particles) after "
            f"{max(0, warmup)} untimed, from the initial state", "seconds": tot}


# DRAM bytes (read + write) per launch from ncu captures.  Per kernel: the
# workload that was captured, its particle count, the bytes per launch, the
# commit whose kernel source was captured, and the summary under profiles/.
# A run of the same kernel on another dam break reports these bytes scaled by
# its particle count (the kernel's traffic is per particle: the state it reads
# and the mask words it writes); a kernel changed since its capture reports
# no traffic until it is captured again.
NCU_CAPTURES = {
    "k_density<3,float,2>": {"workload": "dam_break_3d_256^3", "n_particles": 19507924, "dram_bytes": 3314.1e6,
                             "commit": "08a1c7e", "summary": "profiles/sph_step_dam_break_3d_256cubed_launches.md"},
}
# kernels whose source changed after their capture (their figures are stale)
NCU_STALE = set()


def traffic_from_capture(kernel, workload, n_particles):
    """(DRAM bytes per launch or None, how the figure was obtained)."""
    cap = NCU_CAPTURES.get(kernel)
    if cap is None or kernel in NCU_STALE:
        return None, "no ncu capture of the current kernel"
    if cap["workload"] == workload:
        return cap["dram_bytes"], f"ncu capture of this workload (commit {cap['commit']}, {cap['summary']})"
    scaled = cap["dram_bytes"] * n_particles / cap["n_particles"]
    return scaled, (f"ncu capture of {cap['workload']} ({cap['n_particles']} particles, commit {cap['commit']}, "
                    f"{cap['summary']}) scaled by the particle count")


def timed_steps(S, torch, sim, steps, warmup, barrier=None):
    """Run warmup untimed steps, then time `steps` steps with CUDA events on
    the launching stream (phase events recorded by the library).  Returns
    (ms, phase ms summed, profiled steps, diag of the last step)."""
    stream = torch.cuda.current_stream()
    sim.step(max(3, warmup))
    (barrier or torch.cuda.synchronize)()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    S.sph_profile_begin(sim.ctx, steps)
    e0.record(stream)
    if steps > 1:
        sim.step(steps - 1)
    d = sim.step(1, diag=True)
    e1.record(stream)
    e1.synchronize()
    prof, nprof = S.sph_profile_end(sim.ctx)
    (barrier or torch.cuda.synchronize)()
    return e0.elapsed_time(e1), prof, nprof, d


def dam_break_roofline(S, sim, case, workload, ms, prof, nprof, d):
    """Work counts of the last timed step and the roofline of the dominant
    kernel (the density pass) against the FP32 ALU peak."""
    kind_sorted = sim.state.kind.cpu().numpy()
    r_now = np.stack([t.cpu().numpy() for t in sim.state.r], axis=1)
    cand_fluid, cand_all = candidates_method(r_now, kind_sorted, case.dom_min, case.h, case.dim)
    k_cells = int(round(2.0 * case.h / case.cs))
    pairs_all = int(d.n_pairs)
    pairs_fluid = int(d.n_pairs_fluid)
    dim = case.dim
    steps = max(nprof, 1)
    force_flops = pairs_fluid * FLOPS_PAIR_FORCE[dim]
    dens_flops = cand_all * FLOPS_CAND[dim] + (pairs_all + case.n) * FLOPS_PAIR_DENSITY[dim]
    force_ms = prof["force"] / steps
    dens_ms = prof["density"] / steps
    peaks, peak_src = _peaks()
    alu_peak = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    force_tf = force_flops / (force_ms * 1e-3) / 1e12
    dens_tf = dens_flops / (dens_ms * 1e-3) / 1e12
    kernel = f"k_density<{dim},float,{k_cells}>"
    traffic, tnote = traffic_from_capture(kernel, workload, case.n)
    cap = NCU_CAPTURES.get(kernel, {})
    ms_step = ms / max(nprof, 1)
    return {"bound": "alu", "kernel": kernel, "achieved": dens_tf, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": dens_tf / alu_peak, "traffic": traffic, "traffic_note": tnote,
            "ncu_capture": ({k: cap[k] for k in ("workload", "commit", "summary")}
                            if traffic is not None else None),
            "peak_source": f"FP32 ALU: 152 SMs x 128 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                           f"(max SM clock; SM clock from the {peak_src} peaks file)",
            "flops_per_launch": dens_flops, "launch_ms": dens_ms, "timing": "CUDA events around each launch of "
            "the timed steps (sph_profile_begin/end), on the launching stream",
            "candidates_per_launch": cand_all, "pairs_per_launch": pairs_all,
            "search": {"cells_per_radius": k_cells, "cell_edge_m": case.cs,
                       "note": "candidates_per_launch: the paper's search (cells of edge 2h, 3^D stencil), the "
                               "algorithmic unit; cells of edge h (5^D stencil walked as rows, trimmed by the "
                               "gap test) test fewer of them"},
            "force_kernel": {"achieved": force_tf, "frac": force_tf / alu_peak, "launch_ms": force_ms,
                             "flops_per_launch": force_flops, "pairs_per_launch": pairs_fluid},
            "build_ms": prof["build"] / steps,
            # the whole step against the FP32 ALU peak: the algorithmic FLOPs of
            # both pair passes over the measured time per step
            "step": {"flops_per_step": dens_flops + force_flops,
                     "achieved": (dens_flops + force_flops) / (ms_step * 1e-3) / 1e12,
                     "frac": (dens_flops + force_flops) / (ms_step * 1e-3) / 1e12 / alu_peak}}


def fp64_path(S, torch, case, steps, warmup=1):
    """The plain FP64 GPU path (every kernel templated on double) on the same
    workload: ms per step over `steps` steps after `warmup`."""
    stream = torch.cuda.current_stream()
    sim64 = S.Simulation(case, precision=S.SPH_PREC_F64)
    sim64.step(max(1, warmup))
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    d = sim64.step(steps, diag=True)
    a1.record(stream)
    a1.synchronize()
    ms64 = a0.elapsed_time(a1) / steps
    out = {"value": case.n_fluid / (ms64 * 1e-3), "ms_per_step": ms64, "steps": steps, "warmup": max(1, warmup),
           "pair_interactions_per_s": int(d.n_pairs) / (ms64 * 1e-3), "status": sim64.status()}
    sim64.close()
    del sim64
    return out


def secondary_dam_break(S, torch, case, workload, steps, warmup, fp64_steps):
    """Another dam-break workload in the FP32 form (rate, phases, roofline of
    its density pass) beside its plain FP64 GPU path."""
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)
    ms, prof, nprof, d = timed_steps(S, torch, sim, steps, warmup)
    value = case.n_fluid * steps / (ms * 1e-3)
    out = {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup": max(3, warmup),
           "workload": workload, "n_fluid": case.n_fluid, "n_particles": case.n,
           "pair_interactions_per_s": int(d.n_pairs) * steps / (ms * 1e-3),
           "phase_ms_per_step": {k: v / max(nprof, 1) for k, v in prof.items()},
           "roofline": dam_break_roofline(S, sim, case, workload, ms, prof, nprof, d), "status": sim.status()}
    sim.close()
    if fp64_steps > 0:
        out["fp64_path"] = fp64_path(S, torch, case, fp64_steps)
        out["speedup_vs_fp64"] = value / out["fp64_path"]["value"]
    return out


def dam_break_2d_fp64_config(S, torch, steps=100, warmup=3):
    """The 2D dam break (64 x 64 fluid, 100 steps) in the plain FP64 form it
    is specified in, and the FP32 form on the same workload: 100-step rollouts
    timed with CUDA events (one sph_step call per rollout)."""
    from paper_1710_08259_gb300 import cases as CS
    case = CS.dam_break_2d()
    stream = torch.cuda.current_stream()
    out = {"workload": "dam_break_2d_64x64", "n_fluid": case.n_fluid, "n_particles": case.n, "steps": steps}
    for name, prec in (("fp64", S.SPH_PREC_F64), ("fp32", S.SPH_PREC_F32)):
        best = None
        for rep in range(warmup + 3):
            sim = S.Simulation(case, precision=prec)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            d = sim.step(steps, diag=True)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            status = sim.status()
            sim.close()
            if rep >= warmup and (best is None or ms < best[0]):
                best = (ms, int(d.n_pairs), status)
        ms, pairs, status = best
        out[name] = {"value": case.n_fluid * steps / (ms * 1e-3), "unit": UNIT, "ms_per_rollout": ms,
                     "ms_per_step": ms / steps, "pair_interactions_per_s": pairs * steps / (ms * 1e-3),
                     "status": status, "timing": f"best of 3 rollouts after {warmup} untimed"}
    out["speedup_fp32_vs_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    out["note"] = ("5,074 particles: every kernel is under one wave, so both forms are bound by the 9 launches "
                   "of each step, not by arithmetic")
    return out


WORKLOADS = {
    "large": ("dam_break_3d_256^3", "dam_break_3d_large"),
    "3d": ("dam_break_3d_100^3", "dam_break_3d"),
    "3d_small": ("dam_break_3d_40^3", None),
    "2d": ("dam_break_2d_64x64", "dam_break_2d"),
}


def make_case(name):
    from paper_1710_08259_gb300 import cases as CS
    if name == "large":
        return CS.dam_break_3d_large()
    if name == "3d":
        return CS.dam_break_3d()
    if name == "3d_small":
        return CS.dam_break_3d(n=40, dx=0.005, tank=(0.64, 0.24, 0.24))
    return CS.dam_break_2d()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200,
                    help="timed steps of the headline (default: the large dam break's 200-step run)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default="large", choices=["large", "3d", "2d", "3d_small"],
                    help="headline workload: large = the 256^3 dam break (19.5 M particles, the largest "
                         "configuration), 3d = 100^3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-secondary", dest="secondary", action="store_false",
                    help="skip the 100^3 and 2D FP64 keys")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-example-1a", dest="example_1a", action="store_false")
    ap.add_argument("--no-sampling", dest="sampling", action="store_false")
    ap.add_argument("--no-dem", dest="dem", action="store_false")
    ap.add_argument("--dem-side", type=int, default=100, help="dem leg: spheres per tank edge")
    ap.add_argument("--no-laws", dest="laws", action="store_false")
    ap.add_argument("--leg", default="all", choices=["all", "example_1a", "sampling", "dem", "laws", "batched"],
                    help="example_1a / sampling: run only that leg (--steps steps, --scale, --sides) and "
                         "print its JSON object (for profiling); all: the benchmark line")
    ap.add_argument("--scale", type=int, default=64, help="example_1a leg: refinement of Appendix A")
    ap.add_argument("--sides", default="15,46,100,252", help="sampling leg: cube edges in particles")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.case][0] + "_fp32"

    if args.impl == "reference":
        if world > 1 and rank != 0:
            return 0
        case = make_case(args.case)
        # full oracle steps of the workload; capped so that the whole run stays
        # within a few minutes on the host cores (the 256^3 step takes seconds)
        steps, warmup = max(1, min(args.steps, 20)), max(0, min(args.warmup, 5))
        cb = run_reference(case, steps, warmup)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
                "steps": cb["steps"], "warmup": cb["warmup"], "ms_per_step": 1e3 * cb["seconds"] / cb["steps"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded dam break)",
                "config": {"workload": wl, "n_fluid": case.n_fluid, "n_particles": case.n,
                           "reference": "the CPU FP64 oracle (the paper ships no code)"},
                "cpu_baseline": {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                                 "sample": cb["sample"]},
                "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1710_08259_gb300 import build as B
    B.build()
    from paper_1710_08259_gb300 import sph as S

    sides = tuple(int(x) for x in args.sides.split(","))
    if args.leg == "example_1a":
        print(json.dumps({"leg": "example_1a", **example_1a_rate(S, torch, scale=args.scale,
                                                                  steps=max(2, args.steps), cpu=False)}))
        return 0
    if args.leg == "sampling":
        print(json.dumps({"leg": "sampling", **sampling_rates(S, torch, sides=sides, cpu_side=0)}))
        return 0
    if args.leg == "laws":
        print(json.dumps({"leg": "laws", **laws_rates(S, torch, steps=max(2, args.steps))}))
        return 0
    if args.leg == "dem":
        print(json.dumps({"leg": "dem", **dem_rate(S, torch, n_side=args.dem_side, steps=max(2, args.steps),
                                                   cpu=False)}))
        return 0
    if args.leg == "batched":
        print(json.dumps({"leg": "batched", **batched_rate(S, torch, steps=max(2, args.steps), seq_steps=0)}))
        return 0

    case = make_case(args.case)
    sim = S.Simulation(case, precision=S.SPH_PREC_F32)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(gpu_index=int(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local, period_ms=50)
    sim.step(max(3, args.warmup))
    barrier()
    clocks.start()
    time.sleep(0.2)   # the sampler's first sample lands inside the timed region
    ms, prof, nprof, d = timed_steps(S, torch, sim, args.steps, 0, barrier=barrier)
    clk = clocks.stop()
    ms, units_all = aggregate_replicas(ms, float(case.n_fluid * args.steps), world, dev)
    status = sim.status()
    steps_total = args.steps
    value = units_all / (ms * 1e-3)
    pairs_all = int(d.n_pairs)
    pair_rate = pairs_all * steps_total * world / (ms * 1e-3)
    roof = dam_break_roofline(S, sim, case, WORKLOADS[args.case][0], ms, prof, nprof, d)

    fp64 = fp64_path(S, torch, case, args.fp64_steps) if args.fp64_steps > 0 else None

    # end to end through the C ABI with host buffers: every step, sph_step_host
    # copies the inputs in (over the context's copy streams), steps, and
    # writes the new state back to the page-locked host arrays
    st = sim.state
    host = {"r": [t.cpu().pin_memory() for t in st.r], "v": [t.cpu().pin_memory() for t in st.v],
            "rho": st.rho.cpu().pin_memory(), "p": st.p.cpu().pin_memory(), "id": st.id.cpu().pin_memory(),
            "kind": st.kind.cpu().pin_memory()}
    hview = S.host_state_view(host)
    h2d = sum(t.numel() * t.element_size() for t in host["r"] + host["v"]) + host["id"].numel() * 4 + \
        host["kind"].numel()
    d2h = h2d + 2 * st.n * st.rho.element_size()

    def e2e_step():
        S.sph_step_host(sim.ctx, hview, 1)

    for _ in range(3):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms, e2e_units = aggregate_replicas((time.perf_counter() - t0) * 1e3, float(case.n_fluid * args.e2e_steps),
                                           world, dev)
    e2e_val = e2e_units / (e2e_ms * 1e-3)
    sim.close()
    del host, hview

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.cpu_steps > 0:
        cb = run_reference(case, args.cpu_steps, 0)
        cpu = {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle", "sample": cb["sample"]}

    secondary = {}
    if args.secondary:
        if args.case != "3d":
            secondary["dam_break_3d_100cubed"] = secondary_dam_break(S, torch, make_case("3d"), "dam_break_3d_100^3",
                                                                     200, 10, 3)
        secondary["dam_break_2d_64x64_fp64"] = dam_break_2d_fp64_config(S, torch)

    adj = adjoint_forward_ratio(S, torch) if args.adjoint else None
    batched = batched_rate(S, torch) if args.batched else None
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    ex1a = example_1a_rate(S, torch, cpu=want_cpu) if args.example_1a else None
    sampling = sampling_rates(S, torch, sides=sides, cpu_side=100 if want_cpu else 0) if args.sampling else None
    dem = dem_rate(S, torch, n_side=args.dem_side, cpu=want_cpu) if args.dem else None
    laws = laws_rates(S, torch) if args.laws else None

    kernels_per_step = 9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps_total,
        "warmup": max(3, args.warmup), "ms_per_step": ms / steps_total, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 pair sums, f64 positions",
        "data": "synthetic (seeded dam break)",
        "config": {"workload": wl, "n_fluid": case.n_fluid, "n_particles": case.n, "precision": "fp32+kahan",
                   "l2": "inputs larger than L2 (state + workspace ~%.1f GB)" % (case.n * 300 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "pair_interactions_per_s": pair_rate,
        "n_pairs_per_step": pairs_all,
        "fp64_path": fp64,
        "speedup_vs_fp64": (value / world) / fp64["value"] if fp64 else None,
        "phase_ms_per_step": {k: v / max(nprof, 1) for k, v in prof.items()},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "call": "sph_step_host, page-locked host state", "steps": args.e2e_steps},
        "gpu_launches": kernels_per_step * steps_total,
        "clocks": clk,
        "status": status,
        **secondary,
        "adjoint_forward_ratio": adj["ratio"] if adj else None,
        "adjoint": adj,
        "batched": batched,
        "example_1a": ex1a,
        "sampling": sampling,
        "dem": dem,
        "compiled_laws": laws,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

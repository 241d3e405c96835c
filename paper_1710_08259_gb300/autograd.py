"""Differentiable SPH rollout: torch.autograd.Function over sph_step /
sph_step_adjoint with checkpointing.

Forward: nsteps calls of sph_step from (r0, v0) with viscosity alpha; the
state (r, v, id, kind) is stored every `k` steps, and the steps of the last
segment keep their build and density products (sph_build_save).  Backward:
for each segment, last first, the segment is recomputed from its checkpoint
(not the last one: its products are kept), keeping each recomputed step's
build and density products, then the hand-written adjoint kernels run one
step at a time in reverse on them (sph_adjoint_of_saved, in place),
carrying (dL/dr, dL/dv) and accumulating dL/dalpha on the device.  Memory:
nsteps/k checkpoints, each n x (3 doubles + 3 velocity words + 5 bytes) in
one contiguous buffer, plus two sets of k build products (~100 bytes per
particle each).  The repeated
full segments of both sweeps replay CUDA graphs (the launch sequence of one
segment, captured once), so a small case is not bound by launch overhead.

The loss is whatever the caller builds from the returned final positions
(in the final state's order, given by the returned ids).
"""
from __future__ import annotations

import math
import numpy as np
import torch

from . import sph as S


class _Packed:
    """One particle state in one contiguous device buffer: r (dim x n
    float64), v (dim x n, the working precision), id (n int32) and kind (n
    uint8), so that a snapshot or a restore is a single copy.  The density
    and pressure scratch (rho, p) is not part of the snapshot and may be
    shared between states."""

    def __init__(self, n, dim, tdt, core=None, scratch=None):
        es = 4 if tdt == torch.float32 else 8
        offs, o = {}, 0
        for name, size in (("r", dim * n * 8), ("v", dim * n * es), ("id", n * 4), ("kind", n)):
            offs[name] = o
            o += size
        self.nbytes = (o + 15) // 16 * 16
        self.core = core if core is not None else torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        c = self.core
        self.r = [c[offs["r"] + d * n * 8: offs["r"] + (d + 1) * n * 8].view(torch.float64) for d in range(dim)]
        self.v = [c[offs["v"] + d * n * es: offs["v"] + (d + 1) * n * es].view(tdt) for d in range(dim)]
        self.id = c[offs["id"]: offs["id"] + 4 * n].view(torch.int32)
        self.kind = c[offs["kind"]: offs["kind"] + n]
        if scratch is None:
            scratch = (torch.zeros(n, dtype=tdt, device="cuda"), torch.zeros(n, dtype=tdt, device="cuda"))
        self.rho, self.p = scratch
        self.n, self.dim = n, dim

    def view(self) -> S.SphState:
        st = S.SphState()
        st.n = self.n
        for k in range(3):
            st.r[k] = self.r[k].data_ptr() if k < self.dim else None
            st.v[k] = self.v[k].data_ptr() if k < self.dim else None
        st.rho = self.rho.data_ptr()
        st.p = self.p.data_ptr()
        st.id = self.id.data_ptr()
        st.kind = self.kind.data_ptr()
        return st


class _Engine:
    """A context (one alpha) and the device buffers of one rollout."""

    def __init__(self, case, precision, alpha, graphs=True, reuse_builds=True, **params):
        self.case = case
        self.precision = precision
        self.alpha = float(alpha)
        self.params = S.params_from_case(case, precision=precision, alpha=self.alpha, **params)
        self.ctx = S.sph_create(self.params, case.n)
        self.tdt = torch.float32 if precision == S.SPH_PREC_F32 else torch.float64
        self.graphs = graphs
        self.reuse_builds = reuse_builds
        # the last segment's build + density products, kept by the forward
        # sweep (its reverse steps then recompute nothing); None: not kept
        self.last_rows = None

    def close(self):
        if self.ctx:
            S.sph_destroy(self.ctx)
            self.ctx = None

    def packed(self, core=None, scratch=None):
        return _Packed(self.case.n, self.case.dim, self.tdt, core, scratch)


def _capture(fn):
    """fn's launches captured in a CUDA graph (after fn ran once eagerly, so
    that every kernel it launches is loaded)."""
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def rollout_forward(engine: _Engine, r0, v0, ids0, kind0, nsteps: int, k: int):
    """Run nsteps; return (final state, checkpoints): checkpoints[seg] is the
    packed state at step seg * k.  Full segments after the first replay one
    CUDA graph of k steps when engine.graphs is set."""
    live = engine.packed()
    for d in range(engine.case.dim):
        live.r[d].copy_(r0[d])
        live.v[d].copy_(v0[d])
    live.id.copy_(ids0)
    live.kind.copy_(kind0)
    view = live.view()
    if k <= 0:
        # no checkpoints: every step's build and density products are kept
        # (~100 B per particle and step), so the reverse sweep recomputes nothing
        prods = None
        for s in range(nsteps):
            S.sph_step(engine.ctx, view, 1)
            if prods is None:
                prods = torch.empty((nsteps, S.sph_build_save(engine.ctx)), dtype=torch.uint8, device="cuda")
            S.sph_build_save(engine.ctx, prods[s].data_ptr())
        return live, prods
    nseg = max(1, math.ceil(nsteps / k))
    ckpt = torch.empty((nseg, live.nbytes), dtype=torch.uint8, device="cuda")
    full = nsteps // k

    def seg_steps(m):
        for _ in range(m):
            S.sph_step(engine.ctx, view, 1)

    graph = None
    engine.last_rows = None
    for seg in range(nseg):
        ckpt[seg].copy_(live.core)
        m = min(k, nsteps - seg * k)
        if seg == nseg - 1 and engine.reuse_builds:
            # the last segment keeps its steps' products: the reverse sweep
            # would recompute exactly these
            for j in range(m):
                S.sph_step(engine.ctx, view, 1)
                if engine.last_rows is None:
                    engine.last_rows = torch.empty((m, S.sph_build_save(engine.ctx)), dtype=torch.uint8,
                                                   device="cuda")
                S.sph_build_save(engine.ctx, engine.last_rows[j].data_ptr())
            continue
        if graph is not None and m == k:
            graph.replay()
            continue
        seg_steps(m)
        if engine.graphs and m == k and seg + 1 < full:
            graph = _capture(lambda: seg_steps(k))
    return live, ckpt


def rollout_backward(engine: _Engine, ckpt, nsteps: int, k: int, gr_final, gv_final):
    """Reverse sweep.  gr_final/gv_final: lists of dim device tensors in the
    final state's order.  Returns (gr0, gv0, alpha_bar) in the initial order.

    Each segment, last first: restore its checkpoint, recompute its steps
    storing each step's input state, then run the adjoint kernels one step
    at a time in reverse, carrying (dL/dr, dL/dv) and accumulating dL/dalpha
    on the device.  With engine.graphs, the full segments after the first
    one processed replay one CUDA graph of the whole segment."""
    dim = engine.case.dim
    grA = [g.to(torch.float64).clone() for g in gr_final]
    gvA = [g.to(engine.tdt).clone() for g in gv_final]
    grB = [torch.empty_like(g) for g in grA]
    gvB = [torch.empty_like(g) for g in gvA]
    gA, gB = S.grad_view(grA, gvA), S.grad_view(grB, gvB)
    abar = torch.zeros(1, dtype=torch.float64, device="cuda")
    if k <= 0:
        # every step's products were kept by the forward sweep
        n = engine.case.n
        src, dst = gA, gB
        for s in reversed(range(nsteps)):
            S.sph_adjoint_of_saved(engine.ctx, ckpt[s].data_ptr(), n, src, dst, abar.data_ptr())
            src, dst = dst, src
        if src is gB:
            for d in range(dim):
                grA[d].copy_(grB[d])
                gvA[d].copy_(gvB[d])
        return grA, gvA, abar
    seg_in = engine.packed()
    live = engine.packed()
    live_view = live.view()
    kk = min(k, nsteps)
    n = engine.case.n
    if engine.reuse_builds:
        # each recomputed step's build + density products, kept for its
        # reverse step (the forward sweep left a density pass: sizes known)
        bbytes = S.sph_build_save(engine.ctx)
        rows = torch.empty((max(kk, 1), bbytes), dtype=torch.uint8, device="cuda")
    else:
        # each recomputed step's input state, rebuilt by its reverse step
        rows = torch.empty((max(kk, 1), live.nbytes), dtype=torch.uint8, device="cuda")
        scratch = (live.rho, live.p)
        states = [engine.packed(rows[j], scratch) for j in range(kk)]
        views = [s.view() for s in states]
    nseg = max(1, math.ceil(nsteps / k))

    def segment(m):
        live.core.copy_(seg_in.core)
        for j in range(m):
            if not engine.reuse_builds:
                rows[j].copy_(live.core)
            S.sph_step(engine.ctx, live_view, 1)
            if engine.reuse_builds:
                S.sph_build_save(engine.ctx, rows[j].data_ptr())
        src, dst = gA, gB
        for j in reversed(range(m)):
            if engine.reuse_builds:
                S.sph_adjoint_of_saved(engine.ctx, rows[j].data_ptr(), n, src, dst, abar.data_ptr())
            else:
                S.sph_step_adjoint(engine.ctx, views[j], src, dst, abar.data_ptr())
            src, dst = dst, src
        if src is gB:   # an odd number of steps: the result back into A
            for d in range(dim):
                grA[d].copy_(grB[d])
                gvA[d].copy_(gvB[d])

    graph = None
    full_left = nsteps // k
    last = engine.last_rows if engine.reuse_builds else None
    for seg in reversed(range(nseg)):
        m = min(k, nsteps - seg * k)
        if m <= 0:
            continue
        if seg == nseg - 1 and last is not None:
            # kept by the forward sweep: the adjoint steps alone
            src, dst = gA, gB
            for j in reversed(range(m)):
                S.sph_adjoint_of_saved(engine.ctx, last[j].data_ptr(), n, src, dst, abar.data_ptr())
                src, dst = dst, src
            if src is gB:
                for d in range(dim):
                    grA[d].copy_(grB[d])
                    gvA[d].copy_(gvB[d])
            if m == k:
                full_left -= 1
            continue
        seg_in.core.copy_(ckpt[seg])
        if graph is not None and m == k:
            graph.replay()
            continue
        segment(m)
        if m == k:
            full_left -= 1
            if engine.graphs and full_left > 0:
                graph = _capture(lambda: segment(k))
    return grA, gvA, abar


class SPHRollout(torch.autograd.Function):
    """r_final = rollout(v0, alpha).  Inputs: v0 (n, dim) device tensor in the
    case's particle order, alpha a 0-d tensor.  Outputs: final positions
    (n, dim) float64 and the final ids (int32, not differentiable)."""

    @staticmethod
    def forward(ctx, v0, alpha, case, precision, nsteps, k, params=None, graphs=True, reuse_builds=True):
        dim = case.dim
        eng = _Engine(case, precision, float(alpha.item()), graphs=graphs, reuse_builds=reuse_builds,
                      **(params or {}))
        r0 = [torch.tensor(np.ascontiguousarray(case.r[:, d]), dtype=torch.float64, device="cuda")
              for d in range(dim)]
        v0l = [v0[:, d].detach().to(eng.tdt).contiguous() for d in range(dim)]
        ids0 = torch.tensor(case.id.astype(np.int32), device="cuda")
        kind0 = torch.tensor(case.kind, dtype=torch.uint8, device="cuda")
        st, ckpt = rollout_forward(eng, r0, v0l, ids0, kind0, nsteps, k)
        ctx.eng = eng
        ctx.ckpt = ckpt
        ctx.nsteps = nsteps
        ctx.k = k
        ctx.v0_dtype = v0.dtype
        rf = torch.stack(st.r, dim=1)
        ctx.mark_non_differentiable(st.id)
        return rf, st.id

    @staticmethod
    def backward(ctx, grad_rf, grad_ids):
        eng = ctx.eng
        dim = eng.case.dim
        gr = [grad_rf[:, d].contiguous() for d in range(dim)]
        gv = [torch.zeros(eng.case.n, dtype=eng.tdt, device="cuda") for _ in range(dim)]
        gr0, gv0, abar = rollout_backward(eng, ctx.ckpt, ctx.nsteps, ctx.k, gr, gv)
        eng.close()
        gv0t = torch.stack(gv0, dim=1).to(ctx.v0_dtype)
        return gv0t, abar.reshape(()).to(torch.float64), None, None, None, None, None, None, None


def rollout(v0, alpha, case, precision=S.SPH_PREC_F32, nsteps: int = 200, k: int = 20, graphs: bool = True,
            reuse_builds: bool = True, **params):
    """Differentiable rollout (see SPHRollout); params go to params_from_case
    (e.g. clamp_neg_p=False).  graphs: replay the repeated segments of the
    forward and backward sweeps as CUDA graphs (same kernels, same order:
    the results are identical to the eager sweep).  reuse_builds: each
    reverse step loads the build and density products its recomputed
    forward step saved (sph_build_save / sph_adjoint_of_saved, read in
    place) instead of rebuilding them from the state (the
    same values: identical results).  k <= 0: no checkpoints; the forward
    sweep keeps every step's build products (~100 B per particle and step:
    memory for speed), and the reverse sweep recomputes nothing."""
    return SPHRollout.apply(v0, alpha, case, precision, nsteps, k, params or None, graphs, reuse_builds)


def target_loss(rf, ids, case, target):
    """mean over fluid of |r_final - target|^2 with target indexed by id."""
    tgt = torch.as_tensor(target, dtype=torch.float64, device=rf.device)
    ids_l = ids.long()
    fl = ids_l < case.n_fluid  # fluid particles carry ids 0..n_fluid-1
    d = rf[fl] - tgt[ids_l[fl]]
    return (d * d).sum(dim=1).mean()

"""Differentiable SPH rollout: torch.autograd.Function over sph_step /
sph_step_adjoint with checkpointing.

Forward: nsteps calls of sph_step from (r0, v0) with viscosity alpha; the
state (r, v, id, kind) is stored every `k` steps.  Backward: for each
segment, last first, the segment is recomputed from its checkpoint (storing
each step's input state), then the hand-written adjoint kernels run one step
at a time in reverse, carrying (dL/dr, dL/dv) and accumulating dL/dalpha on
the device.  Memory: nsteps/k checkpoints plus k states, each n x (3 doubles +
3 velocity words + 5 bytes).

The loss is whatever the caller builds from the returned final positions
(in the final state's order, given by the returned ids).
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np
import torch

from . import sph as S


class _Engine:
    """A context (one alpha) and the device state buffers of one rollout."""

    def __init__(self, case, precision, alpha, **params):
        self.case = case
        self.precision = precision
        self.alpha = float(alpha)
        self.params = S.params_from_case(case, precision=precision, alpha=self.alpha, **params)
        self.ctx = S.sph_create(self.params, case.n)
        self.tdt = torch.float32 if precision == S.SPH_PREC_F32 else torch.float64

    def close(self):
        if self.ctx:
            S.sph_destroy(self.ctx)
            self.ctx = None

    def state_from(self, r, v, ids, kind):
        n, dim = self.case.n, self.case.dim
        st = S.DeviceState(r=[r[k].clone() for k in range(dim)], v=[v[k].clone() for k in range(dim)],
                           rho=torch.zeros(n, dtype=self.tdt, device="cuda"),
                           p=torch.zeros(n, dtype=self.tdt, device="cuda"),
                           id=ids.clone(), kind=kind.clone(), n=n, dim=dim)
        return st

    @staticmethod
    def snapshot(st):
        return ([t.clone() for t in st.r], [t.clone() for t in st.v], st.id.clone(), st.kind.clone())


def rollout_forward(engine: _Engine, r0, v0, ids0, kind0, nsteps: int, k: int):
    """Run nsteps, return (final state, checkpoints {step: snapshot})."""
    st = engine.state_from(r0, v0, ids0, kind0)
    view = st.view()
    ckpt = {}
    for s in range(nsteps):
        if s % k == 0:
            ckpt[s] = engine.snapshot(st)
        S.sph_step(engine.ctx, view, 1)
    return st, ckpt


def rollout_backward(engine: _Engine, ckpt, nsteps: int, k: int, gr_final, gv_final):
    """Reverse sweep.  gr_final/gv_final: lists of dim device tensors in the
    final state's order.  Returns (gr0, gv0, alpha_bar) in the initial order."""
    dim = engine.case.dim
    n = engine.case.n
    gr = [g.to(torch.float64).clone() for g in gr_final]
    gv = [g.to(engine.tdt).clone() for g in gv_final]
    gr_alt = [torch.empty_like(g) for g in gr]
    gv_alt = [torch.empty_like(g) for g in gv]
    abar = torch.zeros(1, dtype=torch.float64, device="cuda")
    nseg = math.ceil(nsteps / k)
    for seg in reversed(range(nseg)):
        s0 = seg * k
        s1 = min(s0 + k, nsteps)
        r, v, ids, kind = ckpt[s0]
        st = engine.state_from(r, v, ids, kind)
        view = st.view()
        states = []
        for s in range(s0, s1):
            states.append(engine.state_from(st.r, st.v, st.id, st.kind))
            S.sph_step(engine.ctx, view, 1)
        for s in reversed(range(s0, s1)):
            sn = states[s - s0]
            g1 = S.grad_view(gr, gv)
            g0 = S.grad_view(gr_alt, gv_alt)
            S.sph_step_adjoint(engine.ctx, sn.view(), g1, g0, abar.data_ptr())
            gr, gr_alt = gr_alt, gr
            gv, gv_alt = gv_alt, gv
    return gr, gv, abar


class SPHRollout(torch.autograd.Function):
    """r_final = rollout(v0, alpha).  Inputs: v0 (n, dim) device tensor in the
    case's particle order, alpha a 0-d tensor.  Outputs: final positions
    (n, dim) float64 and the final ids (int32, not differentiable)."""

    @staticmethod
    def forward(ctx, v0, alpha, case, precision, nsteps, k, params=None):
        dim = case.dim
        eng = _Engine(case, precision, float(alpha.item()), **(params or {}))
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
        return gv0t, abar.reshape(()).to(torch.float64), None, None, None, None, None


def rollout(v0, alpha, case, precision=S.SPH_PREC_F32, nsteps: int = 200, k: int = 20, **params):
    """Differentiable rollout (see SPHRollout); params go to params_from_case
    (e.g. clamp_neg_p=False)."""
    return SPHRollout.apply(v0, alpha, case, precision, nsteps, k, params or None)


def target_loss(rf, ids, case, target):
    """mean over fluid of |r_final - target|^2 with target indexed by id."""
    tgt = torch.as_tensor(target, dtype=torch.float64, device=rf.device)
    ids_l = ids.long()
    fl = ids_l < case.n_fluid  # fluid particles carry ids 0..n_fluid-1
    d = rf[fl] - tgt[ids_l[fl]]
    return (d * d).sum(dim=1).mean()

"""PyTorch autograd wrappers of the discrete adjoint (argument marshalling
only: the forward solve, the reverse sweep and the loss run in the CUDA
library).

``HJTube(spec, nsteps)`` holds a grid and a workspace; ``tube(phi0, target,
params)`` returns phi after ``nsteps`` fixed CFL steps and is differentiable
with respect to phi0, the target and the dynamics parameters (the reverse
sweep of ``lsp_hj_adjoint`` with sqrt(N) checkpoints).  The checkpoints live
in the tube's workspace, so only the latest forward of a tube can be
differentiated: a backward through an earlier one raises.  ``tube.loss(phi,
queries)`` is the smoothed tube volume plus the values at query states,
differentiable with respect to phi.
"""
from __future__ import annotations

import torch

from . import binding as B


class _SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, target, params, tube):
        tube._set_params(params)
        phi = phi0.detach().clone().contiguous()
        tgt = target.detach().contiguous() if target is not None else None
        B.lsp_hj_solve_ckpt(tube.grid, tube.opts, phi, tgt, tube.nsteps, tube.ncheck,
                            tube.workspace)
        # the checkpoints of this forward live in the tube's workspace until
        # the next forward on the same tube overwrites them
        tube._generation += 1
        ctx.generation = tube._generation
        ctx.tube = tube
        ctx.params = params.detach().clone()
        ctx.save_for_backward(tgt if tgt is not None else torch.empty(0))
        ctx.has_target = tgt is not None
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        tube = ctx.tube
        if tube._generation != ctx.generation:
            raise RuntimeError(
                "HJTube: the workspace holding this forward's checkpoints was reused by a later "
                "forward on the same tube; call backward before the next forward, or use one "
                "HJTube per live graph")
        (tgt,) = ctx.saved_tensors
        tgt = tgt if ctx.has_target else None
        tube._set_params(ctx.params)  # the sweep needs the forward's dynamics
        lamT = grad_phi.contiguous()
        lam0 = torch.empty_like(lamT)
        lamg = torch.empty_like(lamT) if tgt is not None else None
        dprm = B.lsp_hj_adjoint(tube.grid, tube.opts, tgt, tube.nsteps, tube.ncheck, lamT, lam0,
                                lamg, tube.workspace)
        gp = torch.tensor(dprm[: ctx.params.numel()], dtype=ctx.params.dtype,
                          device=ctx.params.device)
        return lam0, lamg, gp, None


class _LossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, queries, tube):
        value = torch.zeros(1, dtype=torch.float64, device=phi.device)
        grad = torch.empty_like(phi)
        B.lsp_loss_tube(tube.grid, tube.spec.get("dtype", "f32"), phi.contiguous(),
                        queries.contiguous() if queries is not None else None, value, grad)
        ctx.save_for_backward(grad)
        return value[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g.to(grad.dtype), None, None


class HJTube:
    """A fixed-step reachable-tube solve with a discrete-adjoint backward.

    ncheck: checkpoints of the forward (0: ceil(sqrt(nsteps)), recomputed
    segment by segment in the backward); negative: every state and stage
    input is kept (nsteps * rk fields of workspace) and the backward
    recomputes nothing."""

    def __init__(self, spec: dict, nsteps: int, ncheck: int = 0, device="cuda"):
        self.spec = spec
        self.nsteps = int(nsteps)
        self.ncheck = int(ncheck)
        d = spec["ndim"]
        self.grid = B.lsp_grid_create(d, spec["lo"], spec["hi"], spec["n"],
                                      ["periodic" if p else "extrapolate" for p in spec["periodic"]])
        self._params = None
        self._generation = 0  # forwards run so far (checkpoints belong to the last one)
        self._set_params(torch.tensor(spec["params"], dtype=torch.float64))
        self.opts = B.make_opts(spec.get("rk", 3), spec["scheme"], spec.get("dtype", "f32"),
                                spec.get("tube", False), spec.get("cfl", 0.75))
        nbytes = B.lsp_adjoint_workspace_size(self.grid, self.opts, self.nsteps, self.ncheck)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)

    def _set_params(self, params):
        p = [float(v) for v in params.detach().cpu().reshape(-1)]
        if p != self._params:
            B.lsp_set_dynamics(self.grid, self.spec["dyn"], p)
            self._params = p

    def autotune(self, phi):
        """Pick the stage kernel's tile for this grid (lsp_autotune, timed on
        whole RK steps of a scratch copy of phi; phi is not modified).  The
        forward, the recomputed segments and the stage inputs of the reverse
        sweep all run with it.  Returns (tb, ta, ch, minb, pair)."""
        nbytes = B.lsp_workspace_size(self.grid, self.opts)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=phi.device)
        return B.lsp_autotune(self.grid, self.opts, phi, ws)

    def __call__(self, phi0, target, params):
        return _SolveFn.apply(phi0, target, params, self)

    def loss(self, phi, queries):
        return _LossFn.apply(phi, queries, self)

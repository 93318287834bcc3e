"""torch.autograd.Function over the unrolled solve (forward and reverse pass
both run in the library's CUDA kernels; this module only passes pointers)."""
from __future__ import annotations

import torch

from . import lift as G


class UnrolledSolve(torch.autograd.Function):
    """u~ = unlift(PDHG^iters(0; f, lambda, alpha, nu)) with hand-written adjoint.

    ``solver`` is a :class:`paper_1512_01383_gb300.lift.Solver` of the same size
    (quadratic or truncated-quadratic kind); its data and parameters are
    overwritten.  Checkpoints every ``every`` iterations bound the memory of
    the reverse pass.  The solver holds one forward pass at a time: backward
    raises if another forward (or a new f, parameters or a reset) ran on the
    same solver in between; use one solver per pending backward.
    """

    @staticmethod
    def forward(ctx, f, lam, alpha, nu, solver, iters: int, every: int):
        f = f.detach().contiguous().float()
        G.lift_set_data(solver.h, f)
        G.lift_set_params(solver.h, float(lam), float(alpha), float(nu))
        G.lift_unrolled_forward(solver.h, iters, every)
        u = torch.empty((solver.H, solver.W), device=f.device, dtype=torch.float32)
        G.lift_unlift(solver.h, u)
        ctx.solver = solver
        ctx.shapes = (f.shape, lam, alpha, nu)
        ctx.generation = G.lift_unrolled_generation(solver.h)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        solver = ctx.solver
        fshape, lam, alpha, nu = ctx.shapes
        # the handle keeps one forward pass: a later unrolled_solve (or a new
        # f, lambda, alpha, nu, or a reset) on the same solver replaced it
        if G.lift_unrolled_generation(solver.h) != ctx.generation:
            raise G.LiftError(G.LIFT_ERR_ARG, "UnrolledSolve.backward: the solver's stored forward "
                                              "pass is no longer this one's (another forward, new "
                                              "data or parameters, or a reset ran on it since)")
        gu = grad_u.detach().contiguous().float()
        gf = torch.empty(fshape, device=gu.device, dtype=torch.float32)
        gl, ga, gn = G.lift_unrolled_backward(solver.h, gu, gf)

        def scal(ref, v):
            if isinstance(ref, torch.Tensor):
                return torch.tensor(v, dtype=ref.dtype, device=ref.device)
            return None
        return gf, scal(lam, gl), scal(alpha, ga), scal(nu, gn), None, None, None


def unrolled_solve(f, lam, alpha, nu, solver, iters: int, every: int = 50):
    return UnrolledSolve.apply(f, lam, alpha, nu, solver, iters, every)

"""torch.autograd.Function around the MGRIT forward solve and the library's discrete adjoint.

u_T = AdvectionSolve.apply(u0, a, spec) solves u_{n+1} = Phi_n(a) u_n by MGRIT (mgrit_solve) and returns
the final slice, in the shape of u0 (1D: [nx]; 2D, spec["dim"] = 2: [nx, nx] or [nx*nx], y slow).  Its backward pass runs mgrit_adjoint_solve: with lambda_nt = dL/du_T (passed to the
library as u_target = u_T - dL/du_T, since its objective's lambda_nt is u_T - u_target), the adjoint
MGRIT returns dL/du0 = lambda_0 and dL/da.  Only the C-point rows of the forward solution are kept as
checkpoints; the library recomputes the F-points in the backward pass.
"""

from __future__ import annotations

import torch

from . import mgrit_setup


class AdvectionSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, a, spec: dict):
        dim = spec.get("dim", 1)
        h = mgrit_setup(spec["nx"], spec["nt"], spec["order"], spec["m"],
                        wave=spec.get("wave", "sin_kx_cos_t" if dim == 1 else "sin_cos2"), a=float(a),
                        k=spec.get("k", 1.0), a2=spec.get("a2", 1.0), dim=dim, levels=spec.get("levels", 0),
                        max_coarsest=spec.get("max_coarsest", 1), cfl=spec.get("cfl", 0.85), precision=0,
                        gmres_maxit=spec.get("gmres_maxit", 10), gmres_rtol=spec.get("gmres_rtol", 1e-2))
        U, st = h.solve(u0.detach().reshape(-1).contiguous())
        m1 = h.level_info(1)[1]
        ctx.h = h
        ctx.shape = u0.shape
        ctx.checkpoints = U[::m1].contiguous()
        ctx.u_T = U[-1].clone()
        ctx.a_dtype = a.dtype if isinstance(a, torch.Tensor) else torch.float64
        ctx.stats = st
        return U[-1].clone().reshape(u0.shape)

    @staticmethod
    def backward(ctx, grad_uT):
        u_target = (ctx.u_T - grad_uT.reshape(-1)).contiguous()
        dJdu0, dJda, _ = ctx.h.adjoint(u_target, ctx.checkpoints)
        ctx.h.destroy()
        return dJdu0.reshape(ctx.shape), dJda.reshape(()).to(dtype=ctx.a_dtype, device=grad_uT.device), None


def advection_solve(u0, a, **spec):
    """Differentiable MGRIT solve: returns u(T); gradients flow to u0 and the wave-speed amplitude a."""
    return AdvectionSolve.apply(u0, a, spec)

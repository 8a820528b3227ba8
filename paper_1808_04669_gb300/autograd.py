"""torch.autograd binding of the SSP-RK3 rollout and its hand-written adjoint (dg_rk3_vjp).

    u_K = rk3_rollout(mesh, u0, nu, dt, nsteps, checkpoint_every)

u0 and u_K are CUDA float64 tensors of coefficients in the library's orthonormal
basis ([n_tri, 2 n_lat(k)]; the Euclidean inner product is the L2 inner product),
nu a float64 scalar tensor. The backward pass calls the library's adjoint: it
re-runs the forward rollout with checkpoints and sweeps back through each stage
with the transposed residual Jacobian and the symmetric hybrid-mixed solve.
"""
import torch


class _RK3Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, nu, mesh, dt, nsteps, checkpoint_every):
        if not (u0.is_cuda and u0.dtype == torch.float64):
            raise ValueError("u0 must be a CUDA float64 tensor")
        u0c = u0.detach().contiguous()
        nu_f = float(nu.detach().item()) if isinstance(nu, torch.Tensor) else float(nu)
        mesh.set_viscosity(nu_f)
        mesh.set_coefficients(u0c)
        mesh.rk3_step(dt, nsteps)
        out = torch.empty_like(u0c)
        mesh.get_coefficients(out)
        ctx.save_for_backward(u0c)
        ctx.mesh, ctx.dt, ctx.nsteps, ctx.ck, ctx.nu = mesh, dt, nsteps, checkpoint_every, nu_f
        ctx.nu_is_tensor = isinstance(nu, torch.Tensor)
        return out

    @staticmethod
    def backward(ctx, gout):
        (u0c,) = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_viscosity(ctx.nu)
        mesh.set_coefficients(u0c)
        g = gout.detach().contiguous().to(torch.float64)
        u0bar, nubar = mesh.rk3_vjp(ctx.dt, ctx.nsteps, g, checkpoint_every=ctx.ck)
        nu_grad = torch.tensor(nubar, dtype=torch.float64, device=g.device) if ctx.nu_is_tensor else None
        return u0bar, nu_grad, None, None, None, None


def rk3_rollout(mesh, u0, nu, dt, nsteps, checkpoint_every=0):
    """Differentiable nsteps-step SSP-RK3 rollout on mesh (gradients w.r.t. u0 and nu)."""
    return _RK3Rollout.apply(u0, nu, mesh, float(dt), int(nsteps), int(checkpoint_every))

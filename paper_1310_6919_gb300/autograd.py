"""torch.autograd interface: a solve as a differentiable layer.

forward: the MC-PDIPM solve of the problem (b, entry values) on the GPU; outputs the final
iterate (X̄ on E in the supernodal layout, z).  backward: mcsdp_backward, i.e. the implicit
derivatives of the central-path point for the final iterate's mu (the iterate is re-centred
first, so the derivatives are those of a point the outputs lie within the method's
neighbourhood of), with respect to b and to every input entry value.  No computation here:
argument marshalling around binding.Problem."""
import torch

from .binding import Problem


class CentralPathSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, val, n, m, mat, row, col, z0, options):
        P = Problem(n, m, b.detach().cpu().numpy(), mat, row, col, val.detach().cpu().numpy(),
                    **options)
        if z0 is not None:
            P.set_iterate(None, z0)
        P.solve()
        X, z, _ = P.get_iterate()
        ctx.problem = P
        ctx.devices = (b.device, val.device)
        return X, z

    @staticmethod
    def backward(ctx, gX, gz):
        out = ctx.problem.backward(gX, gz)
        return (out["gb"].to(ctx.devices[0]), out["g_entries"].to(ctx.devices[1]), None, None,
                None, None, None, None, None)


def solve_layer(b, val, n, m, mat, row, col, z0=None, **options):
    """(X̄ layout, z) = solve(b, val); differentiable with respect to b and val."""
    return CentralPathSolve.apply(b, val, n, m, mat, row, col, z0, options)

"""Differentiable DMRG energy: torch.autograd.Function around dmrg_solve / dmrg_rdm.

Forward sets the integrals (Sec. 4.1: h, V with eightfold symmetry, physics notation),
runs the convergence scheme (Sec. 4.3) from the context's current MPS and returns the
energy of the last micro-iteration.  Backward returns dE/dh = gamma and
dE/dV = Gamma / 2, the spin-summed RDMs of the final MPS (Gamma^A of Sec. 4.3) computed
by the library's adjoint of the H_eff matvec (dmrg_rdm).  For a converged state these are the exact
derivatives of the eigenvalue (Hellmann-Feynman); V's gradient is the part that is
invariant under V's eight index permutations, so a symmetric change dV of V changes
the energy by sum(grad_V * dV).  torch is used for tensors and streams only.
"""
import torch

from .binding import Context


class DMRGEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, h, V, ctx: Context, econst: float = 0.0):
        ctx.set_integrals(h.detach().cpu().double().numpy(), V.detach().cpu().double().numpy(), econst)
        _, e_last = ctx.solve()
        L = ctx.L
        gamma = torch.empty((L, L), dtype=torch.float64, device="cuda")
        Gamma = torch.empty((L,) * 4, dtype=torch.float64, device="cuda")
        ctx.rdm(gamma, Gamma)
        torch.cuda.current_stream().synchronize()
        fctx.save_for_backward(gamma, Gamma)
        fctx.devices = (h.device, V.device)
        return torch.tensor(e_last, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(fctx, grad_e):
        gamma, Gamma = fctx.saved_tensors
        dh, dV = fctx.devices
        g = grad_e.to(gamma.device)
        return (g * gamma).to(dh), (0.5 * g * Gamma).to(dV), None, None


def dmrg_energy(h, V, ctx: Context, econst: float = 0.0):
    """E(h, V) of the DMRG solve on `ctx`, differentiable in h and V."""
    return DMRGEnergy.apply(h, V, ctx, econst)

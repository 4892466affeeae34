"""torch.autograd functions over the solver: the Mermin free energy of a density-matrix
solve and the eigenpairs of H C = S C diag(eps). The forward passes and the backward
formulas run in the library's kernels (elsi_dm_real / elsi_ev_real and
elsi_dm_adjoint_real / elsi_ev_adjoint_real); this module only wires them into autograd.

KSFreeEnergy.apply(H, S, handle) -> F = E_band - kT S_ent (0-dim tensor);
    backward: dF/dH = P, dF/dS = -W.
KSEigen.apply(H, S, handle, k) -> (eps (n,), C (n, k));
    backward: the first-order perturbation adjoint with the degeneracy guard; the handle
    must compute all n eigenvectors (n_state = n).
H and S are symmetric float64 CUDA tensors; the gradients returned are symmetric.
"""
from __future__ import annotations

import torch

__all__ = ["KSFreeEnergy", "KSEigen", "free_energy", "eigh"]


class KSFreeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, S, handle):
        P, e = handle.dm_real(H.detach().contiguous(), S.detach().contiguous())
        W = handle.get_edm()
        F = e + handle.get_entropy()
        ctx.handle = handle
        ctx.save_for_backward(P, W)
        return torch.tensor(F, dtype=torch.float64, device=H.device)

    @staticmethod
    def backward(ctx, gF):
        P, W = ctx.saved_tensors
        hb, sb = ctx.handle.dm_adjoint(float(gF), P, W)
        return hb, sb, None


class KSEigen(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, S, handle, k):
        if handle.n_state != handle.n:
            raise ValueError("KSEigen needs a handle with n_state = n_basis (all eigenvectors)")
        ev, C = handle.ev_real(H.detach().contiguous(), S.detach().contiguous())
        ctx.handle = handle
        ctx.k = int(k)
        ctx.save_for_backward(ev, C)
        return ev, C[:, :k]

    @staticmethod
    def backward(ctx, gev, gC):
        ev, C = ctx.saved_tensors
        hb, sb = ctx.handle.ev_adjoint(ev, C, gev, gC.contiguous() if gC is not None else None)
        return hb, sb, None, None


def free_energy(H, S, handle):
    return KSFreeEnergy.apply(H, S, handle)


def eigh(H, S, handle, k: int):
    return KSEigen.apply(H, S, handle, k)

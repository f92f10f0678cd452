"""PyTorch adjoints of the CC residual and of the polarizability (marshalling around the C ABI).

* ``CCSDResidual``: Omega(t), the CCSD residual as a function of the amplitudes (ground-state
  equations of Sec. 3, step 1).  Omega is holomorphic in t, so PyTorch's complex convention
  (grad_in = J^H grad_out) gives the backward pass conj(A^T conj(g)) = conj(l A) with l = conj(g):
  one left sigma product (SI Eqs. sigma_sin-ee-left, sigma_double-ee-left) at the same t.
* ``alpha_directional_derivative``: the response function is bilinear in the two operators for a
  fixed Hamiltonian (Eq. CC-CC response function), so the derivative of alpha = -<<X;X>> along an
  operator direction dX is -(<<dX;X>> + <<X;dX>>), read off one linear-response solve with the
  operator pair (X, dX).

Every product runs in libcclr's CUDA kernels; this module only moves arrays and picks entries.
"""
import numpy as np
import torch

from . import AMP_T


def _host(t):
    return np.ascontiguousarray(t.detach().to("cpu").numpy(), dtype=np.complex128)


class CCSDResidual(torch.autograd.Function):
    """Omega(t) for a complex128 amplitude vector t (layout [t_i^a | t_ij^ab packed], length N)
    on the Hamiltonian of ``cc``.  Sets the context's amplitudes to t (H-bar is rebuilt there)."""

    @staticmethod
    def forward(ctx, t, cc):
        cc.cclr_set_amplitudes(AMP_T, _host(t))
        omega = torch.from_numpy(cc.cclr_residual()[0]).to(t.device)
        ctx.cc = cc
        ctx.save_for_backward(t)
        return omega

    @staticmethod
    def backward(ctx, g):
        (t,) = ctx.saved_tensors
        cc = ctx.cc
        cc.cclr_set_amplitudes(AMP_T, _host(t))   # the left sigma is the Jacobian at this t
        lg = cc.cclr_sigma(np.conj(_host(g))[None, :], side=1)[0]
        return torch.from_numpy(np.conj(lg)).to(g.device), None


def ccsd_residual(t, cc):
    """Differentiable Omega(t) (see CCSDResidual)."""
    return CCSDResidual.apply(t, cc)


def alpha_directional_derivative(cc, X, dX, omegas, gamma):
    """d alpha(w + i gamma) / d s of alpha = -<<X + s dX; X + s dX>> at s = 0, for every
    frequency: an array [n_freq].  Needs cc_ground and cc_lambda on ``cc``."""
    ops = np.stack([np.asarray(X, np.complex128), np.asarray(dX, np.complex128)])
    cc.cc_lr_solve(ops, omegas, gamma)
    r = cc.cc_response_function()
    return -(r[:, 0, 1] + r[:, 1, 0])

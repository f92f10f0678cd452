"""PyTorch adjoints of the CC residual, the CC energy and the polarizability (marshalling around the
C ABI; every product and solve runs in libcclr's CUDA kernels).

PyTorch's complex convention: backward receives g = dL/ds* for an output s and returns
dL/dz* = conj(g) ds/dz* + g conj(ds/dz) for an input z.

* ``CCSDResidual``: Omega(t), the CCSD residual as a function of the amplitudes (ground-state
  equations, Sec. 3 step 1).  Omega is holomorphic in t, so the backward pass is
  conj(conj(g)^T A) = conj(l A) with l = conj(g): one left sigma product (SI Eqs.
  sigma_sin-ee-left, sigma_double-ee-left) at the same t.
* ``CCEnergy``: E(t), holomorphic; its derivative is eta of the energy, the right-hand side of the
  Lambda equations t-bar A = -eta (Sec. 2.3), so ``lambda_by_adjoint`` obtains the ground-state
  multipliers as the adjoint solve of the energy: l A = -dE/dt with dE/dt read off autograd.
* ``Polarizability``: alpha(w + i g) = -<<X;Y>> over all operator pairs and frequencies (Eq.
  CC-CC response function), differentiable in the operator matrices.  The response function is
  linear in each operator through xi^X and eta^X; its backward pass runs the adjoint left solves
  l (A + w) = -(eta^Y + F t^Y(w)) on the device (cclr_response_gradient) and contracts the
  results with the operator densities.  Operators parameterised by real numbers (Re/Im X_pq,
  p < q, real X_pp for a Hermitian X) get d Re alpha / d theta and d Im alpha / d theta through
  PyTorch's chain rule.

Arrays stay where they are: CUDA tensors go to the library as device pointers, CPU tensors as
host arrays.
"""
import numpy as np
import torch

from . import AMP_T


def _lib_arg(t):
    """A tensor in the form the binding takes: CUDA tensors as they are (contiguous complex128),
    CPU tensors as numpy arrays.  Lazy conjugation and negation are materialised first: the
    library reads the memory, not the view."""
    t = t.detach().to(torch.complex128).resolve_conj().resolve_neg().contiguous()
    return t if t.is_cuda else t.numpy()


def _as_tensor(a, like):
    return a if torch.is_tensor(a) else torch.from_numpy(np.asarray(a)).to(like.device)


class CCSDResidual(torch.autograd.Function):
    """Omega(t) for a complex128 amplitude vector t (layout [t_i^a | t_ij^ab packed], length N)
    on the Hamiltonian of ``cc``.  Sets the context's amplitudes to t (H-bar is rebuilt there)."""

    @staticmethod
    def forward(ctx, t, cc):
        cc.cclr_set_amplitudes(AMP_T, _lib_arg(t))
        omega = _as_tensor(cc.cclr_residual(like=t if t.is_cuda else None)[0], t)
        ctx.cc = cc
        ctx.save_for_backward(t)
        return omega

    @staticmethod
    def backward(ctx, g):
        (t,) = ctx.saved_tensors
        cc = ctx.cc
        cc.cclr_set_amplitudes(AMP_T, _lib_arg(t))   # the left sigma is the Jacobian at this t
        lg = cc.cclr_sigma(_lib_arg(g.conj()).reshape(1, -1), side=1)
        return _as_tensor(lg, g).reshape(g.shape).conj().resolve_conj(), None


def ccsd_residual(t, cc):
    """Differentiable Omega(t) (see CCSDResidual)."""
    return CCSDResidual.apply(t, cc)


class CCEnergy(torch.autograd.Function):
    """The CCSD correlation energy E(t) (a 0-d complex tensor) at amplitudes t."""

    @staticmethod
    def forward(ctx, t, cc):
        cc.cclr_set_amplitudes(AMP_T, _lib_arg(t))
        e = cc.cclr_residual(like=t if t.is_cuda else None)[1]
        ctx.cc = cc
        ctx.save_for_backward(t)
        return torch.tensor(e, dtype=torch.complex128, device=t.device)

    @staticmethod
    def backward(ctx, g):
        (t,) = ctx.saved_tensors
        cc = ctx.cc
        cc.cclr_set_amplitudes(AMP_T, _lib_arg(t))
        eta = _as_tensor(cc.cclr_eta_ground(like=t if t.is_cuda else None), t)
        return g * eta.conj(), None   # holomorphic: dL/dt* = g conj(dE/dt)


def cc_energy(t, cc):
    """Differentiable E(t) (see CCEnergy)."""
    return CCEnergy.apply(t, cc)


def lambda_by_adjoint(cc, device=None):
    """The ground-state multipliers as the adjoint of the energy: l A = -dE/dt at the context's T,
    with dE/dt from the autograd of ``cc_energy`` and the left solve on the device."""
    t = cc.cclr_get_amplitudes(AMP_T)
    t = torch.from_numpy(t).to(device) if device is not None else torch.from_numpy(t)
    t.requires_grad_(True)
    e = cc_energy(t, cc)
    (gt,) = torch.autograd.grad(e, t, grad_outputs=torch.ones_like(e))
    eta = gt.conj().contiguous()          # grad_output 1 on a holomorphic E gives conj(dE/dt)
    return _as_tensor(cc.cclr_left_solve(_lib_arg(eta)), eta)


class Polarizability(torch.autograd.Function):
    """alpha[f, x, y] = -<<X_x; X_y>>_{w_f + i gamma} for operators ops (n_ops, n, n), after
    cc_ground and cc_lambda on ``cc``.  Backward: per frequency with a non-zero output gradient,
    one cclr_response_gradient call (4 n_ops left solves) and the contraction below.  The operator
    gradients do not depend on the output gradient, so repeated backward passes through the same
    graph (retain_graph=True, e.g. for the rows of the Jacobian) reuse them."""

    @staticmethod
    def forward(ctx, ops, cc, omegas, gamma):
        cc.cc_lr_solve(_lib_arg(ops), omegas, gamma)
        r = cc.cc_response_function()
        ctx.cc, ctx.serial, ctx.args = cc, cc.lr_serial, (list(omegas), float(gamma))
        ctx.G = {}
        ctx.save_for_backward(ops)
        return -torch.from_numpy(r).to(ops.device)

    @staticmethod
    def backward(ctx, g):
        (ops,) = ctx.saved_tensors
        cc = ctx.cc
        grad = torch.zeros_like(ops, dtype=torch.complex128)
        for f in range(g.shape[0]):
            gf = g[f].to(torch.complex128)
            if not bool(torch.any(gf != 0)):
                continue
            if f not in ctx.G:
                if cc.lr_serial != ctx.serial:   # another solve replaced this one's solutions
                    cc.cc_lr_solve(_lib_arg(ops), *ctx.args)
                    ctx.serial = cc.lr_serial
                ctx.G[f] = _as_tensor(cc.cclr_response_gradient(f, like=ops if ops.is_cuda else None), ops)
            grad += alpha_vjp(gf, ctx.G[f])
        return grad, None, None, None


def alpha_vjp(gf, G):
    """dL/dX* for alpha[x, y] = -<<X_x;X_y>> at one frequency, from the output gradient gf (n_ops,
    n_ops) and the operator gradients G (n_ops, 4, n, n) of cclr_response_gradient, where
    d<<X_x;X_y>> = sum G[y,0] o dX_x + conj(sum G[y,1] o dX_x) + sum G[x,3] o dX_y
    + conj(sum G[x,2] o dX_y).  With d alpha/dX_x = -G[y,0], d alpha/dX_x* = -conj(G[y,1]) and
    likewise for X_y, dL/dX* = conj(g) d alpha/dX* + g conj(d alpha/dX)."""
    gc = gf.conj()
    left = torch.einsum("xy,ypq->xpq", gc, G[:, 1].conj()) + torch.einsum("xy,ypq->xpq", gf, G[:, 0].conj())
    right = torch.einsum("xy,xpq->ypq", gc, G[:, 2].conj()) + torch.einsum("xy,xpq->ypq", gf, G[:, 3].conj())
    return -(left + right)


def polarizability(ops, cc, omegas, gamma):
    """Differentiable alpha (n_freq, n_ops, n_ops) (see Polarizability)."""
    return Polarizability.apply(ops, cc, omegas, gamma)


def hermitian_from_params(theta, n):
    """A Hermitian n x n complex128 matrix from n^2 real parameters: X_pp = theta[p] (real
    diagonal), then Re X_pq and Im X_pq for p < q in row-major order of the strict upper
    triangle (X_qp = conj(X_pq)).  Differentiable (torch ops only)."""
    iu = torch.triu_indices(n, n, 1, device=theta.device)
    m = iu.shape[1]
    re = torch.zeros(n, n, dtype=torch.float64, device=theta.device)
    im = torch.zeros(n, n, dtype=torch.float64, device=theta.device)
    re = re.index_put((iu[0], iu[1]), theta[n:n + m]) + torch.diag(theta[:n])
    im = im.index_put((iu[0], iu[1]), theta[n + m:n + 2 * m])
    re = re + torch.triu(re, 1).T
    im = im - im.T
    return torch.complex(re, im)


def hermitian_params(X):
    """The inverse of hermitian_from_params for a Hermitian numpy matrix."""
    n = X.shape[0]
    iu = np.triu_indices(n, 1)
    return np.concatenate([X.diagonal().real, X[iu].real, X[iu].imag])


def alpha_directional_derivative(cc, X, dX, omegas, gamma):
    """d alpha(w + i gamma) / d s of alpha = -<<X + s dX; X + s dX>> at s = 0, for every
    frequency: an array [n_freq].  Needs cc_ground and cc_lambda on ``cc``.  The response
    function is bilinear in the operators, so this reads -(<<dX;X>> + <<X;dX>>) off one solve
    with the operator pair (X, dX); the adjoint gradient above gives the same in every
    direction at once."""
    ops = np.stack([np.asarray(X, np.complex128), np.asarray(dX, np.complex128)])
    cc.cc_lr_solve(ops, omegas, gamma)
    r = cc.cc_response_function()
    return -(r[:, 0, 1] + r[:, 1, 0])


def alpha_field_derivative(new_context, n_occ, n_vir, fock, blocks, V, ops, omegas, gamma, h=1e-4):
    """d alpha / d eps of the polarizability under a static field eps coupled through the
    one-electron operator V (Fock matrix f + eps V, integrals unchanged; orbital-unrelaxed like
    the response functions), by a central difference of two complete device solves (ground
    state, Lambda, response) at eps = +h and -h.  ``new_context()`` returns a fresh Context
    with the caller's options.  Returns (derivative [n_freq, n_ops, n_ops], alpha(+h),
    alpha(-h)).  The analytic form of this derivative is the quadratic response function."""
    fock = np.asarray(fock, np.complex128)
    V = np.asarray(V, np.complex128)
    alphas = []
    for s in (1.0, -1.0):
        cc = new_context()
        try:
            cc.cclr_set_hamiltonian(n_occ, n_vir, fock + s * h * V, blocks)
            cc.cc_ground()
            cc.cc_lambda()
            cc.cc_lr_solve(ops, omegas, gamma)
            alphas.append(-cc.cc_response_function())
        finally:
            cc.close()
    return (alphas[0] - alphas[1]) / (2 * h), alphas[0], alphas[1]

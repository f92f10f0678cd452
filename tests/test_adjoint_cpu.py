"""Host-side checks of the polarizability adjoint (no GPU).

The backward pass of ``autograd.Polarizability`` combines the operator gradients G[k][s] of
cclr_response_gradient into dL/dX* by PyTorch's complex convention.  Here a stand-in context
supplies an explicit response function with the structure of Eq. CC-CC response function,
    f(w; X, Y) = vec(X)^T K_w vec(Y),  K_{-w} = K_w^T,  <<X;Y>>_z = f(z) + conj(f(-z*)),
and its exact operator gradients (shift order w+ig, -w+ig, w-ig, -w-ig).  The adjoint's
gradient must equal PyTorch's own differentiation of the same expression, for complex operators
and through the real parameters of Hermitian ones.
"""
import numpy as np
import pytest
import torch

from paper_2307_14296_b300 import autograd as ag


class ExplicitResponse:
    """A context stand-in: per frequency two random complex matrices P = K_z and Q = K_{-z*}
    (then K_{z*} = Q^T and K_{-z} = P^T)."""

    def __init__(self, n, n_freq, seed):
        rng = np.random.default_rng(seed)
        m = n * n
        self.n = n
        self.P = [rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)) for _ in range(n_freq)]
        self.Q = [rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)) for _ in range(n_freq)]
        self.lr_serial = 0
        self.solves = 0

    def cc_lr_solve(self, ops, omegas, gamma):
        self.ops = np.array(ops, np.complex128)
        self.lr_serial += 1
        self.solves += 1

    def cc_response_function(self):
        v = self.ops.reshape(len(self.ops), -1)
        return np.array([v @ P @ v.T + np.conj(v @ Q @ v.T) for P, Q in zip(self.P, self.Q)])

    def cclr_response_gradient(self, f, like=None):
        v = self.ops.reshape(len(self.ops), -1)
        K = [self.P[f], self.Q[f], self.Q[f].T, self.P[f].T]
        n = self.n
        return np.stack([np.stack([(Ks @ vk).reshape(n, n) for Ks in K]) for vk in v])


def torch_alpha(ops, cc):
    v = ops.reshape(ops.shape[0], -1)
    out = []
    for P, Q in zip(cc.P, cc.Q):
        P, Q = torch.from_numpy(P), torch.from_numpy(Q)
        out.append(-(v @ P @ v.T + (v @ Q @ v.T).conj()))
    return torch.stack(out)


def test_adjoint_gradient_of_complex_operators_matches_torch():
    n, nf, nops = 3, 2, 3
    cc = ExplicitResponse(n, nf, 1)
    rng = np.random.default_rng(2)
    X0 = rng.standard_normal((nops, n, n)) + 1j * rng.standard_normal((nops, n, n))
    c = torch.from_numpy(rng.standard_normal((nf, nops, nops)) + 1j * rng.standard_normal((nf, nops, nops)))
    X = torch.tensor(X0, requires_grad=True)
    (torch.sum(c * ag.polarizability(X, cc, [0.1, 0.2], 0.01)).real).backward()
    Xr = torch.tensor(X0, requires_grad=True)
    (torch.sum(c * torch_alpha(Xr, cc)).real).backward()
    assert torch.allclose(X.grad, Xr.grad, rtol=1e-12, atol=1e-12)


def test_adjoint_gradient_of_hermitian_parameters_matches_torch_and_fd():
    """d Re alpha and d Im alpha with respect to the real parameters of Hermitian operators:
    through hermitian_from_params, against torch and a central difference (alpha is quadratic
    in the parameters, so the difference is exact up to rounding)."""
    n, nf, nops = 4, 2, 2
    cc = ExplicitResponse(n, nf, 3)
    rng = np.random.default_rng(4)
    th0 = rng.standard_normal((nops, n * n))
    c = torch.from_numpy(rng.standard_normal((nf, nops, nops)) + 1j * rng.standard_normal((nf, nops, nops)))
    for part in (lambda z: z.real, lambda z: z.imag):
        th = torch.tensor(th0, requires_grad=True)
        ops = torch.stack([ag.hermitian_from_params(th[k], n) for k in range(nops)])
        part(torch.sum(c * ag.polarizability(ops, cc, [0.1, 0.2], 0.01))).backward()
        thr = torch.tensor(th0, requires_grad=True)
        opr = torch.stack([ag.hermitian_from_params(thr[k], n) for k in range(nops)])
        part(torch.sum(c * torch_alpha(opr, cc))).backward()
        assert torch.allclose(th.grad, thr.grad, rtol=1e-12, atol=1e-12)

        def L(t):
            with torch.no_grad():
                o = torch.stack([ag.hermitian_from_params(torch.from_numpy(t[k]), n) for k in range(nops)])
                return float(part(torch.sum(c * torch_alpha(o, cc))))
        h = 1e-3
        for i in [0, n, n + 1, n * n - 1]:
            d = np.zeros_like(th0)
            d[1, i] = 1.0
            fd = (L(th0 + h * d) - L(th0 - h * d)) / (2 * h)
            assert abs(fd - float(th.grad[1, i])) < 1e-9 * max(1.0, abs(fd))


def test_backward_resolves_again_after_another_solve():
    """A solve between forward and backward replaces the stored solutions; backward repeats the
    forward's solve first."""
    n, nf = 3, 1
    cc = ExplicitResponse(n, nf, 5)
    rng = np.random.default_rng(6)
    X0 = rng.standard_normal((2, n, n)) + 0j
    X = torch.tensor(X0, requires_grad=True)
    a = ag.polarizability(X, cc, [0.1], 0.01)
    cc.cc_lr_solve(rng.standard_normal((2, n, n)), [0.1], 0.01)
    a.real.sum().backward()
    Xr = torch.tensor(X0, requires_grad=True)
    torch_alpha(Xr, cc).real.sum().backward()
    assert cc.solves == 3
    assert torch.allclose(X.grad, Xr.grad, rtol=1e-12, atol=1e-12)


def test_hermitian_parameterisation_round_trip():
    rng = np.random.default_rng(7)
    n = 5
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    X = a + a.conj().T
    th = ag.hermitian_params(X)
    assert th.size == n * n
    Y = ag.hermitian_from_params(torch.from_numpy(th), n).numpy()
    assert np.array_equal(Y, X)


@pytest.mark.parametrize("shape", [(2, 3, 3)])
def test_alpha_vjp_is_linear_in_the_output_gradient(shape):
    """alpha_vjp is linear in the output gradient: the sum of the vjps of two gradients equals the
    vjp of their sum."""
    rng = np.random.default_rng(8)
    nops, n = shape[0], shape[1]
    G = torch.from_numpy(rng.standard_normal((nops, 4, n, n)) + 1j * rng.standard_normal((nops, 4, n, n)))
    g1 = torch.from_numpy(rng.standard_normal((nops, nops)) + 1j * rng.standard_normal((nops, nops)))
    g2 = torch.from_numpy(rng.standard_normal((nops, nops)) + 1j * rng.standard_normal((nops, nops)))
    assert torch.allclose(ag.alpha_vjp(g1, G) + ag.alpha_vjp(g2, G), ag.alpha_vjp(g1 + g2, G), atol=1e-13)


def test_repeated_backward_reuses_the_operator_gradients():
    """Rows of the Jacobian through one graph: the operator gradients are computed once per
    frequency, and every row matches torch's."""
    n, nf = 3, 2
    cc = ExplicitResponse(n, nf, 9)
    calls = []
    orig = cc.cclr_response_gradient
    cc.cclr_response_gradient = lambda f, like=None: (calls.append(f), orig(f, like))[1]
    rng = np.random.default_rng(10)
    X0 = rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n))
    X = torch.tensor(X0, requires_grad=True)
    a = ag.polarizability(X, cc, [0.1, 0.2], 0.01)
    Xr = torch.tensor(X0, requires_grad=True)
    ar = torch_alpha(Xr, cc)
    for idx in [(0, 0, 1), (1, 1, 0), (0, 1, 1)]:
        for gv in (1.0, 1j):
            g = torch.zeros_like(a)
            g[idx] = gv
            (gx,) = torch.autograd.grad(a, X, grad_outputs=g, retain_graph=True)
            (gr,) = torch.autograd.grad(ar, Xr, grad_outputs=g, retain_graph=True)
            assert torch.allclose(gx, gr, rtol=1e-12, atol=1e-12)
    assert sorted(calls) == [0, 1]

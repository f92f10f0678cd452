"""xi, eta and the Hessian product pinned against derivative definitions."""
import numpy as np
import pytest
import synth
from oracle import deriv, hbar, props
from oracle_cases import general_case, rand_amp


@pytest.mark.parametrize("o,v", [(2, 4), (3, 5)])
def test_xi_is_property_projection(o, v):
    inst, F, I = general_case(o, v)
    X = synth.random_hermitian(o + v, 7, 77, 0.3)
    t1, t2 = rand_amp(o, v, 1)
    x1, x2 = props.xi(X, o, t1, t2)
    d1, d2 = deriv.xi(I, t1, t2, X)
    assert np.abs(x1 - d1).max() < 1e-13 and np.abs(x2 - d2).max() < 1e-13


@pytest.mark.parametrize("o,v", [(2, 4), (3, 5)])
def test_eta_is_lagrangian_derivative(o, v):
    inst, F, I = general_case(o, v)
    X = synth.random_hermitian(o + v, 7, 77, 0.3)
    t1, t2 = rand_amp(o, v, 1)
    l1, l2 = rand_amp(o, v, 5)
    e1, e2 = props.eta(X, o, t1, t2, l1, l2)
    for rb in [(1, 0), (0, 1)]:
        r1, r2 = rand_amp(o, v, 3)
        r1, r2 = r1 * rb[0], r2 * rb[1]
        rhs = deriv.eta_dot(I, t1, t2, l1, l2, X, r1, r2)
        assert abs(deriv.dot(e1, e2, r1, r2) - rhs) < 1e-12 * max(1, abs(rhs))


def test_eom_eta_adds_lambda_xi():
    inst, F, I = general_case(3, 5)
    X = synth.random_hermitian(8, 7, 77, 0.3)
    t1, t2 = rand_amp(3, 5, 1)
    l1, l2 = rand_amp(3, 5, 5)
    e1, e2 = props.eta(X, 3, t1, t2, l1, l2)
    m1, m2 = props.eta_eom(X, 3, t1, t2, l1, l2)
    x1, _ = deriv.xi(I, t1, t2, X)
    assert np.abs(m1 - e1 - np.einsum("ijab,jb->ia", l2, x1)).max() < 1e-13
    assert np.abs(m2 - e2).max() == 0


@pytest.mark.parametrize("o,v", [(2, 4), (3, 5)])
def test_hessian_product_is_second_derivative(o, v):
    """(u F) . w == d^2/da db [E + lambda.Omega](t + a u + b w)."""
    inst, F, I = general_case(o, v)
    t1, t2 = rand_amp(o, v, 1)
    l1, l2 = rand_amp(o, v, 5)
    H = hbar.Hbar(I, t1, t2)
    u1, u2 = rand_amp(o, v, 3)
    w1, w2 = rand_amp(o, v, 7)
    for ub in [(1, 0), (0, 1)]:
        for wb in [(1, 0), (0, 1)]:
            a1, a2, b1, b2 = u1 * ub[0], u2 * ub[1], w1 * wb[0], w2 * wb[1]
            f1, f2 = props.hessian_product(H, I, l1, l2, a1, a2)
            rhs = deriv.hessian_dot(I, t1, t2, l1, l2, a1, a2, b1, b2)
            assert abs(deriv.dot(f1, f2, b1, b2) - rhs) < 1e-11 * max(1, abs(rhs))
            # F is symmetric
            g1, g2 = props.hessian_product(H, I, l1, l2, b1, b2)
            assert abs(deriv.dot(g1, g2, a1, a2) - deriv.dot(f1, f2, b1, b2)) < 1e-11 * max(1, abs(rhs))

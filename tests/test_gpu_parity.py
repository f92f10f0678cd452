"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: 1e-9 relative for every FP64 result (the oracle and the GPU differ only in summation
order; observed differences are ~1e-14).  Component tests use random, non-converged amplitudes
of O(0.3) and a non-canonical complex Fock matrix so that every term contributes.
"""
import numpy as np
import pytest

import synth
from layout import from_amp, rel, to_amp
from oracle import ccsd, det, hbar, props, response as R, sigma
from oracle.deriv import antisym
from oracle.ints import Ints

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def pk():
    import os
    os.environ.setdefault("CCLR_WORKSPACE_GB", "4")
    import paper_2307_14296_b300 as pk
    return pk


def make_ctx(pk, inst, fock=None, **opt):
    ctx = pk.Context(0, **opt)
    ctx.cclr_set_hamiltonian(inst.n_occ, inst.n_vir, inst.fock if fock is None else fock,
                             [inst.blocks[k] for k in synth.CLASSES])
    return ctx


def rand_amp(o, v, stream, scale=0.3, seed=1):
    return synth.random_vector((o, v), seed, stream, scale), antisym(synth.random_vector((o, o, v, v), seed, stream + 1, scale))


SIZES = [(2, 2), (3, 5), (4, 7), (5, 9)]


@pytest.mark.parametrize("o,v", SIZES)
def test_components_at_random_amplitudes(pk, o, v):
    inst = synth.make_instance(o, v, seed=7, sd=0.1)
    F = inst.fock + synth.random_hermitian(o + v, 7, 55, 0.2)
    I = Ints.from_instance(inst, fock=F)
    ctx = make_ctx(pk, inst, fock=F)
    t1, t2 = rand_amp(o, v, 1)
    l1, l2 = rand_amp(o, v, 5)
    ctx.cclr_set_amplitudes(pk.AMP_T, to_amp(t1, t2))
    # residual and energy
    res, e = ctx.cclr_residual()
    r1, r2 = ccsd.residual(I, t1, t2)
    assert rel(res, to_amp(r1, r2)) < TOL
    assert abs(e - ccsd.energy(I, t1, t2)) < TOL * max(1, abs(e))
    # right / left sigma on a batch of three vectors
    H = hbar.Hbar(I, t1, t2)
    vecs = [rand_amp(o, v, 11 + 2 * k) for k in range(3)]
    batch = np.stack([to_amp(*x) for x in vecs])
    sr = ctx.cclr_sigma(batch, side=0)
    sl = ctx.cclr_sigma(batch, side=1)
    for k, (a1, a2) in enumerate(vecs):
        assert rel(sr[k], to_amp(*sigma.sigma_right(H, I, a1, a2))) < TOL
        assert rel(sl[k], to_amp(*sigma.sigma_left(H, I, a1, a2))) < TOL
    # xi, eta, EOM eta, Hessian
    X = inst.ops[0]
    assert rel(ctx.cclr_xi(X), to_amp(*props.xi(X, o, t1, t2))) < TOL
    ctx.cclr_set_amplitudes(pk.AMP_LAMBDA, to_amp(l1, l2))
    assert rel(ctx.cclr_eta(X), to_amp(*props.eta(X, o, t1, t2, l1, l2))) < TOL
    assert rel(ctx.cclr_eta(X, eom=True), to_amp(*props.eta_eom(X, o, t1, t2, l1, l2))) < TOL
    hf = ctx.cclr_hessian(batch)
    for k, (a1, a2) in enumerate(vecs):
        assert rel(hf[k], to_amp(*props.hessian_product(H, I, l1, l2, a1, a2))) < TOL
    ctx.close()


@pytest.fixture(scope="module")
def c0_case():
    """The 4 occupied / 20 virtual spinor system (omega 0 and 0.077, gamma 0)."""
    inst = synth.make_instance(4, 20)
    s = R.CCSystem(Ints.from_instance(inst))
    return inst, s


def test_ground_state_and_lambda(pk, c0_case):
    inst, s = c0_case
    ctx = make_ctx(pk, inst, ground_tol=1e-11)
    e, it = ctx.cc_ground()
    assert abs(e - s.e_corr) < TOL * abs(s.e_corr)
    assert rel(ctx.cclr_get_amplitudes(pk.AMP_T), to_amp(s.t1, s.t2)) < 1e-8
    ctx.cc_lambda()
    assert rel(ctx.cclr_get_amplitudes(pk.AMP_LAMBDA), to_amp(s.l1, s.l2)) < 1e-8
    ctx.close()


def test_polarizability_static_and_dynamic(pk, c0_case):
    inst, s = c0_case
    omegas = [0.0, 0.077]
    ctx = make_ctx(pk, inst, tol=1e-10, ground_tol=1e-11)
    ctx.cc_ground()
    ctx.cc_lambda()
    ctx.cc_lr_solve(inst.ops, omegas, 0.0)
    got = ctx.cc_response_function()
    ref = s.response(inst.ops, omegas, tol=1e-11)
    assert rel(got, ref) < TOL
    ctx.close()


def test_damped_response_small(pk):
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    s = R.CCSystem(Ints.from_instance(inst))
    omegas, gamma = [0.05, 0.3], 0.01
    ctx = make_ctx(pk, inst, tol=1e-10, ground_tol=1e-11)
    ctx.cc_ground()
    ctx.cc_lambda()
    ctx.cc_lr_solve(inst.ops, omegas, gamma)
    got = ctx.cc_response_function()
    ref = s.response(inst.ops, [w + 1j * gamma for w in omegas], tol=1e-11)
    assert rel(got, ref) < TOL
    # response vectors themselves
    tvec = ctx.cclr_get_response_vector(1, 0, 0)
    xi = s.xi(inst.ops[1])
    tref = s.davidson(xi, omegas[0] + 1j * gamma, tol=1e-12)[0]
    assert rel(from_amp(tvec, 3, 8)[1], __import__("oracle.deriv", fromlist=["unpack"]).unpack(tref, 3, 8)[1]) < 1e-8
    ctx.close()


def test_two_electron_exact_sum_over_states(pk):
    inst = synth.make_instance(2, 10, seed=11, sd=0.05)
    zs = [0.1 + 0.01j, 0.25 + 0.01j]
    sos, _ = det.fci_response(inst.fock, synth.full_eri(inst), 2, inst.ops, zs)
    ctx = make_ctx(pk, inst, tol=1e-11, ground_tol=1e-12)
    ctx.cc_ground()
    ctx.cc_lambda()
    ctx.cc_lr_solve(inst.ops, [0.1, 0.25], 0.01)
    assert rel(ctx.cc_response_function(), sos) < TOL
    assert rel(ctx.cc_response_function_ci(), sos) < TOL   # both forms are exact for two electrons
    assert rel(ctx.cc_response_function_asym(), sos) < TOL
    ctx.close()


def test_cc_ci_response_function(pk):
    """CC-CI form (EOM-eta, no Hessian term) against the oracle at (3,8), damped frequencies."""
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    s = R.CCSystem(Ints.from_instance(inst))
    omegas, gamma = [0.05, 0.3], 0.01
    ctx = make_ctx(pk, inst, tol=1e-10, ground_tol=1e-11)
    ctx.cc_ground()
    ctx.cc_lambda()
    ctx.cc_lr_solve(inst.ops, omegas, gamma)
    got = ctx.cc_response_function_ci()
    ref = s.response(inst.ops, [w + 1j * gamma for w in omegas], tol=1e-11, form="ci")
    assert rel(got, ref) < TOL
    ctx.close()


def test_asymmetric_response_function(pk):
    """Asymmetric CC-CC form (first-order multipliers from left solves on the device) against the
    oracle's asymmetric form and against the symmetric form, (3,8), static and damped."""
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    s = R.CCSystem(Ints.from_instance(inst))
    omegas, gamma = [0.0, 0.05, 0.3], 0.01
    ctx = make_ctx(pk, inst, tol=1e-11, ground_tol=1e-12)
    ctx.cc_ground()
    ctx.cc_lambda()
    ctx.cc_lr_solve(inst.ops, omegas, gamma)
    got = ctx.cc_response_function_asym()
    ref = s.response(inst.ops, [w + 1j * gamma for w in omegas], tol=1e-12, form="asym")
    assert rel(got, ref) < TOL
    assert rel(got, ctx.cc_response_function()) < TOL
    ctx.close()


def test_eom_ee_two_electron_fci(pk):
    """EOM-EE roots of the GPU Davidson == FCI excitation energies (two electrons)."""
    inst = synth.make_instance(2, 10, seed=11, sd=0.05)
    w = det.fci_energies(inst.fock, synth.full_eri(inst), 2)
    ctx = make_ctx(pk, inst, tol=1e-10, ground_tol=1e-12)
    ctx.cc_ground()
    got, _ = ctx.cc_eom_ee(4)
    assert np.abs(got - (w[1:5] - w[0])).max() < 1e-9 * np.abs(w[1:5] - w[0]).max()
    ctx.close()


def test_eom_ee_roots_and_vectors(pk):
    """(3,8): the lowest four roots against the oracle's dense eigenvalues, and A x = w x for the
    returned right vectors (sigma through the C ABI)."""
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    s = R.CCSystem(Ints.from_instance(inst))
    ref = s.eom_energies(4)
    ctx = make_ctx(pk, inst, tol=1e-10, ground_tol=1e-12)
    ctx.cc_ground()
    got, its = ctx.cc_eom_ee(4)
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()
    for q in range(4):
        x = ctx.cclr_get_eom_vector(q)
        ax = ctx.cclr_sigma(x[None, :], side=0)[0]
        assert np.abs(ax - got[q] * x).max() < 1e-8 * np.abs(got[q]) * np.abs(x).max()
    ctx.close()


def test_eom_ee_tensor_cores_match_fp64(pk):
    """(6,40): split-BF16 roots within 2e-5 relative of the FP64 roots."""
    inst = synth.make_instance(6, 40)
    w = {}
    for prec in (pk.FP64, pk.TC_BF16X3):
        ctx = make_ctx(pk, inst, precision=prec, tol=1e-9, ground_tol=1e-10, batch=4)
        ctx.cc_ground()
        w[prec], _ = ctx.cc_eom_ee(3)
        ctx.close()
    assert np.abs(w[pk.TC_BF16X3] - w[pk.FP64]).max() < 2e-5 * np.abs(w[pk.FP64]).max()


def test_mixed_electric_magnetic_operators(pk):
    """Optical-rotation operator pair (real symmetric mu, imaginary antisymmetric m) through the
    same path: the three response forms against the oracle at (3,8), damped frequencies."""
    from test_oracle_response import mixed_operators
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    ops = mixed_operators(inst.n_occ + inst.n_vir, 4)
    s = R.CCSystem(Ints.from_instance(inst))
    omegas, gamma = [0.05, 0.3], 0.01
    zs = [w + 1j * gamma for w in omegas]
    ctx = make_ctx(pk, inst, tol=1e-10, ground_tol=1e-11)
    ctx.cc_ground()
    ctx.cc_lambda()
    ctx.cc_lr_solve(ops, omegas, gamma)
    assert rel(ctx.cc_response_function(), s.response(ops, zs, tol=1e-11)) < TOL
    assert rel(ctx.cc_response_function_ci(), s.response(ops, zs, tol=1e-11, form="ci")) < TOL
    assert rel(ctx.cc_response_function_asym(), s.response(ops, zs, tol=1e-11, form="asym")) < TOL
    ctx.close()


def test_autograd_residual_backward_is_the_left_sigma(pk):
    """d Re(w^H Omega(t)) along random complex directions d: the autograd gradient (backward =
    conj(left sigma(conj g))) against a 5-point central difference (exact for the quartic Omega)."""
    import torch
    from paper_2307_14296_b300 import autograd as ag
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    ctx = make_ctx(pk, inst)
    n = ctx.N
    rng = np.random.default_rng(5)
    t0 = 0.05 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    t = torch.tensor(t0, requires_grad=True)
    loss = (torch.tensor(w).conj() * ag.ccsd_residual(t, ctx)).sum().real
    loss.backward()
    grad = t.grad.numpy()

    def L(x):
        ctx.cclr_set_amplitudes(pk.AMP_T, x)
        return float((np.conj(w) * ctx.cclr_residual()[0]).sum().real)
    for k in range(3):
        d = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        h = 1e-3
        fd = (L(t0 - 2 * h * d) - 8 * L(t0 - h * d) + 8 * L(t0 + h * d) - L(t0 + 2 * h * d)) / (12 * h)
        assert abs(fd - float(np.real(np.vdot(grad, d)))) < 1e-8 * abs(fd)
    ctx.close()


def test_alpha_directional_derivative_is_exact(pk):
    """alpha is quadratic in the operator, so the central difference along dX is exact: the
    derivative from the bilinear response function matches it to the solver tolerance."""
    from paper_2307_14296_b300 import autograd as ag
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    X = inst.ops[0]
    rng = np.random.default_rng(9)
    a = rng.normal(0, 0.1, X.shape) + 1j * rng.normal(0, 0.1, X.shape)
    dX = (a + a.conj().T) / 2
    omegas, gamma = [0.05, 0.3], 0.01
    ctx = make_ctx(pk, inst, tol=1e-11, ground_tol=1e-12)
    ctx.cc_ground()
    ctx.cc_lambda()
    got = ag.alpha_directional_derivative(ctx, X, dX, omegas, gamma)

    def alpha(op):
        ctx.cc_lr_solve(op[None], omegas, gamma)
        return -ctx.cc_response_function()[:, 0, 0]
    h = 0.1
    fd = (alpha(X + h * dX) - alpha(X - h * dX)) / (2 * h)
    assert np.abs(got - fd).max() < 1e-8 * np.abs(fd).max()
    ctx.close()


def test_tensor_core_response_matches_fp64(pk):
    """(8,40), 16 damped frequencies x 3 operators: the split-BF16 path (tensor-core sigma, FP32
    solver passes over FP32 mirrors of the trial vectors) gives alpha within 2e-5 of the largest
    component of the FP64 result."""
    inst = synth.make_instance(8, 40)
    omegas, gamma = list(np.linspace(0.05, 0.3, 16)), 0.005
    alpha = {}
    for prec in (pk.FP64, pk.TC_BF16X3):
        ctx = make_ctx(pk, inst, precision=prec, tol=1e-7, ground_tol=1e-9, max_subspace=64, batch=8)
        ctx.cc_ground()
        ctx.cc_lambda()
        ctx.cc_lr_solve(inst.ops, omegas, gamma)
        alpha[prec] = -ctx.cc_response_function()
        ctx.close()
    ref = alpha[pk.FP64]
    assert np.abs(alpha[pk.TC_BF16X3] - ref).max() < 2e-5 * np.abs(ref).max()


def test_export_amplitudes_matches_the_getters(pk):
    """cclr_export_amplitudes (the single export call) returns the same bits as
    cclr_get_amplitudes and cclr_get_response_vector for every amplitude set."""
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    ctx = make_ctx(pk, inst, tol=1e-10, ground_tol=1e-11)
    ctx.cc_ground()
    ctx.cc_lambda()
    ctx.cc_lr_solve(inst.ops, [0.05, 0.3], 0.01)
    assert np.array_equal(ctx.cclr_export_amplitudes(0), ctx.cclr_get_amplitudes(pk.AMP_T))
    assert np.array_equal(ctx.cclr_export_amplitudes(1), ctx.cclr_get_amplitudes(pk.AMP_LAMBDA))
    for k, f, s in [(0, 0, 0), (1, 1, 2), (2, 0, 3)]:
        assert np.array_equal(ctx.cclr_export_amplitudes(2, (k * 2 + f) * 4 + s), ctx.cclr_get_response_vector(k, f, s))
    with pytest.raises(pk.CCLRError):
        ctx.cclr_export_amplitudes(2, 3 * 2 * 4)
    ctx.close()

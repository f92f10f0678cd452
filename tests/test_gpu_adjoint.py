"""The adjoint path on the device against the oracle: the polarizability's operator gradient (left
solves l (A + w) = -(eta^Y + F t^Y(w)) and operator densities), the energy's amplitude gradient and
Lambda as the adjoint solve of the energy, and the generic left solve."""
import numpy as np
import pytest
import torch

import synth
from layout import from_amp, rel, to_amp
from oracle import response as R
from oracle.deriv import pack
from oracle.ints import Ints

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import os
    os.environ.setdefault("CCLR_WORKSPACE_GB", "4")
    import paper_2307_14296_b300 as pk
    return pk


def make_ctx(pk, inst, **opt):
    ctx = pk.Context(0, **opt)
    ctx.cclr_set_hamiltonian(inst.n_occ, inst.n_vir, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
    return ctx


@pytest.mark.parametrize("prec", [0, 2])
def test_polarizability_gradient_matches_oracle_central_difference_3x8(pk, prec):
    """d Re and d Im of a random complex combination of all alpha components with respect to the
    real parameters of the three Hermitian operators (Re/Im X_pq, p < q, real X_pp): the adjoint
    gradient (CUDA tensors in and out) against the oracle's central difference (h = 1e-4; alpha
    is quadratic in the parameters, so the difference is exact up to the solve tolerance) along
    three random directions and on individual elements (oo, ov, vv and diagonal)."""
    from paper_2307_14296_b300 import autograd as ag
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    n, nops = inst.n, 3
    omegas, gamma = [0.05, 0.3], 0.01
    zs = [w + 1j * gamma for w in omegas]
    th0 = np.stack([ag.hermitian_params(inst.ops[k]) for k in range(nops)])
    rng = np.random.default_rng(11)
    c = rng.standard_normal((len(omegas), nops, nops)) + 1j * rng.standard_normal((len(omegas), nops, nops))
    dev = torch.device("cuda", 0)
    ctx = make_ctx(pk, inst, precision=prec, tol=1e-10, ground_tol=1e-11, batch=8)
    ctx.cc_ground()
    ctx.cc_lambda()
    grads = []
    for part in (np.real, np.imag):
        th = torch.tensor(th0, device=dev, requires_grad=True)
        ops = torch.stack([ag.hermitian_from_params(th[k], n) for k in range(nops)])
        alpha = ag.polarizability(ops, ctx, omegas, gamma)
        assert alpha.is_cuda
        L = torch.sum(torch.from_numpy(c).to(dev) * alpha)
        (L.real if part is np.real else L.imag).backward()
        assert th.grad.is_cuda
        grads.append(th.grad.cpu().numpy())
    ctx.close()

    S = R.CCSystem(Ints.from_instance(inst))
    A = S.dense_A()

    def oracle_L(th):
        ops = np.stack([ag.hermitian_from_params(torch.from_numpy(th[k]), n).numpy() for k in range(nops)])
        return np.sum(c * -S.response(ops, zs, solver="dense", A=A))

    iu = np.triu_indices(n, 1)
    m = iu[0].size

    def re_at(p, q):
        return n + int(np.flatnonzero((iu[0] == p) & (iu[1] == q))[0])
    dirs = [rng.standard_normal(th0.shape) for _ in range(3)]
    for k, idx in [(0, 1), (1, re_at(0, 1)), (2, re_at(1, 5) + m), (0, re_at(4, 9)), (1, re_at(2, 3) + m)]:
        d = np.zeros_like(th0)
        d[k, idx] = 1.0
        dirs.append(d)
    h = 1e-4
    for d in dirs:
        fd = (oracle_L(th0 + h * d) - oracle_L(th0 - h * d)) / (2 * h)
        for part, g in zip((np.real, np.imag), grads):
            got = float(np.sum(g * d))
            assert abs(got - part(fd)) < 1e-6 * max(abs(part(fd)), 1e-3), (part, got, part(fd))


def test_gradient_agrees_with_bilinearity_at_8x40(pk):
    """Strong-coupling size where the oracle's solves are slow: the adjoint gradient contracted
    with a random Hermitian direction dX of operator 0 equals -(<<dX;X>> + <<X;dX>>) from one
    response solve with the operator pair (X, dX), per frequency (refined split BF16)."""
    from paper_2307_14296_b300 import autograd as ag
    inst = synth.make_instance(8, 40)
    rng = np.random.default_rng(13)
    a = rng.normal(0, 0.1, inst.ops[0].shape) + 1j * rng.normal(0, 0.1, inst.ops[0].shape)
    dX = (a + a.conj().T) / 2
    omegas, gamma = [0.05, 0.3], 0.01
    ctx = make_ctx(pk, inst, precision=pk.TC_BF16X3, tol=1e-10, ground_tol=1e-11, batch=8, max_subspace=64)
    ctx.cc_ground()
    ctx.cc_lambda()
    dev = torch.device("cuda", 0)
    for f in range(len(omegas)):
        X = torch.tensor(inst.ops[:1], device=dev, requires_grad=True)
        alpha = ag.polarizability(X, ctx, omegas, gamma)
        got = []
        # output gradient 1 stands for L = Re(alpha), 1j for L = Re(-1j alpha) = Im(alpha); the
        # returned gradient gives dL = Re sum conj(grad) dX along a direction dX
        for gv in (1.0, 1j):
            g = torch.zeros_like(alpha)
            g[f, 0, 0] = gv
            (gX,) = torch.autograd.grad(alpha, X, grad_outputs=g, retain_graph=True)
            got.append(float(np.real(np.sum(np.conj(gX[0].cpu().numpy()) * dX))))
        ref = ag.alpha_directional_derivative(ctx, inst.ops[0], dX, omegas, gamma)[f]
        assert abs(got[0] - ref.real) < 1e-8 * abs(ref), (got, ref)
        assert abs(got[1] - ref.imag) < 1e-8 * abs(ref), (got, ref)
    ctx.close()


def test_energy_adjoint_is_eta_and_lambda_is_its_left_solve_4x20(pk):
    """dE/dt by autograd (backward = eta of the energy) against a central difference of the
    library's energy (exact: E is quadratic in t), and Lambda as the adjoint solve of the energy,
    l A = -dE/dt, on the device, against the oracle's Lambda and the library's own cc_lambda."""
    from paper_2307_14296_b300 import autograd as ag
    inst = synth.make_instance(4, 20)
    dev = torch.device("cuda", 0)
    ctx = make_ctx(pk, inst, tol=1e-11, ground_tol=1e-11)
    ctx.cc_ground()
    t0 = ctx.cclr_get_amplitudes(pk.AMP_T)
    t = torch.tensor(t0, device=dev, requires_grad=True)
    e = ag.cc_energy(t, ctx)
    (gt,) = torch.autograd.grad(e, t, grad_outputs=torch.ones_like(e))
    eta = gt.conj().cpu().numpy()
    rng = np.random.default_rng(17)
    for _ in range(2):
        d = rng.standard_normal(t0.size) + 1j * rng.standard_normal(t0.size)
        h = 1e-3

        def E(x):
            ctx.cclr_set_amplitudes(pk.AMP_T, x)
            return ctx.cclr_residual()[1]
        fd = (E(t0 + h * d) - E(t0 - h * d)) / (2 * h)
        assert abs(fd - np.sum(eta * d)) < 1e-10 * abs(fd)
    ctx.cclr_set_amplitudes(pk.AMP_T, t0)
    lam = ag.lambda_by_adjoint(ctx, device=dev)
    assert lam.is_cuda
    lam = lam.cpu().numpy()
    S = R.CCSystem(Ints.from_instance(inst))
    assert rel(lam, to_amp(S.l1, S.l2)) < 1e-8    # the library's amplitude layout
    ctx.cc_lambda()
    assert rel(lam, ctx.cclr_get_amplitudes(pk.AMP_LAMBDA)) < 1e-9
    ctx.close()


def test_left_solve_residual_by_oracle_4x20(pk):
    """cclr_left_solve for two random right-hand sides at a complex shift in split BF16 with
    refinement: the oracle's left sigma at the same T gives l (A + w) + b below the tolerance."""
    inst = synth.make_instance(4, 20)
    ctx = make_ctx(pk, inst, precision=pk.TC_BF16X3, tol=1e-9, ground_tol=1e-11, batch=8)
    ctx.cc_ground()
    t = ctx.cclr_get_amplitudes(pk.AMP_T)
    rng = np.random.default_rng(19)
    b = rng.standard_normal((2, ctx.N)) + 1j * rng.standard_normal((2, ctx.N))
    w = -0.2 + 0.01j
    dev = torch.device("cuda", 0)
    lt = ctx.cclr_left_solve(torch.tensor(b, device=dev), w)
    assert lt.is_cuda
    l = lt.cpu().numpy()
    lh = ctx.cclr_left_solve(b, w)
    assert rel(lh, l) < 1e-12
    o, v = inst.n_occ, inst.n_vir
    S = R.CCSystem(Ints.from_instance(inst), t=from_amp(t, o, v), lam=(np.zeros((o, v)), np.zeros((o, o, v, v))))
    for k in range(2):
        lk, bk = pack(*from_amp(l[k], o, v)), pack(*from_amp(b[k], o, v))   # oracle element order
        r = S.sigma_l(lk) + w * lk + bk
        assert np.linalg.norm(r) < 2e-9 * np.linalg.norm(bk), np.linalg.norm(r) / np.linalg.norm(bk)
    ctx.close()


def test_static_field_derivative_3x8(pk):
    """Finite-field d alpha / d eps (Fock f + eps X_z): against the oracle's central difference of
    the same two solves, and, at w = 0 and gamma = 0 where the CC-CC response function is the
    second derivative of the CC energy, the symmetry of the third derivative:
    d alpha_xy / d eps_z = d alpha_xz / d eps_y = d alpha_yz / d eps_x."""
    import dataclasses
    from paper_2307_14296_b300 import autograd as ag
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    blocks = [inst.blocks[k] for k in synth.CLASSES]

    def new_context():
        return pk.Context(0, tol=1e-11, ground_tol=1e-12)
    h = 1e-3
    D = [ag.alpha_field_derivative(new_context, 3, 8, inst.fock, blocks, inst.ops[z], inst.ops, [0.0], 0.0, h=h)[0][0]
         for z in range(3)]
    scale = max(np.abs(d).max() for d in D)
    for x in range(3):
        for y in range(3):
            for z in range(3):
                assert abs(D[z][x, y] - D[y][x, z]) < 1e-6 * scale, (x, y, z)
                assert abs(D[z][x, y] - D[x][y, z]) < 1e-6 * scale, (x, y, z)
    # damped, dynamic: against the oracle's finite field
    om, gamma = [0.2], 0.01
    got = ag.alpha_field_derivative(new_context, 3, 8, inst.fock, blocks, inst.ops[1], inst.ops, om, gamma, h=h)[0]
    ref = []
    for s in (1.0, -1.0):
        i2 = dataclasses.replace(inst, fock=inst.fock + s * h * inst.ops[1])
        ref.append(-R.CCSystem(Ints.from_instance(i2), tol=1e-12).response(inst.ops, [w + 1j * gamma for w in om],
                                                                           tol=1e-12))
    ref = (ref[0] - ref[1]) / (2 * h)
    assert np.abs(got - ref).max() < 1e-7 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def _herm(n, seed, scale):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return scale * (a + a.conj().T) / 2


def test_analytic_field_derivative_matches_oracle_3x8(pk):
    """cclr_field_derivative (the CC-CC response function differentiated through t0, lambda0 and
    the response amplitudes, with first-order multipliers and exact stencils of the device's own
    products) against the oracle's analytic derivative, FP64, static and damped frequencies, and
    against the device's own finite field (central difference of two complete solves)."""
    from paper_2307_14296_b300 import autograd as ag
    inst = synth.make_instance(3, 8, seed=21, sd=0.05)
    V = _herm(inst.n, 7, 0.05)
    om, gamma = [0.0, 0.2], 0.01
    ctx = make_ctx(pk, inst, tol=1e-11, ground_tol=1e-12)
    ctx.cc_ground()
    ctx.cc_lambda()
    ctx.cc_lr_solve(inst.ops, om, gamma)
    before = ctx.cc_response_function()
    got = ctx.cclr_field_derivative(V)
    after = ctx.cc_response_function()
    ref = R.CCSystem(Ints.from_instance(inst), tol=1e-12).field_derivative(inst.ops, V, [w + 1j * gamma for w in om])
    assert rel(got, ref) < 1e-8, rel(got, ref)
    assert np.array_equal(before, after)   # amplitudes and multipliers restored
    blocks = [inst.blocks[k] for k in synth.CLASSES]
    fd = ag.alpha_field_derivative(lambda: pk.Context(0, tol=1e-11, ground_tol=1e-12), 3, 8, inst.fock, blocks, V,
                                   inst.ops, om, gamma, h=1e-3)[0]
    assert rel(-got, fd) < 1e-6, rel(-got, fd)
    ctx.close()


def test_analytic_field_derivative_refined_split_bf16_4x20(pk):
    """The same derivative from split-BF16 solves refined to 1e-10 (products in the FP64-class
    mode) against the oracle at (4,20)."""
    inst = synth.make_instance(4, 20)
    V = _herm(inst.n, 8, 0.05)
    om, gamma = [0.1], 0.01
    ctx = make_ctx(pk, inst, precision=pk.TC_BF16X3, tol=1e-10, ground_tol=1e-11, batch=8)
    ctx.cc_ground()
    ctx.cc_lambda()
    ctx.cc_lr_solve(inst.ops, om, gamma)
    got = ctx.cclr_field_derivative(V)
    ctx.close()
    ref = R.CCSystem(Ints.from_instance(inst), tol=1e-12).field_derivative(inst.ops, V, [w + 1j * gamma for w in om])
    assert rel(got, ref) < 1e-6, rel(got, ref)

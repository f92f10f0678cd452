"""The response chain pinned against exact sum-over-states, finite fields and closed forms."""
import numpy as np
import pytest
import synth
from oracle import ccsd, det, deriv, response as R
from oracle.ints import Ints

ZS = [0.0, 0.077, 0.2 + 0.01j, -0.15 + 0.005j]


@pytest.fixture(scope="module")
def two_electron():
    inst = synth.make_instance(2, 8, seed=11, sd=0.05)
    s = R.CCSystem(Ints.from_instance(inst))
    sos, w = det.fci_response(inst.fock, synth.full_eri(inst), 2, inst.ops, ZS)
    return inst, s, sos


def test_two_electron_sum_over_states_dense(two_electron):
    inst, s, sos = two_electron
    got = s.response(inst.ops, ZS, solver="dense", A=s.dense_A())
    assert np.abs(got - sos).max() < 1e-11 * np.abs(sos).max()


def test_two_electron_sum_over_states_davidson(two_electron):
    inst, s, sos = two_electron
    got = s.response(inst.ops, ZS, solver="davidson", tol=1e-12)
    assert np.abs(got - sos).max() < 1e-10 * np.abs(sos).max()


def test_two_electron_sum_over_states_cc_ci(two_electron):
    """The CC-CI form is exact for two electrons as well (CCSD = FCI)."""
    inst, s, sos = two_electron
    got = s.response(inst.ops, ZS, solver="dense", A=s.dense_A(), form="ci")
    assert np.abs(got - sos).max() < 1e-11 * np.abs(sos).max()


def test_cc_ci_differs_from_cc_cc_beyond_two_electrons():
    """With four electrons the two forms differ (the CC-CI form drops the Hessian term and is
    not the derivative of the CC quasienergy); both keep alpha(-w+ig) = alpha(w+ig)*."""
    inst = synth.make_instance(4, 8, seed=5, sd=0.05)
    s = R.CCSystem(Ints.from_instance(inst))
    A = s.dense_A()
    zs = [0.1 + 0.01j, -0.1 + 0.01j]
    cc = s.response(inst.ops, zs, solver="dense", A=A)
    ci = s.response(inst.ops, zs, solver="dense", A=A, form="ci")
    assert np.abs(ci - cc).max() > 1e-6 * np.abs(cc).max()
    assert np.abs(ci[1] - np.conj(ci[0])).max() < 1e-11 * np.abs(ci).max()


def mixed_operators(n, seed):
    """An electric-dipole-like real symmetric matrix and a magnetic-dipole-like Hermitian matrix
    that is purely imaginary (i times a real antisymmetric one): the operator pair of optical
    rotation, G'(w) = -Im <<mu; m>>."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0, 0.1, (n, n))
    b = rng.normal(0, 0.1, (n, n))
    return np.stack([(a + a.T) / 2 + 0j, 1j * (b - b.T) / 2])


def test_two_electron_mixed_electric_magnetic_operators():
    """<<mu; m>> for an electric and a magnetic-type operator equals the exact sum over states,
    both response forms."""
    inst = synth.make_instance(2, 8, seed=11, sd=0.05)
    ops = mixed_operators(inst.n_occ + inst.n_vir, 4)
    s = R.CCSystem(Ints.from_instance(inst))
    sos, _ = det.fci_response(inst.fock, synth.full_eri(inst), 2, ops, ZS)
    A = s.dense_A()
    for form in ("cc", "ci"):
        got = s.response(ops, ZS, solver="dense", A=A, form=form)
        assert np.abs(got - sos).max() < 1e-11 * np.abs(sos).max()
    assert np.abs(sos[1, 0, 1]) > 1e-6   # the mixed element is not trivially zero


def test_lambda_matches_dense_left_solve():
    inst = synth.make_instance(2, 6, seed=3, sd=0.1)
    s = R.CCSystem(Ints.from_instance(inst))
    A = s.dense_A()
    lam = -np.linalg.solve(A.T, s.eta_ground())
    assert np.abs(deriv.pack(s.l1, s.l2) - lam).max() < 1e-11


def test_finite_field_second_derivative():
    """2 f(0) == d^2 E_CCSD / d e_x d e_y with H -> H + e_x X + e_y Y (Richardson, h = 1e-3)."""
    inst = synth.make_instance(4, 8, seed=3, sd=0.05)
    I = Ints.from_instance(inst)
    X = inst.ops[:2]
    f0 = R.CCSystem(I).response(X, [0.0], half=True, tol=1e-12)[0]

    def E(ex, ey):
        return ccsd.solve(I.with_fock(inst.fock + ex * X[0] + ey * X[1]), tol=1e-13)[2]

    def d2(h):
        return np.array([(E(h, 0) - 2 * E(0, 0) + E(-h, 0)) / h**2,
                         (E(h, h) - E(h, -h) - E(-h, h) + E(-h, -h)) / (4 * h * h)])

    rich = (4 * d2(1e-3) - d2(2e-3)) / 3
    assert abs(rich[0] - 2 * f0[0, 0]) < 1e-7 * abs(f0[0, 0])
    assert abs(rich[1] - 2 * f0[0, 1]) < 1e-7 * abs(f0[0, 0])


def test_no_interaction_closed_form():
    """V = 0: alpha_xy(z) = sum_ia [x_ia y_ai/(D_ia - z) + y_ia x_ai/(D_ia + z)]."""
    o, v = 3, 6
    inst = synth.make_instance(o, v, sd=0.0)
    s = R.CCSystem(Ints.from_instance(inst))
    a = R.polarizability(s.response(inst.ops, ZS, tol=1e-12))
    eps = np.diag(inst.fock).real
    Dia = eps[None, o:] - eps[:o, None]
    for k, z in enumerate(ZS):
        for x in range(3):
            for y in range(3):
                X, Y = inst.ops[x], inst.ops[y]
                ref = np.sum(X[:o, o:] * Y[o:, :o].T / (Dia - z) + Y[:o, o:] * X[o:, :o].T / (Dia + z))
                assert abs(a[k, x, y] - ref) < 1e-11


@pytest.fixture(scope="module")
def correlated():
    inst = synth.make_instance(4, 10, seed=5, sd=0.05)
    return inst, R.CCSystem(Ints.from_instance(inst))


def test_symmetries(correlated):
    inst, s = correlated
    w, g = 0.12, 0.01
    a = R.polarizability(s.response(inst.ops, [w + 1j * g, -w + 1j * g, 0.0], tol=1e-12))
    assert np.abs(a[1] - a[0].conj()).max() < 1e-10           # alpha(-w + ig) = alpha(w + ig)*
    assert np.abs(a[2] - a[2].T).max() < 1e-10                # static alpha is symmetric
    assert np.abs(a[2].imag).max() < 1e-10                    # real without damping at w = 0
    assert np.all(np.diag(a[0]).imag > 0)                     # absorption: Im alpha_xx > 0
    assert np.all(np.diag(a[2]).real > 0)
    a2 = R.polarizability(s.response(2.5 * inst.ops[:1], [w + 1j * g], tol=1e-12))
    assert abs(a2[0, 0, 0] - 6.25 * a[0, 0, 0]) < 1e-10 * abs(a[0, 0, 0])


def test_real_hamiltonian_limit():
    """Real integrals and operators: alpha is real when gamma = 0."""
    inst = synth.make_instance(3, 6, seed=9, sd=0.05)
    for k, b in inst.blocks.items():
        inst.blocks[k] = b.real.astype(complex)
    inst.ops = inst.ops.real.astype(complex)
    s = R.CCSystem(Ints.from_instance(inst))
    a = R.polarizability(s.response(inst.ops, [0.0, 0.1], tol=1e-12))
    assert np.abs(a.imag).max() < 1e-12


def test_derived_quantities():
    alpha = np.diag([1.0, 2.0, 6.0]).astype(complex)[None]
    assert R.mean_alpha(alpha)[0] == 3.0
    assert R.anisotropy(alpha)[0] == 4.5
    alpha = alpha + 1j * np.eye(3)[None]
    assert abs(R.cross_section([0.1], alpha)[0] - 4 * np.pi * 0.1 / 137.035999084) < 1e-15


def test_asymmetric_form_two_electron_sum_over_states(two_electron):
    """The asymmetric CC-CC form (first-order multipliers from left solves) is exact for two
    electrons too."""
    inst, s, sos = two_electron
    got = s.response(inst.ops, ZS, solver="dense", A=s.dense_A(), form="asym")
    assert np.abs(got - sos).max() < 1e-11 * np.abs(sos).max()


@pytest.fixture(scope="module")
def four_electron():
    inst = synth.make_instance(4, 8, seed=5, sd=0.05)
    s = R.CCSystem(Ints.from_instance(inst))
    return inst, s, s.dense_A()


def test_asymmetric_form_equals_symmetric_form(four_electron):
    """Beyond two electrons the asymmetric and symmetric CC-CC forms still agree (Sec. 2.3): the
    identity tbar^Y(z) xi^X = eta^Y t^X(-z) + t^X(-z) F t^Y(z) holds for the exact solutions.
    Dense and Davidson solves, static and damped shifts."""
    inst, s, A = four_electron
    zs = [0.0, 0.1 + 0.01j, -0.07 + 0.02j]
    cc = s.response(inst.ops, zs, solver="dense", A=A)
    asym = s.response(inst.ops, zs, solver="dense", A=A, form="asym")
    assert np.abs(asym - cc).max() < 1e-11 * np.abs(cc).max()
    dav = s.response(inst.ops, zs[1:], tol=1e-12, form="asym")
    assert np.abs(dav - cc[1:]).max() < 1e-9 * np.abs(cc).max()


def test_first_order_multipliers_solve_the_left_equation(four_electron):
    """The left Davidson (op = left sigma) against the dense transpose: tbar (A + w) = -b."""
    inst, s, A = four_electron
    rng = np.random.default_rng(2)
    b = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
    w = 0.12 + 0.01j
    tb = s.davidson(b, -w, tol=1e-12, op=s.sigma_l)[0]
    assert np.abs(tb @ (A + w * np.eye(A.shape[0])) + b).max() < 1e-10 * np.abs(b).max()


def test_asymmetric_form_needs_the_hessian_term(four_electron, monkeypatch):
    """Planted mistake: without F t^Y in the multiplier right-hand side the two forms disagree, so
    the equality above does check that term."""
    inst, s, A = four_electron
    zs = [0.1 + 0.01j]
    cc = s.response(inst.ops, zs, solver="dense", A=A)
    monkeypatch.setattr(s, "hessian", lambda u: np.zeros_like(u))
    bad = s.response(inst.ops, zs, solver="dense", A=A, form="asym")
    assert np.abs(bad - cc).max() > 1e-4 * np.abs(cc).max()


def _herm(n, seed, scale):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return scale * (a + a.conj().T) / 2


def _richardson(fun, h=1e-3):
    """d/d eps at 0 by central differences at h and h/2 with one Richardson step (error O(h^4))."""
    d1 = (fun(h) - fun(-h)) / (2 * h)
    d2 = (fun(h / 2) - fun(-h / 2)) / h
    return (4 * d2 - d1) / 3


ZF = [0.0, 0.1 + 0.01j]


def test_field_derivative_two_electron_matches_fci_finite_field():
    """The analytic static-field derivative of <<X;Y>> (field V on the Fock matrix) against the
    finite-field derivative of the exact sum over states (FCI) for two electrons."""
    inst = synth.make_instance(2, 6, seed=11, sd=0.05)
    V = _herm(8, 3, 0.05)
    got = R.CCSystem(Ints.from_instance(inst)).field_derivative(inst.ops, V, ZF)
    eri = synth.full_eri(inst)
    ref = _richardson(lambda e: det.fci_response(inst.fock + e * V, eri, 2, inst.ops, ZF)[0])
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()


def test_field_derivative_matches_cc_finite_field(four_electron):
    """Four electrons: against the finite-field derivative of the CC-CC response function itself
    (CCSD, Lambda and the response solved again at eps = +-h, +-h/2); dense and Davidson solves."""
    inst, s, A = four_electron
    V = _herm(12, 4, 0.05)
    got = s.field_derivative(inst.ops, V, ZF, A=A)

    def resp(e):
        se = R.CCSystem(s.I.with_fock(inst.fock + e * V), tol=1e-13)
        return se.response(inst.ops, ZF, solver="dense", A=se.dense_A())
    ref = _richardson(resp)
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()
    dav = s.field_derivative(inst.ops, V, ZF[1:], solver="davidson", tol=1e-12)
    assert np.abs(dav - got[1:]).max() < 1e-8 * np.abs(ref).max()


def test_field_derivative_needs_the_multiplier_response(four_electron, monkeypatch):
    """Planted mistake: with the multipliers held at lambda0 in every shifted system (the
    lambda^V terms dropped) the derivative no longer matches, so the pin above checks them."""
    inst, s, A = four_electron
    V = _herm(12, 4, 0.05)
    good = s.field_derivative(inst.ops, V, ZF[1:], A=A)
    orig = R.CCSystem.at
    monkeypatch.setattr(R.CCSystem, "at", lambda self, t=None, lam=None: orig(self, t=t))
    bad = s.field_derivative(inst.ops, V, ZF[1:], A=A)
    assert np.abs(bad - good).max() > 1e-4 * np.abs(good).max()


def test_static_field_derivative_is_a_symmetric_third_derivative(four_electron):
    """At w = 0 and gamma = 0 the CC-CC response function is the second derivative of the CC
    energy, so its field derivative along X_z is the third derivative: d<<X_x;X_y>>/d eps_z is
    symmetric in x, y and z."""
    inst, s, A = four_electron
    D = [s.field_derivative(inst.ops, inst.ops[z], [0.0], A=A)[0] for z in range(3)]
    scale = max(np.abs(d).max() for d in D)
    for x in range(3):
        for y in range(3):
            for z in range(3):
                assert abs(D[z][x, y] - D[y][x, z]) < 1e-10 * scale
                assert abs(D[z][x, y] - D[x][z, y]) < 1e-10 * scale

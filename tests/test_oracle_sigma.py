"""Sigma vectors pinned against derivatives of the CCSD residual and against FCI."""
import numpy as np
import pytest
import synth
from oracle import ccsd, det, deriv, hbar, sigma, response
from oracle.ints import Ints
from oracle_cases import general_case, rand_amp


@pytest.mark.parametrize("o,v", [(2, 4), (3, 5), (4, 6)])
def test_right_sigma_is_jacobian(o, v):
    """A r == d/ds Omega(t + s r) at random (non-converged) t, general complex Fock."""
    inst, F, I = general_case(o, v)
    t1, t2 = rand_amp(o, v, 1)
    H = hbar.Hbar(I, t1, t2)
    for blocks in [(1, 0), (0, 1), (1, 1)]:
        r1, r2 = rand_amp(o, v, 3)
        r1, r2 = r1 * blocks[0], r2 * blocks[1]
        s1, s2 = sigma.sigma_right(H, I, r1, r2)
        d1, d2 = deriv.jacobian_right(I, t1, t2, r1, r2)
        scale = max(np.abs(d1).max(), np.abs(d2).max())
        assert np.abs(s1 - d1).max() < 1e-12 * scale
        assert np.abs(s2 - d2).max() < 1e-12 * scale


@pytest.mark.parametrize("o,v", [(2, 4), (3, 5)])
def test_left_sigma_bilinear_identity(o, v):
    """(l A) . r == l . (A r) for every block pairing."""
    inst, F, I = general_case(o, v)
    t1, t2 = rand_amp(o, v, 1)
    H = hbar.Hbar(I, t1, t2)
    r1, r2 = rand_amp(o, v, 3)
    l1, l2 = rand_amp(o, v, 5)
    for lb in [(1, 0), (0, 1)]:
        for rb in [(1, 0), (0, 1)]:
            a1, a2 = l1 * lb[0], l2 * lb[1]
            b1, b2 = r1 * rb[0], r2 * rb[1]
            L1, L2 = sigma.sigma_left(H, I, a1, a2)
            lhs = deriv.dot(L1, L2, b1, b2)
            rhs = deriv.left_dot(I, t1, t2, a1, a2, b1, b2)
            assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))


def test_dense_jacobian_matches_sigma_columns():
    inst, F, I = general_case(2, 4)
    t1, t2 = rand_amp(2, 4, 1)
    A = deriv.jacobian_dense(I, t1, t2)
    H = hbar.Hbar(I, t1, t2)
    for k in range(A.shape[0]):
        e = np.zeros(A.shape[0], complex)
        e[k] = 1
        r1, r2 = deriv.unpack(e, 2, 4)
        assert np.abs(deriv.pack(*sigma.sigma_right(H, I, r1, r2)) - A[:, k]).max() < 1e-12


def test_two_electron_jacobian_eigenvalues_are_fci_excitations():
    """eig(A) == E_n - E_0 for two electrons (CC-LR poles are exact)."""
    inst = synth.make_instance(2, 6, seed=11, sd=0.05)
    I = Ints.from_instance(inst)
    s = response.CCSystem(I)
    ev = np.sort(np.linalg.eigvals(s.dense_A()).real)
    w = det.fci_energies(inst.fock, synth.full_eri(inst), 2)
    assert np.abs(ev - (w[1:] - w[0])).max() < 1e-11


def test_eom_energies_are_the_lowest_fci_excitations():
    """The oracle's EOM-EE roots (lowest by real part) == the lowest FCI excitation energies."""
    inst = synth.make_instance(2, 8, seed=11, sd=0.05)
    s = response.CCSystem(Ints.from_instance(inst))
    got = s.eom_energies(4)
    w = det.fci_energies(inst.fock, synth.full_eri(inst), 2)
    assert np.abs(got - (w[1:5] - w[0])).max() < 1e-11


def test_pins_detect_planted_mistakes():
    """A plausible slip in one Hbar element (sign, conjugation, index order) breaks the pin."""
    inst, F, I = general_case(3, 5)
    t1, t2 = rand_amp(3, 5, 1)
    r1, r2 = rand_amp(3, 5, 3)
    d1, d2 = deriv.jacobian_right(I, t1, t2, r1, r2)
    plants = {
        "ladder sign": lambda H: setattr(H, "Wabef", -H.Wabef),
        "ring conjugated": lambda H: setattr(H, "Wmbej", H.Wmbej.conj()),
        "Fae transposed": lambda H: setattr(H, "Fae", H.Fae.T.copy()),
        "Wmnie dropped T1": lambda H: setattr(H, "Wmnie", I["ooov"]),
    }
    for name, plant in plants.items():
        H = hbar.Hbar(I, t1, t2)
        plant(H)
        s1, s2 = sigma.sigma_right(H, I, r1, r2)
        err = max(np.abs(s1 - d1).max(), np.abs(s2 - d2).max())
        assert err > 1e-4, name

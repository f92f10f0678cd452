"""Ground-state CCSD oracle pinned against the determinant-space definition."""
import numpy as np
import pytest
import synth
from oracle import ccsd, det
from oracle.ints import Ints
from oracle_cases import general_case, rand_amp


@pytest.mark.parametrize("o,v", [(2, 4), (3, 5), (4, 4)])
def test_residual_equals_projection(o, v):
    """Omega from the factorized equations == <mu|e^-T H e^T|R> at random amplitudes."""
    inst, F, I = general_case(o, v)
    D = det.CCDet(F, synth.full_eri(inst), o)
    t1, t2 = rand_amp(o, v, 1)
    r1, r2 = ccsd.residual(I, t1, t2)
    d1, d2 = D.residual(t1, t2)
    assert np.abs(r1 - d1).max() < 1e-13 * max(1, np.abs(d1).max())
    assert np.abs(r2 - d2).max() < 1e-13 * max(1, np.abs(d2).max())
    assert abs(ccsd.energy(I, t1, t2) - D.energy(t1, t2)) < 1e-13


def test_two_electron_ccsd_is_fci():
    """For two electrons CCSD is exact: E_ref + E_corr is the lowest FCI eigenvalue."""
    inst = synth.make_instance(2, 8, seed=11, sd=0.05)
    I = Ints.from_instance(inst)
    g = synth.full_eri(inst)
    t1, t2, e, _ = ccsd.solve(I)
    D = det.CCDet(inst.fock, g, 2)
    assert abs(e - (det.fci_energies(inst.fock, g, 2)[0] - D.e_ref)) < 1e-12


def test_no_interaction_gives_zero_amplitudes():
    inst = synth.make_instance(3, 6, sd=0.0)
    t1, t2, e, it = ccsd.solve(Ints.from_instance(inst))
    assert np.abs(t1).max() == 0 and np.abs(t2).max() == 0 and e == 0


def test_converged_residual_and_antisymmetry():
    inst = synth.make_instance(4, 8, seed=5)
    I = Ints.from_instance(inst)
    t1, t2, e, _ = ccsd.solve(I, tol=1e-12)
    r1, r2 = ccsd.residual(I, t1, t2)
    assert np.abs(r1).max() < 1e-12 and np.abs(r2).max() < 1e-12
    assert np.abs(t2 + t2.transpose(1, 0, 2, 3)).max() < 1e-15
    assert np.abs(t2 + t2.transpose(0, 1, 3, 2)).max() < 1e-15

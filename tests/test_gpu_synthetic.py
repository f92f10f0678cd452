"""cclr_set_synthetic against the host generator (synth.counter), bit for bit.

The device generates the counter-based instance; the same instance generated on the host goes in
through cclr_set_hamiltonian.  The operators the call returns must equal the host's exactly, and
everything computed from the two Hamiltonians (the CCSD energy, a sigma product) must be
bitwise equal, which holds only if every stored integral is."""
import numpy as np
import pytest

import synth
from synth import counter as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import os
    os.environ.setdefault("CCLR_WORKSPACE_GB", "2")
    import paper_2307_14296_b300 as pk
    return pk


@pytest.mark.parametrize("o,v,seed", [(4, 20, 230714296), (6, 17, 3)])
def test_device_instance_equals_host_generator(pk, o, v, seed):
    sd = synth.integral_sd(o, v)
    inst = C.make_counter_instance(o, v, seed, sd=sd)
    dev = pk.Context(0, tol=1e-10, ground_tol=1e-11)
    ops = dev.cclr_set_synthetic(o, v, seed, sd, 0.1, 3)
    assert np.array_equal(ops, inst.ops)
    host = pk.Context(0, tol=1e-10, ground_tol=1e-11)
    host.cclr_set_hamiltonian(o, v, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
    e_dev, _ = dev.cc_ground()
    e_host, _ = host.cc_ground()
    assert e_dev == e_host
    x = synth.random_vector((2, dev.N), 9, 9, 1e-2)
    assert np.array_equal(dev.cclr_sigma(x), host.cclr_sigma(x))
    assert np.array_equal(dev.cclr_get_amplitudes(pk.AMP_T), host.cclr_get_amplitudes(pk.AMP_T))
    dev.close()
    host.close()


def test_synthetic_rejects_bad_arguments(pk):
    ctx = pk.Context(0)
    with pytest.raises(pk.CCLRError) as e:
        ctx.cclr_set_synthetic(1, 10, 1, 0.01)
    assert e.value.status == pk.CCLR_E_ARG
    with pytest.raises(pk.CCLRError) as e:
        ctx.cclr_set_synthetic(3, 10, 1, float("nan"))
    assert e.value.status == pk.CCLR_E_ARG
    ctx.close()

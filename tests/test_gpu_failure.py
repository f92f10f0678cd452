"""Failure handling through the C ABI, with no GPU fault: every failure is made on the host
(bad inputs, a capped workspace, call-order violations, too few iterations) or by a bounded
device wait that is made to run out on a barrier phase that nothing completes.  Each call
returns its status code and leaves the context (or a new one) usable."""
import numpy as np
import pytest

import synth
from layout import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import os
    os.environ.setdefault("CCLR_WORKSPACE_GB", "4")
    import paper_2307_14296_b300 as pk
    return pk


def blocks(inst):
    return [inst.blocks[k] for k in synth.CLASSES]


def test_bounded_wait_expiry_returns_timeout_and_the_context_recovers(pk):
    inst = synth.make_instance(4, 10)
    ctx = pk.Context(0)
    ctx.cclr_set_hamiltonian(4, 10, inst.fock, blocks(inst))
    A = synth.random_vector((300, 700), 3, 1)
    B = synth.random_vector((260, 700), 3, 2)
    ctx.cclr_debug_expire_next_wait(4096)
    with pytest.raises(pk.CCLRError) as e:
        ctx.cclr_zgemm_nt(A, B, precision=pk.TC_BF16X3)
    assert e.value.status == pk.CCLR_E_TIMEOUT
    for _ in range(2):   # the status word was cleared; the next calls are correct
        assert rel(ctx.cclr_zgemm_nt(A, B, precision=pk.TC_BF16X3), A @ B.T) < 1e-4
    ctx.close()


@pytest.mark.parametrize("where", ["fock", "vvvv", "ooov"])
def test_nonfinite_hamiltonian_is_an_argument_error(pk, where):
    inst = synth.make_instance(3, 6)
    fock, bl = inst.fock.copy(), [b.copy() for b in blocks(inst)]
    if where == "fock":
        fock[1, 2] = np.nan
    else:
        bl[synth.CLASSES.index(where)].flat[3] = complex(0.0, np.inf)
    ctx = pk.Context(0)
    with pytest.raises(pk.CCLRError) as e:
        ctx.cclr_set_hamiltonian(3, 6, fock, bl)
    assert e.value.status == pk.CCLR_E_ARG and "NaN" in str(e.value)
    with pytest.raises(pk.CCLRError) as e:   # no Hamiltonian was kept
        ctx.cc_ground()
    assert e.value.status == pk.CCLR_E_STATE
    ctx.cclr_set_hamiltonian(3, 6, inst.fock, blocks(inst))   # a clean one is accepted
    ctx.cc_ground()
    ctx.close()


def test_nonfinite_operator_or_frequency_is_an_argument_error(pk):
    inst = synth.make_instance(3, 6)
    ctx = pk.Context(0)
    ctx.cclr_set_hamiltonian(3, 6, inst.fock, blocks(inst))
    ctx.cc_ground()
    ctx.cc_lambda()
    ops = inst.ops.copy()
    ops[1, 0, 4] = np.nan
    for bad_ops, om in ((ops, [0.1]), (inst.ops, [np.inf])):
        with pytest.raises(pk.CCLRError) as e:
            ctx.cc_lr_solve(bad_ops, om, 0.0)
        assert e.value.status == pk.CCLR_E_ARG
    ctx.cc_lr_solve(inst.ops, [0.1], 0.0)
    ctx.close()


def test_capped_workspace_is_out_of_memory(pk, monkeypatch):
    inst = synth.make_instance(4, 20)
    monkeypatch.setenv("CCLR_WORKSPACE_GB", "0.0002")   # 200 KiB: the ground state needs more
    ctx = pk.Context(0)
    ctx.cclr_set_hamiltonian(4, 20, inst.fock, blocks(inst))
    with pytest.raises(pk.CCLRError) as e:
        ctx.cc_ground()
    assert e.value.status == pk.CCLR_E_OOM and "workspace" in str(e.value)
    ctx.close()
    monkeypatch.setenv("CCLR_WORKSPACE_GB", "2")
    ctx = pk.Context(0)
    ctx.cclr_set_hamiltonian(4, 20, inst.fock, blocks(inst))
    ctx.cc_ground()
    ctx.close()


def test_call_order_violations_are_state_errors(pk):
    inst = synth.make_instance(3, 6)
    ctx = pk.Context(0)
    with pytest.raises(pk.CCLRError) as e:
        ctx.cc_ground()                       # no Hamiltonian
    assert e.value.status == pk.CCLR_E_STATE
    ctx.cclr_set_hamiltonian(3, 6, inst.fock, blocks(inst))
    for call in (ctx.cc_lambda, lambda: ctx.cc_lr_solve(inst.ops, [0.1], 0.0)):
        with pytest.raises(pk.CCLRError) as e:
            call()
        assert e.value.status == pk.CCLR_E_STATE
    ctx.cc_ground()
    ctx._nops, ctx._nfreq = 3, 1
    with pytest.raises(pk.CCLRError) as e:
        ctx.cc_response_function()           # before cc_lr_solve
    assert e.value.status == pk.CCLR_E_STATE
    for call in (ctx.cc_response_function_asym, lambda: ctx.cclr_field_derivative(np.zeros((2, 2), complex))):
        with pytest.raises(pk.CCLRError) as e:
            call()                           # before cc_lr_solve (V is not read)
        assert e.value.status == pk.CCLR_E_STATE
    ctx.close()


def test_iteration_limit_is_noconv_with_the_iterate_kept(pk):
    inst = synth.make_instance(4, 20)
    ctx = pk.Context(0, maxit=1, ground_tol=1e-13)
    ctx.cclr_set_hamiltonian(4, 20, inst.fock, blocks(inst))
    with pytest.raises(pk.CCLRError) as e:
        ctx.cc_ground()
    assert e.value.status == pk.CCLR_E_NOCONV
    t = ctx.cclr_get_amplitudes(pk.AMP_T)
    assert np.all(np.isfinite(t)) and np.abs(t).max() > 0
    ctx.close()

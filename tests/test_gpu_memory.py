"""Device memory stays flat across repeated solve cycles on one context.

Each cycle (ground state, Lambda, linear response, response function) must release what the
previous cycle allocated: the second and third cycles end with the same free device memory
(within 4 MiB, two of the CUDA driver's 2 MiB pages; one leaked set of response arrays at this size
is ~20 MB).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_repeated_cycles_do_not_grow_device_memory():
    import os
    os.environ.setdefault("CCLR_WORKSPACE_GB", "4")
    import torch
    import paper_2307_14296_b300 as pk
    o, v = 6, 40   # trial vectors of 0.19 MB (11940 amplitudes)
    inst = synth.make_instance(o, v)
    ctx = pk.Context(0, precision=pk.TC_BF16X3, tol=1e-8, ground_tol=1e-8, max_subspace=32, batch=4)
    ctx.cclr_set_hamiltonian(o, v, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
    om = np.array([0.05, 0.2])
    free = []
    for _ in range(3):
        ctx.cc_ground()
        ctx.cc_lambda()
        ctx.cc_lr_solve(inst.ops, om, 0.01)
        ctx.cc_response_function()
        free.append(torch.cuda.mem_get_info(0)[0])
    assert abs(free[2] - free[1]) < 4 << 20, free

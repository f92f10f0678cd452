"""The allocation-free tensor-core GEMM entry point against the context-based one.

cclr_zgemm_nt_noalloc exists for callers that cannot allocate device memory (a framework that owns
all device memory through its own pool, a server with a fixed footprint): it takes device
pointers and keeps its temporaries in one fixed device array inside the library.  This file runs
last (its name sorts after the others) so that a failure here cannot hide other results, and it
also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import synth
from layout import rel

pytestmark = pytest.mark.gpu
TOL = 1e-4   # the bound the tensor-core tests use for three-product split-BF16 contractions


@pytest.fixture(scope="module")
def env():
    import os
    os.environ.setdefault("CCLR_WORKSPACE_GB", "4")
    import torch
    import paper_2307_14296_b300 as pk
    inst = synth.make_instance(4, 10)
    ctx = pk.Context(0)
    ctx.cclr_set_hamiltonian(4, 10, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
    yield pk, torch, ctx
    ctx.close()


@pytest.mark.parametrize("M,N,K", [(300, 500, 250), (40, 30, 20000)])
def test_noalloc_matches_context_gemm_twice(env, M, N, K):
    pk, torch, ctx = env
    A = synth.random_vector((M, K), 3, 1)
    B = synth.random_vector((N, K), 3, 2)
    ref = ctx.cclr_zgemm_nt(A, B, precision=pk.TC_BF16X3)   # existing entry point (context, host data)
    exact = A @ B.T
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    for _ in range(2):                                       # two calls in a row share the scratch
        dC = torch.full((M, N), float("nan"), dtype=torch.complex128, device="cuda")
        st = pk.cclr_zgemm_nt_noalloc(dA, dB, dC, precision=pk.TC_BF16X3)
        torch.cuda.synchronize()
        assert st == pk.CCLR_OK
        got = dC.cpu().numpy()
        assert rel(got, ref) < TOL
        assert rel(got, exact) < TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    pk, torch, ctx = env
    dA = torch.zeros((4096, 4096), dtype=torch.complex128, device="cuda")
    dC = torch.zeros((4096, 4096), dtype=torch.complex128, device="cuda")
    assert pk.cclr_zgemm_nt_noalloc(dA, dA, dC) == pk.CCLR_E_ARG
    assert pk.cclr_zgemm_nt_noalloc(dA, dA, dC, precision=pk.FP64) == pk.CCLR_E_ARG

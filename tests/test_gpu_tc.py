"""Tensor-core (tcgen05) complex GEMM and mixed-precision sigma vectors against FP64.

Bounds: split-BF16 with two slices (three products) keeps ~16 significant bits per operand, so a
contraction is accurate to ~2^-16 relative (1e-4 bound below); three slices (six products) are
limited by FP32 accumulation (1e-5 bound).  The errors must also be clearly nonzero, which shows
that the tensor-core path (not the FP64 one) produced the result.
"""
import numpy as np
import pytest

import synth
from layout import rel, to_amp
from oracle.deriv import antisym

pytestmark = pytest.mark.gpu
BOUND = {2: 1e-4, 3: 1e-5}


@pytest.fixture(scope="module")
def ctx():
    import os
    os.environ.setdefault("CCLR_WORKSPACE_GB", "4")
    import paper_2307_14296_b300 as pk
    inst = synth.make_instance(4, 10)
    c = pk.Context(0)
    c.cclr_set_hamiltonian(4, 10, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
    yield c
    c.close()


@pytest.mark.parametrize("M,N,K", [(256, 256, 512), (300, 500, 250), (64, 129, 4000), (513, 640, 77), (40, 30, 20000)])
@pytest.mark.parametrize("prec", [2, 3])
def test_tc_zgemm_matches_fp64(ctx, M, N, K, prec):
    A = synth.random_vector((M, K), 3, 1)
    B = synth.random_vector((N, K), 3, 2)
    ref = A @ B.T
    got = ctx.cclr_zgemm_nt(A, B, precision=prec)
    err = rel(got, ref)
    assert err < BOUND[prec], err
    assert err > 1e-12  # the BF16 path really ran
    f64 = ctx.cclr_zgemm_nt(A, B, precision=0)
    assert rel(f64, ref) < 1e-13


@pytest.mark.parametrize("M,N,K", [(256, 256, 512), (300, 500, 250), (64, 129, 4000), (513, 640, 77), (40, 30, 20000),
                                   (1000, 130, 1100)])
def test_tc_f64_zgemm_matches_fp64(ctx, M, N, K):
    """The FP64-class mode (five fixed-point digits per row, exact chunk sums).  Each element
    is represented to 2^-39 of its row maximum, and the dropped digit products (i + j >= 5) add at
    most ~2^-36 of max|A_m| max|B_n| per k, so |dC| <= 2^-34 K max|A_m| max|B_n| element-wise
    (the float-float rounding is far below).  With random signs the actual error is ~sqrt(K)
    times smaller: checked in the norm at 1e-10 of the FP64 product (observed 3-4e-11, as the
    digit-level emulation of the scheme predicts)."""
    A = synth.random_vector((M, K), 3, 1)
    B = synth.random_vector((N, K), 3, 2)
    A[:, : K // 3] *= 1e-3          # mixed magnitudes within rows
    B[: N // 2] *= 1e4              # and between rows
    ref = A @ B.T
    got = ctx.cclr_zgemm_nt(A, B, precision=4)
    amax = np.abs(A).max(axis=1)[:, None]
    bmax = np.abs(B).max(axis=1)[None, :]
    bound = 2.0 ** -34 * K * amax * bmax
    assert np.all(np.abs(got - ref) <= bound), float((np.abs(got - ref) / bound).max())
    assert rel(got, ref) < 1e-10, rel(got, ref)


def test_tc_f64_zgemm_special_values(ctx):
    """Zero rows, zero columns and a row of tiny values stay exact in the FP64-class mode."""
    M, N, K = 130, 200, 700
    A = synth.random_vector((M, K), 7, 1)
    B = synth.random_vector((N, K), 7, 2)
    A[5] = 0.0
    B[:, 100:] = 0.0
    A[9] *= 1e-20
    ref = A @ B.T
    got = ctx.cclr_zgemm_nt(A, B, precision=4)
    assert np.all(got[5] == 0.0)
    assert rel(got[9], ref[9]) < 1e-10
    assert rel(got, ref) < 1e-10


@pytest.mark.parametrize("prec", [2, 3])
def test_tc_sigma_matches_fp64(prec):
    import paper_2307_14296_b300 as pk
    o, v = 6, 40
    inst = synth.make_instance(o, v, seed=5)
    c = pk.Context(0)
    c.cclr_set_hamiltonian(o, v, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
    t1 = synth.random_vector((o, v), 1, 1, 0.05)
    t2 = antisym(synth.random_vector((o, o, v, v), 1, 2, 0.05))
    c.cclr_set_amplitudes(pk.AMP_T, to_amp(t1, t2))
    vecs = np.stack([to_amp(synth.random_vector((o, v), 2, 2 * k, 1.0),
                            antisym(synth.random_vector((o, o, v, v), 2, 2 * k + 1, 1.0))) for k in range(8)])
    for side in (0, 1):
        ref = c.cclr_sigma(vecs, side=side, precision=pk.FP64)
        got = c.cclr_sigma(vecs, side=side, precision=prec)
        err = rel(got, ref)
        assert err < BOUND[prec], (side, err)
        assert err > 1e-12
    c.close()


def test_tc_f64_sigma_matches_fp64():
    """Right and left sigma vectors in the FP64-class tensor-core mode against the FP64 (DFMA)
    path: the contractions carry ~1e-11 relative, so the sigma vectors agree to 1e-10."""
    import paper_2307_14296_b300 as pk
    o, v = 6, 40
    inst = synth.make_instance(o, v, seed=5)
    c = pk.Context(0)
    c.cclr_set_hamiltonian(o, v, inst.fock, [inst.blocks[k] for k in synth.CLASSES])
    t1 = synth.random_vector((o, v), 1, 1, 0.05)
    t2 = antisym(synth.random_vector((o, o, v, v), 1, 2, 0.05))
    c.cclr_set_amplitudes(pk.AMP_T, to_amp(t1, t2))
    c.cclr_set_amplitudes(pk.AMP_LAMBDA, to_amp(synth.random_vector((o, v), 3, 1, 0.05),
                                               antisym(synth.random_vector((o, o, v, v), 3, 2, 0.05))))
    vecs = np.stack([to_amp(synth.random_vector((o, v), 2, 2 * k, 1.0),
                            antisym(synth.random_vector((o, o, v, v), 2, 2 * k + 1, 1.0))) for k in range(8)])
    for side in (0, 1):
        ref = c.cclr_sigma(vecs, side=side, precision=pk.FP64)
        got = c.cclr_sigma(vecs, side=side, precision=pk.TC_F64)
        assert rel(got, ref) < 1e-10, (side, rel(got, ref))
    c.close()


@pytest.mark.parametrize("n,nx,ny", [(1, 1, 1), (1001, 3, 5), (70001, 40, 9), (130003, 33, 17), (4097, 8, 8)])
@pytest.mark.parametrize("mirror", [False, True])
def test_solver_gram_block(ctx, n, nx, ny, mirror):
    """The Davidson Gram kernel (FP32 arithmetic, compensated sums) against NumPy's X^H Y: ragged
    lengths (odd n exercises the 16-byte rounding of the mirrored chunk copies), tiles split over
    more than 32 X rows and 8 Y rows.  Bound: FP32 inputs (2^-24 relative) summed with
    compensation, 1e-6 of the largest entry."""
    X = synth.random_vector((nx, n), 5, 1)
    Y = synth.random_vector((ny, n), 5, 2)
    got = ctx.cclr_gram(X, Y, mirror=mirror)
    ref = np.conj(X) @ Y.T
    assert np.abs(got - ref).max() < 1e-6 * np.abs(ref).max()


def test_tile_autotuner_decides_and_stays_correct(ctx):
    """The first two launches of a GEMM shape run the 128-row and the 64-row tile (timed); the
    third uses the faster.  All three results must be correct, and the report lists the shape with
    both timings."""
    M, N, K = 200, 900, 2000
    A = synth.random_vector((M, K), 9, 1)
    B = synth.random_vector((N, K), 9, 2)
    ref = A @ B.T
    for _ in range(3):
        assert rel(ctx.cclr_zgemm_nt(A, B, precision=2), ref) < BOUND[2]
    rep = ctx.cclr_autotune_report()
    key = [k for k in rep if k.startswith(f"{M}x{N}x{(K + 63) // 64 * 64}/2/")]
    assert key, rep
    bn, stages, ms128, ms64 = rep[key[0]]
    assert bn in (64, 128) and ms128 > 0 and ms64 > 0
    assert (bn == 64) == (ms64 < ms128)

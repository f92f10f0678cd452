"""The counter-based synthetic generator (the host side of cclr_set_synthetic), no GPU.

Philox4x32-10 is checked against the published known-answer vectors of its authors' reference
implementation (Random123: zero counter and key, all-ones, and the digits of pi); the series
logarithm and sine / cosine against NumPy's library functions; the normal pairs against their
moments; the instance against the structure of the recipe (Hermitian classes, real diagonals,
sorted orbital energies in their ranges)."""
import numpy as np
import pytest

import synth
from synth import counter as C


@pytest.mark.parametrize("ctr,key,out", [
    ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff,) * 4, (0xffffffff, 0xffffffff), (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
])
def test_philox4x32_10_known_answers(ctr, key, out):
    got = C.philox4x32_10(*[[c] for c in ctr], *key)
    assert tuple(int(w[0]) for w in got) == out


def test_series_logarithm_and_trig_are_accurate():
    rng = np.random.default_rng(1)
    u = np.concatenate([rng.random(100000), [1.0, 0.5, 2.0 ** -53, 1 - 2.0 ** -53]])
    u = u[u > 0]
    assert np.abs(C._ln(u) - np.log(u)).max() < 4e-15
    a = rng.random(100000) * C.HALF_PI
    s, c = C._sincos_quarter(a)
    assert np.abs(s - np.sin(a)).max() < 4e-16 and np.abs(c - np.cos(a)).max() < 4e-16


def test_normal_pairs_have_standard_moments():
    re, im = C.normal_pairs(np.arange(400000, dtype=np.uint64), 3, 11, 1.0)
    z = np.concatenate([re, im])
    assert abs(z.mean()) < 5e-3 and abs(z.var() - 1) < 5e-3 and abs((z ** 4).mean() - 3) < 3e-2
    assert abs(np.corrcoef(re, im)[0, 1]) < 5e-3
    # independent streams and seeds
    re2, _ = C.normal_pairs(np.arange(1000, dtype=np.uint64), 4, 11, 1.0)
    re3, _ = C.normal_pairs(np.arange(1000, dtype=np.uint64), 3, 12, 1.0)
    assert not np.array_equal(re[:1000], re2) and not np.array_equal(re[:1000], re3)


def test_counter_instance_structure():
    o, v = 4, 9
    inst = C.make_counter_instance(o, v, seed=5)
    po, pv = synth.npair(o), synth.npair(v)
    b = inst.blocks
    assert b["oooo"].shape == (po, po) and b["vvvv"].shape == (pv, pv) and b["ovvv"].shape == (o, v, pv)
    for key in ("oooo", "vvvv"):
        assert np.array_equal(b[key], b[key].conj().T)
    m = b["ovov"].reshape(o * v, o * v)
    assert np.array_equal(m, m.conj().T)
    for X in inst.ops:
        assert np.array_equal(X, X.conj().T)
    e = inst.fock.diagonal().real
    assert np.all(np.diff(e[:o]) >= 0) and np.all(np.diff(e[o:]) >= 0)
    assert e[:o].min() >= -2.0 and e[:o].max() < -0.5 and e[o:].min() >= 0.3 and e[o:].max() < 4.0
    assert np.array_equal(inst.fock, np.diag(np.diag(inst.fock)))
    again = C.make_counter_instance(o, v, seed=5)
    assert all(np.array_equal(b[k], again.blocks[k]) for k in synth.CLASSES)
    # an element of a general class is its own index's draw
    re, im = C.normal_pairs(np.array([7], np.uint64), 3, 5, inst.meta["sd"])
    assert b["oovv"].ravel()[7] == re[0] + 1j * im[0]

"""Counter-based synthetic instances: the recipe of the device generator (cclr_set_synthetic).

Same statistics and packed layout as ``synth.make_instance`` but with random numbers that can be
produced for any element independently, on the host or on the device, with identical bits:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
  SC'11): counter (element index low 32 bits, high 32 bits, stream, 0), key (seed low 32 bits,
  seed high 32 bits), ten rounds with the published multipliers and Weyl key increments.
* Two uniforms from the four output words, u1 = ((w0 >> 5) 2^26 + (w1 >> 6) + 1) 2^-53 in (0, 1]
  and u2 = ((w2 >> 5) 2^26 + (w3 >> 6)) 2^-53 in [0, 1), both exact in binary64.
* Box-Muller, (Re, Im) = sd sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2), with the logarithm and the
  sine / cosine evaluated here from their series in a fixed order of correctly rounded additions,
  multiplications, divisions and square roots only (no library transcendental, no fused
  multiply-add), so that NumPy and the CUDA kernels give the same bits:
    ln u = e ln 2 + 2 s sum_j s^2j / (2j + 1),  u = m 2^e, m in [0.5, 1), s = (m - 1) / (m + 1);
    the angle 2 pi u2 is split into quadrant q = floor(4 u2) and a = (4 u2 - q) pi / 2 in [0, pi/2),
    sin a and cos a by their Taylor series in Horner form.
* Streams: 0 orbital energies (element index = spinor index, uniform u from the first two
  words), 1..6 the integral classes oooo, ooov, oovv, ovov, ovvv, vvvv (element index = storage
  index; Hermitian classes draw the element (min(I,J), max(I,J)) of their pair-space matrix,
  element index min * m + max, and conjugate below the diagonal; diagonal elements keep the real
  part), 100 + k the dipole operator k (a Hermitian n x n matrix drawn the same way).

This module draws random numbers and lays them out; it holds none of the coupled-cluster
arithmetic.
"""
from __future__ import annotations

import numpy as np

from . import Instance, integral_sd, npair

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
LN2 = 0.6931471805599453
HALF_PI = 1.5707963267948966
STREAM_EPS, STREAM_OPS = 0, 100
_LOG_TERMS = 20    # s^2j / (2j + 1), j < 20: |s| <= 1/3
_TRIG_TERMS = 13   # Taylor terms up to a^26 / 26!, a < pi / 2


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with ten rounds on arrays of 32-bit counters (held in uint64); returns the four
    output words (uint64 arrays holding 32-bit values)."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0, k1 = k0 & 0xFFFFFFFF, k1 & 0xFFFFFFFF
    for r in range(10):
        if r:
            k0, k1 = (k0 + _W0) & 0xFFFFFFFF, (k1 + _W1) & 0xFFFFFFFF
        p0, p1 = _M0 * c0, _M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ np.uint64(k0), p1 & _MASK,
                          (p0 >> np.uint64(32)) ^ c3 ^ np.uint64(k1), p0 & _MASK)
    return c0, c1, c2, c3


def _words(idx, stream: int, seed: int):
    idx = np.asarray(idx, dtype=np.uint64)
    return philox4x32_10(idx & _MASK, idx >> np.uint64(32), np.full(idx.shape, stream, np.uint64),
                         np.zeros(idx.shape, np.uint64), seed & 0xFFFFFFFF, seed >> 32)


def _u53(a, b):
    return ((a >> np.uint64(5)).astype(np.float64) * 67108864.0 + (b >> np.uint64(6)).astype(np.float64)) * 2.0 ** -53


def _ln(u):
    """ln u for u in (0, 1] (see the module docstring for the fixed evaluation order)."""
    m, e = np.frexp(u)
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    q = np.full_like(s, 1.0 / (2 * _LOG_TERMS - 1))
    for j in range(_LOG_TERMS - 2, -1, -1):
        q = 1.0 / (2 * j + 1) + s2 * q
    return e.astype(np.float64) * LN2 + (2.0 * s) * q


def _sincos_quarter(a):
    """(sin a, cos a) for a in [0, pi/2) by Horner-form Taylor series."""
    a2 = a * a
    S = np.ones_like(a)
    Cc = np.ones_like(a)
    for k in range(_TRIG_TERMS, 0, -1):
        S = 1.0 - (a2 / float((2 * k) * (2 * k + 1))) * S
        Cc = 1.0 - (a2 / float((2 * k - 1) * (2 * k))) * Cc
    return a * S, Cc


def normal_pairs(idx, stream: int, seed: int, sd: float):
    """(Re, Im) = sd (z0, z1), a Box-Muller pair of standard normals per element index."""
    w0, w1, w2, w3 = _words(idx, stream, seed)
    u1 = ((w0 >> np.uint64(5)).astype(np.float64) * 67108864.0 + (w1 >> np.uint64(6)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = _u53(w2, w3)
    r = np.sqrt(np.maximum(0.0, -2.0 * _ln(u1)))   # ln 1 may come out a few ulp above 0
    t4 = 4.0 * u2
    q = np.floor(t4)
    s, c = _sincos_quarter((t4 - q) * HALF_PI)
    qi = q.astype(np.int64)
    cos_t = np.select([qi == 0, qi == 1, qi == 2], [c, -s, -c], s)
    sin_t = np.select([qi == 0, qi == 1, qi == 2], [s, c, -s], -c)
    return sd * (r * cos_t), sd * (r * sin_t)


def uniforms(idx, stream: int, seed: int):
    """u in [0, 1) from the first two words of each element index."""
    w0, w1, _, _ = _words(idx, stream, seed)
    return _u53(w0, w1)


def hermitian(m: int, stream: int, seed: int, sd: float, rows=None) -> np.ndarray:
    """Rows `rows` (default all) of the Hermitian m x m matrix of a stream: element (I, J) is the
    pair drawn at index min(I, J) m + max(I, J), conjugated for I > J, real on the diagonal."""
    rows = np.arange(m) if rows is None else np.asarray(rows)
    I = rows[:, None].astype(np.uint64)
    J = np.arange(m, dtype=np.uint64)[None, :]
    lo, hi = np.minimum(I, J), np.maximum(I, J)
    re, im = normal_pairs(lo * np.uint64(m) + hi, stream, seed, sd)
    im = np.where(I > J, -im, np.where(I == J, 0.0, im))
    return re + 1j * im


def general(shape, stream: int, seed: int, sd: float) -> np.ndarray:
    idx = np.arange(int(np.prod(shape)), dtype=np.uint64)
    re, im = normal_pairs(idx, stream, seed, sd)
    return (re + 1j * im).reshape(shape)


def make_counter_instance(n_occ: int, n_vir: int, seed: int, sd: float | None = None, dip_sd: float = 0.1,
                          n_ops: int = 3, occ_range=(-2.0, -0.5), vir_range=(0.3, 4.0)) -> Instance:
    """The instance cclr_set_synthetic builds on the device (same layout as make_instance)."""
    o, v = n_occ, n_vir
    n = o + v
    if sd is None:
        sd = integral_sd(o, v)
    u = uniforms(np.arange(n, dtype=np.uint64), STREAM_EPS, seed)
    eo = np.sort(occ_range[0] + (occ_range[1] - occ_range[0]) * u[:o])
    ev = np.sort(vir_range[0] + (vir_range[1] - vir_range[0]) * u[o:])
    fock = np.diag(np.concatenate([eo, ev])).astype(np.complex128)
    po, pv = npair(o), npair(v)
    b = {"oooo": hermitian(po, 1, seed, sd), "ooov": general((po, o, v), 2, seed, sd),
         "oovv": general((po, pv), 3, seed, sd), "ovov": hermitian(o * v, 4, seed, sd).reshape(o, v, o, v),
         "ovvv": general((o, v, pv), 5, seed, sd), "vvvv": hermitian(pv, 6, seed, sd)}
    ops = np.stack([hermitian(n, STREAM_OPS + k, seed, dip_sd) for k in range(n_ops)])
    meta = dict(sd=sd, dip_sd=dip_sd, occ_range=occ_range, vir_range=vir_range, generator="counter")
    return Instance(o, v, fock, b, ops, seed, meta)

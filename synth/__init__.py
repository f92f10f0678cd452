"""Seeded synthetic relativistic-CC inputs (shared by the CUDA path's tests/bench and the oracle).

This module draws random numbers and lays them out; it holds none of the coupled-cluster
arithmetic.  It stands in for the molecular Hamiltonians of arXiv 2307.14296 (Sec. 4 and the
SI benchmark section), which need an integral code and basis sets.

Instance recipe (all complex128):
  * spinors 0..o-1 are occupied, o..o+v-1 virtual; Fock f = diag(eps) (canonical), with
    eps_occ ~ U[occ_lo, occ_hi], eps_vir ~ U[vir_lo, vir_hi], each sorted ascending;
  * antisymmetrized integrals <pq||rs> are drawn per canonical element, Re and Im independently
    N(0, sd^2), and every other element follows from <pq||rs> = -<qp||rs> = -<pq||sr> and
    <pq||rs> = conj(<rs||pq>).  Canonical elements whose bra and ket pairs coincide are real;
  * property operators X_k (dipole components) are Hermitian n x n, strict upper triangle
    Re, Im ~ N(0, dip_sd^2), real diagonal N(0, dip_sd^2).

Random streams: numpy's Philox (4x64, 10 rounds) counter-based generator keyed by (seed, stream):
  stream 0 orbital energies, 1..6 the six integral classes, 100+k property operator k.

Storage of the six integral classes (the layout the C ABI takes; pair index of p<q within one
index range is q*(q-1)/2 + p):
  oooo  <ij||kl>  [P(i<j)][P(k<l)]        Hermitian matrix over pairs
  ooov  <ij||ka>  [P(i<j)][k][a]
  oovv  <ij||ab>  [P(i<j)][P(a<b)]
  ovov  <ia||jb>  [i][a][j][b]            Hermitian matrix over (ia)
  ovvv  <ia||bc>  [i][a][P(b<c)]
  vvvv  <ab||cd>  [P(a<b)][P(c<d)]        Hermitian matrix over pairs
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

DEFAULT_SEED = 230714296
CLASSES = ("oooo", "ooov", "oovv", "ovov", "ovvv", "vvvv")


def npair(m: int) -> int:
    return m * (m - 1) // 2


def pair_index(p, q):
    """Packed index of the pair p<q (q*(q-1)/2 + p)."""
    return q * (q - 1) // 2 + p


def pair_table(m: int):
    """Arrays (p, q) listing the pairs p<q of range(m) in packed order."""
    q, p = np.tril_indices(m, -1)  # row q > column p, row-major order == packed order
    return p.astype(np.int64), q.astype(np.int64)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([seed, stream], dtype=np.uint64)))


def _cnormal(g: np.random.Generator, shape, sd: float) -> np.ndarray:
    out = np.empty(shape, dtype=np.complex128)
    out.real = g.normal(0.0, sd, size=shape)
    out.imag = g.normal(0.0, sd, size=shape)
    return out


def _hermitian(g: np.random.Generator, m: int, sd: float, chunk: int = 2048) -> np.ndarray:
    """m x m Hermitian matrix: strict upper triangle drawn, lower = conj transpose, real diagonal.

    Built in column tiles so that m ~ 3e4 (the vv pair space of large systems) fits in memory.
    """
    a = _cnormal(g, (m, m), sd)
    for c0 in range(0, m, chunk):
        c1 = min(m, c0 + chunk)
        # rows below the diagonal in columns c0..c1 take conj of the mirrored upper elements
        for r0 in range(c0, m, chunk):
            r1 = min(m, r0 + chunk)
            blk = a[r0:r1, c0:c1]
            mirror = a[c0:c1, r0:r1].T.conj()
            if r0 == c0:
                low = np.tril(np.ones((r1 - r0, c1 - c0), dtype=bool), -1)
                blk[low] = mirror[low]
            else:
                blk[...] = mirror
    d = np.arange(m)
    a[d, d] = a[d, d].real
    return a


@dataclass
class Instance:
    n_occ: int
    n_vir: int
    fock: np.ndarray                      # (n, n) complex128
    blocks: dict                          # packed integral classes (see module doc)
    ops: np.ndarray                       # (n_ops, n, n) complex128 Hermitian
    seed: int = DEFAULT_SEED
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.n_occ + self.n_vir


def integral_sd(n_occ: int, n_vir: int, sd0: float = 0.02) -> float:
    """Integral standard deviation with the coupling-to-gap ratio of the 4-occupied/20-virtual
    reference system.  A block of random antisymmetrized integrals over P pair (or
    particle-hole) states is a random Hermitian P x P matrix with spectral radius ~2 sd sqrt(2P);
    with sd fixed the ladder block grows past the orbital-energy gaps as n_vir grows (about 8 au
    at 200 virtuals against a smallest doubles gap of 1.6 au) and the CC equations lose their
    solution.  sd0 applies up to the reference size; beyond it sd shrinks as 1/sqrt of the
    largest block dimension, which keeps that spectral radius at the reference value."""
    ref = 20 * 19 // 2                                   # vv pair count of 20 virtuals
    big = max(n_vir * (n_vir - 1) // 2, n_occ * n_vir, n_occ * (n_occ - 1) // 2)
    return sd0 * min(1.0, float(np.sqrt(ref / max(big, 1))))


def make_instance(n_occ: int, n_vir: int, seed: int = DEFAULT_SEED, sd: float | None = None,
                  dip_sd: float = 0.1, n_ops: int = 3, occ_range=(-2.0, -0.5),
                  vir_range=(0.3, 4.0)) -> Instance:
    """sd: integral standard deviation per real component; None -> integral_sd(n_occ, n_vir)."""
    o, v = n_occ, n_vir
    if sd is None:
        sd = integral_sd(o, v)
    g = _rng(seed, 0)
    eo = np.sort(g.uniform(occ_range[0], occ_range[1], size=o))
    ev = np.sort(g.uniform(vir_range[0], vir_range[1], size=v))
    fock = np.diag(np.concatenate([eo, ev])).astype(np.complex128)
    po, pv = npair(o), npair(v)
    b = {}
    b["oooo"] = _hermitian(_rng(seed, 1), po, sd)
    b["ooov"] = _cnormal(_rng(seed, 2), (po, o, v), sd)
    b["oovv"] = _cnormal(_rng(seed, 3), (po, pv), sd)
    b["ovov"] = _hermitian(_rng(seed, 4), o * v, sd).reshape(o, v, o, v)
    b["ovvv"] = _cnormal(_rng(seed, 5), (o, v, pv), sd)
    b["vvvv"] = _hermitian(_rng(seed, 6), pv, sd)
    n = o + v
    ops = np.empty((n_ops, n, n), dtype=np.complex128)
    for k in range(n_ops):
        ops[k] = _hermitian(_rng(seed, 100 + k), n, dip_sd)
    meta = dict(sd=sd, dip_sd=dip_sd, occ_range=occ_range, vir_range=vir_range)
    return Instance(o, v, fock, b, ops, seed, meta)


# ----------------------------------------------------------------------------------------
# Layout conversion (input handling only): packed classes -> full-index blocks, full tensor
# ----------------------------------------------------------------------------------------

def _unpack_pair_axis(x: np.ndarray, axis: int, m: int) -> np.ndarray:
    """Expand a packed pair axis (p<q) into two full axes (p, q), antisymmetric."""
    p, q = pair_table(m)
    x = np.moveaxis(x, axis, 0)
    out = np.zeros((m, m) + x.shape[1:], dtype=x.dtype)
    out[p, q] = x
    out[q, p] = -x
    return np.moveaxis(out, (0, 1), (axis, axis + 1))


def full_blocks(inst: Instance) -> dict:
    """The six integral classes with every index explicit: e.g. 'vvvv' -> [a,b,c,d]."""
    o, v = inst.n_occ, inst.n_vir
    b = inst.blocks
    out = {}
    out["oooo"] = _unpack_pair_axis(_unpack_pair_axis(b["oooo"], 1, o), 0, o)
    out["ooov"] = _unpack_pair_axis(b["ooov"], 0, o)
    out["oovv"] = _unpack_pair_axis(_unpack_pair_axis(b["oovv"], 1, v), 0, o)
    out["ovov"] = b["ovov"].copy()
    out["ovvv"] = _unpack_pair_axis(b["ovvv"], 2, v)
    out["vvvv"] = _unpack_pair_axis(_unpack_pair_axis(b["vvvv"], 1, v), 0, v)
    return out


def full_eri(inst: Instance) -> np.ndarray:
    """Full <pq||rs> over all n spinors (small systems only: n^4 elements)."""
    o, n = inst.n_occ, inst.n
    fb = full_blocks(inst)
    O, V = slice(0, o), slice(o, n)
    sl = {"o": O, "v": V}
    g = np.zeros((n, n, n, n), dtype=np.complex128)

    def put(key, blk):
        g[sl[key[0]], sl[key[1]], sl[key[2]], sl[key[3]]] = blk

    for key, blk in fb.items():
        # the stored class and every element related to it by antisymmetry / Hermiticity
        forms = [(key, blk)]
        forms.append((key[1] + key[0] + key[2:], -blk.transpose(1, 0, 2, 3)))
        forms.append((key[:2] + key[3] + key[2], -blk.transpose(0, 1, 3, 2)))
        forms.append((key[1] + key[0] + key[3] + key[2], blk.transpose(1, 0, 3, 2)))
        for k2, b2 in list(forms):
            forms.append((k2[2:] + k2[:2], b2.transpose(2, 3, 0, 1).conj()))
        for k2, b2 in forms:
            put(k2, b2)
    return g


def random_hermitian(n: int, seed: int, stream: int, sd: float = 0.1) -> np.ndarray:
    """A seeded Hermitian n x n matrix (used for extra perturbation directions in tests)."""
    return _hermitian(_rng(seed, stream), n, sd)


def random_vector(shape, seed: int, stream: int, scale: float = 1.0) -> np.ndarray:
    """Seeded complex Gaussian array (trial vectors, amplitudes for tests)."""
    return _cnormal(_rng(seed, stream), shape, scale)

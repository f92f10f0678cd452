"""Integral classes by occupied/virtual index block (oracle; test infrastructure only).

Convention (SI, Working equations): V^{pq}_{rs} = <pq||rs>; upper indices are the bra
(creators), lower the ket (annihilators).  The six stored classes determine all sixteen blocks
through <pq||rs> = -<qp||rs> = -<pq||sr> and <pq||rs> = conj(<rs||pq>) (Hermiticity of H).
"""
from __future__ import annotations
import numpy as np
import synth


class Ints:
    """Fock blocks and <pq||rs> blocks keyed by 4-letter class strings such as 'ovvo'."""

    def __init__(self, fock: np.ndarray, full_blocks: dict, n_occ: int):
        o = n_occ
        self.o = o
        self.v = fock.shape[0] - o
        self.fock = fock
        self.f_oo = fock[:o, :o]
        self.f_ov = fock[:o, o:]
        self.f_vo = fock[o:, :o]
        self.f_vv = fock[o:, o:]
        self._b = dict(full_blocks)

    @classmethod
    def from_instance(cls, inst, fock=None):
        return cls(inst.fock if fock is None else fock, synth.full_blocks(inst), inst.n_occ)

    def with_fock(self, fock):
        new = Ints.__new__(Ints)
        new.__dict__.update(self.__dict__)
        o = self.o
        new.fock = fock
        new.f_oo, new.f_ov, new.f_vo, new.f_vv = fock[:o, :o], fock[:o, o:], fock[o:, :o], fock[o:, o:]
        return new

    def __getitem__(self, key: str) -> np.ndarray:
        b = self._b
        if key in b:
            return b[key]
        # antisymmetry in the bra pair
        swapped = key[1] + key[0] + key[2:]
        if swapped in ("ooov", "oovv", "ovov", "ovvv", "oooo", "vvvv") or swapped in b:
            out = -self[swapped].transpose(1, 0, 2, 3)
        elif (key[:2] + key[3] + key[2]) in b:
            out = -self[key[:2] + key[3] + key[2]].transpose(0, 1, 3, 2)
        elif (key[1] + key[0] + key[3] + key[2]) in b:
            out = self[key[1] + key[0] + key[3] + key[2]].transpose(1, 0, 3, 2)
        else:
            # Hermiticity: <pq||rs> = conj(<rs||pq>)
            out = self[key[2:] + key[:2]].transpose(2, 3, 0, 1).conj()
        out = np.ascontiguousarray(out)
        b[key] = out
        return out

"""Definition level in the N-electron determinant space (oracle; test infrastructure only).

Everything here is built from creation/annihilation operators, with no coupled-cluster algebra:
  * H = sum_pq h_pq a+_p a_q + 1/4 sum_pqrs <pq||rs> a+_p a+_q a_s a_r, with the bare one-electron
    part recovered from the Fock matrix, h_pq = f_pq - sum_m <pm||qm> (m occupied);
  * T = sum_ia t_i^a a+_a a_i + sum_{i<j,a<b} t_ij^ab a+_a a+_b a_j a_i  (Sec. 2.2, Eq. for T_0);
  * the CC residual Omega_mu = <mu| e^{-T} H e^{T} |R> and energy <R| e^{-T} H e^{T} |R>, with
    |mu> = tau_mu |R> (Sec. 2.3: xi, A, F are all projections of this kind);
  * FCI eigenstates and the exact sum-over-states response function
      <<X;Y>>_z = -sum_{n>0} [ X_0n Y_n0 / (w_n - z) + Y_0n X_n0 / (w_n + z) ]
    (the exact-state form that the paper's Eqs. fre-den-pol / complex-fre-den-pol restate for
    alpha = -<<mu;mu>>, with the sign reading that makes static alpha positive).

Determinants are occupation bitstrings; |D> = a+_{p1} a+_{p2} ... |vac> with p1 < p2 < ...
Only small spaces (C(n, N) up to a few thousand) are practical.
"""
from __future__ import annotations
from itertools import combinations
import numpy as np


class Space:
    """Bases of the N, N-1 and N-2 electron sectors and the operator matrices on them."""

    def __init__(self, n: int, n_elec: int):
        self.n, self.N = n, n_elec
        self.basis = {}
        self.index = {}
        for k in (n_elec, n_elec - 1, n_elec - 2):
            if k < 0:
                continue
            dets = [sum(1 << p for p in c) for c in combinations(range(n), k)]
            self.basis[k] = dets
            self.index[k] = {d: i for i, d in enumerate(dets)}
        self._ann = {}

    def ann(self, p: int, k: int) -> np.ndarray:
        """Matrix of a_p from the k-electron sector to the (k-1)-electron sector."""
        key = (p, k)
        if key not in self._ann:
            src, dst = self.basis[k], self.index[k - 1]
            m = np.zeros((len(self.basis[k - 1]), len(src)))
            for j, d in enumerate(src):
                if d >> p & 1:
                    sign = -1.0 if bin(d & ((1 << p) - 1)).count("1") % 2 else 1.0
                    m[dst[d ^ (1 << p)], j] = sign
            self._ann[key] = m
        return self._ann[key]

    def one_body(self, x: np.ndarray) -> np.ndarray:
        """sum_pq x_pq a+_p a_q on the N-electron sector."""
        N = self.N
        a = np.stack([self.ann(p, N) for p in range(self.n)])        # (n, dN-1, dN)
        return np.einsum("pq,pki,qkj->ij", x, a, a, optimize=True)

    def pair_ann(self):
        """Stack of a_s a_r (r<s) from N to N-2 electrons, with the pair list."""
        N = self.N
        pairs = [(r, s) for s in range(self.n) for r in range(s)]
        mats = np.stack([self.ann(s, N - 1) @ self.ann(r, N) for r, s in pairs])
        return pairs, mats

    def two_body(self, eri: np.ndarray) -> np.ndarray:
        """1/4 sum <pq||rs> a+_p a+_q a_s a_r = sum_{p<q, r<s} <pq||rs> (a_q a_p)^+ (a_s a_r)."""
        pairs, A = self.pair_ann()
        P = np.array(pairs)
        V = eri[P[:, 0][:, None], P[:, 1][:, None], P[:, 0][None, :], P[:, 1][None, :]]
        M = np.einsum("PR,Rkj->Pkj", V, A, optimize=True)
        return np.einsum("Pki,Pkj->ij", A, M, optimize=True)


def hamiltonian(space: Space, fock: np.ndarray, eri: np.ndarray, n_occ: int) -> np.ndarray:
    """N-electron Hamiltonian matrix from the Fock matrix and antisymmetrized integrals."""
    occ = np.arange(n_occ)
    h = fock - np.einsum("pmqm->pq", eri[:, occ][:, :, :, occ])
    return space.one_body(h) + space.two_body(eri)


def reference_index(space: Space, n_occ: int) -> int:
    return space.index[space.N][(1 << n_occ) - 1]


def excitation_ops(space: Space, n_occ: int):
    """Matrices of tau_ia = a+_a a_i and tau_ijab = a+_a a+_b a_j a_i (i<j, a<b) on the N sector."""
    n, N = space.n, space.N
    v = n - n_occ
    a = [space.ann(p, N) for p in range(n)]
    single = np.zeros((n_occ, v) + (len(space.basis[N]),) * 2)
    for i in range(n_occ):
        for e in range(v):
            single[i, e] = a[n_occ + e].T @ a[i]
    pairs, A = space.pair_ann()
    pidx = {p: k for k, p in enumerate(pairs)}
    double = {}
    for j in range(n_occ):
        for i in range(j):
            for b in range(v):
                for e in range(b):
                    # a+_a a+_b a_j a_i with a<b: (a_b a_a)^+ (a_j a_i)
                    double[(i, j, e, b)] = A[pidx[(n_occ + e, n_occ + b)]].T @ A[pidx[(i, j)]]
    return single, double


class CCDet:
    """e^{-T} H e^{T} projections in the determinant space for given f, <pq||rs>."""

    def __init__(self, fock: np.ndarray, eri: np.ndarray, n_occ: int):
        n = fock.shape[0]
        self.o, self.v = n_occ, n - n_occ
        self.space = Space(n, n_occ)
        self.H = hamiltonian(self.space, fock, eri, n_occ)
        self.ref = reference_index(self.space, n_occ)
        self.s_ops, self.d_ops = excitation_ops(self.space, n_occ)
        dim = self.H.shape[0]
        r = np.zeros(dim)
        r[self.ref] = 1.0
        self.r_vec = r
        self.e_ref = self.H[self.ref, self.ref].real
        # |mu> vectors (real, +-1 at one determinant)
        self.s_kets = np.einsum("iajk,k->iaj", self.s_ops, r)
        self.d_keys = list(self.d_ops.keys())
        self.d_kets = np.stack([self.d_ops[k] @ r for k in self.d_keys]) if self.d_keys else np.zeros((0, dim))

    def t_operator(self, t1: np.ndarray, t2: np.ndarray) -> np.ndarray:
        T = np.einsum("ia,iajk->jk", t1, self.s_ops).astype(np.complex128)
        for (i, j, a, b), m in self.d_ops.items():
            T = T + t2[i, j, a, b] * m
        return T

    @staticmethod
    def _exp_apply(T: np.ndarray, vec: np.ndarray, sign: float) -> np.ndarray:
        out = vec.astype(np.complex128)
        term = out.copy()
        for k in range(1, 64):
            term = sign * (T @ term) / k
            if not np.any(term):
                break
            out = out + term
        return out

    def transformed_ref(self, t1, t2, H=None) -> np.ndarray:
        """e^{-T} H e^{T} |R> as a determinant-space vector."""
        T = self.t_operator(t1, t2)
        H = self.H if H is None else H
        return self._exp_apply(T, H @ self._exp_apply(T, self.r_vec, +1.0), -1.0)

    def residual(self, t1, t2, H=None):
        """Omega_mu = <mu| e^{-T} H e^{T} |R> for singles (o,v) and doubles (full antisym)."""
        u = self.transformed_ref(t1, t2, H)
        o, v = self.o, self.v
        w1 = np.einsum("iaj,j->ia", self.s_kets, u)
        w2 = np.zeros((o, o, v, v), dtype=np.complex128)
        if self.d_keys:
            vals = self.d_kets @ u
            for (i, j, a, b), x in zip(self.d_keys, vals):
                w2[i, j, a, b] = x
                w2[j, i, a, b] = -x
                w2[i, j, b, a] = -x
                w2[j, i, b, a] = x
        return w1, w2

    def energy(self, t1, t2, H=None) -> complex:
        """Correlation energy <R| e^{-T} H e^{T} |R> - <R|H|R>."""
        u = self.transformed_ref(t1, t2, H)
        H = self.H if H is None else H
        return u[self.ref] - H[self.ref, self.ref]


def fci_response(fock, eri, n_occ, ops, zs):
    """Exact sum-over-states <<X_x;X_y>>_z for every z in zs: array [len(zs), nx, nx].

    The ground state is the lowest FCI root; X_0n = <0|X|n> with X = sum_pq X_pq a+_p a_q.
    """
    sp = Space(fock.shape[0], n_occ)
    H = hamiltonian(sp, fock, eri, n_occ)
    w, U = np.linalg.eigh(H)
    xs = [U.conj().T @ sp.one_body(x) @ U for x in ops]
    wn = w[1:] - w[0]
    out = np.zeros((len(zs), len(ops), len(ops)), dtype=np.complex128)
    for k, z in enumerate(zs):
        for a, xa in enumerate(xs):
            for b, xb in enumerate(xs):
                out[k, a, b] = -np.sum(xa[0, 1:] * xb[1:, 0] / (wn - z) + xb[0, 1:] * xa[1:, 0] / (wn + z))
    return out, w


def fci_energies(fock, eri, n_occ):
    sp = Space(fock.shape[0], n_occ)
    return np.linalg.eigvalsh(hamiltonian(sp, fock, eri, n_occ))

"""Ground-state CCSD: energy, residual and solver (oracle; test infrastructure only).

The paper solves the closed-shell ground state in a Kramers-unrestricted (spin-orbital) form and
defers the equations to the ExaCorr implementation paper (Sec. 3, step 1).  This restates the
published spin-orbital CCSD equations of Stanton, Gauss, Watts & Bartlett (J. Chem. Phys. 94, 4334
(1991)) for a general complex Hamiltonian: the Fock matrix may have off-diagonal and occupied-
virtual elements (needed for finite-field checks), and the bra/ket placement of every integral is
kept explicit, so nothing relies on real orbitals.  The residual is the projection
Omega_mu = <mu| e^{-T} H e^{T} |R> itself (no denominators folded in); it is pinned against the
determinant-space definition in oracle.det.

Notation: t1[i,a] = t_i^a, t2[i,j,a,b] = t_ij^ab (antisymmetric), I['ovvo'][m,b,e,j] = <mb||ej>.
"""
from __future__ import annotations
import numpy as np

es = lambda s, *a: np.einsum(s, *a, optimize=True)


def tau(t1, t2):
    """tau_ij^ab = t_ij^ab + t_i^a t_j^b - t_i^b t_j^a  (SI Eq. tau)."""
    return t2 + es("ia,jb->ijab", t1, t1) - es("ib,ja->ijab", t1, t1)


def tau_tilde(t1, t2):
    """Stanton-Gauss effective doubles with half the singles product."""
    return t2 + 0.5 * (es("ia,jb->ijab", t1, t1) - es("ib,ja->ijab", t1, t1))


def energy(I, t1, t2) -> complex:
    """E_corr = f_ia t_i^a + 1/4 <ij||ab> t_ij^ab + 1/2 <ij||ab> t_i^a t_j^b."""
    v = I["oovv"]
    return (es("ia,ia->", I.f_ov, t1) + 0.25 * es("ijab,ijab->", v, t2)
            + 0.5 * es("ijab,ia,jb->", v, t1, t1))


def intermediates(I, t1, t2):
    """Stanton-Gauss F and W intermediates (the full Fock diagonal is kept in F_ae, F_mi)."""
    tt = tau_tilde(t1, t2)
    ta = tau(t1, t2)
    Fae = (I.f_vv - 0.5 * es("me,ma->ae", I.f_ov, t1) + es("mf,mafe->ae", t1, I["ovvv"])
           - 0.5 * es("mnaf,mnef->ae", tt, I["oovv"]))
    Fmi = (I.f_oo + 0.5 * es("ie,me->mi", t1, I.f_ov) + es("ne,mnie->mi", t1, I["ooov"])
           + 0.5 * es("inef,mnef->mi", tt, I["oovv"]))
    Fme = I.f_ov + es("nf,mnef->me", t1, I["oovv"])
    x = es("je,mnie->mnij", t1, I["ooov"])
    Wmnij = I["oooo"] + x - x.transpose(0, 1, 3, 2) + 0.25 * es("ijef,mnef->mnij", ta, I["oovv"])
    y = es("mb,amef->abef", t1, I["vovv"])
    Wabef = I["vvvv"] - y + y.transpose(1, 0, 2, 3) + 0.25 * es("mnab,mnef->abef", ta, I["oovv"])
    Wmbej = (I["ovvo"] + es("jf,mbef->mbej", t1, I["ovvv"]) - es("nb,mnej->mbej", t1, I["oovo"])
             - es("jnfb,mnef->mbej", 0.5 * t2 + es("jf,nb->jnfb", t1, t1), I["oovv"]))
    return Fae, Fmi, Fme, Wmnij, Wabef, Wmbej


def _pij(x):
    return x - x.transpose(1, 0, 2, 3)


def _pab(x):
    return x - x.transpose(0, 1, 3, 2)


def residual(I, t1, t2):
    """Omega_1[i,a], Omega_2[i,j,a,b] for the CCSD amplitude equations."""
    Fae, Fmi, Fme, Wmnij, Wabef, Wmbej = intermediates(I, t1, t2)
    ta = tau(t1, t2)
    r1 = (I.f_vo.T + es("ie,ae->ia", t1, Fae) - es("ma,mi->ia", t1, Fmi) + es("imae,me->ia", t2, Fme)
          - es("nf,naif->ia", t1, I["ovov"]) - 0.5 * es("imef,maef->ia", t2, I["ovvv"])
          - 0.5 * es("mnae,nmei->ia", t2, I["oovo"]))
    r2 = I["vvoo"].transpose(2, 3, 0, 1).copy()
    r2 += _pab(es("ijae,be->ijab", t2, Fae - 0.5 * es("mb,me->be", t1, Fme)))
    r2 -= _pij(es("imab,mj->ijab", t2, Fmi + 0.5 * es("je,me->mj", t1, Fme)))
    r2 += 0.5 * es("mnab,mnij->ijab", ta, Wmnij)
    r2 += 0.5 * es("ijef,abef->ijab", ta, Wabef)
    r2 += _pij(_pab(es("imae,mbej->ijab", t2, Wmbej) - es("ie,ma,mbej->ijab", t1, t1, I["ovvo"])))
    r2 += _pij(es("ie,abej->ijab", t1, I["vvvo"]))
    r2 -= _pab(es("ma,mbij->ijab", t1, I["ovoo"]))
    return r1, r2


def denominators(I):
    """Orbital-energy differences D_ia = f_aa - f_ii, D_ijab = f_aa + f_bb - f_ii - f_jj."""
    eo = np.diag(I.f_oo).real
    ev = np.diag(I.f_vv).real
    d1 = ev[None, :] - eo[:, None]
    d2 = ev[None, None, :, None] + ev[None, None, None, :] - eo[:, None, None, None] - eo[None, :, None, None]
    return d1, d2


def solve(I, tol=1e-12, maxit=200, diis=8, verbose=False):
    """Jacobi iterations with DIIS on Omega(t) = 0, from t = 0 (the paper uses CROP; the converged
    amplitudes do not depend on the solver)."""
    o, v = I.o, I.v
    d1, d2 = denominators(I)
    t1 = np.zeros((o, v), dtype=np.complex128)
    t2 = np.zeros((o, o, v, v), dtype=np.complex128)
    vecs, errs = [], []
    for it in range(1, maxit + 1):
        r1, r2 = residual(I, t1, t2)
        norm = np.sqrt(np.vdot(r1, r1).real + 0.25 * np.vdot(r2, r2).real)
        if verbose:
            print(it, norm)
        if norm < tol:
            return t1, t2, energy(I, t1, t2), it
        t1 = t1 - r1 / d1
        t2 = t2 - r2 / d2
        vec = np.concatenate([t1.ravel(), t2.ravel()])
        err = np.concatenate([(r1 / d1).ravel(), (r2 / d2).ravel()])
        vecs.append(vec)
        errs.append(err)
        if len(vecs) > diis:
            vecs.pop(0)
            errs.pop(0)
        if len(vecs) >= 2:
            m = len(vecs)
            B = np.zeros((m + 1, m + 1), dtype=np.complex128)
            E = np.array(errs)
            B[:m, :m] = E.conj() @ E.T
            B[m, :m] = B[:m, m] = -1
            rhs = np.zeros(m + 1, dtype=np.complex128)
            rhs[m] = -1
            try:
                c = np.linalg.solve(B, rhs)[:m]
                vec = c @ np.array(vecs)
                t1 = vec[: o * v].reshape(o, v)
                t2 = vec[o * v:].reshape(o, o, v, v)
            except np.linalg.LinAlgError:
                pass
    raise RuntimeError(f"CCSD did not converge in {maxit} iterations (|Omega|={norm:.3e})")

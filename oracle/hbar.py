"""Similarity-transformed Hamiltonian intermediates (oracle; test infrastructure only).

SI, "EOM-EE sigma-vectors and intermediates", Eqs. F_im ... tau.  Every element is stored
creators-first: W[p,q,r,s] is the coefficient of {p+ q+ s r} in Hbar = e^{-T} H e^{T} (so
W^{pq}_{rs} in the paper's notation, upper = bra), and F[p,q] the coefficient of {p+ q}.
The printed equations carry undefined macros that scramble upper/lower placement; where the
printed placement does not contract consistently, the element below is the standard spin-orbital
one (Gauss & Stanton, J. Chem. Phys. 103, 3561 (1995)), and the derivative tests decide.

Readings against the printed list (each pinned by tests/test_oracle_sigma.py):
  * F_ae: printed "-f^m_a t^e_m" is read as -f_me t_m^a (the only placement that contracts);
  * W_iemn: the Fock term is read as -F_if t_mn^ef (printed with a + sign);
  * the vvvo element (W_efam / W_abei) is used in the standard form.
"""
from __future__ import annotations
import numpy as np
from .ccsd import tau

es = lambda s, *a: np.einsum(s, *a, optimize=True)


class Hbar:
    """One- and two-body elements of Hbar built once from t (SI step 2 of the paper's pipeline)."""

    def __init__(self, I, t1, t2):
        self.t1, self.t2 = t1, t2
        ta = tau(t1, t2)
        self.tau = ta
        oovv = I["oovv"]
        # one-body
        self.Fme = I.f_ov + es("nf,mnef->me", t1, oovv)                                   # Eq. F_me
        self.Fmi = (I.f_oo + es("ie,me->mi", t1, I.f_ov) + es("ne,mnie->mi", t1, I["ooov"])
                    + 0.5 * es("inef,mnef->mi", ta, oovv))                               # Eq. F_im
        self.Fae = (I.f_vv - es("ma,me->ae", t1, I.f_ov) + es("mf,amef->ae", t1, I["vovv"])
                    - 0.5 * es("mnaf,mnef->ae", ta, oovv))                               # Eq. F_ea
        # two-body
        x = es("je,mnie->mnij", t1, I["ooov"])
        self.Wmnij = I["oooo"] + x - x.transpose(0, 1, 3, 2) + 0.5 * es("ijef,mnef->mnij", ta, oovv)  # Eq. W_ijmn
        y = es("mb,amef->abef", t1, I["vovv"])
        self.Wabef = I["vvvv"] - y + y.transpose(1, 0, 2, 3) + 0.5 * es("mnab,mnef->abef", ta, oovv)  # Eq. W_efab
        self.Wmbej = (I["ovvo"] + es("jf,mbef->mbej", t1, I["ovvv"]) - es("nb,mnej->mbej", t1, I["oovo"])
                      - es("jnfb,mnef->mbej", t2 + es("jf,nb->jnfb", t1, t1), oovv))      # Eq. W_mbej
        self.Wmnie = I["ooov"] + es("if,mnfe->mnie", t1, oovv)                              # Eq. W_mnie
        self.Wamef = I["vovv"] - es("na,nmef->amef", t1, oovv)                              # Eq. W_amef
        # bar W_mbej = <mb||ej> - <mn||ef> t_nj^bf  (Eq. barW_mbej)
        Wbar = I["ovvo"] - es("mnef,njbf->mbej", oovv, t2)
        # hole three-index element W_mbij (Eq. W_iemn with m->i, b->e, i->m, j->n)
        z = es("mnie,jnbe->mbij", I["ooov"], t2)
        w = es("ie,mbej->mbij", t1, Wbar)
        self.Wmbij = (I["ovoo"] - es("me,ijbe->mbij", self.Fme, t2) - es("nb,mnij->mbij", t1, self.Wmnij)
                      + 0.5 * es("mbef,ijef->mbij", I["ovvv"], ta)
                      + z - z.transpose(0, 1, 3, 2) + w - w.transpose(0, 1, 3, 2))
        # particle three-index element W_abei (Eq. W_efam with e->a, f->b, a->e, m->i)
        u = es("mbef,miaf->abei", I["ovvv"], t2)
        q = es("ma,mbei->abei", t1, I["ovvo"] - es("mnef,nibf->mbei", oovv, t2))
        self.Wabei = (I["vvvo"] - es("me,miab->abei", self.Fme, t2) + es("if,abef->abei", t1, self.Wabef)
                      + 0.5 * es("mnei,mnab->abei", I["oovo"], ta)
                      - u + u.transpose(1, 0, 2, 3) - q + q.transpose(1, 0, 2, 3))


def g_intermediates(t2, l2):
    """G_ae = -1/2 t_mn^ef l_mn^af and G_mi = 1/2 t_mn^ef l_in^ef (Eqs. G_ea, G_mi)."""
    Gae = -0.5 * es("mnef,mnaf->ae", t2, l2)
    Gmi = 0.5 * es("mnef,inef->mi", t2, l2)
    return Gae, Gmi

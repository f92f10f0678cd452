"""Property vectors of CC linear response (oracle; test infrastructure only).

SI, "Linear response": xi^X (Eq. xi-equation and its programmable form), eta^X
(Eq. eta-equation), EOM eta^X (Faber & Coriani form) and the CC Hessian product (t^X F).
Index placement is read creators-first as in oracle.hbar: X[p,q] = <p|X|q>, so X^a_i -> X[a,i],
V^{pq}_{rs} -> I['....'][p,q,r,s], W^{pq}_{rs} -> the Hbar element of that class, t^{ab}_{ij} ->
t2[i,j,a,b], lambda^{ij}_{ab} -> l2[i,j,a,b].  Two Hbar elements of the (t^X F) singles carry a
particle-hole ordering that the stored W_mbej covers by antisymmetry:
W^{ie}_{mc} = -W_mbej[i,e,c,m] and W^{ek}_{am} = -W_mbej[k,e,a,m].
"""
from __future__ import annotations
import numpy as np

es = lambda s, *a: np.einsum(s, *a, optimize=True)


def _pij(x):
    return x - x.transpose(1, 0, 2, 3)


def _pab(x):
    return x - x.transpose(0, 1, 3, 2)


def xi(X, o, t1, t2):
    """xi^X singles [i,a] and doubles [i,j,a,b]."""
    Xoo, Xov, Xvo, Xvv = X[:o, :o], X[:o, o:], X[o:, :o], X[o:, o:]
    s1 = (Xvo.T + es("ae,ie->ia", Xvv, t1) - es("mi,ma->ia", Xoo, t1)
          - es("me,ie,ma->ia", Xov, t1, t1) + es("me,imae->ia", Xov, t2))
    s2 = _pab(es("bf,ijaf->ijab", Xvv, t2))
    s2 -= _pij(es("mj,imab->ijab", Xoo, t2))
    s2 -= _pij(es("mi,mjab->ijab", es("me,ie->mi", Xov, t1), t2))
    s2 -= _pab(es("fa,ijfb->ijab", es("mf,ma->fa", Xov, t1), t2))
    return s1, s2


def eta(X, o, t1, t2, l1, l2):
    """eta^X singles [i,a] and doubles [i,j,a,b]."""
    Xoo, Xov, Xvo, Xvv = X[:o, :o], X[:o, o:], X[o:, :o], X[o:, o:]
    s1 = (Xov + es("ea,ie->ia", Xvv, l1) - es("im,ma->ia", Xoo, l1)
          - es("ma,me,ie->ia", Xov, t1, l1) - es("ie,me,ma->ia", Xov, t1, l1)
          - 0.5 * es("ni,na->ia", es("mnfe,mife->ni", t2, l2), Xov)
          - 0.5 * es("ea,ie->ia", es("nmfe,nmfa->ea", t2, l2), Xov))
    s2 = _pij(_pab(es("ia,jb->ijab", l1, Xov)))
    s2 += _pab(es("ijae,eb->ijab", l2, Xvv))
    s2 -= _pij(es("imab,jm->ijab", l2, Xoo))
    s2 -= _pab(es("ijam,mb->ijab", es("me,ijae->ijam", t1, l2), Xov))
    s2 -= _pij(es("me,imab,je->ijab", t1, l2, Xov))
    return s1, s2


def eta_eom(X, o, t1, t2, l1, l2):
    """EOM eta^X: eta^X with lambda^{ij}_{ab} xi^X_jb added to the singles."""
    e1, e2 = eta(X, o, t1, t2, l1, l2)
    x1, _ = xi(X, o, t1, t2)
    return e1 + es("ijab,jb->ia", l2, x1), e2


def hessian_product(H, I, l1, l2, u1, u2):
    """(u F): singles [k,c] and doubles [k,l,c,d] for a response vector u = (u1, u2)."""
    t2 = H.t2
    oovv = I["oovv"]
    Fme, Wamef, Wmnie, Wmnij, Wabef, Wmbej = H.Fme, H.Wamef, H.Wmnie, H.Wmnij, H.Wabef, H.Wmbej
    W_iemc = -Wmbej.transpose(0, 1, 3, 2)          # W^{ie}_{mc}[i,e,m,c] = -W_mbej[i,e,c,m]
    W_ekam = -Wmbej.transpose(1, 0, 2, 3)          # W^{ek}_{am}[e,k,a,m] = -W_mbej[k,e,a,m]
    s = es("kica,ia->kc", oovv, u1)
    s -= es("ic,ka,ia->kc", l1, Fme, u1)
    s -= es("ka,ic,ia->kc", l1, Fme, u1)
    s += es("ke,eica,ia->kc", l1, Wamef, u1)
    s -= es("mc,kima,ia->kc", l1, Wmnie, u1)
    s -= es("ma,ikmc,ia->kc", l1, Wmnie, u1)
    s += es("ie,ekac,ia->kc", l1, Wamef, u1)
    s -= 0.5 * es("ic,kjab,ijab->kc", l1, oovv, u2)
    s -= 0.5 * es("ka,ijcb,ijab->kc", l1, oovv, u2)
    s += es("ia,jkbc,ijab->kc", l1, oovv, u2)
    s -= es("mkae,iemc,ia->kc", l2, W_iemc, u1)
    s -= es("imec,ekam,ia->kc", l2, W_ekam, u1)
    s += 0.5 * es("kief,efca,ia->kc", l2, Wabef, u1)
    s += 0.5 * es("mnca,kimn,ia->kc", l2, Wmnij, u1)
    s -= 0.5 * es("fc,kifa,ia->kc", es("mnec,mnef->fc", l2, t2), oovv, u1)
    s -= 0.5 * es("kn,nica,ia->kc", es("mkef,mnef->kn", l2, t2), oovv, u1)
    s -= 0.5 * es("fa,ikfc,ia->kc", es("mnea,mnef->fa", l2, t2), oovv, u1)
    s -= 0.5 * es("in,nkac,ia->kc", es("mief,mnef->in", l2, t2), oovv, u1)
    s -= 0.5 * es("ijac,kb,ijab->kc", l2, Fme, u2)
    s -= 0.5 * es("ikab,jc,ijab->kc", l2, Fme, u2)
    s -= es("ikeb,ejac,ijab->kc", l2, Wamef, u2)
    s += es("mjac,ikmb,ijab->kc", l2, Wmnie, u2)
    s -= 0.25 * es("ijec,ekab,ijab->kc", l2, Wamef, u2)
    s += 0.25 * es("mkab,ijmc,ijab->kc", l2, Wmnie, u2)
    s += 0.5 * es("ijae,ekbc,ijab->kc", l2, Wamef, u2)
    s -= 0.5 * es("imab,jkmc,ijab->kc", l2, Wmnie, u2)

    d = _pab(_pij(es("kc,lida,ia->klcd", l1, oovv, u1)))
    d -= _pij(es("ka,ilcd,ia->klcd", l1, oovv, u1))
    d -= _pab(es("ic,klad,ia->klcd", l1, oovv, u1))
    d -= _pij(es("kicd,la,ia->klcd", l2, Fme, u1))
    d -= _pab(es("klca,id,ia->klcd", l2, Fme, u1))
    d += _pab(es("klce,eida,ia->klcd", l2, Wamef, u1))
    d -= _pij(es("kmcd,lima,ia->klcd", l2, Wmnie, u1))
    d += _pab(_pij(es("mlca,kimd,ia->klcd", l2, Wmnie, u1)))
    d += es("micd,klma,ia->klcd", l2, Wmnie, u1)
    d -= _pab(_pij(es("kied,elca,ia->klcd", l2, Wamef, u1)))
    d -= es("klea,eicd,ia->klcd", l2, Wamef, u1)
    d -= 0.5 * _pab(es("klca,ijdb,ijab->klcd", l2, oovv, u2))
    d -= 0.5 * _pij(es("kicd,ljab,ijab->klcd", l2, oovv, u2))
    d += 0.25 * es("ijcd,klab,ijab->klcd", l2, oovv, u2)
    d += 0.25 * es("klab,ijcd,ijab->klcd", l2, oovv, u2)
    d += _pij(_pab(es("kjcb,lida,ijab->klcd", l2, oovv, u2)))
    d -= 0.5 * _pij(es("ikab,jlcd,ijab->klcd", l2, oovv, u2))
    d -= 0.5 * _pab(es("ijac,klbd,ijab->klcd", l2, oovv, u2))
    return s, d

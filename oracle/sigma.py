"""Right and left EOM-EE sigma vectors (oracle; test infrastructure only).

Right:  sigma = A r        SI Eqs. sigma_sin-ee and sigma_double-ee
Left:   sigma = l A        SI Eqs. sigma_sin-ee-left and sigma_double-ee-left
with A_{mu nu} = <mu| [Hbar, tau_nu] |R> = dOmega_mu/dt_nu (Sec. 2.3 and its table).  Terms follow
the printed order; index placement is read creators-first (see oracle.hbar).  Readings:
  * right singles, 4th term: W_maei r_m^e (the element whose annihilator e and creator m
    contract with r_m^e);
  * left doubles: "-l_ma W_ijmb" is read with the P(ab) antisymmetrizer and "l_ie V_ejab" as
    l_ie W_ejab (the Hbar element), as required by dOmega/dt (tests/test_oracle_sigma.py).
"""
from __future__ import annotations
import numpy as np
from .hbar import g_intermediates

es = lambda s, *a: np.einsum(s, *a, optimize=True)


def _pij(x):
    return x - x.transpose(1, 0, 2, 3)


def _pab(x):
    return x - x.transpose(0, 1, 3, 2)


def sigma_right(H, I, r1, r2):
    """(A r): singles [i,a] and doubles [i,j,a,b] for a trial vector (r1, r2)."""
    t2 = H.t2
    s1 = (es("ae,ie->ia", H.Fae, r1) - es("mi,ma->ia", H.Fmi, r1) + es("me,imae->ia", H.Fme, r2)
          + es("maei,me->ia", H.Wmbej, r1) + 0.5 * es("amef,imef->ia", H.Wamef, r2)
          + 0.5 * es("mnie,mnea->ia", H.Wmnie, r2))
    s2 = -_pab(es("mbij,ma->ijab", H.Wmbij, r1))
    s2 += _pij(es("abej,ie->ijab", H.Wabei, r1))
    s2 += _pab(es("bf,ijaf->ijab", es("bmfe,me->bf", H.Wamef, r1), t2))
    s2 -= _pij(es("nj,inab->ijab", es("nmje,me->nj", H.Wmnie, r1), t2))
    s2 += _pab(es("be,ijae->ijab", H.Fae, r2))
    s2 -= _pij(es("mj,imab->ijab", H.Fmi, r2))
    s2 += 0.5 * es("mnij,mnab->ijab", H.Wmnij, r2)
    s2 += _pij(_pab(es("mbej,imae->ijab", H.Wmbej, r2)))
    s2 -= 0.5 * _pab(es("af,ijfb->ijab", es("nmfe,mnea->af", I["oovv"], r2), t2))
    s2 -= 0.5 * _pij(es("ni,jnba->ijab", es("nmfe,imfe->ni", I["oovv"], r2), t2))
    s2 += 0.5 * es("abef,ijef->ijab", H.Wabef, r2)
    return s1, s2


def sigma_left(H, I, l1, l2):
    """(l A): singles [i,a] and doubles [i,j,a,b] for a left vector (l1, l2)."""
    Gae, Gmi = g_intermediates(H.t2, l2)
    s1 = (es("ie,ea->ia", l1, H.Fae) - es("ma,im->ia", l1, H.Fmi)
          + 0.5 * es("imef,efam->ia", l2, H.Wabei) - 0.5 * es("mnae,iemn->ia", l2, H.Wmbij)
          - es("ef,eifa->ia", Gae, H.Wamef) - es("mn,mina->ia", Gmi, H.Wmnie)
          + es("me,ieam->ia", l1, H.Wmbej))
    s2 = _pab(es("ijae,eb->ijab", l2, H.Fae))
    s2 -= _pij(es("imab,jm->ijab", l2, H.Fmi))
    s2 += 0.5 * es("mnab,ijmn->ijab", l2, H.Wmnij)
    s2 += _pij(_pab(es("imae,jebm->ijab", l2, H.Wmbej)))
    s2 += _pab(es("ijae,be->ijab", I["oovv"], Gae))
    s2 -= _pab(es("ma,ijmb->ijab", l1, H.Wmnie))
    s2 -= _pij(es("imab,mj->ijab", I["oovv"], Gmi))
    s2 += _pij(es("ie,ejab->ijab", l1, H.Wamef))
    s2 += _pij(_pab(es("ia,jb->ijab", l1, H.Fme)))
    s2 += 0.5 * es("ijef,efab->ijab", l2, H.Wabef)
    return s1, s2

"""Derivative definitions of A, xi, eta and F (oracle; test infrastructure only).

The CCSD residual Omega(t) = <mu|e^{-T} H e^{T}|R> is a polynomial of degree 4 in t and contains no
complex conjugates, so every quantity of the response table in Sec. 2.3 is an exact derivative:
  A r         = d/ds Omega(t + s r)                        (degree 4: 5-point stencil, exact)
  xi^X        = Omega(t; f -> X, V -> 0)                   (Omega is linear in the Hamiltonian)
  eta^X . r   = d/ds [E_X + lambda.Omega_X](t + s r)       (degree 2: central difference, exact)
  l A . r     = d/ds lambda.Omega(t + s r)  with lambda -> l
  r F w       = d^2/da db [E + lambda.Omega](t + a r + b w) (degree 4: Richardson-combined
                                                          4-point mixed stencil, exact)
where E_X, Omega_X use the property operator X as the one-body Hamiltonian and no two-body part,
and eta (ground state) = dE/dt.  Only rounding separates these from the closed forms.
"""
from __future__ import annotations
import numpy as np
from . import ccsd
from .ints import Ints


# ---- excitation-vector helpers (unique elements i<j, a<b) -------------------------------------

def antisym(x):
    return x - x.transpose(1, 0, 2, 3) - x.transpose(0, 1, 3, 2) + x.transpose(1, 0, 3, 2)


def unique_index(o, v):
    i, j = np.triu_indices(o, 1)
    a, b = np.triu_indices(v, 1)
    return i, j, a, b


def pack(t1, t2):
    o, v = t1.shape
    i, j, a, b = unique_index(o, v)
    return np.concatenate([t1.ravel(), t2[i[:, None], j[:, None], a[None, :], b[None, :]].ravel()])


def unpack(vec, o, v):
    i, j, a, b = unique_index(o, v)
    t1 = vec[: o * v].reshape(o, v).astype(np.complex128)
    d = vec[o * v:].reshape(len(i), len(a))
    t2 = np.zeros((o, o, v, v), dtype=np.complex128)
    I_, J_, A_, B_ = i[:, None], j[:, None], a[None, :], b[None, :]
    t2[I_, J_, A_, B_] = d
    t2[J_, I_, A_, B_] = -d
    t2[I_, J_, B_, A_] = -d
    t2[J_, I_, B_, A_] = d
    return t1, t2


def dot(x1, x2, y1, y2):
    """Bilinear product over unique excitations: sum_ia x y + 1/4 sum_ijab x y."""
    return np.sum(x1 * y1) + 0.25 * np.sum(x2 * y2)


def property_ints(I, X):
    """Integral set with f -> X and no two-electron part (for xi^X, eta^X)."""
    zero = {k: np.zeros_like(b) for k, b in I._b.items() if k in ("oooo", "ooov", "oovv", "ovov", "ovvv", "vvvv")}
    return Ints(X, zero, I.o)


# ---- stencils ------------------------------------------------------------------------------

def jacobian_right(I, t1, t2, r1, r2, s=None):
    """A r by the 5-point stencil along r."""
    if s is None:
        s = 0.25 * max(1e-3, np.sqrt(dot(t1.conj(), t2.conj(), t1, t2).real + 1.0)) / max(
            1e-300, np.sqrt(dot(r1.conj(), r2.conj(), r1, r2).real))
    vals = {}
    for k in (-2, -1, 1, 2):
        vals[k] = ccsd.residual(I, t1 + k * s * r1, t2 + k * s * r2)
    out = []
    for c in range(2):
        out.append((vals[-2][c] - 8 * vals[-1][c] + 8 * vals[1][c] - vals[2][c]) / (12 * s))
    return out[0], out[1]


def jacobian_dense(I, t1, t2):
    """Dense A over unique excitations, column by column (tiny systems only)."""
    o, v = t1.shape
    n = o * v + len(unique_index(o, v)[0]) * len(unique_index(o, v)[2])
    A = np.zeros((n, n), dtype=np.complex128)
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1.0
        r1, r2 = unpack(e, o, v)
        A[:, k] = pack(*jacobian_right(I, t1, t2, r1, r2, s=0.5))
    return A


def xi(I, t1, t2, X):
    """xi^X_mu = <mu| e^{-T} X e^{T} |R>."""
    return ccsd.residual(property_ints(I, X), t1, t2)


def lagrangian(I, t1, t2, l1, l2):
    """E(t) + lambda . Omega(t)."""
    w1, w2 = ccsd.residual(I, t1, t2)
    return ccsd.energy(I, t1, t2) + dot(l1, l2, w1, w2)


def eta_dot(I, t1, t2, l1, l2, X, r1, r2, s=0.5):
    """eta^X . r (quadratic in s: the central difference is exact)."""
    P = property_ints(I, X)
    f = lambda k: lagrangian(P, t1 + k * r1, t2 + k * r2, l1, l2)
    return (f(s) - f(-s)) / (2 * s)


def left_dot(I, t1, t2, l1, l2, r1, r2):
    """(l A) . r = l . (A r)."""
    a1, a2 = jacobian_right(I, t1, t2, r1, r2)
    return dot(l1, l2, a1, a2)


def eta_ground(I, t1, t2):
    """dE/dt over unique elements: (F_me, <ij||ab>) (E is quadratic in t)."""
    e1 = I.f_ov + np.einsum("mnef,nf->me", I["oovv"], t1)
    return e1, I["oovv"].copy()


def hessian_dot(I, t1, t2, l1, l2, u1, u2, w1, w2, h=0.25):
    """u F w = d^2 L / da db with L = E + lambda.Omega at t + a u + b w."""
    def m(hh):
        L = lambda a, b: lagrangian(I, t1 + a * u1 + b * w1, t2 + a * u2 + b * w2, l1, l2)
        return (L(hh, hh) - L(hh, -hh) - L(-hh, hh) + L(-hh, -hh)) / (4 * hh * hh)
    return (4 * m(h) - m(2 * h)) / 3

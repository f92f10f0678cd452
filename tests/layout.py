"""Amplitude-layout conversion for tests: full (t1[i,a], t2[i,j,a,b]) <-> the C ABI's vector
[t1 | t2 over P(i<j), P(a<b)] with P(p,q) = q(q-1)/2 + p.  Layout only, no method arithmetic."""
import numpy as np
import synth


def to_amp(t1, t2):
    o, v = t1.shape
    p, q = synth.pair_table(o)
    a, b = synth.pair_table(v)
    d = t2[p[:, None], q[:, None], a[None, :], b[None, :]]
    return np.concatenate([t1.ravel(), d.ravel()]).astype(np.complex128)


def from_amp(vec, o, v):
    p, q = synth.pair_table(o)
    a, b = synth.pair_table(v)
    t1 = vec[: o * v].reshape(o, v).copy()
    d = vec[o * v:].reshape(len(p), len(a))
    t2 = np.zeros((o, o, v, v), np.complex128)
    P, Q, A, B = p[:, None], q[:, None], a[None, :], b[None, :]
    t2[P, Q, A, B] = d
    t2[Q, P, A, B] = -d
    t2[P, Q, B, A] = -d
    t2[Q, P, B, A] = d
    return t1, t2


def rel(a, b):
    """max |a - b| / max |b|"""
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(1e-300, np.abs(np.asarray(b)).max()))

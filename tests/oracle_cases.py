"""Small seeded cases shared by the oracle tests (inputs only)."""
import numpy as np
import synth
from oracle.ints import Ints
from oracle.deriv import antisym


def general_case(o=3, v=5, seed=7, sd=0.1, fock_sd=0.2):
    """Non-canonical complex Fock (off-diagonal and occupied-virtual elements) and integrals."""
    inst = synth.make_instance(o, v, seed=seed, sd=sd)
    F = inst.fock + synth.random_hermitian(o + v, seed, 55, fock_sd)
    return inst, F, Ints.from_instance(inst, fock=F)


def rand_amp(o, v, stream, scale=0.3, seed=1):
    t1 = synth.random_vector((o, v), seed, stream, scale)
    t2 = antisym(synth.random_vector((o, o, v, v), seed, stream + 1, scale))
    return t1, t2

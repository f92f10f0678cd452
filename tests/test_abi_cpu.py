"""The C ABI library loads and exports every entry point its header declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "cclr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b((?:cc|cclr)_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_problem_statement_calls():
    names = header_functions()
    for must in ("cc_ground", "cc_lambda", "cc_lr_solve", "cc_response_function", "cclr_set_hamiltonian",
                 "cclr_sigma", "cclr_create", "cclr_destroy", "cclr_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2307_14296_b300 as pk
    lib = ctypes.CDLL(pk.library_path())
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pk.EXPORTS) <= set(header_functions())


def test_default_options_and_errors_without_device():
    import paper_2307_14296_b300 as pk
    o = pk.default_options()
    assert o.tol == 1e-8 and o.maxit == 100 and o.precision == pk.FP64
    # a bad device index is an argument error, not a crash
    h = ctypes.c_void_p()
    st = pk._lib.cclr_create(ctypes.byref(h), 9999, ctypes.byref(o))
    assert st == pk.CCLR_E_ARG and not h
    assert pk._lib.cclr_last_error(None) == b"null context"
    assert pk._lib.cc_ground(None, None, None) == pk.CCLR_E_ARG


def test_layout_roundtrip():
    import numpy as np
    import synth
    from layout import to_amp, from_amp
    from oracle.deriv import antisym
    t1 = synth.random_vector((3, 5), 1, 1)
    t2 = antisym(synth.random_vector((3, 3, 5, 5), 1, 2))
    a, b = from_amp(to_amp(t1, t2), 3, 5)
    assert np.abs(a - t1).max() == 0 and np.abs(b - t2).max() < 1e-14


def test_noalloc_wrapper_rejects_bad_tensors_before_any_gpu_work():
    """cclr_zgemm_nt_noalloc's argument checks run on the host: a wrong dtype, a non-contiguous
    view, a host tensor or mismatched shapes raise ValueError without reaching the library."""
    import torch
    import paper_2307_14296_b300 as pk

    class Fake:   # stands in for a CUDA tensor (attributes only; no GPU here)
        def __init__(self, shape, dtype=torch.complex128, contiguous=True):
            self.shape, self.dtype, self._c, self.is_cuda = tuple(shape), dtype, contiguous, True

        def is_contiguous(self):
            return self._c

        def dim(self):
            return len(self.shape)

    good = dict(A=Fake((8, 5)), B=Fake((6, 5)), C=Fake((8, 6)))
    cases = [
        dict(good, A=torch.zeros((8, 5), dtype=torch.complex128)),   # host tensor
        dict(good, B=Fake((6, 5), dtype=torch.complex64)),            # wrong dtype
        dict(good, C=Fake((8, 6), contiguous=False)),                 # non-contiguous
        dict(good, B=Fake((6, 4))),                                   # K mismatch
        dict(good, C=Fake((8, 5))),                                   # short C
        dict(good, A=Fake((8, 5, 1))),                                # not a matrix
    ]
    for cs in cases:
        with pytest.raises(ValueError):
            pk.cclr_zgemm_nt_noalloc(cs["A"], cs["B"], cs["C"])


def test_header_is_plain_c_and_links_against_the_library(tmp_path):
    """include/cclr.h compiles as C99 without warnings, and a C program that takes the address of
    every declared entry point links against the built library (no call is made)."""
    import shutil
    import subprocess
    import paper_2307_14296_b300 as pk
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = header_functions()
    src = tmp_path / "abi.c"
    src.write_text('#include "cclr.h"\n#include <stdio.h>\nint main(void) {\n  const void *f[] = {'
                   + ", ".join("(const void *)&" + n for n in names) + "};\n"
                   "  printf(\"%d\\n\", (int)(sizeof f / sizeof f[0]));\n  return CCLR_FP32_TC == CCLR_TC_BF16X6 ? 0 : 1;\n}\n")
    lib = pk.library_path()
    out = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-Wno-pedantic", "-I", os.path.join(ROOT, "include"),
                          str(src), lib, "-Wl,-rpath," + os.path.dirname(lib), "-o", str(tmp_path / "abi")],
                         capture_output=True, text=True)
    assert out.returncode == 0, out.stderr

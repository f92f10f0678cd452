"""The host eigensolver of the EOM-EE subspace problems (csrc/zeig.h: Householder reduction to
Hessenberg form, shifted complex QR, back-substitution for the eigenvectors), checked on the CPU
against NumPy's LAPACK eigenvalues and against the eigen-equation itself, on random complex
matrices, a defective-free matrix with a known spectrum, a triangular one and a 1 x 1 case."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2307_14296_b300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("zeig") / "zeig_harness")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "zeig_harness.cpp"), "-o", exe],
                   check=True)
    return exe


def run(exe, A):
    n = A.shape[0]
    text = f"{n}\n" + "\n".join(f"{z.real:.17g} {z.imag:.17g}" for z in A.ravel()) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    w = np.array([complex(float(a), float(b)) for a, b in (line.split() for line in out[:n])])
    res, nrm = (float(x) for x in out[n].split())
    return w, res, nrm


def match(w, ref):
    """largest distance from each reference eigenvalue to the closest computed one"""
    return max(np.min(np.abs(w - r)) for r in ref)


@pytest.mark.parametrize("n", [2, 5, 16, 40, 96])
def test_random_complex_matrices(harness, n):
    rng = np.random.default_rng(2307 + n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    w, res, nrm = run(harness, A)
    ref = np.linalg.eigvals(A)
    scale = np.abs(A).max()
    assert match(w, ref) < 1e-10 * scale * n
    assert res < 1e-11 * n
    assert nrm < 1e-12


def test_known_spectrum_nonnormal(harness):
    """S diag(d) S^-1 with a non-unitary S: the eigenvalues are d (the EOM matrices are
    non-Hermitian with near-degenerate clusters, as here)."""
    rng = np.random.default_rng(7)
    n = 24
    d = np.concatenate([0.7 + 0.01 * np.arange(12), 1.5 + 1e-3 * np.arange(12)]) + 1e-4j * rng.standard_normal(n)
    S = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    A = S @ np.diag(d) @ np.linalg.inv(S)
    w, res, _ = run(harness, A)
    assert match(w, d) < 1e-9
    assert res < 1e-10


def test_triangular_and_scalar(harness):
    rng = np.random.default_rng(3)
    U = np.triu(rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)))
    w, res, _ = run(harness, U)
    assert match(w, np.diag(U)) < 1e-12 * np.abs(U).max()
    assert res < 1e-12
    w1, res1, _ = run(harness, np.array([[2.5 - 0.5j]]))
    assert abs(w1[0] - (2.5 - 0.5j)) < 1e-15 and res1 == 0.0

"""B300-native relativistic CCSD linear response (arXiv 2307.14296), Python binding of libcclr.

Thin ctypes layer over the C ABI in include/cclr.h: it converts numpy arrays (host) or torch CUDA
tensors (device) into pointers and sizes and turns status codes into exceptions.  Every step of
the computation runs in the CUDA library; there is no Python or CPU fallback, and importing this
package fails if libcclr.so has not been built (python paper_2307_14296_b300/build.py).

Vector layout ("amplitude layout"): [singles t_i^a at i*v + a | doubles t_ij^ab at
P(i,j)*Pv + P(a,b)] with P(p,q) = q*(q-1)/2 + p for p < q; unique elements only.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcclr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libcclr.so is missing: build the CUDA library with `python paper_2307_14296_b300/build.py` "
        "(there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

CCLR_OK, CCLR_E_ARG, CCLR_E_NOCONV, CCLR_E_OOM, CCLR_E_CUDA, CCLR_E_STATE, CCLR_E_TIMEOUT = range(7)
FP64, TC_BF16X3, TC_BF16X6, TC_F64 = 0, 2, 3, 4
TC_FP32 = TC_BF16X6   # the FP32-class tensor-core mode
AMP_T, AMP_LAMBDA = 0, 1
EXPORTS = (
    "cclr_default_options", "cclr_create", "cclr_destroy", "cclr_last_error", "cclr_set_hamiltonian",
    "cc_ground", "cc_lambda", "cc_lr_solve", "cc_response_function", "cc_response_function_ci", "cc_response_function_asym",
    "cclr_field_derivative", "cclr_export_amplitudes", "cc_eom_ee",
    "cclr_get_eom_vector",
    "cclr_get_amplitudes",
    "cclr_set_amplitudes", "cclr_get_response_vector", "cclr_sigma", "cclr_residual", "cclr_xi",
    "cclr_eta", "cclr_hessian", "cclr_zgemm_nt", "cclr_kernel_profile", "cclr_get_stats",
    "cclr_zgemm_nt_noalloc", "cclr_kernel_breakdown", "cclr_bench_vector_kernels", "cclr_gram",
    "cclr_debug_expire_next_wait", "cclr_autotune_report", "cclr_response_batch", "cclr_response_gradient",
    "cclr_eta_ground", "cclr_left_solve", "cclr_set_synthetic",
)


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("ground_tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("max_subspace", ctypes.c_int), ("precision", ctypes.c_int), ("batch", ctypes.c_int),
                ("refine", ctypes.c_int), ("refine_tol", ctypes.c_double), ("autotune", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("sigma_calls", ctypes.c_long), ("sigma_vectors", ctypes.c_long),
                ("sigma_seconds", ctypes.c_double), ("total_seconds", ctypes.c_double),
                ("kernel_launches", ctypes.c_long), ("max_residual", ctypes.c_double),
                ("refine_vectors", ctypes.c_long), ("refine_seconds", ctypes.c_double)]


_vp, _i, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_sig = {
    "cclr_default_options": (None, [ctypes.POINTER(Options)]),
    "cclr_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(Options)]),
    "cclr_destroy": (None, [_vp]),
    "cclr_last_error": (ctypes.c_char_p, [_vp]),
    "cclr_set_hamiltonian": (_i, [_vp, _i, _i, _vp, ctypes.POINTER(_vp)]),
    "cc_ground": (_i, [_vp, _vp, ctypes.POINTER(_i)]),
    "cc_lambda": (_i, [_vp, ctypes.POINTER(_i)]),
    "cc_lr_solve": (_i, [_vp, _i, _vp, _i, _vp, _d, _vp]),
    "cc_response_function": (_i, [_vp, _vp]),
    "cc_response_function_ci": (_i, [_vp, _vp]),
    "cc_response_function_asym": (_i, [_vp, _vp]),
    "cclr_field_derivative": (_i, [_vp, _vp, _vp]),
    "cclr_export_amplitudes": (_i, [_vp, _i, _i, _vp, _sz]),
    "cc_eom_ee": (_i, [_vp, _i, _vp, _vp]),
    "cclr_get_eom_vector": (_i, [_vp, _i, _vp, ctypes.c_size_t]),
    "cclr_get_amplitudes": (_i, [_vp, _i, _vp, _sz]),
    "cclr_set_amplitudes": (_i, [_vp, _i, _vp, _sz]),
    "cclr_get_response_vector": (_i, [_vp, _i, _i, _i, _vp, _sz]),
    "cclr_sigma": (_i, [_vp, _i, _i, _vp, _vp, _i, _i]),
    "cclr_residual": (_i, [_vp, _vp, _vp]),
    "cclr_xi": (_i, [_vp, _vp, _vp]),
    "cclr_eta": (_i, [_vp, _vp, _i, _vp]),
    "cclr_hessian": (_i, [_vp, _i, _vp, _vp, _i]),
    "cclr_zgemm_nt": (_i, [_vp, _i, _i, _i, _i, _vp, _vp, _vp]),
    "cclr_kernel_profile": (_i, [_vp, _i, _vp]),
    "cclr_kernel_breakdown": (_i, [_vp, ctypes.c_char_p, _i]),
    "cclr_zgemm_nt_noalloc": (_i, [_i, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "cclr_get_stats": (_i, [_vp, ctypes.POINTER(Stats)]),
    "cclr_bench_vector_kernels": (_i, [_vp, _i, ctypes.c_int64, _i, _i, _i, _i, _vp]),
    "cclr_gram": (_i, [_vp, _i, ctypes.c_int64, _i, _i, _vp, _vp, _vp]),
    "cclr_debug_expire_next_wait": (_i, [_vp, ctypes.c_uint]),
    "cclr_autotune_report": (_i, [_vp, ctypes.c_char_p, _i]),
    "cclr_response_gradient": (_i, [_vp, _i, _vp]),
    "cclr_eta_ground": (_i, [_vp, _vp]),
    "cclr_set_synthetic": (_i, [_vp, _i, _i, ctypes.c_uint64, _d, _d, _i, _vp]),
    "cclr_left_solve": (_i, [_vp, _i, _vp, _d, _d, _vp]),
    "cclr_response_batch": (_i, [ctypes.POINTER(_vp), _i, _i, ctypes.POINTER(_vp), _i, _vp, _d, ctypes.POINTER(_vp),
                                 _vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class CCLRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libcclr status {status}: {msg}")
        self.status = status


def default_options(**kw) -> Options:
    o = Options()
    _lib.cclr_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def _in(x):
    """(pointer, keep-alive) for an input array: a contiguous complex128 CUDA tensor is passed as
    its device pointer after the stream that produced it has finished; anything else as a host
    complex128 array."""
    if _is_torch_cuda(x):
        import torch
        if x.dtype != torch.complex128 or not x.is_contiguous():
            raise ValueError("device arrays must be contiguous complex128 tensors")
        torch.cuda.current_stream(x.device).synchronize()
        return _vp(x.data_ptr()), x
    a = _c128(x)
    return _ptr(a), a


def _out(shape, like=None, out=None):
    """Output array: `out` if given (host or CUDA), else a CUDA tensor on `like`'s device when
    `like` is a CUDA tensor, else a host array."""
    if out is None:
        if _is_torch_cuda(like):
            import torch
            out = torch.empty(shape, dtype=torch.complex128, device=like.device)
        else:
            out = np.zeros(shape, np.complex128)
    if _is_torch_cuda(out):
        import torch
        if out.dtype != torch.complex128 or not out.is_contiguous() or tuple(out.shape) != tuple(shape):
            raise ValueError(f"output must be a contiguous complex128 tensor of shape {tuple(shape)}")
        torch.cuda.current_stream(out.device).synchronize()
        return _vp(out.data_ptr()), out
    if not (isinstance(out, np.ndarray) and out.dtype == np.complex128 and out.flags.c_contiguous
            and out.shape == tuple(shape)):
        raise ValueError(f"output must be a C-contiguous complex128 array of shape {tuple(shape)}")
    return _ptr(out), out


class Context:
    """One libcclr context (device memory, stream, Hamiltonian, amplitudes, response data)."""

    def __init__(self, device: int = 0, **options):
        self._h = _vp()
        self.options = default_options(**options)
        st = _lib.cclr_create(ctypes.byref(self._h), device, ctypes.byref(self.options))
        if st != CCLR_OK:
            raise CCLRError(st, "cclr_create failed (no CUDA device?)")
        self.n_occ = self.n_vir = 0

    def close(self):
        if self._h:
            _lib.cclr_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != CCLR_OK:
            raise CCLRError(st, _lib.cclr_last_error(self._h).decode())

    @property
    def N(self) -> int:
        o, v = self.n_occ, self.n_vir
        return o * v + (o * (o - 1) // 2) * (v * (v - 1) // 2)

    # ---- problem statement
    def cclr_set_hamiltonian(self, n_occ, n_vir, fock, blocks):
        """fock (n x n) and the six packed integral classes (oooo, ooov, oovv, ovov, ovvv, vvvv)."""
        fock = _c128(fock)
        bl = [_c128(b) for b in blocks]
        arr = (_vp * 6)(*[b.ctypes.data for b in bl])
        self._check(_lib.cclr_set_hamiltonian(self._h, n_occ, n_vir, _ptr(fock), arr))
        self.n_occ, self.n_vir = n_occ, n_vir

    def cclr_set_synthetic(self, n_occ, n_vir, seed, sd, dip_sd=0.1, n_ops=3):
        """Generate the counter-based synthetic instance on the device and install it (see
        cclr_set_synthetic in cclr.h); returns the operators (n_ops, n, n) as a host array."""
        n = n_occ + n_vir
        ops = np.zeros((n_ops, n, n), np.complex128)
        self._check(_lib.cclr_set_synthetic(self._h, int(n_occ), int(n_vir), int(seed), float(sd), float(dip_sd),
                                            int(n_ops), _ptr(ops) if n_ops else _vp()))
        self.n_occ, self.n_vir = n_occ, n_vir
        return ops

    def cc_ground(self):
        e = np.zeros(1, np.complex128)
        it = _i()
        self._check(_lib.cc_ground(self._h, _ptr(e), ctypes.byref(it)))
        return complex(e[0]), it.value

    def cc_lambda(self):
        it = _i()
        self._check(_lib.cc_lambda(self._h, ctypes.byref(it)))
        return it.value

    def cc_lr_solve(self, ops, omegas, gamma):
        """ops: (n_ops, n, n) host array or complex128 CUDA tensor."""
        p, ops = _in(ops)
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        its = np.zeros(ops.shape[0] * om.size, np.int32)
        self._check(_lib.cc_lr_solve(self._h, ops.shape[0], p, om.size, _ptr(om), float(gamma), _ptr(its)))
        self._nops, self._nfreq, self._norb = ops.shape[0], om.size, ops.shape[-1]
        self.lr_serial = getattr(self, "lr_serial", 0) + 1
        return its.reshape(ops.shape[0], om.size)

    def cc_response_function(self):
        out = np.zeros((self._nfreq, self._nops, self._nops), np.complex128)
        self._check(_lib.cc_response_function(self._h, _ptr(out)))
        return out

    def cclr_response_gradient(self, f: int, out=None, like=None):
        """Operator gradient of the response function at frequency index f: G[k][s] (n_ops, 4, n, n)
        with d<<X_x;X_y>> = sum G[y,0] dX_x + conj(sum G[y,1] dX_x) + sum G[x,3] dX_y
        + conj(sum G[x,2] dX_y).  Written to `out` (host or CUDA), else to a new array on `like`'s
        device."""
        n = self.n_occ + self.n_vir
        p, out = _out((self._nops, 4, n, n), like, out)
        self._check(_lib.cclr_response_gradient(self._h, int(f), p))
        return out

    def cclr_eta_ground(self, out=None, like=None):
        """dE/dt at the current T (the right-hand side of the Lambda equations)."""
        p, out = _out((self.N,), like, out)
        self._check(_lib.cclr_eta_ground(self._h, p))
        return out

    def cclr_left_solve(self, rhs, w=0.0, out=None):
        """l (A + w) = -b for each row b of rhs ([nrhs, N] or [N]; host or CUDA)."""
        p, b = _in(rhs)
        nrhs = b.shape[0] if b.ndim == 2 else 1
        po, out = _out(tuple(b.shape), b, out)
        self._check(_lib.cclr_left_solve(self._h, nrhs, p, float(complex(w).real), float(complex(w).imag), po))
        return out

    def cc_response_function_ci(self):
        """The CC-CI form (no Hessian term) from the same solutions."""
        out = np.zeros((self._nfreq, self._nops, self._nops), np.complex128)
        self._check(_lib.cc_response_function_ci(self._h, _ptr(out)))
        return out

    def cc_response_function_asym(self):
        """The asymmetric CC-CC form (first-order multipliers from left solves) from the same
        solutions."""
        out = np.zeros((self._nfreq, self._nops, self._nops), np.complex128)
        self._check(_lib.cc_response_function_asym(self._h, _ptr(out)))
        return out

    def cclr_export_amplitudes(self, which, idx=0):
        """T (which 0), Lambda (1) or the response solution idx = (k n_freq + f) 4 + s (2)."""
        out = np.zeros(self.N, np.complex128)
        self._check(_lib.cclr_export_amplitudes(self._h, int(which), int(idx), _ptr(out), out.size))
        return out

    def cclr_field_derivative(self, V):
        """d<<X_x;X_y>>/d eps [n_freq, n_ops, n_ops] for the field eps V on the Fock matrix (V: n x n,
        host or CUDA); d alpha / d eps is its negative."""
        p, keep = _in(V)
        norb = getattr(self, "_norb", None)   # None before cc_lr_solve: the library reports the state
        if norb is not None and tuple(keep.shape) != (norb, norb):
            raise ValueError("V must be an n x n matrix of the operators' size")
        nf, no = getattr(self, "_nfreq", 0), getattr(self, "_nops", 0)
        out = np.zeros((nf, no, no), np.complex128)
        self._check(_lib.cclr_field_derivative(self._h, p, _ptr(out)))
        return out

    def cc_eom_ee(self, n_roots):
        """Lowest n_roots EOM-CCSD excitation energies (complex, ordered by real part) and the
        iteration count."""
        w = np.zeros(n_roots, np.complex128)
        it = _i()
        self._check(_lib.cc_eom_ee(self._h, int(n_roots), _ptr(w), ctypes.byref(it)))
        return w, it.value

    def cclr_get_eom_vector(self, root):
        out = np.zeros(self.N, np.complex128)
        self._check(_lib.cclr_get_eom_vector(self._h, int(root), _ptr(out), out.size))
        return out

    # ---- components
    def cclr_get_amplitudes(self, which=AMP_T, out=None, like=None):
        p, out = _out((self.N,), like, out)
        self._check(_lib.cclr_get_amplitudes(self._h, which, p, self.N))
        return out

    def cclr_set_amplitudes(self, which, vec):
        """vec: host array or complex128 CUDA tensor (amplitude layout)."""
        p, vec = _in(vec)
        n = vec.numel() if _is_torch_cuda(vec) else vec.size
        self._check(_lib.cclr_set_amplitudes(self._h, which, p, n))

    def cclr_get_response_vector(self, k, f, s):
        out = np.zeros(self.N, np.complex128)
        self._check(_lib.cclr_get_response_vector(self._h, k, f, s, _ptr(out), out.size))
        return out

    def cclr_sigma(self, vecs, side=0, precision=FP64, out=None):
        """Right (side 0) or left (side 1) sigma of a batch [nvec, N] (numpy or torch CUDA)."""
        if _is_torch_cuda(vecs):
            import torch
            assert vecs.dtype == torch.complex128 and vecs.is_contiguous()
            nvec = vecs.shape[0] if vecs.dim() == 2 else 1
            if out is None:
                out = torch.empty_like(vecs)
            self._check(_lib.cclr_sigma(self._h, side, nvec, _vp(vecs.data_ptr()), _vp(out.data_ptr()), 1, precision))
            return out
        v = _c128(vecs)
        nvec = v.shape[0] if v.ndim == 2 else 1
        res = np.zeros_like(v)
        self._check(_lib.cclr_sigma(self._h, side, nvec, _ptr(v), _ptr(res), 0, precision))
        return res

    def cclr_residual(self, out=None, like=None):
        """(Omega(T), E_corr); Omega written to `out` (host or CUDA) or a new array on `like`'s device."""
        p, out = _out((self.N,), like, out)
        e = np.zeros(1, np.complex128)
        self._check(_lib.cclr_residual(self._h, p, _ptr(e)))
        return out, complex(e[0])

    def cclr_xi(self, op):
        op = _c128(op)
        out = np.zeros(self.N, np.complex128)
        self._check(_lib.cclr_xi(self._h, _ptr(op), _ptr(out)))
        return out

    def cclr_eta(self, op, eom=False):
        op = _c128(op)
        out = np.zeros(self.N, np.complex128)
        self._check(_lib.cclr_eta(self._h, _ptr(op), int(eom), _ptr(out)))
        return out

    def cclr_hessian(self, vecs):
        if _is_torch_cuda(vecs):
            import torch
            nvec = vecs.shape[0] if vecs.dim() == 2 else 1
            out = torch.empty_like(vecs)
            self._check(_lib.cclr_hessian(self._h, nvec, _vp(vecs.data_ptr()), _vp(out.data_ptr()), 1))
            return out
        v = _c128(vecs)
        nvec = v.shape[0] if v.ndim == 2 else 1
        res = np.zeros_like(v)
        self._check(_lib.cclr_hessian(self._h, nvec, _ptr(v), _ptr(res), 0))
        return res

    def cclr_zgemm_nt(self, A, B, precision=FP64):
        """C = A B^T for complex A (M x K) and B (N x K) through the contraction engine."""
        A, B = _c128(A), _c128(B)
        C = np.zeros((A.shape[0], B.shape[0]), np.complex128)
        self._check(_lib.cclr_zgemm_nt(self._h, precision, A.shape[0], B.shape[0], A.shape[1], _ptr(A), _ptr(B), _ptr(C)))
        return C

    def cclr_gram(self, X, Y, mirror=False):
        """X^H Y (nx x ny) by the solver's FP32-arithmetic Gram kernel, from FP64 rows or from FP32
        mirrors of them."""
        X, Y = _c128(X), _c128(Y)
        out = np.zeros((X.shape[0], Y.shape[0]), np.complex128)
        self._check(_lib.cclr_gram(self._h, int(bool(mirror)), X.shape[1], X.shape[0], Y.shape[0], _ptr(X), _ptr(Y),
                                   _ptr(out)))
        return out

    def cclr_bench_vector_kernels(self, n, nx, ny, m, reps=5, precision=TC_BF16X3) -> dict:
        """Milliseconds per call of the solver's Gram block (nx x ny), residual-norm pass and
        correction pass (m outputs from nx rows) on synthetic device vectors of length n."""
        out = np.zeros(3, np.float64)
        self._check(_lib.cclr_bench_vector_kernels(self._h, precision, int(n), nx, ny, m, reps, _ptr(out)))
        return dict(gram_ms=float(out[0]), norms_ms=float(out[1]), write_ms=float(out[2]))

    def cclr_kernel_profile(self, enable=True) -> dict:
        """Tensor-core kernel timing (CUDA events on the library's stream) since the last call: the
        split-BF16 kernel's launches, ms, executed and useful flops, and under "f64" the same for
        the FP64-class kernel."""
        out = np.zeros(8, np.float64)
        self._check(_lib.cclr_kernel_profile(self._h, int(enable), _ptr(out)))
        d = lambda k: dict(launches=int(out[4 * k]), ms=float(out[4 * k + 1]), flops_exec=float(out[4 * k + 2]),
                           flops_useful=float(out[4 * k + 3]))
        return dict(d(0), f64=d(1))

    def cclr_kernel_breakdown(self) -> dict:
        """Per-kernel {name: (launches, milliseconds)} since the last call (timing switched on by
        cclr_kernel_profile)."""
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(_lib.cclr_kernel_breakdown(self._h, buf, len(buf)))
        out = {}
        for line in buf.value.decode().splitlines():
            name, n, ms = line.rsplit(" ", 2)
            out[name] = (int(n), float(ms))
        return out

    def cclr_debug_expire_next_wait(self, polls: int):
        """Make the next split-BF16 GEMM launch of this context wait first for a barrier phase that
        nothing completes, with `polls` polls per wait (test of the CCLR_E_TIMEOUT path)."""
        self._check(_lib.cclr_debug_expire_next_wait(self._h, int(polls)))

    def cclr_autotune_report(self) -> dict:
        """{shape key: (tile rows, stages, ms of the 128-row tile, ms of the 64-row tile)} decided so far."""
        buf = ctypes.create_string_buffer(1 << 20)
        self._check(_lib.cclr_autotune_report(self._h, buf, len(buf)))
        out = {}
        for line in buf.value.decode().splitlines():
            k, bn, st, m0, m1 = line.split()
            out[k] = (int(bn), int(st), float(m0), float(m1))
        return out

    def cclr_get_stats(self) -> dict:
        s = Stats()
        self._check(_lib.cclr_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}


# module-level names of the C ABI's problem-statement calls
def cclr_create(device=0, **options) -> Context:
    return Context(device, **options)


def cclr_set_hamiltonian(ctx, n_occ, n_vir, fock, blocks):
    return ctx.cclr_set_hamiltonian(n_occ, n_vir, fock, blocks)


def cc_ground(ctx):
    return ctx.cc_ground()


def cc_lambda(ctx):
    return ctx.cc_lambda()


def cc_lr_solve(ctx, ops, omegas, gamma):
    return ctx.cc_lr_solve(ops, omegas, gamma)


def cc_response_function(ctx):
    return ctx.cc_response_function()


def cc_response_function_ci(ctx):
    return ctx.cc_response_function_ci()


def cc_response_function_asym(ctx):
    return ctx.cc_response_function_asym()


def cc_eom_ee(ctx, n_roots):
    return ctx.cc_eom_ee(n_roots)


def _check_noalloc_operands(A, B, C):
    """Argument checks of cclr_zgemm_nt_noalloc, all before any GPU work: complex128 CUDA tensors,
    contiguous, 2-D, A: M x K, B: N x K, C: M x N, on the current device.  Raises ValueError."""
    import torch
    for name, t in (("A", A), ("B", B), ("C", C)):
        if not _is_torch_cuda(t):
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.complex128:
            raise ValueError(f"{name} must be complex128, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.dim() != 2:
            raise ValueError(f"{name} must be a matrix")
    M, K = A.shape
    if tuple(B.shape)[1] != K:
        raise ValueError(f"B has {tuple(B.shape)[1]} columns, A has {K}")
    if tuple(C.shape) != (M, B.shape[0]):
        raise ValueError(f"C must be {M} x {B.shape[0]}, not {tuple(C.shape)[0]} x {tuple(C.shape)[1]}")
    dev = torch.cuda.current_device()
    for name, t in (("A", A), ("B", B), ("C", C)):
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")


def cclr_zgemm_nt_noalloc(A, B, C, precision=TC_BF16X3, stream=None) -> int:
    """C = A B^T on the tensor cores without any device allocation (torch CUDA complex128 tensors,
    contiguous, on the current device; C is written).  For callers that cannot allocate device
    memory; the library keeps its temporaries in one fixed 64 MiB device array shared by all
    calls, so overlapping calls race.  The call synchronizes the stream before it returns.
    Returns the C-ABI status code (0 = success); bad tensors raise ValueError before any GPU work."""
    _check_noalloc_operands(A, B, C)
    M, K = A.shape
    N = B.shape[0]
    s = _vp(stream.cuda_stream) if stream is not None else _vp()
    return _lib.cclr_zgemm_nt_noalloc(precision, M, N, K, _vp(A.data_ptr()), _vp(B.data_ptr()), _vp(C.data_ptr()), s)


def cclr_response_batch(contexts, ops, omegas, gamma):
    """Several systems (contexts with their Hamiltonians set) solved as one batch, one host thread
    per system so that their kernels overlap on the GPU: the response function of each system
    (list of [n_freq, n_ops, n_ops] arrays).  ops: one [n_ops, n, n] array per system."""
    n = len(contexts)
    ops = [_c128(o) for o in ops]
    n_ops = ops[0].shape[0]
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    outs = [np.zeros((om.size, n_ops, n_ops), np.complex128) for _ in range(n)]
    st = np.zeros(n, np.int32)
    h = (_vp * n)(*[c._h for c in contexts])
    po = (_vp * n)(*[o.ctypes.data for o in ops])
    pout = (_vp * n)(*[o.ctypes.data for o in outs])
    r = _lib.cclr_response_batch(h, n, n_ops, po, om.size, _ptr(om), float(gamma), pout, _ptr(st))
    if r != CCLR_OK:
        bad = int(np.flatnonzero(st)[0])
        raise CCLRError(int(st[bad]), f"system {bad}: " + _lib.cclr_last_error(contexts[bad]._h).decode())
    for c in contexts:
        c._nops, c._nfreq = n_ops, om.size
    return outs


def library_path() -> str:
    return LIB_PATH

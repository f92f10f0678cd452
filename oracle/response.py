"""Lambda equations, damped linear-response solves and the response function (oracle).

TEST INFRASTRUCTURE ONLY.

  * Lambda:        lambda A = -eta  (Sec. 2.3, Eq. for t-bar^(0)), eta = dE/dt;
  * response:      (A - z) t^Y(z) = -xi^Y, z = w + i gamma  (Eqs. LR response equation and
                   LR response equation_cpp);
  * Davidson:      the SI "Davidson scheme" steps 1-5, with the readings
                   G' = b^H (sigma - z b), C' = -b^H xi, r = (sigma - z b) beta + xi,
                   correction = -(D - z)^{-1} r with D the orbital-energy differences,
                   modified Gram-Schmidt against the trial space, convergence on ||r||_2;
  * response fn:   <<X;Y>>_z = f(z) + conj(f(-conj z)),
                   f(z) = 1/2 [eta^X t^Y(z) + eta^Y t^X(-z) + (t^X(-z) F) t^Y(z)]
                   (Eq. CC-CC response function with C^{+-w} and P(X,Y) written out; the
                   conjugation flips the real frequency and keeps the damping, which is the
                   reading that reproduces the exact sum over states);
  * asymmetric form: f(z) = 1/2 [eta^X t^Y(z) + t-bar^Y(z) xi^X], symmetrized the same way, with
                   the first-order multipliers t-bar^Y(z) (A + z) = -(eta^Y + F t^Y(z)) from left
                   sigma products (Sec. 2.3, the asymmetric CC-CC form; the printed form omits the
                   C^{+-w} symmetrizer, which the stated equality with the symmetric form needs);
  * static-field derivative d<<X;Y>>_z / d eps for H + eps V on the Fock matrix: the response
                   function above differentiated by the chain rule (field_derivative);
  * polarizability alpha_xy(z) = -<<mu_x; mu_y>>_z, mean alpha, anisotropy, and the absorption
    cross section sigma(w) = 4 pi w / c Im mean-alpha (Eq. abs_cpp; Sec. 5 definitions).
All products in the response function are bilinear (no conjugation) over unique excitations.
"""
from __future__ import annotations
import numpy as np
from . import ccsd, hbar, sigma, props
from .deriv import pack, unpack, dot

C_AU = 137.035999084


class CCSystem:
    """Ground state, Hbar and Lambda for one Hamiltonian (the paper's pipeline steps 1-2)."""

    def __init__(self, I, tol=1e-12, t=None, lam=None):
        self.I, self.o, self.v = I, I.o, I.v
        if t is None:
            t1, t2, e, it = ccsd.solve(I, tol=tol)
            self.ground_iters = it
        else:
            t1, t2 = t
            e = ccsd.energy(I, t1, t2)
        self.t1, self.t2, self.e_corr = t1, t2, e
        self.H = hbar.Hbar(I, t1, t2)
        d1, d2 = ccsd.denominators(I)
        self.D = pack(d1.astype(np.complex128), d2.astype(np.complex128))
        if lam is None:
            lam = self.solve_lambda(tol=tol)
        self.l1, self.l2 = lam

    # -- products on packed unique-element vectors
    def sigma_r(self, vec):
        r1, r2 = unpack(vec, self.o, self.v)
        return pack(*sigma.sigma_right(self.H, self.I, r1, r2))

    def sigma_l(self, vec):
        l1, l2 = unpack(vec, self.o, self.v)
        return pack(*sigma.sigma_left(self.H, self.I, l1, l2))

    def xi(self, X):
        return pack(*props.xi(X, self.o, self.t1, self.t2))

    def eta(self, X):
        return pack(*props.eta(X, self.o, self.t1, self.t2, self.l1, self.l2))

    def eta_eom(self, X):
        return pack(*props.eta_eom(X, self.o, self.t1, self.t2, self.l1, self.l2))

    def hessian(self, u):
        u1, u2 = unpack(u, self.o, self.v)
        return pack(*props.hessian_product(self.H, self.I, self.l1, self.l2, u1, u2))

    def bdot(self, x, y):
        """Bilinear product over unique excitations (packed vectors carry unique elements)."""
        return np.sum(x * y)

    def eta_ground(self):
        I = self.I
        e1 = I.f_ov + np.einsum("mnef,nf->me", I["oovv"], self.t1)
        return pack(e1, I["oovv"])

    def solve_lambda(self, tol=1e-12, maxit=200, diis=8):
        """lambda A = -eta by Jacobi iterations on eta + lambda A with DIIS."""
        eta = self.eta_ground()
        lam = -eta / self.D
        vecs, errs = [], []
        for it in range(maxit):
            res = eta + self.sigma_l(lam)
            if np.linalg.norm(res) < tol:
                self.lambda_iters = it
                return unpack(lam, self.o, self.v)
            lam = lam - res / self.D
            vecs.append(lam)
            errs.append(res / self.D)
            if len(vecs) > diis:
                vecs.pop(0)
                errs.pop(0)
            if len(vecs) >= 2:
                m = len(vecs)
                E = np.array(errs)
                B = np.zeros((m + 1, m + 1), dtype=np.complex128)
                B[:m, :m] = E.conj() @ E.T
                B[m, :m] = B[:m, m] = -1
                rhs = np.zeros(m + 1, dtype=np.complex128)
                rhs[m] = -1
                lam = np.linalg.solve(B, rhs)[:m] @ np.array(vecs)
        raise RuntimeError("Lambda equations did not converge")

    # -- dense references (tiny systems)
    def eom_energies(self, nroots, A=None):
        """Lowest EOM-CCSD excitation energies: the eigenvalues of the CC Jacobian A (SI "EOM-EE
        sigma-vectors and intermediates"), smallest real part first, from the dense A (tiny
        systems only)."""
        A = self.dense_A() if A is None else A
        w = np.linalg.eigvals(A)
        return w[np.argsort(w.real, kind="stable")][:nroots]

    def dense_A(self):
        n = self.D.size
        A = np.zeros((n, n), dtype=np.complex128)
        for k in range(n):
            e = np.zeros(n, dtype=np.complex128)
            e[k] = 1.0
            A[:, k] = self.sigma_r(e)
        return A

    # -- response solves
    def solve_dense(self, A, xi, z):
        return -np.linalg.solve(A - z * np.eye(A.shape[0]), xi)

    def davidson(self, xi, z, tol=1e-10, maxit=200, start="pivot", op=None):
        """Davidson solve of (A - z) t = -xi (SI Davidson scheme, steps 1-5).  With op =
        self.sigma_l (v -> v A, i.e. A^T v) it solves the left system t (A - z) = -xi instead."""
        op = self.sigma_r if op is None else op
        D = self.D
        if start == "pivot":
            b0 = np.zeros_like(xi)
            b0[np.argmax(np.abs(xi))] = 1.0
        else:
            b0 = -xi / (D - z)
        B = [b0 / np.linalg.norm(b0)]
        S = [op(B[0])]
        for it in range(1, maxit + 1):
            Bm, Sm = np.array(B), np.array(S)
            G = Bm.conj() @ (Sm - z * Bm).T
            C = -(Bm.conj() @ xi)
            beta = np.linalg.solve(G, C)
            t = beta @ Bm
            r = beta @ (Sm - z * Bm) + xi
            rn = np.linalg.norm(r)
            if rn < tol:
                return t, it, rn
            c = -r / (D - z)
            for _ in range(2):
                for b in B:
                    c = c - np.vdot(b, c) * b
            cn = np.linalg.norm(c)
            if cn < 1e-14:
                return t, it, rn
            B.append(c / cn)
            S.append(op(B[-1]))
        raise RuntimeError(f"Davidson did not converge (|r|={rn:.3e})")

    def response(self, ops, zs, solver="davidson", tol=1e-11, A=None, half=False, form="cc"):
        """<<X_a; X_b>>_z for all pairs (a, b) and all z: array [len(zs), nops, nops].

        form="cc": the CC-CC response function (Sec. 2.3, Eq. CC-CC response function),
            f(z) = 1/2 [eta^a t^b(z) + eta^b t^a(-z) + (t^a(-z) F) t^b(z)].
        form="ci": the CC-CI response function (Eq. CC-CI response function; EOM-eta of the SI
            "Linear response" section, no Hessian term),
            f(z) = 1/2 [eometa^a t^b(z) - (lam.t^a(-z))(lam.xi^b)
                        + eometa^b t^a(-z) - (lam.t^b(z))(lam.xi^a)],
            lam the ground-state multipliers; P swaps (a, -z) with (b, z).
        form="asym": the asymmetric CC-CC form (Sec. 2.3),
            f(z) = 1/2 [eta^a t^b(z) + tbar^b(z) xi^a],  tbar^b(z) (A + z) = -(eta^b + F t^b(z)),
            which needs solves for operator b only (right and left).
        All three are symmetrized as f(z) + conj(f(-z*)).  With half=True return the unsymmetrized
        f(z) instead (2 f(0) of the CC-CC form is the second derivative of the CC energy with
        respect to static fields).
        """
        assert form in ("cc", "ci", "asym")
        nops = len(ops)
        eta = [self.eta_eom(X) if form == "ci" else self.eta(X) for X in ops]
        xis = [self.xi(X) for X in ops]
        lam = pack(self.l1, self.l2)
        lam_xi = [self.bdot(lam, x) for x in xis]
        cache = {}

        def t_of(k, w):
            key = (k, complex(w))
            if key not in cache:
                if solver == "dense":
                    cache[key] = self.solve_dense(A, xis[k], w)
                else:
                    cache[key] = self.davidson(xis[k], w, tol=tol)[0]
            return cache[key]

        def tbar_of(k, w):
            """First-order multipliers: tbar (A + w) = -(eta^k + F t^k(w))."""
            key = ("left", k, complex(w))
            if key not in cache:
                rhs = eta[k] + self.hessian(t_of(k, w))
                if solver == "dense":
                    cache[key] = -np.linalg.solve(A.T + w * np.eye(A.shape[0]), rhs)
                else:
                    cache[key] = self.davidson(rhs, -w, tol=tol, op=self.sigma_l)[0]
            return cache[key]

        def f(z, a, b):
            if form == "asym":
                return 0.5 * (self.bdot(eta[a], t_of(b, z)) + self.bdot(tbar_of(b, z), xis[a]))
            tx = t_of(a, -z)
            ty = t_of(b, z)
            if form == "ci":
                return 0.5 * (self.bdot(eta[a], ty) - self.bdot(lam, tx) * lam_xi[b]
                              + self.bdot(eta[b], tx) - self.bdot(lam, ty) * lam_xi[a])
            return 0.5 * (self.bdot(eta[a], ty) + self.bdot(eta[b], tx) + self.bdot(self.hessian(tx), ty))

        out = np.zeros((len(zs), nops, nops), dtype=np.complex128)
        for k, z in enumerate(zs):
            for a in range(nops):
                for b in range(nops):
                    out[k, a, b] = f(z, a, b) if half else f(z, a, b) + np.conj(f(-np.conj(z), a, b))
        return out


    # -- static-field derivative of the response function
    def at(self, t=None, lam=None):
        """The same Hamiltonian at other amplitudes and/or multipliers (packed vectors; default the
        converged ones): Hbar rebuilt at t, nothing solved."""
        t = pack(self.t1, self.t2) if t is None else t
        lam = pack(self.l1, self.l2) if lam is None else lam
        return CCSystem(self.I, t=unpack(t, self.o, self.v), lam=unpack(lam, self.o, self.v))

    def field_derivative(self, ops, V, zs, solver="dense", tol=1e-12, A=None):
        """d<<X_a; X_b>>_z / d eps for the field H + eps V (V added to the Fock matrix, orbitals
        unrelaxed), operators fixed: array [len(zs), nops, nops], symmetrized as f'(z) +
        conj(f'(-z*)).  The CC-CC response function (Sec. 2.3) differentiated by the chain rule
        through the ground amplitudes, the multipliers and the response amplitudes; the
        derivatives of the response amplitudes are eliminated with the first-order multipliers
        tbar^k(w) (A + w) = -(eta^k + F t^k(w)):
          f'(w) = 1/2 [eta^a' t^b + eta^b' t^a + t^a F' t^b
                       + tbar^a(-w) (A' t^b + xi^b') + tbar^b(w) (A' t^a + xi^a')],
          t^b = t^b(w), t^a = t^a(-w).
        The field enters as Omega + eps xi^V(t) and E + eps <HF|e^-T V e^T|HF>, so
          t^V = d t0/d eps = -A^-1 xi^V,   lam^V A = -(eta^V + F t^V),
          A' u = D^2 Omega[t^V, u] + D xi^V[u],   xi^k' = D xi^k[t^V],
          eta^k' = D_t eta^k[t^V] + eta^k(lam^V) - eta^k(lam = 0),
          F' u = D_t (F u)[t^V] + F(lam^V) u - F(lam = 0) u + D_t eta^V[u],
        D the directional derivative in the amplitudes.  Every differentiated quantity is a
        polynomial in the amplitudes of degree <= 3 (sigma, Omega), 2 (xi, F) or 1 (eta), so the
        five-point stencil used here is exact up to rounding; eta and F are linear in lambda."""
        nops = len(ops)
        n = self.D.size
        t0 = pack(self.t1, self.t2)
        if solver == "dense" and A is None:
            A = self.dense_A()
        eye = np.eye(n)

        def solve_r(rhs, w):     # (A - w) t = -rhs
            if solver == "dense":
                return -np.linalg.solve(A - w * eye, rhs)
            return self.davidson(rhs, w, tol=tol)[0]

        def solve_l(rhs, w):     # tbar (A + w) = -rhs
            if solver == "dense":
                return -np.linalg.solve(A.T + w * eye, rhs)
            return self.davidson(rhs, -w, tol=tol, op=self.sigma_l)[0]

        def ddir(g, u):
            """d/ds g(t0 + s u) at s = 0 for g a polynomial of degree <= 4 in s (exact stencil)."""
            h = 0.05 / max(np.abs(u).max(), 1e-300)
            vals = {s: g(self.at(t=t0 + s * h * u)) for s in (-2, -1, 1, 2)}
            return (vals[-2] - 8 * vals[-1] + 8 * vals[1] - vals[2]) / (12 * h)

        tV = solve_r(self.xi(V), 0.0)
        lamV = solve_l(self.eta(V) + self.hessian(tV), 0.0)
        sys_l, sys_0 = self.at(lam=lamV), self.at(lam=np.zeros(n, dtype=np.complex128))
        shifted = {s: self.at(t=t0 + s * (0.05 / max(np.abs(tV).max(), 1e-300)) * tV) for s in (-2, -1, 1, 2)}
        hV = 0.05 / max(np.abs(tV).max(), 1e-300)

        def along_tV(g):         # D_t g[t^V] from the four shifted systems
            return (g(shifted[-2]) - 8 * g(shifted[-1]) + 8 * g(shifted[1]) - g(shifted[2])) / (12 * hV)

        eta_p = [along_tV(lambda S, X=X: S.eta(X)) + sys_l.eta(X) - sys_0.eta(X) for X in ops]
        xi_p = [along_tV(lambda S, X=X: S.xi(X)) for X in ops]
        eta = [self.eta(X) for X in ops]
        cache = {}

        def t_of(k, w):
            key = ("r", k, complex(w))
            if key not in cache:
                cache[key] = solve_r(self.xi(ops[k]), w)
            return cache[key]

        def tbar_of(k, w):
            key = ("l", k, complex(w))
            if key not in cache:
                cache[key] = solve_l(eta[k] + self.hessian(t_of(k, w)), w)
            return cache[key]

        def a_prime(u):          # A' u
            return along_tV(lambda S: S.sigma_r(u)) + ddir(lambda S: S.xi(V), u)

        def f_prime(w, a, b):
            tb, ta = t_of(b, w), t_of(a, -w)
            Fp_tb = (along_tV(lambda S: S.hessian(tb)) + sys_l.hessian(tb) - sys_0.hessian(tb)
                     + ddir(lambda S: S.eta(V), tb))
            return 0.5 * (self.bdot(eta_p[a], tb) + self.bdot(eta_p[b], ta) + self.bdot(ta, Fp_tb)
                          + self.bdot(tbar_of(a, -w), a_prime(tb) + xi_p[b])
                          + self.bdot(tbar_of(b, w), a_prime(ta) + xi_p[a]))

        out = np.zeros((len(zs), nops, nops), dtype=np.complex128)
        for k, z in enumerate(zs):
            for a in range(nops):
                for b in range(nops):
                    out[k, a, b] = f_prime(z, a, b) + np.conj(f_prime(-np.conj(z), a, b))
        return out


def polarizability(resp):
    """alpha_xy = -<<mu_x; mu_y>>."""
    return -resp


def mean_alpha(alpha):
    """Isotropic mean (alpha_xx + alpha_yy + alpha_zz)/3 (Sec. 5.2)."""
    return np.trace(alpha, axis1=-2, axis2=-1) / 3.0


def anisotropy(alpha):
    """Delta alpha = alpha_zz - (alpha_xx + alpha_yy)/2 (Sec. 5.2)."""
    return alpha[..., 2, 2] - 0.5 * (alpha[..., 0, 0] + alpha[..., 1, 1])


def cross_section(omega, alpha):
    """sigma(w) = 4 pi w / c Im mean-alpha(w) (Eq. abs_cpp, atomic units)."""
    return 4.0 * np.pi * np.asarray(omega) / C_AU * np.imag(mean_alpha(alpha))

// Eigenvalues and right eigenvectors of a small general complex matrix, on the host, for the
// subspace problems of the EOM-EE Davidson solver.  Textbook algorithm (Golub & Van Loan,
// Matrix Computations, Ch. 7): Householder reduction to upper Hessenberg form, the single-shift
// complex QR iteration with Wilkinson shifts and deflation to the complex Schur form
// A = Z T Z^H, and eigenvectors of the triangular T by back substitution, mapped back with Z.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace cclr {

// A: n x n row-major (overwritten).  On return w[k] are the eigenvalues and column k of V
// (row-major n x n, V[i*n + k]) the unit-norm right eigenvector of w[k].  Returns false if the
// QR iteration did not converge within 60 n sweeps.
inline bool zgeev_small(int n, std::vector<std::complex<double>>& A, std::vector<std::complex<double>>& w,
                        std::vector<std::complex<double>>& V) {
  typedef std::complex<double> zc;
  auto a = [&](int i, int j) -> zc& { return A[(size_t)i * n + j]; };
  std::vector<zc> Z((size_t)n * n, zc(0));
  auto z = [&](int i, int j) -> zc& { return Z[(size_t)i * n + j]; };
  for (int i = 0; i < n; ++i) z(i, i) = 1.0;
  // ---- Householder reduction to Hessenberg form: A <- P A P, Z <- Z P
  for (int k = 0; k + 2 < n; ++k) {
    double alpha2 = 0.0;
    for (int i = k + 1; i < n; ++i) alpha2 += std::norm(a(i, k));
    const double alpha = std::sqrt(alpha2);
    if (alpha == 0.0) continue;
    const zc x0 = a(k + 1, k);
    const zc phase = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : zc(1.0);
    std::vector<zc> v(n, zc(0));
    v[k + 1] = x0 + phase * alpha;
    for (int i = k + 2; i < n; ++i) v[i] = a(i, k);
    double vn2 = 0.0;
    for (int i = k + 1; i < n; ++i) vn2 += std::norm(v[i]);
    if (vn2 == 0.0) continue;
    const double beta = 2.0 / vn2;   // P = I - beta v v^H
    for (int j = 0; j < n; ++j) {   // A <- P A
      zc s(0);
      for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * a(i, j);
      s *= beta;
      for (int i = k + 1; i < n; ++i) a(i, j) -= v[i] * s;
    }
    for (int i = 0; i < n; ++i) {   // A <- A P, Z <- Z P
      zc s(0), t(0);
      for (int j = k + 1; j < n; ++j) { s += a(i, j) * v[j]; t += z(i, j) * v[j]; }
      s *= beta;
      t *= beta;
      for (int j = k + 1; j < n; ++j) { a(i, j) -= s * std::conj(v[j]); z(i, j) -= t * std::conj(v[j]); }
    }
    for (int i = k + 2; i < n; ++i) a(i, k) = 0.0;
  }
  // ---- shifted QR on the active block [lo, hi]
  int hi = n - 1, sweeps = 0;
  while (hi > 0) {
    if (++sweeps > 60 * n) return false;
    int lo = hi;   // find the unreduced block ending at hi
    while (lo > 0) {
      const double s = std::abs(a(lo - 1, lo - 1)) + std::abs(a(lo, lo));
      if (std::abs(a(lo, lo - 1)) <= 1e-15 * (s > 0.0 ? s : 1.0)) { a(lo, lo - 1) = 0.0; break; }
      --lo;
    }
    if (lo == hi) { --hi; sweeps = 0; continue; }
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to a(hi, hi)
    const zc p = a(hi - 1, hi - 1), q = a(hi - 1, hi), r = a(hi, hi - 1), s = a(hi, hi);
    const zc tr = p + s, det = p * s - q * r;
    const zc disc = std::sqrt(tr * tr - 4.0 * det);
    zc mu1 = 0.5 * (tr + disc), mu2 = 0.5 * (tr - disc);
    zc mu = std::abs(mu1 - s) < std::abs(mu2 - s) ? mu1 : mu2;
    if (sweeps % 11 == 10) mu += std::abs(a(hi, hi - 1)) * zc(0.75, 0.25);   // exceptional shift
    // QR step by Givens rotations on H - mu I, applied as a bulge chase
    zc x = a(lo, lo) - mu, y = a(lo + 1, lo);
    for (int k = lo; k < hi; ++k) {
      if (k > lo) { x = a(k, k - 1); y = a(k + 1, k - 1); }
      const double nr = std::sqrt(std::norm(x) + std::norm(y));
      if (nr == 0.0) continue;
      const zc c = x / nr, sn = y / nr;   // G = [c* s*; -s c], G [x; y] = [nr; 0]
      for (int j = (k > lo ? k - 1 : lo); j < n; ++j) {   // rows k, k+1
        const zc u = a(k, j), t = a(k + 1, j);
        a(k, j) = std::conj(c) * u + std::conj(sn) * t;
        a(k + 1, j) = -sn * u + c * t;
      }
      const int rmax = std::min(hi, k + 2);
      for (int i = 0; i <= rmax; ++i) {   // columns k, k+1
        const zc u = a(i, k), t = a(i, k + 1);
        a(i, k) = u * c + t * sn;
        a(i, k + 1) = -u * std::conj(sn) + t * std::conj(c);
      }
      for (int i = 0; i < n; ++i) {
        const zc u = z(i, k), t = z(i, k + 1);
        z(i, k) = u * c + t * sn;
        z(i, k + 1) = -u * std::conj(sn) + t * std::conj(c);
      }
      if (k > lo) a(k + 1, k - 1) = 0.0;
    }
  }
  // ---- eigenvalues and eigenvectors of the triangular T, then V = Z X
  w.assign(n, zc(0));
  for (int k = 0; k < n; ++k) w[k] = a(k, k);
  V.assign((size_t)n * n, zc(0));
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) tnorm = std::max(tnorm, std::abs(a(i, j)));
  const double small = 1e-14 * (tnorm > 0.0 ? tnorm : 1.0);
  std::vector<zc> xk(n);
  for (int k = 0; k < n; ++k) {
    std::fill(xk.begin(), xk.end(), zc(0));
    xk[k] = 1.0;
    for (int i = k - 1; i >= 0; --i) {
      zc s(0);
      for (int j = i + 1; j <= k; ++j) s += a(i, j) * xk[j];
      zc d = a(i, i) - w[k];
      if (std::abs(d) < small) d = small;
      xk[i] = -s / d;
    }
    double nn = 0.0;
    for (int i = 0; i < n; ++i) {
      zc s(0);
      for (int j = 0; j <= k; ++j) s += z(i, j) * xk[j];
      V[(size_t)i * n + k] = s;
      nn += std::norm(s);
    }
    nn = std::sqrt(nn);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + k] /= nn;
  }
  return true;
}

}  // namespace cclr

// Host harness for the EOM-EE subspace eigensolver (paper_2307_14296_b300/csrc/zeig.h), built by
// tests/test_host_zeig.py: reads n and an n x n complex matrix (row-major "re im" pairs) from
// stdin, prints the eigenvalues ("re im" per line) and then the largest relative residual
// |A v_k - w_k v_k| / |A|_max over the eigenpairs and the largest deviation of |v_k| from 1.
#include <cmath>
#include <complex>
#include <cstdio>
#include <vector>

#include "zeig.h"

int main() {
  int n = 0;
  if (std::scanf("%d", &n) != 1 || n < 1) return 2;
  std::vector<std::complex<double>> A((size_t)n * n), w, V;
  for (auto& a : A) {
    double re = 0.0, im = 0.0;
    if (std::scanf("%lf %lf", &re, &im) != 2) return 2;
    a = {re, im};
  }
  const std::vector<std::complex<double>> A0 = A;
  if (!cclr::zgeev_small(n, A, w, V)) return 3;
  double amax = 0.0;
  for (auto& a : A0) amax = std::max(amax, std::abs(a));
  double res = 0.0, nrm = 0.0;
  for (int k = 0; k < n; ++k) {
    double vn = 0.0;
    for (int i = 0; i < n; ++i) {
      std::complex<double> s(0.0);
      for (int j = 0; j < n; ++j) s += A0[(size_t)i * n + j] * V[(size_t)j * n + k];
      s -= w[k] * V[(size_t)i * n + k];
      res = std::max(res, std::abs(s) / (amax > 0.0 ? amax : 1.0));
      vn += std::norm(V[(size_t)i * n + k]);
    }
    nrm = std::max(nrm, std::abs(std::sqrt(vn) - 1.0));
  }
  for (int k = 0; k < n; ++k) std::printf("%.17g %.17g\n", w[k].real(), w[k].imag());
  std::printf("%.6e %.6e\n", res, nrm);
  return 0;
}

// Iterative solvers of libcclr.
//
//  * Ground state: Jacobi updates with the orbital-energy denominators plus DIIS (the paper uses
//    CROP, Sec. 3; the converged amplitudes are solver-independent).
//  * Linear systems (A - z) t = -b (response, SI "Davidson scheme") and t A = -eta (Lambda):
//    a Davidson solver whose trial space is shared by every shift z of one right-hand side.
//    Per iteration and right-hand side: project (G' = B^H (S - z B), C' = -B^H b), solve the small
//    systems in FP64 on the host, form residuals r = (S - z B) beta + b fused with the
//    orbital-energy-denominator preconditioner delta = -(D - z)^{-1} r, orthogonalize the
//    corrections against the trial space (classical Gram-Schmidt, two passes), and add those
//    that bring a new direction.  Sigma vectors of all new trial vectors of all right-hand sides
//    are evaluated in one batched call.  With one shift this is the paper's per-system scheme.
//  * Response function: t^X(z) = B^X beta^X(z) for every shift, so the CC-CC response function
//    reduces to small bilinear forms: eta^X . B^Y, and (B^X F) . B^Y built from one Hessian
//    product per trial vector.
#include "ctx.h"
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>

namespace cclr {

void zsolve(int n, std::vector<zc>& A, std::vector<zc>& b) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::abs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A[(size_t)i * n + k]) > best) { best = std::abs(A[(size_t)i * n + k]); p = i; }
    CCLR_REQUIRE(best > 0.0, CCLR_E_NOCONV, "singular subspace matrix");
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      zc f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      if (f == zc(0)) continue;
      for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    zc s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[(size_t)k * n + j] * b[j];
    b[k] = s / A[(size_t)k * n + k];
  }
}

namespace {

// The solver's vector kernels compute in FP32 (FP64 storage) in the tensor-core modes, whose
// convergence floor (~1e-5 relative) is far above the ~1e-7 error of that arithmetic.
struct Fast32 {
  Ctx& c;
  bool old;
  explicit Fast32(Ctx& cc) : c(cc), old(cc.L.fast32) { c.L.fast32 = c.opt.precision != CCLR_FP64; }
  ~Fast32() { c.L.fast32 = old; }
};

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void to_host(Ctx& c, const cplx* d, zc* h, int64_t n) {
  CCLR_CK(cudaMemcpyAsync(h, d, sizeof(cplx) * n, cudaMemcpyDeviceToHost, c.stream));
  c.sync();
}
void to_dev(Ctx& c, const zc* h, cplx* d, int64_t n) {
  CCLR_CK(cudaMemcpyAsync(d, h, sizeof(cplx) * n, cudaMemcpyHostToDevice, c.stream));
  c.sync();
}

// out[i*ny + j] = sum op(X_i) Y_j for arbitrary nx, ny (tiles of 64), always in FP64: the
// Galerkin matrices and the response-function forms carry their errors into the results, and the
// residual-norm estimates cancel O(|b|^2) terms.
void gram_host(Ctx& c, int nx, const cplx* X, int ny, const cplx* Y, bool herm, std::vector<zc>& out,
               bool = true) {
  out.assign((size_t)nx * ny, zc(0));
  if (nx == 0 || ny == 0) return;
  Launch L = c.L;
  L.fast32 = false;
  Scope sc(c.ws);
  const int64_t scr_n = (int64_t)reduce_blocks() * 64 * 64;
  cplx* scr = c.ws.cplxs(scr_n);
  cplx* dout = c.ws.cplxs(64 * 64);
  std::vector<zc> blk(64 * 64);
  for (int i0 = 0; i0 < nx; i0 += 64)
    for (int j0 = 0; j0 < ny; j0 += 64) {
      const int bx = std::min(64, nx - i0), by = std::min(64, ny - j0);
      gram(L, c.N, bx, X + (int64_t)i0 * c.N, c.N, by, Y + (int64_t)j0 * c.N, c.N, herm, dout, scr, scr_n);
      to_host(c, dout, blk.data(), (int64_t)bx * by);
      for (int i = 0; i < bx; ++i)
        for (int j = 0; j < by; ++j) out[(size_t)(i0 + i) * ny + j0 + j] = blk[(size_t)i * by + j];
    }
}

// y -= sum_j (B_j^H y) B_j over the nb vectors of B, twice; returns |y| after and before
std::pair<double, double> orthogonalize(Ctx& c, int nb, const cplx* B, cplx* y) {
  Scope sc(c.ws);
  cplx* scr = c.ws.cplxs((int64_t)reduce_blocks() * 64);
  cplx* coef = c.ws.cplxs(64);
  cplx* nrm = c.ws.cplxs(1);
  zc h;
  dots(c.L, c.N, 1, y, 0, y, 0, true, nrm, scr);
  to_host(c, nrm, &h, 1);
  const double before = std::sqrt(std::max(0.0, h.real()));
  for (int pass = 0; pass < 2; ++pass)
    for (int j0 = 0; j0 < nb; j0 += 64) {
      const int bj = std::min(64, nb - j0);
      proj(c.L, c.N, bj, B + (int64_t)j0 * c.N, c.N, y, coef, scr);
      std::vector<zc> cf(bj);
      to_host(c, coef, cf.data(), bj);
      for (auto& x : cf) x = -x;
      to_dev(c, cf.data(), coef, bj);
      lincomb(c.L, c.N, bj, B + (int64_t)j0 * c.N, c.N, coef, y, true);
    }
  dots(c.L, c.N, 1, y, 0, y, 0, true, nrm, scr);
  to_host(c, nrm, &h, 1);
  return {std::sqrt(std::max(0.0, h.real())), before};
}

}  // namespace

// ------------------------------------------------------------------------------ ground state
int solve_ground(Ctx& c) {
  const int64_t N = c.N;
  const int kDiis = 8;
  fill_zero(c.L, c.t, N);
  fill_zero(c.L, c.t2, (int64_t)c.o * c.o * c.v * c.v);
  ++data_generation();
  cplx* R = c.dalloc(N);
  cplx* hist_t = c.dalloc(kDiis * N);
  cplx* hist_e = c.dalloc(kDiis * N);
  fill_zero(c.L, hist_t, kDiis * N);   // unused slots enter the DIIS combination with weight 0
  fill_zero(c.L, hist_e, kDiis * N);
  std::vector<zc> Bm;  // kDiis x kDiis Gram of error vectors
  Bm.assign(kDiis * kDiis, zc(0));
  int nh = 0, head = 0, it = 0;
  Scope sc(c.ws);
  cplx* scr = c.ws.cplxs((int64_t)reduce_blocks() * 64);
  cplx* dd = c.ws.cplxs(64);
  bool ok = false;
  double rn = 0.0, tol_eff = c.opt.ground_tol, rn0 = 0.0, best = 1e300;
  int best_it = 0;
  try {
    for (it = 1; it <= c.opt.maxit * 2; ++it) {
      ccsd_residual(c, R);
      zc h;
      dots(c.L, N, 1, R, 0, R, 0, true, dd, scr);
      to_host(c, dd, &h, 1);
      rn = std::sqrt(h.real());
      c.stats.max_residual = rn;
      // tensor-core modes resolve the residual only to a few 1e-6 of its starting size: target
      // 4e-6 of it, and stop at a stagnating residual below 1e-4 of it (8 iterations without a
      // 20% gain)
      if (it == 1) tol_eff = c.opt.precision == CCLR_FP64 ? c.opt.ground_tol : std::max(c.opt.ground_tol, 4e-6 * rn);
      if (it == 1) rn0 = rn;
      if (rn < tol_eff) { ok = true; break; }
      if (rn < 0.8 * best) { best = rn; best_it = it; }
      if (c.opt.precision != CCLR_FP64 && it - best_it >= 8 && best < 1e-4 * rn0) { ok = true; break; }
      // new error vector e = -R/D and new amplitudes t + e into the ring buffer slot
      cplx* e = hist_e + (int64_t)head * N;
      cplx* tn = hist_t + (int64_t)head * N;
      div_shift(c.L, N, R, c.D, cx(0), cx(-1), e);
      copy_vec(c.L, N, c.t, tn);
      axpy(c.L, N, cx(1), e, tn);
      nh = std::min(nh + 1, kDiis);
      // Gram row/column of the new error vector against the stored ones
      std::vector<zc> g(kDiis);
      proj(c.L, N, kDiis, hist_e, N, e, dd, scr);
      to_host(c, dd, g.data(), kDiis);
      for (int j = 0; j < kDiis; ++j) {
        Bm[(size_t)head * kDiis + j] = std::conj(g[j]);
        Bm[(size_t)j * kDiis + head] = g[j];
      }
      head = (head + 1) % kDiis;
      if (nh >= 2) {
        const int m = nh;
        std::vector<int> slots;
        for (int k = 0; k < kDiis && (int)slots.size() < m; ++k) slots.push_back(k);
        std::vector<zc> A((size_t)(m + 1) * (m + 1), zc(0)), rhs(m + 1, zc(0));
        for (int i = 0; i < m; ++i)
          for (int j = 0; j < m; ++j) A[(size_t)i * (m + 1) + j] = Bm[(size_t)slots[i] * kDiis + slots[j]];
        for (int i = 0; i < m; ++i) A[(size_t)i * (m + 1) + m] = A[(size_t)m * (m + 1) + i] = zc(-1);
        rhs[m] = zc(-1);
        bool good = true;
        try { zsolve(m + 1, A, rhs); } catch (const Error&) { good = false; }
        if (good) {
          std::vector<zc> cf(kDiis, zc(0));
          for (int i = 0; i < m; ++i) cf[slots[i]] = rhs[i];
          to_dev(c, cf.data(), dd, kDiis);
          lincomb(c.L, N, kDiis, hist_t, N, dd, c.t, false);
        } else {
          copy_vec(c.L, N, tn, c.t);
        }
      } else {
        copy_vec(c.L, N, tn, c.t);
      }
      expand_t2(c, c.t + c.Ns, c.t2, 1);
    }
  } catch (...) {
    c.dfree(R); c.dfree(hist_t); c.dfree(hist_e);
    throw;
  }
  c.dfree(R); c.dfree(hist_t); c.dfree(hist_e);
  c.e_corr = ccsd_energy(c);
  c.have_t = true;
  if (!ok) throw Error(CCLR_E_NOCONV, "CCSD did not converge: |Omega| = " + std::to_string(rn));
  return it;
}

// ------------------------------------------------------------------------------ Davidson
struct System {            // one right-hand side with its shared trial space
  const cplx* rhs;         // b (device, N)
  std::vector<zc> z;       // shifts
  cplx *B = nullptr, *S = nullptr;
  int L = 0;
  std::vector<zc> BS, Cp;  // maxL x maxL (B^H S), -B^H b
  std::vector<zc> SS, BB;  // maxL x maxL: S^H S, B^H B
  std::vector<zc> Sx;      // S^H b
  double xx = 0.0;         // b^H b
  std::vector<std::vector<zc>> beta;
  std::vector<double> rnorm;
  std::vector<char> conv;
  int iters = 0;
  double best = 1e300;     // best max-residual so far and its iteration (stagnation test)
  int best_it = 0;
};

// Thick restart: compress the trial space onto the span of the current solutions of all shifts
// (QR with column pivoting of the coefficient matrix [beta_1 ... beta_ns], at most kmax columns).
// Sigma vectors transform with the basis (S' = S Q), so no sigma is recomputed.
void restart(Ctx& c, System& s, int maxL, int kmax) {
  const int64_t N = c.N;
  const int L = s.L, ns = (int)s.z.size();
  std::vector<std::vector<zc>> cols(ns, std::vector<zc>(L));
  for (int q = 0; q < ns; ++q)
    for (int i = 0; i < L; ++i) cols[q][i] = s.beta[q][i];
  std::vector<std::vector<zc>> Q;
  std::vector<char> used(ns, 0);
  double first = -1.0;
  while ((int)Q.size() < kmax) {
    int best = -1;
    double bn = 0.0;
    for (int q = 0; q < ns; ++q) {
      if (used[q]) continue;
      double nn = 0.0;
      for (auto& x : cols[q]) nn += std::norm(x);
      if (nn > bn) { bn = nn; best = q; }
    }
    if (best < 0) break;
    const double nrm = std::sqrt(bn);
    if (first < 0) first = nrm;
    if (nrm <= 1e-13 * first) break;
    used[best] = 1;
    std::vector<zc> qv(L);
    for (int i = 0; i < L; ++i) qv[i] = cols[best][i] / nrm;
    for (int q = 0; q < ns; ++q) {
      if (used[q]) continue;
      zc d(0);
      for (int i = 0; i < L; ++i) d += std::conj(qv[i]) * cols[q][i];
      for (int i = 0; i < L; ++i) cols[q][i] -= d * qv[i];
    }
    Q.push_back(qv);
  }
  const int kk = (int)Q.size();
  CCLR_REQUIRE(kk >= 1, CCLR_E_NOCONV, "Davidson restart: empty solution space");
  {
    Scope sc(c.ws);
    cplx* tmp = c.ws.cplxs((int64_t)kk * N);
    cplx* coef = c.ws.cplxs(L);
    for (cplx* X : {s.B, s.S}) {
      for (int j = 0; j < kk; ++j) {
        to_dev(c, Q[j].data(), coef, L);
        lincomb(c.L, N, L, X, N, coef, tmp + (int64_t)j * N, false);
      }
      copy_vec(c.L, (int64_t)kk * N, tmp, X);
    }
  }
  auto congr = [&](std::vector<zc>& M) {   // M' = Q^H M Q
    std::vector<zc> out((size_t)maxL * maxL, zc(0));
    for (int a = 0; a < kk; ++a)
      for (int b = 0; b < kk; ++b) {
        zc acc(0);
        for (int i = 0; i < L; ++i) {
          zc r(0);
          for (int j = 0; j < L; ++j) r += M[(size_t)i * maxL + j] * Q[b][j];
          acc += std::conj(Q[a][i]) * r;
        }
        out[(size_t)a * maxL + b] = acc;
      }
    M.swap(out);
  };
  congr(s.BS);
  congr(s.SS);
  congr(s.BB);
  auto vec = [&](std::vector<zc>& v) {     // v' = Q^H v
    std::vector<zc> out(maxL, zc(0));
    for (int a = 0; a < kk; ++a)
      for (int i = 0; i < L; ++i) out[a] += std::conj(Q[a][i]) * v[i];
    v.swap(out);
  };
  vec(s.Cp);
  vec(s.Sx);
  for (int q = 0; q < ns; ++q) {           // beta in the new basis (re-solved next iteration)
    std::vector<zc> nb(maxL, zc(0));
    for (int a = 0; a < kk; ++a)
      for (int i = 0; i < L; ++i) nb[a] += std::conj(Q[a][i]) * s.beta[q][i];
    s.beta[q].swap(nb);
  }
  s.L = kk;
  c.stats.sigma_calls += 0;
}

// Solve (Op - z) x = -b for every system and shift.  Op(nvec, in, out) acts on N-vectors.
void davidson(Ctx& c, std::vector<System>& sys, const std::function<void(int, const cplx*, cplx*)>& Op,
              int maxL, double tol) {
  static const bool verbose = std::getenv("CCLR_VERBOSE") != nullptr;
  Fast32 f32(c);
  const int64_t N = c.N;
  const int kMaxNew = 4;   // new trial vectors per right-hand side and iteration (worst shifts first)
  Scope sc(c.ws);
  cplx* scr = c.ws.cplxs((int64_t)reduce_blocks() * 64);
  cplx* bdev = c.ws.cplxs(maxL);
  double* r2dev = (double*)c.ws.alloc(sizeof(double) * 2);
  double* rscr = (double*)c.ws.alloc(sizeof(double) * reduce_blocks());
  cplx* delta = c.ws.cplxs(N);
  for (auto& s : sys) {
    s.BS.assign((size_t)maxL * maxL, zc(0));
    s.SS.assign((size_t)maxL * maxL, zc(0));
    s.BB.assign((size_t)maxL * maxL, zc(0));
    s.Cp.assign(maxL, zc(0));
    s.Sx.assign(maxL, zc(0));
    {
      std::vector<zc> g;
      gram_host(c, 1, s.rhs, 1, s.rhs, true, g, true);
      s.xx = g[0].real();
    }
    s.beta.assign(s.z.size(), std::vector<zc>(maxL, zc(0)));
    s.rnorm.assign(s.z.size(), 1e300);
    s.conv.assign(s.z.size(), 0);
    s.L = 0;
    // start: b / D, normalized (preconditioned right-hand side at z = 0)
    div_shift(c.L, N, s.rhs, c.D, cx(0), cx(1), s.B);
    auto nr = orthogonalize(c, 0, s.B, s.B);
    CCLR_REQUIRE(nr.second > 0.0, CCLR_E_ARG, "zero right-hand side");
    scale_vec(c.L, N, cx(1.0 / nr.second), s.B);
    s.L = 1;
  }
  std::vector<int> fresh(sys.size(), 1);   // new vectors at the end of each basis
  for (int it = 1; it <= c.opt.maxit; ++it) {
    // ---- sigma of all new vectors (one batched call; vectors are gathered contiguously)
    int total = 0;
    for (size_t k = 0; k < sys.size(); ++k) total += fresh[k];
    if (total == 0) break;
    {
      Scope s2(c.ws);
      cplx* in = c.ws.cplxs((int64_t)total * N);
      cplx* out = c.ws.cplxs((int64_t)total * N);
      int q = 0;
      for (size_t k = 0; k < sys.size(); ++k)
        for (int j = 0; j < fresh[k]; ++j, ++q)
          copy_vec(c.L, N, sys[k].B + (int64_t)(sys[k].L - fresh[k] + j) * N, in + (int64_t)q * N);
      const int bmax = c.opt.batch > 0 ? c.opt.batch : total;
      double t0 = now();
      for (int q0 = 0; q0 < total; q0 += bmax) {
        const int nb = std::min(bmax, total - q0);
        Op(nb, in + (int64_t)q0 * N, out + (int64_t)q0 * N);
      }
      c.sync();
      c.stats.sigma_seconds += now() - t0;
      q = 0;
      for (size_t k = 0; k < sys.size(); ++k)
        for (int j = 0; j < fresh[k]; ++j, ++q)
          copy_vec(c.L, N, out + (int64_t)q * N, sys[k].S + (int64_t)(sys[k].L - fresh[k] + j) * N);
    }
    bool all_conv = true;
    for (size_t k = 0; k < sys.size(); ++k) {
      System& s = sys[k];
      const int L0 = s.L - fresh[k], f = fresh[k];
      // ---- Gram blocks of the new vectors: B^H S, S^H S, B^H B and S^H b (FP64, host)
      if (f > 0) {
        std::vector<zc> g;
        const cplx* Bn = s.B + (int64_t)L0 * N;
        const cplx* Sn = s.S + (int64_t)L0 * N;
        auto put = [&](std::vector<zc>& M, const std::vector<zc>& blk, int r0, int nr, int c0, int nc, bool herm_fill) {
          for (int i = 0; i < nr; ++i)
            for (int j = 0; j < nc; ++j) {
              M[(size_t)(r0 + i) * maxL + c0 + j] = blk[(size_t)i * nc + j];
              if (herm_fill) M[(size_t)(c0 + j) * maxL + r0 + i] = std::conj(blk[(size_t)i * nc + j]);
            }
        };
        gram_host(c, s.L, s.B, f, Sn, true, g, true);     // B^H S_new: new columns of BS
        put(s.BS, g, 0, s.L, L0, f, false);
        if (L0 > 0) {
          gram_host(c, f, Bn, L0, s.S, true, g, true);    // B_new^H S_old: new rows of BS
          put(s.BS, g, L0, f, 0, L0, false);
        }
        gram_host(c, s.L, s.S, f, Sn, true, g);           // S^H S_new (Hermitian)
        put(s.SS, g, 0, s.L, L0, f, true);
        gram_host(c, s.L, s.B, f, Bn, true, g, true);     // B^H B_new (Hermitian)
        put(s.BB, g, 0, s.L, L0, f, true);
        gram_host(c, f, Bn, 1, s.rhs, true, g, true);     // B_new^H b
        for (int i = 0; i < f; ++i) s.Cp[L0 + i] = -g[i];
        gram_host(c, f, Sn, 1, s.rhs, true, g);           // S_new^H b
        for (int i = 0; i < f; ++i) s.Sx[L0 + i] = g[i];
      }
      fresh[k] = 0;
      // ---- subspace solves; residual norms from the Gram matrices:
      //   |r|^2 = beta^H (S - zB)^H (S - zB) beta + 2 Re beta^H (S^H b - z* B^H b) + b^H b
      const int L = s.L;
      // tensor-core modes: sigma carries ~1e-5 relative error at long K (FP32 accumulation), so
      // the reachable residual is ~1e-5 of |b|; the target is raised to that floor
      const double tol_s = c.opt.precision == CCLR_FP64 ? tol : std::max(tol, 1e-5 * std::sqrt(s.xx));
      std::vector<std::pair<double, int>> order;
      for (size_t q = 0; q < s.z.size(); ++q) {
        const zc z = s.z[q];
        std::vector<zc> G((size_t)L * L), rhs(s.Cp.begin(), s.Cp.begin() + L);
        for (int i = 0; i < L; ++i)
          for (int j = 0; j < L; ++j) G[(size_t)i * L + j] = s.BS[(size_t)i * maxL + j] - z * s.BB[(size_t)i * maxL + j];
        zsolve(L, G, rhs);
        for (int i = 0; i < L; ++i) s.beta[q][i] = rhs[i];
        const zc* b = rhs.data();
        zc quad(0), lin(0);
        for (int i = 0; i < L; ++i) {
          zc row(0);
          for (int j = 0; j < L; ++j) {
            const size_t ij = (size_t)i * maxL + j, ji = (size_t)j * maxL + i;
            const zc Gij = s.SS[ij] - z * std::conj(s.BS[ji]) - std::conj(z) * s.BS[ij] + std::norm(z) * s.BB[ij];
            row += Gij * b[j];
          }
          quad += std::conj(b[i]) * row;
          lin += std::conj(b[i]) * (s.Sx[i] + std::conj(z) * s.Cp[i]);   // Cp = -B^H b
        }
        const double r2 = quad.real() + 2.0 * lin.real() + s.xx;
        s.rnorm[q] = std::sqrt(std::max(0.0, r2));
        // the Gram estimate cancels O(|b|^2) terms: with FP64 Gram blocks it resolves |r| down to
        // ~1e-7 |b|; below that, confirm on the vectors
        const double floor = 1e-7 * std::sqrt(s.xx);
        if (s.rnorm[q] < std::max(tol_s, floor) * 4.0) {
          to_dev(c, rhs.data(), bdev, L);
          residual_precond(c.L, N, L, s.S, s.B, N, bdev, cx(z.real(), z.imag()), s.rhs, c.D, nullptr, delta, r2dev,
                           rscr);
          double e2;
          CCLR_CK(cudaMemcpyAsync(&e2, r2dev, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
          c.sync();
          s.rnorm[q] = std::sqrt(e2);
        }
        s.conv[q] = s.rnorm[q] < tol_s;
        if (!s.conv[q]) order.push_back({s.rnorm[q], (int)q});
        c.stats.max_residual = std::max(c.stats.max_residual, s.rnorm[q]);
      }
      s.iters = it;
      if (verbose)
        std::fprintf(stderr, "[cclr] davidson it %d rhs %zu L %d unconverged %zu/%zu max|r| %.3e tol %.1e\n", it, k, L,
                     order.size(), s.z.size(), order.empty() ? 0.0 : std::max_element(order.begin(), order.end())->first,
                     tol_s);
      if (!order.empty() && c.opt.precision != CCLR_FP64) {
        // tensor-core modes: accept a stagnating solve whose residuals are all within 5x the floor
        double mx = 0.0;
        for (auto& pr : order) mx = std::max(mx, pr.first);
        if (mx < 0.8 * s.best) { s.best = mx; s.best_it = it; }
        if (it - s.best_it >= 4 && mx < 5.0 * tol_s) order.clear();
      }
      if (order.empty()) continue;
      all_conv = false;
      std::sort(order.begin(), order.end(), [](auto& a, auto& b) { return a.first > b.first; });
      if (s.L + kMaxNew > maxL) restart(c, s, maxL, maxL - 2 * kMaxNew);
      int added = 0, tried = 0;
      for (auto& pr : order) {
        // corrections of neighbouring shifts are nearly collinear: try a few, worst first
        if (added >= kMaxNew || s.L >= maxL || tried >= 2 * kMaxNew) break;
        ++tried;
        const int q = pr.second;
        std::vector<zc> bq(s.beta[q].begin(), s.beta[q].begin() + s.L);
        to_dev(c, bq.data(), bdev, s.L);
        cplx* nb = s.B + (int64_t)s.L * N;
        residual_precond(c.L, N, s.L, s.S, s.B, N, bdev, cx(s.z[q].real(), s.z[q].imag()), s.rhs, c.D, nullptr, nb,
                         r2dev, rscr);
        auto nr = orthogonalize(c, s.L, s.B, nb);
        // accept a correction only if at least 1% of it lies outside the trial space
        if (nr.first <= 1e-2 * nr.second || nr.first < 1e-300) continue;
        scale_vec(c.L, N, cx(1.0 / nr.first), nb);
        s.L++;
        fresh[k]++;
        added++;
      }
      if (added == 0)
        throw Error(CCLR_E_NOCONV, "Davidson stagnated: residual " + std::to_string(order.front().first) +
                                       " above tolerance " + std::to_string(tol_s) + " with no new direction");
    }
    if (all_conv) return;
  }
  throw Error(CCLR_E_NOCONV, "Davidson did not converge within maxit iterations");
}

// ------------------------------------------------------------------------------ Lambda
int solve_lambda(Ctx& c) {
  const int64_t N = c.N;
  const int maxL = std::max(8, c.opt.max_subspace);
  cplx* eta = c.dalloc(N);
  eta_ground(c, eta);
  System s;
  s.rhs = eta;
  s.z = {zc(0)};
  s.B = c.dalloc((int64_t)maxL * N);
  s.S = c.dalloc((int64_t)maxL * N);
  std::vector<System> sys{s};
  auto cleanup = [&]() { c.dfree(sys[0].B); c.dfree(sys[0].S); c.dfree(eta); };
  try {
    davidson(c, sys, [&](int nv, const cplx* in, cplx* out) { sigma_left(c, nv, in, out); }, maxL, c.opt.ground_tol);
  } catch (...) {
    cleanup();
    throw;
  }
  // lambda = B beta
  Scope sc(c.ws);
  cplx* bd = c.ws.cplxs(maxL);
  to_dev(c, sys[0].beta[0].data(), bd, sys[0].L);
  lincomb(c.L, N, sys[0].L, sys[0].B, N, bd, c.lam, false);
  expand_t2(c, c.lam + c.Ns, c.l2, 1);
  const int its = sys[0].iters;
  cleanup();
  c.have_lambda = true;
  c.named.erase("F.ready");
  return its;
}

// ------------------------------------------------------------------------------ response
void lr_solve(Ctx& c, int n_ops, const cplx* ops_host, int n_freq, const double* omegas, double gamma,
              int* iters_out) {
  ResponseData& rd = c.rd;
  for (auto p : rd.ops_dev) c.dfree(p);
  for (auto p : rd.xi) c.dfree(p);
  for (auto p : rd.eta) c.dfree(p);
  for (auto p : rd.basis) c.dfree(p);
  for (auto p : rd.sig) c.dfree(p);
  rd = ResponseData();
  const int64_t N = c.N, n = c.n;
  const int maxL = std::max(8, c.opt.max_subspace);
  rd.n_ops = n_ops;
  rd.n_freq = n_freq;
  rd.gamma = gamma;
  rd.omegas.assign(omegas, omegas + n_freq);
  // unique shifts {w+ig, -w+ig, w-ig, -w-ig}
  rd.shift_of.assign((size_t)n_freq * 4, 0);
  for (int f = 0; f < n_freq; ++f) {
    const zc cand[4] = {zc(omegas[f], gamma), zc(-omegas[f], gamma), zc(omegas[f], -gamma), zc(-omegas[f], -gamma)};
    for (int s = 0; s < 4; ++s) {
      int idx = -1;
      for (size_t q = 0; q < rd.shifts.size(); ++q)
        if (std::abs(rd.shifts[q] - cand[s]) < 1e-14) idx = (int)q;
      if (idx < 0) { idx = (int)rd.shifts.size(); rd.shifts.push_back(cand[s]); }
      rd.shift_of[(size_t)f * 4 + s] = idx;
    }
  }
  std::vector<System> sys(n_ops);
  for (int k = 0; k < n_ops; ++k) {
    cplx* X = c.dalloc(n * n);
    CCLR_CK(cudaMemcpyAsync(X, ops_host + (int64_t)k * n * n, sizeof(cplx) * n * n, cudaMemcpyHostToDevice, c.stream));
    rd.ops_dev.push_back(X);
    cplx* xi = c.dalloc(N);
    xi_vec(c, X, xi);
    rd.xi.push_back(xi);
    cplx* et = c.dalloc(N);
    eta_vec(c, X, false, et);
    rd.eta.push_back(et);
    rd.basis.push_back(c.dalloc((int64_t)maxL * N));
    rd.sig.push_back(c.dalloc((int64_t)maxL * N));
    sys[k].rhs = xi;
    sys[k].z = rd.shifts;
    sys[k].B = rd.basis[k];
    sys[k].S = rd.sig[k];
  }
  davidson(c, sys, [&](int nv, const cplx* in, cplx* out) { sigma_right(c, nv, in, out); }, maxL, c.opt.tol);
  rd.nb.resize(n_ops);
  rd.beta.resize(n_ops);
  rd.iters.assign((size_t)n_ops * n_freq, 0);
  for (int k = 0; k < n_ops; ++k) {
    rd.nb[k] = sys[k].L;
    rd.beta[k].assign(rd.shifts.size() * (size_t)maxL, zc(0));
    for (size_t q = 0; q < rd.shifts.size(); ++q)
      for (int i = 0; i < sys[k].L; ++i) rd.beta[k][q * maxL + i] = sys[k].beta[q][i];
    for (int f = 0; f < n_freq; ++f) rd.iters[(size_t)k * n_freq + f] = sys[k].iters;
  }
  if (iters_out)
    for (int i = 0; i < n_ops * n_freq; ++i) iters_out[i] = rd.iters[i];
  // the response function needs the trial vectors and the subspace solutions only
  for (auto& p : rd.sig) c.dfree(p);
  rd.sig.clear();
  rd.solved = true;
}

void response_function(Ctx& c, cplx* out_host) {
  ResponseData& rd = c.rd;
  CCLR_REQUIRE(rd.solved, CCLR_E_STATE, "cc_response_function before cc_lr_solve");
  Fast32 f32(c);
  const int64_t N = c.N;
  const int nop = rd.n_ops, maxL = std::max(8, c.opt.max_subspace);
  // Bilinear forms M^{xy}_{kl} = (b^x_k F) . b^y_l and E^{xy}_l = eta^x . b^y_l.  The Hessian
  // products of the trial vectors are formed in batches and contracted at once (never stored).
  std::vector<std::vector<zc>> M((size_t)nop * nop), E((size_t)nop * nop);
  for (int x = 0; x < nop; ++x)
    for (int y = 0; y < nop; ++y) gram_host(c, 1, rd.eta[x], rd.nb[y], rd.basis[y], false, E[(size_t)x * nop + y], true);
  auto beta = [&](int k, int f, int s) { return &rd.beta[k][(size_t)rd.shift_of[(size_t)f * 4 + s] * maxL]; };
  // The Hessian acts only on the solutions t^X(-z) and t^X(z*) of every frequency.  Their
  // coefficient vectors span few directions: compress them (QR with column pivoting, 1e-12
  // cutoff) to Q_x, form the products F (B^x Q_x) in batches and contract them at once:
  //   M^{xy} = (B^x Q_x F) . B^y,  (t^X F) . t^Y = gamma^T M^{xy} beta^Y,  gamma = Q_x^H beta^X.
  std::vector<std::vector<std::vector<zc>>> Q(nop);
  for (int x = 0; x < nop; ++x) {
    const int Lx = rd.nb[x];
    std::vector<std::vector<zc>> cols;
    for (int f = 0; f < rd.n_freq; ++f)
      for (int s : {3, 2}) cols.emplace_back(beta(x, f, s), beta(x, f, s) + Lx);
    std::vector<char> used(cols.size(), 0);
    double first = -1.0;
    while ((int)Q[x].size() < Lx) {
      int best = -1;
      double bn = 0.0;
      for (size_t q = 0; q < cols.size(); ++q) {
        if (used[q]) continue;
        double nn = 0.0;
        for (auto& v : cols[q]) nn += std::norm(v);
        if (nn > bn) { bn = nn; best = (int)q; }
      }
      if (best < 0) break;
      const double nrm = std::sqrt(bn);
      if (first < 0) first = nrm;
      if (nrm <= 1e-12 * first) break;
      used[best] = 1;
      std::vector<zc> qv(Lx);
      for (int i = 0; i < Lx; ++i) qv[i] = cols[best][i] / nrm;
      for (size_t q = 0; q < cols.size(); ++q) {
        if (used[q]) continue;
        zc d(0);
        for (int i = 0; i < Lx; ++i) d += std::conj(qv[i]) * cols[q][i];
        for (int i = 0; i < Lx; ++i) cols[q][i] -= d * qv[i];
      }
      Q[x].push_back(qv);
    }
    const int rx = (int)Q[x].size();
    for (int y = 0; y < nop; ++y) M[(size_t)x * nop + y].assign((size_t)rx * rd.nb[y], zc(0));
    const int bmax = std::max(1, std::min(c.opt.batch > 0 ? c.opt.batch : 8, rx));
    for (int q0 = 0; q0 < rx; q0 += bmax) {
      const int nb = std::min(bmax, rx - q0);
      Scope sc(c.ws);
      cplx* yv = c.ws.cplxs((int64_t)nb * N);
      cplx* fb = c.ws.cplxs((int64_t)nb * N);
      cplx* coef = c.ws.cplxs(Lx);
      for (int j = 0; j < nb; ++j) {
        to_dev(c, Q[x][q0 + j].data(), coef, Lx);
        lincomb(c.L, N, Lx, rd.basis[x], N, coef, yv + (int64_t)j * N, false);
      }
      hessian_right(c, nb, yv, fb);
      for (int y = 0; y < nop; ++y) {
        std::vector<zc> g;
        gram_host(c, nb, fb, rd.nb[y], rd.basis[y], false, g, true);
        auto& Mxy = M[(size_t)x * nop + y];
        for (int i = 0; i < nb; ++i)
          for (int j = 0; j < rd.nb[y]; ++j) Mxy[(size_t)(q0 + i) * rd.nb[y] + j] = g[(size_t)i * rd.nb[y] + j];
      }
    }
  }
  // f(z) = 1/2 [eta^X t^Y(z) + eta^Y t^X(-z) + (t^X(-z) F) t^Y(z)]
  auto half = [&](int f, int x, int y, int sz, int smz) {
    const zc* by = beta(y, f, sz);
    const zc* bx = beta(x, f, smz);
    const int Lx = rd.nb[x], Ly = rd.nb[y], rx = (int)Q[x].size();
    zc a(0), b(0), q(0);
    for (int j = 0; j < Ly; ++j) a += E[(size_t)x * nop + y][j] * by[j];
    for (int i = 0; i < Lx; ++i) b += E[(size_t)y * nop + x][i] * bx[i];
    const auto& Mxy = M[(size_t)x * nop + y];
    for (int i = 0; i < rx; ++i) {
      zc g(0), r(0);
      for (int l = 0; l < Lx; ++l) g += std::conj(Q[x][i][l]) * bx[l];
      for (int j = 0; j < Ly; ++j) r += Mxy[(size_t)i * Ly + j] * by[j];
      q += g * r;
    }
    return 0.5 * (a + b + q);
  };
  for (int f = 0; f < rd.n_freq; ++f)
    for (int x = 0; x < nop; ++x)
      for (int y = 0; y < nop; ++y) {
        // shifts: 0: w+ig (z), 1: -w+ig (-z*), 2: w-ig (z*), 3: -w-ig (-z)
        const zc val = half(f, x, y, 0, 3) + std::conj(half(f, x, y, 1, 2));
        out_host[((size_t)f * nop + x) * nop + y] = make_double2(val.real(), val.imag());
      }
}

}  // namespace cclr

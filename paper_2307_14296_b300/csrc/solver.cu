// Iterative solvers of libcclr.
//
//  * Ground state: Jacobi updates with the orbital-energy denominators plus DIIS (the paper uses
//    CROP, Sec. 3; the converged amplitudes are solver-independent).
//  * Linear systems (A - z) t = -b (response, SI "Davidson scheme") and t A = -eta (Lambda):
//    a Davidson solver whose trial space is shared by every shift z of one right-hand side.
//    Per iteration and right-hand side: project (G' = B^H (S - z B), C' = -B^H b), solve the small
//    systems in FP64 on the host, form residuals r = (S - z B) beta + b fused with the
//    orbital-energy-denominator preconditioner delta = -(D - z)^{-1} r, project the corrections
//    against the trial space, and add those that bring a new direction.  Sigma vectors of all
//    new trial vectors of all right-hand sides are evaluated in one batched call.  With one
//    shift this is the paper's per-system scheme.
//  * Response function: t^X(z) = B^X beta^X(z) for every shift, so the CC-CC response function
//    reduces to small bilinear forms: eta^X . B^Y, and (B^X F) . B^Y built from one Hessian
//    product per trial vector.
#include "ctx.h"
#include "zeig.h"
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <memory>

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
  explicit Fast32(Ctx& cc) : c(cc), old(cc.L.fast32) { c.L.fast32 = mixed_precision(c.opt.precision); }
  ~Fast32() { c.L.fast32 = old; }
};

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Wall time per solver phase, printed when CCLR_VERBOSE is set (the stream is synchronized at
// every phase boundary then, so those runs are slower)
struct Phases {
  const char* what;
  bool on;
  std::vector<std::pair<std::string, double>> t;
  std::string cur;
  double t0 = 0.0;
  explicit Phases(const char* w) : what(w), on(std::getenv("CCLR_VERBOSE") != nullptr) {}
  void mark(Ctx& c, const char* name) {
    if (!on) return;
    c.sync();
    const double n = now();
    if (!cur.empty()) {
      auto it = std::find_if(t.begin(), t.end(), [&](auto& p) { return p.first == cur; });
      if (it == t.end()) t.push_back({cur, n - t0});
      else it->second += n - t0;
    }
    cur = name;
    t0 = n;
  }
  ~Phases() {
    if (!on || t.empty()) return;
    std::fprintf(stderr, "[cclr] %s phases:", what);
    for (auto& p : t) std::fprintf(stderr, " %s %.3fs", p.first.c_str(), p.second);
    std::fprintf(stderr, "\n");
  }
};

void to_host(Ctx& c, const cplx* d, zc* h, int64_t n) {
  CCLR_CK(cudaMemcpyAsync(h, d, sizeof(cplx) * n, cudaMemcpyDeviceToHost, c.stream));
  c.sync();
}
void to_dev(Ctx& c, const zc* h, cplx* d, int64_t n) {
  CCLR_CK(cudaMemcpyAsync(d, h, sizeof(cplx) * n, cudaMemcpyHostToDevice, c.stream));
  c.sync();
}

// out[i*ny + j] = sum op(X_i) Y_j over row lists of any length, in tiles that the Gram kernel
// takes (FP32 products when the solver's vector kernels run in FP32, FP64 otherwise)
void gram_host(Ctx& c, const Rows& X, const Rows& Y, bool herm, std::vector<zc>& out, bool x32 = false) {
  const int nx = X.total(), ny = Y.total();
  out.assign((size_t)nx * ny, zc(0));
  if (nx == 0 || ny == 0) return;
  Scope sc(c.ws);
  cplx* scr = c.ws.cplxs(gram_scratch_elems());
  cplx* dout = c.ws.cplxs((int64_t)nx * ny);
  gram(c.L, c.N, X, Y, herm, dout, scr, gram_scratch_elems(), x32);
  to_host(c, dout, out.data(), (int64_t)nx * ny);
}

Rows rows(const Ctx& c, const cplx* p, int n) {
  Rows r;
  r.add(p, n, c.N);
  return r;
}

double norm2(Ctx& c, const cplx* x) {
  std::vector<zc> g;
  gram_host(c, rows(c, x, 1), rows(c, x, 1), true, g);
  return std::max(0.0, g[0].real());
}

// Y_q = sum_j X_j W[j*m + q] for m outputs in passes of kVecMatOut (W on the host, nx x m)
void combine(Ctx& c, const Rows& X, int m, const std::vector<zc>& W, cplx* Y) {
  const int nx = X.total();
  Scope sc(c.ws);
  cplx* cdev = c.ws.cplxs((int64_t)nx * kVecMatOut);
  for (int q0 = 0; q0 < m; q0 += kVecMatOut) {
    const int mq = std::min(kVecMatOut, m - q0);
    std::vector<zc> Cq((size_t)nx * mq);
    for (int j = 0; j < nx; ++j)
      for (int q = 0; q < mq; ++q) Cq[(size_t)j * mq + q] = W[(size_t)j * m + q0 + q];
    to_dev(c, Cq.data(), cdev, (int64_t)nx * mq);
    VecMat a;
    a.X = X;
    a.m = mq;
    a.C = cdev;
    a.Y = Y + (int64_t)q0 * c.N;
    a.ldy = c.N;
    vecmat(c.L, c.N, a, nullptr);
  }
}

}  // namespace

// ------------------------------------------------------------------------------ ground state
// Jacobi + DIIS.  In the mixed modes the residuals are first evaluated with split-BF16 tensor-core
// contractions until the residual falls to mixed_floor() of the first one (or stagnates within
// 10x of it); with refinement the iteration then continues, DIIS restarted, with FP64-class
// residuals to ground_tol.
int solve_ground(Ctx& c) {
  const int64_t N = c.N;
  const int kDiis = 8;
  const bool mixed = mixed_precision(c.opt.precision);
  const bool refine = refining(c);
  int phase = mixed ? 1 : 2;
  std::unique_ptr<PrecisionScope> exact;   // the FP64-class arithmetic of the refinement phase
  double t_ref = 0.0;
  long v_ref = 0;
  fill_zero(c.L, c.t, N);
  fill_zero(c.L, c.t2, (int64_t)c.o * c.o * c.v * c.v);
  ++c.data_gen;
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
  Phases ph("ground");
  int it_ref0 = 0;
  try {
    for (it = 1; it <= c.opt.maxit * 2 + (phase == 2 && mixed ? it_ref0 : 0); ++it) {
      ph.mark(c, "residual");
      if (phase == 2 && mixed) { ++v_ref; }
      const double t0 = now();
      ccsd_residual(c, R);
      ph.mark(c, "diis");
      zc h;
      dots(c.L, N, 1, R, 0, R, 0, true, dd, scr);
      to_host(c, dd, &h, 1);
      if (phase == 2 && mixed) t_ref += now() - t0;
      rn = std::sqrt(h.real());
      c.stats.max_residual = rn;
      // mixed modes: the residual carries ~1e-5 relative error (split-BF16 operands, FP32
      // accumulation; the Fock diagonal is exact), so the mixed phase ends at mixed_floor() of the
      // starting residual, or at a stagnating residual below 10x that (8 iterations without a
      // 20% gain)
      if (it == 1) tol_eff = mixed ? std::max(c.opt.ground_tol, mixed_floor(c) * rn) : c.opt.ground_tol;
      if (it == 1) rn0 = rn;
      if (phase == 1) {
        if (rn < 0.8 * best) { best = rn; best_it = it; }
        const bool floor = rn < tol_eff || (it - best_it >= 8 && best < 10.0 * mixed_floor(c) * rn0);
        if (floor && (!refine || rn < c.opt.ground_tol)) { ok = true; break; }
        if (floor) {
          // refinement: the same amplitudes, FP64-class residuals, DIIS restarted
          phase = 2;
          it_ref0 = it;
          exact.reset(new PrecisionScope(c, CCLR_TC_F64));
          nh = 0;
          head = 0;
          std::fill(Bm.begin(), Bm.end(), zc(0));
          continue;
        }
      } else if (rn < c.opt.ground_tol) {
        ok = true;
        break;
      }
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
    ph.mark(c, "");
  } catch (...) {
    c.dfree(R); c.dfree(hist_t); c.dfree(hist_e);
    throw;
  }
  c.dfree(R); c.dfree(hist_t); c.dfree(hist_e);
  c.stats.refine_vectors += v_ref;
  c.stats.refine_seconds += t_ref;
  c.e_corr = ccsd_energy(c);
  c.have_t = true;
  if (!ok) throw Error(CCLR_E_NOCONV, "CCSD did not converge: |Omega| = " + std::to_string(rn));
  return it;
}

// ------------------------------------------------------------------------------ Davidson
struct System {            // one right-hand side with its shared trial space
  const cplx* rhs = nullptr;   // b (device, N)
  std::vector<zc> z;       // shifts
  cplx *B = nullptr, *S = nullptr;
  // FP32 mirrors of B and S (tensor-core modes): the passes whose arithmetic is FP32 anyway
  // (residual norms, candidates, projections) read 8 instead of 16 bytes per element
  void *Bf = nullptr, *Sf = nullptr, *bf = nullptr;   // rows of Np = N rounded up to even elements
  int L = 0;
  std::vector<zc> BS, BB;  // maxL x maxL: B^H S, B^H B
  std::vector<zc> Cp;      // -B^H b
  double xx = 0.0;         // b^H b
  std::vector<std::vector<zc>> beta;
  std::vector<double> rnorm;
  std::vector<char> conv;
  bool done = false;
  int iters = 0;
  double best = 1e300;     // best max-residual so far and its iteration (stagnation test)
  int best_it = 0;
  // anchored residuals (refinement): r0_q (FP32 rows, one per shift) at the coefficients beta0
  void* R0 = nullptr;
  void* Sa = nullptr;      // FP32 mirror of S for the anchored passes (null: they read the FP64 rows)
  std::vector<std::vector<zc>> beta0;
  bool anchor_ok = false;
};

// Orthonormal vectors spanning the columns cols (each of length L): Gram-Schmidt with column
// pivoting, stopping at kmax vectors or when the largest remaining column is below cut times the
// first.  Each new vector is orthogonalised against the ones before it again (two passes): the
// last directions come from columns reduced to ~cut of their size, whose one-pass projections
// would lose orthogonality at eps / cut.  cols is overwritten.  weights (when not null) receives,
// per vector, the norm of its pivot column relative to the first: a bound on the component of any
// column along that vector relative to the largest column.
std::vector<std::vector<zc>> pivoted_orthonormal(std::vector<std::vector<zc>>& cols, int L, double cut, int kmax,
                                                 std::vector<double>* weights = nullptr) {
  const int ns = (int)cols.size();
  std::vector<std::vector<zc>> Q;
  std::vector<char> used(ns, 0);
  double first = -1.0;
  auto dot = [&](const std::vector<zc>& a, const std::vector<zc>& b) {
    zc d(0);
    for (int i = 0; i < L; ++i) d += std::conj(a[i]) * b[i];
    return d;
  };
  while ((int)Q.size() < kmax) {
    int best = -1;
    double bn = 0.0;
    for (int q = 0; q < ns; ++q) {
      if (used[q]) continue;
      double nn = 0.0;
      for (int i = 0; i < L; ++i) nn += std::norm(cols[q][i]);
      if (nn > bn) { bn = nn; best = q; }
    }
    if (best < 0) break;
    if (first < 0) first = std::sqrt(bn);
    if (std::sqrt(bn) <= cut * first) break;
    used[best] = 1;
    std::vector<zc> qv = cols[best];
    for (auto& u : Q) {   // second pass against the earlier vectors
      const zc d = dot(u, qv);
      for (int i = 0; i < L; ++i) qv[i] -= d * u[i];
    }
    double nrm = 0.0;
    for (int i = 0; i < L; ++i) nrm += std::norm(qv[i]);
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0)) continue;
    for (int i = 0; i < L; ++i) qv[i] /= nrm;
    for (int q = 0; q < ns; ++q) {
      if (used[q]) continue;
      const zc d = dot(qv, cols[q]);
      for (int i = 0; i < L; ++i) cols[q][i] -= d * qv[i];
    }
    Q.push_back(qv);
    if (weights) weights->push_back(std::sqrt(bn) / first);
  }
  return Q;
}

// Orthonormal directions (in the coefficient space of the trial vectors) spanning the solutions
// [beta_1 ... beta_ns] of all shifts (pivoted_orthonormal).
std::vector<std::vector<zc>> solution_directions(const System& s, double cut, int kmax) {
  const int L = s.L, ns = (int)s.z.size();
  std::vector<std::vector<zc>> cols(ns, std::vector<zc>(L));
  for (int q = 0; q < ns; ++q)
    for (int i = 0; i < L; ++i) cols[q][i] = s.beta[q][i];
  return pivoted_orthonormal(cols, L, cut, kmax);
}

// Thick restart: compress the trial space onto the span of the current solutions of all shifts
// (QR with column pivoting of the coefficient matrix [beta_1 ... beta_ns], at most kmax columns).
// Sigma vectors transform with the basis (S' = S Q), so no sigma is recomputed.
void restart(Ctx& c, System& s, int maxL, int kmax) {
  const int64_t N = c.N;
  const int L = s.L, ns = (int)s.z.size();
  const std::vector<std::vector<zc>> Q = solution_directions(s, 1e-13, kmax);
  const int kk = (int)Q.size();
  CCLR_REQUIRE(kk >= 1, CCLR_E_NOCONV, "Davidson restart: empty solution space");
  {
    // B' = B Q and S' = S Q, kVecMatOut columns per pass over the old vectors
    Scope sc(c.ws);
    cplx* tmp = c.ws.cplxs((int64_t)kk * N);
    std::vector<zc> W((size_t)L * kk);
    for (int j = 0; j < L; ++j)
      for (int a = 0; a < kk; ++a) W[(size_t)j * kk + a] = Q[a][j];
    for (cplx* X : {s.B, s.S}) {
      combine(c, rows(c, X, L), kk, W, tmp);
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
  congr(s.BB);
  auto vec = [&](std::vector<zc>& v) {     // v' = Q^H v
    std::vector<zc> out(maxL, zc(0));
    for (int a = 0; a < kk; ++a)
      for (int i = 0; i < L; ++i) out[a] += std::conj(Q[a][i]) * v[i];
    v.swap(out);
  };
  vec(s.Cp);
  for (int q = 0; q < ns; ++q) vec(s.beta[q]);   // beta in the new basis (re-solved next iteration)
  s.L = kk;
}

// Projects the nt candidate corrections R (device, nt x N; overwritten) against the trial space
// B[0..L) with two classical Gram-Schmidt passes (R -= B (B^H R), twice: the basis stays
// orthonormal to working precision, so that coefficient-space compressions of the solutions are
// compressions in the vector space), then appends up to kmax of them to B[L..]: Gram-Schmidt
// among the candidates in their own Gram metric, in the given order; a direction is kept only if
// at least 1% of its norm before projection (pre2: squared norms) lies outside the trial space
// and the directions kept before it.  Returns the number appended.  cdev holds >= L * nt
// coefficients.
int add_corrections(Ctx& c, cplx* B, int L, cplx* R, int nt, const double* pre2, int kmax, cplx* cdev,
                    double* vscr, const void* Bf = nullptr, void* Rf = nullptr) {
  const int64_t N = c.N, Np = N + (N & 1);
  if (kmax <= 0 || nt <= 0) return 0;
  // With mirrors the projection runs in FP32 arithmetic whatever the solve's vector arithmetic:
  // the corrections are only directions (B^H B enters the Galerkin matrices exactly, so a basis
  // orthogonal to FP32 level is enough).
  struct Arith32 {
    Ctx& c;
    bool old;
    Arith32(Ctx& cc, bool on) : c(cc), old(cc.L.fast32) { if (on) c.L.fast32 = true; }
    ~Arith32() { c.L.fast32 = old; }
  };
  for (int pass = 0; pass < 2 && L > 0; ++pass) {
    Arith32 a32(c, Bf && Rf);
    std::vector<zc> g;
    if (Bf && Rf) {   // B^H R from the FP32 mirrors (R mirrored here)
      for (int t = 0; t < nt; ++t) to_f32(c.L, R + (int64_t)t * N, (float2*)Rf + (int64_t)t * Np, N);
      Rows b, r;
      b.add(reinterpret_cast<const cplx*>(Bf), L, Np);
      r.add(reinterpret_cast<const cplx*>(Rf), nt, Np);
      gram_host(c, b, r, true, g, true);
    } else {
      gram_host(c, rows(c, B, L), rows(c, R, nt), true, g);
    }
    for (auto& x : g) x = -x;
    to_dev(c, g.data(), cdev, (int64_t)L * nt);
    VecMat a;
    if (Bf) a.X.add(reinterpret_cast<const cplx*>(Bf), L, Np);
    else a.X = rows(c, B, L);
    a.x32 = Bf != nullptr;
    a.m = nt;
    a.C = cdev;
    a.Y = R;
    a.ldy = N;
    a.acc = true;
    vecmat(c.L, N, a, vscr);
  }
  std::vector<zc> RR;
  gram_host(c, rows(c, R, nt), rows(c, R, nt), true, RR);
  auto ip = [&](const std::vector<zc>& u, const std::vector<zc>& v) {   // u^H RR v
    zc acc(0);
    for (int i = 0; i < nt; ++i) {
      zc r(0);
      for (int j = 0; j < nt; ++j) r += RR[(size_t)i * nt + j] * v[j];
      acc += std::conj(u[i]) * r;
    }
    return acc;
  };
  std::vector<std::vector<zc>> T;
  for (int t = 0; t < nt && (int)T.size() < kmax; ++t) {
    std::vector<zc> v(nt, zc(0));
    v[t] = 1.0;
    for (int pass = 0; pass < 2; ++pass)
      for (auto& u : T) {
        const zc d = ip(u, v);
        for (int i = 0; i < nt; ++i) v[i] -= d * u[i];
      }
    const double n2 = ip(v, v).real();
    if (!(n2 > 0.0) || std::sqrt(n2) < 1e-2 * std::sqrt(std::max(0.0, pre2[t]))) continue;
    for (auto& x : v) x /= std::sqrt(n2);
    T.push_back(v);
  }
  const int kk = (int)T.size();
  if (kk == 0) return 0;
  std::vector<zc> W((size_t)nt * kk);
  for (int j = 0; j < nt; ++j)
    for (int a = 0; a < kk; ++a) W[(size_t)j * kk + a] = T[a][j];
  combine(c, rows(c, R, nt), kk, W, B + (int64_t)L * N);
  return kk;
}

// Solve (Op - z) x = -b for every system and shift.  Op(nvec, in, out) acts on N-vectors.
// A system that enters with L > 0 starts from its first L trial vectors (their sigma vectors are
// formed in the first iteration); otherwise from the preconditioned right-hand side.
//
// Per iteration and right-hand side, every pass over the N-vectors is one multi-output kernel:
//   Gram:      B^H [S_new | B_new | b] and S_old^H B_new (the Galerkin matrices B^H S, B^H B)
//   residuals: r_q = (S - z_q B) beta_q + b for up to 16 open shifts per pass (norms only)
//   candidates: delta_q = -(D - z_q)^{-1} r_q for the worst shifts, one pass
//   projection: delta -= B (B^H delta), one classical Gram-Schmidt pass; the basis need not be
//              orthonormal to working precision because B^H B enters the Galerkin matrices
//   selection: Gram-Schmidt among the candidates in their own Gram metric, worst first
//
// coarse: the corrections added after the first iteration are rounded to the coarse grid of their
// largest element (round_coarse: two digits in every view), and the sigma products treat them as
// such (the FP64-class contractions then need 9 instead of 15 digit products on the trial-vector
// operands).  The rounding only changes which vectors span the space; every sigma vector is the
// exact product of the stored vector.  The starting space keeps every digit: rounding a restart
// space would throw away the accuracy it carries.
// anchored (FP64-arithmetic solves that start from an accurate space, i.e. the refinement): the
// residuals of later iterations are r_q = r0_q + (S - z_q B)(beta_q - beta0_q).  The anchor r0_q is
// formed once in float-float after the first subspace solve (and again after a thick restart) and
// kept as FP32 rows (|r0| is near the mixed phase's floor, so FP32 storage errs at ~1e-11 of the
// right-hand side); the increment has coefficients of the size of the corrections and is formed in
// FP32 arithmetic from the FP64 rows (HBM-bound instead of float-float compute-bound).  Without
// device memory for the anchors the float-float passes are kept.
void davidson(Ctx& c, std::vector<System>& sys, const std::function<void(int, const cplx*, cplx*)>& Op,
              int maxL, double tol, bool coarse = false, bool anchored = false) {
  static const bool verbose = std::getenv("CCLR_VERBOSE") != nullptr;
  Fast32 f32(c);
  const bool mixed = mixed_precision(c.opt.precision);
  const int64_t N = c.N;
  const int kMaxNew = 4;   // new trial vectors per right-hand side and iteration (worst shifts first)
  const int kTry = 8;      // candidate corrections formed per right-hand side and iteration
  CCLR_REQUIRE(2 * maxL <= kVecMatMaxRows, CCLR_E_ARG, "max_subspace too large");
  Scope sc(c.ws);
  double* vscr = (double*)c.ws.alloc(sizeof(double) * vecmat_scratch_doubles());
  cplx* cdev = c.ws.cplxs((int64_t)2 * maxL * kVecMatOut);
  cplx* zdev = c.ws.cplxs(kVecMatOut);
  double* n2dev = (double*)c.ws.alloc(sizeof(double) * kVecMatOut);
  cplx* R = c.ws.cplxs((int64_t)kTry * N);
  unsigned* rscr = (unsigned*)c.ws.alloc(sizeof(unsigned));
  auto round_rows = [&](cplx* X, int r0, int nr) {
    if (coarse)
      for (int r = r0; r < r0 + nr; ++r) round_coarse(c.L, X + (int64_t)r * N, N, rscr);
  };
  // coefficients of r_q = S beta_q - z_q B beta_q over the rows [S | B]
  auto resid_coef = [&](const System& s, const std::vector<int>& qs, size_t g0, int m) {
    const int L = s.L;
    std::vector<zc> C((size_t)2 * L * m);
    for (int t = 0; t < m; ++t) {
      const int q = qs[g0 + t];
      for (int j = 0; j < L; ++j) {
        C[(size_t)j * m + t] = s.beta[q][j];
        C[(size_t)(L + j) * m + t] = -s.z[q] * s.beta[q][j];
      }
    }
    to_dev(c, C.data(), cdev, (int64_t)2 * L * m);
  };
  // FP32 mirrors of the trial space in the tensor-core modes; row stride Np (even, as the Gram
  // kernel's 16-byte chunk copies need)
  const int64_t Np = N + (N & 1);
  auto m32 = [&](const void* p, int r0, int nr) {   // rows [r0, r0 + nr) of a mirror
    Rows r;
    r.add(reinterpret_cast<const cplx*>((const float2*)p + (int64_t)r0 * Np), nr, Np);
    return r;
  };
  auto SB = [&](const System& s) {
    return s.Sf ? m32(s.Sf, 0, s.L).add(reinterpret_cast<const cplx*>(s.Bf), s.L, Np)
                : Rows().add(s.S, s.L, N).add(s.B, s.L, N);
  };
  // Mixed modes mirror B, S and b (every FP32-arithmetic pass reads them); FP64-arithmetic solves
  // mirror B alone, for the FP32 projection of new corrections (residuals, candidates and
  // Galerkin blocks stay on the FP64 rows).
  const bool mirrors = c.L.fast32;
  for (auto& s : sys) {
    s.Bf = c.ws.alloc(sizeof(float2) * (size_t)maxL * (size_t)Np);
    s.Sf = mirrors ? c.ws.alloc(sizeof(float2) * (size_t)maxL * (size_t)Np) : nullptr;
    s.bf = mirrors ? c.ws.alloc(sizeof(float2) * (size_t)Np) : nullptr;
    if (s.bf) to_f32(c.L, s.rhs, s.bf, N);
  }
  void* Rf = c.ws.alloc(sizeof(float2) * (size_t)kTry * (size_t)Np);
  auto mirror = [&](const cplx* X, void* Xf, int r0, int nr) {   // rows [r0, r0 + nr) of B or S
    if (Xf)
      for (int r = r0; r < r0 + nr; ++r) to_f32(c.L, X + (int64_t)r * N, (float2*)Xf + (int64_t)r * Np, N);
  };
  // anchors
  struct AnchorMem {
    std::vector<System>& sys;
    ~AnchorMem() {
      for (auto& s : sys) {
        if (s.R0) { cudaFree(s.R0); s.R0 = nullptr; }
        if (s.Sa) { cudaFree(s.Sa); s.Sa = nullptr; }
      }
    }
  } anchor_mem{sys};
  struct Arith32Scope {   // FP32 arithmetic for the anchored passes
    Ctx& c;
    bool old;
    explicit Arith32Scope(Ctx& cc) : c(cc), old(cc.L.fast32) { c.L.fast32 = true; }
    ~Arith32Scope() { c.L.fast32 = old; }
  };
  // Both are taken from free device memory, not the workspace (the sigma products' temporaries
  // live there); the S mirror only while ample memory stays free for the tensor-core slice cache.
  for (auto& s : sys) {
    s.anchor_ok = false;
    s.R0 = s.Sa = nullptr;
    if (anchored && !mixed) {
      if (cudaMalloc(&s.R0, sizeof(float2) * (size_t)Np * s.z.size()) != cudaSuccess) {
        cudaGetLastError();
        s.R0 = nullptr;   // float-float passes
        continue;
      }
      const size_t sa_bytes = sizeof(float2) * (size_t)maxL * (size_t)Np;
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr > sa_bytes + ((size_t)16 << 30) &&
          cudaMalloc(&s.Sa, sa_bytes) != cudaSuccess) {
        cudaGetLastError();
        s.Sa = nullptr;
      }
    }
  }
  // coefficients of the increment (beta_q - beta0_q) over the rows [S | B]
  auto anchored_coef = [&](const System& s, const std::vector<int>& qs, size_t g0, int m) {
    const int L = s.L;
    std::vector<zc> C((size_t)2 * L * m);
    for (int t = 0; t < m; ++t) {
      const int q = qs[g0 + t];
      for (int j = 0; j < L; ++j) {
        const zc d = s.beta[q][j] - s.beta0[q][j];
        C[(size_t)j * m + t] = d;
        C[(size_t)(L + j) * m + t] = -s.z[q] * d;
      }
    }
    to_dev(c, C.data(), cdev, (int64_t)2 * L * m);
  };
  auto anchored_args = [&](const System& s, const std::vector<int>& qs, size_t g0, int m, VecMat& a) {
    anchored_coef(s, qs, g0, m);
    if (s.Sa) {
      a.X = m32(s.Sa, 0, s.L).add(reinterpret_cast<const cplx*>(s.Bf), s.L, Np);
      a.x32 = true;
    } else {
      a.X = Rows().add(s.S, s.L, N).add(s.B, s.L, N);
      a.x32 = false;
    }
    a.m = m;
    a.C = cdev;
    a.add = nullptr;
    a.addq = s.R0;
    a.ldadd = Np;
    for (int t = 0; t < m; ++t) a.arow[t] = qs[g0 + t];
  };
  // the anchor of every shift (float-float pass; also this iteration's residual norms)
  auto compute_anchor = [&](System& s) {
    std::vector<int> all(s.z.size());
    for (size_t q = 0; q < all.size(); ++q) all[q] = (int)q;
    Scope s3(c.ws);
    cplx* Yt = c.ws.cplxs((int64_t)kVecMatOut * N);
    for (size_t g0 = 0; g0 < all.size(); g0 += kVecMatOut) {
      const int m = (int)std::min<size_t>(kVecMatOut, all.size() - g0);
      resid_coef(s, all, g0, m);
      VecMat a;
      a.X = SB(s);
      a.x32 = s.Sf != nullptr;
      a.m = m;
      a.C = cdev;
      a.add = s.rhs;
      a.Y = Yt;
      a.ldy = N;
      a.norm2 = n2dev;
      vecmat(c.L, N, a, vscr);
      double h[kVecMatOut];
      CCLR_CK(cudaMemcpyAsync(h, n2dev, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream));
      for (int t = 0; t < m; ++t)
        to_f32(c.L, Yt + (int64_t)t * N, (float2*)s.R0 + (int64_t)all[g0 + t] * Np, N);
      c.sync();
      for (int t = 0; t < m; ++t) s.rnorm[all[g0 + t]] = std::sqrt(std::max(0.0, h[t]));
    }
    s.beta0 = s.beta;
    for (auto& b0 : s.beta0)   // coefficients of later vectors start from zero
      for (int j = s.L; j < (int)b0.size(); ++j) b0[j] = zc(0);
    s.anchor_ok = true;
  };
  auto residual_norms = [&](System& s, const std::vector<int>& qs) {
    for (size_t g0 = 0; g0 < qs.size(); g0 += kVecMatOut) {
      const int m = (int)std::min<size_t>(kVecMatOut, qs.size() - g0);
      VecMat a;
      std::unique_ptr<Arith32Scope> a32;
      if (s.anchor_ok) {
        anchored_args(s, qs, g0, m, a);
        a32.reset(new Arith32Scope(c));
      } else {
        resid_coef(s, qs, g0, m);
        a.X = SB(s);
        a.x32 = s.Sf != nullptr;
        a.m = m;
        a.C = cdev;
        a.add = s.rhs;
      }
      a.norm2 = n2dev;
      vecmat(c.L, N, a, vscr);
      double h[kVecMatOut];
      CCLR_CK(cudaMemcpyAsync(h, n2dev, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream));
      c.sync();
      for (int t = 0; t < m; ++t) s.rnorm[qs[g0 + t]] = std::sqrt(std::max(0.0, h[t]));
    }
  };
  for (auto& s : sys) {
    s.BS.assign((size_t)maxL * maxL, zc(0));
    s.BB.assign((size_t)maxL * maxL, zc(0));
    s.Cp.assign(maxL, zc(0));
    s.xx = norm2(c, s.rhs);
    s.beta.assign(s.z.size(), std::vector<zc>(maxL, zc(0)));
    s.rnorm.assign(s.z.size(), 1e300);
    s.conv.assign(s.z.size(), 0);
    s.done = false;
    s.best = 1e300;
    s.best_it = 0;
    CCLR_REQUIRE(s.L >= 0 && s.L <= maxL, CCLR_E_ARG, "Davidson: starting space larger than max_subspace");
    if (s.L == 0) {
      // start: b / D, normalized (preconditioned right-hand side at z = 0)
      div_shift(c.L, N, s.rhs, c.Dpre ? c.Dpre : c.D, cx(0), cx(1), s.B);
      const double nb = std::sqrt(norm2(c, s.B));
      CCLR_REQUIRE(nb > 0.0, CCLR_E_ARG, "zero right-hand side");
      scale_vec(c.L, N, cx(1.0 / nb), s.B);
      s.L = 1;
    }
    mirror(s.B, s.Bf, 0, s.L);
  }
  std::vector<int> fresh(sys.size());   // new vectors at the end of each basis
  for (size_t k = 0; k < sys.size(); ++k) fresh[k] = sys[k].L;
  Phases ph("davidson");
  for (int it = 1; it <= c.opt.maxit; ++it) {
    ph.mark(c, "sigma");
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
      struct CoarseFlag {   // the sigma products see coarse inputs while this is alive
        Ctx& c;
        bool old;
        CoarseFlag(Ctx& cc, bool on) : c(cc), old(cc.coarse_sigma) { c.coarse_sigma = on; }
        ~CoarseFlag() { c.coarse_sigma = old; }
      } cf(c, coarse && it > 1);
      for (int q0 = 0; q0 < total; q0 += bmax) {
        const int nb = std::min(bmax, total - q0);
        Op(nb, in + (int64_t)q0 * N, out + (int64_t)q0 * N);
      }
      c.sync();
      c.stats.sigma_seconds += now() - t0;
      q = 0;
      for (size_t k = 0; k < sys.size(); ++k) {
        for (int j = 0; j < fresh[k]; ++j, ++q)
          copy_vec(c.L, N, out + (int64_t)q * N, sys[k].S + (int64_t)(sys[k].L - fresh[k] + j) * N);
        mirror(sys[k].S, sys[k].Sf, sys[k].L - fresh[k], fresh[k]);
        mirror(sys[k].S, sys[k].Sa, sys[k].L - fresh[k], fresh[k]);
      }
    }
    bool all_done = true;
    for (size_t k = 0; k < sys.size(); ++k) {
      System& s = sys[k];
      if (s.done) continue;
      const int L0 = s.L - fresh[k], f = fresh[k];
      // ---- Galerkin matrices: new columns of B^H S and B^H B, new rows of B^H S, B^H b
      ph.mark(c, "gram");
      if (f > 0) {
        std::vector<zc> g;
        const cplx* Bn = s.B + (int64_t)L0 * N;
        const cplx* Sn = s.S + (int64_t)L0 * N;
        const int ny = 2 * f;
        if (s.Sf)
          gram_host(c, m32(s.Bf, 0, s.L), m32(s.Sf, L0, f).add(reinterpret_cast<const cplx*>((const float2*)s.Bf + (int64_t)L0 * Np), f, Np),
                    true, g, true);
        else
          gram_host(c, rows(c, s.B, s.L), Rows().add(Sn, f, N).add(Bn, f, N), true, g);
        for (int i = 0; i < s.L; ++i) {
          for (int j = 0; j < f; ++j) {
            s.BS[(size_t)i * maxL + L0 + j] = g[(size_t)i * ny + j];
            const zc bb = g[(size_t)i * ny + f + j];
            s.BB[(size_t)i * maxL + L0 + j] = bb;
            s.BB[(size_t)(L0 + j) * maxL + i] = std::conj(bb);
          }
        }
        // S_old^H B_new and b^H B_new in one pass (the old rows of B^H b are unchanged: b is fixed
        // and a restart transforms them with the basis)
        Rows sb;
        if (s.Sf) {
          if (L0 > 0) sb = m32(s.Sf, 0, L0);
          sb.add(reinterpret_cast<const cplx*>(s.bf), 1, Np);
          gram_host(c, sb, m32(s.Bf, L0, f), true, g, true);
        } else {
          if (L0 > 0) sb.add(s.S, L0, N);
          sb.add(s.rhs, 1, N);
          gram_host(c, sb, rows(c, Bn, f), true, g);
        }
        for (int i = 0; i < L0; ++i)
          for (int j = 0; j < f; ++j) s.BS[(size_t)(L0 + j) * maxL + i] = std::conj(g[(size_t)i * f + j]);
        for (int j = 0; j < f; ++j) s.Cp[L0 + j] = -std::conj(g[(size_t)L0 * f + j]);
      }
      fresh[k] = 0;
      const int L = s.L;
      // mixed modes: sigma carries ~1e-5 relative error at long K (FP32 accumulation), so the
      // mixed phase stops at mixed_floor() of |b| (the refinement phase, or the caller with
      // refine = 0, takes it from there)
      const double tol_s = mixed ? std::max(tol, mixed_floor(c) * std::sqrt(s.xx)) : tol;
      // ---- subspace solves (B^H S - z B^H B) beta = -B^H b for every shift
      ph.mark(c, "subspace");
      for (size_t q = 0; q < s.z.size(); ++q) {
        const zc z = s.z[q];
        std::vector<zc> G((size_t)L * L), rhs(s.Cp.begin(), s.Cp.begin() + L);
        for (int i = 0; i < L; ++i)
          for (int j = 0; j < L; ++j) G[(size_t)i * L + j] = s.BS[(size_t)i * maxL + j] - z * s.BB[(size_t)i * maxL + j];
        zsolve(L, G, rhs);
        for (int i = 0; i < L; ++i) s.beta[q][i] = rhs[i];
      }
      bool have_all = false;   // the anchor pass gave every shift's norm at this iteration
      if (s.R0 && !s.anchor_ok) {
        ph.mark(c, "anchor");
        compute_anchor(s);
        have_all = true;
      }
      // ---- residual norms of the open shifts; once all are below the target, the shifts
      // locked earlier are checked again at the final trial space.  With FP64 vector arithmetic
      // (FP64 mode, refinement) a pass costs about one DFMA per complex element and output row,
      // so only the kTry open shifts with the largest last norm are recomputed each iteration;
      // every open shift is checked once those are below the target.  Anchored residuals (FP32
      // passes) are cheap enough to refresh every open shift's norm each iteration.
      std::vector<int> open, locked;
      for (size_t q = 0; q < s.z.size(); ++q) (s.conv[q] ? locked : open).push_back((int)q);
      std::vector<std::pair<double, int>> order;
      ph.mark(c, "norms");
      std::vector<int> check = open;
      if (have_all) {
        // norms already fresh
      } else if (!mixed && !s.anchor_ok && (int)open.size() > kTry && it > 1) {
        std::vector<std::pair<double, int>> last;
        for (int q : open) last.push_back({s.rnorm[q], q});
        std::partial_sort(last.begin(), last.begin() + kTry, last.end(), [](auto& a, auto& b) { return a.first > b.first; });
        check.clear();
        for (int t = 0; t < kTry; ++t) check.push_back(last[t].second);
        residual_norms(s, check);
        bool tracked_done = true;
        for (int q : check) tracked_done = tracked_done && s.rnorm[q] < tol_s;
        if (tracked_done) {
          check = open;
          residual_norms(s, check);
        }
      } else {
        residual_norms(s, check);
      }
      for (int q : check) s.conv[q] = s.rnorm[q] < tol_s;
      for (int q : open)
        if (!s.conv[q]) order.push_back({s.rnorm[q], q});
      if (order.empty() && !locked.empty()) {
        if (!have_all) residual_norms(s, locked);
        for (int q : locked) {
          s.conv[q] = s.rnorm[q] < tol_s;
          if (!s.conv[q]) order.push_back({s.rnorm[q], q});
        }
      }
      s.iters = it;
      if (verbose)
        std::fprintf(stderr, "[cclr] davidson it %d rhs %zu L %d unconverged %zu/%zu max|r| %.3e tol %.1e\n", it, k, L,
                     order.size(), s.z.size(), order.empty() ? 0.0 : std::max_element(order.begin(), order.end())->first,
                     tol_s);
      if (!order.empty() && mixed) {
        // mixed modes: accept a stagnating solve whose residuals are all within 5x the floor
        double mx = 0.0;
        for (auto& pr : order) mx = std::max(mx, pr.first);
        if (mx < 0.8 * s.best) { s.best = mx; s.best_it = it; }
        if (it - s.best_it >= 4 && mx < 5.0 * tol_s) order.clear();
      }
      if (order.empty()) {
        s.done = true;
        continue;
      }
      all_done = false;
      std::sort(order.begin(), order.end(), [](auto& a, auto& b) { return a.first > b.first; });
      ph.mark(c, "restart");
      if (s.L + kMaxNew > maxL) {
        restart(c, s, maxL, maxL - 2 * kMaxNew);
        mirror(s.B, s.Bf, 0, s.L);
        mirror(s.S, s.Sf, 0, s.L);
        mirror(s.S, s.Sa, 0, s.L);
        s.anchor_ok = false;   // new basis: anchored again after the next subspace solve
      }
      // ---- preconditioned residuals of kTry shifts, one pass.  The worst shift first, then
      // greedily the shift whose norm times its distance (in z) to the shifts taken is largest:
      // the solutions vary smoothly with z, so corrections of neighbouring shifts are nearly
      // parallel, and spreading them over the shift set spans more of all shifts' errors.
      ph.mark(c, "candidates");
      const int nt = std::min<int>(kTry, (int)order.size());
      std::vector<int> qs(nt);
      std::vector<zc> zq(nt);
      {
        std::vector<char> taken(order.size(), 0);
        for (int t = 0; t < nt; ++t) {
          int bi = 0;
          double bv = -1.0;
          for (size_t i = 0; i < order.size() && t > 0; ++i) {
            if (taken[i]) continue;
            double dmin = 1e300;
            for (int p = 0; p < t; ++p) dmin = std::min(dmin, std::abs(s.z[order[i].second] - s.z[qs[p]]));
            const double v = order[i].first * dmin;
            if (v > bv) { bv = v; bi = (int)i; }
          }
          taken[bi] = 1;
          qs[t] = order[bi].second;
          zq[t] = s.z[qs[t]];
        }
      }
      to_dev(c, zq.data(), zdev, nt);
      double pre2[kVecMatOut];
      {
        VecMat a;
        std::unique_ptr<Arith32Scope> a32;
        if (s.anchor_ok) {
          anchored_args(s, qs, 0, nt, a);
          a32.reset(new Arith32Scope(c));
        } else {
          resid_coef(s, qs, 0, nt);
          a.X = SB(s);
          a.x32 = s.Sf != nullptr;
          a.m = nt;
          a.C = cdev;
          a.add = s.rhs;
        }
        a.Y = R;
        a.ldy = N;
        a.D = c.Dpre ? c.Dpre : c.D;
        a.z = zdev;
        a.norm2 = n2dev;
        a.norm_y = true;
        vecmat(c.L, N, a, vscr);
        CCLR_CK(cudaMemcpyAsync(pre2, n2dev, sizeof(double) * nt, cudaMemcpyDeviceToHost, c.stream));
        c.sync();
      }
      // ---- project out the trial space and append the new directions
      ph.mark(c, "project");
      const int kk = add_corrections(c, s.B, s.L, R, nt, pre2, std::min(kMaxNew, maxL - s.L), cdev, vscr, s.Bf, Rf);
      round_rows(s.B, s.L, kk);
      mirror(s.B, s.Bf, s.L, kk);
      if (kk == 0)
        throw Error(CCLR_E_NOCONV, "Davidson stagnated: residual " + std::to_string(order.front().first) +
                                       " above tolerance " + std::to_string(tol_s) + " with no new direction");
      s.L += kk;
      fresh[k] = kk;
    }
    ph.mark(c, "other");
    // the largest current residual over all systems and shifts (the final one at exit)
    c.stats.max_residual = 0.0;
    for (auto& s : sys)
      for (double r : s.rnorm) c.stats.max_residual = std::max(c.stats.max_residual, r);
    if (all_done) return;
  }
  throw Error(CCLR_E_NOCONV, "Davidson did not converge within maxit iterations");
}

void restart_from_solutions(Ctx& c, std::vector<System>& sys, int maxL, std::vector<cplx*>* bases,
                            std::vector<cplx*>* sigs);

// FP64 iterative refinement of systems solved in a mixed mode (cclr_options.refine): every system
// restarts from the compressed span of its mixed-precision solutions, U = B Q (directions above
// 1e-10 of the largest, at most 16), whose sigma vectors are formed again in the FP64-class
// tensor-core mode from every digit, and the Davidson iteration continues there with FP64-class
// sigma products of coarse corrections and FP64 residuals, norms and projections until every
// residual is below tol.  The phase-1 arrays of each system (B, S) are freed and replaced;
// bases[k] / sigs[k] (when not null) are updated to the new arrays.
void refine_systems(Ctx& c, std::vector<System>& sys, const std::function<void(int, const cplx*, cplx*)>& Op, int maxL,
                    double tol, std::vector<cplx*>* bases, std::vector<cplx*>* sigs) {
  PrecisionScope exact(c, CCLR_TC_F64);
  const double t0 = now();
  const long v0 = c.stats.sigma_vectors;
  restart_from_solutions(c, sys, maxL, bases, sigs);
  davidson(c, sys, Op, maxL, tol, true, true);
  c.stats.refine_vectors += c.stats.sigma_vectors - v0;
  c.stats.refine_seconds += now() - t0;
}

// Replaces every system's trial space by the compressed span of its solutions (see
// refine_systems); the sigma vectors of the new space are formed by the next Davidson call.
void restart_from_solutions(Ctx& c, std::vector<System>& sys, int maxL, std::vector<cplx*>* bases,
                            std::vector<cplx*>* sigs) {
  const int64_t N = c.N;
  for (size_t k = 0; k < sys.size(); ++k) {
    System& s = sys[k];
    const std::vector<std::vector<zc>> Q = solution_directions(s, 1e-10, std::max(1, std::min(16, maxL / 2)));
    const int r = (int)Q.size();
    CCLR_REQUIRE(r >= 1, CCLR_E_NOCONV, "refinement: empty solution space");
    std::vector<zc> W((size_t)s.L * r);
    for (int j = 0; j < s.L; ++j)
      for (int a = 0; a < r; ++a) W[(size_t)j * r + a] = Q[a][j];
    cplx* B2 = c.dalloc((int64_t)maxL * N);
    combine(c, rows(c, s.B, s.L), r, W, B2);
    c.dfree(s.B);
    c.dfree(s.S);
    cplx* S2 = c.dalloc((int64_t)maxL * N);
    s.B = B2;
    s.S = S2;
    s.L = r;
    if (bases) (*bases)[k] = B2;
    if (sigs) (*sigs)[k] = S2;
  }
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
  int its = 0;
  try {
    auto op = [&](int nv, const cplx* in, cplx* out) { sigma_left(c, nv, in, out); };
    davidson(c, sys, op, maxL, c.opt.ground_tol);
    its = sys[0].iters;
    if (refining(c)) {
      refine_systems(c, sys, op, maxL, c.opt.ground_tol, nullptr, nullptr);
      its += sys[0].iters;
    }
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
  cleanup();
  c.have_lambda = true;
  c.named.erase("F.ready");
  return its;
}

// ------------------------------------------------------------------------------ response
// Frees the device arrays of the last linear-response solve.
void release_response(Ctx& c) {
  ResponseData& rd = c.rd;
  for (auto p : rd.ops_dev) c.dfree(p);
  for (auto p : rd.xi) c.dfree(p);
  for (auto p : rd.eta) c.dfree(p);
  for (auto p : rd.basis) c.dfree(p);
  for (auto p : rd.sig) c.dfree(p);
  rd = ResponseData();
}

void lr_solve(Ctx& c, int n_ops, const cplx* ops_host, int n_freq, const double* omegas, double gamma,
              int* iters_out) {
  release_response(c);
  ResponseData& rd = c.rd;
  const int64_t N = c.N, n = c.n;
  const int maxL = std::max(8, c.opt.max_subspace);
  Phases ph("lr_solve");
  ph.mark(c, "setup");
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
    CCLR_CK(cudaMemcpyAsync(X, ops_host + (int64_t)k * n * n, sizeof(cplx) * n * n, cudaMemcpyDefault, c.stream));
    rd.ops_dev.push_back(X);
    PrecisionScope exact(c, exact_precision(c));   // the right-hand sides define the answer
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
  ph.mark(c, "davidson");
  auto op = [&](int nv, const cplx* in, cplx* out) { sigma_right(c, nv, in, out); };
  davidson(c, sys, op, maxL, c.opt.tol);
  std::vector<int> its1(n_ops);
  for (int k = 0; k < n_ops; ++k) its1[k] = sys[k].iters;
  rd.refined = refining(c);
  if (rd.refined) {
    ph.mark(c, "refine");
    refine_systems(c, sys, op, maxL, c.opt.tol, &rd.basis, &rd.sig);
    for (int k = 0; k < n_ops; ++k) sys[k].iters += its1[k];
  }
  ph.mark(c, "finish");
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
  ph.mark(c, "");
}

void response_function(Ctx& c, cplx* out_host) {
  ResponseData& rd = c.rd;
  CCLR_REQUIRE(rd.solved, CCLR_E_STATE, "cc_response_function before cc_lr_solve");
  // refined solutions: the Hessian products in the FP64-class mode, FP64 vector arithmetic (the
  // F term enters small components of <<X;Y>> at the 1e-6 level if formed in FP32 class)
  PrecisionScope exact(c, rd.refined ? CCLR_TC_F64 : c.opt.precision);
  Fast32 f32(c);
  const int64_t N = c.N;
  const int nop = rd.n_ops, maxL = std::max(8, c.opt.max_subspace);
  Phases ph("response_function");
  ph.mark(c, "eta.B");
  // Bilinear forms M^{xy}_{kl} = (b^x_k F) . b^y_l and E^{xy}_l = eta^x . b^y_l.  The Hessian
  // products of the trial vectors are formed in batches and contracted at once (never stored).
  std::vector<std::vector<zc>> M((size_t)nop * nop), E((size_t)nop * nop);
  for (int x = 0; x < nop; ++x)
    for (int y = 0; y < nop; ++y)
      gram_host(c, rows(c, rd.eta[x], 1), rows(c, rd.basis[y], rd.nb[y]), false, E[(size_t)x * nop + y]);
  auto beta = [&](int k, int f, int s) { return &rd.beta[k][(size_t)rd.shift_of[(size_t)f * 4 + s] * maxL]; };
  // The Hessian acts only on the solutions t^X(-z) and t^X(z*) of every frequency.  Their
  // coefficient vectors span few directions: compress them (QR with column pivoting, cutoff
  // 1e-12 of the largest in FP64 mode, 1e-10 for refined solutions; 1e-7 in the unrefined mixed
  // modes, whose sigma products carry ~1e-5 relative error) to Q_x, form the products
  // F (B^x Q_x) in batches and contract them at once:
  //   M^{xy} = (B^x Q_x F) . B^y,  (t^X F) . t^Y = gamma^T M^{xy} beta^Y,  gamma = Q_x^H beta^X.
  // Refined solutions: direction j carries at most a fraction w_j (its pivot weight) of any
  // solution, so a product error eps_p enters the F term at <= w_j eps_p of its size.  Directions
  // with w_j > 1e-4 use the FP64-class mode, 1e-6 < w_j <= 1e-4 the FP32-class split (eps ~1e-7),
  // the rest the three-product split (eps ~2e-5): every contribution stays below ~2e-11.
  const int base_prec = c.opt.precision;   // FP64-class when refined, else the solve's mode
  auto dir_prec = [&](double w) {
    if (!rd.refined) return base_prec;
    return w > 1e-4 ? (int)CCLR_TC_F64 : w > 1e-6 ? (int)CCLR_TC_BF16X6 : (int)CCLR_TC_BF16X3;
  };
  std::vector<std::vector<std::vector<zc>>> Q(nop);
  for (int x = 0; x < nop; ++x) {
    const int Lx = rd.nb[x];
    std::vector<std::vector<zc>> cols;
    for (int f = 0; f < rd.n_freq; ++f)
      for (int s : {3, 2}) cols.emplace_back(beta(x, f, s), beta(x, f, s) + Lx);
    std::vector<double> wts;
    Q[x] = pivoted_orthonormal(cols, Lx, mixed_precision(c.opt.precision) ? 1e-7 : rd.refined ? 1e-10 : 1e-12, Lx,
                               &wts);
    const int rx = (int)Q[x].size();
    for (int y = 0; y < nop; ++y) M[(size_t)x * nop + y].assign((size_t)rx * rd.nb[y], zc(0));
    const int bmax = std::max(1, std::min(c.opt.batch > 0 ? c.opt.batch : 8, rx));
    for (int q0 = 0; q0 < rx;) {
      // one batch: up to bmax consecutive directions of the same precision
      const int p = dir_prec(wts[q0]);
      int nb = 1;
      while (nb < bmax && q0 + nb < rx && dir_prec(wts[q0 + nb]) == p) ++nb;
      PrecisionScope dp(c, p);
      Scope sc(c.ws);
      cplx* yv = c.ws.cplxs((int64_t)nb * N);
      cplx* fb = c.ws.cplxs((int64_t)nb * N);
      std::vector<zc> W((size_t)Lx * nb);
      for (int l = 0; l < Lx; ++l)
        for (int j = 0; j < nb; ++j) W[(size_t)l * nb + j] = Q[x][q0 + j][l];
      ph.mark(c, "combine");
      combine(c, rows(c, rd.basis[x], Lx), nb, W, yv);
      ph.mark(c, "hessian");
      hessian_right(c, nb, yv, fb);
      ph.mark(c, "gram");
      for (int y = 0; y < nop; ++y) {
        std::vector<zc> g;
        gram_host(c, rows(c, fb, nb), rows(c, rd.basis[y], rd.nb[y]), false, g);
        auto& Mxy = M[(size_t)x * nop + y];
        for (int i = 0; i < nb; ++i)
          for (int j = 0; j < rd.nb[y]; ++j) Mxy[(size_t)(q0 + i) * rd.nb[y] + j] = g[(size_t)i * rd.nb[y] + j];
      }
      q0 += nb;
    }
    static const bool verbose = std::getenv("CCLR_VERBOSE") != nullptr;
    if (verbose) {
      int cnt[5] = {0, 0, 0, 0, 0};
      for (double w : wts) cnt[dir_prec(w)]++;
      std::fprintf(stderr, "[cclr] response_function op %d: %d Hessian directions (F64 %d, BF16X6 %d, BF16X3 %d)\n", x,
                   rx, cnt[CCLR_TC_F64], cnt[CCLR_TC_BF16X6], cnt[CCLR_TC_BF16X3]);
    }
  }
  ph.mark(c, "forms");
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

// Gradient of the CC-CC response function with respect to the operators (adjoint method).
// <<X;Y>>_z = f(z) + conj(f(-z*)), f(w) = 1/2 [eta^X t^Y(w) + eta^Y t^X(-w) + (t^X(-w) F) t^Y(w)],
// t^X(w) = -(A - w)^{-1} xi^X, is linear in X and in Y through xi and eta.  Differentiating in
// X at fixed Y (F is symmetric):
//   d f(w) = 1/2 [eta^{dX} t^Y(w) + l^Y(w) xi^{dX}],  l^Y(w) (A + w) = -(eta^Y + F t^Y(w)),
// one left solve (SI left sigma equations) per operator and shift, and the densities of
// xi_density / eta_density turn the products into matrices over X's elements:
//   G[k][s] = 1/2 [eta_density(t^k(w_s)) + xi_density(l^k(w_s))],  w_s the shift s of frequency f
//   (0: w+ig, 1: -w+ig, 2: w-ig, 3: -w-ig), so that for operator perturbations dX_x, dX_y
//   d<<X_x;X_y>> = sum G[y][0] o dX_x + conj(sum G[y][1] o dX_x) + sum G[x][3] o dX_y
//                  + conj(sum G[x][2] o dX_y)        (o: element-wise product, sum over p, q).
// out_host: n_ops x 4 matrices n x n.  Requires cc_lr_solve.
void response_gradient(Ctx& c, int f, cplx* out_host) {
  ResponseData& rd = c.rd;
  CCLR_REQUIRE(rd.solved, CCLR_E_STATE, "cclr_response_gradient before cc_lr_solve");
  CCLR_REQUIRE(f >= 0 && f < rd.n_freq, CCLR_E_ARG, "cclr_response_gradient: frequency index");
  const int64_t N = c.N, n = c.n;
  const int nop = rd.n_ops, maxL = std::max(8, c.opt.max_subspace);
  // per operator (its four shifts share one Davidson run): solution vectors t^k(w_s) and
  // right-hand sides eta^k + F t^k(w_s) (FP64-class when refined)
  std::vector<cplx*> tv, rhs, Bs, Ss;
  auto cleanup = [&]() {
    for (auto p : tv) c.dfree(p);
    for (auto p : rhs) c.dfree(p);
    for (auto p : Bs) c.dfree(p);
    for (auto p : Ss) c.dfree(p);
    tv.clear();
    rhs.clear();
    Bs.clear();
    Ss.clear();
  };
  try {
    for (int k = 0; k < nop; ++k) {
      std::vector<System> sys(4);
      {
        PrecisionScope exact(c, rd.refined ? CCLR_TC_F64 : c.opt.precision);
        Scope sc(c.ws);
        cplx* bd = c.ws.cplxs(maxL);
        for (int q = 0; q < 4; ++q) {
          cplx* t = c.dalloc(N);
          tv.push_back(t);
          const zc* beta = &rd.beta[k][(size_t)rd.shift_of[(size_t)f * 4 + q] * maxL];
          to_dev(c, beta, bd, rd.nb[k]);
          lincomb(c.L, N, rd.nb[k], rd.basis[k], N, bd, t, false);
          cplx* b = c.dalloc(N);
          rhs.push_back(b);
          hessian_right(c, 1, t, b);
          axpy(c.L, N, cx(1), rd.eta[k], b);
          System& s = sys[q];
          s.rhs = b;
          s.z = {-rd.shifts[rd.shift_of[(size_t)f * 4 + q]]};   // l (A - w_l) = -b with w_l = -w_s
          s.B = c.dalloc((int64_t)maxL * N);
          s.S = c.dalloc((int64_t)maxL * N);
          Bs.push_back(s.B);
          Ss.push_back(s.S);
        }
      }
      auto op = [&](int nv, const cplx* in, cplx* out) { sigma_left(c, nv, in, out); };
      davidson(c, sys, op, maxL, c.opt.tol);
      if (refining(c)) refine_systems(c, sys, op, maxL, c.opt.tol, &Bs, &Ss);
      {
        PrecisionScope exact(c, rd.refined ? CCLR_TC_F64 : c.opt.precision);
        Scope sc(c.ws);
        cplx* l = c.ws.cplxs(N);
        cplx* bd = c.ws.cplxs(maxL);
        cplx* D1 = c.ws.cplxs(n * n);
        cplx* D2 = c.ws.cplxs(n * n);
        for (int q = 0; q < 4; ++q) {
          const System& s = sys[q];
          to_dev(c, s.beta[0].data(), bd, s.L);
          lincomb(c.L, N, s.L, s.B, N, bd, l, false);
          eta_density(c, tv[q], D1);
          xi_density(c, l, D2);
          axpy(c.L, n * n, cx(1), D2, D1);
          scale_vec(c.L, n * n, cx(0.5), D1);
          CCLR_CK(cudaMemcpyAsync(out_host + ((size_t)4 * k + q) * n * n, D1, sizeof(cplx) * n * n,
                                  cudaMemcpyDefault, c.stream));
          c.sync();
        }
      }
      cleanup();
    }
  } catch (...) {
    cleanup();
    throw;
  }
}

// Left (adjoint) linear systems l_k (A + w) = -b_k for nrhs right-hand sides (host or device
// memory, cudaMemcpyDefault) with one shift; the Lambda equations are the case b = eta of the
// energy, w = 0.  The same Davidson (and refinement) as the Lambda solve.
void left_solve(Ctx& c, int nrhs, const cplx* rhs, zc w, cplx* out) {
  const int64_t N = c.N;
  const int maxL = std::max(8, c.opt.max_subspace);
  std::vector<System> sys(nrhs);   // refinement replaces B and S: free what the systems hold
  auto cleanup = [&]() {
    for (auto& s : sys) {
      if (s.rhs) c.dfree(const_cast<cplx*>(s.rhs));
      if (s.B) c.dfree(s.B);
      if (s.S) c.dfree(s.S);
    }
  };
  try {
    for (int k = 0; k < nrhs; ++k) {
      cplx* b = c.dalloc(N);
      sys[k].rhs = b;
      CCLR_CK(cudaMemcpyAsync(b, rhs + (int64_t)k * N, sizeof(cplx) * N, cudaMemcpyDefault, c.stream));
      sys[k].z = {-w};
      sys[k].B = c.dalloc((int64_t)maxL * N);
      sys[k].S = c.dalloc((int64_t)maxL * N);
    }
    auto op = [&](int nv, const cplx* in, cplx* o) { sigma_left(c, nv, in, o); };
    davidson(c, sys, op, maxL, c.opt.tol);
    if (refining(c)) refine_systems(c, sys, op, maxL, c.opt.tol, nullptr, nullptr);
    Scope sc(c.ws);
    cplx* bd = c.ws.cplxs(maxL);
    cplx* l = c.ws.cplxs(N);
    for (int k = 0; k < nrhs; ++k) {
      to_dev(c, sys[k].beta[0].data(), bd, sys[k].L);
      lincomb(c.L, N, sys[k].L, sys[k].B, N, bd, l, false);
      CCLR_CK(cudaMemcpyAsync(out + (int64_t)k * N, l, sizeof(cplx) * N, cudaMemcpyDefault, c.stream));
      c.sync();
    }
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
}

// CC-CI response function (Eq. CC-CI response function): no Hessian term; EOM-eta of the SI
// "Linear response" section and the ground-state multipliers lambda,
//   f(z) = 1/2 [eometa^X t^Y(z) - (lam.t^X(-z))(lam.xi^Y) + eometa^Y t^X(-z) - (lam.t^Y(z))(lam.xi^X)],
//   <<X;Y>>_z = f(z) + conj(f(-z*)),
// evaluated in the trial spaces of cc_lr_solve: t^X(w) = B^X beta^X(w).
void response_function_ci(Ctx& c, cplx* out_host) {
  ResponseData& rd = c.rd;
  CCLR_REQUIRE(rd.solved, CCLR_E_STATE, "cc_response_function_ci before cc_lr_solve");
  CCLR_REQUIRE(c.have_lambda, CCLR_E_STATE, "cc_response_function_ci needs Lambda");
  PrecisionScope exact(c, rd.refined ? CCLR_TC_F64 : c.opt.precision);
  Fast32 f32(c);
  const int64_t N = c.N;
  const int nop = rd.n_ops, maxL = std::max(8, c.opt.max_subspace);
  std::vector<std::vector<zc>> E((size_t)nop * nop), Lb(nop);
  std::vector<zc> lam_xi(nop);
  {
    Scope sc(c.ws);
    cplx* eom = c.ws.cplxs(N);
    for (int x = 0; x < nop; ++x) {
      eta_vec(c, rd.ops_dev[x], true, eom);
      for (int y = 0; y < nop; ++y)
        gram_host(c, rows(c, eom, 1), rows(c, rd.basis[y], rd.nb[y]), false, E[(size_t)x * nop + y]);
      gram_host(c, rows(c, c.lam, 1), rows(c, rd.basis[x], rd.nb[x]), false, Lb[x]);
      std::vector<zc> g;
      gram_host(c, rows(c, c.lam, 1), rows(c, rd.xi[x], 1), false, g);
      lam_xi[x] = g[0];
    }
  }
  auto beta = [&](int k, int f, int s) { return &rd.beta[k][(size_t)rd.shift_of[(size_t)f * 4 + s] * maxL]; };
  auto dotL = [&](const std::vector<zc>& a, const zc* b, int L) {
    zc acc(0);
    for (int i = 0; i < L; ++i) acc += a[i] * b[i];
    return acc;
  };
  // shifts: 0: w+ig (z), 1: -w+ig (-z*), 2: w-ig (z*), 3: -w-ig (-z)
  auto half = [&](int f, int x, int y, int sz, int smz) {
    const zc* by = beta(y, f, sz);
    const zc* bx = beta(x, f, smz);
    const int Lx = rd.nb[x], Ly = rd.nb[y];
    const zc a = dotL(E[(size_t)x * nop + y], by, Ly), b = dotL(E[(size_t)y * nop + x], bx, Lx);
    const zc lx = dotL(Lb[x], bx, Lx), ly = dotL(Lb[y], by, Ly);
    return 0.5 * (a - lx * lam_xi[y] + b - ly * lam_xi[x]);
  };
  for (int f = 0; f < rd.n_freq; ++f)
    for (int x = 0; x < nop; ++x)
      for (int y = 0; y < nop; ++y) {
        const zc val = half(f, x, y, 0, 3) + std::conj(half(f, x, y, 1, 2));
        out_host[((size_t)f * nop + x) * nop + y] = make_double2(val.real(), val.imag());
      }
}

// Asymmetric CC-CC response function (Sec. 2.3): with the first-order multipliers of operator Y,
//   tbar^Y(z) (A + z) = -(eta^Y + F t^Y(z))          (left sigma products, as the Lambda solve),
//   f(z) = 1/2 [eta^X t^Y(z) + tbar^Y(z) xi^X],   <<X;Y>>_z = f(z) + conj(f(-z*)).
// It equals the symmetric form for exact solutions; its error is first order in the solution
// errors (the symmetric form's is second order).  Only the shifts z = w + ig and -z* = -w + ig of
// cc_lr_solve are read; the two multiplier systems of one operator and frequency share a Davidson
// run (their trial spaces are the memory of the call).
void response_function_asym(Ctx& c, cplx* out_host) {
  ResponseData& rd = c.rd;
  CCLR_REQUIRE(rd.solved, CCLR_E_STATE, "cc_response_function_asym before cc_lr_solve");
  const int64_t N = c.N;
  const int nop = rd.n_ops, maxL = std::max(8, c.opt.max_subspace);
  const int prec = rd.refined ? CCLR_TC_F64 : c.opt.precision;
  auto beta = [&](int k, int f, int s) { return &rd.beta[k][(size_t)rd.shift_of[(size_t)f * 4 + s] * maxL]; };
  auto dotL = [&](const std::vector<zc>& a, const zc* b, int L) {
    zc acc(0);
    for (int i = 0; i < L; ++i) acc += a[i] * b[i];
    return acc;
  };
  // eta^X . t^Y(z) = (eta^X . B^Y) beta^Y(z)
  std::vector<std::vector<zc>> E((size_t)nop * nop);
  {
    PrecisionScope exact(c, prec);
    Fast32 f32(c);
    for (int x = 0; x < nop; ++x)
      for (int y = 0; y < nop; ++y)
        gram_host(c, rows(c, rd.eta[x], 1), rows(c, rd.basis[y], rd.nb[y]), false, E[(size_t)x * nop + y]);
  }
  std::vector<zc> half((size_t)rd.n_freq * nop * nop * 2);   // [f][x][y][s], s: 0 z, 1 -z*
  for (int f = 0; f < rd.n_freq; ++f)
    for (int y = 0; y < nop; ++y) {   // one operator's two multiplier systems at a time
      std::vector<System> sys(2);   // s: 0 z, 1 -z*
      auto cleanup = [&]() {
        for (auto& s : sys) {
          if (s.rhs) c.dfree(const_cast<cplx*>(s.rhs));
          if (s.B) c.dfree(s.B);
          if (s.S) c.dfree(s.S);
          s.rhs = nullptr;
          s.B = s.S = nullptr;
        }
      };
      try {
        {
          PrecisionScope exact(c, prec);
          Scope sc(c.ws);
          cplx* bd = c.ws.cplxs(maxL);
          cplx* t = c.ws.cplxs(N);
          for (int q = 0; q < 2; ++q) {
              System& s = sys[q];
              to_dev(c, beta(y, f, q), bd, rd.nb[y]);
              lincomb(c.L, N, rd.nb[y], rd.basis[y], N, bd, t, false);
              cplx* b = c.dalloc(N);
              s.rhs = b;
              hessian_right(c, 1, t, b);
              axpy(c.L, N, cx(1), rd.eta[y], b);
              s.z = {-rd.shifts[rd.shift_of[(size_t)f * 4 + q]]};   // tbar (A - w_l) = -b, w_l = -z
              s.B = c.dalloc((int64_t)maxL * N);
              s.S = c.dalloc((int64_t)maxL * N);
            }
        }
        auto op = [&](int nv, const cplx* in, cplx* o) { sigma_left(c, nv, in, o); };
        davidson(c, sys, op, maxL, c.opt.tol);
        if (refining(c)) refine_systems(c, sys, op, maxL, c.opt.tol, nullptr, nullptr);
        PrecisionScope exact(c, prec);
        Fast32 f32(c);
        Scope sc(c.ws);
        cplx* bd = c.ws.cplxs(maxL);
        cplx* l = c.ws.cplxs(N);
        for (int q = 0; q < 2; ++q) {
            const System& s = sys[q];
            to_dev(c, s.beta[0].data(), bd, s.L);
            lincomb(c.L, N, s.L, s.B, N, bd, l, false);
            for (int x = 0; x < nop; ++x) {
              std::vector<zc> g;
              gram_host(c, rows(c, l, 1), rows(c, rd.xi[x], 1), false, g);
              const zc et = dotL(E[(size_t)x * nop + y], beta(y, f, q), rd.nb[y]);
              half[(((size_t)f * nop + x) * nop + y) * 2 + q] = 0.5 * (et + g[0]);
            }
          }
      } catch (...) {
        cleanup();
        throw;
      }
      cleanup();
    }
  for (int f = 0; f < rd.n_freq; ++f)
    for (int x = 0; x < nop; ++x)
      for (int y = 0; y < nop; ++y) {
        const size_t i = (((size_t)f * nop + x) * nop + y) * 2;
        const zc val = half[i] + std::conj(half[i + 1]);
        out_host[((size_t)f * nop + x) * nop + y] = make_double2(val.real(), val.imag());
      }
}

// Static-field derivative of the CC-CC response function (Sec. 2.3 differentiated): d<<X_a;X_b>>_z
// / d eps for H + eps V (V added to the Fock matrix, orbitals unrelaxed), operators fixed, from the
// solutions of the last cc_lr_solve.  The derivatives of the response amplitudes are eliminated
// with the first-order multipliers tbar^k(w) (A + w) = -(eta^k + F t^k(w)):
//   f'(w) = 1/2 [eta^a' t^b + eta^b' t^a + t^a F' t^b + tbar^a(-w) (A' t^b + xi^b')
//                + tbar^b(w) (A' t^a + xi^a')],   t^b = t^b(w), t^a = t^a(-w),
//   <<X_a;X_b>>'_z = f'(z) + conj(f'(-z*)).
// The field enters as Omega + eps xi^V(t) and E + eps <HF|e^-T V e^T|HF>, so with
// t^V = -A^-1 xi^V (ground amplitudes) and lam^V A = -(eta^V + F t^V) (multipliers):
//   A' u = D^2 Omega[t^V, u] + D xi^V[u],   xi^k' = D xi^k[t^V],
//   eta^k' = D_t eta^k[t^V] + eta^k(lam^V) - eta^k(lam = 0),
//   F' u = D_t (F u)[t^V] + F(lam^V) u - F(lam = 0) u + D_t eta^V[u].
// D is the directional derivative in the amplitudes, taken from the library's own products at
// shifted amplitudes: sigma is a cubic in the amplitudes (five-point stencil, exact for degree
// 4), xi and F are quadratics and eta is linear (central differences, exact); eta and F are
// linear in the multipliers.  Products run in the exact mode of the context (FP64, or the
// FP64-class mode of refined solves); the solves are those of cc_lr_solve (refined likewise).
void field_derivative(Ctx& c, const cplx* V_in, cplx* out_host) {
  ResponseData& rd = c.rd;
  CCLR_REQUIRE(rd.solved, CCLR_E_STATE, "cclr_field_derivative before cc_lr_solve");
  CCLR_REQUIRE(c.have_lambda && c.have_hbar, CCLR_E_STATE, "cclr_field_derivative needs T and Lambda");
  const int64_t N = c.N, n = c.n;
  const int nop = rd.n_ops, nv = 4 * nop, maxL = std::max(8, c.opt.max_subspace);
  const int prec = rd.refined ? (int)CCLR_TC_F64 : exact_precision(c);
  const int bmax = c.opt.batch > 0 ? c.opt.batch : nv;
  std::vector<cplx*> owned;
  auto alloc = [&](int64_t m) { cplx* p = c.dalloc(m); owned.push_back(p); return p; };
  cplx* Vd = alloc(n * n);
  cplx* t0 = alloc(N);
  cplx* l0 = alloc(N);
  cplx* tmp = alloc(N);
  cplx* xiV = alloc(N);
  cplx* etaV = alloc(N);
  cplx* tV = alloc(N);
  cplx* lamV = alloc(N);
  cplx* Tv = alloc((int64_t)nv * N);    // t^k(z_s), [k][s]
  cplx* Lv = alloc((int64_t)nv * N);    // tbar^k(z_s)
  cplx* Ap = alloc((int64_t)nv * N);    // A' t^k(z_s)
  cplx* Fp = alloc((int64_t)nv * N);    // F' t^k(z_s)
  cplx* Pv = alloc((int64_t)nv * N);    // products of one batched call
  cplx* etap = alloc((int64_t)nop * N); // eta^k'
  cplx* xip = alloc((int64_t)nop * N);  // xi^k'
  bool moved = false;                   // amplitudes or multipliers differ from the converged ones
  auto set_amps = [&](const cplx* t) {
    copy_vec(c.L, N, t, c.t);
    expand_t2(c, c.t + c.Ns, c.t2, 1);
  };
  auto set_lam = [&](const cplx* l) {
    copy_vec(c.L, N, l, c.lam);
    expand_t2(c, c.lam + c.Ns, c.l2, 1);
    c.named.erase("F.ready");
  };
  auto rebuild = [&]() {
    build_hbar(c);
    c.named.erase("F.ready");
  };
  auto shift_amps = [&](const cplx* u, double h) {   // amplitudes t0 + h u
    copy_vec(c.L, N, t0, tmp);
    axpy(c.L, N, cx(h), u, tmp);
    set_amps(tmp);
  };
  auto restore = [&]() {
    if (!moved) return;
    PrecisionScope exact(c, prec);
    set_amps(t0);
    rebuild();
    set_lam(l0);
    moved = false;
  };
  auto step_for = [&](const cplx* u) {   // stencil step: at most 0.05 per element of h u
    const double nu = std::sqrt(norm2(c, u));
    return nu > 0.0 ? 0.05 / nu : 1.0;
  };
  // batched products of the nv vectors Tv into Pv, then dst += a Pv
  auto batched = [&](void (*fn)(Ctx&, int, const cplx*, cplx*), cplx* dst, cplx a) {
    for (int q0 = 0; q0 < nv; q0 += bmax) {
      const int nb = std::min(bmax, nv - q0);
      fn(c, nb, Tv + (int64_t)q0 * N, Pv + (int64_t)q0 * N);
    }
    axpy(c.L, (int64_t)nv * N, a, Pv, dst);
  };
  auto dot = [&](const cplx* x, const cplx* y) {
    std::vector<zc> g;
    gram_host(c, rows(c, x, 1), rows(c, y, 1), false, g);
    return g[0];
  };
  auto vec = [&](cplx* base, int k, int sidx) { return base + ((int64_t)k * 4 + sidx) * N; };
  try {
    CCLR_CK(cudaMemcpyAsync(Vd, V_in, sizeof(cplx) * n * n, cudaMemcpyDefault, c.stream));
    copy_vec(c.L, N, c.t, t0);
    copy_vec(c.L, N, c.lam, l0);
    {
      PrecisionScope exact(c, prec);
      xi_vec(c, Vd, xiV);
      eta_vec(c, Vd, false, etaV);
    }
    // t^V: (A - 0) t = -xi^V
    {
      std::vector<System> sys(1);
      sys[0].rhs = xiV;
      sys[0].z = {zc(0.0)};
      sys[0].B = c.dalloc((int64_t)maxL * N);
      sys[0].S = c.dalloc((int64_t)maxL * N);
      auto free_sys = [&]() {
        if (sys[0].B) c.dfree(sys[0].B);
        if (sys[0].S) c.dfree(sys[0].S);
        sys[0].B = sys[0].S = nullptr;
      };
      try {
        auto op = [&](int m, const cplx* in, cplx* o) { sigma_right(c, m, in, o); };
        davidson(c, sys, op, maxL, c.opt.tol);
        if (refining(c)) refine_systems(c, sys, op, maxL, c.opt.tol, nullptr, nullptr);
        Scope sc(c.ws);
        cplx* bd = c.ws.cplxs(maxL);
        to_dev(c, sys[0].beta[0].data(), bd, sys[0].L);
        lincomb(c.L, N, sys[0].L, sys[0].B, N, bd, tV, false);
      } catch (...) {
        free_sys();
        throw;
      }
      free_sys();
    }
    // lam^V: lam (A + 0) = -(eta^V + F t^V)
    {
      PrecisionScope exact(c, prec);
      hessian_right(c, 1, tV, tmp);
      axpy(c.L, N, cx(1), etaV, tmp);
    }
    left_solve(c, 1, tmp, zc(0.0), lamV);
    const double hV = step_for(tV);
    fill_zero(c.L, etap, (int64_t)nop * N);
    fill_zero(c.L, xip, (int64_t)nop * N);
    std::vector<zc> half((size_t)rd.n_freq * nop * nop * 2);   // [f][a][b][w], w: 0 z, 1 -z*
    for (int f = 0; f < rd.n_freq; ++f) {
      // response amplitudes t^k(z_s) and first-order multipliers tbar^k(z_s)
      {
        PrecisionScope exact(c, prec);
        Scope sc(c.ws);
        cplx* bd = c.ws.cplxs(maxL);
        for (int k = 0; k < nop; ++k)
          for (int q = 0; q < 4; ++q) {
            to_dev(c, &rd.beta[k][(size_t)rd.shift_of[(size_t)f * 4 + q] * maxL], bd, rd.nb[k]);
            lincomb(c.L, N, rd.nb[k], rd.basis[k], N, bd, vec(Tv, k, q), false);
          }
      }
      {
        std::vector<System> sys((size_t)nv);
        auto free_sys = [&]() {
          for (auto& sy : sys) {
            if (sy.rhs) c.dfree(const_cast<cplx*>(sy.rhs));
            if (sy.B) c.dfree(sy.B);
            if (sy.S) c.dfree(sy.S);
            sy.rhs = nullptr;
            sy.B = sy.S = nullptr;
          }
        };
        try {
          {
            PrecisionScope exact(c, prec);
            for (int k = 0; k < nop; ++k)
              for (int q = 0; q < 4; ++q) {
                System& sy = sys[(size_t)4 * k + q];
                cplx* b = c.dalloc(N);
                sy.rhs = b;
                hessian_right(c, 1, vec(Tv, k, q), b);
                axpy(c.L, N, cx(1), rd.eta[k], b);
                sy.z = {-rd.shifts[rd.shift_of[(size_t)f * 4 + q]]};
                sy.B = c.dalloc((int64_t)maxL * N);
                sy.S = c.dalloc((int64_t)maxL * N);
              }
          }
          auto op = [&](int m, const cplx* in, cplx* o) { sigma_left(c, m, in, o); };
          davidson(c, sys, op, maxL, c.opt.tol);
          if (refining(c)) refine_systems(c, sys, op, maxL, c.opt.tol, nullptr, nullptr);
          Scope sc(c.ws);
          cplx* bd = c.ws.cplxs(maxL);
          for (int i = 0; i < nv; ++i) {
            to_dev(c, sys[i].beta[0].data(), bd, sys[i].L);
            lincomb(c.L, N, sys[i].L, sys[i].B, N, bd, Lv + (int64_t)i * N, false);
          }
        } catch (...) {
          free_sys();
          throw;
        }
        free_sys();
      }
      PrecisionScope exact(c, prec);
      fill_zero(c.L, Ap, (int64_t)nv * N);
      fill_zero(c.L, Fp, (int64_t)nv * N);
      moved = true;
      // multipliers lam^V and 0 at t0: (F(lam^V) - F(0)) u and eta^k(lam^V) - eta^k(0)
      for (int side = 0; side < 2; ++side) {
        const cplx sg = side == 0 ? cx(1) : cx(-1);
        if (side == 0) {
          set_lam(lamV);
        } else {
          fill_zero(c.L, tmp, N);
          set_lam(tmp);
        }
        batched(hessian_right, Fp, sg);
        if (f == 0)
          for (int k = 0; k < nop; ++k) {
            eta_vec(c, rd.ops_dev[k], false, tmp);
            axpy(c.L, N, sg, tmp, etap + (int64_t)k * N);
          }
      }
      set_lam(l0);
      // amplitudes t0 + s hV t^V: D^2 Omega[t^V, u] (five-point), D_t (F u)[t^V], D xi^k[t^V] and
      // D_t eta^k[t^V] (central)
      const int sv[4] = {-2, -1, 1, 2};
      const double c5[4] = {1.0 / 12, -8.0 / 12, 8.0 / 12, -1.0 / 12};
      for (int i = 0; i < 4; ++i) {
        shift_amps(tV, sv[i] * hV);
        rebuild();
        batched(sigma_right, Ap, cx(c5[i] / hV));
        if (sv[i] == -1 || sv[i] == 1) {
          const double w = sv[i] / (2.0 * hV);
          batched(hessian_right, Fp, cx(w));
          if (f == 0)
            for (int k = 0; k < nop; ++k) {
              xi_vec(c, rd.ops_dev[k], tmp);
              axpy(c.L, N, cx(w), tmp, xip + (int64_t)k * N);
              eta_vec(c, rd.ops_dev[k], false, tmp);
              axpy(c.L, N, cx(w), tmp, etap + (int64_t)k * N);
            }
        }
      }
      set_amps(t0);
      rebuild();
      // amplitudes t0 +- h u for every response vector u: D xi^V[u] into A' u, D_t eta^V[u] into F' u
      // (xi and eta read the amplitudes only; the Hbar of t0 stays valid)
      for (int i = 0; i < nv; ++i) {
        const cplx* u = Tv + (int64_t)i * N;
        const double hu = step_for(u);
        for (int sg = -1; sg <= 1; sg += 2) {
          shift_amps(u, sg * hu);
          xi_vec(c, Vd, tmp);
          axpy(c.L, N, cx(sg / (2.0 * hu)), tmp, Ap + (int64_t)i * N);
          eta_vec(c, Vd, false, tmp);
          axpy(c.L, N, cx(sg / (2.0 * hu)), tmp, Fp + (int64_t)i * N);
        }
      }
      set_amps(t0);
      moved = false;
      // f'(w) for w = z (t^b(z), t^a(-z)) and w = -z* (t^b(-z*), t^a(z*))
      for (int a = 0; a < nop; ++a)
        for (int b = 0; b < nop; ++b)
          for (int w = 0; w < 2; ++w) {
            const int sb = w == 0 ? 0 : 1, sa = w == 0 ? 3 : 2;
            const cplx *tb = vec(Tv, b, sb), *ta = vec(Tv, a, sa);
            zc val = dot(etap + (int64_t)a * N, tb) + dot(etap + (int64_t)b * N, ta) + dot(ta, vec(Fp, b, sb));
            copy_vec(c.L, N, vec(Ap, b, sb), tmp);
            axpy(c.L, N, cx(1), xip + (int64_t)b * N, tmp);
            val += dot(vec(Lv, a, sa), tmp);
            copy_vec(c.L, N, vec(Ap, a, sa), tmp);
            axpy(c.L, N, cx(1), xip + (int64_t)a * N, tmp);
            val += dot(vec(Lv, b, sb), tmp);
            half[(((size_t)f * nop + a) * nop + b) * 2 + w] = 0.5 * val;
          }
    }
    for (int f = 0; f < rd.n_freq; ++f)
      for (int a = 0; a < nop; ++a)
        for (int b = 0; b < nop; ++b) {
          const size_t i = (((size_t)f * nop + a) * nop + b) * 2;
          const zc val = half[i] + std::conj(half[i + 1]);
          out_host[((size_t)f * nop + a) * nop + b] = make_double2(val.real(), val.imag());
        }
  } catch (...) {
    try { restore(); } catch (...) {}
    for (auto p : owned) c.dfree(p);
    throw;
  }
  for (auto p : owned) c.dfree(p);
}

// ------------------------------------------------------------------------------ EOM-EE
// Lowest roots of the right eigenproblem A r = w r (EOM-CCSD excitation energies; SI "EOM-EE
// sigma-vectors and intermediates", with the Davidson scheme used for eigenvalues): a
// non-Hermitian Davidson iteration on right sigma products with the orbital-energy-denominator
// preconditioner delta = -(D - w)^{-1} r.  Ritz pairs come from the Galerkin problem
// (B^H S) y = w (B^H B) y (Cholesky of B^H B, then the general complex eigensolver on the host);
// roots are ordered by real part; when the space is full it is compressed onto the lowest Ritz
// vectors.  Starting vectors: unit vectors on the smallest denominators.
namespace {
// B^H B = L L^H (lower L, n x n, ld = ld); false if not positive definite
bool zchol(int n, const std::vector<zc>& A, int ld, std::vector<zc>& Lo) {
  Lo.assign((size_t)n * n, zc(0));
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * ld + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(Lo[(size_t)j * n + k]);
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    Lo[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      zc s = A[(size_t)i * ld + j];
      for (int k = 0; k < j; ++k) s -= Lo[(size_t)i * n + k] * std::conj(Lo[(size_t)j * n + k]);
      Lo[(size_t)i * n + j] = s / ljj;
    }
  }
  return true;
}
}  // namespace

int eom_ee(Ctx& c, int nroots, std::vector<zc>& w_out) {
  static const bool verbose = std::getenv("CCLR_VERBOSE") != nullptr;
  CCLR_REQUIRE(c.have_t && c.have_hbar, CCLR_E_STATE, "cc_eom_ee before cc_ground");
  CCLR_REQUIRE(nroots >= 1 && nroots <= kVecMatOut, CCLR_E_ARG, "cc_eom_ee: n_roots must be 1..16");
  Fast32 f32(c);
  const int64_t N = c.N;
  CCLR_REQUIRE(N > nroots, CCLR_E_ARG, "cc_eom_ee: more roots than excitations");
  const int maxL = std::min<int>(kVecMatMaxRows / 2, std::max(c.opt.max_subspace, 6 * nroots));
  const int nstart = (int)std::min<int64_t>(N, std::max(3 * nroots, 8));
  for (auto p : c.eom_vecs) c.dfree(p);
  c.eom_vecs.clear();
  c.eom_w.clear();
  cplx* B = c.dalloc((int64_t)maxL * N);
  cplx* S = c.dalloc((int64_t)maxL * N);
  auto cleanup = [&]() { c.dfree(B); c.dfree(S); };
  int iters = 0;
  try {
    Scope sc(c.ws);
    double* vscr = (double*)c.ws.alloc(sizeof(double) * vecmat_scratch_doubles());
    cplx* cdev = c.ws.cplxs((int64_t)2 * maxL * kVecMatOut);
    cplx* zdev = c.ws.cplxs(kVecMatOut);
    double* n2dev = (double*)c.ws.alloc(sizeof(double) * kVecMatOut);
    cplx* R = c.ws.cplxs((int64_t)nroots * N);
    // starting vectors: e_k on the nstart smallest denominators
    {
      std::vector<double> D(N);
      CCLR_CK(cudaMemcpyAsync(D.data(), c.D, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream));
      c.sync();
      std::vector<int64_t> idx(N);
      for (int64_t i = 0; i < N; ++i) idx[i] = i;
      std::partial_sort(idx.begin(), idx.begin() + nstart, idx.end(), [&](int64_t a, int64_t b) { return D[a] < D[b]; });
      fill_zero(c.L, B, (int64_t)nstart * N);
      const cplx one = cx(1.0);
      for (int j = 0; j < nstart; ++j)
        CCLR_CK(cudaMemcpyAsync(B + (int64_t)j * N + idx[j], &one, sizeof(cplx), cudaMemcpyHostToDevice, c.stream));
      c.sync();
    }
    std::vector<zc> BS((size_t)maxL * maxL, zc(0)), BB((size_t)maxL * maxL, zc(0));
    int L = nstart, fresh = nstart;
    std::vector<zc> theta(nroots);
    std::vector<std::vector<zc>> Y(nroots);
    std::vector<double> rn(nroots, 1e300);
    double best = 1e300;
    int best_it = 0;
    for (int it = 1; it <= c.opt.maxit; ++it) {
      iters = it;
      {   // sigma of the new vectors, in batches
        const int L0 = L - fresh;
        const int bmax = c.opt.batch > 0 ? c.opt.batch : fresh;
        const double t0 = now();
        for (int q0 = 0; q0 < fresh; q0 += bmax) {
          const int nb = std::min(bmax, fresh - q0);
          sigma_right(c, nb, B + (int64_t)(L0 + q0) * N, S + (int64_t)(L0 + q0) * N);
        }
        c.sync();
        c.stats.sigma_seconds += now() - t0;
        // Galerkin matrices: new columns of B^H S and B^H B, new rows of B^H S
        std::vector<zc> g;
        gram_host(c, rows(c, B, L), Rows().add(S + (int64_t)L0 * N, fresh, N).add(B + (int64_t)L0 * N, fresh, N), true,
                  g);
        const int ny = 2 * fresh;
        for (int i = 0; i < L; ++i)
          for (int j = 0; j < fresh; ++j) {
            BS[(size_t)i * maxL + L0 + j] = g[(size_t)i * ny + j];
            const zc bb = g[(size_t)i * ny + fresh + j];
            BB[(size_t)i * maxL + L0 + j] = bb;
            BB[(size_t)(L0 + j) * maxL + i] = std::conj(bb);
          }
        if (L0 > 0) {
          gram_host(c, rows(c, S, L0), rows(c, B + (int64_t)L0 * N, fresh), true, g);
          for (int i = 0; i < L0; ++i)
            for (int j = 0; j < fresh; ++j) BS[(size_t)(L0 + j) * maxL + i] = std::conj(g[(size_t)i * fresh + j]);
        }
      }
      // Ritz pairs: M = Lo^{-1} (B^H S) Lo^{-H}, y = Lo^{-H} y'
      std::vector<zc> Lo;
      CCLR_REQUIRE(zchol(L, BB, maxL, Lo), CCLR_E_NOCONV, "cc_eom_ee: trial space lost linear independence");
      std::vector<zc> M((size_t)L * L);
      {
        std::vector<zc> T((size_t)L * L);   // T = Lo^{-1} BS (forward substitution, column by column)
        for (int j = 0; j < L; ++j)
          for (int i = 0; i < L; ++i) {
            zc s = BS[(size_t)i * maxL + j];
            for (int k = 0; k < i; ++k) s -= Lo[(size_t)i * L + k] * T[(size_t)k * L + j];
            T[(size_t)i * L + j] = s / Lo[(size_t)i * L + i];
          }
        for (int i = 0; i < L; ++i)   // M = T Lo^{-H}: solve M Lo^H = T row by row
          for (int j = 0; j < L; ++j) {
            zc s = T[(size_t)i * L + j];
            for (int k = 0; k < j; ++k) s -= M[(size_t)i * L + k] * std::conj(Lo[(size_t)j * L + k]);
            M[(size_t)i * L + j] = s / std::conj(Lo[(size_t)j * L + j]);
          }
      }
      std::vector<zc> wv, V;
      CCLR_REQUIRE(zgeev_small(L, M, wv, V), CCLR_E_NOCONV, "cc_eom_ee: subspace eigenproblem did not converge");
      std::vector<int> ord(L);
      for (int i = 0; i < L; ++i) ord[i] = i;
      std::sort(ord.begin(), ord.end(), [&](int a, int b) { return wv[a].real() < wv[b].real(); });
      auto ritz = [&](int col, std::vector<zc>& y) {   // y = Lo^{-H} y' (back substitution)
        y.assign(maxL, zc(0));
        for (int i = L - 1; i >= 0; --i) {
          zc s = V[(size_t)i * L + col];
          for (int k = i + 1; k < L; ++k) s -= std::conj(Lo[(size_t)k * L + i]) * y[k];
          y[i] = s / std::conj(Lo[(size_t)i * L + i]);
        }
      };
      for (int q = 0; q < nroots; ++q) {
        theta[q] = wv[ord[q]];
        ritz(ord[q], Y[q]);
      }
      // residual norms r_q = (S - theta_q B) y_q, all roots in one pass
      auto coef = [&](const std::vector<int>& qs) {
        const int m = (int)qs.size();
        std::vector<zc> C((size_t)2 * L * m);
        for (int t = 0; t < m; ++t)
          for (int j = 0; j < L; ++j) {
            C[(size_t)j * m + t] = Y[qs[t]][j];
            C[(size_t)(L + j) * m + t] = -theta[qs[t]] * Y[qs[t]][j];
          }
        to_dev(c, C.data(), cdev, (int64_t)2 * L * m);
      };
      std::vector<int> all(nroots);
      for (int q = 0; q < nroots; ++q) all[q] = q;
      coef(all);
      {
        VecMat a;
        a.X = Rows().add(S, L, N).add(B, L, N);
        a.m = nroots;
        a.C = cdev;
        a.norm2 = n2dev;
        vecmat(c.L, N, a, vscr);
        double h[kVecMatOut];
        CCLR_CK(cudaMemcpyAsync(h, n2dev, sizeof(double) * nroots, cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        for (int q = 0; q < nroots; ++q) rn[q] = std::sqrt(std::max(0.0, h[q]));
      }
      std::vector<int> open;
      double mx = 0.0;
      for (int q = 0; q < nroots; ++q) {
        const double tol_q =
            mixed_precision(c.opt.precision) ? std::max(c.opt.tol, 1e-5 * std::max(1.0, std::abs(theta[q]))) : c.opt.tol;
        if (rn[q] >= tol_q) open.push_back(q);
        mx = std::max(mx, rn[q] / tol_q);
      }
      if (verbose)
        std::fprintf(stderr, "[cclr] eom it %d L %d open %zu/%d max|r|/tol %.3e lowest %.10f\n", it, L, open.size(),
                     nroots, mx, theta[0].real());
      if (!open.empty() && mixed_precision(c.opt.precision)) {   // stagnation within 5x the floor
        if (mx < 0.8 * best) { best = mx; best_it = it; }
        if (it - best_it >= 4 && mx < 5.0) open.clear();
      }
      if (open.empty()) break;
      if (it == c.opt.maxit) throw Error(CCLR_E_NOCONV, "cc_eom_ee did not converge within maxit iterations");
      // compress onto the lowest Ritz vectors when the space cannot take the new directions
      if (L + (int)open.size() > maxL) {
        const int kk = std::min(L, std::max(2 * nroots, maxL / 2));
        std::vector<std::vector<zc>> Q;   // B^H B-orthonormal combinations of the lowest Ritz vectors
        for (int t = 0; t < kk; ++t) {
          std::vector<zc> y;
          ritz(ord[t], y);
          for (int pass = 0; pass < 2; ++pass)
            for (auto& u : Q) {
              zc d(0);
              for (int i = 0; i < L; ++i) {
                zc r(0);
                for (int j = 0; j < L; ++j) r += BB[(size_t)i * maxL + j] * y[j];
                d += std::conj(u[i]) * r;
              }
              for (int i = 0; i < L; ++i) y[i] -= d * u[i];
            }
          double n2 = 0.0;
          for (int i = 0; i < L; ++i) {
            zc r(0);
            for (int j = 0; j < L; ++j) r += BB[(size_t)i * maxL + j] * y[j];
            n2 += (std::conj(y[i]) * r).real();
          }
          if (!(n2 > 1e-20)) continue;
          for (auto& x : y) x /= std::sqrt(n2);
          Q.push_back(y);
        }
        const int k2 = (int)Q.size();
        std::vector<zc> W((size_t)L * k2);
        for (int j = 0; j < L; ++j)
          for (int a = 0; a < k2; ++a) W[(size_t)j * k2 + a] = Q[a][j];
        Scope s2(c.ws);
        cplx* tmp = c.ws.cplxs((int64_t)k2 * N);
        for (cplx* X : {B, S}) {
          combine(c, rows(c, X, L), k2, W, tmp);
          copy_vec(c.L, (int64_t)k2 * N, tmp, X);
        }
        auto congr = [&](std::vector<zc>& Mx) {
          std::vector<zc> out((size_t)maxL * maxL, zc(0));
          for (int a = 0; a < k2; ++a)
            for (int b = 0; b < k2; ++b) {
              zc acc(0);
              for (int i = 0; i < L; ++i) {
                zc r(0);
                for (int j = 0; j < L; ++j) r += Mx[(size_t)i * maxL + j] * Q[b][j];
                acc += std::conj(Q[a][i]) * r;
              }
              out[(size_t)a * maxL + b] = acc;
            }
          Mx.swap(out);
        };
        congr(BS);
        congr(BB);
        L = k2;
        fresh = 0;
        continue;   // the Ritz pairs of the compressed space are formed before new corrections
      }
      // preconditioned corrections of the open roots, one pass; then projection and selection
      coef(open);
      std::vector<zc> zq(open.size());
      for (size_t t = 0; t < open.size(); ++t) zq[t] = theta[open[t]];
      to_dev(c, zq.data(), zdev, (int64_t)open.size());
      double pre2[kVecMatOut];
      {
        VecMat a;
        a.X = Rows().add(S, L, N).add(B, L, N);
        a.m = (int)open.size();
        a.C = cdev;
        a.Y = R;
        a.ldy = N;
        a.D = c.Dpre ? c.Dpre : c.D;
        a.z = zdev;
        a.norm2 = n2dev;
        a.norm_y = true;
        vecmat(c.L, N, a, vscr);
        CCLR_CK(cudaMemcpyAsync(pre2, n2dev, sizeof(double) * open.size(), cudaMemcpyDeviceToHost, c.stream));
        c.sync();
      }
      const int kk = add_corrections(c, B, L, R, (int)open.size(), pre2, std::min((int)open.size(), maxL - L), cdev,
                                     vscr);
      if (kk == 0) throw Error(CCLR_E_NOCONV, "cc_eom_ee stagnated: no new direction");
      L += kk;
      fresh = kk;
    }
    // eigenvectors x_q = B y_q (unit norm up to the Galerkin metric)
    for (int q = 0; q < nroots; ++q) {
      cplx* v = c.dalloc(N);
      std::vector<zc> W(Y[q].begin(), Y[q].begin() + L);
      combine(c, rows(c, B, L), 1, W, v);
      c.eom_vecs.push_back(v);
    }
    c.eom_w = theta;
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
  w_out = c.eom_w;
  return iters;
}

}  // namespace cclr

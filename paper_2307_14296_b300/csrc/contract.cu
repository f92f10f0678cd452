// Contraction planner: maps "ab,bc->ac"-style tensor contractions onto one GEMM plus at most
// three strided permutations (operands into GEMM order, result into the target layout).
// Operands already in a GEMM-compatible contiguous order are passed straight to the GEMM.
// The GEMM backend is chosen per call by gemm_dispatch (FP64 DFMA or the tensor-core path).
#include "ctx.h"
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>

namespace cclr {

void gemm_dispatch(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A,
                   int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc);

namespace {

struct Spec {
  std::string a, b, c;
};

Spec parse(const char* s) {
  Spec p;
  std::string str(s);
  size_t comma = str.find(','), arrow = str.find("->");
  CCLR_REQUIRE(comma != std::string::npos && arrow != std::string::npos && comma < arrow, CCLR_E_ARG,
               std::string("einsum: bad spec ") + s);
  p.a = str.substr(0, comma);
  p.b = str.substr(comma + 1, arrow - comma - 1);
  p.c = str.substr(arrow + 2);
  return p;
}

// view of t with axes ordered by `letters` (each letter's axis in `have`)
Tensor reorder(const Tensor& t, const std::string& have, const std::string& want) {
  Tensor r = t;
  r.rank = (int)want.size();
  for (size_t k = 0; k < want.size(); ++k) {
    size_t pos = have.find(want[k]);
    r.dim[k] = t.dim[pos];
    r.str[k] = t.str[pos];
  }
  return r;
}

int64_t prod(const Tensor& t, const std::string& have, const std::string& letters, const std::map<char, int64_t>& ext) {
  (void)t; (void)have;
  int64_t p = 1;
  for (char ch : letters) p *= ext.at(ch);
  return p;
}

}  // namespace

void einsum_impl(Ctx& c, const char* spec, cplx alpha, const Tensor& A, const Tensor& B, double beta, const Tensor& C);

// CCLR_TRACE=1 prints every contraction with its GEMM shape and device time (debug aid; it
// synchronizes the stream around each call).
void einsum(Ctx& c, const char* spec, cplx alpha, const Tensor& A, const Tensor& B, double beta, const Tensor& C) {
  static const bool trace = std::getenv("CCLR_TRACE") != nullptr;
  // per-contraction kernel timing: launches are labelled with the spec when asked for
  static const bool detail = std::getenv("CCLR_PROFILE_DETAIL") != nullptr;
  struct Label {
    KernelTimer& k;
    Label(KernelTimer& kt, const char* l, bool on) : k(kt) { if (on) k.label = l; }
    ~Label() { k.label = nullptr; }
  } lab(c.kt, spec, detail);
  if (!trace) return einsum_impl(c, spec, alpha, A, B, beta, C);
  CCLR_CK(cudaStreamSynchronize(c.stream));
  auto t0 = std::chrono::steady_clock::now();
  einsum_impl(c, spec, alpha, A, B, beta, C);
  CCLR_CK(cudaStreamSynchronize(c.stream));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  std::fprintf(stderr, "[cclr] %-28s A%s B%s C%s %9.3f ms\n", spec, std::to_string(A.numel()).c_str(),
               std::to_string(B.numel()).c_str(), std::to_string(C.numel()).c_str(), ms);
}

void einsum_impl(Ctx& c, const char* spec, cplx alpha, const Tensor& A, const Tensor& B, double beta, const Tensor& C) {
  Spec s = parse(spec);
  CCLR_REQUIRE((int)s.a.size() == A.rank && (int)s.b.size() == B.rank && (int)s.c.size() == C.rank, CCLR_E_ARG,
               std::string("einsum: rank mismatch in ") + spec);
  std::map<char, int64_t> ext;
  auto reg = [&](const std::string& l, const Tensor& t) {
    for (size_t k = 0; k < l.size(); ++k) {
      auto it = ext.find(l[k]);
      if (it == ext.end()) ext[l[k]] = t.dim[k];
      else CCLR_REQUIRE(it->second == t.dim[k], CCLR_E_ARG, std::string("einsum: extent mismatch in ") + spec);
    }
  };
  reg(s.a, A);
  reg(s.b, B);
  reg(s.c, C);
  std::string fa, fb, kk;
  for (char ch : s.c) {
    bool ia = s.a.find(ch) != std::string::npos, ib = s.b.find(ch) != std::string::npos;
    CCLR_REQUIRE(ia != ib, CCLR_E_ARG, std::string("einsum: batch or missing index in ") + spec);
    (ia ? fa : fb) += ch;
  }
  for (char ch : s.a) {
    if (s.c.find(ch) != std::string::npos) continue;
    CCLR_REQUIRE(s.b.find(ch) != std::string::npos, CCLR_E_ARG, std::string("einsum: lone index in ") + spec);
    kk += ch;
  }
  for (char ch : s.b)
    if (s.c.find(ch) == std::string::npos)
      CCLR_REQUIRE(s.a.find(ch) != std::string::npos, CCLR_E_ARG, std::string("einsum: lone index in ") + spec);

  const int64_t M = prod(A, s.a, fa, ext), N = prod(B, s.b, fb, ext), K = prod(A, s.a, kk, ext);
  if (M == 0 || N == 0) return;
  Scope scope(c.ws);

  // candidate K orders: as in A, as in B (the one that lets more operands be used in place)
  std::string kB;
  for (char ch : s.b)
    if (kk.find(ch) != std::string::npos) kB += ch;
  std::string korder = kk;
  {
    auto directA = [&](const std::string& ko) {
      return !A.conj && (reorder(A, s.a, fa + ko).contiguous() || reorder(A, s.a, ko + fa).contiguous());
    };
    auto directB = [&](const std::string& ko) {
      return !B.conj && (reorder(B, s.b, ko + fb).contiguous() || reorder(B, s.b, fb + ko).contiguous());
    };
    // on a tie the larger operand keeps its own order: its view (and BF16 slices) are then the
    // same for every contraction that reads it over the same indices
    int sa = (int)directA(kk) + (int)directB(kk), sb = (int)directA(kB) + (int)directB(kB);
    if (sb > sa || (sb == sa && B.numel() > A.numel())) korder = kB;
  }

  cplx al = make_double2(alpha.x, alpha.y);
  // Tensor-core route: both operands K-major ([M][K] and [N][K]); the GEMM then computes
  // C = A' B'^T (or C^T = B' A'^T when the target is laid out [N][M]).
  if (c.opt.precision != CCLR_FP64 && tc_eligible(M, N, K)) {
    // operands go straight from their strided views into BF16 slices (no FP64 copy)
    Tensor va = reorder(A, s.a, fa + korder), vb = reorder(B, s.b, fb + korder);
    al.x *= A.scale * B.scale;
    al.y *= A.scale * B.scale;
    const int nra = (int)fa.size(), nrb = (int)fb.size();
    Tensor cAB = reorder(C, s.c, fa + fb), cBA = reorder(C, s.c, fb + fa);
    if (cAB.contiguous()) {
      tc_gemm_views(c, va, nra, vb, nrb, al, cx(beta), C.p, N);
    } else if (cBA.contiguous()) {
      tc_gemm_views(c, vb, nrb, va, nra, al, cx(beta), C.p, M);
    } else {
      // Strided target: the epilogue writes C through a row-offset map.  The lane side (TMEM
      // rows, stored contiguously across a warp) is the operand holding C's unit-stride index,
      // which is made its fastest row index.
      char unit = 0;
      for (size_t k = 0; k < s.c.size(); ++k)
        if (C.str[k] == 1 && C.dim[k] > 1) unit = s.c[k];
      const bool lane_b = unit == 0 || fb.find(unit) != std::string::npos;
      std::string fl = lane_b ? fb : fa, fr = lane_b ? fa : fb;
      if (unit) {
        fl.erase(fl.find(unit), 1);
        fl += unit;
      }
      if (tc_splits(c, M, N, K, true) == 1 && !fl.empty() && !fr.empty() && fl.size() <= 4 && fr.size() <= 4) {
        const Tensor vl = lane_b ? reorder(B, s.b, fl + korder) : reorder(A, s.a, fl + korder);
        const Tensor vr = lane_b ? reorder(A, s.a, fr + korder) : reorder(B, s.b, fr + korder);
        OutAxes oa;
        oa.nm = (int)fr.size();
        oa.nn = (int)fl.size();
        for (int i = 0; i < oa.nm; ++i) {
          oa.mdim[i] = ext[fr[i]];
          oa.mstr[i] = C.str[s.c.find(fr[i])];
        }
        for (int i = 0; i < oa.nn; ++i) {
          oa.ndim[i] = ext[fl[i]];
          oa.nstr[i] = C.str[s.c.find(fl[i])];
        }
        tc_gemm_views(c, vr, (int)fr.size(), vl, (int)fl.size(), al, cx(beta), C.p, 0, &oa);
      } else {
        cplx* tmp = c.ws.cplxs(M * N);
        tc_gemm_views(c, va, nra, vb, nrb, al, cx(0.0), tmp, N);
        std::vector<int64_t> d;
        for (char ch : fa + fb) d.push_back(ext[ch]);
        permute(c.L, reorder(Tensor::make(tmp, d), fa + fb, s.c), C, cx(1.0), beta != 0.0);
      }
    }
    return;
  }
  // ---- operand A as op(A) = [M x K]
  bool ta = false;
  const cplx* pa;
  int64_t lda;
  {
    Tensor v1 = reorder(A, s.a, fa + korder), v2 = reorder(A, s.a, korder + fa);
    if (!A.conj && v1.contiguous()) {
      ta = false; pa = A.p; lda = K; al.x *= A.scale; al.y *= A.scale;
    } else if (!A.conj && v2.contiguous()) {
      ta = true; pa = A.p; lda = M; al.x *= A.scale; al.y *= A.scale;
    } else {
      cplx* tmp = c.ws.cplxs(M * K);
      std::vector<int64_t> d;
      for (char ch : fa + korder) d.push_back(ext[ch]);
      permute(c.L, v1, Tensor::make(tmp, d), cx(1.0), false);
      ta = false; pa = tmp; lda = K;
    }
  }
  // ---- operand B as op(B) = [K x N]
  bool tb = false;
  const cplx* pb;
  int64_t ldb;
  {
    Tensor v1 = reorder(B, s.b, korder + fb), v2 = reorder(B, s.b, fb + korder);
    if (!B.conj && v1.contiguous()) {
      tb = false; pb = B.p; ldb = N; al.x *= B.scale; al.y *= B.scale;
    } else if (!B.conj && v2.contiguous()) {
      tb = true; pb = B.p; ldb = K; al.x *= B.scale; al.y *= B.scale;
    } else {
      cplx* tmp = c.ws.cplxs(K * N);
      std::vector<int64_t> d;
      for (char ch : korder + fb) d.push_back(ext[ch]);
      permute(c.L, v1, Tensor::make(tmp, d), cx(1.0), false);
      tb = false; pb = tmp; ldb = N;
    }
  }
  // ---- result
  Tensor cAB = reorder(C, s.c, fa + fb), cBA = reorder(C, s.c, fb + fa);
  if (cAB.contiguous()) {
    gemm_dispatch(c, ta, tb, M, N, K, al, pa, lda, pb, ldb, cx(beta), C.p, N);
  } else if (cBA.contiguous()) {
    // C^T [N x M] = op(B)^T op(A)^T
    gemm_dispatch(c, !tb, !ta, N, M, K, al, pb, ldb, pa, lda, cx(beta), C.p, M);
  } else {
    cplx* tmp = c.ws.cplxs(M * N);
    gemm_dispatch(c, ta, tb, M, N, K, al, pa, lda, pb, ldb, cx(0.0), tmp, N);
    std::vector<int64_t> d;
    for (char ch : fa + fb) d.push_back(ext[ch]);
    Tensor t = Tensor::make(tmp, d);
    // permute tmp (axes fa+fb) into C (axes s.c)
    Tensor src = reorder(t, fa + fb, s.c);
    permute(c.L, src, C, cx(1.0), beta != 0.0);
  }
}

}  // namespace cclr

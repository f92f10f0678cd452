// Ground-state CCSD residual/energy and the Hbar intermediates on the device (complex FP64).
//
// Ground state: the spin-orbital CCSD equations (Stanton, Gauss, Watts & Bartlett 1991) for a
// general complex Hamiltonian; the paper's step 1 (Sec. 3) defers them to the ExaCorr paper.
// Hbar: SI Eqs. F_im ... tau (paper's step 2), elements stored creators-first.
// The o^2 v^4 particle-particle ladders run on packed pair indices (a<b, e<f, i<j), which is
// 1/8 of the full-tensor work the paper's TAL-SH code performs.
#include "ctx.h"

namespace cclr {

static inline Tensor T(cplx* p, std::initializer_list<int64_t> d) { return Tensor::make(p, d); }

Tensor Ctx::V(const char* cls) const {
  const int64_t O = o, Vv = v;
  std::string k(cls);
  Tensor oooo_ = T(this->oooo, {O, O, O, O}), ooov_ = T(this->ooov, {O, O, O, Vv});
  Tensor oovv_ = T(this->oovv, {O, O, Vv, Vv}), ovov_ = T(this->ovov, {O, Vv, O, Vv});
  Tensor ovvv_ = T(this->ovvv, {O, Vv, Vv, Vv});
  if (k == "oooo") return oooo_;
  if (k == "ooov") return ooov_;
  if (k == "oovo") return ooov_.perm({0, 1, 3, 2}).neg();
  if (k == "ovoo") return ooov_.perm({2, 3, 0, 1}).cj();
  if (k == "vooo") return ooov_.perm({3, 2, 0, 1}).cj().neg();
  if (k == "oovv") return oovv_;
  if (k == "vvoo") return oovv_.perm({2, 3, 0, 1}).cj();
  if (k == "ovov") return ovov_;
  if (k == "ovvo") return ovov_.perm({0, 1, 3, 2}).neg();
  if (k == "voov") return ovov_.perm({1, 0, 2, 3}).neg();
  if (k == "vovo") return ovov_.perm({1, 0, 3, 2});
  if (k == "ovvv") return ovvv_;
  if (k == "vovv") return ovvv_.perm({1, 0, 2, 3}).neg();
  if (k == "vvov") return ovvv_.perm({2, 3, 0, 1}).cj();
  if (k == "vvvo") return ovvv_.perm({2, 3, 1, 0}).cj().neg();
  throw Error(CCLR_E_ARG, "no full view of integral class " + k);
}

Tensor Ctx::f(const char* blk) const {
  Tensor t;
  t.rank = 2;
  t.str[0] = n;
  t.str[1] = 1;
  const bool ro = blk[0] == 'o', co = blk[1] == 'o';
  t.dim[0] = ro ? o : v;
  t.dim[1] = co ? o : v;
  t.p = fock + (ro ? 0 : (int64_t)o * n) + (co ? 0 : o);
  return t;
}

// ---------------------------------------------------------------- helpers
void expand_t2(Ctx& c, const cplx* packed, cplx* full, int64_t nvec) {
  // packed: nvec contiguous blocks of Po*Pv; full: nvec x (o,o,v,v)
  Tensor X = Tensor::make(full, {nvec, (int64_t)c.o, (int64_t)c.o, (int64_t)c.v, (int64_t)c.v});
  unpack_doubles(c.L, packed, c.Po * c.Pv, X, c.o, c.v);
  if (full == c.t2 || full == c.l2) ++c.data_gen;   // cached tensor-core slices are stale
}

void pack_anti(Ctx& c, const Tensor& X, cplx* D, int64_t nvec, cplx alpha, bool anti, bool acc) {
  pack_doubles_impl(c.L, X, D, nvec, c.o, c.v, alpha, anti, acc, c.po, c.pv);
}

void build_denominators(Ctx& c) {
  std::vector<cplx> F((size_t)c.n * c.n);
  CCLR_CK(cudaMemcpy(F.data(), c.fock, sizeof(cplx) * F.size(), cudaMemcpyDeviceToHost));
  std::vector<double> D((size_t)c.N);
  auto e = [&](int p) { return F[(size_t)p * c.n + p].x; };
  for (int i = 0; i < c.o; ++i)
    for (int a = 0; a < c.v; ++a) D[(size_t)i * c.v + a] = e(c.o + a) - e(i);
  std::vector<int2> po(c.Po), pv(c.Pv);
  int64_t k = 0;
  for (int q = 1; q < c.o; ++q)
    for (int p = 0; p < q; ++p) po[k++] = make_int2(p, q);
  k = 0;
  for (int q = 1; q < c.v; ++q)
    for (int p = 0; p < q; ++p) pv[k++] = make_int2(p, q);
  for (int64_t ij = 0; ij < c.Po; ++ij)
    for (int64_t ab = 0; ab < c.Pv; ++ab)
      D[(size_t)(c.Ns + ij * c.Pv + ab)] =
          e(c.o + pv[ab].x) + e(c.o + pv[ab].y) - e(po[ij].x) - e(po[ij].y);
  CCLR_CK(cudaMemcpy(c.D, D.data(), sizeof(double) * D.size(), cudaMemcpyHostToDevice));
}

static zc fetch(Ctx& c, const cplx* dev) {
  cplx h;
  CCLR_CK(cudaMemcpyAsync(&h, dev, sizeof(cplx), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  return zc(h.x, h.y);
}

zc ccsd_energy(Ctx& c) {
  // E = f_ia t_i^a + 1/4 <ij||ab> t_ij^ab + 1/2 <ij||ab> t_i^a t_j^b
  Scope sc(c.ws);
  const int64_t o = c.o, v = c.v;
  cplx* fov = c.ws.cplxs(o * v);
  permute(c.L, c.f("ov"), T(fov, {o, v}), cx(1), false);
  cplx* g = c.ws.cplxs(o * v);
  Tensor t1 = T(c.t, {o, v});
  einsum(c, "ijab,jb->ia", cx(0.5), c.V("oovv"), t1, 0.0, T(g, {o, v}));
  permute(c.L, T(fov, {o, v}), T(g, {o, v}), cx(1), true);          // g = f_ov + 1/2 V t1
  cplx* out = c.ws.cplxs(2);
  cplx* scr = c.ws.cplxs(reduce_blocks() * 2);
  dots(c.L, o * v, 1, g, 0, c.t, 0, false, out, scr);
  dots(c.L, c.Nd, 1, c.oovv_p, 0, c.t + c.Ns, 0, false, out + 1, scr);
  return fetch(c, out) + fetch(c, out + 1);
}

// Omega(t) in the amplitude layout.  Singles via einsum; doubles accumulated as
//  X4 (terms antisymmetrized by P(ij)P(ab) when packing; P(ab)- or P(ij)-only terms enter with
//  weight 1/2, unpermuted antisymmetric terms with 1/4) plus packed ladder-type GEMMs.
void ccsd_residual(Ctx& c, cplx* R) {
  Scope sc(c.ws);
  const int64_t o = c.o, v = c.v, Po = c.Po, Pv = c.Pv;
  Tensor t1 = T(c.t, {o, v}), t2 = T(c.t2, {o, o, v, v});
  const cplx* t2p = c.t + c.Ns;
  // tau and tau-tilde
  cplx* ta = c.ws.cplxs(o * o * v * v);
  cplx* tt = c.ws.cplxs(o * o * v * v);
  copy_vec(c.L, o * o * v * v, c.t2, ta);
  einsum(c, "ia,jb->ijab", cx(1), t1, t1, 1.0, T(ta, {o, o, v, v}));
  einsum(c, "ib,ja->ijab", cx(-1), t1, t1, 1.0, T(ta, {o, o, v, v}));
  copy_vec(c.L, o * o * v * v, c.t2, tt);
  einsum(c, "ia,jb->ijab", cx(0.5), t1, t1, 1.0, T(tt, {o, o, v, v}));
  einsum(c, "ib,ja->ijab", cx(-0.5), t1, t1, 1.0, T(tt, {o, o, v, v}));
  Tensor Ta = T(ta, {o, o, v, v}), Tt = T(tt, {o, o, v, v});
  cplx* tap = c.ws.cplxs(Po * Pv);
  pack_anti(c, Tensor::make(ta, {1, o, o, v, v}), tap, 1, cx(1), false, false);
  // F and W intermediates (Stanton-Gauss, full Fock diagonal kept)
  cplx *Fae = c.ws.cplxs(v * v), *Fmi = c.ws.cplxs(o * o), *Fme = c.ws.cplxs(o * v);
  Tensor tFae = T(Fae, {v, v}), tFmi = T(Fmi, {o, o}), tFme = T(Fme, {o, v});
  permute(c.L, c.f("vv"), tFae, cx(1), false);
  einsum(c, "me,ma->ae", cx(-0.5), c.f("ov"), t1, 1.0, tFae);
  einsum(c, "mf,mafe->ae", cx(1), t1, c.V("ovvv"), 1.0, tFae);
  einsum(c, "mnaf,mnef->ae", cx(-0.5), Tt, c.V("oovv"), 1.0, tFae);
  permute(c.L, c.f("oo"), tFmi, cx(1), false);
  einsum(c, "ie,me->mi", cx(0.5), t1, c.f("ov"), 1.0, tFmi);
  einsum(c, "ne,mnie->mi", cx(1), t1, c.V("ooov"), 1.0, tFmi);
  einsum(c, "inef,mnef->mi", cx(0.5), Tt, c.V("oovv"), 1.0, tFmi);
  permute(c.L, c.f("ov"), tFme, cx(1), false);
  einsum(c, "nf,mnef->me", cx(1), t1, c.V("oovv"), 1.0, tFme);
  // W_mnij without its tau<mn||ef> part (that part is merged with the ladder's below)
  cplx* Wmn = c.ws.cplxs(o * o * o * o);
  Tensor tW = T(Wmn, {o, o, o, o});
  permute(c.L, c.V("oooo"), tW, cx(1), false);
  einsum(c, "je,mnie->mnij", cx(1), t1, c.V("ooov"), 1.0, tW);
  einsum(c, "ie,mnje->mnij", cx(-1), t1, c.V("ooov"), 1.0, tW);
  cplx* Wmbej = c.ws.cplxs(o * v * v * o);
  Tensor tWm = T(Wmbej, {o, v, v, o});
  permute(c.L, c.V("ovvo"), tWm, cx(1), false);
  einsum(c, "jf,mbef->mbej", cx(1), t1, c.V("ovvv"), 1.0, tWm);
  einsum(c, "nb,mnej->mbej", cx(-1), t1, c.V("oovo"), 1.0, tWm);
  {
    Scope s2(c.ws);
    cplx* u = c.ws.cplxs(o * o * v * v);
    copy_vec(c.L, o * o * v * v, c.t2, u);
    scale_vec(c.L, o * o * v * v, cx(0.5), u);
    einsum(c, "jf,nb->jnfb", cx(1), t1, t1, 1.0, T(u, {o, o, v, v}));
    einsum(c, "jnfb,mnef->mbej", cx(-1), T(u, {o, o, v, v}), c.V("oovv"), 1.0, tWm);
  }
  // ---- singles
  Tensor R1 = T(R, {o, v});
  permute(c.L, c.f("vo").perm({1, 0}), R1, cx(1), false);
  einsum(c, "ie,ae->ia", cx(1), t1, tFae, 1.0, R1);
  einsum(c, "ma,mi->ia", cx(-1), t1, tFmi, 1.0, R1);
  einsum(c, "imae,me->ia", cx(1), t2, tFme, 1.0, R1);
  einsum(c, "nf,naif->ia", cx(-1), t1, c.V("ovov"), 1.0, R1);
  einsum(c, "imef,maef->ia", cx(-0.5), t2, c.V("ovvv"), 1.0, R1);
  einsum(c, "mnae,nmei->ia", cx(-0.5), t2, c.V("oovo"), 1.0, R1);
  // ---- doubles: X4 accumulator (i,j,a,b)
  cplx* x4 = c.ws.cplxs(o * o * v * v);
  Tensor X4 = T(x4, {o, o, v, v});
  fill_zero(c.L, x4, o * o * v * v);
  {
    Scope s2(c.ws);
    cplx* Fb = c.ws.cplxs(v * v);
    copy_vec(c.L, v * v, Fae, Fb);
    einsum(c, "mb,me->be", cx(-0.5), t1, tFme, 1.0, T(Fb, {v, v}));
    einsum(c, "ijae,be->ijab", cx(0.5), t2, T(Fb, {v, v}), 1.0, X4);
    cplx* Fj = c.ws.cplxs(o * o);
    copy_vec(c.L, o * o, Fmi, Fj);
    einsum(c, "je,me->mj", cx(0.5), t1, tFme, 1.0, T(Fj, {o, o}));
    einsum(c, "imab,mj->ijab", cx(-0.5), t2, T(Fj, {o, o}), 1.0, X4);
  }
  einsum(c, "imae,mbej->ijab", cx(1), t2, tWm, 1.0, X4);                // ring
  {
    Scope s2(c.ws);
    cplx* q = c.ws.cplxs(o * o * v * o);
    einsum(c, "ie,mbej->imbj", cx(1), t1, c.V("ovvo"), 0.0, T(q, {o, o, v, o}));
    einsum(c, "ma,imbj->ijab", cx(-1), t1, T(q, {o, o, v, o}), 1.0, X4);
  }
  einsum(c, "ie,abej->ijab", cx(0.5), t1, c.V("vvvo"), 1.0, X4);
  einsum(c, "ma,mbij->ijab", cx(-0.5), t1, c.V("ovoo"), 1.0, X4);
  cplx* R2 = R + c.Ns;
  pack_anti(c, Tensor::make(x4, {1, o, o, v, v}), R2, 1, cx(1), true, false);
  // <ab||ij>
  {
    Tensor vv = c.V("vvoo").perm({2, 3, 0, 1});   // (i,j,a,b), a conjugated view
    Scope s2(c.ws);
    cplx* tmp = c.ws.cplxs(o * o * v * v);
    permute(c.L, vv, T(tmp, {o, o, v, v}), cx(1), false);
    pack_anti(c, Tensor::make(tmp, {1, o, o, v, v}), R2, 1, cx(1), false, true);
  }
  // 1/2 tau_mn^ab W'_mnij  ->  R2[Pij][Pab] += sum_Pmn W'p[Pmn][Pij] tau_p[Pmn][Pab]
  {
    Scope s2(c.ws);
    cplx* Wp = c.ws.cplxs(Po * Po);
    pack_doubles_impl(c.L, Tensor::make(Wmn, {1, o, o, o, o}), Wp, 1, c.o, c.o, cx(1), false, false, c.po, c.po);
    gemm_dispatch(c, true, false, Po, Pv, Po, cx(1), Wp, Po, tap, Pv, cx(1), R2, Pv);
  }
  // ladder, packed: 1/2 tau_ij^ef <ab||ef>
  gemm_dispatch(c, false, true, Po, Pv, Pv, cx(1), tap, Pv, c.vvvv_p, Pv, cx(1), R2, Pv);
  // -1/2 P(ab) tau_ij^ef t_m^b <am||ef>: Z[Pij][(m,a)] = -sum_Pef tau_p <ma||ef>_p, then X[Pij,a,b]
  {
    Scope s2(c.ws);
    cplx* Z = c.ws.cplxs(Po * o * v);
    gemm_dispatch(c, false, true, Po, o * v, Pv, cx(-1), tap, Pv, c.ovvv_p, Pv, cx(0), Z, o * v);
    cplx* X = c.ws.cplxs(Po * v * v);
    einsum(c, "Pma,mb->Pab", cx(1), T(Z, {Po, o, v}), t1, 0.0, T(X, {Po, v, v}));
    pack2(c.L, T(X, {Po, v, v}), R2, Pv, c.pv, cx(-1), true, true);
  }
  // tau tau <mn||ef> (weight 1 over packed pairs): Y[Pij][Pmn] = tau_p . oovv_p^T; R2 += Y tau_p
  {
    Scope s2(c.ws);
    cplx* Y = c.ws.cplxs(Po * Po);
    gemm_dispatch(c, false, true, Po, Po, Pv, cx(1), tap, Pv, c.oovv_p, Pv, cx(0), Y, Po);
    gemm_dispatch(c, false, false, Po, Pv, Po, cx(1), Y, Po, tap, Pv, cx(1), R2, Pv);
  }
}

}  // namespace cclr

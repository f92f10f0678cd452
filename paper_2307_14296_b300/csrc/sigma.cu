// Sigma vectors and property vectors on the device (complex FP64 contractions; the GEMMs go
// through gemm_dispatch, so the tensor-core backend serves the large ones in mixed modes).
//   right sigma  SI Eqs. sigma_sin-ee, sigma_double-ee
//   left sigma   SI Eqs. sigma_sin-ee-left, sigma_double-ee-left
//   xi^X, eta^X, EOM eta^X and (t^X F): SI "Linear response"
// Batched over Z vectors.  Doubles terms are accumulated in one full tensor X4 laid out
// [z][i][a][j][b] so that the o^3 v^3 ring is a single GEMM with no permutation; P(ij)P(ab) is
// applied when X4 is packed (terms carrying only P(ab) or P(ij) enter with weight 1/2, terms
// with neither with weight 1/4).  The o^2 v^4 ladder is a packed GEMM over (e<f).
#include "ctx.h"

namespace cclr {

static inline Tensor T(cplx* p, std::initializer_list<int64_t> d) { return Tensor::make(p, d); }

namespace {

// logical (z,i,j,a,b) view of memory laid out [z][i][a][j][b]
Tensor ring_layout(cplx* p, int64_t Z, int64_t o, int64_t v) {
  Tensor t = Tensor::make(p, {Z, o, o, v, v});
  t.str[0] = o * o * v * v;
  t.str[1] = o * v * v;
  t.str[2] = v;
  t.str[3] = o * v;
  t.str[4] = 1;
  return t;
}

struct Batch {
  cplx *s1, *d2, *full;  // singles [Z][o][v], packed doubles [Z][Po][Pv], full doubles (ring layout)
  Tensor t1, t2;         // views (Z,o,v) and (Z,o,o,v,v)
};

// gather Z vectors of the amplitude layout into contiguous singles/doubles and a full tensor
Batch gather(Ctx& c, int64_t Z, const cplx* in, bool full) {
  Batch b;
  const int64_t o = c.o, v = c.v;
  b.s1 = c.ws.cplxs(Z * o * v);
  b.d2 = c.ws.cplxs(Z * c.Nd);
  Tensor src1 = Tensor::make((cplx*)in, {Z, o * v});
  src1.str[0] = c.N;
  permute(c.L, src1, T(b.s1, {Z, o * v}), cx(1), false);
  Tensor src2 = Tensor::make((cplx*)in + c.Ns, {Z, c.Nd});
  src2.str[0] = c.N;
  permute(c.L, src2, T(b.d2, {Z, c.Nd}), cx(1), false);
  b.t1 = T(b.s1, {Z, o, v});
  b.full = nullptr;
  if (full) {
    b.full = c.ws.cplxs(Z * o * o * v * v);
    b.t2 = ring_layout(b.full, Z, o, v);
    unpack_doubles(c.L, b.d2, c.Nd, b.t2, c.o, c.v);
  }
  return b;
}

void scatter(Ctx& c, int64_t Z, const cplx* s1, const cplx* d2, cplx* out) {
  const int64_t o = c.o, v = c.v;
  Tensor dst1 = Tensor::make(out, {Z, o * v});
  dst1.str[0] = c.N;
  permute(c.L, T((cplx*)s1, {Z, o * v}), dst1, cx(1), false);
  Tensor dst2 = Tensor::make(out + c.Ns, {Z, c.Nd});
  dst2.str[0] = c.N;
  permute(c.L, T((cplx*)d2, {Z, c.Nd}), dst2, cx(1), false);
}

}  // namespace

void sigma_right(Ctx& c, int nvec, const cplx* in, cplx* out) {
  CCLR_REQUIRE(c.have_hbar, CCLR_E_STATE, "sigma: no ground-state amplitudes / Hbar");
  Scope sc(c.ws);
  const int64_t Z = nvec, o = c.o, v = c.v, Po = c.Po, Pv = c.Pv;
  Batch r = gather(c, Z, in, true);
  const size_t cb = c.coarse_sigma ? sizeof(cplx) : 0;   // inputs on the coarse grid (refinement)
  CoarseOperands coarse(c, {{r.s1, cb * Z * o * v}, {r.d2, cb * Z * c.Nd}, {r.full, cb * Z * o * o * v * v}});
  SliceMemo memo(c, r.full, Z * o * o * v * v, 3);   // r_ij^ab is read in three layouts
  Tensor t2 = T(c.t2, {o, o, v, v});
  Tensor Fae = T(c.Fae, {v, v}), Fmi = T(c.Fmi, {o, o}), Fme = T(c.Fme, {o, v});
  Tensor Wmbej = T(c.Wmbej, {o, v, v, o}), Wamef = T(c.Wamef, {v, o, v, v}), Wmnie = T(c.Wmnie, {o, o, o, v});
  // ---- singles
  cplx* s1 = c.ws.cplxs(Z * o * v);
  Tensor S1 = T(s1, {Z, o, v});
  // the Fock-diagonal part of F_ae, F_mi enters exactly as D r at the end
  einsum(c, "ae,zie->zia", cx(1), T(c.Fae_od, {v, v}), r.t1, 0.0, S1);
  einsum(c, "mi,zma->zia", cx(-1), T(c.Fmi_od, {o, o}), r.t1, 1.0, S1);
  einsum(c, "me,zimae->zia", cx(1), Fme, r.t2, 1.0, S1);
  einsum(c, "maei,zme->zia", cx(1), Wmbej, r.t1, 1.0, S1);
  einsum(c, "amef,zimef->zia", cx(0.5), Wamef, r.t2, 1.0, S1);
  einsum(c, "mnie,zmnea->zia", cx(0.5), Wmnie, r.t2, 1.0, S1);
  // ---- doubles
  cplx* x4 = c.ws.cplxs(Z * o * o * v * v);
  Tensor X4 = ring_layout(x4, Z, o, v);
  // ring first (beta = 0 initializes X4); its operand carries the one-index F terms as well
  einsum(c, "zimae,jbme->zijab", cx(1), r.t2, T(c.WringR, {o, v, o, v}), 0.0, X4);
  einsum(c, "mbij,zma->zijab", cx(-0.5), T(c.Wmbij, {o, v, o, o}), r.t1, 1.0, X4);
  einsum(c, "abej,zie->zijab", cx(0.5), T(c.Wabei, {v, v, v, o}), r.t1, 1.0, X4);
  {
    // Terms of the form (W r) t: the packing antisymmetrizer A = (1 - P(ij))(1 - P(ab)) obeys
    // A P(ab) = A P(ij) = -A, so -1/4 Z_af t_ij^fb enters as -1/4 Z_bf t_ij^af (t antisymmetric)
    // and -1/4 Z_ni t_jn^ba as -1/4 Z_nj t_in^ab: the two (W r) intermediates that multiply t the
    // same way are summed first and each pair costs one pass over X4.
    Scope s2(c.ws);
    cplx* bf = c.ws.cplxs(Z * v * v);
    einsum(c, "bmfe,zme->zbf", cx(0.5), Wamef, r.t1, 0.0, T(bf, {Z, v, v}));
    einsum(c, "nmfe,zmnea->zaf", cx(-0.25), c.V("oovv"), r.t2, 1.0, T(bf, {Z, v, v}));
    einsum(c, "zbf,ijaf->zijab", cx(1), T(bf, {Z, v, v}), t2, 1.0, X4);
    cplx* nj = c.ws.cplxs(Z * o * o);
    einsum(c, "nmje,zme->znj", cx(-0.5), Wmnie, r.t1, 0.0, T(nj, {Z, o, o}));
    einsum(c, "nmfe,zimfe->zni", cx(-0.25), c.V("oovv"), r.t2, 1.0, T(nj, {Z, o, o}));
    einsum(c, "znj,inab->zijab", cx(1), T(nj, {Z, o, o}), t2, 1.0, X4);
  }
  // 1/2 P(ab) F_be r_ij^ae and -1/2 P(ij) F_mj r_im^ab are folded into the ring operand (H-bar)
  cplx* s2 = c.ws.cplxs(Z * c.Nd);
  pack_anti(c, X4, s2, Z, cx(1), true, false);
  // ladder 1/2 W_abef r_ij^ef over packed pairs: s2[(z,Pij)][Pab] += r[(z,Pij)][Pef] W[Pab][Pef]
  gemm_dispatch(c, false, true, Z * Po, Pv, Pv, cx(1), r.d2, Pv, c.Wabef_p, Pv, cx(1), s2, Pv);
  // 1/2 W_mnij r_mn^ab: s2_z[Pij][Pab] += sum_Pmn W[Pmn][Pij] r_z[Pmn][Pab]
  for (int64_t z = 0; z < Z; ++z)
    gemm_dispatch(c, true, false, Po, Pv, Po, cx(1), c.Wmnij_p, Po, r.d2 + z * c.Nd, Pv, cx(1), s2 + z * c.Nd, Pv);
  scatter(c, Z, s1, s2, out);
  diag_axpy(c.L, c.N, Z, c.D, in, out);
  c.stats.sigma_calls++;
  c.stats.sigma_vectors += Z;
}

void sigma_left(Ctx& c, int nvec, const cplx* in, cplx* out) {
  CCLR_REQUIRE(c.have_hbar, CCLR_E_STATE, "sigma: no ground-state amplitudes / Hbar");
  Scope sc(c.ws);
  const int64_t Z = nvec, o = c.o, v = c.v, Po = c.Po, Pv = c.Pv;
  Batch l = gather(c, Z, in, true);
  const size_t cb = c.coarse_sigma ? sizeof(cplx) : 0;   // inputs on the coarse grid (refinement)
  CoarseOperands coarse(c, {{l.s1, cb * Z * o * v}, {l.d2, cb * Z * c.Nd}, {l.full, cb * Z * o * o * v * v}});
  SliceMemo memo(c, l.full, Z * o * o * v * v, 3);   // l_ij^ab is read in three layouts
  Tensor t2 = T(c.t2, {o, o, v, v});
  Tensor Fae = T(c.Fae, {v, v}), Fmi = T(c.Fmi, {o, o}), Fme = T(c.Fme, {o, v});
  Tensor Wmbej = T(c.Wmbej, {o, v, v, o}), Wamef = T(c.Wamef, {v, o, v, v}), Wmnie = T(c.Wmnie, {o, o, o, v});
  // G intermediates (Eqs. G_ea, G_mi)
  cplx* gae = c.ws.cplxs(Z * v * v);
  cplx* gmi = c.ws.cplxs(Z * o * o);
  Tensor Gae = T(gae, {Z, v, v}), Gmi = T(gmi, {Z, o, o});
  einsum(c, "mnef,zmnaf->zae", cx(-0.5), t2, l.t2, 0.0, Gae);
  einsum(c, "mnef,zinef->zmi", cx(0.5), t2, l.t2, 0.0, Gmi);
  // ---- singles
  cplx* s1 = c.ws.cplxs(Z * o * v);
  Tensor S1 = T(s1, {Z, o, v});
  // the Fock-diagonal part of F_ae, F_mi enters exactly as D l at the end
  einsum(c, "zie,ea->zia", cx(1), l.t1, T(c.Fae_od, {v, v}), 0.0, S1);
  einsum(c, "zma,im->zia", cx(-1), l.t1, T(c.Fmi_od, {o, o}), 1.0, S1);
  einsum(c, "zimef,efam->zia", cx(0.5), l.t2, T(c.Wabei, {v, v, v, o}), 1.0, S1);
  einsum(c, "zmnae,iemn->zia", cx(-0.5), l.t2, T(c.Wmbij, {o, v, o, o}), 1.0, S1);
  einsum(c, "zef,eifa->zia", cx(-1), Gae, Wamef, 1.0, S1);
  einsum(c, "zmn,mina->zia", cx(-1), Gmi, Wmnie, 1.0, S1);
  einsum(c, "zme,ieam->zia", cx(1), l.t1, Wmbej, 1.0, S1);
  // ---- doubles
  cplx* x4 = c.ws.cplxs(Z * o * o * v * v);
  Tensor X4 = ring_layout(x4, Z, o, v);
  einsum(c, "zimae,jbme->zijab", cx(1), l.t2, T(c.WringL, {o, v, o, v}), 0.0, X4);
  // 1/2 P(ab) l_ij^ae F_eb and -1/2 P(ij) l_im^ab F_jm are folded into the ring operand (H-bar)
  einsum(c, "ijae,zbe->zijab", cx(0.5), c.V("oovv"), Gae, 1.0, X4);
  einsum(c, "zma,ijmb->zijab", cx(-0.5), l.t1, Wmnie, 1.0, X4);
  einsum(c, "imab,zmj->zijab", cx(-0.5), c.V("oovv"), Gmi, 1.0, X4);
  einsum(c, "zie,ejab->zijab", cx(0.5), l.t1, Wamef, 1.0, X4);
  einsum(c, "zia,jb->zijab", cx(1), l.t1, Fme, 1.0, X4);
  cplx* s2 = c.ws.cplxs(Z * c.Nd);
  pack_anti(c, X4, s2, Z, cx(1), true, false);
  // ladder 1/2 l_ij^ef W_efab: s2[(z,Pij)][Pab] += l[(z,Pij)][Pef] W[Pef][Pab]
  gemm_dispatch(c, false, false, Z * Po, Pv, Pv, cx(1), l.d2, Pv, c.Wabef_p, Pv, cx(1), s2, Pv);
  // 1/2 l_mn^ab W_ijmn: s2_z[Pij][Pab] += sum_Pmn W[Pij][Pmn] l_z[Pmn][Pab]
  for (int64_t z = 0; z < Z; ++z)
    gemm_dispatch(c, false, false, Po, Pv, Po, cx(1), c.Wmnij_p, Po, l.d2 + z * c.Nd, Pv, cx(1), s2 + z * c.Nd, Pv);
  scatter(c, Z, s1, s2, out);
  diag_axpy(c.L, c.N, Z, c.D, in, out);
  c.stats.sigma_calls++;
  c.stats.sigma_vectors += Z;
}

// xi^X (SI Eq. xi-equation, programmable form)
void xi_vec(Ctx& c, const cplx* Xd, cplx* out) {
  Scope sc(c.ws);
  const int64_t o = c.o, v = c.v, n = c.n;
  Tensor X = T((cplx*)Xd, {n, n});
  auto blk = [&](bool ro, bool co) {
    Tensor t = X;
    t.dim[0] = ro ? o : v;
    t.dim[1] = co ? o : v;
    t.p = (cplx*)Xd + (ro ? 0 : o * n) + (co ? 0 : o);
    return t;
  };
  Tensor Xoo = blk(true, true), Xov = blk(true, false), Xvo = blk(false, true), Xvv = blk(false, false);
  Tensor t1 = T(c.t, {o, v}), t2 = T(c.t2, {o, o, v, v});
  Tensor S1 = T(out, {o, v});
  permute(c.L, Xvo.perm({1, 0}), S1, cx(1), false);
  einsum(c, "ae,ie->ia", cx(1), Xvv, t1, 1.0, S1);
  einsum(c, "mi,ma->ia", cx(-1), Xoo, t1, 1.0, S1);
  cplx* xmi = c.ws.cplxs(o * o);
  einsum(c, "me,ie->mi", cx(1), Xov, t1, 0.0, T(xmi, {o, o}));
  einsum(c, "mi,ma->ia", cx(-1), T(xmi, {o, o}), t1, 1.0, S1);
  einsum(c, "me,imae->ia", cx(1), Xov, t2, 1.0, S1);
  cplx* x4 = c.ws.cplxs(o * o * v * v);
  Tensor X4 = ring_layout(x4, 1, o, v);
  Tensor X4r = X4;  // drop the z axis for 4-index einsums
  X4r.rank = 4;
  for (int k = 0; k < 4; ++k) { X4r.dim[k] = X4.dim[k + 1]; X4r.str[k] = X4.str[k + 1]; }
  einsum(c, "bf,ijaf->ijab", cx(0.5), Xvv, t2, 0.0, X4r);
  einsum(c, "mj,imab->ijab", cx(-0.5), Xoo, t2, 1.0, X4r);
  einsum(c, "mi,mjab->ijab", cx(-0.5), T(xmi, {o, o}), t2, 1.0, X4r);
  cplx* xfa = c.ws.cplxs(v * v);
  einsum(c, "mf,ma->fa", cx(1), Xov, t1, 0.0, T(xfa, {v, v}));
  einsum(c, "fa,ijfb->ijab", cx(-0.5), T(xfa, {v, v}), t2, 1.0, X4r);
  pack_anti(c, X4, out + c.Ns, 1, cx(1), true, false);
}

// eta^X (SI Eq. eta-equation), optionally EOM eta^X (+ lambda_ij^ab xi^X_jb in the singles)
void eta_vec(Ctx& c, const cplx* Xd, bool eom, cplx* out) {
  CCLR_REQUIRE(c.have_lambda, CCLR_E_STATE, "eta: Lambda not available");
  Scope sc(c.ws);
  const int64_t o = c.o, v = c.v, n = c.n;
  auto blk = [&](bool ro, bool co) {
    Tensor t = T((cplx*)Xd, {n, n});
    t.dim[0] = ro ? o : v;
    t.dim[1] = co ? o : v;
    t.p = (cplx*)Xd + (ro ? 0 : o * n) + (co ? 0 : o);
    return t;
  };
  Tensor Xoo = blk(true, true), Xov = blk(true, false), Xvv = blk(false, false);
  Tensor t1 = T(c.t, {o, v}), t2 = T(c.t2, {o, o, v, v});
  Tensor l1 = T(c.lam, {o, v}), l2 = T(c.l2, {o, o, v, v});
  Tensor S1 = T(out, {o, v});
  permute(c.L, Xov, S1, cx(1), false);
  einsum(c, "ea,ie->ia", cx(1), Xvv, l1, 1.0, S1);
  einsum(c, "im,ma->ia", cx(-1), Xoo, l1, 1.0, S1);
  cplx* tae = c.ws.cplxs(v * v);
  einsum(c, "ma,me->ae", cx(1), Xov, t1, 0.0, T(tae, {v, v}));
  einsum(c, "ae,ie->ia", cx(-1), T(tae, {v, v}), l1, 1.0, S1);
  cplx* tim = c.ws.cplxs(o * o);
  einsum(c, "ie,me->im", cx(1), Xov, t1, 0.0, T(tim, {o, o}));
  einsum(c, "im,ma->ia", cx(-1), T(tim, {o, o}), l1, 1.0, S1);
  cplx* gni = c.ws.cplxs(o * o);
  einsum(c, "mnfe,mife->ni", cx(1), t2, l2, 0.0, T(gni, {o, o}));
  einsum(c, "ni,na->ia", cx(-0.5), T(gni, {o, o}), Xov, 1.0, S1);
  cplx* gea = c.ws.cplxs(v * v);
  einsum(c, "nmfe,nmfa->ea", cx(1), t2, l2, 0.0, T(gea, {v, v}));
  einsum(c, "ea,ie->ia", cx(-0.5), T(gea, {v, v}), Xov, 1.0, S1);
  cplx* x4 = c.ws.cplxs(o * o * v * v);
  Tensor X4 = ring_layout(x4, 1, o, v);
  Tensor X4r = X4;
  X4r.rank = 4;
  for (int k = 0; k < 4; ++k) { X4r.dim[k] = X4.dim[k + 1]; X4r.str[k] = X4.str[k + 1]; }
  einsum(c, "ia,jb->ijab", cx(1), l1, Xov, 0.0, X4r);
  einsum(c, "ijae,eb->ijab", cx(0.5), l2, Xvv, 1.0, X4r);
  einsum(c, "imab,jm->ijab", cx(-0.5), l2, Xoo, 1.0, X4r);
  cplx* q = c.ws.cplxs(o * o * v * o);
  einsum(c, "me,ijae->ijam", cx(1), t1, l2, 0.0, T(q, {o, o, v, o}));
  einsum(c, "ijam,mb->ijab", cx(-0.5), T(q, {o, o, v, o}), Xov, 1.0, X4r);
  cplx* jm = c.ws.cplxs(o * o);
  einsum(c, "me,je->jm", cx(1), t1, Xov, 0.0, T(jm, {o, o}));
  einsum(c, "imab,jm->ijab", cx(-0.5), l2, T(jm, {o, o}), 1.0, X4r);
  pack_anti(c, X4, out + c.Ns, 1, cx(1), true, false);
  if (eom) {
    cplx* xi = c.ws.cplxs(c.N);
    xi_vec(c, Xd, xi);
    einsum(c, "ijab,jb->ia", cx(1), l2, T(xi, {o, v}), 1.0, S1);
  }
}

// Operator densities: the n x n matrices D with l . xi^X = sum_pq D[p,q] X[p,q] (xi_density) and
// eta^X . v = sum_pq D[p,q] X[p,q] (eta_density), the transposes of the xi and eta formulas above
// (both are linear in X; bilinear products over unique excitations, doubles with the weights of
// the antisymmetrizers).  l, v in the amplitude layout; D (device, n x n row-major) is written.
namespace {
struct Blocks {   // the oo, ov, vo, vv views of an n x n matrix
  Tensor oo, ov, vo, vv;
};
Blocks blocks_of(cplx* D, int64_t o, int64_t v) {
  const int64_t n = o + v;
  auto blk = [&](bool ro, bool co) {
    Tensor t = Tensor::make(D, {n, n});
    t.dim[0] = ro ? o : v;
    t.dim[1] = co ? o : v;
    t.p = D + (ro ? 0 : o * n) + (co ? 0 : o);
    return t;
  };
  return Blocks{blk(true, true), blk(true, false), blk(false, true), blk(false, false)};
}
}  // namespace

void xi_density(Ctx& c, const cplx* l, cplx* D) {
  Scope sc(c.ws);
  const int64_t o = c.o, v = c.v, n = c.n;
  fill_zero(c.L, D, n * n);
  Blocks d = blocks_of(D, o, v);
  Tensor t1 = T(c.t, {o, v}), t2 = T(c.t2, {o, o, v, v});
  Tensor l1 = T((cplx*)l, {o, v});
  cplx* l2f = c.ws.cplxs(o * o * v * v);
  expand_t2(c, l + c.Ns, l2f, 1);
  Tensor l2 = T(l2f, {o, o, v, v});
  permute(c.L, l1.perm({1, 0}), d.vo, cx(1), false);                        // X_ai
  einsum(c, "ia,ie->ae", cx(1), l1, t1, 1.0, d.vv);                          // X_ae t_i^e
  einsum(c, "ia,ma->mi", cx(-1), l1, t1, 1.0, d.oo);                         // -X_mi t_m^a
  cplx* k = c.ws.cplxs(o * o);
  Tensor K = T(k, {o, o});
  einsum(c, "ia,ma->im", cx(1), l1, t1, 0.0, K);
  einsum(c, "ie,im->me", cx(-1), t1, K, 1.0, d.ov);                          // -X_me t_i^e t_m^a
  einsum(c, "ia,imae->me", cx(1), l1, t2, 1.0, d.ov);                        // X_me t_im^ae
  einsum(c, "ijab,ijaf->bf", cx(0.5), l2, t2, 1.0, d.vv);                    // P(ab) X_bf t_ij^af
  einsum(c, "ijab,imab->mj", cx(-0.5), l2, t2, 1.0, d.oo);                   // -P(ij) X_mj t_im^ab
  cplx* pim = c.ws.cplxs(o * o);
  einsum(c, "ijab,mjab->im", cx(1), l2, t2, 0.0, T(pim, {o, o}));
  einsum(c, "ie,im->me", cx(-0.5), t1, T(pim, {o, o}), 1.0, d.ov);           // -P(ij) X_me t_i^e t_mj^ab
  cplx* qaf = c.ws.cplxs(v * v);
  einsum(c, "ijab,ijfb->af", cx(1), l2, t2, 0.0, T(qaf, {v, v}));
  einsum(c, "ma,af->mf", cx(-0.5), t1, T(qaf, {v, v}), 1.0, d.ov);           // -P(ab) X_mf t_m^a t_ij^fb
}

void eta_density(Ctx& c, const cplx* vv, cplx* D) {
  CCLR_REQUIRE(c.have_lambda, CCLR_E_STATE, "eta density: Lambda not available");
  Scope sc(c.ws);
  const int64_t o = c.o, v = c.v, n = c.n;
  fill_zero(c.L, D, n * n);
  Blocks d = blocks_of(D, o, v);
  Tensor t1 = T(c.t, {o, v}), t2 = T(c.t2, {o, o, v, v});
  Tensor l1 = T(c.lam, {o, v}), l2 = T(c.l2, {o, o, v, v});
  Tensor v1 = T((cplx*)vv, {o, v});
  cplx* v2f = c.ws.cplxs(o * o * v * v);
  expand_t2(c, vv + c.Ns, v2f, 1);
  Tensor v2 = T(v2f, {o, o, v, v});
  permute(c.L, v1, d.ov, cx(1), true);                                       // X_ia
  einsum(c, "ie,ia->ea", cx(1), l1, v1, 1.0, d.vv);                          // X_ea l_i^e
  einsum(c, "ia,ma->im", cx(-1), v1, l1, 1.0, d.oo);                         // -X_im l_m^a
  cplx* ea = c.ws.cplxs(v * v);
  einsum(c, "ie,ia->ea", cx(1), l1, v1, 0.0, T(ea, {v, v}));
  einsum(c, "me,ea->ma", cx(-1), t1, T(ea, {v, v}), 1.0, d.ov);              // -X_ma t_m^e l_i^e
  cplx* im = c.ws.cplxs(o * o);
  einsum(c, "ia,ma->im", cx(1), v1, l1, 0.0, T(im, {o, o}));
  einsum(c, "im,me->ie", cx(-1), T(im, {o, o}), t1, 1.0, d.ov);              // -X_ie t_m^e l_m^a
  cplx* g = c.ws.cplxs(o * o);
  einsum(c, "mnfe,mife->ni", cx(1), t2, l2, 0.0, T(g, {o, o}));
  einsum(c, "ni,ia->na", cx(-0.5), T(g, {o, o}), v1, 1.0, d.ov);             // -1/2 G_ni X_na
  cplx* h = c.ws.cplxs(v * v);
  einsum(c, "nmfe,nmfa->ea", cx(1), t2, l2, 0.0, T(h, {v, v}));
  einsum(c, "ea,ia->ie", cx(-0.5), T(h, {v, v}), v1, 1.0, d.ov);             // -1/2 H_ea X_ie
  einsum(c, "ijab,ia->jb", cx(1), v2, l1, 1.0, d.ov);                        // P(ij)P(ab) l_i^a X_jb
  cplx* kk = c.ws.cplxs(v * v);
  einsum(c, "ijae,ijab->eb", cx(1), l2, v2, 0.0, T(kk, {v, v}));
  permute(c.L, T(kk, {v, v}), d.vv, cx(0.5), true);                          // P(ab) l_ij^ae X_eb
  einsum(c, "me,eb->mb", cx(-0.5), t1, T(kk, {v, v}), 1.0, d.ov);            // -P(ab) t_m^e l_ij^ae X_mb
  cplx* jj = c.ws.cplxs(o * o);
  einsum(c, "ijab,imab->jm", cx(1), v2, l2, 0.0, T(jj, {o, o}));
  permute(c.L, T(jj, {o, o}), d.oo, cx(-0.5), true);                         // -P(ij) l_im^ab X_jm
  einsum(c, "jm,me->je", cx(-0.5), T(jj, {o, o}), t1, 1.0, d.ov);            // -P(ij) t_m^e l_im^ab X_je
}

// eta of the Lambda equations: dE/dt = (F_me, <ij||ab>) in the amplitude layout
void eta_ground(Ctx& c, cplx* out) {
  copy_vec(c.L, c.Ns, c.Fme, out);
  copy_vec(c.L, c.Nd, c.oovv_p, out + c.Ns);
}

// Hessian product (u F) (SI, "(t^X F)" equations); lambda-only pieces are built once per Lambda.
void hessian_right(Ctx& c, int nvec, const cplx* in, cplx* out) {
  CCLR_REQUIRE(c.have_lambda && c.have_hbar, CCLR_E_STATE, "hessian: Lambda not available");
  const int64_t Z = nvec, o = c.o, v = c.v, Po = c.Po, Pv = c.Pv;
  Tensor t2 = T(c.t2, {o, o, v, v});
  Tensor l1 = T(c.lam, {o, v}), l2 = T(c.l2, {o, o, v, v});
  Tensor Fme = T(c.Fme, {o, v}), Wamef = T(c.Wamef, {v, o, v, v}), Wmnie = T(c.Wmnie, {o, o, o, v});
  Tensor Wmbej = T(c.Wmbej, {o, v, v, o});
  Tensor oovv = c.V("oovv");
  // lambda-only pieces
  if (!c.named.count("F.Y")) {
    cplx* Y = c.dalloc(o * o * v * v);   // <ki||ca> + 1/2 l_ki^ef W_efca + 1/2 W_kimn l_mn^ca
    cplx* G1 = c.dalloc(v * v);          // G1[f,c] = l_mn^ec t_mn^ef
    cplx* G2 = c.dalloc(o * o);          // G2[k,n] = l_mk^ef t_mn^ef
    c.named["F.Y"] = Y;
    c.named["F.G1"] = G1;
    c.named["F.G2"] = G2;
  }
  if (!c.named.count("F.ready")) {
    Scope sc(c.ws);
    cplx* Y = (cplx*)c.named["F.Y"];
    permute(c.L, oovv, T(Y, {o, o, v, v}), cx(1), false);
    // 1/2 sum_ef l_ki^ef W_efca = sum_Pef l_p[Pki][Pef] W_p[Pef][Pca] (packed), then expand
    cplx* lp = c.lam + c.Ns;
    cplx* yp = c.ws.cplxs(Po * Pv);
    gemm_dispatch(c, false, false, Po, Pv, Pv, cx(1), lp, Pv, c.Wabef_p, Pv, cx(0), yp, Pv);
    // 1/2 sum_mn W_kimn l_mn^ca = sum_Pmn W_p[Pki][Pmn] l_p[Pmn][Pca]
    gemm_dispatch(c, false, false, Po, Pv, Po, cx(1), c.Wmnij_p, Po, lp, Pv, cx(1), yp, Pv);
    cplx* yf = c.ws.cplxs(o * o * v * v);
    expand_t2(c, yp, yf, 1);
    permute(c.L, T(yf, {o, o, v, v}), T(Y, {o, o, v, v}), cx(1), true);
    einsum(c, "mnec,mnef->fc", cx(1), l2, t2, 0.0, T((cplx*)c.named["F.G1"], {v, v}));
    einsum(c, "mkef,mnef->kn", cx(1), l2, t2, 0.0, T((cplx*)c.named["F.G2"], {o, o}));
    c.named["F.ready"] = (void*)1;
  }
  Tensor Y = T((cplx*)c.named["F.Y"], {o, o, v, v});
  Tensor G1 = T((cplx*)c.named["F.G1"], {v, v}), G2 = T((cplx*)c.named["F.G2"], {o, o});

  Scope sc(c.ws);
  Batch u = gather(c, Z, in, true);
  SliceMemo memo(c, u.full, Z * o * o * v * v, 7);   // u_ij^ab is read in seven layouts
  Tensor u1 = u.t1, u2 = u.t2;
  cplx* s1 = c.ws.cplxs(Z * o * v);
  Tensor S = T(s1, {Z, o, v});
  auto tmp = [&](std::initializer_list<int64_t> d) {
    int64_t nn = 1;
    for (auto x : d) nn *= x;
    return Tensor::make(c.ws.cplxs(nn), d);
  };
  // ---- singles (k,c)
  einsum(c, "kica,zia->zkc", cx(1), Y, u1, 0.0, S);                          // terms 1, 13, 14
  { Tensor t = tmp({Z, o, o}); einsum(c, "ka,zia->zik", cx(1), Fme, u1, 0.0, t);
    einsum(c, "ic,zik->zkc", cx(-1), l1, t, 1.0, S); }
  { Tensor t = tmp({Z, v, v}); einsum(c, "ic,zia->zca", cx(1), Fme, u1, 0.0, t);
    einsum(c, "ka,zca->zkc", cx(-1), l1, t, 1.0, S); }
  { Tensor t = tmp({Z, v, v}); einsum(c, "eica,zia->zec", cx(1), Wamef, u1, 0.0, t);
    einsum(c, "ke,zec->zkc", cx(1), l1, t, 1.0, S); }
  { Tensor t = tmp({Z, o, o}); einsum(c, "kima,zia->zkm", cx(1), Wmnie, u1, 0.0, t);
    einsum(c, "mc,zkm->zkc", cx(-1), l1, t, 1.0, S); }
  { Tensor t = tmp({Z, o, o}); einsum(c, "ma,zia->zim", cx(1), l1, u1, 0.0, t);
    einsum(c, "ikmc,zim->zkc", cx(-1), Wmnie, t, 1.0, S); }
  { Tensor t = tmp({Z, v, v}); einsum(c, "ie,zia->zea", cx(1), l1, u1, 0.0, t);
    einsum(c, "ekac,zea->zkc", cx(1), Wamef, t, 1.0, S); }
  { Tensor t = tmp({Z, o, o}); einsum(c, "kjab,zijab->zki", cx(1), oovv, u2, 0.0, t);
    einsum(c, "ic,zki->zkc", cx(-0.5), l1, t, 1.0, S); }
  { Tensor t = tmp({Z, v, v}); einsum(c, "ijcb,zijab->zca", cx(1), oovv, u2, 0.0, t);
    einsum(c, "ka,zca->zkc", cx(-0.5), l1, t, 1.0, S); }
  { Tensor t = tmp({Z, o, v}); einsum(c, "ia,zijab->zjb", cx(1), l1, u2, 0.0, t);
    einsum(c, "jkbc,zjb->zkc", cx(1), oovv, t, 1.0, S); }
  { // -l_mk^ae W^{ie}_{mc} u_i^a with W^{ie}_{mc} = -W_mbej[i,e,c,m]
    Tensor t = tmp({Z, o, o, v, o}); einsum(c, "mkae,zia->zmkei", cx(1), l2, u1, 0.0, t);
    einsum(c, "zmkei,iecm->zkc", cx(1), t, Wmbej, 1.0, S); }
  { // -l_im^ec W^{ek}_{am} u_i^a with W^{ek}_{am} = -W_mbej[k,e,a,m]
    Tensor t = tmp({Z, v, o, o, o}); einsum(c, "keam,zia->zekmi", cx(1), Wmbej, u1, 0.0, t);
    einsum(c, "imec,zekmi->zkc", cx(1), l2, t, 1.0, S); }
  { Tensor t = tmp({Z, o, v}); einsum(c, "kifa,zia->zkf", cx(1), oovv, u1, 0.0, t);
    einsum(c, "fc,zkf->zkc", cx(-0.5), G1, t, 1.0, S); }
  { Tensor t = tmp({Z, o, v}); einsum(c, "nica,zia->znc", cx(1), oovv, u1, 0.0, t);
    einsum(c, "kn,znc->zkc", cx(-0.5), G2, t, 1.0, S); }
  { Tensor t = tmp({Z, o, v}); einsum(c, "fa,zia->zif", cx(1), G1, u1, 0.0, t);
    einsum(c, "ikfc,zif->zkc", cx(-0.5), oovv, t, 1.0, S); }
  { Tensor t = tmp({Z, o, v}); einsum(c, "in,zia->zna", cx(1), G2, u1, 0.0, t);
    einsum(c, "nkac,zna->zkc", cx(-0.5), oovv, t, 1.0, S); }
  { Tensor t = tmp({Z, v, v}); einsum(c, "ijac,zijab->zcb", cx(1), l2, u2, 0.0, t);
    einsum(c, "kb,zcb->zkc", cx(-0.5), Fme, t, 1.0, S); }
  { Tensor t = tmp({Z, o, o}); einsum(c, "ikab,zijab->zkj", cx(1), l2, u2, 0.0, t);
    einsum(c, "jc,zkj->zkc", cx(-0.5), Fme, t, 1.0, S); }
  { Tensor t = tmp({Z, o, v, o, v}); einsum(c, "ikeb,zijab->zkeja", cx(1), l2, u2, 0.0, t);
    einsum(c, "zkeja,ejac->zkc", cx(-1), t, Wamef, 1.0, S); }
  { Tensor t = tmp({Z, o, o, o, v}); einsum(c, "ikmb,zijab->zkmja", cx(1), Wmnie, u2, 0.0, t);
    einsum(c, "mjac,zkmja->zkc", cx(1), l2, t, 1.0, S); }
  { Tensor t = tmp({Z, v, o, o, o}); einsum(c, "ekab,zijab->zekij", cx(1), Wamef, u2, 0.0, t);
    einsum(c, "ijec,zekij->zkc", cx(-0.25), l2, t, 1.0, S); }
  { Tensor t = tmp({Z, o, o, o, o}); einsum(c, "mkab,zijab->zmkij", cx(1), l2, u2, 0.0, t);
    einsum(c, "ijmc,zmkij->zkc", cx(0.25), Wmnie, t, 1.0, S); }
  { Tensor t = tmp({Z, v, v}); einsum(c, "ijae,zijab->zeb", cx(1), l2, u2, 0.0, t);
    einsum(c, "ekbc,zeb->zkc", cx(0.5), Wamef, t, 1.0, S); }
  { Tensor t = tmp({Z, o, o}); einsum(c, "imab,zijab->zmj", cx(1), l2, u2, 0.0, t);
    einsum(c, "jkmc,zmj->zkc", cx(-0.5), Wmnie, t, 1.0, S); }

  // ---- doubles (k,l,c,d): X4 weights 1 (P(kl)P(cd)), 1/2 (one P), 1/4 (none)
  cplx* x4 = c.ws.cplxs(Z * o * o * v * v);
  Tensor X4 = ring_layout(x4, Z, o, v);
  fill_zero(c.L, x4, Z * o * o * v * v);
  { Tensor t = tmp({Z, o, v}); einsum(c, "lida,zia->zld", cx(1), oovv, u1, 0.0, t);
    einsum(c, "kc,zld->zklcd", cx(1), l1, t, 1.0, X4); }
  // The remaining terms share their outer operand in groups.  With the packing antisymmetrizer
  // A = (1 - P(kl))(1 - P(cd)) (A P(kl) = A P(cd) = -A, A P(kl) P(cd) = A) every group is rewritten
  // onto one index pattern, its (u-dependent) intermediates are summed, and the group costs one
  // product and one pass over X4.
  { // <il||cd> (-1/2 l_ka u_ia - 1/4 l_ik^ab u_ij^ab)
    Tensor t = tmp({Z, o, o});
    einsum(c, "ka,zia->zki", cx(-0.5), l1, u1, 0.0, t);
    einsum(c, "ikab,zijab->zkj", cx(-0.25), l2, u2, 1.0, t);
    einsum(c, "zki,ilcd->zklcd", cx(1), t, oovv, 1.0, X4); }
  { // <kl||ad> (-1/2 l_ic u_ia - 1/4 l_ij^ac u_ij^ab)
    Tensor t = tmp({Z, v, v});
    einsum(c, "ic,zia->zca", cx(-0.5), l1, u1, 0.0, t);
    einsum(c, "ijac,zijab->zcb", cx(-0.25), l2, u2, 1.0, t);
    einsum(c, "zca,klad->zklcd", cx(1), t, oovv, 1.0, X4); }
  { // l_ki^cd (-1/2 F_la u_ia - 1/2 W_lima u_ia - 1/4 <lj||ab> u_ij^ab)
    Tensor t = tmp({Z, o, o});
    einsum(c, "la,zia->zli", cx(-0.5), Fme, u1, 0.0, t);
    einsum(c, "lima,zia->zlm", cx(-0.5), Wmnie, u1, 1.0, t);
    einsum(c, "ljab,zijab->zli", cx(-0.25), oovv, u2, 1.0, t);
    einsum(c, "kicd,zli->zklcd", cx(1), l2, t, 1.0, X4); }
  { // l_kl^ca (-1/2 F_id u_ia + 1/2 W_eida u_ia (as its transpose) - 1/4 <ij||db> u_ij^ab)
    Tensor t = tmp({Z, v, v});
    einsum(c, "id,zia->zda", cx(-0.5), Fme, u1, 0.0, t);
    einsum(c, "eida,zia->zde", cx(0.5), Wamef, u1, 1.0, t);
    einsum(c, "ijdb,zijab->zda", cx(-0.25), oovv, u2, 1.0, t);
    einsum(c, "klca,zda->zklcd", cx(1), l2, t, 1.0, X4); }
  { // l_mi^cd (1/4 W_klma u_ia + 1/16 <kl||ab> u_mi^ab)
    Tensor t = tmp({Z, o, o, o, o});
    einsum(c, "klma,zia->zklmi", cx(0.25), Wmnie, u1, 0.0, t);
    einsum(c, "klab,zijab->zklij", cx(0.0625), oovv, u2, 1.0, t);
    einsum(c, "micd,zklmi->zklcd", cx(1), l2, t, 1.0, X4); }
  { // ring-shaped terms on l_ml^ca: W_kimd u_ia, <li||da> u_ij^ab (under P(kl)) and
    // -l_ki^ed W_elca u_ia (under P(kl)P(cd), i.e. -W_ekdf u_if at (k,i,d,e))
    Tensor t = tmp({Z, o, o, v, v});
    einsum(c, "kimd,zia->zkmda", cx(1), Wmnie, u1, 0.0, t);
    einsum(c, "lida,zijab->zljdb", cx(1), oovv, u2, 1.0, t);
    einsum(c, "ekdf,zif->zkide", cx(-1), Wamef, u1, 1.0, t);
    einsum(c, "mlca,zkmda->zklcd", cx(1), l2, t, 1.0, X4); }
  { Tensor t = tmp({Z, o, o, v, o}); einsum(c, "klea,zia->zklei", cx(1), l2, u1, 0.0, t);
    einsum(c, "zklei,eicd->zklcd", cx(-0.25), t, Wamef, 1.0, X4); }
  { Tensor t = tmp({Z, o, o, o, o}); einsum(c, "klab,zijab->zklij", cx(1), l2, u2, 0.0, t);
    einsum(c, "zklij,ijcd->zklcd", cx(0.0625), t, oovv, 1.0, X4); }
  cplx* s2 = c.ws.cplxs(Z * c.Nd);
  pack_anti(c, X4, s2, Z, cx(1), true, false);
  scatter(c, Z, s1, s2, out);
  c.stats.sigma_calls++;
  c.stats.sigma_vectors += Z;
}

}  // namespace cclr

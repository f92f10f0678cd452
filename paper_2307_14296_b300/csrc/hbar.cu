// Hbar intermediates (SI, "EOM-EE sigma-vectors and intermediates", Eqs. F_im ... tau), built
// once per ground state (the paper's step 2).  Elements are stored creators-first:
// W[p,q,r,s] multiplies {p+ q+ s r}.  Readings of garbled index placements follow the
// derivative definition dOmega/dt (the oracle's tests pin them):
//   F_ae uses -f_me t_m^a, W_iemn uses -F_if t_mn^ef, the vvvo element is the standard one.
#include "ctx.h"

namespace cclr {

static inline Tensor T(cplx* p, std::initializer_list<int64_t> d) { return Tensor::make(p, d); }

void build_hbar(Ctx& c) {
  ++c.data_gen;
  const int64_t o = c.o, v = c.v, Po = c.Po, Pv = c.Pv;
  auto ensure = [&](cplx*& p, int64_t n) { if (!p) p = c.dalloc(n); };
  ensure(c.Fae, v * v);
  ensure(c.Fmi, o * o);
  ensure(c.Fae_od, v * v);
  ensure(c.Fmi_od, o * o);
  ensure(c.Fme, o * v);
  ensure(c.Wmnij, o * o * o * o);
  ensure(c.Wmnij_p, Po * Po);
  ensure(c.Wabef_p, Pv * Pv);
  ensure(c.Wmbej, o * v * v * o);
  ensure(c.WringR, o * v * o * v);
  ensure(c.WringL, o * v * o * v);
  ensure(c.Wmnie, o * o * o * v);
  ensure(c.Wamef, v * o * v * v);
  ensure(c.Wmbij, o * v * o * o);
  ensure(c.Wabei, v * v * v * o);
  ensure(c.tau, o * o * v * v);
  Scope sc(c.ws);
  Tensor t1 = T(c.t, {o, v}), t2 = T(c.t2, {o, o, v, v});
  // tau (Eq. tau) and its packed form
  copy_vec(c.L, o * o * v * v, c.t2, c.tau);
  Tensor ta = T(c.tau, {o, o, v, v});
  einsum(c, "ia,jb->ijab", cx(1), t1, t1, 1.0, ta);
  einsum(c, "ib,ja->ijab", cx(-1), t1, t1, 1.0, ta);
  cplx* tap = c.ws.cplxs(Po * Pv);
  pack_anti(c, Tensor::make(c.tau, {1, o, o, v, v}), tap, 1, cx(1), false, false);

  // one-body (Eqs. F_me, F_im, F_ea)
  Tensor Fme = T(c.Fme, {o, v}), Fmi = T(c.Fmi, {o, o}), Fae = T(c.Fae, {v, v});
  permute(c.L, c.f("ov"), Fme, cx(1), false);
  einsum(c, "nf,mnef->me", cx(1), t1, c.V("oovv"), 1.0, Fme);
  permute(c.L, c.f("oo"), Fmi, cx(1), false);
  einsum(c, "ie,me->mi", cx(1), t1, c.f("ov"), 1.0, Fmi);
  einsum(c, "ne,mnie->mi", cx(1), t1, c.V("ooov"), 1.0, Fmi);
  einsum(c, "inef,mnef->mi", cx(0.5), ta, c.V("oovv"), 1.0, Fmi);
  permute(c.L, c.f("vv"), Fae, cx(1), false);
  einsum(c, "ma,me->ae", cx(-1), t1, c.f("ov"), 1.0, Fae);
  einsum(c, "mf,amef->ae", cx(1), t1, c.V("vovv"), 1.0, Fae);
  einsum(c, "mnaf,mnef->ae", cx(-0.5), ta, c.V("oovv"), 1.0, Fae);

  // W_mnij (Eq. W_ijmn) full and packed [P(m,n)][P(i,j)]
  Tensor Wmnij = T(c.Wmnij, {o, o, o, o});
  permute(c.L, c.V("oooo"), Wmnij, cx(1), false);
  einsum(c, "je,mnie->mnij", cx(1), t1, c.V("ooov"), 1.0, Wmnij);
  einsum(c, "ie,mnje->mnij", cx(-1), t1, c.V("ooov"), 1.0, Wmnij);
  einsum(c, "ijef,mnef->mnij", cx(0.5), ta, c.V("oovv"), 1.0, Wmnij);
  pack_doubles_impl(c.L, Tensor::make(c.Wmnij, {1, o, o, o, o}), c.Wmnij_p, 1, c.o, c.o, cx(1), false, false, c.po,
                    c.po);

  // W_abef packed [P(a,b)][P(e,f)] (Eq. W_efab):
  //   <ab||ef> - P(ab) t_m^b <am||ef> + 1/2 tau_mn^ab <mn||ef>
  copy_vec(c.L, Pv * Pv, c.vvvv_p, c.Wabef_p);
  {
    Scope s2(c.ws);
    // Y[a][b][Pef] = sum_m <ma||ef>_p t_m^b ; -P(ab) t_mb <am||ef> = +P(ab) Y
    cplx* Y = c.ws.cplxs(v * v * Pv);
    einsum(c, "maP,mb->abP", cx(1), T(c.ovvv_p, {o, v, Pv}), t1, 0.0, T(Y, {v, v, Pv}));
    // Wabef_p[P(a,b)][e f] += Y[a,b,:] - Y[b,a,:]: pack over the leading pair of Y viewed (m, m, R)
    Tensor Yv = T(Y, {v, v, Pv}).perm({2, 0, 1});   // (R=Pef, a, b)
    // write transposed: D[P(a,b)*Pv + Pef] -> use a (Pef, a, b) view and a transposed destination
    cplx* tmp = c.ws.cplxs(Pv * Pv);
    pack2(c.L, Yv, tmp, Pv, c.pv, cx(1), true, false);                  // tmp[Pef][Pab]
    // Wabef_p[Pab][Pef] += tmp^T
    permute(c.L, T(tmp, {Pv, Pv}).perm({1, 0}), T(c.Wabef_p, {Pv, Pv}), cx(1), true);
  }
  gemm_dispatch(c, true, false, Pv, Pv, Po, cx(1), tap, Pv, c.oovv_p, Pv, cx(1), c.Wabef_p, Pv);

  // W_mbej (Eq. W_mbej) and the ring operands
  Tensor Wmbej = T(c.Wmbej, {o, v, v, o});
  permute(c.L, c.V("ovvo"), Wmbej, cx(1), false);
  einsum(c, "jf,mbef->mbej", cx(1), t1, c.V("ovvv"), 1.0, Wmbej);
  einsum(c, "nb,mnej->mbej", cx(-1), t1, c.V("oovo"), 1.0, Wmbej);
  {
    Scope s2(c.ws);
    cplx* u = c.ws.cplxs(o * o * v * v);
    copy_vec(c.L, o * o * v * v, c.t2, u);
    einsum(c, "jf,nb->jnfb", cx(1), t1, t1, 1.0, T(u, {o, o, v, v}));
    einsum(c, "jnfb,mnef->mbej", cx(-1), T(u, {o, o, v, v}), c.V("oovv"), 1.0, Wmbej);
  }
  // right ring operand [(j,b)][(m,e)] = W_mbej[m,b,e,j]; left ring operand = W_mbej[j,e,b,m]
  permute(c.L, Wmbej.perm({3, 1, 0, 2}), T(c.WringR, {o, v, o, v}), cx(1), false);
  permute(c.L, Wmbej.perm({0, 2, 3, 1}), T(c.WringL, {o, v, o, v}), cx(1), false);
  // Davidson preconditioner from the dressed one-body diagonal: Re F_aa - Re F_ii (singles),
  // Re (F_aa + F_bb - F_ii - F_jj) (doubles)
  {
    if (!c.Dpre) c.Dpre = (double*)c.dalloc((c.N + 1) / 2 + 1);
    std::vector<cplx> fa((size_t)v * v), fi((size_t)o * o);
    CCLR_CK(cudaMemcpyAsync(fa.data(), c.Fae, sizeof(cplx) * fa.size(), cudaMemcpyDeviceToHost, c.stream));
    CCLR_CK(cudaMemcpyAsync(fi.data(), c.Fmi, sizeof(cplx) * fi.size(), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    std::vector<double> ea(v), ei(o), D((size_t)c.N);
    for (int a = 0; a < v; ++a) ea[a] = fa[(size_t)a * v + a].x;
    for (int i = 0; i < o; ++i) ei[i] = fi[(size_t)i * o + i].x;
    for (int i = 0; i < o; ++i)
      for (int a = 0; a < v; ++a) D[(size_t)i * v + a] = ea[a] - ei[i];
    int64_t ij = 0;
    for (int q = 1; q < o; ++q)
      for (int p = 0; p < q; ++p, ++ij) {
        int64_t ab = 0;
        for (int bq = 1; bq < v; ++bq)
          for (int bp = 0; bp < bq; ++bp, ++ab)
            D[(size_t)(c.Ns + ij * c.Pv + ab)] = ea[bp] + ea[bq] - ei[p] - ei[q];
      }
    CCLR_CK(cudaMemcpyAsync(c.Dpre, D.data(), sizeof(double) * D.size(), cudaMemcpyHostToDevice, c.stream));
    c.sync();
  }
  // Fae, Fmi without the bare Fock diagonal: sigma adds that part exactly as D r (D the
  // orbital-energy differences), so the tensor-core products carry only the rest
  copy_vec(c.L, v * v, c.Fae, c.Fae_od);
  copy_vec(c.L, o * o, c.Fmi, c.Fmi_od);
  {
    Tensor fv = c.f("vv"), fo = c.f("oo");
    fv.rank = fo.rank = 1;
    fv.str[0] = c.n + 1;
    fo.str[0] = c.n + 1;
    Tensor dv = Tensor::make(c.Fae_od, {v}), dov = Tensor::make(c.Fmi_od, {o});
    dv.str[0] = v + 1;
    dov.str[0] = o + 1;
    permute(c.L, fv, dv, cx(-1), true);
    permute(c.L, fo, dov, cx(-1), true);
  }
  // The one-index F terms of the doubles sigma are ring terms with a Kronecker delta: the ring
  // contracts the amplitudes over (m, e), so (weights as the terms enter the accumulator packed
  // with P(ij)P(ab))
  //   right: 1/2 F_be r_ij^ae - 1/2 F_mj r_im^ab  ->  W[j,b,m,e] += 1/2 d_jm F_be - 1/2 d_be F_mj
  //   left:  1/2 l_ij^ae F_eb - 1/2 l_im^ab F_jm  ->  W[j,b,m,e] += 1/2 d_jm F_eb - 1/2 d_be F_jm
  // and ride in the ring GEMM instead of two read-modify-write passes over the accumulator.
  {
    auto view = [](cplx* p, std::initializer_list<int64_t> d, std::initializer_list<int64_t> st) {
      Tensor t;
      t.p = p;
      t.rank = (int)d.size();
      int i = 0;
      for (int64_t x : d) t.dim[i++] = x;
      i = 0;
      for (int64_t x : st) t.str[i++] = x;
      return t;
    };
    const int64_t sj = v * o * v, sb = o * v, sm = v;   // strides of W[j][b][m][e]
    for (int side = 0; side < 2; ++side) {
      cplx* W = side == 0 ? c.WringR : c.WringL;
      // d_jm: (j, b, e) -> W[j][b][j][e]
      const Tensor djm = view(W, {o, v, v}, {sj + sm, sb, 1});
      const Tensor fae = side == 0 ? view(c.Fae_od, {o, v, v}, {0, v, 1})    // F_be
                                   : view(c.Fae_od, {o, v, v}, {0, 1, v});   // F_eb
      permute(c.L, fae, djm, cx(0.5), true);
      // d_be: (j, b, m) -> W[j][b][m][b]
      const Tensor dbe = view(W, {o, v, o}, {sj, sb + 1, sm});
      const Tensor fmi = side == 0 ? view(c.Fmi_od, {o, v, o}, {1, 0, o})    // F_mj
                                   : view(c.Fmi_od, {o, v, o}, {o, 0, 1});   // F_jm
      permute(c.L, fmi, dbe, cx(-0.5), true);
    }
  }

  // W_mnie (Eq. W_mnie), W_amef (Eq. W_amef)
  Tensor Wmnie = T(c.Wmnie, {o, o, o, v});
  permute(c.L, c.V("ooov"), Wmnie, cx(1), false);
  einsum(c, "if,mnfe->mnie", cx(1), t1, c.V("oovv"), 1.0, Wmnie);
  Tensor Wamef = T(c.Wamef, {v, o, v, v});
  permute(c.L, c.V("vovv"), Wamef, cx(1), false);
  einsum(c, "na,nmef->amef", cx(-1), t1, c.V("oovv"), 1.0, Wamef);

  // W_mbij (Eq. W_iemn with relabelled indices)
  Tensor Wmbij = T(c.Wmbij, {o, v, o, o});
  {
    Scope s2(c.ws);
    permute(c.L, c.V("ovoo"), Wmbij, cx(1), false);
    einsum(c, "me,ijbe->mbij", cx(-1), Fme, t2, 1.0, Wmbij);
    einsum(c, "nb,mnij->mbij", cx(-1), t1, Wmnij, 1.0, Wmbij);
    einsum(c, "mbef,ijef->mbij", cx(0.5), c.V("ovvv"), ta, 1.0, Wmbij);
    einsum(c, "mnie,jnbe->mbij", cx(1), c.V("ooov"), t2, 1.0, Wmbij);
    einsum(c, "mnje,inbe->mbij", cx(-1), c.V("ooov"), t2, 1.0, Wmbij);
    cplx* wb = c.ws.cplxs(o * v * v * o);          // bar W_mbej (Eq. barW_mbej)
    Tensor Wbar = T(wb, {o, v, v, o});
    permute(c.L, c.V("ovvo"), Wbar, cx(1), false);
    einsum(c, "mnef,njbf->mbej", cx(-1), c.V("oovv"), t2, 1.0, Wbar);
    einsum(c, "ie,mbej->mbij", cx(1), t1, Wbar, 1.0, Wmbij);
    einsum(c, "je,mbei->mbij", cx(-1), t1, Wbar, 1.0, Wmbij);
  }

  // W_abei (Eq. W_efam with relabelled indices)
  Tensor Wabei = T(c.Wabei, {v, v, v, o});
  {
    Scope s2(c.ws);
    permute(c.L, c.V("vvvo"), Wabei, cx(1), false);
    einsum(c, "me,miab->abei", cx(-1), Fme, t2, 1.0, Wabei);
    // t_i^f W_abef: unpack the (e,f) pair of W_abef, contract, then unpack (a,b)
    cplx* wf = c.ws.cplxs(Pv * v * v);
    unpack2(c.L, c.Wabef_p, Pv, T(wf, {Pv, v, v}));                        // [Pab][e][f]
    cplx* z = c.ws.cplxs(Pv * v * o);
    einsum(c, "Pef,if->Pei", cx(1), T(wf, {Pv, v, v}), t1, 0.0, T(z, {Pv, v, o}));
    cplx* zf = c.ws.cplxs(v * v * v * o);
    // z is [Pab][(e,i)]; expand the pair into (a,b): view destination (a,b,(e,i)) as (R=(e,i), a, b)
    Tensor dst = T(zf, {v, v, v * o}).perm({2, 0, 1});
    // unpack2 expects D[r*ldd + P]: z stored [P][r] -> transpose first
    cplx* zt = c.ws.cplxs(v * o * Pv);
    permute(c.L, T(z, {Pv, v * o}).perm({1, 0}), T(zt, {v * o, Pv}), cx(1), false);
    unpack2(c.L, zt, Pv, dst);
    permute(c.L, T(zf, {v, v, v, o}), Wabei, cx(1), true);
    einsum(c, "mnei,mnab->abei", cx(0.5), c.V("oovo"), ta, 1.0, Wabei);
    einsum(c, "mbef,miaf->abei", cx(-1), c.V("ovvv"), t2, 1.0, Wabei);
    einsum(c, "maef,mibf->abei", cx(1), c.V("ovvv"), t2, 1.0, Wabei);
    cplx* q = c.ws.cplxs(o * v * v * o);
    Tensor Q = T(q, {o, v, v, o});
    permute(c.L, c.V("ovvo"), Q, cx(1), false);
    einsum(c, "mnef,nibf->mbei", cx(-1), c.V("oovv"), t2, 1.0, Q);
    einsum(c, "ma,mbei->abei", cx(-1), t1, Q, 1.0, Wabei);
    einsum(c, "mb,maei->abei", cx(1), t1, Q, 1.0, Wabei);
  }
  c.have_hbar = true;
}

}  // namespace cclr

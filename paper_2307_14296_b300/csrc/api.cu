// The C ABI of libcclr (declared in include/cclr.h).  Every entry point catches all C++
// exceptions and returns a status; the message is kept in the context for cclr_last_error().
#include "ctx.h"
#include <cstdio>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <thread>

using namespace cclr;

struct cclr_ctx {
  Ctx c;
};

namespace {

bool valid_precision(int p) {
  return p == CCLR_FP64 || p == CCLR_TC_BF16X3 || p == CCLR_TC_BF16X6 || p == CCLR_TC_F64;
}

double wall() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <class F>
cclr_status guard(cclr_ctx* h, F&& fn) {
  if (!h) return CCLR_E_ARG;
  Ctx& c = h->c;
  c.err.clear();
  c.stats = cclr_stats{};
  const long l0 = c.launches;
  const double t0 = wall();
  cclr_status st = CCLR_OK;
  try {
    CCLR_CK(cudaSetDevice(c.device));
    fn(c);
    CCLR_CK(cudaStreamSynchronize(c.stream));
    tc_tune_collect(c);
    if (c.prof) c.prof_collect();
    if (c.kt.on) c.kt.collect();
    static const bool verbose = std::getenv("CCLR_VERBOSE") != nullptr;
    if (verbose) {
      size_t fr = 0, tot = 0;
      cudaMemGetInfo(&fr, &tot);
      std::fprintf(stderr, "[cclr] memory: arrays %.2f GiB (%zu), slice cache %.2f GiB, workspace peak %.2f of %.2f GiB, free %.2f GiB\n",
                   c.persistent_total() / 1073741824.0, c.persistent.size(), tc_cache_bytes(c) / 1073741824.0,
                   c.ws.peak / 1073741824.0, c.ws.cap / 1073741824.0, fr / 1073741824.0);
    }
    if (c.tc_err) {
      int h = 0;
      CCLR_CK(cudaMemcpy(&h, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (h) {
        CCLR_CK(cudaMemset(c.tc_err, 0, sizeof(int)));
        throw Error(CCLR_E_TIMEOUT, "a bounded device wait expired (code " + std::to_string(h) + ")");
      }
    }
  } catch (const Error& e) {
    c.ev_used = 0;
    c.err = e.what();
    st = e.st;
  } catch (const std::exception& e) {
    c.err = e.what();
    st = CCLR_E_ARG;
  }
  c.stats.total_seconds = wall() - t0;
  c.stats.kernel_launches = c.launches - l0;
  return st;
}

void free_all(Ctx& c) {
  tc_release_cache_for(c);
  ++c.data_gen;
  for (void* p : c.persistent) cudaFree(p);
  c.persistent.clear();
  c.persistent_bytes.clear();
  c.named.clear();
  c.rd = ResponseData();
  c.eom_vecs.clear();
  c.eom_w.clear();
  c.fock = c.oooo = c.ooov = c.oovv = c.ovov = c.ovvv = c.vvvv_p = c.oovv_p = c.ovvv_p = nullptr;
  c.D = nullptr;
  c.Dpre = nullptr;
  c.po = c.pv = nullptr;
  c.t = c.t2 = c.lam = c.l2 = nullptr;
  c.Fae = c.Fmi = c.Fme = c.Wmnij = c.Wmnij_p = c.Wabef_p = c.Wmbej = c.WringR = c.WringL = nullptr;
  c.Fae_od = c.Fmi_od = nullptr;
  c.Wmnie = c.Wamef = c.Wmbij = c.Wabei = c.tau = nullptr;
  c.have_ham = c.have_t = c.have_lambda = c.have_hbar = false;
  if (c.ws.base) { cudaFree(c.ws.base); c.ws = Arena(); }
}

// Copies between the library's device arrays and caller memory use cudaMemcpyDefault: with unified
// addressing the runtime reads from the pointer whether it is host (pageable or pinned) or device
// memory, so the amplitude, operator and gradient entry points take either without a flag.
void upload(Ctx& c, cplx* dst, const void* src, int64_t n) {
  CCLR_CK(cudaMemcpyAsync(dst, src, sizeof(cplx) * n, cudaMemcpyDefault, c.stream));
}
void download(Ctx& c, void* dst, const cplx* src, int64_t n) {
  CCLR_CK(cudaMemcpyAsync(dst, src, sizeof(cplx) * n, cudaMemcpyDefault, c.stream));
}

// true when p is device (or managed) memory, false for host memory
bool device_pointer(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// rejects infinities and NaN in n complex values at p (host loop, or a device scan for device p)
void require_finite(Ctx& c, const cplx* p, int64_t n, const char* what) {
  bool ok = true;
  if (device_pointer(p)) {
    Scope sc(c.ws);
    int* bad = (int*)c.ws.alloc(sizeof(int));
    CCLR_CK(cudaMemsetAsync(bad, 0, sizeof(int), c.stream));
    flag_nonfinite(c.L, p, n, bad);
    int h = 0;
    CCLR_CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    ok = h == 0;
  } else {
    for (int64_t i = 0; i < n && ok; ++i) ok = std::isfinite(p[i].x) && std::isfinite(p[i].y);
  }
  if (!ok) throw Error(CCLR_E_ARG, std::string(what) + ": an element is an infinity or NaN");
}

// copy in/out helpers for entry points that accept host or device pointers
struct IO {
  Ctx& c;
  const cplx* in;
  cplx* out;
  cplx* dout;
  int64_t nin, nout;
  bool dev;
  IO(Ctx& cc, const void* i, void* o, int64_t ni, int64_t no, bool on_device)
      : c(cc), nin(ni), nout(no), dev(on_device) {
    if (dev) {
      in = (const cplx*)i;
      out = dout = (cplx*)o;
    } else {
      cplx* di = c.ws.cplxs(ni);
      if (ni) upload(c, di, i, ni);
      in = di;
      dout = c.ws.cplxs(no);
      out = (cplx*)o;
    }
  }
  void finish() {
    if (!dev) {
      CCLR_CK(cudaMemcpyAsync(out, dout, sizeof(cplx) * nout, cudaMemcpyDeviceToHost, c.stream));
      c.sync();
    }
  }
};

}  // namespace

extern "C" {

void cclr_default_options(cclr_options* opt) {
  if (!opt) return;
  opt->tol = 1e-8;
  opt->ground_tol = 1e-10;
  opt->maxit = 100;
  opt->max_subspace = 96;
  opt->precision = CCLR_FP64;
  opt->batch = 0;
  opt->refine = 1;
  opt->refine_tol = 0.0;
  opt->autotune = 1;
}

cclr_status cclr_create(cclr_ctx** out, int device, const cclr_options* opt) {
  if (!out) return CCLR_E_ARG;
  *out = nullptr;
  int nd = 0;
  if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) return CCLR_E_ARG;
  cclr_ctx* h = new cclr_ctx();
  Ctx& c = h->c;
  c.device = device;
  if (opt) c.opt = *opt; else cclr_default_options(&c.opt);
  if (!valid_precision(c.opt.precision)) {
    delete h;
    return CCLR_E_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return CCLR_E_CUDA;
  }
  c.L.s = c.stream;
  c.L.count = &c.launches;
  c.L.kt = &c.kt;
  if (cudaMalloc((void**)&c.tc_err, sizeof(int)) != cudaSuccess || cudaMemset(c.tc_err, 0, sizeof(int)) != cudaSuccess) {
    cudaStreamDestroy(c.stream);
    delete h;
    return CCLR_E_CUDA;
  }
  c.L.err = c.tc_err;
  *out = h;
  return CCLR_OK;
}

void cclr_destroy(cclr_ctx* h) {
  if (!h) return;
  cudaSetDevice(h->c.device);
  free_all(h->c);
  tc_state_free(h->c);
  if (h->c.tc_err) cudaFree(h->c.tc_err);
  for (auto& e : h->c.ev_pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  if (h->c.stream) cudaStreamDestroy(h->c.stream);
  delete h;
}

const char* cclr_last_error(const cclr_ctx* h) {
  if (!h) return "null context";
  return h->c.err.c_str();
}

cclr_status cclr_set_hamiltonian(cclr_ctx* h, int n_occ, int n_vir, const cclr_c128* fock,
                                 const cclr_c128* const blocks[6]) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(n_occ >= 2 && n_vir >= 2, CCLR_E_ARG, "need n_occ >= 2 and n_vir >= 2");
    CCLR_REQUIRE(fock && blocks, CCLR_E_ARG, "null Hamiltonian pointer");
    for (int k = 0; k < 6; ++k) CCLR_REQUIRE(blocks[k], CCLR_E_ARG, "null integral block");
    free_all(c);
    const int64_t o = n_occ, v = n_vir, n = o + v;
    c.o = n_occ; c.v = n_vir; c.n = (int)n;
    c.Po = o * (o - 1) / 2; c.Pv = v * (v - 1) / 2;
    c.Ns = o * v; c.Nd = c.Po * c.Pv; c.N = c.Ns + c.Nd;
    // workspace: a fixed fraction of free device memory (CCLR_WORKSPACE_GB overrides)
    size_t fr = 0, tot = 0;
    CCLR_CK(cudaMemGetInfo(&fr, &tot));
    size_t ws = (size_t)(0.35 * (double)fr);
    if (const char* e = std::getenv("CCLR_WORKSPACE_GB")) ws = (size_t)(atof(e) * (1ull << 30));
    CCLR_CK(cudaMalloc((void**)&c.ws.base, ws));
    c.ws.cap = ws;
    c.ws.top = 0;
    // every uploaded value is checked for infinities and NaN (one flag, read at the end)
    const size_t ws_base = c.ws.mark();
    int* bad = (int*)c.ws.alloc(sizeof(int));
    CCLR_CK(cudaMemsetAsync(bad, 0, sizeof(int), c.stream));
    // pair tables
    std::vector<int2> po(c.Po), pv(c.Pv);
    int64_t k = 0;
    for (int q = 1; q < n_occ; ++q) for (int p = 0; p < q; ++p) po[k++] = make_int2(p, q);
    k = 0;
    for (int q = 1; q < n_vir; ++q) for (int p = 0; p < q; ++p) pv[k++] = make_int2(p, q);
    CCLR_CK(cudaMalloc((void**)&c.po, sizeof(int2) * std::max<int64_t>(1, c.Po)));
    CCLR_CK(cudaMalloc((void**)&c.pv, sizeof(int2) * std::max<int64_t>(1, c.Pv)));
    c.persistent.push_back(c.po);
    c.persistent.push_back(c.pv);
    CCLR_CK(cudaMemcpy(c.po, po.data(), sizeof(int2) * c.Po, cudaMemcpyHostToDevice));
    CCLR_CK(cudaMemcpy(c.pv, pv.data(), sizeof(int2) * c.Pv, cudaMemcpyHostToDevice));
    // Hamiltonian
    c.fock = c.dalloc(n * n);
    upload(c, c.fock, fock, n * n);
    flag_nonfinite(c.L, c.fock, n * n, bad);
    c.oooo = c.dalloc(o * o * o * o);
    c.ooov = c.dalloc(o * o * o * v);
    c.oovv = c.dalloc(o * o * v * v);
    c.ovov = c.dalloc(o * v * o * v);
    c.ovvv = c.dalloc(o * v * v * v);
    c.vvvv_p = c.dalloc(c.Pv * c.Pv);
    c.oovv_p = c.dalloc(c.Po * c.Pv);
    c.ovvv_p = c.dalloc(o * v * c.Pv);
    {
      Scope sc(c.ws);
      cplx* tmp = c.ws.cplxs(c.Po * c.Po);
      upload(c, tmp, blocks[0], c.Po * c.Po);
      flag_nonfinite(c.L, tmp, c.Po * c.Po, bad);
      unpack_doubles(c.L, tmp, c.Po * c.Po, Tensor::make(c.oooo, {1, o, o, o, o}), n_occ, n_occ);
    }
    {
      Scope sc(c.ws);
      cplx* tmp = c.ws.cplxs(c.Po * o * v);
      upload(c, tmp, blocks[1], c.Po * o * v);
      flag_nonfinite(c.L, tmp, c.Po * o * v, bad);
      cplx* tr = c.ws.cplxs(c.Po * o * v);
      permute(c.L, Tensor::make(tmp, {c.Po, o * v}).perm({1, 0}), Tensor::make(tr, {o * v, c.Po}), cx(1), false);
      // full[i][j][k][a] viewed as (R=(k,a), i, j)
      Tensor dst = Tensor::make(c.ooov, {o, o, o * v}).perm({2, 0, 1});
      unpack2(c.L, tr, c.Po, dst);
    }
    upload(c, c.oovv_p, blocks[2], c.Po * c.Pv);
    flag_nonfinite(c.L, c.oovv_p, c.Po * c.Pv, bad);
    unpack_doubles(c.L, c.oovv_p, c.Nd, Tensor::make(c.oovv, {1, o, o, v, v}), n_occ, n_vir);
    upload(c, c.ovov, blocks[3], o * v * o * v);
    flag_nonfinite(c.L, c.ovov, o * v * o * v, bad);
    upload(c, c.ovvv_p, blocks[4], o * v * c.Pv);
    flag_nonfinite(c.L, c.ovvv_p, o * v * c.Pv, bad);
    unpack2(c.L, c.ovvv_p, c.Pv, Tensor::make(c.ovvv, {o * v, v, v}));
    upload(c, c.vvvv_p, blocks[5], c.Pv * c.Pv);
    flag_nonfinite(c.L, c.vvvv_p, c.Pv * c.Pv, bad);
    {
      int h = 0;
      CCLR_CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
      c.sync();
      if (h) {
        free_all(c);
        throw Error(CCLR_E_ARG, "cclr_set_hamiltonian: an infinity or NaN in the Fock matrix or the integrals");
      }
    }
    c.ws.release(ws_base);
    c.D = (double*)c.dalloc((c.N + 1) / 2 + 1);
    c.t = c.dalloc(c.N);
    c.t2 = c.dalloc(o * o * v * v);
    c.lam = c.dalloc(c.N);
    c.l2 = c.dalloc(o * o * v * v);
    fill_zero(c.L, c.t, c.N);
    fill_zero(c.L, c.t2, o * o * v * v);
    c.sync();
    build_denominators(c);
    c.have_ham = true;
  });
}

cclr_status cc_ground(cclr_ctx* h, cclr_c128* e_corr_out, int* iters_out) {
  int its = 0;
  cclr_status st = guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_ham, CCLR_E_STATE, "cc_ground before cclr_set_hamiltonian");
    c.have_lambda = false;
    release_response(c);
    for (auto p : c.eom_vecs) c.dfree(p);
    c.eom_vecs.clear();
    c.eom_w.clear();
    // Hbar defines the sigma products of every later solve: FP64-class when refining
    try {
      its = solve_ground(c);
    } catch (const Error& e) {
      if (e.st == CCLR_E_NOCONV) {
        PrecisionScope exact(c, exact_precision(c));
        build_hbar(c);
      }
      throw;
    }
    PrecisionScope exact(c, exact_precision(c));
    build_hbar(c);
  });
  if (h && (st == CCLR_OK || st == CCLR_E_NOCONV)) {
    if (e_corr_out) { e_corr_out->re = h->c.e_corr.real(); e_corr_out->im = h->c.e_corr.imag(); }
    if (iters_out) *iters_out = its;
  }
  return st;
}

cclr_status cc_lambda(cclr_ctx* h, int* iters_out) {
  int its = 0;
  cclr_status st = guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_hbar, CCLR_E_STATE, "cc_lambda before cc_ground");
    its = solve_lambda(c);
  });
  if (iters_out) *iters_out = its;
  return st;
}

cclr_status cc_lr_solve(cclr_ctx* h, int n_ops, const cclr_c128* ops, int n_freq, const double* omegas, double gamma,
                        int* iters_out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_lambda, CCLR_E_STATE, "cc_lr_solve before cc_lambda");
    CCLR_REQUIRE(n_ops >= 1 && n_freq >= 1 && ops && omegas && gamma >= 0.0, CCLR_E_ARG, "bad cc_lr_solve arguments");
    CCLR_REQUIRE(std::isfinite(gamma), CCLR_E_ARG, "cc_lr_solve: gamma must be finite");
    for (int f = 0; f < n_freq; ++f)
      CCLR_REQUIRE(std::isfinite(omegas[f]), CCLR_E_ARG, "cc_lr_solve: a frequency is an infinity or NaN");
    require_finite(c, (const cplx*)ops, (int64_t)n_ops * c.n * c.n, "cc_lr_solve: operator");
    lr_solve(c, n_ops, (const cplx*)ops, n_freq, omegas, gamma, iters_out);
  });
}

cclr_status cc_response_function(cclr_ctx* h, cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(out, CCLR_E_ARG, "null output");
    response_function(c, (cplx*)out);
  });
}

cclr_status cclr_response_gradient(cclr_ctx* h, int f, cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(out, CCLR_E_ARG, "null output");
    response_gradient(c, f, (cplx*)out);
  });
}

cclr_status cclr_set_synthetic(cclr_ctx* h, int n_occ, int n_vir, uint64_t seed, double sd, double dip_sd,
                               int n_ops, cclr_c128* ops_out) {
  if (!h) return CCLR_E_ARG;
  const int64_t o = n_occ, v = n_vir, n = o + v, Po = o * (o - 1) / 2, Pv = v * (v - 1) / 2;
  const int64_t sizes[6] = {Po * Po, Po * o * v, Po * Pv, o * v * o * v, o * v * Pv, Pv * Pv};
  cplx* blocks[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* eps_u = nullptr;
  cplx* ops = nullptr;
  std::vector<cclr_c128> fock((size_t)(n > 0 ? n * n : 0));
  auto release = [&]() {
    for (auto& b : blocks) { if (b) cudaFree(b); b = nullptr; }
    if (eps_u) cudaFree(eps_u);
    if (ops) cudaFree(ops);
    eps_u = nullptr;
    ops = nullptr;
  };
  // generation into temporary device arrays (not the context's workspace: the Hamiltonian setter
  // below releases and re-creates it)
  cclr_status st = guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(n_occ >= 2 && n_vir >= 2, CCLR_E_ARG, "need n_occ >= 2 and n_vir >= 2");
    CCLR_REQUIRE(std::isfinite(sd) && sd >= 0.0 && std::isfinite(dip_sd) && dip_sd >= 0.0 && n_ops >= 0 &&
                     (n_ops == 0 || ops_out),
                 CCLR_E_ARG, "bad cclr_set_synthetic arguments");
    for (int k = 0; k < 6; ++k) CCLR_CK(cudaMalloc((void**)&blocks[k], sizeof(cplx) * (size_t)std::max<int64_t>(1, sizes[k])));
    CCLR_CK(cudaMalloc((void**)&eps_u, sizeof(double) * (size_t)n));
    if (n_ops > 0) CCLR_CK(cudaMalloc((void**)&ops, sizeof(cplx) * (size_t)(n_ops * n * n)));
    synthetic_instance(c, n_occ, n_vir, seed, sd, dip_sd, n_ops, blocks, eps_u, ops);
    std::vector<double> u((size_t)n);
    CCLR_CK(cudaMemcpyAsync(u.data(), eps_u, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c.stream));
    if (n_ops > 0)
      CCLR_CK(cudaMemcpyAsync(ops_out, ops, sizeof(cplx) * (size_t)(n_ops * n * n), cudaMemcpyDefault, c.stream));
    c.sync();
    // orbital energies: occupied U[-2, -0.5], virtual U[0.3, 4], each range sorted
    std::vector<double> eo((size_t)o), ev((size_t)v);
    for (int64_t p = 0; p < o; ++p) eo[p] = -2.0 + (-0.5 - -2.0) * u[p];
    for (int64_t p = 0; p < v; ++p) ev[p] = 0.3 + (4.0 - 0.3) * u[o + p];
    std::sort(eo.begin(), eo.end());
    std::sort(ev.begin(), ev.end());
    for (int64_t p = 0; p < n; ++p) fock[(size_t)(p * n + p)].re = p < o ? eo[p] : ev[p - o];
  });
  if (st == CCLR_OK) {
    const cclr_c128* bl[6];
    for (int k = 0; k < 6; ++k) bl[k] = (const cclr_c128*)blocks[k];
    st = cclr_set_hamiltonian(h, n_occ, n_vir, fock.data(), bl);
  }
  release();
  return st;
}

cclr_status cclr_eta_ground(cclr_ctx* h, cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_hbar && out, CCLR_E_STATE, "cclr_eta_ground needs T");
    PrecisionScope exact(c, exact_precision(c));
    Scope sc(c.ws);
    cplx* r = c.ws.cplxs(c.N);
    eta_ground(c, r);
    download(c, out, r, c.N);
    c.sync();
  });
}

cclr_status cclr_left_solve(cclr_ctx* h, int nrhs, const cclr_c128* rhs, double w_re, double w_im, cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_hbar, CCLR_E_STATE, "cclr_left_solve needs T");
    CCLR_REQUIRE(nrhs >= 1 && rhs && out && std::isfinite(w_re) && std::isfinite(w_im), CCLR_E_ARG,
                 "bad cclr_left_solve arguments");
    require_finite(c, (const cplx*)rhs, (int64_t)nrhs * c.N, "cclr_left_solve: right-hand side");
    left_solve(c, nrhs, (const cplx*)rhs, zc(w_re, w_im), (cplx*)out);
  });
}

cclr_status cc_response_function_ci(cclr_ctx* h, cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(out, CCLR_E_ARG, "null output");
    response_function_ci(c, (cplx*)out);
  });
}

cclr_status cc_response_function_asym(cclr_ctx* h, cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(out, CCLR_E_ARG, "null output");
    response_function_asym(c, (cplx*)out);
  });
}

cclr_status cclr_field_derivative(cclr_ctx* h, const cclr_c128* V, cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(V && out, CCLR_E_ARG, "null argument");
    CCLR_REQUIRE(c.rd.solved, CCLR_E_STATE, "cclr_field_derivative before cc_lr_solve");
    require_finite(c, (const cplx*)V, c.n * c.n, "cclr_field_derivative: field operator");
    field_derivative(c, (const cplx*)V, (cplx*)out);
  });
}

cclr_status cc_eom_ee(cclr_ctx* h, int n_roots, cclr_c128* energies_out, int* iters_out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(energies_out, CCLR_E_ARG, "null output");
    std::vector<zc> w;
    const int its = eom_ee(c, n_roots, w);
    for (int q = 0; q < n_roots; ++q) energies_out[q] = cclr_c128{w[q].real(), w[q].imag()};
    if (iters_out) *iters_out = its;
  });
}

cclr_status cclr_get_eom_vector(cclr_ctx* h, int root, cclr_c128* dst, size_t n) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(dst && (int64_t)n == c.N, CCLR_E_ARG, "vector buffer length must be o*v + Po*Pv");
    CCLR_REQUIRE(root >= 0 && root < (int)c.eom_vecs.size(), CCLR_E_STATE, "no such EOM root (call cc_eom_ee)");
    download(c, dst, c.eom_vecs[root], (int64_t)n);
  });
}

cclr_status cclr_get_amplitudes(cclr_ctx* h, int which, cclr_c128* dst, size_t n) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(dst && (int64_t)n == c.N, CCLR_E_ARG, "amplitude buffer length must be o*v + Po*Pv");
    const cplx* src = which == CCLR_AMP_T ? c.t : which == CCLR_AMP_LAMBDA ? c.lam : nullptr;
    CCLR_REQUIRE(src, CCLR_E_ARG, "unknown amplitude set");
    CCLR_REQUIRE(which == CCLR_AMP_T ? c.have_t : c.have_lambda, CCLR_E_STATE, "amplitudes not available");
    download(c, dst, src, (int64_t)n);
  });
}

cclr_status cclr_set_amplitudes(cclr_ctx* h, int which, const cclr_c128* src, size_t n) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_ham, CCLR_E_STATE, "no Hamiltonian");
    CCLR_REQUIRE(src && (int64_t)n == c.N, CCLR_E_ARG, "amplitude buffer length must be o*v + Po*Pv");
    if (which == CCLR_AMP_T) {
      upload(c, c.t, src, c.N);
      expand_t2(c, c.t + c.Ns, c.t2, 1);
      c.e_corr = ccsd_energy(c);
      c.have_t = true;
      c.have_lambda = false;
      c.named.erase("F.ready");
      PrecisionScope exact(c, exact_precision(c));
      build_hbar(c);
    } else if (which == CCLR_AMP_LAMBDA) {
      CCLR_REQUIRE(c.have_hbar, CCLR_E_STATE, "set T before Lambda");
      upload(c, c.lam, src, c.N);
      expand_t2(c, c.lam + c.Ns, c.l2, 1);
      c.have_lambda = true;
      c.named.erase("F.ready");
    } else {
      throw Error(CCLR_E_ARG, "unknown amplitude set");
    }
  });
}

cclr_status cclr_get_response_vector(cclr_ctx* h, int k, int f, int s, cclr_c128* dst, size_t n) {
  return guard(h, [&](Ctx& c) {
    ResponseData& rd = c.rd;
    CCLR_REQUIRE(rd.solved, CCLR_E_STATE, "no response solution");
    CCLR_REQUIRE(k >= 0 && k < rd.n_ops && f >= 0 && f < rd.n_freq && s >= 0 && s < 4 && (int64_t)n == c.N && dst,
                 CCLR_E_ARG, "bad response-vector index");
    const int maxL = std::max(8, c.opt.max_subspace);
    Scope sc(c.ws);
    cplx* b = c.ws.cplxs(maxL);
    cplx* t = c.ws.cplxs(c.N);
    const zc* beta = &rd.beta[k][(size_t)rd.shift_of[(size_t)f * 4 + s] * maxL];
    CCLR_CK(cudaMemcpyAsync(b, beta, sizeof(cplx) * rd.nb[k], cudaMemcpyHostToDevice, c.stream));
    lincomb(c.L, c.N, rd.nb[k], rd.basis[k], c.N, b, t, false);
    download(c, dst, t, (int64_t)n);
    c.sync();
  });
}

cclr_status cclr_export_amplitudes(cclr_ctx* h, int which, int idx, cclr_c128* dst, size_t n) {
  if (which == 0 || which == 1) return cclr_get_amplitudes(h, which, dst, n);
  if (which == 2) {
    if (!h) return CCLR_E_ARG;
    const ResponseData& rd = h->c.rd;
    const int nf = std::max(1, rd.n_freq);
    const int s = idx & 3, q = idx >> 2;
    return cclr_get_response_vector(h, idx < 0 ? -1 : q / nf, q % nf, s, dst, n);
  }
  return guard(h, [&](Ctx&) { throw Error(CCLR_E_ARG, "cclr_export_amplitudes: unknown amplitude set"); });
}

cclr_status cclr_sigma(cclr_ctx* h, int side, int nvec, const cclr_c128* in, cclr_c128* out, int on_device,
                       int precision) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_hbar, CCLR_E_STATE, "sigma needs T (cc_ground or cclr_set_amplitudes)");
    CCLR_REQUIRE(nvec >= 1 && in && out && (side == 0 || side == 1), CCLR_E_ARG, "bad sigma arguments");
    CCLR_REQUIRE(valid_precision(precision), CCLR_E_ARG, "unknown precision");
    const int saved = c.opt.precision;
    c.opt.precision = precision;
    try {
      Scope sc(c.ws);
      IO io(c, in, out, (int64_t)nvec * c.N, (int64_t)nvec * c.N, on_device != 0);
      const double t0 = wall();
      if (side == 0) sigma_right(c, nvec, io.in, io.dout);
      else sigma_left(c, nvec, io.in, io.dout);
      c.sync();
      c.stats.sigma_seconds += wall() - t0;
      io.finish();
    } catch (...) {
      c.opt.precision = saved;
      throw;
    }
    c.opt.precision = saved;
  });
}

cclr_status cclr_residual(cclr_ctx* h, cclr_c128* out, cclr_c128* e_corr_out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_t && out, CCLR_E_STATE, "no amplitudes");
    Scope sc(c.ws);
    cplx* R = c.ws.cplxs(c.N);
    ccsd_residual(c, R);
    download(c, out, R, c.N);
    c.sync();
    if (e_corr_out) { zc e = ccsd_energy(c); e_corr_out->re = e.real(); e_corr_out->im = e.imag(); }
  });
}

cclr_status cclr_xi(cclr_ctx* h, const cclr_c128* op, cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_t && op && out, CCLR_E_STATE, "xi needs T");
    PrecisionScope exact(c, exact_precision(c));
    Scope sc(c.ws);
    cplx* X = c.ws.cplxs((int64_t)c.n * c.n);
    upload(c, X, op, (int64_t)c.n * c.n);
    cplx* r = c.ws.cplxs(c.N);
    xi_vec(c, X, r);
    download(c, out, r, c.N);
    c.sync();
  });
}

cclr_status cclr_eta(cclr_ctx* h, const cclr_c128* op, int eom, cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_lambda && op && out, CCLR_E_STATE, "eta needs Lambda");
    PrecisionScope exact(c, exact_precision(c));
    Scope sc(c.ws);
    cplx* X = c.ws.cplxs((int64_t)c.n * c.n);
    upload(c, X, op, (int64_t)c.n * c.n);
    cplx* r = c.ws.cplxs(c.N);
    eta_vec(c, X, eom != 0, r);
    download(c, out, r, c.N);
    c.sync();
  });
}

cclr_status cclr_hessian(cclr_ctx* h, int nvec, const cclr_c128* u, cclr_c128* out, int on_device) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_lambda && u && out && nvec >= 1, CCLR_E_STATE, "hessian needs Lambda");
    PrecisionScope exact(c, exact_precision(c));
    Scope sc(c.ws);
    IO io(c, u, out, (int64_t)nvec * c.N, (int64_t)nvec * c.N, on_device != 0);
    hessian_right(c, nvec, io.in, io.dout);
    c.sync();
    io.finish();
  });
}

cclr_status cclr_zgemm_nt(cclr_ctx* h, int precision, int M, int N, int K, const cclr_c128* A, const cclr_c128* B,
                          cclr_c128* C) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_ham, CCLR_E_STATE, "cclr_zgemm_nt needs a Hamiltonian (device workspace)");
    CCLR_REQUIRE(M > 0 && N > 0 && K > 0 && A && B && C, CCLR_E_ARG, "bad GEMM arguments");
    CCLR_REQUIRE(valid_precision(precision), CCLR_E_ARG, "unknown precision");
    const int saved = c.opt.precision;
    c.opt.precision = precision;
    try {
      Scope sc(c.ws);
      cplx *a = c.ws.cplxs((int64_t)M * K), *b = c.ws.cplxs((int64_t)N * K), *d = c.ws.cplxs((int64_t)M * N);
      upload(c, a, A, (int64_t)M * K);
      upload(c, b, B, (int64_t)N * K);
      gemm_dispatch(c, false, true, M, N, K, cx(1), a, K, b, K, cx(0), d, N);
      CCLR_CK(cudaMemcpyAsync(C, d, sizeof(cplx) * (size_t)M * N, cudaMemcpyDeviceToHost, c.stream));
      c.sync();
    } catch (...) {
      c.opt.precision = saved;
      throw;
    }
    c.opt.precision = saved;
  });
}

cclr_status cclr_gram(cclr_ctx* h, int mirror, int64_t n, int nx, int ny, const cclr_c128* X, const cclr_c128* Y,
                      cclr_c128* out) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_ham, CCLR_E_STATE, "cclr_gram needs a Hamiltonian (device workspace)");
    CCLR_REQUIRE(n >= 1 && nx >= 1 && ny >= 1 && X && Y && out, CCLR_E_ARG, "bad Gram arguments");
    const bool saved = c.L.fast32;
    c.L.fast32 = true;
    try {
      Scope sc(c.ws);
      const int64_t np = n + (n & 1);   // mirror row stride (even)
      cplx *x = c.ws.cplxs((int64_t)nx * n), *y = c.ws.cplxs((int64_t)ny * n), *g = c.ws.cplxs((int64_t)nx * ny);
      cplx* scr = c.ws.cplxs(gram_scratch_elems());
      upload(c, x, X, (int64_t)nx * n);
      upload(c, y, Y, (int64_t)ny * n);
      Rows rx, ry;
      if (mirror) {
        float2* xf = (float2*)c.ws.alloc(sizeof(float2) * (size_t)nx * (size_t)np);
        float2* yf = (float2*)c.ws.alloc(sizeof(float2) * (size_t)ny * (size_t)np);
        for (int r = 0; r < nx; ++r) to_f32(c.L, x + (int64_t)r * n, xf + (int64_t)r * np, n);
        for (int r = 0; r < ny; ++r) to_f32(c.L, y + (int64_t)r * n, yf + (int64_t)r * np, n);
        rx.add(reinterpret_cast<const cplx*>(xf), nx, np);
        ry.add(reinterpret_cast<const cplx*>(yf), ny, np);
      } else {
        rx.add(x, nx, n);
        ry.add(y, ny, n);
      }
      gram(c.L, n, rx, ry, true, g, scr, gram_scratch_elems(), mirror != 0);
      CCLR_CK(cudaMemcpyAsync(out, g, sizeof(cplx) * (size_t)nx * ny, cudaMemcpyDeviceToHost, c.stream));
      c.sync();
    } catch (...) {
      c.L.fast32 = saved;
      throw;
    }
    c.L.fast32 = saved;
  });
}

cclr_status cclr_bench_vector_kernels(cclr_ctx* h, int precision, int64_t n, int nx, int ny, int m, int reps,
                                      double* ms3) {
  return guard(h, [&](Ctx& c) {
    CCLR_REQUIRE(c.have_ham, CCLR_E_STATE, "cclr_bench_vector_kernels needs a Hamiltonian (device workspace)");
    CCLR_REQUIRE(n >= 1 && nx >= 1 && ny >= 1 && m >= 1 && m <= kVecMatOut && nx <= kVecMatMaxRows && reps >= 1 && ms3,
                 CCLR_E_ARG, "bad vector-kernel benchmark arguments");
    CCLR_REQUIRE(valid_precision(precision), CCLR_E_ARG, "unknown precision");
    const bool saved = c.L.fast32;
    c.L.fast32 = mixed_precision(precision);   // the solver's rule: FP32 pairs, else float-float
    cplx *X = nullptr, *Y = nullptr, *C = nullptr, *G = nullptr, *scr = nullptr;
    double *vs = nullptr, *n2 = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
      c.L.fast32 = saved;
      for (cplx* p : {X, Y, C, G, scr}) c.dfree(p);
      c.dfree((cplx*)vs);
      c.dfree((cplx*)n2);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    };
    try {
      X = c.dalloc((int64_t)nx * n);
      Y = c.dalloc((int64_t)std::max(ny, m) * n);   // Gram operand (ny rows) and vecmat outputs (m rows)
      C = c.dalloc((int64_t)nx * m);
      G = c.dalloc((int64_t)nx * ny);
      scr = c.dalloc(gram_scratch_elems());
      vs = (double*)c.dalloc((vecmat_scratch_doubles() + 1) / 2);
      n2 = (double*)c.dalloc(kVecMatOut);
      fill_hash(c.L, X, (int64_t)nx * n, 1);
      fill_hash(c.L, Y, (int64_t)ny * n, 2);
      fill_hash(c.L, C, (int64_t)nx * m, 3);
      CCLR_CK(cudaEventCreate(&e0));
      CCLR_CK(cudaEventCreate(&e1));
      Rows rx, ry;
      rx.add(X, nx, n);
      ry.add(Y, ny, n);
      VecMat norms;   // Y_q = sum_j X_j C_jq, norms only (the solver's residual-norm pass)
      norms.X = rx;
      norms.m = m;
      norms.C = C;
      norms.norm2 = n2;
      VecMat write = norms;   // the same with the outputs stored (candidate corrections)
      write.Y = Y;
      write.ldy = n;
      const int calls = 3;
      for (int k = 0; k < calls; ++k) {
        auto run = [&]() {
          if (k == 0) gram(c.L, n, rx, ry, true, G, scr, gram_scratch_elems());
          else vecmat(c.L, n, k == 1 ? norms : write, vs);
        };
        run();   // warm-up
        CCLR_CK(cudaEventRecord(e0, c.stream));
        for (int r = 0; r < reps; ++r) run();
        CCLR_CK(cudaEventRecord(e1, c.stream));
        CCLR_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CCLR_CK(cudaEventElapsedTime(&ms, e0, e1));
        ms3[k] = ms / reps;
      }
      c.sync();
    } catch (...) {
      cleanup();
      throw;
    }
    cleanup();
  });
}

cclr_status cclr_kernel_profile(cclr_ctx* h, int enable, double* out8) {
  if (!h) return CCLR_E_ARG;
  Ctx& c = h->c;
  if (out8)
    for (int k = 0; k < 2; ++k) {
      out8[4 * k + 0] = (double)c.prof_launches[k];
      out8[4 * k + 1] = c.prof_ms[k];
      out8[4 * k + 2] = c.prof_flops_exec[k];
      out8[4 * k + 3] = c.prof_flops_useful[k];
    }
  for (int k = 0; k < 2; ++k) {
    c.prof_launches[k] = 0;
    c.prof_ms[k] = c.prof_flops_exec[k] = c.prof_flops_useful[k] = 0.0;
  }
  c.prof = enable != 0;
  c.kt.on = enable != 0;
  return CCLR_OK;
}

cclr_status cclr_kernel_breakdown(cclr_ctx* h, char* buf, int cap) {
  if (!h || !buf || cap < 1) return CCLR_E_ARG;
  Ctx& c = h->c;
  auto t = c.kt.totals;
  std::sort(t.begin(), t.end(), [](auto& a, auto& b) { return a.second.second > b.second.second; });
  std::string out;
  for (auto& e : t) {
    char line[256];
    std::snprintf(line, sizeof(line), "%s %ld %.6f\n", e.first.c_str(), e.second.first, e.second.second);
    out += line;
  }
  const size_t n = std::min<size_t>(out.size(), (size_t)cap - 1);
  std::memcpy(buf, out.data(), n);
  buf[n] = 0;
  c.kt.totals.clear();
  return CCLR_OK;
}

cclr_status cclr_debug_expire_next_wait(cclr_ctx* h, unsigned polls) {
  if (!h || polls == 0) return CCLR_E_ARG;
  h->c.dbg_wait_polls = polls;
  return CCLR_OK;
}

cclr_status cclr_response_batch(cclr_ctx* const* ctxs, int n, int n_ops, const cclr_c128* const* ops, int n_freq,
                                const double* omegas, double gamma, cclr_c128* const* out, cclr_status* status) {
  if (!ctxs || n < 1 || !ops || !out || !omegas) return CCLR_E_ARG;
  for (int k = 0; k < n; ++k)
    if (!ctxs[k] || !ops[k] || !out[k]) return CCLR_E_ARG;
  std::vector<cclr_status> st(n, CCLR_OK);
  auto one = [&](int k) {   // the whole response path of system k on its context's stream
    cclr_ctx* h = ctxs[k];
    cclr_status r = cc_ground(h, nullptr, nullptr);
    if (r == CCLR_OK) r = cc_lambda(h, nullptr);
    if (r == CCLR_OK) r = cc_lr_solve(h, n_ops, ops[k], n_freq, omegas, gamma, nullptr);
    if (r == CCLR_OK) r = cc_response_function(h, out[k]);
    st[k] = r;
  };
  std::vector<std::thread> th;
  try {
    for (int k = 1; k < n; ++k) th.emplace_back(one, k);
  } catch (...) {
    for (auto& t : th) t.join();
    return CCLR_E_ARG;
  }
  one(0);
  for (auto& t : th) t.join();
  cclr_status first = CCLR_OK;
  for (int k = 0; k < n; ++k) {
    if (status) status[k] = st[k];
    if (first == CCLR_OK) first = st[k];
  }
  return first;
}

cclr_status cclr_autotune_report(cclr_ctx* h, char* buf, int cap) {
  if (!h || !buf || cap < 1) return CCLR_E_ARG;
  const std::string out = tc_tune_report();
  const size_t n = std::min<size_t>(out.size(), (size_t)cap - 1);
  std::memcpy(buf, out.data(), n);
  buf[n] = 0;
  return CCLR_OK;
}

cclr_status cclr_get_stats(cclr_ctx* h, cclr_stats* out) {
  if (!h || !out) return CCLR_E_ARG;
  *out = h->c.stats;
  return CCLR_OK;
}

}  // extern "C"

// The library context: device, stream, workspace, Hamiltonian, amplitudes, Hbar and solver state.
#pragma once
#include "internal.h"
#include <complex>
#include <map>

namespace cclr {

typedef std::complex<double> zc;

struct ResponseData {
  // per operator k: shared trial space (basis and sigma vectors), projected matrices and the
  // subspace solutions of every shift.
  int n_ops = 0, n_freq = 0;
  double gamma = 0.0;
  std::vector<double> omegas;
  std::vector<zc> shifts;                 // unique shifts z
  std::vector<int> shift_of;              // [f*4+s] -> index into shifts
  std::vector<cplx*> ops_dev;             // property operators (n x n)
  std::vector<cplx*> xi, eta;             // per operator, length N
  std::vector<cplx*> basis, sig;          // per operator, max_subspace x N
  std::vector<int> nb;                    // basis size per operator
  std::vector<std::vector<zc>> H;         // per operator: B^H A B (nb x nb, row-major, stride maxL)
  std::vector<std::vector<zc>> C;         // per operator: -B^H xi
  std::vector<std::vector<zc>> beta;      // per operator: [shift][maxL] subspace solution
  std::vector<int> iters;                 // per (op, freq)
  bool solved = false;
  bool refined = false;                   // solutions from the FP64-class refinement
};

struct Ctx;
// BF16X3 / BF16X6: the modes whose vector passes run in FP32 and whose solves stop at floors
inline bool mixed_precision(int p) { return p == CCLR_TC_BF16X3 || p == CCLR_TC_BF16X6; }
int tc_slices(int precision);        // BF16 slices per operand in a tensor-core precision mode
// While alive, the BF16 slices of the transient operand src (elems complex values, unchanged
// meanwhile) are made once per view and reused by later contractions; workspace for `views`
// views is reserved from the context's arena at construction (declare it after the Scope that
// should release that space).  No effect in the FP64 mode.
struct SliceMemo {
  Ctx& c;
  bool active = false;
  SliceMemo(Ctx& c, const void* src, int64_t elems, int views);
  ~SliceMemo();
  SliceMemo(const SliceMemo&) = delete;
  SliceMemo& operator=(const SliceMemo&) = delete;
};
// While alive, the listed device ranges (pointer, bytes) hold values on a grid of 2^(e - 14), e the
// exponent with |x| < 2^e of the largest element: exactly two FP64-class digits in every operand
// view, so the FP64-class GEMMs skip the digit products that involve their lower digits.
struct CoarseOperands {
  Ctx& c;
  int n = 0;
  CoarseOperands(Ctx& c, std::initializer_list<std::pair<const void*, size_t>> ranges);
  ~CoarseOperands();
  CoarseOperands(const CoarseOperands&) = delete;
  CoarseOperands& operator=(const CoarseOperands&) = delete;
};
struct TcState;                      // per-context state of the tensor-core path (tc_gemm.cu)
void tc_release_cache_for(Ctx& c);   // frees the cached BF16 slices of persistent operands
size_t tc_cache_bytes(Ctx& c);       // bytes held by that cache
void tc_state_free(Ctx& c);          // frees all of it

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Launch L;
  long launches = 0;
  cclr_options opt{};
  std::string err;
  cclr_stats stats{};
  Arena ws;

  // sizes
  int o = 0, v = 0, n = 0;
  int64_t Po = 0, Pv = 0, Ns = 0, Nd = 0, N = 0;
  int2 *po = nullptr, *pv = nullptr;     // pair tables (p, q), p < q, in packed order

  // Hamiltonian
  cplx* fock = nullptr;                                   // n x n
  cplx *oooo = nullptr, *ooov = nullptr, *oovv = nullptr, *ovov = nullptr, *ovvv = nullptr;  // full index
  cplx *vvvv_p = nullptr, *oovv_p = nullptr, *ovvv_p = nullptr;                                 // packed
  double* D = nullptr;                                    // orbital-energy differences, length N
  double* Dpre = nullptr;   // Davidson preconditioner: differences of the dressed one-body diagonal (Re F_aa, Re F_ii)
  bool have_ham = false;

  // amplitudes (t and lambda), amplitude layout and full doubles
  cplx *t = nullptr, *t2 = nullptr;                       // t: N (t1 | t2 packed); t2: o,o,v,v
  cplx *lam = nullptr, *l2 = nullptr;
  bool have_t = false, have_lambda = false;
  zc e_corr = 0.0;

  // Hbar (creators-first elements, see the oracle's definitions)
  cplx *Fae = nullptr, *Fmi = nullptr, *Fme = nullptr;
  cplx *Fae_od = nullptr, *Fmi_od = nullptr;             // Fae, Fmi minus the bare Fock diagonal
  cplx *Wmnij = nullptr, *Wmnij_p = nullptr, *Wabef_p = nullptr, *Wmbej = nullptr;
  cplx *WringR = nullptr, *WringL = nullptr;              // (j,b) x (m,e) operands of the rings
  cplx *Wmnie = nullptr, *Wamef = nullptr, *Wmbij = nullptr, *Wabei = nullptr;
  cplx *tau = nullptr;                                    // o,o,v,v
  bool have_hbar = false;

  std::vector<void*> persistent;                          // all cudaMalloc'd arrays
  std::vector<size_t> persistent_bytes;
  std::map<std::string, void*> named;

  ResponseData rd;
  std::vector<zc> eom_w;            // EOM-EE roots of the last cc_eom_ee and their right vectors
  std::vector<cplx*> eom_vecs;

  // tensor-core status word (bounded-wait expiry) and optional per-launch timing of the
  // tensor-core kernel with CUDA events on the context's stream
  int* tc_err = nullptr;
  // test of the expiry path: the next tensor-core GEMM launch gets this poll limit and a first
  // wait that nothing completes (0 = no test pending)
  uint32_t dbg_wait_polls = 0;
  // sigma inputs rounded to the coarse grid (round_coarse): the sigma products mark their
  // gathered copies as CoarseOperands
  bool coarse_sigma = false;
  TcState* tcs = nullptr;      // slice cache, memos, coarse ranges, autotuner launches
  uint64_t data_gen = 1;       // bumped whenever integrals, T, Lambda or Hbar change
  KernelTimer kt;   // per-kernel timing (switched on with the tensor-core timing)
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  std::vector<int> ev_kind;   // per used pair: 0 split-BF16 kernel, 1 FP64-class kernel
  size_t ev_used = 0;
  // per kernel kind: launches, milliseconds, executed BF16 flops, useful complex flops (8 M N K)
  double prof_ms[2] = {}, prof_flops_exec[2] = {}, prof_flops_useful[2] = {};
  long prof_launches[2] = {};
  void prof_events(cudaEvent_t& a, cudaEvent_t& b, int kind) {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t x, y;
      CCLR_CK(cudaEventCreate(&x));
      CCLR_CK(cudaEventCreate(&y));
      ev_pool.push_back({x, y});
      ev_kind.push_back(0);
    }
    a = ev_pool[ev_used].first;
    b = ev_pool[ev_used].second;
    ev_kind[ev_used] = kind;
    ++ev_used;
  }
  void prof_collect() {  // after a stream synchronize
    for (size_t i = 0; i < ev_used; ++i) {
      float ms = 0.f;
      CCLR_CK(cudaEventElapsedTime(&ms, ev_pool[i].first, ev_pool[i].second));
      prof_ms[ev_kind[i]] += ms;
      ++prof_launches[ev_kind[i]];
    }
    ev_used = 0;
  }

  // helpers
  cplx* dalloc(int64_t n_elems) {
    void* p = nullptr;
    const size_t bytes = sizeof(cplx) * (size_t)(n_elems > 0 ? n_elems : 1);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {   // the tensor-core slice cache yields its memory first
      cudaGetLastError();
      tc_release_cache_for(*this);
      CCLR_CK(cudaMalloc(&p, bytes));
    }
    persistent.push_back(p);
    persistent_bytes.push_back(bytes);
    return (cplx*)p;
  }
  void dfree(void* p) {
    if (!p) return;
    for (size_t i = 0; i < persistent.size(); ++i)
      if (persistent[i] == p) {
        cudaFree(p);
        persistent.erase(persistent.begin() + i);
        persistent_bytes.erase(persistent_bytes.begin() + i);
        return;
      }
  }
  size_t persistent_total() const {
    size_t t = 0;
    for (size_t b : persistent_bytes) t += b;
    return t;
  }
  void sync() { CCLR_CK(cudaStreamSynchronize(stream)); }

  // views of the integral classes with every index explicit (Hermiticity / antisymmetry views)
  Tensor V(const char* cls) const;
  Tensor f(const char* blk) const;     // Fock blocks "oo", "ov", "vo", "vv" as strided views
};

// The contraction arithmetic of c switched for the lifetime of the object
struct PrecisionScope {
  Ctx& c;
  int old;
  PrecisionScope(Ctx& cc, int p) : c(cc), old(cc.opt.precision) { c.opt.precision = p; }
  ~PrecisionScope() { c.opt.precision = old; }
};
// mixed-precision mode with FP64 refinement (cclr_options.refine)
inline bool refining(const Ctx& c) { return mixed_precision(c.opt.precision) && c.opt.refine != 0; }
// the arithmetic of the quantities that define the answer (Hbar, xi, eta, Hessian products)
inline int exact_precision(const Ctx& c) { return refining(c) ? CCLR_TC_F64 : c.opt.precision; }
// floor of the mixed-precision phase relative to the right-hand side
inline double mixed_floor(const Ctx& c) { return c.opt.refine_tol > 0.0 ? c.opt.refine_tol : 2e-5; }

// GEMM backend selection (FP64 DFMA or tensor cores), row-major, see zgemm()
void gemm_dispatch(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A,
                   int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc);


bool tc_eligible(int64_t M, int64_t N, int64_t K);
// C[m*ldc + n] = alpha sum_k vm[m,k] vn[n,k] + beta C on the tensor cores; the first nrm / nrn
// axes of the views are the rows, the remaining axes K (in the same order in both views)
// Output map of a strided GEMM result: element (m, n) at C + moff(m) + noff(n), each a row-major
// decomposition over up to four axes.
struct OutAxes {
  int nm = 0, nn = 0;
  int64_t mdim[4] = {}, mstr[4] = {}, ndim[4] = {}, nstr[4] = {};
};
void tc_gemm_views(Ctx& c, const Tensor& vm, int nrm, const Tensor& vn, int nrn, cplx alpha, cplx beta, cplx* C,
                   int64_t ldc, const OutAxes* oa = nullptr);
// split-K slices the tensor-core GEMM would use for this shape (strided: output through a row map)
int tc_splits(const Ctx& c, int64_t M, int64_t N, int64_t K, bool strided);
void tc_tune_collect(Ctx& c);    // resolves the tile autotuner's timed launches (after a stream sync)
std::string tc_tune_report();    // decided tile shapes, one line per GEMM shape

// equations (ccsd.cu, sigma.cu, props.cu)
void build_denominators(Ctx& c);
zc ccsd_energy(Ctx& c);
void ccsd_residual(Ctx& c, cplx* R);               // R: amplitude layout
void build_hbar(Ctx& c);
void sigma_right(Ctx& c, int nvec, const cplx* in, cplx* out);
void sigma_left(Ctx& c, int nvec, const cplx* in, cplx* out);
void xi_vec(Ctx& c, const cplx* X, cplx* out);
void eta_vec(Ctx& c, const cplx* X, bool eom, cplx* out);
void hessian_right(Ctx& c, int nvec, const cplx* in, cplx* out);
void xi_density(Ctx& c, const cplx* l, cplx* D);     // D: l . xi^X = sum D[p,q] X[p,q]
void eta_density(Ctx& c, const cplx* v, cplx* D);    // D: eta^X . v = sum D[p,q] X[p,q]
void eta_ground(Ctx& c, cplx* out);
void expand_t2(Ctx& c, const cplx* packed, cplx* full, int64_t nvec);   // packed doubles -> o,o,v,v
void pack_anti(Ctx& c, const Tensor& X, cplx* D, int64_t nvec, cplx alpha, bool anti, bool acc);

// solvers (solver.cu)
int solve_ground(Ctx& c);
int solve_lambda(Ctx& c);
void release_response(Ctx& c);   // frees the arrays of the last linear-response solve
void lr_solve(Ctx& c, int n_ops, const cplx* ops_host, int n_freq, const double* omegas, double gamma,
              int* iters_out);
void response_function(Ctx& c, cplx* out_host);
void response_function_ci(Ctx& c, cplx* out_host);
void response_function_asym(Ctx& c, cplx* out_host);
void field_derivative(Ctx& c, const cplx* V, cplx* out_host);   // d<<X;Y>>/d eps, field V on the Fock matrix
void response_gradient(Ctx& c, int f, cplx* out_host);   // operator gradient of <<X;Y>> (adjoint)
void left_solve(Ctx& c, int nrhs, const cplx* rhs, zc w, cplx* out);   // l (A + w) = -b
void synthetic_instance(Ctx& c, int n_occ, int n_vir, uint64_t seed, double sd, double dip_sd, int n_ops,
                        cplx* const blocks[6], double* eps_u, cplx* ops);   // counter-based instance
int eom_ee(Ctx& c, int nroots, std::vector<zc>& w_out);

// small dense complex linear algebra on the host
void zsolve(int n, std::vector<zc>& A, std::vector<zc>& b);   // A (n x n row-major) x = b, in place

}  // namespace cclr

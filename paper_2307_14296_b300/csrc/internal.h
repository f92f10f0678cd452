// Internal declarations of libcclr (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include <stdexcept>
#include <initializer_list>
#include <algorithm>
#include "../../include/cclr.h"

namespace cclr {

typedef double2 cplx;   // interleaved complex FP64, same layout as cclr_c128

struct Error : std::runtime_error {
  cclr_status st;
  Error(cclr_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};

#define CCLR_CK(x)                                                                          \
  do {                                                                                      \
    cudaError_t e_ = (x);                                                                   \
    if (e_ != cudaSuccess)                                                                  \
      throw ::cclr::Error(e_ == cudaErrorMemoryAllocation ? CCLR_E_OOM : CCLR_E_CUDA,       \
                          std::string(#x " failed: ") + cudaGetErrorString(e_) + " at " +  \
                              __FILE__ + ":" + std::to_string(__LINE__));                   \
  } while (0)

#define CCLR_REQUIRE(cond, st, msg) \
  do { if (!(cond)) throw ::cclr::Error(st, msg); } while (0)

constexpr int kMaxRank = 8;

// A strided view of a complex tensor in device memory.  Reads apply conj (if set) and then
// multiply by `scale` (real).  Writes ignore conj/scale.
struct Tensor {
  cplx* p = nullptr;
  int rank = 0;
  int64_t dim[kMaxRank] = {};
  int64_t str[kMaxRank] = {};
  bool conj = false;
  double scale = 1.0;

  int64_t numel() const {
    int64_t n = 1;
    for (int i = 0; i < rank; ++i) n *= dim[i];
    return n;
  }
  static Tensor make(cplx* p, std::initializer_list<int64_t> dims) {
    Tensor t;
    t.p = p;
    t.rank = (int)dims.size();
    int i = 0;
    for (int64_t d : dims) t.dim[i++] = d;
    int64_t s = 1;
    for (int k = t.rank - 1; k >= 0; --k) { t.str[k] = s; s *= t.dim[k]; }
    return t;
  }
  static Tensor make(cplx* p, const std::vector<int64_t>& dims) {
    Tensor t;
    t.p = p;
    t.rank = (int)dims.size();
    for (int i = 0; i < t.rank; ++i) t.dim[i] = dims[i];
    int64_t s = 1;
    for (int k = t.rank - 1; k >= 0; --k) { t.str[k] = s; s *= t.dim[k]; }
    return t;
  }
  // view with axes reordered: new axis k is old axis perm[k]
  Tensor perm(std::initializer_list<int> pm) const {
    Tensor t = *this;
    int k = 0;
    for (int a : pm) { t.dim[k] = dim[a]; t.str[k] = str[a]; ++k; }
    return t;
  }
  Tensor neg() const { Tensor t = *this; t.scale = -scale; return t; }
  Tensor scaled(double s) const { Tensor t = *this; t.scale = scale * s; return t; }
  Tensor cj() const { Tensor t = *this; t.conj = !conj; return t; }
  bool contiguous() const {
    int64_t s = 1;
    for (int k = rank - 1; k >= 0; --k) { if (dim[k] != 1 && str[k] != s) return false; s *= dim[k]; }
    return true;
  }
};

// Bump allocator over one device buffer; mark()/release() bracket temporaries.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, top = 0, peak = 0;
  void* alloc(size_t bytes) {
    size_t a = (top + 255) & ~size_t(255);
    if (a + bytes > cap)
      throw Error(CCLR_E_OOM, "workspace exhausted: need " + std::to_string((a + bytes) >> 20) +
                                  " MiB of " + std::to_string(cap >> 20) + " MiB");
    top = a + bytes;
    if (top > peak) peak = top;
    return base + a;
  }
  cplx* cplxs(int64_t n) { return (cplx*)alloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1)); }
  size_t mark() const { return top; }
  void release(size_t m) { top = m; }
};

struct Scope {  // RAII release of arena temporaries
  Arena& a;
  size_t m;
  explicit Scope(Arena& ar) : a(ar), m(ar.mark()) {}
  ~Scope() { a.release(m); }
};

// ---------------------------------------------------------------- kernels (kernels.cu)
// Per-kernel timing: when on, a pair of CUDA events is recorded on the stream around every
// launch (begin() before, end() after); collect() (after a stream synchronize) adds the
// durations to per-name totals.
struct KernelTimer {
  bool on = false;
  const char* label = nullptr;   // contraction being executed (kept in the names when set)
  std::vector<cudaEvent_t> pool;
  std::vector<std::string> names;
  size_t used = 0;
  std::vector<std::pair<std::string, std::pair<long, double>>> totals;   // name -> (launches, ms)
  cudaEvent_t next(cudaStream_t s) {
    if (used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) throw Error(CCLR_E_CUDA, "cudaEventCreate failed");
      pool.push_back(e);
    }
    cudaEvent_t e = pool[used++];
    if (cudaEventRecord(e, s) != cudaSuccess) throw Error(CCLR_E_CUDA, "cudaEventRecord failed");
    return e;
  }
  void begin(cudaStream_t s) {
    if (on) next(s);
  }
  void end(cudaStream_t s, const char* name) {
    if (!on || used % 2 == 0) return;   // no begin() recorded for this launch
    next(s);
    names.push_back(label ? std::string(label) + " | " + name : std::string(name));
  }
  void collect() {
    // CCLR_PROFILE_DETAIL=2: also print every timed launch, in launch order
    static const bool trace = [] {
      const char* e = std::getenv("CCLR_PROFILE_DETAIL");
      return e != nullptr && e[0] == '2';
    }();
    for (size_t i = 0; i + 1 < used; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pool[i], pool[i + 1]) != cudaSuccess) continue;
      const std::string& nm = names[i / 2];
      if (trace) std::fprintf(stderr, "[cclr] launch %s %.4f ms\n", nm.c_str(), ms);
      auto it = std::find_if(totals.begin(), totals.end(), [&](auto& t) { return t.first == nm; });
      if (it == totals.end()) totals.push_back({nm, {1, ms}});
      else { it->second.first += 1; it->second.second += ms; }
    }
    used = 0;
    names.clear();
  }
};

struct Launch {  // stream + launch counter shared by all kernels of one context
  cudaStream_t s = nullptr;
  long* count = nullptr;
  KernelTimer* kt = nullptr;
  // FP32 arithmetic (FP64 storage) in the solvers' vector kernels (dots, vecmat, Gram blocks);
  // set by the iterative solvers in the tensor-core modes only.
  bool fast32 = false;
  // device status word of the context: kernels with bounded waits record an expiry here (the
  // API layer checks it at the end of every call)
  int* err = nullptr;
};

// dst = alpha * op(src) + (accumulate ? dst : 0), element-wise over dst's shape; src must
// have the same rank/dims (strides arbitrary).
void permute(const Launch& L, const Tensor& src, const Tensor& dst, cplx alpha, bool accumulate);
void fill_zero(const Launch& L, cplx* p, int64_t n);
void flag_nonfinite(const Launch& L, const cplx* p, int64_t n, int* flag);   // *flag = 1 on inf / NaN
// x <- x rounded to the grid 2^(e - 14) of its largest element (|x| < 2^e): 15 significant bits
// relative to that element, exactly two FP64-class digits in any view (scratch: one word)
void round_coarse(const Launch& L, cplx* x, int64_t n, unsigned* scratch);
void fill_hash(const Launch& L, cplx* p, int64_t n, uint64_t seed);   // deterministic values in [-1, 1)^2

// Row-major complex FP64 GEMM: C[MxN] = alpha op(A) op(B) + beta C; op(A)[m,k] = ta ? A[k*lda+m]
// : A[m*lda+k]; op(B)[k,n] = tb ? B[n*ldb+k] : B[k*ldb+n].
void zgemm(const Launch& L, bool ta, bool tb, int64_t M, int64_t N, int64_t K, cplx alpha,
           const cplx* A, int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc);

// Doubles packing.  X is a full antisymmetric view with axes (Z, i, j, a, b) (any strides).
// pack:  D[z][P(i,j)][P(a,b)] = alpha * (anti ? X_ijab - X_jiab - X_ijba + X_jiba : X_ijab)
//                              + (accumulate ? D : 0)
void pack_doubles_impl(const Launch& L, const Tensor& X, cplx* D, int64_t nvec, int o, int v, cplx alpha,
                       bool anti, bool accumulate, const int2* po, const int2* pv);
// unpack: X(Z,i,j,a,b) = D[z][P(i,j)][P(a,b)] with antisymmetry signs (0 on the diagonals)
void unpack_doubles(const Launch& L, const cplx* D, int64_t ld_vec, const Tensor& X, int o, int v);

// Up to four segments of equally strided device vectors, read as one list of rows
// (row j of segment s is p[s] + j * ld[s]).
struct Rows {
  const cplx* p[4] = {};
  int64_t ld[4] = {};
  int cnt[4] = {};
  int ns = 0;
  __host__ __device__ int total() const {
    int t = 0;
    for (int s = 0; s < ns; ++s) t += cnt[s];
    return t;
  }
  Rows& add(const cplx* ptr, int count, int64_t stride) {
    if (count > 0) {
      if (ns == 4) throw Error(CCLR_E_ARG, "Rows: more than four segments");
      p[ns] = ptr; cnt[ns] = count; ld[ns] = stride; ++ns;
    }
    return *this;
  }
  // rows [j0, j0 + n); f32: the rows are FP32 mirrors (strides count float2 elements)
  Rows slice(int j0, int n, bool f32 = false) const {
    Rows r;
    for (int s = 0; s < ns && n > 0; ++s) {
      if (j0 >= cnt[s]) { j0 -= cnt[s]; continue; }
      const int take = std::min(cnt[s] - j0, n);
      const int64_t bytes = (int64_t)j0 * ld[s] * (f32 ? 8 : 16);
      r.add(reinterpret_cast<const cplx*>(reinterpret_cast<const char*>(p[s]) + bytes), take, ld[s]);
      n -= take;
      j0 = 0;
    }
    return r;
  }
};

// Multi-output linear combination over n elements, one pass over the inputs:
//   r_q = sum_j X_j C[j*m + q] + add,  q < m <= 16
//   Y_q = (D ? -r_q / (D - z_q) : r_q) + (acc ? Y_q : 0)
// with optional norm2[q] = |r_q|^2 (or |Y_q|^2 if norm_y).  Products and sums in FP32 pairs
// when Launch::fast32 (FP64 storage), otherwise FP64.  All device pointers; C has X.total() x m
// entries; scratch holds vecmat_scratch_doubles() when norms are requested.
struct VecMat {
  Rows X;
  int m = 0;
  const cplx* C = nullptr;
  const cplx* add = nullptr;
  cplx* Y = nullptr;
  int64_t ldy = 0;
  bool acc = false;
  const double* D = nullptr;
  const cplx* z = nullptr;
  double* norm2 = nullptr;
  bool norm_y = false;
  // X rows hold FP32 complex values (float2; row pointers cast to cplx*, strides in float2
  // elements): the FP32 mirrors of the solver's trial vectors.  Needs Launch::fast32.
  bool x32 = false;
  // optional per-output additive rows (FP32 complex, float2 elements): r_q += addq[arow[q] * ldadd + i]
  // (the stored anchor residuals of the refinement).  Needs Launch::fast32.
  const void* addq = nullptr;
  int64_t ldadd = 0;
  int arow[16] = {};
};
// y[i] = x[i] rounded to FP32 (float2), n complex values (the solver's FP32 mirrors)
void to_f32(const Launch& L, const cplx* x, void* y, int64_t n);
constexpr int kVecMatOut = 16;        // outputs per pass
constexpr int kVecMatMaxRows = 512;   // inputs per pass
int64_t vecmat_scratch_doubles();
void vecmat(const Launch& L, int64_t n, const VecMat& a, double* scratch);

// Vector kernels over n complex elements (batched over nvec contiguous vectors of length n).
void axpy(const Launch& L, int64_t n, cplx a, const cplx* x, cplx* y);                  // y += a x
// out[k] = sum_i op(x_k[i]) * y_k[i] (conj x if herm) for k < nvec, x_k = x + k*ldx
void dots(const Launch& L, int64_t n, int nvec, const cplx* x, int64_t ldx, const cplx* y,
          int64_t ldy, bool herm, cplx* out_dev, cplx* scratch);
// out[j] = sum_i conj(B_j[i]) y[i] for j < nb (B_j = B + j*ldb): Gram-style projections
void proj(const Launch& L, int64_t n, int nb, const cplx* B, int64_t ldb, const cplx* y, cplx* out_dev,
          cplx* scratch);
// y = sum_j c[j] X_j + (accumulate ? y : 0) with coefficients on the device
void lincomb(const Launch& L, int64_t n, int nb, const cplx* X, int64_t ldx, const cplx* c_dev, cplx* y,
             bool accumulate);

int reduce_blocks();
// streaming multiprocessors of the current device (queried once per device)
int num_sms();
// true on the first call for the current device (done: 64 per-device flags), e.g. for per-device
// kernel attributes
bool once_per_device(bool* done);

// Split-K GEMM for skinny shapes: partials P[z] = op(A) op(B) over k in [z*kchunk, (z+1)*kchunk)
// (S slices, each M x N with ld N), then C = alpha * sum_z P[z] + beta * C in a fixed order.
void zgemm_splitk(const Launch& L, bool ta, bool tb, int64_t M, int64_t N, int64_t K, const cplx* A, int64_t lda,
                  const cplx* B, int64_t ldb, cplx* P, int S, int64_t kchunk);
void splitk_reduce(const Launch& L, const cplx* P, int S, int64_t M, int64_t N, cplx alpha, cplx beta, cplx* C,
                   int64_t ldc);

// 3-D pair packing over the last two axes of X (R, m, m):
//   pack2:   D[r*ldd + P(p,q)] = alpha (anti ? X[r,p,q] - X[r,q,p] : X[r,p,q]) (+ D)
//   unpack2: X[r,p,q] = +-D[r*ldd + P(min,max)], 0 for p == q
void pack2(const Launch& L, const Tensor& X, cplx* D, int64_t ldd, const int2* tab, cplx alpha, bool anti, bool acc);
void unpack2(const Launch& L, const cplx* D, int64_t ldd, const Tensor& X);
// Gram block out[i*ny + j] = sum_n op(X_i[n]) Y_j[n] (conj X if herm) over row lists of any
// length (tiles of 64 x 8 rows, longer list first), out_dev holding nx * ny.  FP32 products
// summed in FP32 over runs of 32 elements and in FP64 across runs when Launch::fast32, FP64
// otherwise.  Row starts must be 16-byte aligned; scratch holds gram_scratch_elems().
void gram(const Launch& L, int64_t n, const Rows& X, const Rows& Y, bool herm, cplx* out_dev, cplx* scratch,
          int64_t scratch_elems, bool x32 = false);   // x32: all rows FP32 mirrors (even strides)
inline int64_t gram_scratch_elems() { return (int64_t)num_sms() * 64 * 8; }

// Small element-wise helpers
void scale_vec(const Launch& L, int64_t n, cplx a, cplx* x);
void copy_vec(const Launch& L, int64_t n, const cplx* x, cplx* y);
// y[z*n + i] += D[i] * x[z*n + i] for z < nvec (FP64): the diagonal part of a sigma product
void diag_axpy(const Launch& L, int64_t n, int64_t nvec, const double* D, const cplx* x, cplx* y);
// x_i <- x_i / (D_i - z) * a   (Jacobi update)
void div_shift(const Launch& L, int64_t n, const cplx* x, const double* D, cplx z, cplx a, cplx* y);

// ---------------------------------------------------------------- contraction planner
struct Ctx;
// C[c] = alpha * sum A[a] B[b] + beta * C  for spec "a,b->c" (letters are index names); beta
// is 0 or 1.  Index extents come from the tensors.  Letters present only in one operand are not
// allowed; letters present in all three operands are not allowed.
void einsum(Ctx& c, const char* spec, cplx alpha, const Tensor& A, const Tensor& B, double beta,
            const Tensor& C);

inline cplx cx(double r, double i = 0.0) { return make_double2(r, i); }

}  // namespace cclr

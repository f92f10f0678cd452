// Complex FP64 kernels of libcclr: strided permutation, DFMA GEMM, doubles pack/unpack, and the
// vector kernels of the iterative solvers (dots, projections, linear combinations, the fused
// residual + orbital-energy-denominator preconditioner).  All reductions are deterministic:
// a fixed grid writes partial sums that one block adds in a fixed order.
#include "internal.h"
#include <algorithm>
#include <type_traits>

namespace cclr {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }

inline int grid_for(int64_t n, int per = kThreads) {
  int64_t g = (n + per - 1) / per;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

inline void kbeg(const Launch& L) {   // before a launch: timer start (when per-kernel timing is on)
  if (L.kt) L.kt->begin(L.s);
}
inline void bump(const Launch& L, const char* name) {   // after a launch: count it, timer stop
  if (L.count) ++*L.count;
  if (L.kt) L.kt->end(L.s, name);
}
// kernel name with its shape when every launch is traced (CCLR_PROFILE_DETAIL=2)
inline const char* shaped(const char* name, int a, int b, int c) {
  static const bool on = [] {
    const char* e = std::getenv("CCLR_PROFILE_DETAIL");
    return e != nullptr && e[0] == '2';
  }();
  if (!on) return name;
  static thread_local char buf[96];
  std::snprintf(buf, sizeof buf, "%s[%d,%d,%d]", name, a, b, c);
  return buf;
}

struct PermArgs {
  int rank;
  int64_t dim[kMaxRank];
  int64_t sstr[kMaxRank];
  int64_t dstr[kMaxRank];
  uint32_t mul[kMaxRank];   // Granlund-Montgomery multipliers of dim (32-bit quotients)
  int shr[kMaxRank];
};

// q = n / d for 32-bit n with the multiplier m and shift l of d: q = (umulhi(n, m) + n) >> l
__device__ __forceinline__ uint32_t gm_div(uint32_t n, uint32_t m, int l) {
  return (uint32_t)(((uint64_t)__umulhi(n, m) + n) >> l);
}

template <int AK>
__device__ __forceinline__ cplx scale_alpha(cplx x, cplx alpha, bool conj) {
  if (conj) x.y = -x.y;
  if (AK == 0) {
    if (alpha.x < 0) { x.x = -x.x; x.y = -x.y; }
  } else if (AK == 1) {
    x.x *= alpha.x;
    x.y *= alpha.x;
  } else {
    x = cmul(alpha, x);
  }
  return x;
}

// alpha kinds: 0 -> +-1 real (sign only), 1 -> real, 2 -> complex.  Element-wise in the
// destination's index order; W32: every index is below 2^31 and the multipliers are used.
template <int AK, bool W32>
__global__ void __launch_bounds__(kThreads) k_permute(PermArgs a, const cplx* __restrict__ src, cplx* dst,
                                                      int64_t n, cplx alpha, bool conj, bool acc) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t so = 0, dof = 0;
    if (W32) {
      uint32_t r = (uint32_t)idx;
#pragma unroll
      for (int k = kMaxRank - 1; k >= 0; --k) {
        if (k < a.rank) {
          const uint32_t q = gm_div(r, a.mul[k], a.shr[k]);
          const int64_t c = (int64_t)(r - q * (uint32_t)a.dim[k]);
          r = q;
          so += c * a.sstr[k];
          dof += c * a.dstr[k];
        }
      }
    } else {
      int64_t r = idx;
#pragma unroll
      for (int k = kMaxRank - 1; k >= 0; --k) {
        if (k < a.rank) {
          const int64_t q = r / a.dim[k];
          const int64_t c = r - q * a.dim[k];
          r = q;
          so += c * a.sstr[k];
          dof += c * a.dstr[k];
        }
      }
    }
    cplx x = scale_alpha<AK>(src[so], alpha, conj);
    if (acc) x = cadd(x, dst[dof]);
    dst[dof] = x;
  }
}

// Transposing permutation through shared memory: axis S has unit source stride, axis T unit
// destination stride (S != T).  One 32 x 32 tile of (S, T) per step, the other axes ("batch")
// decoded from the tile index; reads are coalesced along S and writes along T.
struct TileArgs {
  int nb;                      // batch axes
  int64_t bdim[kMaxRank], bsstr[kMaxRank], bdstr[kMaxRank];
  uint32_t bmul[kMaxRank];
  int bshr[kMaxRank];
  int64_t dimS, dimT, sstrT, dstrS;   // extents of S and T, source stride of T, destination stride of S
  uint32_t ntS, ntT;                  // tiles along S and T
  uint32_t mulS, mulT;                // multipliers of ntS, ntT
  int shrS, shrT;
};

template <int AK>
__global__ void __launch_bounds__(256) k_permute_tiled(TileArgs a, const cplx* __restrict__ src, cplx* dst,
                                                       int64_t ntiles, cplx alpha, bool conj, bool acc) {
  __shared__ cplx tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint32_t r = (uint32_t)t;
    const uint32_t qS = gm_div(r, a.mulS, a.shrS);
    const int64_t s0 = (int64_t)(r - qS * a.ntS) * 32;
    r = qS;
    const uint32_t qT = gm_div(r, a.mulT, a.shrT);
    const int64_t t0 = (int64_t)(r - qT * a.ntT) * 32;
    r = qT;
    int64_t sb = 0, db = 0;
#pragma unroll
    for (int k = kMaxRank - 1; k >= 0; --k) {
      if (k < a.nb) {
        const uint32_t q = gm_div(r, a.bmul[k], a.bshr[k]);
        const int64_t c = (int64_t)(r - q * (uint32_t)a.bdim[k]);
        r = q;
        sb += c * a.bsstr[k];
        db += c * a.bdstr[k];
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {   // read: tx along S (unit source stride), rows along T
      const int64_t s = s0 + tx, tt = t0 + ty + 8 * i;
      if (s < a.dimS && tt < a.dimT) tile[ty + 8 * i][tx] = src[sb + s + tt * a.sstrT];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {   // write: tx along T (unit destination stride), rows along S
      const int64_t tt = t0 + tx, s = s0 + ty + 8 * i;
      if (s < a.dimS && tt < a.dimT) {
        cplx x = scale_alpha<AK>(tile[tx][ty + 8 * i], alpha, conj);
        cplx* d = dst + db + tt + s * a.dstrS;
        if (acc) x = cadd(x, *d);
        *d = x;
      }
    }
    __syncthreads();
  }
}

// p[i] = deterministic values in [-1, 1) + i [-1, 1) from a 64-bit mix of (seed, i) (test and
// benchmark operands)
__global__ void k_fill_hash(cplx* p, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull + seed;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    const uint32_t a = (uint32_t)h, b = (uint32_t)(h >> 32);
    p[i] = make_double2((double)a * 0x1p-31 - 1.0, (double)b * 0x1p-31 - 1.0);
  }
}

// *out = largest biased binary64 exponent of the real and imaginary parts (out zeroed beforehand)
__global__ void k_max_bexp(const cplx* __restrict__ x, int64_t n, unsigned* out) {
  unsigned m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx v = x[i];
    m = max(m, max((unsigned)((uint64_t)__double_as_longlong(v.x) >> 52) & 0x7ffu,
                   (unsigned)((uint64_t)__double_as_longlong(v.y) >> 52) & 0x7ffu));
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}
// x <- x rounded to the nearest multiple of 2^(e - 14), e = *bexp - 1022 (|x| < 2^e for all x)
__global__ void k_round_grid(cplx* x, int64_t n, const unsigned* bexp) {
  const unsigned b = *bexp;
  if (b == 0u || b == 0x7ffu) return;
  const int k = (int)b - 1036;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cplx v = x[i];
    v.x = scalbn(rint(scalbn(v.x, -k)), k);
    v.y = scalbn(rint(scalbn(v.y, -k)), k);
    x[i] = v;
  }
}

// *flag = 1 if any real or imaginary part is an infinity or a NaN
__global__ void k_nonfinite(const cplx* __restrict__ p, int64_t n, int* flag) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx x = p[i];
    bad |= !isfinite(x.x) || !isfinite(x.y);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

__global__ void k_fill_zero(cplx* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = make_double2(0.0, 0.0);
}

// ---------------------------------------------------------------------------- DFMA GEMM
// 64x64 output tile per 256-thread block, 4x4 complex outputs per thread, K step 8.  FP64 FMA
// throughput on sm_103 is ~2 DFMA/clk/SM, so this simple shared-memory tiling already runs at
// the FP64 pipe limit (the tile's shared-memory traffic is ~30x below what the pipe consumes).
constexpr int BM = 64, BN = 64, BK = 8;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_zgemm(int64_t M, int64_t N, int64_t K, cplx alpha,
                                               const cplx* __restrict__ A, int64_t lda,
                                               const cplx* __restrict__ B, int64_t ldb, cplx beta,
                                               cplx* __restrict__ C, int64_t ldc, int64_t kchunk, int64_t cz) {
  // split-K: blockIdx.z owns k in [z*kchunk, min(K, (z+1)*kchunk)) and writes C + z*cz
  __shared__ cplx As[BK][BM + 1];
  __shared__ cplx Bs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  C += (int64_t)blockIdx.z * cz;
  cplx acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int e0 = 0; e0 < BM * BK; e0 += 256) {
      const int e = e0 + threadIdx.x;
      int mm, kk;
      if (!TA) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      cplx val = make_double2(0.0, 0.0);
      if (gm < M && gk < kend) val = TA ? A[gk * lda + gm] : A[gm * lda + gk];
      As[kk][mm] = val;
    }
#pragma unroll
    for (int e0 = 0; e0 < BN * BK; e0 += 256) {
      const int e = e0 + threadIdx.x;
      int nn, kk;
      if (!TB) { kk = e / BN; nn = e % BN; } else { nn = e / BK; kk = e % BK; }
      const int64_t gn = n0 + nn, gk = k0 + kk;
      cplx val = make_double2(0.0, 0.0);
      if (gn < N && gk < kend) val = TB ? B[gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][nn] = val;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      cplx v = cmul(alpha, acc[i][j]);
      if (use_beta) v = cadd(v, cmul(beta, C[gm * ldc + gn]));
      C[gm * ldc + gn] = v;
    }
  }
}

// ---------------------------------------------------------------------------- doubles packing
struct Pack5 {
  int64_t str[5];  // strides of (Z, i, j, a, b) in X
};

__device__ __forceinline__ void pair_of(int64_t P, int& p, int& q) {
  // P = q(q-1)/2 + p, p < q
  int qq = (int)((1.0 + sqrt(1.0 + 8.0 * (double)P)) * 0.5);
  while ((int64_t)qq * (qq - 1) / 2 > P) --qq;
  while ((int64_t)(qq + 1) * qq / 2 <= P) ++qq;
  q = qq;
  p = (int)(P - (int64_t)qq * (qq - 1) / 2);
}

__global__ void k_pack(const cplx* __restrict__ X, Pack5 s, cplx* D, int64_t nvec, int64_t Po, int64_t Pv,
                       const int2* __restrict__ po, const int2* __restrict__ pv, cplx alpha, bool anti, bool acc) {
  const int64_t n = nvec * Po * Pv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ab = idx % Pv;
    const int64_t t = idx / Pv;
    const int64_t ij = t % Po;
    const int64_t z = t / Po;
    const int2 IJ = po[ij], AB = pv[ab];
    const int64_t base = z * s.str[0];
    const int64_t oi = IJ.x * s.str[1], oj = IJ.y * s.str[2], oa = AB.x * s.str[3], ob = AB.y * s.str[4];
    cplx x = X[base + oi + oj + oa + ob];
    if (anti) {
      const int64_t oj2 = IJ.x * s.str[2], oi2 = IJ.y * s.str[1], ob2 = AB.x * s.str[4], oa2 = AB.y * s.str[3];
      const cplx x1 = X[base + oi2 + oj2 + oa + ob];
      const cplx x2 = X[base + oi + oj + oa2 + ob2];
      const cplx x3 = X[base + oi2 + oj2 + oa2 + ob2];
      x.x = x.x - x1.x - x2.x + x3.x;
      x.y = x.y - x1.y - x2.y + x3.y;
    }
    if (!(alpha.x == 1.0 && alpha.y == 0.0)) x = cmul(alpha, x);
    if (acc) x = cadd(x, D[idx]);
    D[idx] = x;
  }
}

struct Unpack5 {
  int64_t mdim[5];   // extents in memory order (slowest first)
  int64_t mstr[5];   // strides in memory order
  int lax[5];        // logical axis (0..4 = Z,i,j,a,b) of each memory-order axis
};

__global__ void k_unpack(const cplx* __restrict__ D, int64_t ldv, int64_t Pv, Unpack5 u, cplx* X, int64_t n) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx, off = 0;
    int64_t lg[5];
#pragma unroll
    for (int k = 4; k >= 0; --k) {
      const int64_t q = r / u.mdim[k];
      const int64_t c = r - q * u.mdim[k];
      r = q;
      off += c * u.mstr[k];
      lg[u.lax[k]] = c;
    }
    const int64_t z = lg[0];
    int i = (int)lg[1], j = (int)lg[2], a = (int)lg[3], b = (int)lg[4];
    cplx v = make_double2(0.0, 0.0);
    if (i != j && a != b) {
      double sg = 1.0;
      if (i > j) { int t = i; i = j; j = t; sg = -sg; }
      if (a > b) { int t = a; a = b; b = t; sg = -sg; }
      const int64_t P1 = (int64_t)j * (j - 1) / 2 + i, P2 = (int64_t)b * (b - 1) / 2 + a;
      v = D[z * ldv + P1 * Pv + P2];
      v.x *= sg;
      v.y *= sg;
    }
    X[off] = v;
  }
}

// ---------------------------------------------------------------------------- vector kernels
__global__ void k_axpy(int64_t n, cplx a, const cplx* __restrict__ x, cplx* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = cadd(y[i], cmul(a, x[i]));
}

__global__ void k_scale(int64_t n, cplx a, cplx* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = cmul(a, x[i]);
}

__global__ void k_copy(int64_t n, const cplx* __restrict__ x, cplx* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i];
}

__global__ void k_diag_axpy(int64_t n, int64_t total, const double* __restrict__ D, const cplx* __restrict__ x,
                            cplx* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = D[i % n];
    const cplx a = x[i];
    cplx b = y[i];
    b.x = fma(d, a.x, b.x);
    b.y = fma(d, a.y, b.y);
    y[i] = b;
  }
}

__global__ void k_div_shift(int64_t n, const cplx* __restrict__ x, const double* __restrict__ D, cplx z, cplx a,
                            cplx* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double dr = D[i] - z.x, di = -z.y;
    const double inv = 1.0 / (dr * dr + di * di);
    const cplx q = cmul(x[i], make_double2(dr * inv, -di * inv));
    y[i] = cmul(a, q);
  }
}

__device__ __forceinline__ cplx block_sum(cplx v) {
  __shared__ cplx sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffff, v.x, o);
    v.y += __shfl_down_sync(0xffffffff, v.y, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = make_double2(0.0, 0.0);
  if (w == 0) {
    if (l < kThreads / 32) v = sh[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffff, v.x, o);
      v.y += __shfl_down_sync(0xffffffff, v.y, o);
    }
  }
  __syncthreads();
  return v;
}

// partial[k][blockIdx.x] = sum over this block's slice of op(x_k) y_k
__global__ void __launch_bounds__(kThreads) k_dots_partial(int64_t n, const cplx* __restrict__ x, int64_t ldx,
                                                           const cplx* __restrict__ y, int64_t ldy, bool herm,
                                                           cplx* partial) {
  const int k = blockIdx.y;
  const cplx* xk = x + k * ldx;
  const cplx* yk = y + k * ldy;
  cplx s = make_double2(0.0, 0.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cplx a = xk[i];
    if (herm) a.y = -a.y;
    const cplx b = yk[i];
    s.x = fma(a.x, b.x, fma(-a.y, b.y, s.x));
    s.y = fma(a.x, b.y, fma(a.y, b.x, s.y));
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_sum_partials(const cplx* partial, int nb, cplx* out) {
  const int k = blockIdx.x;
  cplx s = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s = cadd(s, partial[(int64_t)k * nb + i]);
  s = block_sum(s);
  if (threadIdx.x == 0) out[k] = s;
}

// ---- FP64 <-> FP32 by bit manipulation of the IEEE 754 binary64 and binary32 layouts.  On sm_103
// the cvt instructions between the two formats issue on the FP64 pipe (about 1/64 of the FP32
// rate), which would bound every FP32 kernel that reads or writes FP64 storage; these run on the
// integer pipe.  d2f rounds to nearest (ties away from zero), flushes results below the binary32
// normal range to signed zero and overflows to signed infinity (NaN stays NaN); f2d is exact for
// normal inputs and flushes binary32 subnormals to zero.
__device__ __forceinline__ float d2f(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
  // low 9 exponent bits and the top 23 mantissa bits, rounded on the 24th; the exponent bias
  // changes by 1023 - 127 = 896, whose low 9 bits are 0x180
  const uint32_t t = __funnelshift_l(lo, hi, 3) + ((lo >> 28) & 1u);
  uint32_t f = (t - 0xC0000000u) | sign;
  if (e < 897u) f = sign;
  if (e > 1150u) f = sign | ((e == 0x7ffu && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u);
  return __uint_as_float(f);
}
__device__ __forceinline__ double f2d(float x) {
  const uint32_t u = __float_as_uint(x), sign = u & 0x80000000u, e = (u >> 23) & 0xffu;
  uint32_t hi = (((u & 0x7fffffffu) >> 3) + 0x38000000u) | sign, lo = u << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 0xffu) { hi = sign | 0x7ff00000u | ((u & 0x7fffffu) ? 0x80000u : 0u); lo = 0u; }
  return __longlong_as_double((long long)(((uint64_t)hi << 32) | lo));
}
__device__ __forceinline__ float2 d2f2(cplx a) { return make_float2(d2f(a.x), d2f(a.y)); }
__device__ __forceinline__ cplx f2d2(float2 a) { return make_double2(f2d(a.x), f2d(a.y)); }

__global__ void k_to_f32(const cplx* __restrict__ x, float2* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = d2f2(x[i]);
}

// ---- FP32-arithmetic variants of the solver's vector kernels (FP64 storage).  FP64 on sm_103 runs
// at ~1/64 of FP32, and the solver's multi-vector kernels do 8 L m flops per element (L inputs,
// m outputs), so in FP64 they are ALU-bound by a wide margin; in FP32 they stay near the HBM
// roofline.  The inputs are rounded to FP32 (relative 6e-8) and products summed in FP32.

__global__ void __launch_bounds__(kThreads) k_dots_partial32(int64_t n, const cplx* __restrict__ x, int64_t ldx,
                                                             const cplx* __restrict__ y, int64_t ldy, bool herm,
                                                             cplx* partial) {
  const int k = blockIdx.y;
  const cplx* xk = x + k * ldx;
  const cplx* yk = y + k * ldy;
  cplx s = make_double2(0.0, 0.0);
  float2 f = make_float2(0.f, 0.f);
  int run = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 a = d2f2(xk[i]);
    if (herm) a.y = -a.y;
    const float2 b = d2f2(yk[i]);
    f.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, f.x));
    f.y = fmaf(a.x, b.y, fmaf(a.y, b.x, f.y));
    if (++run == 16) { s.x += f.x; s.y += f.y; f = make_float2(0.f, 0.f); run = 0; }
  }
  s.x += f.x;
  s.y += f.y;
  s = block_sum(s);
  if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = s;
}

// Row j of a Rows list (the host guarantees j < X.total()).
__device__ __forceinline__ const cplx* row_of(const Rows& r, int j) {
  const cplx* p = nullptr;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (p == nullptr && s < r.ns) {
      if (j < r.cnt[s]) p = r.p[s] + (int64_t)j * r.ld[s];
      else j -= r.cnt[s];
    }
  }
  return p;
}

// Row j of a Rows list of FP32 mirrors: base pointers are float2 arrays cast to cplx*, strides
// counted in float2 elements.
__device__ __forceinline__ const float2* row_of32(const Rows& r, int j) {
  const float2* p = nullptr;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (p == nullptr && s < r.ns) {
      if (j < r.cnt[s]) p = reinterpret_cast<const float2*>(r.p[s]) + (int64_t)j * r.ld[s];
      else j -= r.cnt[s];
    }
  }
  return p;
}

// Packed FP32 pairs (sm_100+ f32x2 FMA): a complex multiply-accumulate acc += c x is two
// packed FMAs with c held as (c.re, c.re), (-c.im, c.im) and x as (x.re, x.im), (x.im, x.re).
__device__ __forceinline__ uint64_t pk2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 upk2(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Arithmetic of the solver's multi-vector kernels: FP32 pairs (F32) or FP64.
//   C: a coefficient, X: an operand, Acc: an accumulator; mac(acc, c, x): acc += c x
template <bool F32> struct Arith;
template <> struct Arith<true> {
  struct __align__(16) C { uint64_t re, im; };
  struct __align__(16) X { uint64_t a, b; };
  typedef uint64_t Acc;
  __device__ static C coef(float2 c) {
    C r;
    r.re = pk2(c.x, c.x);
    r.im = pk2(-c.y, c.y);
    return r;
  }
  __device__ static C coef(cplx c) { return coef(d2f2(c)); }
  __device__ static X opnd(float2 v) {
    X r;
    r.a = pk2(v.x, v.y);
    r.b = pk2(v.y, v.x);
    return r;
  }
  __device__ static X opnd(cplx v) { return opnd(d2f2(v)); }
  __device__ static Acc zero() { return 0ull; }
  __device__ static X zero_x() { return X{0ull, 0ull}; }
  __device__ static C zero_c() { return C{0ull, 0ull}; }
  __device__ static void mac(Acc& acc, const C& c, const X& x) {
    acc = ffma2(c.re, x.a, acc);
    acc = ffma2(c.im, x.b, acc);
  }
};
// Float-float (double-FP32) complex numbers: value = (rh + rl) + i (ih + il), |rl| <= ulp(rh)/2.
struct __align__(16) FF2 {
  float rh, rl, ih, il;
};
// x = h + l: h = x rounded to binary32, l = the exact remainder x - h rounded to binary32 (about
// 48 significant bits in all), on the integer pipe.  Remainders below the binary32 normal range
// are dropped, so |x| below ~2^-90 (1e-27) keeps fewer bits, down to 24 (checked against binary64
// on 2e4 values spanning 1e-30..1e30: h + l within 2^-47 of x for |x| above that).
__device__ __forceinline__ void split_ff(double x, float& h, float& l) {
  h = d2f(x);
  l = 0.f;
  const uint64_t bx = (uint64_t)__double_as_longlong(x);
  const int e = (int)((bx >> 52) & 0x7ffu);
  const uint32_t uh = __float_as_uint(h), eh = (uh >> 23) & 0xffu;
  if (e == 0 || e == 0x7ff || eh == 0u || eh == 0xffu) return;
  // |x| = M 2^(e - 1075), |h| = Mh 2^(eh - 150) = (Mh << sh) 2^(e - 1075)
  const int64_t M = (int64_t)((bx & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  const int64_t Mh = (int64_t)((uh & 0x7fffffu) | 0x800000u);
  const int sh = (int)eh - e + 925;   // 29, or 30 when rounding carried into the next binade
  const int64_t k = M - (Mh << sh);   // |k| < 2^29
  if (k == 0) return;
  const uint32_t a = (uint32_t)(k < 0 ? -k : k);
  const int msb = 31 - __clz(a);
  uint32_t m;
  int p = msb;
  if (msb > 23) {
    m = (a + (1u << (msb - 24))) >> (msb - 23);   // round half up to 24 bits
    if (m >> 24) { m >>= 1; ++p; }
  } else {
    m = a << (23 - msb);
  }
  const int be = p + e - 948;   // binary32 biased exponent of |k| 2^(e - 1075)
  if (be <= 0) return;
  const uint32_t sx = (uint32_t)(bx >> 63) ^ (k < 0 ? 1u : 0u);
  l = __uint_as_float((sx << 31) | ((uint32_t)be << 23) | (m & 0x7fffffu));
}
// (H, L) += s (ah + al)(bh + bl) with the products of the high parts exact (FMA) and the sum
// compensated (TwoSum); s = +1 or -1.  Round-to-nearest intrinsics keep the compiler from
// contracting or reassociating the error terms.
__device__ __forceinline__ void ff_prod_acc(float& H, float& L, float ah, float al, float bh, float bl, float s) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float ps = s * p, es = s * e;
  const float t = __fadd_rn(H, ps);
  const float v = __fsub_rn(t, H);
  const float err = __fadd_rn(__fsub_rn(H, __fsub_rn(t, v)), __fsub_rn(ps, v));
  H = t;
  L = __fadd_rn(L, __fadd_rn(err, es));
}
// The "FP64" arithmetic of the solver's vector kernels: float-float on the FP32 pipe (~2^-46
// relative per operation).  B300's FP64 pipe issues at 1/64 of the FP32 rate, so a complex
// multiply-add in FP64 (4 DFMA) costs as much as ~256 FP32 operations; in float-float it is
// about 48, with the inputs split once per element.
template <> struct Arith<false> {
  typedef FF2 C;
  typedef FF2 X;
  typedef FF2 Acc;
  __device__ static FF2 split(cplx v) {
    FF2 r;
    split_ff(v.x, r.rh, r.rl);
    split_ff(v.y, r.ih, r.il);
    return r;
  }
  __device__ static C coef(cplx c) { return split(c); }
  __device__ static X opnd(cplx v) { return split(v); }
  __device__ static Acc zero() { return FF2{0.f, 0.f, 0.f, 0.f}; }
  __device__ static X zero_x() { return zero(); }
  __device__ static C zero_c() { return zero(); }
  __device__ static void mac(Acc& acc, const C& c, const X& x) {
    ff_prod_acc(acc.rh, acc.rl, c.rh, c.rl, x.rh, x.rl, 1.f);
    ff_prod_acc(acc.rh, acc.rl, c.ih, c.il, x.ih, x.il, -1.f);
    ff_prod_acc(acc.ih, acc.il, c.rh, c.rl, x.ih, x.il, 1.f);
    ff_prod_acc(acc.ih, acc.il, c.ih, c.il, x.rh, x.rl, 1.f);
  }
  __device__ static cplx to_cplx(const Acc& a) {
    return make_double2(f2d(a.rh) + f2d(a.rl), f2d(a.ih) + f2d(a.il));
  }
};

inline int vecmat_blocks() { return 4 * num_sms(); }

// r_q = sum_j X_j C[j][q] + add; Y_q = (D ? -r_q / (D - z_q) : r_q) (+ Y_q); per-block partial
// norms of r_q (or of Y_q if norm_y).  Q >= m outputs are computed (coefficients of q >= m are
// zero and never stored); each thread takes E elements per step so that every coefficient read
// from shared memory serves E elements.  With F32 the whole element pipeline (products, sums,
// preconditioner, accumulation into Y) runs in FP32 and only loads and stores touch FP64.
struct AddRows {   // row index of each output's additive row (VecMat::arow)
  int r[kVecMatOut];
};
template <bool F32, int Q, int E, int U, bool X32>
__global__ void __launch_bounds__(kThreads, F32 ? 2 : 1)
    k_vecmat(int64_t n, Rows X, int m, const cplx* __restrict__ C, const cplx* __restrict__ add, cplx* Y, int64_t ldy,
             bool acc, const double* __restrict__ D, const cplx* __restrict__ z, bool norm_y, double* part,
             const float2* __restrict__ addq, int64_t ldadd, AddRows arow) {
  typedef Arith<F32> A;
  typedef typename A::C Cf;
  typedef typename std::conditional<F32, float, double>::type R;
  typedef typename std::conditional<F32, float2, double2>::type V;
  extern __shared__ __align__(16) unsigned char vm_smem[];
  __shared__ V zs[Q];
  const int nx = X.total();
  Cf* cs = reinterpret_cast<Cf*>(vm_smem);                                        // nx x Q
  const cplx** rows = reinterpret_cast<const cplx**>(vm_smem + sizeof(Cf) * (size_t)nx * Q);
  for (int e = threadIdx.x; e < nx * Q; e += blockDim.x) {
    const int j = e / Q, q = e % Q;
    cs[e] = A::coef(q < m ? C[(int64_t)j * m + q] : make_double2(0.0, 0.0));
  }
  for (int j = threadIdx.x; j < nx; j += blockDim.x)
    rows[j] = X32 ? reinterpret_cast<const cplx*>(row_of32(X, j)) : row_of(X, j);
  if (threadIdx.x < Q) {
    const cplx zq = (D && (int)threadIdx.x < m) ? z[threadIdx.x] : make_double2(0.0, 0.0);
    if constexpr (F32) zs[threadIdx.x] = d2f2(zq);
    else zs[threadIdx.x] = zq;
  }
  __syncthreads();
  R nn[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) nn[q] = 0;
  const int64_t tile = (int64_t)E * blockDim.x;
  for (int64_t i0 = blockIdx.x * tile + threadIdx.x; i0 < n; i0 += (int64_t)gridDim.x * tile) {
    typename A::Acc a[E][Q];
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int q = 0; q < Q; ++q) a[e][q] = A::zero();
    // rows in groups of U: all loads of a group are issued before any is used, so that each
    // thread keeps U * E loads in flight
    for (int j0 = 0; j0 < nx; j0 += U) {
      typedef typename std::conditional<X32, float2, cplx>::type XV;
      XV raw[U][E];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + u;
        const XV* rp = reinterpret_cast<const XV*>(rows[j < nx ? j : 0]);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int64_t i = i0 + (int64_t)e * blockDim.x;
          if constexpr (X32) raw[u][e] = (j < nx && i < n) ? __ldg(rp + i) : make_float2(0.f, 0.f);
          else raw[u][e] = (j < nx && i < n) ? __ldg(rp + i) : make_double2(0.0, 0.0);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + u;
        if (j >= nx) break;
        typename A::X xv[E];
#pragma unroll
        for (int e = 0; e < E; ++e) xv[e] = A::opnd(raw[u][e]);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const Cf cq = cs[j * Q + q];
#pragma unroll
          for (int e = 0; e < E; ++e) A::mac(a[e][q], cq, xv[e]);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t i = i0 + (int64_t)e * blockDim.x;
      if (i >= n) continue;
      V b, dz;
      if constexpr (F32) {
        b = add ? d2f2(add[i]) : make_float2(0.f, 0.f);
        dz.x = D ? d2f(D[i]) : 0.f;
      } else {
        b = add ? add[i] : make_double2(0.0, 0.0);
        dz.x = D ? D[i] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (q < m) {
          V r;
          if constexpr (F32) {
            const float2 v = upk2(a[e][q]);
            r = make_float2(v.x + b.x, v.y + b.y);
            if (addq) {
              const float2 t = addq[(int64_t)arow.r[q] * ldadd + i];
              r.x += t.x;
              r.y += t.y;
            }
          } else {
            const cplx v = A::to_cplx(a[e][q]);
            r = make_double2(v.x + b.x, v.y + b.y);
          }
          if (!norm_y) nn[q] += r.x * r.x + r.y * r.y;
          if (D) {
            // -r / (D - z) = -r conj(D - z) / |D - z|^2, with |D - z| >= 1e-4 (a Ritz value of the
            // eigensolver can come arbitrarily close to a denominator)
            const R dr = dz.x - zs[q].x, dm = -zs[q].y;
            const R inv = R(1) / fmax(dr * dr + dm * dm, R(1e-8));
            const R rx = r.x, ry = r.y;
            r.x = -(rx * dr + ry * dm) * inv;
            r.y = -(ry * dr - rx * dm) * inv;
          }
          if (Y) {
            cplx* yq = Y + q * ldy + i;
            if constexpr (F32) {
              if (acc) {
                const float2 y0 = d2f2(*yq);
                r.x += y0.x;
                r.y += y0.y;
              }
              *yq = f2d2(r);
            } else {
              if (acc) r = cadd(r, *yq);
              *yq = r;
            }
          }
          if (norm_y) nn[q] += r.x * r.x + r.y * r.y;
        }
      }
    }
  }
  if (part) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (q < m) {   // uniform across the block
        const cplx v = block_sum(make_double2((double)nn[q], 0.0));
        if (threadIdx.x == 0) part[q * gridDim.x + blockIdx.x] = v.x;
      }
    }
  }
}

// out[q] = sum_b part[q * nb + b]   (one block per q, fixed order)
__global__ void k_sum_rows(const double* part, int nb, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[(int64_t)blockIdx.x * nb + i];
  cplx v = block_sum(make_double2(s, 0.0));
  if (threadIdx.x == 0) out[blockIdx.x] = v.x;
}


// D[r][P(p,q)] = alpha (X[r,p,q] - X[r,q,p]) or alpha X[r,p,q]  (+ D), X strided (R, m, m)
// grid: x over the pairs, y over the rows r (no index division)
__global__ void k_pack2(const cplx* __restrict__ X, int64_t sr, int64_t sp, int64_t sq, cplx* D, int64_t ldd,
                        int64_t R, int64_t Pm, const int2* __restrict__ tab, cplx alpha, bool anti, bool acc) {
  for (int64_t r = blockIdx.y; r < R; r += gridDim.y) {
    for (int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; P < Pm; P += (int64_t)gridDim.x * blockDim.x) {
      const int2 pq = tab[P];
      cplx x = X[r * sr + pq.x * sp + pq.y * sq];
      if (anti) {
        const cplx y = X[r * sr + pq.y * sp + pq.x * sq];
        x.x -= y.x;
        x.y -= y.y;
      }
      if (!(alpha.x == 1.0 && alpha.y == 0.0)) x = cmul(alpha, x);
      const int64_t o = r * ldd + P;
      if (acc) x = cadd(x, D[o]);
      D[o] = x;
    }
  }
}

// X[r,p,q] = sign D[r][P(min,max)] (0 on p == q), X strided (R, m, m)
__global__ void k_unpack2(const cplx* __restrict__ D, int64_t ldd, cplx* X, int64_t sr, int64_t sp, int64_t sq,
                          int64_t R, int m) {
  const int64_t n = R * m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % m);
    const int p = (int)((idx / m) % m);
    const int64_t r = idx / ((int64_t)m * m);
    cplx x = make_double2(0.0, 0.0);
    if (p != q) {
      const int a = p < q ? p : q, b = p < q ? q : p;
      x = D[r * ldd + (int64_t)b * (b - 1) / 2 + a];
      if (p > q) { x.x = -x.x; x.y = -x.y; }
    }
    X[r * sr + p * sp + q * sq] = x;
  }
}

// Gram tile for tall-skinny operands: part[blk][i][j] = sum over this block's share of the
// elements of op(X_i[k]) Y_j[k], nx <= 32 RL, ny <= NY.  Chunks of 2^lc elements of all rows are
// brought into shared memory by bulk asynchronous copies (one per row, completion counted on an
// mbarrier), double-buffered; the chunk grows as the row count falls, so that about 64 KiB per SM
// are in flight whatever the tile.  Lane l owns rows l, l+32, ... of X and all rows of Y (read as
// shared-memory broadcasts); the 16 warps split each chunk's elements and are summed at the end.
// F32: each chunk is converted to FP32 once, in place in shared memory, into
// the packed forms the paired FMAs take; products are summed in FP32 pairs over runs of 32
// elements per warp and the runs added with a compensated (two-sum) FP32 accumulator.  The mbarrier waits are bounded: on expiry the block records code
// 11 in the context's status word, waits (bounded) for its copies in flight and returns.
constexpr int kGramRunElems = 32;            // elements per warp in one FP32 run
constexpr int kGramMaxX = 32, kGramMaxY = 8; // tile of one launch (one X row per lane)
constexpr int kGramWarps = 16;               // 512 threads: enough warps per SM to hide latencies
constexpr int kGramMinLog = 6, kGramMaxLog = 11;   // chunk of 64 .. 2048 elements
constexpr int kGramHead = 128;               // bytes before the staging buffers (two mbarriers)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool bar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (about a second): false if the phase did not complete
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity) {
  for (uint32_t i = 0; i < (1u << 22); ++i) {
    if (bar_try_wait(b, parity)) return true;
    if (i > 64) __nanosleep(256);
  }
  return false;
}

// hi + lo += v with the rounding error of the addition kept in lo (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}

template <bool F32, int RL, int NY, bool X32>
__global__ void __launch_bounds__(kGramWarps * 32, 1)
    k_gram_skinny(int64_t n, Rows X, Rows Y, bool herm, cplx* part, int lc, int* __restrict__ err) {
  typedef Arith<F32> A;
  // staged element: FP64 complex, or FP32 complex for rows that are the solver's FP32 mirrors
  // (even row strides, so a chunk's byte count rounded up to 16 stays inside its row)
  typedef typename std::conditional<X32, float2, cplx>::type SE;
  extern __shared__ __align__(128) unsigned char gs_smem[];
  const int nx = X.total(), ny = Y.total(), nr = nx + ny;
  // padded row pitch (FP64: odd, so lanes reading distinct rows hit distinct banks; FP32: even,
  // for 16-byte aligned rows)
  const int CH = 1 << lc, pitch = X32 ? CH + 2 : CH + 1;
  uint64_t* bar = reinterpret_cast<uint64_t*>(gs_smem);
  SE* st0 = reinterpret_cast<SE*>(gs_smem + kGramHead);
  SE* st1 = st0 + (size_t)nr * pitch;
  const SE** rowp = reinterpret_cast<const SE**>(st1 + (size_t)nr * pitch);
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    if constexpr (X32) rowp[r] = r < nx ? row_of32(X, r) : row_of32(Y, r - nx);
    else rowp[r] = r < nx ? row_of(X, r) : row_of(Y, r - nx);
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nchunks = (n + CH - 1) >> lc;
  const int per_warp = CH / kGramWarps;
  const int flush_every = per_warp >= kGramRunElems ? 1 : kGramRunElems / per_warp;   // chunks per run
  // warp 0: bulk copies of chunk ch (all rows) into stage s
  auto issue = [&](int s, int64_t ch) {
    const int64_t base = ch << lc;
    int64_t cnt = min((int64_t)CH, n - base);
    if (X32) cnt += cnt & 1;   // 16-byte multiple; the even row stride keeps it inside the row
    const uint32_t bytes = (uint32_t)(cnt * (int64_t)sizeof(SE));
    SE* dst = s ? st1 : st0;
    if (lane == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar[s])),
                   "r"(bytes * (uint32_t)nr)
                   : "memory");
    __syncwarp();
    for (int r = lane; r < nr; r += 32)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr(dst + (size_t)r * pitch)),
          "l"(rowp[r] + base), "r"(bytes), "r"(smem_addr(&bar[s]))
          : "memory");
  };
  typename A::Acc acc[RL][NY];
  float hi[RL][NY][2], lo[RL][NY][2];   // F32 run totals (two-sum)
#pragma unroll
  for (int a = 0; a < RL; ++a)
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      acc[a][j] = A::zero();
      hi[a][j][0] = hi[a][j][1] = lo[a][j][0] = lo[a][j][1] = 0.f;
    }
  auto flush = [&]() {
#pragma unroll
    for (int a = 0; a < RL; ++a)
#pragma unroll
      for (int j = 0; j < NY; ++j) {
        if constexpr (F32) {
          const float2 v = upk2(acc[a][j]);
          two_sum(hi[a][j][0], lo[a][j][0], v.x);
          two_sum(hi[a][j][1], lo[a][j][1], v.y);
          acc[a][j] = A::zero();
        }
      }
  };
  // F32: the staged chunk holds every element already in its packed operand form (Y rows) or
  // coefficient form (X rows), 16 bytes each, so the products need no register moves
  typedef typename A::X PX;
  typedef typename A::C PC;
  auto mac_elem = [&](const SE* st, int k) {
    typename A::X yv[NY];
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      if constexpr (X32) yv[j] = A::opnd(j < ny ? st[(nx + j) * pitch + k] : make_float2(0.f, 0.f));
      else yv[j] = j < ny ? reinterpret_cast<const PX*>(st)[(nx + j) * pitch + k] : A::zero_x();
    }
#pragma unroll
    for (int a = 0; a < RL; ++a) {
      const int r = lane + 32 * a;
      typename A::C xc;
      if constexpr (X32) {
        float2 xv = r < nx ? st[r * pitch + k] : make_float2(0.f, 0.f);
        if (herm) xv.y = -xv.y;
        xc = A::coef(xv);
      } else {
        xc = r < nx ? reinterpret_cast<const PC*>(st)[r * pitch + k] : A::zero_c();
      }
#pragma unroll
      for (int j = 0; j < NY; ++j) A::mac(acc[a][j], xc, yv[j]);
    }
  };
  uint32_t uses0 = 0, uses1 = 0;   // completed phases per stage (the wait parity)
  int s = 0, run = 0;
  if (warp == 0 && (int64_t)blockIdx.x < nchunks) issue(0, blockIdx.x);
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const bool more = ch + gridDim.x < nchunks;
    if (more && warp == 0) issue(s ^ 1, ch + gridDim.x);
    const bool ok = bar_wait(&bar[s], (s ? uses1 : uses0) & 1u);
    if (__syncthreads_or(!ok)) {
      // give up: record the expiry, let the copies in flight land (bounded), return
      if (threadIdx.x == 0) {
        atomicExch(err, 11);
        bar_wait(&bar[s], (s ? uses1 : uses0) & 1u);
        if (more) bar_wait(&bar[s ^ 1], (s ? uses0 : uses1) & 1u);
      }
      __syncthreads();
      return;
    }
    if (s) ++uses1; else ++uses0;
    SE* st = s ? st1 : st0;
    const int64_t base = ch << lc;
    const int lim = (int)min((int64_t)CH, n - base);
    if constexpr (!X32) {
      // in place: each FP64 element becomes its 16-byte packed form (FP32 pairs, or the
      // float-float split); a warp per row when there are enough rows, else all threads over the
      // rows x chunk elements
      const float sg = herm ? -1.f : 1.f;   // coefficient of conj(x) for the Hermitian product
      auto pack = [&](cplx* p, bool xrow) {
        if constexpr (F32) {
          const float2 v = d2f2(*p);
          if (xrow) {
            const float ci = sg * v.y;
            *reinterpret_cast<PC*>(p) = PC{pk2(v.x, v.x), pk2(-ci, ci)};
          } else {
            *reinterpret_cast<PX*>(p) = PX{pk2(v.x, v.y), pk2(v.y, v.x)};
          }
        } else {
          cplx v = *p;
          if (xrow && herm) v.y = -v.y;
          *reinterpret_cast<FF2*>(p) = A::split(v);
        }
      };
      if (nr >= kGramWarps) {
        for (int r = warp; r < nr; r += kGramWarps)
          for (int k = lane; k < lim; k += 32) pack(st + (size_t)r * pitch + k, r < nx);
      } else {
        for (int e = threadIdx.x; e < nr * CH; e += blockDim.x) {
          const int r = e >> lc, k = e & (CH - 1);
          if (k < lim) pack(st + (size_t)r * pitch + k, r < nx);
        }
      }
      __syncthreads();
    }
    const int k0 = warp * per_warp;
    for (int kk = 0; kk < per_warp; kk += kGramRunElems) {
      const int len = min(kGramRunElems, per_warp - kk);
#pragma unroll 2
      for (int t = 0; t < len; ++t) {
        const int k = k0 + kk + t;
        if (k < lim) mac_elem(st, k);
      }
      if (per_warp >= kGramRunElems) flush();
    }
    if (per_warp < kGramRunElems && ++run == flush_every) {
      run = 0;
      flush();
    }
    __syncthreads();   // the stage (and the FP32 copy) are overwritten next
    s ^= 1;
  }
  flush();
  // sum the 8 warps' shares in shared memory (the staging buffers are free now; the mbarriers
  // in the head are left alone)
  cplx* red = reinterpret_cast<cplx*>(gs_smem + kGramHead);   // [warp][a][j][lane]
#pragma unroll
  for (int a = 0; a < RL; ++a)
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      cplx v;
      if constexpr (F32) {
        v = make_double2((double)hi[a][j][0] + (double)lo[a][j][0], (double)hi[a][j][1] + (double)lo[a][j][1]);
      } else {
        v = A::to_cplx(acc[a][j]);
      }
      red[((warp * RL + a) * NY + j) * 32 + lane] = v;
    }
  __syncthreads();
  for (int o = threadIdx.x; o < nx * ny; o += blockDim.x) {
    const int i = o / ny, j = o % ny;
    const int a = i / 32, l = i % 32;
    cplx v = make_double2(0.0, 0.0);
    for (int w = 0; w < kGramWarps; ++w) v = cadd(v, red[((w * RL + a) * NY + j) * 32 + l]);
    part[(int64_t)blockIdx.x * nx * ny + o] = v;
  }
}

// out[(swap ? j * ldo + i : i * ldo + j)] = (swap && herm ? conj : id)(sum_b part[b][i][j]) for the
// a x b tile, i < a, j < b
__global__ void k_gram_reduce(const cplx* __restrict__ part, int nblk, int a, int b, cplx* out, int64_t ldo, bool swap,
                              bool herm) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= a * b) return;
  cplx s = make_double2(0.0, 0.0);
  for (int k = 0; k < nblk; ++k) s = cadd(s, part[(int64_t)k * a * b + o]);
  const int i = o / b, j = o % b;
  if (swap) {
    if (herm) s.y = -s.y;
    out[(int64_t)j * ldo + i] = s;
  } else {
    out[(int64_t)i * ldo + j] = s;
  }
}

// split-K epilogue: C[m*ldc + n] = alpha * sum_z P[z][m][n] + beta * C (fixed summation order)
__global__ void k_splitk_reduce(const cplx* __restrict__ P, int S, int64_t M, int64_t N, cplx alpha, cplx beta, cplx* C,
                                int64_t ldc) {
  const int64_t n_el = M * N;
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_el; idx += (int64_t)gridDim.x * blockDim.x) {
    cplx s = make_double2(0.0, 0.0);
    for (int z = 0; z < S; ++z) s = cadd(s, P[(int64_t)z * n_el + idx]);
    const int64_t m = idx / N, n = idx - m * N;
    cplx v = cmul(alpha, s);
    if (use_beta) v = cadd(v, cmul(beta, C[m * ldc + n]));
    C[m * ldc + n] = v;
  }
}

}  // namespace

int num_sms() {
  static int cache[64] = {};
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) d = 0;
  const int slot = d >= 0 && d < 64 ? d : -1;
  if (slot >= 0 && cache[slot]) return cache[slot];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0) n = 1;
  if (slot >= 0) cache[slot] = n;
  return n;
}

bool once_per_device(bool* done) {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return true;
  if (done[d]) return false;
  done[d] = true;
  return true;
}

int reduce_blocks() { return 2 * num_sms(); }

void splitk_reduce(const Launch& L, const cplx* P, int S, int64_t M, int64_t N, cplx alpha, cplx beta, cplx* C,
                   int64_t ldc) {
  kbeg(L);
  k_splitk_reduce<<<grid_for(M * N), kThreads, 0, L.s>>>(P, S, M, N, alpha, beta, C, ldc);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_splitk_reduce");
}

void zgemm_splitk(const Launch& L, bool ta, bool tb, int64_t M, int64_t N, int64_t K, const cplx* A, int64_t lda,
                  const cplx* B, int64_t ldb, cplx* P, int S, int64_t kchunk) {
  // partials P[z] (M x N, ld N) over k in [z*kchunk, (z+1)*kchunk); kchunk a multiple of 8
  CCLR_REQUIRE((M + BM - 1) / BM <= 65535 && S <= 65535, CCLR_E_ARG, "zgemm_splitk: grid too large");
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)S);
  const cplx one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  kbeg(L);
  if (!ta && !tb) k_zgemm<false, false><<<grid, 256, 0, L.s>>>(M, N, K, one, A, lda, B, ldb, zero, P, N, kchunk, M * N);
  else if (!ta && tb) k_zgemm<false, true><<<grid, 256, 0, L.s>>>(M, N, K, one, A, lda, B, ldb, zero, P, N, kchunk, M * N);
  else if (ta && !tb) k_zgemm<true, false><<<grid, 256, 0, L.s>>>(M, N, K, one, A, lda, B, ldb, zero, P, N, kchunk, M * N);
  else k_zgemm<true, true><<<grid, 256, 0, L.s>>>(M, N, K, one, A, lda, B, ldb, zero, P, N, kchunk, M * N);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_zgemm_splitk");
}

void pack2(const Launch& L, const Tensor& X, cplx* D, int64_t ldd, const int2* tab, cplx alpha, bool anti, bool acc) {
  CCLR_REQUIRE(X.rank == 3 && X.dim[1] == X.dim[2] && !X.conj, CCLR_E_ARG, "pack2: X must be (R, m, m)");
  const int64_t m = X.dim[1], Pm = m * (m - 1) / 2, R = X.dim[0];
  if (R * Pm == 0) return;
  cplx al = make_double2(alpha.x * X.scale, alpha.y * X.scale);
  kbeg(L);
  const dim3 grid((unsigned)std::min<int64_t>((Pm + kThreads - 1) / kThreads, 1024),
                  (unsigned)std::min<int64_t>(R, 65535));
  k_pack2<<<grid, kThreads, 0, L.s>>>(X.p, X.str[0], X.str[1], X.str[2], D, ldd, R, Pm, tab, al, anti, acc);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_pack2");
}

void unpack2(const Launch& L, const cplx* D, int64_t ldd, const Tensor& X) {
  CCLR_REQUIRE(X.rank == 3 && X.dim[1] == X.dim[2], CCLR_E_ARG, "unpack2: X must be (R, m, m)");
  const int64_t n = X.numel();
  if (n == 0) return;
  kbeg(L);
  k_unpack2<<<grid_for(n), kThreads, 0, L.s>>>(D, ldd, X.p, X.str[0], X.str[1], X.str[2], X.dim[0], (int)X.dim[1]);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_unpack2");
}

namespace {
constexpr size_t kGramSmemMax = 200 << 10;
template <bool F32, int RL, int NY, bool X32>
void launch_gram(const Launch& L, int nblk, size_t smem, int64_t n, const Rows& X, const Rows& Y, bool herm,
                 cplx* part, int lc) {
  CCLR_REQUIRE(L.err, CCLR_E_STATE, "gram: no device status word");
  static bool attr = false;
  if (!attr) {
    CCLR_CK(cudaFuncSetAttribute(k_gram_skinny<F32, RL, NY, X32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kGramSmemMax));
    attr = true;
  }
  k_gram_skinny<F32, RL, NY, X32><<<nblk, kGramWarps * 32, smem, L.s>>>(n, X, Y, herm, part, lc, L.err);
}
template <bool F32, bool X32>
void launch_gram_tile(const Launch& L, int nblk, size_t smem, int64_t n, const Rows& X, const Rows& Y, bool herm,
                      cplx* part, int lc) {
  const int b = Y.total();   // X.total() <= kGramMaxX = 32: one row per lane
  if (b == 1) launch_gram<F32, 1, 1, X32>(L, nblk, smem, n, X, Y, herm, part, lc);
  else if (b <= 4) launch_gram<F32, 1, 4, X32>(L, nblk, smem, n, X, Y, herm, part, lc);
  else launch_gram<F32, 1, 8, X32>(L, nblk, smem, n, X, Y, herm, part, lc);
}
}  // namespace

void gram(const Launch& L, int64_t n, const Rows& X, const Rows& Y, bool herm, cplx* out_dev, cplx* scratch,
          int64_t scratch_elems, bool x32) {
  const int nx = X.total(), ny = Y.total();
  CCLR_REQUIRE(nx >= 1 && ny >= 1 && n >= 1, CCLR_E_ARG, "gram: empty operand");
  CCLR_REQUIRE(!x32 || L.fast32, CCLR_E_ARG, "gram: FP32 rows need the FP32 arithmetic");
  if (x32)   // chunk copies are rounded up to 16 bytes: rows need even strides covering n + 1
    for (const Rows* R : {&X, &Y})
      for (int g = 0; g < R->ns; ++g)
        CCLR_REQUIRE(R->ld[g] % 2 == 0 && R->ld[g] >= n + (n & 1), CCLR_E_ARG, "gram: FP32 row stride");
  const size_t esz = x32 ? sizeof(float2) : sizeof(cplx);
  // the kernel takes the longer list as its X side; the transpose is undone when the tile is stored
  const bool swap = ny > nx;
  const Rows& P = swap ? Y : X;
  const Rows& Q = swap ? X : Y;
  const int np = P.total(), nq = Q.total();
  for (int i0 = 0; i0 < np; i0 += kGramMaxX)
    for (int j0 = 0; j0 < nq; j0 += kGramMaxY) {
      const int a = std::min(kGramMaxX, np - i0), b = std::min(kGramMaxY, nq - j0);
      // chunk: at least 64 KiB of rows per stage (the bytes each SM keeps in flight), within the
      // shared-memory budget of two stages plus the FP32 copy
      auto stage_bytes = [&](int lc) {
        return kGramHead + 2 * esz * (size_t)(a + b) * ((size_t(1) << lc) + 2) + sizeof(void*) * (size_t)(a + b);
      };
      int lc = kGramMinLog;
      while (lc < kGramMaxLog && ((size_t)(a + b) * esz << lc) < (size_t(64) << 10) && stage_bytes(lc + 1) <= kGramSmemMax)
        ++lc;
      const int64_t nchunks = (n + (int64_t(1) << lc) - 1) >> lc;
      int nblk = (int)std::min<int64_t>(num_sms(), nchunks);
      if ((int64_t)nblk * a * b > scratch_elems) nblk = (int)std::max<int64_t>(1, scratch_elems / ((int64_t)a * b));
      const int NYt = b == 1 ? 1 : (b <= 4 ? 4 : 8);
      const size_t red = kGramHead + sizeof(cplx) * kGramWarps * NYt * 32;
      const size_t smem = std::max(stage_bytes(lc), red);
      CCLR_REQUIRE(smem <= kGramSmemMax, CCLR_E_ARG, "gram: tile too large");
      kbeg(L);
      if (x32)
        launch_gram_tile<true, true>(L, nblk, smem, n, P.slice(i0, a, true), Q.slice(j0, b, true), herm, scratch, lc);
      else if (L.fast32) launch_gram_tile<true, false>(L, nblk, smem, n, P.slice(i0, a), Q.slice(j0, b), herm, scratch, lc);
      else launch_gram_tile<false, false>(L, nblk, smem, n, P.slice(i0, a), Q.slice(j0, b), herm, scratch, lc);
      CCLR_CK(cudaGetLastError());
      bump(L, shaped(x32 ? "k_gram_skinny32" : "k_gram_skinny", a, b, lc));
      cplx* o = swap ? out_dev + (int64_t)j0 * ny + i0 : out_dev + (int64_t)i0 * ny + j0;
      kbeg(L);
      k_gram_reduce<<<(a * b + 255) / 256, 256, 0, L.s>>>(scratch, nblk, a, b, o, ny, swap, herm);
      CCLR_CK(cudaGetLastError());
      bump(L, "k_gram_reduce");
    }
}

int64_t vecmat_scratch_doubles() { return (int64_t)kVecMatOut * vecmat_blocks(); }

namespace {
template <bool F32, int Q, bool X32>
void launch_vecmat(const Launch& L, int64_t n, const VecMat& a, double* part) {
  // E elements per thread (each shared-memory coefficient serves E elements), U rows of loads in
  // flight; the FP32 variants stay within 128 registers (two blocks per SM)
  constexpr int E = F32 ? 2 : 1;
  constexpr int U = (F32 && Q == 16) ? 4 : 8;
  const int nx = a.X.total();
  const size_t smem = sizeof(typename Arith<F32>::C) * (size_t)nx * Q + sizeof(void*) * (size_t)nx;
  static bool attr[64] = {};
  if (once_per_device(attr))   // kVecMatMaxRows x 16 coefficients (16 B each) + row table: 132 KiB
    CCLR_CK(cudaFuncSetAttribute(k_vecmat<F32, Q, E, U, X32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 136 << 10));
  AddRows ar;
  for (int q = 0; q < kVecMatOut; ++q) ar.r[q] = a.arow[q];
  k_vecmat<F32, Q, E, U, X32><<<vecmat_blocks(), kThreads, smem, L.s>>>(n, a.X, a.m, a.C, a.add, a.Y, a.ldy, a.acc, a.D, a.z,
                                                              a.norm_y, part, (const float2*)a.addq, a.ldadd, ar);
}
}  // namespace

void vecmat(const Launch& L, int64_t n, const VecMat& a, double* scratch) {
  const int nx = a.X.total();
  CCLR_REQUIRE(a.m >= 1 && a.m <= kVecMatOut && nx >= 1 && nx <= kVecMatMaxRows && a.C, CCLR_E_ARG,
               "vecmat: bad shape");
  CCLR_REQUIRE(!a.D || a.z, CCLR_E_ARG, "vecmat: preconditioner without shifts");
  CCLR_REQUIRE(!a.norm2 || scratch, CCLR_E_ARG, "vecmat: norms without scratch");
  if (n <= 0) return;
  double* part = a.norm2 ? scratch : nullptr;
  kbeg(L);
  CCLR_REQUIRE(!a.x32 || L.fast32, CCLR_E_ARG, "vecmat: FP32 rows need the FP32 arithmetic");
  CCLR_REQUIRE(!a.addq || L.fast32, CCLR_E_ARG, "vecmat: additive FP32 rows need the FP32 arithmetic");
  if (a.x32) {
    if (a.m == 1) launch_vecmat<true, 1, true>(L, n, a, part);
    else if (a.m <= 4) launch_vecmat<true, 4, true>(L, n, a, part);
    else if (a.m <= 8) launch_vecmat<true, 8, true>(L, n, a, part);
    else launch_vecmat<true, 16, true>(L, n, a, part);
  } else if (L.fast32) {
    if (a.m == 1) launch_vecmat<true, 1, false>(L, n, a, part);
    else if (a.m <= 4) launch_vecmat<true, 4, false>(L, n, a, part);
    else if (a.m <= 8) launch_vecmat<true, 8, false>(L, n, a, part);
    else launch_vecmat<true, 16, false>(L, n, a, part);
  } else {
    if (a.m == 1) launch_vecmat<false, 1, false>(L, n, a, part);
    else if (a.m <= 4) launch_vecmat<false, 4, false>(L, n, a, part);
    else if (a.m <= 8) launch_vecmat<false, 8, false>(L, n, a, part);
    else launch_vecmat<false, 16, false>(L, n, a, part);
  }
  CCLR_CK(cudaGetLastError());
  bump(L, shaped("k_vecmat", nx, a.m, a.D ? 1 : 0));
  if (a.norm2) {
    kbeg(L);
    k_sum_rows<<<a.m, kThreads, 0, L.s>>>(part, vecmat_blocks(), a.norm2);
    CCLR_CK(cudaGetLastError());
    bump(L, "k_sum_rows");
  }
}

namespace {
void gm_magic(int64_t d, uint32_t& mul, int& shr) {   // Granlund-Montgomery multiplier of d < 2^31
  int l = 0;
  while ((int64_t(1) << l) < d) ++l;
  shr = l;
  mul = (uint32_t)(((unsigned __int128)1 << 32) * (((uint64_t)1 << l) - (uint64_t)d) / (uint64_t)d + 1);
}
template <int AK>
void launch_permute(const Launch& L, const PermArgs& a, const cplx* src, cplx* dst, int64_t n, cplx al, bool conj,
                    bool acc) {
  // transposing case: the unit-stride source axis is not the unit-stride destination axis
  int S = -1, T = -1;
  for (int k = 0; k < a.rank; ++k) {
    if (a.sstr[k] == 1) S = k;
    if (a.dstr[k] == 1) T = k;
  }
  if (S >= 0 && T >= 0 && S != T && a.dim[S] >= 8 && a.dim[T] >= 8 && n < (int64_t(1) << 31)) {
    TileArgs t{};
    t.dimS = a.dim[S];
    t.dimT = a.dim[T];
    t.sstrT = a.sstr[T];
    t.dstrS = a.dstr[S];
    t.ntS = (uint32_t)((t.dimS + 31) / 32);
    t.ntT = (uint32_t)((t.dimT + 31) / 32);
    gm_magic(t.ntS, t.mulS, t.shrS);
    gm_magic(t.ntT, t.mulT, t.shrT);
    int64_t batch = 1;
    for (int k = 0; k < a.rank; ++k) {
      if (k == S || k == T) continue;
      t.bdim[t.nb] = a.dim[k];
      t.bsstr[t.nb] = a.sstr[k];
      t.bdstr[t.nb] = a.dstr[k];
      gm_magic(a.dim[k], t.bmul[t.nb], t.bshr[t.nb]);
      ++t.nb;
      batch *= a.dim[k];
    }
    const int64_t ntiles = batch * t.ntS * t.ntT;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)num_sms() * 16));
    k_permute_tiled<AK><<<g, 256, 0, L.s>>>(t, src, dst, ntiles, al, conj, acc);
    return;
  }
  const int g = grid_for(n);
  if (n < (int64_t(1) << 31)) k_permute<AK, true><<<g, kThreads, 0, L.s>>>(a, src, dst, n, al, conj, acc);
  else k_permute<AK, false><<<g, kThreads, 0, L.s>>>(a, src, dst, n, al, conj, acc);
}
}  // namespace

void permute(const Launch& L, const Tensor& src, const Tensor& dst, cplx alpha, bool accumulate) {
  CCLR_REQUIRE(src.rank == dst.rank, CCLR_E_ARG, "permute: rank mismatch");
  // drop extent-1 axes and merge neighbours that are contiguous in both source and destination
  PermArgs a{};
  for (int k = 0; k < dst.rank; ++k) {
    CCLR_REQUIRE(src.dim[k] == dst.dim[k], CCLR_E_ARG, "permute: extent mismatch");
    if (dst.dim[k] == 1) continue;
    if (a.rank > 0 && a.sstr[a.rank - 1] == dst.dim[k] * src.str[k] && a.dstr[a.rank - 1] == dst.dim[k] * dst.str[k]) {
      a.dim[a.rank - 1] *= dst.dim[k];
      a.sstr[a.rank - 1] = src.str[k];
      a.dstr[a.rank - 1] = dst.str[k];
    } else {
      a.dim[a.rank] = dst.dim[k];
      a.sstr[a.rank] = src.str[k];
      a.dstr[a.rank] = dst.str[k];
      ++a.rank;
    }
  }
  if (a.rank == 0) {
    a.rank = 1;
    a.dim[0] = 1;
  }
  const int64_t n = dst.numel();
  if (n == 0) return;
  for (int k = 0; k < a.rank; ++k)
    if (a.dim[k] < (int64_t(1) << 31)) gm_magic(a.dim[k], a.mul[k], a.shr[k]);
  cplx al = make_double2(alpha.x * src.scale, alpha.y * src.scale);
  kbeg(L);
  if (al.y == 0.0 && (al.x == 1.0 || al.x == -1.0)) launch_permute<0>(L, a, src.p, dst.p, n, al, src.conj, accumulate);
  else if (al.y == 0.0) launch_permute<1>(L, a, src.p, dst.p, n, al, src.conj, accumulate);
  else launch_permute<2>(L, a, src.p, dst.p, n, al, src.conj, accumulate);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_permute");
}

void to_f32(const Launch& L, const cplx* x, void* y, int64_t n) {
  if (n <= 0) return;
  kbeg(L);
  k_to_f32<<<grid_for(n), kThreads, 0, L.s>>>(x, (float2*)y, n);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_to_f32");
}

void fill_hash(const Launch& L, cplx* p, int64_t n, uint64_t seed) {
  if (n <= 0) return;
  kbeg(L);
  k_fill_hash<<<grid_for(n), kThreads, 0, L.s>>>(p, n, seed);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_fill_hash");
}

void round_coarse(const Launch& L, cplx* x, int64_t n, unsigned* scratch) {
  if (n <= 0) return;
  CCLR_CK(cudaMemsetAsync(scratch, 0, sizeof(unsigned), L.s));
  kbeg(L);
  k_max_bexp<<<grid_for(n), kThreads, 0, L.s>>>(x, n, scratch);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_max_bexp");
  kbeg(L);
  k_round_grid<<<grid_for(n), kThreads, 0, L.s>>>(x, n, scratch);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_round_grid");
}

void flag_nonfinite(const Launch& L, const cplx* p, int64_t n, int* flag) {
  if (n <= 0) return;
  kbeg(L);
  k_nonfinite<<<grid_for(n), kThreads, 0, L.s>>>(p, n, flag);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_nonfinite");
}

void fill_zero(const Launch& L, cplx* p, int64_t n) {
  if (n <= 0) return;
  kbeg(L);
  k_fill_zero<<<grid_for(n), kThreads, 0, L.s>>>(p, n);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_fill_zero");
}

void zgemm(const Launch& L, bool ta, bool tb, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A,
           int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {  // C = beta C
    Tensor c = Tensor::make(C, {M, N});
    c.str[0] = ldc;
    permute(L, c, c, beta, false);
    return;
  }
  const int64_t max_rows = (int64_t)65535 * BM;   // grid.y limit: split the rows into launches
  if (M > max_rows) {
    for (int64_t m0 = 0; m0 < M; m0 += max_rows) {
      const int64_t mm = std::min(max_rows, M - m0);
      zgemm(L, ta, tb, mm, N, K, alpha, ta ? A + m0 : A + m0 * lda, lda, B, ldb, beta, C + m0 * ldc, ldc);
    }
    return;
  }
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  kbeg(L);
  if (!ta && !tb) k_zgemm<false, false><<<grid, 256, 0, L.s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, K, 0);
  else if (!ta && tb) k_zgemm<false, true><<<grid, 256, 0, L.s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, K, 0);
  else if (ta && !tb) k_zgemm<true, false><<<grid, 256, 0, L.s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, K, 0);
  else k_zgemm<true, true><<<grid, 256, 0, L.s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, K, 0);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_zgemm");
}

// Pair tables are uploaded once per Hamiltonian; kept here as a per-process cache keyed by size.
void pack_doubles_impl(const Launch& L, const Tensor& X, cplx* D, int64_t nvec, int o, int v, cplx alpha, bool anti,
                       bool accumulate, const int2* po, const int2* pv) {
  CCLR_REQUIRE(X.rank == 5, CCLR_E_ARG, "pack_doubles: X must have axes (Z,i,j,a,b)");
  CCLR_REQUIRE(!X.conj, CCLR_E_ARG, "pack_doubles: conj view not supported");
  Pack5 s;
  for (int k = 0; k < 5; ++k) s.str[k] = X.str[k];
  // o, v are the ranges of the two pairs (both may be occupied, e.g. for <mn||ij>-type tensors)
  const int64_t Po = (int64_t)o * (o - 1) / 2, Pv = (int64_t)v * (v - 1) / 2;
  const int64_t n = nvec * Po * Pv;
  if (n == 0) return;
  cplx al = make_double2(alpha.x * X.scale, alpha.y * X.scale);
  kbeg(L);
  k_pack<<<grid_for(n), kThreads, 0, L.s>>>(X.p, s, D, nvec, Po, Pv, po, pv, al, anti, accumulate);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_pack");
}

void unpack_doubles(const Launch& L, const cplx* D, int64_t ld_vec, const Tensor& X, int o, int v) {
  CCLR_REQUIRE(X.rank == 5, CCLR_E_ARG, "unpack_doubles: X must have axes (Z,i,j,a,b)");
  Unpack5 u;
  int order[5] = {0, 1, 2, 3, 4};
  // memory order: sort logical axes by decreasing stride (stable)
  for (int a = 0; a < 5; ++a)
    for (int b = a + 1; b < 5; ++b)
      if (X.str[order[b]] > X.str[order[a]]) { int t = order[a]; order[a] = order[b]; order[b] = t; }
  for (int k = 0; k < 5; ++k) {
    u.lax[k] = order[k];
    u.mdim[k] = X.dim[order[k]];
    u.mstr[k] = X.str[order[k]];
  }
  const int64_t n = X.numel();
  if (n == 0) return;
  const int64_t Pv = (int64_t)v * (v - 1) / 2;
  kbeg(L);
  k_unpack<<<grid_for(n), kThreads, 0, L.s>>>(D, ld_vec, Pv, u, X.p, n);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_unpack");
}

void axpy(const Launch& L, int64_t n, cplx a, const cplx* x, cplx* y) {
  if (n <= 0) return;
  kbeg(L);
  k_axpy<<<grid_for(n), kThreads, 0, L.s>>>(n, a, x, y);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_axpy");
}

void scale_vec(const Launch& L, int64_t n, cplx a, cplx* x) {
  if (n <= 0) return;
  kbeg(L);
  k_scale<<<grid_for(n), kThreads, 0, L.s>>>(n, a, x);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_scale");
}

void copy_vec(const Launch& L, int64_t n, const cplx* x, cplx* y) {
  if (n <= 0) return;
  kbeg(L);
  k_copy<<<grid_for(n), kThreads, 0, L.s>>>(n, x, y);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_copy");
}

void diag_axpy(const Launch& L, int64_t n, int64_t nvec, const double* D, const cplx* x, cplx* y) {
  const int64_t total = n * nvec;
  if (total <= 0) return;
  kbeg(L);
  k_diag_axpy<<<grid_for(total), kThreads, 0, L.s>>>(n, total, D, x, y);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_diag_axpy");
}

void div_shift(const Launch& L, int64_t n, const cplx* x, const double* D, cplx z, cplx a, cplx* y) {
  if (n <= 0) return;
  kbeg(L);
  k_div_shift<<<grid_for(n), kThreads, 0, L.s>>>(n, x, D, z, a, y);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_div_shift");
}

void dots(const Launch& L, int64_t n, int nvec, const cplx* x, int64_t ldx, const cplx* y, int64_t ldy, bool herm,
          cplx* out_dev, cplx* scratch) {
  if (nvec <= 0) return;
  dim3 g(reduce_blocks(), nvec);
  kbeg(L);
  if (L.fast32) k_dots_partial32<<<g, kThreads, 0, L.s>>>(n, x, ldx, y, ldy, herm, scratch);
  else k_dots_partial<<<g, kThreads, 0, L.s>>>(n, x, ldx, y, ldy, herm, scratch);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_dots");
  kbeg(L);
  k_sum_partials<<<nvec, kThreads, 0, L.s>>>(scratch, reduce_blocks(), out_dev);
  CCLR_CK(cudaGetLastError());
  bump(L, "k_sum_partials");
}

void proj(const Launch& L, int64_t n, int nb, const cplx* B, int64_t ldb, const cplx* y, cplx* out_dev, cplx* scratch) {
  dots(L, n, nb, B, ldb, y, 0, true, out_dev, scratch);
}

void lincomb(const Launch& L, int64_t n, int nb, const cplx* X, int64_t ldx, const cplx* c_dev, cplx* y,
             bool accumulate) {
  if (n <= 0 || nb <= 0) return;
  Rows r;
  r.add(X, nb, ldx);
  VecMat a;
  a.X = r;
  a.m = 1;
  a.C = c_dev;
  a.Y = y;
  a.ldy = n;
  a.acc = accumulate;
  vecmat(L, n, a, nullptr);
}

}  // namespace cclr

// Complex FP64 kernels of libcclr: strided permutation, DFMA GEMM, doubles pack/unpack, and the
// vector kernels of the iterative solvers (dots, projections, linear combinations, the fused
// residual + orbital-energy-denominator preconditioner).  All reductions are deterministic:
// a fixed grid writes partial sums that one block adds in a fixed order.
#include "internal.h"
#include <algorithm>

namespace cclr {

namespace {

constexpr int kThreads = 256;
constexpr int kReduceBlocks = 296;  // 2 x 148 SMs

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }

inline int grid_for(int64_t n, int per = kThreads) {
  int64_t g = (n + per - 1) / per;
  if (g > 148 * 16) g = 148 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

inline void bump(const Launch& L) { if (L.count) ++*L.count; }

struct PermArgs {
  int rank;
  int64_t dim[kMaxRank];
  int64_t sstr[kMaxRank];
  int64_t dstr[kMaxRank];
};

// alpha kinds: 0 -> +-1 real (sign only), 1 -> real, 2 -> complex
template <int AK>
__global__ void __launch_bounds__(kThreads) k_permute(PermArgs a, const cplx* __restrict__ src, cplx* dst,
                                                      int64_t n, cplx alpha, bool conj, bool acc) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx, so = 0, dof = 0;
#pragma unroll
    for (int k = kMaxRank - 1; k >= 0; --k) {
      if (k < a.rank) {
        int64_t q = r / a.dim[k];
        int64_t c = r - q * a.dim[k];
        r = q;
        so += c * a.sstr[k];
        dof += c * a.dstr[k];
      }
    }
    cplx x = src[so];
    if (conj) x.y = -x.y;
    if (AK == 0) {
      if (alpha.x < 0) { x.x = -x.x; x.y = -x.y; }
    } else if (AK == 1) {
      x.x *= alpha.x;
      x.y *= alpha.x;
    } else {
      x = cmul(alpha, x);
    }
    if (acc) x = cadd(x, dst[dof]);
    dst[dof] = x;
  }
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

// ---- FP32-arithmetic variants of the solver's vector kernels (FP64 storage).  FP64 on sm_103 runs
// at ~1/64 of FP32, and the solver's multi-vector kernels do 8 L m flops per element (L inputs,
// m outputs), so in FP64 they are ALU-bound by a wide margin; in FP32 they stay near the HBM
// roofline.  The inputs are rounded to FP32 (relative 6e-8) and products summed in FP32.
__device__ __forceinline__ float2 f2(cplx a) { return make_float2((float)a.x, (float)a.y); }

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
    float2 a = f2(xk[i]);
    if (herm) a.y = -a.y;
    const float2 b = f2(yk[i]);
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

template <bool F32> struct Arith;
template <> struct Arith<true> {
  typedef float2 T;
  typedef float R;
  __device__ static T cvt(cplx a) { return make_float2((float)a.x, (float)a.y); }
  __device__ static void mac(T& acc, T c, T x) {
    acc.x = fmaf(c.x, x.x, fmaf(-c.y, x.y, acc.x));
    acc.y = fmaf(c.x, x.y, fmaf(c.y, x.x, acc.y));
  }
};
template <> struct Arith<false> {
  typedef double2 T;
  typedef double R;
  __device__ static T cvt(cplx a) { return a; }
  __device__ static void mac(T& acc, T c, T x) {
    acc.x = fma(c.x, x.x, fma(-c.y, x.y, acc.x));
    acc.y = fma(c.x, x.y, fma(c.y, x.x, acc.y));
  }
};

constexpr int kVecMatBlocks = 4 * 148;

// r_q = sum_j X_j C[j][q] + add; Y_q = (D ? -r_q / (D - z_q) : r_q) (+ Y_q); partial norms per
// block.  Q >= m outputs are computed (coefficients of q >= m are zero and never stored).
template <bool F32, int Q>
__global__ void __launch_bounds__(kThreads) k_vecmat(int64_t n, Rows X, int m, const cplx* __restrict__ C,
                                                     const cplx* __restrict__ add, cplx* Y, int64_t ldy, bool acc,
                                                     const double* __restrict__ D, const cplx* __restrict__ z,
                                                     double* part_r, double* part_y) {
  typedef Arith<F32> A;
  typedef typename A::T T;
  typedef typename A::R R;
  extern __shared__ __align__(16) unsigned char vm_smem[];
  const int nx = X.total();
  T* cs = reinterpret_cast<T*>(vm_smem);                                          // nx x Q
  const cplx** rows = reinterpret_cast<const cplx**>(vm_smem + sizeof(T) * (size_t)nx * Q);
  for (int e = threadIdx.x; e < nx * Q; e += blockDim.x) {
    const int j = e / Q, q = e % Q;
    cs[e] = A::cvt(q < m ? C[(int64_t)j * m + q] : make_double2(0.0, 0.0));
  }
  for (int j = threadIdx.x; j < nx; j += blockDim.x) rows[j] = row_of(X, j);
  __syncthreads();
  R nr[Q], ny[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) { nr[q] = 0; ny[q] = 0; }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T a[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) a[q].x = a[q].y = 0;
#pragma unroll 4
    for (int j = 0; j < nx; ++j) {
      const T x = A::cvt(__ldg(rows[j] + i));
#pragma unroll
      for (int q = 0; q < Q; ++q) A::mac(a[q], cs[j * Q + q], x);
    }
    const cplx b = add ? add[i] : make_double2(0.0, 0.0);
    const double di = D ? D[i] : 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (q < m) {
        cplx r = make_double2((double)a[q].x + b.x, (double)a[q].y + b.y);
        nr[q] += (R)(r.x * r.x + r.y * r.y);
        if (D) {
          const cplx zq = z[q];
          const double dr = di - zq.x, dm = -zq.y;
          const double inv = 1.0 / (dr * dr + dm * dm);
          // -r / (D - z) = -r conj(D - z) / |D - z|^2
          r = make_double2(-(r.x * dr + r.y * dm) * inv, -(r.y * dr - r.x * dm) * inv);
        }
        if (Y) {
          cplx* yq = Y + q * ldy + i;
          if (acc) r = cadd(r, *yq);
          *yq = r;
        }
        ny[q] += (R)(r.x * r.x + r.y * r.y);
      }
    }
  }
  if (part_r || part_y) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (q < m) {   // uniform across the block
        if (part_r) {
          const cplx v = block_sum(make_double2((double)nr[q], 0.0));
          if (threadIdx.x == 0) part_r[q * gridDim.x + blockIdx.x] = v.x;
        }
        if (part_y) {
          const cplx v = block_sum(make_double2((double)ny[q], 0.0));
          if (threadIdx.x == 0) part_y[q * gridDim.x + blockIdx.x] = v.x;
        }
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

__global__ void k_sum_real(const double* partial, int nb, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
  cplx v = block_sum(make_double2(s, 0.0));
  if (threadIdx.x == 0) out[0] = v.x;
}

// D[r][P(p,q)] = alpha (X[r,p,q] - X[r,q,p]) or alpha X[r,p,q]  (+ D), X strided (R, m, m)
__global__ void k_pack2(const cplx* __restrict__ X, int64_t sr, int64_t sp, int64_t sq, cplx* D, int64_t ldd,
                        int64_t R, int64_t Pm, const int2* __restrict__ tab, cplx alpha, bool anti, bool acc) {
  const int64_t n = R * Pm;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t P = idx % Pm, r = idx / Pm;
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

// Gram block: part[blk][i][j] = sum over this block's slice of op(X_i[n]) Y_j[n].  Chunks of 16
// elements are staged in shared memory; with F32 the chunk's products are summed in FP32 and
// the chunk sums in FP64.
constexpr int kGramChunk = 16;
template <bool F32>
__global__ void __launch_bounds__(256) k_gram_partial(int64_t n, Rows X, Rows Y, bool herm, cplx* part) {
  typedef Arith<F32> A;
  typedef typename A::T T;
  extern __shared__ __align__(16) unsigned char gr_smem[];
  const int nx = X.total(), ny = Y.total();
  T* xs = reinterpret_cast<T*>(gr_smem);   // nx x kGramChunk
  T* ys = xs + nx * kGramChunk;            // ny x kGramChunk
  const cplx** xrow = reinterpret_cast<const cplx**>(ys + ny * kGramChunk);
  const cplx** yrow = xrow + nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) xrow[i] = row_of(X, i);
  for (int j = threadIdx.x; j < ny; j += blockDim.x) yrow[j] = row_of(Y, j);
  __syncthreads();
  const int nout = nx * ny;
  const int per = (nout + 255) / 256;      // outputs per thread (<= 16)
  cplx acc[16];
  for (int q = 0; q < 16; ++q) acc[q] = make_double2(0.0, 0.0);
  const int64_t nchunks = (n + kGramChunk - 1) / kGramChunk;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t base = ch * kGramChunk;
    for (int e = threadIdx.x; e < nx * kGramChunk; e += 256) {
      const int i = e / kGramChunk, k = e % kGramChunk;
      cplx v = (base + k < n) ? xrow[i][base + k] : make_double2(0.0, 0.0);
      if (herm) v.y = -v.y;
      xs[e] = A::cvt(v);
    }
    for (int e = threadIdx.x; e < ny * kGramChunk; e += 256) {
      const int j = e / kGramChunk, k = e % kGramChunk;
      ys[e] = A::cvt((base + k < n) ? yrow[j][base + k] : make_double2(0.0, 0.0));
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int o = threadIdx.x + 256 * q;
      if (q < per && o < nout) {
        const int i = o / ny, j = o % ny;
        T s;
        s.x = s.y = 0;
#pragma unroll
        for (int k = 0; k < kGramChunk; ++k) A::mac(s, xs[i * kGramChunk + k], ys[j * kGramChunk + k]);
        acc[q].x += (double)s.x;
        acc[q].y += (double)s.y;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int o = threadIdx.x + 256 * q;
    if (q < per && o < nout) part[(int64_t)blockIdx.x * nout + o] = acc[q];
  }
}

__global__ void k_gram_reduce(const cplx* __restrict__ part, int nblk, int nout, cplx* out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  cplx s = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) s = cadd(s, part[(int64_t)b * nout + o]);
  out[o] = s;
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

int reduce_blocks() { return kReduceBlocks; }

void splitk_reduce(const Launch& L, const cplx* P, int S, int64_t M, int64_t N, cplx alpha, cplx beta, cplx* C,
                   int64_t ldc) {
  k_splitk_reduce<<<grid_for(M * N), kThreads, 0, L.s>>>(P, S, M, N, alpha, beta, C, ldc);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void zgemm_splitk(const Launch& L, bool ta, bool tb, int64_t M, int64_t N, int64_t K, const cplx* A, int64_t lda,
                  const cplx* B, int64_t ldb, cplx* P, int S, int64_t kchunk) {
  // partials P[z] (M x N, ld N) over k in [z*kchunk, (z+1)*kchunk); kchunk a multiple of 8
  CCLR_REQUIRE((M + BM - 1) / BM <= 65535 && S <= 65535, CCLR_E_ARG, "zgemm_splitk: grid too large");
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)S);
  const cplx one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  if (!ta && !tb) k_zgemm<false, false><<<grid, 256, 0, L.s>>>(M, N, K, one, A, lda, B, ldb, zero, P, N, kchunk, M * N);
  else if (!ta && tb) k_zgemm<false, true><<<grid, 256, 0, L.s>>>(M, N, K, one, A, lda, B, ldb, zero, P, N, kchunk, M * N);
  else if (ta && !tb) k_zgemm<true, false><<<grid, 256, 0, L.s>>>(M, N, K, one, A, lda, B, ldb, zero, P, N, kchunk, M * N);
  else k_zgemm<true, true><<<grid, 256, 0, L.s>>>(M, N, K, one, A, lda, B, ldb, zero, P, N, kchunk, M * N);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void pack2(const Launch& L, const Tensor& X, cplx* D, int64_t ldd, const int2* tab, cplx alpha, bool anti, bool acc) {
  CCLR_REQUIRE(X.rank == 3 && X.dim[1] == X.dim[2] && !X.conj, CCLR_E_ARG, "pack2: X must be (R, m, m)");
  const int64_t m = X.dim[1], Pm = m * (m - 1) / 2, R = X.dim[0];
  if (R * Pm == 0) return;
  cplx al = make_double2(alpha.x * X.scale, alpha.y * X.scale);
  k_pack2<<<grid_for(R * Pm), kThreads, 0, L.s>>>(X.p, X.str[0], X.str[1], X.str[2], D, ldd, R, Pm, tab, al, anti, acc);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void unpack2(const Launch& L, const cplx* D, int64_t ldd, const Tensor& X) {
  CCLR_REQUIRE(X.rank == 3 && X.dim[1] == X.dim[2], CCLR_E_ARG, "unpack2: X must be (R, m, m)");
  const int64_t n = X.numel();
  if (n == 0) return;
  k_unpack2<<<grid_for(n), kThreads, 0, L.s>>>(D, ldd, X.p, X.str[0], X.str[1], X.str[2], X.dim[0], (int)X.dim[1]);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void gram(const Launch& L, int64_t n, const Rows& X, const Rows& Y, bool herm, cplx* out_dev, cplx* scratch,
          int64_t scratch_elems) {
  const int nx = X.total(), ny = Y.total();
  CCLR_REQUIRE(nx >= 1 && ny >= 1 && nx * ny <= 4096 && nx + ny <= 256, CCLR_E_ARG, "gram: block too large");
  const int nout = nx * ny;
  int nblk = (int)std::min<int64_t>(kReduceBlocks, (n + kGramChunk - 1) / kGramChunk);
  if (nblk < 1) nblk = 1;
  if ((int64_t)nblk * nout > scratch_elems) nblk = (int)std::max<int64_t>(1, scratch_elems / nout);
  const size_t smem = ((L.fast32 ? sizeof(float2) : sizeof(cplx)) * kGramChunk + sizeof(void*)) * (size_t)(nx + ny);
  static bool attr = false;
  if (!attr) {   // up to 256 staged rows of FP64 plus their row pointers: 66 KiB
    CCLR_CK(cudaFuncSetAttribute(k_gram_partial<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 72 << 10));
    CCLR_CK(cudaFuncSetAttribute(k_gram_partial<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 72 << 10));
    attr = true;
  }
  if (L.fast32) k_gram_partial<true><<<nblk, 256, smem, L.s>>>(n, X, Y, herm, scratch);
  else k_gram_partial<false><<<nblk, 256, smem, L.s>>>(n, X, Y, herm, scratch);
  CCLR_CK(cudaGetLastError());
  k_gram_reduce<<<(nout + 255) / 256, 256, 0, L.s>>>(scratch, nblk, nout, out_dev);
  CCLR_CK(cudaGetLastError());
  bump(L);
  bump(L);
}

int64_t vecmat_scratch_doubles() { return 2 * (int64_t)kVecMatOut * kVecMatBlocks; }

namespace {
template <bool F32, int Q>
void launch_vecmat(const Launch& L, int64_t n, const VecMat& a, double* pr, double* py) {
  const int nx = a.X.total();
  const size_t smem = sizeof(typename Arith<F32>::T) * (size_t)nx * Q + sizeof(void*) * (size_t)nx;
  static bool attr = false;
  if (!attr) {   // kVecMatMaxRows x 16 FP64 coefficients + row table: 132 KiB
    CCLR_CK(cudaFuncSetAttribute(k_vecmat<F32, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, 136 << 10));
    attr = true;
  }
  k_vecmat<F32, Q><<<kVecMatBlocks, kThreads, smem, L.s>>>(n, a.X, a.m, a.C, a.add, a.Y, a.ldy, a.acc, a.D, a.z, pr,
                                                           py);
}
}  // namespace

void vecmat(const Launch& L, int64_t n, const VecMat& a, double* scratch) {
  const int nx = a.X.total();
  CCLR_REQUIRE(a.m >= 1 && a.m <= kVecMatOut && nx >= 1 && nx <= kVecMatMaxRows && a.C, CCLR_E_ARG,
               "vecmat: bad shape");
  CCLR_REQUIRE(!a.D || a.z, CCLR_E_ARG, "vecmat: preconditioner without shifts");
  if (n <= 0) return;
  double* pr = a.rnorm2 ? scratch : nullptr;
  double* py = a.ynorm2 ? scratch + (int64_t)kVecMatOut * kVecMatBlocks : nullptr;
  if (L.fast32) {
    if (a.m == 1) launch_vecmat<true, 1>(L, n, a, pr, py);
    else if (a.m <= 4) launch_vecmat<true, 4>(L, n, a, pr, py);
    else launch_vecmat<true, 16>(L, n, a, pr, py);
  } else {
    if (a.m == 1) launch_vecmat<false, 1>(L, n, a, pr, py);
    else if (a.m <= 4) launch_vecmat<false, 4>(L, n, a, pr, py);
    else launch_vecmat<false, 16>(L, n, a, pr, py);
  }
  CCLR_CK(cudaGetLastError());
  bump(L);
  if (a.rnorm2) {
    k_sum_rows<<<a.m, kThreads, 0, L.s>>>(pr, kVecMatBlocks, a.rnorm2);
    CCLR_CK(cudaGetLastError());
    bump(L);
  }
  if (a.ynorm2) {
    k_sum_rows<<<a.m, kThreads, 0, L.s>>>(py, kVecMatBlocks, a.ynorm2);
    CCLR_CK(cudaGetLastError());
    bump(L);
  }
}

void permute(const Launch& L, const Tensor& src, const Tensor& dst, cplx alpha, bool accumulate) {
  CCLR_REQUIRE(src.rank == dst.rank, CCLR_E_ARG, "permute: rank mismatch");
  PermArgs a{};
  a.rank = dst.rank;
  for (int k = 0; k < dst.rank; ++k) {
    CCLR_REQUIRE(src.dim[k] == dst.dim[k], CCLR_E_ARG, "permute: extent mismatch");
    a.dim[k] = dst.dim[k];
    a.sstr[k] = src.str[k];
    a.dstr[k] = dst.str[k];
  }
  const int64_t n = dst.numel();
  if (n == 0) return;
  cplx al = make_double2(alpha.x * src.scale, alpha.y * src.scale);
  const int g = grid_for(n);
  if (al.y == 0.0 && (al.x == 1.0 || al.x == -1.0))
    k_permute<0><<<g, kThreads, 0, L.s>>>(a, src.p, dst.p, n, al, src.conj, accumulate);
  else if (al.y == 0.0)
    k_permute<1><<<g, kThreads, 0, L.s>>>(a, src.p, dst.p, n, al, src.conj, accumulate);
  else
    k_permute<2><<<g, kThreads, 0, L.s>>>(a, src.p, dst.p, n, al, src.conj, accumulate);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void fill_zero(const Launch& L, cplx* p, int64_t n) {
  if (n <= 0) return;
  k_fill_zero<<<grid_for(n), kThreads, 0, L.s>>>(p, n);
  CCLR_CK(cudaGetLastError());
  bump(L);
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
  if (!ta && !tb) k_zgemm<false, false><<<grid, 256, 0, L.s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, K, 0);
  else if (!ta && tb) k_zgemm<false, true><<<grid, 256, 0, L.s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, K, 0);
  else if (ta && !tb) k_zgemm<true, false><<<grid, 256, 0, L.s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, K, 0);
  else k_zgemm<true, true><<<grid, 256, 0, L.s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, K, 0);
  CCLR_CK(cudaGetLastError());
  bump(L);
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
  k_pack<<<grid_for(n), kThreads, 0, L.s>>>(X.p, s, D, nvec, Po, Pv, po, pv, al, anti, accumulate);
  CCLR_CK(cudaGetLastError());
  bump(L);
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
  k_unpack<<<grid_for(n), kThreads, 0, L.s>>>(D, ld_vec, Pv, u, X.p, n);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void axpy(const Launch& L, int64_t n, cplx a, const cplx* x, cplx* y) {
  if (n <= 0) return;
  k_axpy<<<grid_for(n), kThreads, 0, L.s>>>(n, a, x, y);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void scale_vec(const Launch& L, int64_t n, cplx a, cplx* x) {
  if (n <= 0) return;
  k_scale<<<grid_for(n), kThreads, 0, L.s>>>(n, a, x);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void copy_vec(const Launch& L, int64_t n, const cplx* x, cplx* y) {
  if (n <= 0) return;
  k_copy<<<grid_for(n), kThreads, 0, L.s>>>(n, x, y);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void div_shift(const Launch& L, int64_t n, const cplx* x, const double* D, cplx z, cplx a, cplx* y) {
  if (n <= 0) return;
  k_div_shift<<<grid_for(n), kThreads, 0, L.s>>>(n, x, D, z, a, y);
  CCLR_CK(cudaGetLastError());
  bump(L);
}

void dots(const Launch& L, int64_t n, int nvec, const cplx* x, int64_t ldx, const cplx* y, int64_t ldy, bool herm,
          cplx* out_dev, cplx* scratch) {
  if (nvec <= 0) return;
  dim3 g(kReduceBlocks, nvec);
  if (L.fast32) k_dots_partial32<<<g, kThreads, 0, L.s>>>(n, x, ldx, y, ldy, herm, scratch);
  else k_dots_partial<<<g, kThreads, 0, L.s>>>(n, x, ldx, y, ldy, herm, scratch);
  CCLR_CK(cudaGetLastError());
  k_sum_partials<<<nvec, kThreads, 0, L.s>>>(scratch, kReduceBlocks, out_dev);
  CCLR_CK(cudaGetLastError());
  bump(L);
  bump(L);
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

// Counter-based synthetic instance generated on the device (cclr_set_synthetic).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with counter (element index
// low 32 bits, high 32 bits, stream, 0) and key (seed low 32 bits, high 32 bits).  A normal pair
// per element by Box-Muller from two 53-bit uniforms, u1 in (0, 1] and u2 in [0, 1).  ln u1 and
// sin / cos of 2 pi u2 are evaluated from their series with explicitly rounded FP64 operations
// in a fixed order (no library transcendental, no fused multiply-add), the same sequence as the
// host generator, so that both produce identical bits:
//   ln u = e ln 2 + 2 s sum_{j<20} s^2j / (2j + 1),  u = m 2^e, m in [0.5, 1), s = (m - 1)/(m + 1);
//   2 pi u2 = (q + f) pi / 2 with q = floor(4 u2), f = 4 u2 - q; sin and cos of a = f pi / 2 by
//   Horner-form Taylor series to a^26 / 26!.
// Streams: 0 orbital energies, 1..6 the classes oooo, ooov, oovv, ovov, ovvv, vvvv, 100 + k the
// operator k.  Hermitian classes (oooo and vvvv over pairs, ovov over (ia), the operators) draw
// element (min(I, J), max(I, J)) of their m x m matrix at index min m + max, conjugate it below
// the diagonal and keep the real part on the diagonal.
#include "ctx.h"
#include "internal.h"

namespace cclr {
namespace {

constexpr double kLn2 = 0.6931471805599453;
constexpr double kHalfPi = 1.5707963267948966;
constexpr int kLogTerms = 20;
constexpr int kTrigTerms = 13;

__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = (uint32_t)p1;
    c[2] = n2;
    c[3] = (uint32_t)p0;
  }
}

__device__ __forceinline__ void words(uint64_t idx, uint32_t stream, uint64_t seed, uint32_t (&w)[4]) {
  w[0] = (uint32_t)idx;
  w[1] = (uint32_t)(idx >> 32);
  w[2] = stream;
  w[3] = 0u;
  philox4x32_10(w, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// ln u for u in (0, 1] (u normal): the fixed-order series of the header comment
__device__ double ln01(double u) {
  const uint64_t b = (uint64_t)__double_as_longlong(u);
  const int e = (int)((b >> 52) & 0x7ffu) - 1022;
  const double m = __longlong_as_double((long long)((b & 0x800FFFFFFFFFFFFFull) | (1022ull << 52)));
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double s2 = __dmul_rn(s, s);
  double q = __ddiv_rn(1.0, (double)(2 * kLogTerms - 1));
  for (int j = kLogTerms - 2; j >= 0; --j) q = __dadd_rn(__ddiv_rn(1.0, (double)(2 * j + 1)), __dmul_rn(s2, q));
  return __dadd_rn(__dmul_rn((double)e, kLn2), __dmul_rn(__dmul_rn(2.0, s), q));
}

__device__ void sincos_quarter(double a, double& sn, double& cs) {
  const double a2 = __dmul_rn(a, a);
  double S = 1.0, C = 1.0;
  for (int k = kTrigTerms; k >= 1; --k) {
    S = __dsub_rn(1.0, __dmul_rn(__ddiv_rn(a2, (double)((2 * k) * (2 * k + 1))), S));
    C = __dsub_rn(1.0, __dmul_rn(__ddiv_rn(a2, (double)((2 * k - 1) * (2 * k))), C));
  }
  sn = __dmul_rn(a, S);
  cs = C;
}

__device__ double2 normal_pair(uint64_t idx, uint32_t stream, uint64_t seed, double sd) {
  uint32_t w[4];
  words(idx, stream, seed, w);
  const double u1 = __dmul_rn(__dadd_rn(__dadd_rn(__dmul_rn((double)(w[0] >> 5), 67108864.0), (double)(w[1] >> 6)), 1.0),
                              1.1102230246251565e-16);   // 2^-53
  const double u2 = __dmul_rn(__dadd_rn(__dmul_rn((double)(w[2] >> 5), 67108864.0), (double)(w[3] >> 6)),
                              1.1102230246251565e-16);
  const double r = __dsqrt_rn(fmax(0.0, __dmul_rn(-2.0, ln01(u1))));
  const double t4 = __dmul_rn(4.0, u2);
  const int q = (int)t4;   // floor: t4 in [0, 4)
  double sn, cs;
  sincos_quarter(__dmul_rn(__dsub_rn(t4, (double)q), kHalfPi), sn, cs);
  const double ct = q == 0 ? cs : q == 1 ? -sn : q == 2 ? -cs : sn;
  const double st = q == 0 ? sn : q == 1 ? cs : q == 2 ? -sn : -cs;
  return make_double2(__dmul_rn(sd, __dmul_rn(r, ct)), __dmul_rn(sd, __dmul_rn(r, st)));
}

__global__ void k_syn_general(cplx* __restrict__ out, int64_t count, uint32_t stream, uint64_t seed, double sd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = normal_pair((uint64_t)i, stream, seed, sd);
}

__global__ void k_syn_hermitian(cplx* __restrict__ out, int64_t m, uint32_t stream, uint64_t seed, double sd) {
  const int64_t count = m * m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = i / m, J = i - I * m;
    const int64_t lo = I < J ? I : J, hi = I < J ? J : I;
    double2 z = normal_pair((uint64_t)(lo * m + hi), stream, seed, sd);
    if (I > J) z.y = -z.y;
    if (I == J) z.y = 0.0;
    out[i] = z;
  }
}

__global__ void k_syn_uniform(double* __restrict__ out, int n, uint32_t stream, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t w[4];
  words((uint64_t)i, stream, seed, w);
  out[i] = __dmul_rn(__dadd_rn(__dmul_rn((double)(w[0] >> 5), 67108864.0), (double)(w[1] >> 6)), 1.1102230246251565e-16);
}

int syn_grid(int64_t count) {
  const int64_t blocks = (count + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms() * 32));
}

}  // namespace

// Fills the six packed integral classes (device arrays of the sizes cclr_set_hamiltonian takes),
// the n uniforms of the orbital energies (device) and n_ops operators (device, n_ops x n x n).
void synthetic_instance(Ctx& c, int n_occ, int n_vir, uint64_t seed, double sd, double dip_sd, int n_ops,
                        cplx* const blocks[6], double* eps_u, cplx* ops) {
  const int64_t o = n_occ, v = n_vir, n = o + v, Po = o * (o - 1) / 2, Pv = v * (v - 1) / 2;
  const int64_t herm_m[6] = {Po, 0, 0, o * v, 0, Pv};
  const int64_t general_count[6] = {0, Po * o * v, Po * Pv, 0, o * v * Pv, 0};
  for (int k = 0; k < 6; ++k) {
    if (herm_m[k] > 0)
      k_syn_hermitian<<<syn_grid(herm_m[k] * herm_m[k]), 256, 0, c.stream>>>(blocks[k], herm_m[k], (uint32_t)(k + 1),
                                                                          seed, sd);
    else
      k_syn_general<<<syn_grid(general_count[k]), 256, 0, c.stream>>>(blocks[k], general_count[k], (uint32_t)(k + 1),
                                                                    seed, sd);
    CCLR_CK(cudaGetLastError());
  }
  k_syn_uniform<<<(int)((n + 255) / 256), 256, 0, c.stream>>>(eps_u, (int)n, 0u, seed);
  CCLR_CK(cudaGetLastError());
  for (int k = 0; k < n_ops; ++k) {
    k_syn_hermitian<<<syn_grid(n * n), 256, 0, c.stream>>>(ops + (int64_t)k * n * n, n, (uint32_t)(100 + k), seed,
                                                          dip_sd);
    CCLR_CK(cudaGetLastError());
  }
}

}  // namespace cclr

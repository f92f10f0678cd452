// Tensor-core complex GEMM for sm_103a (tcgen05 + TMA + TMEM), used by the mixed-precision
// modes for the two contractions that carry ~90% of the sigma-vector work: the packed
// particle-particle ladder (SI Eq. sigma_double-ee, 1/2 W_abef r_ij^ef) and the ring
// P(ij)P(ab) W_mbej r_im^ae.
//
// C[m*ldc + n] = alpha * sum_k A[m,k] B[n,k] + beta * C     (complex, both operands K-major)
//
// Each complex FP64 operand is split into BF16 slices, x = x_0 + x_1 (+ x_2): x_0 = bf16(x),
// x_1 = bf16(x - x_0), ...; slice products (s,t) with s + t below the slice count are summed in
// FP32 accumulators in tensor memory.  Real and imaginary parts are separate planes; the complex
// product uses four real MMAs per k-step into two accumulators, the minus sign of Ai*Bi coming
// from the instruction descriptor's negate-A bit, so no operand is duplicated in memory.
//
// Tile: 128 rows of the "A-side" MMA operand (= 128 consecutive n, one TMEM lane each) x BN rows
// of the "B-side" operand (= BN consecutive m, TMEM columns).  The kernel is persistent (one CTA
// per SM) and warp-specialised: a TMA producer, a single-thread MMA issuer and four epilogue warps
// that drain one of two TMEM accumulators while the next tile accumulates in the other; stores
// are contiguous along n.  Every mbarrier wait is bounded: on expiry the kernel records an error
// code, stops issuing work, releases TMEM and returns.
#include "ctx.h"
#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>

namespace cclr {

namespace tc {

constexpr int BM = 128;         // MMA M (TMEM lanes) = n-rows per CTA
constexpr int BN = 128;         // MMA N = m-rows per CTA
constexpr int BK = 64;          // K per stage (one 128-byte swizzle row of BF16)
constexpr int STAGES = 3;
constexpr int A_PLANE = BM * BK * 2;           // bytes of one BF16 plane tile
constexpr int B_PLANE = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * A_PLANE + 2 * B_PLANE;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/ + 2 * BN * 8 /*row offsets*/;
constexpr int TMEM_COLS = 2 * BN;              // Cr | Ci
constexpr int MAX_PAIRS = 6;

struct Pairs {
  int n;
  int sa[MAX_PAIRS], sb[MAX_PAIRS];
};

// Strided output: the element (m, n) of the product lives at C + moff(m) + noff(n), each offset a
// row-major decomposition of the index over up to four axes (extents, strides, and the
// Granlund-Montgomery multipliers of the extents: q = (umulhi(i, mul) + i) >> shr).
struct OutMap {
  int nm = 0, nn = 0;
  int64_t mdim[4] = {}, mstr[4] = {}, ndim[4] = {}, nstr[4] = {};
  uint32_t mmul[4] = {}, nmul[4] = {};
  int mshr[4] = {}, nshr[4] = {};
};
__device__ __forceinline__ int64_t out_off(uint32_t i, int na, const int64_t* dim, const int64_t* str,
                                           const uint32_t* mul, const int* shr) {
  int64_t off = 0;
#pragma unroll
  for (int a = 3; a >= 0; --a) {
    if (a >= na) continue;
    const uint32_t q = (uint32_t)(((uint64_t)__umulhi(i, mul[a]) + i) >> shr[a]);
    off += (int64_t)(i - q * (uint32_t)dim[a]) * str[a];
    i = q;
  }
  return off;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: ~2^22 polls with back-off (about a second) unless a limit is given; false on expiry
constexpr uint32_t kWaitPolls = 1u << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint32_t polls = kWaitPolls) {
  for (uint32_t i = 0; i < polls; ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if (i > 64) __nanosleep(256);
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                   // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool negA) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((negA ? 1u : 0u) << 13) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// IEEE 754 binary32 -> binary64 on the integer pipe (exact for normal inputs; binary32
// subnormals flush to zero; infinities and NaN are kept)
__device__ __forceinline__ double epi_f2d(float x) {
  const uint32_t u = __float_as_uint(x), sign = u & 0x80000000u, e = (u >> 23) & 0xffu;
  uint32_t hi = (((u & 0x7fffffffu) >> 3) + 0x38000000u) | sign, lo = u << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 0xffu) { hi = sign | 0x7ff00000u | ((u & 0x7fffffu) ? 0x80000u : 0u); lo = 0u; }
  return __longlong_as_double((long long)(((uint64_t)hi << 32) | lo));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// OR of q over the 384 epilogue threads (named barrier 1; all of them must call it)
__device__ __forceinline__ bool group_any(bool q) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, 384, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)q)
      : "memory");
  return r != 0;
}

// Persistent, warp-specialised kernel: one CTA per SM walks the tiles t = blockIdx.x + i gridDim.x
// (tile = (m-tile fastest, n-tile, split-K slice z)).  Warp 0 lane 0 streams operand tiles into a
// STAGES-deep shared-memory ring with TMA, warp 1 lane 0 issues tcgen05.mma into one of two TMEM
// accumulators (Cr | Ci, 2 x 256 columns), and warps 2..13 drain the other accumulator to C
// (three warps per TMEM lane quarter, 16-column chunks in turn: short-K contractions are bound by
// this read-modify-write of C), so a tile's epilogue overlaps the next tile's MMAs.  Every mbarrier wait is bounded; on expiry the
// kernel records an error code, stops issuing work, waits (bounded) for its MMAs, frees TMEM and
// returns.
constexpr int EPI_WARPS = 12;
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int TC_THREADS = 64 + EPI_THREADS;
// dynamic shared memory of k_tc_zgemm<BN, STAGES>
constexpr int smem_bytes(int bn, int stages) {
  return stages * (2 * A_PLANE + 2 * bn * BK * 2) + 1024 /*align*/ + 256 /*barriers*/ + 2 * bn * 8 /*row offsets*/;
}

template <int BN_, int ST_>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_zgemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int n_rows, int m_rows,
               int kblocks, int kb_per, Pairs pairs, double2 alpha, double2 beta, double2* __restrict__ C, int64_t ldc,
               int64_t cz, int* __restrict__ err, int xtiles, int ytiles, int nsplit, const OutMap om, bool strided,
               uint32_t polls, int expire_first) {
  constexpr int BP_ = BN_ * BK * 2;            // bytes of one B-side BF16 plane tile
  constexpr int SB_ = 2 * A_PLANE + 2 * BP_;     // bytes of one pipeline stage
  constexpr int TC_ = 2 * BN_;                   // TMEM columns of one accumulator (Cr | Ci)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + ST_ * SB_);
  uint64_t* empty = full + ST_;
  uint64_t* tfull = empty + ST_;    // accumulator b holds a finished tile (MMA commit)
  uint64_t* tempty = tfull + 2;        // accumulator b drained (all epilogue threads)
  uint64_t* done = tempty + 2;         // every MMA of this CTA has completed
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int64_t* moff = (int64_t*)(smem + ST_ * SB_ + 256);   // [2][BN_] strided row offsets
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST_; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_THREADS);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * TC_));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int xy = xtiles * ytiles;
  const int ntiles = xy * nsplit;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: the ring runs on across tile boundaries
      int g = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        const int z = t / xy, r = t - z * xy, y = r / xtiles, x = r - y * xtiles;
        const int kb0 = z * kb_per, kb1 = min(kblocks, kb0 + kb_per);
        const int n0 = y * BM, m0 = x * BN_;
        const int iters = (kb1 - kb0) * pairs.n;
        for (int it = 0; it < iters; ++it, ++g) {
          const int s = g % ST_;
          const uint32_t ph = (uint32_t)(g / ST_) & 1u;
          // expire_first (tests of the expiry path): the first wait is for a phase that nothing
          // completes, so it runs out before any copy or MMA is issued
          const uint32_t par = (g == 0 && expire_first) ? ph : (ph ^ 1u);
          if (!mbar_wait(&empty[s], par, polls)) { atomicExch(err, 1); *abort_flag = 1; break; }
          if (*abort_flag) break;
          const int kb = kb0 + it / pairs.n, p = it % pairs.n;
          uint8_t* st = smem + s * SB_;
          mbar_expect_tx(&full[s], SB_);
          tma_load_3d(st, &tmA, kb * BK, n0, 2 * pairs.sa[p] + 0, &full[s]);
          tma_load_3d(st + A_PLANE, &tmA, kb * BK, n0, 2 * pairs.sa[p] + 1, &full[s]);
          tma_load_3d(st + 2 * A_PLANE, &tmB, kb * BK, m0, 2 * pairs.sb[p] + 0, &full[s]);
          tma_load_3d(st + 2 * A_PLANE + BP_, &tmB, kb * BK, m0, 2 * pairs.sb[p] + 1, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer (single thread)
      constexpr uint32_t ID = idesc_bf16(BM, BN_, false), IDN = idesc_bf16(BM, BN_, true);
      int g = 0, tl = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tl) {
        const int z = t / xy;
        const int kb0 = z * kb_per, kb1 = min(kblocks, kb0 + kb_per);
        const int iters = (kb1 - kb0) * pairs.n;
        const int b = tl & 1;
        if (!mbar_wait(&tempty[b], (((uint32_t)tl >> 1) & 1u) ^ 1u, polls)) { atomicExch(err, 4); *abort_flag = 1; break; }
        fence_after();
        const uint32_t cr = tmem + b * TC_, ci = cr + BN_;
        bool ok = true;
        for (int it = 0; it < iters; ++it, ++g) {
          const int s = g % ST_;
          const uint32_t ph = (uint32_t)(g / ST_) & 1u;
          if (!mbar_wait(&full[s], ph, polls)) { atomicExch(err, 2); *abort_flag = 1; ok = false; break; }
          fence_after();
          const uint32_t base = smem_u32(smem + s * SB_);
          const uint32_t ar = base, ai = base + A_PLANE, br = base + 2 * A_PLANE, bi = br + BP_;
#pragma unroll
          for (int ks = 0; ks < BK / 16; ++ks) {
            const uint32_t off = ks * 32;  // 16 BF16 = 32 bytes along K inside the swizzle row
            const uint64_t dar = desc_sw128(ar + off), dai = desc_sw128(ai + off);
            const uint64_t dbr = desc_sw128(br + off), dbi = desc_sw128(bi + off);
            const uint32_t first = (it == 0 && ks == 0) ? 0u : 1u;
            mma_bf16(cr, dar, dbr, ID, first);
            mma_bf16(cr, dai, dbi, IDN, 1u);
            mma_bf16(ci, dar, dbi, ID, first);
            mma_bf16(ci, dai, dbr, ID, 1u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[b]);
      }
      mma_commit(done);
    }
  } else {
    // ---------------- epilogue warps 2..13: TMEM lanes 32 (warp % 4) .. +32, 16-column chunks
    // starting at 16 ch, ch = (warp - 2) / 4, in steps of 48
    const int et = threadIdx.x - 64;                 // 0..EPI_THREADS-1
    const int lg = warp & 3;                         // TMEM lane quarter of this warp
    const int ch = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(lg * 32) << 16;
    // The accumulators are FP32: alpha is applied in FP32 and the result widened on the integer
    // pipe (FP64 arithmetic and FP32 <-> FP64 cvt issue on the FP64 pipe, ~1/64 of the FP32 rate
    // on sm_103); only the beta term uses FP64.
    const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
    const bool beta_one = (beta.x == 1.0 && beta.y == 0.0);
    const float ar = (float)alpha.x, ai = (float)alpha.y;
    // Control flow stays uniform across the epilogue threads: every exit decision is taken
    // through a barrier reduction over named barrier 1, so no thread is left waiting in it.
    int tl = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      const int z = t / xy, r = t - z * xy, y = r / xtiles, x = r - y * xtiles;
      const int n0 = y * BM, m0 = x * BN_;
      const int b = tl & 1;
      double2* Cz = C + (int64_t)z * cz;
      int64_t* mo = moff + b * BN_;
      if (strided && et < BN_) {
        const int m = m0 + et;
        mo[et] = m < m_rows ? out_off((uint32_t)m, om.nm, om.mdim, om.mstr, om.mmul, om.mshr) : 0;
      }
      if (group_any(*abort_flag != 0)) break;   // also publishes this tile's offsets to the group
      const int n = n0 + lg * 32 + lane;
      const int64_t noff = (strided && n < n_rows) ? out_off((uint32_t)n, om.nn, om.ndim, om.nstr, om.nmul, om.nshr) : 0;
      const bool ready = mbar_wait(&tfull[b], ((uint32_t)tl >> 1) & 1u, polls);
      if (group_any(!ready)) {
        if (et == 0) atomicExch(err, 3);
        *abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t acc = tmem + b * TC_ + lane_base;
#pragma unroll 1
      for (int c0 = 16 * ch; c0 < BN_; c0 += 16 * (EPI_WARPS / 4)) {
        uint32_t rr[16], ri[16];
        tmem_ld16(acc + c0, rr);
        tmem_ld16(acc + BN_ + c0, ri);
        if (n < n_rows) {
          // the beta operands of the chunk are all loaded before any is used
          double2 old[16];
          if (use_beta) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int m = m0 + c0 + j;
              if (m < m_rows) old[j] = *(strided ? Cz + mo[c0 + j] + noff : Cz + (int64_t)m * ldc + n);
            }
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int m = m0 + c0 + j;
            if (m < m_rows) {
              const float xr = __uint_as_float(rr[j]), xi = __uint_as_float(ri[j]);
              double2 v = make_double2(epi_f2d(ar * xr - ai * xi), epi_f2d(ar * xi + ai * xr));
              if (use_beta) {
                const double2 o = old[j];
                if (beta_one) {
                  v.x += o.x;
                  v.y += o.y;
                } else {
                  v.x += beta.x * o.x - beta.y * o.y;
                  v.y += beta.x * o.y + beta.y * o.x;
                }
              }
              *(strided ? Cz + mo[c0 + j] + noff : Cz + (int64_t)m * ldc + n) = v;
            }
          }
        }
      }
      fence_before();
      mbar_arrive(&tempty[b]);   // this thread's part of accumulator b has been read
    }
  }
  __syncwarp();
  fence_before();
  __syncthreads();
  if (warp == 2) {
    fence_after();
    // the MMAs may still run if a role gave up early: wait (bounded) for all of them first
    if (!mbar_wait(done, 0, polls) && lane == 0) atomicExch(err, 5);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_));
  }
}

// ------------------------------------------------------------------------------------------
// FP64-class mode (CCLR_TC_F64): the Ozaki splitting (Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012) on BF16 tensor cores.  Every operand row r gets
// the exponent e_r with |x| < 2^e_r for all its elements, and each element is written as five
// signed base-256 digits on the row's grid:
//     x = sum_{s<5} d_s 2^(e_r - 7 - 8 s) + O(2^(e_r - 40)),   |d_s| <= 128,
// each digit stored exactly as a BF16 value.  A digit product d_i d_j (|.| <= 2^14) lies on the
// grid 2^(e_m + e_n - 14 - 8(i + j)) of the output element, so the products of one "group"
// (i + j = g) summed over a chunk of 256 k values stay exact in FP32 for g = 0 (2 real products
// per k: <= 2^23) and g = 1 (4 per k: <= 2^24).  Group 2 (3 pairs, 2^-16 of the result) and
// groups 3..4 (9 pairs, 2^-24) have accumulators of their own: the tensor cores align the
// products of an MMA to the largest term and drop the bits below its window, so small products
// must not share an accumulator with large ones.  Digit pairs with i + j >= 5 (below 2^-40) are
// dropped.  Chunk sums are added into a float-float (hi, lo) running sum per output element, so
// the result carries ~2^-40 relative to the product of the row maxima, like an FP64 GEMM whose
// inputs were rounded to 40 bits.
//
// Kernel k_tc_zgemm_x: tile 128 (n, TMEM lanes) x 64 (m, TMEM columns), pair-major order inside
// each 256-deep chunk, groups in order: each group's accumulator is drained by the epilogue while
// the later groups of the chunk run, and the last group (9 pairs) while the next chunk's first
// three groups run.  TMEM: g0 | g1 | g2 | g34, each Cr (64) | Ci (64) = 512 columns.
// Tiles of 128 x 128 (MMA N = 128: 64-wide tiles run the tensor pipe at about half rate).  The
// four accumulator groups share two TMEM slots of (re, im) x 128 columns in turn.  Warp 0: TMA
// producer; warp 1: MMA issuer; warps 2..17: epilogue (TMEM lane quarter warp % 4, 32 columns
// each), keeping the float-float sums of the tile in a per-CTA global buffer between chunks and
// writing C (alpha, beta in FP64) after the last chunk.
namespace x {
constexpr int NS = 5;                             // digits (slices) per operand
constexpr int BN = 128;                           // MMA N = m rows per tile
constexpr int STAGES = 3;
constexpr int A_PLANE = BM * BK * 2;              // 16 KB
constexpr int B_PLANE = BN * BK * 2;              // 16 KB
constexpr int STAGE_BYTES = 2 * A_PLANE + 2 * B_PLANE;
constexpr int RING_BYTES = STAGES * STAGE_BYTES;
constexpr int CK = 4;                             // k-blocks per chunk (256 K values)
constexpr int EPI_WARPS = 16;
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int THREADS = 64 + EPI_THREADS;
constexpr int COLS = BN / 4;                      // columns of one epilogue thread
constexpr int SMEM_BYTES = RING_BYTES + 256 /*barriers*/ + BN * 8 /*row offsets*/ + 1024 /*align*/;
constexpr int NSLOT = 2;                          // TMEM accumulator slots, (re, im) x BN columns each
constexpr int TMEM_COLS = NSLOT * 2 * BN;
constexpr int MAX_PAIRS = 15;
constexpr int NG = 4;                             // accumulator groups
}  // namespace x

// Digit pairs sorted by accumulator group, and the schedule of the two TMEM slots: the groups
// present take the slots in turn (group order), so before its first pair of a chunk a group waits
// for the drain of the slot's previous user: the group two places earlier in the same chunk, or
// the slot's last user in the previous chunk.
struct PairsX {
  int n;
  int sa[x::MAX_PAIRS], sb[x::MAX_PAIRS], grp[x::MAX_PAIRS];
  int first[x::NG], last[x::NG];   // first / last pair index of each group (-1: group absent)
  int slot[x::NG];                 // TMEM slot of each present group
  int wait_grp[x::NG];             // group whose drain frees the slot
  int wait_same[x::NG];            // 1: that drain belongs to the same chunk, 0: to the previous one
};

// OR of q over the epilogue threads of k_tc_zgemm_x (named barrier 1)
__device__ __forceinline__ bool group_any_x(bool q) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, 512, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)q)
      : "memory");
  return r != 0;
}
static_assert(x::EPI_THREADS == 512, "group_any_x counts 512 epilogue threads");

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// s + e = a + b exactly (Knuth's TwoSum; round-to-nearest FP32)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}
// (H, L) += (h, l), float-float addition with renormalisation
__device__ __forceinline__ void ff_add(float& H, float& L, float h, float l) {
  float s, e;
  two_sum(H, h, s, e);
  e = __fadd_rn(e, __fadd_rn(L, l));
  H = __fadd_rn(s, e);
  L = __fsub_rn(e, __fsub_rn(H, s));
}

__global__ void __launch_bounds__(x::THREADS, 1)
    k_tc_zgemm_x(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int n_rows, int m_rows,
                 int kblocks, int kb_per, PairsX pairs, double2 alpha, float alpha_pow2, double2 beta,
                 double2* __restrict__ C, int64_t ldc, int64_t cz, int* __restrict__ err, int xtiles, int ytiles,
                 int nsplit, const OutMap om, bool strided, float2* __restrict__ fstate) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + x::RING_BYTES);
  uint64_t* empty = full + x::STAGES;
  uint64_t* gfull = empty + x::STAGES;   // chunk sums of group g ready (MMA commit)
  uint64_t* gempty = gfull + x::NG;      // the slot of group g drained (all epilogue threads)
  uint64_t* done = gempty + x::NG;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int64_t* moff = (int64_t*)(smem + x::RING_BYTES + 256);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < x::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < x::NG; ++b) {
      mbar_init(&gfull[b], 1);
      mbar_init(&gempty[b], x::EPI_THREADS);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(x::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int xy = xtiles * ytiles;
  const int ntiles = xy * nsplit;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: per chunk, the pairs in order, each over the chunk's k-blocks
      int g = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        const int z = t / xy, r = t - z * xy, y = r / xtiles, xx = r - y * xtiles;
        const int kb0 = z * kb_per, kb1 = min(kblocks, kb0 + kb_per);
        const int n0 = y * BM, m0 = xx * x::BN;
        for (int c0 = kb0; c0 < kb1 && !stop; c0 += x::CK) {
          const int c1 = min(kb1, c0 + x::CK);
          for (int p = 0; p < pairs.n && !stop; ++p)
            for (int kb = c0; kb < c1; ++kb, ++g) {
              const int s = g % x::STAGES;
              const uint32_t ph = (uint32_t)(g / x::STAGES) & 1u;
              if (!mbar_wait(&empty[s], ph ^ 1u)) { atomicExch(err, 11); *abort_flag = 1; stop = true; break; }
              if (*abort_flag) { stop = true; break; }
              uint8_t* st = smem + s * x::STAGE_BYTES;
              mbar_expect_tx(&full[s], x::STAGE_BYTES);
              tma_load_3d(st, &tmA, kb * BK, n0, 2 * pairs.sa[p] + 0, &full[s]);
              tma_load_3d(st + x::A_PLANE, &tmA, kb * BK, n0, 2 * pairs.sa[p] + 1, &full[s]);
              tma_load_3d(st + 2 * x::A_PLANE, &tmB, kb * BK, m0, 2 * pairs.sb[p] + 0, &full[s]);
              tma_load_3d(st + 2 * x::A_PLANE + x::B_PLANE, &tmB, kb * BK, m0, 2 * pairs.sb[p] + 1, &full[s]);
            }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer (single thread)
      constexpr uint32_t ID = idesc_bf16(BM, x::BN, false), IDN = idesc_bf16(BM, x::BN, true);
      int g = 0, cc = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok && !*abort_flag; t += gridDim.x) {
        const int z = t / xy;
        const int kb0 = z * kb_per, kb1 = min(kblocks, kb0 + kb_per);
        for (int c0 = kb0; c0 < kb1 && ok; c0 += x::CK, ++cc) {
          const int c1 = min(kb1, c0 + x::CK);
          for (int p = 0; p < pairs.n && ok; ++p) {
            const int grp = pairs.grp[p];
            if (p == pairs.first[grp]) {
              // the slot of this group must have been drained by its previous user
              const uint32_t par = ((uint32_t)cc & 1u) ^ (pairs.wait_same[grp] ? 0u : 1u);
              if (!mbar_wait(&gempty[pairs.wait_grp[grp]], par)) { atomicExch(err, 14); *abort_flag = 1; ok = false; break; }
              fence_after();
            }
            const uint32_t cr = tmem + (uint32_t)pairs.slot[grp] * 2 * x::BN, ci = cr + x::BN;
            for (int kb = c0; kb < c1; ++kb, ++g) {
              const int s = g % x::STAGES;
              const uint32_t ph = (uint32_t)(g / x::STAGES) & 1u;
              if (!mbar_wait(&full[s], ph)) { atomicExch(err, 12); *abort_flag = 1; ok = false; break; }
              fence_after();
              const uint32_t base = smem_u32(smem + s * x::STAGE_BYTES);
              const uint32_t ar = base, ai = base + x::A_PLANE, br = base + 2 * x::A_PLANE, bi = br + x::B_PLANE;
#pragma unroll
              for (int ks = 0; ks < BK / 16; ++ks) {
                const uint32_t off = ks * 32;
                const uint64_t dar = desc_sw128(ar + off), dai = desc_sw128(ai + off);
                const uint64_t dbr = desc_sw128(br + off), dbi = desc_sw128(bi + off);
                const uint32_t first = (kb == c0 && ks == 0 && p == pairs.first[grp]) ? 0u : 1u;
                mma_bf16(cr, dar, dbr, ID, first);
                mma_bf16(cr, dai, dbi, IDN, 1u);
                mma_bf16(ci, dar, dbi, ID, first);
                mma_bf16(ci, dai, dbr, ID, 1u);
              }
              mma_commit(&empty[s]);
            }
            if (ok && p == pairs.last[grp]) mma_commit(&gfull[grp]);
          }
        }
      }
      mma_commit(done);
    }
  } else {
    // ---------------- epilogue warps 2..17: TMEM lane quarter warp % 4 (rows n0 + 32 (warp % 4) ..),
    // columns COLS ch .. COLS ch + COLS - 1, ch = (warp - 2) / 4.  Per chunk the exact sums of
    // groups 0 and 1 are added to the running float-float sums (each drained as soon as it is
    // complete), and the FP32 sums of groups 2 and 3..4 (~2^-16 and ~2^-24 of the result) to
    // their low words.  The running sums of the CTA's tile live in its slice of fstate,
    // [hi | lo][col][row] float2 (re, im): a warp's 32 rows are contiguous, and every element is
    // touched by one thread only.
    const int et = threadIdx.x - 64;
    const int lg = warp & 3;
    const int ch = (warp - 2) >> 2;
    const int row = lg * 32 + lane;                       // TMEM lane = n - n0
    const uint32_t lane_base = (uint32_t)(lg * 32) << 16;
    const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
    const bool beta_one = (beta.x == 1.0 && beta.y == 0.0);
    float2* hi = fstate + (size_t)blockIdx.x * 2 * BM * x::BN + row;   // element (col, row) at hi[col * BM]
    float2* lo = hi + BM * x::BN;
    const bool has1 = pairs.first[1] >= 0;
    const uint32_t s0 = tmem + lane_base + (uint32_t)pairs.slot[0] * 2 * x::BN + x::COLS * ch;
    const uint32_t s1 = tmem + lane_base + (uint32_t)(has1 ? pairs.slot[1] : 0) * 2 * x::BN + x::COLS * ch;
    int cc = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      const int z = t / xy, r = t - z * xy, y = r / xtiles, xx = r - y * xtiles;
      const int kb0 = z * kb_per, kb1 = min(kblocks, kb0 + kb_per);
      const int n0 = y * BM, m0 = xx * x::BN;
      const int nch = (kb1 - kb0 + x::CK - 1) / x::CK;
      double2* Cz = C + (int64_t)z * cz;
      if (group_any_x(false)) break;   // the previous tile's row offsets are no longer read
      if (strided && et < x::BN) {
        const int m = m0 + et;
        moff[et] = m < m_rows ? out_off((uint32_t)m, om.nm, om.mdim, om.mstr, om.mmul, om.mshr) : 0;
      }
      if (group_any_x(*abort_flag != 0)) break;   // also publishes this tile's offsets
      const int n = n0 + row;
      const int64_t noff = (strided && n < n_rows) ? out_off((uint32_t)n, om.nn, om.ndim, om.nstr, om.nmul, om.nshr) : 0;
      for (int ci = 0; ci < nch; ++ci, ++cc) {
        const uint32_t cpar = (uint32_t)cc & 1u;
        const bool firstc = ci == 0;
        // groups 0 and 1 one after the other, each an exact chunk sum added to the float-float
        // sums (group 0's slot is free for group 2 while group 1 still runs)
        for (int gx = 0; gx < 2; ++gx) {
          if (gx == 1 && !has1) break;   // same for every thread
          const bool ready = mbar_wait(&gfull[gx], cpar);
          if (group_any_x(!ready)) { if (et == 0) atomicExch(err, 13); *abort_flag = 1; stop = true; break; }
          fence_after();
          const uint32_t sb = gx == 0 ? s0 : s1;
#pragma unroll 2
          for (int q = 0; q < x::COLS / 8; ++q) {
            uint32_t a_re[8], a_im[8];
            tmem_ld8(sb + 8 * q, a_re);
            tmem_ld8(sb + x::BN + 8 * q, a_im);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int col = x::COLS * ch + 8 * q + j;
              if (firstc && gx == 0) {
                hi[col * BM] = make_float2(__uint_as_float(a_re[j]), __uint_as_float(a_im[j]));
                lo[col * BM] = make_float2(0.0f, 0.0f);
              }
            }
            if (!(firstc && gx == 0)) {
              // all eight columns' running sums are loaded before any is stored, so that the
              // loads (L2 hits) overlap instead of waiting behind the stores of earlier columns
              float2 h[8], l[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int col = x::COLS * ch + 8 * q + j;
                h[j] = hi[col * BM];
                l[j] = lo[col * BM];
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int col = x::COLS * ch + 8 * q + j;
                ff_add(h[j].x, l[j].x, __uint_as_float(a_re[j]), 0.0f);
                ff_add(h[j].y, l[j].y, __uint_as_float(a_im[j]), 0.0f);
                hi[col * BM] = h[j];
                lo[col * BM] = l[j];
              }
            }
          }
          fence_before();
          mbar_arrive(&gempty[gx]);
        }
        if (stop) break;
        for (int gq = 2; gq < x::NG; ++gq) {
          if (pairs.first[gq] < 0) continue;   // group absent (same for every thread)
          const bool ready = mbar_wait(&gfull[gq], cpar);
          if (group_any_x(!ready)) { if (et == 0) atomicExch(err, 13); *abort_flag = 1; stop = true; break; }
          fence_after();
          const uint32_t gbase = tmem + lane_base + (uint32_t)pairs.slot[gq] * 2 * x::BN + x::COLS * ch;
#pragma unroll 2
          for (int q = 0; q < x::COLS / 8; ++q) {
            uint32_t q_re[8], q_im[8];
            float2 l8[8];
            tmem_ld8(gbase + 8 * q, q_re);
            tmem_ld8(gbase + x::BN + 8 * q, q_im);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int col = x::COLS * ch + 8 * q + j;
              l8[j] = lo[col * BM];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int col = x::COLS * ch + 8 * q + j;
              l8[j].x = __fadd_rn(l8[j].x, __uint_as_float(q_re[j]));
              l8[j].y = __fadd_rn(l8[j].y, __uint_as_float(q_im[j]));
              lo[col * BM] = l8[j];
            }
          }
          fence_before();
          mbar_arrive(&gempty[gq]);
        }
        if (stop) break;
      }
      if (stop) break;
      // C = alpha (hi + lo) + beta C in FP64 (a split without k-blocks contributes zero)
#pragma unroll 4
      for (int j = 0; j < x::COLS; ++j) {
        const int col = x::COLS * ch + j;
        const int m = m0 + col;
        if (n < n_rows && m < m_rows) {
          const float2 h = nch > 0 ? hi[col * BM] : make_float2(0.0f, 0.0f);
          const float2 l = nch > 0 ? lo[col * BM] : make_float2(0.0f, 0.0f);
          double2 v;
          if (alpha_pow2 != 0.0f) {   // real power-of-two alpha: exact FP32 scaling
            v = make_double2(epi_f2d(h.x * alpha_pow2) + epi_f2d(l.x * alpha_pow2),
                             epi_f2d(h.y * alpha_pow2) + epi_f2d(l.y * alpha_pow2));
          } else {
            const double cr_ = epi_f2d(h.x) + epi_f2d(l.x), ci_ = epi_f2d(h.y) + epi_f2d(l.y);
            v = make_double2(alpha.x * cr_ - alpha.y * ci_, alpha.x * ci_ + alpha.y * cr_);
          }
          double2* dst = strided ? Cz + moff[col] + noff : Cz + (int64_t)m * ldc + n;
          if (use_beta) {
            const double2 o = *dst;
            if (beta_one) {
              v.x += o.x;
              v.y += o.y;
            } else {
              v.x += beta.x * o.x - beta.y * o.y;
              v.y += beta.x * o.y + beta.y * o.x;
            }
          }
          *dst = v;
        }
      }
    }
  }
  __syncwarp();
  fence_before();
  __syncthreads();
  if (warp == 2) {
    fence_after();
    if (!mbar_wait(done, 0) && lane == 0) atomicExch(err, 15);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(x::TMEM_COLS));
  }
}

// Largest biased binary64 exponent of |re| and |im| over each operand row (the row exponent of
// the fixed-point digits is that value - 1022, so that |x| < 2^e).  rexp is zeroed beforehand.
__device__ __forceinline__ uint32_t bexp64(double v) { return (uint32_t)((uint64_t)__double_as_longlong(v) >> 52) & 0x7ffu; }

// Signed base-256 digits of x on the grid of a row whose largest biased exponent is eb_row: the
// fixed-point integer X = round(x / 2^(eb_row - 1061)) (|X| <= 2^39; subnormal x counts as 0)
// is written as X = sum_s d_s 2^(32 - 8 s) with d_0 in [-128, 128] and d_1..d_4 in [-128, 127],
// read from the bytes of U = X + kDigitOffset (>= 0): kDigitOffset holds 128 in each of the five
// digit positions, so the low four bytes of U are d_4..d_1 + 128 and U >> 32 is d_0 + 128.
// Returns U (integer pipe only).
constexpr int64_t kDigitOffset = 0x8080808080ll;
__device__ __forceinline__ uint64_t ozaki_offset(double v, uint32_t eb_row) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const uint32_t eb = (uint32_t)(b >> 52) & 0x7ffu;
  int64_t X = 0;
  if (eb != 0u) {
    const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int rs = (int)eb_row - (int)eb + 14;   // >= 14: x / 2^(e - 39) = M 2^-rs
    if (rs < 64) X = (int64_t)((M + (1ull << (rs - 1))) >> rs);
    if (b >> 63) X = -X;
  }
  return (uint64_t)(X + kDigitOffset);
}
// d_s + 128 from U
__device__ __forceinline__ uint32_t ozaki_byte(uint64_t U, int s) {
  return s == 0 ? (uint32_t)(U >> 32) : ((uint32_t)U >> (32 - 8 * s)) & 0xffu;
}
// BF16 bits of d 2^p (|d| <= 256, exact); values below the BF16 normal range flush to zero
__device__ __forceinline__ uint32_t bf16_digit(int d, int p) {
  if (d == 0) return 0u;
  const uint32_t a = (uint32_t)(d < 0 ? -d : d);
  const int msb = 31 - __clz(a);
  const int be = msb + p + 127;
  if (be <= 0) return 0u;
  const uint32_t sign = d < 0 ? 0x8000u : 0u;
  if (be >= 255) return sign | 0x7f80u;   // beyond the binary32 range: infinity
  const uint32_t frac = (a << (7 - msb)) & 0x7fu;
  return sign | ((uint32_t)be << 7) | frac;
}
// binary32 bits of (byte - 128) 2^p for a row whose digit scales are normal binary32 numbers:
// 2^23 + byte is exact in binary32 (exponent-bias construction), the subtraction of 2^23 + 128 is
// exact, and so is the power-of-two scaling (overflow gives infinity, as bf16_digit).  Its top
// 16 bits are the BF16 digit (at most 8 significant bits).
__device__ __forceinline__ uint32_t digit_f32_bits(uint32_t byte, float scale) {
  return __float_as_uint(__fmul_rn(__fsub_rn(__uint_as_float(0x4B000000u | byte), 8388736.0f), scale));
}
// the digit planes of one element pair (k, k+1) of a row: out32[plane] = bf16(k) | bf16(k+1) << 16
// (only the first nd digit planes are formed: the rest are zero on coarse operands and never read)
__device__ __forceinline__ void ozaki_pair(const double2 (&xv)[2], uint32_t eb_row, uint32_t (&out)[2 * x::NS], int nd) {
  if (eb_row == 0x7ffu) {   // infinity or NaN in the row: propagate NaN
#pragma unroll
    for (int q = 0; q < 2 * x::NS; ++q) out[q] = 0x7fc07fc0u;
    return;
  }
  const uint64_t u[4] = {ozaki_offset(xv[0].x, eb_row), ozaki_offset(xv[0].y, eb_row),
                         ozaki_offset(xv[1].x, eb_row), ozaki_offset(xv[1].y, eb_row)};
  if (eb_row >= 935u && eb_row <= 1156u) {   // every 2^p_s, p_s = eb_row - 1029 - 8 s, a normal binary32
#pragma unroll
    for (int s = 0; s < x::NS; ++s) {
      if (s >= nd) break;
      const float scale = __uint_as_float((uint32_t)((int)eb_row - 1029 - 8 * s + 127) << 23);
      uint32_t f[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) f[t] = digit_f32_bits(ozaki_byte(u[t], s), scale);
      out[2 * s + 0] = __byte_perm(f[0], f[2], 0x7632);   // top halves: bf16(k) | bf16(k+1) << 16
      out[2 * s + 1] = __byte_perm(f[1], f[3], 0x7632);
    }
    return;
  }
#pragma unroll
  for (int s = 0; s < x::NS; ++s) {
    if (s >= nd) break;
    const int p = (int)eb_row - 1029 - 8 * s;
    uint32_t h[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) h[t] = bf16_digit((int)ozaki_byte(u[t], s) - 128, p);
    out[2 * s + 0] = h[0] | (h[2] << 16);
    out[2 * s + 1] = h[1] | (h[3] << 16);
  }
}

// Strided complex FP64 view -> BF16 slice planes [slice][re|im][rows][Kpad].  The view is given
// as up to 8 axes, the first nr of which form the row index and the rest the K index (row-major
// order within each group), so any permutation of a tensor is split in one pass.  Index decoding
// divides by the axis extents with Granlund-Montgomery multipliers (q = (umulhi(n, m) + n) >> l,
// exact for 32-bit n).
struct ViewArgs {
  int rank, nr;
  int64_t dim[kMaxRank];
  int64_t str[kMaxRank];
  uint32_t mul[kMaxRank];
  int shr[kMaxRank];
};

__device__ __forceinline__ int64_t view_off(const ViewArgs& v, int a0, int a1, uint32_t i) {
  int64_t off = 0;
#pragma unroll
  for (int a = kMaxRank - 1; a >= 0; --a) {
    if (a < a0 || a >= a1) continue;
    const uint32_t q = (uint32_t)(((uint64_t)__umulhi(i, v.mul[a]) + i) >> v.shr[a]);
    off += (int64_t)(i - q * (uint32_t)v.dim[a]) * v.str[a];
    i = q;
  }
  return off;
}

// IEEE 754 binary64 -> binary32 on the integer pipe (round to nearest, ties away from zero;
// results below the binary32 normal range flush to zero).  The FP64 <-> FP32 cvt instructions
// issue on the FP64 pipe, about 1/64 of the FP32 rate on sm_103.
__device__ __forceinline__ float split_d2f(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
  const uint32_t t = __funnelshift_l(lo, hi, 3) + ((lo >> 28) & 1u);
  uint32_t f = (t - 0xC0000000u) | sign;   // rebias 1023 -> 127 (896; low 9 bits 0x180)
  if (e < 897u) f = sign;
  if (e > 1150u) f = sign | ((e == 0x7ffu && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u);
  return __uint_as_float(f);
}
// bfloat16 = the top 16 bits of a binary32, rounded to nearest even
__device__ __forceinline__ uint32_t bf16_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}

// Work items are (row, chunk of 64 element pairs), strided over all warps of the grid, so that
// operands with few long rows and with many short rows both fill the GPU; each lane converts
// pairs of consecutive K elements and stores them as packed bf16x2.  x is rounded to FP32
// (24 bits) and cut into slices s_0 + s_1 + s_2 in FP32 arithmetic (each difference is exact).
constexpr int kSplitPairs = 64;
// With rexp (the FP64-class mode) each pair is written as the row's five fixed-point digits instead.
__global__ void __launch_bounds__(256) k_split_view(const double2* __restrict__ X, ViewArgs v, int64_t rows, int64_t K,
                                                    bool conj, int nsl, __nv_bfloat16* __restrict__ out, int64_t Kpad,
                                                    uint32_t nchunk, uint32_t chunk_mul, int chunk_shr,
                                                    const uint32_t* __restrict__ rexp, int nd) {
  const int64_t plane = rows * Kpad;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t* o32 = reinterpret_cast<uint32_t*>(out);
  const int64_t pairs = Kpad / 2;
  const int64_t items = rows * (int64_t)nchunk;
  for (int64_t w = warp0; w < items; w += nwarps) {
    const uint32_t wi = (uint32_t)w;
    const uint32_t r = (uint32_t)(((uint64_t)__umulhi(wi, chunk_mul) + wi) >> chunk_shr);
    const uint32_t c = wi - r * nchunk;
    const int64_t roff = view_off(v, 0, v.nr, r);
#pragma unroll
    for (int h = 0; h < kSplitPairs / 32; ++h) {
      const int64_t p = (int64_t)c * kSplitPairs + h * 32 + lane;
      if (p >= pairs) break;
      const int64_t e2 = (int64_t)r * (Kpad / 2) + p;   // index of the bf16 pair within a plane
      if (rexp) {
        double2 xv[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int64_t k = 2 * p + t;
          xv[t] = make_double2(0.0, 0.0);
          if (k < K) xv[t] = X[roff + view_off(v, v.nr, v.rank, (uint32_t)k)];
          if (conj) xv[t].y = -xv[t].y;
        }
        uint32_t o[2 * x::NS];
        ozaki_pair(xv, rexp[r], o, nd);
#pragma unroll
        for (int q = 0; q < 2 * x::NS; ++q)
          if (q < 2 * nd) o32[(q * plane) / 2 + e2] = o[q];   // zero digit planes are not read
        continue;
      }
      float re[2], im[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int64_t k = 2 * p + t;
        double2 x = make_double2(0.0, 0.0);
        if (k < K) x = X[roff + view_off(v, v.nr, v.rank, (uint32_t)k)];
        re[t] = split_d2f(x.x);
        im[t] = split_d2f(conj ? -x.y : x.y);
      }
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        if (s >= nsl) break;
        uint32_t br[2], bi[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          br[t] = bf16_bits(re[t]);
          bi[t] = bf16_bits(im[t]);
          re[t] -= __uint_as_float(br[t] << 16);
          im[t] -= __uint_as_float(bi[t] << 16);
        }
        o32[((2 * s + 0) * plane) / 2 + e2] = br[0] | (br[1] << 16);
        o32[((2 * s + 1) * plane) / 2 + e2] = bi[0] | (bi[1] << 16);
      }
    }
  }
}

// Transposing split, for views whose unit-stride index is a row index while the K index runs
// with a large stride (e.g. the ring-layout doubles contracted over (m, n, e)): a tile of 32
// consecutive values of the unit-stride row axis U x 64 K values is read into shared memory with
// loads contiguous along U, then written as BF16 slices contiguous along K.  Tiles are
// (other row indices, U chunk, K chunk), K chunk fastest.
struct SplitT {
  int u;                         // the unit-stride row axis of the view
  int64_t rstride[kMaxRank];     // row-index stride of every row axis in the [rows][Kpad] output
  uint32_t n_cu, n_ck;           // U chunks of 32, K chunks of 64
  uint32_t mul_cu, mul_ck;       // Granlund-Montgomery multipliers of n_cu, n_ck
  int shr_cu, shr_ck;
};

__global__ void __launch_bounds__(256) k_split_view_t(const double2* __restrict__ X, ViewArgs v, SplitT s,
                                                      int64_t rows, int64_t K, bool conj, int nsl,
                                                      __nv_bfloat16* __restrict__ out, int64_t Kpad, int64_t ntiles,
                                                      const uint32_t* __restrict__ rexp, int nd) {
  __shared__ double2 tile[64][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t plane = rows * Kpad;
  uint32_t* o32 = reinterpret_cast<uint32_t*>(out);
  const int64_t dimU = v.dim[s.u];
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint32_t r = (uint32_t)t;
    const uint32_t q1 = (uint32_t)(((uint64_t)__umulhi(r, s.mul_ck) + r) >> s.shr_ck);
    const uint32_t ck = r - q1 * s.n_ck;
    const uint32_t q2 = (uint32_t)(((uint64_t)__umulhi(q1, s.mul_cu) + q1) >> s.shr_cu);
    const uint32_t cu = q1 - q2 * s.n_cu;
    uint32_t o = q2;   // index over the row axes other than U (row-major)
    int64_t soff = 0, rbase = 0;
#pragma unroll
    for (int a = kMaxRank - 1; a >= 0; --a) {
      if (a >= v.nr || a == s.u) continue;
      const uint32_t q = (uint32_t)(((uint64_t)__umulhi(o, v.mul[a]) + o) >> v.shr[a]);
      const int64_t idx = (int64_t)(o - q * (uint32_t)v.dim[a]);
      soff += idx * v.str[a];
      rbase += idx * s.rstride[a];
      o = q;
    }
    const int64_t u0 = (int64_t)cu * 32, k0 = (int64_t)ck * 64;
    // read: lanes along U (unit stride), warps over K
    for (int kk = warp; kk < 64; kk += 8) {
      const int64_t k = k0 + kk;
      double2 x = make_double2(0.0, 0.0);
      if (k < K && u0 + lane < dimU) x = X[soff + (u0 + lane) + view_off(v, v.nr, v.rank, (uint32_t)k)];
      tile[kk][lane] = x;
    }
    __syncthreads();
    // write: warp w takes rows w, w+8, w+16, w+24 of the tile; lane p the K pair (2p, 2p+1)
    for (int j = warp; j < 32; j += 8) {
      if (u0 + j >= dimU) continue;
      const int64_t row = rbase + (u0 + j) * s.rstride[s.u];
      if (rexp) {
        double2 xv[2] = {tile[2 * lane][j], tile[2 * lane + 1][j]};
        if (conj) { xv[0].y = -xv[0].y; xv[1].y = -xv[1].y; }
        uint32_t o[2 * x::NS];
        ozaki_pair(xv, rexp[row], o, nd);
        const int64_t e2 = row * (Kpad / 2) + (k0 / 2) + lane;
#pragma unroll
        for (int q = 0; q < 2 * x::NS; ++q)
          if (q < 2 * nd) o32[(q * plane) / 2 + e2] = o[q];   // zero digit planes are not read
        continue;
      }
      float re[2], im[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const double2 x = tile[2 * lane + e][j];
        re[e] = split_d2f(x.x);
        im[e] = split_d2f(conj ? -x.y : x.y);
      }
      const int64_t e2 = row * (Kpad / 2) + (k0 / 2) + lane;
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) {
        if (sl >= nsl) break;
        uint32_t br[2], bi[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          br[e] = bf16_bits(re[e]);
          bi[e] = bf16_bits(im[e]);
          re[e] -= __uint_as_float(br[e] << 16);
          im[e] -= __uint_as_float(bi[e] << 16);
        }
        o32[((2 * sl + 0) * plane) / 2 + e2] = br[0] | (br[1] << 16);
        o32[((2 * sl + 1) * plane) / 2 + e2] = bi[0] | (bi[1] << 16);
      }
    }
    __syncthreads();
  }
}

// Row exponents of the FP64-class digits: rexp[r] = largest biased binary64 exponent of |re| and
// |im| over row r of the view (rexp zeroed beforehand; atomicMax per warp).  Same work items as
// k_split_view.
__global__ void __launch_bounds__(256) k_rowexp(const double2* __restrict__ X, ViewArgs v, int64_t rows, int64_t K,
                                                uint32_t nchunk, uint32_t chunk_mul, int chunk_shr,
                                                uint32_t* __restrict__ rexp) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t items = rows * (int64_t)nchunk;
  for (int64_t w = warp0; w < items; w += nwarps) {
    const uint32_t wi = (uint32_t)w;
    const uint32_t r = (uint32_t)(((uint64_t)__umulhi(wi, chunk_mul) + wi) >> chunk_shr);
    const uint32_t c = wi - r * nchunk;
    const int64_t roff = view_off(v, 0, v.nr, r);
    uint32_t m = 0;
    for (int h = 0; h < 2 * kSplitPairs / 32; ++h) {
      const int64_t k = (int64_t)c * 2 * kSplitPairs + h * 32 + lane;
      if (k < K) {
        const double2 xv = X[roff + view_off(v, v.nr, v.rank, (uint32_t)k)];
        m = max(m, max(bexp64(xv.x), bexp64(xv.y)));
      }
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0 && m) atomicMax(&rexp[r], m);
  }
}

// Row exponents for the transposing split's views (same tiles as k_split_view_t).
__global__ void __launch_bounds__(256) k_rowexp_t(const double2* __restrict__ X, ViewArgs v, SplitT s, int64_t K,
                                                  int64_t ntiles, uint32_t* __restrict__ rexp) {
  __shared__ uint32_t red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t dimU = v.dim[s.u];
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint32_t r = (uint32_t)t;
    const uint32_t q1 = (uint32_t)(((uint64_t)__umulhi(r, s.mul_ck) + r) >> s.shr_ck);
    const uint32_t ck = r - q1 * s.n_ck;
    const uint32_t q2 = (uint32_t)(((uint64_t)__umulhi(q1, s.mul_cu) + q1) >> s.shr_cu);
    const uint32_t cu = q1 - q2 * s.n_cu;
    uint32_t o = q2;
    int64_t soff = 0, rbase = 0;
#pragma unroll
    for (int a = kMaxRank - 1; a >= 0; --a) {
      if (a >= v.nr || a == s.u) continue;
      const uint32_t q = (uint32_t)(((uint64_t)__umulhi(o, v.mul[a]) + o) >> v.shr[a]);
      const int64_t idx = (int64_t)(o - q * (uint32_t)v.dim[a]);
      soff += idx * v.str[a];
      rbase += idx * s.rstride[a];
      o = q;
    }
    const int64_t u0 = (int64_t)cu * 32, k0 = (int64_t)ck * 64;
    if (threadIdx.x < 32) red[threadIdx.x] = 0;
    __syncthreads();
    uint32_t m = 0;
    for (int kk = warp; kk < 64; kk += 8) {
      const int64_t k = k0 + kk;
      if (k < K && u0 + lane < dimU) {
        const double2 xv = X[soff + (u0 + lane) + view_off(v, v.nr, v.rank, (uint32_t)k)];
        m = max(m, max(bexp64(xv.x), bexp64(xv.y)));
      }
    }
    if (m) atomicMax(&red[lane], m);
    __syncthreads();
    if (threadIdx.x < 32 && u0 + threadIdx.x < dimU && red[threadIdx.x])
      atomicMax(&rexp[rbase + (u0 + threadIdx.x) * s.rstride[s.u]], red[threadIdx.x]);
    __syncthreads();
  }
}

}  // namespace tc

namespace {

// The tensor-map encoder lives in the driver library; resolve it through the runtime so that
// libcclr loads (and its CPU-side checks run) on machines without a GPU driver.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    CCLR_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    CCLR_REQUIRE(p && q == cudaDriverEntryPointSuccess, CCLR_E_CUDA, "cuTensorMapEncodeTiled not available");
    fn = (EncodeTiledFn)p;
  }
  return fn;
}

CUtensorMap make_map(const __nv_bfloat16* p, int64_t rows, int64_t Kpad, int nplanes, int box_rows) {
  CUtensorMap tm;
  cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)(Kpad * 2), (cuuint64_t)(rows * Kpad * 2)};
  cuuint32_t box[3] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_tiled()(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)p, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CCLR_REQUIRE(r == CUDA_SUCCESS, CCLR_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return tm;
}

// BF16 slices of one GEMM operand (rows x K, zero-padded to Kpad) with its TMA descriptor
struct Slices {
  __nv_bfloat16* p = nullptr;
  int64_t rows = 0, K = 0, Kpad = 0;
  int nsl = 0;
  int ndig = 0;   // FP64-class digits that can be nonzero (2 for operands on a coarse grid)
  CUtensorMap tm;
};

}  // namespace

// Per-context state of the tensor-core path: the slice cache of persistent operands, the memos of
// transient operands, the coarse operand ranges and the autotuner's timed launches.
struct CacheEntry {
  Slices s;
  uint64_t gen = 0;    // data generation of the last use
  bool integral = false;
};
struct Memo {
  const void* src = nullptr;
  char* base = nullptr;
  size_t cap = 0, used = 0;
  std::vector<std::pair<std::string, Slices>> entries;
};
struct TunePending {
  std::string key;
  int cfg;
  cudaEvent_t a, b;
};
struct TcState {
  std::map<std::string, CacheEntry> cache;
  uint64_t cache_gen = 0;
  std::vector<Memo> memos;
  std::vector<std::pair<const char*, const char*>> coarse;   // device ranges on a coarse grid
  std::vector<TunePending> pending;
};
TcState& tcs(Ctx& c) {
  if (!c.tcs) c.tcs = new TcState();
  return *c.tcs;
}

namespace {

// Device ranges whose values lie on a coarse fixed-point grid (CoarseOperands): their FP64-class
// digits beyond the second are zero.
bool is_coarse(Ctx& c, const void* p) {
  const char* q = (const char*)p;
  for (auto& r : tcs(c).coarse)
    if (q >= r.first && q < r.second) return true;
  return false;
}

// Slices of persistent operands (integrals, Hbar, amplitudes) are kept keyed by pointer and view
// layout.  Those of the integrals live until the Hamiltonian changes; the others for one
// generation of the context's data (bumped whenever amplitudes, Lambda or Hbar change).  When the
// cache is full, integral slices not read in the current generation are evicted, largest first.
size_t entry_bytes(const CacheEntry& e) { return sizeof(__nv_bfloat16) * 2 * e.s.nsl * e.s.rows * e.s.Kpad; }

// View arguments of the split kernel: axes of extent 1 dropped, neighbours that are contiguous
// in memory merged (within the row group and within the K group), division multipliers set.
tc::ViewArgs view_args(const Tensor& v, int nr) {
  std::vector<int64_t> d[2], st[2];
  for (int i = 0; i < v.rank; ++i) {
    const int g = i < nr ? 0 : 1;
    if (v.dim[i] == 1) continue;
    if (!d[g].empty() && st[g].back() == v.dim[i] * v.str[i]) {
      d[g].back() *= v.dim[i];
      st[g].back() = v.str[i];
    } else {
      d[g].push_back(v.dim[i]);
      st[g].push_back(v.str[i]);
    }
  }
  for (int g = 0; g < 2; ++g)
    if (d[g].empty()) { d[g].push_back(1); st[g].push_back(0); }
  tc::ViewArgs a{};
  a.nr = (int)d[0].size();
  a.rank = a.nr + (int)d[1].size();
  for (int i = 0; i < a.rank; ++i) {
    const int g = i < a.nr ? 0 : 1, j = i < a.nr ? i : i - a.nr;
    const int64_t dim = d[g][j];
    CCLR_REQUIRE(dim >= 1 && dim < (int64_t(1) << 31), CCLR_E_ARG, "tensor-core split: axis extent too large");
    int l = 0;
    while ((int64_t(1) << l) < dim) ++l;
    a.dim[i] = dim;
    a.str[i] = st[g][j];
    a.shr[i] = l;
    a.mul[i] = (uint32_t)(((unsigned __int128)1 << 32) * (((uint64_t)1 << l) - (uint64_t)dim) / (uint64_t)dim + 1);
  }
  return a;
}

// rexp != nullptr: the FP64-class digits (nsl = 5); rexp holds `rows` words of scratch on the stream's device
// nd: digit planes written in digit mode (2 for operands on the coarse grid, whose higher digits
// are zero and never read; else all five)
void launch_split(const Tensor& v, int nr, int64_t rows, int64_t K, int64_t Kpad, int nsl, __nv_bfloat16* dst,
                  cudaStream_t stream, uint32_t* rexp = nullptr, int nd = tc::x::NS) {
  CCLR_REQUIRE(rows < (int64_t(1) << 31) && K < (int64_t(1) << 31), CCLR_E_ARG, "tensor-core split: operand too large");
  CCLR_REQUIRE(!rexp || nsl == tc::x::NS, CCLR_E_ARG, "tensor-core split: digit count");
  const tc::ViewArgs a = view_args(v, nr);
  const int sms = num_sms();
  if (rexp) CCLR_CK(cudaMemsetAsync(rexp, 0, sizeof(uint32_t) * (size_t)rows, stream));
  // transposing variant: a row axis has unit stride while the innermost K axis does not
  int u = -1;
  for (int i = 0; i < a.nr; ++i)
    if (a.str[i] == 1 && a.dim[i] >= 16) u = i;
  if (u >= 0 && a.str[a.rank - 1] != 1) {
    tc::SplitT st{};
    st.u = u;
    int64_t rs = 1;
    for (int i = a.nr - 1; i >= 0; --i) {
      st.rstride[i] = rs;
      rs *= a.dim[i];
    }
    const int64_t n_other = rows / a.dim[u];
    const int64_t n_cu = (a.dim[u] + 31) / 32, n_ck = Kpad / 64;
    const int64_t ntiles = n_other * n_cu * n_ck;
    CCLR_REQUIRE(ntiles < (int64_t(1) << 32), CCLR_E_ARG, "tensor-core split: operand too large");
    auto magic = [](int64_t d, uint32_t& mul, int& shr) {
      int l = 0;
      while ((int64_t(1) << l) < d) ++l;
      shr = l;
      mul = (uint32_t)(((unsigned __int128)1 << 32) * (((uint64_t)1 << l) - (uint64_t)d) / (uint64_t)d + 1);
    };
    st.n_cu = (uint32_t)n_cu;
    st.n_ck = (uint32_t)n_ck;
    magic(n_cu, st.mul_cu, st.shr_cu);
    magic(n_ck, st.mul_ck, st.shr_ck);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sms * 8));
    if (rexp) tc::k_rowexp_t<<<g, 256, 0, stream>>>(v.p, a, st, K, ntiles, rexp);
    tc::k_split_view_t<<<g, 256, 0, stream>>>(v.p, a, st, rows, K, v.conj, nsl, dst, Kpad, ntiles, rexp, nd);
    return;
  }
  const int64_t nchunk = (Kpad / 2 + tc::kSplitPairs - 1) / tc::kSplitPairs;
  CCLR_REQUIRE(rows * nchunk < (int64_t(1) << 32), CCLR_E_ARG, "tensor-core split: operand too large");
  int l = 0;
  while ((int64_t(1) << l) < nchunk) ++l;
  const uint32_t mul = (uint32_t)(((unsigned __int128)1 << 32) * (((uint64_t)1 << l) - (uint64_t)nchunk) / (uint64_t)nchunk + 1);
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((rows * nchunk + 7) / 8, (int64_t)sms * 16));
  if (rexp) tc::k_rowexp<<<g, 256, 0, stream>>>(v.p, a, rows, K, (uint32_t)nchunk, mul, l, rexp);
  tc::k_split_view<<<g, 256, 0, stream>>>(v.p, a, rows, K, v.conj, nsl, dst, Kpad, (uint32_t)nchunk, mul, l, rexp, nd);
}

void make_slices(Ctx& c, const Tensor& v, int nr, int nsl, Slices& s, __nv_bfloat16* dst, int nd = tc::x::NS) {
  int64_t rows = 1, K = 1;
  for (int i = 0; i < v.rank; ++i) (i < nr ? rows : K) *= v.dim[i];
  s.rows = rows;
  s.K = K;
  s.Kpad = (K + tc::BK - 1) / tc::BK * tc::BK;
  s.nsl = nsl;
  s.p = dst;
  Scope sc(c.ws);
  uint32_t* rexp = nsl == tc::x::NS ? (uint32_t*)c.ws.alloc(sizeof(uint32_t) * (size_t)rows) : nullptr;
  c.kt.begin(c.stream);
  launch_split(v, nr, rows, K, s.Kpad, nsl, dst, c.stream, rexp, nd);
  CCLR_CK(cudaGetLastError());
  c.kt.end(c.stream, rexp ? "k_split_view(f64 digits)" : "k_split_view");
  c.launches += rexp ? 2 : 1;
  s.tm = make_map(dst, rows, s.Kpad, 2 * nsl, 128);
}

bool is_integral(const Ctx& c, const void* p) {
  const void* arr[] = {c.oooo, c.ooov, c.oovv, c.ovov, c.ovvv, c.vvvv_p, c.oovv_p, c.ovvv_p};
  for (const void* q : arr)
    if (q && q == p) return true;
  return false;
}

bool is_persistent(const Ctx& c, const void* p) {
  const void* arr[] = {c.Fae, c.Fmi, c.Fae_od, c.Fmi_od, c.Fme, c.Wmnij, c.Wmnij_p, c.Wabef_p, c.Wmbej, c.WringR, c.WringL, c.Wmnie,
                       c.Wamef, c.Wmbij, c.Wabei, c.tau, c.t2, c.l2, c.oooo, c.ooov, c.oovv, c.ovov, c.ovvv,
                       c.vvvv_p, c.oovv_p, c.ovvv_p, c.t, c.lam};
  for (const void* q : arr)
    if (q && q == p) return true;
  for (auto& kv : c.named)
    if (kv.second == p && kv.first.rfind("F.", 0) == 0 && kv.first != "F.ready") return true;
  return false;
}

// Slices of a transient operand that several contractions of one call read in the same view
// (the unpacked trial vectors of a sigma product: e.g. r_mn^ea over (m, n, e) for two singles
// terms) are split once.  A SliceMemo names the operand, which must not change while it is
// alive, and reserves workspace for its slices; memos nest.

// Slices of view v (first nr axes = rows): from the cache for persistent operands, from the memo
// of a transient operand named by a SliceMemo, else into the workspace.
Slices get_slices_any(Ctx& c, const Tensor& v, int nr, int nsl);
Slices get_slices(Ctx& c, const Tensor& v, int nr, int nsl) {
  Slices s = get_slices_any(c, v, nr, nsl);
  s.ndig = (nsl == tc::x::NS && is_coarse(c, v.p)) ? 2 : nsl;
  return s;
}
Slices get_slices_any(Ctx& c, const Tensor& v, int nr, int nsl) {
  // transient operands on the coarse grid get only their two nonzero digit planes written (the
  // persistent cache always holds all five)
  const int nd = (nsl == tc::x::NS && is_coarse(c, v.p)) ? 2 : tc::x::NS;
  TcState& T = tcs(c);
  auto& cache = T.cache;
  if (T.cache_gen != c.data_gen) {
    for (auto it = cache.begin(); it != cache.end();) {
      if (it->second.integral) {
        ++it;
        continue;
      }
      cudaFree(it->second.s.p);
      it = cache.erase(it);
    }
    T.cache_gen = c.data_gen;
  }
  int64_t elems = 1;
  for (int i = 0; i < v.rank; ++i) elems *= v.dim[i];
  int64_t K = 1;
  for (int i = nr; i < v.rank; ++i) K *= v.dim[i];
  const int64_t Kpad = (K + tc::BK - 1) / tc::BK * tc::BK;
  const size_t bytes = sizeof(__nv_bfloat16) * 2 * nsl * (size_t)(elems / K) * (size_t)Kpad;
  Slices s;
  static const double cap_gb = std::getenv("CCLR_TC_CACHE_GB") ? atof(std::getenv("CCLR_TC_CACHE_GB")) : 32.0;
  if (is_persistent(c, v.p)) {
    std::string key = std::to_string((uintptr_t)v.p) + "|" + std::to_string(nr) + "|" + std::to_string(nsl) + "|" +
                      std::to_string((int)v.conj);
    for (int i = 0; i < v.rank; ++i) key += "|" + std::to_string(v.dim[i]) + ":" + std::to_string(v.str[i]);
    auto it = cache.find(key);
    if (it != cache.end()) {
      it->second.gen = c.data_gen;
      return it->second.s;
    }
    const double cap = cap_gb * (double)(1ull << 30);
    size_t cached = tc_cache_bytes(c);
    while ((double)(cached + bytes) > cap) {   // evict the largest integral entry idle this generation
      auto victim = cache.end();
      for (auto e = cache.begin(); e != cache.end(); ++e)
        if (e->second.integral && e->second.gen != c.data_gen &&
            (victim == cache.end() || entry_bytes(e->second) > entry_bytes(victim->second)))
          victim = e;
      if (victim == cache.end()) break;
      cached -= entry_bytes(victim->second);
      cudaFree(victim->second.s.p);
      cache.erase(victim);
    }
    __nv_bfloat16* dst = nullptr;
    if ((double)(cached + bytes) <= cap && cudaMalloc((void**)&dst, bytes) == cudaSuccess) {
      make_slices(c, v, nr, nsl, s, dst);
      cache[key] = CacheEntry{s, c.data_gen, is_integral(c, v.p)};
      return s;
    }
    cudaGetLastError();  // out of memory for the cache: fall through to a workspace copy
  }
  for (auto it = T.memos.rbegin(); it != T.memos.rend(); ++it) {
    if (it->src != v.p) continue;
    std::string key = std::to_string(nr) + "|" + std::to_string(nsl) + "|" + std::to_string((int)v.conj);
    for (int i = 0; i < v.rank; ++i) key += "|" + std::to_string(v.dim[i]) + ":" + std::to_string(v.str[i]);
    for (auto& e : it->entries)
      if (e.first == key) return e.second;
    const size_t at = (it->used + 255) & ~size_t(255);
    if (at + bytes <= it->cap) {
      make_slices(c, v, nr, nsl, s, (__nv_bfloat16*)(it->base + at), nd);
      it->used = at + bytes;
      it->entries.push_back({key, s});
      return s;
    }
    break;
  }
  make_slices(c, v, nr, nsl, s, (__nv_bfloat16*)c.ws.alloc(bytes), nd);
  return s;
}

}  // namespace

CoarseOperands::CoarseOperands(Ctx& cc, std::initializer_list<std::pair<const void*, size_t>> ranges) : c(cc) {
  for (auto& r : ranges)
    if (r.first && r.second) {
      tcs(c).coarse.push_back({(const char*)r.first, (const char*)r.first + r.second});
      ++n;
    }
}
CoarseOperands::~CoarseOperands() {
  for (int i = 0; i < n; ++i) tcs(c).coarse.pop_back();
}

SliceMemo::SliceMemo(Ctx& cc, const void* src, int64_t elems, int views) : c(cc) {
  if (c.opt.precision == CCLR_FP64 || src == nullptr) return;
  // each view: nsl slices x (re, im) BF16 planes, K padded to a multiple of BK per row
  const size_t want = (size_t)views * 2 * sizeof(__nv_bfloat16) * (size_t)tc_slices(c.opt.precision) *
                      (size_t)((double)elems * 1.05 + 65536.0);
  const size_t avail = c.ws.cap > c.ws.top ? (c.ws.cap - c.ws.top) / 2 : 0;   // leave half for the call
  const size_t cap = std::min(want, avail);
  if (cap < ((size_t)1 << 20)) return;
  Memo m;
  m.src = src;
  m.base = (char*)c.ws.alloc(cap);
  m.cap = cap;
  tcs(c).memos.push_back(std::move(m));
  active = true;
}
SliceMemo::~SliceMemo() {
  if (active) tcs(c).memos.pop_back();
}

namespace {

// Digit pairs (i, j) with i + j < 5, i < nda (A-side digits), j < ndb (B-side digits), sorted by
// group: group i + j for i + j < 3, group 3 otherwise
tc::PairsX pairs_x(int nda = tc::x::NS, int ndb = tc::x::NS) {
  tc::PairsX p{};
  p.n = 0;
  for (int g = 0; g < tc::x::NS; ++g)
    for (int i = 0; i <= g; ++i) {
      if (i >= nda || g - i >= ndb) continue;
      p.sa[p.n] = i;
      p.sb[p.n] = g - i;
      p.grp[p.n] = std::min(g, tc::x::NG - 1);
      ++p.n;
    }
  for (int q = 0; q < tc::x::NG; ++q) {
    p.first[q] = -1;
    p.last[q] = -1;
  }
  for (int k = 0; k < p.n; ++k) {
    if (p.first[p.grp[k]] < 0) p.first[p.grp[k]] = k;
    p.last[p.grp[k]] = k;
  }
  // TMEM slots: the groups present take slots 0, 1, 0, 1 in group order; a group waits for the
  // drain of the slot's previous user (two groups earlier in the chunk, else the slot's last user
  // in the previous chunk)
  std::vector<int> present;
  for (int q = 0; q < tc::x::NG; ++q) {
    p.slot[q] = 0;
    p.wait_grp[q] = q;
    p.wait_same[q] = 0;
    if (p.first[q] >= 0) present.push_back(q);
  }
  const int np = (int)present.size();
  for (int k = 0; k < np; ++k) {
    const int q = present[k];
    p.slot[q] = k & 1;
    if (k >= 2) {
      p.wait_grp[q] = present[k - 2];
      p.wait_same[q] = 1;
    } else {
      int m = np - 1;
      while ((m & 1) != (k & 1)) --m;
      p.wait_grp[q] = present[m];
      p.wait_same[q] = 0;
    }
  }
  return p;
}

tc::Pairs pairs_for(int nsl) {
  tc::Pairs pairs{};
  if (nsl == 2) {
    pairs.n = 3;
    const int sa[3] = {0, 0, 1}, sb[3] = {0, 1, 0};
    for (int i = 0; i < 3; ++i) { pairs.sa[i] = sa[i]; pairs.sb[i] = sb[i]; }
  } else {
    pairs.n = 6;
    const int sa[6] = {0, 0, 1, 0, 1, 2}, sb[6] = {0, 1, 0, 2, 1, 0};
    for (int i = 0; i < 6; ++i) { pairs.sa[i] = sa[i]; pairs.sb[i] = sb[i]; }
  }
  return pairs;
}

}  // namespace

void tc_release_cache_for(Ctx& c) {   // cudaFree waits for the kernels still reading the slices
  if (!c.tcs) return;
  for (auto& kv : c.tcs->cache) cudaFree(kv.second.s.p);
  c.tcs->cache.clear();
}
size_t tc_cache_bytes(Ctx& c) {
  size_t t = 0;
  if (c.tcs)
    for (auto& kv : c.tcs->cache) t += entry_bytes(kv.second);
  return t;
}
void tc_state_free(Ctx& c) {
  if (!c.tcs) return;
  tc_release_cache_for(c);
  for (auto& p : c.tcs->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  delete c.tcs;
  c.tcs = nullptr;
}

int tc_slices(int precision) {
  return precision == CCLR_TC_BF16X3 ? 2 : precision == CCLR_TC_F64 ? tc::x::NS : 3;
}

bool tc_eligible(int64_t M, int64_t N, int64_t K) {
  // below ~2^18 complex multiply-adds the FP64 kernel is as fast as a tensor-core launch (a few
  // us) and keeps full accuracy; above it the FP64 pipe (~7.6 GFLOP/s per SM on sm_103) loses by
  // orders of magnitude.  Short K is zero-padded to 64.
  return K >= 1 && M >= 1 && N >= 1 && M <= INT32_MAX && N <= INT32_MAX &&
         (double)M * (double)N * (double)K >= 262144.0;
}

// C[m*ldc + n] = alpha sum_k vm[m,k] vn[n,k] + beta C, vm / vn views whose first nr axes are the
// rows (m resp. n) and whose remaining axes are K (same order in both).
// split-K slices for an output of M x N with K (1 = none): when the output has fewer tiles than
// SMs, each slice >= 4 k-blocks
namespace {

// ---- tile autotuner of the split-BF16 kernel (cclr_options.autotune).  Two tile shapes:
// 128 m-rows with 3 pipeline stages and 64 m-rows with 4 stages (the narrower tile gives more
// CTAs and less padding on small or skinny outputs; the wider one halves the A-side reloads).
// Tuning is online: the first launch of a GEMM shape (M, N, K, slice count, output map, SM
// count) uses the first shape and the second launch the second, each timed with CUDA events on
// the context's stream; later launches of that shape use the faster one.  No extra work is run.
// With CCLR_AUTOTUNE_CACHE set, decisions are read from and appended to that file.
struct TileCfg {
  int bn, stages;
};
constexpr TileCfg kTileCfgs[2] = {{128, 3}, {64, 4}};
struct TuneState {
  int best = -1;           // decided configuration
  int launched[2] = {};    // timed launches issued per configuration
  float ms[2] = {-1.f, -1.f};
};
// decisions are shared by all contexts of the process (guarded by tune_mutex)
std::map<std::string, TuneState>& tune_table() {
  static std::map<std::string, TuneState> t;
  return t;
}
std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
std::string tune_key(int64_t M, int64_t N, int64_t K, int nsl, bool strided) {
  return std::to_string(M) + "x" + std::to_string(N) + "x" + std::to_string(K) + "/" + std::to_string(nsl) + "/" +
         (strided ? "s" : "c") + "/" + std::to_string(num_sms());
}
const char* tune_cache_path() { return std::getenv("CCLR_AUTOTUNE_CACHE"); }
void tune_load() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = tune_cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char key[256];
  int best = 0;
  while (std::fscanf(f, "%255s %d", key, &best) == 2)
    if (best == 0 || best == 1) tune_table()[key].best = best;
  std::fclose(f);
}
// the configuration the next launch of this shape uses (no state change)
int tune_peek(const Ctx& c, const std::string& key) {
  if (!c.opt.autotune) return 0;
  std::lock_guard<std::mutex> lk(tune_mutex());
  tune_load();
  auto it = tune_table().find(key);
  if (it == tune_table().end()) return 0;
  const TuneState& t = it->second;
  if (t.best >= 0) return t.best;
  return t.launched[0] == 0 ? 0 : (t.launched[1] == 0 ? 1 : 0);
}

}  // namespace

// Resolves the timed launches of the tile autotuner on this context (after a stream synchronize).
void tc_tune_collect(Ctx& c) {
  if (!c.tcs) return;
  std::lock_guard<std::mutex> lk(tune_mutex());
  for (auto& p : c.tcs->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      TuneState& t = tune_table()[p.key];
      t.ms[p.cfg] = ms;
      if (t.best < 0 && t.ms[0] >= 0.f && t.ms[1] >= 0.f) {
        t.best = t.ms[1] < t.ms[0] ? 1 : 0;
        if (const char* path = tune_cache_path())
          if (FILE* f = std::fopen(path, "a")) {
            std::fprintf(f, "%s %d\n", p.key.c_str(), t.best);
            std::fclose(f);
          }
      }
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  c.tcs->pending.clear();
}

// Decided tile shapes of the autotuner as text, "key bn stages ms0 ms1" per line.
std::string tc_tune_report() {
  std::lock_guard<std::mutex> lk(tune_mutex());
  std::string out;
  for (auto& kv : tune_table()) {
    const TuneState& t = kv.second;
    if (t.best < 0) continue;
    char line[320];
    std::snprintf(line, sizeof line, "%s %d %d %.4f %.4f\n", kv.first.c_str(), kTileCfgs[t.best].bn,
                  kTileCfgs[t.best].stages, t.ms[0], t.ms[1]);
    out += line;
  }
  return out;
}

namespace {

// (bn: the m-rows of a tile, tc::BN or tc::x::BN)
void tc_split_plan(int64_t M, int64_t N, int64_t K, int& S, int& kb_per, int bn = tc::BN) {
  const int kblocks = (int)((K + tc::BK - 1) / tc::BK);
  const int64_t tiles = ((M + bn - 1) / bn) * ((N + tc::BM - 1) / tc::BM);
  const int sms = num_sms();
  S = 1;
  kb_per = kblocks;
  if (tiles < sms && kblocks >= 8) {
    S = (int)std::min<int64_t>((sms + tiles - 1) / tiles, kblocks / 4);
    kb_per = (kblocks + S - 1) / S;
    S = (kblocks + kb_per - 1) / kb_per;   // no empty slice
  }
}
}  // namespace

int tc_splits(const Ctx& c, int64_t M, int64_t N, int64_t K, bool strided) {
  int S, kb;
  int bn = tc::x::BN;
  if (c.opt.precision != CCLR_TC_F64) {
    const int64_t Kpad = (K + tc::BK - 1) / tc::BK * tc::BK;
    bn = kTileCfgs[tune_peek(c, tune_key(M, N, Kpad, tc_slices(c.opt.precision), strided))].bn;
  }
  tc_split_plan(M, N, K, S, kb, bn);
  return S;
}

namespace {
tc::OutMap out_map(const OutAxes& a) {
  tc::OutMap m;
  auto fill = [](int n, const int64_t* dim, const int64_t* str, int64_t* d, int64_t* st, uint32_t* mul, int* shr) {
    for (int i = 0; i < n; ++i) {
      CCLR_REQUIRE(dim[i] >= 1 && dim[i] < (int64_t(1) << 31), CCLR_E_ARG, "tc_gemm: output axis too large");
      d[i] = dim[i];
      st[i] = str[i];
      int l = 0;
      while ((int64_t(1) << l) < dim[i]) ++l;
      shr[i] = l;
      mul[i] = (uint32_t)(((unsigned __int128)1 << 32) * (((uint64_t)1 << l) - (uint64_t)dim[i]) / (uint64_t)dim[i] + 1);
    }
  };
  CCLR_REQUIRE(a.nm >= 1 && a.nm <= 4 && a.nn >= 1 && a.nn <= 4, CCLR_E_ARG, "tc_gemm: output map rank");
  m.nm = a.nm;
  m.nn = a.nn;
  fill(a.nm, a.mdim, a.mstr, m.mdim, m.mstr, m.mmul, m.mshr);
  fill(a.nn, a.ndim, a.nstr, m.ndim, m.nstr, m.nmul, m.nshr);
  return m;
}
}  // namespace

// FP64-class GEMM (CCLR_TC_F64) on the digit slices sn (n rows) and sm (m rows): k_tc_zgemm_x.
void tc_gemm_x(Ctx& c, const Slices& sn, const Slices& sm, cplx alpha, cplx beta, cplx* C, int64_t ldc,
               const OutAxes* oa) {
  const int64_t M = sm.rows, N = sn.rows;
  static bool attr[64] = {};
  if (once_per_device(attr))
    CCLR_CK(cudaFuncSetAttribute(tc::k_tc_zgemm_x, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::x::SMEM_BYTES));
  const int kblocks = (int)(sn.Kpad / tc::BK);
  int S = 1, kb_per = kblocks;
  tc_split_plan(M, N, sn.Kpad, S, kb_per, tc::x::BN);
  CCLR_REQUIRE(!oa || S == 1, CCLR_E_ARG, "tc_gemm: strided output with split-K");
  const tc::OutMap om = oa ? out_map(*oa) : tc::OutMap();
  cplx* P = S > 1 ? c.ws.cplxs((int64_t)S * M * N) : nullptr;
  const int64_t ytiles = (N + tc::BM - 1) / tc::BM, xtiles = (M + tc::x::BN - 1) / tc::x::BN;
  CCLR_REQUIRE(xtiles * ytiles * S < (int64_t)INT32_MAX, CCLR_E_ARG, "tc_gemm: too many tiles");
  const int grid = (int)std::min<int64_t>(xtiles * ytiles * S, num_sms());
  float2* fstate = (float2*)c.ws.alloc(sizeof(float2) * 2 * (size_t)grid * tc::BM * tc::x::BN);
  const CUtensorMap tmB = make_map(sm.p, sm.rows, sm.Kpad, 2 * sm.nsl, tc::x::BN);
  const tc::PairsX pairs = pairs_x(sn.ndig, sm.ndig);
  // a real power-of-two alpha is applied exactly to the float-float sums (no FP64 multiply)
  float apow2 = 0.0f;
  if (S == 1 && alpha.y == 0.0 && alpha.x != 0.0) {
    int e = 0;
    const double f = std::frexp(std::fabs(alpha.x), &e);
    if (f == 0.5 && e > -100 && e < 100) apow2 = (float)alpha.x;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c.prof) c.prof_events(e0, e1, 1);
  if (e0) CCLR_CK(cudaEventRecord(e0, c.stream));
  c.kt.begin(c.stream);
  if (S > 1)
    tc::k_tc_zgemm_x<<<grid, tc::x::THREADS, tc::x::SMEM_BYTES, c.stream>>>(
        sn.tm, tmB, (int)N, (int)M, kblocks, kb_per, pairs, make_double2(1.0, 0.0), 1.0f, make_double2(0.0, 0.0), P, N,
        M * N, c.tc_err, (int)xtiles, (int)ytiles, S, om, false, fstate);
  else
    tc::k_tc_zgemm_x<<<grid, tc::x::THREADS, tc::x::SMEM_BYTES, c.stream>>>(
        sn.tm, tmB, (int)N, (int)M, kblocks, kb_per, pairs, alpha, apow2, beta, C, ldc, 0, c.tc_err, (int)xtiles,
        (int)ytiles, 1, om, oa != nullptr, fstate);
  const cudaError_t le = cudaGetLastError();
  CCLR_REQUIRE(le == cudaSuccess, CCLR_E_CUDA,
               std::string("FP64-class tensor-core GEMM launch failed (") + cudaGetErrorString(le) + ") M=" +
                   std::to_string(M) + " N=" + std::to_string(N) + " K=" + std::to_string(sn.K));
  c.kt.end(c.stream, "k_tc_zgemm_x");
  if (e1) {
    CCLR_CK(cudaEventRecord(e1, c.stream));
    c.prof_flops_exec[1] += 8.0 * (double)M * N * sn.K * pairs.n;
    c.prof_flops_useful[1] += 8.0 * (double)M * N * sn.K;
  }
  ++c.launches;
  if (S > 1) splitk_reduce(c.L, P, S, M, N, alpha, beta, C, ldc);
}

void tc_gemm_views(Ctx& c, const Tensor& vm, int nrm, const Tensor& vn, int nrn, cplx alpha, cplx beta, cplx* C,
                   int64_t ldc, const OutAxes* oa) {
  const int nsl = tc_slices(c.opt.precision);
  Scope sc(c.ws);
  const Slices sn = get_slices(c, vn, nrn, nsl);   // MMA A-side: rows = n (TMEM lanes)
  const Slices sm = get_slices(c, vm, nrm, nsl);   // MMA B-side: rows = m
  CCLR_REQUIRE(sn.K == sm.K, CCLR_E_ARG, "tc_gemm: K mismatch");
  if (!c.tc_err) {  // device status word, checked by the API layer at the end of every call
    CCLR_CK(cudaMalloc((void**)&c.tc_err, sizeof(int)));
    CCLR_CK(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.stream));
  }
  if (c.opt.precision == CCLR_TC_F64) {
    tc_gemm_x(c, sn, sm, alpha, beta, C, ldc, oa);
    return;
  }
  const tc::Pairs pairs = pairs_for(nsl);
  const int64_t M = sm.rows, N = sn.rows;
  const bool strided = oa != nullptr;
  const std::string key = tune_key(M, N, sn.Kpad, nsl, strided);
  const int cfg = tune_peek(c, key);
  const int bn = kTileCfgs[cfg].bn;
  const int kblocks = (int)(sn.Kpad / tc::BK);
  int S = 1, kb_per = kblocks;
  tc_split_plan(M, N, sn.Kpad, S, kb_per, bn);
  CCLR_REQUIRE(!oa || S == 1, CCLR_E_ARG, "tc_gemm: strided output with split-K");
  const tc::OutMap om = oa ? out_map(*oa) : tc::OutMap();
  cplx* P = nullptr;
  if (S > 1) P = c.ws.cplxs((int64_t)S * M * N);
  const int64_t ytiles = (N + tc::BM - 1) / tc::BM, xtiles = (M + bn - 1) / bn;
  CCLR_REQUIRE(xtiles * ytiles * S < (int64_t)INT32_MAX, CCLR_E_ARG, "tc_gemm: too many tiles");
  // the B-side map with this tile's box (the cached maps have 128-row boxes)
  const CUtensorMap tmB = bn == 128 ? sm.tm : make_map(sm.p, sm.rows, sm.Kpad, 2 * sm.nsl, bn);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c.prof) c.prof_events(e0, e1, 0);
  if (e0) CCLR_CK(cudaEventRecord(e0, c.stream));
  // a launch of an undecided shape is timed for the autotuner
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  bool timed = false;
  if (c.opt.autotune) {
    std::lock_guard<std::mutex> lk(tune_mutex());
    TuneState& t = tune_table()[key];
    timed = t.best < 0 && t.launched[cfg] == 0;
    if (timed) t.launched[cfg] = 1;
  }
  if (timed) {
    CCLR_CK(cudaEventCreate(&t0));
    CCLR_CK(cudaEventCreate(&t1));
    CCLR_CK(cudaEventRecord(t0, c.stream));
  }
  {
    // persistent: one CTA per SM (or per tile when there are fewer)
    const int grid = (int)std::min<int64_t>(xtiles * ytiles * S, num_sms());
    // a pending expiry test (cclr_debug_expire_next_wait) applies to this launch only
    const uint32_t polls = c.dbg_wait_polls ? c.dbg_wait_polls : tc::kWaitPolls;
    const int expire = c.dbg_wait_polls ? 1 : 0;
    c.dbg_wait_polls = 0;
    c.kt.begin(c.stream);
    auto launch = [&](auto kernel, int smem, bool* attr) {
      if (once_per_device(attr))
        CCLR_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      if (S > 1)
        kernel<<<grid, tc::TC_THREADS, smem, c.stream>>>(sn.tm, tmB, (int)N, (int)M, kblocks, kb_per, pairs,
                                                         make_double2(1.0, 0.0), make_double2(0.0, 0.0), P, N, M * N,
                                                         c.tc_err, (int)xtiles, (int)ytiles, S, om, false, polls, expire);
      else
        kernel<<<grid, tc::TC_THREADS, smem, c.stream>>>(sn.tm, tmB, (int)N, (int)M, kblocks, kb_per, pairs, alpha, beta,
                                                         C, ldc, 0, c.tc_err, (int)xtiles, (int)ytiles, 1, om, strided,
                                                         polls, expire);
    };
    static bool attr128[64] = {}, attr64[64] = {};
    if (bn == 128) launch(tc::k_tc_zgemm<128, 3>, tc::smem_bytes(128, 3), attr128);
    else launch(tc::k_tc_zgemm<64, 4>, tc::smem_bytes(64, 4), attr64);
    const cudaError_t le = cudaGetLastError();
    CCLR_REQUIRE(le == cudaSuccess, CCLR_E_CUDA,
                 std::string("tensor-core GEMM launch failed (") + cudaGetErrorString(le) + ") M=" + std::to_string(M) +
                     " N=" + std::to_string(N) + " K=" + std::to_string(sn.K) + " S=" + std::to_string(S));
    c.kt.end(c.stream, bn == 128 ? "k_tc_zgemm" : "k_tc_zgemm<64>");
  }
  if (t0) {
    CCLR_CK(cudaEventRecord(t1, c.stream));
    tcs(c).pending.push_back({key, cfg, t0, t1});
  }
  if (e1) {
    CCLR_CK(cudaEventRecord(e1, c.stream));
    c.prof_flops_exec[0] += 8.0 * (double)M * N * sn.K * pairs.n;
    c.prof_flops_useful[0] += 8.0 * (double)M * N * sn.K;
  }
  ++c.launches;
  if (S > 1) splitk_reduce(c.L, P, S, M, N, alpha, beta, C, ldc);
}

bool tc_gemm_try(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A, int64_t lda,
                 const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc) {
  if (!tc_eligible(M, N, K)) return false;
  // 2-axis views (rows, K) of op(A) and op(B)^T; transposed storage is read with swapped strides
  Tensor vm = Tensor::make((cplx*)A, {M, K}), vn = Tensor::make((cplx*)B, {N, K});
  if (ta) { vm.str[0] = 1; vm.str[1] = lda; } else { vm.str[0] = lda; vm.str[1] = 1; }
  if (tb) { vn.str[0] = ldb; vn.str[1] = 1; } else { vn.str[0] = 1; vn.str[1] = ldb; }
  tc_gemm_views(c, vm, 1, vn, 1, alpha, beta, C, ldc);
  return true;
}

// ---------------------------------------------------------------------------------------------
// Building blocks of the allocation-free GEMM entry point (noalloc.cu): the same slicing, kernel
// and split-K choice as tc_gemm_views, with every temporary placed in caller-provided scratch.
// Scratch layout: [status word, 256 B][slices of B (n rows)][slices of A (m rows)][split-K partials]

namespace {
struct RawPlan {
  int64_t Kpad, bytes_sn, bytes_sm, bytes_p;
  int S, kb_per, kblocks;
};
RawPlan raw_plan(int nsl, int64_t M, int64_t N, int64_t K) {
  RawPlan p{};
  p.Kpad = (K + tc::BK - 1) / tc::BK * tc::BK;
  p.bytes_sn = (int64_t)sizeof(__nv_bfloat16) * 2 * nsl * N * p.Kpad;
  p.bytes_sm = (int64_t)sizeof(__nv_bfloat16) * 2 * nsl * M * p.Kpad;
  p.kblocks = (int)(p.Kpad / tc::BK);
  tc_split_plan(M, N, p.Kpad, p.S, p.kb_per);   // the same split-K choice as the context's GEMMs
  p.bytes_p = p.S > 1 ? (int64_t)sizeof(cplx) * p.S * M * N : 0;
  return p;
}
int64_t up256(int64_t b) { return (b + 255) / 256 * 256; }
}  // namespace

int64_t tc_raw_scratch_bytes(int precision, int64_t M, int64_t N, int64_t K) {
  const RawPlan p = raw_plan(tc_slices(precision), M, N, K);
  return 256 + up256(p.bytes_sn) + up256(p.bytes_sm) + up256(p.bytes_p);
}

// C[m*N + n] = sum_k A[m*K + k] B[n*K + k] on `stream`, synchronously; returns the status word
// (0 = every bounded wait completed).
int tc_raw_gemm_nt(int precision, int64_t M, int64_t N, int64_t K, const cplx* A, const cplx* B, cplx* C, char* scratch,
                   cudaStream_t stream) {
  const int nsl = tc_slices(precision);
  const RawPlan p = raw_plan(nsl, M, N, K);
  int* err = (int*)scratch;
  __nv_bfloat16* sn = (__nv_bfloat16*)(scratch + 256);
  __nv_bfloat16* sm = (__nv_bfloat16*)(scratch + 256 + up256(p.bytes_sn));
  cplx* P = (cplx*)(scratch + 256 + up256(p.bytes_sn) + up256(p.bytes_sm));
  CCLR_CK(cudaMemsetAsync(err, 0, sizeof(int), stream));   // the shared scratch keeps the last call's flag
  auto split = [&](const cplx* X, int64_t rows, __nv_bfloat16* dst) {
    launch_split(Tensor::make(const_cast<cplx*>(X), {rows, K}), 1, rows, K, p.Kpad, nsl, dst, stream);
    CCLR_CK(cudaGetLastError());
  };
  split(B, N, sn);
  split(A, M, sm);
  const CUtensorMap tn = make_map(sn, N, p.Kpad, 2 * nsl, 128), tm = make_map(sm, M, p.Kpad, 2 * nsl, 128);
  static bool attr[64] = {};
  if (once_per_device(attr))   // per device: a call on another device needs its own attribute
    CCLR_CK(cudaFuncSetAttribute(tc::k_tc_zgemm<tc::BN, tc::STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::SMEM_BYTES));
  const tc::Pairs pairs = pairs_for(nsl);
  const int64_t ytiles = (N + tc::BM - 1) / tc::BM, xtiles = (M + tc::BN - 1) / tc::BN;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  CCLR_REQUIRE(xtiles * ytiles * p.S < (int64_t)INT32_MAX, CCLR_E_ARG, "tc_gemm: too many tiles");
  {
    const int grid = (int)std::min<int64_t>(xtiles * ytiles * p.S, num_sms());
    if (p.S > 1)
      tc::k_tc_zgemm<tc::BN, tc::STAGES><<<grid, tc::TC_THREADS, tc::SMEM_BYTES, stream>>>(tn, tm, (int)N, (int)M, p.kblocks, p.kb_per, pairs, one,
                                                            zero, P, N, M * N, err, (int)xtiles, (int)ytiles, p.S,
                                                            tc::OutMap(), false, tc::kWaitPolls, 0);
    else
      tc::k_tc_zgemm<tc::BN, tc::STAGES><<<grid, tc::TC_THREADS, tc::SMEM_BYTES, stream>>>(tn, tm, (int)N, (int)M, p.kblocks, p.kb_per, pairs, one,
                                                            zero, C, N, 0, err, (int)xtiles, (int)ytiles, 1,
                                                            tc::OutMap(), false, tc::kWaitPolls, 0);
    CCLR_CK(cudaGetLastError());
  }
  if (p.S > 1) {
    Launch L;
    L.s = stream;
    splitk_reduce(L, P, p.S, M, N, one, zero, C, N);
  }
  int h = 0;
  CCLR_CK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CCLR_CK(cudaStreamSynchronize(stream));
  return h;
}

}  // namespace cclr

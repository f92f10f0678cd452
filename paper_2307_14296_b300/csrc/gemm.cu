// GEMM backend selection.  CCLR_FP64 runs every contraction on the FP64 DFMA kernel; the
// tensor-core modes route K-major contractions to the tcgen05 kernel (tc_gemm.cu).
// Skinny shapes (few output tiles, long K: e.g. the singles projections of o^2 v^3 terms) are
// split along K so that every SM works; the partial tiles are summed in a fixed order.
#include "ctx.h"
#include <algorithm>

namespace cclr {

bool tc_gemm_try(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A, int64_t lda,
                 const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc);

void gemm_dispatch(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A,
                   int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc) {
  if (c.opt.precision != CCLR_FP64 && tc_gemm_try(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc)) return;
  const int64_t tiles = ((M + 63) / 64) * ((N + 63) / 64);
  const int64_t sms = num_sms();
  if (tiles < 2 * sms && K >= 32) {
    // FP64 split-K: enough slices for ~2 blocks per SM, each slice at least 16 deep (FP64 runs at
    // a few GFLOP/s per SM, so even a 30 x 30 x 200 product wants more than one SM)
    int64_t S = std::min<int64_t>({(2 * sms + tiles - 1) / tiles, K / 16, 256});
    if (S >= 2) {
      int64_t kchunk = ((K + S - 1) / S + 7) / 8 * 8;
      S = (K + kchunk - 1) / kchunk;
      Scope sc(c.ws);
      cplx* P = c.ws.cplxs(S * M * N);
      zgemm_splitk(c.L, ta, tb, M, N, K, A, lda, B, ldb, P, (int)S, kchunk);
      splitk_reduce(c.L, P, (int)S, M, N, alpha, beta, C, ldc);
      return;
    }
  }
  zgemm(c.L, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

}  // namespace cclr

// GEMM backend selection.  CCLR_FP64 runs every contraction on the FP64 DFMA kernel; the
// tensor-core modes route large contractions to the tcgen05 kernels (tc_gemm.cu).
#include "ctx.h"

namespace cclr {

bool tc_gemm_try(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A, int64_t lda,
                 const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc);

void gemm_dispatch(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A,
                   int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc) {
  if (c.opt.precision != CCLR_FP64 && tc_gemm_try(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc)) return;
  zgemm(c.L, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

// Until the tensor-core kernels are enabled every call falls back to FP64.
__attribute__((weak)) bool tc_gemm_try(Ctx&, bool, bool, int64_t, int64_t, int64_t, cplx, const cplx*, int64_t,
                                       const cplx*, int64_t, cplx, cplx*, int64_t) {
  return false;
}

}  // namespace cclr

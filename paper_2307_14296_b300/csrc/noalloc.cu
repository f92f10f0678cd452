// Allocation-free variant of the tensor-core complex GEMM (cclr_zgemm_nt_noalloc).
//
// Some callers cannot call cudaMalloc: a host framework that owns the whole device memory
// through its own pool, a server that forbids allocation after start-up so that its memory
// footprint stays fixed, or code running where an allocation may block or fail (a callback
// inside another library's stream work).  For them this entry point takes device pointers for
// inputs and outputs and keeps every temporary (BF16 operand slices, split-K partial tiles and
// the kernel's status word) in one file-scope device array of fixed size.  Every process that
// loads the library holds that array on each device it uses until the process exits.
#include "ctx.h"

namespace cclr {
int64_t tc_raw_scratch_bytes(int precision, int64_t M, int64_t N, int64_t K);
int tc_raw_gemm_nt(int precision, int64_t M, int64_t N, int64_t K, const cplx* A, const cplx* B, cplx* C, char* scratch,
                   cudaStream_t stream);
}  // namespace cclr

using namespace cclr;

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;   // 64 MiB, documented in include/cclr.h

// Shared by every call on a device; calls that overlap on the GPU race on it.
static __device__ __align__(256) char g_scratch[kNoAllocScratchBytes];

// Device address of g_scratch per device, resolved once (the name g_scratch is only a host-side
// stand-in in host code and must never be passed to a kernel).
constexpr int kMaxDevices = 64;
char* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" cclr_status cclr_zgemm_nt_noalloc(int precision, int M, int N, int K, const cclr_c128* A, const cclr_c128* B,
                                             cclr_c128* C, void* stream) {
  if (precision != CCLR_TC_BF16X3 && precision != CCLR_TC_BF16X6) return CCLR_E_ARG;
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return CCLR_E_ARG;
  if ((size_t)tc_raw_scratch_bytes(precision, M, N, K) > kNoAllocScratchBytes) return CCLR_E_ARG;   // too large
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CCLR_E_CUDA;
  if (!g_scratch_addr[dev]) {
    // one-time set-up on this device, with the device current (do this before any stream capture)
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return CCLR_E_CUDA;
    g_scratch_addr[dev] = (char*)p;
  }
  try {
    const int st = tc_raw_gemm_nt(precision, M, N, K, (const cplx*)A, (const cplx*)B, (cplx*)C, g_scratch_addr[dev],
                                  (cudaStream_t)stream);
    return st == 0 ? CCLR_OK : CCLR_E_TIMEOUT;
  } catch (const Error& e) {
    return e.st;
  } catch (...) {
    return CCLR_E_CUDA;
  }
}

// hs_gemm_static: the tensor-core block GEMM of hs_gemm for callers that must
// not allocate device memory themselves.
//
// Who needs it: applications whose memory manager owns all device memory (a
// pooling allocator that forbids out-of-band cudaMalloc), latency-critical
// loops that cannot afford the device-wide synchronisation cudaMalloc and
// cudaFree may imply, and plugins hosted by a framework that does not let
// extensions change the device memory footprint. hs_gemm needs a context,
// whose workspace grows with cudaMalloc; this entry point needs neither.
//
// Its scratch (the split, K-padded copies of A and B) lives in the file-scope
// array g_scratch below, kScratchBytes in size. Every GPU that loads this
// library holds that array until the process exits. Host code cannot use the
// array's name as a device address, so the first call on each device, with
// that device current, looks the address up once with cudaGetSymbolAddress
// and caches it; that first call should come before any stream capture.
//
// Every call uses the same array and leaves the last call's data in it. The
// split kernel writes every element a call reads (padding columns included),
// so nothing in the array needs clearing; the caller's status word is set to
// zero at the start of each call. Each device has its own copy of the array;
// calls whose GPU work overlaps on one device (say, on two streams) race on
// it: order them on one stream.
#include <mutex>

#include "hs_ctx.cuh"

namespace hs {
namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB of operand scratch
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once).
hs_status scratch_address(void** out) {
  int dev = 0;
  HS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(HS_ERR_INVALID_ARG, "device %d beyond the supported %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return fail(HS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return HS_OK;
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" hs_status hs_gemm_static(hs_precision precision, int M, int N, int K, const double* A, int lda,
                                    const double* B, int ldb, double* C, int ldc, int* status_out,
                                    void* stream) {
  if (M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < N || (M > 0 && N > 0 && (!A || !B || !C)) ||
      !status_out)
    return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (precision != HS_PREC_TF32X3 && precision != HS_PREC_TF32 && precision != HS_PREC_BF16X3)
    return fail(HS_ERR_INVALID_ARG, "hs_gemm_static supports the tensor-core precisions only");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* base = nullptr;
  HS_TRY(scratch_address(&base));
  HS_CUDA(cudaMemsetAsync(status_out, 0, sizeof(int), s));
  if (M == 0 || N == 0) return HS_OK;
  if (K == 0) {
    HS_CUDA(cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * N, M, s));
    return HS_OK;
  }
  const int pad = tc_pad(precision), eb = tc_elem_bytes(precision);
  const long long Kp = ((long long)K + pad - 1) / pad * pad;
  // A_hi, A_lo, B_hi, B_lo back to back (each a multiple of 128 bytes)
  const size_t need = 2 * (size_t)(M + (long long)N) * Kp * eb;
  if (need > kScratchBytes)
    return fail(HS_ERR_SHAPE,
                "hs_gemm_static: 2*(M+N)*Kp*%d = %zu bytes exceed the static scratch of %zu bytes "
                "(M=%d N=%d K=%d, K padded to %lld)",
                eb, need, kScratchBytes, M, N, K, Kp);
  unsigned char* a_hi = static_cast<unsigned char*>(base);
  unsigned char* a_lo = a_hi + (size_t)M * Kp * eb;
  unsigned char* b_hi = a_lo + (size_t)M * Kp * eb;
  unsigned char* b_lo = b_hi + (size_t)N * Kp * eb;
  const int mode = tc_mode(precision);
  HS_CUDA(launch_split_pad(A, M, K, lda, a_hi, a_lo, Kp, mode, s));
  HS_CUDA(launch_split_pad(B, N, K, ldb, b_hi, b_lo, Kp, mode, s));
  TcProblem t;
  t.M = M;
  t.N = N;
  t.Kp = (int)Kp;
  t.ldc = ldc;
  t.a_hi = a_hi;
  t.a_lo = a_lo;
  t.b_hi = b_hi;
  t.b_lo = b_lo;
  t.c = C;
  HS_CUDA(launch_gemm_tc(precision, &t, 1, status_out, s));
  return HS_OK;
}

// Grouped FP64 GEMM (DFMA) for the block contractions in FP64 mode:
// C[m, n] = alpha * sum_k A[m, k] B[n, k], both operands K-major (row-major
// M x K and N x K). One CTA per 64 x 64 output tile of any problem of the group.
#include "hs_internal.cuh"

namespace hs {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ int cdiv(int a, int b) { return (a + b - 1) / b; }

__global__ void __launch_bounds__(NT) gemm_f64_nt_kernel(GemmGroup g, const double* __restrict__ A,
                                                         const double* __restrict__ B,
                                                         double* __restrict__ C, double alpha) {
  int t = blockIdx.x;
  int pi = 0;
  for (; pi < g.n; ++pi) {
    const int tiles = cdiv(g.p[pi].M, BM) * cdiv(g.p[pi].N, BN);
    if (t < tiles) break;
    t -= tiles;
  }
  if (pi >= g.n) return;
  const GemmProblem P = g.p[pi];
  const int tn_count = cdiv(P.N, BN);
  const int m0 = (t / tn_count) * BM, n0 = (t % tn_count) * BN;
  const double* Ap = A + P.a_off;
  const double* Bp = B + P.b_off;
  double* Cp = C + P.c_off;

  __shared__ double As[BK][BM + 2];
  __shared__ double Bs[BK][BN + 2];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < P.K; k0 += BK) {
#pragma unroll
    for (int i = 0; i < (BM * BK) / NT; ++i) {
      const int idx = threadIdx.x + i * NT;
      const int r = idx / BK, c = idx % BK;
      const int gm = m0 + r, gk = k0 + c;
      As[c][r] = (gm < P.M && gk < P.K) ? Ap[(long long)gm * P.lda + gk] : 0.0;
      const int gn = n0 + r;
      Bs[c][r] = (gn < P.N && gk < P.K) ? Bp[(long long)gn * P.ldb + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= P.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < P.N) Cp[(long long)gm * P.ldc + gn] = alpha * acc[i][j];
    }
  }
}
}  // namespace

cudaError_t launch_gemm_f64(const GemmGroup& g, const double* A, const double* B, double* C,
                            double alpha, cudaStream_t s) {
  long long tiles = 0;
  for (int i = 0; i < g.n; ++i)
    tiles += (long long)((g.p[i].M + BM - 1) / BM) * ((g.p[i].N + BN - 1) / BN);
  if (tiles == 0) return cudaSuccess;
  gemm_f64_nt_kernel<<<(unsigned)tiles, NT, 0, s>>>(g, A, B, C, alpha);
  return cudaGetLastError();
}

}  // namespace hs

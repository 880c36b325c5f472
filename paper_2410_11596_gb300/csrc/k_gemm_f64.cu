// Grouped FP64 GEMM (DFMA) for the block contractions in FP64 mode:
// C[m, n] = alpha * sum_k A[m, k] B[n, k] (+ C[m, n] when accumulating), both
// operands K-major (row-major M x K and N x K). One CTA per 64 x 64 output
// tile of any problem of the group.
#include "hs_internal.cuh"

namespace hs {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ int cdiv(int a, int b) { return (a + b - 1) / b; }

// With nsplit > 1 every tile is computed as nsplit partial sums over
// consecutive K ranges, written to `part` (problem i at part_off[i], split s
// at s * M * N, row-major M x N) and summed by splitk_reduce_kernel in a fixed
// order (deterministic).
struct SplitK {
  int nsplit;
  long long part_off[kMaxProblems];
};

__global__ void __launch_bounds__(NT) gemm_f64_nt_kernel(GemmGroup g, const double* __restrict__ A,
                                                         const double* __restrict__ B,
                                                         double* __restrict__ C, double alpha, bool accumulate,
                                                         SplitK sk, double* __restrict__ part) {
  hs_pdl_enter();
  int t = blockIdx.x / sk.nsplit;
  const int split = blockIdx.x % sk.nsplit;
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
  const int kchunk = cdiv(cdiv(P.K, sk.nsplit), BK) * BK;
  const int kbeg = split * kchunk;
  const int kend = min(P.K, kbeg + kchunk);
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

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int i = 0; i < (BM * BK) / NT; ++i) {
      const int idx = threadIdx.x + i * NT;
      const int r = idx / BK, c = idx % BK;
      const int gm = m0 + r, gk = k0 + c;
      As[c][r] = (gm < P.M && gk < kend) ? Ap[(long long)gm * P.lda + gk] : 0.0;
      const int gn = n0 + r;
      Bs[c][r] = (gn < P.N && gk < kend) ? Bp[(long long)gn * P.ldb + gk] : 0.0;
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
  double* out = Cp;
  long long ld = P.ldc;
  if (sk.nsplit > 1) {
    out = part + sk.part_off[pi] + (long long)split * P.M * P.N;
    ld = P.N;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= P.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < P.N) {
        double& o = out[(long long)gm * ld + gn];
        o = (accumulate && sk.nsplit == 1) ? o + alpha * acc[i][j] : alpha * acc[i][j];
      }
    }
  }
}

__global__ void splitk_reduce_kernel(GemmGroup g, SplitK sk, const double* __restrict__ part,
                                     double* __restrict__ C, bool accumulate) {
  hs_pdl_enter();
  for (int pi = 0; pi < g.n; ++pi) {
    const GemmProblem P = g.p[pi];
    const long long mn = (long long)P.M * P.N;
    const double* src = part + sk.part_off[pi];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mn;
         e += (long long)gridDim.x * blockDim.x) {
      double v = 0.0;
      for (int s = 0; s < sk.nsplit; ++s) v += src[s * mn + e];
      double& o = C[P.c_off + (e / P.N) * P.ldc + (e % P.N)];
      o = accumulate ? o + v : v;
    }
  }
}
}  // namespace

cudaError_t launch_gemm_f64(const GemmGroup& g, const double* A, const double* B, double* C,
                            double alpha, cudaStream_t s, double* part, long long part_elems, bool accumulate) {
  long long tiles = 0;
  int kmax = 0;
  for (int i = 0; i < g.n; ++i) {
    tiles += (long long)((g.p[i].M + BM - 1) / BM) * ((g.p[i].N + BN - 1) / BN);
    kmax = g.p[i].K > kmax ? g.p[i].K : kmax;
  }
  if (tiles == 0) return cudaSuccess;
  // split K when the output tiles cannot fill the GPU (3 resident CTAs on each
  // of its SMs) and each split still gets several K steps
  const long long kTarget = 3LL * device_sms();
  SplitK sk{};
  sk.nsplit = 1;
  if (part && tiles < kTarget) {
    int ns = (int)((kTarget + tiles - 1) / tiles);
    ns = ns < kmax / (4 * BK) ? ns : kmax / (4 * BK);
    ns = ns < 64 ? ns : 64;
    long long need = 0;
    for (int i = 0; i < g.n; ++i) need += (long long)g.p[i].M * g.p[i].N;
    while (ns > 1 && need * ns > part_elems) --ns;
    if (ns > 1) {
      sk.nsplit = ns;
      long long off = 0;
      for (int i = 0; i < g.n; ++i) {
        sk.part_off[i] = off;
        off += (long long)g.p[i].M * g.p[i].N * ns;
      }
    }
  }
  hs_launch(gemm_f64_nt_kernel, (unsigned)(tiles * sk.nsplit), NT, 0, s, g, A, B, C, alpha, accumulate, sk, part);
  if (sk.nsplit > 1) {
    long long mn = 0;
    for (int i = 0; i < g.n; ++i) mn = (long long)g.p[i].M * g.p[i].N > mn ? (long long)g.p[i].M * g.p[i].N : mn;
    long long gx = (mn + 255) / 256;
    if (gx > 4096) gx = 4096;
    hs_launch(splitk_reduce_kernel, (unsigned)gx, 256, 0, s, g, sk, part, C, accumulate);
  }
  return cudaGetLastError();
}

}  // namespace hs

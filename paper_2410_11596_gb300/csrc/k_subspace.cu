// Kernels of the warm-started subspace eigensolver for the CTMRG projector
// (the truncation of Sec. II.A needs only the chi eigenpairs of largest
// modulus of each parity block of the enlarged corner, not all of them).
#include <cmath>

#include "hs_internal.cuh"

namespace hs {

namespace {

unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// Counter-based hash (splitmix64 finaliser) -> uniform in (-1, 1).
__device__ __forceinline__ double hash_uniform(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// rows [r0, m) of X (m x n, row-major) get seeded pseudo-random entries
__global__ void fill_random_rows_kernel(double* __restrict__ X, int r0, int m, int n, unsigned long long seed) {
  hs_pdl_enter();
  const long long total = (long long)(m - r0) * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    X[(long long)r0 * n + e] = hash_uniform(seed * 0x100000001B3ull + (unsigned long long)e);
}

// Cholesky G = L L^T (lower) of an m x m SPD matrix and L^{-1}, in FP64, by
// one CTA in shared memory (m <= kMaxSub). Right-looking: step j takes the
// pivot, scales column j of L and row j of L^{-1}, then applies the rank-1
// updates of both (forward substitution of L X = I carried along the
// factorisation). One m x (m+1) array holds both triangles: L[i][c] at
// (i, c) and L^{-1}[i][c] at (c, i + 1), c <= i. On a non-positive pivot the
// status word is set and Linv is left unspecified.
constexpr int kMaxChol = 160;  // m (m + 1) doubles of shared memory
// Rayleigh-Ritz problems up to kMaxSub (the Jacobi kernel below); subspaces
// above kMaxChol take the library Cholesky route (hs_api.cu)
constexpr int kMaxSub = 192;

__global__ void __launch_bounds__(1024) chol_inv_kernel(const double* __restrict__ G0, int m0,
                                                        double* __restrict__ Linv0, const double* __restrict__ G1,
                                                        int m1, double* __restrict__ Linv1, int* __restrict__ status) {
  hs_pdl_enter();
  // one CTA per matrix (blockIdx.x)
  const double* G = blockIdx.x ? G1 : G0;
  double* Linv = blockIdx.x ? Linv1 : Linv0;
  const int m = blockIdx.x ? m1 : m0;
  if (m <= 0) return;
  extern __shared__ double sh[];
  const int ld = m + 1;
  double* A = sh;
  for (int e = threadIdx.x; e < m * ld; e += blockDim.x) {
    const int i = e / ld, c = e - (e / ld) * ld;
    A[e] = c <= i ? 0.5 * (G[i * m + c] + G[c * m + i]) : (c == i + 1 ? 1.0 : 0.0);
  }
  __shared__ int bad;
  __shared__ double s_rp;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  for (int j = 0; j < m; ++j) {
    // the pivot's square root and reciprocal once (FP64 square roots and
    // divisions are long sequences on the FP64 pipe)
    if (threadIdx.x == 0) {
      const double d = A[j * ld + j];
      const bool ok = d > 0.0;
      const double piv = ok ? sqrt(d) : 1.0;
      A[j * ld + j] = piv;
      s_rp = 1.0 / piv;
      if (!ok) bad = 1;
    }
    __syncthreads();
    const double rp = s_rp;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[i * ld + j] *= rp;
    for (int c = threadIdx.x; c <= j; c += blockDim.x) A[c * ld + j + 1] *= rp;
    __syncthreads();
    for (int r = j + 1 + ty; r < m; r += ny) {
      const double lrj = A[r * ld + j];
      for (int c = j + 1 + tx; c <= r; c += 32) A[r * ld + c] -= lrj * A[c * ld + j];
      for (int c = tx; c <= j; c += 32) A[c * ld + r + 1] -= lrj * A[c * ld + j + 1];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, c = e - (e / m) * m;
    Linv[e] = c <= i ? A[c * ld + i + 1] : 0.0;
  }
  if (threadIdx.x == 0 && bad) *status = 1;
}

// res[i] = || Zr_i - theta_i Xr_i || for the m rows (theta from FP32 values).
__global__ void residual_kernel(const double* __restrict__ Zr, const double* __restrict__ Xr,
                                const float* __restrict__ theta, int m, int n, double* __restrict__ res) {
  hs_pdl_enter();
  const int i = blockIdx.x;
  if (i >= m) return;
  const double t = (double)theta[i];
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = Zr[(long long)i * n + j] - t * Xr[(long long)i * n + j];
    s += v * v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) res[i] = sqrt(red[0]);
}

// Canonical sign: the entry of largest modulus of each row is made positive.
__global__ void row_sign_kernel(double* __restrict__ X, int m, int n) {
  hs_pdl_enter();
  const int i = blockIdx.x;
  if (i >= m) return;
  double best = -1.0, val = 0.0;
  int bj = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = X[(long long)i * n + j];
    if (fabs(v) > best || (fabs(v) == best && j < bj)) {
      best = fabs(v);
      val = v;
      bj = j;
    }
  }
  __shared__ double sb[256], sv[256];
  __shared__ int sj[256];
  sb[threadIdx.x] = best;
  sv[threadIdx.x] = val;
  sj[threadIdx.x] = bj;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double b2 = sb[threadIdx.x + o];
      const int j2 = sj[threadIdx.x + o];
      if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && j2 < sj[threadIdx.x])) {
        sb[threadIdx.x] = b2;
        sv[threadIdx.x] = sv[threadIdx.x + o];
        sj[threadIdx.x] = j2;
      }
    }
    __syncthreads();
  }
  const double sgn = sv[0] < 0.0 ? -1.0 : 1.0;
  if (sgn < 0.0)
    for (int j = threadIdx.x; j < n; j += blockDim.x) X[(long long)i * n + j] = -X[(long long)i * n + j];
}

// Row i of a stacked pair (m0 rows of n0 entries, then rows of n1 entries):
// offset of its first entry and its length.
__device__ __forceinline__ void pair_row(int i, int m0, int n0, int n1, long long& off, int& n) {
  if (i < m0) {
    off = (long long)i * n0;
    n = n0;
  } else {
    off = (long long)m0 * n0 + (long long)(i - m0) * n1;
    n = n1;
  }
}

// row_sign_kernel over both blocks of a stacked pair (one CTA per row). The
// magnitudes compare as integers (IEEE bits without the sign) and the sign
// flips as a bit: FP64 compares and negations would take the FP64 pipe.
__global__ void row_sign_pair_kernel(double* __restrict__ X, int m0, int n0, int n1) {
  hs_pdl_enter();
  long long off;
  int n;
  pair_row(blockIdx.x, m0, n0, n1, off, n);
  unsigned long long* u = reinterpret_cast<unsigned long long*>(X + off);
  constexpr unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
  unsigned long long best = 0, val = 0;
  int bj = 0x7FFFFFFF;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const unsigned long long v = u[j], a = v & kMag;
    if (a > best || (a == best && j < bj)) {
      best = a;
      val = v;
      bj = j;
    }
  }
  __shared__ unsigned long long sb[256], sv[256];
  __shared__ int sj[256];
  sb[threadIdx.x] = best;
  sv[threadIdx.x] = val;
  sj[threadIdx.x] = bj;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const unsigned long long b2 = sb[threadIdx.x + o];
      const int j2 = sj[threadIdx.x + o];
      if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && j2 < sj[threadIdx.x])) {
        sb[threadIdx.x] = b2;
        sv[threadIdx.x] = sv[threadIdx.x + o];
        sj[threadIdx.x] = j2;
      }
    }
    __syncthreads();
  }
  if ((sv[0] >> 63) && sb[0] != 0)
    for (int j = threadIdx.x; j < n; j += blockDim.x) u[j] ^= 0x8000000000000000ull;
}

// residual_kernel over both blocks of a stacked pair (theta and res stacked).
__global__ void residual_pair_kernel(const double* __restrict__ Zr, const double* __restrict__ Xr,
                                     const float* __restrict__ theta, int m0, int n0, int n1,
                                     double* __restrict__ res) {
  hs_pdl_enter();
  const int i = blockIdx.x;
  long long off;
  int n;
  pair_row(i, m0, n0, n1, off, n);
  const double t = (double)theta[i];
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = Zr[off + j] - t * Xr[off + j];
    s += v * v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) res[i] = sqrt(red[0]);
}

// PT block b row j = X_b row idx[b][j]; P block b column j likewise.
__global__ void gather_rows_kernel(const double* __restrict__ X0, int n0, const double* __restrict__ X1, int n1,
                                   const int* __restrict__ idx, int chi, const SelectOut* __restrict__ sel,
                                   double* __restrict__ PT, double* __restrict__ P) {
  hs_pdl_enter();
  const int b = blockIdx.y, j = blockIdx.x;
  const int cb = sel->chi_new[b];
  if (j >= cb) return;
  const int n = b ? n1 : n0;
  const double* src = (b ? X1 : X0) + (long long)idx[b * chi + j] * n;
  const long long off = b ? (long long)sel->chi_new[0] * n0 : 0;
  double* prow = PT + off + (long long)j * n;
  double* pcol = P + off + j;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = src[i];
    prow[i] = v;
    pcol[(long long)i * cb] = v;
  }
}

// Indices of the m eigenvalues of largest modulus of one ascending spectrum
// (both ends of the array), in descending modulus.
__global__ void top_abs_kernel(const float* __restrict__ w, int n, int m, int* __restrict__ idx) {
  hs_pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int lo = 0, hi = n - 1;
  for (int j = 0; j < m && lo <= hi; ++j) {
    if (fabsf(w[lo]) > fabsf(w[hi])) idx[j] = lo++;
    else idx[j] = hi--;
  }
}

// row j of X (FP64, m x n) = column idx[j] of V (FP32, column-major n x n)
__global__ void rows_from_columns_kernel(const float* __restrict__ V, int n, const int* __restrict__ idx,
                                         double* __restrict__ X) {
  hs_pdl_enter();
  const int j = blockIdx.x;
  const float* src = V + (long long)idx[j] * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[(long long)j * n + i] = (double)src[i];
}

// Each row of X (m x n) scaled to unit Euclidean norm (zero rows untouched).
__global__ void row_normalize_kernel(double* __restrict__ X, int m, int n) {
  hs_pdl_enter();
  const int i = blockIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = X[(long long)i * n + j];
    s += v * v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double nrm = sqrt(red[0]);
  if (nrm > 0.0) {
    const double inv = 1.0 / nrm;
    for (int j = threadIdx.x; j < n; j += blockDim.x) X[(long long)i * n + j] *= inv;
  }
}

// out row i = X row idx[i], i < m (rows of n doubles).
__global__ void gather_rows_idx_kernel(const double* __restrict__ X, const int* __restrict__ idx, int n,
                                       double* __restrict__ out) {
  hs_pdl_enter();
  const long long src = (long long)idx[blockIdx.x] * n, dst = (long long)blockIdx.x * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) out[dst + j] = X[src + j];
}

// One term of the Chebyshev three-term recurrence on rows:
// Y = alpha (Z - T) + beta Yold, T and Yold optional (null: zero).
__global__ void cheb_step_kernel(double* __restrict__ Y, const double* __restrict__ Z, const double* __restrict__ T,
                                 const double* __restrict__ Yold, long long count, double alpha, double beta) {
  hs_pdl_enter();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    double v = Z[e];
    if (T) v -= T[e];
    v *= alpha;
    if (Yold) v += beta * Yold[e];
    Y[e] = v;
  }
}

// Stacked pair gather: out block b row i = X block b row idx[...]; CTA j <
// cnt0 takes block 0 (idx[j]), the rest block 1 (idx[j], rows of n1).
__global__ void gather_rows_idx_pair_kernel(const double* __restrict__ X, long long src_off1, int n0, int n1,
                                            const int* __restrict__ idx, int cnt0, double* __restrict__ out,
                                            long long dst_off1) {
  hs_pdl_enter();
  const int j = blockIdx.x, b = j >= cnt0;
  const int n = b ? n1 : n0;
  const long long src = (b ? src_off1 : 0) + (long long)idx[j] * n;
  const long long dst = (b ? dst_off1 : 0) + (long long)(j - (b ? cnt0 : 0)) * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) out[dst + k] = X[src + k];
}

// As gather_rows_idx_pair_kernel, each output row j multiplied by sgn[j].
__global__ void gather_rows_idx_sign_pair_kernel(const double* __restrict__ X, long long src_off1, int n0, int n1,
                                                 const int* __restrict__ idx, const double* __restrict__ sgn,
                                                 int cnt0, double* __restrict__ out, long long dst_off1) {
  hs_pdl_enter();
  const int j = blockIdx.x, b = j >= cnt0;
  const int n = b ? n1 : n0;
  const long long src = (b ? src_off1 : 0) + (long long)idx[j] * n;
  const long long dst = (b ? dst_off1 : 0) + (long long)(j - (b ? cnt0 : 0)) * n;
  const double f = sgn[j];
  for (int k = threadIdx.x; k < n; k += blockDim.x) out[dst + k] = f * X[src + k];
}

// cheb_step_kernel over a stacked pair: entries below count0 use alpha0.
__global__ void cheb_step_pair_kernel(double* __restrict__ Y, const double* __restrict__ Z,
                                      const double* __restrict__ T, const double* __restrict__ Yold, long long count,
                                      long long count0, double alpha0, double alpha1, double beta) {
  hs_pdl_enter();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    double v = Z[e];
    if (T) v -= T[e];
    v *= e < count0 ? alpha0 : alpha1;
    if (Yold) v += beta * Yold[e];
    Y[e] = v;
  }
}

// Symmetric eigen-decomposition of one small FP32 matrix by the cyclic Jacobi
// method (Golub and Van Loan, Sec. 8.5) with the round-robin ordering, so that
// the m/2 rotations of a round touch disjoint rows and columns and are applied
// together: A <- J^T A J, V <- V J. The Rayleigh matrices of the warm-started
// subspace iteration are nearly diagonal, where Jacobi converges
// quadratically in a few sweeps. Output as cuSOLVER's syevd: eigenvalues
// ascending in w, eigenvectors as the columns of the column-major m x m array
// A (overwritten). A rotation is skipped when |A_pq| <= tol sqrt|A_pp A_qq|,
// tol = max(4e-7, sqrt(m) eps_32) (the relative criterion of Demmel and
// Veselic, SIAM J. Matrix Anal. Appl. 13, 1992), or when |A_pq| is below
// 1e-7 max|A_ii| (FP32 rounding noise of the input); converged after a sweep
// without rotations. After kMaxSweeps without that, *status = 1.
//
// One cluster of kJacobiCtas CTAs per matrix. Every CTA of the cluster runs
// the same rotations on its own copy of A (identical arithmetic on identical
// data, so the copies and the convergence decision agree bit for bit) and
// accumulates V only for its slice of the eigenvector components: the work of
// a round is shared-memory bound, and V is the larger half of it. A is kept as
// its upper triangle, so a 2 x 2 block of a round is read and written once.
constexpr int kMaxSweeps = 40;
constexpr int kJacobiCtas = 8;

// Blocks (a, b), a <= b, of the pair grid that a thread updates in every
// round, packed a << 16 | b, and V entries (pair, component) packed the same
// way (at most kBlkPerThread and kVPerThread per thread).
constexpr int kBlkPerThread = 5;
constexpr int kVPerThread = 4;

// Pair k of round r in the round-robin ordering of M players (player M-1
// fixed, the others rotating), as (p, q) with p < q.
__device__ __forceinline__ int2 rr_pair(int k, int r, int M) {
  int p, q;
  if (k == 0) {
    p = r;
    q = M - 1;
  } else {
    p = r + k;
    if (p >= M - 1) p -= M - 1;
    q = r - k;
    if (q < 0) q += M - 1;
    if (p > q) {
      const int t = p;
      p = q;
      q = t;
    }
  }
  return make_int2(p, q);
}

__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}

__global__ void __launch_bounds__(1024) jacobi_eig_kernel(float* __restrict__ A0, int m0, float* __restrict__ w0,
                                                         float* __restrict__ A1, int m1, float* __restrict__ w1,
                                                         int* __restrict__ status) {
  hs_pdl_enter();
  const int mat = blockIdx.x / kJacobiCtas, g = cluster_rank();
  float* Ag = mat ? A1 : A0;
  float* wg = mat ? w1 : w0;
  const int m = mat ? m1 : m0;
  if (m <= 0) return;  // the whole cluster returns
  extern __shared__ float shj[];
  const int ld = m + 1;
  const int mc = (m + kJacobiCtas - 1) / kJacobiCtas;  // components per CTA
  const int i0 = g * mc, nc = max(0, min(m, i0 + mc) - i0);
  float* A = shj;                                           // upper triangle of m x ld
  float* Vt = A + m * ld;                                   // m x mc: Vt[j * mc + i] = component i0 + i of vector j
  float2* cs = reinterpret_cast<float2*>(Vt + ((m * mc + 1) & ~1));  // (cos, sin) per pair (8-byte aligned)
  const int M = (m + 1) & ~1;  // even player count (index m is a dummy when m is odd)
  const int npair = M / 2;
  const float kRelTol = fmaxf(4e-7f, sqrtf((float)m) * 6e-8f);
  __shared__ float dmax_part[32];
  float dm = 0.f;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    if (j < i) continue;
    const float v = 0.5f * (Ag[i * m + j] + Ag[j * m + i]);
    A[i * ld + j] = v;
    if (i == j) dm = fmaxf(dm, fabsf(v));
  }
  for (int e = threadIdx.x; e < m * mc; e += blockDim.x) {
    const int j = e / mc, i = e % mc;
    Vt[e] = i0 + i == j ? 1.f : 0.f;
  }
  // every CTA of the cluster has read Ag before any of them overwrites it
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if ((threadIdx.x & 31) == 0) dmax_part[threadIdx.x >> 5] = dm;
  // this thread's blocks of the upper block triangle, in row-major order
  int blk[kBlkPerThread];
  int nblk = 0;
  {
    int a = 0, off = 0;  // off: flat index of block (a, a); row a holds blocks b = a .. npair-1
#pragma unroll
    for (int t = 0; t < kBlkPerThread; ++t) {
      const int f = threadIdx.x + t * blockDim.x;
      blk[t] = -1;
      if (f < npair * (npair + 1) / 2) {
        while (f >= off + (npair - a)) {
          off += npair - a;
          ++a;
        }
        blk[t] = (a << 16) | (a + f - off);
        nblk = t + 1;
      }
    }
  }
  // this thread's V entries: pair b, local component i (consecutive threads
  // take consecutive components)
  int ven[kVPerThread];
  int nven = 0;
#pragma unroll
  for (int t = 0; t < kVPerThread; ++t) {
    const int f = threadIdx.x + t * blockDim.x;
    ven[t] = -1;
    if (nc > 0 && f < npair * nc) {
      ven[t] = ((f / nc) << 16) | (f % nc);
      nven = t + 1;
    }
  }
  __syncthreads();
  float dmax = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) dmax = fmaxf(dmax, dmax_part[w]);
  // off-diagonal entries below this are rounding noise of the FP32 matrix
  const float abs_floor = 1e-7f * dmax;
  bool converged = false;
  for (int sweep = 0; sweep < kMaxSweeps && !converged; ++sweep) {
    int nrot = 0;  // rotations in this sweep (the same in every thread)
    for (int r = 0; r < M - 1; ++r) {
      int rotates = 0;
      for (int k = threadIdx.x; k < npair; k += blockDim.x) {
        const int2 pq = rr_pair(k, r, M);
        float c = 1.f, sn = 0.f;
        if (pq.y < m) {
          const float apq = A[pq.x * ld + pq.y];
          const float app = A[pq.x * ld + pq.x], aqq = A[pq.y * ld + pq.y];
          // rotate unless A_pq is negligible against its diagonal pair
          if (fabsf(apq) > abs_floor && fabsf(apq) > 1e-30f && fabsf(apq) > kRelTol * sqrtf(fabsf(app * aqq))) {
            const float th = (aqq - app) / (2.f * apq);
            const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
            c = rsqrtf(t * t + 1.f);
            sn = t * c;
            rotates = 1;
          }
        }
        cs[k] = make_float2(c, sn);
      }
      const int rrot = __syncthreads_count(rotates);
      if (rrot == 0) continue;  // nothing rotates in this round (block-uniform)
      nrot += rrot;
      // A <- J^T A J: the rotations act on disjoint pairs, so every 2 x 2 block
      // (rows of pair a, columns of pair b) transforms on its own; an entry
      // lives at its upper-triangle position (min, max)
#pragma unroll
      for (int t = 0; t < kBlkPerThread; ++t) {
        if (t >= nblk) break;
        const int a = blk[t] >> 16, b = blk[t] & 0xffff;
        const float2 ra_ = cs[a], rb_ = cs[b];
        // neither pair rotates: the block stays as it is
        if (ra_.x == 1.f && ra_.y == 0.f && rb_.x == 1.f && rb_.y == 0.f) continue;
        const int2 ia = rr_pair(a, r, M), ib = rr_pair(b, r, M);
        const bool ra = ia.y < m, rb = ib.y < m;
        // (pa, pb), (pa, qb), (qa, pb), (qa, qb) at their upper positions
        const int e00 = min(ia.x, ib.x) * ld + max(ia.x, ib.x);
        const int e01 = min(ia.x, ib.y) * ld + max(ia.x, ib.y);
        const int e10 = min(ia.y, ib.x) * ld + max(ia.y, ib.x);
        const int e11 = min(ia.y, ib.y) * ld + max(ia.y, ib.y);
        const float a00 = A[e00];
        const float a01 = rb ? A[e01] : 0.f;
        const float a10 = ra ? A[e10] : 0.f;
        const float a11 = (ra && rb) ? A[e11] : 0.f;
        const float t00 = ra_.x * a00 - ra_.y * a10, t01 = ra_.x * a01 - ra_.y * a11;
        const float t10 = ra_.y * a00 + ra_.x * a10, t11 = ra_.y * a01 + ra_.x * a11;
        const float n00 = rb_.x * t00 - rb_.y * t01, n01 = rb_.y * t00 + rb_.x * t01;
        const float n10 = rb_.x * t10 - rb_.y * t11, n11 = rb_.y * t10 + rb_.x * t11;
        A[e00] = n00;
        if (rb) A[e01] = n01;
        // on the diagonal block (a == b) entry (qa, pa) is (pa, qa) again
        if (ra && a != b) A[e10] = n10;
        if (ra && rb) A[e11] = n11;
      }
      // V <- V J on this CTA's components
#pragma unroll
      for (int t = 0; t < kVPerThread; ++t) {
        if (t >= nven) break;
        const int b = ven[t] >> 16, i = ven[t] & 0xffff;
        const float2 rb_ = cs[b];
        if (rb_.x == 1.f && rb_.y == 0.f) continue;  // no rotation (or the dummy pair)
        const int2 ib = rr_pair(b, r, M);
        const float vp = Vt[ib.x * mc + i], vq = Vt[ib.y * mc + i];
        Vt[ib.x * mc + i] = rb_.x * vp - rb_.y * vq;
        Vt[ib.y * mc + i] = rb_.y * vp + rb_.x * vq;
      }
      __syncthreads();
    }
    converged = nrot == 0;  // a sweep without a rotation: every A_pq is negligible
  }
  if (!converged && g == 0 && threadIdx.x == 0) atomicExch(status, 1);
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  // ascending order by rank (ties by index); vectors as columns, column-major
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const float lj = A[j * ld + j];
    int rank = 0;
    for (int i = 0; i < m; ++i) {
      const float li = A[i * ld + i];
      rank += (li < lj) || (li == lj && i < j);
    }
    if (g == 0) wg[rank] = lj;
    for (int i = 0; i < nc; ++i) Ag[(long long)rank * m + i0 + i] = Vt[j * mc + i];
  }
}

}  // namespace

size_t jacobi_smem_bytes(int m) {
  const int mc = (m + kJacobiCtas - 1) / kJacobiCtas;
  return (size_t)(m * (m + 1) + ((m * mc + 1) & ~1)) * sizeof(float) + (size_t)((m + 1) / 2 + 1) * sizeof(float2);
}

cudaError_t launch_jacobi_eig_pair(float* A0, int m0, float* w0, float* A1, int m1, float* w1, int* status,
                                   cudaStream_t s) {
  const int m = m0 > m1 ? m0 : m1;
  if (m <= 0) return cudaSuccess;
  // m <= kMaxSub keeps the (m/2)(m/2 + 1)/2 blocks of a round within kBlkPerThread per thread
  // and the (m/2) ceil(m / kJacobiCtas) V entries within kVPerThread
  static_assert((kMaxSub / 2 + 1) * (kMaxSub / 2 + 2) / 2 <= kBlkPerThread * 1024, "block grid too large");
  static_assert((kMaxSub / 2 + 1) * ((kMaxSub + kJacobiCtas - 1) / kJacobiCtas) <= kVPerThread * 1024,
                "V slice too large");
  if (m > kMaxSub) return cudaErrorInvalidValue;
  // set once per device
  const cudaError_t attr_err =
      ensure_smem_attr(reinterpret_cast<const void*>(jacobi_eig_kernel), (int)jacobi_smem_bytes(kMaxSub));
  if (attr_err != cudaSuccess) return attr_err;
  hs_launch_cluster(jacobi_eig_kernel, 2 * kJacobiCtas, 1024, jacobi_smem_bytes(m), s, kJacobiCtas, A0, m0, w0, A1,
                    m1, w1, status);
  return cudaGetLastError();
}

cudaError_t launch_row_normalize(double* X, int m, int n, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  hs_launch(row_normalize_kernel, m, 256, 0, s, X, m, n);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows_idx(const double* X, const int* idx, int m, int n, double* out, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  hs_launch(gather_rows_idx_kernel, m, 256, 0, s, X, idx, n, out);
  return cudaGetLastError();
}

cudaError_t launch_cheb_step(double* Y, const double* Z, const double* T, const double* Yold, long long count,
                             double alpha, double beta, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  hs_launch(cheb_step_kernel, grid_for(count), 256, 0, s, Y, Z, T, Yold, count, alpha, beta);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows_idx_pair(const double* X, long long src_off1, int n0, int n1, const int* idx,
                                        int cnt0, int cnt1, double* out, long long dst_off1, cudaStream_t s) {
  if (cnt0 + cnt1 <= 0) return cudaSuccess;
  hs_launch(gather_rows_idx_pair_kernel, cnt0 + cnt1, 256, 0, s, X, src_off1, n0, n1, idx, cnt0, out, dst_off1);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows_idx_sign_pair(const double* X, long long src_off1, int n0, int n1, const int* idx,
                                             const double* sgn, int cnt0, int cnt1, double* out, long long dst_off1,
                                             cudaStream_t s) {
  if (cnt0 + cnt1 <= 0) return cudaSuccess;
  hs_launch(gather_rows_idx_sign_pair_kernel, cnt0 + cnt1, 256, 0, s, X, src_off1, n0, n1, idx, sgn, cnt0, out,
            dst_off1);
  return cudaGetLastError();
}

cudaError_t launch_cheb_step_pair(double* Y, const double* Z, const double* T, const double* Yold, long long count,
                                  long long count0, double alpha0, double alpha1, double beta, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  hs_launch(cheb_step_pair_kernel, grid_for(count), 256, 0, s, Y, Z, T, Yold, count, count0, alpha0, alpha1, beta);
  return cudaGetLastError();
}

cudaError_t launch_top_rows(const float* w, const float* V, int n, int m, int* idx, double* X, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  hs_launch(top_abs_kernel, 1, 32, 0, s, w, n, m, idx);
  hs_launch(rows_from_columns_kernel, m, 256, 0, s, V, n, idx, X);
  return cudaGetLastError();
}

cudaError_t launch_fill_random_rows(double* X, int r0, int m, int n, unsigned long long seed, cudaStream_t s) {
  if (r0 >= m) return cudaSuccess;
  hs_launch(fill_random_rows_kernel, grid_for((long long)(m - r0) * n), 256, 0, s, X, r0, m, n, seed);
  return cudaGetLastError();
}

cudaError_t launch_chol_inv(const double* G0, int m0, double* Linv0, const double* G1, int m1, double* Linv1,
                            int* status, cudaStream_t s) {
  if (m0 < 0 || m1 < 0 || m0 > kMaxChol || m1 > kMaxChol) return cudaErrorInvalidValue;
  if (m0 == 0 && m1 == 0) return cudaSuccess;
  const int mm = m0 > m1 ? m0 : m1;
  const size_t smem = (size_t)mm * (mm + 1) * sizeof(double);
  // set once per device
  const cudaError_t attr_err = ensure_smem_attr(reinterpret_cast<const void*>(chol_inv_kernel),
                                                kMaxChol * (kMaxChol + 1) * (int)sizeof(double));
  if (attr_err != cudaSuccess) return attr_err;
  hs_launch(chol_inv_kernel, 2, 1024, smem, s, G0, m0, Linv0, G1, m1, Linv1, status);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* Zr, const double* Xr, const float* theta, int m, int n, double* res,
                            cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  hs_launch(residual_kernel, m, 256, 0, s, Zr, Xr, theta, m, n, res);
  return cudaGetLastError();
}

cudaError_t launch_row_sign_pair(double* X, int m0, int n0, int m1, int n1, cudaStream_t s) {
  if (m0 + m1 <= 0) return cudaSuccess;
  hs_launch(row_sign_pair_kernel, m0 + m1, 256, 0, s, X, m0, n0, n1);
  return cudaGetLastError();
}

cudaError_t launch_residual_pair(const double* Zr, const double* Xr, const float* theta, int m0, int n0, int m1,
                                 int n1, double* res, cudaStream_t s) {
  if (m0 + m1 <= 0) return cudaSuccess;
  hs_launch(residual_pair_kernel, m0 + m1, 256, 0, s, Zr, Xr, theta, m0, n0, n1, res);
  return cudaGetLastError();
}

cudaError_t launch_row_sign(double* X, int m, int n, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  hs_launch(row_sign_kernel, m, 256, 0, s, X, m, n);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double* X0, int n0, const double* X1, int n1, const int* idx, int chi,
                               const SelectOut* sel, double* PT, double* P, cudaStream_t s) {
  dim3 grid((unsigned)chi, 2);
  hs_launch(gather_rows_kernel, grid, 256, 0, s, X0, n0, X1, n1, idx, chi, sel, PT, P);
  return cudaGetLastError();
}

namespace {
// Rows of a parity block of C' over [(alpha, x)] (FSO order of fused2(c, q),
// parity b) carried from boundary sectors c_old to c_new: entry (alpha, x) of
// sector tuple (p_alpha, p_x) keeps its value when alpha < c_old[p_alpha] (the
// kept states of a sector are in pick order, largest |eigenvalue| first, so
// the first ones correspond), and is zero for a state the old boundary did not
// have.
__global__ void remap_rows_kernel(const double* __restrict__ src, int rows, int old_n, double* __restrict__ dst,
                                  int new_n, int b, Sect c_old, Sect c_new, Sect q) {
  hs_pdl_enter();
  const Fused fo = fused2(c_old, q), fn = fused2(c_new, q);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)rows * new_n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / new_n), j = (int)(e % new_n);
    double v = 0.0;
    for (int t = 0; t < 4; ++t) {
      if (tuple_parity(t) != b) continue;
      const long long off = tuple_offset(fn, t), size = tuple_size(fn, t);
      if (j < off || j >= off + size) continue;
      const int pa = tuple_bit(t, 2, 0), px = tuple_bit(t, 2, 1);
      const int al = (int)((j - off) / q.n[px]), xl = (int)((j - off) % q.n[px]);
      if (al < c_old.n[pa]) v = src[(long long)r * old_n + tuple_offset(fo, t) + (long long)al * q.n[px] + xl];
    }
    dst[e] = v;
  }
}
}  // namespace

namespace {
// X (rows x n) += amp * seeded uniform noise in (-1, 1)
__global__ void perturb_rows_kernel(double* __restrict__ X, int rows, int n, double amp, unsigned long long seed) {
  hs_pdl_enter();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)rows * n;
       e += (long long)gridDim.x * blockDim.x)
    X[e] += amp * hash_uniform(seed * 0x100000001B3ull + (unsigned long long)e);
}
}  // namespace

cudaError_t launch_remap_rows(const double* src, int rows, int old_n, double* dst, int new_n, int b, Sect c_old,
                              Sect c_new, Sect q, unsigned long long seed, cudaStream_t s) {
  if (rows <= 0 || new_n <= 0) return cudaSuccess;
  hs_launch(remap_rows_kernel, grid_for((long long)rows * new_n), 256, 0, s, src, rows, old_n, dst, new_n, b, c_old,
            c_new, q);
  // a row that lived mostly on states the new boundary lacks is left nearly
  // zero: a little noise (about 1% of an entry of a unit row) keeps the rows
  // independent for the Cholesky-QR that follows
  hs_launch(perturb_rows_kernel, grid_for((long long)rows * new_n), 256, 0, s, dst, rows, new_n,
            0.01 / sqrt((double)new_n), seed);
  return cudaGetLastError();
}

int max_subspace() { return kMaxSub; }
int max_chol() { return kMaxChol; }

namespace {
// Row-major L^{-1} from the library route: zero the entries above the
// diagonal (left over from G) and raise *bad if the factorisation or the
// inversion failed (info[0], info[1]).
__global__ void tidy_linv_kernel(double* __restrict__ L, int m, const int* __restrict__ info, int* __restrict__ bad) {
  hs_pdl_enter();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * m;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), c = (int)(e % m);
    if (c > i) L[e] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (info[0] != 0 || info[1] != 0)) *bad = 1;
}
}  // namespace

cudaError_t launch_tidy_linv(double* L, int m, const int* info, int* bad, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  long long g = ((long long)m * m + 255) / 256;
  if (g > 1024) g = 1024;
  hs_launch(tidy_linv_kernel, (unsigned)g, 256, 0, s, L, m, info, bad);
  return cudaGetLastError();
}

}  // namespace hs

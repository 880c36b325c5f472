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
  const long long total = (long long)(m - r0) * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    X[(long long)r0 * n + e] = hash_uniform(seed * 0x100000001B3ull + (unsigned long long)e);
}

// In-place Cholesky G = L L^T (lower) of an m x m SPD matrix and L^{-1}, in
// FP64, by one CTA in shared memory (m <= kMaxSub). On a non-positive pivot
// the status word is set and Linv is left unspecified.
constexpr int kMaxSub = 160;

__global__ void __launch_bounds__(256) chol_inv_kernel(const double* __restrict__ G, int m,
                                                       double* __restrict__ Linv, int* __restrict__ status) {
  extern __shared__ double sh[];
  double* L = sh;  // m x m, lower triangle used
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e / m, c = e % m;
    L[e] = r >= c ? 0.5 * (G[r * m + c] + G[c * m + r]) : 0.0;
  }
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      const double d = L[j * m + j];
      if (!(d > 0.0)) bad = 1;
      L[j * m + j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double piv = L[j * m + j];
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) L[i * m + j] /= piv;
    __syncthreads();
    // trailing update of the lower triangle
    const int rem = m - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int r = j + 1 + e / rem, c = j + 1 + e % rem;
      if (c <= r) L[r * m + c] -= L[r * m + j] * L[c * m + j];
    }
    __syncthreads();
  }
  // L^{-1} by forward substitution, one column of the identity per thread,
  // built directly in Linv (each thread reads and writes only its column)
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    for (int r = 0; r < m; ++r) {
      double v = r == c ? 1.0 : 0.0;
      for (int k = c; k < r; ++k) v -= L[r * m + k] * Linv[k * m + c];
      Linv[r * m + c] = r < c ? 0.0 : v / L[r * m + r];
    }
  }
  if (threadIdx.x == 0 && bad) *status = 1;
}

// res[i] = || Zr_i - theta_i Xr_i || for the m rows (theta from FP32 values).
__global__ void residual_kernel(const double* __restrict__ Zr, const double* __restrict__ Xr,
                                const float* __restrict__ theta, int m, int n, double* __restrict__ res) {
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

// PT block b row j = X_b row idx[b][j]; P block b column j likewise.
__global__ void gather_rows_kernel(const double* __restrict__ X0, int n0, const double* __restrict__ X1, int n1,
                                   const int* __restrict__ idx, int chi, const SelectOut* __restrict__ sel,
                                   double* __restrict__ PT, double* __restrict__ P) {
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
  const int j = blockIdx.x;
  const float* src = V + (long long)idx[j] * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[(long long)j * n + i] = (double)src[i];
}

// Each row of X (m x n) scaled to unit Euclidean norm (zero rows untouched).
__global__ void row_normalize_kernel(double* __restrict__ X, int m, int n) {
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
  if (nrm > 0.0)
    for (int j = threadIdx.x; j < n; j += blockDim.x) X[(long long)i * n + j] /= nrm;
}

// out row i = X row idx[i], i < m (rows of n doubles).
__global__ void gather_rows_idx_kernel(const double* __restrict__ X, const int* __restrict__ idx, int n,
                                       double* __restrict__ out) {
  const long long src = (long long)idx[blockIdx.x] * n, dst = (long long)blockIdx.x * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) out[dst + j] = X[src + j];
}

// One term of the Chebyshev three-term recurrence on rows:
// Y = alpha (Z - T) + beta Yold, T and Yold optional (null: zero).
__global__ void cheb_step_kernel(double* __restrict__ Y, const double* __restrict__ Z, const double* __restrict__ T,
                                 const double* __restrict__ Yold, long long count, double alpha, double beta) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    double v = Z[e];
    if (T) v -= T[e];
    v *= alpha;
    if (Yold) v += beta * Yold[e];
    Y[e] = v;
  }
}

// Symmetric eigen-decomposition of one small FP32 matrix per CTA by the
// cyclic Jacobi method (Golub and Van Loan, Sec. 8.5) with the round-robin
// ordering, so that the m/2 rotations of a round touch disjoint rows and
// columns and are applied together: A <- J^T A J, V <- V J. The Rayleigh
// matrices of the warm-started subspace iteration are nearly diagonal, where
// Jacobi converges quadratically in a few sweeps. Output as cuSOLVER's syevd:
// eigenvalues ascending in w, eigenvectors as the columns of the column-major
// m x m array A (overwritten). A rotation is skipped when |A_pq| <= tol
// sqrt|A_pp A_qq|, tol = max(4e-7, sqrt(m) eps_32) (the relative criterion of
// Demmel and Veselic, SIAM J. Matrix Anal. Appl. 13, 1992), or when |A_pq| is
// below 1e-7 max|A_ii| (FP32 rounding noise of the input); converged after a
// sweep without rotations.
// After kMaxSweeps without that, *status = 1.
constexpr int kMaxSweeps = 40;

__global__ void __launch_bounds__(1024) jacobi_eig_kernel(float* __restrict__ A0, int m0, float* __restrict__ w0,
                                                         float* __restrict__ A1, int m1, float* __restrict__ w1,
                                                         int* __restrict__ status) {
  float* Ag = blockIdx.x ? A1 : A0;
  float* wg = blockIdx.x ? w1 : w0;
  const int m = blockIdx.x ? m1 : m0;
  if (m <= 0) return;
  extern __shared__ float shj[];
  const int ld = m + 1;
  float* A = shj;                 // m x ld
  float* V = A + m * ld;          // m x ld, V[i * ld + j] = component i of vector j
  float* cs = V + m * ld;         // cos, sin per pair
  int* pq = reinterpret_cast<int*>(cs + 2 * ((m + 1) / 2 + 1));
  __shared__ int nrot, rrot;
  const int M = (m + 1) & ~1;     // even player count (index m is a dummy when m is odd)
  const int npair = M / 2;
  const float kRelTol = fmaxf(4e-7f, sqrtf((float)m) * 6e-8f);
  __shared__ float dmax_part[32];
  float dm = 0.f;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    const float v = 0.5f * (Ag[i * m + j] + Ag[j * m + i]);
    A[i * ld + j] = v;
    V[i * ld + j] = i == j ? 1.f : 0.f;
    if (i == j) dm = fmaxf(dm, fabsf(v));
  }
  for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if ((threadIdx.x & 31) == 0) dmax_part[threadIdx.x >> 5] = dm;
  __syncthreads();
  float dmax = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) dmax = fmaxf(dmax, dmax_part[w]);
  // off-diagonal entries below this are rounding noise of the FP32 matrix
  const float abs_floor = 1e-7f * dmax;
  bool converged = false;
  for (int sweep = 0; sweep < kMaxSweeps && !converged; ++sweep) {
    if (threadIdx.x == 0) nrot = 0;
    __syncthreads();
    for (int r = 0; r < M - 1; ++r) {
      if (threadIdx.x == 0) rrot = 0;
      __syncthreads();
      // round-robin pairing: player M-1 fixed, the others rotate
      for (int k = threadIdx.x; k < npair; k += blockDim.x) {
        int p = k == 0 ? M - 1 : (r + k) % (M - 1);
        int q = (r + M - 1 - k) % (M - 1);
        if (k == 0) q = r;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        float c = 1.f, sn = 0.f;
        if (q < m) {
          const float apq = A[p * ld + q];
          const float app = A[p * ld + p], aqq = A[q * ld + q];
          // rotate unless A_pq is negligible against its diagonal pair
          if (fabsf(apq) > abs_floor && fabsf(apq) > 1e-30f && fabsf(apq) > kRelTol * sqrtf(fabsf(app * aqq))) {
            const float th = (aqq - app) / (2.f * apq);
            const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
            c = rsqrtf(t * t + 1.f);
            sn = t * c;
            atomicAdd(&rrot, 1);
          }
        }
        pq[2 * k] = p;
        pq[2 * k + 1] = q;
        cs[2 * k] = c;
        cs[2 * k + 1] = sn;
      }
      __syncthreads();
      if (rrot == 0) continue;  // nothing rotates in this round (block-uniform)
      if (threadIdx.x == 0) nrot += rrot;
      // A <- J^T A J: the rotations act on disjoint pairs, so every 2 x 2 block
      // (rows of pair a, columns of pair b) transforms on its own; V <- V J
      const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int a = threadIdx.x >> 5; a < npair; a += nw) {
        const int pa = pq[2 * a], qa = pq[2 * a + 1];
        const float ca = cs[2 * a], sa = cs[2 * a + 1];
        const bool ra = qa < m;
        for (int b = lane; b < npair; b += 32) {
          const int pb = pq[2 * b], qb = pq[2 * b + 1];
          const float cb = cs[2 * b], sb = cs[2 * b + 1];
          const bool rb = qb < m;
          const float a00 = A[pa * ld + pb];
          const float a01 = rb ? A[pa * ld + qb] : 0.f;
          const float a10 = ra ? A[qa * ld + pb] : 0.f;
          const float a11 = (ra && rb) ? A[qa * ld + qb] : 0.f;
          const float t00 = ca * a00 - sa * a10, t01 = ca * a01 - sa * a11;
          const float t10 = sa * a00 + ca * a10, t11 = sa * a01 + ca * a11;
          A[pa * ld + pb] = cb * t00 - sb * t01;
          if (rb) A[pa * ld + qb] = sb * t00 + cb * t01;
          if (ra) A[qa * ld + pb] = cb * t10 - sb * t11;
          if (ra && rb) A[qa * ld + qb] = sb * t10 + cb * t11;
        }
      }
      for (int i = threadIdx.x >> 5; i < m; i += nw) {
        for (int b = lane; b < npair; b += 32) {
          const int pb = pq[2 * b], qb = pq[2 * b + 1];
          if (qb >= m) continue;
          const float cb = cs[2 * b], sb = cs[2 * b + 1];
          const float vp = V[i * ld + pb], vq = V[i * ld + qb];
          V[i * ld + pb] = cb * vp - sb * vq;
          V[i * ld + qb] = sb * vp + cb * vq;
        }
      }
      __syncthreads();
    }
    converged = nrot == 0;  // a sweep without a rotation: every A_pq is negligible
    __syncthreads();
  }
  if (!converged && threadIdx.x == 0) atomicExch(status, 1);
  // ascending order by rank (ties by index); vectors as columns, column-major
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const float lj = A[j * ld + j];
    int rank = 0;
    for (int i = 0; i < m; ++i) {
      const float li = A[i * ld + i];
      rank += (li < lj) || (li == lj && i < j);
    }
    wg[rank] = lj;
    for (int i = 0; i < m; ++i) Ag[(long long)rank * m + i] = V[i * ld + j];
  }
}

}  // namespace

size_t jacobi_smem_bytes(int m) {
  return (size_t)(2 * m * (m + 1) + 2 * ((m + 1) / 2 + 1)) * sizeof(float) + (size_t)((m + 1) / 2 + 1) * 2 * sizeof(int);
}

cudaError_t launch_jacobi_eig_pair(float* A0, int m0, float* w0, float* A1, int m1, float* w1, int* status,
                                   cudaStream_t s) {
  const int m = m0 > m1 ? m0 : m1;
  if (m <= 0) return cudaSuccess;
  if (m > kMaxSub) return cudaErrorInvalidValue;
  // set once per process (thread-safe static initialisation)
  static const cudaError_t attr_err = cudaFuncSetAttribute(jacobi_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)jacobi_smem_bytes(kMaxSub));
  if (attr_err != cudaSuccess) return attr_err;
  jacobi_eig_kernel<<<2, 1024, jacobi_smem_bytes(m), s>>>(A0, m0, w0, A1, m1, w1, status);
  return cudaGetLastError();
}

cudaError_t launch_row_normalize(double* X, int m, int n, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  row_normalize_kernel<<<m, 256, 0, s>>>(X, m, n);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows_idx(const double* X, const int* idx, int m, int n, double* out, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  gather_rows_idx_kernel<<<m, 256, 0, s>>>(X, idx, n, out);
  return cudaGetLastError();
}

cudaError_t launch_cheb_step(double* Y, const double* Z, const double* T, const double* Yold, long long count,
                             double alpha, double beta, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  cheb_step_kernel<<<grid_for(count), 256, 0, s>>>(Y, Z, T, Yold, count, alpha, beta);
  return cudaGetLastError();
}

cudaError_t launch_top_rows(const float* w, const float* V, int n, int m, int* idx, double* X, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  top_abs_kernel<<<1, 32, 0, s>>>(w, n, m, idx);
  rows_from_columns_kernel<<<m, 256, 0, s>>>(V, n, idx, X);
  return cudaGetLastError();
}

cudaError_t launch_fill_random_rows(double* X, int r0, int m, int n, unsigned long long seed, cudaStream_t s) {
  if (r0 >= m) return cudaSuccess;
  fill_random_rows_kernel<<<grid_for((long long)(m - r0) * n), 256, 0, s>>>(X, r0, m, n, seed);
  return cudaGetLastError();
}

cudaError_t launch_chol_inv(const double* G, int m, double* Linv, int* status, cudaStream_t s) {
  if (m <= 0 || m > kMaxSub) return cudaErrorInvalidValue;
  const size_t smem = (size_t)m * m * sizeof(double);
  // set once per process (thread-safe static initialisation)
  static const cudaError_t attr_err = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxSub * kMaxSub * (int)sizeof(double));
  if (attr_err != cudaSuccess) return attr_err;
  chol_inv_kernel<<<1, 256, smem, s>>>(G, m, Linv, status);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* Zr, const double* Xr, const float* theta, int m, int n, double* res,
                            cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  residual_kernel<<<m, 256, 0, s>>>(Zr, Xr, theta, m, n, res);
  return cudaGetLastError();
}

cudaError_t launch_row_sign(double* X, int m, int n, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  row_sign_kernel<<<m, 256, 0, s>>>(X, m, n);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double* X0, int n0, const double* X1, int n1, const int* idx, int chi,
                               const SelectOut* sel, double* PT, double* P, cudaStream_t s) {
  dim3 grid((unsigned)chi, 2);
  gather_rows_kernel<<<grid, 256, 0, s>>>(X0, n0, X1, n1, idx, chi, sel, PT, P);
  return cudaGetLastError();
}

int max_subspace() { return kMaxSub; }

}  // namespace hs

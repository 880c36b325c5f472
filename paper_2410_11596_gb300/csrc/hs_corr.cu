// Correlation length of a converged real C4v environment (an observable of
// Sec. III; the paper reports energies and spectra, the correlation length
// is the standard companion quantity): xi = -1 / ln|lambda_2 / lambda_1| of
// the column transfer matrix
//   E[(alpha, l, beta), (alpha', r, beta')] = sum_{u,d} T[alpha,u,alpha'] a[u,l,d,r] T[beta',d,beta]
// (top edge left to right, bottom edge right to left). For real C4v tensors
// E is symmetric, so its extremal eigenvalues come from a Lanczos iteration
// with full re-orthogonalisation: the vectors live on the device, E v is three
// dense GEMMs and two permutes in the plain combined basis, and the small
// tridiagonal eigenproblem is solved on the host by Jacobi rotations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hs_ctx.cuh"

namespace hs {
namespace {

unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// out[j] = <V_j, w> for the m rows of V (n long); one block per row
__global__ void multi_dot_kernel(const double* __restrict__ V, int m, long long n, const double* __restrict__ w,
                                 double* __restrict__ out) {
  hs_pdl_enter();
  const int j = blockIdx.x;
  if (j >= m) return;
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += V[j * n + i] * w[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

// w -= sum_j c[j] V_j
__global__ void multi_axpy_kernel(const double* __restrict__ V, int m, long long n, const double* __restrict__ c,
                                  double* __restrict__ w) {
  hs_pdl_enter();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s += c[j] * V[j * n + i];
    w[i] -= s;
  }
}

// dst = src * f
__global__ void scale_copy_kernel(const double* __restrict__ src, double f, long long n, double* __restrict__ dst) {
  hs_pdl_enter();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i] * f;
}

// seeded start vector (splitmix64 -> uniform in (-1, 1))
__global__ void start_vector_kernel(double* __restrict__ v, long long n) {
  hs_pdl_enter();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long x = (unsigned long long)i + 0x9E3779B97F4A7C15ull * 7;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    v[i] = (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

// eigenvalues of a small symmetric matrix (row-major, m x m) by cyclic Jacobi
std::vector<double> host_sym_eigvals(std::vector<double> A, int m) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) (i == j ? dia : off) += A[i * m + j] * A[i * m + j];
    if (off <= 1e-30 * dia) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[p * m + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double th = (A[q * m + q] - A[p * m + p]) / (2 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1));
        const double c = 1 / std::sqrt(t * t + 1), s = t * c;
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double ap = A[p * m + k], aq = A[q * m + k];
          A[p * m + k] = c * ap - s * aq;
          A[q * m + k] = s * ap + c * aq;
        }
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double ap = A[k * m + p], aq = A[k * m + q];
          A[k * m + p] = c * ap - s * aq;
          A[k * m + q] = s * ap + c * aq;
        }
      }
  }
  std::vector<double> w(m);
  for (int i = 0; i < m; ++i) w[i] = A[i * m + i];
  return w;
}

Z2Mat dmat(std::initializer_list<long long> rows, std::initializer_list<long long> cols) {
  Fused r = fused0(), c = fused0();
  for (long long v : rows) r.leg[r.k++] = make_sect((int)v, 0);
  for (long long v : cols) c.leg[c.k++] = make_sect((int)v, 0);
  return mat(r, c);
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" hs_status hs_correlation_length(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, int max_iter,
                                           double tol, double* lam_out, double* xi_out) {
  HS_TRY(check_ctx(ctx));
  if (!env || !A || !lam_out || !xi_out || d <= 0 || D != env->D || max_iter < 4 || max_iter > 400 || !(tol > 0))
    return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (env->dtype != HS_F64) return fail(HS_ERR_UNSUPPORTED, "the correlation length needs a real environment");
  cudaStream_t s = ctx->stream;
  const long long chi = env->chi_even + env->chi_odd, q = (long long)D * D;
  const long long n = chi * q * chi;
  const hs_precision prec = env->precision;
  // dense plain-basis T, a and their operand layouts
  DBuf* r = ctx->hb;
  HS_TRY(r[9].ensure(chi * chi * 8));
  HS_TRY(r[10].ensure(n * 8));
  HS_TRY(r[11].ensure(n * 8));
  HS_TRY(r[12].ensure(q * q * q * q * 8));
  HS_TRY(r[13].ensure(q * q * q * q * 8));
  HS_TRY(r[14].ensure(chi * q * q * chi * 8));
  HS_TRY(r[15].ensure(chi * q * q * chi * 8));
  double *Td = r[10].d(), *TB = r[11].d(), *ad = r[12].d(), *aB = r[13].d(), *W1 = r[14].d(), *W2 = r[15].d();
  HS_CUDA(launch_env_to_dense(env->C, env->T, D, env->chi_even, env->chi_odd, env->basis == HS_BASIS_HERMITIAN,
                              r[9].d(), Td, s));
  HS_CUDA(launch_double_layer_dense(A, d, D, false, ad, s));
  HS_TRY(permute(ctx, dmat({q, q}, {q, q}), dmat({q, q}, {q, q}), {1, 2, 0, 3}, ad, aB));         // [(l,d)|(u,r)]
  HS_TRY(permute(ctx, dmat({chi, q}, {chi}), dmat({chi}, {chi, q}), {2, 0, 1}, Td, TB));          // [b|(b',d)]
  // Lanczos basis (rows) and work vectors
  const int mmax = max_iter + 1;
  HS_TRY(ctx->gb[7].ensure((size_t)mmax * n * 8));
  HS_TRY(ctx->gb[8].ensure(n * 8));
  HS_TRY(ctx->gb[9].ensure(n * 8));
  HS_TRY(ctx->gb[10].ensure((size_t)(mmax + 1) * 8));
  double *V = ctx->gb[7].d(), *w = ctx->gb[8].d(), *vt = ctx->gb[9].d(), *coef = ctx->gb[10].d();
  auto matvec = [&](const double* v, double* out) -> hs_status {
    HS_TRY(permute(ctx, dmat({chi, q}, {chi}), dmat({q, chi}, {chi}), {1, 2, 0}, v, vt));          // [(r,b')|a']
    HS_TRY(dense_gemm_any(ctx, prec, (int)(chi * q), (int)(q * chi), (int)chi, Td, vt, W1));     // [(a,u)|(r,b')]
    HS_TRY(permute(ctx, dmat({chi, q}, {q, chi}), dmat({chi, chi}, {q, q}), {0, 3, 1, 2}, W1, W2)); // [(a,b')|(u,r)]
    HS_TRY(dense_gemm_any(ctx, prec, (int)(chi * chi), (int)(q * q), (int)(q * q), W2, aB, W1));  // [(a,b')|(l,d)]
    HS_TRY(permute(ctx, dmat({chi, chi}, {q, q}), dmat({chi, q}, {chi, q}), {0, 2, 1, 3}, W1, W2)); // [(a,l)|(b',d)]
    return dense_gemm_any(ctx, prec, (int)(chi * q), (int)chi, (int)(chi * q), W2, TB, out);     // [(a,l)|b]
  };
  auto norm = [&](const double* x) -> double {
    hs_launch(multi_dot_kernel, 1, 256, 0, s, x, 1, n, x, coef);
    double h = 0.0;
    cudaMemcpyAsync(&h, coef, 8, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return std::sqrt(h);
  };
  hs_launch(start_vector_kernel, grid_for(n), 256, 0, s, w, n);
  HS_CUDA(cudaGetLastError());
  double nb = norm(w);
  hs_launch(scale_copy_kernel, grid_for(n), 256, 0, s, w, 1.0 / nb, n, V);
  std::vector<double> alpha, beta;
  std::vector<double> c(mmax + 1);
  double l1 = 0.0, l2 = 0.0, l1_old = -1.0, l2_old = -1.0;
  bool converged = false;
  for (int j = 0; j < max_iter; ++j) {
    HS_TRY(matvec(V + (long long)j * n, w));
    // full re-orthogonalisation against V_0..V_j, twice (classical Gram-Schmidt)
    double a_j = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      hs_launch(multi_dot_kernel, j + 1, 256, 0, s, V, j + 1, n, w, coef);
      HS_CUDA(cudaMemcpyAsync(c.data(), coef, (j + 1) * 8, cudaMemcpyDeviceToHost, s));
      HS_CUDA(cudaStreamSynchronize(s));
      if (pass == 0) a_j = c[j];
      else a_j += c[j];
      hs_launch(multi_axpy_kernel, grid_for(n), 256, 0, s, V, j + 1, n, coef, w);
    }
    alpha.push_back(a_j);
    const double b = norm(w);
    // eigenvalues of the tridiagonal matrix so far
    const int m = (int)alpha.size();
    std::vector<double> Tm((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) {
      Tm[i * m + i] = alpha[i];
      if (i + 1 < m) Tm[i * m + i + 1] = Tm[(i + 1) * m + i] = beta[i];
    }
    std::vector<double> th = host_sym_eigvals(Tm, m);
    std::sort(th.begin(), th.end(), [](double x, double y) { return std::fabs(x) > std::fabs(y); });
    l1 = std::fabs(th[0]);
    l2 = m > 1 ? std::fabs(th[1]) : 0.0;
    if (m >= 4 && std::fabs(l1 - l1_old) <= tol * l1 && std::fabs(l2 - l2_old) <= tol * l1) {
      converged = true;
      break;
    }
    l1_old = l1;
    l2_old = l2;
    if (!(b > 1e-14 * l1)) {  // invariant subspace found: the Ritz values are exact
      converged = true;
      break;
    }
    beta.push_back(b);
    hs_launch(scale_copy_kernel, grid_for(n), 256, 0, s, w, 1.0 / b, n, V + (long long)(j + 1) * n);
  }
  HS_CUDA(cudaGetLastError());
  lam_out[0] = l1;
  lam_out[1] = l2;
  *xi_out = (l2 <= 0.0) ? 0.0 : (l2 >= l1 ? INFINITY : -1.0 / std::log(l2 / l1));
  if (!converged) return fail(HS_ERR_TIMEOUT, "Lanczos did not converge in %d iterations", max_iter);
  return HS_OK;
}

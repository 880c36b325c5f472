// Normalised corner spectrum of a CTMRG environment (arXiv 2410.11596
// Sec. III.A, the gauge-invariant spectrum of the corner C): the singular
// values of C divided by the largest, in descending order, computed on the
// GPU.
//
// Real environments: C is block diagonal in the boundary parity (Sec. II.B),
// so its singular values are those of the two blocks; one FP64 SVD per block
// (cuSOLVER gesvd, values only), then a merge kernel. Complex (graded)
// environments: C = J M J with J = diag(1, i) by parity (Sec. II.C), M the
// stored matrix with its odd-odd block negated; J is unitary, so the singular
// values of C are those of the real M.
#include "hs_ctx.cuh"

using namespace hs;

namespace {

// out[r] = v / max for the two descending lists s0 (n0) and s1 (n1) merged in
// descending order (ties: list 0 first); one CTA. max = the larger head.
__global__ void merge_spectrum_kernel(const double* __restrict__ s0, int n0, const double* __restrict__ s1, int n1,
                                      double* __restrict__ out) {
  hs_pdl_enter();
  const double top = fmax(n0 > 0 ? s0[0] : 0.0, n1 > 0 ? s1[0] : 0.0);
  const double inv = top > 0.0 ? 1.0 / top : 0.0;
  for (int i = threadIdx.x; i < n0 + n1; i += blockDim.x) {
    const bool first = i < n0;
    const double v = first ? s0[i] : s1[i - n0];
    const double* o = first ? s1 : s0;
    const int no = first ? n1 : n0;
    // number of entries of the other list that come before v
    int lo = 0, hi = no;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      const bool before = first ? (o[mid] > v) : (o[mid] >= v);
      if (before)
        lo = mid + 1;
      else
        hi = mid;
    }
    out[(first ? i : i - n0) + lo] = v * inv;
  }
}

}  // namespace

// Singular values (descending) of the n x n matrix X (device, overwritten) into s.
static hs_status svd_values(hs_ctx ctx, double* X, int n, double* s, int slot) {
  if (n == 0) return HS_OK;
  int lwork = 0;
  HS_SOLVER(cusolverDnDgesvd_bufferSize(ctx->solver, n, n, &lwork));
  HS_TRY(ctx->solver_dev.ensure(((size_t)lwork + 8) * sizeof(double)));
  HS_SOLVER(cusolverDnDgesvd(ctx->solver, 'N', 'N', n, n, X, n, s, nullptr, n, nullptr, n, ctx->solver_dev.d(), lwork,
                             nullptr, static_cast<int*>(ctx->info.p) + slot));
  return HS_OK;
}

extern "C" hs_status hs_corner_spectrum(hs_ctx ctx, const hs_env* env, double* out) {
  HS_TRY(check_ctx(ctx));
  if (!env || !out || !env->C) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = ctx->stream;
  const int c0 = env->chi_even, c1 = env->chi_odd, chi = c0 + c1;
  if (c0 < 0 || c1 < 0 || chi == 0) return fail(HS_ERR_SHAPE, "empty corner");
  DBuf& work = ctx->hb[9];
  DBuf& sv = ctx->hb[10];
  HS_TRY(sv.ensure((size_t)(chi + 2) * sizeof(double)));
  HS_CUDA(cudaMemsetAsync(ctx->info.p, 0, 2 * sizeof(int), s));
  double* s0 = sv.d();
  double* s1 = s0 + (env->dtype == HS_C128 ? chi : c0);
  int n0 = c0, n1 = c1;
  if (env->dtype == HS_C128) {
    // M = C~ with the odd-odd block negated, one SVD of the whole chi x chi matrix
    HS_TRY(work.ensure((size_t)chi * chi * sizeof(double)));
    HS_CUDA(launch_graded_sign(env->C, work.d(), c0, c1, c0, c1, chi, 1, s));
    HS_TRY(svd_values(ctx, work.d(), chi, s0, 0));
    n0 = chi;
    n1 = 0;
  } else {
    // block diagonal: block 1 follows block 0 (c0 x c0, then c1 x c1)
    const long long e = (long long)c0 * c0 + (long long)c1 * c1;
    HS_TRY(work.ensure((size_t)e * sizeof(double)));
    HS_CUDA(cudaMemcpyAsync(work.d(), env->C, (size_t)e * sizeof(double), cudaMemcpyDeviceToDevice, s));
    HS_TRY(svd_values(ctx, work.d(), c0, s0, 0));
    HS_TRY(svd_values(ctx, work.d() + (long long)c0 * c0, c1, s1, 1));
  }
  hs_launch(merge_spectrum_kernel, 1, 256, 0, s, s0, n0, s1, n1, out);
  HS_CUDA(cudaGetLastError());
  ctx->launches += 1;
  int hinfo[2];
  HS_CUDA(cudaMemcpyAsync(hinfo, ctx->info.p, sizeof hinfo, cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  if (hinfo[0] != 0 || hinfo[1] != 0) return fail(HS_ERR_SOLVER, "gesvd info = (%d, %d)", hinfo[0], hinfo[1]);
  return HS_OK;
}

extern "C" hs_status hs_from_hermitian_basis(hs_ctx ctx, const hs_z2_tensor* t, double* a_dense) {
  HS_TRY(check_ctx(ctx));
  if (!t || !t->data || !a_dense || t->D <= 0) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (t->basis != HS_BASIS_HERMITIAN) return fail(HS_ERR_INVALID_ARG, "tensor is not in the Hermitian basis");
  if (t->dtype != HS_F64 && t->dtype != HS_C128) return fail(HS_ERR_DTYPE, "unknown dtype");
  const int D = t->D;
  if (t->n_even != D * (D + 1) / 2 || t->n_odd != D * (D - 1) / 2 || t->v_even != t->n_even ||
      t->h_even != t->n_even || t->v_odd != t->n_odd || t->h_odd != t->n_odd)
    return fail(HS_ERR_SHAPE, "not a double layer of bond dimension %d (sectors changed)", D);
  HS_CUDA(launch_from_hermitian(t->data, D, t->dtype == HS_C128, a_dense, ctx->stream));
  ctx->launches += 1;
  return HS_OK;
}

// Complex C4v CTMRG in the plain combined basis: the comparison path for the
// graded (Hermitian-basis) complex CTMRG of hs_graded.cu (arXiv 2410.11596
// Sec. II.C: in the eigenbasis of the swap every block is purely real or
// purely imaginary, so a product takes one real multiplication per pair where
// the plain basis takes four). Here nothing of that is used: every tensor is a
// general complex array, every product is a complex GEMM made of four FP64
// GEMMs on planar real and imaginary parts, and the truncation is the complex
// Hermitian eigen-decomposition of H = C' C'^dagger (cuSOLVER, FP64).
//
// The move follows the graded one step by step (same leg orders, the same
// reading of the truncation: keep the chi largest singular values of C' and
// renormalise with U_k^dagger on incoming and U_k on outgoing boundary legs).
// Environments are stored interleaved complex128: C[chi, chi], T[chi, D^2, chi].
#include <algorithm>

#include "hs_ctx.cuh"

using namespace hs;

namespace {

// workspace slots: planar pairs 0..15 (zd[0..31]), the interleave scratch, H
constexpr int kScratch = 36, kHz = 37;

unsigned grid_of(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// Traced-boundary C0[d, r] = sum_{u,l} a[u,l,d,r] delta(u) delta(l) and
// T0[alpha = d, x = r, beta = u] = sum_l a[u,l,d,r] delta(l), from the dense
// complex double layer (interleaved); delta = sum_k |k k'>.
__global__ void zinit_kernel(const double* __restrict__ a, int D, double* __restrict__ C, double* __restrict__ T) {
  hs_pdl_enter();
  const int q = D * D;
  const long long nT = (long long)q * q * q;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nT + (long long)q * q;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nT) {
      const int u = (int)(e % q), r = (int)((e / q) % q), d = (int)(e / q / q);  // T[d, r, u]
      double re = 0.0, im = 0.0;
      for (int k = 0; k < D; ++k) {
        const int l = k + D * k;
        const long long src = (((long long)u * q + l) * q + d) * q + r;
        re += a[2 * src];
        im += a[2 * src + 1];
      }
      T[2 * e] = re;
      T[2 * e + 1] = im;
    } else {
      const long long f = e - nT;
      const int d = (int)(f / q), r = (int)(f % q);
      double re = 0.0, im = 0.0;
      for (int k = 0; k < D; ++k)
        for (int k2 = 0; k2 < D; ++k2) {
          const long long src = (((long long)(k + D * k) * q + (k2 + D * k2)) * q + d) * q + r;
          re += a[2 * src];
          im += a[2 * src + 1];
        }
      C[2 * f] = re;
      C[2 * f + 1] = im;
    }
  }
}

// Kept vectors from the ascending eigenvalues w (n) and the column-major
// eigenvectors V (n x n, interleaved) of the row-major H read as column-major,
// i.e. of conj(H): column j is conj(u_j). Row i of P^T (planar) is
// u_{n-1-i}, row i of P^dagger is its conjugate (i < k); the selection record
// takes the singular values sqrt(w).
__global__ void zselect_kernel(const double* __restrict__ w, const double* __restrict__ V, int n, int k,
                               double* __restrict__ ptr, double* __restrict__ pti, double* __restrict__ pcr,
                               double* __restrict__ pci, SelectOut* __restrict__ sel) {
  hs_pdl_enter();
  const int i = blockIdx.x;
  if (i < k) {
    const double* col = V + 2LL * (long long)(n - 1 - i) * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double re = col[2 * j], im = col[2 * j + 1];
      ptr[(long long)i * n + j] = re;   // u = conj(column)
      pti[(long long)i * n + j] = -im;
      pcr[(long long)i * n + j] = re;   // conj(u) = column
      pci[(long long)i * n + j] = im;
    }
  }
  if (i == 0 && threadIdx.x == 0) {
    sel->chi_new[0] = k;
    sel->chi_new[1] = 0;
    sel->lam_max = sqrt(fmax(w[n - 1], 0.0));
    sel->lam_cut = sqrt(fmax(w[n - k], 0.0));
    sel->lam_next = k < n ? sqrt(fmax(w[n - k - 1], 0.0)) : 0.0;
    double disc = 0.0;
    for (int j = 0; j < n - k; ++j) disc += sqrt(fmax(w[j], 0.0));
    sel->discarded = disc;
  }
}

struct ZB {
  double* re;
  double* im;
};

// planar pair i of the context's dense-complex workspace, n doubles each
hs_status zb(hs_ctx ctx, int i, long long n, ZB* out) {
  HS_TRY(ctx->zd[2 * i].ensure((size_t)n * sizeof(double)));
  HS_TRY(ctx->zd[2 * i + 1].ensure((size_t)n * sizeof(double)));
  *out = {ctx->zd[2 * i].d(), ctx->zd[2 * i + 1].d()};
  return HS_OK;
}

Z2Mat dn(std::initializer_list<long long> dims) {
  Fused r = fused0(), c = fused0();
  const int n = (int)dims.size();
  int i = 0;
  for (long long v : dims) {
    if (i < n - 1)
      r.leg[r.k++] = make_sect((int)v, 0);
    else
      c.leg[c.k++] = make_sect((int)v, 0);
    ++i;
  }
  return mat(r, c);
}

// C = A B^T (or A conj(B)^T) for M x K and N x K planar complex operands: four FP64 GEMMs
hs_status zmul(hs_ctx ctx, long long M, long long N, long long K, ZB A, ZB B, ZB C, bool conj_b, double* flops) {
  cudaStream_t s = ctx->stream;
  GemmGroup g{};
  g.n = 1;
  g.p[0] = GemmProblem{(int)M, (int)N, (int)K, (int)K, (int)K, (int)N, 0, 0, 0};
  HS_TRY(ctx->splitk.ensure(kSplitKElems * sizeof(double)));
  double* part = ctx->splitk.d();
  const double sb = conj_b ? -1.0 : 1.0;
  PhaseScope ps(ctx, HS_PHASE_GEMM);
  HS_CUDA(launch_gemm_f64(g, A.re, B.re, C.re, 1.0, s, part, kSplitKElems, false));
  HS_CUDA(launch_gemm_f64(g, A.im, B.im, C.re, -sb, s, part, kSplitKElems, true));
  HS_CUDA(launch_gemm_f64(g, A.re, B.im, C.im, sb, s, part, kSplitKElems, false));
  HS_CUDA(launch_gemm_f64(g, A.im, B.re, C.im, 1.0, s, part, kSplitKElems, true));
  ctx->launches += 4;
  const double f = 8.0 * M * (double)N * K;
  *flops += f;
  ctx->phase_flops[HS_PHASE_GEMM] += f;
  return HS_OK;
}

hs_status zperm(hs_ctx ctx, const Z2Mat& in, const Z2Mat& out, std::initializer_list<int> perm, ZB src, ZB dst) {
  PhaseScope ps(ctx, HS_PHASE_PERMUTE);
  HS_TRY(permute(ctx, in, out, perm, src.re, dst.re));
  return permute(ctx, in, out, perm, src.im, dst.im);
}

// interleaved [n | 2] <-> planar (re, im)
hs_status deinterleave(hs_ctx ctx, const double* src, long long n, ZB dst) {
  HS_TRY(ctx->zd[kScratch].ensure((size_t)(2 * n) * sizeof(double)));
  HS_TRY(permute(ctx, dn({n, 2}), dn({2, n}), {1, 0}, src, ctx->zd[kScratch].d()));
  HS_CUDA(cudaMemcpyAsync(dst.re, ctx->zd[kScratch].d(), (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  HS_CUDA(cudaMemcpyAsync(dst.im, ctx->zd[kScratch].d() + n, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice,
                          ctx->stream));
  return HS_OK;
}

hs_status interleave(hs_ctx ctx, ZB src, long long n, double* dst) {
  HS_TRY(ctx->zd[kScratch].ensure((size_t)(2 * n) * sizeof(double)));
  HS_CUDA(cudaMemcpyAsync(ctx->zd[kScratch].d(), src.re, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  HS_CUDA(cudaMemcpyAsync(ctx->zd[kScratch].d() + n, src.im, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice,
                          ctx->stream));
  return permute(ctx, dn({2, n}), dn({n, 2}), {1, 0}, ctx->zd[kScratch].d(), dst);
}

}  // namespace

namespace hs {

size_t zdense_tensor_bytes(int D) {
  const size_t q = (size_t)D * D;
  return 2 * q * q * q * q * sizeof(double);
}

hs_status zdense_double_layer(hs_ctx ctx, const double* A, int d, int D, hs_z2_tensor* out) {
  HS_CUDA(launch_double_layer_dense(A, d, D, true, out->data, ctx->stream));
  ctx->launches += 1;
  return HS_OK;
}

hs_status zdense_init(hs_ctx ctx, const hs_z2_tensor* a, int chi_max, hs_env* env) {
  cudaStream_t s = ctx->stream;
  const int D = a->D, q = D * D;
  size_t cb, tb;
  HS_TRY(hs_env_bytes(D, chi_max, &cb, &tb));
  if (env->C_bytes < 2 * cb || env->T_bytes < 2 * tb)
    return fail(HS_ERR_WORKSPACE, "complex dense environments need twice hs_env_bytes (%zu/%zu)", 2 * cb, 2 * tb);
  env->chi_even = q;
  env->chi_odd = 0;
  env->q_even = q;
  env->q_odd = 0;
  const long long nT = (long long)q * q * q;
  hs_launch(zinit_kernel, grid_of(nT + (long long)q * q), 256, 0, s, (const double*)a->data, D, env->C, env->T);
  HS_CUDA(cudaGetLastError());
  SelectOut* dsel = static_cast<SelectOut*>(ctx->sel.p);
  HS_CUDA(launch_normalize_max_to(env->C, 2LL * q * q, static_cast<unsigned long long*>(ctx->scratch.p) + 2,
                                  &dsel->log_norm_C, s));
  HS_CUDA(launch_normalize_max(env->T, 2 * nT, static_cast<unsigned long long*>(ctx->scratch.p), dsel, s));
  HS_CUDA(cudaMemcpyAsync(ctx->h_sel, dsel, sizeof(SelectOut), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  env->log_norm_C = ctx->h_sel->log_norm_C;
  env->log_norm_T = ctx->h_sel->log_norm_T;
  // planar private copy of a (real part, then imaginary part)
  const long long na = (long long)q * q * q * q;
  HS_TRY(ctx->ga.ensure((size_t)(2 * na) * sizeof(double)));
  HS_TRY(permute(ctx, dn({na, 2}), dn({2, na}), {1, 0}, a->data, ctx->ga.d()));
  ctx->ga_src = a->data;
  const size_t c = (size_t)env->chi_max, n = c * q;
  HS_TRY(ctx->w.ensure(n * sizeof(double)));
  HS_TRY(ctx->zd[kHz].ensure(2 * n * n * sizeof(double)));  // H interleaved, vectors in place
  // the complex Hermitian eigen-decomposition's workspace
  size_t dw = 0, hw = 0;
  HS_SOLVER(cusolverDnXsyevd_bufferSize(ctx->solver, ctx->params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                        (int64_t)n, CUDA_C_64F, ctx->zd[kHz].p, (int64_t)n, CUDA_R_64F, ctx->w.p,
                                        CUDA_C_64F, &dw, &hw));
  HS_TRY(ctx->solver_dev.ensure(dw + 256));
  if (ctx->solver_host.size() < hw + 1) ctx->solver_host.resize(hw + 1);
  return HS_OK;
}

hs_status zdense_move(hs_ctx ctx, const hs_z2_tensor* a, hs_env* env, int chi, hs_move_info* info) {
  if (ctx->ga_src != a->data)
    return fail(HS_ERR_INVALID_ARG, "the double layer changed since hs_ctmrg_init (private copy is stale)");
  if (env->precision != HS_PREC_F64 || env->eig_mode != HS_EIG_F64)
    return fail(HS_ERR_UNSUPPORTED, "complex dense CTMRG runs FP64 GEMMs and the FP64 eigen-decomposition only");
  cudaStream_t s = ctx->stream;
  const long long c = env->chi_even + env->chi_odd, q = env->q_even + env->q_odd;
  const long long n = c * q;
  const int k = (int)std::min<long long>(chi, n);
  double flops = 0.0;
  const long long na = q * q * q * q;
  const ZB A2{ctx->ga.d(), ctx->ga.d() + na};
  ZB Cz, Tz, Ct, Tq, X1, X2, X2p, X3, Cp, H, PT, PTc, V1, V1t, Pp, Y, Yp, Z, Zp, Cn, Tn;
  HS_TRY(zb(ctx, 0, c * c, &Cz));
  HS_TRY(zb(ctx, 1, c * q * c, &Tz));
  HS_TRY(zb(ctx, 2, c * c, &Ct));
  HS_TRY(zb(ctx, 3, c * q * c, &Tq));
  HS_TRY(zb(ctx, 4, c * q * c, &X1));
  HS_TRY(zb(ctx, 5, n * n, &X2));   // X2, then X3, then H
  HS_TRY(zb(ctx, 6, n * n, &X2p));  // X2p, then C'
  HS_TRY(zb(ctx, 7, (long long)k * n, &PT));
  HS_TRY(zb(ctx, 8, (long long)k * n, &PTc));
  HS_TRY(zb(ctx, 9, n * k, &V1));
  HS_TRY(zb(ctx, 10, n * k, &V1t));
  HS_TRY(zb(ctx, 11, (long long)k * k, &Cn));
  HS_TRY(zb(ctx, 12, (long long)k * q * c, &Pp));
  HS_TRY(zb(ctx, 13, (long long)k * q * q * c, &Y));
  HS_TRY(zb(ctx, 14, (long long)k * q * q * c, &Yp));
  HS_TRY(zb(ctx, 15, (long long)k * q * k, &Tn));
  X3 = X2;
  Cp = X2p;
  H = X2;
  Z = Y;
  Zp = Yp;

  HS_TRY(deinterleave(ctx, env->C, c * c, Cz));
  HS_TRY(deinterleave(ctx, env->T, c * q * c, Tz));
  // ---- enlarged corner C'[(alpha,d),(eps,r)] = T[alpha,x,beta] C[beta,gamma] T[gamma,y,eps] a[y,x,d,r]
  HS_TRY(zperm(ctx, dn({c, c}), dn({c, c}), {1, 0}, Cz, Ct));
  HS_TRY(zperm(ctx, dn({c, q, c}), dn({q, c, c}), {1, 2, 0}, Tz, Tq));          // Tq[(x, beta) | alpha]
  HS_TRY(zmul(ctx, c * q, c, c, Tz, Ct, X1, false, &flops));                      // X1[(alpha,x) | gamma]
  HS_TRY(zmul(ctx, c * q, q * c, c, X1, Tq, X2, false, &flops));                  // X2[(alpha,x) | (y,eps)]
  HS_TRY(zperm(ctx, dn({c, q, q, c}), dn({c, c, q, q}), {0, 3, 2, 1}, X2, X2p));  // (a,x,y,e) -> (a,e,y,x)
  HS_TRY(zmul(ctx, c * c, q * q, q * q, X2p, A2, X3, false, &flops));             // X3[(alpha,eps) | (d,r)]
  HS_TRY(zperm(ctx, dn({c, c, q, q}), dn({c, q, c, q}), {0, 2, 1, 3}, X3, Cp));   // C'[(alpha,d) | (eps,r)]
  // ---- truncation: eigenvectors of H = C' C'^dagger (complex Hermitian, FP64)
  HS_TRY(zmul(ctx, n, n, n, Cp, Cp, H, true, &flops));
  double* Hz = ctx->zd[kHz].d();
  HS_TRY(interleave(ctx, H, n * n, Hz));
  {
    PhaseScope ps(ctx, HS_PHASE_EIG);
    HS_CUDA(cudaMemsetAsync(ctx->info.p, 0, sizeof(int), s));
    HS_SOLVER(cusolverDnXsyevd(ctx->solver, ctx->params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                               (int64_t)n, CUDA_C_64F, Hz, (int64_t)n, CUDA_R_64F, ctx->w.p, CUDA_C_64F,
                               ctx->solver_dev.p, ctx->solver_dev.bytes, ctx->solver_host.data(),
                               ctx->solver_host.size(), static_cast<int*>(ctx->info.p)));
  }
  SelectOut* dsel = static_cast<SelectOut*>(ctx->sel.p);
  {
    PhaseScope ps(ctx, HS_PHASE_SELECT);
    hs_launch(zselect_kernel, k, 256, 0, s, (const double*)ctx->w.d(), (const double*)Hz, (int)n, k, PT.re, PT.im,
              PTc.re, PTc.im, dsel);
    HS_CUDA(cudaGetLastError());
    ctx->launches += 1;
  }
  // ---- C_new = P^dagger C' P (PT = P^T, PTc = P^dagger)
  HS_TRY(zmul(ctx, n, k, n, Cp, PT, V1, false, &flops));                            // V1 = C' P
  HS_TRY(zperm(ctx, dn({n, k}), dn({k, n}), {1, 0}, V1, V1t));
  HS_TRY(zmul(ctx, k, k, n, PTc, V1t, Cn, false, &flops));                          // C_new
  // ---- T_new[a', r, b'] = conj(P[(alpha,d),a']) T[alpha,x,beta] a[u,x,d,r] P[(beta,u),b']
  HS_TRY(zperm(ctx, dn({k, c, q}), dn({q, k, c}), {2, 0, 1}, PTc, Pp));            // Pp[(d, a') | alpha]
  HS_TRY(zmul(ctx, q * k, q * c, c, Pp, Tq, Y, false, &flops));                     // Y[(d,a') | (x,beta)]
  HS_TRY(zperm(ctx, dn({q, k, q, c}), dn({k, c, q, q}), {1, 3, 0, 2}, Y, Yp));     // Yp[(a',beta) | (d,x)]
  HS_TRY(zmul(ctx, k * c, q * q, q * q, Yp, A2, Z, false, &flops));                 // Z[(a',beta) | (u,r)]
  HS_TRY(zperm(ctx, dn({k, c, q, q}), dn({k, q, c, q}), {0, 3, 1, 2}, Z, Zp));     // Zp[(a',r) | (beta,u)]
  HS_TRY(zmul(ctx, k * q, k, c * q, Zp, PT, Tn, false, &flops));                   // T_new[(a',r) | b']
  // ---- back to interleaved storage, normalised by the largest real or imaginary part
  HS_TRY(interleave(ctx, Cn, (long long)k * k, env->C));
  HS_TRY(interleave(ctx, Tn, (long long)k * q * k, env->T));
  {
    PhaseScope ps(ctx, HS_PHASE_NORMALIZE);
    HS_CUDA(launch_normalize_max_to(env->C, 2LL * k * k, static_cast<unsigned long long*>(ctx->scratch.p) + 2,
                                    &dsel->log_norm_C, s));
    HS_CUDA(launch_normalize_max(env->T, 2LL * k * q * k, static_cast<unsigned long long*>(ctx->scratch.p), dsel, s));
    ctx->launches += 4;
  }
  HS_CUDA(cudaMemcpyAsync(ctx->h_sel, dsel, sizeof(SelectOut), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaMemcpyAsync(ctx->h_info, ctx->info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  harvest_profile(ctx);
  if (*ctx->h_info != 0) return fail(HS_ERR_SOLVER, "eigensolver info %d", *ctx->h_info);
  const SelectOut sel = *ctx->h_sel;
  env->chi_even = k;
  env->chi_odd = 0;
  env->log_norm_C = sel.log_norm_C;
  env->log_norm_T = sel.log_norm_T;
  env->moves += 1;
  if (!std::isfinite(env->log_norm_T) || !std::isfinite(env->log_norm_C))
    return fail(HS_ERR_NONFINITE, "environment is not finite after the move");
  if (info) {
    memset(info, 0, sizeof *info);
    info->chi_even = k;
    info->n_even = (int)n;
    info->lam_max = sel.lam_max;
    info->lam_cut = sel.lam_cut;
    info->lam_next = sel.lam_next;
    const bool discarded = k < n;
    info->gap = discarded ? (sel.lam_cut - sel.lam_next) / sel.lam_max : INFINITY;
    info->log_norm_C = env->log_norm_C;
    info->log_norm_T = env->log_norm_T;
    info->gemm_flops = flops;
    info->flags = (discarded && info->gap < 1e-9) ? 1 : 0;
    info->subspace_reason = -1;
  }
  return HS_OK;
}

}  // namespace hs

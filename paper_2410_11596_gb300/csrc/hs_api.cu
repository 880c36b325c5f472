// C ABI of libhs (include/hs.h): context, workspace, the C4v CTMRG move of
// arXiv 2410.11596 (Sec. II.A, Fig. 1(d)) in the Hermitian Z2 basis
// (Sec. II.B).
#include "hs_ctx.cuh"

using namespace hs;

namespace hs {

namespace {
thread_local std::string g_err;
}

hs_status fail(hs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

const char* last_error() { return g_err.c_str(); }

hs_status check_ctx(hs_ctx ctx) {
  if (!ctx) return fail(HS_ERR_INVALID_ARG, "null context");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(HS_ERR_CUDA, "cudaSetDevice failed");
  return HS_OK;
}

Sect q_sect(int D, hs_basis b) {
  const int q = D * D;
  return b == HS_BASIS_HERMITIAN ? make_sect(D * (D + 1) / 2, D * (D - 1) / 2) : make_sect(q, 0);
}

Z2Mat mat(Fused r, Fused c) {
  Z2Mat m;
  m.r = r;
  m.c = c;
  return m;
}

hs_status gemm(hs_ctx ctx, hs_gemm_backend be, const GemmGroup& g, const double* A, const double* B,
               double* C) {
  if (be == HS_GEMM_CUBLAS) {
    const double one = 1.0, zero = 0.0;
    for (int i = 0; i < g.n; ++i) {
      const GemmProblem& p = g.p[i];
      if (p.K == 0) {
        HS_CUDA(cudaMemset2DAsync(C + p.c_off, sizeof(double) * p.ldc, 0, sizeof(double) * p.N, p.M,
                                  ctx->stream));
        continue;
      }
      HS_BLAS(cublasDgemm(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, p.N, p.M, p.K, &one, B + p.b_off,
                          p.ldb, A + p.a_off, p.lda, &zero, C + p.c_off, p.ldc));
    }
    return HS_OK;
  }
  HS_CUDA(launch_gemm_f64(g, A, B, C, 1.0, ctx->stream));
  return HS_OK;
}

hs_status permute(hs_ctx ctx, const Z2Mat& in, const Z2Mat& out, std::initializer_list<int> perm,
                  const double* src, double* dst) {
  int p[4] = {0, 0, 0, 0};
  int i = 0;
  for (int v : perm) p[i++] = v;
  const PermPlan plan = make_perm_plan(in, out, p);
  HS_CUDA(launch_permute_f64(plan, src, dst, 1.0, ctx->stream));
  return HS_OK;
}

namespace {

size_t a_elems(int D, hs_basis b) {
  const Sect q = q_sect(D, b);
  return (size_t)z2_elems(mat(fused2(q, q), fused2(q, q)));
}

hs_status eig_workspace(hs_ctx ctx, int nmax) {
  size_t dev = 0, host = 0;
  HS_SOLVER(cusolverDnXsyevd_bufferSize(ctx->solver, ctx->params, CUSOLVER_EIG_MODE_VECTOR,
                                        CUBLAS_FILL_MODE_LOWER, nmax, CUDA_R_64F, nullptr, nmax,
                                        CUDA_R_64F, nullptr, CUDA_R_64F, &dev, &host));
  HS_TRY(ctx->solver_dev.ensure(dev + 256));
  if (ctx->solver_host.size() < host + 1) ctx->solver_host.resize(host + 1);
  return HS_OK;
}

// In-place FP64 symmetric eigen-decomposition of one n x n block.
hs_status eig_block(hs_ctx ctx, double* A, int n, double* w, int slot) {
  if (n == 0) return HS_OK;
  HS_SOLVER(cusolverDnXsyevd(ctx->solver, ctx->params, CUSOLVER_EIG_MODE_VECTOR,
                             CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A, n, CUDA_R_64F, w, CUDA_R_64F,
                             ctx->solver_dev.p, ctx->solver_dev.bytes, ctx->solver_host.data(),
                             ctx->solver_host.size(), static_cast<int*>(ctx->info.p) + slot));
  return HS_OK;
}

}  // namespace
}  // namespace hs

// ---------------------------------------------------------------------------

extern "C" {

int hs_abi_version(void) { return HS_ABI_VERSION; }

const char* hs_last_error(void) { return hs::last_error(); }

hs_status hs_create(hs_ctx* out, int device, void* stream) {
  if (!out) return fail(HS_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(HS_ERR_CUDA, "no CUDA device available");
  }
  if (device < 0 || device >= ndev) return fail(HS_ERR_INVALID_ARG, "device %d out of range", device);
  HS_CUDA(cudaSetDevice(device));
  hs_ctx c = new hs_ctx_s();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cusolverDnCreate(&c->solver) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnSetStream(c->solver, c->stream) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnCreateParams(&c->params) != CUSOLVER_STATUS_SUCCESS) {
    hs_destroy(c);
    return fail(HS_ERR_SOLVER, "cuSOLVER initialisation failed");
  }
  if (cublasCreate(&c->blas) != CUBLAS_STATUS_SUCCESS ||
      cublasSetStream(c->blas, c->stream) != CUBLAS_STATUS_SUCCESS ||
      cublasSetMathMode(c->blas, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS) {
    hs_destroy(c);
    return fail(HS_ERR_SOLVER, "cuBLAS initialisation failed");
  }
  if (cudaMallocHost(&c->h_sel, sizeof(SelectOut)) != cudaSuccess ||
      cudaMallocHost(&c->h_info, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    hs_destroy(c);
    return fail(HS_ERR_CUDA, "pinned allocation failed");
  }
  hs_status st;
  if ((st = c->sel.ensure(sizeof(SelectOut))) != HS_OK || (st = c->info.ensure(4 * sizeof(int))) != HS_OK ||
      (st = c->scratch.ensure(64)) != HS_OK) {
    hs_destroy(c);
    return st;
  }
  *out = c;
  return HS_OK;
}

hs_status hs_destroy(hs_ctx ctx) {
  if (!ctx) return HS_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  DBuf* bufs[] = {&ctx->big1, &ctx->big2, &ctx->x1, &ctx->pt, &ctx->pp, &ctx->w, &ctx->lam,
                  &ctx->idx, &ctx->sel, &ctx->scratch, &ctx->info, &ctx->solver_dev};
  for (DBuf* b : bufs) b->release();
  for (DBuf& b : ctx->r) b.release();
  if (ctx->h_sel) cudaFreeHost(ctx->h_sel);
  if (ctx->h_info) cudaFreeHost(ctx->h_info);
  if (ctx->params) cusolverDnDestroyParams(ctx->params);
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  if (ctx->blas) cublasDestroy(ctx->blas);
  delete ctx;
  return HS_OK;
}

hs_status hs_sync(hs_ctx ctx) {
  HS_TRY(check_ctx(ctx));
  HS_CUDA(cudaStreamSynchronize(ctx->stream));
  return HS_OK;
}

size_t hs_z2_tensor_bytes(int D, hs_basis basis, hs_dtype dtype) {
  if (D <= 0 || dtype != HS_F64) return 0;
  return a_elems(D, basis) * sizeof(double);
}

hs_status hs_make_double_layer(hs_ctx ctx, const double* A, int d, int D, hs_dtype dtype,
                               double* a_out) {
  HS_TRY(check_ctx(ctx));
  if (!A || !a_out || d <= 0 || D <= 0) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (dtype != HS_F64 && dtype != HS_C128) return fail(HS_ERR_DTYPE, "unknown dtype");
  HS_CUDA(launch_double_layer_dense(A, d, D, dtype == HS_C128, a_out, ctx->stream));
  return HS_OK;
}

hs_status hs_to_hermitian_basis(hs_ctx ctx, const double* a_dense, int D, hs_dtype dtype,
                                double herm_tol, hs_z2_tensor* out) {
  HS_TRY(check_ctx(ctx));
  if (!a_dense || !out || !out->data || D <= 0) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (dtype != HS_F64)
    return fail(HS_ERR_UNSUPPORTED, "complex double layers are not supported by this build");
  const size_t need = hs_z2_tensor_bytes(D, HS_BASIS_HERMITIAN, dtype);
  if (out->capacity_bytes < need)
    return fail(HS_ERR_WORKSPACE, "output holds %zu bytes, %zu needed", out->capacity_bytes, need);
  HS_CUDA(cudaMemsetAsync(ctx->scratch.p, 0, 2 * sizeof(unsigned long long), ctx->stream));
  HS_CUDA(launch_rotate_dense_to_blocks(a_dense, D, out->data,
                                        static_cast<unsigned long long*>(ctx->scratch.p),
                                        ctx->stream));
  unsigned long long m[2];
  HS_CUDA(cudaMemcpyAsync(m, ctx->scratch.p, sizeof m, cudaMemcpyDeviceToHost, ctx->stream));
  HS_CUDA(cudaStreamSynchronize(ctx->stream));
  double mo, ma;
  memcpy(&mo, &m[0], 8);
  memcpy(&ma, &m[1], 8);
  const Sect q = q_sect(D, HS_BASIS_HERMITIAN);
  out->D = D;
  out->n_even = q.n[0];
  out->n_odd = q.n[1];
  out->basis = HS_BASIS_HERMITIAN;
  out->dtype = dtype;
  if (!(mo <= herm_tol * ma))
    return fail(HS_ERR_NOT_HERMITIAN, "odd-total blocks reach %.3e of max %.3e (tol %.1e)", mo, ma,
                herm_tol);
  return HS_OK;
}

hs_status hs_double_layer_hermitian(hs_ctx ctx, const double* A, int d, int D, hs_dtype dtype,
                                    hs_basis basis, hs_z2_tensor* out) {
  HS_TRY(check_ctx(ctx));
  if (!A || !out || !out->data || d <= 0 || D <= 0) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (dtype != HS_F64)
    return fail(HS_ERR_UNSUPPORTED, "complex double layers are not supported by this build");
  if (basis != HS_BASIS_DENSE && basis != HS_BASIS_HERMITIAN)
    return fail(HS_ERR_INVALID_ARG, "unknown basis");
  const size_t need = hs_z2_tensor_bytes(D, basis, dtype);
  if (out->capacity_bytes < need)
    return fail(HS_ERR_WORKSPACE, "output holds %zu bytes, %zu needed", out->capacity_bytes, need);
  HS_CUDA(launch_double_layer_blocks(A, d, D, basis == HS_BASIS_HERMITIAN, out->data, ctx->stream));
  const Sect q = q_sect(D, basis);
  out->D = D;
  out->n_even = q.n[0];
  out->n_odd = q.n[1];
  out->basis = basis;
  out->dtype = dtype;
  return HS_OK;
}

hs_status hs_env_bytes(int D, int chi_max, size_t* C_bytes, size_t* T_bytes) {
  if (D <= 0 || chi_max <= 0 || !C_bytes || !T_bytes) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  const size_t chi = (size_t)(chi_max > D * D ? chi_max : D * D);
  *C_bytes = chi * chi * sizeof(double);
  *T_bytes = chi * (size_t)D * D * chi * sizeof(double);
  return HS_OK;
}

hs_status hs_workspace_query(int D, int chi, hs_precision precision, size_t* bytes) {
  if (D <= 0 || chi <= 0 || !bytes) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  (void)precision;
  const size_t q = (size_t)D * D, c = (size_t)(chi > (int)q ? chi : (int)q);
  *bytes = 2 * c * c * q * q * sizeof(double) + 3 * c * c * q * sizeof(double);
  return HS_OK;
}

hs_status hs_ctmrg_init(hs_ctx ctx, const hs_z2_tensor* a, int chi_max, hs_precision precision,
                        hs_gemm_backend backend, hs_env* env) {
  HS_TRY(check_ctx(ctx));
  if (!a || !env || !a->data || !env->C || !env->T) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (precision != HS_PREC_F64)
    return fail(HS_ERR_UNSUPPORTED, "precision %d is not implemented in this build", (int)precision);
  const int D = a->D, q = D * D;
  if (chi_max < 1) return fail(HS_ERR_SHAPE, "chi_max must be positive");
  size_t cb, tb;
  HS_TRY(hs_env_bytes(D, chi_max, &cb, &tb));
  if (env->C_bytes < cb || env->T_bytes < tb)
    return fail(HS_ERR_WORKSPACE, "environment buffers too small (%zu/%zu needed)", cb, tb);
  const bool herm = a->basis == HS_BASIS_HERMITIAN;
  const Sect qs = q_sect(D, a->basis);
  env->D = D;
  env->chi_max = chi_max > q ? chi_max : q;
  env->q_even = qs.n[0];
  env->q_odd = qs.n[1];
  env->chi_even = qs.n[0];
  env->chi_odd = qs.n[1];
  env->basis = a->basis;
  env->precision = precision;
  env->gemm_backend = backend;
  env->moves = 0;
  HS_CUDA(launch_ctmrg_init(a->data, D, herm, env->C, env->T, ctx->stream));
  // normalise like every later move
  const Z2Mat Cm = mat(fused1(qs), fused1(qs)), Tm = mat(fused2(qs, qs), fused1(qs));
  HS_CUDA(launch_normalize_max(env->C, z2_elems(Cm), static_cast<unsigned long long*>(ctx->scratch.p),
                               static_cast<SelectOut*>(ctx->sel.p), ctx->stream));
  HS_CUDA(cudaMemcpyAsync(&ctx->h_sel->log_norm_C, &static_cast<SelectOut*>(ctx->sel.p)->log_norm_T,
                          sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  HS_CUDA(launch_normalize_max(env->T, z2_elems(Tm), static_cast<unsigned long long*>(ctx->scratch.p) + 1,
                               static_cast<SelectOut*>(ctx->sel.p), ctx->stream));
  HS_CUDA(cudaMemcpyAsync(&ctx->h_sel->log_norm_T, &static_cast<SelectOut*>(ctx->sel.p)->log_norm_T,
                          sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  HS_CUDA(cudaStreamSynchronize(ctx->stream));
  env->log_norm_C = ctx->h_sel->log_norm_C;
  env->log_norm_T = ctx->h_sel->log_norm_T;
  // workspace for the moves
  const size_t c = (size_t)env->chi_max;
  const size_t big = c * c * (size_t)q * q;
  HS_TRY(ctx->big1.ensure(big * sizeof(double)));
  HS_TRY(ctx->big2.ensure(big * sizeof(double)));
  HS_TRY(ctx->x1.ensure(c * q * c * sizeof(double)));
  HS_TRY(ctx->pt.ensure(c * c * q * sizeof(double)));
  HS_TRY(ctx->pp.ensure(c * c * q * sizeof(double)));
  HS_TRY(ctx->w.ensure(c * q * sizeof(double)));
  HS_TRY(ctx->lam.ensure(c * sizeof(double)));
  HS_TRY(ctx->idx.ensure(2 * c * sizeof(int)));
  HS_TRY(eig_workspace(ctx, (int)(c * q)));
  return HS_OK;
}

hs_status hs_ctmrg_move(hs_ctx ctx, const hs_z2_tensor* a, hs_env* env, int chi,
                        hs_move_info* info) {
  HS_TRY(check_ctx(ctx));
  if (!a || !env || !a->data) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (a->D != env->D || a->basis != env->basis)
    return fail(HS_ERR_SHAPE, "tensor and environment disagree on D or basis");
  if (chi < 1 || chi > env->chi_max) return fail(HS_ERR_SHAPE, "chi %d outside [1, %d]", chi, env->chi_max);
  cudaStream_t s = ctx->stream;
  const hs_gemm_backend be = env->gemm_backend;
  const Sect q = make_sect(env->q_even, env->q_odd);
  const Sect c = make_sect(env->chi_even, env->chi_odd);
  double* B1 = ctx->big1.d();
  double* B2 = ctx->big2.d();
  double flops = 0;

  // enlarged corner C'[(alpha,d)|(eps,r)] = T C T a
  const Z2Mat Tcr = mat(fused2(c, q), fused1(c)), Cm = mat(fused1(c), fused1(c));
  const Z2Mat X1 = mat(fused2(c, q), fused1(c));
  const Z2Mat X2 = mat(fused2(c, q), fused2(c, q));
  const Z2Mat X2p = mat(fused2(c, c), fused2(q, q));
  const Z2Mat Am = mat(fused2(q, q), fused2(q, q));
  const Z2Mat X3 = mat(fused2(c, c), fused2(q, q));
  const Z2Mat Cp = mat(fused2(c, q), fused2(c, q));
  GemmGroup g1 = make_z2_gemm(Tcr, Cm, X1), g2 = make_z2_gemm(X1, Tcr, X2),
            g3 = make_z2_gemm(X2p, Am, X3);
  flops += gemm_flops(g1) + gemm_flops(g2) + gemm_flops(g3);
  HS_TRY(gemm(ctx, be, g1, env->T, env->C, ctx->x1.d()));
  HS_TRY(gemm(ctx, be, g2, ctx->x1.d(), env->T, B1));
  HS_TRY(permute(ctx, X2, X2p, {0, 2, 3, 1}, B1, B2));  // (a,x,e,y) -> (a,e,y,x)
  HS_TRY(gemm(ctx, be, g3, B2, a->data, B1));
  HS_TRY(permute(ctx, X3, Cp, {0, 2, 1, 3}, B1, B2));   // (a,e,d,r) -> (a,d,e,r)

  // one FP64 eigen-decomposition per parity block
  const int n0 = (int)z2_rows(Cp, 0), n1 = (int)z2_rows(Cp, 1);
  double* V0 = B2;
  double* V1 = B2 + (long long)n0 * n0;
  double* w0 = ctx->w.d();
  double* w1 = w0 + n0;
  HS_CUDA(cudaMemsetAsync(ctx->info.p, 0, 2 * sizeof(int), s));
  HS_TRY(eig_block(ctx, V0, n0, w0, 0));
  HS_TRY(eig_block(ctx, V1, n1, w1, 1));
  SelectOut* dsel = static_cast<SelectOut*>(ctx->sel.p);
  int* didx = static_cast<int*>(ctx->idx.p);
  HS_CUDA(launch_select(w0, n0, w1, n1, chi, didx, ctx->lam.d(), dsel, s));
  HS_CUDA(cudaMemcpyAsync(ctx->h_sel, dsel, sizeof(SelectOut), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaMemcpyAsync(ctx->h_info, ctx->info.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  if (ctx->h_info[0] != 0 || ctx->h_info[1] != 0)
    return fail(HS_ERR_SOLVER, "syevd info = (%d, %d)", ctx->h_info[0], ctx->h_info[1]);
  if (!std::isfinite(ctx->h_sel->lam_max) || ctx->h_sel->lam_max <= 0)
    return fail(HS_ERR_NONFINITE, "enlarged corner has no finite non-zero eigenvalue");
  const SelectOut sel = *ctx->h_sel;
  const Sect cn = make_sect(sel.chi_new[0], sel.chi_new[1]);

  // projector and renormalised edge T_new = P^T (T a) P
  const Z2Mat PT = mat(fused1(cn), fused2(c, q));
  const Z2Mat Pp = mat(fused2(q, cn), fused1(c));
  const Z2Mat Y = mat(fused2(q, cn), fused2(c, q));
  const Z2Mat Yp = mat(fused2(cn, c), fused2(q, q));
  const Z2Mat Zm = mat(fused2(cn, c), fused2(q, q));
  const Z2Mat Zp = mat(fused2(cn, q), fused2(c, q));
  const Z2Mat Tn = mat(fused2(cn, q), fused1(cn));
  HS_CUDA(launch_gather_pt(V0, n0, V1, n1, didx, chi, dsel, ctx->pt.d(), s));
  HS_TRY(permute(ctx, PT, Pp, {2, 0, 1}, ctx->pt.d(), ctx->pp.d()));  // (a',a,d) -> (d,a',a)
  GemmGroup g4 = make_z2_gemm(Pp, Tcr, Y), g5 = make_z2_gemm(Yp, Am, Zm), g6 = make_z2_gemm(Zp, PT, Tn);
  flops += gemm_flops(g4) + gemm_flops(g5) + gemm_flops(g6);
  HS_TRY(gemm(ctx, be, g4, ctx->pp.d(), env->T, B1));
  HS_TRY(permute(ctx, Y, Yp, {1, 2, 0, 3}, B1, B2));    // (d,a',b,x) -> (a',b,d,x)
  HS_TRY(gemm(ctx, be, g5, B2, a->data, B1));
  HS_TRY(permute(ctx, Zm, Zp, {0, 3, 1, 2}, B1, B2));   // (a',b,u,r) -> (a',r,b,u)
  HS_TRY(gemm(ctx, be, g6, B2, ctx->pt.d(), env->T));

  // C <- diag(lambda)/max|lambda|, T <- T/max|T|
  HS_CUDA(launch_diag_corner(ctx->lam.d(), cn.n[0], cn.n[1], dsel, env->C, s));
  HS_CUDA(launch_normalize_max(env->T, z2_elems(Tn), static_cast<unsigned long long*>(ctx->scratch.p),
                               dsel, s));
  HS_CUDA(cudaMemcpyAsync(&ctx->h_sel->log_norm_C, &dsel->log_norm_C, 2 * sizeof(double),
                          cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  env->chi_even = cn.n[0];
  env->chi_odd = cn.n[1];
  env->log_norm_C = ctx->h_sel->log_norm_C;
  env->log_norm_T = ctx->h_sel->log_norm_T;
  env->moves += 1;
  if (!std::isfinite(env->log_norm_T))
    return fail(HS_ERR_NONFINITE, "edge tensor is not finite after the move");
  if (info) {
    info->chi_even = cn.n[0];
    info->chi_odd = cn.n[1];
    info->n_even = n0;
    info->n_odd = n1;
    info->lam_max = sel.lam_max;
    info->lam_cut = sel.lam_cut;
    info->lam_next = sel.lam_next;
    const bool discarded = cn.n[0] + cn.n[1] < n0 + n1;
    info->gap = discarded ? (sel.lam_cut - sel.lam_next) / sel.lam_max : INFINITY;
    info->log_norm_C = env->log_norm_C;
    info->log_norm_T = env->log_norm_T;
    info->gemm_flops = flops;
    info->flags = (discarded && info->gap < 1e-9) ? 1 : 0;
  }
  return HS_OK;
}

hs_status hs_env_to_dense(hs_ctx ctx, const hs_env* env, double* C_dense, double* T_dense) {
  HS_TRY(check_ctx(ctx));
  if (!env || !C_dense || !T_dense) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  HS_CUDA(launch_env_to_dense(env->C, env->T, env->D, env->chi_even, env->chi_odd,
                              env->basis == HS_BASIS_HERMITIAN, C_dense, T_dense, ctx->stream));
  return HS_OK;
}

}  // extern "C"

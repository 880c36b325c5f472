// C4v CTMRG for complex tensors in the eigenbasis of S (arXiv 2410.11596
// Sec. II.C). Every tensor is a graded matrix (GMat): dense real storage whose
// odd-total entries carry the imaginary parts, multiplied with the sign rule
// of Eq. (2)-(3) (make_graded_gemm), so that every product is a real GEMM at a
// quarter of the cost of the complex one.
//
// Truncation (the paper leaves it open for complex tensors). The enlarged
// corner C' is complex symmetric, but its eigenvalues come in complex-
// conjugate pairs of equal modulus, so "keep the chi largest" is not defined
// for them. The move uses the singular value decomposition C' = U S V^dagger,
// keeps the chi largest singular values and inserts U_k U_k^dagger on every
// boundary bond: each boundary tensor, oriented clockwise, is renormalised as
// U_k^dagger on its incoming leg and U_k on its outgoing leg,
//   C_new = U_k^dagger C' U_k,  T_new = U_k^dagger (T a) U_k.
// For real tensors this is the eigenvalue rule (singular values |lambda|).
// In graded form C' = J M J with J = diag(1, i) by row parity and M real
// (the odd-odd block of the stored C' negated), so U = J U~ with U~ the left
// singular vectors of M: the top eigenvectors of H = M M^T. U's graded
// storage is U~ itself, and every new boundary state is even (chi_odd = 0
// after the first move).
#include <algorithm>
#include <cmath>

#include "hs_ctx.cuh"

namespace hs {

namespace {

GMat gmat(Fused r, Fused c) {
  GMat m;
  m.r = r;
  m.c = c;
  m.pad = 1;
  return m;
}

hs_status gpermute(hs_ctx ctx, const GMat& in, const GMat& out, std::initializer_list<int> perm,
                   const double* src, double* dst) {
  int p[kMaxLegs] = {0};
  int i = 0;
  for (int v : perm) p[i++] = v;
  PermPlan plan;
  if (!make_graded_perm_plan(in, out, p, &plan)) return fail(HS_ERR_SHAPE, "graded permute has too many legs");
  PhaseScope ps(ctx, HS_PHASE_PERMUTE);
  HS_CUDA(launch_permute_f64(plan, src, dst, 1.0, ctx->stream));
  if (plan.nbox > 0) ctx->launches += 1;
  return HS_OK;
}

// Write the conjugate of graded matrix m (stored at buf) right after it.
hs_status gconj(hs_ctx ctx, const GMat& m, double* buf) {
  PhaseScope ps(ctx, HS_PHASE_PERMUTE);
  HS_CUDA(launch_graded_sign(buf, buf + g_elems(m), fused_size(m.r, 0), fused_size(m.r, 1), fused_size(m.c, 0),
                             fused_size(m.c, 1), g_ld(m), 0, ctx->stream));
  ctx->launches += 1;
  return HS_OK;
}

// C~ = A~ B~^T (graded); B points at B~ followed by its conjugate. FP64
// kernel, or the tensor cores in the TF32/BF16 precisions (A, B and conj(B)
// split into padded hi/lo operands, the four sub-products in one launch).
hs_status ggemm(hs_ctx ctx, hs_precision prec, const GMat& Am, const double* A, const GMat& Bm, const double* B,
                const GMat& Cm, double* C, double* flops) {
  if (g_cols(Am) != g_cols(Bm)) return fail(HS_ERR_SHAPE, "graded GEMM: K mismatch");
  const GemmGroup g = make_graded_gemm(Am, Bm, Cm, g_elems(Bm));
  const double f = gemm_flops(g);
  *flops += f;
  if (prec == HS_PREC_F64) {
    PhaseScope ps(ctx, HS_PHASE_GEMM);
    HS_TRY(gemm(ctx, HS_GEMM_OWN, g, A, B, C));
    ctx->phase_flops[HS_PHASE_GEMM] += f;
    return HS_OK;
  }
  const int pad = tc_pad(prec), eb = tc_elem_bytes(prec), mode = tc_mode(prec);
  const long long K = g_cols(Am), Kp = (K + pad - 1) / pad * pad;
  const long long ra = g_rows(Am), rb = g_rows(Bm);
  HS_TRY(ctx->sx_hi.ensure((size_t)ra * Kp * eb));
  HS_TRY(ctx->sx_lo.ensure((size_t)ra * Kp * eb));
  HS_TRY(ctx->sy_hi.ensure((size_t)2 * rb * Kp * eb));
  HS_TRY(ctx->sy_lo.ensure((size_t)2 * rb * Kp * eb));
  ctx->sx_hi.zkey = ctx->sx_lo.zkey = ctx->sy_hi.zkey = ctx->sy_lo.zkey = 0;
  {
    PhaseScope ps(ctx, HS_PHASE_PERMUTE);
    HS_CUDA(launch_split_pad(A, ra, (int)K, g_ld(Am), ctx->sx_hi.p, ctx->sx_lo.p, Kp, mode, ctx->stream));
    // B~ and its conjugate (stored g_elems(Bm) apart) split back to back
    HS_CUDA(launch_split_pad(B, rb, (int)K, g_ld(Bm), ctx->sy_hi.p, ctx->sy_lo.p, Kp, mode, ctx->stream));
    HS_CUDA(launch_split_pad(B + g_elems(Bm), rb, (int)K, g_ld(Bm), static_cast<char*>(ctx->sy_hi.p) + rb * Kp * eb,
                             static_cast<char*>(ctx->sy_lo.p) + rb * Kp * eb, Kp, mode, ctx->stream));
    ctx->launches += 3;
  }
  TcProblem pr[4];
  int np = 0;
  for (int i = 0; i < g.n; ++i) {
    const GemmProblem& q = g.p[i];
    TcProblem& t = pr[np++];
    t.M = q.M;
    t.N = q.N;
    t.Kp = (int)Kp;
    t.ldc = q.ldc;
    const long long arow = q.a_off / g_ld(Am);
    const bool conj = q.b_off >= g_elems(Bm);
    const long long brow = (q.b_off - (conj ? g_elems(Bm) : 0)) / g_ld(Bm) + (conj ? rb : 0);
    t.a_hi = static_cast<const char*>(ctx->sx_hi.p) + arow * Kp * eb;
    t.a_lo = static_cast<const char*>(ctx->sx_lo.p) + arow * Kp * eb;
    t.b_hi = static_cast<const char*>(ctx->sy_hi.p) + brow * Kp * eb;
    t.b_lo = static_cast<const char*>(ctx->sy_lo.p) + brow * Kp * eb;
    t.c = C + q.c_off;
  }
  HS_TRY(ctx->splitk.ensure(kSplitKElems * sizeof(double)));
  PhaseScope ps(ctx, HS_PHASE_GEMM_TC);
  HS_CUDA(launch_gemm_tc(prec, pr, np, static_cast<int*>(ctx->tc_err.p), ctx->stream, ctx->splitk.d(),
                         kSplitKElems));
  ctx->launches += 1;
  ctx->phase_flops[HS_PHASE_GEMM_TC] += f;
  return HS_OK;
}

}  // namespace

hs_status graded_double_layer(hs_ctx ctx, const double* A, int d, int D, hs_z2_tensor* out) {
  HS_CUDA(launch_double_layer_graded(A, d, D, out->data, ctx->stream));
  return HS_OK;
}

size_t graded_tensor_bytes(int D) {
  const size_t q = (size_t)D * D;
  return q * q * q * q * sizeof(double);
}

hs_status graded_init(hs_ctx ctx, const hs_z2_tensor* a, int chi_max, hs_env* env) {
  const int D = a->D, q = D * D;
  const Sect qs = q_sect(D, HS_BASIS_HERMITIAN);
  env->chi_even = qs.n[0];
  env->chi_odd = qs.n[1];
  cudaStream_t s = ctx->stream;
  HS_CUDA(launch_ctmrg_init_graded(a->data, D, env->C, env->T, s));
  SelectOut* dsel = static_cast<SelectOut*>(ctx->sel.p);
  HS_CUDA(launch_normalize_max_to(env->C, (long long)q * q, static_cast<unsigned long long*>(ctx->scratch.p),
                                  &dsel->log_norm_C, s));
  HS_CUDA(launch_normalize_max(env->T, (long long)q * q * q, static_cast<unsigned long long*>(ctx->scratch.p) + 1,
                               dsel, s));
  HS_CUDA(cudaMemcpyAsync(&ctx->h_sel->log_norm_C, &dsel->log_norm_C, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                          s));
  // private copy of a~ followed by its conjugate: the B operand of G3 and G5
  const size_t na = (size_t)q * q * q * q;
  HS_TRY(ctx->ga.ensure(2 * na * sizeof(double)));
  HS_CUDA(cudaMemcpyAsync(ctx->ga.p, a->data, na * sizeof(double), cudaMemcpyDeviceToDevice, s));
  const GMat Am = gmat(fused2(qs, qs), fused2(qs, qs));
  HS_TRY(gconj(ctx, Am, ctx->ga.d()));
  ctx->ga_src = a->data;
  HS_CUDA(cudaStreamSynchronize(s));
  env->log_norm_C = ctx->h_sel->log_norm_C;
  env->log_norm_T = ctx->h_sel->log_norm_T;
  // workspace for the moves (dense graded sizes)
  const size_t c = (size_t)env->chi_max, n = c * q;
  HS_TRY(ctx->big1.ensure(n * n * sizeof(double)));
  HS_TRY(ctx->big2.ensure(n * n * sizeof(double)));
  HS_TRY(ctx->gb[0].ensure(2 * c * q * c * sizeof(double)));  // Tq + conj
  HS_TRY(ctx->gb[1].ensure(2 * c * c * sizeof(double)));      // C^T + conj
  HS_TRY(ctx->gb[2].ensure(c * q * c * sizeof(double)));      // X1
  HS_TRY(ctx->gb[3].ensure(n * n * sizeof(double)));          // M, then H = M M^T
  HS_TRY(ctx->gb[4].ensure(2 * c * n * sizeof(double)));      // PT + conj
  HS_TRY(ctx->gb[5].ensure(2 * c * n * sizeof(double)));      // V1, V1^T + conj
  HS_TRY(ctx->gb[6].ensure(c * n * sizeof(double)));          // Loewdin scratch
  HS_TRY(ctx->w.ensure(n * sizeof(double)));
  HS_TRY(ctx->lam.ensure(c * sizeof(double)));    // selection of the subspace eigensolver
  HS_TRY(ctx->idx.ensure(2 * c * sizeof(int)));
  HS_TRY(eig_workspace(ctx, (int)n));
  return HS_OK;
}

hs_status graded_move(hs_ctx ctx, const hs_z2_tensor* a, hs_env* env, int chi, hs_move_info* info) {
  if (ctx->ga_src != a->data)
    return fail(HS_ERR_INVALID_ARG, "the double layer changed since hs_ctmrg_init (private copy is stale)");
  cudaStream_t s = ctx->stream;
  const Sect q = make_sect(env->q_even, env->q_odd);
  const Sect c = make_sect(env->chi_even, env->chi_odd);
  const long long nchi = (long long)c.n[0] + c.n[1], nq = (long long)q.n[0] + q.n[1];
  const long long n = nchi * nq;
  const int k = (int)std::min<long long>(chi, n);
  const Sect cn = make_sect(k, 0);
  double flops = 0.0;
  const hs_precision prec = env->precision;
  double* B1 = ctx->big1.d();
  double* B2 = ctx->big2.d();
  double* Tq = ctx->gb[0].d();
  double* Ct = ctx->gb[1].d();
  double* X1 = ctx->gb[2].d();
  double* Mh = ctx->gb[3].d();
  double* PT = ctx->gb[4].d();
  double* V1 = ctx->gb[5].d();
  double* Lw = ctx->gb[6].d();
  double* A2 = ctx->ga.d();
  SelectOut* dsel = static_cast<SelectOut*>(ctx->sel.p);

  // layouts (legs in brackets: rows | columns)
  const GMat Tm = gmat(fused2(c, q), fused1(c));          // T[(alpha, x) | beta]
  const GMat Tqm = gmat(fused2(q, c), fused1(c));         // Tq[(x, beta) | alpha]
  const GMat Cm = gmat(fused1(c), fused1(c));             // C[beta | gamma]
  const GMat X1m = gmat(fused2(c, q), fused1(c));         // X1[(alpha, x) | gamma]
  const GMat X2m = gmat(fused2(c, q), fused2(q, c));      // X2[(alpha, x) | (y, eps)]
  const GMat X2pm = gmat(fused2(c, c), fused2(q, q));     // X2p[(alpha, eps) | (y, x)]
  const GMat Am = gmat(fused2(q, q), fused2(q, q));       // a~[(u, l) | (d, r)]
  const GMat X3m = gmat(fused2(c, c), fused2(q, q));      // X3[(alpha, eps) | (d, r)]
  const GMat Cpm = gmat(fused2(c, q), fused2(c, q));      // C'[(alpha, d) | (eps, r)]
  const GMat PTm = gmat(fused1(cn), fused2(c, q));        // PT[a' | (alpha, d)]
  const GMat V1m = gmat(fused2(c, q), fused1(cn));        // V1[(alpha, d) | b']
  const GMat V1tm = gmat(fused1(cn), fused2(c, q));       // V1t[b' | (alpha, d)]
  const GMat Cnm = gmat(fused1(cn), fused1(cn));          // C_new[a' | b']
  const GMat Ppm = gmat(fused2(q, cn), fused1(c));        // P'[(d, a') | alpha]
  const GMat Ym = gmat(fused2(q, cn), fused2(q, c));      // Y[(d, a') | (x, beta)]
  const GMat Ypm = gmat(fused2(cn, c), fused2(q, q));     // Yp[(a', beta) | (d, x)]
  const GMat Zm = gmat(fused2(cn, c), fused2(q, q));      // Z[(a', beta) | (u, r)]
  const GMat Zpm = gmat(fused2(cn, q), fused2(c, q));     // Zp[(a', r) | (beta, u)]
  const GMat Tnm = gmat(fused2(cn, q), fused1(cn));       // T_new[(a', r) | b']

  // ---- enlarged corner C'[(alpha,d),(eps,r)] = T[alpha,x,beta] C[beta,gamma] T[gamma,y,eps] a[y,x,d,r]
  HS_TRY(gpermute(ctx, Tm, Tqm, {1, 2, 0}, env->T, Tq));
  HS_TRY(gconj(ctx, Tqm, Tq));
  HS_TRY(gpermute(ctx, Cm, Cm, {1, 0}, env->C, Ct));
  HS_TRY(gconj(ctx, Cm, Ct));
  HS_TRY(ggemm(ctx, prec, Tm, env->T, Cm, Ct, X1m, X1, &flops));             // G1: X1 = T C
  HS_TRY(ggemm(ctx, prec, X1m, X1, Tqm, Tq, X2m, B1, &flops));               // G2: X2 = X1 T
  HS_TRY(gpermute(ctx, X2m, X2pm, {0, 3, 2, 1}, B1, B2));              // (a,x,y,e) -> (a,e,y,x)
  HS_TRY(ggemm(ctx, prec, X2pm, B2, Am, A2, X3m, B1, &flops));               // G3: X3 = X2p a
  HS_TRY(gpermute(ctx, X3m, Cpm, {0, 2, 1, 3}, B1, B2));               // (a,e,d,r) -> (a,d,e,r)
  double* Cp = B2;

  // ---- truncation: left singular vectors of C' from H = M M^T
  const long long r0 = fused_size(Cpm.r, 0), r1 = fused_size(Cpm.r, 1);
  {
    PhaseScope ps(ctx, HS_PHASE_SELECT);
    HS_CUDA(launch_graded_sign(Cp, B1, r0, r1, r0, r1, n, 1, s));  // M in B1
    ctx->launches += 1;
  }
  // H = M M^T (tensor cores in the TF32/BF16 precisions, which time themselves)
  if (prec == HS_PREC_F64) {
    PhaseScope ps(ctx, HS_PHASE_GEMM);
    HS_TRY(dense_gemm_any(ctx, prec, (int)n, (int)n, (int)n, B1, B1, Mh));
    ctx->phase_flops[HS_PHASE_GEMM] += 2.0 * n * (double)n * n;
  } else {
    HS_TRY(dense_gemm_any(ctx, prec, (int)n, (int)n, (int)n, B1, B1, Mh));
  }
  flops += 2.0 * n * (double)n * n;
  const bool f32 = env->eig_mode != HS_EIG_F64;
  // the subspace eigensolver on H (one block; H is symmetric positive
  // semi-definite, so the chi largest |eigenvalues| are the chi largest
  // singular values squared), warm-started from the previous move's Ritz
  // vectors; the full FP32 eigen-decomposition when it does not apply
  const bool sub_mode = env->eig_mode == HS_EIG_SUBSPACE || env->eig_mode == HS_EIG_SUBSPACE_ADAPTIVE;
  bool sub_done = false;
  int sub_iters = 0, sub_reason = -1, msub[2] = {0, 0};
  double sub_resid = 0.0;
  if (sub_mode) {
    ctx->cp_f32 = false;
    ctx->sH_fresh = false;
    ctx->sel_ready = false;
    HS_TRY(subspace_projector(ctx, env, k, (int)n, 0, Mh, Mh + n * n, ctx->w.d(), msub, &sub_done, &sub_iters, &flops,
                              &sub_reason, &sub_resid));
  }
  if (sub_done) {
    // the converged round's selection (ctx->idx / sel) picks the kept Ritz vectors
    PhaseScope ps(ctx, HS_PHASE_SELECT);
    HS_CUDA(launch_gather_rows(ctx->sxr.d(0), (int)n, ctx->sxr.d(1), 0, static_cast<int*>(ctx->idx.p), k, dsel, PT,
                               V1, s));
    HS_CUDA(launch_row_sign(PT, k, (int)n, s));
    HS_CUDA(cudaMemsetAsync(ctx->info.p, 0, sizeof(int), s));
    ctx->launches += 2;
  } else {
    PhaseScope ps(ctx, HS_PHASE_EIG);
    HS_CUDA(cudaMemsetAsync(ctx->info.p, 0, sizeof(int), s));
    if (!f32) {
      HS_TRY(eig_single(ctx, false, Mh, (int)n, ctx->w.p));
    } else {
      HS_TRY(ctx->c32.ensure((size_t)n * n * sizeof(float)));
      HS_TRY(ctx->w32.ensure((size_t)n * sizeof(float)));
      HS_TRY(eig_workspace32(ctx, (int)n));
      HS_CUDA(launch_cast_f64_f32(Mh, static_cast<float*>(ctx->c32.p), n * n, s));
      HS_TRY(eig_single(ctx, true, ctx->c32.p, (int)n, ctx->w32.p));
    }
  }
  if (!sub_done) {
    PhaseScope ps(ctx, HS_PHASE_SELECT);
    if (!f32)
      HS_CUDA(launch_graded_select(ctx->w.d(), Mh, (int)n, k, PT, dsel, s));
    else
      HS_CUDA(launch_graded_select32(static_cast<const float*>(ctx->w32.p), static_cast<const float*>(ctx->c32.p),
                                     (int)n, k, PT, dsel, s));
    HS_CUDA(launch_row_sign(PT, k, (int)n, s));  // canonical sign: largest entry of each row positive
    ctx->launches += 2;
  }
  if (sub_mode) {
    // warm start of the next move: the Ritz vectors, or the m eigenvectors of
    // largest eigenvalue after a full decomposition
    const int mnext = sub_done ? msub[0] : std::min(std::min(k + oversample(k), (int)n), max_subspace());
    HS_TRY(ctx->ws_pt.ensure(((size_t)mnext * n + 1) * sizeof(double)));
    HS_TRY(ctx->sf_idx.ensure(((size_t)mnext + 1) * sizeof(int)));
    if (sub_done)
      HS_CUDA(cudaMemcpyAsync(ctx->ws_pt.d(), ctx->sxr.d(0), (size_t)mnext * n * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
    else
      HS_CUDA(launch_top_rows(static_cast<const float*>(ctx->w32.p), static_cast<const float*>(ctx->c32.p), (int)n,
                              mnext, static_cast<int*>(ctx->sf_idx.p), ctx->ws_pt.d(), s));
    ctx->ws_env = env;
    ctx->ws_valid = true;
    ctx->ws_c[0] = ctx->ws_c[1] = -1;  // graded rows are not remapped
    ctx->ws_k[0] = k;
    ctx->ws_k[1] = 0;
    ctx->ws_m[0] = mnext;
    ctx->ws_m[1] = 0;
    ctx->ws_n[0] = (int)n;
    ctx->ws_n[1] = 0;
    ctx->ws_moves += 1;
  }
  // Ritz vectors are orthonormal to ~1e-6 (FP32 Rayleigh-Ritz), FP32 eigenvectors to ~1e-7
  if (f32) HS_TRY(lowdin_rows(ctx, HS_PREC_F64, PT, k, (int)n, Lw, sub_done ? 1 : 2));
  HS_TRY(gconj(ctx, PTm, PT));
  double* PTc = PT + g_elems(PTm);

  // ---- C_new = P^dagger C' P
  HS_TRY(ggemm(ctx, prec, Cpm, Cp, PTm, PT, V1m, V1, &flops));               // V1 = C' P
  double* V1t = B1;
  HS_TRY(gpermute(ctx, V1m, V1tm, {2, 0, 1}, V1, V1t));
  HS_TRY(gconj(ctx, V1tm, V1t));
  HS_TRY(ggemm(ctx, prec, PTm, PTc, V1tm, V1t, Cnm, env->C, &flops));        // C_new = conj(P)^T V1

  // ---- T_new[a', r, b'] = conj(P[(alpha,d),a']) T[alpha,x,beta] a[u,x,d,r] P[(beta,u),b']
  double* Pp = V1;
  HS_TRY(gpermute(ctx, PTm, Ppm, {2, 0, 1}, PTc, Pp));                 // (a',alpha,d) -> (d,a',alpha)
  HS_TRY(ggemm(ctx, prec, Ppm, Pp, Tqm, Tq, Ym, B1, &flops));                // G4: Y = conj(P') T
  HS_TRY(gpermute(ctx, Ym, Ypm, {1, 3, 0, 2}, B1, B2));                // (d,a',x,b) -> (a',b,d,x)
  HS_TRY(ggemm(ctx, prec, Ypm, B2, Am, A2, Zm, B1, &flops));                 // G5: Z = Yp a
  HS_TRY(gpermute(ctx, Zm, Zpm, {0, 3, 1, 2}, B1, B2));                // (a',b,u,r) -> (a',r,b,u)
  HS_TRY(ggemm(ctx, prec, Zpm, B2, PTm, PT, Tnm, env->T, &flops));           // G6: T_new = Zp P

  // ---- normalise
  {
    PhaseScope ps(ctx, HS_PHASE_NORMALIZE);
    HS_CUDA(launch_normalize_max_to(env->C, g_elems(Cnm), static_cast<unsigned long long*>(ctx->scratch.p) + 2,
                                    &dsel->log_norm_C, s));
    HS_CUDA(launch_normalize_max(env->T, g_elems(Tnm), static_cast<unsigned long long*>(ctx->scratch.p), dsel, s));
    ctx->launches += 4;
  }
  HS_CUDA(cudaMemcpyAsync(ctx->h_sel, dsel, sizeof(SelectOut), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaMemcpyAsync(ctx->h_info, ctx->info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  harvest_profile(ctx);
  if (*ctx->h_info != 0) return fail(HS_ERR_SOLVER, "eigensolver info %d", *ctx->h_info);
  SelectOut sel = *ctx->h_sel;
  if (sub_done) {
    // the subspace selection ranks eigenvalues of H: singular values are their square roots
    sel.lam_max = std::sqrt(std::fabs(sel.lam_max));
    sel.lam_cut = std::sqrt(std::fabs(sel.lam_cut));
    sel.lam_next = std::sqrt(std::fabs(sel.lam_next));
  }
  env->chi_even = k;
  env->chi_odd = 0;
  env->log_norm_C = sel.log_norm_C;
  env->log_norm_T = sel.log_norm_T;
  env->moves += 1;
  if (!std::isfinite(env->log_norm_T) || !std::isfinite(env->log_norm_C))
    return fail(HS_ERR_NONFINITE, "environment is not finite after the move");
  if (info) {
    info->chi_even = k;
    info->chi_odd = 0;
    info->n_even = (int)n;
    info->n_odd = 0;
    info->lam_max = sel.lam_max;
    info->lam_cut = sel.lam_cut;
    info->lam_next = sel.lam_next;
    const bool discarded = k < n;
    info->gap = discarded ? (sel.lam_cut - sel.lam_next) / sel.lam_max : INFINITY;
    info->log_norm_C = env->log_norm_C;
    info->log_norm_T = env->log_norm_T;
    info->gemm_flops = flops;
    info->flags = ((discarded && info->gap < 1e-9) ? 1 : 0) | (sub_mode ? (sub_done ? 2 : 4) : 0);
    info->subspace_iters = sub_iters;
    info->subspace_reason = sub_reason;
    info->subspace_resid = sub_resid;
  }
  return HS_OK;
}

}  // namespace hs

// HOTRG coarse-graining in the Hermitian Z2 basis (arXiv 2410.11596 Sec. II.A,
// Ref. xie12; Sec. II.B: in HOTRG essentially every step involves only the
// combined bra-ket spaces, so every contraction and eigen-decomposition below
// is block-sparse).
//
// Tensor T[u, l, d, r] in FSO storage [(u, l) | (d, r)]; u and d carry the
// vertical sectors v, l and r the horizontal sectors h. A vertical step stacks
// two copies (top one's d = bottom one's u = k):
//   M[u, (l1 l2), d, (r1 r2)] = sum_k T[u, l1, k, r1] T[k, l2, d, r2]
// and truncates each fused horizontal leg with the top-chi eigenvectors of a
// Gram matrix, built without forming M:
//   A1[(l1 k), (l1' k')] = sum_{u r1} T[u l1 k r1] T[u l1' k' r1]
//   A2[(k l2), (k' l2')] = sum_{d r2} T[k l2 d r2] T[k' l2' d r2]
//   G[(l1 l2), (l1' l2')] = sum_{k k'} A1 A2.
// The right Gram matrix is the same on the mirrored tensor (l <-> r). The
// new tensor is T'[u, L, d, R] = sum U[(l1 l2), L] M[...] U[(r1 r2), R].
#include "hs_ctx.cuh"

using namespace hs;

namespace {

// Gram matrix of the fused left leg of T (layout Tm) into G, FSO
// [(l1 l2) | (l1' l2')]. Workspace: hb[0..5].
hs_status gram_left(hs_ctx ctx, const double* T, Sect v, Sect h, double* G) {
  DBuf* b = ctx->hb;
  const Z2Mat Tm = mat(fused2(v, h), fused2(v, h));
  const Z2Mat Tp = mat(fused2(h, v), fused2(v, h));      // [(l, d) | (u, r)]
  const Z2Mat A1 = mat(fused2(h, v), fused2(h, v));      // [(l1, k) | (l1', k')]
  const Z2Mat A2 = mat(fused2(v, h), fused2(v, h));      // [(k, l2) | (k', l2')]
  const Z2Mat A1p = mat(fused2(h, h), fused2(v, v));     // [(l1, l1') | (k, k')]
  const Z2Mat A2p = mat(fused2(h, h), fused2(v, v));     // [(l2, l2') | (k, k')]
  const Z2Mat Gp = mat(fused2(h, h), fused2(h, h));      // [(l1, l1') | (l2, l2')]
  const Z2Mat Gm = mat(fused2(h, h), fused2(h, h));      // [(l1, l2) | (l1', l2')]
  HS_TRY(b[0].ensure(z2_elems(Tp) * 8));
  HS_TRY(b[1].ensure(z2_elems(A1) * 8));
  HS_TRY(b[2].ensure(z2_elems(A2) * 8));
  HS_TRY(b[3].ensure(z2_elems(A1p) * 8));
  HS_TRY(b[4].ensure(z2_elems(A2p) * 8));
  HS_TRY(b[5].ensure(z2_elems(Gp) * 8));
  HS_TRY(permute(ctx, Tm, Tp, {1, 2, 0, 3}, T, b[0].d()));
  HS_TRY(gemm(ctx, HS_GEMM_OWN, make_z2_gemm(Tp, Tp, A1), b[0].d(), b[0].d(), b[1].d()));
  HS_TRY(gemm(ctx, HS_GEMM_OWN, make_z2_gemm(Tm, Tm, A2), T, T, b[2].d()));
  HS_TRY(permute(ctx, A1, A1p, {0, 2, 1, 3}, b[1].d(), b[3].d()));
  HS_TRY(permute(ctx, A2, A2p, {1, 3, 0, 2}, b[2].d(), b[4].d()));
  HS_TRY(gemm(ctx, HS_GEMM_OWN, make_z2_gemm(A1p, A2p, Gp), b[3].d(), b[4].d(), b[5].d()));
  HS_TRY(permute(ctx, Gp, Gm, {0, 2, 1, 3}, b[5].d(), G));
  return HS_OK;
}

// gram_left with the three products on the tensor cores: each operand is
// split straight from its source by the split's permute (no separate permute
// pass), the products come out in FP64.
hs_status gram_left_tc(hs_ctx ctx, hs_precision prec, const double* T, Sect v, Sect h, double* G) {
  DBuf* b = ctx->hb;
  const Z2Mat Tm = mat(fused2(v, h), fused2(v, h));
  const Z2Mat Tp = mat(fused2(h, v), fused2(v, h));      // [(l, d) | (u, r)]
  const Z2Mat A1 = mat(fused2(h, v), fused2(h, v));      // [(l1, k) | (l1', k')]
  const Z2Mat A2 = mat(fused2(v, h), fused2(v, h));      // [(k, l2) | (k', l2')]
  const Z2Mat A1p = mat(fused2(h, h), fused2(v, v));     // [(l1, l1') | (k, k')]
  const Z2Mat A2p = mat(fused2(h, h), fused2(v, v));     // [(l2, l2') | (k, k')]
  const Z2Mat Gp = mat(fused2(h, h), fused2(h, h));      // [(l1, l1') | (l2, l2')]
  const Z2Mat Gm = mat(fused2(h, h), fused2(h, h));      // [(l1, l2) | (l1', l2')]
  HS_TRY(b[1].ensure(z2_elems(A1) * 8));
  HS_TRY(b[2].ensure(z2_elems(A2) * 8));
  HS_TRY(b[5].ensure(z2_elems(Gp) * 8));
  HS_TRY(tc_split(ctx, prec, Tm, Tp, {1, 2, 0, 3}, T, ctx->sx_hi, ctx->sx_lo));
  HS_TRY(tc_run(ctx, prec, Tp, ctx->sx_hi, ctx->sx_lo, Tp, ctx->sx_hi, ctx->sx_lo, A1, b[1].d()));
  HS_TRY(tc_split(ctx, prec, Tm, Tm, {0, 1, 2, 3}, T, ctx->sy_hi, ctx->sy_lo));
  HS_TRY(tc_run(ctx, prec, Tm, ctx->sy_hi, ctx->sy_lo, Tm, ctx->sy_hi, ctx->sy_lo, A2, b[2].d()));
  HS_TRY(tc_split(ctx, prec, A1, A1p, {0, 2, 1, 3}, b[1].d(), ctx->sx_hi, ctx->sx_lo));
  HS_TRY(tc_split(ctx, prec, A2, A2p, {1, 3, 0, 2}, b[2].d(), ctx->sy_hi, ctx->sy_lo));
  HS_TRY(tc_run(ctx, prec, A1p, ctx->sx_hi, ctx->sx_lo, A2p, ctx->sy_hi, ctx->sy_lo, Gp, b[5].d()));
  HS_TRY(permute(ctx, Gp, Gm, {0, 2, 1, 3}, b[5].d(), G));
  return HS_OK;
}

unsigned long long* scratch(hs_ctx ctx, int i) { return static_cast<unsigned long long*>(ctx->scratch.p) + i; }

}  // namespace

extern "C" size_t hs_hotrg_tensor_bytes(int D, int chi) {
  if (D <= 0 || chi <= 0) return 0;
  const size_t x = (size_t)(chi > D * D ? chi : D * D);
  return x * x * x * x * sizeof(double);
}

// ln Z / N of a run of `steps` coarse-graining steps. Each step halves the
// number of tensors, so the normalisation factor of step k is shared by 2^k
// sites; the last tensor, closed on itself, stands for the rest of the
// lattice. The terms are added in step order.
extern "C" hs_status hs_hotrg_log_z(const double* log_norms, int steps, double trace, double* log_z) {
  if (!log_norms || !log_z || steps < 1) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (!(trace > 0.0) || !std::isfinite(trace)) return fail(HS_ERR_NONFINITE, "trace %g is not positive", trace);
  double sum = 0.0, w = 1.0;
  for (int k = 1; k <= steps; ++k) {
    w *= 0.5;
    sum += log_norms[k] * w;
  }
  const double v = (log_norms[0] + sum) + std::log(trace) * w;
  if (!std::isfinite(v)) return fail(HS_ERR_NONFINITE, "ln Z is not finite");
  *log_z = v;
  return HS_OK;
}

extern "C" hs_status hs_hotrg_init(hs_ctx ctx, const hs_z2_tensor* a, hs_z2_tensor* t, double* log_norm) {
  HS_TRY(check_ctx(ctx));
  if (!a || !t || !a->data || !t->data || !log_norm) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  const Sect q = make_sect(a->n_even, a->n_odd);
  const Z2Mat Am = mat(fused2(q, q), fused2(q, q));
  const size_t nb = z2_elems(Am) * sizeof(double);
  if (t->capacity_bytes < nb) return fail(HS_ERR_WORKSPACE, "tensor buffer holds %zu bytes, %zu needed", t->capacity_bytes, nb);
  HS_CUDA(cudaMemcpyAsync(t->data, a->data, nb, cudaMemcpyDeviceToDevice, ctx->stream));
  SelectOut* dsel = static_cast<SelectOut*>(ctx->sel.p);
  HS_CUDA(launch_normalize_max_to(t->data, z2_elems(Am), scratch(ctx, 3), &dsel->log_norm_T, ctx->stream));
  HS_CUDA(cudaMemcpyAsync(log_norm, &dsel->log_norm_T, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  HS_CUDA(cudaStreamSynchronize(ctx->stream));
  t->D = a->D;
  t->n_even = a->n_even;
  t->n_odd = a->n_odd;
  t->basis = a->basis;
  t->dtype = a->dtype;
  t->v_even = t->h_even = a->n_even;
  t->v_odd = t->h_odd = a->n_odd;
  return HS_OK;
}

extern "C" hs_status hs_hotrg_step(hs_ctx ctx, hs_z2_tensor* t, int chi, int direction, hs_precision precision,
                                   hs_hotrg_info* info) {
  HS_TRY(check_ctx(ctx));
  if (!t || !t->data || chi < 1 || (direction != 0 && direction != 1))
    return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (precision != HS_PREC_F64 && precision != HS_PREC_TF32X3 && precision != HS_PREC_TF32 &&
      precision != HS_PREC_BF16X3)
    return fail(HS_ERR_INVALID_ARG, "unknown precision %d", (int)precision);
  const bool tc = precision != HS_PREC_F64;
  cudaStream_t s = ctx->stream;
  DBuf* b = ctx->hb;
  // the step always stacks vertically; a horizontal step works on the tensor
  // turned by 90 degrees, R[u, l, d, r] = T[l, d, r, u] (R's left leg is T's
  // upper one, so side 0 of a horizontal step is the upper legs), and turns it back
  Sect v = make_sect(t->v_even, t->v_odd), h = make_sect(t->h_even, t->h_odd);
  const Z2Mat T0m = mat(fused2(v, h), fused2(v, h));
  double* T = t->data;
  if (direction == 1) {
    const Z2Mat Rm = mat(fused2(h, v), fused2(h, v));
    HS_TRY(b[6].ensure(z2_elems(T0m) * 8));
    HS_TRY(permute(ctx, T0m, Rm, {3, 0, 1, 2}, t->data, b[6].d()));
    T = b[6].d();
    const Sect tmp = v;
    v = h;
    h = tmp;
  }
  const Z2Mat Tm = mat(fused2(v, h), fused2(v, h));
  const Z2Mat Gm = mat(fused2(h, h), fused2(h, h));
  const int n0 = (int)z2_rows(Gm, 0), n1 = (int)z2_rows(Gm, 1);
  HS_TRY(b[7].ensure(z2_elems(Gm) * 8));
  HS_TRY(b[8].ensure(z2_elems(Gm) * 8));
  HS_TRY(b[9].ensure(z2_elems(Tm) * 8));
  HS_TRY(b[10].ensure((size_t)2 * (n0 + n1) * 8));
  HS_TRY(b[11].ensure((size_t)2 * 2 * chi * sizeof(int) + 2 * sizeof(SelectOut) + 2 * chi * 8));
  double* GL = b[7].d();
  double* GR = b[8].d();
  double* Tmir = b[9].d();
  double* wL = b[10].d();
  double* wR = wL + n0 + n1;
  SelectOut* selL = reinterpret_cast<SelectOut*>(b[11].p);
  SelectOut* selR = selL + 1;
  int* idxL = reinterpret_cast<int*>(selL + 2);
  int* idxR = idxL + 2 * chi;
  double* lam = reinterpret_cast<double*>(idxR + 2 * chi);

  // Gram matrices of the fused left leg and (on the mirrored tensor) of the
  // fused right leg; one eigen-decomposition per parity block of each
  HS_TRY(permute(ctx, Tm, Tm, {0, 3, 2, 1}, T, Tmir));
  if (tc) {
    HS_TRY(gram_left_tc(ctx, precision, T, v, h, GL));
    HS_TRY(gram_left_tc(ctx, precision, Tmir, v, h, GR));
  } else {
    HS_TRY(gram_left(ctx, T, v, h, GL));
    HS_TRY(gram_left(ctx, Tmir, v, h, GR));
  }
  HS_TRY(eig_workspace(ctx, n0 > n1 ? n0 : n1));
  HS_CUDA(cudaMemsetAsync(ctx->info.p, 0, 2 * sizeof(int), s));
  HS_TRY(eig_pair(ctx, false, GL, n0, wL, GL + (long long)n0 * n0, n1, wL + n0));
  HS_CUDA(launch_select(wL, n0, wL + n0, n1, chi, idxL, lam, selL, s));
  HS_TRY(eig_pair(ctx, false, GR, n0, wR, GR + (long long)n0 * n0, n1, wR + n0));
  HS_CUDA(launch_select(wR, n0, wR + n0, n1, chi, idxR, lam, selR, s));
  SelectOut hsel[2];
  int hinfo[2];
  HS_CUDA(cudaMemcpyAsync(hsel, selL, sizeof hsel, cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaMemcpyAsync(hinfo, ctx->info.p, sizeof hinfo, cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  if (hinfo[0] != 0 || hinfo[1] != 0) return fail(HS_ERR_SOLVER, "syevd info = (%d, %d)", hinfo[0], hinfo[1]);
  const int side = hsel[0].discarded <= hsel[1].discarded ? 0 : 1;
  const SelectOut sel = hsel[side];
  const Sect hn = make_sect(sel.chi_new[0], sel.chi_new[1]);

  // isometry rows UT[L | (l1, l2)]
  const Z2Mat UT = mat(fused1(hn), fused2(h, h));
  HS_TRY(b[12].ensure(z2_elems(UT) * 8));
  double* Gs = side == 0 ? GL : GR;
  HS_CUDA(launch_gather_pt(Gs, n0, Gs + (long long)n0 * n0, n1, side == 0 ? idxL : idxR, chi,
                           side == 0 ? selL : selR, b[12].d(), s));

  // M'[(u, l1, r1) | (l2, d, r2)] = T_top[(u, l, r) | d] T_bot[(l, d, r) | u]^T
  const Z2Mat Ttop = mat(fused3(v, h, h), fused1(v)), Tbot = mat(fused3(h, v, h), fused1(v));
  const Z2Mat Mm = mat(fused3(v, h, h), fused3(h, v, h));
  const Z2Mat Mp = mat(fused4(v, v, h, h), fused2(h, h));    // [(u, d, r1, r2) | (l1, l2)]
  const Z2Mat Ym = mat(fused4(v, v, h, h), fused1(hn));      // [(u, d, r1, r2) | L]
  const Z2Mat Yp = mat(fused3(v, hn, v), fused2(h, h));      // [(u, L, d) | (r1, r2)]
  const Z2Mat T3 = mat(fused3(v, hn, v), fused1(hn));        // [(u, L, d) | R]
  const Z2Mat Tn = mat(fused2(v, hn), fused2(v, hn));        // [(u, L) | (d, R)]
  HS_TRY(b[0].ensure(z2_elems(Ttop) * 8));
  HS_TRY(b[1].ensure(z2_elems(Tbot) * 8));
  HS_TRY(b[13].ensure(z2_elems(Mm) * 8));
  HS_TRY(b[14].ensure(z2_elems(Mp) * 8));
  HS_TRY(b[15].ensure(z2_elems(Ym) * 8));
  if (tc) {
    // every operand split straight from its source layout by the split's permute
    HS_TRY(tc_split(ctx, precision, Tm, Ttop, {0, 1, 3, 2}, T, ctx->sx_hi, ctx->sx_lo));
    HS_TRY(tc_split(ctx, precision, Tm, Tbot, {1, 2, 3, 0}, T, ctx->sy_hi, ctx->sy_lo));
    HS_TRY(tc_run(ctx, precision, Ttop, ctx->sx_hi, ctx->sx_lo, Tbot, ctx->sy_hi, ctx->sy_lo, Mm, b[13].d()));
    HS_TRY(tc_split(ctx, precision, Mm, Mp, {0, 4, 2, 5, 1, 3}, b[13].d(), ctx->sx_hi, ctx->sx_lo));
    HS_TRY(tc_split(ctx, precision, UT, UT, {0, 1, 2}, b[12].d(), ctx->sy_hi, ctx->sy_lo));
    HS_TRY(tc_run(ctx, precision, Mp, ctx->sx_hi, ctx->sx_lo, UT, ctx->sy_hi, ctx->sy_lo, Ym, b[15].d()));
    HS_TRY(tc_split(ctx, precision, Ym, Yp, {0, 4, 1, 2, 3}, b[15].d(), ctx->sx_hi, ctx->sx_lo));
    HS_TRY(tc_run(ctx, precision, Yp, ctx->sx_hi, ctx->sx_lo, UT, ctx->sy_hi, ctx->sy_lo, T3, b[14].d()));
  } else {
    HS_TRY(permute(ctx, Tm, Ttop, {0, 1, 3, 2}, T, b[0].d()));
    HS_TRY(permute(ctx, Tm, Tbot, {1, 2, 3, 0}, T, b[1].d()));
    HS_TRY(gemm(ctx, HS_GEMM_OWN, make_z2_gemm(Ttop, Tbot, Mm), b[0].d(), b[1].d(), b[13].d()));
    HS_TRY(permute(ctx, Mm, Mp, {0, 4, 2, 5, 1, 3}, b[13].d(), b[14].d()));
    HS_TRY(gemm(ctx, HS_GEMM_OWN, make_z2_gemm(Mp, UT, Ym), b[14].d(), b[12].d(), b[15].d()));
    HS_TRY(permute(ctx, Ym, Yp, {0, 4, 1, 2, 3}, b[15].d(), b[13].d()));
    HS_TRY(gemm(ctx, HS_GEMM_OWN, make_z2_gemm(Yp, UT, T3), b[13].d(), b[12].d(), b[14].d()));
  }
  const size_t need = z2_elems(Tn) * 8;
  if (t->capacity_bytes < need)
    return fail(HS_ERR_WORKSPACE, "tensor buffer holds %zu bytes, %zu needed", t->capacity_bytes, need);
  if (direction == 0) {
    HS_TRY(permute(ctx, T3, Tn, {0, 1, 2, 3}, b[14].d(), t->data));
  } else {
    // turn back: T[u, l, d, r] = R[r, u, l, d]
    HS_TRY(permute(ctx, T3, Tn, {0, 1, 2, 3}, b[14].d(), b[13].d()));
    const Z2Mat Back = mat(fused2(hn, v), fused2(hn, v));
    HS_TRY(permute(ctx, Tn, Back, {1, 2, 3, 0}, b[13].d(), t->data));
  }
  const long long nt = (long long)(need / 8);
  SelectOut* dsel = static_cast<SelectOut*>(ctx->sel.p);
  HS_CUDA(launch_normalize_max_to(t->data, nt, scratch(ctx, 4), &dsel->log_norm_T, s));
  // the trace sum_{u,l} T[u,l,u,l] is the trace of the block-diagonal matrix
  const Sect vn = direction == 0 ? v : hn, hh = direction == 0 ? hn : v;
  const Z2Mat Out = mat(fused2(vn, hh), fused2(vn, hh));
  HS_CUDA(launch_block_trace(t->data, (int)z2_rows(Out, 0), (int)z2_rows(Out, 1), &dsel->lam_next, s));
  double hout[2];
  HS_CUDA(cudaMemcpyAsync(&hout[0], &dsel->log_norm_T, sizeof(double), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaMemcpyAsync(&hout[1], &dsel->lam_next, sizeof(double), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  t->v_even = vn.n[0];
  t->v_odd = vn.n[1];
  t->h_even = hh.n[0];
  t->h_odd = hh.n[1];
  if (info) {
    info->h_even = hn.n[0];
    info->h_odd = hn.n[1];
    info->side = side;
    info->discarded_left = hsel[0].discarded;
    info->discarded_right = hsel[1].discarded;
    info->log_norm = hout[0];
    info->trace = hout[1];
  }
  if (!std::isfinite(hout[0]) || !std::isfinite(hout[1])) return fail(HS_ERR_NONFINITE, "HOTRG tensor not finite");
  return HS_OK;
}

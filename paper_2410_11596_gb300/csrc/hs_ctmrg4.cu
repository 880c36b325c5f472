// Directional CTMRG without lattice symmetry (arXiv 2410.11596, Sec. II.A
// without its C4v assumption): four corners and four edges, one side of the
// boundary moved at a time, its bonds truncated with oblique projectors from
// the SVD of the two quarters (enlarged corners) on that side. Every tensor
// keeps the Z2 block layout of the Hermitian basis (Sec. II.B), or the
// one-block layout of the plain basis; the contractions are the Z2 block
// GEMMs and permutes of the C4v path, the SVD one Jacobi SVD per parity block.
//
// Frames. Turning the lattice by 90 degrees counter-clockwise moves the top
// side to the left. In frame g the frame's corner j is corner (j + g) mod 4,
// its edge j is edge (j + g) mod 4, its bond b is bond (b + g) mod 4, and its
// double layer is a turned g times: leg j of a_g is leg (j - g) mod 4 of a
// (a_1[u, l, d, r] = a[l, d, r, u]). Moving side `direction` is moving the
// left side of frame f = direction, so the move is written once, for the
// left side:
//
//   Q1 = T4 C1 T1 a        the frame's upper-left quarter  [(L, d) | (T, r)]
//   Q4 = quarter of frame f-1, the lower-left one          [(B, r) | (L, u)]
//   X  = Q1^T Q4^T = U S V^T, one SVD per parity block; keep chi
//   P_a^T = S^-1/2 V^T Q4,  P_b^T = S^-1/2 U^T Q1^T        [c | (L, q)]
//   C1 <- P_a^T (C1 T1),  T4 <- P_a^T (T4 a) P_b,  C4 <- (T3 C4) P_b
//
// with L, T, B the frame's left, top and bottom bonds and q the double-layer
// leg. Each updated tensor is divided by its largest modulus.

#include "hs_ctx.cuh"

#include <algorithm>

namespace hs {
namespace {

constexpr double kSvCutoff = 1e-12;  // singular values below this fraction of the largest are never kept

int mod4(int x) { return ((x % 4) + 4) % 4; }

// Blocks of 256 threads for a grid-stride loop over n elements: one per 256
// elements, at most 32 per SM.
unsigned grid_of(long long n) {
  const long long g = (n + 255) / 256;
  return (unsigned)std::max(1ll, std::min(g, 32ll * device_sms()));
}

// dst row r = scale[r] * (src row idx[r]), rows of n elements.
__global__ void gather_scale_rows_kernel(const double* __restrict__ src, int n, const int* __restrict__ idx,
                                         const double* __restrict__ scale, double* __restrict__ dst) {
  hs_pdl_enter();
  const long long s = (long long)idx[blockIdx.x] * n, d = (long long)blockIdx.x * n;
  const double f = scale[blockIdx.x];
  for (int j = threadIdx.x; j < n; j += blockDim.x) dst[d + j] = f * src[s + j];
}

// Dense [r0 + r1, c0 + c1] copy of a two-block Z2 matrix (block 0 r0 x c0,
// then block 1 r1 x c1, each row-major and tightly packed).
__global__ void corner_dense_kernel(const double* __restrict__ C, int r0, int r1, int c0, int c1,
                                    double* __restrict__ Cd) {
  hs_pdl_enter();
  const int cols = c0 + c1;
  const long long n = (long long)(r0 + r1) * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / cols), b = (int)(e % cols);
    const int pa = a >= r0, pb = b >= c0;
    double v = 0.0;
    if (pa == pb)
      v = pa ? C[(long long)r0 * c0 + (long long)(a - r0) * c1 + (b - c0)] : C[(long long)a * c0 + b];
    Cd[e] = v;
  }
}

cudaError_t launch_gather_scale_rows(const double* src, int n, const int* idx, const double* scale, int m,
                                     double* dst, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  hs_launch(gather_scale_rows_kernel, m, 128, 0, s, src, n, idx, scale, dst);
  return cudaGetLastError();
}

// Workspace slots in ctx->d4.
enum {
  kAq = 0,   // a_g as [(d, r) | (u, l)], g = 0..3: B operand of the quarter's last GEMM
  kAr = 4,   // a_g as [(u, r) | (l, d)]: B operand of the edge update
  kQ1 = 8, kQ4, kQ1t, kQ4t, kY1, kY2, kY3, kP1, kP2, kX, kU, kV, kS, kWork, kInfo,
  kVl, kVr, kPa, kPb, kW1, kW2, kOut0, kOut1, kOut2, kIdx, kScale, kLog,
  kSlots
};
static_assert(kSlots <= (int)(sizeof(((hs_ctx_s*)nullptr)->d4) / sizeof(DBuf)), "d4 slots");

Sect bond(const hs_env4* e, int b) { return make_sect(e->chi_even[mod4(b)], e->chi_odd[mod4(b)]); }

struct Flops {
  double f = 0;
  void add(const GemmGroup& g) { f += gemm_flops(g); }
};

hs_status gemm4(hs_ctx ctx, Flops& fl, const Z2Mat& A, const Z2Mat& B, const Z2Mat& C, const double* a,
                const double* b, double* c) {
  const GemmGroup g = make_z2_gemm(A, B, C);
  fl.add(g);
  return gemm(ctx, HS_GEMM_OWN, g, a, b, c);
}

// The upper-left quarter of frame g, Q[(left bond, d) | (top bond, r)] =
// sum T4[alpha, x, b] C1[b, g] T1[g, y, beta] a_g[y, x, d, r], into Q.
hs_status quarter(hs_ctx ctx, const hs_env4* env, int g, Sect q, double* Q, Flops& fl) {
  const Sect cL = bond(env, g - 1), cT = bond(env, g);
  const double* T4 = env->T[mod4(g - 1)];
  const double* C1 = env->C[mod4(g)];
  const double* T1 = env->T[mod4(g)];
  double* P1 = ctx->d4[kP1].d();
  double* P2 = ctx->d4[kP2].d();
  double* Y1 = ctx->d4[kY1].d();
  double* Y2 = ctx->d4[kY2].d();
  double* Y3 = ctx->d4[kY3].d();
  const Z2Mat T4m = mat(fused2(cL, q), fused1(cL));
  const Z2Mat C1m = mat(fused1(cL), fused1(cT)), C1t = mat(fused1(cT), fused1(cL));
  const Z2Mat T1m = mat(fused2(cT, q), fused1(cT)), T1p = mat(fused2(q, cT), fused1(cT));
  const Z2Mat Y1m = mat(fused2(cL, q), fused1(cT));
  const Z2Mat Y2m = mat(fused2(cL, q), fused2(q, cT));
  const Z2Mat Y2p = mat(fused2(cL, cT), fused2(q, q));
  const Z2Mat Aq = mat(fused2(q, q), fused2(q, q));
  const Z2Mat Y3m = mat(fused2(cL, cT), fused2(q, q));
  const Z2Mat Qm = mat(fused2(cL, q), fused2(cT, q));
  HS_TRY(permute(ctx, C1m, C1t, {1, 0}, C1, P1));                      // C1^T [g | b]
  HS_TRY(permute(ctx, T1m, T1p, {1, 2, 0}, T1, P2));                   // T1 as [(y, beta) | g]
  HS_TRY(gemm4(ctx, fl, T4m, C1t, Y1m, T4, P1, Y1));                   // [(alpha, x) | g]
  HS_TRY(gemm4(ctx, fl, Y1m, T1p, Y2m, Y1, P2, Y2));                   // [(alpha, x) | (y, beta)]
  HS_TRY(permute(ctx, Y2m, Y2p, {0, 3, 2, 1}, Y2, Y3));                // [(alpha, beta) | (y, x)]
  HS_TRY(gemm4(ctx, fl, Y2p, Aq, Y3m, Y3, ctx->d4[kAq + mod4(g)].d(), Y2));  // [(alpha, beta) | (d, r)]
  HS_TRY(permute(ctx, Y3m, Qm, {0, 2, 1, 3}, Y2, Q));                  // [(alpha, d) | (beta, r)]
  return HS_OK;
}

hs_status ensure_workspace(hs_ctx ctx, int chi_max, int q) {
  const size_t c = (size_t)chi_max, cq = c * q, d = sizeof(double);
  const size_t big = cq * cq * d;
  for (int k : {kQ1, kQ4, kQ1t, kQ4t, kY2, kY3, kX, kU, kV, kW1, kW2}) HS_TRY(ctx->d4[k].ensure(big));
  for (int k : {kY1, kP2, kVl, kVr, kPa, kPb, kOut1}) HS_TRY(ctx->d4[k].ensure(c * cq * d));
  for (int k : {kP1, kOut0, kOut2}) HS_TRY(ctx->d4[k].ensure(c * c * d));
  HS_TRY(ctx->d4[kS].ensure(2 * cq * d));
  HS_TRY(ctx->d4[kInfo].ensure(4 * sizeof(int)));
  HS_TRY(ctx->d4[kIdx].ensure(2 * c * sizeof(int)));
  HS_TRY(ctx->d4[kScale].ensure(2 * c * d));
  HS_TRY(ctx->d4[kLog].ensure(8 * d));
  HS_TRY(ctx->d4_h.ensure(2 * cq * d + 2 * c * (sizeof(int) + d) + 16 * d));
  if (!ctx->gesvdj) HS_SOLVER(cusolverDnCreateGesvdjInfo(&ctx->gesvdj));
  return HS_OK;
}

// SVD of the row-major block X (m x n, tightly packed): the min(m, n)
// singular values to S, the left singular vectors as contiguous columns of L
// (m long), the right ones of R (n long); status to *dinfo. Both methods work
// on the tall orientation. polar: cuSOLVER Xgesvdp (polar factor, then a
// symmetric eigensolver), falling back to the Jacobi SVD where it reports a
// failure; else the one-sided Jacobi SVD (gesvdj).
hs_status block_svd(hs_ctx ctx, bool polar, double* X, int m, int n, double* S, double* L, double* R, int* dinfo) {
  cudaStream_t s = ctx->stream;
  HS_SOLVER(cusolverDnSetStream(ctx->solver, s));
  // column-major view of the tall orientation: X^T (n x m) when n >= m,
  // else X itself (m x n, a transposed copy)
  const bool tall_t = n >= m;
  const int rows = tall_t ? n : m, cols = tall_t ? m : n;
  double* A = X;
  if (!tall_t) {
    A = ctx->d4[kW1].d();
    HS_TRY(permute(ctx, mat(fused1(make_sect(m, 0)), fused1(make_sect(n, 0))),
                   mat(fused1(make_sect(n, 0)), fused1(make_sect(m, 0))), {1, 0}, X, A));
  }
  double* U = tall_t ? R : L;  // rows long
  double* V = tall_t ? L : R;  // cols long
  size_t dbytes = 0, hbytes = 0;
  const cusolverStatus_t q = !polar ? CUSOLVER_STATUS_NOT_SUPPORTED :
      cusolverDnXgesvdp_bufferSize(ctx->solver, ctx->params, CUSOLVER_EIG_MODE_VECTOR, 1, rows, cols, CUDA_R_64F, A,
                                   rows, CUDA_R_64F, S, CUDA_R_64F, U, rows, CUDA_R_64F, V, cols, CUDA_R_64F, &dbytes,
                                   &hbytes);
  if (q == CUSOLVER_STATUS_SUCCESS) {
    HS_TRY(ctx->d4[kWork].ensure(std::max<size_t>(dbytes, 8)));
    if (ctx->d4_work_host.size() < hbytes) ctx->d4_work_host.resize(hbytes);
    // the polar path overwrites A; keep X for the fallback
    double* A2 = ctx->d4[kW2].d();
    HS_CUDA(cudaMemcpyAsync(A2, A, (size_t)rows * cols * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double err_sigma = 0.0;
    const cusolverStatus_t st = cusolverDnXgesvdp(
        ctx->solver, ctx->params, CUSOLVER_EIG_MODE_VECTOR, 1, rows, cols, CUDA_R_64F, A2, rows, CUDA_R_64F, S,
        CUDA_R_64F, U, rows, CUDA_R_64F, V, cols, CUDA_R_64F, ctx->d4[kWork].p, dbytes,
        hbytes ? ctx->d4_work_host.data() : nullptr, hbytes, dinfo, &err_sigma);
    int hinfo = 0;
    if (st == CUSOLVER_STATUS_SUCCESS) {
      HS_CUDA(cudaMemcpyAsync(&hinfo, dinfo, sizeof(int), cudaMemcpyDeviceToHost, s));
      HS_CUDA(cudaStreamSynchronize(s));
      if (hinfo == 0 && std::isfinite(err_sigma)) return HS_OK;
    }
    HS_CUDA(cudaMemsetAsync(dinfo, 0, sizeof(int), s));
  }
  int lwork = 0;
  HS_SOLVER(cusolverDnDgesvdj_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, 1, rows, cols, A, rows, S, U, rows,
                                         V, cols, &lwork, ctx->gesvdj));
  HS_TRY(ctx->d4[kWork].ensure((size_t)std::max(lwork, 1) * sizeof(double)));
  HS_SOLVER(cusolverDnDgesvdj(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, 1, rows, cols, A, rows, S, U, rows, V, cols,
                              ctx->d4[kWork].d(), lwork, dinfo, ctx->gesvdj));
  ctx->d4_svd_fallbacks += polar;
  return HS_OK;
}

// Normalise x (n entries) by its largest modulus; the log goes to device slot k of kLog.
hs_status normalise(hs_ctx ctx, double* x, long long n, int k) {
  HS_CUDA(launch_normalize_max_to(x, n, static_cast<unsigned long long*>(ctx->scratch.p) + k,
                                  ctx->d4[kLog].d() + k, ctx->stream));
  ctx->launches += 2;
  return HS_OK;
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" {

hs_status hs_ctmrg4_init(hs_ctx ctx, const hs_z2_tensor* a, int chi_max, hs_env4* env) {
  HS_TRY(check_ctx(ctx));
  if (!a || !env || !a->data) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  for (int k = 0; k < 4; ++k)
    if (!env->C[k] || !env->T[k]) return fail(HS_ERR_INVALID_ARG, "null environment buffer %d", k);
  if (a->dtype != HS_F64) return fail(HS_ERR_UNSUPPORTED, "the directional CTMRG takes real double layers only");
  if (chi_max < 1) return fail(HS_ERR_SHAPE, "chi_max must be positive");
  const int D = a->D, q = D * D;
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
  for (int b = 0; b < 4; ++b) {
    env->chi_even[b] = qs.n[0];
    env->chi_odd[b] = qs.n[1];
  }
  env->basis = a->basis;
  env->moves = 0;
  env->svd = HS_SVD_JACOBI;
  HS_TRY(ensure_workspace(ctx, env->chi_max, q));
  HS_TRY(ctx->scratch.ensure(64 * sizeof(unsigned long long)));
  const Z2Mat Am = mat(fused2(qs, qs), fused2(qs, qs));
  const size_t ab = (size_t)z2_elems(Am) * sizeof(double);
  double* ag = ctx->d4[kY2].d();  // a_g in its own (u, l, d, r) layout, for the traced-boundary init
  for (int g = 0; g < 4; ++g) {
    HS_TRY(ctx->d4[kAq + g].ensure(ab));
    HS_TRY(ctx->d4[kAr + g].ensure(ab));
    HS_TRY(permute(ctx, Am, Am, {mod4(2 - g), mod4(3 - g), mod4(0 - g), mod4(1 - g)}, a->data,
                   ctx->d4[kAq + g].d()));
    HS_TRY(permute(ctx, Am, Am, {mod4(0 - g), mod4(3 - g), mod4(1 - g), mod4(2 - g)}, a->data,
                   ctx->d4[kAr + g].d()));
    HS_TRY(permute(ctx, Am, Am, {mod4(0 - g), mod4(1 - g), mod4(2 - g), mod4(3 - g)}, a->data, ag));
    // frame g: its upper-left corner is C[g], its left edge T[g - 1]
    HS_CUDA(launch_ctmrg_init(ag, D, herm, env->C[g], env->T[mod4(g - 1)], ctx->stream));
    ctx->launches += 1;
  }
  const Z2Mat Cm = mat(fused1(qs), fused1(qs)), Tm = mat(fused2(qs, qs), fused1(qs));
  for (int k = 0; k < 4; ++k) {
    HS_TRY(normalise(ctx, env->C[k], z2_elems(Cm), k));
    HS_TRY(normalise(ctx, env->T[k], z2_elems(Tm), 4 + k));
  }
  double* hlog = static_cast<double*>(ctx->d4_h.p);
  HS_CUDA(cudaMemcpyAsync(hlog, ctx->d4[kLog].p, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  HS_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < 4; ++k) {
    env->log_norm_C[k] = hlog[k];
    env->log_norm_T[k] = hlog[4 + k];
  }
  ctx->d4_src = a->data;
  return HS_OK;
}

hs_status hs_ctmrg4_move(hs_ctx ctx, const hs_z2_tensor* a, hs_env4* env, int chi, int direction,
                         hs_move4_info* info, double* sv_out) {
  HS_TRY(check_ctx(ctx));
  if (!a || !env || !a->data) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (direction < 0 || direction > 3) return fail(HS_ERR_INVALID_ARG, "direction must be 0..3");
  if (chi < 1 || chi > env->chi_max) return fail(HS_ERR_SHAPE, "chi must be in [1, chi_max]");
  if (env->svd != HS_SVD_JACOBI && env->svd != HS_SVD_POLAR) return fail(HS_ERR_INVALID_ARG, "unknown SVD mode");
  if (a->data != ctx->d4_src || a->D != env->D)
    return fail(HS_ERR_INVALID_ARG, "the double layer is not the one given to hs_ctmrg4_init");
  const int f = direction;
  const Sect q = make_sect(env->q_even, env->q_odd);
  const Sect L = bond(env, f - 1), T = bond(env, f), B = bond(env, f - 2);
  cudaStream_t s = ctx->stream;
  Flops fl;

  // the side's two quarters and X = Q1^T Q4^T
  double* Q1 = ctx->d4[kQ1].d();
  double* Q4 = ctx->d4[kQ4].d();
  HS_TRY(quarter(ctx, env, f, q, Q1, fl));
  HS_TRY(quarter(ctx, env, f - 1, q, Q4, fl));
  const Z2Mat Q1m = mat(fused2(L, q), fused2(T, q)), Q1t = mat(fused2(T, q), fused2(L, q));
  const Z2Mat Q4m = mat(fused2(B, q), fused2(L, q)), Q4t = mat(fused2(L, q), fused2(B, q));
  const Z2Mat Xm = mat(fused2(T, q), fused2(B, q));
  HS_TRY(permute(ctx, Q1m, Q1t, {2, 3, 0, 1}, Q1, ctx->d4[kQ1t].d()));
  HS_TRY(permute(ctx, Q4m, Q4t, {2, 3, 0, 1}, Q4, ctx->d4[kQ4t].d()));
  HS_TRY(gemm4(ctx, fl, Q1t, Q4m, Xm, ctx->d4[kQ1t].d(), Q4, ctx->d4[kX].d()));

  // one SVD per parity block, into contiguous columns: Lv the left singular
  // vectors of X_p (over its rows j, m_p long), Rv the right ones (over its
  // columns j', n_p long).
  int m[2], n[2], r[2];
  long long roff[2], loff[2], soff[2];
  for (int p = 0; p < 2; ++p) {
    m[p] = (int)z2_rows(Xm, p);
    n[p] = (int)z2_cols(Xm, p);
    r[p] = std::min(m[p], n[p]);
  }
  roff[0] = loff[0] = soff[0] = 0;
  roff[1] = (long long)n[0] * r[0];
  loff[1] = (long long)m[0] * r[0];
  soff[1] = r[0];
  double* Rv = ctx->d4[kU].d();
  double* Lv = ctx->d4[kV].d();
  double* S = ctx->d4[kS].d();
  int* dinfo = static_cast<int*>(ctx->d4[kInfo].p);
  HS_CUDA(cudaMemsetAsync(dinfo, 0, 2 * sizeof(int), s));
  for (int p = 0; p < 2; ++p)
    if (r[p] > 0)
      HS_TRY(block_svd(ctx, env->svd == HS_SVD_POLAR, ctx->d4[kX].d() + z2_block_off(Xm, p), m[p], n[p],
                       S + soff[p], Lv + loff[p], Rv + roff[p], dinfo + p));
  // singular values and status to the host: the kept sectors fix every shape below
  const int rt = r[0] + r[1];
  if (rt == 0) return fail(HS_ERR_SHAPE, "empty SVD");
  double* hs_ = static_cast<double*>(ctx->d4_h.p);
  int* hinfo = reinterpret_cast<int*>(hs_ + rt);
  HS_CUDA(cudaMemcpyAsync(hs_, S, rt * sizeof(double), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaMemcpyAsync(hinfo, dinfo, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  if (hinfo[0] != 0 || hinfo[1] != 0) return fail(HS_ERR_SOLVER, "SVD info = (%d, %d)", hinfo[0], hinfo[1]);

  // keep the chi largest over both blocks (ties: block 0, then lower index)
  struct Cand {
    double s;
    int b, col;
  };
  std::vector<Cand> cand;
  cand.reserve(rt);
  for (int p = 0; p < 2; ++p)
    for (int c = 0; c < r[p]; ++c) cand.push_back({hs_[soff[p] + c], p, c});
  std::stable_sort(cand.begin(), cand.end(), [](const Cand& x, const Cand& y) { return x.s > y.s; });
  const double smax = cand[0].s;
  if (!(smax > 0.0) || !std::isfinite(smax)) return fail(HS_ERR_NONFINITE, "largest singular value %g", smax);
  int keep = 0;
  while (keep < (int)cand.size() && keep < chi && cand[keep].s > kSvCutoff * smax) ++keep;
  int k[2] = {0, 0};
  std::vector<int> hidx[2];
  std::vector<double> hscale[2];
  for (int i = 0; i < keep; ++i) {
    const Cand& c = cand[i];
    ++k[c.b];
    hidx[c.b].push_back(c.col);
    hscale[c.b].push_back(1.0 / std::sqrt(c.s));
  }
  int* pidx = reinterpret_cast<int*>(hinfo + 4);
  double* pscale = reinterpret_cast<double*>(pidx + 2 * env->chi_max + 2);
  for (int p = 0; p < 2; ++p)
    for (int i = 0; i < k[p]; ++i) {
      pidx[p * env->chi_max + i] = hidx[p][i];
      pscale[p * env->chi_max + i] = hscale[p][i];
    }
  int* didx = static_cast<int*>(ctx->d4[kIdx].p);
  double* dscale = ctx->d4[kScale].d();
  HS_CUDA(cudaMemcpyAsync(didx, pidx, 2 * env->chi_max * sizeof(int), cudaMemcpyHostToDevice, s));
  HS_CUDA(cudaMemcpyAsync(dscale, pscale, 2 * env->chi_max * sizeof(double), cudaMemcpyHostToDevice, s));

  const Sect cn = make_sect(k[0], k[1]);
  // the kept left and right singular vectors as rows, each scaled by s^-1/2:
  // VlT over (T, q), VrT over (B, q)
  const Z2Mat VlT = mat(fused1(cn), fused2(T, q)), VrT = mat(fused1(cn), fused2(B, q));
  double* Vl = ctx->d4[kVl].d();
  double* Vr = ctx->d4[kVr].d();
  for (int p = 0; p < 2; ++p) {
    HS_CUDA(launch_gather_scale_rows(Lv + loff[p], m[p], didx + p * env->chi_max, dscale + p * env->chi_max, k[p],
                                     Vl + z2_block_off(VlT, p), s));
    HS_CUDA(launch_gather_scale_rows(Rv + roff[p], n[p], didx + p * env->chi_max, dscale + p * env->chi_max, k[p],
                                     Vr + z2_block_off(VrT, p), s));
    ctx->launches += (k[p] > 0) * 2;
  }
  // P_a^T = VrT Q4 and P_b^T = VlT Q1^T, both [c | (L, q)]
  const Z2Mat PT = mat(fused1(cn), fused2(L, q));
  double* PaT = ctx->d4[kPa].d();
  double* PbT = ctx->d4[kPb].d();
  HS_TRY(gemm4(ctx, fl, VrT, Q4t, PT, Vr, ctx->d4[kQ4t].d(), PaT));
  HS_TRY(gemm4(ctx, fl, VlT, Q1m, PT, Vl, Q1, PbT));

  double* P1 = ctx->d4[kP1].d();
  double* P2 = ctx->d4[kP2].d();
  double* W1 = ctx->d4[kW1].d();
  double* W2 = ctx->d4[kW2].d();
  double* out0 = ctx->d4[kOut0].d();
  double* out1 = ctx->d4[kOut1].d();
  double* out2 = ctx->d4[kOut2].d();

  // C1 <- P_a^T (C1 T1): Y[(x, e) | b] = T1[g, x, e] C1[b, g], then [e | (b, x)]
  {
    const Z2Mat T1m = mat(fused2(T, q), fused1(T)), T1p = mat(fused2(q, T), fused1(T));
    const Z2Mat C1m = mat(fused1(L), fused1(T));
    const Z2Mat Ym = mat(fused2(q, T), fused1(L)), Yp = mat(fused1(T), fused2(L, q));
    const Z2Mat C1n = mat(fused1(cn), fused1(T));
    HS_TRY(permute(ctx, T1m, T1p, {1, 2, 0}, env->T[f], P2));
    HS_TRY(gemm4(ctx, fl, T1p, C1m, Ym, P2, env->C[f], W1));
    HS_TRY(permute(ctx, Ym, Yp, {1, 2, 0}, W1, W2));
    HS_TRY(gemm4(ctx, fl, PT, Yp, C1n, PaT, W2, out0));
  }
  // T4 <- P_a^T (T4 a) P_b
  {
    const Z2Mat PaTp = mat(fused2(cn, q), fused1(L));
    const Z2Mat T4m = mat(fused2(L, q), fused1(L)), T4p = mat(fused2(q, L), fused1(L));
    const Z2Mat W1m = mat(fused2(cn, q), fused2(q, L)), W1p = mat(fused2(cn, L), fused2(q, q));
    const Z2Mat Ar = mat(fused2(q, q), fused2(q, q));
    const Z2Mat W2m = mat(fused2(cn, L), fused2(q, q)), W2p = mat(fused2(cn, q), fused2(L, q));
    const Z2Mat T4n = mat(fused2(cn, q), fused1(cn));
    double* Y1 = ctx->d4[kY1].d();
    HS_TRY(permute(ctx, PT, PaTp, {0, 2, 1}, PaT, Y1));                   // [(c, d) | alpha]
    HS_TRY(permute(ctx, T4m, T4p, {1, 2, 0}, env->T[mod4(f - 1)], P2));  // [(x, beta) | alpha]
    HS_TRY(gemm4(ctx, fl, PaTp, T4p, W1m, Y1, P2, W1));                   // [(c, d) | (x, beta)]
    HS_TRY(permute(ctx, W1m, W1p, {0, 3, 2, 1}, W1, W2));                 // [(c, beta) | (x, d)]
    HS_TRY(gemm4(ctx, fl, W1p, Ar, W2m, W2, ctx->d4[kAr + f].d(), W1));  // [(c, beta) | (u, r)]
    HS_TRY(permute(ctx, W2m, W2p, {0, 3, 1, 2}, W1, W2));                 // [(c, r) | (beta, u)]
    HS_TRY(gemm4(ctx, fl, W2p, PT, T4n, W2, PbT, out1));                  // [(c, r) | k]
  }
  // C4 <- (T3 C4) P_b
  {
    const Z2Mat C4m = mat(fused1(B), fused1(L)), C4t = mat(fused1(L), fused1(B));
    const Z2Mat T3m = mat(fused2(B, q), fused1(B));
    const Z2Mat Vm = mat(fused2(B, q), fused1(L)), Vp = mat(fused1(B), fused2(L, q));
    const Z2Mat C4n = mat(fused1(B), fused1(cn));
    HS_TRY(permute(ctx, C4m, C4t, {1, 0}, env->C[mod4(f - 1)], P1));
    HS_TRY(gemm4(ctx, fl, T3m, C4t, Vm, env->T[mod4(f - 2)], P1, W1));   // [(alpha, x) | g]
    HS_TRY(permute(ctx, Vm, Vp, {0, 2, 1}, W1, W2));                      // [alpha | (g, x)]
    HS_TRY(gemm4(ctx, fl, Vp, PT, C4n, W2, PbT, out2));                   // [alpha | k]
  }
  // normalise and store
  const long long n0 = (long long)cn.n[0] * T.n[0] + (long long)cn.n[1] * T.n[1];
  const long long n1 = z2_elems(mat(fused2(cn, q), fused1(cn)));
  const long long n2 = (long long)B.n[0] * cn.n[0] + (long long)B.n[1] * cn.n[1];
  HS_TRY(normalise(ctx, out0, n0, 0));
  HS_TRY(normalise(ctx, out1, n1, 1));
  HS_TRY(normalise(ctx, out2, n2, 2));
  HS_CUDA(cudaMemcpyAsync(env->C[f], out0, n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  HS_CUDA(cudaMemcpyAsync(env->T[mod4(f - 1)], out1, n1 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  HS_CUDA(cudaMemcpyAsync(env->C[mod4(f - 1)], out2, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double* hlog = pscale + 2 * env->chi_max;
  HS_CUDA(cudaMemcpyAsync(hlog, ctx->d4[kLog].p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  if (!std::isfinite(hlog[0]) || !std::isfinite(hlog[1]) || !std::isfinite(hlog[2]))
    return fail(HS_ERR_NONFINITE, "environment is not finite after the move");
  env->log_norm_C[f] = hlog[0];
  env->log_norm_T[mod4(f - 1)] = hlog[1];
  env->log_norm_C[mod4(f - 1)] = hlog[2];
  env->chi_even[mod4(f - 1)] = k[0];
  env->chi_odd[mod4(f - 1)] = k[1];
  env->moves += 1;
  if (info) {
    info->direction = f;
    info->chi_even = k[0];
    info->chi_odd = k[1];
    info->m_even = m[0];
    info->m_odd = m[1];
    info->n_even = n[0];
    info->n_odd = n[1];
    info->s_max = smax;
    info->s_cut = cand[keep - 1].s;
    info->s_next = keep < (int)cand.size() ? cand[keep].s : 0.0;
    info->gap = keep < (int)cand.size() ? (info->s_cut - info->s_next) / smax : INFINITY;
    info->gemm_flops = fl.f;
  }
  if (sv_out)
    for (int i = 0; i < keep; ++i) sv_out[i] = cand[i].s / smax;
  return HS_OK;
}

hs_status hs_env4_to_dense(hs_ctx ctx, const hs_env4* env, double* const* C_dense, double* const* T_dense) {
  HS_TRY(check_ctx(ctx));
  if (!env || !C_dense || !T_dense) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  for (int k = 0; k < 4; ++k)
    if (!C_dense[k] || !T_dense[k] || !env->C[k] || !env->T[k]) return fail(HS_ERR_INVALID_ARG, "null buffer");
  const bool herm = env->basis == HS_BASIS_HERMITIAN;
  HS_TRY(ctx->d4[kOut0].ensure((size_t)env->chi_max * env->chi_max * sizeof(double)));
  for (int k = 0; k < 4; ++k) {
    const Sect in = bond(env, k - 1), out = bond(env, k);
    hs_launch(corner_dense_kernel, grid_of((long long)(in.n[0] + in.n[1]) * (out.n[0] + out.n[1])), 256, 0,
              ctx->stream, env->C[k], in.n[0], in.n[1], out.n[0], out.n[1], C_dense[k]);
    HS_CUDA(cudaGetLastError());
    // the edge through the C4v converter; its corner part (read from the
    // edge's own buffer, at least chi^2 entries long) goes to scratch
    const Sect e = bond(env, k);
    HS_CUDA(launch_env_to_dense(env->T[k], env->T[k], env->D, e.n[0], e.n[1], herm, ctx->d4[kOut0].d(), T_dense[k],
                                ctx->stream));
  }
  return HS_OK;
}

}  // extern "C"

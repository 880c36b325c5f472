// C ABI of libhs (include/hs.h): context, workspace, the C4v CTMRG move of
// arXiv 2410.11596 (Sec. II.A, Fig. 1(d)) in the Hermitian Z2 basis
// (Sec. II.B).
#include <algorithm>
#include <utility>

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

Z2Mat mat(Fused r, Fused c, int pad) {
  Z2Mat m;
  m.r = r;
  m.c = c;
  m.pad = pad;
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
  HS_TRY(ctx->splitk.ensure(kSplitKElems * sizeof(double)));
  HS_CUDA(launch_gemm_f64(g, A, B, C, 1.0, ctx->stream, ctx->splitk.d(), kSplitKElems));
  if (g.n > 0) ctx->launches += 1;
  return HS_OK;
}

// make_perm_plan through the context's cache, keyed by the two layouts and
// the permutation.
const PermPlan& cached_plan(hs_ctx ctx, const Z2Mat& in, const Z2Mat& out, const int* perm) {
  int key[2 * (2 + 2 * 2 * kMaxFused) + 2 + kMaxLegs];
  int k = 0;
  for (const Z2Mat* m : {&in, &out}) {
    for (const Fused* f : {&m->r, &m->c}) {
      key[k++] = f->k;
      for (int j = 0; j < kMaxFused; ++j) {
        key[k++] = j < f->k ? f->leg[j].n[0] : 0;
        key[k++] = j < f->k ? f->leg[j].n[1] : 0;
      }
    }
    key[k++] = m->pad;
  }
  for (int j = 0; j < kMaxLegs; ++j) key[k++] = perm[j];
  std::string ks(reinterpret_cast<const char*>(key), k * sizeof(int));
  auto it = ctx->plan_cache.find(ks);
  if (it != ctx->plan_cache.end()) return it->second;
  if (ctx->plan_cache.size() > 4096) ctx->plan_cache.clear();  // bound the cache
  return ctx->plan_cache.emplace(std::move(ks), make_perm_plan(in, out, perm)).first->second;
}

hs_status permute(hs_ctx ctx, const Z2Mat& in, const Z2Mat& out, std::initializer_list<int> perm,
                  const double* src, double* dst) {
  int p[kMaxLegs] = {0};
  int i = 0;
  for (int v : perm) p[i++] = v;
  const PermPlan& plan = cached_plan(ctx, in, out, p);
  HS_CUDA(launch_permute_f64(plan, src, dst, 1.0, ctx->stream));
  if (plan.nbox > 0) ctx->launches += 1;
  return HS_OK;
}

namespace {
int take_event(hs_ctx c) {
  if (c->next_event >= (int)c->events.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    c->events.push_back(e);
  }
  return c->next_event++;
}
}  // namespace

PhaseScope::PhaseScope(hs_ctx c, int phase) : c_(c), phase_(phase), e0_(-1) {
  if (!c_->prof || !((c_->prof_mask >> phase) & 1u)) return;
  e0_ = take_event(c_);
  if (e0_ >= 0) cudaEventRecord(c_->events[e0_], c_->stream);
}

PhaseScope::~PhaseScope() {
  if (!c_->prof || e0_ < 0) return;
  const int e1 = take_event(c_);
  if (e1 < 0) return;
  cudaEventRecord(c_->events[e1], c_->stream);
  c_->recs.push_back({phase_, e0_, e1});
}

void harvest_profile(hs_ctx ctx) {
  for (const auto& r : ctx->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->events[r.e0], ctx->events[r.e1]) == cudaSuccess)
      ctx->phase_ms[r.phase] += ms;
  }
  cudaGetLastError();
  ctx->recs.clear();
  ctx->next_event = 0;
}

int tc_pad(hs_precision p) { return p == HS_PREC_BF16X3 ? 64 : 32; }
int tc_elem_bytes(hs_precision p) { return p == HS_PREC_BF16X3 ? 2 : 4; }
int tc_mode(hs_precision p) { return p == HS_PREC_BF16X3 ? 2 : 1; }

namespace {

size_t a_elems(int D, hs_basis b) {
  const Sect q = q_sect(D, b);
  return (size_t)z2_elems(mat(fused2(q, q), fused2(q, q)));
}

// One cuSOLVER handle with its stream-bound workspaces.
struct Solver {
  cusolverDnHandle_t h;
  cusolverDnParams_t prm;
  DBuf* dev;
  std::vector<char>* host;
};

Solver solver_of(hs_ctx ctx, int which, bool f32) {
  if (which == 0) return {ctx->solver, ctx->params, f32 ? &ctx->solver32_dev : &ctx->solver_dev,
                          f32 ? &ctx->solver32_host : &ctx->solver_host};
  return {ctx->solver2, ctx->params2, f32 ? &ctx->solver2_32_dev : &ctx->solver2_dev,
          f32 ? &ctx->solver2_32_host : &ctx->solver2_host};
}

hs_status eig_ws(const Solver& sv, int nmax, bool f32) {
  size_t dev = 0, host = 0;
  const cudaDataType t = f32 ? CUDA_R_32F : CUDA_R_64F;
  HS_SOLVER(cusolverDnXsyevd_bufferSize(sv.h, sv.prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, nmax, t,
                                        nullptr, nmax, t, nullptr, t, &dev, &host));
  HS_TRY(sv.dev->ensure(dev + 256));
  if (sv.host->size() < host + 1) sv.host->resize(host + 1);
  return HS_OK;
}

hs_status eig_workspace_impl(hs_ctx ctx, int nmax) {
  HS_TRY(eig_ws(solver_of(ctx, 0, false), nmax, false));
  return eig_ws(solver_of(ctx, 1, false), nmax, false);
}

hs_status eig32_workspace(hs_ctx ctx, int nmax) {
  HS_TRY(eig_ws(solver_of(ctx, 0, true), nmax, true));
  return eig_ws(solver_of(ctx, 1, true), nmax, true);
}

// In-place symmetric eigen-decomposition (vectors) of one n x n block on
// solver `which`; FP32 when f32, else FP64.
hs_status eig_any(hs_ctx ctx, int which, bool f32, void* A, int n, void* w, int slot) {
  if (n == 0) return HS_OK;
  const Solver sv = solver_of(ctx, which, f32);
  const cudaDataType t = f32 ? CUDA_R_32F : CUDA_R_64F;
  HS_SOLVER(cusolverDnXsyevd(sv.h, sv.prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, t, A, n, t, w, t,
                             sv.dev->p, sv.dev->bytes, sv.host->data(), sv.host->size(),
                             static_cast<int*>(ctx->info.p) + slot));
  return HS_OK;
}

// Both parity blocks: block 0 on the context stream, block 1 on the second
// stream from a helper thread (cuSOLVER's syevd blocks its calling thread).
hs_status eig_pair_impl(hs_ctx ctx, bool f32, void* A0, int n0, void* w0, void* A1, int n1, void* w1) {
  if (n0 == 0 || n1 == 0) {
    HS_TRY(eig_any(ctx, 0, f32, A0, n0, w0, 0));
    return eig_any(ctx, 0, f32, A1, n1, w1, 1);
  }
  HS_CUDA(cudaEventRecord(ctx->ev_fork, ctx->stream));
  HS_CUDA(cudaStreamWaitEvent(ctx->stream2, ctx->ev_fork, 0));
  hs_status st1 = HS_OK;
  std::string err1;
  std::thread th([&] {
    cudaSetDevice(ctx->device);
    st1 = eig_any(ctx, 1, f32, A1, n1, w1, 1);
    if (st1 != HS_OK) err1 = last_error();
  });
  const hs_status st0 = eig_any(ctx, 0, f32, A0, n0, w0, 0);
  th.join();
  HS_CUDA(cudaEventRecord(ctx->ev_join, ctx->stream2));
  HS_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  if (st0 != HS_OK) return st0;
  if (st1 != HS_OK) return fail(st1, "%s", err1.c_str());
  return HS_OK;
}

}  // namespace

hs_status eig_pair(hs_ctx ctx, bool f32, void* A0, int n0, void* w0, void* A1, int n1, void* w1) {
  return eig_pair_impl(ctx, f32, A0, n0, w0, A1, n1, w1);
}
hs_status eig_single(hs_ctx ctx, bool f32, void* A, int n, void* w) { return eig_any(ctx, 0, f32, A, n, w, 0); }
hs_status eig_workspace32(hs_ctx ctx, int nmax) { return eig32_workspace(ctx, nmax); }
hs_status eig_workspace(hs_ctx ctx, int nmax) { return eig_workspace_impl(ctx, nmax); }

// Write the operand `layout` (legs = src legs permuted by perm) of a
// tensor-core GEMM as split, K-padded hi/lo arrays.
hs_status tc_split_any(hs_ctx ctx, hs_precision prec, const Z2Mat& src_layout, const Z2Mat& layout,
                       std::initializer_list<int> perm, const void* src, bool src_f32, DBuf& hi, DBuf& lo);

hs_status tc_split(hs_ctx ctx, hs_precision prec, const Z2Mat& src_layout, const Z2Mat& layout,
                   std::initializer_list<int> perm, const double* src, DBuf& hi, DBuf& lo) {
  return tc_split_any(ctx, prec, src_layout, layout, perm, src, false, hi, lo);
}

// As tc_split, from an FP32 source (an FP32 tensor-core GEMM output).
hs_status tc_split_f32(hs_ctx ctx, hs_precision prec, const Z2Mat& src_layout, const Z2Mat& layout,
                       std::initializer_list<int> perm, const float* src, DBuf& hi, DBuf& lo) {
  return tc_split_any(ctx, prec, src_layout, layout, perm, src, true, hi, lo);
}

// Sizes the split buffers of the padded operand layout P and zeroes their K
// padding unless the last split into them had the same layout (a split
// writes every entry of the layout but none of the padding).
hs_status split_dest(hs_ctx ctx, hs_precision prec, const Z2Mat& P, DBuf& hi, DBuf& lo) {
  const int eb = tc_elem_bytes(prec);
  const size_t nb = (size_t)z2_elems(P) * eb;
  HS_TRY(hi.ensure(nb));
  HS_TRY(lo.ensure(nb));
  unsigned long long key = 0x9E3779B97F4A7C15ull ^ (unsigned long long)eb;
  for (int p = 0; p < 2; ++p)
    for (long long v : {z2_rows(P, p), z2_cols(P, p), z2_ld(P, p)})
      key = (key ^ (unsigned long long)v) * 0x100000001B3ull;
  key |= 1;
  if (hi.zkey != key || lo.zkey != key) {
    // only the K padding of each block row (the rest is written below)
    for (int p = 0; p < 2; ++p) {
      const long long rows = z2_rows(P, p), cols = z2_cols(P, p), ld = z2_ld(P, p);
      if (rows == 0 || ld == cols) continue;
      const size_t off = (size_t)(z2_block_off(P, p) + cols) * eb;
      for (DBuf* b : {&hi, &lo})
        HS_CUDA(cudaMemset2DAsync(static_cast<char*>(b->p) + off, (size_t)ld * eb, 0, (size_t)(ld - cols) * eb,
                                  (size_t)rows, ctx->stream));
    }
    hi.zkey = lo.zkey = key;
  }
  return HS_OK;
}

hs_status tc_split_any(hs_ctx ctx, hs_precision prec, const Z2Mat& src_layout, const Z2Mat& layout,
                       std::initializer_list<int> perm, const void* src, bool src_f32, DBuf& hi, DBuf& lo) {
  const Z2Mat P = mat(layout.r, layout.c, tc_pad(prec));
  PhaseScope ps(ctx, HS_PHASE_PERMUTE);
  HS_TRY(split_dest(ctx, prec, P, hi, lo));
  int pm[kMaxLegs] = {0}, i = 0;
  for (int v : perm) pm[i++] = v;
  const PermPlan& plan = cached_plan(ctx, src_layout, P, pm);
  if (src_f32)
    HS_CUDA(launch_permute_split_f32(plan, static_cast<const float*>(src), hi.p, lo.p, tc_mode(prec), ctx->stream));
  else
    HS_CUDA(launch_permute_split(plan, static_cast<const double*>(src), hi.p, lo.p, tc_mode(prec), ctx->stream));
  if (plan.nbox > 0) ctx->launches += 1;
  return HS_OK;
}

// C[R|N] = A[R|K] B[N|K]^T on the tensor cores from split operands (logical
// layouts A, B; buffers padded as written by tc_split), FP64 C in layout Cm.
hs_status tc_run(hs_ctx ctx, hs_precision prec, const Z2Mat& A, const DBuf& ahi, const DBuf& alo,
                 const Z2Mat& B, const DBuf& bhi, const DBuf& blo, const Z2Mat& Cm, double* C, bool out_f32) {
  const int pad = tc_pad(prec), eb = tc_elem_bytes(prec);
  const size_t ce = out_f32 ? sizeof(float) : sizeof(double);
  char* Cb = reinterpret_cast<char*>(C);
  const Z2Mat Ap = mat(A.r, A.c, pad), Bp = mat(B.r, B.c, pad);
  TcProblem pr[2];
  int n = 0;
  for (int p = 0; p < 2; ++p) {
    TcProblem& t = pr[n];
    t.M = (int)z2_rows(Ap, p);
    t.N = (int)z2_rows(Bp, p);
    t.Kp = (int)z2_ld(Ap, p);
    if (t.M == 0 || t.N == 0) continue;
    if (z2_cols(Ap, p) == 0) {  // empty contraction: the block is zero
      HS_CUDA(cudaMemset2DAsync(Cb + z2_block_off(Cm, p) * ce, ce * z2_ld(Cm, p), 0, ce * t.N, t.M, ctx->stream));
      continue;
    }
    t.ldc = (int)z2_ld(Cm, p);
    t.a_hi = static_cast<const char*>(ahi.p) + z2_block_off(Ap, p) * eb;
    t.a_lo = static_cast<const char*>(alo.p) + z2_block_off(Ap, p) * eb;
    t.b_hi = static_cast<const char*>(bhi.p) + z2_block_off(Bp, p) * eb;
    t.b_lo = static_cast<const char*>(blo.p) + z2_block_off(Bp, p) * eb;
    t.c = reinterpret_cast<double*>(Cb + z2_block_off(Cm, p) * ce);
    t.out_f32 = out_f32 ? 1 : 0;
    ++n;
  }
  HS_TRY(ctx->splitk.ensure(kSplitKElems * sizeof(double)));
  PhaseScope ps(ctx, HS_PHASE_GEMM_TC);
  HS_CUDA(launch_gemm_tc(prec, pr, n, static_cast<int*>(ctx->tc_err.p), ctx->stream, ctx->splitk.d(), kSplitKElems));
  if (n > 0) ctx->launches += 1;
  return HS_OK;
}

// Destination map of a GEMM output block of parity p (layout Cm: two-leg
// rows L0 L1, two-leg columns L2 L3) written as the padded split operand P,
// whose legs are Cm's permuted by perm. False when the epilogue cannot write
// it (other leg counts, a destination whose innermost leg is neither L1 nor
// L3, offsets beyond 32 bits).
bool make_ps_desc(const Z2Mat& Cm, const Z2Mat& P, const int perm[4], int p, void* hi, void* lo, PsDesc& d) {
  if (Cm.r.k != 2 || Cm.c.k != 2 || P.r.k != 2 || P.c.k != 2) return false;
  if (perm[3] != 1 && perm[3] != 3) return false;
  if (z2_elems(P) >= (1ll << 31)) return false;
  const Sect L[4] = {Cm.r.leg[0], Cm.r.leg[1], Cm.c.leg[0], Cm.c.leg[1]};
  // the destination's legs must be the source's permuted
  const Sect Dl[4] = {P.r.leg[0], P.r.leg[1], P.c.leg[0], P.c.leg[1]};
  for (int k = 0; k < 4; ++k)
    if (Dl[k].n[0] != L[perm[k]].n[0] || Dl[k].n[1] != L[perm[k]].n[1]) return false;
  memset(&d, 0, sizeof d);
  d.hi = hi;
  d.lo = lo;
  d.limit = (int)z2_elems(P);
  d.mode = perm[3] == 1 ? 1 : 2;
  int rt[2], ct[2], nr = 0, nc = 0;
  for (int t = 0; t < 4; ++t)
    if (tuple_parity(t) == p) rt[nr++] = ct[nc++] = t;
  d.rsplit = (int)tuple_size(Cm.r, rt[0]);
  d.csplit = (int)tuple_size(Cm.c, ct[0]);
  for (int a = 0; a < 2; ++a) {
    const int nri = L[1].n[tuple_bit(rt[a], 2, 1)], nci = L[3].n[tuple_bit(ct[a], 2, 1)];
    d.rin[a] = nri > 0 ? nri : 1;
    d.cin[a] = nci > 0 ? nci : 1;
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int par[4] = {tuple_bit(rt[a], 2, 0), tuple_bit(rt[a], 2, 1), tuple_bit(ct[b], 2, 0),
                          tuple_bit(ct[b], 2, 1)};
      const int tr = (par[perm[0]] << 1) | par[perm[1]], tc = (par[perm[2]] << 1) | par[perm[3]];
      const int q = tuple_parity(tr);
      const long long ld = z2_ld(P, q);
      const long long base = z2_block_off(P, q) + tuple_offset(P.r, tr) * ld + tuple_offset(P.c, tc);
      long long co[4];
      co[perm[0]] = (long long)L[perm[1]].n[par[perm[1]]] * ld;
      co[perm[1]] = ld;
      co[perm[2]] = L[perm[3]].n[par[perm[3]]];
      co[perm[3]] = 1;
      d.base[a][b] = (int)base;
      for (int k = 0; k < 4; ++k) d.co[a][b][k] = (int)co[k];
    }
  return true;
}

// As tc_run, with the output (layout Cm) written straight as the split
// operand `layout` (Cm's legs permuted by perm) into hi/lo by the GEMM's
// epilogue. Where the epilogue cannot (BF16 split, an empty contraction,
// unsupported leg order) the output goes through the FP32 buffer tmp and
// the permute/split kernel instead.
hs_status tc_run_split(hs_ctx ctx, hs_precision prec, const Z2Mat& A, const DBuf& ahi, const DBuf& alo,
                       const Z2Mat& B, const DBuf& bhi, const DBuf& blo, const Z2Mat& Cm, const Z2Mat& layout,
                       std::initializer_list<int> perm, DBuf& hi, DBuf& lo, float* tmp) {
  const int pad = tc_pad(prec), eb = tc_elem_bytes(prec);
  const Z2Mat Ap = mat(A.r, A.c, pad), Bp = mat(B.r, B.c, pad), P = mat(layout.r, layout.c, pad);
  int pm[4] = {0, 0, 0, 0}, i = 0;
  for (int v : perm) {
    if (i < 4) pm[i] = v;
    ++i;
  }
  bool fused = eb == 4 && i == 4;
  for (int p = 0; p < 2 && fused; ++p)
    if (z2_rows(Ap, p) > 0 && z2_rows(Bp, p) > 0 && z2_cols(Ap, p) == 0) fused = false;
  PsDesc desc[2];
  TcProblem pr[2];
  int n = 0;
  if (fused) {
    HS_TRY(split_dest(ctx, prec, P, hi, lo));
    for (int p = 0; p < 2 && fused; ++p) {
      TcProblem& t = pr[n];
      t.M = (int)z2_rows(Ap, p);
      t.N = (int)z2_rows(Bp, p);
      t.Kp = (int)z2_ld(Ap, p);
      if (t.M == 0 || t.N == 0) continue;
      if (!make_ps_desc(Cm, P, pm, p, hi.p, lo.p, desc[n])) {
        fused = false;
        break;
      }
      t.ldc = t.N;
      t.a_hi = static_cast<const char*>(ahi.p) + z2_block_off(Ap, p) * eb;
      t.a_lo = static_cast<const char*>(alo.p) + z2_block_off(Ap, p) * eb;
      t.b_hi = static_cast<const char*>(bhi.p) + z2_block_off(Bp, p) * eb;
      t.b_lo = static_cast<const char*>(blo.p) + z2_block_off(Bp, p) * eb;
      t.c = nullptr;
      t.ps = &desc[n];
      ++n;
    }
  }
  if (!fused) {
    HS_TRY(tc_run(ctx, prec, A, ahi, alo, B, bhi, blo, Cm, reinterpret_cast<double*>(tmp), true));
    return tc_split_any(ctx, prec, Cm, layout, perm, tmp, true, hi, lo);
  }
  for (int p = 0; p < 2; ++p)
    ctx->phase_flops[HS_PHASE_GEMM_TC_SPLIT] += 2.0 * z2_rows(A, p) * (double)z2_rows(B, p) * z2_cols(A, p);
  PhaseScope ps(ctx, HS_PHASE_GEMM_TC);
  PhaseScope ps2(ctx, HS_PHASE_GEMM_TC_SPLIT);
  HS_CUDA(launch_gemm_tc(prec, pr, n, static_cast<int*>(ctx->tc_err.p), ctx->stream, nullptr, 0));
  if (n > 0) ctx->launches += 1;
  return HS_OK;
}

// C[R|N] = X[R|K] a[N|K]^T with X written from `src` (layout Xsrc) by `perm`
// and a the split copy of the double layer made by hs_ctmrg_init.
hs_status tc_a_gemm(hs_ctx ctx, hs_precision prec, const Z2Mat& Xsrc, const Z2Mat& X,
                    std::initializer_list<int> perm, const double* src, const Z2Mat& Am, const Z2Mat& Cm,
                    double* C, bool f32 = false) {
  HS_TRY(tc_split_any(ctx, prec, Xsrc, X, perm, src, f32, ctx->tc_x_hi, ctx->tc_x_lo));
  return tc_run(ctx, prec, X, ctx->tc_x_hi, ctx->tc_x_lo, Am, ctx->tc_a_hi, ctx->tc_a_lo, Cm, C, f32);
}

// A dense r x c matrix as a one-block Z2 layout.
Z2Mat dense2(long long r, long long c) { return mat(fused1(make_sect((int)r, 0)), fused1(make_sect((int)c, 0))); }

// Canonical sign, FP64 re-orthonormalisation and projection of the kept rows
// PT (already gathered): the largest entry of each row is made positive,
// `lowdin` Loewdin steps PT <- (3/2 I - 1/2 PT PT^T) PT in FP64 (each step
// squares the departure from orthonormality: 1e-6 -> 1e-12 -> rounding), then
// the new corner is the projection C = PT C' PT^T of each block (FP64, or on
// the tensor cores in the TF32/BF16 precisions), normalised by its largest entry.
hs_status finish_projector(hs_ctx ctx, int n0, int n1, SelectOut* dsel, Sect c, Sect q, Sect cn, const double* C0,
                           const double* C1, hs_env* env, double* flops, int lowdin, bool canonical_sign = true) {
  cudaStream_t s = ctx->stream;
  const int k[2] = {cn.n[0], cn.n[1]};
  const int n[2] = {n0, n1};
  const double* Cp[2] = {C0, C1};
  const long long npt = (long long)k[0] * n[0] + (long long)k[1] * n[1];
  HS_TRY(ctx->pcol.ensure(npt * sizeof(double)));
  HS_TRY(ctx->pt2.ensure(npt * sizeof(double)));
  HS_TRY(ctx->wproj.ensure(npt * sizeof(double)));
  HS_TRY(ctx->gram.ensure(((long long)k[0] * k[0] + (long long)k[1] * k[1] + 1) * sizeof(double)));
  HS_TRY(ctx->splitk.ensure(kSplitKElems * sizeof(double)));
  double* PT = ctx->pt.d();
  double* PT2 = ctx->pt2.d();
  double* P = ctx->pcol.d();
  double* G = ctx->gram.d();
  double* W = ctx->wproj.d();
  const long long ptoff[2] = {0, (long long)k[0] * n[0]};
  const long long goff[2] = {0, (long long)k[0] * k[0]};
  auto group = [&](auto fill) {
    GemmGroup g{};
    for (int p = 0; p < 2; ++p) {
      if (k[p] == 0 || n[p] == 0) continue;
      g.p[g.n++] = fill(p);
    }
    return g;
  };
  const Z2Mat PTm = mat(fused1(cn), fused2(c, q)), Pm = mat(fused2(c, q), fused1(cn));
  {
    PhaseScope ps(ctx, HS_PHASE_SELECT);
    if (canonical_sign) {
      HS_CUDA(launch_row_sign_pair(PT, k[0], n[0], k[1], n[1], s));
      ctx->launches += 1;
    }
    HS_TRY(permute(ctx, PTm, Pm, {1, 2, 0}, PT, P));
    ctx->launches += 1;
  }
  if (env->precision != HS_PREC_F64) {
    // tensor-core precisions: the projection below runs on tcgen05 with FP32
    // accumulation, so orthonormality beyond that level buys nothing; the
    // Loewdin steps run on the tensor cores too (both blocks per launch)
    HS_TRY(lowdin_rows_pair(ctx, env->precision, PT, k, n, PT2, lowdin));
    lowdin = 0;
  }
  for (int step = 0; step < lowdin; ++step) {
    PhaseScope ps(ctx, HS_PHASE_GEMM);
    // G = PT PT^T
    GemmGroup gg = group([&](int p) {
      return GemmProblem{k[p], k[p], n[p], n[p], n[p], k[p], ptoff[p], ptoff[p], goff[p]};
    });
    HS_CUDA(launch_gemm_f64(gg, PT, PT, G, 1.0, s, ctx->splitk.d(), kSplitKElems));
    HS_CUDA(launch_lowdin(G, k[0], k[1], s));
    // PT2 = M PT, i.e. C = M (P)^T with P the column layout
    GemmGroup gm = group([&](int p) {
      return GemmProblem{k[p], n[p], k[p], k[p], k[p], n[p], goff[p], ptoff[p], ptoff[p]};
    });
    HS_CUDA(launch_gemm_f64(gm, G, P, PT2, 1.0, s, ctx->splitk.d(), kSplitKElems));
    *flops += gemm_flops(gg) + gemm_flops(gm);
    ctx->phase_flops[HS_PHASE_GEMM] += gemm_flops(gg) + gemm_flops(gm);
    HS_TRY(permute(ctx, PTm, Pm, {1, 2, 0}, PT2, P));  // columns of the updated vectors
    HS_CUDA(cudaMemcpyAsync(PT, PT2, npt * sizeof(double), cudaMemcpyDeviceToDevice, s));
    ctx->launches += 3;
  }
  // W = PT C' (C' symmetric), C_new = W PT^T, block by block into env->C.
  // With tensor-core precisions both products run on tcgen05 (C' split once
  // per move, PT and W split here); otherwise both run on the FP64 kernel.
  const hs_precision prec = env->precision;
  if (prec == HS_PREC_F64) {
    PhaseScope ps(ctx, HS_PHASE_GEMM);
    GemmGroup gw = group([&](int p) {
      return GemmProblem{k[p], n[p], n[p], n[p], n[p], n[p], ptoff[p], (long long)(Cp[p] - C0), ptoff[p]};
    });
    GemmGroup gc = group([&](int p) {
      return GemmProblem{k[p], k[p], n[p], n[p], n[p], k[p], ptoff[p], ptoff[p], goff[p]};
    });
    HS_CUDA(launch_gemm_f64(gw, PT, C0, W, 1.0, s, ctx->splitk.d(), kSplitKElems));
    HS_CUDA(launch_gemm_f64(gc, W, PT, env->C, 1.0, s, ctx->splitk.d(), kSplitKElems));
    *flops += gemm_flops(gw) + gemm_flops(gc);
    ctx->phase_flops[HS_PHASE_GEMM] += gemm_flops(gw) + gemm_flops(gc);
  } else {
    // both blocks per launch: W = PT C' (C' split once per move), C_new = W PT^T
    if (!ctx->sH_fresh || ctx->sH_n[0] != n[0] || ctx->sH_n[1] != n[1]) {
      const size_t es = ctx->cp_f32 ? sizeof(float) : sizeof(double);
      if (reinterpret_cast<const char*>(Cp[1]) != reinterpret_cast<const char*>(Cp[0]) + (size_t)n[0] * n[0] * es)
        return fail(HS_ERR_INVALID_ARG, "corner blocks not stacked");
      HS_TRY(split_corner(ctx, prec, Cp[0], n[0], n[1]));
    }
    const Z2Mat PL = zd(k[0], k[1], n[0], n[1]), HL = zd(n[0], n[1], n[0], n[1]), CL = zd(k[0], k[1], k[0], k[1]);
    HS_TRY(tc_split(ctx, prec, PL, PL, {0, 1}, PT, ctx->sx_hi, ctx->sx_lo));
    HS_TRY(tc_run(ctx, prec, PL, ctx->sx_hi, ctx->sx_lo, HL, ctx->sH_hi, ctx->sH_lo, PL, W));
    HS_TRY(tc_split(ctx, prec, PL, PL, {0, 1}, W, ctx->sy_hi, ctx->sy_lo));
    HS_TRY(tc_run(ctx, prec, PL, ctx->sy_hi, ctx->sy_lo, PL, ctx->sx_hi, ctx->sx_lo, CL, env->C));
    for (int p = 0; p < 2; ++p) {
      const double f = 2.0 * k[p] * (double)n[p] * n[p] + 2.0 * k[p] * (double)k[p] * n[p];
      *flops += f;
      ctx->phase_flops[HS_PHASE_GEMM_TC] += f;
    }
  }
  HS_CUDA(launch_normalize_max_to(env->C, goff[1] + (long long)k[1] * k[1],
                                  static_cast<unsigned long long*>(ctx->scratch.p) + 2, &dsel->log_norm_C, s));
  ctx->launches += 4;
  return HS_OK;
}

// Order the kept rows PT of this move (k_b rows of length n_b per block,
// stacked) like the previous move's: the new boundary states are a gauge
// choice, and the warm start of the next move's subspace iteration is only
// valid when that choice is stationary. Kept states come ordered by |lambda|;
// where two of them have nearly equal |lambda| (D = 7: the spectrum drifts by
// ~0.5% per move and close pairs change order) the order, and with it the
// coordinates of the next C', changes from move to move. Here, per block,
// the new rows in order of their clearest overlap each take the position of
// the previous row they overlap most (|O_ij|, O = PT PT_prev^T, FP64), with
// that row's sign, when the overlap is above 1/2 and the position is still
// free; the other rows fill the free positions in their order. *moved: rows
// that moved or changed sign.
hs_status align_kept_rows(hs_ctx ctx, const int k[2], const int n[2], int* moved) {
  cudaStream_t s = ctx->stream;
  *moved = 0;
  const long long off1 = (long long)k[0] * n[0];
  const long long npt = off1 + (long long)k[1] * n[1];
  const long long no = (long long)k[0] * k[0] + (long long)k[1] * k[1];
  HS_TRY(ctx->ovl.ensure((size_t)(no + 1) * sizeof(double)));
  HS_TRY(ctx->ovl_idx.ensure((size_t)(k[0] + k[1] + 1) * sizeof(int)));
  HS_TRY(ctx->pt_tmp.ensure((size_t)(npt + 1) * sizeof(double)));
  HS_TRY(ctx->h_ovl.ensure((size_t)(no + 1) * sizeof(double) + (size_t)(k[0] + k[1] + 1) * (sizeof(int) + sizeof(double))));
  HS_TRY(ctx->splitk.ensure(kSplitKElems * sizeof(double)));
  const long long poff[2] = {0, off1}, ooff[2] = {0, (long long)k[0] * k[0]};
  GemmGroup g{};
  for (int b = 0; b < 2; ++b)
    if (k[b] > 0) g.p[g.n++] = GemmProblem{k[b], k[b], n[b], n[b], n[b], k[b], poff[b], poff[b], ooff[b]};
  HS_CUDA(launch_gemm_f64(g, ctx->pt.d(), ctx->pt_prev.d(), ctx->ovl.d(), 1.0, s, ctx->splitk.d(), kSplitKElems));
  ctx->launches += 1;
  double* ho = static_cast<double*>(ctx->h_ovl.p);
  double* hsgn = ho + no + 1;
  int* hidx = reinterpret_cast<int*>(hsgn + k[0] + k[1] + 1);
  HS_CUDA(cudaMemcpyAsync(ho, ctx->ovl.p, (size_t)no * sizeof(double), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  for (int b = 0; b < 2; ++b) {
    const int kb = k[b];
    const double* O = ho + ooff[b];
    int* ib = hidx + (b ? k[0] : 0);
    // each new row's best previous row; rows with the clearest match first,
    // each taking its previous row's position when that is still free and
    // the overlap is above 1/2; the rest fill the free positions in order
    std::vector<int> best(kb, 0), pos(kb, -1), order(kb);
    std::vector<double> ov(kb, 0.0);
    for (int i = 0; i < kb; ++i) {
      for (int j = 1; j < kb; ++j)
        if (std::fabs(O[(long long)i * kb + j]) > std::fabs(O[(long long)i * kb + best[i]])) best[i] = j;
      ov[i] = std::fabs(O[(long long)i * kb + best[i]]);
      order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ov[x] > ov[y]; });
    std::vector<char> taken(kb, 0);
    for (int i : order)
      if (ov[i] > 0.5 && !taken[best[i]]) {
        pos[i] = best[i];
        taken[best[i]] = 1;
      }
    int free_j = 0;
    for (int i = 0; i < kb; ++i) {
      if (pos[i] >= 0) continue;
      while (taken[free_j]) ++free_j;
      pos[i] = free_j;
      taken[free_j] = 1;
    }
    double* sb = hsgn + (b ? k[0] : 0);
    for (int i = 0; i < kb; ++i) {
      ib[pos[i]] = i;
      // a matched row takes the sign of the previous row it continues
      sb[pos[i]] = (pos[i] == best[i] && O[(long long)i * kb + best[i]] < 0.0) ? -1.0 : 1.0;
      *moved += pos[i] != i || sb[pos[i]] < 0.0;
    }
  }
  if (*moved == 0) return HS_OK;
  HS_TRY(ctx->ovl_sgn.ensure((size_t)(k[0] + k[1] + 1) * sizeof(double)));
  HS_CUDA(cudaMemcpyAsync(ctx->ovl_idx.p, hidx, (size_t)(k[0] + k[1]) * sizeof(int), cudaMemcpyHostToDevice, s));
  HS_CUDA(cudaMemcpyAsync(ctx->ovl_sgn.p, hsgn, (size_t)(k[0] + k[1]) * sizeof(double), cudaMemcpyHostToDevice, s));
  HS_CUDA(launch_gather_rows_idx_sign_pair(ctx->pt.d(), off1, n[0], n[1], static_cast<const int*>(ctx->ovl_idx.p),
                                           ctx->ovl_sgn.d(), k[0], k[1], ctx->pt_tmp.d(), off1, s));
  HS_CUDA(cudaMemcpyAsync(ctx->pt.d(), ctx->pt_tmp.d(), (size_t)npt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ctx->launches += 1;
  return HS_OK;
}

// Keep this move's final kept rows for the next move's align_kept_rows.
hs_status keep_pt(hs_ctx ctx, const int k[2], const int n[2]) {
  const long long npt = (long long)k[0] * n[0] + (long long)k[1] * n[1];
  HS_TRY(ctx->pt_prev.ensure((size_t)(npt + 1) * sizeof(double)));
  HS_CUDA(cudaMemcpyAsync(ctx->pt_prev.d(), ctx->pt.d(), (size_t)npt * sizeof(double), cudaMemcpyDeviceToDevice,
                          ctx->stream));
  ctx->pt_prev_valid = true;
  for (int b = 0; b < 2; ++b) {
    ctx->pt_prev_k[b] = k[b];
    ctx->pt_prev_n[b] = n[b];
  }
  return HS_OK;
}

// FP32-eigenvector projector (HS_EIG_F32_PROJECTED): gather the kept FP32
// eigenvectors, then finish_projector.
hs_status project_f32(hs_ctx ctx, const float* V0f, int n0, const float* V1f, int n1, const int* didx, int chi,
                      SelectOut* dsel, Sect c, Sect q, Sect cn, const double* C0, const double* C1, hs_env* env,
                      double* flops) {
  const long long npt = (long long)cn.n[0] * n0 + (long long)cn.n[1] * n1;
  HS_TRY(ctx->pcol.ensure(npt * sizeof(double)));
  {
    PhaseScope ps(ctx, HS_PHASE_SELECT);
    HS_CUDA(launch_gather_p32(V0f, n0, V1f, n1, didx, chi, dsel, ctx->pt.d(), ctx->pcol.d(), ctx->stream));
    ctx->launches += 1;
  }
  return finish_projector(ctx, n0, n1, dsel, c, q, cn, C0, C1, env, flops, 2);
}

// ---- warm-started subspace eigensolver (HS_EIG_SUBSPACE) ----


// Orthonormalise the rows of X_b (m_b x n_b) of both parity blocks (m_b = 0
// skips one): one Cholesky-QR pass with FP64 products, X <- L^{-1} X with
// X X^T = L L^T, leaves an orthogonality error of about eps cond(X)^2
// (Yamamoto et al., 2015), which one Loewdin step in the move's GEMM
// precision squares away. The two factorisations share one launch.
// Non-positive pivots raise *bad (device).
hs_status orthonormalise_rows(hs_ctx ctx, hs_precision prec, double* const X[2], const int m[2], const int n[2],
                              double* const Xc[2], int* bad) {
  const int mm = std::max(m[0], m[1]);
  if (mm == 0) return HS_OK;
  HS_TRY(ctx->schol.ensure(4 * (size_t)mm * mm * sizeof(double)));
  double* G[2] = {ctx->schol.d(), ctx->schol.d() + 2LL * mm * mm};
  double* Li[2] = {G[0] + (long long)mm * mm, G[1] + (long long)mm * mm};
  // stacked pairs (block 1 right after block 0 in X and Xc) run both
  // blocks in one launch per step
  const long long mn0 = (long long)m[0] * n[0];
  const bool stacked = m[0] > 0 && m[1] > 0 && X[1] == X[0] + mn0 && Xc[1] == Xc[0] + mn0;
  if (stacked) {
    GemmGroup gg{2, {GemmProblem{m[0], m[0], n[0], n[0], n[0], m[0], 0, 0, 0},
                     GemmProblem{m[1], m[1], n[1], n[1], n[1], m[1], mn0, mn0, G[1] - G[0]}}};
    HS_TRY(gemm(ctx, HS_GEMM_OWN, gg, X[0], X[0], G[0]));
  } else {
    for (int b = 0; b < 2; ++b)
      if (m[b] > 0)
        HS_TRY(gemm(ctx, HS_GEMM_OWN, GemmGroup{1, {GemmProblem{m[b], m[b], n[b], n[b], n[b], m[b], 0, 0, 0}}},
                    X[b], X[b], G[b]));
  }
  if (mm <= max_chol()) {
    HS_CUDA(launch_chol_inv(G[0], m[0], Li[0], G[1], m[1], Li[1], bad, ctx->stream));
    ctx->launches += 1;
  } else {
    // beyond the one-CTA kernel's shared memory: cuSOLVER potrf + trtri. In the
    // column-major view of the row-major G the upper factor U (G = U^T U) is
    // the row-major L = U^T, and U^{-1} is the row-major L^{-1}
    int* linfo = static_cast<int*>(ctx->info.p) + 4;  // potrf, trtri
    for (int b = 0; b < 2; ++b) {
      if (m[b] == 0) continue;
      HS_CUDA(cudaMemcpyAsync(Li[b], G[b], (size_t)m[b] * m[b] * sizeof(double), cudaMemcpyDeviceToDevice,
                              ctx->stream));
      size_t dw = 0, hw = 0, dw2 = 0, hw2 = 0;
      HS_SOLVER(cusolverDnXpotrf_bufferSize(ctx->solver, ctx->params, CUBLAS_FILL_MODE_UPPER, m[b], CUDA_R_64F,
                                            Li[b], m[b], CUDA_R_64F, &dw, &hw));
      HS_SOLVER(cusolverDnXtrtri_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, m[b],
                                            CUDA_R_64F, Li[b], m[b], &dw2, &hw2));
      HS_TRY(ctx->solver_dev.ensure(std::max(dw, dw2) + 256));
      if (ctx->solver_host.size() < std::max(hw, hw2) + 1) ctx->solver_host.resize(std::max(hw, hw2) + 1);
      HS_CUDA(cudaMemsetAsync(linfo, 0, 2 * sizeof(int), ctx->stream));
      HS_SOLVER(cusolverDnXpotrf(ctx->solver, ctx->params, CUBLAS_FILL_MODE_UPPER, m[b], CUDA_R_64F, Li[b], m[b],
                                 CUDA_R_64F, ctx->solver_dev.p, ctx->solver_dev.bytes, ctx->solver_host.data(),
                                 ctx->solver_host.size(), linfo));
      HS_SOLVER(cusolverDnXtrtri(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, m[b], CUDA_R_64F, Li[b],
                                 m[b], ctx->solver_dev.p, ctx->solver_dev.bytes, ctx->solver_host.data(),
                                 ctx->solver_host.size(), linfo + 1));
      HS_CUDA(launch_tidy_linv(Li[b], m[b], linfo, bad, ctx->stream));
      ctx->launches += 2;
    }
  }
  if (stacked) {
    HS_TRY(permute(ctx, zd(m[0], m[1], n[0], n[1]), zd(n[0], n[1], m[0], m[1]), {1, 0}, X[0], Xc[0]));
    GemmGroup gl{2, {GemmProblem{m[0], n[0], m[0], m[0], m[0], n[0], 0, 0, 0},
                     GemmProblem{m[1], n[1], m[1], m[1], m[1], n[1], Li[1] - Li[0], mn0, mn0}}};
    HS_TRY(gemm(ctx, HS_GEMM_OWN, gl, Li[0], Xc[0], X[0]));
    HS_TRY(lowdin_rows_pair(ctx, prec, X[0], m, n, Xc[0], 1));
    return HS_OK;
  }
  for (int b = 0; b < 2; ++b)
    if (m[b] > 0) {
      HS_TRY(permute(ctx, dense2(m[b], n[b]), dense2(n[b], m[b]), {1, 0}, X[b], Xc[b]));
      HS_TRY(gemm(ctx, HS_GEMM_OWN, GemmGroup{1, {GemmProblem{m[b], n[b], m[b], m[b], m[b], n[b], 0, 0, 0}}},
                  Li[b], Xc[b], X[b]));
      HS_TRY(lowdin_rows(ctx, prec, X[b], m[b], n[b], Xc[b], 1));
    }
  return HS_OK;
}

// Orthonormal rows spanning the rows of Xsrc (stacked blocks, m_b x n_b
// row-major, overwritten) into X, by Householder QR of each block (cuSOLVER
// geqrf + orgqr on the column-major n_b x m_b view, whose Q is the row-major
// m_b x n_b result). Backward stable for any conditioning, but about four
// times the time of the Cholesky-QR pass on these shapes with GB300's FP64
// rate, so it serves only where that pass broke down.
hs_status orthonormalise_rows_qr(hs_ctx ctx, double* Xsrc, const int m[2], const int n[2], double* X) {
  cudaStream_t s = ctx->stream;
  HS_SOLVER(cusolverDnSetStream(ctx->solver, s));
  const long long off1 = (long long)m[0] * n[0];
  int* qinfo = static_cast<int*>(ctx->info.p) + 6;
  for (int b = 0; b < 2; ++b) {
    if (m[b] == 0) continue;
    double* A = Xsrc + (b ? off1 : 0);
    int lw1 = 0, lw2 = 0;
    HS_TRY(ctx->lam.ensure(((size_t)m[b] + 1) * sizeof(double)));  // tau (the selection is rebuilt later)
    double* tau = ctx->lam.d();
    HS_SOLVER(cusolverDnDgeqrf_bufferSize(ctx->solver, n[b], m[b], A, n[b], &lw1));
    HS_SOLVER(cusolverDnDorgqr_bufferSize(ctx->solver, n[b], m[b], m[b], A, n[b], tau, &lw2));
    HS_TRY(ctx->solver_dev.ensure((size_t)std::max(std::max(lw1, lw2), 1) * sizeof(double)));
    HS_SOLVER(cusolverDnDgeqrf(ctx->solver, n[b], m[b], A, n[b], tau, ctx->solver_dev.d(), std::max(lw1, 1), qinfo));
    HS_SOLVER(cusolverDnDorgqr(ctx->solver, n[b], m[b], m[b], A, n[b], tau, ctx->solver_dev.d(), std::max(lw2, 1),
                               qinfo + 1));
    HS_CUDA(cudaMemcpyAsync(X + (b ? off1 : 0), A, (size_t)m[b] * n[b] * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  return HS_OK;
}

// C[M x N] = A[M x K] B[N x K]^T for dense FP64 row-major operands: on the
// tensor cores (operands split into sx / sy) in the TF32/BF16 precisions,
// with the FP64 kernel otherwise.
hs_status dense_gemm_any(hs_ctx ctx, hs_precision prec, int M, int N, int K, const double* A, const double* B,
                         double* C) {
  if (prec == HS_PREC_F64)
    return gemm(ctx, HS_GEMM_OWN, GemmGroup{1, {GemmProblem{M, N, K, K, K, N, 0, 0, 0}}}, A, B, C);
  HS_TRY(tc_split(ctx, prec, dense2(M, K), dense2(M, K), {0, 1}, A, ctx->sx_hi, ctx->sx_lo));
  HS_TRY(tc_split(ctx, prec, dense2(N, K), dense2(N, K), {0, 1}, B, ctx->sy_hi, ctx->sy_lo));
  HS_TRY(tc_run(ctx, prec, dense2(M, K), ctx->sx_hi, ctx->sx_lo, dense2(N, K), ctx->sy_hi, ctx->sy_lo,
                dense2(M, N), C));
  ctx->phase_flops[HS_PHASE_GEMM_TC] += 2.0 * M * (double)N * K;
  return HS_OK;
}

// Loewdin orthonormalisation of the m rows of X (n long), for rows already
// close to orthonormal: X <- (3/2 I - 1/2 X X^T) X, `steps` times.
hs_status lowdin_rows(hs_ctx ctx, hs_precision prec, double* X, int m, int n, double* Xc, int steps) {
  HS_TRY(ctx->schol.ensure(2 * (size_t)m * m * sizeof(double)));
  double* G = ctx->schol.d();
  for (int st = 0; st < steps; ++st) {
    HS_TRY(dense_gemm_any(ctx, prec, m, m, n, X, X, G));
    HS_CUDA(launch_lowdin(G, m, 0, ctx->stream));
    HS_TRY(permute(ctx, dense2(m, n), dense2(n, m), {1, 0}, X, Xc));
    HS_TRY(dense_gemm_any(ctx, prec, m, n, m, G, Xc, X));
    ctx->launches += 1;
  }
  return HS_OK;
}

// Chebyshev-filtered power step on block b after a Rayleigh-Ritz step that
// did not converge (Ritz vectors in sxr[b], their products with H in szr[b],
// FP32 Ritz values theta, kept_b of them in the selection). The spectrum of
// C' falls off slowly past the cut, so plain power steps gain little there;
// a Chebyshev polynomial T_deg(H / a) damps |lambda| <= a and amplifies the
// states just above the cut by T_deg(|lambda| / a) (Zhou and Saad, 2007).
// a is an interior Ritz magnitude of the window, an estimate of the largest
// |lambda| outside it. The filter also grows the top of the spectrum by
// orders of magnitude more than the cut, which would swamp the rows in
// rounding; so the Ritz pairs with |theta| >= kLock a are locked: they take
// two plain power steps and their span is projected out after every product
// of the filtered rows. X receives the locked rows, then
// the filtered ones (not normalised). Returns false in *used when no interior
// magnitude exists (the caller then takes a plain step).
constexpr int kMaxSubRows = 256;  // bound on the subspace rows (max_subspace() is smaller)

hs_status cheb_filter_block(hs_ctx ctx, hs_precision prec, int b, int m, int n, const double* H,
                            const float* theta, int kept_b, double* X, bool* used) {
  constexpr int kDeg = 8;
  constexpr double kLock = 8.0, kEdge = 0.3;
  *used = false;
  cudaStream_t s = ctx->stream;
  const bool tc = prec != HS_PREC_F64;
  std::vector<int> ord(m);
  for (int i = 0; i < m; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int x, int y) { return std::fabs((double)theta[x]) > std::fabs((double)theta[y]); });
  int r = kept_b + 2 + (int)(kEdge * (m - kept_b - 2));
  r = std::max(0, std::min(r, m - 1));
  const double a = std::fabs((double)theta[ord[r]]);
  if (!(a > 0.0) || r <= kept_b) return HS_OK;
  std::vector<int> idx;
  idx.reserve(m);
  for (int i = 0; i < m; ++i)
    if (std::fabs((double)theta[i]) >= kLock * a) idx.push_back(i);
  const int mL = (int)idx.size(), mU = m - mL;
  for (int i = 0; i < m; ++i)
    if (std::fabs((double)theta[i]) < kLock * a) idx.push_back(i);
  // per-block regions of the pinned and device index buffers: the copy is
  // asynchronous, so block 1 must not overwrite block 0's staging
  HS_TRY(ctx->sf_idx.ensure(2 * (size_t)kMaxSubRows * sizeof(int)));
  HS_TRY(ctx->h_idx.ensure(2 * (size_t)kMaxSubRows * sizeof(int)));
  if (m > kMaxSubRows) return fail(HS_ERR_INVALID_ARG, "subspace of %d rows", m);
  int* didx = static_cast<int*>(ctx->sf_idx.p) + b * kMaxSubRows;
  int* hidx = static_cast<int*>(ctx->h_idx.p) + b * kMaxSubRows;
  std::copy(idx.begin(), idx.end(), hidx);
  HS_CUDA(cudaMemcpyAsync(didx, hidx, (size_t)m * sizeof(int), cudaMemcpyHostToDevice, s));
  const size_t mn = (size_t)m * n * sizeof(double);
  for (auto* buf : {&ctx->sf_y[0], &ctx->sf_y[1], &ctx->sf_y[2], &ctx->sf_z, &ctx->sf_t, &ctx->sf_q, &ctx->sf_qt})
    HS_TRY(buf->ensure(mn));
  HS_TRY(ctx->sf_s.ensure((size_t)m * m * sizeof(double)));
  const double* Xr = ctx->sxr.d(b);
  const double* Zr = ctx->szr.d(b);
  const DBuf hhi = tc ? sH_block(ctx, prec, true, b) : DBuf{}, hlo = tc ? sH_block(ctx, prec, false, b) : DBuf{};
  // product of mr rows of Y (m x n) with H into Z
  auto hprod = [&](const double* Y, int mr, double* Z) -> hs_status {
    if (tc) {
      HS_TRY(tc_split(ctx, prec, dense2(mr, n), dense2(mr, n), {0, 1}, Y, ctx->sx_hi, ctx->sx_lo));
      HS_TRY(tc_run(ctx, prec, dense2(mr, n), ctx->sx_hi, ctx->sx_lo, dense2(n, n), hhi, hlo, dense2(mr, n), Z));
      ctx->phase_flops[HS_PHASE_GEMM_TC] += 2.0 * mr * (double)n * n;
    } else {
      HS_TRY(gemm(ctx, HS_GEMM_OWN, GemmGroup{1, {GemmProblem{mr, n, n, n, n, n, 0, 0, 0}}}, Y, H, Z));
      ctx->phase_flops[HS_PHASE_GEMM] += 2.0 * mr * (double)n * n;
    }
    return HS_OK;
  };
  // locked rows: two power steps (the first is their rows of Zr); the ratio
  // to the largest |lambda| outside the window is at most 1 / kLock per step
  if (mL > 0) {
    HS_CUDA(launch_gather_rows_idx(Zr, didx, mL, n, ctx->sf_z.d(), s));
    HS_CUDA(launch_row_normalize(ctx->sf_z.d(), mL, n, s));
    HS_TRY(hprod(ctx->sf_z.d(), mL, X));
    ctx->launches += 2;
  }
  if (mU > 0) {
    double* Q = ctx->sf_q.d();
    double* Qt = ctx->sf_qt.d();
    double* Z = ctx->sf_z.d();
    double* T = ctx->sf_t.d();
    double* S = ctx->sf_s.d();
    double* Y[3] = {ctx->sf_y[0].d(), ctx->sf_y[1].d(), ctx->sf_y[2].d()};
    if (mL > 0) {
      HS_CUDA(launch_gather_rows_idx(Xr, didx, mL, n, Q, s));
      HS_TRY(permute(ctx, dense2(mL, n), dense2(n, mL), {1, 0}, Q, Qt));
      ctx->launches += 1;
    }
    HS_CUDA(launch_gather_rows_idx(Xr, didx + mL, mU, n, Y[0], s));
    HS_CUDA(launch_gather_rows_idx(Zr, didx + mL, mU, n, Z, s));
    ctx->launches += 2;
    const long long cnt = (long long)mU * n;
    // Z <- Z - (Z Q^T) Q: the part of Z outside the locked span (into T, then combined)
    auto project = [&]() -> hs_status {
      if (mL == 0) return HS_OK;
      HS_TRY(dense_gemm_any(ctx, prec, mU, mL, n, Z, Q, S));
      HS_TRY(dense_gemm_any(ctx, prec, mU, n, mL, S, Qt, T));
      return HS_OK;
    };
    HS_TRY(project());
    HS_CUDA(launch_cheb_step(Y[1], Z, mL > 0 ? T : nullptr, nullptr, cnt, 1.0 / a, 0.0, s));
    ctx->launches += 1;
    int prev = 0, cur = 1;
    for (int j = 2; j <= kDeg; ++j) {
      const int next = 3 - prev - cur;
      HS_TRY(hprod(Y[cur], mU, Z));
      HS_TRY(project());
      HS_CUDA(launch_cheb_step(Y[next], Z, mL > 0 ? T : nullptr, Y[prev], cnt, 2.0 / a, -1.0, s));
      ctx->launches += 1;
      prev = cur;
      cur = next;
    }
    HS_CUDA(cudaMemcpyAsync(X + (long long)mL * n, Y[cur], (size_t)cnt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  *used = true;
  return HS_OK;
}

// A block-diagonal pair as one Z2 layout: block p is r_p x c_p (stacked).
Z2Mat zd(long long r0, long long r1, long long c0, long long c1, int pad) {
  return mat(fused1(make_sect((int)r0, (int)r1)), fused1(make_sect((int)c0, (int)c1)), pad);
}

// A view of part of a buffer (never grown or freed through the view).
DBuf view(const DBuf& b, long long byte_off) {
  DBuf v;
  v.p = static_cast<char*>(b.p) + byte_off;
  v.bytes = 0;
  return v;
}

// The split C' block b (dense n_b x n_b) inside the stacked split sH_hi/lo.
DBuf sH_block(hs_ctx ctx, hs_precision prec, bool hi, int b) {
  const Z2Mat P = zd(ctx->sH_n[0], ctx->sH_n[1], ctx->sH_n[0], ctx->sH_n[1], tc_pad(prec));
  return view(hi ? ctx->sH_hi : ctx->sH_lo, z2_block_off(P, b) * tc_elem_bytes(prec));
}

// Both C' blocks (stacked: block 1 right after block 0) split once per move.
hs_status split_corner(hs_ctx ctx, hs_precision prec, const double* H0, int n0, int n1) {
  HS_TRY(tc_split_any(ctx, prec, zd(n0, n1, n0, n1), zd(n0, n1, n0, n1), {0, 1}, H0, ctx->cp_f32, ctx->sH_hi,
                      ctx->sH_lo));
  ctx->sH_n[0] = n0;
  ctx->sH_n[1] = n1;
  ctx->sH_fresh = true;
  return HS_OK;
}

// `steps` Loewdin steps X <- (3/2 I - 1/2 X X^T) X on the rows of both blocks
// of a stacked pair (m_b rows of n_b), each product one tensor-core launch
// for both blocks; with FP64 products block by block.
hs_status lowdin_rows_pair(hs_ctx ctx, hs_precision prec, double* X, const int m[2], const int n[2], double* Xc,
                           int steps) {
  if (prec == HS_PREC_F64) {
    for (int b = 0; b < 2; ++b)
      if (m[b] > 0 && n[b] > 0)
        HS_TRY(lowdin_rows(ctx, prec, X + (b ? (long long)m[0] * n[0] : 0), m[b], n[b], Xc, steps));
    return HS_OK;
  }
  const Z2Mat XL = zd(m[0], m[1], n[0], n[1]), GL = zd(m[0], m[1], m[0], m[1]), XT = zd(n[0], n[1], m[0], m[1]);
  HS_TRY(ctx->schol.ensure(((size_t)m[0] * m[0] + (size_t)m[1] * m[1] + 1) * sizeof(double)));
  double* G = ctx->schol.d();
  for (int st = 0; st < steps; ++st) {
    // G = X X^T (the split X serves as both operands)
    HS_TRY(tc_split(ctx, prec, XL, XL, {0, 1}, X, ctx->sx_hi, ctx->sx_lo));
    HS_TRY(tc_run(ctx, prec, XL, ctx->sx_hi, ctx->sx_lo, XL, ctx->sx_hi, ctx->sx_lo, GL, G));
    HS_CUDA(launch_lowdin(G, m[0], m[1], ctx->stream));
    // X <- G X: G split as A, X^T written straight into the split B operand
    HS_TRY(tc_split(ctx, prec, GL, GL, {0, 1}, G, ctx->sy_hi, ctx->sy_lo));
    HS_TRY(tc_split(ctx, prec, XL, XT, {1, 0}, X, ctx->sx_hi, ctx->sx_lo));
    HS_TRY(tc_run(ctx, prec, GL, ctx->sy_hi, ctx->sy_lo, XT, ctx->sx_hi, ctx->sx_lo, XL, X));
    ctx->launches += 1;
    for (int b = 0; b < 2; ++b) ctx->phase_flops[HS_PHASE_GEMM_TC] += 4.0 * m[b] * (double)m[b] * n[b];
  }
  return HS_OK;
}

// cheb_filter_block for both parity blocks at once (tensor-core precisions):
// the locked rows, the filtered rows and every product stacked over the
// blocks, so that each split, product and projection is one launch for both.
// Each block has its own interior magnitude a_b and lock; a block without an
// interior magnitude locks every row (two plain power steps). Writes the
// new basis into ctx->sx (not normalised).
hs_status cheb_filter_pair(hs_ctx ctx, hs_precision prec, const int m[2], const int n[2], const float* theta,
                           const int kept[2]) {
  constexpr int kDeg = 8;
  constexpr double kLock = 8.0, kEdge = 0.3;
  cudaStream_t s = ctx->stream;
  double a[2] = {0.0, 0.0};
  int mL[2] = {0, 0}, mU[2] = {0, 0};
  std::vector<int> idxL[2], idxU[2];
  for (int b = 0; b < 2; ++b) {
    if (m[b] == 0) continue;
    const float* th = theta + (b ? m[0] : 0);
    std::vector<int> ord(m[b]);
    for (int i = 0; i < m[b]; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int x, int y) { return std::fabs((double)th[x]) > std::fabs((double)th[y]); });
    int r = kept[b] + 2 + (int)(kEdge * (m[b] - kept[b] - 2));
    r = std::max(0, std::min(r, m[b] - 1));
    a[b] = std::fabs((double)th[ord[r]]);
    const bool filt = a[b] > 0.0 && r > kept[b];
    for (int i = 0; i < m[b]; ++i) {
      if (!filt || std::fabs((double)th[i]) >= kLock * a[b])
        idxL[b].push_back(i);
      else
        idxU[b].push_back(i);
    }
    mL[b] = (int)idxL[b].size();
    mU[b] = (int)idxU[b].size();
    if (!filt) a[b] = 1.0;  // unused (no filtered rows)
  }
  // row orders to the device through pinned staging: locked rows of both
  // blocks, then unlocked rows of both blocks
  const int ntot = m[0] + m[1];
  HS_TRY(ctx->sf_idx.ensure(((size_t)ntot + 4) * sizeof(int)));
  HS_TRY(ctx->h_idx.ensure(((size_t)ntot + 4) * sizeof(int)));
  int* hidx = static_cast<int*>(ctx->h_idx.p);
  int k = 0;
  for (int b = 0; b < 2; ++b)
    for (int i : idxL[b]) hidx[k++] = i;
  for (int b = 0; b < 2; ++b)
    for (int i : idxU[b]) hidx[k++] = i;
  int* didx = static_cast<int*>(ctx->sf_idx.p);
  HS_CUDA(cudaMemcpyAsync(didx, hidx, (size_t)ntot * sizeof(int), cudaMemcpyHostToDevice, s));
  const int* dL = didx;
  const int* dU = didx + mL[0] + mL[1];
  const long long mn = (long long)m[0] * n[0] + (long long)m[1] * n[1];
  for (auto* buf : {&ctx->sf_y[0], &ctx->sf_y[1], &ctx->sf_y[2], &ctx->sf_z, &ctx->sf_t, &ctx->sf_q, &ctx->sf_xl})
    HS_TRY(buf->ensure((size_t)(mn + 2) * sizeof(double)));
  HS_TRY(ctx->sf_s.ensure(((size_t)m[0] * m[0] + (size_t)m[1] * m[1] + 2) * sizeof(double)));
  const Z2Mat LL = zd(mL[0], mL[1], n[0], n[1]), UL = zd(mU[0], mU[1], n[0], n[1]), HL = zd(n[0], n[1], n[0], n[1]),
              LT = zd(n[0], n[1], mL[0], mL[1]), SL = zd(mU[0], mU[1], mL[0], mL[1]);
  const long long xoff1 = (long long)m[0] * n[0];
  auto hprod = [&](const Z2Mat& RL, const double* Y, double* Z) -> hs_status {
    HS_TRY(tc_split(ctx, prec, RL, RL, {0, 1}, Y, ctx->sx_hi, ctx->sx_lo));
    HS_TRY(tc_run(ctx, prec, RL, ctx->sx_hi, ctx->sx_lo, HL, ctx->sH_hi, ctx->sH_lo, RL, Z));
    for (int b = 0; b < 2; ++b)
      ctx->phase_flops[HS_PHASE_GEMM_TC] += 2.0 * z2_rows(RL, b) * (double)n[b] * n[b];
    return HS_OK;
  };
  double* XL = ctx->sf_xl.d();
  // locked rows: two power steps (the first is their rows of Zr)
  if (mL[0] + mL[1] > 0) {
    double* Zl = ctx->sf_z.d();
    HS_CUDA(launch_gather_rows_idx_pair(ctx->szr.d(0), xoff1, n[0], n[1], dL, mL[0], mL[1], Zl,
                                        (long long)mL[0] * n[0], s));
    for (int b = 0; b < 2; ++b)
      HS_CUDA(launch_row_normalize(Zl + (b ? (long long)mL[0] * n[0] : 0), mL[b], n[b], s));
    HS_TRY(hprod(LL, Zl, XL));
    ctx->launches += 3;
  }
  double* Y[3] = {ctx->sf_y[0].d(), ctx->sf_y[1].d(), ctx->sf_y[2].d()};
  int cur = 0;
  if (mU[0] + mU[1] > 0) {
    double* Q = ctx->sf_q.d();
    double* Z = ctx->sf_z.d();
    double* T = ctx->sf_t.d();
    double* S = ctx->sf_s.d();
    const bool proj = mL[0] + mL[1] > 0;
    if (proj) {
      // the locked span, split once in both orientations (B of S = Z Q^T and of T = S Q)
      HS_CUDA(launch_gather_rows_idx_pair(ctx->sxr.d(0), xoff1, n[0], n[1], dL, mL[0], mL[1], Q,
                                          (long long)mL[0] * n[0], s));
      HS_TRY(tc_split(ctx, prec, LL, LL, {0, 1}, Q, ctx->sf_qh, ctx->sf_ql));
      HS_TRY(tc_split(ctx, prec, LL, LT, {1, 0}, Q, ctx->sf_qth, ctx->sf_qtl));
      ctx->launches += 1;
    }
    const long long uoff1 = (long long)mU[0] * n[0];
    HS_CUDA(launch_gather_rows_idx_pair(ctx->sxr.d(0), xoff1, n[0], n[1], dU, mU[0], mU[1], Y[0], uoff1, s));
    HS_CUDA(launch_gather_rows_idx_pair(ctx->szr.d(0), xoff1, n[0], n[1], dU, mU[0], mU[1], Z, uoff1, s));
    ctx->launches += 2;
    const long long cnt = uoff1 + (long long)mU[1] * n[1];
    // Z <- Z - (Z Q^T) Q: the part of Z outside the locked span (T holds the second term)
    auto project = [&]() -> hs_status {
      if (!proj) return HS_OK;
      HS_TRY(tc_split(ctx, prec, UL, UL, {0, 1}, Z, ctx->sx_hi, ctx->sx_lo));
      HS_TRY(tc_run(ctx, prec, UL, ctx->sx_hi, ctx->sx_lo, LL, ctx->sf_qh, ctx->sf_ql, SL, S));
      HS_TRY(tc_split(ctx, prec, SL, SL, {0, 1}, S, ctx->sy_hi, ctx->sy_lo));
      HS_TRY(tc_run(ctx, prec, SL, ctx->sy_hi, ctx->sy_lo, LT, ctx->sf_qth, ctx->sf_qtl, UL, T));
      return HS_OK;
    };
    HS_TRY(project());
    HS_CUDA(launch_cheb_step_pair(Y[1], Z, proj ? T : nullptr, nullptr, cnt, uoff1, 1.0 / a[0], 1.0 / a[1], 0.0, s));
    ctx->launches += 1;
    int prev = 0;
    cur = 1;
    for (int j = 2; j <= kDeg; ++j) {
      const int next = 3 - prev - cur;
      HS_TRY(hprod(UL, Y[cur], Z));
      HS_TRY(project());
      HS_CUDA(launch_cheb_step_pair(Y[next], Z, proj ? T : nullptr, Y[prev], cnt, uoff1, 2.0 / a[0], 2.0 / a[1], -1.0,
                                    s));
      ctx->launches += 1;
      prev = cur;
      cur = next;
    }
  }
  // assemble the new basis per block: locked rows, then filtered rows
  for (int b = 0; b < 2; ++b) {
    if (m[b] == 0) continue;
    double* Xb = ctx->sx.d(b);
    if (mL[b] > 0)
      HS_CUDA(cudaMemcpyAsync(Xb, XL + (b ? (long long)mL[0] * n[0] : 0), (size_t)mL[b] * n[b] * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
    if (mU[b] > 0)
      HS_CUDA(cudaMemcpyAsync(Xb + (long long)mL[b] * n[b], Y[cur] + (b ? (long long)mU[0] * n[0] : 0),
                              (size_t)mU[b] * n[b] * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  return HS_OK;
}

// Spare rows of the subspace beyond k kept states: 24, or k/3 when that is
// more, so that a block of many kept states (the dense basis, whose spectrum
// interleaves both parity sectors) keeps the same relative margin past the cut.
int oversample(int k) { return std::max(24, (k + 2) / 3); }

// Subspace iteration on both parity blocks H_b (n_b x n_b, FP64 in place in
// the C' buffer), warm-started from the previous move's kept rows. On success
// (*done) w[0 .. m0+m1) holds the Ritz values of block 0 then block 1
// (ascending per block), sxr[b] the matching Ritz vectors as rows, and
// m_out the subspace sizes; otherwise the caller falls back.
hs_status subspace_projector(hs_ctx ctx, hs_env* env, int chi, int n0, int n1, double* H0, double* H1, double* w,
                             int* m_out, bool* done, int* iters, double* flops, int* reason, double* resid) {
  *done = false;
  *iters = 0;
  *resid = 0.0;
  const int n[2] = {n0, n1};
  double* H[2] = {H0, H1};
  *reason = 1;
  if (!(ctx->ws_valid && ctx->ws_env == env)) return HS_OK;
  *reason = 2;
  // sector sizes changed since the stored rows: carry them over to the new
  // boundary sectors (the states both boundaries have), then orthonormalise
  const Sect c_now = make_sect(env->chi_even, env->chi_odd), q_now = make_sect(env->q_even, env->q_odd);
  const bool remap = !(ctx->ws_n[0] == n0 && ctx->ws_n[1] == n1);
  if (remap && (ctx->ws_c[0] < 0 || n0 != c_now.n[0] * q_now.n[0] + c_now.n[1] * q_now.n[1] ||
                n1 != c_now.n[0] * q_now.n[1] + c_now.n[1] * q_now.n[0]))
    return HS_OK;
  constexpr int kMinOver = 8, kMaxIt = 8;
  cudaStream_t s = ctx->stream;
  const bool tc = env->precision != HS_PREC_F64;
  // residual tolerance relative to max|theta|: above the rounding floor of
  // the products H X (about 2e-6 with 3-pass TF32 at n ~ 2600)
  const double kTol = tc ? 1e-5 : 1e-6;
  // adaptive mode: while the environment still changes from move to move, the
  // projector needs no more accuracy than that change. Its measure: the
  // residual of the warm start in the previous move's first round (how far
  // the kept subspace turned in one move); tol = 0.1 of it, between kTol and
  // 1e-3, so that it is kTol again at the fixed point
  const bool adaptive = env->eig_mode == HS_EIG_SUBSPACE_ADAPTIVE && ctx->prev_spec_env == env &&
                        ctx->prev_first_resid > 0.0;
  const double tol_move = adaptive ? std::min(1e-3, std::max(kTol, 0.1 * ctx->prev_first_resid)) : kTol;
  const hs_precision prec = env->precision;
  int m[2];
  for (int b = 0; b < 2; ++b) {
    // k + oversample(k) rows, at most the block and the Rayleigh-Ritz kernels' limit;
    // at least 8 rows beyond the kept ones unless the subspace is the block
    m[b] = n[b] == 0 ? 0 : std::min(std::min(ctx->ws_k[b] + oversample(ctx->ws_k[b]), n[b]), max_subspace());
    *reason = 3;
    if (m[b] < n[b] && m[b] < ctx->ws_k[b] + kMinOver) return HS_OK;
  }
  int* bad = static_cast<int*>(ctx->info.p) + 2;
  HS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  HS_CUDA(cudaMemsetAsync(static_cast<int*>(ctx->info.p) + 6, 0, 2 * sizeof(int), s));  // Householder QR status
  HS_TRY(eig32_workspace(ctx, m[0] > m[1] ? m[0] : m[1]));
  // the selection issued by every round writes chi indices per block and chi values
  HS_TRY(ctx->idx.ensure(2 * (size_t)chi * sizeof(int)));
  HS_TRY(ctx->lam.ensure((size_t)chi * sizeof(double)));
  // stacked buffers: block 1 after block 0
  const long long mn0 = (long long)m[0] * n[0], mn1 = (long long)m[1] * n[1];
  for (Stacked* t : {&ctx->sx, &ctx->sz, &ctx->sxc, &ctx->szc, &ctx->sxr, &ctx->szr})
    HS_TRY(t->ensure(mn0, mn1, sizeof(double)));
  HS_TRY(ctx->sbm.ensure((long long)m[0] * m[0], (long long)m[1] * m[1], sizeof(double)));
  HS_TRY(ctx->sbw.ensure((long long)m[0] * m[0], (long long)m[1] * m[1], sizeof(float)));
  HS_TRY(ctx->sres.ensure(m[0], m[1], sizeof(double)));
  const Z2Mat XL = zd(m[0], m[1], n[0], n[1]), XT = zd(n[0], n[1], m[0], m[1]), BL = zd(m[0], m[1], m[0], m[1]),
              HL = zd(n[0], n[1], n[0], n[1]);
  // warm start: the previous move's rows (same stacking when the subspace
  // sizes are unchanged), random rows where the subspace grew
  const long long wsoff[2] = {0, (long long)ctx->ws_m[0] * ctx->ws_n[0]};
  const int kb[2] = {std::min(ctx->ws_m[0], m[0]), std::min(ctx->ws_m[1], m[1])};
  bool all_warm = true;
  if (remap) {
    const Sect c_old = make_sect(ctx->ws_c[0], ctx->ws_c[1]);
    for (int b = 0; b < 2; ++b) {
      if (m[b] == 0) continue;
      if (kb[b] > 0)
        HS_CUDA(launch_remap_rows(ctx->ws_pt.d() + wsoff[b], kb[b], ctx->ws_n[b], ctx->sx.d(b), n[b], b, c_old, c_now,
                                  q_now, 0x7e3a0000ull + 2 * (unsigned long long)env->moves + b, s));
      HS_CUDA(launch_fill_random_rows(ctx->sx.d(b), kb[b], m[b], n[b],
                                      0x5eed0000ull + 2 * (unsigned long long)env->moves + b, s));
    }
    all_warm = false;
  } else if (kb[0] == m[0] && kb[1] == m[1] && ctx->ws_m[0] == m[0]) {
    HS_CUDA(cudaMemcpyAsync(ctx->sx.d(0), ctx->ws_pt.d(), (size_t)(mn0 + mn1) * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
  } else {
    for (int b = 0; b < 2; ++b) {
      if (m[b] == 0) continue;
      if (kb[b] > 0)
        HS_CUDA(cudaMemcpyAsync(ctx->sx.d(b), ctx->ws_pt.d() + wsoff[b], (size_t)kb[b] * n[b] * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
      HS_CUDA(launch_fill_random_rows(ctx->sx.d(b), kb[b], m[b], n[b],
                                      0x5eed0000ull + 2 * (unsigned long long)env->moves + b, s));
      if (kb[b] < m[b]) all_warm = false;
    }
  }
  if (all_warm) {
    // the previous move's Ritz / eigen-vectors: orthonormal up to FP32 rounding
    HS_TRY(lowdin_rows_pair(ctx, prec, ctx->sx.d(0), m, n, ctx->sxc.d(0), tc ? 1 : 2));
  } else {
    double* const Xo[2] = {ctx->sx.d(0), ctx->sx.d(1)};
    double* const Xco[2] = {ctx->sxc.d(0), ctx->sxc.d(1)};
    HS_TRY(orthonormalise_rows(ctx, prec, Xo, m, n, Xco, bad));
  }
  if (tc && !(ctx->sH_fresh && ctx->sH_n[0] == n0 && ctx->sH_n[1] == n1)) {
    const size_t es = ctx->cp_f32 ? sizeof(float) : sizeof(double);
    if (reinterpret_cast<const char*>(H1) != reinterpret_cast<const char*>(H0) + (size_t)n0 * n0 * es)
      return fail(HS_ERR_INVALID_ARG, "corner blocks not stacked");
    HS_TRY(split_corner(ctx, prec, H0, n0, n1));
  }
  HS_TRY(ctx->sth.ensure((size_t)(m[0] + m[1] + 2) * sizeof(float)));
  float* th = static_cast<float*>(ctx->sth.p);
  // pinned read-back of the Ritz values, residuals and status words (a copy
  // into pageable memory would block the host before the stream drains)
  const int mt = m[0] + m[1];
  HS_TRY(ctx->h_sub.ensure((size_t)mt * (sizeof(double) + sizeof(float)) + 8 * sizeof(int)));
  double* hres = static_cast<double*>(ctx->h_sub.p);
  float* hth = reinterpret_cast<float*>(hres + mt);
  int* hstat = reinterpret_cast<int*>(hth + mt);  // Jacobi status of both blocks, Cholesky status
  double prev_worst = INFINITY;
  ctx->sx_save_valid = false;
  for (int it = 0; it < kMaxIt; ++it) {
    *iters = it + 1;
    // Z = X H (H symmetric), Rayleigh matrix B = X Z^T (symmetric); with
    // tensor cores each product is one launch for both blocks and the split
    // X serves as the A operand of both
    if (tc) {
      HS_TRY(tc_split(ctx, prec, XL, XL, {0, 1}, ctx->sx.d(0), ctx->sx_hi, ctx->sx_lo));
      HS_TRY(tc_run(ctx, prec, XL, ctx->sx_hi, ctx->sx_lo, HL, ctx->sH_hi, ctx->sH_lo, XL, ctx->sz.d(0)));
      HS_TRY(tc_split(ctx, prec, XL, XL, {0, 1}, ctx->sz.d(0), ctx->sy_hi, ctx->sy_lo));
      // the Rayleigh matrix straight in FP32, the Jacobi eigensolver's input
      // (the tensor-core accumulators are FP32: nothing is lost)
      HS_TRY(tc_run(ctx, prec, XL, ctx->sx_hi, ctx->sx_lo, XL, ctx->sy_hi, ctx->sy_lo, BL,
                    reinterpret_cast<double*>(ctx->sbw.as<float>(0)), true));
      for (int b = 0; b < 2; ++b)
        ctx->phase_flops[HS_PHASE_GEMM_TC] += 2.0 * m[b] * (double)n[b] * n[b] + 2.0 * m[b] * (double)m[b] * n[b];
    } else {
      for (int b = 0; b < 2; ++b) {
        if (m[b] == 0) continue;
        HS_TRY(gemm(ctx, HS_GEMM_OWN, GemmGroup{1, {GemmProblem{m[b], n[b], n[b], n[b], n[b], n[b], 0, 0, 0}}},
                    ctx->sx.d(b), H[b], ctx->sz.d(b)));
        HS_TRY(gemm(ctx, HS_GEMM_OWN, GemmGroup{1, {GemmProblem{m[b], m[b], n[b], n[b], n[b], m[b], 0, 0, 0}}},
                    ctx->sx.d(b), ctx->sz.d(b), ctx->sbm.d(b)));
        ctx->phase_flops[HS_PHASE_GEMM] += 2.0 * m[b] * (double)n[b] * n[b] + 2.0 * m[b] * (double)m[b] * n[b];
      }
    }
    for (int b = 0; b < 2; ++b) *flops += 2.0 * m[b] * (double)n[b] * n[b];
    if (!tc) {
      HS_CUDA(launch_cast_f64_f32(ctx->sbm.d(0), ctx->sbw.as<float>(0),
                                  (long long)m[0] * m[0] + (long long)m[1] * m[1], s));
      ctx->launches += 1;
    }
    {
      // Rayleigh-Ritz: both m x m FP32 problems by one-CTA Jacobi kernels
      PhaseScope ps(ctx, HS_PHASE_EIG);
      HS_CUDA(cudaMemsetAsync(ctx->info.p, 0, 2 * sizeof(int), s));
      HS_CUDA(launch_jacobi_eig_pair(ctx->sbw.as<float>(0), m[0], th, ctx->sbw.as<float>(1), m[1], th + m[0],
                                     static_cast<int*>(ctx->info.p), s));
      ctx->launches += 1;
    }
    // Ritz vectors Xr = W^T X and Zr = W^T Z (W column-major = W^T row-major)
    HS_CUDA(launch_cast_f32_f64(ctx->sbw.as<float>(0), ctx->sbm.d(0),
                                (long long)m[0] * m[0] + (long long)m[1] * m[1], s));
    ctx->launches += 1;
    if (tc) {
      // W split once; X^T and Z^T written straight into the split B operand
      HS_TRY(tc_split(ctx, prec, BL, BL, {0, 1}, ctx->sbm.d(0), ctx->sx_hi, ctx->sx_lo));
      HS_TRY(tc_split(ctx, prec, XL, XT, {1, 0}, ctx->sx.d(0), ctx->sy_hi, ctx->sy_lo));
      HS_TRY(tc_run(ctx, prec, BL, ctx->sx_hi, ctx->sx_lo, XT, ctx->sy_hi, ctx->sy_lo, XL, ctx->sxr.d(0)));
      HS_TRY(tc_split(ctx, prec, XL, XT, {1, 0}, ctx->sz.d(0), ctx->sy_hi, ctx->sy_lo));
      HS_TRY(tc_run(ctx, prec, BL, ctx->sx_hi, ctx->sx_lo, XT, ctx->sy_hi, ctx->sy_lo, XL, ctx->szr.d(0)));
      for (int b = 0; b < 2; ++b) ctx->phase_flops[HS_PHASE_GEMM_TC] += 4.0 * m[b] * (double)m[b] * n[b];
    } else {
      for (int b = 0; b < 2; ++b) {
        if (m[b] == 0) continue;
        HS_TRY(permute(ctx, dense2(m[b], n[b]), dense2(n[b], m[b]), {1, 0}, ctx->sx.d(b), ctx->sxc.d(b)));
        HS_TRY(permute(ctx, dense2(m[b], n[b]), dense2(n[b], m[b]), {1, 0}, ctx->sz.d(b), ctx->szc.d(b)));
        HS_TRY(dense_gemm_any(ctx, prec, m[b], n[b], m[b], ctx->sbm.d(b), ctx->sxc.d(b), ctx->sxr.d(b)));
        HS_TRY(dense_gemm_any(ctx, prec, m[b], n[b], m[b], ctx->sbm.d(b), ctx->szc.d(b), ctx->szr.d(b)));
      }
    }
    HS_CUDA(launch_residual_pair(ctx->szr.d(0), ctx->sxr.d(0), th, m[0], n[0], m[1], n[1], ctx->sres.d(0), s));
    ctx->launches += 1;
    // this round's selection, issued ahead of the readback: when the round
    // converges it is the move's selection, and the move needs no second
    // round trip to the host for it
    HS_CUDA(launch_cast_f32_f64(th, w, m[0] + m[1], s));
    {
      PhaseScope ps(ctx, HS_PHASE_SELECT);
      HS_CUDA(launch_select(w, m[0], w + m[0], m[1], chi, static_cast<int*>(ctx->idx.p), ctx->lam.d(),
                            static_cast<SelectOut*>(ctx->sel.p), s));
    }
    HS_CUDA(cudaMemcpyAsync(ctx->h_sel, ctx->sel.p, sizeof(SelectOut), cudaMemcpyDeviceToHost, s));
    ctx->launches += 2;
    HS_CUDA(cudaMemcpyAsync(hth, th, (size_t)mt * sizeof(float), cudaMemcpyDeviceToHost, s));
    HS_CUDA(cudaMemcpyAsync(hres, ctx->sres.d(0), (size_t)mt * sizeof(double), cudaMemcpyDeviceToHost, s));
    // info[0], info[1]: Jacobi status; info[2]: Cholesky status (bad);
    // info[6], info[7]: status of a Householder redo's geqrf, orgqr
    HS_CUDA(cudaMemcpyAsync(hstat, ctx->info.p, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
    HS_CUDA(cudaStreamSynchronize(s));
    const int hbad = hstat[2];
    if (hstat[6] != 0 || hstat[7] != 0) {  // a Householder redo reported an error: fall back
      *reason = 4;
      return HS_OK;
    }
    if (hbad && tc && ctx->sx_save_valid && it + 1 < kMaxIt) {
      // the last Cholesky-QR broke down (the filtered rows were numerically
      // dependent): this round ran on a broken basis. Orthonormalise the
      // rows it started from by Householder QR and run the round again.
      // (Tensor-core products only: with FP64 products the fallback's FP32
      // eigenvectors with two FP64 Loewdin steps are the more accurate
      // projector, and that mode is about accuracy)
      HS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
      HS_TRY(orthonormalise_rows_qr(ctx, ctx->sx_save.d(), m, n, ctx->sx.d(0)));
      ctx->sx_save_valid = false;
      ctx->qr_redos += 1;
      prev_worst = INFINITY;
      continue;
    }
    *reason = hbad ? 4 : 7;
    if (hbad || hstat[0] || hstat[1]) return HS_OK;  // fall back
    // the states the selection can keep: the chi largest |theta| across both
    // blocks, plus two more per block; all of them must have converged, and no
    // block may keep states near the edge of its subspace
    std::vector<std::pair<double, int>> cand;
    double tmax = 0.0;
    for (int i = 0; i < m[0] + m[1]; ++i) {
      cand.push_back({std::fabs((double)hth[i]), i});
      tmax = std::max(tmax, std::fabs((double)hth[i]));
    }
    std::sort(cand.begin(), cand.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    const int keep = std::min(chi, m[0] + m[1]);
    int kept[2] = {0, 0};
    bool ok = tmax > 0.0;
    double worst = 0.0;
    for (int r = 0; r < (int)cand.size() && r < keep + 4; ++r) {
      const int i = cand[r].second, b = i >= m[0] ? 1 : 0;
      if (r < keep) ++kept[b];
      worst = std::max(worst, tmax > 0.0 ? hres[i] / tmax : 1.0);
    }
    *resid = worst;
    *reason = 5;
    if (it == 0) {
      ctx->prev_first_resid = worst;
      ctx->prev_spec_env = env;
    }
    // the residual cannot go below the rounding of the products H X (the
    // tensor-core products carry about 2^-22 of each term; at D = 6 the floor
    // is 2e-6, at D = 7, n ~ 4800, 1e-5..3e-5): a round that has stalled
    // there (less than a factor 2 better than the previous round, within
    // kFloorMax) is accepted as converged, and the floor it found serves as
    // the tolerance of the next moves (times kFloorMargin)
    // (tensor-core products only: with FP64 products the floor lies below kTol)
    const double kFloorMax = tc ? 10.0 * kTol : kTol, kFloorMargin = 1.5;
    const double accept = std::max(tol_move, std::min(kFloorMax, kFloorMargin * ctx->resid_floor));
    bool at_floor = false;
    if (worst > accept) {
      ok = false;
      if (it >= 1 && worst <= kFloorMax && worst > 0.5 * prev_worst) ok = at_floor = true;
    }
    for (int b = 0; b < 2; ++b)
      if (m[b] < n[b] && kept[b] > m[b] - oversample(ctx->ws_k[b]) / 2) {
        ok = false;
        *reason = 6;
      }
    if (ok && at_floor) ctx->resid_floor = worst;
    if (ok && worst <= tol_move) ctx->resid_floor = 0.0;  // below the tolerance again: no floor in the way
    if (ok) {
      *reason = 0;
      for (int b = 0; b < 2; ++b) m_out[b] = m[b];
      ctx->sel_ready = true;  // w, the selection and its host copy are this round's
      *done = true;
      return HS_OK;
    }
    if (it + 1 == kMaxIt) return HS_OK;  // fall back
    // hopeless attempts (far from tolerance and not closing in fast) fall back early
    if (it >= 1 && worst > 30.0 * kTol && worst > 0.5 * prev_worst) return HS_OK;
    prev_worst = worst;
    if (tc) {
      // next basis: Chebyshev-filtered steps, both blocks per launch
      HS_TRY(cheb_filter_pair(ctx, prec, m, n, hth, kept));
      for (int b = 0; b < 2; ++b)
        if (m[b] > 0) HS_CUDA(launch_row_normalize(ctx->sx.d(b), m[b], n[b], s));
    } else {
      for (int b = 0; b < 2; ++b)
        if (m[b] > 0) {
          // next basis: a Chebyshev-filtered step where possible, else a plain
          // power step (rows of Zr = theta_i x_i + residual)
          bool filtered = false;
          HS_TRY(cheb_filter_block(ctx, prec, b, m[b], n[b], H[b], hth + (b ? m[0] : 0), kept[b], ctx->sx.d(b),
                                   &filtered));
          if (!filtered)
            HS_CUDA(cudaMemcpyAsync(ctx->sx.d(b), ctx->szr.d(b), (size_t)m[b] * n[b] * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
          HS_CUDA(launch_row_normalize(ctx->sx.d(b), m[b], n[b], s));
        }
    }
    {
      // far from convergence the rows can be far from orthogonal (the Loewdin
      // iteration alone diverges there): Cholesky-QR first, its input kept in
      // case it breaks down
      HS_TRY(ctx->sx_save.ensure((size_t)(mn0 + mn1 + 2) * sizeof(double)));
      HS_CUDA(cudaMemcpyAsync(ctx->sx_save.d(), ctx->sx.d(0), (size_t)(mn0 + mn1) * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
      ctx->sx_save_valid = ctx->sx.d(1) == ctx->sx.d(0) + mn0;
      double* const Xo[2] = {ctx->sx.d(0), ctx->sx.d(1)};
      double* const Xco[2] = {ctx->sxc.d(0), ctx->sxc.d(1)};
      HS_TRY(orthonormalise_rows(ctx, prec, Xo, m, n, Xco, bad));
    }
  }
  return HS_OK;
}

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
  if (cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cusolverDnCreate(&c->solver2) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnSetStream(c->solver2, c->stream2) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnCreateParams(&c->params2) != CUSOLVER_STATUS_SUCCESS) {
    cudaGetLastError();
    hs_destroy(c);
    return fail(HS_ERR_SOLVER, "second solver initialisation failed");
  }
  if (cublasCreate(&c->blas) != CUBLAS_STATUS_SUCCESS ||
      cublasSetStream(c->blas, c->stream) != CUBLAS_STATUS_SUCCESS ||
      cublasSetMathMode(c->blas, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS) {
    hs_destroy(c);
    return fail(HS_ERR_SOLVER, "cuBLAS initialisation failed");
  }
  if (cudaMallocHost(&c->h_sel, sizeof(SelectOut)) != cudaSuccess ||
      cudaMallocHost(&c->h_info, 8 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->h_tc_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    hs_destroy(c);
    return fail(HS_ERR_CUDA, "pinned allocation failed");
  }
  hs_status st;
  if ((st = c->sel.ensure(sizeof(SelectOut))) != HS_OK || (st = c->info.ensure(8 * sizeof(int))) != HS_OK ||
      (st = c->scratch.ensure(64)) != HS_OK || (st = c->tc_err.ensure(64)) != HS_OK) {
    hs_destroy(c);
    return st;
  }
  if (cudaMemset(c->tc_err.p, 0, 64) != cudaSuccess) {
    hs_destroy(c);
    return fail(HS_ERR_CUDA, "cudaMemset failed");
  }
  *out = c;
  return HS_OK;
}

hs_status hs_destroy(hs_ctx ctx) {
  if (!ctx) return HS_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  DBuf* bufs[] = {&ctx->big1,    &ctx->big2,    &ctx->x1,      &ctx->pt,      &ctx->pp,
                  &ctx->w,       &ctx->lam,     &ctx->idx,     &ctx->sel,     &ctx->scratch,
                  &ctx->info,    &ctx->solver_dev, &ctx->tc_a_hi, &ctx->tc_a_lo, &ctx->tc_x_hi,
                  &ctx->tc_x_lo, &ctx->tc_b_hi, &ctx->tc_b_lo, &ctx->tc_err};
  for (DBuf* b : bufs) b->release();
  for (DBuf& b : ctx->r) b.release();
  for (DBuf& b : ctx->hb) b.release();
  for (DBuf& b : ctx->gb) b.release();
  for (DBuf& b : ctx->zr) b.release();
  for (DBuf& b : ctx->zd) b.release();
  for (DBuf& b : ctx->d4) b.release();
  for (DBuf* b : {&ctx->pt_prev, &ctx->ovl, &ctx->ovl_idx, &ctx->ovl_sgn, &ctx->pt_tmp, &ctx->sx_save}) b->release();
  ctx->h_ovl.release();
  ctx->d4_h.release();
  if (ctx->gesvdj) cusolverDnDestroyGesvdjInfo(ctx->gesvdj);
  ctx->ga.release();
  ctx->ps_hi.release();
  ctx->ps_lo.release();
  DBuf* more[] = {&ctx->c32,  &ctx->w32,   &ctx->pcol,         &ctx->pt2,   &ctx->gram,
                  &ctx->wproj, &ctx->solver32_dev, &ctx->splitk, &ctx->ws_pt, &ctx->sth,
                  &ctx->sx_hi, &ctx->sx_lo, &ctx->sy_hi, &ctx->sy_lo, &ctx->schol};
  for (Stacked* t : {&ctx->sx, &ctx->sz, &ctx->sxc, &ctx->szc, &ctx->sxr, &ctx->szr, &ctx->sbm, &ctx->sbw, &ctx->sres})
    t->release();
  ctx->sH_hi.release();
  ctx->sH_lo.release();
  for (auto* t : {&ctx->sf_y[0], &ctx->sf_y[1], &ctx->sf_y[2], &ctx->sf_z, &ctx->sf_t, &ctx->sf_s, &ctx->sf_q,
                  &ctx->sf_qt, &ctx->sf_idx, &ctx->sf_xl, &ctx->sf_qh, &ctx->sf_ql, &ctx->sf_qth, &ctx->sf_qtl})
    t->release();
  for (DBuf* b : more) b->release();
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  if (ctx->h_sel) cudaFreeHost(ctx->h_sel);
  if (ctx->h_info) cudaFreeHost(ctx->h_info);
  if (ctx->h_tc_err) cudaFreeHost(ctx->h_tc_err);
  ctx->h_sub.release();
  ctx->h_idx.release();
  if (ctx->stream2) cudaStreamSynchronize(ctx->stream2);
  DBuf* s2b[] = {&ctx->solver2_dev, &ctx->solver2_32_dev};
  for (DBuf* b : s2b) b->release();
  if (ctx->params2) cusolverDnDestroyParams(ctx->params2);
  if (ctx->solver2) cusolverDnDestroy(ctx->solver2);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->stream2) cudaStreamDestroy(ctx->stream2);
  if (ctx->params) cusolverDnDestroyParams(ctx->params);
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  if (ctx->blas) cublasDestroy(ctx->blas);
  delete ctx;
  return HS_OK;
}

hs_status hs_sync(hs_ctx ctx) {
  HS_TRY(check_ctx(ctx));
  HS_CUDA(cudaMemcpyAsync(ctx->h_tc_err, ctx->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HS_CUDA(cudaStreamSynchronize(ctx->stream));
  if (*ctx->h_tc_err != 0) {
    const int code = *ctx->h_tc_err;
    HS_CUDA(cudaMemsetAsync(ctx->tc_err.p, 0, sizeof(int), ctx->stream));
    return fail(HS_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM gave up (code %d)", code);
  }
  return HS_OK;
}

size_t hs_z2_tensor_bytes(int D, hs_basis basis, hs_dtype dtype) {
  if (D <= 0) return 0;
  if (dtype == HS_C128) return basis == HS_BASIS_HERMITIAN ? graded_tensor_bytes(D) : zdense_tensor_bytes(D);
  if (dtype != HS_F64) return 0;
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
  out->v_even = out->h_even = q.n[0];
  out->v_odd = out->h_odd = q.n[1];
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
  if (dtype != HS_F64 && dtype != HS_C128) return fail(HS_ERR_DTYPE, "unknown dtype");
  if (basis != HS_BASIS_DENSE && basis != HS_BASIS_HERMITIAN)
    return fail(HS_ERR_INVALID_ARG, "unknown basis");
  const size_t need = hs_z2_tensor_bytes(D, basis, dtype);
  if (out->capacity_bytes < need)
    return fail(HS_ERR_WORKSPACE, "output holds %zu bytes, %zu needed", out->capacity_bytes, need);
  if (dtype == HS_C128 && basis == HS_BASIS_HERMITIAN)
    HS_TRY(graded_double_layer(ctx, A, d, D, out));
  else if (dtype == HS_C128)
    HS_TRY(zdense_double_layer(ctx, A, d, D, out));
  else
    HS_CUDA(launch_double_layer_blocks(A, d, D, basis == HS_BASIS_HERMITIAN, out->data, ctx->stream));
  const Sect q = q_sect(D, basis);
  out->D = D;
  out->n_even = q.n[0];
  out->n_odd = q.n[1];
  out->v_even = out->h_even = q.n[0];
  out->v_odd = out->h_odd = q.n[1];
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

hs_status hs_selftest_bounded_wait(hs_ctx ctx, long long limit, int* result) {
  HS_TRY(check_ctx(ctx));
  if (!result || limit < 1) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  HS_TRY(ctx->info.ensure(8 * sizeof(int)));
  int* d = static_cast<int*>(ctx->info.p);
  HS_CUDA(launch_wait_selftest(limit, d, ctx->stream));
  HS_CUDA(cudaMemcpyAsync(result, d, 7 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HS_CUDA(cudaStreamSynchronize(ctx->stream));
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
  if (precision != HS_PREC_F64 && precision != HS_PREC_TF32X3 && precision != HS_PREC_TF32 &&
      precision != HS_PREC_BF16X3)
    return fail(HS_ERR_INVALID_ARG, "unknown precision %d", (int)precision);
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
  env->eig_mode = HS_EIG_F64;
  env->dtype = a->dtype;
  ctx->ws_valid = false;  // no warm start for the subspace eigensolver yet
  ctx->prev_first_resid = 0.0;
  ctx->resid_floor = 0.0;
  ctx->pt_prev_valid = false;
  if (a->dtype == HS_C128) return herm ? graded_init(ctx, a, chi_max, env) : zdense_init(ctx, a, chi_max, env);
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
  if (precision != HS_PREC_F64) {
    // split, padded copy of the double layer: the B operand of both a-GEMMs
    const int pad = tc_pad(precision), eb = tc_elem_bytes(precision);
    const Z2Mat Am = mat(fused2(qs, qs), fused2(qs, qs)), Amp = mat(fused2(qs, qs), fused2(qs, qs), pad);
    const size_t nb = (size_t)z2_elems(Amp) * eb;
    HS_TRY(ctx->tc_a_hi.ensure(nb));
    HS_TRY(ctx->tc_a_lo.ensure(nb));
    HS_CUDA(cudaMemsetAsync(ctx->tc_a_hi.p, 0, nb, ctx->stream));
    HS_CUDA(cudaMemsetAsync(ctx->tc_a_lo.p, 0, nb, ctx->stream));
    const int ident[kMaxLegs] = {0, 1, 2, 3, 0, 0};
    HS_CUDA(launch_permute_split(make_perm_plan(Am, Amp, ident), a->data, ctx->tc_a_hi.p, ctx->tc_a_lo.p,
                                 tc_mode(precision), ctx->stream));
    ctx->tc_a_src = a->data;
    ctx->tc_a_prec = precision;
    const size_t xb = (c * c * ((size_t)q * q + pad)) * eb;
    HS_TRY(ctx->tc_x_hi.ensure(xb));
    HS_TRY(ctx->tc_x_lo.ensure(xb));
  }
  return HS_OK;
}

hs_status hs_ctmrg_move(hs_ctx ctx, const hs_z2_tensor* a, hs_env* env, int chi,
                        hs_move_info* info) {
  HS_TRY(check_ctx(ctx));
  if (!a || !env || !a->data) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (a->D != env->D || a->basis != env->basis)
    return fail(HS_ERR_SHAPE, "tensor and environment disagree on D or basis");
  if (chi < 1 || chi > env->chi_max) return fail(HS_ERR_SHAPE, "chi %d outside [1, %d]", chi, env->chi_max);
  if (env->dtype != a->dtype) return fail(HS_ERR_DTYPE, "tensor and environment disagree on dtype");
  if (env->dtype == HS_C128)
    return env->basis == HS_BASIS_DENSE ? zdense_move(ctx, a, env, chi, info) : graded_move(ctx, a, env, chi, info);
  cudaStream_t s = ctx->stream;
  const hs_gemm_backend be = env->gemm_backend;
  const bool tc = env->precision != HS_PREC_F64;
  ctx->sH_fresh = false;
  ctx->sel_ready = false;
  // with tensor-core GEMMs the corner chain stays in FP32 (the accumulators'
  // values, so nothing is lost), except for the FP64 eigensolver
  ctx->cp_f32 = tc && env->eig_mode != HS_EIG_F64;
  const bool f32c = ctx->cp_f32;
  if (tc && (ctx->tc_a_src != a->data || ctx->tc_a_prec != (int)env->precision))
    return fail(HS_ERR_INVALID_ARG, "the double layer changed since hs_ctmrg_init (tensor-core copy is stale)");
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
  ctx->phase_flops[tc ? HS_PHASE_GEMM_TC : HS_PHASE_GEMM] += gemm_flops(g1) + gemm_flops(g2) + gemm_flops(g3);
  if (!tc) {
    PhaseScope ps(ctx, HS_PHASE_GEMM);
    HS_TRY(gemm(ctx, be, g1, env->T, env->C, ctx->x1.d()));
    HS_TRY(gemm(ctx, be, g2, ctx->x1.d(), env->T, B1));
  } else {
    // the split edge serves as A of G1, B of G2 here and B of G4 below; the
    // corner (symmetric) is its own K-major B operand
    HS_TRY(tc_split(ctx, env->precision, Tcr, Tcr, {0, 1, 2}, env->T, ctx->tc_b_hi, ctx->tc_b_lo));
    HS_TRY(tc_split(ctx, env->precision, Cm, Cm, {0, 1}, env->C, ctx->sy_hi, ctx->sy_lo));
    HS_TRY(tc_run(ctx, env->precision, Tcr, ctx->tc_b_hi, ctx->tc_b_lo, Cm, ctx->sy_hi, ctx->sy_lo, X1,
                  ctx->x1.d()));
    HS_TRY(tc_split(ctx, env->precision, X1, X1, {0, 1, 2}, ctx->x1.d(), ctx->tc_x_hi, ctx->tc_x_lo));
    if (f32c) {
      // X2 goes straight from G2's accumulators into the permuted split A of G3
      HS_TRY(tc_run_split(ctx, env->precision, X1, ctx->tc_x_hi, ctx->tc_x_lo, Tcr, ctx->tc_b_hi, ctx->tc_b_lo, X2,
                          X2p, {0, 2, 3, 1}, ctx->ps_hi, ctx->ps_lo, reinterpret_cast<float*>(B1)));
    } else {
      HS_TRY(tc_run(ctx, env->precision, X1, ctx->tc_x_hi, ctx->tc_x_lo, Tcr, ctx->tc_b_hi, ctx->tc_b_lo, X2, B1));
    }
  }
  // C' = X3 with legs (a,e,d,r) -> (a,d,e,r). With the subspace solver and
  // tensor cores, G3 writes X3 straight into the split C' operand; the FP32
  // C' itself is formed (from that split) only when a fallback eigensolver
  // needs it
  const bool subspace_mode = env->eig_mode == HS_EIG_SUBSPACE || env->eig_mode == HS_EIG_SUBSPACE_ADAPTIVE;
  const bool cp_fused = f32c && subspace_mode;
  // the split C' is TF32x3 (FP32 pairs): a fallback joins it; a BF16x3 split
  // went through X3 in B1
  const bool cp_join = cp_fused && tc_elem_bytes(env->precision) == 4;
  if (cp_fused) {
    HS_TRY(tc_run_split(ctx, env->precision, X2p, ctx->ps_hi, ctx->ps_lo, Am, ctx->tc_a_hi, ctx->tc_a_lo, X3, Cp,
                        {0, 2, 1, 3}, ctx->sH_hi, ctx->sH_lo, reinterpret_cast<float*>(B1)));
    ctx->sH_n[0] = (int)z2_rows(Cp, 0);
    ctx->sH_n[1] = (int)z2_rows(Cp, 1);
    ctx->sH_fresh = true;
  } else if (tc && f32c) {
    HS_TRY(tc_run(ctx, env->precision, X2p, ctx->ps_hi, ctx->ps_lo, Am, ctx->tc_a_hi, ctx->tc_a_lo, X3, B1, true));
  } else if (tc) {
    HS_TRY(tc_a_gemm(ctx, env->precision, X2, X2p, {0, 2, 3, 1}, B1, Am, X3, B2, false));
    std::swap(B1, B2);  // X3 now in B1, as on the FP64 path
  } else {
    {
      PhaseScope ps(ctx, HS_PHASE_PERMUTE);
      HS_TRY(permute(ctx, X2, X2p, {0, 2, 3, 1}, B1, B2));  // (a,x,e,y) -> (a,e,y,x)
    }
    PhaseScope ps(ctx, HS_PHASE_GEMM);
    HS_TRY(gemm(ctx, be, g3, B2, a->data, B1));
  }
  bool cp_ready = false;
  auto form_corner = [&]() -> hs_status {
    if (cp_ready) return HS_OK;
    PhaseScope ps(ctx, HS_PHASE_PERMUTE);
    if (cp_join) {
      const Z2Mat Pc = mat(Cp.r, Cp.c, tc_pad(env->precision));
      HS_CUDA(launch_join_split_f32(ctx->sH_hi.p, ctx->sH_lo.p, z2_rows(Pc, 0), z2_cols(Pc, 0), z2_ld(Pc, 0),
                                    z2_block_off(Pc, 1), z2_rows(Pc, 1), z2_cols(Pc, 1), z2_ld(Pc, 1),
                                    reinterpret_cast<float*>(B2), s));
      ctx->launches += 1;
    } else if (f32c) {
      const int pm[kMaxLegs] = {0, 2, 1, 3, 0, 0};
      HS_CUDA(launch_permute_f32(cached_plan(ctx, X3, Cp, pm), reinterpret_cast<const float*>(B1),
                                 reinterpret_cast<float*>(B2), s));
      ctx->launches += 1;
    } else {
      HS_TRY(permute(ctx, X3, Cp, {0, 2, 1, 3}, B1, B2));
    }
    cp_ready = true;
    return HS_OK;
  };
  if (!cp_fused) HS_TRY(form_corner());

  // one eigen-decomposition per parity block (C' blocks stacked in B2: FP32
  // values when f32c, else FP64)
  const int n0 = (int)z2_rows(Cp, 0), n1 = (int)z2_rows(Cp, 1);
  double* V0 = B2;
  double* V1 = f32c ? reinterpret_cast<double*>(reinterpret_cast<float*>(B2) + (long long)n0 * n0)
                    : B2 + (long long)n0 * n0;
  double* w0 = ctx->w.d();
  double* w1 = w0 + n0;
  HS_CUDA(cudaMemsetAsync(ctx->info.p, 0, 2 * sizeof(int), s));
  if (env->eig_mode != HS_EIG_F64 && env->eig_mode != HS_EIG_F32_PROJECTED && !subspace_mode)
    return fail(HS_ERR_INVALID_ARG, "unknown eig mode");
  // subspace eigensolver first (when a warm start exists); its Ritz values
  // replace the spectra, ns0/ns1 are the sizes passed to the selection
  bool sub_done = false;
  int sub_iters = 0, ns0 = n0, ns1 = n1, sub_reason = -1;
  double sub_resid = 0.0;
  if (subspace_mode) {
    int msub[2] = {0, 0};
    HS_TRY(subspace_projector(ctx, env, chi, n0, n1, V0, V1, w0, msub, &sub_done, &sub_iters, &flops, &sub_reason,
                              &sub_resid));
    if (sub_done) {
      ns0 = msub[0];
      ns1 = msub[1];
      w1 = w0 + ns0;
    }
  }
  const bool f32eig = env->eig_mode == HS_EIG_F32_PROJECTED || (subspace_mode && !sub_done);
  float* V0f = nullptr;
  float* V1f = nullptr;
  if (sub_done) {
    // Ritz pairs ready
  } else if (!f32eig) {
    PhaseScope ps(ctx, HS_PHASE_EIG);
    HS_TRY(eig_pair(ctx, false, V0, n0, w0, V1, n1, w1));
  } else {
    const long long nn = (long long)n0 * n0 + (long long)n1 * n1;
    HS_TRY(ctx->c32.ensure(nn * sizeof(float)));
    HS_TRY(ctx->w32.ensure((size_t)(n0 + n1) * sizeof(float)));
    HS_TRY(eig32_workspace(ctx, n0 > n1 ? n0 : n1));
    V0f = static_cast<float*>(ctx->c32.p);
    V1f = V0f + (long long)n0 * n0;
    float* w32 = static_cast<float*>(ctx->w32.p);
    PhaseScope ps(ctx, HS_PHASE_EIG);
    HS_TRY(form_corner());
    if (f32c)
      HS_CUDA(cudaMemcpyAsync(V0f, V0, nn * sizeof(float), cudaMemcpyDeviceToDevice, s));
    else
      HS_CUDA(launch_cast_f64_f32(V0, V0f, nn, s));
    HS_TRY(eig_pair(ctx, true, V0f, n0, w32, V1f, n1, w32 + n0));
    HS_CUDA(launch_cast_f32_f64(w32, w0, n0 + n1, s));
    ctx->launches += 2;
  }
  SelectOut* dsel = static_cast<SelectOut*>(ctx->sel.p);
  int* didx = static_cast<int*>(ctx->idx.p);
  if (!(sub_done && ctx->sel_ready)) {
    // (a converged subspace round has issued the selection and read it back)
    {
      PhaseScope ps(ctx, HS_PHASE_SELECT);
      HS_CUDA(launch_select(w0, ns0, w1, ns1, chi, didx, ctx->lam.d(), dsel, s));
      ctx->launches += 1;
    }
    HS_CUDA(cudaMemcpyAsync(ctx->h_sel, dsel, sizeof(SelectOut), cudaMemcpyDeviceToHost, s));
    HS_CUDA(cudaMemcpyAsync(ctx->h_info, ctx->info.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    HS_CUDA(cudaStreamSynchronize(s));
    if (ctx->h_info[0] != 0 || ctx->h_info[1] != 0)
      return fail(HS_ERR_SOLVER, "syevd info = (%d, %d)", ctx->h_info[0], ctx->h_info[1]);
  }
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
  const Z2Mat Zpq = mat(fused2(cn, q), fused2(q, c)), PTq = mat(fused1(cn), fused2(q, c));
  if (sub_done) {
    const long long npt = (long long)cn.n[0] * n0 + (long long)cn.n[1] * n1;
    HS_TRY(ctx->pcol.ensure(npt * sizeof(double)));
    {
      PhaseScope ps(ctx, HS_PHASE_SELECT);
      HS_CUDA(launch_gather_rows(ctx->sxr.d(0), n0, ctx->sxr.d(1), n1, didx, chi, dsel, ctx->pt.d(),
                                 ctx->pcol.d(), s));
      ctx->launches += 1;
    }
    // a poor warm start (this move's first round far from converged) means
    // the boundary gauge moved: order the kept rows like the previous move's
    const int kk[2] = {cn.n[0], cn.n[1]}, nn[2] = {n0, n1};
    bool aligned = false;
    if (ctx->pt_prev_valid && ctx->pt_prev_k[0] == kk[0] && ctx->pt_prev_k[1] == kk[1] &&
        ctx->pt_prev_n[0] == n0 && ctx->pt_prev_n[1] == n1 && ctx->prev_first_resid > 1e-3) {
      // canonical signs first (the rows no previous row matches keep them)
      HS_CUDA(launch_row_sign_pair(ctx->pt.d(), kk[0], n0, kk[1], n1, s));
      ctx->launches += 1;
      int moved = 0;
      HS_TRY(align_kept_rows(ctx, kk, nn, &moved));
      aligned = true;
    }
    // converged Ritz vectors are orthonormal to ~1e-6 (FP32 Rayleigh-Ritz):
    // one FP64 Loewdin step brings them to ~1e-12
    HS_TRY(finish_projector(ctx, n0, n1, dsel, c, q, cn, V0, V1, env, &flops, 1, !aligned));
    HS_TRY(keep_pt(ctx, kk, nn));
  } else if (!f32eig) {
    PhaseScope ps(ctx, HS_PHASE_SELECT);
    HS_CUDA(launch_gather_pt(V0, n0, V1, n1, didx, chi, dsel, ctx->pt.d(), s));
    ctx->launches += 1;
  } else {
    HS_TRY(project_f32(ctx, V0f, n0, V1f, n1, didx, chi, dsel, c, q, cn, V0, V1, env, &flops));
    const int kk[2] = {cn.n[0], cn.n[1]}, nn[2] = {n0, n1};
    HS_TRY(keep_pt(ctx, kk, nn));
  }
  if (subspace_mode) {
    // the next move starts from the whole subspace of each block: the Ritz
    // vectors of this move, or after a fallback the m largest-|lambda| FP32
    // eigenvectors, m = kept + 24 (at most the block size)
    int mnext[2];
    for (int b = 0; b < 2; ++b) {
      const int nb = b ? n1 : n0;
      mnext[b] = std::min(std::min(cn.n[b] + oversample(cn.n[b]), nb), max_subspace());
      if (sub_done) mnext[b] = b ? ns1 : ns0;
    }
    const long long nws = (long long)mnext[0] * n0 + (long long)mnext[1] * n1;
    HS_TRY(ctx->ws_pt.ensure((nws + 1) * sizeof(double)));
    HS_TRY(ctx->sf_idx.ensure(((size_t)mnext[0] + mnext[1] + 1) * sizeof(int)));
    double* dst[2] = {ctx->ws_pt.d(), ctx->ws_pt.d() + (long long)mnext[0] * n0};
    if (sub_done) {
      // the Ritz vectors, stacked exactly as the warm start wants them
      HS_CUDA(cudaMemcpyAsync(dst[0], ctx->sxr.d(0), (size_t)nws * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else if (f32eig) {
      for (int b = 0; b < 2; ++b) {
        const int nb = b ? n1 : n0;
        if (mnext[b] == 0) continue;
        const float* wb = static_cast<float*>(ctx->w32.p) + (b ? n0 : 0);
        HS_CUDA(launch_top_rows(wb, b ? V1f : V0f, nb, mnext[b], static_cast<int*>(ctx->sf_idx.p), dst[b], s));
      }
    }
    ctx->ws_env = env;
    ctx->ws_valid = sub_done || f32eig;
    ctx->ws_c[0] = c.n[0];
    ctx->ws_c[1] = c.n[1];
    ctx->ws_k[0] = cn.n[0];
    ctx->ws_k[1] = cn.n[1];
    ctx->ws_m[0] = mnext[0];
    ctx->ws_m[1] = mnext[1];
    ctx->ws_n[0] = n0;
    ctx->ws_n[1] = n1;
    ctx->ws_moves += 1;
  }
  GemmGroup g4 = make_z2_gemm(Pp, Tcr, Y), g5 = make_z2_gemm(Yp, Am, Zm), g6 = make_z2_gemm(Zp, PT, Tn);
  flops += gemm_flops(g4) + gemm_flops(g5) + gemm_flops(g6);
  ctx->phase_flops[tc ? HS_PHASE_GEMM_TC : HS_PHASE_GEMM] += gemm_flops(g4) + gemm_flops(g5) + gemm_flops(g6);
  {
    PhaseScope ps(ctx, HS_PHASE_PERMUTE);
    HS_TRY(permute(ctx, PT, Pp, {2, 0, 1}, ctx->pt.d(), ctx->pp.d()));  // (a',a,d) -> (d,a',a)
  }
  if (!tc) {
    {
      PhaseScope ps(ctx, HS_PHASE_GEMM);
      HS_TRY(gemm(ctx, be, g4, ctx->pp.d(), env->T, B1));
    }
    {
      PhaseScope ps(ctx, HS_PHASE_PERMUTE);
      HS_TRY(permute(ctx, Y, Yp, {1, 2, 0, 3}, B1, B2));  // (d,a',b,x) -> (a',b,d,x)
    }
    {
      PhaseScope ps(ctx, HS_PHASE_GEMM);
      HS_TRY(gemm(ctx, be, g5, B2, a->data, B1));
    }
    {
      PhaseScope ps(ctx, HS_PHASE_PERMUTE);
      HS_TRY(permute(ctx, Zm, Zp, {0, 3, 1, 2}, B1, B2));  // (a',b,u,r) -> (a',r,b,u)
    }
    PhaseScope ps(ctx, HS_PHASE_GEMM);
    HS_TRY(gemm(ctx, be, g6, B2, ctx->pt.d(), env->T));
  } else {
    HS_TRY(tc_split(ctx, env->precision, Pp, Pp, {0, 1, 2}, ctx->pp.d(), ctx->tc_x_hi, ctx->tc_x_lo));
    // Y and Z only feed the next GEMM: the epilogues of G4 and G5 write them
    // as its permuted split A operand. Z's contraction legs (b,u) are taken
    // in the order (u,b) (PT's columns alike), so that its destination runs
    // along the rows of G5's output
    HS_TRY(tc_run_split(ctx, env->precision, Pp, ctx->tc_x_hi, ctx->tc_x_lo, Tcr, ctx->tc_b_hi, ctx->tc_b_lo, Y, Yp,
                        {1, 2, 0, 3}, ctx->ps_hi, ctx->ps_lo, reinterpret_cast<float*>(B1)));
    HS_TRY(tc_run_split(ctx, env->precision, Yp, ctx->ps_hi, ctx->ps_lo, Am, ctx->tc_a_hi, ctx->tc_a_lo, Zm, Zpq,
                        {0, 3, 2, 1}, ctx->tc_x_hi, ctx->tc_x_lo, reinterpret_cast<float*>(B1)));
    HS_TRY(tc_split(ctx, env->precision, PT, PTq, {0, 2, 1}, ctx->pt.d(), ctx->tc_b_hi, ctx->tc_b_lo));
    HS_TRY(tc_run(ctx, env->precision, Zpq, ctx->tc_x_hi, ctx->tc_x_lo, PTq, ctx->tc_b_hi, ctx->tc_b_lo, Tn, env->T));
  }

  // C <- diag(lambda)/max|lambda|, T <- T/max|T|
  if (!f32eig && !sub_done) {
    PhaseScope ps(ctx, HS_PHASE_SELECT);
    HS_CUDA(launch_diag_corner(ctx->lam.d(), cn.n[0], cn.n[1], dsel, env->C, s));
    ctx->launches += 1;
  }
  {
    PhaseScope ps(ctx, HS_PHASE_NORMALIZE);
    HS_CUDA(launch_normalize_max(env->T, z2_elems(Tn), static_cast<unsigned long long*>(ctx->scratch.p),
                                 dsel, s));
    ctx->launches += 2;
  }
  HS_CUDA(cudaMemcpyAsync(&ctx->h_sel->log_norm_C, &dsel->log_norm_C, 2 * sizeof(double),
                          cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaMemcpyAsync(ctx->h_tc_err, ctx->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  harvest_profile(ctx);
  if (*ctx->h_tc_err != 0) {
    const int code = *ctx->h_tc_err;
    HS_CUDA(cudaMemsetAsync(ctx->tc_err.p, 0, sizeof(int), s));
    return fail(HS_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM gave up (code %d)", code);
  }
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
    info->flags = ((discarded && info->gap < 1e-9) ? 1 : 0) |
                  (subspace_mode ? (sub_done ? 2 : 4) : 0);
    info->subspace_iters = sub_iters;
    info->subspace_reason = sub_reason;
    info->subspace_resid = sub_resid;
  }
  return HS_OK;
}

hs_status hs_profile_enable(hs_ctx ctx, int enable) {
  HS_TRY(check_ctx(ctx));
  HS_CUDA(cudaStreamSynchronize(ctx->stream));
  harvest_profile(ctx);
  ctx->prof = enable != 0;
  for (double& v : ctx->phase_ms) v = 0;
  for (double& v : ctx->phase_flops) v = 0;
  ctx->launches = 0;
  return HS_OK;
}

hs_status hs_profile_phases(hs_ctx ctx, unsigned mask) {
  HS_TRY(check_ctx(ctx));
  ctx->prof_mask = mask;
  return HS_OK;
}

hs_status hs_profile_read(hs_ctx ctx, double* phase_ms, double* phase_flops, int n_phases,
                          long long* launches) {
  HS_TRY(check_ctx(ctx));
  if (n_phases < 0) return fail(HS_ERR_INVALID_ARG, "negative phase count");
  for (int i = 0; i < n_phases; ++i) {
    if (phase_ms) phase_ms[i] = i < HS_PHASE_COUNT ? ctx->phase_ms[i] : 0.0;
    if (phase_flops) phase_flops[i] = i < HS_PHASE_COUNT ? ctx->phase_flops[i] : 0.0;
  }
  if (launches) *launches = ctx->launches;
  return HS_OK;
}

hs_status hs_gemm(hs_ctx ctx, hs_precision precision, int M, int N, int K, const double* A, int lda,
                  const double* B, int ldb, double* C, int ldc) {
  HS_TRY(check_ctx(ctx));
  if (M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < N || (M > 0 && N > 0 && (!A || !B || !C)))
    return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (M == 0 || N == 0) return HS_OK;
  if (precision == HS_PREC_F64) {
    GemmGroup g{};
    g.n = 1;
    g.p[0] = GemmProblem{M, N, K, lda, ldb, ldc, 0, 0, 0};
    HS_CUDA(launch_gemm_f64(g, A, B, C, 1.0, ctx->stream));
    return HS_OK;
  }
  if (precision != HS_PREC_TF32X3 && precision != HS_PREC_TF32 && precision != HS_PREC_BF16X3)
    return fail(HS_ERR_INVALID_ARG, "unknown precision %d", (int)precision);
  if (K == 0) {
    HS_CUDA(cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * N, M, ctx->stream));
    return HS_OK;
  }
  const int pad = tc_pad(precision), eb = tc_elem_bytes(precision);
  const long long Kp = ((long long)K + pad - 1) / pad * pad;
  HS_TRY(ctx->tc_x_hi.ensure((size_t)M * Kp * eb));
  HS_TRY(ctx->tc_x_lo.ensure((size_t)M * Kp * eb));
  HS_TRY(ctx->tc_b_hi.ensure((size_t)N * Kp * eb));
  HS_TRY(ctx->tc_b_lo.ensure((size_t)N * Kp * eb));
  ctx->tc_x_hi.zkey = ctx->tc_x_lo.zkey = ctx->tc_b_hi.zkey = ctx->tc_b_lo.zkey = 0;
  HS_CUDA(launch_split_pad(A, M, K, lda, ctx->tc_x_hi.p, ctx->tc_x_lo.p, Kp, tc_mode(precision), ctx->stream));
  HS_CUDA(launch_split_pad(B, N, K, ldb, ctx->tc_b_hi.p, ctx->tc_b_lo.p, Kp, tc_mode(precision), ctx->stream));
  TcProblem t;
  t.M = M;
  t.N = N;
  t.Kp = (int)Kp;
  t.ldc = ldc;
  t.a_hi = ctx->tc_x_hi.p;
  t.a_lo = ctx->tc_x_lo.p;
  t.b_hi = ctx->tc_b_hi.p;
  t.b_lo = ctx->tc_b_lo.p;
  t.c = C;
  HS_CUDA(launch_gemm_tc(precision, &t, 1, static_cast<int*>(ctx->tc_err.p), ctx->stream));
  return HS_OK;
}

hs_status hs_env_to_dense(hs_ctx ctx, const hs_env* env, double* C_dense, double* T_dense) {
  HS_TRY(check_ctx(ctx));
  if (!env || !C_dense || !T_dense) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (env->dtype == HS_C128 && env->basis == HS_BASIS_DENSE) {
    // stored dense already (interleaved complex128)
    const size_t chi = (size_t)(env->chi_even + env->chi_odd), q = (size_t)env->D * env->D;
    HS_CUDA(cudaMemcpyAsync(C_dense, env->C, 2 * chi * chi * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    HS_CUDA(cudaMemcpyAsync(T_dense, env->T, 2 * chi * q * chi * sizeof(double), cudaMemcpyDeviceToDevice,
                            ctx->stream));
    return HS_OK;
  }
  if (env->dtype == HS_C128) {
    HS_CUDA(launch_env_to_dense_graded(env->C, env->T, env->D, env->chi_even, env->chi_odd, C_dense, T_dense,
                                       ctx->stream));
    return HS_OK;
  }
  HS_CUDA(launch_env_to_dense(env->C, env->T, env->D, env->chi_even, env->chi_odd,
                              env->basis == HS_BASIS_HERMITIAN, C_dense, T_dense, ctx->stream));
  return HS_OK;
}

}  // extern "C"

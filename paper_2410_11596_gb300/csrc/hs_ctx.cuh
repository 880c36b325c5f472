// Context of libhs and the helpers shared by the C-ABI translation units.
#pragma once

#include <cublas_v2.h>
#include <cusolverDn.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hs_internal.cuh"

namespace hs {

// Records the message of the last failure on this thread and returns st.
hs_status fail(hs_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
const char* last_error();

#define HS_CUDA(x)                                                                        \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess)                                                                \
      return ::hs::fail(HS_ERR_CUDA, "%s failed: %s (%s:%d)", #x, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                              \
  } while (0)
#define HS_SOLVER(x)                                                                      \
  do {                                                                                    \
    cusolverStatus_t e_ = (x);                                                            \
    if (e_ != CUSOLVER_STATUS_SUCCESS)                                                    \
      return ::hs::fail(HS_ERR_SOLVER, "%s failed: cusolver status %d (%s:%d)", #x, (int)e_, \
                        __FILE__, __LINE__);                                              \
  } while (0)
#define HS_BLAS(x)                                                                        \
  do {                                                                                    \
    cublasStatus_t e_ = (x);                                                              \
    if (e_ != CUBLAS_STATUS_SUCCESS)                                                      \
      return ::hs::fail(HS_ERR_SOLVER, "%s failed: cublas status %d (%s:%d)", #x, (int)e_,  \
                        __FILE__, __LINE__);                                              \
  } while (0)
#define HS_TRY(x)               \
  do {                          \
    hs_status s_ = (x);         \
    if (s_ != HS_OK) return s_; \
  } while (0)

// Split-K workspace of the FP64 GEMM, in doubles (32 MB).
constexpr long long kSplitKElems = 4ll << 20;

// Device buffer that only grows.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  // key of the padded split layout whose pad entries are known to be zero
  // (0: unknown). Only tc_split sets it; every other writer clears it.
  unsigned long long zkey = 0;
  hs_status ensure(size_t want) {
    if (want <= bytes) return HS_OK;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    zkey = 0;
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(HS_ERR_CUDA, "cudaMalloc of %zu bytes failed", want);
    }
    bytes = want;
    return HS_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    zkey = 0;
  }
  double* d() const { return static_cast<double*>(p); }
};

// The two parity blocks of one subspace quantity back to back in one
// allocation (block 1 starts at off[1] elements).
struct Stacked {
  DBuf buf;
  long long off[2] = {0, 0};
  hs_status ensure(long long e0, long long e1, size_t esize) {
    off[0] = 0;
    off[1] = e0;
    return buf.ensure((size_t)(e0 + e1 + 2) * esize);
  }
  double* d(int b) const { return buf.d() + off[b]; }
  template <class T>
  T* as(int b) const {
    return static_cast<T*>(buf.p) + off[b];
  }
  void release() { buf.release(); }
};

// Pinned host buffer, grown on demand (device-to-host copies into pageable
// memory block the host until the stream drains).
struct PinnedBuf {
  void* p = nullptr;
  size_t bytes = 0;
  hs_status ensure(size_t want) {
    if (want <= bytes) return HS_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    if (cudaMallocHost(&p, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(HS_ERR_CUDA, "cudaMallocHost of %zu bytes failed", want);
    }
    bytes = want;
    return HS_OK;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
  }
};

}  // namespace hs

struct hs_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  cusolverDnHandle_t solver = nullptr;
  cusolverDnParams_t params = nullptr;
  cublasHandle_t blas = nullptr;
  // move workspace
  hs::DBuf big1, big2, x1, pt, pp, w, lam, idx, sel, scratch, info, solver_dev;
  std::vector<char> solver_host;
  hs::SelectOut* h_sel = nullptr;  // pinned
  int* h_info = nullptr;           // pinned
  // observables workspace
  hs::DBuf r[16];
  // tensor-core operands: split double layer (cached per source/precision),
  // split A operand of the current GEMM, split B for hs_gemm, error word
  hs::DBuf tc_a_hi, tc_a_lo, tc_x_hi, tc_x_lo, tc_b_hi, tc_b_lo, tc_err;
  // split operands written by a GEMM epilogue (X2 permuted, then Y permuted)
  hs::DBuf ps_hi, ps_lo;
  const double* tc_a_src = nullptr;
  int tc_a_prec = -1;
  int* h_tc_err = nullptr;  // pinned
  // FP32-eigenvector mode: FP32 copy of C', FP32 eigenvalues, P (columns),
  // updated PT, Gram/Loewdin matrices, W = PT C'
  hs::DBuf c32, w32, pcol, pt2, gram, wproj, solver32_dev;
  std::vector<char> solver32_host;
  // second solver: the odd block's eigen-decomposition runs on its own
  // stream and handle, driven from a helper thread, beside the even block's
  cudaStream_t stream2 = nullptr;
  cusolverDnHandle_t solver2 = nullptr;
  cusolverDnParams_t params2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  hs::DBuf solver2_dev, solver2_32_dev;
  std::vector<char> solver2_host, solver2_32_host;
  // HOTRG workspace
  hs::DBuf hb[16];
  // complex (graded) CTMRG: private copy of a~ followed by its conjugate, and scratch
  hs::DBuf ga;
  const double* ga_src = nullptr;
  hs::DBuf gb[12];
  // complex observables (planar real / imaginary parts)
  hs::DBuf zr[40];
  // complex CTMRG in the plain basis (hs_zdense.cu)
  hs::DBuf zd[40];
  // directional CTMRG (hs_ctmrg4.cu): the rotated double layers in their two
  // operand layouts, move scratch, SVD workspace and its host staging
  hs::DBuf d4[40];
  hs::PinnedBuf d4_h;
  const double* d4_src = nullptr;
  gesvdjInfo_t gesvdj = nullptr;
  std::vector<char> d4_work_host;
  long long d4_svd_fallbacks = 0;  // blocks that took the Jacobi SVD
  // split-K partial sums of the FP64 GEMM
  hs::DBuf splitk;
  // subspace eigensolver: warm start (previous kept rows, per block) and
  // per-block iteration buffers
  const void* ws_env = nullptr;
  bool ws_valid = false;
  int ws_k[2] = {0, 0}, ws_n[2] = {0, 0}, ws_m[2] = {0, 0};  // kept counts, block sizes, stored rows
  int ws_c[2] = {-1, -1};  // boundary sectors of the C' the stored rows belong to (-1: not remappable)
  long long ws_moves = 0;
  bool sH_fresh = false;  // sH_hi/lo hold the split blocks of this move's C'
  bool sel_ready = false; // this move's selection is done and its host copy read back
  // this move's enlarged corner C' (and the GEMM outputs before it) are FP32
  // (the tensor-core accumulators' values) rather than FP64
  bool cp_f32 = false;
  int sH_n[2] = {0, 0};
  // per-block subspace quantities stacked (block 1 after block 0), so that
  // one launch covers both parity blocks; sH_hi/lo hold the split C' blocks in
  // their padded Z2 layout
  hs::Stacked sx, sz, sxc, szc, sxr, szr, sbm, sbw, sres;
  hs::DBuf ws_pt, sth, sH_hi, sH_lo, sx_hi, sx_lo, sy_hi, sy_lo, schol;
  // Chebyshev filter of the subspace eigensolver: three recurrence terms, the
  // product, the projection and its coefficients, the locked rows (and their
  // transpose), and the row order
  hs::DBuf sf_y[3], sf_z, sf_t, sf_s, sf_q, sf_qt, sf_idx, sf_xl, sf_qh, sf_ql, sf_qth, sf_qtl;
  // pinned staging: Ritz values, residuals and status words (device to
  // host), the filter's row order (host to device)
  hs::PinnedBuf h_sub, h_idx;
  // adaptive subspace tolerance: the warm start's residual in the previous
  // move's first round, and the environment it belongs to
  double prev_first_resid = 0.0;
  // the previous move's kept rows (final PT, both blocks stacked), for
  // ordering this move's kept rows like them (align_kept_rows)
  hs::DBuf pt_prev, ovl, ovl_idx, ovl_sgn, pt_tmp;
  // the subspace rows before the last Cholesky-QR (for the Householder redo
  // when that breaks down) and the count of such redos
  hs::DBuf sx_save;
  bool sx_save_valid = false;
  long long qr_redos = 0;
  hs::PinnedBuf h_ovl;
  bool pt_prev_valid = false;
  int pt_prev_k[2] = {0, 0}, pt_prev_n[2] = {0, 0};
  // the subspace residual at which a previous move stalled on the rounding
  // of its products (0: none yet); the tolerance of later moves follows it
  double resid_floor = 0.0;
  const void* prev_spec_env = nullptr;
  // permute plans by layout pair and permutation (building one takes a few
  // microseconds of host time, and every move repeats the same few dozen)
  std::unordered_map<std::string, hs::PermPlan> plan_cache;
  // profiling: events between phases, harvested after the move's last sync
  bool prof = false;
  unsigned prof_mask = ~0u;  // phases that record events when prof is on
  std::vector<cudaEvent_t> events;
  int next_event = 0;
  struct Rec {
    int phase, e0, e1;
  };
  std::vector<Rec> recs;
  double phase_ms[HS_PHASE_COUNT] = {};
  double phase_flops[HS_PHASE_COUNT] = {};
  long long launches = 0;
};

namespace hs {

hs_status check_ctx(hs_ctx ctx);
Sect q_sect(int D, hs_basis b);
Z2Mat mat(Fused r, Fused c, int pad = 1);
// C = A B^T on the chosen backend.
hs_status gemm(hs_ctx ctx, hs_gemm_backend be, const GemmGroup& g, const double* A, const double* B,
               double* C);
// make_perm_plan through the context's cache (perm: kMaxLegs entries).
const PermPlan& cached_plan(hs_ctx ctx, const Z2Mat& in, const Z2Mat& out, const int* perm);
// The open double layers of the two-site network and their adjoint (dA =, not +=).
cudaError_t launch_open_double_layers(const double* A, int d, int D, double* aoL, double* aoR, cudaStream_t s);
cudaError_t launch_open_double_layers_vjp(const double* daoL, const double* daoR, const double* A, int d, int D,
                                          double* dA, cudaStream_t s);
hs_status permute(hs_ctx ctx, const Z2Mat& in, const Z2Mat& out, std::initializer_list<int> perm,
                  const double* src, double* dst);

// Eigen-decompositions of the two parity blocks (block 1 on the second
// stream); FP32 when f32. Shared with the HOTRG step.
hs_status eig_pair(hs_ctx ctx, bool f32, void* A0, int n0, void* w0, void* A1, int n1, void* w1);
hs_status eig_workspace(hs_ctx ctx, int nmax);
// One symmetric eigen-decomposition (vectors in place, column-major) on the
// context stream; FP32 when f32 (workspace from eig_workspace32).
hs_status eig_single(hs_ctx ctx, bool f32, void* A, int n, void* w);
hs_status eig_workspace32(hs_ctx ctx, int nmax);
// C[M x N] = A[M x K] B[N x K]^T, dense row-major FP64 (tensor cores in the
// TF32/BF16 precisions, else the FP64 kernel).
hs_status dense_gemm_any(hs_ctx ctx, hs_precision prec, int M, int N, int K, const double* A, const double* B,
                         double* C);
// Complex (graded) CTMRG, hs_graded.cu.
hs_status graded_double_layer(hs_ctx ctx, const double* A, int d, int D, hs_z2_tensor* out);
size_t graded_tensor_bytes(int D);
hs_status graded_init(hs_ctx ctx, const hs_z2_tensor* a, int chi_max, hs_env* env);
hs_status graded_move(hs_ctx ctx, const hs_z2_tensor* a, hs_env* env, int chi, hs_move_info* info);
// Complex CTMRG in the plain basis (hs_zdense.cu): the comparison path.
size_t zdense_tensor_bytes(int D);
hs_status zdense_double_layer(hs_ctx ctx, const double* A, int d, int D, hs_z2_tensor* out);
hs_status zdense_init(hs_ctx ctx, const hs_z2_tensor* a, int chi_max, hs_env* env);
hs_status zdense_move(hs_ctx ctx, const hs_z2_tensor* a, hs_env* env, int chi, hs_move_info* info);
// Loewdin re-orthonormalisation of the m rows of X (n long), `steps` times.
hs_status lowdin_rows(hs_ctx ctx, hs_precision prec, double* X, int m, int n, double* Xc, int steps);
// Stacked parity-block pairs (block 1 right after block 0): the pair as one
// Z2 layout, views into buffers, the split C' blocks, batched Loewdin steps.
Z2Mat zd(long long r0, long long r1, long long c0, long long c1, int pad = 1);
DBuf view(const DBuf& b, long long byte_off);
DBuf sH_block(hs_ctx ctx, hs_precision prec, bool hi, int b);
// H0 holds FP32 values when ctx->cp_f32 is set.
hs_status split_corner(hs_ctx ctx, hs_precision prec, const double* H0, int n0, int n1);
hs_status lowdin_rows_pair(hs_ctx ctx, hs_precision prec, double* X, const int m[2], const int n[2], double* Xc,
                           int steps);

// Tensor-core operands: tc_split writes the operand `layout` (src_layout's legs
// permuted by perm) of a tcgen05 GEMM as split, K-padded hi/lo arrays; tc_run
// computes C[R|N] = A[R|K] B[N|K]^T from two such operands into C (FP64 in
// layout Cm, or FP32 when out_f32).
hs_status tc_split(hs_ctx ctx, hs_precision prec, const Z2Mat& src_layout, const Z2Mat& layout,
                   std::initializer_list<int> perm, const double* src, DBuf& hi, DBuf& lo);
hs_status tc_run(hs_ctx ctx, hs_precision prec, const Z2Mat& A, const DBuf& ahi, const DBuf& alo, const Z2Mat& B,
                 const DBuf& bhi, const DBuf& blo, const Z2Mat& Cm, double* C, bool out_f32 = false);

// Warm-started subspace eigensolver of hs_api.cu: on success (*done) the
// Ritz values of both blocks are in w (block 0 then 1), the Ritz vectors in
// ctx->sxr, the selection of the chi largest |values| in ctx->sel / idx / lam;
// otherwise the caller falls back to a full eigen-decomposition.
hs_status subspace_projector(hs_ctx ctx, hs_env* env, int chi, int n0, int n1, double* H0, double* H1, double* w,
                             int* m_out, bool* done, int* iters, double* flops, int* reason, double* resid);
// Spare subspace rows beyond k kept states.
int oversample(int k);

// Tensor-core precisions: elements per 128-byte row (the K padding unit),
// bytes per element, split mode of the permute/split kernels.
int tc_pad(hs_precision p);
int tc_elem_bytes(hs_precision p);
int tc_mode(hs_precision p);

// Records a CUDA event pair around a phase when profiling is on.
class PhaseScope {
 public:
  PhaseScope(hs_ctx c, int phase);
  ~PhaseScope();

 private:
  hs_ctx c_;
  int phase_, e0_;
};

// Accumulates the recorded phases (call after the stream has synchronised).
void harvest_profile(hs_ctx ctx);

}  // namespace hs

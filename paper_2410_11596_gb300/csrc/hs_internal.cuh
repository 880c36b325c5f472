// Internal declarations of libhs: sector-ordered ("FSO") block layouts, the
// descriptors the kernels consume, and the kernel launchers.
//
// Z2 block structure (arXiv 2410.11596, Sec. II.B): every leg carries a
// parity split (even, odd). A tensor is stored as a block-diagonal matrix
// over a grouping of its legs into row legs and column legs; a group of legs
// is "fused" by enumerating the parity tuples of its legs grouped by total
// parity (even group first), tuples in lexicographic order (first leg most
// significant bit), local indices row-major inside each tuple.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <set>
#include <tuple>
#include <utility>
#include <cuda_runtime.h>

#include "../../include/hs.h"

#define HS_HD __host__ __device__ __forceinline__

namespace hs {

// Sector sizes of one leg.
// Programmatic dependent launch. Every kernel of the library is launched by
// hs_launch with programmatic stream serialisation allowed and opens with
// hs_pdl_enter(): it first waits until the previous kernel in the stream has
// completed and its writes are visible (griddepcontrol.wait, before any
// global memory access), then lets the next kernel be scheduled
// (griddepcontrol.launch_dependents). The next kernel's launch and prologue
// so overlap this kernel's run, while the data order stays that of the stream.
__device__ __forceinline__ void hs_pdl_enter() {
#if defined(__CUDA_ARCH__)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
inline cudaError_t hs_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args&&... args) {
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// hs_launch of a grid of clusters of `cluster` CTAs along x.
template <typename... KArgs, typename... Args>
inline cudaError_t hs_launch_cluster(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                     unsigned cluster, Args&&... args) {
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = cluster;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Opt a kernel in to `bytes` of dynamic shared memory on the current device.
// The attribute belongs to the device's context, so it is set once per
// (kernel, device, size) rather than once per process.
inline cudaError_t ensure_smem_attr(const void* func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::set<std::tuple<const void*, int, int>> done;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(func, dev, bytes);
  if (done.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert(key);
  return e;
}

// Number of SMs of the current device (cached per device; 148 if unknown).
inline int device_sms() {
  constexpr int kDevs = 64;
  static int cache[kDevs] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
  if (dev < kDevs && cache[dev] > 0) return cache[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  if (dev < kDevs) cache[dev] = n;
  return n;
}

struct Sect {
  int n[2];
};

HS_HD Sect make_sect(int e, int o) {
  Sect s;
  s.n[0] = e;
  s.n[1] = o;
  return s;
}

// A group of up to 4 legs fused into one matrix index.
constexpr int kMaxFused = 4;
struct Fused {
  int k;
  Sect leg[kMaxFused];
};

HS_HD Fused fused0() {
  Fused f;
  f.k = 0;
  return f;
}
HS_HD Fused fused1(Sect a) {
  Fused f;
  f.k = 1;
  f.leg[0] = a;
  return f;
}
HS_HD Fused fused2(Sect a, Sect b) {
  Fused f;
  f.k = 2;
  f.leg[0] = a;
  f.leg[1] = b;
  return f;
}
HS_HD Fused fused3(Sect a, Sect b, Sect c) {
  Fused f;
  f.k = 3;
  f.leg[0] = a;
  f.leg[1] = b;
  f.leg[2] = c;
  return f;
}
HS_HD Fused fused4(Sect a, Sect b, Sect c, Sect d) {
  Fused f;
  f.k = 4;
  f.leg[0] = a;
  f.leg[1] = b;
  f.leg[2] = c;
  f.leg[3] = d;
  return f;
}

HS_HD int tuple_parity(int t) { return __builtin_popcount((unsigned)t) & 1; }

// Parity of leg j inside tuple t of a k-leg group (leg 0 = most significant).
HS_HD int tuple_bit(int t, int k, int j) { return (t >> (k - 1 - j)) & 1; }

HS_HD long long tuple_size(const Fused& f, int t) {
  long long s = 1;
  for (int j = 0; j < f.k; ++j) s *= f.leg[j].n[tuple_bit(t, f.k, j)];
  return s;
}

// Number of fused indices of total parity P.
HS_HD long long fused_size(const Fused& f, int P) {
  long long s = 0;
  for (int t = 0; t < (1 << f.k); ++t)
    if (tuple_parity(t) == P) s += tuple_size(f, t);
  return s;
}

// Offset of tuple t inside its parity group.
HS_HD long long tuple_offset(const Fused& f, int t) {
  long long s = 0;
  const int P = tuple_parity(t);
  for (int u = 0; u < t; ++u)
    if (tuple_parity(u) == P) s += tuple_size(f, u);
  return s;
}

// Block-diagonal Z2 matrix: block p = rows of parity p x cols of parity p.
// Each block's row stride is its column count rounded up to `pad` elements
// (pad = 1: tightly packed; the tensor-core operands use 32 so that rows are
// whole 128-byte swizzle atoms and 16-byte aligned for TMA).
struct Z2Mat {
  Fused r, c;
  int pad;
};

HS_HD long long z2_rows(const Z2Mat& m, int p) { return fused_size(m.r, p); }
HS_HD long long z2_cols(const Z2Mat& m, int p) { return fused_size(m.c, p); }
HS_HD long long z2_ld(const Z2Mat& m, int p) {
  const long long c = z2_cols(m, p);
  const long long a = m.pad > 1 ? m.pad : 1;
  return (c + a - 1) / a * a;
}
HS_HD long long z2_block_off(const Z2Mat& m, int p) {
  return p == 0 ? 0 : z2_rows(m, 0) * z2_ld(m, 0);
}
HS_HD long long z2_elems(const Z2Mat& m) {
  return z2_rows(m, 0) * z2_ld(m, 0) + z2_rows(m, 1) * z2_ld(m, 1);
}

// ---- permutation of a Z2 matrix into another grouping/order of its legs ----

// One dense box: out[i0..i5] = in[...] for i_j < dim[j] (up to 6 legs; the
// leading unused dimensions have extent 1).
constexpr int kMaxLegs = 6;
struct Box {
  long long out_off, in_off;
  int dim[kMaxLegs];
  long long out_stride[kMaxLegs], in_stride[kMaxLegs];
  long long count;   // product of dims
  long long start;   // prefix sum of counts over earlier boxes
  // division by dim[j] of 32-bit indices (fast_div in hs_bits.cuh)
  unsigned mag[kMaxLegs];
  unsigned char sh1[kMaxLegs], sh2[kMaxLegs];
  int lo;            // first non-trivial dim: dims [0, lo) have extent 1
  // chunked traversal: rows (all dims but the innermost) x nch chunks of
  // kPermVec innermost elements; division by nch as for the dims
  int fits32;        // every offset of the box and rows * nch below 2^31
  unsigned rows, nch, magc;
  unsigned char sh1c, sh2c;
  // tiled transpose (fits32 boxes whose input-contiguous dim ji is not the
  // innermost output dim): kPermTile x kPermTile tiles over (dim ji, the
  // innermost dim), the other dims a batch (nbd dims, outermost first);
  // ji < 0: not tiled
  int ji, nbd;
  // plane mode (plane > 0): both extents small, a CTA stages `plane` whole
  // (dim ji x innermost dim) planes at a time; psz = their product
  int plane;
  unsigned psz, magp, magpi, magpo;
  unsigned char sh1p, sh2p, sh1pi, sh2pi, sh1po, sh2po;
  unsigned ntile_i, ntile_o, nbatch, magto, magti;
  unsigned char sh1to, sh2to, sh1ti, sh2ti;
  int bdim[kMaxLegs];
  unsigned bin_stride[kMaxLegs], bout_stride[kMaxLegs], bmag[kMaxLegs];
  unsigned char bsh1[kMaxLegs], bsh2[kMaxLegs];
};
constexpr int kPermVec = 4;
constexpr int kPermTile = 32;
constexpr int kPermPlaneElems = 2048;  // staged elements per plane-mode step

constexpr int kMaxBoxes = 32;  // even-parity tuples of 6 legs

struct PermPlan {
  int nbox;
  long long total;
  Box box[kMaxBoxes];
};

// Build the plan that maps matrix `in` (legs L0..L{n-1}; the first in.r.k are
// rows) to matrix `out` whose leg j is input leg perm[j]. Both even-total.
PermPlan make_perm_plan(const Z2Mat& in, const Z2Mat& out, const int* perm);

// ---- graded dense matrices (complex tensors, Sec. II.C) ----------------------
//
// For complex A the double layer in the eigenbasis of S is not block sparse,
// but each block is purely real (even total parity) or purely imaginary (odd):
// Sec. II.C. A graded matrix stores all four parity blocks as one dense
// row-major real matrix, rows and columns each in FSO order (even group
// first); an entry of odd total parity holds the imaginary part of the
// complex value, an even one the real part. The product of two graded
// matrices is graded (the rule f of Eq. (2)-(3)): with x = i^[p(r)!=p(k)] x~,
//   C~[r, k] = sum_j s A~[r, j] B~[j, k],  s = -1 iff p(j) != p(r) = p(k).
struct GMat {
  Fused r, c;
  int pad;
};

HS_HD long long g_rows(const GMat& m) { return fused_size(m.r, 0) + fused_size(m.r, 1); }
HS_HD long long g_cols(const GMat& m) { return fused_size(m.c, 0) + fused_size(m.c, 1); }
HS_HD long long g_ld(const GMat& m) {
  const long long a = m.pad > 1 ? m.pad : 1;
  return (g_cols(m) + a - 1) / a * a;
}
HS_HD long long g_elems(const GMat& m) { return g_rows(m) * g_ld(m); }
HS_HD long long g_row0(const GMat& m, int p) { return p ? fused_size(m.r, 0) : 0; }
HS_HD long long g_col0(const GMat& m, int p) { return p ? fused_size(m.c, 0) : 0; }

// Permutation plan between two graded matrices (all parity tuples; at most
// five legs). Returns false if the tuples do not fit the plan.
bool make_graded_perm_plan(const GMat& in, const GMat& out, const int* perm, PermPlan* plan);

// ---- grouped GEMM ----------------------------------------------------------

// C[m, n] = alpha * sum_k A[m, k] B[n, k] (+ beta C): both operands K-major.
struct GemmProblem {
  int M, N, K;
  int lda, ldb, ldc;
  long long a_off, b_off, c_off;  // element offsets
};

constexpr int kMaxProblems = 4;

struct GemmGroup {
  int n;
  GemmProblem p[kMaxProblems];
};

// The two block GEMMs of a Z2 product C[R|N] = A[R|K] B[N|K]^T.
GemmGroup make_z2_gemm(const Z2Mat& A, const Z2Mat& B, const Z2Mat& C);
// The four sub-GEMMs of a graded product C~[R|N] = A~[R|K] B~[N|K]^T: the
// output block (pr, pc) is A~'s row block pr times B~'s row block pc over the
// whole K; the diagonal blocks (pr == pc) read the conjugate copy of B~ (its
// odd-total entries negated), stored `bconj_off` elements after B~.
GemmGroup make_graded_gemm(const GMat& A, const GMat& B, const GMat& C, long long bconj_off);
double gemm_flops(const GemmGroup& g);

// ---- kernel launchers (device code in k_*.cu) -------------------------------

cudaError_t launch_permute_f64(const PermPlan& plan, const double* in, double* out, double scale,
                               cudaStream_t s);
// Same permutation, writing the operand split for the tensor cores:
// mode 1: hi = tf32(x), lo = fp32(x - hi) as float; mode 2: bf16 hi/lo pair.
// The padded columns of `out` must have been zeroed by the caller.
// FP32 sources (values that came out of the tensor-core GEMMs' FP32 accumulators).
cudaError_t launch_permute_f32(const PermPlan& plan, const float* in, float* out, cudaStream_t s);
cudaError_t launch_permute_split_f32(const PermPlan& plan, const float* in, void* hi, void* lo, int mode,
                                     cudaStream_t s);
// FP32 values of a TF32x3-split block pair (padded rows of ld0/ld1 elements,
// block 1 at element off1) into out, tightly packed, block 1 after block 0.
cudaError_t launch_join_split_f32(const void* hi, const void* lo, long long rows0, long long cols0, long long ld0,
                                  long long off1, long long rows1, long long cols1, long long ld1, float* out,
                                  cudaStream_t s);
cudaError_t launch_permute_split(const PermPlan& plan, const double* in, void* hi, void* lo, int mode,
                                 cudaStream_t s);

// Split a row-major FP64 matrix [rows, cols] (row stride ld_src) into padded
// hi/lo operands [rows, ld_dst] (zeros in columns cols..ld_dst-1); mode as above.
cudaError_t launch_split_pad(const double* src, long long rows, int cols, long long ld_src, void* hi,
                             void* lo, long long ld_dst, int mode, cudaStream_t s);

// ---- tensor-core (tcgen05) block GEMM ------------------------------------------

// One block problem: C[M, N] (FP64, row stride ldc) = A[M, Kp] B[N, Kp]^T with
// A and B given as hi/lo splits (FP32 for TF32, BF16 for BF16), rows Kp apart.
// Output of a tensor-core GEMM written straight as the split (TF32 hi, FP32
// lo) operand of the next GEMM, with its four legs permuted. The output block
// has rows (L0, L1) and columns (L2, L3), each fused from two parity tuples:
// rows [0, rsplit) are tuple 0, the rest tuple 1, with inner leg extents
// rin[t] (columns likewise). Entry (i0, i1 | j0, j1) of row tuple tr and
// column tuple tc goes to element base[tr][tc] + co[tr][tc] . (i0, i1, j0, j1)
// of hi and lo (4-byte elements, fewer than limit). mode 1: the destination's
// innermost leg is L1 (a warp stores 32 consecutive rows); mode 2: it is L3
// (stores run along the columns, staged through shared memory).
struct PsDesc {
  void* hi;
  void* lo;
  int limit;
  int rsplit, csplit;
  int rin[2], cin[2];
  int base[2][2];
  int co[2][2][4];
  int mode;
};

struct TcProblem {
  int M, N, Kp, ldc;
  const void* a_hi;
  const void* a_lo;
  const void* b_hi;
  const void* b_lo;
  double* c;        // FP64 output, or FP32 (c read as float*, ldc in floats) when out_f32
  int out_f32 = 0;  // the accumulators are FP32, so an FP32 output loses nothing (one split-K sum rounds once)
  const PsDesc* ps = nullptr;  // when set, the output goes there instead of c (never split along K)
};

// Up to four problems per launch. precision: HS_PREC_TF32X3, HS_PREC_TF32 or HS_PREC_BF16X3. err receives a
// non-zero code if a bounded wait inside the kernel gave up.
// part/part_elems: optional FP64 workspace for split-K partials (used when a
// problem's output tiles cannot fill the GPU); nullptr disables splitting.
cudaError_t launch_gemm_tc(int precision, const TcProblem* probs, int nprob, int* err, cudaStream_t s,
                           double* part = nullptr, long long part_elems = 0);
// part/part_elems: optional workspace for split-K partial sums (used when the
// output tiles alone cannot fill the GPU); nullptr disables splitting.
// accumulate: C += alpha A B^T instead of C = alpha A B^T.
cudaError_t launch_gemm_f64(const GemmGroup& g, const double* A, const double* B, double* C,
                            double alpha, cudaStream_t s, double* part = nullptr, long long part_elems = 0,
                            bool accumulate = false);

// A[p,u,l,d,r] (real) -> a~ blocks in FSO [(u,l)|(d,r)]; hermitian selects the
// rotation by U^T on every leg, otherwise the plain combined basis.
cudaError_t launch_double_layer_blocks(const double* A, int d, int D, bool hermitian, double* out,
                                       cudaStream_t s);
// Dense double layer (D^2)^4 from A, real (cplx = false) or complex128.
cudaError_t launch_double_layer_dense(const double* A, int d, int D, bool cplx, double* out,
                                      cudaStream_t s);
// Rotate a dense real double layer into all 16 parity blocks; writes the
// even-total ones (FSO) and atomically maxes |odd| and |all| into maxes[0..1].
cudaError_t launch_rotate_dense_to_blocks(const double* a, int D, double* out,
                                          unsigned long long* maxes, cudaStream_t s);

// Inverse rotation: the stored blocks of a~ (real FSO [(u,l)|(d,r)], or a
// graded complex matrix) back to the dense plain combined basis (D^2)^4
// (interleaved complex128 when graded).
cudaError_t launch_from_hermitian(const double* t, int D, bool graded, double* out, cudaStream_t s);

// Traced-boundary initial C0 and T0 (FSO) from the stored blocks of a.
cudaError_t launch_ctmrg_init(const double* a_blocks, int D, bool hermitian, double* C, double* T,
                              cudaStream_t s);

struct SelectOut {
  int chi_new[2];
  int pad[2];
  double lam_max, lam_cut, lam_next;
  double log_norm_C, log_norm_T;
  double discarded;  // sum of |lambda| over the states not kept
};

// Choose the chi eigenvalues of largest modulus across the two blocks.
cudaError_t launch_select(const double* w0, int n0, const double* w1, int n1, int chi,
                          int* idx /* [2][chi] */, double* lam /* new diag, FSO order */,
                          SelectOut* out, cudaStream_t s);
// P^T rows: block p row j = eigenvector idx[p][j] of V_p (column-major n_p x n_p).
// The new sector sizes are read on the device from sel.
cudaError_t launch_gather_pt(const double* V0, int n0, const double* V1, int n1, const int* idx,
                             int chi, const SelectOut* sel, double* PT, cudaStream_t s);
// C <- diag(lam) / max|lam| in FSO blocks (c0 x c0, c1 x c1).
cudaError_t launch_diag_corner(const double* lam, int c0, int c1, SelectOut* sel, double* C,
                               cudaStream_t s);
// T <- T / max|T| over n entries; log of the factor into sel->log_norm_T.
cudaError_t launch_normalize_max(double* T, long long n, unsigned long long* scratch,
                                 SelectOut* sel, cudaStream_t s);

// FP32-eigenvector mode: casts, gather of the kept vectors into PT (rows) and
// P (columns, FP64), the Loewdin update M = 1.5 I - 0.5 G of each block of G,
// and a max-abs normalisation that writes its log to *log_out.
cudaError_t launch_cast_f64_f32(const double* src, float* dst, long long n, cudaStream_t s);
cudaError_t launch_cast_f32_f64(const float* src, double* dst, long long n, cudaStream_t s);
cudaError_t launch_gather_p32(const float* V0, int n0, const float* V1, int n1, const int* idx, int chi,
                              const SelectOut* sel, double* PT, double* P, cudaStream_t s);
cudaError_t launch_lowdin(double* G, int k0, int k1, cudaStream_t s);
cudaError_t launch_normalize_max_to(double* x, long long n, unsigned long long* scratch, double* log_out,
                                    cudaStream_t s);

// Sum of the diagonals of a block-diagonal FSO matrix with square blocks
// (n0 x n0 then n1 x n1) into *out.
cudaError_t launch_block_trace(const double* x, int n0, int n1, double* out, cudaStream_t s);

// Warm-started subspace eigensolver kernels (k_subspace.cu).
cudaError_t launch_fill_random_rows(double* X, int r0, int m, int n, unsigned long long seed, cudaStream_t s);
// Cholesky factor inverses L_b^{-1} of two SPD matrices G_b (m_b <= max_subspace(),
// m_b = 0 skips one), one CTA each; *status = 1 on a non-positive pivot.
cudaError_t launch_chol_inv(const double* G0, int m0, double* Linv0, const double* G1, int m1, double* Linv1,
                            int* status, cudaStream_t s);
cudaError_t launch_residual(const double* Zr, const double* Xr, const float* theta, int m, int n, double* res,
                            cudaStream_t s);
cudaError_t launch_row_sign(double* X, int m, int n, cudaStream_t s);
// Over a stacked pair: m0 rows of n0 entries, then m1 rows of n1 (theta and
// res stacked likewise).
cudaError_t launch_row_sign_pair(double* X, int m0, int n0, int m1, int n1, cudaStream_t s);
cudaError_t launch_residual_pair(const double* Zr, const double* Xr, const float* theta, int m0, int n0, int m1,
                                 int n1, double* res, cudaStream_t s);
cudaError_t launch_gather_rows(const double* X0, int n0, const double* X1, int n1, const int* idx, int chi,
                               const SelectOut* sel, double* PT, double* P, cudaStream_t s);
int max_subspace();
// Warm-start rows of parity block b of C' moved from boundary sectors c_old to
// c_new (same double-layer sectors q): entries of states both boundaries have
// are kept, the others zero; then seeded noise of about 1% of an entry of a
// unit row, so that no row is left (nearly) zero.
cudaError_t launch_remap_rows(const double* src, int rows, int old_n, double* dst, int new_n, int b, Sect c_old,
                              Sect c_new, Sect q, unsigned long long seed, cudaStream_t s);
// Largest m of launch_chol_inv (one CTA, shared memory).
int max_chol();
// After a library Cholesky + triangular inverse: zero the strictly upper part of
// the row-major L^{-1} (m x m) and set *bad if info[0] or info[1] is non-zero.
cudaError_t launch_tidy_linv(double* L, int m, const int* info, int* bad, cudaStream_t s);
// Two small symmetric FP32 eigen-decompositions (one CTA each; m <= max_subspace()),
// output as syevd: ascending eigenvalues, vectors as columns (column-major, in place);
// *status = 1 if a matrix did not converge.
cudaError_t launch_jacobi_eig_pair(float* A0, int m0, float* w0, float* A1, int m1, float* w1, int* status,
                                   cudaStream_t s);
cudaError_t launch_row_normalize(double* X, int m, int n, cudaStream_t s);
// out row i = X row idx[i] for i < m (idx on the device; rows of n).
cudaError_t launch_gather_rows_idx(const double* X, const int* idx, int m, int n, double* out, cudaStream_t s);
// Stacked pairs (block 1 at the given element offsets): gather of cnt_b rows
// of block b by idx (cnt0 entries for block 0, then cnt1), and the
// Chebyshev term with alpha0 on the first count0 entries, alpha1 after.
cudaError_t launch_gather_rows_idx_pair(const double* X, long long src_off1, int n0, int n1, const int* idx,
                                        int cnt0, int cnt1, double* out, long long dst_off1, cudaStream_t s);
// As launch_gather_rows_idx_pair, output row j scaled by sgn[j] (device, cnt0 + cnt1 entries).
cudaError_t launch_gather_rows_idx_sign_pair(const double* X, long long src_off1, int n0, int n1, const int* idx,
                                             const double* sgn, int cnt0, int cnt1, double* out, long long dst_off1,
                                             cudaStream_t s);
cudaError_t launch_cheb_step_pair(double* Y, const double* Z, const double* T, const double* Yold, long long count,
                                  long long count0, double alpha0, double alpha1, double beta, cudaStream_t s);
// Y = alpha (Z - T) + beta Yold over count entries; T and Yold may be null.
cudaError_t launch_cheb_step(double* Y, const double* Z, const double* T, const double* Yold, long long count,
                             double alpha, double beta, cudaStream_t s);
// X (m x n rows, FP64) = the m eigenvectors of largest |eigenvalue| of one
// FP32 eigen-decomposition (ascending w, column-major V); idx is scratch (m ints).
cudaError_t launch_top_rows(const float* w, const float* V, int n, int m, int* idx, double* X, cudaStream_t s);

// ---- graded (complex) kernels, k_graded.cu --------------------------------

// dst = src with a sign on part of a graded matrix (rows split r0 | r1,
// columns c0 | c1, row stride ld; dst may equal src):
//   mode 0: negate entries of odd total parity (complex conjugation);
//   mode 1: negate the odd-odd block (C~ -> M with C = J M J, J = diag(1, i)).
cudaError_t launch_graded_sign(const double* src, double* dst, long long r0, long long r1, long long c0,
                               long long c1, long long ld, int mode, cudaStream_t s);
// a~ of a complex A (interleaved complex128) as a graded [(u,l)|(d,r)] matrix.
cudaError_t launch_double_layer_graded(const double* A, int d, int D, double* out, cudaStream_t s);
// Traced-boundary C0 [d | r] and T0 [(alpha, x) | beta] (graded, chi0 = D^2
// with the sectors of one double-layer leg) from the graded a~.
cudaError_t launch_ctmrg_init_graded(const double* a, int D, double* C, double* T, cudaStream_t s);
// Truncation from the ascending eigenvalues w (n) of H = M M^T with vectors V
// (column-major n x n): keep k = min(chi, n) largest, singular values
// sqrt(w); PT rows = the kept vectors in descending order; sel->chi_new =
// {k, 0}; lam_* from the singular values. FP32 variant reads float w and V.
cudaError_t launch_graded_select(const double* w, const double* V, int n, int chi, double* PT, SelectOut* sel,
                                 cudaStream_t s);
cudaError_t launch_graded_select32(const float* w, const float* V, int n, int chi, double* PT, SelectOut* sel,
                                   cudaStream_t s);
// Complex dense views (interleaved complex128, plain combined basis) of a
// graded environment with boundary sectors (c0, c1).
cudaError_t launch_env_to_dense_graded(const double* C, const double* T, int D, int c0, int c1, double* Cd,
                                       double* Td, cudaStream_t s);

// Adjoints used by the gradient through the CTMRG iterations: of the traced
// init (dC0, dT0 -> da += , FSO a), of the dense views of the environment
// (dCd, dTd -> dC += , dT +=, FSO), and of the plain real double layer
// (da_plain -> dA +=).
cudaError_t launch_ctmrg_init_vjp(const double* dC, const double* dT, int D, bool hermitian, double* da,
                                  cudaStream_t s);
cudaError_t launch_env_to_dense_vjp(const double* dCd, const double* dTd, int D, int c0, int c1, bool hermitian,
                                    double* dC, double* dT, cudaStream_t s);
cudaError_t launch_double_layer_vjp(const double* da_plain, const double* A, int d, int D, double* dA,
                                    cudaStream_t s);

// The tensor-core GEMM's bounded mbarrier wait on barriers with known outcomes
// (7 ints to the device array out; k_gemm_tc.cu).
cudaError_t launch_wait_selftest(long long limit, int* out, cudaStream_t s);

// Dense views of an FSO environment (rotated back to the plain combined basis).
cudaError_t launch_env_to_dense(const double* C, const double* T, int D, int c0, int c1,
                                bool hermitian, double* Cd, double* Td, cudaStream_t s);

}  // namespace hs

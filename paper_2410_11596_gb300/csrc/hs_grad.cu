// Gradient of the C4v CTMRG bond energy through the CTMRG iterations
// (differentiation of the whole contraction with respect to the iPEPS tensor,
// the use of CTMRG environments in variational optimisation that arXiv
// 2410.11596 Sec. III.A refers to). FP64, on the GPU, in the Hermitian basis
// (Sec. II.B) or the dense one.
//
// The forward pass is the FP64 path of hs_ctmrg_move (FP64 block GEMMs, the
// FP64 eigen-decomposition of each parity block), from the double layer and
// the traced-boundary start through `moves` moves to the two-site energy, each
// step recorded on a tape with the arrays it read and wrote. The reverse pass
// runs the tape backwards:
//   * a block GEMM C = A B^T gives dA += dC B and dB += dC^T A (transposed
//     operands by the permute kernels, products by the FP64 GEMM kernel with
//     accumulation);
//   * a leg permutation gives the inverse permutation of the cotangent;
//   * the eigen-decomposition C'_b = V diag(w) V^T of each parity block, of
//     which the kept columns V_k and (on the diagonal of the new corner) the kept
//     eigenvalues are used: dC'_b = sym(V (diag(dw) + F o (V^T dV)) V^T),
//     F_il = 1 / (w_l - w_i) (i != l), the standard adjoint of a symmetric
//     eigen-decomposition with distinct eigenvalues (dV has only kept columns);
//   * every max-abs normalisation: dx = dy / m. The energy is unchanged when C
//     or T is rescaled at any point (the next move's kept eigenvectors and the
//     normalised outputs do not change, and E = Tr(rho h) / Tr rho), so the
//     part of the exact adjoint along x, which carries the derivative of m,
//     contracts to zero against dE;
//   * the traced initialisation, the dense views of the final environment,
//     the open double layers and the double layer have their own adjoint kernels.
// A perturbation of A that breaks the C4v symmetry makes C' non-symmetric; the
// eigen-decomposition reads one triangle of it, and the adjoint above is the
// derivative along C4v-symmetric perturbations of A (the ones that keep the
// C4v CTMRG defined).
#include <algorithm>
#include <functional>
#include <memory>

#include "hs_ctx.cuh"

using namespace hs;

namespace {

unsigned grid_of(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (unsigned)g;
}

__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, long long n, double alpha) {
  hs_pdl_enter();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] += alpha * x[e];
}

// y += x / m, m = exp(*log_m) (the normalisation factor of the forward pass)
__global__ void add_scaled_kernel(double* __restrict__ y, const double* __restrict__ x, long long n,
                                  const double* __restrict__ log_m) {
  hs_pdl_enter();
  const double s = exp(-*log_m);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] += s * x[e];
}

// M[j][i] = dw_j (i = idx_j), W[j][i] / (w[idx_j] - w[i]) otherwise (k x n)
__global__ void eig_mix_kernel(const double* __restrict__ W, const double* __restrict__ w, const int* __restrict__ idx,
                               const double* __restrict__ dw, int k, int n, double* __restrict__ M) {
  hs_pdl_enter();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)k * n;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), i = (int)(e % n);
    const int l = idx[j];
    M[e] = i == l ? dw[j] : W[e] / (w[l] - w[i]);
  }
}

// dC += (X + X^T) / 2 for an n x n block
__global__ void sym_add_kernel(double* __restrict__ dC, const double* __restrict__ X, int n) {
  hs_pdl_enter();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    dC[e] += 0.5 * (X[e] + X[(long long)c * n + r]);
  }
}

// dw[j] = dCn[j][j] / lam_max for block b (k x k, FSO offset off)
__global__ void diag_take_kernel(const double* __restrict__ dCn, long long off, int k, double inv,
                                 double* __restrict__ dw) {
  hs_pdl_enter();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x)
    dw[j] = dCn[off + (long long)j * k + j] * inv;
}

// drho4[s1, s1', s2, s2'] for E = Tr(rho h) / Tr rho with rho[(s1 s2), (s1' s2')] =
// rho4[s1, s1', s2, s2']: dE/drho[I, J] = h[J, I] / t0 - t1 / t0^2 delta_IJ
__global__ void energy_adj_kernel(const double* __restrict__ rho4, const double* __restrict__ h, int d,
                                  double* __restrict__ drho4, double* __restrict__ out) {
  hs_pdl_enter();
  const int n = d * d;
  __shared__ double t[2];
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int I = 0; I < n; ++I)
      for (int J = 0; J < n; ++J) {
        const int s1 = I / d, s2 = I % d, u1 = J / d, u2 = J % d;
        const double r = rho4[((s1 * d + u1) * d + s2) * d + u2];
        if (I == J) t0 += r;
        t1 += r * h[J * n + I];
      }
    t[0] = t0;
    t[1] = t1;
    out[0] = t1 / t0;
    out[1] = t0;
    out[2] = t1;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int I = e / n, J = e % n;
    const int s1 = I / d, s2 = I % d, u1 = J / d, u2 = J % d;
    drho4[((s1 * d + u1) * d + s2) * d + u2] = h[J * n + I] / t[0] - (I == J ? t[1] / (t[0] * t[0]) : 0.0);
  }
}

// ---- the tape ----

struct Arr {
  DBuf v, g;
  long long n = 0;
};

struct Tape {
  hs_ctx ctx;
  std::vector<std::unique_ptr<Arr>> a;
  std::vector<std::function<hs_status()>> back;
  DBuf logs;  // device slots for the normalisation logs
  int nlog = 0;
  std::vector<DBuf*> tmp;

  explicit Tape(hs_ctx c) : ctx(c) {}
  ~Tape() {
    for (auto& x : a) {
      x->v.release();
      x->g.release();
    }
    for (DBuf* t : tmp) {
      t->release();
      delete t;
    }
    logs.release();
  }
  hs_status make(long long n, int* id) {
    auto x = std::make_unique<Arr>();
    x->n = n;
    HS_TRY(x->v.ensure((size_t)std::max<long long>(n, 1) * sizeof(double)));
    *id = (int)a.size();
    a.push_back(std::move(x));
    return HS_OK;
  }
  double* v(int id) { return a[id]->v.d(); }
  double* g(int id) { return a[id]->g.d(); }
  long long n(int id) { return a[id]->n; }
  // a scratch buffer that lives until the tape ends
  hs_status scratch(long long n, double** p) {
    DBuf* b = new DBuf();
    tmp.push_back(b);
    HS_TRY(b->ensure((size_t)std::max<long long>(n, 1) * sizeof(double)));
    *p = b->d();
    return HS_OK;
  }
};

Z2Mat transposed(const Z2Mat& m) { return mat(m.c, m.r, m.pad); }

// out leg j = in leg p[j] for the transpose of a [r-legs | c-legs] layout
void transpose_perm(const Z2Mat& m, int* p) {
  for (int j = 0; j < kMaxLegs; ++j) p[j] = 0;
  for (int j = 0; j < m.c.k; ++j) p[j] = m.r.k + j;
  for (int j = 0; j < m.r.k; ++j) p[m.c.k + j] = j;
}

hs_status permute_p(hs_ctx ctx, const Z2Mat& in, const Z2Mat& out, const int* p, const double* src, double* dst) {
  const PermPlan& plan = cached_plan(ctx, in, out, p);
  HS_CUDA(launch_permute_f64(plan, src, dst, 1.0, ctx->stream));
  if (plan.nbox > 0) ctx->launches += 1;
  return HS_OK;
}

hs_status gemm_acc(hs_ctx ctx, const Z2Mat& Am, const double* A, const Z2Mat& Bm, const double* B, const Z2Mat& Cm,
                   double* C, bool acc) {
  HS_TRY(ctx->splitk.ensure(kSplitKElems * sizeof(double)));
  const GemmGroup g = make_z2_gemm(Am, Bm, Cm);
  HS_CUDA(launch_gemm_f64(g, A, B, C, 1.0, ctx->stream, ctx->splitk.d(), kSplitKElems, acc));
  if (g.n > 0) ctx->launches += 1;
  return HS_OK;
}

// C = A B^T (layouts Am [R|K], Bm [N|K], Cm [R|N]); reverse: dA += dC B, dB += dC^T A
hs_status t_gemm(Tape& t, int A, const Z2Mat& Am, int B, const Z2Mat& Bm, const Z2Mat& Cm, int* C) {
  HS_TRY(t.make(z2_elems(Cm), C));
  HS_TRY(gemm_acc(t.ctx, Am, t.v(A), Bm, t.v(B), Cm, t.v(*C), false));
  const int c = *C;
  t.back.push_back([&t, A, Am, B, Bm, Cm, c]() -> hs_status {
    hs_ctx ctx = t.ctx;
    int p[kMaxLegs];
    double *Bt, *Ct, *At;
    // dA[R|K] += dC[R|N] (B^T)[K|N]^T
    HS_TRY(t.scratch(t.n(B), &Bt));
    transpose_perm(Bm, p);
    HS_TRY(permute_p(ctx, Bm, transposed(Bm), p, t.v(B), Bt));
    HS_TRY(gemm_acc(ctx, Cm, t.g(c), transposed(Bm), Bt, Am, t.g(A), true));
    // dB[N|K] += (dC^T)[N|R] (A^T)[K|R]^T
    HS_TRY(t.scratch(t.n(c), &Ct));
    HS_TRY(t.scratch(t.n(A), &At));
    transpose_perm(Cm, p);
    HS_TRY(permute_p(ctx, Cm, transposed(Cm), p, t.g(c), Ct));
    transpose_perm(Am, p);
    HS_TRY(permute_p(ctx, Am, transposed(Am), p, t.v(A), At));
    HS_TRY(gemm_acc(ctx, transposed(Cm), Ct, transposed(Am), At, Bm, t.g(B), true));
    return HS_OK;
  });
  return HS_OK;
}

// Y = X with legs permuted (out leg j = in leg perm[j]); reverse: dX += inverse permutation of dY
hs_status t_perm(Tape& t, int X, const Z2Mat& in, const Z2Mat& out, std::initializer_list<int> perm, int* Y) {
  int p[kMaxLegs] = {0}, q[kMaxLegs] = {0}, i = 0;
  for (int v : perm) p[i++] = v;
  for (int j = 0; j < i; ++j) q[p[j]] = j;
  HS_TRY(t.make(z2_elems(out), Y));
  HS_TRY(permute_p(t.ctx, in, out, p, t.v(X), t.v(*Y)));
  const int y = *Y;
  std::vector<int> qv(q, q + kMaxLegs);
  t.back.push_back([&t, X, in, out, qv, y]() -> hs_status {
    double* tmp;
    HS_TRY(t.scratch(t.n(X), &tmp));
    HS_TRY(permute_p(t.ctx, out, in, qv.data(), t.g(y), tmp));
    hs_launch(axpy_kernel, grid_of(t.n(X)), 256, 0, t.ctx->stream, t.g(X), (const double*)tmp, t.n(X), 1.0);
    HS_CUDA(cudaGetLastError());
    return HS_OK;
  });
  return HS_OK;
}

// Y = X / max|X|; reverse: dX += dY / m (see the header comment)
hs_status t_norm(Tape& t, int X, int* Y) {
  HS_TRY(t.make(t.n(X), Y));
  const int y = *Y, slot = t.nlog++;
  if (slot >= 4096) return fail(HS_ERR_SHAPE, "too many normalisations on the tape");
  HS_CUDA(cudaMemcpyAsync(t.v(y), t.v(X), (size_t)t.n(X) * sizeof(double), cudaMemcpyDeviceToDevice, t.ctx->stream));
  HS_CUDA(launch_normalize_max_to(t.v(y), t.n(X), static_cast<unsigned long long*>(t.ctx->scratch.p) + 2,
                                  t.logs.d() + slot, t.ctx->stream));
  t.back.push_back([&t, X, y, slot]() -> hs_status {
    hs_launch(add_scaled_kernel, grid_of(t.n(X)), 256, 0, t.ctx->stream, t.g(X), (const double*)t.g(y), t.n(X),
              (const double*)(t.logs.d() + slot));
    HS_CUDA(cudaGetLastError());
    return HS_OK;
  });
  return HS_OK;
}

// The projector step of a move: eigen-decomposition of each parity block of
// C' (layout Cpm, two square blocks n0, n1), the chi states of largest
// |eigenvalue| kept; outputs C_new = diag(kept) / max|kept| (layout [cn|cn])
// and PT (rows: kept eigenvectors, layout [cn|(c,q)]). New sectors in *cn.
hs_status t_eig(Tape& t, int Cp, int n0, int n1, int chi, const Fused& rowm, Sect* cn, int* Cn, int* PT) {
  hs_ctx ctx = t.ctx;
  cudaStream_t s = ctx->stream;
  int V, W;
  const long long nn = (long long)n0 * n0 + (long long)n1 * n1;
  HS_TRY(t.make(nn, &V));
  HS_TRY(t.make(n0 + n1, &W));
  HS_CUDA(cudaMemcpyAsync(t.v(V), t.v(Cp), (size_t)nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  HS_TRY(eig_workspace(ctx, std::max(n0, n1)));
  HS_CUDA(cudaMemsetAsync(ctx->info.p, 0, 2 * sizeof(int), s));
  HS_TRY(eig_pair(ctx, false, t.v(V), n0, t.v(W), t.v(V) + (long long)n0 * n0, n1, t.v(W) + n0));
  HS_TRY(ctx->idx.ensure(2 * (size_t)chi * sizeof(int)));
  HS_TRY(ctx->lam.ensure((size_t)chi * sizeof(double)));
  SelectOut* dsel = static_cast<SelectOut*>(ctx->sel.p);
  HS_CUDA(launch_select(t.v(W), n0, t.v(W) + n0, n1, chi, static_cast<int*>(ctx->idx.p), ctx->lam.d(), dsel, s));
  SelectOut hsel;
  int hinfo[2];
  std::vector<int> hidx(2 * (size_t)chi);
  HS_CUDA(cudaMemcpyAsync(&hsel, dsel, sizeof hsel, cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaMemcpyAsync(hinfo, ctx->info.p, sizeof hinfo, cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaMemcpyAsync(hidx.data(), ctx->idx.p, hidx.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  if (hinfo[0] != 0 || hinfo[1] != 0) return fail(HS_ERR_SOLVER, "syevd info = (%d, %d)", hinfo[0], hinfo[1]);
  if (!(hsel.lam_max > 0.0)) return fail(HS_ERR_NONFINITE, "enlarged corner has no non-zero eigenvalue");
  *cn = make_sect(hsel.chi_new[0], hsel.chi_new[1]);
  const Z2Mat Cnm = mat(fused1(*cn), fused1(*cn)), PTm = mat(fused1(*cn), rowm);
  HS_TRY(t.make(z2_elems(Cnm), Cn));
  HS_TRY(t.make(z2_elems(PTm), PT));
  HS_CUDA(launch_gather_pt(t.v(V), n0, t.v(V) + (long long)n0 * n0, n1, static_cast<int*>(ctx->idx.p), chi, dsel,
                           t.v(*PT), s));
  HS_CUDA(launch_diag_corner(ctx->lam.d(), cn->n[0], cn->n[1], dsel, t.v(*Cn), s));
  ctx->launches += 3;
  // device copy of the picks per block
  int Ix;
  HS_TRY(t.make((2 * (long long)chi + 1) / 2 + 1, &Ix));
  int* didx = reinterpret_cast<int*>(t.v(Ix));
  HS_CUDA(cudaMemcpyAsync(didx, ctx->idx.p, 2 * (size_t)chi * sizeof(int), cudaMemcpyDeviceToDevice, s));
  const int k[2] = {cn->n[0], cn->n[1]}, n[2] = {n0, n1};
  const double inv = 1.0 / hsel.lam_max;
  const int cn_id = *Cn, pt_id = *PT;
  t.back.push_back([&t, Cp, V, W, didx, k, n, chi, inv, cn_id, pt_id]() -> hs_status {
    hs_ctx ctx = t.ctx;
    cudaStream_t s = ctx->stream;
    long long voff = 0, ptoff = 0, coff = 0;
    for (int b = 0; b < 2; ++b) {
      const int nb = n[b], kb = k[b];
      if (nb > 0 && kb > 0) {
        const double* Vb = t.v(V) + voff;  // column-major: row i of Vb (row-major) is eigenvector i
        const double* wb = t.v(W) + (b ? n[0] : 0);
        const double* dPT = t.g(pt_id) + ptoff;
        const double* PTb = t.v(pt_id) + ptoff;
        double *dw, *Wm, *Mm, *VT, *Q, *QT, *PTT, *X;
        HS_TRY(t.scratch(kb, &dw));
        HS_TRY(t.scratch((long long)kb * nb, &Wm));
        HS_TRY(t.scratch((long long)kb * nb, &Mm));
        HS_TRY(t.scratch((long long)nb * nb, &VT));
        HS_TRY(t.scratch((long long)kb * nb, &Q));
        HS_TRY(t.scratch((long long)kb * nb, &QT));
        HS_TRY(t.scratch((long long)kb * nb, &PTT));
        HS_TRY(t.scratch((long long)nb * nb, &X));
        auto dm = [](long long r, long long c) { return mat(fused1(make_sect((int)r, 0)), fused1(make_sect((int)c, 0))); };
        const int tp[kMaxLegs] = {1, 0, 0, 0, 0, 0};
        hs_launch(diag_take_kernel, 1, 256, 0, s, (const double*)t.g(cn_id), coff, kb, inv, dw);
        HS_CUDA(cudaGetLastError());
        // W = dPT V_rm^T (k x n): W[j][i] = dV[:, idx_j] . v_i
        HS_TRY(gemm_acc(ctx, dm(kb, nb), dPT, dm(nb, nb), Vb, dm(kb, nb), Wm, false));
        hs_launch(eig_mix_kernel, grid_of((long long)kb * nb), 256, 0, s, (const double*)Wm, wb,
                  (const int*)(didx + b * chi), (const double*)dw, kb, nb, Mm);
        HS_CUDA(cudaGetLastError());
        // Q = M V_rm (k x n), then X = Q^T PT (n x n) = V (M^T) V_k^T
        HS_TRY(permute_p(ctx, dm(nb, nb), dm(nb, nb), tp, Vb, VT));
        HS_TRY(gemm_acc(ctx, dm(kb, nb), Mm, dm(nb, nb), VT, dm(kb, nb), Q, false));
        HS_TRY(permute_p(ctx, dm(kb, nb), dm(nb, kb), tp, Q, QT));
        HS_TRY(permute_p(ctx, dm(kb, nb), dm(nb, kb), tp, PTb, PTT));
        HS_TRY(gemm_acc(ctx, dm(nb, kb), QT, dm(nb, kb), PTT, dm(nb, nb), X, false));
        hs_launch(sym_add_kernel, grid_of((long long)nb * nb), 256, 0, s, t.g(Cp) + voff, (const double*)X, nb);
        HS_CUDA(cudaGetLastError());
      }
      voff += (long long)nb * nb;
      ptoff += (long long)kb * nb;
      coff += (long long)kb * kb;
    }
    return HS_OK;
  });
  return HS_OK;
}

}  // namespace

extern "C" hs_status hs_ctmrg_energy_grad(hs_ctx ctx, const double* A, int d, int D, hs_basis basis, int chi,
                                          int moves, const double* h, double* energy_out, double* dA_out) {
  HS_TRY(check_ctx(ctx));
  if (!A || !h || !energy_out || !dA_out || d <= 0 || D <= 0 || chi < 1 || moves < 0)
    return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (basis != HS_BASIS_DENSE && basis != HS_BASIS_HERMITIAN) return fail(HS_ERR_INVALID_ARG, "unknown basis");
  cudaStream_t s = ctx->stream;
  const bool herm = basis == HS_BASIS_HERMITIAN;
  const int q = D * D;
  const Sect qs = q_sect(D, basis);
  Tape t(ctx);
  HS_TRY(t.logs.ensure(4096 * sizeof(double)));
  ctx->ws_valid = false;  // the tape's moves are not a warm start for later moves
  const long long nA = (long long)d * D * D * D * D;
  int iA;
  HS_TRY(t.make(nA, &iA));
  HS_CUDA(cudaMemcpyAsync(t.v(iA), A, (size_t)nA * sizeof(double), cudaMemcpyDeviceToDevice, s));
  // ---- double layer in the chosen basis
  const Z2Mat Am = mat(fused2(qs, qs), fused2(qs, qs));
  int ia;
  HS_TRY(t.make(z2_elems(Am), &ia));
  HS_CUDA(launch_double_layer_blocks(t.v(iA), d, D, herm, t.v(ia), s));
  t.back.push_back([&t, iA, ia, d, D, herm, q]() -> hs_status {
    double* plain = t.g(ia);
    if (herm) {
      HS_TRY(t.scratch((long long)q * q * q * q, &plain));
      HS_CUDA(launch_from_hermitian(t.g(ia), D, false, plain, t.ctx->stream));
    }
    HS_CUDA(launch_double_layer_vjp(plain, t.v(iA), d, D, t.g(iA), t.ctx->stream));
    return HS_OK;
  });
  // ---- traced-boundary start
  Sect c = qs;
  int iC, iT;
  {
    const Z2Mat Cm = mat(fused1(c), fused1(c)), Tm = mat(fused2(c, qs), fused1(c));
    int c0, t0;
    HS_TRY(t.make(z2_elems(Cm), &c0));
    HS_TRY(t.make(z2_elems(Tm), &t0));
    HS_CUDA(launch_ctmrg_init(t.v(ia), D, herm, t.v(c0), t.v(t0), s));
    t.back.push_back([&t, ia, c0, t0, D, herm]() -> hs_status {
      HS_CUDA(launch_ctmrg_init_vjp(t.g(c0), t.g(t0), D, herm, t.g(ia), t.ctx->stream));
      return HS_OK;
    });
    HS_TRY(t_norm(t, c0, &iC));
    HS_TRY(t_norm(t, t0, &iT));
  }
  // ---- the moves (the FP64 path of hs_ctmrg_move)
  const Sect qq = qs;
  for (int mv = 0; mv < moves; ++mv) {
    const Z2Mat Tcr = mat(fused2(c, qq), fused1(c)), Cm = mat(fused1(c), fused1(c));
    const Z2Mat X1 = mat(fused2(c, qq), fused1(c)), X2 = mat(fused2(c, qq), fused2(c, qq));
    const Z2Mat X2p = mat(fused2(c, c), fused2(qq, qq)), X3 = mat(fused2(c, c), fused2(qq, qq));
    const Z2Mat Cp = mat(fused2(c, qq), fused2(c, qq));
    int x1, x2, x2p, x3, cp;
    HS_TRY(t_gemm(t, iT, Tcr, iC, Cm, X1, &x1));
    HS_TRY(t_gemm(t, x1, X1, iT, Tcr, X2, &x2));
    HS_TRY(t_perm(t, x2, X2, X2p, {0, 2, 3, 1}, &x2p));
    HS_TRY(t_gemm(t, x2p, X2p, ia, Am, X3, &x3));
    HS_TRY(t_perm(t, x3, X3, Cp, {0, 2, 1, 3}, &cp));
    Sect cn;
    int icn, ipt;
    HS_TRY(t_eig(t, cp, (int)z2_rows(Cp, 0), (int)z2_rows(Cp, 1), chi, fused2(c, qq), &cn, &icn, &ipt));
    const Z2Mat PT = mat(fused1(cn), fused2(c, qq)), Pp = mat(fused2(qq, cn), fused1(c));
    const Z2Mat Y = mat(fused2(qq, cn), fused2(c, qq)), Yp = mat(fused2(cn, c), fused2(qq, qq));
    const Z2Mat Zm = mat(fused2(cn, c), fused2(qq, qq)), Zp = mat(fused2(cn, qq), fused2(c, qq));
    const Z2Mat Tn = mat(fused2(cn, qq), fused1(cn));
    int pp, y, yp, z, zp, tn;
    HS_TRY(t_perm(t, ipt, PT, Pp, {2, 0, 1}, &pp));
    HS_TRY(t_gemm(t, pp, Pp, iT, Tcr, Y, &y));
    HS_TRY(t_perm(t, y, Y, Yp, {1, 2, 0, 3}, &yp));
    HS_TRY(t_gemm(t, yp, Yp, ia, Am, Zm, &z));
    HS_TRY(t_perm(t, z, Zm, Zp, {0, 3, 1, 2}, &zp));
    HS_TRY(t_gemm(t, zp, Zp, ipt, PT, Tn, &tn));
    HS_TRY(t_norm(t, tn, &iT));
    iC = icn;
    c = cn;
  }
  // ---- two-site energy from the dense views of the environment
  const long long ch = c.n[0] + c.n[1];
  auto dl = [](std::initializer_list<long long> rows, std::initializer_list<long long> cols) {
    Fused r = fused0(), cc = fused0();
    for (long long v : rows) r.leg[r.k++] = make_sect((int)v, 0);
    for (long long v : cols) cc.leg[cc.k++] = make_sect((int)v, 0);
    return mat(r, cc);
  };
  int cd, td;
  HS_TRY(t.make(ch * ch, &cd));
  HS_TRY(t.make(ch * q * ch, &td));
  HS_CUDA(launch_env_to_dense(t.v(iC), t.v(iT), D, c.n[0], c.n[1], herm, t.v(cd), t.v(td), s));
  {
    const int c0 = c.n[0], c1 = c.n[1];
    const int ic = iC, it = iT;
    t.back.push_back([&t, cd, td, ic, it, D, c0, c1, herm]() -> hs_status {
      HS_CUDA(launch_env_to_dense_vjp(t.g(cd), t.g(td), D, c0, c1, herm, t.g(ic), t.g(it), t.ctx->stream));
      return HS_OK;
    });
  }
  const long long d2 = (long long)d * d, qx = q;
  int tsw, e1, ct, ee, ep, z1, z1p, z2, z2p, lb, rb, lbp, rbp, rho4, aol, aor;
  HS_TRY(t_perm(t, td, dl({ch, qx}, {ch}), dl({qx, ch}, {ch}), {1, 2, 0}, &tsw));       // Tsw[(x, b) | a]
  HS_TRY(t_gemm(t, cd, dl({ch}, {ch}), tsw, dl({qx, ch}, {ch}), dl({ch}, {qx, ch}), &e1));  // E1[t | (l, a')]
  HS_TRY(t_perm(t, cd, dl({ch}, {ch}), dl({ch}, {ch}), {1, 0}, &ct));                    // C^T
  HS_TRY(t_gemm(t, e1, dl({ch, qx}, {ch}), ct, dl({ch}, {ch}), dl({ch, qx}, {ch}), &ee));  // E[(t, l) | b]
  HS_TRY(t_perm(t, ee, dl({ch, qx}, {ch}), dl({qx, ch}, {ch}), {1, 2, 0}, &ep));         // Ep[(l, b) | t]
  HS_TRY(t_gemm(t, ep, dl({qx, ch}, {ch}), tsw, dl({qx, ch}, {ch}), dl({qx, ch}, {qx, ch}), &z1));
  HS_TRY(t_perm(t, z1, dl({qx, ch}, {qx, ch}), dl({qx, qx, ch}, {ch}), {0, 2, 3, 1}, &z1p));
  HS_TRY(t_gemm(t, z1p, dl({qx, qx, ch}, {ch}), tsw, dl({qx, ch}, {ch}), dl({qx, qx, ch}, {qx, ch}), &z2));
  // open double layers: aoL[(s, s', r) | (l, u, d)], aoR[(s, s', l) | (r, u, d)]
  const long long nao = d2 * qx * qx * qx * qx;
  HS_TRY(t.make(nao, &aol));
  HS_TRY(t.make(nao, &aor));
  HS_CUDA(launch_open_double_layers(t.v(iA), d, D, t.v(aol), t.v(aor), s));
  t.back.push_back([&t, aol, aor, iA, d, D, nA]() -> hs_status {
    double* tmp;
    HS_TRY(t.scratch(nA, &tmp));
    HS_CUDA(launch_open_double_layers_vjp(t.g(aol), t.g(aor), t.v(iA), d, D, tmp, t.ctx->stream));
    hs_launch(axpy_kernel, grid_of(nA), 256, 0, t.ctx->stream, t.g(iA), (const double*)tmp, nA, 1.0);
    HS_CUDA(cudaGetLastError());
    return HS_OK;
  });
  HS_TRY(t_perm(t, z2, dl({qx * qx, ch, qx}, {ch}), dl({ch, ch, qx * qx}, {qx}), {1, 3, 0, 2}, &z2p));
  HS_TRY(t_gemm(t, z2p, dl({ch, ch}, {qx * qx, qx}), aol, dl({d2, qx}, {qx * qx, qx}), dl({ch, ch}, {d2, qx}), &lb));
  HS_TRY(t_gemm(t, z2p, dl({ch, ch}, {qx * qx, qx}), aor, dl({d2, qx}, {qx * qx, qx}), dl({ch, ch}, {d2, qx}), &rb));
  HS_TRY(t_perm(t, lb, dl({ch * ch, d2}, {qx}), dl({d2, ch * ch}, {qx}), {1, 0, 2}, &lbp));
  HS_TRY(t_perm(t, rb, dl({ch * ch, d2}, {qx}), dl({d2, ch * ch}, {qx}), {1, 0, 2}, &rbp));
  HS_TRY(t_gemm(t, lbp, dl({d2}, {ch * ch, qx}), rbp, dl({d2}, {ch * ch, qx}), dl({d2}, {d2}), &rho4));
  // energy and its cotangent (dE = 1)
  double* eout;
  HS_TRY(t.scratch(4, &eout));
  HS_TRY(t.a[rho4]->g.ensure((size_t)t.n(rho4) * sizeof(double)));
  for (auto& x : t.a)
    if (x.get() != t.a[rho4].get()) {
      HS_TRY(x->g.ensure((size_t)std::max<long long>(x->n, 1) * sizeof(double)));
      HS_CUDA(cudaMemsetAsync(x->g.p, 0, (size_t)std::max<long long>(x->n, 1) * sizeof(double), s));
    }
  hs_launch(energy_adj_kernel, 1, 256, 0, s, (const double*)t.v(rho4), h, d, t.g(rho4), eout);
  HS_CUDA(cudaGetLastError());
  // ---- reverse pass
  for (auto it = t.back.rbegin(); it != t.back.rend(); ++it) HS_TRY((*it)());
  HS_CUDA(cudaMemcpyAsync(dA_out, t.g(iA), (size_t)nA * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double he[3];
  HS_CUDA(cudaMemcpyAsync(he, eout, sizeof he, cudaMemcpyDeviceToHost, s));
  HS_CUDA(cudaStreamSynchronize(s));
  *energy_out = he[0];
  if (!std::isfinite(he[0])) return fail(HS_ERR_NONFINITE, "energy is not finite");
  return HS_OK;
}

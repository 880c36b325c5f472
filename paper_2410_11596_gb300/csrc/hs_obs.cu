// Observables of a converged C4v environment (arXiv 2410.11596 Sec. III.A):
// the two-site reduced density matrix of a bond and the one-site environment
// eps of Eq. (4). Both are evaluated once per environment, in FP64, as a chain
// of permutes and GEMMs over the environment expanded to the plain combined
// basis; they need the individual bra and ket tensors, which carry no Z2
// symmetry (Sec. II.B).
//
// Networks (C corner, T edge, * open site):
//   rho:  C T T C / T * * T / C T T C        eps:  C T C / T * T / C T C
#include "hs_ctx.cuh"

using namespace hs;

namespace {

// Open double layer of one site with its physical legs kept:
//   out[(s, s', m) | (c0, u, dd)] = A[s, ...] A[s', ...]
// where m is the open auxiliary leg (right leg r if open_right, else left l)
// and c0 the other horizontal leg; combined index x = ket + D * bra.
__global__ void open_double_layer_kernel(const double* __restrict__ A, int d, int D, bool open_right,
                                         double* __restrict__ out) {
  hs_pdl_enter();
  const int q = D * D;
  const long long total = (long long)d * d * q * q * q * q;
  const long long D4 = (long long)D * D * D * D;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    const int xd = (int)(r % q);
    r /= q;
    const int xu = (int)(r % q);
    r /= q;
    const int xc = (int)(r % q);
    r /= q;
    const int xm = (int)(r % q);
    r /= q;
    const int sb = (int)(r % d);
    const int sk = (int)(r / d);
    const int xl = open_right ? xc : xm, xr = open_right ? xm : xc;
    const long long ik = (((long long)(xu % D) * D + xl % D) * D + xd % D) * D + xr % D;
    const long long ib = (((long long)(xu / D) * D + xl / D) * D + xd / D) * D + xr / D;
    out[e] = A[sk * D4 + ik] * A[sb * D4 + ib];
  }
}

// dA from the cotangents of the two open double layers (layouts of
// open_double_layer_kernel: left site open on r, right site open on l). A
// appears in each as the ket factor (index s) and as the bra factor (s'):
//   dA[p, u, l, d, r] = sum over the other factor's indices of dao * A.
__global__ void open_double_layer_vjp_kernel(const double* __restrict__ daoL, const double* __restrict__ daoR,
                                             const double* __restrict__ A, int d, int D, double* __restrict__ dA) {
  hs_pdl_enter();
  const int q = D * D;
  const long long D4 = (long long)D * D * D * D;
  const long long nA = d * D4;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nA;
       e += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(e / D4);
    long long t = e % D4;
    const int ir = (int)(t % D);
    t /= D;
    const int id = (int)(t % D);
    t /= D;
    const int il = (int)(t % D);
    const int iu = (int)(t / D);
    double acc = 0.0;
    for (int s2 = 0; s2 < d; ++s2)
      for (long long o = 0; o < D4; ++o) {
        long long oo = o;
        const int jr = (int)(oo % D);
        oo /= D;
        const int jd = (int)(oo % D);
        oo /= D;
        const int jl = (int)(oo % D);
        const int ju = (int)(oo / D);
        const double a_other = A[s2 * D4 + o];
        // this element as the ket factor: combined index = mine + D * other
        const int ku = iu + D * ju, kl = il + D * jl, kd = id + D * jd, kr = ir + D * jr;
        // this element as the bra factor: combined index = other + D * mine
        const int bu = ju + D * iu, bl = jl + D * il, bd = jd + D * id, br = jr + D * ir;
        // left site: [(s, s', m = r) | (l, u, d)]; right site: [(s, s', m = l) | (r, u, d)]
        const long long kL = ((((((long long)p * d + s2) * q + kr) * q + kl) * q + ku) * q + kd);
        const long long bL = ((((((long long)s2 * d + p) * q + br) * q + bl) * q + bu) * q + bd);
        const long long kR = ((((((long long)p * d + s2) * q + kl) * q + kr) * q + ku) * q + kd);
        const long long bR = ((((((long long)s2 * d + p) * q + bl) * q + br) * q + bu) * q + bd);
        acc += (daoL[kL] + daoL[bL] + daoR[kR] + daoR[bR]) * a_other;
      }
    dA[e] = acc;
  }
}

// rho[(s1 s2), (s1' s2')] = rho4[s1, s1', s2, s2']; mirror the upper triangle
// when requested; tr[0] = Tr rho, tr[1] = Tr(rho h).
__global__ void finish_rho_kernel(const double* __restrict__ rho4, int d, bool mirror,
                                  const double* __restrict__ h, double* __restrict__ rho,
                                  double* __restrict__ tr) {
  hs_pdl_enter();
  const int n = d * d;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int I = e / n, J = e % n;
    if (mirror && I > J) {
      const int t = I;
      I = J;
      J = t;
    }
    const int s1 = I / d, s2 = I % d, t1 = J / d, t2 = J % d;
    rho[e] = rho4[((s1 * d + t1) * d + s2) * d + t2];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int I = 0; I < n; ++I) {
      t0 += rho[I * n + I];
      if (h)
        for (int J = 0; J < n; ++J) t1 += rho[I * n + J] * h[J * n + I];
    }
    tr[0] = t0;
    tr[1] = t1;
  }
}

// One-site reduced density matrix from the one-site environment eps (plain
// combined basis, legs (u, l, d, r), x = ket + D * bra on every leg):
//   rho1[s, s'] = sum_x eps[x_u, x_l, x_d, x_r] A[s, ket(x)] conj(A[s', bra(x)]),
// one CTA per (s, s'); complex eps, A and rho1 interleaved.
__global__ void one_site_rho_kernel(const double* __restrict__ eps, const double* __restrict__ A, int d, int D,
                                    bool cplx, double* __restrict__ rho) {
  hs_pdl_enter();
  const int sk = blockIdx.x / d, sb = blockIdx.x % d;
  const int q = D * D;
  const long long D4 = (long long)D * D * D * D;
  const long long total = (long long)q * q * q * q;
  double re = 0.0, im = 0.0;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int xr = (int)(e % q), xd = (int)((e / q) % q), xl = (int)((e / q / q) % q), xu = (int)(e / q / q / q);
    const long long ik = (((long long)(xu % D) * D + xl % D) * D + xd % D) * D + xr % D;
    const long long ib = (((long long)(xu / D) * D + xl / D) * D + xd / D) * D + xr / D;
    if (!cplx) {
      re += eps[e] * A[sk * D4 + ik] * A[sb * D4 + ib];
      continue;
    }
    const double kr = A[2 * (sk * D4 + ik)], ki = A[2 * (sk * D4 + ik) + 1];
    const double br = A[2 * (sb * D4 + ib)], bi = -A[2 * (sb * D4 + ib) + 1];  // conj
    const double pr = kr * br - ki * bi, pi = kr * bi + ki * br;
    const double er = eps[2 * e], ei = eps[2 * e + 1];
    re += er * pr - ei * pi;
    im += er * pi + ei * pr;
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x / 32] = re;
    red[1][threadIdx.x / 32] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    if (cplx) {
      rho[2 * blockIdx.x] = a;
      rho[2 * blockIdx.x + 1] = b;
    } else {
      rho[blockIdx.x] = a;
    }
  }
}

// tr[0] = Tr rho1, tr[1] = Tr(rho1 h) (h a real d x d matrix, may be null);
// complex: tr = (Re, Im) of each.
__global__ void finish_rho1_kernel(const double* __restrict__ rho, int d, bool cplx, const double* __restrict__ h,
                                   double* __restrict__ tr) {
  hs_pdl_enter();
  if (threadIdx.x != 0) return;
  double t0r = 0.0, t0i = 0.0, t1r = 0.0, t1i = 0.0;
  for (int i = 0; i < d; ++i) {
    t0r += cplx ? rho[2 * (i * d + i)] : rho[i * d + i];
    t0i += cplx ? rho[2 * (i * d + i) + 1] : 0.0;
    if (h)
      for (int j = 0; j < d; ++j) {
        t1r += (cplx ? rho[2 * (i * d + j)] : rho[i * d + j]) * h[j * d + i];
        t1i += cplx ? rho[2 * (i * d + j) + 1] * h[j * d + i] : 0.0;
      }
  }
  if (cplx) {
    tr[0] = t0r;
    tr[1] = t0i;
    tr[2] = t1r;
    tr[3] = t1i;
  } else {
    tr[0] = t0r;
    tr[1] = t1r;
  }
}

// Cotangent of rho for E = Re Tr(rho h) / Tr rho:
//   drho[I, J] = dE (conj(1 / t0) h[J, I] - conj(t1 / t0^2) delta_IJ),
// t0 = Tr rho, t1 = Tr(rho h) as written by the finish kernels (real: tr =
// (t0, t1); complex: tr = (Re t0, Im t0, Re t1, Im t1), drho interleaved).
__global__ void energy_cotangent_kernel(const double* __restrict__ tr, const double* __restrict__ h, int n,
                                        bool cplx, double dE, double* __restrict__ drho) {
  hs_pdl_enter();
  const double t0r = tr[0], t0i = cplx ? tr[1] : 0.0;
  const double t1r = cplx ? tr[2] : tr[1], t1i = cplx ? tr[3] : 0.0;
  // a = 1 / t0, b = t1 / t0^2 (complex division by |t0|^2)
  const double m2 = t0r * t0r + t0i * t0i;
  const double ar = t0r / m2, ai = -t0i / m2;
  const double sr = ar * ar - ai * ai, si = 2.0 * ar * ai;  // 1 / t0^2
  const double br = t1r * sr - t1i * si, bi = t1r * si + t1i * sr;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int I = e / n, J = e % n;
    const double hv = h ? h[J * n + I] : 0.0;
    // conj(a) hv - conj(b) delta
    const double re = ar * hv - (I == J ? br : 0.0);
    const double im = -ai * hv + (I == J ? bi : 0.0);
    if (cplx) {
      drho[2 * e] = dE * re;
      drho[2 * e + 1] = dE * im;
    } else {
      drho[e] = dE * re;
    }
  }
}

unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// A dense tensor with up to 4 groups of legs as an all-even Z2 matrix.
Z2Mat dense(std::initializer_list<long long> dims) {
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

GemmGroup dense_gemm(long long M, long long N, long long K) {
  GemmGroup g{};
  g.n = 1;
  g.p[0].M = (int)M;
  g.p[0].N = (int)N;
  g.p[0].K = (int)K;
  g.p[0].lda = (int)K;
  g.p[0].ldb = (int)K;
  g.p[0].ldc = (int)N;
  return g;
}

// Complex A (interleaved complex128): open double layer with planar output
//   out[(s, s', m) | (k0, k1, k2)] = A[s, kets] conj(A[s', bras]),
// where (m, k0, k1, k2) are the legs legs[0..3] (0 u, 1 l, 2 d, 3 r) and each
// combined index is x = ket + D * bra.
__global__ void open_double_layer_c_kernel(const double* __restrict__ A, int d, int D, int4 legs,
                                           double* __restrict__ re, double* __restrict__ im) {
  hs_pdl_enter();
  const int q = D * D;
  const long long total = (long long)d * d * q * q * q * q;
  const long long D4 = (long long)D * D * D * D;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    int x[4];
    const int x2 = (int)(r % q);
    r /= q;
    const int x1 = (int)(r % q);
    r /= q;
    const int x0 = (int)(r % q);
    r /= q;
    const int xm = (int)(r % q);
    r /= q;
    const int sb = (int)(r % d);
    const int sk = (int)(r / d);
    x[legs.x] = xm;
    x[legs.y] = x0;
    x[legs.z] = x1;
    x[legs.w] = x2;
    const long long ik = (((long long)(x[0] % D) * D + x[1] % D) * D + x[2] % D) * D + x[3] % D;
    const long long ib = (((long long)(x[0] / D) * D + x[1] / D) * D + x[2] / D) * D + x[3] / D;
    const double kr = A[2 * (sk * D4 + ik)], ki = A[2 * (sk * D4 + ik) + 1];
    const double br = A[2 * (sb * D4 + ib)], bi = A[2 * (sb * D4 + ib) + 1];
    re[e] = kr * br + ki * bi;
    im[e] = ki * br - kr * bi;
  }
}

// Complex rho[(s1 s2), (s1' s2')] = rho4[s1, s1', s2, s2'] (planar in,
// interleaved out); tr[0..1] = Tr rho, tr[2..3] = Tr(rho h) for real h.
__global__ void finish_rho_c_kernel(const double* __restrict__ re4, const double* __restrict__ im4, int d,
                                    const double* __restrict__ h, double* __restrict__ rho, double* __restrict__ tr) {
  hs_pdl_enter();
  const int n = d * d;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int I = e / n, J = e % n;
    const int s1 = I / d, s2 = I % d, t1 = J / d, t2 = J % d;
    const int src = ((s1 * d + t1) * d + s2) * d + t2;
    rho[2 * e] = re4[src];
    rho[2 * e + 1] = im4[src];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0, f = 0.0;
    for (int I = 0; I < n; ++I) {
      a += rho[2 * (I * n + I)];
      b += rho[2 * (I * n + I) + 1];
      if (h)
        for (int J = 0; J < n; ++J) {
          c += rho[2 * (I * n + J)] * h[J * n + I];
          f += rho[2 * (I * n + J) + 1] * h[J * n + I];
        }
    }
    tr[0] = a;
    tr[1] = b;
    tr[2] = c;
    tr[3] = f;
  }
}

struct ZBuf {
  double* re;
  double* im;
};

// planar buffer pair i (0 <= i < 20) of the context, at least n doubles each
ZBuf zbuf(hs_ctx ctx, int i, long long n) {
  if (i < 0 || 2 * i + 1 >= (int)(sizeof(ctx->zr) / sizeof(ctx->zr[0]))) return {nullptr, nullptr};
  if (ctx->zr[2 * i].ensure(n * 8) != HS_OK || ctx->zr[2 * i + 1].ensure(n * 8) != HS_OK) return {nullptr, nullptr};
  return {ctx->zr[2 * i].d(), ctx->zr[2 * i + 1].d()};
}

// complex C = A B^T (or A conj(B)^T) from planar parts: four FP64 GEMMs, two accumulating
hs_status zgemm(hs_ctx ctx, const GemmGroup& g, ZBuf A, ZBuf B, ZBuf C, bool conj_b = false) {
  cudaStream_t s = ctx->stream;
  HS_TRY(ctx->splitk.ensure(kSplitKElems * sizeof(double)));
  double* part = ctx->splitk.d();
  const double sb = conj_b ? -1.0 : 1.0;
  HS_CUDA(launch_gemm_f64(g, A.re, B.re, C.re, 1.0, s, part, kSplitKElems, false));
  HS_CUDA(launch_gemm_f64(g, A.im, B.im, C.re, -sb, s, part, kSplitKElems, true));
  HS_CUDA(launch_gemm_f64(g, A.re, B.im, C.im, sb, s, part, kSplitKElems, false));
  HS_CUDA(launch_gemm_f64(g, A.im, B.re, C.im, 1.0, s, part, kSplitKElems, true));
  ctx->launches += 4;
  return HS_OK;
}

// dA of a complex A from the cotangents g1, g2 of the two open double layers
// (planar; layouts of open_double_layer_c_kernel with legs1 / legs2). For a
// real energy the cotangent convention is g = dE/dRe + i dE/dIm; a site's
// a[s, s', ...] = A[s, ket] conj(A[s', bra]) gives
//   dA[p, mine] += g[p, s', (mine as ket, other as bra)] A[s', other]
//                + conj(g[s, p, (other as ket, mine as bra)]) A[s, other].
__global__ void open_double_layer_c_vjp_kernel(const double* __restrict__ g1r, const double* __restrict__ g1i,
                                               int4 legs1, const double* __restrict__ g2r,
                                               const double* __restrict__ g2i, int4 legs2,
                                               const double* __restrict__ A, int d, int D, double* __restrict__ dA) {
  hs_pdl_enter();
  const int q = D * D;
  const long long D4 = (long long)D * D * D * D;
  const long long nA = d * D4;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nA;
       e += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(e / D4);
    long long t = e % D4;
    int mine[4];
    mine[3] = (int)(t % D);
    t /= D;
    mine[2] = (int)(t % D);
    t /= D;
    mine[1] = (int)(t % D);
    mine[0] = (int)(t / D);
    double ar = 0.0, ai = 0.0;
    for (int s2 = 0; s2 < d; ++s2)
      for (long long o = 0; o < D4; ++o) {
        long long oo = o;
        int oth[4];
        oth[3] = (int)(oo % D);
        oo /= D;
        oth[2] = (int)(oo % D);
        oo /= D;
        oth[1] = (int)(oo % D);
        oth[0] = (int)(oo / D);
        int xk[4], xb[4];
        for (int l = 0; l < 4; ++l) {
          xk[l] = mine[l] + D * oth[l];  // this element as the ket factor
          xb[l] = oth[l] + D * mine[l];  // this element as the bra factor
        }
        const double Or = A[2 * (s2 * D4 + o)], Oi = A[2 * (s2 * D4 + o) + 1];
        for (int site = 0; site < 2; ++site) {
          const int4 L = site ? legs2 : legs1;
          const double* gr = site ? g2r : g1r;
          const double* gi = site ? g2i : g1i;
          const long long ik =
              ((((((long long)p * d + s2) * q + xk[L.x]) * q + xk[L.y]) * q + xk[L.z]) * q + xk[L.w]);
          const long long ib =
              ((((((long long)s2 * d + p) * q + xb[L.x]) * q + xb[L.y]) * q + xb[L.z]) * q + xb[L.w]);
          // g_ket * A_other + conj(g_bra) * A_other
          const double cr = gr[ik] + gr[ib], ci = gi[ik] - gi[ib];
          ar += cr * Or - ci * Oi;
          ai += cr * Oi + ci * Or;
        }
      }
    dA[2 * e] = ar;
    dA[2 * e + 1] = ai;
  }
}

hs_status zpermute(hs_ctx ctx, const Z2Mat& in, const Z2Mat& out, std::initializer_list<int> perm, ZBuf src,
                   ZBuf dst) {
  HS_TRY(permute(ctx, in, out, perm, src.re, dst.re));
  return permute(ctx, in, out, perm, src.im, dst.im);
}

}  // namespace

// Two-site rho of a complex (graded, oriented) environment: the network of
// the oracle's clockwise ring, in complex arithmetic on planar FP64 parts.
// Chain (C, T dense from the graded environment; boundary tensors clockwise):
//   H[a,x,b] = C[a,c] T[c,x,e] C[e,b]
//   L[b,d1,l1,u1,t] = T[b,d1,c] H[c,l1,e] T[e,u1,t]  (also the right chain R[t,u2,r2,d2,b])
//   LB[(b,t)|(s1,s1',m)] = L a1 over (d1,l1,u1); RB[(t,b)|(s2,s2',m)] = L a2 over (u2,r2,d2)
//   rho4[(s1,s1')|(s2,s2')] = sum_{b,t,m} LB RB
hs_status rdm_complex(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, hs_rdm_kind kind,
                      const double* h, double* out, double* tr_out) {
  cudaStream_t s = ctx->stream;
  const long long chi = env->chi_even + env->chi_odd, q = (long long)D * D, d2 = (long long)d * d;
  const long long c2 = chi * chi, cqc = chi * q * chi, c2q2 = c2 * q * q, c2q3 = c2q2 * q;
  // interleaved dense environment, then planar
  HS_TRY(ctx->r[0].ensure(2 * c2 * 8));
  HS_TRY(ctx->r[1].ensure(2 * cqc * 8));
  if (env->basis == HS_BASIS_DENSE) {
    // a complex environment of the plain basis is stored dense already
    HS_CUDA(cudaMemcpyAsync(ctx->r[0].d(), env->C, 2 * c2 * 8, cudaMemcpyDeviceToDevice, s));
    HS_CUDA(cudaMemcpyAsync(ctx->r[1].d(), env->T, 2 * cqc * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    HS_CUDA(launch_env_to_dense_graded(env->C, env->T, D, env->chi_even, env->chi_odd, ctx->r[0].d(), ctx->r[1].d(),
                                       s));
  }
  ZBuf Cz = zbuf(ctx, 0, c2), Tz = zbuf(ctx, 1, cqc), Ctz = zbuf(ctx, 2, c2), Tqz = zbuf(ctx, 3, cqc),
       H1 = zbuf(ctx, 4, cqc), Hz = zbuf(ctx, 5, cqc), Hq = zbuf(ctx, 6, cqc), L1 = zbuf(ctx, 7, c2q2),
       L2 = zbuf(ctx, 8, c2q3), L2p = zbuf(ctx, 9, c2q3);
  if (!L2p.re) return fail(HS_ERR_CUDA, "workspace allocation failed");
  {
    // de-interleave: permute [n | 2] -> [2 | n]
    HS_TRY(ctx->r[2].ensure(2 * cqc * 8));
    HS_TRY(permute(ctx, dense({c2, 2}), dense({2, c2}), {1, 0}, ctx->r[0].d(), ctx->r[2].d()));
    HS_CUDA(cudaMemcpyAsync(Cz.re, ctx->r[2].d(), c2 * 8, cudaMemcpyDeviceToDevice, s));
    HS_CUDA(cudaMemcpyAsync(Cz.im, ctx->r[2].d() + c2, c2 * 8, cudaMemcpyDeviceToDevice, s));
    HS_TRY(permute(ctx, dense({cqc, 2}), dense({2, cqc}), {1, 0}, ctx->r[1].d(), ctx->r[2].d()));
    HS_CUDA(cudaMemcpyAsync(Tz.re, ctx->r[2].d(), cqc * 8, cudaMemcpyDeviceToDevice, s));
    HS_CUDA(cudaMemcpyAsync(Tz.im, ctx->r[2].d() + cqc, cqc * 8, cudaMemcpyDeviceToDevice, s));
  }
  HS_TRY(zpermute(ctx, dense({chi, chi}), dense({chi, chi}), {1, 0}, Cz, Ctz));                 // C^T
  HS_TRY(zpermute(ctx, dense({chi, q, chi}), dense({q, chi, chi}), {1, 2, 0}, Tz, Tqz));       // Tq[(x,e)|c]
  HS_TRY(zgemm(ctx, dense_gemm(chi, q * chi, chi), Cz, Tqz, H1));                               // H1[a|(x,e)]
  HS_TRY(zgemm(ctx, dense_gemm(chi * q, chi, chi), H1, Ctz, Hz));                               // H[(a,x)|b]
  HS_TRY(zpermute(ctx, dense({chi, q, chi}), dense({q, chi, chi}), {1, 2, 0}, Hz, Hq));        // Hq[(l,e)|c]
  if (kind == HS_RDM_ENV_ONE_SITE) {
    // eps[u,l,d,r] = H[a,u,b] T[b,r,b'] H[b',d,a'] T[a',l,a] (the clockwise ring of Eq. (4))
    ZBuf Y1 = zbuf(ctx, 7, c2q2), Y2 = zbuf(ctx, 8, c2q3), Y2p = zbuf(ctx, 9, c2q3), Tl = zbuf(ctx, 10, cqc),
         E3 = zbuf(ctx, 11, q * q * q * q);
    if (!E3.re) return fail(HS_ERR_CUDA, "workspace allocation failed");
    HS_TRY(zgemm(ctx, dense_gemm(chi * q, q * chi, chi), Hz, Tqz, Y1));                        // [(a,u)|(r,b')]
    HS_TRY(zgemm(ctx, dense_gemm(chi * q * q, q * chi, chi), Y1, Hq, Y2));                     // [(a,u,r)|(d,a')]
    HS_TRY(zpermute(ctx, dense({chi, q, q, q, chi}), dense({q, q, q, chi, chi}), {1, 2, 3, 4, 0}, Y2, Y2p));
    HS_TRY(zpermute(ctx, dense({chi, q, chi}), dense({q, chi, chi}), {1, 0, 2}, Tz, Tl));      // Tl[l|(a',a)]
    HS_TRY(zgemm(ctx, dense_gemm(q * q * q, q, chi * chi), Y2p, Tl, E3));                       // [(u,r,d)|l]
    // eps[u,l,d,r] (interleaved complex): permute each part, then interleave
    ZBuf Eo = zbuf(ctx, 12, q * q * q * q);
    if (!Eo.re) return fail(HS_ERR_CUDA, "workspace allocation failed");
    HS_TRY(zpermute(ctx, dense({q, q, q, q}), dense({q, q, q, q}), {0, 3, 2, 1}, E3, Eo));
    const long long n4 = q * q * q * q;
    HS_TRY(ctx->r[2].ensure(2 * n4 * 8));
    HS_CUDA(cudaMemcpyAsync(ctx->r[2].d(), Eo.re, n4 * 8, cudaMemcpyDeviceToDevice, s));
    HS_CUDA(cudaMemcpyAsync(ctx->r[2].d() + n4, Eo.im, n4 * 8, cudaMemcpyDeviceToDevice, s));
    return permute(ctx, dense({2, n4}), dense({n4, 2}), {1, 0}, ctx->r[2].d(), out);
  }
  HS_TRY(zgemm(ctx, dense_gemm(chi * q, q * chi, chi), Tz, Hq, L1));                            // L1[(b,d1)|(l1,e)]
  HS_TRY(zgemm(ctx, dense_gemm(chi * q * q, q * chi, chi), L1, Tqz, L2));                       // L2[(b,d1,l1)|(u1,t)]
  HS_TRY(zpermute(ctx, dense({chi, q, q, q, chi}), dense({chi, chi, q, q, q}), {0, 4, 1, 2, 3}, L2, L2p));
  // open double layers: a1[(s,s',r) | (d,l,u)], a2[(s,s',l) | (u,r,d)]
  const long long nao = d2 * q * q * q * q;
  ZBuf a1 = zbuf(ctx, 10, nao), a2 = zbuf(ctx, 11, nao);
  if (!a2.re) return fail(HS_ERR_CUDA, "workspace allocation failed");
  hs_launch(open_double_layer_c_kernel, grid_for(nao), 256, 0, s, A, d, D, make_int4(3, 2, 1, 0), a1.re, a1.im);
  HS_CUDA(cudaGetLastError());
  hs_launch(open_double_layer_c_kernel, grid_for(nao), 256, 0, s, A, d, D, make_int4(1, 0, 3, 2), a2.re, a2.im);
  HS_CUDA(cudaGetLastError());
  ctx->launches += 2;
  ZBuf LB = zbuf(ctx, 1, c2 * d2 * q), RB = zbuf(ctx, 2, c2 * d2 * q);  // reuse (T, C^T no longer needed)
  ZBuf LBp = zbuf(ctx, 4, c2 * d2 * q), RBp = zbuf(ctx, 5, c2 * d2 * q), R4 = zbuf(ctx, 0, d2 * d2);
  if (!R4.re) return fail(HS_ERR_CUDA, "workspace allocation failed");
  HS_TRY(zgemm(ctx, dense_gemm(c2, d2 * q, q * q * q), L2p, a1, LB));                           // LB[(b,t)|(s,s',m)]
  HS_TRY(zgemm(ctx, dense_gemm(c2, d2 * q, q * q * q), L2p, a2, RB));                           // RB[(t,b)|(s,s',m)]
  HS_TRY(zpermute(ctx, dense({chi, chi, d, d, q}), dense({d, d, chi, chi, q}), {2, 3, 0, 1, 4}, LB, LBp));
  HS_TRY(zpermute(ctx, dense({chi, chi, d, d, q}), dense({d, d, chi, chi, q}), {2, 3, 1, 0, 4}, RB, RBp));
  HS_TRY(zgemm(ctx, dense_gemm(d2, d2, c2 * q), LBp, RBp, R4));                                 // rho4
  hs_launch(finish_rho_c_kernel, 1, 256, 0, s, R4.re, R4.im, d, h, out, tr_out);
  HS_CUDA(cudaGetLastError());
  ctx->launches += 1;
  return HS_OK;
}

// Adjoint of rdm_complex with the environment fixed: drho (interleaved
// complex d^4, cotangent dE/dRe rho + i dE/dIm rho) -> dA (interleaved complex).
hs_status rdm_vjp_complex(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, const double* drho,
                          double* dA_out) {
  cudaStream_t s = ctx->stream;
  const long long chi = env->chi_even + env->chi_odd, q = (long long)D * D, d2 = (long long)d * d;
  const long long c2 = chi * chi, c2q3 = c2 * q * q * q, nb = c2 * d2 * q;
  // forward: leaves L2p (slot 9), LB (1), RB (2), LBp (4), RBp (5)
  HS_TRY(ctx->r[3].ensure(2 * d2 * d2 * 8 + 4 * 8));
  HS_TRY(rdm_complex(ctx, env, A, d, D, HS_RDM_TWO_SITE, nullptr, ctx->r[3].d(), ctx->r[3].d() + 2 * d2 * d2));
  ZBuf L2p = zbuf(ctx, 9, c2q3), LBp = zbuf(ctx, 4, nb), RBp = zbuf(ctx, 5, nb);
  // cotangent of rho4[s1, s1', s2, s2'] and of its transpose
  ZBuf G = zbuf(ctx, 12, d2 * d2), G4 = zbuf(ctx, 13, d2 * d2), G4t = zbuf(ctx, 14, d2 * d2);
  if (!G4t.re) return fail(HS_ERR_CUDA, "workspace allocation failed");
  HS_TRY(ctx->r[4].ensure(2 * d2 * d2 * 8));
  HS_TRY(permute(ctx, dense({d2 * d2, 2}), dense({2, d2 * d2}), {1, 0}, drho, ctx->r[4].d()));
  HS_CUDA(cudaMemcpyAsync(G.re, ctx->r[4].d(), d2 * d2 * 8, cudaMemcpyDeviceToDevice, s));
  HS_CUDA(cudaMemcpyAsync(G.im, ctx->r[4].d() + d2 * d2, d2 * d2 * 8, cudaMemcpyDeviceToDevice, s));
  HS_TRY(zpermute(ctx, dense({d, d, d, d}), dense({d, d, d, d}), {0, 2, 1, 3}, G, G4));
  HS_TRY(zpermute(ctx, dense({d2, d2}), dense({d2, d2}), {1, 0}, G4, G4t));
  // gLBp = G4 conj(RBp), gRBp = G4^T conj(LBp): B operands transposed to [(b,t,m) | (s,s')]
  ZBuf RBq = zbuf(ctx, 15, nb), LBq = zbuf(ctx, 16, nb), gLBp = zbuf(ctx, 17, nb), gRBp = zbuf(ctx, 18, nb);
  if (!gRBp.re) return fail(HS_ERR_CUDA, "workspace allocation failed");
  HS_TRY(zpermute(ctx, dense({d2, c2 * q}), dense({c2 * q, d2}), {1, 0}, RBp, RBq));
  HS_TRY(zpermute(ctx, dense({d2, c2 * q}), dense({c2 * q, d2}), {1, 0}, LBp, LBq));
  HS_TRY(zgemm(ctx, dense_gemm(d2, c2 * q, d2), G4, RBq, gLBp, true));
  HS_TRY(zgemm(ctx, dense_gemm(d2, c2 * q, d2), G4t, LBq, gRBp, true));
  // back to [(s, s', m) | (b, t)] and [(s, s', m) | (t, b)] (LB rows (b,t), RB rows (t,b))
  ZBuf gLm = zbuf(ctx, 15, nb), gRm = zbuf(ctx, 16, nb);
  HS_TRY(zpermute(ctx, dense({d, d, chi, chi, q}), dense({d, d, q, chi, chi}), {0, 1, 4, 2, 3}, gLBp, gLm));
  HS_TRY(zpermute(ctx, dense({d, d, chi, chi, q}), dense({d, d, q, chi, chi}), {0, 1, 4, 3, 2}, gRBp, gRm));
  // open double layers: g_a = g_B^T conj(L2p) with L2p^T[(k0,k1,k2) | (x0, x4)]
  ZBuf L2pT = zbuf(ctx, 8, c2q3);
  if (!L2pT.re) return fail(HS_ERR_CUDA, "workspace allocation failed");
  HS_TRY(zpermute(ctx, dense({c2, q * q * q}), dense({q * q * q, c2}), {1, 0}, L2p, L2pT));
  const long long nao = d2 * q * q * q * q;
  ZBuf g1 = zbuf(ctx, 10, nao), g2 = zbuf(ctx, 11, nao);
  HS_TRY(zgemm(ctx, dense_gemm(d2 * q, q * q * q, c2), gLm, L2pT, g1, true));
  HS_TRY(zgemm(ctx, dense_gemm(d2 * q, q * q * q, c2), gRm, L2pT, g2, true));
  const long long nA = (long long)d * D * D * D * D;
  hs_launch(open_double_layer_c_vjp_kernel, grid_for(nA), 256, 0, s, g1.re, g1.im, make_int4(3, 2, 1, 0), g2.re, g2.im,
                                                               make_int4(1, 0, 3, 2), A, d, D, dA_out);
  HS_CUDA(cudaGetLastError());
  ctx->launches += 1;
  return HS_OK;
}

// Shared forward chain of the two-site network up to the half-network blocks:
// on return r[8] = Z2 [(l,u,t')|(d,b')], r[9] = Z2p [(t',b')|(l,u,d)],
// r[10]/r[11] = open double layers of the left/right site, r[12]/r[13] =
// LB/RB [(t',b')|(s,s',m)], r[14]/r[15] = LBp/RBp [(s,s')|(t',b',m)],
// r[6] = rho4 [(s1,s1')|(s2,s2')]. kind selects how far it goes.
hs_status rdm_chain(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, hs_rdm_kind kind,
                    double* eps_out) {
  cudaStream_t s = ctx->stream;
  const hs_gemm_backend be = env->gemm_backend;
  const long long chi = env->chi_even + env->chi_odd, q = (long long)D * D;
  const long long c2 = chi * chi, cqc = chi * q * chi, c2q2 = c2 * q * q, c2q3 = c2q2 * q;
  DBuf* r = ctx->r;
  HS_TRY(r[0].ensure(c2 * 8));
  HS_TRY(r[1].ensure(cqc * 8));
  HS_TRY(r[2].ensure(cqc * 8));
  HS_TRY(r[3].ensure(cqc * 8));
  HS_TRY(r[4].ensure(cqc * 8));
  HS_TRY(r[5].ensure(cqc * 8));
  HS_TRY(r[6].ensure((c2q2 > c2 ? c2q2 : c2) * 8));
  HS_TRY(r[7].ensure(c2q2 * 8));
  HS_TRY(r[8].ensure(c2q3 * 8));
  HS_TRY(r[9].ensure(c2q3 * 8));
  double *Cd = r[0].d(), *Td = r[1].d(), *Tsw = r[2].d(), *E1 = r[3].d(), *E = r[4].d(),
         *Ep = r[5].d(), *Z1 = r[6].d(), *Z1p = r[7].d(), *Z2 = r[8].d(), *Z2p = r[9].d();

  // environment in the plain combined basis
  HS_CUDA(launch_env_to_dense(env->C, env->T, D, env->chi_even, env->chi_odd,
                              env->basis == HS_BASIS_HERMITIAN, Cd, Td, s));
  // Tsw[(x, b) | a] = T[a, x, b]
  HS_TRY(permute(ctx, dense({chi, q, chi}), dense({q, chi, chi}), {1, 2, 0}, Td, Tsw));
  // half ring E[t, l, b] = C[t, a] T[a, l, a'] C[a', b]
  HS_TRY(gemm(ctx, be, dense_gemm(chi, q * chi, chi), Cd, Tsw, E1));          // E1[t | (l, a')]
  HS_TRY(permute(ctx, dense({chi, chi}), dense({chi, chi}), {1, 0}, Cd, Z1));  // C^T in Z1
  HS_TRY(gemm(ctx, be, dense_gemm(chi * q, chi, chi), E1, Z1, E));             // E[(t, l) | b]
  // Z1[l, b, u, t'] = E[t, l, b] T[t, u, t']
  HS_TRY(permute(ctx, dense({chi, q, chi}), dense({q, chi, chi}), {1, 2, 0}, E, Ep));   // Ep[(l,b)|t]
  HS_TRY(gemm(ctx, be, dense_gemm(q * chi, q * chi, chi), Ep, Tsw, Z1));
  // Z2[l, u, t', d, b'] = Z1[l, b, u, t'] T[b, d, b']
  HS_TRY(permute(ctx, dense({q, chi, q, chi}), dense({q, q, chi, chi}), {0, 2, 3, 1}, Z1, Z1p));
  HS_TRY(gemm(ctx, be, dense_gemm(q * q * chi, q * chi, chi), Z1p, Tsw, Z2));

  if (kind == HS_RDM_ENV_ONE_SITE) {
    // Z2 plays Y2[u, l, a', r, b']; eps[u,l,r,d] = Y2[u,l,a',r,b'] H[a',d,b'], H = E
    HS_TRY(r[12].ensure(cqc * 8));
    HS_TRY(r[13].ensure(q * q * q * q * 8));
    HS_TRY(permute(ctx, dense({q * q, chi, q, chi}), dense({q * q, q, chi, chi}), {0, 2, 1, 3}, Z2, Z2p));
    HS_TRY(permute(ctx, dense({chi, q, chi}), dense({q, chi, chi}), {1, 0, 2}, E, r[12].d()));  // Hd[d|(a',b')]
    HS_TRY(gemm(ctx, be, dense_gemm(q * q * q, q, chi * chi), Z2p, r[12].d(), r[13].d()));     // [(u,l,r)|d]
    HS_TRY(permute(ctx, dense({q * q, q, q}), dense({q * q, q, q}), {0, 2, 1}, r[13].d(), eps_out));
    return HS_OK;
  }

  const long long d2 = (long long)d * d;
  HS_TRY(r[10].ensure(d2 * q * q * q * q * 8));
  HS_TRY(r[11].ensure(d2 * q * q * q * q * 8));
  HS_TRY(r[12].ensure(c2 * d2 * q * 8));
  HS_TRY(r[13].ensure(c2 * d2 * q * 8));
  HS_TRY(r[14].ensure(c2 * d2 * q * 8));
  HS_TRY(r[15].ensure(c2 * d2 * q * 8));
  double *aoL = r[10].d(), *aoR = r[11].d(), *LB = r[12].d(), *RB = r[13].d(), *LBp = r[14].d(),
         *RBp = r[15].d();
  const long long nao = d2 * q * q * q * q;
  hs_launch(open_double_layer_kernel, grid_for(nao), 256, 0, s, A, d, D, true, aoL);
  HS_CUDA(cudaGetLastError());
  hs_launch(open_double_layer_kernel, grid_for(nao), 256, 0, s, A, d, D, false, aoR);
  HS_CUDA(cudaGetLastError());
  // Z2p[(t', b') | (l, u, d)]
  HS_TRY(permute(ctx, dense({q * q, chi, q, chi}), dense({chi, chi, q * q, q}), {1, 3, 0, 2}, Z2, Z2p));
  // LB[(t', b') | (s, s', m)] over (l, u, d); RB over (r, u, d) of the mirror site
  HS_TRY(gemm(ctx, be, dense_gemm(c2, d2 * q, q * q * q), Z2p, aoL, LB));
  HS_TRY(gemm(ctx, be, dense_gemm(c2, d2 * q, q * q * q), Z2p, aoR, RB));
  // [(s, s') | (t', b', m)]
  HS_TRY(permute(ctx, dense({c2, d2, q}), dense({d2, c2, q}), {1, 0, 2}, LB, LBp));
  HS_TRY(permute(ctx, dense({c2, d2, q}), dense({d2, c2, q}), {1, 0, 2}, RB, RBp));
  HS_TRY(gemm(ctx, be, dense_gemm(d2, d2, c2 * q), LBp, RBp, Z1));  // rho4[(s1,s1') | (s2,s2')]
  return HS_OK;
}

static hs_status rdm_vjp_after_chain(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, const double* drho,
                                     double* dA_out);

namespace hs {
// The open double layers of the two-site network (left site open on r, right
// site open on l) and their adjoint, for the gradient through the iterations.
cudaError_t launch_open_double_layers(const double* A, int d, int D, double* aoL, double* aoR, cudaStream_t s) {
  const long long q = (long long)D * D, nao = (long long)d * d * q * q * q * q;
  hs_launch(open_double_layer_kernel, grid_for(nao), 256, 0, s, A, d, D, true, aoL);
  hs_launch(open_double_layer_kernel, grid_for(nao), 256, 0, s, A, d, D, false, aoR);
  return cudaGetLastError();
}
cudaError_t launch_open_double_layers_vjp(const double* daoL, const double* daoR, const double* A, int d, int D,
                                          double* dA, cudaStream_t s) {
  const long long nA = (long long)d * D * D * D * D;
  hs_launch(open_double_layer_vjp_kernel, grid_for(nA), 256, 0, s, daoL, daoR, A, d, D, dA);
  return cudaGetLastError();
}
}  // namespace hs

extern "C" hs_status hs_rdm(hs_ctx ctx, const hs_env* env, const double* A, int d, int D,
                            hs_dtype dtype, hs_rdm_kind kind, const double* h, double* out,
                            double* tr_out) {
  HS_TRY(check_ctx(ctx));
  if (!env || !A || !out || d <= 0 || D != env->D) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (dtype != HS_F64 && dtype != HS_C128) return fail(HS_ERR_DTYPE, "unknown dtype");
  if (kind != HS_RDM_TWO_SITE && kind != HS_RDM_ENV_ONE_SITE && kind != HS_RDM_ONE_SITE)
    return fail(HS_ERR_INVALID_ARG, "unknown rdm kind");
  if (kind != HS_RDM_ENV_ONE_SITE && !tr_out) return fail(HS_ERR_INVALID_ARG, "tr_out is required");
  if ((dtype == HS_C128) != (env->dtype == HS_C128)) return fail(HS_ERR_DTYPE, "A and environment disagree on dtype");
  if (kind == HS_RDM_ONE_SITE) {
    // eps first (workspace), then the contraction with A and conj(A)
    const bool cplx = dtype == HS_C128;
    const long long q = (long long)D * D, n4 = q * q * q * q;
    DBuf& eps = ctx->hb[11];
    HS_TRY(eps.ensure((size_t)n4 * (cplx ? 2 : 1) * sizeof(double)));
    if (cplx)
      HS_TRY(rdm_complex(ctx, env, A, d, D, HS_RDM_ENV_ONE_SITE, nullptr, eps.d(), nullptr));
    else
      HS_TRY(rdm_chain(ctx, env, A, d, D, HS_RDM_ENV_ONE_SITE, eps.d()));
    hs_launch(one_site_rho_kernel, d * d, 256, 0, ctx->stream, eps.d(), A, d, D, cplx, out);
    HS_CUDA(cudaGetLastError());
    hs_launch(finish_rho1_kernel, 1, 32, 0, ctx->stream, out, d, cplx, h, tr_out);
    HS_CUDA(cudaGetLastError());
    ctx->launches += 2;
    return HS_OK;
  }
  if (dtype == HS_C128) return rdm_complex(ctx, env, A, d, D, kind, h, out, tr_out);
  HS_TRY(rdm_chain(ctx, env, A, d, D, kind, out));
  if (kind == HS_RDM_ENV_ONE_SITE) return HS_OK;
  hs_launch(finish_rho_kernel, 1, 256, 0, ctx->stream, ctx->r[6].d(), d, env->basis == HS_BASIS_HERMITIAN, h, out,
                                                tr_out);
  HS_CUDA(cudaGetLastError());
  return HS_OK;
}

extern "C" hs_status hs_rdm_vjp(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, hs_dtype dtype,
                                const double* drho, double* dA_out) {
  HS_TRY(check_ctx(ctx));
  if (!env || !A || !drho || !dA_out || d <= 0 || D != env->D) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (dtype != HS_F64 && dtype != HS_C128) return fail(HS_ERR_DTYPE, "unknown dtype");
  if ((dtype == HS_C128) != (env->dtype == HS_C128)) return fail(HS_ERR_DTYPE, "A and environment disagree on dtype");
  if (dtype == HS_C128) return rdm_vjp_complex(ctx, env, A, d, D, drho, dA_out);
  HS_TRY(rdm_chain(ctx, env, A, d, D, HS_RDM_TWO_SITE, nullptr));
  return rdm_vjp_after_chain(ctx, env, A, d, D, drho, dA_out);
}

extern "C" hs_status hs_energy_vjp(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, hs_dtype dtype,
                                   const double* h, double dE, double* dA_out) {
  HS_TRY(check_ctx(ctx));
  if (!env || !A || !h || !dA_out || d <= 0 || D != env->D) return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (dtype != HS_F64 && dtype != HS_C128) return fail(HS_ERR_DTYPE, "unknown dtype");
  if ((dtype == HS_C128) != (env->dtype == HS_C128)) return fail(HS_ERR_DTYPE, "A and environment disagree on dtype");
  const bool cplx = dtype == HS_C128;
  const int n = d * d;
  // rho (scratch), its traces, the cotangent
  DBuf& w = ctx->hb[12];
  HS_TRY(w.ensure((size_t)(2 * n * n * (cplx ? 2 : 1) + 8) * sizeof(double)));
  double* rho = w.d();
  double* drho = rho + (long long)n * n * (cplx ? 2 : 1);
  double* tr = drho + (long long)n * n * (cplx ? 2 : 1);
  if (cplx) {
    HS_TRY(rdm_complex(ctx, env, A, d, D, HS_RDM_TWO_SITE, h, rho, tr));
  } else {
    HS_TRY(rdm_chain(ctx, env, A, d, D, HS_RDM_TWO_SITE, nullptr));
    hs_launch(finish_rho_kernel, 1, 256, 0, ctx->stream, ctx->r[6].d(), d, env->basis == HS_BASIS_HERMITIAN, h, rho,
              tr);
    HS_CUDA(cudaGetLastError());
  }
  hs_launch(energy_cotangent_kernel, 1, 256, 0, ctx->stream, (const double*)tr, h, n, cplx, dE, drho);
  HS_CUDA(cudaGetLastError());
  ctx->launches += 2;
  if (cplx) return rdm_vjp_complex(ctx, env, A, d, D, drho, dA_out);
  return rdm_vjp_after_chain(ctx, env, A, d, D, drho, dA_out);
}

// Reverse pass of the real two-site chain; rdm_chain(HS_RDM_TWO_SITE) must have
// run on the same environment and A just before (its buffers r[8..15]).
static hs_status rdm_vjp_after_chain(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, const double* drho,
                                     double* dA_out) {
  cudaStream_t s = ctx->stream;
  const hs_gemm_backend be = env->gemm_backend;
  const long long chi = env->chi_even + env->chi_odd, q = (long long)D * D, c2 = chi * chi,
                  d2 = (long long)d * d;
  DBuf* r = ctx->r;
  double *Z2 = r[8].d(), *Z2p = r[9].d(), *LB = r[12].d(), *RB = r[13].d();
  // rho[(s1 s2), (s1' s2')] = rho4[s1, s1', s2, s2']: cotangent of rho4 and its transpose
  HS_TRY(ctx->hb[0].ensure(2 * d2 * d2 * 8));
  double* drho4 = ctx->hb[0].d();
  double* drho4T = drho4 + d2 * d2;
  HS_TRY(permute(ctx, dense({d, d, d, d}), dense({d, d, d, d}), {0, 2, 1, 3}, drho, drho4));
  HS_TRY(permute(ctx, dense({d2, d2}), dense({d2, d2}), {1, 0}, drho4, drho4T));
  // RBq/LBq[(t', b', m) | (s, s')]
  HS_TRY(ctx->hb[1].ensure(c2 * d2 * q * 8));
  HS_TRY(ctx->hb[2].ensure(c2 * d2 * q * 8));
  HS_TRY(ctx->hb[3].ensure(c2 * d2 * q * 8));
  HS_TRY(ctx->hb[4].ensure(c2 * d2 * q * 8));
  double *LBq = ctx->hb[1].d(), *RBq = ctx->hb[2].d(), *dLB = ctx->hb[3].d(), *dRB = ctx->hb[4].d();
  HS_TRY(permute(ctx, dense({c2, d2, q}), dense({c2, q, d2}), {0, 2, 1}, LB, LBq));
  HS_TRY(permute(ctx, dense({c2, d2, q}), dense({c2, q, d2}), {0, 2, 1}, RB, RBq));
  // dLB[(s1,s1') | (t',b',m)] = drho4 RB ; dRB[(s2,s2') | (t',b',m)] = drho4^T LB
  HS_TRY(gemm(ctx, be, dense_gemm(d2, c2 * q, d2), drho4, RBq, dLB));
  HS_TRY(gemm(ctx, be, dense_gemm(d2, c2 * q, d2), drho4T, LBq, dRB));
  // [(s, s', m) | (t', b')]
  HS_TRY(ctx->hb[5].ensure(c2 * d2 * q * 8));
  HS_TRY(ctx->hb[6].ensure(c2 * d2 * q * 8));
  double *dLBm = ctx->hb[5].d(), *dRBm = ctx->hb[6].d();
  HS_TRY(permute(ctx, dense({d2, c2, q}), dense({d2, q, c2}), {0, 2, 1}, dLB, dLBm));
  HS_TRY(permute(ctx, dense({d2, c2, q}), dense({d2, q, c2}), {0, 2, 1}, dRB, dRBm));
  // Z2t[(l, u, d) | (t', b')] from Z2[(l,u), t', d, b']
  HS_TRY(permute(ctx, dense({q * q, chi, q, chi}), dense({q * q, q, chi, chi}), {0, 2, 1, 3}, Z2, Z2p));
  // cotangents of the open double layers: dao[(s, s', m) | (c0, u, d)]
  const long long nao = d2 * q * q * q * q;
  HS_TRY(ctx->hb[7].ensure(nao * 8));
  HS_TRY(ctx->hb[8].ensure(nao * 8));
  HS_TRY(gemm(ctx, be, dense_gemm(d2 * q, q * q * q, c2), dLBm, Z2p, ctx->hb[7].d()));
  HS_TRY(gemm(ctx, be, dense_gemm(d2 * q, q * q * q, c2), dRBm, Z2p, ctx->hb[8].d()));
  const long long nA = (long long)d * D * D * D * D;
  hs_launch(open_double_layer_vjp_kernel, grid_for(nA), 256, 0, s, ctx->hb[7].d(), ctx->hb[8].d(), A, d, D, dA_out);
  HS_CUDA(cudaGetLastError());
  return HS_OK;
}

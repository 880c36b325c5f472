// Small kernels of the C4v CTMRG move (arXiv 2410.11596 Sec. II.A, Fig. 1(d)):
// traced-boundary initialisation, selection of the kept eigenvalues across the
// two parity blocks, projector gather, corner/edge normalisation, and the
// dense view of an environment.
#include <cmath>

#include "hs_internal.cuh"

namespace hs {

namespace {

unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// Position of T[alpha, x, beta] in FSO [(alpha, x) | beta]; -1 if odd total.
__device__ __forceinline__ long long t_pos(int pa, int ia, int px, int ix, int pb, int ib, Sect c,
                                           Sect q) {
  if ((pa + px + pb) & 1) return -1;
  const Fused R = fused2(c, q);
  const int tr = (pa << 1) | px;
  const int P = pb;
  const long long CP = c.n[P];
  const long long row = tuple_offset(R, tr) + (long long)ia * q.n[px] + ix;
  const long long off = P ? fused_size(R, 0) * (long long)c.n[0] : 0;
  return off + row * CP + ib;
}

// Position of a[u, l, d, r] in FSO [(u, l) | (d, r)] (all legs sectors q).
__device__ __forceinline__ long long a_pos(int pu, int iu, int pl, int il, int pd, int id, int pr,
                                           int ir, Sect q) {
  if ((pu + pl + pd + pr) & 1) return -1;
  const Fused f = fused2(q, q);
  const int tr = (pu << 1) | pl, tc = (pd << 1) | pr;
  const int P = tuple_parity(tr);
  const long long CP = fused_size(f, P);
  const long long row = tuple_offset(f, tr) + (long long)iu * q.n[pl] + il;
  const long long col = tuple_offset(f, tc) + (long long)id * q.n[pr] + ir;
  const long long off = P ? fused_size(f, 0) * fused_size(f, 0) : 0;
  return off + row * CP + col;
}

// Traced state k of one leg: Hermitian basis index k (even), or the plain
// combined index k + D k (dense basis, a single all-even sector).
__device__ __forceinline__ int traced_local(int k, int D, bool hermitian) {
  return hermitian ? k : k * (D + 1);
}

__global__ void init_T_kernel(const double* __restrict__ a, int D, bool hermitian,
                              double* __restrict__ T) {
  hs_pdl_enter();
  const int q = D * D;
  const int qe = hermitian ? D * (D + 1) / 2 : q;
  const Sect s = make_sect(qe, q - qe);
  const long long total = (long long)q * q * q;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int u = (int)(e % q), r = (int)((e / q) % q), dd = (int)(e / q / q);
    const int pd = dd >= qe, pr = r >= qe, pu = u >= qe;
    const long long pos = t_pos(pd, dd - pd * qe, pr, r - pr * qe, pu, u - pu * qe, s, s);
    if (pos < 0) continue;
    double acc = 0.0;
    for (int k = 0; k < D; ++k) {
      const long long ap = a_pos(pu, u - pu * qe, 0, traced_local(k, D, hermitian), pd, dd - pd * qe,
                                 pr, r - pr * qe, s);
      acc += a[ap];
    }
    T[pos] = acc;  // T0[alpha = d, x = r, beta = u]
  }
}

__global__ void init_C_kernel(const double* __restrict__ a, int D, bool hermitian,
                              double* __restrict__ C) {
  hs_pdl_enter();
  const int q = D * D;
  const int qe = hermitian ? D * (D + 1) / 2 : q;
  const Sect s = make_sect(qe, q - qe);
  const long long total = (long long)q * q;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % q), dd = (int)(e / q);
    const int pd = dd >= qe, pr = r >= qe;
    if (pd != pr) continue;
    double acc = 0.0;
    for (int k = 0; k < D; ++k)
      for (int m = 0; m < D; ++m) {
        const long long ap = a_pos(0, traced_local(k, D, hermitian), 0, traced_local(m, D, hermitian),
                                   pd, dd - pd * qe, pr, r - pr * qe, s);
        acc += a[ap];
      }
    const long long n = s.n[pd];
    const long long off = pd ? (long long)qe * qe : 0;
    C[off + (dd - pd * qe) * n + (r - pr * qe)] = acc;
  }
}

// Merge the two ascending spectra; keep the chi of largest modulus.
__global__ void select_kernel(const double* __restrict__ w0g, int n0, const double* __restrict__ w1g,
                              int n1, int chi, int* __restrict__ idx, double* __restrict__ lam,
                              SelectOut* out, bool staged) {
  hs_pdl_enter();
  // both spectra staged in shared memory (the merge below is a serial walk),
  // followed by the picked values and their blocks. The walk compares
  // magnitudes as integers (IEEE bit patterns without the sign order like
  // |x| for finite values): FP64 compares would run on the slow FP64 pipe.
  extern __shared__ double wsh[];
  const int keep = min(chi, n0 + n1);
  const double* w0 = w0g;
  const double* w1 = w1g;
  double* pv = wsh + (staged ? n0 + n1 : 0);
  unsigned char* pb = reinterpret_cast<unsigned char*>(pv + keep);
  if (staged) {
    for (int i = threadIdx.x; i < n0; i += blockDim.x) wsh[i] = w0g[i];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) wsh[n0 + i] = w1g[i];
    w0 = wsh;
    w1 = wsh + n0;
  }
  // sum of |w| over both spectra
  __shared__ double part[256];
  __shared__ unsigned long long first_bits, last_bits;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n0 + n1; i += blockDim.x) acc += fabs(i < n0 ? w0g[i] : w1g[i - n0]);
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    constexpr unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long* u0 = reinterpret_cast<const unsigned long long*>(w0);
    const unsigned long long* u1 = reinterpret_cast<const unsigned long long*>(w1);
    int lo0 = 0, hi0 = n0 - 1, lo1 = 0, hi1 = n1 - 1, cnt0 = 0, cnt1 = 0;
    unsigned long long fb = 0, lb = 0;
    for (int s = 0; s <= keep; ++s) {
      // candidates in tie order: block 0 low end, block 0 high end, block 1 low, block 1 high
      int best_b = -1, best_i = -1;
      unsigned long long best = 0;
      bool any = false;
      if (lo0 <= hi0) {
        const unsigned long long a = u0[lo0] & kMag, c = u0[hi0] & kMag;
        best = a; best_b = 0; best_i = lo0; any = true;
        if (c > best) { best = c; best_i = hi0; }
      }
      if (lo1 <= hi1) {
        const unsigned long long a = u1[lo1] & kMag, c = u1[hi1] & kMag;
        if (!any || a > best) { best = a; best_b = 1; best_i = lo1; any = true; }
        if (c > best) { best = c; best_b = 1; best_i = hi1; }
      }
      if (s == keep) {
        out->lam_next = any ? __longlong_as_double((long long)best) : 0.0;
        break;
      }
      if (s == 0) fb = best;
      lb = best;
      if (best_b == 0) {
        idx[cnt0++] = best_i;
        pv[s] = w0[best_i];
        if (best_i == lo0) ++lo0; else --hi0;
      } else {
        idx[chi + cnt1++] = best_i;
        pv[s] = w1[best_i];
        if (best_i == lo1) ++lo1; else --hi1;
      }
      pb[s] = (unsigned char)best_b;
    }
    // new diagonal in FSO order: block 0's picks, then block 1's, each in pick order
    int j0 = 0, j1 = cnt0;
    for (int s = 0; s < keep; ++s) lam[pb[s] ? j1++ : j0++] = pv[s];
    out->chi_new[0] = cnt0;
    out->chi_new[1] = cnt1;
    first_bits = fb;
    last_bits = lb;
  }
  __syncthreads();
  // discarded weight: sum |w| minus the kept magnitudes (parallel)
  double k = 0.0;
  for (int s = threadIdx.x; s < keep; s += blockDim.x) k += fabs(pv[s]);
  __syncthreads();
  part[threadIdx.x] -= k;
  __syncthreads();
  if (threadIdx.x == 0) {
    double disc = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) disc += part[t];
    out->discarded = disc;
    out->lam_max = __longlong_as_double((long long)first_bits);
    out->lam_cut = __longlong_as_double((long long)last_bits);
  }
}

// select_kernel for small spectra (n0 + n1 <= kRankMax), by ranks instead of
// a serial merge: element e's rank is the number of elements that come before
// it in the merge order (larger |w| first; on equal |w| block 0 first, then
// the low end of a block before its high end, then the element nearer its end),
// so the kept states, their pick order and every output equal the merge's.
// One CTA of kRankMax threads.
constexpr int kRankMax = 1024;

__global__ void __launch_bounds__(kRankMax) select_rank_kernel(const double* __restrict__ w0g, int n0,
                                                               const double* __restrict__ w1g, int n1, int chi,
                                                               int* __restrict__ idx, double* __restrict__ lam,
                                                               SelectOut* out) {
  hs_pdl_enter();
  __shared__ unsigned long long mag[kRankMax];
  __shared__ unsigned tie[kRankMax];  // block << 31 | side << 30 | distance from the end
  __shared__ short inv[kRankMax];     // element of each rank
  __shared__ int pre[kRankMax];       // block-1 picks among ranks < r (inclusive scan, then shifted)
  __shared__ double part[kRankMax / 32];
  constexpr unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
  const int N = n0 + n1, keep = min(chi, N), t = threadIdx.x;
  double wv = 0.0;
  if (t < N) {
    const int b = t >= n0, i = b ? t - n0 : t, nb = b ? n1 : n0;
    wv = b ? w1g[i] : w0g[i];
    const unsigned long long u = (unsigned long long)__double_as_longlong(wv);
    const int side = (u >> 63) ? 0 : 1;  // negative values come off the low end
    mag[t] = u & kMag;
    tie[t] = ((unsigned)b << 31) | ((unsigned)side << 30) | (unsigned)(side ? nb - 1 - i : i);
  }
  __syncthreads();
  int rank = 0;
  if (t < N) {
    const unsigned long long me = mag[t];
    const unsigned mt = tie[t];
    for (int f = 0; f < N; ++f) {
      const unsigned long long o = mag[f];
      rank += (o > me) || (o == me && tie[f] < mt);
    }
    inv[rank] = (short)t;
  }
  // sum of |w| over both spectra minus the kept ones: the discarded weight
  double dw = (t < N && rank >= keep) ? fabs(wv) : 0.0;
  for (int o = 16; o > 0; o >>= 1) dw += __shfl_xor_sync(0xffffffffu, dw, o);
  if ((t & 31) == 0) part[t >> 5] = dw;
  __syncthreads();
  // block-1 flags in pick order, inclusive scan
  pre[t] = (t < keep && inv[t] >= n0) ? 1 : 0;
  __syncthreads();
  for (int o = 1; o < kRankMax; o <<= 1) {
    const int v = t >= o ? pre[t - o] : 0;
    __syncthreads();
    pre[t] += v;
    __syncthreads();
  }
  const int ones = keep > 0 ? pre[keep - 1] : 0, cnt0 = keep - ones;
  if (t < keep) {
    const int e = inv[t], b = e >= n0, i = b ? e - n0 : e;
    const int before1 = pre[t] - b;  // block-1 picks among ranks < t
    const double v = b ? w1g[i] : w0g[i];
    if (b) {
      idx[chi + before1] = i;
      lam[cnt0 + before1] = v;
    } else {
      const int p0 = t - before1;
      idx[p0] = i;
      lam[p0] = v;
    }
  }
  if (t == 0) {
    double disc = 0.0;
    for (int w = 0; w < kRankMax / 32; ++w) disc += part[w];
    out->discarded = disc;
    out->chi_new[0] = cnt0;
    out->chi_new[1] = ones;
    out->lam_max = keep > 0 ? __longlong_as_double((long long)mag[inv[0]]) : 0.0;
    out->lam_cut = keep > 0 ? __longlong_as_double((long long)mag[inv[keep - 1]]) : 0.0;
    out->lam_next = keep < N ? __longlong_as_double((long long)mag[inv[keep]]) : 0.0;
  }
}

__global__ void gather_pt_kernel(const double* __restrict__ V0, int n0, const double* __restrict__ V1,
                                 int n1, const int* __restrict__ idx, int chi,
                                 const SelectOut* __restrict__ sel, double* __restrict__ PT) {
  hs_pdl_enter();
  const int b = blockIdx.y, j = blockIdx.x;
  if (j >= sel->chi_new[b]) return;
  const int n = b ? n1 : n0;
  const double* src = (b ? V1 : V0) + (long long)idx[b * chi + j] * n;
  double* dst = PT + (b ? (long long)sel->chi_new[0] * n0 : 0) + (long long)j * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

__global__ void diag_corner_kernel(const double* __restrict__ lam, SelectOut* sel, double* C,
                                   int chi) {
  hs_pdl_enter();
  const int c0 = sel->chi_new[0], c1 = sel->chi_new[1];
  const long long total = (long long)c0 * c0 + (long long)c1 * c1;
  // one FP64 division per block (it is a long sequence on the FP64 pipe)
  __shared__ double s_inv;
  if (threadIdx.x == 0) s_inv = 1.0 / sel->lam_max;
  __syncthreads();
  const double inv = s_inv;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r, c, base;
    if (e < (long long)c0 * c0) {
      r = e / c0;
      c = e % c0;
      base = 0;
    } else {
      const long long f = e - (long long)c0 * c0;
      r = f / c1;
      c = f % c1;
      base = c0;
    }
    C[e] = (r == c) ? lam[base + r] * inv : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sel->log_norm_C = log(sel->lam_max);
}

__global__ void absmax_kernel(const double* __restrict__ x, long long n, unsigned long long* m) {
  hs_pdl_enter();
  double v = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    v = fmax(v, fabs(x[e]));
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(m, (unsigned long long)__double_as_longlong(v));
}

__global__ void scale_kernel(double* __restrict__ x, long long n, const unsigned long long* m,
                             SelectOut* sel) {
  hs_pdl_enter();
  const double mx = __longlong_as_double((long long)*m);
  // one FP64 division per block (it is a long sequence on the FP64 pipe)
  __shared__ double s_inv;
  if (threadIdx.x == 0) s_inv = 1.0 / mx;
  __syncthreads();
  const double inv = s_inv;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e] *= inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) sel->log_norm_T = log(mx);
}

__global__ void cast_f64_f32_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
  hs_pdl_enter();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    b[e] = (float)a[e];
}

__global__ void cast_f32_f64_kernel(const float* __restrict__ a, double* __restrict__ b, long long n) {
  hs_pdl_enter();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    b[e] = (double)a[e];
}

// Row j of block b of PT, and column j of block b of P (n_b x c_b row-major).
__global__ void gather_p32_kernel(const float* __restrict__ V0, int n0, const float* __restrict__ V1, int n1,
                                  const int* __restrict__ idx, int chi, const SelectOut* __restrict__ sel,
                                  double* __restrict__ PT, double* __restrict__ P) {
  hs_pdl_enter();
  const int b = blockIdx.y, j = blockIdx.x;
  const int cb = sel->chi_new[b];
  if (j >= cb) return;
  const int n = b ? n1 : n0;
  const float* src = (b ? V1 : V0) + (long long)idx[b * chi + j] * n;
  const long long off = b ? (long long)sel->chi_new[0] * n0 : 0;
  double* prow = PT + off + (long long)j * n;
  double* pcol = P + off + j;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = (double)src[i];
    prow[i] = v;
    pcol[(long long)i * cb] = v;
  }
}

__global__ void lowdin_kernel(double* __restrict__ G, int k0, int k1) {
  hs_pdl_enter();
  const long long total = (long long)k0 * k0 + (long long)k1 * k1;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r, c;
    if (e < (long long)k0 * k0) {
      r = e / k0;
      c = e % k0;
    } else {
      const long long f = e - (long long)k0 * k0;
      r = f / k1;
      c = f % k1;
    }
    G[e] = (r == c ? 1.5 : 0.0) - 0.5 * G[e];
  }
}

__global__ void scale_to_kernel(double* __restrict__ x, long long n, const unsigned long long* m, double* log_out) {
  hs_pdl_enter();
  const double mx = __longlong_as_double((long long)*m);
  __shared__ double s_inv;
  if (threadIdx.x == 0) s_inv = 1.0 / mx;
  __syncthreads();
  const double inv = s_inv;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e] *= inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) *log_out = log(mx);
}

__device__ __forceinline__ int pair_index(int k, int l, int D) {
  return k * (2 * D - k - 1) / 2 + (l - k - 1);
}

__global__ void env_to_dense_kernel(const double* __restrict__ C, const double* __restrict__ T, int D,
                                    int c0, int c1, bool hermitian, double* __restrict__ Cd,
                                    double* __restrict__ Td) {
  hs_pdl_enter();
  const int q = D * D, chi = c0 + c1;
  const int qe = hermitian ? D * (D + 1) / 2 : q;
  const Sect cs = make_sect(c0, c1), qs = make_sect(qe, q - qe);
  const long long nT = (long long)chi * q * chi, nC = (long long)chi * chi;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nT + nC;
       e += (long long)gridDim.x * blockDim.x) {
    if (e >= nT) {
      const long long f = e - nT;
      const int a = (int)(f / chi), b = (int)(f % chi);
      const int pa = a >= c0, pb = b >= c0;
      double v = 0.0;
      if (pa == pb) {
        const int n = pa ? c1 : c0;
        v = C[(pa ? (long long)c0 * c0 : 0) + (long long)(a - pa * c0) * n + (b - pb * c0)];
      }
      Cd[f] = v;
      continue;
    }
    const int b = (int)(e % chi), x = (int)((e / chi) % q), a = (int)(e / chi / q);
    const int pa = a >= c0, pb = b >= c0;
    int nX = 1, X[2];
    double w[2];
    if (!hermitian) {
      X[0] = x;
      w[0] = 1.0;
    } else {
      const int i = x % D, ib = x / D;
      if (i == ib) {
        X[0] = i;
        w[0] = 1.0;
      } else {
        const int k = min(i, ib), l = max(i, ib);
        const int m = pair_index(k, l, D);
        const double r = 0.70710678118654752440;
        nX = 2;
        X[0] = D + m;
        w[0] = r;
        X[1] = qe + m;
        w[1] = (i < ib) ? r : -r;  // (ket k, bra l) enters the odd state with +, (ket l, bra k) with -
      }
    }
    double v = 0.0;
    for (int t = 0; t < nX; ++t) {
      const int px = X[t] >= qe;
      const long long pos = t_pos(pa, a - pa * c0, px, X[t] - px * qe, pb, b - pb * c0, cs, qs);
      if (pos >= 0) v += w[t] * T[pos];
    }
    Td[e] = v;
  }
}

// Graded environment (complex path) -> interleaved complex dense views in the
// plain combined basis: C[a, b] and T[a, x, b] with x = i + D * ibar; an entry
// of odd total parity is i times the stored number.
__global__ void env_to_dense_graded_kernel(const double* __restrict__ C, const double* __restrict__ T, int D,
                                           int c0, int c1, double* __restrict__ Cd, double* __restrict__ Td) {
  hs_pdl_enter();
  const int q = D * D, chi = c0 + c1;
  const int qe = D * (D + 1) / 2, qo = q - qe;
  const Fused fr = fused2(make_sect(c0, c1), make_sect(qe, qo));
  const long long f0 = fused_size(fr, 0);
  const long long nT = (long long)chi * q * chi, nC = (long long)chi * chi;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nT + nC;
       e += (long long)gridDim.x * blockDim.x) {
    if (e >= nT) {
      const long long f = e - nT;
      const int a = (int)(f / chi), b = (int)(f % chi);
      const double v = C[f];
      const bool odd = (a >= c0) != (b >= c0);
      Cd[2 * f] = odd ? 0.0 : v;
      Cd[2 * f + 1] = odd ? v : 0.0;
      continue;
    }
    const int b = (int)(e % chi), x = (int)((e / chi) % q), a = (int)(e / chi / q);
    const int pa = a >= c0, pb = b >= c0;
    int nX = 1, X[2];
    double w[2];
    const int i = x % D, ib = x / D;
    if (i == ib) {
      X[0] = i;
      w[0] = 1.0;
    } else {
      const int k = min(i, ib), l = max(i, ib);
      const int m = pair_index(k, l, D);
      const double r = 0.70710678118654752440;
      nX = 2;
      X[0] = D + m;
      w[0] = r;
      X[1] = qe + m;
      w[1] = (i < ib) ? r : -r;
    }
    double re = 0.0, im = 0.0;
    for (int t = 0; t < nX; ++t) {
      const int px = X[t] >= qe;
      const int tt = (pa << 1) | px;
      const long long row = ((pa ^ px) ? f0 : 0) + tuple_offset(fr, tt) +
                            (long long)(a - pa * c0) * (px ? qo : qe) + (X[t] - px * qe);
      const double v = w[t] * T[row * chi + b];
      if ((pa + px + pb) & 1)
        im += v;
      else
        re += v;
    }
    Td[2 * e] = re;
    Td[2 * e + 1] = im;
  }
}

}  // namespace

cudaError_t launch_env_to_dense_graded(const double* C, const double* T, int D, int c0, int c1, double* Cd,
                                       double* Td, cudaStream_t s) {
  const long long chi = c0 + c1, q = (long long)D * D;
  hs_launch(env_to_dense_graded_kernel, grid_for(chi * q * chi + chi * chi), 256, 0, s, C, T, D, c0, c1, Cd, Td);
  return cudaGetLastError();
}

cudaError_t launch_ctmrg_init(const double* a_blocks, int D, bool hermitian, double* C, double* T,
                              cudaStream_t s) {
  const long long q = (long long)D * D;
  hs_launch(init_T_kernel, grid_for(q * q * q), 256, 0, s, a_blocks, D, hermitian, T);
  hs_launch(init_C_kernel, grid_for(q * q), 256, 0, s, a_blocks, D, hermitian, C);
  return cudaGetLastError();
}

cudaError_t launch_select(const double* w0, int n0, const double* w1, int n1, int chi, int* idx,
                          double* lam, SelectOut* out, cudaStream_t s) {
  if (n0 + n1 <= kRankMax) {
    hs_launch(select_rank_kernel, 1, kRankMax, 0, s, w0, n0, w1, n1, chi, idx, lam, out);
    return cudaGetLastError();
  }
  constexpr size_t kSmemMax = 160 * 1024;
  const int keep = chi < n0 + n1 ? chi : n0 + n1;
  const size_t picks = (size_t)keep * (sizeof(double) + 1);
  size_t smem = (size_t)(n0 + n1) * sizeof(double) + picks;
  const bool staged = smem <= kSmemMax;
  if (!staged) smem = picks;
  if (smem > kSmemMax) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    // opt in beyond the default 48 KB only when needed (once per device)
    const cudaError_t attr_err = ensure_smem_attr(reinterpret_cast<const void*>(select_kernel), (int)kSmemMax);
    if (attr_err != cudaSuccess) return attr_err;
  }
  hs_launch(select_kernel, 1, 256, smem, s, w0, n0, w1, n1, chi, idx, lam, out, staged);
  return cudaGetLastError();
}

cudaError_t launch_gather_pt(const double* V0, int n0, const double* V1, int n1, const int* idx,
                                 int chi, const SelectOut* sel, double* PT, cudaStream_t s) {
  dim3 grid((unsigned)chi, 2);
  hs_launch(gather_pt_kernel, grid, 256, 0, s, V0, n0, V1, n1, idx, chi, sel, PT);
  return cudaGetLastError();
}

cudaError_t launch_diag_corner(const double* lam, int c0, int c1, SelectOut* sel, double* C,
                               cudaStream_t s) {
  const long long n = (long long)c0 * c0 + (long long)c1 * c1;
  hs_launch(diag_corner_kernel, grid_for(n), 256, 0, s, lam, sel, C, c0 + c1);
  return cudaGetLastError();
}

cudaError_t launch_normalize_max(double* T, long long n, unsigned long long* scratch,
                                 SelectOut* sel, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  hs_launch(absmax_kernel, grid_for(n), 256, 0, s, T, n, scratch);
  hs_launch(scale_kernel, grid_for(n), 256, 0, s, T, n, scratch, sel);
  return cudaGetLastError();
}

cudaError_t launch_cast_f64_f32(const double* src, float* dst, long long n, cudaStream_t s) {
  hs_launch(cast_f64_f32_kernel, grid_for(n), 256, 0, s, src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_cast_f32_f64(const float* src, double* dst, long long n, cudaStream_t s) {
  hs_launch(cast_f32_f64_kernel, grid_for(n), 256, 0, s, src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_gather_p32(const float* V0, int n0, const float* V1, int n1, const int* idx, int chi,
                              const SelectOut* sel, double* PT, double* P, cudaStream_t s) {
  dim3 grid((unsigned)chi, 2);
  hs_launch(gather_p32_kernel, grid, 256, 0, s, V0, n0, V1, n1, idx, chi, sel, PT, P);
  return cudaGetLastError();
}

cudaError_t launch_lowdin(double* G, int k0, int k1, cudaStream_t s) {
  const long long n = (long long)k0 * k0 + (long long)k1 * k1;
  hs_launch(lowdin_kernel, grid_for(n), 256, 0, s, G, k0, k1);
  return cudaGetLastError();
}

cudaError_t launch_normalize_max_to(double* x, long long n, unsigned long long* scratch, double* log_out,
                                    cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  hs_launch(absmax_kernel, grid_for(n), 256, 0, s, x, n, scratch);
  hs_launch(scale_to_kernel, grid_for(n), 256, 0, s, x, n, scratch, log_out);
  return cudaGetLastError();
}

__global__ void block_trace_kernel(const double* __restrict__ x, int n0, int n1, double* out) {
  hs_pdl_enter();
  double v = 0.0;
  for (int i = threadIdx.x; i < n0 + n1; i += blockDim.x)
    v += i < n0 ? x[(long long)i * n0 + i] : x[(long long)n0 * n0 + (long long)(i - n0) * n1 + (i - n0)];
  __shared__ double red[256];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

cudaError_t launch_block_trace(const double* x, int n0, int n1, double* out, cudaStream_t s) {
  hs_launch(block_trace_kernel, 1, 256, 0, s, x, n0, n1, out);
  return cudaGetLastError();
}

// ---- adjoints for the gradient through the CTMRG iterations (hs_grad.cu) ----

namespace {

// Adjoint of init_T_kernel: da[a_pos(u, traced k, d, r)] += dT[t_pos(d, r, u)].
// One thread per (d, r, u): the positions it adds to are its own.
__global__ void init_T_vjp_kernel(const double* __restrict__ dT, int D, bool hermitian, double* __restrict__ da) {
  hs_pdl_enter();
  const int q = D * D;
  const int qe = hermitian ? D * (D + 1) / 2 : q;
  const Sect s = make_sect(qe, q - qe);
  const long long total = (long long)q * q * q;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int u = (int)(e % q), r = (int)((e / q) % q), dd = (int)(e / q / q);
    const int pd = dd >= qe, pr = r >= qe, pu = u >= qe;
    const long long pos = t_pos(pd, dd - pd * qe, pr, r - pr * qe, pu, u - pu * qe, s, s);
    if (pos < 0) continue;
    const double g = dT[pos];
    for (int k = 0; k < D; ++k)
      da[a_pos(pu, u - pu * qe, 0, traced_local(k, D, hermitian), pd, dd - pd * qe, pr, r - pr * qe, s)] += g;
  }
}

// Adjoint of init_C_kernel: da[a_pos(traced k, traced m, d, r)] += dC[d, r].
__global__ void init_C_vjp_kernel(const double* __restrict__ dC, int D, bool hermitian, double* __restrict__ da) {
  hs_pdl_enter();
  const int q = D * D;
  const int qe = hermitian ? D * (D + 1) / 2 : q;
  const Sect s = make_sect(qe, q - qe);
  const long long total = (long long)q * q;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % q), dd = (int)(e / q);
    const int pd = dd >= qe, pr = r >= qe;
    if (pd != pr) continue;
    const long long n = s.n[pd];
    const long long off = pd ? (long long)qe * qe : 0;
    const double g = dC[off + (dd - pd * qe) * n + (r - pr * qe)];
    for (int k = 0; k < D; ++k)
      for (int m = 0; m < D; ++m)
        da[a_pos(0, traced_local(k, D, hermitian), 0, traced_local(m, D, hermitian), pd, dd - pd * qe, pr,
                 r - pr * qe, s)] += g;
  }
}

// Adjoint of env_to_dense_kernel: every stored entry of C and T collects the
// dense entries it was copied (C) or rotated (T, the double-layer leg x back
// to the plain basis) into: dT[(a, X, b)] = sum_x U[x, X] dTd[a, x, b].
__global__ void env_to_dense_vjp_kernel(const double* __restrict__ dCd, const double* __restrict__ dTd, int D, int c0,
                                        int c1, bool hermitian, double* __restrict__ dC, double* __restrict__ dT) {
  hs_pdl_enter();
  const int q = D * D, chi = c0 + c1;
  const int qe = hermitian ? D * (D + 1) / 2 : q;
  const Sect cs = make_sect(c0, c1), qs = make_sect(qe, q - qe);
  const long long nT = (long long)chi * q * chi, nC = (long long)chi * chi;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nT + nC;
       e += (long long)gridDim.x * blockDim.x) {
    if (e >= nT) {
      const long long f = e - nT;
      const int a = (int)(f / chi), b = (int)(f % chi);
      const int pa = a >= c0, pb = b >= c0;
      if (pa != pb) continue;
      const int n = pa ? c1 : c0;
      dC[(pa ? (long long)c0 * c0 : 0) + (long long)(a - pa * c0) * n + (b - pb * c0)] += dCd[f];
      continue;
    }
    // e enumerates (a, X, b) with X a basis state of the double-layer leg
    const int b = (int)(e % chi), X = (int)((e / chi) % q), a = (int)(e / chi / q);
    const int pa = a >= c0, pb = b >= c0, px = X >= qe;
    const long long pos = t_pos(pa, a - pa * c0, px, X - px * qe, pb, b - pb * c0, cs, qs);
    if (pos < 0) continue;
    double v;
    if (!hermitian) {
      v = dTd[((long long)a * q + X) * chi + b];
    } else if (X < D) {
      v = dTd[((long long)a * q + X * (D + 1)) * chi + b];  // (k k'): x = k + D k
    } else {
      // pair state (k, l), k < l: plain (ket k, bra l) and (ket l, bra k)
      int m = px ? X - qe : X - D, k = 0;
      while (m >= D - 1 - k) {
        m -= D - 1 - k;
        ++k;
      }
      const int l = k + 1 + m;
      const double r = 0.70710678118654752440;
      const double s2 = px ? -r : r;
      v = r * dTd[((long long)a * q + (k + D * l)) * chi + b] + s2 * dTd[((long long)a * q + (l + D * k)) * chi + b];
    }
    dT[pos] += v;
  }
}

}  // namespace

cudaError_t launch_ctmrg_init_vjp(const double* dC, const double* dT, int D, bool hermitian, double* da,
                                  cudaStream_t s) {
  const long long q = (long long)D * D;
  hs_launch(init_T_vjp_kernel, grid_for(q * q * q), 256, 0, s, dT, D, hermitian, da);
  hs_launch(init_C_vjp_kernel, grid_for(q * q), 256, 0, s, dC, D, hermitian, da);
  return cudaGetLastError();
}

cudaError_t launch_env_to_dense_vjp(const double* dCd, const double* dTd, int D, int c0, int c1, bool hermitian,
                                    double* dC, double* dT, cudaStream_t s) {
  const long long chi = c0 + c1, q = (long long)D * D;
  hs_launch(env_to_dense_vjp_kernel, grid_for(chi * q * chi + chi * chi), 256, 0, s, dCd, dTd, D, c0, c1, hermitian,
            dC, dT);
  return cudaGetLastError();
}

cudaError_t launch_env_to_dense(const double* C, const double* T, int D, int c0, int c1,
                                bool hermitian, double* Cd, double* Td, cudaStream_t s) {
  const long long chi = c0 + c1, q = (long long)D * D;
  hs_launch(env_to_dense_kernel, grid_for(chi * q * chi + chi * chi), 256, 0, s, C, T, D, c0, c1, hermitian,
                                                                         Cd, Td);
  return cudaGetLastError();
}

}  // namespace hs

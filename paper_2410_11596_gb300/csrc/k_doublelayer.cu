// Double-layer tensor a = sum_s A_s (x) conj(A_s) (arXiv 2410.11596 Sec. II.A,
// Fig. 1(b)) and its form in the eigenbasis of the bra-ket swap S (Sec. II.B).
//
// A basis state X of one combined leg is a combination of at most two plain
// states (ket i, bra ibar), x = i + D*ibar:
//   X <  D           : (k k')                   coefficient 1
//   D <= X < q_even  : (k l' + l k')/sqrt2, k<l  lexicographic pair X - D
//   X >= q_even      : (k l' - l k')/sqrt2, k<l  pair X - q_even
#include <cmath>

#include "hs_internal.cuh"

namespace hs {

namespace {

struct Terms {
  int n;
  int ket[2], bra[2];
  double c[2];
};

// Pair number m -> (k, l), k < l, lexicographic.
__device__ __forceinline__ void pair_of(int m, int D, int* k, int* l) {
  int kk = 0;
  while (m >= D - 1 - kk) {
    m -= D - 1 - kk;
    ++kk;
  }
  *k = kk;
  *l = kk + 1 + m;
}

__device__ __forceinline__ Terms basis_terms(int X, int D, bool hermitian) {
  Terms t;
  if (!hermitian) {
    t.n = 1;
    t.ket[0] = X % D;
    t.bra[0] = X / D;
    t.c[0] = 1.0;
    return t;
  }
  const int qe = D * (D + 1) / 2;
  if (X < D) {
    t.n = 1;
    t.ket[0] = X;
    t.bra[0] = X;
    t.c[0] = 1.0;
    return t;
  }
  int k, l;
  const bool odd = X >= qe;
  pair_of(odd ? X - qe : X - D, D, &k, &l);
  const double r = 0.70710678118654752440;
  t.n = 2;
  t.ket[0] = k;
  t.bra[0] = l;
  t.c[0] = r;
  t.ket[1] = l;
  t.bra[1] = k;
  t.c[1] = odd ? -r : r;
  return t;
}

// FSO position of element (X_u, X_l, X_d, X_r) of a [(u,l)|(d,r)] matrix whose
// legs all have sectors (qe, qo); returns -1 for odd-total elements.
__device__ __forceinline__ long long fso4(int Xu, int Xl, int Xd, int Xr, int qe, int qo) {
  const Sect s = make_sect(qe, qo);
  const Fused f = fused2(s, s);
  const int pu = Xu >= qe, pl = Xl >= qe, pd = Xd >= qe, pr = Xr >= qe;
  if ((pu + pl + pd + pr) & 1) return -1;
  const int iu = Xu - pu * qe, il = Xl - pl * qe, id = Xd - pd * qe, ir = Xr - pr * qe;
  const int tr = (pu << 1) | pl, tc = (pd << 1) | pr;
  const int P = tuple_parity(tr);
  const long long CP = fused_size(f, P);
  const long long row = tuple_offset(f, tr) + (long long)iu * s.n[pl] + il;
  const long long col = tuple_offset(f, tc) + (long long)id * s.n[pr] + ir;
  const long long off = P ? fused_size(f, 0) * fused_size(f, 0) : 0;
  return off + row * CP + col;
}

__global__ void double_layer_blocks_kernel(const double* __restrict__ A, int d, int D,
                                           bool hermitian, double* __restrict__ out) {
  hs_pdl_enter();
  const int q = D * D;
  const int qe = hermitian ? D * (D + 1) / 2 : q;
  const int qo = q - qe;
  const long long total = (long long)q * q * q * q;
  const long long D4 = (long long)D * D * D * D;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int Xr = (int)(e % q), Xd = (int)((e / q) % q), Xl = (int)((e / q / q) % q),
              Xu = (int)(e / q / q / q);
    const long long pos = fso4(Xu, Xl, Xd, Xr, qe, qo);
    if (pos < 0) continue;
    const Terms tu = basis_terms(Xu, D, hermitian), tl = basis_terms(Xl, D, hermitian),
                td = basis_terms(Xd, D, hermitian), tr = basis_terms(Xr, D, hermitian);
    double acc = 0.0;
    for (int a = 0; a < tu.n; ++a)
      for (int b = 0; b < tl.n; ++b)
        for (int c = 0; c < td.n; ++c)
          for (int g = 0; g < tr.n; ++g) {
            const double coef = tu.c[a] * tl.c[b] * td.c[c] * tr.c[g];
            const long long ik = (((long long)tu.ket[a] * D + tl.ket[b]) * D + td.ket[c]) * D + tr.ket[g];
            const long long ib = (((long long)tu.bra[a] * D + tl.bra[b]) * D + td.bra[c]) * D + tr.bra[g];
            double s = 0.0;
            for (int p = 0; p < d; ++p) s += A[p * D4 + ik] * A[p * D4 + ib];
            acc += coef * s;
          }
    out[pos] = acc;
  }
}

// Complex A (interleaved complex128): a~ in the eigenbasis of S as a graded
// [(u,l)|(d,r)] matrix (Sec. II.C): the real part of every even-total entry,
// the imaginary part of every odd-total one (the other part vanishes).
__global__ void double_layer_graded_kernel(const double* __restrict__ A, int d, int D, double* __restrict__ out) {
  hs_pdl_enter();
  const int q = D * D;
  const int qe = D * (D + 1) / 2, qo = q - qe;
  const Fused f = fused2(make_sect(qe, qo), make_sect(qe, qo));
  const long long f0 = fused_size(f, 0);
  const long long total = (long long)q * q * q * q;
  const long long D4 = (long long)D * D * D * D;
  const long long q2 = (long long)q * q;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int Xr = (int)(e % q), Xd = (int)((e / q) % q), Xl = (int)((e / q / q) % q),
              Xu = (int)(e / q / q / q);
    const int pu = Xu >= qe, pl = Xl >= qe, pd = Xd >= qe, pr = Xr >= qe;
    const long long row = ((pu ^ pl) ? f0 : 0) + tuple_offset(f, (pu << 1) | pl) +
                          (long long)(Xu - pu * qe) * (pl ? qo : qe) + (Xl - pl * qe);
    const long long col = ((pd ^ pr) ? f0 : 0) + tuple_offset(f, (pd << 1) | pr) +
                          (long long)(Xd - pd * qe) * (pr ? qo : qe) + (Xr - pr * qe);
    const Terms tu = basis_terms(Xu, D, true), tl = basis_terms(Xl, D, true), td = basis_terms(Xd, D, true),
                tr = basis_terms(Xr, D, true);
    double re = 0.0, im = 0.0;
    for (int a = 0; a < tu.n; ++a)
      for (int b = 0; b < tl.n; ++b)
        for (int c = 0; c < td.n; ++c)
          for (int g = 0; g < tr.n; ++g) {
            const double coef = tu.c[a] * tl.c[b] * td.c[c] * tr.c[g];
            const long long ik = (((long long)tu.ket[a] * D + tl.ket[b]) * D + td.ket[c]) * D + tr.ket[g];
            const long long ib = (((long long)tu.bra[a] * D + tl.bra[b]) * D + td.bra[c]) * D + tr.bra[g];
            double sr = 0.0, si = 0.0;
            for (int p = 0; p < d; ++p) {
              const double kr = A[2 * (p * D4 + ik)], ki = A[2 * (p * D4 + ik) + 1];
              const double br = A[2 * (p * D4 + ib)], bi = A[2 * (p * D4 + ib) + 1];
              sr += kr * br + ki * bi;  // ket * conj(bra)
              si += ki * br - kr * bi;
            }
            re += coef * sr;
            im += coef * si;
          }
    out[row * q2 + col] = ((pu + pl + pd + pr) & 1) ? im : re;
  }
}

__global__ void double_layer_dense_kernel(const double* __restrict__ A, int d, int D, bool cplx,
                                          double* __restrict__ out) {
  hs_pdl_enter();
  const int q = D * D;
  const long long total = (long long)q * q * q * q;
  const long long D4 = (long long)D * D * D * D;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int xr = (int)(e % q), xd = (int)((e / q) % q), xl = (int)((e / q / q) % q),
              xu = (int)(e / q / q / q);
    const long long ik = (((long long)(xu % D) * D + xl % D) * D + xd % D) * D + xr % D;
    const long long ib = (((long long)(xu / D) * D + xl / D) * D + xd / D) * D + xr / D;
    if (!cplx) {
      double s = 0.0;
      for (int p = 0; p < d; ++p) s += A[p * D4 + ik] * A[p * D4 + ib];
      out[e] = s;
    } else {
      double re = 0.0, im = 0.0;
      for (int p = 0; p < d; ++p) {
        const double ar = A[2 * (p * D4 + ik)], ai = A[2 * (p * D4 + ik) + 1];
        const double br = A[2 * (p * D4 + ib)], bi = -A[2 * (p * D4 + ib) + 1];
        re += ar * br - ai * bi;
        im += ar * bi + ai * br;
      }
      out[2 * e] = re;
      out[2 * e + 1] = im;
    }
  }
}

__global__ void rotate_dense_kernel(const double* __restrict__ a, int D, double* __restrict__ out,
                                    unsigned long long* maxes) {
  hs_pdl_enter();
  const int q = D * D;
  const int qe = D * (D + 1) / 2, qo = q - qe;
  const long long total = (long long)q * q * q * q;
  double mall = 0.0, modd = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int Xr = (int)(e % q), Xd = (int)((e / q) % q), Xl = (int)((e / q / q) % q),
              Xu = (int)(e / q / q / q);
    const Terms tu = basis_terms(Xu, D, true), tl = basis_terms(Xl, D, true),
                td = basis_terms(Xd, D, true), tr = basis_terms(Xr, D, true);
    double acc = 0.0;
    for (int i = 0; i < tu.n; ++i)
      for (int j = 0; j < tl.n; ++j)
        for (int k = 0; k < td.n; ++k)
          for (int m = 0; m < tr.n; ++m) {
            const long long x = (((long long)(tu.ket[i] + D * tu.bra[i]) * q + (tl.ket[j] + D * tl.bra[j])) * q +
                                 (td.ket[k] + D * td.bra[k])) * q + (tr.ket[m] + D * tr.bra[m]);
            acc += tu.c[i] * tl.c[j] * td.c[k] * tr.c[m] * a[x];
          }
    const long long pos = fso4(Xu, Xl, Xd, Xr, qe, qo);
    mall = fmax(mall, fabs(acc));
    if (pos < 0)
      modd = fmax(modd, fabs(acc));
    else
      out[pos] = acc;
  }
  atomicMax(&maxes[0], (unsigned long long)__double_as_longlong(modd));
  atomicMax(&maxes[1], (unsigned long long)__double_as_longlong(mall));
}

// Index of the Hermitian basis state pair (k, l), k < l, lexicographic (the
// inverse of pair_of).
__device__ __forceinline__ int pair_index(int k, int l, int D) { return k * (D - 1) - k * (k - 1) / 2 + (l - k - 1); }

// The (at most two) basis states X of one leg that contain the plain state
// x = i + D*ibar, with the coefficient U[x, X] of x in X (Sec. II.B).
__device__ __forceinline__ Terms plain_terms(int x, int D) {
  Terms t;
  const int i = x % D, ib = x / D;
  if (i == ib) {
    t.n = 1;
    t.ket[0] = i;  // ket[] holds the basis state X here
    t.c[0] = 1.0;
    return t;
  }
  const int qe = D * (D + 1) / 2;
  const int k = i < ib ? i : ib, l = i < ib ? ib : i;
  const int m = pair_index(k, l, D);
  const double r = 0.70710678118654752440;
  t.n = 2;
  t.ket[0] = D + m;  // (k l' + l k')/sqrt2
  t.c[0] = r;
  t.ket[1] = qe + m;  // (k l' - l k')/sqrt2: + for (ket k, bra l), - for (ket l, bra k)
  t.c[1] = i < ib ? r : -r;
  return t;
}

// a[x_u, x_l, x_d, x_r] = sum_X U[x_u, X_u] .. U[x_r, X_r] a~[X_u, .., X_r]: the
// stored blocks of a~ (real FSO, or a graded complex matrix) back to the
// plain combined basis; complex output interleaved.
__global__ void from_hermitian_kernel(const double* __restrict__ t, int D, bool graded, double* __restrict__ out) {
  hs_pdl_enter();
  const int q = D * D;
  const int qe = D * (D + 1) / 2, qo = q - qe;
  const Fused f = fused2(make_sect(qe, qo), make_sect(qe, qo));
  const long long f0 = fused_size(f, 0);
  const long long q2 = (long long)q * q;
  const long long total = q2 * q2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int xr = (int)(e % q), xd = (int)((e / q) % q), xl = (int)((e / q / q) % q), xu = (int)(e / q / q / q);
    const Terms tu = plain_terms(xu, D), tl = plain_terms(xl, D), td = plain_terms(xd, D), tr = plain_terms(xr, D);
    double re = 0.0, im = 0.0;
    for (int a = 0; a < tu.n; ++a)
      for (int b = 0; b < tl.n; ++b)
        for (int c = 0; c < td.n; ++c)
          for (int g = 0; g < tr.n; ++g) {
            const int Xu = tu.ket[a], Xl = tl.ket[b], Xd = td.ket[c], Xr = tr.ket[g];
            const double coef = tu.c[a] * tl.c[b] * td.c[c] * tr.c[g];
            if (!graded) {
              const long long pos = fso4(Xu, Xl, Xd, Xr, qe, qo);
              if (pos >= 0) re += coef * t[pos];
              continue;
            }
            const int pu = Xu >= qe, pl = Xl >= qe, pd = Xd >= qe, pr = Xr >= qe;
            const long long row = ((pu ^ pl) ? f0 : 0) + tuple_offset(f, (pu << 1) | pl) +
                                  (long long)(Xu - pu * qe) * (pl ? qo : qe) + (Xl - pl * qe);
            const long long col = ((pd ^ pr) ? f0 : 0) + tuple_offset(f, (pd << 1) | pr) +
                                  (long long)(Xd - pd * qe) * (pr ? qo : qe) + (Xr - pr * qe);
            const double v = t[row * q2 + col];
            if ((pu + pl + pd + pr) & 1)
              im += coef * v;
            else
              re += coef * v;
          }
    if (graded) {
      out[2 * e] = re;
      out[2 * e + 1] = im;
    } else {
      out[e] = re;
    }
  }
}

unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

cudaError_t launch_double_layer_blocks(const double* A, int d, int D, bool hermitian, double* out,
                                       cudaStream_t s) {
  const long long q = (long long)D * D;
  hs_launch(double_layer_blocks_kernel, grid_for(q * q * q * q), 256, 0, s, A, d, D, hermitian, out);
  return cudaGetLastError();
}

cudaError_t launch_double_layer_graded(const double* A, int d, int D, double* out, cudaStream_t s) {
  const long long q = (long long)D * D, total = q * q * q * q;
  long long g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  hs_launch(double_layer_graded_kernel, (unsigned)g, 256, 0, s, A, d, D, out);
  return cudaGetLastError();
}

cudaError_t launch_double_layer_dense(const double* A, int d, int D, bool cplx, double* out,
                                      cudaStream_t s) {
  const long long q = (long long)D * D;
  hs_launch(double_layer_dense_kernel, grid_for(q * q * q * q), 256, 0, s, A, d, D, cplx, out);
  return cudaGetLastError();
}

namespace {
// Adjoint of the plain double layer a[x] = sum_p A[p, ket(x)] A[p, bra(x)]
// (real A): dA[p, i] += sum_j (da[x(ket i, bra j)] + da[x(ket j, bra i)]) A[p, j],
// i, j multi-indices (u, l, d, r) and x the combined index of each leg.
__global__ void double_layer_vjp_kernel(const double* __restrict__ da, const double* __restrict__ A, int d, int D,
                                        double* __restrict__ dA) {
  hs_pdl_enter();
  const long long D4 = (long long)D * D * D * D;
  const int q = D * D;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)d * D4;
       e += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(e / D4);
    const long long i = e % D4;
    const int iu = (int)(i / D / D / D), il = (int)((i / D / D) % D), id = (int)((i / D) % D), ir = (int)(i % D);
    double acc = 0.0;
    for (long long j = 0; j < D4; ++j) {
      const int ju = (int)(j / D / D / D), jl = (int)((j / D / D) % D), jd = (int)((j / D) % D), jr = (int)(j % D);
      const long long xk = (((long long)(iu + D * ju) * q + (il + D * jl)) * q + (id + D * jd)) * q + (ir + D * jr);
      const long long xb = (((long long)(ju + D * iu) * q + (jl + D * il)) * q + (jd + D * id)) * q + (jr + D * ir);
      acc += (da[xk] + da[xb]) * A[p * D4 + j];
    }
    dA[e] += acc;
  }
}
}  // namespace

cudaError_t launch_double_layer_vjp(const double* da_plain, const double* A, int d, int D, double* dA,
                                    cudaStream_t s) {
  const long long D4 = (long long)D * D * D * D;
  hs_launch(double_layer_vjp_kernel, grid_for(d * D4), 256, 0, s, da_plain, A, d, D, dA);
  return cudaGetLastError();
}

cudaError_t launch_from_hermitian(const double* t, int D, bool graded, double* out, cudaStream_t s) {
  const long long q = (long long)D * D;
  hs_launch(from_hermitian_kernel, grid_for(q * q * q * q), 256, 0, s, t, D, graded, out);
  return cudaGetLastError();
}

cudaError_t launch_rotate_dense_to_blocks(const double* a, int D, double* out,
                                          unsigned long long* maxes, cudaStream_t s) {
  const long long q = (long long)D * D;
  hs_launch(rotate_dense_kernel, grid_for(q * q * q * q), 256, 0, s, a, D, out, maxes);
  return cudaGetLastError();
}

}  // namespace hs

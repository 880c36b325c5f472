// Kernels of the complex (graded) CTMRG path, arXiv 2410.11596 Sec. II.C:
// in the eigenbasis of S every block of a complex double layer is purely real
// (even total parity) or purely imaginary (odd), so each tensor is stored as
// real numbers with the parity deciding the factor 1 or i (layout GMat in
// hs_internal.cuh).
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

__global__ void graded_sign_kernel(const double* __restrict__ src, double* __restrict__ dst, long long r0,
                                   long long r1, long long c0, long long c1, long long ld, int mode) {
  hs_pdl_enter();
  const long long cols = c0 + c1, total = (r0 + r1) * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / cols, c = e % cols;
    const int pr = r >= r0, pc = c >= c0;
    const bool neg = mode == 0 ? (pr != pc) : (pr && pc);
    const double v = src[r * ld + c];
    dst[r * ld + c] = neg ? -v : v;
  }
}

// Full FSO index of (Xa, Xb) in a fused pair of double-layer legs (qe, qo).
__device__ __forceinline__ long long pair_fso(int Xa, int Xb, int qe, int qo) {
  const Fused f = fused2(make_sect(qe, qo), make_sect(qe, qo));
  const int pa = Xa >= qe, pb = Xb >= qe;
  const int t = (pa << 1) | pb;
  const long long base = (pa ^ pb) ? fused_size(f, 0) : 0;
  return base + tuple_offset(f, t) + (long long)(Xa - pa * qe) * (pb ? qo : qe) + (Xb - pb * qe);
}

// C0[d | r] = sum_{k, m < D} a~[(k, m) | (d, r)]; T0[(alpha, x) | beta] =
// sum_{k < D} a~[(beta, k) | (alpha, x)]: the traced states (k k') are the
// first D even states of a leg.
__global__ void init_graded_kernel(const double* __restrict__ a, int D, double* __restrict__ C,
                                   double* __restrict__ T) {
  hs_pdl_enter();
  const int q = D * D, qe = D * (D + 1) / 2, qo = q - qe;
  const long long q2 = (long long)q * q, nT = (long long)q * q * q;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nT + q2;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nT) {
      // T0 position e = row (alpha, x) * q + beta with rows in FSO order
      const long long row = e / q;
      const int beta = (int)(e % q);
      // invert the FSO row index of (alpha, x)
      const Fused f = fused2(make_sect(qe, qo), make_sect(qe, qo));
      long long rr = row;
      int P = 0;
      if (rr >= fused_size(f, 0)) {
        rr -= fused_size(f, 0);
        P = 1;
      }
      int alpha = 0, x = 0;
      for (int t = 0; t < 4; ++t) {
        if (tuple_parity(t) != P) continue;
        const long long sz = tuple_size(f, t);
        if (rr < sz) {
          const int pa = (t >> 1) & 1, px = t & 1;
          const int nx = px ? qo : qe;
          alpha = (int)(rr / nx) + pa * qe;
          x = (int)(rr % nx) + px * qe;
          break;
        }
        rr -= sz;
      }
      const long long col = pair_fso(alpha, x, qe, qo);
      double acc = 0.0;
      for (int k = 0; k < D; ++k) acc += a[pair_fso(beta, k, qe, qo) * q2 + col];
      T[e] = acc;
    } else {
      const long long f = e - nT;
      const int dd = (int)(f / q), r = (int)(f % q);
      const long long col = pair_fso(dd, r, qe, qo);
      double acc = 0.0;
      for (int k = 0; k < D; ++k)
        for (int m = 0; m < D; ++m) acc += a[pair_fso(k, m, qe, qo) * q2 + col];
      C[f] = acc;
    }
  }
}

template <typename F>
__global__ void graded_select_kernel(const F* __restrict__ w, const F* __restrict__ V, int n, int chi,
                                     double* __restrict__ PT, SelectOut* sel) {
  hs_pdl_enter();
  const int k = chi < n ? chi : n;
  const int j = blockIdx.x;
  if (j >= k) return;
  const F* src = V + (long long)(n - 1 - j) * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) PT[(long long)j * n + i] = (double)src[i];
  if (j == 0 && threadIdx.x == 0) {
    auto sv = [&](int i) { return sqrt(fmax((double)w[i], 0.0)); };
    sel->chi_new[0] = k;
    sel->chi_new[1] = 0;
    sel->pad[0] = sel->pad[1] = 0;
    sel->lam_max = sv(n - 1);
    sel->lam_cut = sv(n - k);
    sel->lam_next = k < n ? sv(n - k - 1) : 0.0;
    double disc = 0.0;
    for (int i = 0; i < n - k; ++i) disc += sv(i);
    sel->discarded = disc;
  }
}

}  // namespace

cudaError_t launch_graded_sign(const double* src, double* dst, long long r0, long long r1, long long c0,
                               long long c1, long long ld, int mode, cudaStream_t s) {
  const long long total = (r0 + r1) * (c0 + c1);
  if (total == 0) return cudaSuccess;
  hs_launch(graded_sign_kernel, grid_for(total), 256, 0, s, src, dst, r0, r1, c0, c1, ld, mode);
  return cudaGetLastError();
}

cudaError_t launch_ctmrg_init_graded(const double* a, int D, double* C, double* T, cudaStream_t s) {
  const long long q = (long long)D * D;
  hs_launch(init_graded_kernel, grid_for(q * q * q + q * q), 256, 0, s, a, D, C, T);
  return cudaGetLastError();
}

cudaError_t launch_graded_select(const double* w, const double* V, int n, int chi, double* PT, SelectOut* sel,
                                 cudaStream_t s) {
  const int k = chi < n ? chi : n;
  if (k <= 0) return cudaErrorInvalidValue;
  hs_launch(graded_select_kernel<double>, k, 256, 0, s, w, V, n, chi, PT, sel);
  return cudaGetLastError();
}

cudaError_t launch_graded_select32(const float* w, const float* V, int n, int chi, double* PT, SelectOut* sel,
                                   cudaStream_t s) {
  const int k = chi < n ? chi : n;
  if (k <= 0) return cudaErrorInvalidValue;
  hs_launch(graded_select_kernel<float>, k, 256, 0, s, w, V, n, chi, PT, sel);
  return cudaGetLastError();
}

}  // namespace hs

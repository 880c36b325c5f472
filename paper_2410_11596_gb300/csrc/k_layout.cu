// Host-side planning of FSO permutations and block GEMMs (Z2 bookkeeping,
// arXiv 2410.11596 Sec. II.B), plus the generic permute kernel.
#include <cuda_bf16.h>

#include "hs_internal.cuh"

namespace hs {

namespace {

// Strides of each leg of a Z2 matrix inside the sub-block (tr, tc).
void leg_strides(const Z2Mat& m, const int* par, long long* stride, long long* off) {
  int tr = 0, tc = 0;
  for (int j = 0; j < m.r.k; ++j) tr = (tr << 1) | par[j];
  for (int j = 0; j < m.c.k; ++j) tc = (tc << 1) | par[m.r.k + j];
  const int P = tuple_parity(tr);
  const long long CP = z2_ld(m, P);
  *off = z2_block_off(m, P) + tuple_offset(m.r, tr) * CP + tuple_offset(m.c, tc);
  long long s = CP;
  for (int j = m.r.k - 1; j >= 0; --j) {
    stride[j] = s;
    s *= m.r.leg[j].n[par[j]];
  }
  s = 1;
  for (int j = m.c.k - 1; j >= 0; --j) {
    stride[m.r.k + j] = s;
    s *= m.c.leg[j].n[par[m.r.k + j]];
  }
}

Sect leg_of(const Z2Mat& m, int j) { return j < m.r.k ? m.r.leg[j] : m.c.leg[j - m.r.k]; }

}  // namespace

PermPlan make_perm_plan(const Z2Mat& in, const Z2Mat& out, const int* perm) {
  PermPlan plan{};
  const int n = out.r.k + out.c.k;
  long long start = 0;
  for (int bits = 0; bits < (1 << n); ++bits) {
    if (tuple_parity(bits)) continue;
    int pout[kMaxLegs] = {0}, pin[kMaxLegs] = {0};
    for (int j = 0; j < n; ++j) {
      pout[j] = (bits >> (n - 1 - j)) & 1;
      pin[perm[j]] = pout[j];
    }
    long long ostr[kMaxLegs], istr_leg[kMaxLegs], ooff, ioff;
    leg_strides(out, pout, ostr, &ooff);
    leg_strides(in, pin, istr_leg, &ioff);
    Box b{};
    b.out_off = ooff;
    b.in_off = ioff;
    b.count = 1;
    const int pad = kMaxLegs - n;
    for (int j = 0; j < kMaxLegs; ++j) {
      b.dim[j] = 1;
      b.out_stride[j] = 0;
      b.in_stride[j] = 0;
    }
    for (int j = 0; j < n; ++j) {
      b.dim[pad + j] = leg_of(out, j).n[pout[j]];
      b.out_stride[pad + j] = ostr[j];
      b.in_stride[pad + j] = istr_leg[perm[j]];
      b.count *= b.dim[pad + j];
    }
    if (b.count == 0) continue;
    b.start = start;
    start += b.count;
    plan.box[plan.nbox++] = b;
  }
  plan.total = start;
  return plan;
}

GemmGroup make_z2_gemm(const Z2Mat& A, const Z2Mat& B, const Z2Mat& C) {
  GemmGroup g{};
  for (int p = 0; p < 2; ++p) {
    GemmProblem q{};
    q.M = (int)z2_rows(A, p);
    q.K = (int)z2_cols(A, p);
    q.N = (int)z2_rows(B, p);
    if (q.M == 0 || q.N == 0) continue;
    q.lda = (int)z2_ld(A, p);
    q.ldb = (int)z2_ld(B, p);
    q.ldc = (int)z2_ld(C, p);
    q.a_off = z2_block_off(A, p);
    q.b_off = z2_block_off(B, p);
    q.c_off = z2_block_off(C, p);
    g.p[g.n++] = q;
  }
  return g;
}

double gemm_flops(const GemmGroup& g) {
  double f = 0;
  for (int i = 0; i < g.n; ++i) f += 2.0 * g.p[i].M * (double)g.p[i].N * g.p[i].K;
  return f;
}

// ---- permute: one dense box per blockIdx.y, grid-stride over its elements ----

__global__ void permute_f64_kernel(PermPlan plan, const double* __restrict__ in,
                                   double* __restrict__ out, double scale) {
  const Box& b = plan.box[blockIdx.y];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < b.count; e += stride) {
    long long r = e, io = b.in_off, oo = b.out_off;
#pragma unroll
    for (int j = kMaxLegs - 1; j > 0; --j) {
      const int ij = (int)(r % b.dim[j]);
      r /= b.dim[j];
      io += ij * b.in_stride[j];
      oo += ij * b.out_stride[j];
    }
    io += r * b.in_stride[0];
    oo += r * b.out_stride[0];
    out[oo] = scale * in[io];
  }
}

template <int MODE>
__global__ void permute_split_kernel(PermPlan plan, const double* __restrict__ in, void* __restrict__ hi,
                                     void* __restrict__ lo) {
  const Box& b = plan.box[blockIdx.y];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < b.count; e += stride) {
    long long r = e, io = b.in_off, oo = b.out_off;
#pragma unroll
    for (int j = kMaxLegs - 1; j > 0; --j) {
      const int ij = (int)(r % b.dim[j]);
      r /= b.dim[j];
      io += ij * b.in_stride[j];
      oo += ij * b.out_stride[j];
    }
    io += r * b.in_stride[0];
    oo += r * b.out_stride[0];
    const double x = in[io];
    if (MODE == 1) {
      float h;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=f"(h) : "f"((float)x));
      static_cast<float*>(hi)[oo] = h;
      static_cast<float*>(lo)[oo] = (float)(x - (double)h);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
      static_cast<__nv_bfloat16*>(hi)[oo] = h;
      static_cast<__nv_bfloat16*>(lo)[oo] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
    }
  }
}

cudaError_t launch_permute_split(const PermPlan& plan, const double* in, void* hi, void* lo, int mode,
                                 cudaStream_t s) {
  if (plan.nbox == 0) return cudaSuccess;
  long long maxc = 0;
  for (int i = 0; i < plan.nbox; ++i) maxc = plan.box[i].count > maxc ? plan.box[i].count : maxc;
  long long gx = (maxc + 255) / 256;
  if (gx > 2048) gx = 2048;
  dim3 grid((unsigned)gx, (unsigned)plan.nbox);
  if (mode == 1)
    permute_split_kernel<1><<<grid, 256, 0, s>>>(plan, in, hi, lo);
  else
    permute_split_kernel<2><<<grid, 256, 0, s>>>(plan, in, hi, lo);
  return cudaGetLastError();
}

template <int MODE>
__global__ void split_pad_kernel(const double* __restrict__ src, long long rows, int cols, long long ld_src,
                                 void* __restrict__ hi, void* __restrict__ lo, long long ld_dst) {
  const long long total = rows * ld_dst;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / ld_dst;
    const int c = (int)(e % ld_dst);
    const double x = c < cols ? src[r * ld_src + c] : 0.0;
    if (MODE == 1) {
      float h;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=f"(h) : "f"((float)x));
      static_cast<float*>(hi)[e] = h;
      static_cast<float*>(lo)[e] = (float)(x - (double)h);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
      static_cast<__nv_bfloat16*>(hi)[e] = h;
      static_cast<__nv_bfloat16*>(lo)[e] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
    }
  }
}

cudaError_t launch_split_pad(const double* src, long long rows, int cols, long long ld_src, void* hi,
                             void* lo, long long ld_dst, int mode, cudaStream_t s) {
  const long long total = rows * ld_dst;
  if (total == 0) return cudaSuccess;
  long long gx = (total + 255) / 256;
  if (gx > 4096) gx = 4096;
  if (mode == 1)
    split_pad_kernel<1><<<(unsigned)gx, 256, 0, s>>>(src, rows, cols, ld_src, hi, lo, ld_dst);
  else
    split_pad_kernel<2><<<(unsigned)gx, 256, 0, s>>>(src, rows, cols, ld_src, hi, lo, ld_dst);
  return cudaGetLastError();
}

cudaError_t launch_permute_f64(const PermPlan& plan, const double* in, double* out, double scale,
                               cudaStream_t s) {
  if (plan.nbox == 0) return cudaSuccess;
  long long maxc = 0;
  for (int i = 0; i < plan.nbox; ++i) maxc = plan.box[i].count > maxc ? plan.box[i].count : maxc;
  long long gx = (maxc + 255) / 256;
  if (gx > 2048) gx = 2048;
  dim3 grid((unsigned)gx, (unsigned)plan.nbox);
  permute_f64_kernel<<<grid, 256, 0, s>>>(plan, in, out, scale);
  return cudaGetLastError();
}

}  // namespace hs

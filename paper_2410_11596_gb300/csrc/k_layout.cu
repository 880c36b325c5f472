// Host-side planning of FSO permutations and block GEMMs (Z2 bookkeeping,
// arXiv 2410.11596 Sec. II.B), plus the generic permute kernel.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "hs_bits.cuh"
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

// Chunked-traversal fields of a box (dims, strides, offsets and count set).
void set_chunks(Box& b) {
  const long long inner = b.dim[kMaxLegs - 1];
  long long in_max = b.in_off, out_max = b.out_off;
  for (int j = 0; j < kMaxLegs; ++j) {
    in_max += (long long)(b.dim[j] - 1) * b.in_stride[j];
    out_max += (long long)(b.dim[j] - 1) * b.out_stride[j];
  }
  const long long rows = inner > 0 ? b.count / inner : 0;
  const long long nch = (inner + kPermVec - 1) / kPermVec;
  const long long lim = 1ll << 31;
  b.fits32 = inner > 0 && in_max < lim && out_max < lim && rows * nch < lim && b.count < lim;
  for (int j = 0; j < kMaxLegs; ++j)
    if (b.in_stride[j] >= lim || b.out_stride[j] >= lim) b.fits32 = 0;
  b.rows = (unsigned)rows;
  b.nch = (unsigned)(nch > 0 ? nch : 1);
  fast_div_magic(b.nch, &b.magc, &b.sh1c, &b.sh2c);
  // tiled transpose when the input's contiguous dim is another one and both
  // extents fill whole tiles (for smaller extents the chunked traversal,
  // whose loads stay within L2-resident lines, is faster than staging tiles
  // that are mostly empty)
  b.ji = -1;
  b.nbd = 0;
  b.plane = 0;
  const int jo = kMaxLegs - 1;
  if (!b.fits32 || b.out_stride[jo] != 1 || b.in_stride[jo] == 1 || b.dim[jo] < 2) return;
  int ji = -1;
  for (int j = b.lo; j < jo; ++j)
    if (b.in_stride[j] == 1 && b.dim[j] >= 2) ji = j;
  if (ji < 0) return;
  const long long psz = (long long)b.dim[ji] * b.dim[jo];
  if (b.dim[ji] >= kPermTile && b.dim[jo] >= kPermTile) {
    b.ji = ji;  // tiled
  } else if (psz <= kPermPlaneElems / 2) {
    // whole planes, several per step
    b.ji = ji;
    b.plane = (int)std::min<long long>(16, kPermPlaneElems / psz);
    b.psz = (unsigned)psz;
    fast_div_magic(b.psz, &b.magp, &b.sh1p, &b.sh2p);
    fast_div_magic((unsigned)b.dim[ji], &b.magpi, &b.sh1pi, &b.sh2pi);
    fast_div_magic((unsigned)b.dim[jo], &b.magpo, &b.sh1po, &b.sh2po);
  } else {
    return;
  }
  b.ntile_i = (unsigned)((b.dim[ji] + kPermTile - 1) / kPermTile);
  b.ntile_o = (unsigned)((b.dim[jo] + kPermTile - 1) / kPermTile);
  b.nbatch = (unsigned)(b.count / ((long long)b.dim[ji] * b.dim[jo]));
  fast_div_magic(b.ntile_o, &b.magto, &b.sh1to, &b.sh2to);
  fast_div_magic(b.ntile_i, &b.magti, &b.sh1ti, &b.sh2ti);
  for (int j = b.lo; j < jo; ++j) {
    if (j == ji) continue;
    const int k = b.nbd++;
    b.bdim[k] = b.dim[j];
    b.bin_stride[k] = (unsigned)b.in_stride[j];
    b.bout_stride[k] = (unsigned)b.out_stride[j];
    fast_div_magic((unsigned)b.dim[j], &b.bmag[k], &b.bsh1[k], &b.bsh2[k]);
  }
}

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
    for (int j = 0; j < kMaxLegs; ++j) fast_div_magic((unsigned)b.dim[j], &b.mag[j], &b.sh1[j], &b.sh2[j]);
    b.lo = n > 0 ? kMaxLegs - n : kMaxLegs - 1;
    set_chunks(b);
    b.start = start;
    start += b.count;
    plan.box[plan.nbox++] = b;
  }
  plan.total = start;
  return plan;
}

namespace {

// Strides of each leg of a graded matrix inside the parity tuple `par`.
void graded_leg_strides(const GMat& m, const int* par, long long* stride, long long* off) {
  int tr = 0, tc = 0;
  for (int j = 0; j < m.r.k; ++j) tr = (tr << 1) | par[j];
  for (int j = 0; j < m.c.k; ++j) tc = (tc << 1) | par[m.r.k + j];
  const long long ld = g_ld(m);
  const long long row = g_row0(m, tuple_parity(tr)) + tuple_offset(m.r, tr);
  const long long col = g_col0(m, tuple_parity(tc)) + tuple_offset(m.c, tc);
  *off = row * ld + col;
  long long s = ld;
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

Sect gleg_of(const GMat& m, int j) { return j < m.r.k ? m.r.leg[j] : m.c.leg[j - m.r.k]; }

}  // namespace

bool make_graded_perm_plan(const GMat& in, const GMat& out, const int* perm, PermPlan* plan_out) {
  PermPlan plan{};
  const int n = out.r.k + out.c.k;
  if (n > kMaxLegs || (1 << n) > kMaxBoxes) return false;
  long long start = 0;
  for (int bits = 0; bits < (1 << n); ++bits) {
    int pout[kMaxLegs] = {0}, pin[kMaxLegs] = {0};
    for (int j = 0; j < n; ++j) {
      pout[j] = (bits >> (n - 1 - j)) & 1;
      pin[perm[j]] = pout[j];
    }
    long long ostr[kMaxLegs], istr_leg[kMaxLegs], ooff, ioff;
    graded_leg_strides(out, pout, ostr, &ooff);
    graded_leg_strides(in, pin, istr_leg, &ioff);
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
      b.dim[pad + j] = gleg_of(out, j).n[pout[j]];
      b.out_stride[pad + j] = ostr[j];
      b.in_stride[pad + j] = istr_leg[perm[j]];
      b.count *= b.dim[pad + j];
    }
    if (b.count == 0) continue;
    for (int j = 0; j < kMaxLegs; ++j) fast_div_magic((unsigned)b.dim[j], &b.mag[j], &b.sh1[j], &b.sh2[j]);
    b.lo = n > 0 ? kMaxLegs - n : kMaxLegs - 1;
    set_chunks(b);
    b.start = start;
    start += b.count;
    plan.box[plan.nbox++] = b;
  }
  plan.total = start;
  *plan_out = plan;
  return true;
}

GemmGroup make_graded_gemm(const GMat& A, const GMat& B, const GMat& C, long long bconj_off) {
  GemmGroup g{};
  for (int pr = 0; pr < 2; ++pr)
    for (int pc = 0; pc < 2; ++pc) {
      GemmProblem q{};
      q.M = (int)fused_size(A.r, pr);
      q.N = (int)fused_size(B.r, pc);
      q.K = (int)g_cols(A);
      if (q.M == 0 || q.N == 0) continue;
      q.lda = (int)g_ld(A);
      q.ldb = (int)g_ld(B);
      q.ldc = (int)g_ld(C);
      q.a_off = g_row0(A, pr) * g_ld(A);
      q.b_off = g_row0(B, pc) * g_ld(B) + (pr == pc ? bconj_off : 0);
      q.c_off = g_row0(C, pr) * g_ld(C) + g_col0(C, pc);
      g.p[g.n++] = q;
    }
  return g;
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

// Input and output offsets of element e of box b (row-major over b.dim).
// Boxes below 2^31 elements decode with 32-bit multiply-high divisions.
__device__ __forceinline__ void box_offsets(const Box& b, long long e, long long& io, long long& oo) {
  io = b.in_off;
  oo = b.out_off;
  if (b.count < (1ll << 31)) {
    // only the box's own dims (the leading extent-1 dims add nothing)
    unsigned r = (unsigned)e;
    for (int j = kMaxLegs - 1; j > b.lo; --j) {
      const unsigned qd = fast_div(r, b.mag[j], b.sh1[j], b.sh2[j]);
      const unsigned ij = r - qd * (unsigned)b.dim[j];
      r = qd;
      io += (long long)ij * b.in_stride[j];
      oo += (long long)ij * b.out_stride[j];
    }
    io += (long long)r * b.in_stride[b.lo];
    oo += (long long)r * b.out_stride[b.lo];
  } else {
    long long r = e;
#pragma unroll
    for (int j = kMaxLegs - 1; j > 0; --j) {
      const int ij = (int)(r % b.dim[j]);
      r /= b.dim[j];
      io += ij * b.in_stride[j];
      oo += ij * b.out_stride[j];
    }
    io += r * b.in_stride[0];
    oo += r * b.out_stride[0];
  }
}

// 32-bit start offsets of row `row` of box b (fits32): every dim but the
// innermost, decoded once per chunk of kPermVec innermost elements.
__device__ __forceinline__ void row_offsets32(const Box& b, unsigned row, unsigned& io, unsigned& oo) {
  io = (unsigned)b.in_off;
  oo = (unsigned)b.out_off;
  unsigned r = row;
  for (int j = kMaxLegs - 2; j > b.lo; --j) {
    const unsigned qd = fast_div(r, b.mag[j], b.sh1[j], b.sh2[j]);
    const unsigned ij = r - qd * (unsigned)b.dim[j];
    r = qd;
    io += ij * (unsigned)b.in_stride[j];
    oo += ij * (unsigned)b.out_stride[j];
  }
  if (b.lo < kMaxLegs - 1) {
    io += r * (unsigned)b.in_stride[b.lo];
    oo += r * (unsigned)b.out_stride[b.lo];
  }
}

// Threads a box needs: a CTA of 256 per tile (tiled), one per chunk
// (fits32) or one per element.
long long max_work(const PermPlan& plan) {
  long long w = 0;
  for (int i = 0; i < plan.nbox; ++i) {
    const Box& b = plan.box[i];
    const long long t = b.plane > 0 ? 256LL * ((b.nbatch + b.plane - 1) / b.plane)
                        : b.ji >= 0  ? 256LL * b.nbatch * b.ntile_i * b.ntile_o
                        : b.fits32   ? (long long)b.rows * b.nch
                                     : b.count;
    w = t > w ? t : w;
  }
  return w;
}

// Tiled transpose of box b: each CTA stages a tile (rows along the innermost
// output dim, columns along the input's contiguous dim) in shared memory, so
// both the loads and the stores run along contiguous addresses. `store`
// writes one value at an output offset.
template <class T, class Store>
__device__ __forceinline__ void permute_tiled(const Box& b, const T* __restrict__ in, Store store) {
  __shared__ T tile[kPermTile][kPermTile + 1];
  constexpr int jo = kMaxLegs - 1;
  const unsigned di = (unsigned)b.dim[b.ji], dout = (unsigned)b.dim[jo];
  const unsigned is_o = (unsigned)b.in_stride[jo], os_i = (unsigned)b.out_stride[b.ji];
  const unsigned ntiles = b.nbatch * b.ntile_i * b.ntile_o;
  for (unsigned t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const unsigned t1 = fast_div(t, b.magto, b.sh1to, b.sh2to);
    const unsigned to = t - t1 * b.ntile_o;
    unsigned r = fast_div(t1, b.magti, b.sh1ti, b.sh2ti);
    const unsigned ti = t1 - r * b.ntile_i;
    unsigned io = (unsigned)b.in_off, oo = (unsigned)b.out_off;
    for (int k = b.nbd - 1; k >= 0; --k) {
      const unsigned q = fast_div(r, b.bmag[k], b.bsh1[k], b.bsh2[k]);
      const unsigned ik = r - q * (unsigned)b.bdim[k];
      r = q;
      io += ik * b.bin_stride[k];
      oo += ik * b.bout_stride[k];
    }
    const unsigned i0 = ti * kPermTile, o0 = to * kPermTile;
    const unsigned ni = di - i0 < (unsigned)kPermTile ? di - i0 : (unsigned)kPermTile;
    const unsigned no = dout - o0 < (unsigned)kPermTile ? dout - o0 : (unsigned)kPermTile;
    for (unsigned e = threadIdx.x; e < kPermTile * kPermTile; e += blockDim.x) {
      const unsigned rr = e / kPermTile, cc = e % kPermTile;  // rr along the output dim, cc along the input's
      if (rr < no && cc < ni) tile[rr][cc] = in[io + (o0 + rr) * is_o + i0 + cc];
    }
    __syncthreads();
    for (unsigned e = threadIdx.x; e < kPermTile * kPermTile; e += blockDim.x) {
      const unsigned rr = e / kPermTile, cc = e % kPermTile;  // rr along the input's dim, cc along the output's
      if (rr < ni && cc < no) store(oo + (i0 + rr) * os_i + o0 + cc, tile[cc][rr]);
    }
    __syncthreads();
  }
}

// Offsets of batch item r of box b (its dims other than ji and the innermost).
__device__ __forceinline__ void batch_offsets(const Box& b, unsigned r, unsigned& io, unsigned& oo) {
  io = (unsigned)b.in_off;
  oo = (unsigned)b.out_off;
  for (int k = b.nbd - 1; k >= 0; --k) {
    const unsigned q = fast_div(r, b.bmag[k], b.bsh1[k], b.bsh2[k]);
    const unsigned ik = r - q * (unsigned)b.bdim[k];
    r = q;
    io += ik * b.bin_stride[k];
    oo += ik * b.bout_stride[k];
  }
}

// Plane-mode transpose of box b: a CTA stages b.plane whole (dim ji x
// innermost dim) planes in shared memory, read in input order and written in
// output order, both along contiguous runs.
template <class T, class Store>
__device__ __forceinline__ void permute_planes(const Box& b, const T* __restrict__ in, Store store) {
  __shared__ T buf[kPermPlaneElems];
  __shared__ unsigned s_io[16], s_oo[16];
  constexpr int jo = kMaxLegs - 1;
  const unsigned pi = (unsigned)b.dim[b.ji], po = (unsigned)b.dim[jo];
  const unsigned is_o = (unsigned)b.in_stride[jo], os_i = (unsigned)b.out_stride[b.ji];
  const unsigned P = (unsigned)b.plane, groups = (b.nbatch + P - 1) / P;
  for (unsigned g = blockIdx.x; g < groups; g += gridDim.x) {
    const unsigned b0 = g * P, np = b.nbatch - b0 < P ? b.nbatch - b0 : P;
    if (threadIdx.x < np) batch_offsets(b, b0 + threadIdx.x, s_io[threadIdx.x], s_oo[threadIdx.x]);
    __syncthreads();
    const unsigned tot = np * b.psz;
    for (unsigned e = threadIdx.x; e < tot; e += blockDim.x) {  // input order: i fastest
      const unsigned p = fast_div(e, b.magp, b.sh1p, b.sh2p), rem = e - p * b.psz;
      const unsigned o = fast_div(rem, b.magpi, b.sh1pi, b.sh2pi), i = rem - o * pi;
      buf[e] = in[s_io[p] + o * is_o + i];
    }
    __syncthreads();
    for (unsigned e = threadIdx.x; e < tot; e += blockDim.x) {  // output order: o fastest
      const unsigned p = fast_div(e, b.magp, b.sh1p, b.sh2p), rem = e - p * b.psz;
      const unsigned i = fast_div(rem, b.magpo, b.sh1po, b.sh2po), o = rem - i * po;
      store(s_oo[p] + i * os_i + o, buf[p * b.psz + o * pi + i]);
    }
    __syncthreads();
  }
}

// The kernels take the plan's boxes by value in a parameter block sized to
// the plan (NB boxes of 192 bytes): a full 32-box plan is a 6 KB parameter
// block, which makes every launch of the common 2- and 8-box plans slower.
template <int NB>
struct PlanArg {
  Box box[NB];
};

// Each thread moves a chunk of kPermVec consecutive innermost elements (one
// index decode per chunk, loads issued before the stores); boxes beyond the
// 32-bit range go element by element. T: double or float (scale 1 only).
template <int NB, class T, bool SCALE>
__global__ void permute_kernel(PlanArg<NB> plan, const T* __restrict__ in, T* __restrict__ out, double scale) {
  hs_pdl_enter();
  const Box& b = plan.box[blockIdx.y];
  // plain copies (SCALE false) keep off the FP64 pipe entirely
  auto put = [&](unsigned long long o, T v) {
    if (SCALE)
      out[o] = (T)(scale * v);
    else
      out[o] = v;
  };
  if (b.plane > 0) {
    permute_planes(b, in, [&](unsigned o, T v) { put(o, v); });
    return;
  }
  if (b.ji >= 0) {
    permute_tiled(b, in, [&](unsigned o, T v) { put(o, v); });
    return;
  }
  if (b.fits32) {
    const unsigned inner = (unsigned)b.dim[kMaxLegs - 1];
    const unsigned istr = (unsigned)b.in_stride[kMaxLegs - 1], ostr = (unsigned)b.out_stride[kMaxLegs - 1];
    const unsigned total = b.rows * b.nch;
    for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < total; c += gridDim.x * blockDim.x) {
      const unsigned row = fast_div(c, b.magc, b.sh1c, b.sh2c);
      const unsigned i0 = (c - row * b.nch) * kPermVec;
      unsigned io, oo;
      row_offsets32(b, row, io, oo);
      io += i0 * istr;
      oo += i0 * ostr;
      const unsigned nv = inner - i0 < (unsigned)kPermVec ? inner - i0 : (unsigned)kPermVec;
      T v[kPermVec];
#pragma unroll
      for (int k = 0; k < kPermVec; ++k)
        if ((unsigned)k < nv) v[k] = in[io + k * istr];
#pragma unroll
      for (int k = 0; k < kPermVec; ++k)
        if ((unsigned)k < nv) put(oo + k * ostr, v[k]);
    }
    return;
  }
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < b.count; e += stride) {
    long long io, oo;
    box_offsets(b, e, io, oo);
    put((unsigned long long)oo, in[io]);
  }
}

// An FP32 value: TF32x3 through one FP32 subtraction (split_f32_tf32x3);
// BF16x3 through the general split of its exact FP64 value.
template <int MODE>
__device__ __forceinline__ void store_split(float x, void* hi, void* lo, long long o) {
  if (MODE == 1) {
    uint32_t h, l;
    split_f32_tf32x3(__float_as_uint(x), h, l);
    static_cast<uint32_t*>(hi)[o] = h;
    static_cast<uint32_t*>(lo)[o] = l;
  } else {
    uint32_t h, l;
    unsigned long long w;
    if (!f32_widen_fast(__float_as_uint(x), w)) w = 0ull;  // subnormal: below the split's range anyway
    split_f64(f64_from_bits(w), 8, 8, false, h, l);
    static_cast<unsigned short*>(hi)[o] = (unsigned short)(h >> 16);
    static_cast<unsigned short*>(lo)[o] = (unsigned short)(l >> 16);
  }
}

template <int MODE>
__device__ __forceinline__ void store_split(double x, void* hi, void* lo, long long o) {
  if (MODE == 1) {
    uint32_t h, l;
    split_tf32x3(x, h, l);
    static_cast<uint32_t*>(hi)[o] = h;
    static_cast<uint32_t*>(lo)[o] = l;
  } else {
    uint32_t h, l;
    split_f64(x, 8, 8, false, h, l);
    static_cast<unsigned short*>(hi)[o] = (unsigned short)(h >> 16);
    static_cast<unsigned short*>(lo)[o] = (unsigned short)(l >> 16);
  }
}

template <int MODE, int NB, class T>
__global__ void permute_split_kernel(PlanArg<NB> plan, const T* __restrict__ in, void* __restrict__ hi,
                                     void* __restrict__ lo) {
  hs_pdl_enter();
  const Box& b = plan.box[blockIdx.y];
  if (b.plane > 0) {
    permute_planes(b, in, [&](unsigned o, T v) { store_split<MODE>(v, hi, lo, (long long)o); });
    return;
  }
  if (b.ji >= 0) {
    permute_tiled(b, in, [&](unsigned o, T v) { store_split<MODE>(v, hi, lo, (long long)o); });
    return;
  }
  if (b.fits32) {
    const unsigned inner = (unsigned)b.dim[kMaxLegs - 1];
    const unsigned istr = (unsigned)b.in_stride[kMaxLegs - 1], ostr = (unsigned)b.out_stride[kMaxLegs - 1];
    const unsigned total = b.rows * b.nch;
    for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < total; c += gridDim.x * blockDim.x) {
      const unsigned row = fast_div(c, b.magc, b.sh1c, b.sh2c);
      const unsigned i0 = (c - row * b.nch) * kPermVec;
      unsigned io, oo;
      row_offsets32(b, row, io, oo);
      io += i0 * istr;
      oo += i0 * ostr;
      const unsigned nv = inner - i0 < (unsigned)kPermVec ? inner - i0 : (unsigned)kPermVec;
      T v[kPermVec];
#pragma unroll
      for (int k = 0; k < kPermVec; ++k)
        if ((unsigned)k < nv) v[k] = in[io + k * istr];
#pragma unroll
      for (int k = 0; k < kPermVec; ++k)
        if ((unsigned)k < nv) store_split<MODE>(v[k], hi, lo, (long long)(oo + k * ostr));
    }
    return;
  }
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < b.count; e += stride) {
    long long io, oo;
    box_offsets(b, e, io, oo);
    store_split<MODE>(in[io], hi, lo, oo);
  }
}

template <class T>
cudaError_t launch_permute_split_t(const PermPlan& plan, const T* in, void* hi, void* lo, int mode, cudaStream_t s) {
  if (plan.nbox == 0) return cudaSuccess;
  const long long maxc = max_work(plan);
  long long gx = (maxc + 255) / 256;
  if (gx > 2048) gx = 2048;
  dim3 grid((unsigned)gx, (unsigned)plan.nbox);
  auto go = [&](auto nb) {
    constexpr int NB = decltype(nb)::value;
    PlanArg<NB> arg;
    for (int i = 0; i < plan.nbox; ++i) arg.box[i] = plan.box[i];
    if (mode == 1)
      hs_launch(permute_split_kernel<1, NB, T>, grid, 256, 0, s, arg, in, hi, lo);
    else
      hs_launch(permute_split_kernel<2, NB, T>, grid, 256, 0, s, arg, in, hi, lo);
  };
  if (plan.nbox <= 2)
    go(std::integral_constant<int, 2>{});
  else if (plan.nbox <= 8)
    go(std::integral_constant<int, 8>{});
  else
    go(std::integral_constant<int, kMaxBoxes>{});
  return cudaGetLastError();
}

cudaError_t launch_permute_split(const PermPlan& plan, const double* in, void* hi, void* lo, int mode,
                                 cudaStream_t s) {
  return launch_permute_split_t(plan, in, hi, lo, mode, s);
}

cudaError_t launch_permute_split_f32(const PermPlan& plan, const float* in, void* hi, void* lo, int mode,
                                     cudaStream_t s) {
  return launch_permute_split_t(plan, in, hi, lo, mode, s);
}

template <int MODE>
__global__ void split_pad_kernel(const double* __restrict__ src, long long rows, int cols, long long ld_src,
                                 void* __restrict__ hi, void* __restrict__ lo, long long ld_dst) {
  hs_pdl_enter();
  const long long total = rows * ld_dst;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / ld_dst;
    const int c = (int)(e % ld_dst);
    store_split<MODE>(c < cols ? src[r * ld_src + c] : 0.0, hi, lo, e);
  }
}

cudaError_t launch_split_pad(const double* src, long long rows, int cols, long long ld_src, void* hi,
                             void* lo, long long ld_dst, int mode, cudaStream_t s) {
  const long long total = rows * ld_dst;
  if (total == 0) return cudaSuccess;
  long long gx = (total + 255) / 256;
  if (gx > 4096) gx = 4096;
  if (mode == 1)
    hs_launch(split_pad_kernel<1>, (unsigned)gx, 256, 0, s, src, rows, cols, ld_src, hi, lo, ld_dst);
  else
    hs_launch(split_pad_kernel<2>, (unsigned)gx, 256, 0, s, src, rows, cols, ld_src, hi, lo, ld_dst);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_permute_t(const PermPlan& plan, const T* in, T* out, double scale, cudaStream_t s) {
  if (plan.nbox == 0) return cudaSuccess;
  const long long maxc = max_work(plan);
  long long gx = (maxc + 255) / 256;
  if (gx > 2048) gx = 2048;
  dim3 grid((unsigned)gx, (unsigned)plan.nbox);
  auto go = [&](auto nb) {
    constexpr int NB = decltype(nb)::value;
    PlanArg<NB> arg;
    for (int i = 0; i < plan.nbox; ++i) arg.box[i] = plan.box[i];
    if (scale != 1.0)
      hs_launch(permute_kernel<NB, T, true>, grid, 256, 0, s, arg, in, out, scale);
    else
      hs_launch(permute_kernel<NB, T, false>, grid, 256, 0, s, arg, in, out, scale);
  };
  if (plan.nbox <= 2)
    go(std::integral_constant<int, 2>{});
  else if (plan.nbox <= 8)
    go(std::integral_constant<int, 8>{});
  else
    go(std::integral_constant<int, kMaxBoxes>{});
  return cudaGetLastError();
}

cudaError_t launch_permute_f64(const PermPlan& plan, const double* in, double* out, double scale,
                               cudaStream_t s) {
  return launch_permute_t(plan, in, out, scale, s);
}

cudaError_t launch_permute_f32(const PermPlan& plan, const float* in, float* out, cudaStream_t s) {
  return launch_permute_t(plan, in, out, 1.0, s);
}

namespace {

// out[r * cols + c] = hi[r * ld + c] + lo[r * ld + c] for both blocks of a
// TF32x3-split pair (hi a TF32 value, lo the FP32 remainder: the sum is the
// split FP32 value exactly).
__global__ void join_split_f32_kernel(const uint32_t* __restrict__ hi, const uint32_t* __restrict__ lo,
                                      long long rows0, long long cols0, long long ld0, long long off1,
                                      long long rows1, long long cols1, long long ld1, float* __restrict__ out) {
  hs_pdl_enter();
  const long long n0 = rows0 * cols0, total = n0 + rows1 * cols1;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const bool b = e >= n0;
    const long long f = b ? e - n0 : e, cols = b ? cols1 : cols0;
    const long long r = f / cols, c = f - r * cols;
    const long long src = (b ? off1 : 0) + r * (b ? ld1 : ld0) + c;
    out[e] = __uint_as_float(hi[src]) + __uint_as_float(lo[src]);
  }
}

}  // namespace

cudaError_t launch_join_split_f32(const void* hi, const void* lo, long long rows0, long long cols0, long long ld0,
                                  long long off1, long long rows1, long long cols1, long long ld1, float* out,
                                  cudaStream_t s) {
  const long long total = rows0 * cols0 + rows1 * cols1;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  const long long cap = 16LL * device_sms();  // grid-stride loop: 16 blocks per SM
  if (blocks > cap) blocks = cap;
  hs_launch(join_split_f32_kernel, (unsigned)blocks, 256, 0, s, static_cast<const uint32_t*>(hi),
            static_cast<const uint32_t*>(lo), rows0, cols0, ld0, off1, rows1, cols1, ld1, out);
  return cudaGetLastError();
}

}  // namespace hs

// Host check of the destination map of the tensor-core GEMM's split
// epilogue: for the four contractions whose outputs are written as the next
// GEMM's permuted split operand, every output entry's destination (the
// descriptor from make_ps_desc, decoded as the epilogue decodes it: its
// column walk of mode 1 and its per-column division of mode 2) must equal
// the destination the permute plan of the same layouts gives it. Prints
// "ok" when all agree.
#include <cstdio>
#include <vector>
#include "hs_internal.cuh"
namespace hs {
bool make_ps_desc(const Z2Mat& Cm, const Z2Mat& P, const int perm[4], int p, void* hi, void* lo, PsDesc& d);
Z2Mat mat(Fused r, Fused c, int pad);
}
using namespace hs;
static int check(const Z2Mat& src, const Z2Mat& dstl, const int perm[4], const char* name) {
  const Z2Mat P = mat(dstl.r, dstl.c, 32);
  int pm[kMaxLegs] = {perm[0], perm[1], perm[2], perm[3], 0, 0};
  PermPlan plan = make_perm_plan(src, P, pm);
  std::vector<long long> ref(z2_elems(src), -1);
  for (int b = 0; b < plan.nbox; ++b) {
    const Box& x = plan.box[b];
    long long cnt = x.count;
    for (long long e = 0; e < cnt; ++e) {
      long long rem = e, in = x.in_off, out = x.out_off;
      for (int j = kMaxLegs - 1; j >= 0; --j) {
        long long i = rem % x.dim[j];
        rem /= x.dim[j];
        in += i * x.in_stride[j];
        out += i * x.out_stride[j];
      }
      ref[in] = out;
    }
  }
  int bad = 0;
  long long n = 0;
  for (int p = 0; p < 2; ++p) {
    const int M = (int)z2_rows(src, p), N = (int)z2_cols(src, p);
    if (M == 0 || N == 0) continue;
    PsDesc d;
    if (!make_ps_desc(src, P, perm, p, nullptr, nullptr, d)) { printf("%s: no desc\n", name); return 1; }
    for (int r = 0; r < M; ++r) {
      const int tr = r >= d.rsplit;
      const int rin = tr ? d.rin[1] : d.rin[0];
      const int rr = r - (tr ? d.rsplit : 0), i0 = rr / rin, i1 = rr - i0 * rin;
      const int R[2] = {d.base[tr][0] + d.co[tr][0][0] * i0 + d.co[tr][0][1] * i1,
                        d.base[tr][1] + d.co[tr][1][0] * i0 + d.co[tr][1][1] * i1};
      // mode-1 walk over chunks of 32 columns
      for (int c0 = 0; c0 < N; c0 += 32) {
        int tc = c0 >= d.csplit, cin = tc ? d.cin[1] : d.cin[0];
        const int cc = c0 - (tc ? d.csplit : 0);
        int j0 = cc / cin, j1 = cc - j0 * cin;
        for (int j = 0; j < 32 && c0 + j < N; ++j) {
          const int col = c0 + j;
          const int o = R[tc] + d.co[tr][tc][2] * j0 + d.co[tr][tc][3] * j1;
          // division form (mode 2)
          const int tc2 = col >= d.csplit, cin2 = tc2 ? d.cin[1] : d.cin[0];
          const int cc2 = col - (tc2 ? d.csplit : 0), k0 = cc2 / cin2, k1 = cc2 - k0 * cin2;
          const int o2 = R[tc2] + d.co[tr][tc2][2] * k0 + d.co[tr][tc2][3] * k1;
          const long long want = ref[z2_block_off(src, p) + (long long)r * N + col];
          if (o != want || o2 != want || o < 0 || o >= d.limit) {
            if (bad < 5) printf("%s p%d r%d c%d: %d %d want %lld\n", name, p, r, col, o, o2, want);
            ++bad;
          }
          ++n;
          if (++j1 == cin) { j1 = 0; ++j0; }
          if (col + 1 == d.csplit) { tc = 1; j0 = 0; j1 = 0; cin = d.cin[1]; }
        }
      }
    }
  }
  if (bad) printf("%s: %lld entries, %d wrong\n", name, n, bad);
  return bad;
}
int main() {
  int fails = 0;
  // sector sizes (even, odd) of the legs c (corner), q (double layer), cn
  // (kept): small and ragged, the D=6 chi=144 workload, an empty sector
  const Sect cs[3][3] = {{{{5, 3}}, {{2, 3}}, {{4, 2}}}, {{{76, 68}}, {{18, 18}}, {{76, 68}}}, {{{5, 0}}, {{2, 3}}, {{3, 1}}}};
  for (auto& t : cs) {
    const Sect c = t[0], q = t[1], cn = t[2];
    { const int pm[4] = {0, 2, 3, 1}; fails += check(mat(fused2(c, q), fused2(c, q), 1), mat(fused2(c, c), fused2(q, q), 1), pm, "X2->X2p"); }
    { const int pm[4] = {0, 2, 1, 3}; fails += check(mat(fused2(c, c), fused2(q, q), 1), mat(fused2(c, q), fused2(c, q), 1), pm, "X3->Cp"); }
    { const int pm[4] = {1, 2, 0, 3}; fails += check(mat(fused2(q, cn), fused2(c, q), 1), mat(fused2(cn, c), fused2(q, q), 1), pm, "Y->Yp"); }
    { const int pm[4] = {0, 3, 2, 1}; fails += check(mat(fused2(cn, c), fused2(q, q), 1), mat(fused2(cn, q), fused2(q, c), 1), pm, "Z->Zpq"); }
  }
  // layouts the epilogue cannot write are refused (the GEMM then goes through
  // the FP32 output and the permute/split kernel): a destination whose
  // innermost leg is a row or column outer leg, and legs that do not match
  {
    const Sect c = {{5, 3}}, q = {{2, 3}}, cn = {{4, 2}};
    const int pz[4] = {0, 3, 1, 2};  // Z -> Zp with contraction legs (b, u): innermost is L2
    PsDesc d;
    if (make_ps_desc(mat(fused2(cn, c), fused2(q, q), 1), mat(fused2(cn, q), fused2(c, q), 32), pz, 0, nullptr,
                     nullptr, d)) {
      printf("accepted an L2-innermost destination\n");
      ++fails;
    }
    const int px[4] = {0, 2, 3, 1};
    if (make_ps_desc(mat(fused2(c, q), fused2(c, q), 1), mat(fused2(c, c), fused2(q, cn), 32), px, 0, nullptr,
                     nullptr, d)) {
      printf("accepted mismatched legs\n");
      ++fails;
    }
  }
  printf(fails ? "FAIL\n" : "ok\n");
  return fails != 0;
}

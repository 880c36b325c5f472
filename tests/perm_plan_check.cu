// Host dump of the permute plans' element maps: for each case read from
// stdin, build the plan (make_perm_plan for Z2 block matrices,
// make_graded_perm_plan for graded ones) and print, for every element of the
// input matrix (flat index in its storage), the flat index its boxes send it
// to in the output matrix (-1 if no box covers it). The test compares the
// map with the one the layout's definition gives.
//
// A case is one line of integers:
//   mode kr kc  e_0 o_0 ... e_{n-1} o_{n-1}  kr_out  perm_0 ... perm_{n-1}  pad_out
// mode 0: Z2 block matrices, 1: graded matrices; n = kr + kc legs; the
// input's first kr legs are its rows, the output's leg j is input leg
// perm[j] and its first kr_out legs are its rows.
//
// Mode 2 prints the block GEMMs of a Z2 product C[R|N] = A[R|K] B[N|K]^T
// (make_z2_gemm) instead:
//   2 kr kk kn  e_0 o_0 ... (kr + kk + kn legs: R, then K, then N)  padA padB padC
// as "n elemsA elemsB elemsC" and per problem "M N K lda ldb ldc a_off b_off c_off".
// Mode 3 does the same for the graded product of complex tensors
// (make_graded_gemm, the conjugate copy of B stored right after B).
#include <cstdio>
#include <vector>
#include "hs_internal.cuh"

using namespace hs;

static Fused group(const Sect* s, int k) {
  Fused f = fused0();
  f.k = k;
  for (int j = 0; j < k; ++j) f.leg[j] = s[j];
  return f;
}

int main() {
  int mode, kr, kc;
  while (std::scanf("%d %d %d", &mode, &kr, &kc) == 3) {
    if (mode == 2 || mode == 3) {
      int kn, pa, pb, pc;
      if (std::scanf("%d", &kn) != 1) return 1;
      const int n = kr + kc + kn;
      if (kr < 1 || kc < 1 || kn < 1 || kr > kMaxFused || kc > kMaxFused || kn > kMaxFused || n > 12) {
        std::printf("bad case\n");
        return 1;
      }
      Sect s[12];
      for (int j = 0; j < n; ++j)
        if (std::scanf("%d %d", &s[j].n[0], &s[j].n[1]) != 2) return 1;
      if (std::scanf("%d %d %d", &pa, &pb, &pc) != 3) return 1;
      GemmGroup g;
      long long ea, eb, ec;
      if (mode == 2) {
        Z2Mat A, B, C;
        A.r = group(s, kr);
        A.c = group(s + kr, kc);
        A.pad = pa;
        B.r = group(s + kr + kc, kn);
        B.c = group(s + kr, kc);
        B.pad = pb;
        C.r = group(s, kr);
        C.c = group(s + kr + kc, kn);
        C.pad = pc;
        g = make_z2_gemm(A, B, C);
        ea = z2_elems(A);
        eb = z2_elems(B);
        ec = z2_elems(C);
      } else {
        GMat A, B, C;
        A.r = group(s, kr);
        A.c = group(s + kr, kc);
        A.pad = pa;
        B.r = group(s + kr + kc, kn);
        B.c = group(s + kr, kc);
        B.pad = pb;
        C.r = group(s, kr);
        C.c = group(s + kr + kc, kn);
        C.pad = pc;
        g = make_graded_gemm(A, B, C, g_elems(B));
        ea = g_elems(A);
        eb = g_elems(B);
        ec = g_elems(C);
      }
      std::printf("%d %lld %lld %lld", g.n, ea, eb, ec);
      for (int i = 0; i < g.n; ++i) {
        const GemmProblem& q = g.p[i];
        std::printf(" %d %d %d %d %d %d %lld %lld %lld", q.M, q.N, q.K, q.lda, q.ldb, q.ldc, q.a_off, q.b_off,
                    q.c_off);
      }
      std::printf("\n");
      continue;
    }
    const int n = kr + kc;
    if (kr < 1 || kc < 1 || kr > kMaxFused || kc > kMaxFused || n > kMaxLegs) {
      std::printf("bad case\n");
      return 1;
    }
    Sect s[kMaxLegs], so[kMaxLegs];
    for (int j = 0; j < n; ++j)
      if (std::scanf("%d %d", &s[j].n[0], &s[j].n[1]) != 2) return 1;
    int kro, perm[kMaxLegs] = {0, 0, 0, 0, 0, 0}, pad;
    if (std::scanf("%d", &kro) != 1) return 1;
    for (int j = 0; j < n; ++j)
      if (std::scanf("%d", &perm[j]) != 1 || perm[j] < 0 || perm[j] >= n) return 1;
    if (std::scanf("%d", &pad) != 1) return 1;
    if (kro < 1 || n - kro < 1 || kro > kMaxFused || n - kro > kMaxFused) {
      std::printf("bad case\n");
      return 1;
    }
    for (int j = 0; j < n; ++j) so[j] = s[perm[j]];
    PermPlan plan{};
    long long nin, nout;
    if (mode == 0) {
      Z2Mat in, out;
      in.r = group(s, kr);
      in.c = group(s + kr, kc);
      in.pad = 1;
      out.r = group(so, kro);
      out.c = group(so + kro, n - kro);
      out.pad = pad;
      plan = make_perm_plan(in, out, perm);
      nin = z2_elems(in);
      nout = z2_elems(out);
    } else {
      GMat in, out;
      in.r = group(s, kr);
      in.c = group(s + kr, kc);
      in.pad = 1;
      out.r = group(so, kro);
      out.c = group(so + kro, n - kro);
      out.pad = pad;
      if (!make_graded_perm_plan(in, out, perm, &plan)) {
        std::printf("unsupported\n");
        continue;
      }
      nin = g_elems(in);
      nout = g_elems(out);
    }
    std::vector<long long> map(nin, -1);
    bool inside = true;
    for (int b = 0; b < plan.nbox; ++b) {
      const Box& x = plan.box[b];
      for (long long e = 0; e < x.count; ++e) {
        long long rem = e, i = x.in_off, o = x.out_off;
        for (int j = kMaxLegs - 1; j >= 0; --j) {
          const long long t = rem % x.dim[j];
          rem /= x.dim[j];
          i += t * x.in_stride[j];
          o += t * x.out_stride[j];
        }
        if (i < 0 || i >= (long long)map.size() || o < 0 || o >= nout) {
          inside = false;
          continue;
        }
        map[i] = o;
      }
    }
    if (!inside) {
      std::printf("out of range\n");
      return 1;
    }
    std::printf("%lld %lld", (long long)map.size(), nout);
    for (long long v : map) std::printf(" %lld", v);
    std::printf("\n");
  }
  return 0;
}

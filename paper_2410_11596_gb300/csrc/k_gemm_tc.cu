// Tensor-core block GEMM for the CTMRG contractions on sm_103a (tcgen05 + TMEM
// + TMA). Inside one parity block the contraction is a dense GEMM
// (arXiv 2410.11596 Sec. II.B: "product of block diagonal matrices"), so it
// runs on the 5th-generation tensor cores:
//
//   C[M, N] (FP64) = A[M, K] B[N, K]^T,  A and B split as x = hi + lo
//     TF32x3 : acc_main += A_hi B_hi ; acc_corr += A_hi B_lo + A_lo B_hi  (tf32 hi, fp32 lo)
//     TF32   : acc_main += A_hi B_hi
//     BF16x3 : as TF32x3 with a bf16 hi/lo split
//   C = (double)(acc_main + acc_corr), one FP32 add, widened on the bit pattern
// The small cross terms get their own accumulator: folded into the main one
// they lose their low bits to its (truncating) accumulation, about a tenth of
// the accuracy gain of the extra passes on K = 512; the single rounding of
// the final FP32 add is of the order of the accumulation's own.
//
// CTA tile 128 x 128, K step 128 bytes (one 128-byte swizzle atom per row).
// The kernel is persistent: one CTA per SM walks the output tiles
// (blockIdx.x, + gridDim.x, ...). Warp roles:
//   warp 0 lane 0   TMA producer: operand tiles into a multi-stage shared ring
//                   (128-byte swizzle), across tile boundaries;
//   warp 1 lane 0   MMA issuer: tcgen05.mma into one of two TMEM accumulator
//                   buffers, so that tile i+1 accumulates while tile i drains;
//   warps 2..9      epilogue: TMEM -> registers -> FP64, staged through shared
//                   memory so that each warp store writes 16-byte pairs of
//                   eight rows; warp w reads TMEM lanes 32(w%4)... and half
//                   of the tile's columns (two warps per SM sub-partition,
//                   so that one hides the other's latency).
// mbarriers: full (TMA bytes landed), empty (MMAs that read the stage are
// done, via tcgen05.commit), tfull (accumulator ready), tempty (the eight
// epilogue warps have read the accumulator).
//
// Every wait is bounded. A wait that gives up sets *err and an abort flag in
// shared memory; the other roles then stop, the kernel drains what it issued
// (again with bounded waits), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <algorithm>
#include <mutex>

#include "hs_bits.cuh"
#include "hs_internal.cuh"

namespace hs {

namespace {

constexpr int BM = 128, BN = 128;
constexpr int kEpiWarps = 8;              // two per TMEM lane quarter, each on half the columns
constexpr int NT = 32 * (2 + kEpiWarps);  // TMA warp, MMA warp, epilogue warps
constexpr int ROW_BYTES = 128;
constexpr int TILE_BYTES = BM * ROW_BYTES;  // BN == BM
constexpr long long WAIT_LIMIT = 20000000;  // try_wait rounds before giving up (seconds)

constexpr int kMaxPairs = 4;  // operand pairs of one launch (the four graded sub-products)
template <int NM>
struct MapsN {
  CUtensorMap a[NM][2];  // [operand pair][hi, lo]
  CUtensorMap b[NM][2];
};
using Maps = MapsN<kMaxPairs>;

// One launch unit: a K range [k0, k0 + Kp) of an operand pair (map); with
// split-K every range writes its own FP64 partial (c, row stride ldc) and a
// reduction kernel sums them.
constexpr int kMaxUnits = 32;
struct Prob {
  int M, N, Kp, ldc;
  int k0, map;
  int f32;  // output FP32 (c read as float*)
  int psi;  // index of the permuted split output in Group::ps, or -1
  double* c;
  int tile_start, tiles_n;
};

struct Group {
  int n;
  Prob p[kMaxUnits];
  PsDesc ps[kMaxPairs];
};

// PsDesc fields of row tuple tr (0 or 1, runtime) without indexing the
// parameter arrays by it.
__device__ __forceinline__ int ps_base(const PsDesc& D, int tr, int tc) {
  return tr ? D.base[1][tc] : D.base[0][tc];
}
__device__ __forceinline__ int ps_co(const PsDesc& D, int tr, int tc, int k) {
  return tr ? D.co[1][tc][k] : D.co[0][tc][k];
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait (limit try_wait rounds); on timeout records the code and
// raises the abort flag.
__device__ __forceinline__ bool mbar_wait_n(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                            int* err, int code, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  atomicExch(err, code);
  return false;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, int code) {
  return mbar_wait_n(bar, parity, abort_flag, err, code, WAIT_LIMIT);
}

// Drain wait after an abort: bounded, never raises anything.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try(bar, parity)) return;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row core
// groups 1024 bytes apart (rows are 128 bytes), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::tf32 / kind::f16: D = f32, A/B format
// (2 = tf32, 1 = bf16), both K-major, N = BN, M = BM.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int EB>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  if (EB == 4) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc(2)), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc(1)), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int NPASS, int EB>
struct Cfg {
  static constexpr int TILES = NPASS == 1 ? 2 : 4;  // A_hi, B_hi (+ A_lo, B_lo)
  static constexpr int STAGE_BYTES = TILES * TILE_BYTES;
  static constexpr int STAGES = NPASS == 1 ? 5 : 3;
  static constexpr uint32_t ACC_COLS = NPASS == 1 ? BN : 2 * BN;  // one accumulator buffer
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;              // double buffered
  static constexpr int K_PER_TILE = ROW_BYTES / EB;                // elements per 128-byte row
  static constexpr int STG_LD = 10;                                // staging row stride (doubles, 16-byte rows)
  static constexpr int STG_BYTES = kEpiWarps * 32 * STG_LD * 8;    // one 32 x 8 block per epilogue warp
  static constexpr int BAR_BYTES = 256;
  static constexpr int SMEM = STAGES * STAGE_BYTES + STG_BYTES + BAR_BYTES + 1024;
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static_assert(2 * STAGES + 6 <= BAR_BYTES / 8 - 2, "barrier area");
};

// Output tile t of the launch: its unit and corner.
struct TileRef {
  int pi, m0, n0;
};

__device__ __forceinline__ TileRef tile_of(const Group& g, int t) {
  int pi = 0;
  while (pi + 1 < g.n && t >= g.p[pi + 1].tile_start) ++pi;
  t -= g.p[pi].tile_start;
  return {pi, (t / g.p[pi].tiles_n) * BM, (t % g.p[pi].tiles_n) * BN};
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int NPASS, int EB, int NM, bool PS>
__global__ void __launch_bounds__(NT, 1) gemm_tc_kernel(const __grid_constant__ MapsN<NM> maps, const Group g,
                                                        int total_tiles, int* __restrict__ err) {
  hs_pdl_enter();
  using K = Cfg<NPASS, EB>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  double* stage_c = reinterpret_cast<double*>(smem + K::STAGES * K::STAGE_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + K::STAGES * K::STAGE_BYTES + K::STG_BYTES);
  uint64_t* empty = full + K::STAGES;
  uint64_t* tfull = empty + K::STAGES;   // [2]
  uint64_t* tempty = tfull + 2;          // [2]
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(K::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < K::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), kEpiWarps);
    }
    mbar_init(smem_u32(drain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: every K step of every tile of this CTA ----
    long long it = 0;
    for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x) {
      const TileRef r = tile_of(g, t);
      const Prob& P = g.p[r.pi];
      const CUtensorMap* mA0 = &maps.a[P.map][0];
      const CUtensorMap* mA1 = &maps.a[P.map][1];
      const CUtensorMap* mB0 = &maps.b[P.map][0];
      const CUtensorMap* mB1 = &maps.b[P.map][1];
      const int ktiles = P.Kp / K::K_PER_TILE;
      for (int kt = 0; kt < ktiles; ++kt) {
        const int s = (int)(it % K::STAGES);
        const long long n = it / K::STAGES;
        if (n > 0 && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((n - 1) & 1), abort_flag, err, 1)) break;
        if (*abort_flag) break;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, K::STAGE_BYTES);
        const uint32_t st = smem_u32(smem + s * K::STAGE_BYTES);
        const int kc = P.k0 + kt * K::K_PER_TILE;
        tma_load_2d(st, mA0, kc, r.m0, fb);
        tma_load_2d(st + TILE_BYTES, mB0, kc, r.n0, fb);
        if (NPASS == 3) {
          tma_load_2d(st + 2 * TILE_BYTES, mA1, kc, r.m0, fb);
          tma_load_2d(st + 3 * TILE_BYTES, mB1, kc, r.n0, fb);
        }
        ++it;
      }
    }
    if (*abort_flag) {
      // copies still in flight sit in the last STAGES issued steps (earlier
      // ones were consumed); let them land before the CTA can exit
      for (long long j = it > K::STAGES ? it - K::STAGES : 0; j < it; ++j)
        mbar_drain(smem_u32(&full[j % K::STAGES]), (uint32_t)((j / K::STAGES) & 1));
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    long long it = 0;
    bool any = false;
    int local = 0;
    for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x, ++local) {
      const TileRef r = tile_of(g, t);
      const int ktiles = g.p[r.pi].Kp / K::K_PER_TILE;
      const int buf = local & 1, use = local >> 1;
      if (use > 0 && !mbar_wait(smem_u32(&tempty[buf]), (uint32_t)((use - 1) & 1), abort_flag, err, 4)) break;
      fence_after();
      const uint32_t d = tmem + (uint32_t)buf * K::ACC_COLS;
      bool ok = true;
      for (int kt = 0; kt < ktiles; ++kt) {
        const int s = (int)(it % K::STAGES);
        const long long n = it / K::STAGES;
        if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(n & 1), abort_flag, err, 2)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t st = smem_u32(smem + s * K::STAGE_BYTES);
        const uint64_t a_hi = sdesc(st), b_hi = sdesc(st + TILE_BYTES);
        const uint64_t a_lo = sdesc(st + 2 * TILE_BYTES), b_lo = sdesc(st + 3 * TILE_BYTES);
#pragma unroll
        for (int kk = 0; kk < ROW_BYTES / 32; ++kk) {
          const uint64_t off = (uint64_t)((kk * 32) >> 4);
          const uint32_t acc = (kt | kk) != 0;
          mma<EB>(d, a_hi + off, b_hi + off, acc);
          if (NPASS == 3) {
            mma<EB>(d + BN, a_hi + off, b_lo + off, acc);
            mma<EB>(d + BN, a_lo + off, b_hi + off, 1);
          }
        }
        any = true;
        mma_commit(smem_u32(&empty[s]));
        ++it;
      }
      if (!ok) break;
      mma_commit(smem_u32(&tfull[buf]));  // arrives once this tile's MMAs are done
    }
    if (*abort_flag && any) {
      mma_commit(smem_u32(drain));
      mbar_drain(smem_u32(drain), 0);
    }
  } else if (warp >= 2) {
    // ---- epilogue: TMEM -> registers -> shared staging -> coalesced FP64 stores ----
    const int q = warp & 3;               // TMEM lane quarter this warp may read
    const int half = (warp - 2) / 4;      // columns [64 half, 64 half + 64) of the tile
    double* stg = stage_c + (warp - 2) * 32 * K::STG_LD;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int local = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++local) {
      const TileRef r = tile_of(g, t);
      const Prob& P = g.p[r.pi];
      const int ktiles = P.Kp / K::K_PER_TILE;
      const int buf = local & 1, use = local >> 1;
      bool ok = mbar_wait(smem_u32(&tfull[buf]), (uint32_t)(use & 1), abort_flag, err, 3);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      fence_after();
      const uint32_t d = tmem + (uint32_t)buf * K::ACC_COLS + lane_base;
      const int row0 = r.m0 + q * 32;
      // 16-byte stores (FP64) / 8-byte stores (FP32) when every row start is aligned
      const bool vec = P.f32 ? (P.ldc % 2 == 0) && ((reinterpret_cast<uintptr_t>(P.c) & 7) == 0)
                             : (P.ldc % 2 == 0) && ((reinterpret_cast<uintptr_t>(P.c) & 15) == 0);
      // permuted split output: this lane's row (row0 + lane) as its row tuple
      // and its destination offsets for column tuples 0 and 1; in mode 2 also
      // those of the four rows (lane / 4) + 8 k this lane stores
      const int psi = (PS && EB == 4) ? P.psi : -1;
      int ps_tr = 0, ps_r0 = 0, ps_r1 = 0;
      if (psi >= 0) {
        const PsDesc& D = g.ps[psi];
        const int row = row0 + lane;
        if (row < P.M) {
          ps_tr = row >= D.rsplit ? 1 : 0;
          const int rin = ps_tr ? D.rin[1] : D.rin[0];
          const int rr = row - (ps_tr ? D.rsplit : 0);
          const int i0 = rr / rin, i1 = rr - i0 * rin;
          ps_r0 = ps_base(D, ps_tr, 0) + ps_co(D, ps_tr, 0, 0) * i0 + ps_co(D, ps_tr, 0, 1) * i1;
          ps_r1 = ps_base(D, ps_tr, 1) + ps_co(D, ps_tr, 1, 0) * i0 + ps_co(D, ps_tr, 1, 1) * i1;
        }
      }
      for (int c = 64 * half; c < 64 * half + 64 && r.n0 + c < P.N; c += 32) {
        uint32_t r0[32], r1[32];
        if (ktiles > 0) {
          tmem_ld32(d + c, r0);
          if (NPASS == 3) tmem_ld32(d + BN + c, r1);
          tmem_wait_ld();
        }
        if (psi >= 0 && g.ps[psi].mode == 1) {
          // destination innermost along the rows: lane = row, one column per
          // step; the columns' destination offsets (for row tuples 0 and 1)
          // computed once per chunk, one column per lane, into a table
          const PsDesc& D = g.ps[psi];
          uint32_t* hi = static_cast<uint32_t*>(D.hi);
          uint32_t* lo = static_cast<uint32_t*>(D.lo);
          int* ctab = reinterpret_cast<int*>(stg);  // [row tuple][32 columns]
          const int col0 = r.n0 + c;
          int ctc = 0, co0 = 0, co1 = 0;
          if (col0 + lane < P.N) {
            const int col = col0 + lane;
            ctc = col >= D.csplit ? 1 : 0;
            const int cin = ctc ? D.cin[1] : D.cin[0];
            const int cc = col - (ctc ? D.csplit : 0);
            const int j0 = cc / cin, j1 = cc - j0 * cin;
            co0 = ps_co(D, 0, 0, 2) * j0 + ps_co(D, 0, 0, 3) * j1;
            co1 = ps_co(D, 1, 0, 2) * j0 + ps_co(D, 1, 0, 3) * j1;
            if (ctc) {
              co0 = ps_co(D, 0, 1, 2) * j0 + ps_co(D, 0, 1, 3) * j1;
              co1 = ps_co(D, 1, 1, 2) * j0 + ps_co(D, 1, 1, 3) * j1;
            }
          }
          const unsigned tcmask = __ballot_sync(0xffffffffu, ctc);
          __syncwarp();  // the previous chunk's readers are done
          ctab[lane] = co0;
          ctab[32 + lane] = co1;
          __syncwarp();
          const int* mytab = ctab + (ps_tr ? 32 : 0);
          const int nvalid = P.N - col0;
          // rows past the problem store nothing; every store stays below the limit
          const unsigned lim = row0 + lane < P.M ? (unsigned)D.limit : 0u;
          // join the accumulators first (frees the correction's registers)
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float f = 0.f;
            if (ktiles > 0) {
              f = __uint_as_float(r0[j]);
              if (NPASS == 3) f += __uint_as_float(r1[j]);
            }
            r0[j] = __float_as_uint(f);
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j >= nvalid) break;  // warp-uniform
            uint32_t h, l;
            split_f32_tf32x3_fin(r0[j], h, l);
            const int o = ((tcmask >> j) & 1u ? ps_r1 : ps_r0) + mytab[j];
            if ((unsigned)o < lim) {
              hi[o] = h;
              lo[o] = l;
            }
          }
          continue;
        }
        if (psi >= 0) {
          // destination innermost along the columns: 16 columns of the 32
          // rows staged at a time (row i's columns rotated by (i / 2) % 16,
          // so that neither the row writes nor the column reads conflict);
          // each half-warp then stores 16 consecutive columns of one row
          const PsDesc& D = g.ps[psi];
          uint32_t* hi = static_cast<uint32_t*>(D.hi);
          uint32_t* lo = static_cast<uint32_t*>(D.lo);
          float* stf = reinterpret_cast<float*>(stg);         // 32 x 16
          int4* rinfo = reinterpret_cast<int4*>(stf + 512);  // per row: offsets for column tuples 0, 1; row tuple
          const int cl = lane & 15, hw = lane >> 4, sw = (lane >> 1) & 15;
          __syncwarp();  // the previous chunk's readers are done
          rinfo[lane] = make_int4(ps_r0, ps_r1, ps_tr, 0);
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              float f = 0.f;
              if (ktiles > 0) {
                f = __uint_as_float(r0[16 * hf + t]);
                if (NPASS == 3) f += __uint_as_float(r1[16 * hf + t]);
              }
              stf[lane * 16 + (t ^ sw)] = f;
            }
            __syncwarp();
            // this lane's column: tuple and offsets for row tuples 0 and 1
            const int col = r.n0 + c + 16 * hf + cl;
            const bool cok = col < P.N;
            const int tc = col >= D.csplit ? 1 : 0;
            const int cin = tc ? D.cin[1] : D.cin[0];
            const int cc = col - (tc ? D.csplit : 0);
            const int j0 = cc / cin, j1 = cc - j0 * cin;
            const int cp0 = (tc ? D.co[0][1][2] : D.co[0][0][2]) * j0 + (tc ? D.co[0][1][3] : D.co[0][0][3]) * j1;
            const int cp1 = (tc ? D.co[1][1][2] : D.co[1][0][2]) * j0 + (tc ? D.co[1][1][3] : D.co[1][0][3]) * j1;
#pragma unroll 2
            for (int st = 0; st < 16; ++st) {
              const int i = 2 * st + hw;
              const int4 ri = rinfo[i];
              const int o = (tc ? ri.y : ri.x) + (ri.z ? cp1 : cp0);
              uint32_t hh, ll;
              split_f32_tf32x3_fin(__float_as_uint(stf[i * 16 + (cl ^ ((i >> 1) & 15))]), hh, ll);
              if (cok && row0 + i < P.M && (unsigned)o < (unsigned)D.limit) {
                hi[o] = hh;
                lo[o] = ll;
              }
            }
            __syncwarp();
          }
          continue;
        }
        if (P.f32) {
          // FP32 output: the accumulator sums as they are, staged as above
          float* stf = reinterpret_cast<float*>(stg);
#pragma unroll
          for (int h = 0; h < 4; ++h) {
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
              float v[2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                float f = 0.f;
                if (ktiles > 0) {
                  f = __uint_as_float(r0[8 * h + j + u]);
                  if (NPASS == 3) f += __uint_as_float(r1[8 * h + j + u]);
                }
                v[u] = f;
              }
              *reinterpret_cast<float2*>(&stf[lane * 2 * K::STG_LD + j]) = make_float2(v[0], v[1]);
            }
            __syncwarp();
            const int col = r.n0 + c + 8 * h + 2 * (lane & 3);
#pragma unroll
            for (int i0 = 0; i0 < 32; i0 += 8) {
              const int i = i0 + (lane >> 2);
              const int row = row0 + i;
              if (row < P.M && col < P.N) {
                const float2 x = *reinterpret_cast<const float2*>(&stf[i * 2 * K::STG_LD + 2 * (lane & 3)]);
                float* dst = reinterpret_cast<float*>(P.c) + (long long)row * P.ldc + col;
                if (vec && col + 1 < P.N) {
                  *reinterpret_cast<float2*>(dst) = x;
                } else {
                  dst[0] = x.x;
                  if (col + 1 < P.N) dst[1] = x.y;
                }
              }
            }
            __syncwarp();
          }
          continue;
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          // this lane's row, 8 columns, widened to FP64 on the bit patterns;
          // the correction joins the main accumulator with one FP32 add
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            double v[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              uint32_t x = 0u;
              if (ktiles > 0) {
                float f = __uint_as_float(r0[8 * h + j + u]);
                if (NPASS == 3) f += __uint_as_float(r1[8 * h + j + u]);
                x = __float_as_uint(f);
              }
              unsigned long long w;
              if (!f32_widen_fast(x, w)) w = f64_bits((double)__uint_as_float(x));  // subnormal
              v[u] = f64_from_bits(w);
            }
            *reinterpret_cast<double2*>(&stg[lane * K::STG_LD + j]) = make_double2(v[0], v[1]);
          }
          __syncwarp();
          // four lanes per row, two columns each: eight rows per warp store
          const int col = r.n0 + c + 8 * h + 2 * (lane & 3);
#pragma unroll
          for (int i0 = 0; i0 < 32; i0 += 8) {
            const int i = i0 + (lane >> 2);
            const int row = row0 + i;
            if (row < P.M && col < P.N) {
              const double2 x = *reinterpret_cast<const double2*>(&stg[i * K::STG_LD + 2 * (lane & 3)]);
              double* dst = P.c + (long long)row * P.ldc + col;
              if (vec && col + 1 < P.N) {
                *reinterpret_cast<double2*>(dst) = x;
              } else {
                dst[0] = x.x;
                if (col + 1 < P.N) dst[1] = x.y;
              }
            }
          }
          __syncwarp();
        }
      }
      // this warp is done reading the accumulator buffer
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(K::TMEM_COLS)
                 : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D map over a row-major [rows, Kp] operand, box = 128 rows x 128 bytes.
bool make_map(CUtensorMap* m, const void* base, int rows, int Kp, int eb) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * eb};
  const cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / eb), (cuuint32_t)BM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(m, eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// make_map through a small per-thread cache: encoding a map is a driver call
// of a few microseconds, and the same operands recur every move. A map
// depends only on (base, rows, Kp, eb), the key, so an entry never goes stale.
bool make_map_cached(CUtensorMap* m, const void* base, int rows, int Kp, int eb) {
  struct Entry {
    const void* base;
    int rows, Kp, eb;
    CUtensorMap map;
  };
  constexpr int kEntries = 128;
  thread_local Entry cache[kEntries] = {};
  unsigned long long h = reinterpret_cast<unsigned long long>(base) >> 7;
  h = (h ^ (unsigned long long)rows * 0x9E3779B97F4A7C15ull ^ (unsigned long long)Kp * 0xC2B2AE3D27D4EB4Full ^
       (unsigned long long)eb) * 0x100000001B3ull;
  Entry& e = cache[(h >> 32) % kEntries];
  if (e.base == base && e.rows == rows && e.Kp == Kp && e.eb == eb && base != nullptr) {
    *m = e.map;
    return true;
  }
  if (!make_map(&e.map, base, rows, Kp, eb)) {
    e.base = nullptr;
    return false;
  }
  e.base = base;
  e.rows = rows;
  e.Kp = Kp;
  e.eb = eb;
  *m = e.map;
  return true;
}

// Split-K sums of every split problem of one launch (blockIdx.y = problem),
// partials added in split order (deterministic).
// The partials are FP32 (each is one FP32 accumulator's sum, so FP32 storage
// loses nothing and halves the epilogue's stores), rows padded to an even
// length ldp for 8-byte stores; they are summed in FP64.
struct SplitRed {
  const float* part;
  int nsplit, M, N, ldc, ldp;
  double* c;
  int f32;  // write FP32 (c read as float*)
};
struct SplitReds {
  SplitRed r[kMaxPairs];
};

__global__ void tc_splitk_reduce_kernel(const SplitReds reds) {
  hs_pdl_enter();
  const SplitRed& r = reds.r[blockIdx.y];
  const long long mn = (long long)r.M * r.N, stride = (long long)r.M * r.ldp;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mn;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / r.N, col = e - row * r.N;
    double v = 0.0;
    for (int s = 0; s < r.nsplit; ++s) {
      // widened on the bit pattern (the FP64 pipe, which a conversion would use, is GB300's scarce one)
      const uint32_t x = __float_as_uint(r.part[s * stride + row * r.ldp + col]);
      unsigned long long w;
      if (!f32_widen_fast(x, w)) w = f64_bits((double)__uint_as_float(x));  // subnormal
      v += f64_from_bits(w);
    }
    if (r.f32)
      reinterpret_cast<float*>(r.c)[row * r.ldc + col] = (float)v;
    else
      r.c[row * r.ldc + col] = v;
  }
}

// Launch with the tensor maps of the first NM operand pairs only: the maps
// are kernel parameters (512 bytes per pair), and a smaller parameter block
// launches faster.
template <int NPASS, int EB, int NM, bool PS>
cudaError_t launch_tc(const Maps& all, const Group& g, int grid, int tiles, int* err, cudaStream_t s) {
  using K = Cfg<NPASS, EB>;
  // set once per device and instantiation
  const cudaError_t attr_err =
      ensure_smem_attr(reinterpret_cast<const void*>(gemm_tc_kernel<NPASS, EB, NM, PS>), K::SMEM);
  if (attr_err != cudaSuccess) return attr_err;
  MapsN<NM> maps;
  for (int j = 0; j < NM; ++j)
    for (int h = 0; h < 2; ++h) {
      maps.a[j][h] = all.a[j][h];
      maps.b[j][h] = all.b[j][h];
    }
  hs_launch(gemm_tc_kernel<NPASS, EB, NM, PS>, grid, NT, K::SMEM, s, maps, g, tiles, err);
  return cudaGetLastError();
}

template <int NPASS, int EB>
cudaError_t run(const TcProblem* probs, int nprob, int* err, cudaStream_t s, double* part, long long part_elems) {
  using K = Cfg<NPASS, EB>;
  Maps maps;
  memset(&maps, 0, sizeof maps);
  Group g{};
  int tiles = 0, nmap = 0;
  SplitReds reds{};  // one reduction per split problem (at most one per operand pair)
  SplitRed* red = reds.r;
  int nred = 0;
  // split-K partials in FP32 (part holds part_elems doubles = 2 part_elems floats)
  float* partf = reinterpret_cast<float*>(part);
  const long long part_felems = 2 * part_elems;
  long long part_used = 0;
  const int sms = device_sms();
  for (int i = 0; i < nprob; ++i) {
    const TcProblem& p = probs[i];
    if (p.M <= 0 || p.N <= 0) continue;
    if (p.Kp <= 0 || p.Kp % K::K_PER_TILE != 0) return cudaErrorInvalidValue;
    const int j = nmap++;
    if (!make_map_cached(&maps.a[j][0], p.a_hi, p.M, p.Kp, EB) ||
        !make_map_cached(&maps.b[j][0], p.b_hi, p.N, p.Kp, EB))
      return cudaErrorInvalidValue;
    if (NPASS == 3 && (!make_map_cached(&maps.a[j][1], p.a_lo, p.M, p.Kp, EB) ||
                       !make_map_cached(&maps.b[j][1], p.b_lo, p.N, p.Kp, EB)))
      return cudaErrorInvalidValue;
    const int tiles_n = (p.N + BN - 1) / BN;
    const int ptiles = ((p.M + BM - 1) / BM) * tiles_n;
    const int ktiles = p.Kp / K::K_PER_TILE;
    int psi = -1;
    if (p.ps) {
      if (EB != 4 || p.ps->mode < 1 || p.ps->mode > 2) return cudaErrorInvalidValue;
      psi = j;
      g.ps[j] = *p.ps;
    }
    // split K when this problem's tiles cannot fill the SMs and each
    // split keeps at least 4 K steps; partials go to `part` (not for a
    // permuted split output). Up to 16 splits: a narrow product with a long
    // contraction (the subspace steps: M, N ~ 100, K ~ 2600) otherwise
    // streams its whole K through a handful of SMs
    int ns = 1;
    if (part && ptiles < sms && psi < 0) {
      ns = (sms + ptiles - 1) / ptiles;
      ns = ns < ktiles / 4 ? ns : ktiles / 4;
      ns = ns < 16 ? ns : 16;
      const long long need = (long long)ns * p.M * ((p.N + 1) & ~1);
      if (ns < 2 || part_used + need > part_felems || g.n + ns > kMaxUnits) ns = 1;
    }
    const int kper = (ktiles + ns - 1) / ns;
    ns = (ktiles + kper - 1) / kper;  // no empty K range
    for (int sidx = 0; sidx < ns; ++sidx) {
      const int kb = sidx * kper, ke = (kb + kper < ktiles) ? kb + kper : ktiles;
      if (g.n >= kMaxUnits) return cudaErrorInvalidValue;
      Prob& q = g.p[g.n++];
      q.M = p.M;
      q.N = p.N;
      q.k0 = kb * K::K_PER_TILE;
      q.Kp = (ke > kb ? ke - kb : 0) * K::K_PER_TILE;
      q.map = j;
      q.psi = psi;
      if (ns > 1) {
        const int ldp = (p.N + 1) & ~1;
        q.c = reinterpret_cast<double*>(partf + part_used + (long long)sidx * p.M * ldp);
        q.ldc = ldp;
        q.f32 = 1;
      } else {
        q.c = p.c;
        q.ldc = p.ldc;
        q.f32 = p.out_f32;
      }
      q.tiles_n = tiles_n;
      q.tile_start = tiles;
      tiles += ptiles;
    }
    if (ns > 1) {
      if (nred >= kMaxPairs) return cudaErrorInvalidValue;
      const int ldp = (p.N + 1) & ~1;
      red[nred++] = {partf + part_used, ns, p.M, p.N, p.ldc, ldp, p.c, p.out_f32};
      part_used += (long long)ns * p.M * ldp;
    }
  }
  if (tiles == 0) return cudaSuccess;
  const int grid = tiles < sms ? tiles : sms;
  // launches with a permuted split output take their own instantiation (the
  // split epilogue; at most two operand pairs), the others the plain one
  bool ps = false;
  for (int u = 0; u < g.n; ++u) ps = ps || g.p[u].psi >= 0;
  if (ps && (EB != 4 || nmap > 2)) return cudaErrorInvalidValue;
  cudaError_t e = ps           ? (nmap <= 1 ? launch_tc<NPASS, EB, 1, true>(maps, g, grid, tiles, err, s)
                                            : launch_tc<NPASS, EB, 2, true>(maps, g, grid, tiles, err, s))
                  : nmap <= 1 ? launch_tc<NPASS, EB, 1, false>(maps, g, grid, tiles, err, s)
                  : nmap <= 2 ? launch_tc<NPASS, EB, 2, false>(maps, g, grid, tiles, err, s)
                              : launch_tc<NPASS, EB, kMaxPairs, false>(maps, g, grid, tiles, err, s);
  if (e != cudaSuccess) return e;
  if (nred > 0) {
    long long mn = 0;
    for (int r = 0; r < nred; ++r) mn = std::max(mn, (long long)red[r].M * red[r].N);
    long long gx = (mn + 255) / 256;
    if (gx > 4096) gx = 4096;
    hs_launch(tc_splitk_reduce_kernel, dim3((unsigned)gx, (unsigned)nred), 256, 0, s, reds);
  }
  return cudaGetLastError();
}

// The GEMM kernel's bounded wait, run on barriers whose outcome is known:
// out[0..2] a wait (limit rounds) on a barrier nothing completes: the result
// (0), the recorded code (7) and the abort flag (1); out[3..4] a second wait
// with the abort flag raised: returns at once (0) and records nothing (0);
// out[5..6] a wait on a barrier completed by one arrival: 1 and nothing
// recorded. One thread; no copy or MMA is in flight.
__global__ void wait_selftest_kernel(long long limit, int* out) {
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int abort_flag, err[3];
  if (threadIdx.x != 0) return;
  abort_flag = 0;
  err[0] = err[1] = err[2] = 0;
  mbar_init(smem_u32(&bar[0]), 1);
  mbar_init(smem_u32(&bar[1]), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const bool w0 = mbar_wait_n(smem_u32(&bar[0]), 0, &abort_flag, &err[0], 7, limit);
  out[0] = w0;
  out[1] = err[0];
  out[2] = abort_flag;
  const bool w1 = mbar_wait_n(smem_u32(&bar[0]), 0, &abort_flag, &err[1], 9, limit);
  out[3] = w1;
  out[4] = err[1];
  abort_flag = 0;
  mbar_arrive(smem_u32(&bar[1]));
  const bool w2 = mbar_wait_n(smem_u32(&bar[1]), 0, &abort_flag, &err[2], 11, limit);
  out[5] = w2;
  out[6] = err[2];
}

}  // namespace

cudaError_t launch_wait_selftest(long long limit, int* out, cudaStream_t s) {
  if (limit < 1 || limit > WAIT_LIMIT) return cudaErrorInvalidValue;
  wait_selftest_kernel<<<1, 32, 0, s>>>(limit, out);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(int precision, const TcProblem* probs, int nprob, int* err, cudaStream_t s,
                           double* part, long long part_elems) {
  if (nprob > kMaxPairs) return cudaErrorInvalidValue;
  switch (precision) {
    case HS_PREC_TF32X3:
      return run<3, 4>(probs, nprob, err, s, part, part_elems);
    case HS_PREC_TF32:
      return run<1, 4>(probs, nprob, err, s, part, part_elems);
    case HS_PREC_BF16X3:
      return run<3, 2>(probs, nprob, err, s, part, part_elems);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace hs

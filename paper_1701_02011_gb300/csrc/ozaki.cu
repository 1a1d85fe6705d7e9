// Split-precision FP64 contraction on tcgen05 (see ozaki.cuh).
#include <cuda_bf16.h>

#include <cstdint>
#include <stdexcept>

#include "ozaki.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

namespace dsrg {
namespace {

// k per stage (a 32-byte row of bf16 digits), stage buffers, and stages per
// exact window: digits are balanced, |d| <= 64, so a level sum over one
// window has at most 8 pairs x 480 products of |d d'| <= 2^12,
// 8 x 480 x 4096 < 2^24, and is exact in FP32
constexpr int OZ_BM = 128, OZ_BK = 16, OZ_NBUF = 4, OZ_WIN = 30;
// fewest stages per k split
constexpr int OZ_SPLIT_MIN = 8;
// row tiles per rasterisation group
constexpr int OZ_GROUP = 8;
constexpr int OZ_THREADS = 256;  // 8 warps: lane quadrant (warp % 4) x column half (warp / 4)
constexpr int OZ_CTA_THREADS = OZ_THREADS + 32;  // and a ninth warp that issues the bulk copies
constexpr int OZ_TILE_ELEMS = OZ_BM * OZ_BK;  // A stage tile of one slice: 2048 bf16 = 4 KiB
constexpr int OZ_TILE_BYTES = OZ_TILE_ELEMS * 2;
// exponents are stored as 2048 + frexp exponent of the row / column maximum (0: all zero)
constexpr unsigned OZ_EBIAS = 2048;
// default budget of a bounded wait, and the fixed budget of the waits that
// drain copies and products in flight after a wait ran out (SM clock cycles,
// about 2 s at 2 GHz)
constexpr long long OZ_WAIT_CYCLES = 1LL << 32;

__device__ int g_oz_status;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major operand in the 32-byte swizzled
// layout (rows of 16 bf16, 8-row groups 256 bytes apart; the 16-byte chunk c
// of row r sits at chunk c ^ ((r >> 2) & 1)).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused when swizzled)
  d |= (uint64_t)(256 >> 4) << 32;           // stride byte offset: 8 rows x 32 B
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)6 << 61;                    // 32-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N columns (a multiple of 16, at most 256).
__host__ __device__ constexpr uint32_t oz_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// non-blocking test of the phase
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// bounded wait: false if the phase did not complete within `budget` SM clock
// cycles (tested once without blocking, then polled with try_wait)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, long long budget) {
  const long long t0 = clock64();
  while (true) {
    if (mbar_test(bar, phase)) return true;
    if (clock64() - t0 > budget) return false;
    if (mbar_try(bar, phase)) return true;
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// global -> shared bulk copy (bytes a multiple of 16, both addresses 16-byte
// aligned), completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define OZ_R32(a)                                                                                                   \
  "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]),      \
      "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(a[16]),        \
      "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]), "=r"(a[24]),       \
      "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]), "=r"(a[31])
#define OZ_W32(a)                                                                                                   \
  "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]),    \
      "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15]), "r"(a[16]), "r"(a[17]), "r"(a[18]),   \
      "r"(a[19]), "r"(a[20]), "r"(a[21]), "r"(a[22]), "r"(a[23]), "r"(a[24]), "r"(a[25]), "r"(a[26]), "r"(a[27]),   \
      "r"(a[28]), "r"(a[29]), "r"(a[30]), "r"(a[31])
#define OZ_P32                                                                                                      \
  "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, " \
  "%24, %25, %26, %27, %28, %29, %30, %31}"
#define OZ_Q32                                                                                                      \
  "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, "     \
  "%24, %25, %26, %27, %28, %29, %30, %31, %32}"

// 32 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 " OZ_P32 ", [%32];" : OZ_R32(r) : "r"(taddr) : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], " OZ_Q32 ";" ::"r"(taddr), OZ_W32(r) : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

struct OzArgs {
  const __nv_bfloat16* As;  // [S][MT][KT] tiles
  const __nv_bfloat16* Bs;  // [S][NT][KT] tiles
  const int* ea;            // [MT*128]
  const int* fb;            // [NT*128]
  int S, MT, NT, KT;
  long long M, N;
  double alpha;
  double* C;
  // C offsets: row m -> decoded with (nM, eM, cM), column n -> (nN, eN, cN)
  int nM, nN;
  int eM[4], eN[4];
  long long cM[4], cN[4];
  int rowfast;  // C's row index has the smaller stride (epilogue writes along rows)
  int* status;
  long long wait_cycles;  // budget of each bounded wait (clock cycles)
  // split over k tiles: CTA z covers [z*ktper, (z+1)*ktper) and writes its
  // scaled partial tile to part[z][MT*128][NT*BN] instead of C
  int splits, ktper;
  double* part;
};

__device__ __forceinline__ long long c_offset(long long lin, int nd, const int* ext, const long long* st) {
  long long o = 0;
  for (int d = nd - 1; d >= 0; --d) {
    long long q = lin / ext[d];
    o += (lin - q * ext[d]) * st[d];
    lin = q;
  }
  return o;
}

// paired FP32 arithmetic on two floats held in one 64-bit register
__device__ __forceinline__ uint64_t f2_pack(uint32_t a, uint32_t b) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, uint32_t& a, uint32_t& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(a), "=r"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// (double)f * 2^k assembled from the bit pattern of the float f (sign,
// re-biased exponent, mantissa) with integer instructions; zero gives zero and
// subnormal, non-finite or out-of-range cases take the library path.
__device__ __forceinline__ double f32_to_f64_scaled(uint32_t u, int k) {
  if ((u << 1) == 0) return 0.0;
  const uint32_t ex = (u >> 23) & 0xFFu;
  const int e = (int)ex - 127 + 1023 + k;
  if (ex == 0 || ex == 255 || e <= 0 || e >= 2047) return ldexp((double)__uint_as_float(u), k);
  const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)e << 52) |
                                  ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// barrier 1 over the 8 warps of the tile (the copy warp does not take part);
// the _and form returns whether every thread's pred was true
__device__ __forceinline__ void tile_sync() { asm volatile("bar.sync 1, %0;" ::"n"(OZ_THREADS) : "memory"); }
__device__ __forceinline__ bool tile_sync_and(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(OZ_THREADS)
      : "memory");
  return r != 0;
}

// Thread 0: every digit pair (t, u), t + u <= S + 1, of one stage into the
// accumulator of level t + u.  For a fixed A slice t the levels
// t + 1 .. S + 1 are adjacent in TMEM and the B slices 1 .. S + 1 - t adjacent
// in shared memory, so one MMA of N = BN (S + 1 - t) columns (pieces of at
// most 256) covers them and reads A_t once.  The first stage of a window
// overwrites: the t = 1 MMAs cover every level.  descA0 / descB0 describe
// the first A / B tile of buffer 0; boff is the buffer's byte offset (the
// descriptors differ only in the start-address field, bytes / 16).
template <int BN, int S>
__device__ __forceinline__ void oz_issue_stage(uint32_t tm, uint64_t descA0, uint64_t descB0, uint32_t boff,
                                               bool fresh) {
  constexpr int B_TILE_BYTES = BN * OZ_BK * 2;
  constexpr int UMAX = 256 / BN;
  const uint64_t dA = descA0 + (boff >> 4), dB = descB0 + (boff >> 4);
#pragma unroll
  for (int t = 1; t <= S; ++t) {
#pragma unroll
    for (int u0 = 1; u0 <= S + 1 - t; u0 += UMAX) {
      const int nu = (S + 1 - t) - u0 + 1 < UMAX ? (S + 1 - t) - u0 + 1 : UMAX;
      mma_bf16(tm + (uint32_t)((t + u0 - 2) * BN), dA + (uint64_t)(((t - 1) * OZ_TILE_BYTES) >> 4),
               dB + (uint64_t)(((u0 - 1) * B_TILE_BYTES) >> 4), oz_idesc(nu * BN), (fresh && t == 1) ? 0u : 1u);
    }
  }
}

// One CTA: a 128 x BN tile of C.  Warps 0-7: warp w reads TMEM lanes
// 32 (w % 4) .. and column half w / 4; its thread 0 issues the MMAs.  Warp 8
// (lane 0) issues the bulk copies.  The k range is walked in stages of 16;
// four shared-memory buffers rotate: the copy warp refills a buffer as soon
// as the MMAs of the stage that used it have completed, so copies run up to
// three stages ahead of the tensor cores, and the MMA thread only waits for
// data.  Every level c = t + u has its own TMEM accumulator (S levels x BN
// columns); after every OZ_WIN stages (an exact window) warps 0-7 fold the
// level sums, scaled by 2^(-7c), into float-float (hi, lo) running sums held
// in registers.
template <int BN>
__global__ void __launch_bounds__(OZ_CTA_THREADS, 1) k_ozaki_mma(const OzArgs a) {
  constexpr uint32_t TMEM_COLS = 512;  // S <= 8 level accumulators of BN <= 64 columns
  constexpr int B_TILE_BYTES = BN * OZ_BK * 2;
  // columns per warp in the fold and epilogue: two column halves for BN >= 64;
  // for BN = 32 the second half of the warps sits out
  constexpr int HALF = BN >= 64 ? BN / 2 : BN;
  constexpr int NCH = HALF / 32;
  static_assert(8 * BN <= (int)TMEM_COLS, "TMEM columns");
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_load[OZ_NBUF], bar_mma[OZ_NBUF], bar_win;
  __shared__ uint32_t tmem_base;
  __shared__ long long colC[BN], rowC[OZ_BM];
  __shared__ int colE[BN];
  __shared__ int issued[OZ_NBUF];  // copies issued per buffer (copy warp), read at the end
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool copier = warp == OZ_THREADS / 32;
  const int quad = warp & 3, half = (warp >> 2) & 1;  // TMEM lanes 32*quad.., columns half*HALF..
  const int row = quad * 32 + (tid & 31);
  // grouped rasterisation: consecutive CTAs walk the column tiles of a group
  // of OZ_GROUP row tiles, so the CTAs running together share their A and B
  // digit tiles in L2
  int mt, nt;
  {
    const int lin = blockIdx.y * a.MT + blockIdx.x;
    const int per = OZ_GROUP * a.NT;
    const int first = (lin / per) * OZ_GROUP;
    const int gm = a.MT - first < OZ_GROUP ? a.MT - first : OZ_GROUP;
    const int within = lin - (lin / per) * per;
    mt = first + within % gm;
    nt = within / gm;
  }
  const int z = blockIdx.z;
  const int kt0 = a.splits > 1 ? z * a.ktper : 0;
  const int kt1 = a.splits > 1 ? (kt0 + a.ktper < a.KT ? kt0 + a.ktper : a.KT) : a.KT;
  const int S = a.S;
  const size_t stage_bytes = (size_t)S * (OZ_TILE_BYTES + B_TILE_BYTES);
  const int ns = kt1 - kt0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < OZ_NBUF; ++i) {
      mbar_init(&bar_load[i], 1);
      mbar_init(&bar_mma[i], 1);
      issued[i] = 0;
    }
    mbar_init(&bar_win, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int t = tid; t < BN; t += OZ_CTA_THREADS) {
    long long n = (long long)nt * BN + t;
    colC[t] = n < a.N ? c_offset(n, a.nN, a.eN, a.cN) : -1;
    colE[t] = a.fb[(long long)nt * BN + t] - (int)OZ_EBIAS;
  }
  for (int t = tid; t < OZ_BM; t += OZ_CTA_THREADS) {
    long long m = (long long)mt * OZ_BM + t;
    rowC[t] = m < a.M ? c_offset(m, a.nM, a.eM, a.cM) : -1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tmem_base;
  // matrix descriptors of the first A and B digit tiles of buffer 0; the
  // others differ only in the start-address field (byte offset / 16)
  const uint64_t descA0 = sdesc(smem_u32(smem));
  const uint64_t descB0 = sdesc(smem_u32(smem + (size_t)S * OZ_TILE_BYTES));

  // ---- copy warp: stage k (relative to kt0) into buffer k % OZ_NBUF, once
  // the MMAs of stage k - OZ_NBUF (the buffer's last use) have completed
  if (copier) {
    if ((tid & 31) == 0) {
      uint32_t ph_mma[OZ_NBUF] = {};
      for (int k = 0; k < ns; ++k) {
        const int b = k % OZ_NBUF, kt = kt0 + k;
        if (k >= OZ_NBUF) {
          if (!mbar_wait(&bar_mma[b], ph_mma[b], a.wait_cycles)) break;  // the MMA thread stopped
          ph_mma[b] ^= 1;
        }
        unsigned char* base = smem + (size_t)b * stage_bytes;
        mbar_expect_tx(&bar_load[b], (uint32_t)(S * (OZ_TILE_BYTES + B_TILE_BYTES)));
        for (int s2 = 0; s2 < S; ++s2) {
          bulk_g2s(base + (size_t)s2 * OZ_TILE_BYTES, a.As + ((size_t)(s2 * a.MT + mt) * a.KT + kt) * OZ_TILE_ELEMS,
                   OZ_TILE_BYTES, &bar_load[b]);
          bulk_g2s(base + (size_t)S * OZ_TILE_BYTES + (size_t)s2 * B_TILE_BYTES,
                   a.Bs + ((size_t)(s2 * a.NT + nt) * a.KT + kt) * (BN * OZ_BK), B_TILE_BYTES, &bar_load[b]);
        }
        issued[b] += 1;
      }
    }
  }

  // ---- warps 0-7: MMAs (thread 0), folds, epilogue
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  const uint32_t col0 = (uint32_t)(half * HALF);
  const bool active = !copier && (BN >= 64 || half == 0);
  uint32_t rhi[NCH][32], rlo[NCH][32];
#pragma unroll
  for (int j = 0; j < NCH; ++j)
#pragma unroll
    for (int q = 0; q < 32; ++q) rhi[j][q] = rlo[j][q] = 0u;
  bool ok = true;
  int consumed[OZ_NBUF] = {};                  // thread 0: loads waited for per buffer
  uint32_t ph_load[OZ_NBUF] = {}, ph_win = 0;  // thread 0 / every tile thread
  bool win_pending = false;                    // thread 0
  if (!copier) {
    for (int k = 0; k < ns; ++k) {
      const int b = k % OZ_NBUF;
      const bool fresh = (k % OZ_WIN) == 0;
      const bool wend = (k % OZ_WIN) == OZ_WIN - 1 || k == ns - 1;
      if (tid == 0) {
        if (ok) {
          if (mbar_wait(&bar_load[b], ph_load[b], a.wait_cycles)) {
            ph_load[b] ^= 1;
            consumed[b] += 1;
          } else {
            ok = false;
          }
        }
        if (ok) {
          tc_fence_after();
          switch (S) {
            case 1: oz_issue_stage<BN, 1>(tm, descA0, descB0, (uint32_t)(b * stage_bytes), fresh); break;
            case 2: oz_issue_stage<BN, 2>(tm, descA0, descB0, (uint32_t)(b * stage_bytes), fresh); break;
            case 3: oz_issue_stage<BN, 3>(tm, descA0, descB0, (uint32_t)(b * stage_bytes), fresh); break;
            case 4: oz_issue_stage<BN, 4>(tm, descA0, descB0, (uint32_t)(b * stage_bytes), fresh); break;
            case 5: oz_issue_stage<BN, 5>(tm, descA0, descB0, (uint32_t)(b * stage_bytes), fresh); break;
            case 6: oz_issue_stage<BN, 6>(tm, descA0, descB0, (uint32_t)(b * stage_bytes), fresh); break;
            case 7: oz_issue_stage<BN, 7>(tm, descA0, descB0, (uint32_t)(b * stage_bytes), fresh); break;
            default: oz_issue_stage<BN, 8>(tm, descA0, descB0, (uint32_t)(b * stage_bytes), fresh); break;
          }
          mma_commit(&bar_mma[b]);  // the buffer is free once these complete
        }
        if (wend) {  // completes once every MMA issued so far has completed
          mma_commit(&bar_win);
          win_pending = true;
        }
      }
      if (!wend) continue;
      const bool w = mbar_wait(&bar_win, ph_win, a.wait_cycles);
      if (w) ph_win ^= 1;
      if (tid == 0 && w) win_pending = false;
      ok = tile_sync_and(ok && w);
      tc_fence_after();
      if (!ok) break;
      // fold the window: (hi, lo) += acc_c * 2^(-7c), two-sum in paired FP32
      if (active) {
        for (int c = 2; c <= S + 1; ++c) {
          const float scale = exp2f(-7.0f * (float)c);
          const uint64_t sc2 = f2_pack(__float_as_uint(scale), __float_as_uint(scale));
#pragma unroll
          for (int j = 0; j < NCH; ++j) {
            uint32_t acc[32];
            tmem_ld32(tm + lane_off + (uint32_t)((c - 2) * BN) + col0 + 32 * j, acc);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 32; q += 2) {
              const uint64_t x = f2_mul(f2_pack(acc[q], acc[q + 1]), sc2);
              const uint64_t h = f2_pack(rhi[j][q], rhi[j][q + 1]);
              const uint64_t s_ = f2_add(h, x);
              const uint64_t bp = f2_sub(s_, h);
              const uint64_t err = f2_add(f2_sub(h, f2_sub(s_, bp)), f2_sub(x, bp));
              uint64_t l = f2_add(f2_pack(rlo[j][q], rlo[j][q + 1]), err);
              const uint64_t s2 = f2_add(s_, l);
              l = f2_sub(l, f2_sub(s2, s_));
              f2_unpack(s2, rhi[j][q], rhi[j][q + 1]);
              f2_unpack(l, rlo[j][q], rlo[j][q + 1]);
            }
          }
        }
      }
      // the accumulators are read; the next window may overwrite them
      tc_fence_before();
      tile_sync();
      tc_fence_after();
    }
  }
  // every warp: the copy warp's count of issued copies is visible after this
  __syncthreads();
  // after a timed-out wait: wait once more (the fixed default budget) for
  // copies issued but not consumed and for every MMA issued, before the
  // shared memory and TMEM are released
  if (!ok && tid == 0) {
    for (int i = 0; i < OZ_NBUF; ++i)
      if (issued[i] > consumed[i]) mbar_wait(&bar_load[i], ph_load[i], OZ_WAIT_CYCLES);
    if (win_pending) mbar_wait(&bar_win, ph_win, OZ_WAIT_CYCLES);
  }
  // epilogue: the scaled tile 2^(ea[m] + fb[n]) (hi + lo) goes to shared
  // memory (the stage buffers are free once the last MMA has completed and
  // every copy was consumed; rows padded by one double against bank
  // conflicts), then consecutive threads write consecutive columns of C
  // (alpha times, accumulated) or of the split-k partial part[z]
  constexpr int LDT = BN + 1;
  double* stile = reinterpret_cast<double*>(smem);
  if (ok && active) {
    const int em = a.ea[(long long)mt * OZ_BM + row] - (int)OZ_EBIAS;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int cc = (int)col0 + 32 * j;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int k = em + colE[cc + q] + 2;  // x = 2^(e + 1) sum_t d_t 2^(-7t) on both sides
        stile[row * LDT + cc + q] = f32_to_f64_scaled(rhi[j][q], k) + f32_to_f64_scaled(rlo[j][q], k);
      }
    }
  }
  __syncthreads();
  if (ok && !copier) {
    if (a.splits > 1) {
      const long long ldp = (long long)a.NT * BN;
      double* pz = a.part + ((long long)z * a.MT * OZ_BM + (long long)mt * OZ_BM) * ldp + (long long)nt * BN;
      for (int i = tid; i < OZ_BM * BN; i += OZ_THREADS) {
        const int r = i / BN, c = i - r * BN;
        const bool live = (long long)mt * OZ_BM + r < a.M && colC[c] >= 0;
        pz[(long long)r * ldp + c] = live ? stile[r * LDT + c] : 0.0;
      }
    } else {
      // eight read-modify-writes per thread with all loads issued first;
      // consecutive threads on C's contiguous index (rows when rowfast)
      constexpr int U = 8;
      static_assert((OZ_BM * BN) % (U * OZ_THREADS) == 0, "epilogue tiling");
      for (int base = 0; base < OZ_BM * BN; base += U * OZ_THREADS) {
        long long off[U];
        double cv[U], tv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = base + u * OZ_THREADS + tid;
          int r, c;
          if (a.rowfast) {
            c = i / OZ_BM;
            r = i - c * OZ_BM;
          } else {
            r = i / BN;
            c = i - r * BN;
          }
          const long long oc = colC[c], orow = rowC[r];
          off[u] = oc >= 0 && orow >= 0 ? orow + oc : -1;
          tv[u] = stile[r * LDT + c];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) cv[u] = off[u] >= 0 ? a.C[off[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (off[u] >= 0) a.C[off[u]] = cv[u] + a.alpha * tv[u];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TMEM_COLS)
                              : "memory");
  if (!ok && tid == 0) atomicExch(a.status ? a.status : &g_oz_status, 1);
}

// C[m, n] += alpha * sum_z part[z][m][n] (z in order)
template <int BN>
__global__ void k_ozaki_reduce(const OzArgs a) {
  const long long Mp = (long long)a.MT * OZ_BM, ldp = (long long)a.NT * BN;
  const long long total = a.M * a.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long m = i / a.N, n = i - m * a.N;
    double s = 0.0;
    for (int z = 0; z < a.splits; ++z) s += a.part[((long long)z * Mp + m) * ldp + n];
    a.C[c_offset(m, a.nM, a.eM, a.cM) + c_offset(n, a.nN, a.eN, a.cN)] += a.alpha * s;
  }
}

// The same sum with one warp per output element, for many splits over few
// outputs (one thread would chain hundreds of dependent loads): lane l adds
// z = l, l + 32, ... in order, then a fixed shuffle tree combines the lanes.
template <int BN>
__global__ void k_ozaki_reduce_warp(const OzArgs a) {
  const long long Mp = (long long)a.MT * OZ_BM, ldp = (long long)a.NT * BN;
  const long long total = a.M * a.N;
  const int lane = threadIdx.x & 31;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = wid; i < total; i += nw) {
    const long long m = i / a.N, n = i - m * a.N;
    double s = 0.0;
    for (int z = lane; z < a.splits; z += 32) s += a.part[((long long)z * Mp + m) * ldp + n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) a.C[c_offset(m, a.nM, a.eM, a.cM) + c_offset(n, a.nN, a.eN, a.cN)] += a.alpha * s;
  }
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------
struct OzPack {
  const double* src;
  int nR, nK;
  int eR[4], eK[4];
  long long sR[4], sK[4];
  long long R, K;      // logical sizes (both < 2^31)
  int T, KT;           // tiles along rows (TR each) and k (64 each)
  int TR;              // rows per tile: 128 (A) or BN (B)
  int S;
  int vec;             // 1: every full 8-group is 64 contiguous, 16-byte aligned bytes
  FastDiv fR[4], fK[4];  // divisors of eR, eK
};

// whether pack_load8 may read a full k group with 16-byte loads: unit
// innermost k stride, groups that never cross a carry of the k multi-index
// (innermost extent a multiple of 8), every other stride even and the base
// 16-byte aligned, so every group starts on a 16-byte boundary
inline int pack_vec_ok(const OzPack& p) {
  if (p.nK < 1 || p.sK[p.nK - 1] != 1 || p.eK[p.nK - 1] % 8 != 0) return 0;
  if (reinterpret_cast<uintptr_t>(p.src) % 16 != 0) return 0;
  for (int d = 0; d < p.nK - 1; ++d)
    if (p.sK[d] % 2 != 0) return 0;
  for (int d = 0; d < p.nR; ++d)
    if (p.sR[d] % 2 != 0) return 0;
  return 1;
}

// Operand preparation runs in two passes over the padded operand viewed as
// rows x (8-element k groups).  Work item i is one (row r, group q); when the
// source's innermost k index is contiguous the groups of a row are adjacent
// items (reads coalesce along k), otherwise the rows are (reads coalesce along
// the row index).
//   pass 1: eu[r] = 2048 + max over k of the binary exponent ex with
//           |x| < 2^ex (frexp), 0 for an all-zero row (eu zeroed beforehand);
//   pass 2: the S balanced 7-bit digits of x 2^(-e) go to the swizzled tiles,
//           eight bf16 (16 bytes) per store.
constexpr int PACK_T = 256;

// Everything below works on the bit patterns with integer instructions: the
// FP64 pipe of this SM is narrow, and even a comparison with 0.0 runs there.
__device__ __forceinline__ unsigned exp_code(long long bits) {
  if ((bits << 1) == 0) return 0u;  // +-0
  const int be = (int)((bits >> 52) & 0x7FF);
  return (unsigned)((be ? be - 1022 : -1022) + (int)OZ_EBIAS);
}

// work item i -> (row r, group q); i, Rpad, Q < 2^32
__device__ __forceinline__ void pack_item(unsigned i, const FastDiv& fQ, const FastDiv& fR, bool kfast, unsigned& r,
                                          unsigned& q) {
  if (kfast) {
    r = fast_div(i, fQ);
    q = i - r * fQ.d;
  } else {
    q = fast_div(i, fR);
    r = i - q * fR.d;
  }
}

// bit patterns of the (up to) 8 source values of group q of row r; zero
// outside R x K
__device__ __forceinline__ void pack_load8(const OzPack& p, unsigned r, unsigned q, long long x[8]) {
  const unsigned k0 = q * 8u;
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 0;
  if (r >= (unsigned long long)p.R || k0 >= (unsigned long long)p.K) return;
  const long long* src = reinterpret_cast<const long long*>(p.src);
  long long roff = 0;
  {
    unsigned lin = r;
    for (int d = p.nR - 1; d >= 0; --d) {
      const unsigned qd = fast_div(lin, p.fR[d]);
      roff += (long long)(lin - qd * p.fR[d].d) * p.sR[d];
      lin = qd;
    }
  }
  // multi-index of k0, then step through the next 7 with carries
  int idx[4];
  long long off = 0;
  {
    unsigned lin = k0;
    for (int d = p.nK - 1; d >= 0; --d) {
      const unsigned qd = fast_div(lin, p.fK[d]);
      idx[d] = (int)(lin - qd * p.fK[d].d);
      off += (long long)idx[d] * p.sK[d];
      lin = qd;
    }
  }
  if (p.vec && k0 + 8 <= (unsigned long long)p.K) {
    const longlong2* v = reinterpret_cast<const longlong2*>(src + roff + off);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const longlong2 t = v[h];
      x[2 * h] = t.x;
      x[2 * h + 1] = t.y;
    }
    return;
  }
  const int last = p.nK - 1;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (k0 + j >= (unsigned long long)p.K) break;
    x[j] = src[roff + off];
    if (j == 7) break;
    int d = last;
    ++idx[d];
    off += p.sK[d];
    while (idx[d] == p.eK[d] && d > 0) {
      off -= (long long)p.eK[d] * p.sK[d];
      idx[d] = 0;
      --d;
      ++idx[d];
      off += p.sK[d];
    }
  }
}

// Both operands of a product in one launch: blockIdx.y selects A (0) or B (1).
struct PackPass {
  OzPack p[2];
  unsigned* eu[2];
  __nv_bfloat16* dst[2];
  int kfast[2];
  FastDiv fQ[2], fR[2];
  unsigned W[2];
};

// Each CTA walks one contiguous range of work items, 256 at a time, and each
// thread keeps the maximum of its current row in a register, flushed by an
// atomic max when its row changes and at the end: a few long rows (a short
// side of 8 or 38) would otherwise send millions of atomics to a few words.
__global__ void __launch_bounds__(PACK_T) k_ozaki_rowexp(const PackPass pp) {
  const int o = blockIdx.y;
  const OzPack& p = pp.p[o];
  unsigned* eu = pp.eu[o];
  const int kfast = pp.kfast[o];
  const FastDiv fQ = pp.fQ[o], fR = pp.fR[o];
  const unsigned W = pp.W[o];
  const unsigned long long span = (unsigned long long)gridDim.x * PACK_T;
  const unsigned long long per = (W + span - 1) / span * PACK_T;  // items per CTA
  const unsigned long long lo = blockIdx.x * per;
  const unsigned long long hi = lo + per < W ? lo + per : W;
  long long held = -1;  // row whose maximum is in hv
  unsigned hv = 0;
  for (unsigned long long base = lo; base < hi; base += PACK_T) {
    if (base + threadIdx.x >= hi) break;
    const unsigned i = (unsigned)(base + threadIdx.x);
    unsigned rr, q;
    pack_item(i, fQ, fR, kfast != 0, rr, q);
    if (rr >= (unsigned long long)p.R) continue;
    long long x[8];
    pack_load8(p, rr, q, x);
    unsigned v = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const unsigned c = exp_code(x[j]);
      v = c > v ? c : v;
    }
    if ((long long)rr != held) {
      if (held >= 0 && hv) atomicMax(eu + held, hv);
      held = rr;
      hv = 0;
    }
    hv = v > hv ? v : hv;
  }
  // final flush: one atomic per warp when every lane holds the same row
  const long long r0 = __shfl_sync(0xffffffffu, held, 0);
  if (__all_sync(0xffffffffu, held == r0)) {
    const unsigned m = __reduce_max_sync(0xffffffffu, hv);
    if ((threadIdx.x & 31) == 0 && r0 >= 0 && m) atomicMax(eu + r0, m);
  } else if (held >= 0 && hv) {
    atomicMax(eu + held, hv);
  }
}

// S balanced base-128 digits of each element: V = round(x 2^(7S - 1 - e)),
// |V| <= 2^(7S - 1) (|x| < 2^e, e the row / column exponent), written as
// V = sum_t d_t 128^(S - t) with |d_t| <= 64, so x = 2^(e + 1) sum_t d_t 2^(-7t);
// the digits are extracted from the lowest up with balanced remainders and
// stored as bf16 (exact: |d| <= 64).  One call: group q of row r, S 16-byte
// stores (one per slice tile).
template <int S>
__device__ __forceinline__ void digits_item(const OzPack& p, const unsigned* eu, __nv_bfloat16* dst, unsigned r,
                                            unsigned q) {
  const long long tile_elems = (long long)p.TR * OZ_BK;
  constexpr int F = 7 * S - 1;
  long long x[8];
  pack_load8(p, r, q, x);
  const int e = r < (unsigned long long)p.R ? (int)eu[r] - (int)OZ_EBIAS : 0;
  int dg[S][8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    long long V = 0;
    const long long bits = x[j];
    if ((bits << 1) != 0) {
      const int be = (int)((bits >> 52) & 0x7FF);
      unsigned long long m = (unsigned long long)(bits & ((1LL << 52) - 1));
      int E;
      if (be) {
        m |= 1ULL << 52;
        E = be - 1075;
      } else {
        E = -1074;
      }
      const int sh_ = E + F - e;  // |x| 2^(F - e) = m 2^sh < 2^F
      unsigned long long v;
      if (sh_ >= 0) v = sh_ < 12 ? (m << sh_) : 0;
      else if (-sh_ >= 64) v = 0;
      else v = (m >> (-sh_)) + ((m >> (-sh_ - 1)) & 1ULL);  // to nearest, ties away from zero
      V = bits < 0 ? -(long long)v : (long long)v;
    }
    // V = hi 2^28 + lo, 0 <= lo < 2^28: a digit depends only on the running
    // value mod 128, so the (at most) four lowest digits come from lo in
    // 32-bit arithmetic (lo - d >= 0 stays exact), then the carry joins the
    // upper part for the rest
    constexpr int NL = S - 1 < 4 ? S - 1 : 4;
    int lo = (int)(V & 0xFFFFFFFLL), hi = (int)(V >> 28);
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int d = ((lo + 64) & 127) - 64;
      dg[S - 1 - k][j] = d;
      lo = (lo - d) >> 7;
    }
    hi = lo + hi * (1 << (28 - 7 * NL));
#pragma unroll
    for (int k = NL; k < S - 1; ++k) {
      const int d = ((hi + 64) & 127) - 64;
      dg[S - 1 - k][j] = d;
      hi = (hi - d) >> 7;
    }
    dg[0][j] = hi;  // |hi| <= 64 here
  }
  const unsigned tr = r / p.TR, rr = r - tr * p.TR;  // TR is 32, 64 or 128
  const int tk = (int)(q >> 1), chunk = (int)(q & 1);   // two 8-element chunks per 16-k row
  const long long within = (long long)rr * OZ_BK + ((chunk ^ ((rr >> 2) & 1)) << 3);
#pragma unroll
  for (int t = 1; t <= S; ++t) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      // |d| <= 64: exact in float and in bf16, so the conversion is exact
      const __nv_bfloat162 b2 = __floats2bfloat162_rn((float)dg[t - 1][2 * h], (float)dg[t - 1][2 * h + 1]);
      w[h] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    const long long tile = ((long long)(t - 1) * p.T + tr) * p.KT + tk;
    *reinterpret_cast<uint4*>(dst + tile * tile_elems + within) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// A 16-k row of a digit tile is 32 bytes, one DRAM sector, filled by its two
// 8-element groups, and the two halves are written by neighbouring lanes:
// along k the groups of a row are consecutive items anyway; along rows item
// i takes row (i / 2) mod rows and group 2 ((i / 2) / rows) + i mod 2.  (With
// rows alone along the lanes, the second half of every sector followed a
// whole pass over the rows later, after the sector had left L2: each
// half-sector write then cost a read-modify-write in DRAM, and the digit pass
// moved 2-4x its bytes.)
template <int S>
__global__ void __launch_bounds__(PACK_T) k_ozaki_digits(const PackPass pp) {
  const int o = blockIdx.y;
  const OzPack& p = pp.p[o];
  const unsigned* eu = pp.eu[o];
  __nv_bfloat16* dst = pp.dst[o];
  const int kfast = pp.kfast[o];
  const FastDiv fQ = pp.fQ[o], fR = pp.fR[o];
  const unsigned W = pp.W[o];
  const unsigned stride = gridDim.x * PACK_T;
  for (unsigned i = blockIdx.x * PACK_T + threadIdx.x; i < W; i += stride) {
    unsigned r, q;
    if (kfast) {
      pack_item(i, fQ, fR, true, r, q);
    } else {
      const unsigned j = i >> 1, tk = fast_div(j, fR);
      r = j - tk * fR.d;
      q = 2u * tk + (i & 1u);
    }
    digits_item<S>(p, eu, dst, r, q);
  }
}

inline int oz_pack_grid(long long n) {
  long long b = (n + PACK_T - 1) / PACK_T;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

// rows or k along the coalesced direction of the source (see the pack kernels)
inline int pack_kfast(const OzPack& p) {
  if (p.nK > 0 && p.sK[p.nK - 1] == 1) return 1;
  if (p.nR > 0 && p.sR[p.nR - 1] == 1) return 0;
  return 1;
}

inline int oz_grid(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

size_t oz_smem_bytes(int S, int BN) {
  const size_t tiles = OZ_NBUF * ((size_t)S * OZ_TILE_BYTES + (size_t)S * BN * OZ_BK * 2);  // stage buffers
  const size_t stage = (size_t)OZ_BM * (BN + 1) * sizeof(double);  // epilogue tile
  return (tiles > stage ? tiles : stage) + 1024;
}

// the largest dynamic shared memory any launch of k_ozaki_mma<BN> asks for,
// set once per device (kept out of the launch path, which may be captured)
template <int BN>
void oz_smem_attribute() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  check_cuda(cudaFuncSetAttribute(k_ozaki_mma<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 4096),
             "cudaFuncSetAttribute (ozaki)");
  done[dev] = true;
}

template <int BN>
void oz_launch_bn(const OzArgs& a, int MT, int NT, cudaStream_t st) {
  // at least 120 KiB so that one CTA (one TMEM allocation) occupies an SM
  size_t smem = oz_smem_bytes(a.S, BN);
  if (smem < 120 * 1024) smem = 120 * 1024;
  oz_smem_attribute<BN>();
  k_ozaki_mma<BN><<<dim3(MT, NT, a.splits > 1 ? a.splits : 1), OZ_CTA_THREADS, smem, st>>>(a);
  if (a.splits > 1) {
    // few outputs, many splits: a warp per output keeps loads in flight
    if (a.splits >= 32 && a.M * a.N < 152LL * 256)
      k_ozaki_reduce_warp<BN><<<oz_grid(a.M * a.N * 32), 256, 0, st>>>(a);
    else
      k_ozaki_reduce<BN><<<oz_grid(a.M * a.N), 256, 0, st>>>(a);
  }
}

void oz_launch_mma(const OzArgs& a, int MT, int NT, int BN, cudaStream_t st) {
  if (BN == 32) oz_launch_bn<32>(a, MT, NT, st);
  else oz_launch_bn<64>(a, MT, NT, st);
}
}  // namespace

const void* g_oz_status_alias() { return (const void*)&g_oz_status; }

int ozaki_status(cudaStream_t st, const int* flag) {
  int v = 0;
  if (flag)
    check_cuda(cudaMemcpyAsync(&v, flag, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
  else
    check_cuda(cudaMemcpyFromSymbolAsync(&v, g_oz_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st), "status");
  check_cuda(cudaStreamSynchronize(st), "sync");
  return v;
}

bool ozaki_supported(const GemmArgs& g) {
  // packing indexes (padded rows) x (8-element k groups) with 32 bits
  const long long big = g.M > g.N ? g.M : g.N;
  const long long rows = (big + OZ_BM - 1) / OZ_BM * OZ_BM, groups = (g.K + OZ_BK - 1) / OZ_BK * (OZ_BK / 8);
  return g.M < (1LL << 31) && g.N < (1LL << 31) && g.K < (1LL << 31) && rows * groups < (1LL << 32);
}

namespace {
// tile width (0: the rule below) and k-split mode (0: rule, 1: none, 2: twice the rule)
struct OzChoice {
  int bn = 0;
  int split_mode = 0;
};

void ozaki_run(Workspace& ws, const GemmArgs& g0, int S, int kind, const OzChoice& ch) {
  if (g0.M <= 0 || g0.N <= 0 || g0.K <= 0) return;
  if (g0.nbatch != 1) throw std::runtime_error("split-precision contraction needs nbatch == 1");
  if (S < 1 || S > kOzakiMaxSlices) throw std::runtime_error("split-precision slices must be 1..8");
  if (!ozaki_supported(g0)) throw std::runtime_error("split-precision contraction too large for 32-bit packing");
  // orient so that the longer output side runs along the 128-row A tiles:
  // C^T = B^T A^T just exchanges the roles of the operands
  const bool swap = g0.N > g0.M;
  OzPack pa{}, pb{};
  OzArgs a{};
  auto fill = [&](OzPack& p, const double* src, int nR, const int* eR, const long long* sR) {
    p.src = src;
    p.nR = nR;
    p.nK = g0.nK;
    for (int d = 0; d < 4; ++d) {
      p.eR[d] = eR[d];
      p.sR[d] = sR[d];
      p.eK[d] = g0.eK[d];
    }
    p.K = g0.K;
    p.S = S;
    for (int d = 0; d < 4; ++d) {
      p.fR[d] = make_fastdiv(d < nR ? (unsigned)eR[d] : 1u);
      p.fK[d] = make_fastdiv(d < g0.nK ? (unsigned)g0.eK[d] : 1u);
    }
  };
  long long M, N;
  if (!swap) {
    fill(pa, g0.A, g0.nM, g0.eM, g0.aM);
    for (int d = 0; d < 4; ++d) pa.sK[d] = g0.aK[d];
    fill(pb, g0.B, g0.nN, g0.eN, g0.bN);
    for (int d = 0; d < 4; ++d) pb.sK[d] = g0.bK[d];
    M = g0.M;
    N = g0.N;
    a.nM = g0.nM;
    a.nN = g0.nN;
    for (int d = 0; d < 4; ++d) {
      a.eM[d] = g0.eM[d];
      a.cM[d] = g0.cM[d];
      a.eN[d] = g0.eN[d];
      a.cN[d] = g0.cN[d];
    }
  } else {
    fill(pa, g0.B, g0.nN, g0.eN, g0.bN);
    for (int d = 0; d < 4; ++d) pa.sK[d] = g0.bK[d];
    fill(pb, g0.A, g0.nM, g0.eM, g0.aM);
    for (int d = 0; d < 4; ++d) pb.sK[d] = g0.aK[d];
    M = g0.N;
    N = g0.M;
    a.nM = g0.nN;
    a.nN = g0.nM;
    for (int d = 0; d < 4; ++d) {
      a.eM[d] = g0.eN[d];
      a.cM[d] = g0.cN[d];
      a.eN[d] = g0.eM[d];
      a.cN[d] = g0.cM[d];
    }
  }
  pa.vec = pack_vec_ok(pa);
  pb.vec = pack_vec_ok(pb);
  int BN = ch.bn ? ch.bn : N <= 32 ? 32 : 64;
  // shared memory per CTA is capped at 227 KiB (static arrays take up to 4 KiB)
  while (BN > 32 && oz_smem_bytes(S, BN) + 4096 > 227 * 1024) BN /= 2;
  const int MT = (int)((M + OZ_BM - 1) / OZ_BM), NT = (int)((N + BN - 1) / BN);
  const int KT = (int)((g0.K + OZ_BK - 1) / OZ_BK);
  pa.R = M;
  pa.T = MT;
  pa.TR = OZ_BM;
  pa.KT = KT;
  pb.R = N;
  pb.T = NT;
  pb.TR = BN;
  pb.KT = KT;
  // spread a short output over more CTAs by splitting the k tiles
  int splits = 1, ktper = KT;
  const long long ctas = (long long)MT * NT;
  if (ch.split_mode != 1 && ctas < 2 * 152 && KT >= 2 * OZ_SPLIT_MIN) {
    long long sp = (2 * 152 + ctas - 1) / ctas;
    if (ch.split_mode == 2) sp *= 2;
    if (sp > KT / OZ_SPLIT_MIN) sp = KT / OZ_SPLIT_MIN;
    if (sp >= 2) {
      ktper = (KT + (int)sp - 1) / (int)sp;
      splits = (KT + ktper - 1) / ktper;
    }
  }
  cudaStream_t st = ws.stream;
  size_t capA, capB, capE, capP = 0;
  const size_t nA = (size_t)S * MT * KT * OZ_TILE_ELEMS, nB = (size_t)S * NT * KT * BN * OZ_BK;
  double* bufA = ws.get((nA + 3) / 4, capA);  // bf16 digit tiles in double-sized blocks
  double* bufB = ws.get((nB + 3) / 4, capB);
  const size_t nE = (size_t)MT * OZ_BM + (size_t)NT * BN;
  double* bufE = ws.get((nE + 1) / 2, capE);
  double* part = nullptr;
  if (splits > 1) part = ws.get((size_t)splits * MT * OZ_BM * NT * BN, capP);
  int* ea = (int*)bufE;
  int* fb = ea + (size_t)MT * OZ_BM;
  // algorithmic bytes: each operand element read twice (8 B each), S bf16 digits written
  int r = ws.begin(K_OZAKI_PACK, 0.0, (16.0 + 2.0 * S) * (double)(M + N) * (double)g0.K);
  if (r >= 0) {
    ws.recs[r].m = M;
    ws.recs[r].n = N;
    ws.recs[r].k = g0.K;
  }
  check_cuda(cudaMemsetAsync(ea, 0, nE * sizeof(int), st), "cudaMemsetAsync (exponents)");
  PackPass pp{};
  long long w1max = 1, w2max = 1;
  PackPass pd{};
  for (int o = 0; o < 2; ++o) {
    const OzPack& p = o ? pb : pa;
    const long long rows = (long long)p.T * p.TR;
    const long long q1 = (p.K + 7) / 8, q2 = (long long)p.KT * (OZ_BK / 8);
    pp.p[o] = pd.p[o] = p;
    pp.eu[o] = pd.eu[o] = (unsigned*)(o ? fb : ea);
    pp.dst[o] = pd.dst[o] = (__nv_bfloat16*)(o ? bufB : bufA);
    pp.kfast[o] = pd.kfast[o] = pack_kfast(p);
    pp.fR[o] = pd.fR[o] = make_fastdiv((unsigned)rows);
    pp.fQ[o] = make_fastdiv((unsigned)q1);
    pd.fQ[o] = make_fastdiv((unsigned)q2);
    pp.W[o] = (unsigned)(rows * q1);
    pd.W[o] = (unsigned)(rows * q2);
    w1max = std::max(w1max, rows * q1);
    w2max = std::max(w2max, rows * q2);
  }
  k_ozaki_rowexp<<<dim3((unsigned)oz_pack_grid(w1max), 2), PACK_T, 0, st>>>(pp);
  const dim3 g2((unsigned)oz_pack_grid(w2max), 2);
  switch (S) {
    case 1: k_ozaki_digits<1><<<g2, PACK_T, 0, st>>>(pd); break;
    case 2: k_ozaki_digits<2><<<g2, PACK_T, 0, st>>>(pd); break;
    case 3: k_ozaki_digits<3><<<g2, PACK_T, 0, st>>>(pd); break;
    case 4: k_ozaki_digits<4><<<g2, PACK_T, 0, st>>>(pd); break;
    case 5: k_ozaki_digits<5><<<g2, PACK_T, 0, st>>>(pd); break;
    case 6: k_ozaki_digits<6><<<g2, PACK_T, 0, st>>>(pd); break;
    case 7: k_ozaki_digits<7><<<g2, PACK_T, 0, st>>>(pd); break;
    default: k_ozaki_digits<8><<<g2, PACK_T, 0, st>>>(pd); break;
  }
  ws.end(r);
  ws.launches += 1;  // two pack kernels (begin() counted one; the memset is not a kernel)
  a.As = (const __nv_bfloat16*)bufA;
  a.Bs = (const __nv_bfloat16*)bufB;
  a.ea = ea;
  a.fb = fb;
  a.S = S;
  a.MT = MT;
  a.NT = NT;
  a.KT = KT;
  a.M = M;
  a.N = N;
  a.alpha = g0.alpha;
  a.C = g0.C;
  a.status = ws.oz_status;
  a.wait_cycles = ws.wait_cycles > 0 ? ws.wait_cycles : OZ_WAIT_CYCLES;
  a.splits = splits;
  a.ktper = ktper;
  a.part = part;
  a.rowfast = (a.nM > 0 && a.nN > 0 && a.cM[a.nM - 1] < a.cN[a.nN - 1]) || (a.nN == 0 && a.nM > 0) ? 1 : 0;
  // timed as the tensor-core kernel whatever the contraction (kind is the
  // step it belongs to); flops: the FP64 product it computes, executed:
  // digit pairs with t + u <= S + 1 over the padded tiles
  (void)kind;
  const double pairs = (double)S * (S + 1) / 2.0;
  r = ws.begin(K_OZAKI_MMA, 2.0 * (double)M * (double)N * (double)g0.K, 0.0,
               2.0 * pairs * (double)MT * OZ_BM * (double)NT * BN * (double)KT * OZ_BK);
  if (r >= 0) {
    ws.recs[r].m = M;
    ws.recs[r].n = N;
    ws.recs[r].k = g0.K;
  }
  oz_launch_mma(a, MT, NT, BN, st);
  ws.end(r);
  if (splits > 1) ws.launches++;
  ws.put(bufA, capA);
  ws.put(bufB, capB);
  ws.put(bufE, capE);
  if (part) ws.put(part, capP);
}

}  // namespace

// Tile width and k split of a split product: fixed rules, or with ws.tune the
// fastest of a few candidates, timed once per (M, N, K, slices) and device on
// the caller's operands with alpha = 0 (C keeps its values bit for bit) and
// cached for the process.  No timing while the stream is being captured.
namespace {
struct OzKey {
  long long M, N, K;
  int S, dev;
  bool operator<(const OzKey& o) const {
    if (M != o.M) return M < o.M;
    if (N != o.N) return N < o.N;
    if (K != o.K) return K < o.K;
    if (S != o.S) return S < o.S;
    return dev < o.dev;
  }
};
std::mutex g_tune_mu;
std::map<OzKey, OzChoice> g_tune;

OzChoice choose(Workspace& ws, const GemmArgs& g0, int S, int kind) {
  OzChoice def;
  if (!ws.tune) return def;
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  const OzKey key{g0.M, g0.N, g0.K, S, dev};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  int stored[2];
  if (tune_cache_lookup("tile", g0.M, g0.N, g0.K, S, 2, stored)) {
    OzChoice c;
    c.bn = stored[0];
    c.split_mode = stored[1];
    if (c.bn == 32 || c.bn == 64) {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune[key] = c;
      return c;
    }
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  check_cuda(cudaStreamIsCapturing(ws.stream, &cs), "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) return def;
  // candidates: tile widths up to about twice the shorter output side, and
  // the k-split rule, no split, twice the rule when the rule splits
  const long long nshort = g0.M < g0.N ? g0.M : g0.N;
  const long long KT = (g0.K + OZ_BK - 1) / OZ_BK;
  std::vector<OzChoice> cands;
  for (int bn : {32, 64}) {
    if (bn != 32 && bn / 2 >= nshort) continue;
    const long long big = g0.M > g0.N ? g0.M : g0.N;
    const long long ctas = ((big + OZ_BM - 1) / OZ_BM) * ((nshort + bn - 1) / bn);
    const bool splits = ctas < 2 * 152 && KT >= 2 * OZ_SPLIT_MIN;
    for (int sm = 0; sm < (splits ? 3 : 1); ++sm) {
      OzChoice c;
      c.bn = bn;
      c.split_mode = sm;
      cands.push_back(c);
    }
  }
  GemmArgs gz = g0;
  gz.alpha = 0.0;
  const bool prof = ws.profiling;
  const long long launches = ws.launches;
  ws.profiling = false;
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
  check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  OzChoice best = def;
  float best_ms = 1e30f;
  for (const OzChoice& c : cands) {
    ozaki_run(ws, gz, S, kind, c);  // first run: packing buffers, caches
    check_cuda(cudaEventRecord(e0, ws.stream), "cudaEventRecord");
    ozaki_run(ws, gz, S, kind, c);
    check_cuda(cudaEventRecord(e1, ws.stream), "cudaEventRecord");
    check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ws.profiling = prof;
  ws.launches = launches;
  const int v[2] = {best.bn, best.split_mode};
  tune_cache_store("tile", g0.M, g0.N, g0.K, S, 2, v);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
  return best;
}
}  // namespace

void ozaki_gemm(Workspace& ws, const GemmArgs& g0, int S, int kind) {
  if (g0.M <= 0 || g0.N <= 0 || g0.K <= 0) return;
  ozaki_run(ws, g0, S, kind, choose(ws, g0, S, kind));
}

}  // namespace dsrg

// ---------------------------------------------------------------------------
// C entry point
// ---------------------------------------------------------------------------
#include "../../include/dsrg.h"

namespace dsrg {
int set_error(int code, const char* msg);
}

extern "C" int dsrg_split_gemm(long long M, long long N, long long K, const double* A, long long lda, const double* B,
                               long long ldb, double* C, long long ldc, double alpha, int slices, void* stream) {
  using namespace dsrg;
  if (M < 0 || N < 0 || K < 0 || M >= (1LL << 31) || N >= (1LL << 31) || K >= (1LL << 31))
    return set_error(DSRG_ERR_ARG, "split gemm: sizes must be in [0, 2^31)");
  if (slices < 1 || slices > kOzakiMaxSlices) return set_error(DSRG_ERR_ARG, "split gemm: slices must be 1..8");
  if (M == 0 || N == 0 || K == 0) return DSRG_OK;
  if (!A || !B || !C) return set_error(DSRG_ERR_ARG, "split gemm: NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  try {
    Workspace ws(st);
    int zero = 0;
    check_cuda(cudaMemcpyToSymbolAsync(g_oz_status_alias(), &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st),
               "status reset");
    GemmArgs g{};
    g.A = A;
    g.B = B;
    g.C = C;
    g.alpha = alpha;
    g.nM = 1;
    g.eM[0] = (int)M;
    g.aM[0] = lda;
    g.cM[0] = ldc;
    g.nN = 1;
    g.eN[0] = (int)N;
    g.bN[0] = 1;
    g.cN[0] = 1;
    g.nK = 1;
    g.eK[0] = (int)K;
    g.aK[0] = 1;
    g.bK[0] = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.nbatch = 1;
    ozaki_gemm(ws, g, slices, K_OZAKI_MMA);
    check_cuda(cudaGetLastError(), "split gemm launch");
    if (ozaki_status(st, nullptr))
      return set_error(DSRG_ERR_TIMEOUT, "split gemm: a bounded wait in the kernel ran out");
  } catch (const Error& e) {
    return set_error(e.code, e.what());
  } catch (const std::exception& e) {
    return set_error(DSRG_ERR_INTERNAL, e.what());
  }
  return DSRG_OK;
}

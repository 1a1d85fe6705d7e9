// Split-precision FP64 contraction on tcgen05 (see ozaki.cuh).
#include <cuda_bf16.h>

#include <cstdint>
#include <stdexcept>

#include "ozaki.cuh"

namespace dsrg {
namespace {

constexpr int OZ_BM = 128, OZ_BK = 64;
constexpr int OZ_THREADS = 256;  // 8 warps: lane quadrant (warp % 4) x column half (warp / 4)
constexpr int OZ_TILE_ELEMS = OZ_BM * OZ_BK;  // A tile: 8192 bf16 = 16 KiB
constexpr int OZ_TILE_BYTES = OZ_TILE_ELEMS * 2;
constexpr long long OZ_WAIT_LIMIT = 1LL << 22;

__device__ int g_oz_status;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzled
// layout (rows of 64 bf16, 8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = BN.
template <int BN>
__host__ __device__ constexpr uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
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

// bounded wait: false if the phase did not complete in time
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  for (long long i = 0; i < OZ_WAIT_LIMIT; ++i)
    if (mbar_try(bar, phase)) return true;
  return false;
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
  int* status;
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

// One CTA: a 128 x BN tile of C.  Thread t owns TMEM lane t (tile row t).
// TMEM columns: level accumulator [0,BN), running hi [BN,2BN), lo [2BN,3BN).
template <int BN>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_ozaki_mma(const OzArgs a) {
  constexpr uint32_t TMEM_COLS = BN == 128 ? 512 : BN == 64 ? 256 : 128;
  constexpr int B_TILE_BYTES = BN * OZ_BK * 2;
  constexpr uint32_t IDESC = oz_idesc<BN>();
  // columns per warp in the fold and epilogue: two column halves for BN >= 64;
  // for BN = 32 the second half of the warps sits out
  constexpr int HALF = BN >= 64 ? BN / 2 : BN;
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + (size_t)a.S * OZ_TILE_BYTES;
  __shared__ uint64_t bar_mma, bar_load;
  __shared__ uint32_t tmem_base;
  __shared__ long long colC[BN];
  __shared__ int colE[BN];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int quad = warp & 3, half = warp >> 2;  // TMEM lanes 32*quad.., columns half*HALF..
  const int row = quad * 32 + (tid & 31);
  const int mt = blockIdx.x, nt = blockIdx.y, z = blockIdx.z;
  const int kt0 = a.splits > 1 ? z * a.ktper : 0;
  const int kt1 = a.splits > 1 ? (kt0 + a.ktper < a.KT ? kt0 + a.ktper : a.KT) : a.KT;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar_mma, 1);
    mbar_init(&bar_load, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int t = tid; t < BN; t += OZ_THREADS) {
    long long n = (long long)nt * BN + t;
    colC[t] = n < a.N ? c_offset(n, a.nN, a.eN, a.cN) : -1;
    colE[t] = a.fb[(long long)nt * BN + t];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tmem_base;
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  const uint32_t col0 = (uint32_t)(half * HALF);
  const int nchunk = (BN >= 64 || half == 0) ? HALF / 32 : 0;  // 32-column chunks of this warp

  // zero the running float-float sums (hi, lo) of this thread's columns
  {
    uint32_t zr[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) zr[q] = 0u;
#pragma unroll
    for (int j = 0; j < nchunk; ++j) {
      tmem_st32(tm + lane_off + BN + col0 + 32 * j, zr);
      tmem_st32(tm + lane_off + 2 * BN + col0 + 32 * j, zr);
    }
    tmem_wait_st();
  }
  uint32_t ph_mma = 0, ph_load = 0;
  bool ok = true;
  const int S = a.S;
  for (int kt = kt0; kt < kt1 && ok; ++kt) {
    // stage the S digit tiles of A and of B for this k chunk (bulk copies)
    if (tid == 0) {
      mbar_expect_tx(&bar_load, (uint32_t)(S * (OZ_TILE_BYTES + B_TILE_BYTES)));
      for (int s = 0; s < S; ++s) {
        bulk_g2s(sA + (size_t)s * OZ_TILE_BYTES, a.As + ((size_t)(s * a.MT + mt) * a.KT + kt) * OZ_TILE_ELEMS,
                 OZ_TILE_BYTES, &bar_load);
        bulk_g2s(sB + (size_t)s * B_TILE_BYTES, a.Bs + ((size_t)(s * a.NT + nt) * a.KT + kt) * (BN * OZ_BK),
                 B_TILE_BYTES, &bar_load);
      }
    }
    ok = mbar_wait(&bar_load, ph_load);
    ph_load ^= 1;
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    for (int c = 2; c <= S + 1 && ok; ++c) {
      if (tid == 0) {
        uint32_t accum = 0;
        const int t0 = c - S > 1 ? c - S : 1, t1 = c - 1 < S ? c - 1 : S;
        for (int t = t0; t <= t1; ++t) {
          const int u = c - t;
          const uint32_t aA = smem_u32(sA + (size_t)(t - 1) * OZ_TILE_BYTES);
          const uint32_t aB = smem_u32(sB + (size_t)(u - 1) * B_TILE_BYTES);
#pragma unroll
          for (int ks = 0; ks < OZ_BK / 16; ++ks) {
            mma_bf16(tm, sdesc(aA + 32 * ks), sdesc(aB + 32 * ks), IDESC, accum);
            accum = 1;
          }
        }
        mma_commit(&bar_mma);
      }
      ok = mbar_wait(&bar_mma, ph_mma);
      ph_mma ^= 1;
      ok = __syncthreads_and(ok) != 0;
      tc_fence_after();
      if (!ok) break;
      // fold level c: (hi, lo) += acc * 2^(-7c), two-sum in FP32
      const float scale = exp2f(-7.0f * (float)c);
#pragma unroll 1
      for (int j = 0; j < nchunk; ++j) {
        uint32_t acc[32], hi[32], lo[32];
        const uint32_t cc = col0 + 32 * j;
        tmem_ld32(tm + lane_off + cc, acc);
        tmem_ld32(tm + lane_off + BN + cc, hi);
        tmem_ld32(tm + lane_off + 2 * BN + cc, lo);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          float x = __uint_as_float(acc[q]) * scale;
          float h = __uint_as_float(hi[q]);
          float s_ = h + x;
          float bp = s_ - h;
          float err = (h - (s_ - bp)) + (x - bp);
          float l = __uint_as_float(lo[q]) + err;
          float s2 = s_ + l;
          l = l - (s2 - s_);
          hi[q] = __float_as_uint(s2);
          lo[q] = __float_as_uint(l);
        }
        tmem_st32(tm + lane_off + BN + cc, hi);
        tmem_st32(tm + lane_off + 2 * BN + cc, lo);
      }
      tmem_wait_st();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }
  // epilogue: alpha * 2^(ea[m] + fb[n]) * (hi + lo) into C, or the scaled
  // partial into part[z] when K is split
  if (ok) {
    const long long m = (long long)mt * OZ_BM + row;
    const long long offm = m < a.M ? c_offset(m, a.nM, a.eM, a.cM) : -1;
    const int em = a.ea[(long long)mt * OZ_BM + row];
    const long long ldp = (long long)a.NT * BN;
    double* prow = a.splits > 1 ? a.part + ((long long)z * a.MT * OZ_BM + m) * ldp + (long long)nt * BN : nullptr;
#pragma unroll 1
    for (int j = 0; j < nchunk; ++j) {
      uint32_t hi[32], lo[32];
      const int cc = (int)col0 + 32 * j;
      tmem_ld32(tm + lane_off + BN + cc, hi);
      tmem_ld32(tm + lane_off + 2 * BN + cc, lo);
      tmem_wait_ld();
      if (prow) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          double v = (double)__uint_as_float(hi[q]) + (double)__uint_as_float(lo[q]);
          prow[cc + q] = colC[cc + q] >= 0 && offm >= 0 ? ldexp(v, em + colE[cc + q]) : 0.0;
        }
      } else if (offm >= 0) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const long long oc = colC[cc + q];
          if (oc < 0) continue;
          double v = (double)__uint_as_float(hi[q]) + (double)__uint_as_float(lo[q]);
          a.C[offm + oc] += a.alpha * ldexp(v, em + colE[cc + q]);
        }
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
};

__device__ __forceinline__ long long src_offset32(int lin, int nd, const int* ext, const long long* st) {
  long long o = 0;
  for (int d = nd - 1; d >= 0; --d) {
    int q = lin / ext[d];
    o += (long long)(lin - q * ext[d]) * st[d];
    lin = q;
  }
  return o;
}

// One CTA per row r (rows beyond R and rows of padding write zeros):
// e[r] = max over k of the binary exponent ex with |x| < 2^ex (frexp), then
// the S digits of every element of the row go to their swizzled tile slots.
constexpr int PACK_T = 256;

__device__ __forceinline__ int exp_of(double x) {
  if (x == 0.0) return -2000;
  const long long bits = __double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  return be ? be - 1022 : -1022;
}

__global__ void __launch_bounds__(PACK_T) k_ozaki_pack(const OzPack p, int* e_out, __nv_bfloat16* dst) {
  const int r = blockIdx.x;  // over T * TR rows (padded)
  const long long Kp = (long long)p.KT * OZ_BK;
  const bool live = r < p.R;
  const long long roff = live ? src_offset32(r, p.nR, p.eR, p.sR) : 0;
  // row maximum exponent
  int emax = -2000;
  if (live)
    for (int k = threadIdx.x; k < p.K; k += PACK_T) {
      const int ex = exp_of(p.src[roff + src_offset32(k, p.nK, p.eK, p.sK)]);
      emax = ex > emax ? ex : emax;
    }
  __shared__ int sh[PACK_T / 32];
  for (int o = 16; o > 0; o >>= 1) {
    const int v = __shfl_xor_sync(0xffffffffu, emax, o);
    emax = v > emax ? v : emax;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = emax;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < PACK_T / 32 ? sh[threadIdx.x] : -2000;
    for (int o = 16; o > 0; o >>= 1) {
      const int w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (threadIdx.x == 0) sh[0] = v;
  }
  __syncthreads();
  const int e = sh[0];
  if (threadIdx.x == 0) e_out[r] = e;
  const int F = 7 * p.S;
  const long long tile_elems = (long long)p.TR * OZ_BK;
  const int tr = r / p.TR, rr = r - tr * p.TR;
  for (long long k = threadIdx.x; k < Kp; k += PACK_T) {
    double x = 0.0;
    if (live && k < p.K) x = p.src[roff + src_offset32((int)k, p.nK, p.eK, p.sK)];
    unsigned long long v = 0;
    bool neg = false;
    if (x != 0.0) {
      const long long bits = __double_as_longlong(x);
      neg = bits < 0;
      const int be = (int)((bits >> 52) & 0x7FF);
      unsigned long long m = (unsigned long long)(bits & ((1LL << 52) - 1));
      int E;
      if (be) {
        m |= 1ULL << 52;
        E = be - 1075;
      } else {
        E = -1074;
      }
      const int sh_ = E + F - e;  // v = m 2^sh < 2^F
      if (sh_ >= 0) v = sh_ < 12 ? (m << sh_) : 0;
      else v = (-sh_) >= 64 ? 0 : (m >> (-sh_));
    }
    const int tk = (int)(k / OZ_BK), kk = (int)(k - (long long)tk * OZ_BK);
    const int chunk = kk >> 3, j = kk & 7;
    const long long within = (long long)rr * OZ_BK + ((chunk ^ (rr & 7)) << 3) + j;
    for (int t = 1; t <= p.S; ++t) {
      int d = (int)((v >> (7 * (p.S - t))) & 127ULL);
      if (neg) d = -d;
      const long long tile = ((long long)(t - 1) * p.T + tr) * p.KT + tk;
      dst[tile * tile_elems + within] = __float2bfloat16_rn((float)d);
    }
  }
}

inline int oz_grid(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

int* oz_status_ptr() {
  int* p = nullptr;
  check_cuda(cudaGetSymbolAddress((void**)&p, g_oz_status), "cudaGetSymbolAddress (status)");
  return p;
}

size_t oz_smem_bytes(int S, int BN) { return (size_t)S * OZ_TILE_BYTES + (size_t)S * BN * OZ_BK * 2 + 1024; }

template <int BN>
void oz_launch_bn(const OzArgs& a, int MT, int NT, cudaStream_t st) {
  // at least 120 KiB so that one CTA (one TMEM allocation) occupies an SM
  size_t smem = oz_smem_bytes(a.S, BN);
  if (smem < 120 * 1024) smem = 120 * 1024;
  check_cuda(cudaFuncSetAttribute(k_ozaki_mma<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
             "cudaFuncSetAttribute (ozaki)");
  k_ozaki_mma<BN><<<dim3(MT, NT, a.splits > 1 ? a.splits : 1), OZ_THREADS, smem, st>>>(a);
  if (a.splits > 1) k_ozaki_reduce<BN><<<oz_grid(a.M * a.N), 256, 0, st>>>(a);
}

void oz_launch_mma(const OzArgs& a, int MT, int NT, int BN, cudaStream_t st) {
  if (BN == 32) oz_launch_bn<32>(a, MT, NT, st);
  else if (BN == 64) oz_launch_bn<64>(a, MT, NT, st);
  else oz_launch_bn<128>(a, MT, NT, st);
}
}  // namespace

const void* g_oz_status_alias() { return (const void*)&g_oz_status; }

int ozaki_status(cudaStream_t st) {
  int v = 0;
  check_cuda(cudaMemcpyFromSymbolAsync(&v, g_oz_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st), "status");
  check_cuda(cudaStreamSynchronize(st), "sync");
  return v;
}

void ozaki_gemm(Workspace& ws, const GemmArgs& g0, int S, int kind) {
  if (g0.M <= 0 || g0.N <= 0 || g0.K <= 0) return;
  if (g0.nbatch != 1) throw std::runtime_error("split-precision contraction needs nbatch == 1");
  if (S < 1 || S > kOzakiMaxSlices) throw std::runtime_error("split-precision slices must be 1..7");
  if (g0.M >= (1LL << 31) || g0.N >= (1LL << 31) || g0.K >= (1LL << 31))
    throw std::runtime_error("split-precision contraction sizes must stay below 2^31");
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
  const int BN = N <= 32 ? 32 : N <= 64 ? 64 : 128;
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
  if (ctas < 2 * 152 && KT >= 8) {
    long long sp = (2 * 152 + ctas - 1) / ctas;
    if (sp > KT / 4) sp = KT / 4;
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
  int r = ws.begin(K_OZAKI_PACK, 0.0, 8.0 * (double)(M + N) * (double)g0.K * 2.0);
  k_ozaki_pack<<<(unsigned)(MT * OZ_BM), PACK_T, 0, st>>>(pa, ea, (__nv_bfloat16*)bufA);
  k_ozaki_pack<<<(unsigned)(NT * BN), PACK_T, 0, st>>>(pb, fb, (__nv_bfloat16*)bufB);
  ws.end(r);
  ws.launches += 1;
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
  a.status = nullptr;
  a.splits = splits;
  a.ktper = ktper;
  a.part = part;
  // executed tensor-core flops: digit pairs with t + u <= S + 1, padded tiles
  const double pairs = (double)S * (S + 1) / 2.0;
  r = ws.begin(kind, 2.0 * pairs * (double)MT * OZ_BM * (double)NT * BN * (double)KT * OZ_BK, 0.0);
  oz_launch_mma(a, MT, NT, BN, st);
  ws.end(r);
  if (splits > 1) ws.launches++;
  ws.put(bufA, capA);
  ws.put(bufB, capB);
  ws.put(bufE, capE);
  if (part) ws.put(part, capP);
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
  if (slices < 1 || slices > kOzakiMaxSlices) return set_error(DSRG_ERR_ARG, "split gemm: slices must be 1..7");
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
    if (ozaki_status(st)) return set_error(DSRG_ERR_CUDA, "split gemm: a bounded wait in the kernel ran out");
  } catch (const std::exception& e) {
    return set_error(DSRG_ERR_CUDA, e.what());
  }
  return DSRG_OK;
}

// Device kernels of the DSRG-MRPT2/PT3 energy path (sm_103a), FP64.
#include "kernels.cuh"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace dsrg {

// ---------------------------------------------------------------------------
// generic strided contraction
// ---------------------------------------------------------------------------
// One CTA computes a 64 x 64 tile of C with 256 threads (4 x 4 outputs each),
// stepping K by 16.  Operand addresses are separable: off(A[m,k]) =
// offA(m) + offA(k), so the tile's row/column/k offsets are decoded once
// into shared memory and the inner loop is a plain tiled GEMM.
namespace {
constexpr int BK = 16, NT = 256;

__device__ __forceinline__ void decode(long long lin, int nd, const int* ext, const long long* s1,
                                       const long long* s2, long long& o1, long long& o2) {
  o1 = 0;
  o2 = 0;
  for (int d = nd - 1; d >= 0; --d) {
    long long q = lin / ext[d];
    int r = (int)(lin - q * ext[d]);
    o1 += r * s1[d];
    o2 += r * s2[d];
    lin = q;
  }
}

// Tile BM_ x BN_ with 256 threads, each owning a 4 x 4 block of outputs at
// rows tm + (BM_/4) i and columns tn + (BN_/4) j (conflict-free shared reads).
template <int BM_, int BN_, int TAG>
__global__ void __launch_bounds__(NT) k_gemm(const GemmArgs g) {
  constexpr int NTN = BN_ / 4, NTM = BM_ / 4;
  static_assert(NTM * NTN == NT, "tile must give 256 threads 4x4 outputs each");
  __shared__ double As[BK][BM_];
  __shared__ double Bs[BK][BN_];
  __shared__ long long offAm[BM_], offCm[BM_], offBn[BN_], offCn[BN_], offAk[BK], offBk[BK];
  const int tid = threadIdx.x;
  const long long m0 = (long long)blockIdx.x * BM_;
  const long long n0 = (long long)blockIdx.y * BN_;
  long long oAb = 0, oBb = 0, oCb = 0;
  const int split = g.splits > 1 ? (int)blockIdx.z : 0;
  const long long kbeg = g.splits > 1 ? (long long)split * g.kper : 0;
  const long long kend = g.splits > 1 ? (kbeg + g.kper < g.K ? kbeg + g.kper : g.K) : g.K;
  if (g.splits <= 1) {
    long long lin = blockIdx.z;
    for (int d = g.nB - 1; d >= 0; --d) {
      long long q = lin / g.eB[d];
      int r = (int)(lin - q * g.eB[d]);
      oAb += r * g.aB[d];
      oBb += r * g.bB[d];
      oCb += r * g.cB[d];
      lin = q;
    }
  }
  for (int t = tid; t < BM_; t += NT) {
    long long m = m0 + t;
    if (m < g.M) decode(m, g.nM, g.eM, g.aM, g.cM, offAm[t], offCm[t]);
    else { offAm[t] = -1; offCm[t] = -1; }
  }
  for (int t = tid; t < BN_; t += NT) {
    long long n = n0 + t;
    if (n < g.N) decode(n, g.nN, g.eN, g.bN, g.cN, offBn[t], offCn[t]);
    else { offBn[t] = -1; offCn[t] = -1; }
  }
  const int tn = tid % NTN, tm = tid / NTN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (long long k0 = kbeg; k0 < kend; k0 += BK) {
    if (tid < BK) {
      long long k = k0 + tid;
      if (k < kend) decode(k, g.nK, g.eK, g.aK, g.bK, offAk[tid], offBk[tid]);
      else { offAk[tid] = -1; offBk[tid] = -1; }
    }
    __syncthreads();
#pragma unroll
    for (int e = tid; e < BM_ * BK; e += NT) {
      int mm = e % BM_, kk = e / BM_;
      long long om = offAm[mm], ok = offAk[kk];
      As[kk][mm] = (om >= 0 && ok >= 0) ? g.A[oAb + om + ok] : 0.0;
    }
#pragma unroll
    for (int e = tid; e < BN_ * BK; e += NT) {
      int nn = e % BN_, kk = e / BN_;
      long long on = offBn[nn], ok = offBk[kk];
      Bs[kk][nn] = (on >= 0 && ok >= 0) ? g.B[oBb + on + ok] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tm + NTM * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn + NTN * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (g.splits > 1) {
    double* Pp = g.part + (long long)split * g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      long long m = m0 + tm + NTM * i;
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        long long n = n0 + tn + NTN * j;
        if (n < g.N) Pp[m * g.N + n] = acc[i][j];
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long om = offCm[tm + NTM * i];
    if (om < 0) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long long on = offCn[tn + NTN * j];
      if (on < 0) continue;
      g.C[oCb + om + on] += g.alpha * acc[i][j];
    }
  }
}

// Outputs too few to fill tiles: one CTA per output element, its threads
// split K (32-bit index decoding), fixed-order tree reduction.
constexpr int SMALL_T = 128;
__device__ __forceinline__ void decode32(int lin, int nd, const int* ext, const long long* s1, const long long* s2,
                                         long long& o1, long long& o2) {
  o1 = 0;
  o2 = 0;
  for (int d = nd - 1; d >= 0; --d) {
    int q = lin / ext[d];
    int r = lin - q * ext[d];
    o1 += r * s1[d];
    o2 += r * s2[d];
    lin = q;
  }
}

__global__ void __launch_bounds__(SMALL_T) k_gemm_small(const GemmArgs g) {
  const long long out = blockIdx.x;  // over nbatch * M * N
  const long long MN = g.M * g.N;
  const long long b = out / MN, mn = out - b * MN;
  const long long m = mn / g.N, n = mn - m * g.N;
  long long oAb = 0, oBb = 0, oCb = 0;
  {
    long long lin = b;
    for (int d = g.nB - 1; d >= 0; --d) {
      long long q = lin / g.eB[d];
      int r = (int)(lin - q * g.eB[d]);
      oAb += r * g.aB[d];
      oBb += r * g.bB[d];
      oCb += r * g.cB[d];
      lin = q;
    }
  }
  long long oAm, oCm, oBn, oCn;
  decode(m, g.nM, g.eM, g.aM, g.cM, oAm, oCm);
  decode(n, g.nN, g.eN, g.bN, g.cN, oBn, oCn);
  const double* A = g.A + oAb + oAm;
  const double* B = g.B + oBb + oBn;
  const int split = g.splits > 1 ? (int)blockIdx.y : 0;
  const long long kb = g.splits > 1 ? split * g.kper : 0;
  const long long ke = g.splits > 1 ? (kb + g.kper < g.K ? kb + g.kper : g.K) : g.K;
  double acc = 0.0;
  for (long long k = kb + threadIdx.x; k < ke; k += SMALL_T) {
    long long oa, ob;
    decode32((int)k, g.nK, g.eK, g.aK, g.bK, oa, ob);
    acc = fma(A[oa], B[ob], acc);
  }
  __shared__ double sh[SMALL_T];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = SMALL_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (g.splits > 1) g.part[(long long)split * MN + mn] = sh[0];
    else g.C[oCb + oCm + oCn] += g.alpha * sh[0];
  }
}

// Short contractions (K <= 64): one thread per output element, the K-offset
// table staged once per CTA in shared memory.
constexpr int TPO_T = 256, TPO_KMAX = 64;
__global__ void __launch_bounds__(TPO_T) k_gemm_tpo(const GemmArgs g, int mfast) {
  __shared__ long long offA[TPO_KMAX], offB[TPO_KMAX];
  const int K = (int)g.K;
  for (int t = threadIdx.x; t < K; t += TPO_T) decode32(t, g.nK, g.eK, g.aK, g.bK, offA[t], offB[t]);
  __syncthreads();
  const long long total = g.M * g.N * g.nbatch;
  for (long long idx = blockIdx.x * (long long)TPO_T + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * TPO_T) {
    long long m, n, b;
    if (mfast) {
      long long r = idx / g.M;
      m = idx - r * g.M;
      b = r / g.N;
      n = r - b * g.N;
    } else {
      long long r = idx / g.N;
      n = idx - r * g.N;
      b = r / g.M;
      m = r - b * g.M;
    }
    long long oAb = 0, oBb = 0, oCb = 0;
    {
      long long lin = b;
      for (int d = g.nB - 1; d >= 0; --d) {
        long long q = lin / g.eB[d];
        int rr = (int)(lin - q * g.eB[d]);
        oAb += rr * g.aB[d];
        oBb += rr * g.bB[d];
        oCb += rr * g.cB[d];
        lin = q;
      }
    }
    long long oAm, oCm, oBn, oCn;
    decode32((int)m, g.nM, g.eM, g.aM, g.cM, oAm, oCm);
    decode32((int)n, g.nN, g.eN, g.bN, g.cN, oBn, oCn);
    const double* A = g.A + oAb + oAm;
    const double* B = g.B + oBb + oBn;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc = fma(A[offA[k]], B[offB[k]], acc);
    g.C[oCb + oCm + oCn] += g.alpha * acc;
  }
}

// Flat contraction: one thread per output element and k chunk, 32
// consecutive outputs per warp along the output index whose operand stride
// is smallest.  The k multi-index (padded to four dimensions) is decoded once
// per thread and then stepped like an odometer, so the inner loop is two
// loads and one FMA with no index division.  WK warps of a CTA take WK
// consecutive k chunks of the same 32 outputs and are summed in shared memory
// in a fixed order; gridDim.y > 1 leaves one partial per CTA row in part[z]
// for k_gemm_flat_reduce.  Nothing is padded, which matters on an SM with two
// FP64 FMA lanes per clock.
struct FlatK {
  int e[4];
  long long a[4], b[4];    // strides of A and B along the padded k dims
  long long wa[4], wb[4];  // offset change when dim d wraps into dim d-1
  FastDiv fk[4];           // divisors of the padded k dims
  FastDiv fM, fN, fm[4], fn[4], fb[4];
};

// (m, n, batch) of output o and its operand offsets; every index < 2^31
__device__ __forceinline__ void flat_out(const GemmArgs& g, const FlatK& fk, long long o, int mfast, long long& oA,
                                         long long& oB, long long& oC) {
  unsigned m, n, b;
  const unsigned uo = (unsigned)o;
  if (mfast) {
    const unsigned r = fast_div(uo, fk.fM);
    m = uo - r * fk.fM.d;
    b = fast_div(r, fk.fN);
    n = r - b * fk.fN.d;
  } else {
    const unsigned r = fast_div(uo, fk.fN);
    n = uo - r * fk.fN.d;
    b = fast_div(r, fk.fM);
    m = r - b * fk.fM.d;
  }
  long long oAb = 0, oBb = 0, oCb = 0, oAm = 0, oCm = 0, oBn = 0, oCn = 0;
  for (int d = g.nB - 1; d >= 0; --d) {
    const unsigned q = fast_div(b, fk.fb[d]);
    const int rr = (int)(b - q * fk.fb[d].d);
    oAb += rr * g.aB[d];
    oBb += rr * g.bB[d];
    oCb += rr * g.cB[d];
    b = q;
  }
  for (int d = g.nM - 1; d >= 0; --d) {
    const unsigned q = fast_div(m, fk.fm[d]);
    const int rr = (int)(m - q * fk.fm[d].d);
    oAm += rr * g.aM[d];
    oCm += rr * g.cM[d];
    m = q;
  }
  for (int d = g.nN - 1; d >= 0; --d) {
    const unsigned q = fast_div(n, fk.fn[d]);
    const int rr = (int)(n - q * fk.fn[d].d);
    oBn += rr * g.bN[d];
    oCn += rr * g.cN[d];
    n = q;
  }
  oA = oAb + oAm;
  oB = oBb + oBn;
  oC = oCb + oCm + oCn;
}

template <int WK>
__global__ void __launch_bounds__(256) k_gemm_flat(const GemmArgs g, const FlatK fk, const FlatTable tab, long long O,
                                                   int mfast, long long len, double* part) {
  constexpr int OG = 8 / WK;  // groups of 32 outputs per CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int og = warp / WK, wk = warp - og * WK;
  const long long o = ((long long)blockIdx.x * OG + og) * 32 + lane;
  const long long chunk = (long long)blockIdx.y * WK + wk;
  const long long klo = chunk * len;
  const long long khi = klo + len < g.K ? klo + len : g.K;
  double acc = 0.0;
  long long oA = 0, oB = 0, oC = 0;
  if (o < O) flat_out(g, fk, o, mfast, oA, oB, oC);
  const int grp = blockIdx.z;
  if (o < O && klo < khi) {
    int i0, i1, i2, i3;
    long long ka, kb;
    {
      unsigned lin = (unsigned)klo;
      unsigned q = fast_div(lin, fk.fk[3]);
      i3 = (int)(lin - q * fk.fk[3].d);
      lin = q;
      q = fast_div(lin, fk.fk[2]);
      i2 = (int)(lin - q * fk.fk[2].d);
      lin = q;
      q = fast_div(lin, fk.fk[1]);
      i1 = (int)(lin - q * fk.fk[1].d);
      i0 = (int)q;
      ka = i0 * fk.a[0] + i1 * fk.a[1] + i2 * fk.a[2] + i3 * fk.a[3];
      kb = i0 * fk.b[0] + i1 * fk.b[1] + i2 * fk.b[2] + i3 * fk.b[3];
    }
    auto step = [&]() {
      ++i3;
      ka += fk.a[3];
      kb += fk.b[3];
      if (i3 == fk.e[3]) {
        i3 = 0;
        ka += fk.wa[3];
        kb += fk.wb[3];
        ++i2;
        if (i2 == fk.e[2]) {
          i2 = 0;
          ka += fk.wa[2];
          kb += fk.wb[2];
          ++i1;
          if (i1 == fk.e[1]) {
            i1 = 0;
            ka += fk.wa[1];
            kb += fk.wb[1];
            ++i0;
          }
        }
      }
    };
    const int j0 = i0, j1 = i1, j2 = i2, j3 = i3;
    const long long ka0 = ka, kb0 = kb;
    double acc1 = 0.0;
    // the block pairs of this output block, in table order
    for (int pr = tab.first[grp]; pr < tab.first[grp + 1]; ++pr) {
      const double* A = tab.a[pr] + oA;
      const double* B = tab.b[pr] + oB;
      i0 = j0;
      i1 = j1;
      i2 = j2;
      i3 = j3;
      ka = ka0;
      kb = kb0;
      long long k = klo;
      for (; k + 4 <= khi; k += 4) {
        long long pa[4], pb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          pa[u] = ka;
          pb[u] = kb;
          step();
        }
        double av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          av[u] = __ldg(A + pa[u]);
          bv[u] = __ldg(B + pb[u]);
        }
        acc = fma(av[0], bv[0], acc);
        acc1 = fma(av[1], bv[1], acc1);
        acc = fma(av[2], bv[2], acc);
        acc1 = fma(av[3], bv[3], acc1);
      }
      for (; k < khi; ++k) {
        acc = fma(__ldg(A + ka), __ldg(B + kb), acc);
        step();
      }
    }
    acc += acc1;
  }
  if (WK > 1) {
    __shared__ double sh[8][32];
    sh[warp][lane] = acc;
    __syncthreads();
    if (wk == 0)
      for (int w = 1; w < WK; ++w) acc += sh[warp + w][lane];
  }
  if (wk == 0 && o < O) {
    if (gridDim.y > 1) part[((long long)grp * gridDim.y + blockIdx.y) * O + o] = acc;
    else tab.c[grp][oC] += g.alpha * acc;
  }
}

// C_grp[o] += alpha * sum_z part[grp][z][o], z in increasing order (grp = blockIdx.y)
__global__ void k_gemm_flat_reduce(const GemmArgs g, const FlatK fk, const FlatTable tab, long long O, int mfast,
                                   int Z, const double* part) {
  const int grp = blockIdx.y;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < O; o += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < Z; ++z) s += part[((long long)grp * Z + z) * O + o];
    long long oA, oB, oC;
    flat_out(g, fk, o, mfast, oA, oB, oC);
    tab.c[grp][oC] += g.alpha * s;
  }
}

// C[m, n] += alpha * sum_z part[z][m][n], z in increasing order
__global__ void k_gemm_splitk_reduce(const GemmArgs g) {
  const long long MN = g.M * g.N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < MN;
       idx += (long long)gridDim.x * blockDim.x) {
    long long m = idx / g.N, n = idx - m * g.N;
    double s = 0.0;
    for (int z = 0; z < g.splits; ++z) s += g.part[z * MN + idx];
    long long oa, om, ob, on;
    decode(m, g.nM, g.eM, g.aM, g.cM, oa, om);
    decode(n, g.nN, g.eN, g.bN, g.cN, ob, on);
    g.C[om + on] += g.alpha * s;
  }
}

// ---------------------------------------------------------------------------
// elementwise and reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ void nd_offsets(const NdArgs& g, long long lin, long long& oa, long long& ob) {
  oa = 0;
  ob = 0;
  for (int d = g.nd - 1; d >= 0; --d) {
    long long q = lin / g.e[d];
    int r = (int)(lin - q * g.e[d]);
    oa += r * g.sa[d];
    ob += r * g.sb[d];
    lin = q;
  }
}

// offsets of linear index lin; FAST: lin < 2^31, divisions by multiply-high
template <bool FAST>
__device__ __forceinline__ void nd_off(const NdArgs& g, long long lin, long long& oa, long long& ob) {
  if (!FAST) {
    nd_offsets(g, lin, oa, ob);
    return;
  }
  unsigned l = (unsigned)lin;
  oa = 0;
  ob = 0;
  for (int d = g.nd - 1; d >= 0; --d) {
    const unsigned q = fast_div(l, g.fe[d]);
    const int r = (int)(l - q * g.fe[d].d);
    oa += r * g.sa[d];
    ob += r * g.sb[d];
    l = q;
  }
}

template <bool FAST>
__global__ void k_axpy(const NdArgs g, double alpha, const double* __restrict__ A, double* __restrict__ C) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    long long oa, oc;
    nd_off<FAST>(g, i, oa, oc);
    C[oc] += alpha * A[oa];
  }
}

// Compensated (Neumaier) per-thread sums, then a fixed-order tree.
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

constexpr int DOT_THREADS = 256;

template <bool FAST>
__global__ void k_axpy_blocks(const NdArgs g, double alpha, const AxpyBlocks p) {
  const double* __restrict__ A = p.a[blockIdx.y];
  double* __restrict__ C = p.c[blockIdx.y];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    long long oa, oc;
    nd_off<FAST>(g, i, oa, oc);
    C[oc] += alpha * A[oa];
  }
}

// fixed-order compensated tree over the DOT_THREADS pairs (s, c) in shared memory
__device__ __forceinline__ void dot_tree(double* sh_s, double* sh_c) {
  for (int w = DOT_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double s2 = sh_s[threadIdx.x], c2 = sh_c[threadIdx.x];
      neumaier(s2, c2, sh_s[threadIdx.x + w]);
      c2 += sh_c[threadIdx.x + w];
      sh_s[threadIdx.x] = s2;
      sh_c[threadIdx.x] = c2;
    }
    __syncthreads();
  }
}

template <bool FAST>
__global__ void __launch_bounds__(DOT_THREADS) k_dot_blocks(const NdArgs g, const DotBlocks p, double* partial,
                                                           unsigned* ticket, double alpha, double* out) {
  const double* __restrict__ A = p.a[blockIdx.y];
  const double* __restrict__ B = p.b[blockIdx.y];
  double s = 0.0, c = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    long long oa, ob;
    nd_off<FAST>(g, i, oa, ob);
    neumaier(s, c, A[oa] * B[ob]);
  }
  __shared__ double sh_s[DOT_THREADS], sh_c[DOT_THREADS];
  __shared__ bool last;
  sh_s[threadIdx.x] = s;
  sh_c[threadIdx.x] = c;
  __syncthreads();
  dot_tree(sh_s, sh_c);
  const unsigned ncta = gridDim.x * gridDim.y, me = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
    partial[2 * me] = sh_s[0];
    partial[2 * me + 1] = sh_c[0];
    __threadfence();
    last = atomicAdd(ticket, 1u) == ncta - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  s = 0.0;
  c = 0.0;
  for (unsigned i = threadIdx.x; i < ncta; i += DOT_THREADS) {
    neumaier(s, c, __ldcg(partial + 2 * i));
    c += __ldcg(partial + 2 * i + 1);
  }
  sh_s[threadIdx.x] = s;
  sh_c[threadIdx.x] = c;
  __syncthreads();
  dot_tree(sh_s, sh_c);
  if (threadIdx.x == 0) {
    *out = alpha * (sh_s[0] + sh_c[0]);
    *ticket = 0u;
  }
}

// Final reduction of the energy components: out[c] = sum of slots
// [r[c], r[c+1]) for c = 0, 1, 2, each in a fixed order with a double-double
// running sum (Knuth's two-sum), one thread per component.
__global__ void k_sum_slots(const double* __restrict__ slots, int r0, int r1, int r2, int r3, int r4,
                            double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= 3) return;
  const int lo = c == 0 ? r0 : c == 1 ? r2 : r3;
  const int hi = c == 0 ? r1 : c == 1 ? r3 : r4;
  double s = 0.0, e = 0.0;
  for (int i = lo; i < hi; ++i) {
    const double x = slots[i];
    const double t = s + x;
    const double bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
  }
  out[c] = s + e;
}

__global__ void k_add_diagonal(double* D, int n, double v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) D[(long long)i * n + i] += v;
}

__global__ void k_fill(double* p, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

// ---------------------------------------------------------------------------
// regulariser (1 - exp(-s D^2)) / D, limit 0 at D = 0 (Eqs. T1_1st, T2_1st)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double regulariser(double s, double D) {
  double x = s * D * D;
  if (x < 1e-12) return s * D * (1.0 - 0.5 * x);
  return -expm1(-x) / D;
}

// One thread per spatial (a, b, i, j): D and R(D) once, then every stored
// spin block (sa, sb, si, sj) of the [P,P,H,H] arrays (block bits sa | sb<<1 |
// si<<2 | sj<<3, offsets lay.boff, spatial strides lay.st; the three arrays
// share the layout).  Consecutive threads take consecutive j.
__global__ void k_amp2(int nc, int na, int nv, double s, const double* __restrict__ eps,
                       const double* __restrict__ O2, double* __restrict__ T2, double* __restrict__ W2,
                       const Amp2Layout lay) {
  const int h = nc + na, p = na + nv;
  const unsigned hh = (unsigned)h * h, total = (unsigned)p * p * hh;
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const unsigned ab = idx / hh, ij = idx - ab * hh;
    const int a = (int)(ab / p), b = (int)(ab - (unsigned)a * p);
    const int i = (int)(ij / h), j = (int)(ij - (unsigned)i * h);
    const bool internal = (i >= nc) && (j >= nc) && (a < na) && (b < na);
    const double D = eps[i] + eps[j] - eps[nc + a] - eps[nc + b];
    const double R = internal ? 0.0 : regulariser(s, D);
    const long long sp0 = a * lay.st[0] + b * lay.st[1] + i * lay.st[2] + j * lay.st[3];
#pragma unroll
    for (int bits = 0; bits < 16; ++bits) {
      const long long bo = lay.boff[bits];
      if (bo < 0) continue;
      const long long o = bo + sp0;
      const int sa = bits & 1, sb = bits >> 1 & 1, si = bits >> 2 & 1, sj = bits >> 3 & 1;
      double t = 0.0;
      if (sa + sb == si + sj) t = O2[o] * R;
      T2[o] = t;
      if (W2) W2[o] = -D * t;
    }
  }
}

__global__ void k_amp1(int nc, int na, int nv, double s, const double* __restrict__ eps,
                       const double* __restrict__ O1, const double* __restrict__ S, double* __restrict__ T1,
                       double* __restrict__ W1) {
  const int h = nc + na, p = na + nv;
  const int total = 4 * p * h;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int i = idx % (2 * h), a = idx / (2 * h);
    int ia = i % h, aa = a % p;
    bool same_spin = (i / h) == (a / p);
    bool internal = (ia >= nc) && (aa < na);
    double D = eps[ia] - eps[nc + aa];
    double src = S ? S[idx] : 0.0;
    double o = O1 ? O1[idx] : 0.0;
    double t = (internal || !same_spin) ? 0.0 : (o + src) * regulariser(s, D);
    T1[idx] = t;
    if (W1) W1[idx] = (internal || !same_spin) ? 0.0 : -D * t + src;
  }
}

__global__ void k_gamma_eta(int nc, int na, int nv, const double* __restrict__ g1a, const double* __restrict__ g1b,
                            double* __restrict__ gamma, double* __restrict__ eta) {
  const int h = nc + na, p = na + nv;
  const int nG = 4 * h * h, nE = 4 * p * p;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nG + nE; idx += gridDim.x * blockDim.x) {
    if (idx < nG) {
      int c2 = idx % (2 * h), r2 = idx / (2 * h);
      int sr = r2 / h, sc = c2 / h, r = r2 % h, c = c2 % h;
      double v = 0.0;
      if (sr == sc) {
        if (r < nc || c < nc) v = (r == c) ? 1.0 : 0.0;
        else v = (sr == 0 ? g1a : g1b)[(r - nc) * na + (c - nc)];
      }
      gamma[idx] = v;
    } else {
      int k = idx - nG;
      int c2 = k % (2 * p), r2 = k / (2 * p);
      int sr = r2 / p, sc = c2 / p, r = r2 % p, c = c2 % p;
      double v = 0.0;
      if (sr == sc) {
        if (r >= na || c >= na) v = (r == c) ? 1.0 : 0.0;
        else v = (r == c ? 1.0 : 0.0) - (sr == 0 ? g1a : g1b)[r * na + c];
      }
      eta[k] = v;
    }
  }
}

struct BlkPtrs {
  const double* b[4];
};

__global__ void k_cumulant(int na, int rank, BlkPtrs blk, double* __restrict__ out) {
  const int A2 = 2 * na;
  long long total = 1;
  for (int k = 0; k < 2 * rank; ++k) total *= A2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int sp[6], x[6];
    long long r = idx;
    for (int k = 2 * rank - 1; k >= 0; --k) {
      int v = (int)(r % A2);
      r /= A2;
      sp[k] = v / na;
      x[k] = v % na;
    }
    int nbc = 0, nba = 0;
    for (int k = 0; k < rank; ++k) {
      nbc += sp[k];
      nba += sp[rank + k];
    }
    double v = 0.0;
    if (nbc == nba) {
      // stable sort creators and annihilators: alpha first; sign of each permutation
      int pc[3], pa[3], nc_ = 0, na_ = 0;
      for (int s = 0; s < 2; ++s)
        for (int k = 0; k < rank; ++k) {
          if (sp[k] == s) pc[nc_++] = k;
          if (sp[rank + k] == s) pa[na_++] = k;
        }
      int inv = 0;
      for (int i = 0; i < rank; ++i)
        for (int j = i + 1; j < rank; ++j) {
          if (pc[i] > pc[j]) ++inv;
          if (pa[i] > pa[j]) ++inv;
        }
      long long off = 0;
      for (int k = 0; k < rank; ++k) off = off * na + x[pc[k]];
      for (int k = 0; k < rank; ++k) off = off * na + x[rank + pa[k]];
      v = blk.b[nbc][off];
      if (inv & 1) v = -v;
    }
    out[idx] = v;
  }
}

__global__ void k_gamma_delta(int nc, int na, const double* __restrict__ eps, const double* __restrict__ gH,
                              int h, double* __restrict__ G) {
  const int A2 = 2 * na;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < A2 * A2; idx += gridDim.x * blockDim.x) {
    int u2 = idx % A2, x2 = idx / A2;
    int sx = x2 / na, su = u2 / na, x = x2 % na, u = u2 % na;
    double g = gH[(long long)(sx * h + nc + x) * (2 * h) + (su * h + nc + u)];
    G[idx] = g * (eps[nc + x] - eps[nc + u]);
  }
}

inline int grid_for(long long n, int threads, int cap = 152 * 16) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}
}  // namespace

void gemm_tile(long long M, long long N, int* bm, int* bn) {
  if (N <= 16) { *bm = 256; *bn = 16; }
  else if (M <= 16) { *bm = 16; *bn = 256; }
  else if (N <= 32) { *bm = 128; *bn = 32; }
  else if (M <= 32) { *bm = 32; *bn = 128; }
  else { *bm = 64; *bn = 64; }
}

bool gemm_is_small(const GemmArgs& g) { return g.M * g.N * g.nbatch <= 4096 && g.K < (1LL << 31); }

bool gemm_is_short(const GemmArgs& g) {
  return g.K <= TPO_KMAX && g.M < (1LL << 31) && g.N < (1LL << 31) && !gemm_is_small(g);
}

bool gemm_use_flat(const GemmArgs& g) {
  const long long O = g.M * g.N * g.nbatch;
  if (O >= (1LL << 31) || g.K >= (1LL << 31) || g.M >= (1LL << 31) || g.N >= (1LL << 31)) return false;
  // full-size tiles with enough of them keep the register-blocked kernel
  const long long tiles = ((g.M + 63) / 64) * ((g.N + 63) / 64) * g.nbatch;
  return !(g.M >= 64 && g.N >= 64 && g.K > 64 && tiles >= 2 * 152);
}

FlatPlan gemm_flat_plan(const GemmArgs& g, int groups) {
  FlatPlan p{};
  const long long O = g.M * g.N * g.nbatch * (groups > 1 ? groups : 1);
  // about 32 resident warps per SM: enough FMAs in flight to cover latency
  const long long target = 152LL * 1024;
  long long chunks = (target + O - 1) / O;
  const long long maxc = g.K / 16 > 1 ? g.K / 16 : 1;  // at least 16 k per chunk
  if (chunks > maxc) chunks = maxc;
  if (chunks < 1) chunks = 1;
  p.wk = chunks >= 8 ? 8 : chunks >= 4 ? 4 : chunks >= 2 ? 2 : 1;
  long long z = (chunks + p.wk - 1) / p.wk;
  if (z > 65535) z = 65535;
  p.len = (g.K + p.wk * z - 1) / (p.wk * z);
  p.z = (int)((g.K + p.len * p.wk - 1) / (p.len * p.wk));
  // lanes walk the output index whose operand stride is smallest
  const long long sm = g.nM ? (g.aM[g.nM - 1] < g.cM[g.nM - 1] ? g.aM[g.nM - 1] : g.cM[g.nM - 1]) : (1LL << 62);
  const long long sn = g.nN ? (g.bN[g.nN - 1] < g.cN[g.nN - 1] ? g.bN[g.nN - 1] : g.cN[g.nN - 1]) : (1LL << 62);
  p.mfast = sm < sn ? 1 : 0;
  return p;
}

void launch_gemm_flat(const GemmArgs& g, const FlatPlan& p, const FlatTable& tab, double* part, cudaStream_t st) {
  const long long O = g.M * g.N * g.nbatch;
  if (O <= 0 || g.K <= 0 || tab.ngroups <= 0) return;
  FlatK fk{};
  const int pad = 4 - g.nK;
  for (int d = 0; d < 4; ++d) {
    const int s = d - pad;
    fk.e[d] = s >= 0 ? g.eK[s] : 1;
    fk.a[d] = s >= 0 ? g.aK[s] : 0;
    fk.b[d] = s >= 0 ? g.bK[s] : 0;
  }
  for (int d = 1; d < 4; ++d) {
    fk.wa[d] = fk.a[d - 1] - (long long)fk.e[d] * fk.a[d];
    fk.wb[d] = fk.b[d - 1] - (long long)fk.e[d] * fk.b[d];
  }
  for (int d = 0; d < 4; ++d) {
    fk.fk[d] = make_fastdiv((unsigned)fk.e[d]);
    fk.fm[d] = make_fastdiv(d < g.nM ? (unsigned)g.eM[d] : 1u);
    fk.fn[d] = make_fastdiv(d < g.nN ? (unsigned)g.eN[d] : 1u);
    fk.fb[d] = make_fastdiv(d < g.nB ? (unsigned)g.eB[d] : 1u);
  }
  fk.fM = make_fastdiv((unsigned)g.M);
  fk.fN = make_fastdiv((unsigned)g.N);
  const long long per_cta = 32LL * (8 / p.wk);
  dim3 grid((unsigned)((O + per_cta - 1) / per_cta), (unsigned)p.z, (unsigned)tab.ngroups);
  switch (p.wk) {
    case 8: k_gemm_flat<8><<<grid, 256, 0, st>>>(g, fk, tab, O, p.mfast, p.len, part); break;
    case 4: k_gemm_flat<4><<<grid, 256, 0, st>>>(g, fk, tab, O, p.mfast, p.len, part); break;
    case 2: k_gemm_flat<2><<<grid, 256, 0, st>>>(g, fk, tab, O, p.mfast, p.len, part); break;
    default: k_gemm_flat<1><<<grid, 256, 0, st>>>(g, fk, tab, O, p.mfast, p.len, part); break;
  }
  if (p.z > 1) {
    const dim3 rg((unsigned)grid_for(O, 256, (152 * 16 + tab.ngroups - 1) / tab.ngroups), (unsigned)tab.ngroups);
    k_gemm_flat_reduce<<<rg, 256, 0, st>>>(g, fk, tab, O, p.mfast, p.z, part);
  }
}

void launch_gemm(const GemmArgs& g, cudaStream_t st, int kind) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.nbatch <= 0) return;
  int bm, bn;
  gemm_tile(g.M, g.N, &bm, &bn);
  if (kind != 0) { bm = 64; bn = 64; }
  dim3 grid((unsigned)((g.M + bm - 1) / bm), (unsigned)((g.N + bn - 1) / bn),
            (unsigned)(g.splits > 1 ? g.splits : g.nbatch));
  if (kind == 0 && gemm_is_small(g)) {
    dim3 sg((unsigned)(g.M * g.N * g.nbatch), (unsigned)(g.splits > 1 ? g.splits : 1));
    k_gemm_small<<<sg, SMALL_T, 0, st>>>(g);
    if (g.splits > 1) k_gemm_splitk_reduce<<<grid_for(g.M * g.N, 256), 256, 0, st>>>(g);
    return;
  }
  if (kind == 0 && gemm_is_short(g)) {
    // consecutive threads walk the output index whose operand stride is smallest
    long long sm = g.nM ? (g.aM[g.nM - 1] < g.cM[g.nM - 1] ? g.aM[g.nM - 1] : g.cM[g.nM - 1]) : (1LL << 62);
    long long sn = g.nN ? (g.bN[g.nN - 1] < g.cN[g.nN - 1] ? g.bN[g.nN - 1] : g.cN[g.nN - 1]) : (1LL << 62);
    k_gemm_tpo<<<grid_for(g.M * g.N * g.nbatch, TPO_T, 152 * 32), TPO_T, 0, st>>>(g, sm < sn ? 1 : 0);
    return;
  }
  if (kind == 1) k_gemm<64, 64, 1><<<grid, NT, 0, st>>>(g);        // (pr|qs) build from B
  else if (kind == 2) k_gemm<64, 64, 2><<<grid, NT, 0, st>>>(g);   // ladder contraction with T2
  else if (bn == 16) k_gemm<256, 16, 0><<<grid, NT, 0, st>>>(g);    // narrow outputs
  else if (bm == 16) k_gemm<16, 256, 0><<<grid, NT, 0, st>>>(g);
  else if (bn == 32) k_gemm<128, 32, 0><<<grid, NT, 0, st>>>(g);
  else if (bm == 32) k_gemm<32, 128, 0><<<grid, NT, 0, st>>>(g);
  else k_gemm<64, 64, 0><<<grid, NT, 0, st>>>(g);                   // every other contraction
  if (g.splits > 1) k_gemm_splitk_reduce<<<grid_for(g.M * g.N, 256), 256, 0, st>>>(g);
}

namespace {
// Consecutive threads take consecutive linear indices, whose last dimension
// runs fastest.  The dimensions are put in order of decreasing stride,
// weighted wb for the second operand (the one written, for axpy), so that
// the last one is the label with the smallest strides: stride 1 in both
// operands when they share a contiguous label.  In the order the labels
// were written, a permuted view (a transposed two-body class, the Hermitian
// placement of W) put a stride of 10^3 - 10^5 elements on the fastest
// dimension, and every 8-byte access then fetched its own DRAM sectors.
// Only the order of the visits changes; the set of (A, B) element pairs is
// the same.
void nd_order(NdArgs& g, long long wb) {
  int ord[kMaxDims];
  for (int d = 0; d < g.nd; ++d) ord[d] = d;
  std::stable_sort(ord, ord + g.nd, [&](int x, int y) {
    return g.sa[x] + wb * g.sb[x] > g.sa[y] + wb * g.sb[y];
  });
  const NdArgs h = g;
  for (int d = 0; d < g.nd; ++d) {
    g.e[d] = h.e[ord[d]];
    g.sa[d] = h.sa[ord[d]];
    g.sb[d] = h.sb[ord[d]];
  }
}

// orders the dimensions and fills the fast divisors; true when every linear
// index fits 31 bits
bool nd_prepare(NdArgs& g, long long wb) {
  nd_order(g, wb);
  if (g.total >= (1LL << 31)) return false;
  for (int d = 0; d < g.nd; ++d) g.fe[d] = make_fastdiv((unsigned)g.e[d]);
  return true;
}
}  // namespace

void launch_axpy(const NdArgs& g0, double alpha, const double* A, double* C, cudaStream_t st) {
  if (g0.total <= 0) return;
  NdArgs g = g0;
  if (nd_prepare(g, 2)) k_axpy<true><<<grid_for(g.total, 256), 256, 0, st>>>(g, alpha, A, C);
  else k_axpy<false><<<grid_for(g.total, 256), 256, 0, st>>>(g, alpha, A, C);
}

void launch_axpy_blocks(const NdArgs& g0, double alpha, const AxpyBlocks& p, cudaStream_t st) {
  if (g0.total <= 0 || p.n <= 0) return;
  NdArgs g = g0;
  const int gx = grid_for(g.total, 256, (152 * 16 + p.n - 1) / p.n);
  const dim3 grid((unsigned)gx, (unsigned)p.n);
  if (nd_prepare(g, 2)) k_axpy_blocks<true><<<grid, 256, 0, st>>>(g, alpha, p);
  else k_axpy_blocks<false><<<grid, 256, 0, st>>>(g, alpha, p);
}

void launch_dot_blocks(const NdArgs& g0, double alpha, const DotBlocks& p, double* scratch, int scratch_len,
                       unsigned* ticket, double* out, cudaStream_t st) {
  if (p.n <= 0) return;
  NdArgs g = g0;
  int cap = scratch_len / 2 / p.n;
  if (cap < 1) throw std::runtime_error("dot: scratch too small for the spin blocks");
  const int gx = grid_for(g.total > 0 ? g.total : 1, DOT_THREADS, cap);
  const dim3 grid((unsigned)gx, (unsigned)p.n);
  if (nd_prepare(g, 1)) k_dot_blocks<true><<<grid, DOT_THREADS, 0, st>>>(g, p, scratch, ticket, alpha, out);
  else k_dot_blocks<false><<<grid, DOT_THREADS, 0, st>>>(g, p, scratch, ticket, alpha, out);
}

void launch_sum_slots(const double* slots, const int* r, double* out, cudaStream_t st) {
  k_sum_slots<<<1, 32, 0, st>>>(slots, r[0], r[1], r[2], r[3], r[4], out);
}

void launch_add_diagonal(double* D, int n, double v, cudaStream_t st) {
  if (n <= 0) return;
  k_add_diagonal<<<1, 256, 0, st>>>(D, n, v);
}

void launch_fill(double* p, long long n, double v, cudaStream_t st) {
  if (n <= 0) return;
  k_fill<<<grid_for(n, 256), 256, 0, st>>>(p, n, v);
}

void launch_build_gamma_eta(int nc, int na, int nv, const double* g1a, const double* g1b, double* gamma,
                            double* eta, cudaStream_t st) {
  int h = nc + na, p = na + nv;
  long long n = 4LL * h * h + 4LL * p * p;
  k_gamma_eta<<<grid_for(n, 256), 256, 0, st>>>(nc, na, nv, g1a, g1b, gamma, eta);
}

void launch_build_cumulant(int na, int rank, const double* const* blk_dev, double* out, cudaStream_t st) {
  BlkPtrs b{};
  for (int k = 0; k <= rank && k < 4; ++k) b.b[k] = blk_dev[k];
  long long total = 1;
  for (int k = 0; k < 2 * rank; ++k) total *= 2 * na;
  k_cumulant<<<grid_for(total, 256), 256, 0, st>>>(na, rank, b, out);
}

void launch_amp2(int nc, int na, int nv, double s, const double* eps, const double* O2, double* T2, double* W2,
                 const Amp2Layout& lay, cudaStream_t st) {
  long long h = nc + na, p = na + nv;
  long long n = p * p * h * h;  // spatial quadruples, one thread each
  if (n >= (1LL << 32)) throw std::runtime_error("amplitudes: p^2 h^2 must stay below 2^32");
  k_amp2<<<grid_for(n, 256), 256, 0, st>>>(nc, na, nv, s, eps, O2, T2, W2, lay);
}

void launch_amp1(int nc, int na, int nv, double s, const double* eps, const double* O1, const double* S,
                 double* T1, double* W1, cudaStream_t st) {
  long long n = 4LL * (na + nv) * (nc + na);
  k_amp1<<<grid_for(n, 256), 256, 0, st>>>(nc, na, nv, s, eps, O1, S, T1, W1);
}

void launch_gamma_delta(int nc, int na, const double* eps, const double* gamma_H, int h, double* G,
                        cudaStream_t st) {
  if (na == 0) return;
  k_gamma_delta<<<grid_for(4LL * na * na, 256), 256, 0, st>>>(nc, na, eps, gamma_H, h, G);
}

}  // namespace dsrg

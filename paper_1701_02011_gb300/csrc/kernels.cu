// Device kernels of the DSRG-MRPT2/PT3 energy path (sm_103a), FP64.
#include "kernels.cuh"

#include <cmath>

namespace dsrg {

// ---------------------------------------------------------------------------
// generic strided contraction
// ---------------------------------------------------------------------------
// One CTA computes a 64 x 64 tile of C with 256 threads (4 x 4 outputs each),
// stepping K by 16.  Operand addresses are separable: off(A[m,k]) =
// offA(m) + offA(k), so the tile's row/column/k offsets are decoded once
// into shared memory and the inner loop is a plain tiled GEMM.
namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

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

__global__ void k_axpy(const NdArgs g, double alpha, const double* __restrict__ A, double* __restrict__ C) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    long long oa, oc;
    nd_offsets(g, i, oa, oc);
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

__global__ void __launch_bounds__(DOT_THREADS) k_dot_partial(const NdArgs g, const double* __restrict__ A,
                                                            const double* __restrict__ B, double* partial) {
  double s = 0.0, c = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.total;
       i += (long long)gridDim.x * blockDim.x) {
    long long oa, ob;
    nd_offsets(g, i, oa, ob);
    neumaier(s, c, A[oa] * B[ob]);
  }
  __shared__ double sh_s[DOT_THREADS], sh_c[DOT_THREADS];
  sh_s[threadIdx.x] = s;
  sh_c[threadIdx.x] = c;
  __syncthreads();
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
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sh_s[0];
    partial[2 * blockIdx.x + 1] = sh_c[0];
  }
}

__global__ void __launch_bounds__(DOT_THREADS) k_dot_final(const double* partial, int nblk, double alpha,
                                                          double* out) {
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nblk; i += DOT_THREADS) {
    neumaier(s, c, partial[2 * i]);
    c += partial[2 * i + 1];
  }
  __shared__ double sh_s[DOT_THREADS], sh_c[DOT_THREADS];
  sh_s[threadIdx.x] = s;
  sh_c[threadIdx.x] = c;
  __syncthreads();
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
  if (threadIdx.x == 0) *out = alpha * (sh_s[0] + sh_c[0]);
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

__global__ void k_amp2(int nc, int na, int nv, double s, const double* __restrict__ eps,
                       const double* __restrict__ O2, double* __restrict__ T2, double* __restrict__ W2) {
  const int h = nc + na, p = na + nv;
  const long long P2 = 2LL * p, H2 = 2LL * h;
  const long long total = P2 * P2 * H2 * H2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx;
    int j = (int)(r % H2); r /= H2;
    int i = (int)(r % H2); r /= H2;
    int b = (int)(r % P2); r /= P2;
    int a = (int)r;
    int ja = j % h, ia = i % h, bb = b % p, aa = a % p;
    bool internal = (ja >= nc) && (ia >= nc) && (bb < na) && (aa < na);
    double D = eps[ia] + eps[ja] - eps[nc + aa] - eps[nc + bb];
    double t = internal ? 0.0 : O2[idx] * regulariser(s, D);
    T2[idx] = t;
    if (W2) W2[idx] = -D * t;
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

void launch_axpy(const NdArgs& g, double alpha, const double* A, double* C, cudaStream_t st) {
  if (g.total <= 0) return;
  k_axpy<<<grid_for(g.total, 256), 256, 0, st>>>(g, alpha, A, C);
}

void launch_dot(const NdArgs& g, double alpha, const double* A, const double* B, double* scratch,
                int scratch_len, double* out_slot, cudaStream_t st) {
  int nblk = grid_for(g.total, DOT_THREADS, scratch_len / 2);
  k_dot_partial<<<nblk, DOT_THREADS, 0, st>>>(g, A, B, scratch);
  k_dot_final<<<1, DOT_THREADS, 0, st>>>(scratch, nblk, alpha, out_slot);
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
                 cudaStream_t st) {
  long long h = nc + na, p = na + nv;
  long long n = 16 * p * p * h * h;
  k_amp2<<<grid_for(n, 256), 256, 0, st>>>(nc, na, nv, s, eps, O2, T2, W2);
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

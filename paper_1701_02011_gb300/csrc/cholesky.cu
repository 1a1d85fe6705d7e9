// Pivoted incomplete Cholesky factorisation of a two-electron supermatrix on
// the GPU: the three-index factor of Eq. int_fact, (pq|rs) ~ sum_Q B^Q_pq
// B^Q_rs, obtained by Cholesky decomposition with a threshold as for the
// paper's larger applications (Sec. IV, thresholds 1e-6 and 1e-8 a.u.).
// Algorithm of Beebe and Linderberg (1977) as described by Koch, Sanchez de
// Meras and Pedersen (J. Chem. Phys. 118, 9481 (2003)): at step Q the pivot J
// is the largest remaining diagonal D[J] (the smallest index on ties); the
// factorisation stops when D[J] <= tau; the vector is
//   B[Q][i] = (V[J][i] - sum_{Q' < Q} B[Q'][i] B[Q'][J]) / sqrt(D[J])
// and D[i] -= B[Q][i]^2.  Corrections are summed over Q' in increasing order
// with one rounding per product and per sum (no fused multiply-add), so the
// result is reproducible operation by operation.
#include <cmath>
#include <string>

#include "../../include/dsrg.h"
#include "ladder.cuh"

namespace {

constexpr int CH_T = 256;
constexpr int CH_MAX_CTAS = 152 * 4;

struct ChState {
  long long J;     // pivot of the vector being formed
  double dJ;       // its remaining diagonal
  int nvec;        // vectors completed
  int done;        // 1: stopped (threshold or max_vecs)
  unsigned ticket; // CTAs finished in the current launch
};

// (value, index) order of the pivot search: larger value first, then the
// smaller index; NaN never wins
__device__ __forceinline__ bool better(double v, long long i, double bv, long long bi) {
  return v > bv || (v == bv && i < bi);
}

// in-CTA reduction of (value, index) pairs; result in v[0], ix[0]
__device__ void cta_argmax(double* v, long long* ix) {
  for (int w = CH_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w && better(v[threadIdx.x + w], ix[threadIdx.x + w], v[threadIdx.x], ix[threadIdx.x])) {
      v[threadIdx.x] = v[threadIdx.x + w];
      ix[threadIdx.x] = ix[threadIdx.x + w];
    }
    __syncthreads();
  }
}

// The CTA that finishes last combines the per-CTA maxima (fixed order) and
// sets the next pivot, or stops.  finish: the vector of this launch is done.
__device__ void last_cta_pivot(double bv, long long bi, double* pv, long long* pi, ChState* st, double tau,
                               int max_vecs, long long* piv, bool finish) {
  __shared__ double sv[CH_T];
  __shared__ long long si[CH_T];
  __shared__ bool last;
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  cta_argmax(sv, si);
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
    __threadfence();
    last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = -INFINITY;
  long long i = -1;
  for (unsigned c = threadIdx.x; c < gridDim.x; c += CH_T) {
    const double cv = __ldcg(pv + c);
    const long long ci = __ldcg(pi + c);
    if (better(cv, ci, v, i)) {
      v = cv;
      i = ci;
    }
  }
  sv[threadIdx.x] = v;
  si[threadIdx.x] = i;
  __syncthreads();
  cta_argmax(sv, si);
  if (threadIdx.x == 0) {
    if (finish) st->nvec += 1;
    if (!(sv[0] > tau) || si[0] < 0 || st->nvec >= max_vecs) {
      st->done = 1;
    } else {
      st->J = si[0];
      st->dJ = sv[0];
      piv[st->nvec] = si[0];
    }
    st->ticket = 0u;
  }
}

// D = diag(V) and the first pivot
__global__ void __launch_bounds__(CH_T) k_chol_init(const double* __restrict__ V, long long N, double* __restrict__ D,
                                                   double* pv, long long* pi, ChState* st, double tau, int max_vecs,
                                                   long long* piv) {
  double bv = -INFINITY;
  long long bi = -1;
  for (long long i = blockIdx.x * (long long)CH_T + threadIdx.x; i < N; i += (long long)gridDim.x * CH_T) {
    const double d = V[i * N + i];
    D[i] = d;
    if (better(d, i, bv, bi)) {
      bv = d;
      bi = i;
    }
  }
  last_cta_pivot(bv, bi, pv, pi, st, tau, max_vecs, piv, false);
}

// one vector: B[nvec][i], D[i] -= B[nvec][i]^2, and the next pivot
__global__ void __launch_bounds__(CH_T) k_chol_step(const double* __restrict__ V, long long N, double* __restrict__ B,
                                                   double* __restrict__ D, double* pv, long long* pi, ChState* st,
                                                   double tau, int max_vecs, long long* piv) {
  if (st->done) return;
  const long long J = st->J;
  const int Q = st->nvec;
  const double sq = sqrt(st->dJ);
  const double* __restrict__ bJ = B + J;  // B[q][J] at bJ[q * N]
  double bv = -INFINITY;
  long long bi = -1;
  for (long long i = blockIdx.x * (long long)CH_T + threadIdx.x; i < N; i += (long long)gridDim.x * CH_T) {
    // the products of 16 vectors are loaded and formed ahead of their
    // (sequential, increasing-q) additions, so many loads are in flight
    double acc = 0.0;
    int q = 0;
    for (; q + 16 <= Q; q += 16) {
      double pr[16];
#pragma unroll
      for (int u = 0; u < 16; ++u)
        pr[u] = __dmul_rn(__ldg(B + (long long)(q + u) * N + i), __ldg(bJ + (long long)(q + u) * N));
#pragma unroll
      for (int u = 0; u < 16; ++u) acc = __dadd_rn(acc, pr[u]);
    }
    for (; q < Q; ++q) acc = __dadd_rn(acc, __dmul_rn(__ldg(B + (long long)q * N + i), __ldg(bJ + (long long)q * N)));
    const double L = __ddiv_rn(__dsub_rn(V[J * N + i], acc), sq);
    B[(long long)Q * N + i] = L;
    const double d = __dsub_rn(D[i], __dmul_rn(L, L));
    D[i] = d;
    if (better(d, i, bv, bi)) {
      bv = d;
      bi = i;
    }
  }
  last_cta_pivot(bv, bi, pv, pi, st, tau, max_vecs, piv, true);
}

inline int ch_grid(long long N) {
  long long g = (N + CH_T - 1) / CH_T;
  if (g < 1) g = 1;
  if (g > CH_MAX_CTAS) g = CH_MAX_CTAS;
  return (int)g;
}

}  // namespace

extern "C" int dsrg_cholesky(long long N, const double* V, double tau, int max_vecs, double* B, int* nvecs,
                             long long* pivots, void* stream) {
  using namespace dsrg;
  if (nvecs) *nvecs = 0;
  if (N < 0 || max_vecs < 0 || !(tau >= 0.0) || !nvecs) return set_error(DSRG_ERR_ARG, "cholesky: need N >= 0, max_vecs >= 0, tau >= 0, nvecs");
  if (N == 0 || max_vecs == 0) return DSRG_OK;
  if (!V || !B) return set_error(DSRG_ERR_ARG, "cholesky: V and B must be device pointers");
  if (N > (1LL << 40) / N) return set_error(DSRG_ERR_ARG, "cholesky: N too large");
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = ch_grid(N);
  // scratch: D [N], per-CTA maxima, pivots [max_vecs], state
  double* D = nullptr;
  const size_t bytes = (size_t)N * 8 + (size_t)grid * 16 + (size_t)max_vecs * 8 + sizeof(ChState) + 64;
  cudaError_t e = cudaMalloc(&D, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(DSRG_ERR_OOM, (std::string("cholesky scratch: ") + cudaGetErrorString(e)).c_str());
  }
  double* pv = D + N;
  long long* pi = reinterpret_cast<long long*>(pv + grid);
  long long* piv = pi + grid;
  ChState* cs = reinterpret_cast<ChState*>(piv + max_vecs);
  int rc = DSRG_OK;
  try {
    check_cuda(cudaMemsetAsync(cs, 0, sizeof(ChState), st), "cudaMemsetAsync (cholesky)");
    k_chol_init<<<grid, CH_T, 0, st>>>(V, N, D, pv, pi, cs, tau, max_vecs, piv);
    check_cuda(cudaGetLastError(), "cholesky launch");
    ChState h{};
    for (int q = 0; q < max_vecs; ++q) {
      k_chol_step<<<grid, CH_T, 0, st>>>(V, N, B, D, pv, pi, cs, tau, max_vecs, piv);
      check_cuda(cudaGetLastError(), "cholesky launch");
      // every 32 vectors: stop launching once the factorisation has stopped
      if ((q & 31) == 31 || q == max_vecs - 1) {
        check_cuda(cudaMemcpyAsync(&h, cs, sizeof h, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync (cholesky)");
        check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize (cholesky)");
        if (h.done) break;
      }
    }
    check_cuda(cudaMemcpyAsync(&h, cs, sizeof h, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync (cholesky)");
    check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize (cholesky)");
    *nvecs = h.nvec;
    if (pivots && h.nvec > 0)
      check_cuda(cudaMemcpy(pivots, piv, (size_t)h.nvec * sizeof(long long), cudaMemcpyDeviceToHost),
                 "cudaMemcpy (pivots)");
  } catch (const Error& ex) {
    rc = set_error(ex.code, ex.what());
  } catch (const std::exception& ex) {
    rc = set_error(DSRG_ERR_INTERNAL, ex.what());
  }
  cudaFree(D);
  return rc;
}

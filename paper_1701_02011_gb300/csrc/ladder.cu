// Density-fitted particle-particle ladder (paper Eq. scaling_problem with the
// factorised integrals of Eq. int_fact), usable on caller buffers.
#include <stdexcept>
#include <string>

#include "../../include/dsrg.h"
#include "ladder.cuh"

namespace dsrg {

void ladder_core(const double* B, long long n, int naux, int p0, int np, int nh, const double* t,
                 const long long* tst, double* L, double* G, long long bp, cudaStream_t st, Workspace* ws) {
  if (np <= 0 || nh <= 0) return;
  const long long p3 = (long long)np * np * np;
  for (long long r0 = 0; r0 < np; r0 += bp) {
    long long nb = (np - r0 < bp) ? np - r0 : bp;
    check_cuda(cudaMemsetAsync(G, 0, (size_t)(nb * p3) * sizeof(double), st), "cudaMemsetAsync (ladder)");
    {  // G[pp,q,r,s] = sum_Q B[Q, p0+r0+pp, p0+r] B[Q, p0+q, p0+s]
      GemmArgs g{};
      g.A = B + (p0 + r0) * n + p0;
      g.B = B + (long long)p0 * n + p0;
      g.C = G;
      g.alpha = 1.0;
      g.nM = 2;
      g.eM[0] = (int)nb; g.aM[0] = n; g.cM[0] = p3;
      g.eM[1] = np;      g.aM[1] = 1; g.cM[1] = np;
      g.nN = 2;
      g.eN[0] = np; g.bN[0] = n; g.cN[0] = (long long)np * np;
      g.eN[1] = np; g.bN[1] = 1; g.cN[1] = 1;
      g.nK = 1;
      g.eK[0] = naux; g.aK[0] = n * n; g.bK[0] = n * n;
      g.M = nb * np;
      g.N = (long long)np * np;
      g.K = naux;
      g.nbatch = 1;
      if (ws) run_gemm(*ws, g, K_LADDER_BUILD);
      else launch_gemm(g, st, 1);
    }
    {  // L[r0+pp,q,i,j] += sum_{r,s} G[pp,q,r,s] t[r,s,i,j]
      GemmArgs g{};
      g.A = G;
      g.B = t;
      g.C = L + r0 * (long long)np * nh * nh;
      g.alpha = 1.0;
      g.nM = 2;
      g.eM[0] = (int)nb; g.aM[0] = p3;                 g.cM[0] = (long long)np * nh * nh;
      g.eM[1] = np;      g.aM[1] = (long long)np * np; g.cM[1] = (long long)nh * nh;
      g.nK = 2;
      g.eK[0] = np; g.aK[0] = np; g.bK[0] = tst[0];
      g.eK[1] = np; g.aK[1] = 1;  g.bK[1] = tst[1];
      g.nN = 2;
      g.eN[0] = nh; g.bN[0] = tst[2]; g.cN[0] = nh;
      g.eN[1] = nh; g.bN[1] = tst[3]; g.cN[1] = 1;
      g.M = nb * np;
      g.N = (long long)nh * nh;
      g.K = (long long)np * np;
      g.nbatch = 1;
      if (ws) run_gemm(*ws, g, K_LADDER_CONTRACT);
      else launch_gemm(g, st, 2);
    }
  }
}

// Pair-symmetric variant: with t[r,s,i,j] = t[s,r,j,i] (the alpha-beta block
// of a spin-free T2) and (pr|qs) = (qs|pr), L[q,p,i,j] = L[p,q,j,i], so a
// batch of rows p in [e0, e1) builds and contracts (pr|qs) only for
// q >= e0 and writes the rows q >= e1 of the mirror image by a transposed
// copy.  About half of the build and contraction work of ladder_core.
void ladder_core_sym(const double* B, long long n, int naux, int p0, int np, int nh, const double* t,
                     const long long* tst, double* L, double* G, long long max_doubles, cudaStream_t st,
                     Workspace* ws) {
  if (np <= 0 || nh <= 0) return;
  const long long p2 = (long long)np * np, h2 = (long long)nh * nh;
  if (max_doubles < np * p2) throw std::runtime_error("ladder: scratch below one row of (pr|qs)");
  long long e0 = 0;
  while (e0 < np) {
    const long long nf = np - e0;  // q in [e0, np)
    long long nb = max_doubles / (nf * p2);
    if (nb < 1) nb = 1;
    if (nb > nf) nb = nf;
    const long long e1 = e0 + nb;
    check_cuda(cudaMemsetAsync(G, 0, (size_t)(nb * nf * p2) * sizeof(double), st), "cudaMemsetAsync (ladder)");
    const char* outer = ws ? ws->tag : "";
    if (ws) ws->tag = "ladder-build";
    {  // G[e, q - e0, r, s] = sum_Q B[Q, p0+e, p0+r] B[Q, p0+q, p0+s], e in [e0, e1), q in [e0, np)
      GemmArgs g{};
      g.A = B + (p0 + e0) * n + p0;
      g.B = B + (p0 + e0) * n + p0;
      g.C = G;
      g.alpha = 1.0;
      g.nM = 2;
      g.eM[0] = (int)nb; g.aM[0] = n; g.cM[0] = nf * p2;
      g.eM[1] = np;      g.aM[1] = 1; g.cM[1] = np;
      g.nN = 2;
      g.eN[0] = (int)nf; g.bN[0] = n; g.cN[0] = p2;
      g.eN[1] = np;      g.bN[1] = 1; g.cN[1] = 1;
      g.nK = 1;
      g.eK[0] = naux; g.aK[0] = n * n; g.bK[0] = n * n;
      g.M = nb * np;
      g.N = nf * np;
      g.K = naux;
      g.nbatch = 1;
      if (ws) run_gemm(*ws, g, K_LADDER_BUILD);
      else launch_gemm(g, st, 1);
    }
    if (ws) ws->tag = "ladder-contract";
    {  // L[e, q, i, j] += sum_{r,s} G[e, q - e0, r, s] t[r, s, i, j]
      GemmArgs g{};
      g.A = G;
      g.B = t;
      g.C = L + (e0 * np + e0) * h2;
      g.alpha = 1.0;
      g.nM = 2;
      g.eM[0] = (int)nb; g.aM[0] = nf * p2; g.cM[0] = np * h2;
      g.eM[1] = (int)nf; g.aM[1] = p2;      g.cM[1] = h2;
      g.nK = 2;
      g.eK[0] = np; g.aK[0] = np; g.bK[0] = tst[0];
      g.eK[1] = np; g.aK[1] = 1;  g.bK[1] = tst[1];
      g.nN = 2;
      g.eN[0] = nh; g.bN[0] = tst[2]; g.cN[0] = nh;
      g.eN[1] = nh; g.bN[1] = tst[3]; g.cN[1] = 1;
      g.M = nb * nf;
      g.N = h2;
      g.K = p2;
      g.nbatch = 1;
      if (ws) run_gemm(*ws, g, K_LADDER_CONTRACT);
      else launch_gemm(g, st, 2);
    }
    if (e1 < np) {  // L[q, e, i, j] = L[e, q, j, i] for e in [e0, e1), q in [e1, np)
      NdArgs a{};
      a.nd = 4;
      a.e[0] = (int)nb;       a.sa[0] = np * h2; a.sb[0] = h2;
      a.e[1] = (int)(np - e1); a.sa[1] = h2;     a.sb[1] = np * h2;
      a.e[2] = nh;            a.sa[2] = 1;       a.sb[2] = nh;
      a.e[3] = nh;            a.sa[3] = nh;      a.sb[3] = 1;
      a.total = nb * (np - e1) * h2;
      const double* src = L + (e0 * np + e1) * h2;
      double* dst = L + (e1 * np + e0) * h2;
      if (ws) run_axpy(*ws, a, 1.0, src, dst);
      else launch_axpy(a, 1.0, src, dst, st);
    }
    if (ws) ws->tag = outer;
    e0 = e1;
  }
}

long long ladder_batch_rows(int np, long long max_doubles) {
  const long long p3 = (long long)np * np * np;
  long long bp = max_doubles / (p3 > 0 ? p3 : 1);
  if (bp > np) bp = np;
  return bp;
}

int ladder_check_args(int n, int naux, int p0, int np, int nh, const void* B, const void* t, const void* L,
                      std::string& msg) {
  if (n < 1 || naux < 1 || np < 0 || nh < 0 || p0 < 0 || p0 + np > n) {
    msg = "ladder: need n >= 1, naux >= 1, 0 <= p0, p0 + np <= n, np >= 0, nh >= 0";
    return DSRG_ERR_ARG;
  }
  if ((np > 0 && nh > 0) && (!B || !t || !L)) {
    msg = "ladder: B, t and L must be device pointers";
    return DSRG_ERR_ARG;
  }
  return DSRG_OK;
}

}  // namespace dsrg

extern "C" int dsrg_df_ladder(int n, int naux, int p0, int np, int nh, const double* B, const double* t, double* L,
                              void* stream) {
  using namespace dsrg;
  std::string msg;
  int rc = ladder_check_args(n, naux, p0, np, nh, B, t, L, msg);
  if (rc) return set_error(rc, msg.c_str());
  if (np == 0 || nh == 0) return DSRG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const long long p3 = (long long)np * np * np;
  long long bp = ladder_batch_rows(np, 1LL << 27);  // at most 1 GiB of (pr|qs) per batch
  if (bp < 1) bp = 1;
  double* G = nullptr;
  cudaError_t e = cudaMalloc(&G, (size_t)(bp * p3) * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(DSRG_ERR_OOM, (std::string("ladder scratch: ") + cudaGetErrorString(e)).c_str());
  }
  try {
    check_cuda(cudaMemsetAsync(L, 0, (size_t)np * np * nh * nh * sizeof(double), st), "cudaMemsetAsync");
    const long long tst[4] = {(long long)np * nh * nh, (long long)nh * nh, nh, 1};
    ladder_core(B, n, naux, p0, np, nh, t, tst, L, G, bp, st, nullptr);
    check_cuda(cudaGetLastError(), "ladder launch");
    check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  } catch (const std::exception& ex) {
    cudaFree(G);
    return set_error(DSRG_ERR_CUDA, ex.what());
  }
  cudaFree(G);
  return DSRG_OK;
}

// Device kernels of the DSRG-MRPT2/PT3 energy path (sm_103a).
//
// All arithmetic here is FP64.  Tensors are spin-orbital arrays whose every
// slot is an interval of spatial orbitals [lo, hi) times the two spins,
// stored spin-major: index (sigma, x) -> sigma * (hi - lo) + (x - lo).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dsrg {

constexpr int kMaxDims = 8;

// C[m, n] += alpha * sum_k A[m, k] B[k, n] over multi-indices m, n, k and a
// batch multi-index b present in all three operands.  Every group holds up
// to four dimensions with an extent and one stride per operand.
struct GemmArgs {
  const double* A;
  const double* B;
  double* C;
  double alpha;
  int nM, nN, nK, nB;
  int eM[4], eN[4], eK[4], eB[4];
  long long aM[4], aK[4], aB[4];
  long long bN[4], bK[4], bB[4];
  long long cM[4], cN[4], cB[4];
  long long M, N, K, nbatch;
  // split-K (nbatch == 1 only): split z covers k in [z*kper, (z+1)*kper) and
  // stores its partial tile densely in part[z][M][N]; a second kernel adds
  // alpha * sum_z part[z] into C in a fixed order.
  int splits;
  long long kper;
  double* part;
};

// Elementwise / reduction descriptor over an nd-dimensional index space.
struct NdArgs {
  int nd;
  int e[kMaxDims];
  long long sa[kMaxDims];
  long long sb[kMaxDims];
  long long total;
};

// C[idx] += alpha * A[idx] (strides sb for C, sa for A).
void launch_axpy(const NdArgs& g, double alpha, const double* A, double* C, cudaStream_t st);
// partial[slot] = alpha * sum A[idx] * B[idx]; deterministic two-pass reduction.
void launch_dot(const NdArgs& g, double alpha, const double* A, const double* B,
                double* scratch, int scratch_len, double* out_slot, cudaStream_t st);
// Output tile of the generic contraction for an M x N output (kinds 1, 2
// always use 64 x 64).
void gemm_tile(long long M, long long N, int* bm, int* bn);
// true when the output is small enough for one CTA per output element
bool gemm_is_small(const GemmArgs& g);
// true when K is short enough for one thread per output element
bool gemm_is_short(const GemmArgs& g);
// kind 0: generic contraction, 1: DF build of (pr|qs), 2: ladder contraction
void launch_gemm(const GemmArgs& g, cudaStream_t st, int kind = 0);
void launch_fill(double* p, long long n, double v, cudaStream_t st);

// Reference quantities on spin orbitals.
//   gamma over H = core + active (2h x 2h): identity on core, g1 on active;
//   eta over P = active + virtual (2p x 2p): 1 - g1 on active, identity on virtual.
void launch_build_gamma_eta(int nc, int na, int nv, const double* g1a, const double* g1b,
                            double* gamma, double* eta, cudaStream_t st);
// Spin-orbital cumulant of rank r (2 or 3) on the active space from its spin
// blocks blk[m] (first r-m creators/annihilators alpha, last m beta).
void launch_build_cumulant(int na, int rank, const double* const* blk_dev, double* out,
                           cudaStream_t st);

// Amplitudes of Eqs. T2_1st / T2_2nd and the closed form of [H0, A]:
//   T2 = O2 * R(D) (zero if all four indices are active), W2 = -D * T2.
// Layout [2p][2p][2h][2h] with P = [c, n) and H = [0, c + a) in global orbitals.
void launch_amp2(int nc, int na, int nv, double s, const double* eps, const double* O2,
                 double* T2, double* W2, cudaStream_t st);
// T1 = (O1 + S) * R(D), W1 = -D * T1 + S; layout [2p][2h].
void launch_amp1(int nc, int na, int nv, double s, const double* eps, const double* O1,
                 const double* S, double* T1, double* W1, cudaStream_t st);
// G[x,u] = gamma[x,u] * (eps_x - eps_u) on the active block (2a x 2a).
void launch_gamma_delta(int nc, int na, const double* eps, const double* gamma_H, int h,
                        double* G, cudaStream_t st);

}  // namespace dsrg

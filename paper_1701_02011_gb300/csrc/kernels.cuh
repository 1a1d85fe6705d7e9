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

// Division by a run-time invariant divisor d >= 1 through a multiply-high
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, round-up variant): with l = ceil(log2 d) and
// m = floor(2^(32+l) / d) + 1 = 2^32 + mlo, floor(n / d) = floor(m n / 2^(32+l))
// for every 32-bit n.  Index decoding in the element-wise, reduction and flat
// contraction kernels uses it instead of the long instruction sequence of a
// general integer division.
struct FastDiv {
  unsigned d, mlo;
  int l;
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f{};
  f.d = d ? d : 1;
  f.l = 0;
  while ((1ull << f.l) < f.d) ++f.l;
  f.mlo = (unsigned)(((1ull << 32) * ((1ull << f.l) - f.d)) / f.d + 1);
  return f;
}
#ifdef __CUDACC__
__host__ __device__ __forceinline__
#else
inline
#endif
    unsigned
    fast_div(unsigned n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  const unsigned hi = __umulhi(n, f.mlo);
#else
  const unsigned hi = (unsigned)(((unsigned long long)n * f.mlo) >> 32);
#endif
  return (unsigned)(((unsigned long long)hi + n) >> f.l);
}

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
  FastDiv fe[kMaxDims];  // filled by the launchers when total < 2^31
  long long sa[kMaxDims];
  long long sb[kMaxDims];
  long long total;
};

// C[idx] += alpha * A[idx] (strides sb for C, sa for A).
void launch_axpy(const NdArgs& g, double alpha, const double* A, double* C, cudaStream_t st);

// Up to kMaxBlocks spin blocks sharing extents and strides, one launch.
constexpr int kMaxBlocks = 64;
struct AxpyBlocks {
  const double* a[kMaxBlocks];
  double* c[kMaxBlocks];
  int n;
};
struct DotBlocks {
  const double* a[kMaxBlocks];
  const double* b[kMaxBlocks];
  int n;
};
// C_k[idx] += alpha * A_k[idx] for every block k (distinct C blocks)
void launch_axpy_blocks(const NdArgs& g, double alpha, const AxpyBlocks& p, cudaStream_t st);
// *out = alpha * sum_k sum_idx A_k[idx] B_k[idx] in one launch: per-CTA
// compensated partials, and the CTA that finishes last (atomic ticket, reset
// afterwards; no CTA waits) adds them in a fixed order.
void launch_dot_blocks(const NdArgs& g, double alpha, const DotBlocks& p, double* scratch, int scratch_len,
                       unsigned* ticket, double* out, cudaStream_t st);
// Output tile of the generic contraction for an M x N output (kinds 1, 2
// always use 64 x 64).
void gemm_tile(long long M, long long N, int* bm, int* bn);
// true when the output is small enough for one CTA per output element
bool gemm_is_small(const GemmArgs& g);
// true when K is short enough for one thread per output element
bool gemm_is_short(const GemmArgs& g);
// Flat contraction (one thread per output and k chunk, no tile padding) for
// narrow, short or small products.  A plan with z > 1 needs part[z * M*N*nbatch].
struct FlatPlan {
  int wk;         // warps of a CTA on consecutive k chunks of the same outputs (1, 2, 4, 8)
  int z;          // CTA rows over k (partials reduced in a fixed order)
  long long len;  // k per chunk
  int mfast;      // lanes along m (1) or n (0)
};
// Output blocks of one flat launch: block j accumulates the products of the
// operand pairs first[j] .. first[j+1]-1 (same geometry as the GemmArgs,
// whose A, B, C pointers are ignored) into c[j].  Distinct c[j] only.
constexpr int kFlatMaxPairs = 64;
struct FlatTable {
  const double* a[kFlatMaxPairs];
  const double* b[kFlatMaxPairs];
  double* c[kFlatMaxPairs];
  int first[kFlatMaxPairs + 1];
  int ngroups;
};
bool gemm_use_flat(const GemmArgs& g);
// plan for `groups` output blocks (the chunking along k covers the GPU with
// all of them together)
FlatPlan gemm_flat_plan(const GemmArgs& g, int groups = 1);
// part needs groups * z * M*N*nbatch doubles when the plan has z > 1
void launch_gemm_flat(const GemmArgs& g, const FlatPlan& p, const FlatTable& tab, double* part, cudaStream_t st);
// kind 0: generic contraction, 1: DF build of (pr|qs), 2: ladder contraction
void launch_gemm(const GemmArgs& g, cudaStream_t st, int kind = 0);
void launch_fill(double* p, long long n, double v, cudaStream_t st);
// out[0] = sum slots[r0, r1), out[1] = sum slots[r2, r3), out[2] = sum
// slots[r3, r4): compensated, fixed order (the energy components E(2), E3a, E3b)
void launch_sum_slots(const double* slots, const int* r, double* out, cudaStream_t st);
// D[i][i] += v for the n x n row-major D
void launch_add_diagonal(double* D, int n, double v, cudaStream_t st);

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
//   T2 = O2 * R(D) (zero if all four indices are active), W2 = -D * T2, on
// every stored spin block of the [P,P,H,H] layout (P = [c, n), H = [0, c + a)).
// spin-block offsets (block bits: slot k spin at bit k; < 0 = not stored) and
// spatial strides of a [P,P,H,H] array
struct Amp2Layout {
  long long boff[16];
  long long st[4];
};
void launch_amp2(int nc, int na, int nv, double s, const double* eps, const double* O2,
                 double* T2, double* W2, const Amp2Layout& lay, cudaStream_t st);
// T1 = (O1 + S) * R(D), W1 = -D * T1 + S; layout [2p][2h].
void launch_amp1(int nc, int na, int nv, double s, const double* eps, const double* O1,
                 const double* S, double* T1, double* W1, cudaStream_t st);
// G[x,u] = gamma[x,u] * (eps_x - eps_u) on the active block (2a x 2a).
void launch_gamma_delta(int nc, int na, const double* eps, const double* gamma_H, int h,
                        double* G, cudaStream_t st);

}  // namespace dsrg

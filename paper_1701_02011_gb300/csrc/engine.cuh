// Host-side tensor machinery for the DSRG-MRPT2/PT3 energy path.
//
// A spin-orbital tensor slot covers an interval [lo, hi) of spatial orbitals
// (global numbering: core [0,c), active [c,c+a), virtual [c+a,n)) for both
// spins, laid out spin-major.  Contractions intersect the intervals of every
// label across operands, so a term written once over hole (H = core+active)
// and particle (P = active+virtual) ranges automatically restricts to the
// overlap (the active space) where two different ranges meet.  Spin blocks
// that are identically zero are tracked by a bit mask and skipped.
#pragma once
#include <cstdint>
#include <functional>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dsrg.h"
#include "kernels.cuh"

namespace dsrg {

// Exception carrying the DSRG_ERR_* code the C interface returns for it:
// CUDA errors (DSRG_ERR_CUDA, or DSRG_ERR_OOM for a failed allocation),
// DSRG_ERR_TIMEOUT for a bounded wait that ran out.  Other exceptions map
// to DSRG_ERR_INTERNAL.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

struct Iv {
  int lo = 0, hi = 0;
  int len() const { return hi - lo; }
  bool empty() const { return hi <= lo; }
  bool contains(const Iv& o) const { return lo <= o.lo && o.hi <= hi; }
};
inline Iv isect(Iv a, Iv b) { return Iv{a.lo > b.lo ? a.lo : b.lo, a.hi < b.hi ? a.hi : b.hi}; }

constexpr int kMaxRank = 6;

// Spin blocks: block b has spin (bit k of b) on slot k.  A tensor stores
// either every block (dense: rank <= 2 and the cumulants) or only the blocks
// that conserve the alpha count between its first and second half of slots
// (creators | annihilators): 6 of 16 for rank 4.  Each stored block is a
// dense row-major array over the slots' spatial intervals.
constexpr long long kNoBlock = -1;

struct View {
  double* p = nullptr;  // spatial origin: every slot at iv.lo, block offset 0
  int rank = 0;
  Iv iv[kMaxRank];
  long long st[kMaxRank] = {0};      // stride of the spatial index within a block
  long long boff[1 << kMaxRank] = {};  // offset of stored block b from p (kNoBlock if absent)
  uint64_t stored = 0;               // blocks present in memory
  uint64_t mask = 0;                 // blocks that may be non-zero (a subset of stored)
  View sub(const Iv* want) const;
  // the same data with slot k of the result being slot perm[k] of this view
  View permuted(const int* perm) const;
};

class Workspace;

// Kernels whose launches can be timed one by one (opt-in) with CUDA events on
// the launching stream.
enum KernelId {
  K_GEMM = 0, K_LADDER_BUILD, K_LADDER_CONTRACT, K_AXPY, K_DOT, K_AMP, K_OZAKI_PACK, K_OZAKI_MMA, K_CI_MATVEC,
  K_NKERNELS
};
const char* kernel_name(int id);

struct Tensor {
  View v;
  size_t n = 0;    // elements
  size_t cap = 0;  // elements of the underlying block
  Workspace* ws = nullptr;
  Tensor() = default;
  Tensor(const Tensor&) = delete;
  Tensor& operator=(const Tensor&) = delete;
  Tensor(Tensor&& o) noexcept { *this = std::move(o); }
  Tensor& operator=(Tensor&& o) noexcept;
  ~Tensor();
  void release();
};

// Device memory for tensors: blocks are cached by size and reused, so after
// the first energy evaluation no further cudaMalloc happens.
class Workspace {
 public:
  explicit Workspace(cudaStream_t st) : stream(st) {}
  ~Workspace();
  double* get(size_t n, size_t& cap);
  void put(double* p, size_t cap);
  size_t bytes_in_use() const { return in_use_; }
  size_t peak_bytes() const { return peak_; }
  cudaStream_t stream;
  // result slots of scalar reductions (device) and their host copy
  double* results = nullptr;
  int nresults = 0, cap_results = 0;
  double* dot_scratch = nullptr;  // dot_scratch_len doubles, then the ticket of the one-launch dot
  int dot_scratch_len = 0;
  unsigned* dot_ticket = nullptr;  // zero between launches
  int* oz_status = nullptr;        // split-precision kernels' error flag (device; nullptr: file-scope flag)
  long long wait_cycles = 0;       // budget of the split kernels' bounded waits (0: default)
  bool tune = false;               // time tile/split candidates of new split-product shapes
  unsigned long long generation = 0;  // bumped when cached blocks are freed (captured graphs go stale)
  long long launches = 0;
  // > 0: large contractions run as split-precision tensor-core products with
  // this many 7-bit digit slices per operand; 0: FP64 everywhere
  int slices = 0;
  // opt-in per-launch timing
  bool profiling = false;
  const char* tag = "";  // step of the energy being issued (profile output only)
  struct Rec { int id; cudaEvent_t a, b; double flops, xflops, bytes; long long m, n, k; const char* tag; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> ev_pool;
  long long prof_launches[K_NKERNELS] = {0};
  double prof_ms[K_NKERNELS] = {0}, prof_flops[K_NKERNELS] = {0}, prof_bytes[K_NKERNELS] = {0};
  double prof_xflops[K_NKERNELS] = {0};
  // per step of the energy (the tag in force at the launch), in order of first use
  struct StepStat { std::string name; long long launches = 0; double ms = 0, flops = 0; };
  std::vector<StepStat> prof_steps;
  void prof_reset();
  // brackets one launch; call begin() before and end() after it.  flops: the
  // FP64 flops of the contraction it computes (2 M N K); xflops: the flops
  // the hardware executes (split products: digit pairs and tile padding;
  // < 0: same as flops); bytes: algorithmic bytes of element-wise kernels
  int begin(int id, double flops, double bytes, double xflops = -1.0);
  void end(int rec);
  void prof_collect();  // after the stream is synchronised

 private:
  struct Blk { double* p; size_t n; };
  std::vector<Blk> free_;
  size_t in_use_ = 0, peak_ = 0;
  const char* peak_tag_ = "";  // step being issued when the peak was reached
};

// Names the step issued while it is in scope (restores the outer name).
struct ProfTag {
  Workspace& ws;
  const char* prev;
  ProfTag(Workspace& w, const char* t) : ws(w), prev(w.tag) { w.tag = t; }
  ~ProfTag() { ws.tag = prev; }
};

// dense: store every spin block (else rank >= 4 tensors keep only the
// alpha-conserving blocks)
Tensor make_tensor(Workspace& ws, int rank, const Iv* ivs, bool zero = true, bool dense = false);
// Non-owning view of T with slots permuted (slot k of the alias is slot
// perm[k] of T), its mask permuted alike; merge_alias_mask carries the
// blocks written through the alias back into T's mask.
Tensor alias_permuted(Tensor& T, const int* perm);
void merge_alias_mask(Tensor& T, const Tensor& alias, const int* perm);
// Mask of a tensor whose first rank/2 slots are creators and the rest
// annihilators: non-zero only when the alpha counts agree.
uint64_t conserving_mask(int rank);

// C[lc] += alpha * A[la] * B[lb] (labels are characters; labels shared by A and
// B but absent from C are summed).  Returns false if nothing was launched.
bool contract(Workspace& ws, double alpha, const View& A, const char* la, const View& B, const char* lb,
              Tensor& C, const char* lc);
// C[lc] += alpha * A[la] with the same label set.
void axpy(Workspace& ws, double alpha, const View& A, const char* la, Tensor& C, const char* lc);
// alpha * sum over all labels of A[la] * B[lb] (identical label sets); each
// spin block's value lands in the next free device result slot.
void dot(Workspace& ws, double alpha, const View& A, const char* la, const View& B, const char* lb);

// Two-body operator with the symmetries of an antisymmetrised Hermitian
// operator, stored on a few canonical interval classes; a request for any
// other class is served as a permuted view with a sign.
struct Sym2 {
  std::vector<Tensor> cls;
  // Classes too large to keep: V on any four intervals is built on demand,
  // in slabs along the first slot of at most max_elems doubles of working
  // memory each (nullptr: every class a term needs is stored).
  std::function<Tensor(const Iv*)> make;
  long long max_elems = 0;
  bool resolve(const Iv* want, View& out, double& sign) const;
};

// A two-body operator X2 = cv V + cw (W + W^+): V kept on complete canonical
// classes, W given by its excitation block [P,P,H,H] (zero elsewhere), so
// its Hermitian image occupies [H,H,P,P].
struct Op2 {
  const Sym2* V = nullptr;
  double cv = 0.0;
  const Tensor* W = nullptr;
  double cw = 0.0;
};

// C[lc] += alpha * X2[lx] * B[lb].  With skip_v the V part is left out (the
// caller evaluates it another way, e.g. the density-fitted ladder).
bool contract_x2(Workspace& ws, double alpha, const Op2& X, const char* lx, const View& B, const char* lb,
                 Tensor& C, const char* lc, bool skip_v = false);
bool contract_x2_left(Workspace& ws, double alpha, const View& A, const char* la, const Op2& X, const char* lx,
                      Tensor& C, const char* lc);
// alpha * sum X2[pqrs] U[pqrs] over U's intervals
void dot_x2(Workspace& ws, double alpha, const Op2& X, const Tensor& U);
// out[abcd] += alpha * X2[abcd] on out's intervals
void fetch_x2(Workspace& ws, double alpha, const Op2& X, Tensor& out);
// W placed as an operator: its excitation block (herm = 0) or the Hermitian
// image of that block (herm = 1), as a view with permuted slots
View w_place(const Tensor& W, int herm);

void check_cuda(cudaError_t e, const char* what);

// Persistent record of tuning decisions (file named by DSRG_TUNE_CACHE; no
// file: decisions live for the process only).  A decision is a few integers
// stored under (kind, GPU, M, N, K, slices); the GPU is identified by its
// name, SM count and compute capability.  lookup fills `vals` and returns
// true when the file holds the key; store appends a line.
bool tune_cache_lookup(const char* kind, long long M, long long N, long long K, int slices, int nvals, int* vals);
void tune_cache_store(const char* kind, long long M, long long N, long long K, int slices, int nvals,
                      const int* vals);

// launches through the workspace (counted, optionally timed)
void run_gemm(Workspace& ws, const GemmArgs& g, int kind = K_GEMM);
void run_axpy(Workspace& ws, const NdArgs& g, double alpha, const double* A, double* C);

}  // namespace dsrg

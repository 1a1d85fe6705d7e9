// Internal state of a DSRG energy handle.
#pragma once
#include "engine.cuh"

namespace dsrg {

struct Handle {
  int nc = 0, na = 0, nv = 0, n = 0, naux = 0;
  double s = 0.0;
  Iv C, A, V, H, P, G;  // core, active, virtual, hole, particle, general
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Workspace ws;
  // inputs (device)
  double* eps = nullptr;
  double* B = nullptr;
  double* f1raw = nullptr;
  bool has_f1 = false;
  double* blk[9] = {};  // g1a g1b l2aa l2ab l2bb l3aaa l3aab l3abb l3bbb
  // reference quantities on spin orbitals
  Tensor gam, eta, L2, L3, F1;
  // active blocks of gamma and eta minus the identity ([A, A]): dressing a
  // copy of X adds (M - 1) X on the active rows
  Tensor gam_dI, eta_dI;
  // intermediates of the last evaluation
  Tensor T1, T2, T1b, T2b, O1, O2;
  // relaxed energies (Eq. E_relaxed): with `relax` set, an energy also
  // accumulates the all-active blocks of the summed transformed Hamiltonian
  // relative to E0, dense spin-major over [A, A] and [A, A, A, A]:
  // second order (H^(0) + H^(1) + 1/2 [Htilde^(1), A^(1)]) in rx1_2, rx2_2,
  // the third-order terms (1/2 [Htilde^(1), A^(2)] + 1/2 [Htilde^(2), A^(1)])
  // in rx1_3, rx2_3
  bool relax = false;
  Tensor rx1_2, rx2_2, rx1_3, rx2_3;
  // first-order aavv amplitudes of the Dyall-H(0) solve (dense, [V,V,A,A])
  Tensor t_aavv;
  long long launches = 0;
  long long d2h_bytes = 0;
  // result-slot boundaries of the last issued energy: E(2) [res0, res1),
  // E3a [res2, res3), E3b [res3, res4)
  int res[5] = {0, 0, 0, 0, 0};
  bool res_pt3 = false;
  // the PT3 energy captured as a CUDA graph (batch calls); stale when the
  // workspace generation changes or the handle runs eagerly / reloads
  cudaGraphExec_t graph = nullptr;
  unsigned long long graph_gen = 0;
  bool warm = false;  // one eager energy has filled the workspace cache
  void drop_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
  }
  // raw device buffers taken from the workspace (returned on destruction)
  std::vector<std::pair<double*, size_t>> owned;
  double* own(size_t n) {
    size_t cap;
    double* p = ws.get(n, cap);
    owned.push_back({p, cap});
    return p;
  }
  explicit Handle(cudaStream_t st) : stream(st), ws(st) {}
  ~Handle() {
    drop_graph();
    for (auto& b : owned) ws.put(b.first, b.second);
  }
};

Tensor vclass(Handle& h, const Iv* ivs, double coef);
Tensor build_x1(Handle& h, double c_v, const Tensor* W1, double c_w);
void build_v(Handle& h, unsigned classes, Sym2& V, bool on_demand = false);
Tensor dress(Handle& h, const Tensor& X, int slot, const Tensor& M);
Tensor dress(Handle& h, Tensor&& X, int slot, const Tensor& M);  // in place on a temporary
void amplitudes(Handle& h, const Tensor* O1, const Tensor& O2, Tensor& T1, Tensor& T2, Tensor& W1, Tensor& W2);
void df_ladder(Handle& h, const Tensor& T2, Tensor& C2, double coef);
struct Op1Pieces;
void commutator(Handle& h, const Tensor& X1, const Op2& X2, const Tensor& T1, const Tensor& T2, Tensor& C1,
                Tensor& C2, bool df, const Op1Pieces* X1p);
void commutator_A(Handle& h, const Tensor& X1, const Op2& X2, const Tensor& T1, const Tensor& T2, Tensor& O1,
                  Tensor& O2, bool df, const Op1Pieces* X1p);
void scalar(Handle& h, const Tensor& X1, const Op2& X2, const Tensor& T1, const Tensor& T2);
void run_energy(Handle& h, bool pt3, double* e2, double* e3a, double* e3b);
void issue_energy(Handle& h, bool pt3);
void finish_energy(Handle& h, double* e2, double* e3a, double* e3b);

// lowest eigenvalue of the order-2 or order-3 relaxed CASCI problem over the
// determinants with n_alpha, n_beta active electrons, from the blocks the
// last energy (run with relax set) accumulated
struct RelaxResult {
  double e = 0.0, residual = 0.0;
  int steps = 0;
};
long long relax_ndet(int na, int n_alpha, int n_beta);

// first-order aavv amplitudes with Dyall's H(0) at s -> infinity (App. B)
struct DyallResult {
  int iterations = 0, converged = 0;
  double max_residual = 0.0, max_source = 0.0, min_shifted_denominator = 0.0;
  long long pairs_not_converged = 0, small_denominators = 0;
};
DyallResult dyall_aavv(Handle& h, double tol, int max_iter);
// h1[u][u] += eps[nc + u] on both spins of a dense [A, A] block
void launch_active_diagonal(int nc, int na, const double* eps, double* h1, cudaStream_t st);
RelaxResult relaxed_ci(Handle& h, int order, int n_alpha, int n_beta);

}  // namespace dsrg

// C interface (include/dsrg.h) over the GPU energy driver.
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>

#include "../../include/dsrg.h"
#include "dsrg_impl.cuh"
#include "ozaki.cuh"

struct dsrg_handle {
  dsrg::Handle* h;
};

namespace {
thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

// the DSRG_ERR_* code an exception stands for (the code it carries)
int classify(const std::exception& e) {
  if (const auto* d = dynamic_cast<const dsrg::Error*>(&e)) return d->code;
  if (dynamic_cast<const std::bad_alloc*>(&e)) return DSRG_ERR_OOM;
  return DSRG_ERR_INTERNAL;
}

size_t pow_na(int na, int k) {
  size_t r = 1;
  for (int i = 0; i < k; ++i) r *= (size_t)na;
  return r;
}

int validate(const dsrg_inputs* in) {
  if (!in) return fail(DSRG_ERR_ARG, "inputs are NULL");
  if (in->nc < 0 || in->na < 0 || in->nv < 0 || in->naux < 1)
    return fail(DSRG_ERR_ARG, "sizes must be nc, na, nv >= 0 and naux >= 1");
  if (in->nc + in->na + in->nv < 1) return fail(DSRG_ERR_ARG, "no orbitals");
  if (in->na > 16) return fail(DSRG_ERR_ARG, "at most 16 active orbitals are supported");
  if (!(in->s > 0.0) || !std::isfinite(in->s)) return fail(DSRG_ERR_ARG, "flow parameter s must be positive");
  if (!in->eps || !in->B) return fail(DSRG_ERR_ARG, "eps and B are required");
  if (in->na > 0 && (!in->g1a || !in->g1b || !in->l2aa || !in->l2ab || !in->l2bb || !in->l3aaa || !in->l3aab ||
                     !in->l3abb || !in->l3bbb))
    return fail(DSRG_ERR_ARG, "active-space densities and cumulants are required when na > 0");
  if (in->memory != DSRG_MEM_HOST && in->memory != DSRG_MEM_DEVICE) return fail(DSRG_ERR_ARG, "bad memory kind");
  return DSRG_OK;
}

void copy_in(double* dst, const double* src, size_t n, int memory, cudaStream_t st) {
  if (n == 0) return;
  dsrg::check_cuda(cudaMemcpyAsync(dst, src, n * sizeof(double),
                                   memory == DSRG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st),
                   "cudaMemcpyAsync (inputs)");
}

// copy the inputs and rebuild gamma, eta, cumulants and f1 on spin orbitals
void load_inputs(dsrg::Handle& h, const dsrg_inputs* in) {
  using namespace dsrg;
  cudaStream_t st = h.stream;
  const int n = h.n, na = h.na;
  copy_in(h.eps, in->eps, (size_t)n, in->memory, st);
  copy_in(h.B, in->B, (size_t)h.naux * n * n, in->memory, st);
  const double* src[9] = {in->g1a, in->g1b, in->l2aa, in->l2ab, in->l2bb, in->l3aaa, in->l3aab, in->l3abb, in->l3bbb};
  const int rank[9] = {2, 2, 4, 4, 4, 6, 6, 6, 6};
  for (int k = 0; k < 9; ++k)
    if (na > 0) copy_in(h.blk[k], src[k], pow_na(na, rank[k]), in->memory, st);
  {
    Iv hh[2] = {h.H, h.H}, pp[2] = {h.P, h.P};
    h.gam = make_tensor(h.ws, 2, hh, false);
    h.eta = make_tensor(h.ws, 2, pp, false);
    launch_build_gamma_eta(h.nc, na, h.nv, h.blk[0], h.blk[1], h.gam.v.p, h.eta.v.p, st);
    h.gam.v.mask = h.eta.v.mask = conserving_mask(2);
    Iv aa[2] = {h.A, h.A};
    h.gam_dI = make_tensor(h.ws, 2, aa, true);
    h.eta_dI = make_tensor(h.ws, 2, aa, true);
    if (na > 0) {
      axpy(h.ws, 1.0, h.gam.v.sub(aa), "xy", h.gam_dI, "xy");
      axpy(h.ws, 1.0, h.eta.v.sub(aa), "xy", h.eta_dI, "xy");
      launch_add_diagonal(h.gam_dI.v.p, 2 * na, -1.0, st);
      launch_add_diagonal(h.eta_dI.v.p, 2 * na, -1.0, st);
    }
    h.gam_dI.v.mask = h.eta_dI.v.mask = conserving_mask(2);
  }
  {
    Iv a4[4] = {h.A, h.A, h.A, h.A}, a6[6] = {h.A, h.A, h.A, h.A, h.A, h.A};
    h.L2 = make_tensor(h.ws, 4, a4, true, true);  // dense: built whole by k_cumulant
    h.L3 = make_tensor(h.ws, 6, a6, true, true);
    if (na > 0) {
      const double* b2[4] = {h.blk[2], h.blk[3], h.blk[4], nullptr};
      const double* b3[4] = {h.blk[5], h.blk[6], h.blk[7], h.blk[8]};
      launch_build_cumulant(na, 2, b2, h.L2.v.p, st);
      launch_build_cumulant(na, 3, b3, h.L3.v.p, st);
    }
    h.L2.v.mask = conserving_mask(4);
    h.L3.v.mask = conserving_mask(6);
  }
  h.has_f1 = in->f1 != nullptr;
  if (h.has_f1) {
    if (!h.f1raw) h.f1raw = h.own((size_t)n * n);
    copy_in(h.f1raw, in->f1, (size_t)n * n, in->memory, st);
    // spin-orbital [G,G]: f1 on both spin diagonal blocks, its core-core,
    // active-active and virtual-virtual parts removed (those are in H(0))
    Iv gg[2] = {h.G, h.G};
    h.F1 = make_tensor(h.ws, 2, gg, true);
    const int lo[3] = {0, h.nc, h.nc + h.na}, hi[3] = {h.nc, h.nc + h.na, n};
    for (int s = 0; s < 2; ++s)
      for (int bi = 0; bi < 3; ++bi)
        for (int bj = 0; bj < 3; ++bj) {
          if (bi == bj) continue;
          if (hi[bi] <= lo[bi] || hi[bj] <= lo[bj]) continue;
          NdArgs g{};
          g.nd = 2;
          g.e[0] = hi[bi] - lo[bi];
          g.e[1] = hi[bj] - lo[bj];
          g.sa[0] = n;
          g.sa[1] = 1;
          g.sb[0] = h.F1.v.st[0];
          g.sb[1] = h.F1.v.st[1];
          g.total = (long long)g.e[0] * g.e[1];
          launch_axpy(g, 1.0, h.f1raw + (long long)lo[bi] * n + lo[bj],
                      h.F1.v.p + h.F1.v.boff[s * 3] + lo[bi] * h.F1.v.st[0] + lo[bj] * h.F1.v.st[1],
                      st);
        }
    h.F1.v.mask = conserving_mask(2);
  }
  check_cuda(cudaGetLastError(), "launch (load)");
}
}  // namespace

namespace dsrg {
int set_error(int code, const char* msg) { return fail(code, msg ? msg : ""); }
}  // namespace dsrg

extern "C" {

const char* dsrg_last_error(void) { return g_last_error.c_str(); }

int dsrg_init(const dsrg_inputs* in, const dsrg_options* opts, dsrg_handle** out) {
  g_last_error.clear();
  if (!out) return fail(DSRG_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate(in);
  if (rc) return rc;
  if (opts && opts->precision != DSRG_PREC_FP64 && opts->precision != DSRG_PREC_SPLIT)
    return fail(DSRG_ERR_ARG, "unsupported precision");
  int slices = 0;
  if (opts && opts->precision == DSRG_PREC_SPLIT) {
    slices = opts->slices ? opts->slices : 6;
    if (slices < 1 || slices > 8) return fail(DSRG_ERR_ARG, "slices must be 1..8");
  }
  if (opts && opts->wait_limit < 0) return fail(DSRG_ERR_ARG, "wait_limit must be >= 0");
  cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
  bool own = false;
  if (!st) {
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(DSRG_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    own = true;
  }
  dsrg::Handle* h = new (std::nothrow) dsrg::Handle(st);
  if (!h) {
    if (own) cudaStreamDestroy(st);
    return fail(DSRG_ERR_OOM, "host allocation failed");
  }
  h->own_stream = own;
  h->ws.slices = slices;
  h->ws.tune = opts && opts->tune != 0;
  h->ws.wait_cycles = opts ? opts->wait_limit : 0;
  try {
    h->nc = in->nc;
    h->na = in->na;
    h->nv = in->nv;
    h->naux = in->naux;
    h->n = in->nc + in->na + in->nv;
    h->s = in->s;
    h->C = {0, in->nc};
    h->A = {in->nc, in->nc + in->na};
    h->V = {in->nc + in->na, h->n};
    h->H = {0, in->nc + in->na};
    h->P = {in->nc, h->n};
    h->G = {0, h->n};
    h->eps = h->own((size_t)h->n);
    h->B = h->own((size_t)h->naux * h->n * h->n);
    const int rank[9] = {2, 2, 4, 4, 4, 6, 6, 6, 6};
    if (h->na > 0)
      for (int k = 0; k < 9; ++k) h->blk[k] = h->own(pow_na(h->na, rank[k]));
    h->ws.cap_results = 1 << 16;
    dsrg::check_cuda(cudaMalloc(&h->ws.results, h->ws.cap_results * sizeof(double)), "cudaMalloc (results)");
    h->ws.dot_scratch_len = 2 * 152 * 16;
    // dot partials, then the dot's ticket and the split kernels' status flag
    dsrg::check_cuda(cudaMalloc(&h->ws.dot_scratch, (h->ws.dot_scratch_len + 4) * sizeof(double)),
                     "cudaMalloc (scratch)");
    h->ws.dot_ticket = reinterpret_cast<unsigned*>(h->ws.dot_scratch + h->ws.dot_scratch_len);
    h->ws.oz_status = reinterpret_cast<int*>(h->ws.dot_scratch + h->ws.dot_scratch_len + 2);
    dsrg::check_cuda(cudaMemsetAsync(h->ws.dot_ticket, 0, 4 * sizeof(double), st), "cudaMemsetAsync (ticket)");
    load_inputs(*h, in);
    dsrg::check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize (init)");
  } catch (const std::exception& e) {
    int code = classify(e);
    std::string msg = e.what();
    delete h;
    if (own) cudaStreamDestroy(st);
    return fail(code, msg);
  }
  dsrg_handle* hd = new (std::nothrow) dsrg_handle{h};
  if (!hd) {
    delete h;
    if (own) cudaStreamDestroy(st);
    return fail(DSRG_ERR_OOM, "host allocation failed");
  }
  *out = hd;
  return DSRG_OK;
}

int dsrg_load(dsrg_handle* hd, const dsrg_inputs* in) {
  g_last_error.clear();
  if (!hd || !hd->h) return fail(DSRG_ERR_STATE, "NULL handle");
  int rc = validate(in);
  if (rc) return rc;
  dsrg::Handle& h = *hd->h;
  if (in->nc != h.nc || in->na != h.na || in->nv != h.nv || in->naux != h.naux)
    return fail(DSRG_ERR_ARG, "dsrg_load needs the sizes the handle was created with");
  try {
    h.drop_graph();  // the captured energy refers to the old reference tensors
    h.warm = false;
    h.s = in->s;
    load_inputs(h, in);
  } catch (const std::exception& e) {
    return fail(classify(e), e.what());
  }
  return DSRG_OK;
}

namespace {
void reset_status(dsrg::Handle& h) {
  if (h.ws.slices > 0)
    dsrg::check_cuda(cudaMemsetAsync(h.ws.oz_status, 0, sizeof(int), h.stream), "status reset");
}

void check_status(dsrg::Handle& h) {
  dsrg::check_cuda(cudaGetLastError(), "kernel launch");
  if (h.ws.slices > 0 && dsrg::ozaki_status(h.stream, h.ws.oz_status))
    throw dsrg::Error(DSRG_ERR_TIMEOUT, "a bounded wait in the split-precision kernel ran out");
}

void eager_energy(dsrg::Handle& h, bool pt3, dsrg_energies* out) {
  h.drop_graph();  // the handle's tensors move to new buffers
  double e2 = 0, e3a = 0, e3b = 0;
  reset_status(h);
  dsrg::run_energy(h, pt3, &e2, &e3a, &e3b);
  check_status(h);
  h.warm = true;
  h.ws.prof_collect();
  out->e2 = e2;
  out->e3a = e3a;
  out->e3b = e3b;
  out->e3 = e3a + e3b;
}

// Capture one PT3 energy of h (status reset included) as a CUDA graph.  The
// workspace cache is warm, so the captured buffers are the ones the eager
// energy used; they stay reserved by the handle until the graph is dropped.
void capture_energy(dsrg::Handle& h) {
  const bool prof = h.ws.profiling;
  h.ws.profiling = false;
  dsrg::check_cuda(cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
  cudaGraph_t g = nullptr;
  try {
    reset_status(h);
    dsrg::issue_energy(h, true);
  } catch (...) {
    cudaStreamEndCapture(h.stream, &g);
    if (g) cudaGraphDestroy(g);
    h.ws.profiling = prof;
    throw;
  }
  h.ws.profiling = prof;
  dsrg::check_cuda(cudaStreamEndCapture(h.stream, &g), "cudaStreamEndCapture");
  cudaError_t e = cudaGraphInstantiate(&h.graph, g, 0ULL);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h.graph = nullptr;
    dsrg::check_cuda(e, "cudaGraphInstantiate");
  }
  h.graph_gen = h.ws.generation;
}
}  // namespace

static int run(dsrg_handle* hd, bool pt3, dsrg_energies* out) {
  g_last_error.clear();
  if (!hd || !hd->h) return fail(DSRG_ERR_STATE, "NULL handle");
  if (!out) return fail(DSRG_ERR_ARG, "out is NULL");
  try {
    eager_energy(*hd->h, pt3, out);
  } catch (const std::exception& e) {
    return fail(classify(e), e.what());
  }
  return DSRG_OK;
}

int dsrg_pt3_batch(dsrg_handle* const* hs, int n, dsrg_energies* out) {
  g_last_error.clear();
  if (n < 0) return fail(DSRG_ERR_ARG, "n < 0");
  if (n == 0) return DSRG_OK;
  if (!hs || !out) return fail(DSRG_ERR_ARG, "handles and out are required");
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || !hs[i]->h) return fail(DSRG_ERR_STATE, "NULL handle in the batch");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(DSRG_ERR_ARG, "a handle appears twice in the batch");
  }
  try {
    // graphs: captured once per handle (after one eager energy), replayed after
    for (int i = 0; i < n; ++i) {
      dsrg::Handle& h = *hs[i]->h;
      if (h.graph && h.graph_gen != h.ws.generation) h.drop_graph();
      if (!h.graph) {
        if (!h.warm) eager_energy(h, true, &out[i]);
        capture_energy(h);
      }
    }
    // every handle's energy in flight at once, each on its own stream
    for (int i = 0; i < n; ++i) {
      dsrg::Handle& h = *hs[i]->h;
      dsrg::check_cuda(cudaGraphLaunch(h.graph, h.stream), "cudaGraphLaunch");
    }
    for (int i = 0; i < n; ++i) {
      dsrg::Handle& h = *hs[i]->h;
      double e2 = 0, e3a = 0, e3b = 0;
      dsrg::finish_energy(h, &e2, &e3a, &e3b);
      check_status(h);
      out[i].e2 = e2;
      out[i].e3a = e3a;
      out[i].e3b = e3b;
      out[i].e3 = e3a + e3b;
    }
  } catch (const std::exception& e) {
    return fail(classify(e), e.what());
  }
  return DSRG_OK;
}

int dsrg_relaxed(dsrg_handle* hd, int n_alpha, int n_beta, dsrg_relaxed_energies* out) {
  g_last_error.clear();
  if (!hd || !hd->h) return fail(DSRG_ERR_STATE, "NULL handle");
  if (!out) return fail(DSRG_ERR_ARG, "out is required");
  dsrg::Handle& h = *hd->h;
  if (n_alpha < 0 || n_beta < 0 || n_alpha > h.na || n_beta > h.na)
    return fail(DSRG_ERR_ARG, "n_alpha and n_beta must lie in [0, na]");
  const long long ndet = dsrg::relax_ndet(h.na, n_alpha, n_beta);
  if (ndet > 20000) return fail(DSRG_ERR_ARG, "more than 20000 determinants");
  struct Flag {
    dsrg::Handle& h;
    ~Flag() { h.relax = false; }
  } flag{h};
  try {
    h.relax = true;
    dsrg_energies e{};
    eager_energy(h, true, &e);
    h.relax = false;
    const dsrg::RelaxResult r2 = dsrg::relaxed_ci(h, 2, n_alpha, n_beta);
    const dsrg::RelaxResult r3 = dsrg::relaxed_ci(h, 3, n_alpha, n_beta);
    check_status(h);
    h.launches = h.ws.launches;
    h.ws.prof_collect();
    out->e2 = e.e2;
    out->e3a = e.e3a;
    out->e3b = e.e3b;
    out->e3 = e.e3;
    out->e_relaxed2 = r2.e;
    out->e_relaxed3 = r3.e;
    out->residual2 = r2.residual;
    out->residual3 = r3.residual;
    out->ndet = ndet;
    out->steps2 = r2.steps;
    out->steps3 = r3.steps;
  } catch (const std::exception& e) {
    return fail(classify(e), e.what());
  }
  return DSRG_OK;
}

int dsrg_dyall_aavv(dsrg_handle* hd, double tol, int max_iter, dsrg_dyall_result* out) {
  g_last_error.clear();
  if (!hd || !hd->h) return fail(DSRG_ERR_STATE, "NULL handle");
  if (!out || !(tol > 0.0) || max_iter < 1) return fail(DSRG_ERR_ARG, "need out, tol > 0 and max_iter >= 1");
  dsrg::Handle& h = *hd->h;
  try {
    h.drop_graph();
    reset_status(h);
    h.ws.launches = 0;
    const dsrg::DyallResult r = dsrg::dyall_aavv(h, tol, max_iter);
    check_status(h);
    h.launches = h.ws.launches;
    h.ws.prof_collect();
    out->iterations = r.iterations;
    out->converged = r.converged;
    out->max_residual = r.max_residual;
    out->max_source = r.max_source;
    out->min_shifted_denominator = r.min_shifted_denominator;
    out->pairs_not_converged = r.pairs_not_converged;
    out->small_denominators = r.small_denominators;
  } catch (const std::exception& e) {
    return fail(classify(e), e.what());
  }
  return DSRG_OK;
}

int dsrg_pt2(dsrg_handle* hd, dsrg_energies* out) { return run(hd, false, out); }
int dsrg_pt3(dsrg_handle* hd, dsrg_energies* out) { return run(hd, true, out); }

void dsrg_free(dsrg_handle* hd) {
  if (!hd) return;
  if (hd->h) {
    cudaStream_t st = hd->h->stream;
    bool own = hd->h->own_stream;
    cudaStreamSynchronize(st);
    delete hd->h;
    if (own) cudaStreamDestroy(st);
  }
  delete hd;
}

long long dsrg_last_launch_count(const dsrg_handle* hd) {
  if (!hd || !hd->h) return -1;
  return hd->h->launches;
}

int dsrg_profile(dsrg_handle* hd, int enable) {
  g_last_error.clear();
  if (!hd || !hd->h) return fail(DSRG_ERR_STATE, "NULL handle");
  hd->h->ws.profiling = enable != 0;
  hd->h->ws.prof_reset();
  return DSRG_OK;
}

int dsrg_profile_stats(const dsrg_handle* hd, int kernel, const char** name, long long* launches, double* ms,
                       double* flops, double* exec_flops, double* bytes) {
  if (!hd || !hd->h) return fail(DSRG_ERR_STATE, "NULL handle");
  if (kernel < 0 || kernel >= dsrg::K_NKERNELS) return fail(DSRG_ERR_ARG, "kernel index out of range");
  const dsrg::Workspace& w = hd->h->ws;
  if (name) *name = dsrg::kernel_name(kernel);
  if (launches) *launches = w.prof_launches[kernel];
  if (ms) *ms = w.prof_ms[kernel];
  if (flops) *flops = w.prof_flops[kernel];
  if (exec_flops) *exec_flops = w.prof_xflops[kernel];
  if (bytes) *bytes = w.prof_bytes[kernel];
  return DSRG_OK;
}

int dsrg_profile_step(const dsrg_handle* hd, int step, const char** name, long long* launches, double* ms,
                      double* flops) {
  if (!hd || !hd->h) return fail(DSRG_ERR_STATE, "NULL handle");
  const dsrg::Workspace& w = hd->h->ws;
  if (step < 0 || step >= (int)w.prof_steps.size()) return fail(DSRG_ERR_ARG, "step index out of range");
  const auto& x = w.prof_steps[step];
  if (name) *name = x.name.c_str();
  if (launches) *launches = x.launches;
  if (ms) *ms = x.ms;
  if (flops) *flops = x.flops;
  return DSRG_OK;
}

long long dsrg_last_d2h_bytes(const dsrg_handle* hd) {
  if (!hd || !hd->h) return -1;
  return hd->h->d2h_bytes;
}

long long dsrg_peak_bytes(const dsrg_handle* hd) {
  if (!hd || !hd->h) return -1;
  return (long long)hd->h->ws.peak_bytes();
}

int dsrg_fetch(const dsrg_handle* hd, const char* name, double* dst, long long count) {
  g_last_error.clear();
  if (!hd || !hd->h) return fail(DSRG_ERR_STATE, "NULL handle");
  if (!name || !dst) return fail(DSRG_ERR_ARG, "name and dst are required");
  const dsrg::Handle& h = *hd->h;
  const dsrg::Tensor* t = nullptr;
  if (!strcmp(name, "T1")) t = &h.T1;
  else if (!strcmp(name, "T2")) t = &h.T2;
  else if (!strcmp(name, "T1b")) t = &h.T1b;
  else if (!strcmp(name, "T2b")) t = &h.T2b;
  else if (!strcmp(name, "O1")) t = &h.O1;
  else if (!strcmp(name, "O2")) t = &h.O2;
  else if (!strcmp(name, "Hbar1_2")) t = &h.rx1_2;
  else if (!strcmp(name, "Hbar2_2")) t = &h.rx2_2;
  else if (!strcmp(name, "Hbar1_3")) t = &h.rx1_3;
  else if (!strcmp(name, "Hbar2_3")) t = &h.rx2_3;
  else if (!strcmp(name, "Taavv")) t = &h.t_aavv;
  else return fail(DSRG_ERR_ARG, std::string("unknown tensor ") + name);
  if (!t->v.p) return fail(DSRG_ERR_STATE, std::string(name) + " has not been computed");
  // the dense spin-major layout: every spin block, blocks not stored are zero
  long long dense = 1;
  for (int k = 0; k < t->v.rank; ++k) dense *= 2LL * t->v.iv[k].len();
  if (dense != count) return fail(DSRG_ERR_ARG, "element count mismatch");
  try {
    dsrg::Handle& hm = *hd->h;
    dsrg::Tensor d = dsrg::make_tensor(hm.ws, t->v.rank, t->v.iv, true, true);
    const char* lab = "abcdef";
    char l[8] = {0};
    for (int k = 0; k < t->v.rank; ++k) l[k] = lab[k];
    dsrg::View src = t->v;
    src.mask = src.stored;  // copy every stored block
    dsrg::axpy(hm.ws, 1.0, src, l, d, l);
    dsrg::check_cuda(cudaMemcpyAsync(dst, d.v.p, d.n * sizeof(double), cudaMemcpyDeviceToHost, h.stream),
                     "cudaMemcpyAsync (fetch)");
    dsrg::check_cuda(cudaStreamSynchronize(h.stream), "cudaStreamSynchronize (fetch)");
  } catch (const std::exception& ex) {
    return fail(classify(ex), ex.what());
  }
  return DSRG_OK;
}

}  // extern "C"

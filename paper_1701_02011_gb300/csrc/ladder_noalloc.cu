// A variant of dsrg_df_ladder for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at the point where they need the
// ladder: frameworks whose caching allocator reserved all device memory up
// front (a cudaMalloc from inside a library would fail or fragment their
// pool), and embedded or real-time runtimes that forbid allocation after
// start-up.  This entry point takes inputs and outputs from the caller and
// keeps its own scratch in a fixed, file-scope device array instead.
#include <cuda.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/dsrg.h"
#include "ladder.cuh"

namespace {
// (pr|qs) rows of one batch: 2^22 doubles = 32 MiB on every GPU where the
// library's device code is loaded, held until the process exits.
constexpr long long kScratchDoubles = 1LL << 22;
static __device__ __align__(256) double g_ladder_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

// The current context's process-unique id, through driver entry points the
// runtime hands out (the library does not link the driver library itself).
// 0 if the driver cannot tell.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
    return id;
  return 0;
}

// Host code cannot use g_ladder_scratch directly: its name here denotes a
// host-side shadow, not device memory.  The device address is looked up at
// set-up, once per device with that device current, and again whenever the
// device's context has changed since (after cudaDeviceReset the module is
// loaded anew and the array may sit elsewhere).  The runtime creates the
// context on the first runtime call, so the id is read after the lookup.
int scratch_address(double** out, std::string& msg) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    msg = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return DSRG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    msg = "device index out of range for the fixed scratch table";
    return DSRG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long ctx = g_addr[dev] ? current_context_id() : 0;
  if (!g_addr[dev] || ctx == 0 || ctx != g_ctx_id[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_ladder_scratch);
    if (e != cudaSuccess || !p) {
      msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      g_addr[dev] = nullptr;
      return DSRG_ERR_CUDA;
    }
    g_addr[dev] = p;
    g_ctx_id[dev] = current_context_id();
  }
  *out = g_addr[dev];
  return DSRG_OK;
}
}  // namespace

extern "C" int dsrg_df_ladder_noalloc(int n, int naux, int p0, int np, int nh, const double* B, const double* t,
                                      double* L, void* stream) {
  using namespace dsrg;
  std::string msg;
  int rc = ladder_check_args(n, naux, p0, np, nh, B, t, L, msg);
  if (rc) return set_error(rc, msg.c_str());
  if (np == 0 || nh == 0) return DSRG_OK;
  const long long p3 = (long long)np * np * np;
  if (p3 > kScratchDoubles) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "dsrg_df_ladder_noalloc: np = %d needs np^3 = %lld scratch doubles, more than the fixed %lld "
             "(np <= 161); use dsrg_df_ladder",
             np, p3, kScratchDoubles);
    return set_error(DSRG_ERR_ARG, buf);
  }
  double* G = nullptr;
  rc = scratch_address(&G, msg);
  if (rc) return set_error(rc, msg.c_str());
  cudaStream_t st = (cudaStream_t)stream;
  try {
    check_cuda(cudaMemsetAsync(L, 0, (size_t)np * np * nh * nh * sizeof(double), st), "cudaMemsetAsync");
    const long long tst[4] = {(long long)np * nh * nh, (long long)nh * nh, nh, 1};
    // every batch clears its part of the shared scratch before accumulating
    ladder_core(B, n, naux, p0, np, nh, t, tst, L, G, ladder_batch_rows(np, kScratchDoubles), st, nullptr);
    check_cuda(cudaGetLastError(), "ladder launch");
    check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  } catch (const std::exception& ex) {
    return set_error(DSRG_ERR_CUDA, ex.what());
  }
  return DSRG_OK;
}

// Host-side tensor machinery (see engine.cuh).
#include "engine.cuh"
#include "ozaki.cuh"

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <stdexcept>

namespace dsrg {

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess)
    throw Error(e == cudaErrorMemoryAllocation ? DSRG_ERR_OOM : DSRG_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {
std::string gpu_key() {
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  cudaDeviceProp p{};
  check_cuda(cudaGetDeviceProperties(&p, dev), "cudaGetDeviceProperties");
  std::string name = p.name;
  for (char& c : name)
    if (c == ' ' || c == '\t') c = '_';
  return name + "/sm" + std::to_string(p.multiProcessorCount) + "/cc" + std::to_string(p.major) +
         std::to_string(p.minor);
}

std::mutex g_tc_mu;
bool g_tc_loaded = false;
std::map<std::string, std::vector<int>> g_tc;

std::string tc_key(const char* kind, const std::string& gpu, long long M, long long N, long long K, int S) {
  return std::string(kind) + " " + gpu + " " + std::to_string(M) + " " + std::to_string(N) + " " +
         std::to_string(K) + " " + std::to_string(S);
}

// file lines: kind gpu M N K slices nvals v0 v1 ...
void tc_load(const char* path) {
  g_tc_loaded = true;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char kind[64], gpu[256];
  long long M, N, K;
  int S, nv;
  while (fscanf(f, "%63s %255s %lld %lld %lld %d %d", kind, gpu, &M, &N, &K, &S, &nv) == 7) {
    if (nv < 0 || nv > 8) break;
    std::vector<int> v((size_t)nv);
    bool ok = true;
    for (int i = 0; i < nv && ok; ++i) ok = fscanf(f, "%d", &v[(size_t)i]) == 1;
    if (!ok) break;
    g_tc[tc_key(kind, gpu, M, N, K, S)] = v;
  }
  fclose(f);
}
}  // namespace

bool tune_cache_lookup(const char* kind, long long M, long long N, long long K, int slices, int nvals, int* vals) {
  const char* path = getenv("DSRG_TUNE_CACHE");
  if (!path || !*path) return false;
  const std::string key = tc_key(kind, gpu_key(), M, N, K, slices);
  std::lock_guard<std::mutex> lock(g_tc_mu);
  if (!g_tc_loaded) tc_load(path);
  auto it = g_tc.find(key);
  if (it == g_tc.end() || (int)it->second.size() != nvals) return false;
  for (int i = 0; i < nvals; ++i) vals[i] = it->second[(size_t)i];
  return true;
}

void tune_cache_store(const char* kind, long long M, long long N, long long K, int slices, int nvals,
                      const int* vals) {
  const char* path = getenv("DSRG_TUNE_CACHE");
  if (!path || !*path) return;
  const std::string gpu = gpu_key();
  std::lock_guard<std::mutex> lock(g_tc_mu);
  g_tc[tc_key(kind, gpu, M, N, K, slices)] = std::vector<int>(vals, vals + nvals);
  FILE* f = fopen(path, "a");
  if (!f) return;
  std::string line = tc_key(kind, gpu, M, N, K, slices) + " " + std::to_string(nvals);
  for (int i = 0; i < nvals; ++i) line += " " + std::to_string(vals[i]);
  fprintf(f, "%s\n", line.c_str());
  fclose(f);
}

View View::sub(const Iv* want) const {
  View o = *this;
  for (int k = 0; k < rank; ++k) {
    if (!iv[k].contains(want[k])) throw std::runtime_error("view: requested interval outside the tensor");
    o.p += (long long)(want[k].lo - iv[k].lo) * st[k];
    o.iv[k] = want[k];
  }
  return o;
}

View View::permuted(const int* perm) const {
  View o = *this;
  o.stored = 0;
  o.mask = 0;
  for (int k = 0; k < rank; ++k) {
    o.iv[k] = iv[perm[k]];
    o.st[k] = st[perm[k]];
  }
  for (int ob = 0; ob < (1 << rank); ++ob) {
    int b = 0;
    for (int k = 0; k < rank; ++k) b |= ((ob >> k) & 1) << perm[k];
    o.boff[ob] = boff[b];
    if ((stored >> b) & 1) o.stored |= 1ULL << ob;
    if ((mask >> b) & 1) o.mask |= 1ULL << ob;
  }
  return o;
}

const char* kernel_name(int id) {
  switch (id) {
    case K_GEMM: return "k_gemm<0>";
    case K_LADDER_BUILD: return "k_gemm<1>";
    case K_LADDER_CONTRACT: return "k_gemm<2>";
    case K_AXPY: return "k_axpy";
    case K_DOT: return "k_dot";
    case K_AMP: return "k_amp";
    case K_OZAKI_PACK: return "k_ozaki_pack";
    case K_CI_MATVEC: return "k_matvec";
    case K_OZAKI_MMA: return "k_ozaki_mma";
    default: return "?";
  }
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
void Workspace::prof_reset() {
  for (int i = 0; i < K_NKERNELS; ++i) {
    prof_launches[i] = 0;
    prof_ms[i] = prof_flops[i] = prof_bytes[i] = prof_xflops[i] = 0.0;
  }
  prof_steps.clear();
}

int Workspace::begin(int id, double flops, double bytes, double xflops) {
  launches++;
  if (!profiling) return -1;
  Rec r{id, nullptr, nullptr, flops, xflops < 0.0 ? flops : xflops, bytes, 0, 0, 0, tag};
  for (cudaEvent_t* e : {&r.a, &r.b}) {
    if (!ev_pool.empty()) {
      *e = ev_pool.back();
      ev_pool.pop_back();
    } else {
      check_cuda(cudaEventCreate(e), "cudaEventCreate");
    }
  }
  check_cuda(cudaEventRecord(r.a, stream), "cudaEventRecord");
  recs.push_back(r);
  return (int)recs.size() - 1;
}

void Workspace::end(int rec) {
  if (rec < 0) return;
  check_cuda(cudaEventRecord(recs[rec].b, stream), "cudaEventRecord");
}

void Workspace::prof_collect() {
  // DSRG_PROFILE_TOP=n prints the n slowest contractions of the call (stderr)
  const char* top = getenv("DSRG_PROFILE_TOP");
  std::vector<std::pair<float, int>> order;
  for (int i = 0; i < (int)recs.size(); ++i) {
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, recs[i].a, recs[i].b), "cudaEventElapsedTime");
    order.push_back({ms, i});
  }
  if (top && atoi(top) > 0) {
    std::sort(order.begin(), order.end(), [](auto& x, auto& y) { return x.first > y.first; });
    for (int i = 0; i < (int)order.size() && i < atoi(top); ++i) {
      const Rec& r = recs[order[i].second];
      fprintf(stderr, "[dsrg] %-10s %9.3f ms  M=%lld N=%lld K=%lld  %.3f TFLOP/s (executed %.3f) %.0f GB/s  %s\n",
              kernel_name(r.id), order[i].first, r.m, r.n, r.k, r.flops / (order[i].first * 1e-3) / 1e12,
              r.xflops / (order[i].first * 1e-3) / 1e12, r.bytes / (order[i].first * 1e-3) / 1e9,
              r.tag ? r.tag : "");
    }
  }
  for (auto& r : recs) {
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime");
    prof_launches[r.id]++;
    prof_ms[r.id] += ms;
    prof_flops[r.id] += r.flops;
    prof_xflops[r.id] += r.xflops;
    prof_bytes[r.id] += r.bytes;
    const char* t = r.tag ? r.tag : "";
    auto it = std::find_if(prof_steps.begin(), prof_steps.end(), [&](const StepStat& x) { return x.name == t; });
    if (it == prof_steps.end()) {
      prof_steps.push_back(StepStat{t});
      it = prof_steps.end() - 1;
    }
    it->launches++;
    it->ms += ms;
    it->flops += r.flops;
    ev_pool.push_back(r.a);
    ev_pool.push_back(r.b);
  }
  recs.clear();
  if (top && atoi(top) > 0)
    fprintf(stderr, "[dsrg] peak device memory %.3f GB, reached in step %s\n", peak_ / 1e9,
            peak_tag_ ? peak_tag_ : "");
}

namespace {
void run_gemm_fp64(Workspace& ws, const GemmArgs& g0, int kind);

// With ws.tune, a contraction of 5e6 .. 5e7 flops goes to whichever path
// was faster when its (M, N, K, slices) shape was first met: both timed on
// the caller's operands with alpha = 0 (C keeps its values), decision cached
// per device for the process.  Never timed while the stream is captured.
bool split_faster(Workspace& ws, const GemmArgs& g) {
  static std::mutex mu;
  static std::map<std::array<long long, 5>, bool> cache;
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  const std::array<long long, 5> key{g.M, g.N, g.K, (long long)ws.slices, (long long)dev};
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int stored = 0;
  if (tune_cache_lookup("route", g.M, g.N, g.K, ws.slices, 1, &stored)) {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = stored != 0;
    return stored != 0;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  check_cuda(cudaStreamIsCapturing(ws.stream, &cs), "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) return false;
  GemmArgs gz = g;
  gz.alpha = 0.0;
  const bool prof = ws.profiling;
  const long long launches = ws.launches;
  ws.profiling = false;
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
  check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  float ms[2] = {0.f, 0.f};
  for (int path = 0; path < 2; ++path) {
    for (int rep = 0; rep < 2; ++rep) {  // the second run is timed
      check_cuda(cudaEventRecord(e0, ws.stream), "cudaEventRecord");
      if (path == 0) run_gemm_fp64(ws, gz, K_GEMM);
      else ozaki_gemm(ws, gz, ws.slices, (int)K_OZAKI_MMA);
      check_cuda(cudaEventRecord(e1, ws.stream), "cudaEventRecord");
    }
    check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
    check_cuda(cudaEventElapsedTime(&ms[path], e0, e1), "cudaEventElapsedTime");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ws.profiling = prof;
  ws.launches = launches;
  const bool split = ms[1] < ms[0];
  const int v = split ? 1 : 0;
  tune_cache_store("route", g.M, g.N, g.K, ws.slices, 1, &v);
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = split;
  return split;
}

// split-precision tensor-core path for every contraction with enough work
// to pay for the operand slicing (about 40 us on the FP64 units); narrow
// outputs use 32-column tiles, short ones split k over CTAs.  With tuning,
// products of 5e6 .. 5e7 flops, and products whose shorter output side is
// at most 32 (where packing the long operand can cost more than the FP64
// work) up to 1e11 flops, take whichever path was faster on their shape;
// so do products of at least 5e7 flops with k below 32 (contractions over
// the active orbitals only), which stay on the FP64 units untuned.
bool split_route(Workspace& ws, const GemmArgs& g) {
  if (!(ws.slices > 0 && g.nbatch == 1 && ozaki_supported(g))) return false;
  const double fl = 2.0 * (double)g.M * (double)g.N * (double)g.K;
  const bool timed = ws.tune && g.A && g.B && g.C;
  if (g.K < 32) return timed && g.K >= 8 && fl >= 5e7 && split_faster(ws, g);
  const long long nmin = g.M < g.N ? g.M : g.N;
  if (timed && nmin <= 32 && fl >= 5e6 && fl < 1e11) return split_faster(ws, g);
  if (fl >= 5e7) return true;
  if (!timed || fl < 5e6) return false;
  return split_faster(ws, g);
}

// one flat launch over the output blocks of tab (npairs operand pairs)
void run_gemm_flat(Workspace& ws, const GemmArgs& g, const FlatTable& tab, int npairs) {
  const FlatPlan fp = gemm_flat_plan(g, tab.ngroups);
  const size_t O = (size_t)(g.M * g.N * g.nbatch);
  double* fpart = nullptr;
  size_t fcap = 0;
  if (fp.z > 1) fpart = ws.get((size_t)tab.ngroups * fp.z * O, fcap);
  int r = ws.begin(K_GEMM, 2.0 * (double)g.M * (double)g.N * (double)g.K * (double)g.nbatch * npairs, 0.0);
  if (r >= 0) {
    ws.recs[r].m = g.M;
    ws.recs[r].n = g.N;
    ws.recs[r].k = g.K * g.nbatch * npairs;
  }
  launch_gemm_flat(g, fp, tab, fpart, ws.stream);
  ws.end(r);
  if (fp.z > 1) ws.launches++;
  if (fpart) ws.put(fpart, fcap);
}
}  // namespace

void run_gemm(Workspace& ws, const GemmArgs& g0, int kind) {
  if (g0.M <= 0 || g0.N <= 0 || g0.K <= 0 || g0.nbatch <= 0) return;
  if (split_route(ws, g0)) {
    ozaki_gemm(ws, g0, ws.slices, kind == K_GEMM ? (int)K_OZAKI_MMA : kind);
    return;
  }
  run_gemm_fp64(ws, g0, kind);
}

namespace {
void run_gemm_fp64(Workspace& ws, const GemmArgs& g0, int kind) {
  if (kind == K_GEMM && gemm_use_flat(g0)) {
    FlatTable tab{};
    tab.a[0] = g0.A;
    tab.b[0] = g0.B;
    tab.c[0] = g0.C;
    tab.first[0] = 0;
    tab.first[1] = 1;
    tab.ngroups = 1;
    run_gemm_flat(ws, g0, tab, 1);
    return;
  }
  GemmArgs g = g0;
  // Few output tiles but a long contraction: split K over extra CTAs so the
  // whole GPU works on it (partials reduced in a fixed order).  Tiny outputs
  // go to the one-CTA-per-element kernel instead.
  int bm = 64, bn = 64;
  if (kind == K_GEMM) gemm_tile(g.M, g.N, &bm, &bn);
  const long long tiles = ((g.M + bm - 1) / bm) * ((g.N + bn - 1) / bn) * g.nbatch;
  double* part = nullptr;
  size_t cap = 0;
  const bool small = kind == K_GEMM && gemm_is_small(g);
  const bool shortk = kind == K_GEMM && gemm_is_short(g);
  if (small && g.nbatch == 1 && g.K >= 4096) {
    // one CTA per output element: split K until the GPU is covered
    long long outs = g.M * g.N;
    long long s = (4 * 152 + outs - 1) / outs;
    if (s > g.K / 2048) s = g.K / 2048;
    if (s >= 2) {
      long long kper = (g.K + s - 1) / s;
      s = (g.K + kper - 1) / kper;
      if (s >= 2) {
        part = ws.get((size_t)(s * outs), cap);
        g.splits = (int)s;
        g.kper = kper;
        g.part = part;
      }
    }
  } else if (!small && !shortk && g.nbatch == 1 && tiles < 2 * 152 && g.K >= 64) {
    long long s = (4 * 152 + tiles - 1) / tiles;
    if (s > g.K / 32) s = g.K / 32;
    if (s > 4096) s = 4096;
    const long long limit = (1LL << 25) / (g.M * g.N);
    if (s > limit) s = limit;
    if (s >= 2) {
      long long kper = (g.K + s - 1) / s;
      kper = (kper + 15) / 16 * 16;
      s = (g.K + kper - 1) / kper;
      if (s >= 2) {
        part = ws.get((size_t)(s * g.M * g.N), cap);
        g.splits = (int)s;
        g.kper = kper;
        g.part = part;
      }
    }
  }
  int r = ws.begin(kind, 2.0 * (double)g.M * (double)g.N * (double)g.K * (double)g.nbatch, 0.0);
  if (r >= 0) {
    ws.recs[r].m = g.M;
    ws.recs[r].n = g.N;
    ws.recs[r].k = g.K * g.nbatch;
  }
  launch_gemm(g, ws.stream, kind == K_LADDER_BUILD ? 1 : kind == K_LADDER_CONTRACT ? 2 : 0);
  ws.end(r);
  if (g.splits > 1) ws.launches++;  // the split-K reduction
  if (part) ws.put(part, cap);  // stream order keeps later reuse behind the reduction
}
}  // namespace

void run_axpy(Workspace& ws, const NdArgs& g, double alpha, const double* A, double* C) {
  if (g.total <= 0) return;
  int r = ws.begin(K_AXPY, 0.0, 24.0 * (double)g.total);
  launch_axpy(g, alpha, A, C, ws.stream);
  ws.end(r);
}

Workspace::~Workspace() {
  for (auto& r : recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ev_pool) cudaEventDestroy(e);
  for (auto& b : free_) cudaFree(b.p);
  if (results) cudaFree(results);
  if (dot_scratch) cudaFree(dot_scratch);
}

double* Workspace::get(size_t n, size_t& cap) {
  if (n == 0) n = 1;
  size_t best = (size_t)-1;
  int bi = -1;
  for (int i = 0; i < (int)free_.size(); ++i)
    if (free_[i].n >= n && free_[i].n < best && free_[i].n <= 2 * n + (1 << 20)) {
      best = free_[i].n;
      bi = i;
    }
  double* p;
  size_t got = n;
  if (bi >= 0) {
    p = free_[bi].p;
    got = free_[bi].n;
    free_.erase(free_.begin() + bi);
  } else {
    cudaError_t e = cudaMalloc(&p, n * sizeof(double));
    if (e != cudaSuccess) {
      // drop cached blocks and retry once
      cudaGetLastError();
      for (auto& b : free_) cudaFree(b.p);
      free_.clear();
      ++generation;
      check_cuda(cudaMalloc(&p, n * sizeof(double)), "cudaMalloc");
    }
  }
  in_use_ += got * sizeof(double);
  if (in_use_ > peak_) {
    peak_ = in_use_;
    peak_tag_ = tag;
  }
  cap = got;
  return p;
}

void Workspace::put(double* p, size_t cap) {
  if (!p) return;
  in_use_ -= cap * sizeof(double);
  free_.push_back({p, cap});
}

Tensor& Tensor::operator=(Tensor&& o) noexcept {
  if (this != &o) {
    release();
    v = o.v;
    n = o.n;
    cap = o.cap;
    ws = o.ws;
    o.v.p = nullptr;
    o.n = 0;
    o.cap = 0;
    o.ws = nullptr;
  }
  return *this;
}

Tensor::~Tensor() { release(); }

void Tensor::release() {
  if (ws && v.p) ws->put(v.p, cap);
  v.p = nullptr;
  ws = nullptr;
  n = 0;
  cap = 0;
}

Tensor make_tensor(Workspace& ws, int rank, const Iv* ivs, bool zero, bool dense) {
  Tensor t;
  t.v.rank = rank;
  const bool sparse = !dense && rank >= 4 && rank % 2 == 0;
  long long block = 1;  // elements of one spin block
  for (int k = rank - 1; k >= 0; --k) {
    t.v.iv[k] = ivs[k];
    const int L = ivs[k].len() > 0 ? ivs[k].len() : 0;
    block *= L;
  }
  for (int b = 0; b < (1 << kMaxRank); ++b) t.v.boff[b] = kNoBlock;
  long long stride = 1;
  if (sparse) {
    // spatial strides inside a block; the stored blocks one after another
    for (int k = rank - 1; k >= 0; --k) {
      t.v.st[k] = stride;
      stride *= ivs[k].len() > 0 ? ivs[k].len() : 0;
    }
    t.v.stored = conserving_mask(rank);
    long long nb = 0;
    for (int b = 0; b < (1 << rank); ++b)
      if ((t.v.stored >> b) & 1) t.v.boff[b] = nb++ * block;
    t.n = (size_t)(nb * block);
  } else {
    // spin-major slots: index (sigma, x) -> sigma * len + x
    long long ss[kMaxRank];
    for (int k = rank - 1; k >= 0; --k) {
      const int L = ivs[k].len() > 0 ? ivs[k].len() : 0;
      t.v.st[k] = stride;
      ss[k] = (long long)L * stride;
      stride *= 2LL * L;
    }
    t.v.stored = rank >= 6 ? ~0ULL : ((1ULL << (1 << rank)) - 1);
    for (int b = 0; b < (1 << rank); ++b) {
      long long o = 0;
      for (int k = 0; k < rank; ++k)
        if ((b >> k) & 1) o += ss[k];
      t.v.boff[b] = o;
    }
    t.n = (size_t)stride;
  }
  t.ws = &ws;
  t.v.p = ws.get(t.n, t.cap);
  if (zero) check_cuda(cudaMemsetAsync(t.v.p, 0, t.n * sizeof(double), ws.stream), "memset");
  t.v.mask = 0;
  return t;
}

uint64_t conserving_mask(int rank) {
  int h = rank / 2;
  uint64_t m = 0;
  for (int b = 0; b < (1 << rank); ++b) {
    int c = 0, a = 0;
    for (int k = 0; k < h; ++k) c += (b >> k) & 1;
    for (int k = h; k < rank; ++k) a += (b >> k) & 1;
    if (c == a) m |= 1ULL << b;
  }
  return m;
}

// ---------------------------------------------------------------------------
// label bookkeeping
// ---------------------------------------------------------------------------
namespace {
struct Lab {
  char c;
  Iv iv;
  int inA = -1, inB = -1, inC = -1;  // slot index in each operand
};

int find_lab(std::vector<Lab>& L, char c) {
  for (int i = 0; i < (int)L.size(); ++i)
    if (L[i].c == c) return i;
  L.push_back(Lab{c, Iv{-1000000000, 1000000000}});
  return (int)L.size() - 1;
}

void add_operand(std::vector<Lab>& L, const View& X, const char* lx, int which) {
  int r = (int)strlen(lx);
  if (r != X.rank) throw std::runtime_error(std::string("label count mismatch for ") + lx);
  for (int k = 0; k < r; ++k) {
    int i = find_lab(L, lx[k]);
    L[i].iv = isect(L[i].iv, X.iv[k]);
    if (which == 0) L[i].inA = k;
    else if (which == 1) L[i].inB = k;
    else L[i].inC = k;
  }
}

View restrict_view(const View& X, const char* lx, const std::vector<Lab>& L) {
  Iv want[kMaxRank];
  for (int k = 0; k < X.rank; ++k) {
    for (auto& l : L)
      if (l.c == lx[k]) want[k] = l.iv;
  }
  return X.sub(want);
}

inline int spin_bits(const View& X, const char* lx, const std::vector<Lab>& L, int assign) {
  int b = 0;
  for (int k = 0; k < X.rank; ++k)
    for (int i = 0; i < (int)L.size(); ++i)
      if (L[i].c == lx[k]) b |= ((assign >> i) & 1) << k;
  return b;
}

inline long long spin_off(const View& X, int bits, const char* labels = "") {
  if (!((X.stored >> bits) & 1))
    throw std::runtime_error(std::string("spin block ") + std::to_string(bits) + " of '" + labels + "' not stored");
  return X.boff[bits];
}

struct Dim {
  int e;
  long long s1, s2;
};

void fill_group(std::vector<Dim>& d, int& n, int* e, long long* s1, long long* s2) {
  if (d.size() > 4) throw std::runtime_error("contraction group with more than four dimensions");
  // slowest first; fastest (smallest first stride) last
  std::sort(d.begin(), d.end(), [](const Dim& a, const Dim& b) { return a.s1 > b.s1; });
  n = (int)d.size();
  for (int i = 0; i < n; ++i) {
    e[i] = d[i].e;
    s1[i] = d[i].s1;
    s2[i] = d[i].s2;
  }
}
}  // namespace

bool contract(Workspace& ws, double alpha, const View& A, const char* la, const View& B, const char* lb, Tensor& C,
              const char* lc) {
  std::vector<Lab> L;
  add_operand(L, A, la, 0);
  add_operand(L, B, lb, 1);
  add_operand(L, C.v, lc, 2);
  for (auto& l : L)
    if (l.iv.empty()) return false;
  if (L.size() > 16) throw std::runtime_error("too many labels");
  View a = restrict_view(A, la, L), b = restrict_view(B, lb, L), c = restrict_view(C.v, lc, L);
  // the geometry is the same for every spin assignment; only the block
  // offsets differ
  GemmArgs g{};
  g.alpha = alpha;
  {
    std::vector<Dim> M, N, K, Bt;
    for (auto& l : L) {
      int e = l.iv.len();
      bool iA = l.inA >= 0, iB = l.inB >= 0, iC = l.inC >= 0;
      if (iA && iB && iC) Bt.push_back({e, a.st[l.inA], b.st[l.inB]});
      else if (iA && iC) M.push_back({e, a.st[l.inA], c.st[l.inC]});
      else if (iB && iC) N.push_back({e, b.st[l.inB], c.st[l.inC]});
      else if (iA && iB) K.push_back({e, a.st[l.inA], b.st[l.inB]});
      else throw std::runtime_error(std::string("label only in one operand: ") + l.c);
    }
    fill_group(M, g.nM, g.eM, g.aM, g.cM);
    fill_group(N, g.nN, g.eN, g.bN, g.cN);
    fill_group(K, g.nK, g.eK, g.aK, g.bK);
    // batch labels need a C stride too
    std::sort(Bt.begin(), Bt.end(), [](const Dim& x, const Dim& y) { return x.s1 > y.s1; });
    if (Bt.size() > 4) throw std::runtime_error("too many batch labels");
    g.nB = (int)Bt.size();
    for (int i = 0; i < g.nB; ++i) {
      g.eB[i] = Bt[i].e;
      g.aB[i] = Bt[i].s1;
      g.bB[i] = Bt[i].s2;
    }
    // C strides of batch labels, in the same order
    int bi = 0;
    std::vector<std::pair<long long, long long>> cb;
    for (auto& l : L)
      if (l.inA >= 0 && l.inB >= 0 && l.inC >= 0) cb.push_back({a.st[l.inA], c.st[l.inC]});
    std::sort(cb.begin(), cb.end(), [](auto& x, auto& y) { return x.first > y.first; });
    for (auto& x : cb) g.cB[bi++] = x.second;
  }
  g.M = g.N = g.K = g.nbatch = 1;
  for (int i = 0; i < g.nM; ++i) g.M *= g.eM[i];
  for (int i = 0; i < g.nN; ++i) g.N *= g.eN[i];
  for (int i = 0; i < g.nK; ++i) g.K *= g.eK[i];
  for (int i = 0; i < g.nB; ++i) g.nbatch *= g.eB[i];
  if (g.nbatch > 65535) throw std::runtime_error("batch too large");
  struct Pair {
    long long oa, ob, oc;
  };
  std::vector<Pair> pairs;
  for (int assign = 0; assign < (1 << L.size()); ++assign) {
    int ba = spin_bits(a, la, L, assign), bb = spin_bits(b, lb, L, assign), bc = spin_bits(c, lc, L, assign);
    if (!((a.mask >> ba) & 1) || !((b.mask >> bb) & 1)) continue;
    pairs.push_back({spin_off(a, ba, la), spin_off(b, bb, lb), spin_off(c, bc, lc)});
    C.v.mask |= 1ULL << bc;
  }
  if (pairs.empty()) return false;
  g.A = a.p + pairs[0].oa;  // operands of the first spin block: timing data for the route choice
  g.B = b.p + pairs[0].ob;
  g.C = c.p + pairs[0].oc;
  if (!split_route(ws, g) && gemm_use_flat(g)) {
    // all spin blocks in flat launches: pairs that share an output block are
    // summed inside one thread, so no two CTAs of a launch write the same C
    std::stable_sort(pairs.begin(), pairs.end(), [](const Pair& x, const Pair& y) { return x.oc < y.oc; });
    FlatTable tab{};
    int np = 0;
    auto flush = [&]() {
      if (tab.ngroups == 0) return;
      tab.first[tab.ngroups] = np;
      run_gemm_flat(ws, g, tab, np);
      tab = FlatTable{};
      np = 0;
    };
    for (size_t i = 0; i < pairs.size(); ++i) {
      if (np == kFlatMaxPairs) flush();
      const bool new_group = tab.ngroups == 0 || c.p + pairs[i].oc != tab.c[tab.ngroups - 1] || np == 0;
      if (new_group) {
        tab.c[tab.ngroups] = c.p + pairs[i].oc;
        tab.first[tab.ngroups] = np;
        ++tab.ngroups;
      }
      tab.a[np] = a.p + pairs[i].oa;
      tab.b[np] = b.p + pairs[i].ob;
      ++np;
    }
    flush();
    return true;
  }
  for (auto& pr : pairs) {
    g.A = a.p + pr.oa;
    g.B = b.p + pr.ob;
    g.C = c.p + pr.oc;
    run_gemm(ws, g);
  }
  return true;
}

void axpy(Workspace& ws, double alpha, const View& A, const char* la, Tensor& C, const char* lc) {
  std::vector<Lab> L;
  add_operand(L, A, la, 0);
  add_operand(L, C.v, lc, 2);
  for (auto& l : L) {
    if (l.iv.empty()) return;
    if (l.inA < 0 || l.inC < 0) throw std::runtime_error("axpy: label sets differ");
  }
  View a = restrict_view(A, la, L), c = restrict_view(C.v, lc, L);
  NdArgs g{};
  g.nd = (int)L.size();
  g.total = 1;
  for (int i = 0; i < g.nd; ++i) {
    g.e[i] = L[i].iv.len();
    g.sa[i] = a.st[L[i].inA];
    g.sb[i] = c.st[L[i].inC];
    g.total *= g.e[i];
  }
  // every non-zero spin block of A, one launch (the C blocks are distinct)
  AxpyBlocks blk{};
  auto flush = [&]() {
    if (blk.n == 0) return;
    int r = ws.begin(K_AXPY, 0.0, 24.0 * (double)g.total * blk.n);
    launch_axpy_blocks(g, alpha, blk, ws.stream);
    ws.end(r);
    blk.n = 0;
  };
  for (int assign = 0; assign < (1 << L.size()); ++assign) {
    int ba = spin_bits(a, la, L, assign), bc = spin_bits(c, lc, L, assign);
    if (!((a.mask >> ba) & 1)) continue;
    blk.a[blk.n] = a.p + spin_off(a, ba);
    blk.c[blk.n] = c.p + spin_off(c, bc, lc);
    ++blk.n;
    C.v.mask |= 1ULL << bc;
    if (blk.n == kMaxBlocks) flush();
  }
  flush();
}

Tensor alias_permuted(Tensor& T, const int* perm) {
  Tensor a;
  a.v = T.v.permuted(perm);
  return a;  // ws == nullptr: never returned to the workspace
}

void merge_alias_mask(Tensor& T, const Tensor& alias, const int* perm) {
  for (int ab = 0; ab < (1 << T.v.rank); ++ab) {
    if (!((alias.v.mask >> ab) & 1)) continue;
    int b = 0;
    for (int k = 0; k < T.v.rank; ++k) b |= ((ab >> k) & 1) << perm[k];
    T.v.mask |= 1ULL << b;
  }
}

void dot(Workspace& ws, double alpha, const View& A, const char* la, const View& B, const char* lb) {
  std::vector<Lab> L;
  add_operand(L, A, la, 0);
  add_operand(L, B, lb, 1);
  for (auto& l : L) {
    if (l.iv.empty()) return;
    if (l.inA < 0 || l.inB < 0) throw std::runtime_error("dot: label sets differ");
  }
  View a = restrict_view(A, la, L), b = restrict_view(B, lb, L);
  NdArgs g{};
  g.nd = (int)L.size();
  g.total = 1;
  for (int i = 0; i < g.nd; ++i) {
    g.e[i] = L[i].iv.len();
    g.sa[i] = a.st[L[i].inA];
    g.sb[i] = b.st[L[i].inB];
    g.total *= g.e[i];
  }
  // all spin blocks that are non-zero in both operands: one launch, one result slot
  DotBlocks blk{};
  auto flush = [&]() {
    if (blk.n == 0) return;
    if (ws.nresults >= ws.cap_results - 3) throw std::runtime_error("out of result slots");  // last 3: the sums
    int r = ws.nresults++;
    int rec = ws.begin(K_DOT, 2.0 * (double)g.total * blk.n, 16.0 * (double)g.total * blk.n);
    launch_dot_blocks(g, alpha, blk, ws.dot_scratch, ws.dot_scratch_len, ws.dot_ticket, ws.results + r, ws.stream);
    ws.end(rec);
    blk.n = 0;
  };
  for (int assign = 0; assign < (1 << L.size()); ++assign) {
    int ba = spin_bits(a, la, L, assign), bb = spin_bits(b, lb, L, assign);
    if (!((a.mask >> ba) & 1) || !((b.mask >> bb) & 1)) continue;
    blk.a[blk.n] = a.p + spin_off(a, ba);
    blk.b[blk.n] = b.p + spin_off(b, bb);
    if (++blk.n == kMaxBlocks) flush();
  }
  flush();
}

// ---------------------------------------------------------------------------
// symmetric two-body store
// ---------------------------------------------------------------------------
namespace {
// X[w0,w1,w2,w3] = sign * T[w_perm0, w_perm1, w_perm2, w_perm3]
const int kOps[8][4] = {{0, 1, 2, 3}, {1, 0, 2, 3}, {0, 1, 3, 2}, {1, 0, 3, 2},
                        {2, 3, 0, 1}, {3, 2, 0, 1}, {2, 3, 1, 0}, {3, 2, 1, 0}};
const double kSign[8] = {1, -1, -1, 1, 1, -1, -1, 1};
}  // namespace

bool Sym2::resolve(const Iv* want, View& out, double& sign) const {
  for (auto& t : cls) {
    for (int o = 0; o < 8; ++o) {
      const int* pm = kOps[o];
      bool ok = true;
      for (int k = 0; k < 4 && ok; ++k) ok = t.v.iv[k].contains(want[pm[k]]);
      if (!ok) continue;
      // request slot j is class slot k with pm[k] == j
      int inv[4];
      for (int k = 0; k < 4; ++k) inv[pm[k]] = k;
      View v = t.v.permuted(inv).sub(want);
      out = v;
      sign = kSign[o];
      return true;
    }
  }
  return false;
}

static void x2_request(const char* lx, const std::vector<Lab>& L, Iv* want) {
  for (int k = 0; k < 4; ++k) {
    want[k] = Iv{-1000000000, 1000000000};
    for (auto& l : L)
      if (l.c == lx[k]) want[k] = l.iv;
  }
}

// W placed as an operator: identity on [P,P,H,H] or its Hermitian image
View w_place(const Tensor& W, int herm) {
  static const int hp[4] = {2, 3, 0, 1};
  if (!herm) return W.v;
  return W.v.permuted(hp);
}

static bool v_view(const Op2& X, const Iv* want, View& xv, double& sg, const char* what, bool skip) {
  if (!X.V || X.cv == 0.0) return false;
  for (int k = 0; k < 4; ++k)
    if (want[k].lo < -100000000) throw std::runtime_error(std::string("unconstrained two-body label in ") + what);
  if (X.V->resolve(want, xv, sg)) return true;
  if (skip || X.V->make) return false;  // v_slabs serves classes that are not stored
  char buf[256];
  snprintf(buf, sizeof buf, "no stored two-body class covers [%d,%d)x[%d,%d)x[%d,%d)x[%d,%d) for %s", want[0].lo,
           want[0].hi, want[1].lo, want[1].hi, want[2].lo, want[2].hi, want[3].lo, want[3].hi, what);
  throw std::runtime_error(buf);
}

// V on the intervals `want` built on demand, one slab of the first slot at a
// time; each slab's view goes to use().  The engine intersects label
// intervals across operands, so every slab restricts the other operand and
// the output to its own rows.  False when V keeps all its classes.
template <class F>
static bool v_slabs(const Op2& X, const Iv* want, F&& use) {
  if (!X.V || !X.V->make || X.cv == 0.0) return false;
  for (int k = 0; k < 4; ++k)
    if (want[k].empty()) return true;
  // per row of the first slot: the (pr|qs) and (ps|qr) blocks and six spin blocks
  long long row = 8;
  for (int k = 1; k < 4; ++k) row *= want[k].len();
  long long rows = X.V->max_elems / row;
  if (rows < 1) rows = 1;
  for (int lo = want[0].lo; lo < want[0].hi; lo += (int)rows) {
    const int hi = (long long)lo + rows < want[0].hi ? lo + (int)rows : want[0].hi;
    Iv sub[4] = {Iv{lo, hi}, want[1], want[2], want[3]};
    Tensor slab = X.V->make(sub);
    use(slab.v);
  }
  return true;
}

bool contract_x2(Workspace& ws, double alpha, const Op2& X, const char* lx, const View& B, const char* lb, Tensor& C,
                 const char* lc, bool skip_v) {
  std::vector<Lab> L;
  add_operand(L, B, lb, 1);
  add_operand(L, C.v, lc, 2);
  for (auto& l : L)
    if (l.iv.empty()) return false;
  bool any = false;
  Iv want[4];
  x2_request(lx, L, want);
  View xv;
  double sg;
  if (!skip_v) {
    if (v_view(X, want, xv, sg, lx, false))
      any |= contract(ws, alpha * X.cv * sg, xv, lx, B, lb, C, lc);
    else
      v_slabs(X, want, [&](const View& v) { any |= contract(ws, alpha * X.cv, v, lx, B, lb, C, lc); });
  }
  if (X.W && X.cw != 0.0)
    for (int herm = 0; herm < 2; ++herm) any |= contract(ws, alpha * X.cw, w_place(*X.W, herm), lx, B, lb, C, lc);
  return any;
}

bool contract_x2_left(Workspace& ws, double alpha, const View& A, const char* la, const Op2& X, const char* lx,
                      Tensor& C, const char* lc) {
  std::vector<Lab> L;
  add_operand(L, A, la, 0);
  add_operand(L, C.v, lc, 2);
  for (auto& l : L)
    if (l.iv.empty()) return false;
  bool any = false;
  Iv want[4];
  x2_request(lx, L, want);
  View xv;
  double sg;
  if (v_view(X, want, xv, sg, lx, false))
    any |= contract(ws, alpha * X.cv * sg, A, la, xv, lx, C, lc);
  else
    v_slabs(X, want, [&](const View& v) { any |= contract(ws, alpha * X.cv, A, la, v, lx, C, lc); });
  if (X.W && X.cw != 0.0)
    for (int herm = 0; herm < 2; ++herm) any |= contract(ws, alpha * X.cw, A, la, w_place(*X.W, herm), lx, C, lc);
  return any;
}

void dot_x2(Workspace& ws, double alpha, const Op2& X, const Tensor& U) {
  for (int k = 0; k < 4; ++k)
    if (U.v.iv[k].empty()) return;
  View xv;
  double sg;
  if (v_view(X, U.v.iv, xv, sg, "scalar term", false))
    dot(ws, alpha * X.cv * sg, xv, "pqrs", U.v, "pqrs");
  else
    v_slabs(X, U.v.iv, [&](const View& v) { dot(ws, alpha * X.cv, v, "pqrs", U.v, "pqrs"); });
  if (X.W && X.cw != 0.0)
    for (int herm = 0; herm < 2; ++herm) dot(ws, alpha * X.cw, w_place(*X.W, herm), "pqrs", U.v, "pqrs");
}

void fetch_x2(Workspace& ws, double alpha, const Op2& X, Tensor& out) {
  for (int k = 0; k < 4; ++k)
    if (out.v.iv[k].empty()) return;
  View xv;
  double sg;
  if (v_view(X, out.v.iv, xv, sg, "materialised class", false))
    axpy(ws, alpha * X.cv * sg, xv, "abcd", out, "abcd");
  else
    v_slabs(X, out.v.iv, [&](const View& v) { axpy(ws, alpha * X.cv, v, "abcd", out, "abcd"); });
  if (X.W && X.cw != 0.0)
    for (int herm = 0; herm < 2; ++herm) axpy(ws, alpha * X.cw, w_place(*X.W, herm), "abcd", out, "abcd");
}

}  // namespace dsrg

// First-order aavv amplitudes with Dyall's zeroth-order Hamiltonian on the
// GPU (App. B, Eq. t2_aavv), at s -> infinity.  For virtual spin orbitals
// e, f and active u, v (X2[p,q,r,s] multiplies {a+_p a+_q a_s a_r}):
//   0 = V[e,f,u,v] - D t[e,f,u,v] - 1/2 sum_xy Va[x,y,u,v] t[e,f,x,y]
//                                 + sum_xyz Va[x,y,u,v] t[e,f,x,z] g[y,z],
// D = eps_u + eps_v - eps_e - eps_f, Va the all-active block of V, g the
// active 1-RDM.  With t[e,f,:,:] a row vector over the active pairs the
// coupling is one matrix, t K with
//   K[(x,z),(u,v)] = -1/2 Va[x,z,u,v] + sum_y g[y,z] Va[x,y,u,v],
// the same for every virtual pair, so an iteration is one product of the
// amplitudes (pairs x m^2) with K (m^2 x m^2) plus an element-wise update.
// The system is solved by Jacobi iteration preconditioned by the shifted
// denominator, the exact diagonal of the system:
//   Ds = D + Va[u,v,u,v] - sum_y (Va[u,y,u,v] g[y,v] - Va[v,y,u,v] g[y,u]).
// Without the renormalisation of the DSRG (s finite) small shifted
// denominators (intruders) can stop it converging; the call reports the
// residual, the pairs that did not converge and the smallest |Ds| instead
// of hiding them.
#include <cmath>
#include <cstdint>
#include <stdexcept>

#include "dsrg_impl.cuh"

namespace dsrg {
namespace {

constexpr int DY_T = 256;

// non-negative doubles order like their bit patterns
__device__ __forceinline__ void atomic_max_nonneg(double* a, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_nonneg(double* a, double v) {
  atomicMin(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

// K (m^2 x m^2) and the two-body part of the diagonal, diag[u,v] (m x m)
__global__ void k_dy_coupling(int m, const double* __restrict__ Va, const double* __restrict__ g,
                              double* __restrict__ K, double* __restrict__ diag) {
  const long long m2 = (long long)m * m, m3 = m2 * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m2 * m2;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / m2, c = i - r * m2;  // r = (x, z), c = (u, v)
    const int x = (int)(r / m), z = (int)(r % m);
    double k = -0.5 * Va[x * m3 + z * m2 + c];
    for (int y = 0; y < m; ++y) k += g[y * m + z] * Va[x * m3 + y * m2 + c];
    K[i] = k;
    if (i < m2) {
      const int u = (int)(i / m), v = (int)(i % m);
      double d = Va[u * m3 + v * m2 + u * m + v];
      for (int y = 0; y < m; ++y)
        d -= Va[u * m3 + y * m2 + u * m + v] * g[y * m + v] - Va[v * m3 + y * m2 + u * m + v] * g[y * m + u];
      diag[i] = d;
    }
  }
}

// orbital energies of virtual spin orbital e and active spin orbital u
__device__ __forceinline__ double eps_vir(const double* eps, int nc, int na, int nv, int e) {
  return eps[nc + na + e % nv];
}
__device__ __forceinline__ double eps_act(const double* eps, int nc, int na, int u) { return eps[nc + u % na]; }

struct DyDims {
  long long pairs;  // (2 nv)^2 virtual spin-orbital pairs
  int m;            // 2 na active spin orbitals
  int nc, na, nv;
};

// R = V - D t + W (W = t K); t += R / Ds off the u = v diagonal; max |R|.
// One CTA per virtual pair at a time (its m^2 elements are contiguous).  The
// FP64 pipe is the narrow resource here, so per active pair dd = eps_u +
// eps_v and ds = dd + diag come precomputed (pd[uv], pd[m2 + uv]) and the
// preconditioner's reciprocal is taken in FP32: it scales the step only,
// the residual that decides convergence stays FP64.
__global__ void __launch_bounds__(DY_T) k_dy_update(const DyDims d, const double* __restrict__ eps,
                                                     const double* __restrict__ Vs, const double* __restrict__ W,
                                                     const double* __restrict__ pd, double* __restrict__ t,
                                                     double* __restrict__ rmax, int update) {
  const int m2 = d.m * d.m;
  float mx = 0.0f;
  for (long long p = blockIdx.x; p < d.pairs; p += gridDim.x) {
    const int e = (int)(p / (2 * d.nv)), f = (int)(p - (long long)e * 2 * d.nv);
    const double Ef = eps_vir(eps, d.nc, d.na, d.nv, e) + eps_vir(eps, d.nc, d.na, d.nv, f);
    const long long base = p * m2;
    for (int uv = threadIdx.x; uv < m2; uv += DY_T) {
      const double dd = pd[uv];
      if (dd != dd) continue;  // u = v: marked NaN
      const long long i = base + uv;
      const double ti = t[i];
      const double R = fma(-(dd - Ef), ti, Vs[i] + W[i]);
      const float a = fabsf((float)R);
      mx = a == a ? fmaxf(mx, a) : INFINITY;  // a NaN residual counts as divergence
      if (update) t[i] = fma(R, (double)(1.0f / (float)(pd[m2 + uv] - Ef)), ti);
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
  // float max, widened: |R| is compared with the tolerance after the loop
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(rmax, (double)mx);
}

// pd[uv] = eps_u + eps_v (NaN on u = v), pd[m2 + uv] = pd[uv] + diag[uv]
__global__ void k_dy_pairs(int m, int nc, int na, const double* __restrict__ eps, const double* __restrict__ diag,
                           double* __restrict__ pd) {
  const int m2 = m * m;
  for (int uv = blockIdx.x * blockDim.x + threadIdx.x; uv < m2; uv += gridDim.x * blockDim.x) {
    const int u = uv / m, v = uv - u * m;
    const double dd = u == v ? (double)NAN : eps_act(eps, nc, na, u) + eps_act(eps, nc, na, v);
    pd[uv] = dd;
    pd[m2 + uv] = dd + diag[uv];
  }
}

// One warp per virtual pair: its largest |R| against thr (pairs above are
// counted), the smallest |Ds| and the number below 1e-2 over u != v, and
// the largest |V|
struct DyStats {
  double min_ds, max_src;
  unsigned long long bad_pairs, small_ds;
};

__global__ void __launch_bounds__(DY_T) k_dy_stats(const DyDims d, const double* __restrict__ eps,
                                                    const double* __restrict__ Vs, const double* __restrict__ W,
                                                    const double* __restrict__ diag, const double* __restrict__ t,
                                                    double thr, DyStats* st) {
  const long long m2 = (long long)d.m * d.m;
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * blockDim.x / 32;
  for (long long p = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; p < d.pairs; p += nwarps) {
    const int e = (int)(p / (2 * d.nv)), f = (int)(p % (2 * d.nv));
    const double Ef = eps_vir(eps, d.nc, d.na, d.nv, e) + eps_vir(eps, d.nc, d.na, d.nv, f);
    double rmax = 0.0, dmin = INFINITY, vmax = 0.0;
    unsigned long long small = 0;
    for (int uv = lane; uv < m2; uv += 32) {
      const int u = uv / d.m, v = uv % d.m;
      if (u == v) continue;
      const long long i = p * m2 + uv;
      const double D = eps_act(eps, d.nc, d.na, u) + eps_act(eps, d.nc, d.na, v) - Ef;
      const double a = fabs(Vs[i] - D * t[i] + W[i]);
      rmax = a == a ? fmax(rmax, a) : INFINITY;
      const double ds = fabs(D + diag[uv]);
      dmin = fmin(dmin, ds);
      small += ds < 1e-2 ? 1 : 0;
      vmax = fmax(vmax, fabs(Vs[i]));
    }
    for (int o = 16; o > 0; o >>= 1) {
      rmax = fmax(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
      dmin = fmin(dmin, __shfl_down_sync(0xffffffffu, dmin, o));
      vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
      small += __shfl_down_sync(0xffffffffu, small, o);
    }
    if (lane == 0) {
      if (!(rmax <= thr)) atomicAdd(&st->bad_pairs, 1ULL);
      if (small) atomicAdd(&st->small_ds, small);
      if (dmin < INFINITY) atomic_min_nonneg(&st->min_ds, dmin);
      atomic_max_nonneg(&st->max_src, vmax);
    }
  }
}

// a workspace block returned when it goes out of scope
struct DyBuf {
  Workspace& ws;
  double* p = nullptr;
  size_t cap = 0;
  DyBuf(Workspace& w, size_t n) : ws(w) { p = ws.get(n ? n : 1, cap); }
  ~DyBuf() { ws.put(p, cap); }
  DyBuf(const DyBuf&) = delete;
  DyBuf& operator=(const DyBuf&) = delete;
};

inline unsigned dy_grid(long long n, int t) {
  long long g = (n + t - 1) / t;
  if (g > 152LL * 32) g = 152LL * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// W = t K: rows of t are the virtual pairs, K is m^2 x m^2 (row-major)
static void dy_product(Handle& h, const double* t, const double* K, double* W, long long pairs, int m2) {
  check_cuda(cudaMemsetAsync(W, 0, (size_t)pairs * m2 * sizeof(double), h.ws.stream), "cudaMemsetAsync (dyall)");
  GemmArgs g{};
  g.A = t;
  g.B = K;
  g.C = W;
  g.alpha = 1.0;
  g.nM = g.nN = g.nK = 1;
  g.eM[0] = (int)pairs;
  g.aM[0] = m2;
  g.cM[0] = m2;
  g.eN[0] = m2;
  g.bN[0] = 1;
  g.cN[0] = 1;
  g.eK[0] = m2;
  g.aK[0] = 1;
  g.bK[0] = m2;
  g.M = pairs;
  g.N = m2;
  g.K = m2;
  g.nbatch = 1;
  run_gemm(h.ws, g);
}

DyallResult dyall_aavv(Handle& h, double tol, int max_iter) {
  Workspace& ws = h.ws;
  cudaStream_t st = ws.stream;
  DyallResult out;
  h.t_aavv.release();
  if (h.na == 0 || h.nv == 0) {
    out.converged = 1;
    return out;
  }
  ProfTag tag_(ws, "dyall-aavv");
  const int m = 2 * h.na, m2 = m * m;
  const long long pairs = 4LL * h.nv * h.nv;
  if (pairs >= (1LL << 31)) throw Error(DSRG_ERR_ARG, "dyall: too many virtual pairs");
  // V[e,f,u,v], Va and gamma on the active block, dense spin-major
  Iv vvaa[4] = {h.V, h.V, h.A, h.A};
  Tensor Vs = make_tensor(ws, 4, vvaa, true, true);
  {
    Tensor Vc = vclass(h, vvaa, 1.0);
    axpy(ws, 1.0, Vc.v, "abcd", Vs, "abcd");
  }
  Iv aaaa[4] = {h.A, h.A, h.A, h.A};
  Tensor Va = make_tensor(ws, 4, aaaa, true, true);
  {
    Tensor Vc = vclass(h, aaaa, 1.0);
    axpy(ws, 1.0, Vc.v, "abcd", Va, "abcd");
  }
  Iv aa[2] = {h.A, h.A};
  Tensor G = make_tensor(ws, 2, aa, true, true);
  axpy(ws, 1.0, h.gam.v.sub(aa), "ab", G, "ab");
  DyBuf K(ws, (size_t)m2 * m2), diag(ws, (size_t)m2), pd(ws, 2 * (size_t)m2);
  k_dy_coupling<<<dy_grid((long long)m2 * m2, DY_T), DY_T, 0, st>>>(m, Va.v.p, G.v.p, K.p, diag.p);
  k_dy_pairs<<<dy_grid(m2, DY_T), DY_T, 0, st>>>(m, h.nc, h.na, h.eps, diag.p, pd.p);
  check_cuda(cudaGetLastError(), "dyall launch");
  ws.launches += 2;
  // amplitudes, product buffer, reductions
  h.t_aavv = make_tensor(ws, 4, vvaa, true, true);
  double* t = h.t_aavv.v.p;
  DyBuf Wb(ws, (size_t)pairs * m2), sb(ws, 16);
  double* W = Wb.p;
  double* scr = sb.p;
  DyDims d{pairs, m, h.nc, h.na, h.nv};
  const long long n = pairs * m2;
  double vmax = 0.0;
  {
    int it = 0;
    double r = INFINITY;
    for (; it < max_iter; ++it) {
      dy_product(h, t, K.p, W, pairs, m2);
      check_cuda(cudaMemsetAsync(scr, 0, sizeof(double), st), "cudaMemsetAsync (dyall)");
      const int rec = ws.begin(K_AMP, 0.0, 32.0 * (double)n);
      k_dy_update<<<dy_grid(pairs * DY_T, DY_T), DY_T, 0, st>>>(d, h.eps, Vs.v.p, W, pd.p, t, scr, 1);
      ws.end(rec);
      check_cuda(cudaGetLastError(), "dyall launch");
      check_cuda(cudaMemcpyAsync(&r, scr, sizeof r, cudaMemcpyDeviceToHost, st), "copy residual");
      check_cuda(cudaStreamSynchronize(st), "sync");
      if (it == 0) vmax = r;  // t = 0: the residual is V itself
      if (!(r <= 1e8 * (vmax > 0.0 ? vmax : 1.0))) break;  // diverging
      if (r <= tol * vmax) break;
    }
    out.iterations = it < max_iter ? it + 1 : max_iter;
    // residual of the final amplitudes, per pair
    dy_product(h, t, K.p, W, pairs, m2);
    DyStats init{INFINITY, 0.0, 0ULL, 0ULL};
    DyStats* dst = reinterpret_cast<DyStats*>(scr + 2);
    check_cuda(cudaMemcpyAsync(dst, &init, sizeof init, cudaMemcpyHostToDevice, st), "copy stats");
    check_cuda(cudaMemsetAsync(scr, 0, sizeof(double), st), "cudaMemsetAsync (dyall)");
    k_dy_update<<<dy_grid(pairs * DY_T, DY_T), DY_T, 0, st>>>(d, h.eps, Vs.v.p, W, pd.p, t, scr, 0);
    k_dy_stats<<<dy_grid(pairs * 32, DY_T), DY_T, 0, st>>>(d, h.eps, Vs.v.p, W, diag.p, t, tol * vmax, dst);
    check_cuda(cudaGetLastError(), "dyall launch");
    ws.launches += 3;
    DyStats hs{};
    check_cuda(cudaMemcpyAsync(&out.max_residual, scr, sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
    check_cuda(cudaMemcpyAsync(&hs, dst, sizeof hs, cudaMemcpyDeviceToHost, st), "copy stats");
    check_cuda(cudaStreamSynchronize(st), "sync");
    out.max_source = hs.max_src;
    out.pairs_not_converged = (long long)hs.bad_pairs;
    out.min_shifted_denominator = hs.min_ds;
    out.small_denominators = (long long)hs.small_ds;
    out.converged = out.max_residual <= tol * hs.max_src ? 1 : 0;
  }
  return out;
}

}  // namespace dsrg

// One-step relaxed DSRG-MRPT2/PT3 energies on the GPU (Eq. E_relaxed, App. A).
//
// The energy driver (run with Handle::relax) leaves the all-active blocks of
// the summed transformed Hamiltonian Hbar^[k]_{1,2} relative to E0.  Here:
//   1. App. A, Eq. Hbar_DNO with the core folded (Eq. c0_cas cancels the
//      core terms): the active-space operator in true-vacuum order,
//        E_s + sum c^u_v a+_u a_v + 1/4 sum w^{uv}_{xy} a+_u a+_v a_y a_x,
//        E_s = Hbar_0 - sum Hbar^u_v g^u_v
//              - sum Hbar^{uv}_{xy} (1/4 g^{uv}_{xy} - g^u_x g^v_y),
//        c^u_v = Hbar^u_v - sum_xy Hbar^{ux}_{vy} g^x_y,  w = Hbar^{uv}_{xy},
//      g^{uv}_{xy} = lambda^{uv}_{xy} + g^u_x g^v_y - g^u_y g^v_x;
//   2. its matrix over the determinants with the reference's alpha and beta
//      active electron counts (Slater's rules on occupation bit strings);
//   3. its lowest eigenvalue (Eq. energy_relaxed) by Lanczos iteration with
//      full reorthogonalisation (C. Lanczos, J. Res. Natl. Bur. Stand. 45,
//      255 (1950)); the tridiagonal eigenvalue by Sturm-sequence bisection
//      (Barth, Martin and Wilkinson, Numer. Math. 9, 386 (1967)) and its
//      vector by inverse iteration, shifted just below the eigenvalue so the
//      LDL^T factorisation is of a positive definite matrix.
// Active spin orbitals are numbered alpha 0..na-1, beta na..2na-1 (the
// dense spin-major layout), so a determinant is a 2na-bit string.
#include <cmath>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "dsrg_impl.cuh"

namespace dsrg {
namespace {

constexpr int RX_T = 256;
constexpr int LZ_MAX_STEPS = 300;  // Krylov dimension per Lanczos run
constexpr int LZ_MAX_RUNS = 6;     // restarts from the Ritz vector
constexpr long long RELAX_MAX_DET = 20000;

// fixed-order sum of one value per thread of an RX_T-thread block
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = RX_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void k_active_diagonal(int nc, int na, const double* __restrict__ eps, double* __restrict__ h1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * na) return;
  h1[(long long)i * 2 * na + i] += eps[nc + i % na];
}

// step 1 (one CTA): E_s and c from h1 [m][m], h2 [m]^4, g1 [m][m], l2 [m]^4;
// Hbar_0 is the sum of the first nres energy components at res
__global__ void __launch_bounds__(RX_T) k_dno(int m, const double* __restrict__ h1, const double* __restrict__ h2,
                                              const double* __restrict__ g1, const double* __restrict__ l2,
                                              const double* __restrict__ res, int nres, double* __restrict__ Es,
                                              double* __restrict__ c) {
  __shared__ double sh[RX_T];
  const long long m2 = (long long)m * m, m4 = m2 * m2;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < m2; i += RX_T) acc += h1[i] * g1[i];
  for (long long i = threadIdx.x; i < m4; i += RX_T) {
    const int y = (int)(i % m), x = (int)((i / m) % m), v = (int)((i / m2) % m), u = (int)(i / (m2 * m));
    const double gg = g1[u * m + x] * g1[v * m + y];
    const double g2 = l2[i] + gg - g1[u * m + y] * g1[v * m + x];
    acc += h2[i] * (0.25 * g2 - gg);
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    double h0 = 0.0;
    for (int k = 0; k < nres; ++k) h0 += res[k];
    *Es = h0 - s;
  }
  for (long long i = threadIdx.x; i < m2; i += RX_T) {
    const int u = (int)(i / m), v = (int)(i % m);
    double t = h1[i];
    for (int x = 0; x < m; ++x)
      for (int y = 0; y < m; ++y) t -= h2[(((long long)u * m + x) * m + v) * m + y] * g1[x * m + y];
    c[i] = t;
  }
}

__device__ __forceinline__ int below(uint32_t d, int x) { return __popc(d & ((1u << x) - 1u)); }

// step 2: H[I][J] = <D_I| E_s + c + w |D_J>, one thread per element
__global__ void k_ci_matrix(long long ndet, const uint32_t* __restrict__ dets, int m, const double* __restrict__ Es,
                            const double* __restrict__ c, const double* __restrict__ w, double* __restrict__ H) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= ndet * ndet) return;
  const long long I = idx / ndet, J = idx - I * ndet;
  const uint32_t dI = dets[I], dJ = dets[J], diff = dI ^ dJ;
  const int nd = __popc(diff);
  const long long m2 = (long long)m * m, m3 = m2 * m;
  double val = 0.0;
  if (nd == 0) {
    val = *Es;
    for (uint32_t a = dJ; a; a &= a - 1) {
      const int k = __ffs(a) - 1;
      val += c[k * m + k];
      for (uint32_t b = a & (a - 1); b; b &= b - 1) {  // pairs k < l
        const int l = __ffs(b) - 1;
        val += w[k * m3 + l * m2 + k * m + l];
      }
    }
  } else if (nd == 2) {  // a+_q a_p: p occupied in J only, q in I only
    const int p = __ffs(diff & dJ) - 1, q = __ffs(diff & dI) - 1;
    double t = c[q * m + p];
    for (uint32_t a = dJ & dI; a; a &= a - 1) {
      const int k = __ffs(a) - 1;
      t += w[q * m3 + k * m2 + p * m + k];
    }
    const int s = below(dJ, p) + below(dJ ^ (1u << p), q);
    val = (s & 1) ? -t : t;
  } else if (nd == 4) {  // a+_q1 a+_q2 a_p2 a_p1, p1 < p2 in J only, q1 < q2 in I only
    const uint32_t pj = diff & dJ, qi = diff & dI;
    const int p1 = __ffs(pj) - 1, p2 = __ffs(pj & (pj - 1)) - 1;
    const int q1 = __ffs(qi) - 1, q2 = __ffs(qi & (qi - 1)) - 1;
    uint32_t d = dJ;
    int s = below(d, p1);
    d ^= 1u << p1;
    s += below(d, p2);
    d ^= 1u << p2;
    s += below(d, q2);
    d ^= 1u << q2;
    s += below(d, q1);
    const double t = w[q1 * m3 + q2 * m2 + p1 * m + p2];
    val = (s & 1) ? -t : t;
  }
  H[idx] = val;
}

// Lanczos state (device)
struct LzState {
  int done;    // the Krylov space stopped growing or reached its limit
  int steps;   // size of the tridiagonal matrix
  double hmax; // largest |alpha|, beta seen (scale of the breakdown test)
  double lambda, resid;
};

// y = H x, one warp per row
__global__ void k_matvec(long long n, const double* __restrict__ H, const double* __restrict__ x,
                         double* __restrict__ y, const LzState* st) {
  if (st && st->done) return;
  const long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* hr = H + row * n;
  double s = 0.0;
  for (long long j = lane; j < n; j += 32) s += hr[j] * x[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

// out[k] = V[k] . x for k < nv (V rows of length n), one CTA per k
__global__ void __launch_bounds__(RX_T) k_dots(long long n, const double* V, const double* x, double* out,
                                               const LzState* st) {
  if (st && st->done) return;
  __shared__ double sh[RX_T];
  const double* v = V + blockIdx.x * n;
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += RX_T) s += v[i] * x[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// x -= sum_{k < nv} coef[k] V[k]
__global__ void k_subtract(long long n, int nv, const double* __restrict__ V, const double* __restrict__ coef,
                           double* __restrict__ x, const LzState* st) {
  if (st && st->done) return;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = x[i];
  for (int k = 0; k < nv; ++k) t -= coef[k] * V[k * n + i];
  x[i] = t;
}

// alpha_j, beta_j = |w|, breakdown / length test
__global__ void k_lz_next(int j, int mmax, const double* coef, const double* nrm2, double* alpha, double* beta,
                          LzState* st) {
  if (st->done) return;
  const double a = coef[j], b = sqrt(fmax(*nrm2, 0.0));
  alpha[j] = a;
  beta[j] = b;
  st->hmax = fmax(st->hmax, fmax(fabs(a), b));
  st->steps = j + 1;
  if (b <= 1e-12 * st->hmax || j + 1 >= mmax) st->done = 1;
}

// V[j + 1] = w / beta_j
__global__ void k_lz_scale(long long n, int j, const double* __restrict__ w, const double* __restrict__ beta,
                           double* __restrict__ V, const LzState* st) {
  if (st->done) return;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) V[(j + 1) * n + i] = w[i] / beta[j];
}

// number of eigenvalues of the tridiagonal (a, b) below x (Sturm sequence)
__device__ int sturm_count(int k, const double* a, const double* b, double x) {
  int cnt = 0;
  double q = a[0] - x;
  for (int i = 0;; ++i) {
    if (q < 0.0) ++cnt;
    if (i + 1 >= k) break;
    if (q == 0.0) q = 1e-300;
    q = (a[i + 1] - x) - b[i] * b[i] / q;
  }
  return cnt;
}

// lowest eigenvalue of the tridiagonal matrix and its unit eigenvector y
// (single thread; work: 3 k doubles)
__global__ void k_lz_tridiag(const double* __restrict__ a, const double* __restrict__ b, LzState* st,
                             double* __restrict__ y, double* __restrict__ work) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = st->steps;
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 4000; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (sturm_count(k, a, b, mid) >= 1) hi = mid;
    else lo = mid;
  }
  const double lam = 0.5 * (lo + hi);
  // inverse iteration with the shift sigma just below lam: T - sigma is
  // positive definite, so its LDL^T factorisation needs no pivoting
  const double scale = fmax(st->hmax, 1e-300);
  const double sigma = lam - 1e-10 * scale;
  double* d = work;
  double* l = work + k;
  double* z = work + 2 * k;
  d[0] = a[0] - sigma;
  for (int i = 0; i + 1 < k; ++i) {
    l[i] = b[i] / d[i];
    d[i + 1] = (a[i + 1] - sigma) - l[i] * b[i];
  }
  for (int i = 0; i < k; ++i) y[i] = 1.0;
  for (int it = 0; it < 4; ++it) {
    // L z' = y, D z'' = z', L^T z = z''
    z[0] = y[0];
    for (int i = 1; i < k; ++i) z[i] = y[i] - l[i - 1] * z[i - 1];
    for (int i = 0; i < k; ++i) z[i] /= d[i];
    for (int i = k - 2; i >= 0; --i) z[i] -= l[i] * z[i + 1];
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += z[i] * z[i];
    nrm = sqrt(nrm);
    if (!(nrm > 0.0) || !isfinite(nrm)) {  // degenerate scale (e.g. a zero matrix): first basis vector
      for (int i = 0; i < k; ++i) y[i] = i == 0 ? 1.0 : 0.0;
      break;
    }
    for (int i = 0; i < k; ++i) y[i] = z[i] / nrm;
  }
  st->lambda = lam;
}

// x = sum_k y[k] V[k]
__global__ void k_ritz(long long n, int k, const double* __restrict__ V, const double* __restrict__ y,
                       double* __restrict__ x) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = 0.0;
  for (int q = 0; q < k; ++q) t += y[q] * V[q * n + i];
  x[i] = t;
}

// r = Hx - lambda x (Hx given in r)
__global__ void k_resid(long long n, const double* __restrict__ x, double* __restrict__ r, const LzState* st) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) r[i] -= st->lambda * x[i];
}

// V[0] = x / |x|, state reset for a new run
__global__ void k_lz_start(long long n, const double* __restrict__ x, const double* __restrict__ nrm2,
                           double* __restrict__ V, LzState* st) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) V[i] = x[i] / sqrt(*nrm2);
  if (i == 0) {
    st->done = 0;
    st->steps = 0;
    st->hmax = 0.0;
  }
}

// start vector: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) of the
// determinant index, mapped to [-1, 1)
__global__ void k_lz_seed(long long n, double* __restrict__ x) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ULL + 0x2545F4914F6CDD1DULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

inline unsigned grid_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

std::vector<uint32_t> strings(int na, int nel) {
  std::vector<uint32_t> out;
  for (uint32_t b = 0; b < (1u << na); ++b)
    if (__builtin_popcount(b) == nel) out.push_back(b);
  return out;  // ascending
}

}  // namespace

void launch_active_diagonal(int nc, int na, const double* eps, double* h1, cudaStream_t st) {
  if (na <= 0) return;
  k_active_diagonal<<<1, 64, 0, st>>>(nc, na, eps, h1);
}

long long relax_ndet(int na, int n_alpha, int n_beta) {
  auto binom = [](int n, int k) {
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
  };
  if (n_alpha < 0 || n_beta < 0 || n_alpha > na || n_beta > na) return 0;
  return binom(na, n_alpha) * binom(na, n_beta);
}

namespace {
// a workspace block returned when it goes out of scope
struct Scratch {
  Workspace& ws;
  double* p = nullptr;
  size_t cap = 0;
  Scratch(Workspace& w, size_t n) : ws(w) { p = ws.get(n ? n : 1, cap); }
  ~Scratch() { ws.put(p, cap); }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
};

__global__ void k_add(long long n, const double* __restrict__ a, double* __restrict__ b) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] += a[i];
}
}  // namespace

RelaxResult relaxed_ci(Handle& h, int order, int n_alpha, int n_beta) {
  Workspace& ws = h.ws;
  cudaStream_t st = ws.stream;
  const int na = h.na, m = 2 * na;
  const long long ndet = relax_ndet(na, n_alpha, n_beta);
  if (ndet < 1 || ndet > RELAX_MAX_DET)
    throw Error(DSRG_ERR_ARG, "relaxed: the determinant space is empty or larger than 20000");
  const double* res = ws.results + ws.cap_results - 3;  // E(2), E3a, E3b of the last energy
  const int nres = order == 2 ? 1 : 3;
  const long long n1 = (long long)m * m, n2 = n1 * n1;
  Scratch h1(ws, n1), h2(ws, n2), g1(ws, n1), l2(ws, n2), c(ws, n1), Es(ws, 4);
  if (na > 0) {
    // active blocks of Hbar^[order] (dense, spin-major)
    if (!h.rx1_2.v.p || !h.rx2_2.v.p || !h.rx1_3.v.p || !h.rx2_3.v.p)
      throw std::runtime_error("relaxed: no active blocks accumulated");
    check_cuda(cudaMemcpyAsync(h1.p, h.rx1_2.v.p, n1 * 8, cudaMemcpyDeviceToDevice, st), "copy");
    check_cuda(cudaMemcpyAsync(h2.p, h.rx2_2.v.p, n2 * 8, cudaMemcpyDeviceToDevice, st), "copy");
    if (order == 3) {
      k_add<<<grid_for(n1, 256), 256, 0, st>>>(n1, h.rx1_3.v.p, h1.p);
      k_add<<<grid_for(n2, 256), 256, 0, st>>>(n2, h.rx2_3.v.p, h2.p);
      ws.launches += 2;
    }
    // reference densities on the active block, dense spin-major
    Iv aa[2] = {h.A, h.A};
    Tensor G = make_tensor(ws, 2, aa, true, true);
    axpy(ws, 1.0, h.gam.v.sub(aa), "ab", G, "ab");
    Iv a4[4] = {h.A, h.A, h.A, h.A};
    Tensor L = make_tensor(ws, 4, a4, true, true);
    axpy(ws, 1.0, h.L2.v, "abcd", L, "abcd");
    check_cuda(cudaMemcpyAsync(g1.p, G.v.p, n1 * 8, cudaMemcpyDeviceToDevice, st), "copy");
    check_cuda(cudaMemcpyAsync(l2.p, L.v.p, n2 * 8, cudaMemcpyDeviceToDevice, st), "copy");
  }
  k_dno<<<1, RX_T, 0, st>>>(m, h1.p, h2.p, g1.p, l2.p, res, nres, Es.p, c.p);
  check_cuda(cudaGetLastError(), "k_dno launch");
  ws.launches += 1;
  // determinants: alpha string major, strings ascending, alpha bits low
  std::vector<uint32_t> dets;
  {
    const std::vector<uint32_t> sa = strings(na, n_alpha), sb = strings(na, n_beta);
    for (uint32_t a : sa)
      for (uint32_t b : sb) dets.push_back(a | (b << na));
  }
  Scratch dd(ws, (size_t)(ndet + 1) / 2);
  uint32_t* dets_dev = reinterpret_cast<uint32_t*>(dd.p);
  check_cuda(cudaMemcpyAsync(dets_dev, dets.data(), (size_t)ndet * 4, cudaMemcpyHostToDevice, st), "copy dets");
  Scratch H(ws, (size_t)(ndet * ndet));
  k_ci_matrix<<<grid_for(ndet * ndet, 256), 256, 0, st>>>(ndet, dets_dev, m, Es.p, c.p, h2.p, H.p);
  check_cuda(cudaGetLastError(), "k_ci_matrix launch");
  ws.launches += 1;
  // Lanczos with full reorthogonalisation (Gram-Schmidt applied twice)
  const int mmax = (int)(ndet < LZ_MAX_STEPS ? ndet : LZ_MAX_STEPS);
  Scratch V(ws, (size_t)(mmax + 1) * ndet), w(ws, ndet), x(ws, ndet), work(ws, 3 * LZ_MAX_STEPS);
  Scratch sc(ws, 5 * LZ_MAX_STEPS + 16);
  double* coef = sc.p;
  double* coef2 = sc.p + LZ_MAX_STEPS;
  double* alpha = sc.p + 2 * LZ_MAX_STEPS;
  double* beta = sc.p + 3 * LZ_MAX_STEPS;
  double* y = sc.p + 4 * LZ_MAX_STEPS;
  double* nrm = sc.p + 5 * LZ_MAX_STEPS;
  LzState* lst = reinterpret_cast<LzState*>(sc.p + 5 * LZ_MAX_STEPS + 8);
  static_assert(sizeof(LzState) <= 8 * sizeof(double), "Lanczos state slot");
  const unsigned gn = grid_for(ndet, 256), gw = grid_for(ndet * 32, 256);
  k_lz_seed<<<gn, 256, 0, st>>>(ndet, x.p);
  ws.launches += 1;
  RelaxResult out;
  const double tol = 1e-9;
  for (int run = 0; run < LZ_MAX_RUNS; ++run) {
    k_dots<<<1, RX_T, 0, st>>>(ndet, x.p, x.p, nrm, nullptr);
    k_lz_start<<<gn, 256, 0, st>>>(ndet, x.p, nrm, V.p, lst);
    ws.launches += 2;
    const double mv_bytes = 8.0 * (double)ndet * (double)ndet + 16.0 * (double)ndet;
    for (int j = 0; j < mmax; ++j) {
      const double* vj = V.p + (long long)j * ndet;
      const int rec = ws.begin(K_CI_MATVEC, 2.0 * (double)ndet * (double)ndet, mv_bytes);
      k_matvec<<<gw, 256, 0, st>>>(ndet, H.p, vj, w.p, lst);
      ws.end(rec);
      k_dots<<<j + 1, RX_T, 0, st>>>(ndet, V.p, w.p, coef, lst);
      k_subtract<<<gn, 256, 0, st>>>(ndet, j + 1, V.p, coef, w.p, lst);
      k_dots<<<j + 1, RX_T, 0, st>>>(ndet, V.p, w.p, coef2, lst);
      k_subtract<<<gn, 256, 0, st>>>(ndet, j + 1, V.p, coef2, w.p, lst);
      k_dots<<<1, RX_T, 0, st>>>(ndet, w.p, w.p, nrm, lst);
      k_lz_next<<<1, 1, 0, st>>>(j, mmax, coef, nrm, alpha, beta, lst);
      k_lz_scale<<<gn, 256, 0, st>>>(ndet, j, w.p, beta, V.p, lst);
      ws.launches += 7;
    }
    check_cuda(cudaGetLastError(), "lanczos launch");
    k_lz_tridiag<<<1, 1, 0, st>>>(alpha, beta, lst, y, work.p);
    LzState hs{};
    check_cuda(cudaMemcpyAsync(&hs, lst, sizeof hs, cudaMemcpyDeviceToHost, st), "copy lanczos state");
    check_cuda(cudaStreamSynchronize(st), "sync");
    // Ritz vector (unit norm) and its explicit residual |H x - lambda x|
    k_ritz<<<gn, 256, 0, st>>>(ndet, hs.steps, V.p, y, x.p);
    k_matvec<<<gw, 256, 0, st>>>(ndet, H.p, x.p, w.p, nullptr);
    k_resid<<<gn, 256, 0, st>>>(ndet, x.p, w.p, lst);
    k_dots<<<1, RX_T, 0, st>>>(ndet, w.p, w.p, nrm, nullptr);
    ws.launches += 6;
    check_cuda(cudaGetLastError(), "lanczos launch");
    double r2 = 0.0;
    check_cuda(cudaMemcpyAsync(&r2, nrm, sizeof r2, cudaMemcpyDeviceToHost, st), "copy residual");
    check_cuda(cudaStreamSynchronize(st), "sync");
    out.e = hs.lambda;
    out.residual = std::sqrt(r2 > 0.0 ? r2 : 0.0);
    out.steps += hs.steps;
    if (out.residual <= tol * (std::fabs(out.e) > 1.0 ? std::fabs(out.e) : 1.0)) break;
  }
  return out;
}

}  // namespace dsrg

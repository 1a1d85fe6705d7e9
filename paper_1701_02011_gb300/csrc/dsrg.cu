// DSRG-MRPT2/PT3 energy driver on the GPU (FP64 path).
//
// Term lists of the commutators [X, T] (X a Hermitian one- plus two-body
// operator, T an excitation operator) in generalized normal order, derived
// from the Mukherjee-Kutzelnigg Wick theorem (the paper defers them, Sec. III)
// and written here by hand on spin orbitals with gamma, eta = 1 - gamma and
// the two- and three-body cumulants.  Sums over hole (H) and particle (P)
// ranges restrict themselves to the overlap where the ranges meet.
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <vector>

#include "dsrg_impl.cuh"

#include <cstdlib>
#include "ladder.cuh"

namespace dsrg {

namespace {
Tensor mk(Handle& h, std::initializer_list<Iv> ivs, bool zero = true) {
  std::vector<Iv> v(ivs);
  return make_tensor(h.ws, (int)v.size(), v.data(), zero);
}

// every spin block stored: for intermediates whose spin conservation pairs
// other slots than (first half | second half)
Tensor mk_dense(Handle& h, std::initializer_list<Iv> ivs) {
  std::vector<Iv> v(ivs);
  return make_tensor(h.ws, (int)v.size(), v.data(), true, true);
}

void raw_axpy4(Handle& h, double alpha, const double* src, const long long* ss, double* dst, const long long* ds,
               const int* ext) {
  NdArgs g{};
  g.nd = 4;
  g.total = 1;
  for (int i = 0; i < 4; ++i) {
    g.e[i] = ext[i];
    g.sa[i] = ss[i];
    g.sb[i] = ds[i];
    g.total *= ext[i];
  }
  run_axpy(h.ws, g, alpha, src, dst);
}

// J[p,q,r,s] = sum_Q B[Q,p,r] B[Q,q,s] for p in I0, q in I1, r in I2, s in I3,
// contiguous [L0][L1][L2][L3] (Eq. int_fact).
void df_integrals(Handle& h, Iv I0, Iv I1, Iv I2, Iv I3, double* J) {
  long long n = h.n;
  int L1 = I1.len(), L2 = I2.len(), L3 = I3.len();
  GemmArgs g{};
  g.A = h.B + I0.lo * n + I2.lo;
  g.B = h.B + I1.lo * n + I3.lo;
  g.C = J;
  g.alpha = 1.0;
  g.nM = 2;
  g.eM[0] = I0.len(); g.aM[0] = n; g.cM[0] = (long long)L1 * L2 * L3;
  g.eM[1] = L2;       g.aM[1] = 1; g.cM[1] = L3;
  g.nN = 2;
  g.eN[0] = L1; g.bN[0] = n; g.cN[0] = (long long)L2 * L3;
  g.eN[1] = L3; g.bN[1] = 1; g.cN[1] = 1;
  g.nK = 1;
  g.eK[0] = h.naux; g.aK[0] = n * n; g.bK[0] = n * n;
  g.nB = 0;
  g.M = (long long)I0.len() * L2;
  g.N = (long long)L1 * L3;
  g.K = h.naux;
  g.nbatch = 1;
  run_gemm(h.ws, g);
}
}  // namespace

// <pq||rs> on a spin-orbital interval class, times coef.
Tensor vclass(Handle& h, const Iv* ivs, double coef) {
  Tensor V = make_tensor(h.ws, 4, ivs, true);
  int L[4] = {ivs[0].len(), ivs[1].len(), ivs[2].len(), ivs[3].len()};
  for (int k = 0; k < 4; ++k)
    if (L[k] <= 0) return V;
  size_t capJ, capK;
  size_t nJ = (size_t)L[0] * L[1] * L[2] * L[3];
  double* J = h.ws.get(nJ, capJ);
  double* K = h.ws.get(nJ, capK);
  check_cuda(cudaMemsetAsync(J, 0, nJ * sizeof(double), h.ws.stream), "memset");
  check_cuda(cudaMemsetAsync(K, 0, nJ * sizeof(double), h.ws.stream), "memset");
  df_integrals(h, ivs[0], ivs[1], ivs[2], ivs[3], J);  // (pr|qs) at [p,q,r,s]
  df_integrals(h, ivs[0], ivs[1], ivs[3], ivs[2], K);  // (ps|qr) at [p,q,s,r]
  long long sJ[4] = {(long long)L[1] * L[2] * L[3], (long long)L[2] * L[3], L[3], 1};
  long long sK[4] = {(long long)L[1] * L[3] * L[2], (long long)L[3] * L[2], 1, L[2]};
  const View& v = V.v;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      // spin block bits: slot k has spin bit k
      double* dJ = v.p + v.boff[a | b << 1 | a << 2 | b << 3];
      raw_axpy4(h, coef, J, sJ, dJ, v.st, L);
      double* dK = v.p + v.boff[a | b << 1 | b << 2 | a << 3];
      raw_axpy4(h, -coef, K, sK, dK, v.st, L);
    }
  V.v.mask = conserving_mask(4);
  h.ws.put(J, capJ);
  h.ws.put(K, capK);
  return V;
}

// ---------------------------------------------------------------------------
// operators X = c_v (f1 + V) + c_w W, with W given by its excitation blocks
// ---------------------------------------------------------------------------
Tensor build_x1(Handle& h, double c_v, const Tensor* W1, double c_w) {
  Tensor X1 = mk(h, {h.G, h.G});
  if (c_v != 0.0 && h.has_f1) axpy(h.ws, c_v, h.F1.v, "pq", X1, "pq");
  if (W1 && c_w != 0.0) {
    axpy(h.ws, c_w, W1->v, "ai", X1, "ai");
    axpy(h.ws, c_w, W1->v, "ai", X1, "ia");
  }
  return X1;
}

// V on the canonical classes HHHH, HHHP, HHPP, PHPH, PPPH (bits 0..4); with
// on_demand, requests no stored class covers are built from B per use
// Classes larger than the budget are not stored: the terms that read them
// build V from B on their own intervals, a slab at a time within the same
// budget.  The budget is DSRG_V_CLASS_BUDGET_MB if set, else 20 % of the
// device's memory, at most 64 GB per class (the same for every energy of a
// handle, whatever the buffer cache holds): the [P,P,P,H] class (p^3 h;
// 53 GB at p = 308, h = 38) is then built once and read by every term,
// instead of once per term; at p = 504, h = 44 (270 GB) it is still built
// per use.
void build_v(Handle& h, unsigned classes, Sym2& V, bool on_demand) {
  V.cls.clear();
  V.make = nullptr;
  const Iv& H = h.H;
  const Iv& P = h.P;
  double budget;
  if (const char* env = getenv("DSRG_V_CLASS_BUDGET_MB")) {
    budget = atof(env) * 1048576.0;
  } else {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    cudaDeviceProp prop{};
    check_cuda(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
    budget = 0.2 * (double)prop.totalGlobalMem;
    if (budget > 64.0 * 1073741824.0) budget = 64.0 * 1073741824.0;
    if (budget < 8.0 * 1073741824.0) budget = 8.0 * 1073741824.0;
  }
  Iv cl[5][4] = {{H, H, H, H}, {H, H, H, P}, {H, H, P, P}, {P, H, P, H}, {P, P, P, H}};
  for (int c = 0; c < 5; ++c) {
    if (!((classes >> c) & 1)) continue;
    double bytes = 6.0 * 8.0;  // six alpha-conserving spin blocks of doubles
    for (int k = 0; k < 4; ++k) bytes *= cl[c][k].len() > 0 ? cl[c][k].len() : 0;
    if (bytes <= budget) {
      V.cls.push_back(vclass(h, cl[c], 1.0));
    } else {
      Handle* hp = &h;
      V.make = [hp](const Iv* ivs) { return vclass(*hp, ivs, 1.0); };
      V.max_elems = (long long)(budget / 8.0);
    }
  }
  if (on_demand && !V.make) {  // any other interval class: built from B per use
    Handle* hp = &h;
    V.make = [hp](const Iv* ivs) { return vclass(*hp, ivs, 1.0); };
    V.max_elems = (long long)(budget / 8.0);
  }
}

// out[..z..] = sum_x M[z,x] X[..x..] along one slot, M = gamma (hole range)
// or eta (particle range).  Both are the identity outside the active block
// (gamma on core, eta on virtual), so the product is a copy there and a
// small contraction with the active block.
// Active rows of a dressing: out[.., z, ..] += sum_x Ma[z, x] X[.., x, ..]
// over the slot's active orbitals x, z (Ma an [A, A] view).
static void dress_active(Handle& h, const View& X, int slot, const View& Ma, Tensor& out) {
  const int r = X.rank;
  char lx[8], lo[8], lm[3];
  for (int k = 0; k < r; ++k) lx[k] = lo[k] = "abcdef"[k];
  lx[r] = lo[r] = 0;
  lo[slot] = 'z';
  lm[0] = 'z';
  lm[1] = lx[slot];
  lm[2] = 0;
  contract(h.ws, 1.0, Ma, lm, X, lx, out, lo);
}

// (M - 1) on the active block for M = gamma or eta, else nullptr
static const Tensor* dress_delta(const Handle& h, const Tensor& M) {
  if (&M == &h.gam) return &h.gam_dI;
  if (&M == &h.eta) return &h.eta_dI;
  return nullptr;
}

Tensor dress(Handle& h, const Tensor& X, int slot, const Tensor& M) {
  ProfTag tag_(h.ws, "dress");
  const int r = X.v.rank;
  Iv ivs[kMaxRank];
  for (int k = 0; k < r; ++k) ivs[k] = X.v.iv[k];
  ivs[slot] = isect(M.v.iv[0], X.v.iv[slot]);
  const Iv& sl = ivs[slot];
  const bool active = h.na > 0 && !isect(sl, h.A).empty();
  const Tensor* dM = dress_delta(h, M);
  if (dM && !sl.empty() && sl.lo == X.v.iv[slot].lo && sl.hi == X.v.iv[slot].hi && X.n > 0) {
    // same layout as X: a copy of X, plus (M - 1) X on the active rows
    Tensor out = make_tensor(h.ws, r, ivs, false);
    check_cuda(cudaMemcpyAsync(out.v.p, X.v.p, X.n * sizeof(double), cudaMemcpyDeviceToDevice, h.ws.stream),
               "cudaMemcpyAsync (dress)");
    out.v.mask = X.v.mask;
    if (active) dress_active(h, X.v, slot, dM->v, out);
    return out;
  }
  Tensor out = make_tensor(h.ws, r, ivs, true);
  if (sl.empty()) return out;
  char lx[8];
  for (int k = 0; k < r; ++k) lx[k] = "abcdef"[k];
  lx[r] = 0;
  // identity part: the slot's orbitals outside the active space
  Iv parts[2] = {isect(sl, Iv{sl.lo, h.A.lo}), isect(sl, Iv{h.A.hi, sl.hi})};
  for (const Iv& part : parts) {
    if (part.empty()) continue;
    Iv sub[kMaxRank];
    for (int k = 0; k < r; ++k) sub[k] = ivs[k];
    sub[slot] = part;
    axpy(h.ws, 1.0, X.v.sub(sub), lx, out, lx);
  }
  if (active) {
    const Iv aa[2] = {h.A, h.A};
    dress_active(h, X.v, slot, M.v.sub(aa), out);
  }
  return out;
}

// In place on a temporary: (M - 1) X of the active rows goes through a
// small tensor and is added back.
Tensor dress(Handle& h, Tensor&& X, int slot, const Tensor& M) {
  ProfTag tag_(h.ws, "dress-inplace");
  const int r = X.v.rank;
  const Iv sl = isect(M.v.iv[0], X.v.iv[slot]);
  const Tensor* dM = dress_delta(h, M);
  if (!dM || sl.lo != X.v.iv[slot].lo || sl.hi != X.v.iv[slot].hi || X.n == 0)
    return dress(h, static_cast<const Tensor&>(X), slot, M);
  if (h.na == 0 || isect(sl, h.A).empty()) return std::move(X);
  Iv ivs[kMaxRank];
  for (int k = 0; k < r; ++k) ivs[k] = X.v.iv[k];
  ivs[slot] = isect(sl, h.A);
  Tensor act = make_tensor(h.ws, r, ivs, true);
  dress_active(h, X.v, slot, dM->v, act);
  char lx[8];
  for (int k = 0; k < r; ++k) lx[k] = "abcdef"[k];
  lx[r] = 0;
  axpy(h.ws, 1.0, act.v, lx, X, lx);
  return std::move(X);
}

// ---------------------------------------------------------------------------
// amplitudes (Eqs. T1_1st, T2_1st, T1_2nd, T2_2nd) and [H0, A] (closed form)
// ---------------------------------------------------------------------------
// S[a,i] = sum_{x,u active} T2[a,x,i,u] gamma[x,u] (eps_x - eps_u)
static Tensor gamma_source(Handle& h, const Tensor& T2) {
  Tensor S = mk(h, {h.P, h.H});
  if (h.na > 0) {
    Tensor G = mk(h, {h.A, h.A}, false);
    int r = h.ws.begin(K_AMP, 0.0, 0.0);
    launch_gamma_delta(h.nc, h.na, h.eps, h.gam.v.p, h.nc + h.na, G.v.p, h.ws.stream);
    h.ws.end(r);
    G.v.mask = conserving_mask(2);
    contract(h.ws, 1.0, T2.v, "axiu", G.v, "xu", S, "ai");
  }
  S.v.mask = conserving_mask(2);
  return S;
}

void amplitudes(Handle& h, const Tensor* O1, const Tensor& O2, Tensor& T1, Tensor& T2, Tensor& W1, Tensor& W2) {
  ProfTag tag_(h.ws, "amplitudes");
  T2 = mk(h, {h.P, h.P, h.H, h.H}, false);
  W2 = mk(h, {h.P, h.P, h.H, h.H}, false);
  {
    int r = h.ws.begin(K_AMP, 0.0, 24.0 * (double)T2.n);
    Amp2Layout lay{};
    for (int b = 0; b < 16; ++b) {
      lay.boff[b] = ((T2.v.stored >> b) & 1) ? T2.v.boff[b] : -1;
      if (((T2.v.stored >> b) & 1) != ((O2.v.stored >> b) & 1) || ((T2.v.stored >> b) & 1 && T2.v.boff[b] != O2.v.boff[b]))
        throw std::runtime_error("amplitudes: O2 and T2 layouts differ");
    }
    for (int k = 0; k < 4; ++k) {
      lay.st[k] = T2.v.st[k];
      if (O2.v.st[k] != T2.v.st[k] || O2.v.iv[k].lo != T2.v.iv[k].lo || O2.v.iv[k].hi != T2.v.iv[k].hi)
        throw std::runtime_error("amplitudes: O2 and T2 layouts differ");
    }
    launch_amp2(h.nc, h.na, h.nv, h.s, h.eps, O2.v.p, T2.v.p, W2.v.p, lay, h.ws.stream);
    h.ws.end(r);
  }
  T2.v.mask = W2.v.mask = conserving_mask(4);
  Tensor S = gamma_source(h, T2);
  T1 = mk(h, {h.P, h.H}, false);
  W1 = mk(h, {h.P, h.H}, false);
  {
    int r = h.ws.begin(K_AMP, 0.0, 40.0 * (double)T1.n);
    launch_amp1(h.nc, h.na, h.nv, h.s, h.eps, O1 ? O1->v.p : nullptr, S.v.p, T1.v.p, W1.v.p, h.ws.stream);
    h.ws.end(r);
  }
  T1.v.mask = W1.v.mask = conserving_mask(2);
}

// ---------------------------------------------------------------------------
// spin-free particle-particle ladder with (pr|qs) built from B in batches
// ---------------------------------------------------------------------------
// L[p,q,i,j] = sum_{r,s in P} (pr|qs) t[r,s,i,j] with t the alpha-beta block of
// a spin-free T2 (first order, Eq. T2_1st); the spin blocks of
// 1/2 sum_rs <pq||rs> T2[r,s,i,j] follow from L (Eq. scaling_problem).
void df_ladder(Handle& h, const Tensor& T2, Tensor& C2, double coef) {
  ProfTag tag_(h.ws, "ladder");
  const int p = h.na + h.nv, hh = h.nc + h.na;
  if (p == 0 || hh == 0) return;
  const View& tv = T2.v;
  const double* t = tv.p + tv.boff[0b1010];  // spins (alpha, beta, alpha, beta)
  size_t capL;
  size_t nL = (size_t)p * p * hh * hh;
  double* L = h.ws.get(nL, capL);
  check_cuda(cudaMemsetAsync(L, 0, nL * sizeof(double), h.ws.stream), "memset");
  // (pr|qs) in batches of rows within a budget (DSRG_LADDER_BUDGET_MB,
  // default 1024 MB); the first-order alpha-beta amplitudes have
  // t[r,s,i,j] = t[s,r,j,i], so the pair-symmetric form applies
  double budget_mb = 1024.0;
  if (const char* env = getenv("DSRG_LADDER_BUDGET_MB")) budget_mb = atof(env);
  long long maxd = (long long)(budget_mb * 131072.0);
  const long long p3 = (long long)p * p * p;
  if (maxd < p3) maxd = p3;  // one row p with every q >= p0 (the first batch)
  size_t capG;
  double* G = h.ws.get((size_t)maxd, capG);
  const long long tst[4] = {tv.st[0], tv.st[1], tv.st[2], tv.st[3]};
  ladder_core_sym(h.B, h.n, h.naux, h.nc, p, hh, t, tst, L, G, maxd, h.ws.stream, &h.ws);
  h.ws.put(G, capG);
  // scatter into the spin blocks of C2 [2p][2p][2h][2h]
  const View& c = C2.v;
  int ext[4] = {p, p, hh, hh};
  long long sL[4] = {(long long)p * hh * hh, (long long)hh * hh, hh, 1};
  long long sLji[4] = {sL[0], sL[1], 1, hh};      // L[p,q,j,i]
  long long sLqp[4] = {sL[1], sL[0], hh, 1};      // L[q,p,i,j]
  auto blk = [&](int a, int b, int i, int j) {
    const int bits = a | b << 1 | i << 2 | j << 3;
    if (!((c.stored >> bits) & 1)) throw std::runtime_error("ladder: spin block not stored");
    return c.p + c.boff[bits];
  };
  raw_axpy4(h, coef, L, sL, blk(0, 1, 0, 1), c.st, ext);
  raw_axpy4(h, coef, L, sL, blk(1, 0, 1, 0), c.st, ext);
  raw_axpy4(h, -coef, L, sLji, blk(0, 1, 1, 0), c.st, ext);
  raw_axpy4(h, -coef, L, sLji, blk(1, 0, 0, 1), c.st, ext);
  for (int s = 0; s < 2; ++s) {
    raw_axpy4(h, coef, L, sL, blk(s, s, s, s), c.st, ext);
    raw_axpy4(h, -coef, L, sLqp, blk(s, s, s, s), c.st, ext);
  }
  C2.v.mask |= conserving_mask(4);
  h.ws.put(L, capL);
}

// ---------------------------------------------------------------------------
// density-fitted forms of the two excitation-block terms that would read V
// with three particle indices (p^3 h elements: 53 GB at p = 308, h = 38);
// with (pq|rs) = sum_Q B^Q_pq B^Q_rs (Eq. int_fact) they contract small
// three-index intermediates instead
// ---------------------------------------------------------------------------
namespace {
// C[m0,m1][n0,n1] += alpha sum_k A[m0,m1][k..] B[k..][n0,n1] (K of one or two dims)
struct Dims2 {
  int e[2];
  long long a[2], c[2];
};
void gemm22(Handle& h, double alpha, const double* A, const double* B, double* C, Dims2 m, Dims2 nn, int nk,
            const int* ek, const long long* ak, const long long* bk) {
  GemmArgs g{};
  g.A = A;
  g.B = B;
  g.C = C;
  g.alpha = alpha;
  g.nM = 2;
  g.nN = 2;
  g.nK = nk;
  g.M = g.N = g.K = 1;
  for (int i = 0; i < 2; ++i) {
    g.eM[i] = m.e[i];
    g.aM[i] = m.a[i];
    g.cM[i] = m.c[i];
    g.eN[i] = nn.e[i];
    g.bN[i] = nn.a[i];
    g.cN[i] = nn.c[i];
    g.M *= m.e[i];
    g.N *= nn.e[i];
  }
  for (int i = 0; i < nk; ++i) {
    g.eK[i] = ek[i];
    g.aK[i] = ak[i];
    g.bK[i] = bk[i];
    g.K *= ek[i];
  }
  g.nbatch = 1;
  run_gemm(h.ws, g);
}

double* c2_block(Tensor& C2, int s0, int s1, int s2, int s3) {
  const int bits = s0 | s1 << 1 | s2 << 2 | s3 << 3;
  if (!((C2.v.stored >> bits) & 1)) throw std::runtime_error("df term: spin block not stored");
  C2.v.mask |= 1ULL << bits;
  return C2.v.p + C2.v.boff[bits];
}
}  // namespace

// C2[p,q,r,s] += coef (sum_a V[p,q,a,s] T1[a,r] - sum_a V[p,q,a,r] T1[a,s]) on
// the excitation block [P,P,H,H], V = <pq||rs>: with X^Q_pr = sum_a B^Q_pa T1[a,r]
// (per spin), sum_a (pa|qs) T1[a,r] = sum_Q X^Q_pr B^Q_qs and
// sum_a (ps|qa) T1[a,r] = sum_Q B^Q_ps X^Q_qr.  The Coulomb part of the first
// term and the exchange part of the second land in the same spin blocks with
// the same index pairing, as do the other two parts, so each pair is one
// product over a stacked index k < 2Q: U^s = [X^s; B], W^s = [B; X^s] (the
// B^Q_pr block over particles p and holes r copied next to X).
static void df_x2t1(Handle& h, const Tensor& T1, Tensor& C2, double coef) {
  const int p = h.na + h.nv, hh = h.nc + h.na, Q = h.naux;
  if (p == 0 || hh == 0) return;
  const long long n = h.n, n2 = n * n, P0 = h.nc, ph = (long long)p * hh, blk = (long long)Q * ph;
  const View& t = T1.v;
  bool has[2] = {false, false};
  for (int sg = 0; sg < 2; ++sg) has[sg] = (t.mask >> (sg | sg << 1)) & 1;
  if (!has[0] && !has[1]) return;
  // U^s at U + 2s blk: [X^s, Bc]; W^s at W + 2s blk: [Bc, X^s]
  size_t capU, capW;
  double* U = h.ws.get((size_t)(4 * blk), capU);
  double* W = h.ws.get((size_t)(4 * blk), capW);
  check_cuda(cudaMemsetAsync(U, 0, (size_t)(4 * blk) * sizeof(double), h.ws.stream), "memset");
  check_cuda(cudaMemsetAsync(W, 0, (size_t)(4 * blk) * sizeof(double), h.ws.stream), "memset");
  {  // Bc[Q][p][r] = B[Q][P0+p][r] into U^s[1] and W^s[0]
    NdArgs g{};
    g.nd = 3;
    g.e[0] = Q; g.sa[0] = n2; g.sb[0] = ph;
    g.e[1] = p; g.sa[1] = n;  g.sb[1] = hh;
    g.e[2] = hh; g.sa[2] = 1; g.sb[2] = 1;
    g.total = blk;
    for (int sg = 0; sg < 2; ++sg) {
      launch_axpy(g, 1.0, h.B + P0 * n, U + (2 * sg + 1) * blk, h.ws.stream);
      check_cuda(cudaMemcpyAsync(W + 2 * sg * blk, U + (2 * sg + 1) * blk, (size_t)blk * sizeof(double),
                                 cudaMemcpyDeviceToDevice, h.ws.stream), "cudaMemcpyAsync (df)");
    }
    h.ws.launches += 2;
  }
  for (int sg = 0; sg < 2; ++sg) {
    if (!has[sg]) continue;
    const int tb = sg | sg << 1;
    // X^s[Q][p][r] = sum_a B[Q][P0+p][P0+a] T1^{ss}[a][r]
    const int ek[1] = {p};
    const long long ak[1] = {1}, bk[1] = {t.st[0]};
    gemm22(h, 1.0, h.B + P0 * n + P0, t.p + t.boff[tb], U + 2 * sg * blk, Dims2{{Q, p}, {n2, n}, {ph, hh}},
           Dims2{{1, hh}, {0, t.st[1]}, {0, 1}}, 1, ek, ak, bk);
    check_cuda(cudaMemcpyAsync(W + (2 * sg + 1) * blk, U + 2 * sg * blk, (size_t)blk * sizeof(double),
                               cudaMemcpyDeviceToDevice, h.ws.stream), "cudaMemcpyAsync (df)");
  }
  const View& c = C2.v;
  const int ek[1] = {2 * Q};
  const long long kk[1] = {ph};
  for (int s1 = 0; s1 < 2; ++s1)
    for (int s2 = 0; s2 < 2; ++s2) {
      // block (s1, s2, s1, s2) += sum_k U^s1[k][p][r] W^s2[k][q][s]
      // (X^s1_pr B_qs + B_pr X^s2_qs); needs T1^{s1 s1} or T1^{s2 s2}
      if (has[s1] || has[s2])
        gemm22(h, coef, U + 2 * s1 * blk, W + 2 * s2 * blk, c2_block(C2, s1, s2, s1, s2),
               Dims2{{p, hh}, {hh, 1}, {c.st[0], c.st[2]}}, Dims2{{p, hh}, {hh, 1}, {c.st[1], c.st[3]}}, 1, ek, kk,
               kk);
      // block (s2, s1, s1, s2) -= sum_k W^s2[k][p][s] U^s1[k][q][r]
      // (B_ps X^s1_qr + X^s2_ps B_qr)
      if (has[s1] || has[s2])
        gemm22(h, -coef, W + 2 * s2 * blk, U + 2 * s1 * blk, c2_block(C2, s2, s1, s1, s2),
               Dims2{{p, hh}, {hh, 1}, {c.st[0], c.st[3]}}, Dims2{{p, hh}, {hh, 1}, {c.st[1], c.st[2]}}, 1, ek, kk,
               kk);
    }
  h.ws.put(U, capU);
  h.ws.put(W, capW);
}

// C1[p,j] += coef sum_{q,r,s} V[p,q,r,s] D[r,s,q,j] on the excitation block
// [P,H], D antisymmetric in its first two slots ([P,P,H,H]): the exchange
// part equals the Coulomb part, so the sum is
// 2 sum_{Q,r} B^Q_pr Y^Q_rj with Y^Q_rj = sum_{q,s} B^Q_qs D[r,s,q,j] (per spin).
static void df_vd_onebody(Handle& h, const Tensor& D, Tensor& C1, double coef) {
  const int p = h.na + h.nv, hh = h.nc + h.na, Q = h.naux;
  if (p == 0 || hh == 0) return;
  const long long n = h.n, n2 = n * n, P0 = h.nc, ph = (long long)p * hh;
  const View& d = D.v;
  size_t capY;
  double* Y = h.ws.get((size_t)(2 * Q * ph), capY);
  check_cuda(cudaMemsetAsync(Y, 0, (size_t)(2 * Q * ph) * sizeof(double), h.ws.stream), "memset");
  bool has[2] = {false, false};
  for (int sg = 0; sg < 2; ++sg)
    for (int s2 = 0; s2 < 2; ++s2) {
      const int db = sg | s2 << 1 | s2 << 2 | sg << 3;  // D[r s, s s2, q s2, j s]
      if (!((d.mask >> db) & 1)) continue;
      has[sg] = true;
      // Y^s[Q][r][j] += sum_{q in H, s in P} B[Q][q][P0+s] D[r,s,q,j]
      const int ek[2] = {hh, p};
      const long long ak[2] = {n, 1}, bk[2] = {d.st[2], d.st[1]};
      gemm22(h, 1.0, h.B + P0, d.p + d.boff[db], Y + sg * Q * ph, Dims2{{1, Q}, {0, n2}, {0, ph}},
             Dims2{{p, hh}, {d.st[0], d.st[3]}, {hh, 1}}, 2, ek, ak, bk);
    }
  const View& c = C1.v;
  for (int sg = 0; sg < 2; ++sg) {
    if (!has[sg]) continue;
    const int cb = sg | sg << 1;
    if (!((c.stored >> cb) & 1)) throw std::runtime_error("df term: spin block not stored");
    C1.v.mask |= 1ULL << cb;
    // C1^{ss}[p][j] += 2 coef sum_{Q,r} B[Q][P0+p][P0+r] Y^s[Q][r][j]
    const int ek[2] = {Q, p};
    const long long ak[2] = {n2, 1}, bk[2] = {ph, hh};
    gemm22(h, 2.0 * coef, h.B + P0 * n + P0, Y + sg * Q * ph, c.p + c.boff[cb], Dims2{{1, p}, {0, n}, {0, c.st[0]}},
           Dims2{{1, hh}, {0, 1}, {0, c.st[1]}}, 2, ek, ak, bk);
  }
  h.ws.put(Y, capY);
}

// ---------------------------------------------------------------------------
// [X, T] into one output block pair (C1, C2)
// ---------------------------------------------------------------------------
// One-body operator c_f f1 + c_w (W1 + W1^+) as pieces: f1 on [G,G] and W1's
// excitation block [P,H] with its transpose on [H,P].
struct Op1Pieces {
  int n = 0;
  View v[3];
  double c[3];
};

static Op1Pieces op1_pieces(Handle& h, double c_f, const Tensor* W1, double c_w) {
  Op1Pieces o;
  if (c_f != 0.0 && h.has_f1) {
    o.v[o.n] = h.F1.v;
    o.c[o.n++] = c_f;
  }
  if (W1 && c_w != 0.0) {
    o.v[o.n] = W1->v;
    o.c[o.n++] = c_w;
    const int swap[2] = {1, 0};
    o.v[o.n] = W1->v.permuted(swap);
    o.c[o.n++] = c_w;
  }
  return o;
}

// Blocks of [X, T] accumulated into each output pair (C1s[o], C2s[o]),
// o < nout; the output pair's ranges select the blocks (C2 on [P,P,H,H]:
// the excitation blocks).  The dressed copies of T2 depend on T only, so each
// is formed once and serves every output pair before the next is formed.
void commutator(Handle& h, const Tensor& X1, const Op2& X2, const Tensor& T1, const Tensor& T2, Tensor* const* C1s,
                Tensor* const* C2s, int nout, bool df, const Op1Pieces* X1p) {
  Workspace& ws = h.ws;
  ProfTag tag_(ws, "commutator");
  const Tensor& g = h.gam;
  const Tensor& e = h.eta;
  const Tensor& L2 = h.L2;
  const Iv& G = h.G;
  const Iv& H = h.H;
  const Iv& P = h.P;
  const Iv& A = h.A;
  auto exc_of = [&](const Tensor& C2) { return C2.v.iv[0].lo == P.lo && C2.v.iv[0].hi == P.hi; };
  // on the excitation block the V part of the terms with three particle
  // indices of V runs in density-fitted form
  auto dfv_of = [&](const Tensor& C2) { return exc_of(C2) && df && X2.V && X2.cv != 0.0; };
  for (int o = 0; o < nout; ++o) {
    Tensor& C1 = *C1s[o];
    Tensor& C2 = *C2s[o];
    const bool dfv = dfv_of(C2);
    // [X1, T1] one-body: X1 T1 - T1 X1
    ws.tag = "c-x1";
    contract(ws, 1.0, X1.v, "pr", T1.v, "rq", C1, "pq");
    contract(ws, -1.0, T1.v, "pr", X1.v, "rq", C1, "pq");
    // [X1, T2] one-body: (gamma X1 eta - eta X1 gamma)[i,a] T2[a,b,i,j]
    {
      Tensor M1 = mk(h, {G, G});
      Tensor t1 = mk(h, {G, P});
      contract(ws, 1.0, X1.v, "pq", e.v, "qa", t1, "pa");
      contract(ws, 1.0, g.v, "ip", t1.v, "pa", M1, "ia");
      Tensor t2 = mk(h, {G, H});
      contract(ws, 1.0, X1.v, "pq", g.v, "qa", t2, "pa");
      contract(ws, -1.0, e.v, "ip", t2.v, "pa", M1, "ia");
      contract(ws, 1.0, M1.v, "ia", T2.v, "abij", C1, "bj");
    }
    // [X1, T2] two-body, piece by piece so that only non-zero blocks of X1 enter
    {
      Op1Pieces whole;
      whole.n = 1;
      whole.v[0] = X1.v;
      whole.c[0] = 1.0;
      const Op1Pieces& pc = X1p ? *X1p : whole;
      for (int k = 0; k < pc.n; ++k) {
        const double c = pc.c[k];
        contract(ws, c, pc.v[k], "xa", T2.v, "ayij", C2, "xyij");
        contract(ws, -c, pc.v[k], "ya", T2.v, "axij", C2, "xyij");
        contract(ws, -c, T2.v, "xyik", pc.v[k], "kj", C2, "xyij");
        contract(ws, c, T2.v, "xyjk", pc.v[k], "ki", C2, "xyij");
      }
    }
    // [X2, T1] one-body: X2[p,q,s,r] (gamma T1^T eta)[q,r]
    ws.tag = "c-x2t1";
    {
      Tensor tmp = mk(h, {H, P});
      contract(ws, 1.0, g.v, "qi", T1.v, "ai", tmp, "qa");
      Tensor Mq = mk(h, {H, P});
      contract(ws, 1.0, tmp.v, "qa", e.v, "ra", Mq, "qr");
      contract_x2(ws, 1.0, X2, "pqsr", Mq.v, "qr", C1, "ps");
    }
    // [X2, T1] two-body
    if (dfv) df_x2t1(h, T1, C2, X2.cv);
    contract_x2(ws, 1.0, X2, "pqas", T1.v, "ar", C2, "pqrs", dfv);
    contract_x2(ws, -1.0, X2, "pqar", T1.v, "as", C2, "pqrs", dfv);
    contract_x2(ws, 1.0, X2, "qirs", T1.v, "pi", C2, "pqrs");
    contract_x2(ws, -1.0, X2, "pirs", T1.v, "qi", C2, "pqrs");
  }
  // [X2, T2] one-body with three single contractions
  ws.tag = "c-x2t2-1body";
  // dressed copies of T2, one chain at a time (each dressed in place after
  // its first copy), so that at most one is alive: [P,P,H,H] tensors set
  // the memory peak of the large instances
  {
    Tensor D1 = dress(h, dress(h, dress(h, T2, 0, e), 1, e), 2, g);
    for (int o = 0; o < nout; ++o) {
      const bool dfv = dfv_of(*C2s[o]);
      if (dfv) df_vd_onebody(h, D1, *C1s[o], -0.5 * X2.cv);
      contract_x2(ws, -0.5, X2, "pqrs", D1.v, "rsqj", *C1s[o], "pj", dfv);
    }
  }
  {
    Tensor D2 = dress(h, dress(h, dress(h, T2, 0, g), 1, g), 2, e);
    for (int o = 0; o < nout; ++o) contract_x2(ws, -0.5, X2, "pqrs", D2.v, "rsqj", *C1s[o], "pj");
  }
  {
    // hole ladder 1/2 X2 (gamma gamma T2 - eta eta T2) as one product: the
    // eta-dressed tensor lives on the active box inside the gamma-dressed one
    // (eta vanishes on core); then the one-body pair (eta-dressed Ehh plus
    // gamma-dressed Nhh) likewise
    Tensor Nhh = dress(h, dress(h, T2, 2, e), 3, e);
    Tensor D4 = dress(h, Nhh, 0, g);
    Tensor Ehh = dress(h, dress(h, T2, 2, g), 3, g);
    axpy(ws, -1.0, Nhh.v, "abij", Ehh, "abij");
    for (int o = 0; o < nout; ++o) contract_x2(ws, 0.5, X2, "pqrs", Ehh.v, "abpq", *C2s[o], "abrs");
    axpy(ws, 1.0, Nhh.v, "abij", Ehh, "abij");
    Nhh.release();
    Tensor D3 = dress(h, std::move(Ehh), 0, e);
    axpy(ws, 1.0, D4.v, "abij", D3, "abij");
    D4.release();
    for (int o = 0; o < nout; ++o) contract_x2(ws, -0.5, X2, "pqrs", D3.v, "rbpq", *C1s[o], "bs");
  }
  for (int o = 0; o < nout; ++o) {
    Tensor& C1 = *C1s[o];
    // [X2, T2] one-body with a two-body cumulant
    ws.tag = "c-cumulant";
    if (h.na > 0) {
      {
        Tensor Y = mk(h, {P, A});
        contract(ws, 1.0, T2.v, "abij", L2.v, "qbij", Y, "aq");
        Tensor Z = dress(h, Y, 0, e);
        contract_x2(ws, -0.5, X2, "pqrs", Z.v, "rq", C1, "ps");
      }
      {
        Tensor Y = mk(h, {H, A});
        contract(ws, 1.0, T2.v, "abij", L2.v, "abjr", Y, "ir");
        Tensor Z = dress(h, Y, 0, g);
        contract_x2(ws, -0.5, X2, "pqrs", Z.v, "qr", C1, "ps");
      }
      {
        Tensor Y = mk_dense(h, {P, H, A, A});  // conserves a + s = i + q
        contract(ws, 1.0, T2.v, "abij", L2.v, "qbjs", Y, "aiqs");
        contract_x2(ws, -1.0, X2, "pqas", Y.v, "aiqs", C1, "pi");
      }
      {
        Tensor Y = mk(h, {P, P, A, A});
        contract(ws, 1.0, T2.v, "abij", L2.v, "pqij", Y, "abpq");
        contract_x2(ws, -0.25, X2, "pqas", Y.v, "abpq", C1, "bs");
      }
      {
        Tensor Y = mk(h, {P, A});
        contract_x2(ws, 1.0, X2, "pqas", L2.v, "pqjs", Y, "aj");
        contract(ws, -0.5, Y.v, "aj", T2.v, "abij", C1, "bi");
      }
      {
        Tensor Y = mk(h, {C1.v.iv[0], H, A, A});
        contract_x2(ws, 1.0, X2, "pirs", L2.v, "abrs", Y, "piab");
        contract(ws, -0.25, Y.v, "piab", T2.v, "abij", C1, "pj");
      }
      {
        Tensor Y = mk_dense(h, {P, H, A, A});  // conserves b + r = i + p
        contract(ws, 1.0, T2.v, "abij", L2.v, "pajr", Y, "bipr");
        contract_x2(ws, -1.0, X2, "pirs", Y.v, "bipr", C1, "bs");
      }
      {
        Tensor Y = mk(h, {H, A});
        contract_x2(ws, 1.0, X2, "pirs", L2.v, "pars", Y, "ia");
        contract(ws, -0.5, Y.v, "ia", T2.v, "abij", C1, "bj");
      }
    }
  }
  // [X2, T2] two-body: particle ladder 1/2 X2 T2 - X2[p,q,r,b] (gamma T2)[r,b,i,j]
  ws.tag = "c-x2t2-2body";
  for (int o = 0; o < nout; ++o) {
    Tensor& C2 = *C2s[o];
    if (exc_of(C2)) {
      // the V part of the all-particle block is never stored: DF ladder
      if (X2.V && X2.cv != 0.0) {
        if (!df) throw std::runtime_error("particle ladder of V needs the DF path");
        df_ladder(h, T2, C2, X2.cv);
      }
    } else {
      contract_x2(ws, 0.5, X2, "pqrs", T2.v, "rsij", C2, "pqij");
    }
  }
  {
    Tensor gT2 = dress(h, T2, 0, g);
    for (int o = 0; o < nout; ++o) {
      Tensor& C2 = *C2s[o];
      if (exc_of(C2)) {
        if (X2.W && X2.cw != 0.0) {
          // W's excitation block [P,P,H,H] meets both terms only on its [A,A]
          // second pair: one product with (1/2 T2 - gamma T2) on [A,A,H,H];
          // its Hermitian image takes each term on its own
          Iv box[4] = {A, A, H, H};
          Tensor Y = make_tensor(ws, 4, box, true);
          axpy(ws, 0.5, T2.v.sub(box), "rsij", Y, "rsij");
          axpy(ws, -1.0, gT2.v.sub(box), "rsij", Y, "rsij");
          contract(ws, X2.cw, w_place(*X2.W, 0), "pqrs", Y.v, "rsij", C2, "pqij");
          contract(ws, 0.5 * X2.cw, w_place(*X2.W, 1), "pqrs", T2.v, "rsij", C2, "pqij");
          contract(ws, -X2.cw, w_place(*X2.W, 1), "pqrb", gT2.v, "rbij", C2, "pqij");
        }
        if (X2.V && X2.cv != 0.0)
          contract_x2(ws, -1.0, Op2{X2.V, X2.cv, nullptr, 0.0}, "pqrb", gT2.v, "rbij", C2, "pqij");
      } else {
        contract_x2(ws, -1.0, X2, "pqrb", gT2.v, "rbij", C2, "pqij");
      }
    }
  }
  for (int o = 0; o < nout; ++o) {
    Tensor& C2 = *C2s[o];
    const bool exc = exc_of(C2);
    // ring: K[x,y,u,w] = sum_{i,a} (Xbar - Xtilde)[x,i,a,w] T2[a,y,i,u], antisymmetrised.
    // X2 is taken piece by piece (V, then W and its Hermitian image on their
    // own boxes) so that no work is spent where a piece vanishes.
    {
      ProfTag ring_tag(ws, "ring");
      Iv xi = isect(exc ? P : H, C2.v.iv[0]), wi = isect(exc ? H : P, C2.v.iv[3]);
      Iv want[4] = {xi, H, P, wi};
      // y and u must land in C2's slots as well as in T2's
      Iv kiv[4] = {xi, isect(P, C2.v.iv[1]), isect(H, C2.v.iv[2]), wi};
      Tensor K = make_tensor(ws, 4, kiv, true);
      // (Xbar - Xtilde) as one operand: Xtilde (eta on the hole slot, gamma on
      // the particle slot) lives on the active box inside Xbar's
      auto ring_piece = [&](const Tensor& Xs) {
        Tensor Xb = dress(h, dress(h, Xs, 1, g), 2, e);
        {
          Tensor Xt = dress(h, dress(h, Xs, 1, e), 2, g);
          axpy(ws, -1.0, Xt.v, "xiaw", Xb, "xiaw");
        }
        contract(ws, 1.0, Xb.v, "xiaw", T2.v, "ayiu", K, "xyuw");
      };
      if (X2.V && X2.cv != 0.0) {
        // V covers the whole box: W's pieces are added into it, one product
        Tensor Xs = make_tensor(ws, 4, want, true);
        fetch_x2(ws, 1.0, Op2{X2.V, X2.cv, nullptr, 0.0}, Xs);
        if (X2.W && X2.cw != 0.0)
          for (int herm = 0; herm < 2; ++herm) axpy(ws, X2.cw, w_place(*X2.W, herm), "abcd", Xs, "abcd");
        ring_piece(Xs);
      } else if (X2.W && X2.cw != 0.0) {
        for (int herm = 0; herm < 2; ++herm) {
          View wp = w_place(*X2.W, herm);
          Iv box[4];
          bool empty = false;
          for (int k = 0; k < 4; ++k) {
            box[k] = isect(want[k], wp.iv[k]);
            empty |= box[k].empty();
          }
          if (empty) continue;
          Tensor Xs = make_tensor(ws, 4, box, true);
          axpy(ws, X2.cw, wp, "abcd", Xs, "abcd");
          ring_piece(Xs);
        }
      }
      axpy(ws, 1.0, K.v, "xyuw", C2, "xyuw");
      axpy(ws, -1.0, K.v, "xyuw", C2, "yxuw");
      axpy(ws, -1.0, K.v, "xyuw", C2, "xywu");
      axpy(ws, 1.0, K.v, "xyuw", C2, "yxwu");
    }
  }
}

void commutator(Handle& h, const Tensor& X1, const Op2& X2, const Tensor& T1, const Tensor& T2, Tensor& C1,
                Tensor& C2, bool df, const Op1Pieces* X1p) {
  Tensor* c1[1] = {&C1};
  Tensor* c2[1] = {&C2};
  commutator(h, X1, X2, T1, T2, c1, c2, 1, df, X1p);
}

// excitation blocks of [X, T - T^+] = [X, T] + [X, T]^+ (X Hermitian)
void commutator_A(Handle& h, const Tensor& X1, const Op2& X2, const Tensor& T1, const Tensor& T2, Tensor& O1,
                  Tensor& O2, bool df, const Op1Pieces* X1p) {
  O1 = mk(h, {h.P, h.H});
  O2 = mk(h, {h.P, h.P, h.H, h.H});
  // excitation blocks straight into O1, O2; the de-excitation blocks [H H P P]
  // land in O2 through a slot-permuted alias (the commutator only accumulates)
  // (both in one pass, so that the dressed copies of T2 are formed once)
  const int perm[4] = {2, 3, 0, 1};
  Tensor C1d = mk(h, {h.H, h.P});
  Tensor C2d = alias_permuted(O2, perm);
  Tensor* c1[2] = {&O1, &C1d};
  Tensor* c2[2] = {&O2, &C2d};
  commutator(h, X1, X2, T1, T2, c1, c2, 2, df, X1p);
  merge_alias_mask(O2, C2d, perm);
  axpy(h.ws, 1.0, C1d.v, "ia", O1, "ai");
}

// ---------------------------------------------------------------------------
// scalar <[X, T]>: only the X1[H,P] and X2[H,H,P,P] elements enter
// ---------------------------------------------------------------------------
void scalar(Handle& h, const Tensor& X1, const Op2& X2, const Tensor& T1, const Tensor& T2) {
  ProfTag tag_(h.ws, "scalar");
  Workspace& ws = h.ws;
  const Tensor& g = h.gam;
  const Tensor& e = h.eta;
  const Iv& G = h.G;
  const Iv& H = h.H;
  const Iv& P = h.P;
  const Iv& A = h.A;
  {  // [X1, T1]
    Tensor t2 = mk(h, {H, G});
    contract(ws, 1.0, g.v, "ip", X1.v, "pq", t2, "iq");
    Tensor tmp = mk(h, {H, P});
    contract(ws, 1.0, t2.v, "iq", e.v, "qa", tmp, "ia");
    dot(ws, 1.0, T1.v, "ai", tmp.v, "ia");
  }
  if (h.na > 0) {
    const Tensor& L2 = h.L2;
    {  // [X1, T2]
      Tensor Y = mk(h, {P, A});
      contract(ws, 1.0, T2.v, "abij", L2.v, "pbij", Y, "ap");
      Tensor xe = mk(h, {A, P});
      contract(ws, 1.0, X1.v, "pq", e.v, "qa", xe, "pa");
      dot(ws, 0.5, xe.v, "pa", Y.v, "ap");
      Tensor Z = mk(h, {H, A});
      contract(ws, 1.0, T2.v, "abij", L2.v, "abjq", Z, "iq");
      Tensor gx = mk(h, {H, A});
      contract(ws, 1.0, g.v, "ip", X1.v, "pq", gx, "iq");
      dot(ws, 0.5, gx.v, "iq", Z.v, "iq");
    }
    {  // [X2, T1]
      Tensor Y = dress(h, T1, 0, e);
      Tensor U = mk(h, {A, A, P, A});
      contract(ws, 1.0, Y.v, "ri", L2.v, "pqis", U, "pqrs");
      dot_x2(ws, 0.5, X2, U);
      Tensor Y2 = mk(h, {H, P});
      contract(ws, 1.0, g.v, "qi", T1.v, "ai", Y2, "qa");
      Tensor U2 = mk(h, {A, H, A, A});
      contract(ws, 1.0, Y2.v, "qa", L2.v, "pars", U2, "pqrs");
      dot_x2(ws, -0.5, X2, U2);
    }
  }
  // [X2, T2]
  Tensor Dee = dress(h, dress(h, T2, 0, e), 1, e);
  {
    Tensor D = dress(h, dress(h, Dee, 2, g), 3, g);
    const int perm[4] = {2, 3, 0, 1};
    Tensor Dt = alias_permuted(D, perm);  // Dt[p,q,r,s] = D[r,s,p,q], no copy
    dot_x2(ws, 0.25, X2, Dt);
  }
  if (h.na > 0) {
    const Tensor& L2 = h.L2;
    const Tensor& L3 = h.L3;
    {
      Tensor U = mk(h, {A, A, P, P});
      contract(ws, 1.0, Dee.v, "rsij", L2.v, "pqij", U, "pqrs");
      dot_x2(ws, 0.125, X2, U);
    }
    {
      Tensor Dgg = dress(h, dress(h, T2, 2, g), 3, g);
      Tensor U = mk(h, {H, H, A, A});
      contract(ws, 1.0, Dgg.v, "abpq", L2.v, "abrs", U, "pqrs");
      dot_x2(ws, 0.125, X2, U);
    }
    {
      Tensor Dp = dress(h, dress(h, T2, 0, e), 2, g);
      Tensor U = mk(h, {A, H, P, A});
      contract(ws, 1.0, Dp.v, "rbqj", L2.v, "pbjs", U, "pqrs");
      dot_x2(ws, 1.0, X2, U);
    }
    {
      Tensor De = dress(h, T2, 0, e);
      Tensor U = mk(h, {A, A, P, A});
      contract(ws, 1.0, De.v, "rbij", L3.v, "pqbijs", U, "pqrs");
      dot_x2(ws, -0.25, X2, U);
    }
    {
      Tensor Dg = dress(h, T2, 2, g);
      Tensor U = mk(h, {A, H, A, A});
      contract(ws, 1.0, Dg.v, "abqj", L3.v, "pabjrs", U, "pqrs");
      dot_x2(ws, -0.25, X2, U);
    }
  }
}

// E(2), E3a, E3b from their result slots, into the last three slots
// ---------------------------------------------------------------------------
// all-active blocks for the relaxed energies (App. A)
// ---------------------------------------------------------------------------
// H^(0) + H^(1) on [A, A] and [A, A, A, A]: the semicanonical Fock diagonal
// and V (the off-diagonal Fock f^(1) has no all-active block)
static void relax_bare(Handle& h, const Sym2& V) {
  h.rx1_2 = mk_dense(h, {h.A, h.A});
  h.rx2_2 = mk_dense(h, {h.A, h.A, h.A, h.A});
  h.rx1_3 = mk_dense(h, {h.A, h.A});
  h.rx2_3 = mk_dense(h, {h.A, h.A, h.A, h.A});
  int r = h.ws.begin(K_AMP, 0.0, 0.0);
  launch_active_diagonal(h.nc, h.na, h.eps, h.rx1_2.v.p, h.ws.stream);
  h.ws.end(r);
  fetch_x2(h.ws, 1.0, Op2{&V, 1.0, nullptr, 0.0}, h.rx2_2);
}

// [X, A]_act = C + C^+ with C = [X, T] on the all-active block, accumulated
// into acc1, acc2
static void relax_commutator(Handle& h, const Tensor& X1, const Op2& X2, const Tensor& T1, const Tensor& T2,
                             const Op1Pieces* pc, Tensor& acc1, Tensor& acc2) {
  ProfTag tag_(h.ws, "relax-active");
  Tensor C1 = mk(h, {h.A, h.A});
  Tensor C2 = mk(h, {h.A, h.A, h.A, h.A});
  commutator(h, X1, X2, T1, T2, C1, C2, false, pc);
  axpy(h.ws, 1.0, C1.v, "uv", acc1, "uv");
  axpy(h.ws, 1.0, C1.v, "uv", acc1, "vu");
  axpy(h.ws, 1.0, C2.v, "uvxy", acc2, "uvxy");
  axpy(h.ws, 1.0, C2.v, "uvxy", acc2, "xyuv");
}

// zero the all-active (internal) block of an excitation-block tensor
static void zero_internal(Handle& h, Tensor& X) {
  Iv want[4] = {h.A, h.A, h.A, h.A};
  View in = X.v.sub(want);
  const char* l = X.v.rank == 2 ? "ab" : "abcd";
  axpy(h.ws, -1.0, in, l, X, l);
}

static void sum_components(Handle& h) {
  Workspace& ws = h.ws;
  if (ws.nresults > ws.cap_results - 3) throw std::runtime_error("out of result slots");
  int r = ws.begin(K_DOT, 0.0, 8.0 * (double)ws.nresults);
  launch_sum_slots(ws.results, h.res, ws.results + ws.cap_results - 3, ws.stream);
  ws.end(r);
}

// Every kernel and copy of one energy, enqueued on the handle's stream with
// no host synchronisation (so that it can be captured in a CUDA graph); the
// result-slot ranges of E(2), E3a, E3b go to h.res.
void issue_energy(Handle& h, bool pt3) {
  Workspace& ws = h.ws;
  ws.launches = 0;
  ws.nresults = 0;
  h.res_pt3 = pt3;
  const Iv& H = h.H;
  const Iv& P = h.P;
  // first-order amplitudes from the non-diagonal part of H(1)
  ws.tag = "first-order";
  Tensor F1ph = mk(h, {P, H});
  if (h.has_f1) axpy(ws, 1.0, h.F1.v, "ai", F1ph, "ai");
  Tensor Vph;
  {
    Iv cl[4] = {P, P, H, H};
    Vph = vclass(h, cl, 1.0);
  }
  Tensor T1, T2, W1, W2;
  amplitudes(h, &F1ph, Vph, T1, T2, W1, W2);
  Vph.release();
  // Htilde(1) = 2 H(1) + [H(0), A(1)] (Eq. Hbar_1st); V on the classes the terms need
  Sym2 V;
  ws.tag = "build-v";
  // the [P,P,P,H] class is read only by terms evaluated in density-fitted
  // form (df_x2t1, df_vd_onebody) and by small slabs of it: not stored
  build_v(h, pt3 ? 0x0fu : (1u << 2), V, pt3);
  const bool rx = h.relax && pt3 && h.na > 0;
  if (rx) relax_bare(h, V);
  ws.tag = "E2";
  Tensor Xs1 = build_x1(h, 2.0, &W1, 1.0);
  Op2 Xs2{&V, 2.0, &W2, 1.0};
  h.res[0] = ws.nresults;
  scalar(h, Xs1, Xs2, T1, T2);
  h.res[1] = h.res[2] = h.res[3] = h.res[4] = ws.nresults;
  h.T1 = std::move(T1);
  h.T2 = std::move(T2);
  if (!pt3) {
    sum_components(h);
    h.launches = ws.launches;
    ws.tag = "";
    return;
  }
  const Tensor& t1 = h.T1;
  const Tensor& t2 = h.T2;
  // O = 1/2 [Htilde(1), A(1)]_{1,2} = [H(1) + W/2, A(1)]_{1,2}
  ws.tag = "O";
  Tensor O1, O2;
  {
    Tensor X1 = build_x1(h, 1.0, &W1, 0.5);
    Op1Pieces pc = op1_pieces(h, 1.0, &W1, 0.5);
    commutator_A(h, X1, Op2{&V, 1.0, &W2, 0.5}, t1, t2, O1, O2, true, &pc);
    if (rx) relax_commutator(h, X1, Op2{&V, 1.0, &W2, 0.5}, t1, t2, &pc, h.rx1_2, h.rx2_2);
  }
  // second-order amplitudes (Eqs. T1_2nd, T2_2nd) and [H(0), A(2)]
  ws.tag = "second-order";
  Tensor U1, U2, V1, V2;
  amplitudes(h, &O1, O2, U1, U2, V1, V2);
  if (rx) {  // 1/2 [Htilde^(1), A^(2)] = [H^(1) + W/2, A^(2)]
    Tensor X1 = build_x1(h, 1.0, &W1, 0.5);
    Op1Pieces pc = op1_pieces(h, 1.0, &W1, 0.5);
    relax_commutator(h, X1, Op2{&V, 1.0, &W2, 0.5}, U1, U2, &pc, h.rx1_3, h.rx2_3);
  }
  // Htilde(2)_{1,2} excitation blocks = [H0, A(2)] + O - [W, A(1)] / 6,
  // accumulated in place of [H0, A(2)] (not needed otherwise); O is kept for
  // dsrg_fetch only while a [P,P,H,H] tensor is small
  Tensor Z1 = std::move(V1), Z2 = std::move(V2);
  axpy(ws, 1.0, O1.v, "ai", Z1, "ai");
  axpy(ws, 1.0, O2.v, "abij", Z2, "abij");
  const bool keep_o = O2.n * sizeof(double) <= (size_t)1 << 30;
  if (keep_o) {
    h.O1 = std::move(O1);
    h.O2 = std::move(O2);
  } else {
    O1.release();
    O2.release();
    h.O1.release();
    h.O2.release();
  }
  // [W, A(1)]_{1,2}
  ws.tag = "Q";
  Tensor Q1, Q2;
  {
    Tensor Y1 = build_x1(h, 0.0, &W1, 1.0);
    Op1Pieces pc = op1_pieces(h, 0.0, &W1, 1.0);
    commutator_A(h, Y1, Op2{nullptr, 0.0, &W2, 1.0}, t1, t2, Q1, Q2, false, &pc);
  }
  ws.tag = "Z";
  axpy(ws, -1.0 / 6.0, Q1.v, "ai", Z1, "ai");
  axpy(ws, -1.0 / 6.0, Q2.v, "abij", Z2, "abij");
  Q1.release();
  Q2.release();
  Tensor Zx1 = build_x1(h, 0.0, &Z1, 1.0);
  ws.tag = "E3";
  h.res[2] = ws.nresults;
  scalar(h, Xs1, Xs2, U1, U2);
  h.res[3] = ws.nresults;
  scalar(h, Zx1, Op2{nullptr, 0.0, &Z2, 1.0}, t1, t2);
  h.res[4] = ws.nresults;
  if (rx) {
    // 1/2 [Htilde^(2), A^(1)]: only the excitation blocks of Htilde^(2) and
    // their Hermitian images reach the all-active block, and not their own
    // all-active part (it meets only internal amplitudes, which vanish); it is
    // removed so that the W-form operator does not count it twice
    Zx1.release();
    zero_internal(h, Z1);
    zero_internal(h, Z2);
    Tensor X1 = build_x1(h, 0.0, &Z1, 0.5);
    Op1Pieces pc = op1_pieces(h, 0.0, &Z1, 0.5);
    relax_commutator(h, X1, Op2{nullptr, 0.0, &Z2, 0.5}, t1, t2, &pc, h.rx1_3, h.rx2_3);
  }
  h.T1b = std::move(U1);
  h.T2b = std::move(U2);
  sum_components(h);
  h.launches = ws.launches;
  ws.tag = "";
}

// One copy of the three energy components, reduced on the device from the
// result slots of the last issued energy.  Synchronises the stream.
void finish_energy(Handle& h, double* e2, double* e3a, double* e3b) {
  double v[3] = {0.0, 0.0, 0.0};
  h.d2h_bytes = (long long)sizeof v;
  check_cuda(cudaMemcpyAsync(v, h.ws.results + h.ws.cap_results - 3, sizeof v, cudaMemcpyDeviceToHost, h.ws.stream),
             "copy results");
  check_cuda(cudaStreamSynchronize(h.ws.stream), "sync");
  *e2 = v[0];
  *e3a = h.res_pt3 ? v[1] : 0.0;
  *e3b = h.res_pt3 ? v[2] : 0.0;
}

void run_energy(Handle& h, bool pt3, double* e2, double* e3a, double* e3b) {
  issue_energy(h, pt3);
  finish_energy(h, e2, e3a, e3b);
}

}  // namespace dsrg

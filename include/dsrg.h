/*
 * dsrg.h -- C interface of the GB300 DSRG-MRPT2/PT3 energy library.
 *
 * Computes the unrelaxed second- and third-order energies of the driven
 * similarity renormalization group perturbation theory (Li & Evangelista,
 * "Driven similarity renormalization group: Third-order multireference
 * perturbation theory"):
 *   E(2) = <[Htilde(1), T(1)]>                          (Eq. E(2))
 *   E(3) = <[Htilde(1), T(2)]> + <[Htilde(2)_{1,2}, T(1)]>  (Eq. E(3), with the
 *          one- and two-body truncation of Htilde(2) stated after Eq. E(3))
 * with first- and second-order amplitudes of Eqs. T1_1st, T2_1st, T1_2nd and
 * T2_2nd (regulariser (1 - exp(-s D^2)) / D), H(0) the diagonal Fock blocks
 * of Eq. F0th, and two-electron integrals from the factorisation
 * (pq|rs) = sum_Q B^Q_pq B^Q_rs of Eq. int_fact.  The reference enters only
 * through gamma1 and the two- and three-body density cumulants.  E(0) is not
 * computed (it needs the bare one-electron integrals, which are not inputs).
 *
 * Orbitals are numbered core [0, nc), active [nc, nc+na), virtual
 * [nc+na, n), n = nc + na + nv, all spin-free (restricted) quantities.
 *
 * Errors: every int-returning call gives 0 on success or a negative
 * DSRG_ERR_* code; dsrg_last_error() then returns a message for the calling
 * thread.  No call aborts the process.  All computation runs in the
 * library's CUDA kernels on the current device; there is no CPU fallback.
 */
#ifndef DSRG_H
#define DSRG_H

#ifdef __cplusplus
extern "C" {
#endif

#define DSRG_OK 0
#define DSRG_ERR_ARG (-1)     /* invalid size, pointer or parameter          */
#define DSRG_ERR_OOM (-2)     /* device allocation failed                    */
#define DSRG_ERR_CUDA (-3)    /* CUDA runtime or launch error                */
#define DSRG_ERR_STATE (-4)   /* call out of order (e.g. NULL handle)        */
#define DSRG_ERR_INTERNAL (-5)
#define DSRG_ERR_TIMEOUT (-6) /* a bounded wait inside a kernel ran out; the
                                 kernel released its resources and returned,
                                 the results of the call are not valid       */

#define DSRG_MEM_HOST 0   /* input pointers are host memory; copied at load     */
#define DSRG_MEM_DEVICE 1 /* input pointers are device memory on the current GPU;
                             copied at load as well                            */

#define DSRG_PREC_FP64 0  /* every contraction in FP64                          */
#define DSRG_PREC_SPLIT 1 /* large contractions as split-precision tensor-core
                             products (see dsrg_split_gemm); everything else,
                             the regulariser and all reductions stay FP64     */

typedef struct dsrg_handle dsrg_handle;

/*
 * Problem inputs.  Row-major, FP64.  The caller keeps ownership; the
 * library copies everything during dsrg_init / dsrg_load.
 *   eps   [n]              semicanonical Fock diagonals (Eq. F0th)
 *   B     [naux][n][n]     three-index factor, symmetric in its last two
 *                          indices (Eq. int_fact)
 *   g1a, g1b [na][na]      active one-particle density per spin,
 *                          g1[u][v] = <a+_u a_v>
 *   l2aa, l2ab, l2bb [na]^4  two-body cumulant spin blocks,
 *                          l2xy[u][v][w][z] = lambda(a+_u a+_v a_z a_w) with
 *                          the spins of (u,w) and (v,z) given by x and y
 *   l3aaa, l3aab, l3abb, l3bbb [na]^6  three-body cumulant spin blocks,
 *                          l3[u][v][w][x][y][z] is the cumulant of
 *                          a+_u a+_v a+_w a_z a_y a_x; creators and
 *                          annihilators in each slot position carry the
 *                          spins named by the block (alpha first)
 *   f1    [n][n] or NULL   off-diagonal Fock part f^(1) (its core-core,
 *                          active-active and virtual-virtual blocks are
 *                          ignored); NULL means zero
 *   s                      flow parameter (> 0), in Eh^-2
 */
typedef struct {
  int nc, na, nv, naux;
  double s;
  const double *eps;
  const double *B;
  const double *g1a, *g1b;
  const double *l2aa, *l2ab, *l2bb;
  const double *l3aaa, *l3aab, *l3abb, *l3bbb;
  const double *f1;
  int memory; /* DSRG_MEM_HOST or DSRG_MEM_DEVICE */
} dsrg_inputs;

typedef struct {
  int precision;  /* DSRG_PREC_FP64 or DSRG_PREC_SPLIT                       */
  void *stream;   /* cudaStream_t to run on; NULL = the library's own stream */
  int slices;     /* DSRG_PREC_SPLIT: 7-bit digit slices per operand (1..8);
                     0 selects 6                                             */
  int tune;       /* DSRG_PREC_SPLIT: 1 = the first product of each new
                     (M, N, K, slices) shape in the process times a few tile
                     widths and k splits (on the caller's operands with
                     alpha = 0, so nothing changes) and keeps the fastest;
                     0 = fixed rules.  Results differ from the fixed rules
                     only in summation order.  With the environment
                     variable DSRG_TUNE_CACHE naming a file, decisions are
                     read from it (keyed by product shape, slices and GPU
                     model) and new ones appended, so later processes skip
                     the timing.  No counterpart in the paper.           */
  long long wait_limit; /* budget, in SM clock cycles, of every bounded wait
                     inside the split-precision kernel (on copies and
                     tensor-core products it issued itself); 0 selects 2^32
                     (about 2 s).  When a wait runs out the kernel stops
                     work, waits for what it has in flight, frees its tensor
                     memory and the call returns DSRG_ERR_TIMEOUT.  Negative
                     values are DSRG_ERR_ARG.  No counterpart in the paper. */
} dsrg_options;

typedef struct {
  double e2;   /* second-order energy E(2)                                  */
  double e3a;  /* <[Htilde(1), T(2)]>                                        */
  double e3b;  /* <[Htilde(2)_{1,2}, T(1)]>                                  */
  double e3;   /* e3a + e3b                                                  */
} dsrg_energies;

/* Create a handle on the current CUDA device and load the inputs.  On
 * success *out owns device memory until dsrg_free.  opts may be NULL. */
int dsrg_init(const dsrg_inputs *in, const dsrg_options *opts, dsrg_handle **out);

/* Replace the inputs of an existing handle with new ones of the same sizes
 * (no reallocation of the input arrays). */
int dsrg_load(dsrg_handle *h, const dsrg_inputs *in);

/* E(2) only (fills e2; e3* set to 0). Synchronises the handle's stream. */
int dsrg_pt2(dsrg_handle *h, dsrg_energies *out);

/* E(2) and E(3) components.  Synchronises the handle's stream. */
int dsrg_pt3(dsrg_handle *h, dsrg_energies *out);

typedef struct {
  double e2, e3a, e3b, e3;  /* the unrelaxed components, as dsrg_pt3          */
  double e_relaxed2;        /* one-step relaxed DSRG-MRPT2 energy, relative
                               to E0 (lowest eigenvalue of Hbar^[2])         */
  double e_relaxed3;        /* one-step relaxed DSRG-MRPT3 energy, relative
                               to E0 (lowest eigenvalue of Hbar^[3])         */
  double residual2, residual3; /* |H x - e x| of the unit eigenvector found */
  long long ndet;           /* determinants of the CI space                  */
  int steps2, steps3;       /* Lanczos steps taken                           */
} dsrg_relaxed_energies;

/*
 * One-step relaxed energies (paper Eq. E_relaxed with Eq. energy_relaxed;
 * App. A).  Evaluates the PT3 energy and, on the way, the all-active blocks
 * of the summed transformed Hamiltonian Hbar^[k]_{1,2} (k = 2: H^(0) + H^(1)
 * + 1/2 [Htilde(1), A(1)]; k = 3: plus 1/2 [Htilde(1), A(2)] +
 * 1/2 [Htilde(2), A(1)]); folds the core and rewrites the operator in
 * true-vacuum order with the reference's gamma1 and lambda2 (App. A), builds
 * its matrix over the determinants with n_alpha and n_beta electrons in the
 * na active orbitals, and returns the lowest eigenvalue of each (Lanczos on
 * the GPU).  E0 needs the bare integrals, which are not inputs: every energy
 * is relative to it, so e_relaxedk - (e2 [+ e3]) is the relaxation energy.
 * The active-space part of H^(0) is the given Fock diagonal.  The reference's
 * densities must be those of a state with n_alpha, n_beta active electrons
 * (no check is made).  Synchronises the handle's stream; drops a captured
 * batch graph as dsrg_pt3 does.
 * Errors: DSRG_ERR_ARG (out NULL, n_alpha or n_beta outside [0, na], more
 * than 20000 determinants), DSRG_ERR_STATE (NULL handle), otherwise as
 * dsrg_pt3.  Ownership: the caller keeps out.
 */
int dsrg_relaxed(dsrg_handle *h, int n_alpha, int n_beta, dsrg_relaxed_energies *out);

typedef struct {
  int iterations;                 /* Jacobi steps taken                          */
  int converged;                  /* 1: max |residual| <= tol x max |V[e,f,u,v]| */
  double max_residual;            /* largest |residual| of the returned amplitudes */
  double max_source;              /* largest |V[e,f,u,v]|                        */
  double min_shifted_denominator; /* smallest |Ds| over e, f and u != v          */
  long long pairs_not_converged;  /* virtual spin-orbital pairs (e, f) whose
                                     largest |residual| exceeds the tolerance    */
  long long small_denominators;   /* elements with |Ds| < 1e-2                   */
} dsrg_dyall_result;

/*
 * First-order aavv amplitudes with Dyall's zeroth-order Hamiltonian (paper
 * App. B, Eq. t2_aavv) at s -> infinity: for virtual spin orbitals e, f and
 * active u, v,
 *   0 = V[e,f,u,v] - D t[e,f,u,v] - 1/2 sum_xy Va[x,y,u,v] t[e,f,x,y]
 *                                 + sum_xyz Va[x,y,u,v] t[e,f,x,z] gamma[y,z]
 * (D = eps_u + eps_v - eps_e - eps_f, Va the all-active block of V).  Solved
 * by Jacobi iteration preconditioned by the shifted denominator Ds, the exact
 * diagonal of the system (D + Va[u,v,u,v] - sum_y (Va[u,y,u,v] gamma[y,v] -
 * Va[v,y,u,v] gamma[y,u])), until max |residual| <= tol x max |V| or max_iter
 * steps, or until the residual grows past 1e8 x max |V| (small shifted
 * denominators: the intruders App. B discusses).  No counterpart energy is
 * defined by the paper; the amplitudes are fetched as "Taavv".  The split
 * path runs the coupling product on the tensor cores.  Synchronises the
 * handle's stream.  Errors: DSRG_ERR_ARG (tol <= 0, max_iter < 1, out NULL),
 * DSRG_ERR_STATE (NULL handle), otherwise as dsrg_pt3.
 */
int dsrg_dyall_aavv(dsrg_handle *h, double tol, int max_iter, dsrg_dyall_result *out);

/*
 * PT3 energies of n independent instances (the points of a potential-energy
 * scan, any sizes), all in flight at once: handle i's energy runs on its own
 * stream and out[i] receives it.  No counterpart in the paper, which
 * evaluates points one by one; this is the batching of the hot path.  The
 * first call for a handle evaluates one energy eagerly (filling the handle's
 * buffer cache) and captures the energy as a CUDA graph; later calls replay
 * the graphs only, so the host issues n launches instead of thousands.  A
 * handle's graph is dropped by dsrg_pt2/dsrg_pt3 on it (eager evaluation) and
 * by dsrg_load (new inputs); the next batch call captures it again.  Every
 * handle keeps the device buffers of its captured energy, so the batch needs
 * the sum of the handles' peak memory (dsrg_peak_bytes).  The handles must be
 * distinct; handles sharing a stream run one after another.
 * Ownership: the caller keeps hs and out.  Errors: DSRG_ERR_ARG (n < 0, NULL
 * arrays, a repeated handle), DSRG_ERR_STATE (NULL handle), otherwise as
 * dsrg_pt3; after an error some out[i] may be unset.
 */
int dsrg_pt3_batch(dsrg_handle *const *hs, int n, dsrg_energies *out);

/* Release all device memory of the handle (NULL is ignored). */
void dsrg_free(dsrg_handle *h);

/* Message of the last failed call on this thread ("" if none). */
const char *dsrg_last_error(void);

/* Number of this library's kernel launches issued by the last dsrg_pt2 /
 * dsrg_pt3 / dsrg_relaxed / dsrg_dyall_aavv call on the handle (-1 on a
 * NULL handle). */
long long dsrg_last_launch_count(const dsrg_handle *h);

/* Per-kernel timing.  dsrg_profile(h, 1) makes later dsrg_pt2/dsrg_pt3 calls
 * bracket every launch of this library with CUDA events on the handle's
 * stream and accumulate, per kernel, the launch count, the summed device
 * time (ms), the FP64 flops of the contractions it computes (2 M N K each),
 * the flops it executes (split-precision products: every digit pair over the
 * padded tiles; FP64 kernels: the same as flops) and the bytes moved by
 * element-wise kernels; dsrg_profile(h, 0) stops.  Both reset the totals.
 * dsrg_profile_stats reads kernel index 0 .. 7 (generic FP64 contraction,
 * FP64 ladder (pr|qs) build, FP64 ladder contraction, axpy, dot, amplitude
 * kernels, split-precision operand packing, split-precision tensor-core
 * product); *name receives a static string.  DSRG_ERR_ARG past the last
 * index.  dsrg_profile_step reads the same launches grouped by the step of
 * the energy they belong to (first-order amplitudes, ladder build, ladder
 * contraction, ring, ...), in the order the steps first ran; *name stays
 * valid until the next profiled call.  No counterpart in the paper. */
int dsrg_profile(dsrg_handle *h, int enable);
int dsrg_profile_stats(const dsrg_handle *h, int kernel, const char **name, long long *launches, double *ms,
                       double *flops, double *exec_flops, double *bytes);
int dsrg_profile_step(const dsrg_handle *h, int step, const char **name, long long *launches, double *ms,
                      double *flops);

/* Device-to-host bytes read back by the last dsrg_pt2 / dsrg_pt3 call (the
 * per-block partial sums of the energy components; -1 on a NULL handle). */
long long dsrg_last_d2h_bytes(const dsrg_handle *h);

/* Peak device bytes held by the handle's tensor workspace. */
long long dsrg_peak_bytes(const dsrg_handle *h);

/*
 * Density-fitted particle-particle ladder on caller buffers (Eq.
 * scaling_problem with the factorised integrals of Eq. int_fact): for
 * p, q, r, s in [0, np) and i, j in [0, nh)
 *   L[p][q][i][j] = sum_{r,s} (sum_Q B[Q][p0+p][p0+r] B[Q][p0+q][p0+s]) t[r][s][i][j]
 * B: device [naux][n][n]; t: device [np][np][nh][nh]; L: device
 * [np][np][nh][nh], overwritten.  All FP64, row-major, device memory of the
 * current GPU; stream may be NULL (legacy default stream).  With t the
 * alpha-beta block of the spin-free first-order amplitudes this is the
 * spatial ladder from which the energy driver assembles all spin blocks.
 * The (pr|qs) rows are formed in batches in a scratch buffer of at most
 * 1 GiB obtained with cudaMalloc and released before return; the call
 * synchronises `stream`.  Errors: DSRG_ERR_ARG (sizes, p0 + np > n, NULL
 * pointers), DSRG_ERR_OOM (scratch), DSRG_ERR_CUDA.
 */
int dsrg_df_ladder(int n, int naux, int p0, int np, int nh, const double *B, const double *t, double *L,
                   void *stream);

/*
 * dsrg_df_ladder without any device allocation.  No counterpart in the
 * paper: it serves callers that may not call cudaMalloc, such as frameworks
 * whose caching allocator reserved the device memory up front (a library
 * allocation would fail or fragment their pool) and embedded or real-time
 * runtimes that forbid allocation after start-up.  Same arguments,
 * contraction and result as dsrg_df_ladder; no cudaMalloc, cudaFree or
 * allocating library routine is called.  The (pr|qs) rows live in one fixed
 * file-scope device array of 2^22 doubles (32 MiB) that every GPU on which
 * the library's device code is loaded holds until the process exits, so
 * np^3 <= 2^22 (np <= 161) is required; larger np returns DSRG_ERR_ARG with
 * a message.  Set-up: the first call on a device (and the first call after
 * that device's context changed, e.g. after cudaDeviceReset) looks up the
 * array's device address with the device current.  All calls share the
 * array and it keeps the last call's contents (each batch clears what it
 * accumulates into); calls that overlap on the GPU (other streams, other
 * host threads) race on it and must be serialised by the caller.
 * Synchronises `stream`.
 */
int dsrg_df_ladder_noalloc(int n, int naux, int p0, int np, int nh, const double *B, const double *t, double *L,
                           void *stream);

/*
 * Pivoted incomplete Cholesky factorisation of a two-electron supermatrix,
 * giving the three-index factor of Eq. int_fact, (pq|rs) ~ sum_Q B^Q_pq B^Q_rs,
 * as for the Cholesky integrals of the paper's larger applications (Sec. IV,
 * thresholds 1e-6 and 1e-8 a.u.; algorithm of Beebe and Linderberg).
 *   V       device [N][N], FP64, row-major, symmetric positive semidefinite
 *           (for integrals N = n^2 and V[p n + q][r n + s] = (pq|rs)); read
 *           by rows, never written
 *   tau     threshold >= 0: the factorisation stops when the largest
 *           remaining diagonal D[J] = V[J][J] - sum_Q B[Q][J]^2 is <= tau
 *   max_vecs  capacity of B (stops there at the latest)
 *   B       device [max_vecs][N] output: B[Q] = (V[J_Q] - sum_{Q'<Q} B[Q'] B[Q'][J_Q]) / sqrt(D[J_Q]),
 *           J_Q the pivot of step Q (largest D, the smallest index on ties);
 *           rows past *nvecs are left untouched
 *   nvecs   host, receives the number of vectors formed
 *   pivots  host [max_vecs] or NULL, receives J_0 .. J_{nvecs-1}
 * Corrections are summed over Q' in increasing order with one rounding per
 * product and per sum (no fused multiply-add), so results are reproducible
 * operation by operation.  Scratch (N + max_vecs + a few thousand doubles)
 * is allocated and released inside the call; synchronises `stream`.
 * Errors: DSRG_ERR_ARG (sizes, tau < 0, NULL pointers), DSRG_ERR_OOM,
 * DSRG_ERR_CUDA.
 */
int dsrg_cholesky(long long N, const double *V, double tau, int max_vecs, double *B, int *nvecs, long long *pivots,
                  void *stream);

/*
 * Split-precision FP64 matrix product on the tensor cores (no counterpart in
 * the paper: it is the contraction primitive of the mixed-precision path):
 *   C[m][n] += alpha * sum_k A[m][k] B[k][n]
 * A [M][K] (row stride lda), B [K][N] (row stride ldb), C [M][N] (row stride
 * ldc), all FP64 device memory, row-major.  Every row of A and column of B is
 * scaled by a power of two, rounded to a grid of 2^(7*slices - 1) steps and
 * cut into `slices` (1..8) balanced base-128 digits (|d| <= 64) held exactly
 * in BF16; digit products are accumulated exactly in FP32 over 480-long
 * windows of k by tcgen05.mma and added into a two-float running sum, so the
 * result carries about 7*slices bits relative to the product of the row and
 * column maxima (Ozaki et al., Numer. Algorithms 59 (2012) 95).  With one
 * slice, integers |x| <= 63 are held exactly.
 * Scratch is allocated and released inside the call; synchronises `stream`.
 * Errors: DSRG_ERR_ARG (sizes >= 2^31, slices, NULL), DSRG_ERR_OOM (scratch),
 * DSRG_ERR_CUDA (launch failure), DSRG_ERR_TIMEOUT (a bounded wait inside the
 * kernel ran out, default budget).
 */
int dsrg_split_gemm(long long M, long long N, long long K, const double *A, long long lda, const double *B,
                    long long ldb, double *C, long long ldc, double alpha, int slices, void *stream);

/*
 * Intermediate access for testing.  Copies a named spin-orbital tensor of the
 * last dsrg_pt2/dsrg_pt3 call to host memory `dst` (FP64, row-major) if its
 * element count equals `count`.  Names and layouts, with H = core+active
 * (h = nc+na) and P = active+virtual (p = na+nv), each slot spin-major
 * (index sigma*len + x):
 *   "T1" [2p][2h], "T2" [2p][2p][2h][2h]       first-order amplitudes
 *   "T1b" [2p][2h], "T2b" [2p][2p][2h][2h]     second-order amplitudes
 *   "O1" [2p][2h], "O2" [2p][2p][2h][2h]       excitation blocks of
 *                                              1/2 [Htilde(1), A(1)]_{1,2}
 *   "Hbar1_2" [2na][2na], "Hbar2_2" [2na]^4    all-active blocks of
 *                                              H^(0) + H^(1) + 1/2 [Htilde(1), A(1)]
 *   "Hbar1_3" [2na][2na], "Hbar2_3" [2na]^4    all-active blocks of
 *                                              1/2 [Htilde(1), A(2)] + 1/2 [Htilde(2), A(1)]
 *                                              (the last dsrg_relaxed call)
 *   "Taavv" [2nv][2nv][2na][2na]               aavv amplitudes of the last
 *                                              dsrg_dyall_aavv call
 * Spin blocks that change the number of alpha electrons are zero (the library
 * does not store them and fills them in on the copy).  O1 and O2 are kept
 * only while one [P,P,H,H] tensor takes at most 1 GiB (stored blocks);
 * beyond that they are folded into Htilde(2) and released, and fetching
 * them returns DSRG_ERR_STATE.
 * Returns DSRG_ERR_ARG for an unknown name or a wrong count.
 */
int dsrg_fetch(const dsrg_handle *h, const char *name, double *dst, long long count);

#ifdef __cplusplus
}
#endif
#endif /* DSRG_H */

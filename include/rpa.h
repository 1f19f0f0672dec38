/*
 * rpa.h - C ABI of the GB300 static-subspace RPA correlation-energy path.
 *
 * Method: Weinberg et al., "Static subspace approximation for random phase
 * approximation correlation energies" (arXiv:2405.20258).  One q-point's work:
 *
 *   chi0(0)  = -(1/Omega) A^H diag(f(0)) A             Eq. (chi0_partial_occs)
 *   chi~(0)  = v^1/2 chi0(0) v^1/2,  v(G) = 4 pi/|q+G|^2 Eq. (rpaE), symmetrised
 *   C        = N_eig eigenvectors of chi~(0) with the most negative eigenvalues (Method, C_s)
 *   M~       = (A v^1/2 C)^H                            Method, M_s = M C_s
 *   chi_s(k) = -(1/Omega) M~ diag(f(w_k)) M~^H           Method, chi0_s = M_s^+ Delta M_s
 *   E_c      = (1/2pi) sum_k w_k sum_i [ln(1 - l_ki) + l_ki]   Eq. (rpaE), trace in the subspace
 *
 * with A[vc][g] = M_vc(G_g) (Eq. pwMat), row vc = v*n_c + c (k-points first when
 * there are several), and the transition weight f_vc(w) = w_vc 4 D_vc /
 * (D_vc^2 + w^2), D_vc = e_c[c] - e_v[v], w_vc = g_k (f_v - f_c) (1 for integer
 * occupations): the resonant and anti-resonant terms of Delta_vck(q, iw) with
 * the spin factor 2.  The frequencies w_k, weights are
 * Gauss-Legendre points on [0,1] mapped by w = s t/(1-t) (Computational Details).
 *
 * Conventions shared by every entry point
 *  - Complex arrays are interleaved (re, im) pairs, row-major, in DEVICE memory
 *    unless the argument says "host".  The caller owns every array it passes;
 *    the plan owns its workspace and frees it in rpa_plan_destroy.
 *  - All work is enqueued on the plan's CUDA stream.  rpa_plan_create,
 *    rpa_subspace_basis (it reads the eigensolver's status), rpa_plan_frequencies
 *    and rpa_ecorr (both return values to the host) synchronise it.  The mixed
 *    path also cuts digit planes on an internal stream of its own, which every
 *    entry point joins into the plan's stream before it returns, so a caller
 *    sees all of a call's work ordered on the plan's stream.
 *  - Memory: the mixed path's digit planes are sized for the largest q-point
 *    within budgets (about 64 GB for the chi_s planes, 48 GB for the
 *    projection's, which then runs in row chunks); the rest is a few arrays of
 *    the problem's own sizes.
 *  - Errors are returned, never aborted on.  After RPA_EINVAL or RPA_ESTATE the
 *    plan is unchanged and stays usable.  rpa_last_error() gives a message.
 *  - Stages of one q-point must run in order chi0 -> basis -> freq -> ecorr.
 *    The plan holds one q-point's outputs per stage (chi~, the basis, M~ and
 *    chi_s): stages of different q-points may interleave as long as each stage
 *    finds its predecessor's outputs for its own q-point; otherwise (called
 *    early, or after another q-point's stage replaced them) it returns
 *    RPA_ESTATE.
 *  - Output pointers marked "may be NULL" are optional copies of intermediates.
 *  - Not thread-safe per plan: one host thread drives one plan at a time.
 */
#ifndef RPA_H
#define RPA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RPA_OK = 0,
  RPA_EINVAL = 1,    /* bad argument: sizes, NULL pointer, unknown option   */
  RPA_ENOMEM = 2,    /* device or host allocation failed                    */
  RPA_ECUDA = 3,     /* a CUDA runtime call failed                          */
  RPA_EEIG = 4,      /* an eigensolver reported failure (info != 0)         */
  RPA_ENUMERIC = 5,  /* non-finite value or 1 - lambda <= 0 in the energy   */
  RPA_ETIMEOUT = 6,  /* a bounded device wait gave up                       */
  RPA_ESTATE = 7     /* stage called out of order                           */
} rpa_status;

typedef enum {
  RPA_FP64 = 0,         /* every contraction in FP64 (SIMT DFMA)                           */
  RPA_MIXED = 1,        /* contractions on BF16 tensor cores with exact digit slicing
                           (default slices 4, 6, 3: |dE_c| <= 1e-6 Ha on every tested
                           workload), FP64 solves, trace and log-sum                    */
  RPA_MIXED_BF16X3 = 2, /* every contraction on round-to-nearest BF16 hi/lo planes, 3
                           products (hi.hi + hi.lo + lo.hi), FP32 sums over K: the
                           classic split; does not reach 1e-6 Ha (for comparison)      */
  RPA_MIXED_BF16X6 = 3, /* the same with hi/mid/lo planes, 6 products                  */
  RPA_MIXED_TF32X3 = 4  /* every contraction on TF32 hi/lo planes (kind::tf32 tensor cores),
                           3 products, FP32 sums over K (for comparison)                */
} rpa_precision;

typedef enum {
  RPA_ROUTE_CHOLESKY = 0, /* default: ln det(1 - chi_s) = sum ln(1 - l) from a tiled FP64
                             Cholesky factor + the FP64 trace term (the paper evaluates
                             Tr ln through a factorisation)                               */
  RPA_ROUTE_EIG = 1       /* eigenvalues of each chi_s(k): sum ln(1 - l) + l (cuSOLVER)   */
} rpa_energy_route;

typedef enum { RPA_C128 = 0, RPA_C64 = 1 } rpa_dtype;

typedef enum {
  RPA_COULOMB_BARE = 0,  /* v = 4 pi/|q+G|^2 (the interaction of Eq. rpaE)                  */
  RPA_COULOMB_SLAB = 1   /* 1/r cut off at |z| > z_c: v = 4 pi/|q+G|^2 [1 - exp(-|q+G|_par z_c)
                            cos((q+G)_z z_c)] for (q+G)_z on the lattice of a cell of height
                            2 z_c (for slabs; the paper names no truncation)              */
} rpa_coulomb;

/* One q-point.  Arrays are device memory owned by the caller and must stay
 * valid and unchanged until the plan is destroyed. */
typedef struct {
  int n_g;                 /* plane waves N_G >= 1                                  */
  int n_v, n_c;            /* valence / conduction bands, N_vc = n_v*n_c >= 1       */
  int n_eig;               /* subspace size, 1 <= n_eig <= n_g                      */
  int n_freq;              /* Gauss-Legendre points, 1 <= n_freq <= 256             */
  double omega_cell;       /* cell volume Omega (bohr^3) > 0                        */
  const double* qg2;       /* [n_g] |q+G|^2 (bohr^-2) > 0                           */
  const double* e_v;       /* [n_v] valence energies (Ha)                           */
  const double* e_c;       /* [n_c] conduction energies (Ha), e_c[c] > e_v[v]       */
  const void* m;           /* [n_v*n_c][n_g] A = M_vc(G), complex of m_dtype;
                              NULL: drawn on the device by the counter generator    */
  int m_dtype;             /* rpa_dtype of m                                        */
  int iq;                  /* q index fed to the generator (m == NULL)              */
  unsigned long long seed; /* generator seed (m == NULL)                            */
  const int* miller;       /* [n_g][3] Miller indices of G (m == NULL)              */
  /* k-points and occupations, Eq. (chi0_partial_occs): every transition carries the
     pair weight w = g_k (f_v - f_c); zero / NULL fields give one k-point and integer
     occupations (w = 1).  w * Delta must be >= 0, and Delta != 0 where w != 0. */
  int n_k;                 /* k-points folded into the transitions (0 means 1): e_v is
                              then [n_k][n_v], e_c [n_k][n_c], m [n_k][n_v][n_c][n_g]
                              (the generator draws band indices k*n_v+v, k*n_c+c)     */
  const double* k_weight;  /* [n_k] g_k (device); NULL: 1 for every k-point          */
  const double* occ_v;     /* [n_k][n_v] occupations f_v (device); NULL: 1           */
  const double* occ_c;     /* [n_k][n_c] occupations f_c (device); NULL: 0           */
  int coulomb;             /* rpa_coulomb                                            */
  double slab_zc;          /* RPA_COULOMB_SLAB: z_c > 0 (bohr)                       */
  const double* qg_vec;    /* RPA_COULOMB_SLAB: [n_g][3] Cartesian q+G (bohr^-1, device) */
} rpa_qpoint;

typedef struct {
  int precision;           /* rpa_precision                                          */
  int energy_route;        /* rpa_energy_route                                       */
  double omega_scale;      /* s of the frequency map w = s t/(1-t); <= 0 means 0.5 Ha */
  int timing;              /* nonzero: record CUDA events around every stage kernel  */
  int slices_chi0;         /* RPA_MIXED: digit slices of chi~(0) operands (1..8; 0 = 4) */
  int slices_proj;         /* RPA_MIXED: digit slices of the projection (1..8; 0 = 6)  */
  int slices_chis;         /* RPA_MIXED: digit slices of chi_s operands (1..8; 0 = 3)  */
  int debug_stall;         /* test hook, 0 in production: 1 makes the tensor-core
                              producer issue no loads, so every bounded wait of the
                              GEMM runs out and the stage reports RPA_ETIMEOUT     */
  int vc_chunk;            /* q-points with m == NULL: 0 draws the whole A once and keeps
                              it resident; > 0 never holds A whole: the chi~ and the
                              projection stages draw it again, one chunk of at most
                              vc_chunk transitions (whole valence bands of one k-point)
                              at a time, into a buffer of that size                    */
  int reserved[2];         /* zero                                                   */
} rpa_options;

/* Stage timers of rpa_plan_timings. */
typedef enum {
  RPA_T_CHI0 = 0,   /* chi~(0) contraction                                               */
  RPA_T_EIG0 = 1,   /* FP64 eigensolve of chi~(0) and gauge fixing                       */
  RPA_T_PROJ = 2,   /* projection M~                                                     */
  RPA_T_CHIS = 3,   /* chi_s(w_k) contraction for every k                                */
  RPA_T_TRACE = 4,  /* FP64 trace term                                                   */
  RPA_T_EIGS = 5,   /* eigenvalues (or Cholesky) of every chi_s(w_k)                     */
  RPA_T_ENERGY = 6, /* final log-sum and quadrature                                      */
  RPA_T_OTHER = 7,  /* scalars, mirrors, copies                                          */
  RPA_T_SLICE = 8,  /* mixed path: cutting FP64 operands into BF16 digit planes          */
  RPA_N_TIMERS = 9
} rpa_timer;

typedef struct rpa_plan_s* rpa_plan_t;

/* Create a plan for n_q q-points: validate, record the descriptors, allocate
 * workspace for the largest q-point, build the frequency grid on the device.
 * stream: a cudaStream_t (NULL = legacy default stream).  opt may be NULL
 * (FP64, Cholesky route, s = 0.5).  On failure *out is NULL. */
rpa_status rpa_plan_create(rpa_plan_t* out, const rpa_qpoint* q, int n_q,
                           const rpa_options* opt, void* stream);
rpa_status rpa_plan_destroy(rpa_plan_t plan);
const char* rpa_last_error(rpa_plan_t plan);   /* plan may be NULL: last create error */
const char* rpa_status_string(int status);

/* Static polarizability chi~(0) = -(1/Omega) v^1/2 A^H diag(f(0)) A v^1/2,
 * Eq. (chi0_partial_occs) at w = 0 and the symmetrisation of Eq. (rpaE).
 * chi_tilde_out: [n_g][n_g] complex128, full Hermitian matrix, may be NULL. */
rpa_status rpa_chi0_static(rpa_plan_t plan, int iq, void* chi_tilde_out);

/* Subspace basis (Method, C_s): the n_eig eigenpairs of chi~(0) with the most
 * negative eigenvalues, FP64 Hermitian eigensolve, ascending order; each
 * eigenvector's entry of largest modulus (lowest g on ties) is made real > 0.
 * lambda_out: [n_eig] float64, may be NULL.  c_out: [n_g][n_eig] complex128,
 * may be NULL.  Returns RPA_EEIG if the solver fails. */
rpa_status rpa_subspace_basis(rpa_plan_t plan, int iq, double* lambda_out, void* c_out);

/* Projection and frequency-dependent subspace polarizabilities (Method):
 * M~ = (A v^1/2 C)^H, chi_s(k) = -(1/Omega) M~ diag(f(w_k)) M~^H for every
 * quadrature node, and the FP64 trace T_k = -(1/Omega) sum_vc f_vc(w_k) |M~[:,vc]|^2.
 * mtilde_out: [n_eig][n_v*n_c] complex128, may be NULL.
 * chi_s_out:  [n_freq][n_eig][n_eig] complex128 (full Hermitian), may be NULL.
 * trace_out:  [n_freq] float64, may be NULL. */
rpa_status rpa_chi_freq(rpa_plan_t plan, int iq, void* mtilde_out, void* chi_s_out,
                        double* trace_out);

/* Correlation energy of Eq. (rpaE) in the subspace: eigenvalues of every
 * chi_s(k) (FP64), or ln det(1 - chi_s) by Cholesky on the Cholesky route, then
 * E_c = (1/2pi) sum_k w_k [sum_i log1p(-l_ki) + T_k].  Synchronises the stream.
 * ec_host: host float64 [1] (iq >= 0) or [n_q] (iq == -1: every q-point, each
 * run through all stages).  lam_out: [n_freq][n_eig] float64 device, may be
 * NULL (eigenvalue route only).  RPA_ENUMERIC if any 1 - l <= 0 or a value is
 * not finite. */
rpa_status rpa_ecorr(rpa_plan_t plan, int iq, double* ec_host, double* lam_out);

/* The quadrature the plan uses: omega_host, weight_host host float64 [n_freq]
 * of q-point iq (weights include the Jacobian of the map). */
rpa_status rpa_plan_frequencies(rpa_plan_t plan, int iq, double* omega_host, double* weight_host);

/* Device generator of synthetic matrix elements (the counter-based splitmix64
 * and Box-Muller recipe of the input generator): writes A[v][c][g] for
 * v in [v0, v0+nv), c in [c0, c0+nc) to out ([nv*nc][q->n_g] complex of dtype).
 * Uses q->seed, q->iq, q->miller, q->qg2 (device).  Asynchronous on stream. */
rpa_status rpa_generate_m(const rpa_qpoint* q, int v0, int nv, int c0, int nc,
                          void* out, int dtype, void* stream);

/* Device time per stage (ms) accumulated since the previous call, from CUDA
 * events on the plan's stream (plans created with opt->timing != 0; zeros
 * otherwise), and the number of kernels the library itself launched since the
 * previous call (library solvers' internal kernels not counted).  Synchronises
 * the stream.  times_ms: host [RPA_N_TIMERS] or NULL; launches: host or NULL. */
rpa_status rpa_plan_timings(rpa_plan_t plan, double* times_ms, long long* launches);

/* Allocation-free trace term, for callers that cannot allocate device memory
 * where they call it (their device memory is fully reserved by their own pool
 * allocator, or they must not cause the device-wide synchronisation that
 * cudaMalloc/cudaFree can bring).  The paper has no counterpart: it is the
 * trace term of rpa_chi_freq, T_k = -(1/Omega) sum_vc f_vc(w_k) |M~[:,vc]|^2,
 * computed without a plan and without any allocation.
 *   mtilde    [n_eig][n_v*n_c] complex128 (device), e.g. rpa_chi_freq's mtilde_out
 *   e_v, e_c  [n_v], [n_c] band energies (device); omega [n_freq] (device)
 *   trace_out [n_freq] float64 (device), written on `stream` (a cudaStream_t).
 * Scratch is a fixed library array of RPA_STATIC_TRACE_MAX_VC doubles (4 MiB)
 * that every GPU loading the library holds until the process exits; larger
 * n_v*n_c is rejected with RPA_EINVAL (message in rpa_last_error(NULL)).  The
 * first call on a device looks up that array's device address (once per
 * device, with the device current): make that first call before any stream
 * capture.  That address is kept for the life of the process: do not reset the
 * device (cudaDeviceReset) between calls, since the array then belongs to a
 * context that no longer exists.  All calls share the array, so calls that
 * overlap on the GPU race; each call overwrites the entries it reads.
 * Asynchronous: no host sync. */
#define RPA_STATIC_TRACE_MAX_VC 524288
rpa_status rpa_trace_term_static(const void* mtilde, int n_eig, int n_v, int n_c,
                                 const double* e_v, const double* e_c, const double* omega,
                                 int n_freq, double omega_cell, double* trace_out, void* stream);

/* Building blocks of the subspace step (a3), for checking each on its own.  Both
 * allocate their scratch per call and synchronise `stream` (a cudaStream_t, NULL:
 * the legacy default stream).  Errors: RPA_EINVAL, RPA_ENOMEM, RPA_ECUDA,
 * RPA_ETIMEOUT (a grid barrier gave up waiting); message in rpa_last_error(NULL).
 *
 * rpa_tridiagonalize: the Householder reduction that starts the eigensolver,
 * T = Q^H A Q real symmetric tridiagonal, in FP32 (bits = 32: a is complex64) or
 * FP64 (bits = 64: complex128).  a: device, n x n Hermitian, column-major, full
 * storage; overwritten with the reflectors.  d: device, n reals (float or double
 * as bits), the diagonal of T; e: device, n-1 reals, its off-diagonal.
 *
 * rpa_hermitian_eig_jacobi: all eigenpairs of a Hermitian m x m matrix (m <=
 * 4096) by the cyclic two-sided Jacobi solver of the Rayleigh-Ritz step, in FP64.
 * g: device, complex128 column-major, destroyed; theta: device, m doubles,
 * ascending; y: device, complex128 m x m column-major, the eigenvectors in the
 * same order. */
rpa_status rpa_tridiagonalize(int n, int bits, void* a, void* d, void* e, void* stream);
rpa_status rpa_hermitian_eig_jacobi(int m, void* g, double* theta, void* y, void* stream);

/* Transition order of the mixed path's chi~(0) (allocates its scratch per call,
 * synchronises `stream`).  The paper has no counterpart: this is the library's own
 * arrangement of the transitions into the K-blocks of the digit-sliced chi~(0)
 * contraction, each block with its own digit scale, so that a block holds
 * transitions of similar weight f_vc(0) (Eq. chi0_partial_occs: f proportional to
 * |w / Delta|).  order[pos] = the transitions vc < n by decreasing key
 * |ow[vc] / delta[vc]| (0 where either is 0), equal keys by increasing vc: the
 * permutation of a stable sort.  seg_bands > 0 (a q-point drawn in chunks of
 * seg_bands valence bands): sorted within each segment of seg_bands bands of one
 * k-point (the last of a k-point may be shorter), as indices local to the segment's
 * first transition; n is then a multiple of n_v * n_c, transitions numbered
 * (k, v, c) with c fastest.  delta, ow: device, n doubles; order: device, n ints.
 * Errors: RPA_EINVAL (n < 1, n_v or n_c < 1, seg_bands outside 0..n_v, n not a
 * multiple of n_v * n_c when seg_bands > 0, NULL pointer), RPA_ENOMEM, RPA_ECUDA;
 * message in rpa_last_error(NULL). */
rpa_status rpa_transition_order(int n, int n_v, int n_c, int seg_bands, const double* delta,
                                const double* ow, int* order, void* stream);

/* Library version string. */
const char* rpa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RPA_H */

/*
 * ed.h -- C ABI of the GB300 exact-diagonalisation library (libedgb.so).
 *
 * The library applies the Hamiltonian of an impurity or cluster model to a
 * vector inside one (N_up, N_dn) particle-number sector, runs Lanczos (full
 * basis, three-vector, or thick-restart) for the lowest eigenpairs, evaluates
 * continued-fraction Green's functions at Matsubara or real frequencies and
 * one DMFT self-consistency update, all on one GPU; sectors can be solved in
 * batches and impurity solves served as a request stream.  The problem is the
 * one arXiv 1004.3354 solves: diagonalise the impurity Hamiltonian for its
 * lowest states (Sec. 2, after Eq. 3) with a Lanczos/Arnoldi solver built on
 * repeated H*v (Sec. 3), then form G(i w_n) (Eq. 3) for the DMFT loop (Sec. 2).
 *
 * Conventions shared by every call
 *  - Every call returns an ed_status.  ED_OK is 0.  On error, ed_last_error()
 *    gives a message for the calling thread; no C++ exception crosses the ABI.
 *  - Opaque handles (ed_ctx, ed_sector) are owned by the library and freed by
 *    the matching *_destroy call.  Destroying NULL is ED_OK.
 *  - Vector arguments are DEVICE pointers owned by the caller (for instance
 *    torch.Tensor.data_ptr()).  Scalars, model parameters and returned results
 *    are HOST memory.  `stream` is a cudaStream_t passed as void* (NULL = the
 *    legacy default stream).  Calls are stream-ordered: they enqueue work on
 *    `stream` and return without synchronising, except where a host result is
 *    returned, which implies a synchronisation of `stream`.
 *  - Basis and layout: site i is bit i of an n_s-bit spin string; each spin's
 *    strings with the sector's particle number are listed in ascending numeric
 *    order and a string's rank is its position there (combinatorial number
 *    system: rank(s) = sum_k C(p_k, k+1) over the set-bit positions
 *    p_0 < p_1 < ...).  A sector vector is the row-major D_up x D_dn array
 *    X[r_up][r_dn], flat index r_up * D_dn + r_dn.  Fermion sign order: every
 *    spin-up mode precedes every spin-down mode.
 *  - Vector element formats, chosen per sector by ed_prec:
 *      ED_PREC_FP64  IEEE double; arithmetic in native FP64.
 *      ED_PREC_DF64  "double-float": each element is two floats {hi, lo} with
 *                    value hi + lo (8 bytes, |lo| <= ulp(hi)); arithmetic in
 *                    error-free float transformations (about 2^-46 relative).
 *                    Values must lie within float's exponent range.
 *      ED_PREC_FP32  float storage.  The fast H*v path (natural-order
 *                    kernel) sums each element in float in two passes
 *                    (diagonal and down hops; up hops, spin-flip and pair-hop)
 *                    with coefficients rounded to float and adds the two
 *                    partial sums with one rounding: to first order in
 *                    u = 2^-24, |y_i - (Hx)_i| <= u [(n_A + 1) sum_A |H_ij x_j|
 *                    + 4 S_i |x_i| + (n_B + 1) sum_B |H_ij x_j| + |(Hx)_i|],
 *                    with sum_A over the n_A entries of the row's own up string
 *                    (diagonal and down hops), sum_B over the n_B others and
 *                    S_i the summed magnitude of the density terms (T_ii, U,
 *                    U', U' - J) present in state i, from which the diagonal
 *                    is formed (tested element by element; about (n + 3) u
 *                    sum_j |H_ij x_j| for n terms when the diagonal does not
 *                    cancel).  The other H*v kernels (general models) form
 *                    every product and sum in double-float and round once.
 *                    Dot products and norms accumulate in double-float.
 */
#ifndef ED_H
#define ED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ED_ABI_VERSION 3

typedef enum ed_status {
  ED_OK = 0,
  ED_ERR_INVALID = 1,        /* bad argument or model */
  ED_ERR_OOM = 2,            /* the context's HBM budget or the device is exhausted */
  ED_ERR_CUDA = 3,           /* a CUDA runtime call failed (message has the CUDA error) */
  ED_ERR_TIMEOUT = 4,        /* a bounded device wait ran out */
  ED_ERR_NOT_CONVERGED = 5,  /* iteration limit reached; partial results are returned */
  ED_ERR_BUSY = 6            /* resource in use */
} ed_status;

typedef enum ed_prec { ED_PREC_FP64 = 0, ED_PREC_DF64 = 1, ED_PREC_FP32 = 2 } ed_prec;

#define ED_SPIN_UP 0
#define ED_SPIN_DN 1
#define ED_MAX_SITES 31
#define ED_MAX_ORB 8
#define ED_MAX_K 64

/* Sector creation flags. */
#define ED_SECTOR_CSR 1u      /* also build the stored CSR matrix (Fig. 1 layout), FP64 only */
#define ED_SECTOR_GENERIC 2u  /* skip the row-kernel tables: H*v uses the generic kernels only */
#define ED_SECTOR_ACC_DF 4u   /* FP32 vectors: keep double-float sums in H*v (the two-row kernel)
                                 instead of the natural-order kernel's float sums */

typedef struct ed_ctx ed_ctx;
typedef struct ed_sector ed_sector;

/*
 * Model parameters (host memory, copied by ed_sector_create).
 *
 *   H = sum_{ij,s} T_ij c+_is c_js + sum_i U_site[i] n_iu n_id
 *     + sum_{m<m'<n_orb, s,s'} (Up - J delta_ss') n_ms n_m's'
 *     - sum_{m != m' < n_orb} [ Jsf d+_mu d_md d+_m'd d_m'u + Jph d+_mu d+_md d_m'u d_m'd ]
 *
 * Eq. 1 (Hubbard): T = -t, U_site = U, n_orb = 0.  Eq. 2 (Anderson impurity):
 * star-shaped T (T_0k = V_k, T_kk = eps_k, T_00 = eps_d), U_site[0] = U,
 * n_orb = 1.  Sec. 4 (Kanamori): T_mm = eps_m - mu, T_kk = eps_k, T_mk = V_mk,
 * U_site[m] = U on the orbital sites, Up = U', J, Jsf = Jph = J'.  The sums over
 * m, m' run over the impurity-orbital sites orb0 .. orb0 + n_orb - 1.
 * Requirements: 1 <= n_s <= 31; T exactly symmetric; 0 <= n_orb <= 8;
 * 0 <= orb0 and orb0 + n_orb <= n_s; the orbital sites lie within one aligned
 * block of 8 sites counted from the lowest site that carries U_site != 0 or an
 * orbital.  Placing the orbitals on the highest sites makes ascending string
 * order group strings by impurity occupation (the fast layout).
 */
typedef struct ed_model {
  int n_s;
  const double* T;       /* n_s * n_s, row-major */
  const double* U_site;  /* n_s */
  int n_orb;             /* M impurity orbitals ... */
  int orb0;              /* ... on sites orb0 .. orb0 + M - 1 */
  double Up, J, Jsf, Jph;
} ed_model;

/* Sizes of a sector and its tables. */
typedef struct ed_sector_info {
  int n_s, n_up, n_dn, prec;
  uint64_t D_up, D_dn, dim;
  uint64_t hops_up, hops_dn;    /* entries in each spin's hop table */
  uint64_t mix_up;              /* entries in the up-string spin-flip/pair-hop list */
  uint64_t csr_nnz;             /* stored CSR entries (0 without ED_SECTOR_CSR) */
  uint64_t table_bytes;         /* device bytes held by the sector */
  double   nnz_per_row;         /* mean stored entries per row of H (diagonal included) */
  int      kernel;              /* H*v kernel in use: 0 flat, 1 row-staged generic, 2 fast row
                                   kernel, 3 fast two-row kernel (DF64 when the autotuner picks
                                   it; FP32 where 4 does not apply), 4 natural-order float kernel
                                   (the FP32 default) */
} ed_sector_info;

/* ------------------------------------------------------------------ errors */
/* Copy the calling thread's last error message into buf (NUL-terminated). */
int ed_last_error(char* buf, size_t len);
/* Compile-time ABI version of the loaded library. */
int ed_abi_version(void);

/* ----------------------------------------------------------------- context */
/* Bind the calling thread to `device` and create a context whose own device
 * allocations (tables, Lanczos workspaces) may not exceed hbm_budget bytes
 * (0 = no limit beyond the device).  Errors: ED_ERR_INVALID (no such device),
 * ED_ERR_CUDA.
 * A context holds one reduction scratch buffer (device partial sums and a
 * pinned host result word) that ed_dot, ed_lanczos, ed_lanczos_tr and the
 * Green's-function calls of that context all use, whatever stream they are
 * given: calls on one context must therefore be serialised (one thread and one
 * stream at a time, or the caller's own ordering between streams).  Use one
 * context per concurrent caller; the request server keeps private scratch per
 * request for this reason. */
int ed_ctx_create(int device, size_t hbm_budget, ed_ctx** out);
int ed_ctx_destroy(ed_ctx* ctx);
/* Bytes of device memory currently held by the context and its sectors. */
int ed_ctx_bytes_in_use(const ed_ctx* ctx, size_t* out);

/* ------------------------------------------------------------------ sector */
/* Build the sector tables on the device (the model-dependent set-up that replaces
 * constructing H, Table 1's T_setup): both spins' bases, hop tables with
 * fermion signs, spin-flip/pair-hop maps and diagonal tables; with
 * ED_SECTOR_CSR also the explicit CSR matrix (Fig. 1 layout, columns ascending,
 * diagonal always stored).  Synchronises the context's device.
 * Errors: ED_ERR_INVALID (model or particle numbers), ED_ERR_OOM, ED_ERR_CUDA. */
int ed_sector_create(ed_ctx* ctx, const ed_model* model, int n_up, int n_dn,
                     int prec, unsigned flags, ed_sector** out);
int ed_sector_destroy(ed_sector* s);
int ed_sector_get_info(const ed_sector* s, ed_sector_info* out);
/* Copy one spin's basis strings (D_spin uint32, ascending) to host memory. */
int ed_sector_basis(const ed_sector* s, int spin, uint32_t* host_out);
/* Copy one spin's one-body hop table to host memory: for string rank r, entries
 * ptr[r] .. ptr[r+1]-1 give the rank tgt[k] of the string reached by moving one
 * electron along a bond with T_ij != 0 and the matrix element val[k] =
 * T_ij * (-1)^(occupied sites strictly between i and j), i.e. <r|H_1body|tgt>.
 * ptr has D_spin + 1 entries, tgt/val hops_spin entries (ed_sector_info).
 * Any output pointer may be NULL. */
int ed_sector_hops(const ed_sector* s, int spin, uint32_t* ptr, uint32_t* tgt, double* val);
/* Copy rows [row0, row0 + nrows) of the stored CSR (ED_SECTOR_CSR) to host
 * memory: row_ptr (nrows + 1 entries, relative to the first copied row), cols
 * and vals (row_ptr[nrows] entries each).  ED_ERR_INVALID without a CSR. */
int ed_sector_csr_rows(const ed_sector* s, uint64_t row0, uint64_t nrows,
                       uint64_t* row_ptr, uint32_t* cols, double* vals);

/* ------------------------------------------------------------------- apply */
/* y = H x inside the sector, matrix-free (elements formed on the fly, the first
 * improvement suggested at the end of Sec. 3.2).  x and y are device arrays of
 * `dim` elements in the sector's format; y is overwritten; x and y must not
 * overlap.  Stream-ordered, no synchronisation, no allocation. */
int ed_apply_h(ed_sector* s, const void* x, void* y, void* stream);
/* y = H x for n_vec vectors in HOST memory, end to end (the same matrix-free
 * product as ed_apply_h, Sec. 3.2): x_host and y_host hold n_vec vectors of
 * `dim` elements each in the sector's format, one after the other.  Every
 * vector crosses the host link once each way; the copies run on internal
 * streams, pipelined with the applies (the copy-in of vector i + 1 and the
 * copy-out of vector i - 1 overlap H*v of vector i).  Pinned host memory
 * (cudaHostAlloc, cudaHostRegister) gives the link's full rate; pageable memory
 * works at a lower one.  The work is ordered after what is already queued on
 * `stream`, and the call returns when y_host is complete (it synchronises
 * `stream`).  The first call on a sector allocates four device vectors
 * (against the context's budget) and three streams, kept until
 * ed_sector_destroy; calls on one sector must not overlap.  ED_ERR_INVALID for
 * NULL pointers, ED_ERR_OOM if the four vectors do not fit. */
int ed_apply_h_host(ed_sector* s, uint64_t n_vec, const void* x_host, void* y_host, void* stream);
/* y = H x from the stored CSR matrix (the Listing 1 product over Fig. 1's
 * arrays).  Needs ED_SECTOR_CSR and ED_PREC_FP64. */
int ed_apply_h_csr(ed_sector* s, const void* x, void* y, void* stream);

/* ---------------------------------------------------------- vector helpers */
/* Convert n elements between IEEE double and the sector-independent DF64 or
 * FP32 formats on the device (dst and src device arrays). */
int ed_convert(const void* src, int src_prec, void* dst, int dst_prec, uint64_t n, void* stream);
/* Dot product <x, y> of two device vectors of n elements in format `prec`,
 * accumulated in double; the result is written to host memory (synchronises). */
int ed_dot(ed_ctx* ctx, const void* x, const void* y, uint64_t n, int prec, double* result, void* stream);

/* Allocation-free dot product: the same <x, y> as ed_dot (accumulated in double
 * for FP64 vectors, in double-float for DF64 and FP32 vectors, the result
 * written to host memory after synchronising `stream`), for callers that cannot
 * allocate device memory: a host framework that owns every device allocation,
 * a process that must not grow its footprint in the middle of a solve, or code
 * that has no ed_ctx (creating one allocates).  The paper has no counterpart of
 * this call.  Its partial sums live in one fixed 512 KB __device__ array that
 * every GPU loading the library keeps until the process exits; n is limited to
 * 268,435,456 elements (65,536 tiles of 4,096) and a larger n is rejected with
 * ED_ERR_INVALID before any device work.  It calls no cudaMalloc or cudaFree.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  With CUDA's lazy module
 * loading (the default since CUDA
 * 12.2) that first look-up is also what loads the library module holding the
 * array onto the device, so the array's 512 KB become resident at the first
 * call, not when the library is loaded: a caller that will later hand all free
 * device memory to another framework should make one call (n = 1 is enough)
 * before doing so.  Later calls change the device's free memory by nothing.
 * All calls on a device share the one array and each call overwrites it, so
 * calls that overlap on the GPU (other streams or threads) race and must be
 * serialised by the caller. */
int ed_dot_noalloc(const void* x, const void* y, uint64_t n, int prec, double* result, void* stream);

/* ----------------------------------------------------------------- Lanczos */
typedef struct ed_lanczos_opts {
  int k;               /* number of lowest eigenpairs wanted (1..ED_MAX_K) */
  double tol;          /* converged when beta_{j+1} |s_{j,i}| <= tol * max(1, |theta_i|) */
  int max_iter;        /* Lanczos steps at most (the basis holds max_iter + 1 vectors) */
  int check_every;     /* steps between tridiagonal solves (>= 1) */
  uint64_t seed;       /* start vector seed when v0 == NULL */
  const void* v0;      /* optional device start vector (sector format), NULL = seeded */
  int reorth;          /* 1: full CGS2 reorthogonalisation against every basis vector */
} ed_lanczos_opts;

typedef struct ed_lanczos_info {
  int iters;                    /* Lanczos steps taken */
  int n_converged;              /* leading eigenvalues meeting tol */
  double residual[ED_MAX_K];    /* Ritz residual estimates beta |s| */
  double apply_ms;              /* device time in H*v (CUDA events) */
  double total_ms;              /* wall time of the call */
} ed_lanczos_info;

/* Lowest k eigenvalues (host, ascending) and, if evecs != NULL, the Ritz vectors
 * (device, k consecutive vectors of dim elements in the sector's format) of H in
 * the sector, by Lanczos with full reorthogonalisation (Sec. 3: iterative
 * solvers built on repeated H*v).  Allocates its Krylov basis from the context
 * budget for the duration of the call.  Returns ED_ERR_NOT_CONVERGED (with the
 * current estimates filled in) when max_iter is reached.  Synchronises. */
int ed_lanczos(ed_sector* s, const ed_lanczos_opts* opts, double* evals,
               void* evecs, ed_lanczos_info* info, void* stream);

/* -------------------------------------------------------------- autotuner */
#define ED_MAX_TUNE 16

typedef struct ed_tune_result {
  int n_candidates;               /* variants tried, in the order of the arrays */
  int chosen;                     /* index of the fastest, now the sector's H*v; -1: nothing to choose */
  int kernel[ED_MAX_TUNE];        /* 2: one up string per block, 3: two up strings per block,
                                     4: natural-order kernel, four or two (float) / two or one
                                     (double-float) up strings per block */
  int block[ED_MAX_TUNE];         /* threads per block */
  int min_blocks[ED_MAX_TUNE];    /* blocks per SM the register budget is sized for */
  double ms[ED_MAX_TUNE];         /* median device time of one H*v; -1 where it does not apply or fit */
} ed_tune_result;

/* Autotuner of the matrix-free H*v (the hot loop of Sec. 3's iterative
 * solvers; the paper has no tuner): times every variant of the fast row
 * kernels that applies to this sector -- one, two or four up strings per block,
 * times the launch shapes (threads per block, blocks per SM) -- `reps` times each
 * (median, CUDA events, after a warm-up) on internal random vectors, makes the
 * fastest the sector's H*v, and records it in the context's cache under the
 * sector's shape (format, sizes, hop counts), so that sectors of the same shape
 * created later start with it.  The variants of one kernel compute the same y
 * bit for bit; for double-float vectors the kernels (kernel ids 2, 3, 4) sum in
 * different orders and agree to rounding; float sectors that have the
 * natural-order kernel are tuned among its variants only.
 * Sectors without the fast kernel (ED_SECTOR_GENERIC, very short rows) have
 * nothing to tune: n_candidates = 0, chosen = -1.  Allocates two vectors for
 * the duration of the call.  Synchronises. */
int ed_sector_autotune(ed_sector* s, int reps, ed_tune_result* out, void* stream);

/* Choose the H*v variant by index (as in ed_tune_result), or -1 for the
 * untuned default.  ED_ERR_INVALID if the variant does not apply.
 * ed_sector_get_variant reports the variant in use (-1: the untuned default,
 * also for sectors without the fast kernel). */
int ed_sector_set_variant(ed_sector* s, int variant);
int ed_sector_get_variant(const ed_sector* s, int* variant);

/* Save the context's autotune cache as JSON (format "libedgb-autotune-1",
 * with the GPU's name), or merge a saved one into it; entries saved on another
 * GPU model are skipped (n_loaded counts the entries taken).  ED_ERR_INVALID
 * for unreadable or malformed files. */
int ed_tune_cache_save(ed_ctx* ctx, const char* path);
int ed_tune_cache_load(ed_ctx* ctx, const char* path, int* n_loaded);

/* ------------------------------------------------ thick-restart Lanczos */
#define ED_MAX_BASIS 128

typedef struct ed_trlan_opts {
  int k;               /* lowest eigenpairs wanted (1..ED_MAX_K) */
  double tol;          /* converged when beta |y_last,i| <= tol * max(1, |theta_i|) */
  int max_basis;       /* basis size m before a restart: k + 2 <= m <= ED_MAX_BASIS (or >= dim) */
  int keep;            /* Ritz vectors kept at a restart, k..m-2; 0 chooses (m + k) / 2 */
  int max_iter;        /* H*v products at most, over all restarts */
  int check_every;     /* steps between projected eigen-solves (>= 1); a full basis always checks */
  uint64_t seed;       /* start vector seed when v0 == NULL */
  const void* v0;      /* optional device start vector (sector format), NULL = seeded */
} ed_trlan_opts;

typedef struct ed_trlan_info {
  int iters;                    /* H*v products */
  int restarts;                 /* thick restarts */
  int n_converged;              /* leading eigenvalues meeting tol */
  double residual[ED_MAX_K];    /* Ritz residual estimates */
  double apply_ms;              /* device time in H*v (CUDA events) */
  double total_ms;              /* wall time of the call */
  size_t basis_bytes;           /* device bytes of basis, work vector and rotation target
                                   (max_basis + 2 + keep slots of dim elements, each slot padded
                                   to a multiple of 32 elements) */
} ed_trlan_info;

/* Lowest k eigenvalues (host, ascending; NaN past the sector dimension) and,
 * if evecs != NULL, the Ritz vectors (device, k consecutive vectors of dim
 * elements in the sector's format) by thick-restart Lanczos with full CGS2
 * reorthogonalisation.  The paper's solver is implicitly restarted Arnoldi
 * (abstract, Sec. 3); for symmetric H a restart with the unwanted Ritz values
 * as exact shifts keeps the span of the wanted Ritz vectors plus the residual
 * direction, which is what this keeps explicitly, so the device memory is
 * bounded by (max_basis + 2 + keep) vectors however many steps convergence
 * takes.  The projected eigenproblem runs on the device (one-block Jacobi).
 * An exhausted Krylov space with fewer than k values continues from a seeded
 * direction orthogonal to the basis (degenerate multiplets).  Returns
 * ED_ERR_NOT_CONVERGED with the current estimates after max_iter products;
 * ED_ERR_INVALID for arguments outside the ranges above; ED_ERR_OOM when the
 * basis does not fit the context budget.  Synchronises. */
int ed_lanczos_tr(ed_sector* s, const ed_trlan_opts* opts, double* evals, void* evecs,
                  ed_trlan_info* info, void* stream);

/* ------------------------------------------------------- Green's function */
typedef struct ed_state {
  int n_up, n_dn;     /* sector of the state */
  double E;           /* its energy */
  const void* vec;    /* device, dim elements of that sector in format `prec` */
} ed_state;

/* G(i w_n), w_n = (2n+1) pi / beta, n < n_w, of orbital `orbital` and spin
 * `spin` (Eq. 3 with the standard sign, Im G < 0), from the given states by
 * Lanczos continued fractions of depth `depth` in the N+1 and N-1 sectors.
 * Z is taken over the states passed; states with e^{-beta (E - E_min)} below
 * boltz_cut are skipped (Sec. 4 keeps about 20 states with a 1e-5 cutoff).
 * G is host memory, 2*n_w doubles (re, im interleaved).  If coeffs != NULL it
 * receives, per kept state and part (particle, then hole), 2 + 2*depth doubles:
 * [n2, L, a_0..a_{depth-1}, b_0..b_{depth-1}] (b_0 = 0; L = steps taken).
 * Builds the neighbour sectors itself.  Synchronises. */
int ed_greens_cf(ed_ctx* ctx, const ed_model* model, int prec, int n_states,
                 const ed_state* states, double beta, int n_w, int orbital, int spin,
                 int depth, double boltz_cut, double* G, double* coeffs, void* stream);

/* The same Green's function at n_z arbitrary complex frequencies z (host,
 * 2*n_z doubles, re/im interleaved, every Im z > 0; ED_ERR_INVALID otherwise):
 * G(z) = sum_nu w_nu [n+ / (z + E_nu - a_0 - ...) + n- / (z - E_nu + a_0 - ...)].
 * With z = w + i eta it gives the real-frequency spectral function
 * A(w) = -Im G(w + i eta) / pi that Figs. 3 and 5 plot; with z = i w_n it equals
 * ed_greens_cf.  beta still sets the Boltzmann weights of the states.  G: host,
 * 2*n_z doubles; coeffs and all other arguments as ed_greens_cf.  Synchronises. */
int ed_greens_cf_z(ed_ctx* ctx, const ed_model* model, int prec, int n_states,
                   const ed_state* states, double beta, int n_z, const double* z, int orbital,
                   int spin, int depth, double boltz_cut, double* G, double* coeffs, void* stream);

/* ------------------------------------------------- DMFT self-consistency */
/* One DMFT self-consistency update for the one-band Hubbard model (Sec. 2: the
 * lattice problem is mapped onto the Anderson impurity of Eq. 2; Sec. 3.2 runs
 * it on the square lattice).  Inputs (host): the impurity G(i w_n), n < n_w,
 * w_n = (2n+1) pi / beta (2*n_w doubles, re/im interleaved; e.g. from
 * ed_greens_cf) of the AIM with impurity level eps_d and bath eps_in, V_in
 * (n_bath each); the chemical potential mu; a quadrature of the lattice band,
 * energies e and weights w (n_e each, weights summing to 1).  Computes on the
 * device, at z = i w_n,
 *   Delta     = sum_k V_k^2 / (z - eps_k),
 *   Sigma     = z - eps_d - Delta - 1 / G_imp,
 *   G_loc     = sum_j w_j / (z + mu - e_j - Sigma),
 *   Delta_new = z - eps_d - Sigma - 1 / G_loc,
 * and fits the new bath eps_out, V_out (V >= 0) to Delta_new on the first n_fit
 * frequencies by Levenberg-Marquardt started from eps_in, V_in, minimising
 * chi2 = (1/n_fit) sum_n |Delta_new - sum_k V_k^2 / (z - eps_k)|^2.  Optional
 * outputs (host, 2*n_w doubles each, NULL to skip): Sigma, G_loc, Delta_new.
 * ED_ERR_INVALID for sizes out of range (1 <= n_bath <= ED_MAX_SITES,
 * 1 <= n_fit <= n_w, n_e >= 1) or a zero or non-finite G_imp.  Synchronises. */
int ed_dmft_update(ed_ctx* ctx, int n_w, double beta, const double* G_imp, double eps_d, double mu,
                   int n_bath, const double* eps_in, const double* V_in, int n_e, const double* e,
                   const double* w, int n_fit, double* eps_out, double* V_out, double* chi2,
                   double* sigma, double* G_loc, double* delta_new, void* stream);

/* ------------------------------------------------------- batched sectors */
typedef struct ed_batch ed_batch;

typedef struct ed_batch_info {
  int steps;           /* Lanczos steps taken (the last sector to converge) */
  int graph_replays;   /* replays of the one-step CUDA graph */
  int n_sectors;
  double total_ms;     /* wall time of the call */
} ed_batch_info;

/* Build n_sectors sectors (n_up[i], n_dn[i]) of one model for batched solves:
 * all of a model's sectors (the Lehmann sum of Eq. 3 runs over every sector) or
 * many small problems at once.  Tables live on the device; vectors are
 * allocated per ed_batch_lanczos call.  Errors as ed_sector_create. */
int ed_batch_create(ed_ctx* ctx, const ed_model* model, int n_sectors, const int* n_up, const int* n_dn,
                    int prec, ed_batch** out);
int ed_batch_destroy(ed_batch* b);
/* Lowest k (<= 16) eigenvalues of every sector of the batch by Lanczos with full
 * CGS2 reorthogonalisation (opts->reorth must be 1; v0 is ignored; seed seeds
 * every sector's start vector).  All active sectors advance together: each
 * step is one replay of a CUDA graph whose kernels (one H*v over all sectors,
 * dot products, update, CGS2, norm, scaling) each run as a single launch over a
 * device work list of (sector, chunk of elements) items; converged sectors
 * drop out of the list.  evals: host, n_sectors * k (NaN past a sector's
 * dimension); iters: host, n_sectors (may be NULL).  Synchronises. */
int ed_batch_lanczos(ed_batch* b, const ed_lanczos_opts* opts, double* evals, int* iters,
                     ed_batch_info* info, void* stream);

/* Sector packing of the batch: every sector is cut into work items of `chunk`
 * consecutive elements (by default the largest power of two from 256 to 8192
 * that gives at least eight items per SM), and each batched kernel runs one
 * launch over the item list.  ed_batch_set_chunk sets it (a power of two in
 * 64..65536; ED_ERR_INVALID otherwise).  ed_batch_autotune runs `steps`
 * graph-replayed Lanczos steps (2..64) of every sector with each candidate
 * chunk (256 .. 32768), keeps the fastest per step and reports all of them;
 * results do not depend on the chunk beyond the order of floating-point sums.
 * Synchronises. */
typedef struct ed_batch_tune_result {
  int n_candidates;
  int chosen;                       /* index of the chunk now in use */
  int chunk[ED_MAX_TUNE];
  double ms_per_step[ED_MAX_TUNE];  /* wall time per Lanczos step of the whole batch */
} ed_batch_tune_result;
int ed_batch_set_chunk(ed_batch* b, int chunk);
int ed_batch_autotune(ed_batch* b, int steps, ed_batch_tune_result* out, void* stream);

/* ---------------------------------------------------------------- serving */
/* A request server for impurity solves, the work of one DMFT iteration (Sec. 2:
 * each iteration diagonalises a new impurity Hamiltonian and forms G(i w_n) of
 * Eq. 3; Sec. 4 keeps the lowest states above a Boltzmann cutoff).  A server
 * thread admits queued requests while their estimated device footprint fits
 * the budget and a slot is free; admitted requests run concurrently, each on
 * its own stream with its own scratch (continuous batching: requests join and
 * leave as others finish, their kernels overlap on the GPU).
 *  k = 1: ground state by three-vector Lanczos, advanced a few steps per server
 *         pass (replays of captured step graphs), its Ritz vector, then (want_G)
 *         the particle and hole continued fractions of c+_{orbital,spin} at
 *         depth cf_depth and G on n_w Matsubara points at beta.
 *  k > 1: the k lowest states of the sector by thick-restart Lanczos (basis of
 *         max(4k + 8, 20) vectors, at most 64), run by a worker thread of the
 *         server, then (want_G) G from those states with Boltzmann weights at
 *         beta (states below a weight of 1e-5 relative to the lowest skipped),
 *         as ed_greens_cf.
 *  packs: requests whose sector has at most pack_dim states (small sectors,
 *         whose single solves are bound by launch latency) are not run one by
 *         one: the server takes every queued such request with the same k
 *         (up to 64) and solves their sectors together, each Lanczos step one
 *         replay of a CUDA graph whose kernels are single launches over all
 *         their sectors (full CGS2 reorthogonalisation, at most 400 steps,
 *         Ritz vectors from the stored basis), then forms each request's G
 *         from its k states as above.  Packed requests do not take slots of
 *         max_active; one pack runs at a time, on a worker thread.
 * A request's kernels touch only its own buffers (and, in a pack, its own
 * work items), so its result is bitwise the same alone or in a mix.  The
 * server's context must not be used from other threads while the server
 * runs. */
#define ED_SERVE_MAX_K 16
typedef struct ed_server ed_server;

typedef struct ed_server_opts {
  size_t hbm_budget;   /* device bytes the admitted requests may hold together (0 = no limit) */
  int max_active;      /* requests on the GPU at once */
  int prec;            /* vector format of every request */
  double tol;          /* residual tolerance of the eigensolve (relative, as ed_lanczos) */
  int max_iter;        /* Lanczos steps (k = 1) or H*v products (k > 1, thick restart) at most */
  int cf_depth;        /* continued-fraction depth (1..1000) */
  int n_w;             /* Matsubara frequencies */
  double beta;         /* inverse temperature */
  uint64_t seed;       /* start-vector seed */
  uint64_t pack_dim;   /* requests whose sector has at most this many states are solved in packs
                          (0: never); see below */
} ed_server_opts;

typedef struct ed_request {
  const ed_model* model;  /* copied at submission */
  int n_up, n_dn;         /* sector of the states */
  int want_G;             /* also compute G(i w_n) */
  int orbital, spin;      /* operator c+ of the Green's function */
  int k;                  /* lowest states wanted, 1..ED_SERVE_MAX_K (0 means 1) */
} ed_request;

typedef struct ed_result {
  int status;          /* ED_OK, ED_ERR_NOT_CONVERGED or the failure */
  double E0;           /* ground energy of the sector */
  int iters;           /* Lanczos steps (H*v products) of the eigensolve */
  double latency_ms;   /* submission to completion */
  double queue_ms;     /* submission to admission */
  int n_w;             /* G entries written (0 without want_G) */
  int n_E;             /* energies in E (k, or the sector dimension if smaller) */
  double E[ED_SERVE_MAX_K];  /* lowest energies, ascending */
} ed_result;

typedef struct ed_server_stats {
  int queued;               /* submitted, not yet admitted (the queue depth) */
  int active;               /* admitted, not yet finished */
  int done, failed;         /* finished with ED_OK / with an error */
  int max_active_seen;
  size_t bytes_in_flight;   /* estimated footprint of the admitted requests */
  /* Over every finished request (done or failed, polled or not): the number
   * of them, and the 50th / 99th percentiles of submission-to-completion
   * (latency) and submission-to-admission (queue) times in ms, interpolated
   * linearly between order statistics; 0 before the first one finishes. */
  int n_latency;
  double latency_p50_ms, latency_p99_ms;
  double queue_p50_ms, queue_p99_ms;
} ed_server_stats;

/* Start a server on the context's device.  ED_ERR_INVALID on bad options. */
int ed_server_create(ed_ctx* ctx, const ed_server_opts* opts, ed_server** out);
/* Stop the thread and free everything (unpolled results are dropped). */
int ed_server_destroy(ed_server* s);
/* Queue a request; never blocks on the GPU.  ED_ERR_OOM if the request alone
 * exceeds the whole budget, ED_ERR_INVALID for a bad model, sector or k. */
int ed_submit(ed_server* s, const ed_request* req, uint64_t* ticket);
/* Non-blocking: *done = 1 and the result (and G, 2*n_w doubles re/im, if
 * non-NULL) once the request has finished; the ticket is then released.
 * ED_ERR_INVALID for an unknown or already collected ticket. */
int ed_poll(ed_server* s, uint64_t ticket, ed_result* res, double* G, int* done);
int ed_server_get_stats(ed_server* s, ed_server_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* ED_H */

/*
 * fsmlmc.h - C ABI of the GB300 (sm_103a) Frequency-Splitting MLMC trace library.
 *
 * Computes the stochastic traces of arXiv:2212.04430 (Whyte, Stathopoulos,
 * Romero, Orginos, "Optimizing Shift Selection in Multilevel Monte Carlo for
 * Disconnected Diagrams in Lattice QCD"): the shifted Wilson-Dirac solves
 * (D + sigma I) x = z of Eq. (shifted_linear_systems) for Z4 noise z, the
 * Gamma Omega_p insertion of Sec. 1, the level traces of Eq. (fs_trace_est) with
 * the practical variance of Eq. (practical_variance), and the variance sampling
 * algorithm of Sec. 3.1.
 *
 * Conventions
 *   Lattice   dims = {Lx, Ly, Lz, Lt}, all even, >= 2; V = Lx Ly Lz Lt.
 *             site = x + Lx (y + Ly (z + Lz t)).
 *   Operator  Wilson, r = 1, DeGrand-Rossi gamma basis (gamma_5 = diag(1,1,-1,-1)):
 *             (D psi)(x) = (4 + m) psi(x) - 1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x + mu)
 *                                         + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)],
 *             mu = 0..3 is x, y, z, t; the t-hop across the boundary is multiplied by bc_t.
 *   Omega_p   (Omega_p psi)(x) = U_z(x) U_z(x + z) ... U_z(x + (p-1) z) psi(x + p z)   (Sec. 1)
 *   Noise     z(x, s, c) = i^k, k = (Philox4x32-10(ctr = {x, sample, level, job},
 *             key = {seed mod 2^32, seed >> 32}).word0 >> 2(3 s + c)) & 3.
 *   Host layouts (double, interleaved re/im):
 *             spinor  [V][4 spin][3 colour][2]      gauge  [4 mu][V][3][3][2], U_mu(x): x -> x + mu
 *             Gamma   [4][4][2] (row major, complex)
 *
 * Ownership and threading
 *   The caller owns every pointer it passes; the library copies what it needs and
 *   never keeps a caller pointer past the call. Device state (gauge copies, solver
 *   workspaces) belongs to the fs_ctx and is freed by fs_ctx_destroy. A context is
 *   used by one host thread at a time. Work is issued on the context's stream
 *   (fs_set_stream, default: a stream the context creates); calls return after the
 *   results they write are complete.
 *
 * Errors
 *   Every int-returning call returns FS_OK (0) or one of the FS_ERR_* codes below;
 *   fs_last_error(ctx) gives a message for the last failure on that context.
 */
#ifndef FSMLMC_H
#define FSMLMC_H

#include <stddef.h>
#include <stdint.h>

/* Only the functions declared here are exported from the shared library. */
#if defined(__GNUC__)
#define FS_API __attribute__((visibility("default")))
#else
#define FS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum fs_status {
  FS_OK = 0,
  FS_ERR_ARG = 1,      /* invalid argument (null pointer, bad size, odd dimension, ...)   */
  FS_ERR_INPUT = 2,    /* non-finite value in an input array                              */
  FS_ERR_OOM = 3,      /* device allocation failed                                        */
  FS_ERR_BUDGET = 4,   /* request exceeds the memory budget                               */
  FS_ERR_NOCONV = 5,   /* a system hit max_iter; outputs are written, see fs_sys_stats     */
  FS_ERR_TIMEOUT = 6,  /* a bounded wait expired                                          */
  FS_ERR_CUDA = 7,     /* CUDA runtime error                                              */
  FS_ERR_STATE = 8     /* call not valid in the context's state (e.g. no gauge field yet) */
};

/* Storage precision of the Krylov vectors. F64: FP64 storage and arithmetic.
 * F32 / F16 / BF16: that storage with FP32 arithmetic, FP64 reductions and FP64
 * reliable updates (true residual recomputed in FP64). */
enum fs_prec { FS_PREC_F64 = 0, FS_PREC_F32 = 1, FS_PREC_F16 = 2, FS_PREC_BF16 = 3 };

/* Level estimators (all unbiased for the same level trace):
 *   FS_EST_DIFF        z^dag Gamma Omega_p [(D+s_l)^-1 - (D+s_{l+1})^-1] z, Eq. (tele_sum)
 *   FS_EST_SPLIT_EVEN  (s_{l+1}-s_l) [(D+s_l)^-dag z]^dag Gamma Omega_p (D+s_{l+1})^-1 z,
 *                      Eq. (fs_trace_est); the adjoint solve uses gamma_5 z
 *   FS_EST_PRODUCT     (s_{l+1}-s_l) z^dag Gamma Omega_p (D+s_l)^-1 (D+s_{l+1})^-1 z,
 *                      Eq. (tele_sum_prod_disp0), two nested solves
 * The last level is z^dag Gamma Omega_p (D+s_L)^-1 z for all three. Each costs two solves
 * per sample below the last level, at the same two shifts for DIFF and SPLIT_EVEN. Measured on
 * the 16^3x32 job with the same noise (64 vectors per level), SPLIT_EVEN has the smallest
 * multilevel cost (sum_l sqrt(V_l C_l))^2, 16% below DIFF (its V_0 and V_1 are about half of
 * DIFF's) and 19% below PRODUCT: it is the recommended choice (the Python binding's default).
 * The value 0 stays DIFF, so a zero-initialised fs_mlmc_params keeps the difference form. */
enum fs_estimator { FS_EST_DIFF = 0, FS_EST_SPLIT_EVEN = 1, FS_EST_PRODUCT = 2 };

/* Per-system solver status (fs_sys_stats.status). */
enum fs_sys_status { FS_SYS_CONVERGED = 2, FS_SYS_NOCONV = 3 };

typedef struct fs_ctx fs_ctx;

typedef struct fs_solve_params {
  double tol;          /* stop when ||z - (D+sigma) x|| <= tol ||z||  (FP64 true residual)   */
  int max_iter;        /* BiCGStab iterations per system before FS_SYS_NOCONV                */
  int prec;            /* enum fs_prec                                                       */
  int rhs_tile;        /* systems solved together in one batch (1..64); 0 = library choice  */
  int link_compress;   /* 18: full links; 12: two rows stored, third reconstructed          */
  double delta;        /* reliable update when the sloppy residual drops by this factor;
                          0 = library choice                                                 */
  int verify;          /* 1: recompute the full-lattice FP64 residual of every solution      */
  int fallback_iter;   /* a system BiCGStab leaves unconverged (breakdowns past the restart
                          limit, or max_iter) is re-solved by FP64 CGNR on the normal equations
                          M^dag M x = M^dag b, M^dag = gamma5 M gamma5, for at most this many
                          iterations; 0 = 4 * max_iter, < 0 = no fallback                     */
  int lanes;           /* mlmc_level_trace only: tiles solved at the same time, each on a stream
                          and host thread of its own (1..4); 0 = library choice: as many tiles
                          as the job fills, at most 3. A system's result does not depend on its
                          lane. Every lane holds a tile of device memory; a lane whose tile does
                          not fit is dropped and its share goes to the others. */
} fs_solve_params;

typedef struct fs_sys_stats {
  int iters;           /* BiCGStab iterations                                                */
  int status;          /* enum fs_sys_status                                                 */
  int reliable_updates;
  int restarts;
  double true_resid;   /* ||z - (D+sigma) x|| / ||z|| in FP64                                 */
  int fallback_iters;  /* CGNR fallback iterations (0: BiCGStab alone)                        */
  int pad;
} fs_sys_stats;

typedef struct fs_mlmc_params {
  double m;                 /* bare mass                                                   */
  int nlev;                 /* number of shifts = L + 1                                    */
  int p;                    /* z-displacement of Omega_p, 0 <= p < Lz                      */
  const double* sigma;      /* [nlev] shifts, sigma_0 < ... < sigma_L, Eq. (tele_sum)       */
  const int* n_samples;     /* [nlev] N_l noise vectors per level                           */
  const double* gamma;      /* Gamma, 4x4 complex [4][4][2]                                 */
  uint64_t seed;            /* Philox key                                                   */
  uint32_t job;             /* Philox counter word 3                                        */
  int estimator;            /* enum fs_estimator                                            */
  fs_solve_params solve;
  /* Probing and dilution of the noise (Sec. 2.1, Eq. (probing_vectors); Sec. 3.1). A sample
     is then the sum of the level estimator over its pieces: the sample's Z4 vector restricted
     to the sites of one probing colour j < ncolors and, with dilute = 1, to one spin-colour
     index a = 3 s + c < 12; pieces are listed colour-major. */
  const int32_t* colors;    /* [V] probing colour of every site (canonical order), values in
                               [0, ncolors) with every colour used; NULL = no probing          */
  int ncolors;              /* number of colours when colors != NULL                         */
  int dilute;               /* 1: full spin-colour dilution (12 pieces per colour); 0: none  */
  /* Hopping parameter expansion of the last level (Sec. 3.1, the remark after
     Eq. (sampled_single)), applied when m + sigma_L > 0: with D + s = A (1 - kappa H),
     A = 4 + m + s, kappa = 1 / (2A), the last level's samples become
       T_exact + z^dag Gamma Omega_p (kappa H)^K (D + sigma_L)^-1 z,
       T_exact = sum_{k<K} Tr(Gamma Omega_p (kappa H)^k) / A,
     T_exact computed exactly from displacement-p distance-(K-1) probing vectors with full
     spin-colour dilution (12 c FP64 vectors, K - 1 kappa H applications each). Same
     expectation, lower variance. 0 = off; K in 1..8 (the paper uses 4); needs p < Lz
     (FS_ERR_ARG otherwise). */
  int hpe_order;
} fs_mlmc_params;

/* ---- context ------------------------------------------------------------------ */

/* Create a context for a lattice on CUDA device `device`. bc_t = -1 (antiperiodic in t)
 * or +1 (periodic). FS_ERR_ARG for odd or non-positive dims or V >= 2^31 / 24. */
FS_API int fs_ctx_create(fs_ctx** ctx, const int dims[4], int bc_t, int device);
FS_API void fs_ctx_destroy(fs_ctx* ctx);
/* Message of the last error on ctx ("" if none); valid until the next call on ctx. */
FS_API const char* fs_last_error(const fs_ctx* ctx);
/* Issue all work of ctx on `stream` (a cudaStream_t; NULL restores the context's own). */
FS_API int fs_set_stream(fs_ctx* ctx, void* stream);
/* Device memory currently held by ctx, in bytes. */
FS_API size_t fs_ctx_device_bytes(const fs_ctx* ctx);

/* The tile size the autotuner chose for storage precision `prec` and `link_compress` on this
   context, or 0 if it has not run. A library addition (the paper has no counterpart): when a
   call leaves fs_solve_params.rhs_tile = 0 and has at least 16 systems, the first such call
   per precision and link format times a BiCGStab iteration per system on tiles of 8, 16, 32
   and 64 systems (at most the call's system count) and keeps the fastest for the context. */
FS_API int fs_tuned_tile(const fs_ctx* ctx, int prec, int link_compress);
/* The whole tuned shape: the tile as above and, for tiles of 32-system chunks in the inner
   precisions (the persistent hop kernel), the ring depth and resident blocks per SM the same trial
   chose among {default, 3} x {as many as fit, 2} (0 = the default); all 0 if it has not run. The
   shape never changes a result: every system is computed the same way in every launch shape. */
FS_API int fs_tuned_shape(const fs_ctx* ctx, int prec, int link_compress, int* tile, int* ring_depth,
                          int* blocks_per_sm);

/* Upload the gauge field U (host, [4][V][3][3][2] doubles). Builds the FP64 copy used
 * for true residuals and contractions and the lower-precision copies on demand.
 * FS_ERR_INPUT if U holds a non-finite value. */
FS_API int fs_set_gauge(fs_ctx* ctx, const double* U);

/* The Wilson-clover operator (Sec. 4 computes with the clover discretisation): with c_sw != 0
 * every operation of ctx below (wilson_dslash, the solves, the trace estimators) applies
 *   D_sw + sigma I = D + sigma I + C,   C(x) = (c_sw / 2) sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x),
 * sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag) / (8i), Q_{mu nu}(x)
 * the sum of the four counter-clockwise plaquettes of the (mu, nu) plane at x (the paper states no
 * normalisation: this is the reading). C is Hermitian, commutes with gamma_5 and is eigen-
 * decomposed once per gauge field into a table of two complex 6x6 blocks per site (about 2.7 KB
 * per site in FP64 + FP32), so that (A + C)^-1 for every shift costs two 6x6 products per chirality.
 * The table is built now if a gauge field is set, else by the next fs_set_gauge, and rebuilt by
 * every fs_set_gauge; c_sw = 0 frees it and restores the Wilson operator. With the clover term
 * the CGNR fallback runs on the clover M-hat (still M-hat^dag = gamma_5 M-hat gamma_5), the
 * hopping parameter expansion (hpe_order, fs_hpe_exact_trace) is
 * the generalised one of Sec. 3.1, D_sw + sigma = A(x) (1 - K), K = A(x)^-1 H / 2 with
 * A(x) = 4 + m + sigma + C(x): T_exact = sum_{k<K} Tr(Gamma Omega_p K^k A^-1) and the remainder
 * z^dag Gamma Omega_p K^K (D_sw + sigma)^-1 z, and wilson_dslash_noalloc stays the Wilson
 * operator. FS_ERR_INPUT for a non-finite c_sw, FS_ERR_STATE on a lane, 3 when the table does
 * not fit. */
FS_API int fs_set_clover(fs_ctx* ctx, double c_sw);

/* ---- the operations of the paper -------------------------------------------------- */

/* out_k = (D + sigma I) in_k for k < nrhs, full lattice (the operator of
 * Eq. (shifted_linear_systems); D_sw + sigma I with the clover term, fs_set_clover). in/out: host
 * [nrhs][V][4][3][2]. prec selects the storage precision of the device vectors (F64 computes in
 * FP64, others in FP32). */
FS_API int wilson_dslash(fs_ctx* ctx, double m, double sigma, const double* in, double* out, int nrhs,
                  int prec, int link_compress);

/* Solve (D + sigma_j I) x_{j,k} = b_k, Eq. (shifted_linear_systems), for every shift j < nshift
 * and right-hand side k < nrhs, with even-odd preconditioned BiCGStab batched over systems.
 * b: host [nrhs][V][24]; x: host [nshift][nrhs][V][24]; stats (optional): [nshift][nrhs].
 * Returns FS_ERR_NOCONV if any system stopped at max_iter (x and stats still written). */
FS_API int shifted_solve(fs_ctx* ctx, double m, const double* sigma, int nshift, const double* b, int nrhs,
                  double* x, const fs_solve_params* params, fs_sys_stats* stats);

/* shifted_solve on caller-owned device arrays (e.g. torch tensors): b device [nrhs][V][24],
 * x device [nshift][nrhs][V][24] (canonical layout, FP64), both on the context's GPU and
 * 16-byte aligned (FS_ERR_ARG otherwise); sigma and stats stay on the host. The work runs on
 * the context's stream (fs_set_stream) and the call returns when x is written. b is read in
 * place and not checked for non-finite values (they surface as FS_ERR_NOCONV). Same arithmetic
 * as shifted_solve: the solutions are identical. */
FS_API int shifted_solve_dev(fs_ctx* ctx, double m, const double* sigma, int nshift, const double* b, int nrhs,
                      double* x, const fs_solve_params* params, fs_sys_stats* stats);

/* FS-MLMC trace estimate, Eq. (fs_trace_est): for every level l < nlev, N_l Z4 noise
 * vectors z_{s,l} (Philox counter {site, s, l, job}) give samples c_{s,l} of the chosen
 * estimator. Outputs (host, caller-owned):
 *   trace   [nlev][2]   T_l = (1/N_l) sum_s c_{s,l}
 *   var     [nlev]      V_l = (1/N_l) sum_s |c_{s,l}|^2 - |T_l|^2   (Eq. (practical_variance))
 *   samples [sum N_l][2] (optional) every c_{s,l}, level-major
 *   stats   [number of solves] (optional), in the order the solves are listed in
 *           fs_mlmc_num_solves' documentation.
 * The total trace is sum_l T_l and V_FS = sum_l V_l / N_l (Eq. (total_var)). */
FS_API int mlmc_level_trace(fs_ctx* ctx, const fs_mlmc_params* params, double* trace, double* var,
                     double* samples, fs_sys_stats* stats);

/* mlmc_level_trace for several displacements at once: the traces for p[0..np) (distinct, each
 * 0..30, np <= 16; params->p is ignored) from the same solves, as the paper uses one set of
 * inversions for all displacements (Sec. 4); the contraction forms them in one pass. Outputs in
 * the order of p: trace [np][nlev][2], var [np][nlev], samples (optional) [np][sum N_l][2];
 * stats as mlmc_level_trace. With hpe_order every p needs p < Lz and gets its own exact part. */
FS_API int mlmc_level_traces(fs_ctx* ctx, const fs_mlmc_params* params, const int* p, int np, double* trace,
                      double* var, double* samples, fs_sys_stats* stats);

/* Number of shifted solves mlmc_level_trace performs: per level l < L two solves per
 * sample and piece (DIFF: z at s_l then z at s_{l+1}; SPLIT_EVEN: gamma_5 z at s_l then z at
 * s_{l+1}; PRODUCT: z at s_{l+1} then its solution at s_l), one per sample and piece at level
 * L; a sample has ncolors * (dilute ? 12 : 1) pieces when probing (1 without), so the count
 * is the paper's 12 c m N_s for one shift and full dilution. Solves are listed level-major,
 * then by sample, then by piece. -1 if the count exceeds 2^31 - 1 or params is invalid. */
FS_API int fs_mlmc_num_solves(const fs_mlmc_params* params);

/* Exact low orders of the hopping parameter expansion (Sec. 3.1, the remark after
 * Eq. (sampled_single)): out = {re, im} of T = sum_{k<K} Tr(Gamma Omega_p (kappa H)^k) / A,
 * A = 4 + m + sigma, kappa = 1 / (2A), H the hopping term of D (D + sigma = A (1 - kappa H)).
 * Computed with displacement-p distance-(K-1) probing colours (fs_probing_colors) and full
 * spin-colour dilution: 12 c FP64 vectors (pieces of a Z4 vector from `seed`; the result does not
 * depend on it), K - 1 kappa H applications each, one contraction per order. The value
 * mlmc_level_trace adds to every last-level sample with hpe_order = K. params: rhs_tile (0 = 64
 * pieces at a time); the other fields are unused. K in 1..8, 0 <= p < Lz, else FS_ERR_ARG.
 * With the clover term (fs_set_clover) the generalised expansion: T = sum_{k<K} Tr(Gamma Omega_p
 * K^k A^-1), K = A(x)^-1 H / 2, A(x) = A + C(x), every order (order 0 included) from the pieces,
 * with distance-max(K-1, 1) colours. */
FS_API int fs_hpe_exact_trace(fs_ctx* ctx, double m, double sigma, const double* gamma, int p, int K, uint64_t seed,
                       const fs_solve_params* params, double* out);

/* Greedy probing colours (Sec. 2.1): a distance-k colouring of the lattice graph of D (the
 * nearest-neighbour graph of the periodic 4D lattice, hop distance), or, for p > 0, the
 * displacement-p colouring of the symmetric part of Pi_p D^k, in which site x differs in colour
 * from every site within distance k of x + p z and of x - p z (z = lattice axis 2, the axis of
 * Omega_p). Sites are coloured in canonical order, each taking the smallest colour that none of
 * its already coloured conflicting sites has. Host-only (no device work, no context).
 *   dims     lattice sizes, each >= 1; V = Lx Ly Lz Lt < 2^31
 *   k        distance, 1..16; p displacement, 0 <= p < Lz
 *   colors   out: [V] colours (canonical site order), caller-owned
 *   ncolors  out: the number of colours c
 * FS_ERR_ARG for a null pointer or an argument out of range, FS_ERR_OOM if host memory runs
 * out. */
FS_API int fs_probing_colors(const int dims[4], int k, int p, int32_t* colors, int* ncolors);

/* Variance sampling, Sec. 3.1 algorithm, for the m_shifts sampling shifts s_hat
 * (s_hat_0 < ... ) and every displacement p[k], k < np, with Ns Z4 noise vectors
 * (Philox counter {site, k, 0x80000000, job}). For each noise z_k and shift s_i it solves
 * x^(i) = (D+s_i)^-1 z_k and y^(i) = (D+s_i)^-dag z_k = gamma_5 (D+s_i)^-1 gamma_5 z_k, then
 *   a_i  = z_k^dag Gamma Omega_p x^(i)         -> VL[k_p][i]      (Eq. (sampled_single))
 *   b_ij = y^(i)^dag Gamma Omega_p x^(j), j>=i -> Vbar[k_p][i][j] (Eq. (bar_vl))
 * with the practical variance of Eq. (practical_variance). Outputs (host):
 *   VL [np][m_shifts], Vbar [np][m_shifts][m_shifts] (entries j < i set to 0),
 *   a (optional) [Ns][np][m_shifts][2], b (optional) [Ns][np][m_shifts][m_shifts][2],
 *   iters (optional) [m_shifts] mean BiCGStab iterations of the solves at each shift. */
FS_API int variance_sample(fs_ctx* ctx, double m, const double* s_hat, int m_shifts, const double* gamma,
                    const int* p, int np, int Ns, uint64_t seed, uint32_t job,
                    const fs_solve_params* params, double* VL, double* Vbar, double* a, double* b,
                    double* iters);

/* variance_sample with probed and diluted noise (Sec. 2.1, Eq. (probing_vectors); Sec. 3.1):
 * each noise vector z_k is split into pieces, its restrictions to the sites of one colour
 * j < ncolors (colors: [V] in canonical order, values in [0, ncolors), every colour used; NULL =
 * no probing) and, with dilute = 1, to one spin-colour index (12 pieces per colour), and a_i,
 * b_ij are the sums over the pieces. With dilute = 1 every piece lives on one spin s, so
 * gamma_5 z = +-z and y^(i) = +-gamma_5 x^(i) needs no second solve: 12 c m N_s solves in all
 * (Sec. 3.1), against 2 m N_s c' without dilution (c' = ncolors or 1).
 * hpe_order = K > 0: at every sampling shift with m + s_i > 0, a_i is the remainder of the
 * hopping parameter expansion, z^dag Gamma Omega_p (kappa_i H)^K x^(i) (see fs_mlmc_params),
 * so VL is the variance of the expanded estimator; its exact low orders shift every sample
 * alike and are not added (Sec. 3.1: not needed for the sampling). b_ij is unchanged.
 * Outputs and errors as variance_sample; iters averages every solve at the shift. */
FS_API int variance_sample_probed(fs_ctx* ctx, double m, const double* s_hat, int m_shifts, const double* gamma,
                           const int* p, int np, int Ns, uint64_t seed, uint32_t job,
                           const fs_solve_params* params, const int32_t* colors, int ncolors, int dilute,
                           int hpe_order, double* VL, double* Vbar, double* a, double* b, double* iters);

/* The Z4 noise vector (seed, job, level, sample) as integer codes k (z = i^k),
 * host [V][4][3] bytes, generated on the device (bit-exact RNG checks). */
FS_API int fs_noise_codes(fs_ctx* ctx, uint64_t seed, uint32_t job, uint32_t level, uint32_t sample,
                   uint8_t* codes);

/* Sum over all calls since the last reset of the device time of the hopping (dslash)
 * kernel launches of ctx: number of launches, total milliseconds, the algorithmic bytes
 * they moved, and the (site, system) pairs they computed (1320 flop each). Timing is
 * recorded only while enabled (CUDA events around each launch on the context's stream).
 * Any output pointer may be NULL. */
FS_API int fs_profile_enable(fs_ctx* ctx, int enable);
FS_API int fs_profile_read(fs_ctx* ctx, long long* launches, double* total_ms, double* bytes, double* site_systems);
/* The same for the FP64-arithmetic hops on the system-major work lists of a mixed-precision or
 * FP64 solve (the even-odd preparation, the FP64 reliable-update residuals, the odd-site
 * reconstruction and the verification residual): launches, device milliseconds and the
 * (site, system) pairs they computed (1320 flop each on the FP64 pipe). */
FS_API int fs_profile_read_fp64(fs_ctx* ctx, long long* launches, double* total_ms, double* site_systems);

/* ---- serving ---------------------------------------------------------------------
 * A server on one GPU runs FS-MLMC trace jobs (one mlmc_level_trace each) as they arrive.
 * Jobs are admitted when one of `max_active` slots is free and the job's device-memory
 * estimate fits `hbm_budget_bytes` next to the running jobs, least work first with a bound on
 * the wait (fs_server_set_admission; first in, first out on request); every
 * running job has its own worker thread, context and CUDA stream, so their work overlaps
 * on the device, and inside a job the solves are continuously batched. A job's results
 * depend only on its own inputs and are identical alone or in a mix. */
#define FS_JOB_MAX_LEVELS 16

typedef struct fs_server fs_server;

typedef struct fs_job {
  int dims[4];
  int bc_t;
  const double* U;          /* host gauge field [4][V][3][3][2]; copied by fs_server_submit   */
  fs_mlmc_params params;    /* as for mlmc_level_trace; its arrays are copied at submit       */
  double c_sw;              /* the clover coefficient of the job's operator (fs_set_clover);
                               0: Wilson                                                       */
} fs_job;

typedef struct fs_job_result {
  int status;               /* return code of the job's mlmc_level_trace                     */
  int nlev;
  double trace[FS_JOB_MAX_LEVELS][2];
  double var[FS_JOB_MAX_LEVELS];
  long long solves;
  double mean_iters;
  int max_iters;            /* most BiCGStab iterations of one solve                          */
  int noconv;               /* solves that ended FS_SYS_NOCONV                                */
  long long restarts;       /* breakdown restarts summed over the solves                      */
  double latency_ms;        /* completion - submission                                       */
  double queue_ms;          /* admission - submission                                        */
} fs_job_result;

typedef struct fs_server_report {
  long long completed, queued, active, solves;
  size_t reserved_bytes;    /* device-memory estimates of the running jobs                   */
  double p50_ms, p99_ms, max_ms, mean_ms;  /* latency over completed jobs                   */
  double solves_per_s;      /* solves of completed jobs / (last completion - first submission) */
  long long gauge_reuses;   /* jobs whose gauge field was already resident on their worker (same
                               lattice, byte-identical field): no upload, packed copies kept  */
} fs_server_report;

/* FS_ERR_ARG for max_active outside [1, 64] or a zero budget. */
FS_API int fs_server_create(fs_server** server, int device, size_t hbm_budget_bytes, int max_active);
/* Queue a job; FS_ERR_BUDGET if its estimate alone exceeds the budget, FS_ERR_ARG for bad
 * dims or more than FS_JOB_MAX_LEVELS levels. */
FS_API int fs_server_submit(fs_server* server, const fs_job* job, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a job; FS_ERR_TIMEOUT if it is not done yet.
 * A result is returned once, then the ticket is forgotten. */
FS_API int fs_server_poll(fs_server* server, uint64_t ticket, fs_job_result* result, int timeout_ms);
FS_API int fs_server_stats(fs_server* server, fs_server_report* stats);
/* Admission order (a library addition; the paper has no server). least_work_first = 1 (the
 * default): among the queued jobs whose memory estimate fits the budget, the one with the least
 * work (solves x lattice sites) starts first, which shortens the median latency; a job queued for
 * max_wait_ms (default 10000) goes next regardless and no later job passes it, so no job waits
 * for ever. least_work_first = 0: first in, first out. FS_ERR_ARG for other values or a negative
 * wait. */
FS_API int fs_server_set_admission(fs_server* server, int least_work_first, double max_wait_ms);
/* Finishes queued and running jobs, then stops the workers. */
FS_API void fs_server_destroy(fs_server* server);

/* Watchdog of the host solve loops (a library addition; the paper has none): a call on ctx that
 * has run more than `bound` BiCGStab (or CGNR fallback) iterations on one tile returns
 * FS_ERR_TIMEOUT, with that tile's systems left idle and the context usable for the next call.
 * 0 (the default) restores the built-in bound, (2 max_iter + 64)(groups + 1) iterations, which a
 * solve that terminates never reaches. FS_ERR_ARG for a negative bound. */
FS_API int fs_set_iteration_bound(fs_ctx* ctx, long long bound);

/* Number of CUDA kernels this library has launched in the process (all contexts). */
FS_API long long fs_kernel_launches(void);

/* ---- measured arithmetic roofs --------------------------------------------------------
 * The paper has no counterpart; the hop kernels sit at the ridge of this GPU's HBM and FP32
 * roofs, and these measure the FP32 and FP64 roofs on the device itself. fs_measure_peak runs
 * independent fused multiply-add chains (scalar FP32, packed FP32 pairs, or FP64) on every SM of
 * the current device, with as many threads as fit, for about `seconds` (at most 60) on a stream of
 * its own, and writes the rate in TFLOP/s (2 flop per multiply-add) and the elapsed time of the
 * timed launches (CUDA events). The caller samples clocks alongside if it wants a clock-normalised
 * figure. FS_ERR_ARG for a bad kind or time; FS_ERR_CUDA if a CUDA call fails or an error was
 * already pending (left untouched). */
enum fs_peak_kind { FS_PEAK_F32 = 0, FS_PEAK_F32X2 = 1, FS_PEAK_F64 = 2 };
FS_API int fs_measure_peak(int kind, double seconds, double* tflops, double* elapsed_ms);

/* ---- allocation-free variant ------------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that may not
 * allocate device memory while they run: work recorded into a CUDA stream capture,
 * processes that hand out a fixed device-memory budget up front, latency-critical loops
 * that cannot take an allocation's implicit synchronisation. It computes what
 * wilson_dslash computes in FP64, out_k = (D + sigma I) in_k for k < nrhs, on DEVICE
 * buffers in the canonical layouts (U [4][V][3][3][2], in/out [nrhs][V][4][3][2]),
 * without a context and without allocating: its scratch (the even-odd packed gauge
 * field, packed spinors and per-system coefficients) is one fixed 32 MiB static device
 * array that every GPU loading the library holds until process exit.
 * Limits: nrhs <= 64 and 576 V + 384 V nrhs bytes (plus alignment) <= 32 MiB, else
 * FS_ERR_BUDGET; FS_ERR_ARG for bad dims / bc_t / null pointers.
 * The first call on a device looks up the array's device address (that device must be
 * current) and should come before any stream capture. The call is stream ordered on
 * `stream` (a cudaStream_t, NULL = legacy default stream): it returns once its kernels
 * are queued. All calls on a device share the array, so calls whose work overlaps on
 * the GPU (unordered streams) race and corrupt each other; each call rewrites every
 * scratch field it reads, so the contents left by the previous call do not matter.
 * The cached device address does not survive cudaDeviceReset: do not call again in a
 * process after a reset. A CUDA error already pending when the call starts (left by
 * other work) makes it return FS_ERR_CUDA without launching and without clearing that
 * error; a failure of one of its own launches returns FS_ERR_CUDA too. */
FS_API int wilson_dslash_noalloc(const int dims[4], int bc_t, double m, double sigma, const double* U,
                          const double* in, double* out, int nrhs, void* stream);

/* ---- shift selection and sample allocation (host only; paper Sec. 3.2-3.3) --------------
 * Inputs come from variance_sample on m sampling shifts s_hat (increasing; s_hat[0] = 0 in
 * the paper, whose sigma_0 = 0; any first shift serves as sigma_0): VL_hat[i] = V_L(s_hat_i)
 * and the row-major upper triangle Vbar_hat[i*m + j] = Vbar_l(s_hat_i, s_hat_j), j >= i
 * (Eq. (sampled_single), Eq. (bar_vl)). s is the evaluation set (increasing, s[0] = s_hat[0]).
 * All buffers are caller-owned host memory; nothing touches the GPU. FS_ERR_ARG for null
 * pointers, m < 2, n < 2, unordered shifts or s[0] != s_hat[0]; FS_ERR_INPUT for negative or
 * non-finite variances or iteration counts. */

/* Interpolated variances on the evaluation set, in log space with piecewise cubic Hermite
 * interpolating polynomials (linear through two points): VL[k] = V_L(s_k) and
 * Vl[i*n + k] = V_l(s_i, s_k) = (s_k - s_i)^2 Vbar_l(s_i, s_k) for k > i (NaN for k <= i or
 * where no prediction exists), from the three-stage 2-D interpolation of Sec. 3.2. */
FS_API int fs_interp_variances(const double* s_hat, int m, const double* VL_hat, const double* Vbar_hat,
                        const double* s, int n, double* VL /*[n]*/, double* Vl /*[n*n]*/);

/* Eq. (opt_shifts): the L shifts after sigma_0 = s_0 that minimise the multilevel cost
 * C_FS = eps^-2 F^2, F = sum_l sqrt(C_l V_l) (Eq. (ml_cost_shifts)), with V_l from
 * fs_interp_variances and C_l the iteration count of the level's solves: iters_hat at the
 * sampling shifts, next-neighbour interpolated (r(s) = r(s_hat_j), s_hat_{j-1} < s <= s_hat_j),
 * C_l = r(sigma_l) + r(sigma_{l+1}) for l < L, C_L = r(sigma_L). Outputs idx[L+1] (indices
 * into s, idx[0] = 0), V[L+1], C[L+1] and F. FS_ERR_ARG also for L outside [1, n-1] or when
 * no choice of L shifts has predicted variances. */
FS_API int fs_select_shifts(const double* s_hat, int m, const double* VL_hat, const double* Vbar_hat,
                     const double* iters_hat, const double* s, int n, int L, int* idx, double* V, double* C,
                     double* F);

/* Eq. (num_samples), Eq. (total_var): N_l = mu sqrt(V_l / C_l), mu = eps2^-1 sum_l sqrt(V_l C_l)
 * (real-valued; round up for use), and V_FS = sum_l V_l / N_l (= eps2), C_FS = sum_l N_l C_l.
 * mu, V_FS, C_FS may be NULL. FS_ERR_ARG for eps2 <= 0 or nlev < 1; FS_ERR_INPUT for V < 0,
 * C <= 0 or non-finite values. */
FS_API int fs_sample_allocation(const double* V, const double* C, int nlev, double eps2, double* N, double* mu,
                         double* V_FS, double* C_FS);

/* The FS estimate and its variance from the per-level results of mlmc_level_trace(s):
 * total[q] = sum_l trace[q][l] (complex), the level estimates of Eq. (fs_trace_est) summed
 * into the estimate of Tr(Gamma Omega_p (D + sigma_0)^-1), and v_fs[q] = sum_l var[q][l] / N_l,
 * Eq. (total_var) (the levels use independent noise). trace [np][nlev][2] and var [np][nlev]
 * as mlmc_level_traces writes them (np = 1 for mlmc_level_trace), N_l = n_samples[l]; total
 * [np][2], v_fs [np]. Host only. FS_ERR_ARG for null pointers, nlev < 1, np < 1 or a level
 * with no samples; FS_ERR_INPUT for non-finite values. */
FS_API int fs_trace_total(const double* trace, const double* var, const int* n_samples, int nlev, int np,
                          double* total, double* v_fs);

/* Eq. (sampled_prod): the level variance of a pair of sampling shifts,
 * Vl[q][i][j] = (s_hat_j - s_hat_i)^2 Vbar[q][i][j] for j >= i and 0 below the diagonal, from
 * variance_sample's Vbar [np][m][m] (upper triangle) and its m shifts s_hat. Host only.
 * FS_ERR_ARG for null pointers, m < 1 or np < 1; FS_ERR_INPUT for non-finite Vbar. */
FS_API int fs_sampled_level_variances(const double* s_hat, int m, const double* Vbar, int np, double* Vl);

/* The paper's evaluation set (Sec. 3.3): logspace(-5,-2,4) and logspace(log10(0.011),0,76)
 * from s_hat[0] up, with the sampling shifts added, sorted and unique (with s_hat[0] = 0 it
 * starts at 0). With s = NULL only *n is set; otherwise cap must be >= *n. */
FS_API int fs_eval_grid(const double* s_hat, int m, double* s, int cap, int* n);

#ifdef __cplusplus
}
#endif

#endif /* FSMLMC_H */

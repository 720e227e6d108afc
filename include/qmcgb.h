/*
 * qmcgb.h: C ABI of the GB300 (sm_103a) library for the particle-by-particle (PbyP)
 * electron move over a crowd of walkers, after Luo, Doak, Kent, "A High-Performance
 * Design for Hierarchical Parallelism in the QMCPACK Monte Carlo code" (arXiv:2209.14487).
 *
 * A crowd (Sec. III: a subset of the walkers operated on as one batch, in lock-step) holds
 * W walkers of one system.  The calls follow Alg. 1 of the paper:
 *   line 5-6  propose r'_k                      -> qmc_eval_grad_batch, qmc_propose_move_batch
 *   line 7-8  ratio Psi(R')/Psi(R), grad_k      -> qmc_propose_move_batch
 *   line 9    accept / reject (inverse update)  -> qmc_accept_reject_batch
 *   line 11   local energy                      -> qmc_local_energy_batch
 *   lines 1-11 fused over generations           -> qmc_sweep
 *
 * Wavefunction (the paper gives none; the library's reading):
 *   Psi(R) = det A_up det A_dn exp(-U),  A_s[l][j] = phi_j(r_l) (tricubic B-spline orbitals
 *   on a periodic G^3 grid), U = sum_{i<j} u2(r_ij) + sum_{i,I} u1(r_iI) (cubic B-spline
 *   radial functors, minimum image).  Moves: r' = r + tau D + sqrt(tau) chi with the drift
 *   D = grad log Psi limited near nodes (or unlimited, or none), Metropolis(-Hastings)
 *   acceptance, counter-based Philox4x32-10 draws.
 *
 * Conventions:
 *  - Every call returns a qmc_status (QMC_OK = 0).  qmc_status_string() names it.
 *  - Arguments marked "mem" are host pointers (QMC_MEM_HOST) or device pointers
 *    (QMC_MEM_DEVICE) as the call's `mem` argument says.  Calls with device buffers are
 *    asynchronous on the crowd's stream; calls with host buffers copy and synchronise.
 *  - The library owns all device state of a crowd; inputs are copied in; outputs go to
 *    caller-owned buffers.  Positions are double [W][N][3], electrons 0..n_up-1 are spin
 *    up, n_up..N-1 spin down.
 *  - A crowd is not thread safe; distinct crowds may be driven from distinct host
 *    threads and streams (Sec. III, Alg. 4).
 *  - Device-side failures (singular matrix, non-finite energy) are recorded in a status
 *    word that the next synchronising call returns.
 */
#ifndef QMCGB_H
#define QMCGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum qmc_status {
  QMC_OK = 0,
  QMC_ERR_INVALID_ARG = 1, /* bad pointer, size or enum value                         */
  QMC_ERR_OOM = 2,         /* device allocation failed                                */
  QMC_ERR_CUDA = 3,        /* a CUDA runtime call failed                              */
  QMC_ERR_SINGULAR = 4,    /* zero pivot in the FP64 recompute                         */
  QMC_ERR_TIMEOUT = 5,     /* a bounded device wait ran out                            */
  QMC_ERR_NAN = 6,         /* non-finite local energy or ratio (the move is rejected)  */
  QMC_ERR_STATE = 7,       /* call out of order (accept without propose, no orbitals)  */
  QMC_ERR_UNSUPPORTED = 8, /* valid request this build does not serve (size limits)    */
  QMC_ERR_BOUNDS = 9       /* a device bounds check failed (bounds-checked build only) */
} qmc_status;

enum { QMC_MEM_HOST = 0, QMC_MEM_DEVICE = 1 };
enum { QMC_PREC_FP64 = 0, QMC_PREC_MIXED = 1 };
enum { QMC_UPDATE_SM = 0, QMC_UPDATE_DELAYED = 1 };
enum { QMC_J1 = 0, QMC_J2_UU = 1, QMC_J2_UD = 2 };
enum { QMC_DTYPE_F64 = 0, QMC_DTYPE_F32 = 1 };

/* The simulated system (Alg. 1 "R = {r_1 .. r_N}" plus what Psi needs). */
typedef struct qmc_system_desc {
  int n_up, n_dn;  /* electrons per spin; this build requires n_up == n_dn >= 1      */
  int n_orb;       /* orbitals in the table (>= n_up); the first n_up are occupied   */
  int n_ions;      /* electron-ion Jastrow centres (may be 0)                         */
  int grid;        /* G: spline grid points per dimension (>= 4)                      */
  int reserved;
  double L;        /* periodic cubic cell side (bohr)                                 */
} qmc_system_desc;

/* How the crowd is driven. */
enum { QMC_STAGING_AUTO = 0, QMC_STAGING_LDG = 1 };
enum { QMC_LAYOUT_AUTO = 0, QMC_LAYOUT_SHARED = 1, QMC_LAYOUT_COMPACT = 2 };
enum { QMC_ENGINE_AUTO = 0, QMC_ENGINE_SIMT = 1 };

typedef struct qmc_run_desc {
  int n_walkers;    /* W >= 1                                                         */
  int precision;    /* QMC_PREC_FP64: FP64 everywhere; QMC_PREC_MIXED: FP32 orbitals,  *
                     * Jastrow, ratios and inverse, FP64 recompute and energy sums     */
  int update;       /* QMC_UPDATE_SM (rank-1 per accept) or QMC_UPDATE_DELAYED         */
  int delay_rank;   /* k for QMC_UPDATE_DELAYED, 1..64; 0: the library picks k (the   *
                     * largest rank up to 32 its shared-memory plan holds with the       *
                     * inverse in global memory, 8 when the inverse fits in shared       *
                     * memory: the measured optima on GB300); qmc_get_update reports it  */
  int n_recompute;  /* generations between FP64 recomputes of A^-1; 0 = never        */
  int drift;        /* proposal r' = r + tau D + sqrt(tau) chi with Metropolis-Hastings  *
                     * acceptance and D from F = grad log Psi: 1: D = 2 F / (1 +        *
                     * sqrt(1 + 2 tau |F|^2)), the drift limited as in Umrigar,         *
                     * Nightingale, Runge (1993), so tau |D| < sqrt(2 tau) near nodes;  *
                     * 2: D = F (unlimited); 0: no drift (plain Metropolis)             */
  int potential;    /* 1: add the model potential to E_L                              */
  int staging;      /* QMC_STAGING_AUTO (0): each move's 4x4x4 x n orbital stencil is  *
                     * copied to shared memory with one TMA tensor copy when it fits   *
                     * (n_pad <= 256), else in the mixed path with 128 threads by a    *
                     * ring of TMA boxes (256 orbitals x one x-plane, three in flight);*
                     * QMC_STAGING_LDG: the stencil is read with per-thread loads      */
  double tau;       /* time step                                                      */
  uint64_t seed;    /* Philox key: (low 32 bits, walker ^ high 32 bits)               */
  int cta_threads;  /* threads per walker CTA of the move kernel: 128, 160, 256, or 0 *
                     * for the library's choice (128 up to 128 electrons per spin,     *
                     * else 256); the tensor-core flush needs 128 or 256               */
  int engine;       /* QMC_ENGINE_AUTO (0): in the mixed path with the delayed update   *
                     * and the inverse in global memory, windows are flushed on the    *
                     * tensor cores (tcgen05, 3xTF32); QMC_ENGINE_SIMT: CUDA cores     */
  int dmc;          /* 1: diffusion Monte Carlo: fixed-node acceptance (a move that     *
                     * changes the sign of the determinant is rejected) and population *
                     * branching by qmc_dmc_branch; n_walkers is then the capacity     */
  int layout;       /* shared-memory layout of the move kernel: QMC_LAYOUT_AUTO (0) the  *
                     * library's pick (below), QMC_LAYOUT_SHARED: the delayed window's  *
                     * new orbital rows and each sweep's table of draws in shared       *
                     * memory, QMC_LAYOUT_COMPACT: both outside it (the window rows in  *
                     * global memory, where they are kept between calls anyway, and    *
                     * each move's draws computed from the same Philox words when       *
                     * needed), so that larger systems fit and more CTAs share an SM;   *
                     * results are the same either way.  AUTO takes SHARED unless only  *
                     * COMPACT fits (FP64 Sherman-Morrison at n = 768, for one).        */
  double guard_tol; /* mixed path: inverse guard bound (0: the library's 0.1; < 0:      *
                     * off).  After each sweep every walker's FP32 inverses are probed   *
                     * with a fixed sign vector v (v_l = -1 where bit 31 of             *
                     * (l + 1) * 0x9E3779B1 mod 2^32 is set, else +1):                   *
                     * g_s = max over k of |(v^T (A_s B_s - I))_k|; a spin whose g_s   *
                     * exceeds guard_tol (or is not finite) has its inverse, log|det|   *
                     * and sign recomputed in FP64 (LU with partial pivoting) before    *
                     * the walker's E_L -- an early instance of the periodic recompute  *
                     * (Alg. 1 line 3).  Ignored by the FP64 path.                      */
} qmc_run_desc;

/* Per-call statistics of qmc_sweep, accumulated in FP64 over walkers and generations. */
typedef struct qmc_stats {
  double e_sum;          /* sum over walkers and generations of E_L                    */
  double e2_sum;         /* sum of E_L^2                                               */
  long long n_samples;   /* walkers x generations                                      */
  long long n_accept;    /* accepted moves                                             */
  long long n_moves;     /* proposed moves = W x N x generations                       */
  long long n_repair;    /* walkers the guard repaired (one or both inverses recomputed) */
} qmc_stats;

typedef struct qmc_crowd qmc_crowd;

/* Creates a crowd of run->n_walkers walkers of system `sys` on the current CUDA device.
 * `cuda_stream` is a cudaStream_t (may be NULL: the crowd creates its own stream).
 * Allocates all device state (O(W N n) for the orbital rows, O(W n^2) for inverses).
 * Errors: INVALID_ARG (sizes), UNSUPPORTED (n_up != n_dn, grid or n beyond limits), OOM. */
int qmc_crowd_create(const qmc_system_desc* sys, const qmc_run_desc* run, void* cuda_stream,
                     qmc_crowd** out);
int qmc_crowd_destroy(qmc_crowd* crowd);

/* Electron positions, double [W][N][3] (mem).  Values are wrapped into [0, L).  Marks
 * the orbital rows and inverses stale: the next move, energy or explicit
 * qmc_recompute() rebuilds them (Alg. 1 line 3).  Errors: INVALID_ARG (also for a
 * non-finite coordinate in host memory: nothing is loaded); a non-finite coordinate in
 * device memory is replaced by 0 and the next synchronising call returns QMC_ERR_NAN. */
int qmc_load_positions(qmc_crowd* crowd, const double* R, int mem);
/* Ion positions, double [n_ions][3] (host).  Errors: INVALID_ARG (also non-finite). */
int qmc_load_ions(qmc_crowd* crowd, const double* RI);
/* Orbital coefficient table [G][G][G][n_orb] (mem), x slowest, orbital fastest, periodic
 * (node g at x = g L / G), dtype QMC_DTYPE_F64 or F32.  The library adds three ghost
 * layers, pads the orbital dimension and converts to the crowd's precision. */
int qmc_load_orbitals(qmc_crowd* crowd, const void* coefs, int dtype, int mem);
/* Radial functor `kind` with K >= 1 free coefficients c (host) and cutoff rc > 0;
 * u(r) = sum_m c_{i+m} b_m(r/h - i), h = rc/K, i = floor(r/h), three zero coefficients
 * follow c_{K-1}; u = 0 for r >= rc.  K = 0 removes the term. */
int qmc_load_jastrow(qmc_crowd* crowd, int kind, const double* c, int K, double rc);

/* FP64 full recompute: orbital rows from the positions, LU with partial pivoting of
 * each A_s, A_s^-1, log|det A_s| and sign.  Errors: SINGULAR. */
int qmc_recompute(qmc_crowd* crowd);

/* grad_k log Psi(R) for electron iel of every walker: grad [W][3] (mem). */
int qmc_eval_grad_batch(qmc_crowd* crowd, int iel, double* grad, int mem);

/* Proposes electron iel of every walker (Alg. 1 lines 5-8).
 * rnew [W][3] (mem) gives r'; NULL draws r' = r + tau F + sqrt(tau) chi from the
 * crowd's counter-based RNG at its current generation.  Outputs (mem, each may be NULL):
 * ratio [W] = Psi(R')/Psi(R); grad [W][3] = grad_k log Psi(R'); log_ratio [W] =
 * log|ratio|; rnew_out [W][3] = the proposed, wrapped r'.  The proposal stays pending
 * for qmc_accept_reject_batch. */
int qmc_propose_move_batch(qmc_crowd* crowd, int iel, const double* rnew, double* ratio,
                           double* grad, double* log_ratio, double* rnew_out, int mem);

/* Accepts or rejects the pending proposal of electron iel (Alg. 1 line 9).
 * accept [W] (mem, nonzero = accept) or NULL for the Metropolis test with the crowd's RNG;
 * accepted_out [W] (mem, may be NULL) receives the decisions.  Accepting updates the
 * inverse (Sherman-Morrison, or appends to the delayed window), the orbital rows, the
 * position and log|det|.  Errors: STATE if no proposal of iel is pending. */
int qmc_accept_reject_batch(qmc_crowd* crowd, int iel, const uint8_t* accept,
                            uint8_t* accepted_out, int mem);

/* Local energy of every walker (Alg. 1 line 11): eloc [W] (mem).  Applies pending
 * delayed updates first. */
int qmc_local_energy_batch(qmc_crowd* crowd, double* eloc, int mem);

/* n_gen generations in one fused launch per generation: every electron of every walker
 * proposed once in order, pending updates applied, the FP64 recompute every n_recompute
 * generations, then E_L.  eloc [n_gen][W] (mem, may be NULL); stats (host, may be NULL:
 * without it the call does not synchronise). */
int qmc_sweep(qmc_crowd* crowd, int n_gen, double* eloc, int mem, qmc_stats* stats);

/* Getters (host buffers unless mem says otherwise). */
int qmc_get_positions(qmc_crowd* crowd, double* R, int mem);
/* log|Psi| = log|det A_up| + log|det A_dn| - U and sign(Psi), [W] each (host). */
int qmc_get_logpsi(qmc_crowd* crowd, double* logabs, int* sign);
/* A_s^-1 of every walker as double [W][n][n], element [w][j][l] = (A_s^-1)[j][l]
 * (host); applies pending delayed updates first. */
int qmc_get_inverse(qmc_crowd* crowd, int spin, double* out);
/* A_s of every walker as double [W][n][n], [w][l][j] = phi_j(r_l) (host). */
int qmc_get_slater_matrix(qmc_crowd* crowd, int spin, double* out);
int qmc_get_generation(qmc_crowd* crowd, uint32_t* gen);
int qmc_set_generation(qmc_crowd* crowd, uint32_t gen);
/* Number of kernel launches this crowd has issued so far. */
int qmc_get_launch_count(qmc_crowd* crowd, unsigned long long* count);
/* The move kernel's configuration, chosen at creation from the shared memory a CTA may
 * use: 1 in *b_in_smem when the moving spin's inverse is staged in shared memory, 1 in
 * *stencil_tma when each move's orbital stencil arrives by one TMA copy (2: by the ring of
 * TMA boxes, 0: by per-thread loads), the kernel's dynamic
 * shared memory in bytes, its threads per CTA, 1 in *tc_flush when delayed windows
 * are flushed on the tensor cores, and the layout taken (QMC_LAYOUT_SHARED or
 * QMC_LAYOUT_COMPACT).  Any output pointer may be NULL.  Errors: INVALID_ARG. */
int qmc_get_kernel_config(const qmc_crowd* crowd, int* b_in_smem, int* stencil_tma,
                          int* smem_bytes, int* cta_threads, int* tc_flush, int* layout);

/* Checkpoint: positions, generation and RNG seed.  With buf == NULL, *size receives the
 * byte count; otherwise *size must hold at least that many bytes.  Restoring recomputes
 * every derived quantity in FP64 from the positions. */
int qmc_crowd_save(qmc_crowd* crowd, void* buf, size_t* size);
int qmc_crowd_restore(qmc_crowd* crowd, const void* buf, size_t size);

const char* qmc_status_string(int status);
/* ---------------------------------------------------------------------------------------
 * Batches: crowds of different systems (electron counts, grids, ions) swept together,
 * one kernel launch per generation whose CTAs cover every walker of every crowd (the
 * crowd concept of Sec. III applied across systems of different sizes).  Each crowd keeps
 * its own state, RNG key, generation counter and FP64 recompute cadence; the result of a
 * batch sweep equals that of qmc_sweep on each crowd.  Generations without a recompute
 * replay a captured CUDA graph (move launch + counter advance).
 * --------------------------------------------------------------------------------------- */
typedef struct qmc_batch qmc_batch;

/* 1..8 distinct crowds on the current device with the same precision, update kind and
 * cta_threads (UNSUPPORTED otherwise).  The batch launches on crowds[0]'s stream and
 * orders the other crowds' streams around each sweep.  The crowds must outlive the batch.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM. */
int qmc_batch_create(qmc_crowd* const* crowds, int n_crowds, qmc_batch** out);
int qmc_batch_destroy(qmc_batch* batch);
/* n_gen generations of every crowd.  eloc: NULL, or n_crowds pointers (entries may be
 * NULL) to host buffers double [n_gen][W_c] for crowd c's E_L; stats: NULL or n_crowds
 * entries.  Synchronous.
 * Errors: as qmc_sweep. */
int qmc_batch_sweep(qmc_batch* batch, int n_gen, double* const* eloc, qmc_stats* stats);
/* Kernel launches (graph replays count their nodes) issued by the batch so far. */
int qmc_batch_get_launch_count(const qmc_batch* batch, unsigned long long* count);

/* ---------------------------------------------------------------------------------------
 * DMC branching (Alg. 1 lines 13-14; the paper gives no formulas, the readings are):
 * after a generation, walker w's weight is exp(-tau ((E_prev[w] + E_new[w]) / 2 - e_trial))
 * and its multiplicity floor(weight + u) with u the walker's Philox uniform from counter
 * (generation just completed, N, 3, 0); the new population lists walker 0 M_0 times,
 * walker 1 M_1 times, ... (each copy carries the walker's full state: positions, orbital
 * rows, inverses, log|det|), cut at the crowd's capacity (run.n_walkers).  Pending delayed
 * windows are applied first.  The crowd's active walker count becomes n_after.
 * e_prev: double [W] (mem); e_new: double [capacity] (mem) holding the W walkers' E_L
 * after the generation; on return e_new[0..n_after) holds the new population's E_L (the
 * next generation's e_prev).  Needs run.dmc.  Errors: INVALID_ARG; STATE (no
 * DMC crowd, or every multiplicity zero: the crowd is then left unchanged).
 * --------------------------------------------------------------------------------------- */
typedef struct qmc_dmc_stats {
  int n_before;       /* walkers before branching                                     */
  int n_after;        /* walkers after (at most the capacity)                         */
  long long n_wanted; /* sum of multiplicities before the capacity cut                 */
  double w_sum;       /* sum of weights                                               */
  double we_sum;      /* sum of weight x E_new (the mixed estimator's numerator)       */
} qmc_dmc_stats;

int qmc_dmc_branch(qmc_crowd* crowd, const double* e_prev, double* e_new, int mem,
                   double e_trial, qmc_dmc_stats* out);
/* The mixed path's inverse guard (run.guard_tol): values [W] (host, may be NULL) receives
 * max(g_up, g_dn) of every walker's last sweep (before any repair; walker slots as they
 * were at that sweep, so a DMC branch since then reorders them), n_repair (host, may be
 * NULL) the walkers repaired since the crowd was created.  Synchronous.  Errors: INVALID_ARG; STATE (an
 * FP64 crowd or a crowd created with the guard off). */
int qmc_get_guard(qmc_crowd* crowd, double* values, long long* n_repair);
/* Records the accept decisions of qmc_sweep (on = 1) or stops recording (on = 0).  While
 * on, every sweep generation writes walker w's decision for electron i (1 accepted, 0
 * rejected) to entry [w][i] of a library-owned record, which qmc_get_accept_trace copies
 * out: out uint8 [W][N] (host), the decisions of the last generation swept.  Synchronous.
 * Errors: INVALID_ARG; OOM; STATE (qmc_get_accept_trace while not recording). */
int qmc_trace_accepts(qmc_crowd* crowd, int on);
int qmc_get_accept_trace(qmc_crowd* crowd, uint8_t* out);
/* Failure-detection test hook.  Every device wait of the move kernel (a stencil copy, a
 * tensor-core product) is bounded: after about one second the kernel records
 * QMC_ERR_TIMEOUT, leaves the generation, and the crowd rebuilds its rows and inverses
 * from the stored positions at the next call.  With on = 1 the kernel stops issuing its
 * stencil copies but still waits for them, so that a test can make the wait run out with
 * no copy in flight (the next sweep then takes about two seconds and returns
 * QMC_ERR_TIMEOUT); on = 0 issues them again.  Needs a crowd whose stencil arrives by TMA
 * (qmc_get_kernel_config).  Errors: INVALID_ARG (no TMA staging, on not 0 or 1). */
int qmc_test_skip_stencil_copy(qmc_crowd* crowd, int on);
/* Active walkers of the crowd (n_walkers unless DMC branching changed it). */
int qmc_get_walker_count(const qmc_crowd* crowd, int* count);
/* The crowd's update scheme and delay rank (the library's pick when run.delay_rank was 0;
 * 1 for Sherman-Morrison). */
int qmc_get_update(const qmc_crowd* crowd, int* update, int* delay_rank);

/* ---------------------------------------------------------------------------------------
 * Nonlocal pseudopotential in E_L (the locality approximation; the paper's NiO runs use
 * pseudopotentials, its text gives no form, so the channels are synthetic Gaussians):
 * every ion carries channels l = 0..n_l-1 with v_l(r) = amp[l] exp(-(r / width[l])^2) for
 * r < rc.  Each electron i within rc of ion I (d = r_i - R_I, minimum image, r = |d|) adds
 *   sum_l v_l(r) (2l+1) (1/12) sum_q P_l(d.u_q / r) Psi(r_i -> R_I + r u_q) / Psi(R)
 * over the 12 vertices u_q of an icosahedron in a fixed orientation ((0, +-1, +-phi)
 * normalised and its cyclic shifts), P_0 = 1, P_1 = x, P_2 = (3x^2 - 1) / 2.  Every E_L the
 * crowd computes from then on includes it (one extra launch per E_L); batches of crowds
 * (qmc_batch_*) do not serve it and return UNSUPPORTED.  n_l = 0 removes it.
 * amp, width: double [n_l] (host); 0 <= n_l <= 3; width > 0; 0 < rc <= L/2.
 * Errors: INVALID_ARG (nothing changes).
 * --------------------------------------------------------------------------------------- */
int qmc_load_nlpp(qmc_crowd* crowd, int n_l, const double* amp, const double* width, double rc);

/* ---------------------------------------------------------------------------------------
 * Coulomb energy in E_L by Ewald summation (the paper's runs use it; its text gives no
 * form): charges -1 (electrons) and +Z (every ion) in the periodic cube, V = L^3,
 *   E = sum_{a<b} q_a q_b erfc(alpha r_ab) / r_ab   (minimum image of each pair)
 *     + (2 pi / V) sum_{k != 0} exp(-k^2 / (4 alpha^2)) / k^2 |S(k)|^2
 *     - (alpha / sqrt(pi)) sum_a q_a^2 - pi Q^2 / (2 V alpha^2),
 * S(k) = sum_a q_a exp(i k.r_a), k = 2 pi m / L over integer m, 0 < |m|^2 <= mmax^2,
 * Q = sum_a q_a (the last term is the neutralising background's).  The ion-ion part is
 * included.  It adds to the model potential of run.potential.  The minimum-image
 * real-space sum is exact when erfc(alpha L / 2) is negligible (alpha L >~ 10).
 * on: 1 to add the term (Z >= 0, alpha > 0, mmax >= 1), 0 to remove it.  Batches of crowds
 * do not serve it.  Errors: INVALID_ARG; UNSUPPORTED (more than 4096 half-space vectors:
 * mmax above about 12); OOM.
 * --------------------------------------------------------------------------------------- */
int qmc_load_coulomb(qmc_crowd* crowd, int on, double Z, double alpha, int mmax);

/* ---------------------------------------------------------------------------------------
 * Population edits for walker exchange between crowds (one crowd per GPU; Sec. III's
 * walkers are independent, so any walker may move to any crowd of the same system).
 *
 * qmc_dmc_select: the new population is walkers src[0..n_new) of the current one, in
 * that order, repeats allowed (each copy carries the walker's full state, as in
 * qmc_dmc_branch); pending delayed windows are applied first.  src: int [n_new] (mem),
 * every entry in [0, W); 1 <= n_new <= capacity.  Needs run.dmc.  Synchronous.
 * Errors: INVALID_ARG (a bad index or size: nothing changes), STATE (no DMC crowd).
 *
 * qmc_dmc_append: m walkers join at slots W..W+m-1 with positions R: double [m][N][3]
 * (mem), wrapped into the cell; their orbital rows and inverses are built (FP64
 * recompute) and nothing of the other walkers changes.  W + m <= capacity.  Synchronous.
 * Errors: INVALID_ARG (also a non-finite coordinate in host memory); NAN (one in device
 * memory: replaced by 0); SINGULAR (a joining walker's Slater matrix is singular).
 * --------------------------------------------------------------------------------------- */
int qmc_dmc_select(qmc_crowd* crowd, const int* src, int n_new, int mem);
int qmc_dmc_append(qmc_crowd* crowd, const double* R, int m, int mem);

/* Text of the CUDA error behind the calling thread's last QMC_ERR_CUDA ("no error" if none). */
const char* qmc_last_cuda_error(void);

/* ---------------------------------------------------------------------------------------
 * Bounds-checked build.  The same sources compiled with -DQMCGB_CHECK=1 (libqmcgb_check.so,
 * `python -m paper_2209_14487_gb300.build --check`) check, on the device, every walker and
 * electron index a kernel takes, each proposal's spline cell (its 4x4x4 stencil must lie in
 * the ghost-padded table), each stencil item's orbital and point, the delayed window's
 * count before an append, the shared-memory layout against the launch's dynamic shared
 * memory, the TMA stencil copy's size and buffer, the nonlocal pair list's ion indices and
 * the DMC gather's source walkers.  A failed check records its site and value (the first
 * failure of the crowd), skips the access (a bad index is replaced by 0, a bad walker or
 * layout ends the CTA) and makes the call return QMC_ERR_BOUNDS; the crowd then rebuilds
 * its state from the stored positions at the next call.  In the normal build the checks
 * compile to nothing, qmc_build_flags() is 0 and qmc_check_report reports nothing.
 * --------------------------------------------------------------------------------------- */
enum { QMC_BUILD_CHECKED = 1 };
/* QMC_BUILD_CHECKED when this library is the bounds-checked build, else 0. */
int qmc_build_flags(void);
/* The crowd's first failed check since the last report, then cleared: site (host) 0 if
 * none, else 1 walker, 2 electron, 3 spline cell, 4 stencil item, 5 window count,
 * 6 shared-memory layout, 7 stencil copy, 8 pair-list ion, 9 DMC source walker; value
 * (host, may be NULL) the offending index (for a cell: dimension << 32 | cell).
 * Synchronous.  Errors: INVALID_ARG. */
int qmc_check_report(qmc_crowd* crowd, int* site, long long* value);
/* Test hook of the checked build: with on = 1 every proposal of electron 0 gets spline cell
 * G + 5 in x (outside the table), which the cell check records (site 3) and replaces by
 * cell 0 before any load, so the call returns QMC_ERR_BOUNDS; on = 0 removes it.  Errors:
 * INVALID_ARG; UNSUPPORTED in the normal build (no check would stop the access). */
int qmc_test_plant_bad_cell(qmc_crowd* crowd, int on);

/* Allocation-free FP64 inverse of a batch of dense matrices.  The paper has no
 * counterpart: this call exists for callers that must not allocate device memory when
 * they need it, such as code in a host callback, a latency-critical loop where
 * cudaMalloc's implicit synchronisation is not allowed, or a runtime that owns all device
 * memory through its own pool.
 *   a      [batch][n][n] device, row major (not modified)
 *   inv    [batch][n][n] device: inv[b][j][l] = (a_b^-1)[j][l]; filled with NaN when a_b
 *          is singular
 *   logdet [batch] device: log|det a_b| (-inf when singular)
 *   sign   [batch] device: sign of det a_b, 0 when a zero pivot shows a_b singular
 * LU with partial pivoting in FP64, asynchronous on cuda_stream (NULL: legacy default
 * stream).  The LU factors live in one 16 MiB static device array that the library holds
 * on every GPU that loads it until the process exits; a batch larger than 2^21 / n^2
 * matrices runs as several launches in stream order.  Limits: 1 <= n <= 1024 (else
 * QMC_ERR_INVALID_ARG / QMC_ERR_UNSUPPORTED), batch >= 0.  No device memory is allocated
 * or freed and no allocating library routine is called.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) and should come before any stream
 * capture.  All calls share the array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and corrupt each other's results.  Nothing in the
 * array has to start at zero: each launch overwrites the factors it reads. */
int qmc_inverse_noalloc(const double* a, int n, int batch, double* inv, double* logdet,
                        int* sign, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* QMCGB_H */

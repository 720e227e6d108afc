// Internal interface between the CUDA translation units of libqmcgb (not part of the ABI).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace qmcgb {

constexpr int LA_NT = 256;         // threads per CTA of the row, LU and Jastrow kernels
constexpr int LA_NWARP = LA_NT / 32;
constexpr int MAX_K = 64;          // largest delay rank
constexpr int MAX_KNOTS = 64;      // largest radial functor (free coefficients)
constexpr int PEND_STRIDE = 24;    // doubles of pending-proposal state per walker
// Ring-staged stencil (n_pad > 256, mixed path): TMA boxes of RING_ORB orbitals x one
// 4x4 (y, z) plane of the stencil, RING_SLOTS of them in flight per CTA
constexpr int RING_ORB = 256;
constexpr int RING_SLOTS = 3;

// pending-proposal slots (doubles)
enum {
  P_R = 0, P_DISP = 3, P_FP = 6, P_RHOD = 9, P_RHO = 10, P_DU = 11, P_LOGGF = 12,
  P_IEL = 13, P_VALID = 14
};

enum Mode {
  MODE_SWEEP = 0,    // one generation: every electron moved once, windows applied, E_L
  MODE_GRAD = 1,     // grad log Psi of electron iel at the current positions
  MODE_PROPOSE = 2,  // ratio and grad at r' for electron iel, kept pending
  MODE_ACCEPT = 3,   // accept / reject the pending proposal of electron iel
  MODE_ELOC = 4,     // apply windows, E_L
  MODE_FLUSH = 5,    // apply windows only
  MODE_SWEEP_NOE = 6 // MODE_SWEEP without E_L (a recompute comes first)
};

// status bits written by kernels
enum { ST_SINGULAR = 1, ST_NAN = 2, ST_STATE = 4, ST_TIMEOUT = 8, ST_BOUNDS = 16 };

// Bounds-checked build (nvcc -DQMCGB_CHECK=1, libqmcgb_check.so): the index checks below
// record the first failed check (site and offending value) in Params::check_info, set
// ST_BOUNDS and skip the access; in the normal build they compile to nothing.
#ifndef QMCGB_CHECK
#define QMCGB_CHECK 0
#endif
enum CheckSite {
  CK_WALKER = 1,   // CTA's walker index >= W
  CK_ELECTRON = 2, // electron index outside [0, N)
  CK_CELL = 3,     // spline cell outside [0, G - 1] (its 4x4x4 stencil leaves the table)
  CK_ORBITAL = 4,  // stencil item: orbital >= n_pad or point >= 4
  CK_WINDOW = 5,   // delayed window count > k before an append
  CK_SMEM = 6,     // shared-memory layout larger than the launch's dynamic shared memory
  CK_STENCIL = 7,  // TMA stencil copy size != 64 n_pad elements, or its buffer misaligned
  CK_PAIR = 8,     // nonlocal pair list: ion index >= n_ions
  CK_SOURCE = 9    // DMC gather: source walker >= the old population
};

struct Params {
  int W, N, n_up, n;        // n = electrons per spin = occupied orbitals
  int n_pad;                // orbital stride of the table and of the rows
  int n_ions, G, GP;        // GP = G + 3 (ghost layers)
  int drift, potential, update, k;
  int K2, K1;               // free radial coefficients (0 = term absent)
  int b_in_smem;            // inverse of the moving spin staged in shared memory
  int skip_eloc;            // sweep without the local energy (a recompute comes first)
  int nt;                   // threads per CTA of the move kernel: 128, 160 or 256
  int use_tma;              // 1: each move's 4x4x4 x n_pad stencil by one TMA copy; 2: by
                            // a ring of TMA copies of RING_ORB orbitals x one x-plane
  int tc_flush;             // delayed windows flushed on the tensor cores (mixed, B global)
  int inc_jastrow;          // mixed Sherman-Morrison sweep: incremental Jastrow grad/lap
  int compact;              // compact shared memory: the delayed window's V rows stay in
                            // win_V (global) and each move's draws are computed when needed
  int dmc;                  // fixed node: a move that changes the determinant's sign is rejected
  int nl_n;                 // nonlocal pseudopotential channels l < nl_n in E_L (0: none)
  double nl_rc;             // their cutoff; v_l(r) = nl_a[l] exp(-r^2 nl_sinv2[l])
  double nl_a[3], nl_sinv2[3];
  int coul;                 // Ewald Coulomb energy in E_L (electrons -1, ions +coul_Z)
  int coul_mmax, coul_nk;   // |m| <= mmax; coul_nk half-space vectors in coul_m / coul_c
  double coul_alpha, coul_Z, coul_const;  // splitting, ion charge, self + background terms
  const int* coul_m;        // [coul_nk][3] integer vectors m (k = 2 pi m / L)
  const double* coul_c;     // [coul_nk] (4 pi / V) exp(-k^2 / (4 alpha^2)) / k^2
  int eloc_by_gen;          // E_L of generation g goes to eloc_out[(g - eloc_gen0) W + w]
  uint32_t eloc_gen0;
  int stencil_bytes;        // bytes of that copy
  int vs, ks;               // padded strides of the window's V rows and S^-1 rows
  uint32_t gen;
  double L, invL, tau, sqrt_tau, dgrid;   // dgrid = G / L
  double rc2, rc1, h2inv, h1inv;
  double fx_scale, fx_unit;               // 2^32 / L and L / 2^32 (fixed-point positions)
  uint64_t seed;
  const void* table;        // [GP^3][n_pad] T
  const void* jc;           // T [K2+3] like, [K2+3] unlike, [K1+3] electron-ion
  const double* ions;       // [n_ions][3]
  double* R;                // [W][N][3]
  void* rows;               // [W][N][5][n_pad] T: phi, dphi/dx, dphi/dy, dphi/dz, lap phi
  void* binv;               // [W][2][n][n] T: B^T, [k][j] = (A^-1)[j][k]
  double* logdet;           // [W][2]
  int* sign;                // [W][2]
  int* win_m;               // [W][2]
  int* win_P;               // [W][2][MAX_K]
  void* win_V;              // [W][2][k][vs] T
  void* win_S;              // [W][2][k][ks] T  (S^-1)
  void* pend_phi;           // [W][5][n_pad] T
  void* flush_scratch;      // [W][2][k][n] T: tensor-core flush, snapshot rows and Y^T
  void* jgl;                // [W][N][4] T: Jastrow grad U (3) and lap U of every electron
  int* jvalid;              // [W]: jgl holds the walker's current values
  double* pend;             // [W][PEND_STRIDE]
  // inverse guard (mixed sweep): a walker whose probe of A B - I exceeds guard_tol gets
  // its inverses recomputed by the FP64 LU before its E_L
  float guard_tol;
  float* guard_val;         // [W] probe value of the last sweep; null: no guard
  unsigned long long* n_repair;  // [2]: repairs since creation, since the call began
  double* lu_ws;            // [W][2][2 n^2] FP64 workspace of the repair's LU
  uint8_t* accept_trace;    // [W][N]: a sweep's accept decisions (null: not recorded)
  int test_no_copy;         // failure-detection test: stencil copies are not issued
  int test_bad_cell;        // checked-build test: electron 0's proposals get cell G + 5
  int iel;
  const double* rnew_in;    // [W][3] or null
  double* ratio_out;
  double* grad_out;
  double* logratio_out;
  double* rnew_out;
  const uint8_t* accept_in; // [W] or null
  uint8_t* accept_out;
  double* eloc_out;         // [W]
  unsigned long long* n_accept;
  int* status;
  unsigned long long* check_info;  // checked build: site << 56 | value of the first failure
};

#if defined(__CUDACC__)
#if QMCGB_CHECK
__device__ __noinline__ inline void check_record(int* status, unsigned long long* info, int site,
                                                 long long v) {
  atomicOr(status, (int)ST_BOUNDS);
  if (info)
    atomicCAS(info, 0ull, ((unsigned long long)site << 56) |
                              ((unsigned long long)v & ((1ull << 56) - 1)));
}
// true when COND holds; otherwise records (SITE, V) and yields false (the caller skips)
#define QMC_CHECK(STATUS, INFO, COND, SITE, V) \
  ((COND) ? true : (::qmcgb::check_record((STATUS), (INFO), (SITE), (long long)(V)), false))
#else
#define QMC_CHECK(STATUS, INFO, COND, SITE, V) true
#endif
#define QMC_CHECKP(P, COND, SITE, V) QMC_CHECK((P).status, (P).check_info, COND, SITE, V)
#endif


size_t move_smem_bytes(const Params& p, int elem_bytes);
int max_smem_optin();

// The per-walker state a DMC branching step copies (one half of a double buffer).
struct WalkerState {
  double* R;
  void* rows;
  void* binv;
  void* jgl;
  double* logdet;
  int* sign;
  int* jvalid;
  size_t r_elems, rows_bytes, binv_bytes, jgl_bytes;  // per walker
  int n_walkers;                   // walkers in this half (checked build: gather sources)
  int* status;                     // the crowd's status word and check record
  unsigned long long* check_info;
};
cudaError_t launch_branch(const double* e_prev, const double* e_new, int W, int N, double tau,
                          double e_trial, uint64_t seed, uint32_t gen, int cap, int* mult,
                          int* src, int* out, double* sums, cudaStream_t s);
cudaError_t launch_gather(const WalkerState& to, const WalkerState& from, const int* src,
                          int n_new, const double* e_new, double* e_out, cudaStream_t s);

// tmap: host copy of the table's CUtensorMap (128 bytes), or null when p.use_tma == 0.
// The move kernel is compiled once per CTA width (p.nt); these dispatch on it.
template <typename T>
cudaError_t launch_move(const Params& p, int mode, const void* tmap, cudaStream_t s);
int stencil_tma_bytes(const Params& p, int elem_bytes);
// Several crowds in one launch: crowd c owns CTAs [base[c], base[c+1]).
constexpr int MAX_BATCH = 8;
struct BatchArgs {
  CUtensorMap maps[MAX_BATCH];  // each crowd's table map (unused where use_tma == 0)
  int base[MAX_BATCH + 1];
  int n;
};

#define QMCGB_DECLARE_MOVE_WIDTH(NS)                                                      \
  namespace NS {                                                                        \
  template <typename T>                                                                 \
  cudaError_t launch_move(const Params& p, int mode, const void* tmap, cudaStream_t s); \
  template <typename T>                                                                 \
  cudaError_t launch_batch(const Params* d_plist, const BatchArgs& a, int update,       \
                           size_t bytes, cudaStream_t s);                              \
  size_t move_smem_bytes(const Params& p, int elem_bytes);                              \
  }
QMCGB_DECLARE_MOVE_WIDTH(nt128)
QMCGB_DECLARE_MOVE_WIDTH(nt160)
QMCGB_DECLARE_MOVE_WIDTH(nt256)
#undef QMCGB_DECLARE_MOVE_WIDTH
// walkers [w0, w0 + count) (count < 0: through p.W)
template <typename T>
cudaError_t launch_eval_rows(const Params& p, cudaStream_t s, int w0 = 0, int count = -1);
template <typename T>
cudaError_t launch_recompute(const Params& p, double* ws, cudaStream_t s, int w0 = 0,
                             int count = -1);
template <typename T>
cudaError_t launch_pad_table(const Params& p, const void* src, int src_f32, int n_orb,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_jastrow_U(const Params& p, double* U, cudaStream_t s);
cudaError_t launch_wrap_positions(double* R, size_t n3, double L, int* status, cudaStream_t s);
// adds the nonlocal pseudopotential term to eloc[0..W) (nothing when p.nl_n == 0);
// partial: scratch of W * nlpp_partials_per_walker() doubles
template <typename T>
cudaError_t launch_nlpp(const Params& p, double* eloc, double* partial, cudaStream_t s);
int nlpp_partials_per_walker();
// adds the Ewald Coulomb energy to eloc[0..W) (nothing when p.coul == 0)
template <typename T>
cudaError_t launch_ewald(const Params& p, double* eloc, cudaStream_t s);
int ewald_max_vectors();

}  // namespace qmcgb

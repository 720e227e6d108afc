// Crowd runtime behind the C ABI of include/qmcgb.h: device state of a crowd of walkers
// (arXiv:2209.14487, Sec. III "crowd"), its stream, the generation counter of the
// counter-based RNG and the FP64 recompute cadence.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/qmcgb.h"
#include "qmc_internal.h"

using qmcgb::Params;

namespace qmcgb {

// bytes of one stencil copy: the whole 4x4x4 x n_pad stencil, or one ring box
int stencil_tma_bytes(const Params& p, int elem_bytes) {
  return p.use_tma == 2 ? RING_ORB * 16 * elem_bytes : 64 * p.n_pad * elem_bytes;
}

size_t move_smem_bytes(const Params& p, int elem_bytes) {
  if (p.nt == 128) return nt128::move_smem_bytes(p, elem_bytes);
  if (p.nt == 160) return nt160::move_smem_bytes(p, elem_bytes);
  return nt256::move_smem_bytes(p, elem_bytes);
}

template <typename T>
cudaError_t launch_move(const Params& p, int mode, const void* tmap, cudaStream_t s) {
  if (p.nt == 128) return nt128::launch_move<T>(p, mode, tmap, s);
  if (p.nt == 160) return nt160::launch_move<T>(p, mode, tmap, s);
  return nt256::launch_move<T>(p, mode, tmap, s);
}

template <typename T>
cudaError_t launch_batch(int nt, const Params* d_plist, const BatchArgs& a, int update,
                         size_t bytes, cudaStream_t s) {
  if (nt == 128) return nt128::launch_batch<T>(d_plist, a, update, bytes, s);
  if (nt == 160) return nt160::launch_batch<T>(d_plist, a, update, bytes, s);
  return nt256::launch_batch<T>(d_plist, a, update, bytes, s);
}

// Advances the generation counter of every crowd of a batch (after its move launch).
__global__ void batch_advance_kernel(Params* plist, int n) {
  if ((int)threadIdx.x < n) plist[threadIdx.x].gen += 1u;
}

int max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

}  // namespace qmcgb

struct qmc_crowd {
  qmc_system_desc sys;
  qmc_run_desc run;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int es = 8;  // bytes per element of the crowd's precision
  Params p{};
  // device buffers
  double* d_R = nullptr;
  void* d_rows = nullptr;
  void* d_binv = nullptr;
  double* d_logdet = nullptr;
  int* d_sign = nullptr;
  void* d_table = nullptr;
  void* d_jc = nullptr;
  double* d_ions = nullptr;
  int* d_win_m = nullptr;
  int* d_win_P = nullptr;
  void* d_win_V = nullptr;
  void* d_win_S = nullptr;
  void* d_pend_phi = nullptr;
  void* d_jgl = nullptr;        // [W][N][4] incremental Jastrow grad/lap, carried over sweeps
  void* d_flush = nullptr;      // [W][3][k][n] tensor-core flush scratch
  // DMC: the other half of the walker-state double buffer and the branching scratch
  double* d_R2 = nullptr;
  void* d_rows2 = nullptr;
  void* d_binv2 = nullptr;
  void* d_jgl2 = nullptr;
  double* d_nlpart = nullptr;   // [capacity][splits] partial sums of the nonlocal term
  int* d_coul_m = nullptr;      // Ewald reciprocal vectors and their coefficients
  double* d_coul_c = nullptr;
  double* d_logdet2 = nullptr;
  int* d_sign2 = nullptr;
  int* d_jvalid2 = nullptr;
  int* d_mult = nullptr;        // [cap]
  int* d_src = nullptr;         // [cap]
  int* d_bout = nullptr;        // [2]
  double* d_bsums = nullptr;    // [2]
  double* d_e = nullptr;        // [3][cap]: E_prev, E_new staging, gathered E
  int* d_jvalid = nullptr;      // [W]
  double* d_pend = nullptr;
  double* d_ws = nullptr;
  double* d_eloc = nullptr;     // [eloc_cap][W]
  int eloc_cap = 0;
  unsigned long long* d_nacc = nullptr;
  int* d_status = nullptr;
  float* d_guard = nullptr;     // [cap] inverse-guard probe of each walker's last sweep
  unsigned long long* d_nrep = nullptr;  // [2] guard repairs: since creation, this call
  uint8_t* d_trace = nullptr;   // [cap][N] accept decisions of the last sweep generation
  double* d_io = nullptr;       // staging for host I/O, 12 W doubles
  uint8_t* d_io8 = nullptr;     // 2 W bytes
  // host state
  int K2 = 0, K1 = 0;
  double rc2 = 1.0, rc1 = 1.0;
  std::vector<double> c_uu, c_ud, c_1;
  bool has_orbitals = false, has_positions = false, stale = true;
  uint32_t gen = 0;
  unsigned long long launches = 0;
  int test_no_copy = 0;             // failure-detection test hook (stencil copies not issued)
  int test_bad_cell = 0;            // checked-build test hook (a planted out-of-range cell)
  CUtensorMap tmap;  // (128-byte aligned type) the padded table as a 4-D tensor, for the stencil copy
  size_t smem = 0;               // dynamic shared memory of the move kernel
};

namespace {

// Default bound of the mixed path's inverse guard, max_k |(v^T (A B - I))_k| after a
// sweep: above the largest value of healthy walkers measured at n = 64, 256 and 768
// (6.5e-5, 1.5e-2, 2.4e-3), below those of drifted inverses (0.19 and more).
constexpr double kGuardTolDefault = 0.1;

// The last CUDA error a call of this thread returned as QMC_ERR_CUDA.
thread_local cudaError_t g_last_cuda = cudaSuccess;

int cuda_fail(cudaError_t e) {
  g_last_cuda = e;
  return QMC_ERR_CUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_);   \
  } while (0)

// An NVTX range named after the C-ABI call for the call's duration (a profiler's timeline
// shows every call and the kernels it launched; without a tool attached it costs a few
// nanoseconds).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define QMC_RANGE() NvtxRange qmc_range_(__func__)

bool is_mixed(const qmc_crowd* c) { return c->run.precision == QMC_PREC_MIXED; }

bool all_finite(const double* x, size_t n) {
  for (size_t e = 0; e < n; ++e)
    if (!std::isfinite(x[e])) return false;
  return true;
}

int dmalloc(void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return QMC_ERR_OOM;
  }
  return QMC_OK;
}

void free_all(qmc_crowd* c) {
  void* ptrs[] = {c->d_R, c->d_rows, c->d_binv, c->d_logdet, c->d_sign, c->d_table,
                  c->d_jc, c->d_ions, c->d_win_m, c->d_win_P, c->d_win_V, c->d_win_S,
                  c->d_pend_phi, c->d_pend, c->d_ws, c->d_eloc, c->d_nacc, c->d_status,
                  c->d_io, c->d_io8, c->d_jgl, c->d_jvalid, c->d_flush, c->d_R2,
                  c->d_rows2, c->d_binv2, c->d_jgl2, c->d_logdet2, c->d_sign2, c->d_jvalid2,
                  c->d_mult, c->d_src, c->d_bout, c->d_bsums, c->d_e, c->d_coul_m,
                  c->d_coul_c, c->d_nlpart, c->d_guard, c->d_nrep, c->d_trace};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

void sync_params(qmc_crowd* c) {
  Params& p = c->p;
  p.R = c->d_R;
  p.rows = c->d_rows;
  p.binv = c->d_binv;
  p.logdet = c->d_logdet;
  p.sign = c->d_sign;
  p.table = c->d_table;
  p.jc = c->d_jc;
  p.ions = c->d_ions;
  p.win_m = c->d_win_m;
  p.win_P = c->d_win_P;
  p.win_V = c->d_win_V;
  p.win_S = c->d_win_S;
  p.pend_phi = c->d_pend_phi;
  p.jgl = c->d_jgl;
  p.flush_scratch = c->d_flush;
  p.jvalid = c->d_jvalid;
  p.pend = c->d_pend;
  p.status = c->d_status;
  // d_status holds four ints: the status bits, then the checked build's 8-byte record
  p.check_info = reinterpret_cast<unsigned long long*>(c->d_status + 2);
  p.n_accept = c->d_nacc;
  p.guard_val = c->d_guard;
  p.n_repair = c->d_nrep;
  p.lu_ws = c->d_ws;
  p.accept_trace = c->d_trace;
  p.test_no_copy = c->test_no_copy;
  p.test_bad_cell = c->test_bad_cell;
  p.K2 = c->K2;
  p.K1 = (c->K1 > 0 && c->sys.n_ions > 0) ? c->K1 : 0;
  p.rc2 = c->rc2;
  p.rc1 = c->rc1;
  p.h2inv = c->K2 > 0 ? c->K2 / c->rc2 : 1.0;
  p.h1inv = c->K1 > 0 ? c->K1 / c->rc1 : 1.0;
  p.gen = c->gen;
  p.iel = 0;
  p.rnew_in = nullptr;
  p.ratio_out = p.grad_out = p.logratio_out = p.rnew_out = nullptr;
  p.accept_in = nullptr;
  p.accept_out = nullptr;
  p.eloc_out = nullptr;
}

int launch_status(qmc_crowd* c, cudaError_t e) {
  ++c->launches;
  return e == cudaSuccess ? QMC_OK : cuda_fail(e);
}

int gather_population(qmc_crowd* c, int n_new, const double* e_in, double* e_out);

int move(qmc_crowd* c, int mode) {
  const void* tm = c->p.use_tma ? (const void*)&c->tmap : nullptr;
  if (is_mixed(c)) return launch_status(c, qmcgb::launch_move<float>(c->p, mode, tm, c->stream));
  return launch_status(c, qmcgb::launch_move<double>(c->p, mode, tm, c->stream));
}

// Adds the nonlocal pseudopotential and Ewald Coulomb terms to the E_L the last launch
// wrote to p.eloc_out.
int add_nlpp(qmc_crowd* c) {
  if (!c->p.eloc_out) return QMC_OK;
  int st = QMC_OK;
  if (c->p.nl_n > 0 && c->p.n_ions > 0) {
    if (is_mixed(c))
      st = launch_status(c, qmcgb::launch_nlpp<float>(c->p, c->p.eloc_out, c->d_nlpart, c->stream));
    else
      st = launch_status(c, qmcgb::launch_nlpp<double>(c->p, c->p.eloc_out, c->d_nlpart, c->stream));
    if (st) return st;
  }
  if (c->p.coul) {
    if (is_mixed(c)) st = launch_status(c, qmcgb::launch_ewald<float>(c->p, c->p.eloc_out, c->stream));
    else st = launch_status(c, qmcgb::launch_ewald<double>(c->p, c->p.eloc_out, c->stream));
  }
  return st;
}

// The padded table [GP][GP][GP][n_pad] (x slowest) as a 4-D tensor, innermost first, with
// a box of one full 4x4x4 stencil (one copy per move lands it in shared memory), or for
// the ring a box of RING_ORB orbitals x 4 x 4 x 1 (a box is at most 256 elements wide;
// where it passes n_pad the copy fills zeros).
bool encode_table_map(qmc_crowd* c) {
  const Params& p = c->p;
  const cuuint64_t es = (cuuint64_t)c->es;
  const cuuint64_t GP = (cuuint64_t)p.GP, np = (cuuint64_t)p.n_pad;
  cuuint64_t dims[4] = {np, GP, GP, GP};
  cuuint64_t strides[3] = {np * es, GP * np * es, GP * GP * np * es};  // bytes, dims 1..3
  cuuint32_t box[4] = {(cuuint32_t)np, 4, 4, 4};
  if (p.use_tma == 2) {
    box[0] = (cuuint32_t)qmcgb::RING_ORB;
    box[3] = 1;
  }
  cuuint32_t estr[4] = {1, 1, 1, 1};
  std::memset(&c->tmap, 0, sizeof(c->tmap));
  // the driver's encoder, looked up at run time so the library needs no driver at link
  // or load time (hosts without a GPU still load it); looked up once, thread-safely
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      fn = nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }();
  if (!encode) return false;
  CUresult r = encode(
      &c->tmap, is_mixed(c) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
      c->d_table, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int read_status(qmc_crowd* c) {
  int st = 0;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) CK(cudaMemset(c->d_status, 0, sizeof(int)));
  // a generation cut short by a timed-out wait may have updated rows and inverses of
  // moves whose positions it did not store: everything is rebuilt from the positions
  if (st & qmcgb::ST_TIMEOUT) c->stale = true;
  // a failed bounds check (checked build) skipped accesses: nothing of the state is trusted
  if (st & qmcgb::ST_BOUNDS) {
    c->stale = true;
    return QMC_ERR_BOUNDS;
  }
  if (st & qmcgb::ST_SINGULAR) return QMC_ERR_SINGULAR;
  if (st & qmcgb::ST_NAN) return QMC_ERR_NAN;
  if (st & qmcgb::ST_STATE) return QMC_ERR_STATE;
  if (st & qmcgb::ST_TIMEOUT) return QMC_ERR_TIMEOUT;
  return QMC_OK;
}

int upload_jastrow(qmc_crowd* c) {
  const int K2 = c->K2, K1 = c->K1;
  std::vector<double> h((size_t)2 * (K2 + 3) + K1 + 3, 0.0);
  for (int m = 0; m < K2; ++m) {
    h[m] = m < (int)c->c_uu.size() ? c->c_uu[m] : 0.0;
    h[K2 + 3 + m] = m < (int)c->c_ud.size() ? c->c_ud[m] : 0.0;
  }
  for (int m = 0; m < K1; ++m) h[2 * (K2 + 3) + m] = c->c_1[m];
  if (is_mixed(c)) {
    std::vector<float> f(h.begin(), h.end());
    CK(cudaMemcpyAsync(c->d_jc, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else {
    CK(cudaMemcpyAsync(c->d_jc, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  sync_params(c);
  return QMC_OK;
}

int rebuild(qmc_crowd* c) {
  sync_params(c);
  int st;
  if (is_mixed(c)) st = launch_status(c, qmcgb::launch_eval_rows<float>(c->p, c->stream));
  else st = launch_status(c, qmcgb::launch_eval_rows<double>(c->p, c->stream));
  if (st) return st;
  if (is_mixed(c)) st = launch_status(c, qmcgb::launch_recompute<float>(c->p, c->d_ws, c->stream));
  else st = launch_status(c, qmcgb::launch_recompute<double>(c->p, c->d_ws, c->stream));
  if (st) return st;
  CK(cudaMemsetAsync(c->d_pend, 0, sizeof(double) * c->run.n_walkers * qmcgb::PEND_STRIDE,
                     c->stream));
  CK(cudaMemsetAsync(c->d_jvalid, 0, sizeof(int) * c->run.n_walkers, c->stream));
  c->stale = false;
  return QMC_OK;
}

int ensure_ready(qmc_crowd* c) {
  if (!c->has_orbitals || !c->has_positions) return QMC_ERR_STATE;
  if (c->stale) {
    int st = rebuild(c);
    if (st) return st;
  }
  sync_params(c);
  return QMC_OK;
}

int check_iel(const qmc_crowd* c, int iel) {
  return (iel >= 0 && iel < c->p.N) ? QMC_OK : QMC_ERR_INVALID_ARG;
}

}  // namespace

extern "C" {

const char* qmc_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda); }

const char* qmc_status_string(int status) {
  switch (status) {
    case QMC_OK: return "ok";
    case QMC_ERR_INVALID_ARG: return "invalid argument";
    case QMC_ERR_OOM: return "device out of memory";
    case QMC_ERR_CUDA: return "CUDA runtime error";
    case QMC_ERR_SINGULAR: return "singular Slater matrix";
    case QMC_ERR_TIMEOUT: return "bounded device wait ran out";
    case QMC_ERR_NAN: return "non-finite ratio or local energy";
    case QMC_ERR_STATE: return "call out of order or missing input";
    case QMC_ERR_UNSUPPORTED: return "size or option not supported by this build";
    case QMC_ERR_BOUNDS: return "device bounds check failed (checked build)";
    default: return "unknown status";
  }
}

int qmc_build_flags(void) { return QMCGB_CHECK ? QMC_BUILD_CHECKED : 0; }

int qmc_check_report(qmc_crowd* c, int* site, long long* value) {
  QMC_RANGE();
  if (!c || !site) return QMC_ERR_INVALID_ARG;
  unsigned long long rec = 0;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(&rec, c->p.check_info, sizeof(rec), cudaMemcpyDeviceToHost));
  if (rec) CK(cudaMemset(c->p.check_info, 0, sizeof(rec)));
  *site = (int)(rec >> 56);
  if (value) {
    const long long v = (long long)(rec & ((1ull << 56) - 1));
    *value = v >= (1ll << 55) ? v - (1ll << 56) : v;  // sign of the 56-bit field
  }
  return QMC_OK;
}

int qmc_crowd_create(const qmc_system_desc* sys, const qmc_run_desc* run, void* cuda_stream,
                     qmc_crowd** out) {
  QMC_RANGE();
  if (!sys || !run || !out) return QMC_ERR_INVALID_ARG;
  *out = nullptr;
  if (sys->n_up < 1 || sys->n_dn < 0 || sys->n_orb < sys->n_up || sys->n_ions < 0 ||
      sys->grid < 4 || !(sys->L > 0.0) || run->n_walkers < 1 || !(run->tau > 0.0))
    return QMC_ERR_INVALID_ARG;
  if (run->precision != QMC_PREC_FP64 && run->precision != QMC_PREC_MIXED)
    return QMC_ERR_INVALID_ARG;
  if (run->update != QMC_UPDATE_SM && run->update != QMC_UPDATE_DELAYED)
    return QMC_ERR_INVALID_ARG;
  if (run->update == QMC_UPDATE_DELAYED &&
      (run->delay_rank < 0 || run->delay_rank > qmcgb::MAX_K))  // 0: the library picks k
    return QMC_ERR_INVALID_ARG;
  if (run->n_recompute < 0) return QMC_ERR_INVALID_ARG;
  if (run->staging != QMC_STAGING_AUTO && run->staging != QMC_STAGING_LDG)
    return QMC_ERR_INVALID_ARG;
  if (run->cta_threads != 0 && run->cta_threads != 128 && run->cta_threads != 160 &&
      run->cta_threads != 256)
    return QMC_ERR_INVALID_ARG;
  if (run->engine != QMC_ENGINE_AUTO && run->engine != QMC_ENGINE_SIMT) return QMC_ERR_INVALID_ARG;
  if (std::isnan(run->guard_tol)) return QMC_ERR_INVALID_ARG;
  if (run->drift < 0 || run->drift > 2) return QMC_ERR_INVALID_ARG;
  if (sys->n_dn != sys->n_up) return QMC_ERR_UNSUPPORTED;
  if (sys->n_up > 1024 || sys->grid > 1024) return QMC_ERR_UNSUPPORTED;

  qmc_crowd* c = new qmc_crowd();
  c->sys = *sys;
  c->run = *run;
  c->es = run->precision == QMC_PREC_MIXED ? 4 : 8;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return QMC_ERR_CUDA;
    }
    c->own_stream = true;
  }
  Params& p = c->p;
  const int W = run->n_walkers, n = sys->n_up, N = sys->n_up + sys->n_dn;
  p.W = W;
  p.N = N;
  p.n_up = sys->n_up;
  p.n = n;
  p.n_pad = (n + 7) & ~7;
  p.nt = run->cta_threads ? run->cta_threads : (n <= 128 ? 128 : 256);
  // incremental Jastrow gradients and Laplacians in the mixed Sherman-Morrison sweep
  p.inc_jastrow = (run->precision == QMC_PREC_MIXED && run->update == QMC_UPDATE_SM &&
                   2 * n <= p.nt && n % 8 == 0) ? 1 : 0;
  p.n_ions = sys->n_ions;
  p.G = sys->grid;
  p.GP = sys->grid + 3;
  p.drift = run->drift;
  p.dmc = run->dmc ? 1 : 0;
  p.potential = run->potential ? 1 : 0;
  p.update = run->update;
  p.k = run->update == QMC_UPDATE_DELAYED ? run->delay_rank : 1;
  p.vs = n + 1;
  p.ks = p.k + 1;
  p.L = sys->L;
  p.invL = 1.0 / sys->L;
  p.tau = run->tau;
  p.sqrt_tau = std::sqrt(run->tau);
  p.dgrid = sys->grid / sys->L;
  p.fx_scale = 4294967296.0 / sys->L;
  p.fx_unit = sys->L / 4294967296.0;
  p.seed = run->seed;
  // inverse guard of the mixed path: on unless guard_tol < 0
  const bool guard = run->precision == QMC_PREC_MIXED && run->guard_tol >= 0.0;
  p.guard_tol = guard ? (float)(run->guard_tol > 0.0 ? run->guard_tol : kGuardTolDefault) : 0.0f;
  c->run.guard_tol = guard ? (double)p.guard_tol : -1.0;
  const int es = c->es;

  // Shared-memory plan, first that fits: the moving spin's inverse and the TMA-staged
  // stencil, the inverse alone, the stencil alone, neither.  A TMA box is at most 256
  // elements wide, so the staged stencil needs n_pad <= 256.
  const int optin = qmcgb::max_smem_optin();
  // n_pad > 256: the mixed path's ring of smaller boxes (128 threads: two orbitals of each
  // box per thread; the wider kernels are built without the ring's code, which cost them
  // registers)
  const bool ring_ok = run->precision == QMC_PREC_MIXED && p.nt == 128;
  const bool tma_ok = run->staging == QMC_STAGING_AUTO && (p.n_pad <= 256 || ring_ok);
  // The tensor-core flush (mixed delayed path, inverse in global memory, n % 4 == 0) adds
  // a 64 KB operand stage unless it can share the stencil buffer.
  // (its epilogue splits the four TMEM lane quadrants over groups of four warps, and
  // its operand stages over 128 or 256 threads)
  const bool tc_ok = run->engine == QMC_ENGINE_AUTO && run->precision == QMC_PREC_MIXED &&
                     run->update == QMC_UPDATE_DELAYED && n % 4 == 0 &&
                     (p.nt == 128 || p.nt == 256);
  const int plans[4][2] = {{1, 1}, {1, 0}, {0, 1}, {0, 0}};
  size_t smem = 0;
  if (run->layout < QMC_LAYOUT_AUTO || run->layout > QMC_LAYOUT_COMPACT) {
    delete c;
    return QMC_ERR_INVALID_ARG;
  }
  // Layouts to try: the caller's, else shared (every plan), then compact (the window's
  // rows in global memory and the draws computed per move) when no shared plan fits.
  const int lay_first = run->layout == QMC_LAYOUT_COMPACT ? 1 : 0;
  const int lay_last = run->layout == QMC_LAYOUT_SHARED ? 0 : 1;
  auto fits = [&]() -> bool {
    smem = qmcgb::move_smem_bytes(p, es);
    return optin <= 0 || smem <= (size_t)optin;
  };
  // the first plan that fits for delay rank k in the current layout
  auto place_plan = [&](int k) -> bool {
    p.k = k;
    p.ks = k + 1;
    for (const auto& pl : plans) {
      if (pl[1] && !tma_ok) continue;
      p.b_in_smem = pl[0];
      p.use_tma = pl[1] ? (p.n_pad <= 256 ? 1 : 2) : 0;
      p.tc_flush = (tc_ok && !pl[0]) ? 1 : 0;
      p.stencil_bytes = qmcgb::stencil_tma_bytes(p, es);
      if (fits()) return true;
    }
    if (tc_ok) {  // without the tensor-core stage
      for (const auto& pl : plans) {
        if (pl[0] || (pl[1] && !tma_ok)) continue;
        p.b_in_smem = 0;
        p.use_tma = pl[1] ? (p.n_pad <= 256 ? 1 : 2) : 0;
        p.tc_flush = 0;
        p.stencil_bytes = qmcgb::stencil_tma_bytes(p, es);
        if (fits()) return true;
      }
    }
    return false;
  };
  // the first layout and plan that fit (sets p.k, p.ks, p.compact and the plan's fields)
  auto place = [&](int k) -> bool {
    for (int cp = lay_first; cp <= lay_last; ++cp) {
      p.compact = cp;
      if (place_plan(k)) return true;
    }
    return false;
  };
  bool placed = false;
  if (run->update == QMC_UPDATE_DELAYED && run->delay_rank == 0) {
    // the library's pick (measured optima on GB300): the largest rank up to 32 that fits
    // with the inverse in global memory; 8 when the inverse fits in shared memory
    for (int k : {32, 16, 8, 4, 2, 1}) {
      if (place(k)) {
        placed = true;
        break;
      }
    }
    if (placed && p.k > 8 && p.b_in_smem) placed = place(8);
    c->run.delay_rank = p.k;
  } else {
    placed = place(p.k);
  }
  if (!placed) {
    delete c;
    return QMC_ERR_UNSUPPORTED;
  }
  // the incremental sweep pipelines proposals and reads the draw table the compact layout
  // leaves out: a compact crowd takes the plain sweep (and its smaller layout)
  if (p.compact && p.inc_jastrow) {
    p.inc_jastrow = 0;
    smem = qmcgb::move_smem_bytes(p, es);
  }
  // TMEM: a flush holds 128 of the SM's 512 columns while it runs; a CTA whose
  // allocation finds them taken waits for another CTA's flush to end
  c->smem = smem;

  const size_t GP = (size_t)p.GP;
  int st = QMC_OK;
  st |= dmalloc((void**)&c->d_R, sizeof(double) * W * N * 3);
  st |= dmalloc(&c->d_rows, (size_t)es * W * N * 5 * p.n_pad);
  st |= dmalloc(&c->d_binv, (size_t)es * W * 2 * n * n);
  st |= dmalloc((void**)&c->d_logdet, sizeof(double) * W * 2);
  st |= dmalloc((void**)&c->d_sign, sizeof(int) * W * 2);
  st |= dmalloc(&c->d_table, (size_t)es * GP * GP * GP * p.n_pad);
  st |= dmalloc(&c->d_jc, sizeof(double) * (3 * (qmcgb::MAX_KNOTS + 3)));
  st |= dmalloc((void**)&c->d_ions, sizeof(double) * 3 * (sys->n_ions > 0 ? sys->n_ions : 1));
  st |= dmalloc((void**)&c->d_win_m, sizeof(int) * W * 2);
  st |= dmalloc((void**)&c->d_win_P, sizeof(int) * W * 2 * qmcgb::MAX_K);
  if (p.update == QMC_UPDATE_DELAYED) {
    st |= dmalloc(&c->d_win_V, (size_t)es * W * 2 * p.k * p.vs);
    st |= dmalloc(&c->d_win_S, (size_t)es * W * 2 * p.k * p.ks);
  }
  st |= dmalloc(&c->d_pend_phi, (size_t)es * W * 5 * p.n_pad);
  st |= dmalloc(&c->d_jgl, (size_t)es * W * N * 4);
  if (p.tc_flush) st |= dmalloc(&c->d_flush, (size_t)es * W * 3 * p.k * n);
  if (run->dmc) {
    st |= dmalloc((void**)&c->d_R2, sizeof(double) * W * N * 3);
    st |= dmalloc(&c->d_rows2, (size_t)es * W * N * 5 * p.n_pad);
    st |= dmalloc(&c->d_binv2, (size_t)es * W * 2 * n * n);
    st |= dmalloc(&c->d_jgl2, (size_t)es * W * N * 4);
    st |= dmalloc((void**)&c->d_logdet2, sizeof(double) * W * 2);
    st |= dmalloc((void**)&c->d_sign2, sizeof(int) * W * 2);
    st |= dmalloc((void**)&c->d_jvalid2, sizeof(int) * W);
    st |= dmalloc((void**)&c->d_mult, sizeof(int) * W);
    st |= dmalloc((void**)&c->d_src, sizeof(int) * W);
    st |= dmalloc((void**)&c->d_bout, sizeof(int) * 2);
    st |= dmalloc((void**)&c->d_bsums, sizeof(double) * 2);
    st |= dmalloc((void**)&c->d_e, sizeof(double) * 3 * W);
  }
  st |= dmalloc((void**)&c->d_jvalid, sizeof(int) * W);
  st |= dmalloc((void**)&c->d_pend, sizeof(double) * W * qmcgb::PEND_STRIDE);
  st |= dmalloc((void**)&c->d_ws, sizeof(double) * W * 2 * 2 * n * n);
  st |= dmalloc((void**)&c->d_nacc, sizeof(unsigned long long));
  st |= dmalloc((void**)&c->d_status, 4 * sizeof(int));
  if (guard) {
    st |= dmalloc((void**)&c->d_guard, sizeof(float) * W);
    st |= dmalloc((void**)&c->d_nrep, sizeof(unsigned long long) * 2);
  }
  st |= dmalloc((void**)&c->d_io, sizeof(double) * 12 * W);
  st |= dmalloc((void**)&c->d_io8, 2 * (size_t)W);
  if (st) {
    free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return QMC_ERR_OOM;
  }
  cudaMemsetAsync(c->d_win_m, 0, sizeof(int) * W * 2, c->stream);
  cudaMemsetAsync(c->d_jvalid, 0, sizeof(int) * W, c->stream);
  cudaMemsetAsync(c->d_pend, 0, sizeof(double) * W * qmcgb::PEND_STRIDE, c->stream);
  cudaMemsetAsync(c->d_nacc, 0, sizeof(unsigned long long), c->stream);
  cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int), c->stream);
  if (guard) {
    cudaMemsetAsync(c->d_guard, 0, sizeof(float) * W, c->stream);
    cudaMemsetAsync(c->d_nrep, 0, sizeof(unsigned long long) * 2, c->stream);
  }
  cudaMemsetAsync(c->d_table, 0, (size_t)es * GP * GP * GP * p.n_pad, c->stream);
  cudaMemsetAsync(c->d_logdet, 0, sizeof(double) * W * 2, c->stream);
  cudaMemsetAsync(c->d_sign, 0, sizeof(int) * W * 2, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return QMC_ERR_CUDA;
  }
  if (p.use_tma && !encode_table_map(c)) {  // plain loads then, if they fit
    p.use_tma = 0;
    p.stencil_bytes = 0;
    c->smem = qmcgb::move_smem_bytes(p, c->es);
    if (qmcgb::max_smem_optin() > 0 && c->smem > (size_t)qmcgb::max_smem_optin()) {
      free_all(c);
      if (c->own_stream) cudaStreamDestroy(c->stream);
      delete c;
      return QMC_ERR_UNSUPPORTED;
    }
  }
  sync_params(c);
  int js = upload_jastrow(c);
  if (js) {
    free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return js;
  }
  *out = c;
  return QMC_OK;
}

int qmc_crowd_destroy(qmc_crowd* c) {
  QMC_RANGE();
  if (!c) return QMC_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return QMC_OK;
}

int qmc_load_positions(qmc_crowd* c, const double* R, int mem) {
  QMC_RANGE();
  if (!c || !R) return QMC_ERR_INVALID_ARG;
  const size_t n3 = (size_t)c->p.W * c->p.N * 3;
  if (mem == QMC_MEM_HOST && !all_finite(R, n3)) return QMC_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(c->d_R, R, n3 * sizeof(double),
                     mem == QMC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->stream));
  int st = launch_status(c, qmcgb::launch_wrap_positions(c->d_R, n3, c->p.L, c->d_status,
                                                         c->stream));
  if (st) return st;
  if (mem == QMC_MEM_HOST) CK(cudaStreamSynchronize(c->stream));
  c->has_positions = true;
  c->stale = true;
  return QMC_OK;
}

int qmc_load_ions(qmc_crowd* c, const double* RI) {
  QMC_RANGE();
  if (!c) return QMC_ERR_INVALID_ARG;
  if (c->sys.n_ions == 0) return QMC_OK;
  if (!RI || !all_finite(RI, 3 * (size_t)c->sys.n_ions)) return QMC_ERR_INVALID_ARG;
  std::vector<double> h(RI, RI + 3 * c->sys.n_ions);
  for (double& x : h) x = x - c->p.L * std::floor(x / c->p.L);
  CK(cudaMemcpyAsync(c->d_ions, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->stale = true;
  return QMC_OK;
}

int qmc_load_orbitals(qmc_crowd* c, const void* coefs, int dtype, int mem) {
  QMC_RANGE();
  if (!c || !coefs) return QMC_ERR_INVALID_ARG;
  if (dtype != QMC_DTYPE_F64 && dtype != QMC_DTYPE_F32) return QMC_ERR_INVALID_ARG;
  const size_t G = (size_t)c->p.G;
  const size_t bytes = G * G * G * (size_t)c->sys.n_orb * (dtype == QMC_DTYPE_F32 ? 4 : 8);
  const void* src = coefs;
  void* tmp = nullptr;
  if (mem == QMC_MEM_HOST) {
    if (dmalloc(&tmp, bytes)) return QMC_ERR_OOM;
    if (cudaMemcpyAsync(tmp, coefs, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
      cudaFree(tmp);
      return QMC_ERR_CUDA;
    }
    src = tmp;
  }
  sync_params(c);
  cudaError_t e;
  if (is_mixed(c))
    e = qmcgb::launch_pad_table<float>(c->p, src, dtype == QMC_DTYPE_F32, c->sys.n_orb, c->stream);
  else
    e = qmcgb::launch_pad_table<double>(c->p, src, dtype == QMC_DTYPE_F32, c->sys.n_orb, c->stream);
  ++c->launches;
  cudaError_t e2 = cudaStreamSynchronize(c->stream);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e);
  if (e2 != cudaSuccess) return cuda_fail(e2);
  c->has_orbitals = true;
  c->stale = true;
  return QMC_OK;
}

int qmc_load_jastrow(qmc_crowd* c, int kind, const double* coefs, int K, double rc) {
  QMC_RANGE();
  if (!c) return QMC_ERR_INVALID_ARG;
  if (K < 0 || K > qmcgb::MAX_KNOTS || (K > 0 && (!coefs || !(rc > 0.0))))
    return QMC_ERR_INVALID_ARG;
  std::vector<double> v(coefs ? coefs : nullptr, coefs ? coefs + K : nullptr);
  if (kind == QMC_J1) {
    c->K1 = K;
    c->rc1 = K > 0 ? rc : 1.0;
    c->c_1 = v;
  } else if (kind == QMC_J2_UU || kind == QMC_J2_UD) {
    // like and unlike pair functors share one knot grid
    const bool other = kind == QMC_J2_UU ? !c->c_ud.empty() : !c->c_uu.empty();
    if (K > 0 && other && c->K2 > 0 && (K != c->K2 || rc != c->rc2)) return QMC_ERR_INVALID_ARG;
    if (kind == QMC_J2_UU) c->c_uu = v;
    else c->c_ud = v;
    if (K > 0) {
      c->K2 = K;
      c->rc2 = rc;
    } else if (c->c_uu.empty() && c->c_ud.empty()) {
      c->K2 = 0;
    }
  } else {
    return QMC_ERR_INVALID_ARG;
  }
  c->stale = true;
  return upload_jastrow(c);
}

int qmc_recompute(qmc_crowd* c) {
  QMC_RANGE();
  if (!c) return QMC_ERR_INVALID_ARG;
  if (!c->has_orbitals || !c->has_positions) return QMC_ERR_STATE;
  int st = rebuild(c);
  if (st) return st;
  return read_status(c);
}

int qmc_eval_grad_batch(qmc_crowd* c, int iel, double* grad, int mem) {
  QMC_RANGE();
  if (!c || !grad) return QMC_ERR_INVALID_ARG;
  if (check_iel(c, iel)) return QMC_ERR_INVALID_ARG;
  int st = ensure_ready(c);
  if (st) return st;
  c->p.iel = iel;
  c->p.grad_out = mem == QMC_MEM_DEVICE ? grad : c->d_io;
  st = move(c, qmcgb::MODE_GRAD);
  if (st) return st;
  if (mem == QMC_MEM_HOST) {
    CK(cudaMemcpyAsync(grad, c->d_io, sizeof(double) * 3 * c->p.W, cudaMemcpyDeviceToHost,
                       c->stream));
    return read_status(c);
  }
  return QMC_OK;
}

int qmc_propose_move_batch(qmc_crowd* c, int iel, const double* rnew, double* ratio,
                           double* grad, double* log_ratio, double* rnew_out, int mem) {
  QMC_RANGE();
  if (!c) return QMC_ERR_INVALID_ARG;
  if (check_iel(c, iel)) return QMC_ERR_INVALID_ARG;
  int st = ensure_ready(c);
  if (st) return st;
  const int W = c->p.W;
  Params& p = c->p;
  p.iel = iel;
  if (mem == QMC_MEM_DEVICE) {
    p.rnew_in = rnew;
    p.ratio_out = ratio;
    p.grad_out = grad;
    p.logratio_out = log_ratio;
    p.rnew_out = rnew_out;
  } else {
    double* io = c->d_io;
    if (rnew) {
      CK(cudaMemcpyAsync(io + 9 * W, rnew, sizeof(double) * 3 * W, cudaMemcpyHostToDevice,
                         c->stream));
      p.rnew_in = io + 9 * W;
    }
    p.ratio_out = io;
    p.logratio_out = io + W;
    p.grad_out = io + 2 * W;
    p.rnew_out = io + 5 * W;
  }
  st = move(c, qmcgb::MODE_PROPOSE);
  if (st) return st;
  if (mem == QMC_MEM_HOST) {
    const double* io = c->d_io;
    if (ratio) CK(cudaMemcpyAsync(ratio, io, sizeof(double) * W, cudaMemcpyDeviceToHost, c->stream));
    if (log_ratio)
      CK(cudaMemcpyAsync(log_ratio, io + W, sizeof(double) * W, cudaMemcpyDeviceToHost, c->stream));
    if (grad)
      CK(cudaMemcpyAsync(grad, io + 2 * W, sizeof(double) * 3 * W, cudaMemcpyDeviceToHost, c->stream));
    if (rnew_out)
      CK(cudaMemcpyAsync(rnew_out, io + 5 * W, sizeof(double) * 3 * W, cudaMemcpyDeviceToHost,
                         c->stream));
    return read_status(c);
  }
  return QMC_OK;
}

int qmc_accept_reject_batch(qmc_crowd* c, int iel, const uint8_t* accept, uint8_t* accepted_out,
                            int mem) {
  QMC_RANGE();
  if (!c) return QMC_ERR_INVALID_ARG;
  if (check_iel(c, iel)) return QMC_ERR_INVALID_ARG;
  if (!c->has_orbitals || !c->has_positions || c->stale) return QMC_ERR_STATE;
  sync_params(c);
  const int W = c->p.W;
  Params& p = c->p;
  p.iel = iel;
  if (mem == QMC_MEM_DEVICE) {
    p.accept_in = accept;
    p.accept_out = accepted_out;
  } else {
    if (accept) {
      CK(cudaMemcpyAsync(c->d_io8, accept, W, cudaMemcpyHostToDevice, c->stream));
      p.accept_in = c->d_io8;
    }
    p.accept_out = c->d_io8 + W;
  }
  int st = move(c, qmcgb::MODE_ACCEPT);
  if (st) return st;
  if (mem == QMC_MEM_HOST) {
    if (accepted_out)
      CK(cudaMemcpyAsync(accepted_out, c->d_io8 + W, W, cudaMemcpyDeviceToHost, c->stream));
    return read_status(c);
  }
  return QMC_OK;
}

int qmc_local_energy_batch(qmc_crowd* c, double* eloc, int mem) {
  QMC_RANGE();
  if (!c || !eloc) return QMC_ERR_INVALID_ARG;
  int st = ensure_ready(c);
  if (st) return st;
  c->p.eloc_out = mem == QMC_MEM_DEVICE ? eloc : c->d_io;
  st = move(c, qmcgb::MODE_ELOC);
  if (st) return st;
  st = add_nlpp(c);
  if (st) return st;
  if (mem == QMC_MEM_HOST) {
    CK(cudaMemcpyAsync(eloc, c->d_io, sizeof(double) * c->p.W, cudaMemcpyDeviceToHost, c->stream));
    return read_status(c);
  }
  return QMC_OK;
}

int qmc_sweep(qmc_crowd* c, int n_gen, double* eloc, int mem, qmc_stats* stats) {
  QMC_RANGE();
  if (!c || n_gen < 0) return QMC_ERR_INVALID_ARG;
  int st = ensure_ready(c);
  if (st) return st;
  const int W = c->p.W;
  const bool need_buf = stats || (eloc && mem == QMC_MEM_HOST);
  if (need_buf && c->eloc_cap < n_gen) {
    if (c->d_eloc) cudaFree(c->d_eloc);
    c->d_eloc = nullptr;
    c->eloc_cap = 0;
    if (dmalloc((void**)&c->d_eloc, sizeof(double) * (size_t)n_gen * W)) return QMC_ERR_OOM;
    c->eloc_cap = n_gen;
  }
  if (stats) CK(cudaMemsetAsync(c->d_nacc, 0, sizeof(unsigned long long), c->stream));
  if (stats && c->d_nrep)
    CK(cudaMemsetAsync(c->d_nrep + 1, 0, sizeof(unsigned long long), c->stream));
  for (int g = 0; g < n_gen; ++g) {
    sync_params(c);
    Params& p = c->p;
    if (eloc && mem == QMC_MEM_DEVICE) p.eloc_out = eloc + (size_t)g * W;
    else if (need_buf) p.eloc_out = c->d_eloc + (size_t)g * W;
    else p.eloc_out = nullptr;
    p.n_accept = stats ? c->d_nacc : nullptr;
    const bool due = c->run.n_recompute > 0 && ((c->gen + 1) % (uint32_t)c->run.n_recompute) == 0;
    if (!due) {
      st = move(c, qmcgb::MODE_SWEEP);
      if (st) return st;
    } else {
      st = move(c, qmcgb::MODE_SWEEP_NOE);
      if (st) return st;
      if (is_mixed(c)) st = launch_status(c, qmcgb::launch_recompute<float>(p, c->d_ws, c->stream));
      else st = launch_status(c, qmcgb::launch_recompute<double>(p, c->d_ws, c->stream));
      if (st) return st;
      if (p.eloc_out) {
        st = move(c, qmcgb::MODE_ELOC);
        if (st) return st;
      }
    }
    st = add_nlpp(c);
    if (st) return st;
    c->gen += 1;
  }
  if (eloc && mem == QMC_MEM_HOST)
    CK(cudaMemcpyAsync(eloc, c->d_eloc, sizeof(double) * (size_t)n_gen * W,
                       cudaMemcpyDeviceToHost, c->stream));
  if (stats) {
    std::vector<double> h((size_t)n_gen * W);
    CK(cudaMemcpyAsync(h.data(), c->d_eloc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    unsigned long long na = 0, nr = 0;
    CK(cudaMemcpyAsync(&na, c->d_nacc, sizeof(na), cudaMemcpyDeviceToHost, c->stream));
    if (c->d_nrep)
      CK(cudaMemcpyAsync(&nr, c->d_nrep + 1, sizeof(nr), cudaMemcpyDeviceToHost, c->stream));
    st = read_status(c);
    double s1 = 0.0, s2 = 0.0;
    for (double e : h) {
      s1 += e;
      s2 += e * e;
    }
    stats->e_sum = s1;
    stats->e2_sum = s2;
    stats->n_samples = (long long)h.size();
    stats->n_accept = (long long)na;
    stats->n_moves = (long long)n_gen * W * c->p.N;
    stats->n_repair = (long long)nr;
    return st;
  }
  if (eloc && mem == QMC_MEM_HOST) return read_status(c);
  return QMC_OK;
}

int qmc_get_positions(qmc_crowd* c, double* R, int mem) {
  QMC_RANGE();
  if (!c || !R) return QMC_ERR_INVALID_ARG;
  const size_t bytes = sizeof(double) * c->p.W * c->p.N * 3;
  CK(cudaMemcpyAsync(R, c->d_R, bytes,
                     mem == QMC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream));
  if (mem == QMC_MEM_HOST) CK(cudaStreamSynchronize(c->stream));
  return QMC_OK;
}

int qmc_get_logpsi(qmc_crowd* c, double* logabs, int* sign) {
  QMC_RANGE();
  if (!c || !logabs || !sign) return QMC_ERR_INVALID_ARG;
  int st = ensure_ready(c);
  if (st) return st;
  const int W = c->p.W;
  if (is_mixed(c)) st = launch_status(c, qmcgb::launch_jastrow_U<float>(c->p, c->d_io, c->stream));
  else st = launch_status(c, qmcgb::launch_jastrow_U<double>(c->p, c->d_io, c->stream));
  if (st) return st;
  std::vector<double> U(W), ld(2 * W);
  std::vector<int> sg(2 * W);
  CK(cudaMemcpyAsync(U.data(), c->d_io, sizeof(double) * W, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(ld.data(), c->d_logdet, sizeof(double) * 2 * W, cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaMemcpyAsync(sg.data(), c->d_sign, sizeof(int) * 2 * W, cudaMemcpyDeviceToHost,
                     c->stream));
  st = read_status(c);
  for (int w = 0; w < W; ++w) {
    logabs[w] = ld[2 * w] + ld[2 * w + 1] - U[w];
    sign[w] = sg[2 * w] * sg[2 * w + 1];
  }
  return st;
}

int qmc_get_inverse(qmc_crowd* c, int spin, double* out) {
  QMC_RANGE();
  if (!c || !out || (spin != 0 && spin != 1)) return QMC_ERR_INVALID_ARG;
  int st = ensure_ready(c);
  if (st) return st;
  st = move(c, qmcgb::MODE_FLUSH);
  if (st) return st;
  const int W = c->p.W, n = c->p.n, es = c->es;
  std::vector<unsigned char> h((size_t)es * W * 2 * n * n);
  CK(cudaMemcpyAsync(h.data(), c->d_binv, h.size(), cudaMemcpyDeviceToHost, c->stream));
  st = read_status(c);
  for (int w = 0; w < W; ++w)
    for (int l = 0; l < n; ++l)
      for (int j = 0; j < n; ++j) {
        const size_t src = (((size_t)w * 2 + spin) * n + l) * n + j;  // B^T[l][j]
        const double v = es == 4 ? (double)((const float*)h.data())[src]
                                 : ((const double*)h.data())[src];
        out[((size_t)w * n + j) * n + l] = v;
      }
  return st;
}

int qmc_get_slater_matrix(qmc_crowd* c, int spin, double* out) {
  QMC_RANGE();
  if (!c || !out || (spin != 0 && spin != 1)) return QMC_ERR_INVALID_ARG;
  int st = ensure_ready(c);
  if (st) return st;
  const int W = c->p.W, n = c->p.n, N = c->p.N, np = c->p.n_pad, es = c->es;
  std::vector<unsigned char> h((size_t)es * W * N * 5 * np);
  CK(cudaMemcpyAsync(h.data(), c->d_rows, h.size(), cudaMemcpyDeviceToHost, c->stream));
  st = read_status(c);
  for (int w = 0; w < W; ++w)
    for (int l = 0; l < n; ++l)
      for (int j = 0; j < n; ++j) {
        const size_t src = (((size_t)w * N + spin * c->p.n_up + l) * 5) * np + j;
        out[((size_t)w * n + l) * n + j] =
            es == 4 ? (double)((const float*)h.data())[src] : ((const double*)h.data())[src];
      }
  return st;
}

int qmc_get_generation(qmc_crowd* c, uint32_t* gen) {
  QMC_RANGE();
  if (!c || !gen) return QMC_ERR_INVALID_ARG;
  *gen = c->gen;
  return QMC_OK;
}

int qmc_set_generation(qmc_crowd* c, uint32_t gen) {
  QMC_RANGE();
  if (!c) return QMC_ERR_INVALID_ARG;
  c->gen = gen;
  return QMC_OK;
}

int qmc_get_kernel_config(const qmc_crowd* c, int* b_in_smem, int* stencil_tma, int* smem_bytes,
                          int* cta_threads, int* tc_flush, int* layout) {
  QMC_RANGE();
  if (!c) return QMC_ERR_INVALID_ARG;
  if (layout) *layout = c->p.compact ? QMC_LAYOUT_COMPACT : QMC_LAYOUT_SHARED;
  if (tc_flush) *tc_flush = c->p.tc_flush;
  if (cta_threads) *cta_threads = c->p.nt;
  if (b_in_smem) *b_in_smem = c->p.b_in_smem;
  if (stencil_tma) *stencil_tma = c->p.use_tma;
  if (smem_bytes) *smem_bytes = (int)c->smem;
  return QMC_OK;
}

int qmc_get_update(const qmc_crowd* c, int* update, int* delay_rank) {
  QMC_RANGE();
  if (!c || !update || !delay_rank) return QMC_ERR_INVALID_ARG;
  *update = c->run.update;
  *delay_rank = c->run.update == QMC_UPDATE_DELAYED ? c->run.delay_rank : 1;
  return QMC_OK;
}

int qmc_get_guard(qmc_crowd* c, double* values, long long* n_repair) {
  QMC_RANGE();
  if (!c) return QMC_ERR_INVALID_ARG;
  if (!c->d_guard) return QMC_ERR_STATE;
  const int W = c->p.W;
  std::vector<float> h(W);
  unsigned long long nr = 0;
  if (values)
    CK(cudaMemcpyAsync(h.data(), c->d_guard, sizeof(float) * W, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaMemcpyAsync(&nr, c->d_nrep, sizeof(nr), cudaMemcpyDeviceToHost, c->stream));
  const int st = read_status(c);
  if (values)
    for (int w = 0; w < W; ++w) values[w] = (double)h[w];
  if (n_repair) *n_repair = (long long)nr;
  return st;
}

int qmc_trace_accepts(qmc_crowd* c, int on) {
  QMC_RANGE();
  if (!c || (on != 0 && on != 1)) return QMC_ERR_INVALID_ARG;
  if (on && !c->d_trace) {
    CK(cudaStreamSynchronize(c->stream));
    if (dmalloc((void**)&c->d_trace, (size_t)c->run.n_walkers * c->p.N)) return QMC_ERR_OOM;
    CK(cudaMemsetAsync(c->d_trace, 0, (size_t)c->run.n_walkers * c->p.N, c->stream));
  } else if (!on && c->d_trace) {
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->d_trace);
    c->d_trace = nullptr;
  }
  sync_params(c);
  return QMC_OK;
}

int qmc_get_accept_trace(qmc_crowd* c, uint8_t* out) {
  QMC_RANGE();
  if (!c || !out) return QMC_ERR_INVALID_ARG;
  if (!c->d_trace) return QMC_ERR_STATE;
  CK(cudaMemcpyAsync(out, c->d_trace, (size_t)c->p.W * c->p.N, cudaMemcpyDeviceToHost,
                     c->stream));
  return read_status(c);
}

int qmc_test_skip_stencil_copy(qmc_crowd* c, int on) {
  QMC_RANGE();
  if (!c || (on != 0 && on != 1)) return QMC_ERR_INVALID_ARG;
  if (on && !c->p.use_tma) return QMC_ERR_INVALID_ARG;
  c->test_no_copy = on;
  sync_params(c);
  return QMC_OK;
}

int qmc_test_plant_bad_cell(qmc_crowd* c, int on) {
  QMC_RANGE();
  if (!c || (on != 0 && on != 1)) return QMC_ERR_INVALID_ARG;
  if (!QMCGB_CHECK) return QMC_ERR_UNSUPPORTED;  // only a checked kernel stops the access
  c->test_bad_cell = on;
  sync_params(c);
  return QMC_OK;
}

int qmc_get_walker_count(const qmc_crowd* c, int* count) {
  QMC_RANGE();
  if (!c || !count) return QMC_ERR_INVALID_ARG;
  *count = c->p.W;
  return QMC_OK;
}

int qmc_load_nlpp(qmc_crowd* c, int n_l, const double* amp, const double* width, double rc) {
  QMC_RANGE();
  if (!c || n_l < 0 || n_l > 3) return QMC_ERR_INVALID_ARG;
  if (n_l > 0) {
    if (!amp || !width || !(rc > 0.0) || rc > 0.5 * c->p.L) return QMC_ERR_INVALID_ARG;
    for (int l = 0; l < n_l; ++l)
      if (!(width[l] > 0.0) || !std::isfinite(amp[l])) return QMC_ERR_INVALID_ARG;
  }
  if (n_l > 0 && !c->d_nlpart &&
      dmalloc((void**)&c->d_nlpart, sizeof(double) * (size_t)c->run.n_walkers *
                                        qmcgb::nlpp_partials_per_walker()))
    return QMC_ERR_OOM;
  c->p.nl_n = n_l;
  c->p.nl_rc = n_l > 0 ? rc : 0.0;
  for (int l = 0; l < 3; ++l) {
    c->p.nl_a[l] = l < n_l ? amp[l] : 0.0;
    c->p.nl_sinv2[l] = l < n_l ? 1.0 / (width[l] * width[l]) : 0.0;
  }
  sync_params(c);
  return QMC_OK;
}

int qmc_load_coulomb(qmc_crowd* c, int on, double Z, double alpha, int mmax) {
  QMC_RANGE();
  if (!c || (on != 0 && on != 1)) return QMC_ERR_INVALID_ARG;
  if (on == 0) {
    c->p.coul = 0;
    sync_params(c);
    return QMC_OK;
  }
  if (!(Z >= 0.0) || !std::isfinite(Z) || !(alpha > 0.0) || !std::isfinite(alpha) || mmax < 1)
    return QMC_ERR_INVALID_ARG;
  // the half space of 0 < |m|^2 <= mmax^2: m0 > 0, or m0 = 0 < m1, or m0 = m1 = 0 < m2
  const double L = c->p.L, V = L * L * L, two_pi = 6.283185307179586476925286766559;
  std::vector<int> m;
  std::vector<double> cf;
  for (int m0 = 0; m0 <= mmax; ++m0)
    for (int m1 = -mmax; m1 <= mmax; ++m1)
      for (int m2 = -mmax; m2 <= mmax; ++m2) {
        const int n2 = m0 * m0 + m1 * m1 + m2 * m2;
        if (n2 == 0 || n2 > mmax * mmax) continue;
        if (m0 == 0 && (m1 < 0 || (m1 == 0 && m2 < 0))) continue;
        const double k2 = (two_pi / L) * (two_pi / L) * n2;
        m.push_back(m0);
        m.push_back(m1);
        m.push_back(m2);
        cf.push_back(2.0 * two_pi / V * std::exp(-k2 / (4.0 * alpha * alpha)) / k2);
      }
  const int nk = (int)cf.size();
  if (nk > qmcgb::ewald_max_vectors()) return QMC_ERR_UNSUPPORTED;
  int* dm = nullptr;
  double* dc = nullptr;
  if (dmalloc((void**)&dm, sizeof(int) * m.size()) || dmalloc((void**)&dc, sizeof(double) * nk)) {
    if (dm) cudaFree(dm);
    return QMC_ERR_OOM;
  }
  cudaError_t e = cudaMemcpy(dm, m.data(), sizeof(int) * m.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dc, cf.data(), sizeof(double) * nk, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dm);
    cudaFree(dc);
    return cuda_fail(e);
  }
  CK(cudaStreamSynchronize(c->stream));  // no launch still reads the previous lists
  if (c->d_coul_m) cudaFree(c->d_coul_m);
  if (c->d_coul_c) cudaFree(c->d_coul_c);
  c->d_coul_m = dm;
  c->d_coul_c = dc;
  const int N = c->p.N, NI = c->p.n_ions;
  const double Q = NI * Z - N, Q2 = N + NI * Z * Z, sqrt_pi = 1.7724538509055160273;
  c->p.coul = 1;
  c->p.coul_mmax = mmax;
  c->p.coul_nk = nk;
  c->p.coul_alpha = alpha;
  c->p.coul_Z = Z;
  c->p.coul_const = -alpha / sqrt_pi * Q2 - 0.5 * two_pi * Q * Q / (2.0 * V * alpha * alpha);
  c->p.coul_m = dm;
  c->p.coul_c = dc;
  sync_params(c);
  return QMC_OK;
}

int qmc_dmc_select(qmc_crowd* c, const int* src, int n_new, int mem) {
  QMC_RANGE();
  if (!c || !src || n_new < 1 || n_new > c->run.n_walkers) return QMC_ERR_INVALID_ARG;
  if (mem != QMC_MEM_HOST && mem != QMC_MEM_DEVICE) return QMC_ERR_INVALID_ARG;
  if (!c->run.dmc) return QMC_ERR_STATE;
  int st = ensure_ready(c);
  if (st) return st;
  // every index is checked on the host before the gather reads with it
  std::vector<int> h(n_new);
  if (mem == QMC_MEM_DEVICE) {
    CK(cudaMemcpyAsync(h.data(), src, sizeof(int) * n_new, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else {
    std::memcpy(h.data(), src, sizeof(int) * n_new);
  }
  for (int v : h)
    if (v < 0 || v >= c->p.W) return QMC_ERR_INVALID_ARG;
  if (c->run.update == QMC_UPDATE_DELAYED) {  // apply pending windows before copying walkers
    st = move(c, qmcgb::MODE_FLUSH);
    if (st) return st;
  }
  CK(cudaMemcpyAsync(c->d_src, h.data(), sizeof(int) * n_new, cudaMemcpyHostToDevice,
                     c->stream));
  st = gather_population(c, n_new, nullptr, nullptr);
  if (st) return st;
  return read_status(c);
}

int qmc_dmc_append(qmc_crowd* c, const double* R, int m, int mem) {
  QMC_RANGE();
  if (!c || !R || m < 1) return QMC_ERR_INVALID_ARG;
  if (mem != QMC_MEM_HOST && mem != QMC_MEM_DEVICE) return QMC_ERR_INVALID_ARG;
  const int W = c->p.W, N = c->p.N;
  if (W + m > c->run.n_walkers) return QMC_ERR_INVALID_ARG;
  if (mem == QMC_MEM_HOST && !all_finite(R, (size_t)m * N * 3)) return QMC_ERR_INVALID_ARG;
  int st = ensure_ready(c);
  if (st) return st;
  const size_t off = (size_t)W * N * 3, n3 = (size_t)m * N * 3;
  CK(cudaMemcpyAsync(c->d_R + off, R, n3 * sizeof(double),
                     mem == QMC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->stream));
  st = launch_status(c, qmcgb::launch_wrap_positions(c->d_R + off, n3, c->p.L, c->d_status,
                                                     c->stream));
  if (st) return st;
  // the new walkers' orbital rows and FP64 inverses, nobody else's (launched with the
  // grown population, of which walkers W .. W + m - 1 are the new ones)
  qmcgb::Params pa = c->p;
  pa.W = W + m;
  if (is_mixed(c)) st = launch_status(c, qmcgb::launch_eval_rows<float>(pa, c->stream, W, m));
  else st = launch_status(c, qmcgb::launch_eval_rows<double>(pa, c->stream, W, m));
  if (st) return st;
  if (is_mixed(c))
    st = launch_status(c, qmcgb::launch_recompute<float>(pa, c->d_ws, c->stream, W, m));
  else
    st = launch_status(c, qmcgb::launch_recompute<double>(pa, c->d_ws, c->stream, W, m));
  if (st) return st;
  CK(cudaMemsetAsync(c->d_pend + (size_t)W * qmcgb::PEND_STRIDE, 0,
                     sizeof(double) * m * qmcgb::PEND_STRIDE, c->stream));
  CK(cudaMemsetAsync(c->d_jvalid + W, 0, sizeof(int) * m, c->stream));
  c->p.W = W + m;
  sync_params(c);
  return read_status(c);
}

}  // extern "C"

namespace {

// The new population is walkers d_src[0..n_new) of the current one: their whole state is
// gathered into the idle half of the double buffer, the halves swap, and the pending
// proposals are dropped.  e_in/e_out: optional device E_L carried along.
int gather_population(qmc_crowd* c, int n_new, const double* e_in, double* e_out) {
  const int N = c->p.N, n = c->p.n, es = c->es;
  qmcgb::WalkerState from{c->d_R, c->d_rows, c->d_binv, c->d_jgl, c->d_logdet, c->d_sign,
                          c->d_jvalid, (size_t)N * 3, (size_t)es * N * 5 * c->p.n_pad,
                          (size_t)es * 2 * n * n, (size_t)es * N * 4, c->p.W,
                          c->d_status, c->p.check_info};
  qmcgb::WalkerState to = from;
  to.R = c->d_R2;
  to.rows = c->d_rows2;
  to.binv = c->d_binv2;
  to.jgl = c->d_jgl2;
  to.logdet = c->d_logdet2;
  to.sign = c->d_sign2;
  to.jvalid = c->d_jvalid2;
  int st = launch_status(c, qmcgb::launch_gather(to, from, c->d_src, n_new, e_in, e_out,
                                                 c->stream));
  if (st) return st;
  std::swap(c->d_R, c->d_R2);
  std::swap(c->d_rows, c->d_rows2);
  std::swap(c->d_binv, c->d_binv2);
  std::swap(c->d_jgl, c->d_jgl2);
  std::swap(c->d_logdet, c->d_logdet2);
  std::swap(c->d_sign, c->d_sign2);
  std::swap(c->d_jvalid, c->d_jvalid2);
  CK(cudaMemsetAsync(c->d_pend, 0, sizeof(double) * c->run.n_walkers * qmcgb::PEND_STRIDE,
                     c->stream));
  c->p.W = n_new;
  sync_params(c);
  return QMC_OK;
}

}  // namespace

extern "C" {

int qmc_dmc_branch(qmc_crowd* c, const double* e_prev, double* e_new, int mem, double e_trial,
                   qmc_dmc_stats* out) {
  QMC_RANGE();
  if (!c || !e_prev || !e_new) return QMC_ERR_INVALID_ARG;
  if (!c->run.dmc) return QMC_ERR_STATE;
  int st = ensure_ready(c);
  if (st) return st;
  const int W = c->p.W, N = c->p.N, cap = c->run.n_walkers;
  if (c->run.update == QMC_UPDATE_DELAYED) {  // apply pending windows before copying walkers
    st = move(c, qmcgb::MODE_FLUSH);
    if (st) return st;
  }
  const double* ep = e_prev;
  const double* en = e_new;
  if (mem == QMC_MEM_HOST) {
    CK(cudaMemcpyAsync(c->d_e, e_prev, sizeof(double) * W, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_e + cap, e_new, sizeof(double) * W, cudaMemcpyHostToDevice,
                       c->stream));
    ep = c->d_e;
    en = c->d_e + cap;
  }
  const uint32_t gen = c->gen > 0 ? c->gen - 1 : 0;  // the generation just completed
  st = launch_status(c, qmcgb::launch_branch(ep, en, W, N, c->p.tau, e_trial, c->run.seed, gen,
                                             cap, c->d_mult, c->d_src, c->d_bout, c->d_bsums,
                                             c->stream));
  if (st) return st;
  int bo[2];
  double sums[2];
  CK(cudaMemcpyAsync(bo, c->d_bout, sizeof(bo), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(sums, c->d_bsums, sizeof(sums), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int n_new = bo[0];
  if (out) {
    out->n_before = W;
    out->n_after = n_new;
    out->n_wanted = bo[1];
    out->w_sum = sums[0];
    out->we_sum = sums[1];
  }
  if (n_new == 0) return QMC_ERR_STATE;  // the population died out: the crowd is unchanged
  double* e_out = c->d_e + 2 * (size_t)cap;
  st = gather_population(c, n_new, en, e_out);
  if (st) return st;
  CK(cudaMemcpyAsync(e_new, e_out, sizeof(double) * n_new,
                     mem == QMC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return QMC_OK;
}

int qmc_get_launch_count(qmc_crowd* c, unsigned long long* count) {
  QMC_RANGE();
  if (!c || !count) return QMC_ERR_INVALID_ARG;
  *count = c->launches;
  return QMC_OK;
}

namespace {
struct SaveHeader {
  uint64_t magic;
  int32_t W, N;
  uint32_t gen, pad;
  uint64_t seed;
};
constexpr uint64_t kMagic = 0x31424743514d51ull;  // "QMQCGB1"
}  // namespace

int qmc_crowd_save(qmc_crowd* c, void* buf, size_t* size) {
  QMC_RANGE();
  if (!c || !size) return QMC_ERR_INVALID_ARG;
  const size_t need = sizeof(SaveHeader) + sizeof(double) * c->p.W * c->p.N * 3;
  if (!buf) {
    *size = need;
    return QMC_OK;
  }
  if (*size < need) return QMC_ERR_INVALID_ARG;
  SaveHeader h{kMagic, c->p.W, c->p.N, c->gen, 0u, c->run.seed};
  std::memcpy(buf, &h, sizeof(h));
  int st = qmc_get_positions(c, (double*)((char*)buf + sizeof(h)), QMC_MEM_HOST);
  *size = need;
  return st;
}

// ---------------------------------------------------------------------------------------
// Batches: several crowds (systems of different sizes) swept by one launch per generation.
// ---------------------------------------------------------------------------------------
struct qmc_batch {
  std::vector<qmc_crowd*> crowds;  // caller's order
  std::vector<int> order;          // launch order: largest systems first
  int update = 0, nt = 256;
  bool mixed = false;
  size_t smem = 0;
  qmcgb::BatchArgs args{};
  std::vector<Params> hp;          // launch order
  Params* d_params = nullptr;
  std::vector<double*> ring;       // per crowd (caller's order): E_L [cap][W]
  int ring_cap = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t graph = nullptr;  // one plain generation: batch move launch + advance
  bool eager_done = false;
  unsigned long long launches = 0;
};

namespace {

void batch_free(qmc_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->d_params) cudaFree(b->d_params);
  for (double* r : b->ring)
    if (r) cudaFree(r);
  if (b->ev) cudaEventDestroy(b->ev);
}

int batch_launch_move(qmc_batch* b) {
  ++b->launches;
  cudaError_t e = b->mixed ? qmcgb::launch_batch<float>(b->nt, b->d_params, b->args, b->update,
                                                         b->smem, b->stream)
                           : qmcgb::launch_batch<double>(b->nt, b->d_params, b->args, b->update,
                                                          b->smem, b->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  ++b->launches;
  qmcgb::batch_advance_kernel<<<1, 32, 0, b->stream>>>(b->d_params, (int)b->order.size());
  e = cudaGetLastError();
  return e == cudaSuccess ? QMC_OK : cuda_fail(e);
}

// Every crowd's stream waits for the batch stream (or the other way round).
int batch_join(qmc_batch* b, bool into_batch) {
  for (qmc_crowd* c : b->crowds) {
    if (c->stream == b->stream) continue;
    cudaStream_t from = into_batch ? c->stream : b->stream;
    cudaStream_t to = into_batch ? b->stream : c->stream;
    CK(cudaEventRecord(b->ev, from));
    CK(cudaStreamWaitEvent(to, b->ev, 0));
  }
  return QMC_OK;
}

}  // namespace

int qmc_batch_create(qmc_crowd* const* crowds, int n_crowds, qmc_batch** out) {
  QMC_RANGE();
  if (!crowds || !out || n_crowds < 1 || n_crowds > qmcgb::MAX_BATCH) return QMC_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n_crowds; ++i) {
    if (!crowds[i]) return QMC_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (crowds[j] == crowds[i]) return QMC_ERR_INVALID_ARG;
    const qmc_crowd* c = crowds[i];
    const qmc_crowd* c0 = crowds[0];
    if (c->run.precision != c0->run.precision || c->run.update != c0->run.update ||
        c->p.nt != c0->p.nt || c->p.nl_n > 0 || c->p.coul)
      return QMC_ERR_UNSUPPORTED;
  }
  qmc_batch* b = new qmc_batch();
  b->crowds.assign(crowds, crowds + n_crowds);
  b->update = crowds[0]->run.update;
  b->nt = crowds[0]->p.nt;
  b->mixed = is_mixed(crowds[0]);
  b->stream = crowds[0]->stream;
  b->order.resize(n_crowds);
  for (int i = 0; i < n_crowds; ++i) b->order[i] = i;
  // longest walkers first: their CTAs start in the first wave
  std::sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    return crowds[x]->p.N > crowds[y]->p.N || (crowds[x]->p.N == crowds[y]->p.N && x < y);
  });
  b->args.n = n_crowds;
  b->args.base[0] = 0;
  for (int q = 0; q < n_crowds; ++q) {
    qmc_crowd* c = crowds[b->order[q]];
    b->args.base[q + 1] = b->args.base[q] + c->p.W;
    std::memcpy(&b->args.maps[q], &c->tmap, sizeof(CUtensorMap));
    b->smem = std::max(b->smem, c->smem);
  }
  b->hp.resize(n_crowds);
  b->ring.assign(n_crowds, nullptr);
  if (dmalloc((void**)&b->d_params, sizeof(Params) * n_crowds) ||
      cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    delete b;
    return QMC_ERR_OOM;
  }
  *out = b;
  return QMC_OK;
}

int qmc_batch_destroy(qmc_batch* b) {
  QMC_RANGE();
  if (!b) return QMC_ERR_INVALID_ARG;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
  return QMC_OK;
}

int qmc_batch_sweep(qmc_batch* b, int n_gen, double* const* eloc, qmc_stats* stats) {
  QMC_RANGE();
  if (!b || n_gen < 0) return QMC_ERR_INVALID_ARG;
  const int nc = (int)b->crowds.size();
  for (qmc_crowd* c : b->crowds) {
    // batches run without the nonlocal and Coulomb terms
    if (c->p.nl_n > 0 || c->p.coul) return QMC_ERR_UNSUPPORTED;
    const int st = ensure_ready(c);
    if (st) return st;
  }
  if (n_gen == 0) return QMC_OK;
  int st = batch_join(b, true);
  if (st) return st;
  if (b->ring_cap < n_gen) {
    for (double*& r : b->ring) {
      if (r) cudaFree(r);
      r = nullptr;
    }
    b->ring_cap = 0;
    for (int i = 0; i < nc; ++i)
      if (dmalloc((void**)&b->ring[i], sizeof(double) * (size_t)n_gen * b->crowds[i]->p.W))
        return QMC_ERR_OOM;
    b->ring_cap = n_gen;
    if (b->graph) {  // the graph holds the old parameters' addresses only, but rebuild anyway
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  // parameters of every crowd (launch order), E_L rows indexed by generation
  auto fill = [&](int g) {
    for (int q = 0; q < nc; ++q) {
      const int ci = b->order[q];
      qmc_crowd* c = b->crowds[ci];
      sync_params(c);
      Params p = c->p;
      p.gen = c->gen + (uint32_t)g;
      p.eloc_out = b->ring[ci];
      p.eloc_by_gen = 1;
      p.eloc_gen0 = c->gen;
      p.n_accept = stats ? c->d_nacc : nullptr;
      p.stencil_bytes = qmcgb::stencil_tma_bytes(p, c->es);
      p.skip_eloc = 0;
      b->hp[q] = p;
    }
  };
  if (stats)
    for (qmc_crowd* c : b->crowds) {
      CK(cudaMemsetAsync(c->d_nacc, 0, sizeof(unsigned long long), b->stream));
      if (c->d_nrep)
        CK(cudaMemsetAsync(c->d_nrep + 1, 0, sizeof(unsigned long long), b->stream));
    }
  auto due = [&](qmc_crowd* c, int g) {
    return c->run.n_recompute > 0 && ((c->gen + (uint32_t)g + 1) % (uint32_t)c->run.n_recompute) == 0;
  };
  fill(0);
  for (int q = 0; q < nc; ++q)  // layouts as launched (the kernel checks this too)
    if (qmcgb::move_smem_bytes(b->hp[q], b->crowds[b->order[q]]->es) > b->smem)
      return QMC_ERR_STATE;
  CK(cudaMemcpyAsync(b->d_params, b->hp.data(), sizeof(Params) * nc, cudaMemcpyHostToDevice,
                     b->stream));
  for (int g = 0; g < n_gen; ++g) {
    bool any_due = false;
    for (qmc_crowd* c : b->crowds) any_due |= due(c, g);
    if (!any_due && !b->graph && !b->eager_done) {
      // the first plain generation runs eagerly (it configures the kernel's shared memory
      // limit, which a stream capture must not do); later ones replay a captured graph
      st = batch_launch_move(b);
      if (st) return st;
      b->eager_done = true;
      continue;
    }
    if (!any_due) {
      // a plain generation: replay the captured graph (batch launch + advance)
      if (!b->graph) {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const int ls = batch_launch_move(b);
        cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
        if (ls) {
          if (graph) cudaGraphDestroy(graph);
          return ls;
        }
        if (ce != cudaSuccess) return cuda_fail(ce);
        ce = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(ce);
        b->launches -= 2;  // counted at replay
      }
      CK(cudaGraphLaunch(b->graph, b->stream));
      b->launches += 2;
      continue;
    }
    // a generation with an FP64 recompute for some crowds: their E_L follows the recompute
    fill(g);
    for (int q = 0; q < nc; ++q) b->hp[q].skip_eloc = due(b->crowds[b->order[q]], g) ? 1 : 0;
    CK(cudaMemcpyAsync(b->d_params, b->hp.data(), sizeof(Params) * nc, cudaMemcpyHostToDevice,
                       b->stream));
    st = batch_launch_move(b);
    if (st) return st;
    for (int q = 0; q < nc; ++q) {
      const int ci = b->order[q];
      qmc_crowd* c = b->crowds[ci];
      if (!due(c, g)) continue;
      Params p = b->hp[q];
      cudaError_t e = is_mixed(c) ? qmcgb::launch_recompute<float>(p, c->d_ws, b->stream)
                                  : qmcgb::launch_recompute<double>(p, c->d_ws, b->stream);
      ++b->launches;
      if (e != cudaSuccess) return cuda_fail(e);
      p.skip_eloc = 0;
      const void* tm = p.use_tma ? (const void*)&c->tmap : nullptr;
      e = is_mixed(c) ? qmcgb::launch_move<float>(p, qmcgb::MODE_ELOC, tm, b->stream)
                      : qmcgb::launch_move<double>(p, qmcgb::MODE_ELOC, tm, b->stream);
      ++b->launches;
      if (e != cudaSuccess) return cuda_fail(e);
    }
    // back to plain parameters for the following generations (generation g + 1)
    fill(g + 1);
    CK(cudaMemcpyAsync(b->d_params, b->hp.data(), sizeof(Params) * nc, cudaMemcpyHostToDevice,
                       b->stream));
  }
  for (qmc_crowd* c : b->crowds) c->gen += (uint32_t)n_gen;
  st = batch_join(b, false);
  if (st) return st;
  CK(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < nc; ++i) {
    qmc_crowd* c = b->crowds[i];
    const size_t cnt = (size_t)n_gen * c->p.W;
    std::vector<double> h(cnt);
    CK(cudaMemcpy(h.data(), b->ring[i], sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    if (eloc && eloc[i]) std::memcpy(eloc[i], h.data(), sizeof(double) * cnt);
    if (stats) {
      double s1 = 0.0, s2 = 0.0;
      for (double e : h) {
        s1 += e;
        s2 += e * e;
      }
      unsigned long long na = 0, nr = 0;
      CK(cudaMemcpy(&na, c->d_nacc, sizeof(na), cudaMemcpyDeviceToHost));
      if (c->d_nrep) CK(cudaMemcpy(&nr, c->d_nrep + 1, sizeof(nr), cudaMemcpyDeviceToHost));
      stats[i].n_repair = (long long)nr;
      stats[i].e_sum = s1;
      stats[i].e2_sum = s2;
      stats[i].n_samples = (long long)cnt;
      stats[i].n_accept = (long long)na;
      stats[i].n_moves = (long long)n_gen * c->p.W * c->p.N;
    }
    st = read_status(c);
    if (st) return st;
  }
  return QMC_OK;
}

int qmc_batch_get_launch_count(const qmc_batch* b, unsigned long long* count) {
  QMC_RANGE();
  if (!b || !count) return QMC_ERR_INVALID_ARG;
  *count = b->launches;
  return QMC_OK;
}

int qmc_crowd_restore(qmc_crowd* c, const void* buf, size_t size) {
  QMC_RANGE();
  if (!c || !buf || size < sizeof(SaveHeader)) return QMC_ERR_INVALID_ARG;
  SaveHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kMagic || h.W != c->p.W || h.N != c->p.N ||
      size < sizeof(h) + sizeof(double) * c->p.W * c->p.N * 3)
    return QMC_ERR_INVALID_ARG;
  c->gen = h.gen;
  c->run.seed = h.seed;
  c->p.seed = h.seed;
  int st = qmc_load_positions(c, (const double*)((const char*)buf + sizeof(h)), QMC_MEM_HOST);
  if (st) return st;
  if (c->has_orbitals) return qmc_recompute(c);
  return QMC_OK;
}

}  // extern "C"

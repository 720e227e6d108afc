// The particle-by-particle move over a crowd of walkers (arXiv:2209.14487, Alg. 1 lines
// 4-11) as one CTA per walker.  Walkers are independent (Alg. 1 line 2), so a walker's
// CTA runs its whole electron loop (Alg. 1 line 4, sequential) without any grid-level
// synchronisation: one launch per generation replaces the per-electron kernel chain of
// the lock-step driver (Sec. II-C, limitations (a)-(b)).  The fine-grained batched calls
// (propose / accept / energy) are other instantiations of the same kernel and device
// functions, so the timed path and the parity-tested path are one code.
//
// Precision: T = double is the FP64 path.  T = float is the mixed path: orbitals,
// Jastrow, ratios, the proposal and the Metropolis test in FP32 on 32-bit fixed-point
// positions, inverse in FP32; log|det| and the local energy accumulate in FP64 and the
// inverse is recomputed in FP64 by a separate kernel.  In the mixed path every warp
// evaluates the (cheap, deterministic) proposal and acceptance itself after each block
// reduction, so the move needs three barriers plus one per accepted move; the FP64 path,
// where GB300's FP64 rate makes redundant scalar work expensive, lets thread 0 do it.
//
// This file is the kernel's implementation, compiled once per CTA width and precision: a
// translation unit defines QMCGB_MOVE_NT (threads per CTA), QMCGB_MOVE_NS (the namespace
// of that width) and QMCGB_MOVE_ELEM (4: the mixed path, 8: the FP64 path) and includes it.  Narrow CTAs suit small determinants: a move is a chain of short
// block reductions, and fewer warps make each barrier and each reduction cheaper.
#if !defined(QMCGB_MOVE_NT) || !defined(QMCGB_MOVE_ELEM)
#error "define QMCGB_MOVE_NT, QMCGB_MOVE_NS and QMCGB_MOVE_ELEM before including qmc_move_impl.cuh"
#endif
#include <cuda.h>

#include <atomic>
#include <cmath>
#include <cstring>

#include "qmc_device.cuh"
#include "qmc_internal.h"
#include "qmc_lu.cuh"

namespace qmcgb {
namespace QMCGB_MOVE_NS {

constexpr int NT = QMCGB_MOVE_NT;  // threads per CTA
constexpr int NWARP = NT / 32;
constexpr int JT = 4;
// Tensor-core flush: operand tiles of 128 rows x 32 K-elements, FP32 split into TF32 hi and
// lo parts; A and B operand stages of 32 KB each.
constexpr int TC_TILE = 128;
constexpr int TC_KC = 32;
constexpr int TC_STAGE_BYTES = 4 * TC_TILE * TC_KC * 4;
constexpr uint32_t TC_COLS = 128;  // TMEM columns a CTA allocates  // Jastrow partner terms cached per thread (N + N_ions <= JT * NT)

// Per-move proposal state (registers of every thread in the mixed path; in the FP64 path
// thread 0 builds it in shared memory and the others copy it).
template <typename T>
struct Prop {
  T F[3], disp[3], logGf;
  T t[3];          // offsets in the spline cell
  int cell[3];
  uint32_t rq[3];  // mixed: fixed-point proposed position
  double rp[3];    // FP64: proposed position
};

template <typename T>
struct Res {
  T rhoD, dU, rho, Fp[3];
};

template <typename T>
struct Scal {
  Prop<T> pr;
  Res<T> rs;
  double logdet[2];
  float lsum[2], lcomp[2];  // mixed path: Kahan sums of log|rhoD| since the kernel began
  int sign[2];
  int accept, m;
  uint32_t tmem;  // TMEM base address of the tensor-core flush
  T wts[48];
  T chi[4];       // compact layout: the current move's Gaussian draws
};

// Constants of the crowd in the path's precision, converted once per kernel (a double to
// float conversion runs on the FP64 pipe, 1/64 rate on GB300).
template <typename T>
struct Cst {
  T L, invL, tau, stau, dgrid, h2inv, h1inv, rc2, rc1, halfL, unit, scale;
};

template <typename T>
__device__ __forceinline__ Cst<T> make_cst(const Params& p) {
  Cst<T> k;
  k.L = (T)p.L;
  k.invL = (T)p.invL;
  k.tau = (T)p.tau;
  k.stau = (T)p.sqrt_tau;
  k.dgrid = (T)p.dgrid;
  k.h2inv = (T)p.h2inv;
  k.h1inv = (T)p.h1inv;
  k.rc2 = (T)p.rc2;
  k.rc1 = (T)p.rc1;
  k.halfL = (T)(0.5 * p.L);
  k.unit = (T)p.fx_unit;
  k.scale = (T)p.fx_scale;
  return k;
}

struct Lay {
  size_t scal, bar, stc, tcs, B, R, Rq, ion, ionq, jc, jgl, phi, part, col, col2, dchi, du, red0,
      red1;
  size_t wP, wV, wS, wy, wz, wc, wb, snap, xb, yb, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Row stride of the inverse staged in shared memory: n + 4 floats (16-byte aligned rows,
// conflict-free float4 reads by one thread per row) or n + 1 doubles.
template <typename T>
__host__ __device__ inline int b_stride(const Params& p) {
  return p.b_in_smem ? p.n + (sizeof(T) == 4 ? 4 : 1) : p.n;
}

template <typename T>
__host__ __device__ inline Lay make_lay(const Params& p) {
  const size_t es = sizeof(T);
  Lay L{};
  size_t o = 0;
  L.scal = o; o += al16(sizeof(Scal<T>));
  L.bar = o; o += 32;  // stencil copies (ring slot 0), tensor-core MMAs, ring slots 1 and 2
  // +128: alignment slack
  L.stc = o; o += p.use_tma == 1 ? al16((size_t)p.stencil_bytes + 128) : 0;
  // the ring's boxes take the place of the partial sums (its consumer combines the four
  // x-planes in registers)
  const size_t part_bytes = p.use_tma == 2 ? al16((size_t)RING_SLOTS * p.stencil_bytes + 128)
                                           : al16((size_t)16 * p.n_pad * es);
  // tensor-core flush staging: shares the stencil buffer (unused during a flush) when that
  // is large enough, else the move's phi', partial sums (or ring) and column (dead during
  // a flush, see accept_update) when those are, else a buffer of its own
  L.tcs = L.stc;
  const size_t move_bufs = al16((size_t)5 * p.n_pad * es) + part_bytes + al16((size_t)p.n_pad * es);
  const bool need_stage = p.tc_flush && !(p.use_tma == 1 && p.stencil_bytes >= TC_STAGE_BYTES);
  const bool over_move = need_stage && es == 4 && move_bufs >= (size_t)TC_STAGE_BYTES + 128;
  if (need_stage && !over_move) {
    L.tcs = o;
    o += al16((size_t)TC_STAGE_BYTES + 128);
  }
  L.B = o; o += al16(p.b_in_smem ? (size_t)p.n * b_stride<T>(p) * es : 0);
  L.R = o; o += es == 8 ? al16((size_t)p.N * 3 * 8) : 0;  // the mixed path moves fixed point
  L.Rq = o; o += al16((size_t)p.N * 3 * 4);
  L.ion = o; o += al16((size_t)p.n_ions * 3 * 8);
  L.ionq = o; o += al16((size_t)p.n_ions * 3 * 4);
  L.jc = o; o += al16((size_t)3 * (MAX_KNOTS + 3) * es);  // any Jastrow the crowd loads later
  L.jgl = o; o += p.inc_jastrow ? al16((size_t)p.N * 4 * es) : 0;
  L.phi = o; o += al16((size_t)5 * p.n_pad * es);
  L.part = o; o += part_bytes;
  L.col = o; o += al16((size_t)p.n_pad * es);
  L.col2 = o; o += p.inc_jastrow ? al16((size_t)p.n_pad * es) : 0;  // the next move's column
  if (over_move) L.tcs = L.phi;
  L.dchi = o; o += p.compact ? 0 : al16((size_t)p.N * 3 * es);
  L.du = o; o += p.compact ? 0 : al16((size_t)p.N * es);
  L.red0 = o; o += al16((size_t)NWARP * 8 * 8);  // eight values per warp, FP64 at most
  L.red1 = o; o += al16((size_t)NWARP * 8 * 8);
  L.wP = L.wV = L.wS = L.wy = L.wz = L.wc = L.wb = L.snap = L.xb = L.yb = o;
  if (p.update == 1) {
    L.wP = o; o += al16((size_t)MAX_K * 4);
    L.wV = o; o += p.compact ? 0 : al16((size_t)p.k * p.vs * es);
    L.wS = o; o += al16((size_t)p.k * p.ks * es);
    L.wy = o; o += al16((size_t)(MAX_K + 1) * es);
    L.wz = o; o += al16((size_t)(MAX_K + 1) * es);
    L.wc = o; o += al16((size_t)(MAX_K + 1) * es);
    L.wb = o; o += al16((size_t)(MAX_K + 1) * es);
    if (!p.tc_flush) {  // the tensor-core flush keeps them in global memory
      L.snap = o; o += al16((size_t)p.k * p.n * es);
      L.xb = o; o += al16((size_t)p.n * p.k * es);
      L.yb = o; o += al16((size_t)p.n * p.k * es);
    }
  }
  L.total = o;
  return L;
}

#if QMCGB_MOVE_ELEM == 4  // host functions shared by both precisions: in the FP32 unit
size_t move_smem_bytes(const Params& p, int elem_bytes) {
  return elem_bytes == 4 ? make_lay<float>(p).total : make_lay<double>(p).total;
}
#endif

template <typename T>
struct Ctx {
  const Params& p;
  Cst<T> k;
  int w, tid, lane, warp;
  int bs;   // row stride of B
  int upd;  // 0: Sherman-Morrison, 1: delayed window (a template constant of the kernel)
  int bsm;  // where B lives: 1 shared, 2 global, 0 decided at run time (template constant)
  Scal<T>* sc;
  T* B;     // inverse (transposed) of the moving spin: shared or global
  T* Bs;    // shared staging buffer (if p.b_in_smem)
  T* Bg;    // this walker's global inverses [2][n][n]
  double* R;
  uint32_t* Rq;
  double* ion;
  uint32_t* ionq;
  T* jc;
  T* jgl;   // incremental sweep: grad U (3) and lap U of every electron [N][4]
  T* phi;
  T* part;
  T* col;
  T* col2;  // incremental sweep: the next move's column, written by the update's row owners
  T* dchi;
  T* du;
  T* red0;
  T* red1;
  int* wP;
  T* wV;
  T* wS;
  T* wy;
  T* wz;
  T* wc;
  T* wb;
  T* snap;
  T* xb;
  T* yb;
  T* rows;  // this walker's global orbital rows [N][5][n_pad]
  T* stc;   // TMA-staged stencil [4][4][4][n_pad] (x, y, z, orbital)
  uint64_t* bar;      // [0] stencil copies, [1] tensor-core MMA completion
  const void* tmap;
  uint32_t tma_phase;
  uint32_t mma_phase;
  float* tcs;         // tensor-core staging: A hi, A lo, B hi, B lo (128 x 32 each)
  bool tc;            // windows flushed on the tensor cores (TMEM held by this CTA)
  bool tc_over_move;  // their operand stage overlays phi', part and col
  bool failed;        // a bounded wait ran out (status set); the sweep stops
  // stencil items of this thread (orbital j, x offset a), at most 4
  int nit;
  int itj[4], ita[4];
};

// ---------------------------------------------------------------------------------------
// Jastrow term geometry: displacement from electron/point (x, q) to partner t (electron
// t < N, ion t - N) and its length; the radial functor of the pair.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void partner_disp(const Ctx<T>& c, const double* x, const uint32_t* q,
                                             int t, T* d, T& r, T& rinv) {
  const Params& p = c.p;
  if constexpr (IsMixed<T>::value) {
    const uint32_t* b = t < p.N ? c.Rq + 3 * t : c.ionq + 3 * (t - p.N);
    disp_fx(q, b, c.k.unit, d);
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    rinv = rsqrtf(r2);
    r = r2 * rinv;
  } else {
    const double* b = t < p.N ? c.R + 3 * t : c.ion + 3 * (t - p.N);
    disp_f64(x, b, p.L, p.invL, d);
    r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    rinv = 1.0 / r;
  }
}

template <typename T>
__device__ __forceinline__ void functor(const Ctx<T>& c, int i, int t, const T*& coef, int& K,
                                        T& hinv, T& rc) {
  const Params& p = c.p;
  if (t < p.N) {
    const bool same = (i < p.n_up) == (t < p.n_up);
    coef = c.jc + (same ? 0 : p.K2 + 3);
    K = p.K2;
    hinv = c.k.h2inv;
    rc = c.k.rc2;
  } else {
    coef = c.jc + 2 * (p.K2 + 3);
    K = p.K1;
    hinv = c.k.h1inv;
    rc = c.k.rc1;
  }
}

__device__ __forceinline__ void term_range(const Params& p, int& t0, int& t1) {
  t0 = p.K2 > 0 ? 0 : p.N;
  t1 = p.K1 > 0 ? p.N + p.n_ions : p.N;
}

// ---------------------------------------------------------------------------------------
// Inverse and delayed window of one spin: staging in and out of shared memory.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ void begin_spin(Ctx<T>& c, int s) {
  const Params& p = c.p;
  const int n = p.n;
  T* Bg = c.Bg + (size_t)s * n * n;
  const bool in_smem = c.bsm == 1 || (c.bsm == 0 && p.b_in_smem);
  if (in_smem) {
    for (int r = c.warp; r < n; r += NWARP)
      for (int j = c.lane; j < n; j += 32) c.Bs[r * c.bs + j] = Bg[(size_t)r * n + j];
  }
  // a compile-time choice where possible, so accesses through c.B are shared-memory ones
  if (c.bsm == 1) c.B = c.Bs;
  else if (c.bsm == 2) c.B = Bg;
  else c.B = in_smem ? c.Bs : Bg;
  if (c.upd == 1) {
    const int ws = c.w * 2 + s;
    const int m = p.win_m[ws];
    const T* gV = (const T*)p.win_V + (size_t)ws * p.k * p.vs;
    const T* gS = (const T*)p.win_S + (size_t)ws * p.k * p.ks;
    for (int e = c.tid; e < m; e += NT) c.wP[e] = p.win_P[ws * MAX_K + e];
    if (p.compact) c.wV = const_cast<T*>(gV);  // the V rows are used where they are stored
    else
      for (int e = c.tid; e < m * p.vs; e += NT) c.wV[e] = gV[e];
    for (int e = c.tid; e < m * p.ks; e += NT) c.wS[e] = gS[e];
    if (c.tid == 0) c.sc->m = m;
  } else if (c.tid == 0) {
    c.sc->m = 0;
  }
  __syncthreads();
}

template <typename T>
__device__ void end_spin(Ctx<T>& c, int s, bool store) {
  const Params& p = c.p;
  const int n = p.n;
  __syncthreads();
  if (!store) return;
  if (p.b_in_smem) {
    T* Bg = c.Bg + (size_t)s * n * n;
    for (int r = c.warp; r < n; r += NWARP)
      for (int j = c.lane; j < n; j += 32) Bg[(size_t)r * n + j] = c.Bs[r * c.bs + j];
  }
  if (c.upd == 1) {
    const int ws = c.w * 2 + s;
    const int m = c.sc->m;
    T* gV = (T*)p.win_V + (size_t)ws * p.k * p.vs;
    T* gS = (T*)p.win_S + (size_t)ws * p.k * p.ks;
    for (int e = c.tid; e < m; e += NT) p.win_P[ws * MAX_K + e] = c.wP[e];
    if (!p.compact)
      for (int e = c.tid; e < m * p.vs; e += NT) gV[e] = c.wV[e];
    for (int e = c.tid; e < m * p.ks; e += NT) gS[e] = c.wS[e];
    if (c.tid == 0) p.win_m[ws] = m;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// Delayed window (Woodbury).  The window holds m replaced rows p_l (all distinct) with
// their new orbital rows Phi_l; with A_cur = A_0 + P V, V_l = Phi_l - a_{p_l} and
// B = A_0^-1, every product V B is evaluated as Phi B - P^T (a_p^T B = e_p^T), the form
// in which rounding errors of B are damped as in Sherman-Morrison.  S = I + V B P and its
// inverse is bordered one accept at a time.
// ---------------------------------------------------------------------------------------

// Column pp of the current inverse: B[:,pp] - (B P) S^-1 (V B[:,pp]); y and z = S^-1 y
// are kept for a following accept.
template <typename T>
__device__ void compute_column(Ctx<T>& c, int pp) {
  const Params& p = c.p;
  const int n = p.n;
  const T* brow = c.B + (size_t)pp * c.bs;
  const int m = c.sc->m;
  if (m == 0) {
    for (int j = c.tid; j < n; j += NT) c.col[j] = brow[j];
    return;
  }
  for (int l = c.warp; l < m; l += NWARP) {
    const T* v = c.wV + (size_t)l * p.vs;
    T acc = 0;
    for (int j = c.lane; j < n; j += 32) acc += v[j] * brow[j];
    acc = warp_sum(acc);
    if (c.lane == 0) c.wy[l] = acc - (c.wP[l] == pp ? T(1) : T(0));
  }
  __syncthreads();
  for (int l = c.tid; l < m; l += NT) {
    const T* srow = c.wS + (size_t)l * p.ks;
    T acc = 0;
    for (int q = 0; q < m; ++q) acc += srow[q] * c.wy[q];
    c.wz[l] = acc;
  }
  __syncthreads();
  for (int j = c.tid; j < n; j += NT) {
    T acc = brow[j];
    for (int l = 0; l < m; ++l) acc -= c.B[(size_t)c.wP[l] * c.bs + j] * c.wz[l];
    c.col[j] = acc;
  }
}

// B <- B - (B P) S^-1 (V B); in B^T form B^T[k] -= sum_b Y[k][b] B^T[p_b] with
// X[k][l] = B^T[k].Phi_l - delta(k, p_l) and Y = X S^-T.
template <typename T>
__device__ void flush_window_simt(Ctx<T>& c) {
  const Params& p = c.p;
  const int m = c.sc->m;
  if (m == 0) return;
  const int n = p.n, bs = c.bs;
  for (int l = c.warp; l < m; l += NWARP)
    for (int j = c.lane; j < n; j += 32) c.snap[l * n + j] = c.B[(size_t)c.wP[l] * bs + j];
  for (int e = c.tid; e < n * m; e += NT) {
    const int k = e / m, l = e - k * m;
    const T* brow = c.B + (size_t)k * bs;
    const T* v = c.wV + (size_t)l * p.vs;
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int j = 0;
    for (; j + 4 <= n; j += 4) {
      a0 += brow[j] * v[j];
      a1 += brow[j + 1] * v[j + 1];
      a2 += brow[j + 2] * v[j + 2];
      a3 += brow[j + 3] * v[j + 3];
    }
    for (; j < n; ++j) a0 += brow[j] * v[j];
    c.xb[e] = (a0 + a1) + (a2 + a3) - (k == c.wP[l] ? T(1) : T(0));
  }
  __syncthreads();
  for (int e = c.tid; e < n * m; e += NT) {
    const int k = e / m, b = e - k * m;
    const T* srow = c.wS + (size_t)b * p.ks;
    const T* xrow = c.xb + (size_t)k * m;
    T acc = 0;
    for (int l = 0; l < m; ++l) acc += xrow[l] * srow[l];
    c.yb[e] = acc;
  }
  __syncthreads();
  for (int k = c.warp; k < n; k += NWARP) {
    const T* yrow = c.yb + (size_t)k * m;
    T* brow = c.B + (size_t)k * bs;
    for (int j = c.lane; j < n; j += 32) {
      T acc = 0;
      for (int b = 0; b < m; ++b) acc += yrow[b] * c.snap[b * n + j];
      brow[j] -= acc;
    }
  }
  __syncthreads();
  if (c.tid == 0) c.sc->m = 0;
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// The flush on the tensor cores (mixed path, inverse in global memory).  The two products
// of the flush, X = B^T Phi^T and B^T -= Y snap, run as tcgen05 kind::tf32 MMAs of 128-row
// tiles with FP32 operands split into TF32 hi + lo parts (3 MMAs per K-step: hi.hi,
// hi.lo, lo.hi), accumulated in FP32 in TMEM; the small m x m product Y = X S^-T stays on
// the CUDA cores.  Operand tiles are staged through shared memory in the K-major layout
// without swizzling: the float4 slot e of a 128 x 32 tile (row 8 (e >> 6) + (e & 7),
// K-group (e >> 3) & 7) sits at byte 16 e, so core matrices are 128 B apart along K and
// 1024 B apart along the rows.
// ---------------------------------------------------------------------------------------

// Slot e of a stage: its row and first K index (within the tile).
__device__ __forceinline__ void tc_slot(int e, int& r, int& kk) {
  r = ((e >> 6) << 3) + (e & 7);
  kk = ((e >> 3) & 7) << 2;
}

__device__ __forceinline__ void tc_store_split(float* hi, float* lo, int e, float4 v) {
  float4 h, l;
  tf32_split(v.x, h.x, l.x);
  tf32_split(v.y, h.y, l.y);
  tf32_split(v.z, h.z, l.z);
  tf32_split(v.w, h.w, l.w);
  reinterpret_cast<float4*>(hi)[e] = h;
  reinterpret_cast<float4*>(lo)[e] = l;
}

// Issues the 3xTF32 MMAs of one staged chunk (ksteps K-steps of 8) into TMEM column base d
// and commits them to the MMA mbarrier; thread 0 only.
__device__ __forceinline__ void tc_issue_chunk(const float* st, uint32_t d, uint32_t idesc,
                                               int ksteps, bool first, uint64_t* bar) {
  tc_fence_after_sync();
  const float* ahi = st;
  const float* alo = st + TC_TILE * TC_KC;
  const float* bhi = st + 2 * TC_TILE * TC_KC;
  const float* blo = st + 3 * TC_TILE * TC_KC;
  for (int s = 0; s < ksteps; ++s) {
    const int off = s * 64;  // two core matrices (8 K-elements) per step
    const uint64_t a_h = tc_smem_desc(ahi + off, 128, 1024);
    const uint64_t a_l = tc_smem_desc(alo + off, 128, 1024);
    const uint64_t b_h = tc_smem_desc(bhi + off, 128, 1024);
    const uint64_t b_l = tc_smem_desc(blo + off, 128, 1024);
    tc_mma_tf32(d, a_h, b_h, idesc, (first && s == 0) ? 0u : 1u);
    tc_mma_tf32(d, a_h, b_l, idesc, 1u);
    tc_mma_tf32(d, a_l, b_h, idesc, 1u);
  }
  tc_commit(bar);
}

// Waits for the chunk's MMAs (bounded); on a timeout every thread learns of it, the status
// word records it, and the copies get one more bounded wait.  False on timeout.
template <typename T>
__device__ bool tc_wait(Ctx<T>& c) {
  const bool ok = mbar_wait_bounded(c.bar + 1, c.mma_phase);
  c.mma_phase ^= 1u;
  if (__syncthreads_or(!ok)) {
    if (c.tid == 0) atomicOr(c.p.status, ST_TIMEOUT);
    if (!ok) mbar_wait_bounded(c.bar + 1, c.mma_phase ^ 1u);
    c.failed = true;
    return false;
  }
  return true;
}

// Global rows of B^T for a stage: slots e = tid, tid + NT, ... (1024 slots per 128 x 32).
constexpr int TC_SLOTS = TC_TILE * TC_KC / 4;
constexpr int TC_PER_T = TC_SLOTS / NT;

template <typename T>
__device__ __forceinline__ void tc_load_bt(const Ctx<T>& c, int r0, int k0, float4* v) {
  const int n = c.p.n;
#pragma unroll
  for (int q = 0; q < TC_PER_T; ++q) {
    int r, kk;
    tc_slot(c.tid + q * NT, r, kk);
    r += r0;
    kk += k0;
    v[q] = (r < n && kk < n)
               ? __ldcg(reinterpret_cast<const float4*>(c.B + (size_t)r * c.bs + kk))
               : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Releases the flush's TMEM (every MMA has completed or its wait ran out twice).
template <typename T>
__device__ __forceinline__ void tc_release(Ctx<T>& c) {
  tc_fence_before_sync();
  __syncthreads();
  if (c.warp == 0) tmem_dealloc(c.sc->tmem, TC_COLS);
}

// One row tile of the flush for a window of mp <= 32 columns, the X accumulator of rows
// r0..r0+127 in TMEM columns 0..mp-1: Y = (X - P) S^-T by the warps of the four lane
// quadrants, one row per thread, written as the update's A operand (hi/lo, K = mp); then
// B^T[r0..][j0..] -= Y snap[.][j0..] for every 128-column tile j0 (K = mp in one chunk),
// snap's rows j read as float4 runs of the [n][mp] snapshot, the tile's B^T loaded before
// the MMAs and read-modify-written after them.  False (TMEM released) if a wait ran out.
template <typename T>
__device__ bool flush_tile_update_tc(Ctx<T>& c, int r0, uint32_t tm, uint32_t lane_base,
                                     uint32_t id2, const float* snapt) {
  const Params& p = c.p;
  const int m = c.sc->m, n = p.n, bs = c.bs;
  const int mp = (m + 15) & ~15;
  float* st = c.tcs;
  float* ahi = st;
  float* alo = st + TC_TILE * TC_KC;
  float* bhi = st + 2 * TC_TILE * TC_KC;
  float* blo = st + 3 * TC_TILE * TC_KC;
  if (c.warp < 4) {
    // 16 columns of Y at a time from 16 columns of X at a time (registers stay few: the
    // flush runs inside the move loop)
    const int rr = c.warp * 32 + c.lane, r = r0 + rr;
    for (int bh = 0; bh < mp; bh += 16) {
      float y[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) y[q] = 0.f;
      for (int lc = 0; lc < mp; lc += 16) {
        float x[16];
        tmem_ld16(tm + lane_base + (uint32_t)lc, x);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int l = lc + q;
          x[q] = (l < m && r < n) ? x[q] - ((r == c.wP[l]) ? 1.f : 0.f) : 0.f;
        }
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          if (bh + b < m) {
            const float* srow = c.wS + (size_t)(bh + b) * p.ks + lc;
            float acc = y[b];
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (lc + q < m) acc += x[q] * srow[q];
            y[b] = acc;
          }
        }
      }
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const int e = ((rr >> 3) << 6) | (((bh >> 2) + g) << 3) | (rr & 7);
        tc_store_split(ahi, alo, e, make_float4(y[4 * g], y[4 * g + 1], y[4 * g + 2], y[4 * g + 3]));
      }
    }
  }
  tc_fence_before_sync();  // X is read from TMEM before the update's MMAs overwrite it
  // The tile of B^T moves through shared memory in two halves of 64 columns (the B operand's
  // stage, free once the MMAs are done), so that its global reads and writes are coalesced
  // (a warp takes two whole 256-byte row pieces) while each thread still handles one row
  // against its TMEM lane; float4 slot c of row r sits at c ^ (r & 15) (no bank conflicts)
  constexpr int HALF_F4 = TC_TILE * 16;        // float4 of a 128 x 64 half tile
  constexpr int PER_T = 2 * HALF_F4 / NT;      // both halves' float4 per thread
  float4* buf = reinterpret_cast<float4*>(bhi);  // bhi, blo: 32 KB, contiguous
  const int rq = (c.warp & 3) * 32 + c.lane;   // this thread's row of the tile (TMEM lane)
  const int cg = c.warp >> 2;                  // its group of columns
  constexpr int NG = NWARP / 4;                // groups: 64 / NG columns of a half each
  for (int j0 = 0; j0 < n; j0 += TC_TILE) {
    float4 pre[PER_T];  // the tile, loaded before the MMAs (coalesced)
#pragma unroll
    for (int q = 0; q < PER_T; ++q) {
      const int idx = c.tid + q * NT;
      const int h = idx / HALF_F4, e = idx - h * HALF_F4;
      const int row = e >> 4, c4 = e & 15;
      const int r = r0 + row, j = j0 + 64 * h + 4 * c4;
      pre[q] = (r < n && j < n)
                   ? __ldcg(reinterpret_cast<const float4*>(c.B + (size_t)r * bs + j))
                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // snap as the B operand: rows j, K = b; all of this thread's runs loaded first
    float4 z[TC_PER_T];
#pragma unroll
    for (int q = 0; q < TC_PER_T; ++q) {
      int rr, b;
      tc_slot(c.tid + q * NT, rr, b);
      const int j = j0 + rr;
      z[q] = (j < n && b < mp)
                 ? __ldcg(reinterpret_cast<const float4*>(snapt + (size_t)j * mp + b))
                 : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < TC_PER_T; ++q) {
      int rr, b;
      tc_slot(c.tid + q * NT, rr, b);
      if (b < mp) tc_store_split(bhi, blo, c.tid + q * NT, z[q]);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (c.tid == 0) tc_issue_chunk(st, tm, id2, mp / 8, true, c.bar + 1);
    if (!tc_wait(c)) {
      tc_release(c);
      return false;
    }
    tc_fence_after_sync();
    for (int h = 0; h < 2; ++h) {
      if (j0 + 64 * h >= n) break;  // uniform
#pragma unroll
      for (int q = 0; q < PER_T; ++q) {
        const int idx = c.tid + q * NT;
        if (idx / HALF_F4 == h) {
          const int e = idx - h * HALF_F4, row = e >> 4, c4 = e & 15;
          buf[row * 16 + (c4 ^ (row & 15))] = pre[q];
        }
      }
      __syncthreads();
      constexpr int COLS = 64 / NG;  // columns of this thread's group in a half
#pragma unroll
      for (int cc = 0; cc < COLS; cc += 16) {
        const int c0 = 64 * h + cg * COLS + cc;  // column within the tile
        float d[16];
        tmem_ld16(tm + lane_base + (uint32_t)c0, d);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c4 = ((c0 - 64 * h) >> 2) + q;
          float4& v = buf[rq * 16 + (c4 ^ (rq & 15))];
          float4 b = v;
          b.x -= d[4 * q];
          b.y -= d[4 * q + 1];
          b.z -= d[4 * q + 2];
          b.w -= d[4 * q + 3];
          v = b;
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < PER_T; ++q) {
        const int idx = c.tid + q * NT;
        if (idx / HALF_F4 == h) {
          const int e = idx - h * HALF_F4, row = e >> 4, c4 = e & 15;
          const int r = r0 + row, j = j0 + 64 * h + 4 * c4;
          if (r < n && j < n)  // n % 4 == 0: whole float4 groups in or out
            *reinterpret_cast<float4*>(c.B + (size_t)r * bs + j) =
                buf[row * 16 + (c4 ^ (row & 15))];
        }
      }
      __syncthreads();
    }
    tc_fence_before_sync();
    __syncthreads();
  }
  return true;
}

// The window's rows of B^T before the update (snap), X^T and Y^T live in the walker's
// global scratch [3][k][n] (L2-resident), which keeps the flush's shared memory to the
// operand stages: delay ranks up to 64 fit next to the staged stencil.
template <typename T>
__device__ void flush_window_tc(Ctx<T>& c) {
  if constexpr (IsMixed<T>::value) {
    const Params& p = c.p;
    const int m = c.sc->m;
    if (m == 0) return;
    const int n = p.n, bs = c.bs;
    const int mp = (m + 15) & ~15;  // N of the first product, K of the second
    float* scr = (float*)p.flush_scratch + (size_t)c.w * 3 * p.k * n;
    float* snapg = scr;                      // [m][n]: B^T[p_b][j]
    float* xt = scr + (size_t)p.k * n;       // [m][n]: X^T[l][r]
    float* yt = scr + (size_t)2 * p.k * n;   // [m][n]: Y^T[b][r]
    // Row tiles one at a time when the window has at most 32 columns (and the scratch holds
    // the snapshot as [n][mp]): Y's rows depend on X's same rows only, so each tile goes
    // X -> Y (from TMEM into registers, S^-1 from shared memory) -> B^T -= Y snap while
    // its rows of B^T are still in L2.  Only for n >= 512: a smaller inverse stays in L2
    // between the passes anyway, and there the three-pass order measured faster (pw512,
    // n = 256: 42.2 against 43.7 ms per generation)
    const bool fused = mp <= TC_KC && mp <= 3 * p.k && n >= 512;
    if (c.warp == 0) tmem_alloc(&c.sc->tmem, TC_COLS);
    // snapshot of the window's rows of B^T before the update ([m][n], or [n][mp] with the
    // columns m..mp-1 zero when fused, so that a row of the update's B operand is one
    // contiguous run)
    if (fused) {
      for (int e = c.tid; e < mp * n; e += NT) {
        const int l = e / n, j = e - l * n;
        snapg[(size_t)j * mp + l] = l < m ? c.B[(size_t)c.wP[l] * bs + j] : 0.f;
      }
    } else {
      for (int e = c.tid; e < m * n; e += NT) {
        const int l = e / n, j = e - l * n;
        snapg[e] = c.B[(size_t)c.wP[l] * bs + j];
      }
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tm = c.sc->tmem;
    const uint32_t lane_base = (uint32_t)((c.warp & 3) * 32) << 16;
    float* st = c.tcs;
    float* ahi = st;
    float* alo = st + TC_TILE * TC_KC;
    float* bhi = st + 2 * TC_TILE * TC_KC;
    float* blo = st + 3 * TC_TILE * TC_KC;
    // ---- X = B^T Phi^T - P (per 128-row tile, K = n in chunks of 32; the B^T chunks are
    // loaded two ahead, so two of them are in flight while a chunk's MMAs run)
    const uint32_t id1 = tc_idesc_tf32((uint32_t)mp);
    const uint32_t id2 = tc_idesc_tf32((uint32_t)TC_TILE);
    for (int r0 = 0; r0 < n; r0 += TC_TILE) {
      // stages chunk k0 from v, issues its MMAs, reloads v with chunk k0 + 2 TC_KC, waits
      auto x_chunk = [&](int k0, float4 (&v)[TC_PER_T]) -> bool {
#pragma unroll
        for (int q = 0; q < TC_PER_T; ++q) tc_store_split(ahi, alo, c.tid + q * NT, v[q]);
        for (int e = c.tid; e < mp * 8; e += NT) {  // Phi rows l < m, zero rows up to mp
          int l, kk;
          tc_slot(e, l, kk);
          kk += k0;
          float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
          if (l < m) {
            const T* vr = c.wV + (size_t)l * p.vs;
            f.x = kk < n ? vr[kk] : 0.f;
            f.y = kk + 1 < n ? vr[kk + 1] : 0.f;
            f.z = kk + 2 < n ? vr[kk + 2] : 0.f;
            f.w = kk + 3 < n ? vr[kk + 3] : 0.f;
          }
          tc_store_split(bhi, blo, e, f);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (c.tid == 0) tc_issue_chunk(st, tm, id1, TC_KC / 8, k0 == 0, c.bar + 1);
        if (k0 + 2 * TC_KC < n) tc_load_bt(c, r0, k0 + 2 * TC_KC, v);
        return tc_wait(c);
      };
      float4 va[TC_PER_T], vb[TC_PER_T];
      tc_load_bt(c, r0, 0, va);
      tc_load_bt(c, r0, TC_KC, vb);  // zeros (no loads) past n
      bool ok = true;
      for (int k0 = 0; k0 < n && ok; k0 += 2 * TC_KC) {
        ok = x_chunk(k0, va);
        if (ok && k0 + TC_KC < n) ok = x_chunk(k0 + TC_KC, vb);
      }
      if (!ok) {
        tc_release(c);
        return;
      }
      tc_fence_after_sync();
      if (fused) {
        if (!flush_tile_update_tc(c, r0, tm, lane_base, id2, snapg)) return;
        continue;
      }
      // epilogue: row r of the tile is TMEM lane r; warps of one lane quadrant split columns
      const int r = r0 + (c.warp & 3) * 32 + c.lane;
      for (int c0 = (c.warp >> 2) * 16; c0 < mp; c0 += (NWARP / 4) * 16) {
        float x[16];
        tmem_ld16(tm + lane_base + (uint32_t)c0, x);
        if (r < n) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int l = c0 + q;
            if (l < m) xt[(size_t)l * n + r] = x[q] - (r == c.wP[l] ? 1.f : 0.f);
          }
        }
      }
      tc_fence_before_sync();
      __syncthreads();
    }
    if (fused) {
      tc_release(c);
      if (c.tid == 0) c.sc->m = 0;
      __syncthreads();
      return;
    }
    // ---- Y = X S^-T (m x m on the CUDA cores; X^T rows from the L2-resident scratch)
    for (int e = c.tid; e < n * m; e += NT) {
      const int b = e / n, r = e - b * n;
      const T* srow = c.wS + (size_t)b * p.ks;
      float acc = 0.f;
      for (int l = 0; l < m; ++l) acc += xt[(size_t)l * n + r] * srow[l];
      yt[e] = acc;
    }
    __syncthreads();
    // ---- B^T -= Y snap (per 128 x 128 output tile, K = mp in chunks of 32)
    // epilogue geometry: row r of the tile is TMEM lane r; the warps of one lane quadrant
    // split the columns into EP_IT groups of 16 per thread
    constexpr int EP_STEP = (NWARP / 4) * 16;
    constexpr int EP_IT = TC_TILE / EP_STEP;
    // groups loaded ahead of the MMAs (at 256 threads, whose register cap is 128, half)
    constexpr int EP_PF = NT >= 256 ? EP_IT / 2 : EP_IT;
    for (int r0 = 0; r0 < n; r0 += TC_TILE) {
      for (int j0 = 0; j0 < n; j0 += TC_TILE) {
        // this thread's part of the B^T tile, loaded while the operands are staged and the
        // MMAs run (only the epilogue below writes the tile)
        const int r = r0 + (c.warp & 3) * 32 + c.lane;
        const int jb = j0 + (c.warp >> 2) * 16;
        float4 bt[EP_PF][4];
#pragma unroll
        for (int it = 0; it < EP_PF; ++it) {
          const int j = jb + it * EP_STEP;
#pragma unroll
          for (int q = 0; q < 4; ++q)  // n % 4 == 0: whole float4 groups in or out
            bt[it][q] = (r < n && j + 4 * q < n)
                            ? __ldcg(reinterpret_cast<const float4*>(c.B + (size_t)r * bs + j) + q)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int b0 = 0; b0 < mp; b0 += TC_KC) {
          for (int e = c.tid; e < TC_SLOTS; e += NT) {
            int rr, kk;
            tc_slot(e, rr, kk);
            const int k = r0 + rr, b = b0 + kk;
            float4 y = make_float4(0.f, 0.f, 0.f, 0.f), z = y;
            if (k < n) {
              y.x = b < m ? yt[(size_t)b * n + k] : 0.f;
              y.y = b + 1 < m ? yt[(size_t)(b + 1) * n + k] : 0.f;
              y.z = b + 2 < m ? yt[(size_t)(b + 2) * n + k] : 0.f;
              y.w = b + 3 < m ? yt[(size_t)(b + 3) * n + k] : 0.f;
            }
            const int j = j0 + rr;  // the B operand's rows are output columns j
            if (j < n) {
              z.x = b < m ? snapg[(size_t)b * n + j] : 0.f;
              z.y = b + 1 < m ? snapg[(size_t)(b + 1) * n + j] : 0.f;
              z.z = b + 2 < m ? snapg[(size_t)(b + 2) * n + j] : 0.f;
              z.w = b + 3 < m ? snapg[(size_t)(b + 3) * n + j] : 0.f;
            }
            tc_store_split(ahi, alo, e, y);
            tc_store_split(bhi, blo, e, z);
          }
          fence_proxy_async_smem();
          __syncthreads();
          const int ks = (mp - b0 < TC_KC ? mp - b0 : TC_KC) / 8;
          if (c.tid == 0) tc_issue_chunk(st, tm, id2, ks, b0 == 0, c.bar + 1);
          if (!tc_wait(c)) {
            tc_release(c);
            return;
          }
        }
        tc_fence_after_sync();
#pragma unroll
        for (int it = 0; it < EP_IT; ++it) {
          const int c0 = (c.warp >> 2) * 16 + it * EP_STEP;
          float d[16];
          tmem_ld16(tm + lane_base + (uint32_t)c0, d);
          const int j = j0 + c0;
          float4* brow = reinterpret_cast<float4*>(c.B + (size_t)r * bs + j);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (r < n && j + 4 * q < n) {
              float4 bv = it < EP_PF ? bt[it < EP_PF ? it : 0][q] : __ldcg(brow + q);
              bv.x -= d[4 * q];
              bv.y -= d[4 * q + 1];
              bv.z -= d[4 * q + 2];
              bv.w -= d[4 * q + 3];
              brow[q] = bv;
            }
          }
        }
        tc_fence_before_sync();
        __syncthreads();
      }
    }
    tc_release(c);
    if (c.tid == 0) c.sc->m = 0;
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void flush_window(Ctx<T>& c) {
  if (c.tc) flush_window_tc(c);
  else flush_window_simt(c);
}

// ---------------------------------------------------------------------------------------
// The move.
// ---------------------------------------------------------------------------------------

// grad_i log Psi at the current positions (the drift F of Alg. 1 line 5): det part
// sum_j dA[i][j] col_j, Jastrow part -sum u'(r) d/r.  Every thread receives F.  Caches
// u(r_old) per partner term in `uo`.  `pf` holds this thread's prefetched gradient-row
// entries (orbital j = tid) when `use_pf` is set.
template <typename T>
__device__ void eval_grad(Ctx<T>& c, int i, const T* pf, bool use_pf, T* uo, T* F) {
  const Params& p = c.p;
  const int n = p.n, n_pad = p.n_pad;
  T v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (use_pf) {
    if (c.tid < n) {
      const T cj = c.col[c.tid];
      v[0] = pf[0] * cj;
      v[1] = pf[1] * cj;
      v[2] = pf[2] * cj;
    }
  } else {
    const T* rw = c.rows + (size_t)i * 5 * n_pad;
    for (int j = c.tid; j < n; j += NT) {
      const T cj = c.col[j];
      v[0] += rw[n_pad + j] * cj;
      v[1] += rw[2 * n_pad + j] * cj;
      v[2] += rw[3 * n_pad + j] * cj;
    }
  }
  int t0, t1;
  term_range(p, t0, t1);
  // partner t (use = false: a placeholder partner in range whose term is discarded)
  auto term = [&](int t, bool use, T& u_out) {
    T d[3], r, rinv;
    partner_disp(c, c.R + 3 * i, c.Rq + 3 * i, t, d, r, rinv);
    const T* coef; int K; T hinv, rc;
    functor(c, i, t, coef, K, hinv, rc);
    T u, du, d2u;
    radial(coef, K, hinv, rc, r, u, du, d2u);
    u_out = u;
    const T f = (use && r > T(0)) ? du * rinv : T(0);
    v[3] += f * d[0];
    v[4] += f * d[1];
    v[5] += f * d[2];
  };
#pragma unroll
  for (int q = 0; q < JT; ++q) {
    if (t0 + q * NT < t1) {
      const int t = t0 + c.tid + q * NT;
      term(t < t1 ? t : t1 - 1, t < t1 && t != i, uo[q]);
    }
  }
  for (int t = t0 + c.tid + JT * NT; t < t1; t += NT) {
    T dummy;
    term(t, t != i, dummy);
  }
  block_allreduce8<NWARP>(v, c.red0);
  for (int k = 0; k < 3; ++k) F[k] = v[k] - v[3 + k];
}

// The drift D(F) = scale F of the proposal (Alg. 1 line 5 read as drift-diffusion): with
// drift == 1 limited as in Umrigar, Nightingale and Runge (1993) with a = 1, scale =
// 2 / (1 + sqrt(1 + 2 tau |F|^2)), so tau |D| < sqrt(2 tau) near a node; drift == 2: D = F;
// drift == 0: no drift.
// The mixed path forms it as 2 r / (1 + r) with r = 1 / sqrt(1 + 2 tau |F|^2) from the
// approximate reciprocal square root and division (a few ulps; the forward and the
// reverse Green's function use the same function, so the Metropolis-Hastings balance is
// exact for it).
template <typename T>
__device__ __forceinline__ T drift_scale(int drift, T tau, const T* F) {
  if (drift == 1) {
    const T f2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    if constexpr (sizeof(T) == 4) {
      const float r = rsqrtf(1.0f + 2.0f * tau * f2);
      return __fdividef(2.0f * r, 1.0f + r);
    } else {
      return T(2) / (T(1) + sqrt(T(1) + T(2) * tau * f2));
    }
  }
  return drift == 2 ? T(1) : T(0);
}

// The proposal r' (given, or r + tau D(F) + sqrt(tau) chi), its spline cell and the
// forward Green's-function exponent.
template <typename T>
__device__ __forceinline__ void make_proposal(const Ctx<T>& c, int i, const T* F, const T* chi,
                                              const double* rgiven, Prop<T>& pr) {
  const Params& p = c.p;
  const T tau = c.k.tau, stau = c.k.stau;
  T gf = 0;
  const T sc = drift_scale(p.drift, tau, F);
  for (int k = 0; k < 3; ++k) pr.F[k] = sc * F[k];
  if constexpr (IsMixed<T>::value) {
    const uint32_t* qi = c.Rq + 3 * i;
    if (!rgiven) {
      // lanes 0-2 of every warp take one dimension each, then share it over the warp
      const int k = c.lane < 3 ? c.lane : 0;
      const float Fk = k == 0 ? pr.F[0] : (k == 1 ? pr.F[1] : pr.F[2]);
      const float d = tau * Fk + stau * chi[k];
      const float dw = d - c.k.L * rintf(d * c.k.invL);  // same point mod L, |dw| <= L/2
      const uint32_t q = qi[k] + (uint32_t)__float2int_rn(dw * c.k.scale);
      const unsigned long long prod = (unsigned long long)q * (unsigned long long)p.G;
      const int cell = (int)(prod >> 32);
      const float t = (float)(uint32_t)prod * 0x1p-32f;
      const float x = d - tau * Fk;
      const unsigned full = 0xffffffffu;
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        pr.disp[kk] = __shfl_sync(full, d, kk);
        pr.rq[kk] = __shfl_sync(full, q, kk);
        pr.cell[kk] = __shfl_sync(full, cell, kk);
        pr.t[kk] = __shfl_sync(full, t, kk);
        const float xk = __shfl_sync(full, x, kk);
        gf += xk * xk;
      }
      pr.logGf = -gf / (T(2) * tau);
      return;
    }
    for (int k = 0; k < 3; ++k) {
      uint32_t q;
      if (rgiven) {
        q = to_fixed(wrap_coord(rgiven[k], p.L, p.invL), p.fx_scale);
        pr.disp[k] = (float)(int32_t)(q - qi[k]) * c.k.unit;
      } else {
        const float d = tau * pr.F[k] + stau * chi[k];
        pr.disp[k] = d;
        const float dw = d - c.k.L * rintf(d * c.k.invL);  // same point mod L, |dw| <= L/2
        q = qi[k] + (uint32_t)__float2int_rn(dw * c.k.scale);
      }
      pr.rq[k] = q;
      const unsigned long long prod = (unsigned long long)q * (unsigned long long)p.G;
      pr.cell[k] = (int)(prod >> 32);
      pr.t[k] = (float)(uint32_t)prod * 0x1p-32f;
      const float x = pr.disp[k] - tau * pr.F[k];
      gf += x * x;
    }
  } else {
    const double* ri = c.R + 3 * i;
    if (rgiven) {
      for (int k = 0; k < 3; ++k) pr.rp[k] = wrap_coord(rgiven[k], p.L, p.invL);
      disp_f64(pr.rp, ri, p.L, p.invL, pr.disp);
    } else {
      for (int k = 0; k < 3; ++k) {
        pr.disp[k] = tau * pr.F[k] + stau * chi[k];
        pr.rp[k] = wrap_coord(ri[k] + pr.disp[k], p.L, p.invL);
      }
    }
    for (int k = 0; k < 3; ++k) {
      const double x = pr.disp[k] - tau * pr.F[k];
      gf += x * x;
      const double s = pr.rp[k] * p.dgrid;
      int g = (int)floor(s);
      g = g > p.G - 1 ? p.G - 1 : (g < 0 ? 0 : g);
      pr.cell[k] = g;
      pr.t[k] = s - (double)g;
    }
  }
  pr.logGf = -gf / (T(2) * tau);
}

// Ring-staged stencil (n_pad > 256): box s of a move holds orbitals
// [RING_ORB (s / 4), RING_ORB (s / 4 + 1)) of the stencil's x-plane s % 4, as [y][z][orbital]
// (4 x 4 x RING_ORB); it lands in slot s % RING_SLOTS on that slot's mbarrier.
template <typename T>
__device__ __forceinline__ uint64_t* ring_bar(const Ctx<T>& c, int slot) {
  return slot == 0 ? c.bar : c.bar + 1 + slot;  // c.bar[1] belongs to the tensor cores
}

template <typename T>
__device__ __forceinline__ void ring_issue(const Ctx<T>& c, const Prop<T>& pr, int s) {
  const int slot = s % RING_SLOTS;
  uint64_t* bar = ring_bar(c, slot);
  fence_proxy_async_smem();  // the slot's previous box was read through the generic proxy
  mbar_arrive_expect_tx(bar, (uint32_t)c.p.stencil_bytes);
  tma_load_4d(c.stc + (size_t)slot * RING_ORB * 16, c.tmap, (s >> 2) * RING_ORB, pr.cell[2],
              pr.cell[1], pr.cell[0] + (s & 3), bar);
}

// Ratio Psi(R')/Psi(R) and grad_i log Psi(R') (Alg. 1 lines 7-8): Jastrow difference over
// all partners, tricubic orbital VGL at r', determinant ratio phi'.col.  Every thread
// gets rhoD and dU; rho and Fp = grad log Psi(R') on every thread in the mixed path and
// on thread 0 in the FP64 path.  phi' stays in shared memory.
template <typename T>
__device__ bool ratio_grad(Ctx<T>& c, int i, const Prop<T>& pr, const T* uo, bool cached,
                           Res<T>& rs) {
  const Params& p = c.p;
  const int n = p.n, n_pad = p.n_pad, GP = p.GP;
  const T* table = (const T*)p.table;
  T cf[16];
  const bool tma = p.use_tma == 1;
  // the ring serves the mixed path with 128 threads (the host enables it only there; the
  // other widths' kernels are compiled without it)
  const bool ring = IsMixed<T>::value && NT == 128 && p.use_tma == 2;
  const int nslab = 4 * ((n + RING_ORB - 1) / RING_ORB);
  if (tma) {
    if (c.tid == 0 && !p.test_no_copy) {  // the whole 4x4x4 x n_pad stencil in one copy
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(c.bar, (uint32_t)p.stencil_bytes);
      tma_load_4d(c.stc, c.tmap, 0, pr.cell[2], pr.cell[1], pr.cell[0], c.bar);
    }
  } else if (ring) {
    if (c.tid == 0 && !p.test_no_copy)  // the first boxes fly during the Jastrow terms
      for (int s = 0; s < RING_SLOTS && s < nslab; ++s) ring_issue(c, pr, s);
  } else if (c.nit > 0) {
    stencil_load(table, GP, n_pad, pr.cell[0], pr.cell[1], pr.cell[2], c.itj[0], c.ita[0], cf);
  }
  T wreg[36];  // x, y, z weights (mixed path: computed by every thread)
  if constexpr (IsMixed<T>::value) {
    basis12(pr.t[1], wreg + 12);
    basis12(pr.t[2], wreg + 24);
  } else {
    if (c.tid < 36) c.sc->wts[c.tid] = basis_one((T)pr.t[c.tid / 12], c.tid % 12);
  }
  T v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int t0, t1;
  term_range(p, t0, t1);
  // partner t (use = false: a placeholder partner in range whose term is discarded)
  auto term = [&](int t, bool use, bool have_old, T uold) {
    T dn[3], rn, rninv;
    partner_disp(c, pr.rp, pr.rq, t, dn, rn, rninv);
    const T* coef; int K; T hinv, rc;
    functor(c, i, t, coef, K, hinv, rc);
    T un, dun, d2n;
    radial(coef, K, hinv, rc, rn, un, dun, d2n);
    if (!have_old) {
      T dol[3], ro, roinv, duo, d2o;
      partner_disp(c, c.R + 3 * i, c.Rq + 3 * i, t, dol, ro, roinv);
      radial(coef, K, hinv, rc, ro, uold, duo, d2o);
    }
    const T f = (use && rn > T(0)) ? dun * rninv : T(0);
    v[4] += use ? un - uold : T(0);
    v[5] += f * dn[0];
    v[6] += f * dn[1];
    v[7] += f * dn[2];
  };
  // the cached terms: a slot q is skipped only when no thread has a partner in it
#pragma unroll
  for (int q = 0; q < JT; ++q) {
    if (t0 + q * NT < t1) {
      const int t = t0 + c.tid + q * NT;
      term(t < t1 ? t : t1 - 1, t < t1 && t != i, cached, uo[q]);
    }
  }
  for (int t = t0 + c.tid + JT * NT; t < t1; t += NT) term(t, t != i, false, T(0));
  const T* wts;
  if constexpr (IsMixed<T>::value) {
    wts = wreg;
  } else {
    __syncthreads();  // weights in shared memory
    wts = c.sc->wts;
  }
  if constexpr (IsMixed<T>::value && NT == 128) {
    if (ring) {
      // each box as it lands: every thread reduces its RING_ORB / NT orbitals' 4 x 4 (y, z)
      // values and adds the x-plane's share of value, gradient and Laplacian (the
      // x-weights of stencil_combine, in the same order); after plane 3 of a chunk its
      // orbitals' rows are final.  Then every thread is past the slot and thread 0
      // refills it with the box RING_SLOTS ahead.
      constexpr int NJ = RING_ORB / NT;
      T wx[12];
      basis12(pr.t[0], wx);
      const T dinv = c.k.dgrid;
      T acc[NJ][5];
#pragma unroll
      for (int u = 0; u < NJ; ++u)
#pragma unroll
        for (int r = 0; r < 5; ++r) acc[u][r] = T(0);
      const uint32_t ph0 = c.tma_phase;
      bool ok = true;
      int s = 0;
      for (; s < nslab; ++s) {
        const int slot = s % RING_SLOTS, a = s & 3;
        ok = mbar_wait_bounded(ring_bar(c, slot), ((ph0 >> slot) ^ (uint32_t)(s / RING_SLOTS)) & 1u);
        if (ok) {
          const T* sl = c.stc + (size_t)slot * RING_ORB * 16 + c.tid;
          // plane a's x-weights (value, first, second derivative) by selects: a register
          // array indexed at run time would live in local memory
          T xa = wx[0], xd = wx[4], xl = wx[8];
#pragma unroll
          for (int q = 1; q < 4; ++q)
            if (a == q) {
              xa = wx[q];
              xd = wx[4 + q];
              xl = wx[8 + q];
            }
#pragma unroll
          for (int u = 0; u < NJ; ++u) {
#pragma unroll
            for (int bc = 0; bc < 16; ++bc) cf[bc] = sl[bc * RING_ORB + u * NT];
            T o4[4];
            stencil_reduce(cf, wts, o4);
            acc[u][0] += xa * o4[0];
            acc[u][1] += xd * o4[0];
            acc[u][2] += xa * o4[1];
            acc[u][3] += xa * o4[2];
            acc[u][4] += xl * o4[0] + xa * o4[3];
          }
          if (a == 3) {
#pragma unroll
            for (int u = 0; u < NJ; ++u) {
              const int j = (s >> 2) * RING_ORB + c.tid + u * NT;
              if (j < n) {
                const T o5[5] = {acc[u][0], acc[u][1] * dinv, acc[u][2] * dinv, acc[u][3] * dinv,
                                 acc[u][4] * dinv * dinv};
#pragma unroll
                for (int q = 0; q < 5; ++q) c.phi[q * n_pad + j] = o5[q];
                const T cj = c.col[j];
                v[0] += o5[0] * cj;
                v[1] += o5[1] * cj;
                v[2] += o5[2] * cj;
                v[3] += o5[3] * cj;
              }
#pragma unroll
              for (int r = 0; r < 5; ++r) acc[u][r] = T(0);
            }
          }
        }
        if (__syncthreads_or(!ok)) break;  // uniform: every thread leaves together
        if (c.tid == 0 && s + RING_SLOTS < nslab && !p.test_no_copy) ring_issue(c, pr, s + RING_SLOTS);
      }
      if (s < nslab) {
        // a box that never landed: record it, give every box still in flight one more
        // bounded wait, and leave the kernel
        if (c.tid == 0) atomicOr(p.status, ST_TIMEOUT);
        for (int t = s; t < nslab && t < s + RING_SLOTS; ++t) {
          const int slot = t % RING_SLOTS;
          mbar_wait_bounded(ring_bar(c, slot), ((ph0 >> slot) ^ (uint32_t)(t / RING_SLOTS)) & 1u);
        }
        return false;
      }
      // each slot's phase after this move's boxes
      uint32_t ph = ph0;
      for (int slot = 0; slot < RING_SLOTS; ++slot) {
        const int uses = nslab / RING_SLOTS + (slot < nslab % RING_SLOTS ? 1 : 0);
        if (uses & 1) ph ^= 1u << slot;
      }
      c.tma_phase = ph;
    }
  }
  if (!ring) {
  bool ok = true;
  if (tma) {
    ok = mbar_wait_bounded(c.bar, c.tma_phase);
    c.tma_phase ^= 1u;
  }
  // with TMA staging, the shared-memory reads of the first two items are issued together
  if (tma && c.nit >= 2) {
    T cg[16];
    const T* sa = c.stc + (size_t)(c.ita[0] * 16) * n_pad + c.itj[0];
    const T* sb = c.stc + (size_t)(c.ita[1] * 16) * n_pad + c.itj[1];
#pragma unroll
    for (int bc = 0; bc < 16; ++bc) {
      cf[bc] = sa[(size_t)bc * n_pad];
      cg[bc] = sb[(size_t)bc * n_pad];
    }
    T o4[4], o4b[4];
    stencil_reduce(cf, wts, o4);
    stencil_reduce(cg, wts, o4b);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      c.part[(c.ita[0] * 4 + r) * n_pad + c.itj[0]] = o4[r];
      c.part[(c.ita[1] * 4 + r) * n_pad + c.itj[1]] = o4b[r];
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < c.nit && !(tma && c.nit >= 2 && q < 2)) {
      if (tma) {
        const T* sb = c.stc + (size_t)(c.ita[q] * 16) * n_pad + c.itj[q];
#pragma unroll
        for (int bc = 0; bc < 16; ++bc) cf[bc] = sb[(size_t)bc * n_pad];
      } else if (q > 0) {
        stencil_load(table, GP, n_pad, pr.cell[0], pr.cell[1], pr.cell[2], c.itj[q], c.ita[q], cf);
      }
      T o4[4];
      stencil_reduce(cf, wts, o4);
      const int j = c.itj[q], a = c.ita[q];
#pragma unroll
      for (int r = 0; r < 4; ++r) c.part[(a * 4 + r) * n_pad + j] = o4[r];
    }
  }
  // items beyond four per thread, two per pass so that both items' loads are in flight
  int it = c.tid + 4 * NT;
  for (; it + NT < 4 * n; it += 2 * NT) {
    const int j = it % n, a = it / n, j2 = (it + NT) % n, a2 = (it + NT) / n;
    T cg[16];
    if (tma) {
      const T* sa = c.stc + (size_t)(a * 16) * n_pad + j;
      const T* sb = c.stc + (size_t)(a2 * 16) * n_pad + j2;
#pragma unroll
      for (int bc = 0; bc < 16; ++bc) {
        cf[bc] = sa[(size_t)bc * n_pad];
        cg[bc] = sb[(size_t)bc * n_pad];
      }
    } else {
      stencil_load(table, GP, n_pad, pr.cell[0], pr.cell[1], pr.cell[2], j, a, cf);
      stencil_load(table, GP, n_pad, pr.cell[0], pr.cell[1], pr.cell[2], j2, a2, cg);
    }
    T o4[4], o4b[4];
    stencil_reduce(cf, wts, o4);
    stencil_reduce(cg, wts, o4b);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      c.part[(a * 4 + r) * n_pad + j] = o4[r];
      c.part[(a2 * 4 + r) * n_pad + j2] = o4b[r];
    }
  }
  for (; it < 4 * n; it += NT) {
    const int j = it % n, a = it / n;
    if (tma) {
      const T* sb = c.stc + (size_t)(a * 16) * n_pad + j;
      for (int bc = 0; bc < 16; ++bc) cf[bc] = sb[(size_t)bc * n_pad];
    } else {
      stencil_load(table, GP, n_pad, pr.cell[0], pr.cell[1], pr.cell[2], j, a, cf);
    }
    T o4[4];
    stencil_reduce(cf, wts, o4);
#pragma unroll
    for (int r = 0; r < 4; ++r) c.part[(a * 4 + r) * n_pad + j] = o4[r];
  }
  if (tma) {
    // a stencil copy that never lands: record it, give the copy one more bounded wait,
    // and leave the kernel (uniformly, every thread sees the vote)
    if (__syncthreads_or(!ok)) {
      if (c.tid == 0) atomicOr(p.status, ST_TIMEOUT);
      if (!ok) mbar_wait_bounded(c.bar, c.tma_phase ^ 1u);
      return false;
    }
  } else {
    __syncthreads();
  }
  const T dinv = c.k.dgrid;
  for (int j = c.tid; j < n; j += NT) {
    T wx[12];
    if constexpr (IsMixed<T>::value) {
      basis12(pr.t[0], wx);
    } else {
      for (int q = 0; q < 12; ++q) wx[q] = c.sc->wts[q];
    }
    T o5[5];
    stencil_combine(c.part, n_pad, j, wx, dinv, o5);
#pragma unroll
    for (int q = 0; q < 5; ++q) c.phi[q * n_pad + j] = o5[q];
    const T cj = c.col[j];
    v[0] += o5[0] * cj;
    v[1] += o5[1] * cj;
    v[2] += o5[2] * cj;
    v[3] += o5[3] * cj;
  }
  }  // !ring
  block_allreduce8<NWARP>(v, c.red1);
  rs.rhoD = v[0];
  rs.dU = v[4];
  if constexpr (IsMixed<T>::value) {
    rs.rho = v[0] * __expf(-v[4]);
    const T ir = T(1) / v[0];
    for (int k = 0; k < 3; ++k) rs.Fp[k] = v[1 + k] * ir - v[5 + k];
  } else if (c.tid == 0) {  // FP64 scalar work on one thread; the caller syncs
    rs.rho = v[0] * exp(-v[4]);
    for (int k = 0; k < 3; ++k) rs.Fp[k] = v[1 + k] / v[0] - v[5 + k];
  }
  return true;
}

// Metropolis(-Hastings): A = rho^2 G(r<-r')/G(r'<-r) with drift (G(b<-a) =
// exp(-|b - a - tau D(F(a))|^2 / (2 tau))), rho^2 without;
// accept iff u < A; rho = 0 or non-finite rejects (a non-finite ratio also sets the NaN
// status), and with DMC (fixed node) so does a change of the determinant's sign.  The decision is that of FP64 arithmetic on the
// move's ratio, displacement and drifts with the 53-bit uniform of the Philox draw
// (walker w, electron i): the mixed path evaluates A in FP32 with the 24-bit uniform of
// the same draw, and only where u lies within those roundings of A (about one move in
// 10^5) does every thread take the decision again in FP64.
// (Everything by value: taking the address of the kernel parameter block or of register
// values would move them to local memory for the whole kernel.)
static __device__ __noinline__ int metropolis_fp64_redo(uint64_t seed, uint32_t gen, int drift,
                                                        double tau, float3 disp, float3 Fp,
                                                        float rho, float logGf, int w, int i) {
  const double u = accept_uniform(seed, (uint32_t)w, gen, (uint32_t)i);
  double A = (double)rho * (double)rho;
  if (drift) {
    const double F[3] = {(double)Fp.x, (double)Fp.y, (double)Fp.z};
    const double d[3] = {(double)disp.x, (double)disp.y, (double)disp.z};
    const double sc = drift_scale(drift, tau, F);
    double gb = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double x = -d[q] - tau * sc * F[q];
      gb += x * x;
    }
    A *= exp(-gb / (2.0 * tau) - (double)logGf);
  }
  return u < A ? 1 : 0;
}

template <typename T>
__device__ __forceinline__ int metropolis(const Params& p, const Cst<T>& k, const Prop<T>& pr,
                                          const Res<T>& rs, T u, int w, int i) {
  const T rho = rs.rho;
  if (!isfinite(rho)) {  // rejected, and reported as a non-finite ratio
    if (threadIdx.x == 0) atomicOr(p.status, ST_NAN);
    return 0;
  }
  if (rho == T(0)) return 0;
  if (p.dmc && rs.rhoD < T(0)) return 0;  // fixed node: no crossing of a nodal surface
  T A, scale = T(1);
  if (p.drift) {
    T gb = 0;
    const T sc = drift_scale(p.drift, k.tau, rs.Fp);
    for (int q = 0; q < 3; ++q) {
      const T x = -pr.disp[q] - k.tau * sc * rs.Fp[q];
      gb += x * x;
    }
    const T e1 = gb / (T(2) * k.tau);
    A = rho * rho * exp(-e1 - pr.logGf);
    scale += e1 + fabs(pr.logGf);
  } else {
    A = rho * rho;
  }
  if constexpr (IsMixed<T>::value) {
    // |A32 - A| <= 2^-19 (1 + |exponent terms|) A, |u24 - u53| <= 2^-24
    const float margin = 0x1p-19f * scale * A + 0x1p-23f;
    if (!(fabsf(u - A) > margin))
      return metropolis_fp64_redo(p.seed, p.gen, p.drift, p.tau,
                                  make_float3(pr.disp[0], pr.disp[1], pr.disp[2]),
                                  make_float3(rs.Fp[0], rs.Fp[1], rs.Fp[2]), rho, pr.logGf,
                                  w, i);
  }
  return u < A ? 1 : 0;
}

// Accepting the pending move of electron i (row pp of spin s): inverse update, rows of A,
// dA, d2A replaced, position and log|det| updated.
template <typename T>
__device__ void accept_update(Ctx<T>& c, int i, int s, int pp, const Prop<T>& pr, T rhoD) {
  const Params& p = c.p;
  const int n = p.n, n_pad = p.n_pad, bs = c.bs;
  T* rw = c.rows + (size_t)i * 5 * n_pad;
  if (c.upd == 0) {
    // Sherman-Morrison: v_k = phi'.B^T[k], then B^T[k] -= col (v_k - delta_k,pp) / rhoD:
    // by row owners (2 or 4 threads per row) in FP32, else one thread per row for v
    // (f_k in `part`) and one warp per row for the update.
    const T invr = T(1) / rhoD;
    T* fk = c.part;
    // threads per row: 4 or 2 when the CTA covers the rows that way (float4 reads of a
    // part of the row each, combined by shuffles), else one thread per row
    int tpr = 0;
    if constexpr (sizeof(T) == 4) {
      if (bs % 4 == 0) {
        if (4 * n <= NT && n % 16 == 0) tpr = 4;
        else if (2 * n <= NT && n % 8 == 0) tpr = 2;
      }
    }
    if (tpr) {
      if constexpr (sizeof(T) == 4) {
        // row owners: the tpr threads of row k dot phi' with their parts of the row
        // (float4 reads), combine by shuffles and update the same parts, so the two passes
        // need no barrier between them
        const int k = c.tid / tpr, qd = c.tid % tpr, nq = n / tpr;  // nq floats per part
        float4* r4 = reinterpret_cast<float4*>(c.B + (size_t)(k < n ? k : 0) * bs + qd * nq);
        const float4* p4 = reinterpret_cast<const float4*>(c.phi + qd * nq);
        const float4* c4 = reinterpret_cast<const float4*>(c.col + qd * nq);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (k < n) {
          for (int q = 0; q < nq / 4; ++q) {
            const float4 b = r4[q], f = p4[q];
            a0 += b.x * f.x;
            a1 += b.y * f.y;
            a2 += b.z * f.z;
            a3 += b.w * f.w;
          }
        }
        float acc = (a0 + a1) + (a2 + a3);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (tpr == 4) acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (k < n) {
          const float f = (acc - (k == pp ? 1.f : 0.f)) * invr;
          for (int q = 0; q < nq / 4; ++q) {
            float4 b = r4[q];
            const float4 cv = c4[q];
            b.x -= cv.x * f;
            b.y -= cv.y * f;
            b.z -= cv.z * f;
            b.w -= cv.w * f;
            r4[q] = b;
          }
        }
      }
    } else {
      for (int k = c.tid; k < n; k += NT) {
        const T* row = c.B + (size_t)k * bs;
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int j = 0;
        for (; j + 4 <= n; j += 4) {
          a0 += row[j] * c.phi[j];
          a1 += row[j + 1] * c.phi[j + 1];
          a2 += row[j + 2] * c.phi[j + 2];
          a3 += row[j + 3] * c.phi[j + 3];
        }
        for (; j < n; ++j) a0 += row[j] * c.phi[j];
        fk[k] = ((a0 + a1) + (a2 + a3) - (k == pp ? T(1) : T(0))) * invr;
      }
      __syncthreads();
      // B^T[k][j] -= col[j] f_k: each warp takes rows warp, warp + NWARP, ...; four rows at
      // a time with every load issued before the stores (the compiler cannot prove that
      // the row, col and f pointers do not alias)
      for (int k0 = c.warp; k0 < n; k0 += 4 * NWARP) {
        T f[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int k = k0 + r * NWARP;
          f[r] = k < n ? fk[k] : T(0);
        }
        for (int j0 = 0; j0 < n; j0 += 64) {
          const int ja = j0 + c.lane, jb = j0 + 32 + c.lane;
          const T ca = ja < n ? c.col[ja] : T(0), cb = jb < n ? c.col[jb] : T(0);
          T va[4], vb[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int k = k0 + r * NWARP;
            const T* row = c.B + (size_t)k * bs;
            va[r] = (k < n && ja < n) ? row[ja] : T(0);
            vb[r] = (k < n && jb < n) ? row[jb] : T(0);
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int k = k0 + r * NWARP;
            T* row = c.B + (size_t)k * bs;
            if (k < n && ja < n) row[ja] = va[r] - ca * f[r];
            if (k < n && jb < n) row[jb] = vb[r] - cb * f[r];
          }
        }
      }
    }
  } else {
    // Delayed: a row already in the window is applied first; then append p_m = pp,
    // Phi_m = phi', border S^-1 with b = y, c_l = Phi_m.B[:,p_l], d = Phi_m.B[:,pp]
    // and sigma = d - c.z (= rhoD).
    int m = c.sc->m;
#if QMCGB_CHECK
    // the window holds at most k - 1 rows before an append (a full window was flushed);
    // a bad count is recorded and the window restarted empty (its rows are lost)
    if (!QMC_CHECKP(p, m >= 0 && m < p.k && m < MAX_K, CK_WINDOW, m)) m = 0;
#endif
    bool dup = false;
    for (int l = 0; l < m; ++l) dup |= (c.wP[l] == pp);
    // with the flush's operand stage over phi', the five new rows go out and phi' itself
    // moves into the window's free slot m before any flush can overwrite it
    const bool over = c.tc_over_move;
    if (over) {
      for (int j = c.tid; j < n; j += NT) {
#pragma unroll
        for (int q = 0; q < 5; ++q) rw[q * n_pad + j] = c.phi[q * n_pad + j];
      }
      T* vs = c.wV + (size_t)m * p.vs;
      for (int j = c.tid; j < n; j += NT) vs[j] = c.phi[j];
      __syncthreads();
    }
    if (dup) {
      flush_window(c);  // applies slots l < m; slot m is not read
      if (over) {  // the saved row to slot 0
        const T* vs = c.wV + (size_t)m * p.vs;
        for (int j = c.tid; j < n; j += NT) c.wV[j] = vs[j];
      }
      m = 0;
    }
    T* vm = c.wV + (size_t)m * p.vs;
    if (!over)
      for (int j = c.tid; j < n; j += NT) vm[j] = c.phi[j];
    if (c.tid == 0) c.wP[m] = pp;
    __syncthreads();
    for (int l = c.warp; l <= m; l += NWARP) {
      const T* brow = c.B + (size_t)(l < m ? c.wP[l] : pp) * bs;
      T acc = 0;
      for (int j = c.lane; j < n; j += 32) acc += vm[j] * brow[j];
      acc = warp_sum(acc);
      if (c.lane == 0) c.wc[l] = acc;
    }
    __syncthreads();
    if (m == 0) {
      if (c.tid == 0) c.wS[0] = T(1) / c.wc[0];
    } else {
      for (int b = c.tid; b < m; b += NT) {  // w = c^T S^-1
        T acc = 0;
        for (int l = 0; l < m; ++l) acc += c.wc[l] * c.wS[(size_t)l * p.ks + b];
        c.wb[b] = acc;
      }
      if (c.warp == NWARP - 1) {
        T acc = 0;
        for (int l = c.lane; l < m; l += 32) acc += c.wc[l] * c.wz[l];
        acc = warp_sum(acc);
        if (c.lane == 0) c.wc[MAX_K] = T(1) / (c.wc[m] - acc);  // 1 / sigma
      }
      __syncthreads();
      const T isg = c.wc[MAX_K];
      const int m1 = m + 1;
      for (int e = c.tid; e < m1 * m1; e += NT) {
        const int a = e / m1, b = e - a * m1;
        T* sab = c.wS + (size_t)a * p.ks + b;
        if (a < m && b < m) *sab += c.wz[a] * c.wb[b] * isg;
        else if (a < m) *sab = -c.wz[a] * isg;
        else if (b < m) *sab = -c.wb[b] * isg;
        else *sab = isg;
      }
    }
    if (c.tid == 0) c.sc->m = m + 1;
    __syncthreads();
    if (m + 1 >= p.k) flush_window(c);
  }
  if (!(c.upd == 1 && c.tc_over_move)) {
    for (int j = c.tid; j < n; j += NT) {
#pragma unroll
      for (int q = 0; q < 5; ++q) rw[q * n_pad + j] = c.phi[q * n_pad + j];
    }
  }
  if (c.tid == 0) {
    for (int k = 0; k < 3; ++k) {
      if constexpr (IsMixed<T>::value) c.Rq[3 * i + k] = pr.rq[k];
      else c.R[3 * i + k] = pr.rp[k];
    }
    if constexpr (IsMixed<T>::value) {
      const float y = logf(fabsf(rhoD)) - c.sc->lcomp[s];
      const float t = c.sc->lsum[s] + y;
      c.sc->lcomp[s] = (t - c.sc->lsum[s]) - y;
      c.sc->lsum[s] = t;
    } else {
      c.sc->logdet[s] += log(fabs(rhoD));
    }
    if (rhoD < T(0)) c.sc->sign[s] = -c.sc->sign[s];
  }
  __syncthreads();
}

// Local energy (Alg. 1 line 11): E_L = -1/2 sum_i [lap_i log Psi + |grad_i log Psi|^2] + V,
// with grad_i log D = sum_j dA[i][j] Ainv[j][i], lap_i D / D = sum_j d2A[i][j] Ainv[j][i];
// one warp per electron, lanes over partners (no atomics); FP64 accumulation.
template <typename T>
__device__ double local_energy(Ctx<T>& c) {
  const Params& p = c.p;
  const int N = p.N, n = p.n, n_pad = p.n_pad, NI = p.n_ions;
  double kin = 0.0, pot = 0.0;
  for (int i = c.warp; i < N; i += NWARP) {
    T v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = c.lane; t < N + NI; t += 32) {
      if (t == i) continue;
      T d[3], r, rinv;
      partner_disp(c, c.R + 3 * i, c.Rq + 3 * i, t, d, r, rinv);
      const bool jas = t < N ? p.K2 > 0 : p.K1 > 0;
      if (jas && r > T(0)) {
        const T* coef; int K; T hinv, rc;
        functor(c, i, t, coef, K, hinv, rc);
        T u, du, d2u;
        radial(coef, K, hinv, rc, r, u, du, d2u);
        const T f = du * rinv;
        v[0] += f * d[0];
        v[1] += f * d[1];
        v[2] += f * d[2];
        v[3] += d2u + T(2) * f;
      }
      if (p.potential && r < c.k.halfL) {
        if (t < N) {
          if (t > i) v[8] += exp(-r * r);
        } else {
          v[8] += T(-2) * exp(T(-0.5) * r * r);
        }
      }
    }
    const int s = i < p.n_up ? 0 : 1;
    const int pp = i - s * p.n_up;
    const T* brow = c.Bg + ((size_t)s * n + pp) * n;
    const T* rw = c.rows + (size_t)i * 5 * n_pad;
    for (int j = c.lane; j < n; j += 32) {
      const T b = brow[j];
      v[4] += rw[n_pad + j] * b;
      v[5] += rw[2 * n_pad + j] * b;
      v[6] += rw[3 * n_pad + j] * b;
      v[7] += rw[4 * n_pad + j] * b;
    }
    {
      const T t8 = warp_sum8_transposed(v);  // lane 4q holds the total of value q
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = __shfl_sync(0xffffffffu, t8, 4 * q);
      v[8] = warp_sum(v[8]);
    }
    if (c.lane == 0) {
      T gd2 = 0, gg = 0;
      for (int k = 0; k < 3; ++k) {
        gd2 += v[4 + k] * v[4 + k];
        const T g = v[4 + k] - v[k];
        gg += g * g;
      }
      kin += (double)(T(-0.5) * ((v[7] - gd2) - v[3] + gg));
      pot += (double)v[8];
    }
  }
  double v2[2] = {kin, pot};
  block_sum_to0<NWARP, 2>(v2, (double*)c.red0);
  return v2[0] + v2[1];  // meaningful on thread 0
}

// ---------------------------------------------------------------------------------------
// Incremental Jastrow (mixed Sherman-Morrison sweep).  c.jgl[i] holds grad_i U and lap_i U
// of every electron at the current positions; an accepted move of electron i replaces
// c.jgl[i] by the values at r' (summed afresh over all partners in the ratio) and adds
// each electron partner's change of its pair term.  The drift then needs no Jastrow pass,
// and E_L no pair derivatives.  Between sweeps the values stay in global memory (p.jgl,
// valid while p.jvalid[w] is set: a recompute, new positions or a fine-grained accept
// clear it); every electron's entry is recomputed whenever its own move is accepted.
// ---------------------------------------------------------------------------------------

// grad U and lap U of every electron over all partners (one warp per electron).
template <typename T>
__device__ void jastrow_gl_all(Ctx<T>& c) {
  const Params& p = c.p;
  const int N = p.N, NI = p.n_ions;
  for (int i = c.warp; i < N; i += NWARP) {
    T g0 = 0, g1 = 0, g2 = 0, l = 0;
    for (int t = c.lane; t < N + NI; t += 32) {
      const bool jas = t < N ? p.K2 > 0 : p.K1 > 0;
      if (t == i || !jas) continue;
      T d[3], r, rinv;
      partner_disp(c, c.R + 3 * i, c.Rq + 3 * i, t, d, r, rinv);
      if (r > T(0)) {
        const T* coef; int K; T hinv, rc;
        functor(c, i, t, coef, K, hinv, rc);
        T u, du, d2u;
        radial(coef, K, hinv, rc, r, u, du, d2u);
        const T f = du * rinv;
        g0 += f * d[0];
        g1 += f * d[1];
        g2 += f * d[2];
        l += d2u + T(2) * f;
      }
    }
    g0 = warp_sum(g0);
    g1 = warp_sum(g1);
    g2 = warp_sum(g2);
    l = warp_sum(l);
    if (c.lane == 0) {
      c.jgl[4 * i] = g0;
      c.jgl[4 * i + 1] = g1;
      c.jgl[4 * i + 2] = g2;
      c.jgl[4 * i + 3] = l;
    }
  }
}

// Determinant part of electron i's drift, dA_i . B[:,p] (col), by one all-reduce.
template <typename T>
__device__ void det_grad(Ctx<T>& c, int i, T* det) {
  const int n = c.p.n, n_pad = c.p.n_pad;
  T v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const T* rw = c.rows + (size_t)i * 5 * n_pad;
  for (int j = c.tid; j < n; j += NT) {
    const T cj = c.col[j];
    v[0] += rw[n_pad + j] * cj;
    v[1] += rw[2 * n_pad + j] * cj;
    v[2] += rw[3 * n_pad + j] * cj;
  }
  block_allreduce8<NWARP>(v, c.red0);
  det[0] = v[0];
  det[1] = v[1];
  det[2] = v[2];
}

// What a move leaves for the accept and the next electron's drift (incremental sweep).
template <typename T>
struct IncOut {
  T dg[JT][4];    // per cached partner slot: change of the partner's grad U (3) and lap U
  T g[4];         // grad U and lap U of the moving electron at r'
  T a[3], b[3];   // dA_{i+1} . B[:,p+1] and dA_{i+1} . B[:,p]
  T e;            // phi' . B[:,p+1]
};

// The ratio of the incremental sweep, in three parts so that the sweep can start a move
// before the previous move's inverse update: stencil_issue (the TMA copy of the stencil),
// jas_inc (the Jastrow terms) and spo_inc (the spline, the determinant sums and the
// all-reduce).  Every partner term is evaluated at r and at r' (u, u', u''), giving the
// moving electron's fresh grad U and lap U at r' and the partners' changes for an accept;
// when `nxt`, the sums a, b, e from which the next electron's determinant drift follows
// after this move (`pf`: that electron's dA entries for orbital j = tid).
template <typename T>
__device__ __forceinline__ void stencil_issue(Ctx<T>& c, const Prop<T>& pr) {
  if (c.p.use_tma == 1 && c.tid == 0 && !c.p.test_no_copy) {  // the whole stencil in one copy
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(c.bar, (uint32_t)c.p.stencil_bytes);
    tma_load_4d(c.stc, c.tmap, 0, pr.cell[2], pr.cell[1], pr.cell[0], c.bar);
  }
}

// jv: dU, grad U (3) and lap U partial sums of this thread's partner slots.
template <typename T>
__device__ __forceinline__ void jas_inc(Ctx<T>& c, int i, const Prop<T>& pr, T* jv,
                                        IncOut<T>& io) {
  const Params& p = c.p;
  int t0, t1;
  term_range(p, t0, t1);
#pragma unroll
  for (int q = 0; q < 5; ++q) jv[q] = T(0);
  // partner slot q of this thread: t = t0 + tid + q NT
  auto slot = [&](int q) {
    const int tq = t0 + c.tid + q * NT;
    const bool use = tq < t1 && tq != i;
    const int t = tq < t1 ? tq : t1 - 1;
    T dn[3], rn, rninv, dol[3], ro, roinv;
    partner_disp(c, pr.rp, pr.rq, t, dn, rn, rninv);
    partner_disp(c, c.R + 3 * i, c.Rq + 3 * i, t, dol, ro, roinv);
    const T* coef; int K; T hinv, rc;
    functor(c, i, t, coef, K, hinv, rc);
    T un, dun, d2n, uo, duo, d2o;
    radial(coef, K, hinv, rc, rn, un, dun, d2n);
    radial(coef, K, hinv, rc, ro, uo, duo, d2o);
    const bool un_ok = use && rn > T(0), uo_ok = use && ro > T(0);
    const T fn = un_ok ? dun * rninv : T(0), fo = uo_ok ? duo * roinv : T(0);
    const T ln = un_ok ? d2n + T(2) * fn : T(0), lo = uo_ok ? d2o + T(2) * fo : T(0);
    jv[0] += use ? un - uo : T(0);
    jv[1] += fn * dn[0];
    jv[2] += fn * dn[1];
    jv[3] += fn * dn[2];
    jv[4] += ln;
    // partner t's pair term: grad_t u = -(u'/r) d, lap_t u = u'' + 2 u'/r
    io.dg[q][0] = fo * dol[0] - fn * dn[0];
    io.dg[q][1] = fo * dol[1] - fn * dn[1];
    io.dg[q][2] = fo * dol[2] - fn * dn[2];
    io.dg[q][3] = ln - lo;
  };
#pragma unroll
  for (int q = 0; q < JT; ++q) io.dg[q][0] = io.dg[q][1] = io.dg[q][2] = io.dg[q][3] = T(0);
  if (t1 - t0 > NT && t1 - t0 <= 2 * NT) {
    // two slots in one block, so their independent chains interleave (the common case:
    // a little more than one partner per thread)
    slot(0);
    slot(1);
  } else {
#pragma unroll
    for (int q = 0; q < JT; ++q)
      if (t0 + q * NT < t1) slot(q);  // slot q has partners for some thread (uniform)
  }
}

// False when the stencil copy timed out (uniform).
template <typename T>
__device__ bool spo_inc(Ctx<T>& c, int i, int pp, const Prop<T>& pr, Res<T>& rs, bool nxt,
                        const T* pf, const T* jv, IncOut<T>& io) {
  const Params& p = c.p;
  const int n = p.n, n_pad = p.n_pad, GP = p.GP;
  const T* table = (const T*)p.table;
  const bool tma = p.use_tma == 1;  // the ring (n_pad > 256) never meets this path
  T cf[16];
  T wreg[36];
  basis12(pr.t[1], wreg + 12);
  basis12(pr.t[2], wreg + 24);
  T v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = T(0);
#pragma unroll
  for (int q = 0; q < 5; ++q) v[4 + q] = jv[q];
  const T* wts = wreg;
  bool ok = true;
  if (tma) {
    ok = mbar_wait_bounded(c.bar, c.tma_phase);
    c.tma_phase ^= 1u;
  }
  if (tma && c.nit >= 2) {
    T cg[16];
    const T* sa = c.stc + (size_t)(c.ita[0] * 16) * n_pad + c.itj[0];
    const T* sb = c.stc + (size_t)(c.ita[1] * 16) * n_pad + c.itj[1];
#pragma unroll
    for (int bc = 0; bc < 16; ++bc) {
      cf[bc] = sa[(size_t)bc * n_pad];
      cg[bc] = sb[(size_t)bc * n_pad];
    }
    T o4[4], o4b[4];
    stencil_reduce(cf, wts, o4);
    stencil_reduce(cg, wts, o4b);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      c.part[(c.ita[0] * 4 + r) * n_pad + c.itj[0]] = o4[r];
      c.part[(c.ita[1] * 4 + r) * n_pad + c.itj[1]] = o4b[r];
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < c.nit && !(tma && c.nit >= 2 && q < 2)) {
      if (tma) {
        const T* sb = c.stc + (size_t)(c.ita[q] * 16) * n_pad + c.itj[q];
#pragma unroll
        for (int bc = 0; bc < 16; ++bc) cf[bc] = sb[(size_t)bc * n_pad];
      } else {
        stencil_load(table, GP, n_pad, pr.cell[0], pr.cell[1], pr.cell[2], c.itj[q], c.ita[q], cf);
      }
      T o4[4];
      stencil_reduce(cf, wts, o4);
      const int j = c.itj[q], a = c.ita[q];
#pragma unroll
      for (int r = 0; r < 4; ++r) c.part[(a * 4 + r) * n_pad + j] = o4[r];
    }
  }
  for (int it = c.tid + 4 * NT; it < 4 * n; it += NT) {  // items beyond four per thread
    const int j = it % n, a = it / n;
    if (tma) {
      const T* sb = c.stc + (size_t)(a * 16) * n_pad + j;
      for (int bc = 0; bc < 16; ++bc) cf[bc] = sb[(size_t)bc * n_pad];
    } else {
      stencil_load(table, GP, n_pad, pr.cell[0], pr.cell[1], pr.cell[2], j, a, cf);
    }
    T o4[4];
    stencil_reduce(cf, wts, o4);
#pragma unroll
    for (int r = 0; r < 4; ++r) c.part[(a * 4 + r) * n_pad + j] = o4[r];
  }
  if (tma) {
    if (__syncthreads_or(!ok)) {
      if (c.tid == 0) atomicOr(p.status, ST_TIMEOUT);
      if (!ok) mbar_wait_bounded(c.bar, c.tma_phase ^ 1u);
      return false;
    }
  } else {
    __syncthreads();
  }
  const T dinv = c.k.dgrid;
  const T* bnext = c.B + (size_t)(pp + 1) * c.bs;  // read only when nxt (pp + 1 < n)
  for (int j = c.tid; j < n; j += NT) {  // n <= NT on this path: j == tid
    T wx[12];
    basis12(pr.t[0], wx);
    T o5[5];
    stencil_combine(c.part, n_pad, j, wx, dinv, o5);
#pragma unroll
    for (int q = 0; q < 5; ++q) c.phi[q * n_pad + j] = o5[q];
    const T cj = c.col[j];
    v[0] += o5[0] * cj;
    v[1] += o5[1] * cj;
    v[2] += o5[2] * cj;
    v[3] += o5[3] * cj;
    if (nxt) {
      const T bn = bnext[j];
      v[9] += pf[0] * bn;
      v[10] += pf[1] * bn;
      v[11] += pf[2] * bn;
      v[12] += pf[0] * cj;
      v[13] += pf[1] * cj;
      v[14] += pf[2] * cj;
      v[15] += o5[0] * bn;
    }
  }
  block_allreduce16<NWARP>(v, c.red1);
  rs.rhoD = v[0];
  rs.dU = v[4];
  rs.rho = v[0] * __expf(-v[4]);
  const T ir = T(1) / v[0];
  for (int k = 0; k < 3; ++k) rs.Fp[k] = v[1 + k] * ir - v[5 + k];
  io.g[0] = v[5];
  io.g[1] = v[6];
  io.g[2] = v[7];
  io.g[3] = v[8];
  for (int k = 0; k < 3; ++k) {
    io.a[k] = v[9 + k];
    io.b[k] = v[12 + k];
  }
  io.e = v[15];
  return true;
}

// The Sherman-Morrison update of an accepted move by row owners (2 or 4 threads per row,
// n <= NT / 2) with the new rows of A written to HBM and log|det| advanced; no barrier
// (the caller's publishes it).  The caller has already moved the electron.
template <typename T>
__device__ __forceinline__ void sm_rows_update(Ctx<T>& c, int i, int s, int pp, T rhoD,
                                               T* cnext) {
  const Params& p = c.p;
  const int n = p.n, n_pad = p.n_pad, bs = c.bs;
  if constexpr (sizeof(T) == 4) {
    const int tpr = (4 * n <= NT && n % 16 == 0) ? 4 : 2;
    const float invr = 1.f / rhoD;
    const int k = c.tid / tpr, qd = c.tid % tpr, nq = n / tpr;
    float4* r4 = reinterpret_cast<float4*>(c.B + (size_t)(k < n ? k : 0) * bs + qd * nq);
    const float4* p4 = reinterpret_cast<const float4*>(c.phi + qd * nq);
    const float4* c4 = reinterpret_cast<const float4*>(c.col + qd * nq);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (k < n) {
      for (int q = 0; q < nq / 4; ++q) {
        const float4 b = r4[q], f = p4[q];
        a0 += b.x * f.x;
        a1 += b.y * f.y;
        a2 += b.z * f.z;
        a3 += b.w * f.w;
      }
    }
    float acc = (a0 + a1) + (a2 + a3);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (tpr == 4) acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (k < n) {
      const float f = (acc - (k == pp ? 1.f : 0.f)) * invr;
      for (int q = 0; q < nq / 4; ++q) {
        float4 b = r4[q];
        const float4 cv = c4[q];
        b.x -= cv.x * f;
        b.y -= cv.y * f;
        b.z -= cv.z * f;
        b.w -= cv.w * f;
        r4[q] = b;
        if (cnext && k == pp + 1) reinterpret_cast<float4*>(cnext + qd * nq)[q] = b;
      }
    }
    T* rw = c.rows + (size_t)i * 5 * n_pad;
    for (int j = c.tid; j < n; j += NT) {
#pragma unroll
      for (int q = 0; q < 5; ++q) rw[q * n_pad + j] = c.phi[q * n_pad + j];
    }
    if (c.tid == 0) {
      const float y = logf(fabsf(rhoD)) - c.sc->lcomp[s];
      const float t = c.sc->lsum[s] + y;
      c.sc->lcomp[s] = (t - c.sc->lsum[s]) - y;
      c.sc->lsum[s] = t;
      if (rhoD < 0.f) c.sc->sign[s] = -c.sc->sign[s];
    }
  }
}

// Accepted move of electron i: partners' accumulators change by their pair term's
// difference, the electron's own become the fresh sums at r' (the caller's barrier in
// the inverse update publishes them).
template <typename T>
__device__ __forceinline__ void accept_inc(Ctx<T>& c, int i, const IncOut<T>& io) {
  const Params& p = c.p;
  int t0, t1;
  term_range(p, t0, t1);
#pragma unroll
  for (int q = 0; q < JT; ++q) {
    const int t = t0 + c.tid + q * NT;
    if (t0 + q * NT < t1 && t < t1 && t < p.N && t != i) {
#pragma unroll
      for (int k = 0; k < 4; ++k) c.jgl[4 * t + k] += io.dg[q][k];
    }
  }
  if (c.tid == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) c.jgl[4 * i + k] = io.g[k];
  }
}

// E_L of the incremental sweep.  The Jastrow derivatives come from c.jgl, so what is left
// is independent per electron: one thread per electron forms its determinant gradient and
// Laplacian (four dots with its rows and the inverse column, float4 reads when aligned);
// the potential's electron pairs are split evenly, two threads per folded row of the pair
// triangle (row r holds (r, col + 1) for col >= r and (N - 1 - r, N - 1 - col) for
// col < r), and every thread takes its electron's ion terms.  FP64 accumulation.
template <typename T>
__device__ double local_energy_inc(Ctx<T>& c) {
  const Params& p = c.p;
  const int N = p.N, n = p.n, n_pad = p.n_pad, NI = p.n_ions;
  double kin = 0.0;
  T pot = 0;
  const bool vec = (n % 4 == 0) && (n_pad % 4 == 0);
  for (int i = c.tid; i < N; i += NT) {
    const int s = i < p.n_up ? 0 : 1;
    const int pp = i - s * p.n_up;
    const T* brow = c.Bg + ((size_t)s * n + pp) * n;
    const T* rw = c.rows + (size_t)i * 5 * n_pad;
    T gx = 0, gy = 0, gz = 0, l = 0;
    if constexpr (sizeof(T) == 4) {
      if (vec) {
        const float4* b4 = reinterpret_cast<const float4*>(brow);
        const float4* x4 = reinterpret_cast<const float4*>(rw + n_pad);
        const float4* y4 = reinterpret_cast<const float4*>(rw + 2 * n_pad);
        const float4* z4 = reinterpret_cast<const float4*>(rw + 3 * n_pad);
        const float4* l4 = reinterpret_cast<const float4*>(rw + 4 * n_pad);
        for (int q = 0; q < n / 4; ++q) {
          const float4 b = b4[q], x = x4[q], y = y4[q], z = z4[q], w = l4[q];
          gx += x.x * b.x + x.y * b.y + x.z * b.z + x.w * b.w;
          gy += y.x * b.x + y.y * b.y + y.z * b.z + y.w * b.w;
          gz += z.x * b.x + z.y * b.y + z.z * b.z + z.w * b.w;
          l += w.x * b.x + w.y * b.y + w.z * b.z + w.w * b.w;
        }
      }
    }
    if (!(sizeof(T) == 4 && vec)) {
      for (int j = 0; j < n; ++j) {
        const T b = brow[j];
        gx += rw[n_pad + j] * b;
        gy += rw[2 * n_pad + j] * b;
        gz += rw[3 * n_pad + j] * b;
        l += rw[4 * n_pad + j] * b;
      }
    }
    const T ux = c.jgl[4 * i], uy = c.jgl[4 * i + 1], uz = c.jgl[4 * i + 2];
    const T gd2 = gx * gx + gy * gy + gz * gz;
    const T gg = (gx - ux) * (gx - ux) + (gy - uy) * (gy - uy) + (gz - uz) * (gz - uz);
    kin += (double)(T(-0.5) * ((l - gd2) - c.jgl[4 * i + 3] + gg));
    if (p.potential) {
      for (int t = N; t < N + NI; ++t) {
        T d[3], r, rinv;
        partner_disp(c, c.R + 3 * i, c.Rq + 3 * i, t, d, r, rinv);
        if (r < c.k.halfL) pot += T(-2) * exp(T(-0.5) * r * r);
      }
    }
  }
  if (p.potential && N >= 2) {
    const int half = (N - 1) / 2;
    for (int u = c.tid; u < 2 * (N / 2); u += NT) {
      const int r = u >> 1;
      const int c0 = (u & 1) ? half : 0, c1 = (u & 1) ? N - 1 : half;
      for (int col = c0; col < c1; ++col) {
        const bool first = col >= r;
        const int i = first ? r : N - 1 - r;
        const int t = first ? col + 1 : N - 1 - col;
        T d[3], rr, rinv;
        partner_disp(c, c.R + 3 * i, c.Rq + 3 * i, t, d, rr, rinv);
        if (rr < c.k.halfL) pot += exp(-rr * rr);
      }
    }
  }
  double v2[2] = {kin, (double)pot};
  block_sum_to0<NWARP, 2>(v2, (double*)c.red0);
  return v2[0] + v2[1];  // meaningful on thread 0
}

// ---------------------------------------------------------------------------------------
// Inverse guard (mixed path).  After a sweep each spin's FP32 inverse B is probed with the
// sign vector v (v_l = +-1): y = A^T v, then z_k = B^T[k] . y - v_k = (v^T (A B - I))_k,
// a random-sign combination of column k of the residual, for every k at O(n^2) cost.
// Double-float (Neumaier) sums keep z accurate to FP32 relative precision, so the probe
// measures the stored inverse rather than its own rounding.  A spin whose max |z_k|
// exceeds p.guard_tol (or is not finite) has its inverse recomputed by the FP64 LU before
// the walker's E_L, as an early instance of the periodic recompute (Alg. 1 line 3).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ bool probe_negative(int l) {
  return (((uint32_t)(l + 1) * 0x9E3779B1u) >> 31) != 0u;
}

// s + c += x with the rounding error of the addition kept in c (Neumaier).
__device__ __forceinline__ void nsum(float& s, float& c, float x) {
  const float t = s + x;
  c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
  s = t;
}

__device__ __forceinline__ float nan_max(float a, float b) { return (b > a || b != b) ? b : a; }

// g[s] = max_k |(v^T (A_s B_s - I))_k| for both spins; every thread receives them.  Both
// passes serve both spins at once (one column of A, then one row of B^T, per thread), with
// the loads of a thread issued in batches ahead of their sums.
template <typename T>
__device__ void inverse_probe(Ctx<T>& c, float* g) {
  const Params& p = c.p;
  const int n = p.n, n_pad = p.n_pad;
  float* yhi = (float*)c.part;  // [2][n_pad]: y_s as an unevaluated sum hi + lo
  float* ylo = yhi + 2 * n_pad;
  float* red = (float*)c.red1;  // [2][NWARP]
  constexpr int U = 8;
  for (int t = c.tid; t < 2 * n; t += NT) {
    const int s = t >= n ? 1 : 0, j = t - s * n;
    const T* a = c.rows + (size_t)s * p.n_up * 5 * n_pad + j;  // A_s[l][j] at a + 5 n_pad l
    float sm0 = 0.0f, cm0 = 0.0f, sm1 = 0.0f, cm1 = 0.0f;
    int l = 0;
    for (; l + U <= n; l += U) {
      float x[U];
#pragma unroll
      for (int q = 0; q < U; ++q) x[q] = (float)a[(size_t)(l + q) * 5 * n_pad];
#pragma unroll
      for (int q = 0; q < U; q += 2) {
        nsum(sm0, cm0, probe_negative(l + q) ? -x[q] : x[q]);
        nsum(sm1, cm1, probe_negative(l + q + 1) ? -x[q + 1] : x[q + 1]);
      }
    }
    for (; l < n; ++l) {
      const float x = (float)a[(size_t)l * 5 * n_pad];
      nsum(sm0, cm0, probe_negative(l) ? -x : x);
    }
    nsum(sm0, cm0, sm1);
    cm0 += cm1;
    const float hi = sm0 + cm0;
    yhi[s * n_pad + j] = hi;
    ylo[s * n_pad + j] = cm0 - (hi - sm0);
  }
  __syncthreads();
  float worst0 = 0.0f, worst1 = 0.0f;
  for (int t = c.tid; t < 2 * n; t += NT) {
    const int s = t >= n ? 1 : 0, k = t - s * n;
    const T* b = c.Bg + ((size_t)s * n + k) * n;
    const float* yh = yhi + s * n_pad;
    const float* yl = ylo + s * n_pad;
    float sm[4] = {0.0f, 0.0f, 0.0f, 0.0f}, cm[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    auto term = [&](int q, float bj, int j) {
      const float h = yh[j], pr = bj * h;
      const float er = fmaf(bj, h, -pr);
      nsum(sm[q], cm[q], pr);
      cm[q] += er + bj * yl[j];
    };
    int j = 0;
    if constexpr (sizeof(T) == 4) {
      if ((n & 3) == 0) {
        const float4* b4 = reinterpret_cast<const float4*>(b);
        for (; j + 4 * U <= n; j += 4 * U) {
          float4 x[U];
#pragma unroll
          for (int q = 0; q < U; ++q) x[q] = b4[(j >> 2) + q];
#pragma unroll
          for (int q = 0; q < U; ++q) {
            term(0, x[q].x, j + 4 * q);
            term(1, x[q].y, j + 4 * q + 1);
            term(2, x[q].z, j + 4 * q + 2);
            term(3, x[q].w, j + 4 * q + 3);
          }
        }
      }
    }
    for (; j < n; ++j) term(0, (float)b[j], j);
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      nsum(sm[0], cm[0], sm[q]);
      cm[0] += cm[q];
    }
    nsum(sm[0], cm[0], probe_negative(k) ? 1.0f : -1.0f);
    const float z = fabsf(sm[0] + cm[0]);
    if (s == 0) worst0 = nan_max(worst0, z);
    else worst1 = nan_max(worst1, z);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    worst0 = nan_max(worst0, __shfl_xor_sync(0xffffffffu, worst0, o));
    worst1 = nan_max(worst1, __shfl_xor_sync(0xffffffffu, worst1, o));
  }
  if (c.lane == 0) {
    red[c.warp] = worst0;
    red[NWARP + c.warp] = worst1;
  }
  __syncthreads();
  for (int s = 0; s < 2; ++s) {
    float m = red[s * NWARP];
#pragma unroll
    for (int q = 1; q < NWARP; ++q) m = nan_max(m, red[s * NWARP + q]);
    g[s] = m;
  }
  __syncthreads();  // red and the y buffers are free again
}

// FP64 recompute of spin s of this walker (the move kernel's share of the periodic
// recompute): A_s from the current orbital rows, LU with partial pivoting in the walker's
// slice of the workspace, B^T, log|det| and sign replaced.
template <typename T>
__device__ void repair_inverse(Ctx<T>& c, int s) {
  const Params& p = c.p;
  const int n = p.n, n_pad = p.n_pad;
  int* piv = (int*)c.part;
  LuShared<NT>* sh = (LuShared<NT>*)c.red0;
  {
    double* LU = p.lu_ws + (size_t)c.w * 4 * n * n + (size_t)s * 2 * n * n;
    double* X = LU + (size_t)n * n;
    const T* A = c.rows + (size_t)s * p.n_up * 5 * n_pad;
    for (int e = c.tid; e < n * n; e += NT) {
      const int l = e / n, j = e - l * n;
      LU[e] = (double)A[(size_t)l * 5 * n_pad + j];
    }
    __syncthreads();
    double logabs;
    int sgn;
    const bool ok = lu_invert_cta<NT>(LU, X, n, piv, sh, logabs, sgn);
    if (ok) {
      T* Bt = c.Bg + (size_t)s * n * n;
      for (int e = c.tid; e < n * n; e += NT) {
        const int k = e / n, i = e - k * n;  // B^T[k][i] = (A^-1)[i][k]
        Bt[e] = (T)X[(size_t)i * n + k];
      }
    }
    if (c.tid == 0) {
      if (!ok) atomicOr(p.status, ST_SINGULAR);
      c.sc->logdet[s] = logabs;
      c.sc->sign[s] = sgn;
      c.sc->lsum[s] = c.sc->lcomp[s] = 0.0f;
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void prefetch_grad_rows(const Ctx<T>& c, int i, T* pf) {
  if (i < c.p.N && c.tid < c.p.n) {
    const T* rw = c.rows + (size_t)i * 5 * c.p.n_pad + c.tid;
    pf[0] = rw[c.p.n_pad];
    pf[1] = rw[2 * c.p.n_pad];
    pf[2] = rw[3 * c.p.n_pad];
  }
}

// The Gaussian draws chi of move i (in shared memory: the proposal indexes them by lane)
// and its acceptance uniform: from the sweep's table, or (compact layout) computed from the
// same Philox words here, every thread writing the same values to one shared slot (all
// threads are at the same move: barriers separate consecutive proposals on this path).
// The incremental sweep, which pipelines proposals, never runs in the compact layout.
template <typename T>
__device__ __forceinline__ const T* chi_of(const Ctx<T>& c, int i) {
  if (!c.p.compact) return c.dchi + 3 * i;
  T d4[4];
  draws_t<T>(c.p.seed, (uint32_t)c.w, c.p.gen, (uint32_t)i, d4);
  c.sc->chi[0] = d4[0];
  c.sc->chi[1] = d4[1];
  c.sc->chi[2] = d4[2];
  return c.sc->chi;
}
template <typename T>
__device__ __forceinline__ T u_of(const Ctx<T>& c, int i) {
  return c.p.compact ? accept_uniform_t<T>(c.p.seed, (uint32_t)c.w, c.p.gen, (uint32_t)i)
                     : c.du[i];
}

// Proposal of electron i shared by every thread: the mixed path computes it in each
// thread; the FP64 path on thread 0, then copied through shared memory.
template <typename T>
__device__ __forceinline__ void shared_proposal(Ctx<T>& c, int i, const T* F, const T* chi,
                                                const double* rgiven, Prop<T>& pr) {
  if constexpr (IsMixed<T>::value) {
    make_proposal(c, i, F, chi, rgiven, pr);
  } else {
    if (c.tid == 0) make_proposal(c, i, F, chi, rgiven, c.sc->pr);
    __syncthreads();
    pr = c.sc->pr;
  }
#if QMCGB_CHECK
  // the electron index and the spline cell of r' (its 4x4x4 stencil must lie in the
  // ghost-padded table); a bad cell is recorded and replaced by cell 0 before any load
  if (c.p.test_bad_cell && i == 0) pr.cell[0] = c.p.G + 5;  // test hook: a planted bad cell
  QMC_CHECKP(c.p, i >= 0 && i < c.p.N, CK_ELECTRON, i);
  for (int k = 0; k < 3; ++k)
    if (!QMC_CHECKP(c.p, pr.cell[k] >= 0 && pr.cell[k] < c.p.G, CK_CELL,
                    ((long long)k << 32) | (uint32_t)pr.cell[k]))
      pr.cell[k] = 0;
#endif
}

// Offset of this generation's E_L in p.eloc_out: a batch sweep keeps one row per
// generation ([gen - eloc_gen0][W]); single-crowd calls write row 0.
__device__ __forceinline__ size_t eloc_slot(const Params& p) {
  return p.eloc_by_gen ? (size_t)(p.gen - p.eloc_gen0) * p.W : 0;
}

// The body of one walker's CTA (walker w of the crowd described by p); smem is the CTA's
// dynamic shared memory, tmap the crowd's table tensor map.
template <typename T, int MODE, int UPD, int BSM>
__device__ __forceinline__ void move_body(const Params& p, const int w, const CUtensorMap* tmap,
                                          unsigned char* smem) {
  const Lay lay = make_lay<T>(p);
  const int N = p.N, n = p.n, n_pad = p.n_pad;
#if QMCGB_CHECK
  {
    uint32_t dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    // uniform per CTA: the whole walker is skipped
    if (!QMC_CHECKP(p, w >= 0 && w < p.W, CK_WALKER, w)) return;
    if (!QMC_CHECKP(p, lay.total <= dyn, CK_SMEM, lay.total)) return;
    if (p.use_tma) {
      // the copy's size, and its 128-byte aligned buffer (all ring slots) inside the room
      // the layout gave it
      const bool ring = p.use_tma == 2;
      const size_t sb = (ring ? (size_t)RING_SLOTS : 1) * (size_t)p.stencil_bytes;
      const uintptr_t base = reinterpret_cast<uintptr_t>(smem + (ring ? lay.part : lay.stc));
      const uintptr_t a = (base + 127) & ~(uintptr_t)127;
      const int want = (ring ? RING_ORB * 16 : 64 * n_pad) * (int)sizeof(T);
      if (!QMC_CHECKP(p, p.stencil_bytes == want && a + sb <= base + al16(sb + 128), CK_STENCIL,
                      p.stencil_bytes))
        return;
    }
  }
#endif
  Ctx<T> c{p};
  c.k = make_cst<T>(p);
  c.w = w;
  c.tid = threadIdx.x;
  c.lane = threadIdx.x & 31;
  c.warp = threadIdx.x >> 5;
  c.bs = b_stride<T>(p);
  c.upd = UPD;
  c.bsm = BSM;
  c.sc = (Scal<T>*)(smem + lay.scal);
  c.Bs = (T*)(smem + lay.B);
  c.Bg = (T*)p.binv + (size_t)w * 2 * n * n;
  c.B = c.Bg;
  c.R = (double*)(smem + lay.R);
  c.Rq = (uint32_t*)(smem + lay.Rq);
  c.ion = (double*)(smem + lay.ion);
  c.ionq = (uint32_t*)(smem + lay.ionq);
  c.jc = (T*)(smem + lay.jc);
  c.jgl = (T*)(smem + lay.jgl);
  c.phi = (T*)(smem + lay.phi);
  c.part = (T*)(smem + lay.part);
  c.col = (T*)(smem + lay.col);
  c.col2 = (T*)(smem + lay.col2);
  c.dchi = (T*)(smem + lay.dchi);
  c.du = (T*)(smem + lay.du);
  c.red0 = (T*)(smem + lay.red0);
  c.red1 = (T*)(smem + lay.red1);
  c.wP = (int*)(smem + lay.wP);
  c.wV = (T*)(smem + lay.wV);
  c.wS = (T*)(smem + lay.wS);
  c.wy = (T*)(smem + lay.wy);
  c.wz = (T*)(smem + lay.wz);
  c.wc = (T*)(smem + lay.wc);
  c.wb = (T*)(smem + lay.wb);
  c.snap = (T*)(smem + lay.snap);
  c.xb = (T*)(smem + lay.xb);
  c.yb = (T*)(smem + lay.yb);
  c.rows = (T*)p.rows + (size_t)w * N * 5 * n_pad;
  c.bar = (uint64_t*)(smem + lay.bar);
  c.stc = (T*)((reinterpret_cast<uintptr_t>(smem + (p.use_tma == 2 ? lay.part : lay.stc)) + 127) &
               ~(uintptr_t)127);
  c.tmap = tmap;
  c.tma_phase = 0;
  c.mma_phase = 0;
  c.tcs = (float*)((reinterpret_cast<uintptr_t>(smem + lay.tcs) + 127) & ~(uintptr_t)127);
  c.tc = false;
  c.tc_over_move = lay.tcs == lay.phi;
  c.failed = false;
  c.nit = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int it = c.tid + q * NT;
    c.itj[q] = it < 4 * n ? it % n : 0;
    c.ita[q] = it < 4 * n ? it / n : 0;
    if (it < 4 * n) c.nit = q + 1;
#if QMCGB_CHECK
    if (!QMC_CHECKP(p, c.itj[q] < n_pad && c.ita[q] < 4, CK_ORBITAL, it)) c.itj[q] = c.ita[q] = 0;
#endif
  }
  Scal<T>* sc = c.sc;

  const double* Rg = p.R + (size_t)w * N * 3;
  for (int e = c.tid; e < N * 3; e += NT) {
    const double x = Rg[e];
    if constexpr (IsMixed<T>::value) c.Rq[e] = to_fixed(x, p.fx_scale);
    else c.R[e] = x;
  }
  for (int e = c.tid; e < p.n_ions * 3; e += NT) {
    const double x = p.ions[e];
    c.ion[e] = x;
    if constexpr (IsMixed<T>::value) c.ionq[e] = to_fixed(x, p.fx_scale);
  }
  const int njc = 2 * (p.K2 + 3) + p.K1 + 3;
  for (int e = c.tid; e < njc; e += NT) c.jc[e] = ((const T*)p.jc)[e];
  if (c.tid == 0) {
    sc->logdet[0] = p.logdet[w * 2];
    sc->logdet[1] = p.logdet[w * 2 + 1];
    sc->sign[0] = p.sign[w * 2];
    sc->sign[1] = p.sign[w * 2 + 1];
    sc->lsum[0] = sc->lsum[1] = sc->lcomp[0] = sc->lcomp[1] = 0.0f;
    sc->m = 0;
    if (p.use_tma || p.tc_flush) {
      mbar_init(c.bar, 1);
      mbar_init(c.bar + 1, 1);
      if (p.use_tma == 2) {
        mbar_init(c.bar + 2, 1);
        mbar_init(c.bar + 3, 1);
      }
      mbar_fence_init();
    }
    sc->accept = 0;
  }
  // delayed windows of the mixed path with the inverse in global memory are flushed on
  // the tensor cores (TMEM is allocated for each flush)
  if constexpr (IsMixed<T>::value && UPD == 1 && BSM != 1) c.tc = p.tc_flush && !p.b_in_smem;
  __syncthreads();

  int t0, t1;
  term_range(p, t0, t1);
  const bool cache_ok = p.drift && (t1 - t0) <= JT * NT;
  const bool pf_ok = n <= NT;
  T uo[JT];
#pragma unroll
  for (int q = 0; q < JT; ++q) uo[q] = T(0);
  T F[3] = {0, 0, 0};
  Prop<T> pr;
  Res<T> rs;

  bool moved = false;
  if constexpr (MODE == MODE_SWEEP) {
    for (int e = c.tid; e < N && !p.compact; e += NT) {
      T d4[4];
      draws_t<T>(p.seed, (uint32_t)w, p.gen, (uint32_t)e, d4);
      c.dchi[3 * e] = d4[0];
      c.dchi[3 * e + 1] = d4[1];
      c.dchi[3 * e + 2] = d4[2];
      c.du[e] = d4[3];
    }
    T pf[3] = {0, 0, 0};
    if (pf_ok) prefetch_grad_rows(c, 0, pf);
    // incremental Jastrow (mixed Sherman-Morrison): the accumulators come from the previous
    // sweep when still valid, else from one pass over all pairs
    bool inc = false;
    if constexpr (IsMixed<T>::value && UPD == 0)
      inc = p.inc_jastrow && 2 * n <= NT && n % 8 == 0 && b_stride<T>(p) % 4 == 0 &&
            (t1 - t0) <= JT * NT;
    if (inc) {
      if (p.jvalid[w]) {
        const T* gsrc = (const T*)p.jgl + (size_t)w * N * 4;
        for (int e = c.tid; e < N * 4; e += NT) c.jgl[e] = gsrc[e];
      } else {
        jastrow_gl_all(c);
      }
    }
    __syncthreads();
    unsigned long long nacc = 0;
    if constexpr (IsMixed<T>::value && UPD == 0) {
      if (inc) {
        // Software-pipelined: once move i is decided (and its accumulators and position
        // published), move i+1's drift, proposal, stencil copy and Jastrow terms are issued
        // before move i's inverse update, so their latencies overlap it.
        for (int s = 0; s < 2 && !c.failed; ++s) {
          begin_spin(c, s);
          T det[3] = {0, 0, 0};
          T jv[5];
          IncOut<T> io;
          int i = s * p.n_up;
          compute_column(c, 0);
          if (p.drift) {
            det_grad(c, i, det);
            for (int k = 0; k < 3; ++k) F[k] = det[k] - c.jgl[4 * i + k];
          }
          bool nxt = p.drift && n > 1;
          if (nxt) prefetch_grad_rows(c, i + 1, pf);
          shared_proposal(c, i, F, c.dchi + 3 * i, nullptr, pr);
          stencil_issue(c, pr);
          jas_inc(c, i, pr, jv, io);
          for (int pp = 0; pp < n; ++pp) {
            i = s * p.n_up + pp;
            // false only when a stencil copy timed out (status set; uniform over the CTA)
            if (!spo_inc(c, i, pp, pr, rs, nxt, pf, jv, io)) {
              c.failed = true;
              break;
            }
            const int acc = metropolis(p, c.k, pr, rs, c.du[i], w, i);
            nacc += acc;
            if (p.accept_trace && c.tid == 0) p.accept_trace[(size_t)w * N + i] = (uint8_t)acc;
            if (acc) {
              accept_inc(c, i, io);
              if (c.tid == 0)
                for (int k = 0; k < 3; ++k) c.Rq[3 * i + k] = pr.rq[k];
            }
            if (nxt) {  // the next electron's determinant drift after this move
              const T f = acc ? io.e / rs.rhoD : T(0);
              for (int k = 0; k < 3; ++k) det[k] = io.a[k] - f * io.b[k];
            }
            const T rhoD = rs.rhoD;
            __syncthreads();  // accumulators and the moved position are visible
            const bool more = pp + 1 < n;
            if (more) {
              const int i1 = i + 1;
              if (p.drift)
                for (int k = 0; k < 3; ++k) F[k] = det[k] - c.jgl[4 * i1 + k];
              nxt = p.drift && pp + 2 < n;
              if (nxt) prefetch_grad_rows(c, i1 + 1, pf);
              shared_proposal(c, i1, F, c.dchi + 3 * i1, nullptr, pr);
              stencil_issue(c, pr);
              jas_inc(c, i1, pr, jv, io);
            }
            // the next move's column is row pp + 1 of the updated inverse: its row owners
            // write it to col2 as they update it (or it is copied when nothing changes), so
            // the next move needs no column pass and no barrier of its own here; the barrier
            // inside its ratio (before the column and the updated rows are read) orders it
            if (acc) {
              sm_rows_update(c, i, s, pp, rhoD, more ? c.col2 : nullptr);
            } else if (more) {
              const T* bn = c.B + (size_t)(pp + 1) * c.bs;
              for (int j = c.tid; j < n; j += NT) c.col2[j] = bn[j];
            }
            if (more) {
              T* t = c.col;
              c.col = c.col2;
              c.col2 = t;
            }
          }
          if (c.failed) break;
          end_spin(c, s, true);
        }
      }
    }
    for (int s = 0; s < 2 && !inc; ++s) {
      begin_spin(c, s);
      for (int pp = 0; pp < n; ++pp) {
        const int i = s * p.n_up + pp;
        compute_column(c, pp);
        if (p.drift) eval_grad(c, i, pf, pf_ok, uo, F);
        if (pf_ok) prefetch_grad_rows(c, i + 1, pf);  // row i+1 is not touched by move i
        shared_proposal(c, i, F, chi_of(c, i), nullptr, pr);
        // false only when a stencil copy timed out (status set; uniform over the CTA)
        if (!ratio_grad(c, i, pr, uo, cache_ok, rs)) {
          c.failed = true;
          break;
        }
        int acc;
        if constexpr (IsMixed<T>::value) {
          acc = metropolis(p, c.k, pr, rs, u_of(c, i), w, i);
        } else {
          if (c.tid == 0) {
            sc->rs = rs;
            sc->accept = metropolis(p, c.k, pr, rs, u_of(c, i), w, i);
          }
          __syncthreads();
          rs = sc->rs;
          acc = sc->accept;
        }
        nacc += acc;
        if (p.accept_trace && c.tid == 0) p.accept_trace[(size_t)w * N + i] = (uint8_t)acc;
        if (acc) accept_update(c, i, s, pp, pr, rs.rhoD);
        if (c.failed) break;  // a tensor-core flush timed out
      }
      if (c.failed) break;
      flush_window(c);
      if (c.failed) break;
      end_spin(c, s, true);
    }
    if (c.failed) return;
    moved = true;
    if constexpr (IsMixed<T>::value) {
      if (p.guard_val && !p.skip_eloc) {
        float g[2];
        inverse_probe(c, g);
        if (c.tid == 0) p.guard_val[w] = (g[1] > g[0] || g[1] != g[1]) ? g[1] : g[0];
        bool rep = false;
        for (int s = 0; s < 2; ++s) {
          if (!(g[s] <= p.guard_tol)) {  // uniform; a NaN repairs too
            repair_inverse(c, s);
            rep = true;
          }
        }
        if (rep && c.tid == 0 && p.n_repair) {
          atomicAdd(p.n_repair, 1ull);
          atomicAdd(p.n_repair + 1, 1ull);
        }
      }
    }
    if (!p.skip_eloc) {
      double e;
      if constexpr (IsMixed<T>::value && UPD == 0)
        e = inc ? local_energy_inc(c) : local_energy(c);
      else
        e = local_energy(c);
      if (c.tid == 0) {
        if (p.eloc_out) p.eloc_out[eloc_slot(p) + w] = e;
        if (!isfinite(e)) atomicOr(p.status, ST_NAN);
      }
    }
    if (inc) {  // carried to the next sweep
      T* gdst = (T*)p.jgl + (size_t)w * N * 4;
      for (int e = c.tid; e < N * 4; e += NT) gdst[e] = c.jgl[e];
      if (c.tid == 0) p.jvalid[w] = 1;
    }
    if (c.tid == 0 && p.n_accept) atomicAdd(p.n_accept, nacc);
  } else if constexpr (MODE == MODE_GRAD || MODE == MODE_PROPOSE) {
    const int i = p.iel;
    const int s = i < p.n_up ? 0 : 1;
    const int pp = i - s * p.n_up;
    begin_spin(c, s);
    compute_column(c, pp);
    if (p.drift) eval_grad<T>(c, i, nullptr, false, uo, F);
    if constexpr (MODE == MODE_GRAD) {
      if (c.tid == 0)
        for (int k = 0; k < 3; ++k) p.grad_out[w * 3 + k] = (double)F[k];
    } else {
      T chi[3] = {0, 0, 0};
      if (!p.rnew_in) {
        T d4[4];
        draws_t<T>(p.seed, (uint32_t)w, p.gen, (uint32_t)i, d4);
        chi[0] = d4[0];
        chi[1] = d4[1];
        chi[2] = d4[2];
      }
      shared_proposal(c, i, F, chi, p.rnew_in ? p.rnew_in + 3 * w : nullptr, pr);
      if (!ratio_grad(c, i, pr, uo, cache_ok, rs)) return;
      T* pphi = (T*)p.pend_phi + (size_t)w * 5 * n_pad;
      for (int j = c.tid; j < n; j += NT)
        for (int q = 0; q < 5; ++q) pphi[q * n_pad + j] = c.phi[q * n_pad + j];
      if (c.tid == 0) {
        double* pd = p.pend + (size_t)w * PEND_STRIDE;
        double rp[3];
        for (int k = 0; k < 3; ++k) {
          if constexpr (IsMixed<T>::value) {
            pd[P_R + k] = (double)pr.rq[k];
            rp[k] = (double)pr.rq[k] * p.fx_unit;
          } else {
            pd[P_R + k] = pr.rp[k];
            rp[k] = pr.rp[k];
          }
          pd[P_DISP + k] = (double)pr.disp[k];
          pd[P_FP + k] = (double)rs.Fp[k];
        }
        pd[P_RHOD] = (double)rs.rhoD;
        pd[P_RHO] = (double)rs.rho;
        pd[P_DU] = (double)rs.dU;
        pd[P_LOGGF] = (double)pr.logGf;
        pd[P_IEL] = (double)i;
        pd[P_VALID] = 1.0;
        if (p.ratio_out) p.ratio_out[w] = (double)rs.rho;
        if (p.logratio_out) p.logratio_out[w] = log(fabs((double)rs.rhoD)) - (double)rs.dU;
        if (p.grad_out)
          for (int k = 0; k < 3; ++k) p.grad_out[w * 3 + k] = (double)rs.Fp[k];
        if (p.rnew_out)
          for (int k = 0; k < 3; ++k) p.rnew_out[w * 3 + k] = rp[k];
      }
    }
    end_spin(c, s, false);
  } else if constexpr (MODE == MODE_ACCEPT) {
    const int i = p.iel;
    const int s = i < p.n_up ? 0 : 1;
    const int pp = i - s * p.n_up;
    double* pd = p.pend + (size_t)w * PEND_STRIDE;
    const bool valid = pd[P_VALID] == 1.0 && (int)pd[P_IEL] == i;
    if (!valid) {
      if (c.tid == 0) atomicOr(p.status, ST_STATE);
      return;  // uniform across the CTA
    }
    begin_spin(c, s);
    compute_column(c, pp);
    const T* pphi = (const T*)p.pend_phi + (size_t)w * 5 * n_pad;
    for (int j = c.tid; j < n; j += NT)
      for (int q = 0; q < 5; ++q) c.phi[q * n_pad + j] = pphi[q * n_pad + j];
    for (int k = 0; k < 3; ++k) {
      if constexpr (IsMixed<T>::value) pr.rq[k] = (uint32_t)pd[P_R + k];
      else pr.rp[k] = pd[P_R + k];
      pr.disp[k] = (T)pd[P_DISP + k];
      rs.Fp[k] = (T)pd[P_FP + k];
    }
    rs.rhoD = (T)pd[P_RHOD];
    rs.rho = (T)pd[P_RHO];
    rs.dU = (T)pd[P_DU];
    pr.logGf = (T)pd[P_LOGGF];
    __syncthreads();  // every thread has read the pending state
    if (c.tid == 0) {
      int acc;
      if (p.accept_in) acc = p.accept_in[w] != 0;
      else
        acc = metropolis(p, c.k, pr, rs,
                         accept_uniform_t<T>(p.seed, (uint32_t)w, p.gen, (uint32_t)i), w, i);
      sc->accept = acc;
      if (p.accept_out) p.accept_out[w] = (uint8_t)acc;
      pd[P_VALID] = 0.0;
      if (p.jvalid) p.jvalid[w] = 0;  // the incremental sweep's accumulators are stale
    }
    __syncthreads();
    if (sc->accept) accept_update(c, i, s, pp, pr, rs.rhoD);
    end_spin(c, s, true);
    moved = true;
  } else if constexpr (MODE == MODE_ELOC) {
    for (int s = 0; s < 2; ++s) {
      begin_spin(c, s);
      flush_window(c);
      end_spin(c, s, true);
    }
    if (!p.skip_eloc) {
      const double e = local_energy(c);
      if (c.tid == 0) {
        p.eloc_out[eloc_slot(p) + w] = e;
        if (!isfinite(e)) atomicOr(p.status, ST_NAN);
      }
    }
  }
  __syncthreads();
  if (moved) {
    double* Rw = p.R + (size_t)w * N * 3;
    for (int e = c.tid; e < N * 3; e += NT) {
      if constexpr (IsMixed<T>::value) Rw[e] = (double)c.Rq[e] * p.fx_unit;
      else Rw[e] = c.R[e];
    }
    if (c.tid == 0) {
      p.logdet[w * 2] = sc->logdet[0] + (double)sc->lsum[0];
      p.logdet[w * 2 + 1] = sc->logdet[1] + (double)sc->lsum[1];
      p.sign[w * 2] = sc->sign[0];
      p.sign[w * 2 + 1] = sc->sign[1];
    }
  }
}

// Two CTAs per SM; with the inverse in global memory at 256 threads the shared memory
// already holds one CTA per SM, so the register cap is lifted to that of one CTA.
template <typename T, int MODE, int UPD, int BSM>
__global__ void __launch_bounds__(NT, (BSM == 2 && NT >= 256) ? 1 : 2)
    move_kernel(const Params p, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(16) unsigned char smem[];
  move_body<T, MODE, UPD, BSM>(p, blockIdx.x, &tmap, smem);
}

// One generation of several crowds in one launch (the mixed-size batch): CTA b runs walker
// b - base[c] of crowd c, with the crowd's parameters copied from global memory into
// shared memory.  Where the inverse lives is decided per crowd at run time.
template <typename T, int UPD>
__global__ void __launch_bounds__(NT, 2) move_kernel_batch(const Params* __restrict__ plist,
                                                           const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) Params sp;
  int cr = 0;
  while (cr + 1 < a.n && (int)blockIdx.x >= a.base[cr + 1]) ++cr;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(plist + cr);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sp);
  for (int e = threadIdx.x; e < (int)(sizeof(Params) / 4); e += NT) dst[e] = src[e];
  __syncthreads();
  // the crowd's layout must fit the launch's dynamic shared memory (uniform per CTA)
  uint32_t dyn;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  const int w = (int)blockIdx.x - a.base[cr];
  if (make_lay<T>(sp).total > dyn || w >= sp.W) {
    if (threadIdx.x == 0) atomicOr(sp.status, ST_STATE);
    return;
  }
  move_body<T, MODE_SWEEP, UPD, 0>(sp, w, &a.maps[cr], smem);
}

// Lets a kernel instantiation use up to the device's opt-in shared memory per CTA (set
// once per process and device; crowds of any size then launch it without resetting it).
template <typename T, int MODE, int UPD, int BSM>
static cudaError_t allow_max_smem() {
  static std::atomic<int> done_for{-1};  // one per kernel instantiation (crowds may be
                                          // driven from several host threads)
  auto kern = move_kernel<T, MODE, UPD, BSM>;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || done_for.load() == dev) return e;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) done_for = dev;
  return e;
}

template <typename T, int MODE, int UPD, int BSM>
static cudaError_t launch_upd(const Params& p, size_t bytes, const CUtensorMap& tm,
                              cudaStream_t s) {
  if (bytes > 48 * 1024) {
    const cudaError_t e = allow_max_smem<T, MODE, UPD, BSM>();
    if (e != cudaSuccess) return e;
  }
  move_kernel<T, MODE, UPD, BSM><<<p.W, NT, bytes, s>>>(p, tm);
  return cudaGetLastError();
}

// The sweep is specialised on where the inverse lives; the fine-grained calls are not.
template <typename T, int MODE>
static cudaError_t launch_mode(const Params& p, size_t bytes, const CUtensorMap& tm,
                               cudaStream_t s) {
  if constexpr (MODE == MODE_SWEEP) {
    if (p.update == 1)
      return p.b_in_smem ? launch_upd<T, MODE, 1, 1>(p, bytes, tm, s)
                         : launch_upd<T, MODE, 1, 2>(p, bytes, tm, s);
    return p.b_in_smem ? launch_upd<T, MODE, 0, 1>(p, bytes, tm, s)
                       : launch_upd<T, MODE, 0, 2>(p, bytes, tm, s);
  } else {
    return p.update == 1 ? launch_upd<T, MODE, 1, 0>(p, bytes, tm, s)
                         : launch_upd<T, MODE, 0, 0>(p, bytes, tm, s);
  }
}

template <typename T>
cudaError_t launch_move(const Params& p_in, int mode, const void* tmap, cudaStream_t s) {
  Params p = p_in;
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  if (p.use_tma && tmap) std::memcpy(&tm, tmap, sizeof(tm));
  else p.use_tma = 0;
  p.stencil_bytes = stencil_tma_bytes(p, (int)sizeof(T));
  const size_t bytes = make_lay<T>(p).total;
  p.skip_eloc = 0;
  switch (mode) {
    case MODE_SWEEP: return launch_mode<T, MODE_SWEEP>(p, bytes, tm, s);
    case MODE_SWEEP_NOE: p.skip_eloc = 1; return launch_mode<T, MODE_SWEEP>(p, bytes, tm, s);
    case MODE_GRAD: return launch_mode<T, MODE_GRAD>(p, bytes, tm, s);
    case MODE_PROPOSE: return launch_mode<T, MODE_PROPOSE>(p, bytes, tm, s);
    case MODE_ACCEPT: return launch_mode<T, MODE_ACCEPT>(p, bytes, tm, s);
    case MODE_ELOC: return launch_mode<T, MODE_ELOC>(p, bytes, tm, s);
    case MODE_FLUSH: p.skip_eloc = 1; return launch_mode<T, MODE_ELOC>(p, bytes, tm, s);
    default: return cudaErrorInvalidValue;
  }
}


template <typename T, int UPD>
static cudaError_t launch_batch_upd(const Params* d_plist, const BatchArgs& a, size_t bytes,
                                    cudaStream_t s) {
  static std::atomic<int> done_for{-1};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (done_for.load() != dev) {
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int avail = optin - (int)sizeof(Params) - 16;  // the static Params copy
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(move_kernel_batch<T, UPD>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, avail);
    if (e != cudaSuccess) return e;
    done_for = dev;
  }
  move_kernel_batch<T, UPD><<<a.base[a.n], NT, bytes, s>>>(d_plist, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch(const Params* d_plist, const BatchArgs& a, int update, size_t bytes,
                         cudaStream_t s) {
  return update == 1 ? launch_batch_upd<T, 1>(d_plist, a, bytes, s)
                     : launch_batch_upd<T, 0>(d_plist, a, bytes, s);
}

// one precision per translation unit (QMCGB_MOVE_ELEM = 4 or 8), so the units compile in
// parallel
#if QMCGB_MOVE_ELEM == 4
template cudaError_t launch_batch<float>(const Params*, const BatchArgs&, int, size_t,
                                         cudaStream_t);
template cudaError_t launch_move<float>(const Params&, int, const void*, cudaStream_t);
#else
template cudaError_t launch_batch<double>(const Params*, const BatchArgs&, int, size_t,
                                          cudaStream_t);
template cudaError_t launch_move<double>(const Params&, int, const void*, cudaStream_t);
#endif

}  // namespace QMCGB_MOVE_NS
}  // namespace qmcgb

// Nonlocal pseudopotential term of the local energy (Alg. 1 line 11) in the locality
// approximation, as a kernel of its own that adds to the E_L a sweep has written (the
// move kernel's registers stay those of the move).
//
// Every ion carries channels l < p.nl_n with v_l(r) = a_l exp(-r^2 / s_l^2) for r < nl_rc.
// Electron i at d = r_i - R_I (minimum image), r = |d| < nl_rc, adds
//   sum_l v_l(r) (2l+1) (1/12) sum_q P_l(d.u_q / r) Psi(r_i -> R_I + r u_q) / Psi(R)
// over the 12 vertices u_q of an icosahedron (a spherical design exact to degree 5),
// P_0 = 1, P_1 = x, P_2 = (3x^2 - 1)/2.  Each ratio is a virtual move of electron i: the
// orbitals' values at the point dotted with electron i's column of A^-1, times
// exp(-(U_i(point) - U_i(r_i))).
//
// NL_SPLIT CTAs per walker (more CTAs than SMs, two resident per SM).  A CTA's warps first
// list the (electron, ion) pairs within the cutoff of their electrons (the walker's 32
// warps take electrons gw, gw + 32, ...), then take the listed pairs' batches of quadrature
// points in turn, so the few pairs spread evenly; lanes run over orbitals for the
// determinant and over partners for the Jastrow sums.  Each CTA writes its FP64 sum to a
// partial slot; a second kernel adds a walker's partials to E_L in a fixed order, so E_L
// stays deterministic.  The mixed path works
// in FP32 on 32-bit fixed-point positions like the move kernel; the FP64 path in double.
#include <cmath>

#include "qmc_device.cuh"
#include "qmc_internal.h"

namespace qmcgb {
namespace {

constexpr int NL_NT = 256;
constexpr int NL_NW = NL_NT / 32;
constexpr int NL_SPLIT = 4;  // CTAs per walker
constexpr int NL_QB = 2;     // quadrature points evaluated together
constexpr int NL_NQB = 12 / NL_QB;
constexpr int NL_SEG = 64;   // pairs a warp lists for the CTA (more: it does them itself)

// Vertex q of the icosahedron: (0, +-1, +-phi) / sqrt(1 + phi^2) for q < 4 and its cyclic
// shifts (+-1, +-phi, 0), (+-phi, 0, +-1) for q / 4 = 1, 2; bits 0 and 1 of q are the signs.
template <typename T>
__device__ __forceinline__ void ico_vertex(int q, T* u) {
  const T nrm = T(0.52573111211913360603);  // 1 / sqrt(1 + phi^2)
  const T phn = T(0.85065080835203993218);  // phi / sqrt(1 + phi^2)
  const T v[3] = {T(0), (q & 1) ? -nrm : nrm, (q & 2) ? -phn : phn};
  const int sft = q >> 2;
#pragma unroll
  for (int k = 0; k < 3; ++k) u[k] = v[(k + sft) % 3];
}

// A point: FP64 coordinates, or fixed point in the mixed path.
template <typename T> struct Pt { double x[3]; };
template <> struct Pt<float> { uint32_t q[3]; };

template <typename T>
struct NlCtx {
  const Params& p;
  const Pt<T>* R;    // electrons (shared memory)
  const Pt<T>* ion;  // ions (shared memory)
  const T* jc;       // radial coefficients (shared memory)
  T unit, scale, L, invL, h2inv, h1inv, rc2, rc1;
  int lane;
};

template <typename T>
__device__ __forceinline__ void disp(const NlCtx<T>& c, const Pt<T>& a, const Pt<T>& b, T* d,
                                     T& r) {
  if constexpr (IsMixed<T>::value) {
    disp_fx(a.q, b.q, c.unit, d);
  } else {
    disp_f64(a.x, b.x, c.p.L, c.p.invL, d);
  }
  r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

// out[b] = sum over partners t != i (electrons, then ions) of u(|x[b] - r_t|) for B points
// at once (independent chains): the warp totals.
template <typename T, int B>
__device__ void jastrow_sums(const NlCtx<T>& c, int i, const Pt<T>* x, T* out) {
  const Params& p = c.p;
  const int N = p.N;
  const int t0 = p.K2 > 0 ? 0 : N, t1 = p.K1 > 0 ? N + p.n_ions : N;
  T acc[B];
#pragma unroll
  for (int b = 0; b < B; ++b) acc[b] = 0;
  for (int t = t0 + c.lane; t < t1; t += 32) {
    if (t == i) continue;
    const Pt<T>& pt = t < N ? c.R[t] : c.ion[t - N];
    const T* coef;
    int K;
    T hinv, rc;
    if (t < N) {
      coef = c.jc + (((i < p.n_up) == (t < p.n_up)) ? 0 : p.K2 + 3);
      K = p.K2;
      hinv = c.h2inv;
      rc = c.rc2;
    } else {
      coef = c.jc + 2 * (p.K2 + 3);
      K = p.K1;
      hinv = c.h1inv;
      rc = c.rc1;
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      T d[3], r, u, du, d2u;
      disp(c, x[b], pt, d, r);
      radial(coef, K, hinv, rc, r, u, du, d2u);
      acc[b] += u;
    }
  }
#pragma unroll
  for (int b = 0; b < B; ++b) out[b] = warp_sum(acc[b]);
}

// Quadrature point q of the pair (electron, ion I at distance r): R_I + r u_q, its spline
// cell and value weights.
template <typename T>
__device__ __forceinline__ void quad_point(const NlCtx<T>& c, const Pt<T>& ion, T r, int q,
                                           T* u, Pt<T>& xq, int* cell, T (*wt)[4]) {
  const Params& p = c.p;
  ico_vertex(q, u);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T t;
    if constexpr (IsMixed<T>::value) {  // fixed point wraps by itself
      xq.q[k] = ion.q[k] + (uint32_t)__float2int_rn(r * u[k] * c.scale);
      const unsigned long long prod = (unsigned long long)xq.q[k] * (unsigned long long)p.G;
      cell[k] = (int)(prod >> 32);
      t = (float)(uint32_t)prod * 0x1p-32f;
    } else {
      double x = ion.x[k] + r * u[k];
      x -= p.L * floor(x * p.invL);
      xq.x[k] = x;
      const double sg = x * p.dgrid;
      int g = (int)floor(sg);
      g = g > p.G - 1 ? p.G - 1 : (g < 0 ? 0 : g);
      cell[k] = g;
      t = sg - (double)g;
    }
    const T t2 = t * t, t3 = t2 * t, sm = T(1) - t, sixth = T(1) / T(6);
    wt[k][0] = sm * sm * sm * sixth;
    wt[k][1] = (T(3) * t3 - T(6) * t2 + T(4)) * sixth;
    wt[k][2] = (T(-3) * t3 + T(3) * t2 + T(3) * t + T(1)) * sixth;
    wt[k][3] = t3 * sixth;
  }
}

// The contribution of quadrature points q0 .. q0 + NL_QB - 1 of the pair (electron i, ion
// I), u0 = U_i at r_i: sum_l v_l(r) (2l+1) (1/12) sum_q P_l(d.u_q / r) Psi(q) / Psi, the
// same on every lane.
template <typename T>
__device__ double pair_batch(const NlCtx<T>& c, const T* table, const T* Bw, int i, int I,
                             T u0, int q0) {
  const Params& p = c.p;
  const int n = p.n, n_pad = p.n_pad, GP = p.GP, lane = c.lane;
  const int s = i < p.n_up ? 0 : 1;
  const T* bcol = Bw + ((size_t)s * n + (i - s * p.n_up)) * n;  // column of A^-1
  T d[3], r;
  disp(c, c.R[i], c.ion[I], d, r);  // r_i - R_I
  const T rinv = T(1) / r;
  T u[NL_QB][3];
  Pt<T> xq[NL_QB];
  int cell[NL_QB][3];
  T wt[NL_QB][3][4];
#pragma unroll
  for (int b = 0; b < NL_QB; ++b) quad_point(c, c.ion[I], r, q0 + b, u[b], xq[b], cell[b], wt[b]);
  // the orbitals' values at the points, dotted with the inverse's column
  T det[NL_QB];
#pragma unroll
  for (int b = 0; b < NL_QB; ++b) det[b] = 0;
  for (int j = lane; j < n; j += 32) {
    const T bj = bcol[j];
#pragma unroll
    for (int b = 0; b < NL_QB; ++b) {
      T v = 0;
#pragma unroll 1
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          const T* row = table + (((size_t)(cell[b][0] + a) * GP + cell[b][1] + bb) * GP +
                                  cell[b][2]) * (size_t)n_pad + j;
          const T wab = wt[b][0][a] * wt[b][1][bb];
#pragma unroll
          for (int e = 0; e < 4; ++e) v += wab * wt[b][2][e] * __ldg(row + (size_t)e * n_pad);
        }
      det[b] += v * bj;
    }
  }
  T u1[NL_QB];
  jastrow_sums<T, NL_QB>(c, i, xq, u1);
  T acc0 = 0, acc1 = 0, acc2 = 0;
#pragma unroll
  for (int b = 0; b < NL_QB; ++b) {
    const T dt = warp_sum(det[b]);
    T rho;
    if constexpr (IsMixed<T>::value) rho = dt * __expf(u0 - u1[b]);
    else rho = dt * exp(u0 - u1[b]);
    const T cth = (d[0] * u[b][0] + d[1] * u[b][1] + d[2] * u[b][2]) * rinv;
    acc0 += rho;
    acc1 += cth * rho;
    acc2 += (T(1.5) * cth * cth - T(0.5)) * rho;
  }
  const double acc[3] = {(double)acc0, (double)acc1, (double)acc2};
  const double r2 = (double)r * (double)r;
  double e = 0.0;
  for (int l = 0; l < p.nl_n; ++l)
    e += p.nl_a[l] * exp(-r2 * p.nl_sinv2[l]) * (double)(2 * l + 1) * acc[l] / 12.0;
  return e;
}

// A pair within the cutoff, listed for the CTA's warps: electron, ion, U_i at r_i.
template <typename T> struct NlPair { int i, I; T u0; };

// Shared-memory layout (byte offsets, each 16-byte aligned): electrons, ions, radial
// coefficients, the warps' FP64 partial sums.
struct NlLay {
  size_t R, ion, jc, pairs, cnt, red, total;
};

__host__ __device__ inline size_t nl_al16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename T>
__host__ __device__ inline NlLay nl_lay(const Params& p) {
  NlLay L;
  const size_t njc = 2 * (size_t)(p.K2 + 3) + p.K1 + 3;
  L.R = 0;
  L.ion = nl_al16(L.R + (size_t)p.N * sizeof(Pt<T>));
  L.jc = nl_al16(L.ion + (size_t)p.n_ions * sizeof(Pt<T>));
  L.pairs = nl_al16(L.jc + njc * sizeof(T));  // NL_SEG listed pairs per warp
  L.cnt = nl_al16(L.pairs + (size_t)NL_NW * NL_SEG * sizeof(NlPair<T>));
  L.red = nl_al16(L.cnt + NL_NW * sizeof(int));
  L.total = L.red + NL_NW * sizeof(double);
  return L;
}

template <typename T>
__global__ void __launch_bounds__(NL_NT, 2) nlpp_kernel(const Params p, double* partial) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int w = blockIdx.x, N = p.N, NI = p.n_ions, n = p.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#if QMCGB_CHECK
  if (!QMC_CHECKP(p, w < p.W, CK_WALKER, w)) return;
#endif
  const int gw = blockIdx.y * NL_NW + warp;  // this warp among the walker's
  const NlLay lay = nl_lay<T>(p);
  Pt<T>* R = reinterpret_cast<Pt<T>*>(smem + lay.R);
  Pt<T>* ion = reinterpret_cast<Pt<T>*>(smem + lay.ion);
  T* jc = reinterpret_cast<T*>(smem + lay.jc);
  NlPair<T>* pairs = reinterpret_cast<NlPair<T>*>(smem + lay.pairs);
  int* cnt = reinterpret_cast<int*>(smem + lay.cnt);
  double* red = reinterpret_cast<double*>(smem + lay.red);
  const int njc = 2 * (p.K2 + 3) + p.K1 + 3;
  const double* Rg = p.R + (size_t)w * N * 3;
  for (int e = threadIdx.x; e < (N + NI) * 3; e += NL_NT) {
    const double x = e < N * 3 ? Rg[e] : p.ions[e - N * 3];
    Pt<T>* dst = e < N * 3 ? R : ion;
    const int k = e < N * 3 ? e : e - N * 3;
    if constexpr (IsMixed<T>::value) dst[k / 3].q[k % 3] = to_fixed(x, p.fx_scale);
    else dst[k / 3].x[k % 3] = x;
  }
  for (int e = threadIdx.x; e < njc; e += NL_NT) jc[e] = ((const T*)p.jc)[e];
  __syncthreads();
  NlCtx<T> c{p, R, ion, jc, (T)p.fx_unit, (T)p.fx_scale, (T)p.L, (T)p.invL,
             (T)p.h2inv, (T)p.h1inv, (T)p.rc2, (T)p.rc1, lane};
  const T* table = (const T*)p.table;
  const T* Bw = (const T*)p.binv + (size_t)w * 2 * n * n;
  double vsum = 0.0;  // lane 0 of each warp
  // 1. each warp lists the pairs within the cutoff of its electrons (lanes over ions),
  //    with U_i of each such electron; a warp with more than NL_SEG does the rest itself
  int listed = 0;  // the same on every lane
  for (int i = gw; i < N; i += NL_NW * NL_SPLIT) {
    bool have_u0 = false;
    T u0 = 0;
    for (int I0 = 0; I0 < NI; I0 += 32) {
      const int I = I0 + lane;
      bool in = false;
      if (I < NI) {
        T d[3], r;
        disp(c, R[i], ion[I], d, r);  // r_i - R_I
        in = r < (T)p.nl_rc && r > T(0);
      }
      unsigned m = __ballot_sync(0xffffffffu, in);
      if (m && !have_u0) {
        jastrow_sums<T, 1>(c, i, &R[i], &u0);
        have_u0 = true;
      }
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        if (listed < NL_SEG) {
          if (lane == 0) pairs[warp * NL_SEG + listed] = NlPair<T>{i, I0 + b, u0};
          ++listed;
        } else {
          for (int qb = 0; qb < NL_NQB; ++qb) {
            const double e = pair_batch(c, table, Bw, i, I0 + b, u0, qb * NL_QB);
            if (lane == 0) vsum += e;
          }
        }
      }
    }
  }
  if (lane == 0) cnt[warp] = listed;
  __syncthreads();
  // 2. the listed pairs' quadrature batches, dealt to the warps in turn (in the order of
  //    the warps' lists, so every E_L is the same from run to run)
  int total = 0;
#pragma unroll
  for (int q = 0; q < NL_NW; ++q) total += cnt[q];
  for (int k = warp; k < total * NL_NQB; k += NL_NW) {
    int pidx = k / NL_NQB, seg = 0;
    const int qb = k - pidx * NL_NQB;
    while (pidx >= cnt[seg]) {
      pidx -= cnt[seg];
      ++seg;
    }
    NlPair<T> pe = pairs[seg * NL_SEG + pidx];
#if QMCGB_CHECK
    if (!QMC_CHECKP(p, pe.I >= 0 && pe.I < NI, CK_PAIR, pe.I)) pe.I = 0;
    if (!QMC_CHECKP(p, pe.i >= 0 && pe.i < N, CK_ELECTRON, pe.i)) pe.i = 0;
#endif
    const double e = pair_batch(c, table, Bw, pe.i, pe.I, pe.u0, qb * NL_QB);
    if (lane == 0) vsum += e;
  }
  double v1[1] = {vsum};
  block_sum_to0<NL_NW, 1>(v1, red);
  if (threadIdx.x == 0) partial[(size_t)w * NL_SPLIT + blockIdx.y] = v1[0];
}

// eloc[w] += the walker's partial sums, in order.
__global__ void nlpp_add_kernel(const double* __restrict__ partial, double* eloc, int W,
                                int* status) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  double e = eloc[w];
  for (int q = 0; q < NL_SPLIT; ++q) e += partial[(size_t)w * NL_SPLIT + q];
  eloc[w] = e;
  if (!isfinite(e)) atomicOr(status, ST_NAN);
}

}  // namespace

int nlpp_partials_per_walker() { return NL_SPLIT; }

template <typename T>
cudaError_t launch_nlpp(const Params& p, double* eloc, double* partial, cudaStream_t s) {
  if (p.nl_n <= 0 || p.n_ions == 0 || p.W == 0) return cudaSuccess;
  const size_t bytes = nl_lay<T>(p).total;
  if (bytes > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        nlpp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  nlpp_kernel<T><<<dim3(p.W, NL_SPLIT), NL_NT, bytes, s>>>(p, partial);
  nlpp_add_kernel<<<(p.W + 255) / 256, 256, 0, s>>>(partial, eloc, p.W, p.status);
  return cudaGetLastError();
}

template cudaError_t launch_nlpp<float>(const Params&, double*, double*, cudaStream_t);
template cudaError_t launch_nlpp<double>(const Params&, double*, double*, cudaStream_t);

}  // namespace qmcgb

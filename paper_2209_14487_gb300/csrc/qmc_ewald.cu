// Coulomb energy of the local energy (Alg. 1 line 11) by Ewald summation, as a kernel of
// its own that adds to the E_L a sweep has written.
//
// Charges -1 (electrons) and +Z (ions) in the periodic cube of volume V = L^3:
//   E = sum_{a<b} q_a q_b erfc(alpha r_ab) / r_ab          (minimum image of each pair)
//     + sum_{k in half space} c_k |S(k)|^2,  c_k = (4 pi / V) exp(-k^2 / (4 alpha^2)) / k^2
//     + const                                 (-(alpha/sqrt(pi)) sum q^2 - pi Q^2/(2 V alpha^2))
// with S(k) = sum_a q_a exp(i k.r_a), k = 2 pi m / L, 0 < |m|^2 <= mmax^2; the half space
// (m0 > 0, or m0 = 0 and m1 > 0, or m0 = m1 = 0 and m2 > 0) counts each +-k pair once.
// The host lists the vectors m and their c_k and the constant.
//
// One CTA per walker.  Real space: threads over the partners b > a of each particle a.
// Reciprocal space: each thread owns up to EW_KPT vectors (S(k) in registers); the
// particles pass through shared memory in chunks as per-dimension phase tables
// exp(i 2 pi m x / L), m = 0..mmax (one sincos and mmax complex products per coordinate),
// so exp(i k.r) is two complex products.  FP32 in the mixed path, FP64 otherwise; every
// energy sum in FP64, combined in a fixed order (deterministic E_L).
#include <cmath>

#include "qmc_device.cuh"
#include "qmc_internal.h"

namespace qmcgb {
namespace {

constexpr int EW_NT = 256;
constexpr int EW_NW = EW_NT / 32;
constexpr int EW_KPT = 16;  // reciprocal vectors per thread (at most EW_NT * EW_KPT)
constexpr int EW_CH = 64;   // particles per shared-memory chunk

template <typename T> struct Cx { T re, im; };

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

template <typename T>
__device__ __forceinline__ T erfc_t(T x) {
  if constexpr (sizeof(T) == 4) return erfcf(x);
  else return erfc(x);
}

template <typename T>
__global__ void __launch_bounds__(EW_NT) ewald_kernel(const Params p, double* eloc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int w = blockIdx.x, tid = threadIdx.x, N = p.N, NI = p.n_ions, M = N + NI;
#if QMCGB_CHECK
  if (!QMC_CHECKP(p, w < p.W, CK_WALKER, w)) return;
#endif
  const int mm1 = p.coul_mmax + 1;
  Cx<T>* tab = reinterpret_cast<Cx<T>*>(smem);  // [EW_CH][3][mm1]
  double* red = reinterpret_cast<double*>(smem + (size_t)EW_CH * 3 * mm1 * sizeof(Cx<T>));
  const double* Rg = p.R + (size_t)w * N * 3;
  const T Z = (T)p.coul_Z, alpha = (T)p.coul_alpha;
  auto pos = [&](int a) { return a < N ? Rg + 3 * a : p.ions + 3 * (a - N); };
  // ---- real space
  double ereal = 0.0;
  for (int a = 0; a < M; ++a) {
    const double* xa = pos(a);
    const T qa = a < N ? T(-1) : Z;
    for (int b = a + 1 + tid; b < M; b += EW_NT) {
      const double* xb = pos(b);
      const T qb = b < N ? T(-1) : Z;
      T r2 = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double x = xa[k] - xb[k];
        x -= p.L * rint(x * p.invL);
        r2 += (T)x * (T)x;
      }
      const T r = sqrt(r2);
      ereal += (double)(qa * qb * erfc_t(alpha * r) / r);
    }
  }
  // ---- reciprocal space
  int mv[EW_KPT][3];
  Cx<T> S[EW_KPT];
#pragma unroll
  for (int j = 0; j < EW_KPT; ++j) {
    const int kk = tid + j * EW_NT;
    const bool on = kk < p.coul_nk;
#pragma unroll
    for (int d = 0; d < 3; ++d) mv[j][d] = on ? p.coul_m[3 * kk + d] : 0;
    S[j] = {T(0), T(0)};
  }
  const T tw = T(6.283185307179586476925286766559) / (T)p.L;
  for (int c0 = 0; c0 < M; c0 += EW_CH) {
    const int nch = M - c0 < EW_CH ? M - c0 : EW_CH;
    __syncthreads();  // the previous chunk's tables are read
    for (int e = tid; e < nch * 3; e += EW_NT) {
      const int pa = e / 3, d = e - 3 * pa;
      const T x = (T)pos(c0 + pa)[d];
      T sn, cs;
      if constexpr (sizeof(T) == 4) sincosf(tw * x, &sn, &cs);
      else sincos(tw * x, &sn, &cs);
      const Cx<T> base = {cs, sn};
      Cx<T>* row = tab + (size_t)(pa * 3 + d) * mm1;
      Cx<T> v = {T(1), T(0)};
      for (int m = 0; m < mm1; ++m) {
        row[m] = v;
        v = cmul(v, base);
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EW_KPT; ++j) {
      if (tid + j * EW_NT >= p.coul_nk) break;
      const int m0 = mv[j][0], m1 = mv[j][1], m2 = mv[j][2];
      const int a0 = m0 < 0 ? -m0 : m0, a1 = m1 < 0 ? -m1 : m1, a2 = m2 < 0 ? -m2 : m2;
      const T s0 = m0 < 0 ? T(-1) : T(1), s1 = m1 < 0 ? T(-1) : T(1), s2 = m2 < 0 ? T(-1) : T(1);
      Cx<T> acc = {T(0), T(0)};
      for (int pa = 0; pa < nch; ++pa) {
        const Cx<T>* row = tab + (size_t)pa * 3 * mm1;
        Cx<T> e0 = row[a0], e1 = row[mm1 + a1], e2 = row[2 * mm1 + a2];
        e0.im *= s0;  // exp(-i t) = conj(exp(i t))
        e1.im *= s1;
        e2.im *= s2;
        const Cx<T> ph = cmul(cmul(e0, e1), e2);
        const T q = c0 + pa < N ? T(-1) : Z;
        acc.re += q * ph.re;
        acc.im += q * ph.im;
      }
      S[j].re += acc.re;
      S[j].im += acc.im;
    }
  }
  double erec = 0.0;
#pragma unroll
  for (int j = 0; j < EW_KPT; ++j) {
    const int kk = tid + j * EW_NT;
    if (kk < p.coul_nk)
      erec += p.coul_c[kk] * ((double)S[j].re * (double)S[j].re +
                              (double)S[j].im * (double)S[j].im);
  }
  double v[1] = {ereal + erec};
  block_sum_to0<EW_NW, 1>(v, red);
  if (tid == 0) {
    const double e = eloc[w] + v[0] + p.coul_const;
    eloc[w] = e;
    if (!isfinite(e)) atomicOr(p.status, ST_NAN);
  }
}

}  // namespace

int ewald_max_vectors() { return EW_NT * EW_KPT; }

template <typename T>
cudaError_t launch_ewald(const Params& p, double* eloc, cudaStream_t s) {
  if (!p.coul || p.W == 0) return cudaSuccess;
  const size_t bytes =
      (size_t)EW_CH * 3 * (p.coul_mmax + 1) * sizeof(Cx<T>) + EW_NW * sizeof(double);
  if (bytes > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        ewald_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  ewald_kernel<T><<<p.W, EW_NT, bytes, s>>>(p, eloc);
  return cudaGetLastError();
}

template cudaError_t launch_ewald<float>(const Params&, double*, cudaStream_t);
template cudaError_t launch_ewald<double>(const Params&, double*, cudaStream_t);

}  // namespace qmcgb

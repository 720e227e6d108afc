// Set-up and recompute kernels: orbital rows from positions (Alg. 1 line 3), the FP64
// full recompute of A^-1 and log|det| by LU with partial pivoting, the ghost-padded
// orbital table, the Jastrow exponent U for log|Psi|, and position wrapping.
#include <cmath>

#include "qmc_device.cuh"
#include "qmc_internal.h"
#include "qmc_lu.cuh"

namespace qmcgb {

// One CTA per (walker, electron) of walkers w0, w0 + 1, ...: phi, grad phi, lap phi of the
// occupied orbitals at r_i.
template <typename T>
__global__ void __launch_bounds__(LA_NT) eval_rows_kernel(const Params p, int w0) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* part = (T*)smem;  // [16][n_pad]
  __shared__ T wts[48];
  __shared__ int cell[3];
  __shared__ T tt[3];
  const int wl = blockIdx.x / p.N, i = blockIdx.x - wl * p.N, w = w0 + wl;
  const int n = p.n, n_pad = p.n_pad;
#if QMCGB_CHECK
  if (!QMC_CHECKP(p, w >= 0 && w < p.W, CK_WALKER, w)) return;
#endif
  if (threadIdx.x < 3) {
    const int d = threadIdx.x;
    const double x = p.R[((size_t)w * p.N + i) * 3 + d];
    if constexpr (IsMixed<T>::value) {
      const uint32_t q = to_fixed(x, p.fx_scale);
      const unsigned long long prod = (unsigned long long)q * (unsigned long long)p.G;
      cell[d] = (int)(prod >> 32);
      tt[d] = (float)(uint32_t)prod * 0x1p-32f;
    } else {
      const double s = x * p.dgrid;
      int g = (int)floor(s);
      g = g > p.G - 1 ? p.G - 1 : (g < 0 ? 0 : g);
      cell[d] = g;
      tt[d] = s - (double)g;
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) basis12(tt[threadIdx.x], wts + 12 * threadIdx.x);
  __syncthreads();
  const T* table = (const T*)p.table;
  for (int it = threadIdx.x; it < 4 * n; it += LA_NT) {
    T cf[16], o4[4];
    stencil_load(table, p.GP, n_pad, cell[0], cell[1], cell[2], it % n, it / n, cf);
    stencil_reduce(cf, wts, o4);
    const int j = it % n, a = it / n;
    for (int q = 0; q < 4; ++q) part[(a * 4 + q) * n_pad + j] = o4[q];
  }
  __syncthreads();
  T* rw = (T*)p.rows + ((size_t)w * p.N + i) * 5 * n_pad;
  for (int j = threadIdx.x; j < n; j += LA_NT) {
    T o5[5];
    stencil_combine(part, n_pad, j, wts, (T)p.dgrid, o5);
    for (int q = 0; q < 5; ++q) rw[q * n_pad + j] = o5[q];
  }
}

// One CTA per (walker, spin) of walkers w0, w0 + 1, ...: FP64 LU with partial pivoting
// (row exchanges) of A_s, then the columns of A_s^-1 by forward/back substitution; writes
// B^T = (A^-1)^T in the crowd's precision, log|det A_s| and its sign, and empties the
// delayed window.  `ws` is scratch: 2 n^2 doubles per CTA.
template <typename T>
__global__ void __launch_bounds__(LA_NT) recompute_kernel(const Params p, double* ws, int w0) {
  extern __shared__ __align__(16) unsigned char smem[];
  int* piv = (int*)smem;  // [n]
  __shared__ LuShared<LA_NT> sh;
  const int ws_id = blockIdx.x, s = ws_id & 1, w = w0 + (ws_id >> 1);
  const int n = p.n, n_pad = p.n_pad;
#if QMCGB_CHECK
  if (!QMC_CHECKP(p, w >= 0 && w < p.W, CK_WALKER, w)) return;
#endif
  const int tid = threadIdx.x;
  double* LU = ws + (size_t)(w - w0) * 4 * n * n + (size_t)s * 2 * n * n;
  double* X = LU + (size_t)n * n;
  const T* rows = (const T*)p.rows + (size_t)w * p.N * 5 * n_pad;
  for (int e = tid; e < n * n; e += LA_NT) {
    const int l = e / n, j = e - l * n;
    LU[e] = (double)rows[((size_t)(s * p.n_up + l)) * 5 * n_pad + j];
  }
  __syncthreads();
  double logabs;
  int sign;
  if (!lu_invert_cta<LA_NT>(LU, X, n, piv, &sh, logabs, sign)) {
    if (tid == 0) {
      atomicOr(p.status, ST_SINGULAR);
      p.logdet[w * 2 + s] = -INFINITY;
      p.sign[w * 2 + s] = 0;
    }
    return;
  }
  T* Bg = (T*)p.binv + ((size_t)w * 2 + s) * n * n;
  for (int e = tid; e < n * n; e += LA_NT) {
    const int k = e / n, i = e - k * n;  // B^T[k][i] = (A^-1)[i][k]
    Bg[e] = (T)X[(size_t)i * n + k];
  }
  if (tid == 0) {
    p.logdet[w * 2 + s] = logabs;
    p.sign[w * 2 + s] = sign;
    if (p.win_m) p.win_m[w * 2 + s] = 0;
  }
}

// Orbital table [G][G][G][n_orb] (f64 or f32) -> [(G+3)^3][n_pad] in T with one ghost
// layer before and two after each dimension (padded index x holds node (x-1) mod G), so
// that a cell's 4^3 stencil is contiguous in z and never wraps.
template <typename T>
__global__ void pad_table_kernel(const Params p, const void* src, int src_f32, int n_orb, T* dst) {
  const size_t GP = (size_t)p.GP, total = GP * GP * GP * (size_t)p.n_pad;
  const int G = p.G;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % p.n_pad);
    const size_t cidx = idx / p.n_pad;
    const int z = (int)(cidx % GP), y = (int)((cidx / GP) % GP), x = (int)(cidx / (GP * GP));
    if (j >= p.n) {
      dst[idx] = T(0);
      continue;
    }
    const int gx = (x - 1 + G) % G, gy = (y - 1 + G) % G, gz = (z - 1 + G) % G;
    const size_t s = (((size_t)gx * G + gy) * G + gz) * (size_t)n_orb + j;
    dst[idx] = src_f32 ? (T)((const float*)src)[s] : (T)((const double*)src)[s];
  }
}

// U(R) per walker in FP64 accumulation (for log|Psi| queries).
template <typename T>
__global__ void __launch_bounds__(LA_NT) jastrow_U_kernel(const Params p, double* U) {
  __shared__ double red[LA_NWARP];
  const int w = blockIdx.x, N = p.N, NI = p.n_ions;
#if QMCGB_CHECK
  if (!QMC_CHECKP(p, w < p.W, CK_WALKER, w)) return;
#endif
  const double* R = p.R + (size_t)w * N * 3;
  const T* jc = (const T*)p.jc;
  double acc = 0.0;
  if (p.K2 > 0) {
    for (int q = threadIdx.x; q < N * N; q += LA_NT) {
      const int i = q / N, j = q - i * N;
      if (j <= i) continue;
      double d[3];
      disp_f64(R + 3 * i, R + 3 * j, p.L, p.invL, d);
      const T r = (T)sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const bool same = (i < p.n_up) == (j < p.n_up);
      T u, du, d2u;
      radial(jc + (same ? 0 : p.K2 + 3), p.K2, (T)p.h2inv, (T)p.rc2, r, u, du, d2u);
      acc += (double)u;
    }
  }
  if (p.K1 > 0) {
    for (int q = threadIdx.x; q < N * NI; q += LA_NT) {
      const int i = q / NI, I = q - i * NI;
      double d[3];
      disp_f64(R + 3 * i, p.ions + 3 * I, p.L, p.invL, d);
      const T r = (T)sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      T u, du, d2u;
      radial(jc + 2 * (p.K2 + 3), p.K1, (T)p.h1inv, (T)p.rc1, r, u, du, d2u);
      acc += (double)u;
    }
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < LA_NWARP; ++q) t += red[q];
    U[w] = t;
  }
}

// Wraps positions into [0, L); a non-finite coordinate is replaced by 0 and reported
// (ST_NAN), so that no later kernel indexes the table with it.
__global__ void wrap_kernel(double* R, size_t n3, double L, int* status) {
  const double invL = 1.0 / L;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n3;
       e += (size_t)gridDim.x * blockDim.x) {
    const double x = R[e];
    if (isfinite(x)) {
      R[e] = wrap_coord(x, L, invL);
    } else {
      R[e] = 0.0;
      atomicOr(status, (int)ST_NAN);
    }
  }
}

template <typename T>
cudaError_t launch_eval_rows(const Params& p, cudaStream_t s, int w0, int count) {
  if (count < 0) count = p.W - w0;
  if (count <= 0) return cudaSuccess;
  const size_t bytes = (size_t)16 * p.n_pad * sizeof(T);
  if (bytes + 1024 > 48 * 1024) {  // the dynamic part plus the kernel's static shared memory
    cudaError_t e = cudaFuncSetAttribute(eval_rows_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  eval_rows_kernel<T><<<count * p.N, LA_NT, bytes, s>>>(p, w0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_recompute(const Params& p, double* ws, cudaStream_t s, int w0, int count) {
  if (count < 0) count = p.W - w0;
  if (count <= 0) return cudaSuccess;
  recompute_kernel<T><<<count * 2, LA_NT, (size_t)p.n * sizeof(int), s>>>(p, ws, w0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pad_table(const Params& p, const void* src, int src_f32, int n_orb,
                             cudaStream_t s) {
  pad_table_kernel<T><<<1024, 256, 0, s>>>(p, src, src_f32, n_orb, (T*)p.table);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jastrow_U(const Params& p, double* U, cudaStream_t s) {
  jastrow_U_kernel<T><<<p.W, LA_NT, 0, s>>>(p, U);
  return cudaGetLastError();
}

cudaError_t launch_wrap_positions(double* R, size_t n3, double L, int* status, cudaStream_t s) {
  wrap_kernel<<<256, 256, 0, s>>>(R, n3, L, status);
  return cudaGetLastError();
}

template cudaError_t launch_eval_rows<double>(const Params&, cudaStream_t, int, int);
template cudaError_t launch_eval_rows<float>(const Params&, cudaStream_t, int, int);
template cudaError_t launch_recompute<double>(const Params&, double*, cudaStream_t, int, int);
template cudaError_t launch_recompute<float>(const Params&, double*, cudaStream_t, int, int);
template cudaError_t launch_pad_table<double>(const Params&, const void*, int, int, cudaStream_t);
template cudaError_t launch_pad_table<float>(const Params&, const void*, int, int, cudaStream_t);
template cudaError_t launch_jastrow_U<double>(const Params&, double*, cudaStream_t);
template cudaError_t launch_jastrow_U<float>(const Params&, double*, cudaStream_t);

}  // namespace qmcgb

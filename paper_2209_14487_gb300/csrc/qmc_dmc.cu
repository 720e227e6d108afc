// DMC reweighting and branching of a crowd on the device (arXiv:2209.14487, Alg. 1 lines
// 13-14): weights from the local energies before and after a generation, multiplicities
// from the walkers' counter-based uniforms, and the gather of the surviving and copied
// walkers' state into the other half of a double buffer.
#include <cmath>

#include "qmc_device.cuh"
#include "qmc_internal.h"

namespace qmcgb {
namespace {

constexpr int BT = 1024;  // threads of the branching kernel (one CTA)

// One CTA: weight w = exp(-tau ((E_prev + E_new) / 2 - E_T)), multiplicity
// M = floor(w + u) with u from Philox counter (gen, N, 3, 0) and the walker's key, the new
// population (walker 0 M_0 times, walker 1 M_1 times, ...) cut at `cap`, and the sums of
// w and w E_new.  mult: scratch [W].  out: [0] new size, [1] total before the cut.
__global__ void __launch_bounds__(BT) branch_kernel(const double* __restrict__ e_prev,
                                                    const double* __restrict__ e_new, int W,
                                                    int N, double tau, double e_trial,
                                                    uint64_t seed, uint32_t gen, int cap,
                                                    int* mult, int* src, int* out,
                                                    double* sums) {
  __shared__ double red[BT / 32][2];
  double sw = 0.0, swe = 0.0;
  for (int w = threadIdx.x; w < W; w += BT) {
    const double wt = exp(-tau * (0.5 * (e_prev[w] + e_new[w]) - e_trial));
    uint32_t x[4] = {gen, (uint32_t)N, 3u, 0u};
    philox4x32_10(x, (uint32_t)seed, (uint32_t)w ^ (uint32_t)(seed >> 32));
    const double u = uniform53(x[0], x[1]);
    const double m = floor(wt + u);
    mult[w] = isfinite(m) ? (m < 0.0 ? 0 : (m > 1e6 ? 1000000 : (int)m)) : 0;
    sw += wt;
    swe += wt * e_new[w];
  }
  sw = warp_sum(sw);
  swe = warp_sum(swe);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = sw;
    red[threadIdx.x >> 5][1] = swe;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < BT / 32; ++q) {
      a += red[q][0];
      b += red[q][1];
    }
    sums[0] = a;
    sums[1] = b;
    // exclusive scan of the multiplicities into slot ranges (small populations: serial)
    long long d = 0;
    for (int w = 0; w < W; ++w) {
      const int m = mult[w];
      mult[w] = (int)(d < cap ? d : cap);
      d += m;
    }
    out[0] = (int)(d < cap ? d : cap);
    out[1] = (int)(d < 0x7fffffff ? d : 0x7fffffff);
  }
  __syncthreads();
  const int total = out[0];
  for (int w = threadIdx.x; w < W; w += BT) {
    const int d0 = mult[w];
    const int d1 = w + 1 < W ? mult[w + 1] : total;
    for (int d = d0; d < d1 && d < cap; ++d) src[d] = w;
  }
}

__device__ __forceinline__ void copy_bytes(void* dst, const void* src, size_t bytes) {
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) | bytes) & 15) == 0) {
    uint4* d = reinterpret_cast<uint4*>(dst);
    const uint4* s = reinterpret_cast<const uint4*>(src);
    for (size_t e = threadIdx.x; e < bytes / 16; e += blockDim.x) d[e] = s[e];
  } else {
    uint8_t* d = reinterpret_cast<uint8_t*>(dst);
    const uint8_t* s = reinterpret_cast<const uint8_t*>(src);
    for (size_t e = threadIdx.x; e < bytes; e += blockDim.x) d[e] = s[e];
  }
}

// CTA d copies walker src[d]'s state from the `from` buffers into slot d of `to`.
__global__ void gather_kernel(WalkerState to, WalkerState from, const int* __restrict__ src,
                              const double* __restrict__ e_new, double* e_out) {
  const int d = blockIdx.x, w = src[d];
#if QMCGB_CHECK
  if (!QMC_CHECK(from.status, from.check_info, w >= 0 && w < from.n_walkers, CK_SOURCE, w)) return;
#endif
  copy_bytes(to.R + (size_t)d * to.r_elems, from.R + (size_t)w * to.r_elems,
             sizeof(double) * to.r_elems);
  copy_bytes((char*)to.rows + (size_t)d * to.rows_bytes,
             (const char*)from.rows + (size_t)w * to.rows_bytes, to.rows_bytes);
  copy_bytes((char*)to.binv + (size_t)d * to.binv_bytes,
             (const char*)from.binv + (size_t)w * to.binv_bytes, to.binv_bytes);
  copy_bytes((char*)to.jgl + (size_t)d * to.jgl_bytes,
             (const char*)from.jgl + (size_t)w * to.jgl_bytes, to.jgl_bytes);
  if (threadIdx.x < 2) {
    to.logdet[2 * d + threadIdx.x] = from.logdet[2 * w + threadIdx.x];
    to.sign[2 * d + threadIdx.x] = from.sign[2 * w + threadIdx.x];
  }
  if (threadIdx.x == 0) {
    to.jvalid[d] = from.jvalid[w];
    if (e_out) e_out[d] = e_new[w];
  }
}

}  // namespace

cudaError_t launch_branch(const double* e_prev, const double* e_new, int W, int N, double tau,
                          double e_trial, uint64_t seed, uint32_t gen, int cap, int* mult,
                          int* src, int* out, double* sums, cudaStream_t s) {
  branch_kernel<<<1, BT, 0, s>>>(e_prev, e_new, W, N, tau, e_trial, seed, gen, cap, mult, src,
                                 out, sums);
  return cudaGetLastError();
}

cudaError_t launch_gather(const WalkerState& to, const WalkerState& from, const int* src,
                          int n_new, const double* e_new, double* e_out, cudaStream_t s) {
  if (n_new <= 0) return cudaSuccess;
  gather_kernel<<<n_new, 256, 0, s>>>(to, from, src, e_new, e_out);
  return cudaGetLastError();
}

}  // namespace qmcgb

// Allocation-free FP64 batched inverse (see qmc_inverse_noalloc in include/qmcgb.h).
//
// Some callers cannot allocate device memory at the moment they need this operation: code
// running inside a host callback or a latency-critical loop, where cudaMalloc's implicit
// synchronisation is not allowed or not affordable, or an embedding runtime that hands all
// device memory to its own pool and forbids other allocations.  This entry point serves
// them with a workspace that is part of the library image: a file-scope device array of
// fixed size that every GPU loading the library holds until the process exits.
#include <cmath>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "../../include/qmcgb.h"
#include "qmc_internal.h"

namespace {

// LU factors of the matrices of one launch: 2^21 doubles (16 MiB).  A launch takes as
// many n x n matrices as fit; larger batches run as several launches in stream order.
constexpr size_t kScratchDoubles = size_t(1) << 21;
constexpr int kMaxN = 1024;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_lu_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_lu_scratch on the current device; resolved once per device.  In
// host code the symbol itself only names a host-side stand-in, so kernels get this
// address instead.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QMC_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return QMC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_lu_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return QMC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return QMC_OK;
}

// One CTA per matrix: LU with partial pivoting (row exchanges) in the scratch slot, then
// column c of A^-1 by forward/back substitution written straight into the output (which
// doubles as the solve buffer), log|det| and sign (0 when a zero pivot makes A singular).
__global__ void __launch_bounds__(kThreads) inverse_lu_kernel(const double* __restrict__ a,
                                                              int n, double* lu_all,
                                                              double* inv, double* logdet,
                                                              int* sign) {
  extern __shared__ int piv[];  // [n]
  __shared__ double red_v[kThreads / 32];
  __shared__ int red_i[kThreads / 32];
  __shared__ int s_piv, s_sing, s_sign;
  __shared__ double s_logabs;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t nn = (size_t)n * n;
  double* LU = lu_all + (size_t)b * nn;
  const double* A = a + (size_t)b * nn;
  double* X = inv + (size_t)b * nn;
  for (size_t e = tid; e < nn; e += kThreads) LU[e] = A[e];
  if (tid == 0) { s_sing = 0; s_sign = 1; s_logabs = 0.0; }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += kThreads) {
      const double v = fabs(LU[(size_t)i * n + k]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = red_v[0];
      int ib = red_i[0];
      for (int q = 1; q < kThreads / 32; ++q)
        if (red_v[q] > bv || (red_v[q] == bv && red_i[q] < ib)) { bv = red_v[q]; ib = red_i[q]; }
      piv[k] = ib;
      s_piv = ib;
      if (!(bv > 0.0)) s_sing = 1;
    }
    __syncthreads();
    if (s_sing) break;
    const int pk = s_piv;
    if (pk != k) {
      for (int j = tid; j < n; j += kThreads) {
        const double t = LU[(size_t)k * n + j];
        LU[(size_t)k * n + j] = LU[(size_t)pk * n + j];
        LU[(size_t)pk * n + j] = t;
      }
    }
    __syncthreads();
    const double akk = LU[(size_t)k * n + k];
    if (tid == 0) {
      if (pk != k) s_sign = -s_sign;
      if (akk < 0.0) s_sign = -s_sign;
      s_logabs += log(fabs(akk));
    }
    for (int i = k + 1 + tid; i < n; i += kThreads) LU[(size_t)i * n + k] /= akk;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = tid; e < m * m; e += kThreads) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      LU[(size_t)i * n + j] -= LU[(size_t)i * n + k] * LU[(size_t)k * n + j];
    }
    __syncthreads();
  }
  if (s_sing) {
    for (size_t e = tid; e < nn; e += kThreads) X[e] = NAN;
    if (tid == 0) {
      logdet[b] = -INFINITY;
      sign[b] = 0;
    }
    return;
  }
  for (int c = tid; c < n; c += kThreads) {
    for (int i = 0; i < n; ++i) X[(size_t)i * n + c] = (i == c) ? 1.0 : 0.0;
    for (int k = 0; k < n; ++k) {
      const int pk = piv[k];
      if (pk != k) {
        const double t = X[(size_t)k * n + c];
        X[(size_t)k * n + c] = X[(size_t)pk * n + c];
        X[(size_t)pk * n + c] = t;
      }
    }
    for (int i = 0; i < n; ++i) {
      double acc = X[(size_t)i * n + c];
      for (int j = 0; j < i; ++j) acc -= LU[(size_t)i * n + j] * X[(size_t)j * n + c];
      X[(size_t)i * n + c] = acc;
    }
    for (int i = n - 1; i >= 0; --i) {
      double acc = X[(size_t)i * n + c];
      for (int j = i + 1; j < n; ++j) acc -= LU[(size_t)i * n + j] * X[(size_t)j * n + c];
      X[(size_t)i * n + c] = acc / LU[(size_t)i * n + i];
    }
  }
  if (tid == 0) {
    logdet[b] = s_logabs;
    sign[b] = s_sign;
  }
}

}  // namespace

extern "C" int qmc_inverse_noalloc(const double* a, int n, int batch, double* inv, double* logdet,
                                   int* sign, void* cuda_stream) {
  if (batch < 0 || n < 1) return QMC_ERR_INVALID_ARG;
  if (n > kMaxN) return QMC_ERR_UNSUPPORTED;
  if (batch == 0) return QMC_OK;
  // an NVTX range over the launches, as for every other C-ABI call
  struct Range {
    Range() { nvtxRangePushA("qmc_inverse_noalloc"); }
    ~Range() { nvtxRangePop(); }
  } range;
  if (!a || !inv || !logdet || !sign) return QMC_ERR_INVALID_ARG;
  double* scratch = nullptr;
  int st = scratch_address(&scratch);
  if (st) return st;
  const size_t nn = (size_t)n * n;
  const int per_launch = (int)(kScratchDoubles / nn);  // >= 2 for n <= 1024
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const size_t smem = sizeof(int) * (size_t)n;
  for (int b0 = 0; b0 < batch; b0 += per_launch) {
    const int cnt = batch - b0 < per_launch ? batch - b0 : per_launch;
    inverse_lu_kernel<<<cnt, kThreads, smem, stream>>>(a + (size_t)b0 * nn, n, scratch,
                                                        inv + (size_t)b0 * nn, logdet + b0,
                                                        sign + b0);
    if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
  }
  return QMC_OK;
}

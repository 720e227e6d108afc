// FP64 LU with partial pivoting and the inverse by substitution, run by one CTA: the full
// recompute of A^-1, log|det A| and its sign (Alg. 1 line 3, repeated every n_recompute
// generations), shared by the periodic recompute kernel and the move kernel's repair of a
// walker whose FP32 inverse has drifted.
#pragma once
#include <cmath>

namespace qmcgb {

// Shared scalars of one CTA's factorisation (NTH threads).
template <int NTH>
struct LuShared {
  double red_v[NTH / 32];
  int red_i[NTH / 32];
  int piv_k, sing, sign;
  double logabs;
};

// LU (n x n, row major, global memory) holds A on entry; on return it holds the factors
// (unit lower triangle below the diagonal, U on and above it) and X (n x n, row major)
// holds A^-1: column c solves L U x = P e_c, where the permuted unit vector's 1 sits at
// row pos(c), so the forward substitution starts there.  piv: n ints of shared memory.
// Returns false (uniformly) when a zero pivot shows A singular; logabs and sign are the
// determinant's on every thread.  Every thread of the CTA calls it.
template <int NTH>
__device__ bool lu_invert_cta(double* __restrict__ LU, double* __restrict__ X, int n,
                              int* piv, LuShared<NTH>* sh, double& logabs, int& sign) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    sh->sing = 0;
    sh->sign = 1;
    sh->logabs = 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += NTH) {
      const double v = fabs(LU[(size_t)i * n + k]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) {
      sh->red_v[warp] = best;
      sh->red_i[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = sh->red_v[0];
      int ib = sh->red_i[0];
      for (int q = 1; q < NTH / 32; ++q)
        if (sh->red_v[q] > b || (sh->red_v[q] == b && sh->red_i[q] < ib)) {
          b = sh->red_v[q];
          ib = sh->red_i[q];
        }
      piv[k] = ib;
      sh->piv_k = ib;
      if (!(b > 0.0)) sh->sing = 1;
    }
    __syncthreads();
    if (sh->sing) break;
    const int pk = sh->piv_k;
    if (pk != k) {
      for (int j = tid; j < n; j += NTH) {
        const double t = LU[(size_t)k * n + j];
        LU[(size_t)k * n + j] = LU[(size_t)pk * n + j];
        LU[(size_t)pk * n + j] = t;
      }
    }
    __syncthreads();
    const double akk = LU[(size_t)k * n + k];
    if (tid == 0) {
      if (pk != k) sh->sign = -sh->sign;
      if (akk < 0.0) sh->sign = -sh->sign;
      sh->logabs += log(fabs(akk));
    }
    for (int i = k + 1 + tid; i < n; i += NTH) LU[(size_t)i * n + k] /= akk;
    __syncthreads();
    // rank-1 update of the trailing block: rows over warps, columns over lanes (row k of
    // U is read by every warp, from L1)
    for (int i = k + 1 + warp; i < n; i += NTH / 32) {
      const double lik = LU[(size_t)i * n + k];
      double* ri = LU + (size_t)i * n;
      const double* rk = LU + (size_t)k * n;
      for (int j = k + 1 + lane; j < n; j += 32) ri[j] -= lik * rk[j];
    }
    __syncthreads();
  }
  if (sh->sing) {
    logabs = -INFINITY;
    sign = 0;
    return false;
  }
  for (int col = tid; col < n; col += NTH) {
    // row of the 1 in P e_col after the row exchanges k <-> piv[k], k = 0..n-1
    int pos = col;
    for (int k = 0; k < n; ++k) {
      const int pk = piv[k];
      if (pos == k) pos = pk;
      else if (pos == pk) pos = k;
    }
    // forward substitution L y = P e_col: y is 0 above pos and 1 at pos; every lane of a
    // warp runs the same rows (over the zeros above its own pos, which add nothing), with
    // four partial sums so that the FP64 products do not wait on one another
    for (int i = 0; i < n; ++i) {
      const double* li = LU + (size_t)i * n;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int j = 0;
      for (; j + 4 <= i; j += 4) {
        a0 += li[j] * X[(size_t)j * n + col];
        a1 += li[j + 1] * X[(size_t)(j + 1) * n + col];
        a2 += li[j + 2] * X[(size_t)(j + 2) * n + col];
        a3 += li[j + 3] * X[(size_t)(j + 3) * n + col];
      }
      for (; j < i; ++j) a0 += li[j] * X[(size_t)j * n + col];
      X[(size_t)i * n + col] = i < pos ? 0.0 : (i == pos ? 1.0 : -((a0 + a1) + (a2 + a3)));
    }
    // back substitution U x = y
    for (int i = n - 1; i >= 0; --i) {
      const double* ui = LU + (size_t)i * n;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int j = i + 1;
      for (; j + 4 <= n; j += 4) {
        a0 += ui[j] * X[(size_t)j * n + col];
        a1 += ui[j + 1] * X[(size_t)(j + 1) * n + col];
        a2 += ui[j + 2] * X[(size_t)(j + 2) * n + col];
        a3 += ui[j + 3] * X[(size_t)(j + 3) * n + col];
      }
      for (; j < n; ++j) a0 += ui[j] * X[(size_t)j * n + col];
      X[(size_t)i * n + col] = (X[(size_t)i * n + col] - ((a0 + a1) + (a2 + a3))) / ui[i];
    }
  }
  __syncthreads();
  logabs = sh->logabs;
  sign = sh->sign;
  return true;
}

}  // namespace qmcgb

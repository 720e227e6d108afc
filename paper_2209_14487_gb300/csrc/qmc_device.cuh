// Device helpers of the PbyP move (arXiv:2209.14487, Alg. 1 lines 5-11) for sm_103a.
#pragma once
#include <cstdint>

#include "qmc_internal.h"

namespace qmcgb {

// ---------------------------------------------------------------------------------------
// Precision traits.  FP64: positions and every quantity in double.  Mixed: orbitals,
// Jastrow, ratios and the inverse in float; electron and ion positions additionally held
// as 32-bit fixed point (x = q L / 2^32), so the minimum image is an integer subtraction
// and the spline cell an integer multiply (no FP64 arithmetic in the hot loop).
// ---------------------------------------------------------------------------------------
template <typename T> struct IsMixed { static constexpr bool value = false; };
template <> struct IsMixed<float> { static constexpr bool value = true; };

// ---------------------------------------------------------------------------------------
// Counter-based RNG: Philox4x32-10 (Salmon et al., SC'11), stateless per (walker, draw).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// 53-bit uniform in (0, 1]: (k + 1/2) 2^-53, k = (a >> 5) 2^26 + (b >> 6).
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
  const unsigned long long k = ((unsigned long long)(a >> 5) << 26) | (unsigned long long)(b >> 6);
  return __dadd_rn(__ull2double_rn(k), 0.5) * 0x1p-53;
}

// The draws of one proposal: out = (chi_x, chi_y, chi_z, u_accept).  Key (seed_lo,
// walker ^ seed_hi); counter (gen, electron, slot, 0); Box-Muller on slots 0 and 1,
// the acceptance uniform from slot 2.
__device__ __forceinline__ void move_draws(uint64_t seed, uint32_t walker, uint32_t gen,
                                           uint32_t iel, double* out) {
  const uint32_t k0 = (uint32_t)seed, k1 = walker ^ (uint32_t)(seed >> 32);
  const double two_pi = 6.283185307179586476925286766559;
  uint32_t c[4] = {gen, iel, 0u, 0u};
  philox4x32_10(c, k0, k1);
  double u1 = uniform53(c[0], c[1]), u2 = uniform53(c[2], c[3]);
  double rad = sqrt(-2.0 * log(u1));
  out[0] = rad * cos(two_pi * u2);
  out[1] = rad * sin(two_pi * u2);
  uint32_t c2[4] = {gen, iel, 1u, 0u};
  philox4x32_10(c2, k0, k1);
  double u3 = uniform53(c2[0], c2[1]), u4 = uniform53(c2[2], c2[3]);
  out[2] = sqrt(-2.0 * log(u3)) * cos(two_pi * u4);
  uint32_t c3[4] = {gen, iel, 2u, 0u};
  philox4x32_10(c3, k0, k1);
  out[3] = uniform53(c3[0], c3[1]);
}

__device__ __forceinline__ double accept_uniform(uint64_t seed, uint32_t walker, uint32_t gen,
                                                 uint32_t iel) {
  uint32_t c[4] = {gen, iel, 2u, 0u};
  philox4x32_10(c, (uint32_t)seed, walker ^ (uint32_t)(seed >> 32));
  return uniform53(c[0], c[1]);
}

// FP32 draws of the mixed path from the same Philox words: 24-bit uniforms
// (x >> 8 + 1/2) 2^-24 and an FP32 Box-Muller transform.
__device__ __forceinline__ float uniform24(uint32_t x) {
  return ((float)(x >> 8) + 0.5f) * 0x1p-24f;
}

__device__ __forceinline__ void move_draws_f32(uint64_t seed, uint32_t walker, uint32_t gen,
                                               uint32_t iel, float* out) {
  const uint32_t k0 = (uint32_t)seed, k1 = walker ^ (uint32_t)(seed >> 32);
  uint32_t c[4] = {gen, iel, 0u, 0u};
  philox4x32_10(c, k0, k1);
  const float rad = sqrtf(-2.0f * logf(uniform24(c[0])));
  float sn, cs;
  sincospif(2.0f * uniform24(c[2]), &sn, &cs);
  out[0] = rad * cs;
  out[1] = rad * sn;
  uint32_t c2[4] = {gen, iel, 1u, 0u};
  philox4x32_10(c2, k0, k1);
  out[2] = sqrtf(-2.0f * logf(uniform24(c2[0]))) * cospif(2.0f * uniform24(c2[2]));
  uint32_t c3[4] = {gen, iel, 2u, 0u};
  philox4x32_10(c3, k0, k1);
  out[3] = uniform24(c3[0]);
}

__device__ __forceinline__ float accept_uniform_f32(uint64_t seed, uint32_t walker, uint32_t gen,
                                                    uint32_t iel) {
  uint32_t c[4] = {gen, iel, 2u, 0u};
  philox4x32_10(c, (uint32_t)seed, walker ^ (uint32_t)(seed >> 32));
  return uniform24(c[0]);
}

// Draws in the path's precision: FP64 Box-Muller for T = double, FP32 for T = float.
template <typename T>
__device__ __forceinline__ void draws_t(uint64_t seed, uint32_t walker, uint32_t gen,
                                        uint32_t iel, T* out) {
  if constexpr (sizeof(T) == 8) {
    move_draws(seed, walker, gen, iel, out);
  } else {
    move_draws_f32(seed, walker, gen, iel, out);
  }
}

template <typename T>
__device__ __forceinline__ T accept_uniform_t(uint64_t seed, uint32_t walker, uint32_t gen,
                                              uint32_t iel) {
  if constexpr (sizeof(T) == 8) return accept_uniform(seed, walker, gen, iel);
  else return accept_uniform_f32(seed, walker, gen, iel);
}

// ---------------------------------------------------------------------------------------
// Uniform cubic B-spline basis: weight q of a cell at t (q = 0..3 value, 4..7 first
// derivative, 8..11 second derivative, all in cell units).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T basis_one(T t, int q) {
  const T t2 = t * t, t3 = t2 * t, s = T(1) - t;
  const T sixth = T(1) / T(6);
  switch (q) {
    case 0: return s * s * s * sixth;
    case 1: return (T(3) * t3 - T(6) * t2 + T(4)) * sixth;
    case 2: return (T(-3) * t3 + T(3) * t2 + T(3) * t + T(1)) * sixth;
    case 3: return t3 * sixth;
    case 4: return T(-0.5) * s * s;
    case 5: return T(1.5) * t2 - T(2) * t;
    case 6: return T(-1.5) * t2 + t + T(0.5);
    case 7: return T(0.5) * t2;
    case 8: return s;
    case 9: return T(3) * t - T(2);
    case 10: return T(-3) * t + T(1);
    default: return t;
  }
}

// All twelve weights of one dimension at t (value, first, second derivative).
template <typename T>
__device__ __forceinline__ void basis12(T t, T* w) {
  const T t2 = t * t, t3 = t2 * t, s = T(1) - t;
  const T sixth = T(1) / T(6);
  w[0] = s * s * s * sixth;
  w[1] = (T(3) * t3 - T(6) * t2 + T(4)) * sixth;
  w[2] = (T(-3) * t3 + T(3) * t2 + T(3) * t + T(1)) * sixth;
  w[3] = t3 * sixth;
  w[4] = T(-0.5) * s * s;
  w[5] = T(1.5) * t2 - T(2) * t;
  w[6] = T(-1.5) * t2 + t + T(0.5);
  w[7] = T(0.5) * t2;
  w[8] = s;
  w[9] = T(3) * t - T(2);
  w[10] = T(-3) * t + T(1);
  w[11] = t;
}

// Radial functor u(r) with K free coefficients c[0..K-1] followed by three zeros:
// i = floor(r h^-1) (at most K-1), u = sum_m c[i+m] b_m(t); zero for r >= rc.
// FP32: branch-free; the knot index is clamped (every read stays inside the K + 3
// coefficients, also for r = NaN or inf) and the result is selected to zero outside
// [0, rc), so the terms of neighbouring partners can be evaluated interleaved.
template <typename T>
__device__ __forceinline__ void radial(const T* __restrict__ c, int K, T hinv, T rc, T r, T& u,
                                       T& du, T& d2u) {
  if constexpr (sizeof(T) == 8) {  // FP64 arithmetic is scarce: skip partners beyond rc
    if (!(r < rc)) {
      u = du = d2u = T(0);
      return;
    }
  }
  const T x = r * hinv;
  int i;
  if constexpr (sizeof(T) == 4) i = __float2int_rd(x);
  else i = __double2int_rd(x);
  i = i > K - 1 ? K - 1 : (i < 0 ? 0 : i);
  const T t = x - T(i);
  const T t2 = t * t, t3 = t2 * t, s = T(1) - t;
  const T sixth = T(1) / T(6);
  const T c0 = c[i], c1 = c[i + 1], c2 = c[i + 2], c3 = c[i + 3];
  const T uu = (c0 * s * s * s + c1 * (T(3) * t3 - T(6) * t2 + T(4)) +
                c2 * (T(-3) * t3 + T(3) * t2 + T(3) * t + T(1)) + c3 * t3) * sixth;
  const T dd = (c0 * (T(-0.5) * s * s) + c1 * (T(1.5) * t2 - T(2) * t) +
                c2 * (T(-1.5) * t2 + t + T(0.5)) + c3 * (T(0.5) * t2)) * hinv;
  const T d2 = (c0 * s + c1 * (T(3) * t - T(2)) + c2 * (T(-3) * t + T(1)) + c3 * t) * hinv * hinv;
  const bool in = r < rc;
  u = in ? uu : T(0);
  du = in ? dd : T(0);
  d2u = in ? d2 : T(0);
}

// ---------------------------------------------------------------------------------------
// Minimum-image displacements.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void disp_f64(const double* a, const double* b, double L, double invL,
                                         double* d) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double x = a[k] - b[k];
    d[k] = x - L * rint(x * invL);
  }
}

// Fixed point: the signed 32-bit difference is the minimum image exactly.
__device__ __forceinline__ void disp_fx(const uint32_t* a, const uint32_t* b, float unit,
                                        float* d) {
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = (float)(int32_t)(a[k] - b[k]) * unit;
}

__device__ __forceinline__ uint32_t to_fixed(double x, double scale) {
  return (uint32_t)__double2ull_rn(x * scale);
}

__device__ __forceinline__ double wrap_coord(double x, double L, double invL) {
  double y = x - L * floor(x * invL);
  return y;
}

// ---------------------------------------------------------------------------------------
// Reductions.
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums V values over a CTA of NW warps; thread 0 receives the totals in v.  `red` holds
// NW * V values; the caller syncs before `red` is reused.
template <int NW, int V, typename R>
__device__ __forceinline__ void block_sum_to0(R* v, R* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < V; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < V; ++q) red[warp * V + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < V; ++q) {
      R acc = red[q];
      for (int wi = 1; wi < NW; ++wi) acc += red[wi * V + q];
      v[q] = acc;
    }
  }
}

// Eight values summed over a warp by recursive halving (9 shuffles instead of 40): lane L
// ends with the warp total of value 4*bit4(L) + 2*bit3(L) + bit2(L).
template <typename R>
__device__ __forceinline__ R warp_sum8_transposed(const R* v) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  R a[4], b[2];
  const bool u4 = lane & 16, u3 = lane & 8, u2 = lane & 4;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const R send = u4 ? v[q] : v[q + 4];
    const R keep = u4 ? v[q + 4] : v[q];
    a[q] = keep + __shfl_xor_sync(full, send, 16);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const R send = u3 ? a[q] : a[q + 2];
    const R keep = u3 ? a[q + 2] : a[q];
    b[q] = keep + __shfl_xor_sync(full, send, 8);
  }
  R c = (u2 ? b[1] : b[0]) + __shfl_xor_sync(full, u2 ? b[0] : b[1], 4);
  c += __shfl_xor_sync(full, c, 2);
  c += __shfl_xor_sync(full, c, 1);
  return c;
}

// Sums eight values over a CTA of NW warps and hands every thread all eight totals (one
// barrier).  `red` holds NW * 8 values and must not be rewritten before every warp has
// read it.
template <int NW, typename R>
__device__ __forceinline__ void block_allreduce8(R* v, R* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const R c = warp_sum8_transposed(v);
  if ((lane & 3) == 0) red[warp * 8 + (lane >> 2)] = c;
  __syncthreads();
  R t = R(0);
  if (lane < 8) {
#pragma unroll
    for (int w = 0; w < NW; ++w) t += red[w * 8 + lane];
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __shfl_sync(0xffffffffu, t, q);
}

// Sixteen values summed over a CTA of NW warps, every thread receives all totals (one
// barrier).  `red` holds NW * 16 values.
template <int NW, typename R>
__device__ __forceinline__ void block_allreduce16(R* v, R* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const R c0 = warp_sum8_transposed(v);
  const R c1 = warp_sum8_transposed(v + 8);
  if ((lane & 3) == 0) {
    red[warp * 16 + (lane >> 2)] = c0;
    red[warp * 16 + 8 + (lane >> 2)] = c1;
  }
  __syncthreads();
  R t = R(0);
  if (lane < 16) {
#pragma unroll
    for (int w = 0; w < NW; ++w) t += red[w * 16 + lane];
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __shfl_sync(0xffffffffu, t, q);
}

// ---------------------------------------------------------------------------------------
// TMA and mbarrier helpers (inline PTX, sm_90+ forms available on sm_103a).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One 4-D tile of a tensor map into shared memory, completing on `bar`.
// Coordinates are innermost first; c0 * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2,
                                            int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"((unsigned long long)tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `parity` of `bar`, for at most about one second of wall time (and at
// most 2^22 polls); false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
  return false;
}

// ---------------------------------------------------------------------------------------
// tcgen05 (fifth-generation tensor core) helpers: TMEM allocation, the kind::tf32 MMA with
// both operands in shared memory and the accumulator in TMEM, completion through an
// mbarrier, and TMEM loads for the epilogue.  All cta_group::1 (one SM per tile).
// ---------------------------------------------------------------------------------------

// Allocates `ncols` TMEM columns (a power of two, 32..512) for the CTA; the base address
// is written to *dst.  Executed by one whole warp.  The CTA keeps its permit to allocate
// again (an allocation lives for one flush).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(dst)),
               "r"(ncols)
               : "memory");
}

// Frees a TMEM allocation; by the warp that allocated it.
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand without swizzling: core matrices of
// 8 rows x 16 bytes stored as 128 contiguous bytes, `lbo` bytes apart along K and `sbo`
// bytes apart along M (or N).  Bits 46-48 hold the descriptor version (0b001).
__device__ __forceinline__ uint64_t tc_smem_desc(const void* base, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = smem_addr(base);
  return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, both operands K-major,
// dense, M = 128 and N (a multiple of 16, 16..256).
__device__ __forceinline__ uint32_t tc_idesc_tf32(uint32_t n_cols) {
  return (1u << 4)              // D format: F32
         | (2u << 7)            // A format: TF32
         | (2u << 10)           // B format: TF32
         | ((n_cols >> 3) << 17)  // N / 8
         | ((128u >> 4) << 24);   // M / 16
}

// D[tmem] (+)= A[smem] . B[smem]^T for one K-step of 8 TF32 elements; one thread issues.
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// One arrival on `bar` once every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (lane = warp quadrant base +
// lane id, encoded in taddr's upper half); waits for the load before returning.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// x = hi + lo with hi, lo TF32 (round to nearest): the split of the 3xTF32 products
// A.B ~ Ahi.Bhi + Ahi.Blo + Alo.Bhi, which keep FP32 accuracy on the TF32 pipe.
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hi));
  lo = __uint_as_float(l);
}

// ---------------------------------------------------------------------------------------
// Tricubic B-spline orbital stencil: for item (j, a) the 16 coefficients of orbital j at
// x offset a (4 y rows x 4 consecutive z) -- one coalesced read per (y, z) across the
// orbital lanes of a warp (orbital-fastest table with three ghost layers, so the stencil
// of cell (cx, cy, cz) starts at padded index (cx, cy, cz) and never wraps).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void stencil_load(const T* __restrict__ table, int GP, int n_pad,
                                             int cx, int cy, int cz, int j, int a, T* cf) {
  const T* base = table + (((size_t)(cx + a) * GP + cy) * GP + cz) * (size_t)n_pad + j;
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int c = 0; c < 4; ++c) cf[b * 4 + c] = __ldg(base + ((size_t)b * GP + c) * n_pad);
}

// Partial sums over (y, z) of one item: value, d/dy, d/dz and the y+z second derivatives,
// with the y and z basis weights w[12 * dim + q].
template <typename T>
__device__ __forceinline__ void stencil_reduce(const T* cf, const T* w, T* out4) {
  T v = 0, gy = 0, gz = 0, l = 0;
  const T* wy = w + 12;
  const T* wz = w + 24;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T x = cf[b * 4 + c];
      s0 += wz[c] * x;
      s1 += wz[4 + c] * x;
      s2 += wz[8 + c] * x;
    }
    v += wy[b] * s0;
    gy += wy[4 + b] * s0;
    gz += wy[b] * s1;
    l += wy[8 + b] * s0 + wy[b] * s2;
  }
  out4[0] = v;
  out4[1] = gy;
  out4[2] = gz;
  out4[3] = l;
}

// Combines the four x offsets of orbital j: phi, grad (3) and Laplacian.
template <typename T>
__device__ __forceinline__ void stencil_combine(const T* part, int n_pad, int j, const T* w,
                                                T dinv, T* o5) {
  T v = 0, gx = 0, gy = 0, gz = 0, l = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const T pv = part[(a * 4 + 0) * n_pad + j];
    const T py = part[(a * 4 + 1) * n_pad + j];
    const T pz = part[(a * 4 + 2) * n_pad + j];
    const T pl = part[(a * 4 + 3) * n_pad + j];
    v += w[a] * pv;
    gx += w[4 + a] * pv;
    gy += w[a] * py;
    gz += w[a] * pz;
    l += w[8 + a] * pv + w[a] * pl;
  }
  o5[0] = v;
  o5[1] = gx * dinv;
  o5[2] = gy * dinv;
  o5[3] = gz * dinv;
  o5[4] = l * dinv * dinv;
}

}  // namespace qmcgb

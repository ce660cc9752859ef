// Kernels of the eMAGPIE hot path (arXiv 2511.01793) for sm_103a.
//
//   k_amp_prep     a_k = sqrt(max(d_k, 0)) reordered into the FFT storage order
//   k_prep         per-minibatch probe-only arrays: max|Q|^2, gains G_l, MAGPIE
//                  weights W_z, W_R and restricted probes Q_l (Sec. 3.2)
//   k_step<M>      one CTA per scan position: gather, exit wave, 2-D FFT, modulus
//                  replacement (Def. 2.1), inverse FFT, MAGPIE object step,
//                  ePIE probe step, geometric-mean joint step (Eq. geomean)
//   k_apply        deterministic combine of the minibatch into object and probe
//   k_misfit<M>    Phi_k = 1/2 ||Q . P_k z - R_k||^2 (Eq. exit_misfit), per position
//   k_simulate<M>  d_k = |F(Q . P_k z)|^2 (Sec. 2.1 data model)
//   k_fft2<M>      batched 2-D DFT of natural-order tiles
#include <cooperative_groups.h>
#include <math.h>
#include <stdint.h>

#include "emg_fft.cuh"
#include "emg_internal.h"

namespace emg {
namespace {
#ifdef EMG_BOUNDS_CHECK
__device__ unsigned g_bounds_error;
__device__ __forceinline__ bool in_bounds(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  atomicOr(&g_bounds_error, 1u << site);
  return false;
}
#define EMG_INB(i, n, site) in_bounds((long long)(i), (long long)(n), (site))
#else
#define EMG_INB(i, n, site) true
#endif
}  // namespace

#ifdef EMG_BOUNDS_CHECK
namespace {
// Exercises the recording path of the checks: index n against a bound of n
// fails the check, so the store is skipped (buf holds n + 1 floats regardless).
__global__ void k_bounds_probe(float* buf, int n) {
  if (threadIdx.x == 0 && EMG_INB(n, n, kBcLevel)) buf[n] = 1.f;
}
}  // namespace
#endif

cudaError_t bounds_probe(unsigned* out) {
#ifdef EMG_BOUNDS_CHECK
  float* buf = nullptr;
  const int n = 32;
  cudaError_t e = cudaMalloc(&buf, (n + 1) * sizeof(float));
  if (e != cudaSuccess) return e;
  k_bounds_probe<<<1, 32>>>(buf, n);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(buf);
  if (e != cudaSuccess) return e;
  return bounds_errors_take(out);
#else
  *out = 0;
  return cudaErrorNotSupported;
#endif
}

cudaError_t bounds_errors_take(unsigned* out) {
#ifdef EMG_BOUNDS_CHECK
  unsigned zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_bounds_error, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bounds_error, &zero, sizeof(unsigned));
  return e;
#else
  *out = 0;
  return cudaErrorNotSupported;
#endif
}
}  // namespace emg

namespace emg {

namespace {

template <int M> struct StepThreads;
template <> struct StepThreads<16> { static constexpr int value = 64; };
template <> struct StepThreads<32> { static constexpr int value = 128; };
template <> struct StepThreads<64> { static constexpr int value = 256; };
template <> struct StepThreads<128> { static constexpr int value = 512; };

__device__ __forceinline__ float2 czero() { return make_float2(0.f, 0.f); }

// Programmatic dependent launch: the minibatch kernels (prep -> step ->
// combine) are launched so that each may start while its predecessor drains.
// pdl_wait() blocks until the predecessor grid has finished and its writes are
// visible; everything before it may only read data that no predecessor
// writes (scan order, positions, amplitudes).  pdl_trigger() lets the
// successor launch.  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float2 gather_obj(const float2* __restrict__ z, int n_rows, int n_cols,
                                             int gr, int gc) {
  if ((unsigned)gr < (unsigned)n_rows && (unsigned)gc < (unsigned)n_cols)
    return z[(size_t)gr * n_cols + gc];
  return czero();
}

// num / den with 0/0 read as 0 (den == 0 gives 0).
__device__ __forceinline__ float safe_div(float num, float den) { return den != 0.f ? num / den : 0.f; }
__device__ __forceinline__ float2 safe_cdiv(float2 num, float den) {
  return den != 0.f ? make_float2(num.x / den, num.y / den) : czero();
}

// Principal square root of w (Kahan, "Branch cuts for complex elementary functions", 1987).
__device__ __forceinline__ float2 csqrt_principal(float2 w) {
  const float mag = sqrtf(fmaf(w.x, w.x, w.y * w.y));
  if (mag == 0.f) return czero();
  const float t = sqrtf(0.5f * (fabsf(w.x) + mag));
  if (w.x >= 0.f) return make_float2(t, w.y / (2.f * t));
  return make_float2(fabsf(w.y) / (2.f * t), copysignf(t, w.y));
}

// y with y^2 = x * xp and Re(y conj(x)) >= 0 (Eq. geomean); ties keep the principal root.
__device__ __forceinline__ float2 geometric_mean_aligned(float2 x, float2 xp) {
  float2 y = csqrt_principal(cmul(x, xp));
  if (fmaf(y.x, x.x, y.y * x.y) < 0.f) y = make_float2(-y.x, -y.y);
  return y;
}

// y with y^2 = x * xp and Re(y conj(x)) >= 0 (Eq. geomean), branch-free.
// With w = x xp = u + i v, s = (|u| + |w|)/2, t = sqrt(s), h = 1/(2t):
// (t, v h) squares to w when u >= 0 (Kahan's half-angle form), and (v h, t)
// squares to w when u < 0 (its real part is (v^2 - 4 s^2)/(4 s) = u); either
// root is then negated if it points away from x.  Square roots come from rsqrtf.
__device__ __forceinline__ float2 geometric_mean_aligned_fast(float2 x, float2 xp) {
  const float2 w = cmul(x, xp);
  const float n = fmaf(w.x, w.x, w.y * w.y);
  const float mag = n * rsqrtf(n);
  const float s = 0.5f * (fabsf(w.x) + mag);
  const float rt = rsqrtf(s);
  const float t = s * rt, vh = w.y * (0.5f * rt);
  float2 y = w.x >= 0.f ? make_float2(t, vh) : make_float2(vh, t);
  const float sgn = fmaf(y.x, x.x, y.y * x.y) < 0.f ? -1.f : 1.f;
  y = n > 0.f ? make_float2(sgn * y.x, sgn * y.y) : czero();
  return y;
}

// c + a b, c - a b and c + conj(a) b as chains of two fused multiply-adds per part.
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfnma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}

// y with y^2 = x * xp and Re(y conj(x)) >= 0 (Eq. geomean), branch-free, in
// the half-angle form of geometric_mean_aligned_fast with s' = 2 s, so that
// t = sqrt(s) = s' r / sqrt(2) and v h = v r / sqrt(2) for r = 1 / sqrt(s').
// A floor of 1e-37 under both square roots gives y = 0 for w = 0 without a
// branch; it changes no result for |w|^2 above about 1e-29.  The sign flip
// is applied to the sign bit when Re(y conj(x)) < 0.
__device__ __forceinline__ float2 geomean_aligned_root(float2 x, float2 xp) {
  const float2 w = cmul(x, xp);
  const float n = fmaf(w.x, w.x, w.y * w.y);
  const float mag = n * rsqrtf(n + 1e-37f);
  const float s2 = fabsf(w.x) + mag;
  const float rr = rsqrtf(s2 + 1e-37f) * 0.70710678118654752f;
  const float t = s2 * rr, vh = w.y * rr;
  const float yx = w.x >= 0.f ? t : vh, yy = w.x >= 0.f ? vh : t;
  const unsigned sbit = fmaf(yx, x.x, yy * x.y) < 0.f ? 0x80000000u : 0u;
  return make_float2(__uint_as_float(__float_as_uint(yx) ^ sbit), __uint_as_float(__float_as_uint(yy) ^ sbit));
}

// a5 (finest level) + a6 + a7 at one pixel: with MG the fine MAGPIE step from
// the prolonged coarse correction pro, z^+ = zp + G_0 (R - Q zp) with
// zp = z_k + pro, else z^+ = z_k + G_0 (R - Q z_k); Q^+ = Q + conj(z_k)(R - Q z_k)/mu_k;
// with JOINT their aligned geometric means with z_k and Q (Eq. geomean).
template <bool MG, bool JOINT>
__device__ __forceinline__ void update_pixel(float2 zk, float2 q, float2 g0, float2 R, float2 pro, float inv_mu,
                                             float2& zn, float2& qn) {
  const float2 res = cfnma(q, zk, R);
  float2 zplus;
  if constexpr (MG) {
    const float2 zp = cadd(zk, pro);
    zplus = cfma(g0, cfnma(q, zp, R), zp);
  } else {
    zplus = cfma(g0, res, zk);
  }
  const float2 qplus = cfma_conj(zk, cscale(res, inv_mu), q);
  if constexpr (JOINT) {
    zn = geomean_aligned_root(zk, zplus);
    qn = geomean_aligned_root(q, qplus);
  } else {
    zn = zplus;
    qn = qplus;
  }
}

// Atomic object scatter of one patch pixel (EMG_SCATTER_ATOMIC): weighted mean
// (combine 0) adds w z~ and w, the summed corrections (combine 1) add z~ - z_k.
__device__ __forceinline__ void scatter_atomic(float2* num, float* den, int combine, int n_rows, int n_cols, int gr,
                                               int gc, float2 zn, float2 zk, float w) {
  if ((unsigned)gr >= (unsigned)n_rows || (unsigned)gc >= (unsigned)n_cols) return;
  const size_t gi = (size_t)gr * n_cols + gc;
  if (combine == 0) {
    atomicAdd(num + gi, make_float2(w * zn.x, w * zn.y));
    atomicAdd(den + gi, w);
  } else {
    atomicAdd(num + gi, make_float2(zn.x - zk.x, zn.y - zk.y));
  }
}

template <typename T>
__device__ __forceinline__ T lerp4(T a, T b, T c, T d);
template <>
__device__ __forceinline__ float lerp4<float>(float a, float b, float c, float d) {
  return 0.5625f * a + 0.1875f * b + 0.1875f * c + 0.0625f * d;
}
template <>
__device__ __forceinline__ float2 lerp4<float2>(float2 a, float2 b, float2 c, float2 d) {
  return make_float2(lerp4<float>(a.x, b.x, c.x, d.x), lerp4<float>(a.y, b.y, c.y, d.y));
}

// (I_H^h y)(r, c) for a coarse array of side mc with row stride `stride`.
// kind 0: piecewise constant (4 (I_h^H)^T); kind 1: cell-centred bilinear, edge clamp.
template <typename T>
__device__ __forceinline__ T prolong_at(const T* y, int stride, int mc, int r, int c, int kind) {
  const int i = r >> 1, j = c >> 1;
  const T v = y[i * stride + j];
  if (kind == 0) return v;
  const int i2 = (r & 1) ? min(i + 1, mc - 1) : max(i - 1, 0);
  const int j2 = (c & 1) ? min(j + 1, mc - 1) : max(j - 1, 0);
  return lerp4<T>(v, y[i2 * stride + j], y[i * stride + j2], y[i2 * stride + j2]);
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = sh[0];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) r = fmaxf(r, sh[i]);
  __syncthreads();
  return r;
}

// Sum over the block of per-thread FP32 partials: FP32 warp trees, then the
// NT/32 warp sums added in FP64 by one thread in a fixed order; the result is
// broadcast.  Deterministic; avoids FP64 work in every thread.
template <int NT>
__device__ __forceinline__ double block_sum_f(float v, float* shf, double* shd) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) r += (double)shf[i];
    shd[0] = r;
  }
  __syncthreads();
  return shd[0];
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sh[0];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) r += sh[i];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// a_k in storage order: amp[k][e_r][e_c] = sqrt(max(d[k][f(e_r)][f(e_c)], 0)).
// Warp-level max (sum) of v, written by lane 0 of each warp to sh[warp]; after
// a barrier, partials_max / partials_sum combine them in warp order, as
// block_max and block_sum_f do, so a caller can let one existing barrier serve.
__device__ __forceinline__ void warp_partial_max(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
}
__device__ __forceinline__ void warp_partial_sum(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
}
template <int NT>
__device__ __forceinline__ float partials_max(const float* sh) {
  float r = sh[0];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) r = fmaxf(r, sh[i]);
  return r;
}
template <int NT>
__device__ __forceinline__ double partials_sum(const float* sh) {
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) r += (double)sh[i];
  return r;
}

template <int M>
__global__ void __launch_bounds__(256) k_amp_prep(const float* __restrict__ d, float* __restrict__ amp,
                                                  int n_pos) {
  // One warp per storage row: the frequency row it needs is read whole with
  // consecutive lanes on consecutive words (the source may be host memory read
  // over the CPU-GPU link), then permuted through shared memory.
  constexpr int PL = (M + 31) / 32;
  __shared__ float rows[8][M];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* buf = rows[warp];
  const size_t n_rows = (size_t)n_pos * M;
  for (size_t g = (size_t)blockIdx.x * 8 + warp; g < n_rows; g += (size_t)gridDim.x * 8) {
    const size_t k = g / M;
    const int er = (int)(g % M);
    const float* src = d + (k * M + storage_to_freq<M>(er)) * M;
    float v[PL];
#pragma unroll
    for (int j = 0; j < PL; ++j)
      if (lane + 32 * j < M) v[j] = src[lane + 32 * j];
#pragma unroll
    for (int j = 0; j < PL; ++j)
      if (lane + 32 * j < M) buf[lane + 32 * j] = v[j];
    __syncwarp();
    float* dst = amp + g * M;
#pragma unroll
    for (int j = 0; j < PL; ++j) {
      const int ec = lane + 32 * j;
      if (ec < M) dst[ec] = sqrtf(fmaxf(buf[storage_to_freq<M>(ec)], 0.f));
    }
    __syncwarp();
  }
}

// a_k of the positions idx[0..b) into their slots of amp, read from d (any
// device-readable address, e.g. pinned host memory).  A small grid that runs
// beside the step kernels: each warp keeps kGatherRows rows of loads in flight.
#ifndef EMG_GATHER_BLOCKS
#define EMG_GATHER_BLOCKS 38
#endif
#ifndef EMG_GATHER_ROWS
#define EMG_GATHER_ROWS 4
#endif
#ifndef EMG_GATHER_WARPS
#define EMG_GATHER_WARPS 8
#endif
constexpr int kGatherRows = EMG_GATHER_ROWS, kGatherWarps = EMG_GATHER_WARPS, kGatherBlocks = EMG_GATHER_BLOCKS;
template <int M>
__global__ void __launch_bounds__(kGatherWarps * 32) k_amp_gather(const float* __restrict__ d,
                                                                 const int32_t* __restrict__ idx, int b,
                                                                 float* __restrict__ amp) {
  constexpr int PL = (M + 31) / 32, RW = kGatherRows;
  static_assert(M % RW == 0, "row groups stay within one position");
  __shared__ __align__(16) float rows[kGatherWarps][RW][M];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_groups = b * (M / RW);
  // rows of M >= 128 floats at a 16-byte aligned source: one 16-byte load per
  // lane and 128 columns, fewer and larger reads over the CPU-GPU link
  constexpr int PV = M / 128;
  const bool vec = PV > 0 && (reinterpret_cast<uintptr_t>(d) & 15) == 0;
  for (int g = blockIdx.x * kGatherWarps + warp; g < n_groups; g += gridDim.x * kGatherWarps) {
    const int kk = g / (M / RW), er0 = (g % (M / RW)) * RW;
    const size_t k = (size_t)idx[kk];
    if constexpr (PV > 0) {
      if (vec) {
        float4 v4[RW][PV];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
          const float4* src = reinterpret_cast<const float4*>(d + (k * M + storage_to_freq<M>(er0 + r)) * M);
#pragma unroll
          for (int j = 0; j < PV; ++j) v4[r][j] = src[lane + 32 * j];
        }
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
          for (int j = 0; j < PV; ++j) *reinterpret_cast<float4*>(&rows[warp][r][4 * (lane + 32 * j)]) = v4[r][j];
      }
    }
    if (!vec) {
      float v[RW][PL];
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const float* src = d + (k * M + storage_to_freq<M>(er0 + r)) * M;
#pragma unroll
        for (int j = 0; j < PL; ++j)
          if (lane + 32 * j < M) v[r][j] = src[lane + 32 * j];
      }
#pragma unroll
      for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int j = 0; j < PL; ++j)
          if (lane + 32 * j < M) rows[warp][r][lane + 32 * j] = v[r][j];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      float* dst = amp + (k * M + er0 + r) * M;
#pragma unroll
      for (int j = 0; j < PL; ++j) {
        const int ec = lane + 32 * j;
        if (ec < M) dst[ec] = sqrtf(fmaxf(rows[warp][r][storage_to_freq<M>(ec)], 0.f));
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Probe-only arrays of one minibatch (single CTA; O(m^2) work).
constexpr int kPrepThreads = 1024;

__global__ void __launch_bounds__(kPrepThreads) k_prep(const PrepArgs a) {
  __shared__ float redf[kPrepThreads / 32];
  const int tid = threadIdx.x;
  const int m = a.m;
  float mx = 0.f;
  for (int p = tid; p < m * m; p += kPrepThreads) mx = fmaxf(mx, cabs2(a.probe[p]));
  const float MQ = block_max<kPrepThreads>(mx, redf);
  if (tid == 0 && a.mq_next) *a.mq_next = 0u;

  // level 0: u_0 = alpha (M_Q - |Q|^2), G_0, combine weight
  for (int p = tid; p < m * m; p += kPrepThreads) {
    const float2 q = a.probe[p];
    const float a2 = cabs2(q);
    const float u = a.alpha * (MQ - a2);
    a.u[0][p] = u;
    a.G[0][p] = safe_cdiv(cconj(q), u + a2);
    a.wq[p] = fmaf(a.w_eps, MQ, a2);
  }
  for (int l = 0; l + 1 < a.levels; ++l) {
    __syncthreads();
    const int mf = m >> l, mc = mf >> 1;
    const float2* Qf = (l == 0) ? a.probe : a.Q[l];
    const float* uf = a.u[l];
    // coarse: T = I_h^H |Q_l|^2, Q_{l+1} = I_h^H Q_l, u_{l+1} = W_u^H I_h^H u_l, G_{l+1}
    for (int pc = tid; pc < mc * mc; pc += kPrepThreads) {
      const int i = pc / mc, j = pc % mc;
      float t = 0.f, ur = 0.f;
      float2 qs = czero();
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int pf = (2 * i + dy) * mf + 2 * j + dx;
          const float2 q = Qf[pf];
          t += cabs2(q);
          qs = cadd(qs, q);
          ur += uf[pf];
        }
      t *= 0.25f;
      ur *= 0.25f;
      qs = cscale(qs, 0.25f);
      const float aH = cabs2(qs);
      const float uH = safe_div(aH, t) * ur;
      a.T[l][pc] = t;
      a.Q[l + 1][pc] = qs;
      a.u[l + 1][pc] = uH;
      a.G[l + 1][pc] = safe_cdiv(cconj(qs), uH + aH);
    }
    __syncthreads();
    // fine: W_z = |Q_l|^2 / S, W_R = (I_H^h Q_{l+1}) conj(Q_l) / S, S = I_H^h T
    for (int pf = tid; pf < mf * mf; pf += kPrepThreads) {
      const int r = pf / mf, c = pf % mf;
      const float S = prolong_at<float>(a.T[l], mc, mc, r, c, a.prolong);
      const float2 pq = prolong_at<float2>(a.Q[l + 1], mc, mc, r, c, a.prolong);
      const float2 q = Qf[pf];
      a.Wz[l][pf] = safe_div(cabs2(q), S);
      a.WR[l][pf] = safe_cdiv(cmulc(pq, q), S);
    }
  }
}

// max|Q|^2 into *slot (float bits, atomicMax; the slot starts at 0).
__device__ __forceinline__ void warp_atomic_max(unsigned* slot, float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, __float_as_uint(v));
}

__global__ void __launch_bounds__(256) k_probe_max(const float2* __restrict__ probe, int n,
                                                   unsigned* __restrict__ slot) {
  float mx = 0.f;
  for (int p = blockIdx.x * 256 + threadIdx.x; p < n; p += gridDim.x * 256) mx = fmaxf(mx, cabs2(probe[p]));
  warp_atomic_max(slot, mx);
}

// Tiled probe-only prep: one CTA per tile x tile block of level-0 pixels.
// The CTA rebuilds the restriction pyramid of its tile plus a halo of
// 2^(L-1) px (bilinear prolongation reads one coarse neighbour per level) in
// shared memory and writes the level arrays of its own pixels.
constexpr int kPrepTileThreads = 256;

// Bounded wait of the fused prep: 1 s of %globaltimer, then the error flag.
constexpr unsigned long long kFusedPrepWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct PrepRegion {
  int lo_r, lo_c, h, w;   // region of one level, in that level's pixels
};

__device__ __forceinline__ PrepRegion prep_region(int m, int R0, int C0, int tile, int halo, int l) {
  PrepRegion g;
  const int lr = max(0, R0 - halo), hr = min(m, R0 + tile + halo);
  const int lc = max(0, C0 - halo), hc = min(m, C0 + tile + halo);
  g.lo_r = lr >> l;
  g.lo_c = lc >> l;
  g.h = (hr >> l) - g.lo_r;
  g.w = (hc >> l) - g.lo_c;
  return g;
}

// Prolongation at level-l pixel (r, c) from a coarse array stored on a region
// (row stride g.w, origin g.lo_r, g.lo_c); mc = full coarse side for clamping.
template <typename T>
__device__ __forceinline__ T prolong_region(const T* y, const PrepRegion& g, int mc, int r, int c, int kind) {
  const int i = r >> 1, j = c >> 1;
  const T v = y[(i - g.lo_r) * g.w + (j - g.lo_c)];
  if (kind == 0) return v;
  const int i2 = (r & 1) ? min(i + 1, mc - 1) : max(i - 1, 0);
  const int j2 = (c & 1) ? min(j + 1, mc - 1) : max(j - 1, 0);
  return lerp4<T>(v, y[(i2 - g.lo_r) * g.w + (j - g.lo_c)], y[(i - g.lo_r) * g.w + (j2 - g.lo_c)],
                  y[(i2 - g.lo_r) * g.w + (j2 - g.lo_c)]);
}

// The probe-only arrays of one tile (index `t`) of the probe, computed by
// `nt` threads of a CTA with `smp` as shared scratch (prep_tile_smem bytes).
__device__ __forceinline__ void prep_tile_body(const PrepArgs& a, int t, int tid, int nt, float2* smp) {
  const int m = a.m, L = a.levels, tile = a.tile, halo = a.halo;
  const int tiles_per_row = m / tile;
  const int R0 = (t / tiles_per_row) * tile, C0 = (t % tiles_per_row) * tile;
  const float MQ = __uint_as_float(*a.mq_read);
  if (t == 0 && tid == 0) *a.mq_next = 0u;

  // carve shared memory: per level Q_l (float2), u_l (float), T_l (float, level l+1 region)
  float2* Qs[kMaxLevels];
  float* us[kMaxLevels];
  float* Ts[kMaxLevels];
  {
    char* base = (char*)smp;
    size_t off = 0;
    for (int l = 0; l < L; ++l) {
      const PrepRegion g = prep_region(m, R0, C0, tile, halo, l);
      Qs[l] = (float2*)(base + off);
      off += (size_t)g.h * g.w * sizeof(float2);
      us[l] = (float*)(base + off);
      off += (size_t)g.h * g.w * sizeof(float);
      if (l + 1 < L) {
        const PrepRegion gc = prep_region(m, R0, C0, tile, halo, l + 1);
        Ts[l] = (float*)(base + off);
        off += (size_t)gc.h * gc.w * sizeof(float);
      }
      off = (off + 15) & ~(size_t)15;
    }
  }
  // level 0
  {
    const PrepRegion g = prep_region(m, R0, C0, tile, halo, 0);
    for (int p = tid; p < g.h * g.w; p += nt) {
      const int r = g.lo_r + p / g.w, c = g.lo_c + p % g.w;
      const float2 q = a.probe[r * m + c];
      const float a2 = cabs2(q);
      const float u = a.alpha * (MQ - a2);
      Qs[0][p] = q;
      us[0][p] = u;
      if (r >= R0 && r < R0 + tile && c >= C0 && c < C0 + tile) {
        a.G[0][r * m + c] = safe_cdiv(cconj(q), u + a2);
        a.wq[r * m + c] = fmaf(a.w_eps, MQ, a2);
      }
    }
  }
  for (int l = 0; l + 1 < L; ++l) {
    __syncthreads();
    const PrepRegion gf = prep_region(m, R0, C0, tile, halo, l);
    const PrepRegion gc = prep_region(m, R0, C0, tile, halo, l + 1);
    const int mf = m >> l, mc = mf >> 1;
    const int tr0 = R0 >> (l + 1), tc0 = C0 >> (l + 1), tsz = tile >> (l + 1);
    // coarse: T = I_h^H |Q_l|^2, Q_{l+1} = I_h^H Q_l, u_{l+1} = W_u^H I_h^H u_l, G_{l+1}
    for (int p = tid; p < gc.h * gc.w; p += nt) {
      const int i = p / gc.w, j = p % gc.w;
      float t = 0.f, ur = 0.f;
      float2 qs = czero();
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int pf = (2 * i + dy) * gf.w + 2 * j + dx;
          const float2 q = Qs[l][pf];
          t += cabs2(q);
          qs = cadd(qs, q);
          ur += us[l][pf];
        }
      t *= 0.25f;
      ur *= 0.25f;
      qs = cscale(qs, 0.25f);
      const float aH = cabs2(qs);
      const float uH = safe_div(aH, t) * ur;
      Ts[l][p] = t;
      Qs[l + 1][p] = qs;
      us[l + 1][p] = uH;
      const int gi = gc.lo_r + i, gj = gc.lo_c + j;
      if (gi >= tr0 && gi < tr0 + tsz && gj >= tc0 && gj < tc0 + tsz) {
        a.Q[l + 1][gi * mc + gj] = qs;
        a.G[l + 1][gi * mc + gj] = safe_cdiv(cconj(qs), uH + aH);
      }
    }
    __syncthreads();
    // fine weights of the tile's level-l pixels: W_z = |Q_l|^2 / S, W_R = (I_H^h Q_{l+1}) conj(Q_l) / S
    const int fr0 = R0 >> l, fc0 = C0 >> l, fsz = tile >> l;
    for (int p = tid; p < fsz * fsz; p += nt) {
      const int r = fr0 + p / fsz, c = fc0 + p % fsz;
      const float S = prolong_region<float>(Ts[l], gc, mc, r, c, a.prolong);
      const float2 pq = prolong_region<float2>(Qs[l + 1], gc, mc, r, c, a.prolong);
      const float2 q = Qs[l][(r - gf.lo_r) * gf.w + (c - gf.lo_c)];
      a.Wz[l][r * mf + c] = safe_div(cabs2(q), S);
      a.WR[l][r * mf + c] = safe_cdiv(cmulc(pq, q), S);
    }
  }
}

__global__ void __launch_bounds__(kPrepTileThreads) k_prep_tile(const PrepArgs a) {
  extern __shared__ float2 smp[];
  pdl_trigger();
  pdl_wait();  // the probe and max|Q|^2 come from the previous combine
  prep_tile_body(a, blockIdx.x, threadIdx.x, kPrepTileThreads, smp);
}

__host__ size_t prep_tile_smem(const PrepArgs& a) {
  // worst-case region sizes over tiles (interior tile)
  size_t bytes = 0;
  for (int l = 0; l < a.levels; ++l) {
    const int side = min(a.m, a.tile + 2 * a.halo) >> l;
    bytes += (size_t)side * side * (sizeof(float2) + sizeof(float));
    if (l + 1 < a.levels) {
      const int sc = min(a.m, a.tile + 2 * a.halo) >> (l + 1);
      bytes += (size_t)sc * sc * sizeof(float);
    }
    bytes = (bytes + 15) & ~(size_t)15;
  }
  return bytes;
}

constexpr size_t kPrepTileSmemMax = 96 * 1024;

// ---------------------------------------------------------------------------
// One scan position per CTA.
template <int M>
__host__ __device__ constexpr size_t level_floats2(int l) {
  return (size_t)(M >> l) * ((M >> l) + 1);
}

template <int M>
__host__ __device__ inline size_t step_smem_elems(int levels) {
  size_t n = level_floats2<M>(0);
  for (int l = 1; l < levels; ++l) n += 2 * level_floats2<M>(l);
  return n;
}

// NATURAL_AMP = true is the variant used by the allocation-free entry point:
// a.amp then holds the caller's intensities d_k in natural order and the
// amplitude sqrt(max(d, 0)) is formed on the fly.
template <int M, bool NATURAL_AMP = false>
__global__ void __launch_bounds__(StepThreads<M>::value) k_step(const StepArgs a) {
  constexpr int NT = StepThreads<M>::value;
  constexpr int S = M + 1;
  constexpr int N1 = FftPlan<M>::N1, N2 = FftPlan<M>::N2;
  extern __shared__ float2 sm[];
  __shared__ double redd[NT / 32];
  __shared__ float redf[NT / 32];
  const int tid = threadIdx.x;
  const int kb = blockIdx.x;
  int k = a.order[kb];
  if (!EMG_INB(k, a.n_pos, kBcOrder)) k = 0;
  const bool slot_ok = EMG_INB(kb, a.b, kBcPatchWrite);
  const int o_r = a.pos[2 * k], o_c = a.pos[2 * k + 1];
  float2* buf = sm;

  // a1: z_k = P_k z, psi = Q z_k, mu_k = max |z_k|^2
  float mu_l = 0.f;
  for (int p = tid; p < M * M; p += NT) {
    const int r = p / M, c = p % M;
    const float2 zk = gather_obj(a.object, a.n_rows, a.n_cols, o_r + r, o_c + c);
    buf[r * S + c] = cmul(a.probe[p], zk);
    mu_l = fmaxf(mu_l, cabs2(zk));
  }
  const float mu = block_max<NT>(mu_l, redf);

  // a2: Psi = F psi (rows, then column pass A)
  fft2_fwd_until_col_b<M, NT>(buf, tid);

  // a2 (column pass B) + a3: Psi' = a_k Psi / |Psi| (scaled by 1/M^2) + a4 start
  const float* amp = a.amp + (size_t)k * M * M;
  const float inv_m2 = 1.f / (float)(M * M);
  float acc = 0.f;
  for (int s = tid; s < M * N2; s += NT) {
    const int k2 = s / M, c = s % M;
    float2 v[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = buf[(i + N1 * k2) * S + c];
    Dft<N1, false>::run(v);
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      const float am = NATURAL_AMP
                           ? sqrtf(fmaxf(amp[storage_to_freq<M>(i + N1 * k2) * M + storage_to_freq<M>(c)], 0.f))
                           : amp[(i + N1 * k2) * M + c];
      const float p2 = cabs2(v[i]);
      if (p2 > 0.f) {
        const float inv = rsqrtf(p2);
        const float dm = fmaf(p2, inv, -am);
        acc = fmaf(dm, dm, acc);
        v[i] = cscale(v[i], am * inv * inv_m2);
      } else {
        acc = fmaf(am, am, acc);
        v[i] = make_float2(am * inv_m2, 0.f);
      }
    }
    Dft<N1, true>::run(v);
#pragma unroll
    for (int i = 0; i < N1; ++i) buf[(i + N1 * k2) * S + c] = v[i];
  }
  __syncthreads();
  // a4: R = F^-1 Psi' (natural order)
  fft2_inv_after_col_b<M, NT>(buf, tid);
  const double phi = block_sum<NT>((double)acc, redd) * (0.5 / (double)(M * M));

  // a5: MAGPIE multigrid object step, patch-local (levels > 1)
  float2* Zl[kMaxLevels];
  float2* Rl[kMaxLevels];
  {
    size_t off = level_floats2<M>(0);
    for (int l = 1; l < a.levels; ++l) {
      Zl[l] = sm + off;
      off += level_floats2<M>(l);
      Rl[l] = sm + off;
      off += level_floats2<M>(l);
    }
  }
  if (a.levels > 1) {
    // restrict level 0 -> 1: z_1 = I_h^H (W_z z_k), R_1 = I_h^H (W_R R)
    {
      constexpr int mc = M / 2, sc = mc + 1;
      const float* Wz = a.lv.Wz[0];
      const float2* WR = a.lv.WR[0];
      for (int p = tid; p < mc * mc; p += NT) {
        const int i = p / mc, j = p % mc;
        float2 zs = czero(), rs = czero();
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const int r = 2 * i + dy, c = 2 * j + dx;
            const float2 zk = gather_obj(a.object, a.n_rows, a.n_cols, o_r + r, o_c + c);
            zs = cadd(zs, cscale(zk, Wz[r * M + c]));
            rs = cadd(rs, cmul(WR[r * M + c], buf[r * S + c]));
          }
        Zl[1][i * sc + j] = cscale(zs, 0.25f);
        Rl[1][i * sc + j] = cscale(rs, 0.25f);
      }
    }
    __syncthreads();
    for (int l = 1; l + 1 < a.levels; ++l) {
      const int mf = M >> l, sf = mf + 1, mc = mf >> 1, sc = mc + 1;
      const float* Wz = a.lv.Wz[l];
      const float2* WR = a.lv.WR[l];
      for (int p = tid; p < mc * mc; p += NT) {
        const int i = p / mc, j = p % mc;
        float2 zs = czero(), rs = czero();
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const int r = 2 * i + dy, c = 2 * j + dx;
            zs = cadd(zs, cscale(Zl[l][r * sf + c], Wz[r * mf + c]));
            rs = cadd(rs, cmul(WR[r * mf + c], Rl[l][r * sf + c]));
          }
        Zl[l + 1][i * sc + j] = cscale(zs, 0.25f);
        Rl[l + 1][i * sc + j] = cscale(rs, 0.25f);
      }
      __syncthreads();
    }
    // coarsest level: correction c = G (R - Q z), stored over z
    {
      const int l = a.levels - 1;
      const int ml = M >> l, sl = ml + 1;
      const float2* G = a.lv.G[l];
      const float2* Q = a.lv.Q[l];
      for (int p = tid; p < ml * ml; p += NT) {
        const int i = p / ml, j = p % ml;
        const float2 z = Zl[l][i * sl + j];
        Zl[l][i * sl + j] = cmul(G[p], csub(Rl[l][i * sl + j], cmul(Q[p], z)));
      }
      __syncthreads();
    }
    // back up: c_l = I_H^h c_{l+1} + G_l (R_l - Q_l (z_l + I_H^h c_{l+1}))
    for (int l = a.levels - 2; l >= 1; --l) {
      const int ml = M >> l, sl = ml + 1, mc = ml >> 1, sc = mc + 1;
      const float2* G = a.lv.G[l];
      const float2* Q = a.lv.Q[l];
      for (int p = tid; p < ml * ml; p += NT) {
        const int i = p / ml, j = p % ml;
        const float2 pro = prolong_at<float2>(Zl[l + 1], sc, mc, i, j, a.prolong);
        const float2 zp = cadd(Zl[l][i * sl + j], pro);
        Zl[l][i * sl + j] = cadd(pro, cmul(G[p], csub(Rl[l][i * sl + j], cmul(Q[p], zp))));
      }
      __syncthreads();
    }
  }

  // a5 (finest level) + a6 + a7: z+, Q+, geometric-mean joint step
  const float inv_mu = mu > 0.f ? 1.f / mu : 0.f;
  const float2* G0 = a.lv.G[0];
  const float MQ = a.s_num ? __uint_as_float(*a.mq) : 0.f;  // combine weight of the atomic scatter
  float2* zt = a.zt + (size_t)kb * M * M;
  float2* qt = a.qt + (size_t)kb * M * M;
  float acc_after = 0.f;
  for (int p = tid; p < M * M; p += NT) {
    const int r = p / M, c = p % M;
    const float2 zk = gather_obj(a.object, a.n_rows, a.n_cols, o_r + r, o_c + c);
    const float2 q = a.probe[p];
    const float2 R = buf[r * S + c];
    const float2 res = csub(R, cmul(q, zk));
    float2 zplus;
    if (a.levels == 1) {
      zplus = cadd(zk, cmul(G0[p], res));
    } else {
      constexpr int mc = M / 2, sc = mc + 1;
      const float2 pro = prolong_at<float2>(Zl[1], sc, mc, r, c, a.prolong);
      const float2 zp = cadd(zk, pro);
      zplus = cadd(zp, cmul(G0[p], csub(R, cmul(q, zp))));
    }
    const float2 qplus = cadd(q, cscale(cconjmul(zk, res), inv_mu));
    float2 zn, qn;
    if (a.joint) {
      zn = geometric_mean_aligned(zk, zplus);
      qn = geometric_mean_aligned(q, qplus);
    } else {
      zn = zplus;
      qn = qplus;
    }
    if (a.s_num)
      scatter_atomic(a.s_num, a.s_den, a.combine, a.n_rows, a.n_cols, o_r + r, o_c + c, zn, zk,
                     fmaf(a.w_eps, MQ, cabs2(q)));
    else if (slot_ok)
      zt[p] = zn;
    if (slot_ok) qt[p] = qn;
    if (a.verify) acc_after += cabs2(csub(cmul(qn, zn), R));
  }
  double phi_after = 0.0;
  if (a.verify) phi_after = 0.5 * block_sum<NT>((double)acc_after, redd);
  if (tid == 0) {
    a.mu[kb] = mu;
    a.phi[kb] = phi;
    if (a.verify) a.phi_after[kb] = phi_after;
  }
}

// ---------------------------------------------------------------------------
// One scan position per cluster of C CTAs (m = 64, 128: C = 2; m = 256: C = 8).
//
// CTA `rank` owns patch rows [rank m/C, (rank+1) m/C) for the gather, the row
// FFT passes, the multigrid passes and the update, and storage columns
// [rank m/C, (rank+1) m/C) for the column FFT passes and the modulus
// replacement.  The two transposes between row and column slabs go through
// distributed shared memory; the multigrid up-pass reads the coarse rows
// adjacent to its slab from the neighbouring ranks (bilinear prolongation).
// Per CTA the shared memory is one row slab, one column slab and the object
// slab, so a minibatch of B positions occupies C B SMs.
namespace cg = cooperative_groups;

// Pixels per unrolled group in the update pass of the cluster step kernel.
#ifndef EMG_UPDATE_GROUP
#define EMG_UPDATE_GROUP 8
#endif


// Cluster barrier arrive without release semantics, for barriers that order
// execution only (every CTA of the cluster resident; no CTA exits while a
// neighbour still reads its shared memory).  A release arrive would first
// wait for all of the thread's outstanding loads and stores.
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

template <int M> struct ClusterSize;
template <> struct ClusterSize<16> { static constexpr int value = 2; };
template <> struct ClusterSize<32> { static constexpr int value = 2; };
template <> struct ClusterSize<64> { static constexpr int value = 2; };
template <> struct ClusterSize<128> { static constexpr int value = 2; };
template <> struct ClusterSize<256> { static constexpr int value = 8; };

template <int M, int C>
struct CTile {
  static constexpr int H = M / C;              // rows of a row slab, columns of a column slab
  static constexpr int SR = M + 1, SC = H + 1;  // odd strides: conflict-free lines
  static constexpr int N1 = FftPlan<M>::N1, N2 = FftPlan<M>::N2;
  static constexpr int NT = H * N1;            // one pass-A slot per thread
  static constexpr int PER = H * M / NT;       // slab pixels per thread
  static constexpr int SLOTS = H * N2 / NT;    // column pass-B slots per thread
  static constexpr size_t smem_elems = (size_t)H * SR + (size_t)M * SC + (size_t)H * M;
  static_assert(H * M % NT == 0 && H * N2 % NT == 0 && NT <= 1024, "slab must split evenly");
};

// Row slab (after the row passes) -> column slabs of all C CTAs.
template <int M, int C>
__device__ __forceinline__ void cluster_rows_to_cols(cg::cluster_group& cl, int rank, const float2* rowbuf,
                                                     float2* colbuf, int tid) {
  using T = CTile<M, C>;
  for (int s = tid; s < T::H * M; s += T::NT) {
    const int lr = s / M, e = s % M, d = e / T::H;
    float2* dst = d == rank ? colbuf : cl.map_shared_rank(colbuf, d);
    dst[(rank * T::H + lr) * T::SC + (e % T::H)] = rowbuf[lr * T::SR + e];
  }
}

// Column slab -> row slabs of all C CTAs.
template <int M, int C>
__device__ __forceinline__ void cluster_cols_to_rows(cg::cluster_group& cl, int rank, const float2* colbuf,
                                                     float2* rowbuf, int tid) {
  using T = CTile<M, C>;
  for (int s = tid; s < M * T::H; s += T::NT) {
    const int r = s / T::H, lc = s % T::H, d = r / T::H;
    float2* dst = d == rank ? rowbuf : cl.map_shared_rank(rowbuf, d);
    dst[(r % T::H) * T::SR + rank * T::H + lc] = colbuf[r * T::SC + lc];
  }
}

// Writes v into slot [rank] of `arr` in every CTA of the cluster.
template <int C, typename V>
__device__ __forceinline__ void cluster_publish(cg::cluster_group& cl, int rank, V* arr, V v) {
#pragma unroll
  for (int d = 0; d < C; ++d) *(d == rank ? &arr[rank] : cl.map_shared_rank(&arr[rank], d)) = v;
}

// (I_H^h y)(lr, c) for a coarse row slab stored with one halo row above and
// below (y points at my first row, row stride sl); lr is the local fine row.
template <typename T>
__device__ __forceinline__ T prolong_halo(const T* y, int sl, int wc, int lr, int c, int kind) {
  const int i = lr >> 1, j = c >> 1;
  const T v = y[i * sl + j];
  if (kind == 0) return v;
  const int i2 = (lr & 1) ? i + 1 : i - 1;
  const int j2 = (c & 1) ? min(j + 1, wc - 1) : max(j - 1, 0);
  return lerp4<T>(v, y[i2 * sl + j], y[i * sl + j2], y[i2 * sl + j2]);
}

// Stores coarse value v of local row i, column j (a slab of hl rows, row stride
// sl, y at my first row) where the halo rows of the prolongation read it: my
// first row into the upper neighbour's bottom halo row (my own top halo row
// at the patch's top edge), my last row into the lower neighbour's top halo
// row (my own bottom halo row at the bottom edge).  A cluster barrier makes
// the rows visible before they are read.
template <int C, typename T>
__device__ __forceinline__ void push_halo(cg::cluster_group& cl, int rank, T* y, int sl, int hl, int i, int j, T v) {
  if (i == 0) *(rank > 0 ? cl.map_shared_rank(y, rank - 1) + hl * sl + j : y - sl + j) = v;
  if (i == hl - 1) *(rank < C - 1 ? cl.map_shared_rank(y, rank + 1) - sl + j : y + hl * sl + j) = v;
}

// RIN = true: the revised exit waves R_k and the misfit partials come from the
// tensor-core DFT pair (a2-a4 done elsewhere); the kernel gathers z_k and runs
// a5-a7 only.
template <int M, int C, bool RIN = false>
__global__ void __launch_bounds__(CTile<M, C>::NT, 1) k_stepc(const StepArgs a) {
  using TL = CTile<M, C>;
  constexpr int NT = TL::NT, H = TL::H, SR = TL::SR, SC = TL::SC;
  constexpr int N1 = TL::N1, N2 = TL::N2, PER = TL::PER, SLOTS = TL::SLOTS;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) float2 sm[];  // 16-byte aligned: the update pass reads pixel pairs
  float2* rowbuf = sm;                     // H x SR: my patch rows
  float2* colbuf = sm + H * SR;            // M x SC: my storage columns (all rows); multigrid buffers later
  float2* zbuf = colbuf + M * SC;          // H x M: z_k on my rows (gathered once)
  __shared__ float xf[C];
  __shared__ double xd[C], xd2[C];
  __shared__ double redd[2];
  __shared__ float redf[NT / 32];
  __shared__ int ticket_sh;
  const int tid = threadIdx.x;
  int kb = blockIdx.x / C;
  if constexpr (!RIN) {
    if (a.prep_clusters > 0) {
      // role by ticket, taken before this launch lets the next one start: a
      // cluster only ever waits for clusters that started before it
      if (rank == 0 && tid == 0) ticket_sh = (int)(atomicAdd(a.sync, 1u) - a.ticket_base);
      cl.sync();  // every CTA of the cluster is running; rank 0's ticket is visible
      const int t = *cl.map_shared_rank(&ticket_sh, 0);
      if (t < a.prep_clusters) {
        pdl_trigger();
        pdl_wait();  // the probe and max|Q|^2 come from the previous combine
        const int tile = t * C + rank;
        if (tile < a.prep_tiles) {
          prep_tile_body(a.prep, tile, tid, NT, sm);
          __syncthreads();
          if (tid == 0) {
            __threadfence();
            atomicAdd(a.sync + 1, 1u);
          }
        }
        cl.sync();  // no CTA leaves while a peer may still read rank 0's ticket
        return;
      }
      kb = t - a.prep_clusters;
    }
  }
  int k = a.order[kb];
  if (!EMG_INB(k, a.n_pos, kBcOrder)) k = 0;
  const bool slot_ok = EMG_INB(kb, a.b, kBcPatchWrite);
  const int o_r = a.pos[2 * k], o_c = a.pos[2 * k + 1];
  const int row0 = rank * H;

  // amplitudes of my spectral slots: issued now, consumed after the row passes
  float am_reg[SLOTS][N1];
  if constexpr (!RIN) {
    const float* amp = a.amp + (size_t)k * M * M + rank * H;
#pragma unroll
    for (int t = 0; t < SLOTS; ++t) {
      const int s = tid + t * NT, k2 = s / H, lc = s % H;
#pragma unroll
      for (int i = 0; i < N1; ++i) am_reg[t][i] = __ldg(amp + (i + N1 * k2) * M + lc);
    }
  }
  pdl_trigger();
  pdl_wait();  // object, probe, max|Q|^2 and level arrays come from earlier kernels
  const float MQ = __uint_as_float(*a.mq);
  cluster_arrive_relaxed();  // completed (wait) before the first distributed shared memory access

  // a1: gather my rows, psi = Q z_k, partial mu_k
  float mu_l = 0.f;
  // pixels of a thread whose gather loads are in flight together (more costs
  // registers that the small tiles need for their occupancy)
#ifdef EMG_GATHER_UNROLL
  constexpr int kGatherUnroll = EMG_GATHER_UNROLL;
#else
  constexpr int kGatherUnroll = M >= 128 ? 8 : 4;
#endif
#pragma unroll (kGatherUnroll)
  for (int t = 0; t < PER; ++t) {
    const int p = tid + t * NT;
    const int lr = p / M, c = p % M, r = row0 + lr;
    const float2 zk = gather_obj(a.object, a.n_rows, a.n_cols, o_r + r, o_c + c);
    zbuf[p] = zk;
    if constexpr (RIN)
      rowbuf[lr * SR + c] = a.r_in[(size_t)kb * M * M + r * M + c];
    else
      rowbuf[lr * SR + c] = cmul(a.probe[r * M + c], zk);
    mu_l = fmaxf(mu_l, cabs2(zk));
  }
  // per-warp maxima of |z_k|^2; the barrier also orders the gather before the row passes
  warp_partial_max(mu_l, redf);
  __syncthreads();
  if constexpr (!RIN) {
    // a2: row passes on my rows
    gpass_a_fwd<M, H, SR, 1, NT>(rowbuf, tid);
    __syncthreads();
    gpass_b<M, H, SR, 1, NT, false>(rowbuf, tid);
    __syncthreads();
  }
  cl.barrier_wait();  // all CTAs of the cluster resident
  // transpose 1: my rows x all storage columns -> column slabs
  if constexpr (!RIN) cluster_rows_to_cols<M, C>(cl, rank, rowbuf, colbuf, tid);
  if (tid == 0) cluster_publish<C>(cl, rank, xf, partials_max<NT>(redf));
  cl.sync();
  float mu = xf[0];
#pragma unroll
  for (int d = 1; d < C; ++d) mu = fmaxf(mu, xf[d]);

  if constexpr (!RIN) {
  // a2 (columns) + a3 + a4 (columns) on my storage columns
  gpass_a_fwd<M, H, 1, SC, NT>(colbuf, tid);
  __syncthreads();
  const float inv_m2 = 1.f / (float)(M * M);
  float acc = 0.f;
#pragma unroll
  for (int t = 0; t < SLOTS; ++t) {
    const int s = tid + t * NT, k2 = s / H, lc = s % H;
    float2 v[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = colbuf[(i + N1 * k2) * SC + lc];
    Dft<N1, false>::run(v);
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      const float am = am_reg[t][i];
      const float p2 = cabs2(v[i]);
      if (p2 > 0.f) {
        const float inv = rsqrtf(p2);
        const float dm = fmaf(p2, inv, -am);
        acc = fmaf(dm, dm, acc);
        v[i] = cscale(v[i], am * inv * inv_m2);
      } else {
        acc = fmaf(am, am, acc);
        v[i] = make_float2(am * inv_m2, 0.f);
      }
    }
    Dft<N1, true>::run(v);
#pragma unroll
    for (int i = 0; i < N1; ++i) colbuf[(i + N1 * k2) * SC + lc] = v[i];
  }
  __syncthreads();
  gpass_a_inv<M, H, 1, SC, NT>(colbuf, tid);
  // per-warp misfit partials; the barrier also orders the pass before the transpose
  warp_partial_sum(acc, redf);
  __syncthreads();
  // transpose 2: all rows x my columns -> row slabs
  cluster_cols_to_rows<M, C>(cl, rank, colbuf, rowbuf, tid);
  if (tid == 0) cluster_publish<C>(cl, rank, xd, partials_sum<NT>(redf));
  cl.sync();
  // a4: inverse row passes -> R (natural order) on my rows
  gpass_b<M, H, SR, 1, NT, true>(rowbuf, tid);
  __syncthreads();
  gpass_a_inv<M, H, SR, 1, NT>(rowbuf, tid);
  __syncthreads();
  }  // !RIN

  if constexpr (!RIN) {
    if (a.prep_clusters > 0 && a.levels > 1) {
      // the level arrays of this minibatch come from the prep clusters of this launch
      if (tid == 0) {
        const unsigned long long t0 = globaltimer_ns();
        while (ld_acquire_u32(a.sync + 1) < a.prep_target) {
          if (globaltimer_ns() - t0 > kFusedPrepWaitNs) {
            atomicExch(a.sync + 2, 1u);
            break;
          }
        }
      }
      __syncthreads();
    }
  }
  // a5: MAGPIE multigrid on row slabs; level-l buffers (l >= 1) reuse colbuf.
  // Z_l keeps one halo row above and below my rows for the prolongation.
  float2* Zl[kMaxLevels];
  float2* Rl[kMaxLevels];
  {
    size_t off = 0;
    for (int l = 1; l < a.levels; ++l) {
      const int wl = M >> l, hl = wl / C, sl = wl + 1;
      Zl[l] = colbuf + off + sl;
      off += (size_t)(hl + 2) * sl;
      Rl[l] = colbuf + off;
      off += (size_t)hl * sl;
    }
  }
  // Copies the rows of the coarse correction at level l adjacent to my slab
  // (from the neighbouring ranks, or my own edge row where the patch ends).
  auto fill_halo = [&](int l) {
    const int wl = M >> l, hl = wl / C, sl = wl + 1;
    float2* Z = Zl[l];
    const float2* Zup = rank > 0 ? cl.map_shared_rank(Zl[l], rank - 1) : Z;
    const float2* Zdn = rank < C - 1 ? cl.map_shared_rank(Zl[l], rank + 1) : Z;
    for (int j = tid; j < wl; j += NT) {
      Z[-sl + j] = rank > 0 ? Zup[(hl - 1) * sl + j] : Z[j];
      Z[hl * sl + j] = rank < C - 1 ? Zdn[j] : Z[(hl - 1) * sl + j];
    }
  };
  const bool halo = a.prolong != 0;
  // With three levels (and slabs that split evenly over the threads) every
  // level array the coarse levels need is loaded into registers here, beside
  // the loads of the first restriction, so the coarse phases wait on no load.
  constexpr int wc1 = M / 2, hc1 = wc1 / C, wc2 = M / 4, hc2 = wc2 / C;
  constexpr bool kL3 = hc2 >= 1 && hc2 * wc2 >= NT && (hc2 * wc2) % NT == 0 && (hc1 * wc1) % NT == 0;
  constexpr int Q12 = kL3 ? hc2 * wc2 / NT : 1, QUP = kL3 ? hc1 * wc1 / NT : 1;
  const bool l3 = kL3 && a.levels == 3;
  float2 pf_wz1[Q12][2];     // W_z,1 at (2i + dy, 2j .. 2j + 1): (dx 0, dx 1) per dy
  float4 pf_wr1[Q12][2];     // W_R,1 at the same pixels
  float2 pf_g2[Q12], pf_q2[Q12], pf_g1[QUP], pf_q1[QUP];
  if (a.levels > 1) {
    if (l3) {
#pragma unroll
      for (int t = 0; t < Q12; ++t) {
        const int p = tid + t * NT, i = p / wc2, j = p % wc2;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const int r = rank * hc1 + 2 * i + dy, c = 2 * j;
          const int wi = EMG_INB(r * wc1 + c + 1, wc1 * wc1, kBcLevel) ? r * wc1 + c : 0;
          pf_wz1[t][dy] = __ldcg(reinterpret_cast<const float2*>(a.lv.Wz[1] + wi));
          pf_wr1[t][dy] = __ldcg(reinterpret_cast<const float4*>(a.lv.WR[1] + wi));
        }
        const int li = EMG_INB((rank * hc2 + i) * wc2 + j, wc2 * wc2, kBcLevel) ? (rank * hc2 + i) * wc2 + j : 0;
        pf_g2[t] = __ldcg(a.lv.G[2] + li);
        pf_q2[t] = __ldcg(a.lv.Q[2] + li);
      }
#pragma unroll
      for (int t = 0; t < QUP; ++t) {
        const int p = tid + t * NT, i = p / wc1, j = p % wc1;
        const int li = EMG_INB((rank * hc1 + i) * wc1 + j, wc1 * wc1, kBcLevel) ? (rank * hc1 + i) * wc1 + j : 0;
        pf_g1[t] = __ldcg(a.lv.G[1] + li);
        pf_q1[t] = __ldcg(a.lv.Q[1] + li);
      }
    }
    {  // restrict level 0 -> 1: z_1 = I_h^H (W_z z_k), R_1 = I_h^H (W_R R)
      constexpr int wc = M / 2, hc = wc / C, sc = wc + 1;
      constexpr int PC = hc * wc / NT;
      static_assert(hc * wc % NT == 0, "coarse slab must split evenly");
      const float* Wz = a.lv.Wz[0];
      const float2* WR = a.lv.WR[0];
      float2* __restrict__ const Z1w = Zl[1];
      float2* __restrict__ const R1w = Rl[1];
#pragma unroll
      for (int t = 0; t < PC; ++t) {
        const int p = tid + t * NT;
        const int i = p / wc, j = p % wc;
        float2 zs = czero(), rs = czero();
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const int lr = 2 * i + dy, r = row0 + lr, c = 2 * j;
          // the weights of the pixel pair (c, c + 1) in one load each (c is even)
          const float2 wz = __ldcg(reinterpret_cast<const float2*>(Wz + r * M + c));
          const float4 wr = __ldcg(reinterpret_cast<const float4*>(WR + r * M + c));
          zs = cadd(zs, cscale(zbuf[lr * M + c], wz.x));
          rs = cfma(make_float2(wr.x, wr.y), rowbuf[lr * SR + c], rs);
          zs = cadd(zs, cscale(zbuf[lr * M + c + 1], wz.y));
          rs = cfma(make_float2(wr.z, wr.w), rowbuf[lr * SR + c + 1], rs);
        }
        Z1w[i * sc + j] = cscale(zs, 0.25f);
        R1w[i * sc + j] = cscale(rs, 0.25f);
      }
    }
    __syncthreads();
    if (l3) {
      {  // restrict 1 -> 2 from the prefetched weights, and at once the coarsest step
         // on the same level-2 pixel (it needs nothing from other threads)
        constexpr int sf = wc1 + 1, sc = wc2 + 1;
        const float2* __restrict__ const Zf = Zl[1];
        const float2* __restrict__ const Rf = Rl[1];
        float2* __restrict__ const Zc = Zl[2];
#pragma unroll
        for (int t = 0; t < Q12; ++t) {
          const int p = tid + t * NT, i = p / wc2, j = p % wc2;
          float2 zs = czero(), rs = czero();
#pragma unroll
          for (int dy = 0; dy < 2; ++dy) {
            const int lr = 2 * i + dy, c = 2 * j;
            zs = cadd(zs, cscale(Zf[lr * sf + c], pf_wz1[t][dy].x));
            rs = cfma(make_float2(pf_wr1[t][dy].x, pf_wr1[t][dy].y), Rf[lr * sf + c], rs);
            zs = cadd(zs, cscale(Zf[lr * sf + c + 1], pf_wz1[t][dy].y));
            rs = cfma(make_float2(pf_wr1[t][dy].z, pf_wr1[t][dy].w), Rf[lr * sf + c + 1], rs);
          }
          const float2 z2 = cscale(zs, 0.25f), r2 = cscale(rs, 0.25f);
          // coarsest level 2: correction c = G (R - Q z), stored over z
          const float2 cc = cmul(pf_g2[t], cfnma(pf_q2[t], z2, r2));
          Zc[i * sc + j] = cc;
          if (halo) push_halo<C>(cl, rank, Zc, sc, hc2, i, j, cc);
        }
      }
      if (halo) cl.sync();  // the pushed halo rows of level 2 are in place
      __syncthreads();
      {  // back up to level 1
        constexpr int sl = wc1 + 1, sc = wc2 + 1;
        float2* __restrict__ const Zw = Zl[1];
        const float2* __restrict__ const Rw = Rl[1];
        const float2* __restrict__ const Zc = Zl[2];
#pragma unroll
        for (int t = 0; t < QUP; ++t) {
          const int p = tid + t * NT, i = p / wc1, j = p % wc1;
          const float2 pro = prolong_halo<float2>(Zc, sc, wc2, i, j, a.prolong);
          const float2 zp = cadd(Zw[i * sl + j], pro);
          const float2 cc = cfma(pf_g1[t], cfnma(pf_q1[t], zp, Rw[i * sl + j]), pro);
          Zw[i * sl + j] = cc;
          if (halo) push_halo<C>(cl, rank, Zw, sl, hc1, i, j, cc);
        }
      }
    } else {
    for (int l = 1; l + 1 < a.levels; ++l) {
      const int wf = M >> l, sf = wf + 1, hf = wf / C, wc = wf >> 1, hc = wc / C, sc = wc + 1;
      const float* Wz = a.lv.Wz[l];
      const float2* WR = a.lv.WR[l];
      const float2* __restrict__ const Zf = Zl[l];
      const float2* __restrict__ const Rf = Rl[l];
      float2* __restrict__ const Zc = Zl[l + 1];
      float2* __restrict__ const Rc = Rl[l + 1];
      for (int p = tid; p < hc * wc; p += NT) {
        const int i = p / wc, j = p % wc;
        float2 zs = czero(), rs = czero();
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const int lr = 2 * i + dy, r = rank * hf + lr, c = 2 * j + dx;
            const int wi = EMG_INB(r * wf + c, wf * wf, kBcLevel) ? r * wf + c : 0;
            zs = cadd(zs, cscale(Zf[lr * sf + c], __ldcg(Wz + wi)));
            rs = cadd(rs, cmul(__ldcg(WR + wi), Rf[lr * sf + c]));
          }
        Zc[i * sc + j] = cscale(zs, 0.25f);
        Rc[i * sc + j] = cscale(rs, 0.25f);
      }
      __syncthreads();
    }
    {  // coarsest level: correction c = G (R - Q z), stored over z
      const int l = a.levels - 1;
      const int wl = M >> l, hl = wl / C, sl = wl + 1;
      const float2* G = a.lv.G[l];
      const float2* Q = a.lv.Q[l];
      float2* __restrict__ const Zw = Zl[l];
      const float2* __restrict__ const Rw = Rl[l];
      for (int p = tid; p < hl * wl; p += NT) {
        const int i = p / wl, j = p % wl, gi = rank * hl + i;
        const int li = EMG_INB(gi * wl + j, wl * wl, kBcLevel) ? gi * wl + j : 0;
        const float2 z = Zw[i * sl + j];
        Zw[i * sl + j] = cmul(__ldcg(G + li), csub(Rw[i * sl + j], cmul(__ldcg(Q + li), z)));
      }
    }
    // back up: c_l = I_H^h c_{l+1} + G_l (R_l - Q_l (z_l + I_H^h c_{l+1}))
    for (int l = a.levels - 2; l >= 1; --l) {
      if (halo) {
        cl.sync();
        fill_halo(l + 1);
      }
      __syncthreads();
      const int wl = M >> l, hl = wl / C, sl = wl + 1, wc = wl >> 1, sc = wc + 1;
      const float2* G = a.lv.G[l];
      const float2* Q = a.lv.Q[l];
      float2* __restrict__ const Zw = Zl[l];
      const float2* __restrict__ const Rw = Rl[l];
      const float2* __restrict__ const Zc = Zl[l + 1];
#pragma unroll 4
      for (int p = tid; p < hl * wl; p += NT) {
        const int i = p / wl, j = p % wl, gi = rank * hl + i;
        const int li = EMG_INB(gi * wl + j, wl * wl, kBcLevel) ? gi * wl + j : 0;
        const float2 pro = prolong_halo<float2>(Zc, sc, wc, i, j, a.prolong);
        const float2 zp = cadd(Zw[i * sl + j], pro);
        Zw[i * sl + j] = cadd(pro, cmul(__ldcg(G + li), csub(Rw[i * sl + j], cmul(__ldcg(Q + li), zp))));
      }
    }
    }  // generic levels
    if (halo) {
      cl.sync();
      if (!l3) fill_halo(1);  // three levels: the halo rows were pushed
    }
    __syncthreads();
  }

  // a5 (finest level) + a6 + a7; the level-0 gain G_0 = conj(Q)/(u_0 + |Q|^2)
  // comes from the probe prep of this minibatch
  const float inv_mu = mu > 0.f ? 1.f / mu : 0.f;
  float2* zt = a.zt + (size_t)kb * M * M;
  float2* qt = a.qt + (size_t)kb * M * M;
  const float2* Z1 = Zl[1];
  const float2* G0 = a.lv.G[0];
  float acc_after = 0.f;
  // Groups of UG pixels: the probe and gain loads of a group are issued
  // together, and the loop body stays small enough for the instruction cache.
  constexpr int UG0 = EMG_UPDATE_GROUP < PER ? EMG_UPDATE_GROUP : PER;
  constexpr int UG = PER % UG0 == 0 ? UG0 : 1;
  // The common case (multigrid, joint step, ordered combine, no verify) runs a
  // loop without the mode branches over pairs of adjacent pixels, with 16-byte
  // probe and gain loads and patch stores, and the prolongation's loads shared
  // by the pair; the arithmetic per pixel is the same as in the general loop.
  constexpr int UGP = UG >= 2 && PER % 2 == 0 ? UG / 2 : 0;
  const bool pairs = UGP > 0 && a.levels > 1 && a.joint && !a.s_num && !a.verify && slot_ok &&
                     ((reinterpret_cast<uintptr_t>(a.probe) | reinterpret_cast<uintptr_t>(G0) |
                       reinterpret_cast<uintptr_t>(zt) | reinterpret_cast<uintptr_t>(qt)) & 15) == 0;
  if constexpr (UGP > 0) {
    if (pairs) {
      constexpr int PP = PER / 2;
      constexpr int SL1 = M / 2 + 1, WC1 = M / 2;
#pragma unroll 1
      for (int t0 = 0; t0 < PP; t0 += UGP) {
        float4 qv[UGP], gv[UGP];
#pragma unroll
        for (int u = 0; u < UGP; ++u) {
          const int off = row0 * M + 2 * (tid + (t0 + u) * NT);
          qv[u] = __ldg(reinterpret_cast<const float4*>(a.probe + off));
          gv[u] = __ldcg(reinterpret_cast<const float4*>(G0 + off));
        }
#pragma unroll
        for (int u = 0; u < UGP; ++u) {
          const int p0 = 2 * (tid + (t0 + u) * NT);
          const int lr = p0 / M, c0 = p0 % M, r = row0 + lr;
          const float4 zk2 = *reinterpret_cast<const float4*>(zbuf + p0);
          // coarse-level correction at both pixels: the rows and the centre column are shared
          float2 pro[2];
          {
            const int i = lr >> 1, j = c0 >> 1;
            const float2* y0 = Z1 + i * SL1;
            const float2 v = y0[j];
            if (a.prolong == 0) {
              pro[0] = pro[1] = v;
            } else {
              const float2* y1 = Z1 + ((lr & 1) ? i + 1 : i - 1) * SL1;
              const int jm = max(j - 1, 0), jp = min(j + 1, WC1 - 1);
              pro[0] = lerp4<float2>(v, y1[j], y0[jm], y1[jm]);
              pro[1] = lerp4<float2>(v, y1[j], y0[jp], y1[jp]);
            }
          }
          float2 zo[2], qo[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float2 zk = h ? make_float2(zk2.z, zk2.w) : make_float2(zk2.x, zk2.y);
            const float2 q = h ? make_float2(qv[u].z, qv[u].w) : make_float2(qv[u].x, qv[u].y);
            const float2 g0 = h ? make_float2(gv[u].z, gv[u].w) : make_float2(gv[u].x, gv[u].y);
            update_pixel<true, true>(zk, q, g0, rowbuf[lr * SR + c0 + h], pro[h], inv_mu, zo[h], qo[h]);
          }
          *reinterpret_cast<float4*>(zt + r * M + c0) = make_float4(zo[0].x, zo[0].y, zo[1].x, zo[1].y);
          *reinterpret_cast<float4*>(qt + r * M + c0) = make_float4(qo[0].x, qo[0].y, qo[1].x, qo[1].y);
        }
      }
    }
  }
#pragma unroll 1
  for (int t0 = 0; t0 < (pairs ? 0 : PER); t0 += UG) {
  float2 qv[UG], gv[UG];
#pragma unroll
  for (int u = 0; u < UG; ++u) {
    qv[u] = __ldg(a.probe + row0 * M + tid + (t0 + u) * NT);
    gv[u] = __ldcg(G0 + row0 * M + tid + (t0 + u) * NT);
  }
#pragma unroll
  for (int u = 0; u < UG; ++u) {
    const int t = t0 + u;
    const int p = tid + t * NT;
    const int lr = p / M, c = p % M, r = row0 + lr;
    const float2 zk = zbuf[p];
    const float2 q = qv[u];
    const float2 R = rowbuf[lr * SR + c];
    const float2 pro = a.levels == 1 ? czero() : prolong_halo<float2>(Z1, M / 2 + 1, M / 2, lr, c, a.prolong);
    float2 zn, qn;
    if (a.levels == 1) {
      if (a.joint)
        update_pixel<false, true>(zk, q, gv[u], R, pro, inv_mu, zn, qn);
      else
        update_pixel<false, false>(zk, q, gv[u], R, pro, inv_mu, zn, qn);
    } else {
      if (a.joint)
        update_pixel<true, true>(zk, q, gv[u], R, pro, inv_mu, zn, qn);
      else
        update_pixel<true, false>(zk, q, gv[u], R, pro, inv_mu, zn, qn);
    }
    if (a.s_num)
      scatter_atomic(a.s_num, a.s_den, a.combine, a.n_rows, a.n_cols, o_r + r, o_c + c, zn, zk, fmaf(a.w_eps, MQ, cabs2(q)));
    else if (slot_ok)
      zt[r * M + c] = zn;
    if (slot_ok) qt[r * M + c] = qn;
    if (a.verify) acc_after += cabs2(csub(cmul(qn, zn), R));
  }
  }
  if (a.verify) {
    const double part = 0.5 * block_sum_f<NT>(acc_after, redf, redd);
    if (tid == 0) cluster_publish<C>(cl, rank, xd2, part);
  }
  // With halo rows read from the neighbours (bilinear prolongation, other
  // than three levels) a neighbour may still read my coarse rows: no CTA leaves
  // before all arrive.  The verify mode also publishes xd2, which needs the
  // release / acquire pair.  Otherwise no CTA touches another's shared memory
  // after the last cluster barrier, and each may leave when done.
  if (a.verify) {
    cl.sync();
  } else if (halo && !l3 && a.levels > 1) {
    cluster_arrive_relaxed();
    cluster_wait();
  }
  if (rank == 0 && tid == 0) {
    double phi = 0.0, after = 0.0;
#pragma unroll
    for (int d = 0; d < C; ++d) {
      if constexpr (!RIN) phi += xd[d];
      after += xd2[d];
    }
    if constexpr (RIN)
      for (int t = 0; t < a.r_tiles; ++t) phi += a.r_partial[(size_t)kb * a.r_tiles + t];
    a.mu[kb] = mu;
    a.phi[kb] = phi * (0.5 / (double)(M * M));
    if (a.verify) a.phi_after[kb] = after;
  }
}

// ---------------------------------------------------------------------------
// Forward transform of one tile per cluster (any m): modes
//   0 misfit partial (1/2 m^2) sum (|F psi| - a_k)^2 per position,
//   1 intensity |F psi|^2 in natural order,
//   2 F x of a natural-order tile.
template <int M, int C, int MODE>
__global__ void __launch_bounds__(CTile<M, C>::NT, 1) k_fwdc(const FwdArgs a) {
  using TL = CTile<M, C>;
  constexpr int NT = TL::NT, H = TL::H, SR = TL::SR, SC = TL::SC, N1 = TL::N1, N2 = TL::N2;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ float2 sm[];
  float2* rowbuf = sm;
  float2* colbuf = sm + H * SR;
  __shared__ double xd[C];
  __shared__ double redd[2];
  __shared__ float redf[NT / 32];
  const int tid = threadIdx.x;
  const int t = blockIdx.x / C;
  const int row0 = rank * H;
  cluster_arrive_relaxed();
  if (MODE == 2) {
    const float2* x = a.in + (size_t)t * M * M;
    for (int p = tid; p < H * M; p += NT) rowbuf[(p / M) * SR + p % M] = x[row0 * M + p];
  } else {
    const int o_r = a.pos[2 * t], o_c = a.pos[2 * t + 1];
    for (int p = tid; p < H * M; p += NT) {
      const int lr = p / M, c = p % M, r = row0 + lr;
      rowbuf[lr * SR + c] = cmul(a.probe[r * M + c], gather_obj(a.object, a.n_rows, a.n_cols, o_r + r, o_c + c));
    }
  }
  __syncthreads();
  gpass_a_fwd<M, H, SR, 1, NT>(rowbuf, tid);
  __syncthreads();
  gpass_b<M, H, SR, 1, NT, false>(rowbuf, tid);
  __syncthreads();
  cl.barrier_wait();
  cluster_rows_to_cols<M, C>(cl, rank, rowbuf, colbuf, tid);
  cl.sync();
  gpass_a_fwd<M, H, 1, SC, NT>(colbuf, tid);
  __syncthreads();
  gpass_b<M, H, 1, SC, NT, false>(colbuf, tid);
  __syncthreads();
  float acc = 0.f;
  for (int p = tid; p < M * H; p += NT) {
    const int er = p / H, lc = p % H, ec = rank * H + lc;
    const float2 v = colbuf[er * SC + lc];
    const size_t nat = (size_t)storage_to_freq<M>(er) * M + storage_to_freq<M>(ec);
    if (MODE == 0) {
      const float dm = sqrtf(cabs2(v)) - a.amp[(size_t)t * M * M + er * M + ec];
      acc = fmaf(dm, dm, acc);
    } else if (MODE == 1) {
      a.out_intensity[(size_t)t * M * M + nat] = cabs2(v);
    } else {
      a.out[(size_t)t * M * M + nat] = v;
    }
  }
  if (MODE == 0) {
    const double part = block_sum_f<NT>(acc, redf, redd);
    if (tid == 0) cluster_publish<C>(cl, rank, xd, part);
    cl.sync();
    if (rank == 0 && tid == 0) {
      double tot = 0.0;
#pragma unroll
      for (int d = 0; d < C; ++d) tot += xd[d];
      a.partial[t] = tot * (0.5 / (double)(M * M));
    }
  }
}

// Inverse 2-D DFT (with 1/m^2) of natural-order tiles, one tile per cluster.
template <int M, int C>
__global__ void __launch_bounds__(CTile<M, C>::NT, 1) k_ifftc(const FwdArgs a) {
  using TL = CTile<M, C>;
  constexpr int NT = TL::NT, H = TL::H, SR = TL::SR, SC = TL::SC;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ float2 sm[];
  float2* rowbuf = sm;
  float2* colbuf = sm + H * SR;
  const int tid = threadIdx.x;
  const int t = blockIdx.x / C;
  const float2* x = a.in + (size_t)t * M * M;
  const float sc = 1.f / (float)(M * M);
  cluster_arrive_relaxed();
  for (int p = tid; p < M * H; p += NT) {
    const int er = p / H, lc = p % H, ec = rank * H + lc;
    colbuf[er * SC + lc] = cscale(x[(size_t)storage_to_freq<M>(er) * M + storage_to_freq<M>(ec)], sc);
  }
  __syncthreads();
  gpass_b<M, H, 1, SC, NT, true>(colbuf, tid);
  __syncthreads();
  gpass_a_inv<M, H, 1, SC, NT>(colbuf, tid);
  __syncthreads();
  cl.barrier_wait();
  cluster_cols_to_rows<M, C>(cl, rank, colbuf, rowbuf, tid);
  cl.sync();
  gpass_b<M, H, SR, 1, NT, true>(rowbuf, tid);
  __syncthreads();
  gpass_a_inv<M, H, SR, 1, NT>(rowbuf, tid);
  __syncthreads();
  float2* y = a.out + (size_t)t * M * M + rank * H * M;
  for (int p = tid; p < H * M; p += NT) y[p] = rowbuf[(p / M) * SR + p % M];
}

// ---------------------------------------------------------------------------
// Wirtinger gradient of the exit-wave misfit per position (Sec. 2.1), with the
// revised exit wave recomputed: forward FFT, modulus replacement, inverse FFT,
// then gz = conj(Q) (psi - R), gq = conj(z_k) (psi - R) on the patch.
template <int M, int C>
__global__ void __launch_bounds__(CTile<M, C>::NT, 1) k_gradc(const GradArgs a) {
  using TL = CTile<M, C>;
  constexpr int NT = TL::NT, H = TL::H, SR = TL::SR, SC = TL::SC, N1 = TL::N1, N2 = TL::N2, SLOTS = TL::SLOTS;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ float2 sm[];
  float2* rowbuf = sm;
  float2* colbuf = sm + H * SR;
  float2* zbuf = colbuf + M * SC;
  __shared__ double xd[C];
  __shared__ float redf[NT / 32];
  const int tid = threadIdx.x;
  const int kb = blockIdx.x / C;
  const int k = a.first + kb;
  const int o_r = a.pos[2 * k], o_c = a.pos[2 * k + 1];
  const int row0 = rank * H;
  constexpr int PER = TL::PER;
  // amplitudes of my spectral slots: issued now, consumed after the row passes
  float am_reg[SLOTS][N1];
  {
    const float* amp = a.amp + (size_t)k * M * M + rank * H;
#pragma unroll
    for (int t = 0; t < SLOTS; ++t) {
      const int s = tid + t * NT, k2 = s / H, lc = s % H;
#pragma unroll
      for (int i = 0; i < N1; ++i) am_reg[t][i] = __ldg(amp + (i + N1 * k2) * M + lc);
    }
  }
  cluster_arrive_relaxed();
  // gather: the loads of 8 pixels of a thread in flight together
#pragma unroll 8
  for (int t = 0; t < PER; ++t) {
    const int p = tid + t * NT;
    const int lr = p / M, c = p % M, r = row0 + lr;
    const float2 zk = gather_obj(a.object, a.n_rows, a.n_cols, o_r + r, o_c + c);
    zbuf[p] = zk;
    rowbuf[lr * SR + c] = cmul(a.probe[r * M + c], zk);
  }
  __syncthreads();
  gpass_a_fwd<M, H, SR, 1, NT>(rowbuf, tid);
  __syncthreads();
  gpass_b<M, H, SR, 1, NT, false>(rowbuf, tid);
  __syncthreads();
  cl.barrier_wait();
  cluster_rows_to_cols<M, C>(cl, rank, rowbuf, colbuf, tid);
  cl.sync();
  gpass_a_fwd<M, H, 1, SC, NT>(colbuf, tid);
  __syncthreads();
  const float inv_m2 = 1.f / (float)(M * M);
  float acc = 0.f;
#pragma unroll
  for (int t = 0; t < SLOTS; ++t) {
    const int s = tid + t * NT, k2 = s / H, lc = s % H;
    float2 v[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = colbuf[(i + N1 * k2) * SC + lc];
    Dft<N1, false>::run(v);
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      const float am = am_reg[t][i];
      const float p2 = cabs2(v[i]);
      if (p2 > 0.f) {
        const float inv = rsqrtf(p2);
        const float dm = fmaf(p2, inv, -am);
        acc = fmaf(dm, dm, acc);
        v[i] = cscale(v[i], am * inv * inv_m2);
      } else {
        acc = fmaf(am, am, acc);
        v[i] = make_float2(am * inv_m2, 0.f);
      }
    }
    Dft<N1, true>::run(v);
#pragma unroll
    for (int i = 0; i < N1; ++i) colbuf[(i + N1 * k2) * SC + lc] = v[i];
  }
  __syncthreads();
  gpass_a_inv<M, H, 1, SC, NT>(colbuf, tid);
  // per-warp misfit partials; the barrier also orders the pass before the transpose
  warp_partial_sum(acc, redf);
  __syncthreads();
  cluster_cols_to_rows<M, C>(cl, rank, colbuf, rowbuf, tid);
  if (tid == 0) cluster_publish<C>(cl, rank, xd, partials_sum<NT>(redf));
  cl.sync();
  gpass_b<M, H, SR, 1, NT, true>(rowbuf, tid);
  __syncthreads();
  gpass_a_inv<M, H, SR, 1, NT>(rowbuf, tid);
  __syncthreads();
  float2* gz = a.gz + (size_t)kb * M * M;
  float2* gq = a.gq + (size_t)kb * M * M;
  // patch gradients; the probe loads of 8 pixels of a thread are issued together
  constexpr int UG = PER < 8 ? PER : 8;
#pragma unroll 1
  for (int t0 = 0; t0 < PER; t0 += UG) {
    float2 qv[UG];
#pragma unroll
    for (int u = 0; u < UG; ++u) {
      const int p = tid + (t0 + u) * NT;
      qv[u] = __ldg(a.probe + (row0 + p / M) * M + p % M);
    }
#pragma unroll
    for (int u = 0; u < UG; ++u) {
      const int p = tid + (t0 + u) * NT;
      const int lr = p / M, c = p % M, r = row0 + lr;
      const float2 zk = zbuf[p];
      const float2 q = qv[u];
      const float2 e = csub(cmul(q, zk), rowbuf[lr * SR + c]);
      gz[r * M + c] = cconjmul(q, e);
      gq[r * M + c] = cconjmul(zk, e);
    }
  }
  if (rank == 0 && tid == 0) {
    double tot = 0.0;
#pragma unroll
    for (int d = 0; d < C; ++d) tot += xd[d];
    a.phi[kb] = tot * (0.5 / (double)(M * M));
  }
}

// Object gradient sum_k P_k^T gz_k over 16 x 16 tiles and probe gradient
// sum_k gq_k, each in position order (deterministic); optionally added to the
// existing values (later chunks of positions).
__global__ void __launch_bounds__(kApplyThreads) k_grad_reduce(const GradReduceArgs a) {
  extern __shared__ int glist[];
  __shared__ int warp_count[kApplyThreads / 32];
  __shared__ int total;
  __shared__ float2 part_s[kApplyProbeGroups][32];
  const int tid = threadIdx.x;
  const int n_tiles = a.tiles_x * a.tiles_y;
  const int m = a.m;
  const size_t mm = (size_t)m * m;
  if ((int)blockIdx.x < n_tiles) {
    if (!a.grad_object) return;
    const int ty = blockIdx.x / a.tiles_x, tx = blockIdx.x % a.tiles_x;
    const int r0 = ty * kApplyTile, c0 = tx * kApplyTile;
    if (tid == 0) total = 0;
    __syncthreads();
    for (int base = 0; base < a.b; base += kApplyThreads) {
      const int kb = base + tid;
      int pr = 0, pc = 0;
      bool hit = false;
      if (kb < a.b) {
        pr = a.pos[2 * (a.first + kb)];
        pc = a.pos[2 * (a.first + kb) + 1];
        hit = pr < r0 + kApplyTile && pr + m > r0 && pc < c0 + kApplyTile && pc + m > c0;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, hit);
      const int lane = tid & 31, warp = tid >> 5;
      if (lane == 0) warp_count[warp] = __popc(mask);
      __syncthreads();
      int off = total;
      for (int w = 0; w < warp; ++w) off += warp_count[w];
      if (hit) {
        const int slot = off + __popc(mask & ((1u << lane) - 1u));
        glist[3 * slot] = kb;
        glist[3 * slot + 1] = pr;
        glist[3 * slot + 2] = pc;
      }
      __syncthreads();
      if (tid == 0) {
        int t = total;
        for (int w = 0; w < kApplyThreads / 32; ++w) t += warp_count[w];
        total = t;
      }
      __syncthreads();
    }
    const int cnt = total;
    const int row = r0 + tid / kApplyTile, col = c0 + tid % kApplyTile;
    if (row >= a.n_rows || col >= a.n_cols) return;
    float2 g = czero();
    for (int t = 0; t < cnt; ++t) {
      const int lr = row - glist[3 * t + 1], lc = col - glist[3 * t + 2];
      if ((unsigned)lr < (unsigned)m && (unsigned)lc < (unsigned)m)
        g = cadd(g, a.gz[(size_t)glist[3 * t] * mm + lr * m + lc]);
    }
    const size_t gi = (size_t)row * a.n_cols + col;
    a.grad_object[gi] = a.accumulate ? cadd(a.grad_object[gi], g) : g;
  } else {
    if (!a.grad_probe) return;
    const int lane = tid & 31, g = tid >> 5;
    const int p = (blockIdx.x - n_tiles) * 32 + lane;
    float2 sum = czero();
    if (p < (int)mm)
      for (int kb = g; kb < a.b; kb += kApplyProbeGroups) sum = cadd(sum, a.gq[(size_t)kb * mm + p]);
    part_s[g][lane] = sum;
    __syncthreads();
    if (g != 0 || p >= (int)mm) return;
    float2 tot = part_s[0][lane];
#pragma unroll
    for (int i = 1; i < kApplyProbeGroups; ++i) tot = cadd(tot, part_s[i][lane]);
    a.grad_probe[p] = a.accumulate ? cadd(a.grad_probe[p], tot) : tot;
  }
}

// ---------------------------------------------------------------------------
// a8 + a9: deterministic combine.  Blocks [0, tiles) own object tiles of
// kApplyTile x kApplyTileW pixels (kApplyPx pixels per thread, kApplyTile
// apart in the row); the remaining blocks own kApplyProbePx probe pixels each
// (kApplyProbePx / 32 per lane), with 8 thread groups summing disjoint
// position subsets that are then added in a fixed order.  Each thread issues
// the loads of all its pixels together, and the grid of the bench-sized
// object and probe is resident at once after the step.  The new probe's
// max|Q|^2 goes to a.mq_next for the next prep.
#ifndef EMG_APPLY_MIN_BLOCKS
#define EMG_APPLY_MIN_BLOCKS 4
#endif
#ifndef EMG_APPLY_CHUNK
#define EMG_APPLY_CHUNK 4
#endif
constexpr int kApplyChunk = EMG_APPLY_CHUNK;  // covering patches whose loads a thread issues together
__global__ void __launch_bounds__(kApplyThreads, EMG_APPLY_MIN_BLOCKS) k_apply(const ApplyArgs a) {
  constexpr int PX = kApplyPx, PP = kApplyProbePx / 32;
  extern __shared__ int list[];  // [b][3] = (kb, row, col) of patches overlapping the tile
  __shared__ int warp_count[kApplyThreads / 32];
  __shared__ int total;
  __shared__ float2 part_s[kApplyProbeGroups][kApplyProbePx];
  __shared__ int part_n[kApplyProbeGroups][kApplyProbePx];
  const int tid = threadIdx.x;
  const int n_tiles = a.tiles_x * a.tiles_y;
  const int m = a.m;
  const size_t mm = (size_t)m * m;
  pdl_trigger();
  if ((int)blockIdx.x < n_tiles && a.s_num) {
    // atomic scatter: the step kernel has accumulated this tile's sums; finalise and reset them
    const int ty = blockIdx.x / a.tiles_x, tx = blockIdx.x % a.tiles_x;
    const int row = ty * kApplyTile + tid / kApplyTile;
    if (row >= a.n_rows) return;
    pdl_wait();
#pragma unroll
    for (int h = 0; h < PX; ++h) {
      const int col = tx * kApplyTileW + tid % kApplyTile + h * kApplyTile;
      if (col >= a.n_cols) continue;
      const size_t gi = (size_t)row * a.n_cols + col;
      if (a.combine == 0) {
        const float den = a.s_den[gi];
        if (den > 0.f) {
          a.object[gi] = cscale(a.s_num[gi], 1.f / den);
          a.s_num[gi] = czero();
          a.s_den[gi] = 0.f;
        }
      } else {
        const float2 dz = a.s_num[gi];
        if (dz.x != 0.f || dz.y != 0.f) {
          a.object[gi] = cadd(a.object[gi], dz);
          a.s_num[gi] = czero();
        }
      }
    }
  } else if ((int)blockIdx.x < n_tiles) {
    const int ty = blockIdx.x / a.tiles_x, tx = blockIdx.x % a.tiles_x;
    const int r0 = ty * kApplyTile, c0 = tx * kApplyTileW;
    if (tid == 0) total = 0;
    __syncthreads();
    // ordered compaction of the minibatch patches that overlap this tile
    for (int base = 0; base < a.b; base += kApplyThreads) {
      const int kb = base + tid;
      int pr = 0, pc = 0;
      bool hit = false;
      if (kb < a.b) {
        int k = a.order[kb];
        if (!EMG_INB(k, a.n_pos, kBcApplyOrder)) k = 0;
        pr = a.pos[2 * k];
        pc = a.pos[2 * k + 1];
        hit = pr < r0 + kApplyTile && pr + m > r0 && pc < c0 + kApplyTileW && pc + m > c0;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, hit);
      const int lane = tid & 31, warp = tid >> 5;
      if (lane == 0) warp_count[warp] = __popc(mask);
      __syncthreads();
      int off = total;
      for (int w = 0; w < warp; ++w) off += warp_count[w];
      if (hit) {
        const int slot = off + __popc(mask & ((1u << lane) - 1u));
        list[3 * slot] = kb;
        list[3 * slot + 1] = pr;
        list[3 * slot + 2] = pc;
      }
      __syncthreads();
      if (tid == 0) {
        int t = total;
        for (int w = 0; w < kApplyThreads / 32; ++w) t += warp_count[w];
        total = t;
      }
      __syncthreads();
    }
    const int cnt = total;
    const int row = r0 + tid / kApplyTile, col0 = c0 + tid % kApplyTile;
    if (cnt == 0 || row >= a.n_rows || col0 >= a.n_cols) return;
    pdl_wait();  // patches z~_k and weights come from the step and prep kernels
    float2 num[PX];
    float den[PX];
    bool covered[PX];
#pragma unroll
    for (int h = 0; h < PX; ++h) {
      num[h] = czero();
      den[h] = 0.f;
      covered[h] = false;
    }
    // patches in minibatch order; loads of kApplyChunk patches at all pixels are issued together
    for (int t0 = 0; t0 < cnt; t0 += kApplyChunk) {
      float2 v[PX][kApplyChunk];
      float w[PX][kApplyChunk];
      bool in[PX][kApplyChunk];
#pragma unroll
      for (int u = 0; u < kApplyChunk; ++u) {
        const int t = t0 + u;
#pragma unroll
        for (int h = 0; h < PX; ++h) in[h][u] = false;
        if (t < cnt) {
          const int kb = list[3 * t], lr = row - list[3 * t + 1], lc = col0 - list[3 * t + 2];
          const bool ok = (unsigned)lr < (unsigned)m && EMG_INB(kb, a.b, kBcApplyPatch);
          // all pixels from one base address: pixel h is h kApplyTile columns on
          const float2* zrow = a.zt + (size_t)kb * mm + lr * m + lc;
          const float* wrow = a.wq + lr * m + lc;
#pragma unroll
          for (int h = 0; h < PX; ++h) {
            in[h][u] = ok && (unsigned)(lc + h * kApplyTile) < (unsigned)m && col0 + h * kApplyTile < a.n_cols;
            if (in[h][u]) {
              v[h][u] = zrow[h * kApplyTile];
              w[h][u] = a.combine == 0 ? wrow[h * kApplyTile] : 1.f;
            }
          }
        }
      }
#pragma unroll
      for (int h = 0; h < PX; ++h)
#pragma unroll
        for (int u = 0; u < kApplyChunk; ++u) {
          if (in[h][u]) {
            covered[h] = true;
            if (a.combine == 0) {
              num[h] = make_float2(fmaf(w[h][u], v[h][u].x, num[h].x), fmaf(w[h][u], v[h][u].y, num[h].y));
            } else {
              num[h] = cadd(num[h], v[h][u]);
            }
            den[h] += w[h][u];
          }
        }
    }
#pragma unroll
    for (int h = 0; h < PX; ++h) {
      if (!covered[h]) continue;
      const size_t gi = (size_t)row * a.n_cols + col0 + h * kApplyTile;
      if (!EMG_INB(gi, (size_t)a.n_rows * a.n_cols, kBcApplyObject)) continue;
      if (a.combine == 0) {
        a.object[gi] = safe_cdiv(num[h], den[h]);
      } else {
        const float2 z = a.object[gi];
        a.object[gi] = cadd(z, csub(num[h], cscale(z, den[h])));
      }
    }
  } else {
    pdl_wait();  // probes Q~_k come from the step kernel
    const int lane = tid & 31, g = tid >> 5;
    const int p0 = (blockIdx.x - n_tiles) * kApplyProbePx + lane;
    float2 s[PP];
#pragma unroll
    for (int h = 0; h < PP; ++h) s[h] = czero();
    int cnt = 0;
    if (p0 < (int)mm) {
      for (int kb0 = g; kb0 < a.b; kb0 += 4 * kApplyProbeGroups) {
        float2 v[PP][4];
        float mu[4];
        // mu_k and Q~_k are loaded together; slots with mu_k = 0 are skipped when summing
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int kb = kb0 + u * kApplyProbeGroups;
          mu[u] = 0.f;
          if (kb < a.b) {
            mu[u] = a.mu[kb];
            const float2* qrow = a.qt + (size_t)kb * mm + p0;
#pragma unroll
            for (int h = 0; h < PP; ++h)
              if (p0 + 32 * h < (int)mm) v[h][u] = qrow[32 * h];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (mu[u] > 0.f) {
#pragma unroll
            for (int h = 0; h < PP; ++h)
              if (p0 + 32 * h < (int)mm) s[h] = cadd(s[h], v[h][u]);
            ++cnt;
          }
        }
      }
    }
#pragma unroll
    for (int h = 0; h < PP; ++h) {
      part_s[g][lane + 32 * h] = s[h];
      part_n[g][lane + 32 * h] = cnt;
    }
    __syncthreads();
    if (tid >= kApplyProbePx) return;
    const int p = (blockIdx.x - n_tiles) * kApplyProbePx + tid;
    float a2 = 0.f;
    if (p < (int)mm) {
      float2 tot = part_s[0][tid];
      int n = part_n[0][tid];
#pragma unroll
      for (int i = 1; i < kApplyProbeGroups; ++i) {
        tot = cadd(tot, part_s[i][tid]);
        n += part_n[i][tid];
      }
      float2 q = a.probe[p];
      if (n > 0) {
        q = (a.combine == 0) ? cscale(tot, 1.f / (float)n) : cadd(q, csub(tot, cscale(q, (float)n)));
        a.probe[p] = q;
      }
      a2 = cabs2(q);
    }
    if (a.mq_next) warp_atomic_max(a.mq_next, a2);
  }
}

// ---------------------------------------------------------------------------
// Phi_k = (1/2 M^2) sum (|F psi| - a_k)^2 per position (Parseval form of Eq. exit_misfit).
template <int M>
__global__ void __launch_bounds__(StepThreads<M>::value)
    k_misfit(const float2* __restrict__ object, const float2* __restrict__ probe,
             const int32_t* __restrict__ pos, const float* __restrict__ amp, int n_rows, int n_cols,
             double* __restrict__ partial) {
  constexpr int NT = StepThreads<M>::value;
  constexpr int S = M + 1;
  constexpr int N1 = FftPlan<M>::N1, N2 = FftPlan<M>::N2;
  extern __shared__ float2 sm[];
  __shared__ double redd[NT / 32];
  const int tid = threadIdx.x;
  const int k = blockIdx.x;
  const int o_r = pos[2 * k], o_c = pos[2 * k + 1];
  float2* buf = sm;
  for (int p = tid; p < M * M; p += NT) {
    const int r = p / M, c = p % M;
    buf[r * S + c] = cmul(probe[p], gather_obj(object, n_rows, n_cols, o_r + r, o_c + c));
  }
  __syncthreads();
  fft2_fwd_until_col_b<M, NT>(buf, tid);
  const float* ak = amp + (size_t)k * M * M;
  float acc = 0.f;
  for (int s = tid; s < M * N2; s += NT) {
    const int k2 = s / M, c = s % M;
    float2 v[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = buf[(i + N1 * k2) * S + c];
    Dft<N1, false>::run(v);
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      const float dm = sqrtf(cabs2(v[i])) - ak[(i + N1 * k2) * M + c];
      acc = fmaf(dm, dm, acc);
    }
  }
  const double tot = block_sum<NT>((double)acc, redd);
  if (tid == 0) partial[k] = tot * (0.5 / (double)(M * M));
}

// Deterministic single-block sum: out = scale * sum x[0..n).
constexpr int kSumThreads = 1024;
__global__ void __launch_bounds__(kSumThreads) k_sum(const double* __restrict__ x, int n,
                                                     double scale, double* __restrict__ out) {
  __shared__ double redd[kSumThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kSumThreads) s += x[i];
  s = block_sum<kSumThreads>(s, redd);
  if (threadIdx.x == 0) *out = s * scale;
}

// ---------------------------------------------------------------------------
// Data model of Sec. 2.1: d_k = |F(Q . P_k z)|^2 in natural order.
template <int M>
__global__ void __launch_bounds__(StepThreads<M>::value)
    k_simulate(const float2* __restrict__ object, const float2* __restrict__ probe,
               const int32_t* __restrict__ pos, int n_rows, int n_cols, float* __restrict__ out) {
  constexpr int NT = StepThreads<M>::value;
  constexpr int S = M + 1;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int k = blockIdx.x;
  const int o_r = pos[2 * k], o_c = pos[2 * k + 1];
  float2* buf = sm;
  for (int p = tid; p < M * M; p += NT) {
    const int r = p / M, c = p % M;
    buf[r * S + c] = cmul(probe[p], gather_obj(object, n_rows, n_cols, o_r + r, o_c + c));
  }
  __syncthreads();
  fft2_fwd_until_col_b<M, NT>(buf, tid);
  pass_b<M, true, NT, false>(buf, tid);
  __syncthreads();
  float* dk = out + (size_t)k * M * M;
  for (int p = tid; p < M * M; p += NT) {
    const int er = p / M, ec = p % M;
    dk[storage_to_freq<M>(er) * M + storage_to_freq<M>(ec)] = cabs2(buf[er * S + ec]);
  }
}

// Batched 2-D DFT of natural-order tiles.
template <int M>
__global__ void __launch_bounds__(StepThreads<M>::value)
    k_fft2(const float2* in, float2* out, int inverse) {
  constexpr int NT = StepThreads<M>::value;
  constexpr int S = M + 1;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const float2* x = in + (size_t)blockIdx.x * M * M;
  float2* y = out + (size_t)blockIdx.x * M * M;
  float2* buf = sm;
  if (!inverse) {
    for (int p = tid; p < M * M; p += NT) buf[(p / M) * S + p % M] = x[p];
    __syncthreads();
    fft2_fwd_until_col_b<M, NT>(buf, tid);
    pass_b<M, true, NT, false>(buf, tid);
    __syncthreads();
    for (int p = tid; p < M * M; p += NT) {
      const int er = p / M, ec = p % M;
      y[storage_to_freq<M>(er) * M + storage_to_freq<M>(ec)] = buf[er * S + ec];
    }
  } else {
    const float s = 1.f / (float)(M * M);
    for (int p = tid; p < M * M; p += NT) {
      const int er = p / M, ec = p % M;
      buf[er * S + ec] = cscale(x[storage_to_freq<M>(er) * M + storage_to_freq<M>(ec)], s);
    }
    __syncthreads();
    pass_b<M, true, NT, true>(buf, tid);
    __syncthreads();
    fft2_inv_after_col_b<M, NT>(buf, tid);
    for (int p = tid; p < M * M; p += NT) y[p] = buf[(p / M) * S + p % M];
  }
}

// dp_avg probe scaling (Sec. 4.1): partial sums of a^2 = max(d, 0).
constexpr int kNormThreads = 256;
__global__ void __launch_bounds__(kNormThreads) k_sum_sq(const float* __restrict__ amp, size_t n,
                                                         double* __restrict__ partial) {
  __shared__ double redd[kNormThreads / 32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)kNormThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kNormThreads) {
    const float v = amp[i];
    s += (double)(v * v);
  }
  s = block_sum<kNormThreads>(s, redd);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kSumThreads) k_scale_probe(const double* __restrict__ partial,
                                                             int n_partial, int m, int n_pos,
                                                             float2* __restrict__ probe) {
  __shared__ double redd[kSumThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n_partial; i += kSumThreads) s += partial[i];
  const double sum_d = block_sum<kSumThreads>(s, redd);
  double q2 = 0.0;
  for (int p = threadIdx.x; p < m * m; p += kSumThreads) q2 += (double)cabs2(probe[p]);
  const double norm2 = block_sum<kSumThreads>(q2, redd);
  const double dp_avg = sqrt(sum_d / (double)n_pos) / (double)m;
  const float scale = norm2 > 0.0 ? (float)(dp_avg / sqrt(norm2)) : 0.f;
  for (int p = threadIdx.x; p < m * m; p += kSumThreads) probe[p] = cscale(probe[p], scale);
}

template <int M>
cudaError_t set_step_smem() {
  return cudaFuncSetAttribute(k_step<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              step_smem_limit());
}

template <int M>
cudaError_t launch_step_t(int b, const StepArgs& a, cudaStream_t s) {
  const size_t bytes = step_smem_elems<M>(a.levels) * sizeof(float2);
  k_step<M><<<b, StepThreads<M>::value, bytes, s>>>(a);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_misfit_t(const float2* object, const float2* probe, const int32_t* pos,
                            const float* amp, int n_rows, int n_cols, int n_pos, double* partial,
                            cudaStream_t s) {
  const size_t bytes = level_floats2<M>(0) * sizeof(float2);
  k_misfit<M><<<n_pos, StepThreads<M>::value, bytes, s>>>(object, probe, pos, amp, n_rows, n_cols,
                                                          partial);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_simulate_t(const float2* object, const float2* probe, const int32_t* pos,
                              int n_rows, int n_cols, int n_pos, float* out, cudaStream_t s) {
  const size_t bytes = level_floats2<M>(0) * sizeof(float2);
  k_simulate<M><<<n_pos, StepThreads<M>::value, bytes, s>>>(object, probe, pos, n_rows, n_cols, out);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_fft2_t(const float2* in, float2* out, int count, int inverse, cudaStream_t s) {
  const size_t bytes = level_floats2<M>(0) * sizeof(float2);
  k_fft2<M><<<count, StepThreads<M>::value, bytes, s>>>(in, out, inverse);
  return cudaGetLastError();
}

template <int M>
cudaError_t set_aux_smem() {
  const int bytes = (int)(level_floats2<M>(0) * sizeof(float2));
  cudaError_t e = cudaFuncSetAttribute(k_misfit<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_simulate<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft2<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

#define EMG_DISPATCH_M(m, CALL)        \
  switch (m) {                         \
    case 16: { constexpr int M = 16; return CALL; }   \
    case 32: { constexpr int M = 32; return CALL; }   \
    case 64: { constexpr int M = 64; return CALL; }   \
    case 128: { constexpr int M = 128; return CALL; } \
    default: return cudaErrorInvalidValue;            \
  }

}  // namespace

// Dynamic shared memory per CTA; 227 KB minus room for the kernels' static reductions.
// Launch with programmatic stream serialisation (see pdl_wait / pdl_trigger).
template <typename Kernel, typename... Args>
cudaError_t launch_pdl(Kernel kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

int step_smem_limit() { return 227 * 1024 - 1024; }

size_t step_smem_bytes(int m, int levels) {
  switch (m) {
    case 16: return step_smem_elems<16>(levels) * sizeof(float2);
    case 32: return step_smem_elems<32>(levels) * sizeof(float2);
    case 64: return step_smem_elems<64>(levels) * sizeof(float2);
    case 128: return step_smem_elems<128>(levels) * sizeof(float2);
    default: return 0;
  }
}

cudaError_t set_cluster_attrs();

cudaError_t upload_twiddles() {
  float2 h[256];
  for (int t = 0; t < 256; ++t) {
    const double ang = -2.0 * M_PI * (double)t / 256.0;
    double c = cos(ang), s = sin(ang);
    if (fabs(c) < 1e-15) c = 0.0;
    if (fabs(s) < 1e-15) s = 0.0;
    h[t] = make_float2((float)c, (float)s);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_twiddle, h, sizeof(h));
  if (e != cudaSuccess) return e;
  if ((e = set_step_smem<16>()) != cudaSuccess) return e;
  if ((e = set_step_smem<32>()) != cudaSuccess) return e;
  if ((e = set_step_smem<64>()) != cudaSuccess) return e;
  if ((e = set_step_smem<128>()) != cudaSuccess) return e;
  if ((e = set_cluster_attrs()) != cudaSuccess) return e;
  if ((e = set_aux_smem<16>()) != cudaSuccess) return e;
  if ((e = set_aux_smem<32>()) != cudaSuccess) return e;
  if ((e = set_aux_smem<64>()) != cudaSuccess) return e;
  if ((e = set_aux_smem<128>()) != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_prep_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrepTileSmemMax);
  return e;
}

cudaError_t launch_amp_prep(const float* d, float* amp, int m, int n_pos, cudaStream_t s) {
  const size_t rows = (size_t)n_pos * m;
  int blocks = (int)((rows + 7) / 8);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks == 0) return cudaSuccess;
  switch (m) {
    case 16: k_amp_prep<16><<<blocks, 256, 0, s>>>(d, amp, n_pos); break;
    case 32: k_amp_prep<32><<<blocks, 256, 0, s>>>(d, amp, n_pos); break;
    case 64: k_amp_prep<64><<<blocks, 256, 0, s>>>(d, amp, n_pos); break;
    case 128: k_amp_prep<128><<<blocks, 256, 0, s>>>(d, amp, n_pos); break;
    case 256: k_amp_prep<256><<<blocks, 256, 0, s>>>(d, amp, n_pos); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Shared memory each gather block reserves in all (its row buffer plus unused
// dynamic shared memory, within the 48 KB a launch may ask for without opting
// in).  At the bench size a block that large does not fit beside two step
// CTAs, so the gathers run on the SMs the step leaves free instead of slowing
// its CTAs: end to end 1.57M -> 1.62M positions/s (20 KB per block gave 1.44M).
#ifndef EMG_GATHER_BLOCK_SMEM
#define EMG_GATHER_BLOCK_SMEM (46 * 1024)
#endif
cudaError_t launch_amp_gather(const float* d, const int32_t* idx, int b, float* amp, int m, cudaStream_t s) {
  const int groups = b * (m / kGatherRows);
  int blocks = (groups + kGatherWarps - 1) / kGatherWarps;
  if (blocks > kGatherBlocks) blocks = kGatherBlocks;
  if (blocks == 0) return cudaSuccess;
  const dim3 th(kGatherWarps * 32);
  const size_t rows_bytes = (size_t)kGatherWarps * kGatherRows * m * sizeof(float);
  const size_t pad = rows_bytes < EMG_GATHER_BLOCK_SMEM ? EMG_GATHER_BLOCK_SMEM - rows_bytes : 0;
  switch (m) {
    case 16: k_amp_gather<16><<<blocks, th, pad, s>>>(d, idx, b, amp); break;
    case 32: k_amp_gather<32><<<blocks, th, pad, s>>>(d, idx, b, amp); break;
    case 64: k_amp_gather<64><<<blocks, th, pad, s>>>(d, idx, b, amp); break;
    case 128: k_amp_gather<128><<<blocks, th, pad, s>>>(d, idx, b, amp); break;
    case 256: k_amp_gather<256><<<blocks, th, pad, s>>>(d, idx, b, amp); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#ifndef EMG_PREP_TILE
#define EMG_PREP_TILE 8
#endif
bool prep_tiled_config(PrepArgs& a) {
  int tile = EMG_PREP_TILE;
  while (tile < (1 << (a.levels - 1))) tile *= 2;
  if (tile > a.m) tile = a.m;
  a.tile = tile;
  a.halo = (a.prolong == 1) ? (1 << (a.levels - 1)) : 0;
  if ((tile >> (a.levels - 1)) < 1) return false;
  return prep_tile_smem(a) <= kPrepTileSmemMax;
}

template <int M, int C>
constexpr size_t stepc_smem_bytes() {
  return CTile<M, C>::smem_elems * sizeof(float2);
}

// Clusters of the step kernel that can be resident at once (CTAs per SM from
// the occupancy calculator x SMs / cluster size), or 0 if unknown.
template <int M, int C>
int stepc_resident_clusters() {
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stepc<M, C>, CTile<M, C>::NT,
                                                    stepc_smem_bytes<M, C>()) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms / C;
}

int step_resident_clusters(int m, int cluster) {
  switch (m * 16 + cluster) {
    case 16 * 16 + 2: return stepc_resident_clusters<16, 2>();
    case 32 * 16 + 2: return stepc_resident_clusters<32, 2>();
    case 64 * 16 + 2: return stepc_resident_clusters<64, 2>();
    case 64 * 16 + 4: return stepc_resident_clusters<64, 4>();
    case 128 * 16 + 2: return stepc_resident_clusters<128, 2>();
    case 128 * 16 + 4: return stepc_resident_clusters<128, 4>();
    case 128 * 16 + 8: return stepc_resident_clusters<128, 8>();
    case 256 * 16 + 8: return stepc_resident_clusters<256, 8>();
    default: return 0;
  }
}

int fused_prep_tiles(PrepArgs& a, int m, int cluster) {
  size_t smem = 0;
  switch (m * 16 + cluster) {
    case 16 * 16 + 2: smem = stepc_smem_bytes<16, 2>(); break;
    case 32 * 16 + 2: smem = stepc_smem_bytes<32, 2>(); break;
    case 64 * 16 + 2: smem = stepc_smem_bytes<64, 2>(); break;
    case 64 * 16 + 4: smem = stepc_smem_bytes<64, 4>(); break;
    case 128 * 16 + 2: smem = stepc_smem_bytes<128, 2>(); break;
    case 128 * 16 + 4: smem = stepc_smem_bytes<128, 4>(); break;
    case 128 * 16 + 8: smem = stepc_smem_bytes<128, 8>(); break;
    case 256 * 16 + 8: smem = stepc_smem_bytes<256, 8>(); break;
    default: return 0;
  }
  int tile = 32;
  while (tile < (1 << (a.levels - 1))) tile *= 2;
  if (tile > m) tile = m;
  a.tile = tile;
  a.halo = (a.prolong == 1) ? (1 << (a.levels - 1)) : 0;
  if ((tile >> (a.levels - 1)) < 1 || prep_tile_smem(a) > smem) return 0;
  return (m / tile) * (m / tile);
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s) {
  PrepArgs t = a;
  if (a.mq_read && prep_tiled_config(t)) {
    const int tiles = (t.m / t.tile) * (t.m / t.tile);
    cudaError_t e = launch_pdl(k_prep_tile, dim3(tiles), dim3(kPrepTileThreads), prep_tile_smem(t), s, t);
    if (e != cudaSuccess) return e;
  } else {
    k_prep<<<1, kPrepThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_probe_max(const float2* probe, int m, unsigned* slot, cudaStream_t s) {
  const int n = m * m;
  int blocks = (n + 255) / 256;
  if (blocks > 64) blocks = 64;
  k_probe_max<<<blocks, 256, 0, s>>>(probe, n, slot);
  return cudaGetLastError();
}

// Launch of a C-CTA cluster kernel with programmatic stream serialisation.
template <typename Kernel, typename... Args>
cudaError_t launch_cluster_pdl(Kernel kernel, int cluster, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                               Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = cluster;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename Kernel, typename... Args>
cudaError_t launch_cluster_plain(Kernel kernel, int cluster, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                 Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int M, int MODE>
cudaError_t launch_fwdc_t(int count, const FwdArgs& a, cudaStream_t s) {
  constexpr int C = ClusterSize<M>::value;
  using TL = CTile<M, C>;
  cudaError_t e = launch_cluster_plain(k_fwdc<M, C, MODE>, C, dim3(C * count), dim3(TL::NT),
                                       TL::smem_elems * sizeof(float2), s, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int M>
cudaError_t launch_ifftc_t(int count, const FwdArgs& a, cudaStream_t s) {
  constexpr int C = ClusterSize<M>::value;
  using TL = CTile<M, C>;
  cudaError_t e = launch_cluster_plain(k_ifftc<M, C>, C, dim3(C * count), dim3(TL::NT),
                                       TL::smem_elems * sizeof(float2), s, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int M>
cudaError_t launch_gradc_t(int b, const GradArgs& a, cudaStream_t s) {
  constexpr int C = ClusterSize<M>::value;
  using TL = CTile<M, C>;
  cudaError_t e = launch_cluster_plain(k_gradc<M, C>, C, dim3(C * b), dim3(TL::NT),
                                       TL::smem_elems * sizeof(float2), s, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename Kernel>
cudaError_t set_cluster_smem(Kernel k, size_t elems) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(elems * sizeof(float2)));
}

template <int M>
cudaError_t set_grad_attrs() {
  constexpr int C = ClusterSize<M>::value;
  return set_cluster_smem(k_gradc<M, C>, CTile<M, C>::smem_elems);
}

// Dynamic shared-memory limits of the cluster kernels (once per device).
cudaError_t set_cluster_attrs() {
  cudaError_t e;
  if ((e = set_cluster_smem(k_stepc<16, 2>, CTile<16, 2>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_stepc<32, 2>, CTile<32, 2>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_stepc<64, 4>, CTile<64, 4>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_stepc<128, 4>, CTile<128, 4>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_stepc<128, 8>, CTile<128, 8>::smem_elems)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_stepc<64, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(CTile<64, 2>::smem_elems * sizeof(float2)))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_stepc<128, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(CTile<128, 2>::smem_elems * sizeof(float2)))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_stepc<256, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(CTile<256, 8>::smem_elems * sizeof(float2)))) != cudaSuccess)
    return e;
  if ((e = set_cluster_smem(k_stepc<128, 2, true>, CTile<128, 2>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_stepc<128, 4, true>, CTile<128, 4>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_stepc<128, 8, true>, CTile<128, 8>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_stepc<256, 8, true>, CTile<256, 8>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_fwdc<256, 8, 0>, CTile<256, 8>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_fwdc<256, 8, 1>, CTile<256, 8>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_fwdc<256, 8, 2>, CTile<256, 8>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_cluster_smem(k_ifftc<256, 8>, CTile<256, 8>::smem_elems)) != cudaSuccess) return e;
  if ((e = set_grad_attrs<16>()) != cudaSuccess) return e;
  if ((e = set_grad_attrs<32>()) != cudaSuccess) return e;
  if ((e = set_grad_attrs<64>()) != cudaSuccess) return e;
  if ((e = set_grad_attrs<128>()) != cudaSuccess) return e;
  if ((e = set_grad_attrs<256>()) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_grad_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024)) !=
      cudaSuccess)
    return e;
  return cudaSuccess;
}

template <int M, int C>
cudaError_t launch_stepc_t(int b, const StepArgs& a, cudaStream_t s) {
  using TL = CTile<M, C>;
  cudaError_t e = launch_cluster_pdl(k_stepc<M, C>, C, dim3(C * (b + a.prep_clusters)), dim3(TL::NT),
                                     TL::smem_elems * sizeof(float2), s, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int M, int C>
cudaError_t launch_stepc_rin_t(int b, const StepArgs& a, cudaStream_t s) {
  using TL = CTile<M, C>;
  cudaError_t e = launch_cluster_pdl(k_stepc<M, C, true>, C, dim3(C * b), dim3(TL::NT),
                                     TL::smem_elems * sizeof(float2), s, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_step_rin(int m, int b, const StepArgs& a, cudaStream_t s) {
  switch (m * 16 + a.cluster) {
    case 128 * 16 + 2: return launch_stepc_rin_t<128, 2>(b, a, s);
    case 128 * 16 + 4: return launch_stepc_rin_t<128, 4>(b, a, s);
    case 128 * 16 + 8: return launch_stepc_rin_t<128, 8>(b, a, s);
    case 256 * 16 + 8: return launch_stepc_rin_t<256, 8>(b, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step(int m, int b, const StepArgs& a, cudaStream_t s) {
  switch (m * 16 + a.cluster) {
    case 16 * 16 + 1: return launch_step_t<16>(b, a, s);
    case 16 * 16 + 2: return launch_stepc_t<16, 2>(b, a, s);
    case 32 * 16 + 1: return launch_step_t<32>(b, a, s);
    case 32 * 16 + 2: return launch_stepc_t<32, 2>(b, a, s);
    case 64 * 16 + 2: return launch_stepc_t<64, 2>(b, a, s);
    case 64 * 16 + 4: return launch_stepc_t<64, 4>(b, a, s);
    case 128 * 16 + 2: return launch_stepc_t<128, 2>(b, a, s);
    case 128 * 16 + 4: return launch_stepc_t<128, 4>(b, a, s);
    case 128 * 16 + 8: return launch_stepc_t<128, 8>(b, a, s);
    case 256 * 16 + 8: return launch_stepc_t<256, 8>(b, a, s);
    default: return cudaErrorInvalidValue;
  }
}

// CTAs per position by default: 4 for m = 128 where every CTA keeps a row at
// the coarsest level (measured faster than 2), else the one choice built.
int default_cluster(int m, int levels) {
  if (m <= 32) return 1;
  if (m == 256) return 8;
  if (m == 128 && step_supported(m, levels, 4)) return 4;
  return 2;
}

// Copies, per problem, the order row of the current epoch into the buffer its
// captured minibatch kernels read.  One block per problem.
__global__ void __launch_bounds__(256) k_batch_orders(const int32_t* const* src, int32_t* const* dst, const int* n,
                                                      const int* epoch) {
  const int q = blockIdx.x;
  const int len = n[q];
  const int32_t* from = src[q] + (size_t)(*epoch) * len;
  for (int i = threadIdx.x; i < len; i += 256) dst[q][i] = from[i];
}

__global__ void k_epoch_advance(int* epoch) { *epoch += 1; }

cudaError_t launch_batch_orders(const int32_t* const* src, int32_t* const* dst, const int* n, int count,
                                const int* epoch, cudaStream_t s) {
  k_batch_orders<<<count, 256, 0, s>>>(src, dst, n, epoch);
  return cudaGetLastError();
}

cudaError_t launch_epoch_advance(int* epoch, cudaStream_t s) {
  k_epoch_advance<<<1, 1, 0, s>>>(epoch);
  return cudaGetLastError();
}

cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t s) {
  const int n_tiles = a.tiles_x * a.tiles_y;
  const int n_probe = (a.m * a.m + kApplyProbePx - 1) / kApplyProbePx;
  const size_t bytes = (size_t)a.b * 3 * sizeof(int);
  cudaError_t e = launch_pdl(k_apply, dim3(n_tiles + n_probe), dim3(kApplyThreads), bytes, s, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_misfit(int m, const float2* object, const float2* probe, const int32_t* pos,
                          const float* amp, int n_rows, int n_cols, int n_pos, double* partial,
                          cudaStream_t s) {
  if (m == 256) {
    FwdArgs f{};
    f.object = object;
    f.probe = probe;
    f.pos = pos;
    f.amp = amp;
    f.n_rows = n_rows;
    f.n_cols = n_cols;
    f.partial = partial;
    return launch_fwdc_t<256, 0>(n_pos, f, s);
  }
  EMG_DISPATCH_M(m, (launch_misfit_t<M>(object, probe, pos, amp, n_rows, n_cols, n_pos, partial, s)));
}

cudaError_t launch_sum(const double* x, int n, double scale, double* out, cudaStream_t s) {
  k_sum<<<1, kSumThreads, 0, s>>>(x, n, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_simulate(int m, const float2* object, const float2* probe, const int32_t* pos,
                            int n_rows, int n_cols, int n_pos, float* out, cudaStream_t s) {
  if (m == 256) {
    FwdArgs f{};
    f.object = object;
    f.probe = probe;
    f.pos = pos;
    f.n_rows = n_rows;
    f.n_cols = n_cols;
    f.out_intensity = out;
    return launch_fwdc_t<256, 1>(n_pos, f, s);
  }
  EMG_DISPATCH_M(m, (launch_simulate_t<M>(object, probe, pos, n_rows, n_cols, n_pos, out, s)));
}

cudaError_t launch_fft2(int m, const float2* in, float2* out, int count, int inverse,
                        cudaStream_t s) {
  if (m == 256) {
    FwdArgs f{};
    f.in = in;
    f.out = out;
    return inverse ? launch_ifftc_t<256>(count, f, s) : launch_fwdc_t<256, 2>(count, f, s);
  }
  EMG_DISPATCH_M(m, (launch_fft2_t<M>(in, out, count, inverse, s)));
}

template <int M>
int gradient_wave_t() {
  constexpr int C = ClusterSize<M>::value;
  using TL = CTile<M, C>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * 4096);
  cfg.blockDim = dim3(TL::NT);
  cfg.dynamicSmemBytes = TL::smem_elems * sizeof(float2);
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = C;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_gradc<M, C>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int gradient_positions_per_wave(int m) {
  switch (m) {
    case 16: return gradient_wave_t<16>();
    case 32: return gradient_wave_t<32>();
    case 64: return gradient_wave_t<64>();
    case 128: return gradient_wave_t<128>();
    case 256: return gradient_wave_t<256>();
    default: return 0;
  }
}

cudaError_t launch_gradient(int m, int b, const GradArgs& a, cudaStream_t s) {
  switch (m) {
    case 16: return launch_gradc_t<16>(b, a, s);
    case 32: return launch_gradc_t<32>(b, a, s);
    case 64: return launch_gradc_t<64>(b, a, s);
    case 128: return launch_gradc_t<128>(b, a, s);
    case 256: return launch_gradc_t<256>(b, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_grad_reduce(const GradReduceArgs& a, cudaStream_t s) {
  const int n_tiles = a.tiles_x * a.tiles_y;
  const int n_probe = (a.m * a.m + 31) / 32;
  k_grad_reduce<<<n_tiles + n_probe, kApplyThreads, (size_t)a.b * 3 * sizeof(int), s>>>(a);
  return cudaGetLastError();
}

// Whether the step kernel for probe side m with `cluster` CTAs per position
// supports `levels` multigrid levels.
bool step_supported(int m, int levels, int cluster) {
  const bool built = (cluster == 1 && m <= 32) || (cluster == 2 && m <= 128) || (cluster == 4 && (m == 64 || m == 128)) ||
                     (cluster == 8 && m >= 128);
  if (!built) return false;
  if (cluster == 1) return step_smem_bytes(m, levels) <= (size_t)step_smem_limit();
  if ((m >> (levels - 1)) < cluster) return false;  // every CTA needs a row at the coarsest level
  size_t need = 0;
  for (int l = 1; l < levels; ++l) {
    const size_t wl = (size_t)m >> l, hl = wl / cluster;
    need += (2 * hl + 2) * (wl + 1);
  }
  return need <= (size_t)m * (m / cluster + 1);
}

cudaError_t launch_normalize_probe(const float* amp, int m, int n_pos, float2* probe,
                                   double* scratch, int scratch_len, cudaStream_t s) {
  const size_t n = (size_t)n_pos * m * m;
  int blocks = (int)((n + kNormThreads - 1) / kNormThreads);
  if (blocks > scratch_len) blocks = scratch_len;
  k_sum_sq<<<blocks, kNormThreads, 0, s>>>(amp, n, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_scale_probe<<<1, kSumThreads, 0, s>>>(scratch, blocks, m, n_pos, probe);
  return cudaGetLastError();
}

}  // namespace emg

// ===========================================================================
// Allocation-free minibatch step: emg_step_minibatch_noalloc (include/emagpie.h).
//
// For callers that may not allocate device memory: code that runs inside a
// memory pool or arena it does not own, code that must not grow the device
// footprint after start-up, or code under a host-side policy that forbids
// cudaMalloc on its hot path.  They pass every input and output; the only
// scratch is the fixed array below, which every GPU that loads this library
// holds until the process exits.
// ===========================================================================
#include <string.h>

#include <mutex>

#include "../../include/emagpie.h"

namespace emg {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[EMG_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_base[256] = {nullptr};

struct NoAllocLayout {
  size_t idx, mq, wq, zt, qt, mu, phi, phi_after, total;
  size_t G[kMaxLevels], Q[kMaxLevels], u[kMaxLevels], Wz[kMaxLevels], WR[kMaxLevels], T[kMaxLevels];
};

// Byte offsets of every scratch array of one call, each 256-byte aligned.
NoAllocLayout noalloc_layout(int m, int levels, int b) {
  NoAllocLayout L{};
  size_t bytes = 0;
  auto take = [&](size_t n) {
    const size_t off = (bytes + 255) & ~(size_t)255;
    bytes = off + n;
    return off;
  };
  L.idx = take((size_t)b * sizeof(int32_t));
  L.mq = take(2 * sizeof(unsigned));
  for (int l = 0; l < levels; ++l) {
    const size_t n = (size_t)(m >> l) * (m >> l);
    L.G[l] = take(n * sizeof(float2));
    L.Q[l] = take(n * sizeof(float2));
    L.u[l] = take(n * sizeof(float));
    if (l + 1 < levels) {
      L.Wz[l] = take(n * sizeof(float));
      L.WR[l] = take(n * sizeof(float2));
      L.T[l] = take(n / 4 * sizeof(float));
    }
  }
  L.wq = take((size_t)m * m * sizeof(float));
  L.zt = take((size_t)b * m * m * sizeof(float2));
  L.qt = take((size_t)b * m * m * sizeof(float2));
  L.mu = take((size_t)b * sizeof(float));
  L.phi = take((size_t)b * sizeof(double));
  L.phi_after = take((size_t)b * sizeof(double));
  L.total = bytes;
  return L;
}

// Once per device, with that device current: twiddles, kernel attributes and
// the device address of the scratch array (a host-side name of a __device__
// array is not a device address, so it is looked up here).
cudaError_t noalloc_setup(int dev, unsigned char** base) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  if (g_noalloc_base[dev]) {
    *base = g_noalloc_base[dev];
    return cudaSuccess;
  }
  cudaError_t e = upload_twiddles();
  if (e != cudaSuccess) return e;
  const int lim = step_smem_limit();
  if ((e = cudaFuncSetAttribute(k_step<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) ||
      (e = cudaFuncSetAttribute(k_step<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) ||
      (e = cudaFuncSetAttribute(k_step<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) ||
      (e = cudaFuncSetAttribute(k_step<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)))
    return e;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_noalloc_base[dev] = (unsigned char*)p;
  *base = (unsigned char*)p;
  return cudaSuccess;
}

// The minibatch's position indices travel inside the launch parameters, which
// the runtime copies when the launch is enqueued: the caller may overwrite its
// host array as soon as the call returns, pinned or not.
constexpr int kNoAllocMaxIdx = 2048;
struct NoAllocIdx {
  int32_t v[kNoAllocMaxIdx];
};

__global__ void k_noalloc_idx(const NoAllocIdx p, int b, int32_t* __restrict__ out) {
  for (int i = threadIdx.x; i < b; i += blockDim.x) out[i] = p.v[i];
}

template <int M>
cudaError_t launch_step_natural(int b, const StepArgs& a, cudaStream_t s) {
  const size_t bytes = step_smem_elems<M>(a.levels) * sizeof(float2);
  k_step<M, true><<<b, StepThreads<M>::value, bytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace
}  // namespace emg

extern "C" emg_status emg_step_minibatch_noalloc(float* object, int32_t n_rows, int32_t n_cols,
                                                 float* probe, int32_t m, const int32_t* pos,
                                                 const float* intensity, int32_t n_pos,
                                                 const int32_t* idx, int32_t b,
                                                 const emg_params* p, emg_stream_t stream) {
  using namespace emg;
  if (!object || !probe || !pos || !intensity || !idx || !p) return EMG_EINVAL;
  if (n_rows < 1 || n_cols < 1 || n_pos < 1 || b < 1 || b > n_pos || b > kNoAllocMaxIdx) return EMG_EINVAL;
  if (m != 16 && m != 32 && m != 64 && m != 128) return EMG_ENOTSUP;  // m = 256 needs a cluster
  if (!(p->alpha > 0.f) || !isfinite(p->alpha) || !(p->w_eps >= 0.f) || !isfinite(p->w_eps))
    return EMG_EINVAL;
  if (p->levels < 1 || p->levels > kMaxLevels || (m >> (p->levels - 1)) < 2) return EMG_EINVAL;
  if (p->prolong != EMG_PROLONG_CONST && p->prolong != EMG_PROLONG_BILINEAR) return EMG_EINVAL;
  if (p->combine != EMG_COMBINE_WAVG && p->combine != EMG_COMBINE_SUM) return EMG_EINVAL;
  if (p->joint != 0 && p->joint != 1) return EMG_EINVAL;
  if (p->scatter != EMG_SCATTER_DETERMINISTIC) return EMG_ENOTSUP;
  if (p->dft != EMG_DFT_FFT32) return p->dft == EMG_DFT_BF16X3 ? EMG_ENOTSUP : EMG_EINVAL;
  if (step_smem_bytes(m, p->levels) > (size_t)step_smem_limit()) return EMG_ENOTSUP;
  for (int i = 0; i < b; ++i)
    if (idx[i] < 0 || idx[i] >= n_pos) return EMG_EINVAL;
  const NoAllocLayout L = noalloc_layout(m, p->levels, b);
  if (L.total > (size_t)EMG_NOALLOC_SCRATCH_BYTES) return EMG_EINVAL;  // beyond the fixed scratch

  int dev = 0;
  unsigned char* base = nullptr;
  if (cudaGetDevice(&dev) != cudaSuccess || noalloc_setup(dev, &base) != cudaSuccess) return EMG_ECUDA;
  const cudaStream_t s = (cudaStream_t)stream;
  int32_t* d_idx = (int32_t*)(base + L.idx);
  {
    NoAllocIdx pv;
    memcpy(pv.v, idx, (size_t)b * sizeof(int32_t));
    k_noalloc_idx<<<1, 256, 0, s>>>(pv, b, d_idx);
    if (cudaGetLastError() != cudaSuccess) return EMG_ECUDA;
  }

  unsigned* d_mq = (unsigned*)(base + L.mq);
  if (cudaMemsetAsync(d_mq, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return EMG_ECUDA;
  if (launch_probe_max((const float2*)probe, m, d_mq, s) != cudaSuccess) return EMG_ECUDA;

  PrepArgs pa{};
  StepArgs sa{};
  pa.probe = (const float2*)probe;
  pa.mq_read = d_mq;
  pa.mq_next = d_mq + 1;
  pa.m = m;
  pa.levels = p->levels;
  pa.prolong = p->prolong;
  pa.alpha = p->alpha;
  pa.w_eps = p->w_eps;
  pa.wq = (float*)(base + L.wq);
  for (int l = 0; l < p->levels; ++l) {
    pa.G[l] = (float2*)(base + L.G[l]);
    pa.Q[l] = (float2*)(base + L.Q[l]);
    pa.u[l] = (float*)(base + L.u[l]);
    sa.lv.G[l] = pa.G[l];
    sa.lv.Q[l] = pa.Q[l];
    if (l + 1 < p->levels) {
      pa.Wz[l] = (float*)(base + L.Wz[l]);
      pa.WR[l] = (float2*)(base + L.WR[l]);
      pa.T[l] = (float*)(base + L.T[l]);
      sa.lv.Wz[l] = pa.Wz[l];
      sa.lv.WR[l] = pa.WR[l];
    }
  }
  sa.object = (const float2*)object;
  sa.probe = (const float2*)probe;
  sa.pos = pos;
  sa.amp = intensity;
  sa.order = d_idx;
  sa.n_rows = n_rows;
  sa.n_cols = n_cols;
  sa.n_pos = n_pos;
  sa.b = b;
  sa.levels = p->levels;
  sa.prolong = p->prolong;
  sa.joint = p->joint;
  sa.verify = 0;
  sa.alpha = p->alpha;
  sa.mq = d_mq;
  sa.zt = (float2*)(base + L.zt);
  sa.qt = (float2*)(base + L.qt);
  sa.mu = (float*)(base + L.mu);
  sa.phi = (double*)(base + L.phi);
  sa.phi_after = (double*)(base + L.phi_after);
  ApplyArgs aa{};
  aa.object = (float2*)object;
  aa.probe = (float2*)probe;
  aa.pos = pos;
  aa.order = d_idx;
  aa.b = b;
  aa.n_pos = n_pos;
  aa.n_rows = n_rows;
  aa.n_cols = n_cols;
  aa.m = m;
  aa.combine = p->combine;
  aa.zt = sa.zt;
  aa.qt = sa.qt;
  aa.mu = sa.mu;
  aa.wq = pa.wq;
  aa.mq_next = d_mq + 1;
  aa.tiles_x = apply_tiles_x(n_cols);
  aa.tiles_y = apply_tiles_y(n_rows);

  cudaError_t e = launch_prep(pa, s);
  if (e == cudaSuccess) {
    switch (m) {
      case 16: e = launch_step_natural<16>(b, sa, s); break;
      case 32: e = launch_step_natural<32>(b, sa, s); break;
      case 64: e = launch_step_natural<64>(b, sa, s); break;
      default: e = launch_step_natural<128>(b, sa, s); break;
    }
  }
  if (e == cudaSuccess) e = launch_apply(aa, s);
  return e == cudaSuccess ? EMG_OK : EMG_ECUDA;
}

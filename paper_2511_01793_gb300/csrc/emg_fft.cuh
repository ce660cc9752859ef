// Shared-memory 2-D FFT of an m x m complex64 tile for sm_103a.
//
// The operator is the unnormalised forward 2-D DFT F of Sec. 2.1 (arXiv
// 2511.01793); the inverse passes are unnormalised too and the caller folds
// the 1/m^2 of F^-1 into its pointwise step.
//
// Each 1-D transform of length M = N1 * N2 is one Cooley-Tukey split:
//   pass A: for each n1, an N2-point DFT over x[n1 + N1 n2]; multiply output
//           k2 by W_M^(n1 k2); write back to the same slots;
//   pass B: for each k2, an N1-point DFT over the pass-A outputs; write back to
//           the same slots.
// Both passes read and write one fixed set of addresses per thread, so the
// transform is in place without hazards inside a pass.  The output leaves
// frequency k2 + N2 k1 at slot k1 + N1 k2 ("storage order"); the inverse
// passes consume storage order and produce natural order, so a forward
// transform, a pointwise step and an inverse transform never need an explicit
// bit-reversal.  Small DFTs (N <= 16) run in registers; twiddles come from a
// table computed on the host in FP64.
//
// Layout: element (r, c) of the tile lives at buf[r * S + c] with S = M + 1.
// Consecutive lanes always take consecutive lines (rows or columns), so every
// shared-memory access of a warp is bank-conflict free for odd S.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace emg {

// W_256^t = exp(-2 pi i t / 256), t = 0..255; filled once per device by the host.
// Defined here: this header belongs to exactly one translation unit.
__constant__ float2 c_twiddle[256];

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}

// x * W_N^k (forward) or x * W_N^-k (inverse); k is a compile-time constant
// after unrolling, so the trivial factors 1, -1, -i, +i cost nothing.
template <int N, bool INV>
__device__ __forceinline__ float2 tw_mul(float2 x, int k) {
  if (k == 0) return x;
  if (2 * k == N) return make_float2(-x.x, -x.y);
  if (4 * k == N) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
  if (4 * k == 3 * N) return INV ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
  const float2 w = c_twiddle[k * (256 / N)];
  return INV ? cmulc(x, w) : cmul(x, w);
}

// In-register N-point DFT, natural order in and out (radix-2, decimation in time).
template <int N, bool INV>
struct Dft {
  static __device__ __forceinline__ void run(float2 (&v)[N]) {
    float2 e[N / 2], o[N / 2];
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    Dft<N / 2, INV>::run(e);
    Dft<N / 2, INV>::run(o);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const float2 t = tw_mul<N, INV>(o[k], k);
      v[k] = cadd(e[k], t);
      v[k + N / 2] = csub(e[k], t);
    }
  }
};
template <bool INV>
struct Dft<1, INV> {
  static __device__ __forceinline__ void run(float2 (&)[1]) {}
};

template <int M> struct FftPlan;
template <> struct FftPlan<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct FftPlan<32> { static constexpr int N1 = 4, N2 = 8; };
template <> struct FftPlan<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct FftPlan<128> { static constexpr int N1 = 8, N2 = 16; };
template <> struct FftPlan<256> { static constexpr int N1 = 16, N2 = 16; };

// Storage slot -> frequency of the 1-D transform.
template <int M>
__host__ __device__ __forceinline__ int storage_to_freq(int e) {
  return e / FftPlan<M>::N1 + FftPlan<M>::N2 * (e % FftPlan<M>::N1);
}

// W_M^(j k) for runtime j and compile-time k (warp-uniform j: constant-cache broadcast).
template <int M>
__device__ __forceinline__ float2 stage_twiddle(int j, int k) {
  return c_twiddle[((j * k) & (M - 1)) * (256 / M)];
}

// ---- forward / inverse passes over LINES lines of length M -------------------
// Element e of line l lives at buf[l * LS + e * ES].  Slot s of a pass maps to
// (j = s / LINES, line = s % LINES): consecutive lanes take consecutive lines.

template <int M, int LINES, int LS, int ES, int NT>
__device__ __forceinline__ void gpass_a_fwd(float2* buf, int tid) {
  constexpr int N1 = FftPlan<M>::N1, N2 = FftPlan<M>::N2;
  for (int s = tid; s < LINES * N1; s += NT) {
    const int j = s / LINES, line = s % LINES;
    float2* p = buf + line * LS + j * ES;
    float2 v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = p[N1 * n2 * ES];
    Dft<N2, false>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmul(v[k2], stage_twiddle<M>(j, k2));
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) p[N1 * k2 * ES] = v[k2];
  }
}

template <int M, int LINES, int LS, int ES, int NT>
__device__ __forceinline__ void gpass_a_inv(float2* buf, int tid) {
  constexpr int N1 = FftPlan<M>::N1, N2 = FftPlan<M>::N2;
  for (int s = tid; s < LINES * N1; s += NT) {
    const int j = s / LINES, line = s % LINES;
    float2* p = buf + line * LS + j * ES;
    float2 v[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) v[k2] = p[N1 * k2 * ES];
#pragma unroll
    for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmulc(v[k2], stage_twiddle<M>(j, k2));
    Dft<N2, true>::run(v);
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) p[N1 * n2 * ES] = v[n2];
  }
}

template <int M, int LINES, int LS, int ES, int NT, bool INV>
__device__ __forceinline__ void gpass_b(float2* buf, int tid) {
  constexpr int N1 = FftPlan<M>::N1, N2 = FftPlan<M>::N2;
  for (int s = tid; s < LINES * N2; s += NT) {
    const int k2 = s / LINES, line = s % LINES;
    float2* p = buf + line * LS + N1 * k2 * ES;
    float2 v[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = p[i * ES];
    Dft<N1, INV>::run(v);
#pragma unroll
    for (int i = 0; i < N1; ++i) p[i * ES] = v[i];
  }
}

// Full m x m tile, row stride M + 1: rows (COL = false) or columns (COL = true).
template <int M, bool COL, int NT>
__device__ __forceinline__ void pass_a_fwd(float2* buf, int tid) {
  gpass_a_fwd<M, M, COL ? 1 : M + 1, COL ? M + 1 : 1, NT>(buf, tid);
}

template <int M, bool COL, int NT>
__device__ __forceinline__ void pass_a_inv(float2* buf, int tid) {
  gpass_a_inv<M, M, COL ? 1 : M + 1, COL ? M + 1 : 1, NT>(buf, tid);
}

template <int M, bool COL, int NT, bool INV>
__device__ __forceinline__ void pass_b(float2* buf, int tid) {
  gpass_b<M, M, COL ? 1 : M + 1, COL ? M + 1 : 1, NT, INV>(buf, tid);
}

// Forward transform up to (not including) the column pass B, which callers
// usually fuse with their spectral step.
template <int M, int NT>
__device__ __forceinline__ void fft2_fwd_until_col_b(float2* buf, int tid) {
  pass_a_fwd<M, false, NT>(buf, tid);
  __syncthreads();
  pass_b<M, false, NT, false>(buf, tid);
  __syncthreads();
  pass_a_fwd<M, true, NT>(buf, tid);
  __syncthreads();
}

// Inverse transform after the column pass B (storage order in, natural out, x M^2).
template <int M, int NT>
__device__ __forceinline__ void fft2_inv_after_col_b(float2* buf, int tid) {
  pass_a_inv<M, true, NT>(buf, tid);
  __syncthreads();
  pass_b<M, false, NT, true>(buf, tid);
  __syncthreads();
  pass_a_inv<M, false, NT>(buf, tid);
  __syncthreads();
}

}  // namespace emg

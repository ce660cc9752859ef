// FP64 reductions of the reconstruction quality on the GPU.
//
// Blind ptychography recovers (z, Q) only up to the scaling (c z, Q / c),
// c complex and non-zero: the exit waves Q . P_k z, and with them the data of
// Sec. 2.1, do not change.  A reconstruction is therefore compared with a
// reference after the best c over a region of the object (the pixels the
// scan illuminates well):
//
//   c = <z, z_ref> / <z, z>        (sums over the region; <a, b> = sum conj(a) b)
//   object error = ||c z - z_ref|| / ||z_ref||            (over the region)
//   probe error  = ||Q / c - Q_ref|| / ||Q_ref||          (whole probe)
//   phase RMS    = sqrt(mean over the region of arg(c z conj(z_ref))^2)
//
// and the region is { p : sum_k |Q_ref(p - o_k)|^2 >= frac * max }, the summed
// illumination of the scan (the paper's figures compare reconstructions over
// the scanned field, Sec. 4.1).
//
// Every sum is taken in FP64.  Each kernel uses a fixed grid and a fixed
// reduction tree, and the partial sums are added in block order, so results
// are bitwise repeatable.  The illumination of a pixel is summed over the
// positions in index order, as a sequential loop would.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/emagpie.h"

namespace emg {
namespace {

constexpr int kMetThreads = 256;
constexpr int kMetBlocks = 304;  // 2 per SM on 152 SMs; fixed, so the sums are repeatable
constexpr int kPosChunk = 512;   // positions staged in shared memory at a time

struct D2 {
  double x, y;
};

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int s = kMetThreads / 2; s > 0; s >>= 1) {
    if (tid < s) sh[tid] += sh[tid + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Partial sums over the region: |z|^2, conj(z) z_ref (re, im), |z_ref|^2, count.
__global__ void __launch_bounds__(kMetThreads) k_align_pass1(const float2* __restrict__ z,
                                                             const float2* __restrict__ zr,
                                                             const uint8_t* __restrict__ region, size_t n,
                                                             double* __restrict__ part) {
  __shared__ double sh[kMetThreads];
  double zz = 0.0, cr = 0.0, ci = 0.0, rr = 0.0, cnt = 0.0;
  for (size_t i = (size_t)blockIdx.x * kMetThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kMetThreads) {
    if (region && !region[i]) continue;
    const float2 a = z[i], b = zr[i];
    const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
    zz += ax * ax + ay * ay;
    cr += ax * bx + ay * by;  // conj(a) b
    ci += ax * by - ay * bx;
    rr += bx * bx + by * by;
    cnt += 1.0;
  }
  double* out = part + (size_t)blockIdx.x * 5;
  const double v[5] = {zz, cr, ci, rr, cnt};
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const double s = block_sum_d(v[j], sh);
    if (threadIdx.x == 0) out[j] = s;
  }
}

// Sums the per-block partials in block order; with `finish` = 0 it also forms
// c = <z, z_ref> / <z, z> into res[0..1] (res[2] = ||z_ref||^2, res[3] = count).
__global__ void k_align_final1(const double* __restrict__ part, int blocks, double* __restrict__ res) {
  if (threadIdx.x != 0) return;
  double s[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < blocks; ++b)
    for (int j = 0; j < 5; ++j) s[j] += part[(size_t)b * 5 + j];
  res[0] = s[0] > 0.0 ? s[1] / s[0] : 0.0;
  res[1] = s[0] > 0.0 ? s[2] / s[0] : 0.0;
  res[2] = s[3];
  res[3] = s[4];
}

// Partial sums: |c z - z_ref|^2 and arg(c z conj(z_ref))^2 over the region,
// and (blocks covering the probe) |Q / c - Q_ref|^2, |Q_ref|^2.
__global__ void __launch_bounds__(kMetThreads) k_align_pass2(const float2* __restrict__ z,
                                                             const float2* __restrict__ zr,
                                                             const uint8_t* __restrict__ region, size_t n,
                                                             const float2* __restrict__ q,
                                                             const float2* __restrict__ qr, size_t nq,
                                                             const double* __restrict__ res,
                                                             double* __restrict__ part) {
  __shared__ double sh[kMetThreads];
  const double c_x = res[0], c_y = res[1];
  double e_obj = 0.0, e_ph = 0.0, e_q = 0.0, q_rr = 0.0;
  const size_t stride = (size_t)gridDim.x * kMetThreads;
  for (size_t i = (size_t)blockIdx.x * kMetThreads + threadIdx.x; i < n; i += stride) {
    if (region && !region[i]) continue;
    const float2 a = z[i], b = zr[i];
    const double wx = c_x * a.x - c_y * a.y, wy = c_x * a.y + c_y * a.x;  // c z
    const double dx = wx - b.x, dy = wy - b.y;
    e_obj += dx * dx + dy * dy;
    const double px = wx * b.x + wy * b.y, py = wy * b.x - wx * b.y;   // c z conj(z_ref)
    const double ph = atan2(py, px);
    e_ph += ph * ph;
  }
  const double cc = c_x * c_x + c_y * c_y;
  for (size_t i = (size_t)blockIdx.x * kMetThreads + threadIdx.x; i < nq; i += stride) {
    const float2 a = q[i], b = qr[i];
    // Q / c = Q conj(c) / |c|^2
    const double wx = cc > 0.0 ? (a.x * c_x + a.y * c_y) / cc : 0.0;
    const double wy = cc > 0.0 ? (a.y * c_x - a.x * c_y) / cc : 0.0;
    const double dx = wx - b.x, dy = wy - b.y;
    e_q += dx * dx + dy * dy;
    q_rr += (double)b.x * b.x + (double)b.y * b.y;
  }
  double* out = part + (size_t)blockIdx.x * 4;
  const double v[4] = {e_obj, e_ph, e_q, q_rr};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double s = block_sum_d(v[j], sh);
    if (threadIdx.x == 0) out[j] = s;
  }
}

__global__ void k_align_final2(const double* __restrict__ part, int blocks, double* __restrict__ res) {
  if (threadIdx.x != 0) return;
  double s[4] = {0, 0, 0, 0};
  for (int b = 0; b < blocks; ++b)
    for (int j = 0; j < 4; ++j) s[j] += part[(size_t)b * 4 + j];
  const double rr = res[2], cnt = res[3];
  res[4] = rr > 0.0 ? sqrt(s[0] / rr) : 0.0;
  res[5] = s[3] > 0.0 ? sqrt(s[2] / s[3]) : 0.0;
  res[6] = cnt > 0.0 ? sqrt(s[1] / cnt) : 0.0;
}

// Summed illumination of each object pixel, positions in index order, and
// the largest value per block.
__global__ void __launch_bounds__(kMetThreads) k_illumination(const float2* __restrict__ qr, int m,
                                                              const int32_t* __restrict__ pos, int n_pos,
                                                              int n_rows, int n_cols, double* __restrict__ illum,
                                                              double* __restrict__ part_max) {
  __shared__ int2 sp[kPosChunk];
  __shared__ double sh[kMetThreads];
  const size_t n = (size_t)n_rows * n_cols;
  double mx = 0.0;
  // every block walks the same number of rounds, so the barriers stay uniform
  const size_t stride = (size_t)gridDim.x * kMetThreads;
  const size_t rounds = (n + stride - 1) / stride;
  for (size_t rd = 0; rd < rounds; ++rd) {
    const size_t i = rd * stride + (size_t)blockIdx.x * kMetThreads + threadIdx.x;
    const bool live = i < n;
    const int r = live ? (int)(i / n_cols) : 0, c = live ? (int)(i % n_cols) : 0;
    double s = 0.0;
    for (int k0 = 0; k0 < n_pos; k0 += kPosChunk) {
      const int cnt = min(kPosChunk, n_pos - k0);
      __syncthreads();
      for (int j = threadIdx.x; j < cnt; j += kMetThreads) sp[j] = make_int2(pos[2 * (k0 + j)], pos[2 * (k0 + j) + 1]);
      __syncthreads();
      if (live) {
        for (int j = 0; j < cnt; ++j) {
          const int lr = r - sp[j].x, lc = c - sp[j].y;
          if ((unsigned)lr < (unsigned)m && (unsigned)lc < (unsigned)m) {
            const float2 q = qr[lr * m + lc];
            s += (double)q.x * q.x + (double)q.y * q.y;
          }
        }
      }
    }
    if (live) {
      illum[i] = s;
      mx = fmax(mx, s);
    }
  }
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int s = kMetThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part_max[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kMetThreads) k_region_mask(const double* __restrict__ illum, size_t n,
                                                             const double* __restrict__ part_max, int blocks,
                                                             double frac, uint8_t* __restrict__ region) {
  __shared__ double thr;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int b = 0; b < blocks; ++b) mx = fmax(mx, part_max[b]);
    thr = frac * mx;
  }
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * kMetThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kMetThreads)
    region[i] = illum[i] >= thr ? 1 : 0;
}

}  // namespace
}  // namespace emg

extern "C" emg_status emg_aligned_errors(const float* object, const float* object_ref, int32_t n_rows,
                                         int32_t n_cols, const float* probe, const float* probe_ref, int32_t m,
                                         const uint8_t* region, double* out, emg_stream_t stream) {
  using namespace emg;
  if (!object || !object_ref || !probe || !probe_ref || !out || n_rows < 1 || n_cols < 1 || m < 1)
    return EMG_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)n_rows * n_cols, nq = (size_t)m * m;
  double* scratch = nullptr;  // 5 + 4 partials per block, then 7 results
  const size_t words = (size_t)kMetBlocks * 9 + 8;
  if (cudaMalloc(&scratch, words * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return EMG_ENOMEM;
  }
  double* p1 = scratch;
  double* p2 = scratch + (size_t)kMetBlocks * 5;
  double* res = scratch + (size_t)kMetBlocks * 9;
  double host[7];
  cudaError_t e = cudaSuccess;
  k_align_pass1<<<kMetBlocks, kMetThreads, 0, s>>>((const float2*)object, (const float2*)object_ref, region, n, p1);
  if ((e = cudaGetLastError()) == cudaSuccess) {
    k_align_final1<<<1, 32, 0, s>>>(p1, kMetBlocks, res);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_align_pass2<<<kMetBlocks, kMetThreads, 0, s>>>((const float2*)object, (const float2*)object_ref, region, n,
                                                     (const float2*)probe, (const float2*)probe_ref, nq, res, p2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_align_final2<<<1, 32, 0, s>>>(p2, kMetBlocks, res);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(scratch);
  if (e != cudaSuccess) return EMG_ECUDA;
  out[0] = host[0];  // c (re, im)
  out[1] = host[1];
  out[2] = host[4];  // object relative error
  out[3] = host[5];  // probe relative error
  out[4] = host[6];  // RMS phase difference
  return EMG_OK;
}

extern "C" emg_status emg_illuminated_region(const float* probe_ref, int32_t m, const int32_t* pos, int32_t n_pos,
                                             int32_t n_rows, int32_t n_cols, double frac, uint8_t* region,
                                             emg_stream_t stream) {
  using namespace emg;
  if (!probe_ref || !pos || !region || m < 1 || n_pos < 1 || n_rows < 1 || n_cols < 1 || !(frac >= 0.0) ||
      !isfinite(frac))
    return EMG_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)n_rows * n_cols;
  double* scratch = nullptr;
  if (cudaMalloc(&scratch, (n + kMetBlocks) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return EMG_ENOMEM;
  }
  k_illumination<<<kMetBlocks, kMetThreads, 0, s>>>((const float2*)probe_ref, m, pos, n_pos, n_rows, n_cols,
                                                    scratch, scratch + n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_region_mask<<<kMetBlocks, kMetThreads, 0, s>>>(scratch, n, scratch + n, kMetBlocks, frac, region);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(scratch);
  return e == cudaSuccess ? EMG_OK : EMG_ECUDA;
}

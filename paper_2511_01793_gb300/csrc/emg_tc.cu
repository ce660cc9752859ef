// Batched 2-D DFT on the fifth-generation tensor cores (tcgen05) of sm_103a:
// BF16 operands, each split into a high and a low part, with the three leading
// products accumulated in FP32 (x y ~ xh yh + xh yl + xl yh); the precision
// variant of the FFT pair a2 / a4 of the eMAGPIE step (Sec. 2.1, Eq. for R_k).
//
// A 2-D DFT of an m x m tile is two 1-D passes.  Each pass is one GEMM over all
// rows of all tiles of a batch: a row x (m complex values stored as interleaved
// (re, im) bf16 pairs, K = 2m) times the 2m x 2m real matrix of the complex map
// x -> x G, G = F or conj(F), F[c][v] = exp(-2 pi i c v / m).  The output row is
// interleaved the same way, so each thread of the epilogue holds (re, im) pairs
// and can write them transposed per tile (the next pass then transforms the
// other axis), replace the modulus (a3) or store FP32.
//
// Persistent kernel, one CTA per SM, each looping over 128 x 256 output tiles
// (consecutive CTAs take the two 128-row halves of a 256-row block, so the
// block's B, the DFT matrix, is read from L2 by both at about the same time).
// Warp 0 streams A and B chunks of 32 bf16 along K through a four-stage
// shared-memory ring with plain per-CTA TMA loads (64-byte swizzle); warp 1 owns all 512 columns of tensor memory
// as two 256-column accumulators and issues tcgen05.mma from one lane; warps
// 2-9 drain an accumulator with tcgen05.ld (two warps per lane quadrant, each
// half of the columns) and run the epilogue while the MMAs of the next tile
// fill the other accumulator.  Every mbarrier wait is bounded in
// time: on expiry the kernel records an error flag, waits (bounded) for what it
// issued, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <new>

#include "emg_internal.h"

namespace emg {
namespace {

constexpr int kBM = 128;                            // accumulator rows = TMEM lanes
constexpr int kBN = 256;                            // accumulator columns (FP32)
constexpr int kBK = 32;                             // bf16 per 64-byte swizzled row
constexpr int kStages = 4;
constexpr int kSwizzleBytes = kBK * 2;              // one swizzle atom row
constexpr int kTileA = kBM * kBK * 2;               // 8 KB
constexpr int kTileB = kBN * kBK * 2;               // 16 KB
constexpr int kStageBytes = 2 * kTileA + 2 * kTileB;  // A hi, A lo, B hi, B lo
constexpr int kTcSmem = kStages * kStageBytes + 1024;  // + alignment slack
constexpr int kEpiWarps = 8;                        // two per TMEM lane quadrant, each half the columns
constexpr int kTcThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kTmemCols = 2 * kBN;             // two accumulators
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per wait

// tcgen05.mma instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(addr), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the phase of `bar` with the given parity to complete; gives up
// after kWaitNs or as soon as *abort is set by another role of the CTA.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* abort) {
  const uint32_t addr = smem_u32(bar);
  if (mbar_try(addr, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (;;) {
    if (mbar_try(addr, parity)) return true;
    if (*abort || gtimer() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with 64-byte swizzling:
// start address >> 4 (bits 0-13), leading byte offset (unused for this layout,
// bits 16-29), stride byte offset 512 B = 8 rows x 64 B (bits 32-45), the
// descriptor version 1 (bits 46-48), base offset 0 (tiles are 1024-byte
// aligned), swizzle mode 4 = 64 B (bits 61-63).
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8 * kSwizzleBytes) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of the warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive floats (64-byte aligned) through the read-only path.
__device__ __forceinline__ void load16(const float* p, float (&v)[16]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float4 t4 = __ldg(q + j);
    v[4 * j] = t4.x;
    v[4 * j + 1] = t4.y;
    v[4 * j + 2] = t4.z;
    v[4 * j + 3] = t4.w;
  }
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// (re, im) -> high and low bf16 pairs: hi = bf16(x), lo = bf16(x - hi).
__device__ __forceinline__ void split_pair(float re, float im, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat16 hr = __float2bfloat16_rn(re), hm = __float2bfloat16_rn(im);
  hi = (uint32_t)__bfloat16_as_ushort(hr) | ((uint32_t)__bfloat16_as_ushort(hm) << 16);
  lo = bf16_bits(re - __bfloat162float(hr)) | (bf16_bits(im - __bfloat162float(hm)) << 16);
}

struct TcPassArgs {
  int m;                    // transform size; K = 2m, each tile has m rows
  int tiles_n, m_tiles;     // output tiles along N and along M
  uint32_t* out_hi;         // split outputs, bf16 pairs [rows][m]
  uint32_t* out_lo;
  float2* out_f32;          // FP32 outputs [rows][m]
  float scale;              // FP32 outputs: multiplier; modulus mode: 1/m^2 folded into Psi'
  const float* amp_t;       // modulus mode: a_k transposed, [N][m][m], a_k^T[v][u] = a_k[u][v]
  const int32_t* order;     // modulus mode: position of tile kb
  double* partial;          // modulus mode: sum (|Psi| - a)^2 per output tile and epilogue warp
  int* err;                 // set to 1 when a bounded wait gives up
};

// Epilogue modes.
enum { kEpiSplitT = 0, kEpiModulus = 1, kEpiF32 = 2, kEpiF32T = 3 };

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int EPI>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_dft(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
             const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
             const TcPassArgs a) {
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kStages];   // stage loaded (TMA bytes arrived)
  __shared__ __align__(8) uint64_t empty_bar[kStages];  // stage consumed by the MMAs
  __shared__ __align__(8) uint64_t accf_bar[2];         // accumulator complete
  __shared__ __align__(8) uint64_t acce_bar[2];         // accumulator drained by the epilogue warps
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t tiles_s = (raw + 1023u) & ~1023u;
  const int KC = 2 * a.m / kBK;

  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], kEpiWarps);
    }
    mbar_init(&drain_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // visible to the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();  // barriers initialised and the TMEM address published
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  // CTA pairs (2c, 2c + 1) take the two 128-row halves of the same output
  // block, so both read that block's B rows from L2 at about the same time.
  const int rank = (int)(blockIdx.x & 1), n_cl = (int)(gridDim.x >> 1), cl_id = (int)(blockIdx.x >> 1);
  const int pairs = ((a.m_tiles + 1) >> 1) * a.tiles_n;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;  // chunks issued so far (the ring position runs on across tiles)
      for (int pr = cl_id; pr < pairs && !abort_sh; pr += n_cl) {
        const int m_tile = 2 * (pr / a.tiles_n) + rank, n_tile = pr % a.tiles_n;
        for (int kc = 0; kc < KC; ++kc, ++it) {
          const uint32_t s = it % kStages;
          if (it >= kStages && !mbar_wait(&empty_bar[s], ((it / kStages) + 1) & 1, &abort_sh)) {
            abort_sh = 1;
            atomicExch(a.err, 1);
            break;
          }
          const uint32_t st = tiles_s + s * kStageBytes;
          mbar_expect_tx(&full_bar[s], kStageBytes);
          tma_load_2d(st, &mAh, &full_bar[s], kc * kBK, m_tile * kBM);
          tma_load_2d(st + kTileA, &mAl, &full_bar[s], kc * kBK, m_tile * kBM);
          // the block's B rows, in two boxes of kBN / 2 rows
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t bo = (uint32_t)h * (kTileB / 2);
            tma_load_2d(st + 2 * kTileA + bo, &mBh, &full_bar[s], kc * kBK, n_tile * kBN + h * (kBN / 2));
            tma_load_2d(st + 2 * kTileA + kTileB + bo, &mBl, &full_bar[s], kc * kBK, n_tile * kBN + h * (kBN / 2));
          }
        }
      }
      if (abort_sh) {  // let the copies already issued land before the CTA exits
        const volatile int never = 0;
        for (uint32_t j = it > kStages ? it - kStages : 0; j < it; ++j)
          mbar_wait(&full_bar[j % kStages], (j / kStages) & 1, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      uint32_t it = 0;
      int local = 0;
      for (int pr = cl_id; pr < pairs && ok; pr += n_cl, ++local) {
        const int buf = local & 1;
        if (local >= 2 && !mbar_wait(&acce_bar[buf], ((local >> 1) + 1) & 1, &abort_sh)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * kBN);
        for (int kc = 0; kc < KC; ++kc, ++it) {
          const uint32_t s = it % kStages;
          if (!mbar_wait(&full_bar[s], (it / kStages) & 1, &abort_sh)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = tiles_s + s * kStageBytes;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint64_t ah = sw_desc(st + kk * 32);
            const uint64_t al = sw_desc(st + kTileA + kk * 32);
            const uint64_t bh = sw_desc(st + 2 * kTileA + kk * 32);
            const uint64_t bl = sw_desc(st + 2 * kTileA + kTileB + kk * 32);
            umma_bf16(d, ah, bh, (kc | kk) != 0);
            umma_bf16(d, ah, bl, 1);
            umma_bf16(d, al, bh, 1);
          }
          umma_commit(&empty_bar[s]);  // the stage is free once these MMAs have read it
        }
        if (ok) umma_commit(&accf_bar[buf]);
      }
      if (!ok) {
        abort_sh = 1;
        atomicExch(a.err, 1);
        umma_commit(&drain_bar);  // every MMA issued so far completes before the TMEM is freed
        const volatile int never = 0;
        mbar_wait(&drain_bar, 0, &never);
      }
    }
  } else {
    const int q = warp & 3;              // this warp may access TMEM lanes 32 q .. 32 q + 31
    const int ew = warp - 2;             // epilogue warp 0 .. 7
    const int c_lo = (ew >> 2) * (kBN / 2);  // its half of the accumulator columns
    const int m = a.m;
    int local = 0;
    for (int pr = cl_id; pr < pairs; pr += n_cl, ++local) {
      const int buf = local & 1;
      const int m_tile = 2 * (pr / a.tiles_n) + rank, n_tile = pr % a.tiles_n;
      const int t = m_tile * a.tiles_n + n_tile;
      const bool real = m_tile < a.m_tiles;  // the second half of the last block may lie past the rows
      const int gr = m_tile * kBM + q * 32 + lane;  // global row
      const int kb = gr / m, r = gr % m;
      // modulus replacement: the first chunk's amplitudes are fetched while the MMAs still run
      float am_next[16];
      const float* amp_row = nullptr;
      if constexpr (EPI == kEpiModulus) {
        if (real) {
          amp_row = a.amp_t + ((size_t)a.order[kb] * m + r) * m;
          load16(amp_row + ((n_tile * kBN + c_lo) >> 1), am_next);
        }
      }
      const bool got = mbar_wait(&accf_bar[buf], (local >> 1) & 1, &abort_sh);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0) {
          abort_sh = 1;
          atomicExch(a.err, 1);
        }
        break;
      }
      tc_fence_after();
      const uint32_t tb = tmem + (uint32_t)(buf * kBN) + ((uint32_t)(q * 32) << 16);
      float acc = 0.f;
#pragma unroll 1
      for (int c0 = c_lo; c0 < c_lo + kBN / 2; c0 += 32) {
        float v[32];
        __syncwarp();
        tmem_ld32(tb + (uint32_t)c0, v);
        if (!real) continue;
        const int u0 = (n_tile * kBN + c0) >> 1;  // first complex column of the chunk
        if constexpr (EPI == kEpiSplitT) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            uint32_t hi, lo;
            split_pair(v[2 * j], v[2 * j + 1], hi, lo);
            const size_t o = ((size_t)kb * m + u0 + j) * m + r;
            a.out_hi[o] = hi;
            a.out_lo[o] = lo;
          }
        } else if constexpr (EPI == kEpiModulus) {
          float am[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) am[j] = am_next[j];
          if (c0 + 32 < c_lo + kBN / 2) load16(amp_row + u0 + 16, am_next);  // the next chunk's, in flight
          uint32_t hi[16], lo[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float re = v[2 * j], im = v[2 * j + 1];
            const float p2 = re * re + im * im;
            if (p2 > 0.f) {
              const float inv = rsqrtf(p2);
              const float dm = fmaf(p2, inv, -am[j]);
              acc = fmaf(dm, dm, acc);
              const float f = am[j] * inv * a.scale;
              re *= f;
              im *= f;
            } else {
              acc = fmaf(am[j], am[j], acc);
              re = am[j] * a.scale;
              im = 0.f;
            }
            split_pair(re, im, hi[j], lo[j]);
          }
          uint4* oh = reinterpret_cast<uint4*>(a.out_hi + (size_t)gr * m + u0);
          uint4* ol = reinterpret_cast<uint4*>(a.out_lo + (size_t)gr * m + u0);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            oh[j] = make_uint4(hi[4 * j], hi[4 * j + 1], hi[4 * j + 2], hi[4 * j + 3]);
            ol[j] = make_uint4(lo[4 * j], lo[4 * j + 1], lo[4 * j + 2], lo[4 * j + 3]);
          }
        } else if constexpr (EPI == kEpiF32) {
          float4* o = reinterpret_cast<float4*>(a.out_f32 + (size_t)gr * m + u0);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            o[j] = make_float4(v[4 * j] * a.scale, v[4 * j + 1] * a.scale, v[4 * j + 2] * a.scale,
                               v[4 * j + 3] * a.scale);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            a.out_f32[((size_t)kb * m + u0 + j) * m + r] = make_float2(v[2 * j] * a.scale, v[2 * j + 1] * a.scale);
        }
      }
      // the accumulator is free for the tile after next once every epilogue warp has read it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce_bar[buf]);
      if constexpr (EPI == kEpiModulus) {
        double dsum = (double)acc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, off);
        if (lane == 0 && real) a.partial[(size_t)t * kEpiWarps + ew] = dsum;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Complex64 tiles -> high / low bf16 pairs (same order).
__global__ void __launch_bounds__(256) k_tc_split(const float2* __restrict__ in, uint32_t* __restrict__ hi,
                                                  uint32_t* __restrict__ lo, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 x = in[i];
    uint32_t h, l;
    split_pair(x.x, x.y, h, l);
    hi[i] = h;
    lo[i] = l;
  }
}

// a1 for the tensor-core path: psi_k = Q . P_k z for the b positions of a
// minibatch (zero outside the object), split into high / low bf16 pairs,
// rows (kb, r) of m pairs.
__global__ void __launch_bounds__(256) k_tc_psi(const float2* __restrict__ object, const float2* __restrict__ probe,
                                                const int32_t* __restrict__ pos, const int32_t* __restrict__ order,
                                                int n_rows, int n_cols, int m, int b, uint32_t* __restrict__ hi,
                                                uint32_t* __restrict__ lo) {
  const size_t mm = (size_t)m * m, n = (size_t)b * mm;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int kb = (int)(i / mm), p = (int)(i % mm), r = p / m, c = p % m;
    const int k = order[kb];
    const int orow = pos[2 * k] + r, ocol = pos[2 * k + 1] + c;
    float2 z = make_float2(0.f, 0.f);
    if (orow >= 0 && orow < n_rows && ocol >= 0 && ocol < n_cols) z = object[(size_t)orow * n_cols + ocol];
    const float2 q = probe[p];
    uint32_t h, l;
    split_pair(q.x * z.x - q.y * z.y, q.x * z.y + q.y * z.x, h, l);
    hi[i] = h;
    lo[i] = l;
  }
}

// a_k^T[v][u] = sqrt(max(d_k[u][v], 0)).
__global__ void __launch_bounds__(256) k_tc_amp(const float* __restrict__ d, float* __restrict__ amp_t, int m,
                                                size_t n) {
  const size_t mm = (size_t)m * m;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t k = i / mm;
    const int p = (int)(i % mm), v = p / m, u = p % m;
    amp_t[i] = sqrtf(fmaxf(d[k * mm + (size_t)u * m + v], 0.f));
  }
}

// Exercises the give-up path of the bounded wait: one thread waits on an
// mbarrier that nothing arrives on, exactly as the roles of k_tc_dft wait, and
// records the expiry in *err.  No copy or MMA is in flight, so nothing else
// needs draining.
__global__ void k_wait_selftest(int* err) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, &abort_flag)) *err = 1;
}

// ---------------------------------------------------------------------------
// Host side

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_tc_mu;
EncodeTiledFn g_encode = nullptr;

cudaError_t get_encoder(EncodeTiledFn* out) {
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (!g_encode) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<EncodeTiledFn>(p);
  }
  *out = g_encode;
  return cudaSuccess;
}

// 2-D bf16 tensor of `rows` rows of `inner` elements, boxes of kBK x box_rows, 64-byte swizzle.
cudaError_t make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  EncodeTiledFn enc = nullptr;
  cudaError_t e = get_encoder(&enc);
  if (e != cudaSuccess) return e;
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {inner * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

uint16_t host_bf16(double x) {  // round to nearest even (finite inputs)
  const float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

double host_bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

// The 2m x 2m real matrices of x -> x F and x -> x conj(F), stored K-major
// (row n = output component, column k = input component), high and low parts.
struct TcTables {
  uint16_t* d = nullptr;  // [4][2m][2m]: fwd hi, fwd lo, inv hi, inv lo
  CUtensorMap map[4];
};

TcTables g_tables[64][2];  // per device, m = 128 / 256

cudaError_t get_tables(int m, const TcTables** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  TcTables& t = g_tables[dev][m == 256 ? 1 : 0];
  {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    if (t.d) {
      *out = &t;
      return cudaSuccess;
    }
  }
  const int K = 2 * m;
  const size_t per = (size_t)K * K;
  uint16_t* h = (uint16_t*)malloc(4 * per * sizeof(uint16_t));
  if (!h) return cudaErrorMemoryAllocation;
  for (int inv = 0; inv < 2; ++inv) {
    uint16_t* th = h + (size_t)(2 * inv) * per;
    uint16_t* tl = th + per;
    for (int v = 0; v < m; ++v)
      for (int c = 0; c < m; ++c) {
        const int t_ = (int)(((long long)c * v) % m);
        double gr = cos(2.0 * M_PI * t_ / m), gi = -sin(2.0 * M_PI * t_ / m);
        if (fabs(gr) < 1e-15) gr = 0.0;
        if (fabs(gi) < 1e-15) gi = 0.0;
        if (inv) gi = -gi;
        // out re (row 2v): re x_c * gr - im x_c * gi; out im (row 2v+1): re x_c * gi + im x_c * gr
        const double val[4] = {gr, -gi, gi, gr};
        const size_t idx[4] = {(size_t)(2 * v) * K + 2 * c, (size_t)(2 * v) * K + 2 * c + 1,
                               (size_t)(2 * v + 1) * K + 2 * c, (size_t)(2 * v + 1) * K + 2 * c + 1};
        for (int j = 0; j < 4; ++j) {
          const uint16_t hv = host_bf16(val[j]);
          th[idx[j]] = hv;
          tl[idx[j]] = host_bf16(val[j] - host_bf16_value(hv));
        }
      }
  }
  uint16_t* d = nullptr;
  e = cudaMalloc(&d, 4 * per * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMemcpy(d, h, 4 * per * sizeof(uint16_t), cudaMemcpyHostToDevice);
  free(h);
  TcTables nt;
  for (int j = 0; e == cudaSuccess && j < 4; ++j) e = make_map(&nt.map[j], d + j * per, K, K, kBN / 2);
  if (e != cudaSuccess) {
    if (d) cudaFree(d);
    return e;
  }
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (t.d) {  // another thread won
    cudaFree(d);
  } else {
    nt.d = d;
    t = nt;
  }
  *out = &t;
  return cudaSuccess;
}

template <int EPI>
cudaError_t launch_pass(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                        int rows, int sms, TcPassArgs a, cudaStream_t s) {
  a.tiles_n = 2 * a.m / kBN;
  a.m_tiles = rows / kBM;
  const int pairs = ((a.m_tiles + 1) / 2) * a.tiles_n;
  const int npairs = pairs < sms / 2 ? pairs : sms / 2;
  k_tc_dft<EPI><<<2 * npairs, kTcThreads, kTcSmem, s>>>(ah, al, bh, bl, a);
  return cudaGetLastError();
}

cudaError_t set_tc_attrs() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_tc_dft<kEpiSplitT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_tc_dft<kEpiModulus>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_tc_dft<kEpiF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem)) !=
      cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_tc_dft<kEpiF32T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
}

int grid_for(size_t n) {
  size_t blocks = (n + 255) / 256;
  return (int)(blocks > 152 * 32 ? 152 * 32 : blocks);
}

}  // namespace

struct TcWork {
  int m = 0, cap = 0;       // transform size, tiles of capacity
  uint32_t* buf[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [ping-pong][hi, lo]: bf16 pairs [cap m][m]
  CUtensorMap amap[2][2];   // the two buffers as A operands
  const TcTables* tables = nullptr;
  int* d_err = nullptr;
  int sms = 0;              // persistent grid: one CTA per SM
};

bool tc_supported(int m) { return m == 128 || m == 256; }

cudaError_t tc_work_create(TcWork** out, int m, int cap) {
  *out = nullptr;
  if (!tc_supported(m) || cap < 1) return cudaErrorInvalidValue;
  static std::once_flag attrs_once;
  static cudaError_t attrs_err = cudaSuccess;
  std::call_once(attrs_once, [] { attrs_err = set_tc_attrs(); });
  if (attrs_err != cudaSuccess) return attrs_err;
  TcWork* w = new (std::nothrow) TcWork();
  if (!w) return cudaErrorMemoryAllocation;
  w->m = m;
  w->cap = cap;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&w->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || w->sms < 1) {
    delete w;
    return cudaErrorInvalidDevice;
  }
  const size_t pairs = (size_t)cap * m * m;
  cudaError_t e = get_tables(m, &w->tables);
  for (int i = 0; e == cudaSuccess && i < 2; ++i)
    for (int j = 0; e == cudaSuccess && j < 2; ++j) {
      e = cudaMalloc(&w->buf[i][j], pairs * sizeof(uint32_t));
      if (e == cudaSuccess) e = make_map(&w->amap[i][j], w->buf[i][j], 2 * (uint64_t)m, (uint64_t)cap * m, kBM);
    }
  if (e == cudaSuccess) e = cudaMalloc(&w->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(w->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    tc_work_destroy(w);
    return e;
  }
  *out = w;
  return cudaSuccess;
}

void tc_work_destroy(TcWork* w) {
  if (!w) return;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      if (w->buf[i][j]) cudaFree(w->buf[i][j]);
  if (w->d_err) cudaFree(w->d_err);
  delete w;
}

int* tc_error_flag(TcWork* w) { return w->d_err; }

int tc_tiles_per_position(int m) { return (m / kBM) * (2 * m / kBN) * kEpiWarps; }  // per epilogue warp

cudaError_t tc_dft2(TcWork* w, const float2* in, float2* out, int count, int inverse, cudaStream_t s) {
  if (count < 1 || count > w->cap) return cudaErrorInvalidValue;
  const int m = w->m, rows = count * m;
  const size_t n = (size_t)count * m * m;
  k_tc_split<<<grid_for(n), 256, 0, s>>>(in, w->buf[0][0], w->buf[0][1], n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const CUtensorMap* B = &w->tables->map[inverse ? 2 : 0];
  TcPassArgs a{};
  a.m = m;
  a.err = w->d_err;
  a.out_hi = w->buf[1][0];
  a.out_lo = w->buf[1][1];
  a.scale = 1.f;
  if ((e = launch_pass<kEpiSplitT>(w->amap[0][0], w->amap[0][1], B[0], B[1], rows, w->sms, a, s)) != cudaSuccess) return e;
  a.out_hi = a.out_lo = nullptr;
  a.out_f32 = out;
  a.scale = inverse ? 1.f / (float)(m * m) : 1.f;
  return launch_pass<kEpiF32T>(w->amap[1][0], w->amap[1][1], B[0], B[1], rows, w->sms, a, s);
}

cudaError_t tc_exit_waves(TcWork* w, const TcStepArgs& t, cudaStream_t s) {
  if (t.b < 1 || t.b > w->cap) return cudaErrorInvalidValue;
  const int m = w->m, rows = t.b * m;
  const size_t n = (size_t)t.b * m * m;
  k_tc_psi<<<grid_for(n), 256, 0, s>>>(t.object, t.probe, t.pos, t.order, t.n_rows, t.n_cols, m, t.b, w->buf[0][0],
                                       w->buf[0][1]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const CUtensorMap* F = &w->tables->map[0];
  const CUtensorMap* G = &w->tables->map[2];
  TcPassArgs a{};
  a.m = m;
  a.err = w->d_err;
  a.scale = 1.f;
  // a2, rows: psi -> (psi F)^T per tile
  a.out_hi = w->buf[1][0];
  a.out_lo = w->buf[1][1];
  if ((e = launch_pass<kEpiSplitT>(w->amap[0][0], w->amap[0][1], F[0], F[1], rows, w->sms, a, s)) != cudaSuccess) return e;
  // a2, columns, and a3: Psi^T, modulus replaced, 1/m^2 folded in
  a.out_hi = w->buf[0][0];
  a.out_lo = w->buf[0][1];
  a.amp_t = t.amp_t;
  a.order = t.order;
  a.partial = t.partial;
  a.scale = 1.f / (float)(m * m);
  if ((e = launch_pass<kEpiModulus>(w->amap[1][0], w->amap[1][1], F[0], F[1], rows, w->sms, a, s)) != cudaSuccess) return e;
  // a4: inverse over the frequency rows (transposed back), then over the columns
  a.amp_t = nullptr;
  a.order = nullptr;
  a.partial = nullptr;
  a.scale = 1.f;
  a.out_hi = w->buf[1][0];
  a.out_lo = w->buf[1][1];
  if ((e = launch_pass<kEpiSplitT>(w->amap[0][0], w->amap[0][1], G[0], G[1], rows, w->sms, a, s)) != cudaSuccess) return e;
  a.out_hi = a.out_lo = nullptr;
  a.out_f32 = t.R;
  return launch_pass<kEpiF32>(w->amap[1][0], w->amap[1][1], G[0], G[1], rows, w->sms, a, s);
}

cudaError_t launch_wait_selftest(int* err, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(err);
  return cudaGetLastError();
}

cudaError_t launch_tc_amp(const float* d, float* amp_t, int m, int n_pos, cudaStream_t s) {
  const size_t n = (size_t)n_pos * m * m;
  k_tc_amp<<<grid_for(n), 256, 0, s>>>(d, amp_t, m, n);
  return cudaGetLastError();
}

}  // namespace emg

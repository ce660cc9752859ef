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
#include <stdlib.h>
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

// (re, im) -> high and low bf16 pairs: hi = bf16(x), lo = bf16(x - hi), re in the
// low half of each word (one packed conversion per pair).
__device__ __forceinline__ uint32_t pack_bf16x2(float re, float im) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(re, im);
  return *reinterpret_cast<const uint32_t*>(&p);
}
__device__ __forceinline__ void split_pair(float re, float im, uint32_t& hi, uint32_t& lo) {
  hi = pack_bf16x2(re, im);
  lo = pack_bf16x2(re - __uint_as_float(hi << 16), im - __uint_as_float(hi & 0xFFFF0000u));
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
  int rows16;               // radix-16 pass: output row k stored at r16_perm(k)
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

// ---------------------------------------------------------------------------
// Radix-16 pass (m = 256): each 1-D DFT of length 256 = 16 x 16 as two 16-point
// DFT GEMMs with a twiddle multiply between them, both on chip:
//   n = 16 n1 + n2, k = k1 + 16 k2,
//   Y[n2][k1] = sum_n1 x[16 n1 + n2] W16^(n1 k1)            (stage 1)
//   X[k1 + 16 k2] = sum_n2 W16^(n2 k2) W256^(n2 k1) Y[n2][k1]  (stage 2)
// Rows hold their elements in digit-swapped order (logical index 16 n1 + n2 at
// position 16 n2 + n1), so the stage-1 input of each n2 is 32 contiguous bf16:
// one TMA box of 128 rows, exactly the A chunk of the dense pass.  Per block of
// 128 rows, warp 1 issues the stage-1 MMAs of all 16 n2 (N = 16 per half of the
// k1 range) into all 512 TMEM columns; the epilogue warps multiply by the
// twiddles, split into BF16 high and low parts and write the stage-2 operands
// (8 k1 at a time) into shared memory in the same 64-byte swizzled layout that
// TMA produces; warp 1 then issues the stage-2 MMAs (N = 32) into the columns
// just drained, and the epilogue warps write the outputs.  The same 32 x 32
// real matrix of the 16-point DFT serves both stages.  Every wait is bounded.
constexpr int kR16Stages = 4;
constexpr int kR16Tile = kBM * kBK * 2;                   // 8 KB: 128 rows x 32 bf16
constexpr int kR16StageBytes = 2 * kR16Tile;              // A hi, A lo
constexpr int kR16BBytes = 32 * kBK * 2;                  // 2 KB: the 32 x 32 matrix, hi or lo
constexpr int kR16A2Bytes = 8 * kR16Tile;                 // 64 KB: stage-2 operands of 8 k1, hi or lo
constexpr int kR16Smem = kR16Stages * kR16StageBytes + 2 * kR16BBytes + 2 * kR16A2Bytes + 1024;
// Chunks kR16XFirst .. kR16XFirst + 7 of a block are staged in the stage-2 operand
// area (free from the end of the previous block's stage-2 MMAs until the
// epilogue writes it), so that most of a block's loads are in flight while the
// previous block's outputs drain; the others go through the ring.
constexpr int kR16XChunks = 2 * kR16A2Bytes / kR16StageBytes;  // 8
constexpr int kR16XFirst = 4;
static_assert(kR16XFirst + kR16XChunks <= 16, "staged chunks within the 16 of a block");
constexpr uint32_t kIdescN16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(16 >> 3) << 17) |
                               ((uint32_t)(kBM >> 4) << 24);
constexpr uint32_t kIdescN32 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(32 >> 3) << 17) |
                               ((uint32_t)(kBM >> 4) << 24);

// W_256^j, j = 0..255, filled on the host in FP64 (once per device).
__constant__ float2 c_tw256[256];

__device__ __forceinline__ void umma_bf16_n(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 16 consecutive FP32 columns of the warp's 32 TMEM lanes; completes with tmem_ld_wait.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// Position of logical element n = 16 n1 + n2 in a digit-swapped row (an involution).
__host__ __device__ __forceinline__ int r16_perm(int n) { return ((n & 15) << 4) | (n >> 4); }
__device__ __forceinline__ bool r16_staged(int n2) { return n2 >= kR16XFirst && n2 < kR16XFirst + kR16XChunks; }

template <int EPI>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_fft16(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
               const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
               const TcPassArgs a, const int inverse) {
  static_assert(EPI != kEpiF32, "the radix-16 pass writes transposed outputs only");
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kR16Stages];   // stage-1 operands of one n2 landed
  __shared__ __align__(8) uint64_t empty_bar[kR16Stages];  // ... and consumed by their MMAs
  __shared__ __align__(8) uint64_t x_bar[kR16XChunks];      // chunks staged in the stage-2 operand area landed
  __shared__ __align__(8) uint64_t b_bar;                   // the DFT matrix landed
  __shared__ __align__(8) uint64_t d1_bar;                  // stage-1 accumulators complete
  __shared__ __align__(8) uint64_t a2_bar[2];               // stage-2 operands of a k1 half written
  __shared__ __align__(8) uint64_t s2_bar[2];               // stage-2 accumulators of a half complete
  __shared__ __align__(8) uint64_t acce_bar;                // all accumulators drained
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t ring = (raw + 1023u) & ~1023u;
  const uint32_t bsm = ring + kR16Stages * kR16StageBytes;  // B hi, then B lo
  const uint32_t a2h = bsm + 2 * kR16BBytes;                // 8 tiles of stage-2 A, hi
  const uint32_t a2l = a2h + kR16A2Bytes;                   // ... lo
  const int m = a.m;
  const int n_blocks = a.m_tiles;

  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < kR16Stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
#pragma unroll
    for (int s = 0; s < kR16XChunks; ++s) mbar_init(&x_bar[s], 1);
    mbar_init(&b_bar, 1);
    mbar_init(&d1_bar, 1);
    mbar_init(&a2_bar[0], kEpiWarps);
    mbar_init(&a2_bar[1], kEpiWarps);
    mbar_init(&s2_bar[0], 1);
    mbar_init(&s2_bar[1], 1);
    mbar_init(&acce_bar, kEpiWarps);
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
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      // the 16-point DFT matrix (32 x 32 real, K-major), once per CTA
      mbar_expect_tx(&b_bar, 2 * kR16BBytes);
      tma_load_2d(bsm, &mBh, &b_bar, 0, 0);
      tma_load_2d(bsm + kR16BBytes, &mBl, &b_bar, 0, 0);
      uint32_t it = 0;                // ring slots filled so far
      int x_local = -1, x_count = 0;  // block and count of the chunks last staged in the operand area
      int local = 0;
      for (int blk = blockIdx.x; blk < n_blocks && !abort_sh; blk += gridDim.x, ++local) {
        for (int n2 = 0; n2 < 16; ++n2) {
          uint32_t st;
          uint64_t* bar;
          if (r16_staged(n2)) {
            // the operand area is free once the previous block's stage-2 MMAs are complete
            if (n2 == kR16XFirst && local > 0 && !mbar_wait(&s2_bar[1], (local - 1) & 1, &abort_sh)) {
              abort_sh = 1;
              atomicExch(a.err, 1);
              break;
            }
            st = a2h + (uint32_t)(n2 - kR16XFirst) * kR16StageBytes;
            bar = &x_bar[n2 - kR16XFirst];
            if (x_local != local) x_count = 0;
            x_local = local;
            ++x_count;
          } else {
            const uint32_t s = it % kR16Stages;
            if (it >= kR16Stages && !mbar_wait(&empty_bar[s], ((it / kR16Stages) + 1) & 1, &abort_sh)) {
              abort_sh = 1;
              atomicExch(a.err, 1);
              break;
            }
            st = ring + s * kR16StageBytes;
            bar = &full_bar[s];
            ++it;
          }
          mbar_expect_tx(bar, kR16StageBytes);
          tma_load_2d(st, &mAh, bar, n2 * kBK, blk * kBM);
          tma_load_2d(st + kR16Tile, &mAl, bar, n2 * kBK, blk * kBM);
        }
      }
      if (abort_sh) {  // let the copies already issued land before the CTA exits
        const volatile int never = 0;
        mbar_wait(&b_bar, 0, &never);
        for (uint32_t j = it > kR16Stages ? it - kR16Stages : 0; j < it; ++j)
          mbar_wait(&full_bar[j % kR16Stages], (j / kR16Stages) & 1, &never);
        for (int j = 0; j < x_count; ++j) mbar_wait(&x_bar[j], x_local & 1, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(&b_bar, 0, &abort_sh);
      uint32_t it = 0;
      int local = 0;
      for (int blk = blockIdx.x; ok && blk < n_blocks; blk += gridDim.x, ++local) {
        if (local > 0 && !mbar_wait(&acce_bar, (local - 1) & 1, &abort_sh)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // stage 1: for each n2, a 16-point DFT of the 128 rows' n1 elements;
        // half h of the k1 range lands in columns h * 256 + n2 * 16
        for (int n2 = 0; n2 < 16; ++n2) {
          const bool staged = r16_staged(n2);
          const uint32_t s = it % kR16Stages;
          if (!mbar_wait(staged ? &x_bar[n2 - kR16XFirst] : &full_bar[s],
                         staged ? (uint32_t)(local & 1) : (it / kR16Stages) & 1, &abort_sh)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st =
              staged ? a2h + (uint32_t)(n2 - kR16XFirst) * kR16StageBytes : ring + s * kR16StageBytes;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t d = tmem + (uint32_t)(h * 256 + n2 * 16);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
              const uint64_t ah = sw_desc(st + kk * 32), al = sw_desc(st + kR16Tile + kk * 32);
              const uint64_t bh = sw_desc(bsm + h * 1024 + kk * 32);
              const uint64_t bl = sw_desc(bsm + kR16BBytes + h * 1024 + kk * 32);
              umma_bf16_n(d, ah, bh, kIdescN16, kk != 0);
              umma_bf16_n(d, ah, bl, kIdescN16, 1);
              umma_bf16_n(d, al, bh, kIdescN16, 1);
            }
          }
          if (!staged) {
            umma_commit(&empty_bar[s]);
            ++it;
          }
        }
        if (!ok) break;
        umma_commit(&d1_bar);
        // stage 2, one k1 half at a time: 16-point DFTs over n2 into columns h * 256 + j * 32
        for (int h = 0; h < 2; ++h) {
          if (!mbar_wait(&a2_bar[h], local & 1, &abort_sh)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll 1
          for (int j = 0; j < 8; ++j) {
            const uint32_t d = tmem + (uint32_t)(h * 256 + j * 32);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
              const uint64_t ah = sw_desc(a2h + j * kR16Tile + kk * 32), al = sw_desc(a2l + j * kR16Tile + kk * 32);
              const uint64_t bh = sw_desc(bsm + kk * 32), bl = sw_desc(bsm + kR16BBytes + kk * 32);
              umma_bf16_n(d, ah, bh, kIdescN32, kk != 0);
              umma_bf16_n(d, ah, bl, kIdescN32, 1);
              umma_bf16_n(d, al, bh, kIdescN32, 1);
            }
          }
          umma_commit(&s2_bar[h]);
        }
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
    const int q = warp & 3;            // TMEM lane quadrant of this warp
    const int ew = warp - 2;           // epilogue warp 0 .. 7
    const int hw = ew >> 2;            // which half of the n2 (stage 1) or of the k1 (stage 2) range
    const int t = q * 32 + lane;       // row within the block = TMEM lane
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    const float tsign = inverse ? -1.f : 1.f;
    int local = 0;
    bool alive = true;
    for (int blk = blockIdx.x; alive && blk < n_blocks; blk += gridDim.x, ++local) {
      const int grow = blk * kBM + t, kb = grow / m, sr = grow % m;  // stored row sr of tile kb
      bool got = mbar_wait(&d1_bar, local & 1, &abort_sh);
      if (!__all_sync(0xffffffffu, got)) {
        alive = false;
        break;
      }
      tc_fence_after();
      // stage-1 results -> twiddled, split stage-2 operands (row t; my 8 n2: chunks 2 hw, 2 hw + 1)
      for (int h = 0; h < 2; ++h) {
        if (h == 1) {  // the stage-2 operand buffer is free once the half-0 MMAs are done
          got = mbar_wait(&s2_bar[0], local & 1, &abort_sh);
          if (!__all_sync(0xffffffffu, got)) {
            alive = false;
            break;
          }
          tc_fence_after();
        }
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
          const int n2b = 8 * hw + 4 * g, c = n2b >> 2;
          uint32_t v[4][16];
#pragma unroll
          for (int i = 0; i < 4; ++i) tmem_ld16_issue(tl + (uint32_t)(h * 256 + (n2b + i) * 16), v[i]);
          tmem_ld_wait();
          const uint32_t off = (uint32_t)((t >> 3) * 512 + (t & 7) * 64 + ((c ^ ((t >> 1) & 3)) << 4));
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int k1 = 8 * h + j;
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float2 w = c_tw256[(n2b + i) * k1];
              const float re = __uint_as_float(v[i][2 * j]), im = __uint_as_float(v[i][2 * j + 1]);
              const float wi = tsign * w.y;
              split_pair(re * w.x - im * wi, re * wi + im * w.x, hi[i], lo[i]);
            }
            sts128(a2h + j * kR16Tile + off, hi[0], hi[1], hi[2], hi[3]);
            sts128(a2l + j * kR16Tile + off, lo[0], lo[1], lo[2], lo[3]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the MMAs read these operands
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&a2_bar[h]);  // one arrival per epilogue warp
      }
      if (!alive) break;
      // stage-2 results: X[k1 + 16 k2], my 4 k1 of each half
      float acc = 0.f;
      // modulus: the 16 amplitudes of the next (h, jj) step are loaded one step ahead
      const float* amp_tile = nullptr;
      float am[16], am_next[16];
      if constexpr (EPI == kEpiModulus) {
        amp_tile = a.amp_t + (size_t)a.order[kb] * m * m + sr;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          const int k = 4 * hw + 16 * k2;  // h = 0, jj = 0
          am_next[k2] = __ldg(amp_tile + (size_t)(a.rows16 ? r16_perm(k) : k) * m);
        }
      }
      for (int h = 0; h < 2; ++h) {
        got = mbar_wait(&s2_bar[h], local & 1, &abort_sh);
        if (!__all_sync(0xffffffffu, got)) {
          alive = false;
          break;
        }
        tc_fence_after();
#pragma unroll 1
        for (int jj = 0; jj < 4; ++jj) {
          const int j = 4 * hw + jj, k1 = 8 * h + j;
          float v[32];
          if constexpr (EPI == kEpiModulus) {
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) am[k2] = am_next[k2];
            const int step = 4 * h + jj + 1;  // the next step, if any
            if (step < 8) {
              const int k1n = 8 * (step >> 2) + 4 * hw + (step & 3);
#pragma unroll
              for (int k2 = 0; k2 < 16; ++k2) {
                const int k = k1n + 16 * k2;
                am_next[k2] = __ldg(amp_tile + (size_t)(a.rows16 ? r16_perm(k) : k) * m);
              }
            }
          }
          __syncwarp();
          tmem_ld32(tl + (uint32_t)(h * 256 + j * 32), v);
          // transposed outputs: frequency k = k1 + 16 k2 of stored input row sr goes to
          // position sr of output row k (r16_perm(k) with rows16); a warp writes 128 contiguous bytes
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            const int k = k1 + 16 * k2;
            const size_t o = ((size_t)kb * m + (a.rows16 ? r16_perm(k) : k)) * m + sr;
            float re = v[2 * k2], im = v[2 * k2 + 1];
            if constexpr (EPI == kEpiF32T) {
              a.out_f32[o] = make_float2(re * a.scale, im * a.scale);
            } else {
              if constexpr (EPI == kEpiModulus) {
                const float p2 = re * re + im * im;
                if (p2 > 0.f) {
                  const float inv = rsqrtf(p2);
                  const float dm = fmaf(p2, inv, -am[k2]);
                  acc = fmaf(dm, dm, acc);
                  const float f = am[k2] * inv * a.scale;
                  re *= f;
                  im *= f;
                } else {
                  acc = fmaf(am[k2], am[k2], acc);
                  re = am[k2] * a.scale;
                  im = 0.f;
                }
              }
              uint32_t hv, lv;
              split_pair(re, im, hv, lv);
              a.out_hi[o] = hv;
              a.out_lo[o] = lv;
            }
          }
        }
      }
      if (!alive) break;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce_bar);  // one arrival per epilogue warp
      if constexpr (EPI == kEpiModulus) {
        double dsum = (double)acc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, off);
        if (lane == 0) a.partial[(size_t)blk * kEpiWarps + ew] = dsum;
      }
    }
    if (!alive && lane == 0) {
      abort_sh = 1;
      atomicExch(a.err, 1);
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

// Complex64 -> high / low bf16 pairs, element by element.
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
    const float2 q = probe[r * m + c];
    uint32_t h, l;
    split_pair(q.x * z.x - q.y * z.y, q.x * z.y + q.y * z.x, h, l);
    hi[i] = h;
    lo[i] = l;
  }
}

// Radix-16 layout (m = 256): tiles with rows and elements digit-swapped.  Each
// block permutes kR16Rows rows at a time: they are read in natural order
// (coalesced, all loads of a thread in flight together), permuted in shared
// memory (padded by one word per 16 against bank conflicts) and written in
// stored order (coalesced).  With object == nullptr the rows come from `in`
// (tc_dft2); otherwise they are psi_k = Q . P_k z of minibatch slot kb.
constexpr int kR16Rows = 4;
__global__ void __launch_bounds__(256) k_tc_rows16(const float2* __restrict__ in, const float2* __restrict__ object,
                                                   const float2* __restrict__ probe, const int32_t* __restrict__ pos,
                                                   const int32_t* __restrict__ order, int n_rows, int n_cols,
                                                   int n_tiles, uint32_t* __restrict__ hi, uint32_t* __restrict__ lo) {
  constexpr int m = 256, R = kR16Rows;
  __shared__ uint32_t sh[R][2][m + m / 16];
  const int c = threadIdx.x;
  const int pc = r16_perm(c);
  for (int row0 = blockIdx.x * R; row0 < n_tiles * m; row0 += gridDim.x * R) {  // m is a multiple of R
    float2 x[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int row = row0 + i, kb = row / m, r = row % m;
      if (object == nullptr) {
        x[i] = in[(size_t)row * m + c];
      } else {
        const int k = order[kb];
        const int orow = pos[2 * k] + r, ocol = pos[2 * k + 1] + c;
        float2 z = make_float2(0.f, 0.f);
        if (orow >= 0 && orow < n_rows && ocol >= 0 && ocol < n_cols) z = object[(size_t)orow * n_cols + ocol];
        const float2 q = probe[r * m + c];
        x[i] = make_float2(q.x * z.x - q.y * z.y, q.x * z.y + q.y * z.x);
      }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
      uint32_t h, l;
      split_pair(x[i].x, x[i].y, h, l);
      sh[i][0][pc + (pc >> 4)] = h;
      sh[i][1][pc + (pc >> 4)] = l;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int row = row0 + i, kb = row / m, r = row % m;
      const size_t o = ((size_t)kb * m + r16_perm(r)) * m + c;
      hi[o] = sh[i][0][c + (c >> 4)];
      lo[o] = sh[i][1][c + (c >> 4)];
    }
    __syncthreads();
  }
}

// The amplitudes in the layout the dense modulus pass reads: a_k^T[v][u] = sqrt(max(d_k[u][v], 0)).
__global__ void __launch_bounds__(256) k_tc_amp(const float* __restrict__ d, float* __restrict__ amp_t, int m,
                                                size_t n) {
  const size_t mm = (size_t)m * m;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t k = i / mm;
    const int p = (int)(i % mm), v = p / m, u = p % m;
    amp_t[i] = sqrtf(fmaxf(d[k * mm + (size_t)u * m + v], 0.f));
  }
}

// ... and in the layout the radix-16 modulus pass reads (m = 256): a_k with rows
// and columns digit-swapped.  One block per row, permuted in shared memory as in
// k_tc_rows16 so that reads and writes are coalesced.
__global__ void __launch_bounds__(256) k_tc_amp16(const float* __restrict__ d, float* __restrict__ amp_s,
                                                  int n_pos) {
  constexpr int m = 256, R = kR16Rows;
  __shared__ float sh[R][m + m / 16];
  const int c = threadIdx.x;
  const int pc = r16_perm(c);
  for (int row0 = blockIdx.x * R; row0 < n_pos * m; row0 += gridDim.x * R) {
    float v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = d[(size_t)(row0 + i) * m + c];
#pragma unroll
    for (int i = 0; i < R; ++i) sh[i][pc + (pc >> 4)] = sqrtf(fmaxf(v[i], 0.f));
    __syncthreads();
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int row = row0 + i, k = row / m, r = row % m;
      amp_s[((size_t)k * m + r16_perm(r)) * m + c] = sh[i][c + (c >> 4)];
    }
    __syncthreads();
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

// The radix-16 pass: the 32 x 32 real matrices of x -> x W16 and x -> x conj(W16)
// (K-major, high and low parts), their tensor maps (one 32 x 32 box), and the
// twiddles W_256^j in constant memory; per device.
struct TcTables16 {
  uint16_t* d = nullptr;  // [4][32][32]: fwd hi, fwd lo, inv hi, inv lo
  CUtensorMap map[4];
};
TcTables16 g_tables16[64];

cudaError_t get_tables16(const TcTables16** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  TcTables16& t = g_tables16[dev];
  {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    if (t.d) {
      *out = &t;
      return cudaSuccess;
    }
  }
  constexpr int K = 32, per = K * K;
  uint16_t h[4 * per];
  memset(h, 0, sizeof(h));
  for (int inv = 0; inv < 2; ++inv) {
    uint16_t* th = h + (2 * inv) * per;
    uint16_t* tl = th + per;
    for (int v = 0; v < 16; ++v)
      for (int c = 0; c < 16; ++c) {
        const int t_ = (c * v) % 16;
        double gr = cos(2.0 * M_PI * t_ / 16), gi = -sin(2.0 * M_PI * t_ / 16);
        if (fabs(gr) < 1e-15) gr = 0.0;
        if (fabs(gi) < 1e-15) gi = 0.0;
        if (inv) gi = -gi;
        const double val[4] = {gr, -gi, gi, gr};
        const int idx[4] = {(2 * v) * K + 2 * c, (2 * v) * K + 2 * c + 1, (2 * v + 1) * K + 2 * c,
                            (2 * v + 1) * K + 2 * c + 1};
        for (int j = 0; j < 4; ++j) {
          const uint16_t hv = host_bf16(val[j]);
          th[idx[j]] = hv;
          tl[idx[j]] = host_bf16(val[j] - host_bf16_value(hv));
        }
      }
  }
  float2 tw[256];
  for (int j = 0; j < 256; ++j) tw[j] = make_float2((float)cos(2.0 * M_PI * j / 256), (float)-sin(2.0 * M_PI * j / 256));
  uint16_t* d = nullptr;
  e = cudaMalloc(&d, sizeof(h));
  if (e == cudaSuccess) e = cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tw256, tw, sizeof(tw));
  TcTables16 nt;
  for (int j = 0; e == cudaSuccess && j < 4; ++j) e = make_map(&nt.map[j], d + j * per, K, K, 32);
  if (e != cudaSuccess) {
    if (d) cudaFree(d);
    return e;
  }
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (t.d) {
    cudaFree(d);
  } else {
    nt.d = d;
    t = nt;
  }
  *out = &t;
  return cudaSuccess;
}

template <int EPI>
cudaError_t launch_pass16(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                          int rows, int sms, TcPassArgs a, int inverse, cudaStream_t s) {
  a.tiles_n = 1;
  a.m_tiles = rows / kBM;  // blocks of 128 rows
  const int grid = a.m_tiles < sms ? a.m_tiles : sms;
  k_tc_fft16<EPI><<<grid, kTcThreads, kR16Smem, s>>>(ah, al, bh, bl, a, inverse);
  return cudaGetLastError();
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
  if ((e = cudaFuncSetAttribute(k_tc_fft16<kEpiSplitT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kR16Smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_tc_fft16<kEpiModulus>, cudaFuncAttributeMaxDynamicSharedMemorySize, kR16Smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_tc_fft16<kEpiF32T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kR16Smem)) !=
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
  const TcTables16* tables16 = nullptr;  // the radix-16 pass (m = 256)
  int* d_err = nullptr;
  int sms = 0;              // persistent grid: one CTA per SM
};

bool tc_supported(int m) { return m == 128 || m == 256; }

// m = 256 runs the radix-16 pass unless EMG_TC_RADIX16=0 (read once per process,
// so that every work area and the transposed amplitudes agree on the layout).
bool tc_radix16(int m) {
  static const bool on = [] {
    const char* v = getenv("EMG_TC_RADIX16");
    return !(v && v[0] == '0');
  }();
  return m == 256 && on;
}

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
  if (e == cudaSuccess && tc_radix16(m)) e = get_tables16(&w->tables16);
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

int tc_tiles_per_position(int m) {  // partial sums per position: one per output tile and epilogue warp
  return tc_radix16(m) ? (m / kBM) * kEpiWarps : (m / kBM) * (2 * m / kBN) * kEpiWarps;
}

cudaError_t tc_dft2(TcWork* w, const float2* in, float2* out, int count, int inverse, cudaStream_t s) {
  if (count < 1 || count > w->cap) return cudaErrorInvalidValue;
  const int m = w->m, rows = count * m;
  const size_t n = (size_t)count * m * m;
  const bool r16 = tc_radix16(m);
  if (r16)
    k_tc_rows16<<<rows / kR16Rows, 256, 0, s>>>(in, nullptr, nullptr, nullptr, nullptr, 0, 0, count, w->buf[0][0],
                                               w->buf[0][1]);
  else
    k_tc_split<<<grid_for(n), 256, 0, s>>>(in, w->buf[0][0], w->buf[0][1], n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (r16) {
    const CUtensorMap* B = &w->tables16->map[inverse ? 2 : 0];
    TcPassArgs a{};
    a.m = m;
    a.err = w->d_err;
    a.out_hi = w->buf[1][0];
    a.out_lo = w->buf[1][1];
    a.scale = 1.f;
    a.rows16 = 0;  // [kc][r]: rows natural, elements digit-swapped
    if ((e = launch_pass16<kEpiSplitT>(w->amap[0][0], w->amap[0][1], B[0], B[1], rows, w->sms, a, inverse, s)) !=
        cudaSuccess)
      return e;
    a.out_hi = a.out_lo = nullptr;
    a.out_f32 = out;
    a.scale = inverse ? 1.f / (float)(m * m) : 1.f;
    return launch_pass16<kEpiF32T>(w->amap[1][0], w->amap[1][1], B[0], B[1], rows, w->sms, a, inverse, s);
  }
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
  const bool r16 = tc_radix16(m);
  if (r16)
    k_tc_rows16<<<rows / kR16Rows, 256, 0, s>>>(nullptr, t.object, t.probe, t.pos, t.order, t.n_rows, t.n_cols,
                                                t.b, w->buf[0][0], w->buf[0][1]);
  else
    k_tc_psi<<<grid_for(n), 256, 0, s>>>(t.object, t.probe, t.pos, t.order, t.n_rows, t.n_cols, m, t.b,
                                         w->buf[0][0], w->buf[0][1]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (r16) {
    // The same four passes, each a radix-16 pass with transposed outputs.  Tile
    // layouts (rows x elements; "swapped" = stored at r16_perm of the index):
    // psi [r][c] both swapped -> [kc][r] both swapped -> (modulus) [kr][kc] both
    // swapped -> [c][kr] elements swapped -> R [r][c] natural.
    const CUtensorMap* F = &w->tables16->map[0];
    const CUtensorMap* G = &w->tables16->map[2];
    TcPassArgs a{};
    a.m = m;
    a.err = w->d_err;
    a.scale = 1.f;
    a.out_hi = w->buf[1][0];
    a.out_lo = w->buf[1][1];
    a.rows16 = 1;
    if ((e = launch_pass16<kEpiSplitT>(w->amap[0][0], w->amap[0][1], F[0], F[1], rows, w->sms, a, 0, s)) !=
        cudaSuccess)
      return e;
    a.out_hi = w->buf[0][0];
    a.out_lo = w->buf[0][1];
    a.amp_t = t.amp_t;
    a.order = t.order;
    a.partial = t.partial;
    a.scale = 1.f / (float)(m * m);
    if ((e = launch_pass16<kEpiModulus>(w->amap[1][0], w->amap[1][1], F[0], F[1], rows, w->sms, a, 0, s)) !=
        cudaSuccess)
      return e;
    a.amp_t = nullptr;
    a.order = nullptr;
    a.partial = nullptr;
    a.scale = 1.f;
    a.out_hi = w->buf[1][0];
    a.out_lo = w->buf[1][1];
    a.rows16 = 0;
    if ((e = launch_pass16<kEpiSplitT>(w->amap[0][0], w->amap[0][1], G[0], G[1], rows, w->sms, a, 1, s)) !=
        cudaSuccess)
      return e;
    a.out_hi = a.out_lo = nullptr;
    a.out_f32 = t.R;
    return launch_pass16<kEpiF32T>(w->amap[1][0], w->amap[1][1], G[0], G[1], rows, w->sms, a, 1, s);
  }
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
  if (tc_radix16(m)) {
    const int groups = n_pos * m / kR16Rows, grid = groups < 65536 ? groups : 65536;
    k_tc_amp16<<<grid, 256, 0, s>>>(d, amp_t, n_pos);
  } else {
    k_tc_amp<<<grid_for(n), 256, 0, s>>>(d, amp_t, m, n);
  }
  return cudaGetLastError();
}

}  // namespace emg

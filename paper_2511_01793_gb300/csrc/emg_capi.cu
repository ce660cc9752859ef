// C ABI of the eMAGPIE hot path: context, validation, scratch ownership and
// the minibatch / epoch drivers (Sec. 3 stochastic sweep of arXiv 2511.01793).
#include <math.h>
#include <algorithm>
#include <cmath>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/emagpie.h"
#include "emg_internal.h"

using emg::ApplyArgs;
using emg::kMaxLevels;
using emg::PrepArgs;
using emg::StepArgs;

// Kernel kinds counted and timed by the profiling hooks.
enum { kKindPrep = 0, kKindStep = 1, kKindApply = 2, kKindOther = 3, kKindDft = 4, kKinds = 5 };
// Epochs whose misfit histories emg_reconstruct_host stages in the pinned scratch
// (h_scalar holds 64 doubles: two histories and the wait flag).
constexpr int kHostStageEpochs = 31;

// A captured epoch and the state it was captured for.
struct EpochGraph {
  cudaGraphExec_t exec = nullptr;
  float2* object = nullptr;
  float2* probe = nullptr;
  int verify = -1;
  int cluster = -1;
  const float* src = nullptr;
  int64_t counts[kKinds] = {0, 0, 0, 0, 0};
};

struct emg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_rows = 0, n_cols = 0, m = 0, n_pos = 0;
  emg_params par{};
  int verify = 0;
  int cluster = 1;                // CTAs per position in the step kernel (a tuning knob)
  int64_t epoch = 0;
  std::string err;
  int last_b = 0;

  // caller-bound state
  float2* object = nullptr;
  float2* probe = nullptr;

  // library-owned device buffers
  int32_t* d_pos = nullptr;       // [N][2]
  float* d_amp = nullptr;         // [N][m][m] storage order
  float2* d_zt = nullptr;         // [B][m][m]
  float2* d_qt = nullptr;         // [B][m][m]
  float* d_mu = nullptr;          // [B]
  double* d_phi = nullptr;        // [N]
  double* d_phi_after = nullptr;  // [B]
  double* d_partial = nullptr;    // [N] misfit partials
  double* d_scalar = nullptr;     // [64] assorted scalar results
  double* d_norm = nullptr;       // [1024] normalisation partials
  unsigned* d_mq = nullptr;       // [2] max|Q|^2 slots (float bits), alternating per minibatch
  // Fused probe prep (cluster step kernels, FFT path): [0] tickets, [1] prep
  // tiles done, [2] bounded wait gave up.  Both counters grow across the
  // launches that follow a max|Q|^2 seed; the host keeps their expected values.
  unsigned* d_sync = nullptr;
  unsigned ticket_base = 0, prep_done_base = 0;
  int resident_cluster = -1, resident_clusters = 0;  // step clusters resident at once, for `cluster`
  int fuse_prep = 1;              // probe prep inside the step launch where it fits (emg_set_prep_fusion)
  unsigned prep_wait_extra = 0;   // test hook: added to the prep count a launch waits for
  int32_t* d_epoch_order = nullptr;  // [N] order read by the captured epoch graph

  // One epoch captured as a CUDA graph (replayed per epoch on `stream`), and
  // the variant that also reads each minibatch's data from pinned host memory.
  cudaStream_t cap_stream = nullptr;
  EpochGraph graph, sgraph;
  // While the streamed variant is captured: its host source, the side stream
  // that reads it ahead of the step kernels, and the event that orders them.
  const float* stream_src = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_side = nullptr;
  float* d_wq = nullptr;          // [m][m]
  void* d_levels = nullptr;       // all multigrid arrays
  int32_t* d_orders = nullptr;    // [cap_orders]
  size_t cap_orders = 0;
  int32_t* h_orders = nullptr;    // pinned staging of the order rows, [cap_h_orders]
  size_t cap_h_orders = 0;
  cudaEvent_t ev_orders = nullptr;  // the last copy out of h_orders
  double* d_hist = nullptr;       // [2][cap_hist]
  size_t cap_hist = 0;
  float* d_stage_d = nullptr;     // [N][m][m] intensity staging (host input path)
  float2* d_own_object = nullptr; // host-buffer path state
  float2* d_own_probe = nullptr;
  int cap_minibatch = 0;          // minibatch capacity of the per-minibatch buffers
  int grad_chunk_req = 0;         // positions per gradient launch asked for (0: automatic)
  int grad_chunk = 0;             // positions per gradient launch in use (0: not chosen yet)
  float2* d_gz = nullptr;         // [grad_chunk][m][m] when it exceeds the minibatch
  float2* d_gq = nullptr;
  // second pair of gradient patch buffers: the sums of one chunk run on the
  // side stream while the next chunk's patches are computed
  float2* d_gz2 = nullptr;
  float2* d_gq2 = nullptr;
  cudaEvent_t ev_grad[3] = {nullptr, nullptr, nullptr};  // chunk computed; sums of buffer 0 / 1 done
  double* h_scalar = nullptr;     // pinned [64]

  // kernel timing (emg_set_profiling): CUDA events around each launch, per kernel kind
  int profile = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_marks;
  size_t ev_used = 0;
  int64_t launches[kKinds] = {0, 0, 0, 0, 0};

  // tensor-core DFT path (par.dft == EMG_DFT_BF16X3)
  emg::TcWork* tc = nullptr;
  float* d_amp_t = nullptr;       // [N][m][m] a_k transposed
  float2* d_tc_r = nullptr;       // [B][m][m] R_k
  double* d_tc_part = nullptr;    // [B][tiles] misfit partial sums
  // atomic object scatter (par.scatter == EMG_SCATTER_ATOMIC)
  float2* d_snum = nullptr;       // [n_rows][n_cols]
  float* d_sden = nullptr;        // [n_rows][n_cols]

  std::vector<int32_t> h_pos;
  PrepArgs prep{};
  emg::LevelArrays lv{};
};

// Several independent contexts whose epochs replay as one graph: one branch
// per context, forked after a kernel that selects every context's order row
// for the current epoch on the device.
struct emg_batch {
  std::vector<emg_ctx*> ctxs;
  int device = 0;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> forks;
  cudaGraphExec_t graph = nullptr;
  std::vector<const void*> key;   // per context: d_orders, object, probe, cluster, verify
  int32_t** d_src = nullptr;      // [count] device pointers to each context's order rows
  int32_t** d_dst = nullptr;      // [count] each context's epoch order buffer
  int* d_n = nullptr;             // [count] positions per context
  int* d_epoch = nullptr;         // current epoch within the call
  std::string err;
};

namespace {

std::mutex g_init_mu;
bool g_init_done[256] = {false};

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

emg_status fail(emg_ctx* c, emg_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

emg_status cuda_fail(emg_ctx* c, cudaError_t e, const char* where) {
  return fail(c, EMG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define EMG_CUDA(ctx, call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
  } while (0)

// Brackets one launch with a pair of events on the context's stream when profiling.
// NVTX range for the lifetime of a scope (a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

const char* const kKindNames[kKinds] = {"emg:prep", "emg:step", "emg:apply", "emg:other", "emg:dft"};

struct LaunchMark {
  emg_ctx* c;
  int kind;
  cudaEvent_t stop = nullptr;
  NvtxRange range;
  LaunchMark(emg_ctx* ctx, int k, int n = 1) : c(ctx), kind(k), range(kKindNames[k]) {
    c->launches[k] += n;
    if (!c->profile) return;
    if (c->ev_used + 2 > c->ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->ev_pool.push_back(e);
      }
    }
    cudaEvent_t start = c->ev_pool[c->ev_used++];
    stop = c->ev_pool[c->ev_used++];
    cudaEventRecord(start, c->stream);
    c->ev_marks.push_back({k, {start, stop}});
  }
  ~LaunchMark() {
    if (stop) cudaEventRecord(stop, c->stream);
  }
};

cudaError_t ensure_device_init(int dev) {
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  if (g_init_done[dev]) return cudaSuccess;
  cudaError_t e = emg::upload_twiddles();
  if (e == cudaSuccess) g_init_done[dev] = true;
  return e;
}

bool valid_m(int m) { return m == 16 || m == 32 || m == 64 || m == 128 || m == 256; }

emg_status validate_params(emg_ctx* c, const emg_params* p, int m, int n_pos) {
  if (!p) return fail(c, EMG_EINVAL, "params is NULL");
  if (!(p->alpha > 0.f) || !isfinite(p->alpha)) return fail(c, EMG_EINVAL, "alpha must be finite and > 0");
  if (p->levels < 1 || p->levels > kMaxLevels) return fail(c, EMG_EINVAL, "levels out of range [1, 7]");
  if ((m >> (p->levels - 1)) < 2) return fail(c, EMG_EINVAL, "m / 2^(levels-1) must be >= 2");
  if (p->minibatch < 1 || p->minibatch > 4096 || p->minibatch > n_pos)
    return fail(c, EMG_EINVAL, "minibatch must be in [1, min(n_pos, 4096)]");
  if (p->prolong != EMG_PROLONG_CONST && p->prolong != EMG_PROLONG_BILINEAR)
    return fail(c, EMG_EINVAL, "prolong must be EMG_PROLONG_CONST or EMG_PROLONG_BILINEAR");
  if (p->combine != EMG_COMBINE_WAVG && p->combine != EMG_COMBINE_SUM)
    return fail(c, EMG_EINVAL, "combine must be EMG_COMBINE_WAVG or EMG_COMBINE_SUM");
  if (p->scatter != EMG_SCATTER_DETERMINISTIC && p->scatter != EMG_SCATTER_ATOMIC)
    return fail(c, EMG_EINVAL, "unknown scatter mode");
  if (p->scatter == EMG_SCATTER_ATOMIC && p->combine == EMG_COMBINE_WAVG && !(p->w_eps > 0.f))
    return fail(c, EMG_EINVAL, "the atomic weighted-mean scatter needs w_eps > 0 (coverage is read from the weights)");
  if (p->joint != 0 && p->joint != 1) return fail(c, EMG_EINVAL, "joint must be 0 or 1");
  if (!(p->w_eps >= 0.f) || !isfinite(p->w_eps)) return fail(c, EMG_EINVAL, "w_eps must be finite and >= 0");
  if (p->dft != EMG_DFT_FFT32 && p->dft != EMG_DFT_BF16X3) return fail(c, EMG_EINVAL, "unknown dft mode");
  if (p->dft == EMG_DFT_BF16X3 && !emg::tc_supported(m))
    return fail(c, EMG_ENOTSUP, "the tensor-core DFT is built for m = 128 and 256");
  if (!emg::step_supported(m, p->levels, emg::default_cluster(m, p->levels)))
    return fail(c, EMG_ENOTSUP, "too many multigrid levels for this probe size");
  return EMG_OK;
}

// Host-side fault injection (emg_debug_fail_alloc): the library's device
// allocation after this many successful ones fails once; -1 disables.
std::atomic<int> g_fail_alloc_after{-1};

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  int n = g_fail_alloc_after.load();
  while (n >= 0 && !g_fail_alloc_after.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 0) return cudaErrorMemoryAllocation;
  return cudaMalloc((void**)p, count * sizeof(T));
}

void free_all(emg_ctx* c) {
  cudaFree(c->d_pos);
  cudaFree(c->d_amp);
  cudaFree(c->d_zt);
  cudaFree(c->d_qt);
  cudaFree(c->d_mu);
  cudaFree(c->d_phi);
  cudaFree(c->d_phi_after);
  cudaFree(c->d_partial);
  cudaFree(c->d_scalar);
  cudaFree(c->d_norm);
  cudaFree(c->d_mq);
  cudaFree(c->d_sync);
  cudaFree(c->d_epoch_order);
  if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
  if (c->sgraph.exec) cudaGraphExecDestroy(c->sgraph.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_side) cudaEventDestroy(c->ev_side);
  cudaFree(c->d_wq);
  cudaFree(c->d_levels);
  cudaFree(c->d_orders);
  if (c->ev_orders) cudaEventSynchronize(c->ev_orders);
  if (c->h_orders) cudaFreeHost(c->h_orders);
  if (c->ev_orders) cudaEventDestroy(c->ev_orders);
  cudaFree(c->d_hist);
  cudaFree(c->d_stage_d);
  cudaFree(c->d_own_object);
  cudaFree(c->d_own_probe);
  cudaFree(c->d_gz);
  cudaFree(c->d_gq);
  cudaFree(c->d_gz2);
  cudaFree(c->d_gq2);
  for (cudaEvent_t& ev : c->ev_grad)
    if (ev) cudaEventDestroy(ev);
  if (c->h_scalar) cudaFreeHost(c->h_scalar);
  emg::tc_work_destroy(c->tc);
  c->tc = nullptr;
  cudaFree(c->d_amp_t);
  cudaFree(c->d_tc_r);
  cudaFree(c->d_tc_part);
  cudaFree(c->d_snum);
  cudaFree(c->d_sden);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
}

// Carves the multigrid level arrays out of one allocation.
emg_status alloc_levels(emg_ctx* c) {
  const int m = c->m, L = c->par.levels;
  size_t bytes = 0;
  auto take = [&](size_t b) {
    size_t off = (bytes + 255) & ~(size_t)255;
    bytes = off + b;
    return off;
  };
  size_t offG[kMaxLevels], offQ[kMaxLevels], offWz[kMaxLevels], offWR[kMaxLevels], offU[kMaxLevels],
      offT[kMaxLevels];
  for (int l = 0; l < L; ++l) {
    const size_t n = (size_t)(m >> l) * (m >> l);
    offG[l] = take(n * sizeof(float2));
    offQ[l] = take(n * sizeof(float2));
    offU[l] = take(n * sizeof(float));
    if (l + 1 < L) {
      offWz[l] = take(n * sizeof(float));
      offWR[l] = take(n * sizeof(float2));
      offT[l] = take(n / 4 * sizeof(float));
    }
  }
  cudaError_t e = cudaMalloc(&c->d_levels, bytes);
  if (e != cudaSuccess) return fail(c, EMG_ENOMEM, "cudaMalloc(levels) failed");
  char* base = (char*)c->d_levels;
  PrepArgs& pa = c->prep;
  memset(&pa, 0, sizeof(pa));
  memset(&c->lv, 0, sizeof(c->lv));
  for (int l = 0; l < L; ++l) {
    pa.G[l] = (float2*)(base + offG[l]);
    pa.Q[l] = (float2*)(base + offQ[l]);
    pa.u[l] = (float*)(base + offU[l]);
    c->lv.G[l] = pa.G[l];
    c->lv.Q[l] = pa.Q[l];
    if (l + 1 < L) {
      pa.Wz[l] = (float*)(base + offWz[l]);
      pa.WR[l] = (float2*)(base + offWR[l]);
      pa.T[l] = (float*)(base + offT[l]);
      c->lv.Wz[l] = pa.Wz[l];
      c->lv.WR[l] = pa.WR[l];
    }
  }
  pa.m = m;
  pa.levels = L;
  pa.prolong = c->par.prolong;
  pa.alpha = c->par.alpha;
  pa.w_eps = c->par.w_eps;
  pa.wq = c->d_wq;
  return EMG_OK;
}

// Copies n order entries to d_orders through the pinned staging buffer (a
// true asynchronous copy; the buffer is reused once the previous copy is done).
emg_status upload_orders(emg_ctx* c, const int32_t* src, size_t n, cudaStream_t s) {
  if (c->ev_orders) EMG_CUDA(c, cudaEventSynchronize(c->ev_orders));
  if (n > c->cap_h_orders) {
    if (c->h_orders) cudaFreeHost(c->h_orders);
    c->h_orders = nullptr;
    c->cap_h_orders = 0;
    if (cudaMallocHost(&c->h_orders, n * sizeof(int32_t)) != cudaSuccess)
      return fail(c, EMG_ENOMEM, "cudaMallocHost(orders) failed");
    c->cap_h_orders = n;
  }
  memcpy(c->h_orders, src, n * sizeof(int32_t));
  EMG_CUDA(c, cudaMemcpyAsync(c->d_orders, c->h_orders, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (!c->ev_orders) EMG_CUDA(c, cudaEventCreateWithFlags(&c->ev_orders, cudaEventDisableTiming));
  EMG_CUDA(c, cudaEventRecord(c->ev_orders, s));
  return EMG_OK;
}

emg_status ensure_orders(emg_ctx* c, size_t n) {
  if (n <= c->cap_orders) return EMG_OK;
  cudaFree(c->d_orders);
  c->d_orders = nullptr;
  c->cap_orders = 0;
  if (cudaMalloc(&c->d_orders, n * sizeof(int32_t)) != cudaSuccess)
    return fail(c, EMG_ENOMEM, "cudaMalloc(orders) failed");
  c->cap_orders = n;
  return EMG_OK;
}

emg_status ensure_hist(emg_ctx* c, size_t n) {
  if (n <= c->cap_hist) return EMG_OK;
  cudaFree(c->d_hist);
  c->d_hist = nullptr;
  c->cap_hist = 0;
  if (cudaMalloc(&c->d_hist, 2 * n * sizeof(double)) != cudaSuccess)
    return fail(c, EMG_ENOMEM, "cudaMalloc(history) failed");
  c->cap_hist = n;
  return EMG_OK;
}

uint64_t splitmix_next(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t x = s;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

void permutation(uint64_t seed, int64_t epoch, int32_t n, int32_t* out) {
  uint64_t s = seed + (uint64_t)epoch * 0x9E3779B97F4A7C15ull;
  for (int32_t i = 0; i < n; ++i) out[i] = i;
  for (int32_t i = n - 1; i >= 1; --i) {
    const uint64_t j = splitmix_next(s) % (uint64_t)(i + 1);
    const int32_t t = out[i];
    out[i] = out[j];
    out[j] = t;
  }
}

// Seeds max|Q|^2 of the bound probe into slot 0 before a call's first minibatch.
emg_status seed_probe_max(emg_ctx* c, cudaStream_t s) {
  EMG_CUDA(c, cudaMemsetAsync(c->d_mq, 0, 2 * sizeof(unsigned), s));
  EMG_CUDA(c, cudaMemsetAsync(c->d_sync, 0, 2 * sizeof(unsigned), s));
  c->ticket_base = c->prep_done_base = 0;
  LaunchMark mk(c, kKindOther);
  cudaError_t e = emg::launch_probe_max(c->probe, c->m, c->d_mq, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_probe_max launch");
  return EMG_OK;
}

// One rank's part of a minibatch split across ranks: the step covers slots
// [s0, s1) and writes z~_k, Q~_k, mu_k of slot k to zt + k m^2, qt + k m^2,
// mu + k (caller-owned buffers of all slots); with `step` false the step is
// skipped and the combine reads every slot from those buffers.
struct ShardPart {
  int s0, s1;
  float2* zt;
  float2* qt;
  float* mu;
  bool step, apply;
};

// Enqueues one minibatch: probe prep, per-position step, combine.  `seq` is the
// minibatch's index within the current call: it selects which max|Q|^2 slot
// the prep reads and which one the combine fills.
emg_status enqueue_minibatch(emg_ctx* c, const int32_t* d_idx, int b, double* d_phi_out, int seq,
                             cudaStream_t strm, const ShardPart* sh = nullptr) {
  if (!c->object || !c->probe) return fail(c, EMG_EINVAL, "no state bound");
  const size_t mm = (size_t)c->m * c->m;
  // the slots this call steps (all of them unless a shard says otherwise)
  const int s0 = sh ? sh->s0 : 0, nb = sh ? sh->s1 - sh->s0 : b;
  const bool do_step = !sh || sh->step, do_apply = !sh || sh->apply;
  float2* zt_all = sh ? sh->zt : c->d_zt;
  float2* qt_all = sh ? sh->qt : c->d_qt;
  float* mu_all = sh ? sh->mu : c->d_mu;
  if (do_step) {
  PrepArgs pa = c->prep;
  pa.probe = c->probe;  // the probe bound right now (emg_reconstruct_host swaps it)
  pa.mq_read = c->d_mq + (seq & 1);
  pa.mq_next = c->d_mq + ((seq + 1) & 1);
  cudaError_t e;
  if (c->stream_src) {  // this minibatch's amplitudes, read from host memory on the side stream
    {
      LaunchMark mk(c, kKindOther);
      e = emg::launch_amp_gather(c->stream_src, d_idx + s0, nb, c->d_amp, c->m, c->side);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "k_amp_gather launch");
    EMG_CUDA(c, cudaEventRecord(c->ev_side, c->side));
  }
  // The probe prep runs inside the cluster step launch (FFT path) when the
  // launch fits in one wave of resident clusters: there it overlaps the gather
  // and transforms.  Otherwise it is its own kernel before the step.
  PrepArgs pf = pa;
  int fused_tiles = (c->fuse_prep && !c->tc && c->cluster >= 2) ? emg::fused_prep_tiles(pf, c->m, c->cluster) : 0;
  if (fused_tiles > 0) {
    const int prep_clusters = (fused_tiles + c->cluster - 1) / c->cluster;
    if (c->resident_cluster != c->cluster) {
      c->resident_clusters = emg::step_resident_clusters(c->m, c->cluster);
      c->resident_cluster = c->cluster;
    }
    if (nb + prep_clusters > c->resident_clusters || nb == 0) fused_tiles = 0;
  }
  if (fused_tiles == 0) {
    {
      LaunchMark mk(c, kKindPrep);
      e = emg::launch_prep(pa, strm);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "k_prep launch");
  }
  if (c->stream_src) EMG_CUDA(c, cudaStreamWaitEvent(strm, c->ev_side, 0));
  StepArgs sa{};
  sa.object = c->object;
  sa.probe = c->probe;
  sa.pos = c->d_pos;
  sa.amp = c->d_amp;
  sa.order = d_idx + s0;
  sa.mq = pa.mq_read;
  sa.n_rows = c->n_rows;
  sa.n_pos = c->n_pos;
  sa.b = nb;
  sa.n_cols = c->n_cols;
  sa.levels = c->par.levels;
  sa.prolong = c->par.prolong;
  sa.joint = c->par.joint;
  sa.verify = c->verify;
  sa.cluster = c->cluster;
  sa.alpha = c->par.alpha;
  sa.lv = c->lv;
  sa.zt = zt_all + (size_t)s0 * mm;
  sa.qt = qt_all + (size_t)s0 * mm;
  sa.mu = mu_all + s0;
  sa.phi = d_phi_out + s0;
  sa.phi_after = c->d_phi_after;
  sa.combine = c->par.combine;
  sa.w_eps = c->par.w_eps;
  const bool atomic = c->par.scatter == EMG_SCATTER_ATOMIC;
  sa.s_num = atomic ? c->d_snum : nullptr;
  sa.s_den = atomic ? c->d_sden : nullptr;
  sa.sync = c->d_sync;
  if (fused_tiles > 0) {
    sa.prep = pf;
    sa.prep_tiles = fused_tiles;
    sa.prep_clusters = (fused_tiles + c->cluster - 1) / c->cluster;
    sa.ticket_base = c->ticket_base;
    sa.prep_target = c->prep_done_base + (unsigned)fused_tiles + c->prep_wait_extra;
    c->ticket_base += (unsigned)(nb + sa.prep_clusters);
    c->prep_done_base += (unsigned)fused_tiles;
  }
  if (nb == 0) {
    // an empty share: only the prep ran (the combine needs its weights)
  } else if (c->tc) {
    emg::TcStepArgs ta{};
    ta.object = c->object;
    ta.probe = c->probe;
    ta.pos = c->d_pos;
    ta.order = d_idx + s0;
    ta.n_rows = c->n_rows;
    ta.n_cols = c->n_cols;
    ta.b = nb;
    ta.amp_t = c->d_amp_t;
    ta.R = c->d_tc_r;
    ta.partial = c->d_tc_part;
    {
      LaunchMark mk(c, kKindDft, 5);
      e = emg::tc_exit_waves(c->tc, ta, strm);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core DFT launch");
    sa.r_in = c->d_tc_r;
    sa.r_partial = c->d_tc_part;
    sa.r_tiles = emg::tc_tiles_per_position(c->m);
    {
      LaunchMark mk(c, kKindStep);
      e = emg::launch_step_rin(c->m, nb, sa, strm);
    }
  } else {
    LaunchMark mk(c, kKindStep);
    e = emg::launch_step(c->m, nb, sa, strm);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "k_step launch");
  }  // do_step
  if (!do_apply) return EMG_OK;
  const bool atomic = c->par.scatter == EMG_SCATTER_ATOMIC;
  cudaError_t e;
  ApplyArgs aa{};
  aa.object = c->object;
  aa.probe = c->probe;
  aa.pos = c->d_pos;
  aa.order = d_idx;
  aa.b = b;
  aa.n_pos = c->n_pos;
  aa.n_rows = c->n_rows;
  aa.n_cols = c->n_cols;
  aa.m = c->m;
  aa.combine = c->par.combine;
  aa.zt = zt_all;
  aa.qt = qt_all;
  aa.mu = mu_all;
  aa.wq = c->d_wq;
  aa.mq_next = c->d_mq + ((seq + 1) & 1);
  aa.tiles_x = emg::apply_tiles_x(c->n_cols);
  aa.tiles_y = emg::apply_tiles_y(c->n_rows);
  aa.s_num = atomic ? c->d_snum : nullptr;
  aa.s_den = atomic ? c->d_sden : nullptr;
  {
    LaunchMark mk(c, kKindApply);
    e = emg::launch_apply(aa, strm);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "k_apply launch");
  return EMG_OK;
}

// Reads (synchronously) the flag the tensor-core kernels set when one of their
// bounded waits gave up; callers invoke it where they synchronise anyway.
emg_status check_tc_flag(emg_ctx* c) {
  unsigned gave_up = 0;
  EMG_CUDA(c, cudaMemcpy(&gave_up, c->d_sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (gave_up) {
    EMG_CUDA(c, cudaMemset(c->d_sync + 2, 0, sizeof(unsigned)));
    return fail(c, EMG_ETIMEOUT, "the step kernel's bounded wait for the fused probe prep gave up");
  }
  if (!c->tc) return EMG_OK;
  int flag = 0;
  EMG_CUDA(c, cudaMemcpy(&flag, emg::tc_error_flag(c->tc), sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) return fail(c, EMG_ETIMEOUT, "a bounded wait in the tensor-core DFT kernel gave up");
  return EMG_OK;
}

emg_status check_bound(emg_ctx* c) {
  if (!c->object || !c->probe) return fail(c, EMG_EINVAL, "no state bound (call emg_bind_state)");
  return EMG_OK;
}

// Enqueues one epoch reading its order from d_epoch_order: the max|Q|^2 seed
// and every minibatch (used inside graph capture).
emg_status enqueue_epoch(emg_ctx* c, cudaStream_t s) {
  emg_status st = seed_probe_max(c, s);
  if (st == EMG_OK && c->stream_src) {
    EMG_CUDA(c, cudaEventRecord(c->ev_side, s));
    EMG_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_side, 0));
  }
  const int N = c->n_pos, B = c->par.minibatch;
  int seq = 0;
  for (int b0 = 0; st == EMG_OK && b0 < N; b0 += B) {
    const int b = (N - b0 < B) ? N - b0 : B;
    st = enqueue_minibatch(c, c->d_epoch_order + b0, b, c->d_phi + b0, seq++, s);
  }
  return st;
}

// Captures one epoch (probe-max seed + all minibatches reading d_epoch_order)
// as a graph for the currently bound state; reused until the state changes.
// With `src` (pinned host intensities) each minibatch's amplitudes are read
// from it on the side stream, and the minibatch's step waits for them.
emg_status ensure_epoch_graph(emg_ctx* c, EpochGraph& G, const float* src) {
  if (G.exec && G.object == c->object && G.probe == c->probe && G.verify == c->verify &&
      G.cluster == c->cluster && G.src == src)
    return EMG_OK;
  if (G.exec) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  int64_t before[kKinds];
  for (int i = 0; i < kKinds; ++i) before[i] = c->launches[i];
  EMG_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  c->stream_src = src;
  emg_status st = enqueue_epoch(c, c->cap_stream);
  c->stream_src = nullptr;
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
  for (int i = 0; i < kKinds; ++i) {
    G.counts[i] = c->launches[i] - before[i];
    c->launches[i] = before[i];
  }
  if (st != EMG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture");
  const cudaError_t ie = cudaGraphInstantiate(&G.exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    G.exec = nullptr;
    return cuda_fail(c, ie, "cudaGraphInstantiate");
  }
  G.object = c->object;
  G.probe = c->probe;
  G.verify = c->verify;
  G.cluster = c->cluster;
  G.src = src;
  return EMG_OK;
}

// Drops the captured epochs (they hold the buffers and settings they were captured with).
void drop_graphs(emg_ctx* c) {
  for (EpochGraph* G : {&c->graph, &c->sgraph}) {
    if (G->exec) cudaGraphExecDestroy(G->exec);
    *G = EpochGraph();
  }
}

emg_status set_minibatch_impl(emg_ctx* c, int32_t B) {
  if (B < 1 || B > c->n_pos) return fail(c, EMG_EINVAL, "minibatch must be in 1..n_pos");
  if (B == c->par.minibatch) return EMG_OK;
  EMG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (B > c->cap_minibatch) {
    const size_t mm = (size_t)c->m * c->m;
    float2 *zt = nullptr, *qt = nullptr, *r = nullptr;
    float* mu = nullptr;
    double *after = nullptr, *part = nullptr;
    emg::TcWork* tc = nullptr;
    bool ok = !dmalloc(&zt, (size_t)B * mm) && !dmalloc(&qt, (size_t)B * mm) && !dmalloc(&mu, (size_t)B) &&
              !dmalloc(&after, (size_t)B);
    if (ok && c->tc)
      ok = emg::tc_work_create(&tc, c->m, B) == cudaSuccess && !dmalloc(&r, (size_t)B * mm) &&
           !dmalloc(&part, (size_t)B * emg::tc_tiles_per_position(c->m));
    if (!ok) {
      cudaFree(zt);
      cudaFree(qt);
      cudaFree(mu);
      cudaFree(after);
      cudaFree(r);
      cudaFree(part);
      if (tc) emg::tc_work_destroy(tc);
      cudaGetLastError();
      return fail(c, EMG_ENOMEM, "minibatch buffers");
    }
    cudaFree(c->d_zt);
    cudaFree(c->d_qt);
    cudaFree(c->d_mu);
    cudaFree(c->d_phi_after);
    c->d_zt = zt;
    c->d_qt = qt;
    c->d_mu = mu;
    c->d_phi_after = after;
    if (c->tc) {
      emg::tc_work_destroy(c->tc);
      cudaFree(c->d_tc_r);
      cudaFree(c->d_tc_part);
      c->tc = tc;
      c->d_tc_r = r;
      c->d_tc_part = part;
    }
    c->cap_minibatch = B;
  }
  EMG_CUDA(c, cudaMemsetAsync(c->d_phi_after, 0xff, (size_t)c->cap_minibatch * sizeof(double), c->stream));
  c->par.minibatch = B;
  // the gradient may have used the minibatch buffers for its patches
  cudaFree(c->d_gz);
  cudaFree(c->d_gq);
  cudaFree(c->d_gz2);
  cudaFree(c->d_gq2);
  c->d_gz = c->d_gq = c->d_gz2 = c->d_gq2 = nullptr;
  c->grad_chunk = 0;
  drop_graphs(c);
  return EMG_OK;
}

emg_status set_scatter_impl(emg_ctx* c, int32_t mode) {
  if (mode != EMG_SCATTER_DETERMINISTIC && mode != EMG_SCATTER_ATOMIC) return fail(c, EMG_EINVAL, "unknown scatter mode");
  if (mode == EMG_SCATTER_ATOMIC && c->par.combine == EMG_COMBINE_WAVG && !(c->par.w_eps > 0.f))
    return fail(c, EMG_EINVAL, "the atomic weighted-mean scatter needs w_eps > 0 (coverage is read from the weights)");
  if (mode == c->par.scatter) return EMG_OK;
  EMG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (mode == EMG_SCATTER_ATOMIC && !c->d_snum) {
    const size_t npx = (size_t)c->n_rows * c->n_cols;
    if (dmalloc(&c->d_snum, npx) || dmalloc(&c->d_sden, npx)) {
      cudaFree(c->d_snum);
      c->d_snum = nullptr;
      c->d_sden = nullptr;
      cudaGetLastError();
      return fail(c, EMG_ENOMEM, "atomic scatter accumulators");
    }
    EMG_CUDA(c, cudaMemsetAsync(c->d_snum, 0, npx * sizeof(float2), c->stream));
    EMG_CUDA(c, cudaMemsetAsync(c->d_sden, 0, npx * sizeof(float), c->stream));
  }
  c->par.scatter = mode;
  drop_graphs(c);
  return EMG_OK;
}

// `stream_src`: pinned host intensities that epoch 0 reads minibatch by
// minibatch (graph path only; the amplitudes of all positions are in place
// after it, since an epoch visits every position).
// With `flag_out` (pinned host memory; FFT path only) the call does not wait:
// it queues the copies of the misfit histories and of the bounded-wait flag
// and leaves synchronising and checking the flag to the caller.
emg_status run_epochs_impl(emg_ctx* c, int32_t n_epochs, const int32_t* order, double* running,
                           double* misfit, const float* stream_src = nullptr, unsigned* flag_out = nullptr) {
  if (n_epochs < 0) return fail(c, EMG_EINVAL, "n_epochs < 0");
  if (n_epochs == 0) return EMG_OK;
  const int N = c->n_pos, B = c->par.minibatch;
  std::vector<int32_t> h((size_t)n_epochs * N);
  if (order) {
    std::vector<unsigned char> seen(N);
    for (int32_t e = 0; e < n_epochs; ++e) {
      std::fill(seen.begin(), seen.end(), 0);
      for (int i = 0; i < N; ++i) {
        const int32_t v = order[(size_t)e * N + i];
        if (v < 0 || v >= N || seen[v]) return fail(c, EMG_EINVAL, "order row is not a permutation of 0..n_pos-1");
        seen[v] = 1;
      }
    }
    memcpy(h.data(), order, h.size() * sizeof(int32_t));
  } else {
    for (int32_t e = 0; e < n_epochs; ++e) permutation(c->par.seed, c->epoch + e, N, h.data() + (size_t)e * N);
  }
  emg_status st = ensure_orders(c, h.size());
  if (st != EMG_OK) return st;
  if ((st = ensure_hist(c, n_epochs)) != EMG_OK) return st;
  if ((st = upload_orders(c, h.data(), h.size(), c->stream)) != EMG_OK) return st;
  // Profiling times each launch with events, so it runs the epochs as direct
  // launches; otherwise each epoch replays the captured graph.
  const bool use_graph = !c->profile;
  if (!use_graph && stream_src) return fail(c, EMG_EINVAL, "streamed intensities need the graph path");
  if (use_graph && stream_src && (st = ensure_epoch_graph(c, c->sgraph, stream_src)) != EMG_OK) return st;
  if (use_graph && (n_epochs > 1 || !stream_src) && (st = ensure_epoch_graph(c, c->graph, nullptr)) != EMG_OK)
    return st;
  for (int32_t e = 0; e < n_epochs; ++e) {
    const int32_t* ord = c->d_orders + (size_t)e * N;
    if (use_graph) {
      const EpochGraph& G = (e == 0 && stream_src) ? c->sgraph : c->graph;
      EMG_CUDA(c, cudaMemcpyAsync(c->d_epoch_order, ord, (size_t)N * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                  c->stream));
      EMG_CUDA(c, cudaGraphLaunch(G.exec, c->stream));
      for (int i = 0; i < kKinds; ++i) c->launches[i] += G.counts[i];
    } else {
      if ((st = seed_probe_max(c, c->stream)) != EMG_OK) return st;
      int seq = 0;
      for (int b0 = 0; b0 < N; b0 += B) {
        const int b = (N - b0 < B) ? N - b0 : B;
        if ((st = enqueue_minibatch(c, ord + b0, b, c->d_phi + b0, seq++, c->stream)) != EMG_OK) return st;
      }
    }
    if (running) {
      c->launches[kKindOther] += 1;
      cudaError_t ce = emg::launch_sum(c->d_phi, N, 1.0, c->d_hist + e, c->stream);
      if (ce != cudaSuccess) return cuda_fail(c, ce, "k_sum launch");
    }
    if (misfit) {
      c->launches[kKindOther] += 2;
      cudaError_t ce = emg::launch_misfit(c->m, c->object, c->probe, c->d_pos, c->d_amp, c->n_rows,
                                          c->n_cols, N, c->d_partial, c->stream);
      if (ce != cudaSuccess) return cuda_fail(c, ce, "k_misfit launch");
      ce = emg::launch_sum(c->d_partial, N, 1.0, c->d_hist + c->cap_hist + e, c->stream);
      if (ce != cudaSuccess) return cuda_fail(c, ce, "k_sum launch");
    }
  }
  c->epoch += n_epochs;
  if (running)
    EMG_CUDA(c, cudaMemcpyAsync(running, c->d_hist, n_epochs * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (misfit)
    EMG_CUDA(c, cudaMemcpyAsync(misfit, c->d_hist + c->cap_hist, n_epochs * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  if (flag_out && !c->tc) {
    EMG_CUDA(c, cudaMemcpyAsync(flag_out, c->d_sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    return EMG_OK;
  }
  if (running || misfit) {
    EMG_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_tc_flag(c);
  }
  EMG_CUDA(c, cudaGetLastError());
  return EMG_OK;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Stopping criterion of Sec. 4.1 with the noise-floor rule of Sec. 4.3 (see the header).
int32_t stopping_epoch(const double* r, int n, int window, int patience, double floor) {
  double best = 0.0;
  bool have_best = false;
  int count = 0;
  for (int t = 1; t <= n; ++t) {
    if (floor > 0.0 && r[t - 1] < 0.9 * floor) return t;
    if (t < window) continue;
    double sum = 0.0;
    for (int i = 0; i < window; ++i) sum += r[t - 1 - i];
    const double avg = sum / window;
    if (have_best && avg >= best) {
      if (++count >= patience) return t;
    } else {
      count = 0;
      best = avg;
      have_best = true;
    }
  }
  return 0;
}

// Device address through which a kernel may read pinned, mapped host memory
// (over the CPU-GPU link), or NULL for any other pointer.
const float* mapped_host_pointer(const float* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? (const float*)at.devicePointer : nullptr;
}

emg_status set_intensity_impl(emg_ctx* c, const float* intensity) {
  const size_t n = (size_t)c->n_pos * c->m * c->m;
  const float* src = intensity;
  const float* mapped = (c->tc || is_device_pointer(intensity)) ? nullptr : mapped_host_pointer(intensity);
  if (mapped) {
    // pinned host data: the amplitude kernel reads it in place, one pass over the link
    src = mapped;
  } else if (!is_device_pointer(intensity)) {
    if (!c->d_stage_d && cudaMalloc(&c->d_stage_d, n * sizeof(float)) != cudaSuccess)
      return fail(c, EMG_ENOMEM, "cudaMalloc(intensity staging) failed");
    EMG_CUDA(c, cudaMemcpyAsync(c->d_stage_d, intensity, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    src = c->d_stage_d;
  }
  cudaError_t e = emg::launch_amp_prep(src, c->d_amp, c->m, c->n_pos, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_amp_prep launch");
  if (c->tc) {
    e = emg::launch_tc_amp(src, c->d_amp_t, c->m, c->n_pos, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_tc_amp launch");
  }
  return EMG_OK;
}

// Phi of the bound state (FP64 sum), synchronising.
emg_status misfit_now(emg_ctx* c, double* out) {
  cudaError_t e = emg::launch_misfit(c->m, c->object, c->probe, c->d_pos, c->d_amp, c->n_rows, c->n_cols,
                                     c->n_pos, c->d_partial, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_misfit launch");
  e = emg::launch_sum(c->d_partial, c->n_pos, 1.0, c->d_scalar, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_sum launch");
  EMG_CUDA(c, cudaMemcpyAsync(c->h_scalar, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  EMG_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = c->h_scalar[0];
  return EMG_OK;
}

// One trial of the search: `epochs` epochs from the saved state (copied into
// the private buffers, which are bound), after one untimed epoch that captures
// the graph.  Returns the device time and the misfit at the end.
emg_status tune_trial(emg_ctx* c, const float2* o0, const float2* p0, float2* tz, float2* tq, int64_t epoch0,
                      int epochs, cudaEvent_t e0, cudaEvent_t e1, double* ms, double* phi_end) {
  const size_t nz = (size_t)c->n_rows * c->n_cols, nq = (size_t)c->m * c->m;
  emg_status st = EMG_OK;
  for (int pass = 0; pass < 2 && st == EMG_OK; ++pass) {
    EMG_CUDA(c, cudaMemcpyAsync(tz, o0, nz * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    EMG_CUDA(c, cudaMemcpyAsync(tq, p0, nq * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    c->epoch = epoch0;
    if (pass == 1) EMG_CUDA(c, cudaEventRecord(e0, c->stream));
    st = run_epochs_impl(c, pass == 0 ? 1 : epochs, nullptr, nullptr, nullptr);
    if (pass == 1 && st == EMG_OK) EMG_CUDA(c, cudaEventRecord(e1, c->stream));
  }
  if (st != EMG_OK) return st;
  EMG_CUDA(c, cudaEventSynchronize(e1));
  float f = 0.f;
  EMG_CUDA(c, cudaEventElapsedTime(&f, e0, e1));
  *ms = f;
  return misfit_now(c, phi_end);
}

}  // namespace

extern "C" {

emg_status emg_default_params(emg_params* p) {
  if (!p) return EMG_EINVAL;
  p->alpha = 0.01f;
  p->levels = 1;
  p->minibatch = 1;
  p->prolong = EMG_PROLONG_CONST;
  p->combine = EMG_COMBINE_WAVG;
  p->scatter = EMG_SCATTER_DETERMINISTIC;
  p->joint = 1;
  p->w_eps = 1e-6f;
  p->dft = EMG_DFT_FFT32;
  p->seed = 0;
  return EMG_OK;
}

const char* emg_status_string(emg_status s) {
  switch (s) {
    case EMG_OK: return "EMG_OK";
    case EMG_EINVAL: return "EMG_EINVAL";
    case EMG_ENOMEM: return "EMG_ENOMEM";
    case EMG_ECUDA: return "EMG_ECUDA";
    case EMG_ETIMEOUT: return "EMG_ETIMEOUT";
    case EMG_ENOTSUP: return "EMG_ENOTSUP";
  }
  return "EMG_UNKNOWN";
}

emg_status emg_create(emg_ctx** out, const emg_problem* pr, const emg_params* par, emg_stream_t stream) {
  NvtxRange nvtx_range("emg_create");
  if (!out) return EMG_EINVAL;
  *out = nullptr;
  if (!pr || !par) return EMG_EINVAL;
  if (pr->n_rows < 1 || pr->n_cols < 1 || pr->n_pos < 1 || !pr->pos || !pr->intensity) return EMG_EINVAL;
  if (!valid_m(pr->m)) return EMG_ENOTSUP;
  if ((int64_t)pr->n_rows * pr->n_cols > ((int64_t)1 << 34)) return EMG_EINVAL;
  emg_ctx* c = new (std::nothrow) emg_ctx();
  if (!c) return EMG_ENOMEM;
  emg_status st = validate_params(c, par, pr->m, pr->n_pos);
  if (st != EMG_OK) {
    delete c;
    return st;
  }
  c->n_rows = pr->n_rows;
  c->n_cols = pr->n_cols;
  c->m = pr->m;
  c->n_pos = pr->n_pos;
  c->par = *par;
  c->cluster = emg::default_cluster(pr->m, par->levels);
  c->stream = (cudaStream_t)stream;
  auto bail = [&](emg_status s) {
    free_all(c);
    delete c;
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bail(EMG_ECUDA);
  if (ensure_device_init(c->device) != cudaSuccess) return bail(EMG_ECUDA);
  const int N = c->n_pos, m = c->m, B = par->minibatch;
  const size_t mm = (size_t)m * m;
  if (dmalloc(&c->d_pos, (size_t)2 * N) || dmalloc(&c->d_amp, (size_t)N * mm) ||
      dmalloc(&c->d_zt, (size_t)B * mm) || dmalloc(&c->d_qt, (size_t)B * mm) ||
      dmalloc(&c->d_mu, (size_t)B) || dmalloc(&c->d_phi, (size_t)N) ||
      dmalloc(&c->d_phi_after, (size_t)B) || dmalloc(&c->d_partial, (size_t)N) ||
      dmalloc(&c->d_scalar, (size_t)64) || dmalloc(&c->d_norm, (size_t)1024) || dmalloc(&c->d_mq, (size_t)2) || dmalloc(&c->d_sync, (size_t)4) ||
      dmalloc(&c->d_epoch_order, (size_t)N) ||
      dmalloc(&c->d_wq, mm))
    return bail(EMG_ENOMEM);
  if (cudaMallocHost(&c->h_scalar, 64 * sizeof(double)) != cudaSuccess) return bail(EMG_ENOMEM);
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_side, cudaEventDisableTiming) != cudaSuccess)
    return bail(EMG_ECUDA);
  if (alloc_levels(c) != EMG_OK) return bail(EMG_ENOMEM);
  if (par->scatter == EMG_SCATTER_ATOMIC) {
    const size_t npx = (size_t)c->n_rows * c->n_cols;
    if (dmalloc(&c->d_snum, npx) || dmalloc(&c->d_sden, npx)) return bail(EMG_ENOMEM);
    if (cudaMemsetAsync(c->d_snum, 0, npx * sizeof(float2), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_sden, 0, npx * sizeof(float), c->stream) != cudaSuccess)
      return bail(EMG_ECUDA);
  }
  if (par->dft == EMG_DFT_BF16X3) {
    if (emg::tc_work_create(&c->tc, m, B) != cudaSuccess || dmalloc(&c->d_amp_t, (size_t)N * mm) ||
        dmalloc(&c->d_tc_r, (size_t)B * mm) || dmalloc(&c->d_tc_part, (size_t)B * emg::tc_tiles_per_position(m)))
      return bail(EMG_ENOMEM);
  }
  c->h_pos.resize((size_t)2 * N);
  if (cudaMemcpyAsync(c->h_pos.data(), pr->pos, c->h_pos.size() * sizeof(int32_t), cudaMemcpyDefault,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(EMG_ECUDA);
  for (int32_t v : c->h_pos)
    if (v <= -(1 << 24) || v >= (1 << 24)) return bail(EMG_EINVAL);
  if (cudaMemcpyAsync(c->d_pos, c->h_pos.data(), c->h_pos.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess)
    return bail(EMG_ECUDA);
  if (cudaMemsetAsync(c->d_phi_after, 0xff, (size_t)B * sizeof(double), c->stream) != cudaSuccess)
    return bail(EMG_ECUDA);
  c->cap_minibatch = B;
  if (cudaMemsetAsync(c->d_sync, 0, 4 * sizeof(unsigned), c->stream) != cudaSuccess) return bail(EMG_ECUDA);
  if (set_intensity_impl(c, pr->intensity) != EMG_OK) return bail(EMG_ECUDA);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(EMG_ECUDA);
  *out = c;
  return EMG_OK;
}

emg_status emg_set_intensity(emg_ctx* c, const float* intensity) {
  if (!c) return EMG_EINVAL;
  if (!intensity) return fail(c, EMG_EINVAL, "intensity is NULL");
  DeviceGuard g(c->device);
  return set_intensity_impl(c, intensity);
}

emg_status emg_bind_state(emg_ctx* c, float* object, float* probe) {
  if (!c) return EMG_EINVAL;
  if (!object || !probe) return fail(c, EMG_EINVAL, "object or probe is NULL");
  c->object = (float2*)object;
  c->probe = (float2*)probe;
  return EMG_OK;
}

emg_status emg_normalize_probe(emg_ctx* c) {
  if (!c) return EMG_EINVAL;
  emg_status st = check_bound(c);
  if (st != EMG_OK) return st;
  DeviceGuard g(c->device);
  cudaError_t e = emg::launch_normalize_probe(c->d_amp, c->m, c->n_pos, c->probe, c->d_norm, 1024, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "normalize launch");
  return EMG_OK;
}

emg_status emg_step_minibatch(emg_ctx* c, const int32_t* idx, int32_t b, double* sampled_misfit) {
  NvtxRange nvtx_range("emg_step_minibatch");
  if (!c) return EMG_EINVAL;
  emg_status st = check_bound(c);
  if (st != EMG_OK) return st;
  if (!idx) return fail(c, EMG_EINVAL, "idx is NULL");
  if (b < 1 || b > c->par.minibatch) return fail(c, EMG_EINVAL, "b must be in [1, params.minibatch]");
  for (int i = 0; i < b; ++i)
    if (idx[i] < 0 || idx[i] >= c->n_pos) return fail(c, EMG_EINVAL, "idx entry out of range");
  DeviceGuard g(c->device);
  if ((st = ensure_orders(c, (size_t)c->n_pos)) != EMG_OK) return st;
  if ((st = upload_orders(c, idx, (size_t)b, c->stream)) != EMG_OK) return st;
  if ((st = seed_probe_max(c, c->stream)) != EMG_OK) return st;
  if ((st = enqueue_minibatch(c, c->d_orders, b, c->d_phi, 0, c->stream)) != EMG_OK) return st;
  c->last_b = b;
  if (sampled_misfit) {
    cudaError_t e = emg::launch_sum(c->d_phi, b, 1.0, c->d_scalar, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_sum launch");
    EMG_CUDA(c, cudaMemcpyAsync(c->h_scalar, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    EMG_CUDA(c, cudaStreamSynchronize(c->stream));
    *sampled_misfit = c->h_scalar[0];
    return check_tc_flag(c);
  }
  return EMG_OK;
}

// Checks shared by the two halves of a minibatch split across ranks.
emg_status shard_args(emg_ctx* c, const int32_t* idx, int32_t b, const void* zt, const void* qt, const void* mu) {
  if (!c) return EMG_EINVAL;
  emg_status st = check_bound(c);
  if (st != EMG_OK) return st;
  if (!idx || !zt || !qt || !mu) return fail(c, EMG_EINVAL, "idx, zt, qt and mu must not be NULL");
  if (b < 1 || b > c->par.minibatch) return fail(c, EMG_EINVAL, "b must be in [1, params.minibatch]");
  if (c->par.scatter == EMG_SCATTER_ATOMIC)
    return fail(c, EMG_ENOTSUP, "a split minibatch exchanges patches; the atomic scatter has none");
  for (int i = 0; i < b; ++i)
    if (idx[i] < 0 || idx[i] >= c->n_pos) return fail(c, EMG_EINVAL, "idx entry out of range");
  return EMG_OK;
}

emg_status emg_shard_step(emg_ctx* c, const int32_t* idx, int32_t b, int32_t slot_begin, int32_t slot_end,
                          float* zt, float* qt, float* mu) {
  NvtxRange nvtx_range("emg_shard_step");
  emg_status st = shard_args(c, idx, b, zt, qt, mu);
  if (st != EMG_OK) return st;
  if (slot_begin < 0 || slot_end < slot_begin || slot_end > b)
    return fail(c, EMG_EINVAL, "need 0 <= slot_begin <= slot_end <= b");
  DeviceGuard g(c->device);
  if ((st = ensure_orders(c, (size_t)c->n_pos)) != EMG_OK) return st;
  if ((st = upload_orders(c, idx, (size_t)b, c->stream)) != EMG_OK) return st;
  if ((st = seed_probe_max(c, c->stream)) != EMG_OK) return st;
  ShardPart sh{slot_begin, slot_end, (float2*)zt, (float2*)qt, mu, true, false};
  return enqueue_minibatch(c, c->d_orders, b, c->d_phi, 0, c->stream, &sh);
}

emg_status emg_shard_apply(emg_ctx* c, const int32_t* idx, int32_t b, const float* zt, const float* qt,
                           const float* mu) {
  NvtxRange nvtx_range("emg_shard_apply");
  emg_status st = shard_args(c, idx, b, zt, qt, mu);
  if (st != EMG_OK) return st;
  DeviceGuard g(c->device);
  if ((st = ensure_orders(c, (size_t)c->n_pos)) != EMG_OK) return st;
  if ((st = upload_orders(c, idx, (size_t)b, c->stream)) != EMG_OK) return st;
  ShardPart sh{0, 0, (float2*)zt, (float2*)qt, (float*)mu, false, true};
  if ((st = enqueue_minibatch(c, c->d_orders, b, c->d_phi, 0, c->stream, &sh)) != EMG_OK) return st;
  c->last_b = b;
  return EMG_OK;
}

emg_status emg_position_stats(emg_ctx* c, double* out, int32_t b) {
  if (!c) return EMG_EINVAL;
  if (!out || b < 1 || b > c->last_b) return fail(c, EMG_EINVAL, "b must be in [1, last minibatch size]");
  DeviceGuard g(c->device);
  std::vector<double> phi(b), after(b);
  std::vector<float> mu(b);
  EMG_CUDA(c, cudaMemcpyAsync(phi.data(), c->d_phi, b * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  EMG_CUDA(c, cudaMemcpyAsync(after.data(), c->d_phi_after, b * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  EMG_CUDA(c, cudaMemcpyAsync(mu.data(), c->d_mu, b * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  EMG_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < b; ++i) {
    out[3 * i] = phi[i];
    out[3 * i + 1] = c->verify ? after[i] : NAN;
    out[3 * i + 2] = mu[i];
  }
  return EMG_OK;
}

emg_status emg_set_verify(emg_ctx* c, int32_t verify) {
  if (!c) return EMG_EINVAL;
  c->verify = verify ? 1 : 0;
  return EMG_OK;
}

emg_status emg_run_epochs(emg_ctx* c, int32_t n_epochs, const int32_t* order, double* running_misfit,
                          double* misfit) {
  NvtxRange nvtx_range("emg_run_epochs");
  if (!c) return EMG_EINVAL;
  emg_status st = check_bound(c);
  if (st != EMG_OK) return st;
  DeviceGuard g(c->device);
  return run_epochs_impl(c, n_epochs, order, running_misfit, misfit);
}

emg_status emg_misfit(emg_ctx* c, double* out) {
  if (!c) return EMG_EINVAL;
  emg_status st = check_bound(c);
  if (st != EMG_OK) return st;
  if (!out) return fail(c, EMG_EINVAL, "out is NULL");
  DeviceGuard g(c->device);
  cudaError_t e = emg::launch_misfit(c->m, c->object, c->probe, c->d_pos, c->d_amp, c->n_rows, c->n_cols,
                                     c->n_pos, c->d_partial, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_misfit launch");
  e = emg::launch_sum(c->d_partial, c->n_pos, 1.0, c->d_scalar, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_sum launch");
  EMG_CUDA(c, cudaMemcpyAsync(c->h_scalar, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  EMG_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = c->h_scalar[0];
  return check_tc_flag(c);
}

emg_status emg_set_epoch(emg_ctx* c, int64_t epoch) {
  if (!c) return EMG_EINVAL;
  if (epoch < 0) return fail(c, EMG_EINVAL, "epoch < 0");
  c->epoch = epoch;
  return EMG_OK;
}

emg_status emg_stopping_epoch(const double* r, int32_t n, int32_t window, int32_t patience, double floor,
                              int32_t* out) {
  if (!out || n < 0 || (n > 0 && !r) || window < 1 || patience < 1 || !(floor >= 0.0) || !isfinite(floor))
    return EMG_EINVAL;
  *out = stopping_epoch(r, n, window, patience, floor);
  return EMG_OK;
}

emg_status emg_run_until(emg_ctx* c, int32_t max_epochs, int32_t window, int32_t patience, double floor,
                         int32_t* epochs_run, double* misfit) {
  if (!c) return EMG_EINVAL;
  emg_status st = check_bound(c);
  if (st != EMG_OK) return st;
  if (!epochs_run || max_epochs < 0 || window < 1 || patience < 1 || !(floor >= 0.0) || !isfinite(floor))
    return fail(c, EMG_EINVAL, "invalid stopping parameters");
  DeviceGuard g(c->device);
  std::vector<double> r;
  r.reserve((size_t)max_epochs);
  *epochs_run = 0;
  for (int32_t e = 0; e < max_epochs; ++e) {
    double phi = 0.0;
    if ((st = run_epochs_impl(c, 1, nullptr, nullptr, &phi)) != EMG_OK) return st;
    r.push_back(phi);
    if (misfit) misfit[e] = phi;
    *epochs_run = e + 1;
    if (stopping_epoch(r.data(), (int)r.size(), window, patience, floor) != 0) break;
  }
  return EMG_OK;
}

emg_status emg_schedule_permutation(uint64_t seed, int64_t epoch, int32_t n, int32_t* out) {
  if (n < 0 || (n > 0 && !out) || epoch < 0) return EMG_EINVAL;
  permutation(seed, epoch, n, out);
  return EMG_OK;
}

emg_status emg_reconstruct_host(emg_ctx* c, const float* intensity, float* object, float* probe,
                                int32_t n_epochs, const int32_t* order, double* running_misfit,
                                double* misfit) {
  NvtxRange nvtx_range("emg_reconstruct_host");
  if (!c) return EMG_EINVAL;
  if (!intensity || !object || !probe) return fail(c, EMG_EINVAL, "NULL host buffer");
  DeviceGuard g(c->device);
  const size_t nz = (size_t)c->n_rows * c->n_cols, nq = (size_t)c->m * c->m;
  if (!c->d_own_object && cudaMalloc(&c->d_own_object, nz * sizeof(float2)) != cudaSuccess)
    return fail(c, EMG_ENOMEM, "cudaMalloc(object) failed");
  if (!c->d_own_probe && cudaMalloc(&c->d_own_probe, nq * sizeof(float2)) != cudaSuccess)
    return fail(c, EMG_ENOMEM, "cudaMalloc(probe) failed");
  // Pinned host intensities on the FFT path are read minibatch by minibatch
  // during the first epoch, overlapping the transfer with the earlier steps.
  const float* streamed = (n_epochs > 0 && !c->tc && !c->profile && !is_device_pointer(intensity))
                              ? mapped_host_pointer(intensity)
                              : nullptr;
  emg_status st = streamed ? EMG_OK : set_intensity_impl(c, intensity);
  if (st != EMG_OK) return st;
  EMG_CUDA(c, cudaMemcpyAsync(c->d_own_object, object, nz * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
  EMG_CUDA(c, cudaMemcpyAsync(c->d_own_probe, probe, nq * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
  float2* keep_o = c->object;
  float2* keep_p = c->probe;
  c->object = c->d_own_object;
  c->probe = c->d_own_probe;
  // Everything is queued and waited for once: the misfit histories land in the
  // context's pinned scratch when they fit (a copy to pageable memory would
  // wait), and the bounded-wait flag is read there after the one wait.
  const bool staged = !c->tc && n_epochs <= kHostStageEpochs;
  double* h_run = staged && running_misfit ? c->h_scalar : running_misfit;
  double* h_mis = staged && misfit ? c->h_scalar + kHostStageEpochs : misfit;
  unsigned* h_flag = staged ? reinterpret_cast<unsigned*>(c->h_scalar + 2 * kHostStageEpochs) : nullptr;
  if (h_flag) *h_flag = 0u;
  st = run_epochs_impl(c, n_epochs, order, h_run, h_mis, streamed, h_flag);
  c->object = keep_o;
  c->probe = keep_p;
  if (st != EMG_OK) return st;
  EMG_CUDA(c, cudaMemcpyAsync(object, c->d_own_object, nz * sizeof(float2), cudaMemcpyDeviceToHost, c->stream));
  EMG_CUDA(c, cudaMemcpyAsync(probe, c->d_own_probe, nq * sizeof(float2), cudaMemcpyDeviceToHost, c->stream));
  EMG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (staged) {
    if (running_misfit) memcpy(running_misfit, h_run, (size_t)n_epochs * sizeof(double));
    if (misfit) memcpy(misfit, h_mis, (size_t)n_epochs * sizeof(double));
    if (*h_flag) {
      EMG_CUDA(c, cudaMemset(c->d_sync + 2, 0, sizeof(unsigned)));
      return fail(c, EMG_ETIMEOUT, "the step kernel's bounded wait for the fused probe prep gave up");
    }
  }
  return EMG_OK;
}

emg_status emg_simulate_intensity(const float* object, int32_t n_rows, int32_t n_cols, const float* probe,
                                  int32_t m, const int32_t* pos, int32_t n_pos, float* out,
                                  emg_stream_t stream) {
  if (!object || !probe || !pos || !out || n_rows < 1 || n_cols < 1 || n_pos < 0) return EMG_EINVAL;
  if (!valid_m(m)) return EMG_ENOTSUP;
  if (n_pos == 0) return EMG_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || ensure_device_init(dev) != cudaSuccess) return EMG_ECUDA;
  cudaError_t e = emg::launch_simulate(m, (const float2*)object, (const float2*)probe, pos, n_rows, n_cols,
                                       n_pos, out, (cudaStream_t)stream);
  return e == cudaSuccess ? EMG_OK : EMG_ECUDA;
}

emg_status emg_fft2(const float* in, float* out, int32_t m, int32_t count, int32_t inverse,
                    emg_stream_t stream) {
  if (!in || !out || count < 0 || (inverse != 0 && inverse != 1)) return EMG_EINVAL;
  if (!valid_m(m)) return EMG_ENOTSUP;
  if (count == 0) return EMG_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || ensure_device_init(dev) != cudaSuccess) return EMG_ECUDA;
  cudaError_t e = emg::launch_fft2(m, (const float2*)in, (float2*)out, count, inverse, (cudaStream_t)stream);
  return e == cudaSuccess ? EMG_OK : EMG_ECUDA;
}

emg_status emg_debug_bounds_errors(uint32_t* mask) {
  if (!mask) return EMG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || ensure_device_init(dev) != cudaSuccess) return EMG_ECUDA;
  unsigned m = 0;
  const cudaError_t e = emg::bounds_errors_take(&m);
  *mask = m;
  if (e == cudaErrorNotSupported) return EMG_ENOTSUP;
  return e == cudaSuccess ? EMG_OK : EMG_ECUDA;
}

emg_status emg_debug_bounds_selftest(uint32_t* mask) {
  if (!mask) return EMG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || ensure_device_init(dev) != cudaSuccess) return EMG_ECUDA;
  unsigned m = 0;
  const cudaError_t e = emg::bounds_probe(&m);
  *mask = m;
  if (e == cudaErrorNotSupported) return EMG_ENOTSUP;
  return e == cudaSuccess ? EMG_OK : EMG_ECUDA;
}

emg_status emg_debug_fail_alloc(int32_t after) {
  if (after < -1) return EMG_EINVAL;
  g_fail_alloc_after.store(after);
  return EMG_OK;
}

emg_status emg_selftest_bounded_wait(int32_t* gave_up) {
  if (!gave_up) return EMG_EINVAL;
  *gave_up = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || ensure_device_init(dev) != cudaSuccess) return EMG_ECUDA;
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return EMG_ENOMEM;
  int h = 0;
  cudaError_t e = cudaMemset(flag, 0, sizeof(int));
  if (e == cudaSuccess) e = emg::launch_wait_selftest(flag, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(flag);
  if (e != cudaSuccess) return EMG_ECUDA;
  *gave_up = h;
  return EMG_OK;
}

emg_status emg_dft2_bf16x3(const float* in, float* out, int32_t m, int32_t count, int32_t inverse,
                           emg_stream_t stream) {
  if (!in || !out || in == out || count < 0 || (inverse != 0 && inverse != 1)) return EMG_EINVAL;
  if (!emg::tc_supported(m)) return EMG_ENOTSUP;
  if (count == 0) return EMG_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || ensure_device_init(dev) != cudaSuccess) return EMG_ECUDA;
  const cudaStream_t s = (cudaStream_t)stream;
  emg::TcWork* w = nullptr;
  if (emg::tc_work_create(&w, m, count) != cudaSuccess) return EMG_ENOMEM;
  cudaError_t e = emg::tc_dft2(w, (const float2*)in, (float2*)out, count, inverse, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, emg::tc_error_flag(w), sizeof(int), cudaMemcpyDeviceToHost);
  emg::tc_work_destroy(w);
  if (e != cudaSuccess) return EMG_ECUDA;
  return flag ? EMG_ETIMEOUT : EMG_OK;
}

emg_status emg_dft_bf16x3_form(int32_t m, int32_t* radix16) {
  if (!radix16) return EMG_EINVAL;
  if (!emg::tc_supported(m)) return EMG_ENOTSUP;
  *radix16 = emg::tc_radix16(m) ? 1 : 0;
  return EMG_OK;
}

emg_status emg_misfit_gradient(emg_ctx* c, const float* object, const float* probe, float* grad_object,
                               float* grad_probe, double* misfit) {
  NvtxRange nvtx_range("emg_misfit_gradient");
  if (!c) return EMG_EINVAL;
  if (!object || !probe) return fail(c, EMG_EINVAL, "object or probe is NULL");
  DeviceGuard g(c->device);
  const int N = c->n_pos;
  if (c->grad_chunk == 0) {
    // By default a multiple of the position clusters that can be resident at
    // once, about 128 positions per launch; the chunking fixes the order of the sums.
    const int pw = emg::gradient_positions_per_wave(c->m);
    int chunk = c->grad_chunk_req > 0 ? c->grad_chunk_req : pw > 0 ? pw * ((128 + pw - 1) / pw) : c->par.minibatch;
    if (chunk > N) chunk = N;
    if (chunk > c->par.minibatch) {
      const size_t bytes = (size_t)chunk * c->m * c->m * sizeof(float2);
      if (cudaMalloc(&c->d_gz, bytes) != cudaSuccess || cudaMalloc(&c->d_gq, bytes) != cudaSuccess) {
        cudaFree(c->d_gz);
        c->d_gz = nullptr;
        cudaGetLastError();
        return fail(c, EMG_ENOMEM, "cudaMalloc(gradient patches) failed");
      }
    }
    c->grad_chunk = chunk;
  }
  const int B = c->grad_chunk;
  const bool sums = grad_object || grad_probe;
  // With the sums asked for and more than one chunk, the sums of chunk i run on
  // the side stream while chunk i + 1's patches are computed into the other
  // buffer pair; the sums stay in chunk order on the side stream, so the
  // result is the same bitwise.  Without a second pair the chunks run in turn.
  bool overlap = sums && N > B;
  if (overlap && !c->d_gz2) {
    const size_t bytes = (size_t)B * c->m * c->m * sizeof(float2);
    if (cudaMalloc(&c->d_gz2, bytes) != cudaSuccess || cudaMalloc(&c->d_gq2, bytes) != cudaSuccess) {
      cudaFree(c->d_gz2);
      c->d_gz2 = nullptr;
      cudaGetLastError();
      overlap = false;
    }
  }
  for (int j = 0; overlap && j < 3; ++j)
    if (!c->ev_grad[j] && cudaEventCreateWithFlags(&c->ev_grad[j], cudaEventDisableTiming) != cudaSuccess) {
      c->ev_grad[j] = nullptr;
      cudaGetLastError();
      overlap = false;
    }
  for (int first = 0, chunk = 0; first < N; first += B, ++chunk) {
    const int b = (N - first < B) ? N - first : B;
    const int pair = overlap ? (chunk & 1) : 0;
    float2* gz = pair ? c->d_gz2 : (c->d_gz ? c->d_gz : c->d_zt);
    float2* gq = pair ? c->d_gq2 : (c->d_gq ? c->d_gq : c->d_qt);
    // the pair is free once the sums of chunk - 2 (which used it) are done
    if (overlap && chunk >= 2) EMG_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_grad[1 + pair], 0));
    emg::GradArgs ga{};
    ga.object = (const float2*)object;
    ga.probe = (const float2*)probe;
    ga.pos = c->d_pos;
    ga.amp = c->d_amp;
    ga.first = first;
    ga.n_rows = c->n_rows;
    ga.n_cols = c->n_cols;
    ga.gz = gz;
    ga.gq = gq;
    ga.phi = c->d_phi + first;
    cudaError_t e = emg::launch_gradient(c->m, b, ga, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_gradc launch");
    c->launches[kKindOther] += 1;
    if (sums) {
      const cudaStream_t rs = overlap ? c->side : c->stream;
      if (overlap) {
        EMG_CUDA(c, cudaEventRecord(c->ev_grad[0], c->stream));
        EMG_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_grad[0], 0));
      }
      emg::GradReduceArgs ra{};
      ra.pos = c->d_pos;
      ra.first = first;
      ra.b = b;
      ra.n_rows = c->n_rows;
      ra.n_cols = c->n_cols;
      ra.m = c->m;
      ra.accumulate = first > 0;
      ra.gz = gz;
      ra.gq = gq;
      ra.grad_object = (float2*)grad_object;
      ra.grad_probe = (float2*)grad_probe;
      ra.tiles_x = (c->n_cols + emg::kApplyTile - 1) / emg::kApplyTile;
      ra.tiles_y = (c->n_rows + emg::kApplyTile - 1) / emg::kApplyTile;
      e = emg::launch_grad_reduce(ra, rs);
      if (e != cudaSuccess) return cuda_fail(c, e, "k_grad_reduce launch");
      c->launches[kKindOther] += 1;
      if (overlap) EMG_CUDA(c, cudaEventRecord(c->ev_grad[1 + pair], c->side));
    }
  }
  if (overlap) {  // the caller's stream sees every sum
    EMG_CUDA(c, cudaEventRecord(c->ev_grad[0], c->side));
    EMG_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_grad[0], 0));
  }
  if (misfit) {
    cudaError_t e = emg::launch_sum(c->d_phi, N, 1.0, c->d_scalar, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_sum launch");
    EMG_CUDA(c, cudaMemcpyAsync(c->h_scalar, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    EMG_CUDA(c, cudaStreamSynchronize(c->stream));
    *misfit = c->h_scalar[0];
  }
  return EMG_OK;
}

emg_status emg_set_gradient_chunk(emg_ctx* c, int32_t positions) {
  if (!c) return EMG_EINVAL;
  if (positions < 0) return fail(c, EMG_EINVAL, "gradient chunk < 0");
  DeviceGuard g(c->device);
  EMG_CUDA(c, cudaStreamSynchronize(c->stream));
  cudaFree(c->d_gz);
  cudaFree(c->d_gq);
  cudaFree(c->d_gz2);
  cudaFree(c->d_gq2);
  c->d_gz = c->d_gq = c->d_gz2 = c->d_gq2 = nullptr;
  c->grad_chunk_req = positions;
  c->grad_chunk = 0;
  return EMG_OK;
}

emg_status emg_debug_prep_wait_extra(emg_ctx* c, uint32_t extra) {
  if (!c) return EMG_EINVAL;
  DeviceGuard g(c->device);
  EMG_CUDA(c, cudaStreamSynchronize(c->stream));
  c->prep_wait_extra = extra;
  drop_graphs(c);
  return EMG_OK;
}

emg_status emg_set_prep_fusion(emg_ctx* c, int32_t enable) {
  if (!c) return EMG_EINVAL;
  if (enable != 0 && enable != 1) return fail(c, EMG_EINVAL, "enable must be 0 or 1");
  if (enable != c->fuse_prep) {
    DeviceGuard g(c->device);
    EMG_CUDA(c, cudaStreamSynchronize(c->stream));
    c->fuse_prep = enable;
    drop_graphs(c);
  }
  return EMG_OK;
}

emg_status emg_set_cluster(emg_ctx* c, int32_t cluster) {
  if (!c) return EMG_EINVAL;
  if (!emg::step_supported(c->m, c->par.levels, cluster))
    return fail(c, EMG_ENOTSUP, "cluster size not built or not valid for this probe size and level count");
  c->cluster = cluster;
  return EMG_OK;
}

emg_status emg_set_minibatch(emg_ctx* c, int32_t minibatch) {
  if (!c) return EMG_EINVAL;
  DeviceGuard g(c->device);
  return set_minibatch_impl(c, minibatch);
}

emg_status emg_set_scatter(emg_ctx* c, int32_t scatter) {
  if (!c) return EMG_EINVAL;
  DeviceGuard g(c->device);
  return set_scatter_impl(c, scatter);
}

emg_status emg_autotune_search(emg_ctx* c, const emg_tune_request* req, emg_tune_result* res) {
  NvtxRange nvtx_range("emg_autotune_search");
  if (!c) return EMG_EINVAL;
  if (!req || !res) return fail(c, EMG_EINVAL, "request or result is NULL");
  if (req->n_minibatch < 0 || (req->n_minibatch > 0 && !req->minibatch) || req->trial_epochs < 1)
    return fail(c, EMG_EINVAL, "minibatch candidates or trial epochs invalid");
  for (int i = 0; i < req->n_minibatch; ++i)
    if (req->minibatch[i] < 1 || req->minibatch[i] > c->n_pos)
      return fail(c, EMG_EINVAL, "minibatch candidate outside 1..n_pos");
  if (req->allow_atomic && c->par.combine == EMG_COMBINE_WAVG && !(c->par.w_eps > 0.f))
    return fail(c, EMG_EINVAL, "the atomic weighted-mean scatter needs w_eps > 0");
  emg_status st = check_bound(c);
  if (st != EMG_OK) return st;
  DeviceGuard g(c->device);
  const size_t nz = (size_t)c->n_rows * c->n_cols, nq = (size_t)c->m * c->m;
  float2 *tz = nullptr, *tq = nullptr;
  if (cudaMalloc(&tz, nz * sizeof(float2)) != cudaSuccess || cudaMalloc(&tq, nq * sizeof(float2)) != cudaSuccess) {
    cudaFree(tz);
    cudaGetLastError();
    return fail(c, EMG_ENOMEM, "autotune scratch");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float2* keep_o = c->object;
  float2* keep_p = c->probe;
  const int64_t keep_epoch = c->epoch;
  const int keep_profile = c->profile;
  const int keep_b = c->par.minibatch, keep_cl = c->cluster, keep_sc = c->par.scatter;
  int64_t keep_launches[kKinds];
  for (int i = 0; i < kKinds; ++i) keep_launches[i] = c->launches[i];
  c->profile = 0;
  double phi0 = 0.0;
  st = misfit_now(c, &phi0);
  c->object = tz;
  c->probe = tq;
  // 1. B: the largest misfit decrease per second, ln(Phi_0 / Phi_end) / t
  int best_b = c->par.minibatch;
  double best_rate = -1e300, best_ms = 0.0;
  std::vector<int32_t> cands(req->minibatch, req->minibatch + req->n_minibatch);
  if (cands.empty()) cands.push_back(c->par.minibatch);
  for (int32_t b : cands) {
    if (st != EMG_OK) break;
    if ((st = set_minibatch_impl(c, b)) != EMG_OK) break;
    double ms = 0.0, phi = 0.0;
    if ((st = tune_trial(c, keep_o, keep_p, tz, tq, keep_epoch, req->trial_epochs, e0, e1, &ms, &phi)) != EMG_OK)
      break;
    const double rate = phi > 0.0 && phi0 > 0.0 ? std::log(phi0 / phi) / (ms * 1e-3) : (phi0 > 0.0 ? 1e300 : 0.0);
    if (rate > best_rate) {
      best_rate = rate;
      best_b = b;
      best_ms = ms / req->trial_epochs;
    }
  }
  if (st == EMG_OK) st = set_minibatch_impl(c, best_b);
  // 2. the FFT tiling at that B: time per epoch (results do not depend on it)
  int best_cluster = c->cluster;
  if (st == EMG_OK && req->tune_tiling) {
    double t_best = 1e300;
    for (int cand : {1, 2, 4, 8}) {
      if (!emg::step_supported(c->m, c->par.levels, cand)) continue;
      c->cluster = cand;
      double ms = 0.0, phi = 0.0;
      if ((st = tune_trial(c, keep_o, keep_p, tz, tq, keep_epoch, 1, e0, e1, &ms, &phi)) != EMG_OK) break;
      if (ms < t_best) {
        t_best = ms;
        best_cluster = cand;
      }
    }
    c->cluster = best_cluster;
    if (st == EMG_OK) best_ms = t_best;
  }
  // 3. the scatter mode, when non-repeatable sums are allowed
  if (st == EMG_OK && req->allow_atomic) {
    const int keep_scatter = c->par.scatter;
    const int other = keep_scatter == EMG_SCATTER_ATOMIC ? EMG_SCATTER_DETERMINISTIC : EMG_SCATTER_ATOMIC;
    double ms_keep = 0.0, ms_other = 0.0, phi = 0.0;
    st = tune_trial(c, keep_o, keep_p, tz, tq, keep_epoch, 1, e0, e1, &ms_keep, &phi);
    if (st == EMG_OK) st = set_scatter_impl(c, other);
    if (st == EMG_OK) st = tune_trial(c, keep_o, keep_p, tz, tq, keep_epoch, 1, e0, e1, &ms_other, &phi);
    if (st == EMG_OK && ms_other >= ms_keep) st = set_scatter_impl(c, keep_scatter);
    if (st == EMG_OK) best_ms = std::min(ms_keep, ms_other);
  }
  cudaStreamSynchronize(c->stream);
  c->object = keep_o;
  c->probe = keep_p;
  c->epoch = keep_epoch;
  c->profile = keep_profile;
  if (st != EMG_OK) {  // leave the settings as they were (best effort; the error is reported)
    c->cluster = keep_cl;
    set_minibatch_impl(c, keep_b);
    set_scatter_impl(c, keep_sc);
  }
  for (int i = 0; i < kKinds; ++i) c->launches[i] = keep_launches[i];
  drop_graphs(c);  // captured with the private buffers
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(tz);
  cudaFree(tq);
  if (st != EMG_OK) return st;
  res->minibatch = c->par.minibatch;
  res->cluster = c->cluster;
  res->scatter = c->par.scatter;
  res->ms_per_epoch = best_ms;
  res->misfit_rate = best_rate;
  return EMG_OK;
}

emg_status emg_autotune(emg_ctx* c, int32_t* chosen, double* ms_per_minibatch) {
  NvtxRange nvtx_range("emg_autotune");
  if (!c) return EMG_EINVAL;
  emg_status st = check_bound(c);
  if (st != EMG_OK) return st;
  DeviceGuard g(c->device);
  const int cands[] = {1, 2, 4, 8};
  const size_t nz = (size_t)c->n_rows * c->n_cols, nq = (size_t)c->m * c->m;
  float2 *tz = nullptr, *tq = nullptr;
  if (cudaMalloc(&tz, nz * sizeof(float2)) != cudaSuccess || cudaMalloc(&tq, nq * sizeof(float2)) != cudaSuccess) {
    cudaFree(tz);
    return fail(c, EMG_ENOMEM, "autotune scratch");
  }
  float2* keep_o = c->object;
  float2* keep_p = c->probe;
  const int keep_cluster = c->cluster, keep_profile = c->profile;
  int best = keep_cluster;
  double best_ms = 1e30;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int B = c->par.minibatch;
  std::vector<int32_t> idx(B);
  for (int i = 0; i < B; ++i) idx[i] = (int32_t)(((int64_t)i * 7919) % c->n_pos);
  for (int cand : cands) {
    if (!emg::step_supported(c->m, c->par.levels, cand)) continue;
    c->cluster = cand;
    c->profile = 0;
    cudaMemcpyAsync(tz, keep_o, nz * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tq, keep_p, nq * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream);
    c->object = tz;
    c->probe = tq;
    if ((st = ensure_orders(c, (size_t)c->n_pos)) != EMG_OK) break;
    cudaMemcpyAsync(c->d_orders, idx.data(), B * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    st = seed_probe_max(c, c->stream);
    for (int r = 0; r < 2 && st == EMG_OK; ++r) st = enqueue_minibatch(c, c->d_orders, B, c->d_phi, r, c->stream);
    cudaEventRecord(e0, c->stream);
    const int reps = 6;
    for (int r = 0; r < reps && st == EMG_OK; ++r) {
      if (r % 2 == 0) st = seed_probe_max(c, c->stream);
      if (st == EMG_OK) st = enqueue_minibatch(c, c->d_orders, B, c->d_phi, r, c->stream);
    }
    cudaEventRecord(e1, c->stream);
    if (st != EMG_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = cuda_fail(c, cudaGetLastError(), "autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / reps < best_ms) {
      best_ms = ms / reps;
      best = cand;
    }
  }
  cudaStreamSynchronize(c->stream);
  c->object = keep_o;
  c->probe = keep_p;
  c->profile = keep_profile;
  c->cluster = best;
  for (int i = 0; i < kKinds; ++i) c->launches[i] = 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(tz);
  cudaFree(tq);
  if (st != EMG_OK) return st;
  if (chosen) *chosen = best;
  if (ms_per_minibatch) *ms_per_minibatch = best_ms;
  return EMG_OK;
}

emg_status emg_batch_create(emg_batch** out, emg_ctx* const* ctxs, int32_t count) {
  if (!out) return EMG_EINVAL;
  *out = nullptr;
  if (!ctxs || count < 1) return EMG_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!ctxs[i] || ctxs[i]->device != ctxs[0]->device || !ctxs[i]->object || !ctxs[i]->probe) return EMG_EINVAL;
  emg_batch* b = new (std::nothrow) emg_batch();
  if (!b) return EMG_ENOMEM;
  b->ctxs.assign(ctxs, ctxs + count);
  b->device = ctxs[0]->device;
  DeviceGuard g(b->device);
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&b->d_src, count * sizeof(int32_t*)) == cudaSuccess &&
            cudaMalloc(&b->d_dst, count * sizeof(int32_t*)) == cudaSuccess &&
            cudaMalloc(&b->d_n, count * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->d_epoch, sizeof(int)) == cudaSuccess;
  for (int i = 0; ok && i < count; ++i) {
    cudaStream_t f;
    ok = cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->forks.push_back(f);
  }
  if (!ok) {
    emg_batch_destroy(b);
    return EMG_ENOMEM;
  }
  *out = b;
  return EMG_OK;
}

emg_status emg_batch_run_epochs(emg_batch* b, int32_t n_epochs, emg_stream_t stream) {
  NvtxRange nvtx_range("emg_batch_run_epochs");
  if (!b || n_epochs < 0) return EMG_EINVAL;
  if (n_epochs == 0) return EMG_OK;
  DeviceGuard g(b->device);
  const int K = (int)b->ctxs.size();
  const cudaStream_t s = (cudaStream_t)stream;
  // every context's orders for this call (its default schedule), uploaded once
  std::vector<int32_t*> src(K), dst(K);
  std::vector<int> ns(K);
  std::vector<const void*> key;
  for (int i = 0; i < K; ++i) {
    emg_ctx* c = b->ctxs[i];
    const int N = c->n_pos;
    std::vector<int32_t> h((size_t)n_epochs * N);
    for (int32_t e = 0; e < n_epochs; ++e) permutation(c->par.seed, c->epoch + e, N, h.data() + (size_t)e * N);
    emg_status st = ensure_orders(c, h.size());
    if (st != EMG_OK) return st;
    if (cudaMemcpyAsync(c->d_orders, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return EMG_ECUDA;
    src[i] = c->d_orders;
    dst[i] = c->d_epoch_order;
    ns[i] = N;
    key.insert(key.end(), {c->d_orders, c->object, c->probe, (const void*)(intptr_t)c->cluster,
                           (const void*)(intptr_t)c->verify, (const void*)(intptr_t)c->profile,
                           (const void*)(intptr_t)c->par.minibatch, (const void*)(intptr_t)c->par.scatter,
                           c->d_zt});
  }
  if (cudaMemcpyAsync(b->d_src, src.data(), K * sizeof(int32_t*), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->d_dst, dst.data(), K * sizeof(int32_t*), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->d_n, ns.data(), K * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(b->d_epoch, 0, sizeof(int), s) != cudaSuccess)
    return EMG_ECUDA;
  if (!b->graph || key != b->key) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return EMG_ECUDA;
    cudaError_t ce = emg::launch_batch_orders(b->d_src, b->d_dst, b->d_n, K, b->d_epoch, b->cap);
    cudaEvent_t fork_ev, join_ev;
    cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming);
    cudaEventRecord(fork_ev, b->cap);
    emg_status st = ce == cudaSuccess ? EMG_OK : EMG_ECUDA;
    std::vector<cudaEvent_t> joins;
    for (int i = 0; i < K && st == EMG_OK; ++i) {
      cudaStreamWaitEvent(b->forks[i], fork_ev, 0);
      emg_ctx* c = b->ctxs[i];
      const int keep_profile = c->profile;
      c->profile = 0;
      int64_t before[kKinds];
      for (int k2 = 0; k2 < kKinds; ++k2) before[k2] = c->launches[k2];
      st = enqueue_epoch(c, b->forks[i]);
      for (int k2 = 0; k2 < kKinds; ++k2) {
        c->graph.counts[k2] = c->launches[k2] - before[k2];
        c->launches[k2] = before[k2];
      }
      c->profile = keep_profile;
      cudaEvent_t j;
      cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
      cudaEventRecord(j, b->forks[i]);
      cudaStreamWaitEvent(b->cap, j, 0);
      joins.push_back(j);
    }
    if (st == EMG_OK) ce = emg::launch_epoch_advance(b->d_epoch, b->cap);
    cudaGraph_t gr = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->cap, &gr);
    cudaEventDestroy(fork_ev);
    cudaEventDestroy(join_ev);
    for (cudaEvent_t j : joins) cudaEventDestroy(j);
    if (st != EMG_OK || ce != cudaSuccess || ee != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return st != EMG_OK ? st : EMG_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (ie != cudaSuccess) {
      b->graph = nullptr;
      return EMG_ECUDA;
    }
    b->key = key;
  }
  for (int32_t e = 0; e < n_epochs; ++e) {
    if (cudaGraphLaunch(b->graph, s) != cudaSuccess) return EMG_ECUDA;
    for (emg_ctx* c : b->ctxs)
      for (int k2 = 0; k2 < kKinds; ++k2) c->launches[k2] += c->graph.counts[k2];
  }
  for (emg_ctx* c : b->ctxs) c->epoch += n_epochs;
  return cudaGetLastError() == cudaSuccess ? EMG_OK : EMG_ECUDA;
}

void emg_batch_destroy(emg_batch* b) {
  if (!b) return;
  {
    DeviceGuard g(b->device);
    if (b->cap) cudaStreamSynchronize(b->cap);
    cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaStream_t f : b->forks) cudaStreamDestroy(f);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->d_src);
    cudaFree(b->d_dst);
    cudaFree(b->d_n);
    cudaFree(b->d_epoch);
  }
  delete b;
}

emg_status emg_set_profiling(emg_ctx* c, int32_t enable) {
  if (!c) return EMG_EINVAL;
  c->profile = enable ? 1 : 0;
  return EMG_OK;
}

emg_status emg_profile_read(emg_ctx* c, double* ms, int64_t* launches) {
  if (!c) return EMG_EINVAL;
  if (!ms || !launches) return fail(c, EMG_EINVAL, "NULL output");
  DeviceGuard g(c->device);
  EMG_CUDA(c, cudaStreamSynchronize(c->stream));
  double acc[kKinds] = {0, 0, 0, 0, 0};
  for (auto& mk : c->ev_marks) {
    float t = 0.f;
    EMG_CUDA(c, cudaEventElapsedTime(&t, mk.second.first, mk.second.second));
    acc[mk.first] += t;
  }
  for (int i = 0; i < kKinds; ++i) {
    ms[i] = acc[i];
    launches[i] = c->launches[i];
    c->launches[i] = 0;
  }
  c->ev_marks.clear();
  c->ev_used = 0;
  return EMG_OK;
}

emg_status emg_last_error(const emg_ctx* c, const char** msg) {
  if (!c || !msg) return EMG_EINVAL;
  *msg = c->err.c_str();
  return EMG_OK;
}

void emg_destroy(emg_ctx* c) {
  if (!c) return;
  {
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_all(c);
  }
  delete c;
}

}  // extern "C"

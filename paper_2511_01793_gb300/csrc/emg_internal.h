// Internal interface between the C ABI layer (emg_capi.cu) and the kernels
// (emg_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace emg {

constexpr int kMaxLevels = 7;

// Index-check sites of the bounds-check build (-DEMG_BOUNDS_CHECK): bit i of
// the device error word (emg_debug_bounds_errors) records a failed check at
// site i; the access is then skipped (a load reads 0 or index 0 instead).
enum BoundsSite : int {
  kBcOrder = 0,        // step kernels: order entry outside 0..n_pos-1
  kBcPatchWrite = 1,   // step kernels: minibatch slot outside 0..b-1
  kBcLevel = 2,        // step kernel: multigrid level array index
  kBcApplyOrder = 3,   // combine: order entry outside 0..n_pos-1
  kBcApplyPatch = 4,   // combine: patch slot outside 0..b-1
  kBcApplyObject = 5,  // combine: object index
};
// Reads and clears the error word (cudaErrorNotSupported without the checks).
cudaError_t bounds_errors_take(unsigned* out);
// One failing check (site kBcLevel) whose access is skipped; then bounds_errors_take.
cudaError_t bounds_probe(unsigned* out);

// Probe-only multigrid arrays of one minibatch (Sec. 3.2, Eq. def_weights and
// Eq. downsampled_terms).  Level l has side m >> l.
//   G[l]  = conj(Q_l) / (u_l + |Q_l|^2)               (closed-form gain, 0/0 := 0)
//   Q[l]  = I_h^H Q_{l-1} (Q[0] is the probe itself)
//   Wz[l] = |Q_l|^2 / (I_H^h I_h^H |Q_l|^2)            (l < L-1)
//   WR[l] = (I_H^h Q_{l+1}) conj(Q_l) / (I_H^h I_h^H |Q_l|^2)  (l < L-1)
struct LevelArrays {
  const float2* G[kMaxLevels];
  const float2* Q[kMaxLevels];
  const float* Wz[kMaxLevels];
  const float2* WR[kMaxLevels];
};

struct PrepArgs {
  const float2* probe;
  int m, levels, prolong;
  float alpha, w_eps;
  // max|Q|^2 of the probe as float bits: read from mq_read; mq_next is reset
  // to 0 for the combine that follows to fill (atomicMax).
  const unsigned* mq_read;
  unsigned* mq_next;
  int tile, halo;               // tiled prep: level-0 tile side and halo (px)
  float* wq;                    // [m*m] |Q|^2 + w_eps max|Q|^2 (object-combine weight)
  float* u[kMaxLevels];         // per-level rPIE weight u_l (scratch)
  float* T[kMaxLevels];         // per-level I_h^H |Q_l|^2 (side (m >> l) / 2, scratch)
  float2* G[kMaxLevels];
  float2* Q[kMaxLevels];        // Q[0] unused (the probe)
  float* Wz[kMaxLevels];
  float2* WR[kMaxLevels];
};

struct StepArgs {
  const float2* object;
  const float2* probe;
  const int32_t* pos;
  const float* amp;             // sqrt(max(d,0)) in the FFT's storage order, [N][m][m]
  const int32_t* order;         // positions of this minibatch, [b]
  const unsigned* mq;           // max|Q|^2 of the probe (float bits), read by the cluster step
  int n_rows, n_cols;
  int n_pos, b;                 // positions of the problem and of this minibatch (index checks)
  int levels, prolong, joint, verify;
  int cluster;                  // CTAs per position: 1 (m <= 32 only), 2, 4 or 8 (m = 256)
  float alpha;                  // rPIE constant (level-0 gain formed in the cluster step)
  LevelArrays lv;
  float2* zt;                   // [b][m*m] joint-step object patches z~_k
  float2* qt;                   // [b][m*m] joint-step probes Q~_k
  float* mu;                    // [b] max |z_k|^2
  double* phi;                  // [b] Phi_k at the snapshot
  double* phi_after;            // [b] Phi~_k(Q~, z~_k) (verify only)
  // atomic object scatter (EMG_SCATTER_ATOMIC): z~_k goes straight into object-sized
  // accumulators instead of zt; null for the deterministic scatter
  int combine;
  float w_eps;                  // weight floor of the weighted mean, relative to max|Q|^2
  float2* s_num;                // [n_rows][n_cols] sum w z~ (weighted mean) or sum (z~ - z_k)
  float* s_den;                 // [n_rows][n_cols] sum w (weighted mean)
  // tensor-core DFT path: R_k from outside and the misfit partial sums of each position
  const float2* r_in;           // [b][m][m] natural order, or null (FFT path)
  const double* r_partial;      // [b][r_tiles] sums of (|Psi| - a)^2
  int r_tiles;
  // Probe prep fused into the launch (prep_clusters > 0, cluster kernels on the
  // FFT path): every cluster takes a ticket (sync[0] - ticket_base) when it
  // starts; tickets below prep_clusters compute the tiles of `prep`, the rest
  // take the minibatch's positions in ticket order and, before the multigrid
  // phase, wait (bounded) until sync[1] reaches prep_target.  Both counters
  // grow across the launches of an epoch and are zeroed with max|Q|^2.
  PrepArgs prep;
  int prep_clusters, prep_tiles;
  unsigned ticket_base, prep_target;
  unsigned* sync;               // [0] tickets, [1] prep tiles done, [2] wait gave up (error flag)
};

struct ApplyArgs {
  float2* object;
  float2* probe;
  const int32_t* pos;
  const int32_t* order;
  int b, n_rows, n_cols, m, combine;
  int n_pos;                    // positions of the problem (index checks)
  const float2* zt;
  const float2* qt;
  const float* mu;
  const float* wq;
  unsigned* mq_next;            // receives max|Q|^2 of the combined probe (atomicMax, float bits)
  int tiles_x, tiles_y;         // object tiles of kApplyTile x kApplyTile pixels
  float2* s_num;                // atomic scatter: the step's accumulators, finalised and reset here
  float* s_den;
};

// Forward-only cluster kernels (m up to 256): misfit partials, simulated
// intensities, forward / inverse 2-D DFT of natural-order tiles.
struct FwdArgs {
  const float2* object;
  const float2* probe;
  const int32_t* pos;
  const float* amp;             // storage order (misfit)
  int n_rows, n_cols;
  double* partial;              // [count] misfit per position (mode 0)
  float* out_intensity;         // [count][m][m] natural order (mode 1)
  const float2* in;             // [count][m][m] natural order (modes 2, 3)
  float2* out;                  // [count][m][m] natural order (modes 2, 3)
};

// Wirtinger gradients of the exit-wave misfit per position (Sec. 2.1):
// gz_k = conj(Q) (psi_k - R_k), gq_k = conj(z_k) (psi_k - R_k).
struct GradArgs {
  const float2* object;
  const float2* probe;
  const int32_t* pos;
  const float* amp;
  int first, n_rows, n_cols;    // positions first .. first + b - 1
  float2* gz;                   // [b][m][m]
  float2* gq;                   // [b][m][m]
  double* phi;                  // [b]
};

// Sums the patch gradients of one chunk into the object / probe gradients.
struct GradReduceArgs {
  const int32_t* pos;
  int first, b, n_rows, n_cols, m, accumulate;
  const float2* gz;
  const float2* gq;
  float2* grad_object;          // [n_rows][n_cols] or null
  float2* grad_probe;           // [m][m] or null
  int tiles_x, tiles_y;
};

cudaError_t launch_gradient(int m, int b, const GradArgs& a, cudaStream_t s);
// Positions whose gradient clusters are resident on the device at once (0 if unknown).
int gradient_positions_per_wave(int m);
cudaError_t launch_grad_reduce(const GradReduceArgs& a, cudaStream_t s);
bool step_supported(int m, int levels, int cluster);
int default_cluster(int m, int levels);
// Copies, for each of `count` problems, its order row `*epoch` into its epoch buffer.
cudaError_t launch_batch_orders(const int32_t* const* src, int32_t* const* dst, const int* n, int count,
                                const int* epoch, cudaStream_t s);
cudaError_t launch_epoch_advance(int* epoch, cudaStream_t s);

// Combine object tiles: kApplyTile rows x kApplyTileW columns, kApplyPx pixels
// per thread (the gradient sums use kApplyTile^2 tiles, one pixel per thread).
#ifndef EMG_APPLY_PX
#define EMG_APPLY_PX 2
#endif
#ifndef EMG_APPLY_PROBE_PX
#define EMG_APPLY_PROBE_PX 2
#endif
constexpr int kApplyTile = 16;
constexpr int kApplyPx = EMG_APPLY_PX;
constexpr int kApplyTileW = kApplyTile * kApplyPx;
constexpr int kApplyThreads = 256;
constexpr int kApplyProbeGroups = 8;   // probe blocks: kApplyProbePx pixels x 8 position groups
constexpr int kApplyProbePx = 32 * EMG_APPLY_PROBE_PX;
inline int apply_tiles_x(int n_cols) { return (n_cols + kApplyTileW - 1) / kApplyTileW; }
inline int apply_tiles_y(int n_rows) { return (n_rows + kApplyTile - 1) / kApplyTile; }

cudaError_t upload_twiddles();
cudaError_t launch_amp_prep(const float* d, float* amp, int m, int n_pos, cudaStream_t s);
// a_k of positions idx[0..b) (device indices) from d, which may be mapped host memory.
cudaError_t launch_amp_gather(const float* d, const int32_t* idx, int b, float* amp, int m, cudaStream_t s);
cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s);
// Fused probe prep for the cluster step kernel: sets a.tile / a.halo for it
// and returns its tile count, or 0 when it does not fit beside the step.
int fused_prep_tiles(PrepArgs& a, int m, int cluster);
// Step-kernel clusters that can be resident on the device at once (0 if unknown).
int step_resident_clusters(int m, int cluster);
cudaError_t launch_probe_max(const float2* probe, int m, unsigned* slot, cudaStream_t s);
// Fills tile/halo of a and returns true when the tiled prep fits in shared memory.
bool prep_tiled_config(PrepArgs& a);
cudaError_t launch_step(int m, int b, const StepArgs& a, cudaStream_t s);
// The step with R_k and the misfit partials given (a.r_in, a.r_partial): m = 128 (cluster 2, 4), 256 (8).
cudaError_t launch_step_rin(int m, int b, const StepArgs& a, cudaStream_t s);
cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t s);
cudaError_t launch_misfit(int m, const float2* object, const float2* probe, const int32_t* pos,
                          const float* amp, int n_rows, int n_cols, int n_pos, double* partial,
                          cudaStream_t s);
cudaError_t launch_sum(const double* x, int n, double scale, double* out, cudaStream_t s);
cudaError_t launch_simulate(int m, const float2* object, const float2* probe, const int32_t* pos,
                            int n_rows, int n_cols, int n_pos, float* out, cudaStream_t s);
cudaError_t launch_fft2(int m, const float2* in, float2* out, int count, int inverse,
                        cudaStream_t s);
cudaError_t launch_normalize_probe(const float* amp, int m, int n_pos, float2* probe,
                                   double* scratch, int scratch_len, cudaStream_t s);
size_t step_smem_bytes(int m, int levels);

// Tensor-core DFT pair (BF16 split into three products, FP32 accumulation) for
// m = 128 and 256; see emg_tc.cu.  A TcWork holds the split operand buffers of
// up to `cap` tiles and their TMA descriptors.
struct TcWork;
struct TcStepArgs {
  const float2* object;
  const float2* probe;
  const int32_t* pos;
  const int32_t* order;         // [b] positions of the minibatch
  int n_rows, n_cols, b;
  const float* amp_t;           // [N][m][m] a_k transposed
  float2* R;                    // [b][m][m] out: revised exit waves, natural order
  double* partial;              // [b][tc_tiles_per_position(m)] out: sums of (|Psi| - a)^2
};
bool tc_supported(int m);
bool tc_radix16(int m);  // m = 256 and EMG_TC_RADIX16 is not "0..."
cudaError_t tc_work_create(TcWork** out, int m, int cap);
void tc_work_destroy(TcWork* w);
int* tc_error_flag(TcWork* w);
int tc_tiles_per_position(int m);
// count tiles of m x m complex64: out = F x (inverse = 0) or F^-1 x (inverse = 1).
cudaError_t tc_dft2(TcWork* w, const float2* in, float2* out, int count, int inverse, cudaStream_t s);
// a1-a4 of a minibatch: psi_k, Psi_k, modulus replacement, R_k.
cudaError_t tc_exit_waves(TcWork* w, const TcStepArgs& a, cudaStream_t s);
cudaError_t launch_tc_amp(const float* d, float* amp_t, int m, int n_pos, cudaStream_t s);
// One bounded mbarrier wait that nothing satisfies; sets *err when it gives up.
cudaError_t launch_wait_selftest(int* err, cudaStream_t s);
int step_smem_limit();

}  // namespace emg

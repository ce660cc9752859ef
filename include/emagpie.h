/*
 * emagpie.h - C ABI of the GB300 (sm_103a) eMAGPIE hot path.
 *
 * eMAGPIE (arXiv 2511.01793) jointly reconstructs a complex object z
 * (n_rows x n_cols) and a complex probe Q (m x m) from far-field intensities
 * d_k = |F(Q . P_k z)|^2 + noise, k = 0..N-1 (Sec. 2.1).  One epoch visits a
 * random permutation of the scan positions (Sec. 3, stochastic sweep) in
 * minibatches of B positions.  For each position k of a minibatch the library:
 *
 *   1. gathers z_k = P_k z (zero outside the object) and forms psi = Q . z_k;
 *   2. takes Psi = F psi, replaces its modulus by a_k = sqrt(max(d_k, 0)) and
 *      takes R_k = F^-1 of the result (Def. 2.1, revised exit wave);
 *   3. computes the MAGPIE object step z+ with L multigrid levels (Sec. 3.2)
 *      and the ePIE probe step Q+ (Sec. 4, Eq. qplus_proximal);
 *   4. fuses them into the geometric-mean, phase-aligned joint step
 *      (z~, Q~) of Eq. (geomean);
 * then combines the B patches into the object and the B probe estimates into
 * the probe (see emg_params.combine).  All positions of a minibatch see the
 * same snapshot (z, Q); B = 1 is exactly the paper's sequential sweep.
 *
 * Conventions shared by every entry point:
 *  - Complex arrays are complex64: interleaved (re, im) float pairs, row-major.
 *  - F is the unnormalised forward 2-D DFT; F^-1 carries 1/m^2; DC at [0][0].
 *  - The caller owns every pointer it passes; the library owns the scratch it
 *    allocates in emg_create and frees it in emg_destroy.
 *  - Calls are asynchronous on the context's stream unless they write host
 *    memory, in which case they synchronise that stream before returning.
 *  - No C++ exception or abort crosses this ABI.  Argument errors return
 *    EMG_EINVAL before any device work is enqueued; CUDA errors return
 *    EMG_ECUDA; emg_last_error() gives a message for the last failure.
 *  - One context per stream; a context is not thread-safe.
 */
#ifndef EMAGPIE_H
#define EMAGPIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum emg_status {
  EMG_OK = 0,
  EMG_EINVAL = 1,   /* invalid argument (detected before any launch) */
  EMG_ENOMEM = 2,   /* device or pinned host allocation failed */
  EMG_ECUDA = 3,    /* a CUDA call or kernel failed */
  EMG_ETIMEOUT = 4, /* a bounded device wait gave up */
  EMG_ENOTSUP = 5   /* valid request that this library does not implement */
} emg_status;

enum { EMG_PROLONG_CONST = 0, EMG_PROLONG_BILINEAR = 1 };
enum { EMG_COMBINE_WAVG = 0, EMG_COMBINE_SUM = 1 };
enum { EMG_SCATTER_DETERMINISTIC = 0, EMG_SCATTER_ATOMIC = 1 };
enum { EMG_DFT_FFT32 = 0, EMG_DFT_BF16X3 = 1 };

/* Same object as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* emg_stream_t;

typedef struct emg_ctx emg_ctx;     /* opaque, library-owned */
typedef struct emg_batch emg_batch; /* opaque, library-owned */

/*
 * The problem of Sec. 2.1: object size, probe size m, scan positions P_k
 * and data d_k.
 *  pos        device int32 [n_pos][2]: (row, col) of the top-left corner of
 *             patch k in object pixels.  A patch may extend past the object;
 *             P_k zero-pads (Sec. 2.1).  |row|, |col| must be < 2^24.
 *  intensity  device float32 [n_pos][m][m]: d_k with DC at [0][0].  Negative
 *             values are clamped to 0 before the square root.  Read only
 *             during emg_create (the library keeps sqrt(d) in its own layout).
 *  m          16, 32, 64, 128 or 256.
 */
typedef struct emg_problem {
  int32_t n_rows, n_cols;
  int32_t m;
  int32_t n_pos;
  const int32_t* pos;
  const float* intensity;
} emg_problem;

/*
 * Hyper-parameters (Sec. 3, 3.2 and 4).
 *  alpha      rPIE constant of the object weight u_Q = alpha (max|Q|^2 - |Q|^2), > 0.
 *  levels     multigrid levels L >= 1 of the MAGPIE object step; m / 2^(L-1) >= 2.
 *             L = 2 is the paper's pair of levels; L > 2 applies it recursively.
 *  minibatch  positions per minibatch B >= 1 (1 = the paper's sequential sweep).
 *  prolong    EMG_PROLONG_CONST: I_H^h = 4 (I_h^H)^T, piecewise-constant (paper);
 *             EMG_PROLONG_BILINEAR: cell-centred bilinear, edge-clamped.
 *             Restriction I_h^H is always the 2x2 average.
 *  combine    EMG_COMBINE_WAVG: covered object pixels become
 *               sum_k w_k z~_k / sum_k w_k, w_k(p) = |Q(p - o_k)|^2 + w_eps max|Q|^2,
 *             and the probe the mean of Q~_k over positions with max|z_k| > 0;
 *             EMG_COMBINE_SUM: z += sum_k (z~_k - z_k), Q += sum_k (Q~_k - Q).
 *  scatter    EMG_SCATTER_DETERMINISTIC (default): the combine sums the B patches
 *             of every object pixel in minibatch order (bitwise repeatable);
 *             EMG_SCATTER_ATOMIC: the step kernel adds each patch into
 *             object-sized FP32 accumulators with atomics and the combine only
 *             finalises them (equal up to rounding order, not bitwise
 *             repeatable; the weighted mean then needs w_eps > 0).
 *  joint      1: geometric-mean joint step (eMAGPIE); 0: take z+ and Q+ as they
 *             are (the rPIE-style simultaneous update of Sec. 2.2).
 *  w_eps      weight floor of the object combine, relative to max|Q|^2, >= 0.
 *  dft        EMG_DFT_FFT32: the FFT pair a2 / a4 as FP32 shared-memory FFTs
 *             inside the step kernel (default);
 *             EMG_DFT_BF16X3: the pair as tensor-core GEMMs in BF16 with every
 *             operand split into high and low parts (see emg_dft2_bf16x3);
 *             m = 128 or 256 only (EMG_ENOTSUP otherwise).  The misfit of
 *             emg_misfit is always evaluated on the FP32 path.  The tensor-
 *             core kernels bound every wait; one that gives up is reported as
 *             EMG_ETIMEOUT by the next call that synchronises (emg_misfit,
 *             emg_run_epochs with host output, a sampled emg_step_minibatch).
 *  seed       schedule seed used when emg_run_epochs gets no order array.
 */
typedef struct emg_params {
  float alpha;
  int32_t levels;
  int32_t minibatch;
  int32_t prolong;
  int32_t combine;
  int32_t scatter;
  int32_t joint;
  float w_eps;
  int32_t dft;
  uint64_t seed;
} emg_params;

/* Fills *p with alpha 0.01, L 1, B 1, CONST, WAVG, DETERMINISTIC, joint 1, w_eps 1e-6,
 * EMG_DFT_FFT32, seed 0. */
emg_status emg_default_params(emg_params* p);

/* Human-readable name of a status code (static string). */
const char* emg_status_string(emg_status s);

/*
 * Creates a context bound to `stream` on the current CUDA device, validates
 * the problem and parameters, allocates the scratch (sqrt-intensities in the
 * FFT's storage order, per-minibatch patch buffers, multigrid level arrays)
 * and derives a_k = sqrt(max(d_k, 0)) from problem->intensity.
 * On failure *out is NULL and nothing stays allocated.
 */
emg_status emg_create(emg_ctx** out, const emg_problem* problem,
                      const emg_params* params, emg_stream_t stream);

/*
 * Replaces the data d_k (same shape as at creation).  `intensity` may be a
 * device pointer or a host pointer.  Pinned host memory is read in place by
 * the amplitude kernel, asynchronously on the context's stream (through a
 * device staging copy on the tensor-core DFT path); pageable memory is staged
 * synchronously.  The caller keeps pinned data unchanged until the stream has
 * passed this call.
 */
emg_status emg_set_intensity(emg_ctx* ctx, const float* intensity);

/*
 * Binds the caller-owned state: object = device complex64 [n_rows][n_cols],
 * probe = device complex64 [m][m].  Both are updated in place by the step
 * entry points.  Fails with EMG_EINVAL for a NULL pointer.
 */
emg_status emg_bind_state(emg_ctx* ctx, float* object, float* probe);

/*
 * Scales the bound probe to the data, Q <- Q dp_avg / ||Q||_2 with
 * dp_avg = sqrt(sum_ij mean_k d_k[i][j]) / m (Sec. 4.1).
 */
emg_status emg_normalize_probe(emg_ctx* ctx);

/*
 * One minibatch: positions idx[0..b-1] (host int32, each in [0, n_pos)),
 * 1 <= b <= the context's minibatch size (params.minibatch, or the last
 * emg_set_minibatch).  Updates the bound object and probe.
 * If sampled_misfit (host) is not NULL it receives sum_k Phi_k at the
 * snapshot, Phi_k = 1/2 ||Q . z_k - R_k||^2 (Eq. exit_misfit), and the call
 * synchronises.
 */
emg_status emg_step_minibatch(emg_ctx* ctx, const int32_t* idx, int32_t b,
                              double* sampled_misfit);

/*
 * Per-position diagnostics of the last emg_step_minibatch, copied to host
 * out[b][3] = { Phi_k at the snapshot, Phi~_k(Q~, z~_k) after the joint step
 * (the sampled surrogate of Eq. quadratic_surrogate, Prop. 3.2), max|z_k|^2 }.
 * Phi~ after is NaN unless emg_set_verify(ctx, 1) was called.  Synchronises.
 */
emg_status emg_position_stats(emg_ctx* ctx, double* out, int32_t b);

/* verify = 1 makes the step kernel also evaluate Phi~_k after the joint step. */
emg_status emg_set_verify(emg_ctx* ctx, int32_t verify);

/*
 * Runs n_epochs epochs.  order: host int32 [n_epochs][n_pos], each row a
 * permutation of 0..n_pos-1, or NULL to draw the permutation of epoch e from
 * emg_schedule_permutation(params.seed, e, n_pos) where e counts the epochs
 * this context has run (see emg_set_epoch).  Each epoch is cut into
 * consecutive minibatches of the context's minibatch size (the last may be
 * shorter).  running_misfit (host [n_epochs] or NULL) receives the sum over
 * the epoch of the sampled Phi_k; misfit (host [n_epochs] or NULL) receives
 * Phi(Q, z) at the end of each epoch from a separate forward pass.  The call
 * synchronises iff it writes host output.
 */
emg_status emg_run_epochs(emg_ctx* ctx, int32_t n_epochs, const int32_t* order,
                          double* running_misfit, double* misfit);

/*
 * Exit-wave misfit and its Wirtinger gradients (Sec. 2.1) at an arbitrary
 * (object, probe), which need not be the bound state:
 *   Phi = 1/2 sum_k ||Q . P_k z - R_k(Q, P_k z)||^2,
 *   grad_z Phi = sum_k P_k^T [conj(Q) (Q . P_k z - R_k)],
 *   grad_Q Phi = sum_k conj(P_k z) (Q . P_k z - R_k),
 * in the convention d/dRe + i d/dIm (twice the conjugate Wirtinger derivative,
 * the convention PyTorch uses for complex autograd).  R_k is recomputed (no
 * exit waves are stored); positions are processed in chunks (by default a
 * multiple of the position clusters that can be resident at once, about 128
 * positions; see emg_set_gradient_chunk) and summed in a fixed order, so
 * results repeat bitwise for a given chunk size.  The first call may allocate
 * the chunk's patch buffers.
 *  object, probe            device complex64 [n_rows][n_cols], [m][m] (read only)
 *  grad_object, grad_probe  device complex64, same shapes, overwritten; either may be NULL
 *  misfit                   host double or NULL (synchronises when not NULL)
 */
emg_status emg_misfit_gradient(emg_ctx* ctx, const float* object, const float* probe,
                               float* grad_object, float* grad_probe, double* misfit);

/*
 * Positions per launch of emg_misfit_gradient: 0 (the default) chooses a
 * multiple of the position clusters that can be resident at once, about 128
 * positions; n > 0 takes n.  The chunk only
 * changes speed and the rounding order of the sums.  Synchronises the
 * context's stream and frees the previous chunk's buffers.  EMG_EINVAL for
 * n < 0.
 */
emg_status emg_set_gradient_chunk(emg_ctx* ctx, int32_t positions);

/* Phi(Q, z) = 1/2 sum_k ||Q . P_k z - R_k||^2 of the bound state (host *out; synchronises). */
emg_status emg_misfit(emg_ctx* ctx, double* out);

/* Sets the epoch counter used by the default schedule (checkpoint / resume). */
emg_status emg_set_epoch(emg_ctx* ctx, int64_t epoch);

/*
 * Host-only: the stopping criterion of Sec. 4.1 and the noise-floor rule of
 * Sec. 4.3 applied to residuals r[0..n-1] (r[t-1] = Phi after outer iteration
 * t).  For t >= window the moving average of the last `window` residuals is
 * formed; a check counts when that average is not below the best of the
 * earlier averages (an improvement resets the count), and the run stops at the
 * first t at which the count reaches `patience`.  With floor > 0 (Phi at the
 * true object and probe on the noisy data) it also stops at the first t with
 * r_t < 0.9 floor.  *out receives that t (1-based), or 0 if the run does not
 * stop within the n residuals.  EMG_EINVAL for n < 0, window or patience < 1,
 * a negative or non-finite floor, or a NULL pointer that is needed.
 */
emg_status emg_stopping_epoch(const double* r, int32_t n, int32_t window, int32_t patience, double floor,
                              int32_t* out);

/*
 * Runs epochs (default schedule) one at a time, evaluating Phi after each as
 * emg_misfit does, until the rules of emg_stopping_epoch stop the run or
 * max_epochs have run.  epochs_run (host) receives the number of epochs;
 * misfit (host [max_epochs], or NULL) the residual after each.  Synchronises
 * once per epoch.
 */
emg_status emg_run_until(emg_ctx* ctx, int32_t max_epochs, int32_t window, int32_t patience, double floor,
                         int32_t* epochs_run, double* misfit);

/*
 * Host-only: the default schedule's permutation of 0..n-1 for one epoch.
 * SplitMix64 (Steele, Lea, Flood 2014) seeded with
 * seed + epoch * 0x9E3779B97F4A7C15 (mod 2^64), then Fisher-Yates from
 * i = n-1 down to 1 swapping i with (next() mod (i + 1)).  out: host [n].
 */
emg_status emg_schedule_permutation(uint64_t seed, int64_t epoch, int32_t n, int32_t* out);

/*
 * End-to-end call on host buffers: takes intensity (host [n_pos][m][m]) as
 * emg_set_intensity does, copies object (host complex64 [n_rows][n_cols]) and
 * probe (host complex64 [m][m]) to library-owned device buffers, runs
 * n_epochs as emg_run_epochs does and copies object and probe back.  The
 * context's bound device state is not touched.  Synchronises once: for up to
 * 31 epochs the misfit histories and the flag of the step kernel's bounded
 * wait come back through the context's pinned scratch beside the object and
 * the probe; a wait that gave up returns EMG_ETIMEOUT after the copies.
 */
emg_status emg_reconstruct_host(emg_ctx* ctx, const float* intensity, float* object,
                                float* probe, int32_t n_epochs, const int32_t* order,
                                double* running_misfit, double* misfit);

/*
 * Forward model of Sec. 2.1 without a context: d_k = |F(Q . P_k z)|^2 for
 * k = 0..n_pos-1.  object device complex64 [n_rows][n_cols], probe device
 * complex64 [m][m], pos device int32 [n_pos][2], out device float32
 * [n_pos][m][m] (DC at [0][0]).  Asynchronous on `stream`.
 */
emg_status emg_simulate_intensity(const float* object, int32_t n_rows, int32_t n_cols,
                                  const float* probe, int32_t m, const int32_t* pos,
                                  int32_t n_pos, float* out, emg_stream_t stream);

/*
 * One minibatch split across ranks (one process per GPU, each with its own
 * context on identical state and data).  The minibatch's slots 0..b-1 (slot k
 * holds position idx[k]) are divided among the ranks; each rank steps its own
 * slots against the shared snapshot (z, Q), the ranks exchange the results
 * (one all-gather of the slot buffers), and every rank then combines all b
 * slots in slot order, so all ranks end with bitwise the same state, equal to
 * emg_step_minibatch on one GPU.  The paper's sweep has batch 1 (Sec. 4.4);
 * this is the minibatch reading of the sweep with its positions spread over
 * devices.
 *
 * emg_shard_step: probe prep and the per-position step (a0-a7) for slots
 *   [slot_begin, slot_end); writes z~_k to zt + k m^2, Q~_k to qt + k m^2
 *   (complex64) and max|z_k|^2 to mu + k for each of those slots.  The bound
 *   object and probe are not changed.  slot_begin == slot_end is allowed (the
 *   rank has no position in this minibatch).
 * emg_shard_apply: the combine (a8, a9) of all b slots read from zt, qt, mu,
 *   which by then hold every rank's slots; updates the bound object and probe.
 *  idx, b   host int32 [b], the whole minibatch, the same on every rank
 *  zt, qt   device complex64 [>= b][m][m], caller-owned
 *  mu       device float32 [>= b], caller-owned
 * EMG_ENOTSUP with the atomic scatter (it has no per-slot patches to
 * exchange).  Asynchronous on the context's stream; the caller orders its
 * exchange on that stream between the two calls.
 */
emg_status emg_shard_step(emg_ctx* ctx, const int32_t* idx, int32_t b, int32_t slot_begin,
                          int32_t slot_end, float* zt, float* qt, float* mu);
emg_status emg_shard_apply(emg_ctx* ctx, const int32_t* idx, int32_t b, const float* zt,
                           const float* qt, const float* mu);

/*
 * Reconstruction errors with the scale ambiguity removed, reduced on the GPU
 * in FP64.  Blind ptychography determines (z, Q) only up to (c z, Q / c) for a
 * complex c != 0: the exit waves Q . P_k z of Sec. 2.1, and so the data, do
 * not change.  The call takes the best c over a region of the object,
 *   c = <z, z_ref> / <z, z>     (<a, b> = sum over the region of conj(a) b),
 * and returns in out (host double[5]):
 *   out[0], out[1]  Re c, Im c
 *   out[2]          ||c z - z_ref|| / ||z_ref|| over the region
 *   out[3]          ||Q / c - Q_ref|| / ||Q_ref|| over the whole probe
 *   out[4]          RMS over the region of arg(c z conj(z_ref)) (radians)
 *  object, object_ref  device complex64 [n_rows][n_cols]
 *  probe, probe_ref    device complex64 [m][m]
 *  region              device uint8 [n_rows][n_cols], nonzero = inside; NULL = every pixel
 * Sums run in a fixed order, so the result is bitwise repeatable.  Allocates
 * a small scratch buffer (EMG_ENOMEM if that fails) and synchronises `stream`.
 */
emg_status emg_aligned_errors(const float* object, const float* object_ref, int32_t n_rows,
                              int32_t n_cols, const float* probe, const float* probe_ref, int32_t m,
                              const uint8_t* region, double* out, emg_stream_t stream);

/*
 * The well-illuminated region of the scan, the comparison region of
 * emg_aligned_errors: region[p] = 1 where sum_k |probe_ref(p - o_k)|^2 >=
 * frac * (its maximum over the object), else 0 (o_k = pos[k], the patch
 * corners of Sec. 2.1; pixels a patch does not cover add nothing).  The sums
 * are FP64 over k = 0..n_pos-1 in index order.
 *  probe_ref  device complex64 [m][m]
 *  pos        device int32 [n_pos][2]
 *  region     device uint8 [n_rows][n_cols], written
 * Allocates n_rows n_cols doubles of scratch and synchronises `stream`.
 */
emg_status emg_illuminated_region(const float* probe_ref, int32_t m, const int32_t* pos,
                                  int32_t n_pos, int32_t n_rows, int32_t n_cols, double frac,
                                  uint8_t* region, emg_stream_t stream);

/*
 * Batched 2-D DFT of count m x m complex64 tiles (device, natural order in
 * and out): inverse = 0 gives F x (unnormalised), inverse = 1 gives F^-1 x
 * (with 1/m^2).  in and out may alias.  Asynchronous on `stream`.
 */
emg_status emg_fft2(const float* in, float* out, int32_t m, int32_t count, int32_t inverse,
                    emg_stream_t stream);

/*
 * The same batched 2-D DFT on the tensor cores (the precision variant of the
 * FFT pair of Sec. 2.1).  Every operand is split into high and low parts in
 * BF16 (x = xh + xl, xh = bf16(x), xl = bf16(x - xh)) and the products
 * xh yh + xh yl + xl yh accumulate in FP32.  At m = 128 (and at m = 256 with
 * the environment variable EMG_TC_RADIX16=0) each 1-D pass is one GEMM of the
 * rows of all tiles with the 2m x 2m real matrix of x -> x F (or x conj(F)):
 * relative error of order 3 u^2 per pass, u = 2^-8.  At m = 256 each 1-D
 * pass is by default a radix-16 pass (256 = 16 x 16): two 16-point DFT
 * products with an FP32 twiddle multiply between them, 1/8 of the flops of the
 * dense GEMM and about twice its error (about 2e-4 in the L2 norm per 2-D
 * transform, against about 1e-7 for emg_fft2); emg_dft_bf16x3_form reports
 * which form runs.
 *  in, out  device complex64 [count][m][m], natural order; may not alias
 *  m        128 or 256 (EMG_ENOTSUP otherwise)
 * Allocates and frees its split buffers and synchronises the stream.
 * EMG_ETIMEOUT when a bounded wait inside the kernel gave up.
 */
emg_status emg_dft2_bf16x3(const float* in, float* out, int32_t m, int32_t count, int32_t inverse,
                           emg_stream_t stream);

/*
 * Which form the tensor-core DFT of size m takes in this process (the
 * variable EMG_TC_RADIX16 is read once per process): *radix16 = 1 for radix-16
 * passes (m = 256 by default), 0 for dense GEMM passes.  EMG_ENOTSUP if m is
 * not 128 or 256, EMG_EINVAL if radix16 is NULL.  Host only; launches nothing.
 */
emg_status emg_dft_bf16x3_form(int32_t m, int32_t* radix16);

/*
 * Check of the failure path of the tensor-core kernel's waits: one CTA waits,
 * with the same bounded mbarrier wait, on a barrier that nothing arrives on.
 * The wait gives up after its limit (1 s) and records that in a device flag,
 * as a stalled pipeline would; *gave_up receives the flag (1 expected).  The
 * device stays usable.  Synchronises the device.  EMG_EINVAL for NULL.
 */
emg_status emg_selftest_bounded_wait(int32_t* gave_up);

/*
 * Host-side fault injection for tests: the library's next device allocation
 * after `after` successful ones fails once (as if the device were out of
 * memory); -1 disables.  Process-wide.  EMG_EINVAL for after < -1.
 */
emg_status emg_debug_fail_alloc(int32_t after);

/*
 * Bounds-check build only (compiled with -DEMG_BOUNDS_CHECK): *mask receives
 * the error word and the word is cleared.  Bit i set: an index check at site
 * i failed and its access was skipped (sites: 0 order entry and 1 minibatch
 * slot in the step kernels, 2 multigrid level index, 3 order entry, 4 patch
 * slot and 5 object index in the combine).  Synchronous.  EMG_ENOTSUP (with
 * *mask = 0) in a build without the checks.
 */
emg_status emg_debug_bounds_errors(uint32_t* mask);

/*
 * Bounds-check build only: runs one check that must fail (an index equal to
 * its bound, site 2), whose store is skipped, and returns the error word in
 * *mask (bit 2 expected), clearing it.  Synchronises the device.  EMG_ENOTSUP
 * in a build without the checks.
 */
emg_status emg_debug_bounds_selftest(uint32_t* mask);

/*
 * FFT tiling: the number of CTAs that share one scan position in the step
 * kernel (1 or 2 for m <= 32; 2 or 4 for m = 64; 2, 4 or 8 for m = 128; 8 for
 * m = 256).  It changes speed only: results are identical for every valid
 * choice.  EMG_ENOTSUP when the choice is not built or leaves a CTA without a
 * row at the coarsest level.
 */
emg_status emg_set_cluster(emg_ctx* ctx, int32_t cluster);

/*
 * Where the probe prep of a minibatch runs: 1 (the default) inside the step
 * launch of the cluster kernels, beside the gather and transforms, when the
 * launch fits in one wave of resident clusters; 0 always as its own kernel
 * before the step.  Speed only: the results are identical.  Synchronises.
 * EMG_EINVAL for other values.
 */
emg_status emg_set_prep_fusion(emg_ctx* ctx, int32_t enable);

/*
 * Test hook for the failure path of the fused prep's wait: each later step
 * launch waits for `extra` more prep tiles than it has, so its bounded wait
 * (1 s) runs out, sets the device flag and the kernel goes on; the next call
 * that synchronises returns EMG_ETIMEOUT.  0 (the default) restores normal
 * operation.  Synchronises.
 */
emg_status emg_debug_prep_wait_extra(emg_ctx* ctx, uint32_t extra);

/*
 * Autotuner: times a few minibatches (on private copies of the bound state,
 * which is left untouched) for every valid FFT tiling and keeps the fastest.
 * chosen (host, or NULL) receives it, ms_per_minibatch (host, or NULL) its
 * time.  Synchronises.
 */
emg_status emg_autotune(emg_ctx* ctx, int32_t* chosen, double* ms_per_minibatch);

/*
 * Minibatch size B (1..n_pos) after creation.  B is part of the method: it
 * sets how many positions share one snapshot and one combine (reading of the
 * minibatch combine), so it changes results, not only speed.  Synchronises;
 * grows the per-minibatch buffers when B exceeds every earlier size.
 * EMG_EINVAL outside 1..n_pos, EMG_ENOMEM when the buffers cannot grow (the
 * context keeps its previous B).
 */
emg_status emg_set_minibatch(emg_ctx* ctx, int32_t minibatch);

/*
 * Object scatter mode after creation (EMG_SCATTER_DETERMINISTIC or
 * EMG_SCATTER_ATOMIC; see emg_params.scatter).  Synchronises; allocates the
 * atomic accumulators on first use.  EMG_EINVAL for an unknown mode or for the
 * atomic weighted mean with w_eps = 0.
 */
emg_status emg_set_scatter(emg_ctx* ctx, int32_t scatter);

typedef struct {
  const int32_t* minibatch;  /* host [n_minibatch]: candidate B values (1..n_pos) */
  int32_t n_minibatch;       /* 0: keep the context's B */
  int32_t trial_epochs;      /* >= 1: epochs each B candidate runs */
  int32_t tune_tiling;       /* 1: also choose the FFT tiling (emg_set_cluster) */
  int32_t allow_atomic;      /* 1: also try the other scatter mode; the atomic one
                                is not bitwise repeatable */
} emg_tune_request;

typedef struct {
  int32_t minibatch, cluster, scatter;  /* the configuration now set on the context */
  double ms_per_epoch;                  /* its device time per epoch */
  double misfit_rate;                   /* ln(Phi_0 / Phi_end) per second in the B trial */
} emg_tune_result;

/*
 * Autotuner over B, the FFT tiling and the scatter mode.  Every trial starts
 * from a private copy of the bound state at the context's epoch counter; the
 * bound state and the counter are left untouched.  B: each candidate runs
 * trial_epochs epochs, and the one with the largest misfit decrease per
 * second, ln(Phi_0 / Phi_end) / t, wins (B changes the iterates, so speed
 * alone cannot choose it).  Tiling and scatter mode: the fastest epoch at that
 * B (the tiling leaves results unchanged; the scatter modes differ by
 * rounding).  The winners are set on the context and returned in *result.
 * Synchronises.  EMG_EINVAL for invalid requests.
 */
emg_status emg_autotune_search(emg_ctx* ctx, const emg_tune_request* request, emg_tune_result* result);

/*
 * Batches of independent reconstructions (problems of different object, probe
 * and scan sizes).  emg_batch_create groups `count` contexts on one device,
 * each with its state bound; the contexts stay owned by the caller and must
 * outlive the batch.  emg_batch_run_epochs runs n_epochs epochs of every
 * context with its default schedule (emg_schedule_permutation from its own
 * seed and epoch counter), each epoch as ONE launch of a CUDA graph that holds
 * one branch per context; results equal running each context alone.
 * Asynchronous on `stream`.
 */
emg_status emg_batch_create(emg_batch** out, emg_ctx* const* ctxs, int32_t count);
emg_status emg_batch_run_epochs(emg_batch* batch, int32_t n_epochs, emg_stream_t stream);
void emg_batch_destroy(emg_batch* batch);

/*
 * Kernel timing for measurement (not part of the method).  enable = 1 makes
 * every later launch of the minibatch path record a pair of CUDA events on the
 * context's stream.  emg_profile_read synchronises and returns, per kernel
 * kind {probe prep, per-position step, combine, other, tensor-core DFT passes},
 * the summed event time in milliseconds (ms[5], host) and the number of
 * launches (launches[5], host; counted whether or not profiling is on) since
 * the last read, then resets.
 */
emg_status emg_set_profiling(emg_ctx* ctx, int32_t enable);
emg_status emg_profile_read(emg_ctx* ctx, double* ms, int64_t* launches);

/*
 * Allocation-free variant of emg_step_minibatch, without a context.  The paper
 * has no counterpart: it exists for callers that may not allocate device
 * memory (code running inside a memory pool or arena it does not own, code
 * whose device footprint must not grow after start-up, or code under a policy
 * that forbids cudaMalloc on its hot path).  The caller passes every input and
 * output; the call performs no device or pinned allocation of any kind.
 *
 *  object      device complex64 [n_rows][n_cols], updated in place
 *  probe       device complex64 [m][m], updated in place
 *  pos         device int32 [n_pos][2] patch corners, |row|, |col| < 2^24
 *  intensity   device float32 [n_pos][m][m] data d_k in natural order (DC at [0][0])
 *  idx, b      host int32 [b] positions of this minibatch, 1 <= b <= n_pos,
 *              b <= 2048; the indices are copied into the launch parameters
 *              before the call returns, so the caller may reuse idx at once
 *              (pinned or pageable)
 *  m           16, 32, 64 or 128 (EMG_ENOTSUP for 256)
 *  params      as for emg_create (minibatch and seed are ignored; dft must be
 *              EMG_DFT_FFT32, EMG_ENOTSUP for EMG_DFT_BF16X3)
 *
 * The result equals emg_step_minibatch on the same inputs.  Its only scratch
 * is one fixed device array of EMG_NOALLOC_SCRATCH_BYTES per GPU, part of the
 * library image, held until the process exits.  A call needs about
 * m^2 (16 b + 45) bytes of it; a larger request is rejected with EMG_EINVAL
 * before any work is enqueued (at m = 128 that allows b <= 29, at m = 32
 * b <= 500).  No part of the scratch needs to start at zero: each call writes
 * every element it later reads.  All calls share the array, so calls that
 * overlap on the GPU (other streams or threads) race and give wrong results;
 * serialise them.  The first call on each device does a one-time set-up with
 * that device current (constant tables, kernel attributes, the scratch
 * address); make that first call before any stream capture.  Asynchronous on
 * `stream` otherwise.
 */
#define EMG_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
emg_status emg_step_minibatch_noalloc(float* object, int32_t n_rows, int32_t n_cols,
                                      float* probe, int32_t m, const int32_t* pos,
                                      const float* intensity, int32_t n_pos,
                                      const int32_t* idx, int32_t b,
                                      const emg_params* params, emg_stream_t stream);

/* Message of the last failure on this context (static until the next call). */
emg_status emg_last_error(const emg_ctx* ctx, const char** msg);

/* Frees everything the context owns; NULL is a no-op. */
void emg_destroy(emg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* EMAGPIE_H */

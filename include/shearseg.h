/*
 * shearseg.h -- C ABI of the GB300 (sm_103a) shearlet-regularised convex
 * multi-label segmentation library (Haeuser & Steidl, "Convex Multiclass
 * Segmentation with Shearlet Regularization", arXiv:1112.1805).
 *
 * Conventions shared by every entry point:
 *   - Images are planar, row-major float32: a channel/label plane is [H][W],
 *     stacks are label-major [K][H][W] (the paper stacks the q label layers one
 *     after the other, Sec. 3 "Segmentation Model"; rows instead of its
 *     column-major vec, which leaves the model unchanged because the filter set
 *     is closed under transposition).  The first frequency coordinate omega_1
 *     belongs to the row axis (length H).
 *   - Shearlet coefficients are [nch][eta][H][W] with eta = 2^(J+2) - 3 filters
 *     per channel in the order: low-pass; then for each scale j = 0..J-1 the
 *     horizontal-cone shears k = -2^j+1..2^j-1, the vertical-cone shears (same
 *     k), the glued seam shearlet k = -2^j and the glued one k = +2^j
 *     (Sec. 2, "Finite Discrete Shearlets" and the Theorem's system).
 *   - Sizes: W even; H and W/2 products of powers of 2, 3 and 5; 8 <= H, W <=
 *     2048.  Labels 2 <= K <= 16; channels C in {1, 3}; scales 1 <= J <= 6.
 *   - Device pointers are caller-owned CUDA device memory unless the argument
 *     says "host".  Calls that take a bank or a state run on the device the
 *     bank was built on, which must be the current device.  The library never
 *     frees caller memory and never returns memory it allocated for the
 *     caller.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Work is enqueued asynchronously on that stream unless
 *     the function says it synchronises.
 *   - Every function returns SHF_OK (0) or a negative SHF_ERR_* code and never
 *     throws; shf_last_error() gives a thread-local message for the last
 *     failure.  There is no CPU fallback: without a usable sm_103a device every
 *     compute entry point fails with SHF_ERR_CUDA.
 */
#ifndef SHEARSEG_H
#define SHEARSEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHF_OK 0
#define SHF_ERR_ARG (-1)       /* null pointer, K/J/C/size out of range        */
#define SHF_ERR_SIZE (-2)      /* H or W/2 not 2^a 3^b 5^c, odd W, too large    */
#define SHF_ERR_OOM (-3)       /* device allocation failed                     */
#define SHF_ERR_CUDA (-4)      /* CUDA runtime or launch error                 */
#define SHF_ERR_NONFINITE (-5) /* NaN/Inf in an input image or codebook        */
#define SHF_ERR_TIMEOUT (-6)   /* a bounded device wait gave up (nl_admm_sync) */
#define SHF_ERR_STATE (-7)     /* handle used inconsistently (sizes, J, K)     */
#define SHF_ERR_IO (-8)        /* checkpoint file could not be read/written    */

/* Opaque, library-owned objects. */
typedef struct shf_bank shf_bank;   /* filter bank + FFT tables for one (H, W, J) */
typedef struct seg_state seg_state; /* ADMM state for one image                   */

/* ADMM parameters (Sec. 3).  gamma > 0 is the ADMM step; Lambda (host, J+1
 * floats) holds the weights of eq. problemSegmentation: Lambda[0] for the
 * low-pass, Lambda[j+1] for scale j, shared by all shears of a scale.  The
 * soft-shrinkage threshold of a coefficient is gamma * Lambda[.].
 * max_iters bounds seg_admm_solve; it stops earlier once
 * ||u - w||_2 / sqrt(K H W) < tol, checked every check_every iterations. */
typedef struct {
  float gamma;
  int J;
  const float* Lambda;
  int max_iters;
  float tol;
  int check_every;
} seg_params;

/* Library version (major*10000 + minor*100 + patch). */
int shf_version(void);

/* Thread-local text of the last error ("" if none).  Valid until the next
 * failing call on the same thread. */
const char* shf_last_error(void);

/* ---------------------------------------------------------------------------
 * Filter bank, Sec. 2 "Finite Discrete Shearlets" (shearlet spectra
 * psi1_hat(4^-j xi_1) psi2_hat(2^j xi_2/xi_1 + k) on the cones, glued seam
 * shearlets, scaling function varphi) and the Theorem (Parseval frame).
 * Built on the device in FP64 and stored as FP32 on the half plane
 * [eta][H][W/2+1] (the spectra are real and even).  Readings: frequencies are
 * normalised per axis, xi_a = omega_a 4^J / N_a, so that the J scales reach the
 * Nyquist frequency for any (N, J); on the Nyquist line of an even axis each
 * filter is replaced by the root mean square of its values at the two DFT
 * partners, which keeps sum_f W_f^2 = 1 and makes coefficients of real images
 * real.  Enqueued on `stream`; *out is usable once the stream reaches it.
 * Errors: SHF_ERR_ARG (null out, J out of range), SHF_ERR_SIZE, SHF_ERR_OOM,
 * SHF_ERR_CUDA. */
int shfilters_build(int H, int W, int J, void* stream, shf_bank** out);

/* Releases the bank (synchronises the device).  NULL is accepted. */
int shfilters_destroy(shf_bank* bank);

/* eta = 2^(J+2) - 3 (Remark 1: 61 images for four scales), H, W, J.  Any
 * output pointer may be NULL. */
int shfilters_info(const shf_bank* bank, int* eta, int* H, int* W, int* J);

/* Copies the FP32 half-plane bank [eta][H][W/2+1] into device memory dst. */
int shfilters_copy(const shf_bank* bank, float* dst, void* stream);

/* ---------------------------------------------------------------------------
 * Shearlet transform S (eq. wichtig: one fft2 per channel, then per filter a
 * pointwise product with the real spectrum and an ifft2).
 * u: device [nch][H][W]; coef: device [nch][eta][H][W] (must not alias u).
 * Temporary device memory is taken stream-ordered from the default pool and
 * returned before the call's work completes.  Errors: SHF_ERR_ARG,
 * SHF_ERR_OOM, SHF_ERR_CUDA. */
int shearlet_analyze(const shf_bank* bank, const float* u, int nch, float* coef, void* stream);

/* Adjoint S^T (the synthesis paragraph after the Theorem: fft2 of every
 * coefficient image, product with the same spectra, sum over the filters,
 * one ifft2).  By eq. important, shearlet_synthesize(shearlet_analyze(u)) = u.
 * coef: device [nch][eta][H][W]; u: device [nch][H][W]. */
int shearlet_synthesize(const shf_bank* bank, const float* coef, int nch, float* u, void* stream);

/* Allocation-free form of shearlet_analyze.  The paper has no counterpart: it
 * exists for callers that must not allocate device memory when they run a
 * transform -- a real-time loop that cannot stall on the allocator, a plugin
 * whose host application owns all device memory, a tool that forbids
 * allocation after start-up.  Same arguments, layout and result as
 * shearlet_analyze; the caller still provides u and coef.  Its temporaries
 * live in one fixed 32 MiB array inside the library image, which every GPU
 * that loads the library keeps reserved until the process exits; the call
 * itself allocates nothing (no cudaMalloc, no pool, no library allocation).
 * Limit: nch * (eta + 1) * H * (W/2 + 1) * 8 bytes must not exceed 32 MiB
 * (e.g. one 512 x 512 channel at J = 3: 31.6 MB, or two 256 x 256 channels
 * at J = 4: 32.8 MB); larger requests fail with SHF_ERR_SIZE and a message
 * giving both numbers.  The device the bank was built on must be the current
 * device (its tables and the array are then on the same GPU); otherwise the
 * call fails with SHF_ERR_STATE.  The first call on each device looks up the
 * array's device address with that device current; make that first call
 * before any stream capture.
 * Every call on a device shares the one array and leaves its contents behind
 * (nothing needs clearing: each call writes every element it reads), so calls
 * whose work overlaps on the GPU -- other streams, other host threads --
 * race on it and must be serialised by the caller. */
int shearlet_analyze_noalloc(const shf_bank* bank, const float* u, int nch, float* coef, void* stream);

/* ---------------------------------------------------------------------------
 * ADMM for eq. problemSegmentationADMM (Sec. 3): splitting (I_q (x) S) u = v,
 * u = w; per iteration
 *   u   = 1/2 [ S^T (v - b_v) + (w - b_w) - gamma s ]         (A^T A = 2 I)
 *   v   = soft-shrink(b_v + S u, gamma Lambda)               (v-step)
 *   w   = pixelwise projection of b_w + u onto the simplex   (w-step)
 *   b_v = b_v + S u - v,  b_w = b_w + u - w                  (eq. ADMM_b)
 * with the data term s[k] = sum_ch (f[ch] - c[k][ch])^2 (eq. computationOfs,
 * p = 2, and its RGB form).  The initial state is v = b_v = w = b_w = 0.
 * The library stores b_v and the synthesis S^T(v - b_v) instead of v and b_v
 * (v = soft(g), b_v = clip(g) with the same g), so v itself is not kept.
 *
 * f: device [C][H][W]; codebook: HOST [K][C]; params: host.  The state keeps
 * the bank pointer (the bank must outlive it), copies f and the parameters,
 * and owns its device buffers.  If `stream` is NULL the state creates and owns
 * a private non-blocking stream; otherwise all its work goes to `stream`.
 * Errors: SHF_ERR_ARG, SHF_ERR_STATE (params->J differs from the bank's),
 * SHF_ERR_NONFINITE (NaN/Inf in the codebook or parameters), SHF_ERR_OOM,
 * SHF_ERR_CUDA. */
int seg_admm_init(const shf_bank* bank, const float* f, int C, const float* codebook, int K,
                  const seg_params* params, void* stream, seg_state** out);

/* New image of the same size (f device, or host if f_on_host != 0; a host
 * image should be pinned for the copy to be asynchronous), recomputes the
 * data term and returns the state to v = b_v = w = b_w = 0, iteration 0. */
int seg_admm_reset(seg_state* st, const float* f, int f_on_host);

/* Enqueues n_iters ADMM iterations on the state's stream (replays of a CUDA
 * graph of one iteration, captured on first use when the stream allows it;
 * the last iteration of each call records the events of
 * seg_admm_kernel_times). */
int seg_admm_step(seg_state* st, int n_iters);

/* ---------------------------------------------------------------------------
 * Work plan and autotuner (no counterpart in the paper: how the iteration of
 * Sec. 3 is cut into kernel launches).  Power-of-two sizes (fast = 1) run the
 * register-FFT kernels over waves of (label, filter) pairs whose coefficient
 * spectra take about wave_mib MiB: the filters of one label when a label's
 * spectra exceed the budget, else whole labels (as many as fit, balanced), so
 * that one launch of each kernel covers several labels; each synthesis
 * (gather) launch runs col_ctas_per_sm resident CTAs per SM (0: as many as
 * fit) and each analysis (fan) launch as many as fit, each CTA on a balanced
 * range of the wave's (label, column tile, filter) triples.  Other
 * sizes (fast = 0) run the general kernels with tiles of tile_cols
 * half-spectrum columns and tile_rows rows and `groups` filter
 * groups in the synthesis sums.  On the fast path the plan also names the
 * FFT kernels: the v-step's (8, 16, 12, 20 or 32 values per thread, one row
 * or a pair of rows per thread group) and the fan's and gather's (8, 16, 12
 * or 20 values per thread), among those that exist for the size, and whether
 * the iteration's launches overlap (serial).  Fields of the other path
 * are 0 in seg_admm_get_plan and ignored by seg_admm_set_plan.  The plan
 * changes the grouping of the FP32 synthesis sums (wave_mib,
 * col_ctas_per_sm, groups) and the order of the FFT arithmetic (row_kernel,
 * col_kernel), so results are bitwise reproducible for a fixed plan on a
 * given GPU model, and agree within rounding across plans.
 * ------------------------------------------------------------------------- */
typedef struct {
  int fast;          /* read-only: 1 power-of-two path, 0 general path        */
  int wave_mib;      /* fast: MiB of coefficient spectra per wave, [1, 4096]  */
  int col_ctas_per_sm; /* fast: gather CTAs per SM, [0, 32], 0 = all that fit */
  int tile_cols;     /* general: half-spectrum columns per column tile        */
  int tile_rows;     /* general: rows per row block                           */
  int groups;        /* general: filter groups of the synthesis partial sums  */
  float us_per_iter; /* seg_admm_tune: measured microseconds per iteration    */
  int row_kernel;    /* fast: v-step FFT kernel, 0 default for the width, 1 8
                        values per thread, 2 16 values (half widths 64..1024,
                        powers of two), 3 pairs of rows (half widths 64, 128),
                        4 12, 20 or 32 values (half widths 12 T or 20 T, T =
                        2..32: 24..384 and 40..640; and 1024 = 32 x 32)       */
  int col_kernel;    /* fast: fan and gather FFT kernel, 0 default for the
                        height, 1 8 values per thread, 2 16 values (heights
                        512, 1024, 2048), 3 12 or 20 values (heights 12 T or
                        20 T, T = 2..128)                                     */
  int serial;        /* fast: 0 (default) each kernel of the iteration is
                        launched with programmatic dependent launch (its CTAs
                        start while the previous kernel drains), 1 plain
                        stream order; no effect on the results            */
  int sms;           /* fast: SMs the fan, v-step and gather launches size
                        their resident grids for, [0, 65536]; 0 (default) or
                        more than the GPU has: all of them.  A share lets the
                        images of a batch run side by side
                        (seg_admm_batch_tune chooses it)                     */
} seg_plan;

/* The state's current plan. */
int seg_admm_get_plan(const seg_state* st, seg_plan* out);

/* Installs a plan (reallocating the plan's scratch; the iterate is kept).
 * Synchronises the state's stream.  Errors: SHF_ERR_ARG for values out of
 * range or a tile shape the kernels do not support at this size (the old plan
 * stays), SHF_ERR_OOM. */
int seg_admm_set_plan(seg_state* st, const seg_plan* p);

/* Autotuner: times `iters` iterations (after one warm-up; replays of the plain
 * iteration graph, without the per-kernel timing events) of each candidate
 * plan twice and keeps the better time, varying one parameter at a time
 * around the best so far (fast: wave budget, then col_ctas_per_sm, then the
 * v-step's FFT kernel together with serial, then the column FFT kernel;
 * general: groups, then tile_cols, then tile_rows), and installs the fastest.
 * The iterate and the iteration count are saved before and restored after the
 * trials (needs memory for one copy of b_v, w, b_w, u and the u-spectra).
 * best (may be NULL) receives the plan with its time.  Synchronises.  Errors:
 * SHF_ERR_ARG (iters < 1), SHF_ERR_OOM, SHF_ERR_CUDA. */
int seg_admm_tune(seg_state* st, int iters, seg_plan* best);

/* Iterates until ||u - w||_2 / sqrt(K H W) < tol (checked every check_every
 * iterations) or max_iters total iterations; synchronises.  Outputs may be
 * NULL. */
int seg_admm_solve(seg_state* st, int* iters_done, float* final_residual);

/* Readout selectors for seg_admm_get / seg_admm_set. */
#define SEG_U 0      /* float [K][H][W]       last u                          */
#define SEG_W 1      /* float [K][H][W]       last w (in the simplex)         */
#define SEG_BW 2     /* float [K][H][W]       dual b_w                        */
#define SEG_BV 3     /* float [K][eta][H][W]  dual b_v                        */
#define SEG_S 4      /* float [K][H][W]       data term s                     */
#define SEG_LABELS 5 /* int32 [H][W]          argmax_k w (ties: lowest k)     */
#define SEG_GAP 6    /* float [H][W]          largest minus second largest w  */
#define SEG_ENERGY 7 /* double [1]            <w,s> + sum Lambda ||(S w)_f||_1 */
#define SEG_ITER 8   /* int32 [1]             iterations done (host only)     */
#define SEG_STV 9    /* float [K][H][W]       S^T (v - b_v) feeding next u    */
#define SEG_V 10     /* float [K][eta][H][W]  v (set only: with SEG_BV set
                        first, recomputes S^T (v - b_v))                        */

/* Copies component `what` into dst (device, or host if dst_on_host != 0).
 * Synchronises the state's stream when dst is on the host or what is
 * SEG_ENERGY or SEG_ITER.  Errors: SHF_ERR_ARG for an unknown selector. */
int seg_admm_get(seg_state* st, int what, void* dst, int dst_on_host);

/* Overwrites a state component from src (device, or host if src_on_host) --
 * used to resume or to start from a given state.  Accepts SEG_W, SEG_BW,
 * SEG_BV, SEG_STV and SEG_V. */
int seg_admm_set(seg_state* st, int what, const void* src, int src_on_host);

/* Checkpoint / resume: raw FP32 state (the carried synthesis spectrum of
 * v - b_v, b_v, w, b_w, s, u) behind a header with H, W, K, J, eta, C, the
 * iteration count, gamma and Lambda; a resumed run continues bit for bit.
 * load requires a state with the same H, W, K, J.  Synchronise. */
int seg_admm_save(seg_state* st, const char* path);
int seg_admm_load(seg_state* st, const char* path);

/* ---------------------------------------------------------------------------
 * Unrolled solve for differentiation.  The iteration is the one above; its
 * reverse mode is not in the paper (it follows from the iteration map: the
 * Jacobian of the simplex projection on the active face, the 0/1 masks of the
 * clipping |g| < gamma Lambda, and S / S^T exchanged).
 * seg_admm_unrolled_fwd returns the state to v = b_v = w = b_w = 0, runs T
 * iterations on the general-size kernels and keeps the state of every
 * ckpt_every-th iteration on the device.  seg_admm_unrolled_bwd takes dL/dw_T
 * (device [K][H][W]) of a loss of the final w, recomputes each segment from
 * its checkpoint, runs the adjoint iterations backwards and returns
 * dL/dcodebook (HOST [K][C]), dL/dLambda (HOST [J+1]), and optionally dL/df
 * (device [C][H][W]) and dL/ds (device [K][H][W]).  It synchronises and leaves
 * the state at an intermediate iterate.  Errors: SHF_ERR_STATE when the
 * forward has not run, SHF_ERR_OOM, SHF_ERR_CUDA. */
int seg_admm_unrolled_fwd(seg_state* st, int T, int ckpt_every);
int seg_admm_unrolled_bwd(seg_state* st, const float* dL_dw, float* dL_dcodebook, float* dL_dLambda, float* dL_df,
                          float* dL_ds);

/* The reverse sweep of seg_admm_unrolled_bwd in two parts, so that states on
 * different streams sweep concurrently.  _enqueue queues the sweep on the
 * state's stream and returns at once; dL_dw (device [K][H][W]) is read by a
 * queued copy and must stay valid until _grads returns.  _grads waits for the
 * sweep and writes the same outputs as seg_admm_unrolled_bwd.  Errors:
 * SHF_ERR_STATE (no forward; _grads without _enqueue), and those of
 * seg_admm_unrolled_bwd. */
int seg_admm_unrolled_bwd_enqueue(seg_state* st, const float* dL_dw);
int seg_admm_unrolled_grads(seg_state* st, float* dL_dcodebook, float* dL_dLambda, float* dL_df, float* dL_ds);

/* Instrumentation (no counterpart in the paper): time spent in each kind of
 * kernel during the most recent iteration, measured by CUDA events recorded
 * on the state's stream before every launch (event nodes inside the replayed
 * graph).  ms[i] gets the milliseconds of kind i summed over its launches,
 * launches[i] (may be NULL) their number; both need room for 8 entries.  *nk
 * (may be NULL) gets the number of kinds.  Waits for that iteration to finish.
 * Errors: SHF_ERR_STATE before the first iteration, and when an iteration has
 * more than 8192 launches (the timing events are created for the current
 * plan when an iteration is first run on the state's own stream). */
int seg_admm_kernel_times(seg_state* st, float* ms, int* launches, int* nk);

/* Name of kernel kind i of seg_admm_kernel_times ("" when out of range). */
const char* seg_admm_kernel_name(int i);

/* ---------------------------------------------------------------------------
 * Batched solves (no counterpart in the paper): n independent images of uneven
 * sizes, channel and label counts, each the problem of Sec. 3 with its own
 * parameters.  Image i: f[i] device [C[i]][H[i]][W[i]], codebooks[i] host
 * [K[i]][C[i]], params[i] host (its J selects the filter bank; banks are
 * built once per distinct (H, W, J) and shared).  One ADMM iteration of every
 * image is captured as one CUDA graph with one branch per image, the branches
 * on separate streams so that they run concurrently, joined on `stream`
 * (NULL: the batch creates its own stream).  Errors: those of
 * shfilters_build and seg_admm_init for any image (nothing is left allocated).
 */
typedef struct seg_batch seg_batch;
int seg_admm_batch_init(int n, const int* H, const int* W, const int* C, const int* K, const float* const* f,
                        const float* const* codebooks, const seg_params* params, void* stream, seg_batch** out);

/* Enqueues n_iters iterations of every image (replays of the batch graph). */
int seg_admm_batch_step(seg_batch* batch, int n_iters);

/* Borrows image i's state for seg_admm_get/set/save/load/reset (owned by the
 * batch: do not destroy it).  Its work goes to the image's own stream; call
 * seg_admm_batch_sync first to order it after the batch's iterations. */
int seg_admm_batch_image(seg_batch* batch, int i, seg_state** out);

/* Lanes of a batch iteration: with lanes = L in [1, n) the n images form L
 * chains that run side by side, each image (taken in decreasing order of
 * H W K eta) joining the chain with the least such work so far and starting
 * when the chain's previous image has finished its iteration; 0 (the
 * default), or L >= n, runs every image concurrently.  Fewer images at once
 * compete less for the L2 cache.  The results do not depend on it (every
 * image runs the same kernels on its own buffers).  Takes effect at the next
 * seg_admm_batch_step.  Errors: SHF_ERR_ARG (NULL batch, lanes < 0). */
int seg_admm_batch_set_lanes(seg_batch* batch, int lanes);
int seg_admm_batch_get_lanes(const seg_batch* batch, int* lanes);

/* Runs seg_admm_tune on the first image of every distinct (path, H, W, J, K)
 * (with sms = 0) and installs its plan on the other images of that shape;
 * then times `iters` iterations of the whole batch (twice, the better time
 * kept) for 0 to 4 lanes (seg_admm_batch_set_lanes), and at the fastest for
 * every fast image's sms set to all SMs, a half, a third and a quarter of
 * them, keeping the fastest of each.  The iterates are saved before and
 * restored after the batch-wide trials (a copy of every image's b_v, w, b_w,
 * u and u-spectra; without memory for them those trials are skipped).  The
 * batch graph is recaptured at the next step.  Synchronises. */
int seg_admm_batch_tune(seg_batch* batch, int iters);

/* Waits for the batch's stream. */
int seg_admm_batch_sync(seg_batch* batch);

/* Releases every state and bank of the batch.  NULL is accepted. */
int seg_admm_batch_destroy(seg_batch* batch);

/* ---------------------------------------------------------------------------
 * TV-regularised segmentation, the comparison model of Sec. 4 (eq. TVreg):
 *   min_u <u, s> + lambda sum_pixels |(I_q (x) grad) u| + iota_C(u)
 * with |(I_q (x) grad) u|(x) = (|grad u_1(x)|^2 + ... + |grad u_q(x)|^2)^(1/2)
 * (per_label = 0: the labels coupled per pixel, as eq. TVreg writes it) or
 * sum_k |grad u_k(x)| (per_label = 1: the alternative the paper mentions).
 * The paper fixes neither the difference scheme nor the solver; readings:
 * grad is the forward difference with periodic boundary, and the ADMM is the
 * one of Sec. 3 with S replaced by grad (splitting v = (I_q (x) grad) u,
 * w = u, same gamma):
 *   u   = (I + grad^T grad)^(-1) [ grad^T (v - b_v) + (w - b_w) - gamma s ]
 *   v   = group shrinkage of b_v + grad u by gamma lambda, b_v += grad u - v
 *   w   = pixelwise projection of b_w + u onto the simplex, b_w += u - w
 * from v = b_v = w = b_w = 0.  I + grad^T grad is diagonal in the DFT basis
 * (symbol 1 + 4 sin^2(pi n1/H) + 4 sin^2(pi n2/W)), so the u-step is one
 * filtered 2-D FFT per label.  Gradients and their duals are [K][2][H][W]
 * (component 0 along the row axis).
 * ------------------------------------------------------------------------- */
typedef struct tv_state tv_state;
typedef struct {
  float gamma;   /* ADMM step, > 0                                           */
  float lambda;  /* regularisation weight, >= 0 (threshold gamma * lambda)   */
  int per_label; /* 0: labels coupled per pixel (eq. TVreg); 1: per label    */
} tv_params;

/* f: device [C][H][W]; codebook: HOST [K][C]; sizes as for shfilters_build
 * (H and W/2 products of 2, 3 and 5, W even, 8..2048).  The state owns its
 * buffers and, if `stream` is NULL, a private stream.  Synchronises.  Errors:
 * SHF_ERR_ARG, SHF_ERR_SIZE, SHF_ERR_NONFINITE, SHF_ERR_OOM, SHF_ERR_CUDA. */
int tv_admm_init(int H, int W, const float* f, int C, const float* codebook, int K, const tv_params* params,
                 void* stream, tv_state** out);

/* New image of the same size (device, or host if f_on_host), data term
 * recomputed, state back to zero.  Synchronises. */
int tv_admm_reset(tv_state* st, const float* f, int f_on_host);

/* Enqueues n_iters iterations (replays of a CUDA graph of one iteration when
 * the stream can be captured). */
int tv_admm_step(tv_state* st, int n_iters);

/* Readouts as seg_admm_get: SEG_U, SEG_W, SEG_BW, SEG_S ([K][H][W]), SEG_BV
 * and SEG_V ([K][2][H][W]), SEG_LABELS, SEG_GAP ([H][W]), SEG_ENERGY (double:
 * <w, s> + lambda TV(w)), SEG_ITER (int, host only).  Host destinations and
 * SEG_ENERGY synchronise. */
int tv_admm_get(tv_state* st, int what, void* dst, int dst_on_host);

/* Overwrites SEG_W, SEG_BW, SEG_BV or SEG_V (v itself; set SEG_BV first,
 * since the state keeps v - b_v, which setting SEG_BV leaves unchanged) and
 * rebuilds the next u-step's right-hand side.  Synchronises. */
int tv_admm_set(tv_state* st, int what, const void* src, int src_on_host);

/* Instrumentation (no counterpart in the paper): runs n iterations launched
 * one by one with CUDA events between the kernels and writes the mean
 * milliseconds of each of the iteration's 5 kernels to ms (room for 5), *nk
 * (may be NULL) = 5.  Advances the iterate by n.  Synchronises. */
int tv_admm_kernel_times(tv_state* st, int n, float* ms, int* nk);
const char* tv_admm_kernel_name(int i);

int tv_admm_sync(tv_state* st);
/* Releases the state (synchronises its stream).  NULL is accepted. */
int tv_admm_destroy(tv_state* st);

/* ---------------------------------------------------------------------------
 * NL-means-regularised segmentation, the second comparison model of Sec. 4:
 * the gradient of the TV model replaced by a matrix D from patch similarities
 * of f.  Every pixel i, in raster order, picks min(mt, 2 mt - l) new
 * neighbours j (l: the neighbours it already has) among the candidates of the
 * varpi x varpi search window with the smallest patch distance
 *   d_a(i, j) = sum_{|t1|, |t2| <= h} G_a(t) sum_ch (f(i + t) - f(j + t))^2,
 * h = ceil((p - 1)/2), G_a the Gaussian of standard deviation a normalised to
 * sum 1, and links are symmetric (w(i, j) = w(j, i) = 1).  D has m = 2 mt
 * blocks: block b, row i is -1 at i and +1 at i's b-th neighbour (zero when i
 * has fewer neighbours).  The regulariser is the isotropic
 *   lambda sum_i (sum_k sum_b ((D u_k)_b(i))^2)^(1/2),
 * minimised with the ADMM of Sec. 3 with S replaced by D:
 *   u   = (I + D^T D)^(-1) [ D^T (v - b_v) + (w - b_w) - gamma s ]
 *   v   = group shrinkage of b_v + D u by gamma lambda, b_v += D u - v
 *   w   = pixelwise projection of b_w + u onto the simplex, b_w += u - w.
 * Readings (the paper leaves them open): the window is clipped to the image,
 * f is mirrored at the border inside patches (index -1 -> 1), distances run
 * over all channels and are computed in FP64 with every operation rounded
 * separately, ties go to the lower raster index, candidates already linked or
 * holding 2 mt neighbours are passed over, and the u-step solve runs
 * solve_steps Chebyshev iterations on the spectrum bound [1, 1 + 4 deg_max]
 * of I + D^T D = I + 2 L from the previous u (0: as many as give a relative
 * error of 1e-7).  The paper's values: p = 5, varpi = 15, a = 2, mt = 5.
 * Coefficients and duals are [K][m][H][W].
 * ------------------------------------------------------------------------- */
typedef struct nl_state nl_state;
typedef struct {
  float gamma;     /* ADMM step, > 0                                          */
  float lambda;    /* regularisation weight, >= 0                            */
  int patch;       /* p, 1..9                                                */
  int window;      /* varpi, odd, 3..15                                      */
  float a;         /* standard deviation of the patch Gaussian, > 0          */
  int neighbours;  /* mt, 1..8 (m = 2 mt blocks of D)                        */
  int solve_steps; /* Chebyshev iterations per u-step, 0 = automatic         */
} nl_params;

/* f: device [C][H][W] (H, W in 8..2048); codebook: HOST [K][C].  Builds the
 * neighbour graph of f (patch distances and their ranking on the GPU, the
 * sequential selection on the host), the data term and the zero state.
 * Synchronises.  Errors: SHF_ERR_ARG, SHF_ERR_SIZE, SHF_ERR_NONFINITE,
 * SHF_ERR_OOM, SHF_ERR_CUDA. */
int nl_admm_init(int H, int W, const float* f, int C, const float* codebook, int K, const nl_params* params,
                 void* stream, nl_state** out);

/* New image of the same size (device, or host if f_on_host): graph, data
 * term and state rebuilt.  Synchronises. */
int nl_admm_reset(nl_state* st, const float* f, int f_on_host);

/* The graph: nbr HOST [H W][2 mt] (increasing index, -1 padded), deg HOST
 * [H W], solve_steps (Chebyshev iterations per u-step); any may be NULL. */
int nl_admm_graph(const nl_state* st, int* nbr, int* deg, int* solve_steps);

/* Enqueues n_iters iterations (replays of a CUDA graph of one iteration).
 * For K <= 4 and images whose pixels fit one resident grid at two pixels per
 * thread, the u-step's Chebyshev steps run in one cooperative launch with a
 * grid barrier between steps; every barrier wait gives up after one second,
 * which nl_admm_sync then reports as SHF_ERR_TIMEOUT (a barrier cannot wait
 * that long unless the GPU is broken: all CTAs of the launch are resident). */
int nl_admm_step(nl_state* st, int n_iters);

/* Readouts as tv_admm_get, with SEG_BV and SEG_V of shape [K][m][H][W]. */
int nl_admm_get(nl_state* st, int what, void* dst, int dst_on_host);

/* Overwrites SEG_W, SEG_BW, SEG_U (the u-step's starting point), SEG_BV or
 * SEG_V (set SEG_BV first) and rebuilds the right-hand side.  Synchronises. */
int nl_admm_set(nl_state* st, int what, const void* src, int src_on_host);

/* Instrumentation: n iterations with events around the u-step solve, the
 * prox kernel and the right-hand side; mean milliseconds into ms (room for
 * 3), *nk = 3.  Advances the iterate.  Synchronises. */
int nl_admm_kernel_times(nl_state* st, int n, float* ms, int* nk);
const char* nl_admm_kernel_name(int i);

/* Waits for the state's stream; SHF_ERR_TIMEOUT if a grid barrier of the
 * Chebyshev solve gave up since the last call (the iterate is then invalid). */
int nl_admm_sync(nl_state* st);

/* Self-test of the bounded wait in the Chebyshev solve's grid barrier: runs,
 * on the state's stream, a two-CTA cooperative launch of that barrier with a
 * target that no CTA reaches, waits, and returns what nl_admm_sync reports:
 * SHF_ERR_TIMEOUT when the wait gave up after its one-second bound, as it
 * should.  No fault, trap or hang; the state and its iterate are untouched
 * and stay usable.  Synchronises. */
int nl_admm_barrier_selftest(nl_state* st);
/* Releases the state (synchronises its stream).  NULL is accepted. */
int nl_admm_destroy(nl_state* st);

/* Waits for the state's stream. */
int seg_admm_sync(seg_state* st);

/* Releases the state (synchronises its stream).  NULL is accepted. */
int seg_admm_destroy(seg_state* st);

#ifdef __cplusplus
}
#endif

#endif /* SHEARSEG_H */

/*
 * kb.h -- C ABI of the B300 (sm_103a) KBMOD shift-and-stack library, libkb_b300.so.
 *
 * The method is the GPU search of Smotherman et al. 2021 ("Sifting Through the Static: Moving
 * Object Detection in Difference Images", arXiv 2109.03296): PSF-matched likelihood images
 * psi/phi are summed along every linear trajectory of a velocity grid from every start pixel
 * (Section 3: Psi_coadd = sum psi_i, Phi_coadd = sum phi_i, nu = Psi/sqrt(Phi)); the sigma-G
 * percentile clip of Section 3.1 (Eqs. 1-5) is applied to each trajectory's lightcurve inside
 * the search (Section 3.2), the clipped likelihood sum LH' is thresholded, and the best K
 * trajectories of every start pixel are kept on the device (Section 3.2).  Coadded mean and
 * median postage stamps are cut along surviving trajectories (Section 3.3).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless the comment says HOST.
 *    The library never allocates device memory in these calls; scratch space is the caller's
 *    workspace, sized by the matching *_workspace_size query.
 *  - Images are row-major float32 planes stacked epoch-major: element (t, y, x) of a [T][H][W]
 *    array is at t*H*W + y*W + x; x is the column (fastest), y the row.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream).  A call returns once its kernels are enqueued.
 *  - Every call returns a kb_status.  KB_OK (0) means enqueued; any other value means nothing
 *    was enqueued (argument errors are found on the host before any launch) or, for
 *    KB_ERR_CUDA, that a CUDA runtime call failed.  kb_last_error() describes the last failure
 *    of the calling thread.
 *  - Integer-pixel trajectory positions are x_t = x0 + round(vx * dt_t), y_t = y0 + round(vy * dt_t)
 *    with dt_t = (float)(t_t - t_0) (difference in float64, then rounded to float32), the
 *    product taken as one IEEE float32 multiply and round() = floor(d + 0.5f) (round half up).
 */
#ifndef KB_B300_H
#define KB_B300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KB_API __attribute__((visibility("default")))
#else
#define KB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define KB_OK 0
#define KB_ERR_INVALID_ARG 1   /* a null pointer, a bad size or a bad parameter value */
#define KB_ERR_UNSUPPORTED 2   /* a valid request beyond the library's limits (e.g. T > KB_MAX_T) */
#define KB_ERR_CUDA 3          /* a CUDA runtime call failed; kb_last_error() names it */
#define KB_ERR_WORKSPACE 4     /* the workspace is null, misaligned or smaller than required */
#define KB_ERR_TIMEOUT 5       /* a bounded device-side wait gave up (see kb_wait_check) */

/* Host-side fault injection, for tests of a caller's failure handling: every entry point named
 * in the environment variable KB_FAULT_INJECT (a comma-separated list of names such as
 * "kb_search,kb_collect", or "*" for all) returns KB_ERR_CUDA with the message
 * "<name>: injected fault (KB_FAULT_INJECT)" after checking its arguments and before any device
 * work.  The variable is read at every call; unset or empty, nothing is injected. */

#define KB_MAX_T 128           /* epochs per stack */
#define KB_MAX_K 32            /* results kept per start pixel */
#define KB_WORKSPACE_ALIGN 256 /* required alignment of a workspace pointer, in bytes */

/* Parameters of the search (Sections 3.1-3.2). */
typedef struct kb_search_params {
  int32_t k_per_pixel; /* K: results kept per start pixel, 1..KB_MAX_K (the paper keeps 8) */
  float lh_min;        /* keep a trajectory only if its clipped sum LH' >= lh_min (paper: 10) */
  int32_t min_obs;     /* minimum number of valid epochs (paper: 15) */
  int32_t clip;        /* 1 = apply the sigma-G clip, 0 = keep every valid epoch */
  float q_lo;          /* lower quantile of sigma_G (paper: 0.25), 0 <= q_lo < q_hi <= 1 */
  float q_mid;         /* centre quantile, the median (0.5) */
  float q_hi;          /* upper quantile of sigma_G (paper: 0.75) */
  float n_sigma;       /* keep points within median +- n_sigma * sigma_G (paper: 2) */
  int32_t clip_on;     /* lightcurve that is clipped: 0 = flux psi_t/phi_t,
                          1 = per-epoch likelihood psi_t/sqrt(phi_t) (Section 3.1, "likelihood
                          and/or flux values") */
  int32_t x_lo, x_hi;  /* start-pixel window [x_lo, x_hi) x [y_lo, y_hi); the whole image is */
  int32_t y_lo, y_hi;  /* 0..W, 0..H */
  int32_t bound_rows;  /* start-pixel rows per term of the pruning bound (an implementation
                          choice; the results do not depend on it): 0 = automatic (2 when
                          1.5 T <= lh_min^2 or lh_min <= 0, else 1), 1 = every start pixel on its
                          own, 2 = blocks of two vertically adjacent start pixels, whose sum
                          bounds both (half the bound-pass work, looser). */
} kb_search_params;

/* Library version (major*10000 + minor*100 + patch). */
KB_API int kb_version(void);

/* Message describing the calling thread's last failure ("" if none).  The pointer stays valid
 * until the next failing call on the same thread. */
KB_API const char* kb_last_error(void);

/* Fills p with the paper's settings for the whole image: K = 8, LH' >= 10, min_obs = 15,
 * sigma-G clip on the flux with quantiles 0.25/0.5/0.75 and n_sigma = 2 (Sections 3.1, 3.2,
 * 4.3).  The window is set to [0, W) x [0, H). */
KB_API void kb_search_params_default(kb_search_params* p, int H, int W);

/*
 * kb_make_psi_phi -- PSF-matched likelihood images (Section 3, first paragraph; the formula
 * itself is KBMOD's: psi_t = (I_t / var_t) (x) PSF_t, phi_t = (1 / var_t) (x) PSF_t^2).
 *
 *   psi[t,y,x] = sum_{u,v in [-r,r]} w[t,y+v,x+u] * img[t,y+v,x+u] * psf[t,v+r,u+r]
 *   phi[t,y,x] = sum_{u,v in [-r,r]} w[t,y+v,x+u] * psf[t,v+r,u+r]^2
 *
 * with r = k/2 and w = 1/var, where w = 0 outside the image and at masked pixels (mask != 0,
 * var not finite or <= 0, img not finite); psi = phi = 0 is written at masked pixels
 * (Section 3: masked pixels carry no data).  This is a correlation; for the symmetric PSFs of
 * the paper it equals the convolution.  No renormalisation at the edges.
 *
 *   img, var  [T][H][W] float32 (device).       mask  [T][H][W] uint8 (device) or NULL.
 *   psf       [T][k][k] float32 (device), k odd, 1 <= k <= 31.
 *   psi, phi  [T][H][W] float32 (device) outputs; must not alias the inputs.
 * Errors: KB_ERR_INVALID_ARG for null pointers, T/H/W < 1, even k or k > 31.
 */
KB_API int kb_make_psi_phi(const float* img, const float* var, const uint8_t* mask, const float* psf,
                    int T, int H, int W, int k, float* psi, float* phi, void* stream);

/*
 * kb_search_workspace_size -- bytes of workspace kb_search needs for these sizes (the result
 * depends on T, H, W, n_traj and the window of p).  Returns KB_ERR_INVALID_ARG / UNSUPPORTED
 * for the same argument errors kb_search reports.
 */
KB_API int kb_search_workspace_size(int T, int H, int W, int n_traj, const kb_search_params* p,
                             size_t* bytes);

/*
 * kb_search -- exhaustive integer-pixel shift-and-stack search with the in-line sigma-G clip,
 * threshold and per-start-pixel top-K (Section 3 pointer arithmetic; Section 3.1 clip and
 * recomputed sum LH'; Section 3.2 clip before the per-pixel selection).
 *
 * For every start pixel (x0, y0) of the window and every trajectory j (vx[j], vy[j]):
 *   1. epoch t is valid iff (x_t, y_t) is inside the image and phi > 0 there (psi, phi finite);
 *      a trajectory with fewer than min_obs valid epochs is discarded;
 *   2. the lightcurve a_t (flux psi/phi, or psi/sqrt(phi) with clip_on = 1) of the valid
 *      epochs gives the q_lo, q_mid, q_hi percentiles by linear interpolation between order
 *      statistics (h = (n-1) q); sigma_G = C (x_hi - x_lo), C = 1/(sqrt2 (erfinv(2 q_hi - 1) -
 *      erfinv(2 q_lo - 1))) (Eq. 3 solved for sigma_G; Eq. 4 as printed drops its sqrt2);
 *      epoch t is kept iff x_mid - n_sigma sigma_G <= a_t <= x_mid + n_sigma sigma_G;
 *   3. over the kept epochs LH' = sum psi / sqrt(sum phi) and the flux alpha = sum psi / sum phi;
 *      discarded if no epoch is kept;
 *   4. kept in the start pixel's list if LH' >= lh_min; each list holds the K best, ordered by
 *      LH' descending and, for equal LH', by ascending trajectory index.
 * The result equals evaluating every pair; pairs are skipped only when an upper bound on LH'
 * proves they cannot enter the list.
 *
 *   psi, phi     [T][H][W] float32 (device).
 *   times        [T] float64, HOST pointer, finite; read during the call only.
 *   vx, vy       [n_traj] float32 (device), pixels per unit of `times`.
 *   p            HOST pointer to the parameters.
 *   out_*        (device) [npix][K] with npix = (x_hi - x_lo) * (y_hi - y_lo), start pixels in
 *                row-major order of the window; out_mask is [npix][K][ceil(T/32)] uint32
 *                (bit t%32 of word t/32 set = epoch t kept).  Empty slots: out_idx = -1,
 *                out_lh = -inf, out_flux = 0, counts 0, mask 0.
 *   workspace    device scratch of at least kb_search_workspace_size() bytes, aligned to
 *                KB_WORKSPACE_ALIGN; its contents on entry do not matter.  It must not be used
 *                by another call until this one has finished on the stream.
 * Velocities must be finite; a track offset beyond +-2^24 pixels is clamped there (it is off
 * the image either way).
 * Errors: KB_ERR_INVALID_ARG (null pointers, sizes, non-finite times or parameters, bad window,
 * K outside 1..KB_MAX_K, bound_rows outside 0..2), KB_ERR_UNSUPPORTED (T > KB_MAX_T,
 * n_traj > 2^24, H or W > 2^20, an image plane beyond 2^31 pixels, a device of more than 256
 * SMs), KB_ERR_WORKSPACE, KB_ERR_CUDA.
 */
KB_API int kb_search(const float* psi, const float* phi, const double* times, int T, int H, int W,
              const float* vx, const float* vy, int n_traj, const kb_search_params* p,
              float* out_lh, float* out_flux, int32_t* out_idx, uint16_t* out_nvalid,
              uint16_t* out_nkept, uint32_t* out_mask, void* workspace, size_t ws_bytes,
              void* stream);

/*
 * kb_search_no_alloc -- kb_search for callers that must not allocate device memory.  Some
 * callers cannot call cudaMalloc or hand out a workspace: a plug-in running inside a host program
 * whose device memory is owned by another allocator (a caching or fixed-size pool it may not grow),
 * or code that must keep a fixed device footprint after start-up.  This entry point takes the
 * same arguments as kb_search minus the workspace and uses scratch memory built into the library
 * instead: one array of KB_STATIC_SCRATCH_BYTES in device global memory, which every GPU that
 * loads the library holds until the process exits.  The paper has no counterpart; it is a
 * packaging of kb_search.
 *
 *  - Sizes whose kb_search_workspace_size exceeds KB_STATIC_SCRATCH_BYTES are rejected with
 *    KB_ERR_UNSUPPORTED (use kb_search with a workspace for them).
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture on the device.
 *  - All calls share the one array, and it keeps whatever the last call left in it (kb_search
 *    does not depend on the workspace's previous contents).  Calls whose work overlaps on the
 *    GPU (different streams, or threads without ordering) race on the array: serialise them.
 *  - No allocation of any kind (no cudaMalloc, no cudaFree, no allocating library routine).
 *  - The looked-up address is kept for the life of the process: a cudaDeviceReset between calls
 *    is not supported (the array may move when the module reloads).
 *  - kb_search_no_alloc_stats reads the counters of the last call on the current device,
 *    including the device-side error flags (a bounded wait that gave up).
 * Errors: as kb_search, plus KB_ERR_UNSUPPORTED for sizes beyond the built-in scratch and
 * KB_ERR_CUDA if the address lookup fails.  KB_FAULT_INJECT=kb_search_no_alloc injects a failure
 * after the size check (the call also runs kb_search's own checks and injection point).
 */
#define KB_STATIC_SCRATCH_BYTES (32u << 20)
KB_API int kb_search_no_alloc(const float* psi, const float* phi, const double* times, int T,
                              int H, int W, const float* vx, const float* vy, int n_traj,
                              const kb_search_params* p, float* out_lh, float* out_flux,
                              int32_t* out_idx, uint16_t* out_nvalid, uint16_t* out_nkept,
                              uint32_t* out_mask, void* stream);

/*
 * kb_search_no_alloc_stats -- kb_search_stats of the last kb_search_no_alloc call on the current
 * device (HOST array stats[4], same meaning; synchronises the stream).  A search whose
 * device-side wait gave up returns KB_OK with partial lists; stats[3] != 0 tells the caller.
 * Errors: KB_ERR_INVALID_ARG (null pointer, or no kb_search_no_alloc call on this device yet),
 * KB_ERR_CUDA.  The paper has no counterpart.
 */
KB_API int kb_search_no_alloc_stats(unsigned long long* stats, void* stream);

/*
 * kb_search_stats -- counters of the last kb_search that used `workspace` (device counters
 * copied to the HOST array stats[4]; synchronises the stream):
 *   stats[0] trajectory-epochs covered (start pixels x trajectories x T),
 *   stats[1] (pixel, trajectory) pairs whose bound required a full clipped evaluation,
 *   stats[2] pairs inserted into a top-K list,
 *   stats[3] device-side error flags (0 = none; bit 0x1 if a bounded wait gave up; bit 0x2 if
 *            a device-side bounds check failed -- only the checked build libkb_b300_checked.so,
 *            with the search kernel compiled with KB_BOUNDS_CHECK=1, makes those checks).
 */
KB_API int kb_search_stats(const void* workspace, unsigned long long* stats, void* stream);

/*
 * kb_search_stage_counts -- candidate counts at the stages of the last kb_search that used
 * `workspace`, the per-stage counts Section 3.1 (Fig. 3) and Section 3.4 (Fig. 4) report for the
 * pipeline (HOST array out[4]; synchronises the stream).  Over the (pixel, trajectory) pairs
 * the search evaluated in full (kb_search_stats()[1]):
 *   out[0] pairs with n_valid >= max(min_obs, 1) (eligible for the clip),
 *   out[1] pairs whose clipped LH' reached lh_min,
 *   out[2] the sum of n_kept over the out[1] pairs, out[3] the sum of their n_valid
 *          (out[2] / out[3] = the mean kept fraction of the clip).
 * Pruned pairs are not counted.  A pair is pruned only when its bound is below lh_min or below
 * the K-th LH' of its start pixel's full list, so while no list is full every pair that reaches
 * lh_min is evaluated (out[1..3] are then the exhaustive counts), and with lh_min <= 0 and K at
 * least the number of trajectories every pair is (all four are).
 */
KB_API int kb_search_stage_counts(const void* workspace, unsigned long long* out, void* stream);

/*
 * kb_search_pass_counts -- the shared-memory traffic of the last kb_search that used `workspace`
 * (HOST array out[4]; synchronises the stream), counted from the staging plan of every
 * (tile, chunk of 32 trajectories, epoch) the search swept:
 *   out[0] bytes of the pruning bound's words the search kernel read from staged shared memory
 *          (per bound-pass thread and trajectory two 4-byte words, or one with two-row-block
 *          bounds in 32-wide tiles; as many per thread when the chunk's trajectories share one
 *          offset in that epoch),
 *   out[1] bytes of the per-trajectory offsets it read with them (16 per four trajectories and
 *          warp),
 *   out[2] bytes staged into shared memory by the tensor-memory copies,
 *   out[3] iterations that read the bound from global memory instead (no staged box).
 * Measurement utility: the paper has no counterpart.
 * kb_batch_pass_counts: the same over the last run of a batch (kb_batch, below).
 * Errors: KB_ERR_INVALID_ARG (null pointer), KB_ERR_CUDA.
 */
KB_API int kb_search_pass_counts(const void* workspace, unsigned long long* out, void* stream);

/*
 * kb_stamps -- coadded postage stamps along trajectories (Section 3.3: per-pixel median over
 * the epochs of the trajectory; also the mean).  For candidate c and stamp pixel (sy, sx) in
 * [-radius, radius]^2, the values img[t, y_t + sy, x_t + sx] of every epoch t that is inside the
 * image, not masked (as in kb_make_psi_phi) and, if keep_mask is given, set in keep_mask[c]
 * are combined: mean = their average, median = the middle value (mean of the two middle values
 * for an even count); NaN if no epoch contributes.
 *
 *   img, var     [T][H][W] float32 (device); mask [T][H][W] uint8 (device) or NULL.
 *   times        [T] float64 HOST pointer.
 *   x0, y0       [n] int32 start pixels; vx, vy [n] float32 (device).
 *   keep_mask    [n][ceil(T/32)] uint32 (device) or NULL for all valid epochs.
 *   out_mean, out_median  [n][2r+1][2r+1] float32 (device).
 * Errors: KB_ERR_INVALID_ARG (null pointers, sizes, radius outside 0..15), KB_ERR_UNSUPPORTED
 * (T > KB_MAX_T).
 */
KB_API int kb_stamps(const float* img, const float* var, const uint8_t* mask, const double* times,
              int T, int H, int W, const int32_t* x0, const int32_t* y0, const float* vx,
              const float* vy, const uint32_t* keep_mask, int n, int radius, float* out_mean,
              float* out_median, void* stream);

/*
 * Batched search -- many stacks (CCDs, pointings) searched as one unit.  The paper searches each
 * CCD's stack on its own (Section 2: 2580 independent searches, Section 4.1); here either the
 * tiles of all stacks are handed out from one counter to one persistent kernel, or the stacks'
 * kernels run concurrently on a few streams (schedule mode), so that no SM idles at the end of
 * a stack, and the whole sequence (per-stack preparation + the search) can be replayed as one
 * CUDA graph.  Each stack's results are exactly those of kb_search on it.
 *
 *   kb_stack       one stack: the arguments of kb_search (psi, phi, times, sizes, velocities,
 *                  search parameters and the six output arrays), with the same meaning, layout
 *                  and ownership; each stack has its own T (up to KB_MAX_T), H, W and n_traj.
 *   kb_schedule    scheduling knobs; the results never depend on them:
 *                    tile_order   1: each stack's tiles in decreasing predicted cost (pixels
 *                                 with psi^2/phi >= hot_nu2 in the footprints of the epochs
 *                                 whose offsets span at most score_span pixels); 0: row-major.
 *                    stack_order  1: stacks in decreasing trajectory-epoch count; 0: as given.
 *                    mode         0: one persistent launch over the tiles of all stacks;
 *                                 1: one launch per stack (the single-stack kernel, whose
 *                                 arguments live in parameter space), spread over four
 *                                 streams of the batch, so that a stack's kernel starts on the
 *                                 SMs that the previous one's last tiles leave idle.
 *                    tile_cols    1 or 2: columns summed by each thread of the bound pass, i.e.
 *                                 tiles 32 or 64 pixels wide (stacks with two-row-block bounds;
 *                                 single-row bounds always take 32); 0: automatic, per stack
 *                                 64 wide when its window holds at least 8 tiles of that width
 *                                 per SM, else 32 (mode 0: 64 for every stack).
 *                  kb_schedule_default: {tile_order 1, hot_nu2 64, score_span 64, stack_order 1,
 *                  mode 1, tile_cols 0} (kb_search uses the same tile order and width rule).
 *   kb_batch       opaque handle: kb_batch_create validates every stack (the checks of
 *                  kb_search), lays out the workspace and writes the batch tables to the device
 *                  (synchronous copies); the stacks' buffers must stay valid while it is used.
 *
 * kb_batch_workspace_size: bytes of the caller-owned workspace (KB_WORKSPACE_ALIGN-aligned).
 * kb_batch_run: enqueues the batch on `stream` (kernel launches only).
 * kb_batch_run_graph: on first use captures kb_batch_run into a CUDA graph on a stream of the
 *   batch's own; every call replays it, ordered after the work already on `stream` and before
 *   the work enqueued on it later.  A schedule change drops the graph (re-captured on the next
 *   call).
 * kb_batch_set_schedule / kb_batch_get_schedule: knobs above (set waits for the device).
 * kb_batch_autotune: times the batch (kb_batch_run, best of `reps`) under schedules chosen by
 *   coordinate descent from the default (mode and stack order, tile order and tile width,
 *   hot_nu2 in {64, 16, 144}, score_span in {64, 32, 128}), keeps the fastest and returns it in
 *   *best (nullable).  Runs the batch about 10 x reps times; its outputs are those of a normal
 *   run.
 * kb_batch_stats: after a run, done_ns[i] = ns from the start of the run to the completion of
 *   stack i's last tile (the caller's order), totals[4] = {trajectory-epochs, full evaluations,
 *   insertions, error flags} of the run (blocks the host).
 * kb_batch_destroy: frees the handle (not the workspace or the stacks' buffers).
 * Errors: as kb_search per stack (the message names the stack), KB_ERR_INVALID_ARG for bad
 * schedules, KB_ERR_WORKSPACE, KB_ERR_CUDA.
 */
typedef struct kb_stack {
  const float* psi;
  const float* phi;
  const double* times; /* HOST */
  int T, H, W;
  const float* vx;
  const float* vy;
  int n_traj;
  kb_search_params params;
  float* out_lh;
  float* out_flux;
  int32_t* out_idx;
  uint16_t* out_nvalid;
  uint16_t* out_nkept;
  uint32_t* out_mask;
} kb_stack;

typedef struct kb_schedule {
  int tile_order;
  float hot_nu2;
  int score_span;
  int stack_order;
  int mode;
  int tile_cols;
} kb_schedule;

typedef struct kb_batch kb_batch;

KB_API void kb_schedule_default(kb_schedule* s);
KB_API int kb_batch_workspace_size(const kb_stack* stacks, int n, size_t* bytes);
KB_API int kb_batch_create(const kb_stack* stacks, int n, void* workspace, size_t ws_bytes,
                           kb_batch** out);
KB_API int kb_batch_run(kb_batch* b, void* stream);
KB_API int kb_batch_run_graph(kb_batch* b, void* stream);
KB_API int kb_batch_set_schedule(kb_batch* b, const kb_schedule* s);
KB_API int kb_batch_get_schedule(const kb_batch* b, kb_schedule* s);
KB_API int kb_batch_autotune(kb_batch* b, void* stream, int reps, kb_schedule* best);
KB_API int kb_batch_stats(kb_batch* b, unsigned long long* done_ns, unsigned long long* totals,
                          void* stream);
KB_API int kb_batch_pass_counts(kb_batch* b, unsigned long long* out, void* stream);
KB_API void kb_batch_destroy(kb_batch* b);

/*
 * kb_stamp_filter -- central-moment filter of coadded stamps (Section 3.3: a candidate is kept
 * only if the moments of its median coadd are those of a compact source at the trajectory's
 * position; the paper's limits are 0.5, 0.5, 1.5, 36.5, 36.5 for x, y, xy, xx, yy, strictly).
 * With S the stamp, (dx, dy) = (column - radius, row - radius), NaN pixels (no contributing
 * epoch) left out and the weights w = S - min S (the smallest non-NaN pixel):
 *   M0 = sum w,  x = sum dx w / M0,  y = sum dy w / M0,  xy = sum dx dy w / M0,
 *   xx = sum dx^2 w / M0,  yy = sum dy^2 w / M0   (sums in float64)
 * and the stamp passes iff M0 > 0, |x| < lim[0], |y| < lim[1], |xy| < lim[2], xx < lim[3] and
 * yy < lim[4].  (Uniform weights over 21 x 21 give xx = yy = 36.67: a flat or noise-like stamp
 * sits just above the paper's 36.5, and light concentrated at the centre pulls it below.)
 *
 *   stamps       [n][2r+1][2r+1] float32 (device), e.g. kb_stamps' out_median.
 *   limits       [5] float32 HOST array, or NULL for the paper's limits.
 *   out_moments  [n][6] float32 (device, nullable): M0, x, y, xy, xx, yy.
 *   out_pass     [n] uint8 (device): 1 = passes.
 * Errors: KB_ERR_INVALID_ARG (null pointers, n < 0, radius outside 0..15, NaN limits).
 */
KB_API int kb_stamp_filter(const float* stamps, int n, int radius, const float* limits,
                           float* out_moments, uint8_t* out_pass, void* stream);

/*
 * kb_cluster -- de-duplication of candidates (the clustering step that follows the stamp filter
 * in the paper's pipeline, Fig. 3; the paper does not give its algorithm).  In priority order
 * (index 0 first, e.g. kb_collect's LH' order), candidate i is kept unless its track agrees
 * within `radius` pixels, at the first epoch and at the last, with a candidate kept before it:
 *   |p_i(0) - p_j(0)| <= radius  and  |p_i(dt) - p_j(dt)| <= radius,
 *   p(t) = (x0 + vx t, y0 + vy t), distances in float64, dt = t_last - t_0.
 * out_rep[i] = i for a kept candidate, else the first (lowest-index) kept candidate it
 * duplicates; -1 for candidates that take no part (valid[i] == 0, or a start pixel outside
 * 0 .. 2^20 - 1, as kb_candidate_tracks gives empty slots).
 *
 *   x0, y0       [n] int32 start pixels; vx, vy [n] float32 (device).
 *   valid        [n] uint8 (device) or NULL: e.g. kb_stamp_filter's out_pass.
 *   out_keep     [n] uint8 (device): 1 = kept.   out_rep [n] int32 (device).
 *   workspace    kb_cluster_workspace_size(n) bytes, KB_WORKSPACE_ALIGN-aligned.
 *   rounds       (nullable, host) the number of parallel rounds run.
 * The greedy order is resolved in rounds: a candidate is dropped as soon as an earlier duplicate
 * is kept, and kept once its earlier duplicates are all decided and none is kept (a group of
 * mutual duplicates takes two rounds).  The call reads a round counter back every 4 rounds, so
 * it BLOCKS the host until the result is final (it is not capturable in a CUDA graph).
 * Errors: KB_ERR_INVALID_ARG (null pointers, n < 0, radius < 1 or not finite, dt not finite),
 * KB_ERR_UNSUPPORTED (n > 2^24), KB_ERR_WORKSPACE.
 */
KB_API int kb_cluster_workspace_size(int n, size_t* bytes);
KB_API int kb_cluster(const int32_t* x0, const int32_t* y0, const float* vx, const float* vy,
                      const uint8_t* valid, int n, double dt, double radius, uint8_t* out_keep,
                      int32_t* out_rep, void* workspace, size_t ws_bytes, int* rounds,
                      void* stream);

/*
 * kb_collect -- GPU-to-host handoff of the survivors (Section 3.1 reworked handoff; Section 3.2
 * returns the per-pixel results to the CPU): gathers every filled slot of a kb_search result
 * and orders them by LH' descending, then start pixel, then slot; the first n_max are written.
 *
 *   lh, idx      [npix][K] kb_search outputs (device).
 *   cand_pix     [n_max] int32 (device): window pixel index (row-major) of each survivor.
 *   cand_slot    [n_max] int32 (device): its slot in that pixel's list.
 *   count        [1] int32 (device): total number of filled slots (may exceed n_max).
 *   workspace    kb_collect_workspace_size(n_max) bytes, aligned to KB_WORKSPACE_ALIGN.
 * Errors: KB_ERR_INVALID_ARG (null pointers, sizes, K outside 1..KB_MAX_K), KB_ERR_UNSUPPORTED
 * (npix * K >= 2^32 or n_max > 2^24), KB_ERR_WORKSPACE.
 */
KB_API int kb_collect_workspace_size(int n_max, size_t* bytes);
KB_API int kb_collect(const float* lh, const int32_t* idx, int npix, int K, int n_max,
               int32_t* cand_pix, int32_t* cand_slot, int32_t* count, void* workspace,
               size_t ws_bytes, void* stream);

/*
 * kb_candidate_tracks -- start pixel and velocity of collected survivors, for kb_stamps.
 * For i < n with cand_pix[i] >= 0: x0[i] = x_lo + cand_pix[i] % wx, y0[i] = y_lo + cand_pix[i] / wx,
 * traj[i] = idx[cand_pix[i] * K + cand_slot[i]], out_vx/out_vy = vx/vy[traj[i]].  Entries with
 * cand_pix[i] < 0 get traj = -1 and a start pixel far outside any image (their stamps are NaN).
 * All arrays are device arrays; idx is the kb_search output of the window (x_lo, y_lo, wx).
 */
KB_API int kb_candidate_tracks(const int32_t* cand_pix, const int32_t* cand_slot, int n,
                               const int32_t* idx, int K, const float* vx, const float* vy,
                               int x_lo, int y_lo, int wx, int32_t* x0, int32_t* y0,
                               float* out_vx, float* out_vy, int32_t* traj, void* stream);

/*
 * Sub-pixel evaluation of single trajectories, its backward pass, and refinement off the velocity
 * grid.  Section 4.1 evaluates single given trajectories along their own tracks, and spaces the
 * search grid so that neighbouring trajectories stay within about two PSF widths of each other
 * over the run; the grid spacing thus bounds how closely a found trajectory follows its object.
 * These calls evaluate a trajectory at a real-valued start and velocity: psi_t and phi_t are read
 * at (x0 + vx dt_t, y0 + vy dt_t), dt_t = times[t] - times[0], by bilinear interpolation (pixel
 * centres at integer coordinates; the cell of a position is (floor x, floor y); taps outside the
 * image read zero), and over a FIXED set of kept epochs (the clip is not re-run)
 *     Psi = sum_{t kept} psi_t(.),  Phi = sum_{t kept} phi_t(.),
 *     L = Psi / sqrt(Phi),  alpha = Psi / Phi        (Eq. 1 and 2 on the kept epochs).
 * L is piecewise bilinear in (x0, y0, vx, vy); its gradient is the one-sided derivative on the
 * cell containing the position.  Positions x0 + vx dt_t are formed in float-float arithmetic
 * (about 48 significant bits, so the cell of an epoch is the one of the exact position unless it
 * lies within ~1e-11 px of a cell edge), the bilinear weights and the sums in float32.  A candidate
 * whose Phi is not > 0 (no kept tap inside the image with phi > 0) gets L = alpha = NaN and a zero
 * gradient.
 *
 * Common arguments:
 *   psi, phi   [T][H][W] float32 (device), as written by kb_make_psi_phi.
 *   times      [T] float64 HOST pointer (finite).
 *   params     [n][4] float32 (device, 16-byte aligned: rows are read as float4): x0, y0 in
 *              pixels, vx, vy in pixels per unit of times.
 *   keep       [n][ceil(T/32)] uint32 (device): bit t of word t/32 set = epoch t kept (the
 *              out_mask layout of kb_search); NULL keeps every epoch.
 * All outputs are caller-owned device arrays.  n = 0 enqueues nothing.
 * Errors: KB_ERR_INVALID_ARG (null pointers, bad sizes, a params or [n][4] gradient array not
 * 16-byte aligned, non-finite times or bad refine parameters), KB_ERR_UNSUPPORTED (T > KB_MAX_T,
 * sides > 2^20).
 */

/* kb_traj_eval_fwd -- out_lh, out_flux [n]; out_grad [n][4] (nullable, 16-byte aligned)
 * receives dL/d(params). */
KB_API int kb_traj_eval_fwd(const float* psi, const float* phi, const double* times, int T, int H,
                            int W, const float* params, const uint32_t* keep, int n,
                            float* out_lh, float* out_flux, float* out_grad, void* stream);

/*
 * kb_traj_eval_bwd -- vector-Jacobian product of kb_traj_eval_fwd.  With upstream weights
 * gL = grad_lh[c] and gA = grad_flux[c] (either array nullable, read as zeros):
 *   out_grad_params [n][4] (nullable, 16-byte aligned, overwritten) = gL dL/dparams +
 *   gA dalpha/dparams;
 *   grad_psi, grad_phi [T][H][W] (nullable, ACCUMULATED with atomic adds, in no fixed order):
 *   each kept in-image tap of weight w on epoch t adds cPsi w to grad_psi and cPhi w to grad_phi,
 *   cPsi = gL / sqrt(Phi) + gA / Phi,  cPhi = -gL Psi / (2 Phi^1.5) - gA Psi / Phi^2.
 */
KB_API int kb_traj_eval_bwd(const float* psi, const float* phi, const double* times, int T, int H,
                            int W, const float* params, const uint32_t* keep, int n,
                            const float* grad_lh, const float* grad_flux, float* out_grad_params,
                            float* grad_psi, float* grad_phi, void* stream);

/* Adam (Kingma & Ba 2015) settings of kb_refine; kb_refine_params_default gives 20 steps,
 * lr_pos 0.1 px, lr_vel 0.2 px per unit of times, beta1 0.9, beta2 0.999, eps 1e-8. */
typedef struct kb_refine_params {
  int n_steps;  /* 0..100000 */
  float lr_pos; /* step size of x0, y0 (>= 0) */
  float lr_vel; /* step size of vx, vy (>= 0) */
  float beta1;  /* [0, 1) */
  float beta2;  /* [0, 1) */
  float eps;    /* > 0 */
} kb_refine_params;

KB_API void kb_refine_params_default(kb_refine_params* rp);

/*
 * kb_refine -- gradient ascent of L from each candidate's params with Adam, the kept set fixed.
 * Step k = 1..n_steps evaluates L and g = dL/dparams at the current params and moves them by
 * lr mhat / (sqrt(vhat) + eps), m = beta1 m + (1 - beta1) g, v = beta2 v + (1 - beta2) g^2,
 * mhat = m / (1 - beta1^k), vhat = v / (1 - beta2^k); lr is lr_pos for x0, y0 and lr_vel for
 * vx, vy.  The gradient and the moments are float32; the parameters are carried in
 * float-float between steps and rounded to float32 once at the end.  params are updated in place;
 * out_lh, out_flux [n] are L and alpha at the returned (rounded) params; out_lh_start [n]
 * (nullable) is L at the given params.  Where Phi <= 0 is met the ascent of that candidate stops
 * there (params as they were, rounded; L = alpha = NaN).
 */
KB_API int kb_refine(const float* psi, const float* phi, const double* times, int T, int H, int W,
                     float* params, const uint32_t* keep, int n, const kb_refine_params* rp,
                     float* out_lh, float* out_flux, float* out_lh_start, void* stream);

/*
 * kb_candidate_params -- refine inputs of collected survivors: for i < n with cand_pix[i] >= 0,
 * out_params[i] = (x_lo + cand_pix[i] % wx, y_lo + cand_pix[i] / wx, vx[traj], vy[traj]) with
 * traj = idx[cand_pix[i] * K + cand_slot[i]], and out_keep[i] (nullable; needs mask) = that
 * slot's kept-epoch mask from kb_search's out_mask [npix][K][ceil(T/32)].  Other entries get NaN
 * params (kb_refine then reports NaN) and an all-zero mask.  All arrays are device arrays;
 * out_params [n][4] must be 16-byte aligned (KB_ERR_INVALID_ARG otherwise).
 */
KB_API int kb_candidate_params(const int32_t* cand_pix, const int32_t* cand_slot, int n,
                               const int32_t* idx, const uint32_t* mask, int K, int T,
                               const float* vx, const float* vy, int x_lo, int y_lo, int wx,
                               float* out_params, uint32_t* out_keep, void* stream);

/*
 * kb_l2_probe -- measurement utility, not part of the method: reads the device buffer `buf`
 * (`bytes`, 16-byte aligned; choose it smaller than the L2 so that it stays resident) `reps`
 * times with 16-byte loads cached in L2 only, from `blocks` blocks of 512 threads.  The caller
 * times the call (CUDA events): bytes x reps / time is the L2 read bandwidth.  scratch: `blocks`
 * floats (device), written only in a case that the probe data never meet.
 */
KB_API int kb_l2_probe(const void* buf, size_t bytes, int reps, float* scratch, int blocks,
                       void* stream);

/*
 * kb_smem_probe -- measurement utility, not part of the method: `blocks` blocks of 1024 threads
 * each stream `iters` x 32 shared-memory loads per warp, 32-bit and lane-contiguous (one 128-byte
 * wavefront per load instruction, no bank conflict), the access of the search kernel's bound
 * pass.  The caller times the call (CUDA events): blocks x 32 warps x iters x 32 x 128 bytes /
 * time is the shared-memory read bandwidth the bound pass can reach.  scratch: `blocks` uint32
 * (device), written only in a case the probe data never meet.
 */
KB_API int kb_smem_probe(int blocks, int iters, unsigned int* scratch, void* stream);

/*
 * kb_wait_check -- failure detection without a fault: runs the bounded device-side waits of the
 * search kernel on waits that cannot complete and reports what the device saw.  One thread waits
 * on an mbarrier phase that nothing completes, first as a producer retiring a ring slot, then as
 * a consumer waiting for a staged box (each gives up after limit_ns of %globaltimer, as the
 * search kernel's waits do after 2 s), then once more as a consumer with its block's abort flag
 * raised (it must return at the flag, as the other warps of a search block do after one wait has
 * given up).  The device writes its status; the call copies it back (synchronising the stream).
 *   limit_ns  1e3 .. 1e10 ns; the kernel runs for about 2 limit_ns.
 *   out       HOST [4] (nullable): status bits (0x1 producer wait gave up, 0x2 consumer wait gave
 *             up, 0x4 consumer wait ended by the abort flag), then each wait's duration in ns.
 * Returns KB_ERR_TIMEOUT when all three gave up as designed (the expected outcome: the device
 * reported the timeouts and the context stays usable), KB_ERR_CUDA if a wait reported success or
 * ignored the abort flag, KB_ERR_INVALID_ARG for a limit outside the range.  A search whose wait
 * gives up reports it in kb_search_stats()[3] (kb_batch_stats totals[3]) bit 0x1.
 */
KB_API int kb_wait_check(unsigned long long limit_ns, unsigned long long* out, void* stream);

/* Number of kernels this library has launched in the process so far (all entry points). */
KB_API unsigned long long kb_launch_count(void);

/*
 * kb_profile_events -- when both are non-NULL (cudaEvent_t passed as void*), every following
 * kb_search on this thread records `start` on its stream immediately before the main search
 * kernel and `stop` immediately after it, so the caller can time that kernel alone with
 * cudaEventElapsedTime.  Pass NULL, NULL to stop.  The events are owned by the caller.
 */
KB_API void kb_profile_events(void* start, void* stop);

#ifdef __cplusplus
}
#endif

#endif /* KB_B300_H */

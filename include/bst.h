/*
 * bst.h -- C ABI of libbst: filtered backprojection of parallel-beam
 * sinograms through the backprojection-slice theorem (BST) on one GPU.
 *
 * Method: Theorem 2.1 (Eq. 3) of "Low-complexity Distributed Tomographic
 * Backprojection for large datasets": the 2D Fourier transform of the
 * backprojection b = B y (Eq. 2) at the polar point sigma (cos t, sin t) is
 * y^(sigma, t) / sigma.  Sec. 2 evaluates it in stages P0..P8: zero padding,
 * a 1D FFT along the detector, a 1/sigma (or filter) weight, polar-to-
 * Cartesian interpolation in the Fourier domain, a 2D inverse FFT and an
 * fftshift/crop, O(N^2 log N) per slice instead of the O(N^3) slant stack.
 *
 * Conventions (the paper fixes none; these are this library's):
 *   - N detector samples at t_i = (i - N/2) dt, dt = 2/N (t in [-1, 1));
 *   - images are N x N with volume[r][c] at u = ((c - N/2) dt, (r - N/2) dt):
 *     the column index follows u1, the row index u2; theta = 0 has t = u1;
 *   - V angles theta_j (radians, float32), strictly increasing, in [0, pi);
 *   - pad factor alpha in {1, 2}; FFT length M = alpha N; supported M are
 *     2^a (16 <= M <= 4096) and 3 * 2^a (48 <= M <= 3072); N is even;
 *   - sinogram[slices][V][N], volume[slices][N][N]: row-major, contiguous
 *     float32, device memory owned by the caller; the library never frees or
 *     retains caller pointers;
 *   - the ordinary-frequency Fourier convention, so Eq. 3 holds with
 *     constant 1; bilinear interpolation in (signed radius, angle) by default
 *     (Kaiser-Bessel gridding on request, bst_plan_set_gridding); the Nyquist
 *     bin is zero; the DC bin is averaged over angles (bilinear).
 *
 * Every call is asynchronous on the given stream.  The returned status
 * covers argument validation and launch errors only; errors detected on the
 * device are sticky in the plan and reported by bst_plan_status().  Calls on
 * one plan may be issued from one host thread at a time.
 *
 * A plan belongs to the device that was current at bst_plan_create (its
 * tables live there).  Every call that launches work for a plan or builds
 * tables for it must be made with that device current, and returns
 * BST_ERR_INVALID_ARGUMENT otherwise; so do the ragged-batch calls, whose
 * plans must all belong to the current device.
 */
#ifndef BST_H
#define BST_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BST_OK = 0,
    BST_ERR_INVALID_ARGUMENT = 1,   /* null pointer, bad count, bad angles, aliasing */
    BST_ERR_UNSUPPORTED_SIZE = 2,   /* M = alpha N not a supported FFT length, N odd */
    BST_ERR_WORKSPACE_TOO_SMALL = 3,
    BST_ERR_CUDA = 4,               /* a CUDA runtime call or launch failed */
    BST_ERR_TIMEOUT = 5,            /* a bounded device-side wait gave up */
    BST_ERR_OUT_OF_MEMORY = 6       /* a plan-owned allocation failed */
} bst_status_t;

typedef enum {
    BST_W_FILTER = 0,      /* FBP: P4 weight W[k] = g[k] (g = NULL: ramp, g = 1) */
    BST_W_BACKPROJECT = 1  /* plain B: W[k] = 1/sigma_k = M dt / k, W[0] = 0 */
} bst_mode_t;

/* Interpolation kernel of stage P5 (Sec. 2 names the step, not the kernel). */
typedef enum {
    BST_GRID_BILINEAR = 0,      /* bilinear in (signed radius, angle), gather form */
    BST_GRID_KAISER_BESSEL = 1  /* KB convolution gridding with deapodization */
} bst_gridding_t;

/* Memory layout of the polar spectrum between the ray and gridding stages
 * (an implementation choice; the paper's stages P3-P5 fix the values only). */
typedef enum {
    BST_LAYOUT_PACKED = 0,  /* Z[V][M] complex64, natural order of k */
    BST_LAYOUT_PAIRED = 1   /* Z[V][M/2] pairs (Z[k], Z[-k]): one 16-byte load serves a
                               Cartesian point and its mirror (bilinear gridding only) */
} bst_layout_t;

/* Launch shape of the forward path (extension; no passage: the paper fixes
 * the stages, not how they are tiled).  Results are identical up to
 * rounding whatever the shape. */
typedef struct {
    int max_radix;    /* largest Stockham radix: 16 or 8 */
    int layout;       /* bst_layout_t */
    int chunk_pairs;  /* slice pairs per launch of each stage, 1..256 */
    int pair_fast;    /* 1: gridding blocks ordered pair-fastest within a chunk */
    int max_lanes;    /* streams alternating chunks, 1 or 2 */
    int grid_xchg;    /* paired layout only: 1 feeds the first column-FFT pass of both
                         columns of a pair from registers (partner lanes swap the halves
                         of their gathered point pairs), 0 goes through shared memory */
} bst_fwd_config_t;

typedef struct bst_plan_s* bst_plan_t;
typedef void* bst_stream_t;   /* a cudaStream_t; NULL is the legacy default stream */

/* Create a plan for N = rays detector samples, V = angles projections and pad
 * factor alpha (extension; no passage: the paper's problem statement, Sec. 1,
 * fixes the sizes N and V; the plan holds the tables of stages P3 and P5).
 * angles_rad_host: host array of V float32 angles, copied.
 * Builds the plan's device tables (twiddles, angle directions, bracket
 * lookup) on the current device.  Errors: INVALID_ARGUMENT (null, V < 2,
 * non-finite, unsorted or out-of-range angles), UNSUPPORTED_SIZE, CUDA,
 * OUT_OF_MEMORY.  On error *plan is NULL. */
bst_status_t bst_plan_create(bst_plan_t* plan, int rays, int angles,
                             const float* angles_rad_host, int pad_factor);

/* Free the plan's device tables (synchronises the device first). NULL is a no-op. */
bst_status_t bst_plan_destroy(bst_plan_t plan);

/* Device workspace in bytes that bst_fbp / bst_backproject need for `slices`
 * slices (extension; no passage -- the memory budget of Sec. 4 bounds what a
 * GPU holds at once; here the caller allocates it): the padded polar
 * spectrum Z[chunk][V][M] and the column-transformed
 * grid T[chunk][N][M] (complex64) for a chunk of slice pairs sized to stay
 * resident in L2 where possible.  0 for an invalid plan or slices <= 0. */
size_t bst_workspace_bytes(bst_plan_t plan, int slices);

/* BST filtered backprojection (Sec. 2 stages P0..P8 with the FBP weight
 * x = B[F y], Sec. 1): volume[s] = FBP(sinogram[s]) for s < slices.
 *   d_sino    [slices][V][N] float32, device
 *   d_g       [M/2] float32 filter taps in BST form (g[k] = h^(sigma_k)/|sigma_k|),
 *             device, or NULL for the ramp |sigma| (g = 1)
 *   d_volume  [slices][N][N] float32, device, must not overlap d_sino
 *   d_ws      device workspace of ws_bytes >= bst_workspace_bytes(plan, slices)
 * Slices are transformed two at a time as the real and imaginary parts of
 * one complex line; an odd last slice is paired with zeros.
 * Errors: INVALID_ARGUMENT, WORKSPACE_TOO_SMALL, CUDA. */
bst_status_t bst_fbp(bst_plan_t plan, const float* d_sino, int slices,
                     const float* d_g, float* d_volume,
                     void* d_ws, size_t ws_bytes, bst_stream_t stream);

/* Plain BST backprojection b = B y via Eq. 3 (weight 1/sigma).  The DC bin
 * is zero, so b is defined up to an additive constant (Eq. 3 holds for
 * sigma > 0 only).  Arguments as bst_fbp. */
bst_status_t bst_backproject(bst_plan_t plan, const float* d_sino, int slices,
                             float* d_volume, void* d_ws, size_t ws_bytes,
                             bst_stream_t stream);

/* BST filtered backprojection with the pre-reconstruction stages fused into
 * its first stage (the paper's stages N and C of Sec. 3, and window P1):
 *   normalization (Sec. 1 (a)), when d_flat != NULL: d_sino holds photon
 *     counts I and y = -log[(I - D)/(I0 - D)], both differences clamped to
 *     >= 1e-6; d_flat (I0) and d_dark (D, or NULL for 0) are [slices][N],
 *     the detector row of each slice;
 *   centering (Sec. 1 (b)): the measured rays are y(t - beta); they are
 *     shifted back by `shift` = beta in detector samples (|shift| < N) with
 *     the exact band-limited shift on the padded grid (spectrum times
 *     exp(+2 pi i k shift / M));
 *   window (P1): kb_beta > 0 multiplies the centered rays by the
 *     Kaiser-Bessel window I0(kb_beta sqrt(1 - (t/h)^2)) / I0(kb_beta),
 *     |t| <= h = kb_halfwidth (detector units, t in [-1, 1)).
 * All zero/NULL: identical to bst_fbp.  Other arguments as bst_fbp.
 * Errors: INVALID_ARGUMENT, WORKSPACE_TOO_SMALL, CUDA. */
bst_status_t bst_fbp_prep(bst_plan_t plan, const float* d_sino, int slices,
                          const float* d_dark, const float* d_flat, float shift,
                          float kb_beta, float kb_halfwidth, const float* d_g,
                          float* d_volume, void* d_ws, size_t ws_bytes, bst_stream_t stream);

/* Device workspace in bytes for radon_adjoint and bst_fbp_filter_grad. */
size_t bst_adjoint_workspace_bytes(bst_plan_t plan, int slices);

/* Exact adjoint (transpose) of the discrete operator of bst_fbp (mode
 * FILTER, taps d_g) or bst_backproject (mode BACKPROJECT, d_g ignored): a
 * Fourier-slice projector (the FST dual of Sec. 2): 2D FFT of the zero-
 * extended image, Cartesian-to-polar transpose of the bilinear gridding,
 * weight, 1D inverse FFT along t, crop to N samples.
 *   d_volume [slices][N][N] -> d_sino [slices][V][N], device float32.
 * The first call builds the plan's cell lists of the gridding (device
 * memory owned by the plan); it synchronises the stream.
 * Errors: INVALID_ARGUMENT (also for a plan with KB gridding),
 * WORKSPACE_TOO_SMALL, CUDA, OUT_OF_MEMORY. */
bst_status_t radon_adjoint(bst_plan_t plan, bst_mode_t mode, const float* d_g,
                           const float* d_volume, int slices, float* d_sino,
                           void* d_ws, size_t ws_bytes, bst_stream_t stream);

/* Gradient of sum(grad_vol * FBP(sino; g)) with respect to the M/2 filter
 * taps g (the autograd backward of bst_fbp's d_g).  Extension; no passage:
 * the paper defines the filter weight of stage P4 (Sec. 1's filter F in
 * BST form), not its gradient, which this library adds for learning taps:
 *   d_grad_g[m] = sum over slices, angles j and |k| = m of
 *                 Re(conj(lambda_j[k]) * Y_j[k]),
 * Y = dt * DFT of the padded rays, lambda = grad_vol pulled back through the
 * crop, 2D transform, gridding and DC mean.  Deterministic (fixed reduction
 * order).  d_grad_g is overwritten.  Workspace: bst_adjoint_workspace_bytes.
 * A plan with KB gridding is rejected (INVALID_ARGUMENT). */
bst_status_t bst_fbp_filter_grad(bst_plan_t plan, const float* d_sino,
                                 const float* d_grad_vol, int slices,
                                 float* d_grad_g, void* d_ws, size_t ws_bytes,
                                 bst_stream_t stream);

/* Backward of x = FBP(sino; g) for autograd: both gradients of
 * <grad_vol, x> from one polar pull-back of grad_vol per chunk of slices.
 *   d_grad_sino [slices][V][N]: the adjoint applied to grad_vol (as
 *               radon_adjoint, mode FILTER, taps d_g), or NULL to skip;
 *   d_grad_g    [M/2]: as bst_fbp_filter_grad (overwritten), or NULL to skip
 *               (then d_sino may be NULL).
 * Results equal those of the two separate calls.  Workspace:
 * bst_adjoint_workspace_bytes.  A plan with KB gridding is rejected.
 * Errors: INVALID_ARGUMENT (nothing requested, aliasing), WORKSPACE_TOO_SMALL,
 * CUDA, OUT_OF_MEMORY. */
bst_status_t bst_fbp_backward(bst_plan_t plan, const float* d_sino,
                              const float* d_grad_vol, int slices, const float* d_g,
                              float* d_grad_sino, float* d_grad_g, void* d_ws,
                              size_t ws_bytes, bst_stream_t stream);

/* Device workspace in bytes for brute_backproject with a filter (0 without). */
size_t brute_workspace_bytes(bst_plan_t plan, int slices, int filtered);

/* Slant-stack backprojection, the O(N^3)-per-slice comparator of Sec. 2:
 * b[r][c] = sum_j w_j y_j(u . xi_j) with linear interpolation along t and
 * trapezoid angular weights w_j = (theta_{j+1} - theta_{j-1})/2 (Eq. 2).
 * d_g == NULL: plain B.  Otherwise each angle is first filtered along t with
 * h_k = |sigma_k| g[k] (h_0 = dsigma/4 g[0], h_{M/2} = 0) on the plan's padded
 * grid (SS filtered backprojection, x = B[F y]); the filtered sinogram goes
 * to d_ws (brute_workspace_bytes(plan, slices, 1) bytes).
 * Errors: INVALID_ARGUMENT, WORKSPACE_TOO_SMALL, CUDA. */
bst_status_t brute_backproject(bst_plan_t plan, const float* d_sino, int slices,
                               const float* d_g, float* d_volume,
                               void* d_ws, size_t ws_bytes, bst_stream_t stream);

/* BST filtered backprojection exactly as bst_fbp, for callers that cannot
 * allocate device memory where they reconstruct (an external memory manager
 * owns the device's memory, or a cudaMalloc/cudaFree, which may synchronise
 * the device, is not acceptable in the calling loop).  The paper has no
 * counterpart: this is a deployment variant of the same operator.
 * The call allocates nothing: its scratch is a fixed 8 MiB device array
 * inside the library (bst_noalloc_scratch_bytes()), present on every GPU
 * that loads the library until the process exits.  Plans whose one-pair
 * workspace, (V M + 4 ceil(N/4) M) * 8 bytes, exceeds it (for example
 * N = V > 512 at pad factor 2) are rejected with WORKSPACE_TOO_SMALL.
 * bst_plan_create looks up the array's device address on the plan's device
 * (loading the library's device code there, which places the array in
 * device memory, when the CUDA runtime loads modules lazily), so a call
 * itself does no set-up and allocates nothing.  cudaDeviceReset ends every
 * plan of that device; plans created after it refresh the address.
 * All calls on a device share the one array, so calls that overlap on the
 * GPU (different streams or host threads without ordering) race and corrupt
 * each other's results; serialise them.  No scratch content carries over
 * between calls (every byte read is written earlier in the same call).
 * Other arguments and errors as bst_fbp. */
bst_status_t bst_fbp_noalloc(bst_plan_t plan, const float* d_sino, int slices,
                             const float* d_g, float* d_volume, bst_stream_t stream);

/* Size in bytes of bst_fbp_noalloc's fixed scratch array. */
size_t bst_noalloc_scratch_bytes(void);

/* Device workspace in bytes for bst_fbp_host: two staging buffers per
 * direction for chunks of about 512 MiB of input, plus the forward workspace. */
size_t bst_host_workspace_bytes(bst_plan_t plan, int slices);

/* BST filtered backprojection of a volume in host memory:
 *   h_sino    [slices][V][N] float32, host (page-locked for full overlap)
 *   h_volume  [slices][N][N] float32, host
 *   d_g       as bst_fbp (device memory or NULL)
 *   d_ws      device workspace of bst_host_workspace_bytes(plan, slices)
 * Chunks of slices are uploaded, reconstructed and downloaded with the copies
 * of one chunk overlapping the computation of its neighbours (the overlap of
 * data movement and GPU stages of Sec. 3), on `stream` and two plan-owned copy
 * streams.  Asynchronous: the host buffers must stay valid until `stream`
 * completes, which it does after the last download.  Errors as bst_fbp. */
bst_status_t bst_fbp_host(bst_plan_t plan, const float* h_sino, int slices,
                          const float* d_g, float* h_volume,
                          void* d_ws, size_t ws_bytes, bst_stream_t stream);

/* FFT radix schedule of the plan's forward path: the largest radix of the
 * Stockham passes, 16 (fewer passes) or 8 (fewer registers per thread).
 * Results are identical up to rounding.  Errors: INVALID_ARGUMENT. */
bst_status_t bst_plan_set_schedule(bst_plan_t plan, int max_radix);
int bst_plan_get_schedule(bst_plan_t plan);

/* Interpolation kernel of stage P5 for bst_fbp, bst_backproject,
 * bst_fbp_prep, bst_fbp_host and bst_fbp_noalloc on this plan.
 *   BST_GRID_BILINEAR (width ignored): the default.
 *   BST_GRID_KAISER_BESSEL, width W in {2, 4, 6, 8} bins: classical
 *     convolution gridding.  Each polar sample Y_j[k] of P3, times the P4
 *     weight, is given the area of its polar cell dtheta_j |sigma_k| dsigma
 *     (dsigma / 4 for the DC cell; dtheta_j the trapezoid weights on the half
 *     circle), spread onto the Cartesian frequency grid with the separable
 *     kernel phi(x) = (I0(beta sqrt(1 - (2x/W)^2)) - 1) / (I0(beta) - 1) (KB
 *     without its pedestal) over the W points x in (-W/2, W/2] of each axis,
 *     beta =
 *     pi sqrt((W / alpha)^2 (alpha - 1/2)^2 - 0.8), and after the 2D inverse
 *     FFT each pixel is divided by C(c_p / M) C(r_p / M), C the Fourier
 *     transform of phi.  The result approximates the direct polar sum
 *     sum_{j,k} a_jk exp(2 pi i omega_jk . u) (relative error ~3e-6 at W = 6,
 *     alpha = 2), which bilinear interpolation reaches only to ~1e-1.  At
 *     alpha = 1 the grid has no guard band: accurate inside the inscribed
 *     disk, ill-conditioned (deapodization gain up to ~1e7) at the edge.
 * Builds the plan's KB tables synchronously (a kernel table, the
 * deapodization and, per strip of four Cartesian columns, the samples whose
 * footprint meets it with their work items: about 4 (1 + (W - 1) / 4) V M
 * bytes, ~90 MB at N = V = 2048, alpha = 2, W = 6); synchronises the device.  radon_adjoint, bst_fbp_filter_grad and the ragged batch need a
 * bilinear plan and reject a KB one.  Errors: INVALID_ARGUMENT (kind, width),
 * OUT_OF_MEMORY, CUDA (the plan then stays bilinear). */
bst_status_t bst_plan_set_gridding(bst_plan_t plan, int kind, int width);
/* The plan's gridding kind and width (2 for bilinear). Errors: INVALID_ARGUMENT. */
bst_status_t bst_plan_get_gridding(bst_plan_t plan, int* kind, int* width);

/* Launch shape of the plan's forward path (bst_fbp, bst_backproject,
 * bst_fbp_prep, bst_fbp_host, bst_fbp_noalloc).  Extension; no passage.
 * bst_plan_set_forward_config validates every field (max_radix 16 or 8,
 * layout a bst_layout_t, chunk_pairs 1..256, pair_fast 0 or 1, max_lanes 1
 * or 2) and changes nothing on error; bst_workspace_bytes follows the new
 * chunk and lane counts, so size workspaces after setting it.  A plan starts
 * with radix 16, the packed layout, chunks sized to about 64 MiB of
 * workspace, block order column-fastest and two lanes.  A Kaiser-Bessel plan
 * always uses the packed layout.  Errors: INVALID_ARGUMENT. */
bst_status_t bst_plan_set_forward_config(bst_plan_t plan, const bst_fwd_config_t* config);
bst_status_t bst_plan_get_forward_config(bst_plan_t plan, bst_fwd_config_t* config);

/* Autotuner (extension; no passage): time the plan's forward path on a
 * synthetic batch of about 256 MiB (`slices` slices, at least 4, and at
 * least 64 where the default chunk is one pair; <= 0 picks that size) under
 * each candidate launch shape -- radix 16 or 8; packed or
 * paired layout (bilinear plans); the plan's default chunk and, where that
 * is one pair, chunks of 2, 4 and 8 pairs; either block order -- keep the fastest
 * (the best of three timed runs each, after one warm-up run) and return its
 * radix in *chosen (may be NULL).  Allocates and frees its own buffers;
 * synchronises the device. */
bst_status_t bst_plan_autotune(bst_plan_t plan, int slices, int* chosen);

/* ---- ragged batch: sinograms of mixed sizes in one persistent launch ----- */
typedef struct bst_ragged_s* bst_ragged_t;

/* A batch of `items` sinograms, item i reconstructed with plans[i] (plans are
 * borrowed and must outlive the batch).  Items sharing a plan are paired two
 * slices per complex line, in order.  Supported FFT lengths: 256, 512, 768,
 * 1024, 1536, 2048, 3072, 4096.  Errors: INVALID_ARGUMENT, UNSUPPORTED_SIZE,
 * CUDA, OUT_OF_MEMORY. */
bst_status_t bst_ragged_create(bst_ragged_t* batch, int items, const bst_plan_t* plans);
/* Device workspace of the batch: a private Z and T region per pair of items. */
size_t bst_ragged_workspace_bytes(bst_ragged_t batch);
/* Number of pair-items (pairs of items sharing a plan, plus unpaired items). */
int bst_ragged_pair_items(bst_ragged_t batch);
/* Bind device buffers: d_sinos[i] [V_i][N_i], d_volumes[i] [N_i][N_i] (host
 * arrays of device pointers), d_g[i] filter taps or NULL (d_g itself may be
 * NULL: ramp for all; paired items must share their taps).  Builds and
 * uploads the work queue; drops a captured graph.  The queue runs in phases
 * (every ray unit, then every gridding unit, then every row unit, the
 * largest pair-items first); flags bit 1 overlaps neighbouring pair-items'
 * stages instead (stage s of pair-item k at step k + s); bit 0 is a diagnostic that leaves the ray stage of the
 * first pair-item unqueued, so that its dependent units wait until the spin
 * limit and the launch reports BST_ERR_TIMEOUT (used to test the bounded
 * waits).  Every plan must use
 * bilinear gridding (INVALID_ARGUMENT otherwise). */
bst_status_t bst_ragged_bind(bst_ragged_t batch, const float* const* d_sinos, const float* const* d_g,
                             float* const* d_volumes, void* d_ws, size_t ws_bytes, int flags);
/* Iterations (each with a ~256 ns sleep) a dependency wait may spin before it
 * gives up with BST_ERR_TIMEOUT (default 2^22, env BST_SPIN_LIMIT). */
bst_status_t bst_ragged_set_spin_limit(bst_ragged_t batch, int iterations);
/* Reconstruct the bound batch: one cooperative persistent launch (one block
 * per SM claims units of the three stages of every item in dependency order).
 * use_graph != 0: the counter reset and the launch are captured into a CUDA
 * graph on first use and replayed.  Asynchronous on `stream`. */
bst_status_t bst_ragged_fbp(bst_ragged_t batch, int use_graph, bst_stream_t stream);
/* Synchronise `stream`; return and clear the batch's device error (TIMEOUT). */
bst_status_t bst_ragged_status(bst_ragged_t batch, bst_stream_t stream);
bst_status_t bst_ragged_destroy(bst_ragged_t batch);

/* Synchronise `stream` and return the plan's sticky device error (BST_OK if
 * none, BST_ERR_CUDA if the stream reported an error). */
bst_status_t bst_plan_status(bst_plan_t plan, bst_stream_t stream);

/* Static English description of a status code. */
const char* bst_status_string(bst_status_t status);

/* FFT length M of a plan (0 for NULL). */
int bst_plan_fft_length(bst_plan_t plan);

/* Per-stage kernel timing (instrumentation, not part of the method).
 * While enabled, every kernel launch of the plan is followed by a CUDA event
 * record on its stream.  bst_plan_timing synchronises those events, adds the
 * device time of each launch to stage_ms[stage] and its count to
 * launches[stage] (arrays of n entries, n <= 8, caller-owned host memory),
 * and clears the record.  Stages: 0 ray FFT + weight, 1 gridding + column
 * inverse FFT, 2 row inverse FFT + crop, 3 slant-stack prefilter,
 * 4 slant-stack backprojection, 5 adjoint row FFT, 6 adjoint column FFT,
 * 7 adjoint polar gather + inverse FFT along t. */
bst_status_t bst_plan_set_timing(bst_plan_t plan, int enable);
bst_status_t bst_plan_timing(bst_plan_t plan, double* stage_ms, long long* launches, int n);

#ifdef __cplusplus
}
#endif

#endif /* BST_H */

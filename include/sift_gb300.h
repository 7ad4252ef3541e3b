/*
 * sift_gb300.h — C ABI of the GPU-resident, bitwise-deterministic SIFT extractor
 * for NVIDIA GB300 (sm_103a).
 *
 * What it computes (PySIFT, arXiv 2605.17869, §3.2 "GPU Pipeline Stages" and
 * Eq. 1): Gaussian scale-space pyramid built by separable blurs with 4-sigma
 * truncation, difference of Gaussians, 3x3x3 extrema with a contrast gate,
 * sub-pixel refinement solved by Cramer's rule (up to 5 iterations) with Hessian
 * edge rejection, 36-bin orientation histograms smoothed with [1/4, 1/2, 1/4]
 * and refined by a parabola, and 4x4x8 gradient descriptors with the 0.2 clip.
 * Everything stays in device memory (§3.3): outputs are written into device
 * buffers that callers wrap with DLPack.
 *
 * Determinism (§5, "Bitwise Deterministic GPU Execution"): no kernel uses
 * atomics; histograms are per-lane private and merged in a fixed order, and
 * keypoints are compacted by prefix scans in canonical order
 * (octave, layer, row, column, orientation peak). An image's output is
 * bit-identical whether it is extracted alone or inside any batch.
 *
 * Conventions
 *  - Images are FP32 grayscale in [0, 1], row-major, with a row pitch given in
 *    elements (pitch >= W). Image pointers are device pointers owned by the
 *    caller; the extractor only reads them, and they must stay valid until the
 *    work queued on the stream has run.
 *  - Streams are passed as `void*` holding a cudaStream_t (NULL = legacy
 *    default stream). Calls are asynchronous: they queue work and return
 *    without waiting for the GPU. Argument errors are reported synchronously;
 *    counts and truncation are device-side results.
 *  - Output buffers are caller-owned device memory with capacity max_kpts
 *    keypoints (descriptors: max_kpts x 128 floats, row-major).
 *  - A handle owns its device workspace, plans and CUDA graphs. It is not
 *    thread-safe: use one handle per host thread, and order calls on one
 *    handle on a single stream (the workspace is reused by the next call).
 *  - No entry point aborts; each returns a sift_status. sift_last_error()
 *    gives a message for the last failure on a handle.
 */
#ifndef SIFT_GB300_H
#define SIFT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SIFT_OK = 0,
  SIFT_W_TRUNCATED = 1,   /* a capacity was hit; output kept in canonical order */
  SIFT_PENDING = 2,       /* serving: request not finished yet */
  SIFT_E_INVALID = -1,    /* bad argument (null pointer, size < min_octave_side, ...) */
  SIFT_E_OOM = -2,        /* device allocation failed */
  SIFT_E_CUDA = -3,       /* a CUDA runtime call failed */
  SIFT_E_BUDGET = -4,     /* serving: request can never fit the memory budget */
  SIFT_E_TIMEOUT = -5,    /* a bounded wait ran out */
  SIFT_E_NOTFOUND = -6    /* serving: unknown ticket */
} sift_status;

/* Extraction parameters. sift_params_default() gives plain SIFT as evaluated
 * here: 3 scales per octave, sigma0 1.6, assumed input blur 0.5, no
 * upsampling (and, when it is switched on, none above 4,000,000 input
 * pixels), octaves while min side >= 16, contrast threshold 0.04/3, edge
 * ratio 10, border 5, 5 refinement iterations, pre-gate 0.5 x threshold,
 * secondary orientation peaks at >= 0.8 of the maximum, capacity and top-K
 * cap of 8192 keypoints per image. sift_create() and sift_octave_geometry()
 * reject (SIFT_E_INVALID) values outside the ranges given per field, and a
 * sigma0 whose largest blur radius (ceil(4 sigma)) exceeds 16 pixels. */
typedef struct {
  int n_scales;          /* S: scales per octave (2..6) */
  float sigma0;          /* base scale of each octave; > 0 */
  float init_blur;       /* blur already present in the input; >= 0 */
  int upsample;          /* 1: first octave from the 2x bilinear magnified input */
  int min_octave_side;   /* keep octaves while min(H_o, W_o) >= this; >= 16,
                            above the largest blur radius and 2 x border */
  float contrast_thr;    /* |interpolated DoG| must be >= this; > 0 */
  float edge_ratio;      /* principal curvature ratio limit r; > 0 */
  int border;            /* candidates need b <= x < W-b, b <= y < H-b; >= 1 */
  int max_refine_iter;   /* refinement iterations (paper: 5); >= 1 */
  float prefilter_ratio; /* candidates need |D| > prefilter_ratio * contrast_thr; >= 0 */
  float ori_peak_ratio;  /* orientation peaks >= ratio * histogram maximum; (0, 1] */
  int max_kpts;          /* output capacity and top-K cap (by response); > 0 */
  int upright;           /* 1: orientation fixed to 0, one keypoint per extremum */
  int dsp;               /* 1: DSP-SIFT pooling (§3.2): histograms of 5 relative
                            scales {1/2, 1/sqrt2, 1, sqrt2, 2}, each a 32 x 32
                            sample patch, pooled before normalisation; 0 or 1 */
  int rootsift;          /* 1: RootSIFT epilogue (L1 normalise, square root, §3.2) */
  int upsample_max_px;   /* with upsample = 1, an image of more than this many
                            input pixels keeps its own resolution as the first
                            octave (the paper's VRAM-adaptive suppression of the
                            double image above 4 MP, §1 and §5); decided per
                            image, also within a batch; 0: no limit; >= 0 */
  int fp16_pyramid;      /* 1: the levels of every octave above 0 are stored as
                            IEEE binary16 (rounded to nearest, ties to even) and
                            read back into FP32 for all arithmetic; octave 0 stays
                            FP32 (§3.2, "fp16 storage with fp32 compute (octave 0
                            in fp32)"), halving those octaves' pyramid memory and
                            traffic; 0 or 1 (default 0) */
} sift_params;

/* Keypoint outputs: structure of arrays in device memory, capacity max_kpts.
 * x, y, sigma are in input-image pixels (x right, y down); angle is in degrees
 * in [0, 360), measured from +x towards +y; response is |interpolated DoG|;
 * octave is the pyramid octave (0 = first, the magnified one when upsampling);
 * layer is the DoG layer 1..S. */
typedef struct {
  float *x, *y, *sigma, *angle, *response;
  int *octave, *layer;
} sift_kpts_dev;

typedef struct sift_handle sift_handle;
typedef struct sift_server sift_server;

/* Fill *p with the defaults above (max_kpts = 8192). */
sift_status sift_params_default(sift_params *p);

/* Create a handle. The handle copies *p and creates its streams, events and
 * pinned host descriptors on the current device; device workspace is allocated
 * lazily on the first extraction and grown when a larger input arrives.
 * Errors: SIFT_E_INVALID on a null or out-of-range parameter; SIFT_E_CUDA if
 * no CUDA device is usable (nothing is created then). */
sift_status sift_create(const sift_params *p, sift_handle **out);

/* Release a handle and all device memory, graphs and streams it owns. The
 * caller must make sure no work queued by this handle is still running. */
sift_status sift_destroy(sift_handle *h);

/* Extract keypoints and descriptors of one image (Eq. 1, Pyr -> DoG -> Ext ->
 * Ori -> Desc, all on the device).
 *   img_dev      device pointer, H x W floats, row pitch pitch_elems (>= W)
 *   stream       cudaStream_t the work is queued on
 *   out_kpts     caller-owned SoA buffers, capacity max_kpts each
 *   out_desc_dev caller-owned, max_kpts x 128 floats
 *   out_count_dev caller-owned device int: number of keypoints written
 * Keypoints beyond max_kpts are dropped keeping the largest responses (ties:
 * canonical order); the kept ones are written in canonical order.
 * Returns SIFT_OK once the work is queued; SIFT_E_INVALID for bad arguments
 * (including min(H, W) below min_octave_side, and an image whose first octave
 * is too large to address: its n_scales + 3 levels of H_0 rows by W_0 rounded
 * up to 32 floats must hold fewer than 2^32 floats, i.e. up to about 21,800 x
 * 21,800 pixels at n_scales = 3, where H_0 x W_0 is 2H x 2W when the image is
 * magnified), SIFT_E_OOM / SIFT_E_CUDA on allocation or launch failure. */
sift_status sift_extract(sift_handle *h, const float *img_dev, int H, int W, int pitch_elems,
                         void *stream, sift_kpts_dev out_kpts, float *out_desc_dev,
                         int *out_count_dev);

/* Extract n images of arbitrary sizes in one pass: every stage runs as one
 * persistent kernel per octave level over a flattened tile queue covering all
 * images, captured in a CUDA graph. Each image's output is bit-identical to
 * its sift_extract() output.
 *   imgs_dev[i], H[i], W[i], pitch_elems[i]  host arrays describing image i
 *   out_kpts[i], out_desc[i]                 host arrays of device buffers
 *   out_counts_dev                           device int[n]
 * A batch of more than 128 images runs as consecutive launches of at most 128
 * (outputs unchanged); sift_pack_outputs and sift_last_stats then refuse.
 * With the tuning's batch_lanes at k > 1 (default 2), a batch of 2 to 128
 * images is cut into min(k, n) contiguous parts of about equal pixel counts
 * that run concurrently: the first on `stream`, each other one on a stream of
 * the handle that waits for `stream` at the call and that `stream` waits for
 * before returning, so work queued on `stream` afterwards sees every part.
 * Each part has its own graph and scratch buffers; outputs are unchanged.
 * Errors as sift_extract. */
sift_status sift_extract_batch(sift_handle *h, int n, const float *const *imgs_dev,
                               const int *H, const int *W, const int *pitch_elems, void *stream,
                               const sift_kpts_dev *out_kpts, float *const *out_desc,
                               int *out_counts_dev);

/* Allocation-free extraction of one image, for callers that cannot call
 * cudaMalloc: plug-ins whose host framework owns all device memory, and
 * real-time loops that forbid any allocation after start-up. The paper has no
 * counterpart; this is a deployment variant of sift_extract().
 * No handle: it takes the parameters directly, because creating a handle
 * allocates. Its scratch memory (descriptor and workspace) is a fixed 64 MiB
 * __device__ array inside the library, which every GPU that loads the library
 * holds until the process exits. It allocates nothing: no cudaMalloc,
 * cudaFree, stream-ordered or pinned allocation, and no CUDA graph.
 *   Arguments, outputs and results are those of sift_extract() (same kernels,
 *   bit-identical output). Returns SIFT_E_BUDGET if the image needs more than
 *   the fixed scratch (about 1.6 Mpx without upsampling, about 0.4 Mpx with
 *   it), SIFT_E_INVALID for bad arguments, SIFT_E_CUDA on a launch failure.
 *   The first call on a device (which must be the current device) resolves the
 *   scratch array's device address and sets kernel attributes; make that
 *   first call before any stream capture.
 *   Every call shares the one scratch array, and it keeps the last call's
 *   contents (nothing in it needs clearing). Calls whose GPU work overlaps,
 *   e.g. on two unordered streams, race on it: order them on one stream. */
sift_status sift_extract_noalloc(const sift_params *p, const float *img_dev, int H, int W,
                                 int pitch_elems, void *stream, sift_kpts_dev out_kpts,
                                 float *out_desc_dev, int *out_count_dev);

/* Symmetric ratio-test matcher (§3.4 "Descriptor Matching", first backend).
 * The similarity matrix of two descriptor sets is formed from fp16
 * tensor-core products (tcgen05, FP32 accumulation): for every descriptor
 * its nearest neighbour in the other set (largest dot product, ties to the
 * smaller index) and the second nearest. A pair (i, j) is kept when each is
 * the other's nearest neighbour and both pass Lowe's ratio test
 * d1 < ratio * d2 on the unit-vector distance d = sqrt(2 - 2 s).
 *   desc_a: n_a x 128 FP32 (device, row-major, 16-byte aligned, unit
 *   vectors, e.g. an extraction's output); desc_b: n_b x 128 likewise.
 *   out_match_a: device, n_a ints: j for a kept pair (i, j), else -1; -2 in
 *   every entry if a bounded device wait gave up (the run is not valid).
 * Asynchronous on `stream`; the handle keeps a small workspace that grows with
 * n_a + n_b. Errors: SIFT_E_INVALID for a null pointer, n_a or n_b outside
 * [0, 65536] or ratio outside (0, 1]; SIFT_E_OOM / SIFT_E_CUDA. With fewer
 * than two descriptors on either side no pair is kept. */
sift_status sift_match(sift_handle *h, const float *desc_a, int n_a, const float *desc_b, int n_b,
                       float ratio, void *stream, int *out_match_a);

/* Pack the outputs of the last extraction call on this handle (at most 128
 * images; after a larger batch, which runs as several launches, the call is
 * refused) into one device block, for a single device-to-host copy. Queue it on the
 * extraction's stream, after the extraction and before the next one.
 * Layout, N = the total kept keypoints of the batch, images in batch order:
 * N x 128 float descriptors, then N floats each of x, y, sigma, angle,
 * response, then N int32 each of octave, layer (540 bytes per keypoint; the
 * per-image counts split it). dst_dev: device, 16-byte aligned, at least
 * 540 x images x max_kpts bytes. Asynchronous. Errors: SIFT_E_INVALID for a
 * null or misaligned dst, a short dst, no extraction yet, or a last batch of
 * more than 128 images; SIFT_E_CUDA. */
sift_status sift_pack_outputs(sift_handle *h, void *stream, void *dst_dev, size_t dst_bytes);

/* GPU MAGSAC++ homography verification (§3.6 "GPU MAGSAC++"): the best of
 * n_hyp minimal-sample homographies under the MAGSAC++ score.
 *   xa, xb: device, n x 2 FP32 (x, y) points of the two images, 8-byte aligned;
 *   correspondence i is xa[i] -> xb[i] (e.g. matched keypoints), n >= 4.
 *   samples: device, n_hyp x 4 int32 indices into [0, n): the random draw is
 *   the caller's (the Python binding draws 4 distinct indices per hypothesis
 *   from a seeded generator). An index outside [0, n) makes that hypothesis
 *   invalid; it is never read.
 *   sigma_max: upper bound of the inlier noise in pixels (> 0).
 * Per hypothesis: the normalised DLT in FP64 (Hartley normalisation, the 8 x 8
 * system with h33 = 1 by pivoted elimination, de-normalised, H[2][2] = 1); a
 * sample is invalid (score +inf) if three of its points are collinear in
 * either image or the system is (near-)singular. Score: the sum over all
 * correspondences of the MAGSAC++ loss of the forward transfer error
 * r = |pi(H xa) - xb|: the chi (4 degrees of freedom) likelihood marginalised
 * over the noise sigma in [0, sigma_max], truncated at k sigma_max with k the
 * 0.99 chi quantile (3.644), as an M-estimator loss; lower is better.
 * Outputs (device): H_out 9 doubles, row-major, of the best hypothesis
 * (smallest score, ties to the smaller index; zeros if none is valid);
 * best_out its index or -1; score_out its score (+inf if none);
 * inliers_out n bytes, 1 where r <= k sigma_max under H_out; scores_out
 * (optional, may be NULL) the n_hyp scores. Scores are bitwise reproducible.
 * Asynchronous on `stream`; the handle keeps a workspace of about 80 bytes
 * per hypothesis. Errors: SIFT_E_INVALID for a null pointer, misaligned
 * points, n outside [4, 2^24], n_hyp outside [1, 2^20] or sigma_max outside
 * (0, 1e6); SIFT_E_OOM / SIFT_E_CUDA. */
sift_status sift_magsac(sift_handle *h, const float *xa, const float *xb, int n, const int *samples,
                        int n_hyp, float sigma_max, void *stream, double *H_out, int *best_out,
                        float *score_out, unsigned char *inliers_out, float *scores_out);

/* Statistics of the last extraction on this handle, read after synchronising
 * its stream. stats receives, per image i of the last call (up to max_images):
 *   stats[4*i+0] candidates (extrema after the gate), stats[4*i+1] refined
 *   keypoints, stats[4*i+2] oriented keypoints before the cap,
 *   stats[4*i+3] truncation flags (bit 0 candidate capacity, bit 1 oriented
 *   capacity, bit 2 top-K cap applied).
 * Returns SIFT_W_TRUNCATED if any capacity was exceeded, else SIFT_OK;
 * SIFT_E_INVALID if the last batch had more than 128 images (it ran as several
 * launches, and the statistics cover one launch); SIFT_E_TIMEOUT if a wait of
 * the single-pass keypoint compaction gave up (a bounded wait for another
 * block's published count; it is not expected to happen): that run's counts
 * and keypoints are then not valid, though every write stayed within its
 * buffers and the handle remains usable. Tests exercise that path through the
 * environment variables SIFT_TEST_LOOKBACK_SPINS (poll limit of one wait) and
 * SIFT_TEST_LOOKBACK_HOLD (index of a compaction block that never publishes
 * its count), read when a handle is created. */
sift_status sift_last_stats(sift_handle *h, int *stats, int max_images);

/* Pyramid geometry for an H x W input under the handle's parameters:
 * *n_octaves octaves; *total_elems floats for sift_build_pyramid's packed
 * layout [octave][level 0..S+2][H_o][W_o] (no padding). */
sift_status sift_pyramid_size(sift_handle *h, int H, int W, int *n_octaves, size_t *total_elems);

/* Octave geometry of an H x W input under *p, computed on the host alone (no
 * handle and no device): the image is magnified when upsample is set and H*W
 * is at most upsample_max_px (0: no limit; §1 and §5), octave 0 is then
 * 2H x 2W, each further octave halves both sides rounding down (§3.2), and
 * octaves are kept while the smaller side is at least min_octave_side.
 *   *n_octaves, *magnified   outputs (magnified: 1 or 0)
 *   heights, widths          host arrays: octave o's size for o < min(*n_octaves,
 *                            cap); either may be NULL when cap is 0
 * Errors: SIFT_E_INVALID for a null p, n_octaves or magnified, invalid
 * parameters, H or W below 1, or cap < 0 (or cap > 0 with a NULL array). */
sift_status sift_octave_geometry(const sift_params *p, int H, int W, int *n_octaves,
                                 int *magnified, int *heights, int *widths, int cap);

/* Build the Gaussian pyramid of one image (the first stage of sift_extract,
 * same kernels: §3.2's scale space of separable 4-sigma blurs, incremental
 * levels and decimated octaves) and copy it, packed as above, into out_dev
 * (capacity out_elems floats). For inspection and tests. SIFT_E_INVALID if
 * out_elems is below sift_pyramid_size()'s total or pitch_elems < W. */
sift_status sift_build_pyramid(sift_handle *h, const float *img_dev, int H, int W,
                               int pitch_elems, void *stream, float *out_dev, size_t out_elems);

/* Per-kernel timing. When enabled, the graphs captured afterwards carry CUDA
 * event nodes around every launch, and sift_kernel_times() returns, for the
 * last extraction, the summed device time in milliseconds and the launch count
 * of each kernel class:
 *   0 blur levels, 1 base level (blur of the input / magnified input),
 *   2 DoG extrema scan, 3 decimation (no separate launch: it is fused into
 *   the first level blur of each octave), 4 candidate and keypoint
 *   compaction and the top-K cap, 5 descriptor, 6 refinement,
 *   7 orientation. Classes at or above n_classes are left out. While profiling
 * is on, sift_extract_batch runs a batch as one lane, so that every kernel is
 * timed alone. Reading synchronises the handle's last run. */
sift_status sift_set_profiling(sift_handle *h, int enable);
sift_status sift_kernel_times(sift_handle *h, double *ms, int *launches, int n_classes);

/* Number of CUDA kernels the last extraction on this handle launched (one
 * graph replay per lane; a batch run as k lanes counts each lane's kernels).
 * Host-only: no synchronisation. */
sift_status sift_last_launch_count(sift_handle *h, int *kernels);

/* Autotuner. The tuning is the set of launch shapes the extraction uses
 * (tile heights and persistent-grid sizes). Tiles and grids decide only
 * which CTA computes what, never the arithmetic, so every tuning gives
 * bit-identical outputs. Its JSON form, every key optional:
 *   {"blur_tile_rows": [[r_1, ..., r_{S+2}], ...],  per octave, one entry per
 *                                                   level blur; 32 or 64 rows
 *                                                   (binary16 levels of the
 *                                                   fp16 mode always use 32);
 *                                                   a flat list sets octave 0
 *    "blur_ctas_per_sm": [c_0, c_1, ...],           level blurs, per octave
 *    "extrema_ctas_per_sm": c, "orientation_ctas_per_sm": c,
 *    "descriptor_ctas_per_sm": c, "compaction_ctas_per_sm": c,
 *    "batch_lanes": k}                              sift_extract_batch: whole
 *                                                   batch in one pass (1), or
 *                                                   up to k concurrent parts
 *                                                   (2, the default, to 4)
 * with c the resident CTAs per SM of that persistent grid, 0 (the default)
 * meaning the kernel's occupancy maximum and larger values capped by it.
 * sift_set_tuning changes only the keys given (SIFT_E_INVALID on a malformed
 * string, an unknown key or a value out of range); sift_get_tuning writes the
 * full tuning (SIFT_E_INVALID if len is too small).
 *
 * sift_autotune: for each level blur of octave 0, time 32- and 64-row tiles
 * on a synthetic H x W pyramid on `stream` and keep the faster. */
sift_status sift_autotune(sift_handle *h, int H, int W, void *stream);
sift_status sift_get_tuning(sift_handle *h, char *json, size_t len);
sift_status sift_set_tuning(sift_handle *h, const char *json);

/* Autotune on a real batch: the arguments of sift_extract_batch (1 to 128
 * images), plus from_cache (host, may be NULL) set to 1 when the tuning came
 * from the cache. Coordinate descent over whole extraction steps of this
 * batch on `stream` (each run as sift_extract_batch runs it, lanes included),
 * from the defaults: 64-row tiles per level of the three
 * largest octaves, then fewer resident CTAs per SM for their level blurs and
 * for the extrema, orientation, descriptor and compaction grids, then 1 to 4
 * lanes (batch_lanes); a change is kept only if the step gets at least 1%
 * faster, and the result is re-timed against the defaults at the end. The chosen tuning stays on the handle, and on return
 * the output buffers hold this batch's results (a run with that tuning;
 * identical to sift_extract_batch's). Synchronises `stream` while timing.
 * With a tuning cache set (sift_set_tuning_cache), the batch's signature
 * (device and sift_batch_signature) is looked up first: a hit applies the
 * stored tuning and runs the batch once, without timing; a miss tunes and then
 * stores the result. SIFT_E_INVALID also for an unreadable cache file or an
 * invalid entry, and when the cache cannot be written. */
sift_status sift_autotune_batch(sift_handle *h, int n, const float *const *imgs_dev, const int *H,
                                const int *W, const int *pitch_elems, void *stream,
                                const sift_kpts_dev *out_kpts, float *const *out_desc,
                                int *out_counts_dev, int *from_cache);

/* Tuning cache file used by sift_autotune_batch on this handle (path copied;
 * NULL or "" switches the cache off). The file is JSON,
 * {"version": 1, "entries": {"<signature>": <tuning JSON>, ...}}, rewritten
 * through a temporary file and a rename, so readers never see a partial file;
 * with concurrent writers the last rename wins. */
sift_status sift_set_tuning_cache(sift_handle *h, const char *path);

/* Host only. The batch part of a tuning-cache signature: every parameter that
 * changes the work, the image count, total pixels, longest side and a 64-bit
 * FNV-1a hash of the sorted (H, W) list (a reordered batch has the same
 * signature). sift_autotune_batch prefixes "sm<major><minor>x<SMs>;".
 * SIFT_E_INVALID on invalid parameters or sizes, or if len is too small. */
sift_status sift_batch_signature(const sift_params *p, int n, const int *H, const int *W,
                                 char *out, size_t len);

/* Host only: read or write one entry of a tuning cache file. get returns
 * SIFT_E_NOTFOUND when the file or the entry does not exist and SIFT_E_INVALID
 * for a malformed file or a too-small buffer; put replaces or appends the
 * entry (json must be one JSON object) and refuses (SIFT_E_INVALID) to
 * overwrite a file it cannot parse. Signatures may not contain '"', '\\' or
 * control characters. */
sift_status sift_tuning_cache_get(const char *path, const char *signature, char *json, size_t len);
sift_status sift_tuning_cache_put(const char *path, const char *signature, const char *json);

/* ---------------------------------------------------------------- serving
 * Continuous batching: a scheduler thread admits submitted requests while
 * their device-memory estimate fits the budget and a slot is free, forms a
 * step batch of everything admitted, and runs it on one of several worker
 * streams, so steps overlap on the device. Requests that arrive while other
 * steps are running join the next step. Pyramids and outputs stay on the
 * device (§3.3: results are handed to other frameworks by DLPack, without a
 * copy); results are library-owned until released. */
typedef struct {
  sift_status status;   /* SIFT_OK, SIFT_W_TRUNCATED or an error (SIFT_E_TIMEOUT:
                           a compaction wait of the request's step gave up, as in
                           sift_last_stats; its results are not valid) */
  int count;            /* keypoints in the buffers below */
  sift_kpts_dev kpts;   /* device buffers, valid until sift_serve_release */
  float *desc;          /* device, count x 128 */
  double submit_to_done_ms; /* host-measured latency of this request */
} sift_result;

/* mem_budget_bytes: device memory the server may use for in-flight requests;
 * max_slots: most requests in flight at once. The server uses the handle's
 * parameters; the handle itself must not be used while the server lives. */
sift_status sift_serve_create(sift_handle *h, size_t mem_budget_bytes, int max_slots,
                              sift_server **out);
/* Queue one image. img_dev must stay valid until the request completes (poll
 * returns something other than SIFT_PENDING). SIFT_E_BUDGET if the image
 * alone exceeds the budget. */
sift_status sift_serve_submit(sift_server *s, const float *img_dev, int H, int W, int pitch_elems,
                              uint64_t *ticket);
/* Non-blocking: SIFT_PENDING while queued or running; otherwise fills *out. */
sift_status sift_serve_poll(sift_server *s, uint64_t ticket, sift_result *out);
/* Block until the request is done or timeout_ms passes (SIFT_E_TIMEOUT). */
sift_status sift_serve_wait(sift_server *s, uint64_t ticket, int timeout_ms, sift_result *out);
/* Free a finished request's result buffers. */
sift_status sift_serve_release(sift_server *s, uint64_t ticket);
/* Device-side timing of the server's finished steps (a step is one batched
 * extraction on one of the server's lanes, each lane a stream of its own),
 * oldest first: for up to max_steps of the most recent steps, the lane, the number of images, and the times of CUDA events
 * recorded on the lane's stream before the step's first launch and after its
 * result read-back, in ms after an event recorded when the server was created.
 * (The server keeps the last 65536 steps.)
 * Steps of different lanes whose [start, end] intervals intersect were on the
 * device at the same time, which is how continuous batching overlaps requests
 * that arrive while others run. *n_out receives the number written.
 * SIFT_E_INVALID for a null server or n_out, a negative max_steps, or a null
 * array with max_steps > 0. Host-only: no synchronisation. */
sift_status sift_serve_steps(sift_server *s, int max_steps, int *lane, int *n_images,
                             double *start_ms, double *end_ms, int *n_out);
/* Stop the scheduler (waits for running steps) and free the server. */
sift_status sift_serve_destroy(sift_server *s);

/* Message describing the last error on the handle (never NULL). */
const char *sift_last_error(sift_handle *h);

/* Library version string. */
const char *sift_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SIFT_GB300_H */

// Internal definitions shared by the CUDA translation units of the extractor.
//
// Data layout in device memory (one "engine" = one workspace + descriptor):
//  * Pyramid: per image, per octave o, levels 0..S+2 stored back to back, each
//    H_o rows of `pitch` elements (pitch = W_o rounded up to 32). Elements are
//    FP32, or IEEE binary16 for the octaves above 0 in the fp16 storage mode
//    (OctDev::half); arithmetic is FP32 throughout.
//  * Candidate bitmap: per image, per octave, per DoG layer 1..S, H_o rows of
//    ceil(W_o / 30) 32-bit words; bit k (< 30) of word w in row y marks pixel
//    x = 30 w + k (one word is the row of one extrema strip). Walking the
//    bitmap in memory order is the canonical order (octave, layer, row,
//    column).
//  * Keypoint-stage arrays are per image slices of global arrays; every slice
//    is addressed through the per-image fields of ImgDev.
// All geometry lives in a device-side descriptor (Desc) written before each
// launch, so the captured CUDA graphs depend only on the number of octaves.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace sift {

constexpr int kMaxImg = 128;       // images per device launch (larger batches are split)
constexpr int kMaxOct = 14;        // octaves (2^14 px sides)
constexpr int kMaxScales = 6;      // S <= 6
constexpr int kMaxLevels = kMaxScales + 3;
constexpr int kMaxR = 16;          // largest blur radius supported (halo 16)
constexpr int kOriBins = 36;       // §3.2: 36-bin orientation histogram
constexpr int kMaxPeaks = kOriBins / 2;  // strict circular maxima of 36 bins
constexpr int kDescLen = 128;      // 4 x 4 x 8
constexpr int kBlurTW = 128;       // blur tile width (32 lanes x float4)
constexpr int kBlurHalo = 16;      // staged columns left/right of a blur tile
constexpr int kBmCols = 30;        // columns per bitmap word = extrema strip width (one warp)
constexpr int kExtTH = 32;         // extrema tile rows (one warp streams down them)
constexpr int kChunk = 2048;       // compaction chunk (words or slots)

// Tile-queue kinds: blur with tile height 16/32/64, extrema tiles, decimation.
enum TileKind { TK_BLUR16 = 0, TK_BLUR32 = 1, TK_BLUR64 = 2, TK_EXT = 3, TK_COUNT = 4 };

// Rejection codes of the refinement (0 = kept).
enum RefCode { RC_KEEP = 0, RC_SINGULAR = 1, RC_NOCONV = 2, RC_BOUNDS = 3, RC_CONTRAST = 4, RC_EDGE = 5 };

// Truncation flags per image.
enum { TF_CAND = 1, TF_ORI = 2, TF_TOPK = 4 };

struct OctDev {
  int H, W, pitch, wpr;        // size, row pitch (elements), bitmap words per row
  long long lvl;               // offset of level 0 in the pyramid array, in floats (4-byte units)
  long long lstride;           // elements between consecutive levels (H * pitch)
  long long bm;                // word offset of layer 1's bitmap
  int half;                    // 1: this octave's levels are stored as binary16
  int pad;
};

struct ImgDev {
  const float *src;            // input image (device)
  int H, W, spitch;            // input size and pitch (elements)
  int src_vec_ok;              // 1 if 16-byte aligned rows (vector loads allowed)
  int up;                      // 1 if the first octave is the 2x magnified input
  int n_oct, oct0;             // octaves and index of the first OctDev
  long long bm_begin, bm_words;  // bitmap slice
  int bmc0, bmc_n;             // bitmap chunks [bmc0, bmc0 + bmc_n)
  int cand_cap;                // candidate slots
  long long cand_off;          // slice start in cand / ref / code / npk arrays
  int cc0, cc_n;               // candidate-slot chunks
  int ori_cap;                 // oriented keypoint slots
  long long ori_off;
  int kcap;                    // output capacity (top-K)
  long long fin_off;           // slice start in the final index list
  float *ox, *oy, *osig, *oang, *oresp;
  int *ooct, *olay;
  float *odesc;
  int *ocount;
};

// Dynamic per-image results written by kernels.
struct ImgCounters {
  int n_cand_raw, n_cand, n_ori_raw, n_ori, n_fin, n_ref, flags;
  // Kept keypoints of octave 0 (fp16 storage mode only): the list is in
  // canonical order, so they are its first n_fin0 entries and the keypoints of
  // the binary16 octaves the rest.
  int n_fin0;
};

struct RefRec {               // refined keypoint (octave-local coordinates)
  int o, s, y, x;
  float dx, dy, ds, resp;
};

struct Desc {
  int n_img, n_oct_max, n_scales, upsample;
  float sigma0, contrast_thr, prefilter, edge_ratio;
  int border, max_iter, upright, rootsift;
  float ori_peak_ratio, pad_f[3];
  int n_bm_chunks, n_cc_chunks, dsp, fp16;  // fp16: octaves above 0 stored as binary16
  // workspace arrays
  float *pyr;
  uint32_t *bm;
  int4 *cand;
  RefRec *ref;
  int *code;
  int *npk;
  float *angs;                 // kMaxPeaks per candidate slot
  int2 *ori;                   // (candidate slot, peak index)
  uint32_t *okey;              // response bits of oriented keypoints
  int *fin;                    // final indices into the oriented list
  // Single-pass scan statuses (scan.cuh): per block of the candidate and of
  // the oriented compaction, per image (totals: candidates, then final; 2 x
  // kMaxImg), per image (global offset of its first slot: candidates, then
  // oriented; 2 x kMaxImg), and the word that records a wait that gave up.
  unsigned long long *lb_bm, *lb_cc, *lb_img, *lb_start, *lb_err;
  unsigned lb_epoch;           // this run's epoch, 1 .. 2^30 - 1
  int lb_spins;                // poll limit of one wait
  int lb_hold;                 // test hook: a chunk that never publishes (-1: none)
  int lb_pad;
  ImgCounters *cnt;            // per image
  int *cand_flat;              // [kMaxImg + 1] prefix of n_cand over images
  int *fin_flat;               // [kMaxImg + 1] prefix of n_fin over images
  // geometry
  int tile_pre[TK_COUNT][kMaxOct][kMaxImg + 1];
  int base_pre[2][kMaxImg + 1];  // base-blur tiles (32 rows) of the images with up = 0 / 1
  int bmc_pre[kMaxImg + 1];
  int cc_pre[kMaxImg + 1];
  ImgDev img[kMaxImg];
  OctDev oct[kMaxImg * kMaxOct];
};

// Normalised taps w[0..2R] of one blur, plus the pairs the packed FMAs take
// as operands (prepared on the host so each is one aligned 8-byte constant).
struct BlurTaps {
  float w[2 * kMaxR + 2];     // zero past 2R
  float2 wp[kMaxR + 1];       // (w[2i], w[2i + 1])
  float2 wq[kMaxR + 1];       // (w[2i + 1], w[2i + 2])
  float2 wd[2 * kMaxR + 1];   // (w[j], w[j])
};

// Programmatic dependent launch. Every kernel after the first of a run is
// launched so that its blocks may start while the previous kernel of the
// stream is still finishing. A kernel runs the prologue that needs only the
// descriptor (which the host wrote before the run) and calls pdl_wait before
// it reads anything a previous kernel produced and before it writes any
// global memory; pdl_wait returns once the previous kernel has completed and
// its writes are visible. The level blurs and the extrema scan call
// pdl_trigger when a block starts its last tile, letting their successor's
// blocks take the SMs that the tail frees; other kernels let it launch when
// they exit. In a kernel launched without the attribute both calls do nothing.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// A launch without attributes. Like launch_pdl it returns the status of this
// launch alone: an error an earlier call left in the runtime's last-error
// state is neither reported as this launch's nor cleared.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_plain(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Pyramid element access for the per-keypoint stages, which read octaves of
// either storage type: base = d->pyr + od.lvl, idx in elements of the octave.
__device__ __forceinline__ float lvl_ld(const float *base, bool half, long long idx) {
  if (half) return __half2float(__ldg(reinterpret_cast<const __half *>(base) + idx));
  return __ldg(base + idx);
}

// Index of the image owning flattened item t, given an exclusive prefix pre[0..n].
__device__ __forceinline__ int find_owner(const int *pre, int n, int t) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// reflect-101 for indices in (-n, 2n-1); anything further is clamped (such
// samples only feed outputs outside the image, which are never read).
__device__ __forceinline__ int refl101(int i, int n) {
  i = i < 0 ? -i : i;
  i = i >= n ? 2 * n - 2 - i : i;
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// ---------------------------------------------------------------- launchers
// Pyramid (pyramid.cu)
cudaError_t launch_base_blur(const Desc *d, int R, const BlurTaps &t, int th_kind, bool upsample,
                             int grid, cudaStream_t s);
// pdl: launch as a programmatic dependent of the previous kernel on s.
// storage: 0 FP32 in and out; 1 FP32 source, binary16 output (first level of
// octave 1 in the fp16 storage mode, from_prev_octave only); 2 binary16 in and
// out. Binary16 octaves use 32-row tiles.
cudaError_t launch_level_blur(const Desc *d, int oct, int lvl_out, int R, const BlurTaps &t,
                              int th_kind, int grid, cudaStream_t s, bool from_prev_octave = false,
                              bool pdl = true, int storage = 0);
// Copy one pyramid level (src: the level's first element, `half` for binary16)
// into a dense H x W FP32 plane.
cudaError_t launch_export_level(const float *src, bool half, int pitch, int H, int W, float *dst,
                                cudaStream_t s);
int blur_smem_bytes(int R, int th_kind);
int blur_blocks_per_sm(int R, int th_kind, int mode);
cudaError_t blur_set_attributes();

// Detection (detect.cu)
// pdl: launch as a programmatic dependent of the previous kernel on s.
// half: the octave's levels are binary16 (fp16 storage mode).
cudaError_t launch_extrema(const Desc *d, int oct, int n_scales, int grid, cudaStream_t s,
                           bool pdl = true, bool half = false);
cudaError_t extrema_set_attributes();
// Persistent grid of the extrema scan: SMs x resident blocks per SM.
// Occupancy maxima (resident CTAs per SM) of the persistent keypoint kernels.
int extrema_max_ctas(int n_scales);
int orientation_max_ctas(bool mixed);
int descriptor_max_ctas(bool mixed);
int compact_max_ctas();
cudaError_t cc_compact_occupancy(int *blocks_per_sm);
cudaError_t launch_bm_compact(const Desc *d, int grid, cudaStream_t s);
cudaError_t launch_refine(const Desc *d, int grid, cudaStream_t s);

// Description (describe.cu)
cudaError_t launch_orientation(const Desc *d, int grid, cudaStream_t s, bool mixed = false);
cudaError_t launch_ori_compact(const Desc *d, int grid, cudaStream_t s);
cudaError_t launch_select(const Desc *d, int grid, cudaStream_t s);
// mixed: the pyramid has binary16 octaves (fp16 storage mode).
cudaError_t launch_descriptor(const Desc *d, int grid, cudaStream_t s, bool mixed = false);

// Pack the outputs of the batch described by d into one block (describe.cu).
// The descriptors of the parts of one batch, in batch order (1 to 4).
struct PackSrc {
  const Desc *d[4];
  int n;
};
cudaError_t launch_pack(PackSrc src, void *dst, int n_sm, cudaStream_t s);

// MAGSAC++ homography verification (magsac.cu).
size_t magsac_workspace_bytes(int n_hyp);
cudaError_t launch_magsac(const float *xa, const float *xb, int n, const int *samples, int n_hyp,
                          float sigma_max, void *ws, cudaStream_t s, double *H_out, int *best_out,
                          float *score_out, unsigned char *inliers, float *scores_out);
cudaError_t descriptor_set_attributes();
// Matcher (match.cu)
size_t match_workspace_bytes(int n_a, int n_b);
cudaError_t match_set_attributes();
cudaError_t launch_match(const float *A, int n_a, const float *B, int n_b, float ratio, void *ws,
                         int *out, cudaStream_t s);
int descriptor_smem_bytes();

}  // namespace sift

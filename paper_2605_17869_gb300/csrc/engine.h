// Host-side extraction engine: geometry planning, workspace, descriptor
// upload and per-octave-count CUDA graphs. One engine runs one batch at a time
// on the stream it is given; the server owns several engines so that steps
// overlap on the device.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "../../include/sift_gb300.h"
#include "sift_dev.cuh"

namespace sift {

struct ImgIn {
  const float *src;
  int H, W, pitch;
  sift_kpts_dev k;
  float *desc;
  int *count;
};

enum ProfClass { PC_BLUR = 0, PC_BASE = 1, PC_EXTREMA = 2, PC_DECIMATE = 3, PC_KEYPOINT = 4,
                 PC_DESCRIPTOR = 5, PC_REFINE = 6, PC_ORIENT = 7, PC_COUNT = 8 };

// Launch shapes the autotuner chooses. None of them changes an output bit:
// tiles and grids only decide which CTA computes what.
struct Tuning {
  // Tile-height class (TK_BLUR32 / TK_BLUR64) of the blur that writes level l
  // of octave o; binary16 levels always take 32-row tiles.
  int lvl_kind[kMaxOct][kMaxLevels];
  // Resident CTAs per SM of the persistent grids, 0 meaning the occupancy
  // maximum (larger values are capped by it): the level blurs of octave o, the
  // extrema scans, orientation, descriptor.
  int blur_ctas[kMaxOct];
  int ext_ctas, ori_ctas, desc_ctas;
  int cmp_ctas;  // the two single-pass keypoint compactions
  // sift_extract_batch: k > 1 runs a batch of two or more images as up to k
  // contiguous parts (balanced by pixels) on as many engines and streams at
  // once, so that one part's latency-bound stretches overlap the others'
  // work; 1 runs it on one engine. Outputs are the same either way.
  int batch_lanes;
};
constexpr int kMaxLanes = 4;  // largest batch_lanes

// Poll limit of a single-pass scan wait and the test hook's held block
// (environment SIFT_TEST_LOOKBACK_SPINS / SIFT_TEST_LOOKBACK_HOLD).
void lookback_config(int *spins, int *hold);

// Host-only tuning helpers (tuning.cu).
Tuning default_tuning();
std::string tuning_json(const Tuning &t, int n_scales);
bool parse_tuning(const char *json, int n_scales, const Tuning &base, Tuning *out,
                  std::string *why);
// Key of the tuning cache for a batch: parameters, image count, shapes.
std::string batch_signature(const sift_params &p, int n, const int *H, const int *W);
sift_status cache_get(const char *path, const char *sig, std::string *json);
sift_status cache_put(const char *path, const char *sig, const char *json);

struct WsLayout {
  size_t pyr, bm, cand, ref, code, npk, angs, ori, okey, fin,
      cnt, cand_flat, fin_flat, total;
};

class Engine {
 public:
  explicit Engine(const sift_params &p);
  ~Engine();
  sift_status init();
  // Queue the extraction of n <= kMaxImg images on stream s.
  sift_status run(int n, const ImgIn *imgs, cudaStream_t s);
  // Queue the pyramid stage only (for export); one image.
  sift_status run_pyramid(const ImgIn &img, cudaStream_t s);
  // Whether an H x W input gets the 2x magnified first octave: upsample on
  // and at most upsample_max_px input pixels (0: no limit).
  bool magnify(int H, int W) const;
  // Octave sizes for an input; returns the octave count.
  int octave_sizes(int H, int W, int *hs, int *ws) const;
  // Octave o's levels are stored as binary16 (fp16 storage mode, octaves > 0).
  bool half_octave(int o) const { return P_.fp16_pyramid && o > 0; }
  // Storage mode of the launch that writes level l of octave o (see
  // launch_level_blur): 0 FP32, 1 FP32 source into binary16, 2 binary16.
  int storage(int o, int l) const {
    if (!half_octave(o)) return 0;
    return (l == 1 && !half_octave(o - 1)) ? 1 : 2;
  }
  // Whether an H x W input's first octave is small enough to address with
  // 32-bit offsets within its level stack (n_scales + 3 levels < 2^32 floats).
  bool addressable(int H, int W) const;
  // Workspace bytes a batch needs (serving admission).
  size_t workspace_bytes(int n, const int *H, const int *W) const;
  // Device-side per-image geometry of the last run (valid until the next run).
  const Desc &host_desc() const { return *hdesc_[ring_last_]; }
  const WsLayout &layout() const { return lay_; }
  // Device descriptor of the last run (valid on its stream until the next run).
  const Desc *device_desc() const { return ddesc_; }
  int sm_count() const { return n_sm_; }
  char *workspace() const { return ws_; }

  void set_profiling(bool on);
  bool profiling() const { return profiling_; }
  sift_status kernel_times(double *ms, int *launches, int n_classes);
  sift_status last_stats(int *stats, int max_images);
  int last_launch_count() const { return last_kernels_; }
  // The single-pass scan's gave-up word (device) and the last run's epoch: the
  // run's compaction counts are valid unless the word equals the epoch.
  const unsigned long long *gave_up_word() const { return lb_; }
  unsigned last_epoch() const { return epoch_; }

  Tuning tuning() const { return tun_; }
  void set_tuning(const Tuning &t);
  sift_status autotune(int H, int W, cudaStream_t s);
  // Search the launch shapes on a real batch (n <= kMaxImg) by timing whole
  // extraction steps, and keep the fastest; the outputs end up holding the
  // results of a run with the chosen tuning. step, when given, queues one
  // whole step of the batch on s under this engine's current tuning (the
  // handle runs it as one or several lanes); by default run(n, imgs, s).
  using StepFn = std::function<sift_status()>;
  sift_status autotune_batch(int n, const ImgIn *imgs, cudaStream_t s,
                             const StepFn &step = StepFn());
  // "sm<major><minor>x<SMs>": the device part of a tuning-cache key.
  std::string device_key() const;
  int level_radius(int l) const { return lvl_R_[l]; }

  const sift_params &params() const { return P_; }

  // Fixed-scratch path: everything run() does except allocating. The caller
  // supplies the device descriptor and workspace (see noalloc.cu).
  sift_status init_noalloc();
  sift_status plan_noalloc(const ImgIn &img, Desc *hd, WsLayout *lay, int *max_oct) const {
    return fill_plan(1, &img, *hd, *lay, max_oct);
  }
  cudaError_t enqueue_noalloc(Desc *d_desc, cudaStream_t s, int max_oct, int modes) {
    ddesc_ = d_desc;
    const cudaError_t e = enqueue_all(s, max_oct, modes, nullptr);
    ddesc_ = nullptr;  // not owned: the destructor must not free it
    return e;
  }

  std::string err;
  cudaStream_t last_stream = nullptr;
  int last_n = 0;
  bool last_extract = false;  // the last run was an extraction (outputs described)

 private:
  sift_status fill_plan(int n, const ImgIn *imgs, Desc &hd, WsLayout &lay, int *max_oct) const;
  sift_status ensure_workspace(size_t bytes, cudaStream_t s);
  sift_status upload(Desc *hd, size_t bytes, cudaStream_t s);
  // modes: bit 0 set if an image is processed as is, bit 1 if one is magnified.
  cudaError_t enqueue_pyramid(cudaStream_t s, int max_oct, int modes, std::vector<struct ProfRec> *prof);
  // fork: run the extrema scans of all but the last octave on a side branch
  // (graph capture only; the allocation-free path runs everything in order).
  cudaError_t enqueue_all(cudaStream_t s, int max_oct, int modes, std::vector<struct ProfRec> *prof,
                          bool fork = false);
  sift_status get_graph(int max_oct, int modes, cudaGraphExec_t *out);
  void drop_graphs();
  int grid_blur(int R, int kind, int mode, int ctas = 0) const;
 public:
  // Grid of the single-pass compactions (their scan runs over blocks).
  int compact_grid() const { return grid_of(cmp_max_, tun_.cmp_ctas); }
 private:
  // Single-pass scan statuses: make room for `words`, cleared on allocation.
  sift_status ensure_lb(size_t words, cudaStream_t s);
  int grid_of(int max_ctas, int ctas) const {
    return n_sm_ * std::max(1, ctas > 0 ? std::min(ctas, max_ctas) : max_ctas);
  }
  // Step time (ms, best of 3 x 5 steps) of a batch under tuning t.
  float time_steps(const Tuning &t, const StepFn &step, cudaStream_t s, sift_status *st);

  sift_params P_;
  int dev_ = 0, n_sm_ = 0;
  // Occupancy maxima (resident CTAs per SM) of the extrema scan, orientation
  // and descriptor kernels.
  int ext_max_ = 1, ori_max_ = 1, desc_max_ = 1, cmp_max_ = 1;
  int S_ = 3;
  int base_R_[2] = {0, 0};  // base blur: [0] input as is, [1] 2x magnified input
  BlurTaps base_t_[2] = {};
  int lvl_R_[kMaxLevels] = {};
  BlurTaps lvl_t_[kMaxLevels] = {};
  Tuning tun_{};

  char *ws_ = nullptr;
  size_t ws_cap_ = 0;
  // Scan statuses (scan.cuh), kept apart from the workspace so that no other
  // data ever lands in them: [0] the gave-up word, then 2 x kMaxImg image
  // totals, then the chunks of the run. Epochs tell runs apart.
  unsigned long long *lb_ = nullptr;
  size_t lb_cap_ = 0;
  unsigned epoch_ = 0;
  int lb_spins_ = 0, lb_hold_ = -1;
  WsLayout lay_{};
  Desc *ddesc_ = nullptr;
  static constexpr int kRing = 3;
  Desc *hdesc_[kRing] = {};
  cudaEvent_t hevt_[kRing] = {};
  int ring_ = 0, ring_last_ = 0;
  cudaEvent_t done_ = nullptr;   // recorded after each run
  cudaStream_t cap_ = nullptr;   // capture stream
  // Side branches of the captured graph: octave o's last two levels and extrema
  // scan run on side_[o % kSides].
  static constexpr int kSides = 3;
  cudaStream_t side_[kSides] = {};
  cudaEvent_t fork_ev_[kMaxOct] = {};
  cudaEvent_t join_ev_[kSides] = {};

  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<struct ProfRec> *prof = nullptr;
    int kernels = 0;
  };
  int kernels_ = 0;       // kernels enqueued by the current capture
  int last_kernels_ = 0;  // kernels in the last replayed graph
  std::map<int, GraphEntry> graphs_;
  bool profiling_ = false;
  std::vector<struct ProfRec> *last_prof_ = nullptr;
  bool inited_ = false;
};

// Base-blur modes a plan needs: bit m set when some image has up == m.
inline int base_modes(const Desc &hd) {
  return (hd.base_pre[0][hd.n_img] > 0 ? 1 : 0) | (hd.base_pre[1][hd.n_img] > 0 ? 2 : 0);
}

struct ProfRec {
  cudaEvent_t a, b;
  int cls;
};

// Gaussian taps with 4-sigma truncation, computed in double and rounded to
// float: radius ceil(4 sigma), w_k = exp(-k^2 / 2 sigma^2) / sum.
int gaussian_taps(double sigma, BlurTaps *t);
sift_status validate_params(const sift_params &p, std::string *why);

}  // namespace sift

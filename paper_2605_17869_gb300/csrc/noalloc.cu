// sift_extract_noalloc: one-image extraction that allocates nothing.
//
// Some callers cannot call cudaMalloc: a plug-in hosted by a framework whose
// memory manager owns all device memory (an allocation behind its back can
// fail or fragment its pool), or a real-time loop that forbids allocation
// after start-up so that no call can stall or run out of memory mid-stream.
// This entry point serves them. Its scratch memory (the device descriptor and
// every workspace slice) lives in one file-scope __device__ array of fixed
// size, created when the library's device code is loaded, so a call makes no
// allocation of any kind: no cudaMalloc / cudaFree / cudaMallocAsync, no
// pinned host buffer, no CUDA graph. The geometry is written into the array
// by a one-warp set-up kernel that receives it as a launch parameter.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "engine.h"
#include "scan.cuh"

namespace sift {

namespace {

// 64 MiB: fits one image of up to about 1.6 Mpx without upsampling (e.g.
// 1600x1000), or about 0.4 Mpx with the 2x magnified first octave.
constexpr size_t kScratchBytes = 64ull << 20;
constexpr int kMaxDevices = 64;
constexpr size_t kDescBytes = (sizeof(Desc) + 255) / 256 * 256;

// Shared by every call on a device; it keeps the last call's contents. No
// part of it needs to start at zero: every kernel writes all the entries it
// later reads. Calls whose work overlaps on the GPU (different streams, no
// ordering between them) race on it.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Single-pass scan statuses (scan.cuh) of every call on a device, apart from
// the scratch so that no other data ever lands in them: [0] the gave-up word,
// 2 x kMaxImg image totals, 2 x kMaxImg image starts, then one word per block
// of each compaction (up to 16384 blocks each). Zero at load time; calls are
// told apart by epochs.
constexpr size_t kLbWords = 1 + 4 * kMaxImg + 2 * 16384;
static __device__ unsigned long long g_lb[kLbWords];

// The part of a one-image Desc that is not a per-image table.
struct SetupArgs {
  unsigned char head[offsetof(Desc, tile_pre)];
  int tiles[TK_COUNT][kMaxOct];
  int base_tiles[2];
  int bmc_n, cc_n;
  ImgDev img;
  OctDev oct[kMaxOct];
};

__global__ void k_noalloc_setup(Desc *d, SetupArgs a) {
  const int lane = threadIdx.x;
  unsigned char *dst = reinterpret_cast<unsigned char *>(d);
  for (int i = lane; i < (int)sizeof(a.head); i += 32) dst[i] = a.head[i];
  for (int i = lane; i < TK_COUNT * kMaxOct; i += 32) {
    const int k = i / kMaxOct, o = i % kMaxOct;
    d->tile_pre[k][o][0] = 0;
    d->tile_pre[k][o][1] = a.tiles[k][o];
  }
  if (lane < 2) {
    d->base_pre[lane][0] = 0;
    d->base_pre[lane][1] = a.base_tiles[lane];
  }
  if (lane == 0) {
    d->bmc_pre[0] = 0;
    d->bmc_pre[1] = a.bmc_n;
    d->cc_pre[0] = 0;
    d->cc_pre[1] = a.cc_n;
    d->img[0] = a.img;
  }
  for (int o = lane; o < a.img.n_oct; o += 32) d->oct[o] = a.oct[o];
}

// Per-device set-up state. Only a successful set-up is kept: after a failure
// (for example a call made before the device's context is usable) the next
// call on that device tries again.
struct DeviceScratch {
  std::mutex mu;
  void *ptr = nullptr;  // device address of g_scratch on this device, once set up
  unsigned long long *lb = nullptr;  // device address of g_lb
  unsigned epoch = 0;   // the last call's scan epoch (guarded by g_plan_mu)
};
DeviceScratch g_dev[kMaxDevices];

// Resolve the scratch array's device address and set the kernels'
// shared-memory limits on the current device. Returns the failing call's
// status, or cudaSuccess.
cudaError_t setup_device(DeviceScratch &ds) {
  std::lock_guard<std::mutex> lk(ds.mu);
  if (ds.ptr) return cudaSuccess;
  void *ptr = nullptr, *lb = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&lb, g_lb);
  if (e == cudaSuccess) ds.lb = static_cast<unsigned long long *>(lb);
  if (e == cudaSuccess) e = blur_set_attributes();
  if (e == cudaSuccess) e = descriptor_set_attributes();
  if (e == cudaSuccess) e = extrema_set_attributes();
  if (e == cudaSuccess && ptr) ds.ptr = ptr;
  return e == cudaSuccess && !ptr ? cudaErrorInvalidSymbol : e;
}

std::mutex g_plan_mu;
Desc g_host_desc;  // host-side planning buffer (static storage, not allocated per call)

}  // namespace

}  // namespace sift

using namespace sift;

extern "C" sift_status sift_extract_noalloc(const sift_params *p, const float *img_dev, int H,
                                            int W, int pitch_elems, void *stream,
                                            sift_kpts_dev out_kpts, float *out_desc_dev,
                                            int *out_count_dev) {
  if (!p || !img_dev || !out_desc_dev || !out_count_dev || !out_kpts.x || !out_kpts.y ||
      !out_kpts.sigma || !out_kpts.angle || !out_kpts.response || !out_kpts.octave ||
      !out_kpts.layer)
    return SIFT_E_INVALID;
  if (validate_params(*p, nullptr) != SIFT_OK) return SIFT_E_INVALID;
  if (H < p->min_octave_side || W < p->min_octave_side || pitch_elems < W) return SIFT_E_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SIFT_E_CUDA;
  // First call on this device (which must be current): resolve the device
  // address of the scratch array and set the kernels' shared-memory limits.
  // A failed set-up is not remembered; the next call retries it.
  DeviceScratch &ds = g_dev[dev];
  if (setup_device(ds) != cudaSuccess) return SIFT_E_CUDA;

  Engine eng(*p);  // planning and launch sequencing only; it allocates nothing
  const sift_status ist = eng.init_noalloc();  // parameters were validated above
  if (ist != SIFT_OK) return ist;
  if (!eng.addressable(H, W)) return SIFT_E_BUDGET;  // far beyond the scratch array
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_plan_mu);
  Desc &hd = g_host_desc;
  WsLayout lay;
  int M = 0;
  ImgIn in{img_dev, H, W, pitch_elems, out_kpts, out_desc_dev, out_count_dev};
  if (eng.plan_noalloc(in, &hd, &lay, &M) != SIFT_OK) return SIFT_E_INVALID;
  if (kDescBytes + lay.total > kScratchBytes) return SIFT_E_BUDGET;  // image too large

  char *base = static_cast<char *>(ds.ptr);
  Desc *d_desc = reinterpret_cast<Desc *>(base);
  char *ws = base + kDescBytes;
  hd.pyr = reinterpret_cast<float *>(ws + lay.pyr);
  hd.bm = reinterpret_cast<uint32_t *>(ws + lay.bm);
  hd.cand = reinterpret_cast<int4 *>(ws + lay.cand);
  hd.ref = reinterpret_cast<RefRec *>(ws + lay.ref);
  hd.code = reinterpret_cast<int *>(ws + lay.code);
  hd.npk = reinterpret_cast<int *>(ws + lay.npk);
  hd.angs = reinterpret_cast<float *>(ws + lay.angs);
  hd.ori = reinterpret_cast<int2 *>(ws + lay.ori);
  hd.okey = reinterpret_cast<uint32_t *>(ws + lay.okey);
  hd.fin = reinterpret_cast<int *>(ws + lay.fin);
  hd.cnt = reinterpret_cast<ImgCounters *>(ws + lay.cnt);
  hd.cand_flat = reinterpret_cast<int *>(ws + lay.cand_flat);
  hd.fin_flat = reinterpret_cast<int *>(ws + lay.fin_flat);

  const int gc = eng.compact_grid();
  if (1 + 4 * kMaxImg + 2 * (size_t)gc > kLbWords) return SIFT_E_BUDGET;
  if (ds.epoch >= kLbEpochMask) {  // epochs wrapped: clear every earlier status
    if (cudaMemsetAsync(ds.lb, 0, sizeof(g_lb), s) != cudaSuccess) return SIFT_E_CUDA;
    ds.epoch = 0;
  }
  hd.lb_err = ds.lb;
  hd.lb_img = ds.lb + 1;
  hd.lb_start = hd.lb_img + 2 * kMaxImg;
  hd.lb_bm = hd.lb_start + 2 * kMaxImg;
  hd.lb_cc = hd.lb_bm + gc;
  hd.lb_epoch = ++ds.epoch;
  lookback_config(&hd.lb_spins, &hd.lb_hold);

  SetupArgs a;
  std::memcpy(a.head, &hd, sizeof(a.head));
  for (int k = 0; k < TK_COUNT; k++)
    for (int o = 0; o < kMaxOct; o++) a.tiles[k][o] = hd.tile_pre[k][o][1];
  for (int m = 0; m < 2; m++) a.base_tiles[m] = hd.base_pre[m][1];
  a.bmc_n = hd.bmc_pre[1];
  a.cc_n = hd.cc_pre[1];
  a.img = hd.img[0];
  for (int o = 0; o < kMaxOct; o++) a.oct[o] = o < hd.img[0].n_oct ? hd.oct[o] : OctDev{};
  // launch_plain reports this launch's own status; an error that an earlier,
  // unrelated call left in the runtime is not taken for ours.
  cudaError_t e = launch_plain(k_noalloc_setup, 1, 32, 0, s, d_desc, a);
  if (e == cudaSuccess) e = eng.enqueue_noalloc(d_desc, s, M, base_modes(hd));
  return e == cudaSuccess ? SIFT_OK : SIFT_E_CUDA;
}

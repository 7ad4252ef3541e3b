// Gaussian scale space (§3.2, "GPU Pipeline Stages"): separable blurs with
// 4-sigma truncation, the 2x magnified first octave, and octave decimation.
//
// One kernel launch computes one pyramid level for every image of the batch:
// a persistent grid walks a flattened queue of 128 x TH output tiles. A tile
// stages its (TH + 2R) x 160 input window in shared memory (float4 loads on
// interior tiles, reflect-101 indexing on border tiles), runs the row pass
// into a second shared buffer (each lane computes 4 adjacent outputs from
// float4 reads), then the column pass (each lane computes a 4-wide column
// strip of TH/8 rows, register-blocked). Every output pixel is the same
// fixed-order FMA chain over its taps whatever the tile shape, so results do
// not depend on tiling or on which other images share the launch.
#include "sift_dev.cuh"

namespace sift {

namespace {

constexpr int kThreads = 256;
constexpr int kSinW = kBlurTW + 2 * kBlurHalo;  // 160 staged columns

template <int TH> struct KindOf;
template <> struct KindOf<16> { static constexpr int v = TK_BLUR16; };
template <> struct KindOf<32> { static constexpr int v = TK_BLUR32; };
template <> struct KindOf<64> { static constexpr int v = TK_BLUR64; };

// Stage rows [y0 - R, y0 + TH + R) x columns [x0 - 16, x0 + 144) of a plain
// image (pyramid level or input) into s_in, reflect-101 at the borders.
__device__ __forceinline__ void stage_plain(const float *__restrict__ src, int pitch, int H, int W,
                                            bool vec_ok, int x0, int y0, int R, int rows,
                                            float *s_in) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int xb = x0 - kBlurHalo;
  const bool xin = vec_ok && xb >= 0 && xb + kSinW <= W;
  for (int r = warp; r < rows; r += kThreads / 32) {
    const int gy = refl101(y0 - R + r, H);
    const float *row = src + (long long)gy * pitch;
    float *dst = s_in + r * kSinW;
    if (xin) {
      const float4 *r4 = reinterpret_cast<const float4 *>(row + xb);
      float4 *d4 = reinterpret_cast<float4 *>(dst);
      d4[lane] = __ldg(r4 + lane);
      if (lane < kSinW / 4 - 32) d4[32 + lane] = __ldg(r4 + 32 + lane);
    } else {
      for (int c = lane; c < kSinW; c += 32) dst[c] = __ldg(row + refl101(xb + c, W));
    }
  }
}

// Same window, sampled from the 2x bilinear magnification of the input:
// u[2k] = I[k], u[2k+1] = (I[k] + I[k+1]) / 2 (last sample clamped), rows of
// the magnified image formed after its columns.
__device__ __forceinline__ void stage_upsampled(const float *__restrict__ src, int spitch, int h,
                                                int w, int x0, int y0, int R, int rows,
                                                float *s_in) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int H = 2 * h, W = 2 * w;
  const int xb = x0 - kBlurHalo;
  for (int r = warp; r < rows; r += kThreads / 32) {
    const int gy = refl101(y0 - R + r, H);
    const int iy = gy >> 1, fy = gy & 1;
    const int iy1 = min(iy + 1, h - 1);
    const float *ra = src + (long long)iy * spitch;
    const float *rb = src + (long long)iy1 * spitch;
    float *dst = s_in + r * kSinW;
    for (int c = lane; c < kSinW; c += 32) {
      const int gx = refl101(xb + c, W);
      const int ix = gx >> 1, fx = gx & 1;
      const int ix1 = min(ix + 1, w - 1);
      const float a = __ldg(ra + ix);
      float v;
      if (!fy) {
        v = fx ? 0.5f * (a + __ldg(ra + ix1)) : a;
      } else {
        const float c0 = __ldg(rb + ix);
        v = fx ? 0.5f * (0.5f * (a + __ldg(ra + ix1)) + 0.5f * (c0 + __ldg(rb + ix1)))
               : 0.5f * (a + c0);
      }
      dst[c] = v;
    }
  }
}

// Row pass: s_h[r][k] = sum_j w[j] * s_in[r][16 + k - R + j], j = 0..2R in order.
template <int R, int TH>
__device__ __forceinline__ void row_pass(const float *s_in, float *s_h, const BlurTaps &tp) {
  constexpr int ROWS = TH + 2 * R;
  constexpr int OFF = (kBlurHalo - R) & 3;
  constexpr int C0 = (kBlurHalo - R) - OFF;
  constexpr int NV = (OFF + 4 + 2 * R + 3) / 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < ROWS; r += kThreads / 32) {
    const float4 *s4 = reinterpret_cast<const float4 *>(s_in + r * kSinW + C0 + 4 * lane);
    float v[NV * 4];
#pragma unroll
    for (int q = 0; q < NV; q++) {
      const float4 f = s4[q];
      v[4 * q + 0] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
    }
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      float acc = tp.w[0] * v[OFF + k];
#pragma unroll
      for (int j = 1; j <= 2 * R; j++) acc = fmaf(tp.w[j], v[OFF + k + j], acc);
      o[k] = acc;
    }
    reinterpret_cast<float4 *>(s_h + r * kBlurTW)[lane] = make_float4(o[0], o[1], o[2], o[3]);
  }
}

// Column pass + store: lane owns columns 4*lane..4*lane+3, warp owns TH/8 rows.
template <int R, int TH>
__device__ __forceinline__ void col_pass_store(const float *s_h, float *out, int pitch, int H,
                                               int x0, int y0, const BlurTaps &tp) {
  constexpr int V = TH / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int v0 = warp * V;
  float acc[V][4];
#pragma unroll
  for (int i = 0; i < V + 2 * R; i++) {
    const float4 f = reinterpret_cast<const float4 *>(s_h + (v0 + i) * kBlurTW)[lane];
#pragma unroll
    for (int v = 0; v < V; v++) {
      const int j = i - v;
      if (j == 0) {
        acc[v][0] = tp.w[0] * f.x; acc[v][1] = tp.w[0] * f.y;
        acc[v][2] = tp.w[0] * f.z; acc[v][3] = tp.w[0] * f.w;
      } else if (j > 0 && j <= 2 * R) {
        acc[v][0] = fmaf(tp.w[j], f.x, acc[v][0]); acc[v][1] = fmaf(tp.w[j], f.y, acc[v][1]);
        acc[v][2] = fmaf(tp.w[j], f.z, acc[v][2]); acc[v][3] = fmaf(tp.w[j], f.w, acc[v][3]);
      }
    }
  }
  const int x = x0 + 4 * lane;
  if (x < pitch) {
#pragma unroll
    for (int v = 0; v < V; v++) {
      const int y = y0 + v0 + v;
      if (y < H)
        *reinterpret_cast<float4 *>(out + (long long)y * pitch + x) =
            make_float4(acc[v][0], acc[v][1], acc[v][2], acc[v][3]);
    }
  }
}

// MODE 0: level lvl_out from level lvl_out - 1 of octave `oct`.
// MODE 1: octave 0 level 0 from the input image.  MODE 2: same, magnified 2x.
template <int R, int TH, int MODE>
__global__ void __launch_bounds__(kThreads) k_blur(const Desc *__restrict__ d, int oct, int lvl_out,
                                                   BlurTaps tp) {
  constexpr int ROWS = TH + 2 * R;
  extern __shared__ float4 smem4[];
  float *s_in = reinterpret_cast<float *>(smem4);
  float *s_h = s_in + ROWS * kSinW;
  const int n = d->n_img;
  const int *pre = d->tile_pre[KindOf<TH>::v][oct];
  const int total = pre[n];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int b = find_owner(pre, n, t);
    const ImgDev &im = d->img[b];
    const OctDev od = d->oct[im.oct0 + oct];
    const int tiles_x = (od.W + kBlurTW - 1) / kBlurTW;
    const int lt = t - pre[b];
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int x0 = tx * kBlurTW, y0 = ty * TH;
    float *out = d->pyr + od.lvl + (long long)lvl_out * od.lstride;
    if (MODE == 0) {
      const float *src = d->pyr + od.lvl + (long long)(lvl_out - 1) * od.lstride;
      stage_plain(src, od.pitch, od.H, od.W, true, x0, y0, R, ROWS, s_in);
    } else if (MODE == 1) {
      stage_plain(im.src, im.spitch, od.H, od.W, im.src_vec_ok != 0, x0, y0, R, ROWS, s_in);
    } else {
      stage_upsampled(im.src, im.spitch, im.H, im.W, x0, y0, R, ROWS, s_in);
    }
    __syncthreads();
    row_pass<R, TH>(s_in, s_h, tp);
    __syncthreads();
    col_pass_store<R, TH>(s_h, out, od.pitch, od.H, x0, y0, tp);
    __syncthreads();
  }
}

// Fallback for radii without a specialised kernel (non-default parameters):
// same staging and the same per-output tap order, plain loops.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_blur_generic(const Desc *__restrict__ d, int oct,
                                                           int lvl_out, int R, BlurTaps tp) {
  constexpr int TH = 32;
  const int ROWS = TH + 2 * R;
  extern __shared__ float4 smem4[];
  float *s_in = reinterpret_cast<float *>(smem4);
  float *s_h = s_in + ROWS * kSinW;
  const int n = d->n_img;
  const int *pre = d->tile_pre[TK_BLUR32][oct];
  const int total = pre[n];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int b = find_owner(pre, n, t);
    const ImgDev &im = d->img[b];
    const OctDev od = d->oct[im.oct0 + oct];
    const int tiles_x = (od.W + kBlurTW - 1) / kBlurTW;
    const int lt = t - pre[b];
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int x0 = tx * kBlurTW, y0 = ty * TH;
    float *out = d->pyr + od.lvl + (long long)lvl_out * od.lstride;
    if (MODE == 0) {
      const float *src = d->pyr + od.lvl + (long long)(lvl_out - 1) * od.lstride;
      stage_plain(src, od.pitch, od.H, od.W, true, x0, y0, R, ROWS, s_in);
    } else if (MODE == 1) {
      stage_plain(im.src, im.spitch, od.H, od.W, im.src_vec_ok != 0, x0, y0, R, ROWS, s_in);
    } else {
      stage_upsampled(im.src, im.spitch, im.H, im.W, x0, y0, R, ROWS, s_in);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ROWS * kBlurTW; idx += kThreads) {
      const int r = idx / kBlurTW, k = idx - r * kBlurTW;
      const float *row = s_in + r * kSinW + kBlurHalo + k - R;
      float acc = tp.w[0] * row[0];
      for (int j = 1; j <= 2 * R; j++) acc = fmaf(tp.w[j], row[j], acc);
      s_h[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TH * kBlurTW; idx += kThreads) {
      const int r = idx / kBlurTW, k = idx - r * kBlurTW;
      const int y = y0 + r, x = x0 + k;
      float acc = tp.w[0] * s_h[r * kBlurTW + k];
      for (int j = 1; j <= 2 * R; j++) acc = fmaf(tp.w[j], s_h[(r + j) * kBlurTW + k], acc);
      if (y < od.H && x < od.pitch) out[(long long)y * od.pitch + x] = acc;
    }
    __syncthreads();
  }
}

// Octave o > 0, level 0: every second sample of level S of octave o - 1.
__global__ void __launch_bounds__(kThreads) k_decimate(const Desc *__restrict__ d, int oct) {
  const int n = d->n_img;
  const int *pre = d->tile_pre[TK_BLUR32][oct];
  const int total = pre[n];
  const int S = d->n_scales;
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int b = find_owner(pre, n, t);
    const ImgDev &im = d->img[b];
    const OctDev od = d->oct[im.oct0 + oct];
    const OctDev op = d->oct[im.oct0 + oct - 1];
    const int tiles_x = (od.W + kBlurTW - 1) / kBlurTW;
    const int lt = t - pre[b];
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const float *src = d->pyr + op.lvl + (long long)S * op.lstride;
    float *dst = d->pyr + od.lvl;
    for (int idx = threadIdx.x; idx < kBlurTW * 32; idx += kThreads) {
      const int y = ty * 32 + idx / kBlurTW, x = tx * kBlurTW + (idx % kBlurTW);
      if (y < od.H && x < od.W) dst[(long long)y * od.pitch + x] = src[(long long)(2 * y) * op.pitch + 2 * x];
    }
  }
}

template <int R, int TH> constexpr int smem_bytes() {
  return (TH + 2 * R) * (kSinW + kBlurTW) * (int)sizeof(float);
}

int th_of_kind(int kind) { return kind == TK_BLUR16 ? 16 : kind == TK_BLUR64 ? 64 : 32; }

}  // namespace

int blur_smem_bytes(int R, int th_kind) {
  return (th_of_kind(th_kind) + 2 * R) * (kSinW + kBlurTW) * (int)sizeof(float);
}

#define SIFT_FOR_EACH_R(X) X(5) X(7) X(8) X(10) X(13)

cudaError_t blur_set_attributes() {
  cudaError_t e = cudaSuccess;
#define SET(fn, bytes)                                                                 \
  if (e == cudaSuccess)                                                                \
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
#define SET_R(R)                                             \
  SET((k_blur<R, 16, 0>), (smem_bytes<R, 16>()))             \
  SET((k_blur<R, 32, 0>), (smem_bytes<R, 32>()))             \
  SET((k_blur<R, 64, 0>), (smem_bytes<R, 64>()))             \
  SET((k_blur<R, 32, 1>), (smem_bytes<R, 32>()))             \
  SET((k_blur<R, 32, 2>), (smem_bytes<R, 32>()))
  SIFT_FOR_EACH_R(SET_R)
  SET(k_blur_generic<0>, (smem_bytes<kMaxR, 32>()))
  SET(k_blur_generic<1>, (smem_bytes<kMaxR, 32>()))
  SET(k_blur_generic<2>, (smem_bytes<kMaxR, 32>()))
#undef SET_R
#undef SET
  return e;
}

cudaError_t launch_level_blur(const Desc *d, int oct, int lvl_out, int R, const BlurTaps &t,
                              int th_kind, int grid, cudaStream_t s) {
  const int bytes = blur_smem_bytes(R, th_kind);
#define CASE_R(RR)                                                                       \
  case RR:                                                                               \
    if (th_kind == TK_BLUR16) k_blur<RR, 16, 0><<<grid, kThreads, bytes, s>>>(d, oct, lvl_out, t); \
    else if (th_kind == TK_BLUR64) k_blur<RR, 64, 0><<<grid, kThreads, bytes, s>>>(d, oct, lvl_out, t); \
    else k_blur<RR, 32, 0><<<grid, kThreads, bytes, s>>>(d, oct, lvl_out, t);            \
    break;
  switch (R) {
    SIFT_FOR_EACH_R(CASE_R)
    default:
      k_blur_generic<0><<<grid, kThreads, blur_smem_bytes(R, TK_BLUR32), s>>>(d, oct, lvl_out, R, t);
  }
#undef CASE_R
  return cudaGetLastError();
}

cudaError_t launch_base_blur(const Desc *d, int R, const BlurTaps &t, int th_kind, bool upsample,
                             int grid, cudaStream_t s) {
  (void)th_kind;
  const int bytes = blur_smem_bytes(R, TK_BLUR32);
#define CASE_R(RR)                                                                      \
  case RR:                                                                              \
    if (upsample) k_blur<RR, 32, 2><<<grid, kThreads, bytes, s>>>(d, 0, 0, t);          \
    else k_blur<RR, 32, 1><<<grid, kThreads, bytes, s>>>(d, 0, 0, t);                   \
    break;
  switch (R) {
    SIFT_FOR_EACH_R(CASE_R)
    default:
      if (upsample) k_blur_generic<2><<<grid, kThreads, bytes, s>>>(d, 0, 0, R, t);
      else k_blur_generic<1><<<grid, kThreads, bytes, s>>>(d, 0, 0, R, t);
  }
#undef CASE_R
  return cudaGetLastError();
}

int blur_blocks_per_sm(int R, int th_kind, int mode) {
  int nb = 0;
  const int bytes = mode == 0 ? blur_smem_bytes(R, th_kind) : blur_smem_bytes(R, TK_BLUR32);
  cudaError_t e = cudaErrorInvalidValue;
#define OCC(fn) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, bytes);
#define CASE_R(RR)                                                   \
  case RR:                                                           \
    if (mode == 1) { OCC((k_blur<RR, 32, 1>)) }                      \
    else if (mode == 2) { OCC((k_blur<RR, 32, 2>)) }                 \
    else if (th_kind == TK_BLUR16) { OCC((k_blur<RR, 16, 0>)) }      \
    else if (th_kind == TK_BLUR64) { OCC((k_blur<RR, 64, 0>)) }      \
    else { OCC((k_blur<RR, 32, 0>)) }                                \
    break;
  switch (R) {
    SIFT_FOR_EACH_R(CASE_R)
    default:
      if (mode == 0) { OCC(k_blur_generic<0>) }
      else if (mode == 1) { OCC(k_blur_generic<1>) }
      else { OCC(k_blur_generic<2>) }
  }
#undef CASE_R
#undef OCC
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

cudaError_t launch_decimate(const Desc *d, int oct, int grid, cudaStream_t s) {
  k_decimate<<<grid, kThreads, 0, s>>>(d, oct);
  return cudaGetLastError();
}

}  // namespace sift

// Gaussian scale space (§3.2, "GPU Pipeline Stages"): separable blurs with
// 4-sigma truncation, the 2x magnified first octave (k_base_poly, a polyphase
// filter of the input, below), and octave decimation.
//
// One kernel launch computes one pyramid level for every image of the batch:
// a persistent grid walks a flattened queue of 128 x TH output tiles. A tile
// stages its (TH + 2R) x 160 input window in shared memory with cp.async
// (16-byte copies on interior tiles, reflect-101 element copies on border
// tiles; every copy of the tile is in flight before the one wait), runs the
// column pass (each thread: a 4-column x TH/8-row block, packed two-lane FP32
// FMAs) into a second shared buffer, then the row pass (each lane: 4 adjacent
// outputs from float4 reads) and stores float4 rows.
//
// Every output pixel is the same fixed-order chain of FP32 operations whatever
// the tile: out(y, x) = sum_i w_i * c_i with c_i = sum_j w_j * in(y - R + j,
// x - R + i), each c_i summed over j ascending and the outer sum split into
// two ascending chains of alternate taps whose grouping depends only on the
// parity of x - R (row_pass_store). Results therefore do not depend on tiling
// or on which other images share the launch.
#include <type_traits>

#include "sift_dev.cuh"

namespace sift {

namespace {

constexpr int kThreads = 320;                   // 10 warps
constexpr int kWarps = kThreads / 32;
constexpr int kSinW = kBlurTW + 2 * kBlurHalo;  // 160 staged columns
constexpr int kNG = kSinW / 4;                  // 40 float4 column groups

template <int TH> struct KindOf;
template <> struct KindOf<32> { static constexpr int v = TK_BLUR32; };
template <> struct KindOf<64> { static constexpr int v = TK_BLUR64; };

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async16_u(unsigned dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Issue (without waiting) the copies of rows [y0 - R, y0 + TH + R) x columns
// [x0 - 16, x0 + 144) of a plain image (pyramid level or input) into s_in,
// reflect-101 at the borders.
// 16-byte path (16-byte aligned rows): thread t copies float4 column group
// t % 40 of rows t / 40, t / 40 + 8, ...; a group that crosses or lies past an
// image edge copies its four reflected columns one by one. Element path
// (unaligned input rows): thread t copies column t % 160 of rows t / 160,
// t / 160 + 2, .... Reflection is only computed where the window crosses an
// image edge.
__device__ __forceinline__ void stage_plain_issue(const float *__restrict__ src, int pitch, int H,
                                                  int W, bool vec_ok, int x0, int y0, int R,
                                                  int rows, float *s_in) {
  const int xb = x0 - kBlurHalo;
  const int yb = y0 - R;
  const bool yin = yb >= 0 && yb + rows <= H;
  const int tid = threadIdx.x;
  if (vec_ok) {
    constexpr int RPP = kThreads / kNG;  // rows per pass (8)
    const int g = tid % kNG, r0 = tid / kNG;
    const int c = xb + 4 * g;
    float *dst = s_in + r0 * kSinW + 4 * g;
    if (c >= 0 && c + 4 <= W) {
      const float *col = src + c;
      if (yin) {
        const float *p = col + (long long)(yb + r0) * pitch;
        for (int r = r0; r < rows; r += RPP, p += (long long)RPP * pitch, dst += RPP * kSinW)
          cp_async16(dst, p);
      } else {
        for (int r = r0; r < rows; r += RPP, dst += RPP * kSinW)
          cp_async16(dst, col + (long long)refl101(yb + r, H) * pitch);
      }
    } else {
      const int c0 = refl101(c, W), c1 = refl101(c + 1, W), c2 = refl101(c + 2, W),
                c3 = refl101(c + 3, W);
      for (int r = r0; r < rows; r += RPP, dst += RPP * kSinW) {
        const float *row = src + (long long)(yin ? yb + r : refl101(yb + r, H)) * pitch;
        cp_async4(dst, row + c0);
        cp_async4(dst + 1, row + c1);
        cp_async4(dst + 2, row + c2);
        cp_async4(dst + 3, row + c3);
      }
    }
  } else {
    constexpr int RPP = kThreads / kSinW;  // rows per pass (2)
    const int c = tid % kSinW, r0 = tid / kSinW;
    const float *col = src + refl101(xb + c, W);
    float *dst = s_in + r0 * kSinW + c;
    for (int r = r0; r < rows; r += RPP, dst += RPP * kSinW)
      cp_async4(dst, col + (long long)(yin ? yb + r : refl101(yb + r, H)) * pitch);
  }
}

__device__ __forceinline__ void stage_plain(const float *__restrict__ src, int pitch, int H, int W,
                                            bool vec_ok, int x0, int y0, int R, int rows,
                                            float *s_in) {
  stage_plain_issue(src, pitch, H, W, vec_ok, x0, y0, R, rows, s_in);
  cp_async_wait_all();
}

// Same window, sampled from the 2x bilinear magnification of the input:
// u[2k] = I[k], u[2k+1] = (I[k] + I[k+1]) / 2 (last sample clamped), rows of
// the magnified image formed after its columns.
__device__ __forceinline__ void stage_upsampled(const float *__restrict__ src, int spitch, int h,
                                                int w, int x0, int y0, int R, int rows,
                                                float *s_in) {
  const int H = 2 * h, W = 2 * w;
  const int xb = x0 - kBlurHalo;
  for (int idx = threadIdx.x; idx < rows * kSinW; idx += kThreads) {
    const int r = idx / kSinW, c = idx - r * kSinW;
    const int gy = refl101(y0 - R + r, H);
    const int iy = gy >> 1, fy = gy & 1;
    const int iy1 = min(iy + 1, h - 1);
    const float *ra = src + (long long)iy * spitch;
    const float *rb = src + (long long)iy1 * spitch;
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
    s_in[idx] = v;
  }
}

// Staged columns the row pass reads: float4 groups [RowSpan<R>::G0, G1).
template <int R> struct RowSpan {
  static constexpr int OFF = (kBlurHalo - R) & 3;      // first tap's offset in the first group
  static constexpr int C0 = (kBlurHalo - R) - OFF;     // first column read by lane 0
  static constexpr int NV = (OFF + 4 + 2 * R + 3) / 4; // float4 groups read per lane
  static constexpr int G0 = C0 / 4;
  static constexpr int G1 = G0 + 31 + NV;
};

// How the staged window holds its values (binary16 octaves of the fp16 storage
// mode use 32-row tiles only):
//   SK_F32  FP32 values;
//   SK_H16  binary16 values (a binary16 level, MODE 0);
//   SK_R16  FP32 values still to be rounded to binary16 (the decimated base of
//           the first binary16 octave, MODE 3 from an FP32 octave);
//   SK_P16  32-bit words whose low half is the binary16 value (the decimated
//           base of a later binary16 octave: the word holding sample 2x of a
//           binary16 row, copied whole by a 4-byte cp.async).
enum StageKind { SK_F32 = 0, SK_H16 = 1, SK_R16 = 2, SK_P16 = 3 };

template <int MODE, int ST> __host__ __device__ constexpr int stage_kind() {
  return ST == 0 ? SK_F32 : MODE == 0 ? SK_H16 : ST == 1 ? SK_R16 : SK_P16;
}

// Staged elements idx, idx + 1 (idx even) as FP32; binary16 values widen
// exactly, and SK_R16 rounds to binary16 first (what the level stores).
template <int KIND>
__device__ __forceinline__ float2 staged_pair(const float *s, int idx) {
  if constexpr (KIND == SK_H16) {
    return __half22float2(reinterpret_cast<const __half2 *>(s)[idx >> 1]);
  } else if constexpr (KIND == SK_P16) {
    const uint2 w = reinterpret_cast<const uint2 *>(s)[idx >> 1];
    const unsigned lo = __byte_perm(w.x, w.y, 0x5410);  // the two low halves
    return __half22float2(*reinterpret_cast<const __half2 *>(&lo));
  } else {
    const float2 f = reinterpret_cast<const float2 *>(s)[idx >> 1];
    if constexpr (KIND == SK_R16) return __half22float2(__float22half2_rn(f));
    return f;
  }
}

// Column pass: s_v[v][c] = sum_j w[j] * s_in[v + j][c], j = 0..2R in order,
// for the column groups the row pass reads. Thread item = one float4 column
// group x V = TH/8 rows. KIND: how s_in holds the window (StageKind).
template <int R, int TH, int KIND = SK_F32>
__device__ __forceinline__ void col_pass(const float *s_in, float *s_v, const BlurTaps &tp) {
  static_assert(TH == 32 || KIND == SK_F32, "binary16 windows use 32-row tiles");
  if constexpr (TH == 32) {
    // 32-row tiles: items of 8 rows x one column pair (float2), 4 x 72..80
    // items; 8 rows per item halve the staged reads per output compared with
    // 4-row items, at the same FMA order.
    constexpr int V = 8;
    constexpr int NP = 2 * (RowSpan<R>::G1 - RowSpan<R>::G0);
    constexpr int ITEMS = (TH / V) * NP;
    for (int it = threadIdx.x; it < ITEMS; it += kThreads) {
      const int rb = it / NP, c = 4 * RowSpan<R>::G0 + 2 * (it - rb * NP);
      const int e0 = rb * V * kSinW + c;  // staged element of the item's first tap
      float2 acc[V];
#pragma unroll
      for (int i = 0; i < V + 2 * R; i++) {
        const float2 f = staged_pair<KIND>(s_in, e0 + i * kSinW);
#pragma unroll
        for (int v = 0; v < V; v++) {
          const int j = i - v;
          if (j == 0) acc[v] = __fmul2_rn(tp.wd[0], f);
          else if (j > 0 && j <= 2 * R) acc[v] = __ffma2_rn(tp.wd[j], f, acc[v]);
        }
      }
      float *dst = s_v + rb * V * kSinW + c;
#pragma unroll
      for (int v = 0; v < V; v++) *reinterpret_cast<float2 *>(dst + v * kSinW) = acc[v];
    }
    return;
  }
  constexpr int V = TH / 8;
  constexpr int NG = RowSpan<R>::G1 - RowSpan<R>::G0;
  constexpr int ITEMS = (TH / V) * NG;
  for (int it = threadIdx.x; it < ITEMS; it += kThreads) {
    const int rb = it / NG, g = RowSpan<R>::G0 + it - rb * NG;
    const float *src = s_in + rb * V * kSinW + 4 * g;
    float2 acc[V][2];
#pragma unroll
    for (int i = 0; i < V + 2 * R; i++) {
      const float4 f = *reinterpret_cast<const float4 *>(src + i * kSinW);
      const float2 lo = make_float2(f.x, f.y), hi = make_float2(f.z, f.w);
#pragma unroll
      for (int v = 0; v < V; v++) {
        const int j = i - v;
        if (j == 0) {
          acc[v][0] = __fmul2_rn(tp.wd[0], lo);
          acc[v][1] = __fmul2_rn(tp.wd[0], hi);
        } else if (j > 0 && j <= 2 * R) {
          acc[v][0] = __ffma2_rn(tp.wd[j], lo, acc[v][0]);
          acc[v][1] = __ffma2_rn(tp.wd[j], hi, acc[v][1]);
        }
      }
    }
    float *dst = s_v + rb * V * kSinW + 4 * g;
#pragma unroll
    for (int v = 0; v < V; v++)
      *reinterpret_cast<float4 *>(dst + v * kSinW) =
          make_float4(acc[v][0].x, acc[v][0].y, acc[v][1].x, acc[v][1].y);
  }
}

// Row pass + store: out[y0 + v][x0 + k] from s_v[v][16 + k - R + i], i = 0..2R.
// Lane l of a warp produces outputs x0 + 4l .. x0 + 4l + 3 of one row. The
// taps are taken two at a time by packed FMAs whose operand pairs are aligned
// (even, odd) column pairs of the row, so with s the output's first tap
// column (each lane of a packed FMA is an ordinary FP32 fma):
//   s even: a = (w0 v[s], w1 v[s+1]), a += (w2i, w2i+1)(v[s+2i], v[s+2i+1]) for
//           i = 1..R-1, out = fma(w2R, v[s+2R], a.x) + a.y;
//   s odd:  a = (w1 v[s+1], w2 v[s+2]), a += (w2i+1, w2i+2)(v[s+2i+1], v[s+2i+2])
//           for i = 1..R-1, out = fma(w0, v[s], a.x) + a.y.
// The parity of s is that of the output's column, so the order of operations
// is a fixed function of the pixel, independent of tiling.
// Store four adjacent outputs: FP32, or (DH) rounded to binary16.
template <bool DH>
__device__ __forceinline__ void store4(float *out, long long idx, float a, float b, float c, float e) {
  if (DH) {
    const __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, e);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned *>(&lo);
    u.y = *reinterpret_cast<const unsigned *>(&hi);
    *reinterpret_cast<uint2 *>(reinterpret_cast<__half *>(out) + idx) = u;
  } else {
    *reinterpret_cast<float4 *>(out + idx) = make_float4(a, b, c, e);
  }
}

template <int R, int TH, bool DH = false>
__device__ __forceinline__ void row_pass_store(const float *s_v, float *out, int pitch, int H,
                                               int x0, int y0, const BlurTaps &tp) {
  constexpr int OFF = RowSpan<R>::OFF;
  constexpr int NV = RowSpan<R>::NV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = x0 + 4 * lane;
  const bool xok = x < pitch;
  const float *sp = s_v + warp * kSinW + RowSpan<R>::C0 + 4 * lane;
  long long oi = (long long)(y0 + warp) * pitch + x;
  for (int v = warp; v < TH; v += kWarps, sp += kWarps * kSinW, oi += (long long)kWarps * pitch) {
    const float4 *s4 = reinterpret_cast<const float4 *>(sp);
    float in[NV * 4];
#pragma unroll
    for (int q = 0; q < NV; q++) {
      const float4 f = s4[q];
      in[4 * q + 0] = f.x; in[4 * q + 1] = f.y; in[4 * q + 2] = f.z; in[4 * q + 3] = f.w;
    }
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int s = OFF + k;
      if ((s & 1) == 0) {
        float2 a = __fmul2_rn(tp.wp[0], make_float2(in[s], in[s + 1]));
#pragma unroll
        for (int i = 1; i < R; i++)
          a = __ffma2_rn(tp.wp[i], make_float2(in[s + 2 * i], in[s + 2 * i + 1]), a);
        o[k] = __fadd_rn(fmaf(tp.w[2 * R], in[s + 2 * R], a.x), a.y);
      } else {
        float2 a = __fmul2_rn(tp.wq[0], make_float2(in[s + 1], in[s + 2]));
#pragma unroll
        for (int i = 1; i < R; i++)
          a = __ffma2_rn(tp.wq[i], make_float2(in[s + 2 * i + 1], in[s + 2 * i + 2]), a);
        o[k] = __fadd_rn(fmaf(tp.w[0], in[s], a.x), a.y);
      }
    }
    if (y0 + v < H && xok) store4<DH>(out, oi, o[0], o[1], o[2], o[3]);
  }
}

// The same output from scalar operations, for the generic kernel: row points
// at the output's first tap column s, odd tells the parity of s.
__device__ __forceinline__ float row_tap_sum(const float *row, bool odd, int R, const float *w) {
  float ax, ay;
  if (!odd) {
    ax = __fmul_rn(w[0], row[0]);
    ay = __fmul_rn(w[1], row[1]);
    for (int i = 1; i < R; i++) {
      ax = fmaf(w[2 * i], row[2 * i], ax);
      ay = fmaf(w[2 * i + 1], row[2 * i + 1], ay);
    }
    return __fadd_rn(fmaf(w[2 * R], row[2 * R], ax), ay);
  }
  ax = __fmul_rn(w[1], row[1]);
  ay = __fmul_rn(w[2], row[2]);
  for (int i = 1; i < R; i++) {
    ax = fmaf(w[2 * i + 1], row[2 * i + 1], ax);
    ay = fmaf(w[2 * i + 2], row[2 * i + 2], ay);
  }
  return __fadd_rn(fmaf(w[0], row[0], ax), ay);
}

// MODE 0: level lvl_out from level lvl_out - 1 of octave `oct`.
// MODE 1: octave 0 level 0 from the input image.  MODE 2: same, magnified 2x.
// MODE 3: level 1 of octave `oct` > 0 from its level 0, decimated on the fly
//         from level S of octave oct - 1; level 0 itself is stored on the way.
struct TileGeo {
  const float *src;  // staging source: level lvl_out - 1 (MODE 0), the input (1, 2),
                     // level S of the previous octave (3)
  float *out;        // level lvl_out of the tile's octave
  float *out0;       // level 0 of the tile's octave (MODE 3 stores it)
  int spitch;        // source pitch (elements)
  int pitch, H, W;   // the octave's pitch and size
  int sh, sw;        // input size (MODE 2)
  int vec;           // 16-byte aligned source rows
  int x0, y0;
};

// Geometry of flattened tile t. Image b's octaves sit at fixed slots
// oct[b * kMaxOct + o], so no ImgDev read is needed for pyramid levels.
// Element st of plane p, for planes of 4-byte (half false) or 2-byte elements.
__device__ __forceinline__ float *elem_ptr(float *p, long long st, bool half) {
  return half ? reinterpret_cast<float *>(reinterpret_cast<__half *>(p) + st) : p + st;
}

// ST: storage of the source and the output. 0: FP32 in and out; 1: FP32 source,
// binary16 output (the first level of octave 1 in the fp16 storage mode);
// 2: binary16 in and out (octaves above 1, and every level after the first of
// octave 1).
template <int TH, int MODE, int ST = 0>
__device__ __forceinline__ TileGeo tile_geo(const Desc *__restrict__ d, const int *pre, int oct,
                                            int lvl_out, int t) {
  TileGeo g;
  const int b = find_owner(pre, d->n_img, t);
  const OctDev od = d->oct[b * kMaxOct + oct];
  g.pitch = od.pitch;
  g.H = od.H;
  g.W = od.W;
  float *lv = d->pyr + od.lvl;
  g.out0 = lv;
  g.out = elem_ptr(lv, (long long)lvl_out * od.lstride, ST != 0);
  g.sh = 0;
  g.sw = 0;
  if (MODE == 0) {
    g.src = elem_ptr(lv, (long long)(lvl_out - 1) * od.lstride, ST == 2);
    g.spitch = od.pitch;
    g.vec = 1;
  } else if (MODE == 3) {
    const OctDev op = d->oct[b * kMaxOct + oct - 1];
    g.src = elem_ptr(d->pyr + op.lvl, (long long)d->n_scales * op.lstride, ST == 2);
    g.spitch = op.pitch;
    g.vec = 0;
  } else {
    const ImgDev &im = d->img[b];
    g.src = im.src;
    g.spitch = im.spitch;
    g.sh = im.H;
    g.sw = im.W;
    g.vec = im.src_vec_ok;
  }
  const int tiles_x = (od.W + kBlurTW - 1) / kBlurTW;
  const int lt = t - pre[b];
  const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
  g.x0 = tx * kBlurTW;
  g.y0 = ty * TH;
  return g;
}

// Issue the copies of the window of octave o > 0's level 0 without storing
// that level first: sample (y, x) of level 0 is sample (2y, 2x) of level S of
// octave o - 1, so the window is gathered from there (reflect-101 applied in
// octave o's own domain), element by element.
// DEC 2: src holds FP32 samples, spitch in floats. DEC 1: src is a binary16
// plane seen as 32-bit words (spitch in halves): word gy * spitch + gx holds
// halves 2 (gy * spitch + gx) and the next, the first of which is sample
// (2 gy, 2 gx) (SK_P16).
template <int DEC = 2>
__device__ __forceinline__ void stage_decim_issue(const float *__restrict__ src, int spitch, int H,
                                                  int W, int x0, int y0, int R, int rows,
                                                  float *s_in) {
  const int xb = x0 - kBlurHalo, yb = y0 - R;
  const bool yin = yb >= 0 && yb + rows <= H;
  constexpr int RPP = kThreads / kSinW;  // rows per pass (2)
  const int c = threadIdx.x % kSinW, r0 = threadIdx.x / kSinW;
  const float *col = src + DEC * refl101(xb + c, W);
  float *dst = s_in + r0 * kSinW + c;
  for (int r = r0; r < rows; r += RPP, dst += RPP * kSinW)
    cp_async4(dst, col + (long long)(DEC * (yin ? yb + r : refl101(yb + r, H))) * spitch);
}

// Store the tile's own rows / columns of the staged (decimated) level 0:
// FP32, or (DH) rounded to binary16 (exact for SK_P16 words, whose low
// halves are binary16 values already).
template <int R, int TH, bool DH = false, int KIND = SK_F32>
__device__ __forceinline__ void store_level0(const float *s_in, float *out0, int pitch, int H,
                                             int x0, int y0) {
  for (int q = threadIdx.x; q < TH * (kBlurTW / 4); q += kThreads) {
    const int v = q / (kBlurTW / 4), g = q - v * (kBlurTW / 4);
    const int y = y0 + v, x = x0 + 4 * g;
    if (y < H && x < pitch) {
      const int e = (R + v) * kSinW + kBlurHalo + 4 * g;
      const float2 a = staged_pair<KIND == SK_P16 ? SK_P16 : SK_F32>(s_in, e);
      const float2 b = staged_pair<KIND == SK_P16 ? SK_P16 : SK_F32>(s_in, e + 2);
      store4<DH>(out0, (long long)y * pitch + x, a.x, a.y, b.x, b.y);
    }
  }
}

// Staging by plain loads for the binary16 modes of the generic-radius kernel
// (k_blur uses cp.async for them): a binary16 source (ST 2) is widened to FP32
// on the way into shared memory, and the decimated base of a binary16 octave
// (MODE 3, ST 1 or 2) is rounded to binary16 first, so that the level-1 blur
// reads the values level 0 stores.
// Rows [y0 - R, y0 + rows - R) x columns [x0 - 16, x0 + 144), reflect-101 in
// the octave's own domain; MODE 3 samples (2y, 2x) of the previous octave.
template <int MODE, int ST>
__device__ __forceinline__ void stage_sync(const TileGeo &g, int R, int rows, float *s_in) {
  const int xb = g.x0 - kBlurHalo, yb = g.y0 - R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const __half *src16 = reinterpret_cast<const __half *>(g.src);
  for (int r = warp; r < rows; r += kWarps) {
    const int gy = refl101(yb + r, g.H);
    const long long row = (long long)(MODE == 3 ? 2 * gy : gy) * g.spitch;
    for (int c = lane; c < kSinW; c += 32) {
      const int gx = refl101(xb + c, g.W);
      const long long idx = row + (MODE == 3 ? 2 * gx : gx);
      float v = ST == 2 ? __half2float(src16[idx]) : g.src[idx];
      if (MODE == 3) v = __half2float(__float2half_rn(v));
      s_in[r * kSinW + c] = v;
    }
  }
}

// Interior tile of a 16-byte aligned plane (no staged row or column outside
// the image): a fixed, fully unrolled copy schedule, thread t copying float4
// group t % 40 of rows t / 40 + 8 i, so the copies cost almost nothing but
// the copy instructions themselves.
template <int ROWS>
__device__ __forceinline__ void stage_interior(const float *__restrict__ src, int pitch, int xb,
                                               int yb, float *s_in) {
  constexpr int RPP = kThreads / kNG;  // 8
  constexpr int NIT = (ROWS + RPP - 1) / RPP;
  const int tid = threadIdx.x;
  const int g = tid % kNG, r0 = tid / kNG;
  const unsigned d0 = smem_u32(s_in + r0 * kSinW + 4 * g);
  const float *p = src + (long long)(yb + r0) * pitch + (xb + 4 * g);
  const long long step = (long long)RPP * pitch;
#pragma unroll
  for (int i = 0; i < NIT; i++)
    if (i + 1 < NIT || r0 + i * RPP < ROWS) cp_async16_u(d0 + i * RPP * kSinW * 4, p + i * step);
}

// The window of a binary16 level (MODE 0, ST 2), kept as binary16 in shared
// memory (rows of kSinW halves) and widened by the column pass. Every group of
// 8 columns that lies inside the image is one 16-byte cp.async copy (rows
// start on 64-byte boundaries and xb is a multiple of 16; a row outside the
// image is its reflect-101 row); a group that crosses or lies past a left or
// right edge is copied element by element through registers with reflect-101
// (cp.async has no 2-byte copy).
__device__ __forceinline__ void stage_half_issue(const TileGeo &g, int R, int rows, __half *s_in) {
  const __half *src = reinterpret_cast<const __half *>(g.src);
  const int xb = g.x0 - kBlurHalo, yb = g.y0 - R;
  constexpr int NG8 = kSinW / 8;  // 20 groups of 8 halves per row
  const bool yin = yb >= 0 && yb + rows <= g.H;
  for (int i = threadIdx.x; i < rows * NG8; i += kThreads) {
    const int r = i / NG8, c8 = i - r * NG8;
    const int gx = xb + 8 * c8;
    const __half *row = src + (long long)(yin ? yb + r : refl101(yb + r, g.H)) * g.spitch;
    __half *dst = s_in + r * kSinW + 8 * c8;
    if (gx >= 0 && gx + 8 <= g.W) {
      cp_async16(dst, row + gx);
    } else {
#pragma unroll
      for (int k = 0; k < 8; k++) dst[k] = row[refl101(gx + k, g.W)];
    }
  }
}

template <int R, int TH, int MODE, int ST = 0>
__device__ __forceinline__ void issue_stage(const TileGeo &g, float *dst) {
  constexpr int ROWS = TH + 2 * R;
  if constexpr (MODE == 0 && ST == 2) {
    stage_half_issue(g, R, ROWS, reinterpret_cast<__half *>(dst));
  } else if constexpr (MODE == 3) {  // FP32 samples (ST 0, 1) or binary16 words (ST 2)
    stage_decim_issue<ST == 2 ? 1 : 2>(g.src, g.spitch, g.H, g.W, g.x0, g.y0, R, ROWS, dst);
  } else {
    static_assert(ST == 0, "binary16 output is MODE 3 (ST 1) or MODE 0 / 3 (ST 2)");
    const int xb = g.x0 - kBlurHalo, yb = g.y0 - R;
    if (g.vec && xb >= 0 && xb + kSinW <= g.W && yb >= 0 && yb + ROWS <= g.H)
      stage_interior<ROWS>(g.src, g.spitch, xb, yb, dst);
    else
      stage_plain_issue(g.src, g.spitch, g.H, g.W, g.vec != 0, g.x0, g.y0, R, ROWS, dst);
  }
}

// The block's tiles are t0, t0 + grid, t0 + 2 grid, .... Their geometry is
// resolved 32 tiles at a time, one tile per lane of warp 0, into a ring of two
// 32-entry chunks in shared memory: the lanes' owner searches and descriptor
// loads overlap, and chunk m + 1 is filled half-way through chunk m, so no
// tile waits on a dependent chain of global loads.
// One staging buffer per block, but its copies run ahead: once the column pass
// of tile i has read the staged window, the block issues tile i + 1's copies
// into it and they land while the row pass of tile i runs (MODE 2 stages
// synchronously). With three or four blocks per SM this measured faster than
// a second buffer with fewer blocks.
constexpr int kGeoChunk = 32;
template <int R, int TH, int MODE, int ST = 0>
__global__ void __launch_bounds__(kThreads, TH == 32 ? (MODE == 0 ? 4 : 3) : 1)
    k_blur(const Desc *__restrict__ d, int oct, int lvl_out, BlurTaps tp) {
  constexpr int ROWS = TH + 2 * R;
  static_assert(MODE != 2, "the magnified base is k_base_poly");
  extern __shared__ float4 smem4[];
  __shared__ TileGeo geo[2 * kGeoChunk];
  // A binary16 level (MODE 0, ST 2) is staged as binary16: half the bytes.
  constexpr int KIND = stage_kind<MODE, ST>();
  constexpr bool H16 = KIND == SK_H16;
  float *s_in = reinterpret_cast<float *>(smem4);
  float *s_v = s_in + (H16 ? ROWS * kSinW / 2 : ROWS * kSinW);
  // The base blur of images kept at their size (MODE 1) takes the queue of
  // those images only.
  const int *pre = MODE == 1 ? d->base_pre[0] : d->tile_pre[KindOf<TH>::v][oct];
  const int total = pre[d->n_img];
  const int t0 = blockIdx.x, G = gridDim.x;
  if (t0 >= total) return;
  const int n_mine = (total - t0 + G - 1) / G;  // tiles of this block
  auto fill_chunk = [&](int m) {                // tiles 32 m .. 32 m + 31, by warp 0
    const int k = m * kGeoChunk + (int)threadIdx.x;
    if (k < n_mine) geo[k & (2 * kGeoChunk - 1)] = tile_geo<TH, MODE, ST>(d, pre, oct, lvl_out, t0 + k * G);
  };
  if (threadIdx.x < 32) fill_chunk(0);
  __syncthreads();
  pdl_wait();  // the source level is the previous kernel's output
  issue_stage<R, TH, MODE, ST>(geo[0], s_in);
  for (int k = 0; k < n_mine; k++) {
    if (k + 1 == n_mine) pdl_trigger();  // successors launch during this block's last tile
    const TileGeo &g = geo[k & (2 * kGeoChunk - 1)];
    const TileGeo &gn = geo[(k + 1) & (2 * kGeoChunk - 1)];
    cp_async_wait_all();
    __syncthreads();
    if (MODE == 3) store_level0<R, TH, ST != 0, KIND>(s_in, g.out0, g.pitch, g.H, g.x0, g.y0);
    col_pass<R, TH, KIND>(s_in, s_v, tp);
    __syncthreads();
    if (k + 1 < n_mine) issue_stage<R, TH, MODE, ST>(gn, s_in);
    row_pass_store<R, TH, ST != 0>(s_v, g.out, g.pitch, g.H, g.x0, g.y0, tp);
    if (threadIdx.x < 32 && (k & (kGeoChunk - 1)) == kGeoChunk / 2)
      fill_chunk(k / kGeoChunk + 1);
    // No barrier here: the barrier after the next copy-wait orders every
    // warp's row pass (reads of s_v) before the next column pass writes s_v,
    // and the column pass (reads of s_in) before s_in is restaged.
  }
}

// Fallback for radii without a specialised kernel (non-default parameters):
// same staging and the same per-output order of operations, plain loops. ST as
// for k_blur (MODE 0 and 3 only).
template <int MODE, int ST = 0>
__global__ void __launch_bounds__(kThreads) k_blur_generic(const Desc *__restrict__ d, int oct,
                                                           int lvl_out, int R, BlurTaps tp) {
  pdl_trigger();
  pdl_wait();
  constexpr int TH = 32;
  const int ROWS = TH + 2 * R;
  extern __shared__ float4 smem4[];
  float *s_in = reinterpret_cast<float *>(smem4);
  float *s_v = s_in + ROWS * kSinW;
  const int n = d->n_img;
  const int *pre = (MODE == 1 || MODE == 2) ? d->base_pre[MODE - 1] : d->tile_pre[TK_BLUR32][oct];
  const int total = pre[n];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int b = find_owner(pre, n, t);
    const ImgDev &im = d->img[b];
    const OctDev od = d->oct[im.oct0 + oct];
    const int tiles_x = (od.W + kBlurTW - 1) / kBlurTW;
    const int lt = t - pre[b];
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int x0 = tx * kBlurTW, y0 = ty * TH;
    float *out = elem_ptr(d->pyr + od.lvl, (long long)lvl_out * od.lstride, ST != 0);
    if (ST != 0) {
      TileGeo g{};
      if (MODE == 3) {
        const OctDev op = d->oct[im.oct0 + oct - 1];
        g.src = elem_ptr(d->pyr + op.lvl, (long long)d->n_scales * op.lstride, ST == 2);
        g.spitch = op.pitch;
      } else {
        g.src = elem_ptr(d->pyr + od.lvl, (long long)(lvl_out - 1) * od.lstride, ST == 2);
        g.spitch = od.pitch;
      }
      g.H = od.H;
      g.W = od.W;
      g.x0 = x0;
      g.y0 = y0;
      stage_sync<MODE, ST>(g, R, ROWS, s_in);
    } else if (MODE == 0) {
      const float *src = d->pyr + od.lvl + (long long)(lvl_out - 1) * od.lstride;
      stage_plain(src, od.pitch, od.H, od.W, true, x0, y0, R, ROWS, s_in);
    } else if (MODE == 1) {
      stage_plain(im.src, im.spitch, od.H, od.W, im.src_vec_ok != 0, x0, y0, R, ROWS, s_in);
    } else if (MODE == 3) {
      const OctDev op = d->oct[im.oct0 + oct - 1];
      stage_decim_issue(d->pyr + op.lvl + (long long)d->n_scales * op.lstride, op.pitch, od.H, od.W,
                        x0, y0, R, ROWS, s_in);
      cp_async_wait_all();
    } else {
      stage_upsampled(im.src, im.spitch, im.H, im.W, x0, y0, R, ROWS, s_in);
    }
    __syncthreads();
    if (MODE == 3) {
      for (int q = threadIdx.x; q < TH * kBlurTW; q += kThreads) {
        const int v = q / kBlurTW, k = q - v * kBlurTW;
        if (y0 + v < od.H && x0 + k < od.pitch) {
          const long long i = (long long)(y0 + v) * od.pitch + x0 + k;
          const float val = s_in[(R + v) * kSinW + kBlurHalo + k];
          if (ST != 0) reinterpret_cast<__half *>(d->pyr + od.lvl)[i] = __float2half_rn(val);
          else d->pyr[od.lvl + i] = val;
        }
      }
    }
    for (int idx = threadIdx.x; idx < TH * kSinW; idx += kThreads) {
      const int v = idx / kSinW, c = idx - v * kSinW;
      float acc = tp.w[0] * s_in[v * kSinW + c];
      for (int j = 1; j <= 2 * R; j++) acc = fmaf(tp.w[j], s_in[(v + j) * kSinW + c], acc);
      s_v[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TH * kBlurTW; idx += kThreads) {
      const int v = idx / kBlurTW, k = idx - v * kBlurTW;
      const int y = y0 + v, x = x0 + k;
      const int sc = kBlurHalo + k - R;  // first tap column; its parity is that of x - R
      const float acc = row_tap_sum(s_v + v * kSinW + sc, (sc & 1) != 0, R, tp.w);
      if (y < od.H && x < od.pitch) {
        if (ST != 0) reinterpret_cast<__half *>(out)[(long long)y * od.pitch + x] = __float2half_rn(acc);
        else out[(long long)y * od.pitch + x] = acc;
      }
    }
    __syncthreads();
  }
}

// Shared memory: the staging buffer (binary16 for a binary16 level, ST 2 with
// MODE 0) plus the column-pass output.
template <int R, int TH, int MODE, int ST = 0> constexpr int smem_bytes() {
  return (TH + 2 * R) * kSinW * (MODE == 0 && ST == 2 ? 2 : 4) + TH * kSinW * (int)sizeof(float);
}

int th_of_kind(int kind) { return kind == TK_BLUR64 ? 64 : 32; }



int generic_smem_bytes(int R) { return (2 * 32 + 2 * R) * kSinW * (int)sizeof(float); }

// ------------------------------------------------- magnified base, polyphase
//
// The base level of a magnified first octave is G = g * U(I): U the 2x bilinear
// magnification (u[2k] = I[k], u[2k+1] = (I[k] + I[k+1]) / 2, last sample
// clamped), g the base Gaussian with reflect-101 on the magnified grid. Both
// are linear, so output sample 2k + p (p = 0, 1) of a row is a 2Q + 1 tap
// filter c_p of the input around k, with c_p[q] = sum_t g[t] * (weight of
// I[k + q] in u[2k + p + t]), Q = (R + 2) / 2. The reflection and the clamp
// are exact on an extended input I_e[i] = I[refl101(2i, 2n) / 2]
// (reflect-101 on the left, half-sample symmetric on the right, which is what
// the magnified grid's reflection maps back to). A tile of 128 x 32 outputs
// stages (64 + 2Q) x (16 + 2Q) input samples, filters its rows into 128
// columns at input-row resolution, then its columns into 32 rows: about 12
// FMAs per output against 22 for the two passes on the magnified grid, and no
// magnified window. Each output is the same fixed chain (sum over q
// ascending, rows then columns) whatever the tile.
constexpr int kPolyThreads = 256;
constexpr int kPolyMaxQ = kMaxR / 2 + 1;

struct PolyTaps {
  float c[2][2 * kPolyMaxQ + 1];
};

template <int Q>
__global__ void __launch_bounds__(kPolyThreads) k_base_poly(const Desc *__restrict__ d, PolyTaps pt) {
  constexpr int NR = 16 + 2 * Q, NC = 64 + 2 * Q, NT = 2 * Q + 1;
  __shared__ float sI[NR * NC];
  __shared__ __align__(16) float sH[NR * kBlurTW];
  const int *pre = d->base_pre[1];
  const int total = pre[d->n_img];
  const int G = gridDim.x;
  for (int t = blockIdx.x; t < total; t += G) {
    if (t + G >= total) pdl_trigger();  // successors launch during this block's last tile
    const TileGeo g = tile_geo<32, 2>(d, pre, 0, 0, t);
    const int kx0 = g.x0 >> 1, ky0 = g.y0 >> 1;
    const int iyb = ky0 - Q, ixb = kx0 - Q;
    if (iyb >= 0 && iyb + NR <= g.sh && ixb >= 0 && ixb + NC <= g.sw) {
      // Interior: the window needs no reflection; warp w copies rows w, w + 8, ...
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int r = warp; r < NR; r += kPolyThreads / 32) {
        const float *srow = g.src + (long long)(iyb + r) * g.spitch + ixb;
        for (int c = lane; c < NC; c += 32) cp_async4(sI + r * NC + c, srow + c);
      }
    } else {
      for (int idx = threadIdx.x; idx < NR * NC; idx += kPolyThreads) {
        const int r = idx / NC, c = idx - r * NC;
        const int iy = refl101(2 * (iyb + r), g.H) >> 1;
        const int ix = refl101(2 * (ixb + c), g.W) >> 1;
        cp_async4(sI + idx, g.src + (long long)iy * g.spitch + ix);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    // Rows: outputs 2j and 2j + 1 of input row r share the taps sI[r][j .. j + 2Q].
    for (int idx = threadIdx.x; idx < NR * (kBlurTW / 2); idx += kPolyThreads) {
      const int r = idx / (kBlurTW / 2), j = idx - r * (kBlurTW / 2);
      const float *row = sI + r * NC + j;
      float a = 0.f, b = 0.f;
#pragma unroll
      for (int q = 0; q < NT; q++) {
        const float v = row[q];
        a = fmaf(pt.c[0][q], v, a);
        b = fmaf(pt.c[1][q], v, b);
      }
      *reinterpret_cast<float2 *>(sH + r * kBlurTW + 2 * j) = make_float2(a, b);
    }
    __syncthreads();
    // Columns: output rows 2j and 2j + 1 of a 4-column group share the taps
    // sH[j .. j + 2Q][4 g4 .. 4 g4 + 3].
    for (int idx = threadIdx.x; idx < 16 * (kBlurTW / 4); idx += kPolyThreads) {
      const int j = idx / (kBlurTW / 4), g4 = idx - j * (kBlurTW / 4);
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
#pragma unroll
      for (int q = 0; q < NT; q++) {
        const float4 v = *reinterpret_cast<const float4 *>(sH + (j + q) * kBlurTW + 4 * g4);
        const float c0 = pt.c[0][q], c1 = pt.c[1][q];
        a.x = fmaf(c0, v.x, a.x);
        a.y = fmaf(c0, v.y, a.y);
        a.z = fmaf(c0, v.z, a.z);
        a.w = fmaf(c0, v.w, a.w);
        b.x = fmaf(c1, v.x, b.x);
        b.y = fmaf(c1, v.y, b.y);
        b.z = fmaf(c1, v.z, b.z);
        b.w = fmaf(c1, v.w, b.w);
      }
      const int X = g.x0 + 4 * g4, Y = g.y0 + 2 * j;
#pragma unroll
      for (int p = 0; p < 2; p++) {
        if (Y + p >= g.H) break;
        const float4 v = p ? b : a;
        float *o = g.out + (long long)(Y + p) * g.pitch + X;
        if (X + 3 < g.W) {
          *reinterpret_cast<float4 *>(o) = v;
        } else {
          if (X < g.W) o[0] = v.x;
          if (X + 1 < g.W) o[1] = v.y;
          if (X + 2 < g.W) o[2] = v.z;
        }
      }
    }
    __syncthreads();  // the next tile reuses sI and sH
  }
}

PolyTaps make_poly_taps(const BlurTaps &t, int R) {
  const int Q = (R + 2) / 2;
  PolyTaps p{};
  for (int ph = 0; ph < 2; ph++)
    for (int q = -Q; q <= Q; q++) {
      double c = 0.0;
      for (int tt = -R; tt <= R; tt++) {
        const int n = ph + tt;  // magnified offset from 2k
        double w = 0.0;
        if ((n & 1) == 0) w = (n / 2 == q) ? 1.0 : 0.0;
        else w = ((n - 1) / 2 == q || (n + 1) / 2 == q) ? 0.5 : 0.0;
        c += (double)t.w[tt + R] * w;
      }
      p.c[ph][q + Q] = (float)c;
    }
  return p;
}

}  // namespace

int blur_smem_bytes(int R, int th_kind) {
  const int th = th_of_kind(th_kind);
  return ((th + 2 * R) + th) * kSinW * (int)sizeof(float);
}

#define SIFT_FOR_EACH_R(X) X(5) X(7) X(8) X(10) X(13)

cudaError_t blur_set_attributes() {
  cudaError_t e = cudaSuccess;
#define SET(fn, bytes)                                                                 \
  if (e == cudaSuccess)                                                                \
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
#define SET_R(R)                                             \
  SET((k_blur<R, 32, 0>), (smem_bytes<R, 32, 0>()))          \
  SET((k_blur<R, 64, 0>), (smem_bytes<R, 64, 0>()))          \
  SET((k_blur<R, 32, 3>), (smem_bytes<R, 32, 3>()))          \
  SET((k_blur<R, 64, 3>), (smem_bytes<R, 64, 3>()))          \
  SET((k_blur<R, 32, 1>), (smem_bytes<R, 32, 1>()))          \
  SET((k_blur<R, 32, 0, 2>), (smem_bytes<R, 32, 0, 2>()))    \
  SET((k_blur<R, 32, 3, 1>), (smem_bytes<R, 32, 3>()))       \
  SET((k_blur<R, 32, 3, 2>), (smem_bytes<R, 32, 3>()))
  SIFT_FOR_EACH_R(SET_R)
  SET(k_blur_generic<0>, generic_smem_bytes(kMaxR))
  SET(k_blur_generic<3>, generic_smem_bytes(kMaxR))
  SET((k_blur_generic<0, 2>), generic_smem_bytes(kMaxR))
  SET((k_blur_generic<3, 1>), generic_smem_bytes(kMaxR))
  SET((k_blur_generic<3, 2>), generic_smem_bytes(kMaxR))
  SET(k_blur_generic<1>, generic_smem_bytes(kMaxR))
  SET(k_blur_generic<2>, generic_smem_bytes(kMaxR))
#undef SET_R
#undef SET
  return e;
}

cudaError_t launch_level_blur(const Desc *d, int oct, int lvl_out, int R, const BlurTaps &t,
                              int th_kind, int grid, cudaStream_t s, bool from_prev_octave,
                              bool pdl, int storage) {
  const bool m3 = from_prev_octave;
  if (storage != 0 && (th_kind == TK_BLUR64 || storage > 2 || (storage == 1 && !m3)))
    return cudaErrorInvalidValue;  // binary16 octaves use 32-row tiles
  // A programmatic dependent of the previous kernel on s, or (pdl false) a plain
  // launch that waits for everything before it (a branch after an event wait).
  auto go = [&](auto kern, size_t smem, auto... args) -> cudaError_t {
    if (pdl) return launch_pdl(kern, grid, kThreads, smem, s, d, oct, lvl_out, args...);
    return launch_plain(kern, grid, kThreads, smem, s, d, oct, lvl_out, args...);
  };
#define CASE_R(RR)                                                                        \
  case RR:                                                                                \
    if (storage == 1) return go(k_blur<RR, 32, 3, 1>, smem_bytes<RR, 32, 3>(), t);          \
    if (storage == 2)                                                                     \
      return m3 ? go(k_blur<RR, 32, 3, 2>, smem_bytes<RR, 32, 3>(), t)                      \
                : go(k_blur<RR, 32, 0, 2>, smem_bytes<RR, 32, 0, 2>(), t);                  \
    if (th_kind == TK_BLUR64)                                                             \
      return m3 ? go(k_blur<RR, 64, 3>, smem_bytes<RR, 64, 3>(), t)                         \
                : go(k_blur<RR, 64, 0>, smem_bytes<RR, 64, 0>(), t);                        \
    return m3 ? go(k_blur<RR, 32, 3>, smem_bytes<RR, 32, 3>(), t)                           \
              : go(k_blur<RR, 32, 0>, smem_bytes<RR, 32, 0>(), t);
  switch (R) {
    SIFT_FOR_EACH_R(CASE_R)
    default:
      if (storage == 1) return go(k_blur_generic<3, 1>, generic_smem_bytes(R), R, t);
      if (storage == 2)
        return m3 ? go(k_blur_generic<3, 2>, generic_smem_bytes(R), R, t)
                  : go(k_blur_generic<0, 2>, generic_smem_bytes(R), R, t);
      return m3 ? go(k_blur_generic<3>, generic_smem_bytes(R), R, t)
                : go(k_blur_generic<0>, generic_smem_bytes(R), R, t);
  }
#undef CASE_R
}

namespace {
// One pyramid level copied out as a dense H x W FP32 plane (binary16 levels
// widened), for the pyramid export.
__global__ void k_export_level(const float *__restrict__ src, int half, int pitch, int H, int W,
                               float *__restrict__ dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W || y >= H) return;
  const long long i = (long long)y * pitch + x;
  dst[(long long)y * W + x] =
      half ? __half2float(reinterpret_cast<const __half *>(src)[i]) : src[i];
}
}  // namespace

cudaError_t launch_export_level(const float *src, bool half, int pitch, int H, int W, float *dst,
                                cudaStream_t s) {
  return launch_plain(k_export_level, dim3((W + 127) / 128, H), 128, 0, s, src, half ? 1 : 0,
                      pitch, H, W, dst);
}

cudaError_t launch_base_blur(const Desc *d, int R, const BlurTaps &t, int th_kind, bool upsample,
                             int grid, cudaStream_t s) {
  (void)th_kind;
#define CASE_R(RR)                                                                             \
  case RR:                                                                                     \
    if (upsample)                                                                              \
      return launch_plain(k_base_poly<(RR + 2) / 2>, grid, kPolyThreads, 0, s, d,              \
                          make_poly_taps(t, RR));                                              \
    return launch_plain(k_blur<RR, 32, 1>, grid, kThreads, smem_bytes<RR, 32, 1>(), s, d, 0, 0, t);
  switch (R) {
    SIFT_FOR_EACH_R(CASE_R)
    default:
      if (upsample)
        return launch_plain(k_blur_generic<2>, grid, kThreads, generic_smem_bytes(R), s, d, 0, 0, R, t);
      return launch_plain(k_blur_generic<1>, grid, kThreads, generic_smem_bytes(R), s, d, 0, 0, R, t);
  }
#undef CASE_R
}

int blur_blocks_per_sm(int R, int th_kind, int mode) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define OCC(fn, bytes) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, bytes);
#define CASE_R(RR)                                                                       \
  case RR:                                                                               \
    if (mode == 1) { OCC((k_blur<RR, 32, 1>), (smem_bytes<RR, 32, 1>())) }                \
    else if (mode == 2) { e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_base_poly<(RR + 2) / 2>, kPolyThreads, 0); } \
    else if (th_kind == TK_BLUR64) { OCC((k_blur<RR, 64, 0>), (smem_bytes<RR, 64, 0>())) } \
    else { OCC((k_blur<RR, 32, 0>), (smem_bytes<RR, 32, 0>())) }                          \
    break;
  switch (R) {
    SIFT_FOR_EACH_R(CASE_R)
    default:
      if (mode == 0) { OCC(k_blur_generic<0>, generic_smem_bytes(R)) }
      else if (mode == 1) { OCC(k_blur_generic<1>, generic_smem_bytes(R)) }
      else { OCC(k_blur_generic<2>, generic_smem_bytes(R)) }
  }
#undef CASE_R
#undef OCC
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

}  // namespace sift

// GPU MAGSAC++ homography verification (§3.6 "GPU MAGSAC++").
//
// Hypotheses: one thread per minimal sample of 4 correspondences fits the
// homography by the normalised DLT in FP64. Each image's 4 points are moved to
// centroid 0 and mean distance sqrt(2). The 8 x 8 system of the DLT with
// h33 = 1 is then solved by Gaussian elimination with partial pivoting, and the
// result is de-normalised and scaled to H[2][2] = 1. A sample is degenerate
// (score +inf) in four cases:
//   - an index lies outside [0, n);
//   - three of its normalised points in either image span a triangle of area
//     below 1e-6;
//   - the system is singular, or its solution has |(h, 1)| above 1e9 (the unit
//     null vector's last entry below 1e-9);
//   - |H[2][2]| falls below 1e-12 of the largest entry.
//
// Scoring: one block per hypothesis sums the MAGSAC++ loss over all
// correspondences. The loss is the chi (4 degrees of freedom) likelihood
// marginalised over the noise sigma in [0, sigma_max], truncated at
// k sigma_max (k the 0.99 chi quantile), as an M-estimator loss:
//   rho(r) = P (s^2 gamma(5/2, x) + r^2 / 2 (Gamma(3/2, x) - Gamma(3/2, k^2 / 2))),
//   x = r^2 / (2 s^2), P = 2^(3/2) / (4 s), s = sigma_max; rho(k s) beyond.
// The incomplete gamma functions of half-integer order come from erfc and exp
// by the recurrence Gamma(a + 1, x) = a Gamma(a, x) + x^a e^-x, starting from
// Gamma(1/2, x) = sqrt(pi) erfc(sqrt(x)). The residual is the forward transfer
// error |pi(H x) - x'| in FP32. Each thread adds its correspondences in index
// order, and the block combines the threads in a fixed tree: the scores are
// bitwise reproducible.
//
// Selection: one block takes the smallest score (ties to the smaller index)
// and marks the inliers of its model (r <= k sigma_max).
#include <algorithm>
#include <cmath>

#include "sift_dev.cuh"

namespace sift {

namespace {

constexpr int kFitThreads = 32;  // most FP64 solver threads per block
constexpr int kScoreThreads = 256;
constexpr int kSelectThreads = 1024;

struct MagsacConst {
  float kk_s2;     // (k sigma_max)^2
  float inv_2s2;   // 1 / (2 sigma_max^2)
  float s2;        // sigma_max^2
  float pref;      // C(4) 2^(3/2) / sigma_max
  float g15_k;     // Gamma(3/2, k^2 / 2)
  float rho_max;   // rho(k sigma_max)
};

__device__ __forceinline__ float magsac_rho(float r2, const MagsacConst &c) {
  if (!(r2 < c.kk_s2)) return c.rho_max;  // beyond the truncation, +inf or NaN
  const float x = r2 * c.inv_2s2;
  const float sx = sqrtf(x), ex = expf(-x);
  const float g15 = 0.886226925452758f * erfcf(sx) + sx * ex;  // Gamma(3/2, x)
  const float g25 = 1.5f * g15 + x * sx * ex;                   // Gamma(5/2, x)
  const float l25 = 1.329340388179137f - g25;                   // gamma(5/2, x)
  return c.pref * (c.s2 * l25 + 0.5f * r2 * (g15 - c.g15_k));
}

// Squared forward transfer error of (a -> b) under H (row-major, FP32).
__device__ __forceinline__ float transfer_r2(const float *H, float2 a, float2 b) {
  const float q0 = fmaf(H[0], a.x, fmaf(H[1], a.y, H[2]));
  const float q1 = fmaf(H[3], a.x, fmaf(H[4], a.y, H[5]));
  const float q2 = fmaf(H[6], a.x, fmaf(H[7], a.y, H[8]));
  if (q2 == 0.f) return INFINITY;
  const float dx = q0 / q2 - b.x, dy = q1 / q2 - b.y;
  return dx * dx + dy * dy;
}

// Hartley normalisation of 4 points in place; returns (s, cx, cy).
__device__ void normalise4(double p[4][2], double *s, double *cx, double *cy) {
  double mx = 0.0, my = 0.0;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    mx += p[j][0];
    my += p[j][1];
  }
  mx /= 4.0;
  my /= 4.0;
  double d = 0.0;
#pragma unroll
  for (int j = 0; j < 4; j++) d += sqrt((p[j][0] - mx) * (p[j][0] - mx) + (p[j][1] - my) * (p[j][1] - my));
  d /= 4.0;
  const double sc = d > 0.0 ? 1.4142135623730951 / d : 1.0;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    p[j][0] = sc * p[j][0] - sc * mx;
    p[j][1] = sc * p[j][1] - sc * my;
  }
  *s = sc;
  *cx = mx;
  *cy = my;
}

__device__ bool collinear4(const double p[4][2]) {
  const int tri[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  for (int t = 0; t < 4; t++) {
    const int i = tri[t][0], j = tri[t][1], m = tri[t][2];
    const double a = 0.5 * fabs((p[j][0] - p[i][0]) * (p[m][1] - p[i][1]) -
                                (p[j][1] - p[i][1]) * (p[m][0] - p[i][0]));
    if (a < 1e-6) return true;
  }
  return false;
}

// Column C of Gaussian elimination with partial pivoting on the 8 x 9
// augmented system: the row r >= C with the largest |M[r][C]| (the first on
// ties) becomes the pivot row, the rows below are reduced. False if the
// column is all zero (singular system).
template <int C>
__device__ __forceinline__ bool elim_step(double (&M)[8][9], double (&rinv)[8]) {
  int piv = C;
  double best = fabs(M[C][C]);
#pragma unroll
  for (int r = C + 1; r < 8; r++) {
    const double a = fabs(M[r][C]);
    if (a > best) {
      best = a;
      piv = r;
    }
  }
  if (best == 0.0) return false;
#pragma unroll
  for (int r = C + 1; r < 8; r++) {
    const bool sw = piv == r;
#pragma unroll
    for (int k = C; k < 9; k++) {
      const double t = M[C][k];
      M[C][k] = sw ? M[r][k] : t;
      M[r][k] = sw ? t : M[r][k];
    }
  }
  rinv[C] = 1.0 / M[C][C];
#pragma unroll
  for (int r = C + 1; r < 8; r++) {
    const double f = M[r][C] * rinv[C];
#pragma unroll
    for (int k = C; k < 9; k++) M[r][k] -= f * M[C][k];
  }
  return true;
}

__global__ void __launch_bounds__(kFitThreads) k_magsac_fit(const float2 *__restrict__ xa,
                                                            const float2 *__restrict__ xb, int n,
                                                            const int *__restrict__ samples,
                                                            int n_hyp, double *__restrict__ models,
                                                            int *__restrict__ valid) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= n_hyp) return;
  int idx[4];
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    idx[j] = samples[4 * h + j];
    ok = ok && idx[j] >= 0 && idx[j] < n;
  }
  if (!ok) {
    valid[h] = 0;
    return;
  }
  double pa[4][2], pb[4][2];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const float2 a = xa[idx[j]], b = xb[idx[j]];
    pa[j][0] = a.x;
    pa[j][1] = a.y;
    pb[j][0] = b.x;
    pb[j][1] = b.y;
  }
  double sa, ax, ay, sb, bx, by;
  normalise4(pa, &sa, &ax, &ay);
  normalise4(pb, &sb, &bx, &by);
  if (collinear4(pa) || collinear4(pb)) {
    valid[h] = 0;
    return;
  }
  // A h = 0 with h33 = 1: rows (x, y, 1, 0, 0, 0, -u x, -u y | u) and
  // (0, 0, 0, x, y, 1, -v x, -v y | v) (signs flipped from the DLT rows).
  double M[8][9];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const double x = pa[j][0], y = pa[j][1], u = pb[j][0], v = pb[j][1];
    const double r0[9] = {x, y, 1.0, 0.0, 0.0, 0.0, -u * x, -u * y, u};
    const double r1[9] = {0.0, 0.0, 0.0, x, y, 1.0, -v * x, -v * y, v};
#pragma unroll
    for (int c = 0; c < 9; c++) {
      M[2 * j][c] = r0[c];
      M[2 * j + 1][c] = r1[c];
    }
  }
  // One instantiation per pivot column (elim_step<C>), so every index is a
  // compile-time constant and M stays in registers: the pivot row is swapped
  // in by selects, and each pivot's reciprocal is taken once.
  double rinv[8];
  bool ok8 = elim_step<0>(M, rinv) && elim_step<1>(M, rinv) && elim_step<2>(M, rinv) &&
             elim_step<3>(M, rinv) && elim_step<4>(M, rinv) && elim_step<5>(M, rinv) &&
             elim_step<6>(M, rinv) && elim_step<7>(M, rinv);
  if (!ok8) {
    valid[h] = 0;
    return;
  }
  double hn[9];
  hn[8] = 1.0;
#pragma unroll
  for (int c = 7; c >= 0; c--) {
    double acc = M[c][8];
#pragma unroll
    for (int k = c + 1; k < 8; k++) acc -= M[c][k] * hn[k];
    hn[c] = acc * rinv[c];
  }
  double nn = 1.0;
  for (int k = 0; k < 8; k++) nn += hn[k] * hn[k];
  if (!(nn <= 1e18)) {  // the null vector's h33 component below 1e-9 (or not finite)
    valid[h] = 0;
    return;
  }
  // H = Tb^-1 Hn Ta with Ta = [[sa, 0, -sa ax], [0, sa, -sa ay], [0, 0, 1]] and
  // Tb^-1 = [[1/sb, 0, bx], [0, 1/sb, by], [0, 0, 1]].
  double G[9];  // Hn Ta
  for (int r = 0; r < 3; r++) {
    const double a0 = hn[3 * r], a1 = hn[3 * r + 1], a2 = hn[3 * r + 2];
    G[3 * r] = a0 * sa;
    G[3 * r + 1] = a1 * sa;
    G[3 * r + 2] = a2 - a0 * sa * ax - a1 * sa * ay;
  }
  double H[9];
  for (int c = 0; c < 3; c++) {
    H[c] = G[c] / sb + bx * G[6 + c];
    H[3 + c] = G[3 + c] / sb + by * G[6 + c];
    H[6 + c] = G[6 + c];
  }
  double mx = 0.0;
  for (int k = 0; k < 9; k++) mx = fmax(mx, fabs(H[k]));
  if (!(fabs(H[8]) >= 1e-12 * mx)) {
    valid[h] = 0;
    return;
  }
  const double inv = 1.0 / H[8];
  for (int k = 0; k < 9; k++) models[9 * h + k] = H[k] * inv;
  models[9 * h + 8] = 1.0;
  valid[h] = 1;
}

__global__ void __launch_bounds__(kScoreThreads) k_magsac_score(const float2 *__restrict__ xa,
                                                                const float2 *__restrict__ xb,
                                                                int n, const double *__restrict__ models,
                                                                const int *__restrict__ valid,
                                                                int n_hyp, MagsacConst c,
                                                                float *__restrict__ scores) {
  __shared__ float red[kScoreThreads / 32];
  const int tid = threadIdx.x;
  for (int h = blockIdx.x; h < n_hyp; h += gridDim.x) {
    if (!valid[h]) {  // block-uniform
      if (tid == 0) scores[h] = INFINITY;
      continue;
    }
    float H[9];
#pragma unroll
    for (int k = 0; k < 9; k++) H[k] = (float)models[9 * h + k];
    float acc = 0.f;
    for (int i = tid; i < n; i += kScoreThreads) acc += magsac_rho(transfer_r2(H, xa[i], xb[i]), c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
      float s = red[0];
#pragma unroll
      for (int w = 1; w < kScoreThreads / 32; w++) s += red[w];
      scores[h] = s;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void better(float &v, int &i, float v2, int i2) {
  if (v2 < v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

__global__ void __launch_bounds__(kSelectThreads) k_magsac_select(
    const float2 *__restrict__ xa, const float2 *__restrict__ xb, int n,
    const double *__restrict__ models, const float *__restrict__ scores, int n_hyp, MagsacConst c,
    double *__restrict__ H_out, int *__restrict__ best_out, float *__restrict__ score_out,
    unsigned char *__restrict__ inliers, float *__restrict__ scores_out) {
  __shared__ float sv[kSelectThreads / 32];
  __shared__ int si[kSelectThreads / 32];
  __shared__ float s_H[9];
  __shared__ int s_best;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float v = INFINITY;
  int bi = 0x7fffffff;
  for (int h = tid; h < n_hyp; h += kSelectThreads) {
    const float s = scores[h];
    if (scores_out) scores_out[h] = s;
    better(v, bi, s, h);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    better(v, bi, v2, i2);
  }
  if (lane == 0) {
    sv[warp] = v;
    si[warp] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    float bv = sv[0];
    int b = si[0];
    for (int w = 1; w < kSelectThreads / 32; w++) better(bv, b, sv[w], si[w]);
    const int best = (bv < INFINITY) ? b : -1;
    s_best = best;
    *best_out = best;
    *score_out = best >= 0 ? bv : INFINITY;
    for (int k = 0; k < 9; k++) {
      const double e = best >= 0 ? models[9 * best + k] : 0.0;
      H_out[k] = e;
      s_H[k] = (float)e;
    }
  }
  __syncthreads();
  const int best = s_best;
  for (int i = tid; i < n; i += kSelectThreads)
    inliers[i] = (best >= 0 && transfer_r2(s_H, xa[i], xb[i]) <= c.kk_s2) ? 1 : 0;
}

// Gamma(3/2, x) and gamma(5/2, x) in double (host), by the same recurrences.
double upper_g15(double x) { return 0.5 * std::sqrt(M_PI) * std::erfc(std::sqrt(x)) + std::sqrt(x) * std::exp(-x); }
double lower_g25(double x) {
  return 0.75 * std::sqrt(M_PI) - (1.5 * upper_g15(x) + x * std::sqrt(x) * std::exp(-x));
}

// k: the 0.99 quantile of the chi distribution with 4 degrees of freedom.
// P(chi^2_4 <= 2y) = 1 - e^-y (1 + y); Newton on e^-y (1 + y) = 0.01.
double chi4_quantile_099() {
  double y = 6.0;
  for (int it = 0; it < 60; it++) {
    const double f = std::exp(-y) * (1.0 + y) - 0.01;
    const double df = -std::exp(-y) * y;
    const double step = f / df;
    y -= step;
    if (std::fabs(step) < 1e-15 * y) break;
  }
  return std::sqrt(2.0 * y);
}

MagsacConst make_const(float sigma_max) {
  const double s = sigma_max, k = chi4_quantile_099();
  const double pref = 0.25 * std::pow(2.0, 1.5) / s;
  const double xk = 0.5 * k * k;
  MagsacConst c;
  c.kk_s2 = (float)(k * k * s * s);
  c.inv_2s2 = (float)(1.0 / (2.0 * s * s));
  c.s2 = (float)(s * s);
  c.pref = (float)pref;
  c.g15_k = (float)upper_g15(xk);
  c.rho_max = (float)(pref * (s * s * lower_g25(xk)));  // the r^2 term vanishes at k sigma_max
  return c;
}

}  // namespace

size_t magsac_workspace_bytes(int n_hyp) {
  return (size_t)n_hyp * (9 * sizeof(double) + sizeof(int) + sizeof(float)) + 256;
}

cudaError_t launch_magsac(const float *xa, const float *xb, int n, const int *samples, int n_hyp,
                          float sigma_max, void *ws, cudaStream_t s, double *H_out, int *best_out,
                          float *score_out, unsigned char *inliers, float *scores_out) {
  char *p = static_cast<char *>(ws);
  double *models = reinterpret_cast<double *>(p);
  int *valid = reinterpret_cast<int *>(p + (size_t)n_hyp * 9 * sizeof(double));
  float *scores = reinterpret_cast<float *>(p + (size_t)n_hyp * (9 * sizeof(double) + sizeof(int)));
  const MagsacConst c = make_const(sigma_max);
  const float2 *a = reinterpret_cast<const float2 *>(xa);
  const float2 *b = reinterpret_cast<const float2 *>(xb);
  int dev = 0, n_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  // The FP64 solver is bound by each SM's FP64 rate: spread the hypotheses over
  // every SM (ceil(n_hyp / SMs) threads per block, at most 32).
  const int fit_threads = std::max(1, std::min(kFitThreads, (n_hyp + n_sm - 1) / n_sm));
  cudaError_t e = launch_plain(k_magsac_fit, (n_hyp + fit_threads - 1) / fit_threads, fit_threads,
                               0, s, a, b, n, samples, n_hyp, models, valid);
  if (e != cudaSuccess) return e;
  const int grid = n_hyp < 8 * n_sm ? n_hyp : 8 * n_sm;
  e = launch_plain(k_magsac_score, grid, kScoreThreads, 0, s, a, b, n, models, valid, n_hyp, c,
                   scores);
  if (e != cudaSuccess) return e;
  return launch_plain(k_magsac_select, 1, kSelectThreads, 0, s, a, b, n, models, scores, n_hyp, c,
                      H_out, best_out, score_out, inliers, scores_out);
}

}  // namespace sift

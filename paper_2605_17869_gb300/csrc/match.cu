// Symmetric ratio-test matcher (§3.4 "Descriptor Matching", first backend):
// the similarity matrix of two descriptor sets from fp16 tensor-core products,
// nearest neighbours in both directions, mutual consistency and Lowe's ratio
// test on both sides.
//
// The similarity matrix is a dense N x M x 128 contraction, so it runs on the
// 5th-generation tensor cores. Both sets are first converted once to fp16 in
// the core-matrix layout the tensor core reads. Then every CTA of a 2-D grid
// takes one 128-row block of one set and one 256-row tile of the other:
// both arrive in shared memory by two bulk copies on an mbarrier, one thread
// issues 8 tcgen05.mma (M = 128, N = 256, K = 16, FP32 accumulation in TMEM)
// and commits them to a second mbarrier (both waits bounded), and each warp
// reads its 32 accumulator rows back with tcgen05.ld, reducing each row to
// the tile's best index and two best similarities. A merge kernel combines
// the tiles per row in tile order (ties keep the smaller index); running the
// grid with the sets swapped gives the other side, and a last kernel applies
// the mutual check and the ratio tests. The tensor core's accumulation order
// is fixed, so results are reproducible.
#include <cuda_fp16.h>

#include "sift_dev.cuh"

namespace sift {

namespace {

constexpr int kMM = 128;      // A rows per CTA (TMEM lanes)
constexpr int kMN = 256;      // B rows per tile (accumulator columns)
constexpr int kDim = 128;     // descriptor length (K)
constexpr int kMThreads = 128;
constexpr int kSmemA = kMM * kDim * 2;   // 32 KB of fp16
constexpr int kSmemB = kMN * kDim * 2;   // 64 KB of fp16
constexpr unsigned kMaxPolls = 1u << 22;

__device__ __forceinline__ unsigned saddr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of a K-major operand without swizzle: 8 x 8
// fp16 core matrices of 128 contiguous bytes, the next core matrix along K at
// +128 bytes (leading byte offset), the next 8-row group at +2048 bytes (stride
// byte offset); bits 46-47 hold the descriptor version (1).
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
  const unsigned long long lbo = 128 >> 4, sbo = 2048 >> 4;
  return (unsigned long long)((addr >> 4) & 0x3FFFu) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B fp16 (formats 0), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr unsigned kIdesc = (1u << 4) | ((unsigned)(kMN >> 3) << 17) | ((unsigned)(kMM >> 4) << 24);

__device__ __forceinline__ void mbar_init(unsigned long long *m) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(m)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *m, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded: gives up after kMaxPolls polls (each may suspend the thread briefly).
__device__ __forceinline__ bool mbar_wait(unsigned long long *m, unsigned parity) {
  for (unsigned i = 0; i < kMaxPolls; i++)
    if (mbar_try_wait(m, parity)) return true;
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// A descriptor set (FP32, kDim per row, row-major) as fp16 core matrices in
// global memory, the layout the tensor core reads from shared memory: core
// matrix (row / 8, k / 8) at byte (row / 8) * 2048 + (k / 8) * 128, 8 rows x
// 16 bytes inside; rows n .. n_pad - 1 are zero. A 128-row block is then 32
// contiguous KB and a 256-row tile 64 contiguous KB. Thread: 8 elements.
__global__ void k_to_core_matrices(const float *__restrict__ src, int n, int n_pad,
                                   unsigned char *dst) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;  // (row, k-group) chunk
  if (c >= n_pad * (kDim / 8)) return;
  const int row = c >> 4, kg = c & 15;
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (row < n) {
    const float4 *p = reinterpret_cast<const float4 *>(src + (size_t)row * kDim + kg * 8);
    const float4 a = __ldg(p), b = __ldg(p + 1);
    const __half2 h0 = __floats2half2_rn(a.x, a.y), h1 = __floats2half2_rn(a.z, a.w);
    const __half2 h2 = __floats2half2_rn(b.x, b.y), h3 = __floats2half2_rn(b.z, b.w);
    v = make_uint4(*reinterpret_cast<const unsigned *>(&h0), *reinterpret_cast<const unsigned *>(&h1),
                   *reinterpret_cast<const unsigned *>(&h2), *reinterpret_cast<const unsigned *>(&h3));
  }
  *reinterpret_cast<uint4 *>(dst + (size_t)(row >> 3) * 2048 + kg * 128 + (row & 7) * 16) = v;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(m)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(m))
      : "memory");
}

// One 128-row block of A (blockIdx.x) against one 256-row tile of B
// (blockIdx.y), both already in core-matrix layout: per row of the block, the
// tile's best column (ties: smaller index), best and second-best similarity,
// written to the tile's slot of the partial arrays ([tile][row]). Columns past
// n_b are ignored.
__global__ void __launch_bounds__(kMThreads, 1)
    k_match_tile(const unsigned char *__restrict__ Acm, int n_a, const unsigned char *__restrict__ Bcm,
                 int n_b, int n_a_pad, int *p_best, float *p_s1, float *p_s2, int *err) {
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char *sA = sm;
  unsigned char *sB = sm + kSmemA;
  __shared__ __align__(8) unsigned long long bar_copy, bar_mma;
  __shared__ unsigned tmem_sh;
  const int warp = threadIdx.x >> 5;
  const int r0 = blockIdx.x * kMM, j0 = blockIdx.y * kMN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_sh)),
                 "r"(kMN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar_copy);
    mbar_init(&bar_mma);
    mbar_arrive_expect_tx(&bar_copy, kSmemA + kSmemB);
    bulk_g2s(sA, Acm + (size_t)r0 * kDim * 2, kSmemA, &bar_copy);
    bulk_g2s(sB, Bcm + (size_t)j0 * kDim * 2, kSmemB, &bar_copy);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_sh;
  bool ok = true;
  if (threadIdx.x == 0) {
    ok = mbar_wait(&bar_copy, 0);
    if (ok) {
#pragma unroll
      for (int kk = 0; kk < kDim / 16; kk++) {
        const unsigned long long da = smem_desc(saddr(sA) + kk * 256);
        const unsigned long long db = smem_desc(saddr(sB) + kk * 256);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(kIdesc), "r"(kk)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              saddr(&bar_mma))
          : "memory");
    }
  }
  if (__syncthreads_or(!ok)) {  // the copies never landed: flag, wait once more, free, exit
    if (threadIdx.x == 0) {
      *err = 1;
      mbar_wait(&bar_copy, 0);
    }
  } else {
    ok = mbar_wait(&bar_mma, 0);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        *err = 1;
        mbar_wait(&bar_mma, 0);
      }
    } else {
      tc_fence_after();
      float s1 = -INFINITY, s2 = -INFINITY;
      int b1 = -1;
#pragma unroll 1
      for (int ch = 0; ch < kMN / 32; ch++) {
        unsigned v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
            "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
            "%30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
              "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
              "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
              "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(tmem + ((unsigned)(32 * warp) << 16) + (unsigned)(ch * 32)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 32; c++) {
          const int j = j0 + ch * 32 + c;
          const float s = __uint_as_float(v[c]);
          if (j < n_b) {
            if (s > s1) {
              s2 = s1;
              s1 = s;
              b1 = j;
            } else if (s > s2) {
              s2 = s;
            }
          }
        }
      }
      const int row = r0 + (int)threadIdx.x;
      if (row < n_a) {
        const size_t o = (size_t)blockIdx.y * n_a_pad + row;
        p_best[o] = b1;
        p_s1[o] = s1;
        p_s2[o] = s2;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMN)
                 : "memory");
  }
}

// Per row: merge the tiles' partial results in tile order (so ties keep the
// smaller column index): best, best and second-best similarity.
__global__ void k_match_merge(int n, int n_pad, int n_tiles, const int *p_best, const float *p_s1,
                              const float *p_s2, int *best, float *s1o, float *s2o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s1 = -INFINITY, s2 = -INFINITY;
  int b1 = -1;
  for (int t = 0; t < n_tiles; t++) {
    const size_t o = (size_t)t * n_pad + i;
    const float a1 = p_s1[o], a2 = p_s2[o];
    if (a1 > s1) {
      s2 = fmaxf(s1, a2);
      s1 = a1;
      b1 = p_best[o];
    } else {
      s2 = fmaxf(s2, a1);
    }
  }
  best[i] = b1;
  s1o[i] = s1;
  s2o[i] = s2;
}

__device__ __forceinline__ float unit_distance(float s) { return sqrtf(fmaxf(0.f, 2.f - 2.f * s)); }

// Mutual nearest neighbours passing the ratio test on both sides; -1 else,
// -2 for every row if a bounded device wait gave up.
__global__ void k_match_final(int n_a, int n_b, float ratio, const int *best_a, const float *s1_a,
                              const float *s2_a, const int *best_b, const float *s1_b,
                              const float *s2_b, const int *err, int *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_a) return;
  int m = -1;
  if (*err) {
    m = -2;
  } else if (n_a >= 2 && n_b >= 2) {
    const int j = best_a[i];
    if (j >= 0 && best_b[j] == i && unit_distance(s1_a[i]) < ratio * unit_distance(s2_a[i]) &&
        unit_distance(s1_b[j]) < ratio * unit_distance(s2_b[j]))
      m = j;
  }
  out[i] = m;
}

}  // namespace

static inline size_t pad256(int n) { return (size_t)((n + kMN - 1) / kMN) * kMN; }
static inline size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Workspace: error word, both sets in core-matrix layout, per-tile partials of
// both directions, merged per-row results of both sides.
size_t match_workspace_bytes(int n_a, int n_b) {
  const size_t pa = pad256(n_a), pb = pad256(n_b);
  const size_t ta = pa / kMN, tb = pb / kMN;
  return 256 + align256(pa * kDim * 2) + align256(pb * kDim * 2) + align256(tb * pa * 12) +
         align256(ta * pb * 12) + align256(pa * 12) + align256(pb * 12);
}

cudaError_t match_set_attributes() {
  return cudaFuncSetAttribute(k_match_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSmemA + kSmemB);
}

cudaError_t launch_match(const float *A, int n_a, const float *B, int n_b, float ratio, void *ws,
                         int *out, cudaStream_t s) {
  const size_t pa = pad256(n_a), pb = pad256(n_b);
  const int ta = (int)(pa / kMN), tb = (int)(pb / kMN);
  char *w = static_cast<char *>(ws);
  int *err = reinterpret_cast<int *>(w);
  size_t o = 256;
  auto take = [&](size_t bytes) {
    char *p = w + o;
    o += align256(bytes);
    return p;
  };
  unsigned char *Acm = reinterpret_cast<unsigned char *>(take(pa * kDim * 2));
  unsigned char *Bcm = reinterpret_cast<unsigned char *>(take(pb * kDim * 2));
  char *pab = take((size_t)tb * pa * 12);  // A rows against B tiles
  char *pba = take((size_t)ta * pb * 12);  // B rows against A tiles
  char *ra = take(pa * 12);
  char *rb = take(pb * 12);
  int *pab_best = reinterpret_cast<int *>(pab);
  float *pab_s1 = reinterpret_cast<float *>(pab_best + (size_t)tb * pa);
  float *pab_s2 = pab_s1 + (size_t)tb * pa;
  int *pba_best = reinterpret_cast<int *>(pba);
  float *pba_s1 = reinterpret_cast<float *>(pba_best + (size_t)ta * pb);
  float *pba_s2 = pba_s1 + (size_t)ta * pb;
  int *best_a = reinterpret_cast<int *>(ra);
  float *s1_a = reinterpret_cast<float *>(best_a + pa);
  float *s2_a = s1_a + pa;
  int *best_b = reinterpret_cast<int *>(rb);
  float *s1_b = reinterpret_cast<float *>(best_b + pb);
  float *s2_b = s1_b + pb;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess || n_a == 0) return e;
  if (n_b > 0) {
    e = launch_plain(k_to_core_matrices, (int)((pa * 16 + 255) / 256), 256, 0, s, A, n_a, (int)pa,
                     Acm);
    if (e == cudaSuccess)
      e = launch_plain(k_to_core_matrices, (int)((pb * 16 + 255) / 256), 256, 0, s, B, n_b,
                       (int)pb, Bcm);
    if (e == cudaSuccess)
      e = launch_plain(k_match_tile, dim3((n_a + kMM - 1) / kMM, tb), kMThreads, kSmemA + kSmemB,
                       s, Acm, n_a, Bcm, n_b, (int)pa, pab_best, pab_s1, pab_s2, err);
    if (e == cudaSuccess)
      e = launch_plain(k_match_tile, dim3((n_b + kMM - 1) / kMM, ta), kMThreads, kSmemA + kSmemB,
                       s, Bcm, n_b, Acm, n_a, (int)pb, pba_best, pba_s1, pba_s2, err);
    if (e == cudaSuccess)
      e = launch_plain(k_match_merge, (n_a + 255) / 256, 256, 0, s, n_a, (int)pa, tb, pab_best,
                       pab_s1, pab_s2, best_a, s1_a, s2_a);
    if (e == cudaSuccess)
      e = launch_plain(k_match_merge, (n_b + 255) / 256, 256, 0, s, n_b, (int)pb, ta, pba_best,
                       pba_s1, pba_s2, best_b, s1_b, s2_b);
    if (e != cudaSuccess) return e;
  }
  return launch_plain(k_match_final, (n_a + 255) / 256, 256, 0, s, n_a, n_b, ratio, best_a, s1_a,
                      s2_a, best_b, s1_b, s2_b, err, out);
}

}  // namespace sift

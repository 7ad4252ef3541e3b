// Symmetric ratio-test matcher (§3.3 "Descriptor Matching", first backend):
// the similarity matrix of two descriptor sets from fp16 tensor-core products,
// nearest neighbours in both directions, mutual consistency and Lowe's ratio
// test on both sides.
//
// The similarity matrix is a dense N x M x 128 contraction, so it runs on the
// 5th-generation tensor cores: a CTA stages 128 rows of set A as fp16 in
// shared memory once, then, for every 256-row tile of set B, stages the tile,
// issues 8 tcgen05.mma (M = 128, N = 256, K = 16, FP32 accumulation in TMEM)
// from one thread, waits on the commit's mbarrier (bounded), and reads its
// accumulator rows back with tcgen05.ld, keeping each row's best index and two
// best similarities in registers. Running the same kernel with the sets
// swapped gives the column side; a last kernel applies the mutual check and
// the ratio tests. Ties go to the smaller index; the accumulation order of the
// tensor core is fixed, so results are reproducible.
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

// Rows [r0, r0 + R) of a set (FP32, kDim per row, row-major) into shared memory
// as fp16 core matrices: core matrix (row / 8, k / 8) at byte
// (row / 8) * 2048 + (k / 8) * 128, row-major 8 x 16 bytes inside. Rows past n
// are zero. Thread t converts 8 consecutive elements of a row per step.
template <int R>
__device__ __forceinline__ void stage_fp16(const float *__restrict__ src, int n, int r0,
                                           unsigned char *dst) {
  for (int c = threadIdx.x; c < R * (kDim / 8); c += kMThreads) {
    const int row = c >> 4, kg = c & 15;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r0 + row < n) {
      const float4 *p = reinterpret_cast<const float4 *>(src + (size_t)(r0 + row) * kDim + kg * 8);
      const float4 a = __ldg(p), b = __ldg(p + 1);
      const __half2 h0 = __floats2half2_rn(a.x, a.y), h1 = __floats2half2_rn(a.z, a.w);
      const __half2 h2 = __floats2half2_rn(b.x, b.y), h3 = __floats2half2_rn(b.z, b.w);
      v = make_uint4(*reinterpret_cast<const unsigned *>(&h0), *reinterpret_cast<const unsigned *>(&h1),
                     *reinterpret_cast<const unsigned *>(&h2), *reinterpret_cast<const unsigned *>(&h3));
    }
    *reinterpret_cast<uint4 *>(dst + (row >> 3) * 2048 + kg * 128 + (row & 7) * 16) = v;
  }
}

// Per row i of A (n_a rows): the index of the row of B (n_b rows) with the
// largest fp16 dot product (ties: smaller index), that value and the second
// largest. A row with no candidate keeps (-1, -inf, -inf).
__global__ void __launch_bounds__(kMThreads, 1)
    k_match_rows(const float *__restrict__ A, int n_a, const float *__restrict__ B, int n_b,
                 int *best, float *s1_out, float *s2_out, int *err) {
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char *sA = sm;
  unsigned char *sB = sm + kSmemA;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ unsigned tmem_sh;
  const int warp = threadIdx.x >> 5;
  const int r0 = blockIdx.x * kMM;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_sh)),
                 "r"(kMN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) mbar_init(&mbar);
  stage_fp16<kMM>(A, n_a, r0, sA);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_sh;
  float s1 = -INFINITY, s2 = -INFINITY;
  int b1 = -1;
  bool stalled = false;
  for (int t = 0, j0 = 0; j0 < n_b; j0 += kMN, t++) {
    stage_fp16<kMN>(B, n_b, j0, sB);
    // generic-proxy shared-memory writes -> visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
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
              saddr(&mbar))
          : "memory");
    }
    const bool ok = mbar_wait(&mbar, t & 1);
    if (__syncthreads_or(!ok)) {
      stalled = true;
      if (threadIdx.x == 0) {
        *err = 1;
        mbar_wait(&mbar, t & 1);  // a second bounded chance for the MMAs in flight
      }
      break;
    }
    tc_fence_after();
    // This warp's 32 accumulator rows (TMEM lanes 32 w ..), 32 columns at a time.
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
    tc_fence_before();
    __syncthreads();  // accumulator and B tile are read before the next tile reuses them
  }
  const int row = r0 + (int)threadIdx.x;
  if (!stalled && row < n_a) {
    best[row] = b1;
    s1_out[row] = s1;
    s2_out[row] = s2;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMN)
                 : "memory");
  }
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

size_t match_workspace_bytes(int n_a, int n_b) {
  const size_t rows = (size_t)n_a + (size_t)n_b;
  return 256 + rows * 3 * 4;
}

cudaError_t match_set_attributes() {
  return cudaFuncSetAttribute(k_match_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSmemA + kSmemB);
}

cudaError_t launch_match(const float *A, int n_a, const float *B, int n_b, float ratio, void *ws,
                         int *out, cudaStream_t s) {
  char *w = static_cast<char *>(ws);
  int *err = reinterpret_cast<int *>(w);
  int *best_a = reinterpret_cast<int *>(w + 256);
  float *s1_a = reinterpret_cast<float *>(best_a + n_a);
  float *s2_a = s1_a + n_a;
  int *best_b = reinterpret_cast<int *>(s2_a + n_a);
  float *s1_b = reinterpret_cast<float *>(best_b + n_b);
  float *s2_b = s1_b + n_b;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess || n_a == 0) return e;
  if (n_b > 0) {
    k_match_rows<<<(n_a + kMM - 1) / kMM, kMThreads, kSmemA + kSmemB, s>>>(A, n_a, B, n_b, best_a,
                                                                           s1_a, s2_a, err);
    k_match_rows<<<(n_b + kMM - 1) / kMM, kMThreads, kSmemA + kSmemB, s>>>(B, n_b, A, n_a, best_b,
                                                                           s1_b, s2_b, err);
  }
  k_match_final<<<(n_a + 255) / 256, 256, 0, s>>>(n_a, n_b, ratio, best_a, s1_a, s2_a, best_b,
                                                  s1_b, s2_b, err, out);
  return cudaGetLastError();
}

}  // namespace sift

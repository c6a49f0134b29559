// k_umma.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05), FP32 accumulate in TMEM.
//
// D[M x N] = A[M x K] . B[K x N] for the message-passing network's layer products (M = vertices,
// N, K in {64, 192}).  Operands are kept in global memory already in the shared-memory image the
// MMA reads ("K-major, no swizzle" core-matrix layout), so one bulk copy per operand tile moves them
// into shared memory:
//   element (r, k) of a block of R rows  ->  byte (k / 16) * (R * 32) + ((k % 16) / 8) * 128
//                                              + (r / 8) * 256 + (r % 8) * 16 + (k % 8) * 2
// i.e. for each 16-wide K step, 8 x 8 core matrices of 128 contiguous bytes, the two K halves of a row
// group side by side (leading-dimension offset 128 B) and row groups 256 B apart (stride offset).
// A is stored as consecutive blocks of 128 rows; B (the weights, N x K with K contiguous) as one block.
//
// One CTA of 4 warps per 128-row tile (grid-strided): thread 0 issues the bulk copies (completion on
// an mbarrier) and the K/16 MMAs (completion committed to a second mbarrier); then each warp reads
// its 32 TMEM lanes (= rows) with tcgen05.ld and hands the FP32 row to the epilogue.  Every wait is
// bounded (about one second): on expiry the CTA records an error, stops issuing, waits (bounded)
// for what it issued, frees its TMEM and returns.
#pragma once
#include <cuda_bf16.h>

#include "gp_internal.cuh"

namespace gp {

__host__ __device__ __forceinline__ int64_t umma_off(int64_t r, int64_t k, int64_t R) {
  return (k >> 4) * (R * 32) + ((k & 15) >> 3) * 128 + (r >> 3) * 256 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// true once the phase with the given parity has completed; false after ~limit_ns
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, uint64_t limit_ns) {
  const uint32_t a = smem_u32(bar);
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, unsigned ncols) {  // one full warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, unsigned ncols) {  // one full warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, byte offsets between core matrices along K (lbo)
// and along M/N (sbo); bit 46 holds the descriptor version of this MMA generation.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor: D FP32, A and B BF16, both K-major, N and M sizes.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // one second
constexpr int kUmmaErrTimeout = 1;

template <int N>
constexpr unsigned umma_tmem_cols() {
  return N <= 32 ? 32u : N <= 64 ? 64u : N <= 128 ? 128u : 256u;
}

// Epilogue interface: epi(row, col0, v[16]) for every 16-column chunk of every row < M.
template <int N, int K, class Epi>
__global__ void __launch_bounds__(128) k_umma_gemm(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                   int64_t mtiles, int64_t M, Epi epi, int* err) {
  constexpr unsigned A_BYTES = 128u * K * 2u, B_BYTES = (unsigned)N * K * 2u;
  constexpr unsigned NCOLS = umma_tmem_cols<N>();
  constexpr uint32_t IDESC = umma_idesc_bf16(128, N);
  static_assert(K % 16 == 0 && N % 16 == 0 && N <= 256, "shape");
  extern __shared__ __align__(1024) uint8_t umma_sm[];
  uint8_t* sA = umma_sm;
  uint8_t* sB = umma_sm + A_BYTES;
  __shared__ __align__(8) uint64_t bar_ld, bar_mma;
  __shared__ uint32_t s_taddr;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) tmem_alloc(&s_taddr, NCOLS);
  if (threadIdx.x == 0) {
    mbar_init(&bar_ld, 1);
    mbar_init(&bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  unsigned ph_ld = 0, ph_mma = 0;
  bool issued_ld = false, issued_mma = false;
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar_ld, B_BYTES);
    bulk_g2s(sB, B, B_BYTES, &bar_ld);
  }
  issued_ld = true;
  if (!mbar_wait(&bar_ld, ph_ld, kWaitLimitNs)) s_fail = 1;
  ph_ld ^= 1;
  __syncthreads();
  if (!s_fail) issued_ld = false;
  for (int64_t t = blockIdx.x; t < mtiles && !s_fail; t += gridDim.x) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(&bar_ld, A_BYTES);
      bulk_g2s(sA, A + (size_t)t * A_BYTES, A_BYTES, &bar_ld);
    }
    issued_ld = true;
    if (!mbar_wait(&bar_ld, ph_ld, kWaitLimitNs)) s_fail = 1;
    ph_ld ^= 1;
    __syncthreads();
    if (s_fail) break;
    issued_ld = false;
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int s = 0; s < K / 16; s++) {
        const uint64_t ad = umma_desc(a0 + (uint32_t)s * 128u * 32u, 128u, 256u);
        const uint64_t bd = umma_desc(b0 + (uint32_t)s * (uint32_t)N * 32u, 128u, 256u);
        umma_bf16(taddr, ad, bd, IDESC, s > 0 ? 1u : 0u);
      }
      umma_commit(&bar_mma);
    }
    issued_mma = true;
    if (!mbar_wait(&bar_mma, ph_mma, kWaitLimitNs)) s_fail = 1;
    ph_mma ^= 1;
    __syncthreads();
    if (s_fail) break;
    issued_mma = false;
    tc_fence_after();
    const int64_t row = t * 128 + warp * 32 + lane;
    const uint32_t lane_addr = taddr + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c = 0; c < N / 16; c++) {
      float v[16];
      tmem_ld16(lane_addr + (uint32_t)(c * 16), v);
      if (row < M) epi(row, c * 16, v);
    }
    if (threadIdx.x == 0) {  // algorithmic bytes: the A tile, the outputs (and B once per CTA)
      const int64_t rows = (M - t * 128) < 128 ? (M - t * 128) : 128;
      atomicAdd(&d_alg_bytes[F_MPNN], (unsigned long long)A_BYTES +
                                          (unsigned long long)rows * N * Epi::kOutBytes +
                                          (t == blockIdx.x ? (unsigned long long)B_BYTES : 0ull));
    }
    tc_fence_before();
    __syncthreads();
  }
  if (s_fail) {
    // drain what this CTA issued (bounded), then release TMEM
    if (issued_ld) mbar_wait(&bar_ld, ph_ld ^ 1, kWaitLimitNs);
    if (issued_mma) mbar_wait(&bar_mma, ph_mma ^ 1, kWaitLimitNs);
    if (threadIdx.x == 0) atomicOr(err, kUmmaErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

// Failure-path check of the bounded waits: allocates tensor memory as the GEMM does, waits on an
// mbarrier that nothing arrives at (limit `limit_ns`), then releases the tensor memory and records
// the timeout, leaving the context usable.
__global__ void __launch_bounds__(128) k_wait_selftest(uint64_t limit_ns, int* err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_taddr;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) tmem_alloc(&s_taddr, 32);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!mbar_wait(&bar, 0, limit_ns)) s_fail = 1;  // no arrival: the wait must give up
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0 && s_fail) atomicOr(err, kUmmaErrTimeout);
  if (warp == 0) tmem_dealloc(s_taddr, 32);
}

template <int N, int K>
constexpr size_t umma_smem_bytes() {
  return 128u * K * 2u + (size_t)N * K * 2u;
}

// Row-major BF16 [R x K] -> the tiled image (rows padded to R_pad with zeros); R_block = rows per block.
__global__ void k_umma_tile(const __nv_bfloat16* __restrict__ src, int64_t R, int64_t R_pad, int K, int R_block,
                            __nv_bfloat16* __restrict__ dst) {
  const int64_t total = R_pad * (int64_t)K;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / K, k = i % K;
    const int64_t blk = r / R_block, rr = r % R_block;
    const __nv_bfloat16 v = r < R ? src[r * K + k] : __float2bfloat16(0.0f);
    dst[(blk * R_block * K * 2 + umma_off(rr, k, R_block)) / 2] = v;
  }
}

struct EpiStoreF32 {
  static constexpr unsigned kOutBytes = 4;  // FP32 per output
  float* C;
  int ldc;
  __device__ __forceinline__ void operator()(int64_t row, int col0, const float* v) const {
    float4* p = (float4*)(C + row * ldc + col0);
#pragma unroll
    for (int i = 0; i < 4; i++) p[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  }
};

template <int N, int K, class Epi>
cudaError_t umma_gemm(const void* A_tiled, const void* B_tiled, int64_t M, Epi epi, int* err, cudaStream_t s) {
  const int64_t mtiles = (M + 127) / 128;
  if (mtiles == 0) return cudaSuccess;
  // at most 512 / NCOLS CTAs of this kernel may hold tensor memory on an SM at once: extra shared
  // memory keeps the others off the SM rather than blocked in the allocation
  constexpr size_t need = umma_smem_bytes<N, K>();
  constexpr size_t per_sm = 233472;  // 228 KB of shared memory per SM
  constexpr size_t fit = per_sm / (512 / umma_tmem_cols<N>() + 1) + 1024;
  constexpr size_t smem = need > fit ? need : fit;
  auto kern = k_umma_gemm<N, K, Epi>;
  cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t cap = (int64_t)num_sms() * (int64_t)(per_sm / smem);
  const unsigned grid = (unsigned)(mtiles < cap ? mtiles : cap);
  launch_begin(F_MPNN, s);
  kern<<<grid, 128, smem, s>>>((const uint8_t*)A_tiled, (const uint8_t*)B_tiled, mtiles, M, epi, err);
  launch_end(F_MPNN, s);
  return cudaGetLastError();
}

}  // namespace gp

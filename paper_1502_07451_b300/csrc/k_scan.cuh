// k_scan.cuh -- exclusive prefix sums (reduce-then-scan, three launches, no inter-block waits; inputs of
// at most a few tiles: one block in one launch, the tiles in turn with a running carry).
#pragma once
#include "gp_internal.cuh"

namespace gp {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;  // consecutive items per thread
constexpr int kScanTile = kScanThreads * kScanItems;

template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const Tin* __restrict__ in, int64_t n,
                                                              Tout* __restrict__ partial) {
  __shared__ Tout sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  Tout s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    const int64_t idx = base + i;
    if (idx < n) s += (Tout)in[idx];
  }
  s = block_sum<Tout>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Exclusive scan of the thread values of a block; returns the thread's exclusive prefix and
// writes the block total to *total.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T x, T* sh, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  T inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = (lane < nw) ? sh[lane] : T(0);
    T winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= o) winc += y;
    }
    if (lane < nw) sh[lane] = winc - w;
    if (lane == 31) sh[32] = winc;
  }
  __syncthreads();
  T r = sh[wid] + inc - x;
  *total = sh[32];
  __syncthreads();
  return r;
}

template <class T>
__global__ void __launch_bounds__(1024) k_scan_partials(T* __restrict__ partial, int64_t nb) {
  __shared__ T sh[33];
  T carry = 0;
  for (int64_t b = 0; b < nb; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    T x = (i < nb) ? partial[i] : T(0);
    T tot;
    T ex = block_exclusive_scan<T>(x, sh, &tot);
    if (i < nb) partial[i] = carry + ex;
    carry += tot;
  }
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const Tin* __restrict__ in, int64_t n,
                                                            const Tout* __restrict__ partial,
                                                            Tout* __restrict__ out) {
  __shared__ Tout sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  Tout v[kScanItems];
  Tout s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    const int64_t idx = base + i;
    v[i] = (idx < n) ? (Tout)in[idx] : Tout(0);
    s += v[i];
  }
  Tout tot;
  Tout run = block_exclusive_scan<Tout>(s, sh, &tot) + partial[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    const int64_t idx = base + i;
    if (idx < n) out[idx] = run;
    run += v[i];
    if (idx == n - 1) out[n] = run;
  }
}

// One block over every tile of a short input, in order, carrying the running total.
template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_one_block(const Tin* __restrict__ in, int64_t n,
                                                                 Tout* __restrict__ out) {
  __shared__ Tout sh[33];
  Tout carry = 0;
  for (int64_t t0 = 0; t0 < n; t0 += kScanTile) {
    const int64_t base = t0 + (int64_t)threadIdx.x * kScanItems;
    Tout v[kScanItems];
    Tout sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
      const int64_t idx = base + i;
      v[i] = (idx < n) ? (Tout)in[idx] : Tout(0);
      sum += v[i];
    }
    Tout tot;
    Tout run = block_exclusive_scan<Tout>(sum, sh, &tot) + carry;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
      const int64_t idx = base + i;
      if (idx < n) out[idx] = run;
      run += v[i];
      if (idx == n - 1) out[n] = run;
    }
    carry += tot;
  }
}

constexpr int64_t kScanOneBlockTiles = 4;  // up to here one launch beats three

template <class Tin, class Tout>
static void scan_impl(const Tin* in, Tout* out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    GP_CUDA(cudaMemsetAsync(out, 0, sizeof(Tout), s));
    return;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb <= kScanOneBlockTiles) {
    GP_LAUNCH(F_SCAN, (k_scan_one_block<Tin, Tout>), 1, kScanThreads, 0, s, in, n, out);
    GP_CHECK_LAUNCH();
    return;
  }
  Tout* partial = dnew<Tout>(nb, s);
  GP_LAUNCH(F_SCAN, (k_scan_reduce<Tin, Tout>), (unsigned)nb, kScanThreads, 0, s, in, n, partial);
  GP_LAUNCH(F_SCAN, (k_scan_partials<Tout>), 1, 1024, 0, s, partial, nb);
  GP_LAUNCH(F_SCAN, (k_scan_down<Tin, Tout>), (unsigned)nb, kScanThreads, 0, s, in, n, partial, out);
  GP_CHECK_LAUNCH();
  dfree(partial, s);
}

void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  scan_impl<int32_t, int64_t>(in, out, n, s);
}
void scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  scan_impl<int64_t, int64_t>(in, out, n, s);
}
void scan_u8_to_i32(const uint8_t* in, int32_t* out, int64_t n, cudaStream_t s) {
  scan_impl<uint8_t, int32_t>(in, out, n, s);
}

}  // namespace gp

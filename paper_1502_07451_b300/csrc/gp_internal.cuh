// gp_internal.cuh -- shared declarations of the CUDA implementation (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "../../include/gp.h"

namespace gp {

// ------------------------------------------------------------------------------------------------
// Fixed algorithm constants (they change results; the CPU oracle uses the same values).
// ------------------------------------------------------------------------------------------------
constexpr int kMatchRounds = 4;     // handshake rounds per coarsening level
constexpr int kCapDiv = 8;          // merged vertex weight <= bound / 8
constexpr int64_t kCoarsest = 128;  // stop coarsening at <= 128 vertices
constexpr int kStallNum = 95;       // stop when a matching keeps > 95/100 of the vertices
constexpr int kStallDen = 100;
constexpr int kMaxLevels = GP_MAX_LEVELS;
constexpr int kTrials = 8;          // greedy growing trials
constexpr int kRefineRounds = 8;    // gain rounds per level
constexpr int64_t kSumLimit = int64_t(1) << 61;
constexpr int64_t kMaxN = (int64_t(1) << 31) - 2;

// ------------------------------------------------------------------------------------------------
// Kernel families (profiling / accounting ids).
// ------------------------------------------------------------------------------------------------
enum Family {
  F_VALIDATE = 0, F_TRANSPOSE, F_LEVELS, F_SYM_MERGE, F_MATCH_PICK, F_MATCH_CONFIRM, F_TWOHOP,
  F_CMAP, F_CONTRACT_MERGE, F_SCAN, F_GGGP, F_GAIN, F_SELECT, F_APPLY, F_PROJECT, F_MAKESPAN,
  F_CUT, F_MISC, F_BATCH, F_MPNN, F_PROPOSE, F_REFINE, F_LISTSCHED, F_COUNT
};
extern const char* const kFamilyName[F_COUNT];

// ------------------------------------------------------------------------------------------------
// Checked build (-DGP_CHECKED, libgp_checked.so): every data-dependent index the kernels gather with
// (neighbour ids, match partners, coarse ids, level positions) is tested against its range before the
// access; a failing test records the check's site number in a device word (the first one wins) and the
// access is skipped, so a corrupt input turns into a recorded site instead of an out-of-range access.
// Without GP_CHECKED the test is the constant `true` and compiles away.
// ------------------------------------------------------------------------------------------------
#ifdef GP_CHECKED
__device__ int d_check_site;
__device__ __forceinline__ bool gp_in_range(int64_t i, int64_t n, int site) {
  if ((uint64_t)i < (uint64_t)n) return true;
  atomicCAS(&d_check_site, 0, site);
  return false;
}
#define GP_IN(i, n, site) ::gp::gp_in_range((int64_t)(i), (int64_t)(n), (site))
#else
#define GP_IN(i, n, site) true
#endif

// Device counters of algorithmic bytes per family (added by kernels, one atomic per block).  The
// library is a single translation unit, so the definition lives here.
__device__ unsigned long long d_alg_bytes[F_COUNT];

// ------------------------------------------------------------------------------------------------
// Launch bookkeeping (host).
// ------------------------------------------------------------------------------------------------
void launch_begin(int family, cudaStream_t s);
void launch_end(int family, cudaStream_t s);
bool prof_on();

#define GP_LAUNCH(fam, kern, grid, block, smem, stream, ...)                  \
  do {                                                                        \
    ::gp::launch_begin((fam), (stream));                                      \
    kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                 \
    ::gp::launch_end((fam), (stream));                                        \
  } while (0)


// ------------------------------------------------------------------------------------------------
// Error helpers.
// ------------------------------------------------------------------------------------------------
struct Fail {
  gp_status st;
};
#define GP_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      if (e_ == cudaErrorMemoryAllocation) throw ::gp::Fail{GP_ERR_OOM}; \
      throw ::gp::Fail{GP_ERR_CUDA};                   \
    }                                                  \
  } while (0)
#define GP_CHECK_LAUNCH() GP_CUDA(cudaGetLastError())

// stream-ordered allocation from the device pool
void* dalloc(size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);
template <class T>
T* dnew(int64_t count, cudaStream_t s) {
  return (T*)dalloc(sizeof(T) * (size_t)(count > 0 ? count : 1), s);
}

int num_sms();
int device_id();

// Blocks of a grid-stride kernel whose scattered accesses (atomics and stores at data-dependent
// positions) cover `scatter_bytes`: when those are larger than half of the L2, at most as many blocks
// as fit on the device at once, so that the grid's passes cover the index range once, in order, and
// the positions a stretch of it scatters to stay in L2 while it is written (a larger grid runs in
// waves, each sweeping the whole range again after the previous wave's lines were evicted); else
// grid_for's bound (more blocks than fit: later blocks balance the load).  resident_blocks: blocks
// per SM of `kern` at `threads` threads (occupancy query, cached); l2_bytes: the device's L2 size.
int resident_blocks(const void* kern, int threads, size_t smem);
int64_t l2_bytes();
inline unsigned grid_scatter(const void* kern, int64_t work, int per_block, int threads, int64_t scatter_bytes,
                             int max_per_sm = 16) {
  const int64_t want = (work + per_block - 1) / per_block;
  const int64_t per_sm = scatter_bytes > l2_bytes() / 2 ? resident_blocks(kern, threads, 0) : max_per_sm;
  const int64_t cap = (int64_t)num_sms() * per_sm;
  return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

// ------------------------------------------------------------------------------------------------
// Device helpers.
// ------------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
// tie-break hash of the unordered pair {a, b}, a = smaller id
__host__ __device__ __forceinline__ uint64_t pair_hash(uint64_t seed, uint32_t a, uint32_t b) {
  return mix64(seed ^ mix64(((uint64_t)a << 32) | (uint64_t)b));
}

// Edge key of the matching order: larger W first, then larger hash, then smaller (min, max).
// `nm` holds ~((min << 32) | max) so that every component is "larger is better".
struct EdgeKey {
  int64_t W;
  uint64_t h;
  uint64_t nm;
};
__device__ __forceinline__ bool key_better(const EdgeKey& x, const EdgeKey& y) {
  if (x.W != y.W) return x.W > y.W;
  if (x.h != y.h) return x.h > y.h;
  return x.nm > y.nm;
}
__device__ __forceinline__ EdgeKey key_none() { return EdgeKey{-1, 0, 0}; }
__device__ __forceinline__ EdgeKey make_key(int64_t W, uint64_t seed, uint32_t v, uint32_t u) {
  const uint32_t mn = v < u ? v : u, mx = v < u ? u : v;
  return EdgeKey{W, pair_hash(seed, mn, mx), ~(((uint64_t)mn << 32) | (uint64_t)mx)};
}
__device__ __forceinline__ int32_t key_other(const EdgeKey& k, uint32_t v) {
  const uint64_t mm = ~k.nm;
  const uint32_t mn = (uint32_t)(mm >> 32), mx = (uint32_t)mm;
  return (int32_t)(mn == v ? mx : mn);
}
__device__ __forceinline__ EdgeKey warp_best_key(EdgeKey k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    EdgeKey q;
    q.W = __shfl_xor_sync(0xffffffffu, k.W, o);
    q.h = __shfl_xor_sync(0xffffffffu, k.h, o);
    q.nm = __shfl_xor_sync(0xffffffffu, k.nm, o);
    if (key_better(q, k)) k = q;
  }
  return k;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ unsigned long long warp_sumu64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block-wide sum (all threads get the result).  `sh` needs 32 slots.
template <class T>
__device__ __forceinline__ T block_sum(T x, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

// accounting: add bytes to a family's counter once per block
__device__ __forceinline__ void account(int fam, unsigned long long bytes_this_thread,
                                        unsigned long long* sh) {
  unsigned long long s = block_sum<unsigned long long>(bytes_this_thread, sh);
  if (threadIdx.x == 0 && s) atomicAdd(&d_alg_bytes[fam], s);
}

// ------------------------------------------------------------------------------------------------
// Thread-block clusters.  Level-synchronous loops (topological levels, makespan) run in ONE cluster
// of up to 16 CTAs x 1024 threads and separate levels with the hardware cluster barrier; data that
// other CTAs wrote before the barrier is read with L2-only loads (__ldcg).
// ------------------------------------------------------------------------------------------------
// Bulk L2 prefetch of [p, p + bytes) spread over the threads of the grid (16-byte aligned chunks of
// up to 64 KiB; the unaligned head and tail are left to demand loads).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t a0 = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  const uintptr_t a1 = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  if (a1 <= a0) return;
  constexpr uintptr_t kChunk = 65536;
  const uintptr_t nch = (a1 - a0 + kChunk - 1) / kChunk;
  const uintptr_t tid = (uintptr_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uintptr_t nt = (uintptr_t)gridDim.x * blockDim.x;
  for (uintptr_t c = tid; c < nch; c += nt) {
    const uintptr_t s = a0 + c * kChunk;
    const uintptr_t e = (s + kChunk < a1) ? s + kChunk : a1;
    const unsigned sz = (unsigned)(e - s);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"(sz) : "memory");
  }
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;\n" ::: "memory");
}
// Split form: work placed between arrive and wait overlaps the barrier.  The release waits for the
// thread's earlier memory operations, so loads issued after the arrive do not delay it.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory"); }

// Largest cluster (16 if the device allows non-portable sizes, else 8) that can be resident for
// `fn` with `block` threads per CTA; 0 if none.
int cluster_max(const void* fn, int block, size_t smem);

template <typename... KArgs, typename... Args>
cudaError_t launch_cluster(int family, void (*kern)(KArgs...), int csize, int block, size_t smem, cudaStream_t s,
                           Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)csize);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  launch_begin(family, s);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
  launch_end(family, s);
  return e;
}

// ------------------------------------------------------------------------------------------------
// Level graph in padded CSR: row v occupies [start[v], start[v] + deg[v]) of adj / W.
// ------------------------------------------------------------------------------------------------
struct LevelGraph {
  int64_t n = 0;
  int64_t cap = 0;       // capacity of adj / W
  int64_t a = 0;         // entries held (0: not known, cap is used as the estimate)
  int64_t* start = nullptr;
  int32_t* deg = nullptr;
  int32_t* adj = nullptr;
  int64_t* W = nullptr;
  int64_t* vC = nullptr;
  int64_t* vG = nullptr;
  int8_t* fix = nullptr;  // fixed vertices: 0 pinned to the CPU, 1 to the GPU, -1 free; null: none
};

// ------------------------------------------------------------------------------------------------
// Host launchers (implemented in the k_*.cu files).
// ------------------------------------------------------------------------------------------------

// scans: exclusive prefix sum of in[0..n) into out[0..n], out[n] = total.  `total_host` may be NULL.
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
void scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
void scan_u8_to_i32(const uint8_t* in, int32_t* out, int64_t n, cudaStream_t s);

// row merge: for every row r of a "two-source" description, gather entries, map columns,
// drop column == self_col(r), sort by column, add up equal columns, write at out_start[r].
struct TwoSrc {
  // row r takes entries from segment A = [a_beg[ra], a_beg[ra] + a_len(ra)) and optionally
  // segment B, mapping column c -> map[c] when map != NULL.
  const int64_t* a_start;  // per source row start
  const int32_t* a_deg;    // per source row length (NULL: a_start[r+1] - a_start[r])
  const int32_t* a_col;
  const int32_t* a_w32;    // weights int32 (or NULL)
  const int64_t* a_w64;    // weights int64 (or NULL)
  const int64_t* b_start;
  const int32_t* b_deg;
  const int32_t* b_col;
  const int32_t* b_w32;
  const int64_t* b_w64;
  const int32_t* row_a;    // source row of segment A for output row r (NULL: r)
  const int32_t* row_b;    // source row of segment B (NULL: r); -1 = none
  const int32_t* map;      // column map (NULL: identity)
  int32_t drop_self;       // drop mapped column == r
  int64_t map_n;           // entries of `map` (checked build: the ids it is indexed with; 0 = unknown)
};
// Writes deg_out[r] and the merged row at out_start[r] (capacity = raw length).
// raw_bound >= total raw entries (sizes the scratch of the long-row tier).
void merge_rows(const TwoSrc& src, int64_t nrows, int64_t ncols, const int64_t* out_start,
                int32_t* deg_out, int32_t* adj_out, int64_t* W_out, int family, int64_t raw_bound,
                cudaStream_t s);

// coarsening
void match_level(const LevelGraph& g, int64_t capC, int64_t capG, uint64_t seed, int rounds,
                 bool twohop, int32_t* mate, cudaStream_t s);
// rep flags + scan: cmap (partial) and number of coarse vertices written to *nc_dev
void coarse_count(const LevelGraph& g, const int32_t* mate, int32_t* cmap, int64_t* nc_dev, cudaStream_t s);
// fill the coarse level (requires cg.n set and arrays allocated with cg.cap = g's entry total)
void contract_level(const LevelGraph& g, const int32_t* mate, int32_t* cmap, LevelGraph& cg,
                    cudaStream_t s);

// initial split
void gggp(const LevelGraph& g, int64_t BC, int64_t BG, int64_t SG, uint64_t seed, uint8_t* part,
          int32_t* trial_dev, cudaStream_t s);
void gggp_grow_one(const LevelGraph& g, int64_t BC, int64_t BG, int64_t start, uint8_t* part,
                   int64_t* cut_dev, cudaStream_t s);

void project(int64_t n, const int32_t* cmap, const uint8_t* part_c, uint8_t* part_f, cudaStream_t s);

}  // namespace gp

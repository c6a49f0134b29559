// gp_api.cu -- the C-ABI (include/gp.h) of the B300 multilevel CPU/GPU bipartitioner.
// Single translation unit: the kernel headers are included here.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <vector>

#include "gp_internal.cuh"
#include "k_scan.cuh"
#include "k_rows.cuh"
#include "k_graph.cuh"
#include "k_coarsen.cuh"
#include "k_initial.cuh"
#include "k_refine.cuh"
#include "k_makespan.cuh"
#include "k_batch.cuh"
#include "k_umma.cuh"
#include "k_mpnn.cuh"
#include "k_propose.cuh"
#include "k_create.cuh"
#include "k_listsched.cuh"

namespace gp {

const char* const kFamilyName[F_COUNT] = {
    "validate", "transpose", "levels", "sym_merge", "match_pick", "match_confirm", "twohop", "cmap",
    "contract_merge", "scan", "gggp", "gain", "select", "apply", "project", "makespan", "cut", "misc", "batch", "mpnn", "propose", "refine", "listsched"};

// ------------------------------------------------------------------------------------------------
// launch accounting and optional per-launch event timing
// ------------------------------------------------------------------------------------------------
static std::atomic<long long> g_launches{0};
static std::atomic<int> g_prof{0};
struct EvRec {
  int fam;
  cudaEvent_t a, b;
};
static std::mutex g_ev_mu;
static std::vector<EvRec> g_ev;
static std::vector<cudaEvent_t> g_ev_pool;
static thread_local cudaEvent_t t_pending = nullptr;
static double g_fam_ms[F_COUNT];
static long long g_fam_launches[F_COUNT];

static cudaEvent_t ev_get() {
  std::lock_guard<std::mutex> lk(g_ev_mu);
  if (!g_ev_pool.empty()) {
    cudaEvent_t e = g_ev_pool.back();
    g_ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

bool prof_on() { return g_prof.load() != 0; }

void launch_begin(int family, cudaStream_t s) {
  g_launches.fetch_add(1);
  if (prof_on()) {
    t_pending = ev_get();
    if (t_pending) cudaEventRecord(t_pending, s);
  }
  (void)family;
}

void launch_end(int family, cudaStream_t s) {
  if (prof_on() && t_pending) {
    cudaEvent_t b = ev_get();
    if (b) {
      cudaEventRecord(b, s);
      std::lock_guard<std::mutex> lk(g_ev_mu);
      g_ev.push_back(EvRec{family, t_pending, b});
    }
    t_pending = nullptr;
  }
}

static void prof_collect() {
  std::lock_guard<std::mutex> lk(g_ev_mu);
  for (auto& r : g_ev) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g_fam_ms[r.fam] += ms;
      g_fam_launches[r.fam] += 1;
    }
    g_ev_pool.push_back(r.a);
    g_ev_pool.push_back(r.b);
  }
  g_ev.clear();
}

int cluster_max(const void* fn, int block, size_t smem) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, int>> cache;  // ((fn, device), size)
  const int dev = device_id();
  std::lock_guard<std::mutex> lk(mu);
  for (auto& c : cache)
    if (c.first.first == fn && c.first.second == dev) return c.second;
  int best = 0;
  for (int cs : {16, 8, 4, 2, 1}) {
    if (cs > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters >= 1) {
      best = cs;
      break;
    }
    cudaGetLastError();
  }
  cache.push_back({{fn, dev}, best});
  if (getenv("GP_LOG")) fprintf(stderr, "[gp] cluster size %d for %p (block %d, smem %zu)\n", best, fn, block, smem);
  return best;
}

// ------------------------------------------------------------------------------------------------
// device memory: the current device's stream-ordered pool, kept cached across calls
// ------------------------------------------------------------------------------------------------
static std::mutex g_dev_mu;
static bool g_pool_set[64];
static int g_sms[64];

int device_id() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

int num_sms() {
  const int d = device_id();
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (d >= 0 && d < 64 && g_sms[d] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    g_sms[d] = v > 0 ? v : 1;
  }
  return (d >= 0 && d < 64) ? g_sms[d] : 1;
}

int64_t l2_bytes() {
  static int64_t v[64];
  const int d = device_id();
  if (d < 0 || d >= 64) return (int64_t)1 << 62;
  if (v[d] == 0) {
    int b = 0;
    cudaDeviceGetAttribute(&b, cudaDevAttrL2CacheSize, d);
    v[d] = b > 0 ? b : ((int64_t)1 << 62);
  }
  return v[d];
}

int resident_blocks(const void* kern, int threads, size_t smem) {
  struct Key {
    const void* k;
    int t;
    size_t m;
    int d;
  };
  static std::vector<std::pair<Key, int>> cache;
  static std::mutex mu;
  const int d = device_id();
  std::lock_guard<std::mutex> lk(mu);
  for (auto& e : cache)
    if (e.first.k == kern && e.first.t == threads && e.first.m == smem && e.first.d == d) return e.second;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  cache.push_back({{kern, threads, smem, d}, occ});
  return occ;
}

static void pool_setup() {
  const int d = device_id();
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (d < 0 || d >= 64 || g_pool_set[d]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  g_pool_set[d] = true;
}

// Host-side fault injection for the error paths (nothing is done to the GPU): GP_FAULT=oom makes every
// device allocation fail as out of memory, GP_FAULT=cuda as a failed runtime call, and GP_FAULT=timeout
// makes the partition report an expired device wait after its kernels completed normally.
static bool fault_is(const char* what) {
  const char* f = getenv("GP_FAULT");
  return f && strcmp(f, what) == 0;
}

void* dalloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (fault_is("oom")) throw Fail{GP_ERR_OOM};
  if (fault_is("cuda")) throw Fail{GP_ERR_CUDA};
  GP_CUDA(cudaMallocAsync(&p, bytes ? bytes : 1, s));
  return p;
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// per-call allocations released at scope exit (stream-ordered)
struct Arena {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Arena(cudaStream_t st) : s(st) {}
  template <class T>
  T* get(int64_t count) {
    T* p = dnew<T>(count, s);
    ptrs.push_back(p);
    return p;
  }
  ~Arena() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

// A second stream forked from `s` (it starts after everything already queued on `s`); join() makes
// `s` wait for it, and the destructor joins too, so that frees queued on `s` afterwards (error paths
// included) come after the side stream's work.  One side stream per device, created on first use.
struct StreamFork {
  cudaStream_t main, side = nullptr;
  cudaEvent_t ev = nullptr;
  bool joined = false;
  explicit StreamFork(cudaStream_t s) : main(s) {
    static std::mutex mu;
    static cudaStream_t streams[64];
    const int d = device_id();
    {
      std::lock_guard<std::mutex> lk(mu);
      if (d >= 0 && d < 64 && !streams[d]) cudaStreamCreateWithFlags(&streams[d], cudaStreamNonBlocking);
      side = (d >= 0 && d < 64) ? streams[d] : nullptr;
    }
    if (!side || cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      side = main;  // no second stream: run in order
      ev = nullptr;
      return;
    }
    cudaEventRecord(ev, main);
    cudaStreamWaitEvent(side, ev, 0);
  }
  void join() {
    if (joined) return;
    joined = true;
    if (!ev) return;
    cudaEventRecord(ev, side);
    cudaStreamWaitEvent(main, ev, 0);
  }
  void detach() { joined = true; }  // the side stream's work goes on; the main stream does not wait
  ~StreamFork() {
    join();
    if (ev) cudaEventDestroy(ev);
  }
};

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static gp_status host_bounds(int64_t SC, int64_t SG, double r_cpu, double tol, int64_t* BC, int64_t* BG) {
  if (!(tol >= 0.0 && tol <= 1.0)) return GP_ERR_INVALID;
  if (std::isnan(r_cpu) || r_cpu > 1.0) return GP_ERR_INVALID;
  if (SC < 0 || SG < 0) return GP_ERR_INVALID;
  const __int128 ppm = (__int128)llround(tol * 1e6);
  const __int128 scale = (__int128)1000000 + ppm;
  if (r_cpu < 0.0) {
    const __int128 den = (__int128)SC + (__int128)SG;
    const __int128 t = den == 0 ? 0 : ((__int128)SC * (__int128)SG) / den;
    *BC = (int64_t)((t * scale) / 1000000);
    *BG = *BC;
  } else {
    const __int128 rq = (__int128)llround(r_cpu * 4294967296.0);
    const __int128 tc = ((__int128)SC * rq) >> 32;
    const __int128 tg = ((__int128)SG * (((__int128)1 << 32) - rq)) >> 32;
    *BC = (int64_t)((tc * scale) / 1000000);
    *BG = (int64_t)((tg * scale) / 1000000);
  }
  return GP_OK;
}

static int makespan_group(int64_t n, int64_t m) {
  const double avg = n > 0 ? (double)m / (double)n : 0.0;
  if (avg <= 3.0) return 2;
  if (avg <= 6.0) return 4;
  if (avg <= 12.0) return 8;
  if (avg <= 24.0) return 16;
  return 32;
}

// the cut of a mapping over the directed out-CSR (G lanes per row from the average out-degree)
static void launch_cut(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                       const uint8_t* part, unsigned long long* cut, int* bad, cudaStream_t s) {
  if (n <= 0) return;
  switch (makespan_group(n, m)) {
#define GP_CUTG(GG) \
  case GG: GP_LAUNCH(F_CUT, k_cut<GG>, grid_for(n * GG, 256), 256, 0, s, n, off, cols, w, part, cut, bad); break;
    GP_CUTG(2) GP_CUTG(4) GP_CUTG(8) GP_CUTG(16) GP_CUTG(32)
#undef GP_CUTG
  }
}

}  // namespace gp

using namespace gp;

struct gp_graph {
  int dev = 0;
  int64_t n = 0, m = 0, a0 = 0;
  int32_t nlev = 0;
  int64_t SC = 0, SG = 0;
  int64_t max_width = 0;
  int64_t* off = nullptr;
  int32_t* cols = nullptr;
  int32_t* w = nullptr;
  int32_t* cC = nullptr;
  int32_t* cG = nullptr;
  int64_t* lev_ptr = nullptr;
  int32_t* lev_vtx = nullptr;
  int32_t* level = nullptr;
  int64_t* lo_off = nullptr;
  int32_t* lo_src = nullptr;
  int32_t* lo_w = nullptr;
  int32_t* lo_cC = nullptr;
  int32_t* lo_cG = nullptr;
  int64_t* in_off = nullptr;  // vertex-indexed in-CSR (entries in no particular order within a row)
  int32_t* in_src = nullptr;
  int32_t* in_w = nullptr;
  bool in_sorted = false;     // in-rows sorted by (source, cost): set before the network first reads them
  // deferred levels (gp_graph_create_deferred): the level traversal and the level-ordered in-CSR run on
  // a side stream after creation returns; lev_event marks their end, lev_host receives {vertices
  // placed, levels, widest level}, and levels_ready() waits for them once
  bool lev_pending = false;
  gp_status lev_status = GP_OK;
  cudaEvent_t lev_event = nullptr;
  int64_t* lev_host = nullptr;  // pinned slot of 4 int64
  std::mutex lev_mu;
  std::shared_ptr<void> block;  // device block shared by the handles of one gp_graph_create_batch call
  LevelGraph L0;
  gp_trace trace;
  std::vector<void*> owned;
  template <class T>
  T* own(int64_t count, cudaStream_t s) {
    T* p = dnew<T>(count, s);
    owned.push_back(p);
    return p;
  }
};

// Pinned host slots of 4 int64 (carved from 64 KiB pinned chunks, recycled): targets of the deferred
// level results' device-to-host copies, so that creating a graph allocates no pinned memory.
static std::mutex g_slot_mu;
static std::vector<int64_t*> g_slot_free;
static int64_t* pinned_slot_alloc() {
  std::lock_guard<std::mutex> lk(g_slot_mu);
  if (g_slot_free.empty()) {
    void* chunk = nullptr;
    if (cudaMallocHost(&chunk, 65536) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int i = 0; i < 65536 / 32; i++) g_slot_free.push_back((int64_t*)chunk + 4 * i);
  }
  int64_t* p = g_slot_free.back();
  g_slot_free.pop_back();
  return p;
}
static void pinned_slot_free(int64_t* p) {
  std::lock_guard<std::mutex> lk(g_slot_mu);
  g_slot_free.push_back(p);
}

// Waits (once) for a deferred creation's level work and takes its results: GP_ERR_NOT_DAG when the
// traversal placed fewer than n vertices (a cycle).  A no-op for a graph created without deferral.
static gp_status levels_ready(const gp_graph* cg) {
  gp_graph* g = const_cast<gp_graph*>(cg);
  std::lock_guard<std::mutex> lk(g->lev_mu);
  if (!g->lev_pending) return g->lev_status;
  if (cudaEventSynchronize(g->lev_event) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  g->nlev = (int32_t)g->lev_host[1];
  g->max_width = g->lev_host[2];
  g->lev_status = g->lev_host[0] == g->n ? GP_OK : GP_ERR_NOT_DAG;
  g->lev_pending = false;
  return g->lev_status;
}

static void graph_free(gp_graph* g) {
  if (!g) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(g->dev);
  cudaDeviceSynchronize();  // includes deferred level work on the side stream
  if (g->lev_event) cudaEventDestroy(g->lev_event);
  if (g->lev_host) pinned_slot_free(g->lev_host);
  for (void* p : g->owned) cudaFree(p);
  g->block.reset();  // the shared block is freed with its last handle
  cudaSetDevice(cur);
  delete g;
}

// The makespan kernel in one cluster sized to the widest level (G lanes per vertex): the
// distributed-shared-memory ring variant when two adjacent levels fit its ring, else (or when
// GP_MAKESPAN_KERNEL=cluster) the variant that reads every predecessor from global memory.
static cudaError_t launch_makespan(const gp_graph* g, const uint8_t* part, unsigned long long* fp,
                                   unsigned long long* ms, int* bad, int64_t* fin, cudaStream_t s,
                                   unsigned* grid_bar = nullptr) {
  const int G = makespan_group(g->n, g->m);
  const int32_t nlev = g->nlev;
  const char* forced = getenv("GP_MAKESPAN_KERNEL");
  const bool small_ids = g->m < ((int64_t)1 << 31) && g->n < ((int64_t)1 << 31);
  const bool dsm = g->max_width <= kMsR && small_ids && !(forced && strcmp(forced, "cluster") == 0);
  // levels wider than a cluster's groups: one cooperative grid (grid_bar: a zeroed counter)
  const bool grid = !dsm && small_ids && grid_bar && (int64_t)g->max_width * G > 16 * 1024 &&
                    !(forced && strcmp(forced, "cluster") == 0);
  if (grid) {
    int coop = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (coop) {
      switch (G) {
#define GP_MSG(GG)                                                                                     \
  case GG: {                                                                                           \
    int per_sm = 0;                                                                                    \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_makespan_grid<GG>, 1024, 0) != cudaSuccess || \
        per_sm < 1)                                                                                    \
      break;                                                                                           \
    const int64_t want = ((int64_t)g->max_width * GG + 1023) / 1024;                                   \
    const int64_t cap = (int64_t)num_sms() * per_sm;                                                   \
    const unsigned blocks = (unsigned)(want < cap ? want : cap);                                       \
    const int64_t* a0 = (const int64_t*)g->lev_ptr;                                                    \
    const int32_t* a1 = (const int32_t*)g->lev_vtx;                                                    \
    const int64_t* a2 = (const int64_t*)g->lo_off;                                                     \
    const int32_t* a3 = (const int32_t*)g->lo_src;                                                     \
    const int32_t* a4 = (const int32_t*)g->lo_w;                                                       \
    const int32_t* a5 = (const int32_t*)g->lo_cC;                                                      \
    const int32_t* a6 = (const int32_t*)g->lo_cG;                                                      \
    int32_t nl = nlev;                                                                                 \
    void* args[] = {&nl, (void*)&a0, (void*)&a1, (void*)&a2, (void*)&a3, (void*)&a4, (void*)&a5, (void*)&a6, \
                    (void*)&part, (void*)&fp, (void*)&ms, (void*)&bad, (void*)&fin, (void*)&grid_bar};    \
    launch_begin(F_MAKESPAN, s);                                                                       \
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_makespan_grid<GG>, dim3(blocks),  \
                                                      dim3(1024), args, 0, s);                         \
    launch_end(F_MAKESPAN, s);                                                                         \
    return e;                                                                                          \
  }
        GP_MSG(2) GP_MSG(4) GP_MSG(8) GP_MSG(16) GP_MSG(32)
#undef GP_MSG
      }
    }
  }
  switch (G) {
#define GP_MS(GG)                                                                                      \
  case GG: {                                                                                           \
    if (dsm) {                                                                                         \
      const cudaError_t e = cudaFuncSetAttribute(k_makespan_dsm<GG>,                                   \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMsRingBytes); \
      if (e != cudaSuccess) return e;                                                                  \
    }                                                                                                  \
    const int cmax = dsm ? cluster_max((const void*)k_makespan_dsm<GG>, 1024, kMsRingBytes)            \
                         : cluster_max((const void*)k_makespan<GG>, 1024, 0);                          \
    if (cmax <= 0) return cudaErrorLaunchFailure;                                                      \
    int64_t want = (g->max_width * GG + 1023) / 1024;                                                  \
    if (dsm && want > 8) want = 8; /* each value goes to every CTA: 8 measured fastest at 1,000-wide levels */ \
    const int cs = (int)(want < 1 ? 1 : (want < cmax ? want : cmax));                                  \
    if (dsm)                                                                                           \
      return launch_cluster(F_MAKESPAN, k_makespan_dsm<GG>, cs, 1024, kMsRingBytes, s, nlev,           \
                            (const int64_t*)g->lev_ptr, (const int32_t*)g->lev_vtx, (const int64_t*)g->lo_off, \
                            (const int32_t*)g->lo_src, (const int32_t*)g->lo_w, (const int32_t*)g->lo_cC, \
                            (const int32_t*)g->lo_cG, part, fp, ms, bad, fin);                         \
    return launch_cluster(F_MAKESPAN, k_makespan<GG>, cs, 1024, 0, s, nlev, (const int64_t*)g->lev_ptr, \
                          (const int32_t*)g->lev_vtx, (const int64_t*)g->lo_off, (const int32_t*)g->lo_src, \
                          (const int32_t*)g->lo_w, (const int32_t*)g->lo_cC, (const int32_t*)g->lo_cG, part, \
                          fp, ms, bad, fin);                                                           \
  }
    GP_MS(2) GP_MS(4) GP_MS(8) GP_MS(16) GP_MS(32)
#undef GP_MS
  }
  return cudaErrorInvalidValue;
}

extern "C" {

const char* gp_status_string(gp_status s) {
  switch (s) {
    case GP_OK: return "ok";
    case GP_ERR_INVALID: return "invalid argument or malformed graph";
    case GP_ERR_NOT_DAG: return "graph has a cycle";
    case GP_ERR_OOM: return "out of memory";
    case GP_ERR_CUDA: return "CUDA error";
    case GP_ERR_TIMEOUT: return "device wait timed out";
    case GP_ERR_OVERFLOW: return "summed cost exceeds 2^61";
  }
  return "unknown status";
}

int64_t gp_launch_count(void) { return (int64_t)g_launches.load(); }

gp_status gp_prof_enable(int on) {
  g_prof.store(on ? 1 : 0);
  return GP_OK;
}

gp_status gp_prof_reset(void) {
  prof_collect();
  for (int i = 0; i < F_COUNT; i++) {
    g_fam_ms[i] = 0;
    g_fam_launches[i] = 0;
  }
  unsigned long long z[F_COUNT] = {0};
  if (cudaMemcpyToSymbol(d_alg_bytes, z, sizeof(z)) != cudaSuccess) return GP_ERR_CUDA;
  return GP_OK;
}

gp_status gp_prof_read(int kernel, int64_t* launches, double* total_ms, int64_t* alg_bytes) {
  if (kernel < 0 || kernel >= F_COUNT) return GP_ERR_INVALID;
  prof_collect();
  unsigned long long b[F_COUNT];
  if (cudaMemcpyFromSymbol(b, d_alg_bytes, sizeof(b)) != cudaSuccess) return GP_ERR_CUDA;
  if (launches) *launches = g_fam_launches[kernel];
  if (total_ms) *total_ms = g_fam_ms[kernel];
  if (alg_bytes) *alg_bytes = (int64_t)b[kernel];
  return GP_OK;
}

const char* gp_kernel_name(int kernel) {
  if (kernel < 0 || kernel >= F_COUNT) return nullptr;
  return kFamilyName[kernel];
}

gp_status gp_bounds(int64_t sum_cpu, int64_t sum_gpu, double r_cpu, double tol, int64_t* bound_cpu,
                    int64_t* bound_gpu) {
  if (!bound_cpu || !bound_gpu) return GP_ERR_INVALID;
  return host_bounds(sum_cpu, sum_gpu, r_cpu, tol, bound_cpu, bound_gpu);
}

}  // extern "C"

// Graph creation.  deferred: the level traversal and the level-ordered in-CSR run on the side stream
// and creation returns once the symmetrised graph is built (levels_ready() collects them).
static gp_status graph_create(int64_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                              const int32_t* edge_cost, const int32_t* cpu_cost, const int32_t* gpu_cost,
                              int ptr_kind, void* stream, gp_graph** out, bool deferred) {
  if (!out) return GP_ERR_INVALID;
  *out = nullptr;
  if (n < 0 || m < 0 || n > kMaxN || (ptr_kind != 0 && ptr_kind != 1)) return GP_ERR_INVALID;
  if (!offsets || (m > 0 && (!cols || !edge_cost)) || (n > 0 && (!cpu_cost || !gpu_cost))) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  gp_graph* g = new gp_graph();
  try {
    pool_setup();
    g->dev = device_id();
    g->n = n;
    g->m = m;
    memset(&g->trace, 0, sizeof(g->trace));
    g->off = g->own<int64_t>(n + 1, s);
    g->cols = g->own<int32_t>(m, s);
    g->w = g->own<int32_t>(m, s);
    g->cC = g->own<int32_t>(n, s);
    g->cG = g->own<int32_t>(n, s);
    const cudaMemcpyKind kind = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    GP_CUDA(cudaMemcpyAsync(g->off, offsets, sizeof(int64_t) * (n + 1), kind, s));
    if (m) {
      GP_CUDA(cudaMemcpyAsync(g->cols, cols, sizeof(int32_t) * m, kind, s));
      GP_CUDA(cudaMemcpyAsync(g->w, edge_cost, sizeof(int32_t) * m, kind, s));
    }
    if (n) {
      GP_CUDA(cudaMemcpyAsync(g->cC, cpu_cost, sizeof(int32_t) * n, kind, s));
      GP_CUDA(cudaMemcpyAsync(g->cG, gpu_cost, sizeof(int32_t) * n, kind, s));
    }
    Arena A(s);
    // ---- validation (sizes, ids, costs) and exact sums
    int* flags = A.get<int>(1);
    unsigned long long* sums = A.get<unsigned long long>(6);
    GP_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), s));
    GP_CUDA(cudaMemsetAsync(sums, 0, 6 * sizeof(unsigned long long), s));
    const int64_t vwork = n > m ? n : m;
    GP_LAUNCH(F_VALIDATE, k_validate, grid_for(vwork + 1, 256, 8), 256, 0, s, n, m, g->off, g->cols, g->w, g->cC,
              g->cG, flags, sums);
    GP_CHECK_LAUNCH();
    int hflags = 0;
    unsigned long long hs[6];
    GP_CUDA(cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (hflags & VF_INVALID) throw Fail{GP_ERR_INVALID};
    const unsigned __int128 sw = ((unsigned __int128)hs[1] << 64) | hs[0];
    const unsigned __int128 sc = ((unsigned __int128)hs[3] << 64) | hs[2];
    const unsigned __int128 sg = ((unsigned __int128)hs[5] << 64) | hs[4];
    if (sw > (unsigned __int128)kSumLimit || sc > (unsigned __int128)kSumLimit || sg > (unsigned __int128)kSumLimit)
      throw Fail{GP_ERR_OVERFLOW};
    g->SC = (int64_t)sc;
    g->SG = (int64_t)sg;
    // ---- transpose (in-CSR) and self-loop check
    int32_t* indeg = A.get<int32_t>(n);
    int64_t* in_off = g->in_off = g->own<int64_t>(n + 1, s);
    int32_t* in_src = g->in_src = g->own<int32_t>(m, s);
    int32_t* in_w = g->in_w = g->own<int32_t>(m, s);
    GP_CUDA(cudaMemsetAsync(indeg, 0, sizeof(int32_t) * (n > 0 ? n : 1), s));
    // grids of the scattering kernels: resident only, when their scatter targets exceed half the L2
    if (m)
      GP_LAUNCH(F_TRANSPOSE, k_indeg, grid_scatter((const void*)k_indeg, m, 256, 256, 4 * n, 8), 256, 0, s, m,
                g->cols, indeg);
    scan_i32_to_i64(indeg, in_off, n, s);
    GP_CUDA(cudaMemsetAsync(indeg, 0, sizeof(int32_t) * (n > 0 ? n : 1), s));  // reused as fill cursor
    unsigned long long* fill_next = A.get<unsigned long long>(1);
    GP_CUDA(cudaMemsetAsync(fill_next, 0, sizeof(unsigned long long), s));
    if (n) {
      switch (makespan_group(n, m)) {  // lanes per row from the average out-degree
#define GP_FI(GG)                                                                                           \
  case GG:                                                                                                  \
    GP_LAUNCH(F_TRANSPOSE, k_fill_in<GG>, grid_scatter((const void*)k_fill_in<GG>, n * GG, 256, 256, 8 * m + 4 * n), \
              256, 0, s, n, g->off, g->cols, g->w, in_off, indeg, in_src, in_w, flags, fill_next);          \
    break;
        GP_FI(2) GP_FI(4) GP_FI(8) GP_FI(16) GP_FI(32)
#undef GP_FI
      }
    }
    GP_CHECK_LAUNCH();
    // ---- symmetrisation: row v = out-row(v) + in-row(v), merged (Sec. III.B: one cost per transfer).
    // It needs only the two CSRs, so it runs on one stream while the level traversal (one cluster of
    // SMs) runs on another: the side stream takes the symmetrisation, or with deferral the levels.
    LevelGraph& L = g->L0;
    L.n = n;
    L.cap = 2 * m;
    L.start = g->own<int64_t>(n + 1, s);
    L.deg = g->own<int32_t>(n, s);
    L.adj = g->own<int32_t>(2 * m, s);
    L.W = g->own<int64_t>(2 * m, s);
    L.vC = g->own<int64_t>(n, s);
    L.vG = g->own<int64_t>(n, s);
    int64_t* rawlen = A.get<int64_t>(n);
    unsigned long long* a0 = A.get<unsigned long long>(1);
    GP_CUDA(cudaMemsetAsync(a0, 0, sizeof(unsigned long long), s));
    g->lev_vtx = g->own<int32_t>(n, s);
    g->lev_ptr = g->own<int64_t>(n + 2, s);
    g->level = g->own<int32_t>(n, s);
    g->lo_off = g->own<int64_t>(n + 1, s);
    g->lo_src = g->own<int32_t>(m, s);
    g->lo_w = g->own<int32_t>(m, s);
    g->lo_cC = g->own<int32_t>(n, s);
    g->lo_cG = g->own<int32_t>(n, s);
    if (deferred && n) {
      // unplaced positions of a cyclic graph must read as -1 in the level-ordered in-CSR build
      GP_CUDA(cudaMemsetAsync(g->lev_vtx, 0xff, sizeof(int32_t) * n, s));
      g->lev_host = pinned_slot_alloc();
      if (!g->lev_host || cudaEventCreateWithFlags(&g->lev_event, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        throw Fail{GP_ERR_CUDA};
      }
    }
    StreamFork fork(s);  // the side stream starts here, after everything above
    const cudaStream_t sl = deferred ? fork.side : s;  // the levels
    const cudaStream_t ss = deferred ? s : fork.side;  // the symmetrisation
    Arena AL(sl);  // temporaries of the level work, freed in its stream's order
    // ---- topological levels (Kahn: sources, then one CTA while levels are narrow, then one cluster)
    int32_t* rem = AL.get<int32_t>(n);
    unsigned long long* tail = AL.get<unsigned long long>(4);  // 3 rotating level counters + total
    int32_t* nlev_dev = AL.get<int32_t>(1);
    longlong2* frec = AL.get<longlong2>(n);
    GP_CUDA(cudaMemsetAsync(tail, 0, 4 * sizeof(unsigned long long), sl));
    GP_CUDA(cudaMemsetAsync(nlev_dev, 0, sizeof(int32_t), sl));
    int64_t* resume = AL.get<int64_t>(4);  // {level, begin, end, done} where the one-CTA kernel stopped
    GP_CUDA(cudaMemsetAsync(resume, 0, 4 * sizeof(int64_t), sl));
    if (n) {
      GP_LAUNCH(F_LEVELS, k_levels_init, grid_for(n, 256, 8), 256, 0, sl, n, (const int64_t*)g->off,
                (const int32_t*)g->cols, (const int64_t*)in_off, rem, g->lev_vtx, g->level, tail, frec);
      if (m < ((int64_t)1 << 31)) {
        // narrow levels in one CTA: it stops at the first level of more than ~1,300 out-entries (at the
        // average out-degree), where the cluster kernel's ~3.5 us per level becomes the cheaper one
        const double deg = (double)m / (double)n;
        int64_t mw = (int64_t)(1300.0 / (deg > 1.0 ? deg : 1.0));
        mw = mw < 32 ? 32 : (mw > 4096 ? 4096 : mw);
        GP_CUDA(cudaFuncSetAttribute(k_levels_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLevCtaSmem));
        GP_LAUNCH(F_LEVELS, k_levels_cta, 1, 1024, kLevCtaSmem, sl, n, (const int64_t*)g->off,
                  (const int32_t*)g->cols, rem, g->lev_vtx, g->lev_ptr, g->level, tail, nlev_dev, frec, resume, mw);
      }
      const int G = makespan_group(n, m);
      int ok = 0;
      switch (G) {
#define GP_LEV(GG)                                                                                       \
  case GG: {                                                                                            \
    const int cs = cluster_max((const void*)k_levels<GG>, 1024, 0);                                     \
    if (cs > 0) {                                                                                       \
      GP_CUDA(launch_cluster(F_LEVELS, k_levels<GG>, cs, 1024, 0, sl, (const int64_t*)g->off,            \
                             (const int32_t*)g->cols, rem, g->lev_vtx, g->lev_ptr, g->level, tail, nlev_dev, \
                             frec, (const int64_t*)resume));                                            \
      ok = 1;                                                                                           \
    }                                                                                                   \
  } break;
        GP_LEV(2) GP_LEV(4) GP_LEV(8) GP_LEV(16) GP_LEV(32)
#undef GP_LEV
      }
      if (!ok) throw Fail{GP_ERR_CUDA};
    }
    // the symmetrisation, beside the traversal
    if (n) {
      GP_LAUNCH(F_SYM_MERGE, k_rawlen_sym, grid_for(n, 256), 256, 0, ss, n, g->off, in_off, rawlen);
      GP_LAUNCH(F_MISC, k_widen, grid_for(n, 256), 256, 0, ss, n, g->cC, g->cG, L.vC, L.vG);
    }
    scan_i64(rawlen, L.start, n, ss);
    {
      TwoSrc src{};
      src.a_start = g->off;
      src.a_col = g->cols;
      src.a_w32 = g->w;
      src.b_start = in_off;
      src.b_col = in_src;
      src.b_w32 = in_w;
      src.drop_self = 0;
      merge_rows_unordered(src, n, n, L.start, L.deg, L.adj, L.W, F_SYM_MERGE, 2 * m, ss);
    }
    if (n) GP_LAUNCH(F_MISC, k_sum_deg, grid_for(n, 256, 8), 256, 0, ss, n, L.deg, a0);
    GP_CHECK_LAUNCH();
    // ---- level-ordered in-CSR for the makespan (after the traversal, on its stream); its inputs
    // are the traversal's positions, which exist whether or not the graph turns out acyclic
    auto lo_csr = [&]() {
      int32_t* pos_of = AL.get<int32_t>(n);
      int32_t* lo_deg = AL.get<int32_t>(n);
      if (n) GP_LAUNCH(F_TRANSPOSE, k_lo_prep, grid_for(n, 256), 256, 0, sl, n, g->lev_vtx, in_off, g->cC, g->cG,
                       pos_of, lo_deg, g->lo_cC, g->lo_cG);
      scan_i32_to_i64(lo_deg, g->lo_off, n, sl);
      if (n) {
        switch (makespan_group(n, m)) {  // lanes per position from the average in-degree
#define GP_LF(GG)                                                                                          \
  case GG:                                                                                                 \
    GP_LAUNCH(F_TRANSPOSE, k_lo_fill<GG>, grid_scatter((const void*)k_lo_fill<GG>, n * GG, 256, 256, 4 * n), 256, \
              0, sl, n, g->lev_vtx, in_off, in_src, in_w, pos_of, g->lo_off, g->lo_src, g->lo_w);          \
    break;
          GP_LF(2) GP_LF(4) GP_LF(8) GP_LF(16) GP_LF(32)
#undef GP_LF
        }
      }
    };
    if (!deferred) {
      unsigned long long htail = 0;
      int32_t hnlev = 0;
      GP_CUDA(cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaMemcpyAsync(&htail, tail + 3, sizeof(htail), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaMemcpyAsync(&hnlev, nlev_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaStreamSynchronize(s));
      if ((hflags & VF_SELFLOOP) || (n > 0 && (int64_t)htail != n)) throw Fail{GP_ERR_NOT_DAG};
      g->nlev = hnlev;
      {
        std::vector<int64_t> lp((size_t)hnlev + 1);
        if (n) GP_CUDA(cudaMemcpy(lp.data(), g->lev_ptr, sizeof(int64_t) * (hnlev + 1), cudaMemcpyDeviceToHost));
        int64_t mw = 0;
        for (int l = 0; l < hnlev; l++) mw = std::max(mw, lp[l + 1] - lp[l]);
        g->max_width = mw;
      }
      lo_csr();
      fork.join();  // the first stream waits for the symmetrisation
    } else if (n) {
      // the traversal's results, read by levels_ready(): vertices placed, levels, widest level
      lo_csr();
      int64_t* res3 = AL.get<int64_t>(3);
      GP_LAUNCH(F_MISC, k_level_summary, 1, 256, 0, sl, tail + 3, nlev_dev, (const int64_t*)g->lev_ptr, res3);
      GP_CUDA(cudaMemcpyAsync(g->lev_host, res3, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, sl));
      GP_CUDA(cudaEventRecord(g->lev_event, sl));
      g->lev_pending = true;
      fork.detach();
    }
    unsigned long long ha0 = 0;
    GP_CUDA(cudaMemcpyAsync(&ha0, a0, sizeof(ha0), cudaMemcpyDeviceToHost, s));
    if (deferred) GP_CUDA(cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (deferred && (hflags & VF_SELFLOOP)) throw Fail{GP_ERR_NOT_DAG};
    g->a0 = (int64_t)ha0;
    *out = g;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    graph_free(g);
    return f.st;
  }
}

extern "C" {

gp_status gp_graph_create(int64_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                          const int32_t* edge_cost, const int32_t* cpu_cost, const int32_t* gpu_cost,
                          int ptr_kind, void* stream, gp_graph** out) {
  return graph_create(n, m, offsets, cols, edge_cost, cpu_cost, gpu_cost, ptr_kind, stream, out, false);
}

gp_status gp_graph_create_deferred(int64_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                                   const int32_t* edge_cost, const int32_t* cpu_cost, const int32_t* gpu_cost,
                                   int ptr_kind, void* stream, gp_graph** out) {
  return graph_create(n, m, offsets, cols, edge_cost, cpu_cost, gpu_cost, ptr_kind, stream, out, true);
}

gp_status gp_graph_destroy(gp_graph* g) {
  if (!g) return GP_ERR_INVALID;
  graph_free(g);
  return GP_OK;
}

gp_status gp_graph_info(const gp_graph* g, int64_t* n, int64_t* m, int64_t* a0, int32_t* nlevels, int64_t* sum_cpu,
                        int64_t* sum_gpu) {
  if (!g) return GP_ERR_INVALID;
  if (nlevels) {
    const gp_status ls = levels_ready(g);
    if (ls != GP_OK) return ls;
  }
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (a0) *a0 = g->a0;
  if (nlevels) *nlevels = g->nlev;
  if (sum_cpu) *sum_cpu = g->SC;
  if (sum_gpu) *sum_gpu = g->SG;
  return GP_OK;
}

gp_status gp_graph_export(const gp_graph* g, int64_t* off, int32_t* adj, int64_t* W, int32_t* level, void* stream) {
  if (!g) return GP_ERR_INVALID;
  if (level) {
    const gp_status ls = levels_ready(g);
    if (ls != GP_OK) return ls;
  }
  cudaStream_t s = (cudaStream_t)stream;
  try {
    Arena A(s);
    const int64_t n = g->n;
    int64_t* coff = A.get<int64_t>(n + 1);
    int32_t* cadj = A.get<int32_t>(g->a0);
    int64_t* cW = A.get<int64_t>(g->a0);
    // level-0 rows are kept in no particular order; sort them (by neighbour) for the export
    int32_t* sdeg = A.get<int32_t>(n);
    int32_t* sadj = A.get<int32_t>(g->L0.cap);
    int64_t* sW = A.get<int64_t>(g->L0.cap);
    TwoSrc src{};
    src.a_start = g->L0.start;
    src.a_deg = g->L0.deg;
    src.a_col = g->L0.adj;
    src.a_w64 = g->L0.W;
    merge_rows(src, n, n, g->L0.start, sdeg, sadj, sW, F_MISC, g->L0.cap, s);
    scan_i32_to_i64(sdeg, coff, n, s);
    if (n) GP_LAUNCH(F_MISC, k_compact_rows, grid_for(n * 32, 256), 256, 0, s, n, g->L0.start, sdeg, sadj, sW, coff,
                     cadj, cW);
    GP_CHECK_LAUNCH();
    if (off) GP_CUDA(cudaMemcpyAsync(off, coff, sizeof(int64_t) * (n + 1), cudaMemcpyDefault, s));
    if (adj && g->a0) GP_CUDA(cudaMemcpyAsync(adj, cadj, sizeof(int32_t) * g->a0, cudaMemcpyDefault, s));
    if (W && g->a0) GP_CUDA(cudaMemcpyAsync(W, cW, sizeof(int64_t) * g->a0, cudaMemcpyDefault, s));
    if (level && n) GP_CUDA(cudaMemcpyAsync(level, g->level, sizeof(int32_t) * n, cudaMemcpyDefault, s));
    GP_CUDA(cudaStreamSynchronize(s));
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

// device-side per-level record of one partition call
struct TraceDev {
  int32_t rounds[kMaxLevels + 1];
  long long moves[kMaxLevels + 1];
  int32_t bal[kMaxLevels + 1];
  long long balmoves[kMaxLevels + 1];
  unsigned long long cut;
  unsigned long long a_last;
  int32_t trial;
  int32_t bad;
  Ctl ctl;
  unsigned grid_bar;  // arrivals at the grid refinement's barrier
  int32_t tail_err;   // a grid refinement barrier wait expired
};

// Coarse split of the V-cycle: every coarse vertex holds members of one proposed side (its pin).
__global__ void k_pins_to_part(int64_t n, const int8_t* __restrict__ pin, uint8_t* __restrict__ part,
                               int32_t* trial) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    part[i] = (uint8_t)pin[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) *trial = -1;
}

// The multilevel bipartitioner.  fixed: NULL, or one pin per vertex (host or device; -1 free, 0 CPU,
// 1 GPU).  restrict_only = false: the pins hold through every step (gp_partition_fixed).
// restrict_only = true (the learned V-cycle, every vertex pinned to its proposed side): the pins only
// keep the matching to same-side pairs; the coarsest level's split is its pins and refinement moves
// any vertex.
static gp_status partition_impl(gp_graph* g, const int8_t* fixed, double r_cpu, double tol, uint64_t seed,
                                uint8_t* part_out, gp_result* res, void* stream, bool restrict_only = false) {
  if (!g || (!part_out && g->n > 0)) return GP_ERR_INVALID;
  int64_t BC, BG;
  gp_status st = host_bounds(g->SC, g->SG, r_cpu, tol, &BC, &BG);
  if (st != GP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  gp_result R;
  memset(&R, 0, sizeof(R));
  R.bound_cpu = BC;
  R.bound_gpu = BG;
  gp_trace T;
  memset(&T, 0, sizeof(T));
  T.gggp_trial = -1;
  const int64_t n = g->n;
  if (n == 0) {
    R.feasible = 1;
    g->trace = T;
    if (res) *res = R;
    return GP_OK;
  }
  try {
    Arena A(s);
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    const bool prof = prof_on();
    if (prof)
      for (auto& e : ev) cudaEventCreate(&e);
    if (prof) cudaEventRecord(ev[0], s);
    std::vector<LevelGraph> L;
    std::vector<int32_t*> cmaps;
    L.push_back(g->L0);
    L[0].a = g->a0;
    T.n[0] = n;
    T.a[0] = g->a0;
    const int64_t capC = BC / kCapDiv, capG = BG / kCapDiv;
    TraceDev* td = A.get<TraceDev>(1);
    GP_CUDA(cudaMemsetAsync(td, 0, sizeof(TraceDev), s));
    // entries of each coarse level, summed on the device and read with the next level's vertex count
    // (one host round trip per level); until then a level's kernels size their lane groups from the
    // bound the fine level gives (c.cap), which changes no result
    unsigned long long* adev = A.get<unsigned long long>(kMaxLevels + 2);
    GP_CUDA(cudaMemsetAsync(adev, 0, sizeof(unsigned long long) * (kMaxLevels + 2), s));
    int64_t* hbuf = pinned_slot_alloc();  // [0]: the coarse vertex count (int32), [1]: entries
    if (!hbuf) throw Fail{GP_ERR_OOM};
    struct SlotGuard {
      int64_t* p;
      ~SlotGuard() { pinned_slot_free(p); }
    } slot_guard{hbuf};
    if (fixed) {  // pinned vertices: a device copy, checked before any level uses it
      int8_t* fx = A.get<int8_t>(n);
      int* bad = A.get<int>(1);
      GP_CUDA(cudaMemcpyAsync(fx, fixed, (size_t)n, cudaMemcpyDefault, s));
      GP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
      GP_LAUNCH(F_MISC, k_fix_check, grid_for(n, 256), 256, 0, s, n, (const int8_t*)fx, bad);
      GP_CUDA(cudaMemcpyAsync(hbuf, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaStreamSynchronize(s));
      if (*(int*)hbuf) throw Fail{GP_ERR_INVALID};
      L[0].fix = fx;
    }
    int lev = 0;
    auto take_entries = [&](int l) {  // level l's entries, copied to hbuf[1] before the last sync
      L[l].a = hbuf[1];
      T.a[l] = hbuf[1];
    };
    bool pending_a = false;  // L[lev].a still to be taken from hbuf[1]
    while (L[lev].n > kCoarsest && lev < kMaxLevels) {
      const LevelGraph& f = L[lev];
      int32_t* mate = dnew<int32_t>(f.n, s);
      int32_t* cmap = A.get<int32_t>(f.n + 1);
      match_level(f, capC, capG, seed, kMatchRounds, true, mate, s);
      coarse_count(f, mate, cmap, nullptr, s);
      int32_t* hnc = (int32_t*)&hbuf[0];
      GP_CUDA(cudaMemcpyAsync(hnc, cmap + f.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      if (pending_a) GP_CUDA(cudaMemcpyAsync(&hbuf[1], adev + lev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaStreamSynchronize(s));
      const int32_t nc = *hnc;
      if (pending_a) {
        take_entries(lev);
        pending_a = false;
      }
      if ((int64_t)nc * kStallDen > f.n * kStallNum) {
        dfree(mate, s);
        break;
      }
      LevelGraph c;
      c.n = nc;
      c.cap = T.a[lev];  // the coarse rows hold at most the fine entries
      contract_level(f, mate, cmap, c, s);
      dfree(mate, s);
      A.ptrs.push_back(c.start);
      A.ptrs.push_back(c.deg);
      A.ptrs.push_back(c.adj);
      A.ptrs.push_back(c.W);
      A.ptrs.push_back(c.vC);
      A.ptrs.push_back(c.vG);
      if (c.fix) A.ptrs.push_back(c.fix);
      GP_LAUNCH(F_MISC, k_sum_deg, grid_for(nc, 256, 8), 256, 0, s, (int64_t)nc, c.deg, adev + lev + 1);
      cmaps.push_back(cmap);
      c.a = 0;  // taken at the next level's round trip
      L.push_back(c);
      lev++;
      T.n[lev] = nc;
      pending_a = true;
    }
    if (pending_a) {  // the coarsest level's entries
      GP_CUDA(cudaMemcpyAsync(&hbuf[1], adev + lev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaStreamSynchronize(s));
      take_entries(lev);
    }
    const int Lc = lev;
    if (prof) cudaEventRecord(ev[1], s);
    std::vector<uint8_t*> parts(Lc + 1, nullptr);
    parts[Lc] = A.get<uint8_t>(L[Lc].n);
    if (restrict_only) {
      // the coarsest split is the proposed sides; from here on no vertex is pinned
      GP_LAUNCH(F_GGGP, k_pins_to_part, grid_for(L[Lc].n, 256), 256, 0, s, L[Lc].n, (const int8_t*)L[Lc].fix,
                parts[Lc], &td->trial);
      GP_CHECK_LAUNCH();
      for (auto& lg : L) lg.fix = nullptr;
    } else {
      gggp(L[Lc], BC, BG, g->SG, seed, parts[Lc], &td->trial, s);
    }
    if (prof) cudaEventRecord(ev[2], s);
    Ctl hctl;
    memset(&hctl, 0, sizeof(hctl));
    hctl.BC = BC;
    hctl.BG = BG;
    GP_CUDA(cudaMemcpyAsync(&td->ctl, &hctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    refine_loads(L[Lc], parts[Lc], &td->ctl, s);
    Cands cand;
    cand.id = A.get<int32_t>(n);
    cand.gain = A.get<long long>(n);
    cand.cd = A.get<long long>(n);
    cand.cs = A.get<long long>(n);
    cand.gainv = A.get<long long>(n);
    cand.stamp = A.get<int32_t>(n);
    cand.dirty[0] = A.get<int32_t>(n);
    cand.dirty[1] = A.get<int32_t>(n);
    GP_CUDA(cudaMemsetAsync(cand.stamp, 0xff, sizeof(int32_t) * n, s));
    // the coarse levels (at most kTailMaxVertices vertices each) in one CTA launch, the next ones (up to
    // kClusterTailMaxVertices) in one cluster launch, then the rest in one cooperative grid launch (level
    // by level, a launch per step, where the device has no cooperative launch)
    auto tail_args = [&](int a, int b, double gscale) {  // levels b (coarser) down to a
      TailArgs ta;
      memset(&ta, 0, sizeof(ta));
      ta.lo = a;
      ta.hi = b;
      ta.top_part = b < Lc ? parts[b + 1] : nullptr;
      for (int l = b; l >= a; l--) {
        if (l < Lc) parts[l] = A.get<uint8_t>(L[l].n);
        TailLevel& t = ta.lev[l - a];
        t.g = L[l];
        t.cmap = l < Lc ? cmaps[l] : nullptr;
        t.part = parts[l];
        t.G = group_for_degree(gscale * (double)T.a[l] / (double)(T.n[l] > 0 ? T.n[l] : 1));
        t.idbits = idbits_for(L[l].n);
      }
      return ta;
    };
    int lo = Lc + 1;
    while (lo - 1 >= 0 && L[lo - 1].n <= kTailMaxVertices && Lc - (lo - 1) + 1 <= kTailMaxLevels) lo--;
    if (lo <= Lc) {
      const TailArgs ta = tail_args(lo, Lc, 1.0);
      GP_LAUNCH(F_REFINE, k_refine_tail<kTailCta>, 1, 1024, 0, s, ta, &td->ctl, cand, td->rounds, td->moves,
                td->bal, td->balmoves, (unsigned*)nullptr, (int*)nullptr);
    }
    {
      int lo2 = lo;
      while (lo2 - 1 >= 0 && L[lo2 - 1].n <= kClusterTailMaxVertices && lo - (lo2 - 1) <= kTailMaxLevels) lo2--;
      const int cs = lo2 < lo ? cluster_max((const void*)k_refine_tail<kTailCluster>, 1024, 0) : 0;
      if (lo2 < lo && cs > 0) {
        const TailArgs ta = tail_args(lo2, lo - 1, 0.25);
        GP_CUDA(launch_cluster(F_REFINE, k_refine_tail<kTailCluster>, cs, 1024, 0, s, ta, &td->ctl, cand, td->rounds,
                               td->moves, td->bal, td->balmoves, (unsigned*)nullptr, (int*)nullptr));
        lo = lo2;
      }
    }
    // the grid's gain passes with about eight row entries per lane (its CTAs hold half the threads a
    // launch per step did; refine 2.90 -> 2.87 ms per step on the 1M workload, 20.0 -> 19.4 ms on the 16M
    // one, against about four; sixteen was slower)
    if (lo > 0 && lo <= kTailMaxLevels &&
        launch_refine_grid(tail_args(0, lo - 1, 0.125), &td->ctl, cand, td->rounds, td->moves, td->bal, td->balmoves,
                           &td->grid_bar, &td->tail_err, g->lev_event, s))
      lo = 0;
    for (int l = lo - 1; l >= 0; l--) {
      if (l < Lc) {  // the coarsest level holds the growing's split
        parts[l] = A.get<uint8_t>(L[l].n);
        project(L[l].n, cmaps[l], parts[l + 1], parts[l], s);
      }
      refine_level_run(L[l], parts[l], &td->ctl, cand, l, (double)T.a[l] / (double)(T.n[l] > 0 ? T.n[l] : 1), s);
      GP_LAUNCH(F_MISC, k_ref_end, 1, 1, 0, s, &td->ctl, l, td->rounds, td->moves, td->bal, td->balmoves);
    }
    if (prof) cudaEventRecord(ev[3], s);
    launch_cut(n, g->m, g->off, g->cols, g->w, parts[0], &td->cut, &td->bad, s);
    GP_CHECK_LAUNCH();
    GP_CUDA(cudaMemcpyAsync(part_out, parts[0], (size_t)n, cudaMemcpyDefault, s));
    if (prof) cudaEventRecord(ev[4], s);
    TraceDev h;
    GP_CUDA(cudaMemcpyAsync(&h, td, sizeof(TraceDev), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (h.tail_err || fault_is("timeout")) throw Fail{GP_ERR_TIMEOUT};
    R.cut = (int64_t)h.cut;
    R.load_cpu = h.ctl.LC;
    R.load_gpu = h.ctl.LG;
    R.feasible = (h.ctl.LC <= BC && h.ctl.LG <= BG) ? 1 : 0;
    R.levels = Lc;
    R.coarsest_n = (int32_t)L[Lc].n;
    int32_t rounds = 0;
    for (int l = 0; l <= Lc; l++) {
      T.rounds[l] = h.rounds[l];
      T.moves[l] = h.moves[l];
      T.balanced[l] = h.bal[l];
      T.bal_moves[l] = h.balmoves[l];
      rounds += h.rounds[l];
    }
    R.rounds = rounds;
    T.levels = Lc;
    T.gggp_trial = h.trial;
    if (prof) {
      for (int i = 0; i < 4; i++) cudaEventElapsedTime(&R.ms[i], ev[i], ev[i + 1]);
      for (auto& e : ev) cudaEventDestroy(e);
    }
    g->trace = T;
    if (res) *res = R;
    return levels_ready(g);  // a deferred creation's cycle check (its traversal ran beside this call)
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_partition(gp_graph* g, double r_cpu, double tol, uint64_t seed, uint8_t* part_out, gp_result* res,
                       void* stream) {
  return partition_impl(g, nullptr, r_cpu, tol, seed, part_out, res, stream);
}

gp_status gp_partition_fixed(gp_graph* g, const int8_t* fixed, double r_cpu, double tol, uint64_t seed,
                             uint8_t* part_out, gp_result* res, void* stream) {
  return partition_impl(g, fixed, r_cpu, tol, seed, part_out, res, stream);
}

// Checked build: the site of the first failed index test since the last clear (0: none); -1 without
// GP_CHECKED.
int32_t gp_checked_site(int32_t clear) {
#ifdef GP_CHECKED
  int site = 0;
  if (cudaMemcpyFromSymbol(&site, d_check_site, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return -2;
  }
  if (clear) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(d_check_site, &zero, sizeof(int)) != cudaSuccess) cudaGetLastError();
  }
  return site;
#else
  (void)clear;
  return -1;
#endif
}

#ifdef GP_CHECKED
// One thread gathers through an index it tests first: idx is out of range, so the test records site 99
// and the gather does not happen.
__global__ void k_checked_selftest(const int32_t* __restrict__ a, int64_t n, int64_t idx, int32_t* out) {
  int32_t v = -1;
  if (GP_IN(idx, n, 99)) v = a[idx];
  *out = v;
}
#endif

gp_status gp_selftest_checked(void* stream) {
#ifdef GP_CHECKED
  cudaStream_t s = (cudaStream_t)stream;
  try {
    int32_t* buf = dnew<int32_t>(5, s);
    GP_CUDA(cudaMemsetAsync(buf, 0, 5 * sizeof(int32_t), s));
    GP_LAUNCH(F_MISC, k_checked_selftest, 1, 1, 0, s, (const int32_t*)buf, (int64_t)4, (int64_t)1000000, buf + 4);
    GP_CHECK_LAUNCH();
    int32_t v = 0;
    GP_CUDA(cudaMemcpyAsync(&v, buf + 4, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    dfree(buf, s);
    return v == -1 ? GP_OK : GP_ERR_CUDA;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
#else
  (void)stream;
  return GP_ERR_INVALID;  // the unchecked build has no test to skip the gather: nothing is launched
#endif
}

gp_status gp_selftest_grid_wait_timeout(void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    unsigned* bar = A.get<unsigned>(1);
    int* err = A.get<int>(1);
    GP_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
    GP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    void* args[] = {(void*)&bar, (void*)&err};
    launch_begin(F_MISC, s);
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_grid_wait_selftest, dim3(2), dim3(32), args, 0, s);
    launch_end(F_MISC, s);
    GP_CUDA(e);
    int herr = 0;
    GP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    return herr ? GP_ERR_TIMEOUT : GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_last_trace(const gp_graph* g, gp_trace* trace) {
  if (!g || !trace) return GP_ERR_INVALID;
  *trace = g->trace;
  return GP_OK;
}

gp_status gp_cut(const gp_graph* g, const uint8_t* part, int64_t* cut, void* stream) {
  if (!g || !cut || (!part && g->n > 0)) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    Arena A(s);
    const int64_t n = g->n;
    const uint8_t* p = part;
    if (n && !is_device_ptr(part)) {
      uint8_t* d = A.get<uint8_t>(n);
      GP_CUDA(cudaMemcpyAsync(d, part, (size_t)n, cudaMemcpyDefault, s));
      p = d;
    }
    unsigned long long* c = A.get<unsigned long long>(1);
    int* bad = A.get<int>(1);
    GP_CUDA(cudaMemsetAsync(c, 0, sizeof(unsigned long long), s));
    GP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    launch_cut(n, g->m, g->off, g->cols, g->w, p, c, bad, s);
    GP_CHECK_LAUNCH();
    unsigned long long hc = 0;
    int hb = 0;
    GP_CUDA(cudaMemcpyAsync(&hc, c, sizeof(hc), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (hb) return GP_ERR_INVALID;
    *cut = (int64_t)hc;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_makespan(const gp_graph* g, const uint8_t* part, int64_t* makespan, int64_t* finish_out, void* stream) {
  if (!g || !makespan || (!part && g->n > 0)) return GP_ERR_INVALID;
  {
    const gp_status ls = levels_ready(g);
    if (ls != GP_OK) return ls;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n;
  if (n == 0) {
    *makespan = 0;
    return GP_OK;
  }
  try {
    Arena A(s);
    const uint8_t* p = part;
    if (!is_device_ptr(part)) {
      uint8_t* d = A.get<uint8_t>(n);
      GP_CUDA(cudaMemcpyAsync(d, part, (size_t)n, cudaMemcpyDefault, s));
      p = d;
    }
    int64_t* fin = nullptr;
    const bool fin_host = finish_out && !is_device_ptr(finish_out);
    if (finish_out) fin = fin_host ? A.get<int64_t>(n) : finish_out;
    unsigned long long* fp = A.get<unsigned long long>(n);
    struct Small {
      unsigned long long ms;
      int bad;
      unsigned grid_bar;  // the grid kernel's barrier counter
    };
    Small* sm = A.get<Small>(1);
    GP_CUDA(cudaMemsetAsync(sm, 0, sizeof(Small), s));
    GP_CUDA(launch_makespan(g, p, fp, &sm->ms, &sm->bad, fin, s, &sm->grid_bar));
    Small h;
    GP_CUDA(cudaMemcpyAsync(&h, sm, sizeof(Small), cudaMemcpyDeviceToHost, s));
    if (fin_host) GP_CUDA(cudaMemcpyAsync(finish_out, fin, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (h.bad & 2) return GP_ERR_TIMEOUT;  // a bounded device wait gave up
    if (h.bad) return GP_ERR_INVALID;
    *makespan = (int64_t)h.ms;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

// ------------------------------------------------------------------------------------------------
// step-level entry points (device CSR in, device results out)
// ------------------------------------------------------------------------------------------------
static LevelGraph view_of(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W, const int64_t* vC,
                          const int64_t* vG, Arena& A, cudaStream_t s) {
  LevelGraph L;
  L.n = n;
  int64_t a = 0;
  GP_CUDA(cudaMemcpyAsync(&a, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  L.cap = a;
  L.start = const_cast<int64_t*>(off);
  L.deg = A.get<int32_t>(n);
  L.adj = const_cast<int32_t*>(adj);
  L.W = const_cast<int64_t*>(W);
  L.vC = const_cast<int64_t*>(vC);
  L.vG = const_cast<int64_t*>(vG);
  if (n) GP_LAUNCH(F_MISC, k_deg_from_off, grid_for(n, 256), 256, 0, s, n, off, L.deg);
  GP_CHECK_LAUNCH();
  return L;
}

gp_status gp_step_match(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W, const int64_t* vC,
                        const int64_t* vG, int64_t cap_cpu, int64_t cap_gpu, uint64_t seed, int32_t rounds,
                        int32_t twohop, int32_t* mate_out, void* stream) {
  if (n < 0 || n > kMaxN || !off || (n > 0 && (!vC || !vG || !mate_out)) || rounds < 0) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    LevelGraph L = view_of(n, off, adj, W, vC, vG, A, s);
    match_level(L, cap_cpu, cap_gpu, seed, rounds, twohop != 0, mate_out, s);
    GP_CUDA(cudaStreamSynchronize(s));
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_step_contract(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W, const int64_t* vC,
                           const int64_t* vG, const int32_t* mate, int32_t* cmap_out, int64_t* coff, int32_t* cadj,
                           int64_t* cW, int64_t* cvC, int64_t* cvG, int64_t* nc_out, int64_t* ac_out, void* stream) {
  if (n < 0 || n > kMaxN || !off || !nc_out || !ac_out || !coff) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    LevelGraph L = view_of(n, off, adj, W, vC, vG, A, s);
    int64_t a = 0;
    GP_CUDA(cudaMemcpyAsync(&a, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    int32_t* cmap = A.get<int32_t>(n + 1);
    coarse_count(L, mate, cmap, nullptr, s);
    int32_t nc = 0;
    GP_CUDA(cudaMemcpyAsync(&nc, cmap + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    LevelGraph C;
    C.n = nc;
    C.cap = a;
    if (n) contract_level(L, mate, cmap, C, s);
    if (n) {
      A.ptrs.push_back(C.start);
      A.ptrs.push_back(C.deg);
      A.ptrs.push_back(C.adj);
      A.ptrs.push_back(C.W);
      A.ptrs.push_back(C.vC);
      A.ptrs.push_back(C.vG);
      GP_CUDA(cudaMemcpyAsync(cmap_out, cmap, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    scan_i32_to_i64(C.deg, coff, nc, s);
    if (nc) GP_LAUNCH(F_MISC, k_compact_rows, grid_for((int64_t)nc * 32, 256), 256, 0, s, (int64_t)nc, C.start, C.deg,
                      C.adj, C.W, coff, cadj, cW);
    if (nc) {
      GP_CUDA(cudaMemcpyAsync(cvC, C.vC, sizeof(int64_t) * nc, cudaMemcpyDeviceToDevice, s));
      GP_CUDA(cudaMemcpyAsync(cvG, C.vG, sizeof(int64_t) * nc, cudaMemcpyDeviceToDevice, s));
    }
    GP_CHECK_LAUNCH();
    int64_t ac = 0;
    GP_CUDA(cudaMemcpyAsync(&ac, coff + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    *nc_out = nc;
    *ac_out = ac;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_step_gggp(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W, const int64_t* vC,
                       const int64_t* vG, int64_t bound_cpu, int64_t bound_gpu, uint64_t seed, uint8_t* part_out,
                       int32_t* trial_out, void* stream) {
  if (n < 0 || n > kMaxN || !off || !trial_out || (n > 0 && !part_out)) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    LevelGraph L = view_of(n, off, adj, W, vC, vG, A, s);
    long long* sg = A.get<long long>(1);
    sum_i64(vG, n, sg, s);
    long long SG = 0;
    GP_CUDA(cudaMemcpyAsync(&SG, sg, sizeof(SG), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    int32_t* t = A.get<int32_t>(1);
    GP_CUDA(cudaMemsetAsync(t, 0xff, sizeof(int32_t), s));
    if (n) gggp(L, bound_cpu, bound_gpu, SG, seed, part_out, t, s);
    GP_CUDA(cudaMemcpyAsync(trial_out, t, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_step_gggp_grow(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W, const int64_t* vC,
                            const int64_t* vG, int64_t bound_cpu, int64_t bound_gpu, int64_t start, uint8_t* part_out,
                            int64_t* cut_out, void* stream) {
  if (n <= 0 || n > kMaxN || !off || start < 0 || start >= n || !part_out || !cut_out) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    LevelGraph L = view_of(n, off, adj, W, vC, vG, A, s);
    int64_t* c = A.get<int64_t>(1);
    gggp_grow_one(L, bound_cpu, bound_gpu, start, part_out, c, s);
    GP_CUDA(cudaMemcpyAsync(cut_out, c, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_step_refine(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W, const int64_t* vC,
                         const int64_t* vG, int64_t bound_cpu, int64_t bound_gpu, uint8_t* part, int64_t* stats,
                         void* stream) {
  if (n < 0 || n > kMaxN || !off || (n > 0 && !part)) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    LevelGraph L = view_of(n, off, adj, W, vC, vG, A, s);
    Ctl* ctl = A.get<Ctl>(1);
    Ctl hc;
    memset(&hc, 0, sizeof(hc));
    hc.BC = bound_cpu;
    hc.BG = bound_gpu;
    GP_CUDA(cudaMemcpyAsync(ctl, &hc, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    Cands cand;
    cand.id = A.get<int32_t>(n);
    cand.gain = A.get<long long>(n);
    cand.cd = A.get<long long>(n);
    cand.cs = A.get<long long>(n);
    cand.gainv = A.get<long long>(n);
    cand.stamp = A.get<int32_t>(n);
    cand.dirty[0] = A.get<int32_t>(n);
    cand.dirty[1] = A.get<int32_t>(n);
    if (n) {
      int64_t a = 0;
      GP_CUDA(cudaMemcpyAsync(&a, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaMemsetAsync(cand.stamp, 0xff, sizeof(int32_t) * n, s));
      GP_CUDA(cudaStreamSynchronize(s));
      refine_loads(L, part, ctl, s);
      refine_level_run(L, part, ctl, cand, 0, (double)a / (double)n, s);
    }
    GP_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (stats) {
      stats[0] = hc.rounds;
      stats[1] = hc.balanced;
      stats[2] = hc.moves;
      stats[3] = hc.bal_moves;
      stats[4] = hc.LC;
      stats[5] = hc.LG;
    }
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

}  // extern "C"

// the no-allocation makespan variant (its scratch array must share this translation unit)
#include "gp_noalloc.cu"

#include "gp_listsched.cu"

#include "gp_kway.cu"
// many graphs in one persistent launch
#include "gp_batch.cu"
// the learned proposal (message-passing network on the tensor cores)
#include "gp_mpnn.cu"

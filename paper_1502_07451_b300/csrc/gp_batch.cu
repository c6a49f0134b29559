// gp_batch.cu -- gp_batch_partition and its autotuner: the host side of the persistent batch kernel
// (k_batch.cuh).
//
// A call fills one descriptor per graph, orders the graphs largest first, and replays a captured
// CUDA graph holding the queue reset, the persistent launch and the copy of the per-graph results.
// The captured graph, the descriptor buffers and the workspace live in a per-device context and
// are reused by later calls of the same shape.  Graphs too large for a CTA's workspace (and any
// graph the kernel defers) go through the single-graph path in the same call.
//
// This file is included at the end of gp_api.cu (the library is one translation unit).

namespace gp {

struct SchedDef {
  int nt, minb;
  BatchSched s;
  const char* name;
};
static const SchedDef kSched[] = {
    {512, 2, {0, 256}, "cta512x2"},
    {256, 4, {0, 256}, "cta256x4"},
    {1024, 1, {0, 256}, "cta1024x1"},
    {512, 1, {0, 256}, "cta512x1"},
    {512, 2, {1, 256}, "cta512x2_wide_rows"},
    {512, 2, {-1, 256}, "cta512x2_narrow_rows"},
    {512, 2, {0, 128}, "cta512x2_hash128"},
    {512, 2, {-2, 256}, "cta512x2_quarter_rows"},
    {512, 2, {-3, 256}, "cta512x2_eighth_rows"},
    {512, 2, {-4, 256}, "cta512x2_sixteenth_rows"},
    {256, 4, {-1, 256}, "cta256x4_narrow_rows"},
    {256, 4, {-2, 256}, "cta256x4_quarter_rows"},
};
constexpr int kNumSched = (int)(sizeof(kSched) / sizeof(kSched[0]));

// graphs with more adjacency entries than this always take the single-graph path (they fill the
// GPU on their own)
constexpr int64_t kBatchMaxEntries = int64_t(1) << 23;

typedef void (*BatchKernel)(const BatchGraph*, const int32_t*, int32_t, unsigned*, char*, unsigned long long,
                            BatchOut*, BatchSched);

static BatchKernel sched_kernel(int i) {
  const SchedDef& d = kSched[i];
  if (d.nt == 256) return k_batch<256, 4>;
  if (d.nt == 1024) return k_batch<1024, 1>;
  if (d.minb == 1) return k_batch<512, 1>;
  return k_batch<512, 2>;
}

// Workspace of one CTA for graphs of at most n vertices and a entries: fixed per-vertex scratch
// plus coarse levels (their entries add up to about 5 a on the generated DAGs; a graph that needs
// more is deferred).
static unsigned long long slot_bytes_for(int64_t n, int64_t a) {
  const unsigned long long b = 160ull * (unsigned long long)n + 72ull * (unsigned long long)a + (2ull << 20);
  return (b + 255ull) & ~255ull;
}

struct BatchCtx {
  std::mutex mu;
  int cap = 0;
  BatchGraph* d_graphs = nullptr;
  int32_t* d_order = nullptr;
  BatchOut* d_out = nullptr;
  unsigned* d_queue = nullptr;
  BatchGraph* h_graphs = nullptr;
  int32_t* h_order = nullptr;
  BatchOut* h_out = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  uint8_t* d_stage = nullptr;
  uint8_t* h_stage = nullptr;
  size_t stage_bytes = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  int key_sched = -1, key_count = -1, key_slots = -1;
  unsigned long long key_slot_bytes = 0;
  int tuned = -1;
};
static BatchCtx g_bctx[64];
static std::atomic<int> g_sched_forced{-1};

static void ctx_drop_exec(BatchCtx& c) {
  if (c.exec) cudaGraphExecDestroy(c.exec);
  c.exec = nullptr;
  c.key_sched = -1;
}

static void ctx_reserve(BatchCtx& c, int count) {
  if (count <= c.cap) return;
  ctx_drop_exec(c);
  int cap = c.cap ? c.cap : 64;
  while (cap < count) cap *= 2;
  cudaFree(c.d_graphs);
  cudaFree(c.d_order);
  cudaFree(c.d_out);
  cudaFreeHost(c.h_graphs);
  cudaFreeHost(c.h_order);
  cudaFreeHost(c.h_out);
  c.d_graphs = nullptr;
  c.d_order = nullptr;
  c.d_out = nullptr;
  c.h_graphs = nullptr;
  c.h_order = nullptr;
  c.h_out = nullptr;
  c.cap = 0;
  GP_CUDA(cudaMalloc(&c.d_graphs, sizeof(BatchGraph) * cap));
  GP_CUDA(cudaMalloc(&c.d_order, sizeof(int32_t) * cap));
  GP_CUDA(cudaMalloc(&c.d_out, sizeof(BatchOut) * cap));
  GP_CUDA(cudaMallocHost(&c.h_graphs, sizeof(BatchGraph) * cap));
  GP_CUDA(cudaMallocHost(&c.h_order, sizeof(int32_t) * cap));
  GP_CUDA(cudaMallocHost(&c.h_out, sizeof(BatchOut) * cap));
  if (!c.d_queue) GP_CUDA(cudaMalloc(&c.d_queue, 256));
  if (!c.cap_stream) GP_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
  c.cap = cap;
}

static void ctx_workspace(BatchCtx& c, size_t bytes) {
  if (bytes <= c.ws_bytes) return;
  ctx_drop_exec(c);
  cudaFree(c.ws);
  c.ws = nullptr;
  c.ws_bytes = 0;
  GP_CUDA(cudaMalloc(&c.ws, bytes));
  c.ws_bytes = bytes;
}

static void ctx_stage(BatchCtx& c, size_t bytes) {
  if (bytes <= c.stage_bytes) return;
  cudaFree(c.d_stage);
  cudaFreeHost(c.h_stage);
  c.d_stage = nullptr;
  c.h_stage = nullptr;
  c.stage_bytes = 0;
  size_t b = 1 << 20;
  while (b < bytes) b *= 2;
  GP_CUDA(cudaMalloc(&c.d_stage, b));
  GP_CUDA(cudaMallocHost(&c.h_stage, b));
  c.stage_bytes = b;
}

struct BatchJob {
  int idx;               // caller's index
  int64_t BC, BG;
  uint64_t seed;
  const float* logits;   // learned path: the graph's logits (device), else null
  uint8_t* dst;          // caller's split buffer
  bool dst_host;
  size_t stage_off;
};

// Runs the persistent kernel over `jobs` (all with n > 0) with schedule `si`; fills out[j].
// Returns the kernel's device time in ms (events on `s`).
static float run_persistent(BatchCtx& c, int si, gp_graph* const* graphs, const std::vector<BatchJob>& jobs,
                            bool want_ms, std::vector<BatchOut>& out, cudaStream_t s) {
  const int K = (int)jobs.size();
  out.assign(K, BatchOut{});
  if (K == 0) return 0.f;
  ctx_reserve(c, K);
  int64_t nmax = 0, amax = 0;
  size_t stage = 0;
  for (const BatchJob& j : jobs) {
    const gp_graph* g = graphs[j.idx];
    nmax = std::max(nmax, g->n);
    amax = std::max(amax, g->a0);
    if (j.dst_host) stage += (size_t)g->n;
  }
  if (stage) ctx_stage(c, stage);
  const SchedDef& sd = kSched[si];
  const BatchKernel kern = sched_kernel(si);
  const int dsm = (sd.nt / 32) * kBatchWarpSmem;
  GP_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
  int per_sm = 0;
  GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, sd.nt, dsm));
  if (per_sm < 1) throw Fail{GP_ERR_CUDA};
  int slots = std::min(K, per_sm * num_sms());
  unsigned long long sb = slot_bytes_for(nmax, amax);
  // GP_BATCH_SLOT_LIMIT=<bytes> caps a CTA's workspace (graphs that outgrow it are deferred): a
  // check that deferral leaves every result unchanged
  if (const char* lim = getenv("GP_BATCH_SLOT_LIMIT")) {
    const unsigned long long l = strtoull(lim, nullptr, 10) & ~255ull;
    if (l >= 4096 && l < sb) sb = l;
  }
  // keep the workspace within a quarter of the free memory (fewer slots if needed)
  size_t freeb = 0, totalb = 0;
  GP_CUDA(cudaMemGetInfo(&freeb, &totalb));
  const size_t budget = (size_t)c.ws_bytes + freeb / 4;
  while (slots > 1 && (size_t)slots * sb > budget) slots--;
  ctx_workspace(c, (size_t)slots * sb);
  // descriptors, largest first
  for (int j = 0; j < K; j++) {
    const gp_graph* g = graphs[jobs[j].idx];
    BatchGraph& B = c.h_graphs[j];
    B.start = g->L0.start;
    B.deg = g->L0.deg;
    B.adj = g->L0.adj;
    B.W = g->L0.W;
    B.vC = g->L0.vC;
    B.vG = g->L0.vG;
    B.n = g->n;
    B.a0 = g->a0;
    B.BC = jobs[j].BC;
    B.BG = jobs[j].BG;
    B.SC = g->SC;
    B.SG = g->SG;
    B.logits = jobs[j].logits;
    B.seed = jobs[j].seed;
    B.off = g->off;
    B.cols = g->cols;
    B.w = g->w;
    B.lev_ptr = g->lev_ptr;
    B.lev_vtx = g->lev_vtx;
    B.lo_off = g->lo_off;
    B.lo_src = g->lo_src;
    B.lo_w = g->lo_w;
    B.lo_cC = g->lo_cC;
    B.lo_cG = g->lo_cG;
    B.nlev = g->nlev;
    B.want_makespan = want_ms ? 1 : 0;
    B.part = jobs[j].dst_host ? c.d_stage + jobs[j].stage_off : jobs[j].dst;
    c.h_order[j] = j;
  }
  std::sort(c.h_order, c.h_order + K, [&](int x, int y) {
    const int64_t wx = c.h_graphs[x].a0 + c.h_graphs[x].n, wy = c.h_graphs[y].a0 + c.h_graphs[y].n;
    return wx != wy ? wx > wy : x < y;
  });
  GP_CUDA(cudaMemcpyAsync(c.d_graphs, c.h_graphs, sizeof(BatchGraph) * K, cudaMemcpyHostToDevice, s));
  GP_CUDA(cudaMemcpyAsync(c.d_order, c.h_order, sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
  if (!c.exec || c.key_sched != si || c.key_count != K || c.key_slots != slots || c.key_slot_bytes != sb) {
    ctx_drop_exec(c);
    cudaGraph_t graph = nullptr;
    GP_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(c.d_queue, 0, sizeof(unsigned), c.cap_stream);
    kern<<<slots, sd.nt, dsm, c.cap_stream>>>(c.d_graphs, c.d_order, K, c.d_queue, c.ws, sb, c.d_out, sd.s);
    cudaMemcpyAsync(c.h_out, c.d_out, sizeof(BatchOut) * K, cudaMemcpyDeviceToHost, c.cap_stream);
    const cudaError_t e = cudaStreamEndCapture(c.cap_stream, &graph);
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      GP_CUDA(e);
    }
    const cudaError_t ei = cudaGraphInstantiate(&c.exec, graph, 0);
    cudaGraphDestroy(graph);
    GP_CUDA(ei);
    c.key_sched = si;
    c.key_count = K;
    c.key_slots = slots;
    c.key_slot_bytes = sb;
  }
  cudaEvent_t e0, e1;
  GP_CUDA(cudaEventCreate(&e0));
  GP_CUDA(cudaEventCreate(&e1));
  launch_begin(F_BATCH, s);
  cudaEventRecord(e0, s);
  const cudaError_t el = cudaGraphLaunch(c.exec, s);
  cudaEventRecord(e1, s);
  launch_end(F_BATCH, s);
  if (el != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    GP_CUDA(el);
  }
  if (stage) GP_CUDA(cudaMemcpyAsync(c.h_stage, c.d_stage, stage, cudaMemcpyDeviceToHost, s));
  const cudaError_t es = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (es == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GP_CUDA(es);
  for (int j = 0; j < K; j++) {
    out[j] = c.h_out[j];
    if (jobs[j].dst_host && out[j].status == kBatchDone)
      memcpy(jobs[j].dst, c.h_stage + jobs[j].stage_off, (size_t)graphs[jobs[j].idx]->n);
  }
  return ms;
}

// Shared by gp_batch_partition and gp_batch_autotune: validate, plan, run with schedule si.
static gp_status batch_run(int32_t count, gp_graph* const* graphs, const double* r_cpu, double tol,
                           const uint64_t* seeds, uint8_t* const* parts, gp_result* res, int64_t* makespans,
                           cudaStream_t s, int si, float* kernel_ms, const float* const* logits_of = nullptr) {
  if (count < 0 || (count > 0 && !graphs)) return GP_ERR_INVALID;
  if (kernel_ms) *kernel_ms = 0.f;
  if (count == 0) return GP_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
  for (int i = 0; i < count; i++)
    if (graphs[i]) {
      const gp_status ls = levels_ready(graphs[i]);  // the makespans read the levels
      if (ls != GP_OK) return ls;
    }
  std::vector<BatchJob> kjobs, direct;
  std::vector<int64_t> BCs(count), BGs(count);
  size_t stage = 0;
  for (int i = 0; i < count; i++) {
    const gp_graph* g = graphs[i];
    if (!g || g->dev != dev) return GP_ERR_INVALID;
    if (g->n > 0 && (!parts || !parts[i])) return GP_ERR_INVALID;
    int64_t BC, BG;
    const gp_status st = host_bounds(g->SC, g->SG, r_cpu ? r_cpu[i] : -1.0, tol, &BC, &BG);
    if (st != GP_OK) return st;
    BCs[i] = BC;
    BGs[i] = BG;
  }
  try {
    pool_setup();
    for (int i = 0; i < count; i++) {
      const gp_graph* g = graphs[i];
      BatchJob j;
      j.idx = i;
      j.BC = BCs[i];
      j.BG = BGs[i];
      j.seed = seeds ? seeds[i] : 0ull;
      j.logits = logits_of ? logits_of[i] : nullptr;
      j.dst = g->n > 0 ? parts[i] : nullptr;
      j.dst_host = g->n > 0 && !is_device_ptr(parts[i]);
      j.stage_off = 0;
      if (g->n == 0) {
        if (res) {
          gp_result R;
          memset(&R, 0, sizeof(R));
          R.bound_cpu = BCs[i];
          R.bound_gpu = BGs[i];
          R.feasible = 1;
          res[i] = R;
        }
        if (makespans) makespans[i] = 0;
        continue;
      }
      if (g->a0 > kBatchMaxEntries) {
        direct.push_back(j);
      } else {
        if (j.dst_host) {
          j.stage_off = stage;
          stage += (size_t)g->n;
        }
        kjobs.push_back(j);
      }
    }
    std::vector<BatchOut> out;
    float ms = 0.f;
    {
      BatchCtx& c = g_bctx[dev];
      std::lock_guard<std::mutex> lk(c.mu);
      ms = run_persistent(c, si, graphs, kjobs, makespans != nullptr, out, s);
    }
    if (kernel_ms) *kernel_ms = ms;
    for (size_t k = 0; k < kjobs.size(); k++) {
      const BatchJob& j = kjobs[k];
      const BatchOut& o = out[k];
      if (o.status != kBatchDone) {
        direct.push_back(j);
        continue;
      }
      if (res) {
        gp_result R;
        memset(&R, 0, sizeof(R));
        R.cut = o.cut;
        R.load_cpu = o.LC;
        R.load_gpu = o.LG;
        R.bound_cpu = j.BC;
        R.bound_gpu = j.BG;
        R.feasible = o.feasible;
        R.levels = o.levels;
        R.rounds = o.rounds;
        R.coarsest_n = o.coarsest_n;
        R.ms[0] = ms;
        res[j.idx] = R;
      }
      if (makespans) makespans[j.idx] = o.makespan;
    }
    for (const BatchJob& j : direct) {
      gp_graph* g = graphs[j.idx];
      gp_result R;
      const double r = r_cpu ? r_cpu[j.idx] : -1.0;
      gp_status st = j.logits ? gp_partition_learned(g, nullptr, j.logits, r, tol, j.dst, &R, s)
                              : gp_partition(g, r, tol, j.seed, j.dst, &R, s);
      if (st != GP_OK) return st;
      if (res) res[j.idx] = R;
      if (makespans) {
        int64_t msv = 0;
        st = gp_makespan(g, j.dst, &msv, nullptr, s);
        if (st != GP_OK) return st;
        makespans[j.idx] = msv;
      }
    }
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

static int current_schedule(int dev) {
  const int f = g_sched_forced.load();
  if (f >= 0 && f < kNumSched) return f;
  const int t = (dev >= 0 && dev < 64) ? g_bctx[dev].tuned : -1;
  return (t >= 0 && t < kNumSched) ? t : 0;
}

}  // namespace gp

extern "C" {

gp_status gp_batch_partition(int32_t count, gp_graph* const* graphs, const double* r_cpu, double tol,
                             const uint64_t* seeds, uint8_t* const* parts, gp_result* res, int64_t* makespans,
                             void* stream) {
  int dev = 0;
  cudaGetDevice(&dev);
  return batch_run(count, graphs, r_cpu, tol, seeds, parts, res, makespans, (cudaStream_t)stream,
                   current_schedule(dev), nullptr);
}

int32_t gp_batch_schedule_count(void) { return kNumSched; }

const char* gp_batch_schedule_name(int32_t i) { return (i >= 0 && i < kNumSched) ? kSched[i].name : nullptr; }

gp_status gp_batch_set_schedule(int32_t i) {
  if (i < -1 || i >= kNumSched) return GP_ERR_INVALID;
  g_sched_forced.store(i);
  return GP_OK;
}

gp_status gp_batch_autotune(int32_t count, gp_graph* const* graphs, const double* r_cpu, double tol,
                            const uint64_t* seeds, int32_t* best, float* ms_out, void* stream) {
  if (count <= 0 || !graphs || !best) return GP_ERR_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // scratch splits on the device (the results are discarded)
  int64_t tot = 0;
  for (int i = 0; i < count; i++) {
    if (!graphs[i]) return GP_ERR_INVALID;
    tot += graphs[i]->n;
  }
  uint8_t* scratch = nullptr;
  if (cudaMalloc(&scratch, (size_t)(tot > 0 ? tot : 1)) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_OOM;
  }
  std::vector<uint8_t*> parts(count);
  int64_t o = 0;
  for (int i = 0; i < count; i++) {
    parts[i] = scratch + o;
    o += graphs[i]->n;
  }
  int bi = 0;
  float bms = 0.f;
  gp_status st = GP_OK;
  for (int si = 0; si < kNumSched && st == GP_OK; si++) {
    float ms = 0.f;
    st = batch_run(count, graphs, r_cpu, tol, seeds, parts.data(), nullptr, nullptr, s, si, nullptr);  // warm-up
    if (st == GP_OK) st = batch_run(count, graphs, r_cpu, tol, seeds, parts.data(), nullptr, nullptr, s, si, &ms);
    if (ms_out) ms_out[si] = ms;
    if (st == GP_OK && (si == 0 || ms < bms)) {
      bi = si;
      bms = ms;
    }
  }
  cudaFree(scratch);
  if (st != GP_OK) return st;
  {
    std::lock_guard<std::mutex> lk(g_bctx[dev].mu);
    g_bctx[dev].tuned = bi;
  }
  *best = bi;
  return GP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// gp_graph_create_batch: gp_graph_create for many DAGs, in one persistent launch.
// ------------------------------------------------------------------------------------------------
namespace gp {

constexpr int64_t kCreateBatchMaxN = int64_t(1) << 20;  // larger DAGs take gp_graph_create
constexpr int kCreateThreads = 512;

struct CreateLayout {
  size_t bytes = 0;
  size_t add(size_t b) {
    const size_t a = (bytes + 255) & ~(size_t)255;
    bytes = a + (b ? b : 1);
    return a;
  }
};

}  // namespace gp

extern "C" gp_status gp_graph_create_batch(int32_t count, const int64_t* n, const int64_t* m,
                                           const int64_t* const* offsets, const int32_t* const* cols,
                                           const int32_t* const* edge_cost, const int32_t* const* cpu_cost,
                                           const int32_t* const* gpu_cost, int ptr_kind, void* stream,
                                           gp_graph** out, gp_status* status) {
  if (count < 0 || (count > 0 && (!n || !m || !offsets || !cols || !edge_cost || !cpu_cost || !gpu_cost || !out ||
                                   !status)) ||
      (ptr_kind != 0 && ptr_kind != 1))
    return GP_ERR_INVALID;
  for (int i = 0; i < count; i++) {
    out[i] = nullptr;
    status[i] = GP_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> kern, single;
  for (int i = 0; i < count; i++) {
    const bool ok = n[i] >= 0 && m[i] >= 0 && n[i] <= kMaxN && offsets[i] && (m[i] == 0 || (cols[i] && edge_cost[i])) &&
                    (n[i] == 0 || (cpu_cost[i] && gpu_cost[i]));
    if (!ok) continue;  // status stays GP_ERR_INVALID
    if (n[i] > kCreateBatchMaxN || m[i] >= (int64_t(1) << 31)) single.push_back(i);
    else kern.push_back(i);
  }
  try {
    pool_setup();
    const int dev = device_id();
    const int K = (int)kern.size();
    if (K > 0) {
      // one device block: every graph's inputs, then every graph's derived arrays
      CreateLayout lay;
      std::vector<CreateJob> jobs(K);
      std::vector<size_t> o_in(K * 5), o_dv(K * 17);
      for (int k = 0; k < K; k++) {
        const int64_t nn = n[kern[k]], mm = m[kern[k]];
        size_t* q = &o_in[k * 5];
        q[0] = lay.add(8 * (nn + 1));
        q[1] = lay.add(4 * mm);
        q[2] = lay.add(4 * mm);
        q[3] = lay.add(4 * nn);
        q[4] = lay.add(4 * nn);
      }
      for (int k = 0; k < K; k++) {
        const int64_t nn = n[kern[k]], mm = m[kern[k]];
        size_t* q = &o_dv[k * 17];
        const size_t sz[17] = {(size_t)(8 * (nn + 1)), (size_t)(4 * mm), (size_t)(4 * mm), (size_t)(4 * nn),
                               (size_t)(8 * (nn + 2)), (size_t)(4 * nn), (size_t)(8 * (nn + 1)), (size_t)(4 * mm),
                               (size_t)(4 * mm), (size_t)(4 * nn), (size_t)(4 * nn), (size_t)(8 * (nn + 1)),
                               (size_t)(4 * nn), (size_t)(8 * mm), (size_t)(16 * mm), (size_t)(8 * nn),
                               (size_t)(8 * nn)};
        for (int t = 0; t < 17; t++) q[t] = lay.add(sz[t]);
      }
      char* base = (char*)dalloc(lay.bytes, s);
      std::shared_ptr<void> block(base, [dev](void* p) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(dev);
        cudaFree(p);
        cudaSetDevice(cur);
      });
      int64_t nmax = 0;
      for (int k = 0; k < K; k++) {
        const int i = kern[k];
        CreateJob& J = jobs[k];
        const size_t* q = &o_in[k * 5];
        const size_t* r = &o_dv[k * 17];
        J.n = n[i];
        J.m = m[i];
        J.off = (const int64_t*)(base + q[0]);
        J.cols = (const int32_t*)(base + q[1]);
        J.w = (const int32_t*)(base + q[2]);
        J.cC = (const int32_t*)(base + q[3]);
        J.cG = (const int32_t*)(base + q[4]);
        J.in_off = (int64_t*)(base + r[0]);
        J.in_src = (int32_t*)(base + r[1]);
        J.in_w = (int32_t*)(base + r[2]);
        J.lev_vtx = (int32_t*)(base + r[3]);
        J.lev_ptr = (int64_t*)(base + r[4]);
        J.level = (int32_t*)(base + r[5]);
        J.lo_off = (int64_t*)(base + r[6]);
        J.lo_src = (int32_t*)(base + r[7]);
        J.lo_w = (int32_t*)(base + r[8]);
        J.lo_cC = (int32_t*)(base + r[9]);
        J.lo_cG = (int32_t*)(base + r[10]);
        J.start = (int64_t*)(base + r[11]);
        J.deg = (int32_t*)(base + r[12]);
        J.adj = (int32_t*)(base + r[13]);
        J.W = (int64_t*)(base + r[14]);
        J.vC = (int64_t*)(base + r[15]);
        J.vG = (int64_t*)(base + r[16]);
        nmax = std::max(nmax, J.n);
      }
      // inputs
      if (ptr_kind == 0) {
        for (int k = 0; k < K; k++) {
          const int i = kern[k];
          const CreateJob& J = jobs[k];
          GP_CUDA(cudaMemcpyAsync((void*)J.off, offsets[i], 8 * (size_t)(J.n + 1), cudaMemcpyHostToDevice, s));
          if (J.m) {
            GP_CUDA(cudaMemcpyAsync((void*)J.cols, cols[i], 4 * (size_t)J.m, cudaMemcpyHostToDevice, s));
            GP_CUDA(cudaMemcpyAsync((void*)J.w, edge_cost[i], 4 * (size_t)J.m, cudaMemcpyHostToDevice, s));
          }
          if (J.n) {
            GP_CUDA(cudaMemcpyAsync((void*)J.cC, cpu_cost[i], 4 * (size_t)J.n, cudaMemcpyHostToDevice, s));
            GP_CUDA(cudaMemcpyAsync((void*)J.cG, gpu_cost[i], 4 * (size_t)J.n, cudaMemcpyHostToDevice, s));
          }
        }
      } else {
        std::vector<CopyJob> cj(K);
        for (int k = 0; k < K; k++) {
          const int i = kern[k];
          const CreateJob& J = jobs[k];
          cj[k] = CopyJob{J.n, J.m, offsets[i], cols[i], edge_cost[i], cpu_cost[i], gpu_cost[i],
                          (int64_t*)J.off, (int32_t*)J.cols, (int32_t*)J.w, (int32_t*)J.cC, (int32_t*)J.cG};
        }
        CopyJob* dcj = dnew<CopyJob>(K, s);
        GP_CUDA(cudaMemcpyAsync(dcj, cj.data(), sizeof(CopyJob) * K, cudaMemcpyHostToDevice, s));
        GP_LAUNCH(F_VALIDATE, k_copy_inputs, (unsigned)std::min<int64_t>(K, (int64_t)num_sms() * 8), 256, 0, s,
                  (const CopyJob*)dcj, K);
        GP_CHECK_LAUNCH();
        dfree(dcj, s);
      }
      // the persistent launch
      std::vector<int32_t> order(K);
      for (int k = 0; k < K; k++) order[k] = k;
      std::sort(order.begin(), order.end(), [&](int a, int b) {
        const int64_t wa = jobs[a].n + jobs[a].m, wb = jobs[b].n + jobs[b].m;
        return wa != wb ? wa > wb : a < b;
      });
      const int dsm = (kCreateThreads / 32) * kBatchWarpSmem;
      auto kernfn = k_create_batch<kCreateThreads>;
      GP_CUDA(cudaFuncSetAttribute((const void*)kernfn, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
      int per_sm = 0;
      GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernfn, kCreateThreads, dsm));
      if (per_sm < 1) throw Fail{GP_ERR_CUDA};
      const int slots = std::min(K, per_sm * num_sms());
      const unsigned long long sb = ((unsigned long long)nmax * 48ull + (1ull << 16) + 255ull) & ~255ull;
      char* ws = (char*)dalloc((size_t)slots * sb, s);
      CreateJob* djobs = dnew<CreateJob>(K, s);
      int32_t* dorder = dnew<int32_t>(K, s);
      CreateOut* dout = dnew<CreateOut>(K, s);
      unsigned* dq = dnew<unsigned>(1, s);
      GP_CUDA(cudaMemcpyAsync(djobs, jobs.data(), sizeof(CreateJob) * K, cudaMemcpyHostToDevice, s));
      GP_CUDA(cudaMemcpyAsync(dorder, order.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
      GP_CUDA(cudaMemsetAsync(dq, 0, sizeof(unsigned), s));
      GP_LAUNCH(F_BATCH, kernfn, (unsigned)slots, kCreateThreads, dsm, s, (const CreateJob*)djobs,
                (const int32_t*)dorder, K, dq, ws, sb, dout);
      GP_CHECK_LAUNCH();
      std::vector<CreateOut> hout(K);
      GP_CUDA(cudaMemcpyAsync(hout.data(), dout, sizeof(CreateOut) * K, cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaStreamSynchronize(s));
      dfree(ws, s);
      dfree(djobs, s);
      dfree(dorder, s);
      dfree(dout, s);
      dfree(dq, s);
      for (int k = 0; k < K; k++) {
        const int i = kern[k];
        const CreateOut& o = hout[k];
        status[i] = (gp_status)o.status;
        if (o.status != GP_OK) continue;
        const CreateJob& J = jobs[k];
        gp_graph* g = new gp_graph();
        g->dev = dev;
        g->n = J.n;
        g->m = J.m;
        g->a0 = o.a0;
        g->nlev = o.nlev;
        g->SC = o.SC;
        g->SG = o.SG;
        g->max_width = o.max_width;
        memset(&g->trace, 0, sizeof(g->trace));
        g->off = (int64_t*)J.off;
        g->cols = (int32_t*)J.cols;
        g->w = (int32_t*)J.w;
        g->cC = (int32_t*)J.cC;
        g->cG = (int32_t*)J.cG;
        g->in_off = J.in_off;
        g->in_src = J.in_src;
        g->in_w = J.in_w;
        g->lev_vtx = J.lev_vtx;
        g->lev_ptr = J.lev_ptr;
        g->level = J.level;
        g->lo_off = J.lo_off;
        g->lo_src = J.lo_src;
        g->lo_w = J.lo_w;
        g->lo_cC = J.lo_cC;
        g->lo_cG = J.lo_cG;
        g->L0.n = J.n;
        g->L0.cap = 2 * J.m;
        g->L0.start = J.start;
        g->L0.deg = J.deg;
        g->L0.adj = J.adj;
        g->L0.W = J.W;
        g->L0.vC = J.vC;
        g->L0.vG = J.vG;
        g->block = block;
        out[i] = g;
      }
    }
    for (int i : single) status[i] = gp_graph_create(n[i], m[i], offsets[i], cols[i], edge_cost[i], cpu_cost[i],
                                                      gpu_cost[i], ptr_kind, stream, &out[i]);
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    for (int i = 0; i < count; i++)
      if (out[i]) {
        gp_graph_destroy(out[i]);
        out[i] = nullptr;
        status[i] = f.st;
      }
    return f.st;
  }
}

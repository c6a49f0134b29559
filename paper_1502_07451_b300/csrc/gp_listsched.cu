// gp_listsched.cu -- gp_makespan_workers / gp_batch_makespan_workers: the makespan of a mapping on a
// fixed number of CPU and GPU workers (the list schedule of k_listsched.cuh), for one graph or many.
//
// This file is included at the end of gp_api.cu (the library is one translation unit).

namespace gp {

static gp_status listsched_run(int32_t count, const gp_graph* const* graphs, const uint8_t* const* parts,
                               int32_t Pc, int32_t Pg, int64_t* makespans, int64_t* finish_out, cudaStream_t s) {
  if (count < 0 || (count > 0 && (!graphs || !parts || !makespans))) return GP_ERR_INVALID;
  if (Pc < 1 || Pg < 1 || Pc + Pg > kLsMaxWorkers) return GP_ERR_INVALID;
  if (count == 0) return GP_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return GP_ERR_CUDA;
  int64_t total = 0;
  for (int32_t i = 0; i < count; i++) {
    const gp_graph* g = graphs[i];
    if (!g || g->dev != dev || (!parts[i] && g->n > 0)) return GP_ERR_INVALID;
    total += g->n;
  }
  try {
    pool_setup();
    Arena A(s);
    LsRec* rec = A.get<LsRec>(total);
    LsWait* wait = A.get<LsWait>(2 * total);
    long long* fin = A.get<long long>(total);
    std::vector<LsJob> jobs(count);
    std::vector<int> order(count);
    int64_t base = 0;
    for (int32_t i = 0; i < count; i++) {
      const gp_graph* g = graphs[i];
      const uint8_t* p = parts[i];
      if (g->n > 0 && !is_device_ptr(p)) {
        uint8_t* d = A.get<uint8_t>(g->n);
        GP_CUDA(cudaMemcpyAsync(d, p, (size_t)g->n, cudaMemcpyHostToDevice, s));
        p = d;
      }
      LsJob& J = jobs[i];
      J.n = g->n;
      J.off = g->off;
      J.cols = g->cols;
      J.w = g->w;
      J.cC = g->cC;
      J.cG = g->cG;
      J.in_off = g->in_off;
      J.part = p;
      J.rec = rec + base;
      J.wait = wait + 2 * base;
      J.fin = fin + base;
      base += g->n;
      order[i] = i;
    }
    // largest graphs first, so that the last graph a warp takes is a small one
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return graphs[a]->n + graphs[a]->m > graphs[b]->n + graphs[b]->m; });
    LsJob* djobs = A.get<LsJob>(count);
    int* dorder = A.get<int>(count);
    unsigned* queue = A.get<unsigned>(1);
    LsOut* dout = A.get<LsOut>(count);
    GP_CUDA(cudaMemcpyAsync(djobs, jobs.data(), sizeof(LsJob) * count, cudaMemcpyHostToDevice, s));
    GP_CUDA(cudaMemcpyAsync(dorder, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    GP_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned), s));
    int per_sm = 0;
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_listsched, 256, 0));
    if (per_sm < 1) per_sm = 1;
    const int64_t warps_needed = count;
    const int64_t blocks_needed = (warps_needed + 7) / 8;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    const unsigned blocks = (unsigned)(blocks_needed < cap ? blocks_needed : cap);
    GP_LAUNCH(F_LISTSCHED, k_listsched, blocks, 256, 0, s, count, (const LsJob*)djobs, (const int*)dorder, Pc, Pg,
              queue, dout);
    GP_CHECK_LAUNCH();
    std::vector<LsOut> hout(count);
    GP_CUDA(cudaMemcpyAsync(hout.data(), dout, sizeof(LsOut) * count, cudaMemcpyDeviceToHost, s));
    if (finish_out && count == 1 && graphs[0]->n > 0)
      GP_CUDA(cudaMemcpyAsync(finish_out, fin, sizeof(int64_t) * graphs[0]->n, cudaMemcpyDefault, s));
    GP_CUDA(cudaStreamSynchronize(s));
    gp_status st = GP_OK;
    for (int32_t i = 0; i < count; i++) {
      if (hout[i].status & 2) return GP_ERR_TIMEOUT;  // the event loop ran past its iteration bound
      if (hout[i].status & 1) st = GP_ERR_INVALID;
      makespans[i] = (int64_t)hout[i].makespan;
    }
    return st;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

}  // namespace gp

extern "C" gp_status gp_makespan_workers(const gp_graph* g, const uint8_t* part, int32_t workers_cpu,
                                         int32_t workers_gpu, int64_t* makespan, int64_t* finish_out,
                                         void* stream) {
  if (!g || !makespan) return GP_ERR_INVALID;
  if (g->n == 0) {
    if (workers_cpu < 1 || workers_gpu < 1 || workers_cpu + workers_gpu > kLsMaxWorkers) return GP_ERR_INVALID;
    *makespan = 0;
    return GP_OK;
  }
  const gp_graph* gs[1] = {g};
  const uint8_t* ps[1] = {part};
  return listsched_run(1, gs, ps, workers_cpu, workers_gpu, makespan, finish_out, (cudaStream_t)stream);
}

extern "C" gp_status gp_batch_makespan_workers(int32_t count, gp_graph* const* graphs, const uint8_t* const* parts,
                                               int32_t workers_cpu, int32_t workers_gpu, int64_t* makespans,
                                               void* stream) {
  return listsched_run(count, (const gp_graph* const*)graphs, parts, workers_cpu, workers_gpu, makespans, nullptr,
                       (cudaStream_t)stream);
}

// gp_noalloc.cu -- gp_makespan_noalloc: the makespan evaluation for callers that must not allocate.
//
// gp_makespan allocates its per-call scratch (one 8-byte word per vertex plus a few control words)
// from the device memory pool.  Some callers cannot do that: code that runs while a stream is being
// captured into a CUDA graph in a mode that forbids allocation, latency-critical loops where an
// allocation may stall or fail at the worst moment, and hosts that hand every byte of device memory
// to their own allocator and forbid anyone else from calling cudaMalloc.  This entry point takes its
// scratch from a fixed array compiled into the library instead, and allocates nothing.
//
// The array is a file-scope device variable: every GPU that loads the library holds it (8 MiB + 64
// bytes) until the process exits, and every call on that GPU shares it.  Two calls whose work
// overlaps on the same GPU (different streams, different host threads) would overwrite each other's
// scratch: serialise them.  Graphs with more than GP_MAKESPAN_NOALLOC_MAX_N vertices are rejected.
//
// This file is included at the end of gp_api.cu (the library is one translation unit).

namespace gp {

// words [0, 8): control (result, flags); words [8, 8 + max n): finish times
static __device__ __align__(256) unsigned long long g_noalloc_scratch[8 + GP_MAKESPAN_NOALLOC_MAX_N];

static std::mutex g_noalloc_mu;
static unsigned long long* g_noalloc_addr[64];  // device address of the array, per device

// Looks the array's device address up once per device, with that device current.  In host code the
// name g_noalloc_scratch is only a host-side stand-in, never a device address.
static gp_status noalloc_scratch(int dev, unsigned long long** out) {
  if (dev < 0 || dev >= 64) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return GP_ERR_CUDA;
    }
    g_noalloc_addr[dev] = (unsigned long long*)p;
  }
  *out = g_noalloc_addr[dev];
  return GP_OK;
}

}  // namespace gp

extern "C" gp_status gp_makespan_noalloc(const gp_graph* g, const uint8_t* part, int64_t* makespan,
                                         int64_t* finish_out, void* stream) {
  if (!g || !makespan || (!part && g->n > 0)) return GP_ERR_INVALID;
  if (g->n > GP_MAKESPAN_NOALLOC_MAX_N) return GP_ERR_INVALID;  // scratch holds at most this many
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != g->dev) return GP_ERR_INVALID;
  const int64_t n = g->n;
  if (n == 0) {
    *makespan = 0;
    return GP_OK;
  }
  {
    const gp_status ls = levels_ready(g);  // a deferred creation's levels (allocates nothing)
    if (ls != GP_OK) return ls;
  }
  // no staging copies here: the mapping and the finish times must already be device memory
  if (!is_device_ptr(part) || (finish_out && !is_device_ptr(finish_out))) return GP_ERR_INVALID;
  unsigned long long* base = nullptr;
  const gp_status st = noalloc_scratch(dev, &base);
  if (st != GP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* msp = base;                  // word 0: makespan
  int* badp = (int*)(base + 1);                    // word 1: bit 0 a part value > 1, bit 1 a wait gave up
  unsigned long long* fp = base + 8;               // finish times, written before they are read
  // the control words must start at zero; the finish area needs no clearing
  if (cudaMemsetAsync(base, 0, 8 * sizeof(unsigned long long), s) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  unsigned* grid_bar = (unsigned*)(base + 2);       // word 2: the grid kernel's barrier counter
  if (launch_makespan(g, part, fp, msp, badp, finish_out, s, grid_bar) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  unsigned long long ctl[2];
  if (cudaMemcpyAsync(ctl, base, sizeof(ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  if ((int)ctl[1] & 2) return GP_ERR_TIMEOUT;  // a bounded device wait gave up
  if ((int)ctl[1]) return GP_ERR_INVALID;
  *makespan = (int64_t)ctl[0];
  return GP_OK;
}

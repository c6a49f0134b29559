// gp_noalloc.cu -- gp_makespan_noalloc: the makespan evaluation for callers that must not allocate.
//
// gp_makespan allocates its per-call scratch (one 8-byte word per vertex plus a few control words)
// from the device memory pool.  Some callers cannot do that: hosts that hand every byte of device
// memory to their own allocator at start-up and forbid anyone else from allocating (a serving
// process that reserves the GPU's memory for its own arenas, a runtime embedding this library in a
// fixed memory budget), and latency-critical loops where an allocation may stall on the driver or
// fail at the worst moment.  This entry point takes its scratch from a fixed array compiled into the
// library instead, and allocates nothing.  It reads the result back to the host, so it synchronises
// its stream before it returns.
//
// The array is a file-scope device variable: every GPU that loads the library holds it (8 MiB + 64
// bytes) until the process exits, and every call on that GPU shares it.  Two calls whose work
// overlaps on the same GPU (different streams, different host threads) would overwrite each other's
// scratch: serialise them.  Graphs with more than GP_MAKESPAN_NOALLOC_MAX_N vertices are rejected.
//
// In host code the array's name is only a host-side stand-in.  Its device address is looked up with
// cudaGetSymbolAddress, with the device current, on the first call on that device, and again on the
// first call after that device's context was replaced (cudaDeviceReset): the address is cached per
// device together with the unique id of the context it belongs to.
//
// This file is included at the end of gp_api.cu (the library is one translation unit).
#include <cuda.h>  // driver types for the context id (entry points resolved through the runtime)

namespace gp {

// words [0, 8): control (result, flags); words [8, 8 + max n): finish times
static __device__ __align__(256) unsigned long long g_noalloc_scratch[8 + GP_MAKESPAN_NOALLOC_MAX_N];

static std::mutex g_noalloc_mu;
struct NoallocSlot {
  unsigned long long ctx_id;   // unique id of the context the address belongs to (0: none yet)
  unsigned long long* addr;    // device address of g_noalloc_scratch in that context
};
static NoallocSlot g_noalloc_slot[64];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 when none is current or the driver does not
// offer the query).
static unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)f;
    cudaGetLastError();
  });
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// The array's device address on device `dev` (current), looked up once per device and context.
static gp_status noalloc_scratch(int dev, unsigned long long** out) {
  if (dev < 0 || dev >= 64) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoallocSlot& slot = g_noalloc_slot[dev];
  const unsigned long long id = current_ctx_id();
  if (!slot.addr || id == 0 || id != slot.ctx_id) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      slot.addr = nullptr;
      return GP_ERR_CUDA;
    }
    slot.addr = (unsigned long long*)p;
    slot.ctx_id = id ? id : current_ctx_id();
  }
  *out = slot.addr;
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

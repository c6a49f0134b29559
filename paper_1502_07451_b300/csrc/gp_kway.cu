// gp_kway.cu -- gp_partition_kway: k device classes by recursive bisection on the 2-way path.
//
// The paper names a third kind of processor (an FPGA) as future work (Sec. VI) and defines neither
// its costs nor the k-class form of Eq. (1)-(2).  This project's reading: every task has one time
// per class; a group of classes acts as one device whose time for a task folds its classes' times
// like parallel resistors, comb(x, y) = floor(x*y / (x+y)) (0 when both are 0), left to right (so
// Eq. (1)'s T* for k classes is the group time of all of them, and k = 2 is the 2-way problem);
// bisect(V', [lo, hi)) splits the subgraph induced by V' between the groups [lo, mid) and [mid, hi),
// mid = lo + ceil((hi - lo) / 2), with gp_partition (Eq. (1) bounds from the two group sums), and
// recurses into both sides; one class left takes every vertex of its side.
//
// Every step runs on the device: the group times, the induced subgraph of each side (flags, an
// exclusive scan for the new ids, per-row kept counts, a scan for the row pointers, a fill), and
// each bisection through gp_graph_create_deferred + gp_partition on device arrays.  The host only
// walks the recursion (k - 1 bisections).
//
// This file is included at the end of gp_api.cu (the library is one translation unit).

namespace gp {

constexpr int kKwayMax = 255;

// comb(x, y) folded over classes [a, b) of vertex `orig`
__device__ __forceinline__ long long kway_group_time(const int32_t* __restrict__ costs, int64_t n_all,
                                                     int32_t orig, int a, int b) {
  long long t = costs[(int64_t)a * n_all + orig];
  for (int c = a + 1; c < b; c++) {
    const long long y = costs[(int64_t)c * n_all + orig];
    t = (t + y == 0) ? 0 : (long long)(((__int128)t * y) / (t + y));
  }
  return t;
}

__global__ void k_kway_group_times(int64_t n, const int32_t* __restrict__ orig, const int32_t* __restrict__ costs,
                                   int64_t n_all, int lo, int mid, int hi, int32_t* __restrict__ cA,
                                   int32_t* __restrict__ cB) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = orig ? orig[v] : (int32_t)v;
    cA[v] = (int32_t)kway_group_time(costs, n_all, o, lo, mid);
    cB[v] = (int32_t)kway_group_time(costs, n_all, o, mid, hi);
  }
}

// costs >= 0 for every class, and each class's sum (for the overflow check)
__global__ void k_kway_check(int64_t n, int k, const int32_t* __restrict__ costs, unsigned long long* sums,
                             int* bad) {
  for (int c = 0; c < k; c++) {
    unsigned long long s = 0;
    bool b = false;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
      const int32_t x = costs[(int64_t)c * n + v];
      b |= x < 0;
      s += (unsigned long long)(x > 0 ? x : 0);
    }
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) *bad = 1;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(&sums[c], s);
  }
}

__global__ void k_kway_side_flags(int64_t n, const uint8_t* __restrict__ part, int side, uint8_t* __restrict__ flag) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = part[v] == side;
}

// kept entries of each kept row (a warp per row)
__global__ void k_kway_count(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                             const uint8_t* __restrict__ part, int side, const int32_t* __restrict__ newid,
                             int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += warps) {
    if (part[v] != side) continue;
    int c = 0;
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) c += part[cols[e]] == side;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[newid[v]] = c;
  }
}

// the kept entries, renumbered, in their row order; the child's original ids
__global__ void k_kway_fill(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                            const int32_t* __restrict__ w, const uint8_t* __restrict__ part, int side,
                            const int32_t* __restrict__ newid, const int32_t* __restrict__ orig,
                            const int64_t* __restrict__ coff, int32_t* __restrict__ ccols, int32_t* __restrict__ cw,
                            int32_t* __restrict__ corig) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += warps) {
    if (part[v] != side) continue;
    const int32_t nv = newid[v];
    if (lane == 0) corig[nv] = orig ? orig[v] : (int32_t)v;
    int64_t pos = coff[nv];
    for (int64_t b = off[v]; b < off[v + 1]; b += 32) {
      const int64_t e = b + lane;
      int32_t u = -1;
      bool keep = false;
      if (e < off[v + 1]) {
        u = cols[e];
        keep = part[u] == side;
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int64_t q = pos + __popc(m & lt);
        ccols[q] = newid[u];
        cw[q] = w[e];
      }
      pos += __popc(m);
    }
  }
}

__global__ void k_kway_assign(int64_t n, const int32_t* __restrict__ orig, uint8_t cls, uint8_t* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    out[orig ? orig[v] : v] = cls;
}

// cut over directed entries with different classes, and each class's load
__global__ void k_kway_totals(int64_t n, int k, const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                              const int32_t* __restrict__ w, const int32_t* __restrict__ costs,
                              const uint8_t* __restrict__ cls, unsigned long long* cut, unsigned long long* loads) {
  unsigned long long c = 0;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
    const int64_t v = b + lane;
    int cv = -1;
    unsigned long long ld = 0;
    if (v < n) {
      cv = cls[v];
      for (int64_t e = off[v]; e < off[v + 1]; e++)
        if (cls[cols[e]] != cv) c += (unsigned long long)w[e];
      ld = (unsigned long long)costs[(int64_t)cv * n + v];
    }
    // one atomic per class present in the warp
    const unsigned grp = __match_any_sync(0xffffffffu, cv);
    unsigned long long sum = 0;
    for (unsigned gm = grp; gm; gm &= gm - 1) sum += __shfl_sync(grp, ld, __ffs(gm) - 1);
    if (cv >= 0 && lane == __ffs(grp) - 1 && sum) atomicAdd(&loads[cv], sum);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cut, c);
}

struct KwayNode {
  int64_t n, m;
  const int64_t* off;
  const int32_t* cols;
  const int32_t* w;
  const int32_t* orig;  // nullptr: identity (the root)
  int lo, hi;
};

struct KwayRun {
  int64_t n_all;
  const int32_t* costs;
  double tol;
  uint64_t seed;
  uint8_t* cls;  // device, n_all
  int32_t feasible = 1;
  int32_t bisections = 0;
  cudaStream_t s;
};

static void kway_bisect(KwayRun& R, const KwayNode& N, Arena& A) {
  cudaStream_t s = R.s;
  if (N.n == 0) return;
  if (N.hi - N.lo == 1) {
    GP_LAUNCH(F_MISC, k_kway_assign, grid_for(N.n, 256), 256, 0, s, N.n, N.orig, (uint8_t)N.lo, R.cls);
    GP_CHECK_LAUNCH();
    return;
  }
  const int mid = N.lo + (N.hi - N.lo + 1) / 2;
  int32_t* cA = A.get<int32_t>(N.n);
  int32_t* cB = A.get<int32_t>(N.n);
  GP_LAUNCH(F_MISC, k_kway_group_times, grid_for(N.n, 256), 256, 0, s, N.n, N.orig, R.costs, R.n_all, N.lo, mid,
            N.hi, cA, cB);
  GP_CHECK_LAUNCH();
  uint8_t* part = A.get<uint8_t>(N.n);
  {
    gp_graph* h = nullptr;
    gp_status st = graph_create(N.n, N.m, N.off, N.cols, N.w, cA, cB, 1, s, &h, true);
    if (st != GP_OK) throw Fail{st};
    gp_result res;
    st = gp_partition(h, -1.0, R.tol, R.seed, part, &res, s);
    graph_free(h);
    if (st != GP_OK) throw Fail{st};
    R.bisections++;
    if (!res.feasible) R.feasible = 0;
  }
  for (int side = 0; side < 2; side++) {
    uint8_t* flag = A.get<uint8_t>(N.n);
    int32_t* newid = A.get<int32_t>(N.n + 1);
    GP_LAUNCH(F_MISC, k_kway_side_flags, grid_for(N.n, 256), 256, 0, s, N.n, (const uint8_t*)part, side, flag);
    scan_u8_to_i32(flag, newid, N.n, s);
    int32_t cn = 0;
    GP_CUDA(cudaMemcpyAsync(&cn, newid + N.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    KwayNode C;
    C.lo = side ? mid : N.lo;
    C.hi = side ? N.hi : mid;
    C.n = cn;
    if (cn == 0) continue;
    int32_t* cnt = A.get<int32_t>(cn);
    int64_t* coff = A.get<int64_t>(cn + 1);
    GP_LAUNCH(F_MISC, k_kway_count, grid_for(N.n * 32, 256), 256, 0, s, N.n, N.off, N.cols, (const uint8_t*)part,
              side, (const int32_t*)newid, cnt);
    scan_i32_to_i64(cnt, coff, cn, s);
    int64_t cm = 0;
    GP_CUDA(cudaMemcpyAsync(&cm, coff + cn, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    int32_t* ccols = A.get<int32_t>(cm);
    int32_t* cw = A.get<int32_t>(cm);
    int32_t* corig = A.get<int32_t>(cn);
    GP_LAUNCH(F_MISC, k_kway_fill, grid_for(N.n * 32, 256), 256, 0, s, N.n, N.off, N.cols, N.w, (const uint8_t*)part,
              side, (const int32_t*)newid, N.orig, (const int64_t*)coff, ccols, cw, corig);
    GP_CHECK_LAUNCH();
    C.m = cm;
    C.off = coff;
    C.cols = ccols;
    C.w = cw;
    C.orig = corig;
    kway_bisect(R, C, A);
  }
}

}  // namespace gp

extern "C" gp_status gp_partition_kway(int64_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                                       const int32_t* edge_cost, int32_t k, const int32_t* costs, int ptr_kind,
                                       double tol, uint64_t seed, uint8_t* cls_out, int64_t* cut, int64_t* loads,
                                       int32_t* feasible, int32_t* bisections, void* stream) {
  if (k < 1 || k > kKwayMax || n < 0 || m < 0 || n > kMaxN || (ptr_kind != 0 && ptr_kind != 1)) return GP_ERR_INVALID;
  if (!offsets || (m > 0 && (!cols || !edge_cost)) || (n > 0 && (!costs || !cls_out)) || !cut || !loads)
    return GP_ERR_INVALID;
  if (!(tol >= 0.0 && tol <= 1.0)) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    const int64_t* d_off = offsets;
    const int32_t* d_cols = cols;
    const int32_t* d_w = edge_cost;
    const int32_t* d_costs = costs;
    if (ptr_kind == 0) {
      int64_t* o = A.get<int64_t>(n + 1);
      GP_CUDA(cudaMemcpyAsync(o, offsets, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
      d_off = o;
      if (m > 0) {
        int32_t* c = A.get<int32_t>(m);
        int32_t* w = A.get<int32_t>(m);
        GP_CUDA(cudaMemcpyAsync(c, cols, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        GP_CUDA(cudaMemcpyAsync(w, edge_cost, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        d_cols = c;
        d_w = w;
      }
      if (n > 0) {
        int32_t* c = A.get<int32_t>((int64_t)k * n);
        GP_CUDA(cudaMemcpyAsync(c, costs, sizeof(int32_t) * k * n, cudaMemcpyHostToDevice, s));
        d_costs = c;
      }
    }
    // validation in the precedence of gp_graph_create: INVALID (any class's negative cost, the CSR),
    // then OVERFLOW (a class sum above 2^61), then NOT_DAG
    unsigned long long* sums = A.get<unsigned long long>(k + 2);  // [k]: cut, [k + 1]: bad flag
    GP_CUDA(cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * (k + 2), s));
    if (n > 0)
      GP_LAUNCH(F_MISC, k_kway_check, grid_for(n, 256, 4), 256, 0, s, n, k, d_costs, sums, (int*)(sums + k + 1));
    GP_CHECK_LAUNCH();
    std::vector<unsigned long long> hs(k + 2);
    GP_CUDA(cudaMemcpyAsync(hs.data(), sums, sizeof(unsigned long long) * (k + 2), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (hs[k + 1]) return GP_ERR_INVALID;
    gp_graph* h0 = nullptr;
    // the CSR's own checks (structure, edge costs, acyclicity), with class 0's times as both costs
    const gp_status st0 = graph_create(n, m, d_off, d_cols, d_w, d_costs, d_costs, 1, s, &h0, false);
    if (h0) graph_free(h0);
    if (st0 == GP_ERR_INVALID) return st0;
    for (int c = 0; c < k; c++)
      if (hs[c] > (unsigned long long)kSumLimit) return GP_ERR_OVERFLOW;
    if (st0 != GP_OK) return st0;  // the transfers' sum (OVERFLOW), a cycle (NOT_DAG), OOM, CUDA
    const bool cls_dev = n == 0 || is_device_ptr(cls_out);
    uint8_t* d_cls = cls_dev ? cls_out : A.get<uint8_t>(n);
    KwayRun R;
    R.n_all = n;
    R.costs = d_costs;
    R.tol = tol;
    R.seed = seed;
    R.cls = d_cls;
    R.s = s;
    KwayNode root;
    root.n = n;
    root.m = m;
    root.off = d_off;
    root.cols = d_cols;
    root.w = d_w;
    root.orig = nullptr;
    root.lo = 0;
    root.hi = k;
    kway_bisect(R, root, A);
    GP_CUDA(cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * (k + 1), s));
    if (n > 0)
      GP_LAUNCH(F_MISC, k_kway_totals, grid_for(n, 256, 4), 256, 0, s, n, k, d_off, d_cols, d_w, d_costs,
                (const uint8_t*)d_cls, sums + k, sums);
    GP_CHECK_LAUNCH();
    if (!cls_dev) GP_CUDA(cudaMemcpyAsync(cls_out, d_cls, (size_t)n, cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(hs.data(), sums, sizeof(unsigned long long) * (k + 1), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < k; c++) loads[c] = (int64_t)hs[c];
    *cut = (int64_t)hs[k];
    if (feasible) *feasible = R.feasible;
    if (bisections) *bisections = R.bisections;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

// gp_mpnn.cu -- C-ABI of the learned proposal: the tensor-core GEMM step, the network, its
// training, and the learned partition.  Included at the end of gp_api.cu (one translation unit).

namespace gp {

__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ src, int64_t R, int64_t C,
                                 __nv_bfloat16* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R * C; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / C, c = i % C;
    dst[c * R + r] = src[i];
  }
}

template <int N, int K>
static gp_status step_mma(int64_t M, const void* A, const void* B, float* C, cudaStream_t s) {
  Arena ar(s);
  const int64_t Mp = (M + 127) / 128 * 128;
  __nv_bfloat16* At = ar.get<__nv_bfloat16>(Mp * K);
  __nv_bfloat16* Bt = ar.get<__nv_bfloat16>((int64_t)K * N);
  __nv_bfloat16* Bkm = ar.get<__nv_bfloat16>((int64_t)K * N);
  int* err = ar.get<int>(1);
  GP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  GP_LAUNCH(F_MPNN, k_umma_tile, grid_for(Mp * K, 256), 256, 0, s, (const __nv_bfloat16*)A, M, Mp, K, 128, At);
  GP_LAUNCH(F_MPNN, k_transpose_bf16, grid_for((int64_t)K * N, 256), 256, 0, s, (const __nv_bfloat16*)B, (int64_t)K,
            (int64_t)N, Bkm);
  GP_LAUNCH(F_MPNN, k_umma_tile, grid_for((int64_t)K * N, 256), 256, 0, s, (const __nv_bfloat16*)Bkm, (int64_t)N,
            (int64_t)N, K, N, Bt);
  GP_CHECK_LAUNCH();
  GP_CUDA((umma_gemm<N, K>(At, Bt, M, EpiStoreF32{C, N}, err, s)));
  int herr = 0;
  GP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  return herr ? GP_ERR_TIMEOUT : GP_OK;
}

}  // namespace gp

extern "C" {

gp_status gp_selftest_wait_timeout(int32_t limit_ms, void* stream) {
  if (limit_ms < 1 || limit_ms > 2000) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    int* err = A.get<int>(1);
    GP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    GP_LAUNCH(F_MISC, k_wait_selftest, 1, 128, 0, s, (uint64_t)limit_ms * 1000000ull, err);
    GP_CHECK_LAUNCH();
    int herr = 0;
    GP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    return herr ? GP_ERR_TIMEOUT : GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_step_mma_bf16(int64_t M, int32_t N, int32_t K, const void* A, const void* B, float* C, void* stream) {
  if (M < 0 || M > kMaxN || (M > 0 && (!A || !B || !C))) return GP_ERR_INVALID;
  if (M > 0 && (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C))) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    if (N == 64 && K == 192) return step_mma<64, 192>(M, A, B, C, s);
    if (N == 192 && K == 64) return step_mma<192, 64>(M, A, B, C, s);
    if (N == 64 && K == 64) return step_mma<64, 64>(M, A, B, C, s);
    return GP_ERR_INVALID;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// The network: parameters, forward, backward, Adam; the learned partition.
// ------------------------------------------------------------------------------------------------
struct gp_model {
  int dev = 0;
  float* P = nullptr;  // FP32 master parameters
  float* m = nullptr;  // Adam moments
  float* v = nullptr;
  float* g = nullptr;  // last gradient
  __nv_bfloat16* Wf = nullptr;  // tiled BF16 layer weights, forward operand (3 x 64 x 192)
  __nv_bfloat16* Wb = nullptr;  // backward operand (3 x 192 x 64)
  int64_t step = 0;
};

namespace gp {

constexpr int64_t kWPer = (int64_t)kCat * kHid;

static void model_free(gp_model* M) {
  if (!M) return;
  cudaFree(M->P);
  cudaFree(M->m);
  cudaFree(M->v);
  cudaFree(M->g);
  cudaFree(M->Wf);
  cudaFree(M->Wb);
  delete M;
}

static gp_status model_alloc(gp_model** out) {
  gp_model* M = new gp_model();
  M->dev = device_id();
  if (cudaMalloc(&M->P, sizeof(float) * kPN) != cudaSuccess || cudaMalloc(&M->m, sizeof(float) * kPN) != cudaSuccess ||
      cudaMalloc(&M->v, sizeof(float) * kPN) != cudaSuccess || cudaMalloc(&M->g, sizeof(float) * kPN) != cudaSuccess ||
      cudaMalloc(&M->Wf, sizeof(__nv_bfloat16) * 3 * kWPer) != cudaSuccess ||
      cudaMalloc(&M->Wb, sizeof(__nv_bfloat16) * 3 * kWPer) != cudaSuccess) {
    cudaGetLastError();
    model_free(M);
    return GP_ERR_OOM;
  }
  *out = M;
  return GP_OK;
}

// upload parameters (and moments, or zeros), rebuild the tiled weights
static void model_upload(gp_model* M, const float* P, const float* m, const float* v, cudaStream_t s) {
  GP_CUDA(cudaMemcpyAsync(M->P, P, sizeof(float) * kPN, cudaMemcpyHostToDevice, s));
  if (m)
    GP_CUDA(cudaMemcpyAsync(M->m, m, sizeof(float) * kPN, cudaMemcpyHostToDevice, s));
  else
    GP_CUDA(cudaMemsetAsync(M->m, 0, sizeof(float) * kPN, s));
  if (v)
    GP_CUDA(cudaMemcpyAsync(M->v, v, sizeof(float) * kPN, cudaMemcpyHostToDevice, s));
  else
    GP_CUDA(cudaMemsetAsync(M->v, 0, sizeof(float) * kPN, s));
  GP_CUDA(cudaMemsetAsync(M->g, 0, sizeof(float) * kPN, s));
  GP_LAUNCH(F_MPNN, k_mp_tile_weights, 96, 256, 0, s, M->P, M->Wf, M->Wb);
  GP_CHECK_LAUNCH();
  GP_CUDA(cudaStreamSynchronize(s));
}

// He-normal initial weights from a counter-based generator (splitmix64, Box-Muller), zero biases
static void model_init_host(uint64_t seed, std::vector<float>& P) {
  P.assign((size_t)kPN, 0.0f);
  uint64_t ctr = 0;
  auto unif = [&]() {
    const uint64_t z = mix64(seed + 0x9E3779B97F4A7C15ULL * (++ctr));
    return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int64_t off, int64_t count, double sd) {
    for (int64_t i = 0; i < count; i += 2) {
      const double u1 = unif(), u2 = unif();
      const double r = std::sqrt(-2.0 * std::log(u1));
      P[(size_t)(off + i)] = (float)(sd * r * std::cos(6.283185307179586 * u2));
      if (i + 1 < count) P[(size_t)(off + i + 1)] = (float)(sd * r * std::sin(6.283185307179586 * u2));
    }
  };
  fill(kPWin, kNFeat * kHid, std::sqrt(2.0 / kNFeat));
  for (int l = 1; l <= 3; l++) fill(p_W(l), kWPer, std::sqrt(2.0 / kCat));
  fill(kPWo, kHid, std::sqrt(1.0 / kHid));
}

// Sorts the handle's in-rows by (source, cost) once, so that the network's FP32 neighbour sums run
// in a fixed order (the transpose fills rows in no particular order).
static void mp_prepare(const gp_graph* gc, cudaStream_t s) {
  gp_graph* g = const_cast<gp_graph*>(gc);
  // the sort below permutes the in-rows in place, and a deferred creation's level-ordered in-CSR build
  // (on the side stream) reads them: wait for it first
  const gp_status ls = levels_ready(g);
  if (ls != GP_OK) throw Fail{ls};
  if (g->in_sorted || g->n == 0 || g->m == 0) {
    g->in_sorted = true;
    return;
  }
  Arena A(s);
  int32_t* long_rows = A.get<int32_t>(g->n);
  unsigned* cnt = A.get<unsigned>(1);
  unsigned long long* ta = A.get<unsigned long long>(g->m);
  unsigned long long* tb = A.get<unsigned long long>(g->m);
  GP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned), s));
  GP_LAUNCH(F_MPNN, k_sort_rows_short, grid_for(g->n * 32, 256), 256, 0, s, g->n, (const int64_t*)g->in_off,
            g->in_src, g->in_w, long_rows, cnt);
  GP_LAUNCH(F_MPNN, k_sort_rows_long, (unsigned)num_sms(), 1024, 0, s, (const int64_t*)g->in_off, g->in_src,
            g->in_w, (const int32_t*)long_rows, (const unsigned*)cnt, ta, tb);
  GP_CHECK_LAUNCH();
  g->in_sorted = true;
}

static MpGraph mp_graph(const gp_graph* g) {
  const gp_status ls = levels_ready(g);  // the features read the levels
  if (ls != GP_OK) throw Fail{ls};
  MpGraph G;
  G.n = g->n;
  G.m = g->m;
  G.off = g->off;
  G.cols = g->cols;
  G.w = g->w;
  G.in_off = g->in_off;
  G.in_src = g->in_src;
  G.in_w = g->in_w;
  G.cC = g->cC;
  G.cG = g->cG;
  G.level = g->level;
  G.nlev = g->nlev;
  G.levf = nullptr;
  return G;
}

struct MpWork {
  int64_t n = 0, np = 0;
  float *X = nullptr, *inv_in = nullptr, *inv_out = nullptr, *e_out = nullptr, *e_in = nullptr;
  __nv_bfloat16* H[4] = {nullptr, nullptr, nullptr, nullptr};
  __nv_bfloat16* Ct[3] = {nullptr, nullptr, nullptr};
  float *logit = nullptr, *dlogit = nullptr;
  double *loss_part = nullptr, *loss = nullptr;
  float *dZ = nullptr, *dC = nullptr, *part = nullptr;
  __nv_bfloat16* dZt = nullptr;
  int* err = nullptr;
  int nblk_logit = 1, nblk_dw = 1;
};

static void mp_work(MpWork& W, const MpGraph& G, bool train, Arena& A, cudaStream_t s) {
  const int64_t n = G.n, np = (n + 127) / 128 * 128, m = G.m;
  W.n = n;
  W.np = np;
  W.X = A.get<float>(n * kNFeat);
  W.inv_in = A.get<float>(n);
  W.inv_out = A.get<float>(n);
  W.e_out = A.get<float>(m);
  W.e_in = A.get<float>(m);
  const int nh = train ? 4 : 2, nc = train ? 3 : 1;
  for (int i = 0; i < nh; i++) W.H[i] = A.get<__nv_bfloat16>(n * kHid);
  for (int i = 0; i < nc; i++) W.Ct[i] = A.get<__nv_bfloat16>(np * kCat);
  W.logit = A.get<float>(n);
  W.err = A.get<int>(1);
  GP_CUDA(cudaMemsetAsync(W.err, 0, sizeof(int), s));
  W.nblk_logit = (int)grid_for(n, 256, 4);
  if (train) {
    W.dlogit = A.get<float>(n);
    W.loss_part = A.get<double>(W.nblk_logit);
    W.loss = A.get<double>(1);
    W.dZ = A.get<float>(n * kHid);
    W.dZt = A.get<__nv_bfloat16>(np * kHid);
    W.dC = A.get<float>(n * kCat);
    const int64_t want = (n + kDwStage - 1) / kDwStage;
    const int64_t cap = (int64_t)num_sms() * 2;
    W.nblk_dw = (int)(want < 1 ? 1 : (want < cap ? want : cap));
    W.part = A.get<float>((int64_t)W.nblk_dw * (kCat + 1) * kHid);
  }
}

// logits of every vertex into W.logit (and, with labels, dlogit and the summed loss)
static void mp_forward(const gp_model* M, const MpGraph& G, MpWork& W, const uint8_t* label, bool train,
                       cudaStream_t s) {
  const int64_t n = G.n;
  const int64_t vm = n > G.m ? n : G.m;
  GP_LAUNCH(F_MPNN, k_mp_prep, grid_for(vm, 256), 256, 0, s, G, W.X, W.inv_in, W.inv_out, W.e_out, W.e_in);
  GP_LAUNCH(F_MPNN, k_mp_input, grid_for(n * kHid, 256), 256, 0, s, n, (const float*)W.X, (const float*)M->P, W.H[0]);
  GP_CHECK_LAUNCH();
  for (int l = 1; l <= 3; l++) {
    __nv_bfloat16* Ct = train ? W.Ct[l - 1] : W.Ct[0];
    const __nv_bfloat16* Hin = train ? W.H[l - 1] : W.H[(l - 1) & 1];
    __nv_bfloat16* Hout = train ? W.H[l] : W.H[l & 1];
    GP_LAUNCH(F_MPNN, k_mp_aggregate, grid_for(n * 32, 256), 256, 0, s, G, (const float*)W.inv_in,
              (const float*)W.inv_out, (const float*)W.e_out, (const float*)W.e_in, Hin, Ct);
    GP_CHECK_LAUNCH();
    GP_CUDA((umma_gemm<kHid, kCat>(Ct, M->Wf + (l - 1) * kWPer, n, EpiRelu{M->P + p_b(l), Hout}, W.err, s)));
  }
  const __nv_bfloat16* H3 = train ? W.H[3] : W.H[1];
  GP_LAUNCH(F_MPNN, k_mp_logits, W.nblk_logit, 256, 0, s, n, H3, (const float*)M->P, W.logit, label, W.dlogit,
            label ? W.loss_part : nullptr);
  if (label) GP_LAUNCH(F_MPNN, k_sum_parts, 1, 32, 0, s, W.nblk_logit, (const double*)W.loss_part, W.loss);
  GP_CHECK_LAUNCH();
}

// parameter gradient of the mean loss into grad (device, kPN floats)
static void mp_backward(const gp_model* M, const MpGraph& G, MpWork& W, float* grad, cudaStream_t s) {
  const int64_t n = G.n;
  const float scale = 1.0f / (float)n;
  GP_LAUNCH(F_MPNN, k_mp_dout, kHid + 1, 256, 0, s, n, (const float*)W.dlogit, (const __nv_bfloat16*)W.H[3], scale,
            grad);
  GP_LAUNCH(F_MPNN, k_mp_dz_top, grid_for(n * (kHid / 2), 256), 256, 0, s, n, (const float*)W.dlogit,
            (const float*)M->P, (const __nv_bfloat16*)W.H[3], W.dZ, W.dZt);
  GP_CHECK_LAUNCH();
  for (int l = 3; l >= 1; l--) {
    GP_LAUNCH(F_MPNN, k_mp_dw<kCat>, W.nblk_dw, 256, 0, s, n, (const __nv_bfloat16*)W.Ct[l - 1], (const float*)nullptr,
              (const float*)W.dZ, W.part);
    GP_LAUNCH(F_MPNN, k_mp_dw_reduce, grid_for((kCat + 1) * kHid, 256), 256, 0, s, W.nblk_dw, kCat,
              (const float*)W.part, scale, grad, p_W(l), p_b(l));
    GP_CHECK_LAUNCH();
    GP_CUDA((umma_gemm<kCat, kHid>(W.dZt, M->Wb + (l - 1) * kWPer, n, EpiStoreF32{W.dC, kCat}, W.err, s)));
    GP_LAUNCH(F_MPNN, k_mp_agg_back, grid_for(n * 32, 256), 256, 0, s, G, (const float*)W.inv_in,
              (const float*)W.inv_out, (const float*)W.e_out, (const float*)W.e_in, (const float*)W.dC,
              (const __nv_bfloat16*)W.H[l - 1], W.dZ, l - 1 >= 1 ? W.dZt : (__nv_bfloat16*)nullptr);
    GP_CHECK_LAUNCH();
  }
  GP_LAUNCH(F_MPNN, k_mp_dw<kNFeat>, W.nblk_dw, 256, 0, s, n, (const __nv_bfloat16*)nullptr, (const float*)W.X,
            (const float*)W.dZ, W.part);
  GP_LAUNCH(F_MPNN, k_mp_dw_reduce, grid_for((kNFeat + 1) * kHid, 256), 256, 0, s, W.nblk_dw, kNFeat,
            (const float*)W.part, scale, grad, kPWin, kPBin);
  GP_CHECK_LAUNCH();
}

static const uint8_t* device_labels(const uint8_t* labels, int64_t n, Arena& A, cudaStream_t s) {
  if (is_device_ptr(labels)) return labels;
  uint8_t* d = A.get<uint8_t>(n);
  GP_CUDA(cudaMemcpyAsync(d, labels, (size_t)n, cudaMemcpyHostToDevice, s));
  return d;
}

static gp_status mp_check(const gp_model* M, const gp_graph* g) {
  if (!M || !g) return GP_ERR_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != g->dev || dev != M->dev) return GP_ERR_INVALID;
  return GP_OK;
}

// the split proposed by the logits (device), into part (device)
static void propose_split(const gp_graph* g, const float* logit, int64_t BC, int64_t BG, uint8_t* part, Arena& A,
                          cudaStream_t s) {
  const int64_t n = g->n;
  unsigned long long* key = A.get<unsigned long long>(n);
  unsigned long long* hist = A.get<unsigned long long>(1024);
  PropSel* dsel = A.get<PropSel>(1);
  PropSel hs;
  memset(&hs, 0, sizeof(hs));
  const int64_t D = g->SG - BG;  // GPU load that has to leave
  hs.rem[0] = BC;
  hs.rem[1] = D > 0 ? D - 1 : 0;
  hs.active[0] = 1;
  hs.active[1] = D > 0 ? 1 : 0;
  GP_CUDA(cudaMemcpyAsync(dsel, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
  GP_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 1024, s));
  GP_LAUNCH(F_PROPOSE, k_prop_keys, grid_for(n, 256), 256, 0, s, n, logit, key, dsel);
  for (int p = 0; p < 8; p++) {
    const int shift = 56 - 8 * p;
    GP_LAUNCH(F_PROPOSE, k_prop_hist, grid_for(n, 256, 4), 256, 0, s, n, (const unsigned long long*)key,
              (const int64_t*)g->L0.vC, (const int64_t*)g->L0.vG, (const PropSel*)dsel, shift, hist);
    GP_LAUNCH(F_PROPOSE, k_prop_pick, 1, 64, 0, s, dsel, shift, hist);
  }
  GP_CHECK_LAUNCH();
  GP_CUDA(cudaMemcpyAsync(&hs, dsel, sizeof(hs), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  if (hs.bad) throw Fail{GP_ERR_INVALID};
  const int64_t kC = hs.found[0] ? (int64_t)hs.less[0] : n;
  const int64_t kG = D <= 0 ? 0 : (hs.found[1] ? (int64_t)hs.less[1] + 1 : n);
  const int64_t k = kC < kG ? kC : kG;
  int mode;
  unsigned long long thr = 0;
  if (k == 0) {
    mode = 0;
  } else if (k >= n) {
    mode = 1;
  } else if (kC <= kG) {
    mode = 2;
    thr = hs.prefix[0];
  } else {
    mode = 3;
    thr = hs.prefix[1];
  }
  GP_LAUNCH(F_PROPOSE, k_prop_assign, grid_for(n, 256), 256, 0, s, n, (const unsigned long long*)key, thr, mode, part);
  GP_CHECK_LAUNCH();
}

}  // namespace gp

extern "C" {

gp_status gp_model_create(uint64_t seed, gp_model** out) {
  if (!out) return GP_ERR_INVALID;
  *out = nullptr;
  gp_model* M = nullptr;
  gp_status st = model_alloc(&M);
  if (st != GP_OK) return st;
  try {
    std::vector<float> P;
    model_init_host(seed, P);
    model_upload(M, P.data(), nullptr, nullptr, (cudaStream_t)0);
    *out = M;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    model_free(M);
    return f.st;
  }
}

gp_status gp_model_destroy(gp_model* M) {
  if (!M) return GP_ERR_INVALID;
  cudaDeviceSynchronize();
  model_free(M);
  return GP_OK;
}

int64_t gp_model_param_count(void) { return kPN; }

gp_status gp_model_get_params(const gp_model* M, float* params) {
  if (!M || !params) return GP_ERR_INVALID;
  if (cudaMemcpy(params, M->P, sizeof(float) * kPN, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  return GP_OK;
}

gp_status gp_model_set_params(gp_model* M, const float* params) {
  if (!M || !params) return GP_ERR_INVALID;
  for (int64_t i = 0; i < kPN; i++)
    if (!std::isfinite(params[i])) return GP_ERR_INVALID;
  try {
    model_upload(M, params, nullptr, nullptr, (cudaStream_t)0);
    M->step = 0;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

static const char kModelMagic[8] = {'G', 'P', 'M', 'P', 'N', 'N', '0', '1'};

// Checkpoint layout (little-endian): magic "GPMPNN01", uint32 version, uint32 parameter count, int64
// Adam step, float32 parameters / first moments / second moments, and from version 2 on a uint64
// FNV-1a (64-bit) checksum of every byte after the magic up to the checksum.  Version 1 files (no
// checksum) still load.
static uint64_t fnv1a64(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 0x100000001b3ULL;
  }
  return h;
}
static const uint64_t kFnvBasis = 0xcbf29ce484222325ULL;

gp_status gp_model_save(const gp_model* M, const char* path) {
  if (!M || !path) return GP_ERR_INVALID;
  std::vector<float> buf((size_t)kPN * 3);
  if (cudaMemcpy(buf.data(), M->P, sizeof(float) * kPN, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + kPN, M->m, sizeof(float) * kPN, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + 2 * kPN, M->v, sizeof(float) * kPN, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  FILE* f = fopen(path, "wb");
  if (!f) return GP_ERR_INVALID;
  const uint32_t ver = 2, np = (uint32_t)kPN;
  const int64_t step = M->step;
  uint64_t h = kFnvBasis;
  h = fnv1a64(h, &ver, 4);
  h = fnv1a64(h, &np, 4);
  h = fnv1a64(h, &step, 8);
  h = fnv1a64(h, buf.data(), sizeof(float) * buf.size());
  bool ok = fwrite(kModelMagic, 1, 8, f) == 8 && fwrite(&ver, 4, 1, f) == 1 && fwrite(&np, 4, 1, f) == 1 &&
            fwrite(&step, 8, 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size() &&
            fwrite(&h, 8, 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  return ok ? GP_OK : GP_ERR_INVALID;
}

gp_status gp_model_load(const char* path, gp_model** out) {
  if (!path || !out) return GP_ERR_INVALID;
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return GP_ERR_INVALID;
  char mg[8];
  uint32_t ver = 0, np = 0;
  int64_t step = 0;
  uint64_t sum = 0;
  std::vector<float> buf((size_t)kPN * 3);
  bool ok = fread(mg, 1, 8, f) == 8 && memcmp(mg, kModelMagic, 8) == 0 && fread(&ver, 4, 1, f) == 1 &&
            (ver == 1 || ver == 2) && fread(&np, 4, 1, f) == 1 && np == (uint32_t)kPN && fread(&step, 8, 1, f) == 1 &&
            fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  if (ok && ver == 2) {
    ok = fread(&sum, 8, 1, f) == 1;
    uint64_t h = kFnvBasis;
    h = fnv1a64(h, &ver, 4);
    h = fnv1a64(h, &np, 4);
    h = fnv1a64(h, &step, 8);
    h = fnv1a64(h, buf.data(), sizeof(float) * buf.size());
    ok = ok && h == sum;
  }
  if (ok) {  // nothing may follow
    char extra;
    ok = fread(&extra, 1, 1, f) == 0;
  }
  fclose(f);
  if (!ok) return GP_ERR_INVALID;
  for (float x : buf)
    if (!std::isfinite(x)) return GP_ERR_INVALID;
  gp_model* M = nullptr;
  gp_status st = model_alloc(&M);
  if (st != GP_OK) return st;
  try {
    model_upload(M, buf.data(), buf.data() + kPN, buf.data() + 2 * kPN, (cudaStream_t)0);
    M->step = step;
    *out = M;
    return GP_OK;
  } catch (Fail& e) {
    cudaGetLastError();
    model_free(M);
    return e.st;
  }
}

gp_status gp_model_forward(const gp_model* M, const gp_graph* g, float* logits_out, void* stream) {
  gp_status st = mp_check(M, g);
  if (st != GP_OK) return st;
  if (g->n > 0 && !logits_out) return GP_ERR_INVALID;
  if (g->n == 0) return GP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    MpWork W;
    mp_prepare(g, s);
    const MpGraph G = mp_graph(g);
    mp_work(W, G, false, A, s);
    mp_forward(M, G, W, nullptr, false, s);
    GP_CUDA(cudaMemcpyAsync(logits_out, W.logit, sizeof(float) * g->n, cudaMemcpyDefault, s));
    int herr = 0;
    GP_CUDA(cudaMemcpyAsync(&herr, W.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    return herr ? GP_ERR_TIMEOUT : GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

// forward + backward (+ Adam when lr > 0); grad_out (host, nullable), loss_out (host, nullable)
static gp_status model_step(gp_model* M, const gp_graph* g, const uint8_t* labels, float lr, float* grad_out,
                            double* loss_out, cudaStream_t s) {
  gp_status st = mp_check(M, g);
  if (st != GP_OK) return st;
  if (g->n <= 0 || !labels) return GP_ERR_INVALID;
  try {
    pool_setup();
    Arena A(s);
    MpWork W;
    mp_prepare(g, s);
    const MpGraph G = mp_graph(g);
    mp_work(W, G, true, A, s);
    const uint8_t* lab = device_labels(labels, g->n, A, s);
    mp_forward(M, G, W, lab, true, s);
    mp_backward(M, G, W, M->g, s);
    if (lr > 0.0f) {
      M->step += 1;
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.0f - (float)std::pow((double)b1, (double)M->step);
      const float c2 = 1.0f - (float)std::pow((double)b2, (double)M->step);
      GP_LAUNCH(F_MPNN, k_adam, grid_for(kPN, 256), 256, 0, s, kPN, M->P, (const float*)M->g, M->m, M->v, lr, b1, b2,
                1e-8f, c1, c2);
      GP_LAUNCH(F_MPNN, k_mp_tile_weights, 96, 256, 0, s, (const float*)M->P, M->Wf, M->Wb);
      GP_CHECK_LAUNCH();
    }
    double loss = 0.0;
    int herr = 0;
    GP_CUDA(cudaMemcpyAsync(&loss, W.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(&herr, W.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (grad_out) GP_CUDA(cudaMemcpyAsync(grad_out, M->g, sizeof(float) * kPN, cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (herr) return GP_ERR_TIMEOUT;
    if (loss_out) *loss_out = loss / (double)g->n;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_model_grad(gp_model* M, const gp_graph* g, const uint8_t* labels, float* grad_out, double* loss_out,
                        void* stream) {
  if (!grad_out) return GP_ERR_INVALID;
  return model_step(M, g, labels, 0.0f, grad_out, loss_out, (cudaStream_t)stream);
}

gp_status gp_model_train_step(gp_model* M, const gp_graph* g, const uint8_t* labels, float lr, double* loss_out,
                              void* stream) {
  if (!(lr > 0.0f) || !std::isfinite(lr)) return GP_ERR_INVALID;
  return model_step(M, g, labels, lr, nullptr, loss_out, (cudaStream_t)stream);
}

gp_status gp_partition_learned(gp_graph* g, const gp_model* M, const float* logits, double r_cpu, double tol,
                               uint8_t* part_out, gp_result* res, void* stream) {
  if (!g || (!M && !logits) || (!part_out && g->n > 0)) return GP_ERR_INVALID;
  if (M) {
    gp_status st = mp_check(M, g);
    if (st != GP_OK) return st;
  }
  int64_t BC, BG;
  gp_status st = host_bounds(g->SC, g->SG, r_cpu, tol, &BC, &BG);
  if (st != GP_OK) return st;
  gp_result R;
  memset(&R, 0, sizeof(R));
  R.bound_cpu = BC;
  R.bound_gpu = BG;
  const int64_t n = g->n;
  if (n == 0) {
    R.feasible = 1;
    if (res) *res = R;
    return GP_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    const bool prof = prof_on();
    if (prof)
      for (auto& e : ev) cudaEventCreate(&e);
    if (prof) cudaEventRecord(ev[0], s);
    float* lg = A.get<float>(n);
    int herr = 0;
    if (logits) {
      GP_CUDA(cudaMemcpyAsync(lg, logits, sizeof(float) * n, cudaMemcpyDefault, s));
    } else {
      MpWork W;
      mp_prepare(g, s);
      const MpGraph G = mp_graph(g);
      mp_work(W, G, false, A, s);
      mp_forward(M, G, W, nullptr, false, s);
      GP_CUDA(cudaMemcpyAsync(lg, W.logit, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
      GP_CUDA(cudaMemcpyAsync(&herr, W.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    if (prof) cudaEventRecord(ev[1], s);
    uint8_t* part = A.get<uint8_t>(n);
    propose_split(g, lg, BC, BG, part, A, s);  // synchronises
    if (herr) return GP_ERR_TIMEOUT;
    if (prof) cudaEventRecord(ev[2], s);
    // refinement of level 0 only (flat mode)
    Ctl* ctl = A.get<Ctl>(1);
    Ctl hc;
    memset(&hc, 0, sizeof(hc));
    hc.BC = BC;
    hc.BG = BG;
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
    GP_CUDA(cudaMemsetAsync(cand.stamp, 0xff, sizeof(int32_t) * n, s));
    refine_loads(g->L0, part, ctl, s);
    // one cooperative grid launch for the level (a launch per step where the grid does not fit)
    int* terr = A.get<int>(1);
    GP_CUDA(cudaMemsetAsync(terr, 0, sizeof(int), s));
    {
      TailArgs ta;
      memset(&ta, 0, sizeof(ta));
      ta.lev[0].g = g->L0;
      ta.lev[0].part = part;
      ta.lev[0].G = group_for_degree(0.25 * (double)g->a0 / (double)n);
      ta.lev[0].idbits = idbits_for(n);
      int32_t* t_rounds = A.get<int32_t>(1);
      int32_t* t_bal = A.get<int32_t>(1);
      long long* t_moves = A.get<long long>(1);
      long long* t_balmoves = A.get<long long>(1);
      unsigned* bar = A.get<unsigned>(1);
      GP_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
      if (!launch_refine_grid(ta, ctl, cand, t_rounds, t_moves, t_bal, t_balmoves, bar, terr, g->lev_event, s))
        refine_level_run(g->L0, part, ctl, cand, 0, (double)g->a0 / (double)n, s);
    }
    unsigned long long* cut = A.get<unsigned long long>(1);
    int* bad = A.get<int>(1);
    GP_CUDA(cudaMemsetAsync(cut, 0, sizeof(unsigned long long), s));
    GP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    launch_cut(n, g->m, g->off, g->cols, g->w, part, cut, bad, s);
    GP_CHECK_LAUNCH();
    GP_CUDA(cudaMemcpyAsync(part_out, part, (size_t)n, cudaMemcpyDefault, s));
    if (prof) cudaEventRecord(ev[3], s);
    unsigned long long hcut = 0;
    int hterr = 0;
    GP_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(&hcut, cut, sizeof(hcut), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(&hterr, terr, sizeof(int), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (hterr) return GP_ERR_TIMEOUT;
    R.cut = (int64_t)hcut;
    R.load_cpu = hc.LC;
    R.load_gpu = hc.LG;
    R.feasible = (hc.LC <= BC && hc.LG <= BG) ? 1 : 0;
    R.levels = 0;
    R.rounds = hc.rounds;
    R.coarsest_n = (int32_t)n;
    if (prof) {
      for (int i = 0; i < 3; i++) cudaEventElapsedTime(&R.ms[i], ev[i], ev[i + 1]);
      for (auto& e : ev) cudaEventDestroy(e);
    }
    if (res) *res = R;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

gp_status gp_partition_learned_vcycle(gp_graph* g, const gp_model* M, const float* logits, double r_cpu,
                                      double tol, uint64_t seed, uint8_t* part_out, gp_result* res, void* stream) {
  if (!g || (!M && !logits) || (!part_out && g->n > 0)) return GP_ERR_INVALID;
  if (M) {
    gp_status st = mp_check(M, g);
    if (st != GP_OK) return st;
  }
  int64_t BC, BG;
  gp_status st = host_bounds(g->SC, g->SG, r_cpu, tol, &BC, &BG);
  if (st != GP_OK) return st;
  const int64_t n = g->n;
  if (n == 0) return partition_impl(g, nullptr, r_cpu, tol, seed, part_out, res, stream);
  cudaStream_t s = (cudaStream_t)stream;
  try {
    pool_setup();
    Arena A(s);
    const bool prof = prof_on();
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (prof) {
      for (auto& e : ev) cudaEventCreate(&e);
      cudaEventRecord(ev[0], s);
    }
    float* lg = A.get<float>(n);
    int herr = 0;
    if (logits) {
      GP_CUDA(cudaMemcpyAsync(lg, logits, sizeof(float) * n, cudaMemcpyDefault, s));
    } else {
      MpWork W;
      mp_prepare(g, s);
      const MpGraph G = mp_graph(g);
      mp_work(W, G, false, A, s);
      mp_forward(M, G, W, nullptr, false, s);
      GP_CUDA(cudaMemcpyAsync(lg, W.logit, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
      GP_CUDA(cudaMemcpyAsync(&herr, W.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    uint8_t* prop = A.get<uint8_t>(n);
    propose_split(g, lg, BC, BG, prop, A, s);  // synchronises
    if (herr) return GP_ERR_TIMEOUT;
    float net_ms = 0.0f;
    if (prof) {
      cudaEventRecord(ev[1], s);
      cudaEventSynchronize(ev[1]);
      cudaEventElapsedTime(&net_ms, ev[0], ev[1]);
      for (auto& e : ev) cudaEventDestroy(e);
    }
    // the proposed sides (0 / 1) pin every vertex for the matching only
    gp_result R;
    st = partition_impl(g, (const int8_t*)prop, r_cpu, tol, seed, part_out, &R, stream, true);
    if (st != GP_OK) return st;
    R.ms[4] = net_ms;
    if (res) *res = R;
    return GP_OK;
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// The learned path for many graphs: one network forward over their disjoint union, then the
// persistent batch kernel in learned mode (proposal + refinement of level 0 per graph).
// ------------------------------------------------------------------------------------------------
namespace gp {

// Logits of every vertex of the graphs `sel` (all with n > 0) into one device buffer; base[i] is
// graph sel[i]'s first vertex.
static float* mp_union_logits(const gp_model* M, gp_graph* const* graphs, const std::vector<int>& sel,
                              std::vector<int64_t>& base, Arena& A, cudaStream_t s, int* err_dev) {
  const int K = (int)sel.size();
  std::vector<MpPiece> pieces(K);
  int64_t N = 0, Mtot = 0;
  base.assign(K, 0);
  int32_t maxlev = 0;
  for (int i = 0; i < K; i++) {
    const gp_status ls = levels_ready(graphs[sel[i]]);  // the features read the levels
    if (ls != GP_OK) throw Fail{ls};
  }
  for (int i = 0; i < K; i++) mp_prepare(graphs[sel[i]], s);
  for (int i = 0; i < K; i++) {
    const gp_graph* g = graphs[sel[i]];
    MpPiece& P = pieces[i];
    P.n = g->n;
    P.m = g->m;
    P.vb = N;
    P.eb = Mtot;
    P.off = g->off;
    P.cols = g->cols;
    P.w = g->w;
    P.in_off = g->in_off;
    P.in_src = g->in_src;
    P.in_w = g->in_w;
    P.cC = g->cC;
    P.cG = g->cG;
    P.level = g->level;
    P.nlev = g->nlev;
    base[i] = N;
    N += g->n;
    Mtot += g->m;
    maxlev = std::max(maxlev, g->nlev);
  }
  if (N > kMaxN || Mtot >= ((int64_t)1 << 31)) throw Fail{GP_ERR_INVALID};  // int32 ids in the union
  MpPiece* dp = A.get<MpPiece>(K);
  GP_CUDA(cudaMemcpyAsync(dp, pieces.data(), sizeof(MpPiece) * K, cudaMemcpyHostToDevice, s));
  MpGraph G;
  G.n = N;
  G.m = Mtot;
  int64_t* off = A.get<int64_t>(N + 1);
  int32_t* cols = A.get<int32_t>(Mtot);
  int32_t* w = A.get<int32_t>(Mtot);
  int64_t* in_off = A.get<int64_t>(N + 1);
  int32_t* in_src = A.get<int32_t>(Mtot);
  int32_t* in_w = A.get<int32_t>(Mtot);
  int32_t* cC = A.get<int32_t>(N);
  int32_t* cG = A.get<int32_t>(N);
  int32_t* level = A.get<int32_t>(N);
  float* levf = A.get<float>(N);
  GP_LAUNCH(F_MPNN, k_mp_union, (unsigned)std::min<int64_t>(K, (int64_t)num_sms() * 8), 256, 0, s,
            (const MpPiece*)dp, K, off, cols, w, in_off, in_src, in_w, cC, cG, level, levf);
  GP_LAUNCH(F_MPNN, k_mp_union_tail, 1, 1, 0, s, N, Mtot, off, in_off);
  GP_CHECK_LAUNCH();
  G.off = off;
  G.cols = cols;
  G.w = w;
  G.in_off = in_off;
  G.in_src = in_src;
  G.in_w = in_w;
  G.cC = cC;
  G.cG = cG;
  G.level = level;
  G.nlev = maxlev;
  G.levf = levf;
  MpWork W;
  mp_work(W, G, false, A, s);
  mp_forward(M, G, W, nullptr, false, s);
  GP_CUDA(cudaMemcpyAsync(err_dev, W.err, sizeof(int), cudaMemcpyDeviceToDevice, s));
  return W.logit;
}

}  // namespace gp

extern "C" gp_status gp_batch_partition_learned(int32_t count, gp_graph* const* graphs, const gp_model* M,
                                                const double* r_cpu, double tol, uint8_t* const* parts,
                                                gp_result* res, int64_t* makespans, void* stream) {
  if (count < 0 || (count > 0 && (!graphs || !M))) return GP_ERR_INVALID;
  if (count == 0) return GP_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || dev != M->dev) return GP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> sel;
  for (int i = 0; i < count; i++) {
    if (!graphs[i] || graphs[i]->dev != dev) return GP_ERR_INVALID;
    if (graphs[i]->n > 0) sel.push_back(i);
  }
  try {
    pool_setup();
    Arena A(s);
    std::vector<const float*> lg((size_t)count, nullptr);
    int* err = A.get<int>(1);
    GP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (!sel.empty()) {
      std::vector<int64_t> base;
      const float* L = mp_union_logits(M, graphs, sel, base, A, s, err);
      for (size_t k = 0; k < sel.size(); k++) lg[(size_t)sel[k]] = L + base[k];
    }
    int herr = 0;
    GP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (herr) return GP_ERR_TIMEOUT;
    return batch_run(count, graphs, r_cpu, tol, nullptr, parts, res, makespans, s, current_schedule(dev), nullptr,
                     lg.data());
  } catch (Fail& f) {
    cudaGetLastError();
    return f.st;
  }
}

// k_mpnn.cuh -- the learned proposal's message-passing network: features, aggregation, the three
// layer products on the tensor cores (k_umma.cuh), logits, loss, backward pass and Adam.
//
// Network (a project addition; the paper's initial split comes from METIS, Sec. III.A):
//   x_v  = [log1p(cpu)/16, log1p(gpu)/16, log1p(indeg)/4, log1p(outdeg)/4, level/max(1, levels-1)]
//   h0   = relu(x W_in + b_in)
//   c_v  = [h_v | sum_{u->v} e h_u / max(1, indeg v) | sum_{v->u} e h_u / max(1, outdeg v)],
//          e = log1p(transfer cost)/16 per directed entry
//   h_l  = relu(c W_l + b_l), l = 1..3 (W_l 192 x 64, BF16 on the tensor cores, FP32 accumulate)
//   logit = h3 . w_o + b_o;   loss = mean softplus(logit) - y logit
// Neighbour sums run in FP32 in row order; the in-CSR's rows are sorted by (source, cost) before the
// network first reads a graph (k_sort_rows_*) and the out-CSR's order is the caller's, so the
// network's outputs are deterministic.  The backward pass works on the summed loss and divides the
// parameter gradients by n at the end.
#pragma once
#include <cuda_bf16.h>

#include "gp_internal.cuh"
#include "k_umma.cuh"

namespace gp {

constexpr int kHid = 64, kNFeat = 5, kCat = 3 * kHid;
// flat parameter vector: W_in, b_in, W1, b1, W2, b2, W3, b3, w_o, b_o (row-major)
constexpr int64_t kPWin = 0, kPBin = kPWin + kNFeat * kHid;
constexpr int64_t kPW1 = kPBin + kHid;
constexpr int64_t kLayerStride = (int64_t)kCat * kHid + kHid;
__host__ __device__ constexpr int64_t p_W(int l) { return kPW1 + (l - 1) * kLayerStride; }
__host__ __device__ constexpr int64_t p_b(int l) { return p_W(l) + (int64_t)kCat * kHid; }
constexpr int64_t kPWo = p_W(4), kPBo = kPWo + kHid, kPN = kPBo + 1;
static_assert(kPN == 37505, "parameter count");
constexpr int64_t kTileC = 128LL * kCat;  // BF16 elements per 128-row tile of c
constexpr int64_t kTileZ = 128LL * kHid;  // per 128-row tile of dz

struct MpGraph {
  int64_t n, m;
  const int64_t* off;
  const int32_t* cols;
  const int32_t* w;
  const int64_t* in_off;
  const int32_t* in_src;
  const int32_t* in_w;
  const int32_t* cC;
  const int32_t* cG;
  const int32_t* level;
  int32_t nlev;
  const float* levf;  // nullable: the level feature per vertex (a union of graphs with their own depths)
};

// features, inverse degrees, per-entry edge features (out-CSR order and in-CSR order)
__global__ void k_mp_prep(MpGraph G, float* __restrict__ X, float* __restrict__ inv_in, float* __restrict__ inv_out,
                          float* __restrict__ e_out, float* __restrict__ e_in) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  const float lev_den = 1.0f / (float)(G.nlev > 1 ? G.nlev - 1 : 1);
  for (int64_t v = tid; v < G.n; v += st) {
    const int64_t id = G.in_off[v + 1] - G.in_off[v], od = G.off[v + 1] - G.off[v];
    float* x = X + v * kNFeat;
    x[0] = log1pf((float)G.cC[v]) * 0.0625f;
    x[1] = log1pf((float)G.cG[v]) * 0.0625f;
    x[2] = log1pf((float)id) * 0.25f;
    x[3] = log1pf((float)od) * 0.25f;
    x[4] = G.levf ? G.levf[v] : (float)G.level[v] * lev_den;
    inv_in[v] = 1.0f / (float)(id > 1 ? id : 1);
    inv_out[v] = 1.0f / (float)(od > 1 ? od : 1);
  }
  for (int64_t e = tid; e < G.m; e += st) {
    e_out[e] = log1pf((float)G.w[e]) * 0.0625f;
    e_in[e] = log1pf((float)G.in_w[e]) * 0.0625f;
  }
}

// h0 = relu(x W_in + b_in), BF16 [n x 64]
__global__ void k_mp_input(int64_t n, const float* __restrict__ X, const float* __restrict__ P,
                           __nv_bfloat16* __restrict__ H) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * kHid; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / kHid;
    const int j = (int)(i % kHid);
    float z = P[kPBin + j];
#pragma unroll
    for (int f = 0; f < kNFeat; f++) z = fmaf(X[v * kNFeat + f], P[kPWin + f * kHid + j], z);
    H[i] = __float2bfloat16(z > 0.0f ? z : 0.0f);
  }
}

// Sum over the entries [b, e) of a row of wt(entry) * rows[idx(entry)] (two features per lane, lane
// owns features 2*lane, 2*lane+1 of a 64-wide row), in row order.
template <class RowF>
__device__ __forceinline__ void warp_row_sum(int64_t b, int64_t e, const int32_t* __restrict__ idx,
                                             const float* __restrict__ ew, RowF row, float& a0, float& a1) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = b; base < e; base += 32) {
    const int cnt = (int)((e - base) < 32 ? (e - base) : 32);
    int32_t my_u = 0;
    float my_w = 0.0f;
    if (lane < cnt) {
      my_u = idx[base + lane];
      my_w = ew[base + lane];
    }
    int j = 0;
    for (; j + 4 <= cnt; j += 4) {  // four independent row loads in flight
      float2 h[4];
#pragma unroll
      for (int q = 0; q < 4; q++)
        h[q] = row(__shfl_sync(0xffffffffu, my_u, j + q), __shfl_sync(0xffffffffu, my_w, j + q));
#pragma unroll
      for (int q = 0; q < 4; q++) {
        a0 += h[q].x;
        a1 += h[q].y;
      }
    }
    for (; j < cnt; j++) {
      const float2 h = row(__shfl_sync(0xffffffffu, my_u, j), __shfl_sync(0xffffffffu, my_w, j));
      a0 += h.x;
      a1 += h.y;
    }
  }
}

__device__ __forceinline__ void store_tile2(__nv_bfloat16* __restrict__ T, int64_t v, int k, int R, int K,
                                            float x, float y) {
  const int64_t tile = v / R, r = v % R;
  __nv_bfloat162 p;
  p.x = __float2bfloat16(x);
  p.y = __float2bfloat16(y);
  *(__nv_bfloat162*)(T + tile * (int64_t)R * K + umma_off(r, k, R) / 2) = p;
}

// c_v = [h_v | ain_v | aout_v] written into the tiled A image of the layer product (warp per vertex)
__global__ void __launch_bounds__(256) k_mp_aggregate(MpGraph G, const float* __restrict__ inv_in,
                                                      const float* __restrict__ inv_out,
                                                      const float* __restrict__ e_out, const float* __restrict__ e_in,
                                                      const __nv_bfloat16* __restrict__ H,
                                                      __nv_bfloat16* __restrict__ Ct) {
  __shared__ unsigned long long sacc[32];
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const __nv_bfloat162* H2 = (const __nv_bfloat162*)H;
  unsigned long long bytes = 0;
  auto row = [&](int32_t u, float wgt) {
    const float2 h = __bfloat1622float2(H2[(int64_t)u * 32 + lane]);
    return make_float2(wgt * h.x, wgt * h.y);
  };
  for (int64_t v = gw; v < G.n; v += nw) {
    const float2 self = __bfloat1622float2(H2[v * 32 + lane]);
    float i0 = 0.0f, i1 = 0.0f, o0 = 0.0f, o1 = 0.0f;
    warp_row_sum(G.in_off[v], G.in_off[v + 1], G.in_src, e_in, row, i0, i1);
    warp_row_sum(G.off[v], G.off[v + 1], G.cols, e_out, row, o0, o1);
    const float si = inv_in[v], so = inv_out[v];
    const int k = 2 * lane;
    // per vertex: ranges (32), own row (128), inverse degrees (8), c (384); per entry: id, weight, row
    if (lane == 0)
      bytes += 552ull + 136ull * (unsigned long long)(G.in_off[v + 1] - G.in_off[v] + G.off[v + 1] - G.off[v]);
    store_tile2(Ct, v, k, 128, kCat, self.x, self.y);
    store_tile2(Ct, v, kHid + k, 128, kCat, i0 * si, i1 * si);
    store_tile2(Ct, v, 2 * kHid + k, 128, kCat, o0 * so, o1 * so);
  }
  account(F_MPNN, bytes, sacc);
}

// forward epilogue: h = relu(acc + b), BF16 row-major
struct EpiRelu {
  static constexpr unsigned kOutBytes = 2;  // BF16 per output
  const float* bias;
  __nv_bfloat16* H;
  __device__ __forceinline__ void operator()(int64_t row, int col0, const float* v) const {
    __align__(16) __nv_bfloat162 o[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const float a = v[2 * i] + bias[col0 + 2 * i], b = v[2 * i + 1] + bias[col0 + 2 * i + 1];
      o[i].x = __float2bfloat16(a > 0.0f ? a : 0.0f);
      o[i].y = __float2bfloat16(b > 0.0f ? b : 0.0f);
    }
    uint4* dst = (uint4*)(H + row * kHid + col0);
    dst[0] = *(const uint4*)&o[0];
    dst[1] = *(const uint4*)&o[4];
  }
};

// logits; with labels also dlogit = sigmoid(logit) - y (summed loss) and per-block loss partials
__global__ void __launch_bounds__(256) k_mp_logits(int64_t n, const __nv_bfloat16* __restrict__ H,
                                                   const float* __restrict__ P, float* __restrict__ logit,
                                                   const uint8_t* __restrict__ label, float* __restrict__ dlogit,
                                                   double* __restrict__ loss_part) {
  __shared__ double sh[32];
  double loss = 0.0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const uint4* hp = (const uint4*)(H + v * kHid);
    float z = P[kPBo];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const uint4 u = hp[q];
      const __nv_bfloat162* b2 = (const __nv_bfloat162*)&u;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const float2 f = __bfloat1622float2(b2[i]);
        z = fmaf(f.x, P[kPWo + q * 8 + 2 * i], z);
        z = fmaf(f.y, P[kPWo + q * 8 + 2 * i + 1], z);
      }
    }
    logit[v] = z;
    if (label) {
      const float y = label[v] == 0 ? 1.0f : 0.0f;
      const float s = 1.0f / (1.0f + expf(-z));
      dlogit[v] = s - y;
      const double zd = (double)z;
      loss += (zd > 0 ? zd + log1p(exp(-zd)) : log1p(exp(zd))) - (double)y * zd;
    }
  }
  if (loss_part) {
    loss = block_sum<double>(loss, sh);
    if (threadIdx.x == 0) loss_part[blockIdx.x] = loss;
  }
}

// dz3 = dlogit w_o * [h3 > 0]: FP32 row-major and the tiled BF16 A image of the dc product
__global__ void k_mp_dz_top(int64_t n, const float* __restrict__ dlogit, const float* __restrict__ P,
                            const __nv_bfloat16* __restrict__ H, float* __restrict__ dZ,
                            __nv_bfloat16* __restrict__ dZt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * (kHid / 2);
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / (kHid / 2);
    const int k = (int)(i % (kHid / 2)) * 2;
    const float2 h = __bfloat1622float2(((const __nv_bfloat162*)H)[i]);
    const float d = dlogit[v];
    const float a = h.x > 0.0f ? d * P[kPWo + k] : 0.0f;
    const float b = h.y > 0.0f ? d * P[kPWo + k + 1] : 0.0f;
    dZ[v * kHid + k] = a;
    dZ[v * kHid + k + 1] = b;
    store_tile2(dZt, v, k, 128, kHid, a, b);
  }
}

// dh_prev = dc[:, 0:64] + sum_{v->u} e / max(1, indeg u) dc_u[64:128] + sum_{u->v} e / max(1, outdeg u)
// dc_u[128:192]; dz_prev = dh_prev * [h_prev > 0] (warp per vertex)
__global__ void __launch_bounds__(256) k_mp_agg_back(MpGraph G, const float* __restrict__ inv_in,
                                                     const float* __restrict__ inv_out,
                                                     const float* __restrict__ e_out, const float* __restrict__ e_in,
                                                     const float* __restrict__ dC, const __nv_bfloat16* __restrict__ Hp,
                                                     float* __restrict__ dZ, __nv_bfloat16* __restrict__ dZt) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int k = 2 * lane;
  auto row_in = [&](int32_t u, float wgt) {  // v -> u: v fed ain_u
    const float2 d = *(const float2*)(dC + (int64_t)u * kCat + kHid + k);
    const float s = wgt * inv_in[u];
    return make_float2(s * d.x, s * d.y);
  };
  auto row_out = [&](int32_t u, float wgt) {  // u -> v: v fed aout_u
    const float2 d = *(const float2*)(dC + (int64_t)u * kCat + 2 * kHid + k);
    const float s = wgt * inv_out[u];
    return make_float2(s * d.x, s * d.y);
  };
  for (int64_t v = gw; v < G.n; v += nw) {
    float a0 = 0.0f, a1 = 0.0f;
    warp_row_sum(G.off[v], G.off[v + 1], G.cols, e_out, row_in, a0, a1);
    warp_row_sum(G.in_off[v], G.in_off[v + 1], G.in_src, e_in, row_out, a0, a1);
    const float2 self = *(const float2*)(dC + v * kCat + k);
    const float2 h = __bfloat1622float2(((const __nv_bfloat162*)Hp)[v * 32 + lane]);
    const float d0 = h.x > 0.0f ? self.x + a0 : 0.0f;
    const float d1 = h.y > 0.0f ? self.y + a1 : 0.0f;
    dZ[v * kHid + k] = d0;
    dZ[v * kHid + k + 1] = d1;
    if (dZt) store_tile2(dZt, v, k, 128, kHid, d0, d1);
  }
}

// Parameter gradient of one layer, partials per block: part[b][k][j] = sum over the block's
// vertices of c_v[k] dz_v[j] (k < K) and, in row K, sum of dz_v[j] (the bias).  c comes from the
// tiled BF16 image (K = 192) or from the FP32 features (K = 5).  Vertices are split into equal
// contiguous ranges per block; the sums inside a block run in vertex order.
constexpr int kDwStage = 32;
template <int K>
__global__ void __launch_bounds__(256) k_mp_dw(int64_t n, const __nv_bfloat16* __restrict__ Ct,
                                               const float* __restrict__ X, const float* __restrict__ dZ,
                                               float* __restrict__ part) {
  constexpr int ROWS = K + 1, OUT = ROWS * kHid;
  constexpr int PER = (OUT + 255) / 256;
  __shared__ float cs[kDwStage][ROWS];
  __shared__ float zs[kDwStage][kHid];
  float acc[PER];
#pragma unroll
  for (int i = 0; i < PER; i++) acc[i] = 0.0f;
  const int64_t per_blk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t v0 = (int64_t)blockIdx.x * per_blk, v1 = (v0 + per_blk < n) ? v0 + per_blk : n;
  for (int64_t sb = v0; sb < v1; sb += kDwStage) {
    const int cnt = (int)((v1 - sb) < kDwStage ? (v1 - sb) : kDwStage);
    for (int i = threadIdx.x; i < kDwStage * ROWS; i += blockDim.x) {
      const int s = i / ROWS, k = i % ROWS;
      float x = 0.0f;
      if (s < cnt) {
        const int64_t v = sb + s;
        if (k == K)
          x = 1.0f;
        else if (K == kCat)
          x = __bfloat162float(Ct[(v / 128) * kTileC + umma_off(v % 128, k, 128) / 2]);
        else
          x = X[v * kNFeat + k];
      }
      cs[s][k] = x;
    }
    for (int i = threadIdx.x; i < kDwStage * kHid; i += blockDim.x) {
      const int s = i / kHid, j = i % kHid;
      zs[s][j] = s < cnt ? dZ[(sb + s) * kHid + j] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; i++) {
      const int o = threadIdx.x + 256 * i;
      if (o < OUT) {
        const int k = o / kHid, j = o % kHid;
        float a = acc[i];
        for (int s = 0; s < cnt; s++) a = fmaf(cs[s][k], zs[s][j], a);
        acc[i] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < PER; i++) {
    const int o = threadIdx.x + 256 * i;
    if (o < OUT) part[(int64_t)blockIdx.x * OUT + o] = acc[i];
  }
}

// grad[w_off + k*64 + j] = scale * sum_b part[b][k][j] (k < K), grad[b_off + j] = scale * sum_b part[b][K][j]
__global__ void k_mp_dw_reduce(int nblk, int K, const float* __restrict__ part, float scale, float* __restrict__ grad,
                               int64_t w_off, int64_t b_off) {
  const int OUT = (K + 1) * kHid;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < OUT; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += (double)part[(int64_t)b * OUT + o];
    const int k = o / kHid, j = o % kHid;
    grad[k < K ? w_off + o : b_off + j] = (float)(s * scale);
  }
}

// output-layer gradient: dw_o[j] = scale * sum_v dlogit_v h3_v[j], db_o = scale * sum_v dlogit_v
__global__ void k_mp_dout(int64_t n, const float* __restrict__ dlogit, const __nv_bfloat16* __restrict__ H,
                          float scale, float* __restrict__ grad) {
  __shared__ double sh[32];
  const int j = blockIdx.x;  // 0..64 (64 = the bias)
  double s = 0.0;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x)
    s += (double)dlogit[v] * (j < kHid ? (double)__bfloat162float(H[v * kHid + j]) : 1.0);
  s = block_sum<double>(s, sh);
  if (threadIdx.x == 0) grad[j < kHid ? kPWo + j : kPBo] = (float)(s * scale);
}

__global__ void k_sum_parts(int nparts, const double* __restrict__ parts, double* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nparts; i++) s += parts[i];
    *out = s;
  }
}

// Adam (bias-corrected), FP32 master parameters
__global__ void k_adam(int64_t np, float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 tiled copies of W_l: forward operand (64 rows j, K = 192 k: W^T) and backward operand
// (192 rows k, K = 64 j: W)
__global__ void k_mp_tile_weights(const float* __restrict__ P, __nv_bfloat16* __restrict__ Wf,
                                  __nv_bfloat16* __restrict__ Wb) {
  const int per = kCat * kHid;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * per; i += gridDim.x * blockDim.x) {
    const int l = i / per, r = i % per;
    const int k = r / kHid, j = r % kHid;
    const __nv_bfloat16 x = __float2bfloat16(P[p_W(l + 1) + r]);
    Wf[(int64_t)l * per + umma_off(j, k, kHid) / 2] = x;
    Wb[(int64_t)l * per + umma_off(k, j, kCat) / 2] = x;
  }
}

}  // namespace gp

namespace gp {

// One graph's arrays inside a disjoint union: vertex base vb, entry base eb.
struct MpPiece {
  int64_t n, m, vb, eb;
  const int64_t* off;
  const int32_t* cols;
  const int32_t* w;
  const int64_t* in_off;
  const int32_t* in_src;
  const int32_t* in_w;
  const int32_t* cC;
  const int32_t* cG;
  const int32_t* level;
  int32_t nlev;
};

// Copies every piece into the union arrays, shifting vertex ids and row offsets (block per piece,
// grid-strided over pieces).
__global__ void k_mp_union(const MpPiece* __restrict__ P, int npieces, int64_t* __restrict__ off,
                           int32_t* __restrict__ cols, int32_t* __restrict__ w, int64_t* __restrict__ in_off,
                           int32_t* __restrict__ in_src, int32_t* __restrict__ in_w, int32_t* __restrict__ cC,
                           int32_t* __restrict__ cG, int32_t* __restrict__ level, float* __restrict__ levf) {
  for (int p = blockIdx.x; p < npieces; p += gridDim.x) {
    const MpPiece Q = P[p];
    const float den = 1.0f / (float)(Q.nlev > 1 ? Q.nlev - 1 : 1);
    for (int64_t v = threadIdx.x; v < Q.n; v += blockDim.x) {
      const int64_t o = Q.vb + v;
      off[o] = Q.off[v] + Q.eb;
      in_off[o] = Q.in_off[v] + Q.eb;
      cC[o] = Q.cC[v];
      cG[o] = Q.cG[v];
      level[o] = Q.level[v];
      levf[o] = (float)Q.level[v] * den;
    }
    for (int64_t e = threadIdx.x; e < Q.m; e += blockDim.x) {
      const int64_t o = Q.eb + e;
      cols[o] = Q.cols[e] + (int32_t)Q.vb;
      w[o] = Q.w[e];
      in_src[o] = Q.in_src[e] + (int32_t)Q.vb;
      in_w[o] = Q.in_w[e];
    }
  }
}

__global__ void k_mp_union_tail(int64_t N, int64_t M, int64_t* off, int64_t* in_off) {
  off[N] = M;
  in_off[N] = M;
}

}  // namespace gp

namespace gp {

// ------------------------------------------------------------------------------------------------
// Deterministic row order for the network's neighbour sums: every row of a CSR (entries
// (id, weight), int32 both) sorted by (id, weight).  Rows of <= 32 entries: a warp's shuffle
// bitonic network; longer rows: a block's stable LSD radix sort (8-bit digits) through scratch.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long row_key(int32_t id, int32_t w) {
  return ((unsigned long long)(uint32_t)id << 32) | (unsigned long long)(uint32_t)w;
}

__global__ void __launch_bounds__(256) k_sort_rows_short(int64_t n, const int64_t* __restrict__ off,
                                                         int32_t* __restrict__ ids, int32_t* __restrict__ w,
                                                         int32_t* __restrict__ long_rows, unsigned* long_cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = gw; r < n; r += nw) {
    const int64_t b = off[r], len = off[r + 1] - b;
    if (len <= 1) continue;
    if (len > 32) {
      if (lane == 0) long_rows[atomicAdd(long_cnt, 1u)] = (int32_t)r;
      continue;
    }
    unsigned long long x = lane < len ? row_key(ids[b + lane], w[b + lane]) : ~0ull;
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
      for (int j = kk >> 1; j > 0; j >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, j);
        const bool keep_min = ((lane & j) == 0) == ((lane & kk) == 0);
        x = keep_min ? (x < y ? x : y) : (x > y ? x : y);
      }
    }
    if (lane < len) {
      ids[b + lane] = (int32_t)(x >> 32);
      w[b + lane] = (int32_t)(uint32_t)x;
    }
  }
}

__global__ void __launch_bounds__(1024) k_sort_rows_long(const int64_t* __restrict__ off, int32_t* __restrict__ ids,
                                                         int32_t* __restrict__ w, const int32_t* __restrict__ rows,
                                                         const unsigned* cnt, unsigned long long* __restrict__ ta,
                                                         unsigned long long* __restrict__ tb) {
  __shared__ unsigned hist[256];
  __shared__ unsigned binbase[256];
  __shared__ int wcnt[32][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const unsigned lt = lanemask_lt();
  const unsigned nrows = *cnt;
  for (unsigned ri = blockIdx.x; ri < nrows; ri += gridDim.x) {
    const int32_t r = rows[ri];
    const int64_t b = off[r], N = off[r + 1] - b;
    unsigned long long* src = ta + b;
    unsigned long long* dst = tb + b;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) src[i] = row_key(ids[b + i], w[b + i]);
    __syncthreads();
    for (int shift = 0; shift < 64; shift += 8) {
      for (int x = threadIdx.x; x < 256; x += blockDim.x) hist[x] = 0;
      __syncthreads();
      for (int64_t i = threadIdx.x; i < N; i += blockDim.x) atomicAdd(&hist[(src[i] >> shift) & 255ull], 1u);
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int x = 0; x < 256; x++) {
          binbase[x] = run;
          run += hist[x];
        }
      }
      __syncthreads();
      for (int64_t tile = 0; tile < N; tile += blockDim.x) {  // stable scatter, one tile at a time
        const int64_t i = tile + threadIdx.x;
        const bool valid = i < N;
        for (int x = lane; x < 256; x += 32) wcnt[wid][x] = 0;
        __syncwarp();
        unsigned long long key = 0;
        int dg = 0, rank = 0;
        if (valid) {
          key = src[i];
          dg = (int)((key >> shift) & 255ull);
        }
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
          const unsigned peers = __match_any_sync(act, dg);
          rank = __popc(peers & lt);
          if (rank == 0) wcnt[wid][dg] = __popc(peers);
        }
        __syncthreads();
        unsigned tilecnt = 0;
        if (threadIdx.x < 256) {
          int run = 0;
          for (int q = 0; q < nwarps; q++) {
            const int c = wcnt[q][threadIdx.x];
            wcnt[q][threadIdx.x] = run;
            run += c;
          }
          tilecnt = (unsigned)run;
        }
        __syncthreads();
        if (valid) dst[binbase[dg] + wcnt[wid][dg] + rank] = key;
        __syncthreads();
        if (threadIdx.x < 256) binbase[threadIdx.x] += tilecnt;
        __syncthreads();
      }
      unsigned long long* t = src;
      src = dst;
      dst = t;
    }
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {  // 8 passes: the result is back in ta
      const unsigned long long k = src[i];
      ids[b + i] = (int32_t)(k >> 32);
      w[b + i] = (int32_t)(uint32_t)k;
    }
    __syncthreads();
  }
}

}  // namespace gp

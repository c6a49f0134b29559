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

// FMA-pipe throughput probe (measurement aid for the roofline of the SIMT
// K.v forms): 8 independent multiply-add chains per thread.
#include "common.cuh"

namespace {
template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == (T)1234.5) out[blockIdx.x] = s;   // keeps the chains live
}
}  // namespace

extern "C" mfto_status mfto_fma_probe(mfto_form form, int32_t blocks, int32_t iters,
                                      double* ms_out) {
  if (!ms_out || blocks < 1 || iters < 1) return MFTO_INVALID_ARG;
  if (form != MFTO_FORM_F64 && form != MFTO_FORM_F32) return MFTO_UNSUPPORTED;
  void* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess) return MFTO_OOM;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto launch = [&]() {
    if (form == MFTO_FORM_F64)
      fma_chains<double><<<blocks, 256>>>((double*)out, iters, 0.999999, 1e-7);
    else
      fma_chains<float><<<blocks, 256>>>((float*)out, iters, 0.999999f, 1e-7f);
  };
  launch();  // warm-up
  cudaEventRecord(a);
  launch();
  cudaEventRecord(b);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return MFTO_CUDA_ERROR;
  *ms_out = ms;
  return MFTO_OK;
}

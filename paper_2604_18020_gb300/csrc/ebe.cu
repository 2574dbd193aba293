// Element-by-element K.v over an arbitrary connectivity table: the shape of
// the synthetic hot-path microbenchmark of Sec. 5 ("Hot-Path Microbenchmark",
// Tab. profiling), where the element DOF indices are random instead of the
// structured mesh's, so that no locality can be exploited.
//
//   y = sum_e B_e^T (E_e KE) B_e v      (Eq. matfree, no Dirichlet rows)
//
// Three ways, all through the same 24 x 24 unit element matrix KE:
//   staged FP64 -- the unfused three-stage pipeline the paper times as
//                  t_full64: a gather kernel (V_e = v[edof_e], [n][24]), a
//                  batched element contraction (Y_e = V_e KE, written and
//                  read back through HBM) and a scatter kernel
//                  (y[edof_e] += E_e Y_e with FP64 atomics);
//   fused FP64  -- one kernel: gather, contraction and atomic scatter of an
//                  element in one thread, nothing but v and y in memory;
//   fused FP32  -- the same in FP32 (the paper's t_fused form).
// The scatter adds with atomics because an arbitrary table has no owner per
// DOF: the sums are not bit-reproducible (order of the additions varies).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

struct mfto_ebe {
  int64_t n_elem = 0, n_dof = 0;
  cudaStream_t stream = nullptr;
  double* Ve = nullptr;   // [n_elem][24] gathered element vectors (staged path)
  double* Ye = nullptr;   // [n_elem][24] element products (staged path)
  double* KE64 = nullptr;
  float* KE32 = nullptr;
  int32_t* d_bad = nullptr;   // set when an index falls outside [0, n_dof)
  int32_t* h_bad = nullptr;
  cudaEvent_t ev[4] = {};
  int64_t launches = 0;
  char msg[512] = {};
};

namespace {

constexpr int kEbeBlock = 256;
constexpr int kContractRows = 64;   // elements per CTA of the staged contraction

mfto_status efail(mfto_ebe* e, mfto_status code, const char* fmt, ...) {
  if (e) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(e->msg, sizeof(e->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define ECUDA(e, call)                                                              \
  do {                                                                              \
    cudaError_t err_ = (call);                                                      \
    if (err_ != cudaSuccess)                                                        \
      return efail((e), MFTO_CUDA_ERROR, "%s: %s", #call, cudaGetErrorString(err_)); \
  } while (0)

__device__ __forceinline__ bool in_range(int32_t d, int64_t n_dof, int32_t* bad) {
  if (d >= 0 && d < n_dof) return true;
  *bad = 1;
  return false;
}

// V_e[a] = v[edof_e[a]], one thread per (element, local DOF): the table and
// V are read and written in order, v is gathered.
__global__ void __launch_bounds__(kEbeBlock)
ebe_gather(const int32_t* __restrict__ edof, const double* __restrict__ v,
           double* __restrict__ Ve, int64_t n, int64_t n_dof, int32_t* bad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = edof[t];
    Ve[t] = in_range(d, n_dof, bad) ? v[d] : 0.0;
  }
}

// Y_e = V_e KE (KE symmetric) for kContractRows elements per CTA: the rows
// and KE staged in shared memory, each thread computing six outputs.
__global__ void __launch_bounds__(kEbeBlock)
ebe_contract(const double* __restrict__ Ve, const double* __restrict__ KE,
             double* __restrict__ Ye, int64_t n_elem) {
  __shared__ double ke[576];
  __shared__ double rows[kContractRows * 24];
  for (int i = threadIdx.x; i < 576; i += blockDim.x) ke[i] = KE[i];
  for (int64_t e0 = (int64_t)blockIdx.x * kContractRows; e0 < n_elem;
       e0 += (int64_t)gridDim.x * kContractRows) {
    const int ne = n_elem - e0 < kContractRows ? (int)(n_elem - e0) : kContractRows;
    __syncthreads();
    for (int i = threadIdx.x; i < ne * 24; i += blockDim.x) rows[i] = Ve[e0 * 24 + i];
    __syncthreads();
    for (int o = threadIdx.x; o < ne * 24; o += blockDim.x) {
      const int r = o / 24, a = o - 24 * r;
      double acc = 0.0;
#pragma unroll
      for (int b = 0; b < 24; ++b) acc = fma(rows[r * 24 + b], ke[b * 24 + a], acc);
      Ye[e0 * 24 + o] = acc;
    }
  }
}

// y[edof_e[a]] += E_e Y_e[a]
__global__ void __launch_bounds__(kEbeBlock)
ebe_scatter(const int32_t* __restrict__ edof, const double* __restrict__ E,
            const double* __restrict__ Ye, double* __restrict__ y, int64_t n, int64_t n_dof,
            int32_t* bad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = edof[t];
    if (in_range(d, n_dof, bad)) atomicAdd(&y[d], E[t / 24] * Ye[t]);
  }
}

// One element per thread: 24 indices (six 16-byte loads of the table row),
// 24 gathered values, the 24 x 24 contraction against KE in shared memory
// (every thread reads the same entry at once: a broadcast) and 24 atomics.
template <typename T>
__global__ void __launch_bounds__(kEbeBlock)
ebe_fused(const int32_t* __restrict__ edof, const T* __restrict__ E, const T* __restrict__ KE,
          const T* __restrict__ v, T* __restrict__ y, int64_t n_elem, int64_t n_dof,
          int32_t* bad) {
  __shared__ T ke[576];
  for (int i = threadIdx.x; i < 576; i += blockDim.x) ke[i] = KE[i];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_elem;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t idx[24];
    const int4* row = reinterpret_cast<const int4*>(edof + 24 * e);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int4 w = row[q];
      idx[4 * q] = w.x;
      idx[4 * q + 1] = w.y;
      idx[4 * q + 2] = w.z;
      idx[4 * q + 3] = w.w;
    }
    T ve[24];
#pragma unroll
    for (int b = 0; b < 24; ++b) ve[b] = in_range(idx[b], n_dof, bad) ? v[idx[b]] : T(0);
    const T Ee = E[e];
#pragma unroll
    for (int a = 0; a < 24; ++a) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < 24; ++b) acc = fma(ke[a * 24 + b], ve[b], acc);
      if (idx[a] >= 0 && idx[a] < n_dof) atomicAdd(&y[idx[a]], Ee * acc);
    }
  }
}

int grid_for(int64_t work, int per_thread) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (work + (int64_t)kEbeBlock * per_thread - 1) / ((int64_t)kEbeBlock * per_thread);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, 32LL * sms));
}

}  // namespace

extern "C" mfto_status mfto_ebe_create(int64_t n_elem, int64_t n_dof, const double* h_KE,
                                       void* stream, mfto_ebe** out) {
  if (!out || !h_KE) return MFTO_INVALID_ARG;
  *out = nullptr;
  if (n_elem < 1 || n_dof < 1 || n_dof > INT32_MAX || n_elem > (INT32_MAX / 24))
    return MFTO_INVALID_ARG;
  mfto_ebe* e = new mfto_ebe();
  e->n_elem = n_elem;
  e->n_dof = n_dof;
  e->stream = static_cast<cudaStream_t>(stream);
  float ke32[576];
  for (int i = 0; i < 576; ++i) ke32[i] = (float)h_KE[i];
  const size_t rows = sizeof(double) * 24 * (size_t)n_elem;
  auto fail = [&](cudaError_t err) {
    mfto_ebe_destroy(e);
    return err == cudaErrorMemoryAllocation ? MFTO_OOM : MFTO_CUDA_ERROR;
  };
  cudaError_t err;
  if ((err = cudaMalloc((void**)&e->Ve, rows)) != cudaSuccess) return fail(err);
  if ((err = cudaMalloc((void**)&e->Ye, rows)) != cudaSuccess) return fail(err);
  if ((err = cudaMalloc((void**)&e->KE64, sizeof(double) * 576)) != cudaSuccess) return fail(err);
  if ((err = cudaMalloc((void**)&e->KE32, sizeof(float) * 576)) != cudaSuccess) return fail(err);
  if ((err = cudaMalloc((void**)&e->d_bad, sizeof(int32_t))) != cudaSuccess) return fail(err);
  if ((err = cudaMallocHost((void**)&e->h_bad, sizeof(int32_t))) != cudaSuccess) return fail(err);
  for (cudaEvent_t& ev : e->ev)
    if ((err = cudaEventCreate(&ev)) != cudaSuccess) return fail(err);
  if ((err = cudaMemcpy(e->KE64, h_KE, sizeof(double) * 576, cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return fail(err);
  if ((err = cudaMemcpy(e->KE32, ke32, sizeof(float) * 576, cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return fail(err);
  *out = e;
  return MFTO_OK;
}

extern "C" mfto_status mfto_ebe_destroy(mfto_ebe* e) {
  if (!e) return MFTO_OK;
  void* ptrs[] = {e->Ve, e->Ye, e->KE64, e->KE32, e->d_bad};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (e->h_bad) cudaFreeHost(e->h_bad);
  for (cudaEvent_t ev : e->ev)
    if (ev) cudaEventDestroy(ev);
  delete e;
  return MFTO_OK;
}

extern "C" const char* mfto_ebe_last_error(const mfto_ebe* e) { return e ? e->msg : ""; }

extern "C" mfto_status mfto_ebe_launch_count(const mfto_ebe* e, int64_t* n) {
  if (!e || !n) return MFTO_INVALID_ARG;
  *n = e->launches;
  return MFTO_OK;
}

extern "C" mfto_status mfto_ebe_kv(mfto_ebe* e, int32_t variant, const int32_t* d_edof,
                                   const void* d_E, const void* d_v, void* d_y,
                                   float* h_stage_ms) {
  if (!e) return MFTO_INVALID_ARG;
  if (!d_edof || !d_E || !d_v || !d_y)
    return efail(e, MFTO_INVALID_ARG, "mfto_ebe_kv: null pointer");
  if (reinterpret_cast<uintptr_t>(d_edof) % 16 != 0)
    return efail(e, MFTO_INVALID_ARG, "mfto_ebe_kv: the table must be 16-byte aligned");
  if (variant < MFTO_EBE_STAGED_F64 || variant > MFTO_EBE_FUSED_F32)
    return efail(e, MFTO_INVALID_ARG, "mfto_ebe_kv: unknown variant %d", variant);
  cudaStream_t s = e->stream;
  const int64_t n = 24 * e->n_elem;
  const size_t ybytes = (variant == MFTO_EBE_FUSED_F32 ? sizeof(float) : sizeof(double)) *
                        (size_t)e->n_dof;
  ECUDA(e, cudaMemsetAsync(e->d_bad, 0, sizeof(int32_t), s));
  const bool timed = h_stage_ms != nullptr;
  if (timed) ECUDA(e, cudaEventRecord(e->ev[0], s));
  if (variant == MFTO_EBE_STAGED_F64) {
    ebe_gather<<<grid_for(n, 4), kEbeBlock, 0, s>>>(d_edof, static_cast<const double*>(d_v),
                                                      e->Ve, n, e->n_dof, e->d_bad);
    ECUDA(e, cudaGetLastError());
    if (timed) ECUDA(e, cudaEventRecord(e->ev[1], s));
    const int64_t blocks = (e->n_elem + kContractRows - 1) / kContractRows;
    ebe_contract<<<(int)std::min<int64_t>(blocks, INT32_MAX), kEbeBlock, 0, s>>>(
        e->Ve, e->KE64, e->Ye, e->n_elem);
    ECUDA(e, cudaGetLastError());
    if (timed) ECUDA(e, cudaEventRecord(e->ev[2], s));
    ECUDA(e, cudaMemsetAsync(d_y, 0, ybytes, s));
    ebe_scatter<<<grid_for(n, 4), kEbeBlock, 0, s>>>(d_edof, static_cast<const double*>(d_E),
                                                       e->Ye, static_cast<double*>(d_y), n,
                                                       e->n_dof, e->d_bad);
    ECUDA(e, cudaGetLastError());
    e->launches += 3;
  } else {
    ECUDA(e, cudaMemsetAsync(d_y, 0, ybytes, s));
    if (variant == MFTO_EBE_FUSED_F64)
      ebe_fused<double><<<grid_for(e->n_elem, 1), kEbeBlock, 0, s>>>(
          d_edof, static_cast<const double*>(d_E), e->KE64, static_cast<const double*>(d_v),
          static_cast<double*>(d_y), e->n_elem, e->n_dof, e->d_bad);
    else
      ebe_fused<float><<<grid_for(e->n_elem, 1), kEbeBlock, 0, s>>>(
          d_edof, static_cast<const float*>(d_E), e->KE32, static_cast<const float*>(d_v),
          static_cast<float*>(d_y), e->n_elem, e->n_dof, e->d_bad);
    ECUDA(e, cudaGetLastError());
    e->launches += 1;
  }
  if (timed) ECUDA(e, cudaEventRecord(e->ev[3], s));
  ECUDA(e, cudaMemcpyAsync(e->h_bad, e->d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ECUDA(e, cudaStreamSynchronize(s));
  if (timed) {
    if (variant == MFTO_EBE_STAGED_F64) {
      ECUDA(e, cudaEventElapsedTime(&h_stage_ms[0], e->ev[0], e->ev[1]));
      ECUDA(e, cudaEventElapsedTime(&h_stage_ms[1], e->ev[1], e->ev[2]));
      ECUDA(e, cudaEventElapsedTime(&h_stage_ms[2], e->ev[2], e->ev[3]));
    } else {
      ECUDA(e, cudaEventElapsedTime(&h_stage_ms[0], e->ev[0], e->ev[3]));
    }
  }
  if (*e->h_bad)
    return efail(e, MFTO_INVALID_ARG, "mfto_ebe_kv: an index lies outside [0, n_dof)");
  return MFTO_OK;
}

// Compliance and sensitivities for callers that cannot allocate device
// memory.
//
// mfto_compliance_sens needs a handle, and mfto_create allocates the
// handle's workspace with cudaMalloc.  Some callers cannot do that: programs
// whose device memory is owned entirely by another allocator (a framework's
// caching pool, or a budget reserved in full at start-up), and latency-bound
// loops that cannot accept the device-wide synchronisation cudaMalloc may
// cause.  This entry point computes the same quantities with no handle and no
// allocation.
// Its only scratch (the unit element matrix, the per-block partial sums, the
// reduction ticket and the result) is the file-scope array below, which every
// GPU that loads the library holds until the process exits.
#include <math.h>

#include <mutex>

#include "common.cuh"

#define MFTO_NOALLOC_BLOCKS 2048   // partial-sum slots: at most 2048 x 256 elements

struct NoAllocScratch {
  double ke[576];                        // unit KE of the current call
  double partials[MFTO_NOALLOC_BLOCKS];  // one compliance partial per block
  double result;                         // sum_e E_e ce_e
  unsigned int ticket;                   // last-block counter, cleared every call
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

namespace {

// Same arithmetic as the handle's compliance kernel (one thread per element,
// u_e^T KE u_e with KE from the scratch array, fixed-order sums), with one
// block per 256 elements and the partials in the static scratch.
__global__ void __launch_bounds__(MFTO_BLOCK)
compliance_noalloc_kernel(const double* __restrict__ rho, const double* __restrict__ u,
                          double* __restrict__ dc, NoAllocScratch* scr, Grid g, double E0,
                          double Emin, double penal) {
  __shared__ double ke[576];
  __shared__ double sh[64];
  __shared__ bool s_last;
  for (int t = threadIdx.x; t < 576; t += blockDim.x) ke[t] = scr->ke[t];
  __syncthreads();
  const int n = g.nelx * g.nely * g.nelz;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (e < n) {
    const int i = e % g.nelx, j = (e / g.nelx) % g.nely, k = e / (g.nelx * g.nely);
    double ue[24];
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int m = (i + (l & 1)) + g.nx * ((j + ((l >> 1) & 1)) + g.ny * (k + (l >> 2)));
      ue[3 * l + 0] = u[3 * m + 0];
      ue[3 * l + 1] = u[3 * m + 1];
      ue[3 * l + 2] = u[3 * m + 2];
    }
    double ce = 0.0;
#pragma unroll 4
    for (int a = 0; a < 24; ++a) {
      double row = 0.0;
#pragma unroll
      for (int b = 0; b < 24; ++b) row += ke[a * 24 + b] * ue[b];
      ce += ue[a] * row;
    }
    const double r = rho[e];
    acc = (Emin + (E0 - Emin) * pow(r, penal)) * ce;
    if (dc) dc[e] = -penal * pow(r, penal - 1.0) * (E0 - Emin) * ce;
  }
  const double bs = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    scr->partials[blockIdx.x] = bs;
    __threadfence();
    s_last = atomicAdd(&scr->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&scr->partials[b]);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    scr->result = s;
    scr->ticket = 0u;
  }
}

std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_addr[128];   // device address of the array, per device

}  // namespace

extern "C" mfto_status mfto_compliance_sens_noalloc(const mfto_mesh* mesh, double E0, double Emin,
                                                    double nu, double penal,
                                                    const double* d_rho_phys, const double* d_u,
                                                    double* d_dc, double* h_c_out,
                                                    void* stream) {
  if (!mesh || !d_rho_phys || !d_u || !h_c_out) return MFTO_INVALID_ARG;
  if (mesh->nelx < 1 || mesh->nely < 1 || mesh->nelz < 1 || !(mesh->h > 0.0))
    return MFTO_INVALID_ARG;
  if (!(nu > -1.0 && nu < 0.5) || !(E0 > 0.0) || Emin < 0.0 || !(penal >= 1.0))
    return MFTO_INVALID_ARG;
  const int64_t n_elem = (int64_t)mesh->nelx * mesh->nely * mesh->nelz;
  if (n_elem > (int64_t)MFTO_NOALLOC_BLOCKS * MFTO_BLOCK) return MFTO_TOO_LARGE;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return MFTO_CUDA_ERROR;
  NoAllocScratch* scr = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name
    // of the array is not a device address, so look the address up
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return MFTO_CUDA_ERROR;
      }
      g_scratch_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    scr = g_scratch_addr[dev];
  }
  double ke[576];
  mfto_unit_ke(1.0, nu, mesh->h, ke);
  if (cudaMemcpyAsync(scr->ke, ke, sizeof(ke), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int), st) != cudaSuccess)
    return MFTO_CUDA_ERROR;
  const Grid g = make_grid(*mesh);
  const int blocks = (int)((n_elem + MFTO_BLOCK - 1) / MFTO_BLOCK);
  compliance_noalloc_kernel<<<blocks, MFTO_BLOCK, 0, st>>>(d_rho_phys, d_u, d_dc, scr, g, E0, Emin,
                                                          penal);
  if (cudaGetLastError() != cudaSuccess) return MFTO_CUDA_ERROR;
  double c = 0.0;
  if (cudaMemcpyAsync(&c, &scr->result, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MFTO_CUDA_ERROR;
  *h_c_out = c;
  return MFTO_OK;
}

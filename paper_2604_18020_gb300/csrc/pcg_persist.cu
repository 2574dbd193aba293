// Persistent FP32 Jacobi-PCG (Sec. 3.6): the whole inner iteration loop of
// the mixed-precision solve in one cooperative launch.
//
// The per-iteration kernels of pcg.cu cost two launches and two grid-wide
// reductions through a last-block ticket per iteration.  At the 10^5 - 10^6
// element sizes of the benchmark meshes one iteration's work is a few
// microseconds, so those fixed costs dominate.  Here every CTA stays resident
// for the whole solve and each iteration is
//   A  p_new = z + beta p_old folded into the K.v gather, q = K p_new (the
//      column-streaming body of kv_column.cuh over this CTA's column tiles),
//      this CTA's share of p_new.q  ->  partial row 0;
//      grid barrier; every CTA sums the partials in block order, so every CTA
//      holds the same alpha = rz / p.q and takes the same branch;
//   B  u += alpha p_new; r -= alpha q; z = r / d; shares of r.z and r.r
//      ->  partial rows 1, 2;
//      grid barrier; every CTA forms beta = r.z / rz and the stop test.
// The vector update and the r.z, r.r accumulation are those of
// pcg_update_f32; p.q sums each node's three products in FP32 before the
// double-float accumulation (as pcg_kv_col_kernel does).  Values written by
// other CTAs inside the launch are read with ld.global.cg (L2), never
// through L1.  Every barrier wait is bounded: on timeout the kernel raises
// bar_error and returns; the host reports it.
#include <math.h>

#include "cg_update.cuh"
#include "common.cuh"
#include "kv_column.cuh"

namespace {

constexpr int kItersPerLaunch = 4096;   // iterations per launch before the host looks

// Grid barrier on one monotonic counter: each CTA adds 1 with release
// semantics (no return value, no reset) and polls the counter with acquire
// loads until it reaches (barriers passed so far) x G.  The counter is zeroed
// before every launch.  Every wait is bounded: after MFTO_SPIN_LIMIT polls
// the CTA raises *error and stops waiting, and no later barrier waits once
// *error is set.

__device__ __forceinline__ void grid_barrier_count(unsigned int* count, unsigned int target,
                                                   int32_t* error) {
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_add(count, 1u);
    volatile int32_t* verr = error;
    unsigned int spins = 0;
    while (ld_acquire(count) < target) {
      if (*verr) break;
      if (++spins > MFTO_SPIN_LIMIT) { atomicExch(error, 1); break; }
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(MFTO_BLOCK, 2)
pcg_persist_f32(const float* __restrict__ E, const uint8_t* __restrict__ fixed,
                const float* __restrict__ dinv, ModeCoef<float> K, Grid g, ColTiling tl,
                int n_node, float* u, float* r, float* z, float* p0, float* p1, float* q,
                PcgScalars* s, double* part, unsigned int* bar, int max_iters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[64];
  if (*(volatile int32_t*)&s->done) return;   // uniform: written before the launch
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  double rz = s->rz, beta = s->beta, rr = s->rr, pq = s->pq, alpha = s->alpha;
  const double rtol2ff = s->rtol2ff;
  const int maxit = s->maxit;
  int it = s->it;
  int done = 0, status = s->status;
  unsigned int nbar = 0;   // barrier arrivals expected so far
  for (int k = 0; k < max_iters; ++k) {
    float* p_old = (it & 1) ? p1 : p0;
    float* p_new = (it & 1) ? p0 : p1;
    // ---- A: p_new, q = K p_new, share of p_new.q
    {
      const DFloat red = kv_column_body(E, fixed, K, g, tl,
                                        ColLoadDirectionL2{z, p_old, (float)beta},
                                        ColPcg{p_new, q}, reinterpret_cast<float*>(smem_raw));
      const double bs = block_sum_w0(col_warp_finish(red), sh);
      if (tid == 0) part[blockIdx.x] = bs;
    }
    nbar += G;
    grid_barrier_count(bar, nbar, &s->bar_error);
    if (*(volatile int32_t*)&s->bar_error) break;
    {
      double t[1];
      grid_allsum<1>(part, G, t, sh);
      pq = t[0];
    }
    if (!(pq > 0.0) || !isfinite(pq)) {
      done = 1;
      status = MFTO_BREAKDOWN;
      alpha = 0.0;
      break;
    }
    alpha = rz / pq;
    // ---- B: u, r, z; shares of r.z and r.r
    {
      DotAcc<float> d0, d1;
      cg_update_f32<true>(u, p_new, q, r, z, dinv, 3 * n_node, (float)alpha,
                          blockIdx.x * blockDim.x + tid, G * blockDim.x, d0, d1);
      const double b0 = block_sum_w0(d0.finish(), sh);
      const double b1 = block_sum_w0(d1.finish(), sh);
      if (tid == 0) {
        part[MFTO_RED_SLOTS + blockIdx.x] = b0;
        part[2 * MFTO_RED_SLOTS + blockIdx.x] = b1;
      }
    }
    nbar += G;
    grid_barrier_count(bar, nbar, &s->bar_error);
    if (*(volatile int32_t*)&s->bar_error) break;
    double t[2];
    grid_allsum<2>(part + MFTO_RED_SLOTS, G, t, sh);
    it += 1;
    rr = t[1];
    beta = t[0] / rz;
    rz = t[0];
    if (!isfinite(t[0]) || !isfinite(t[1])) {
      done = 1;
      status = MFTO_BREAKDOWN;
    } else if (t[1] <= rtol2ff) {
      done = 1;
      status = MFTO_OK;
    } else if (it >= maxit) {
      done = 1;
      status = MFTO_NOT_CONVERGED;
    }
    if (done) break;
  }
  if (blockIdx.x == 0 && tid == 0) {
    s->rz = rz;
    s->beta = beta;
    s->rr = rr;
    s->pq = pq;
    s->alpha = alpha;
    s->it = it;
    s->status = status;
    s->done = done;
  }
}

int persist_smem() { return (int)ColShape::smem_bytes; }
constexpr size_t kBarBytes = 128;   // the barrier counter, alone in its line

}  // namespace

mfto_status pcg_persist_init(mfto_handle* h) {
  h->persist_grid = 0;
  int dev = 0, coop = 0;
  MFTO_CUDA(h, cudaGetDevice(&dev));
  MFTO_CUDA(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return MFTO_OK;
  const int smem = persist_smem();
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_persist_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem));
  int per_sm = 0;
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_persist_f32,
                                                             MFTO_BLOCK, smem));
  if (per_sm < 1) return MFTO_OK;
  // column tiles sized for the resident CTAs, one tile per CTA where possible
  const Grid g = make_grid(h->mesh);
  const int64_t gmax = (int64_t)per_sm * h->num_sms;
  const ColTiling tl = col_tiling(g, col_chunk(g, gmax, 4));
  int64_t grid = tl.count();
  if (grid > gmax) grid = gmax;
  if (grid > MFTO_RED_SLOTS) grid = MFTO_RED_SLOTS;
  if (grid < 1) grid = 1;
  h->persist_tiling[0] = tl.tx;
  h->persist_tiling[1] = tl.ty;
  h->persist_tiling[2] = tl.tz;
  h->persist_tiling[3] = tl.nzc;
  if (!h->d_bar) {
    MFTO_CUDA(h, cudaMalloc(&h->d_bar, kBarBytes));
    MFTO_CUDA(h, cudaMemsetAsync(h->d_bar, 0, kBarBytes, h->stream));
  }
  h->persist_grid = (int)grid;
  return MFTO_OK;
}

// Runs the FP32 CG started by pcg_start<float> to its end (tolerance, cap or
// breakdown); host_s receives the final scalars.
mfto_status pcg_persist_iterate(mfto_handle* h, const PcgVecs<float>& v, PcgScalars* host_s) {
  if (h->persist_grid < 1)
    return mfto_fail(h, MFTO_UNSUPPORTED, "persistent CG: cooperative launch unavailable");
  const Grid g = make_grid(h->mesh);
  int n_node = (int)h->n_node;
  int max_iters = kItersPerLaunch;
  const float* E = v.E;
  const uint8_t* fixed = h->d_fixed;
  const float* dinv = v.dinv;
  ModeCoef<float> K = h->mc32;
  float *u = v.u, *r = v.r, *z = v.z, *p0 = v.p0, *p1 = v.p1, *q = v.q;
  PcgScalars* s = v.s;
  double* part = v.part_a;
  ColTiling tl;
  tl.fixed_tiles = nullptr;
  tl.tx = h->persist_tiling[0];
  tl.ty = h->persist_tiling[1];
  tl.tz = h->persist_tiling[2];
  tl.nzc = h->persist_tiling[3];
  unsigned int* bar = h->d_bar;
  void* args[] = {(void*)&E, (void*)&fixed, (void*)&dinv, (void*)&K, (void*)&g, (void*)&tl,
                  (void*)&n_node, (void*)&u, (void*)&r, (void*)&z, (void*)&p0, (void*)&p1,
                  (void*)&q, (void*)&s, (void*)&part, (void*)&bar, (void*)&max_iters};
  if (h->kv_timing && !h->ev.cg_start) {
    MFTO_CUDA(h, cudaEventCreate(&h->ev.cg_start));
    MFTO_CUDA(h, cudaEventCreate(&h->ev.cg_stop));
  }
  for (;;) {
    MFTO_CUDA(h, cudaMemcpyAsync(host_s, v.s, sizeof(PcgScalars), cudaMemcpyDeviceToHost,
                                 h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
    if (host_s->bar_error)
      return mfto_fail(h, MFTO_CUDA_ERROR, "persistent CG: a grid barrier wait gave up");
    if (host_s->done) break;
    const int it_before = host_s->it;
    // barrier counters and the error flag start at zero
    MFTO_CUDA(h, cudaMemsetAsync(h->d_bar, 0, kBarBytes, h->stream));
    MFTO_CUDA(h, cudaMemsetAsync(&v.s->bar_error, 0, sizeof(int32_t), h->stream));
    if (h->kv_timing) MFTO_CUDA(h, cudaEventRecord(h->ev.cg_start, h->stream));
    h->launches++;
    MFTO_CUDA(h, cudaLaunchCooperativeKernel((const void*)pcg_persist_f32, dim3(h->persist_grid),
                                             dim3(MFTO_BLOCK), args, (size_t)persist_smem(),
                                             h->stream));
    if (h->kv_timing) {
      MFTO_CUDA(h, cudaEventRecord(h->ev.cg_stop, h->stream));
      MFTO_CUDA(h, cudaMemcpyAsync(host_s, v.s, sizeof(PcgScalars), cudaMemcpyDeviceToHost,
                                   h->stream));
      MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
      float ms = 0.f;
      MFTO_CUDA(h, cudaEventElapsedTime(&ms, h->ev.cg_start, h->ev.cg_stop));
      h->ev.cg_launches++;
      h->ev.cg_ms += ms;
      // K.v applications of the launch: completed iterations, plus the one
      // whose p.q broke down
      h->ev.cg_iterations += host_s->it - it_before +
                             (host_s->status == MFTO_BREAKDOWN && host_s->done ? 1 : 0);
    }
  }
  return MFTO_OK;
}

extern "C" mfto_status mfto_set_cg_engine(mfto_handle* h, int32_t engine) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, engine >= 0 && engine <= 2, "mfto_set_cg_engine: engine must be 0, 1 or 2");
  if (engine == 1 && h->persist_grid < 1)
    return mfto_fail(h, MFTO_UNSUPPORTED, "mfto_set_cg_engine: cooperative launch unavailable");
  if (h->cg_engine != engine) pcg_graph_release(h);   // captured chunks hold the engine's kernels
  h->cg_engine = engine;
  return MFTO_OK;
}

extern "C" mfto_status mfto_cg_timing_read(mfto_handle* h, int64_t* launches,
                                           int64_t* iterations, double* total_ms) {
  if (!h) return MFTO_INVALID_ARG;
  if (launches) *launches = h->ev.cg_launches;
  if (iterations) *iterations = h->ev.cg_iterations;
  if (total_ms) *total_ms = h->ev.cg_ms;
  h->ev.cg_launches = 0;
  h->ev.cg_iterations = 0;
  h->ev.cg_ms = 0.0;
  return MFTO_OK;
}

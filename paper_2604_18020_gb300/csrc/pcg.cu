// Jacobi-preconditioned CG (Sec. 3.6) with warm start, templated on the
// vector type: FP64 for the plain solver, FP32 for the inner solve of the
// iterative refinement (ir.cu).  Dot products are always accumulated in FP64
// (the product of two FP32 values is exact in FP64).
//
// Iteration (left Jacobi, Hestenes-Stiefel):
//   q = K p;  alpha = rz / p.q;  u += alpha p;  r -= alpha q;
//   stop if ||r|| <= rtol ||f|| or it = maxit;
//   z = r / d;  beta = r.z / rz;  p = z + beta p.
// Two kernels per iteration, all scalars stay on the device:
//   A  p_new = z + beta p_old folded into the K.v gather; q = K p_new;
//      p_new.q reduced by the last block, which forms alpha;
//   B  u, r, z updated; r.z and r.r reduced by the last block, which forms
//      beta, counts the iteration and raises `done`.
// Once `done` is set every later kernel returns at entry, so a chunk of
// iterations may be launched past convergence without changing the result.
// The host launches chunks of check_every iterations (captured once into a
// CUDA graph) and reads the scalars after each chunk.
#include <math.h>

#include <vector>

#include "cg_update.cuh"

#include "common.cuh"
#include "kv_node.cuh"

struct PcgGraph {
  const void* key[3] = {nullptr, nullptr, nullptr};
  int chunk = 0;
  bool timed = false;
  int variant = 0;
  int form = 0;
  int engine = 0;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;  // 2 per K.v launch when timed
};

namespace {

// r = f - Ku, z = r / d; r.z, r.r, f.f reduced; the solver state is reset.
// f may alias r (each entry is read before it is written); Ku may be NULL.
// rz_prev > 0 continues an earlier direction (the caller left it in p0):
// the first K.v then uses p = z + (r.z / rz_prev) p0 instead of p = z.
template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_init(const T* f, const T* __restrict__ Ku, const T* __restrict__ dinv, T* r,
         T* __restrict__ z, int n, double rtol, int maxit, double rz_prev, PcgScalars* s,
         double* partials) {
  __shared__ double sh[64];
  DotAcc<T> d0, d1, d2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const T fi = f[i];
    const T ri = fi - (Ku ? Ku[i] : T(0));
    const T zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    d0.add_prod(ri, zi);
    d1.add_prod(ri, ri);
    d2.add_prod(fi, fi);
  }
  const double acc[3] = {d0.finish(), d1.finish(), d2.finish()};
  double tot[3];
  if (last_block_reduce<3, DotAcc<T>::kWarpReduced>(acc, partials, &s->ticket_a, tot, sh) &&
      threadIdx.x == 0) {
    s->rz = tot[0];
    s->rr = tot[1];
    s->ff = tot[2];
    s->rtol2ff = rtol * rtol * tot[2];
    s->beta = rz_prev > 0.0 ? tot[0] / rz_prev : 0.0;
    s->alpha = 0.0;
    s->it = 0;
    s->maxit = maxit;
    s->status = MFTO_OK;
    s->tc_error = 0;
    s->done = (tot[2] == 0.0 || tot[1] <= s->rtol2ff) ? 1 : 0;
    if (!isfinite(tot[0]) || !isfinite(tot[1])) { s->done = 1; s->status = MFTO_BREAKDOWN; }
  }
}

// A (dense node-centric variant): p_new = z + beta p_old, q = K p_new, alpha
// (p_new.q accumulated in FP64 per DOF: this variant exists for comparison)
template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_kv_step(const T* __restrict__ E, const T* __restrict__ z, const T* __restrict__ p_old,
            T* __restrict__ p_new, T* __restrict__ q, const uint8_t* __restrict__ fixed,
            const T* __restrict__ ke_g, Grid g, int n_node, PcgScalars* s, double* partials) {
  if (*(volatile int32_t*)&s->done) return;  // uniform over the grid
  __shared__ T ke[576];
  __shared__ double sh[64];
  for (int t = threadIdx.x; t < 576; t += blockDim.x) ke[t] = ke_g[t];
  __syncthreads();
  const LoadDirection<T> ld{z, p_old, (T)s->beta};
  double acc[1] = {0.0};
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < n_node;
       node += gridDim.x * blockDim.x) {
    T a[3];
    node_kv<T>(node, E, fixed, ke, g, ld, a[0], a[1], a[2]);
    const uint8_t fm = fixed[node];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T pn = ((fm >> c) & 1) ? T(0) : ld(3 * node + c);
      const T qc = ((fm >> c) & 1) ? pn : a[c];
      p_new[3 * node + c] = pn;
      q[3 * node + c] = qc;
      acc[0] += (double)pn * (double)qc;
    }
  }
  double tot[1];
  if (last_block_reduce<1>(acc, partials, &s->ticket_b, tot, sh) && threadIdx.x == 0) {
    s->pq = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      s->done = 1;
      s->status = MFTO_BREAKDOWN;
      s->alpha = 0.0;
    } else {
      s->alpha = s->rz / tot[0];
    }
  }
}

// B: u += alpha p; r -= alpha q; z = r / d; beta = r.z / rz; convergence test
template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_update(T* __restrict__ u, const T* __restrict__ p, const T* __restrict__ q,
           T* __restrict__ r, T* __restrict__ z, const T* __restrict__ dinv, int n,
           PcgScalars* s, double* partials) {
  if (*(volatile int32_t*)&s->done) return;
  __shared__ double sh[64];
  const T alpha = (T)s->alpha;
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    u[i] += alpha * p[i];
    const T ri = r[i] - alpha * q[i];
    const T zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    acc[0] += (double)ri * (double)zi;
    acc[1] += (double)ri * (double)ri;
  }
  double tot[2];
  if (last_block_reduce<2>(acc, partials, &s->ticket_c, tot, sh) && threadIdx.x == 0) {
    s->it += 1;
    s->rr = tot[1];
    s->beta = tot[0] / s->rz;
    s->rz = tot[0];
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      s->done = 1;
      s->status = MFTO_BREAKDOWN;
    } else if (tot[1] <= s->rtol2ff) {
      s->done = 1;
      s->status = MFTO_OK;
    } else if (s->it >= s->maxit) {
      s->done = 1;
      s->status = MFTO_NOT_CONVERGED;
    }
  }
}

// B for FP32 vectors: groups of 4 DOFs per thread in a grid-stride loop over
// few, fat blocks (cg_update.cuh), so the per-thread cost of the reductions
// is spread over many DOFs; warps finish in double-float, blocks in FP64.
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_update_f32(float* __restrict__ u, const float* __restrict__ p, const float* __restrict__ q,
               float* __restrict__ r, float* __restrict__ z, const float* __restrict__ dinv,
               int n, PcgScalars* s, double* partials) {
  int done = 0;
  const float alpha = flag_and_scalar_f32(&s->done, &s->alpha, &done);
  if (done) return;
  __shared__ double sh[64];
  DotAcc<float> d0, d1;
  cg_update_f32<false>(u, p, q, r, z, dinv, n, alpha, blockIdx.x * blockDim.x + threadIdx.x,
                       gridDim.x * blockDim.x, d0, d1);
  const DFloat acc[2] = {d0.finish_df(), d1.finish_df()};
  double tot[2];
  if (last_block_reduce_df<2>(acc, partials, &s->ticket_c, tot, sh) && threadIdx.x == 0) {
    s->it += 1;
    s->rr = tot[1];
    s->beta = tot[0] / s->rz;
    s->rz = tot[0];
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      s->done = 1;
      s->status = MFTO_BREAKDOWN;
    } else if (tot[1] <= s->rtol2ff) {
      s->done = 1;
      s->status = MFTO_OK;
    } else if (s->it >= s->maxit) {
      s->done = 1;
      s->status = MFTO_NOT_CONVERGED;
    }
  }
}

template <typename T>
void launch_update(const mfto_handle* h, cudaStream_t st, const PcgVecs<T>& v, T* p_new);
template <>
void launch_update<double>(const mfto_handle* h, cudaStream_t st, const PcgVecs<double>& v,
                           double* p_new) {
  pcg_update<double><<<reduction_blocks(h->n_dof, MFTO_BLOCK), MFTO_BLOCK, 0, st>>>(
      v.u, p_new, v.q, v.r, v.z, v.dinv, (int)h->n_dof, v.s, v.part_b);
}
template <>
void launch_update<float>(const mfto_handle* h, cudaStream_t st, const PcgVecs<float>& v,
                          float* p_new) {
  // two resident blocks per SM, at most one float4 group per thread per pass
  int64_t blocks = (h->n_dof / 4 + MFTO_BLOCK - 1) / MFTO_BLOCK;
  if (blocks > 2 * (int64_t)h->num_sms) blocks = 2 * (int64_t)h->num_sms;
  if (blocks < 1) blocks = 1;
  pcg_update_f32<<<(int)blocks, MFTO_BLOCK, 0, st>>>(v.u, p_new, v.q, v.r, v.z, v.dinv,
                                                     (int)h->n_dof, v.s, v.part_b);
}

template <typename T>
const T* ke_of(const mfto_handle* h);
template <>
const double* ke_of<double>(const mfto_handle* h) { return h->d_ke64; }
template <>
const float* ke_of<float>(const mfto_handle* h) { return h->d_ke32; }

template <typename T>
mfto_status enqueue_chunk(mfto_handle* h, cudaStream_t st, const PcgVecs<T>& v, int chunk,
                          cudaEvent_t* ev) {
  const Grid g = make_grid(h->mesh);
  const int nb_node = reduction_blocks(h->n_node, MFTO_BLOCK);
  for (int it = 0; it < chunk; ++it) {
    T* p_old = (it & 1) ? v.p1 : v.p0;
    T* p_new = (it & 1) ? v.p0 : v.p1;
    if (sizeof(T) == 4 && cg2_active(h, v.form)) {
      mfto_status s = cg2_enqueue(h, st, reinterpret_cast<const PcgVecs<float>&>(v),
                                  (const float*)p_old, (float*)p_new, it & 1,
                                  ev ? ev[2 * it] : nullptr, ev ? ev[2 * it + 1] : nullptr);
      if (s != MFTO_OK) return s;
      continue;
    }
    // external record nodes: a plain record inside a capture would only add a
    // dependency edge, not record the event on each graph launch
    if (ev) MFTO_CUDA(h, cudaEventRecordWithFlags(ev[2 * it], st, cudaEventRecordExternal));
    if (sizeof(T) == 4 && tc_form(v.form)) {
      mfto_status s = pcg_kv_tc_launch(h, v.form, (const float*)v.E, (const float*)v.z,
                                       (const float*)p_old, (float*)p_new, (float*)v.q, v.s,
                                       v.part_a, st);
      if (s != MFTO_OK) return s;
    } else if (h->kv_variant != 1) {
      mfto_status s = pcg_kv_tile_launch<T>(h, v.E, v.z, p_old, p_new, v.q, v.s, v.part_a, st);
      if (s != MFTO_OK) return s;
    } else {
      pcg_kv_step<T><<<nb_node, MFTO_BLOCK, 0, st>>>(v.E, v.z, p_old, p_new, v.q, h->d_fixed,
                                                     ke_of<T>(h), g, (int)h->n_node, v.s,
                                                     v.part_a);
    }
    if (ev) MFTO_CUDA(h, cudaEventRecordWithFlags(ev[2 * it + 1], st, cudaEventRecordExternal));
    launch_update<T>(h, st, v, p_new);
  }
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

void destroy_graph(PcgGraph* pg) {
  if (!pg) return;
  if (pg->exec) cudaGraphExecDestroy(pg->exec);
  for (cudaEvent_t e : pg->ev) cudaEventDestroy(e);
  delete pg;
}

template <typename T>
mfto_status get_graph(mfto_handle* h, const PcgVecs<T>& v, int slot, PcgGraph** out) {
  const int chunk = h->p.check_every;
  PcgGraph* pg = h->pcg_graph[slot];
  if (pg && pg->key[0] == v.E && pg->key[1] == v.u && pg->key[2] == v.s && pg->chunk == chunk &&
      pg->timed == h->kv_timing && pg->variant == h->kv_variant && pg->form == v.form &&
      pg->engine == h->cg_engine) {
    *out = pg;
    return MFTO_OK;
  }
  destroy_graph(pg);
  h->pcg_graph[slot] = nullptr;
  pg = new PcgGraph();
  pg->key[0] = v.E;
  pg->key[1] = v.u;
  pg->key[2] = v.s;
  pg->chunk = chunk;
  pg->timed = h->kv_timing;
  pg->variant = h->kv_variant;
  pg->form = v.form;
  pg->engine = h->cg_engine;
  if (pg->timed) {
    pg->ev.resize(2 * chunk);
    for (auto& e : pg->ev) cudaEventCreate(&e);
  }
  // Captured on a private stream (the caller's stream may be the legacy
  // default stream, which cannot be captured); launched on the caller's.
  cudaGraph_t graph = nullptr;
  if (!h->cap_stream &&
      cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    destroy_graph(pg);
    return mfto_fail(h, MFTO_CUDA_ERROR, "PCG graph: cannot create the capture stream");
  }
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    destroy_graph(pg);
    return mfto_fail(h, MFTO_CUDA_ERROR, "PCG graph capture: %s", cudaGetErrorString(e));
  }
  mfto_status s = enqueue_chunk<T>(h, h->cap_stream, v, chunk, pg->timed ? pg->ev.data() : nullptr);
  e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (s != MFTO_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    destroy_graph(pg);
    return s != MFTO_OK ? s
                        : mfto_fail(h, MFTO_CUDA_ERROR, "PCG graph capture: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&pg->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    destroy_graph(pg);
    return mfto_fail(h, MFTO_CUDA_ERROR, "PCG graph instantiate: %s", cudaGetErrorString(e));
  }
  h->pcg_graph[slot] = pg;
  *out = pg;
  return MFTO_OK;
}

}  // namespace

namespace {
__global__ void fill_f32(float* x, int n, float v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}
}  // namespace

// Device time of one FP32 inner CG iteration as the graph engines run it
// (the captured chunk of K.v and vector-update launches, replayed `chunks`
// times after one untimed replay) on the handle's FP32 work vectors: unit
// moduli, a right-hand side of ones, a tolerance no iterate reaches.
mfto_status pcg_time_iterations(mfto_handle* h, int chunks, float* us_per_iter) {
  const int n = (int)h->n_dof;
  const int nb = reduction_blocks(h->n_dof, MFTO_BLOCK);
  const bool timed = h->kv_timing;
  h->kv_timing = false;
  h->launches += 2;
  fill_f32<<<nb, MFTO_BLOCK, 0, h->stream>>>(h->d_E32, (int)h->n_elem, 1.f);
  fill_f32<<<nb, MFTO_BLOCK, 0, h->stream>>>(h->d_r32, n, 1.f);
  MFTO_LAUNCH_CHECK(h);
  MFTO_CUDA(h, cudaMemsetAsync(h->d_e32, 0, sizeof(float) * h->n_dof, h->stream));
  mfto_status s = diag_launch(h, MFTO_FORM_F32, h->d_E32, h->d_dinv32, true);
  const PcgVecs<float> v{h->d_E32, h->d_e32, h->d_r32, h->d_z32, h->d_p0_32, h->d_p1_32,
                         h->d_q32, h->d_dinv32, h->d_pcg32, h->d_partials, h->d_partials2,
                         MFTO_FORM_F32};
  if (s == MFTO_OK) s = pcg_start<float>(h, v, h->d_r32, nullptr, 1e-30, 1 << 30, 0.0);
  if (s == MFTO_OK && cg2_active(h, MFTO_FORM_F32)) s = cg2_seed(h, v, 0.0);
  PcgGraph* pg = nullptr;
  if (s == MFTO_OK) s = get_graph<float>(h, v, 1, &pg);
  h->kv_timing = timed;
  if (s != MFTO_OK) return s;
  cudaEvent_t a, b;
  MFTO_CUDA(h, cudaEventCreate(&a));
  MFTO_CUDA(h, cudaEventCreate(&b));
  cudaError_t e = cudaGraphLaunch(pg->exec, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
  for (int c = 0; c < chunks && e == cudaSuccess; ++c) e = cudaGraphLaunch(pg->exec, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess)
    return mfto_fail(h, MFTO_CUDA_ERROR, "CG iteration timing: %s", cudaGetErrorString(e));
  h->launches += 2 * (int64_t)pg->chunk * (chunks + 1);
  *us_per_iter = 1000.f * ms / (float)(chunks * pg->chunk);
  return MFTO_OK;
}

// Device time of the FP32 CG K.v launch of engine 2 on this handle's mesh,
// launch shape and work vectors: `launches` launches of the first inner
// iteration's K.v (the same kernel, grid and arguments as in the CG graphs;
// unit moduli, a right-hand side of ones) captured back to back in one CUDA
// graph, one untimed replay, then `reps` replays between two events.  Each
// launch repeats the same work (it reads z and the seeded partials, writes
// p_new, q and its p.q partials), so the time per launch is the kernel's
// duration plus the gap between consecutive kernels of a graph, without the
// cost of event nodes between launches.  Overwrites the FP32 work vectors.
mfto_status pcg_time_kv(mfto_handle* h, int launches, int reps, bool events,
                        double* us_per_launch) {
  if (!cg2_active(h, MFTO_FORM_F32))
    return mfto_fail(h, MFTO_INVALID_ARG,
                     "K.v burst timing: needs CG engine 2 and the FP32 column K.v");
  const int n = (int)h->n_dof;
  const int nb = reduction_blocks(h->n_dof, MFTO_BLOCK);
  h->launches += 2;
  fill_f32<<<nb, MFTO_BLOCK, 0, h->stream>>>(h->d_E32, (int)h->n_elem, 1.f);
  fill_f32<<<nb, MFTO_BLOCK, 0, h->stream>>>(h->d_r32, n, 1.f);
  MFTO_LAUNCH_CHECK(h);
  MFTO_CUDA(h, cudaMemsetAsync(h->d_e32, 0, sizeof(float) * h->n_dof, h->stream));
  mfto_status s = diag_launch(h, MFTO_FORM_F32, h->d_E32, h->d_dinv32, true);
  const PcgVecs<float> v{h->d_E32, h->d_e32, h->d_r32, h->d_z32, h->d_p0_32, h->d_p1_32,
                         h->d_q32, h->d_dinv32, h->d_pcg32, h->d_partials, h->d_partials2,
                         MFTO_FORM_F32};
  if (s == MFTO_OK) s = pcg_start<float>(h, v, h->d_r32, nullptr, 1e-30, 1 << 30, 0.0);
  if (s == MFTO_OK) s = cg2_seed(h, v, 0.0);
  if (s != MFTO_OK) return s;
  if (!h->cap_stream)
    MFTO_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  // with events: an external record node before and after every launch, as
  // mfto_kv_timing places them in the CG graphs
  std::vector<cudaEvent_t> ev(events ? 2 * launches : 0, nullptr);
  for (auto& x : ev)
    if (s == MFTO_OK && cudaEventCreate(&x) != cudaSuccess)
      s = mfto_fail(h, MFTO_CUDA_ERROR, "K.v burst timing: cannot create events");
  auto destroy_events = [&]() {
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
  };
  if (s != MFTO_OK) {
    destroy_events();
    return s;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    destroy_events();
    return mfto_fail(h, MFTO_CUDA_ERROR, "K.v burst capture: %s", cudaGetErrorString(e));
  }
  for (int i = 0; i < launches && s == MFTO_OK; ++i) {
    if (events && cudaEventRecordWithFlags(ev[2 * i], h->cap_stream, cudaEventRecordExternal) !=
                      cudaSuccess)
      s = mfto_fail(h, MFTO_CUDA_ERROR, "K.v burst capture: event record");
    if (s == MFTO_OK) s = cg2_enqueue_kv(h, h->cap_stream, v, h->d_p0_32, h->d_p1_32, 0);
    if (s == MFTO_OK && events &&
        cudaEventRecordWithFlags(ev[2 * i + 1], h->cap_stream, cudaEventRecordExternal) !=
            cudaSuccess)
      s = mfto_fail(h, MFTO_CUDA_ERROR, "K.v burst capture: event record");
  }
  e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (s != MFTO_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    destroy_events();
    return s != MFTO_OK ? s : mfto_fail(h, MFTO_CUDA_ERROR, "K.v burst capture: %s",
                                        cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    destroy_events();
    return mfto_fail(h, MFTO_CUDA_ERROR, "K.v burst instantiate: %s", cudaGetErrorString(e));
  }
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  // with events: the mean of the per-launch event intervals of the last replay
  double ev_ms = 0.0;
  for (int i = 0; events && i < launches && e == cudaSuccess; ++i) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
    ev_ms += t;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  destroy_events();
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess)
    return mfto_fail(h, MFTO_CUDA_ERROR, "K.v burst timing: %s", cudaGetErrorString(e));
  h->launches += (int64_t)launches * (reps + 1);
  *us_per_launch = events ? 1000.0 * ev_ms / launches : 1000.0 * ms / ((double)reps * launches);
  return MFTO_OK;
}

extern "C" mfto_status mfto_cg_kv_time(mfto_handle* h, int32_t launches, int32_t reps,
                                       int32_t events, double* us_per_launch) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, us_per_launch && launches >= 1 && launches <= 4096 && reps >= 1 &&
                      (events == 0 || events == 1),
               "mfto_cg_kv_time: launches in [1, 4096], reps >= 1, events 0 or 1, non-null "
               "output");
  return pcg_time_kv(h, launches, reps, events != 0, us_per_launch);
}

void pcg_graph_release(mfto_handle* h) {
  for (int i = 0; i < MFTO_PCG_SLOTS; ++i) {
    destroy_graph(h->pcg_graph[i]);
    h->pcg_graph[i] = nullptr;
  }
}

template <typename T>
mfto_status pcg_start(mfto_handle* h, const PcgVecs<T>& v, const T* rhs, const T* Ku, double rtol,
                      int maxit, double rz_prev) {
  const int nb_dof = reduction_blocks(h->n_dof, MFTO_BLOCK);
  // the first iteration reads its previous direction from p0: zero unless a
  // direction is continued
  if (!(rz_prev > 0.0)) {
    rz_prev = 0.0;
    MFTO_CUDA(h, cudaMemsetAsync(v.p0, 0, sizeof(T) * h->n_dof, h->stream));
  }
  h->launches++;
  pcg_init<T><<<nb_dof, MFTO_BLOCK, 0, h->stream>>>(rhs, Ku, v.dinv, v.r, v.z, (int)h->n_dof,
                                                    rtol, maxit, rz_prev, v.s, v.part_a);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

template <typename T>
mfto_status pcg_iterate(mfto_handle* h, const PcgVecs<T>& v, int slot, PcgScalars* host_s) {
  PcgGraph* pg = nullptr;
  mfto_status s = get_graph<T>(h, v, slot, &pg);
  if (s != MFTO_OK) return s;
  int it_before = 0;
  for (;;) {
    MFTO_CUDA(h, cudaMemcpyAsync(host_s, v.s, sizeof(PcgScalars), cudaMemcpyDeviceToHost, h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
    const int progress = host_s->it;   // iterations completed so far
    if (pg->timed) {
      // harvest the K.v launches of the previous chunk that did work
      const int ran = progress - it_before +
                      (host_s->done && host_s->status == MFTO_BREAKDOWN ? 1 : 0);
      for (int i = 0; i < ran && i < pg->chunk; ++i) {
        float ms = 0.f;
        MFTO_CUDA(h, cudaEventElapsedTime(&ms, pg->ev[2 * i], pg->ev[2 * i + 1]));
        const int f = sizeof(T) == 8 ? 0 : 1;
        h->ev.total_ms[f] += ms;
        h->ev.launches[f]++;
      }
      it_before = progress;
    }
    if (host_s->tc_error)
      return mfto_fail(h, MFTO_CUDA_ERROR, "a completion wait (tensor-core or bulk copy) timed out");
    if (host_s->done) break;
    MFTO_CUDA(h, cudaGraphLaunch(pg->exec, h->stream));
    h->launches += 2 * (int64_t)pg->chunk;
  }
  return MFTO_OK;
}

template mfto_status pcg_start<double>(mfto_handle*, const PcgVecs<double>&, const double*,
                                       const double*, double, int, double);
template mfto_status pcg_start<float>(mfto_handle*, const PcgVecs<float>&, const float*,
                                      const float*, double, int, double);
template mfto_status pcg_iterate<double>(mfto_handle*, const PcgVecs<double>&, int, PcgScalars*);
template mfto_status pcg_iterate<float>(mfto_handle*, const PcgVecs<float>&, int, PcgScalars*);

mfto_status pcg_run(mfto_handle* h, const double* E, const double* f, double* u,
                    mfto_solve_stats* st) {
  mfto_status s = diag_launch(h, MFTO_FORM_F64, E, h->d_dinv, true);
  if (s != MFTO_OK) return s;
  s = kv_launch(h, MFTO_FORM_F64, E, u, h->d_q);
  if (s != MFTO_OK) return s;
  const PcgVecs<double> v{E, u, h->d_r, h->d_z, h->d_p0, h->d_p1, h->d_q, h->d_dinv,
                          h->d_pcg, h->d_partials, h->d_partials2, MFTO_FORM_F64};
  s = pcg_start<double>(h, v, f, h->d_q, h->p.rtol, h->p.maxit);
  if (s != MFTO_OK) return s;
  s = pcg_iterate<double>(h, v, 0, h->h_pcg);
  if (s != MFTO_OK) return s;
  if (h->h_pcg->ff == 0.0) MFTO_CUDA(h, cudaMemsetAsync(u, 0, sizeof(double) * h->n_dof, h->stream));
  if (st) {
    st->iterations = h->h_pcg->it;
    st->status = h->h_pcg->status;
    st->fnorm = sqrt(h->h_pcg->ff);
    st->rel_residual = h->h_pcg->ff > 0.0 ? sqrt(h->h_pcg->rr / h->h_pcg->ff) : 0.0;
  }
  return MFTO_OK;
}

extern "C" mfto_status mfto_pcg(mfto_handle* h, const double* E, const double* f, double* u,
                                mfto_solve_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, E && f && u, "mfto_pcg: null pointer");
  return pcg_run(h, E, f, u, st);
}

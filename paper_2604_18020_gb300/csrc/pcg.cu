// FP64 Jacobi-preconditioned CG (Sec. 3.6) with warm start.
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

#include "common.cuh"
#include "kv_node.cuh"

struct PcgGraph {
  const void* E = nullptr;
  const void* u = nullptr;
  int chunk = 0;
  bool timed = false;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;  // 2 per K.v launch when timed
};

namespace {

__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_init(const double* __restrict__ f, const double* __restrict__ Ku, const double* __restrict__ dinv,
         double* __restrict__ r, double* __restrict__ z, int n, double rtol, int maxit,
         PcgScalars* s, double* partials) {
  __shared__ double sh[64];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double ri = f[i] - Ku[i];
    const double zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    acc[0] += ri * zi;
    acc[1] += ri * ri;
    acc[2] += f[i] * f[i];
  }
  double tot[3];
  if (last_block_reduce<3>(acc, partials, &s->ticket_a, tot, sh) && threadIdx.x == 0) {
    s->rz = tot[0];
    s->rr = tot[1];
    s->ff = tot[2];
    s->rtol2ff = rtol * rtol * tot[2];
    s->beta = 0.0;
    s->alpha = 0.0;
    s->it = 0;
    s->maxit = maxit;
    s->status = MFTO_OK;
    s->done = (tot[2] == 0.0 || tot[1] <= s->rtol2ff) ? 1 : 0;
    if (!isfinite(tot[0]) || !isfinite(tot[1])) { s->done = 1; s->status = MFTO_BREAKDOWN; }
  }
}

// A: p_new = z + beta p_old (own nodes written), q = K p_new, alpha = rz / p_new.q
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_kv_step(const double* __restrict__ E, const double* __restrict__ z,
            const double* __restrict__ p_old, double* __restrict__ p_new,
            double* __restrict__ q, const uint8_t* __restrict__ fixed,
            const double* __restrict__ ke_g, Grid g, int n_node, PcgScalars* s,
            double* partials) {
  if (*(volatile int32_t*)&s->done) return;  // uniform over the grid
  __shared__ double ke[576];
  __shared__ double sh[64];
  for (int t = threadIdx.x; t < 576; t += blockDim.x) ke[t] = ke_g[t];
  __syncthreads();
  const double beta = s->beta;
  const LoadDirection<double> ld{z, p_old, beta};
  double acc[1] = {0.0};
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < n_node;
       node += gridDim.x * blockDim.x) {
    double a[3];
    node_kv<double>(node, E, fixed, ke, g, ld, a[0], a[1], a[2]);
    const uint8_t fm = fixed[node];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double pn = ((fm >> c) & 1) ? 0.0 : ld(3 * node + c);
      const double qc = ((fm >> c) & 1) ? pn : a[c];
      p_new[3 * node + c] = pn;
      q[3 * node + c] = qc;
      acc[0] += pn * qc;
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
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_update(double* __restrict__ u, const double* __restrict__ p, const double* __restrict__ q,
           double* __restrict__ r, double* __restrict__ z, const double* __restrict__ dinv,
           int n, PcgScalars* s, double* partials) {
  if (*(volatile int32_t*)&s->done) return;
  __shared__ double sh[64];
  const double alpha = s->alpha;
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    u[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    const double zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    acc[0] += ri * zi;
    acc[1] += ri * ri;
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

}  // namespace

static mfto_status enqueue_chunk(mfto_handle* h, cudaStream_t st, const double* E, double* u,
                                 int chunk, cudaEvent_t* ev) {
  const Grid g = make_grid(h->mesh);
  const int nb_node = reduction_blocks(h->n_node, MFTO_BLOCK);
  const int nb_dof = reduction_blocks(h->n_dof, MFTO_BLOCK);
  for (int it = 0; it < chunk; ++it) {
    double* p_old = (it & 1) ? h->d_p1 : h->d_p0;
    double* p_new = (it & 1) ? h->d_p0 : h->d_p1;
    // external record nodes: a plain record inside a capture would only add a
    // dependency edge, not record the event on each graph launch
    if (ev) MFTO_CUDA(h, cudaEventRecordWithFlags(ev[2 * it], st, cudaEventRecordExternal));
    if (h->kv_variant == 0) {
      mfto_status s = pcg_kv_tile_launch<double>(h, E, h->d_z, p_old, p_new, h->d_q, h->d_pcg,
                                                 h->d_partials, st);
      if (s != MFTO_OK) return s;
    } else {
      pcg_kv_step<<<nb_node, MFTO_BLOCK, 0, st>>>(E, h->d_z, p_old, p_new, h->d_q, h->d_fixed,
                                                  h->d_ke64, g, (int)h->n_node, h->d_pcg,
                                                  h->d_partials);
    }
    if (ev) MFTO_CUDA(h, cudaEventRecordWithFlags(ev[2 * it + 1], st, cudaEventRecordExternal));
    pcg_update<<<nb_dof, MFTO_BLOCK, 0, st>>>(u, p_new, h->d_q, h->d_r, h->d_z,
                                                    h->d_dinv, (int)h->n_dof, h->d_pcg,
                                                    h->d_partials2);
  }
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

static void destroy_graph(PcgGraph* pg) {
  if (!pg) return;
  if (pg->exec) cudaGraphExecDestroy(pg->exec);
  for (cudaEvent_t e : pg->ev) cudaEventDestroy(e);
  delete pg;
}

void pcg_graph_release(mfto_handle* h) {
  destroy_graph(h->pcg_graph);
  h->pcg_graph = nullptr;
}

static mfto_status get_graph(mfto_handle* h, const double* E, double* u, PcgGraph** out) {
  const int chunk = h->p.check_every;
  PcgGraph* pg = h->pcg_graph;
  if (pg && pg->E == E && pg->u == u && pg->chunk == chunk && pg->timed == h->kv_timing) {
    *out = pg;
    return MFTO_OK;
  }
  pcg_graph_release(h);
  pg = new PcgGraph();
  pg->E = E;
  pg->u = u;
  pg->chunk = chunk;
  pg->timed = h->kv_timing;
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
  mfto_status s = enqueue_chunk(h, h->cap_stream, E, u, chunk, pg->timed ? pg->ev.data() : nullptr);
  e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (s != MFTO_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    destroy_graph(pg);
    return s != MFTO_OK ? s : mfto_fail(h, MFTO_CUDA_ERROR, "PCG graph capture: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&pg->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    destroy_graph(pg);
    return mfto_fail(h, MFTO_CUDA_ERROR, "PCG graph instantiate: %s", cudaGetErrorString(e));
  }
  h->pcg_graph = pg;
  *out = pg;
  return MFTO_OK;
}

mfto_status pcg_run(mfto_handle* h, const double* E, const double* f, double* u,
                    mfto_solve_stats* st) {
  const int nb_dof = reduction_blocks(h->n_dof, MFTO_BLOCK);
  mfto_status s = diag_launch(h, MFTO_FORM_F64, E, h->d_dinv, true);
  if (s != MFTO_OK) return s;
  s = kv_launch(h, MFTO_FORM_F64, E, u, h->d_q);
  if (s != MFTO_OK) return s;
  MFTO_CUDA(h, cudaMemsetAsync(h->d_p0, 0, sizeof(double) * h->n_dof, h->stream));
  h->launches++;
  pcg_init<<<nb_dof, MFTO_BLOCK, 0, h->stream>>>(f, h->d_q, h->d_dinv, h->d_r, h->d_z,
                                                 (int)h->n_dof, h->p.rtol, h->p.maxit,
                                                 h->d_pcg, h->d_partials);
  MFTO_LAUNCH_CHECK(h);
  PcgGraph* pg = nullptr;
  s = get_graph(h, E, u, &pg);
  if (s != MFTO_OK) return s;
  int it_before = 0;
  for (;;) {
    MFTO_CUDA(h, cudaMemcpyAsync(h->h_pcg, h->d_pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost,
                                 h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
    if (pg->timed) {
      // harvest the K.v launches of the previous chunk that did work
      const int ran = h->h_pcg->it - it_before + (h->h_pcg->status == MFTO_BREAKDOWN ? 1 : 0);
      for (int i = 0; i < ran && i < pg->chunk; ++i) {
        float ms = 0.f;
        MFTO_CUDA(h, cudaEventElapsedTime(&ms, pg->ev[2 * i], pg->ev[2 * i + 1]));
        h->ev.total_ms += ms;
        h->ev.launches++;
      }
      it_before = h->h_pcg->it;
    }
    if (h->h_pcg->done) break;
    MFTO_CUDA(h, cudaGraphLaunch(pg->exec, h->stream));
    h->launches += 2 * (int64_t)pg->chunk;
  }
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

// Mixed-precision solve: FP64 iterative refinement around an FP32 inner
// Jacobi-PCG (the residual-correction loop of Sec. 3.5, with the outer
// residual, norms and accumulation in FP64 and the inner solve's dot products
// in FP64 as well).
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace {

__global__ void __launch_bounds__(MFTO_BLOCK)
to_f32(const double* __restrict__ a, float* __restrict__ b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// r = f - Ku (FP64); r.r and f.f reduced (sum[0], sum[1]); r stored as FP32
// (the right-hand side of the inner solve).
__global__ void __launch_bounds__(MFTO_BLOCK)
ir_residual(const double* __restrict__ f, const double* __restrict__ Ku,
            float* __restrict__ r32, int n, MiscScalars* s, double* partials) {
  __shared__ double sh[64];
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double ri = f[i] - Ku[i];
    r32[i] = (float)ri;
    acc[0] += ri * ri;
    acc[1] += f[i] * f[i];
  }
  double tot[2];
  if (last_block_reduce<2>(acc, partials, &s->ticket, tot, sh) && threadIdx.x == 0) {
    s->sum[0] = tot[0];
    s->sum[1] = tot[1];
  }
}

// u += e (the FP32 correction added in FP64)
__global__ void __launch_bounds__(MFTO_BLOCK)
ir_accumulate(double* __restrict__ u, const float* __restrict__ e, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    u[i] += (double)e[i];
}

}  // namespace

mfto_status mfto_to_f32(mfto_handle* h, const double* a, float* b, int64_t n) {
  h->launches++;
  to_f32<<<reduction_blocks(n, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(a, b, (int)n);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

mfto_status ir_run(mfto_handle* h, mfto_form inner, double inner_tol, const double* E,
                   const double* f, double* u, mfto_ir_stats* st) {
  if (inner != MFTO_FORM_F32 && !tc_form(inner))
    return mfto_fail(h, MFTO_UNSUPPORTED, "mfto_ir_solve: unsupported inner form %d", (int)inner);
  if (!(inner_tol > 0.0 && inner_tol < 1.0))
    return mfto_fail(h, MFTO_INVALID_ARG, "mfto_ir_solve: inner_tol must lie in (0, 1)");
  const int n = (int)h->n_dof;
  const int nb_dof = reduction_blocks(h->n_dof, MFTO_BLOCK);
  const int nb_el = reduction_blocks(h->n_elem, MFTO_BLOCK);
  mfto_ir_stats local;
  mfto_ir_stats* out = st ? st : &local;
  memset(out, 0, sizeof(*out));
  // FP32 modulus and inverse Jacobi diagonal, once per solve
  h->launches++;
  to_f32<<<nb_el, MFTO_BLOCK, 0, h->stream>>>(E, h->d_E32, (int)h->n_elem);
  MFTO_LAUNCH_CHECK(h);
  mfto_status s = diag_launch(h, MFTO_FORM_F32, h->d_E32, h->d_dinv32, true);
  if (s != MFTO_OK) return s;
  // inner solve K e = r: the FP32 right-hand side is written into the inner
  // residual buffer, which pcg_init turns into r = rhs in place
  const PcgVecs<float> v{h->d_E32, h->d_e32, h->d_r32, h->d_z32, h->d_p0_32, h->d_p1_32,
                         h->d_q32, h->d_dinv32, h->d_pcg32, h->d_partials, h->d_partials2,
                         (int)inner};
  double prev = 0.0;
  double rz_prev = 0.0;   // > 0: the next inner solve continues the last direction
  int stalls = 0;
  out->status = MFTO_NOT_CONVERGED;
  for (int outer = 0;; ++outer) {
    s = kv_launch(h, MFTO_FORM_F64, E, u, h->d_q);
    if (s != MFTO_OK) return s;
    out->kv_f64++;
    h->launches++;
    ir_residual<<<nb_dof, MFTO_BLOCK, 0, h->stream>>>(f, h->d_q, h->d_r32, n, h->d_misc,
                                                      h->d_partials);
    MFTO_LAUNCH_CHECK(h);
    MFTO_CUDA(h, cudaMemcpyAsync(h->h_misc, h->d_misc, sizeof(MiscScalars),
                                 cudaMemcpyDeviceToHost, h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
    const double rr = h->h_misc->sum[0], ff = h->h_misc->sum[1];
    out->fnorm = sqrt(ff);
    if (ff == 0.0) {
      MFTO_CUDA(h, cudaMemsetAsync(u, 0, sizeof(double) * h->n_dof, h->stream));
      out->rel_residual = 0.0;
      out->status = MFTO_OK;
      break;
    }
    const double rel = sqrt(rr / ff);
    out->rel_residual = rel;
    if (outer < 64) out->history[outer] = rel;
    if (!isfinite(rel)) { out->status = MFTO_BREAKDOWN; break; }
    if (rel <= h->p.rtol) { out->status = MFTO_OK; break; }
    if (outer > 0) {
      stalls = rel > 0.9 * prev ? stalls + 1 : 0;
      if (stalls >= 2) { out->status = MFTO_STALLED; break; }
    }
    if (outer >= h->max_outer) { out->status = MFTO_NOT_CONVERGED; break; }
    prev = rel;
    // inner solve from e = 0
    MFTO_CUDA(h, cudaMemsetAsync(h->d_e32, 0, sizeof(float) * h->n_dof, h->stream));
    s = pcg_start<float>(h, v, h->d_r32, nullptr, inner_tol, h->inner_maxit, rz_prev);
    if (s != MFTO_OK) return s;
    if (cg2_active(h, inner)) {
      s = cg2_seed(h, v, rz_prev);
      if (s != MFTO_OK) return s;
    }
    if (h->cg_engine == 1 && inner == MFTO_FORM_F32 && h->kv_variant == 0)
      s = pcg_persist_iterate(h, v, h->h_pcg32);
    else
      s = pcg_iterate<float>(h, v, 1, h->h_pcg32);
    if (s != MFTO_OK) return s;
    const PcgScalars& fin = *h->h_pcg32;
    out->inner_iterations += fin.it;
    if (fin.status == MFTO_BREAKDOWN) { out->status = MFTO_BREAKDOWN; break; }
    // Continued direction (reliable updating): the next inner solve starts
    // from the true FP64 residual but keeps the last search direction p_{k-1}
    // and the r.z of the iteration that formed it, rho_{k-1} = rho_k / beta_k,
    // so the first new direction is z + (rho / rho_{k-1}) p_{k-1}.  Iteration j
    // writes its direction into p1 (j even) or p0 (j odd); the next solve reads
    // p0 first.
    rz_prev = 0.0;
    if (h->ir_mode == MFTO_IR_CONTINUE && fin.it >= 1 && fin.beta > 0.0 &&
               isfinite(fin.rz / fin.beta)) {
      if (fin.it & 1)
        MFTO_CUDA(h, cudaMemcpyAsync(h->d_p0_32, h->d_p1_32, sizeof(float) * h->n_dof,
                                     cudaMemcpyDeviceToDevice, h->stream));
      rz_prev = fin.rz / fin.beta;
    }
    h->launches++;
    ir_accumulate<<<nb_dof, MFTO_BLOCK, 0, h->stream>>>(u, h->d_e32, n);
    MFTO_LAUNCH_CHECK(h);
    out->outer_iterations++;
  }
  return MFTO_OK;
}

extern "C" mfto_status mfto_ir_solve(mfto_handle* h, mfto_form inner, double inner_tol,
                                     const double* E, const double* f, double* u,
                                     mfto_ir_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, E && f && u, "mfto_ir_solve: null pointer");
  return ir_run(h, inner, inner_tol, E, f, u, st);
}

extern "C" mfto_status mfto_set_solver(mfto_handle* h, mfto_form form, double inner_tol,
                                       int32_t inner_maxit, int32_t max_outer) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, form == MFTO_FORM_F64 || form == MFTO_FORM_F32 || tc_form(form),
               "mfto_set_solver: unsupported form");
  MFTO_REQUIRE(h, inner_tol > 0.0 && inner_tol < 1.0, "mfto_set_solver: inner_tol in (0, 1)");
  MFTO_REQUIRE(h, inner_maxit >= 1 && max_outer >= 1, "mfto_set_solver: caps must be >= 1");
  h->solver_form = form;
  h->inner_tol = inner_tol;
  h->inner_maxit = inner_maxit;
  h->max_outer = max_outer;
  return MFTO_OK;
}

extern "C" mfto_status mfto_set_ir_mode(mfto_handle* h, int32_t mode) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, mode == MFTO_IR_RESTART || mode == MFTO_IR_CONTINUE,
               "mfto_set_ir_mode: mode must be MFTO_IR_RESTART or MFTO_IR_CONTINUE");
  h->ir_mode = mode;
  return MFTO_OK;
}

// Matrix-free estimate of the condition number kappa(K) of the stiffness
// matrix on the free DOFs (Sec. 3.5, "Condition number of the SIMP stiffness
// matrix", and the kappa results of Sec. 5): lambda_max by power iteration,
// lambda_min by inverse iteration with Jacobi-PCG inner solves, both through
// the FP64 K.v only.
//
// The start vectors are zeroed on the fixed DOFs; the masked K.v (identity
// rows there) and the PCG solves then keep every iterate zero on them, so
// the estimate is that of K_ff.  Each step's eigenvalue estimate is the
// Rayleigh quotient of the current unit vector:
//   power:   w = K v;  lambda = v.w;  v = w / ||w||;
//   inverse: x = K^-1 v (PCG from 0 to rtol);  mu = v.x;  v = x / ||x||;
//            lambda_min = 1 / mu;
// each loop stops when its estimate changes by less than its relative
// tolerance, or at its step cap.  Dot products are FP64 on the device
// (fixed-order block partials); the scalar recurrences run on the host.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace {

// a.b and b.b -> s->sum[0], s->sum[1]
__global__ void __launch_bounds__(MFTO_BLOCK)
dot2_kernel(const double* __restrict__ a, const double* __restrict__ b, int n, MiscScalars* s,
            double* partials) {
  __shared__ double sh[64];
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double bi = b[i];
    acc[0] += a[i] * bi;
    acc[1] += bi * bi;
  }
  double tot[2];
  if (last_block_reduce<2>(acc, partials, &s->ticket, tot, sh) && threadIdx.x == 0) {
    s->sum[0] = tot[0];
    s->sum[1] = tot[1];
  }
}

// dst = c src
__global__ void __launch_bounds__(MFTO_BLOCK)
scale_kernel(const double* __restrict__ src, double* __restrict__ dst, double c, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = c * src[i];
}

// zero the fixed DOFs of v
__global__ void __launch_bounds__(MFTO_BLOCK)
mask_kernel(double* __restrict__ v, const uint8_t* __restrict__ fixed, int n_node) {
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < n_node; nd += gridDim.x * blockDim.x) {
    const uint8_t fm = fixed[nd];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if ((fm >> c) & 1) v[3 * nd + c] = 0.0;
  }
}

// (a.b, b.b) on the host
mfto_status dot2(mfto_handle* h, const double* a, const double* b, double* ab, double* bb) {
  h->launches++;
  dot2_kernel<<<reduction_blocks(h->n_dof, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(
      a, b, (int)h->n_dof, h->d_misc, h->d_partials);
  MFTO_LAUNCH_CHECK(h);
  MFTO_CUDA(h, cudaMemcpyAsync(h->h_misc, h->d_misc, sizeof(MiscScalars), cudaMemcpyDeviceToHost,
                               h->stream));
  MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  *ab = h->h_misc->sum[0];
  *bb = h->h_misc->sum[1];
  return MFTO_OK;
}

mfto_status scale(mfto_handle* h, const double* src, double* dst, double c) {
  h->launches++;
  scale_kernel<<<reduction_blocks(h->n_dof, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(
      src, dst, c, (int)h->n_dof);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

mfto_status mask_and_normalise(mfto_handle* h, double* v) {
  h->launches++;
  mask_kernel<<<reduction_blocks(h->n_node, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(
      v, h->d_fixed, (int)h->n_node);
  MFTO_LAUNCH_CHECK(h);
  double ab = 0.0, vv = 0.0;
  mfto_status s = dot2(h, v, v, &ab, &vv);
  if (s != MFTO_OK) return s;
  if (!(vv > 0.0) || !isfinite(vv))
    return mfto_fail(h, MFTO_INVALID_ARG, "mfto_kappa: a start vector is zero on the free DOFs");
  return scale(h, v, v, 1.0 / sqrt(vv));
}

}  // namespace

extern "C" void mfto_default_kappa_params(mfto_kappa_params* p) {
  if (!p) return;
  p->power_maxit = 50;
  p->power_tol = 1e-6;
  p->inverse_maxit = 50;
  p->inverse_tol = 1e-4;
  p->inner_rtol = 1e-8;
  p->inner_maxit = 2000;
}

extern "C" mfto_status mfto_kappa(mfto_handle* h, const double* E, double* v_power,
                                  double* v_inverse, double* work, const mfto_kappa_params* prm,
                                  mfto_kappa_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, E && v_power && v_inverse && work && st, "mfto_kappa: null pointer");
  mfto_kappa_params p;
  if (prm) p = *prm; else mfto_default_kappa_params(&p);
  MFTO_REQUIRE(h, p.power_maxit >= 1 && p.inverse_maxit >= 1 && p.inner_maxit >= 1,
               "mfto_kappa: caps must be >= 1");
  MFTO_REQUIRE(h, p.power_tol >= 0.0 && p.inverse_tol >= 0.0 && p.inner_rtol > 0.0,
               "mfto_kappa: tolerances must be >= 0 (inner_rtol > 0)");
  memset(st, 0, sizeof(*st));
  // ---- power iteration
  mfto_status s = mask_and_normalise(h, v_power);
  if (s != MFTO_OK) return s;
  double lam = 0.0, lam_prev = 0.0;
  for (int k = 1; k <= p.power_maxit; ++k) {
    s = kv_launch(h, MFTO_FORM_F64, E, v_power, work);
    if (s != MFTO_OK) return s;
    double vw = 0.0, ww = 0.0;
    s = dot2(h, v_power, work, &vw, &ww);
    if (s != MFTO_OK) return s;
    lam = vw;
    st->power_steps = k;
    if (!(ww > 0.0) || !isfinite(ww))
      return mfto_fail(h, MFTO_BREAKDOWN, "mfto_kappa: K v vanished in power iteration");
    s = scale(h, work, v_power, 1.0 / sqrt(ww));
    if (s != MFTO_OK) return s;
    if (k > 1 && fabs(lam - lam_prev) <= p.power_tol * fabs(lam)) break;
    lam_prev = lam;
  }
  st->lambda_max = lam;
  // ---- inverse iteration (the handle's PCG with the inner tolerance and cap)
  s = mask_and_normalise(h, v_inverse);
  if (s != MFTO_OK) return s;
  const double rtol_saved = h->p.rtol;
  const int32_t maxit_saved = h->p.maxit;
  h->p.rtol = p.inner_rtol;
  h->p.maxit = p.inner_maxit;
  double mu = 0.0, mu_prev = 0.0;
  for (int k = 1; k <= p.inverse_maxit; ++k) {
    s = [&]() -> mfto_status {
      MFTO_CUDA(h, cudaMemsetAsync(work, 0, sizeof(double) * h->n_dof, h->stream));
      return MFTO_OK;
    }();
    if (s != MFTO_OK) break;
    mfto_solve_stats ss;
    s = pcg_run(h, E, v_inverse, work, &ss);
    if (s != MFTO_OK) break;
    st->inner_iterations += ss.iterations;
    if (ss.status != MFTO_OK) st->inner_capped++;
    double vx = 0.0, xx = 0.0;
    s = dot2(h, v_inverse, work, &vx, &xx);
    if (s != MFTO_OK) break;
    mu = vx;
    st->inverse_steps = k;
    if (!(xx > 0.0) || !isfinite(xx) || !(mu > 0.0)) {
      s = mfto_fail(h, MFTO_BREAKDOWN, "mfto_kappa: inverse iteration broke down");
      break;
    }
    s = scale(h, work, v_inverse, 1.0 / sqrt(xx));
    if (s != MFTO_OK) break;
    if (k > 1 && fabs(mu - mu_prev) <= p.inverse_tol * fabs(mu)) break;
    mu_prev = mu;
  }
  h->p.rtol = rtol_saved;
  h->p.maxit = maxit_saved;
  if (s != MFTO_OK) return s;
  st->lambda_min = 1.0 / mu;
  st->kappa = st->lambda_max / st->lambda_min;
  return MFTO_OK;
}

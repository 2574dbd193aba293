// Compliance and sensitivities, the OC bisection update and one SIMP
// iteration (Sec. 3.1, Sec. 3.6 warm start).
#include <math.h>

#include "common.cuh"

namespace {

// ce_e = u_e^T KE u_e;  c = sum_e E_e ce_e;  dc_e = -p rho^(p-1) (E0-Emin) ce_e;
// grayness sum 4 rho (1 - rho).  One thread per element, fixed-order sums.
// The element energy is evaluated in the per-axis (sum, difference) mode
// basis of modes.cuh: with x = T u_e (the three butterfly stages per
// component) and KE = T^T Kt T / 8, u_e^T KE u_e = x . (Kt / 8) x, the sparse
// mode operator the K.v applies (about 150 FP64 operations instead of the
// 1,200 of the dense quadratic form).
__global__ void __launch_bounds__(MFTO_BLOCK)
compliance_kernel(const double* __restrict__ rho, const double* __restrict__ u,
                  double* __restrict__ dc, ModeCoef<double> K, Grid g,
                  double E0, double Emin, double penal, MiscScalars* s, double* partials) {
  __shared__ double sh[64];
  const int n = g.nelx * g.nely * g.nelz;
  double acc[2] = {0.0, 0.0};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int i = e % g.nelx, j = (e / g.nelx) % g.nely, k = e / (g.nelx * g.nely);
    double x[3][8];
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int m = (i + (l & 1)) + g.nx * ((j + ((l >> 1) & 1)) + g.ny * (k + (l >> 2)));
      x[0][l] = u[3 * m + 0];
      x[1][l] = u[3 * m + 1];
      x[2][l] = u[3 * m + 2];
    }
    // butterflies (v0, v1) -> (v0 + v1, v1 - v0) along x, y, z
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ax = 0; ax < 3; ++ax)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          if (m & (1 << ax)) continue;
          const double v0 = x[c][m], v1 = x[c][m | (1 << ax)];
          x[c][m] = v0 + v1;
          x[c][m | (1 << ax)] = v1 - v0;
        }
    double y[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int m = 0; m < 8; ++m) y[c][m] = K.diag[c][m] * x[c][m];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (a == b) continue;
        const int t = 3 - a - b;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const int tb = mt << t;
          y[a][(1 << a) | tb] = fma(K.lamM[mt], x[b][(1 << b) | tb], y[a][(1 << a) | tb]);
          y[a][(1 << b) | tb] = fma(K.muM[mt], x[b][(1 << a) | tb], y[a][(1 << b) | tb]);
        }
      }
    double ce = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int m = 0; m < 8; ++m) ce = fma(x[c][m], y[c][m], ce);
    const double r = rho[e];
    const double E = Emin + (E0 - Emin) * pow(r, penal);
    acc[0] += E * ce;
    acc[1] += 4.0 * r * (1.0 - r);
    if (dc) dc[e] = -penal * pow(r, penal - 1.0) * (E0 - Emin) * ce;
  }
  double tot[2];
  if (last_block_reduce<2>(acc, partials, &s->ticket, tot, sh) && threadIdx.x == 0) {
    s->sum[0] = tot[0];
    s->sum[1] = tot[1];
  }
}

// OC with bisection on lambda.  One cooperative grid of one CTA per SM.  A
// first pass forms per element a_e = rho_e sqrt(max(0, -dc_e) n) and the
// move-limit bounds, so that the candidate of a midpoint lambda is
// a_e / sqrt(lambda) (the same value as rho_e sqrt(max(0, -dc_e) / (lambda / n))
// up to rounding): each evaluation of the candidate volume is then one FP64
// multiply and a clamp per element, on values kept in registers (G > 0: up
// to G elements per thread) or re-read from the scratch arrays (G == 0,
// larger meshes).  An evaluation sums the candidate field, crosses a
// counting grid barrier (release-add of one arrival per CTA, acquire-polls
// until every CTA has arrived; bounded), and warp 0 of every CTA adds the
// per-CTA partials in the same order, so every CTA takes the same branch.
// Partials are double-buffered by evaluation parity.
//
// The bisection starts from [0, 1e9].  While its lower end is still 0, its
// midpoints are lambda_k = 1e9 / 2^k (k = 1, 2, ...: each the previous one
// halved, so exact down to the subnormal range), and it moves the upper end
// down until the first k* whose candidate volume exceeds the target.  That
// volume is nondecreasing in k (every step of its evaluation is monotone:
// rounded products, clamps and fixed-order rounded sums), so k* is found by
// a binary search over k, started at the previous call's k* (a hint that
// leaves the result unchanged and normally settles it in two evaluations),
// and the bisection then continues from exactly the state it would have
// reached step by step.  The candidate of the last midpoint is written by a
// final pass.
template <int G>
__global__ void __launch_bounds__(MFTO_BLOCK)
oc_kernel(const double* __restrict__ rho, const double* __restrict__ dc,
          double* __restrict__ rho_new, double* __restrict__ a_s, double* __restrict__ lo_s,
          double* __restrict__ hi_s, int n, double volfrac, double move, MiscScalars* s,
          double* partials, int k_end, int k_hint) {
  __shared__ double sh[64];
  const double target = volfrac * (double)n;
  const int first = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  double ra[G > 0 ? G : 1], rlo[G > 0 ? G : 1], rhi[G > 0 ? G : 1];
  if constexpr (G > 0) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int e = first + g * stride;
      ra[g] = 0.0;
      rlo[g] = 0.0;
      rhi[g] = 0.0;
      if (e < n) {
        const double r = rho[e];
        ra[g] = r * sqrt(fmax(0.0, -dc[e]) * (double)n);
        rlo[g] = fmax(0.0, r - move);
        rhi[g] = fmin(1.0, r + move);
      }
    }
  } else {
    for (int e = first; e < n; e += stride) {
      const double r = rho[e];
      a_s[e] = r * sqrt(fmax(0.0, -dc[e]) * (double)n);
      lo_s[e] = fmax(0.0, r - move);
      hi_s[e] = fmin(1.0, r + move);
    }
  }
  // the candidate sum at the scale sc = 1 / sqrt(lambda)
  auto volume = [&](double sc) {
    double acc = 0.0;
    if constexpr (G > 0) {
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (first + g * stride < n) acc += fmax(rlo[g], fmin(rhi[g], ra[g] * sc));
    } else {
      for (int e = first; e < n; e += stride) acc += fmax(lo_s[e], fmin(hi_s[e], a_s[e] * sc));
    }
    return acc;
  };
  unsigned int arrivals = 0;   // grid-barrier arrivals expected so far
  auto grid_sync = [&]() {
    arrivals += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
      red_release_add(&s->bar_count, 1u);
      volatile int32_t* verr = &s->error;
      unsigned int spins = 0;
      while (ld_acquire(&s->bar_count) < arrivals) {
        if (*verr) break;
        if (++spins > MFTO_SPIN_LIMIT) { atomicExch(&s->error, 1); break; }
      }
    }
    __syncthreads();
  };
  // 1 / sqrt(lambda) of each evaluation: formed once per CTA (the FP64 pipe
  // runs 2 operations per clock per SM) and handed over in shared memory
  __shared__ double s_sc, s_tot;
  int evals = 0;
  // the candidate volume at lambda, identical in every CTA
  auto eval_total = [&](double lam) {
    double* buf = partials + (evals & 1) * MFTO_RED_SLOTS;
    ++evals;
    if (threadIdx.x == 0) s_sc = 1.0 / sqrt(lam);
    __syncthreads();
    const double bs = block_sum(volume(s_sc), sh);
    if (threadIdx.x == 0) buf[blockIdx.x] = bs;
    grid_sync();
    if (threadIdx.x < 32) {
      double t = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) t += __ldcg(&buf[b]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (threadIdx.x == 0) s_tot = t;
    }
    __syncthreads();
    return s_tot;
  };
  // lambda_k = 1e9 halved k times (0 <= k <= k_end; exact for k <= 1083)
  auto lam_of = [](int k) {
    if (k <= 1083) return ldexp(1e9, -k);
    double x = ldexp(1e9, -1083);
    for (int i = 1083; i < k; ++i) x = 0.5 * x;
    return x;
  };
  const double target_v = target;
  double l1 = 0.0, l2 = 1e9, total = 0.0, last = -1.0;
  int step = 0, kstar = 0;
  // the phase with lower end 0: k* = the first k in [1, k_end) whose volume
  // exceeds the target (k_end: the first k with lambda_k = 0, where the
  // step-by-step bisection stops); klo: volume known <= target (0: none
  // evaluated), khi: volume known > target (k_end: none found yet)
  if (k_end > 1) {
    int klo = 0, khi = k_end;
    double vlo = 0.0, vhi = 0.0;
    auto probe = [&](int k) {
      const double v = eval_total(lam_of(k));
      if (v > target_v) { khi = k; vhi = v; } else { klo = k; vlo = v; }
    };
    if (k_hint >= 1 && k_hint < k_end) {
      probe(k_hint);
      if (khi == k_hint && k_hint - 1 >= 1) probe(k_hint - 1);
      else if (klo == k_hint && k_hint + 1 < k_end) probe(k_hint + 1);
    }
    if (klo != k_end - 1 && khi == k_end) probe(k_end - 1);   // is there a k* at all?
    while (khi - klo > 1 && !*(volatile int32_t*)&s->error) probe((klo + khi) / 2);
    kstar = khi;
    if (khi < k_end) {
      l1 = lam_of(khi);
      l2 = lam_of(khi - 1);
      last = l1;
      total = vhi;
      step = khi;
    } else {
      l2 = lam_of(k_end - 1);
      last = l2;
      total = vlo;
      step = k_end - 1;
    }
  }
  // Stops at the relative bracket width 1e-10, or when the midpoint no
  // longer lies strictly inside the bracket (lambda underflow when the target
  // is unreachable from above), and after at most 4096 steps in any case.
  while (l1 + l2 > 0.0 && (l2 - l1) / (l1 + l2) > 1e-10 && step < 4096) {
    const double lmid = 0.5 * (l1 + l2);
    if (!(l1 < lmid && lmid < l2)) break;   // uniform: every block holds the same l1, l2
    total = eval_total(lmid);
    last = lmid;
    if (total > target) l1 = lmid; else l2 = lmid;
    ++step;
    if (*(volatile int32_t*)&s->error) break;
  }
  // the candidate of the last midpoint (rho itself if no step ran), and
  // change = max |rho_new - rho|
  const double sc = last > 0.0 ? 1.0 / sqrt(last) : 0.0;
  double mx = 0.0;
  auto write = [&](int e, double a, double lo, double hi) {
    const double r = rho[e];
    const double rn = last > 0.0 ? fmax(lo, fmin(hi, a * sc)) : r;
    rho_new[e] = rn;
    mx = fmax(mx, fabs(rn - r));
  };
  if constexpr (G > 0) {
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (first + g * stride < n) write(first + g * stride, ra[g], rlo[g], rhi[g]);
  } else {
    for (int e = first; e < n; e += stride) write(e, a_s[e], lo_s[e], hi_s[e]);
  }
  double* buf = partials + 2 * MFTO_RED_SLOTS;
  const double bm = block_max(mx, sh);
  if (threadIdx.x == 0) buf[blockIdx.x] = bm;
  grid_sync();
  if (blockIdx.x == 0) {
    double m2 = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m2 = fmax(m2, __ldcg(&buf[b]));
    m2 = block_max(m2, sh);
    if (threadIdx.x == 0) {
      s->change = m2;
      s->volume = total / (double)n;
      s->lambda = 0.5 * (l1 + l2);
      s->oc_steps = step;
      s->oc_evals = evals;
      s->oc_kstar = kstar;
    }
  }
}

constexpr int kOcRegs = 8;   // elements per thread held in registers

}  // namespace

mfto_status compliance_launch(mfto_handle* h, const double* rho, const double* u, double* dc,
                              double* c_out, double* gray_out) {
  const Grid g = make_grid(h->mesh);
  const int nb = reduction_blocks(h->n_elem, MFTO_BLOCK);
  h->launches++;
  compliance_kernel<<<nb, MFTO_BLOCK, 0, h->stream>>>(rho, u, dc, h->mc64, g, h->p.E0,
                                                     h->p.Emin, h->p.penal, h->d_misc,
                                                     h->d_partials);
  MFTO_LAUNCH_CHECK(h);
  MFTO_CUDA(h, cudaMemcpyAsync(h->h_misc, h->d_misc, sizeof(MiscScalars), cudaMemcpyDeviceToHost,
                               h->stream));
  MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  if (c_out) *c_out = h->h_misc->sum[0];
  if (gray_out) *gray_out = h->h_misc->sum[1] / (double)h->n_elem;
  return MFTO_OK;
}

mfto_status oc_launch(mfto_handle* h, const double* rho, const double* dc, double* rho_new,
                      mfto_iter_stats* st) {
  // one CTA per SM (co-resident: the kernels use far fewer registers and no
  // dynamic shared memory); elements in registers when they fit
  int blocks = h->num_sms;
  const int need = (int)((h->n_elem + MFTO_BLOCK - 1) / MFTO_BLOCK);
  const bool regs = h->n_elem <= (int64_t)blocks * MFTO_BLOCK * kOcRegs;
  if (!regs) {
    // larger meshes re-read the scratch arrays every step: more CTAs in flight
    int per_sm = 0;
    MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oc_kernel<0>,
                                                               MFTO_BLOCK, 0));
    blocks = (per_sm < 4 ? (per_sm < 1 ? 1 : per_sm) : 4) * h->num_sms;
  }
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  MFTO_CUDA(h, cudaMemsetAsync(&h->d_misc->error, 0, sizeof(int32_t), h->stream));
  MFTO_CUDA(h, cudaMemsetAsync(&h->d_misc->bar_count, 0, sizeof(unsigned int), h->stream));
  int n = (int)h->n_elem;
  double volfrac = h->p.volfrac, move = h->p.move;
  MiscScalars* s = h->d_misc;
  double* partials = h->d_partials2;
  double* a_s = h->d_oc;
  double* lo_s = h->d_oc + h->n_elem;
  double* hi_s = h->d_oc + 2 * h->n_elem;
  // k_end: the first k at which 1e9 halved k times is 0 (the bisection's
  // midpoint with lower end 0 no longer lies inside its bracket)
  static const int k_end = [] {
    double x = 1e9;
    int k = 0;
    while (x > 0.0) {
      x = 0.5 * x;
      ++k;
    }
    return k;
  }();
  int k_hint = h->oc_hint;
  void* args[] = {(void*)&rho, (void*)&dc, (void*)&rho_new, &a_s, &lo_s, &hi_s, &n, &volfrac,
                  &move, &s, &partials, (void*)&k_end, &k_hint};
  h->launches++;
  const void* fn = regs ? (const void*)oc_kernel<kOcRegs> : (const void*)oc_kernel<0>;
  MFTO_CUDA(h, cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(MFTO_BLOCK), args, 0, h->stream));
  MFTO_CUDA(h, cudaMemcpyAsync(h->h_misc, h->d_misc, sizeof(MiscScalars), cudaMemcpyDeviceToHost,
                               h->stream));
  MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->h_misc->error)
    return mfto_fail(h, MFTO_CUDA_ERROR, "OC: a grid barrier wait gave up (bounded spin)");
  h->oc_hint = (h->h_misc->oc_kstar >= 1 && h->h_misc->oc_kstar < k_end) ? h->h_misc->oc_kstar : 0;
  if (st) {
    st->change = h->h_misc->change;
    st->volume = h->h_misc->volume;
    st->lambda = h->h_misc->lambda;
  }
  return MFTO_OK;
}

extern "C" mfto_status mfto_compliance_sens(mfto_handle* h, const double* rho_phys,
                                            const double* u, double* c_out, double* dc) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, rho_phys && u && c_out, "mfto_compliance_sens: null pointer");
  return compliance_launch(h, rho_phys, u, dc, c_out, nullptr);
}

extern "C" mfto_status mfto_oc_update(mfto_handle* h, const double* rho, const double* dc,
                                      double* rho_new, mfto_iter_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, rho && dc && rho_new, "mfto_oc_update: null pointer");
  MFTO_REQUIRE(h, rho != rho_new, "mfto_oc_update: rho_new must not alias rho");
  return oc_launch(h, rho, dc, rho_new, st);
}

extern "C" mfto_status mfto_simp_step(mfto_handle* h, double* rho, double* u, const double* f,
                                      double* rho_phys_out, mfto_iter_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, rho && u && f, "mfto_simp_step: null pointer");
  double* rho_phys = rho_phys_out ? rho_phys_out : h->d_rho_phys;
  // filter, then (three-field form) project: rho -> rho_bar -> rho_phys
  const bool proj = projection_active(h);
  mfto_status s = filter_launch(h, rho, proj ? h->d_rho_bar : rho_phys, 0);
  if (s != MFTO_OK) return s;
  if (proj) {
    s = project_launch(h, h->d_rho_bar, rho_phys);
    if (s != MFTO_OK) return s;
  }
  s = modulus_launch(h, MFTO_FORM_F64, rho_phys, h->d_E);
  if (s != MFTO_OK) return s;
  mfto_solve_stats ss;
  if (learned_active(h)) {
    mfto_learned_stats ls;
    s = learned_run(h, h->d_E, rho_phys, f, u, &ls);
    if (s != MFTO_OK) return s;
    ss.iterations = ls.inner_iterations + ls.fp64_iterations;
    ss.status = ls.status;
    ss.rel_residual = ls.rel_residual;
    ss.fnorm = ls.fnorm;
  } else if (gmg_active(h)) {
    s = gmg_solve(h, h->d_E, f, u, &ss);
    if (s != MFTO_OK) return s;
} else if (h->solver_form == MFTO_FORM_F64) {
    s = pcg_run(h, h->d_E, f, u, &ss);
    if (s != MFTO_OK) return s;
  } else {
    mfto_ir_stats is;
    s = ir_run(h, (mfto_form)h->solver_form, h->inner_tol, h->d_E, f, u, &is);
    if (s != MFTO_OK) return s;
    ss.iterations = is.inner_iterations;
    ss.status = is.status;
    ss.rel_residual = is.rel_residual;
    ss.fnorm = is.fnorm;
  }
  double c = 0.0, gray = 0.0;
  s = compliance_launch(h, rho_phys, u, h->d_dc_phys, &c, &gray);
  if (s != MFTO_OK) return s;
  if (proj) {   // dc/drho_bar = dc/drho_phys * drho_phys/drho_bar
    s = project_chain_launch(h, h->d_rho_bar, h->d_dc_phys);
    if (s != MFTO_OK) return s;
  }
  s = filter_launch(h, h->d_dc_phys, h->d_dc, 1);
  if (s != MFTO_OK) return s;
  mfto_iter_stats local;
  mfto_iter_stats* out = st ? st : &local;
  // the OC candidate goes to scratch (the bisection re-reads rho every step)
  s = oc_launch(h, rho, h->d_dc, h->d_dc_phys, out);
  if (s != MFTO_OK) return s;
  MFTO_CUDA(h, cudaMemcpyAsync(rho, h->d_dc_phys, sizeof(double) * h->n_elem,
                               cudaMemcpyDeviceToDevice, h->stream));
  out->compliance = c;
  out->grayness = gray;
  out->cg_iterations = ss.iterations;
  out->cg_status = ss.status;
  out->rel_residual = ss.rel_residual;
  return MFTO_OK;
}

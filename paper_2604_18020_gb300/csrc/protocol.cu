// Three-field SIMP (Sec. 3.1: density filter, smoothed Heaviside projection)
// and the 120-iteration continuation protocol of the benchmark runs (Sec.
// 4.1: four phases of penalty, projection sharpness, OC move limit and
// filter radius; restart from the selected design when the compliance
// exceeds 1.12 times the selected compliance; the selected iterate is the
// lowest compliance among iterates with p >= 3 and grayness < 0.25).
//
// Projection, with eta = 0.5 by default:
//   rho_phys = (tanh(beta eta) + tanh(beta (rho_bar - eta))) / D,
//   D = tanh(beta eta) + tanh(beta (1 - eta)),
// clipped to [0, 1] (rounding can put it a few ulps below 0 at rho_bar = 0);
// sensitivity chain dc/drho_bar = dc/drho_phys * beta (1 - tanh^2(beta
// (rho_bar - eta))) / D before the filter transpose.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace {

__global__ void __launch_bounds__(MFTO_BLOCK)
project_kernel(const double* __restrict__ rho_bar, double* __restrict__ rho_phys, int n,
               double beta, double eta, double th_eta, double den) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const double hv = (th_eta + tanh(beta * (rho_bar[e] - eta))) / den;
    rho_phys[e] = fmin(1.0, fmax(0.0, hv));
  }
}

__global__ void __launch_bounds__(MFTO_BLOCK)
project_chain_kernel(const double* __restrict__ rho_bar, double* __restrict__ dc, int n,
                     double beta, double eta, double den) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const double t = tanh(beta * (rho_bar[e] - eta));
    dc[e] = dc[e] * (beta * (1.0 - t * t) / den);
  }
}

// The paper's schedule: (first, last iteration, p, beta, move, r_min target
// or a negative value for "unchanged").
struct Phase {
  int first, last;
  double penal, beta, move, rmin_target;
};
const Phase kSchedule[4] = {
    {1, 15, 1.5, 1.0, 0.20, -1.0},
    {16, 40, 3.5, 4.0, 0.15, 1.35},
    {41, 65, 4.5, 16.0, 0.08, 1.25},
    {66, 120, 4.5, 32.0, 0.05, 1.20},
};

// (p, beta, move, r_min) of 1-based iteration it: values held within a phase,
// r_min ramped linearly from the previous phase's end value to the phase's
// target, which it reaches at the phase's last iteration.
void phase_params(int it, double rmin0, double* penal, double* beta, double* move,
                  double* rmin) {
  double r_start = rmin0;
  for (const Phase& ph : kSchedule) {
    const double r_end = ph.rmin_target < 0.0 ? r_start : ph.rmin_target;
    if (it <= ph.last) {
      *penal = ph.penal;
      *beta = ph.beta;
      *move = ph.move;
      if (ph.rmin_target < 0.0) {
        *rmin = r_start;
      } else {
        const int k = it - ph.first + 1, n = ph.last - ph.first + 1;
        *rmin = r_start + (r_end - r_start) * k / n;
      }
      return;
    }
    r_start = r_end;
  }
  const Phase& ph = kSchedule[3];
  *penal = ph.penal;
  *beta = ph.beta;
  *move = ph.move;
  *rmin = r_start;
}

}  // namespace

bool projection_active(const mfto_handle* h) { return h->proj_beta > 0.0; }

static void projection_constants(const mfto_handle* h, double* th_eta, double* den) {
  *th_eta = tanh(h->proj_beta * h->proj_eta);
  *den = *th_eta + tanh(h->proj_beta * (1.0 - h->proj_eta));
}

mfto_status project_launch(mfto_handle* h, const double* rho_bar, double* rho_phys) {
  double th_eta, den;
  projection_constants(h, &th_eta, &den);
  h->launches++;
  project_kernel<<<reduction_blocks(h->n_elem, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(
      rho_bar, rho_phys, (int)h->n_elem, h->proj_beta, h->proj_eta, th_eta, den);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

mfto_status project_chain_launch(mfto_handle* h, const double* rho_bar, double* dc) {
  double th_eta, den;
  projection_constants(h, &th_eta, &den);
  h->launches++;
  project_chain_kernel<<<reduction_blocks(h->n_elem, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(
      rho_bar, dc, (int)h->n_elem, h->proj_beta, h->proj_eta, den);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

extern "C" mfto_status mfto_set_projection(mfto_handle* h, double beta, double eta) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, beta >= 0.0 && isfinite(beta), "mfto_set_projection: beta must be >= 0");
  MFTO_REQUIRE(h, eta > 0.0 && eta < 1.0, "mfto_set_projection: eta must lie in (0, 1)");
  h->proj_beta = beta;
  h->proj_eta = eta;
  return MFTO_OK;
}

extern "C" mfto_status mfto_project(mfto_handle* h, const double* rho_bar, double* rho_phys,
                                    double* dc) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, rho_bar && (rho_phys || dc), "mfto_project: null pointer");
  MFTO_REQUIRE(h, projection_active(h), "mfto_project: projection is off (beta = 0)");
  mfto_status s = MFTO_OK;
  if (rho_phys) s = project_launch(h, rho_bar, rho_phys);
  if (s == MFTO_OK && dc) s = project_chain_launch(h, rho_bar, dc);
  return s;
}

extern "C" void mfto_default_protocol_params(mfto_protocol_params* p) {
  if (!p) return;
  p->n_iter = 120;
  p->rmin0 = 1.5;
  p->eta = 0.5;
  p->restart_factor = 1.12;
  p->select_min_penal = 3.0;
  p->select_max_gray = 0.25;
  p->cold_start = 0;
}

extern "C" mfto_status mfto_simp_protocol(mfto_handle* h, double* rho, double* u, const double* f,
                                          double* rho_selected, const mfto_protocol_params* prm,
                                          double* compliance, double* grayness,
                                          int32_t* restarted, mfto_protocol_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, rho && u && f && rho_selected && prm && st, "mfto_simp_protocol: null pointer");
  MFTO_REQUIRE(h, prm->n_iter >= 1 && prm->rmin0 > 0.0 && prm->restart_factor >= 1.0,
               "mfto_simp_protocol: need n_iter >= 1, rmin0 > 0, restart_factor >= 1");
  MFTO_REQUIRE(h, prm->eta > 0.0 && prm->eta < 1.0, "mfto_simp_protocol: eta must lie in (0, 1)");
  memset(st, 0, sizeof(*st));
  const mfto_params saved = h->p;
  const double saved_beta = h->proj_beta, saved_eta = h->proj_eta;
  const size_t bytes = sizeof(double) * h->n_elem;
  bool have_sel = false;
  double sel_c = 0.0;
  mfto_status s = MFTO_OK;
  for (int it = 1; it <= prm->n_iter && s == MFTO_OK; ++it) {
    double penal, beta, move, rmin;
    phase_params(it, prm->rmin0, &penal, &beta, &move, &rmin);
    h->p.penal = penal;
    h->p.move = move;
    if (rmin != h->p.rmin) {
      h->p.rmin = rmin;
      s = filter_setup(h);   // stencil and row sums of the new radius
      if (s != MFTO_OK) break;
    }
    h->proj_beta = beta;
    h->proj_eta = prm->eta;
    // the design entering this iteration (the one its compliance belongs to)
    s = [&]() -> mfto_status {
      MFTO_CUDA(h, cudaMemcpyAsync(h->d_rho_in, rho, bytes, cudaMemcpyDeviceToDevice, h->stream));
      return MFTO_OK;
    }();
    if (s != MFTO_OK) break;
    if (prm->cold_start) {
      s = [&]() -> mfto_status {
        MFTO_CUDA(h, cudaMemsetAsync(u, 0, sizeof(double) * h->n_dof, h->stream));
        return MFTO_OK;
      }();
      if (s != MFTO_OK) break;
    }
    mfto_iter_stats is;
    s = mfto_simp_step(h, rho, u, f, nullptr, &is);
    if (s != MFTO_OK) break;
    st->cg_iterations += is.cg_iterations;
    if (compliance) compliance[it - 1] = is.compliance;
    if (grayness) grayness[it - 1] = is.grayness;
    const bool restart = have_sel && is.compliance > prm->restart_factor * sel_c;
    const bool eligible = penal >= prm->select_min_penal && is.grayness < prm->select_max_gray;
    const bool better = eligible && (!have_sel || is.compliance < sel_c);
    if (restarted) restarted[it - 1] = restart ? 1 : 0;
    s = [&]() -> mfto_status {
      if (better) {
        MFTO_CUDA(h, cudaMemcpyAsync(rho_selected, h->d_rho_in, bytes, cudaMemcpyDeviceToDevice,
                                     h->stream));
      }
      if (restart) {
        MFTO_CUDA(h, cudaMemcpyAsync(rho, rho_selected, bytes, cudaMemcpyDeviceToDevice,
                                     h->stream));
      }
      return MFTO_OK;
    }();
    if (better) {
      have_sel = true;
      sel_c = is.compliance;
      st->selected_iteration = it;
      st->selected_compliance = is.compliance;
    }
    if (restart) st->restarts++;
    st->iterations = it;
  }
  // the handle's parameters as the caller left them
  const bool refilter = h->p.rmin != saved.rmin;
  h->p = saved;
  h->proj_beta = saved_beta;
  h->proj_eta = saved_eta;
  if (refilter) {
    const mfto_status s2 = filter_setup(h);
    if (s == MFTO_OK) s = s2;
  }
  if (s == MFTO_OK) MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  return s;
}

// The learned solve: FP64 iterative refinement (the residual-correction loop
// of Sec. 3.5, as in ir.cu) whose inner solve is a flexible PCG in FP32 with
// a network correction.  The network (nn.cu) maps (node density, load
// direction) on the padded node grid to a displacement direction.
//
// Inner flexible PCG (K e = r, e0 = 0), FP32 vectors, FP64 dot products:
//   z_k = D^-1 r_k, except at correction iterations where
//         z_k = +-N(rho, r_k) (the sign makes z_k.r_k > 0; the scale of z_k
//         does not matter): k = 0 of the first outer step (the initial
//         guess) and, when `every` > 0, k = 0 of every later inner solve and
//         every `every`-th iteration;
//   beta_k = z_k.(r_k - r_{k-1}) / z_{k-1}.r_{k-1}   (Polak-Ribiere)
//   p_k = z_k + beta_k p_{k-1};  q = K p_k;  alpha = z_k.r_k / p_k.q
//   (= r_k.p_k / p_k.q, the exact line search, since r_k.p_{k-1} = 0).
// With a fixed preconditioner the Polak-Ribiere beta equals the usual one;
// it is what keeps the recurrence consistent when z changes form.  The first
// correction of the first outer step (u = 0, r = f) is the network's initial
// guess, scaled optimally in the energy norm by the line search.
//
// Fallback: when two outer steps in a row reduce the FP64 residual by less
// than 10 % the network is switched off (plain Jacobi inner PCG, the mixed
// form of ir.cu); if that stalls too, plain FP64 Jacobi-PCG finishes the
// solve from the current iterate.  A solve is accepted (status OK) only when
// the FP64 residual ||f - Ku|| / ||f||, recomputed from u, is <= rtol.
#include <math.h>
#include <string.h>

#include "common.cuh"

struct mfto_nn;
mfto_status nn_infer(mfto_nn* n, cudaStream_t st, int D, int H, int W, const float* x, float* y);
int nn_levels(const mfto_nn* n);
long long nn_max_voxels(const mfto_nn* n);
const char* nn_message(const mfto_nn* n);
mfto_status nn_train_forward(mfto_nn* n, cudaStream_t st, int D, int H, int W, const float* x,
                             float** out);
mfto_status nn_train_backward(mfto_nn* n, cudaStream_t st, int D, int H, int W, float lr);

// decision of one correction (device)
struct FpcgCtl {
  double cr, cq, cc, rr;
  int32_t use;
  float sgn;
  unsigned int ticket;
};

struct LearnedWs {
  mfto_nn* nn = nullptr;
  int every = 0;
  int levels = 0;
  int D = 0, H = 0, W = 0;
  float* x = nullptr;            // network input [4][D][H][W]
  float* y = nullptr;            // network output [3][D][H][W]
  float* c = nullptr;            // network direction on the DOFs [n_dof]
  double* uk = nullptr;          // FP64 scratch of the sample builder [n_dof]
  unsigned int* amax = nullptr;  // bit pattern of a max |.| (non-negative float)
  FpcgCtl* ctl = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

struct VoxGrid {
  int D, H, W;
};

int round_up(int a, int m) { return (a + m - 1) / m * m; }

void grid_dims(const mfto_mesh& m, int levels, int* D, int* H, int* W) {
  const int mult = 1 << (levels - 1);
  *D = round_up(m.nelz + 1, mult);
  *H = round_up(m.nely + 1, mult);
  *W = round_up(m.nelx + 1, mult);
}

// channel 0: mean density of the elements around each node (0 on padding)
__global__ void __launch_bounds__(MFTO_BLOCK)
density_channel(const double* __restrict__ rho, float* __restrict__ x0, Grid g, VoxGrid vg) {
  const int V = vg.D * vg.H * vg.W;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int i = v % vg.W, j = (v / vg.W) % vg.H, k = v / (vg.W * vg.H);
  float out = 0.f;
  if (i < g.nx && j < g.ny && k < g.nz) {
    double s = 0.0;
    int cnt = 0;
    for (int ce = 0; ce < 8; ++ce) {
      const int ei = i - 1 + (ce & 1), ej = j - 1 + ((ce >> 1) & 1), ek = k - 1 + (ce >> 2);
      if (ei < 0 || ej < 0 || ek < 0 || ei >= g.nelx || ej >= g.nely || ek >= g.nelz) continue;
      s += rho[ei + g.nelx * (ej + g.nely * ek)];
      ++cnt;
    }
    out = (float)(s / cnt);
  }
  x0[v] = out;
}

// *slot = max(*slot, max |a_i|) as the bit pattern of a non-negative float
// (ordered like the unsigned integers, so the result is order-independent)
template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
absmax_kernel(const T* __restrict__ a, int n, unsigned int* slot) {
  __shared__ double sh[64];
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)a[i]));
  m = block_max(m, sh);
  if (threadIdx.x == 0) atomicMax(slot, __float_as_uint((float)m));
}

__device__ __forceinline__ float inv_of(const unsigned int* amax) {
  const float m = __uint_as_float(*amax);
  return m > 0.f ? 1.f / m : 0.f;
}

// channels 1..3 (or a target): a[3 n + c] / max |a| on the real nodes, 0 on
// padding; the optional mask is 1 on the free DOFs of the real nodes.
template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
dof_channels(const T* __restrict__ a, float* __restrict__ out, float* __restrict__ mask,
             const uint8_t* __restrict__ fixed, const unsigned int* __restrict__ amax, Grid g,
             VoxGrid vg) {
  const int V = vg.D * vg.H * vg.W;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int i = v % vg.W, j = (v / vg.W) % vg.H, k = v / (vg.W * vg.H);
  const bool real = i < g.nx && j < g.ny && k < g.nz;
  const int node = real ? i + g.nx * (j + g.ny * k) : 0;
  const float inv = inv_of(amax);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    out[(size_t)c * V + v] = real ? (float)a[3 * node + c] * inv : 0.f;
    if (mask) mask[(size_t)c * V + v] = (real && !((fixed[node] >> c) & 1)) ? 1.f : 0.f;
  }
}

// network output [3][D][H][W] -> DOF vector, zero on the fixed DOFs
template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
to_dofs_kernel(const float* __restrict__ y, T* __restrict__ c, const uint8_t* __restrict__ fixed,
               Grid g, VoxGrid vg, int n_node) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= n_node) return;
  const int i = node % g.nx, j = (node / g.nx) % g.ny, k = node / (g.nx * g.ny);
  const size_t V = (size_t)vg.D * vg.H * vg.W;
  const size_t v = (size_t)i + (size_t)vg.W * (j + (size_t)vg.H * k);
  const uint8_t fm = fixed[node];
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) c[3 * node + cc] = ((fm >> cc) & 1) ? T(0) : (T)y[cc * V + v];
}

// r = f - Ku;  e = u* - u_k (in place in uk)
__global__ void __launch_bounds__(MFTO_BLOCK)
sample_pair(const double* __restrict__ f, const double* __restrict__ Ku,
            const double* __restrict__ ustar, double* __restrict__ r, double* __restrict__ uk, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    r[i] = f[i] - Ku[i];
    uk[i] = ustar[i] - uk[i];
  }
}

// Flexible-PCG update: e += alpha p; r -= alpha q; z = r / d; the
// Polak-Ribiere beta from z.r_new and z.r_old; convergence test.
__global__ void __launch_bounds__(MFTO_BLOCK)
fpcg_update(float* __restrict__ u, const float* __restrict__ p, const float* __restrict__ q,
            float* __restrict__ r, float* __restrict__ z, const float* __restrict__ dinv,
            int n_node, PcgScalars* s, double* partials) {
  if (*(volatile int32_t*)&s->done) return;
  __shared__ double sh[64];
  const float alpha = (float)s->alpha;
  DotAcc<float> d0, d1, d2;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < n_node; nd += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int i = 3 * nd + c;
      u[i] += alpha * p[i];
      const float r_old = r[i];
      const float ri = r_old - alpha * q[i];
      const float zi = ri * dinv[i];
      r[i] = ri;
      z[i] = zi;
      d0.add_prod(ri, zi);
      d1.add_prod(ri, ri);
      d2.add_prod(r_old, zi);
    }
  }
  const double acc[3] = {d0.finish(), d1.finish(), d2.finish()};
  double tot[3];
  if (last_block_reduce<3, true>(acc, partials, &s->ticket_c, tot, sh) && threadIdx.x == 0) {
    s->it += 1;
    s->rr = tot[1];
    s->beta = (tot[0] - tot[2]) / s->rz;
    s->rz = tot[0];
    if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
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

// Dots of a network direction c with the current residual r and the last
// q = K p; the last block decides whether and with which sign c replaces z,
// and sets beta and r.z to match (r_old = r + alpha q).
__global__ void __launch_bounds__(MFTO_BLOCK)
fpcg_corr_dots(const float* __restrict__ c, const float* __restrict__ r,
               const float* __restrict__ q, int n, PcgScalars* s, FpcgCtl* ctl,
               double* partials) {
  if (*(volatile int32_t*)&s->done) return;
  __shared__ double sh[64];
  DotAcc<float> d0, d1, d2, d3;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float ci = c[i];
    d0.add_prod(ci, r[i]);
    d1.add_prod(ci, q[i]);
    d2.add_prod(ci, ci);
    d3.add_prod(r[i], r[i]);
  }
  const double acc[4] = {d0.finish(), d1.finish(), d2.finish(), d3.finish()};
  double tot[4];
  if (last_block_reduce<4, true>(acc, partials, &ctl->ticket, tot, sh) && threadIdx.x == 0) {
    ctl->cr = tot[0];
    ctl->cq = tot[1];
    ctl->cc = tot[2];
    ctl->rr = tot[3];
    const bool use = isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2]) &&
                     fabs(tot[0]) > 1e-6 * sqrt(tot[2] * tot[3]) && s->rz > 0.0;
    ctl->use = use ? 1 : 0;
    if (use) {
      const double sg = tot[0] >= 0.0 ? 1.0 : -1.0;
      ctl->sgn = (float)sg;
      // beta = sgn c.(r - r_old) / rz_prev with r - r_old = -alpha q
      s->beta = -sg * s->alpha * tot[1] / s->rz;
      s->rz = sg * tot[0];
    }
  }
}

__global__ void __launch_bounds__(MFTO_BLOCK)
fpcg_apply(const float* __restrict__ c, float* __restrict__ z, int n, const PcgScalars* s,
           const FpcgCtl* ctl) {
  if (*(volatile const int32_t*)&s->done || !ctl->use) return;
  const float sg = ctl->sgn;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    z[i] = sg * c[i];
}

__global__ void __launch_bounds__(MFTO_BLOCK)
to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// r = f - Ku (FP64) into r32; r.r and f.f (sum[0], sum[1])
__global__ void __launch_bounds__(MFTO_BLOCK)
residual_kernel(const double* __restrict__ f, const double* __restrict__ Ku,
                float* __restrict__ r32, int n, MiscScalars* s, double* partials) {
  __shared__ double sh[64];
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double ri = f[i] - Ku[i];
    if (r32) r32[i] = (float)ri;
    acc[0] += ri * ri;
    acc[1] += f[i] * f[i];
  }
  double tot[2];
  if (last_block_reduce<2>(acc, partials, &s->ticket, tot, sh) && threadIdx.x == 0) {
    s->sum[0] = tot[0];
    s->sum[1] = tot[1];
  }
}

__global__ void __launch_bounds__(MFTO_BLOCK)
accumulate_kernel(double* __restrict__ u, const float* __restrict__ e, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    u[i] += (double)e[i];
}

// a = f.c, b = c.Kc (sum[0], sum[1])
__global__ void __launch_bounds__(MFTO_BLOCK)
energy_dots(const double* __restrict__ f, const double* __restrict__ c,
            const double* __restrict__ Kc, int n, MiscScalars* s, double* partials) {
  __shared__ double sh[64];
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    acc[0] += f[i] * c[i];
    acc[1] += c[i] * Kc[i];
  }
  double tot[2];
  if (last_block_reduce<2>(acc, partials, &s->ticket, tot, sh) && threadIdx.x == 0) {
    s->sum[0] = tot[0];
    s->sum[1] = tot[1];
  }
}

// d loss / d output on the grid for loss = 1 - a^2 / (b S):
//   d loss / d c = (2 a^2 / b^2 Kc - 2 a / b f) / S, zero on fixed DOFs and
// padding; the loss goes to sum[2] (1 and a zero gradient when b <= 0).
__global__ void __launch_bounds__(MFTO_BLOCK)
energy_grad(const double* __restrict__ f, const double* __restrict__ Kc,
            const uint8_t* __restrict__ fixed, MiscScalars* s, double S, float* __restrict__ g,
            Grid gr, VoxGrid vg) {
  const int V = vg.D * vg.H * vg.W;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const double a = s->sum[0], b = s->sum[1];
  const bool ok = b > 0.0 && S > 0.0;
  if (v == 0) s->sum[2] = ok ? 1.0 - a * a / (b * S) : 1.0;
  const int i = v % vg.W, j = (v / vg.W) % vg.H, k = v / (vg.W * vg.H);
  const bool real = ok && i < gr.nx && j < gr.ny && k < gr.nz;
  const int node = real ? i + gr.nx * (j + gr.ny * k) : 0;
  const double ca = ok ? 2.0 * a * a / (b * b * S) : 0.0;
  const double cf = ok ? 2.0 * a / (b * S) : 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float out = 0.f;
    if (real && !((fixed[node] >> c) & 1)) out = (float)(ca * Kc[3 * node + c] - cf * f[3 * node + c]);
    g[(size_t)c * V + v] = out;
  }
}

unsigned nblk(int64_t n) { return (unsigned)((n + MFTO_BLOCK - 1) / MFTO_BLOCK); }

VoxGrid vox(const LearnedWs* w) { return VoxGrid{w->D, w->H, w->W}; }

mfto_status ensure_ws(mfto_handle* h, int levels) {
  LearnedWs*& w = h->learned;
  if (!w) w = new LearnedWs();
  if (w->x && w->levels == levels) return MFTO_OK;
  if (w->x) { cudaFree(w->x); cudaFree(w->y); w->x = w->y = nullptr; }
  w->levels = levels;
  grid_dims(h->mesh, levels, &w->D, &w->H, &w->W);
  const size_t V = (size_t)w->D * w->H * w->W;
  MFTO_CUDA(h, cudaMalloc(&w->x, sizeof(float) * 4 * V));
  MFTO_CUDA(h, cudaMalloc(&w->y, sizeof(float) * 3 * V));
  if (!w->c) MFTO_CUDA(h, cudaMalloc(&w->c, sizeof(float) * h->n_dof));
  if (!w->uk) MFTO_CUDA(h, cudaMalloc(&w->uk, sizeof(double) * h->n_dof));
  if (!w->amax) MFTO_CUDA(h, cudaMalloc(&w->amax, sizeof(unsigned int) * 2));
  if (!w->ctl) {
    MFTO_CUDA(h, cudaMalloc(&w->ctl, sizeof(FpcgCtl)));
    MFTO_CUDA(h, cudaMemsetAsync(w->ctl, 0, sizeof(FpcgCtl), h->stream));
  }
  if (!w->ev0) {
    MFTO_CUDA(h, cudaEventCreate(&w->ev0));
    MFTO_CUDA(h, cudaEventCreate(&w->ev1));
  }
  return MFTO_OK;
}

// features: channel 0 from rho_phys (when given), channels 1..3 from the load
template <typename T>
mfto_status build_features(mfto_handle* h, const double* rho_phys, const T* load) {
  LearnedWs* w = h->learned;
  const Grid g = make_grid(h->mesh);
  const VoxGrid vg = vox(w);
  const size_t V = (size_t)w->D * w->H * w->W;
  if (rho_phys) {
    h->launches++;
    density_channel<<<nblk(V), MFTO_BLOCK, 0, h->stream>>>(rho_phys, w->x, g, vg);
  }
  MFTO_CUDA(h, cudaMemsetAsync(w->amax, 0, sizeof(unsigned int), h->stream));
  h->launches += 2;
  absmax_kernel<T><<<reduction_blocks(h->n_dof, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(
      load, (int)h->n_dof, w->amax);
  dof_channels<T><<<nblk(V), MFTO_BLOCK, 0, h->stream>>>(load, w->x + V, nullptr, h->d_fixed,
                                                         w->amax, g, vg);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

mfto_status build_target(mfto_handle* h, const double* u, float* y, float* mask) {
  LearnedWs* w = h->learned;
  const Grid g = make_grid(h->mesh);
  const size_t V = (size_t)w->D * w->H * w->W;
  MFTO_CUDA(h, cudaMemsetAsync(w->amax + 1, 0, sizeof(unsigned int), h->stream));
  h->launches += 2;
  absmax_kernel<double><<<reduction_blocks(h->n_dof, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(
      u, (int)h->n_dof, w->amax + 1);
  dof_channels<double><<<nblk(V), MFTO_BLOCK, 0, h->stream>>>(u, y, mask, h->d_fixed, w->amax + 1,
                                                              g, vox(w));
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

mfto_status run_network(mfto_handle* h) {
  LearnedWs* w = h->learned;
  MFTO_CUDA(h, cudaEventRecord(w->ev0, h->stream));
  mfto_status s = nn_infer(w->nn, h->stream, w->D, w->H, w->W, w->x, w->y);
  if (s != MFTO_OK) return mfto_fail(h, s, "network: %s", nn_message(w->nn));
  MFTO_CUDA(h, cudaEventRecord(w->ev1, h->stream));
  h->launches++;
  to_dofs_kernel<float><<<nblk(h->n_node), MFTO_BLOCK, 0, h->stream>>>(
      w->y, w->c, h->d_fixed, make_grid(h->mesh), vox(w), (int)h->n_node);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

// inner flexible PCG from e = 0 on the right-hand side already in v.r
mfto_status fpcg_inner(mfto_handle* h, const PcgVecs<float>& v, double tol, int maxit,
                       bool first_correction, mfto_learned_stats* st) {
  LearnedWs* w = h->learned;
  const int n = (int)h->n_dof;
  int nb_node = (int)((h->n_node + MFTO_BLOCK - 1) / MFTO_BLOCK);
  if (nb_node > MFTO_RED_SLOTS) nb_node = MFTO_RED_SLOTS;
  const int nb_dof = reduction_blocks(h->n_dof, MFTO_BLOCK);
  MFTO_CUDA(h, cudaMemsetAsync(v.u, 0, sizeof(float) * h->n_dof, h->stream));
  // q enters the first correction's dots (multiplied by alpha = 0): keep it finite
  MFTO_CUDA(h, cudaMemsetAsync(v.q, 0, sizeof(float) * h->n_dof, h->stream));
  mfto_status s = pcg_start<float>(h, v, v.r, nullptr, tol, maxit);
  if (s != MFTO_OK) return s;
  const int chunk_cap = h->p.check_every;
  int parity = 0;
  bool timed = false;   // a network call awaits its event pair
  for (;;) {
    MFTO_CUDA(h, cudaMemcpyAsync(h->h_pcg32, v.s, sizeof(PcgScalars), cudaMemcpyDeviceToHost,
                                 h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->h_pcg32->tc_error)
      return mfto_fail(h, MFTO_CUDA_ERROR, "tensor-core completion wait timed out");
    if (timed) {
      float ms = 0.f;
      MFTO_CUDA(h, cudaEventElapsedTime(&ms, w->ev0, w->ev1));
      st->nn_ms += ms;
      timed = false;
    }
    if (h->h_pcg32->done) break;
    const int k = h->h_pcg32->it;
    const bool correct =
        w->nn && (k == 0 ? first_correction : (w->every > 0 && k % w->every == 0));
    if (correct) {
      s = build_features<float>(h, nullptr, v.r);
      if (s == MFTO_OK) s = run_network(h);
      if (s != MFTO_OK) return s;
      h->launches += 2;
      fpcg_corr_dots<<<nb_dof, MFTO_BLOCK, 0, h->stream>>>(w->c, v.r, v.q, n, v.s, w->ctl,
                                                           v.part_a);
      fpcg_apply<<<nb_dof, MFTO_BLOCK, 0, h->stream>>>(w->c, v.z, n, v.s, w->ctl);
      MFTO_LAUNCH_CHECK(h);
      st->nn_calls++;
      timed = true;
    }
    // iterations up to the next correction (or check point)
    int run = chunk_cap;
    if (w->nn && w->every > 0) {
      const int next = (k / w->every + 1) * w->every;
      if (next - k < run) run = next - k;
    }
    for (int it = 0; it < run; ++it) {
      float* p_old = parity ? v.p1 : v.p0;
      float* p_new = parity ? v.p0 : v.p1;
      parity ^= 1;
      if (tc_form(v.form))
        s = pcg_kv_tc_launch(h, v.form, v.E, v.z, p_old, p_new, v.q, v.s, v.part_a, h->stream);
      else
        s = pcg_kv_tile_launch<float>(h, v.E, v.z, p_old, p_new, v.q, v.s, v.part_a, h->stream);
      if (s != MFTO_OK) return s;
      h->launches++;
      fpcg_update<<<nb_node, MFTO_BLOCK, 0, h->stream>>>(v.u, p_new, v.q, v.r, v.z, v.dinv,
                                                         (int)h->n_node, v.s, v.part_b);
      MFTO_LAUNCH_CHECK(h);
    }
  }
  return MFTO_OK;
}

}  // namespace

bool learned_active(const mfto_handle* h) { return h->learned && h->learned->nn; }

void learned_release(mfto_handle* h) {
  LearnedWs* w = h->learned;
  if (!w) return;
  void* ptrs[] = {w->x, w->y, w->c, w->uk, w->amax, w->ctl};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (w->ev0) cudaEventDestroy(w->ev0);
  if (w->ev1) cudaEventDestroy(w->ev1);
  delete w;
  h->learned = nullptr;
}

mfto_status learned_run(mfto_handle* h, const double* E, const double* rho_phys, const double* f,
                        double* u, mfto_learned_stats* st) {
  LearnedWs* w = h->learned;
  if (!w || !w->nn) return mfto_fail(h, MFTO_INVALID_ARG, "learned solve: no network attached");
  const int n = (int)h->n_dof;
  const int nb_dof = reduction_blocks(h->n_dof, MFTO_BLOCK);
  const int nb_el = reduction_blocks(h->n_elem, MFTO_BLOCK);
  mfto_learned_stats local;
  mfto_learned_stats* out = st ? st : &local;
  memset(out, 0, sizeof(*out));
  mfto_nn* net = w->nn;
  h->launches++;
  to_f32_kernel<<<nb_el, MFTO_BLOCK, 0, h->stream>>>(E, h->d_E32, (int)h->n_elem);
  MFTO_LAUNCH_CHECK(h);
  mfto_status s = diag_launch(h, MFTO_FORM_F32, h->d_E32, h->d_dinv32, true);
  if (s != MFTO_OK) return s;
  // density channel once per solve
  {
    const size_t V = (size_t)w->D * w->H * w->W;
    h->launches++;
    density_channel<<<nblk(V), MFTO_BLOCK, 0, h->stream>>>(rho_phys, w->x, make_grid(h->mesh),
                                                           vox(w));
    MFTO_LAUNCH_CHECK(h);
  }
  const PcgVecs<float> v{h->d_E32, h->d_e32, h->d_r32, h->d_z32, h->d_p0_32, h->d_p1_32,
                         h->d_q32, h->d_dinv32, h->d_pcg32, h->d_partials, h->d_partials2,
                         (int)MFTO_FORM_F32};
  double prev = 0.0;
  int stalls = 0;
  int mode = 0;  // 0: network inner FPCG; 1: plain Jacobi inner PCG; 2: FP64 PCG
  out->status = MFTO_NOT_CONVERGED;
  for (int outer = 0;; ++outer) {
    s = kv_launch(h, MFTO_FORM_F64, E, u, h->d_q);
    if (s != MFTO_OK) return s;
    h->launches++;
    residual_kernel<<<nb_dof, MFTO_BLOCK, 0, h->stream>>>(f, h->d_q, h->d_r32, n, h->d_misc,
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
    if (mode == 2) { out->status = MFTO_NOT_CONVERGED; break; }   // FP64 PCG ran: its outcome is final
    if (outer > 0) {
      stalls = rel > 0.9 * prev ? stalls + 1 : 0;
      if (stalls >= 2) {
        ++mode;
        stalls = 0;
        out->fallback = mode;
      }
    }
    if (outer >= h->max_outer && mode < 2) { mode = 2; out->fallback = 2; }
    prev = rel;
    if (mode == 2) {
      mfto_solve_stats ps;
      s = pcg_run(h, E, f, u, &ps);
      if (s != MFTO_OK) return s;
      out->fp64_iterations += ps.iterations;
      continue;   // the next pass recomputes the true residual and decides
    }
    // the network's first direction: the initial guess (first outer step)
    // and, with every > 0, the start of each later inner solve
    w->nn = mode == 0 ? net : nullptr;
    s = fpcg_inner(h, v, h->inner_tol, h->inner_maxit, outer == 0 || w->every > 0, out);
    w->nn = net;
    if (s != MFTO_OK) { w->nn = net; return s; }
    out->inner_iterations += h->h_pcg32->it;
    if (h->h_pcg32->status == MFTO_BREAKDOWN) {
      // a breakdown of the flexible recurrence: retry this step without the network
      if (mode == 0) { mode = 1; out->fallback = 1; continue; }
      out->status = MFTO_BREAKDOWN;
      break;
    }
    h->launches++;
    accumulate_kernel<<<nb_dof, MFTO_BLOCK, 0, h->stream>>>(u, h->d_e32, n);
    MFTO_LAUNCH_CHECK(h);
    out->outer_iterations++;
  }
  w->nn = net;
  return MFTO_OK;
}

// ------------------------------------------------------------------ C ABI

extern "C" mfto_status mfto_nn_grid(const mfto_mesh* m, int32_t levels, int32_t dims[3]) {
  if (!m || !dims || levels < 2 || levels > 6 || m->nelx < 1 || m->nely < 1 || m->nelz < 1)
    return MFTO_INVALID_ARG;
  int D, H, W;
  grid_dims(*m, levels, &D, &H, &W);
  dims[0] = D;
  dims[1] = H;
  dims[2] = W;
  return MFTO_OK;
}

extern "C" mfto_status mfto_nn_features(mfto_handle* h, int32_t levels, const double* rho_phys,
                                        const double* load, float* x_out) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, rho_phys && load && x_out, "mfto_nn_features: null pointer");
  MFTO_REQUIRE(h, levels >= 2 && levels <= 6, "mfto_nn_features: levels in [2, 6]");
  mfto_status s = ensure_ws(h, levels);
  if (s != MFTO_OK) return s;
  s = build_features<double>(h, rho_phys, load);
  if (s != MFTO_OK) return s;
  const size_t V = (size_t)h->learned->D * h->learned->H * h->learned->W;
  MFTO_CUDA(h, cudaMemcpyAsync(x_out, h->learned->x, sizeof(float) * 4 * V,
                               cudaMemcpyDeviceToDevice, h->stream));
  return MFTO_OK;
}

extern "C" mfto_status mfto_nn_target(mfto_handle* h, int32_t levels, const double* u,
                                      float* y_out, float* mask_out) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, u && y_out && mask_out, "mfto_nn_target: null pointer");
  MFTO_REQUIRE(h, levels >= 2 && levels <= 6, "mfto_nn_target: levels in [2, 6]");
  mfto_status s = ensure_ws(h, levels);
  if (s != MFTO_OK) return s;
  return build_target(h, u, y_out, mask_out);
}

extern "C" mfto_status mfto_nn_to_dofs(mfto_handle* h, int32_t levels, const float* y,
                                       double* c_out) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, y && c_out, "mfto_nn_to_dofs: null pointer");
  MFTO_REQUIRE(h, levels >= 2 && levels <= 6, "mfto_nn_to_dofs: levels in [2, 6]");
  mfto_status s = ensure_ws(h, levels);
  if (s != MFTO_OK) return s;
  h->launches++;
  to_dofs_kernel<double><<<nblk(h->n_node), MFTO_BLOCK, 0, h->stream>>>(
      y, c_out, h->d_fixed, make_grid(h->mesh), vox(h->learned), (int)h->n_node);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

extern "C" mfto_status mfto_nn_sample(mfto_handle* h, int32_t levels, const double* E,
                                      const double* rho_phys, const double* f,
                                      const double* u_star, int32_t k_iters, float* x_out,
                                      float* y_out, float* mask_out) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, E && rho_phys && f && u_star && x_out && y_out && mask_out,
               "mfto_nn_sample: null pointer");
  MFTO_REQUIRE(h, levels >= 2 && levels <= 6, "mfto_nn_sample: levels in [2, 6]");
  MFTO_REQUIRE(h, k_iters >= 0, "mfto_nn_sample: k_iters >= 0");
  mfto_status s = ensure_ws(h, levels);
  if (s != MFTO_OK) return s;
  LearnedWs* w = h->learned;
  const size_t V = (size_t)w->D * w->H * w->W;
  if (k_iters == 0) {
    s = build_features<double>(h, rho_phys, f);
    if (s == MFTO_OK) s = build_target(h, u_star, y_out, mask_out);
  } else {
    // k Jacobi-PCG iterations from zero: the residual and the error of that
    // iterate form one (load, displacement) pair
    MFTO_CUDA(h, cudaMemsetAsync(w->uk, 0, sizeof(double) * h->n_dof, h->stream));
    const int keep_maxit = h->p.maxit;
    const double keep_rtol = h->p.rtol;
    h->p.maxit = k_iters;
    h->p.rtol = 0.0;
    mfto_solve_stats ps;
    s = pcg_run(h, E, f, w->uk, &ps);
    h->p.maxit = keep_maxit;
    h->p.rtol = keep_rtol;
    if (s != MFTO_OK) return s;
    s = kv_launch(h, MFTO_FORM_F64, E, w->uk, h->d_q);
    if (s != MFTO_OK) return s;
    h->launches++;
    sample_pair<<<reduction_blocks(h->n_dof, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(
        f, h->d_q, u_star, h->d_r, w->uk, (int)h->n_dof);
    MFTO_LAUNCH_CHECK(h);
    s = build_features<double>(h, rho_phys, h->d_r);
    if (s == MFTO_OK) s = build_target(h, w->uk, y_out, mask_out);
  }
  if (s != MFTO_OK) return s;
  MFTO_CUDA(h, cudaMemcpyAsync(x_out, w->x, sizeof(float) * 4 * V, cudaMemcpyDeviceToDevice,
                               h->stream));
  return MFTO_OK;
}

extern "C" mfto_status mfto_set_learned(mfto_handle* h, mfto_nn* nn, int32_t every) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, every >= 0, "mfto_set_learned: every >= 0");
  if (!nn) {
    if (h->learned) h->learned->nn = nullptr;
    return MFTO_OK;
  }
  const int levels = nn_levels(nn);
  mfto_status s = ensure_ws(h, levels);
  if (s != MFTO_OK) return s;
  LearnedWs* w = h->learned;
  if ((long long)w->D * w->H * w->W > nn_max_voxels(nn))
    return mfto_fail(h, MFTO_TOO_LARGE, "mfto_set_learned: network made for %lld voxels, grid has %lld",
                     nn_max_voxels(nn), (long long)w->D * w->H * w->W);
  w->nn = nn;
  w->every = every;
  return MFTO_OK;
}

extern "C" mfto_status mfto_learned_solve(mfto_handle* h, const double* E, const double* rho_phys,
                                          const double* f, double* u, mfto_learned_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, E && rho_phys && f && u, "mfto_learned_solve: null pointer");
  return learned_run(h, E, rho_phys, f, u, st);
}

extern "C" mfto_status mfto_nn_train_energy(mfto_handle* h, mfto_nn* nn, const double* E,
                                            const double* rho_phys, const double* f,
                                            double compliance, float lr, double* loss) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, nn && E && rho_phys && f, "mfto_nn_train_energy: null pointer");
  MFTO_REQUIRE(h, compliance > 0.0 && lr > 0.f, "mfto_nn_train_energy: compliance, lr > 0");
  mfto_status s = ensure_ws(h, nn_levels(nn));
  if (s != MFTO_OK) return s;
  LearnedWs* w = h->learned;
  s = build_features<double>(h, rho_phys, f);
  if (s != MFTO_OK) return s;
  float* out = nullptr;
  s = nn_train_forward(nn, h->stream, w->D, w->H, w->W, w->x, &out);
  if (s != MFTO_OK) return mfto_fail(h, s, "network: %s", nn_message(nn));
  const Grid g = make_grid(h->mesh);
  h->launches += 3;
  to_dofs_kernel<double><<<nblk(h->n_node), MFTO_BLOCK, 0, h->stream>>>(out, w->uk, h->d_fixed, g,
                                                                        vox(w), (int)h->n_node);
  MFTO_LAUNCH_CHECK(h);
  s = kv_launch(h, MFTO_FORM_F64, E, w->uk, h->d_q);
  if (s != MFTO_OK) return s;
  energy_dots<<<reduction_blocks(h->n_dof, MFTO_BLOCK), MFTO_BLOCK, 0, h->stream>>>(
      f, w->uk, h->d_q, (int)h->n_dof, h->d_misc, h->d_partials);
  energy_grad<<<nblk((int64_t)w->D * w->H * w->W), MFTO_BLOCK, 0, h->stream>>>(
      f, h->d_q, h->d_fixed, h->d_misc, compliance, out, g, vox(w));
  MFTO_LAUNCH_CHECK(h);
  s = nn_train_backward(nn, h->stream, w->D, w->H, w->W, lr);
  if (s != MFTO_OK) return mfto_fail(h, s, "network: %s", nn_message(nn));
  if (loss) {
    MFTO_CUDA(h, cudaMemcpyAsync(h->h_misc, h->d_misc, sizeof(MiscScalars), cudaMemcpyDeviceToHost,
                                 h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
    *loss = h->h_misc->sum[2];
  }
  return MFTO_OK;
}

int64_t learned_bytes(const mfto_handle* h) {
  const LearnedWs* w = h->learned;
  if (!w) return 0;
  int64_t b = 0;
  if (w->x) b += (int64_t)sizeof(float) * 7 * (int64_t)w->D * w->H * w->W;
  if (w->c) b += (int64_t)sizeof(float) * h->n_dof;
  if (w->uk) b += (int64_t)sizeof(double) * h->n_dof;
  if (w->amax) b += (int64_t)sizeof(unsigned int) * 2;
  if (w->ctl) b += (int64_t)sizeof(FpcgCtl);
  return b;
}

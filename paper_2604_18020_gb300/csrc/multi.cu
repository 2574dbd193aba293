// Several load cases at once (multi-RHS): one K.V launch for all of them,
// sharing the moduli, the fixed-DOF masks and the index arithmetic, and a
// mixed-precision solve (FP64 refinement per load case around one FP32
// inner CG that advances every case together, each with its own scalars).
// Vectors of the nrhs cases are stored one after the other: [nrhs][n_dof].
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "kv_column.cuh"
#include "kv_tile.cuh"

namespace {

// Block-variant K.V over nrhs cases (see kv_block_body in kv_tile.cuh): per
// block, the masks and moduli are staged once, then each case is staged,
// contracted and summed into its owned nodes in turn.
//   ld(r, idx)  -> input value of case r at DOF idx
//   epi(r, node, acc, pn, fm, red) -> what the owner does for case r
//   active(r)   -> false for cases to skip (converged)
template <typename T, typename Ld, typename Epi, typename Act>
__device__ __forceinline__ void kv_block_multi(const T* __restrict__ E,
                                               const uint8_t* __restrict__ fixed,
                                               const ModeCoef<T>& K, const Grid& g, int nrhs,
                                               const Ld& ld, const Epi& epi, const Act& active,
                                               T* smem, DotAcc<T>* red) {
  using B = BlockShape;
  T* vs = smem;                                                     // [3][NV]
  T* out = vs + 3 * B::NV;                                          // [24][256]
  uint8_t* ms = reinterpret_cast<uint8_t*>(out + 24 * MFTO_BLOCK);  // [NV]
  const int tid = threadIdx.x;
  const int tx = (g.nx + B::OX - 1) / B::OX, ty = (g.ny + B::OY - 1) / B::OY;
  const int tz = (g.nz + B::OZ - 1) / B::OZ;
  const int n_blocks = tx * ty * tz;
  const int ex = tid & 7, ey = (tid >> 3) & 7, ez = tid >> 6;
  for (int b = blockIdx.x; b < n_blocks; b += gridDim.x) {
    const int bx = b % tx, by = (b / tx) % ty, bz = b / (tx * ty);
    const int ox = bx * B::OX, oy = by * B::OY, oz = bz * B::OZ;
    for (int idx = tid; idx < B::NV; idx += MFTO_BLOCK) {
      const int lx = idx % B::VX, ly = (idx / B::VX) % B::VY, lz = idx / (B::VX * B::VY);
      const int gi = ox - 1 + lx, gj = oy - 1 + ly, gk = oz - 1 + lz;
      ms[idx] = (gi >= 0 && gj >= 0 && gk >= 0 && gi < g.nx && gj < g.ny && gk < g.nz)
                    ? fixed[gi + g.nx * (gj + g.ny * gk)] : (uint8_t)0;
    }
    const int ei = ox - 1 + ex, ej = oy - 1 + ey, ek = oz - 1 + ez;
    T Ee = 0;
    if (ei >= 0 && ej >= 0 && ek >= 0 && ei < g.nelx && ej < g.nely && ek < g.nelz)
      Ee = E[ei + g.nelx * (ej + g.nely * ek)];
    __syncthreads();
    for (int r = 0; r < nrhs; ++r) {
      if (!active(r)) continue;                       // uniform over the block
      for (int idx = tid; idx < B::NV; idx += MFTO_BLOCK) {
        const int lx = idx % B::VX, ly = (idx / B::VX) % B::VY, lz = idx / (B::VX * B::VY);
        const int gi = ox - 1 + lx, gj = oy - 1 + ly, gk = oz - 1 + lz;
        T a = 0, bb = 0, c = 0;
        if (gi >= 0 && gj >= 0 && gk >= 0 && gi < g.nx && gj < g.ny && gk < g.nz) {
          const int node = gi + g.nx * (gj + g.ny * gk);
          const uint8_t fm = ms[idx];
          a = (fm & 1) ? T(0) : ld(r, 3 * node + 0);
          bb = (fm & 2) ? T(0) : ld(r, 3 * node + 1);
          c = (fm & 4) ? T(0) : ld(r, 3 * node + 2);
        }
        vs[idx] = a;
        vs[B::NV + idx] = bb;
        vs[2 * B::NV + idx] = c;
      }
      __syncthreads();
      {
        T x[3][8];
#pragma unroll
        for (int l = 0; l < 8; ++l) {
          const int vi = (ex + (l & 1)) + B::VX * ((ey + ((l >> 1) & 1)) + B::VY * (ez + (l >> 2)));
          x[0][l] = vs[vi];
          x[1][l] = vs[B::NV + vi];
          x[2][l] = vs[2 * B::NV + vi];
        }
        element_apply<T>(x, Ee, K);
#pragma unroll
        for (int l = 0; l < 8; ++l)
#pragma unroll
          for (int c = 0; c < 3; ++c) out[(3 * l + c) * MFTO_BLOCK + tid] = x[c][l];
      }
      __syncthreads();
      if (tid < B::NO) {
        const int ix = tid % B::OX, iy = (tid / B::OX) % B::OY, iz = tid / (B::OX * B::OY);
        const int gi = ox + ix, gj = oy + iy, gk = oz + iz;
        if (gi < g.nx && gj < g.ny && gk < g.nz) {
          T acc[3] = {0, 0, 0};
#pragma unroll
          for (int ec = 0; ec < 2; ++ec)
#pragma unroll
            for (int eb = 0; eb < 2; ++eb)
#pragma unroll
              for (int ea = 0; ea < 2; ++ea) {
                const int e = (ix + ea) + B::BX * ((iy + eb) + B::BY * (iz + ec));
                const int corner = (1 - ea) + 2 * (1 - eb) + 4 * (1 - ec);
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c] += out[(3 * corner + c) * MFTO_BLOCK + e];
              }
          const int vi = (ix + 1) + B::VX * ((iy + 1) + B::VY * (iz + 1));
          const T pn[3] = {vs[vi], vs[B::NV + vi], vs[2 * B::NV + vi]};
          epi(r, gi + g.nx * (gj + g.ny * gk), acc, pn, ms[vi], red[r]);
        }
      }
      __syncthreads();
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
kv_multi_kernel(const T* __restrict__ E, const T* __restrict__ V, T* __restrict__ Y,
                const uint8_t* __restrict__ fixed, ModeCoef<T> K, Grid g, int nrhs, int n_dof) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DotAcc<T> red[MFTO_MAX_RHS];
  auto ld = [&](int r, int i) { return V[(size_t)r * n_dof + i]; };
  auto epi = [&](int r, int node, const T (&acc)[3], const T (&pn)[3], uint8_t fm, DotAcc<T>&) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t i = (size_t)r * n_dof + 3 * node + c;
      Y[i] = ((fm >> c) & 1) ? V[i] : acc[c];
    }
  };
  kv_block_multi<T>(E, fixed, K, g, nrhs, ld, epi, [](int) { return true; },
                    reinterpret_cast<T*>(smem_raw), red);
}

// CG step A for every active case: p_new = z + beta p_old, q = K p_new, p.q
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_kv_multi(const float* __restrict__ E, const float* __restrict__ Z, const float* __restrict__ P0,
             float* __restrict__ P1, float* __restrict__ Q, const uint8_t* __restrict__ fixed,
             ModeCoef<float> K, Grid g, int n_dof, MultiScalars* s, double* partials) {
  if (*(volatile int32_t*)&s->all_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[64];
  const int nrhs = s->nrhs;
  float beta[MFTO_MAX_RHS];
  int32_t done[MFTO_MAX_RHS];
#pragma unroll
  for (int r = 0; r < MFTO_MAX_RHS; ++r) {
    beta[r] = r < nrhs ? (float)s->beta[r] : 0.f;
    done[r] = r < nrhs ? s->done[r] : 1;
  }
  DotAcc<float> red[MFTO_MAX_RHS];
  auto ld = [&](int r, int i) {
    const size_t o = (size_t)r * n_dof + i;
    return Z[o] + beta[r] * P0[o];
  };
  auto epi = [&](int r, int node, const float (&acc)[3], const float (&pn)[3], uint8_t fm,
                 DotAcc<float>& d) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)r * n_dof + 3 * node + c;
      const float qc = ((fm >> c) & 1) ? pn[c] : acc[c];
      P1[o] = pn[c];
      Q[o] = qc;
      d.add_prod(pn[c], qc);
    }
  };
  kv_block_multi<float>(E, fixed, K, g, nrhs, ld, epi, [&](int r) { return !done[r]; },
                        reinterpret_cast<float*>(smem_raw), red);
  double part[MFTO_MAX_RHS];
#pragma unroll
  for (int r = 0; r < MFTO_MAX_RHS; ++r) part[r] = red[r].finish();
  double tot[MFTO_MAX_RHS];
  if (last_block_reduce<MFTO_MAX_RHS, true>(part, partials, &s->ticket_b, tot, sh) &&
      threadIdx.x == 0) {
    for (int r = 0; r < nrhs; ++r) {
      if (s->done[r]) continue;
      s->pq[r] = tot[r];
      if (!(tot[r] > 0.0) || !isfinite(tot[r])) {
        s->done[r] = 1;
        s->status[r] = MFTO_BREAKDOWN;
        s->alpha[r] = 0.0;
      } else {
        s->alpha[r] = s->rz[r] / tot[r];
      }
    }
  }
}

// CG step B for every active case
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_update_multi(float* __restrict__ U, const float* __restrict__ P, const float* __restrict__ Q,
                 float* __restrict__ R, float* __restrict__ Z, const float* __restrict__ dinv,
                 int n_node, int n_dof, MultiScalars* s, double* partials) {
  if (*(volatile int32_t*)&s->all_done) return;
  __shared__ double sh[64];
  const int nrhs = s->nrhs;
  float alpha[MFTO_MAX_RHS];
  int32_t done[MFTO_MAX_RHS];
#pragma unroll
  for (int r = 0; r < MFTO_MAX_RHS; ++r) {
    alpha[r] = r < nrhs ? (float)s->alpha[r] : 0.f;
    done[r] = r < nrhs ? s->done[r] : 1;
  }
  DotAcc<float> d[2 * MFTO_MAX_RHS];
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < n_node; nd += gridDim.x * blockDim.x) {
#pragma unroll
    for (int r = 0; r < MFTO_MAX_RHS; ++r) {
      if (done[r]) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t i = (size_t)r * n_dof + 3 * nd + c;
        U[i] += alpha[r] * P[i];
        const float ri = R[i] - alpha[r] * Q[i];
        const float zi = ri * dinv[3 * nd + c];
        R[i] = ri;
        Z[i] = zi;
        d[2 * r].add_prod(ri, zi);
        d[2 * r + 1].add_prod(ri, ri);
      }
    }
  }
  double part[2 * MFTO_MAX_RHS];
#pragma unroll
  for (int k = 0; k < 2 * MFTO_MAX_RHS; ++k) part[k] = d[k].finish();
  double tot[2 * MFTO_MAX_RHS];
  if (last_block_reduce<2 * MFTO_MAX_RHS, true>(part, partials, &s->ticket_c, tot, sh) &&
      threadIdx.x == 0) {
    int all = 1;
    for (int r = 0; r < nrhs; ++r) {
      if (!s->done[r]) {
        s->it[r] += 1;
        s->rr[r] = tot[2 * r + 1];
        s->beta[r] = tot[2 * r] / s->rz[r];
        s->rz[r] = tot[2 * r];
        if (!isfinite(tot[2 * r]) || !isfinite(tot[2 * r + 1])) {
          s->done[r] = 1;
          s->status[r] = MFTO_BREAKDOWN;
        } else if (tot[2 * r + 1] <= s->rtol2ff[r]) {
          s->done[r] = 1;
          s->status[r] = MFTO_OK;
        } else if (s->it[r] >= s->maxit) {
          s->done[r] = 1;
          s->status[r] = MFTO_NOT_CONVERGED;
        }
      }
      all &= s->done[r];
    }
    s->all_done = all;
  }
}

// The same two CG steps with the column K.v (kv_column.cuh) and 16-byte
// vector updates: grid row blockIdx.y is load case r, so every case has its
// own tiles, partial rows (2r, 2r + 1 of the partial buffers) and tickets,
// and a converged case's blocks return at entry.  The last case to finish
// raises all_done.
__device__ __forceinline__ void multi_case_done(MultiScalars* s) {
  if (atomicAdd(&s->ndone, 1) + 1 >= s->nrhs) s->all_done = 1;
}

template <int MINB>
__global__ void __launch_bounds__(MFTO_BLOCK, MINB)
pcg_kv_multi_col(const float* __restrict__ E, const float* __restrict__ Z,
                 const float* __restrict__ P0, float* __restrict__ P1, float* __restrict__ Q,
                 const uint8_t* __restrict__ fixed, ModeCoef<float> K, Grid g, ColTiling tl,
                 int n_dof, MultiScalars* s, double* partials) {
  const int r = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[64];
  const size_t o = (size_t)r * n_dof;
  DotAcc<float> acc;
  bool skipped = false;   // the case is done: uniform over the case's blocks
  acc.s = kv_column_body(E, fixed, K, g, tl, ColLoadDirection{Z + o, P0 + o, 0.f},
                         ColPcg{P1 + o, Q + o}, reinterpret_cast<float*>(smem_raw),
                         ColPreFlagBeta{&s->done[r], &s->beta[r]}, &skipped);
  if (skipped) return;
  const DFloat w[1] = {acc.finish_df()};
  double tot[1];
  if (row_reduce_df<1>(w, partials + (size_t)2 * r * MFTO_RED_SLOTS, &s->ticket_kv[r], tot, sh) &&
      threadIdx.x == 0) {
    s->pq[r] = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      s->done[r] = 1;
      s->status[r] = MFTO_BREAKDOWN;
      s->alpha[r] = 0.0;
      multi_case_done(s);
    } else {
      s->alpha[r] = s->rz[r] / tot[0];
    }
  }
}

__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_update_multi_col(float* __restrict__ U, const float* __restrict__ P,
                     const float* __restrict__ Q, float* __restrict__ R, float* __restrict__ Z,
                     const float* __restrict__ dinv, int n_dof, MultiScalars* s,
                     double* partials) {
  const int r = blockIdx.y;
  int done = 0;
  const float alpha = flag_and_scalar_f32(&s->done[r], &s->alpha[r], &done);
  if (done) return;
  __shared__ double sh[64];
  const size_t o = (size_t)r * n_dof;
  DotAcc<float> d0, d1;
  // groups of 4 consecutive DOFs (a case's vectors start at r n_dof, which
  // need not be 16-byte aligned, so scalar accesses); each group's products
  // are summed in FP32 before the double-float accumulation
  float* u = U + o;
  const float* p = P + o;
  const float* q = Q + o;
  float* rv = R + o;
  float* z = Z + o;
  for (int g4 = blockIdx.x * blockDim.x + threadIdx.x; 4 * g4 < n_dof;
       g4 += gridDim.x * blockDim.x) {
    float t0 = 0.f, t1 = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = 4 * g4 + c;
      if (i < n_dof) {
        u[i] += alpha * p[i];
        const float ri = rv[i] - alpha * q[i];
        const float zi = ri * dinv[i];
        rv[i] = ri;
        z[i] = zi;
        t0 = fmaf(ri, zi, t0);
        t1 = fmaf(ri, ri, t1);
      }
    }
    d0.add(t0);
    d1.add(t1);
  }
  const DFloat w[2] = {d0.finish_df(), d1.finish_df()};
  double tot[2];
  if (row_reduce_df<2>(w, partials + (size_t)2 * r * MFTO_RED_SLOTS, &s->ticket_up[r], tot, sh) &&
      threadIdx.x == 0) {
    s->it[r] += 1;
    s->rr[r] = tot[1];
    s->beta[r] = tot[0] / s->rz[r];
    s->rz[r] = tot[0];
    int fin = 1;
    if (!isfinite(tot[0]) || !isfinite(tot[1])) s->status[r] = MFTO_BREAKDOWN;
    else if (tot[1] <= s->rtol2ff[r]) s->status[r] = MFTO_OK;
    else if (s->it[r] >= s->maxit) s->status[r] = MFTO_NOT_CONVERGED;
    else fin = 0;
    if (fin) {
      s->done[r] = 1;
      multi_case_done(s);
    }
  }
}

// Outer FP64 residual of every case: R = F - KU; r.r, f.f per case; the FP32
// right-hand side of the inner solve (zero for cases marked converged).
__global__ void __launch_bounds__(MFTO_BLOCK)
ir_residual_multi(const double* __restrict__ F, const double* __restrict__ KU,
                  float* __restrict__ R32, int n_dof, int nrhs, unsigned int converged,
                  MiscScalars* s, double* partials, double* out) {
  __shared__ double sh[64];
  double acc[2 * MFTO_MAX_RHS];
#pragma unroll
  for (int k = 0; k < 2 * MFTO_MAX_RHS; ++k) acc[k] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_dof; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int r = 0; r < MFTO_MAX_RHS; ++r) {
      if (r >= nrhs) break;
      const size_t o = (size_t)r * n_dof + i;
      const double ri = F[o] - KU[o];
      R32[o] = ((converged >> r) & 1u) ? 0.f : (float)ri;
      acc[2 * r] += ri * ri;
      acc[2 * r + 1] += F[o] * F[o];
    }
  }
  double tot[2 * MFTO_MAX_RHS];
  if (last_block_reduce<2 * MFTO_MAX_RHS>(acc, partials, &s->ticket, tot, sh) &&
      threadIdx.x == 0) {
    for (int k = 0; k < 2 * MFTO_MAX_RHS; ++k) out[k] = tot[k];
  }
}

// r.z of the direction each case continues with (0: a new start, p = z)
struct RzPrev {
  double v[MFTO_MAX_RHS];
};

// Inner solve start for every case: r = rhs (in place), z = r / d, sums.
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_init_multi(float* R, float* __restrict__ Z, const float* __restrict__ dinv, int n_dof,
               int nrhs, double rtol, int maxit, RzPrev rz_prev, MultiScalars* s,
               double* partials) {
  __shared__ double sh[64];
  DotAcc<float> d[2 * MFTO_MAX_RHS];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_dof; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int r = 0; r < MFTO_MAX_RHS; ++r) {
      if (r >= nrhs) break;
      const size_t o = (size_t)r * n_dof + i;
      const float ri = R[o];
      const float zi = ri * dinv[i];
      Z[o] = zi;
      d[2 * r].add_prod(ri, zi);
      d[2 * r + 1].add_prod(ri, ri);
    }
  }
  double part[2 * MFTO_MAX_RHS];
#pragma unroll
  for (int k = 0; k < 2 * MFTO_MAX_RHS; ++k) part[k] = d[k].finish();
  double tot[2 * MFTO_MAX_RHS];
  if (last_block_reduce<2 * MFTO_MAX_RHS, true>(part, partials, &s->ticket_a, tot, sh) &&
      threadIdx.x == 0) {
    int all = 1;
    for (int r = 0; r < MFTO_MAX_RHS; ++r) {
      const bool live = r < nrhs;
      s->rz[r] = live ? tot[2 * r] : 0.0;
      s->rr[r] = live ? tot[2 * r + 1] : 0.0;
      s->ff[r] = s->rr[r];                       // the inner right-hand side is r0
      s->rtol2ff[r] = rtol * rtol * s->ff[r];
      s->alpha[r] = 0.0;
      s->beta[r] = (live && rz_prev.v[r] > 0.0) ? s->rz[r] / rz_prev.v[r] : 0.0;
      s->it[r] = 0;
      s->status[r] = MFTO_OK;
      s->done[r] = (!live || s->ff[r] == 0.0) ? 1 : 0;
      all &= s->done[r];
    }
    int nd = 0;
    for (int r = 0; r < nrhs; ++r) nd += s->done[r];
    s->ndone = nd;
    s->nrhs = nrhs;
    s->maxit = maxit;
    s->all_done = all;
  }
}

__global__ void __launch_bounds__(MFTO_BLOCK)
ir_accumulate_multi(double* __restrict__ U, const float* __restrict__ E32, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    U[i] += (double)E32[i];
}

size_t block_smem(size_t esz) {
  return esz * (3 * BlockShape::NV + 24 * MFTO_BLOCK) + BlockShape::NV;
}

}  // namespace

static unsigned multi_grid(const mfto_handle* h, int per_sm) {
  const Grid g = make_grid(h->mesh);
  const int64_t nb = (int64_t)((g.nx + 6) / 7) * ((g.ny + 6) / 7) * ((g.nz + 2) / 3);
  int64_t grid = (int64_t)per_sm * h->num_sms;
  if (grid > nb) grid = nb;
  if (grid > MFTO_RED_SLOTS) grid = MFTO_RED_SLOTS;
  return (unsigned)grid;
}

mfto_status multi_init(mfto_handle* h) {
  MFTO_CUDA(h, cudaFuncSetAttribute(kv_multi_kernel<double>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)block_smem(8)));
  MFTO_CUDA(h, cudaFuncSetAttribute(kv_multi_kernel<float>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)block_smem(4)));
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_kv_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)block_smem(4)));
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ_multi[0],
                                                             kv_multi_kernel<double>, MFTO_BLOCK,
                                                             block_smem(8)));
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ_multi[1],
                                                             kv_multi_kernel<float>, MFTO_BLOCK,
                                                             block_smem(4)));
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ_multi[2], pcg_kv_multi,
                                                             MFTO_BLOCK, block_smem(4)));
  for (int i = 0; i < 3; ++i)
    if (h->occ_multi[i] < 1) h->occ_multi[i] = 1;
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_kv_multi_col<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kColSmem));
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_kv_multi_col<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kColSmem));
  return MFTO_OK;
}

static mfto_status kv_multi_launch(mfto_handle* h, mfto_form form, const void* E, const void* V,
                                   void* Y, int nrhs) {
  const Grid g = make_grid(h->mesh);
  h->launches++;
  if (form == MFTO_FORM_F64) {
    kv_multi_kernel<double><<<multi_grid(h, h->occ_multi[0]), MFTO_BLOCK, block_smem(8),
                              h->stream>>>((const double*)E, (const double*)V, (double*)Y,
                                           h->d_fixed, h->mc64, g, nrhs, (int)h->n_dof);
  } else if (form == MFTO_FORM_F32) {
    kv_multi_kernel<float><<<multi_grid(h, h->occ_multi[1]), MFTO_BLOCK, block_smem(4),
                             h->stream>>>((const float*)E, (const float*)V, (float*)Y,
                                          h->d_fixed, h->mc32, g, nrhs, (int)h->n_dof);
  } else {
    return mfto_fail(h, MFTO_UNSUPPORTED, "mfto_kv_multi: forms F64 and F32 only");
  }
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

extern "C" mfto_status mfto_kv_multi(mfto_handle* h, mfto_form form, const void* E,
                                     const void* V, void* Y, int32_t nrhs) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, E && V && Y, "mfto_kv_multi: null pointer");
  MFTO_REQUIRE(h, V != Y, "mfto_kv_multi: Y must not alias V");
  MFTO_REQUIRE(h, nrhs >= 1 && nrhs <= MFTO_MAX_RHS, "mfto_kv_multi: nrhs must lie in 1..8");
  return kv_multi_launch(h, form, E, V, Y, nrhs);
}

// ---- the multi-RHS inner CG: graph-captured chunks, like pcg.cu --------------

struct MultiGraph {
  const void* key = nullptr;
  int chunk = 0;
  int nrhs = 0, variant = 0, kind = 0, nzc = 0;
  cudaGraphExec_t exec = nullptr;
};

static mfto_status multi_chunk(mfto_handle* h, cudaStream_t st, int chunk, int nrhs) {
  const Grid g = make_grid(h->mesh);
  int nb_node = (int)((h->n_node + MFTO_BLOCK - 1) / MFTO_BLOCK);
  if (nb_node > MFTO_RED_MAX_BLOCKS) nb_node = MFTO_RED_MAX_BLOCKS;
  // column kernels: one grid row per case, the K.v tiling of a single case
  int grid = 0;
  const ColTiling tl = col_launch_tiling(h, h->occ_col[h->col_kind], &grid);
  int64_t nb_up = ((int64_t)h->n_dof / 4 + MFTO_BLOCK) / MFTO_BLOCK;
  if (nb_up > 2 * (int64_t)h->num_sms) nb_up = 2 * (int64_t)h->num_sms;
  for (int it = 0; it < chunk; ++it) {
    float* p_old = (it & 1) ? h->m_p1 : h->m_p0;
    float* p_new = (it & 1) ? h->m_p0 : h->m_p1;
    if (h->kv_variant == 0) {
      const dim3 gk((unsigned)grid, (unsigned)nrhs);
      if (h->col_kind == 1)
        pcg_kv_multi_col<3><<<gk, MFTO_BLOCK, kColSmem, st>>>(
            h->d_E32, h->m_z32, p_old, p_new, h->m_q32, h->d_fixed, h->mc32, g, tl,
            (int)h->n_dof, h->m_pcg, h->d_partials);
      else
        pcg_kv_multi_col<2><<<gk, MFTO_BLOCK, kColSmem, st>>>(
            h->d_E32, h->m_z32, p_old, p_new, h->m_q32, h->d_fixed, h->mc32, g, tl,
            (int)h->n_dof, h->m_pcg, h->d_partials);
      pcg_update_multi_col<<<dim3((unsigned)nb_up, (unsigned)nrhs), MFTO_BLOCK, 0, st>>>(
          h->m_e32, p_new, h->m_q32, h->m_r32, h->m_z32, h->d_dinv32, (int)h->n_dof, h->m_pcg,
          h->d_partials2);
    } else {
      pcg_kv_multi<<<multi_grid(h, h->occ_multi[2]), MFTO_BLOCK, block_smem(4), st>>>(
          h->d_E32, h->m_z32, p_old, p_new, h->m_q32, h->d_fixed, h->mc32, g, (int)h->n_dof,
          h->m_pcg, h->d_partials);
      pcg_update_multi<<<nb_node, MFTO_BLOCK, 0, st>>>(h->m_e32, p_new, h->m_q32, h->m_r32,
                                                       h->m_z32, h->d_dinv32, (int)h->n_node,
                                                       (int)h->n_dof, h->m_pcg, h->d_partials2);
    }
  }
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

void multi_graph_release(mfto_handle* h) {
  MultiGraph* mg = reinterpret_cast<MultiGraph*>(h->m_graph);
  if (mg) {
    if (mg->exec) cudaGraphExecDestroy(mg->exec);
    delete mg;
  }
  h->m_graph = nullptr;
}

static mfto_status multi_graph(mfto_handle* h, int nrhs, MultiGraph** out) {
  MultiGraph* mg = reinterpret_cast<MultiGraph*>(h->m_graph);
  if (mg && mg->key == h->d_E32 && mg->chunk == h->p.check_every && mg->nrhs == nrhs &&
      mg->variant == h->kv_variant && mg->kind == h->col_kind && mg->nzc == h->col_nzc) {
    *out = mg;
    return MFTO_OK;
  }
  multi_graph_release(h);
  mg = new MultiGraph();
  mg->key = h->d_E32;
  mg->chunk = h->p.check_every;
  mg->nrhs = nrhs;
  mg->variant = h->kv_variant;
  mg->kind = h->col_kind;
  mg->nzc = h->col_nzc;
  if (!h->cap_stream &&
      cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete mg;
    return mfto_fail(h, MFTO_CUDA_ERROR, "multi-RHS graph: cannot create the capture stream");
  }
  cudaGraph_t graph = nullptr;
  MFTO_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  mfto_status s = multi_chunk(h, h->cap_stream, mg->chunk, nrhs);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (s != MFTO_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    delete mg;
    return s != MFTO_OK ? s : mfto_fail(h, MFTO_CUDA_ERROR, "multi-RHS graph capture failed");
  }
  e = cudaGraphInstantiate(&mg->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    delete mg;
    return mfto_fail(h, MFTO_CUDA_ERROR, "multi-RHS graph instantiate failed");
  }
  h->m_graph = mg;
  *out = mg;
  return MFTO_OK;
}

mfto_status mfto_to_f32(mfto_handle* h, const double* a, float* b, int64_t n);  // ir.cu

extern "C" mfto_status mfto_ir_solve_multi(mfto_handle* h, double inner_tol, const double* E,
                                           const double* F, double* U, int32_t nrhs,
                                           mfto_ir_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, E && F && U && st, "mfto_ir_solve_multi: null pointer");
  MFTO_REQUIRE(h, nrhs >= 1 && nrhs <= h->max_rhs,
               "mfto_ir_solve_multi: nrhs must lie in 1..max_rhs of mfto_create");
  MFTO_REQUIRE(h, inner_tol > 0.0 && inner_tol < 1.0, "mfto_ir_solve_multi: inner_tol in (0,1)");
  const int n = (int)h->n_dof;
  const size_t total = (size_t)nrhs * n;
  const int nb = reduction_blocks(h->n_dof, MFTO_BLOCK);
  for (int r = 0; r < nrhs; ++r) {
    memset(&st[r], 0, sizeof(mfto_ir_stats));
    st[r].status = MFTO_NOT_CONVERGED;
  }
  mfto_status s = mfto_to_f32(h, E, h->d_E32, h->n_elem);
  if (s != MFTO_OK) return s;
  s = diag_launch(h, MFTO_FORM_F32, h->d_E32, h->d_dinv32, true);
  if (s != MFTO_OK) return s;
  double prev[MFTO_MAX_RHS] = {0};
  int stalls[MFTO_MAX_RHS] = {0};
  RzPrev rzp;                 // continued directions (MFTO_IR_CONTINUE), per case
  for (int r = 0; r < MFTO_MAX_RHS; ++r) rzp.v[r] = 0.0;
  unsigned int converged = 0, stopped = 0;
  double* d_out = h->m_out;   // per-case r.r, f.f of the outer residual
  double out[2 * MFTO_MAX_RHS];
  for (int outer = 0;; ++outer) {
    s = kv_multi_launch(h, MFTO_FORM_F64, E, U, h->m_q64, nrhs);
    if (s != MFTO_OK) return s;
    h->launches++;
    ir_residual_multi<<<nb, MFTO_BLOCK, 0, h->stream>>>(F, h->m_q64, h->m_r32, n, nrhs,
                                                        converged | stopped, h->d_misc,
                                                        h->d_partials, d_out);
    MFTO_LAUNCH_CHECK(h);
    MFTO_CUDA(h, cudaMemcpyAsync(out, d_out, sizeof(out), cudaMemcpyDeviceToHost, h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
    unsigned int newly = 0;
    for (int r = 0; r < nrhs; ++r) {
      if (((converged | stopped) >> r) & 1u) continue;
      const double rr = out[2 * r], ff = out[2 * r + 1];
      st[r].fnorm = sqrt(ff);
      const double rel = ff > 0.0 ? sqrt(rr / ff) : 0.0;
      st[r].rel_residual = rel;
      st[r].kv_f64++;
      if (outer < 64) st[r].history[outer] = rel;
      if (rel <= h->p.rtol) { st[r].status = MFTO_OK; newly |= 1u << r; continue; }
      if (!isfinite(rel)) { st[r].status = MFTO_BREAKDOWN; stopped |= 1u << r; continue; }
      if (outer > 0) {
        stalls[r] = rel > 0.9 * prev[r] ? stalls[r] + 1 : 0;
        if (stalls[r] >= 2) { st[r].status = MFTO_STALLED; stopped |= 1u << r; continue; }
      }
      if (outer >= h->max_outer) { st[r].status = MFTO_NOT_CONVERGED; stopped |= 1u << r; continue; }
      prev[r] = rel;
    }
    converged |= newly;
    const unsigned int all = (nrhs >= 32 ? 0xffffffffu : ((1u << nrhs) - 1u));
    if (((converged | stopped) & all) == all) break;
    if (newly) {
      // the right-hand sides written above still hold the just-converged
      // cases: clear them so their inner solves are empty
      for (int r = 0; r < nrhs; ++r)
        if ((newly >> r) & 1u)
          MFTO_CUDA(h, cudaMemsetAsync(h->m_r32 + (size_t)r * n, 0, sizeof(float) * n, h->stream));
    }
    for (int r = 0; r < nrhs; ++r)
      if ((stopped >> r) & 1u)
        MFTO_CUDA(h, cudaMemsetAsync(h->m_r32 + (size_t)r * n, 0, sizeof(float) * n, h->stream));
    // inner solve of every live case from e = 0; a case continuing its
    // direction keeps it in p0, the others start from p = z
    MFTO_CUDA(h, cudaMemsetAsync(h->m_e32, 0, sizeof(float) * total, h->stream));
    for (int r = 0; r < nrhs; ++r) {
      if (((converged | stopped) >> r) & 1u) rzp.v[r] = 0.0;
      if (!(rzp.v[r] > 0.0))
        MFTO_CUDA(h, cudaMemsetAsync(h->m_p0 + (size_t)r * n, 0, sizeof(float) * n, h->stream));
    }
    h->launches++;
    pcg_init_multi<<<nb, MFTO_BLOCK, 0, h->stream>>>(h->m_r32, h->m_z32, h->d_dinv32, n, nrhs,
                                                     inner_tol, h->inner_maxit, rzp, h->m_pcg,
                                                     h->d_partials);
    MFTO_LAUNCH_CHECK(h);
    MultiGraph* mg = nullptr;
    s = multi_graph(h, nrhs, &mg);
    if (s != MFTO_OK) return s;
    for (;;) {
      MFTO_CUDA(h, cudaMemcpyAsync(h->h_mpcg, h->m_pcg, sizeof(MultiScalars),
                                   cudaMemcpyDeviceToHost, h->stream));
      MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
      if (h->h_mpcg->all_done) break;
      MFTO_CUDA(h, cudaGraphLaunch(mg->exec, h->stream));
      h->launches += 2 * (int64_t)mg->chunk;
    }
    for (int r = 0; r < nrhs; ++r) {
      if (((converged | stopped) >> r) & 1u) continue;
      const MultiScalars& fin = *h->h_mpcg;
      st[r].inner_iterations += fin.it[r];
      st[r].outer_iterations++;
      // continued direction: iteration j wrote its direction into p1 (j even)
      // or p0 (j odd); the next inner solve reads p0 first
      rzp.v[r] = 0.0;
      if (h->ir_mode == MFTO_IR_CONTINUE && fin.it[r] >= 1 && fin.status[r] != MFTO_BREAKDOWN &&
          fin.beta[r] > 0.0 && isfinite(fin.rz[r] / fin.beta[r])) {
        if (fin.it[r] & 1)
          MFTO_CUDA(h, cudaMemcpyAsync(h->m_p0 + (size_t)r * n, h->m_p1 + (size_t)r * n,
                                       sizeof(float) * n, cudaMemcpyDeviceToDevice, h->stream));
        rzp.v[r] = fin.rz[r] / fin.beta[r];
      }
    }
    h->launches++;
    ir_accumulate_multi<<<nb, MFTO_BLOCK, 0, h->stream>>>(U, h->m_e32, total);
    MFTO_LAUNCH_CHECK(h);
  }
  return MFTO_OK;
}

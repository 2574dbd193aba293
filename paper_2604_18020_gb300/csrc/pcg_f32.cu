// FP32 inner CG without grid-wide tickets (CG engine 2): the Jacobi-PCG of
// Sec. 3.6 with the same per-entry arithmetic as the two-kernel graph engine
// (pcg.cu), but every dot product is reduced by the kernel that consumes it.
//
//   A(k)  column K.v (kv_column.cuh): its pre-step sums the per-block shares
//         of r.z and r.r left by B(k-1) (or by the seed), decides
//         convergence, forms beta = r.z / (r.z)_prev while the first node
//         layers are in flight, then p = z + beta p_old, q = K p, and writes
//         its block's share of p.q;
//   B(k)  vector update: sums A(k)'s shares of p.q while its first vector
//         groups are in flight, forms alpha, updates u, r, z and writes its
//         block's shares of r.z and r.r.
// Every block of a launch sums the same partials in the same fixed order, so
// all blocks reach bit-identical scalars and the same decisions; block 0
// alone publishes them.  Scalars that a launch reads from the previous one
// while block 0 writes the next value (r.z, the iteration count) are
// double-buffered by iteration parity, which is fixed per launch in the
// captured chunk (chunks have an even number of iterations).  beta is r.z
// times the reciprocal of the previous r.z, which B formed (the K.v kernel
// holds no FP64 division).  This removes
// the fence, ticket atomic and last-block pass that end each kernel of the
// graph engine.
#include <math.h>

#include "cg_update.cuh"
#include "common.cuh"
#include "kv_column.cuh"
#include "kv_tcol.cuh"

namespace {

// Thread 0's sum of the 8 warps' double-float values of K rows, as a
// balanced tree ((w0 + w1) + (w2 + w3)) + ((w4 + w5) + (w6 + w7)): the same
// fixed order in every block, three dependent additions instead of eight.
static_assert(MFTO_BLOCK / 32 == 8, "warp tree over 8 warps");
template <int K>
__device__ __forceinline__ void warp_tree8(const float2 (&sh)[K][MFTO_BLOCK / 32], DFloat (&t)[K]) {
  DFloat a[K][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < K; ++c)
      a[c][i] = df_add(DFloat{sh[c][2 * i].x, sh[c][2 * i].y},
                       DFloat{sh[c][2 * i + 1].x, sh[c][2 * i + 1].y});
#pragma unroll
  for (int c = 0; c < K; ++c) t[c] = df_add(df_add(a[c][0], a[c][1]), df_add(a[c][2], a[c][3]));
}

// Sums of K rows of double-float partials pf[c * MFTO_RED_SLOTS + b], b < nb,
// in a fixed order: threads stride the blocks, then a shuffle tree in each
// warp, then a balanced tree over the warps (warp_tree8).  partials_load
// issues a thread's first kPartAhead loads (so that they can go out before
// other memory traffic of the launch);
// partials_sum adds them and any further strides.  Thread 0 gets the FP64
// totals (the same bits in every block); the other threads get 0.  FP64
// instructions stay in one thread: the FP64 pipe issues a warp instruction
// at a small fraction of the FP32 rate whatever the number of active lanes.
// One barrier; call uniformly, once per launch.  Three loads ahead cover the
// update kernel's blocks (at most 4 per SM, 608 on 152 SMs) in one pass;
// measured 0.3 % faster per CG iteration at 216k than four.
constexpr int kPartAhead = 3;
template <int K>
struct PartialLoads {
  float2 x[kPartAhead][K];
};

template <int K>
__device__ __forceinline__ PartialLoads<K> partials_load(const float2* __restrict__ pf, int nb) {
  PartialLoads<K> L;
#pragma unroll
  for (int j = 0; j < kPartAhead; ++j) {
    const int b = threadIdx.x + j * blockDim.x;
#pragma unroll
    for (int c = 0; c < K; ++c)
      L.x[j][c] = b < nb ? __ldcg(&pf[c * MFTO_RED_SLOTS + b]) : make_float2(0.f, 0.f);
  }
  return L;
}

template <int K>
__device__ __forceinline__ void partials_sum(const PartialLoads<K>& L, const float2* __restrict__ pf,
                                             int nb, double (&out)[K]) {
  __shared__ float2 sh[K][MFTO_BLOCK / 32];
  DFloat t[K];
#pragma unroll
  for (int c = 0; c < K; ++c) t[c] = DFloat{0.f, 0.f};
#pragma unroll
  for (int j = 0; j < kPartAhead; ++j) {
    if (threadIdx.x + j * blockDim.x < nb) {
#pragma unroll
      for (int c = 0; c < K; ++c) t[c] = df_add(t[c], DFloat{L.x[j][c].x, L.x[j][c].y});
    }
  }
  for (int b = threadIdx.x + kPartAhead * blockDim.x; b < nb; b += blockDim.x) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const float2 y = __ldcg(&pf[c * MFTO_RED_SLOTS + b]);
      t[c] = df_add(t[c], DFloat{y.x, y.y});
    }
  }
#pragma unroll
  for (int c = 0; c < K; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      DFloat w;
      w.hi = __shfl_down_sync(0xffffffffu, t[c].hi, o);
      w.lo = __shfl_down_sync(0xffffffffu, t[c].lo, o);
      t[c] = df_add(t[c], w);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) sh[c][warp] = make_float2(t[c].hi, t[c].lo);
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < K; ++c) out[c] = 0.0;
  if (threadIdx.x == 0) {
    DFloat t2[K];
    warp_tree8<K>(sh, t2);
#pragma unroll
    for (int c = 0; c < K; ++c) out[c] = (double)t2[c].hi + (double)t2[c].lo;
  }
}

// Block sum of K double-float values held in lane 0 of each warp (as
// DotAcc<float>::finish_df leaves them), written by thread 0 as this
// block's partials pf[c * MFTO_RED_SLOTS + blockIdx.x].
template <int K>
__device__ __forceinline__ void publish_block_df(const DFloat (&v)[K], float2* pf) {
  __shared__ float2 sh[K][MFTO_BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) sh[c][warp] = make_float2(v[c].hi, v[c].lo);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    DFloat t2[K];
    warp_tree8<K>(sh, t2);
#pragma unroll
    for (int c = 0; c < K; ++c)
      pf[c * MFTO_RED_SLOTS + blockIdx.x] = make_float2(t2[c].hi, t2[c].lo);
  }
}

// Pre-step of A(k): r.z and r.r of the current iterate from B(k-1)'s
// partials, the convergence and cap tests, beta.  par = k & 1.
struct ColPreCg2 {
  const float2* pb;   // B's partials: row 0 r.z, row 1 r.r
  int nb;             // B's blocks
  PcgScalars* s;
  int par;
  // the partials and (thread 0) the scalars, loaded together: one round trip
  struct State {
    PartialLoads<2> part;
    int done, k, maxit;
    double rtol2ff, rinv;
  };
  __device__ __forceinline__ State issue() const {
    State st;
    st.part = partials_load<2>(pb, nb);
    st.done = st.k = st.maxit = 0;
    st.rtol2ff = st.rinv = 0.0;
    if (threadIdx.x == 0) {
      st.done = *(const volatile int32_t*)&s->done;
      st.k = s->it2[par ^ 1] + 1;                   // iterations completed so far
      st.maxit = s->maxit;
      st.rtol2ff = s->rtol2ff;
      st.rinv = s->rinv2[par ^ 1];
    }
    return st;
  }
  template <typename Load>
  __device__ __forceinline__ bool run(Load& ld) const { return run(ld, issue()); }
  // thread 0 decides for the block and broadcasts through shared memory
  template <typename Load>
  __device__ __forceinline__ bool run(Load& ld, const State& st) const {
    __shared__ float s_beta;
    __shared__ int s_skip;
    const bool lead = threadIdx.x == 0;
    int done = st.done;
    const int k = st.k, maxit = st.maxit;
    const double rtol2ff = st.rtol2ff, rinv = st.rinv;
    double tot[2];
    partials_sum<2>(st.part, pb, nb, tot);
    if (lead) {
      double beta = 0.0;
      if (!done) {
        const double rz = tot[0], rr = tot[1];
        int status = MFTO_OK;
        if (!isfinite(rz) || !isfinite(rr)) {
          done = 1;
          status = MFTO_BREAKDOWN;
        } else if (rr <= rtol2ff) {
          done = 1;
        } else if (k >= maxit) {
          done = 1;
          status = MFTO_NOT_CONVERGED;
        } else {
          beta = rz * rinv;
        }
        if (blockIdx.x == 0) {
          s->rz2[par] = rz;
          s->it2[par] = k;
          s->it = k;
          s->rr = rr;
          s->beta = rz * rinv;
          s->rz = rz;
          if (done) {
            s->status = status;
            s->done = 1;
          }
        }
      }
      s_skip = done;
      s_beta = (float)beta;
    }
    __syncthreads();
    if (s_skip) return false;
    ld.beta = s_beta;
    return true;
  }
};

template <int MINB>
__global__ void __launch_bounds__(MFTO_BLOCK, MINB)
cg2_kv_kernel(const float* __restrict__ E, const float* __restrict__ z,
              const float* __restrict__ p_old, float* __restrict__ p_new, float* __restrict__ q,
              const uint8_t* __restrict__ fixed, ModeCoef<float> K, Grid g, ColTiling tl,
              PcgScalars* s, const double* part_b, int nb_b, double* part_a, int par) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DotAcc<float> acc;
  bool skipped = false;   // uniform over the grid
  acc.s = kv_column_body(E, fixed, K, g, tl, ColLoadDirection{z, p_old, 0.f}, ColPcg{p_new, q},
                         reinterpret_cast<float*>(smem_raw),
                         ColPreCg2{reinterpret_cast<const float2*>(part_b), nb_b, s, par},
                         &skipped);
  if (skipped) return;
  const DFloat w[1] = {acc.finish_df()};
  publish_block_df<1>(w, reinterpret_cast<float2*>(part_a));
}

// A(k) with the tensor-core column K.v (TF32 forms, kv_tcol.cuh).
template <bool SPLIT>
__global__ void __launch_bounds__(MFTO_BLOCK, 2)
cg2_kv_tcol_kernel(const float* __restrict__ E, const float* __restrict__ z,
                   const float* __restrict__ p_old, float* __restrict__ p_new,
                   float* __restrict__ q, const uint8_t* __restrict__ fixed,
                   const unsigned char* __restrict__ btile, Grid g, TcolTiling tl, PcgScalars* s,
                   const double* part_b, int nb_b, double* part_a, int par) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  DotAcc<float> acc;
  bool skipped = false;   // uniform over the grid
  acc.s = kv_tcol_body<TcolDefault, SPLIT>(
      E, fixed, btile, g, tl, ColLoadDirection{z, p_old, 0.f}, ColPcg{p_new, q}, smem,
      ColPreCg2{reinterpret_cast<const float2*>(part_b), nb_b, s, par}, &skipped, &s->tc_error);
  if (skipped) return;
  const DFloat w[1] = {acc.finish_df()};
  publish_block_df<1>(w, reinterpret_cast<float2*>(part_a));
}

// B(k): u += alpha p; r -= alpha q; z = r / d over groups of 4 DOFs
// (cg_update.cuh's per-group arithmetic); the first group's loads are
// issued before alpha is formed.
__global__ void __launch_bounds__(MFTO_BLOCK)
cg2_update_kernel(float* __restrict__ u, const float* __restrict__ p, const float* __restrict__ q,
                  float* __restrict__ r, float* __restrict__ z, const float* __restrict__ dinv,
                  int n, PcgScalars* s, const double* part_a, int nb_a, double* part_b,
                  int par) {
  const int n4 = n >> 2;
  const int first = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  float4* u4 = reinterpret_cast<float4*>(u);
  float4* r4 = reinterpret_cast<float4*>(r);
  float4* z4 = reinterpret_cast<float4*>(z);
  const float4* p4 = reinterpret_cast<const float4*>(p);
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const float4* d4 = reinterpret_cast<const float4*>(dinv);
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // the p.q partials go out first: the block's decision waits for them,
  // while the vector groups are only needed after it
  const float2* pa = reinterpret_cast<const float2*>(part_a);
  const PartialLoads<1> pl = partials_load<1>(pa, nb_a);
  float4 uu = zero4, pp = zero4, qq = zero4, rr = zero4, dd = zero4;
  if (first < n4) {
    uu = u4[first];
    pp = p4[first];
    qq = q4[first];
    rr = r4[first];
    dd = d4[first];
  }
  // the scalars go out with the partials' loads (one round trip for both);
  // thread 0 decides for the block, as in the K.v's pre-step
  __shared__ float s_alpha;
  __shared__ int s_skip;
  const bool lead = threadIdx.x == 0;
  int done = 0, it = 0;
  double rz = 0.0;
  if (lead) {
    done = *(const volatile int32_t*)&s->done;
    rz = s->rz2[par];
    it = s->it2[par];
  }
  double tot[1];
  partials_sum<1>(pl, pa, nb_a, tot);
  // the block's alpha goes out first; block 0 records the FP64 scalars
  // (alpha, the reciprocal of r.z for the next beta) after the broadcast,
  // off the other threads' path
  const bool was_done = done != 0;
  const double pq = tot[0];
  double alpha64 = 0.0;
  if (lead) {
    if (!done) {
      if (!(pq > 0.0) || !isfinite(pq))
        done = 1;
      else
        alpha64 = rz / pq;
    }
    s_skip = done;
    s_alpha = (float)alpha64;
  }
  __syncthreads();
  if (lead && blockIdx.x == 0 && !was_done) {
    s->pq = pq;
    if (done) {
      s->alpha = 0.0;
      s->status = MFTO_BREAKDOWN;
      s->done = 1;
    } else {
      s->alpha = alpha64;
      s->it = it + 1;
      s->rinv2[par] = 1.0 / rz;   // for the next beta
    }
  }
  if (s_skip) return;
  const float alpha = s_alpha;
  DotAcc<float> d0, d1;
  for (int i = first; i < n4; i += stride) {
    // the next group's loads go out before this group is computed
    const int nx = i + stride;
    float4 un = zero4, pn = zero4, qn = zero4, rn_ = zero4, dn = zero4;
    if (nx < n4) {
      un = u4[nx];
      pn = p4[nx];
      qn = q4[nx];
      rn_ = r4[nx];
      dn = d4[nx];
    }
    uu.x += alpha * pp.x; uu.y += alpha * pp.y; uu.z += alpha * pp.z; uu.w += alpha * pp.w;
    float4 rn, zn;
    rn.x = rr.x - alpha * qq.x; rn.y = rr.y - alpha * qq.y;
    rn.z = rr.z - alpha * qq.z; rn.w = rr.w - alpha * qq.w;
    zn.x = rn.x * dd.x; zn.y = rn.y * dd.y; zn.z = rn.z * dd.z; zn.w = rn.w * dd.w;
    u4[i] = uu;
    r4[i] = rn;
    z4[i] = zn;
    d0.add(dot4(rn, zn));
    d1.add(dot4(rn, rn));
    uu = un; pp = pn; qq = qn; rr = rn_; dd = dn;
  }
  // the n mod 4 trailing DOFs, by the threads whose first index is below n mod 4
  if (first < (n & 3)) {
    const int i = 4 * n4 + first;
    u[i] += alpha * p[i];
    const float ri = r[i] - alpha * q[i];
    const float zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    d0.add(ri * zi);
    d1.add(ri * ri);
  }
  const DFloat w[2] = {d0.finish_df(), d1.finish_df()};
  publish_block_df<2>(w, reinterpret_cast<float2*>(part_b));
}

// After pcg_init: B's partial rows hold the initial r.z and r.r in slot 0
// and zeros elsewhere (so A(0) sums exactly them), the reciprocal of the
// previous r.z is the continued direction's (or 0: beta = 0) and no
// iteration is complete.
__global__ void cg2_seed_kernel(PcgScalars* s, double* part_b, int nb_b, double rz_prev) {
  float2* pf = reinterpret_cast<float2*>(part_b);
  const double rz = s->rz, rr = s->rr;
  for (int b = threadIdx.x; b < nb_b; b += blockDim.x) {
    float2 a = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    if (b == 0) {
      const float rzh = (float)rz, rrh = (float)rr;
      a = make_float2(rzh, (float)(rz - (double)rzh));
      c = make_float2(rrh, (float)(rr - (double)rrh));
    }
    pf[b] = a;
    pf[MFTO_RED_SLOTS + b] = c;
  }
  if (threadIdx.x == 0) {
    s->rinv2[1] = rz_prev > 0.0 ? 1.0 / rz_prev : 0.0;
    s->it2[1] = -1;
  }
}

int update_blocks(const mfto_handle* h) {
  int64_t b = (h->n_dof / 4 + MFTO_BLOCK - 1) / MFTO_BLOCK;
  const int64_t cap = 4 * (int64_t)h->num_sms;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

bool cg2_active(const mfto_handle* h, int form) {
  return h->cg_engine == 2 && ((form == MFTO_FORM_F32 && h->kv_variant == 0) || tcol_form(form));
}

mfto_status cg2_attrs(mfto_handle* h) {
  const int csm = (int)kColSmem;
  MFTO_CUDA(h, cudaFuncSetAttribute(cg2_kv_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(cg2_kv_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(cg2_kv_tcol_kernel<false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, tcol_smem_bytes(2)));
  MFTO_CUDA(h, cudaFuncSetAttribute(cg2_kv_tcol_kernel<true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, tcol_smem_bytes(2)));
  return MFTO_OK;
}

mfto_status cg2_seed(mfto_handle* h, const PcgVecs<float>& v, double rz_prev) {
  h->launches++;
  cg2_seed_kernel<<<1, MFTO_BLOCK, 0, h->stream>>>(v.s, v.part_b, update_blocks(h), rz_prev);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

// One iteration (A then B) of engine 2 on stream st; par = iteration parity.
mfto_status cg2_enqueue(mfto_handle* h, cudaStream_t st, const PcgVecs<float>& v,
                        const float* p_old, float* p_new, int par, cudaEvent_t ev0,
                        cudaEvent_t ev1) {
  int grid = 0;
  const int kind = h->col_kind;
  const Grid g = make_grid(h->mesh);
  const int nb_b = update_blocks(h);
  if (ev0) MFTO_CUDA(h, cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal));
  if (tcol_form(v.form)) {
    const bool split = v.form == MFTO_FORM_TF32X3;
    const TcolTiling tt = tcol_launch_tiling(h, h->occ_tc[split ? 3 : 1], &grid);
    const size_t smt = tcol_smem_bytes(2);
    if (split)
      cg2_kv_tcol_kernel<true><<<grid, MFTO_BLOCK, smt, st>>>(
          v.E, v.z, p_old, p_new, v.q, h->d_fixed, h->d_btc, g, tt, v.s, v.part_b, nb_b,
          v.part_a, par);
    else
      cg2_kv_tcol_kernel<false><<<grid, MFTO_BLOCK, smt, st>>>(
          v.E, v.z, p_old, p_new, v.q, h->d_fixed, h->d_btc, g, tt, v.s, v.part_b, nb_b,
          v.part_a, par);
    if (ev1) MFTO_CUDA(h, cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal));
    cg2_update_kernel<<<nb_b, MFTO_BLOCK, 0, st>>>(v.u, p_new, v.q, v.r, v.z, v.dinv,
                                                   (int)h->n_dof, v.s, v.part_a, grid, v.part_b,
                                                   par);
    MFTO_LAUNCH_CHECK(h);
    return MFTO_OK;
  }
  const ColTiling tl = col_launch_tiling(h, h->occ_col[kind], &grid);
  const size_t sm = kColSmem;
  if (kind == 1)
    cg2_kv_kernel<3><<<grid, MFTO_BLOCK, sm, st>>>(v.E, v.z, p_old, p_new, v.q, h->d_fixed,
                                                   h->mc32, g, tl, v.s, v.part_b, nb_b, v.part_a,
                                                   par);
  else
    cg2_kv_kernel<2><<<grid, MFTO_BLOCK, sm, st>>>(v.E, v.z, p_old, p_new, v.q, h->d_fixed,
                                                   h->mc32, g, tl, v.s, v.part_b, nb_b, v.part_a,
                                                   par);
  if (ev1) MFTO_CUDA(h, cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal));
  cg2_update_kernel<<<nb_b, MFTO_BLOCK, 0, st>>>(v.u, p_new, v.q, v.r, v.z, v.dinv,
                                                 (int)h->n_dof, v.s, v.part_a, grid, v.part_b,
                                                 par);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

// A(k) alone, as cg2_enqueue issues it for the FP32 SIMT form (burst timing
// of the K.v launch, pcg.cu).
mfto_status cg2_enqueue_kv(mfto_handle* h, cudaStream_t st, const PcgVecs<float>& v,
                           const float* p_old, float* p_new, int par) {
  int grid = 0;
  const int kind = h->col_kind;
  const Grid g = make_grid(h->mesh);
  const int nb_b = update_blocks(h);
  const ColTiling tl = col_launch_tiling(h, h->occ_col[kind], &grid);
  if (kind == 1)
    cg2_kv_kernel<3><<<grid, MFTO_BLOCK, kColSmem, st>>>(v.E, v.z, p_old, p_new, v.q,
                                                         h->d_fixed, h->mc32, g, tl, v.s,
                                                         v.part_b, nb_b, v.part_a, par);
  else
    cg2_kv_kernel<2><<<grid, MFTO_BLOCK, kColSmem, st>>>(v.E, v.z, p_old, p_new, v.q,
                                                         h->d_fixed, h->mc32, g, tl, v.s,
                                                         v.part_b, nb_b, v.part_a, par);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

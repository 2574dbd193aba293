// Internal definitions shared by the library's translation units: the handle,
// error plumbing, deterministic block reductions and a bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/mfto.h"

// Mode-space coefficients for unit modulus; the 1/8 of the inverse transform
// is folded in.  diag[i][m]: out[i][m] += diag[i][m] in[i][m];
// lamM[t], muM[t]: off-diagonal couplings lam*M(t), mu*M(t) (t = mode bit of
// the remaining axis).  Applied by element_apply() in kv_tile.cuh.
template <typename T>
struct ModeCoef {
  T diag[3][8];
  T lamM[2], muM[2];
};

#define MFTO_BLOCK 256            // threads per block of the element/node kernels
#define MFTO_RED_MAX_BLOCKS 1024  // grid cap of the grid-stride vector kernels
#define MFTO_RED_SLOTS 16384      // partial-sum slots per row of one grid reduction
#define MFTO_PCG_SLOTS 2          // cached PCG graphs: FP64 solver, FP32 inner solver
#define MFTO_TC_BTILE 4096        // bytes of one tensor-core B operand (KE, one part)
#define MFTO_MAX_RHS 8            // load cases of the multi-RHS calls
#define MFTO_RED_ROWS 16          // rows of the partial-sum buffers (2 per load case)

// Device-resident scalars of the PCG driver and the other reductions.  Each
// reduction site owns a ticket counter (reset by the last block).
struct PcgScalars {
  double rz;        // r.z of the current iterate
  double pq;        // p.q
  double alpha, beta;
  double rr;        // r.r
  double ff;        // f.f
  double rtol2ff;   // rtol^2 * f.f
  int32_t it, maxit, done, status;
  unsigned int ticket_a, ticket_b, ticket_c;
  int32_t tc_error;         // a tensor-core or bulk-copy completion wait gave up
  int32_t bar_error;        // a grid-barrier wait of the persistent CG gave up
  // ticket-free FP32 CG (pcg_f32.cu): r.z, its reciprocal and the
  // completed-iteration count of iteration k in slot k & 1
  double rz2[2];
  double rinv2[2];
  int32_t it2[2];
};

// Scalars of the multi-RHS inner CG: one set per load case, plus the flag
// raised when every case is done.
struct MultiScalars {
  double rz[MFTO_MAX_RHS], pq[MFTO_MAX_RHS], alpha[MFTO_MAX_RHS], beta[MFTO_MAX_RHS];
  double rr[MFTO_MAX_RHS], ff[MFTO_MAX_RHS], rtol2ff[MFTO_MAX_RHS];
  int32_t done[MFTO_MAX_RHS], status[MFTO_MAX_RHS], it[MFTO_MAX_RHS];
  int32_t all_done, maxit, nrhs;
  unsigned int ticket_a, ticket_b, ticket_c;
  // column kernels (one grid row per case): per-case tickets, and the count
  // of cases done (the last case to finish raises all_done)
  unsigned int ticket_kv[MFTO_MAX_RHS], ticket_up[MFTO_MAX_RHS];
  int32_t ndone;
};

struct MiscScalars {
  double sum[4];            // results of small reductions
  double lambda, change, volume;
  int32_t oc_steps;
  int32_t oc_evals;         // candidate-volume evaluations (grid barriers) of the last OC
  int32_t oc_kstar;         // its first-phase index k* (the next call's starting guess)
  int32_t error;            // set by device code that gave up on a wait
  unsigned int ticket;
  unsigned int bar_count, bar_gen;
};

struct KvEventPool {
  std::vector<cudaEvent_t> start, stop;
  std::vector<int> form;      // form index (0 FP64, 1 FP32) of each recorded pair
  int used = 0;
  int64_t launches[2] = {0, 0};
  double total_ms[2] = {0.0, 0.0};
  // persistent CG launches (pcg_persist.cu): launches, CG iterations, device time
  int64_t cg_launches = 0, cg_iterations = 0;
  double cg_ms = 0.0;
  cudaEvent_t cg_start = nullptr, cg_stop = nullptr;
};

struct mfto_handle {
  mfto_mesh mesh;
  mfto_params p;
  int64_t n_elem, n_node, n_dof;
  cudaStream_t stream;
  cudaStream_t cap_stream;  // private stream used only to capture CUDA graphs
  int num_sms;
  // device copies of the unit element matrix (row-major 24x24)
  double* d_ke64;
  float* d_ke32;
  double ke_diag;           // KE[l][l] (equal for every local DOF on a cube)
  ModeCoef<double> mc64;    // mode-space element operator (kv_tile.cuh)
  ModeCoef<float> mc32;
  int kv_variant;           // 0: tiled mode-space kernel, 1: node-centric dense KE
  int cg_engine;            // FP32 inner CG: 0 two kernels per iteration, 1 persistent,
                            // 2 two ticket-free kernels per iteration
  int persist_grid;         // CTAs of the persistent CG launch (0: unavailable)
  int persist_tiling[4];    // its column tiling: tiles in x, y, z and node layers per chunk
  int occ_kv32, occ_pcg32;  // resident CTAs per SM of the FP32 block kernels
  int occ_col[2];           // ... of the FP32 column kernel kinds (kv_tile.cu)
  int col_nzc;              // node layers per z-chunk of the column kernels (0: automatic)
  int col_kind;             // column kernel kind (mfto_kv_autotune)
  int tcol_nzc;             // node layers per z-chunk of the tensor-core column kernel (0: automatic)
  unsigned int* d_bar;      // tree grid-barrier counters of the persistent CG (zeroed)
  int occ_tc[12];           // ... of the tensor-core kernels, [2 * (2 kind + split) + pcg]
  int occ_multi[3];         // ... of the multi-RHS kernels (F64 K.V, F32 K.V, F32 CG step)
  unsigned char* d_btc;     // tensor-core B operands: [kind][hi | lo]
  uint8_t* d_fixed;         // per-node mask
  // cone filter
  int32_t n_stencil;
  int32_t* d_stencil_off;   // [3 * n_stencil]
  double* d_stencil_w;      // [n_stencil]
  double* d_filter_W;       // row sums W_e
  // PCG workspace (FP64)
  double *d_r, *d_z, *d_p0, *d_p1, *d_q, *d_dinv;
  double* d_oc;             // [3][n_elem] OC bisection scratch (simp.cu)
  int oc_hint;              // k* of the previous OC update (0: none), simp.cu
  uint8_t* d_tile_fixed;    // column K.v xy tiles that stage a fixed node (kv_column.cuh)
  double* d_partials;       // [MFTO_RED_ROWS * MFTO_RED_SLOTS]
  double* d_partials2;      // [MFTO_RED_ROWS * MFTO_RED_SLOTS]
  PcgScalars* d_pcg;
  MiscScalars* d_misc;
  PcgScalars* h_pcg;        // pinned mirror
  MiscScalars* h_misc;      // pinned mirror
  // SIMP step workspace
  double *d_rho_phys, *d_E, *d_dc, *d_dc_phys;
  double *d_rho_bar, *d_rho_in;   // filtered field (projection on); design entering a step
  double proj_beta, proj_eta;     // Heaviside projection (beta = 0: off), mfto_set_projection
  // FP32 workspace of the inner solve of the iterative refinement
  float *d_r32, *d_z32, *d_p0_32, *d_p1_32, *d_q32, *d_dinv32, *d_e32, *d_E32;
  PcgScalars* d_pcg32;
  PcgScalars* h_pcg32;      // pinned mirror
  // multi-RHS workspace ([max_rhs][n_dof] each), allocated when max_rhs > 1
  int max_rhs;
  double* m_q64;
  float *m_r32, *m_z32, *m_p0, *m_p1, *m_q32, *m_e32;
  MultiScalars* m_pcg;
  MultiScalars* h_mpcg;     // pinned mirror
  double* m_out;            // [2 * MFTO_MAX_RHS] outer residual sums
  struct MultiGraph* m_graph;  // captured chunk of the multi-RHS inner CG
  // solver used by mfto_simp_step (mfto_set_solver)
  int32_t solver_form;      // MFTO_FORM_F64: plain FP64 PCG; else IR with this inner form
  double inner_tol;
  int32_t inner_maxit;
  int32_t max_outer;
  int32_t ir_mode;          // MFTO_IR_RESTART or MFTO_IR_CONTINUE (mfto_set_ir_mode)
  // learned solve (learned.cu): network, correction period and its buffers
  struct LearnedWs* learned;
  // geometric multigrid hierarchy and V-cycle solver (gmg.cu)
  struct GmgWs* gmg;
  // bytes of the workspace mfto_create allocated (mfto_device_bytes)
  int64_t ws_bytes;
  // PCG graph cache: one captured chunk of check_every iterations per solver
  struct PcgGraph* pcg_graph[MFTO_PCG_SLOTS];
  // kernels launched on behalf of this handle (graph kernel nodes included)
  int64_t launches;
  // timing
  bool kv_timing;
  KvEventPool ev;
  char msg[512];
};

// --------------------------------------------------------------- errors
mfto_status mfto_fail(mfto_handle* h, mfto_status code, const char* fmt, ...);

#define MFTO_CUDA(h, call)                                                   \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return mfto_fail((h), MFTO_CUDA_ERROR, "%s: %s (%s:%d)", #call,        \
                       cudaGetErrorString(e_), __FILE__, __LINE__);          \
  } while (0)

#define MFTO_LAUNCH_CHECK(h) MFTO_CUDA(h, cudaGetLastError())

#define MFTO_REQUIRE(h, cond, msg)                                           \
  do {                                                                       \
    if (!(cond)) return mfto_fail((h), MFTO_INVALID_ARG, "%s", msg);        \
  } while (0)

// --------------------------------------------------------- index helpers
struct Grid {
  int nelx, nely, nelz;   // elements
  int nx, ny, nz;         // nodes per axis (nel + 1)
};

static inline Grid make_grid(const mfto_mesh& m) {
  Grid g;
  g.nelx = m.nelx; g.nely = m.nely; g.nelz = m.nelz;
  g.nx = m.nelx + 1; g.ny = m.nely + 1; g.nz = m.nelz + 1;
  return g;
}

static inline int reduction_blocks(int64_t n, int block) {
  int64_t b = (n + block - 1) / block;
  if (b > MFTO_RED_MAX_BLOCKS) b = MFTO_RED_MAX_BLOCKS;
  if (b < 1) b = 1;
  return (int)b;
}

// ----------------------------------------------------- device reductions
// Sum of one double over the block in a fixed order (warp shuffles, then
// warp 0 over the per-warp sums).  The result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (warp == 0) {
    v = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Sum over the warps of values that live in lane 0 of each warp (every other
// lane's value is ignored): the per-warp results of DotAcc<float>::finish.
// One FP64 add per warp instead of a shuffle tree over every lane (the FP64
// pipe is narrow).  The result is valid in thread 0; fixed order.
__device__ __forceinline__ double block_sum_w0(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) t += sh[w];
  }
  return t;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (warp == 0) {
    v = lane < nw ? sh[lane] : -1.0e300;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  }
  return v;
}

// Dot-product accumulators.  FP64 vectors accumulate in FP64.  FP32 vectors
// accumulate in double-float (an unevaluated sum hi + lo of two FP32 values,
// ~48-bit significand): each product is split exactly with an FMA
// (TwoProduct), sums use TwoSum, a warp combines its 32 pairs with shuffles,
// and only then is the pair converted to FP64 for the block and grid sums.
// On this GPU the FP64 pipe, conversions included, runs at a small fraction
// of the FP32 rate, so one conversion per warp instead of one FP64
// operation per term keeps the reductions off the critical path without
// giving up FP64-level accuracy.
struct DFloat {
  float hi, lo;
};

__device__ __forceinline__ DFloat df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float err = (a - (s - bb)) + (b - bb);
  return {s, err};
}

__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b) {
  DFloat s = df_two_sum(a.hi, b.hi);
  const float lo = s.lo + a.lo + b.lo;
  const float hi = s.hi + lo;
  return {hi, lo - (hi - s.hi)};
}

__device__ __forceinline__ DFloat df_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

template <typename T>
struct DotAcc;

template <>
struct DotAcc<double> {
  static constexpr bool kWarpReduced = false;   // finish(): one partial per thread
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s += a * b; }
  // every thread returns its own FP64 partial
  __device__ __forceinline__ double finish() const { return s; }
};

template <>
struct DotAcc<float> {
  static constexpr bool kWarpReduced = true;    // finish(): one partial per warp (lane 0)
  DFloat s{0.f, 0.f};
  __device__ __forceinline__ void add_prod(float a, float b) { s = df_add(s, df_prod(a, b)); }
  // adds one FP32 value (e.g. a short FP32 sum of products)
  __device__ __forceinline__ void add(float t) { s = df_add(s, DFloat{t, 0.f}); }
  // must be called by all 32 lanes of the warp: lane 0 returns the warp's
  // sum as a double-float pair (the other lanes hold partial sums)
  __device__ __forceinline__ DFloat finish_df() const {
    DFloat v = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      DFloat w;
      w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
      w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
      v = df_add(v, w);
    }
    return v;
  }
  // as finish_df, converted to FP64 by lane 0 alone (the other lanes return
  // 0 and execute no FP64 instruction: the FP64 pipe is 1/64 of FP32 here)
  __device__ __forceinline__ double finish() const {
    const DFloat v = finish_df();
    double r = 0.0;
    if ((threadIdx.x & 31) == 0) r = (double)v.hi + (double)v.lo;
    return r;
  }
};

// Block sum of double-float values that live in lane 0 of each warp; the
// result is valid in thread 0 (FP32 arithmetic only).  sh: 32 float2.
__device__ __forceinline__ DFloat block_sum_df(DFloat v, float2* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = make_float2(v.hi, v.lo);
  __syncthreads();
  DFloat t{0.f, 0.f};
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) t = df_add(t, DFloat{sh[w].x, sh[w].y});
  }
  return t;
}

// last_block_reduce for FP32 dot products held as double-float pairs in lane
// 0 of each warp (DotAcc<float>::finish_df): block partials are published as
// pairs, and the last block sums them with warp 0 in double-float, in block
// order, converting to FP64 once per total.  No FP64 instruction runs outside
// that conversion.  out[0..K) is valid in every thread of the last block.
template <int K>
__device__ __forceinline__ bool last_block_reduce_df(const DFloat (&v)[K], double* partials,
                                                     unsigned int* ticket, double* out,
                                                     double* sh) {
  __shared__ bool s_last;
  float2* shf = reinterpret_cast<float2*>(sh);          // [0, 32): warp values
  float2* pf = reinterpret_cast<float2*>(partials);     // one pair per double slot
  const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
  const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  DFloat bs[K];
#pragma unroll
  for (int c = 0; c < K; ++c) bs[c] = block_sum_df(v[c], shf);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) pf[c * MFTO_RED_SLOTS + bid] = make_float2(bs[c].hi, bs[c].lo);
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == nb - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      DFloat t{0.f, 0.f};
      for (int b = threadIdx.x; b < (int)nb; b += 32) {
        const float2 x = __ldcg(&pf[c * MFTO_RED_SLOTS + b]);
        t = df_add(t, DFloat{x.x, x.y});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        DFloat w;
        w.hi = __shfl_down_sync(0xffffffffu, t.hi, o);
        w.lo = __shfl_down_sync(0xffffffffu, t.lo, o);
        t = df_add(t, w);
      }
      if (threadIdx.x == 0) sh[32 + c] = (double)t.hi + (double)t.lo;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < K; ++c) out[c] = sh[32 + c];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// last_block_reduce_df over the blocks of one grid row (blockIdx.y fixed):
// bid = blockIdx.x among gridDim.x blocks, the row's own partial rows and
// ticket.  Used where each grid row is an independent problem (a load case).
template <int K>
__device__ __forceinline__ bool row_reduce_df(const DFloat (&v)[K], double* partials,
                                              unsigned int* ticket, double* out, double* sh) {
  __shared__ bool s_last;
  float2* shf = reinterpret_cast<float2*>(sh);
  float2* pf = reinterpret_cast<float2*>(partials);
  const unsigned int nb = gridDim.x, bid = blockIdx.x;
  DFloat bs[K];
#pragma unroll
  for (int c = 0; c < K; ++c) bs[c] = block_sum_df(v[c], shf);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) pf[c * MFTO_RED_SLOTS + bid] = make_float2(bs[c].hi, bs[c].lo);
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == nb - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      DFloat t{0.f, 0.f};
      for (int b = threadIdx.x; b < (int)nb; b += 32) {
        const float2 x = __ldcg(&pf[c * MFTO_RED_SLOTS + b]);
        t = df_add(t, DFloat{x.x, x.y});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        DFloat w;
        w.hi = __shfl_down_sync(0xffffffffu, t.hi, o);
        w.lo = __shfl_down_sync(0xffffffffu, t.lo, o);
        t = df_add(t, w);
      }
      if (threadIdx.x == 0) sh[32 + c] = (double)t.hi + (double)t.lo;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < K; ++c) out[c] = sh[32 + c];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// A solver's done flag and one FP64 scalar, read in a single round trip by
// thread 0 (the scalar converted to FP32 there) and broadcast through shared
// memory: *done_out and the returned value are the same in every thread.
// Call once per kernel, before anything else uses shared memory.
__device__ __forceinline__ float flag_and_scalar_f32(const int32_t* done, const double* p,
                                                     int* done_out) {
  __shared__ float s_val;
  __shared__ int s_done;
  if (threadIdx.x == 0) {
    const int d = *(const volatile int32_t*)done;
    const double v = *p;
    s_done = d;
    s_val = (float)v;
  }
  __syncthreads();
  *done_out = s_done;
  return s_val;
}


// Publish K per-block partial sums and let the last block to arrive reduce
// them in block-index order.  Returns true in every thread of that last
// block, with out[0..K) holding the totals (valid in all its threads).
// W0: the values live in lane 0 of each warp only (DotAcc<float>::finish),
// so the block stage sums the warps' values instead of every lane's.
template <int K, bool W0 = false>
__device__ __forceinline__ bool last_block_reduce(const double (&v)[K],
                                                  double* partials,
                                                  unsigned int* ticket,
                                                  double* out, double* sh) {
  // partials: K rows of MFTO_RED_SLOTS slots; the grid (any shape) must not
  // have more than MFTO_RED_SLOTS blocks.
  __shared__ bool s_last;
  const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
  const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  double bs[K];
#pragma unroll
  for (int c = 0; c < K; ++c) bs[c] = W0 ? block_sum_w0(v[c], sh) : block_sum(v[c], sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) partials[c * MFTO_RED_SLOTS + bid] = bs[c];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == nb - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
#pragma unroll
  for (int c = 0; c < K; ++c) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)nb; b += blockDim.x)
      s += __ldcg(&partials[c * MFTO_RED_SLOTS + b]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) sh[32 + c] = s;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < K; ++c) out[c] = sh[32 + c];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Sum of K doubles over the block in a fixed order; every thread receives
// the totals.  sh must hold 8 K doubles (256 threads).
template <int K>
__device__ __forceinline__ void block_allsum(double (&v)[K], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  __syncthreads();
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh[w * K + k];
    v[k] = t;
  }
}

// Totals of K partial rows (G entries each), identical in every thread of
// every CTA.
template <int K>
__device__ __forceinline__ void grid_allsum(const double* part, int G, double (&out)[K],
                                            double* sh) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) t += __ldcg(part + k * MFTO_RED_SLOTS + b);
    out[k] = t;
  }
  block_allsum<K>(out, sh);
}

// Grid-wide barrier for a cooperative launch.  Every wait is bounded: after
// MFTO_SPIN_LIMIT polls the block sets *error and stops waiting; once *error
// is set no later barrier waits at all, so the kernel always terminates.
#define MFTO_SPIN_LIMIT (1u << 24)
__device__ __forceinline__ void grid_barrier(unsigned int* count,
                                             unsigned int* gen,
                                             int32_t* error) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = gen;
    volatile int32_t* verr = error;
    const unsigned int g = *vgen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      *count = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned int spins = 0;
      while (*vgen == g) {
        if (*verr) break;
        if (++spins > MFTO_SPIN_LIMIT) { atomicExch(error, 1); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Release-add and acquire-load of a global counter (grid barriers that count
// arrivals: each block adds 1 and waits until the count reaches the number
// of arrivals expected so far).
__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------------ host-side entries
// (defined in the .cu files, used across them)
mfto_status kv_launch(mfto_handle* h, mfto_form form, const void* E,
                      const void* v, void* y);
mfto_status diag_launch(mfto_handle* h, mfto_form form, const void* E,
                        void* diag, bool inverse);
mfto_status modulus_launch(mfto_handle* h, mfto_form form,
                           const double* rho_phys, void* E);
mfto_status filter_launch(mfto_handle* h, const double* x, double* y,
                          int transpose);
mfto_status filter_setup(mfto_handle* h);
bool projection_active(const mfto_handle* h);
mfto_status project_launch(mfto_handle* h, const double* rho_bar, double* rho_phys);
mfto_status project_chain_launch(mfto_handle* h, const double* rho_bar, double* dc);
mfto_status compliance_launch(mfto_handle* h, const double* rho_phys,
                              const double* u, double* dc, double* c_out,
                              double* gray_out);
mfto_status oc_launch(mfto_handle* h, const double* rho, const double* dc,
                      double* rho_new, mfto_iter_stats* st);
mfto_status pcg_run(mfto_handle* h, const double* E, const double* f,
                    double* u, mfto_solve_stats* st);
mfto_status ir_run(mfto_handle* h, mfto_form inner, double inner_tol, const double* E,
                   const double* f, double* u, mfto_ir_stats* st);

// The vectors of one PCG solve (see pcg.cu).
template <typename T>
struct PcgVecs {
  const T* E;
  T *u, *r, *z, *p0, *p1, *q, *dinv;
  PcgScalars* s;
  double *part_a, *part_b;
  int form;                 // K.v form of this solve
};
mfto_status learned_run(mfto_handle* h, const double* E, const double* rho_phys, const double* f,
                        double* u, mfto_learned_stats* st);
bool learned_active(const mfto_handle* h);
void learned_release(mfto_handle* h);
bool gmg_active(const mfto_handle* h);
mfto_status gmg_sweep_col_launch(mfto_handle* h, bool first, const float* E, const float* b,
                                 const float* dinv, float omega, const float* x, float* xo,
                                 float* t);
// Multigrid Chebyshev launches fused into the FP32 column K.v (kv_tile.cu).
enum { GMG_CHEB_FIRST = 0, GMG_CHEB_BEGIN = 1, GMG_CHEB_STEP = 2 };
mfto_status gmg_cheb_col_launch(mfto_handle* h, int mode, const float* E, const float* in,
                                const float* b, const float* dinv, float inv_theta, float c1,
                                float c2, float* r, float* dn, const float* x, float* xo);
int64_t gmg_bytes(const mfto_handle* h);
int64_t learned_bytes(const mfto_handle* h);
void gmg_release(mfto_handle* h);
mfto_status gmg_solve(mfto_handle* h, const double* E, const double* f, double* u,
                      mfto_solve_stats* st);
void mode_coefficients(double nu, double h, ModeCoef<double>* c64, ModeCoef<float>* c32);
mfto_status tc_init(mfto_handle* h);
mfto_status multi_init(mfto_handle* h);
void multi_graph_release(mfto_handle* h);
mfto_status tc_upload_b(mfto_handle* h, const double* ke);
bool tc_form(int form);
mfto_status kv_tc_launch(mfto_handle* h, int form, const float* E, const float* v, float* y,
                         cudaStream_t st);
mfto_status pcg_kv_tc_launch(mfto_handle* h, int form, const float* E, const float* z,
                             const float* p_old, float* p_new, float* q, PcgScalars* s,
                             double* partials, cudaStream_t st);
template <typename T>
mfto_status pcg_start(mfto_handle* h, const PcgVecs<T>& v, const T* rhs, const T* Ku, double rtol,
                      int maxit, double rz_prev = 0.0);
template <typename T>
mfto_status pcg_iterate(mfto_handle* h, const PcgVecs<T>& v, int slot, PcgScalars* host_s);
void pcg_graph_release(mfto_handle* h);
mfto_status pcg_time_iterations(mfto_handle* h, int chunks, float* us_per_iter);
mfto_status pcg_persist_init(mfto_handle* h);
// ticket-free FP32 CG, engine 2 (pcg_f32.cu)
bool cg2_active(const mfto_handle* h, int form);
mfto_status cg2_attrs(mfto_handle* h);
mfto_status cg2_seed(mfto_handle* h, const PcgVecs<float>& v, double rz_prev);
mfto_status cg2_enqueue_kv(mfto_handle* h, cudaStream_t st, const PcgVecs<float>& v,
                           const float* p_old, float* p_new, int par);
mfto_status cg2_enqueue(mfto_handle* h, cudaStream_t st, const PcgVecs<float>& v,
                        const float* p_old, float* p_new, int par, cudaEvent_t ev0,
                        cudaEvent_t ev1);
mfto_status pcg_persist_iterate(mfto_handle* h, const PcgVecs<float>& v, PcgScalars* host_s);
mfto_status kv_tile_init(mfto_handle* h);
template <typename T>
mfto_status kv_tile_launch(mfto_handle* h, const T* E, const T* v, T* y, cudaStream_t st);
template <typename T>
mfto_status pcg_kv_tile_launch(mfto_handle* h, const T* E, const T* z, const T* p_old, T* p_new,
                               T* q, PcgScalars* s, double* partials, cudaStream_t st);
void kv_timing_begin(mfto_handle* h, int form);
void kv_timing_end(mfto_handle* h);
mfto_status kv_timing_harvest(mfto_handle* h, bool sync);

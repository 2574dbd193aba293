// Many independent problems of uneven size (structured meshes of their own
// dimensions) solved together: every step of the mixed-precision solve is
// one persistent launch over all instances, and the inner CG chunks are
// captured into one CUDA graph.
//
// Work list: each instance is cut into element blocks (BX x BY x BZ elements,
// the owned nodes are the (BX-1) x (BY-1) x (BZ-1) interior); the blocks of
// all instances are numbered consecutively, instance by instance.  A
// persistent grid (resident CTAs x SMs) walks this list; a CTA maps a global
// block number to its instance by binary search over the instances' first
// block numbers.  Per-instance sums (CG dot products, residual norms) are
// formed per block and reduced per instance, in block order, by the last CTA
// to finish -- deterministic and without atomics on the data.
//
// The block shape is a template parameter; mfto_batch_autotune times the
// candidates on the batch itself and keeps the fastest.
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "kv_tile.cuh"

#define MFTO_BATCH_MAX 256
#define MFTO_BATCH_SHAPES 4

struct BatchInst {
  int nelx, nely, nelz, nx, ny, nz;
  long long elem_off, node_off;
  int kv_blk0, kv_nblk;      // element blocks in the K.V work list (current shape)
  int up_blk0, up_nblk;      // node blocks of the vector kernels
};

struct BatchScal {
  double rz, pq, alpha, beta, rr, ff, rtol2ff;
  int32_t it, done, status, pad;
};

struct BatchCtl {
  int32_t count, all_done, maxit, pad;
  unsigned int ticket_a, ticket_b, ticket_c, ticket_d;
};

struct BatchGraph {
  int chunk = 0;
  int shape = -1;
  cudaGraphExec_t exec = nullptr;
};

struct mfto_batch {
  int count;
  mfto_params p;
  double h;
  cudaStream_t stream, cap_stream;
  int num_sms;
  std::vector<mfto_mesh> meshes;
  std::vector<long long> elem_off, node_off;
  long long n_elem, n_node, n_dof;
  int shape;
  int kv_total[MFTO_BATCH_SHAPES];
  int up_total;
  int occ_kv64[MFTO_BATCH_SHAPES], occ_kv32[MFTO_BATCH_SHAPES], occ_pcg[MFTO_BATCH_SHAPES];
  BatchInst* d_inst[MFTO_BATCH_SHAPES];
  uint8_t* d_fixed;
  ModeCoef<double> mc64;
  ModeCoef<float> mc32;
  double ke_diag;
  float *r32, *z32, *p0, *p1, *q32, *e32, *dinv32, *E32;
  double* q64;
  BatchScal* d_scal;
  BatchScal* h_scal;
  BatchCtl* d_ctl;
  BatchCtl* h_ctl;
  double *d_part_a, *d_part_b;     // [2][max blocks]
  double* d_res;                   // [2 * count] outer residual sums
  int* d_mask;                     // [count] 1 = instance converged/stopped
  double* d_rzp;                   // [count] r.z of a continued direction (0: p = z)
  int ir_mode;                     // MFTO_IR_RESTART or MFTO_IR_CONTINUE
  BatchGraph* graph;
  int64_t launches;
  char msg[512];
};

namespace {

template <int S>
struct Shape;
template <> struct Shape<0> { static constexpr int BX = 8, BY = 8, BZ = 4; };
template <> struct Shape<1> { static constexpr int BX = 8, BY = 4, BZ = 8; };
template <> struct Shape<2> { static constexpr int BX = 4, BY = 8, BZ = 8; };
template <> struct Shape<3> { static constexpr int BX = 16, BY = 4, BZ = 4; };

template <int S>
struct ShapeDims {
  static constexpr int BX = Shape<S>::BX, BY = Shape<S>::BY, BZ = Shape<S>::BZ;
  static constexpr int VX = BX + 1, VY = BY + 1, VZ = BZ + 1;
  static constexpr int NV = VX * VY * VZ;
  static constexpr int OX = BX - 1, OY = BY - 1, OZ = BZ - 1;
  static constexpr int NO = OX * OY * OZ;
  static_assert(BX * BY * BZ == MFTO_BLOCK, "one element per thread");
  static_assert(NO <= MFTO_BLOCK, "owned nodes per block");
};

int shape_blocks(int s, int nx, int ny, int nz) {
  static const int O[MFTO_BATCH_SHAPES][3] = {{7, 7, 3}, {7, 3, 7}, {3, 7, 7}, {15, 3, 3}};
  return ((nx + O[s][0] - 1) / O[s][0]) * ((ny + O[s][1] - 1) / O[s][1]) *
         ((nz + O[s][2] - 1) / O[s][2]);
}

template <typename T>
size_t batch_smem() { return sizeof(T) * (3 * 512 + 24 * MFTO_BLOCK) + 512; }

// instance holding global block gb (first[] ascending, first[0] = 0)
__device__ __forceinline__ int find_inst(const int* first, int count, int gb) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= gb) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One element block of one instance (pointers already offset to it).
template <typename T, int S, typename Ld, typename Epi>
__device__ __forceinline__ void batch_block(const T* __restrict__ E, const uint8_t* __restrict__ fixed,
                                            const ModeCoef<T>& K, const BatchInst& in, int lb,
                                            const Ld& ld, const Epi& epi, T* smem,
                                            DotAcc<T>& red) {
  using D = ShapeDims<S>;
  T* vs = smem;                                                     // [3][512]
  T* out = vs + 3 * 512;                                            // [24][256]
  uint8_t* ms = reinterpret_cast<uint8_t*>(out + 24 * MFTO_BLOCK);  // [512]
  const int tid = threadIdx.x;
  const int tx = (in.nx + D::OX - 1) / D::OX, ty = (in.ny + D::OY - 1) / D::OY;
  const int bx = lb % tx, by = (lb / tx) % ty, bz = lb / (tx * ty);
  const int ox = bx * D::OX, oy = by * D::OY, oz = bz * D::OZ;
  for (int idx = tid; idx < D::NV; idx += MFTO_BLOCK) {
    const int lx = idx % D::VX, ly = (idx / D::VX) % D::VY, lz = idx / (D::VX * D::VY);
    const int gi = ox - 1 + lx, gj = oy - 1 + ly, gk = oz - 1 + lz;
    T a = 0, b = 0, c = 0;
    uint8_t fm = 0;
    if (gi >= 0 && gj >= 0 && gk >= 0 && gi < in.nx && gj < in.ny && gk < in.nz) {
      const int node = gi + in.nx * (gj + in.ny * gk);
      fm = fixed[node];
      a = ld(3 * node + 0);
      b = ld(3 * node + 1);
      c = ld(3 * node + 2);
      a = (fm & 1) ? T(0) : a;
      b = (fm & 2) ? T(0) : b;
      c = (fm & 4) ? T(0) : c;
    }
    vs[idx] = a;
    vs[512 + idx] = b;
    vs[1024 + idx] = c;
    ms[idx] = fm;
  }
  const int ex = tid % D::BX, ey = (tid / D::BX) % D::BY, ez = tid / (D::BX * D::BY);
  const int ei = ox - 1 + ex, ej = oy - 1 + ey, ek = oz - 1 + ez;
  T Ee = 0;
  if (ei >= 0 && ej >= 0 && ek >= 0 && ei < in.nelx && ej < in.nely && ek < in.nelz)
    Ee = E[ei + in.nelx * (ej + in.nely * ek)];
  __syncthreads();
  {
    T x[3][8];
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int vi = (ex + (l & 1)) + D::VX * ((ey + ((l >> 1) & 1)) + D::VY * (ez + (l >> 2)));
      x[0][l] = vs[vi];
      x[1][l] = vs[512 + vi];
      x[2][l] = vs[1024 + vi];
    }
    element_apply<T>(x, Ee, K);
#pragma unroll
    for (int l = 0; l < 8; ++l)
#pragma unroll
      for (int c = 0; c < 3; ++c) out[(3 * l + c) * MFTO_BLOCK + tid] = x[c][l];
  }
  __syncthreads();
  if (tid < D::NO) {
    const int ix = tid % D::OX, iy = (tid / D::OX) % D::OY, iz = tid / (D::OX * D::OY);
    const int gi = ox + ix, gj = oy + iy, gk = oz + iz;
    if (gi < in.nx && gj < in.ny && gk < in.nz) {
      T acc[3] = {0, 0, 0};
#pragma unroll
      for (int ec = 0; ec < 2; ++ec)
#pragma unroll
        for (int eb = 0; eb < 2; ++eb)
#pragma unroll
          for (int ea = 0; ea < 2; ++ea) {
            const int e = (ix + ea) + D::BX * ((iy + eb) + D::BY * (iz + ec));
            const int corner = (1 - ea) + 2 * (1 - eb) + 4 * (1 - ec);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] += out[(3 * corner + c) * MFTO_BLOCK + e];
          }
      const int vi = (ix + 1) + D::VX * ((iy + 1) + D::VY * (iz + 1));
      const T pn[3] = {vs[vi], vs[512 + vi], vs[1024 + vi]};
      epi(gi + in.nx * (gj + in.ny * gk), acc, pn, ms[vi], red);
    }
  }
  __syncthreads();
}

// Per-instance totals of per-block partials (rows of NR values, blocks
// [blk0, blk0 + nblk) of each instance): one warp per instance, lanes stride
// the blocks, shuffle tree -- a fixed order.
template <int NR>
__device__ __forceinline__ void per_instance_sums(const double* part, int stride,
                                                  const BatchInst* inst, int count, bool kv,
                                                  double* tot /* [count][NR] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < count; i += blockDim.x >> 5) {
    const int b0 = kv ? inst[i].kv_blk0 : inst[i].up_blk0;
    const int nb = kv ? inst[i].kv_nblk : inst[i].up_nblk;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double s = 0.0;
      for (int b = lane; b < nb; b += 32) s += __ldcg(&part[r * stride + b0 + b]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) tot[i * NR + r] = s;
    }
  }
}

__device__ __forceinline__ bool batch_last_cta(unsigned int* ticket) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// plain batched K.V (the outer FP64 residual, the autotuner's timing)
template <typename T, int S>
__global__ void __launch_bounds__(MFTO_BLOCK)
batch_kv_kernel(const T* __restrict__ E, const T* __restrict__ V, T* __restrict__ Y,
                const uint8_t* __restrict__ fixed, ModeCoef<T> K, const BatchInst* __restrict__ inst,
                int count, int total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int first[MFTO_BATCH_MAX];
  for (int i = threadIdx.x; i < count; i += blockDim.x) first[i] = inst[i].kv_blk0;
  __syncthreads();
  for (int gb = blockIdx.x; gb < total; gb += gridDim.x) {
    const int i = find_inst(first, count, gb);
    const BatchInst in = inst[i];
    const T* Ei = E + in.elem_off;
    const T* Vi = V + 3 * in.node_off;
    T* Yi = Y + 3 * in.node_off;
    DotAcc<T> red;
    batch_block<T, S>(Ei, fixed + in.node_off, K, in, gb - in.kv_blk0, TileLoadPlain<T>{Vi},
                      TileStore<T>{Vi, Yi}, reinterpret_cast<T*>(smem_raw), red);
  }
}

// inner CG step A over all live instances
template <int S>
__global__ void __launch_bounds__(MFTO_BLOCK)
batch_pcg_kv(const float* __restrict__ E, const float* __restrict__ Z, const float* __restrict__ P0,
             float* __restrict__ P1, float* __restrict__ Q, const uint8_t* __restrict__ fixed,
             ModeCoef<float> K, const BatchInst* __restrict__ inst, BatchScal* sc, BatchCtl* ctl,
             double* part, int total) {
  if (*(volatile int32_t*)&ctl->all_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int first[MFTO_BATCH_MAX];
  __shared__ double sh[64];
  const int count = ctl->count;
  for (int i = threadIdx.x; i < count; i += blockDim.x) first[i] = inst[i].kv_blk0;
  __syncthreads();
  for (int gb = blockIdx.x; gb < total; gb += gridDim.x) {
    const int i = find_inst(first, count, gb);
    const BatchInst in = inst[i];
    double pq = 0.0;
    if (!sc[i].done) {                       // uniform over the CTA
      const float beta = (float)sc[i].beta;
      const long long o = 3 * in.node_off;
      DotAcc<float> red;
      batch_block<float, S>(E + in.elem_off, fixed + in.node_off, K, in, gb - in.kv_blk0,
                            TileLoadDirection<float>{Z + o, P0 + o, beta},
                            TilePcg<float>{P1 + o, Q + o}, reinterpret_cast<float*>(smem_raw), red);
      pq = block_sum_w0(red.finish(), sh);
    }
    if (threadIdx.x == 0) part[gb] = pq;
  }
  if (batch_last_cta(&ctl->ticket_b)) {
    __shared__ double tot[MFTO_BATCH_MAX];
    per_instance_sums<1>(part, 0, inst, count, true, tot);
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
      if (sc[i].done) continue;
      sc[i].pq = tot[i];
      if (!(tot[i] > 0.0) || !isfinite(tot[i])) {
        sc[i].done = 1;
        sc[i].status = MFTO_BREAKDOWN;
        sc[i].alpha = 0.0;
      } else {
        sc[i].alpha = sc[i].rz / tot[i];
      }
    }
    if (threadIdx.x == 0) ctl->ticket_b = 0u;
  }
}

// node-block walk of the vector kernels: calls f(i, node) for each node
template <typename F>
__device__ __forceinline__ void for_instance_nodes(const int* first, const BatchInst* inst,
                                                   int count, int gb, const F& f) {
  const int i = find_inst(first, count, gb);
  const BatchInst& in = inst[i];
  const int n_node = in.nx * in.ny * in.nz;
  const int local = (gb - in.up_blk0) * MFTO_BLOCK + threadIdx.x;
  f(i, local < n_node ? in.node_off + local : -1LL);
}

// inner CG step B over all live instances
__global__ void __launch_bounds__(MFTO_BLOCK)
batch_update(float* __restrict__ U, const float* __restrict__ P, const float* __restrict__ Q,
             float* __restrict__ R, float* __restrict__ Z, const float* __restrict__ dinv,
             const BatchInst* __restrict__ inst, BatchScal* sc, BatchCtl* ctl, double* part,
             int total, int stride) {
  if (*(volatile int32_t*)&ctl->all_done) return;
  __shared__ int first[MFTO_BATCH_MAX];
  __shared__ double sh[64];
  const int count = ctl->count;
  for (int i = threadIdx.x; i < count; i += blockDim.x) first[i] = inst[i].up_blk0;
  __syncthreads();
  for (int gb = blockIdx.x; gb < total; gb += gridDim.x) {
    DotAcc<float> d0, d1;
    int inst_i = 0;
    for_instance_nodes(first, inst, count, gb, [&](int i, long long node) {
      inst_i = i;
      if (node < 0 || sc[i].done) return;
      const float alpha = (float)sc[i].alpha;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long k = 3 * node + c;
        U[k] += alpha * P[k];
        const float ri = R[k] - alpha * Q[k];
        const float zi = ri * dinv[k];
        R[k] = ri;
        Z[k] = zi;
        d0.add_prod(ri, zi);
        d1.add_prod(ri, ri);
      }
    });
    (void)inst_i;
    const double a = block_sum_w0(d0.finish(), sh);
    const double b = block_sum_w0(d1.finish(), sh);
    if (threadIdx.x == 0) {
      part[gb] = a;
      part[stride + gb] = b;
    }
  }
  if (batch_last_cta(&ctl->ticket_c)) {
    __shared__ double tot[2 * MFTO_BATCH_MAX];
    per_instance_sums<2>(part, stride, inst, count, false, tot);
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
      BatchScal& s = sc[i];
      if (s.done) continue;
      s.it += 1;
      s.rr = tot[2 * i + 1];
      s.beta = tot[2 * i] / s.rz;
      s.rz = tot[2 * i];
      if (!isfinite(tot[2 * i]) || !isfinite(tot[2 * i + 1])) {
        s.done = 1;
        s.status = MFTO_BREAKDOWN;
      } else if (tot[2 * i + 1] <= s.rtol2ff) {
        s.done = 1;
        s.status = MFTO_OK;
      } else if (s.it >= ctl->maxit) {
        s.done = 1;
        s.status = MFTO_NOT_CONVERGED;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int all = 1;
      for (int i = 0; i < count; ++i) all &= sc[i].done;
      ctl->all_done = all;
      ctl->ticket_c = 0u;
    }
  }
}

// inner solve start: r = rhs (in place), z = r / d, r.z and r.r per instance
__global__ void __launch_bounds__(MFTO_BLOCK)
batch_init(float* R, float* __restrict__ Z, const float* __restrict__ dinv,
           const BatchInst* __restrict__ inst, BatchScal* sc, BatchCtl* ctl, double* part,
           int total, int stride, double rtol, int maxit, int count,
           const double* __restrict__ rz_prev) {
  __shared__ int first[MFTO_BATCH_MAX];
  __shared__ double sh[64];
  for (int i = threadIdx.x; i < count; i += blockDim.x) first[i] = inst[i].up_blk0;
  __syncthreads();
  for (int gb = blockIdx.x; gb < total; gb += gridDim.x) {
    DotAcc<float> d0, d1;
    for_instance_nodes(first, inst, count, gb, [&](int, long long node) {
      if (node < 0) return;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long k = 3 * node + c;
        const float ri = R[k];
        const float zi = ri * dinv[k];
        Z[k] = zi;
        d0.add_prod(ri, zi);
        d1.add_prod(ri, ri);
      }
    });
    const double a = block_sum_w0(d0.finish(), sh);
    const double b = block_sum_w0(d1.finish(), sh);
    if (threadIdx.x == 0) {
      part[gb] = a;
      part[stride + gb] = b;
    }
  }
  if (batch_last_cta(&ctl->ticket_a)) {
    __shared__ double tot[2 * MFTO_BATCH_MAX];
    per_instance_sums<2>(part, stride, inst, count, false, tot);
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
      BatchScal& s = sc[i];
      s.rz = tot[2 * i];
      s.rr = tot[2 * i + 1];
      s.ff = s.rr;
      s.rtol2ff = rtol * rtol * s.ff;
      s.alpha = 0.0;
      s.beta = rz_prev[i] > 0.0 ? s.rz / rz_prev[i] : 0.0;   // continued direction
      s.it = 0;
      s.status = MFTO_OK;
      s.done = s.ff == 0.0 ? 1 : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int all = 1;
      for (int i = 0; i < count; ++i) all &= sc[i].done;
      ctl->count = count;
      ctl->maxit = maxit;
      ctl->all_done = all;
      ctl->ticket_a = 0u;
    }
  }
}

// outer FP64 residual: R32 = F - KU (zero for masked instances), r.r, f.f
__global__ void __launch_bounds__(MFTO_BLOCK)
batch_residual(const double* __restrict__ F, const double* __restrict__ KU, float* __restrict__ R32,
               const int* __restrict__ mask, const BatchInst* __restrict__ inst, BatchCtl* ctl,
               double* part, int total, int stride, int count, double* res) {
  __shared__ int first[MFTO_BATCH_MAX];
  __shared__ double sh[64];
  for (int i = threadIdx.x; i < count; i += blockDim.x) first[i] = inst[i].up_blk0;
  __syncthreads();
  for (int gb = blockIdx.x; gb < total; gb += gridDim.x) {
    double a = 0.0, b = 0.0;
    for_instance_nodes(first, inst, count, gb, [&](int i, long long node) {
      if (node < 0) return;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long k = 3 * node + c;
        const double ri = F[k] - KU[k];
        R32[k] = mask[i] ? 0.f : (float)ri;
        a += ri * ri;
        b += F[k] * F[k];
      }
    });
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
      part[gb] = a;
      part[stride + gb] = b;
    }
  }
  if (batch_last_cta(&ctl->ticket_d)) {
    per_instance_sums<2>(part, stride, inst, count, false, res);
    if (threadIdx.x == 0) ctl->ticket_d = 0u;
  }
}

// inverse Jacobi diagonal of every instance (FP32), one node per thread
__global__ void __launch_bounds__(MFTO_BLOCK)
batch_diag(const float* __restrict__ E, const uint8_t* __restrict__ fixed, float* __restrict__ dinv,
           const BatchInst* __restrict__ inst, int count, int total, float ke_diag) {
  __shared__ int first[MFTO_BATCH_MAX];
  for (int i = threadIdx.x; i < count; i += blockDim.x) first[i] = inst[i].up_blk0;
  __syncthreads();
  for (int gb = blockIdx.x; gb < total; gb += gridDim.x) {
    for_instance_nodes(first, inst, count, gb, [&](int i, long long node) {
      if (node < 0) return;
      const BatchInst& in = inst[i];
      const int local = (int)(node - in.node_off);
      const int a = local % in.nx, b = (local / in.nx) % in.ny, c = local / (in.nx * in.ny);
      float s = 0.f;
      for (int ce = 0; ce < 8; ++ce) {
        const int ei = a - 1 + (ce & 1), ej = b - 1 + ((ce >> 1) & 1), ek = c - 1 + (ce >> 2);
        if (ei < 0 || ej < 0 || ek < 0 || ei >= in.nelx || ej >= in.nely || ek >= in.nelz) continue;
        s += E[in.elem_off + ei + in.nelx * (ej + in.nely * ek)];
      }
      const uint8_t fm = fixed[node];
      for (int k = 0; k < 3; ++k) dinv[3 * node + k] = ((fm >> k) & 1) ? 1.f : 1.f / (ke_diag * s);
    });
  }
}

__global__ void __launch_bounds__(MFTO_BLOCK)
batch_to_f32(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void __launch_bounds__(MFTO_BLOCK)
batch_accumulate(double* __restrict__ U, const float* __restrict__ e, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    U[i] += (double)e[i];
}

mfto_status bfail(mfto_batch* b, mfto_status code, const char* msg) {
  if (b) snprintf(b->msg, sizeof(b->msg), "%s", msg);
  return code;
}

#define BCUDA(b, call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      if (b) snprintf((b)->msg, sizeof((b)->msg), "%s: %s", #call, cudaGetErrorString(e_)); \
      return MFTO_CUDA_ERROR;                                                             \
    }                                                                                     \
  } while (0)

unsigned persistent_grid(const mfto_batch* b, int per_sm, int total) {
  long long g = (long long)per_sm * b->num_sms;
  if (g > total) g = total;
  if (g < 1) g = 1;
  return (unsigned)g;
}

template <int S>
mfto_status shape_attrs(mfto_batch* b) {
  BCUDA(b, cudaFuncSetAttribute(batch_kv_kernel<double, S>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem<double>()));
  BCUDA(b, cudaFuncSetAttribute(batch_kv_kernel<float, S>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem<float>()));
  BCUDA(b, cudaFuncSetAttribute(batch_pcg_kv<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)batch_smem<float>()));
  BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ_kv64[S], batch_kv_kernel<double, S>,
                                                         MFTO_BLOCK, batch_smem<double>()));
  BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ_kv32[S], batch_kv_kernel<float, S>,
                                                         MFTO_BLOCK, batch_smem<float>()));
  BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ_pcg[S], batch_pcg_kv<S>,
                                                         MFTO_BLOCK, batch_smem<float>()));
  if (b->occ_kv64[S] < 1) b->occ_kv64[S] = 1;
  if (b->occ_kv32[S] < 1) b->occ_kv32[S] = 1;
  if (b->occ_pcg[S] < 1) b->occ_pcg[S] = 1;
  return MFTO_OK;
}

template <typename T>
mfto_status launch_kv(mfto_batch* b, int S, const T* E, const T* V, T* Y, cudaStream_t st,
                      const ModeCoef<T>& K) {
  const int* occ = sizeof(T) == 8 ? b->occ_kv64 : b->occ_kv32;
  const unsigned grid = persistent_grid(b, occ[S], b->kv_total[S]);
  const size_t smem = batch_smem<T>();
  b->launches++;
  switch (S) {
    case 0: batch_kv_kernel<T, 0><<<grid, MFTO_BLOCK, smem, st>>>(E, V, Y, b->d_fixed, K, b->d_inst[0], b->count, b->kv_total[0]); break;
    case 1: batch_kv_kernel<T, 1><<<grid, MFTO_BLOCK, smem, st>>>(E, V, Y, b->d_fixed, K, b->d_inst[1], b->count, b->kv_total[1]); break;
    case 2: batch_kv_kernel<T, 2><<<grid, MFTO_BLOCK, smem, st>>>(E, V, Y, b->d_fixed, K, b->d_inst[2], b->count, b->kv_total[2]); break;
    default: batch_kv_kernel<T, 3><<<grid, MFTO_BLOCK, smem, st>>>(E, V, Y, b->d_fixed, K, b->d_inst[3], b->count, b->kv_total[3]); break;
  }
  BCUDA(b, cudaGetLastError());
  return MFTO_OK;
}

mfto_status launch_pcg_kv(mfto_batch* b, cudaStream_t st, const float* P0, float* P1) {
  const int S = b->shape;
  const unsigned grid = persistent_grid(b, b->occ_pcg[S], b->kv_total[S]);
  const size_t smem = batch_smem<float>();
  b->launches++;
  switch (S) {
    case 0: batch_pcg_kv<0><<<grid, MFTO_BLOCK, smem, st>>>(b->E32, b->z32, P0, P1, b->q32, b->d_fixed, b->mc32, b->d_inst[0], b->d_scal, b->d_ctl, b->d_part_a, b->kv_total[0]); break;
    case 1: batch_pcg_kv<1><<<grid, MFTO_BLOCK, smem, st>>>(b->E32, b->z32, P0, P1, b->q32, b->d_fixed, b->mc32, b->d_inst[1], b->d_scal, b->d_ctl, b->d_part_a, b->kv_total[1]); break;
    case 2: batch_pcg_kv<2><<<grid, MFTO_BLOCK, smem, st>>>(b->E32, b->z32, P0, P1, b->q32, b->d_fixed, b->mc32, b->d_inst[2], b->d_scal, b->d_ctl, b->d_part_a, b->kv_total[2]); break;
    default: batch_pcg_kv<3><<<grid, MFTO_BLOCK, smem, st>>>(b->E32, b->z32, P0, P1, b->q32, b->d_fixed, b->mc32, b->d_inst[3], b->d_scal, b->d_ctl, b->d_part_a, b->kv_total[3]); break;
  }
  BCUDA(b, cudaGetLastError());
  return MFTO_OK;
}

int part_stride(const mfto_batch* b) {
  int m = b->up_total;
  for (int s = 0; s < MFTO_BATCH_SHAPES; ++s) m = m > b->kv_total[s] ? m : b->kv_total[s];
  return m;
}

mfto_status enqueue_chunk(mfto_batch* b, cudaStream_t st, int chunk) {
  const unsigned ug = persistent_grid(b, 8, b->up_total);
  for (int it = 0; it < chunk; ++it) {
    float* p_old = (it & 1) ? b->p1 : b->p0;
    float* p_new = (it & 1) ? b->p0 : b->p1;
    mfto_status s = launch_pcg_kv(b, st, p_old, p_new);
    if (s != MFTO_OK) return s;
    b->launches++;
    batch_update<<<ug, MFTO_BLOCK, 0, st>>>(b->e32, p_new, b->q32, b->r32, b->z32, b->dinv32,
                                            b->d_inst[b->shape], b->d_scal, b->d_ctl, b->d_part_b,
                                            b->up_total, part_stride(b));
    BCUDA(b, cudaGetLastError());
  }
  return MFTO_OK;
}

mfto_status get_graph(mfto_batch* b, BatchGraph** out) {
  BatchGraph* g = b->graph;
  if (g && g->chunk == b->p.check_every && g->shape == b->shape) {
    *out = g;
    return MFTO_OK;
  }
  if (g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
    b->graph = nullptr;
  }
  g = new BatchGraph();
  g->chunk = b->p.check_every;
  g->shape = b->shape;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { delete g; return bfail(b, MFTO_CUDA_ERROR, "batch graph capture failed"); }
  const int64_t l0 = b->launches;
  mfto_status s = enqueue_chunk(b, b->cap_stream, g->chunk);
  b->launches = l0;   // counted per graph launch instead
  e = cudaStreamEndCapture(b->cap_stream, &graph);
  if (s != MFTO_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    delete g;
    return s != MFTO_OK ? s : bfail(b, MFTO_CUDA_ERROR, "batch graph capture failed");
  }
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { delete g; return bfail(b, MFTO_CUDA_ERROR, "batch graph instantiate failed"); }
  b->graph = g;
  *out = g;
  return MFTO_OK;
}

mfto_status upload_inst(mfto_batch* b) {
  std::vector<BatchInst> h(b->count);
  for (int s = 0; s < MFTO_BATCH_SHAPES; ++s) {
    int kv = 0, up = 0;
    for (int i = 0; i < b->count; ++i) {
      const mfto_mesh& m = b->meshes[i];
      BatchInst& in = h[i];
      in.nelx = m.nelx; in.nely = m.nely; in.nelz = m.nelz;
      in.nx = m.nelx + 1; in.ny = m.nely + 1; in.nz = m.nelz + 1;
      in.elem_off = b->elem_off[i];
      in.node_off = b->node_off[i];
      in.kv_blk0 = kv;
      in.kv_nblk = shape_blocks(s, in.nx, in.ny, in.nz);
      kv += in.kv_nblk;
      in.up_blk0 = up;
      in.up_nblk = (in.nx * in.ny * in.nz + MFTO_BLOCK - 1) / MFTO_BLOCK;
      up += in.up_nblk;
    }
    b->kv_total[s] = kv;
    b->up_total = up;
    BCUDA(b, cudaMemcpyAsync(b->d_inst[s], h.data(), sizeof(BatchInst) * b->count,
                             cudaMemcpyHostToDevice, b->stream));
  }
  return MFTO_OK;
}

void free_batch(mfto_batch* b) {
  if (!b) return;
  if (b->graph) {
    if (b->graph->exec) cudaGraphExecDestroy(b->graph->exec);
    delete b->graph;
  }
  void* ptrs[] = {b->d_fixed, b->r32, b->z32, b->p0, b->p1, b->q32, b->e32, b->dinv32, b->E32,
                  b->q64, b->d_scal, b->d_ctl, b->d_part_a, b->d_part_b, b->d_res, b->d_mask,
                  b->d_rzp,
                  b->d_inst[0], b->d_inst[1], b->d_inst[2], b->d_inst[3]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->h_scal) cudaFreeHost(b->h_scal);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

}  // namespace

extern "C" mfto_status mfto_batch_create(int32_t count, const mfto_mesh* meshes,
                                         const mfto_params* params, const uint8_t* h_fixed,
                                         void* stream, mfto_batch** out) {
  if (!out) return MFTO_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || count > MFTO_BATCH_MAX || !meshes || !params || !h_fixed) return MFTO_INVALID_ARG;
  if (!(params->nu > -1.0 && params->nu < 0.5) || params->check_every < 2 ||
      params->check_every % 2 || params->maxit < 1 || !(params->rtol > 0.0))
    return MFTO_INVALID_ARG;
  mfto_batch* b = new mfto_batch();
  b->count = count;
  b->p = *params;
  b->stream = (cudaStream_t)stream;
  b->h = meshes[0].h;
  b->shape = 0;
  long long ne = 0, nn = 0;
  for (int i = 0; i < count; ++i) {
    const mfto_mesh& m = meshes[i];
    if (m.nelx < 1 || m.nely < 1 || m.nelz < 1 || m.h != b->h) { free_batch(b); return MFTO_INVALID_ARG; }
    b->meshes.push_back(m);
    b->elem_off.push_back(ne);
    b->node_off.push_back(nn);
    ne += (long long)m.nelx * m.nely * m.nelz;
    nn += (long long)(m.nelx + 1) * (m.nely + 1) * (m.nelz + 1);
  }
  b->elem_off.push_back(ne);
  b->node_off.push_back(nn);
  b->n_elem = ne;
  b->n_node = nn;
  b->n_dof = 3 * nn;
  if (b->n_dof > (long long)INT32_MAX) { free_batch(b); return MFTO_TOO_LARGE; }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    free_batch(b);
    return MFTO_CUDA_ERROR;
  }
  // block totals of the largest shape decide the partial-sum buffers
  int max_blocks = 0, up = 0;
  for (int s = 0; s < MFTO_BATCH_SHAPES; ++s) {
    int kv = 0;
    for (int i = 0; i < count; ++i)
      kv += shape_blocks(s, meshes[i].nelx + 1, meshes[i].nely + 1, meshes[i].nelz + 1);
    max_blocks = max_blocks > kv ? max_blocks : kv;
  }
  for (int i = 0; i < count; ++i)
    up += (int)(((long long)(meshes[i].nelx + 1) * (meshes[i].nely + 1) * (meshes[i].nelz + 1) +
                 MFTO_BLOCK - 1) / MFTO_BLOCK);
  max_blocks = max_blocks > up ? max_blocks : up;
  bool ok = true;
  auto A = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
  };
  const size_t nd32 = sizeof(float) * b->n_dof;
  A((void**)&b->d_fixed, b->n_node);
  A((void**)&b->r32, nd32);
  A((void**)&b->z32, nd32);
  A((void**)&b->p0, nd32);
  A((void**)&b->p1, nd32);
  A((void**)&b->q32, nd32);
  A((void**)&b->e32, nd32);
  A((void**)&b->dinv32, nd32);
  A((void**)&b->E32, sizeof(float) * b->n_elem);
  A((void**)&b->q64, sizeof(double) * b->n_dof);
  A((void**)&b->d_scal, sizeof(BatchScal) * count);
  A((void**)&b->d_ctl, sizeof(BatchCtl));
  A((void**)&b->d_part_a, sizeof(double) * 2 * max_blocks);
  A((void**)&b->d_part_b, sizeof(double) * 2 * max_blocks);
  A((void**)&b->d_res, sizeof(double) * 2 * count);
  A((void**)&b->d_rzp, sizeof(double) * count);
  A((void**)&b->d_mask, sizeof(int) * count);
  for (int s = 0; s < MFTO_BATCH_SHAPES; ++s) A((void**)&b->d_inst[s], sizeof(BatchInst) * count);
  if (ok && (cudaMallocHost(&b->h_scal, sizeof(BatchScal) * count) != cudaSuccess ||
             cudaMallocHost(&b->h_ctl, sizeof(BatchCtl)) != cudaSuccess))
    ok = false;
  if (!ok) {
    cudaGetLastError();
    free_batch(b);
    return MFTO_OOM;
  }
  mfto_status s = upload_inst(b);
  if (s == MFTO_OK) s = shape_attrs<0>(b);
  if (s == MFTO_OK) s = shape_attrs<1>(b);
  if (s == MFTO_OK) s = shape_attrs<2>(b);
  if (s == MFTO_OK) s = shape_attrs<3>(b);
  if (s != MFTO_OK) { free_batch(b); return s; }
  if (cudaMemcpyAsync(b->d_fixed, h_fixed, b->n_node, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_ctl, 0, sizeof(BatchCtl), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_scal, 0, sizeof(BatchScal) * count, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    free_batch(b);
    return MFTO_CUDA_ERROR;
  }
  // unit element operator (same material and edge for every instance)
  double ke[576];
  mfto_unit_ke(1.0, params->nu, b->h, ke);
  b->ke_diag = ke[0];
  mode_coefficients(params->nu, b->h, &b->mc64, &b->mc32);
  *out = b;
  return MFTO_OK;
}

extern "C" mfto_status mfto_batch_destroy(mfto_batch* b) {
  if (!b) return MFTO_INVALID_ARG;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  return MFTO_OK;
}

extern "C" const char* mfto_batch_last_error(const mfto_batch* b) { return b ? b->msg : "null batch"; }

extern "C" mfto_status mfto_batch_layout(const mfto_batch* b, int64_t* elem_off, int64_t* dof_off) {
  if (!b) return MFTO_INVALID_ARG;
  for (int i = 0; i <= b->count; ++i) {
    if (elem_off) elem_off[i] = b->elem_off[i];
    if (dof_off) dof_off[i] = 3 * b->node_off[i];
  }
  return MFTO_OK;
}

extern "C" mfto_status mfto_batch_kv(mfto_batch* b, mfto_form form, const void* E, const void* V,
                                     void* Y) {
  if (!b) return MFTO_INVALID_ARG;
  if (!E || !V || !Y || V == Y) return bfail(b, MFTO_INVALID_ARG, "mfto_batch_kv: bad pointers");
  if (form == MFTO_FORM_F64)
    return launch_kv<double>(b, b->shape, (const double*)E, (const double*)V, (double*)Y, b->stream, b->mc64);
  if (form == MFTO_FORM_F32)
    return launch_kv<float>(b, b->shape, (const float*)E, (const float*)V, (float*)Y, b->stream, b->mc32);
  return bfail(b, MFTO_UNSUPPORTED, "mfto_batch_kv: forms F64 and F32 only");
}

extern "C" mfto_status mfto_batch_autotune(mfto_batch* b, int32_t reps, double* ms_out,
                                           int32_t* chosen) {
  if (!b || reps < 1) return MFTO_INVALID_ARG;
  // time each block shape on an FP32 K.V of the batch with unit moduli
  BCUDA(b, cudaMemsetAsync(b->r32, 0, sizeof(float) * b->n_dof, b->stream));
  std::vector<float> ones(b->n_elem, 1.0f);
  BCUDA(b, cudaMemcpyAsync(b->E32, ones.data(), sizeof(float) * b->n_elem, cudaMemcpyHostToDevice,
                           b->stream));
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  double best = 1e300;
  int best_s = 0;
  for (int s = 0; s < MFTO_BATCH_SHAPES; ++s) {
    mfto_status st = launch_kv<float>(b, s, b->E32, b->r32, b->z32, b->stream, b->mc32);  // warm-up
    if (st != MFTO_OK) return st;
    BCUDA(b, cudaEventRecord(e0, b->stream));
    for (int r = 0; r < reps; ++r) {
      st = launch_kv<float>(b, s, b->E32, b->r32, b->z32, b->stream, b->mc32);
      if (st != MFTO_OK) return st;
    }
    BCUDA(b, cudaEventRecord(e1, b->stream));
    BCUDA(b, cudaEventSynchronize(e1));
    float ms = 0.f;
    BCUDA(b, cudaEventElapsedTime(&ms, e0, e1));
    const double per = ms / reps;
    if (ms_out) ms_out[s] = per;
    if (per < best) { best = per; best_s = s; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->shape = best_s;
  if (chosen) *chosen = best_s;
  return MFTO_OK;
}

extern "C" mfto_status mfto_batch_set_shape(mfto_batch* b, int32_t shape) {
  if (!b || shape < 0 || shape >= MFTO_BATCH_SHAPES) return MFTO_INVALID_ARG;
  b->shape = shape;
  return MFTO_OK;
}

extern "C" mfto_status mfto_batch_solve(mfto_batch* b, double inner_tol, const double* E,
                                        const double* F, double* U, int32_t inner_maxit,
                                        int32_t max_outer, mfto_ir_stats* st) {
  if (!b) return MFTO_INVALID_ARG;
  if (!E || !F || !U || !st) return bfail(b, MFTO_INVALID_ARG, "mfto_batch_solve: null pointer");
  if (!(inner_tol > 0.0 && inner_tol < 1.0) || inner_maxit < 1 || max_outer < 1)
    return bfail(b, MFTO_INVALID_ARG, "mfto_batch_solve: bad tolerance or caps");
  const int count = b->count;
  const int stride = part_stride(b);
  const unsigned ug = persistent_grid(b, 8, b->up_total);
  for (int i = 0; i < count; ++i) {
    memset(&st[i], 0, sizeof(mfto_ir_stats));
    st[i].status = MFTO_NOT_CONVERGED;
  }
  b->launches++;
  batch_to_f32<<<ug, MFTO_BLOCK, 0, b->stream>>>(E, b->E32, b->n_elem);
  b->launches++;
  batch_diag<<<ug, MFTO_BLOCK, 0, b->stream>>>(b->E32, b->d_fixed, b->dinv32, b->d_inst[b->shape],
                                               count, b->up_total, (float)b->ke_diag);
  BCUDA(b, cudaGetLastError());
  std::vector<int> mask(count, 0);
  std::vector<double> prev(count, 0.0), res(2 * count);
  std::vector<int> stalls(count, 0);
  std::vector<double> rzp(count, 0.0);   // continued directions (MFTO_IR_CONTINUE)
  for (int outer = 0;; ++outer) {
    BCUDA(b, cudaMemcpyAsync(b->d_mask, mask.data(), sizeof(int) * count, cudaMemcpyHostToDevice,
                             b->stream));
    mfto_status s = launch_kv<double>(b, b->shape, E, U, b->q64, b->stream, b->mc64);
    if (s != MFTO_OK) return s;
    b->launches++;
    batch_residual<<<ug, MFTO_BLOCK, 0, b->stream>>>(F, b->q64, b->r32, b->d_mask,
                                                     b->d_inst[b->shape], b->d_ctl, b->d_part_a,
                                                     b->up_total, stride, count, b->d_res);
    BCUDA(b, cudaGetLastError());
    BCUDA(b, cudaMemcpyAsync(res.data(), b->d_res, sizeof(double) * 2 * count,
                             cudaMemcpyDeviceToHost, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    bool any_live = false, changed = false;
    for (int i = 0; i < count; ++i) {
      if (mask[i]) continue;
      const double rr = res[2 * i], ff = res[2 * i + 1];
      const double rel = ff > 0.0 ? sqrt(rr / ff) : 0.0;
      st[i].fnorm = sqrt(ff);
      st[i].rel_residual = rel;
      st[i].kv_f64++;
      if (outer < 64) st[i].history[outer] = rel;
      int stop = 0;
      if (rel <= b->p.rtol) { st[i].status = MFTO_OK; stop = 1; }
      else if (!isfinite(rel)) { st[i].status = MFTO_BREAKDOWN; stop = 1; }
      else {
        if (outer > 0) {
          stalls[i] = rel > 0.9 * prev[i] ? stalls[i] + 1 : 0;
          if (stalls[i] >= 2) { st[i].status = MFTO_STALLED; stop = 1; }
        }
        if (!stop && outer >= max_outer) { st[i].status = MFTO_NOT_CONVERGED; stop = 1; }
      }
      if (stop) { mask[i] = 1; changed = true; }
      else { prev[i] = rel; any_live = true; }
    }
    if (!any_live) break;
    if (changed) {
      // zero the right-hand sides of instances that stopped in this round
      BCUDA(b, cudaMemcpyAsync(b->d_mask, mask.data(), sizeof(int) * count,
                               cudaMemcpyHostToDevice, b->stream));
      b->launches++;
      batch_residual<<<ug, MFTO_BLOCK, 0, b->stream>>>(F, b->q64, b->r32, b->d_mask,
                                                       b->d_inst[b->shape], b->d_ctl, b->d_part_a,
                                                       b->up_total, stride, count, b->d_res);
      BCUDA(b, cudaGetLastError());
    }
    BCUDA(b, cudaMemsetAsync(b->e32, 0, sizeof(float) * b->n_dof, b->stream));
    // instances that continue their direction keep it in p0; the others start from p = z
    for (int i = 0; i < count; ++i) {
      if (mask[i]) rzp[i] = 0.0;
      if (!(rzp[i] > 0.0)) {
        const long long o = 3 * b->node_off[i];
        const long long n = 3 * ((long long)(b->meshes[i].nelx + 1) * (b->meshes[i].nely + 1) *
                                 (b->meshes[i].nelz + 1));
        BCUDA(b, cudaMemsetAsync(b->p0 + o, 0, sizeof(float) * n, b->stream));
      }
    }
    BCUDA(b, cudaMemcpyAsync(b->d_rzp, rzp.data(), sizeof(double) * count, cudaMemcpyHostToDevice,
                             b->stream));
    b->launches++;
    batch_init<<<ug, MFTO_BLOCK, 0, b->stream>>>(b->r32, b->z32, b->dinv32, b->d_inst[b->shape],
                                                 b->d_scal, b->d_ctl, b->d_part_a, b->up_total,
                                                 stride, inner_tol, inner_maxit, count, b->d_rzp);
    BCUDA(b, cudaGetLastError());
    BatchGraph* g = nullptr;
    s = get_graph(b, &g);
    if (s != MFTO_OK) return s;
    for (;;) {
      BCUDA(b, cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost,
                               b->stream));
      BCUDA(b, cudaStreamSynchronize(b->stream));
      if (b->h_ctl->all_done) break;
      BCUDA(b, cudaGraphLaunch(g->exec, b->stream));
      b->launches += 2 * (int64_t)g->chunk;
    }
    BCUDA(b, cudaMemcpyAsync(b->h_scal, b->d_scal, sizeof(BatchScal) * count,
                             cudaMemcpyDeviceToHost, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < count; ++i) {
      if (mask[i]) continue;
      const BatchScal& fin = b->h_scal[i];
      st[i].inner_iterations += fin.it;
      st[i].outer_iterations++;
      // continued direction: iteration j writes its direction into p1 (j even)
      // or p0 (j odd); the next inner solve reads p0 first
      rzp[i] = 0.0;
      if (b->ir_mode == MFTO_IR_CONTINUE && fin.it >= 1 && fin.status != MFTO_BREAKDOWN &&
          fin.beta > 0.0 && isfinite(fin.rz / fin.beta)) {
        if (fin.it & 1) {
          const long long o = 3 * b->node_off[i];
          const long long n = 3 * ((long long)(b->meshes[i].nelx + 1) * (b->meshes[i].nely + 1) *
                                   (b->meshes[i].nelz + 1));
          BCUDA(b, cudaMemcpyAsync(b->p0 + o, b->p1 + o, sizeof(float) * n,
                                   cudaMemcpyDeviceToDevice, b->stream));
        }
        rzp[i] = fin.rz / fin.beta;
      }
    }
    b->launches++;
    batch_accumulate<<<ug, MFTO_BLOCK, 0, b->stream>>>(U, b->e32, b->n_dof);
    BCUDA(b, cudaGetLastError());
  }
  return MFTO_OK;
}

extern "C" mfto_status mfto_batch_launch_count(const mfto_batch* b, int64_t* n) {
  if (!b || !n) return MFTO_INVALID_ARG;
  *n = b->launches;
  return MFTO_OK;
}

extern "C" mfto_status mfto_batch_set_ir_mode(mfto_batch* b, int32_t mode) {
  if (!b) return MFTO_INVALID_ARG;
  if (mode != MFTO_IR_RESTART && mode != MFTO_IR_CONTINUE)
    return bfail(b, MFTO_INVALID_ARG, "mfto_batch_set_ir_mode: MFTO_IR_RESTART or MFTO_IR_CONTINUE");
  b->ir_mode = mode;
  return MFTO_OK;
}

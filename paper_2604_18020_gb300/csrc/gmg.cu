// Geometric multigrid preconditioner for the masked stiffness operator: the
// follow-on the paper proposes (Sec. 6, "Path to Geometric Multigrid
// Integration": restriction R, prolongation P = R^T, a direct coarsest solve,
// smoothing steps that each apply the operator; Sec. 3.5, "Path forward": the
// low-precision K.v as the smoother inside a V-cycle).
//
// Hierarchy (rebuilt for every modulus field):
//   level 0 is the mesh itself, applied by the FP32 structured K.v;
//   level l + 1 halves the element counts of level l per axis, rounding up;
//   its element matrices are Galerkin products of the children's:
//     A_E = sum_{children c} P_c^T A_c P_c,
//   P_c (24 x 24) the trilinear interpolation from E's 8 corners to child c's
//   8 nodes (per axis weights 1 - s, s at the child's node, s in {0, 1/2, 1}),
//   A_c = E_c D_c KE D_c on level 0 (D_c zeroes the child's fixed DOFs) or the
//   child's stored matrix; rows and columns of E's fixed DOFs are then zeroed.
//   For nested trilinear spaces the assembly of these matrices is exactly
//   Phat^T A Phat, Phat = M_f P M_c (the masked interpolation), so every level
//   is the Galerkin operator plus the identity on its fixed DOFs.  A coarse
//   DOF is fixed where the fine DOF at the same position is.
//   Interior coarse elements of level 1 (all 8 children, no fixed DOF) are
//   formed as sum_c E_c G_c from the unit-modulus child matrices
//   G_c = P_c^T KE P_c.
// V-cycle: nu_pre sweeps from x = 0, residual, restriction, recursion,
// prolongation, nu_post sweeps; the coarsest level is solved with its dense
// inverse (Cholesky on the host in FP64, stored as FP32; a rank-deficient
// operator -- a consistent singular problem -- factorised with a small
// diagonal shift).  Sweeps are l1-Jacobi, x += omega D1^-1 (b - A x), or
// Chebyshev of a chosen degree on [1/30, 1]; the l1 row sums come from the
// element matrices, D1 = sum_E sum_j |(A_E)_ij| (1 on fixed DOFs), so
// lambda_max(D1^-1 A) <= 1 bounds both.  Coarse levels apply their operator
// node by node from the element matrices (each node sums its rows of its
// <= 8 elements: no atomics), with a sweep fused into the same launch; level
// 1 is applied as Phat^T K Phat through the fine FP32 K.v instead when its
// matrices would not stay in L2.  The cycle is replayed from a CUDA graph.
// Outer solvers (CG with z = V(r) and the Polak-Ribiere beta, because the
// cycle runs in FP32): one FP64 CG, or FP64 refinement around FP32 CGs whose
// scalars stay on the device and whose iterations are replayed in graph
// chunks, each continuing the previous one's direction; fixed-order sums
// throughout, so every result is bit-reproducible.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

struct GmgScalars {
  double sum[4];
  unsigned int ticket;
};

// Scalars of the FP32 inner CG when its iterations run from a graph: every
// step reads and writes them on the device; the host polls done / it.
struct GmgCg {
  double rz, alpha, beta, tol2;
  int32_t it, maxit, done, breakdown;
  unsigned int ticket;
};

struct GmgLevel {
  int nx = 0, ny = 0, nz = 0;
  int64_t n_elem = 0, n_node = 0, n_dof = 0;
  uint8_t* d_fixed = nullptr;   // per-node mask (level 0: the handle's, not owned)
  float* d_K = nullptr;         // [n_elem][576] element matrices (levels >= 1)
  float* d_dinv = nullptr;      // 1 / l1 row sums
  float* x = nullptr;           // correction (levels >= 1)
  float* x2 = nullptr;          // its other half when a fused sweep writes a copy
  float* cr = nullptr;          // Chebyshev residual and step (Chebyshev smoother only)
  float* cd = nullptr;
  float* b = nullptr;           // right-hand side (levels >= 1)
  float* t = nullptr;           // operator applied to x
};

struct GmgWs {
  int n_levels = 0;
  GmgLevel lv[MFTO_GMG_MAX_LEVELS];
  mfto_gmg_params prm{};
  float* d_E32 = nullptr;
  float* d_G = nullptr;             // [8][576] unit-modulus child Galerkin matrices
  int cheb = 0;                     // Chebyshev degree in use (cheb_degree resolved)
  bool mf1 = false;                 // level 1 applied as Phat^T K Phat (no matrices read)
  float* mf_s0 = nullptr;           // its two fine-level scratch vectors
  float* mf_s1 = nullptr;
  float* d_cinv = nullptr;          // dense inverse of the coarsest operator
  int n_c = 0;                      // its DOFs
  std::vector<std::vector<uint8_t>> h_fixed;   // per-level node masks
  GmgScalars* d_s = nullptr;
  GmgScalars* h_s = nullptr;
  bool ready = false;               // a hierarchy is built
  bool use_in_simp = false;         // mfto_simp_step solves with mfto_gmg_solve
  // the V-cycle captured as a CUDA graph for one (r, z) pair and parameter set
  cudaGraphExec_t vexec = nullptr;
  const float* vkey_r = nullptr;
  float* vkey_z = nullptr;
  mfto_gmg_params vprm{};
  int64_t vnodes = 0;               // kernels in the graph
  // cchunk inner CG iterations (K.v, step, V-cycle, direction) as one graph
  cudaGraphExec_t cexec = nullptr;
  mfto_gmg_params cprm{};
  int64_t cnodes = 0;
  int cchunk = 0;
  GmgCg* d_cg = nullptr;
  GmgCg* h_cg = nullptr;
};

// Iterations per replayed chunk: the host polls once per chunk, and up to
// chunk - 1 iterations after convergence still run their K.v and V-cycle
// (their CG steps skip).  Four on meshes whose cycle is short; one where a
// cycle costs far more than a poll (above 2M DOFs, a cycle takes > 0.5 ms).
int cg_chunk_len(const mfto_handle* h) { return h->n_dof > 2000000 ? 1 : 4; }

namespace {

constexpr int kB = MFTO_BLOCK;

__host__ __device__ inline int64_t nid(int i, int j, int k, int nx, int ny) {
  return i + (int64_t)(nx + 1) * (j + (int64_t)(ny + 1) * k);
}

int g_sms = 148;   // SM count of the device (set from the handle at setup)

int grid_of(int64_t n) {
  const int64_t want = (n + kB - 1) / kB;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, 16LL * g_sms));
}

// trilinear weight of coarse local node m at child ch's local node n
__device__ __forceinline__ float phi(int ch, int n, int m) {
  float w = 1.0f;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int p = ((ch >> ax) & 1) + ((n >> ax) & 1);   // 0, 1, 2 in fine units
    w *= ((m >> ax) & 1) ? 0.5f * p : 1.0f - 0.5f * p;
  }
  return w;
}

__global__ void __launch_bounds__(kB) gmg_cast(const double* __restrict__ a, float* __restrict__ b,
                                               int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// l1 row sums of level 0 from E_e D_e KE D_e, node by node
__global__ void __launch_bounds__(kB)
gmg_l1_fine(const float* __restrict__ E, const uint8_t* __restrict__ fixed,
            const float* __restrict__ ke, int nx, int ny, int nz, float* __restrict__ dinv) {
  __shared__ float ka[576];
  for (int i = threadIdx.x; i < 576; i += blockDim.x) ka[i] = fabsf(ke[i]);
  __syncthreads();
  const int64_t n_node = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; nd < n_node;
       nd += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(nd % (nx + 1));
    const int j = (int)((nd / (nx + 1)) % (ny + 1));
    const int k = (int)(nd / ((int64_t)(nx + 1) * (ny + 1)));
    double acc[3] = {0.0, 0.0, 0.0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int ex = i - dx, ey = j - dy, ez = k - dz;
          if (ex < 0 || ey < 0 || ez < 0 || ex >= nx || ey >= ny || ez >= nz) continue;
          const int l = dx + 2 * dy + 4 * dz;
          uint8_t fm[8];
#pragma unroll
          for (int lb = 0; lb < 8; ++lb)
            fm[lb] = fixed[nid(ex + (lb & 1), ey + ((lb >> 1) & 1), ez + (lb >> 2), nx, ny)];
          const float Ee = E[ex + (int64_t)nx * (ey + (int64_t)ny * ez)];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int lb = 0; lb < 8; ++lb)
#pragma unroll
              for (int cb = 0; cb < 3; ++cb)
                if (!((fm[lb] >> cb) & 1)) s += ka[(3 * l + c) * 24 + 3 * lb + cb];
            acc[c] += (double)Ee * s;
          }
        }
    const uint8_t fm = fixed[nd];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      dinv[3 * nd + c] = ((fm >> c) & 1) ? 1.0f : (float)(1.0 / acc[c]);
  }
}

// G_c = P_c^T KE P_c for the 8 child positions (one CTA each): the Galerkin
// matrix of a unit-modulus child, so that an interior coarse element of
// level 1 is just sum_c E_c G_c.
__global__ void __launch_bounds__(kB)
gmg_child_galerkin(const float* __restrict__ ke, float* __restrict__ G) {
  __shared__ float T[576];
  const int ch = blockIdx.x;
  for (int idx = threadIdx.x; idx < 576; idx += blockDim.x) {
    const int i = idx / 24, col = idx - 24 * (idx / 24);
    const int m = col / 3, cc = col - 3 * (col / 3);
    float s = 0.0f;
#pragma unroll
    for (int n = 0; n < 8; ++n) s = fmaf(ke[i * 24 + 3 * n + cc], phi(ch, n, m), s);
    T[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 576; idx += blockDim.x) {
    const int row = idx / 24, q = idx - 24 * (idx / 24);
    const int m = row / 3, cc = row - 3 * (row / 3);
    float s = 0.0f;
#pragma unroll
    for (int n = 0; n < 8; ++n) s = fmaf(phi(ch, n, m), T[(3 * n + cc) * 24 + q], s);
    G[ch * 576 + idx] = s;
  }
}

// Element matrices of level l + 1 (dims mx, my, mz) from level l (nx, ny, nz):
// one CTA per coarse element, children one after another through shared
// memory (T = A_c P_c, then M += P_c^T T), M held in registers.
template <bool FINE0>
__global__ void __launch_bounds__(kB)
gmg_galerkin(const float* __restrict__ Kf, const float* __restrict__ E,
             const float* __restrict__ ke, const float* __restrict__ G,
             const uint8_t* __restrict__ fixf, int nx, int ny, int nz,
             const uint8_t* __restrict__ fixc, int mx, int my, int mz, float* __restrict__ Kc) {
  __shared__ float A[576], T[576], KEs[FINE0 ? 576 : 1], Gs[FINE0 ? 8 * 576 : 1];
  if (FINE0) {
    for (int i = threadIdx.x; i < 576; i += blockDim.x) KEs[i] = ke[i];
    for (int i = threadIdx.x; i < 8 * 576; i += blockDim.x) Gs[i] = G[i];
  }
  const int64_t n_c = (int64_t)mx * my * mz;
  for (int64_t e = blockIdx.x; e < n_c; e += gridDim.x) {
    const int I = (int)(e % mx), J = (int)((e / mx) % my), K = (int)(e / ((int64_t)mx * my));
    float acc[3] = {0.0f, 0.0f, 0.0f};
    if (FINE0) {
      // interior element: all 8 children present and no fixed DOF among the
      // 27 fine nodes -> sum_c E_c G_c
      bool fixed_here = false;
      if (threadIdx.x < 27) {
        const int a = threadIdx.x % 3, b = (threadIdx.x / 3) % 3, c = threadIdx.x / 9;
        const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
        fixed_here = i > nx || j > ny || k > nz || fixf[nid(i, j, k, nx, ny)] != 0;
      }
      const bool slow = __syncthreads_or(fixed_here) != 0 || 2 * I + 1 >= nx ||
                        2 * J + 1 >= ny || 2 * K + 1 >= nz;
      if (!slow) {
        float Ec[8];
#pragma unroll
        for (int ch = 0; ch < 8; ++ch)
          Ec[ch] = E[(2 * I + (ch & 1)) + (int64_t)nx * ((2 * J + ((ch >> 1) & 1)) +
                                                         (int64_t)ny * (2 * K + (ch >> 2)))];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int idx = threadIdx.x + r * kB;
          if (idx < 576) {
            float s = 0.0f;
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) s = fmaf(Ec[ch], Gs[ch * 576 + idx], s);
            Kc[e * 576 + idx] = s;
          }
        }
        continue;                                                 // uniform over the CTA
      }
    }
    for (int ch = 0; ch < 8; ++ch) {
      const int fx = 2 * I + (ch & 1), fy = 2 * J + ((ch >> 1) & 1), fz = 2 * K + (ch >> 2);
      if (fx >= nx || fy >= ny || fz >= nz) continue;            // uniform over the CTA
      const int64_t c = fx + (int64_t)nx * (fy + (int64_t)ny * fz);
      __syncthreads();                                            // A, T free again
      for (int idx = threadIdx.x; idx < 576; idx += blockDim.x) {
        if (FINE0) {
          const int r = idx / 24, q = idx - 24 * (idx / 24);
          const int nr = r / 3, nq = q / 3;
          const uint8_t fr = fixf[nid(fx + (nr & 1), fy + ((nr >> 1) & 1), fz + (nr >> 2), nx, ny)];
          const uint8_t fq = fixf[nid(fx + (nq & 1), fy + ((nq >> 1) & 1), fz + (nq >> 2), nx, ny)];
          const bool free_rq = !((fr >> (r % 3)) & 1) && !((fq >> (q % 3)) & 1);
          A[idx] = free_rq ? E[c] * KEs[idx] : 0.0f;
        } else {
          A[idx] = Kf[c * 576 + idx];
        }
      }
      __syncthreads();
      // T[i][3m + cc] = sum_n A[i][3n + cc] phi(ch, n, m)
      for (int idx = threadIdx.x; idx < 576; idx += blockDim.x) {
        const int i = idx / 24, col = idx - 24 * (idx / 24);
        const int m = col / 3, cc = col - 3 * (col / 3);
        float s = 0.0f;
#pragma unroll
        for (int n = 0; n < 8; ++n) s = fmaf(A[i * 24 + 3 * n + cc], phi(ch, n, m), s);
        T[idx] = s;
      }
      __syncthreads();
      // M[3m + cc][q] += sum_n phi(ch, n, m) T[3n + cc][q]
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int idx = threadIdx.x + r * kB;
        if (idx < 576) {
          const int row = idx / 24, q = idx - 24 * (idx / 24);
          const int m = row / 3, cc = row - 3 * (row / 3);
          float s = 0.0f;
#pragma unroll
          for (int n = 0; n < 8; ++n) s = fmaf(phi(ch, n, m), T[(3 * n + cc) * 24 + q], s);
          acc[r] += s;
        }
      }
    }
    // zero the rows and columns of E's fixed DOFs
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int idx = threadIdx.x + r * kB;
      if (idx < 576) {
        const int row = idx / 24, q = idx - 24 * (idx / 24);
        const int nr = row / 3, nq = q / 3;
        const uint8_t fr = fixc[nid(I + (nr & 1), J + ((nr >> 1) & 1), K + (nr >> 2), mx, my)];
        const uint8_t fq = fixc[nid(I + (nq & 1), J + ((nq >> 1) & 1), K + (nq >> 2), mx, my)];
        const bool free_rq = !((fr >> (row % 3)) & 1) && !((fq >> (q % 3)) & 1);
        Kc[e * 576 + idx] = free_rq ? acc[r] : 0.0f;
      }
    }
  }
}

// l1 row sums of a coarse level from its element matrices
__global__ void __launch_bounds__(kB)
gmg_l1_coarse(const float* __restrict__ K, const uint8_t* __restrict__ fixed, int nx, int ny,
              int nz, float* __restrict__ dinv) {
  const int64_t n_node = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; nd < n_node;
       nd += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(nd % (nx + 1));
    const int j = (int)((nd / (nx + 1)) % (ny + 1));
    const int k = (int)(nd / ((int64_t)(nx + 1) * (ny + 1)));
    double acc[3] = {0.0, 0.0, 0.0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int ex = i - dx, ey = j - dy, ez = k - dz;
          if (ex < 0 || ey < 0 || ez < 0 || ex >= nx || ey >= ny || ez >= nz) continue;
          const int l = dx + 2 * dy + 4 * dz;
          const float* Ke = K + (ex + (int64_t)nx * (ey + (int64_t)ny * ez)) * 576;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float s = 0.0f;
            for (int q = 0; q < 24; ++q) s += fabsf(Ke[(3 * l + c) * 24 + q]);
            acc[c] += s;
          }
        }
    const uint8_t fm = fixed[nd];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      dinv[3 * nd + c] = ((fm >> c) & 1) ? 1.0f : (float)(1.0 / acc[c]);
  }
}

// The coarse-level operator's rows of node nd, 8 lanes per node: lane `sub`
// takes the node's three rows of adjacent element sub (corner offsets the bits
// of sub) against that element's 24 input values val(DOF), and the 8 lanes'
// sums are added in a fixed order, so every lane ends with the node's three
// sums (zero for nd >= n_node).  Fixed DOFs are not special here: their
// columns are zero in the element matrices.  Every lane of the warp must call
// it (the shuffles need all 32).
template <class Val>
__device__ __forceinline__ void coarse_rows(const float* __restrict__ K, int nx, int ny, int nz,
                                            int64_t nd, int64_t n_node, int sub, Val val,
                                            float acc[3]) {
  const int dx = sub & 1, dy = (sub >> 1) & 1, dz = sub >> 2;
  acc[0] = acc[1] = acc[2] = 0.0f;
  if (nd < n_node) {
    const int i = (int)(nd % (nx + 1));
    const int j = (int)((nd / (nx + 1)) % (ny + 1));
    const int k = (int)(nd / ((int64_t)(nx + 1) * (ny + 1)));
    const int ex = i - dx, ey = j - dy, ez = k - dz;
    if (ex >= 0 && ey >= 0 && ez >= 0 && ex < nx && ey < ny && ez < nz) {
      const int l = dx + 2 * dy + 4 * dz;
      const float* Ke = K + (ex + (int64_t)nx * (ey + (int64_t)ny * ez)) * 576;
      float xe[24];
#pragma unroll
      for (int lb = 0; lb < 8; ++lb) {
        const int64_t m = nid(ex + (lb & 1), ey + ((lb >> 1) & 1), ez + (lb >> 2), nx, ny);
        xe[3 * lb] = val(3 * m);
        xe[3 * lb + 1] = val(3 * m + 1);
        xe[3 * lb + 2] = val(3 * m + 2);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4* row = reinterpret_cast<const float4*>(Ke + (3 * l + c) * 24);
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const float4 w = row[q];
          s = fmaf(w.x, xe[4 * q], s);
          s = fmaf(w.y, xe[4 * q + 1], s);
          s = fmaf(w.z, xe[4 * q + 2], s);
          s = fmaf(w.w, xe[4 * q + 3], s);
        }
        acc[c] = s;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 1);
    acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 2);
    acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 4);
  }
}

// Coarse-level operator with identity rows on fixed DOFs, one node per 8
// lanes (coarse_rows).  Three forms, so that a smoothing sweep and its
// operator application are one launch:
//   KV_PLAIN:  y = A x;
//   KV_FIRST:  the first sweep from zero, x = omega D1^-1 b (neighbours' values
//              formed on the fly), written to xo, and y = A x;
//   KV_SMOOTH: xo = x + omega D1^-1 (b - A x) (xo distinct from x).
enum { KV_PLAIN = 0, KV_FIRST = 1, KV_SMOOTH = 2 };

template <int MODE>
__global__ void __launch_bounds__(kB)
gmg_kv_coarse(const float* __restrict__ K, const uint8_t* __restrict__ fixed, int nx, int ny,
              int nz, const float* __restrict__ x, const float* __restrict__ b,
              const float* __restrict__ dinv, float omega, float* __restrict__ y,
              float* __restrict__ xo) {
  const int64_t n_node = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  const int sub = threadIdx.x & 7;
  auto val = [&](int64_t d) -> float {
    return MODE == KV_FIRST ? omega * dinv[d] * b[d] : x[d];
  };
  // every lane of a warp runs the same number of trips (the shuffles need all 32)
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 3);
  const int64_t trips = (n_node + groups - 1) / groups;
  for (int64_t tr = 0; tr < trips; ++tr) {
    const int64_t nd = tr * groups + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3);
    float acc[3];
    coarse_rows(K, nx, ny, nz, nd, n_node, sub, val, acc);
    if (sub < 3 && nd < n_node) {
      const int64_t d = 3 * nd + sub;
      const uint8_t fm = fixed[nd];
      const float a = sub == 0 ? acc[0] : (sub == 1 ? acc[1] : acc[2]);
      const float xd = val(d);
      const float yd = ((fm >> sub) & 1) ? xd : a;
      if (MODE == KV_SMOOTH) {
        xo[d] = xd + omega * dinv[d] * (b[d] - yd);
      } else {
        y[d] = yd;
        if (MODE == KV_FIRST) xo[d] = xd;
      }
    }
  }
}

// Chebyshev sweeps on a coarse level with stored element matrices, each
// operator application and the vector update after it in one launch (the
// operator's result is not stored).  With d the step and r the
// preconditioned residual (the recurrences of gmg_cheb_*):
//   CH_FIRST: the first sweep from x = 0 through its first further step:
//             d0 = D1^-1 b / theta formed on the fly, r = D1^-1 b - D1^-1 A d0,
//             dn = c1 d0 + c2 r, x = d0 + dn;
//   CH_BEGIN: a later sweep's start, in = x: r = D1^-1 (b - A x), dn = r / theta,
//             xo = x + dn (xo distinct from x);
//   CH_STEP:  in = d: r -= D1^-1 A d, dn = c1 d + c2 r, x += dn (dn distinct
//             from d).
enum { CH_FIRST = 0, CH_BEGIN = 1, CH_STEP = 2 };

template <int MODE>
__global__ void __launch_bounds__(kB)
gmg_cheb_coarse(const float* __restrict__ K, const uint8_t* __restrict__ fixed, int nx, int ny,
                int nz, const float* __restrict__ in, const float* __restrict__ b,
                const float* __restrict__ dinv, float inv_theta, float c1, float c2,
                float* __restrict__ r, float* __restrict__ dn, float* __restrict__ x,
                float* __restrict__ xo) {
  const int64_t n_node = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  const int sub = threadIdx.x & 7;
  auto val = [&](int64_t q) -> float {
    return MODE == CH_FIRST ? inv_theta * (dinv[q] * b[q]) : in[q];
  };
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 3);
  const int64_t trips = (n_node + groups - 1) / groups;
  for (int64_t tr = 0; tr < trips; ++tr) {
    const int64_t nd = tr * groups + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3);
    float acc[3];
    coarse_rows(K, nx, ny, nz, nd, n_node, sub, val, acc);
    if (sub < 3 && nd < n_node) {
      const int64_t q = 3 * nd + sub;
      const float a = sub == 0 ? acc[0] : (sub == 1 ? acc[1] : acc[2]);
      const float vq = val(q);
      const float t = ((fixed[nd] >> sub) & 1) ? vq : a;
      if (MODE == CH_BEGIN) {
        const float ri = dinv[q] * (b[q] - t);
        const float di = inv_theta * ri;
        r[q] = ri;
        dn[q] = di;
        xo[q] = vq + di;
      } else {
        const float r0 = MODE == CH_FIRST ? dinv[q] * b[q] : r[q];
        const float ri = r0 - dinv[q] * t;
        const float di = c1 * vq + c2 * ri;
        r[q] = ri;
        dn[q] = di;
        x[q] = (MODE == CH_FIRST ? vq : x[q]) + di;
      }
    }
  }
}

// x = omega dinv b (first sweep from x = 0) or x += omega dinv (b - t)
__global__ void __launch_bounds__(kB)
gmg_smooth(float* __restrict__ x, const float* __restrict__ b, const float* __restrict__ t,
           const float* __restrict__ dinv, int64_t n, float omega, int first) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (first) x[i] = omega * dinv[i] * b[i];
    else x[i] += omega * dinv[i] * (b[i] - t[i]);
  }
}

// Chebyshev sweeps (the degree-k Chebyshev iteration for D1^-1 A x = D1^-1 b
// on [1/30, 1], 1 the l1 bound of lambda_max): r is the preconditioned
// residual, d the step.
//   first sweep from x = 0: r = D1^-1 b, d = r / theta, x = d;
//   later sweeps:           r = D1^-1 (b - t), t = A x, d = r / theta, x += d;
//   each further step:      r -= D1^-1 t, t = A d, d = c1 d + c2 r, x += d.
__global__ void __launch_bounds__(kB)
gmg_cheb_first(float* __restrict__ x, float* __restrict__ d, float* __restrict__ r,
               const float* __restrict__ b, const float* __restrict__ dinv, int64_t n,
               float inv_theta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float ri = dinv[i] * b[i];
    const float di = inv_theta * ri;
    r[i] = ri;
    d[i] = di;
    x[i] = di;
  }
}

__global__ void __launch_bounds__(kB)
gmg_cheb_begin(float* __restrict__ x, float* __restrict__ d, float* __restrict__ r,
               const float* __restrict__ b, const float* __restrict__ t,
               const float* __restrict__ dinv, int64_t n, float inv_theta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float ri = dinv[i] * (b[i] - t[i]);
    const float di = inv_theta * ri;
    r[i] = ri;
    d[i] = di;
    x[i] += di;
  }
}

__global__ void __launch_bounds__(kB)
gmg_cheb_step(float* __restrict__ x, float* __restrict__ d, float* __restrict__ r,
              const float* __restrict__ t, const float* __restrict__ dinv, int64_t n, float c1,
              float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float ri = r[i] - dinv[i] * t[i];
    const float di = c1 * d[i] + c2 * ri;
    r[i] = ri;
    d[i] = di;
    x[i] += di;
  }
}

// bc = Phat^T (b - t) (t = NULL: the residual is b); on fixed coarse DOFs
// zero, or xid there when given (the identity rows of a coarse operator
// applied as Phat^T A Phat).  One thread per coarse DOF.
__global__ void __launch_bounds__(kB)
gmg_restrict(const float* __restrict__ bf, const float* __restrict__ tf,
             const uint8_t* __restrict__ fixf, int nx, int ny, int nz,
             const uint8_t* __restrict__ fixc, int mx, int my, int mz, float* __restrict__ bc,
             const float* __restrict__ xid) {
  const int64_t n_cd = 3 * (int64_t)(mx + 1) * (my + 1) * (mz + 1);
  for (int64_t cd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cd < n_cd;
       cd += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cn = cd / 3;
    const int c = (int)(cd - 3 * cn);
    if ((fixc[cn] >> c) & 1) {
      bc[cd] = xid ? xid[cd] : 0.0f;
      continue;
    }
    const int I = (int)(cn % (mx + 1));
    const int J = (int)((cn / (mx + 1)) % (my + 1));
    const int K = (int)(cn / ((int64_t)(mx + 1) * (my + 1)));
    float acc = 0.0f;
    for (int dk = -1; dk <= 1; ++dk) {
      const int k = 2 * K + dk;
      if (k < 0 || k > nz) continue;
      const float wk = dk == 0 ? 1.0f : 0.5f;
      for (int dj = -1; dj <= 1; ++dj) {
        const int j = 2 * J + dj;
        if (j < 0 || j > ny) continue;
        const float wjk = wk * (dj == 0 ? 1.0f : 0.5f);
        for (int di = -1; di <= 1; ++di) {
          const int i = 2 * I + di;
          if (i < 0 || i > nx) continue;
          const int64_t f = nid(i, j, k, nx, ny);
          if ((fixf[f] >> c) & 1) continue;
          const float w = wjk * (di == 0 ? 1.0f : 0.5f);
          const float r = tf ? bf[3 * f + c] - tf[3 * f + c] : bf[3 * f + c];
          acc = fmaf(w, r, acc);
        }
      }
    }
    bc[cd] = acc;
  }
}

// xf += Phat xc on the free fine DOFs (add = 1), or xf = Phat xc (add = 0:
// the fixed fine DOFs written as zero)
__global__ void __launch_bounds__(kB)
gmg_prolong(const float* __restrict__ xc, const uint8_t* __restrict__ fixc, int mx, int my,
            const uint8_t* __restrict__ fixf, int nx, int ny, int nz, float* __restrict__ xf,
            int add) {
  const int64_t n_fn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n_fn;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(f % (nx + 1));
    const int j = (int)((f / (nx + 1)) % (ny + 1));
    const int k = (int)(f / ((int64_t)(nx + 1) * (ny + 1)));
    const uint8_t fm = fixf[f];
    if (fm == 7 && add) continue;
    const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1;
    const int k0 = k >> 1, k1 = (k + 1) >> 1;
    float acc[3] = {0.0f, 0.0f, 0.0f};
    for (int a = 0; a < 2; ++a) {
      const int K = a ? k1 : k0;
      if (a && k1 == k0) continue;
      const float wk = (k1 == k0) ? 1.0f : 0.5f;
      for (int b = 0; b < 2; ++b) {
        const int J = b ? j1 : j0;
        if (b && j1 == j0) continue;
        const float wjk = wk * ((j1 == j0) ? 1.0f : 0.5f);
        for (int d = 0; d < 2; ++d) {
          const int I = d ? i1 : i0;
          if (d && i1 == i0) continue;
          const float w = wjk * ((i1 == i0) ? 1.0f : 0.5f);
          const int64_t cn = nid(I, J, K, mx, my);
          const uint8_t cm = fixc[cn];
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (!((cm >> c) & 1)) acc[c] = fmaf(w, xc[3 * cn + c], acc[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const bool fixed_c = (fm >> c) & 1;
      if (add) {
        if (!fixed_c) xf[3 * f + c] += acc[c];
      } else {
        xf[3 * f + c] = fixed_c ? 0.0f : acc[c];
      }
    }
  }
}

// x = Cinv b, one warp per row
__global__ void __launch_bounds__(kB)
gmg_coarse_solve(const float* __restrict__ cinv, const float* __restrict__ b,
                 float* __restrict__ x, int n) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = w; r < n; r += nw) {
    float s = 0.0f;
    for (int q = lane; q < n; q += 32) s = fmaf(cinv[(int64_t)r * n + q], b[q], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[r] = s;
  }
}

// ---- outer FP64 CG kernels (fixed-order reductions through the handle's partials)

// r = f - q, r32 = r; sums r.r, f.f -> s[0], s[1]
__global__ void __launch_bounds__(kB)
gmg_resid0(const double* __restrict__ f, const double* __restrict__ q, double* __restrict__ r,
           float* __restrict__ r32, int64_t n, GmgScalars* s, double* partials) {
  __shared__ double sh[64];
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = f[i] - q[i];
    r[i] = ri;
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

// z = z32; sums r.z, z.r_old -> s[0], s[1]
__global__ void __launch_bounds__(kB)
gmg_zdot(const float* __restrict__ z32, const double* __restrict__ r,
         const double* __restrict__ r_old, double* __restrict__ z, int64_t n, int first,
         GmgScalars* s, double* partials) {
  __shared__ double sh[64];
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = (double)z32[i];
    z[i] = zi;
    acc[0] += r[i] * zi;
    if (!first) acc[1] += r_old[i] * zi;
  }
  double tot[2];
  if (last_block_reduce<2>(acc, partials, &s->ticket, tot, sh) && threadIdx.x == 0) {
    s->sum[0] = tot[0];
    s->sum[1] = tot[1];
  }
}

// p = z + beta p; first: p = z without reading p (it may hold anything,
// NaN bit patterns included, and 0 * NaN is NaN)
__global__ void __launch_bounds__(kB)
gmg_dir(const double* __restrict__ z, double* __restrict__ p, double beta, int64_t n, int first) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = first ? z[i] : z[i] + beta * p[i];
}

// p.q -> s[3]
__global__ void __launch_bounds__(kB)
gmg_pq(const double* __restrict__ p, const double* __restrict__ q, int64_t n, GmgScalars* s,
       double* partials) {
  __shared__ double sh[64];
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc[0] += p[i] * q[i];
  double tot[1];
  if (last_block_reduce<1>(acc, partials, &s->ticket, tot, sh) && threadIdx.x == 0)
    s->sum[3] = tot[0];
}

// u += alpha p; r_old = r; r -= alpha q; r32 = r; r.r -> s[2]
__global__ void __launch_bounds__(kB)
gmg_update(double* __restrict__ u, double* __restrict__ r, double* __restrict__ r_old,
           const double* __restrict__ p, const double* __restrict__ q, float* __restrict__ r32,
           double alpha, int64_t n, GmgScalars* s, double* partials) {
  __shared__ double sh[64];
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    u[i] += alpha * p[i];
    const double ro = r[i];
    r_old[i] = ro;
    const double rn = ro - alpha * q[i];
    r[i] = rn;
    r32[i] = (float)rn;
    acc[0] += rn * rn;
  }
  double tot[1];
  if (last_block_reduce<1>(acc, partials, &s->ticket, tot, sh) && threadIdx.x == 0)
    s->sum[2] = tot[0];
}

// ---- FP32 inner CG kernels of the mixed solve (FP64 sums)

// r.z, z.r_old -> s[0], s[1]
__global__ void __launch_bounds__(kB)
gmg_dot2_f32(const float* __restrict__ r, const float* __restrict__ r_old,
             const float* __restrict__ z, int64_t n, int first, GmgScalars* s, double* partials) {
  __shared__ double sh[64];
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = z[i];
    acc[0] += (double)r[i] * zi;
    if (!first) acc[1] += (double)r_old[i] * zi;
  }
  double tot[2];
  if (last_block_reduce<2>(acc, partials, &s->ticket, tot, sh) && threadIdx.x == 0) {
    s->sum[0] = tot[0];
    s->sum[1] = tot[1];
  }
}

// first direction of a continued inner CG: p = z + (r.z / (r.z)_prev) p, with
// r.z from the start's dot product (s[0]) and (r.z)_prev the previous inner
// CG's last (cg->rz, read before gmg_cg_start replaces it)
__global__ void __launch_bounds__(kB)
gmg_cont_dir_f32(const float* __restrict__ z, float* __restrict__ p, int64_t n,
                 const GmgScalars* s, const GmgCg* cg) {
  const double prev = cg->rz;
  const float beta = (prev > 0.0 && isfinite(prev)) ? (float)(s->sum[0] / prev) : 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = beta == 0.0f ? z[i] : z[i] + beta * p[i];
}

// first direction of an inner CG: p = z (p itself is not read)
__global__ void __launch_bounds__(kB)
gmg_first_dir_f32(const float* __restrict__ z, float* __restrict__ p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i];
}

// u += e
__global__ void __launch_bounds__(kB)
gmg_correct(double* __restrict__ u, const float* __restrict__ e, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    u[i] += (double)e[i];
}

// ---- FP32 inner CG steps with device-side scalars (graph-replayed chunks)

// start: rz from the first r.z (s[0]); done when there is nothing to do
__global__ void gmg_cg_start(GmgCg* cg, const GmgScalars* s, double tol2, int maxit) {
  cg->rz = s->sum[0];
  cg->alpha = cg->beta = 0.0;
  cg->tol2 = tol2;
  cg->it = 0;
  cg->maxit = maxit;
  cg->breakdown = 0;
  cg->done = (maxit < 1 || !(cg->rz > 0.0)) ? 1 : 0;
}

// p.q, then alpha = rz / p.q (breakdown ends the solve)
__global__ void __launch_bounds__(kB)
gmg_cg_pq(const float* __restrict__ p, const float* __restrict__ q, int64_t n, GmgCg* cg,
          double* partials) {
  if (*(volatile int32_t*)&cg->done) return;
  __shared__ double sh[64];
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc[0] += (double)p[i] * q[i];
  double tot[1];
  if (last_block_reduce<1>(acc, partials, &cg->ticket, tot, sh) && threadIdx.x == 0) {
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      cg->breakdown = 1;
      cg->done = 1;
    } else {
      cg->alpha = cg->rz / tot[0];
    }
  }
}

// e += alpha p; r_old = r; r -= alpha q; done when r.r <= tol2 or at maxit
__global__ void __launch_bounds__(kB)
gmg_cg_update(float* __restrict__ e, float* __restrict__ r, float* __restrict__ r_old,
              const float* __restrict__ p, const float* __restrict__ q, int64_t n, GmgCg* cg,
              double* partials) {
  if (*(volatile int32_t*)&cg->done) return;
  __shared__ double sh[64];
  const float alpha = (float)cg->alpha;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    e[i] += alpha * p[i];
    const float ro = r[i];
    r_old[i] = ro;
    const float rn = ro - alpha * q[i];
    r[i] = rn;
    acc[0] += (double)rn * rn;
  }
  double tot[1];
  if (last_block_reduce<1>(acc, partials, &cg->ticket, tot, sh) && threadIdx.x == 0) {
    cg->it += 1;
    if (!(tot[0] > cg->tol2) || cg->it >= cg->maxit) cg->done = 1;
  }
}

// r.z, z.r_old, then the Polak-Ribiere beta and rz
__global__ void __launch_bounds__(kB)
gmg_cg_beta(const float* __restrict__ r, const float* __restrict__ r_old,
            const float* __restrict__ z, int64_t n, GmgCg* cg, double* partials) {
  if (*(volatile int32_t*)&cg->done) return;
  __shared__ double sh[64];
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = z[i];
    acc[0] += (double)r[i] * zi;
    acc[1] += (double)r_old[i] * zi;
  }
  double tot[2];
  if (last_block_reduce<2>(acc, partials, &cg->ticket, tot, sh) && threadIdx.x == 0) {
    cg->beta = (tot[0] - tot[1]) / cg->rz;
    cg->rz = tot[0];
  }
}

__global__ void __launch_bounds__(kB)
gmg_cg_dir(const float* __restrict__ z, float* __restrict__ p, int64_t n, const GmgCg* cg) {
  if (*(volatile const int32_t*)&cg->done) return;
  const float beta = (float)cg->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// ---------------------------------------------------------------- host side

void level_dims(const mfto_handle* h, const mfto_gmg_params& p, int* n_levels, int dims[][3]) {
  int nx = h->mesh.nelx, ny = h->mesh.nely, nz = h->mesh.nelz;
  int L = 0;
  dims[0][0] = nx; dims[0][1] = ny; dims[0][2] = nz;
  L = 1;
  while (L < p.max_levels) {
    const int64_t dofs = 3LL * (nx + 1) * (ny + 1) * (nz + 1);
    if (dofs <= p.coarse_max_dofs || (nx == 1 && ny == 1 && nz == 1)) break;
    nx = (nx + 1) / 2; ny = (ny + 1) / 2; nz = (nz + 1) / 2;
    dims[L][0] = nx; dims[L][1] = ny; dims[L][2] = nz;
    ++L;
  }
  *n_levels = L;
}

void drop_graph(GmgWs* w) {
  if (w->vexec) cudaGraphExecDestroy(w->vexec);
  w->vexec = nullptr;
  if (w->cexec) cudaGraphExecDestroy(w->cexec);
  w->cexec = nullptr;
  w->vkey_r = nullptr;
  w->vkey_z = nullptr;
}

void free_levels(GmgWs* w) {
  drop_graph(w);
  for (int l = 0; l < MFTO_GMG_MAX_LEVELS; ++l) {
    GmgLevel& v = w->lv[l];
    if (l > 0 && v.d_fixed) cudaFree(v.d_fixed);
    void* ptrs[] = {v.d_K, v.d_dinv, v.x, v.x2, v.b, v.t, v.cr, v.cd};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    v = GmgLevel();
  }
  if (w->d_cinv) cudaFree(w->d_cinv);
  w->d_cinv = nullptr;
  if (w->mf_s0) cudaFree(w->mf_s0);
  if (w->mf_s1) cudaFree(w->mf_s1);
  w->mf_s0 = w->mf_s1 = nullptr;
  w->mf1 = false;
  w->n_levels = 0;
  w->ready = false;
}

mfto_status gmg_alloc(mfto_handle* h, GmgWs* w, const mfto_gmg_params& p) {
  int L;
  int dims[MFTO_GMG_MAX_LEVELS][3];
  level_dims(h, p, &L, dims);
  bool same = L == w->n_levels && w->d_cinv;
  for (int l = 0; same && l < L; ++l)
    same = w->lv[l].nx == dims[l][0] && w->lv[l].ny == dims[l][1] && w->lv[l].nz == dims[l][2];
  if (same) return MFTO_OK;
  free_levels(w);
  const int64_t nc = 3LL * (dims[L - 1][0] + 1) * (dims[L - 1][1] + 1) * (dims[L - 1][2] + 1);
  if (nc > MFTO_GMG_MAX_COARSE)
    return mfto_fail(h, MFTO_TOO_LARGE,
                     "mfto_gmg_setup: the coarsest level has %lld DOFs (at most %d): allow more "
                     "levels", (long long)nc, MFTO_GMG_MAX_COARSE);
  // per-level node masks on the host: level 0 from the handle
  w->h_fixed.assign(L, {});
  w->h_fixed[0].resize(h->n_node);
  MFTO_CUDA(h, cudaMemcpy(w->h_fixed[0].data(), h->d_fixed, h->n_node, cudaMemcpyDeviceToHost));
  for (int l = 1; l < L; ++l) {
    const int nx = dims[l - 1][0], ny = dims[l - 1][1], nz = dims[l - 1][2];
    const int mx = dims[l][0], my = dims[l][1], mz = dims[l][2];
    std::vector<uint8_t>& fc = w->h_fixed[l];
    fc.assign((size_t)(mx + 1) * (my + 1) * (mz + 1), 0);
    for (int K = 0; K <= mz; ++K)
      for (int J = 0; J <= my; ++J)
        for (int I = 0; I <= mx; ++I)
          if (2 * I <= nx && 2 * J <= ny && 2 * K <= nz)
            fc[nid(I, J, K, mx, my)] = w->h_fixed[l - 1][nid(2 * I, 2 * J, 2 * K, nx, ny)];
  }
  w->n_levels = L;
  for (int l = 0; l < L; ++l) {
    GmgLevel& v = w->lv[l];
    v.nx = dims[l][0]; v.ny = dims[l][1]; v.nz = dims[l][2];
    v.n_elem = (int64_t)v.nx * v.ny * v.nz;
    v.n_node = (int64_t)(v.nx + 1) * (v.ny + 1) * (v.nz + 1);
    v.n_dof = 3 * v.n_node;
    auto A = [&](void** ptr, size_t bytes) -> mfto_status {
      const cudaError_t e = cudaMalloc(ptr, bytes);
      if (e == cudaSuccess) return MFTO_OK;
      cudaGetLastError();
      free_levels(w);
      return mfto_fail(h, MFTO_OOM, "mfto_gmg_setup: cudaMalloc of %zu bytes failed", bytes);
    };
    mfto_status s;
    if (l == 0) {
      v.d_fixed = h->d_fixed;
    } else {
      if ((s = A((void**)&v.d_fixed, v.n_node)) != MFTO_OK) return s;
      MFTO_CUDA(h, cudaMemcpy(v.d_fixed, w->h_fixed[l].data(), v.n_node, cudaMemcpyHostToDevice));
      if ((s = A((void**)&v.d_K, sizeof(float) * 576 * v.n_elem)) != MFTO_OK) return s;
      if ((s = A((void**)&v.x, sizeof(float) * v.n_dof)) != MFTO_OK) return s;
      if ((s = A((void**)&v.x2, sizeof(float) * v.n_dof)) != MFTO_OK) return s;
      if ((s = A((void**)&v.b, sizeof(float) * v.n_dof)) != MFTO_OK) return s;
    }
    if ((s = A((void**)&v.d_dinv, sizeof(float) * v.n_dof)) != MFTO_OK) return s;
    if ((s = A((void**)&v.t, sizeof(float) * v.n_dof)) != MFTO_OK) return s;
  }
  w->n_c = (int)nc;
  if (cudaMalloc((void**)&w->d_cinv, sizeof(float) * nc * nc) != cudaSuccess) {
    cudaGetLastError();
    free_levels(w);
    return mfto_fail(h, MFTO_OOM, "mfto_gmg_setup: cudaMalloc of the coarse inverse failed");
  }
  return MFTO_OK;
}

// Dense inverse of the coarsest operator from its element matrices (FP64 on
// the host: Cholesky, then the inverse column by column).
mfto_status coarse_inverse(mfto_handle* h, GmgWs* w) {
  const int L = w->n_levels - 1;
  const GmgLevel& v = w->lv[L];
  const int n = (int)v.n_dof;
  std::vector<float> Ke((size_t)576 * v.n_elem);
  if (L == 0) {   // single level: E_e D_e KE D_e from the moduli and the unit matrix
    std::vector<float> E(v.n_elem), ke(576);
    MFTO_CUDA(h, cudaMemcpyAsync(E.data(), w->d_E32, sizeof(float) * v.n_elem,
                                 cudaMemcpyDeviceToHost, h->stream));
    MFTO_CUDA(h, cudaMemcpyAsync(ke.data(), h->d_ke32, sizeof(float) * 576,
                                 cudaMemcpyDeviceToHost, h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int64_t e = 0; e < v.n_elem; ++e)
      for (int q = 0; q < 576; ++q) Ke[e * 576 + q] = E[e] * ke[q];
  } else {
    MFTO_CUDA(h, cudaMemcpyAsync(Ke.data(), v.d_K, sizeof(float) * 576 * v.n_elem,
                                 cudaMemcpyDeviceToHost, h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  const std::vector<uint8_t>& fx = w->h_fixed[L];
  auto is_fixed = [&](int64_t dof) { return (fx[dof / 3] >> (dof % 3)) & 1; };
  std::vector<double> Am((size_t)n * n, 0.0);
  for (int ez = 0; ez < v.nz; ++ez)
    for (int ey = 0; ey < v.ny; ++ey)
      for (int ex = 0; ex < v.nx; ++ex) {
        const int64_t e = ex + (int64_t)v.nx * (ey + (int64_t)v.ny * ez);
        int64_t dof[24];
        for (int lb = 0; lb < 8; ++lb) {
          const int64_t m = nid(ex + (lb & 1), ey + ((lb >> 1) & 1), ez + (lb >> 2), v.nx, v.ny);
          for (int c = 0; c < 3; ++c) dof[3 * lb + c] = 3 * m + c;
        }
        for (int a = 0; a < 24; ++a) {
          if (is_fixed(dof[a])) continue;
          for (int b = 0; b < 24; ++b)
            if (!is_fixed(dof[b])) Am[dof[a] * n + dof[b]] += Ke[e * 576 + a * 24 + b];
        }
      }
  for (int64_t d = 0; d < n; ++d)
    if (is_fixed(d)) Am[d * n + d] = 1.0;
  // Cholesky, lower triangle in place.  A pivot below 1e-5 of its diagonal
  // entry marks a rank-deficient operator (a consistent singular problem:
  // free rigid motions, as in the MBB preset); it is then factorised again
  // with the diagonal scaled by 1 + delta, delta = 1e-6, 1e-5, ... 1e-2, the
  // first that makes it positive definite (the FP32-rounded element matrices
  // can leave the null space's eigenvalues slightly negative), which keeps
  // the cycle SPD.
  const std::vector<double> A0 = Am;
  double shift = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = Am[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= Am[(size_t)j * n + k] * Am[(size_t)j * n + k];
    // a shifted operator only has to be positive definite
    if (!(s > (shift > 0.0 ? 0.0 : 1e-5 * A0[(size_t)j * n + j])) || !std::isfinite(s)) {
      shift = shift > 0.0 ? 10.0 * shift : 1e-6;
      if (shift > 1.5e-2 || !std::isfinite(s))
        return mfto_fail(h, MFTO_BREAKDOWN,
                         "mfto_gmg_setup: coarsest operator not positive definite");
      Am = A0;
      for (int i = 0; i < n; ++i) Am[(size_t)i * n + i] *= 1.0 + shift;
      j = -1;                           // restart the factorisation
      continue;
    }
    const double d = sqrt(s);
    Am[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = Am[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= Am[(size_t)i * n + k] * Am[(size_t)j * n + k];
      Am[(size_t)i * n + j] = t / d;
    }
  }
  // L^T row-major, so that both substitutions read contiguous rows
  std::vector<double> Lt((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k <= i; ++k) Lt[(size_t)k * n + i] = Am[(size_t)i * n + k];
  std::vector<float> inv((size_t)n * n);
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < c; ++i) col[i] = 0.0;
    for (int i = c; i < n; ++i) {       // L y = e_c (y is zero above row c)
      double t = (i == c) ? 1.0 : 0.0;
      const double* Li = &Am[(size_t)i * n];
      for (int k = c; k < i; ++k) t -= Li[k] * col[k];
      col[i] = t / Li[i];
    }
    for (int i = n - 1; i >= 0; --i) {  // L^T x = y
      double t = col[i];
      const double* Ri = &Lt[(size_t)i * n];
      for (int k = i + 1; k < n; ++k) t -= Ri[k] * col[k];
      col[i] = t / Ri[i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = (float)col[i];
  }
  MFTO_CUDA(h, cudaMemcpy(w->d_cinv, inv.data(), sizeof(float) * inv.size(),
                          cudaMemcpyHostToDevice));
  return MFTO_OK;
}

mfto_status apply_level(mfto_handle* h, GmgWs* w, int l, const float* x, float* y) {
  if (l == 0) return kv_launch(h, (mfto_form)w->prm.smoother_form, w->d_E32, x, y);
  const GmgLevel& v = w->lv[l];
  if (l == 1 && w->mf1) {
    // A_1 x = Phat^T K (Phat x) with the FP32 fine operator: no element
    // matrices read (the stored ones serve the setup only)
    const GmgLevel& f = w->lv[0];
    h->launches++;
    gmg_prolong<<<grid_of(f.n_node), kB, 0, h->stream>>>(x, v.d_fixed, v.nx, v.ny, f.d_fixed, f.nx,
                                                         f.ny, f.nz, w->mf_s0, 0);
    MFTO_LAUNCH_CHECK(h);
    mfto_status s = kv_launch(h, MFTO_FORM_F32, w->d_E32, w->mf_s0, w->mf_s1);
    if (s != MFTO_OK) return s;
    h->launches++;
    gmg_restrict<<<grid_of(v.n_dof), kB, 0, h->stream>>>(w->mf_s1, nullptr, f.d_fixed, f.nx, f.ny,
                                                         f.nz, v.d_fixed, v.nx, v.ny, v.nz, y, x);
    MFTO_LAUNCH_CHECK(h);
    return MFTO_OK;
  }
  h->launches++;
  gmg_kv_coarse<KV_PLAIN><<<grid_of(8 * v.n_node), kB, 0, h->stream>>>(
      v.d_K, v.d_fixed, v.nx, v.ny, v.nz, x, nullptr, nullptr, 0.0f, y, nullptr);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

// Chebyshev coefficients on [1/30, 1]: 1/theta and (c1, c2) per further step
struct ChebCoef {
  float inv_theta;
  float c1[8], c2[8];
};

ChebCoef cheb_coef(int degree) {
  ChebCoef c{};
  const double lmax = 1.0, lmin = 1.0 / 30.0;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  c.inv_theta = (float)(1.0 / theta);
  for (int k = 0; k + 1 < degree && k < 8; ++k) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    c.c1[k] = (float)(rho_new * rho);
    c.c2[k] = (float)(2.0 * rho_new / delta);
    rho = rho_new;
  }
  return c;
}

// `sweeps` Chebyshev sweeps on level l (from zero when first); on exit v.t is
// not A x.
mfto_status cheb_sweeps(mfto_handle* h, GmgWs* w, int l, const float* b, float* x, int sweeps,
                        bool from_zero) {
  const GmgLevel& v = w->lv[l];
  const ChebCoef c = cheb_coef(w->cheb);
  const int g = grid_of(v.n_dof);
  mfto_status s;
  for (int sw = 0; sw < sweeps; ++sw) {
    h->launches++;
    if (sw == 0 && from_zero) {
      gmg_cheb_first<<<g, kB, 0, h->stream>>>(x, v.cd, v.cr, b, v.d_dinv, v.n_dof, c.inv_theta);
    } else {
      if ((s = apply_level(h, w, l, x, v.t)) != MFTO_OK) return s;
      gmg_cheb_begin<<<g, kB, 0, h->stream>>>(x, v.cd, v.cr, b, v.t, v.d_dinv, v.n_dof,
                                              c.inv_theta);
    }
    MFTO_LAUNCH_CHECK(h);
    for (int k = 0; k + 1 < w->cheb; ++k) {
      if ((s = apply_level(h, w, l, v.cd, v.t)) != MFTO_OK) return s;
      h->launches++;
      gmg_cheb_step<<<g, kB, 0, h->stream>>>(x, v.cd, v.cr, v.t, v.d_dinv, v.n_dof, c.c1[k],
                                             c.c2[k]);
      MFTO_LAUNCH_CHECK(h);
    }
  }
  return MFTO_OK;
}

// The same sweeps on a coarse level with stored matrices (degree >= 2), one
// launch per operator application (gmg_cheb_coarse): a sweep from zero is
// degree - 1 launches, a later one degree.  A later sweep writes its iterate
// to `other` and swaps the two; the step alternates between v.cd and v.t (on
// exit v.t is not A x).
mfto_status cheb_sweeps_coarse(mfto_handle* h, GmgWs* w, int l, const float* b, float*& x,
                               float*& other, int sweeps, bool from_zero) {
  const GmgLevel& v = w->lv[l];
  const ChebCoef c = cheb_coef(w->cheb);
  const int gk = grid_of(8 * v.n_node);
  float* d = v.cd;
  float* dn = v.t;
  for (int sw = 0; sw < sweeps; ++sw) {
    int k = 0;
    h->launches++;
    if (sw == 0 && from_zero) {
      gmg_cheb_coarse<CH_FIRST><<<gk, kB, 0, h->stream>>>(
          v.d_K, v.d_fixed, v.nx, v.ny, v.nz, nullptr, b, v.d_dinv, c.inv_theta, c.c1[0],
          c.c2[0], v.cr, d, x, nullptr);
      k = 1;
    } else {
      gmg_cheb_coarse<CH_BEGIN><<<gk, kB, 0, h->stream>>>(
          v.d_K, v.d_fixed, v.nx, v.ny, v.nz, x, b, v.d_dinv, c.inv_theta, 0.0f, 0.0f, v.cr, d,
          nullptr, other);
      std::swap(x, other);
    }
    MFTO_LAUNCH_CHECK(h);
    for (; k + 1 < w->cheb; ++k) {
      h->launches++;
      gmg_cheb_coarse<CH_STEP><<<gk, kB, 0, h->stream>>>(
          v.d_K, v.d_fixed, v.nx, v.ny, v.nz, d, nullptr, v.d_dinv, 0.0f, c.c1[k], c.c2[k], v.cr,
          dn, x, nullptr);
      MFTO_LAUNCH_CHECK(h);
      std::swap(d, dn);
    }
  }
  return MFTO_OK;
}

mfto_status vcycle(mfto_handle* h, GmgWs* w, int l, const float* b, float* x,
                   float** out = nullptr);

// Level 0 with its l1-Jacobi sweeps fused into the FP32 column K.v: the
// pre-smoothed iterate lives in the level's two scratch buffers, the last
// post-sweep writes the caller's x.
mfto_status vcycle_level0_fused(mfto_handle* h, GmgWs* w, const float* b, float* x) {
  const GmgLevel& v = w->lv[0];
  const GmgLevel& c = w->lv[1];
  const mfto_gmg_params& p = w->prm;
  const float om = (float)p.omega;
  float* cur = v.x;
  auto other = [&](const float* q) { return q == v.x ? v.x2 : v.x; };
  mfto_status s;
  if (p.nu_pre == 0) {
    MFTO_CUDA(h, cudaMemsetAsync(cur, 0, sizeof(float) * v.n_dof, h->stream));
  } else {
    if ((s = gmg_sweep_col_launch(h, true, w->d_E32, b, v.d_dinv, om, nullptr, cur, v.t)) !=
        MFTO_OK)
      return s;
    for (int k = 1; k < p.nu_pre; ++k) {
      float* dst = other(cur);
      if ((s = gmg_sweep_col_launch(h, false, w->d_E32, b, v.d_dinv, om, cur, dst, nullptr)) !=
          MFTO_OK)
        return s;
      cur = dst;
    }
    if (p.nu_pre > 1 && (s = apply_level(h, w, 0, cur, v.t)) != MFTO_OK) return s;
  }
  h->launches++;
  gmg_restrict<<<grid_of(c.n_dof), kB, 0, h->stream>>>(
      b, p.nu_pre ? v.t : nullptr, v.d_fixed, v.nx, v.ny, v.nz, c.d_fixed, c.nx, c.ny, c.nz, c.b,
      nullptr);
  MFTO_LAUNCH_CHECK(h);
  float* xc = nullptr;
  if ((s = vcycle(h, w, 1, c.b, c.x, &xc)) != MFTO_OK) return s;
  h->launches++;
  gmg_prolong<<<grid_of(v.n_node), kB, 0, h->stream>>>(xc, c.d_fixed, c.nx, c.ny, v.d_fixed,
                                                       v.nx, v.ny, v.nz, cur, 1);
  MFTO_LAUNCH_CHECK(h);
  if (p.nu_post == 0) {
    MFTO_CUDA(h, cudaMemcpyAsync(x, cur, sizeof(float) * v.n_dof, cudaMemcpyDeviceToDevice,
                                 h->stream));
    return MFTO_OK;
  }
  for (int k = 0; k < p.nu_post; ++k) {
    float* dst = k + 1 == p.nu_post ? x : other(cur);
    if ((s = gmg_sweep_col_launch(h, false, w->d_E32, b, v.d_dinv, om, cur, dst, nullptr)) !=
        MFTO_OK)
      return s;
    cur = dst;
  }
  return MFTO_OK;
}

// Level 0 with Chebyshev sweeps (degree >= 2) fused into the FP32 column K.v
// (gmg_cheb_col_launch): the iterate lives in the level's two scratch buffers,
// the step alternates between v.cd and v.t, and the last post-smoothing
// launch (always a step) writes the caller's x.
mfto_status vcycle_level0_cheb(mfto_handle* h, GmgWs* w, const float* b, float* x) {
  const GmgLevel& v = w->lv[0];
  const GmgLevel& c = w->lv[1];
  const mfto_gmg_params& p = w->prm;
  const ChebCoef cc = cheb_coef(w->cheb);
  float* cur = v.x;
  float* oth = v.x2;
  float* d = v.cd;
  float* dn = v.t;
  // `sweeps` sweeps; the last step of the last one writes `dst` when given
  auto sweeps = [&](int n, bool from_zero, float* dst) -> mfto_status {
    mfto_status s;
    for (int sw = 0; sw < n; ++sw) {
      int k = 0;
      if (sw == 0 && from_zero) {
        if ((s = gmg_cheb_col_launch(h, GMG_CHEB_FIRST, w->d_E32, nullptr, b, v.d_dinv,
                                     cc.inv_theta, cc.c1[0], cc.c2[0], v.cr, d, nullptr, cur)) !=
            MFTO_OK)
          return s;
        k = 1;
      } else {
        if ((s = gmg_cheb_col_launch(h, GMG_CHEB_BEGIN, w->d_E32, cur, b, v.d_dinv,
                                     cc.inv_theta, 0.0f, 0.0f, v.cr, d, nullptr, oth)) != MFTO_OK)
          return s;
        std::swap(cur, oth);
      }
      for (; k + 1 < w->cheb; ++k) {
        const bool last = dst && sw + 1 == n && k + 2 == w->cheb;
        if ((s = gmg_cheb_col_launch(h, GMG_CHEB_STEP, w->d_E32, d, nullptr, v.d_dinv, 0.0f,
                                     cc.c1[k], cc.c2[k], v.cr, dn, cur, last ? dst : cur)) !=
            MFTO_OK)
          return s;
        std::swap(d, dn);
        if (last) cur = dst;
      }
    }
    return MFTO_OK;
  };
  mfto_status s;
  if (p.nu_pre == 0) {
    MFTO_CUDA(h, cudaMemsetAsync(cur, 0, sizeof(float) * v.n_dof, h->stream));
  } else {
    if ((s = sweeps(p.nu_pre, true, nullptr)) != MFTO_OK) return s;
    if ((s = apply_level(h, w, 0, cur, v.t)) != MFTO_OK) return s;
  }
  h->launches++;
  gmg_restrict<<<grid_of(c.n_dof), kB, 0, h->stream>>>(
      b, p.nu_pre ? v.t : nullptr, v.d_fixed, v.nx, v.ny, v.nz, c.d_fixed, c.nx, c.ny, c.nz, c.b,
      nullptr);
  MFTO_LAUNCH_CHECK(h);
  float* xc = nullptr;
  if ((s = vcycle(h, w, 1, c.b, c.x, &xc)) != MFTO_OK) return s;
  h->launches++;
  gmg_prolong<<<grid_of(v.n_node), kB, 0, h->stream>>>(xc, c.d_fixed, c.nx, c.ny, v.d_fixed,
                                                       v.nx, v.ny, v.nz, cur, 1);
  MFTO_LAUNCH_CHECK(h);
  if (p.nu_post == 0) {
    MFTO_CUDA(h, cudaMemcpyAsync(x, cur, sizeof(float) * v.n_dof, cudaMemcpyDeviceToDevice,
                                 h->stream));
    return MFTO_OK;
  }
  return sweeps(p.nu_post, false, x);
}

// One V-cycle from level l: b the right-hand side, x the caller's output
// buffer on level 0; on coarse levels the result lands in lv[l].x or
// lv[l].x2 (fused sweeps alternate between them) and *out says which.
mfto_status vcycle(mfto_handle* h, GmgWs* w, int l, const float* b, float* x, float** out) {
  const int L = w->n_levels - 1;
  const GmgLevel& v = w->lv[l];
  const mfto_gmg_params& p = w->prm;
  mfto_status s;
  if (out) *out = x;
  if (l == L) {
    h->launches++;
    gmg_coarse_solve<<<std::max(1, std::min(1024, (w->n_c + 7) / 8)), kB, 0, h->stream>>>(
        w->d_cinv, b, x, w->n_c);
    MFTO_LAUNCH_CHECK(h);
    return MFTO_OK;
  }
  const int g = grid_of(v.n_dof);
  const int gk = grid_of(8 * v.n_node);
  const float om = (float)p.omega;
  // coarse levels with stored matrices: sweep and operator in one launch
  const bool cheb = w->cheb > 0;
  const bool stored = l > 0 && !(l == 1 && w->mf1);
  const bool fused = stored && !cheb;
  const bool cheb_fused = stored && w->cheb >= 2;
  if (l == 0 && v.x && v.x2 && p.smoother_form == MFTO_FORM_F32 && h->kv_variant == 0) {
    if (!cheb) return vcycle_level0_fused(h, w, b, x);
    if (w->cheb >= 2) return vcycle_level0_cheb(h, w, b, x);
  }
  float* other = fused || cheb_fused ? (x == v.x ? v.x2 : v.x) : nullptr;
  // pre-smoothing; on exit v.t = A x
  if (p.nu_pre == 0) {
    MFTO_CUDA(h, cudaMemsetAsync(x, 0, sizeof(float) * v.n_dof, h->stream));
  } else if (cheb) {
    if ((s = cheb_fused ? cheb_sweeps_coarse(h, w, l, b, x, other, p.nu_pre, true)
                        : cheb_sweeps(h, w, l, b, x, p.nu_pre, true)) != MFTO_OK)
      return s;
    if ((s = apply_level(h, w, l, x, v.t)) != MFTO_OK) return s;
  } else if (fused) {
    h->launches++;
    gmg_kv_coarse<KV_FIRST><<<gk, kB, 0, h->stream>>>(v.d_K, v.d_fixed, v.nx, v.ny, v.nz, nullptr,
                                                      b, v.d_dinv, om, v.t, x);
    MFTO_LAUNCH_CHECK(h);
    for (int k = 1; k < p.nu_pre; ++k) {
      h->launches++;
      gmg_kv_coarse<KV_SMOOTH><<<gk, kB, 0, h->stream>>>(v.d_K, v.d_fixed, v.nx, v.ny, v.nz, x,
                                                         b, v.d_dinv, om, nullptr, other);
      MFTO_LAUNCH_CHECK(h);
      std::swap(x, other);
    }
    if (p.nu_pre > 1 && (s = apply_level(h, w, l, x, v.t)) != MFTO_OK) return s;
  } else {
    for (int k = 0; k < p.nu_pre; ++k) {
      if (k > 0 && (s = apply_level(h, w, l, x, v.t)) != MFTO_OK) return s;
      h->launches++;
      gmg_smooth<<<g, kB, 0, h->stream>>>(x, b, v.t, v.d_dinv, v.n_dof, om, k == 0);
      MFTO_LAUNCH_CHECK(h);
    }
    if ((s = apply_level(h, w, l, x, v.t)) != MFTO_OK) return s;
  }
  const GmgLevel& c = w->lv[l + 1];
  h->launches++;
  gmg_restrict<<<grid_of(c.n_dof), kB, 0, h->stream>>>(
      b, p.nu_pre ? v.t : nullptr, v.d_fixed, v.nx, v.ny, v.nz, c.d_fixed, c.nx, c.ny, c.nz, c.b,
      nullptr);
  MFTO_LAUNCH_CHECK(h);
  float* xc = nullptr;
  if ((s = vcycle(h, w, l + 1, c.b, c.x, &xc)) != MFTO_OK) return s;
  h->launches++;
  gmg_prolong<<<grid_of(v.n_node), kB, 0, h->stream>>>(xc, c.d_fixed, c.nx, c.ny, v.d_fixed,
                                                       v.nx, v.ny, v.nz, x, 1);
  MFTO_LAUNCH_CHECK(h);
  if (cheb) {
    if ((s = cheb_fused ? cheb_sweeps_coarse(h, w, l, b, x, other, p.nu_post, false)
                        : cheb_sweeps(h, w, l, b, x, p.nu_post, false)) != MFTO_OK)
      return s;
    if (out) *out = x;
    return MFTO_OK;
  }
  for (int k = 0; k < p.nu_post; ++k) {
    if (fused) {
      h->launches++;
      gmg_kv_coarse<KV_SMOOTH><<<gk, kB, 0, h->stream>>>(v.d_K, v.d_fixed, v.nx, v.ny, v.nz, x,
                                                         b, v.d_dinv, om, nullptr, other);
      MFTO_LAUNCH_CHECK(h);
      std::swap(x, other);
    } else {
      if ((s = apply_level(h, w, l, x, v.t)) != MFTO_OK) return s;
      h->launches++;
      gmg_smooth<<<g, kB, 0, h->stream>>>(x, b, v.t, v.d_dinv, v.n_dof, om, 0);
      MFTO_LAUNCH_CHECK(h);
    }
  }
  if (out) *out = x;
  return MFTO_OK;
}

// The V-cycle for (r, z) as one graph launch: captured on the handle's
// private capture stream the first time (and again when the buffers, the
// parameters or the hierarchy's storage change), replayed on the stream.
mfto_status vcycle_graph(mfto_handle* h, GmgWs* w, const float* r, float* z) {
  const mfto_gmg_params &a = w->vprm, &b = w->prm;
  const bool same = w->vexec && w->vkey_r == r && w->vkey_z == z &&
                    a.max_levels == b.max_levels && a.coarse_max_dofs == b.coarse_max_dofs &&
                    a.nu_pre == b.nu_pre && a.nu_post == b.nu_post && a.omega == b.omega &&
                    a.smoother_form == b.smoother_form && a.matfree_level1 == b.matfree_level1 &&
                    a.cheb_degree == b.cheb_degree;
  if (!same) {
    drop_graph(w);
    if (!h->cap_stream &&
        cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return mfto_fail(h, MFTO_CUDA_ERROR, "V-cycle graph: cannot create the capture stream");
    cudaStream_t saved = h->stream;
    const bool timing = h->kv_timing;
    const int64_t launches = h->launches;
    h->kv_timing = false;
    h->stream = h->cap_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    mfto_status s = e == cudaSuccess ? vcycle(h, w, 0, r, z) : MFTO_CUDA_ERROR;
    if (e == cudaSuccess) e = cudaStreamEndCapture(h->cap_stream, &graph);
    h->stream = saved;
    h->kv_timing = timing;
    w->vnodes = h->launches - launches;
    h->launches = launches;
    if (s != MFTO_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return s != MFTO_OK ? s
                          : mfto_fail(h, MFTO_CUDA_ERROR, "V-cycle graph capture: %s",
                                      cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&w->vexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      w->vexec = nullptr;
      return mfto_fail(h, MFTO_CUDA_ERROR, "V-cycle graph instantiate: %s", cudaGetErrorString(e));
    }
    w->vkey_r = r;
    w->vkey_z = z;
    w->vprm = w->prm;
  }
  MFTO_CUDA(h, cudaGraphLaunch(w->vexec, h->stream));
  h->launches += w->vnodes;
  return MFTO_OK;
}

// cg_chunk_len inner CG iterations on the handle's FP32 vectors as one graph
mfto_status cg_chunk_graph(mfto_handle* h, GmgWs* w) {
  const mfto_gmg_params &a = w->cprm, &b = w->prm;
  const int chunk = cg_chunk_len(h);
  const bool same = w->cexec && w->cchunk == chunk && a.max_levels == b.max_levels &&
                    a.coarse_max_dofs == b.coarse_max_dofs && a.nu_pre == b.nu_pre &&
                    a.nu_post == b.nu_post && a.omega == b.omega &&
                    a.smoother_form == b.smoother_form && a.matfree_level1 == b.matfree_level1 &&
                    a.cheb_degree == b.cheb_degree;
  if (!same) {
    if (w->cexec) cudaGraphExecDestroy(w->cexec);
    w->cexec = nullptr;
    if (!h->cap_stream &&
        cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return mfto_fail(h, MFTO_CUDA_ERROR, "CG graph: cannot create the capture stream");
    const int64_t n = h->n_dof;
    const int g = reduction_blocks(n, kB);
    float *r32 = h->d_r32, *z32 = h->d_z32, *p32 = h->d_p0_32, *q32 = h->d_q32,
          *e32 = h->d_e32, *ro32 = h->d_p1_32;
    cudaStream_t saved = h->stream;
    const bool timing = h->kv_timing;
    const int64_t launches = h->launches;
    h->kv_timing = false;
    h->stream = h->cap_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    mfto_status s = e == cudaSuccess ? MFTO_OK : MFTO_CUDA_ERROR;
    for (int k = 0; k < chunk && s == MFTO_OK; ++k) {
      s = kv_launch(h, MFTO_FORM_F32, w->d_E32, p32, q32);
      if (s != MFTO_OK) break;
      h->launches += 2;
      gmg_cg_pq<<<g, kB, 0, h->stream>>>(p32, q32, n, w->d_cg, h->d_partials);
      gmg_cg_update<<<g, kB, 0, h->stream>>>(e32, r32, ro32, p32, q32, n, w->d_cg,
                                             h->d_partials);
      s = vcycle(h, w, 0, r32, z32);
      if (s != MFTO_OK) break;
      h->launches += 2;
      gmg_cg_beta<<<g, kB, 0, h->stream>>>(r32, ro32, z32, n, w->d_cg, h->d_partials);
      gmg_cg_dir<<<g, kB, 0, h->stream>>>(z32, p32, n, w->d_cg);
    }
    if (e == cudaSuccess) e = cudaStreamEndCapture(h->cap_stream, &graph);
    h->stream = saved;
    h->kv_timing = timing;
    w->cnodes = h->launches - launches;
    h->launches = launches;
    if (s != MFTO_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return s != MFTO_OK ? s
                          : mfto_fail(h, MFTO_CUDA_ERROR, "CG graph capture: %s",
                                      cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&w->cexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      w->cexec = nullptr;
      return mfto_fail(h, MFTO_CUDA_ERROR, "CG graph instantiate: %s", cudaGetErrorString(e));
    }
    w->cprm = w->prm;
    w->cchunk = chunk;
  }
  return MFTO_OK;
}

mfto_status check_params(mfto_handle* h, const mfto_gmg_params& p) {
  MFTO_REQUIRE(h, p.max_levels >= 1 && p.max_levels <= MFTO_GMG_MAX_LEVELS,
               "mfto_gmg_setup: max_levels in [1, MFTO_GMG_MAX_LEVELS]");
  MFTO_REQUIRE(h, p.coarse_max_dofs >= 3 && p.coarse_max_dofs <= MFTO_GMG_MAX_COARSE,
               "mfto_gmg_setup: coarse_max_dofs in [3, MFTO_GMG_MAX_COARSE]");
  MFTO_REQUIRE(h, p.nu_pre >= 0 && p.nu_post >= 0 && p.nu_pre <= 8 && p.nu_post <= 8,
               "mfto_gmg_setup: sweeps in [0, 8]");
  MFTO_REQUIRE(h, p.omega > 0.0 && p.omega < 2.0, "mfto_gmg_setup: omega in (0, 2)");
  MFTO_REQUIRE(h, p.mixed == 0 || p.mixed == 1, "mfto_gmg_setup: mixed is 0 or 1");
  MFTO_REQUIRE(h, p.inner_tol > 0.0 && p.inner_tol < 1.0, "mfto_gmg_setup: inner_tol in (0, 1)");
  MFTO_REQUIRE(h, p.smoother_form == MFTO_FORM_F32 || tc_form(p.smoother_form),
               "mfto_gmg_setup: smoother_form is MFTO_FORM_F32 or a tensor-core form");
  MFTO_REQUIRE(h, p.matfree_level1 >= -1 && p.matfree_level1 <= 1,
               "mfto_gmg_setup: matfree_level1 is -1, 0 or 1");
  MFTO_REQUIRE(h, p.continue_dir == 0 || p.continue_dir == 1,
               "mfto_gmg_setup: continue_dir is 0 or 1");
  MFTO_REQUIRE(h, p.cheb_degree >= -1 && p.cheb_degree <= 8,
               "mfto_gmg_setup: cheb_degree in [-1, 8]");
  return MFTO_OK;
}

GmgWs* ws(mfto_handle* h) {
  if (!h->gmg) {
    GmgWs* w = new GmgWs();
    mfto_default_gmg_params(&w->prm);
    if (cudaMalloc((void**)&w->d_s, sizeof(GmgScalars)) != cudaSuccess ||
        cudaMallocHost((void**)&w->h_s, sizeof(GmgScalars)) != cudaSuccess ||
        cudaMemset(w->d_s, 0, sizeof(GmgScalars)) != cudaSuccess ||
        cudaMalloc((void**)&w->d_cg, sizeof(GmgCg)) != cudaSuccess ||
        cudaMallocHost((void**)&w->h_cg, sizeof(GmgCg)) != cudaSuccess ||
        cudaMemset(w->d_cg, 0, sizeof(GmgCg)) != cudaSuccess) {
      cudaGetLastError();
      if (w->d_s) cudaFree(w->d_s);
      if (w->h_s) cudaFreeHost(w->h_s);
      if (w->d_cg) cudaFree(w->d_cg);
      if (w->h_cg) cudaFreeHost(w->h_cg);
      delete w;
      return nullptr;
    }
    h->gmg = w;
  }
  return h->gmg;
}

mfto_status read_scalars(mfto_handle* h, GmgWs* w) {
  MFTO_CUDA(h, cudaMemcpyAsync(w->h_s, w->d_s, sizeof(GmgScalars), cudaMemcpyDeviceToHost,
                               h->stream));
  MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  return MFTO_OK;
}

}  // namespace

void gmg_release(mfto_handle* h) {
  if (!h || !h->gmg) return;
  GmgWs* w = h->gmg;
  free_levels(w);
  if (w->d_E32) cudaFree(w->d_E32);
  if (w->d_G) cudaFree(w->d_G);
  if (w->d_s) cudaFree(w->d_s);
  if (w->h_s) cudaFreeHost(w->h_s);
  if (w->d_cg) cudaFree(w->d_cg);
  if (w->h_cg) cudaFreeHost(w->h_cg);
  delete w;
  h->gmg = nullptr;
}

bool gmg_active(const mfto_handle* h) { return h->gmg && h->gmg->use_in_simp; }

int64_t gmg_bytes(const mfto_handle* h) {
  const GmgWs* w = h->gmg;
  if (!w) return 0;
  int64_t b = sizeof(GmgScalars) + sizeof(GmgCg);
  if (w->d_E32) b += (int64_t)sizeof(float) * h->n_elem;
  if (w->d_G) b += (int64_t)sizeof(float) * 8 * 576;
  for (int l = 0; l < w->n_levels; ++l) {
    const GmgLevel& v = w->lv[l];
    b += 2 * (int64_t)sizeof(float) * v.n_dof;                  // dinv, t
    if (l == 0 && v.x) b += 2 * (int64_t)sizeof(float) * v.n_dof;   // fused-sweep scratch
    if (l > 0)
      b += v.n_node + (int64_t)sizeof(float) * (576 * v.n_elem + 3 * v.n_dof);  // mask, K, x, x2, b
  }
  if (w->d_cinv) b += (int64_t)sizeof(float) * w->n_c * w->n_c;
  if (w->mf_s0) b += 2 * (int64_t)sizeof(float) * h->n_dof;
  for (int l = 0; l < w->n_levels; ++l)
    if (w->lv[l].cr) b += 2 * (int64_t)sizeof(float) * w->lv[l].n_dof;
  return b;
}

extern "C" void mfto_default_gmg_params(mfto_gmg_params* p) {
  if (!p) return;
  p->max_levels = MFTO_GMG_MAX_LEVELS;
  p->coarse_max_dofs = 200;
  p->nu_pre = 1;
  p->nu_post = 1;
  p->omega = 1.3;
  p->mixed = 1;
  p->inner_tol = 1e-2;
  p->smoother_form = MFTO_FORM_F32;
  p->matfree_level1 = 0;
  p->continue_dir = 1;
  p->cheb_degree = -1;
}

extern "C" mfto_status mfto_gmg_setup(mfto_handle* h, const double* d_E,
                                      const mfto_gmg_params* prm) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, d_E, "mfto_gmg_setup: null pointer");
  GmgWs* w = ws(h);
  if (!w) return mfto_fail(h, MFTO_OOM, "mfto_gmg_setup: workspace allocation failed");
  mfto_gmg_params p = w->prm;
  if (prm) p = *prm;
  mfto_status s = check_params(h, p);
  if (s != MFTO_OK) return s;
  w->prm = p;
  g_sms = h->num_sms;
  if ((s = gmg_alloc(h, w, p)) != MFTO_OK) return s;
  // level 1 matrix-free when its matrices would not stay in L2 (auto), or as
  // asked; the matrices are still formed for the smoother and level 2
  {
    const bool want = w->n_levels >= 2 &&
                      (p.matfree_level1 == 1 ||
                       (p.matfree_level1 == 0 &&
                        (int64_t)sizeof(float) * 576 * w->lv[1].n_elem > (int64_t)96 << 20));
    if (want && !w->mf_s0) {
      if (cudaMalloc((void**)&w->mf_s0, sizeof(float) * h->n_dof) != cudaSuccess ||
          cudaMalloc((void**)&w->mf_s1, sizeof(float) * h->n_dof) != cudaSuccess) {
        cudaGetLastError();
        return mfto_fail(h, MFTO_OOM, "mfto_gmg_setup: cudaMalloc failed");
      }
    }
    w->mf1 = want;
  }
  // Chebyshev sweeps: as asked, or (cheb_degree = -1) degree 2 up to 4M DOFs,
  // where they were measured faster, l1-Jacobi above
  w->cheb = p.cheb_degree >= 0 ? p.cheb_degree : (h->n_dof <= 4000000 ? 2 : 0);
  if (w->cheb != 1 && p.smoother_form == MFTO_FORM_F32 && w->n_levels >= 2 &&
      !w->lv[0].x) {                        // level-0 scratch of the fused sweeps
    GmgLevel& v = w->lv[0];
    if (cudaMalloc((void**)&v.x, sizeof(float) * v.n_dof) != cudaSuccess ||
        cudaMalloc((void**)&v.x2, sizeof(float) * v.n_dof) != cudaSuccess) {
      cudaGetLastError();
      return mfto_fail(h, MFTO_OOM, "mfto_gmg_setup: cudaMalloc failed");
    }
  }
  if (w->cheb > 0) {                        // Chebyshev step and residual per level
    for (int l = 0; l + 1 < w->n_levels; ++l) {
      GmgLevel& v = w->lv[l];
      if (v.cr) continue;
      if (cudaMalloc((void**)&v.cr, sizeof(float) * v.n_dof) != cudaSuccess ||
          cudaMalloc((void**)&v.cd, sizeof(float) * v.n_dof) != cudaSuccess) {
        cudaGetLastError();
        return mfto_fail(h, MFTO_OOM, "mfto_gmg_setup: cudaMalloc failed");
      }
    }
  }
  if (!w->d_E32 || !w->d_G) {
    if ((!w->d_E32 && cudaMalloc((void**)&w->d_E32, sizeof(float) * h->n_elem) != cudaSuccess) ||
        (!w->d_G && cudaMalloc((void**)&w->d_G, sizeof(float) * 8 * 576) != cudaSuccess)) {
      cudaGetLastError();
      return mfto_fail(h, MFTO_OOM, "mfto_gmg_setup: cudaMalloc failed");
    }
  }
  w->ready = false;
  h->launches++;
  gmg_cast<<<grid_of(h->n_elem), kB, 0, h->stream>>>(d_E, w->d_E32, h->n_elem);
  MFTO_LAUNCH_CHECK(h);
  const GmgLevel& v0 = w->lv[0];
  h->launches++;
  gmg_l1_fine<<<grid_of(v0.n_node), kB, 0, h->stream>>>(w->d_E32, v0.d_fixed, h->d_ke32, v0.nx,
                                                        v0.ny, v0.nz, v0.d_dinv);
  MFTO_LAUNCH_CHECK(h);
  for (int l = 0; l + 1 < w->n_levels; ++l) {
    const GmgLevel& f = w->lv[l];
    const GmgLevel& c = w->lv[l + 1];
    const int g = (int)std::min<int64_t>(c.n_elem, 8LL * h->num_sms);
    h->launches++;
    if (l == 0) {
      h->launches++;
      gmg_child_galerkin<<<8, kB, 0, h->stream>>>(h->d_ke32, w->d_G);
      gmg_galerkin<true><<<g, kB, 0, h->stream>>>(nullptr, w->d_E32, h->d_ke32, w->d_G, f.d_fixed,
                                                  f.nx, f.ny, f.nz, c.d_fixed, c.nx, c.ny, c.nz,
                                                  c.d_K);
    } else {
      gmg_galerkin<false><<<g, kB, 0, h->stream>>>(f.d_K, nullptr, nullptr, nullptr, f.d_fixed,
                                                   f.nx, f.ny, f.nz, c.d_fixed, c.nx, c.ny, c.nz,
                                                   c.d_K);
    }
    MFTO_LAUNCH_CHECK(h);
    h->launches++;
    gmg_l1_coarse<<<grid_of(c.n_node), kB, 0, h->stream>>>(c.d_K, c.d_fixed, c.nx, c.ny, c.nz,
                                                           c.d_dinv);
    MFTO_LAUNCH_CHECK(h);
  }
  if ((s = coarse_inverse(h, w)) != MFTO_OK) return s;
  w->ready = true;
  return MFTO_OK;
}

extern "C" mfto_status mfto_gmg_params_in_use(mfto_handle* h, mfto_gmg_params* p) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, p, "mfto_gmg_params_in_use: null pointer");
  MFTO_REQUIRE(h, h->gmg && h->gmg->ready, "mfto_gmg_params_in_use: call mfto_gmg_setup first");
  *p = h->gmg->prm;
  p->cheb_degree = h->gmg->cheb;
  p->matfree_level1 = h->gmg->mf1 ? 1 : -1;
  return MFTO_OK;
}

extern "C" mfto_status mfto_gmg_levels(mfto_handle* h, int32_t* n_levels, int32_t* dims) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, n_levels && dims, "mfto_gmg_levels: null pointer");
  MFTO_REQUIRE(h, h->gmg && h->gmg->ready, "mfto_gmg_levels: call mfto_gmg_setup first");
  *n_levels = h->gmg->n_levels;
  for (int l = 0; l < h->gmg->n_levels; ++l) {
    dims[3 * l] = h->gmg->lv[l].nx;
    dims[3 * l + 1] = h->gmg->lv[l].ny;
    dims[3 * l + 2] = h->gmg->lv[l].nz;
  }
  return MFTO_OK;
}

extern "C" mfto_status mfto_gmg_apply(mfto_handle* h, int32_t level, const float* d_x,
                                      float* d_y) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, d_x && d_y, "mfto_gmg_apply: null pointer");
  MFTO_REQUIRE(h, h->gmg && h->gmg->ready, "mfto_gmg_apply: call mfto_gmg_setup first");
  MFTO_REQUIRE(h, level >= 0 && level < h->gmg->n_levels, "mfto_gmg_apply: no such level");
  return apply_level(h, h->gmg, level, d_x, d_y);
}

extern "C" mfto_status mfto_gmg_vcycle(mfto_handle* h, const float* d_r, float* d_z) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, d_r && d_z && d_r != d_z, "mfto_gmg_vcycle: null or aliased pointers");
  MFTO_REQUIRE(h, h->gmg && h->gmg->ready, "mfto_gmg_vcycle: call mfto_gmg_setup first");
  return vcycle_graph(h, h->gmg, d_r, d_z);
}

namespace {

// FP64 refinement around FP32 V-cycle CGs (mfto_gmg_params.mixed = 1)
mfto_status gmg_solve_mixed(mfto_handle* h, GmgWs* w, const double* E, const double* f, double* u,
                            mfto_solve_stats* st) {
  const int64_t n = h->n_dof;
  double *r = h->d_r, *q = h->d_q;
  float *r32 = h->d_r32, *z32 = h->d_z32, *p32 = h->d_p0_32, *e32 = h->d_e32, *ro32 = h->d_p1_32;
  const int g = reduction_blocks(n, kB);
  const double rtol = h->p.rtol, itol = w->prm.inner_tol;
  mfto_status s;
  double prev = 0.0;
  int stalls = 0;
  bool cont = false;                   // continue the last inner direction
  st->status = MFTO_NOT_CONVERGED;
  for (int outer = 0; outer <= 50; ++outer) {
    if ((s = kv_launch(h, MFTO_FORM_F64, E, u, q)) != MFTO_OK) return s;
    h->launches++;
    gmg_resid0<<<g, kB, 0, h->stream>>>(f, q, r, r32, n, w->d_s, h->d_partials);
    MFTO_LAUNCH_CHECK(h);
    if ((s = read_scalars(h, w)) != MFTO_OK) return s;
    const double rr = w->h_s->sum[0], ff = w->h_s->sum[1];
    st->fnorm = sqrt(ff);
    if (ff == 0.0) {
      MFTO_CUDA(h, cudaMemsetAsync(u, 0, sizeof(double) * n, h->stream));
      MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
      st->status = MFTO_OK;
      return MFTO_OK;
    }
    const double rel = sqrt(rr / ff);
    st->rel_residual = rel;
    if (rel <= rtol) { st->status = MFTO_OK; break; }
    if (!std::isfinite(rel)) { st->status = MFTO_BREAKDOWN; break; }
    if (outer > 0) {
      stalls = rel > 0.9 * prev ? stalls + 1 : 0;
      if (stalls >= 2) { st->status = MFTO_STALLED; break; }
    }
    if (outer == 50) break;
    prev = rel;
    // FP32 CG on K e = r from e = 0: start, then graph chunks of iterations
    // with the scalars on the device, polled once per chunk
    MFTO_CUDA(h, cudaMemsetAsync(e32, 0, sizeof(float) * n, h->stream));
    if ((s = vcycle_graph(h, w, r32, z32)) != MFTO_OK) return s;
    h->launches += 3;
    gmg_dot2_f32<<<g, kB, 0, h->stream>>>(r32, ro32, z32, n, 1, w->d_s, h->d_partials);
    MFTO_LAUNCH_CHECK(h);
    // continue the previous inner CG's direction (reliable updating), or
    // start from p = z
    if (cont) gmg_cont_dir_f32<<<g, kB, 0, h->stream>>>(z32, p32, n, w->d_s, w->d_cg);
    else gmg_first_dir_f32<<<g, kB, 0, h->stream>>>(z32, p32, n);
    MFTO_LAUNCH_CHECK(h);
    gmg_cg_start<<<1, 1, 0, h->stream>>>(w->d_cg, w->d_s, itol * itol * rr, h->p.maxit);
    MFTO_LAUNCH_CHECK(h);
    if ((s = cg_chunk_graph(h, w)) != MFTO_OK) return s;
    for (;;) {
      MFTO_CUDA(h, cudaGraphLaunch(w->cexec, h->stream));
      h->launches += w->cnodes;
      MFTO_CUDA(h, cudaMemcpyAsync(w->h_cg, w->d_cg, sizeof(GmgCg), cudaMemcpyDeviceToHost,
                                   h->stream));
      MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
      if (w->h_cg->done) break;
    }
    st->iterations += w->h_cg->it;
    cont = w->prm.continue_dir && w->h_cg->it > 0 && !w->h_cg->breakdown;
    h->launches++;
    gmg_correct<<<g, kB, 0, h->stream>>>(u, e32, n);
    MFTO_LAUNCH_CHECK(h);
  }
  MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  return MFTO_OK;
}

}  // namespace

namespace {

// FP64 CG preconditioned by the V-cycle (mfto_gmg_params.mixed = 0)
mfto_status gmg_solve_f64(mfto_handle* h, GmgWs* w, const double* E, const double* f, double* u,
                          mfto_solve_stats* st) {
  mfto_status s;
  const int64_t n = h->n_dof;
  double *r = h->d_r, *z = h->d_z, *pv = h->d_p0, *q = h->d_q, *r_old = h->d_p1;
  float *r32 = h->d_r32, *z32 = h->d_z32;
  const int g = reduction_blocks(n, kB);
  // r = f - K u
  if ((s = kv_launch(h, MFTO_FORM_F64, E, u, q)) != MFTO_OK) return s;
  h->launches++;
  gmg_resid0<<<g, kB, 0, h->stream>>>(f, q, r, r32, n, w->d_s, h->d_partials);
  MFTO_LAUNCH_CHECK(h);
  if ((s = read_scalars(h, w)) != MFTO_OK) return s;
  const double ff = w->h_s->sum[1];
  st->fnorm = sqrt(ff);
  if (ff == 0.0) {
    MFTO_CUDA(h, cudaMemsetAsync(u, 0, sizeof(double) * n, h->stream));
    MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
    st->status = MFTO_OK;
    return MFTO_OK;
  }
  double rr = w->h_s->sum[0];
  st->rel_residual = sqrt(rr / ff);
  const double rtol = h->p.rtol;
  if (st->rel_residual <= rtol) {
    st->status = MFTO_OK;
    return MFTO_OK;
  }
  if ((s = vcycle_graph(h, w, r32, z32)) != MFTO_OK) return s;
  h->launches += 2;
  gmg_zdot<<<g, kB, 0, h->stream>>>(z32, r, r_old, z, n, 1, w->d_s, h->d_partials);
  MFTO_LAUNCH_CHECK(h);
  gmg_dir<<<g, kB, 0, h->stream>>>(z, pv, 0.0, n, 1);
  MFTO_LAUNCH_CHECK(h);
  if ((s = read_scalars(h, w)) != MFTO_OK) return s;
  double rz = w->h_s->sum[0];
  st->status = MFTO_NOT_CONVERGED;
  for (int it = 1; it <= h->p.maxit; ++it) {
    if ((s = kv_launch(h, MFTO_FORM_F64, E, pv, q)) != MFTO_OK) return s;
    h->launches++;
    gmg_pq<<<g, kB, 0, h->stream>>>(pv, q, n, w->d_s, h->d_partials);
    MFTO_LAUNCH_CHECK(h);
    if ((s = read_scalars(h, w)) != MFTO_OK) return s;
    const double pq = w->h_s->sum[3];
    if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rz)) {
      st->status = MFTO_BREAKDOWN;
      st->iterations = it - 1;
      return MFTO_OK;
    }
    const double alpha = rz / pq;
    h->launches++;
    gmg_update<<<g, kB, 0, h->stream>>>(u, r, r_old, pv, q, r32, alpha, n, w->d_s,
                                        h->d_partials);
    MFTO_LAUNCH_CHECK(h);
    if ((s = vcycle_graph(h, w, r32, z32)) != MFTO_OK) return s;
    h->launches++;
    gmg_zdot<<<g, kB, 0, h->stream>>>(z32, r, r_old, z, n, 0, w->d_s, h->d_partials);
    MFTO_LAUNCH_CHECK(h);
    if ((s = read_scalars(h, w)) != MFTO_OK) return s;
    rr = w->h_s->sum[2];
    st->iterations = it;
    st->rel_residual = sqrt(rr / ff);
    if (st->rel_residual <= rtol) {
      st->status = MFTO_OK;
      break;
    }
    if (!std::isfinite(st->rel_residual)) {
      st->status = MFTO_BREAKDOWN;
      break;
    }
    const double rz_new = w->h_s->sum[0], zr_old = w->h_s->sum[1];
    const double beta = (rz_new - zr_old) / rz;
    rz = rz_new;
    h->launches++;
    gmg_dir<<<g, kB, 0, h->stream>>>(z, pv, beta, n, 0);
    MFTO_LAUNCH_CHECK(h);
  }
  MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  return MFTO_OK;
}

}  // namespace

// One solve on the hierarchy already built for E.
static mfto_status gmg_solve_built(mfto_handle* h, const double* E, const double* f, double* u,
                                   mfto_solve_stats* st) {
  memset(st, 0, sizeof(*st));
  mfto_status s;
  GmgWs* w = h->gmg;
  // a tensor-core smoother reports a completion wait that gave up in the
  // handle's error word
  const bool tc = tc_form(w->prm.smoother_form);
  if (tc) MFTO_CUDA(h, cudaMemsetAsync(&h->d_misc->error, 0, sizeof(int32_t), h->stream));
  s = w->prm.mixed ? gmg_solve_mixed(h, w, E, f, u, st) : gmg_solve_f64(h, w, E, f, u, st);
  if (s != MFTO_OK || !tc) return s;
  MFTO_CUDA(h, cudaMemcpyAsync(h->h_misc, h->d_misc, sizeof(MiscScalars), cudaMemcpyDeviceToHost,
                               h->stream));
  MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->h_misc->error)
    return mfto_fail(h, MFTO_CUDA_ERROR, "mfto_gmg_solve: tensor-core completion wait timed out");
  return MFTO_OK;
}

mfto_status gmg_solve(mfto_handle* h, const double* E, const double* f, double* u,
                      mfto_solve_stats* st) {
  mfto_status s = mfto_gmg_setup(h, E, nullptr);
  if (s != MFTO_OK) {
    memset(st, 0, sizeof(*st));
    return s;
  }
  return gmg_solve_built(h, E, f, u, st);
}

extern "C" mfto_status mfto_gmg_solve_multi(mfto_handle* h, const double* d_E, const double* d_F,
                                            double* d_U, int32_t nrhs, mfto_solve_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, d_E && d_F && d_U && st, "mfto_gmg_solve_multi: null pointer");
  MFTO_REQUIRE(h, nrhs >= 1, "mfto_gmg_solve_multi: nrhs >= 1");
  mfto_status s = mfto_gmg_setup(h, d_E, nullptr);           // one hierarchy for every case
  if (s != MFTO_OK) return s;
  for (int32_t r = 0; r < nrhs && s == MFTO_OK; ++r)
    s = gmg_solve_built(h, d_E, d_F + (size_t)r * h->n_dof, d_U + (size_t)r * h->n_dof, &st[r]);
  return s;
}

extern "C" mfto_status mfto_gmg_solve(mfto_handle* h, const double* d_E, const double* d_f,
                                      double* d_u, mfto_solve_stats* st) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, d_E && d_f && d_u && st, "mfto_gmg_solve: null pointer");
  return gmg_solve(h, d_E, d_f, d_u, st);
}

extern "C" mfto_status mfto_set_gmg_solver(mfto_handle* h, int32_t on,
                                           const mfto_gmg_params* prm) {
  if (!h) return MFTO_INVALID_ARG;
  GmgWs* w = ws(h);
  if (!w) return mfto_fail(h, MFTO_OOM, "mfto_set_gmg_solver: workspace allocation failed");
  if (prm) {
    mfto_status s = check_params(h, *prm);
    if (s != MFTO_OK) return s;
    w->prm = *prm;
  }
  w->use_in_simp = on != 0;
  return MFTO_OK;
}

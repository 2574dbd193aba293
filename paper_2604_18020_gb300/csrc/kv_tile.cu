// Launchers of the tiled mode-space K.v (kv_tile.cuh): plain y = K v and the
// CG form that also forms p_new = z + beta p_old, q = K p_new and alpha.
#include "common.cuh"
#include "kv_column.cuh"
#include "kv_tile.cuh"

namespace {

constexpr int kTX = 16, kTY = 12;   // owned nodes per CTA in x, y; 256 threads
using Shape = TileShape<kTX, kTY>;

// FP64 runs the z-streaming ring variant (bound by the FP64 pipe, little halo
// recompute); FP32 runs the one-element-per-thread block variant (bound by
// memory latency otherwise, so it trades halo arithmetic for parallelism).
template <typename T>
struct UseBlock { static constexpr bool value = sizeof(T) == 4; };
static_assert(Shape::NE <= MFTO_BLOCK && Shape::NV <= MFTO_BLOCK, "tile larger than the block");

template <typename T, typename Load, typename Epi>
__device__ __forceinline__ double tile_body(const T* E, const uint8_t* fixed, const ModeCoef<T>& K,
                                            const Grid& g, int nzc, const Load& ld, const Epi& epi,
                                            T* smem) {
  if constexpr (UseBlock<T>::value)
    return kv_block_body<T>(E, fixed, K, g, ld, epi, smem);
  else
    return kv_tile_body<T, kTX, kTY>(E, fixed, K, g, nzc, ld, epi, smem);
}

template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
kv_tile_kernel(const T* __restrict__ E, const T* __restrict__ v, T* __restrict__ y,
               const uint8_t* __restrict__ fixed, ModeCoef<T> K, Grid g, int nzc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_body<T>(E, fixed, K, g, nzc, TileLoadPlain<T>{v}, TileStore<T>{v, y},
               reinterpret_cast<T*>(smem_raw));
}

template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_kv_tile_kernel(const T* __restrict__ E, const T* __restrict__ z, const T* __restrict__ p_old,
                   T* __restrict__ p_new, T* __restrict__ q, const uint8_t* __restrict__ fixed,
                   ModeCoef<T> K, Grid g, int nzc, PcgScalars* s, double* partials) {
  if (*(volatile int32_t*)&s->done) return;  // uniform over the grid
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[64];
  const T beta = (T)s->beta;
  double red[1];
  red[0] = tile_body<T>(E, fixed, K, g, nzc, TileLoadDirection<T>{z, p_old, beta},
                        TilePcg<T>{p_new, q}, reinterpret_cast<T*>(smem_raw));
  double tot[1];
  if (last_block_reduce<1, DotAcc<T>::kWarpReduced>(red, partials, &s->ticket_b, tot, sh) &&
      threadIdx.x == 0) {
    s->pq = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      s->done = 1;
      s->status = MFTO_BREAKDOWN;
      s->alpha = 0.0;
    } else {
      s->alpha = s->rz / tot[0];
    }
  }
}

// FP32, variant 0: column-streaming body (kv_column.cuh).  MINB: resident
// CTAs per SM the register allocation is held to (2: up to 128 registers per
// thread, 3: up to 80); mfto_kv_autotune picks one.
template <int MINB>
__global__ void __launch_bounds__(MFTO_BLOCK, MINB)
kv_col_kernel(const float* __restrict__ E, const float* __restrict__ v, float* __restrict__ y,
              const uint8_t* __restrict__ fixed, ModeCoef<float> K, Grid g, ColTiling tl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  kv_column_body(E, fixed, K, g, tl, ColLoadPlain{v}, ColStore{v, y},
                 reinterpret_cast<float*>(smem_raw));
}

// Multigrid l1-Jacobi sweeps on the level-0 operator (gmg.cu), fused into the
// column K.v: the first sweep from zero loads omega D1^-1 b as its vector and
// writes x and A x; a later sweep loads x and writes x + omega D1^-1 (b - A x)
// to another buffer.  The masked loads give 0 on fixed DOFs, where A is the
// identity and b is 0, so both stay 0 there.
struct ColLoadScaled {
  using Raw = float;
  static constexpr bool kAsync = true;
  static constexpr int kSrc = 2;
  const float* b;
  const float* dinv;
  float omega;
  __device__ __forceinline__ const float* src(int i) const { return i == 0 ? b : dinv; }
  __device__ __forceinline__ float combine(const float (&r)[kSrc]) const { return omega * r[1] * r[0]; }
  __device__ __forceinline__ float operator()(int idx) const { return omega * dinv[idx] * b[idx]; }
};

struct ColSweepFirst {
  float* x;
  float* t;
  __device__ __forceinline__ void operator()(int node, const float (&acc)[3], const float (&pn)[3],
                                             uint8_t fm, DFloat& red) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[3 * node + c] = pn[c];
      t[3 * node + c] = ((fm >> c) & 1) ? pn[c] : acc[c];
    }
  }
};

struct ColSweep {
  const float* b;
  const float* dinv;
  float omega;
  float* xo;
  __device__ __forceinline__ void operator()(int node, const float (&acc)[3], const float (&pn)[3],
                                             uint8_t fm, DFloat& red) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int d = 3 * node + c;
      const float y = ((fm >> c) & 1) ? pn[c] : acc[c];
      xo[d] = pn[c] + omega * dinv[d] * (b[d] - y);
    }
  }
};

template <int MINB, int FIRST>
__global__ void __launch_bounds__(MFTO_BLOCK, MINB)
gmg_sweep_col_kernel(const float* __restrict__ E, const float* __restrict__ b,
                     const float* __restrict__ dinv, float omega, const float* __restrict__ x,
                     float* __restrict__ xo, float* __restrict__ t,
                     const uint8_t* __restrict__ fixed, ModeCoef<float> K, Grid g, ColTiling tl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (FIRST)
    kv_column_body(E, fixed, K, g, tl, ColLoadScaled{b, dinv, omega}, ColSweepFirst{xo, t},
                   reinterpret_cast<float*>(smem_raw));
  else
    kv_column_body(E, fixed, K, g, tl, ColLoadPlain{x}, ColSweep{b, dinv, omega, xo},
                   reinterpret_cast<float*>(smem_raw));
}

// Multigrid Chebyshev sweeps on the level-0 operator, fused into the column
// K.v the same way (the recurrences of the gmg_cheb_* kernels in gmg.cu; d
// the step, r the preconditioned residual, t = A of the loaded vector):
//   ColChebFirst (loads d0 = D1^-1 b / theta): r = D1^-1 b - D1^-1 t,
//     dn = c1 d0 + c2 r, x = d0 + dn;
//   ColChebBegin (loads x): r = D1^-1 (b - t), dn = r / theta, xo = x + dn;
//   ColChebStep (loads d): r -= D1^-1 t, dn = c1 d + c2 r, xo = x + dn (xo
//     may be x, which no other thread reads).
// The written step dn and a Begin's xo are buffers the launch does not load.
struct ColChebFirst {
  const float* b;
  const float* dinv;
  float c1, c2;
  float* r;
  float* dn;
  float* x;
  __device__ __forceinline__ void operator()(int node, const float (&acc)[3], const float (&pn)[3],
                                             uint8_t fm, DFloat& red) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int q = 3 * node + c;
      const float t = ((fm >> c) & 1) ? pn[c] : acc[c];
      const float ri = dinv[q] * b[q] - dinv[q] * t;
      const float di = c1 * pn[c] + c2 * ri;
      r[q] = ri;
      dn[q] = di;
      x[q] = pn[c] + di;
    }
  }
};

struct ColChebBegin {
  const float* b;
  const float* dinv;
  float inv_theta;
  float* r;
  float* dn;
  float* xo;
  __device__ __forceinline__ void operator()(int node, const float (&acc)[3], const float (&pn)[3],
                                             uint8_t fm, DFloat& red) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int q = 3 * node + c;
      const float t = ((fm >> c) & 1) ? pn[c] : acc[c];
      const float ri = dinv[q] * (b[q] - t);
      const float di = inv_theta * ri;
      r[q] = ri;
      dn[q] = di;
      xo[q] = pn[c] + di;
    }
  }
};

struct ColChebStep {
  const float* dinv;
  float c1, c2;
  float* r;
  float* dn;
  const float* x;
  float* xo;
  __device__ __forceinline__ void operator()(int node, const float (&acc)[3], const float (&pn)[3],
                                             uint8_t fm, DFloat& red) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int q = 3 * node + c;
      const float t = ((fm >> c) & 1) ? pn[c] : acc[c];
      const float ri = r[q] - dinv[q] * t;
      const float di = c1 * pn[c] + c2 * ri;
      r[q] = ri;
      dn[q] = di;
      xo[q] = x[q] + di;
    }
  }
};

template <int MINB, int MODE>
__global__ void __launch_bounds__(MFTO_BLOCK, MINB)
gmg_cheb_col_kernel(const float* __restrict__ E, const float* in, const float* b,
                    const float* dinv, float inv_theta, float c1, float c2, float* r, float* dn,
                    const float* x, float* xo, const uint8_t* __restrict__ fixed,
                    ModeCoef<float> K, Grid g, ColTiling tl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  if (MODE == GMG_CHEB_FIRST)
    kv_column_body(E, fixed, K, g, tl, ColLoadScaled{b, dinv, inv_theta},
                   ColChebFirst{b, dinv, c1, c2, r, dn, xo}, sm);
  else if (MODE == GMG_CHEB_BEGIN)
    kv_column_body(E, fixed, K, g, tl, ColLoadPlain{in},
                   ColChebBegin{b, dinv, inv_theta, r, dn, xo}, sm);
  else
    kv_column_body(E, fixed, K, g, tl, ColLoadPlain{in}, ColChebStep{dinv, c1, c2, r, dn, x, xo},
                   sm);
}

template <int MINB>
__global__ void __launch_bounds__(MFTO_BLOCK, MINB)
pcg_kv_col_kernel(const float* __restrict__ E, const float* __restrict__ z,
                  const float* __restrict__ p_old, float* __restrict__ p_new,
                  float* __restrict__ q, const uint8_t* __restrict__ fixed, ModeCoef<float> K,
                  Grid g, ColTiling tl, PcgScalars* s, double* partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[64];
  DotAcc<float> acc;
  bool skipped = false;   // the solve is done: uniform over the grid
  acc.s = kv_column_body(E, fixed, K, g, tl, ColLoadDirection{z, p_old, 0.f}, ColPcg{p_new, q},
                         reinterpret_cast<float*>(smem_raw), ColPreFlagBeta{&s->done, &s->beta},
                         &skipped);
  if (skipped) return;
  const DFloat w[1] = {acc.finish_df()};
  double tot[1];
  if (last_block_reduce_df<1>(w, partials, &s->ticket_b, tot, sh) && threadIdx.x == 0) {
    s->pq = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      s->done = 1;
      s->status = MFTO_BREAKDOWN;
      s->alpha = 0.0;
    } else {
      s->alpha = s->rz / tot[0];
    }
  }
}

// Column kernel kinds, chosen by mfto_kv_autotune: the register allocation
// held to 2 (kind 0, up to 128 registers) or 3 (kind 1, up to 80) resident
// CTAs per SM.
constexpr int kColKinds = 2;

template <typename T>
dim3 tile_grid(const mfto_handle* h, int* nzc_out, int per_sm = 1) {
  const Grid g = make_grid(h->mesh);
  if (UseBlock<T>::value) {
    // grid-stride over 7 x 7 x 3 node blocks; one wave of resident CTAs
    const int64_t nb = (int64_t)((g.nx + 6) / 7) * ((g.ny + 6) / 7) * ((g.nz + 2) / 3);
    int64_t grid = (int64_t)per_sm * h->num_sms;
    if (grid > nb) grid = nb;
    *nzc_out = 0;
    return dim3((unsigned)grid, 1, 1);
  }
  const int tx = (g.nx + kTX - 1) / kTX, ty = (g.ny + kTY - 1) / kTY;
  const int target = (sizeof(T) == 8 ? 2 : 4) * h->num_sms;
  int zch = (target + tx * ty / 2) / (tx * ty);
  if (zch < 1) zch = 1;
  if (zch > g.nz) zch = g.nz;
  int nzc = (g.nz + zch - 1) / zch;
  if (nzc < 4) nzc = g.nz < 4 ? g.nz : 4;
  int tz = (g.nz + nzc - 1) / nzc;
  // the CG form reduces one partial per block
  if ((int64_t)tx * ty * tz > MFTO_RED_SLOTS) return dim3(0, 0, 0);
  *nzc_out = nzc;
  return dim3(tx, ty, tz);
}

template <typename T>
size_t tile_smem() {
  return UseBlock<T>::value ? BlockShape::smem_bytes<T>() : Shape::smem_bytes<T>();
}

template <typename T>
mfto_status set_attrs(mfto_handle* h) {
  const int smem = (int)tile_smem<T>();
  MFTO_CUDA(h, cudaFuncSetAttribute(kv_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_kv_tile_kernel<T>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return MFTO_OK;
}

}  // namespace

// column tiling for a standalone launch: chunks of h->col_nzc node layers if
// set (mfto_kv_autotune), else sized for the resident CTAs
ColTiling col_launch_tiling(const mfto_handle* h, int per_sm, int* grid) {
  const Grid g = make_grid(h->mesh);
  const int64_t ctas = (int64_t)per_sm * h->num_sms;
  ColTiling tl = col_tiling(g, h->col_nzc > 0 ? h->col_nzc : col_chunk(g, ctas, 4));
  tl.fixed_tiles = h->d_tile_fixed;
  int64_t n = tl.count();
  if (n > ctas) n = ctas;
  if (n > MFTO_RED_SLOTS) n = MFTO_RED_SLOTS;
  *grid = (int)n;
  return tl;
}

mfto_status kv_tile_init(mfto_handle* h) {
  mfto_status s = set_attrs<double>(h);
  if (s == MFTO_OK) s = set_attrs<float>(h);
  if (s != MFTO_OK) return s;
  const int csm = (int)kColSmem;
  MFTO_CUDA(h, cudaFuncSetAttribute(kv_col_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(kv_col_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_sweep_col_kernel<2, 0>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_sweep_col_kernel<2, 1>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_sweep_col_kernel<3, 0>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_sweep_col_kernel<3, 1>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_cheb_col_kernel<2, GMG_CHEB_FIRST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_cheb_col_kernel<2, GMG_CHEB_BEGIN>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_cheb_col_kernel<2, GMG_CHEB_STEP>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_cheb_col_kernel<3, GMG_CHEB_FIRST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_cheb_col_kernel<3, GMG_CHEB_BEGIN>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(gmg_cheb_col_kernel<3, GMG_CHEB_STEP>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_kv_col_kernel<2>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_kv_col_kernel<3>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, csm));
  // resident CTAs per SM of each kind (the CG form, which is the heavier one)
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ_col[0], pcg_kv_col_kernel<2>,
                                                             MFTO_BLOCK, csm));
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ_col[1], pcg_kv_col_kernel<3>,
                                                             MFTO_BLOCK, csm));
  for (int k = 0; k < kColKinds; ++k)
    if (h->occ_col[k] < 1) h->occ_col[k] = 1;
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                   &h->occ_kv32, kv_tile_kernel<float>, MFTO_BLOCK, tile_smem<float>()));
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                   &h->occ_pcg32, pcg_kv_tile_kernel<float>, MFTO_BLOCK, tile_smem<float>()));
  if (h->occ_kv32 < 1) h->occ_kv32 = 1;
  if (h->occ_pcg32 < 1) h->occ_pcg32 = 1;
  return MFTO_OK;
}

template <typename T>
static const ModeCoef<T>& coef(const mfto_handle* h);
template <>
const ModeCoef<double>& coef<double>(const mfto_handle* h) { return h->mc64; }
template <>
const ModeCoef<float>& coef<float>(const mfto_handle* h) { return h->mc32; }

// One l1-Jacobi sweep on the FP32 operator fused with it (first: from x = 0,
// writing x and A x; otherwise x -> xo).  Needs the column kernel (variant 0).
mfto_status gmg_sweep_col_launch(mfto_handle* h, bool first, const float* E, const float* b,
                                 const float* dinv, float omega, const float* x, float* xo,
                                 float* t) {
  if (h->kv_variant != 0)
    return mfto_fail(h, MFTO_UNSUPPORTED, "fused sweeps need the column K.v");
  int grid = 0;
  const int kind = h->col_kind;
  const ColTiling tl = col_launch_tiling(h, h->occ_col[kind], &grid);
  const Grid g = make_grid(h->mesh);
  const size_t sm = kColSmem;
  h->launches++;
  if (kind == 1) {
    if (first)
      gmg_sweep_col_kernel<3, 1><<<grid, MFTO_BLOCK, sm, h->stream>>>(
          E, b, dinv, omega, x, xo, t, h->d_fixed, h->mc32, g, tl);
    else
      gmg_sweep_col_kernel<3, 0><<<grid, MFTO_BLOCK, sm, h->stream>>>(
          E, b, dinv, omega, x, xo, t, h->d_fixed, h->mc32, g, tl);
  } else {
    if (first)
      gmg_sweep_col_kernel<2, 1><<<grid, MFTO_BLOCK, sm, h->stream>>>(
          E, b, dinv, omega, x, xo, t, h->d_fixed, h->mc32, g, tl);
    else
      gmg_sweep_col_kernel<2, 0><<<grid, MFTO_BLOCK, sm, h->stream>>>(
          E, b, dinv, omega, x, xo, t, h->d_fixed, h->mc32, g, tl);
  }
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

// One Chebyshev launch on the FP32 operator fused with it (mode and buffers as
// gmg_cheb_col_kernel: in the loaded vector of BEGIN and STEP, x the iterate
// STEP adds to, xo where the new iterate goes).  Needs the column kernel.
mfto_status gmg_cheb_col_launch(mfto_handle* h, int mode, const float* E, const float* in,
                                const float* b, const float* dinv, float inv_theta, float c1,
                                float c2, float* r, float* dn, const float* x, float* xo) {
  if (h->kv_variant != 0)
    return mfto_fail(h, MFTO_UNSUPPORTED, "fused sweeps need the column K.v");
  int grid = 0;
  const int kind = h->col_kind;
  const ColTiling tl = col_launch_tiling(h, h->occ_col[kind], &grid);
  const Grid g = make_grid(h->mesh);
  const size_t sm = kColSmem;
  h->launches++;
#define MFTO_CHEB_COL(MINB, MODE)                                                               \
  gmg_cheb_col_kernel<MINB, MODE><<<grid, MFTO_BLOCK, sm, h->stream>>>(                         \
      E, in, b, dinv, inv_theta, c1, c2, r, dn, x, xo, h->d_fixed, h->mc32, g, tl)
  if (kind == 1) {
    if (mode == GMG_CHEB_FIRST) MFTO_CHEB_COL(3, GMG_CHEB_FIRST);
    else if (mode == GMG_CHEB_BEGIN) MFTO_CHEB_COL(3, GMG_CHEB_BEGIN);
    else MFTO_CHEB_COL(3, GMG_CHEB_STEP);
  } else {
    if (mode == GMG_CHEB_FIRST) MFTO_CHEB_COL(2, GMG_CHEB_FIRST);
    else if (mode == GMG_CHEB_BEGIN) MFTO_CHEB_COL(2, GMG_CHEB_BEGIN);
    else MFTO_CHEB_COL(2, GMG_CHEB_STEP);
  }
#undef MFTO_CHEB_COL
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

template <typename T>
mfto_status kv_tile_launch(mfto_handle* h, const T* E, const T* v, T* y, cudaStream_t st) {
  if (sizeof(T) == 4 && h->kv_variant == 0) {
    int grid = 0;
    const int kind = h->col_kind;
    const ColTiling tl = col_launch_tiling(h, h->occ_col[kind], &grid);
    const Grid g = make_grid(h->mesh);
    const float *Ef = (const float*)E, *vf = (const float*)v;
    float* yf = (float*)y;
    const size_t sm = kColSmem;
    if (kind == 1)
      kv_col_kernel<3><<<grid, MFTO_BLOCK, sm, st>>>(Ef, vf, yf, h->d_fixed, h->mc32, g, tl);
    else
      kv_col_kernel<2><<<grid, MFTO_BLOCK, sm, st>>>(Ef, vf, yf, h->d_fixed, h->mc32, g, tl);
    MFTO_LAUNCH_CHECK(h);
    return MFTO_OK;
  }
  int nzc = 0;
  const dim3 grid = tile_grid<T>(h, &nzc, h->occ_kv32);
  if (grid.x == 0) return mfto_fail(h, MFTO_TOO_LARGE, "mesh too large for the K.v tiling");
  kv_tile_kernel<T><<<grid, MFTO_BLOCK, tile_smem<T>(), st>>>(
      E, v, y, h->d_fixed, coef<T>(h), make_grid(h->mesh), nzc);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

template <typename T>
mfto_status pcg_kv_tile_launch(mfto_handle* h, const T* E, const T* z, const T* p_old, T* p_new,
                               T* q, PcgScalars* s, double* partials, cudaStream_t st) {
  if (sizeof(T) == 4 && h->kv_variant == 0) {
    int grid = 0;
    const int kind = h->col_kind;
    const ColTiling tl = col_launch_tiling(h, h->occ_col[kind], &grid);
    const Grid g = make_grid(h->mesh);
    const float *Ef = (const float*)E, *zf = (const float*)z, *pf = (const float*)p_old;
    float *pn = (float*)p_new, *qf = (float*)q;
    const size_t sm = kColSmem;
    if (kind == 1)
      pcg_kv_col_kernel<3><<<grid, MFTO_BLOCK, sm, st>>>(Ef, zf, pf, pn, qf, h->d_fixed, h->mc32,
                                                         g, tl, s, partials);
    else
      pcg_kv_col_kernel<2><<<grid, MFTO_BLOCK, sm, st>>>(Ef, zf, pf, pn, qf, h->d_fixed, h->mc32,
                                                         g, tl, s, partials);
    MFTO_LAUNCH_CHECK(h);
    return MFTO_OK;
  }
  int nzc = 0;
  const dim3 grid = tile_grid<T>(h, &nzc, h->occ_pcg32);
  if (grid.x == 0) return mfto_fail(h, MFTO_TOO_LARGE, "mesh too large for the K.v tiling");
  pcg_kv_tile_kernel<T><<<grid, MFTO_BLOCK, tile_smem<T>(), st>>>(
      E, z, p_old, p_new, q, h->d_fixed, coef<T>(h), make_grid(h->mesh), nzc, s, partials);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

template mfto_status kv_tile_launch<double>(mfto_handle*, const double*, const double*, double*,
                                            cudaStream_t);
template mfto_status kv_tile_launch<float>(mfto_handle*, const float*, const float*, float*,
                                           cudaStream_t);
template mfto_status pcg_kv_tile_launch<double>(mfto_handle*, const double*, const double*,
                                                const double*, double*, double*, PcgScalars*,
                                                double*, cudaStream_t);
template mfto_status pcg_kv_tile_launch<float>(mfto_handle*, const float*, const float*,
                                               const float*, float*, float*, PcgScalars*,
                                               double*, cudaStream_t);

// Times the FP32 column K.v (as one inner CG iteration with the graph CG
// engines, as a plain K.v otherwise) for every balanced chunk length along z
// and every kernel kind on the handle's FP32 work vectors and keeps the
// fastest pair (mfto_kv, the CG K.v of the FP32 inner solves).
extern "C" mfto_status mfto_kv_autotune(mfto_handle* h, int32_t* nzc_out, int32_t* kind_out,
                                        float* us_out) {
  if (!h) return MFTO_INVALID_ARG;
  const Grid g = make_grid(h->mesh);
  // chunk lengths: every distinct ceil(nz / tz) for up to 64 chunks along z
  // (each the shortest chunk for its chunk count, so the z tiles are as even
  // as the count allows), from the longest chunk down
  std::vector<int> cand;
  for (int tz = 1; tz <= 64 && tz <= g.nz; ++tz) {
    const int c = (g.nz + tz - 1) / tz;
    if (cand.empty() || cand.back() != c) cand.push_back(c);
  }
  MFTO_CUDA(h, cudaMemsetAsync(h->d_r32, 0, sizeof(float) * h->n_dof, h->stream));
  MFTO_CUDA(h, cudaMemsetAsync(h->d_E32, 0, sizeof(float) * h->n_elem, h->stream));
  cudaEvent_t a, b;
  MFTO_CUDA(h, cudaEventCreate(&a));
  MFTO_CUDA(h, cudaEventCreate(&b));
  const int saved_nzc = h->col_nzc, saved_kind = h->col_kind;
  int best = 0, best_kind = 0;
  float best_ms = 0.f;
  // the graph CG engines time one inner CG iteration (the K.v launch with
  // its vector update) per shape, the others the plain K.v
  const bool cg = h->cg_engine != 1;
  for (int kind = 0; kind < kColKinds; ++kind) {
    for (int nzc : cand) {
      h->col_nzc = nzc;
      h->col_kind = kind;
      if (cg) {
        pcg_graph_release(h);
        float us = 0.f;
        mfto_status st = pcg_time_iterations(h, 2, &us);
        if (st != MFTO_OK) {
          h->col_nzc = saved_nzc;
          h->col_kind = saved_kind;
          pcg_graph_release(h);
          cudaEventDestroy(a);
          cudaEventDestroy(b);
          return st;
        }
        if (best == 0 || us < best_ms * 1000.f) { best = nzc; best_kind = kind; best_ms = us / 1000.f; }
        continue;
      }
      const int reps = 20;
      for (int rep = 0; rep < reps + 2; ++rep) {   // 2 warm-up launches
        if (rep == 2) cudaEventRecord(a, h->stream);
        mfto_status st = kv_tile_launch<float>(h, h->d_E32, h->d_r32, h->d_q32, h->stream);
        if (st != MFTO_OK) {
          h->col_nzc = saved_nzc;
          h->col_kind = saved_kind;
          cudaEventDestroy(a);
          cudaEventDestroy(b);
          return st;
        }
      }
      cudaEventRecord(b, h->stream);
      cudaError_t e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e != cudaSuccess) {
        h->col_nzc = saved_nzc;
        h->col_kind = saved_kind;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return mfto_fail(h, MFTO_CUDA_ERROR, "mfto_kv_autotune: %s", cudaGetErrorString(e));
      }
      h->launches += reps + 2;
      ms /= reps;
      if (best == 0 || ms < best_ms) { best = nzc; best_kind = kind; best_ms = ms; }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->col_nzc = best;
  h->col_kind = best_kind;
  pcg_graph_release(h);   // captured CG graphs hold the old launch shape
  if (nzc_out) *nzc_out = best;
  if (kind_out) *kind_out = best_kind;
  if (us_out) *us_out = best_ms * 1000.f;
  return MFTO_OK;
}

extern "C" mfto_status mfto_set_kv_shape(mfto_handle* h, int32_t nzc, int32_t kind) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, nzc >= 0, "mfto_set_kv_shape: nzc must be >= 0");
  MFTO_REQUIRE(h, kind >= 0 && kind < kColKinds, "mfto_set_kv_shape: kind must be 0 or 1");
  h->col_nzc = nzc;
  h->col_kind = kind;
  pcg_graph_release(h);
  return MFTO_OK;
}

// Launchers of the tiled mode-space K.v (kv_tile.cuh): plain y = K v and the
// CG form that also forms p_new = z + beta p_old, q = K p_new and alpha.
#include "common.cuh"
#include "kv_tile.cuh"

namespace {

constexpr int kTX = 16, kTY = 12;   // owned nodes per CTA in x, y; 256 threads
using Shape = TileShape<kTX, kTY>;
static_assert(Shape::NE <= MFTO_BLOCK && Shape::NV <= MFTO_BLOCK, "tile larger than the block");

template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
kv_tile_kernel(const T* __restrict__ E, const T* __restrict__ v, T* __restrict__ y,
               const uint8_t* __restrict__ fixed, ModeCoef<T> K, Grid g, int nzc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  kv_tile_body<T, kTX, kTY>(E, fixed, K, g, nzc, TileLoadPlain<T>{v}, TileStore<T>{v, y},
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
  red[0] = kv_tile_body<T, kTX, kTY>(E, fixed, K, g, nzc, TileLoadDirection<T>{z, p_old, beta},
                                     TilePcg<T>{p_new, q}, reinterpret_cast<T*>(smem_raw));
  double tot[1];
  if (last_block_reduce<1>(red, partials, &s->ticket_b, tot, sh) && threadIdx.x == 0) {
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

template <typename T>
dim3 tile_grid(const mfto_handle* h, int* nzc_out) {
  const Grid g = make_grid(h->mesh);
  const int tx = (g.nx + kTX - 1) / kTX, ty = (g.ny + kTY - 1) / kTY;
  const int target = (sizeof(T) == 8 ? 2 : 4) * h->num_sms;
  int zch = (target + tx * ty / 2) / (tx * ty);
  if (zch < 1) zch = 1;
  if (zch > g.nz) zch = g.nz;
  int nzc = (g.nz + zch - 1) / zch;
  if (nzc < 4) nzc = g.nz < 4 ? g.nz : 4;
  int tz = (g.nz + nzc - 1) / nzc;
  // the CG form reduces one partial per block
  while ((int64_t)tx * ty * tz > MFTO_RED_SLOTS) {
    nzc *= 2;
    tz = (g.nz + nzc - 1) / nzc;
  }
  *nzc_out = nzc;
  return dim3(tx, ty, tz);
}

template <typename T>
mfto_status set_attrs(mfto_handle* h) {
  const int smem = (int)Shape::smem_bytes<T>();
  MFTO_CUDA(h, cudaFuncSetAttribute(kv_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_kv_tile_kernel<T>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return MFTO_OK;
}

}  // namespace

mfto_status kv_tile_init(mfto_handle* h) {
  mfto_status s = set_attrs<double>(h);
  if (s != MFTO_OK) return s;
  return set_attrs<float>(h);
}

template <typename T>
static const ModeCoef<T>& coef(const mfto_handle* h);
template <>
const ModeCoef<double>& coef<double>(const mfto_handle* h) { return h->mc64; }
template <>
const ModeCoef<float>& coef<float>(const mfto_handle* h) { return h->mc32; }

template <typename T>
mfto_status kv_tile_launch(mfto_handle* h, const T* E, const T* v, T* y, cudaStream_t st) {
  int nzc = 0;
  const dim3 grid = tile_grid<T>(h, &nzc);
  kv_tile_kernel<T><<<grid, MFTO_BLOCK, Shape::smem_bytes<T>(), st>>>(
      E, v, y, h->d_fixed, coef<T>(h), make_grid(h->mesh), nzc);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

template <typename T>
mfto_status pcg_kv_tile_launch(mfto_handle* h, const T* E, const T* z, const T* p_old, T* p_new,
                               T* q, PcgScalars* s, double* partials, cudaStream_t st) {
  int nzc = 0;
  const dim3 grid = tile_grid<T>(h, &nzc);
  pcg_kv_tile_kernel<T><<<grid, MFTO_BLOCK, Shape::smem_bytes<T>(), st>>>(
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

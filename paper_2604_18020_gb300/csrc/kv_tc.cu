// K.v with the element contraction on the tcgen05 tensor cores: the TF32,
// split-TF32, BF16, split-BF16, FP16 and split-FP16 forms (FP32 vectors, FP32
// accumulation in tensor memory).
//
// TF32 and split TF32 run the pipelined column kernel of kv_tcol.cuh: the
// staged node layers are the MMA's A operand in place, two TMEM accumulators
// let the MMAs of one element layer overlap the staging of the next and the
// node sums of the previous one.
//
// BF16 and FP16 (2-byte operands: four components of a node fill only half a
// 16-byte core-matrix row, so a node layer cannot serve as the operand) use
// the block kernel below, with the blocking of the FP32 block variant
// (kv_tile.cuh): a 256-thread CTA owns the 7 x 7 x 3 interior nodes of a
// 9 x 9 x 5 node block and evaluates its 8 x 8 x 4 elements, one per thread.
// Each thread writes its element's 24 inputs, scaled by E_e and rounded to
// the form's type, as one row of a 256 x K operand A in shared memory (the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices);
// one thread then issues
//   D[128 x 32] (+)= A[128 x K] * B[K x 32],   two M-tiles,
// with B = KE (rows = outputs, K-major; outputs 24..31 zero) resident in
// shared memory and D in tensor memory (64 columns); the split forms add
// A_hi B_lo + A_lo B_hi (hi = form(x), lo = form(x - hi)).  After the commit
// mbarrier fires, every thread reads its element's 32-column row of D with
// one tcgen05.ld and the node phase sums contributions as in the SIMT path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <string.h>

#include "common.cuh"
#include "kv_tcol.cuh"
#include "kv_tile.cuh"
#include "tc.cuh"

namespace {

constexpr int kTcCols = 64;            // TMEM columns per CTA: two 128 x 32 FP32 tiles
constexpr uint32_t kTcSpin = 1u << 20; // bound of the mbarrier wait

template <int KIND>                    // 1 BF16, 2 FP16
struct TcKind {
  static_assert(KIND == 1 || KIND == 2, "2-byte kinds of the block kernel");
  static constexpr int ESZ = 2;
  static constexpr int KPAD = 32;                       // K per row (24 used)
  static constexpr int ROWB = KPAD * ESZ;               // 64 bytes per row
  static constexpr int KC = ROWB / 16;                  // core matrices along K
  static constexpr int SBO = KC * 128;                  // bytes between 8-row groups
  static constexpr int NKS = 2;                         // MMAs along K (K = 16 each)
  static constexpr int ATILE = 256 * ROWB;
  static constexpr int BTILE = 32 * ROWB;
  static constexpr uint32_t IDESC = make_idesc(KIND == 1 ? 1u : 0u, 128, 32);
};

constexpr int round128(int x) { return (x + 127) / 128 * 128; }

// Shared-memory regions, every one starting on a 128-byte boundary (the
// operands need 16 bytes, the mbarrier 8).
template <int KIND, bool SPLIT>
struct TcLayout {
  using C = TcKind<KIND>;
  static constexpr int R0 = (C::ATILE > 24 * 1024 ? C::ATILE : 24 * 1024);  // A_hi, then out
  static constexpr int OFF_A0 = 0;
  static constexpr int OFF_A1 = round128(OFF_A0 + R0);                       // A_lo (split)
  static constexpr int OFF_B0 = round128(OFF_A1 + (SPLIT ? C::ATILE : 0));
  static constexpr int OFF_B1 = round128(OFF_B0 + C::BTILE);                 // B_lo (split)
  static constexpr int OFF_VS = round128(OFF_B1 + (SPLIT ? C::BTILE : 0));   // [3][405] floats
  static constexpr int OFF_MS = round128(OFF_VS + 3 * BlockShape::NV * 4);   // [405] masks
  static constexpr int OFF_RS = round128(OFF_MS + BlockShape::NV);           // [256] row scales
  static constexpr int OFF_BAR = round128(OFF_RS + 256 * 4);                 // mbarrier, TMEM slot
  static constexpr int BYTES = OFF_BAR + 128;
  static constexpr int ALLOC = BYTES + 128;   // slack to align the dynamic base
};
static_assert(TcLayout<1, false>::OFF_BAR % 128 == 0 && TcLayout<2, true>::OFF_BAR % 128 == 0,
              "aligned regions");

// byte offset of (row, k) in a K-major no-swizzle operand of the kind
template <int KIND>
__host__ __device__ inline int tc_offset(int row, int kbyte) {
  using C = TcKind<KIND>;
  return (row >> 3) * C::SBO + (kbyte >> 4) * 128 + (row & 7) * 16 + (kbyte & 15);
}

// Writes one A row (this thread's element) in the form; returns the factor
// by which the row was scaled (FP16 forms scale each row into [1, 2) to stay
// in range; BF16 returns 1).
template <int KIND, bool SPLIT>
__device__ __forceinline__ float write_a_row(unsigned char* A0, unsigned char* A1, int row,
                                             const float (&a)[24]) {
  {
    float scale = 1.0f, inv = 1.0f;
    if (KIND == 2) {
      float m = 0.f;
#pragma unroll
      for (int k = 0; k < 24; ++k) m = fmaxf(m, fabsf(a[k]));
      if (m > 0.f) {
        const int e = ilogbf(m);
        scale = ldexpf(1.0f, -e);
        inv = ldexpf(1.0f, e);
      }
    }
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) {
      const float x0 = 2 * p < 24 ? a[2 * p] * scale : 0.f;
      const float x1 = 2 * p + 1 < 24 ? a[2 * p + 1] * scale : 0.f;
      if (KIND == 1) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hi[p] = *reinterpret_cast<const uint32_t*>(&h);
        lo[p] = *reinterpret_cast<const uint32_t*>(&l);
      } else {
        const __half2 h = __floats2half2_rn(x0, x1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
        hi[p] = *reinterpret_cast<const uint32_t*>(&h);
        lo[p] = *reinterpret_cast<const uint32_t*>(&l);
      }
    }
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      *reinterpret_cast<uint4*>(A0 + tc_offset<KIND>(row, 16 * kc)) =
          make_uint4(hi[4 * kc], hi[4 * kc + 1], hi[4 * kc + 2], hi[4 * kc + 3]);
      if (SPLIT)
        *reinterpret_cast<uint4*>(A1 + tc_offset<KIND>(row, 16 * kc)) =
            make_uint4(lo[4 * kc], lo[4 * kc + 1], lo[4 * kc + 2], lo[4 * kc + 3]);
    }
    return inv;
  }
}

template <int KIND, bool SPLIT, typename Load, typename Epi>
__device__ __forceinline__ double kv_tc_body(const float* __restrict__ E,
                                             const uint8_t* __restrict__ fixed,
                                             const unsigned char* __restrict__ btile,
                                             const Grid& g, const Load& ld, const Epi& epi,
                                             unsigned char* smem, int32_t* err) {
  using B = BlockShape;
  using C = TcKind<KIND>;
  using L = TcLayout<KIND, SPLIT>;
  unsigned char* A0 = smem + L::OFF_A0;
  unsigned char* A1 = smem + L::OFF_A1;
  unsigned char* B0 = smem + L::OFF_B0;
  unsigned char* B1 = smem + L::OFF_B1;
  float* vs = reinterpret_cast<float*>(smem + L::OFF_VS);
  uint8_t* ms = smem + L::OFF_MS;
  float* rs = reinterpret_cast<float*>(smem + L::OFF_RS);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::OFF_BAR + 8);
  float* out = reinterpret_cast<float*>(A0);   // [24][256], after the MMAs have read A
  const int tid = threadIdx.x, warp = tid >> 5;

  // ---- set-up: B operands, TMEM, mbarrier
  for (int i = tid; i < C::BTILE / 16; i += MFTO_BLOCK) {
    reinterpret_cast<uint4*>(B0)[i] = reinterpret_cast<const uint4*>(btile)[i];
    if (SPLIT) reinterpret_cast<uint4*>(B1)[i] = reinterpret_cast<const uint4*>(btile + C::BTILE)[i];
  }
  if (warp == 0) {
    tmem_alloc(tslot, kTcCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t my_row_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
  const uint32_t a0 = smem_u32(A0), a1 = smem_u32(A1), b0 = smem_u32(B0), b1 = smem_u32(B1);

  const int tx = (g.nx + B::OX - 1) / B::OX, ty = (g.ny + B::OY - 1) / B::OY;
  const int tz = (g.nz + B::OZ - 1) / B::OZ;
  const int n_blocks = tx * ty * tz;
  const int ex = tid & 7, ey = (tid >> 3) & 7, ez = tid >> 6;
  DotAcc<float> red;
  uint32_t phase = 0;
  for (int b = blockIdx.x; b < n_blocks; b += gridDim.x) {
    const int bx = b % tx, by = (b / tx) % ty, bz = b / (tx * ty);
    const int ox = bx * B::OX, oy = by * B::OY, oz = bz * B::OZ;
    // ---- stage the node block and this thread's modulus
    for (int idx = tid; idx < B::NV; idx += MFTO_BLOCK) {
      const int lx = idx % B::VX, ly = (idx / B::VX) % B::VY, lz = idx / (B::VX * B::VY);
      const int gi = ox - 1 + lx, gj = oy - 1 + ly, gk = oz - 1 + lz;
      float va = 0.f, vb = 0.f, vc = 0.f;
      uint8_t fm = 0;
      if (gi >= 0 && gj >= 0 && gk >= 0 && gi < g.nx && gj < g.ny && gk < g.nz) {
        const int node = gi + g.nx * (gj + g.ny * gk);
        fm = fixed[node];
        va = ld(3 * node + 0);
        vb = ld(3 * node + 1);
        vc = ld(3 * node + 2);
        va = (fm & 1) ? 0.f : va;
        vb = (fm & 2) ? 0.f : vb;
        vc = (fm & 4) ? 0.f : vc;
      }
      vs[idx] = va;
      vs[B::NV + idx] = vb;
      vs[2 * B::NV + idx] = vc;
      ms[idx] = fm;
    }
    const int ei = ox - 1 + ex, ej = oy - 1 + ey, ek = oz - 1 + ez;
    float Ee = 0.f;
    if (ei >= 0 && ej >= 0 && ek >= 0 && ei < g.nelx && ej < g.nely && ek < g.nelz)
      Ee = E[ei + g.nelx * (ej + g.nely * ek)];
    __syncthreads();
    // ---- A row of this thread's element: E_e * u_e in the form
    {
      float a[24];
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        const int vi = (ex + (l & 1)) + B::VX * ((ey + ((l >> 1) & 1)) + B::VY * (ez + (l >> 2)));
        a[3 * l + 0] = Ee * vs[vi];
        a[3 * l + 1] = Ee * vs[B::NV + vi];
        a[3 * l + 2] = Ee * vs[2 * B::NV + vi];
      }
      rs[tid] = write_a_row<KIND, SPLIT>(A0, A1, tid, a);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // ---- MMAs (one thread), completion on the mbarrier
    if (tid == 0) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const uint32_t d = tmem + 32 * t;
        const uint32_t arow = (uint32_t)(16 * t * C::SBO);   // 128 rows = 16 row groups
        uint32_t acc = 0;
#pragma unroll
        for (int term = 0; term < (SPLIT ? 3 : 1); ++term) {
          const uint32_t aa = (term == 2 ? a1 : a0) + arow;
          const uint32_t bb = term == 1 ? b1 : b0;
#pragma unroll
          for (int ks = 0; ks < C::NKS; ++ks) {
            const uint64_t da = smem_desc(aa + 256 * ks, 128, C::SBO);
            const uint64_t db = smem_desc(bb + 256 * ks, 128, C::SBO);
            mma_f16(d, da, db, C::IDESC, acc);
            acc = 1;
          }
        }
      }
      mma_commit(bar);
    }
    {
      uint32_t spins = 0;
      bool ok;
      while (!(ok = mbar_try_wait(bar, phase)))
        if (++spins > kTcSpin) break;
      if (!ok) {
        atomicExch(err, 1);
        // keep waiting, still bounded, so TMEM is not read or freed mid-MMA
        for (uint32_t s = 0; s < kTcSpin && !mbar_try_wait(bar, phase); ++s) {
        }
      }
      phase ^= 1u;
    }
    tc_fence_after();
    // ---- read back this element's outputs (A0 is free again: out aliases it)
    {
      float d[32];
      tmem_ld32(my_row_addr, d);
      const float sc = rs[tid];
#pragma unroll
      for (int n = 0; n < 24; ++n) out[n * MFTO_BLOCK + tid] = d[n] * sc;
    }
    tc_fence_before();
    __syncthreads();
    // ---- node phase
    if (tid < B::NO) {
      const int ix = tid % B::OX, iy = (tid / B::OX) % B::OY, iz = tid / (B::OX * B::OY);
      const int gi = ox + ix, gj = oy + iy, gk = oz + iz;
      if (gi < g.nx && gj < g.ny && gk < g.nz) {
        float acc[3] = {0.f, 0.f, 0.f};
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
        const float pn[3] = {vs[vi], vs[B::NV + vi], vs[2 * B::NV + vi]};
        epi(gi + g.nx * (gj + g.ny * gk), acc, pn, ms[vi], red);
      }
    }
    __syncthreads();   // vs, ms, A0/out are rewritten for the next block
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTcCols);
  return red.finish();
}

template <int KIND, bool SPLIT>
__global__ void __launch_bounds__(MFTO_BLOCK)
kv_tc_kernel(const float* __restrict__ E, const float* __restrict__ v, float* __restrict__ y,
             const uint8_t* __restrict__ fixed, const unsigned char* __restrict__ btile, Grid g,
             int32_t* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  kv_tc_body<KIND, SPLIT>(E, fixed, btile, g, TileLoadPlain<float>{v}, TileStore<float>{v, y},
                          smem, err);
}

template <int KIND, bool SPLIT>
__global__ void __launch_bounds__(MFTO_BLOCK)
pcg_kv_tc_kernel(const float* __restrict__ E, const float* __restrict__ z,
                 const float* __restrict__ p_old, float* __restrict__ p_new, float* __restrict__ q,
                 const uint8_t* __restrict__ fixed, const unsigned char* __restrict__ btile, Grid g,
                 PcgScalars* s, double* partials, int32_t* err) {
  if (*(volatile int32_t*)&s->done) return;  // uniform over the grid
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sh[64];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  double red[1];
  red[0] = kv_tc_body<KIND, SPLIT>(E, fixed, btile, g,
                                   TileLoadDirection<float>{z, p_old, (float)s->beta},
                                   TilePcg<float>{p_new, q}, smem, err);
  double tot[1];
  if (last_block_reduce<1, true>(red, partials, &s->ticket_b, tot, sh) && threadIdx.x == 0) {
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


// ---- pipelined column kernels (TF32, split TF32) -------------------------

template <bool SPLIT>
__global__ void __launch_bounds__(MFTO_BLOCK, 2)
kv_tcol_kernel(const float* __restrict__ E, const float* __restrict__ v, float* __restrict__ y,
               const uint8_t* __restrict__ fixed, const unsigned char* __restrict__ btile, Grid g,
               TcolTiling tl, int32_t* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  bool skipped = false;
  kv_tcol_body<TcolDefault, SPLIT>(E, fixed, btile, g, tl, ColLoadPlain{v}, ColStore{v, y}, smem,
                                   ColNoPre{}, &skipped, err);
}

// CG K.v of the ticket graph engine: p = z + beta p_old, q = K p, p.q
// reduced by the last block (alpha formed there).
template <bool SPLIT>
__global__ void __launch_bounds__(MFTO_BLOCK, 2)
pcg_kv_tcol_kernel(const float* __restrict__ E, const float* __restrict__ z,
                   const float* __restrict__ p_old, float* __restrict__ p_new,
                   float* __restrict__ q, const uint8_t* __restrict__ fixed,
                   const unsigned char* __restrict__ btile, Grid g, TcolTiling tl, PcgScalars* s,
                   double* partials, int32_t* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sh[64];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  bool skipped = false;
  DotAcc<float> acc;
  acc.s = kv_tcol_body<TcolDefault, SPLIT>(E, fixed, btile, g, tl, ColLoadDirection{z, p_old, 0.f},
                                           ColPcg{p_new, q}, smem,
                                           ColPreFlagBeta{&s->done, &s->beta}, &skipped, err);
  if (skipped) return;   // uniform over the grid
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

// ---- host side -------------------------------------------------------------

struct FormSpec {
  int kind;     // 0 TF32, 1 BF16, 2 FP16
  bool split;
};

bool form_spec(int form, FormSpec* fs) {
  switch (form) {
    case MFTO_FORM_TF32: *fs = {0, false}; return true;
    case MFTO_FORM_TF32X3: *fs = {0, true}; return true;
    case MFTO_FORM_BF16: *fs = {1, false}; return true;
    case MFTO_FORM_BF16X3: *fs = {1, true}; return true;
    case MFTO_FORM_F16: *fs = {2, false}; return true;
    case MFTO_FORM_F16X3: *fs = {2, true}; return true;
    default: return false;
  }
}

// TF32 rounding on the host, to nearest with ties away from zero (the
// rounding of cvt.rna.tf32.f32 used for A on the device).
float host_tf32(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

template <int KIND>
void build_btile(const double* ke, unsigned char* hi, unsigned char* lo) {
  using C = TcKind<KIND>;
  memset(hi, 0, C::BTILE);
  memset(lo, 0, C::BTILE);
  for (int n = 0; n < 24; ++n)
    for (int k = 0; k < 24; ++k) {
      const float x = (float)ke[n * 24 + k];   // B[k][n] = KE[n][k], stored K-major by n
      const int off = tc_offset<KIND>(n, k * C::ESZ);
      if (KIND == 1) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        memcpy(hi + off, &h, 2);
        memcpy(lo + off, &l, 2);
      } else {
        const __half h = __float2half_rn(x);
        const __half l = __float2half_rn(x - __half2float(h));
        memcpy(hi + off, &h, 2);
        memcpy(lo + off, &l, 2);
      }
    }
}

// B operands of the column kernel: for MMA step s = dy + 2 dz, the 32 x 8
// block B_s[n][k] = KE[3 c_out + i][3 c_in + j] with n = 4 c_out + i (output
// corner c_out, component i < 3) and k = 4 dx + j (input corner
// c_in = dx + 2 dy + 4 dz, component j < 3); rows and columns of the 4th
// components are zero.  hi = tf32(KE), lo = tf32(KE - hi).
void build_btile_tcol(const double* ke, unsigned char* out) {
  memset(out, 0, kTcolBBytes);
  for (int st = 0; st < 4; ++st)
    for (int co = 0; co < 8; ++co)
      for (int i = 0; i < 3; ++i)
        for (int dx = 0; dx < 2; ++dx)
          for (int j = 0; j < 3; ++j) {
            const int ci = dx + 2 * (st & 1) + 4 * (st >> 1);
            const float x = (float)ke[(3 * co + i) * 24 + 3 * ci + j];
            const float hv = host_tf32(x), lv = host_tf32(x - hv);
            const int off = 1024 * st + tcol_b_offset(4 * co + i, 4 * dx + j);
            memcpy(out + off, &hv, 4);
            memcpy(out + kTcolBBytes / 2 + off, &lv, 4);
          }
}

template <int KIND, bool SPLIT>
mfto_status tc_attrs(mfto_handle* h, int* occ_kv, int* occ_pcg) {
  const int smem = TcLayout<KIND, SPLIT>::ALLOC;
  MFTO_CUDA(h, cudaFuncSetAttribute(kv_tc_kernel<KIND, SPLIT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_kv_tc_kernel<KIND, SPLIT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_kv, kv_tc_kernel<KIND, SPLIT>,
                                                             MFTO_BLOCK, smem));
  MFTO_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                   occ_pcg, pcg_kv_tc_kernel<KIND, SPLIT>, MFTO_BLOCK, smem));
  // at most 512 / 64 CTAs of one SM can hold their TMEM columns at once
  const int cap = 512 / kTcCols;
  if (*occ_kv > cap) *occ_kv = cap;
  if (*occ_pcg > cap) *occ_pcg = cap;
  if (*occ_kv < 1) *occ_kv = 1;
  if (*occ_pcg < 1) *occ_pcg = 1;
  return MFTO_OK;
}

// Resident CTAs per SM of a column-kernel launch: as many as shared memory
// holds (dynamic + static + the per-block reservation), at most 2 (the
// register budget of __launch_bounds__) and at most 512 / kTcolCols (TMEM).
// The runtime's occupancy query reports one CTA per SM for kernels that
// allocate tensor memory, so the count is derived here.
template <typename K>
mfto_status tcol_occupancy(mfto_handle* h, K kernel, int dyn, int* occ) {
  int dev = 0, smem_sm = 0, reserved = 0;
  MFTO_CUDA(h, cudaGetDevice(&dev));
  MFTO_CUDA(h, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  MFTO_CUDA(h, cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  cudaFuncAttributes fa;
  MFTO_CUDA(h, cudaFuncGetAttributes(&fa, kernel));
  const int per_block = dyn + (int)fa.sharedSizeBytes + reserved;
  int n = per_block > 0 ? smem_sm / per_block : 1;
  if (n > 2) n = 2;
  if (n > 512 / kTcolCols) n = 512 / kTcolCols;
  if (n < 1) n = 1;
  *occ = n;
  return MFTO_OK;
}

template <bool SPLIT>
mfto_status tcol_attrs(mfto_handle* h, int* occ_kv, int* occ_pcg) {
  MFTO_CUDA(h, cudaFuncSetAttribute(kv_tcol_kernel<SPLIT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, tcol_smem_bytes(1)));
  MFTO_CUDA(h, cudaFuncSetAttribute(pcg_kv_tcol_kernel<SPLIT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, tcol_smem_bytes(2)));
  mfto_status s = tcol_occupancy(h, kv_tcol_kernel<SPLIT>, tcol_smem_bytes(1), occ_kv);
  if (s == MFTO_OK) s = tcol_occupancy(h, pcg_kv_tcol_kernel<SPLIT>, tcol_smem_bytes(2), occ_pcg);
  return s;
}

int tc_index(int kind, bool split) { return 2 * kind + (split ? 1 : 0); }

unsigned grid_for(const mfto_handle* h, int per_sm) {
  const Grid g = make_grid(h->mesh);
  const int64_t nb = (int64_t)((g.nx + 6) / 7) * ((g.ny + 6) / 7) * ((g.nz + 2) / 3);
  int64_t grid = (int64_t)per_sm * h->num_sms;
  if (grid > nb) grid = nb;
  return (unsigned)grid;
}

}  // namespace

int tcol_smem_bytes(int ksrc) {
  return ksrc == 1 ? TcolLayout<TcolDefault, 1>::ALLOC : TcolLayout<TcolDefault, 2>::ALLOC;
}

// Column tiling of a launch of the tensor-core column kernel: chunks of
// h->tcol_nzc node layers if set, else about three tiles per resident CTA
// with chunks of at least 4 layers.
TcolTiling tcol_launch_tiling(const mfto_handle* h, int per_sm, int* grid) {
  using S = TcolDefault;
  const Grid g = make_grid(h->mesh);
  const int64_t ctas = (int64_t)per_sm * h->num_sms;
  int nzc = h->tcol_nzc;
  if (nzc <= 0) {
    const int64_t txy = (int64_t)((g.nx + S::OX - 1) / S::OX) * ((g.ny + S::OY - 1) / S::OY);
    int64_t zch = (3 * ctas + txy - 1) / txy;
    if (zch < 1) zch = 1;
    nzc = (int)((g.nz + zch - 1) / zch);
    if (nzc < 4) nzc = 4;
  }
  const TcolTiling tl = tcol_tiling<S>(g, nzc);
  int64_t n = tl.count();
  if (n > ctas) n = ctas;
  if (n > MFTO_RED_SLOTS) n = MFTO_RED_SLOTS;
  *grid = (int)n;
  return tl;
}

mfto_status tc_init(mfto_handle* h) {
  mfto_status s = MFTO_OK;
  int* o = h->occ_tc;
  if (s == MFTO_OK) s = tcol_attrs<false>(h, &o[0], &o[1]);
  if (s == MFTO_OK) s = tcol_attrs<true>(h, &o[2], &o[3]);
  if (s == MFTO_OK) s = tc_attrs<1, false>(h, &o[4], &o[5]);
  if (s == MFTO_OK) s = tc_attrs<1, true>(h, &o[6], &o[7]);
  if (s == MFTO_OK) s = tc_attrs<2, false>(h, &o[8], &o[9]);
  if (s == MFTO_OK) s = tc_attrs<2, true>(h, &o[10], &o[11]);
  return s;
}

// B operands (KE, hi and lo parts) in the device layouts: [kind][2 *
// MFTO_TC_BTILE], the column kernel's blocks for TF32, hi then lo tiles for
// BF16 and FP16.
mfto_status tc_upload_b(mfto_handle* h, const double* ke) {
  static_assert(kTcolBBytes <= 2 * MFTO_TC_BTILE && TcKind<1>::BTILE <= MFTO_TC_BTILE, "B tile");
  unsigned char packed[3][2 * MFTO_TC_BTILE];
  memset(packed, 0, sizeof(packed));
  build_btile_tcol(ke, packed[0]);
  build_btile<1>(ke, packed[1], packed[1] + TcKind<1>::BTILE);
  build_btile<2>(ke, packed[2], packed[2] + TcKind<2>::BTILE);
  MFTO_CUDA(h, cudaMemcpyAsync(h->d_btc, packed, sizeof(packed), cudaMemcpyHostToDevice, h->stream));
  MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  return MFTO_OK;
}

bool tc_form(int form) {
  FormSpec fs;
  return form_spec(form, &fs);
}

bool tcol_form(int form) { return form == MFTO_FORM_TF32 || form == MFTO_FORM_TF32X3; }

#define MFTO_TC_DISPATCH(KIND_, SPLIT_, CALL)                                          \
  if (fs.kind == KIND_ && fs.split == SPLIT_) {                                         \
    const int occ = h->occ_tc[2 * tc_index(KIND_, SPLIT_) + idx_occ];                   \
    const unsigned grid = grid_for(h, occ);                                             \
    const size_t smem = TcLayout<KIND_, SPLIT_>::ALLOC;                                 \
    const unsigned char* bt = h->d_btc + (size_t)KIND_ * 2 * MFTO_TC_BTILE;             \
    CALL;                                                                               \
  }

mfto_status kv_tc_launch(mfto_handle* h, int form, const float* E, const float* v, float* y,
                         cudaStream_t st) {
  FormSpec fs;
  if (!form_spec(form, &fs)) return mfto_fail(h, MFTO_UNSUPPORTED, "not a tensor-core form");
  const Grid g = make_grid(h->mesh);
  const int idx_occ = 0;
  int32_t* err = &h->d_misc->error;
  if (fs.kind == 0) {
    int grid = 0;
    const TcolTiling tl = tcol_launch_tiling(h, h->occ_tc[2 * tc_index(0, fs.split)], &grid);
    const size_t smem = tcol_smem_bytes(1);
    if (fs.split)
      kv_tcol_kernel<true><<<grid, MFTO_BLOCK, smem, st>>>(E, v, y, h->d_fixed, h->d_btc, g, tl, err);
    else
      kv_tcol_kernel<false><<<grid, MFTO_BLOCK, smem, st>>>(E, v, y, h->d_fixed, h->d_btc, g, tl, err);
    MFTO_LAUNCH_CHECK(h);
    return MFTO_OK;
  }
  MFTO_TC_DISPATCH(1, false, (kv_tc_kernel<1, false><<<grid, MFTO_BLOCK, smem, st>>>(E, v, y, h->d_fixed, bt, g, err)))
  MFTO_TC_DISPATCH(1, true, (kv_tc_kernel<1, true><<<grid, MFTO_BLOCK, smem, st>>>(E, v, y, h->d_fixed, bt, g, err)))
  MFTO_TC_DISPATCH(2, false, (kv_tc_kernel<2, false><<<grid, MFTO_BLOCK, smem, st>>>(E, v, y, h->d_fixed, bt, g, err)))
  MFTO_TC_DISPATCH(2, true, (kv_tc_kernel<2, true><<<grid, MFTO_BLOCK, smem, st>>>(E, v, y, h->d_fixed, bt, g, err)))
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

mfto_status pcg_kv_tc_launch(mfto_handle* h, int form, const float* E, const float* z,
                             const float* p_old, float* p_new, float* q, PcgScalars* s,
                             double* partials, cudaStream_t st) {
  FormSpec fs;
  if (!form_spec(form, &fs)) return mfto_fail(h, MFTO_UNSUPPORTED, "not a tensor-core form");
  const Grid g = make_grid(h->mesh);
  const int idx_occ = 1;
  int32_t* err = &s->tc_error;
  if (fs.kind == 0) {
    int grid = 0;
    const TcolTiling tl = tcol_launch_tiling(h, h->occ_tc[2 * tc_index(0, fs.split) + 1], &grid);
    const size_t smem = tcol_smem_bytes(2);
    if (fs.split)
      pcg_kv_tcol_kernel<true><<<grid, MFTO_BLOCK, smem, st>>>(E, z, p_old, p_new, q, h->d_fixed,
                                                              h->d_btc, g, tl, s, partials, err);
    else
      pcg_kv_tcol_kernel<false><<<grid, MFTO_BLOCK, smem, st>>>(E, z, p_old, p_new, q, h->d_fixed,
                                                               h->d_btc, g, tl, s, partials, err);
    MFTO_LAUNCH_CHECK(h);
    return MFTO_OK;
  }
  MFTO_TC_DISPATCH(1, false, (pcg_kv_tc_kernel<1, false><<<grid, MFTO_BLOCK, smem, st>>>(E, z, p_old, p_new, q, h->d_fixed, bt, g, s, partials, err)))
  MFTO_TC_DISPATCH(1, true, (pcg_kv_tc_kernel<1, true><<<grid, MFTO_BLOCK, smem, st>>>(E, z, p_old, p_new, q, h->d_fixed, bt, g, s, partials, err)))
  MFTO_TC_DISPATCH(2, false, (pcg_kv_tc_kernel<2, false><<<grid, MFTO_BLOCK, smem, st>>>(E, z, p_old, p_new, q, h->d_fixed, bt, g, s, partials, err)))
  MFTO_TC_DISPATCH(2, true, (pcg_kv_tc_kernel<2, true><<<grid, MFTO_BLOCK, smem, st>>>(E, z, p_old, p_new, q, h->d_fixed, bt, g, s, partials, err)))
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

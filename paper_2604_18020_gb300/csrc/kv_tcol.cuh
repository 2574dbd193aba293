// Pipelined tensor-core K.v (tcgen05), column-streaming: the element
// contraction D_e = KE u_e of Eq. (matfree) for every element of one z-layer
// of a tile runs as MMAs whose A operand is the staged node layer itself, so
// no per-element gather is formed at all.
//
// Operand layout.  A tile's node layer is staged in shared memory as one
// 16-byte float4 (x, y, z, 0) per node, at position q = ix + P * iy (node
// pitch P).  The element at position m = ex + P * ey has its 8 corners at
// positions m + dx + P dy of the node layers ez (dz = 0) and ez + 1 (dz = 1).
// In the canonical K-major layout without swizzle, a tcgen05 operand is made
// of core matrices of 8 rows x 16 bytes, rows 16 bytes apart; the descriptor
// gives the byte step between core matrices along M (SBO) and along K (LBO).
// With SBO = 128 (8 positions) and LBO = 16 (one position), the rows m .. m+7
// of the core-matrix pair of one MMA step (K = 8 TF32 values) are exactly the
// corner nodes (dx = 0, dx = 1) of elements m .. m+7 for one (dy, dz): the
// node layer read in place is the element operand.  Four MMA steps, one per
// (dy, dz), cover K = 32 (8 corners x 4 components, the 4th zero), against
// B = KE arranged per step (rows = 24 outputs padded to N = 32, K-major).
// Positions whose element does not exist (the last column ex = P - 1, whose
// dx = 1 corners wrap into the next row, and positions past the tile) give
// rows that are never used.  A tile has 256 positions = two M = 128 MMA tiles.
//
// Split TF32 (SPLIT): every staged value w = v - r (r: a translation common
// to the tile, below) is stored as hi = tf32(w) and lo = tf32(w - hi), KE
// likewise, and D = A_lo B_hi + A_hi B_lo + A_hi B_hi (small products first)
// in FP32 in tensor memory; without SPLIT, r = 0 and only A_hi B_hi.  The
// modulus multiplies the read-back row: E_e (KE u_e).
//
// Pipeline (one CTA, 256 threads, thread t <-> position t; one barrier per
// element layer).  Iteration i (element layer ez = kb - 1 + i):
//   1. stage node layer ez + 1 from a ring filled by asynchronous copies
//      three layers ahead (loader combine, mask, hi/lo split);
//   2. barrier;
//   3. one thread issues the MMAs of element layer ez into TMEM buffer
//      i & 1 and commits them to mbarrier i & 1;
//   4. the owners finish node layer ez - 2 (sums written in iteration i - 1);
//   5. every thread waits for the MMAs of element layer ez - 1 (issued one
//      iteration earlier, so normally complete), reads its row back with
//      tcgen05.ld and forms the column sums of node layer ez - 1: E times the
//      lower-face outputs of element ez - 1 plus the upper-face outputs of
//      element ez - 2 (kept in registers).
// The MMAs of a layer thus overlap the staging of the next layer, the node
// sums of the layer before and the epilogue.  A node's 4 column sums (its
// (dx, dy) corners) are added by its owner in a fixed order, and every
// element row is computed by the same MMA sequence whatever the launch
// shape: results are bit-reproducible.
//
// Tiles own (P - 2) x (R - 1) nodes per layer and recompute a one-element
// halo on the low x / y side and one element layer below their z-chunk (as
// the FP32 column kernel, kv_column.cuh, whose loaders, epilogues and
// pre-steps this body shares).
#pragma once
#include <type_traits>

#include "kv_column.cuh"
#include "tc.cuh"

template <int P_, int R_>
struct TcolShape {
  static constexpr int P = P_;      // positions per node row
  static constexpr int R = R_;      // element rows of a tile
  static constexpr int POS = 256;   // element positions per layer (two M = 128 tiles)
  static constexpr int OX = P - 2;  // owned nodes per row: positions ix = 1 .. P - 2
  static constexpr int OY = R - 1;  // owned node rows iy = 1 .. R - 1
  static constexpr int NODES = (R + 1) * P;   // node positions of a staged layer
  static constexpr int NREAD = POS + P + 1;   // positions the MMAs read
  static constexpr int NPOS = ((NODES > NREAD ? NODES : NREAD) + 7) / 8 * 8;
  static constexpr int NEXTRA = NPOS - POS;   // positions staged by a thread's second slot
  static_assert(P * R <= POS, "a tile's elements fit the two M tiles");
  static_assert(NEXTRA <= POS, "second slots fit one pass");
};

// The launch shape used by the library: 32 x 8 positions, 30 x 7 owned nodes.
using TcolDefault = TcolShape<32, 8>;

constexpr int kTcolRing = 3;            // ring slots (copies three layers ahead)
constexpr int kTcolCols = 128;          // TMEM columns per CTA: two buffers x two 128 x 32 tiles
constexpr uint32_t kTcolSpin = 1u << 20;   // bound of an mbarrier wait (try_wait polls)
constexpr int kTcolBBytes = 8192;       // B operands: [hi | lo][4 steps][32 x 8 TF32]

// Byte offset of B element (n, k) of one MMA step's 32 x 8 block (K-major,
// no swizzle: core matrices 128 B apart along K, 8-row groups 256 B apart).
__host__ __device__ constexpr int tcol_b_offset(int n, int k) {
  return (n >> 3) * 256 + (k >> 2) * 128 + (n & 7) * 16 + (k & 3) * 4;
}

// Shared-memory regions (bytes; every region starts on a 128-byte boundary).
template <typename S, int KSRC>
struct TcolLayout {
  static constexpr int SLOT = S::NPOS * 16;                   // one staged node layer
  static constexpr int NS = 3 * KSRC + 1;                     // ring rows: sources, mask word
  static constexpr int OFF_VH = 0;                            // [3][NPOS] float4, hi
  static constexpr int OFF_VL = OFF_VH + 3 * SLOT;            // [3][NPOS] float4, lo
  static constexpr int OFF_B = OFF_VL + 3 * SLOT;             // [2][4][1024 B]
  static constexpr int OFF_SUM = OFF_B + kTcolBBytes;         // [2][4][256] float4
  static constexpr int OFF_HIST = OFF_SUM + 2 * 4 * 256 * 16; // [4][256] float4
  static constexpr int OFF_RING = OFF_HIST + 4 * 256 * 16;    // [ring][NS][NPOS] float
  static constexpr int OFF_ERING = OFF_RING + kTcolRing * NS * S::NPOS * 4;  // [ring][256] float
  static constexpr int OFF_BAR = (OFF_ERING + kTcolRing * 256 * 4 + 127) / 128 * 128;
  static constexpr int BYTES = OFF_BAR + 128;
  static constexpr int ALLOC = BYTES + 128;   // slack to align the dynamic base
  static_assert(SLOT % 128 == 0 && OFF_SUM % 128 == 0 && OFF_RING % 128 == 0, "aligned regions");
};

// Tiling of the node grid: tile (bx, by, bz) owns nodes [bx OX, +OX) x
// [by OY, +OY) x [bz nzc, +nzc) (clipped to the grid).
struct TcolTiling {
  int tx, ty, tz, nzc;
  __host__ __device__ int count() const { return tx * ty * tz; }
};

template <typename S>
static inline TcolTiling tcol_tiling(const Grid& g, int nzc) {
  TcolTiling t;
  t.tx = (g.nx + S::OX - 1) / S::OX;
  t.ty = (g.ny + S::OY - 1) / S::OY;
  if (nzc < 1) nzc = 1;
  if (nzc > g.nz) nzc = g.nz;
  t.nzc = nzc;
  t.tz = (g.nz + nzc - 1) / nzc;
  return t;
}

// Host side (kv_tc.cu): dynamic shared memory of a launch whose loader has
// ksrc source arrays, the tiling and grid of a launch for a handle (chunks of
// h->tcol_nzc node layers, else automatic), and the forms the kernel runs.
int tcol_smem_bytes(int ksrc);
TcolTiling tcol_launch_tiling(const mfto_handle* h, int per_sm, int* grid);
bool tcol_form(int form);

// Three asynchronous 4-byte copies: the consecutive floats at gsrc into
// shared rows STRIDE bytes apart (zero-filled when !valid).
template <int STRIDE>
__device__ __forceinline__ void tcol_cp4x3(float* sdst, const float* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  const int n = valid ? 4 : 0;
  asm volatile(
      "cp.async.ca.shared.global [%0], [%1], 4, %2;\n"
      "cp.async.ca.shared.global [%0+%3], [%1+4], 4, %2;\n"
      "cp.async.ca.shared.global [%0+%4], [%1+8], 4, %2;\n" ::"r"(d),
      "l"(gsrc), "r"(n), "n"(STRIDE), "n"(2 * STRIDE)
      : "memory");
}

// The body.  Tiles blockIdx.x, blockIdx.x + gridDim.x, ... of tl.  Returns
// this thread's double-float share of the epilogue reduction.  err: set to 1
// when an mbarrier wait gave up (the kernel then still ends; its results are
// not to be used).
template <typename S, bool SPLIT, typename Load, typename Epi, typename Pre>
__device__ __forceinline__ DFloat kv_tcol_body(const float* __restrict__ E,
                                               const uint8_t* __restrict__ fixed,
                                               const unsigned char* __restrict__ btile,
                                               const Grid& g, const TcolTiling& tl, Load ld,
                                               const Epi& epi, unsigned char* smem,
                                               const Pre& pre, bool* skipped, int32_t* err) {
  static_assert(Load::kAsync, "the tensor-core column body stages through asynchronous copies");
  using L = TcolLayout<S, Load::kSrc>;
  constexpr int NS = L::NS;
  constexpr int P = S::P;
  float4* VH = reinterpret_cast<float4*>(smem + L::OFF_VH);
  float4* VL = reinterpret_cast<float4*>(smem + L::OFF_VL);
  float4* SUM = reinterpret_cast<float4*>(smem + L::OFF_SUM);
  float4* HIST = reinterpret_cast<float4*>(smem + L::OFF_HIST);
  float* ring = reinterpret_cast<float*>(smem + L::OFF_RING);
  float* ering = reinterpret_cast<float*>(smem + L::OFF_ERING);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::OFF_BAR + 16);
  const uint32_t* fixed_words = reinterpret_cast<const uint32_t*>(fixed);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int ex = tid % P, ey = tid / P;                 // this thread's position
  const bool elem_pos = ex <= P - 2 && ey <= S::R - 1;  // an element of the tile
  const bool owner = ex >= 1 && ex <= P - 2 && ey >= 1 && ey <= S::R - 1;
  const bool has_extra = tid < S::NEXTRA;
  const int q2 = S::POS + tid;                          // second staged position
  const int ex2 = q2 % P, ey2 = q2 / P;
  DFloat red{0.f, 0.f};
  *skipped = false;
  const int ntiles = tl.count();

  const int nxy = g.nx * g.ny;
  // this thread's place in tile t: in-plane node indices (layer 0) of its two
  // staged positions and of its element, whether they exist, and the tile's
  // reference translation r
  struct Ctx {
    int kb, ke, x0, y0;
    int own_base, extra_base, elem_base;
    bool own_in, extra_in, elem_in;
    float r[3];
  };
  auto ctx_of = [&](int t) {
    const int bx = t % tl.tx, by = (t / tl.tx) % tl.ty, bz = t / (tl.tx * tl.ty);
    Ctx c;
    c.x0 = bx * S::OX - 1;   // node / element origin of position 0
    c.y0 = by * S::OY - 1;
    c.kb = bz * tl.nzc;
    c.ke = min(c.kb + tl.nzc, g.nz);   // owned node layers [kb, ke)
    const int gi = c.x0 + ex, gj = c.y0 + ey, hi = c.x0 + ex2, hj = c.y0 + ey2;
    c.own_in = ey <= S::R && gi >= 0 && gj >= 0 && gi < g.nx && gj < g.ny;
    c.extra_in = has_extra && ey2 <= S::R && hi >= 0 && hj >= 0 && hi < g.nx && hj < g.ny;
    c.elem_in = elem_pos && gi >= 0 && gj >= 0 && gi < g.nelx && gj < g.nely;
    c.own_base = gi + g.nx * gj;
    c.extra_base = hi + g.nx * hj;
    c.elem_base = gi + g.nelx * gj;
    return c;
  };
  // r (split form): the loaded value of the tile's central node of layer
  // kb.  Any translation leaves KE u_e unchanged; subtracting one common to
  // the tile makes the TF32 rounding relative to the tile's deformation
  // instead of its rigid motion, which dominates in soft regions.  As r
  // depends on the operand, the product with the rounded KE picks up the
  // term -(KE_used 1) r per element, which is linear but not symmetric in
  // the operand: with the split KE (KE_hi + KE_lo = KE to about 2^-22) it
  // stays below the rounding of the product itself, with the one-term TF32
  // KE (2^-11) it would not, so the TF32 form keeps r = 0.
  auto reference = [&](Ctx& c) {
#pragma unroll
    for (int k = 0; k < 3; ++k) c.r[k] = 0.f;
    if (!SPLIT) return;
    const int ci = min(max(c.x0 + P / 2, 0), g.nx - 1);
    const int cj = min(max(c.y0 + S::R / 2, 0), g.ny - 1);
    const int node = ci + g.nx * (cj + g.ny * c.kb);
#pragma unroll
    for (int k = 0; k < 3; ++k) c.r[k] = ld(3 * node + k);
  };
  // node layer Lz lives in ring slot and node slot (Lz + 1) mod 3; the
  // slots are passed along as rotating counters (sl)
  auto next_slot = [](int sl) { return sl == 2 ? 0 : sl + 1; };
  // copies of node layer Lz (and the modulus of element layer Lz - 1) into
  // the ring; layers past ke copy nothing but still commit a group
  auto issue = [&](const Ctx& c, int Lz, int sl) {
    const bool lay = Lz >= 0 && Lz <= c.ke && Lz < g.nz;
    float* Rb = ring + sl * NS * S::NPOS;
    {
      const bool in = lay && c.own_in;
      const int node = in ? c.own_base + nxy * Lz : 0;
#pragma unroll
      for (int s = 0; s < Load::kSrc; ++s)
        tcol_cp4x3<S::NPOS * 4>(Rb + 3 * s * S::NPOS + tid, ld.src(s) + 3 * node, in);
      col_cp4(Rb + 3 * Load::kSrc * S::NPOS + tid, fixed_words + (node >> 2), in);
    }
    if (has_extra) {
      const bool in = lay && c.extra_in;
      const int node = in ? c.extra_base + nxy * Lz : 0;
#pragma unroll
      for (int s = 0; s < Load::kSrc; ++s)
        tcol_cp4x3<S::NPOS * 4>(Rb + 3 * s * S::NPOS + q2, ld.src(s) + 3 * node, in);
      col_cp4(Rb + 3 * Load::kSrc * S::NPOS + q2, fixed_words + (node >> 2), in);
    }
    {
      const int el = Lz - 1;
      const bool in = c.elem_in && el >= c.kb - 1 && el >= 0 && el < g.nelz && Lz <= c.ke;
      const int e = in ? c.elem_base + g.nelx * g.nely * el : 0;
      col_cp4(ering + sl * S::POS + tid, E + e, in);
    }
    col_cp_commit();
  };
  // staged value of position q of node layer Lz: masked loaded values, split
  auto stage_one = [&](const Ctx& c, int Lz, int sl, int q, int base, float4* hist_out) {
    const float* Rb = ring + sl * NS * S::NPOS;
    const int node = base + nxy * Lz;   // only its low 2 bits are used
    const uint32_t w = __float_as_uint(Rb[3 * Load::kSrc * S::NPOS + q]);
    const uint32_t fm = (w >> (8 * (node & 3))) & 0xFFu;
    float v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float r[Load::kSrc];
#pragma unroll
      for (int s = 0; s < Load::kSrc; ++s) r[s] = Rb[(3 * s + k) * S::NPOS + q];
      v[k] = ((fm >> k) & 1) ? 0.f : ld.combine(r);
    }
    const float w0 = v[0] - c.r[0], w1 = v[1] - c.r[1], w2 = v[2] - c.r[2];
    float4 hi, lo;
    hi.x = to_tf32(w0);
    hi.y = to_tf32(w1);
    hi.z = to_tf32(w2);
    hi.w = 0.f;
    const int ns = sl * S::NPOS + q;
    VH[ns] = hi;
    if (SPLIT) {
      lo.x = to_tf32(w0 - hi.x);
      lo.y = to_tf32(w1 - hi.y);
      lo.z = to_tf32(w2 - hi.z);
      lo.w = 0.f;
      VL[ns] = lo;
    }
    if (hist_out) *hist_out = make_float4(v[0], v[1], v[2], __uint_as_float(fm));
  };
  auto stage = [&](const Ctx& c, int Lz, int sl) {
    stage_one(c, Lz, sl, tid, c.own_base, &HIST[(Lz & 3) * S::POS + tid]);
    if (has_extra) stage_one(c, Lz, sl, q2, c.extra_base, nullptr);
  };
  auto issue_prologue = [&](const Ctx& c) {
    int sl = c.kb % 3;   // slot of layer kb - 1
#pragma unroll
    for (int j = 0; j < kTcolRing; ++j) {
      issue(c, c.kb - 1 + j, sl);
      sl = next_slot(sl);
    }
  };

  // first tile's prologue copies, then the pre-step while they are in flight
  int t = blockIdx.x;
  if (t < ntiles) issue_prologue(ctx_of(t));
  if (!pre.run(ld)) {
    col_cp_wait<0>();
    *skipped = true;
    return red;
  }
  // ---- set-up: B operands, TMEM, mbarriers
  {
    const uint4* src = reinterpret_cast<const uint4*>(btile);
    uint4* dst = reinterpret_cast<uint4*>(smem + L::OFF_B);
    for (int i = tid; i < kTcolBBytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  if (warp == 0) {
    tmem_alloc(tslot, kTcolCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    // one arrival per M tile: threads 0 and 128 each issue and commit one
    mbar_init(&bar[0], 2);
    mbar_init(&bar[1], 2);
    mbar_init_fence();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t my_lane = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
  const uint32_t vh_addr = smem_u32(VH), vl_addr = smem_u32(VL);
  const uint32_t bh_addr = smem_u32(smem + L::OFF_B), bl_addr = bh_addr + kTcolBBytes / 2;
  constexpr uint32_t IDESC = make_idesc(2u, 128, 32);
  uint32_t phase = 0;   // bit b: parity of mbarrier b's next completion

  // MMAs of M tile j of an element layer whose lower / upper node layers sit
  // in slots sa / sb, into TMEM buffer buf
  auto issue_mmas = [&](int j, int sa, int sb, int buf) {
    const uint32_t lo_off = (uint32_t)(sa * L::SLOT);
    const uint32_t up_off = (uint32_t)(sb * L::SLOT);
    {
      const uint32_t d = tmem + (uint32_t)(buf * 64 + j * 32);
      uint32_t acc = 0;
#pragma unroll
      for (int prod = 0; prod < (SPLIT ? 3 : 1); ++prod) {
        const uint32_t abase = (SPLIT && prod == 0) ? vl_addr : vh_addr;
        const uint32_t bbase = (SPLIT && prod == 1) ? bl_addr : bh_addr;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint32_t a = abase + ((s >> 1) ? up_off : lo_off) +
                             (uint32_t)((128 * j + (s & 1) * P) * 16);
          mma_tf32(d, smem_desc(a, 16, 128), smem_desc(bbase + 1024 * s, 128, 256), IDESC, acc);
          acc = 1;
        }
      }
    }
  };
  // lane 0 of each warp polls the mbarrier; the warp barrier that follows
  // (with tcgen05.fence::after_thread_sync in every thread) orders the
  // warp's TMEM reads after the MMAs it observed complete
  auto wait_bar = [&](int b) {
    const uint32_t par = (phase >> b) & 1u;
    if ((tid & 31) == 0) {
      uint32_t spins = 0;
      bool ok;
      while (!(ok = mbar_try_wait(&bar[b], par)))
        if (++spins > kTcolSpin) break;
      if (!ok) {
        atomicExch(err, 1);
        // keep waiting, still bounded, so TMEM is not read or freed mid-MMA
        for (uint32_t s2 = 0; s2 < kTcolSpin && !mbar_try_wait(&bar[b], par); ++s2) {
        }
      }
    }
    __syncwarp();
    phase ^= 1u << b;
  };

  auto run_tile = [&](const Ctx& c) {
    const int kb = c.kb, ke = c.ke;
    const int n_el = ke - kb + 1;   // element layers kb - 1 .. ke - 1
    const bool own_node = owner && c.own_in;
    // owner's sum of node layer Lz: its (dx, dy) = (0,0), (1,0), (0,1), (1,1)
    // corners, from the columns at positions t, t - 1, t - P, t - P - 1
    auto finish = [&](int Lz) {
      if (!own_node) return;
      const float4* Sm = SUM + (Lz & 1) * 4 * S::POS;
      const float4 a = Sm[tid], b = Sm[S::POS + tid - 1];
      const float4 cc = Sm[2 * S::POS + tid - P], d = Sm[3 * S::POS + tid - P - 1];
      float acc[3];
      acc[0] = ((a.x + b.x) + cc.x) + d.x;
      acc[1] = ((a.y + b.y) + cc.y) + d.y;
      acc[2] = ((a.z + b.z) + cc.z) + d.z;
      const float4 hv = HIST[(Lz & 3) * S::POS + tid];
      const float pn[3] = {hv.x, hv.y, hv.z};
      epi(c.own_base + nxy * Lz, acc, pn, (uint8_t)__float_as_uint(hv.w), red);
    };
    // node layer kb - 1
    int sa = kb % 3;            // slot of node layer ez (kb - 1 at first)
    col_cp_wait<kTcolRing - 1>();
    stage(c, kb - 1, sa);
    issue(c, kb - 1 + kTcolRing, sa);
    int sb = next_slot(sa);     // slot of node layer ez + 1
    float U[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k][0] = U[k][1] = U[k][2] = 0.f;
    float Eprev = 0.f;
    for (int i = 0; i <= n_el; ++i) {
      const int ez = kb - 1 + i;
      const bool mma = i < n_el;
      float Ecur = 0.f;
      if (mma) {
        col_cp_wait<kTcolRing - 1>();
        stage(c, ez + 1, sb);
        Ecur = ering[sb * S::POS + tid];   // modulus of element layer ez
        issue(c, ez + 1 + kTcolRing, sb);
        fence_proxy_async_smem();
      }
      tc_fence_before();
      __syncthreads();
      if (mma && (tid & 127) == 0) {
        tc_fence_after();
        issue_mmas(tid >> 7, sa, sb, i & 1);
        mma_commit(&bar[i & 1]);
      }
      sa = sb;
      sb = next_slot(sb);
      if (ez - 2 >= kb) finish(ez - 2);
      if (i >= 1) {
        const int b = (i - 1) & 1;
        wait_bar(b);
        tc_fence_after();
        float d[32];
        tmem_ld32(my_lane + (uint32_t)(b * 64), d);
        tc_fence_before();
        // column sums of node layer ez - 1
        float4 Sc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Sc[k].x = fmaf(Eprev, d[4 * k + 0], U[k][0]);
          Sc[k].y = fmaf(Eprev, d[4 * k + 1], U[k][1]);
          Sc[k].z = fmaf(Eprev, d[4 * k + 2], U[k][2]);
          Sc[k].w = 0.f;
          U[k][0] = Eprev * d[16 + 4 * k + 0];
          U[k][1] = Eprev * d[16 + 4 * k + 1];
          U[k][2] = Eprev * d[16 + 4 * k + 2];
        }
        if (ez - 1 >= kb) {
          float4* Sm = SUM + ((ez - 1) & 1) * 4 * S::POS;
#pragma unroll
          for (int k = 0; k < 4; ++k) Sm[k * S::POS + tid] = Sc[k];
        }
      }
      Eprev = Ecur;
    }
    __syncthreads();
    finish(ke - 1);
  };

  for (; t < ntiles; t += gridDim.x) {
    Ctx c = ctx_of(t);
    if (t != (int)blockIdx.x) issue_prologue(c);
    reference(c);
    run_tile(c);
  }
  col_cp_wait<0>();   // the trailing (empty) groups
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTcolCols);
  return red;
}

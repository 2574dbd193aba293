// Column-streaming FP32 K.v (Eq. matfree): the element operator of
// modes.cuh applied along z-columns of elements, one column per thread, with
// the per-face halves of the mode transform carried from one element layer
// to the next.
//
// A CTA of 256 threads covers CX x CY = 32 x 8 element columns and walks
// their element layers bottom to top over a chunk of node layers.  It owns
// the interior (CX-1) x (CY-1) nodes of every node layer of the chunk; the
// one-column halo on the low x/y side and one element layer below the chunk
// are recomputed by the neighbouring CTA (no atomics, no second pass).
//
// Per element layer ez a thread
//   1. stages its own node of layer ez+1 (threads 0..40 also the tile's
//      last node row / column) into a shared node layer (the x/y pair as one
//      8-byte word, then z; two buffers, three in kv_column_body_async), with
//      the fixed DOFs zeroed.  The node layers come from a ring in shared memory
//      filled by asynchronous copies two layers ahead (kv_column_body_async;
//      loaders that must read L2 directly stage one layer ahead through
//      registers instead, kv_column_body_regs);
//   2. after the layer's one barrier, finishes node layer ez-1 (below);
//   3. reads the 4 upper corners of its element and forms their face modes
//      (x and y stages of the butterfly); the face modes of the lower corners
//      are those of the previous layer, kept in registers, so each node
//      layer's face transform is computed once per column, not twice;
//   4. completes the z stage, applies the unit mode operator, and undoes the z
//      stage with the modulus folded in: lower = E (s - d), upper = E (s + d);
//   5. adds its lower-face output to the upper-face output of the element
//      below (still in mode space), undoes the y and x stages once per node
//      layer, and publishes the 4 corner sums of the column (12 values: four
//      x/y pairs as 8-byte words, four z);
//   6. one layer later (step 2), the owner of node (ex, ey) sums the 4
//      columns around the node in a fixed order and hands the result to the
//      epilogue.
// The element operator costs 48 (forward) + 48 (mode operator) + 36 (inverse
// z with E) + 12 (face sum) + 24 (inverse y, x) = 168 FP32 operations per
// element, against 1152 for the dense 24 x 24 product; every output is
// written once, by one thread, in a fixed order, so results are
// bit-reproducible and independent of the launch shape.
#pragma once
#include <type_traits>

#include "common.cuh"

struct ColShape {
  static constexpr int CX = 32, CY = 8;            // element columns of a CTA
  static constexpr int NX = CX + 1, NY = CY + 1;   // node tile of one layer
  static constexpr int NV = NX * NY;               // 297 staged nodes
  // a staged node layer: the x/y pairs of its NV nodes (float2), then their z;
  // layers LS floats apart (even, so that every pair is 8-byte aligned)
  static constexpr int LS = 3 * NV + 1;
  static constexpr int OX = CX - 1, OY = CY - 1;   // owned nodes per layer: 31 x 7
  static constexpr int NEXTRA = NV - CX * CY;      // 41 nodes staged by a second thread
  static constexpr size_t smem_bytes = sizeof(float) * (2 * LS + 2 * 12 * CX * CY);
};
static_assert(ColShape::CX * ColShape::CY == MFTO_BLOCK, "one column per thread");
static_assert(ColShape::NEXTRA <= MFTO_BLOCK, "extra nodes fit one pass");

// Tiling of the node grid by column tiles: tile (tx, ty, tz) owns nodes
// [tx OX, +OX) x [ty OY, +OY) x [tz nzc, +nzc) (clipped to the grid).
struct ColTiling {
  int tx, ty, tz, nzc;
  // per xy tile (bx + tx by): nonzero when a node the tile stages is fixed
  // (any z); NULL: every tile is treated as having fixed nodes
  const uint8_t* fixed_tiles;
  __host__ __device__ int count() const { return tx * ty * tz; }
};

static inline ColTiling col_tiling(const Grid& g, int nzc) {
  ColTiling t;
  t.fixed_tiles = nullptr;
  t.tx = (g.nx + ColShape::OX - 1) / ColShape::OX;
  t.ty = (g.ny + ColShape::OY - 1) / ColShape::OY;
  if (nzc < 1) nzc = 1;
  if (nzc > g.nz) nzc = g.nz;
  t.nzc = nzc;
  t.tz = (g.nz + nzc - 1) / nzc;
  return t;
}

// Chunk length along z for a grid of at most `ctas` resident CTAs: split
// the columns into about three tiles per resident CTA (so that the
// grid-stride loop balances), but keep chunks of at least `min_nzc` node
// layers (a chunk of n layers recomputes n + 1 element layers).
static inline int col_chunk(const Grid& g, int64_t ctas, int min_nzc) {
  const int64_t txy = (int64_t)((g.nx + ColShape::OX - 1) / ColShape::OX) *
                      ((g.ny + ColShape::OY - 1) / ColShape::OY);
  int64_t zch = (3 * ctas + txy - 1) / txy;
  if (zch < 1) zch = 1;
  int nzc = (int)((g.nz + zch - 1) / zch);
  if (nzc < min_nzc) nzc = min_nzc;
  if (nzc > g.nz) nzc = g.nz;
  return nzc;
}

// Column tiling and grid of a standalone launch of a column kernel for a
// handle (kv_tile.cu): z-chunks of the autotuned length, else sized for
// per_sm resident CTAs per SM.
struct mfto_handle;
ColTiling col_launch_tiling(const mfto_handle* h, int per_sm, int* grid);

// Loaders of one node's 3 components (already masked by the caller).  A
// loader reads a raw value (raw) and turns it into the loaded value (val);
// only the direction loaders need a scalar for the second step, so a kernel
// can issue its first loads before that scalar is known (the pre-steps
// below).
struct ColLoadPlain {                 // v, through L1
  using Raw = float;
  static constexpr bool kAsync = true;  // staged by asynchronous copies (src / combine)
  static constexpr int kSrc = 1;
  const float* v;
  __device__ __forceinline__ const float* src(int) const { return v; }
  __device__ __forceinline__ float combine(const float (&r)[kSrc]) const { return r[0]; }
  __device__ __forceinline__ Raw raw(int idx) const { return v[idx]; }
  __device__ __forceinline__ float val(Raw r) const { return r; }
  __device__ __forceinline__ float operator()(int idx) const { return v[idx]; }
};

struct ColLoadDirectionL2 {           // z + beta p, from L2 (written inside a persistent launch)
  struct Raw { float z, p; };
  // 4-byte asynchronous copies go through L1, which may hold lines that other
  // CTAs of the same launch have since rewritten: staged through registers
  static constexpr bool kAsync = false;
  const float* z;
  const float* p;
  float beta;
  __device__ __forceinline__ Raw raw(int idx) const { return {__ldcg(z + idx), __ldcg(p + idx)}; }
  __device__ __forceinline__ float val(Raw r) const { return r.z + beta * r.p; }
  __device__ __forceinline__ float operator()(int idx) const { return val(raw(idx)); }
};

struct ColLoadDirection {             // z + beta p, through L1 (separate launches)
  struct Raw { float z, p; };
  static constexpr bool kAsync = true;
  static constexpr int kSrc = 2;
  const float* z;
  const float* p;
  float beta;
  __device__ __forceinline__ const float* src(int i) const { return i == 0 ? z : p; }
  __device__ __forceinline__ float combine(const float (&r)[kSrc]) const { return r[0] + beta * r[1]; }
  __device__ __forceinline__ Raw raw(int idx) const { return {z[idx], p[idx]}; }
  __device__ __forceinline__ float val(Raw r) const { return r.z + beta * r.p; }
  __device__ __forceinline__ float operator()(int idx) const { return val(raw(idx)); }
};

// Pre-steps: run once per launch by every thread of the CTA, after the first
// two node layers of the first tile have been requested from memory and
// before they are used.  run() may set the loader's scalar and returns false
// when the launch has nothing to do (uniform over the grid); the body then
// returns at once, with `*skipped` set.  A pre-step's global loads may go out
// before the body's first copies: issue() starts them and returns them in a
// State, run(ld, state) finishes; run(ld) does both at once.
struct ColNoPre {
  struct State {};
  __device__ __forceinline__ State issue() const { return {}; }
  template <typename Load>
  __device__ __forceinline__ bool run(Load&, const State&) const { return true; }
  template <typename Load>
  __device__ __forceinline__ bool run(Load&) const { return true; }
};

// The done flag and beta of a CG iteration whose scalars a previous launch
// left on the device (one round trip, overlapped with the first loads).
struct ColPreFlagBeta {
  const int32_t* done;
  const double* beta;
  struct State {};
  __device__ __forceinline__ State issue() const { return {}; }
  template <typename Load>
  __device__ __forceinline__ bool run(Load& ld, const State&) const { return run(ld); }
  template <typename Load>
  __device__ __forceinline__ bool run(Load& ld) const {
    int d = 0;
    const float b = flag_and_scalar_f32(done, beta, &d);
    if (d) return false;
    ld.beta = b;
    return true;
  }
};

// Epilogues: what the owner of a node does with its 3 sums.  red accumulates
// the node's p.q (double-float; the three products are summed in FP32 first).
struct ColStore {                     // plain K.v: y = sum, y_fixed = v
  const float* v;
  float* y;
  __device__ __forceinline__ void operator()(int node, const float (&acc)[3], const float (&pn)[3],
                                             uint8_t fm, DFloat& red) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) y[3 * node + c] = ((fm >> c) & 1) ? v[3 * node + c] : acc[c];
  }
};

struct ColPcg {                       // CG: p_new stored, q = K p_new, p_new.q accumulated
  float* p_new;
  float* q;
  __device__ __forceinline__ void operator()(int node, const float (&acc)[3], const float (&pn)[3],
                                             uint8_t fm, DFloat& red) const {
    float qc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      qc[c] = ((fm >> c) & 1) ? pn[c] : acc[c];
      p_new[3 * node + c] = pn[c];
      q[3 * node + c] = qc[c];
    }
    const float t = fmaf(pn[0], qc[0], fmaf(pn[1], qc[1], pn[2] * qc[2]));
    red = df_add(red, DFloat{t, 0.f});
  }
};

// One node's masked values and mask, fetched for a later stage.
struct ColNode {
  float v[3];
  uint8_t fm;
};

// One node's raw loads and mask (in: inside the node grid).
template <typename Raw>
struct ColNodeRaw {
  Raw v[3];
  uint8_t fm;
  bool in;
};

template <typename Load>
__device__ __forceinline__ ColNodeRaw<typename Load::Raw> col_fetch_raw(
    const Load& ld, const uint8_t* __restrict__ fixed, const Grid& g, int gi, int gj, int gk) {
  ColNodeRaw<typename Load::Raw> n;
  n.fm = 0;
  n.in = gi >= 0 && gj >= 0 && gk >= 0 && gi < g.nx && gj < g.ny && gk < g.nz;
  if (n.in) {
    const int node = gi + g.nx * (gj + g.ny * gk);
    n.fm = fixed[node];
#pragma unroll
    for (int c = 0; c < 3; ++c) n.v[c] = ld.raw(3 * node + c);
  }
  return n;
}

template <typename Load>
__device__ __forceinline__ ColNode col_finish(const Load& ld,
                                              const ColNodeRaw<typename Load::Raw>& r) {
  ColNode n{{0.f, 0.f, 0.f}, r.fm};
  if (r.in) {
#pragma unroll
    for (int c = 0; c < 3; ++c) n.v[c] = ((r.fm >> c) & 1) ? 0.f : ld.val(r.v[c]);
  }
  return n;
}

template <typename Load>
__device__ __forceinline__ ColNode col_fetch(const Load& ld, const uint8_t* __restrict__ fixed,
                                             const Grid& g, int gi, int gj, int gk) {
  ColNode n{{0.f, 0.f, 0.f}, 0};
  if (gi >= 0 && gj >= 0 && gk >= 0 && gi < g.nx && gj < g.ny && gk < g.nz) {
    const int node = gi + g.nx * (gj + g.ny * gk);
    const uint8_t fm = fixed[node];
    const float a = ld(3 * node + 0), b = ld(3 * node + 1), c = ld(3 * node + 2);
    n.v[0] = (fm & 1) ? 0.f : a;
    n.v[1] = (fm & 2) ? 0.f : b;
    n.v[2] = (fm & 4) ? 0.f : c;
    n.fm = fm;
  }
  return n;
}

__device__ __forceinline__ float col_modulus(const float* __restrict__ E, const Grid& g, int ei,
                                             int ej, int ek) {
  return (ei >= 0 && ej >= 0 && ek >= 0 && ei < g.nelx && ej < g.nely && ek < g.nelz)
             ? E[ei + g.nelx * (ej + g.nely * ek)]
             : 0.f;
}

// Packed FP32 pairs (sm_100 and later): one instruction applies the same
// IEEE operation, with the same rounding, to both lanes, so a pair computes
// bit for bit what two scalar instructions would.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Values of the three displacement components at the 4 places (a + 2b) of
// one face: corner values, face modes or outputs.  The x and y components
// go through identical butterflies, z stages and modulus scaling, so they
// are held as one packed pair; z is a plain float.
struct ColFace {
  float2 xy[4];
  float z[4];
};

// face modes (x then y stage) of the 4 corners (a + 2b) of one face, per component
__device__ __forceinline__ void face_forward(const float* __restrict__ layer, int base,
                                             ColFace& F) {
  const float2* Lxy = reinterpret_cast<const float2*>(layer) + base;
  const float* Lz = layer + 2 * ColShape::NV + base;
  constexpr int NX = ColShape::NX;
  const float2 c0 = Lxy[0], c1 = Lxy[1], c2 = Lxy[NX], c3 = Lxy[NX + 1];
  const float2 m0 = add2(c0, c1), m1 = sub2(c1, c0), m2 = add2(c2, c3), m3 = sub2(c3, c2);
  F.xy[0] = add2(m0, m2);
  F.xy[2] = sub2(m2, m0);
  F.xy[1] = add2(m1, m3);
  F.xy[3] = sub2(m3, m1);
  const float z0 = Lz[0], z1 = Lz[1], z2 = Lz[NX], z3 = Lz[NX + 1];
  const float n0 = z0 + z1, n1 = z1 - z0, n2 = z2 + z3, n3 = z3 - z2;
  F.z[0] = n0 + n2;
  F.z[2] = n2 - n0;
  F.z[1] = n1 + n3;
  F.z[3] = n3 - n1;
}

// Applies the element to face modes Flo (node layer ez) and Fup (layer ez+1):
// lo, up receive E * (the inverse z stage of the mode operator's output).
// Mode m = f + 4 s of component c: face mode f, z sum (s = 0) or difference.
__device__ __forceinline__ void col_element(const ColFace& Flo, const ColFace& Fup, float E,
                                            const ModeCoef<float>& K, ColFace& lo, ColFace& up) {
  float2 X[8], Y[8];   // components x, y
  float xz[8], yz[8];  // component z
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    X[f] = add2(Flo.xy[f], Fup.xy[f]);       // z sum
    X[f | 4] = sub2(Fup.xy[f], Flo.xy[f]);   // z difference
    xz[f] = Flo.z[f] + Fup.z[f];
    xz[f | 4] = Fup.z[f] - Flo.z[f];
  }
  // component c of mode m
  auto xc = [&](int c, int m) -> float { return c == 0 ? X[m].x : (c == 1 ? X[m].y : xz[m]); };
  auto yc = [&](int c, int m) -> float& { return c == 0 ? Y[m].x : (c == 1 ? Y[m].y : yz[m]); };
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    Y[m].x = K.diag[0][m] * X[m].x;
    Y[m].y = K.diag[1][m] * X[m].y;
    yz[m] = K.diag[2][m] * xz[m];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (i == j) continue;
      const int t = 3 - i - j;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int tb = mt << t;
        float& a = yc(i, (1 << i) | tb);
        a = fmaf(K.lamM[mt], xc(j, (1 << j) | tb), a);
        float& b = yc(i, (1 << j) | tb);
        b = fmaf(K.muM[mt], xc(j, (1 << i) | tb), b);
      }
    }
  // lo = E y - E y', up = E y + E y' (y' the z-difference partner), with
  // E y' rounded once: -(E y') is formed as (-E) y', exactly its negation
  const float2 E2 = make_float2(E, E), nE2 = make_float2(-E, -E);
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const float2 ed = mul2(E2, Y[f | 4]), ned = mul2(nE2, Y[f | 4]);
    lo.xy[f] = fma2(E2, Y[f], ned);
    up.xy[f] = fma2(E2, Y[f], ed);
    const float edz = E * yz[f | 4];
    lo.z[f] = fmaf(E, yz[f], -edz);
    up.z[f] = fmaf(E, yz[f], edz);
  }
}

// The 4 corner values (a + 2b) of summed face modes: inverse y, then x stage.
__device__ __forceinline__ void face_inverse(const ColFace& M, ColFace& S) {
  {
    const float2 a0 = sub2(M.xy[0], M.xy[2]), a2 = add2(M.xy[0], M.xy[2]);
    const float2 a1 = sub2(M.xy[1], M.xy[3]), a3 = add2(M.xy[1], M.xy[3]);
    S.xy[0] = sub2(a0, a1);
    S.xy[1] = add2(a0, a1);
    S.xy[2] = sub2(a2, a3);
    S.xy[3] = add2(a2, a3);
  }
  const float a0 = M.z[0] - M.z[2], a2 = M.z[0] + M.z[2];
  const float a1 = M.z[1] - M.z[3], a3 = M.z[1] + M.z[3];
  S.z[0] = a0 - a1;
  S.z[1] = a0 + a1;
  S.z[2] = a2 - a3;
  S.z[3] = a2 + a3;
}

// Sum of two faces (the upper face of one element and the lower face of the next).
__device__ __forceinline__ void face_add(const ColFace& a, const ColFace& b, ColFace& s) {
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    s.xy[f] = add2(a.xy[f], b.xy[f]);
    s.z[f] = a.z[f] + b.z[f];
  }
}

// The 12 corner sums of one column into shared memory: the x/y pairs of
// corner a at Sm2[a MFTO_BLOCK + tid] (Sm2 = Sm as float2, 8-byte aligned),
// z at Sm[(8 + a) MFTO_BLOCK + tid].
__device__ __forceinline__ void face_store(const ColFace& S, float* Sm, int tid) {
  float2* Sm2 = reinterpret_cast<float2*>(Sm);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    Sm2[a * MFTO_BLOCK + tid] = S.xy[a];
    Sm[(8 + a) * MFTO_BLOCK + tid] = S.z[a];
  }
}

// Owner's sum of one node from the corner sums of the 4 columns around it, in
// the fixed order: columns (ex-1, ey-1), (ex, ey-1), (ex-1, ey), (ex, ey)
// contribute their corners 3, 2, 1, 0.
__device__ __forceinline__ void node_sum(const float* Sm, int tid, float (&acc)[3]) {
  constexpr int B = MFTO_BLOCK, CX = ColShape::CX;
  const float2* Sm2 = reinterpret_cast<const float2*>(Sm);
  auto pair = [&](int a, int i) { return Sm2[a * B + i]; };
  float2 s = pair(3, tid - CX - 1);
  s = add2(s, pair(2, tid - CX));
  s = add2(s, pair(1, tid - 1));
  s = add2(s, pair(0, tid));
  float sz = Sm[(8 + 3) * B + tid - CX - 1];
  sz += Sm[(8 + 2) * B + tid - CX];
  sz += Sm[(8 + 1) * B + tid - 1];
  sz += Sm[(8 + 0) * B + tid];
  acc[0] = s.x;
  acc[1] = s.y;
  acc[2] = sz;
}

// One staged node's 3 values into a node layer (x/y pair, then z).
__device__ __forceinline__ void col_put_node(float* layer, int slot, const float (&v)[3]) {
  reinterpret_cast<float2*>(layer)[slot] = make_float2(v[0], v[1]);
  layer[2 * ColShape::NV + slot] = v[2];
}

__device__ __forceinline__ void face_zero(ColFace& F) {
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    F.xy[f] = make_float2(0.f, 0.f);
    F.z[f] = 0.f;
  }
}
// Tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... of `tl`.  Returns this
// thread's double-float share of the epilogue reduction (sum over the block
// with DotAcc-style finishing by the caller).
//
// One barrier per element layer.  Iteration ez (element layer ez, between
// node layers ez and ez + 1) stages node layer ez + 1, crosses the barrier,
// finishes node layer ez - 1 (the owners sum the corner sums that iteration
// ez - 1 wrote), then computes element ez and writes the corner sums of node
// layer ez.  Node layers and corner sums are double-buffered by layer
// parity; a buffer is rewritten only after the barrier that follows its last
// read.  Node layer ke - 1 is finished after the loop, behind one more
// barrier.
template <typename Load, typename Epi, typename Pre>
__device__ __forceinline__ DFloat kv_column_body_regs(const float* __restrict__ E,
                                                      const uint8_t* __restrict__ fixed,
                                                      const ModeCoef<float>& K, const Grid& g,
                                                      const ColTiling& tl, Load ld,
                                                      const Epi& epi, float* smem,
                                                      const Pre& pre, bool* skipped) {
  using S = ColShape;
  float* nodes = smem;                          // [2][LS], slot of node layer k: k & 1
  float* sums = smem + 2 * S::LS;               // [2][12][256] corner sums, slot k & 1
  const int tid = threadIdx.x;
  const int ex = tid % S::CX, ey = tid / S::CX;
  // second staged node of threads < NEXTRA: the top row (y = CY), then the
  // right column (x = CX)
  const bool has_extra = tid < S::NEXTRA;
  const int xx = tid < S::CX ? tid : S::CX;
  const int xy = tid < S::CX ? S::CY : tid - S::CX;
  const bool owner = ex >= 1 && ey >= 1;
  DFloat red{0.f, 0.f};
  *skipped = false;
  const int ntiles = tl.count();
  bool first = true;
  for (int t = blockIdx.x; t < ntiles || first; t += gridDim.x) {
    const bool live = t < ntiles;   // false only for the pre-step of a CTA without tiles
    const int bx = t % tl.tx, by = (t / tl.tx) % tl.ty, bz = t / (tl.tx * tl.ty);
    const int x0 = bx * S::OX - 1, y0 = by * S::OY - 1;   // node / element origin of column 0
    const int kb = bz * tl.nzc;
    const int ke = min(kb + tl.nzc, g.nz);                // owned node layers [kb, ke)
    const int gi = x0 + ex, gj = y0 + ey;                  // this column's element (and node)
    const int hi = x0 + xx, hj = y0 + xy;                  // the extra node
    const bool own_node = owner && gi < g.nx && gj < g.ny;
    auto stage = [&](int k, const ColNode& own, const ColNode& extra) {
      float* L = nodes + (k & 1) * S::LS;
      col_put_node(L, ey * S::NX + ex, own.v);
      if (has_extra) col_put_node(L, xy * S::NX + xx, extra.v);
    };
    // prologue: node layers kb - 1 and kb requested together (raw), then the
    // pre-step, then layer kb - 1 staged
    ColNodeRaw<typename Load::Raw> r0{}, r0x{}, r1{}, r1x{};
    float Ecur = 0.f;
    if (live) {
      r0 = col_fetch_raw(ld, fixed, g, gi, gj, kb - 1);
      r1 = col_fetch_raw(ld, fixed, g, gi, gj, kb);
      if (has_extra) {
        r0x = col_fetch_raw(ld, fixed, g, hi, hj, kb - 1);
        r1x = col_fetch_raw(ld, fixed, g, hi, hj, kb);
      }
      Ecur = col_modulus(E, g, gi, gj, kb - 1);
    }
    if (first) {
      first = false;
      if (!pre.run(ld)) {
        *skipped = true;
        return red;
      }
    }
    if (!live) break;
    ColNode own = col_finish(ld, r0), extra{{0.f, 0.f, 0.f}, 0};
    if (has_extra) extra = col_finish(ld, r0x);
    stage(kb - 1, own, extra);
    own = col_finish(ld, r1);
    if (has_extra) extra = col_finish(ld, r1x);
    __syncthreads();
    // face modes and upper-face outputs ping-pong between two register sets
    // (the z loop is unrolled by two, so nothing is copied between layers)
    ColFace F0, F1, U0, U1;
    face_forward(nodes + ((kb - 1) & 1) * S::LS, ey * S::NX + ex, F0);
    face_zero(U0);
    ColNode mine = own;          // this column's node of layer ez + 1 (after staging)
    ColNode mine_cur = own;      // of layer ez
    ColNode mine_prev = own;     // of layer ez - 1 (finished in iteration ez)
    // owner's sum of node layer k from the corner sums in slot k & 1:
    // columns (ex-1, ey-1), (ex, ey-1), (ex-1, ey), (ex, ey) contribute their
    // corners 3, 2, 1, 0
    auto finish = [&](int k, const ColNode& nv) {
      if (own_node) {
        float acc[3];
        node_sum(sums + (k & 1) * 12 * MFTO_BLOCK, tid, acc);
        epi(gi + g.nx * (gj + g.ny * k), acc, nv.v, nv.fm, red);
      }
    };
    // one element layer: Flo = face modes of node layer ez (in), Fup = those of
    // ez + 1 (out), upp = upper-face outputs of element ez - 1 (in), up = those
    // of element ez (out)
    auto layer = [&](int ez, const ColFace& Flo, ColFace& Fup, const ColFace& upp, ColFace& up) {
      // stage node layer ez + 1; fetch layer ez + 2 and the next modulus
      stage(ez + 1, own, extra);
      mine_prev = mine_cur;
      mine_cur = mine;
      mine = own;
      const float Ee = Ecur;
      if (ez + 1 < ke) {
        own = col_fetch(ld, fixed, g, gi, gj, ez + 2);
        if (has_extra) extra = col_fetch(ld, fixed, g, hi, hj, ez + 2);
        Ecur = col_modulus(E, g, gi, gj, ez + 1);
      }
      __syncthreads();
      // node layer ez - 1 (its corner sums were written in iteration ez - 1)
      if (ez - 1 >= kb) finish(ez - 1, mine_prev);
      // upper face modes, element operator
      ColFace lo;
      face_forward(nodes + ((ez + 1) & 1) * S::LS, ey * S::NX + ex, Fup);
      col_element(Flo, Fup, Ee, K, lo, up);
      if (ez >= kb) {
        // node layer ez: upper face of element ez - 1 plus lower face of ez
        ColFace Ms, Sc;
        face_add(upp, lo, Ms);
        face_inverse(Ms, Sc);
        face_store(Sc, sums + (ez & 1) * 12 * MFTO_BLOCK, tid);
      }
    };
    for (int ez = kb - 1; ez < ke; ez += 2) {
      layer(ez, F0, F1, U0, U1);
      if (ez + 1 < ke) layer(ez + 1, F1, F0, U1, U0);
    }
    // the last owned node layer; the barrier also ends every read of this
    // tile's node layers before the next tile stages its own
    __syncthreads();
    finish(ke - 1, mine_cur);
  }
  return red;
}

// Asynchronous 4-byte copy global -> shared (zero-filled when !valid: no
// bytes are read) and its group operations.
__device__ __forceinline__ void col_cp4(void* sdst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gsrc),
               "r"(valid ? 4 : 0)
               : "memory");
}
// the 3 consecutive floats at gsrc into 3 shared rows NV floats apart, one
// address register each side, immediate offsets
__device__ __forceinline__ void col_cp4x3(float* sdst, const float* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  const int n = valid ? 4 : 0;
  asm volatile(
      "cp.async.ca.shared.global [%0], [%1], 4, %2;\n"
      "cp.async.ca.shared.global [%0+1188], [%1+4], 4, %2;\n"
      "cp.async.ca.shared.global [%0+2376], [%1+8], 4, %2;\n" ::"r"(d),
      "l"(gsrc), "r"(n)
      : "memory");
}
static_assert(ColShape::NV * 4 == 1188, "row stride of col_cp4x3");
__device__ __forceinline__ void col_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void col_cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Node layers prefetched ahead of the one being staged by the asynchronous
// body; its ring holds kColPrefetch + 1 layers.
constexpr int kColPrefetch = 2;
constexpr int kColRing = kColPrefetch + 1;

// Shared memory of the asynchronous body beyond ColShape::smem_bytes: per
// ring slot, kSrc x 3 source values and the mask word of each staged node,
// and the modulus of each column's element.
template <int KSRC>
constexpr size_t col_ring_bytes() {
  return sizeof(float) * kColRing * ((3 * KSRC + 1) * ColShape::NV + MFTO_BLOCK);
}
// Node layers (three buffers of ColShape::LS floats) and corner sums (two) of
// the asynchronous body.
// (three node buffers, padded to an even float count: the corner sums are
// read and written as 8-byte pairs)
constexpr int kColNodeFloats = 3 * ColShape::LS;
constexpr size_t kColAsyncBase = sizeof(float) * (kColNodeFloats + 2 * 12 * MFTO_BLOCK);

// The column body with its node layers staged by asynchronous copies
// kColPrefetch layers ahead into a ring in shared memory (each thread copies
// and later reads only its own entries, so the ring needs no barrier: the
// copies' wait_group makes them visible to the thread).  Per node the ring
// holds the loader's source values, the 32-bit word of the mask array that
// contains the node's mask byte (the mask array must be readable up to the
// next multiple of 4 bytes) and, per column, the modulus of the element below
// the node layer.  Out-of-grid entries are zero-filled.  Schedule, barrier
// use and arithmetic are those of kv_column_body_regs, except that the node
// layers have three buffers: node layer k stays staged until iteration k + 1,
// so the owner reads its node's staged value back for the epilogue instead of
// carrying it in registers (stage(k + 2) rewrites the buffer, but the owner's
// own slot is written by no other thread, and the face transforms read only
// layers k + 1 and k + 2 by then).
template <typename Load, typename Epi, typename Pre>
__device__ __forceinline__ DFloat kv_column_body_async(const float* __restrict__ E,
                                                       const uint8_t* __restrict__ fixed,
                                                       const ModeCoef<float>& K, const Grid& g,
                                                       const ColTiling& tl, Load ld,
                                                       const Epi& epi, float* smem,
                                                       const Pre& pre, bool* skipped) {
  using S = ColShape;
  constexpr int NS = 3 * Load::kSrc + 1;        // ring rows per node: sources, mask word
  float* nodes = smem;                          // [3][LS], slot of node layer k: (k + 3) % 3
  float* sums = smem + kColNodeFloats;          // [2][12][256] corner sums, slot k & 1
  float* ring = sums + 2 * 12 * MFTO_BLOCK;     // [kColRing][NS][NV]
  float* ering = ring + kColRing * NS * S::NV;  // [kColRing][256]
  const int tid = threadIdx.x;
  const int ex = tid % S::CX, ey = tid / S::CX;
  const bool has_extra = tid < S::NEXTRA;
  const int xx = tid < S::CX ? tid : S::CX;
  const int xy = tid < S::CX ? S::CY : tid - S::CX;
  const int own_slot = ey * S::NX + ex, extra_slot = xy * S::NX + xx;
  const bool owner = ex >= 1 && ey >= 1;
  const uint32_t* fixed_words = reinterpret_cast<const uint32_t*>(fixed);
  DFloat red{0.f, 0.f};
  *skipped = false;
  const int ntiles = tl.count();
  const int nxy = g.nx * g.ny, nexy = g.nelx * g.nely;
  // this thread's place in tile t: its column's node and element and the
  // extra node, as in-plane indices (layer 0) and whether they exist
  struct Ctx {
    int kb, ke, gi, gj;
    int own_base, extra_base, elem_base;
    bool own_in, extra_in, elem_in;
  };
  auto ctx_of = [&](int t) {
    const int bx = t % tl.tx, by = (t / tl.tx) % tl.ty, bz = t / (tl.tx * tl.ty);
    const int x0 = bx * S::OX - 1, y0 = by * S::OY - 1;   // node / element origin of column 0
    Ctx c;
    c.kb = bz * tl.nzc;
    c.ke = min(c.kb + tl.nzc, g.nz);                      // owned node layers [kb, ke)
    c.gi = x0 + ex;                                       // this column's element (and node)
    c.gj = y0 + ey;
    const int hi = x0 + xx, hj = y0 + xy;                 // the extra node
    c.own_in = c.gi >= 0 && c.gj >= 0 && c.gi < g.nx && c.gj < g.ny;
    c.extra_in = hi >= 0 && hj >= 0 && hi < g.nx && hj < g.ny;
    c.elem_in = c.gi >= 0 && c.gj >= 0 && c.gi < g.nelx && c.gj < g.nely;
    c.own_base = c.gi + g.nx * c.gj;
    c.extra_base = hi + g.nx * hj;
    c.elem_base = c.gi + g.nelx * c.gj;
    return c;
  };
  // node layer L (>= -1) sits in ring slot (L + 1) mod kColRing; the slots
  // are carried as rotating counters
  auto next_slot = [](int sl) { return sl == kColRing - 1 ? 0 : sl + 1; };
  // tile t has no fixed node: its mask words are neither copied nor read
  auto clean_of = [&](int t) {
    const int bxy = t % (tl.tx * tl.ty);
    return tl.fixed_tiles != nullptr && tl.fixed_tiles[bxy] == 0;
  };
  // copies of node layer L (and the modulus of element layer L - 1) into
  // ring slot sl; layers past ke copy nothing but still commit a group
  auto issue = [&](const Ctx& c, int L, int sl, auto clean_tag) {
    constexpr bool CLEAN = decltype(clean_tag)::value;
    const bool lay = L >= 0 && L <= c.ke && L < g.nz;
    float* R = ring + sl * NS * S::NV;
    {
      const bool in = lay && c.own_in;
      const int node = in ? c.own_base + nxy * L : 0;
#pragma unroll
      for (int sidx = 0; sidx < Load::kSrc; ++sidx)
        col_cp4x3(R + 3 * sidx * S::NV + own_slot, ld.src(sidx) + 3 * node, in);
      if (!CLEAN) col_cp4(R + 3 * Load::kSrc * S::NV + own_slot, fixed_words + (node >> 2), in);
    }
    if (has_extra) {
      const bool in = lay && c.extra_in;
      const int node = in ? c.extra_base + nxy * L : 0;
#pragma unroll
      for (int sidx = 0; sidx < Load::kSrc; ++sidx)
        col_cp4x3(R + 3 * sidx * S::NV + extra_slot, ld.src(sidx) + 3 * node, in);
      if (!CLEAN)
        col_cp4(R + 3 * Load::kSrc * S::NV + extra_slot, fixed_words + (node >> 2), in);
    }
    {
      const int el = L - 1;
      const bool in = c.elem_in && el >= c.kb - 1 && el >= 0 && el < g.nelz && L <= c.ke;
      const int e = in ? c.elem_base + nexy * el : 0;
      col_cp4(ering + sl * MFTO_BLOCK + tid, E + e, in);
    }
    col_cp_commit();
  };
  // a staged node from ring slot rs: masked loaded values and its mask
  // (q: its place in the staged layer, base: its in-plane node index)
  auto take = [&](int L, int rs, int q, int base, auto clean_tag) {
    constexpr bool CLEAN = decltype(clean_tag)::value;
    const float* R = ring + rs * NS * S::NV;
    const int sl = q;
    ColNode n;
    n.fm = 0;
    if (!CLEAN) {
      const uint32_t w = __float_as_uint(R[3 * Load::kSrc * S::NV + sl]);
      const int node = base + nxy * L;   // only its low 2 bits are used
      n.fm = (uint8_t)(w >> (8 * (node & 3)));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float r[Load::kSrc];
#pragma unroll
      for (int sidx = 0; sidx < Load::kSrc; ++sidx) r[sidx] = R[(3 * sidx + k) * S::NV + sl];
      n.v[k] = (!CLEAN && ((n.fm >> k) & 1)) ? 0.f : ld.combine(r);
    }
    return n;
  };
  // The prologue's copies of a tile always include the mask words: waiting
  // for the tile's clean flag (a global load) before the first copy would
  // put that load's latency in front of every copy; a clean tile just does
  // not read them.
  auto issue_prologue = [&](const Ctx& c) {
    int sl = c.kb % kColRing;   // slot of node layer kb - 1
#pragma unroll
    for (int j = 0; j <= kColPrefetch; ++j) {
      issue(c, c.kb - 1 + j, sl, std::false_type{});
      sl = next_slot(sl);
    }
  };
  // the pre-step's loads, the first tile's prologue copies, then the rest of
  // the pre-step while the copies are in flight
  const typename Pre::State pst = pre.issue();
  int t = blockIdx.x;
  if (t < ntiles) issue_prologue(ctx_of(t));
  if (!pre.run(ld, pst)) {
    col_cp_wait<0>();
    *skipped = true;
    return red;
  }
  // one tile; CLEAN (no fixed node in the tile) compiles the mask work out
  auto run_tile = [&](const Ctx& c, auto clean_tag) {
    constexpr bool CLEAN = decltype(clean_tag)::value;
    const int kb = c.kb, ke = c.ke;
    const bool own_node = owner && c.own_in;
    auto stage = [&](int L, int rs) {
      float* Lb = nodes + ((L + 3) % 3) * S::LS;
      const ColNode own = take(L, rs, own_slot, c.own_base, clean_tag);
      col_put_node(Lb, own_slot, own.v);
      if (has_extra) {
        const ColNode extra = take(L, rs, extra_slot, c.extra_base, clean_tag);
        col_put_node(Lb, extra_slot, extra.v);
      }
      return own;
    };
    // ring slots: rs of the node layer staged next, rp of the one staged
    // before it (free again: its copies landed and were read)
    int rp = c.kb % kColRing;   // node layer kb - 1
    col_cp_wait<kColPrefetch>();
    ColNode mine = stage(kb - 1, rp);
    int rs = next_slot(rp);
    __syncthreads();
    ColFace F0, F1, U0, U1;
    face_forward(nodes + ((kb + 2) % 3) * S::LS, own_slot, F0);
    face_zero(U0);
    // masks of this column's node in node layers ez - 1, ez and ez + 1
    uint8_t fm_cur = mine.fm, fm_prev = mine.fm, fm_next = mine.fm;
    // owner's sum of node layer k from the corner sums in slot k & 1:
    // columns (ex-1, ey-1), (ex, ey-1), (ex-1, ey), (ex, ey) contribute their
    // corners 3, 2, 1, 0
    auto finish = [&](int k, uint8_t fm) {
      if (own_node) {
        float acc[3];
        node_sum(sums + (k & 1) * 12 * MFTO_BLOCK, tid, acc);
        const float* Lk = nodes + ((k + 3) % 3) * S::LS;
        const float2 pxy = reinterpret_cast<const float2*>(Lk)[own_slot];
        const float pn[3] = {pxy.x, pxy.y, Lk[2 * S::NV + own_slot]};
        epi(c.own_base + nxy * k, acc, pn, CLEAN ? (uint8_t)0 : fm, red);
      }
    };
    auto layer = [&](int ez, const ColFace& Flo, ColFace& Fup, const ColFace& upp, ColFace& up) {
      // node layer ez + 1 has landed: stage it, then request layer
      // ez + 1 + kColPrefetch into the ring slot layer ez used
      col_cp_wait<kColPrefetch - 1>();
      fm_prev = fm_cur;
      fm_cur = fm_next;
      fm_next = stage(ez + 1, rs).fm;
      const float Ee = ering[rs * MFTO_BLOCK + tid];
      // layer ez + 1 + kColPrefetch goes into the slot of layer ez
      issue(c, ez + 1 + kColPrefetch, rp, clean_tag);
      rp = rs;
      rs = next_slot(rs);
      __syncthreads();
      // node layer ez - 1 (its corner sums were written in iteration ez - 1)
      if (ez - 1 >= kb) finish(ez - 1, fm_prev);
      ColFace lo;
      face_forward(nodes + ((ez + 4) % 3) * S::LS, own_slot, Fup);
      col_element(Flo, Fup, Ee, K, lo, up);
      if (ez >= kb) {
        // node layer ez: upper face of element ez - 1 plus lower face of ez
        ColFace Ms, Sc;
        face_add(upp, lo, Ms);
        face_inverse(Ms, Sc);
        face_store(Sc, sums + (ez & 1) * 12 * MFTO_BLOCK, tid);
      }
    };
    for (int ez = kb - 1; ez < ke; ez += 2) {
      layer(ez, F0, F1, U0, U1);
      if (ez + 1 < ke) layer(ez + 1, F1, F0, U1, U0);
    }
    // the last owned node layer; the barrier also ends every read of this
    // tile's node layers before the next tile stages its own
    __syncthreads();
    finish(ke - 1, fm_cur);
  };
  for (; t < ntiles; t += gridDim.x) {
    const Ctx c = ctx_of(t);
    if (t != (int)blockIdx.x) issue_prologue(c);
    const bool clean = clean_of(t);
    if (clean)
      run_tile(c, std::true_type{});
    else
      run_tile(c, std::false_type{});
  }
  col_cp_wait<0>();   // the trailing (empty or unused) groups
  return red;
}

template <typename Load, typename Epi, typename Pre>
__device__ __forceinline__ DFloat kv_column_body(const float* __restrict__ E,
                                                 const uint8_t* __restrict__ fixed,
                                                 const ModeCoef<float>& K, const Grid& g,
                                                 const ColTiling& tl, const Load& ld,
                                                 const Epi& epi, float* smem, const Pre& pre,
                                                 bool* skipped) {
  if constexpr (Load::kAsync)
    return kv_column_body_async(E, fixed, K, g, tl, ld, epi, smem, pre, skipped);
  else
    return kv_column_body_regs(E, fixed, K, g, tl, ld, epi, smem, pre, skipped);
}

template <typename Load, typename Epi>
__device__ __forceinline__ DFloat kv_column_body(const float* __restrict__ E,
                                                 const uint8_t* __restrict__ fixed,
                                                 const ModeCoef<float>& K, const Grid& g,
                                                 const ColTiling& tl, const Load& ld,
                                                 const Epi& epi, float* smem) {
  bool skipped;
  return kv_column_body(E, fixed, K, g, tl, ld, epi, smem, ColNoPre{}, &skipped);
}

// Dynamic shared memory of every column-kernel launch whose loader is staged
// asynchronously (at most two source arrays).
constexpr size_t kColSmem = kColAsyncBase + col_ring_bytes<2>();

// Dynamic shared memory of a column-kernel launch with loader Load.
template <typename Load>
constexpr size_t col_smem_bytes() {
  if constexpr (Load::kAsync)
    return kColAsyncBase + col_ring_bytes<Load::kSrc>();
  else
    return ColShape::smem_bytes;
}

// Warp sum of double-float shares; lane 0 returns the warp's total in FP64,
// the other lanes 0 (the convention of DotAcc<float>::finish).
__device__ __forceinline__ double col_warp_finish(DFloat v) {
  DotAcc<float> acc;
  acc.s = v;
  return acc.finish();
}

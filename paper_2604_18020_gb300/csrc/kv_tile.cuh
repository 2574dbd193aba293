// Tiled, node-owned, atomic-free K.v with the element operator applied in the
// per-axis (sum, difference) mode basis (see modes.cuh).
//
// A CTA owns a block of TX x TY x nzc nodes and streams along z.  For every
// element layer ek it needs (elements i in [i0-1, i0+TX), j in [j0-1, j0+TY)),
// it:
//   1. stages node layer ek+1 of v (TX+2 x TY+2 nodes, fixed DOFs zeroed)
//      into a three-layer shared-memory ring (layers ek-1, ek, ek+1: the node
//      phase of layer ek-1 may still read its slot while ek+1 is staged);
//   2. computes each element's 24 outputs: forward butterflies (v -> modes),
//      the 45-term mode operator scaled by E_e, inverse butterflies;
//      lower-face outputs go to buffer L, upper-face outputs to U[cur];
//   3. lets each owned node of layer ek sum its 8 contributions (4 upper faces
//      of element layer ek-1 from U[prev], 4 lower faces of layer ek from L)
//      in a fixed order and stores the result.
// Each output is written once, by one thread, in a fixed order: the result
// is bit-reproducible.  Elements on the x/y halo and one z layer per chunk
// are computed by two CTAs (the price of owning nodes without atomics).
#pragma once
#include "common.cuh"

template <typename T>
struct TileLoadPlain {
  const T* v;
  __device__ __forceinline__ T operator()(int idx) const { return v[idx]; }
};

template <typename T>
struct TileLoadDirection {
  const T* z;
  const T* p;
  T beta;
  __device__ __forceinline__ T operator()(int idx) const { return z[idx] + beta * p[idx]; }
};

// per-axis butterfly on a 24-value element vector, component-major x[c][m]
template <int BIT, typename T>
__device__ __forceinline__ void butterfly_fwd(T (&x)[3][8]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < 8; ++m)
      if (!(m & BIT)) {
        const T a = x[c][m], b = x[c][m | BIT];
        x[c][m] = a + b;        // sum
        x[c][m | BIT] = b - a;  // difference
      }
}

template <int BIT, typename T>
__device__ __forceinline__ void butterfly_inv(T (&x)[3][8]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < 8; ++m)
      if (!(m & BIT)) {
        const T s = x[c][m], d = x[c][m | BIT];
        x[c][m] = s - d;        // corner 0 (factor 1/2 folded into the coefficients)
        x[c][m | BIT] = s + d;  // corner 1
      }
}

// y = E KE x for one element, in place (x[c][corner] -> y[c][corner]).
template <typename T>
__device__ __forceinline__ void element_apply(T (&x)[3][8], T E, const ModeCoef<T>& K) {
  butterfly_fwd<1>(x);
  butterfly_fwd<2>(x);
  butterfly_fwd<4>(x);
  T y[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < 8; ++m) y[c][m] = (E * K.diag[c][m]) * x[c][m];
  const T l0 = E * K.lamM[0], l1 = E * K.lamM[1];
  const T u0 = E * K.muM[0], u1 = E * K.muM[1];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (i == j) continue;
      const int t = 3 - i - j;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int tb = mt << t;
        const T lc = mt ? l1 : l0, uc = mt ? u1 : u0;
        y[i][(1 << i) | tb] += lc * x[j][(1 << j) | tb];
        y[i][(1 << j) | tb] += uc * x[j][(1 << i) | tb];
      }
    }
  butterfly_inv<4>(y);
  butterfly_inv<2>(y);
  butterfly_inv<1>(y);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < 8; ++m) x[c][m] = y[c][m];
}

// Epilogues: what the owner of a node does with its 3 sums.
template <typename T>
struct TileStore {           // plain K.v: y = sum, y_fixed = v
  const T* v;
  T* y;
  __device__ __forceinline__ void operator()(int node, const T (&acc)[3], const T (&pn)[3],
                                             uint8_t fm, DotAcc<T>& red) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) y[3 * node + c] = ((fm >> c) & 1) ? v[3 * node + c] : acc[c];
  }
};

template <typename T>
struct TilePcg {             // CG: p_new stored, q = K p_new, p_new.q accumulated
  T* p_new;
  T* q;
  __device__ __forceinline__ void operator()(int node, const T (&acc)[3], const T (&pn)[3],
                                             uint8_t fm, DotAcc<T>& red) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T qc = ((fm >> c) & 1) ? pn[c] : acc[c];
      p_new[3 * node + c] = pn[c];
      q[3 * node + c] = qc;
      red.add_prod(pn[c], qc);
    }
  }
};

template <int TX, int TY>
struct TileShape {
  static constexpr int VX = TX + 2, VY = TY + 2;      // staged node region
  static constexpr int EX = TX + 1, EY = TY + 1;      // elements per layer
  static constexpr int NV = VX * VY, NE = EX * EY, NN = TX * TY;
  template <typename T>
  static constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)(3 * 3 * NV + 12 * NE + 2 * 12 * NE);
  }
};

// Block (bx, by, bz) owns nodes [bx*TX, +TX) x [by*TY, +TY) x [bz*nzc, +nzc).
// Returns this thread's share of the epilogue reduction (0 for plain K.v),
// to be summed over the block.
template <typename T, int TX, int TY, typename Load, typename Epi>
__device__ __forceinline__ double kv_tile_body(const T* __restrict__ E,
                                               const uint8_t* __restrict__ fixed,
                                               const ModeCoef<T>& K, const Grid& g, int nzc,
                                               const Load& ld, const Epi& epi, T* smem) {
  using S = TileShape<TX, TY>;
  T* vs = smem;                        // [3][3][NV], slot of node layer nk: (nk + 3) % 3
  T* Lb = vs + 3 * 3 * S::NV;          // [12][NE]
  T* Ub = Lb + 12 * S::NE;             // [2][12][NE]
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * nzc;
  const int k_end = min(k0 + nzc, g.nz);   // owned node layers [k0, k_end)
  DotAcc<T> red;

  auto load_layer = [&](int nk) {
    T* dst = vs + ((nk + 3) % 3) * 3 * S::NV;
    for (int idx = tid; idx < S::NV; idx += blockDim.x) {
      const int gi = i0 - 1 + idx % S::VX, gj = j0 - 1 + idx / S::VX;
      T a = 0, b = 0, c = 0;
      if (gi >= 0 && gj >= 0 && gi < g.nx && gj < g.ny && nk >= 0 && nk < g.nz) {
        const int node = gi + g.nx * (gj + g.ny * nk);
        const uint8_t fm = fixed[node];
        a = (fm & 1) ? T(0) : ld(3 * node + 0);
        b = (fm & 2) ? T(0) : ld(3 * node + 1);
        c = (fm & 4) ? T(0) : ld(3 * node + 2);
      }
      dst[idx] = a;
      dst[S::NV + idx] = b;
      dst[2 * S::NV + idx] = c;
    }
  };

  load_layer(k0 - 1);
  int cur = 0;
  for (int ek = k0 - 1; ek < k_end; ++ek) {
    load_layer(ek + 1);
    __syncthreads();
    // ---- element phase: element layer ek
    T* Uc = Ub + cur * 12 * S::NE;
    for (int t = tid; t < S::NE; t += blockDim.x) {
      const int ex = t % S::EX, ey = t / S::EX;
      const int ei = i0 - 1 + ex, ej = j0 - 1 + ey;
      T x[3][8];
      const bool valid = ei >= 0 && ej >= 0 && ek >= 0 && ei < g.nelx && ej < g.nely && ek < g.nelz;
      if (valid) {
#pragma unroll
        for (int l = 0; l < 8; ++l) {
          const T* src = vs + ((ek + (l >> 2) + 3) % 3) * 3 * S::NV + (ex + (l & 1)) +
                         S::VX * (ey + ((l >> 1) & 1));
          x[0][l] = src[0];
          x[1][l] = src[S::NV];
          x[2][l] = src[2 * S::NV];
        }
        element_apply<T>(x, E[ei + g.nelx * (ej + g.nely * ek)], K);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int l = 0; l < 8; ++l) x[c][l] = 0;
      }
#pragma unroll
      for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Lb[(3 * l + c) * S::NE + t] = x[c][l];
          Uc[(3 * l + c) * S::NE + t] = x[c][l + 4];
        }
    }
    __syncthreads();
    // ---- node phase: node layer ek (owned when k0 <= ek < k_end)
    if (ek >= k0) {
      const T* Up = Ub + (cur ^ 1) * 12 * S::NE;
      const T* vcur = vs + ((ek + 3) % 3) * 3 * S::NV;
      for (int t = tid; t < S::NN; t += blockDim.x) {
        const int ix = t % TX, iy = t / TX;
        const int gi = i0 + ix, gj = j0 + iy;
        if (gi >= g.nx || gj >= g.ny) continue;
        T acc[3] = {0, 0, 0};
        // element (ex, ey) = (ix + ea, iy + eb); this node is its corner (1-ea, 1-eb)
#pragma unroll
        for (int half = 0; half < 2; ++half) {      // upper faces of layer ek-1, then lower of ek
          const T* B = half ? Lb : Up;
#pragma unroll
          for (int eb = 0; eb < 2; ++eb)
#pragma unroll
            for (int ea = 0; ea < 2; ++ea) {
              const int e = (ix + ea) + S::EX * (iy + eb);
              const int corner = (1 - ea) + 2 * (1 - eb);
#pragma unroll
              for (int c = 0; c < 3; ++c) acc[c] += B[(3 * corner + c) * S::NE + e];
            }
        }
        const int vi = (ix + 1) + S::VX * (iy + 1);
        const T pn[3] = {vcur[vi], vcur[S::NV + vi], vcur[2 * S::NV + vi]};
        const int node = gi + g.nx * (gj + g.ny * ek);
        epi(node, acc, pn, fixed[node], red);
      }
    }
    cur ^= 1;
  }
  return red.finish();
}

// Block variant (FP32 forms): one element per thread, no layer loop.  A CTA
// of 256 threads computes the 8 x 8 x 4 elements whose corners span a
// 9 x 9 x 5 node block and owns the 7 x 7 x 3 interior nodes (all 8 of their
// elements lie in the block).  Per block: stage the 405 nodes (masked values
// and masks), compute one element per thread into a [24][256] output buffer,
// and let each owned node sum its 8 contributions in a fixed order.  The
// halo costs 256/147 = 1.74 element evaluations per node, cheap in FP32;
// in exchange every thread works and there are two barriers per block.
// Blocks are visited by a grid-stride loop (z fastest after x, y), so the
// grid -- and the number of reduction partials -- stays small.
struct BlockShape {
  static constexpr int BX = 8, BY = 8, BZ = 4;          // elements
  static constexpr int VX = 9, VY = 9, VZ = 5;          // nodes
  static constexpr int NV = VX * VY * VZ;               // 405
  static constexpr int OX = 7, OY = 7, OZ = 3;          // owned nodes
  static constexpr int NO = OX * OY * OZ;               // 147
  template <typename T>
  static constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)(3 * NV + 24 * BX * BY * BZ) + NV;
  }
};

template <typename T, typename Load, typename Epi>
__device__ __forceinline__ double kv_block_body(const T* __restrict__ E,
                                                const uint8_t* __restrict__ fixed,
                                                const ModeCoef<T>& K, const Grid& g,
                                                const Load& ld, const Epi& epi, T* smem) {
  using B = BlockShape;
  static_assert(B::BX * B::BY * B::BZ == MFTO_BLOCK, "one element per thread");
  T* vs = smem;                                                  // [3][NV]
  T* out = vs + 3 * B::NV;                                       // [24][256]
  uint8_t* ms = reinterpret_cast<uint8_t*>(out + 24 * MFTO_BLOCK);  // [NV]
  const int tid = threadIdx.x;
  const int tx = (g.nx + B::OX - 1) / B::OX, ty = (g.ny + B::OY - 1) / B::OY;
  const int tz = (g.nz + B::OZ - 1) / B::OZ;
  const int n_blocks = tx * ty * tz;
  const int ex = tid & 7, ey = (tid >> 3) & 7, ez = tid >> 6;
  DotAcc<T> red;
  for (int b = blockIdx.x; b < n_blocks; b += gridDim.x) {
    const int bx = b % tx, by = (b / tx) % ty, bz = b / (tx * ty);
    const int ox = bx * B::OX, oy = by * B::OY, oz = bz * B::OZ;   // first owned node
    // ---- stage the node block (masked values, masks) and this thread's E
    for (int idx = tid; idx < B::NV; idx += MFTO_BLOCK) {
      const int lx = idx % B::VX, ly = (idx / B::VX) % B::VY, lz = idx / (B::VX * B::VY);
      const int gi = ox - 1 + lx, gj = oy - 1 + ly, gk = oz - 1 + lz;
      T a = 0, bb = 0, c = 0;
      uint8_t fm = 0;
      if (gi >= 0 && gj >= 0 && gk >= 0 && gi < g.nx && gj < g.ny && gk < g.nz) {
        const int node = gi + g.nx * (gj + g.ny * gk);
        fm = fixed[node];
        a = ld(3 * node + 0);
        bb = ld(3 * node + 1);
        c = ld(3 * node + 2);
        a = (fm & 1) ? T(0) : a;
        bb = (fm & 2) ? T(0) : bb;
        c = (fm & 4) ? T(0) : c;
      }
      vs[idx] = a;
      vs[B::NV + idx] = bb;
      vs[2 * B::NV + idx] = c;
      ms[idx] = fm;
    }
    const int ei = ox - 1 + ex, ej = oy - 1 + ey, ek = oz - 1 + ez;
    T Ee = 0;
    if (ei >= 0 && ej >= 0 && ek >= 0 && ei < g.nelx && ej < g.nely && ek < g.nelz)
      Ee = E[ei + g.nelx * (ej + g.nely * ek)];
    __syncthreads();
    // ---- element phase (out-of-domain elements have E = 0: zero outputs)
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
    // ---- node phase: owned node (ox+ix, oy+iy, oz+iz)
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
        epi(gi + g.nx * (gj + g.ny * gk), acc, pn, ms[vi], red);
      }
    }
    __syncthreads();   // vs, ms and out are rewritten for the next block
  }
  return red.finish();
}

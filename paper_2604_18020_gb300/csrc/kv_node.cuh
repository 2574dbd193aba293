// Node-centric gather of the matrix-free K.v (Eq. matfree):
//   y_n = sum_{e owns n} E_e sum_{m in e} KE[l(n,e), l(m,e)] v_m
// for one node n, over the up to 8 elements around it, in a fixed order
// (element corner ce = 0..7, then local node lm = 0..7).  Inputs on fixed
// DOFs are read as zero (the masked operator).  The caller substitutes the
// fixed outputs.  ke points to the 576-entry KE in shared memory; all lanes
// of a warp index it with the same ce, so its loads are broadcasts.
#pragma once
#include "common.cuh"

template <typename T>
struct LoadPlain {
  const T* v;
  __device__ __forceinline__ T operator()(int idx) const { return v[idx]; }
};

// p_new = z + beta * p_old, evaluated on the fly (the CG direction update
// folded into the K.v gather).
template <typename T>
struct LoadDirection {
  const T* z;
  const T* p;
  T beta;
  __device__ __forceinline__ T operator()(int idx) const { return z[idx] + beta * p[idx]; }
};

template <typename T, typename Load>
__device__ __forceinline__ void node_kv(int node, const T* __restrict__ E,
                                        const uint8_t* __restrict__ fixed,
                                        const T* ke, const Grid& g, const Load& ld,
                                        T& acc0, T& acc1, T& acc2) {
  const int i = node % g.nx;
  const int j = (node / g.nx) % g.ny;
  const int k = node / (g.nx * g.ny);
  acc0 = 0; acc1 = 0; acc2 = 0;
#pragma unroll 1
  for (int ce = 0; ce < 8; ++ce) {
    // element (i-1+ea, j-1+eb, k-1+ec); this node is its corner (1-ea, 1-eb, 1-ec)
    const int ea = ce & 1, eb = (ce >> 1) & 1, ec = ce >> 2;
    const int ei = i - 1 + ea, ej = j - 1 + eb, ek = k - 1 + ec;
    if (ei < 0 || ej < 0 || ek < 0 || ei >= g.nelx || ej >= g.nely || ek >= g.nelz) continue;
    const int ln = (1 - ea) + 2 * (1 - eb) + 4 * (1 - ec);
    const T* kr = ke + (3 * ln) * 24;
    T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int lm = 0; lm < 8; ++lm) {
      const int m = (ei + (lm & 1)) + g.nx * ((ej + ((lm >> 1) & 1)) + g.ny * (ek + (lm >> 2)));
      const uint8_t mm = fixed[m];
      const T v0 = (mm & 1) ? T(0) : ld(3 * m + 0);
      const T v1 = (mm & 2) ? T(0) : ld(3 * m + 1);
      const T v2 = (mm & 4) ? T(0) : ld(3 * m + 2);
      s0 += kr[0 * 24 + 3 * lm + 0] * v0 + kr[0 * 24 + 3 * lm + 1] * v1 + kr[0 * 24 + 3 * lm + 2] * v2;
      s1 += kr[1 * 24 + 3 * lm + 0] * v0 + kr[1 * 24 + 3 * lm + 1] * v1 + kr[1 * 24 + 3 * lm + 2] * v2;
      s2 += kr[2 * 24 + 3 * lm + 0] * v0 + kr[2 * 24 + 3 * lm + 1] * v1 + kr[2 * 24 + 3 * lm + 2] * v2;
    }
    const T Ee = E[ei + g.nelx * (ej + g.nely * ek)];
    acc0 += Ee * s0;
    acc1 += Ee * s1;
    acc2 += Ee * s2;
  }
}

// The FP32 CG vector update u += alpha p; r -= alpha q; z = r / d with the
// shares of r.z and r.r, over groups of 4 DOFs (16-byte accesses of the flat
// DOF arrays).  For each group the 4 products of r.z and of r.r are summed in
// FP32 (relative error <= 4 u of the group's absolute sum) and the group sum
// enters the caller's double-float accumulators.  FROM_L2: p and q were
// written by other CTAs of the same launch and are read with ld.global.cg.
#pragma once
#include "common.cuh"

__device__ __forceinline__ float dot4(const float4& a, const float4& b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

template <bool FROM_L2>
__device__ __forceinline__ void cg_update_f32(float* u, const float* p, const float* q, float* r,
                                              float* z, const float* __restrict__ dinv, int n,
                                              float alpha, int first, int stride,
                                              DotAcc<float>& d0, DotAcc<float>& d1) {
  const int n4 = n >> 2;
  float4* u4 = reinterpret_cast<float4*>(u);
  float4* r4 = reinterpret_cast<float4*>(r);
  float4* z4 = reinterpret_cast<float4*>(z);
  const float4* p4 = reinterpret_cast<const float4*>(p);
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const float4* d4 = reinterpret_cast<const float4*>(dinv);
  for (int i = first; i < n4; i += stride) {
    float4 uu = u4[i];
    const float4 pp = FROM_L2 ? __ldcg(p4 + i) : p4[i];
    const float4 qq = FROM_L2 ? __ldcg(q4 + i) : q4[i];
    const float4 rr = r4[i], dd = d4[i];
    uu.x += alpha * pp.x; uu.y += alpha * pp.y; uu.z += alpha * pp.z; uu.w += alpha * pp.w;
    float4 rn, zn;
    rn.x = rr.x - alpha * qq.x; rn.y = rr.y - alpha * qq.y;
    rn.z = rr.z - alpha * qq.z; rn.w = rr.w - alpha * qq.w;
    zn.x = rn.x * dd.x; zn.y = rn.y * dd.y; zn.z = rn.z * dd.z; zn.w = rn.w * dd.w;
    u4[i] = uu;
    r4[i] = rn;
    z4[i] = zn;
    d0.add(dot4(rn, zn));
    d1.add(dot4(rn, rn));
  }
  // the n mod 4 trailing DOFs, by the threads whose first index is below n mod 4
  if (first < (n & 3)) {
    const int i = 4 * n4 + first;
    const float pi = FROM_L2 ? __ldcg(p + i) : p[i];
    const float qi = FROM_L2 ? __ldcg(q + i) : q[i];
    u[i] += alpha * pi;
    const float ri = r[i] - alpha * qi;
    const float zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    d0.add(ri * zi);
    d1.add(ri * ri);
  }
}

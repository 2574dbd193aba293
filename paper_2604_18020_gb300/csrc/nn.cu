// The learned part: a 4-level 3D-conv U-Net on the node grid (input: node
// density and load, 4 channels; output: a displacement direction, 3
// channels), with hand-written forward, backward and Adam kernels.  Weights
// are stored in BF16 for the forward and backward passes (an FP32 master copy
// takes the Adam updates); activations and all accumulation are FP32; every
// reduction (weight and bias gradients, loss) runs in a fixed order.
//
// Architecture (same as the oracle's): encoder levels l = 0..L-2 each
// relu(conv(relu(conv(.)))) with c 2^l channels, 2x2x2 average pooling
// between levels, a bottleneck of c 2^(L-1) channels, decoder levels with
// nearest upsampling and concatenation of the encoder output, and a 1x1x1
// head.  Tensors are [channels][nz][ny][nx] FP32 on a grid padded to a
// multiple of 2^(L-1).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <random>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace {

constexpr int kNT = 128;      // threads of the voxel kernels
constexpr int kCOB = 8;       // output channels per thread (forward)
constexpr int kCIC = 8;       // input-channel chunk staged in shared memory
constexpr int kLossBlocks = 256;  // blocks of the loss reduction

struct Dims {
  int D, H, W;
  __host__ __device__ int V() const { return D * H * W; }
};

__device__ __forceinline__ int koff_ok(int z, int y, int x, int k, int K, const Dims& d, int* idx) {
  const int r = K / 2;
  const int dz = k / (K * K) - r, dy = (k / K) % K - r, dx = k % K - r;
  const int zz = z + dz, yy = y + dy, xx = x + dx;
  if (zz < 0 || yy < 0 || xx < 0 || zz >= d.D || yy >= d.H || xx >= d.W) return 0;
  *idx = zz * d.H * d.W + yy * d.W + xx;
  return 1;
}

// out[co][v] = b[co] + sum_ci sum_k w[co][ci][k] in[ci][v + d_k]  (optional relu)
template <int K>
__global__ void __launch_bounds__(kNT)
conv_fwd(const float* __restrict__ in, int Cin, const __nv_bfloat16* __restrict__ w,
         const float* __restrict__ b, float* __restrict__ out, int Cout, Dims d, int relu) {
  constexpr int KK = K * K * K;
  __shared__ float ws[kCOB][kCIC][KK];
  const int V = d.V();
  const int v = blockIdx.x * kNT + threadIdx.x;
  const int co0 = blockIdx.y * kCOB;
  const int z = v / (d.H * d.W), y = (v / d.W) % d.H, x = v % d.W;
  float acc[kCOB];
#pragma unroll
  for (int j = 0; j < kCOB; ++j) acc[j] = (co0 + j < Cout) ? b[co0 + j] : 0.f;
  for (int ci0 = 0; ci0 < Cin; ci0 += kCIC) {
    __syncthreads();
    for (int t = threadIdx.x; t < kCOB * kCIC * KK; t += kNT) {
      const int j = t / (kCIC * KK), c = (t / KK) % kCIC, k = t % KK;
      ws[j][c][k] = (co0 + j < Cout && ci0 + c < Cin)
                        ? __bfloat162float(w[((size_t)(co0 + j) * Cin + ci0 + c) * KK + k]) : 0.f;
    }
    __syncthreads();
    if (v < V) {
      for (int c = 0; c < kCIC && ci0 + c < Cin; ++c) {
        const float* src = in + (size_t)(ci0 + c) * V;
#pragma unroll
        for (int k = 0; k < KK; ++k) {
          int idx;
          if (!koff_ok(z, y, x, k, K, d, &idx)) continue;
          const float xv = src[idx];
#pragma unroll
          for (int j = 0; j < kCOB; ++j) acc[j] += ws[j][c][k] * xv;
        }
      }
    }
  }
  if (v < V)
#pragma unroll
    for (int j = 0; j < kCOB; ++j)
      if (co0 + j < Cout) out[(size_t)(co0 + j) * V + v] = relu ? fmaxf(acc[j], 0.f) : acc[j];
}

// din[ci][v] = (sum_co sum_k w[co][ci][k] dout[co][v - d_k]) * (gate[ci][v] > 0 if gate)
template <int K>
__global__ void __launch_bounds__(kNT)
conv_bwd_data(const float* __restrict__ dout, int Cout, const __nv_bfloat16* __restrict__ w,
              float* __restrict__ din, int Cin, Dims d, const float* __restrict__ gate) {
  constexpr int KK = K * K * K;
  __shared__ float ws[kCOB][kCIC][KK];   // [ci block][co chunk][k]
  const int V = d.V();
  const int v = blockIdx.x * kNT + threadIdx.x;
  const int ci0 = blockIdx.y * kCOB;
  const int z = v / (d.H * d.W), y = (v / d.W) % d.H, x = v % d.W;
  float acc[kCOB];
#pragma unroll
  for (int j = 0; j < kCOB; ++j) acc[j] = 0.f;
  for (int co0 = 0; co0 < Cout; co0 += kCIC) {
    __syncthreads();
    for (int t = threadIdx.x; t < kCOB * kCIC * KK; t += kNT) {
      const int j = t / (kCIC * KK), c = (t / KK) % kCIC, k = t % KK;
      ws[j][c][k] = (ci0 + j < Cin && co0 + c < Cout)
                        ? __bfloat162float(w[((size_t)(co0 + c) * Cin + ci0 + j) * KK + k]) : 0.f;
    }
    __syncthreads();
    if (v < V) {
      for (int c = 0; c < kCIC && co0 + c < Cout; ++c) {
        const float* src = dout + (size_t)(co0 + c) * V;
#pragma unroll
        for (int k = 0; k < KK; ++k) {
          int idx;
          if (!koff_ok(z, y, x, KK - 1 - k, K, d, &idx)) continue;   // v - d_k
          const float g = src[idx];
#pragma unroll
          for (int j = 0; j < kCOB; ++j) acc[j] += ws[j][c][k] * g;
        }
      }
    }
  }
  if (v < V)
#pragma unroll
    for (int j = 0; j < kCOB; ++j)
      if (ci0 + j < Cin) {
        const size_t o = (size_t)(ci0 + j) * V + v;
        din[o] = (gate && !(gate[o] > 0.f)) ? 0.f : acc[j];
      }
}

// partial[chunk][co][ci][k] = sum_{v in chunk} dout[co][v] in[ci][v + d_k];
// one block per (co, ci, chunk), fixed-order block reduction
template <int K>
__global__ void __launch_bounds__(kNT)
conv_bwd_weight(const float* __restrict__ in, int Cin, const float* __restrict__ dout, int Cout,
                Dims d, int chunk, float* __restrict__ partial) {
  constexpr int KK = K * K * K;
  __shared__ float red[kNT / 32][KK];
  const int V = d.V();
  const int co = blockIdx.x / Cin, ci = blockIdx.x % Cin;
  const int v0 = blockIdx.y * chunk, v1 = min(V, v0 + chunk);
  float acc[KK];
#pragma unroll
  for (int k = 0; k < KK; ++k) acc[k] = 0.f;
  const float* g = dout + (size_t)co * V;
  const float* src = in + (size_t)ci * V;
  for (int v = v0 + threadIdx.x; v < v1; v += kNT) {
    const float gv = g[v];
    const int z = v / (d.H * d.W), y = (v / d.W) % d.H, x = v % d.W;
#pragma unroll
    for (int k = 0; k < KK; ++k) {
      int idx;
      if (koff_ok(z, y, x, k, K, d, &idx)) acc[k] += gv * src[idx];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < KK; ++k) {
    float s = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < KK; k += kNT) {
    float s = 0.f;
    for (int q = 0; q < kNT / 32; ++q) s += red[q][k];
    partial[(((size_t)blockIdx.y * Cout + co) * Cin + ci) * KK + k] = s;
  }
}

// partial[chunk][co] = sum_{v in chunk} dout[co][v]
__global__ void __launch_bounds__(kNT)
bias_grad(const float* __restrict__ dout, int Cout, int V, int chunk, float* __restrict__ partial) {
  __shared__ float red[kNT / 32];
  const int co = blockIdx.x;
  const int v0 = blockIdx.y * chunk, v1 = min(V, v0 + chunk);
  float s = 0.f;
  for (int v = v0 + threadIdx.x; v < v1; v += kNT) s += dout[(size_t)co * V + v];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int q = 0; q < kNT / 32; ++q) t += red[q];
    partial[(size_t)blockIdx.y * Cout + co] = t;
  }
}

// out[i] = sum over chunks of partial[chunk][i] (chunk order)
__global__ void sum_chunks(const float* __restrict__ partial, int n, int chunks, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += partial[(size_t)c * n + i];
  out[i] = s;
}

__global__ void pool_fwd(const float* __restrict__ in, float* __restrict__ out, int C, Dims dc) {
  // dc: coarse dims
  const int Vc = dc.V();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C * Vc) return;
  const int c = i / Vc, v = i % Vc;
  const int z = v / (dc.H * dc.W), y = (v / dc.W) % dc.H, x = v % dc.W;
  const int Hf = 2 * dc.H, Wf = 2 * dc.W;
  const size_t base = (size_t)c * 8 * Vc;
  float s = 0.f;
  for (int q = 0; q < 8; ++q)
    s += in[base + (size_t)(2 * z + (q >> 2)) * Hf * Wf + (2 * y + ((q >> 1) & 1)) * Wf + 2 * x + (q & 1)];
  out[i] = s * 0.125f;
}

// fine[c][v] (+)= coarse[c][v / 2] * scale
__global__ void spread_up(const float* __restrict__ coarse, float* __restrict__ fine, int C, Dims df,
                          float scale, int accumulate) {
  const int Vf = df.V();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C * Vf) return;
  const int c = i / Vf, v = i % Vf;
  const int z = v / (df.H * df.W), y = (v / df.W) % df.H, x = v % df.W;
  const int Hc = df.H / 2, Wc = df.W / 2;
  const float val = coarse[(size_t)c * (Vf / 8) + (z / 2) * Hc * Wc + (y / 2) * Wc + x / 2] * scale;
  fine[i] = accumulate ? fine[i] + val : val;
}

// coarse[c][v] = sum of the 8 children of v in fine (the adjoint of spread_up)
__global__ void gather_up(const float* __restrict__ fine, float* __restrict__ coarse, int C, Dims dc) {
  const int Vc = dc.V();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C * Vc) return;
  const int c = i / Vc, v = i % Vc;
  const int z = v / (dc.H * dc.W), y = (v / dc.W) % dc.H, x = v % dc.W;
  const int Hf = 2 * dc.H, Wf = 2 * dc.W;
  const size_t base = (size_t)c * 8 * Vc;
  float s = 0.f;
  for (int q = 0; q < 8; ++q)
    s += fine[base + (size_t)(2 * z + (q >> 2)) * Hf * Wf + (2 * y + ((q >> 1) & 1)) * Wf + 2 * x + (q & 1)];
  coarse[i] = s;
}

__global__ void copy_f32(const float* __restrict__ a, float* __restrict__ b, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

__global__ void add_f32(const float* __restrict__ a, float* __restrict__ b, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] += a[i];
}

// Masked MSE, first pass: g = 2 (p - t) m (not yet divided by the count),
// per-block partial sums of (p - t)^2 m^2 (row 0) and of m (row 1).  g may
// alias p (each element is read before it is written by the same thread).
__global__ void __launch_bounds__(256)
mse_grad(const float* p, const float* __restrict__ t, const float* __restrict__ m, float* g,
         size_t n, double* __restrict__ partial) {
  __shared__ double sh[64];
  double acc = 0.0, cnt = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float diff = (p[i] - t[i]) * m[i];
    g[i] = 2.f * diff;
    acc += (double)diff * (double)diff;
    cnt += (double)m[i];
  }
  const double bs = block_sum(acc, sh);
  __syncthreads();
  const double bc = block_sum(cnt, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = bs;
    partial[kLossBlocks + blockIdx.x] = bc;
  }
}

// second pass (one block): loss = sum / count and 1 / count, in block order
__global__ void mse_finish(double* partial) {
  if (threadIdx.x != 0) return;
  double s = 0.0, c = 0.0;
  for (int b = 0; b < kLossBlocks; ++b) {
    s += partial[b];
    c += partial[kLossBlocks + b];
  }
  c = c > 1.0 ? c : 1.0;
  partial[2 * kLossBlocks] = s / c;
  partial[2 * kLossBlocks + 1] = 1.0 / c;
}

// g *= 1 / count
__global__ void mse_scale(float* __restrict__ g, size_t n, const double* __restrict__ partial) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) g[i] *= (float)partial[2 * kLossBlocks + 1];
}

__global__ void adam_step(float* __restrict__ w, __nv_bfloat16* __restrict__ wb,
                          const float* __restrict__ g, float* __restrict__ m, float* __restrict__ vv,
                          size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * vv[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  vv[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}

__global__ void to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ---- 3x3x3 convolution on the tensor cores (implicit GEMM, tcgen05) ------
//
// out[co][v] = b[co] + sum_ci sum_k w[co][ci][k] in[ci][v + d_k] as the GEMM
// D[128 voxels x N] = sum_k sum_ci A_k[voxel][ci] B_k[ci][co], N = a slice of
// NS output channels, accumulated in FP32 in tensor memory.  A CTA computes an
// output tile of 8 (x) x 16 (y) voxels of one z-plane (M = 128) and stages its
// input halo tile, 10 x 18 x 3 voxels, 16 input channels at a time, as BF16 in
// the canonical no-swizzle K-major layout: one 16-byte row per (voxel, 8
// channels).  For tap (dx, dy, dz) the A operand is that staged tile read in
// place: the core-matrix rows of output voxels x = 0..7 of one y-row are the
// staged voxels x + dx of y-row y + dy (consecutive, 16 bytes apart), the
// 8-row groups step one staged y-row (SBO = 160 bytes) and the two 8-channel
// halves of the K = 16 step sit one channel part apart (LBO).  The FP32
// activations are split into BF16 hi + lo (two products against the same
// BF16 weights), so the result carries the activations to about 2^-16 and
// the weights as stored.  Per stage one thread issues 27 taps x 2 parts
// MMAs (M = 128, N = NS, K = 16), commits them to an mbarrier (bounded wait),
// and the CTA stages the next 16 channels after they completed; three CTAs
// per SM overlap one another's staging and MMAs.  The epilogue reads each
// voxel's row of D with tcgen05.ld and writes bias + ReLU in FP32 (bias may
// be NULL; with gate given, outputs whose gate value is not positive are
// zero: the ReLU adjoint of the data gradient, which runs through this
// kernel with the adjoint weights of pack_w3).
constexpr int kCtTX = 8, kCtTY = 16;                  // output tile (M = 128)
constexpr int kCtHX = kCtTX + 2, kCtHY = kCtTY + 2;   // staged halo tile, 3 z-planes
constexpr int kCtPos = kCtHX * kCtHY * 3;             // 540 staged voxels
constexpr int kCtPart = kCtPos * 16;                  // one 8-channel part: 8,640 bytes
constexpr int kCtA = 4 * kCtPart;                     // hi 0-7, hi 8-15, lo 0-7, lo 8-15
constexpr int kCtCin = 16;                            // input channels per stage
constexpr uint32_t kCtSpin = 1u << 20;                // bound of the mbarrier wait
template <int NS>
struct CtShape {
  static constexpr int B = 27 * 2 * (NS / 8) * 128;   // packed weights of one stage
  static constexpr int COLS = NS < 32 ? 32 : NS;      // TMEM columns (allocation >= 32)
  static constexpr int SMEM = kCtA + B + 128 + 128;   // + mbarrier / TMEM slot + alignment
};

// Packed weights of one 3x3x3 layer, slice by slice (NS output channels) and
// stage by stage (16 input channels): [tap 27][kc 2][ng NS/8][r 8][c 8] BF16,
// co = slice NS + 8 ng + r, ci = 16 stage + 8 kc + c, zero outside the layer
// (B in the canonical K-major layout: N = output channels, K = input
// channels; LBO = NS/8 x 128 bytes along K, SBO = 128 bytes along N).
// With transpose set, the layer packed is the adjoint of a stored layer with
// Cout inputs and Cin outputs: w'[co][ci][tap] = w[ci][co][26 - tap] (the data
// gradient of a zero-padded 3x3x3 convolution is the zero-padded convolution
// with the channel roles swapped and the taps mirrored).
__global__ void pack_w3(const __nv_bfloat16* __restrict__ w, int Cin, int Cout, int NS, int S,
                        size_t n, int transpose, __nv_bfloat16* __restrict__ out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)(i & 7), r = (int)((i >> 3) & 7);
  size_t q = i >> 6;
  const int ng = (int)(q % (NS / 8));
  q /= NS / 8;
  const int kc = (int)(q % 2);
  q /= 2;
  const int tap = (int)(q % 27);
  q /= 27;
  const int stage = (int)(q % S), slice = (int)(q / S);
  const int co = slice * NS + 8 * ng + r, ci = 16 * stage + 8 * kc + c;
  const size_t src = transpose ? ((size_t)ci * Cout + co) * 27 + (26 - tap)
                               : ((size_t)co * Cin + ci) * 27 + tap;
  out[i] = (co < Cout && ci < Cin) ? w[src] : __float2bfloat16_rn(0.f);
}

template <int NS>
__global__ void __launch_bounds__(128)
conv3_tc(const float* __restrict__ in, int Cin, const __nv_bfloat16* __restrict__ wp,
         const float* __restrict__ bias, float* __restrict__ out, int Cout, Dims d, int relu,
         const float* __restrict__ gate, int tiles_x, int tiles_y, int32_t* err) {
  using C = CtShape<NS>;
  extern __shared__ __align__(16) unsigned char ct_raw[];
  unsigned char* As = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(ct_raw) + 127) & ~(uintptr_t)127);
  unsigned char* Bs = As + kCtA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + C::B);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(Bs + C::B + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int slice = blockIdx.y;
  const int S = (Cin + kCtCin - 1) / kCtCin;
  const int ntiles = tiles_x * tiles_y * d.D;
  const size_t V = (size_t)d.V();
  if (warp == 0) {
    tmem_alloc(tslot, C::COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t a_addr = smem_u32(As), b_addr = smem_u32(Bs);
  constexpr uint32_t IDESC = make_idesc(1u, 128, NS);
  uint32_t phase = 0;
  // staging assignment, the same for every tile and stage: thread t < 120
  // owns staged column xx = t % 10 of rows r = t / 10 + 12 k (row r = z-plane
  // r / 18, y-row r % 18 of the halo tile), for both 8-channel groups
  const bool stager = tid < 120;
  const int xx = tid % kCtHX, r0 = tid / kCtHX;
  auto stage_b = [&](int s) {
    const uint4* src = reinterpret_cast<const uint4*>(wp) + ((size_t)slice * S + s) * (C::B / 16);
    uint4* dst = reinterpret_cast<uint4*>(Bs);
    for (int i = tid; i < C::B / 16; i += 128) dst[i] = src[i];
  };
  if (S == 1) stage_b(0);   // one stage: the weights stay for every tile
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tx = t % tiles_x, ty = (t / tiles_x) % tiles_y, z = t / (tiles_x * tiles_y);
    const int x0 = tx * kCtTX, y0 = ty * kCtTY;
    const int gx = x0 - 1 + xx;
    const bool xin = gx >= 0 && gx < d.W;
    for (int s = 0; s < S; ++s) {
      if (stager) {
#pragma unroll 2
        for (int r = r0; r < 3 * kCtHY; r += 12) {
          const int zz = r / kCtHY, yy = r - zz * kCtHY;
          const int gy = y0 - 1 + yy, gz = z - 1 + zz;
          const bool inside = xin && gy >= 0 && gz >= 0 && gy < d.H && gz < d.D;
          const size_t vox = inside ? ((size_t)gz * d.H + gy) * d.W + gx : 0;
          const int pos = r * kCtHX + xx;
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            const int c0 = s * kCtCin + 8 * g;
            const float* p = in + (size_t)c0 * V + vox;
            float v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = (inside && c0 + c < Cin) ? p[(size_t)c * V] : 0.f;
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
              const float2 hf = __bfloat1622float2(h);
              const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
              hi[q] = *reinterpret_cast<const uint32_t*>(&h);
              lo[q] = *reinterpret_cast<const uint32_t*>(&l);
            }
            *reinterpret_cast<uint4*>(As + g * kCtPart + pos * 16) =
                make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(As + (2 + g) * kCtPart + pos * 16) =
                make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
      }
      if (S > 1) stage_b(s);
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll 1
        for (int tap = 0; tap < 27; ++tap) {
          const int dx = tap % 3, dy = (tap / 3) % 3, dz = tap / 9;
          const uint32_t aoff = (uint32_t)(((dz * kCtHY + dy) * kCtHX + dx) * 16);
          const uint64_t bd = smem_desc(b_addr + tap * (2 * (NS / 8) * 128), (NS / 8) * 128, 128);
#pragma unroll
          for (int part = 0; part < 2; ++part) {   // activations hi, lo
            const uint64_t ad = smem_desc(a_addr + part * 2 * kCtPart + aoff, kCtPart, kCtHX * 16);
            mma_f16(tmem, ad, bd, IDESC, (s | tap | part) ? 1u : 0u);
          }
        }
        mma_commit(bar);
      }
      // the next stage (or tile) rewrites A and B, the epilogue reads D: wait
      // for these MMAs (one lane per warp polls; the warp barrier and the
      // fence order the rest of the warp)
      if ((tid & 31) == 0) {
        uint32_t spins = 0;
        bool ok;
        // back off between polls: the other CTAs of the SM need the issue
        // slots for their staging while these MMAs run
        while (!(ok = mbar_try_wait(bar, phase))) {
          if (++spins > kCtSpin) break;
          __nanosleep(128);
        }
        if (!ok) {
          atomicExch(err, 1);
          for (uint32_t s2 = 0; s2 < kCtSpin && !mbar_try_wait(bar, phase); ++s2) {
          }
        }
      }
      __syncwarp();
      phase ^= 1u;
      tc_fence_after();
    }
    // epilogue: thread tid holds TMEM lane tid = output voxel (x0 + tid % 8, y0 + tid / 8)
    float acc[NS];
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
    if constexpr (NS == 16) {
      tmem_ld16(lane_addr, acc);
    } else {
#pragma unroll
      for (int h = 0; h < NS / 32; ++h) {
        float part[32];
        tmem_ld32(lane_addr + 32 * h, part);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[32 * h + j] = part[j];
      }
    }
    tc_fence_before();   // the next tile's first MMA overwrites D after the next barrier
    const int ox = x0 + (tid & 7), oy = y0 + (tid >> 3);
    if (ox < d.W && oy < d.H) {
      const size_t vox = ((size_t)z * d.H + oy) * d.W + ox;
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const int co = slice * NS + j;
        if (co < Cout) {
          float r = bias ? acc[j] + bias[co] : acc[j];
          if (relu) r = fmaxf(r, 0.f);
          if (gate && !(gate[(size_t)co * V + vox] > 0.f)) r = 0.f;
          out[(size_t)co * V + vox] = r;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, C::COLS);
}

// output-channel slice of a layer: 16 for at most 16 channels, else 32
int ct_ns(int cout) { return cout <= 16 ? 16 : 32; }
size_t ct_packed_elems(int cin, int cout) {
  const int ns = ct_ns(cout);
  const size_t slices = (size_t)((cout + ns - 1) / ns), stages = (size_t)((cin + kCtCin - 1) / kCtCin);
  return slices * stages * (size_t)(ns == 16 ? CtShape<16>::B : CtShape<32>::B) / 2;
}

}  // namespace

__global__ void gate_relu_kernel(float* __restrict__ g, const float* __restrict__ act, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n && !(act[i] > 0.f)) g[i] = 0.f;
}

// ---------------------------------------------------------------- the net

struct NnLayer {
  int cin, cout, k;
  size_t w_off, b_off;       // offsets into the parameter vector
};

struct mfto_nn {
  int base, levels, in_ch, out_ch;
  long long max_vox, max_train_vox;
  cudaStream_t stream;
  std::vector<NnLayer> layers;
  size_t n_params;
  float *w32, *grad, *m1, *m2;   // FP32 master, gradient, Adam moments [n_params]
  __nv_bfloat16* w16;            // BF16 working copy [n_params]
  int adam_t;
  std::vector<float*> bufs;      // 3 slots (in, a, b) per block
  float *gbuf0, *gbuf1, *gbuf2;  // gradient scratch
  float* wpart;                  // gradient chunk partials
  size_t wpart_elems;
  double* lpart;                 // loss partials [2 kLossBlocks], loss, 1 / count
  float* dpred;                  // d loss / d output
  // tensor-core 3x3x3 convolutions: weights packed per layer in the MMA
  // layout (repacked after every weight change), offsets per layer, switch
  __nv_bfloat16* wpack;
  std::vector<size_t> wp_off;
  __nv_bfloat16* wpack_t;        // adjoint layers for the data gradient (training only)
  std::vector<size_t> wpt_off;
  bool wpack_dirty;
  int tc_conv;                   // 1: 3x3x3 convolutions on tcgen05 (default), 0: SIMT FP32
  int32_t* d_err;                // set when a tensor-core wait gave up
  int num_sms;
  int64_t launches;
  char msg[512];
};

namespace {

mfto_status nfail(mfto_nn* n, mfto_status code, const char* msg) {
  if (n) snprintf(n->msg, sizeof(n->msg), "%s", msg);
  return code;
}

#define NCUDA(n, call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      if (n) snprintf((n)->msg, sizeof((n)->msg), "%s: %s", #call, cudaGetErrorString(e_)); \
      return MFTO_CUDA_ERROR;                                                              \
    }                                                                                      \
  } while (0)

enum { SLOT_IN = 0, SLOT_A = 1, SLOT_B = 2 };
float* slot(mfto_nn* n, int bi, int s) { return n->bufs[3 * bi + s]; }
Dims level_dims(const Dims& d, int l) { return Dims{d.D >> l, d.H >> l, d.W >> l}; }
int chan(const mfto_nn* n, int l) { return n->base << l; }

// One 3x3x3 convolution on the tensor cores: cin -> cout channels with the
// packed weights wp (bias and gate may be NULL).
mfto_status conv3_tc_launch(mfto_nn* n, const float* in, int cin, const __nv_bfloat16* wp,
                            const float* bias, float* out, int cout, Dims d, int relu,
                            const float* gate) {
  const int ns = ct_ns(cout);
  const int tiles_x = (d.W + kCtTX - 1) / kCtTX, tiles_y = (d.H + kCtTY - 1) / kCtTY;
  // persistent CTAs: as many as fit on the GPU (shared memory: 4 per SM for
  // 16-channel slices, 3 for 32), at most one per tile
  const size_t tiles = (size_t)tiles_x * tiles_y * d.D;
  const size_t fit = (size_t)n->num_sms * (ns == 16 ? 4 : 3);
  const dim3 grid((unsigned)(tiles < fit ? tiles : fit), (unsigned)((cout + ns - 1) / ns));
  n->launches++;
  if (ns == 16)
    conv3_tc<16><<<grid, 128, CtShape<16>::SMEM, n->stream>>>(in, cin, wp, bias, out, cout, d, relu,
                                                              gate, tiles_x, tiles_y, n->d_err);
  else
    conv3_tc<32><<<grid, 128, CtShape<32>::SMEM, n->stream>>>(in, cin, wp, bias, out, cout, d, relu,
                                                              gate, tiles_x, tiles_y, n->d_err);
  NCUDA(n, cudaGetLastError());
  return MFTO_OK;
}

mfto_status conv_forward(mfto_nn* n, const NnLayer& L, const float* in, float* out, Dims d, int relu) {
  if (L.k == 3 && n->tc_conv) {
    const size_t li = (size_t)(&L - n->layers.data());
    return conv3_tc_launch(n, in, L.cin, n->wpack + n->wp_off[li], n->w32 + L.b_off, out, L.cout, d,
                           relu, nullptr);
  }
  const dim3 grid(cdiv(d.V(), kNT), cdiv(L.cout, kCOB));
  n->launches++;
  if (L.k == 3)
    conv_fwd<3><<<grid, kNT, 0, n->stream>>>(in, L.cin, n->w16 + L.w_off, n->w32 + L.b_off, out, L.cout, d, relu);
  else
    conv_fwd<1><<<grid, kNT, 0, n->stream>>>(in, L.cin, n->w16 + L.w_off, n->w32 + L.b_off, out, L.cout, d, relu);
  NCUDA(n, cudaGetLastError());
  return MFTO_OK;
}

int n_chunks(int V) {
  int c = (V + 4095) / 4096;
  return c > 64 ? 64 : (c < 1 ? 1 : c);
}

// weight and bias gradients of one conv into n->grad; if din, the input
// gradient, gated by `gate` (zero where gate <= 0) when gate is given
mfto_status conv_backward(mfto_nn* n, const NnLayer& L, const float* in, const float* dout,
                          float* din, const float* gate, Dims d) {
  const int V = d.V();
  const int KK = L.k * L.k * L.k;
  const int chunks = n_chunks(V);
  const int chunk = (V + chunks - 1) / chunks;
  const size_t nw = (size_t)L.cout * L.cin * KK;
  if ((size_t)chunks * nw > n->wpart_elems) return nfail(n, MFTO_INVALID_ARG, "weight partials too small");
  n->launches += 4;
  if (L.k == 3)
    conv_bwd_weight<3><<<dim3(L.cout * L.cin, chunks), kNT, 0, n->stream>>>(in, L.cin, dout, L.cout, d, chunk, n->wpart);
  else
    conv_bwd_weight<1><<<dim3(L.cout * L.cin, chunks), kNT, 0, n->stream>>>(in, L.cin, dout, L.cout, d, chunk, n->wpart);
  sum_chunks<<<cdiv(nw, 256), 256, 0, n->stream>>>(n->wpart, (int)nw, chunks, n->grad + L.w_off);
  bias_grad<<<dim3(L.cout, chunks), kNT, 0, n->stream>>>(dout, L.cout, V, chunk, n->wpart);
  sum_chunks<<<cdiv(L.cout, 256), 256, 0, n->stream>>>(n->wpart, L.cout, chunks, n->grad + L.b_off);
  if (din && L.k == 3 && n->tc_conv && n->wpack_t) {
    // the data gradient as the adjoint convolution on the tensor cores
    const size_t li = (size_t)(&L - n->layers.data());
    mfto_status s = conv3_tc_launch(n, dout, L.cout, n->wpack_t + n->wpt_off[li], nullptr, din,
                                    L.cin, d, 0, gate);
    if (s != MFTO_OK) return s;
  } else if (din) {
    n->launches++;
    const dim3 grid(cdiv(V, kNT), cdiv(L.cin, kCOB));
    if (L.k == 3)
      conv_bwd_data<3><<<grid, kNT, 0, n->stream>>>(dout, L.cout, n->w16 + L.w_off, din, L.cin, d, gate);
    else
      conv_bwd_data<1><<<grid, kNT, 0, n->stream>>>(dout, L.cout, n->w16 + L.w_off, din, L.cin, d, gate);
  }
  NCUDA(n, cudaGetLastError());
  return MFTO_OK;
}

// Block indices: encoders 0..L-2, bottleneck L-1, decoders L..2L-2 (level
// L-2 .. 0).  Layer indices: block bi has convs 2 bi (a) and 2 bi + 1 (b);
// the head is last.
// the 3x3x3 layers' weights in the tensor-core kernel's layout
mfto_status pack_weights(mfto_nn* n) {
  for (size_t i = 0; i < n->layers.size(); ++i) {
    const NnLayer& ly = n->layers[i];
    if (ly.k != 3) continue;
    const int ns = ct_ns(ly.cout);
    const int S = (ly.cin + kCtCin - 1) / kCtCin;
    const size_t cnt = ct_packed_elems(ly.cin, ly.cout);
    n->launches++;
    pack_w3<<<cdiv(cnt, 256), 256, 0, n->stream>>>(n->w16 + ly.w_off, ly.cin, ly.cout, ns, S, cnt, 0,
                                                   n->wpack + n->wp_off[i]);
    if (n->wpack_t) {   // the adjoint layer: cout inputs, cin outputs
      const size_t cnt_t = ct_packed_elems(ly.cout, ly.cin);
      n->launches++;
      pack_w3<<<cdiv(cnt_t, 256), 256, 0, n->stream>>>(n->w16 + ly.w_off, ly.cout, ly.cin,
                                                       ct_ns(ly.cin), (ly.cout + kCtCin - 1) / kCtCin,
                                                       cnt_t, 1, n->wpack_t + n->wpt_off[i]);
    }
  }
  NCUDA(n, cudaGetLastError());
  n->wpack_dirty = false;
  return MFTO_OK;
}

mfto_status net_forward(mfto_nn* n, const float* x, float* out, Dims d) {
  const int L = n->levels;
  mfto_status s = MFTO_OK;
  if (n->tc_conv && n->wpack_dirty) {
    s = pack_weights(n);
    if (s != MFTO_OK) return s;
  }
  for (int l = 0; l < L - 1; ++l) {                         // encoders
    const Dims dl = level_dims(d, l);
    if (l == 0) {
      n->launches++;
      copy_f32<<<cdiv((size_t)n->in_ch * dl.V(), 256), 256, 0, n->stream>>>(x, slot(n, 0, SLOT_IN),
                                                                           (size_t)n->in_ch * dl.V());
    }
    s = conv_forward(n, n->layers[2 * l], slot(n, l, SLOT_IN), slot(n, l, SLOT_A), dl, 1);
    if (s == MFTO_OK) s = conv_forward(n, n->layers[2 * l + 1], slot(n, l, SLOT_A), slot(n, l, SLOT_B), dl, 1);
    if (s != MFTO_OK) return s;
    const Dims dn = level_dims(d, l + 1);
    n->launches++;
    pool_fwd<<<cdiv((size_t)chan(n, l) * dn.V(), 256), 256, 0, n->stream>>>(
        slot(n, l, SLOT_B), slot(n, l + 1, SLOT_IN), chan(n, l), dn);
  }
  {                                                          // bottleneck
    const Dims db = level_dims(d, L - 1);
    s = conv_forward(n, n->layers[2 * (L - 1)], slot(n, L - 1, SLOT_IN), slot(n, L - 1, SLOT_A), db, 1);
    if (s == MFTO_OK)
      s = conv_forward(n, n->layers[2 * (L - 1) + 1], slot(n, L - 1, SLOT_A), slot(n, L - 1, SLOT_B), db, 1);
    if (s != MFTO_OK) return s;
  }
  for (int l = L - 2; l >= 0; --l) {                         // decoders
    const int bi = 2 * (L - 1) - l;
    const Dims dl = level_dims(d, l);
    const int c_up = chan(n, l + 1), c_skip = chan(n, l);
    float* cat = slot(n, bi, SLOT_IN);
    n->launches += 2;
    spread_up<<<cdiv((size_t)c_up * dl.V(), 256), 256, 0, n->stream>>>(slot(n, bi - 1, SLOT_B), cat, c_up,
                                                                       dl, 1.f, 0);
    copy_f32<<<cdiv((size_t)c_skip * dl.V(), 256), 256, 0, n->stream>>>(
        slot(n, l, SLOT_B), cat + (size_t)c_up * dl.V(), (size_t)c_skip * dl.V());
    s = conv_forward(n, n->layers[2 * bi], cat, slot(n, bi, SLOT_A), dl, 1);
    if (s == MFTO_OK) s = conv_forward(n, n->layers[2 * bi + 1], slot(n, bi, SLOT_A), slot(n, bi, SLOT_B), dl, 1);
    if (s != MFTO_OK) return s;
  }
  return conv_forward(n, n->layers.back(), slot(n, 2 * (L - 1), SLOT_B), out, d, 0);
}

void gate(mfto_nn* n, float* g, const float* act, size_t cnt) {
  n->launches++;
  gate_relu_kernel<<<cdiv(cnt, 256), 256, 0, n->stream>>>(g, act, cnt);
}

mfto_status net_backward(mfto_nn* n, const float* dout, Dims d) {
  const int L = n->levels;
  float* g0 = n->gbuf0;
  float* g1 = n->gbuf1;
  float* g2 = n->gbuf2;
  const int last = 2 * (L - 1);
  // head: g0 = gradient w.r.t. the pre-activation of the last decoder's b-conv
  mfto_status s = conv_backward(n, n->layers.back(), slot(n, last, SLOT_B), dout, g0,
                                slot(n, last, SLOT_B), d);
  if (s != MFTO_OK) return s;
  std::vector<float*> stash(L - 1, nullptr);
  for (int l = 0; l <= L - 2; ++l) {                         // decoders, level 0 first
    const int bi = 2 * (L - 1) - l;
    const Dims dl = level_dims(d, l);
    s = conv_backward(n, n->layers[2 * bi + 1], slot(n, bi, SLOT_A), g0, g1, slot(n, bi, SLOT_A), dl);
    if (s == MFTO_OK) s = conv_backward(n, n->layers[2 * bi], slot(n, bi, SLOT_IN), g1, g2, nullptr, dl);
    if (s != MFTO_OK) return s;
    const int c_up = chan(n, l + 1), c_skip = chan(n, l);
    // the skip part belongs to the encoder output e_l: keep it in this
    // block's 'a' slot (same size, no longer needed)
    n->launches++;
    copy_f32<<<cdiv((size_t)c_skip * dl.V(), 256), 256, 0, n->stream>>>(
        g2 + (size_t)c_up * dl.V(), slot(n, bi, SLOT_A), (size_t)c_skip * dl.V());
    stash[l] = slot(n, bi, SLOT_A);
    // the upsampled part belongs to the block below, gated by its ReLU
    const Dims dc = level_dims(d, l + 1);
    n->launches++;
    gather_up<<<cdiv((size_t)c_up * dc.V(), 256), 256, 0, n->stream>>>(g2, g0, c_up, dc);
    gate(n, g0, slot(n, bi - 1, SLOT_B), (size_t)c_up * dc.V());
  }
  {                                                          // bottleneck
    const Dims db = level_dims(d, L - 1);
    s = conv_backward(n, n->layers[2 * (L - 1) + 1], slot(n, L - 1, SLOT_A), g0, g1, slot(n, L - 1, SLOT_A), db);
    if (s == MFTO_OK) s = conv_backward(n, n->layers[2 * (L - 1)], slot(n, L - 1, SLOT_IN), g1, g2, nullptr, db);
    if (s != MFTO_OK) return s;
  }
  for (int l = L - 2; l >= 0; --l) {                         // encoders
    const Dims dl = level_dims(d, l);
    const int C = chan(n, l);
    const size_t cnt = (size_t)C * dl.V();
    n->launches += 2;
    spread_up<<<cdiv(cnt, 256), 256, 0, n->stream>>>(g2, g0, C, dl, 0.125f, 0);   // pooling adjoint
    add_f32<<<cdiv(cnt, 256), 256, 0, n->stream>>>(stash[l], g0, cnt);
    gate(n, g0, slot(n, l, SLOT_B), cnt);
    s = conv_backward(n, n->layers[2 * l + 1], slot(n, l, SLOT_A), g0, g1, slot(n, l, SLOT_A), dl);
    if (s == MFTO_OK)
      s = conv_backward(n, n->layers[2 * l], slot(n, l, SLOT_IN), g1, l > 0 ? g2 : nullptr, nullptr, dl);
    if (s != MFTO_OK) return s;
  }
  NCUDA(n, cudaGetLastError());
  return MFTO_OK;
}

mfto_status check_dims(mfto_nn* n, int D, int H, int W, bool train) {
  const int m = 1 << (n->levels - 1);
  if (D < m || H < m || W < m || D % m || H % m || W % m)
    return nfail(n, MFTO_INVALID_ARG, "grid dimensions must be positive multiples of 2^(levels-1)");
  const long long V = (long long)D * H * W;
  if (V > (train ? n->max_train_vox : n->max_vox))
    return nfail(n, MFTO_TOO_LARGE, "grid larger than the network was created for");
  return MFTO_OK;
}

// masked-MSE gradient of n->dpred (in place); the loss stays on the device
mfto_status loss_and_grad(mfto_nn* n, const float* target, const float* mask, size_t cnt) {
  n->launches += 3;
  mse_grad<<<kLossBlocks, 256, 0, n->stream>>>(n->dpred, target, mask, n->dpred, cnt, n->lpart);
  mse_finish<<<1, 32, 0, n->stream>>>(n->lpart);
  mse_scale<<<cdiv(cnt, 256), 256, 0, n->stream>>>(n->dpred, cnt, n->lpart);
  NCUDA(n, cudaGetLastError());
  return MFTO_OK;
}

mfto_status read_loss(mfto_nn* n, double* loss) {
  NCUDA(n, cudaMemcpyAsync(loss, n->lpart + 2 * kLossBlocks, sizeof(double), cudaMemcpyDeviceToHost,
                           n->stream));
  NCUDA(n, cudaStreamSynchronize(n->stream));
  return MFTO_OK;
}

void free_nn(mfto_nn* n) {
  if (!n) return;
  for (float* p : n->bufs)
    if (p) cudaFree(p);
  void* ptrs[] = {n->wpack, n->wpack_t, n->d_err, n->w32, n->grad, n->m1, n->m2, n->w16, n->gbuf0, n->gbuf1, n->gbuf2, n->wpart,
                  n->lpart, n->dpred};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete n;
}

}  // namespace

extern "C" mfto_status mfto_nn_create(int32_t base, int32_t levels, int64_t max_voxels,
                                      int64_t max_train_voxels, uint64_t seed, void* stream,
                                      mfto_nn** out) {
  if (!out) return MFTO_INVALID_ARG;
  *out = nullptr;
  if (base < 1 || base > 64 || levels < 2 || levels > 6 || max_voxels < 1 || max_train_voxels < 0 ||
      max_train_voxels > max_voxels)
    return MFTO_INVALID_ARG;
  mfto_nn* n = new mfto_nn();
  n->base = base;
  n->levels = levels;
  n->in_ch = 4;
  n->out_ch = 3;
  n->max_vox = max_voxels;
  n->max_train_vox = max_train_voxels;
  n->stream = (cudaStream_t)stream;
  // layers in forward order (encoders, bottleneck, decoders, head)
  const int L = levels;
  size_t off = 0;
  auto add = [&](int ci, int co, int k) {
    NnLayer ly;
    ly.cin = ci; ly.cout = co; ly.k = k;
    ly.w_off = off; off += (size_t)co * ci * k * k * k;
    ly.b_off = off; off += co;
    n->layers.push_back(ly);
  };
  int prev = n->in_ch;
  for (int l = 0; l < L - 1; ++l) { add(prev, base << l, 3); add(base << l, base << l, 3); prev = base << l; }
  add(prev, base << (L - 1), 3);
  add(base << (L - 1), base << (L - 1), 3);
  for (int l = L - 2; l >= 0; --l) { add((base << (l + 1)) + (base << l), base << l, 3); add(base << l, base << l, 3); }
  add(base, n->out_ch, 1);
  n->n_params = off;
  bool ok = true;
  auto A = [&](void** p, size_t bytes) {
    if (ok && bytes && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
  };
  A((void**)&n->w32, sizeof(float) * off);
  A((void**)&n->grad, sizeof(float) * off);
  A((void**)&n->m1, sizeof(float) * off);
  A((void**)&n->m2, sizeof(float) * off);
  A((void**)&n->w16, sizeof(__nv_bfloat16) * off);
  // activations for max_voxels
  const long long V = max_voxels;
  const int nb = 2 * (L - 1) + 1;
  n->bufs.assign(3 * nb, nullptr);
  for (int bi = 0; bi < nb && ok; ++bi) {
    const int l = bi < L ? bi : 2 * (L - 1) - bi;
    const long long Vl = V >> (3 * l);
    long long cin;
    if (bi == 0) cin = n->in_ch;
    else if (bi < L) cin = base << (l - 1);
    else cin = (base << (l + 1)) + (base << l);
    A((void**)&n->bufs[3 * bi + SLOT_IN], sizeof(float) * (size_t)(cin * Vl + 1));
    A((void**)&n->bufs[3 * bi + SLOT_A], sizeof(float) * (size_t)((base << l) * Vl + 1));
    A((void**)&n->bufs[3 * bi + SLOT_B], sizeof(float) * (size_t)((base << l) * Vl + 1));
  }
  const long long TV = max_train_voxels;
  const size_t gsz = (size_t)3 * base * TV + 16;           // largest gradient tensor: level-0 concat
  if (TV > 0) {
    A((void**)&n->gbuf0, sizeof(float) * gsz);
    A((void**)&n->gbuf1, sizeof(float) * gsz);
    A((void**)&n->gbuf2, sizeof(float) * gsz);
    size_t wp = 0;
    for (size_t i = 0; i < n->layers.size(); ++i) {
      const NnLayer& ly = n->layers[i];
      const int bi = (int)(i / 2);
      const int l = (i == n->layers.size() - 1) ? 0 : (bi < L ? bi : 2 * (L - 1) - bi);
      const size_t need = (size_t)n_chunks((int)(TV >> (3 * l))) * ((size_t)ly.cout * ly.cin * ly.k * ly.k * ly.k + ly.cout);
      wp = wp > need ? wp : need;
    }
    n->wpart_elems = wp;
    A((void**)&n->wpart, sizeof(float) * wp);
    A((void**)&n->dpred, sizeof(float) * (size_t)(n->out_ch * TV));
  }
  A((void**)&n->lpart, sizeof(double) * (2 * kLossBlocks + 2));
  {
    size_t pk = 0;
    n->wp_off.assign(n->layers.size(), 0);
    for (size_t i = 0; i < n->layers.size(); ++i) {
      n->wp_off[i] = pk;
      if (n->layers[i].k == 3) pk += ct_packed_elems(n->layers[i].cin, n->layers[i].cout);
    }
    A((void**)&n->wpack, sizeof(__nv_bfloat16) * (pk + 8));
    if (TV > 0) {
      size_t pt = 0;
      n->wpt_off.assign(n->layers.size(), 0);
      for (size_t i = 0; i < n->layers.size(); ++i) {
        n->wpt_off[i] = pt;
        if (n->layers[i].k == 3) pt += ct_packed_elems(n->layers[i].cout, n->layers[i].cin);
      }
      A((void**)&n->wpack_t, sizeof(__nv_bfloat16) * (pt + 8));
    }
    A((void**)&n->d_err, sizeof(int32_t));
    n->tc_conv = 1;
    n->wpack_dirty = true;
    int dev = 0;
    n->num_sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (!ok) {
    cudaGetLastError();
    free_nn(n);
    return MFTO_OOM;
  }
  // He-normal initial weights, zero biases (seeded)
  std::vector<float> h(off, 0.f);
  std::mt19937_64 rng(seed);
  for (const NnLayer& ly : n->layers) {
    std::normal_distribution<double> nd(0.0, sqrt(2.0 / (ly.cin * ly.k * ly.k * ly.k)));
    for (size_t i = 0; i < (size_t)ly.cout * ly.cin * ly.k * ly.k * ly.k; ++i) h[ly.w_off + i] = (float)nd(rng);
  }
  if (cudaMemcpyAsync(n->w32, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice, n->stream) != cudaSuccess ||
      cudaMemsetAsync(n->m1, 0, sizeof(float) * off, n->stream) != cudaSuccess ||
      cudaMemsetAsync(n->m2, 0, sizeof(float) * off, n->stream) != cudaSuccess) {
    free_nn(n);
    return MFTO_CUDA_ERROR;
  }
  to_bf16<<<cdiv(off, 256), 256, 0, n->stream>>>(n->w32, n->w16, off);
  if (cudaMemsetAsync(n->d_err, 0, sizeof(int32_t), n->stream) != cudaSuccess ||
      cudaFuncSetAttribute(conv3_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           CtShape<16>::SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(conv3_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           CtShape<32>::SMEM) != cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess) {
    cudaGetLastError();
    free_nn(n);
    return MFTO_CUDA_ERROR;
  }
  *out = n;
  return MFTO_OK;
}

extern "C" mfto_status mfto_nn_destroy(mfto_nn* n) {
  if (!n) return MFTO_INVALID_ARG;
  cudaStreamSynchronize(n->stream);
  free_nn(n);
  return MFTO_OK;
}

extern "C" const char* mfto_nn_last_error(const mfto_nn* n) { return n ? n->msg : "null network"; }

extern "C" mfto_status mfto_nn_num_params(const mfto_nn* n, int64_t* count) {
  if (!n || !count) return MFTO_INVALID_ARG;
  *count = (int64_t)n->n_params;
  return MFTO_OK;
}

extern "C" mfto_status mfto_nn_get_params(mfto_nn* n, float* h_out) {
  if (!n || !h_out) return MFTO_INVALID_ARG;
  NCUDA(n, cudaMemcpyAsync(h_out, n->w32, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost, n->stream));
  NCUDA(n, cudaStreamSynchronize(n->stream));
  return MFTO_OK;
}

extern "C" mfto_status mfto_nn_set_params(mfto_nn* n, const float* h_in) {
  if (!n || !h_in) return MFTO_INVALID_ARG;
  NCUDA(n, cudaMemcpyAsync(n->w32, h_in, sizeof(float) * n->n_params, cudaMemcpyHostToDevice, n->stream));
  to_bf16<<<cdiv(n->n_params, 256), 256, 0, n->stream>>>(n->w32, n->w16, n->n_params);
  NCUDA(n, cudaGetLastError());
  NCUDA(n, cudaStreamSynchronize(n->stream));
  n->wpack_dirty = true;
  n->adam_t = 0;
  NCUDA(n, cudaMemsetAsync(n->m1, 0, sizeof(float) * n->n_params, n->stream));
  NCUDA(n, cudaMemsetAsync(n->m2, 0, sizeof(float) * n->n_params, n->stream));
  return MFTO_OK;
}

extern "C" mfto_status mfto_nn_set_tensor_cores(mfto_nn* n, int32_t on) {
  if (!n || (on != 0 && on != 1)) return MFTO_INVALID_ARG;
  n->tc_conv = on;
  return MFTO_OK;
}

extern "C" mfto_status mfto_nn_tc_status(mfto_nn* n, int32_t* gave_up) {
  if (!n || !gave_up) return MFTO_INVALID_ARG;
  NCUDA(n, cudaMemcpyAsync(gave_up, n->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, n->stream));
  NCUDA(n, cudaStreamSynchronize(n->stream));
  return MFTO_OK;
}

extern "C" mfto_status mfto_nn_forward(mfto_nn* n, int32_t D, int32_t H, int32_t W,
                                       const float* d_in, float* d_out) {
  if (!n || !d_in || !d_out) return MFTO_INVALID_ARG;
  mfto_status s = check_dims(n, D, H, W, false);
  if (s != MFTO_OK) return s;
  return net_forward(n, d_in, d_out, Dims{D, H, W});
}

namespace {
mfto_status adam(mfto_nn* n, float lr) {
  n->adam_t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->adam_t), c2 = 1.f - powf(b2, (float)n->adam_t);
  n->launches++;
  adam_step<<<cdiv(n->n_params, 256), 256, 0, n->stream>>>(n->w32, n->w16, n->grad, n->m1, n->m2,
                                                           n->n_params, lr, b1, b2, 1e-8f, c1, c2);
  NCUDA(n, cudaGetLastError());
  n->wpack_dirty = true;
  return MFTO_OK;
}

mfto_status gradient(mfto_nn* n, int32_t D, int32_t H, int32_t W, const float* d_in,
                     const float* d_target, const float* d_mask) {
  if (!d_in || !d_target || !d_mask) return nfail(n, MFTO_INVALID_ARG, "null pointer");
  mfto_status s = check_dims(n, D, H, W, true);
  if (s != MFTO_OK) return s;
  const Dims d{D, H, W};
  s = net_forward(n, d_in, n->dpred, d);   // output, then overwritten by its gradient
  if (s == MFTO_OK) s = loss_and_grad(n, d_target, d_mask, (size_t)n->out_ch * d.V());
  if (s == MFTO_OK) s = net_backward(n, n->dpred, d);
  return s;
}
}  // namespace

extern "C" mfto_status mfto_nn_gradient(mfto_nn* n, int32_t D, int32_t H, int32_t W,
                                        const float* d_in, const float* d_target,
                                        const float* d_mask, double* loss, float* h_grad) {
  if (!n || !loss) return MFTO_INVALID_ARG;
  mfto_status s = gradient(n, D, H, W, d_in, d_target, d_mask);
  if (s != MFTO_OK) return s;
  if (h_grad)
    NCUDA(n, cudaMemcpyAsync(h_grad, n->grad, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost,
                             n->stream));
  return read_loss(n, loss);
}

extern "C" mfto_status mfto_nn_train_step(mfto_nn* n, int32_t D, int32_t H, int32_t W,
                                          const float* d_in, const float* d_target,
                                          const float* d_mask, float lr, double* loss) {
  if (!n || !(lr > 0.f)) return MFTO_INVALID_ARG;
  mfto_status s = gradient(n, D, H, W, d_in, d_target, d_mask);
  if (s != MFTO_OK) return s;
  s = adam(n, lr);
  if (s != MFTO_OK) return s;
  return loss ? read_loss(n, loss) : MFTO_OK;
}

extern "C" mfto_status mfto_nn_launch_count(const mfto_nn* n, int64_t* count) {
  if (!n || !count) return MFTO_INVALID_ARG;
  *count = n->launches;
  return MFTO_OK;
}

// ---------------------------------------------------------------- internal
// Inference on the caller's stream (used by the learned solve).
mfto_status nn_infer(mfto_nn* n, cudaStream_t st, int D, int H, int W, const float* x, float* y) {
  mfto_status s = check_dims(n, D, H, W, false);
  if (s != MFTO_OK) return s;
  cudaStream_t keep = n->stream;
  n->stream = st;
  s = net_forward(n, x, y, Dims{D, H, W});
  n->stream = keep;
  return s;
}

int nn_levels(const mfto_nn* n) { return n->levels; }
long long nn_max_voxels(const mfto_nn* n) { return n->max_vox; }
const char* nn_message(const mfto_nn* n) { return n->msg; }

// Training with a loss the caller computes from the output (the learned
// solve's energy loss): train_forward leaves the output in the returned
// buffer [3][D][H][W]; the caller overwrites it with d loss / d output and
// calls train_backward, which back-propagates and takes one Adam step.
mfto_status nn_train_forward(mfto_nn* n, cudaStream_t st, int D, int H, int W, const float* x,
                             float** out) {
  mfto_status s = check_dims(n, D, H, W, true);
  if (s != MFTO_OK) return s;
  cudaStream_t keep = n->stream;
  n->stream = st;
  s = net_forward(n, x, n->dpred, Dims{D, H, W});
  n->stream = keep;
  *out = n->dpred;
  return s;
}

mfto_status nn_train_backward(mfto_nn* n, cudaStream_t st, int D, int H, int W, float lr) {
  cudaStream_t keep = n->stream;
  n->stream = st;
  mfto_status s = net_backward(n, n->dpred, Dims{D, H, W});
  if (s == MFTO_OK) s = adam(n, lr);
  n->stream = keep;
  return s;
}

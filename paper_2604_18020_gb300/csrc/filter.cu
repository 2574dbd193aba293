// Cone density filter (Sec. 3.1) and its transpose.
//
//   forward:   y_e = sum_{i in N(e)} w_ei x_i / W_e
//   transpose: y_i = sum_{e in N(i)} w_ei x_e / W_e
// N(e): the stencil offsets of mfto_filter_stencil, truncated at the domain
// boundary; W_e = sum_{i in N(e)} w_ei.  Terms are added in stencil order with
// separate IEEE multiply and add (no fused multiply-add), so the result does
// not depend on the compiler's contraction choices.  The weight matrix is
// symmetric, so the transpose visits the same offsets; it divides x by W
// once per element in a first pass (the same quotients the sum would form
// term by term) and then runs the forward sum on the quotients.
#include "common.cuh"

namespace {

__global__ void __launch_bounds__(MFTO_BLOCK)
filter_kernel(const double* __restrict__ x, double* __restrict__ y,
              const double* __restrict__ W, const int32_t* __restrict__ off,
              const double* __restrict__ w, int n_st, Grid g, int transpose,
              int rowsums_only) {
  extern __shared__ unsigned char smem_raw[];
  double* sw = reinterpret_cast<double*>(smem_raw);
  int* so = reinterpret_cast<int*>(sw + n_st);
  for (int t = threadIdx.x; t < n_st; t += blockDim.x) {
    sw[t] = w[t];
    so[3 * t + 0] = off[3 * t + 0];
    so[3 * t + 1] = off[3 * t + 1];
    so[3 * t + 2] = off[3 * t + 2];
  }
  __syncthreads();
  const int n = g.nelx * g.nely * g.nelz;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int i = e % g.nelx, j = (e / g.nelx) % g.nely, k = e / (g.nelx * g.nely);
    double acc = 0.0;
    for (int t = 0; t < n_st; ++t) {
      const int ii = i + so[3 * t], jj = j + so[3 * t + 1], kk = k + so[3 * t + 2];
      if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nelx || jj >= g.nely || kk >= g.nelz) continue;
      const int nb = ii + g.nelx * (jj + g.nely * kk);
      double term;
      if (rowsums_only)
        term = sw[t];
      else
        term = __dmul_rn(sw[t], x[nb]);
      acc = __dadd_rn(acc, term);
    }
    y[e] = (rowsums_only || transpose) ? acc : __ddiv_rn(acc, W[e]);
  }
}

__global__ void __launch_bounds__(MFTO_BLOCK)
divide_kernel(const double* __restrict__ x, const double* __restrict__ W, double* __restrict__ q,
              int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    q[e] = __ddiv_rn(x[e], W[e]);
}

}  // namespace

static mfto_status launch_filter(mfto_handle* h, const double* x, double* y, int transpose,
                                 int rowsums) {
  const Grid g = make_grid(h->mesh);
  const size_t smem = (size_t)h->n_stencil * (sizeof(double) + 3 * sizeof(int));
  if (smem > 48 * 1024)
    MFTO_CUDA(h, cudaFuncSetAttribute(filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  int blocks = (int)((h->n_elem + MFTO_BLOCK - 1) / MFTO_BLOCK);
  if (blocks > 16 * h->num_sms) blocks = 16 * h->num_sms;
  if (transpose) {   // quotients x / W into the OC scratch (free outside the OC update)
    h->launches++;
    divide_kernel<<<blocks, MFTO_BLOCK, 0, h->stream>>>(x, h->d_filter_W, h->d_oc,
                                                        (int)h->n_elem);
    x = h->d_oc;
  }
  h->launches++;
  filter_kernel<<<blocks, MFTO_BLOCK, smem, h->stream>>>(x, y, h->d_filter_W, h->d_stencil_off,
                                                         h->d_stencil_w, h->n_stencil, g,
                                                         transpose, rowsums);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

mfto_status filter_rowsums(mfto_handle* h) {
  return launch_filter(h, nullptr, h->d_filter_W, 0, 1);
}

mfto_status filter_launch(mfto_handle* h, const double* x, double* y, int transpose) {
  return launch_filter(h, x, y, transpose, 0);
}

extern "C" mfto_status mfto_filter(mfto_handle* h, const double* x, double* y,
                                   int32_t transpose) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, x && y, "mfto_filter: null pointer");
  MFTO_REQUIRE(h, x != y, "mfto_filter: y must not alias x");
  return filter_launch(h, x, y, transpose ? 1 : 0);
}

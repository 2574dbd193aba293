// Matrix-free K.v (Eq. matfree), the Jacobi diagonal (Sec. 3.6) and the SIMP
// modulus (Eq. simp).
//
// K.v here is node-centric: one thread owns one node and gathers the
// contributions of the (up to) 8 elements around it,
//   y_n = sum_{e owns n} E_e sum_{m in e} KE[l(n,e), l(m,e)] v_m,
// so every output is written exactly once, in a fixed summation order, with
// no atomics (Alg. 1 of the paper scatters with atomics instead).  Fixed DOFs
// are masked: their input is read as zero and their output is v itself.
#include "common.cuh"
#include "kv_node.cuh"

namespace {

// Node-centric dense K.v, grid-stride over nodes (see kv_node.cuh).
template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
kv_node_dense(const T* __restrict__ E, const T* __restrict__ v, T* __restrict__ y,
              const uint8_t* __restrict__ fixed, const T* __restrict__ ke_g,
              Grid g, int n_node) {
  __shared__ T ke[576];
  for (int t = threadIdx.x; t < 576; t += blockDim.x) ke[t] = ke_g[t];
  __syncthreads();
  const LoadPlain<T> ld{v};
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < n_node;
       node += gridDim.x * blockDim.x) {
    T a0, a1, a2;
    node_kv<T>(node, E, fixed, ke, g, ld, a0, a1, a2);
    const uint8_t fm = fixed[node];
    y[3 * node + 0] = (fm & 1) ? v[3 * node + 0] : a0;
    y[3 * node + 1] = (fm & 2) ? v[3 * node + 1] : a1;
    y[3 * node + 2] = (fm & 4) ? v[3 * node + 2] : a2;
  }
}

// diag_k = ke_diag * sum_{e owns node(k)} E_e (every diagonal entry of KE is
// the same on a cube), 1 on fixed DOFs; optionally stores the reciprocal.
template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
diag_node(const T* __restrict__ E, T* __restrict__ d, const uint8_t* __restrict__ fixed,
          T ke_diag, Grid g, int n_node, int inverse) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= n_node) return;
  const int i = node % g.nx;
  const int j = (node / g.nx) % g.ny;
  const int k = node / (g.nx * g.ny);
  T s = 0;
  for (int ce = 0; ce < 8; ++ce) {
    const int ei = i - 1 + (ce & 1), ej = j - 1 + ((ce >> 1) & 1), ek = k - 1 + (ce >> 2);
    if (ei < 0 || ej < 0 || ek < 0 || ei >= g.nelx || ej >= g.nely || ek >= g.nelz) continue;
    s += E[ei + g.nelx * (ej + g.nely * ek)];
  }
  const T val = ke_diag * s;
  const uint8_t fm = fixed[node];
  for (int c = 0; c < 3; ++c) {
    const T dv = ((fm >> c) & 1) ? T(1) : val;
    d[3 * node + c] = inverse ? T(1) / dv : dv;
  }
}

template <typename T>
__global__ void __launch_bounds__(MFTO_BLOCK)
modulus_kernel(const double* __restrict__ rho, T* __restrict__ E, double E0, double Emin,
               double penal, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  E[e] = (T)(Emin + (E0 - Emin) * pow(rho[e], penal));
}

}  // namespace

static inline int blocks_for(int64_t n) { return (int)((n + MFTO_BLOCK - 1) / MFTO_BLOCK); }
// grid of a grid-stride node loop: enough blocks to fill the GPU, capped so
// that the fused reductions of the PCG fit their partial-sum slots
static inline int node_blocks(const mfto_handle* h) { return reduction_blocks(h->n_node, MFTO_BLOCK); }

mfto_status kv_launch(mfto_handle* h, mfto_form form, const void* E, const void* v, void* y) {
  const Grid g = make_grid(h->mesh);
  if (form != MFTO_FORM_F64 && form != MFTO_FORM_F32 && !tc_form(form))
    return mfto_fail(h, MFTO_UNSUPPORTED, "mfto_kv: unsupported form %d", (int)form);
  kv_timing_begin(h, form);
  h->launches++;
  if (tc_form(form)) {
    mfto_status s = kv_tc_launch(h, form, (const float*)E, (const float*)v, (float*)y, h->stream);
    kv_timing_end(h);
    return s;
  }
  if (h->kv_variant != 1) {
    mfto_status s = form == MFTO_FORM_F64
        ? kv_tile_launch<double>(h, (const double*)E, (const double*)v, (double*)y, h->stream)
        : kv_tile_launch<float>(h, (const float*)E, (const float*)v, (float*)y, h->stream);
    kv_timing_end(h);
    return s;
  }
  if (form == MFTO_FORM_F64) {
    kv_node_dense<double><<<node_blocks(h), MFTO_BLOCK, 0, h->stream>>>(
        (const double*)E, (const double*)v, (double*)y, h->d_fixed, h->d_ke64, g, (int)h->n_node);
  } else if (form == MFTO_FORM_F32) {
    kv_node_dense<float><<<node_blocks(h), MFTO_BLOCK, 0, h->stream>>>(
        (const float*)E, (const float*)v, (float*)y, h->d_fixed, h->d_ke32, g, (int)h->n_node);
  } else {
    return mfto_fail(h, MFTO_UNSUPPORTED, "mfto_kv: unsupported form %d", (int)form);
  }
  kv_timing_end(h);
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

mfto_status diag_launch(mfto_handle* h, mfto_form form, const void* E, void* d, bool inverse) {
  const Grid g = make_grid(h->mesh);
  h->launches++;
  if (form == MFTO_FORM_F64) {
    diag_node<double><<<blocks_for(h->n_node), MFTO_BLOCK, 0, h->stream>>>(
        (const double*)E, (double*)d, h->d_fixed, h->ke_diag, g, (int)h->n_node, inverse);
  } else if (form == MFTO_FORM_F32) {
    diag_node<float><<<blocks_for(h->n_node), MFTO_BLOCK, 0, h->stream>>>(
        (const float*)E, (float*)d, h->d_fixed, (float)h->ke_diag, g, (int)h->n_node, inverse);
  } else {
    return mfto_fail(h, MFTO_UNSUPPORTED, "mfto_jacobi_diag: unsupported form %d", (int)form);
  }
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

mfto_status modulus_launch(mfto_handle* h, mfto_form form, const double* rho, void* E) {
  const int n = (int)h->n_elem;
  h->launches++;
  if (form == MFTO_FORM_F64) {
    modulus_kernel<double><<<blocks_for(n), MFTO_BLOCK, 0, h->stream>>>(
        rho, (double*)E, h->p.E0, h->p.Emin, h->p.penal, n);
  } else if (form == MFTO_FORM_F32) {
    modulus_kernel<float><<<blocks_for(n), MFTO_BLOCK, 0, h->stream>>>(
        rho, (float*)E, h->p.E0, h->p.Emin, h->p.penal, n);
  } else {
    return mfto_fail(h, MFTO_UNSUPPORTED, "mfto_simp_modulus: unsupported form %d", (int)form);
  }
  MFTO_LAUNCH_CHECK(h);
  return MFTO_OK;
}

extern "C" mfto_status mfto_kv(mfto_handle* h, mfto_form form, const void* E, const void* v,
                               void* y) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, E && v && y, "mfto_kv: null pointer");
  MFTO_REQUIRE(h, v != y, "mfto_kv: y must not alias v");
  return kv_launch(h, form, E, v, y);
}

extern "C" mfto_status mfto_set_kv_variant(mfto_handle* h, int32_t variant) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, variant >= 0 && variant <= 2, "mfto_set_kv_variant: variant must be 0, 1 or 2");
  if (h->kv_variant != variant) pcg_graph_release(h);
  h->kv_variant = variant;
  return MFTO_OK;
}

extern "C" mfto_status mfto_jacobi_diag(mfto_handle* h, mfto_form form, const void* E,
                                        void* d) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, E && d, "mfto_jacobi_diag: null pointer");
  return diag_launch(h, form, E, d, false);
}

extern "C" mfto_status mfto_simp_modulus(mfto_handle* h, mfto_form form, const double* rho,
                                         void* E) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, rho && E, "mfto_simp_modulus: null pointer");
  return modulus_launch(h, form, rho, E);
}

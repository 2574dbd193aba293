// Host entry points: version, parameters, unit element matrix, edof table,
// filter stencil, handle life cycle and K.v timing.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include "common.cuh"
#include "kv_column.cuh"
#include "modes.cuh"

mfto_status mfto_fail(mfto_handle* h, mfto_status code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}

extern "C" const char* mfto_version(void) { return "mfto 0.1 (sm_103a)"; }

extern "C" void mfto_default_params(mfto_params* p) {
  if (!p) return;
  p->E0 = 1.0;
  p->Emin = 1e-9;
  p->nu = 0.3;
  p->penal = 3.0;
  p->rmin = 1.5;
  p->volfrac = 0.3;
  p->move = 0.2;
  p->rtol = 1e-8;
  p->maxit = 10000;
  p->check_every = 32;
  p->max_rhs = 1;
}

// KE = T^-1 Kt T: Kt is the element operator in the per-axis (sum, difference)
// basis built by mode_operator(); T maps the 8 corner values of one component
// to the 8 modes and T^-1 = T^T / 8.
extern "C" mfto_status mfto_unit_ke(double E0, double nu, double h,
                                    double* ke) {
  if (!ke || !(h > 0.0) || !(nu > -1.0 && nu < 0.5)) return MFTO_INVALID_ARG;
  ModeOperator op = mode_operator(E0, nu, h);
  double Kt[24][24];
  memset(Kt, 0, sizeof(Kt));
  for (int t = 0; t < op.n_terms; ++t)
    Kt[3 * op.out_mode[t] + op.out_comp[t]][3 * op.in_mode[t] + op.in_comp[t]] += op.coef[t];
  // T[m][b] = prod_axis (m_axis == 0 ? 1 : (b_axis ? 1 : -1))
  double T[8][8];
  for (int m = 0; m < 8; ++m)
    for (int b = 0; b < 8; ++b) {
      double s = 1.0;
      for (int ax = 0; ax < 3; ++ax)
        if ((m >> ax) & 1) s *= ((b >> ax) & 1) ? 1.0 : -1.0;
      T[m][b] = s;
    }
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int b = 0; b < 8; ++b)
        for (int j = 0; j < 3; ++j) {
          double s = 0.0;
          for (int mo = 0; mo < 8; ++mo) {
            double row = 0.0;
            for (int mi = 0; mi < 8; ++mi) row += Kt[3 * mo + i][3 * mi + j] * T[mi][b];
            s += T[mo][a] * row;
          }
          ke[(3 * a + i) * 24 + 3 * b + j] = s / 8.0;
        }
  return MFTO_OK;
}

extern "C" mfto_status mfto_edof(const mfto_mesh* m, int32_t* edof) {
  if (!m || !edof || m->nelx < 1 || m->nely < 1 || m->nelz < 1) return MFTO_INVALID_ARG;
  const int64_t nx = m->nelx + 1, ny = m->nely + 1;
  if ((int64_t)3 * nx * ny * (m->nelz + 1) > INT32_MAX) return MFTO_INVALID_ARG;
  int64_t e = 0;
  for (int k = 0; k < m->nelz; ++k)
    for (int j = 0; j < m->nely; ++j)
      for (int i = 0; i < m->nelx; ++i, ++e)
        for (int l = 0; l < 8; ++l) {
          const int64_t n = (i + (l & 1)) + nx * ((j + ((l >> 1) & 1)) + ny * (k + (l >> 2)));
          for (int c = 0; c < 3; ++c) edof[e * 24 + 3 * l + c] = (int32_t)(3 * n + c);
        }
  return MFTO_OK;
}

extern "C" mfto_status mfto_filter_stencil(double rmin, int32_t cap,
                                           int32_t* off, double* w,
                                           int32_t* count) {
  if (!(rmin > 0.0) || rmin > 64.0 || !count) return MFTO_INVALID_ARG;
  const int R = (int)ceil(rmin) - 1;
  int n = 0;
  for (int dz = -R; dz <= R; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        const double wt = rmin - sqrt((double)(dx * dx + dy * dy + dz * dz));
        if (wt > 0.0) {
          if (n < cap && off && w) {
            off[3 * n + 0] = dx; off[3 * n + 1] = dy; off[3 * n + 2] = dz;
            w[n] = wt;
          }
          ++n;
        }
      }
  *count = n;
  return n <= cap ? MFTO_OK : MFTO_INVALID_ARG;
}

static mfto_status check_params(mfto_handle* h, const mfto_params* p) {
  MFTO_REQUIRE(h, p, "params is NULL");
  MFTO_REQUIRE(h, p->nu > -1.0 && p->nu < 0.5, "nu must lie in (-1, 0.5)");
  MFTO_REQUIRE(h, p->E0 > 0.0 && p->Emin >= 0.0 && p->Emin < p->E0, "need 0 <= Emin < E0");
  MFTO_REQUIRE(h, p->penal >= 1.0, "penal must be >= 1");
  MFTO_REQUIRE(h, p->rmin > 0.0 && p->rmin <= 64.0, "rmin must lie in (0, 64]");
  MFTO_REQUIRE(h, p->volfrac > 0.0 && p->volfrac <= 1.0, "volfrac must lie in (0, 1]");
  MFTO_REQUIRE(h, p->move > 0.0, "move must be > 0");
  MFTO_REQUIRE(h, p->rtol > 0.0, "rtol must be > 0");
  MFTO_REQUIRE(h, p->maxit >= 1, "maxit must be >= 1");
  MFTO_REQUIRE(h, p->check_every >= 2 && p->check_every % 2 == 0,
               "check_every must be even and >= 2");
  MFTO_REQUIRE(h, p->max_rhs >= 1 && p->max_rhs <= MFTO_MAX_RHS, "max_rhs must lie in 1..8");
  return MFTO_OK;
}

static void free_handle(mfto_handle* h) {
  if (!h) return;
  pcg_graph_release(h);
  multi_graph_release(h);
  learned_release(h);
  gmg_release(h);
  void* ptrs[] = {h->d_ke64, h->d_ke32, h->d_fixed, h->d_stencil_off, h->d_stencil_w,
                  h->d_filter_W, h->d_r, h->d_z, h->d_p0, h->d_p1, h->d_q, h->d_dinv,
                  h->d_partials, h->d_partials2, h->d_pcg, h->d_misc, h->d_rho_phys,
                  h->d_E, h->d_dc, h->d_dc_phys, h->d_r32, h->d_z32, h->d_p0_32,
                  h->d_p1_32, h->d_q32, h->d_dinv32, h->d_e32, h->d_E32, h->d_pcg32,
                  h->d_btc, h->m_q64, h->m_r32, h->m_z32, h->m_p0, h->m_p1, h->m_q32,
                  h->m_e32, h->m_pcg, h->m_out, h->d_bar, h->d_rho_bar, h->d_rho_in, h->d_oc,
                  h->d_tile_fixed};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->h_pcg) cudaFreeHost(h->h_pcg);
  if (h->h_misc) cudaFreeHost(h->h_misc);
  if (h->h_pcg32) cudaFreeHost(h->h_pcg32);
  if (h->h_mpcg) cudaFreeHost(h->h_mpcg);
  if (h->ev.cg_start) cudaEventDestroy(h->ev.cg_start);
  if (h->ev.cg_stop) cudaEventDestroy(h->ev.cg_stop);
  for (size_t i = 0; i < h->ev.start.size(); ++i) {
    cudaEventDestroy(h->ev.start[i]);
    cudaEventDestroy(h->ev.stop[i]);
  }
  delete h;
}

mfto_status filter_rowsums(mfto_handle* h);  // filter.cu

// Mode-space coefficients of the unit element operator (kv_tile.cuh): the
// diagonal terms of mode_operator() and the off-diagonal couplings, with
// the 1/8 of the inverse transform folded in.
void mode_coefficients(double nu, double hh, ModeCoef<double>* c64, ModeCoef<float>* c32) {
  const ModeOperator op = mode_operator(1.0, nu, hh);
  memset(c64, 0, sizeof(*c64));
  for (int t = 0; t < op.n_terms; ++t)
    if (op.out_comp[t] == op.in_comp[t] && op.out_mode[t] == op.in_mode[t])
      c64->diag[op.out_comp[t]][op.out_mode[t]] = op.coef[t] / 8.0;
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
  const double M[2] = {hh / 2.0, hh / 6.0};
  for (int t = 0; t < 2; ++t) {
    c64->lamM[t] = lam * M[t] / 8.0;
    c64->muM[t] = mu * M[t] / 8.0;
  }
  for (int c = 0; c < 3; ++c)
    for (int m = 0; m < 8; ++m) c32->diag[c][m] = (float)c64->diag[c][m];
  for (int t = 0; t < 2; ++t) {
    c32->lamM[t] = (float)c64->lamM[t];
    c32->muM[t] = (float)c64->muM[t];
  }
}

mfto_status filter_setup(mfto_handle* h);

static mfto_status upload_params(mfto_handle* h) {
  double ke[576];
  float ke32[576];
  mfto_unit_ke(1.0, h->p.nu, h->mesh.h, ke);
  for (int i = 0; i < 576; ++i) ke32[i] = (float)ke[i];
  h->ke_diag = ke[0];
  {
    mfto_status s = tc_upload_b(h, ke);
    if (s != MFTO_OK) return s;
  }
  mode_coefficients(h->p.nu, h->mesh.h, &h->mc64, &h->mc32);
  MFTO_CUDA(h, cudaMemcpyAsync(h->d_ke64, ke, sizeof(ke), cudaMemcpyHostToDevice, h->stream));
  MFTO_CUDA(h, cudaMemcpyAsync(h->d_ke32, ke32, sizeof(ke32), cudaMemcpyHostToDevice, h->stream));
  return filter_setup(h);
}

// Cone-filter stencil and row sums of the radius h->p.rmin.
mfto_status filter_setup(mfto_handle* h) {
  int32_t n = 0;
  mfto_filter_stencil(h->p.rmin, 0, nullptr, nullptr, &n);
  std::vector<int32_t> off(3 * n);
  std::vector<double> w(n);
  mfto_filter_stencil(h->p.rmin, n, off.data(), w.data(), &n);
  if (h->d_stencil_off) cudaFree(h->d_stencil_off);
  if (h->d_stencil_w) cudaFree(h->d_stencil_w);
  h->d_stencil_off = nullptr;
  h->d_stencil_w = nullptr;
  if (cudaMalloc(&h->d_stencil_off, sizeof(int32_t) * 3 * n) != cudaSuccess ||
      cudaMalloc(&h->d_stencil_w, sizeof(double) * n) != cudaSuccess)
    return mfto_fail(h, MFTO_OOM, "cudaMalloc of the filter stencil failed");
  h->n_stencil = n;
  MFTO_CUDA(h, cudaMemcpyAsync(h->d_stencil_off, off.data(), sizeof(int32_t) * 3 * n,
                               cudaMemcpyHostToDevice, h->stream));
  MFTO_CUDA(h, cudaMemcpyAsync(h->d_stencil_w, w.data(), sizeof(double) * n,
                               cudaMemcpyHostToDevice, h->stream));
  mfto_status s = filter_rowsums(h);
  if (s != MFTO_OK) return s;
  MFTO_CUDA(h, cudaStreamSynchronize(h->stream));
  return MFTO_OK;
}

extern "C" mfto_status mfto_create(const mfto_mesh* mesh, const mfto_params* params,
                                   const uint8_t* h_fixed, void* stream,
                                   mfto_handle** out) {
  if (!out) return MFTO_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !params || !h_fixed) return MFTO_INVALID_ARG;
  if (mesh->nelx < 1 || mesh->nely < 1 || mesh->nelz < 1 || !(mesh->h > 0.0))
    return MFTO_INVALID_ARG;
  mfto_handle* h = new mfto_handle();
  memset(h->msg, 0, sizeof(h->msg));
  h->mesh = *mesh;
  h->stream = (cudaStream_t)stream;
  h->n_elem = (int64_t)mesh->nelx * mesh->nely * mesh->nelz;
  h->n_node = (int64_t)(mesh->nelx + 1) * (mesh->nely + 1) * (mesh->nelz + 1);
  h->n_dof = 3 * h->n_node;
  if (h->n_dof > (int64_t)INT32_MAX) { free_handle(h); return MFTO_INVALID_ARG; }
  if (check_params(h, params) != MFTO_OK) { free_handle(h); return MFTO_INVALID_ARG; }
  h->max_rhs = params->max_rhs;
  h->p = *params;
  h->solver_form = MFTO_FORM_F64;
  h->inner_tol = 1e-2;
  h->inner_maxit = 10000;
  h->max_outer = 50;
  h->proj_beta = 0.0;       // no projection unless asked (the plain path)
  h->proj_eta = 0.5;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    free_handle(h);
    return MFTO_CUDA_ERROR;
  }
  const size_t nd = sizeof(double) * h->n_dof, ne = sizeof(double) * h->n_elem;
  bool ok = true;
  auto A = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
    if (ok) h->ws_bytes += (int64_t)bytes;
  };
  A((void**)&h->d_ke64, sizeof(double) * 576);
  A((void**)&h->d_ke32, sizeof(float) * 576);
  // padded: the column K.v reads the mask as 32-bit words
  A((void**)&h->d_fixed, h->n_node + 16);
  A((void**)&h->d_filter_W, ne);
  A((void**)&h->d_r, nd);
  A((void**)&h->d_z, nd);
  A((void**)&h->d_p0, nd);
  A((void**)&h->d_p1, nd);
  A((void**)&h->d_q, nd);
  A((void**)&h->d_dinv, nd);
  A((void**)&h->d_partials, sizeof(double) * MFTO_RED_ROWS * MFTO_RED_SLOTS);
  A((void**)&h->d_partials2, sizeof(double) * MFTO_RED_ROWS * MFTO_RED_SLOTS);
  A((void**)&h->d_pcg, sizeof(PcgScalars));
  A((void**)&h->d_misc, sizeof(MiscScalars));
  A((void**)&h->d_rho_phys, ne);
  A((void**)&h->d_E, ne);
  A((void**)&h->d_dc, ne);
  A((void**)&h->d_dc_phys, ne);
  A((void**)&h->d_rho_bar, ne);
  A((void**)&h->d_rho_in, ne);
  A((void**)&h->d_oc, 3 * ne);        // OC bisection: a_e and the move-limit bounds
  const size_t nd32 = sizeof(float) * h->n_dof;
  A((void**)&h->d_r32, nd32);
  A((void**)&h->d_z32, nd32);
  A((void**)&h->d_p0_32, nd32);
  A((void**)&h->d_p1_32, nd32);
  A((void**)&h->d_q32, nd32);
  A((void**)&h->d_dinv32, nd32);
  A((void**)&h->d_e32, nd32);
  A((void**)&h->d_E32, sizeof(float) * h->n_elem);
  A((void**)&h->d_pcg32, sizeof(PcgScalars));
  A((void**)&h->d_btc, 3 * 2 * MFTO_TC_BTILE);
  if (h->max_rhs > 1) {
    const size_t m = (size_t)h->max_rhs;
    A((void**)&h->m_q64, m * nd);
    A((void**)&h->m_r32, m * nd32);
    A((void**)&h->m_z32, m * nd32);
    A((void**)&h->m_p0, m * nd32);
    A((void**)&h->m_p1, m * nd32);
    A((void**)&h->m_q32, m * nd32);
    A((void**)&h->m_e32, m * nd32);
    A((void**)&h->m_pcg, sizeof(MultiScalars));
    A((void**)&h->m_out, sizeof(double) * 2 * MFTO_MAX_RHS);
    if (ok && cudaMallocHost(&h->h_mpcg, sizeof(MultiScalars)) != cudaSuccess) ok = false;
  }
  if (ok && (cudaMallocHost(&h->h_pcg, sizeof(PcgScalars)) != cudaSuccess ||
             cudaMallocHost(&h->h_misc, sizeof(MiscScalars)) != cudaSuccess ||
             cudaMallocHost(&h->h_pcg32, sizeof(PcgScalars)) != cudaSuccess))
    ok = false;
  // column K.v tiles (kv_column.cuh) that stage no fixed node: any z, the
  // tile's node range x0 .. x0 + CX, y0 .. y0 + CY with x0 = OX bx - 1,
  // y0 = OY by - 1
  const int ntx = (int)((h->mesh.nelx + 1 + ColShape::OX - 1) / ColShape::OX);
  const int nty = (int)((h->mesh.nely + 1 + ColShape::OY - 1) / ColShape::OY);
  std::vector<uint8_t> tile_fixed((size_t)ntx * nty, 0);
  {
    const int nx = h->mesh.nelx + 1, ny = h->mesh.nely + 1, nz = h->mesh.nelz + 1;
    std::vector<uint8_t> colfix((size_t)nx * ny, 0);
    for (int64_t n = 0; n < h->n_node; ++n)
      if (h_fixed[n]) colfix[n % ((int64_t)nx * ny)] = 1;
    (void)nz;
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if (!colfix[(size_t)i + (size_t)nx * j]) continue;
        for (int by = 0; by < nty; ++by) {
          const int y0 = ColShape::OY * by - 1;
          if (j < y0 || j > y0 + ColShape::CY) continue;
          for (int bx = 0; bx < ntx; ++bx) {
            const int x0 = ColShape::OX * bx - 1;
            if (i >= x0 && i <= x0 + ColShape::CX) tile_fixed[(size_t)bx + (size_t)ntx * by] = 1;
          }
        }
      }
  }
  A((void**)&h->d_tile_fixed, tile_fixed.size());
  if (!ok) {
    cudaGetLastError();
    free_handle(h);
    return MFTO_OOM;
  }
  if (cudaMemcpy(h->d_tile_fixed, tile_fixed.data(), tile_fixed.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpyAsync(h->d_fixed, h_fixed, h->n_node, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_pcg, 0, sizeof(PcgScalars), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_misc, 0, sizeof(MiscScalars), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_pcg32, 0, sizeof(PcgScalars), h->stream) != cudaSuccess ||
      (h->m_pcg && cudaMemsetAsync(h->m_pcg, 0, sizeof(MultiScalars), h->stream) != cudaSuccess)) {
    free_handle(h);
    return MFTO_CUDA_ERROR;
  }
  mfto_status s = kv_tile_init(h);
  if (s == MFTO_OK) s = pcg_persist_init(h);
  if (s == MFTO_OK) s = cg2_attrs(h);
  if (s == MFTO_OK) h->cg_engine = 2;
  if (s == MFTO_OK) s = tc_init(h);
  if (s == MFTO_OK) s = multi_init(h);
  if (s == MFTO_OK) s = upload_params(h);
  if (s != MFTO_OK) { free_handle(h); return s; }
  *out = h;
  return MFTO_OK;
}

extern "C" mfto_status mfto_destroy(mfto_handle* h) {
  if (!h) return MFTO_INVALID_ARG;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
  return MFTO_OK;
}

extern "C" mfto_status mfto_set_params(mfto_handle* h, const mfto_params* p) {
  if (!h) return MFTO_INVALID_ARG;
  mfto_status s = check_params(h, p);
  if (s != MFTO_OK) return s;
  MFTO_REQUIRE(h, p->max_rhs == h->max_rhs, "mfto_set_params: max_rhs is fixed at mfto_create");
  h->p = *p;
  return upload_params(h);
}

extern "C" const char* mfto_last_error(const mfto_handle* h) {
  return h ? h->msg : "null handle";
}

extern "C" mfto_status mfto_sizes(const mfto_handle* h, int64_t* ne, int64_t* nn,
                                  int64_t* nd) {
  if (!h) return MFTO_INVALID_ARG;
  if (ne) *ne = h->n_elem;
  if (nn) *nn = h->n_node;
  if (nd) *nd = h->n_dof;
  return MFTO_OK;
}

// ------------------------------------------------------------ K.v timing
static const int kEventPool = 4096;

void kv_timing_begin(mfto_handle* h, int form) {
  if (!h->kv_timing) return;
  if (h->ev.used >= kEventPool) kv_timing_harvest(h, true);
  if ((int)h->ev.start.size() <= h->ev.used) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    h->ev.start.push_back(a);
    h->ev.stop.push_back(b);
    h->ev.form.push_back(0);
  }
  h->ev.form[h->ev.used] = form == MFTO_FORM_F64 ? 0 : 1;
  cudaEventRecord(h->ev.start[h->ev.used], h->stream);
}

void kv_timing_end(mfto_handle* h) {
  if (!h->kv_timing) return;
  cudaEventRecord(h->ev.stop[h->ev.used], h->stream);
  h->ev.used++;
}

mfto_status kv_timing_harvest(mfto_handle* h, bool sync) {
  if (h->ev.used == 0) return MFTO_OK;
  if (sync) MFTO_CUDA(h, cudaEventSynchronize(h->ev.stop[h->ev.used - 1]));
  for (int i = 0; i < h->ev.used; ++i) {
    float ms = 0.f;
    MFTO_CUDA(h, cudaEventElapsedTime(&ms, h->ev.start[i], h->ev.stop[i]));
    h->ev.total_ms[h->ev.form[i]] += ms;
    h->ev.launches[h->ev.form[i]]++;
  }
  h->ev.used = 0;
  return MFTO_OK;
}

extern "C" mfto_status mfto_kv_timing(mfto_handle* h, int32_t on) {
  if (!h) return MFTO_INVALID_ARG;
  mfto_status s = kv_timing_harvest(h, true);
  h->kv_timing = on != 0;
  return s;
}

extern "C" mfto_status mfto_launch_count(const mfto_handle* h, int64_t* n) {
  if (!h || !n) return MFTO_INVALID_ARG;
  *n = h->launches;
  return MFTO_OK;
}

extern "C" mfto_status mfto_kv_timing_read(mfto_handle* h, mfto_form form, int64_t* launches,
                                           double* total_ms) {
  if (!h) return MFTO_INVALID_ARG;
  MFTO_REQUIRE(h, form == MFTO_FORM_F64 || form == MFTO_FORM_F32,
               "mfto_kv_timing_read: form must be F64 or F32");
  mfto_status s = kv_timing_harvest(h, true);
  const int f = form == MFTO_FORM_F64 ? 0 : 1;
  if (launches) *launches = h->ev.launches[f];
  if (total_ms) *total_ms = h->ev.total_ms[f];
  h->ev.launches[f] = 0;
  h->ev.total_ms[f] = 0.0;
  return s;
}

extern "C" mfto_status mfto_device_bytes(const mfto_handle* h, int64_t* bytes) {
  if (!h || !bytes) return MFTO_INVALID_ARG;
  int64_t b = h->ws_bytes;
  b += (int64_t)h->n_stencil * (int64_t)(3 * sizeof(int32_t) + sizeof(double));
  if (h->d_bar) b += 128;                       // the persistent CG's barrier line
  b += learned_bytes(h) + gmg_bytes(h);
  *bytes = b;
  return MFTO_OK;
}

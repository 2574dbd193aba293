/*
 * mfto -- matrix-free 3D SIMP topology optimisation on one GB300 (sm_103a).
 *
 * C ABI of the library libmfto.so.  Plain pointers and sizes only.
 *
 * Method (arXiv 2604.18020, "Matrix-Free 3D SIMP Topology Optimization with
 * Fused Gather-GEMM-Scatter Kernels"):
 *   minimise f^T u  s.t.  K(rho) u = f,  mean(rho) = V_f          (Eq. tomin)
 *   K(rho) = sum_e B_e^T E(rho_phys_e) KE B_e                       (Eq. simp)
 *   E(r)   = Emin + (E0 - Emin) r^p
 * with KE the 24x24 unit-modulus stiffness of a trilinear 8-node hexahedron on
 * a structured nelx x nely x nelz grid, K.v applied matrix-free
 * (Eq. matfree, Sec. 3.2-3.3), Jacobi-PCG (Sec. 3.6), cone density filter,
 * analytic sensitivities and OC bisection (Sec. 3.1).
 *
 * Conventions (the paper fixes none of them):
 *   element e = i + nelx*(j + nely*k), i fastest; element edge h (mfto_mesh.h);
 *   node    n = i + (nelx+1)*(j + (nely+1)*k);  DOF = 3*n + c, c = x, y, z;
 *   local node l = a + 2b + 4c for the element corner (i+a, j+b, k+c),
 *   local DOF 3*l + c (the row/column order of mfto_unit_ke);
 *   element fields (rho, E, dc) are [nelz][nely][nelx]; DOF vectors are
 *   [nelz+1][nely+1][nelx+1][3] (node-major, components interleaved).
 *   Fixed DOFs are given by a per-node uint8 mask, bit c set when DOF c is
 *   clamped.  The operator is the masked K:  (Kv)_free = (K P v)_free with P
 *   zeroing fixed DOFs, and (Kv)_fixed = v_fixed; so it is SPD and its Jacobi
 *   diagonal is 1 on fixed DOFs.  Loads f must be zero on fixed DOFs.
 *
 * Memory and streams: every array argument named d_* is a DEVICE pointer
 * owned by the caller (the library never frees it); h_* is a HOST pointer.
 * All device work is enqueued on the stream given at mfto_create; calls that
 * return host scalars synchronise that stream before returning.  Arguments
 * must not alias unless a function says so.
 *
 * Device allocations by the library (everything is freed by the matching
 * destroy call): mfto_create (the handle's workspace and the filter
 * stencil); mfto_set_params and mfto_simp_protocol when the filter radius
 * changes (the stencil is made again); mfto_gmg_setup, and the multigrid
 * solves and SIMP steps that build a hierarchy on first use or when its
 * shape changes (levels, coarse inverse, sweep vectors); the learned-part
 * calls on a handle (mfto_nn_features, mfto_nn_target, mfto_nn_to_dofs,
 * mfto_nn_sample, mfto_set_learned, mfto_nn_train_energy) on first use of a
 * grid depth; and the constructors of the separate objects, mfto_batch_create,
 * mfto_ebe_create and mfto_nn_create.  Every other call works in memory that
 * already exists.  There is no separate workspace-size query: a handle's
 * whole device footprint, workspace and optional parts included, is reported
 * by mfto_device_bytes.  mfto_compliance_sens_noalloc allocates nothing.
 *
 * Errors: every function returns an mfto_status; nothing is thrown across the
 * ABI.  On an error the handle's message is available from mfto_last_error.
 * A CUDA error inside a call is reported as MFTO_CUDA_ERROR and leaves the
 * handle usable only if the CUDA context is.
 */
#ifndef MFTO_H
#define MFTO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mfto_status;
enum {
  MFTO_OK = 0,
  MFTO_INVALID_ARG = 1,     /* null pointer, bad size or unknown enum     */
  MFTO_CUDA_ERROR = 2,      /* a CUDA runtime call or launch failed       */
  MFTO_OOM = 3,             /* cudaMalloc of the workspace failed         */
  MFTO_NOT_CONVERGED = 4,   /* iteration cap reached before the tolerance */
  MFTO_STALLED = 5,         /* residual stopped decreasing (IR / FPCG)    */
  MFTO_BREAKDOWN = 6,       /* NaN/Inf or non-positive curvature in CG    */
  MFTO_UNSUPPORTED = 7,     /* form or feature not available             */
  MFTO_TOO_LARGE = 8        /* problem exceeds a fixed capacity          */
};

/* Arithmetic forms of the K.v contraction (Eq. matfree; the mixed-precision
 * forms of Sec. 3.5).  F64 and F32 run on the FMA pipes; the others keep FP32
 * vectors and moduli, put the element contraction on the tcgen05 tensor cores
 * with FP32 accumulation, and round the operands to the form's type first.
 * The X3 forms split each operand x into hi = round(x) and lo = round(x - hi)
 * and add the products of the lo parts to A_hi B_hi (three products).
 * TF32 forms: A = the element's nodal values (split TF32: minus a
 * translation common to the tile of 30 x 7 owned nodes that contains it; KE
 * annihilates translations, so the product is unchanged and its rounding
 * scales with the deformation, not the rigid motion), the modulus applied to
 * the product.
 * BF16 and FP16 forms: A = E_e u_e; FP16 scales each element's row by a
 * power of two into [1, 2) to stay in range. */
typedef enum {
  MFTO_FORM_F64 = 0,        /* FP64 data, FP64 arithmetic                 */
  MFTO_FORM_F32 = 1,        /* FP32 data, FP32 arithmetic                 */
  MFTO_FORM_TF32 = 2,       /* tensor cores, TF32 operands                */
  MFTO_FORM_TF32X3 = 3,     /* tensor cores, split TF32 (3 products)      */
  MFTO_FORM_BF16 = 4,       /* tensor cores, BF16 operands                */
  MFTO_FORM_BF16X3 = 5,     /* tensor cores, split BF16 (3 products)      */
  MFTO_FORM_F16 = 6,        /* tensor cores, FP16 operands (row-scaled)   */
  MFTO_FORM_F16X3 = 7       /* tensor cores, split FP16 (3 products)      */
} mfto_form;

typedef struct {
  int32_t nelx, nely, nelz; /* elements per axis, each >= 1               */
  double h;                 /* element edge length (> 0)                  */
} mfto_mesh;

typedef struct {
  double E0;                /* solid modulus                              */
  double Emin;              /* void modulus (Eq. simp: rho_min)           */
  double nu;                /* Poisson ratio, in (-1, 0.5)                */
  double penal;             /* SIMP penalty p                             */
  double rmin;              /* cone filter radius (elements), > 0         */
  double volfrac;           /* target mean design density V_f             */
  double move;              /* OC move limit m                            */
  double rtol;              /* PCG stop: ||r|| <= rtol ||f||              */
  int32_t maxit;            /* PCG iteration cap                          */
  int32_t check_every;      /* PCG: host polls convergence every k iters  */
  int32_t max_rhs;          /* load cases of the multi-RHS calls, 1..8    */
} mfto_params;

typedef struct {
  int32_t iterations;       /* CG iterations performed                    */
  int32_t status;           /* MFTO_OK, MFTO_NOT_CONVERGED, MFTO_BREAKDOWN */
  double rel_residual;      /* recursive ||r|| / ||f|| at exit            */
  double fnorm;             /* ||f||                                      */
} mfto_solve_stats;

typedef struct {
  double compliance;        /* c = sum_e E_e u_e^T KE u_e                 */
  double change;            /* max |rho_new - rho|                        */
  double volume;            /* mean(rho_new)                              */
  double grayness;          /* (4/n) sum rho_phys (1 - rho_phys)          */
  double lambda;            /* OC multiplier at exit of the bisection     */
  int32_t cg_iterations;
  int32_t cg_status;
  double rel_residual;
} mfto_iter_stats;

typedef struct {
  int32_t outer_iterations; /* FP64 residual evaluations that led to a correction */
  int32_t inner_iterations; /* CG iterations of all inner solves               */
  int32_t status;           /* MFTO_OK, MFTO_NOT_CONVERGED, MFTO_STALLED,       */
                            /* MFTO_BREAKDOWN                                   */
  int32_t kv_f64;           /* FP64 K.v applications (outer residuals)          */
  double rel_residual;      /* true FP64 ||f - K u|| / ||f|| at exit            */
  double fnorm;             /* ||f||                                            */
  double history[64];       /* rel. residual before each outer step (first 64)  */
} mfto_ir_stats;

typedef struct mfto_handle mfto_handle;

/* Library version string (static storage). */
const char* mfto_version(void);

/* Default parameters: E0=1, Emin=1e-9, nu=0.3, p=3, rmin=1.5, V_f=0.3,
 * move=0.2, rtol=1e-8, maxit=10000, check_every=32, max_rhs=1. */
void mfto_default_params(mfto_params* p);

/* ---------------------------------------------------------------- host -- */

/* Unit element stiffness KE (24x24, row-major, local DOF order above) of the
 * trilinear hexahedron with edge h, modulus E0 and Poisson ratio nu, from the
 * exact integrals of the linear shape functions (Sec. 3.1: KE is the
 * unit-modulus element matrix of Eq. simp).  h_ke_out: 576 doubles. */
mfto_status mfto_unit_ke(double E0, double nu, double h, double* h_ke_out);

/* The element -> DOF table of Sec. 3.2 (edof), [n_elem][24] int32, host.
 * The device kernels never read it (they compute DOFs from (i, j, k)); it is
 * exported so the indexing can be checked exactly. */
mfto_status mfto_edof(const mfto_mesh* mesh, int32_t* h_edof_out);

/* Cone-filter stencil (Sec. 3.1): every offset (dx, dy, dz) with
 * |d|_inf <= ceil(rmin) - 1 and weight w = rmin - |d| > 0, in dz, dy, dx
 * ascending order (dx fastest).  h_offsets: 3*cap int32; h_weights: cap
 * doubles; *count receives the number of offsets (<= cap or
 * MFTO_INVALID_ARG). */
mfto_status mfto_filter_stencil(double rmin, int32_t cap, int32_t* h_offsets,
                                double* h_weights, int32_t* count);

/* -------------------------------------------------------------- handle -- */

/* Create a handle for one mesh.  h_fixed: per-node uint8 mask
 * ([n_node], copied to the device).  stream: a cudaStream_t (0 = legacy
 * default stream) on which every later call enqueues its work.  Allocates the
 * device workspace (PCG vectors and reduction buffers, about 12 FP64 DOF
 * vectors); returns MFTO_OOM if that fails. */
mfto_status mfto_create(const mfto_mesh* mesh, const mfto_params* params,
                        const uint8_t* h_fixed, void* stream,
                        mfto_handle** out);
mfto_status mfto_destroy(mfto_handle* h);
/* Replace the parameters (mesh and fixed set stay). */
mfto_status mfto_set_params(mfto_handle* h, const mfto_params* params);
/* Message of the last failing call on this handle (static per handle). */
const char* mfto_last_error(const mfto_handle* h);
/* Sizes of the mesh: elements, nodes, DOFs. */
mfto_status mfto_sizes(const mfto_handle* h, int64_t* n_elem, int64_t* n_node,
                       int64_t* n_dof);
/* Device memory this handle holds now, in bytes: the workspace of
 * mfto_create (vectors, reduction buffers, scalars, element matrices), the
 * filter stencil, and what optional parts allocated on first use (the
 * multigrid hierarchy, the learned solve's buffers); the caller's arrays are
 * not counted.  For VRAM reports (the paper's memory snapshots). */
mfto_status mfto_device_bytes(const mfto_handle* h, int64_t* bytes);

/* -------------------------------------------------------- device steps -- */

/* SIMP modulus (Eq. simp): d_E[e] = Emin + (E0 - Emin) d_rho_phys[e]^p.
 * FP64 in, FP64 out (form F64) or FP64 in, FP32 out (form F32). */
mfto_status mfto_simp_modulus(mfto_handle* h, mfto_form form,
                              const double* d_rho_phys, void* d_E);

/* Masked matrix-free K.v (Eq. matfree; Alg. 1 computes the same sum):
 * d_y = K(E) d_v.  d_E, d_v, d_y are double for MFTO_FORM_F64 and float for
 * every other form.  d_y must not alias d_v.  A tensor-core form whose
 * completion wait times out sets the handle's device error flag (reported
 * by the next synchronising call) instead of hanging. */
mfto_status mfto_kv(mfto_handle* h, mfto_form form, const void* d_E,
                    const void* d_v, void* d_y);

/* Choose the K.v kernel used by mfto_kv, mfto_pcg and mfto_simp_step:
 * 0 (default) = element operator in the per-axis (sum, difference) mode
 * basis, about 220 arithmetic operations per element; FP64 runs node-owned
 * tiles streaming along z through a shared-memory ring, FP32 runs one
 * z-column of elements per thread with the face transforms carried from
 * layer to layer (about 170 operations per element); 1 = one thread per node
 * gathering its 8 elements with the dense 24x24 KE from shared memory (576
 * multiply-adds per node, the operation count of Alg. 1); 2 = as 0 for FP64,
 * and for FP32 one element per thread over 8 x 8 x 4 element blocks that own
 * their 7 x 7 x 3 interior nodes.  All are atomic-free and bit-reproducible. */
mfto_status mfto_set_kv_variant(mfto_handle* h, int32_t variant);

/* Choose how the FP32 inner Jacobi-PCG of the mixed solve (mfto_ir_solve and
 * mfto_simp_step with an F32 inner form) runs its iterations (Sec. 3.6):
 * 0 = two kernels per iteration (K.v, vector update) replayed
 * from a captured CUDA graph; 1 = one persistent cooperative kernel per
 * inner solve: each iteration's K.v with the direction update, the vector
 * update and both dot products run between two bounded grid barriers, every
 * CTA reducing the per-CTA partials in the same order; 2 (default) = two kernels per
 * iteration from a captured graph like 0, without grid-wide tickets: each
 * kernel sums the per-block partials of the dot products it needs (r.z and
 * r.r in the K.v's pre-step, p.q before the vector update) while its first
 * loads are in flight, every block in the same fixed order.  All compute the
 * same per-entry arithmetic; the dot products add the per-block partials in
 * different orders.  The TF32 and split-TF32 inner forms run 0 or 2 (1 acts
 * as 0 for them); the BF16 and FP16 forms and mfto_set_kv_variant(h, 1)
 * always use 0.
 * MFTO_UNSUPPORTED for 1 without cooperative launch.  A barrier wait that
 * gives up (about a second) makes the solve return MFTO_CUDA_ERROR. */
mfto_status mfto_set_cg_engine(mfto_handle* h, int32_t engine);

/* Autotune the FP32 K.v (variant 0): times the column kernel for every
 * distinct length ceil(nz / t), t = 1 .. 64, of its z-chunks (node layers per
 * CTA tile; longer chunks recompute fewer element layers, shorter ones give
 * more CTAs, and the chunk count sets how evenly the tiles fill the resident
 * CTAs) and each kernel kind
 * (register allocation held to 2 (kind 0) or 3 (kind 1) resident CTAs per
 * SM) on the handle's own work vectors, and keeps the fastest pair for
 * mfto_kv and the FP32 inner CG.  With the graph CG engines (0, 2) the timed
 * unit is one inner CG iteration (the CG K.v with its vector update, from the
 * captured graph), otherwise one plain K.v.  All shapes give bit-identical K.v
 * results.  Returns the chosen chunk length, kind and the time of the timed
 * unit in microseconds (any may be NULL).  Overwrites the handle's FP32 work
 * vectors; synchronises the stream.  Call it after mfto_set_cg_engine. */
mfto_status mfto_kv_autotune(mfto_handle* h, int32_t* nzc, int32_t* kind, float* us);
/* Set the FP32 column K.v's launch shape by hand: z-chunk length nzc (0:
 * automatic) and kernel kind 0 or 1 (as in mfto_kv_autotune). */
mfto_status mfto_set_kv_shape(mfto_handle* h, int32_t nzc, int32_t kind);

/* Jacobi diagonal of the masked K (Sec. 3.6), one element pass:
 * d_diag[k] = sum_{e owning k} E_e KE[l, l], 1 on fixed DOFs. */
mfto_status mfto_jacobi_diag(mfto_handle* h, mfto_form form, const void* d_E,
                             void* d_diag);

/* Jacobi-PCG in FP64 (Sec. 3.6) on K(E) u = f with warm start: d_u holds the
 * initial guess on entry and the solution on exit.  Stops at
 * ||r|| <= rtol ||f|| (recursive residual) or maxit.  Returns MFTO_OK also
 * when the cap is hit; the outcome is in st->status. */
mfto_status mfto_pcg(mfto_handle* h, const double* d_E, const double* d_f,
                     double* d_u, mfto_solve_stats* st);

/* Mixed-precision solve of K(E) u = f: FP64 iterative refinement (Sec. 3.5's
 * residual correction, with the outer loop in FP64) around an inner
 * Jacobi-PCG in a lower precision:
 *   r = f - K u in FP64 (FP64 K.v);  stop if ||r|| <= rtol ||f||;
 *   solve K e = r approximately with the inner PCG (inner form K.v, FP32
 *   vectors, FP64 dot products) to ||r_e|| <= inner_tol ||r||, from e = 0;
 *   u += e in FP64.
 * d_E and d_f FP64; d_u FP64, initial guess on entry, solution on exit.
 * Stops with MFTO_STALLED when the outer residual fails twice in a row to fall
 * below 0.9 of its previous value (the stagnation the paper reports for BF16),
 * MFTO_NOT_CONVERGED after max_outer corrections (mfto_set_solver).
 * inner: any form but MFTO_FORM_F64 (the inner K.v form).  Returns MFTO_OK
 * also when not converged; see st->status.  Synchronises the stream. */
mfto_status mfto_ir_solve(mfto_handle* h, mfto_form inner, double inner_tol,
                          const double* d_E, const double* d_f, double* d_u,
                          mfto_ir_stats* st);

/* How the inner Jacobi-PCG of mfto_ir_solve (and of mfto_simp_step with a
 * mixed solver) starts at each outer step:
 *   MFTO_IR_RESTART (default): from e = 0 with the direction p = z, the
 *     residual correction of Sec. 3.5 as written (each inner solve is a new
 *     Krylov process);
 *   MFTO_IR_CONTINUE: from e = 0 on the new FP64 residual, but keeping the
 *     last search direction: the first direction is z + (rho / rho_prev) p
 *     with rho_prev the r.z that formed p.  This is reliable updating
 *     (residual replacement): one Krylov process whose FP32 recursive
 *     residual is replaced by the true FP64 residual whenever it has fallen by
 *     inner_tol, so the inner iterations add up to about those of one long CG
 *     instead of restarting the superlinear phase at every outer step.
 * Outer residual, accumulation, stopping and stall rules are the same. */
enum { MFTO_IR_RESTART = 0, MFTO_IR_CONTINUE = 1 };
mfto_status mfto_set_ir_mode(mfto_handle* h, int32_t mode);

/* Several load cases at once (multi-RHS).  V and Y hold nrhs DOF vectors
 * one after the other ([nrhs][n_dof]); every case uses the same moduli and
 * fixed set.  mfto_kv_multi: Y_r = K(E) V_r for r < nrhs (1..8), one launch,
 * forms MFTO_FORM_F64 (double) and MFTO_FORM_F32 (float).  The paper treats
 * one load case; this batches the operator it defines (Eq. matfree). */
mfto_status mfto_kv_multi(mfto_handle* h, mfto_form form, const void* d_E, const void* d_V,
                          void* d_Y, int32_t nrhs);

/* Mixed-precision solve of K(E) U_r = F_r for nrhs load cases (nrhs <=
 * max_rhs of mfto_create): the refinement of mfto_ir_solve for every case
 * (FP64 residuals, norms and accumulation), around one inner FP32 CG that
 * advances all live cases together (one launch of the K.v for all cases and
 * one vector update per iteration, a grid row per case, per-case scalars and
 * stopping; mfto_set_ir_mode applies per case).  d_E FP64 [n_elem];
 * d_F, d_U FP64 [nrhs][n_dof] (d_U: initial guesses in, solutions out);
 * st: nrhs entries.  Synchronises the stream. */
mfto_status mfto_ir_solve_multi(mfto_handle* h, double inner_tol, const double* d_E,
                                const double* d_F, double* d_U, int32_t nrhs,
                                mfto_ir_stats* st);

/* ------------------------------------------------------------- batches -- */

/* Many independent problems of uneven size solved together: every step is
 * one persistent launch over all instances (a work list of (instance,
 * element block) items), the inner CG chunks are captured in one CUDA graph,
 * and per-instance sums are reduced deterministically.  The paper solves
 * one problem at a time; a batch applies its operator (Eq. matfree) and its
 * solver (Sec. 3.6, refined as in mfto_ir_solve) to each instance.
 *
 * mfto_batch_create: count (1..256) meshes with the same element edge h,
 * shared parameters (E0, Emin, nu, rtol, maxit, check_every are used),
 * h_fixed: the instances' per-node masks concatenated in instance order.
 * Arrays passed to the batch calls concatenate the instances' arrays in the
 * same order; mfto_batch_layout returns the offsets (count + 1 entries each,
 * elements and DOFs). */
typedef struct mfto_batch mfto_batch;
mfto_status mfto_batch_create(int32_t count, const mfto_mesh* meshes, const mfto_params* params,
                              const uint8_t* h_fixed, void* stream, mfto_batch** out);
mfto_status mfto_batch_destroy(mfto_batch* b);
const char* mfto_batch_last_error(const mfto_batch* b);
mfto_status mfto_batch_layout(const mfto_batch* b, int64_t* h_elem_off, int64_t* h_dof_off);
/* d_Y = K(E) d_V for every instance, one launch (forms F64, F32). */
mfto_status mfto_batch_kv(mfto_batch* b, mfto_form form, const void* d_E, const void* d_V,
                          void* d_Y);
/* Element-block shape of the batch kernels (8x8x4, 8x4x8, 4x8x8, 16x4x4
 * elements = 0..3): mfto_batch_autotune times an FP32 K.V of the batch
 * `reps` times per shape (CUDA events), keeps the fastest, and reports the
 * per-launch times in h_ms_out[4] (may be NULL) and the choice. */
mfto_status mfto_batch_autotune(mfto_batch* b, int32_t reps, double* h_ms_out, int32_t* chosen);
mfto_status mfto_batch_set_shape(mfto_batch* b, int32_t shape);
/* Mixed-precision solve of every instance (FP64 refinement per instance
 * around one FP32 inner CG over all live instances): d_E FP64 [elements],
 * d_F, d_U FP64 [DOFs] (d_U: initial guesses in, solutions out), st: count
 * entries.  Synchronises the stream. */
mfto_status mfto_batch_solve(mfto_batch* b, double inner_tol, const double* d_E, const double* d_F,
                             double* d_U, int32_t inner_maxit, int32_t max_outer,
                             mfto_ir_stats* st);
/* Kernels launched for this batch so far (graph kernel nodes included). */
mfto_status mfto_batch_launch_count(const mfto_batch* b, int64_t* n);
/* Refinement mode of mfto_batch_solve, per instance as in mfto_set_ir_mode:
 * MFTO_IR_RESTART (default, every correction restarts with p = z) or
 * MFTO_IR_CONTINUE (each instance's inner CG continues its previous search
 * direction with beta = r.z / (r.z)_prev).  MFTO_INVALID_ARG otherwise. */
mfto_status mfto_batch_set_ir_mode(mfto_batch* b, int32_t mode);

/* Select the linear solver of mfto_simp_step: form MFTO_FORM_F64 = plain FP64
 * Jacobi-PCG (default); any other form = mfto_ir_solve with that inner form,
 * inner tolerance inner_tol (> 0, < 1), inner iteration cap inner_maxit and
 * at most max_outer corrections. */
mfto_status mfto_set_solver(mfto_handle* h, mfto_form form, double inner_tol,
                            int32_t inner_maxit, int32_t max_outer);

/* Cone density filter (Sec. 3.1): transpose = 0 gives
 * d_y = (H d_x) / W;  transpose = 1 gives d_y = H (d_x / W)
 * (the chain rule for sensitivities).  FP64, element fields. */
mfto_status mfto_filter(mfto_handle* h, const double* d_x, double* d_y,
                        int32_t transpose);

/* Compliance and sensitivity (Sec. 3.1): ce_e = u_e^T KE u_e,
 * *c_out = sum_e E_e ce_e (FP64, fixed reduction order),
 * d_dc[e] = -p rho_phys_e^(p-1) (E0 - Emin) ce_e  (derivative with respect
 * to rho_phys; chain through mfto_filter(transpose=1) for the design field).
 * d_dc may be NULL.  Synchronises the stream. */
mfto_status mfto_compliance_sens(mfto_handle* h, const double* d_rho_phys,
                                 const double* d_u, double* c_out,
                                 double* d_dc);

/* OC update with bisection on the volume multiplier (Sec. 3.1):
 * B_e = max(0, -dc_e) / (lambda / n); candidate rho sqrt(B_e) clipped to
 * [max(0, rho - m), min(1, rho + m)]; lambda bisected on [0, 1e9] while
 * sum(rho_new) > V_f n raises the lower end, until
 * (l2 - l1)/(l1 + l2) <= 1e-10, or until the midpoint no longer lies strictly
 * inside the bracket (lambda underflow), or 4096 steps.  d_rho_new receives
 * the candidate of the last midpoint.  Synchronises the stream; st may be NULL. */
mfto_status mfto_oc_update(mfto_handle* h, const double* d_rho,
                           const double* d_dc, double* d_rho_new,
                           mfto_iter_stats* st);

/* One SIMP iteration (the loop of Sec. 3.1 / 3.7): rho_phys = filter(rho)
 * (then the Heaviside projection when mfto_set_projection turned it on);
 * E = E(rho_phys); Jacobi-PCG on K(E) u = f warm-started from d_u;
 * compliance and sensitivities (through the projection's derivative when
 * on); filter transpose; OC.  d_rho is updated in place, d_u holds the new
 * displacement, d_rho_phys (may be NULL) receives the physical field used in
 * this iteration. */
mfto_status mfto_simp_step(mfto_handle* h, double* d_rho, double* d_u,
                           const double* d_f, double* d_rho_phys,
                           mfto_iter_stats* st);

/* ------------------------------------------------------- learned part -- */

/* The paper has no learned component; this part adds one on top of its
 * solver (Sec. 3.5 refinement, Sec. 3.6 Jacobi-PCG).
 *
 * Network: a 3D convolutional U-Net on the node grid, padded with zeros to a
 * multiple of 2^(levels-1) per axis.  Tensors are FP32 [channels][D][H][W]
 * with D along z (nodes k), H along y (j), W along x (i).  levels - 1
 * encoder levels of two 3x3x3 convolutions + ReLU with base 2^l channels,
 * 2x2x2 average pooling between them, a bottleneck of base 2^(levels-1)
 * channels, decoder levels with nearest upsampling and channel
 * concatenation [upsampled, encoder output], two 3x3x3 convolutions + ReLU,
 * and a 1x1x1 output convolution: 4 input channels (node density, load x, y,
 * z), 3 output channels (displacement direction).  Zero padding at the grid
 * boundary.  Parameters are one FP32 vector, layer by layer in that order,
 * each layer's weights [c_out][c_in][kz][ky][kx] then its biases; the
 * convolutions compute with a BF16 copy of the weights (FP32 activations and
 * accumulation), Adam updates the FP32 master copy.  Reductions (weight and
 * bias gradients, loss) run in a fixed order: results are reproducible.
 *
 * mfto_nn_create: base 1..64 channels, levels 2..6, max_voxels: the largest
 * D*H*W that forward will see (activations are allocated for it),
 * max_train_voxels (<= max_voxels, 0 = inference only): the largest grid of
 * gradient / train_step; seed: He-normal initial weights, zero biases;
 * stream: cudaStream_t of all the network's work.  MFTO_OOM when the
 * buffers do not fit. */
typedef struct mfto_nn mfto_nn;
mfto_status mfto_nn_create(int32_t base, int32_t levels, int64_t max_voxels,
                           int64_t max_train_voxels, uint64_t seed, void* stream, mfto_nn** out);
mfto_status mfto_nn_destroy(mfto_nn* n);
const char* mfto_nn_last_error(const mfto_nn* n);
mfto_status mfto_nn_num_params(const mfto_nn* n, int64_t* count);
/* host copies of the FP32 parameter vector (set_params also resets Adam) */
mfto_status mfto_nn_get_params(mfto_nn* n, float* h_out);
mfto_status mfto_nn_set_params(mfto_nn* n, const float* h_in);
/* Where the 3x3x3 convolutions run: 1 (default) on the tcgen05 tensor cores
 * as implicit GEMMs (BF16 weights; FP32 activations split into BF16 hi + lo,
 * two products; FP32 accumulation in tensor memory), 0 on the FP32 FMA pipe.
 * The switch covers the forward pass and, for networks created with
 * max_train_voxels > 0, the data gradient of the backward pass (the adjoint
 * convolution: channel roles swapped, taps mirrored, the ReLU gate applied in
 * its epilogue); weight and bias gradients and the 1x1x1 head run on the FMA
 * pipe either way.  No paper counterpart (the learned part is this
 * library's). */
mfto_status mfto_nn_set_tensor_cores(mfto_nn* n, int32_t on);
/* *gave_up = 1 if a tensor-core convolution stopped waiting for its MMAs
 * (bounded wait, about a second; its output is then not to be used), else
 * 0.  Synchronises the network's stream. */
mfto_status mfto_nn_tc_status(mfto_nn* n, int32_t* gave_up);
/* d_out [3][D][H][W] = network(d_in [4][D][H][W]); D, H, W multiples of
 * 2^(levels-1); asynchronous.  MFTO_TOO_LARGE above max_voxels. */
mfto_status mfto_nn_forward(mfto_nn* n, int32_t D, int32_t H, int32_t W, const float* d_in,
                            float* d_out);
/* Masked mean squared error of the output against d_target [3][D][H][W]
 * (d_mask 1 where an entry counts, 0 elsewhere; the mean is over the
 * counted entries), its gradient with respect to every parameter (copied to
 * h_grad [num_params] when not NULL) and *loss.  Synchronises the stream. */
mfto_status mfto_nn_gradient(mfto_nn* n, int32_t D, int32_t H, int32_t W, const float* d_in,
                             const float* d_target, const float* d_mask, double* loss,
                             float* h_grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * gradient of mfto_nn_gradient; *loss (may be NULL: no synchronisation) is
 * the loss before the step. */
mfto_status mfto_nn_train_step(mfto_nn* n, int32_t D, int32_t H, int32_t W, const float* d_in,
                               const float* d_target, const float* d_mask, float lr,
                               double* loss);
mfto_status mfto_nn_launch_count(const mfto_nn* n, int64_t* count);

/* Padded network grid {D, H, W} of a mesh's nodes. */
mfto_status mfto_nn_grid(const mfto_mesh* m, int32_t levels, int32_t dims[3]);
/* Network input [4][D][H][W] of a (density, load) pair: channel 0 is the
 * mean rho_phys of the elements around each node, channels 1..3 the load
 * components divided by max |load|; zero on padding. */
mfto_status mfto_nn_features(mfto_handle* h, int32_t levels, const double* d_rho_phys,
                             const double* d_load, float* d_x_out);
/* Training target [3][D][H][W] = u / max |u| on the real nodes (zero on
 * padding) and mask [3][D][H][W] = 1 on the free DOFs of the real nodes. */
mfto_status mfto_nn_target(mfto_handle* h, int32_t levels, const double* d_u, float* d_y_out,
                           float* d_mask_out);
/* Network output [3][D][H][W] -> DOF vector (zero on fixed DOFs). */
mfto_status mfto_nn_to_dofs(mfto_handle* h, int32_t levels, const float* d_y, double* d_c_out);
/* One training sample from a solved state (E, rho_phys, f, u* = K^-1 f):
 * k_iters = 0 gives (features(rho_phys, f), target(u*)); k_iters > 0 runs
 * k_iters Jacobi-PCG iterations from zero to u_k and gives
 * (features(rho_phys, f - K u_k), target(u* - u_k)), the residual and error
 * of a partly converged solve. */
mfto_status mfto_nn_sample(mfto_handle* h, int32_t levels, const double* d_E,
                           const double* d_rho_phys, const double* d_f, const double* d_u_star,
                           int32_t k_iters, float* d_x_out, float* d_y_out, float* d_mask_out);

/* One Adam step (learning rate lr) of the network nn on the energy loss of
 * one state (E, rho_phys, f): with c = the network's displacement direction
 * for (rho_phys, f) on the DOFs (mfto_nn_to_dofs), a = f.c, b = c.Kc,
 *   loss = 1 - a^2 / (b * compliance),
 * the squared energy-norm error of the optimally scaled prediction
 * (a / b) c relative to the solution u* of K u* = f, whose compliance f.u*
 * the caller passes (> 0).  No displacement enters: the loss is minimal
 * (0) exactly when c is parallel to K^-1 f (the minimum of the potential
 * energy).  The gradient uses one FP64 K.v.  The network must have been
 * created with max_train_voxels >= the mesh's padded node grid.  *loss (may
 * be NULL: no synchronisation) is the loss before the step. */
mfto_status mfto_nn_train_energy(mfto_handle* h, mfto_nn* nn, const double* d_E,
                                 const double* d_rho_phys, const double* d_f, double compliance,
                                 float lr, double* loss);

typedef struct {
  int32_t outer_iterations;  /* FP64 refinement steps */
  int32_t inner_iterations;  /* FP32 flexible-PCG iterations */
  int32_t fp64_iterations;   /* FP64 Jacobi-PCG iterations of the last fallback */
  int32_t nn_calls;          /* network evaluations */
  int32_t fallback;          /* 0 none, 1 network switched off, 2 FP64 Jacobi-PCG */
  int32_t status;            /* MFTO_OK only at ||f - Ku|| / ||f|| <= rtol (FP64) */
  double rel_residual, fnorm;
  double nn_ms;              /* device time of the network evaluations */
  double history[64];        /* relative FP64 residual before each outer step */
} mfto_learned_stats;

/* Attach a network to the handle (NULL detaches): mfto_learned_solve and,
 * while attached, mfto_simp_step use it.  every = 0: the network supplies
 * the initial guess only (first iteration of the first inner solve);
 * every > 0: also the first direction of every later inner solve and a
 * correction at every every-th inner iteration.  MFTO_TOO_LARGE if the mesh's padded node grid
 * exceeds the network's max_voxels.  The network must outlive the
 * attachment. */
mfto_status mfto_set_learned(mfto_handle* h, mfto_nn* nn, int32_t every);
/* The learned solve: FP64 iterative refinement (outer residual f - Ku in
 * FP64) around an inner flexible PCG in FP32 (Polak-Ribiere beta) whose
 * preconditioner is Jacobi, replaced by the network's direction for
 * (rho_phys, r) at the correction iterations; the first correction with
 * u = 0 is the network's initial guess, energy-optimally scaled.  Inner
 * tolerance, caps and rtol come from mfto_set_solver and mfto_params.  When
 * two outer steps in a row reduce the residual by less than 10 % the
 * network is switched off; when that stalls too, FP64 Jacobi-PCG finishes
 * from the current iterate.  st->status is MFTO_OK only if the recomputed
 * FP64 residual meets rtol.  Synchronises the stream. */
mfto_status mfto_learned_solve(mfto_handle* h, const double* d_E, const double* d_rho_phys,
                               const double* d_f, double* d_u, mfto_learned_stats* st);

/* ---------------------------------- three-field SIMP, SIMP-120 protocol -- */

/* Smoothed Heaviside projection of the filtered field (Sec. 3.1):
 * rho_phys = (tanh(beta eta) + tanh(beta (rho_bar - eta))) /
 *            (tanh(beta eta) + tanh(beta (1 - eta))), clipped to [0, 1];
 * mfto_simp_step applies it after the filter and chains the sensitivities
 * through its derivative.  beta = 0 turns it off (the plain path, the
 * default); eta in (0, 1), the paper's 0.5. */
mfto_status mfto_set_projection(mfto_handle* h, double beta, double eta);
/* The projection alone (testing): d_rho_phys (may be NULL) = H(d_rho_bar);
 * d_dc (may be NULL) *= H'(d_rho_bar), in place.  MFTO_INVALID_ARG when the
 * projection is off. */
mfto_status mfto_project(mfto_handle* h, const double* d_rho_bar, double* d_rho_phys,
                         double* d_dc);

typedef struct {
  int32_t n_iter;           /* iterations (120; beyond, the last phase holds) */
  double rmin0;             /* filter radius of phase 1                       */
  double eta;               /* projection threshold (0.5)                     */
  double restart_factor;    /* restart when c > factor x selected c (1.12)    */
  double select_min_penal;  /* selectable iterates: p >= this (3.0) ...       */
  double select_max_gray;   /* ... and grayness < this (0.25)                 */
  int32_t cold_start;       /* 1: every solve starts from u = 0 (no warm start) */
} mfto_protocol_params;

typedef struct {
  int32_t iterations;       /* iterations run                                 */
  int32_t selected_iteration; /* 1-based; 0 when no iterate was selectable    */
  double selected_compliance;
  int32_t restarts;
  int32_t cg_iterations;    /* solver iterations of all steps                 */
} mfto_protocol_stats;

void mfto_default_protocol_params(mfto_protocol_params* p);

/* The benchmark protocol of Sec. 4.1 with mfto_simp_step and the handle's
 * solver: iteration i (1-based) runs with the phase values (p, beta, m) =
 * (1.5, 1, 0.20) for i <= 15, (3.5, 4, 0.15) for i <= 40, (4.5, 16, 0.08)
 * for i <= 65, (4.5, 32, 0.05) after; r_min = rmin0 in phase 1 and, in each
 * later phase, ramps linearly from the previous phase's end value to 1.35,
 * 1.25, 1.20, reached at the phase's last iteration.  The compliance of
 * iteration i belongs to the design entering it; when it exceeds
 * restart_factor times the selected compliance the next design is the
 * selected one (the displacement keeps its warm start); otherwise the OC
 * result.  The selected design is the lowest-compliance entering design
 * among iterates with p >= select_min_penal and grayness < select_max_gray.
 * d_rho: initial design in (the paper starts from V_f), final design out;
 * d_rho_selected: the selected design (unchanged if none).  Host arrays of
 * n_iter entries (each may be NULL): compliance, grayness, restarted (1 when
 * a restart followed the iteration).  cold_start = 1 zeroes d_u before every
 * solve (the paper's cold-start hard-problem runs).  The handle's parameters and projection
 * setting are restored at exit.  Synchronises the stream. */
mfto_status mfto_simp_protocol(mfto_handle* h, double* d_rho, double* d_u, const double* d_f,
                               double* d_rho_selected, const mfto_protocol_params* p,
                               double* compliance, double* grayness, int32_t* restarted,
                               mfto_protocol_stats* st);

/* ------------------------------------------- condition-number estimate -- */

typedef struct {
  int32_t power_maxit;      /* power-iteration step cap (50)                   */
  double power_tol;         /* stop when lambda_max changes by < tol (1e-6)    */
  int32_t inverse_maxit;    /* inverse-iteration step cap (50)                 */
  double inverse_tol;       /* stop when 1/lambda_min changes by < tol (1e-4)  */
  double inner_rtol;        /* inner PCG: ||r|| <= rtol ||v||, ||v|| = 1 (1e-8) */
  int32_t inner_maxit;      /* inner PCG iteration cap (2000)                  */
} mfto_kappa_params;

typedef struct {
  double lambda_max;        /* Rayleigh quotient of the last power step        */
  double lambda_min;        /* 1 / (v . K^-1 v) of the last inverse step        */
  double kappa;             /* lambda_max / lambda_min                         */
  int32_t power_steps, inverse_steps;
  int32_t inner_iterations; /* PCG iterations of all inverse steps             */
  int32_t inner_capped;     /* inner solves that stopped at the cap            */
} mfto_kappa_stats;

/* The defaults above: the paper's caps and tolerances (Sec. 3.5). */
void mfto_default_kappa_params(mfto_kappa_params* p);

/* Matrix-free estimate of kappa(K) on the free DOFs (Sec. 3.5, "Condition
 * number of the SIMP stiffness matrix"): power iteration for lambda_max and
 * inverse iteration for lambda_min, every product an FP64 K(E).v of this
 * handle, every inverse step a Jacobi-PCG solve from zero (the paper's
 * SciPy CG is unpreconditioned; converged, both give K^-1 v).  d_E: FP64
 * moduli.  d_v_power, d_v_inverse: the start vectors (n_dof doubles; the
 * caller seeds them); they are zeroed on the fixed DOFs, normalised, and
 * overwritten with the final unit iterates.  d_work: n_dof doubles of
 * scratch.  p may be NULL (defaults).  Capped estimates bound the spectrum
 * from inside, so kappa is not overestimated.  MFTO_INVALID_ARG for a start
 * vector that vanishes on the free DOFs, MFTO_BREAKDOWN for a vanishing
 * iterate.  Synchronises the stream. */
mfto_status mfto_kappa(mfto_handle* h, const double* d_E, double* d_v_power,
                       double* d_v_inverse, double* d_work, const mfto_kappa_params* p,
                       mfto_kappa_stats* st);

/* ------------------------------------------------------------- timing -- */

/* When on, every K.v launch issued by the library on this handle is
 * bracketed by CUDA events on the handle's stream (inside the captured CG
 * graphs as external event nodes); mfto_kv_timing_read synchronises and
 * returns, for the K.v launches of one form (MFTO_FORM_F64 or MFTO_FORM_F32;
 * the mixed solver runs both), the number of timed launches that did work
 * and their summed device time in milliseconds, then resets that form's
 * accumulators. */
mfto_status mfto_kv_timing(mfto_handle* h, int32_t on);
mfto_status mfto_kv_timing_read(mfto_handle* h, mfto_form form, int64_t* launches,
                                double* total_ms);

/* Persistent CG launches timed while mfto_kv_timing is on (they contain the
 * FP32 K.v applications of the inner solves, which then have no launches of
 * their own): number of launches, CG iterations they completed (K.v
 * applications) and their summed device time in milliseconds; resets the
 * accumulators. */
mfto_status mfto_cg_timing_read(mfto_handle* h, int64_t* launches, int64_t* iterations,
                                double* total_ms);

/* Device time of one launch of the FP32 CG K.v as the default inner CG
 * (engine 2, FP32 column K.v) runs it on this handle: the first inner
 * iteration's K.v launch, with the handle's mesh, autotuned launch shape and
 * work vectors (unit moduli, a right-hand side of ones), captured `launches`
 * times back to back into one CUDA graph; after one untimed replay, `reps`
 * replays are timed between two CUDA events on the handle's stream, and
 * *us_per_launch = elapsed / (reps x launches) in microseconds.  Every launch
 * does the work of a CG iteration's K.v, so this is the kernel's duration
 * plus the gap between consecutive graph kernels, without the event nodes
 * that mfto_kv_timing places around every launch (which add several
 * microseconds to each timed launch).  With events = 1 the same graph also
 * holds an external event record node before and after every launch, as
 * mfto_kv_timing places them in the CG graphs, and *us_per_launch is the
 * mean interval between each launch's two events in the last replay: the
 * difference to events = 0 is what those nodes add.  Overwrites the FP32
 * work vectors of the handle (as mfto_kv_autotune does); synchronises the
 * stream.  MFTO_INVALID_ARG unless launches is in [1, 4096], reps >= 1,
 * events is 0 or 1, and the FP32 inner form with CG engine 2 and the column
 * K.v (the defaults) is selected. */
mfto_status mfto_cg_kv_time(mfto_handle* h, int32_t launches, int32_t reps, int32_t events,
                            double* us_per_launch);

/* Number of kernels the library has launched for this handle so far (the
 * kernel nodes of every launched CUDA graph included). */
mfto_status mfto_launch_count(const mfto_handle* h, int64_t* n);

/* ------------------------------------------------- no-allocation variant -- */

/* mfto_compliance_sens for callers that cannot allocate device memory: the
 * same c = sum_e E_e u_e^T KE u_e and (if d_dc is not NULL)
 * d_dc[e] = -p rho_e^(p-1) (E0 - Emin) u_e^T KE u_e, computed without a
 * handle and without any cudaMalloc, cudaFree or allocating library call.
 * It exists for programs whose device memory belongs entirely to another
 * allocator (a framework's caching pool, a budget reserved at start-up) and
 * for latency-bound loops that cannot accept the device-wide synchronisation
 * an allocation may cause.  The paper has no counterpart to this entry point.
 *
 * mesh: the structured grid (elements per axis, edge h); E0, Emin, nu, penal:
 * as in mfto_params; d_rho_phys [n_elem], d_u [n_dof], d_dc [n_elem] or NULL:
 * device arrays in the layouts of this header, owned by the caller; h_c_out:
 * host double receiving c; stream: cudaStream_t of the work (0 = legacy
 * default), synchronised before returning.
 *
 * Capacity: the only scratch is one file-scope device array of 21 KB (unit
 * KE, 2048 per-block partial sums, a ticket and the result) that every GPU
 * which loads the library holds until the process exits; meshes of more than
 * 2048 x 256 = 524,288 elements are rejected with MFTO_TOO_LARGE.  The first
 * call on a device looks up the array's device address (set-up) and keeps it
 * for the rest of the process; make that first call before any stream
 * capture, and do not call the entry point again on a device after a
 * cudaDeviceReset of it (the kept address belongs to the reset context).
 * Every call copies the unit KE in, reads the result back and synchronises
 * the stream before it returns.  The pointers must be memory of the current
 * device.  All calls share the array and it
 * keeps the last call's contents (the ticket is cleared by every call), so
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * and must be serialised by the caller.  Returns MFTO_INVALID_ARG for null
 * pointers or bad sizes or parameters, MFTO_CUDA_ERROR on a CUDA failure. */
mfto_status mfto_compliance_sens_noalloc(const mfto_mesh* mesh, double E0, double Emin,
                                         double nu, double penal, const double* d_rho_phys,
                                         const double* d_u, double* d_dc, double* h_c_out,
                                         void* stream);

/* ------------------------------------------------ geometric multigrid -- */

/* Geometric multigrid for the masked operator, the solver follow-on of Sec. 6
 * ("Path to Geometric Multigrid Integration": restriction, prolongation
 * P = R^T, a direct coarsest solve, smoothing steps that apply the operator)
 * with the FP32 K.v as the fine smoother (Sec. 3.5, "Path forward").
 * Levels: level 0 is the handle's mesh; level l + 1 has ceil(n / 2) elements
 * per axis of level l's n; coarsening stops at the first level with at most
 * coarse_max_dofs DOFs, or after max_levels levels.  Interpolation is
 * trilinear from the coarse nodes (fine coordinates 2I) with the fine fixed
 * DOFs zeroed; a coarse DOF is fixed where the fine DOF at its position is;
 * each coarse level is the Galerkin product Phat^T A Phat (formed element by
 * element: each coarse element's 24 x 24 matrix from its children's) plus the
 * identity on its fixed DOFs.  V-cycle: nu_pre sweeps from x = 0, either
 * l1-Jacobi, x += omega D1^-1 (b - A x) (D1 the l1 row sums of the element
 * matrices), or Chebyshev sweeps of degree cheb_degree for D1^-1 A; residual,
 * restriction, recursion, prolongation, nu_post sweeps; the coarsest level is
 * solved by its dense inverse (FP64 Cholesky on the host, applied in FP32).
 * The cycle runs in FP32, each sweep's vector update inside the launch that
 * applies the operator where the operator is the FP32 column K.v or stored
 * element matrices. */
#define MFTO_GMG_MAX_LEVELS 10
#define MFTO_GMG_MAX_COARSE 1000   /* DOFs of the densely inverted level */
typedef struct {
  int32_t max_levels;       /* 1 .. MFTO_GMG_MAX_LEVELS (default 10)      */
  int32_t coarse_max_dofs;  /* 3 .. MFTO_GMG_MAX_COARSE (default 200)     */
  int32_t nu_pre, nu_post;  /* 0 .. 8 sweeps (default 1, 1)               */
  double omega;             /* l1-Jacobi weight in (0, 2) (default 1.3)   */
  int32_t mixed;            /* mfto_gmg_solve: 0 FP64 CG, 1 FP64 refinement
                               around an FP32 CG (default 1)              */
  double inner_tol;         /* relative tolerance of each FP32 CG, (0, 1)
                               (default 1e-2)                             */
  int32_t smoother_form;    /* K.v form of the level-0 sweeps and residual
                               inside the cycle: MFTO_FORM_F32 (default) or
                               a tensor-core form (TF32, BF16, FP16 and
                               their split variants)                      */
  int32_t matfree_level1;   /* level 1 applied as Phat^T K Phat with the
                               FP32 fine operator instead of its element
                               matrices: 1 always, -1 never, 0 (default)
                               when those matrices exceed 96 MiB          */
  int32_t continue_dir;     /* mixed solve: each FP32 CG after the first
                               continues the previous one's direction,
                               p = z + (r.z / (r.z)_prev) p (1, default),
                               or starts from p = z (0)                   */
  int32_t cheb_degree;      /* 0: l1-Jacobi sweeps with omega; k = 1 .. 8:
                               Chebyshev sweeps of degree k on [1/30, 1]
                               of D1^-1 A (1 = the l1 bound), a sweep
                               costing k operator applications; -1
                               (default): 2 up to 4,000,000 DOFs, else 0  */
} mfto_gmg_params;
void mfto_default_gmg_params(mfto_gmg_params* p);
/* Build the hierarchy for the moduli d_E (FP64 [elements]) with params p
 * (NULL: the handle's current ones, initially the defaults).  Synchronises
 * the stream (the coarsest inverse is formed on the host).  MFTO_TOO_LARGE
 * when the coarsest level would exceed MFTO_GMG_MAX_COARSE DOFs,
 * MFTO_BREAKDOWN when it is not positive definite. */
mfto_status mfto_gmg_setup(mfto_handle* h, const double* d_E, const mfto_gmg_params* p);
/* The parameters of the last setup with its automatic choices resolved
 * (cheb_degree >= 0; matfree_level1 1 or -1 as applied). */
mfto_status mfto_gmg_params_in_use(mfto_handle* h, mfto_gmg_params* p);
/* Levels of the last setup: *n_levels and dims[3 * l + axis] elements. */
mfto_status mfto_gmg_levels(mfto_handle* h, int32_t* n_levels, int32_t* dims);
/* d_y = A_level d_x (FP32 [DOFs of that level]); level 0 is the FP32 K.v. */
mfto_status mfto_gmg_apply(mfto_handle* h, int32_t level, const float* d_x, float* d_y);
/* d_z = V(d_r), one V-cycle on FP32 fine vectors (d_r and d_z distinct). */
mfto_status mfto_gmg_vcycle(mfto_handle* h, const float* d_r, float* d_z);
/* K(E) u = f by CG preconditioned with the V-cycle (Polak-Ribiere beta),
 * after a setup for d_E, from the initial guess in d_u until
 * ||r|| <= rtol ||f|| (the handle's rtol):
 *   mixed = 0: one CG with FP64 vectors, K.v and dot products, at most the
 *     handle's maxit iterations;
 *   mixed = 1: FP64 refinement (r = f - K u with the FP64 K.v, u += e) around
 *     CGs in FP32 (FP32 K.v and vectors, FP64 dot products) that each reduce
 *     their residual by inner_tol, at most maxit iterations each; at most 50
 *     corrections, MFTO_STALLED when the residual fails twice in a row to
 *     fall below 0.9 of the previous one.
 * Outcome in st (iterations = CG iterations, summed over the corrections). */
mfto_status mfto_gmg_solve(mfto_handle* h, const double* d_E, const double* d_f, double* d_u,
                           mfto_solve_stats* st);
/* nrhs load cases with one modulus field (the multi-RHS workload): one
 * hierarchy for d_E, then mfto_gmg_solve's iteration for each case.  d_F and
 * d_U FP64 [nrhs][DOFs] (d_U: initial guesses in, solutions out), st: nrhs
 * entries. */
mfto_status mfto_gmg_solve_multi(mfto_handle* h, const double* d_E, const double* d_F,
                                 double* d_U, int32_t nrhs, mfto_solve_stats* st);
/* on != 0: mfto_simp_step solves with mfto_gmg_solve (params p, NULL keeps the
 * current ones); on = 0: back to the solver of mfto_set_solver. */
mfto_status mfto_set_gmg_solver(mfto_handle* h, int32_t on, const mfto_gmg_params* p);

/* ------------------------------------- element-by-element microbenchmark -- */

/* y = sum_e B_e^T (E_e KE) B_e v over an ARBITRARY element DOF table (no
 * Dirichlet rows): the synthetic hot-path microbenchmark of Sec. 5 (Tab.
 * profiling), whose element DOF indices are random rather than the
 * structured mesh's.  Variants:
 *   MFTO_EBE_STAGED_F64: three kernels, as the paper's unfused FP64 pipeline
 *     (t_full64): gather V_e = v[edof_e] into an [n_elem][24] buffer, the
 *     element contraction Y_e = V_e KE into a second one, and the scatter
 *     y[edof_e] += E_e Y_e with FP64 atomics;
 *   MFTO_EBE_FUSED_F64 / MFTO_EBE_FUSED_F32: one kernel, an element per
 *     thread (gather, contraction, atomic scatter), in FP64 / FP32.
 * The atomics make the sums' order, and so their last bits, vary from run to
 * run.  mfto_ebe_create: n_elem >= 1 (at most 2^31 / 24), 1 <= n_dof < 2^31,
 * h_KE the 576 doubles of the unit element matrix (row-major, e.g. from
 * mfto_unit_ke), stream a cudaStream_t (NULL = legacy stream); it allocates
 * two [n_elem][24] FP64 stage buffers (MFTO_OOM if that fails).
 * mfto_ebe_kv: d_edof int32 [n_elem][24] row-major, 16-byte aligned, entries
 * in [0, n_dof); d_E, d_v, d_y FP64 (FP32 for MFTO_EBE_FUSED_F32) of n_elem,
 * n_dof, n_dof entries; d_y is overwritten.  Synchronises the stream.  With
 * h_stage_ms non-NULL the device times (CUDA events, ms) are written there:
 * gather, contraction and scatter (3 floats, the scatter's zeroing of y
 * included) for the staged variant, one total for the fused ones.  An index
 * outside [0, n_dof) is skipped and the call returns MFTO_INVALID_ARG. */
typedef enum {
  MFTO_EBE_STAGED_F64 = 0,
  MFTO_EBE_FUSED_F64 = 1,
  MFTO_EBE_FUSED_F32 = 2
} mfto_ebe_variant;
typedef struct mfto_ebe mfto_ebe;
mfto_status mfto_ebe_create(int64_t n_elem, int64_t n_dof, const double* h_KE, void* stream,
                            mfto_ebe** out);
mfto_status mfto_ebe_destroy(mfto_ebe* e);
const char* mfto_ebe_last_error(const mfto_ebe* e);
mfto_status mfto_ebe_kv(mfto_ebe* e, int32_t variant, const int32_t* d_edof, const void* d_E,
                        const void* d_v, void* d_y, float* h_stage_ms);
/* Kernels launched by this object so far. */
mfto_status mfto_ebe_launch_count(const mfto_ebe* e, int64_t* n);

/* ------------------------------------------------------- measurement aid -- */

/* Arithmetic-pipe probe: launches `blocks` x 256 threads, each running
 * `iters` iterations of 8 independent fused multiply-add chains in the given
 * form (F64 or F32) on the current device and stream 0, and returns the
 * elapsed device time (CUDA events) in *ms_out.  Work done:
 * blocks * 256 * iters * 8 FMAs.  Used to measure the FMA-pipe peak that the
 * roofline of the FP64 and FP32 K.v forms is quoted against; it has no
 * counterpart in the paper. */
mfto_status mfto_fma_probe(mfto_form form, int32_t blocks, int32_t iters, double* ms_out);

#ifdef __cplusplus
}
#endif
#endif /* MFTO_H */

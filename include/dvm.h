/*
 * dvm.h — C ABI of the GB300 S-model discrete velocity solver.
 *
 * Method: Chikitkin, Kornev & Titarev, "Numerical solution of the Boltzmann
 * equation with S-model collision integral using tensor decompositions"
 * (arXiv:1912.04582).  One explicit time step of the discrete velocity method
 * (Section 3, Algorithms 1 and 2) on every hexahedral cell of an unstructured
 * mesh, with the distribution function of each cell stored on a structured
 * N1 x N2 x N3 velocity grid either as a full tensor or in Tucker format
 * (Sections 4 and 5).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Units      nondimensional: R_g = 1/2, molecular mass m = 1, so that
 *            f^M = n (pi T)^{-3/2} exp(-|xi - u|^2 / T), p = n T / 2 and
 *            nu = p / mu(T) with mu = (Kn / sqrt(pi)) T^omega
 *            (Section 2, shakhov_integral).
 * Grid       xi_{a,i} = ((N_a-1-i) lo_a + i hi_a) / (N_a-1), i = 0..N_a-1
 *            (Section 3: uniform nodes xi_min + (i-1) dxi, endpoints included);
 *            every node has quadrature weight dxi_1 dxi_2 dxi_3.
 * Layout     a full tensor f of one cell is N1*N2*N3 doubles, i3 fastest:
 *            f[(i1*N2 + i2)*N3 + i3].  Arrays over cells are cell-major.
 * Macro      per cell [n, u1, u2, u3, T, q1, q2, q3] (Section 2), with
 *            q = (1/2) sum_nodes w v |v|^2 f.
 * Mesh       hex8 lists vertex ids in VTK order (unit-cube corners
 *            (0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1));
 *            local face l is the quad {0,4,7,3}, {1,2,6,5}, {0,1,5,4},
 *            {3,7,6,2}, {0,3,2,1}, {4,5,6,7} (outward by the right-hand
 *            rule).  Faces shared by two cells are found by vertex sets; every
 *            other (cell, local face) must be listed as a boundary face with a
 *            group id.
 * Errors     every call returns a status: DVM_OK (0), a warning (> 0) or an
 *            error (< 0); dvm_last_error() gives a message for the calling
 *            thread.  No exception crosses the ABI.
 * Ownership  the library copies every input array; the caller keeps its
 *            buffers.  The context owns all device memory it allocates.
 * Streams    all device work of a context is issued on opts.cuda_stream
 *            (NULL = the legacy default stream).  Calls that return host data
 *            synchronise that stream.
 */
#ifndef DVM_GB300_H
#define DVM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DVM_OK 0
#define DVM_NOT_CONVERGED 1
#define DVM_ERR_INVALID_ARG (-1)
#define DVM_ERR_OOM (-2)
#define DVM_ERR_CUDA (-3)
#define DVM_ERR_TIMEOUT (-4)
#define DVM_ERR_NONPHYSICAL (-5)
#define DVM_ERR_UNSUPPORTED (-6)
#define DVM_ERR_STATE (-7)
#define DVM_ERR_IO (-8)

/* boundary condition types (Section 2; Section 6 lists 'in'/'out' = free
 * stream, 'wall', and symmetry 'sym-y'/'sym-z') */
#define DVM_BC_FREESTREAM 0 /* Maxwellian with prescribed n, u, T           */
#define DVM_BC_ZEROGRAD 1   /* ghost value = interior value                  */
#define DVM_BC_SYMMETRY 2   /* f(xi) = f(xi - 2 (xi.e) e), coordinate plane  */
#define DVM_BC_WALL 3       /* diffuse reflection, full accommodation        */

/* storage formats and arithmetic */
#define DVM_FORMAT_FULL 0
#define DVM_FORMAT_TUCKER 1
#define DVM_PREC_FP64 0
#define DVM_PREC_MIXED 1

typedef struct dvm_ctx dvm_ctx;

typedef struct {
  int64_t n_vert;             /* number of vertices                          */
  const double *xyz;          /* [n_vert][3]                                 */
  int64_t n_cell;             /* number of hexahedra (1 .. 2^31-1)           */
  const int64_t *hex8;        /* [n_cell][8] vertex ids, VTK order           */
  int64_t n_bface;            /* number of boundary faces                    */
  const int64_t *bface;       /* [n_bface][2] = (cell, local face 0..5)      */
  const int32_t *bface_group; /* [n_bface] group id 0 .. 4095                */
} dvm_mesh;

typedef struct {
  int32_t N[3];  /* nodes per axis, 2 .. 128 (Tucker format: 2 .. 64)       */
  double lo[3];  /* smallest node per axis                                   */
  double hi[3];  /* largest node per axis (hi > lo)                          */
} dvm_vgrid;

typedef struct {
  double Pr;     /* Prandtl number (Section 2: 2/3)                          */
  double omega;  /* viscosity exponent, mu ~ T^omega                         */
  double Kn;     /* Knudsen number (mean-free-path definition)               */
} dvm_gas;

typedef struct {
  int32_t format;     /* DVM_FORMAT_FULL or DVM_FORMAT_TUCKER                */
  int32_t precision;  /* DVM_PREC_FP64 or DVM_PREC_MIXED                     */
  int32_t rank_cap;   /* Tucker: maximal rank per mode (1 .. min(N, 24))     */
  double tol;         /* Tucker: relative rounding tolerance eps             */
  double cfl;         /* CFL number for the fixed time step (default 0.5)    */
  double dt;          /* if > 0, use this time step instead of the CFL rule  */
  void *cuda_stream;  /* cudaStream_t for all device work (may be NULL)      */
  int32_t variant;    /* Tucker step launch variant: DVM_VARIANT_AUTO (0,
                       * the autotuner times both on the first step and keeps
                       * the faster), DVM_VARIANT_FUSED (one persistent
                       * kernel, one cell per CTA through all phases) or
                       * DVM_VARIANT_PHASED (phase-major: assembly, then per
                       * mode Gram / eigen-solve (one warp per cell) /
                       * projection kernels over chunks of cells).  Both
                       * compute the same values cell by cell.              */
  int64_t max_chunk;  /* Tucker phase-major variant: at most this many cells
                       * per chunk of its per-step work buffers (0: chunks
                       * sized to 1/8 of the free device memory, at most all
                       * cells); bounds the context's memory.  Results do not
                       * depend on it.                                      */
  int32_t engine;     /* mixed-precision Tucker, phase-major variant: how the
                       * dense contractions run.  DVM_ENGINE_AUTO (0): the
                       * first-mode Gram matrices on the tensor cores (exact
                       * integer split, see dvm_gram_tc) when N1 <= 64 and
                       * N2 N3 is a multiple of 8 up to 4096, else on the
                       * CUDA cores; on meshes whose faces all lie on
                       * coordinate planes (and N <= 64), the assembly of
                       * f^{n+1} as one small GEMM per cell of its rank-one
                       * terms (FP32 FMAs).  DVM_ENGINE_CUDA_CORES (1): the
                       * fused variant's arithmetic (Gram matrices from
                       * exact FP32 products summed in double-FP32, the
                       * assembly term by term): the two variants then
                       * agree bit for bit.  Both are accurate to FP32
                       * rounding of f^{n+1}.                              */
  int32_t scheme;     /* time stepping (Section 3): DVM_SCHEME_EXPLICIT (0),
                       * the explicit Euler step of Algorithm 1, or
                       * DVM_SCHEME_LUSGS (1, full format only), the implicit
                       * step of the linear-system equation, [I/dt - dR/df]
                       * (f^{n+1} - f^n) = R^n, solved by one LU-SGS pass: a
                       * forward sweep over the cells in increasing index
                       * order, D_i g_i = R_i - sum_{j<i} M_ij g_j, then a
                       * backward sweep in decreasing order, df_i = g_i -
                       * D_i^{-1} sum_{j>i} M_ij df_j, with the diagonal of
                       * the diagonal_term equation D_i = 1/dt + nu_i +
                       * sum_l |A_l| |xi.e_l| / (2 |V_i|), evaluated as
                       * sum_l |A_l| (xi.e_l)^+ / |V_i| (the same on a closed
                       * cell; f^S and boundary ghosts held at t^n), and
                       * M_ij = |A_l| (xi.e_l)^- / |V_i| for the face l shared
                       * with cell j.  The result depends
                       * on the cell numbering (it fixes the sweep order), not
                       * on how the work is scheduled: cells of one wavefront
                       * of the sweep run in parallel.  Its time step is not
                       * bound by the explicit limit: set cfl (> 0.5) or dt.  */
} dvm_opts;

#define DVM_ENGINE_AUTO 0
#define DVM_ENGINE_CUDA_CORES 1

#define DVM_SCHEME_EXPLICIT 0
#define DVM_SCHEME_LUSGS 1

#define DVM_VARIANT_AUTO 0
#define DVM_VARIANT_FUSED 1
#define DVM_VARIANT_PHASED 2

/* Create a solver context on the current CUDA device.  Builds the face list
 * (interior faces by shared vertex sets, boundary faces from mesh->bface),
 * face area vectors (1/2)(p2-p0)x(p3-p1) and cell volumes, and allocates the
 * state.  Section 3 (ode_system: |V_i|, |A_j|, e_j, sign(i,l)); Section 6
 * (Mesh, Solution).  Errors: INVALID_ARG (bad sizes, unmatched faces,
 * non-positive volumes), OOM, CUDA. */
int dvm_create(dvm_ctx **out, const dvm_mesh *mesh, const dvm_vgrid *vgrid,
               const dvm_gas *gas, const dvm_opts *opts);

/* Assign a boundary condition to a group (Section 2; Section 6 Problem).
 * params[8] = [n, u1, u2, u3, T, 0, 0, 0]: free stream uses all five; a wall
 * uses u (its velocity, tangential) and T (its temperature), its density n_w
 * comes from the impermeability condition; zero-gradient and symmetry ignore
 * params.  Symmetry needs a coordinate-plane face and lo = -hi on that axis
 * (else UNSUPPORTED at init).  Must precede the init call. */
int dvm_set_bc(dvm_ctx *ctx, int32_t group, int32_t type, const double params[8]);

/* Initial state from per-cell Maxwellians (Section 6, f_init): host arrays
 * n[n_cell], u[n_cell][3], T[n_cell].  Computes the moments, the time step
 * (opts.dt, or dt = CFL / max_i [nu_i + sum_l |A_l| xi_max / (2 |V_i|)]) and,
 * for the Tucker format, the rank-1 Tucker form (Section 5).  Errors:
 * INVALID_ARG, STATE (a boundary group without a condition), UNSUPPORTED. */
int dvm_init_maxwellian(dvm_ctx *ctx, const double *n, const double *u, const double *T);

/* Initial state from full tensors f[n_cell][N1*N2*N3]; on_device != 0 means f
 * is a device pointer.  Tucker contexts compress each cell by truncated HOSVD
 * at opts.tol / opts.rank_cap (Section 4, item 1).  May be called again on an
 * initialised context to replace the state; the time step of the solve is
 * then kept. */
int dvm_init_f(dvm_ctx *ctx, const double *f, int32_t on_device);

/* Tucker format only: the state given directly, in the layout the solver keeps
 * (Section 4: f = G x1 U1 x2 U2 x3 U3 per cell).  ranks[n_cell][3] with
 * 1 <= r_a <= min(N_a, rank cap R); core[n_cell][R^3], the r1 x r2 x r3 core
 * at the front of each cell's block (k3 fastest); u_a[n_cell][N_a][R], row i of
 * a cell's factor at i*R, its first r_a columns used (orthonormal columns are
 * not required).  Copied (host or device pointers, on_device as for
 * dvm_init_f); as for the other initialisations the macroparameters are
 * recomputed and the time step is kept once set.  Errors: INVALID_ARG (not a
 * Tucker context, ranks out of range), NONPHYSICAL, CUDA. */
int dvm_init_tucker(dvm_ctx *ctx, const int32_t *ranks, const double *core, const double *u1,
                    const double *u2, const double *u3, int32_t on_device);

/* Tucker format only: the current state into host arrays in the layout of
 * dvm_init_tucker (any pointer may be NULL).  Errors: INVALID_ARG, STATE. */
int dvm_get_tucker(dvm_ctx *ctx, int32_t *ranks, double *core, double *u1, double *u2,
                   double *u3);

/* Advance nsteps explicit Euler steps (Section 3, Algorithm 1 with
 * Algorithm 2 inside; Tucker: Section 5 with one rounding per cell and step).
 * If residual_out is not NULL the call synchronises and stores the residual
 * of the last step, ||U^{n+1}-U^n||_{2,V} / (dt ||U^n||_{2,V}) with
 * U = (n, n u, sum w |xi|^2 f) per cell; with NULL the call only enqueues.
 * Errors: NONPHYSICAL (n <= 0 or T <= 0 seen in a cell), TIMEOUT (Tucker: a
 * bulk shared-memory copy did not complete within its bounded wait; the blocks
 * that saw it returned without writing their results, so the step failed and
 * the state is undefined until the next dvm_init_* or dvm_load), CUDA.  Both
 * device flags are reported only by calls with residual_out, and stay set (every
 * later such call reports them) until the state is initialised again. */
int dvm_step(dvm_ctx *ctx, int32_t nsteps, double *residual_out);

/* Macroparameters of every cell (Section 2): host arrays out[n_cell][8] =
 * [n, u1, u2, u3, T, q1, q2, q3]. */
int dvm_moments(dvm_ctx *ctx, double *out);

/* Run steps until the residual is <= tol or max_steps were made; the residual
 * is checked every check_every steps (>= 1).  Returns DVM_NOT_CONVERGED (1)
 * if max_steps is hit.  steps_out / res_out may be NULL. */
int dvm_solve(dvm_ctx *ctx, double tol, int64_t max_steps, int32_t check_every,
              int64_t *steps_out, double *res_out);

/* Full tensors of cells [cell0, cell0 + ncell) into host out[ncell][N^3]
 * (Tucker cells are expanded). */
int dvm_get_f(dvm_ctx *ctx, int64_t cell0, int64_t ncell, double *out);

/* Scalars: the fixed time step, the number of steps made, the number of faces. */
int dvm_get_dt(dvm_ctx *ctx, double *dt);
int dvm_get_step_count(dvm_ctx *ctx, int64_t *steps);
int dvm_get_num_faces(dvm_ctx *ctx, int64_t *n_face);

/* Geometry as the solver sees it: vol[n_cell]; per face (owner, neighbour or
 * -1, group or -1) into fcell[n_face][3] and (|A|, e1, e2, e3) into
 * fgeo[n_face][4].  Any pointer may be NULL. */
int dvm_get_geometry(dvm_ctx *ctx, double *vol, int64_t *fcell, double *fgeo);

/* Tucker ranks per cell into r[n_cell][3] (full format: N1, N2, N3). */
int dvm_get_ranks(dvm_ctx *ctx, int32_t *r);

/* Launch configuration of the Tucker step: the persistent grid in CTAs
 * chosen by the autotuner on the first step (fused kernel, or the assembly
 * kernel of the phase-major variant), the fused kernel's time in ms for 1..4
 * resident CTAs per SM in tune_ms[1..4] and the phase-major step's in
 * tune_ms[0] (0 where not tried); the variant in use is returned as a negative
 * grid when it is the phase-major one.  Full format: grid = number of cells,
 * tune_ms zeros.  Either pointer may be NULL. */
int dvm_get_launch_config(dvm_ctx *ctx, int32_t *grid, float *tune_ms);

/* Optional per-launch event timing of the step kernels, for measurement:
 * with on != 0 every launch of dvm_step is bracketed by CUDA events on the
 * context's stream (the two-step graph replay is not used meanwhile) and its
 * elapsed time accumulated per kernel class; on == 0 stops.  Either call
 * clears the totals.  Errors: INVALID_ARG, CUDA. */
int dvm_set_kernel_timing(dvm_ctx *ctx, int32_t on);

/* Accumulated launch times (ms) and counts since timing was switched on, per
 * kernel class: [0] full-grid step, [1] fused Tucker step, [2] phase-major
 * assembly, [3] first-mode Gram, [4] second/third-mode Gram, [5] eigen-solves,
 * [6] projections/cores, [7] moments of the new state, [8] phase-major
 * mode-2/3 contractions of all cells.  ms[9], launches[9]; either may be NULL.
 * Synchronises the context's stream. */
int dvm_get_kernel_timing(dvm_ctx *ctx, double *ms, int64_t *launches);

#define DVM_KERNEL_CLASSES 9

/* Bytes of device memory held for the distribution function in its current
 * representation (Tucker: sum over cells of r1 r2 r3 + N1 r1 + N2 r2 + N3 r3
 * values, Section 7), and the total bytes the context allocated. */
int dvm_memory(dvm_ctx *ctx, size_t *f_bytes, size_t *total_bytes);

/* Checkpoint / restart of the state (Section 6: init_type 'restart'): the
 * distribution function (full tensors or cores + factors), the step counter
 * and the time step.  Restarting gives bitwise the same continuation. */
int dvm_save(dvm_ctx *ctx, const char *path);
int dvm_load(dvm_ctx *ctx, const char *path);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of steady-state solves (one request = one
 * mesh / velocity grid / gas / boundary conditions / initial state, run to a
 * residual; Section 3: the steady problem, n the iteration index).
 * A server admits queued requests while the summed device-memory estimate of
 * the running ones stays within its budget and a slot is free, creates each
 * admitted context on its own CUDA stream (so the kernels of different solves
 * overlap on the device), advances every running solve by a few steps per
 * round, and retires a solve when its residual reaches the request's
 * tolerance or its step limit.  A solve's arithmetic depends on its own data
 * only, so its result is the same alone and in a mix.
 */
typedef struct dvm_server dvm_server;

typedef struct {
  dvm_mesh mesh;
  dvm_vgrid vgrid;
  dvm_gas gas;
  dvm_opts opts;            /* opts.cuda_stream is ignored: the server owns streams */
  int32_t n_bc;             /* boundary conditions: groups[n_bc], types[n_bc],      */
  const int32_t *bc_group;  /* params[n_bc][8] (as for dvm_set_bc)                  */
  const int32_t *bc_type;
  const double *bc_params;
  const double *n0;         /* initial Maxwellians, as for dvm_init_maxwellian      */
  const double *u0;
  const double *T0;
  double tol;               /* residual to reach                                    */
  int64_t max_steps;        /* step limit                                           */
  int32_t check_every;      /* steps between residual checks (>= 1)                 */
} dvm_request;

/* request states reported by dvm_server_poll */
#define DVM_REQ_QUEUED 0
#define DVM_REQ_RUNNING 1
#define DVM_REQ_CONVERGED 2
#define DVM_REQ_NOT_CONVERGED 3
#define DVM_REQ_FAILED 4
#define DVM_REQ_CANCELLED 5

/* Device-memory estimate of one request's context (bytes). */
int dvm_estimate_memory(const dvm_request *req, size_t *bytes);

/* Create a server with a device-memory budget (bytes) and at most max_slots
 * concurrently running solves, on the current device. */
int dvm_server_create(dvm_server **out, size_t hbm_budget, int32_t max_slots);

/* Queue a request (every array is copied); its ticket is returned.  Requests
 * whose estimate exceeds the whole budget are rejected (INVALID_ARG). */
int dvm_server_submit(dvm_server *srv, const dvm_request *req, int64_t *ticket);

/* Run the admission / stepping / retirement loop until every queued request
 * has finished or max_seconds of wall time have passed.  Returns the number
 * of requests still queued or running in *pending (may be NULL). */
int dvm_server_run(dvm_server *srv, double max_seconds, int64_t *pending);

/* State of a request: state (DVM_REQ_*), steps made, last residual, latency
 * from submission to retirement in seconds (0 while unfinished).  Any output
 * pointer may be NULL. */
int dvm_server_poll(dvm_server *srv, int64_t ticket, int32_t *state, int64_t *steps,
                    double *residual, double *latency_s);

/* Macroparameters [n_cell][8] of a finished request (kept after its device
 * memory was released). */
int dvm_server_result(dvm_server *srv, int64_t ticket, double *macro);

/* Cancel a request.  A queued request is retired at once (state CANCELLED); a
 * running one keeps its slot until the chunk of steps it has in flight ends, and
 * the next dvm_server_run retires it there (state CANCELLED, its device memory
 * released, dvm_server_result giving the macroparameters reached).  Errors:
 * INVALID_ARG (unknown ticket), STATE (already finished). */
int dvm_server_cancel(dvm_server *srv, int64_t ticket);

/* Message of a failed request ("" otherwise); valid until the server is
 * destroyed. */
const char *dvm_server_error(dvm_server *srv, int64_t ticket);

void dvm_server_destroy(dvm_server *srv);

/* Macroparameters [n, u1, u2, u3, T, q1, q2, q3] of n_cell full tensors that
 * are already in device memory, computed without allocating device memory.
 * The paper has no counterpart: this entry point is for callers that cannot
 * allocate at the point of the call, such as an application whose device
 * memory is handed out by its own pool allocator, or a pipeline that must not
 * pay the implicit device-wide synchronisation of cudaMalloc between kernels
 * it has already queued.
 *   f      device pointer, [n_cell][N1*N2*N3] doubles in the layout above
 *   macro  device pointer, [n_cell][8] doubles, written on cuda_stream (the
 *          call only enqueues; synchronise before reading)
 * The per-cell intermediate sums live in a fixed array inside the library
 * with room for 16384 cells (1 MiB, held by every GPU that loads the library
 * until the process exits); a larger n_cell is rejected with
 * DVM_ERR_INVALID_ARG.  The first call on each device (and the first after that
 * device's context has been replaced, e.g. by cudaDeviceReset) looks up that
 * array's device address with cudaGetSymbolAddress, so make the first call on a
 * device before any stream capture.  Every call uses the same array: calls whose
 * GPU work overlaps (other streams or host threads on the same device) race on
 * it and must be serialised by the caller.  A cell whose density sum is zero
 * gets NaN macroparameters (there is no per-cell status).  Results equal those
 * of dvm_moments on a context initialised with the same tensors, up to
 * summation order. */
int dvm_full_macro_noalloc(const double *f, int64_t n_cell, const dvm_vgrid *vgrid,
                           double *macro, void *cuda_stream);

/* Gram matrices C_j = X_j X_j^T of ncell row-major n x K FP32 matrices on the
 * tensor cores (tcgen05, bf16 MMAs with FP32 accumulators), exact up to FP64
 * rounding for the tensor whose elements are rounded to 35 bits below their
 * row's largest magnitude (an Ozaki-type split into five 7-bit integer slices).
 * This is the Gram step of the mixed-precision Tucker rounding (Section 4 item 4,
 * the truncated SVD of each unfolding), exported as a building block; the paper
 * has no such call.
 *   X       device pointer, [ncell][n][K] floats, 16-byte aligned
 *   n, K    1 <= n <= 64, 8 <= K <= 4096, K a multiple of 8 (else INVALID_ARG)
 *   C       device pointer, [ncell][n][n] doubles, written on cuda_stream (the
 *           call only enqueues; synchronise before reading)
 *   status  device pointer to an int the kernel ORs 2 into if one of its
 *           bounded waits runs out (C is then incomplete); the caller zeroes it
 * Errors: INVALID_ARG, UNSUPPORTED (no such launch on this device), CUDA. */
int dvm_gram_tc(const float *X, int64_t ncell, int32_t n, int32_t K, double *C,
                int32_t *status, void *cuda_stream);

/* Host-side fault injection, for testing the error paths (the paper has no
 * counterpart).  Process-wide; each kind fires once and then disarms:
 *   DVM_FAULT_ALLOC    the device allocation made after `count` more succeed
 *                      fails as out of memory (DVM_ERR_OOM from the call that
 *                      made it, e.g. dvm_create, or a failed serving request);
 *   DVM_FAULT_TIMEOUT  the dvm_step call made after `count` more finds the
 *                      context's device flag set as a timed-out bulk-copy wait
 *                      leaves it (DVM_ERR_TIMEOUT from the next call with
 *                      residual_out, or a failed serving request);
 *   DVM_FAULT_ADMIT    the next `count` admission checks of every server see
 *                      the memory budget as full (requests stay queued);
 *   DVM_FAULT_NONE     disarms all.
 * A negative count disarms that kind.  No device fault is ever raised. */
#define DVM_FAULT_NONE 0
#define DVM_FAULT_ALLOC 1
#define DVM_FAULT_TIMEOUT 2
#define DVM_FAULT_ADMIT 3
int dvm_fault_inject(int32_t kind, int64_t count);

/* The schedule of one sweep of the implicit LU-SGS step (DVM_SCHEME_LUSGS; Section 3,
 * linear-system equation), a host computation with no device work.  The forward
 * sweep visits the cells in increasing index order and the backward sweep in
 * decreasing order; a cell's wavefront is 0 if none of its neighbours comes before
 * it in the sweep, else one more than the largest wavefront of those that do.  The
 * cells of one wavefront depend only on earlier ones, so the step updates them in
 * parallel (one launch per wavefront) with the result of the sequential sweep.
 *   nb       host, [n_cell][6] neighbour cell across each face, -1 on the boundary
 *            (each entry -1 or in [0, n_cell), else INVALID_ARG)
 *   forward  1 forward sweep, 0 backward sweep
 *   order    host, [n_cell] out: the cells by wavefront, increasing index within one
 *   offsets  host, [n_cell + 1] out: wavefront w is order[offsets[w] .. offsets[w+1])
 *   n_waves  out: the number of wavefronts (offsets[0 .. n_waves] are written)
 * Errors: INVALID_ARG (n_cell < 0, null pointers, a neighbour out of range). */
int dvm_lusgs_wavefronts(int64_t n_cell, const int32_t *nb, int32_t forward, int32_t *order,
                         int64_t *offsets, int64_t *n_waves);

void dvm_destroy(dvm_ctx *ctx);

/* Message of the last failed call made by this thread ("" if none). */
const char *dvm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DVM_GB300_H */

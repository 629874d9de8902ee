/*
 * cvweno.h -- C ABI of the GB300 (sm_103a) cell-vertex WENO stabilised DG solver.
 *
 * The library computes, on one GPU, the per-stage stabilised residual of
 * Vedral & Kuzmin, "Cell-vertex WENO schemes with shock-capturing quadrature for
 * high-order finite element discretizations of hyperbolic problems" (arXiv
 * 2601.16911), for du/dt + div f(u) = 0 (Sec. 2, eq. pde) on uniform 1D meshes and
 * uniform structured quadrilateral meshes, DG with tensor Legendre Q_p, p = 1..4:
 *
 *   (a) Hermite (Taylor) data of every cell at its vertices   Sec. 3.2, eq. taylorsol,
 *                                                              eq. pointsnorm
 *   (b) vertex-averaged HWENO candidates                       Sec. 3.2, eq. taylorcand
 *   (c) cell-vertex WENO reconstruction, sensor gamma_e and
 *       viscosity nu_e                                         Sec. 3.2 eq. finalweno,
 *                                                              Sec. 2.2 eq. gamma, snorm,
 *                                                              lostab
 *   (d) shock-capturing quadrature weights alpha_q             Sec. 4, eq. alphaq,
 *                                                              eq. alpha_prelim
 *   (e) volume + face residual with the dissipation added      Sec. 2.1 eq. convop,
 *       (LLF for scalar laws, HLL for Euler), M^{-1}, SSP-RK3  Sec. 2.2 eq. stab, sdstab
 *
 * Conventions (all entry points):
 *   - Every float pointer is a CALLER-OWNED DEVICE pointer, contiguous, laid out
 *     u[var][cell][k] with cell = i + nx*j and k = kx + (p+1)*ky (tensor Legendre
 *     mode, 1D: k = kx).  The library never frees caller memory.
 *   - Host pointers are marked "host".  Streams are cudaStream_t passed as void*;
 *     NULL means the legacy default stream.  Work is stream-ordered; an entry point
 *     only synchronises where it says so.  The scalar stage kernels are launched with
 *     programmatic dependent launch: one may start while the previous kernel on the
 *     stream (the caller's included) finishes, but it reads or writes no memory that
 *     kernel can touch until that kernel has completed.  A caller kernel launched with
 *     the same attribute right after them must wait likewise before reading their
 *     output.
 *   - Errors are returned as cvweno_status; nothing is thrown across the ABI.
 *     Kernels report non-finite values and non-positive density/pressure through a
 *     device status word that cvweno_status_check() (and every synchronising
 *     entry point) reads and clears.
 *   - A mesh owns its tables and scratch (two stage buffers of the state size).
 *     Calls on one mesh must not overlap on different streams.
 *   - CG meshes (kind CVWENO_CG) hold nodal values at the Gauss-Lobatto nodes instead:
 *     u[var][node] (see cvweno_state_size); the sensor and the SC weights are
 *     computed per cell exactly as for DG.  CG residual: Sec. 2.2 (CG form of eq. stab),
 *     P_h by the lumped-mass L2 projection, M^{-1} by the lumped mass with two
 *     defect-correction sweeps.
 */
#ifndef CVWENO_H
#define CVWENO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cvweno_mesh_s* cvweno_mesh;

typedef enum {
  CVWENO_OK = 0,
  CVWENO_ERR_ARG = 1,          /* invalid argument (NULL pointer, bad size, bad combination) */
  CVWENO_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  CVWENO_ERR_NONFINITE = 3,    /* a kernel produced a NaN/Inf */
  CVWENO_ERR_POSITIVITY = 4,   /* Euler: non-positive density or pressure at a node */
  CVWENO_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  CVWENO_ERR_UNSUPPORTED = 6,  /* valid but not implemented (degree, kind, system) */
  CVWENO_ERR_NOMEM = 7,        /* device or host allocation failed */
  CVWENO_ERR_CHECK = 8         /* a bounds check of the checked build (-DCVWENO_CHECK) failed */
} cvweno_status;

enum { CVWENO_DG = 0, CVWENO_CG = 1 };
enum { CVWENO_PERIODIC = 0, CVWENO_TRANSMISSIVE = 1 };
/* flux f: BURGERS 1D u^2/2, 2D (u^2/2, u^2/2); KPP (sin u, cos u) (Sec. 5.3);
 * LINADV (vx u, vy u); EULER ideal gas (rho, rho v, rho E) (Sec. 5.4) */
enum { CVWENO_BURGERS = 0, CVWENO_KPP = 1, CVWENO_LINADV = 2, CVWENO_EULER = 3 };
/* sensor_mode: COMPUTED = eq. gamma; SMOOTH forces gamma_e = 1; TROUBLED forces 0 */
enum { CVWENO_SENSOR_COMPUTED = 0, CVWENO_SENSOR_SMOOTH = 1, CVWENO_SENSOR_TROUBLED = 2 };
/* analytic initial data for cvweno_project; parameter layouts in cvweno_project */
enum {
  CVWENO_IC_CONST = 0,
  CVWENO_IC_SINE_STEP = 1,
  CVWENO_IC_CIRCLE = 2,
  CVWENO_IC_QUADRANTS = 3,
  CVWENO_IC_FOURIER = 4,
  CVWENO_IC_POLY = 5,
  CVWENO_IC_DENSITY_WAVE = 6
};

/* Method parameters.  Defaults (cvweno_default_params) are the paper's:
 * eps = 1e-6, r = 2 (Sec. 3.2, Jiang-Shu), q = 1 (Sec. 5), vertex linear weight
 * 1e-3 (Sec. 3.2), C_gamma = 0.9 (Sec. 5), SC quadrature on, gas gamma = 1.4. */
typedef struct {
  double eps;           /* Jiang-Shu epsilon */
  double r;             /* Jiang-Shu power; must be an integer in [1, 8] */
  double q;             /* exponent q of eq. gamma and of both indicators, >= 1 */
  double gamma_vertex;  /* linear weight of each vertex candidate; cell gets 1 - v_e * this */
  double c_gamma;       /* SC quadrature cutoff: redistribute iff gamma_e < c_gamma */
  int sc_quadrature;    /* 1: shock-capturing quadrature (Sec. 4) on; 0: off */
  int sensor_mode;      /* CVWENO_SENSOR_* */
  double lambda_const;  /* > 0: fixed wave speed for nu_e and LLF (KPP: 1); <= 0: computed */
  double gas_gamma;     /* Euler heat capacity ratio */
  double adv_vx, adv_vy;/* LINADV velocity */
  int hweno_limiter;    /* 1: after every RK stage, cells with computed gamma_e < c_gamma are
                           overwritten by their average-preserving cell-vertex WENO
                           reconstruction (Sec. 3; DG scalar laws only); 0: off */
  int positivity;       /* 1: after every RK stage, the positivity limiter (cvweno_positivity;
                           Euler DG only); 0: off */
} cvweno_params;

typedef struct {
  int dim;              /* 1 or 2 */
  int nx, ny;           /* cells per direction (ny ignored in 1D) */
  int degree;           /* p in 1..4 */
  int kind;             /* CVWENO_DG, or CVWENO_CG (scalar laws, periodic meshes; state =
                           values at the GLL nodes, see cvweno_state_size) */
  int system;           /* CVWENO_BURGERS | KPP | LINADV | EULER (KPP, EULER: 2D only) */
  int bc[4];            /* x-low, x-high, y-low, y-high: PERIODIC or TRANSMISSIVE;
                           periodic sides must come in pairs */
  double x0, x1, y0, y1;/* box [x0,x1] x [y0,y1] (y ignored in 1D) */
  cvweno_params params;
} cvweno_mesh_desc;

/* Fill *p with the paper's parameter values (see cvweno_params). */
void cvweno_default_params(cvweno_params* p);

/* Build the mesh: host tables (vertex patches, colouring), basis tabulations in
 * FP64 rounded once to FP32, device scratch.  The discretisation is that of Sec. 2
 * (the uniform partition of Sec. 2 eq. pde's domain into cells K_e of diameter h_e,
 * Sec. 2.1 DG space V_h of tensor polynomials Q_p; Sec. 2.2 for the CG space) with the
 * vertex patches C(x_i) of Sec. 3.2 (the cells meeting at vertex x_i).  desc and out are host pointers.
 * Returns ERR_ARG for inconsistent sizes/sides, ERR_UNSUPPORTED for degree > 4, 1D
 * Euler/KPP, CG with Euler or a transmissive side, or a non-integer r.  Records the
 * current device as the mesh's device. */
cvweno_status cvweno_mesh_create(const cvweno_mesh_desc* desc, cvweno_mesh* out);

/* Free everything the mesh owns (synchronises its device).  NULL is accepted.  (Resource
 * management; no passage of the paper.) */
cvweno_status cvweno_mesh_destroy(cvweno_mesh m);

/* Sizes (host out-pointers, each may be NULL): cells, DOFs per cell per variable
 * ((p+1)^dim, the dimension of Q_p on one cell, Sec. 2.1), conserved variables (1 or 4;
 * Sec. 5.4 for Euler), vertices x_i (Sec. 3.2; periodic sides identify their vertices),
 * quadrature points per cell ((p+1)^dim Gauss-Legendre, the nodes x_q of Sec. 4). */
cvweno_status cvweno_mesh_info(cvweno_mesh m, int64_t* ncells, int64_t* ndof_per_var, int* nvars,
                               int64_t* nverts, int* nquad);

/* Number of floats of one state (host out-pointer; Sec. 2.1 DG, Sec. 2.2 CG spaces):
 * nvars * ncells * (p+1)^dim for DG,
 * nvars * (p nx) * (p ny) nodal values for CG (GLL nodes of the periodic lattice,
 * node I + (p nx) J). */
cvweno_status cvweno_state_size(cvweno_mesh m, int64_t* nstate);

/* Host copies of the integer mesh tables (host arrays, each may be NULL), the vertex
 * patches C(x_i) of Sec. 3.2 (eq. taylorcand averages over them):
 *   cell_vertices[ncells][2^dim]  vertex of corner c = cx + 2 cy of each cell
 *   vertex_cells[nverts][2^dim]   cells around each vertex in the fixed slot order
 *                                 SW, SE, NW, NE (1D: W, E); -1 where a transmissive
 *                                 side leaves a slot empty
 *   colour[ncells]                a colouring in which no two cells sharing a vertex
 *                                 have the same colour (at most 9 colours) */
cvweno_status cvweno_mesh_tables(cvweno_mesh m, int32_t* cell_vertices, int32_t* vertex_cells, int32_t* colour);

/* L2 projection of an analytic initial datum onto the DG space (12-point Gauss rule
 * per direction), written to u (device, state layout).  ic_params: host array of 64
 * doubles:
 *   CONST: conserved state [0..3]; SINE_STEP: A sin(2 pi k (x-x0)/Lx) + B H(x - s) with
 *   (A, k, B, s); CIRCLE: (cx, cy, R, inside, outside); QUADRANTS (Euler): split (xs, ys)
 *   then (rho, vx, vy, p) of quadrant qx + 2 qy; FOURIER: M then M x (a, kx, ky, phase)
 *   of sum a sin(2 pi (kx (x-x0)/Lx + ky (y-y0)/Ly) + phase); POLY: params[i + 5 j] is
 *   the coefficient of x^i y^j (i, j <= 4); DENSITY_WAVE (Euler):
 *   rho = 1 + A sin(2 pi (kx (x-x0)/Lx + ky (y-y0)/Ly)), velocity (vx, vy), pressure p0
 *   with (A, kx, ky, vx, vy, p0). */
cvweno_status cvweno_project(cvweno_mesh m, int ic_type, const double* ic_params, float* u, void* stream);

/* Stages (a)+(b) only, for inspection: T*[nverts][(p+1)^dim] (device), the vertex
 * candidate's physical derivatives D^k u*_i(x_i), k = kx + (p+1) ky (eq. taylorcand). */
cvweno_status cvweno_vertex_data(cvweno_mesh m, const float* u, float* tstar, void* stream);

/* Stages (a)-(c): smoothness sensor gamma_e (eq. gamma) and viscosity
 * nu_e = lambda_e h_e / (2p) (eq. lostab), both [ncells] device arrays. */
cvweno_status cvweno_sensor(cvweno_mesh m, const float* u, float* gamma, float* nu, void* stream);

/* Stages (a)-(e): dudt = M^{-1} r (device, state layout).  Optional device outputs
 * (NULL to skip): gamma[ncells], nu[ncells], alpha[ncells][nvars][nquad] (the SC
 * weights, 1 where not redistributed; q = qx + (p+1) qy), troubled[ncells] (1 where
 * SC redistributed).  troubled_override (device int32[ncells] or NULL): -1 = decide,
 * 0/1 = force the SC decision of that cell (used to compare decisions taken in
 * another precision). */
cvweno_status cvweno_residual_ex(cvweno_mesh m, const float* u, const int32_t* troubled_override, float* dudt,
                                 float* gamma, float* nu, float* alpha, int32_t* troubled, void* stream);

/* Stages (a)-(e): dudt = M^{-1} r (device, state layout): r is the stabilised residual of
 * Sec. 2.1 eq. convop plus the dissipation of Sec. 2.2 eq. stab / eq. lostab, with the
 * sensor of Sec. 3.2 eq. finalweno and Sec. 2.2 eq. gamma and the quadrature weights of
 * Sec. 4 eq. alphaq; M is the (diagonal, Legendre) mass matrix. */
cvweno_status cvweno_residual(cvweno_mesh m, const float* u, float* dudt, void* stream);

/* One SSP-RK3 step (Shu-Osher form) in place on u (device): the explicit third-order
 * strong-stability-preserving Runge-Kutta scheme of Sec. 5 applied to the semi-discrete
 * system of Sec. 2.2 eq. sdstab, each stage a cvweno_residual evaluation.  dt > 0: that step size,
 * no synchronisation.  dt <= 0: dt = cfl * min(dx, dy) / (dim * max lambda_e), which
 * reads the FP64 maximum back (synchronises) and also checks the status word.
 * dt_used (host, may be NULL) receives the step size. */
cvweno_status cvweno_step(cvweno_mesh m, float* u, double dt, double cfl, double* dt_used, void* stream);

/* nsteps SSP-RK3 steps (Sec. 5, as cvweno_step) of fixed size dt > 0, enqueued without
 * synchronisation.  A 1D
 * scalar DG mesh of at most 128 cells without a limiter (one tile) runs all the steps of
 * the call in one kernel launch (cvweno_step: its one step), unless kernel timing is on;
 * the results are bitwise those of one launch per stage. */
cvweno_status cvweno_advance(cvweno_mesh m, float* u, double dt, int nsteps, void* stream);

/* FP64 totals sum_e int_{K_e} u_h of every conserved variable into totals[nvars]
 * (host): the totals the scheme conserves (Sec. 4: the stabilisation keeps the zero-sum
 * property s_h^e(u_h, 1) = 0, which gives discrete conservation).  Synchronises. */
cvweno_status cvweno_mass_total(cvweno_mesh m, const float* u, double* totals, void* stream);

/* FP64 maximum over cells of lambda_e (the wave speed of Sec. 2.2 eq. lostab, read as
 * max |f'(u_h)| over the cell's nodes; the CFL time step of cvweno_step follows from it)
 * into *lam (host).  Synchronises and checks the status word. */
cvweno_status cvweno_max_wavespeed(cvweno_mesh m, const float* u, double* lam, void* stream);

/* Synchronise the stream, read and clear the mesh's device status word.  (Error
 * reporting; no passage of the paper.) */
cvweno_status cvweno_status_check(cvweno_mesh m, void* stream);

/* HWENO limiter (Sec. 3): out = u, except that every cell whose computed sensor gamma_e
 * is below c_gamma (or every cell, when all_cells is set) is overwritten by its
 * cell-vertex WENO reconstruction u^{e,*} (eq. finalweno) built from the
 * average-corrected vertex candidates, so cell means are kept.  The troubled set
 * ignores sensor_mode.  u and out: device states of the mesh layout, distinct;
 * troubled (device [ncells], may be NULL) receives 1 for limited cells.  DG scalar
 * laws (ERR_UNSUPPORTED otherwise).  Enqueued without synchronisation. */
cvweno_status cvweno_limit(cvweno_mesh m, const float* u, float* out, int all_cells, int32_t* troubled,
                           void* stream);

/* Positivity limiter for the Euler equations (Zhang and Shu's scaling limiter; the paper
 * defers positivity to cited work).  Per cell, at the volume and face Gauss nodes: the
 * density's non-mean modes are scaled by theta_1 so that rho >= eps_e, then the non-mean
 * modes of all variables by theta_2 so that p >= eps_e, eps_e = 1e-3 min(mean density,
 * mean pressure); cell means are kept.  u, out: device Euler states (may be the same
 * array: the limiter is cell-local); theta (device [ncells], may be NULL) receives
 * theta_1 theta_2.  A cell whose mean is not admissible is copied and raises status bit
 * 2 (CVWENO_ERR_POSITIVITY at the next status check).  2D Euler DG meshes. */
cvweno_status cvweno_positivity(cvweno_mesh m, const float* u, float* out, float* theta, void* stream);

/* Per-launch device times, a measurement aid (the paper has no counterpart).
 * cvweno_mesh_set_kernel_timing(m, 1) makes every following step of m (cvweno_step,
 * cvweno_advance) record a timing event before its first kernel and after each kernel
 * it launches; under stream capture the records become event-record nodes, so a graph
 * captured from such a step times each of its replays.  cvweno_kernel_times waits for
 * the last recorded event and writes the durations (ms) of the kernels of the most
 * recent step into ms[capacity] (host), in launch order: DG and Euler one per stage
 * (two with the HWENO or positivity limiter; with timing on, a one-tile 1D mesh also
 * launches stage by stage), CG two per stage in 2D (cells, then the
 * node phase: assembly and both defect-correction sweeps) and four in 1D (cells, node
 * right-hand side, two sweeps); *count receives how many were written.  Timing
 * costs one event record per kernel; turn it off (enable 0) for production runs.  Turning it off keeps the events
 * of the last timed step (and of graphs captured while it was on) readable. */
cvweno_status cvweno_mesh_set_kernel_timing(cvweno_mesh m, int enable);
cvweno_status cvweno_kernel_times(cvweno_mesh m, float* ms, int capacity, int* count);

/* Contraction form of the stage kernel.  enable = 1 runs the sensor's corner products
 * (stage (c): the four vertex candidates mapped into the cell's semi-norm coordinates,
 * Sec. 3.2 eq. finalweno with the semi-norm of Sec. 2.2 eq. snorm) on the tensor cores
 * (tcgen05, split TF32: hi*hi + hi*lo + lo*hi, FP32 accumulation), on 8 x 16 tiles;
 * enable = 0 (the default) runs them as FP32 FMAs on 16 x 8 tiles.  Both forms compute
 * the same stage to FP32 rounding.  2D DG scalar meshes of degree 3 only: returns
 * CVWENO_ERR_UNSUPPORTED for any other mesh when enable = 1, CVWENO_ERR_ARG for enable
 * other than 0 or 1.  A bounded wait for the tensor cores that gives up raises status
 * bit 4, reported as CVWENO_ERR_TIMEOUT at the next status check. */
cvweno_status cvweno_mesh_set_tensor_cores(cvweno_mesh m, int enable);

/* Bounds-checked build.  The library built with -DCVWENO_CHECK (libcvweno_check.so, same
 * entry points) checks, before each global load or store of a stage kernel (and each
 * shared-memory staging store whose offset follows the data's alignment), that the span
 * lies within its array: the state arrays within the mesh's nstate floats, the per-cell
 * outputs and work arrays within its cells.  A failed check skips the access and raises
 * status bit 8, reported as CVWENO_ERR_CHECK at the next status check; nothing traps.
 * This call narrows the extents those checks use for the mesh's later launches (so that
 * the checks themselves can be exercised without an out-of-bounds access):
 *   - state_floats: floats of u_in, u_n and u_out, 0 <= state_floats <= nstate;
 *   - cells: cells of the per-cell outputs, 0 <= cells <= the mesh's cell count;
 *   - both negative: back to the mesh's own extents.
 * Errors: CVWENO_ERR_ARG for a NULL mesh or a value above the mesh's own extent (or one
 * negative and the other not); CVWENO_ERR_UNSUPPORTED in the normal build, which has no
 * checks. */
cvweno_status cvweno_mesh_set_check_extents(cvweno_mesh m, int64_t state_floats, int64_t cells);

/* ---- batches of independent problems ------------------------------------------------
 * Many independent 2D DG meshes of uneven size and degree advanced together: each
 * SSP-RK3 stage of the whole batch is one persistent launch (or one per degree present),
 * and cvweno_batch_advance replays a captured CUDA graph of one step.  The per-mesh
 * arithmetic is that of cvweno_residual / cvweno_step on the same mesh; only the work
 * distribution differs.  The paper advances one problem at a time; batching is a
 * deployment form of its stage (a)-(e) residual.
 *
 * The state of instance k is u[offsets[k] .. offsets[k+1]) of ONE device array, in the
 * state layout of that instance's mesh (cvweno_state_size). */
typedef struct cvweno_batch_s* cvweno_batch;

enum { CVWENO_BATCH_FUSED = 0, CVWENO_BATCH_GROUPED = 1 };

/* Launch shape of a batch stage.  schedule: FUSED = one launch per stage whose CTAs
 * take tiles of every degree; GROUPED = one launch per degree present, forked onto
 * concurrent streams.  tile: 0 = 16x8 cells per CTA, 1 = 8x8.  dynamic: 1 = CTAs claim
 * tiles from a device counter (reset by the last CTA to leave), 0 = static
 * round-robin.  ctas_per_sm: persistent grid = ctas_per_sm x SM count, 0 = as many as
 * fit.  use_graph: cvweno_batch_advance replays a captured graph of one step.
 * ms (output of cvweno_batch_autotune): measured time of one residual pass. */
typedef struct {
  int schedule;
  int tile;
  int dynamic;
  int ctas_per_sm;
  int use_graph;
  float ms;
} cvweno_batch_plan;

/* Create a batch of count >= 1 meshes from descs[count] (host).  Every desc must be
 * 2D, DG, the same scalar system (BURGERS only), degree 1..4, with
 * square cells (dx == dy, so that one set of reference tabulations serves each
 * degree); other checks are those of cvweno_mesh_create.  Default plan: FUSED, 16x8,
 * dynamic, ctas_per_sm 0, use_graph 1.  Records the current device. */
cvweno_status cvweno_batch_create(const cvweno_mesh_desc* descs, int count, cvweno_batch* out);
cvweno_status cvweno_batch_destroy(cvweno_batch b);

/* offsets[count + 1] (host): start of each instance's state in the batch state array;
 * offsets[count] is the total length in floats. */
cvweno_status cvweno_batch_offsets(cvweno_batch b, int64_t* offsets);

/* Replace the launch shape; ERR_ARG for a field out of range. */
cvweno_status cvweno_batch_set_plan(cvweno_batch b, const cvweno_batch_plan* plan);
cvweno_status cvweno_batch_get_plan(cvweno_batch b, cvweno_batch_plan* plan);

/* Time every launch shape on the residual of state u (device, not modified) and keep
 * the fastest; *best (host, may be NULL) receives it.  Synchronises; not capturable. */
cvweno_status cvweno_batch_autotune(cvweno_batch b, const float* u, cvweno_batch_plan* best, void* stream);

/* dudt of every instance (stages (a)-(e) and M^-1), same layout as u; one stage launch
 * (or one per degree).  Enqueued without synchronisation. */
cvweno_status cvweno_batch_residual(cvweno_batch b, const float* u, float* dudt, void* stream);

/* nsteps SSP-RK3 steps of every instance in place, instance k with step dt[k] > 0
 * (host array of count).  Enqueued without synchronisation; with use_graph the first
 * call for a given u captures and instantiates the step graph. */
cvweno_status cvweno_batch_advance(cvweno_batch b, float* u, const double* dt, int nsteps, void* stream);

/* Synchronise, read and clear the per-instance status words.  *first_bad (host, may be
 * NULL) receives the lowest instance index with a raised status, or -1. */
cvweno_status cvweno_batch_status_check(cvweno_batch b, int* first_bad, void* stream);

/* ---- surrogate sensor ---------------------------------------------------------------
 * A small network estimates the sensor gamma_e (eq. gamma) from cell-vertex data.  The
 * paper has no learned component; the plain sensor is both its fallback and its judge.
 * Network: x (12) -> GELU(W1 x + b1) (64) -> GELU(W2 . + b2) (64) -> o = W3 . + b3 (2),
 * GELU in its tanh form; gamma_hat = sigmoid(o0), confidence = sigmoid(o1).
 * Parameters: one FP32 vector of 5,122 values, row-major W1 (64,12), b1 (64), W2 (64,64),
 * b2 (64), W3 (2,64), b3 (2).  Training reads inputs and weights rounded to bfloat16 and
 * computes in FP32; the loss per sample is (gamma_hat - gamma)^2 + 0.1 BCE(confidence, t)
 * with t = 1 iff |gamma_hat - gamma| < 0.05, averaged over the batch; Adam (0.9, 0.999,
 * 1e-8, bias-corrected).  Inference (stand-alone and fused into the stage kernel) runs
 * on the tensor cores with bfloat16 operands and activations, FP32 accumulation.
 * Inputs of a cell (2D DG scalar meshes), for its corners SW, SE, NW, NE in that order:
 * the vertex candidate's cell mean minus the cell mean, and h d_x, h d_y of the
 * candidate at the vertex, all over ||u^e||_e + eps (eq. snorm), clamped to [-8, 8]. */
typedef struct cvweno_mlp_s* cvweno_mlp;

/* params: host [5122] initial parameters (NULL: zeros).  Records the current device. */
cvweno_status cvweno_mlp_create(const float* params, cvweno_mlp* out);
cvweno_status cvweno_mlp_destroy(cvweno_mlp n);

/* The FP32 master parameters into params (host [5122]).  Synchronous. */
cvweno_status cvweno_mlp_get_params(cvweno_mlp n, float* params);

/* Mean loss and gradient over the count samples X (device [count][12]), gamma targets y
 * (device [count]).  loss and grad (host, [1] and [5122]) may be NULL; when either is
 * given the call synchronises.  The sum over samples runs in a fixed order. */
cvweno_status cvweno_mlp_loss_grad(cvweno_mlp n, const float* X, const float* y, int64_t count, float* loss,
                                   float* grad, void* stream);

/* One Adam step with the gradient of the last cvweno_mlp_loss_grad, learning rate lr. */
cvweno_status cvweno_mlp_adam_step(cvweno_mlp n, float lr, void* stream);

/* epochs passes over (X, y) in consecutive minibatches of `batch` samples (the caller
 * shuffles), one Adam step each.  last_loss (host, may be NULL) receives the mean loss of
 * the last minibatch (the call then synchronises). */
cvweno_status cvweno_mlp_train(cvweno_mlp n, const float* X, const float* y, int64_t count, int64_t batch,
                               int epochs, float lr, float* last_loss, void* stream);

/* Network outputs (o0, o1) before the sigmoids into out (device [count][2]), on the tensor
 * cores exactly as the fused stage kernel evaluates them. */
cvweno_status cvweno_mlp_infer(cvweno_mlp n, const float* X, int64_t count, float* out, void* stream);

/* The network inputs of every cell of u into feats (device [ncells][12]), the computed
 * sensor gamma_e (whatever sensor_mode says) into gamma and the semi-norm ||u^e||_e into
 * norm (device [ncells] each, may be NULL).  2D DG scalar meshes; ERR_UNSUPPORTED
 * otherwise. */
cvweno_status cvweno_features(cvweno_mesh m, const float* u, float* feats, float* gamma, float* norm,
                              void* stream);

/* Attach network n (NULL detaches) to mesh m: from then on the stage kernels of m take
 * gamma_e = gamma_hat where confidence >= conf_min, and the plain sensor elsewhere; cells
 * whose ||u^e||_e is at most 1e-5 (|cell mean| + 1) (rounding-level variation) take
 * gamma_e = 1 without the network.  The mesh reads n's weights at
 * every launch: n must outlive its use by m.  Training n after attaching takes effect at
 * the next launch.  2D DG scalar meshes. */
cvweno_status cvweno_mesh_set_surrogate(cvweno_mesh m, cvweno_mlp n, float conf_min);

/* Cells that fell back to the plain sensor since the last reset, over every mesh n is
 * attached to (device counter read back: synchronises); reset != 0 zeroes it. */
cvweno_status cvweno_mlp_fallbacks(cvweno_mlp n, uint64_t* count, int reset, void* stream);

/* One SSP-RK3 step of fixed size dt > 0, in place on the caller's state u (device,
 * state layout of desc), that allocates nothing -- for callers that cannot allocate
 * device or host memory (a library running inside an arena or memory pool it does not
 * own, or an embedding that forbids cudaMalloc after start-up).  It needs no mesh
 * handle: the tabulations are built on the host stack (by the same builder that
 * cvweno_mesh_create uses, so the step equals cvweno_step on that mesh bit for bit), and
 * the two RK stage buffers, the status word and the device copy of the tabulations live
 * in file-scope __device__ storage of fixed size (2 x 4,194,304 floats = 32 MiB, plus
 * under 16 KiB), held on every GPU where it has been created until the process exits.
 * The paper has no counterpart; this is a deployment variant of cvweno_step.
 *   - Argument checks and codes are those of cvweno_mesh_create, in its order.  Beyond
 *     them this variant returns CVWENO_ERR_UNSUPPORTED for CG meshes and for
 *     hweno_limiter = 1 or positivity = 1, and CVWENO_ERR_ARG for states larger than
 *     4,194,304 floats (ncells x (p+1)^dim x nvars).
 *   - The first call on a device looks up the device addresses of that storage with
 *     the device current.  Under CUDA's lazy module loading (the default) that first
 *     call is also when the 32 MiB come into existence on the device: make it at
 *     start-up, before reserving an arena of all free memory and before any stream
 *     capture (or set CUDA_MODULE_LOADING=EAGER).  The addresses are kept for the
 *     process: do not call it across a cudaDeviceReset of the device.
 *   - Every call shares the same storage: calls that overlap on the GPU (different
 *     streams, or different host threads) race and corrupt each other's stages.
 *   - status_out (host, may be NULL): when given, the call synchronises the stream and
 *     stores the device status bits of this step (1 non-finite, 2 non-positive density
 *     or pressure, 8 a failed bounds check of the checked build), returning
 *     CVWENO_ERR_NONFINITE / CVWENO_ERR_POSITIVITY / CVWENO_ERR_CHECK accordingly;
 *     when NULL the call only enqueues work. */
cvweno_status cvweno_step_static(const cvweno_mesh_desc* desc, float* u, double dt, int32_t* status_out,
                                 void* stream);

/* The sine and cosine of the KPP flux (Sec. 5.3: f(u) = (sin u, cos u)), as the stage
 * kernels form them from a deviation d: the Maclaurin series for |d| <= 1, beyond it a
 * reduction d = k pi/2 + r (Cody and Waite) and the series for r.  For testing the FP32
 * forms against a reference.
 *   - d (device, float[n]): the arguments; out (device, float[2n]): sin d in out[0..n),
 *     cos d - 1 in out[n..2n).  Enqueued on `stream` (NULL: the default stream).
 * Errors: CVWENO_ERR_ARG for n < 0 or NULL pointers with n > 0; CVWENO_ERR_CUDA if the
 * launch fails. */
cvweno_status cvweno_kpp_sincos(const float* d, float* out, int n, void* stream);

/* Static description of a status code.  (Error reporting; no passage of the paper.) */
const char* cvweno_status_string(cvweno_status s);

#ifdef __cplusplus
}
#endif

#endif /* CVWENO_H */

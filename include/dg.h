/*
 * dg.h -- C ABI of the GB300 (sm_103a) modal discontinuous Galerkin solver for
 * the 2D compressible Euler equations on unstructured triangle meshes.
 *
 * The method is the one of Fuhry, Giuliani and Krivodonova, "Discontinuous
 * Galerkin methods on graphics processing units for nonlinear hyperbolic
 * conservation laws" (arXiv:1601.07944):
 *   - weak form on each triangle mapped to the reference triangle
 *     {(0,0),(1,0),(0,1)} (Section 2, Eqs. 2ddg, weak2dsys, 2dmap);
 *   - orthonormal modal basis with N_p = (p+1)(p+2)/2 functions (Eq. np), so
 *     the mass matrix is the identity and dc/dt = (volume - surface)/det J
 *     (Eq. 2ddg0);
 *   - volume integral against the basis gradients (Eq. volume, Algorithm 1);
 *   - edge integral of a numerical flux computed once per edge from the traces
 *     of both elements, the right element's points taken in reverse order
 *     (Eqs. surface, edgeint, Algorithm 2), combined per element (Algorithm 3);
 *   - Euler flux with p = (gamma-1)(E - rho|v|^2/2) (Eq. euler, Section 5).
 * Choices this library fixes where the paper leaves them open: the Dubiner
 * basis (collapsed coordinates, ordered by total degree then by the second
 * index), a collapsed Gauss-Jacobi volume rule with p+1 points per direction,
 * Gauss-Legendre edge rules with n_edge_pts points (default p+1, as in the
 * paper's Section 4.3.3), the local Lax-Friedrichs flux and the three-stage
 * SSP Runge-Kutta method (the paper's own classic RK2, read as Heun's method,
 * and RK4 are available through dg_rk_step_method).
 *
 * Conventions for every call:
 *   - Coefficient arrays are element-major, c[e][m][j]: element e, conserved
 *     variable m in (rho, rho u, rho v, E), mode j; float64, contiguous,
 *     N * 4 * N_p values.  They are DEVICE pointers owned by the caller unless a
 *     call says otherwise.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     asynchronous on it unless stated; a caller must not reuse an output before
 *     the stream has reached the call.
 *   - The mesh handle owns its geometry, basis tables and work buffers; calls on
 *     one handle must not overlap in time on different streams.  Calls that take
 *     a mesh run on the device it was created on, which must be the calling
 *     thread's current device (DG_EINVAL otherwise).
 *   - No call aborts.  Every call returns a dg_status; on failure
 *     dg_last_error() returns a message for the calling thread.
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mesh dg_mesh;     /* opaque, library-owned */

typedef enum {
    DG_OK = 0,
    DG_EINVAL = 1,      /* bad argument (null pointer, size, order out of range) */
    DG_ENOMEM = 2,      /* host or device allocation failed */
    DG_ECUDA = 3,       /* a CUDA runtime call failed (message says which) */
    DG_EMESH = 4,       /* mesh fails validation (orientation, neighbours, edges) */
    DG_ENONPHYS = 5,    /* non-physical state met (rho <= 0 or p <= 0) */
    DG_ETIMEOUT = 6,    /* a bounded device wait expired */
    DG_ENOTIMPL = 7     /* valid request this build does not implement */
} dg_status;

/* Arithmetic of the contractions (interpolation to quadrature points, projection
 * onto the basis and lifting of edge fluxes).  The Riemann flux, the Runge-Kutta
 * accumulation and the conserved totals are float64 in every mode. */
typedef enum {
    DG_FP64 = 0,        /* every operation in float64 */
    DG_TF32X1 = 1,      /* contractions on the tensor cores, one TF32 product, FP32 accumulate */
    DG_TF32X3 = 2       /* contractions as split 3xTF32 products, FP32 accumulate */
} dg_precision;

/* Explicit Runge-Kutta methods of dg_rk_step_method.  The paper integrates
 * Eq. 2ddg0 with classic explicit RK methods of order two and four (Section
 * 4.3.1); the three-stage SSP method is the default of dg_rk_step. */
typedef enum {
    DG_SSP_RK3 = 0,     /* three-stage SSP method, third order (Shu-Osher form) */
    DG_RK2 = 1,         /* Heun's method: u + dt/2 (k1 + k2), k2 = L(u + dt k1); second order */
    DG_RK4 = 2          /* the classical four-stage method, fourth order */
} dg_rk_method;

/* Boundary codes in dg_mesh_desc.nbr (Algorithm 2: on a boundary face a ghost
 * state takes the right trace's place in the numerical flux). */
enum {
    DG_BC_WALL = -1,    /* solid wall: U_g = (rho, m - 2 (m.n) n, E), the interior state mirrored */
    DG_BC_STATE = -2    /* a state prescribed at each boundary quadrature point (far field,
                           Dirichlet data), given with dg_set_boundary_state */
};

/* Volume quadrature (Section 4.3.2: the volume integrals of Eq. volume are
 * evaluated with a rule exact for polynomials of degree 2p). */
typedef enum {
    DG_RULE_COLLAPSED = 0,  /* (p+1)^2-point collapsed Gauss grid (Gauss-Legendre x
                               Gauss-Jacobi(1,0)), exact to degree 2p+1; the float64
                               element kernel sum-factorises on it */
    DG_RULE_SYMMETRIC = 1   /* fully symmetric rule of degree 2p with the paper's point
                               counts, 3 / 6 / 12 / 16 / 25 points at p = 1..5 (positive
                               weights, interior points), derived at mesh creation from
                               its moment conditions; contracted directly */
} dg_vol_rule;

/* Host description of a mesh; dg_mesh_create copies everything it needs. */
typedef struct {
    int64_t n_elem;             /* N >= 1 */
    const double *elem_xy;      /* HOST [N][3][2]: vertices, counter-clockwise (det J > 0).
                                   Periodic meshes store each element's coordinates
                                   unwrapped; the two copies of a shared edge must be
                                   translates of each other. */
    const int64_t *nbr;         /* HOST [N][3]: element across local face q, where local
                                   face q runs from vertex q to vertex (q+1) mod 3;
                                   DG_BC_WALL or DG_BC_STATE on a boundary face */
    const int8_t *nbr_face;     /* HOST [N][3]: that neighbour's local face index
                                   (ignored on a boundary face) */
    int p;                      /* polynomial degree, 1 <= p <= 5 */
    int n_edge_pts;             /* Gauss-Legendre points per edge; 0 = p+1 (the paper's rule).
                                   Supported: p+1, and p for p = 3 */
    double gamma;               /* ratio of specific heats (1.4 for air) */
    int vol_rule;               /* dg_vol_rule; 0 (DG_RULE_COLLAPSED) for a zeroed struct */
} dg_mesh_desc;

typedef struct {
    int64_t n_elem;             /* N */
    int64_t n_face;             /* number of distinct edges */
    int p, n_modes, n_vol_pts, n_edge_pts;
    double gamma;
    int64_t n_boundary_face;    /* boundary faces (the first ones of the edge list) */
} dg_mesh_info_t;

/* The mesh and its connectivity (Section 4.2; element maps Eq. 2dmap, edge lengths
 * Eq. len).  Validates the mesh (det J > 0; nbr[nbr[e][q]][nbr_face[e][q]] == e and the face
 * index maps back; the shared edge's endpoints are translates; boundary codes are
 * DG_BC_WALL or DG_BC_STATE), builds the edge list (boundary faces first, in
 * element order, as the paper sorts them), geometry and basis tables on the host
 * and copies them to the current CUDA device.  Synchronous.  *out receives a handle to free with dg_mesh_destroy.
 * The volume rule (vol_rule) is built here; a symmetric rule is derived from its
 * moment conditions (milliseconds).
 * Errors: DG_EINVAL (null pointers, p, n_edge_pts or vol_rule unsupported),
 * DG_EMESH, DG_ENOMEM, DG_ECUDA. */
dg_status dg_mesh_create(const dg_mesh_desc *desc, dg_mesh **out);

/* Frees the handle and its device memory (synchronises the device first).
 * A NULL handle is accepted.  (Resource management: no passage of the paper.) */
dg_status dg_mesh_destroy(dg_mesh *mesh);

/* Sizes of the discretisation (N_p of Eq. np, the volume and edge rules of
 * Sections 4.3.2-4.3.3, the edge count of Section 4.2).  info: HOST, written on
 * DG_OK.  Errors: DG_EINVAL (null pointers). */
dg_status dg_mesh_info(const dg_mesh *mesh, dg_mesh_info_t *info);

/* Physical points of the boundary faces' quadrature points (Eq. 1dmap at the
 * Gauss-Legendre edge nodes): xy[n_boundary_face][n_edge_pts][2], DEVICE, faces in
 * element order (element, then local face), points in the element's
 * counter-clockwise direction along the face.  Asynchronous. */
dg_status dg_boundary_points(const dg_mesh *mesh, double *xy, void *stream);

/* The state prescribed on the DG_BC_STATE faces (Algorithm 2's ghost state for
 * Dirichlet and far-field boundaries, Section 4.3.3): u[n_boundary_face][n_edge_pts][4]
 * conserved variables at the points of dg_boundary_points (DEVICE; entries of
 * wall faces are not read), copied into the mesh.  Required before dg_rhs or a
 * time step on a mesh with DG_BC_STATE faces (DG_EINVAL otherwise); the state is
 * constant in time.  Asynchronous. */
dg_status dg_set_boundary_state(dg_mesh *mesh, const double *u, void *stream);

/* Physical coordinates of the volume quadrature points (Eq. 2dmap applied to the
 * reference rule): xy[N][n_vol_pts][2], DEVICE.  Asynchronous. */
dg_status dg_volume_points(const dg_mesh *mesh, double *xy, void *stream);

/* Values of the solution U = sum_j c_j phi_j (Section 2) at npts reference points
 * (r[k], s[k]) of every element: out[e][k][m], DEVICE [N][npts][4].  r, s are
 * HOST arrays (points inside the reference triangle {(0,0),(1,0),(0,1)}); the
 * basis table at the points is built on the host and copied to a temporary
 * device buffer.  Synchronous (the table is freed before returning). */
dg_status dg_eval_points(dg_mesh *mesh, int npts, const double *r, const double *s, const double *c,
                         double *out, void *stream);

/* det J of every element (twice its area; the Jacobian of Eq. 2dmap):
 * detj[N], DEVICE.  Asynchronous. */
dg_status dg_det_j(const dg_mesh *mesh, double *detj, void *stream);

/* Physical points of npts reference points (r[k], s[k]) in every element
 * (Eq. 2dmap): xy[N][npts][2], DEVICE.  r, s: HOST (inside the reference
 * triangle; DG_EINVAL otherwise).  Synchronous (a temporary device copy of the
 * points is freed before returning). */
dg_status dg_map_points(const dg_mesh *mesh, int npts, const double *r, const double *s, double *xy,
                        void *stream);

/* L2 error of variable var (0..3) of the solution U = sum_j c_j phi_j against
 * given values on a reference rule (r[k], s[k], w[k]) whose weights sum to 1/2
 * over the reference triangle:
 *   err = sqrt( sum_e det J_e sum_k w_k (U_var(r_k) - exact[e][k][var])^2 ),
 * the sum in a fixed order (bitwise repeatable).  r, s, w: HOST [npts];
 * c: DEVICE [N][4][N_p]; exact: DEVICE [N][npts][4] (for example an exact
 * solution evaluated at the points of dg_map_points); err: HOST double.
 * Synchronous (temporary device buffers are freed before returning). */
dg_status dg_l2_error(const dg_mesh *mesh, int npts, const double *r, const double *s, const double *w,
                      const double *c, const double *exact, int var, double *err, void *stream);

/* L2 projection of point values onto the orthonormal basis (Section 2, the
 * initial data u_0):  c[e][m][j] = sum_k w_k u[e][k][m] phi_j(r_k), with u the
 * conserved state at the points returned by dg_volume_points.
 * u: DEVICE [N][n_vol_pts][4]; c: DEVICE [N][4][N_p].  Asynchronous. */
dg_status dg_project_ic(dg_mesh *mesh, const double *u, double *c, void *stream);

/* Right-hand side of Eq. 2ddg0: r = (volume integral - surface integral)/det J for
 * every element, mode and variable, with the local Lax-Friedrichs flux
 *   F_hat = (F(U_l).n + F(U_r).n)/2 - alpha (U_r - U_l)/2,
 *   alpha = max(|v_l.n| + c_l, |v_r.n| + c_r),
 * evaluated once per edge.  c, r: DEVICE [N][4][N_p], must not alias.
 * Asynchronous. */
dg_status dg_rhs(dg_mesh *mesh, const double *c, double *r, dg_precision prec, void *stream);

/* Same result as dg_rhs, for callers that cannot allocate device memory when
 * they call it (for example a host whose device memory is all reserved by another
 * allocator, or a time-critical loop that must not allocate).  The paper has no
 * counterpart: this is a service of the library, not a step of the method.
 * The call allocates nothing.  Its work space (edge traces and edge fluxes,
 * N*3*n_edge_pts*4 + n_face*n_edge_pts*4 doubles) comes from one static device
 * array of 8,388,608 doubles (64 MiB) that every GPU loading this library keeps
 * until the process exits; larger meshes are rejected with DG_EINVAL and a
 * message giving both sizes (use dg_rhs for them).  The first call on a device,
 * made with that device current, looks up the array's device address; make it
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (every slot is written before it is read, so nothing
 * needs clearing); calls that overlap on the GPU, on any stream or thread, race
 * on it.  The current device must be the mesh's device.  The cached address
 * assumes that the device's context is not reset (cudaDeviceReset) while the
 * library stays loaded.  Its launches are not recorded by dg_set_timing.
 * c, r: DEVICE [N][4][N_p], must not alias.  Asynchronous. */
dg_status dg_rhs_noalloc(dg_mesh *mesh, const double *c, double *r, dg_precision prec, void *stream);

/* Time integration of Eq. 2ddg0 (Section 4.3.1; the paper uses classic RK2/RK4,
 * this entry point the SSP method, dg_rk_step_method the paper's): nsteps steps
 * of the three-stage SSP Runge-Kutta method (Shu-Osher form),
 *   u1 = u + dt L(u),  u2 = 3/4 u + 1/4 (u1 + dt L(u1)),
 *   u <- 1/3 u + 2/3 (u2 + dt L(u2)),
 * in place on c (DEVICE [N][4][N_p]).  The stage accumulation is float64 in every
 * precision mode.  Asynchronous.  Long calls replay whole chunks of 16 steps as a
 * CUDA graph, captured once per (c, dt, precision) on an internal stream that is
 * ordered after, and then before, `stream` with events. */
dg_status dg_rk_step(dg_mesh *mesh, double *c, double dt, int nsteps, dg_precision prec,
                     void *stream);

/* nsteps steps of the Runge-Kutta method `method` (see dg_rk_method) in place on c
 * (DEVICE [N][4][N_p]); dg_rk_step is this call with DG_SSP_RK3.  Heun's method
 * runs as u1 = u + dt L(u), u <- 1/2 u + 1/2 (u1 + dt L(u1)); the classical RK4
 * (Section 4.3.1) keeps the running sum u + dt sum_i b_i k_i of its stages in a
 * work array of the mesh (N * 4 * N_p doubles, allocated by the first DG_RK4 call
 * on the handle: make that call before any stream capture).  Each stage is one
 * edge-flux launch and one element launch in every precision mode; the stage
 * accumulation is float64.  Asynchronous; graph replay as for dg_rk_step, keyed
 * also by the method.  Errors: DG_EINVAL (unknown method or precision, nsteps < 0,
 * dt not finite), DG_ENOMEM (the RK4 work array), DG_ECUDA. */
dg_status dg_rk_step_method(dg_mesh *mesh, double *c, double dt, int nsteps, dg_rk_method method,
                            dg_precision prec, void *stream);

/* The fused small-mesh stepper (Section 7.1 finds small meshes bound by kernel
 * launches): on a mesh whose elements fit, in tiles of 4 or 8, in the blocks
 * of one wave of the GPU (at most 4 per SM), a float64 dg_rk_step or
 * dg_rk_step_method call runs the traces of the state and then every stage of
 * all nsteps steps in one cooperative launch, the edge, element and (with
 * dg_set_limiter on) limiter phases of each stage separated by a barrier over
 * the grid (bounded: a wait longer than 2 s records DG_ETIMEOUT for
 * dg_device_status).  The phases run the same code as the separate launches,
 * so the results are bitwise equal.  enable = 0 makes such calls use the
 * separate launches (and CUDA graphs) as on larger meshes; on by default.
 * Errors: DG_EINVAL (null mesh). */
dg_status dg_set_small_mesh_stepper(dg_mesh *mesh, int enable);

/* Barth-Jespersen limiter for p = 1 (Section 4.3.5, Eqs. limit, limitmax,
 * limitmin), in place on c (DEVICE [N][4][3]), variable by variable:
 *   U_i(r) = Ubar_i + alpha_i grad U_i . (r - r_i),
 * Ubar_i the centroid value, U^max / U^min the largest / smallest centroid value
 * of element i and its three neighbours, and alpha_i the smallest over the edge
 * integration points of min(1, (U^max - Ubar_i)/d) where d = U_i(r_qk) - Ubar_i > 0,
 * min(1, (U^min - Ubar_i)/d) where d < 0 (the standard Barth-Jespersen ratio; the
 * paper names the limiter and its bounds).  The linear modes are multiplied by
 * alpha_i; the means are unchanged.  Errors: DG_EINVAL unless p = 1.
 * Asynchronous. */
dg_status dg_limit(dg_mesh *mesh, double *c, void *stream);

/* enable != 0: dg_rk_step and dg_rk_step_method limit every intermediate stage
 * value and the new state with dg_limit's limiter, as the paper does (Section
 * 4.3.1); float64 path only (the mixed modes then return DG_ENOTIMPL, and so does
 * dg_adjoint_step).  Off by default.  Errors: DG_EINVAL if enable and p != 1. */
dg_status dg_set_limiter(dg_mesh *mesh, int enable);

/* Same as dg_rk_step (Section 4.3.1) with c in HOST memory (pinned memory gives
 * the fastest copies): copies c to the device, takes nsteps steps and copies the
 * result back into c.  When c is page-locked memory the device can reach
 * (cudaPointerGetAttributes: cudaMemoryTypeHost) and the call is float64
 * without the limiter on a mesh the fused small-mesh stepper does not take, the
 * first kernel reads c in place and makes the device copy itself, and the copy
 * back runs in chunks behind the last stage on a second stream of the handle
 * (the same results).  Errors as dg_rk_step, and DG_ENOMEM if the device copy of
 * the state cannot be allocated (first call on the handle).  Synchronous. */
dg_status dg_rk_step_host(dg_mesh *mesh, double *c_host, double dt, int nsteps,
                          dg_precision prec, void *stream);

/* Discrete adjoint of dg_rhs (float64; the transpose, step by step, of Eq. 2ddg0
 * and Algorithms 1-3 -- the paper has no adjoint): out = (dR/dc)^T lam, the transpose of the
 * RHS Jacobian at c applied to lam, taken backwards through the edge traces,
 * the Lax-Friedrichs flux (same kink conventions as dg_adjoint_step; on a
 * boundary face through the ghost state: a wall's ghost is the reflected trace,
 * a prescribed ghost is constant), the lift, the volume integral and the 1/det J
 * scaling.  All arrays DEVICE [N][4][N_p]; out must not alias c or lam.
 * Asynchronous. */
dg_status dg_rhs_adjoint(dg_mesh *mesh, const double *c, const double *lam, double *out, void *stream);

/* Discrete adjoint of one SSP-RK3 step (float64; the transpose of dg_rk_step's
 * stages, Section 4.3.1, and of dg_rhs_adjoint's RHS): given the state c_n at the start
 * of the step and lam_np1 = dJ/dc_{n+1}, writes lam_n = dJ/dc_n = (d c_{n+1}/d c_n)^T
 * lam_np1.  The stages are recomputed from c_n.  At a tie of the two wave speeds in
 * alpha the derivative follows the left trace (at a wall the two always tie), and
 * d|x|/dx at x = 0 is taken as 0.  Not with the limiter on (DG_ENOTIMPL).
 * All arrays DEVICE [N][4][N_p]; lam_n must not alias the others.  Asynchronous. */
dg_status dg_adjoint_step(dg_mesh *mesh, const double *c_n, double dt, const double *lam_np1,
                          double *lam_n, void *stream);

/* One float64 SSP-RK3 step of dg_rk_step on c (DEVICE [N][4][N_p], in place)
 * that also writes its two stage values, u1 = c + dt R(c) and
 * u2 = 3/4 c + 1/4 (u1 + dt R(u1)) (Section 4.3.1's stages in Shu-Osher form),
 * into u1 and u2 (DEVICE [N][4][N_p], caller-owned, distinct from c and from each
 * other): the same launches as dg_rk_step, so c comes out with the same bits,
 * and the stage values are those dg_adjoint_step would recompute.  For a
 * backward pass that keeps them (dg_adjoint_step_stages).  Errors: DG_EINVAL
 * (null or aliased buffers, dt not finite, boundary state missing), DG_ENOTIMPL
 * with the limiter on.  Asynchronous. */
dg_status dg_rk_step_stages(dg_mesh *mesh, double *c, double dt, double *u1, double *u2, void *stream);

/* dg_adjoint_step with the step's stage values given (as dg_rk_step_stages
 * writes them) instead of recomputed: the reverse sweep alone, three transposed
 * RHS applications.  The same result, bit for bit, as dg_adjoint_step on c_n.
 * lam_n must not alias the inputs.  Errors as dg_adjoint_step.  Asynchronous. */
dg_status dg_adjoint_step_stages(dg_mesh *mesh, const double *c_n, const double *u1, const double *u2,
                                 double dt, const double *lam_np1, double *lam_n, void *stream);

/* A stable time step (the paper gives none; Section 4.3.1 computes one with a
 * reduction): dt = cfl * r_min / ((2p+1) * s_max), with r_min the smallest
 * inscribed radius (twice the area over the perimeter) of the mesh and s_max the
 * largest |v| + c of the solution c over the volume quadrature points (an exact,
 * order-free maximum).  c: DEVICE.  *dt_out: HOST.  DG_ENONPHYS if rho <= 0 or
 * p <= 0 at a point.  Synchronous. */
dg_status dg_stable_dt(dg_mesh *mesh, const double *c, double cfl, double *dt_out, void *stream);

/* Domain integrals of the conserved variables (Section 2: the basis of Eq. np is
 * orthonormal with phi_1 = sqrt(2) constant),
 *   T_m = sum_e int_{Omega_e} U_m = sum_e det J_e c[e][m][0] / sqrt(2)
 * (only the constant mode has a non-zero mean), as a fixed-order float64
 * reduction, so repeated calls give bitwise equal results.  c: DEVICE.
 * out: HOST double[4].  Synchronous on stream. */
dg_status dg_conserved_totals(dg_mesh *mesh, const double *c, double out[4], void *stream);

/* ---- diagnostics ---------------------------------------------------------- */

/* Kernel kinds reported by dg_kernel_times. */
enum {
    DG_K_TRACES = 0,    /* edge traces of a coefficient array */
    DG_K_FACE = 1,      /* Lax-Friedrichs flux, one thread per edge point */
    DG_K_ELEMENT = 2,   /* volume + lift + 1/det J + stage update (+ next traces) */
    DG_K_PROJECT = 3,   /* L2 projection of point data */
    DG_K_TOTALS = 4,    /* conserved totals reduction */
    DG_K_ADJOINT = 5,   /* adjoint kernels */
    DG_K_OTHER = 6,
    DG_K_STEPPER = 7,   /* fused small-mesh stepper: every stage of a call in one launch */
    DG_NKINDS = 8
};

/* Per-kernel timing, for the kernel runtime distribution of Section 6.1: when
 * enable != 0, every kernel this library launches for the mesh is bracketed by a
 * pair of CUDA events recorded on the launch's own stream.  Enabling or
 * disabling clears the accumulated times.  Errors: DG_EINVAL (null mesh). */
dg_status dg_set_timing(dg_mesh *mesh, int enable);

/* The runtime distribution of Section 6.1: waits for the recorded events and adds
 * their durations, per kernel kind, to ms[DG_NKINDS] and launches[DG_NKINDS] (HOST
 * arrays, overwritten with the totals since timing was enabled).  Errors:
 * DG_EINVAL (null pointers), DG_ECUDA.  Synchronous. */
dg_status dg_kernel_times(dg_mesh *mesh, double ms[8], int64_t launches[8]);

/* The arithmetic peak that Section 6.4's throughput figures are measured against:
 * the device's sustained fused multiply-add rate in float64 and float32
 * (TFLOP/s, 2 flops per FMA) with a register-resident FMA chain over every SM,
 * timed with CUDA events on stream.  Either output may be NULL.  Errors:
 * DG_ECUDA (including a failed scratch allocation).  Synchronous; allocates a
 * small scratch buffer. */
dg_status dg_probe_fma_rate(double *fp64_tflops, double *fp32_tflops, void *stream);

/* Failure detection (no passage of the paper): synchronises stream and reports
 * device-side failures recorded since the last call: DG_EMESH if a kernel of a library built with DG_DEBUG read a connectivity
 * index out of range (it then used index 0 instead; other builds do not check);
 * DG_ETIMEOUT if a bounded wait of the mixed-precision kernels expired (the
 * kernel then skipped its remaining work and released its resources);
 * DG_ENONPHYS if a kernel met rho <= 0 or p <= 0 (or NaN) at a volume or edge
 * quadrature point (the results of that call are then meaningless).  The record
 * is cleared.  Synchronous. */
dg_status dg_device_status(dg_mesh *mesh, void *stream);

/* Device self-check (no passage of the paper) of two arithmetic helpers the
 * kernels use to spare the narrow float64 pipe: on 2^20 values over the float32 normal range (both signs,
 * exact rounding ties, zeros) it counts
 *   mismatches[0]: integer float64 -> float32 conversions (round to nearest even)
 *                  that differ bit for bit from the hardware conversion,
 *   mismatches[1]: integer float32 -> float64 conversions that differ,
 *   mismatches[2]: Newton-refined reciprocals more than 1 ulp from 1/x,
 *   mismatches[3]: Newton-refined square roots more than 1 ulp from sqrt(x),
 *                  or reciprocal square roots more than 2 ulp from 1/sqrt(x)
 *                  (the sound speeds of the edge flux and of its adjoint).
 * HOST int64_t[4].  Synchronous; allocates 32 bytes. */
dg_status dg_self_test(int64_t mismatches[4], void *stream);

/* Message for the last failing call on this thread ("" if none). */
const char *dg_last_error(void);

/* Host-only (needs no GPU): the reference rules (the collapsed volume grid and
 * the Gauss-Legendre edge rule of Sections 4.3.2-4.3.3) and the basis tables of
 * Eq. np this library uses for degree p with ne edge points.  Any pointer may be
 * NULL.  Errors: DG_EINVAL (p outside 0..8, ne outside 1..16).
 *   vol_r, vol_s, vol_w [nq] with nq = (p+1)^2;  edge_x, edge_w [ne];
 *   phi, dphi_r, dphi_s [nq][N_p] at the volume points;  phi_face [3][ne][N_p]
 *   at the edge points of local faces 0, 1, 2 (edge point order: xi ascending,
 *   face q running from reference vertex q to vertex q+1). */
dg_status dg_host_tables(int p, int ne, double *vol_r, double *vol_s, double *vol_w,
                         double *edge_x, double *edge_w, double *phi, double *dphi_r,
                         double *dphi_s, double *phi_face);

/* Host-only (needs no GPU): the volume rule of kind `rule` (dg_vol_rule; the
 * degree-2p rules of Section 4.3.2 with Section 6.1's point counts for
 * DG_RULE_SYMMETRIC) for degree p, as dg_mesh_create builds it.  *nq receives the point count (may be
 * read first with r = s = w = NULL); r, s, w [*nq] receive the reference points
 * and weights (sum 1/2), and phi [*nq][N_p] the basis at the points (any of them
 * may be NULL).  Symmetric rule point order: the orbits S3, S21, S111 in the
 * library's order, an S21 orbit with parameter a as (a, a), (a, 1-2a), (1-2a, a),
 * an S111 orbit (a, b), c = 1-a-b, as (a, b), (b, a), (a, c), (c, a), (b, c), (c, b).
 * Errors: DG_EINVAL (p outside 1..5, unknown rule, nq null). */
dg_status dg_volume_rule(int p, int rule, int *nq, double *r, double *s, double *w, double *phi);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */

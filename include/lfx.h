/*
 * lfx - one semi-implicit BDF time step of incompressible Navier-Stokes with P1-P1 elements,
 * VMS-LES stabilisation and static resistive immersed surfaces, on one GPU (sm_103a).
 *
 * The operation is the fully discrete problem of Section 2.3, Eq.
 * (fullydiscrete_ns_ale_riis_vmsles_quasistatic_unified), with the stabilisation terms of
 * Eqs. (stabilization_form_SUPG), (stabilization_form_VMS), (stabilization_form_LES)
 * (semi-implicit), the stabilisation parameters tau_M, tau_C of Section 2.3, the resistive term
 * of Eq. (riis), the boundary conditions of Section 2.2 and the block linear solve of Section
 * 2.4 (GMRES preconditioned by aSIMPLE, here with Jacobi/Chebyshev smoothing on the device).
 *
 * Conventions for every call:
 *  - Return value: LFX_OK (0) or a negative lfx_status; lfx_last_error() then holds a message
 *    for the calling thread.  No call aborts the process.
 *  - Node numbering at the interface is the caller's; the library renumbers internally and
 *    translates on input and output.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Handles are owned by the
 *    caller and released with the matching *_destroy.  A state borrows its problem, a problem
 *    borrows its mesh: destroy in reverse order.
 *  - Calls on one state are not reentrant; distinct states may be stepped from one thread on
 *    different streams.
 *  - Units are the caller's (the library is unit-agnostic).
 */
#ifndef LFX_H
#define LFX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lfx_status;
enum {
  LFX_OK = 0,
  LFX_ERR_INVALID_ARG = -1,   /* null pointer, size out of range, unknown enum value         */
  LFX_ERR_BAD_MESH = -2,      /* index out of range, zero-volume tetrahedron                 */
  LFX_ERR_OOM = -3,           /* device or host allocation failed                            */
  LFX_ERR_NOT_CONVERGED = -4, /* linear solve hit its iteration cap; the step was still taken */
  LFX_ERR_NONFINITE = -5,     /* NaN/Inf detected in a residual norm                         */
  LFX_ERR_CUDA = -6,          /* a CUDA runtime call failed                                  */
  LFX_ERR_TIMEOUT = -7,       /* a bounded device-side wait gave up                          */
  LFX_ERR_BUDGET = -8         /* serving: request does not fit the device-memory budget      */
};

/* Message of the last failed call on this thread ("" if none).  Valid until the next call. */
const char *lfx_last_error(void);
/* sizeof() of a public struct by name ("lfx_bc", "lfx_options", ...), -1 if unknown; lets a
 * binding check its struct layouts without a GPU. */
int64_t lfx_sizeof(const char *type_name);
/* Total number of CUDA kernels this library has launched in the process (diagnostic counter,
 * including kernels that returned early because a solve had already converged). */
int64_t lfx_launch_count(void);

/* ------------------------------------------------------------------------------------------
 * Mesh (Section 2.3: tetrahedral mesh T^h; Section 2.2: boundary subsets by tag)
 * ------------------------------------------------------------------------------------------ */
typedef struct lfx_mesh lfx_mesh;

/* nodes [n_nodes][3] FP64; tets [n_tets][4] int32 (any orientation: negatively oriented
 * tetrahedra are flipped and counted; zero volume -> LFX_ERR_BAD_MESH); bfaces [n_bfaces][3]
 * int32 with boundary_tags [n_bfaces] (any orientation; outward normals are recomputed).
 * Builds, once, on the host: the node and element renumbering (space-filling curve), the 4x4
 * block-CSR pattern of the node graph, the element -> block-slot map and an element colouring
 * such that no two elements of one colour share a node (atomic-free scatter).  Disconnected
 * pieces (several independent meshes passed together, "batching") are detected and numbered
 * contiguously; they are assembled by the same launches and solved as one block-diagonal
 * system.  Copies all inputs.  Needs no GPU: the device copies are made by the first
 * lfx_problem_create. */
lfx_status lfx_mesh_create(const double *nodes, int64_t n_nodes, const int32_t *tets,
                           int64_t n_tets, const int32_t *bfaces, const int32_t *boundary_tags,
                           int64_t n_bfaces, lfx_mesh **out);
void lfx_mesh_destroy(lfx_mesh *mesh);

typedef struct lfx_mesh_info {
  int64_t n_nodes, n_tets, n_bfaces;
  int64_t nnz_blocks;          /* 4x4 blocks in the pattern (diagonal included)              */
  int32_t n_colors;            /* element colours                                            */
  int32_t n_flipped;           /* tetrahedra whose orientation was fixed                     */
  int32_t max_color_size, min_color_size;
  int64_t n_bad_elements;      /* elements whose shape quality 6 sqrt2 |K| / e_rms^3 is below the
                                  default bad_element_quality (0.1): their geometry is FP64 in
                                  mixed assembly                                               */
  int32_t n_components;        /* connected components: independent meshes batched together  */
  int32_t pad;
} lfx_mesh_info;
lfx_status lfx_mesh_get_info(const lfx_mesh *mesh, lfx_mesh_info *info);

/* Pattern in the caller's node numbering, for inspection and tests: row_ptr [n_nodes+1],
 * col_idx [nnz_blocks] (sorted within each row).  Host buffers supplied by the caller. */
lfx_status lfx_mesh_get_pattern(const lfx_mesh *mesh, int64_t *row_ptr, int32_t *col_idx);
/* Element colours in the caller's element numbering [n_tets]. */
lfx_status lfx_mesh_get_colors(const lfx_mesh *mesh, int32_t *colors);
/* The chunk tables of the chunked assembly, for inspection and tests (host, no device work).
 * sizes = {chunks, chunk colours, passes, runs, slots per pass}.  Non-NULL arrays receive:
 * elem_old [n_tets] (caller element of each internal element), chunk_elem_off [chunks+1] (internal
 * element range of each chunk), chunk_color_off [colours+1] (chunk range of each colour; chunks of
 * one colour share no node), chunk_pass_off [chunks+1], pass_code [passes][slots per pass] (slot =
 * element-in-chunk << 4 | a << 2 | b for block (a, b) of that element, 0xffff idle), pass_run_off
 * [passes+1], run_meta [runs] (first slot | length << 8 | first-writer << 14 | diagonal << 15),
 * run_row, run_col [runs] (the run's matrix block as caller nodes; both or neither). */
lfx_status lfx_mesh_get_chunks(const lfx_mesh *mesh, int64_t sizes[5], int32_t *elem_old, int32_t *chunk_elem_off,
                               int32_t *chunk_color_off, int32_t *chunk_pass_off, uint16_t *pass_code,
                               int32_t *pass_run_off, uint16_t *run_meta, int32_t *run_row, int32_t *run_col);
/* The row tiles of the staged velocity smoothing pass, for inspection and tests (host, no device
 * work).  sizes = {tiles (0: the mesh has none, the plain pass runs), maximum rows per tile,
 * maximum blocks per tile}.  Non-NULL arrays receive tile_row [tiles+1] (the internal block-row
 * range of each tile) and row_node [n_nodes] (the caller node of each internal block row). */
lfx_status lfx_mesh_get_row_tiles(const lfx_mesh *mesh, int64_t sizes[3], int32_t *tile_row, int32_t *row_node);

/* ------------------------------------------------------------------------------------------
 * Problem: physics (Section 2.1), boundary conditions (Section 2.2), RIIS surfaces (Eq. riis),
 * numerics (Sections 2.3-2.4)
 * ------------------------------------------------------------------------------------------ */
enum { LFX_TIME_CONSTANT = 0, LFX_TIME_PULSATILE = 1, LFX_TIME_RAMP = 2, LFX_TIME_FOURIER = 3 };
#define LFX_MAX_FOURIER 16
/* g(t) of Section 2.2.1.  p[]: constant {value}; pulsatile {g_min, g_max, period};
 * ramp {g0, g1, t0, tL}; Fourier {period}: g = a[0] + sum_{k=1..K} a[k] cos(k w t) + b[k] sin(k w t),
 * w = 2 pi / period, K = n_harmonics <= LFX_MAX_FOURIER. */
typedef struct lfx_time_law {
  int32_t kind;
  int32_t n_harmonics;
  double p[4];
  double a[LFX_MAX_FOURIER + 1];
  double b[LFX_MAX_FOURIER + 1];
} lfx_time_law;

enum { LFX_BC_NOSLIP = 0, LFX_BC_DIRICHLET = 1, LFX_BC_NODAL = 2, LFX_BC_NEUMANN = 3, LFX_BC_RESISTANCE = 4 };
enum { LFX_PROFILE_UNIFORM = 0, LFX_PROFILE_PARABOLIC = 1, LFX_PROFILE_WOMERSLEY = 2 };
/* One boundary condition on the faces carrying `tag`.
 *  NOSLIP    u = 0 (fixed domain).
 *  DIRICHLET u = theta g(t) s(x) (Section 2.2.1): s = -n (uniform, unit velocity),
 *            s = -2 (R^2 - r^2)/(pi R^4) n (parabolic, unit flow rate, r = distance to the
 *            barycentre of the tagged faces), or the Womersley profile of unit flow rate per
 *            Fourier harmonic of g (needs time.kind == LFX_TIME_FOURIER).
 *  NODAL     u given per node and per step by lfx_set_dirichlet_nodal.
 *  NEUMANN   sigma n = -h(t) n (Eq. bcs-neumann), h = time law; h = 0 is the natural condition.
 *            With beta > 0, inertial backflow stabilisation (Section 2.2.2): + beta rho/2
 *            |u . n|_- u, semi-implicit: the matrix gains c (u, v) on the faces with
 *            c = -beta rho/2 min(u^EXT . n, 0), integrated at the three edge midpoints of each face.
 *  RESISTANCE sigma n = -(p_0(t) + resistance * int_Gamma u . n) n (Section 2.2.3), p_0 = time
 *            law: implicit, the linear operator carries the rank-one term resistance w w^T
 *            (w_{4a+i} = int_Gamma phi_a n_i) and p_0 enters like Neumann data.  Not available on
 *            meshes of several disconnected pieces (LFX_ERR_INVALID_ARG at state creation).
 * Where tags meet: NOSLIP > DIRICHLET/NODAL > NEUMANN/RESISTANCE.  center/normal: if
 * given_geometry is 0 they are computed as the area-weighted barycentre and outward normal of the
 * tagged faces.  beta must be >= 0, and 0 for kinds other than NEUMANN; resistance >= 0, and 0 for
 * kinds other than RESISTANCE (LFX_ERR_INVALID_ARG otherwise). */
typedef struct lfx_bc {
  int32_t tag, kind, profile, given_geometry;
  lfx_time_law time;
  double theta, radius;
  double center[3], normal[3];
  double beta;
  double resistance;
} lfx_bc;

enum { LFX_RIIS_DISK = 0, LFX_RIIS_SDF_NODAL = 1 };
/* Static resistive immersed surface (Eq. riis with u_ALE = u_Sigma = 0): resistance R, half
 * thickness eps.  DISK: flat disk (center, unit normal, radius); its signed distance is the
 * plane distance inside the rim and the signed distance to the rim circle outside.
 * SDF_NODAL: signed distance given at the nodes (caller numbering), copied.  Inside an element
 * the signed distance is the P1 interpolant of its nodal values. */
typedef struct lfx_riis {
  int32_t kind, pad;
  double resistance, eps;
  double center[3], normal[3], radius;
  const double *sdf_nodal;
} lfx_riis;

enum { LFX_PREC_FP64 = 0, LFX_PREC_MIXED = 1 };
enum { LFX_ASM_AUTO = 0, LFX_ASM_COLORS = 1, LFX_ASM_CHUNKS = 2, LFX_ASM_PERSISTENT = 3 };
/* Smoothers of the aSIMPLE blocks.  LFX_SMOOTH_AMG (Schur block only): one V-cycle of a
 * smoothed-aggregation AMG hierarchy of S = C - D diag(F)^-1 G, Chebyshev smoothing (s_steps
 * pre and post) on every level, dense solve on the coarsest. */
enum { LFX_SMOOTH_JACOBI = 0, LFX_SMOOTH_CHEBYSHEV = 1, LFX_SMOOTH_AMG = 2 };
enum { LFX_STAB_NONE = 0, LFX_STAB_SUPG_PSPG = 1, LFX_STAB_VMS_LES = 2 };
enum { LFX_DIFF_GRAD_GRAD = 0, LFX_DIFF_SYMGRAD_GRAD = 1, LFX_DIFF_SYMGRAD_SYMGRAD = 2 };

typedef struct lfx_options {
  /* discretisation */
  int32_t stab;                 /* LFX_STAB_*, default VMS-LES                                 */
  int32_t diffusion;            /* LFX_DIFF_*, default grad-grad (Eq. diffusion-term)          */
  double c_r;                   /* C_r in tau_M (not printed in the paper); default 30         */
  double f[3];                  /* constant body force f; default 0                            */
  int32_t pin_pressure_node;    /* caller node whose pressure is fixed (all-Dirichlet flows);
                                   -1 = none.  Value per step: lfx_set_pressure_pin.           */
  int32_t precision;            /* LFX_PREC_FP64 (default) or LFX_PREC_MIXED                   */
  /* linear solve: GMRES(restart) right-preconditioned by aSIMPLE */
  int32_t gmres_restart;        /* default 64                                                  */
  int32_t gmres_max_iters;      /* total Arnoldi steps cap; default 1000                       */
  double gmres_rtol;            /* stop when ||b - A x|| <= rtol ||b||; default 1e-10         */
  int32_t reorthogonalize;      /* classical Gram-Schmidt once (0, default) or twice (1); in mixed
                                   precision the FP32 inner solve orthogonalises twice only if 2  */
  /* aSIMPLE: velocity block F and Schur approximation S = C - D diag(F)^-1 G */
  int32_t f_smoother, f_steps;  /* LFX_SMOOTH_*, steps; default Chebyshev, 6                   */
  double f_omega, f_ratio;      /* Jacobi damping; Chebyshev lmax/lmin; default 0.7, 60        */
  int32_t s_smoother, s_steps;  /* default AMG with 1 Chebyshev step pre and post               */
  double s_omega, s_ratio;      /* default 0.7, 30                                             */
  int32_t n_power;              /* 0 (default): Chebyshev lmax = Gershgorin bound (holds for every
                                   eigenvalue); > 0: this many power-iteration steps x 1.1       */
  /* mixed precision (LFX_PREC_MIXED) */
  int32_t smoother_bf16;        /* store the preconditioner blocks in BF16 (FP32 arithmetic)   */
  int32_t outer_restart;        /* FP64 flexible GMRES restart; default 8                       */
  int32_t outer_max_iters;      /* default 40                                                   */
  double inner_rtol;            /* FP32 inner GMRES tolerance per outer step; default 1e-4.
                                   With inner_adaptive it is the tightest tolerance used      */
  int32_t inner_max_iters;      /* default 60                                                   */
  double bad_element_quality;   /* elements with 6 sqrt2 |K| / e_rms^3 below this keep FP64
                                   geometry in mixed assembly; default 0.1                       */
  /* Schur AMG (s_smoother == LFX_SMOOTH_AMG) */
  int32_t amg_refresh;          /* rebuild the hierarchy every this many steps (0 = build once) */
  int32_t amg_coarse_size;      /* dense solve below this many unknowns; default 2000          */
  double amg_theta;             /* strength threshold on coarse levels; default 0.08           */
  double amg_alpha;             /* scaling of the coarse correction; default 1.0               */
  /* batching: a mesh made of several disconnected meshes is stepped as one system.  With
   * batch_segmented (default 1) the Krylov solvers run one Arnoldi process per component in
   * lockstep (own Hessenberg matrix, rotations and stopping test ||r_c|| <= rtol ||b_c|| each,
   * shared launches), so every component takes about the steps it would take alone.  With
   * batch_segmented = 0 the union is one Krylov system, and batch_normalize (default 1) scales
   * each component's rows by 1/||its rhs|| every step so that the union's relative tolerance
   * approximates every component's own (a Schur AMG hierarchy built at an earlier step then
   * keeps that step's scale, which slows it when the scales drift) */
  int32_t batch_normalize;
  int32_t batch_segmented;
  /* mixed precision: each inner solve's tolerance from the outer flexible GMRES's residual
   * estimate r and its target tol = gmres_rtol ||b|| (default 1): 1/2 sqrt(tol / r) for the first
   * inner solve of an outer cycle (two outer steps reach tol), 1/2 tol / r for the later ones (this
   * step reaches it), kept within [inner_rtol, 0.1]; for a segmented batch the tightest over the
   * members still running */
  int32_t inner_adaptive;
  /* fully implicit formulation (Eq. u_star in its implicit form and the implicit LES term of
   * Section 2.3), linearised by Newton's method (Section 2.4): each step first solves the
   * semi-implicit system, then runs Newton iterations from that solution.  Each iteration
   * evaluates R(U) = A(U) U - b(U) with the semi-implicit system assembled at the iterate (u^EXT,
   * p^EXT := U), stops once ||R|| <= newton_rtol ||b|| (b: the step's semi-implicit right-hand
   * side; Dirichlet rows s (U_r - g_r)), and otherwise assembles the Jacobian of the element
   * residual (u* = u, tau_M(u*), tau_C(u*), r_M(u, p) at the iterate, derived analytically) with
   * the right-hand side J U - R(U) and solves for the next iterate with the configured Krylov
   * method.  Not with backflow stabilisation or resistance conditions (LFX_ERR_INVALID_ARG at
   * problem creation). */
  int32_t implicit;             /* 0 (default): semi-implicit; 1: fully implicit with Newton     */
  int32_t newton_max_iters;     /* default 10; the step returns LFX_ERR_NOT_CONVERGED past it   */
  /* assembly launch shape of the semi-implicit system: LFX_ASM_COLORS (one launch per element
   * colour, each CTA scattering its elements' blocks), LFX_ASM_CHUNKS (compact 32-element chunks,
   * their blocks reduced in shared memory and written once per chunk, one launch per chunk colour),
   * LFX_ASM_PERSISTENT (the chunks in one cooperative launch, colours separated by bounded grid-wide
   * waits; LFX_ERR_TIMEOUT from lfx_step if a wait gives up), or LFX_ASM_AUTO (default): the first
   * assembly on the problem times each of the three on the device (two assemblies each) and the
   * problem keeps the fastest for all its states (lfx_problem_assembly_tuning reports it).  The
   * Newton system of the fully implicit formulation is timed and chosen apart from it, at its own
   * first assembly, since its kernels fit the SMs differently. */
  int32_t assembly;
  double newton_rtol;           /* default 1e-10                                                 */
  /* velocity smoothing passes of the BF16 smoother (smoother_bf16 = 1): 1 (default) the staged
   * pass, whose persistent CTAs copy whole row tiles of F sub-blocks into shared memory with bulk
   * asynchronous copies while the previous tile is processed (LFX_ERR_TIMEOUT from lfx_step if a
   * bounded wait for a tile gives up); 0 the plain pass, each lane loading its blocks itself.  Both
   * compute the same sums in the same order. */
  int32_t staged_f;
  int32_t pad2;
} lfx_options;
void lfx_options_default(lfx_options *opt);

typedef struct lfx_problem lfx_problem;
/* rho, mu > 0 (Section 2.1.2), dt > 0, bdf_order 1..3 (Eq. bdf).  bcs [n_bcs], riis [n_riis]
 * (n_riis <= 8) are copied; opt may be NULL for defaults; n_bcs x (H + 1) <= 1024, where H = 1, or
 * 1 + 2 x (the largest number of Womersley harmonics).  Precomputes the Dirichlet profiles, the
 * Neumann load vectors, the nodal signed distances and every element's geometry, all resident on
 * the device (the mesh does not move). */
lfx_status lfx_problem_create(const lfx_mesh *mesh, double rho, double mu, double dt,
                              int32_t bdf_order, const lfx_bc *bcs, int32_t n_bcs,
                              const lfx_riis *riis, int32_t n_riis, const lfx_options *opt,
                              lfx_problem **out);
void lfx_problem_destroy(lfx_problem *problem);
/* The assembly launch shape of the problem (options.assembly, or the autotuner's choice once a state
 * of it has assembled; 0 before that) and the tuning times in ms per assembly of the three shapes
 * (ms[0..2] = colours, chunks, persistent; 0 where not timed).  Host-only. */
lfx_status lfx_problem_assembly_tuning(const lfx_problem *problem, int32_t *mode, float ms[3]);

/* ------------------------------------------------------------------------------------------
 * State: BDF history (u^n, ..., u^{n+1-sigma}; p likewise) resident on the device
 * ------------------------------------------------------------------------------------------ */
typedef struct lfx_state lfx_state;
/* u_hist [bdf_order][n_nodes][3], p_hist [bdf_order][n_nodes] (level 0 = u^n), t0 = t^n.
 * Host pointers, copied. */
lfx_status lfx_state_create(lfx_problem *problem, const double *u_hist, const double *p_hist,
                            double t0, lfx_state **out);
void lfx_state_destroy(lfx_state *state);
/* CUDA stream (cudaStream_t, NULL = legacy default stream) used by every later call on it. */
lfx_status lfx_set_stream(lfx_state *state, void *cuda_stream);

/* Per-step data for the next lfx_step: nodal Dirichlet values for one NODAL tag, u [n_nodes][3]
 * (caller numbering, only the tag's nodes are read), host pointer, copied. */
lfx_status lfx_set_dirichlet_nodal(lfx_state *state, int32_t tag, const double *u);
/* Pressure value at the pinned node (options.pin_pressure_node) for the next step. */
lfx_status lfx_set_pressure_pin(lfx_state *state, double value);

typedef struct lfx_step_stats {
  int32_t iterations;           /* Arnoldi steps (FP64 path) or inner steps summed (mixed)     */
  int32_t outer_iterations;     /* outer FGMRES steps (mixed), 0 for FP64                      */
  double rel_residual;          /* final ||b - A x|| / ||b|| (FP64)                            */
  double t;                     /* time reached                                                */
  float ms_assembly, ms_solve, ms_total;   /* device time per phase (CUDA events)              */
  int32_t converged;
  float ms_assembly_kernels;    /* the assembly kernel's launches alone (CUDA events)          */
  int32_t n_assembly_launches;  /* launches of the assembly kernel in this step: element colours,
                                   chunk colours, or 1 for the persistent launch                */
  float ms_spmv;                /* device time of a sample of the Arnoldi block SpMV launches of
                                   the (inner) Krylov solve in this step: one in five, at most four
                                   (CUDA events)                                                 */
  int32_t n_spmv;               /* their number (FP64 matrix on the FP64 path, FP32 in mixed)   */
  int32_t newton_iterations;    /* Newton updates taken (fully implicit formulation), else 0    */
  float ms_newton_assembly;     /* device time of the Newton loop's assemblies: the residual
                                   checks and the Jacobians (CUDA events)                        */
  int32_t n_fpass;              /* plain F passes of the preconditioner timed in this step (those
                                   of its first application)                                     */
  float ms_fpass_median;        /* their mean duration per pass (CUDA events)                     */
  int32_t assembly_mode;        /* LFX_ASM_* launch shape the step's assembly used                */
  int32_t reserved[2];
} lfx_step_stats;

/* One BDF step t^n -> t^{n+1}: BDF/EXT fields, coloured assembly of the linearised block system,
 * Neumann and Dirichlet data, the preconditioned Krylov solve, history shift; with
 * options.implicit, Newton iterations of the fully implicit formulation follow the semi-implicit
 * solve.  Arithmetic: FP64 on the FP64 path.  In mixed precision every element term is formed in
 * double-float arithmetic (pairs of FP32 numbers, 48-bit significand) and the matrix is stored as
 * FP32 high and low parts; elements below options.bad_element_quality take their geometry in FP64;
 * the RIIS delta and the right-hand side are FP64; the outer flexible GMRES works on FP64 vectors
 * with the double-float operator, the inner GMRES and aSIMPLE in FP32 (BF16 storage optional).
 * Returns LFX_ERR_NOT_CONVERGED after still advancing the state if a solve (or Newton) hit its
 * cap.  Every other error returns before the history is shifted, so the state keeps its time
 * level and history: after LFX_ERR_TIMEOUT (a bounded device wait gave up) the step can be
 * repeated as it is, after LFX_ERR_NONFINITE once lfx_state_set has replaced the history.
 * stats may be NULL. */
lfx_status lfx_step(lfx_state *state, lfx_step_stats *stats);

/* Newton residual history of the last step (fully implicit formulation): res[k] = ||R(U_k)|| /
 * ||b|| for the iterates U_0 (the semi-implicit solution), U_1, ...; *n entries, of which the first
 * min(*n, capacity) are written to the caller's host array.  0 entries for semi-implicit steps. */
lfx_status lfx_state_newton_residuals(const lfx_state *state, double *res, int32_t capacity, int32_t *n);

/* ------------------------------------------------------------------------------------------
 * Moving domain (arbitrary Lagrangian-Eulerian form, Sections 2.1-2.3): the mesh follows a
 * displacement d from the reference configuration x^ given at creation.
 * ------------------------------------------------------------------------------------------ */
/* Makes the state a moving-mesh state with the displacement levels d^n, d^{n-1}, ...:
 * d_hist [bdf_order][n_nodes][3] (caller numbering, host, copied).  Every later step then needs
 * lfx_set_boundary_displacement first.  The boundary conditions must be NOSLIP, NODAL or NEUMANN
 * without backflow stabilisation (LFX_ERR_INVALID_ARG otherwise; the Dirichlet profiles and the
 * resistance and backflow terms are tied to the reference configuration), on a mesh of one piece.
 * Builds, once, the lifting operator: the P1 Laplacian of the reference mesh (Eq. lifting, with
 * sigma^L = grad d, i.e. harmonic extension). */
lfx_status lfx_state_set_displacement(lfx_state *state, const double *d_hist);
/* The displacement d^{n+1} of the next step at n listed nodes (caller numbering; d [n][3], host,
 * copied).  lfx_step extends it into the domain by the lifting problem (Eq. lifting: K d = 0 on the
 * other nodes, zero normal flux on the rest of the boundary; conjugate gradients with Jacobi
 * scaling on the device, from d^n, to a relative residual of 1e-12), assembles the step on the
 * configuration x^ + d^{n+1} (element geometry and Neumann loads recomputed there) with the
 * advection velocity u* = u^EXT - u_ALE, u_ALE = (alpha d^{n+1} - sum_j beta_j d^{n-j}) / dt the BDF
 * derivative of the displacement (Eq. u_star; Section 2.3), and then shifts the displacement levels.
 * LFX_ERR_NOT_CONVERGED from lfx_step if the lifting does not converge in 20000 iterations. */
lfx_status lfx_set_boundary_displacement(lfx_state *state, int64_t n, const int32_t *nodes, const double *d);
/* The displacement of the current time level (after a step: d^{n+1}), d [n_nodes][3] caller
 * numbering, host; *lifting_iterations (nullable) = CG iterations of the last lifting. */
lfx_status lfx_state_get_displacement(const lfx_state *state, double *d, int32_t *lifting_iterations);

/* Replace the history (same layout as lfx_state_create) and the time; host pointers, copied
 * on the state's stream before the call returns. */
lfx_status lfx_state_set(lfx_state *state, const double *u_hist, const double *p_hist, double t);

/* Copy the latest solution to the host in caller numbering: u [n_nodes][3], p [n_nodes]. */
lfx_status lfx_state_get(const lfx_state *state, double *u, double *p);

/* ------------------------------------------------------------------------------------------
 * Building blocks of the step, exposed for parity tests (all act on the state's stream)
 * ------------------------------------------------------------------------------------------ */
/* Assemble the system of the next step (BDF/EXT + assembly + Neumann + Dirichlet) without
 * solving; then copy it out: block values [nnz_blocks][4][4] in the order of
 * lfx_mesh_get_pattern (caller numbering), rhs [n_nodes][4]. FP64 host buffers. */
lfx_status lfx_debug_assemble(lfx_state *state, int32_t apply_bcs, double *blocks, double *rhs);
/* The Newton system of the fully implicit formulation (options.implicit need not be set) at the
 * iterate U [n_nodes][4] (caller numbering, host): the Jacobian J(U) of the element residuals summed
 * (block values as in lfx_debug_assemble) and the right-hand side J(U) U - R(U) with the Neumann data,
 * both before Dirichlet rows; the BDF fields are those of the state's next step.  FP64 host buffers. */
lfx_status lfx_debug_assemble_newton(lfx_state *state, const double *U, double *blocks, double *rhs);
/* Failure path of the persistent assembly, for tests: one assembly with the first grid-wide wait's
 * target set out of reach and its poll limit at 4096, so that the wait runs out; every CTA then
 * returns.  LFX_ERR_TIMEOUT is the expected result; the state stays usable (the next lfx_step
 * assembles anew).  Needs a problem whose assembly is the persistent launch (options.assembly).  */
lfx_status lfx_debug_persistent_timeout(lfx_state *state);
/* Failure path of the staged velocity smoothing pass, for tests: assembles the next step's system,
 * then applies the BF16 aSIMPLE preconditioner once with every wait for a staged tile given no
 * polls, so that each wait runs out at once; each CTA waits (bounded) for its copies in flight and
 * returns.  LFX_ERR_TIMEOUT is the expected result; the state stays usable (the next lfx_step
 * assembles anew).  Needs a mixed-precision state with smoother_bf16 and staged_f set. */
lfx_status lfx_debug_staged_timeout(lfx_state *state);
/* y = A x with the last assembled matrix; x, y [n_nodes][4] FP64 host buffers, caller numbering. */
lfx_status lfx_debug_spmv(lfx_state *state, const double *x, double *y);
/* z = P^-1 r with the aSIMPLE preconditioner of the last assembled matrix (FP64 path);
 * r, z [n_nodes][4] host buffers, caller numbering.  Also returns the lambda_max values of
 * diag(F)^-1 F and diag(S)^-1 S that set the Chebyshev intervals. */
lfx_status lfx_debug_precond(lfx_state *state, const double *r, double *z, double *lam_f,
                             double *lam_s);
/* Solve the last assembled system (after lfx_debug_assemble with BCs) from x0 = 0 with the
 * configured Krylov method; x [n_nodes][4] host buffer. */
lfx_status lfx_debug_solve(lfx_state *state, double *x, lfx_step_stats *stats);

/* The Schur AMG hierarchy of the FP64 path (s_smoother == LFX_SMOOTH_AMG) as the device holds it
 * after its set-up (a step or lfx_debug_precond / lfx_debug_solve): level `level` >= 1 below the
 * matrix-free level 0.  sizes = {n_l, nnz(A_l), n_{l+1}, nnz(P_l)} (n_{l+1} = nnz(P_l) = 0 at the
 * coarsest level; nnz(A_l) = 0 there too, its dense inverse being all the device keeps; P_0 is
 * level 0's prolongator, reported with level = 0 and nnz(A_0) = 0).  If the array pointers are
 * non-NULL they receive A_l (a_rp [n_l+1], a_ci, a_v) and P_l (p_rp [n_l+1], p_ci, p_v), CSR with
 * int32 indices and FP64 values, and *lam the Gershgorin bound of lambda_max(D^-1 A_l) that sets
 * the level's Chebyshev interval.  Host buffers; LFX_ERR_INVALID_ARG before the set-up or for a
 * level out of range. */
lfx_status lfx_debug_amg_level(lfx_state *state, int32_t level, int64_t sizes[4], int32_t *a_rp,
                               int32_t *a_ci, double *a_v, int32_t *p_rp, int32_t *p_ci, double *p_v,
                               double *lam);
/* One device V-cycle of that hierarchy over levels 1 .. L-1 (the part below the matrix-free level
 * 0, run by the same launch as inside the preconditioner): x1 = V(b1), b1 and x1 [n_1] FP64 host
 * buffers in level-1 numbering.  Needs at least 3 levels. */
lfx_status lfx_debug_amg_vcycle(lfx_state *state, const double *b1, double *x1);

/* The same host set-up of the Schur AMG hierarchy, run on the host alone for a caller-held matrix
 * (no state, no device work: tests of the host logic run without a GPU).  The matrix is the 4x4
 * block-CSR system of a step in host memory: row_ptr [n_nodes+1], col_idx [nnz_blocks] (the node
 * graph, which also drives the finest aggregation), diag_idx [n_nodes] (position of block (i,i)),
 * blocks [nnz_blocks][4][4] FP64 row-major with unknowns (u_x, u_y, u_z, p) per node.  The set-up
 * forms S = C - D diag(F)^-1 G explicitly, then aggregates, smooths the prolongators, forms the
 * Galerkin coarse operators, their Gershgorin bounds and the dense inverse of the coarsest one,
 * with opt's amg_coarse_size and amg_theta (NULL = defaults).  It runs whole at every call and
 * reports level `level`: sizes = {levels, n_l, nnz(A_l), n_{l+1}, nnz(P_l)}, with n_{l+1} and nnz(P_l)
 * 0 at the coarsest level.  Non-NULL arrays receive A_l (a_rp [n_l+1], a_ci, a_v; A_0 = S), P_l
 * (p_rp [n_l+1], p_ci, p_v), *lam (the Gershgorin bound of lambda_max(D^-1 A_l), 0 at the coarsest
 * level) and, at the coarsest level, coarse_inv [n_l][n_l] (A_l^-1, row-major).  Host buffers,
 * CSR with int32 indices.  LFX_ERR_INVALID_ARG for NULL inputs, a pattern or diagonal index out of
 * range, or a level beyond the last. */
lfx_status lfx_debug_amg_host(int64_t n_nodes, const int32_t *row_ptr, const int32_t *col_idx,
                              const int32_t *diag_idx, const double *blocks, const lfx_options *opt,
                              int32_t level, int64_t sizes[5], int32_t *a_rp, int32_t *a_ci, double *a_v,
                              int32_t *p_rp, int32_t *p_ci, double *p_v, double *lam, double *coarse_inv);

/* ------------------------------------------------------------------------------------------
 * Allocation-free preconditioner application (the paper has no counterpart: this is a service
 * for callers that cannot allocate device memory where they need the preconditioner, e.g. a
 * solver embedded in a framework that owns all device memory through its own pool, or a
 * time-critical loop that must not pay for an allocation, which may synchronise the device, or
 * risk its failure midway).
 *
 * z = P^-1 r with the aSIMPLE preconditioner (the same kernels as lfx_step's) for a 4x4
 * block-CSR matrix the caller already holds on the device: row_ptr [n_nodes+1], col_idx
 * [nnz_blocks], diag_idx [n_nodes] (position of block (i,i)), trans_idx [nnz_blocks] (position of
 * block (j,i) for block (i,j)), blocks [nnz_blocks][4][4] FP64 row-major with unknowns
 * (u_x, u_y, u_z, p) per node; r, z [n_nodes][4] FP64.  All pointers are device pointers and the
 * caller owns them; z must not alias r.  opt selects the smoothers (Jacobi or Chebyshev only;
 * NULL = defaults with a 6-step Chebyshev Schur smoother).
 *
 * No memory is allocated: all intermediate arrays live in one 16 MiB static device array that
 * every GPU loading the library holds until process exit; n_nodes above 65536 is rejected with
 * LFX_ERR_INVALID_ARG.  The first call on a device (and the first after that device's context
 * was reset) looks the array's address up with the device current; make that first call before
 * any stream capture begins.  Every call reuses the same array and clears
 * it first, so calls whose work overlaps on the GPU (different streams, or different host
 * threads) race and must be serialised by the caller.  Work is queued on cuda_stream (NULL =
 * legacy default stream); the call does not synchronise. */
lfx_status lfx_asimple_apply_noalloc(int64_t n_nodes, const int32_t *row_ptr, const int32_t *col_idx,
                                     const int32_t *diag_idx, const int32_t *trans_idx,
                                     const double *blocks, const double *r, double *z,
                                     const lfx_options *opt, void *cuda_stream);

/* Shape of the algebraic-multigrid hierarchy of the Schur approximation (s_smoother ==
 * LFX_SMOOTH_AMG; Section 2.4 lists AMG among the block approximations of aSIMPLE), as built at
 * the last set-up: *n_levels levels (0 until the first step or debug call builds it); rows[l]
 * and nnz[l] = rows and stored nonzeros of the level-l operator (level 0 = the explicit
 * S = C - D diag(F)^-1 G, the last level = the dense-inverted coarsest one), written for
 * l < min(*n_levels, capacity) into caller-owned host arrays.  Host-only; no device work. */
lfx_status lfx_state_amg_levels(const lfx_state *state, int32_t *n_levels, int64_t *rows, int64_t *nnz,
                                int32_t capacity);

/* ------------------------------------------------------------------------------------------
 * Device memory: optional allocator hook (e.g. a framework's caching allocator)
 * ------------------------------------------------------------------------------------------ */
typedef void *(*lfx_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lfx_free_fn)(void *ptr, void *ctx);
/* Route every later device allocation through alloc/free (NULL, NULL restores cudaMalloc).  alloc
 * returns device memory aligned to at least 16 bytes (a pointer that is not is handed back to free
 * and the allocation fails with LFX_ERR_OOM), or NULL on failure.  Each allocation is released
 * through the free function (and ctx) that was current when it was made, so the hook may change
 * while handles are alive, provided the earlier free function stays callable until they are
 * destroyed.  The hook is process-wide and not synchronised: set it while no other call of the
 * library is running.  Giving one function without the other is LFX_ERR_INVALID_ARG. */
lfx_status lfx_set_allocator(lfx_alloc_fn alloc, lfx_free_fn free_fn, void *ctx);
/* Device bytes held by a state together with its problem and mesh (for admission control). */
lfx_status lfx_state_device_bytes(const lfx_state *state, int64_t *bytes);
/* Device bytes a new state of this problem will take (excluding the mesh and problem, which are
 * already resident), an upper estimate used for admission. */
lfx_status lfx_problem_state_bytes(const lfx_problem *problem, int64_t *bytes);

/* ------------------------------------------------------------------------------------------
 * Serving (not in the paper): continuous batching of independent simulations on one GPU.
 * Requests wait FIFO until the device-memory budget admits them; admitted simulations keep
 * their state resident, each on its own stream, and n_workers host threads step them
 * round-robin one step at a time, so kernels of different simulations overlap.  When one
 * finishes, its result is copied to host memory, its device memory released and waiting
 * requests are admitted.  Results are independent of the mix (no shared reductions).
 * ------------------------------------------------------------------------------------------ */
typedef struct lfx_server lfx_server;
/* hbm_budget_bytes: device memory that admitted states may occupy in total (> 0);
 * n_workers: host threads stepping simulations (1..64).  Uses the current CUDA device. */
lfx_status lfx_server_create(int64_t hbm_budget_bytes, int32_t n_workers, lfx_server **out);
/* Queue a simulation of `problem` (borrowed; must outlive the request) from the history
 * u_hist [bdf_order][n_nodes][3], p_hist [bdf_order][n_nodes] (copied) at t0, for n_steps
 * steps.  LFX_ERR_BUDGET if it can never fit the budget. */
lfx_status lfx_server_submit(lfx_server *server, lfx_problem *problem, const double *u_hist,
                             const double *p_hist, double t0, int32_t n_steps, int64_t *ticket);
/* done = 1 once all steps ran (or the request failed: the failure status is returned). */
lfx_status lfx_server_poll(lfx_server *server, int64_t ticket, int32_t *done, int32_t *steps_done,
                           lfx_step_stats *last);
/* Final u [n_nodes][3], p [n_nodes] (caller numbering) of a finished request; frees the ticket. */
lfx_status lfx_server_result(lfx_server *server, int64_t ticket, double *u, double *p);
/* Per-step latencies in ms (wall time of each lfx_step, up to capacity entries), their count,
 * the device bytes currently admitted, the queue length and the peak number of simulations
 * resident at once. */
lfx_status lfx_server_stats(lfx_server *server, float *latency_ms, int64_t capacity, int64_t *n_latencies,
                            int64_t *used_bytes, int64_t *n_waiting, int64_t *max_active);
/* Stops the workers after their current step and frees every remaining state. */
void lfx_server_destroy(lfx_server *server);

/* One step of each of n independent simulations (distinct states, each on its own stream set
 * with lfx_set_stream; states on the same stream run one after another): the steps run
 * concurrently, one host thread per state, so their kernels overlap on the device; stats [n]
 * (nullable) receive each step's statistics.  Returns LFX_OK, or the first failure in state order
 * (a hard error before LFX_ERR_NOT_CONVERGED), with the state's index in lfx_last_error().
 * Every state has advanced unless its own step failed.  Many small meshes are batched more tightly
 * by passing them to lfx_mesh_create together as one disconnected mesh: one state then steps all
 * of them with the same launches (one Krylov process per piece, batch_segmented). */
lfx_status lfx_batch_step(lfx_state *const *states, int32_t n, lfx_step_stats *stats);

#ifdef __cplusplus
}
#endif
#endif /* LFX_H */

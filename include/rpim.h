/*
 * rpim.h -- C ABI of the GB300 (sm_103a) RPIM stiffness-assembly library.
 *
 * The library follows the three stages of the pipeline described in Sec. 2
 * of the paper: (1) assemble the global stiffness matrix by integrating the
 * "element stiffness matrix of each field node" over its background cell,
 * (2) enforce displacement boundary conditions by the penalty method,
 * (3) solve the system and recover stresses. The method is the radial point
 * interpolation method (RPIM) with multiquadric radial basis and linear
 * polynomial augmentation (Sec. 1, refs. [23,24]).
 *
 * Conventions
 *  - Every array argument is a DEVICE pointer owned by the caller unless it
 *    is marked "host". Arrays are dense, C order, double or integer as typed.
 *  - Calls are ordered on `stream` (a cudaStream_t; NULL = legacy default
 *    stream). A call that must report sizes or convergence synchronises
 *    `stream`; each entry's comment says so.
 *  - DOF numbering: 3*node + {0:x, 1:y, 2:z}, nodes in the caller's order.
 *  - K is stored as a 3x3-block CSR matrix ("BSR"): `rowptr` (int64,
 *    n_nodes+1), `cols` (int32, ascending within a row), values as 9 doubles
 *    per block, row-major inside the block. K is symmetric: block (J,I) is
 *    the transpose of block (I,J), bit for bit.
 *  - Errors are returned as rpim_status codes, never by trapping; a kernel
 *    that meets an error records it on the device and the next synchronising
 *    call of the same pattern returns it. rpim_last_error() gives a
 *    thread-local message (for example the failing point index).
 *  - Thread safety: one pattern must not be used from two host threads at
 *    once; distinct patterns are independent.
 */
#ifndef RPIM_H
#define RPIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rpim_stream_t; /* same type as cudaStream_t */

typedef enum {
    RPIM_OK = 0,
    RPIM_E_ARG = 1,       /* invalid argument (null pointer, bad size, bad parameter)      */
    RPIM_E_CUDA = 2,      /* a CUDA runtime call failed                                     */
    RPIM_E_OOM = 3,       /* device or host allocation failed                               */
    RPIM_E_SUPPORT = 4,   /* a point has fewer than 4 or more than RPIM_MAX_SUPPORT nodes,  
                           * or a node lies in no point's support                          */
    RPIM_E_SINGULAR = 5,  /* degenerate support: the moment problem is singular             */
    RPIM_E_NOCONV = 6,    /* PCG reached max_iter before the tolerance                      */
    RPIM_E_NONFINITE = 7, /* a NaN or infinity was met in the inputs or the iteration       */
    RPIM_E_TIMEOUT = 8    /* reserved: a bounded device wait gave up                        */
} rpim_status;

/* Largest support (nodes per point) the shape-function kernel accepts. */
#define RPIM_MAX_SUPPORT 216

/*
 * RPIM parameters. Radii are in units of the nodal spacing h:
 *   support radius r_s = alpha_s * h;
 *   multiquadric R(r) = (r^2 + (alpha_c h)^2)^q, written in the local
 *   coordinates xi = (x - x_point)/h as (|xi|^2 + alpha_c^2)^q (the shape
 *   functions do not depend on this scaling);
 *   gauss_order: points per axis of the cell quadrature rule; only 2 is
 *   implemented (2x2x2 Gauss-Legendre per node cell).
 */
typedef struct {
    double alpha_s;
    double alpha_c;
    double q;
    double h;
    int32_t gauss_order;
} rpim_params;

typedef struct rpim_pattern rpim_pattern; /* opaque, owned by the library */

typedef struct {
    int64_t n_nodes;     /* field nodes                                        */
    int64_t n_points;    /* volume integration points = 8 n_nodes              */
    int64_t n_entries;   /* sum over points of the support size                */
    int64_t nnz_blocks;  /* 3x3 blocks of K                                    */
    int32_t max_support; /* largest support size                               */
    int32_t min_support; /* smallest support size                              */
    int32_t max_row;     /* largest number of blocks in a row                  */
    int32_t device;      /* CUDA device the pattern lives on                   */
} rpim_pattern_info;

/*
 * Stage 1a (Sec. 2): build everything that depends only on the node cloud.
 * Computes on the device, in order: the 2x2x2 Gauss points of every node
 * cell (point 8*i + a + 2b + 4c of cell i), a uniform-grid cell list of the
 * nodes (cell edge >= r_s), the support of every point (nodes with
 * |x_i - x_g|^2 <= r_s^2, ascending node id), the node -> point incidence,
 * and the BSR pattern of K (block (I,J) present iff some point supports both
 * I and J).
 *   xyz      [n_nodes*3]  node coordinates (device, read during the call only)
 *   cell_lo  [n_nodes*3]  lower corner of each node's cell (device)
 *   cell_hi  [n_nodes*3]  upper corner (device)
 *   params   host pointer
 *   out      host: receives the new pattern (free with rpim_pattern_free)
 *   nnz_blocks host, optional: number of 3x3 blocks of K
 * Synchronises `stream` (sizes come back to the host).
 * Errors: RPIM_E_ARG, RPIM_E_SUPPORT (a support outside 4..RPIM_MAX_SUPPORT,
 * point index in rpim_last_error; or a node that no point's support reaches,
 * whose row of K would be empty: node index), RPIM_E_OOM, RPIM_E_CUDA.
 */
rpim_status rpim_build_pattern(int64_t n_nodes, const double *xyz, const double *cell_lo,
                               const double *cell_hi, const rpim_params *params,
                               rpim_stream_t stream, rpim_pattern **out, int64_t *nnz_blocks);

/*
 * Batched stage 1a: one pattern for many independent node clouds
 * ("instances", e.g. hundreds of blocks of a parameter study). Instance i
 * owns the next inst[i].n_nodes nodes of xyz/cell_lo/cell_hi and has its own
 * support radius alpha_s*h and spacing h (alpha_c, q and gauss_order are
 * common). Every instance gets its own uniform grid, so supports never mix
 * instances and K is block diagonal; each stage then runs in one launch
 * over all instances. rpim_build_pattern is the one-instance case.
 *   inst     host [n_inst]
 * Synchronises. Errors as rpim_build_pattern.
 */
typedef struct {
    int64_t n_nodes; /* nodes of this instance (consecutive)           */
    double alpha_s;  /* support radius in units of h                   */
    double h;        /* nodal spacing of this instance                 */
} rpim_instance;

rpim_status rpim_build_pattern_batched(int32_t n_inst, const rpim_instance *inst, const double *xyz,
                                       const double *cell_lo, const double *cell_hi, double alpha_c,
                                       double q, int32_t gauss_order, rpim_stream_t stream,
                                       rpim_pattern **out, int64_t *nnz_blocks);

/*
 * Shape functions used by every later stage of a pattern (assembly, point
 * loads, stresses, gradients). RPIM_SHAPE_RPIM (the default) is the radial
 * point interpolation of Sec. 1. RPIM_SHAPE_MLS is moving least squares, one
 * of the alternatives the paper plans (Sec. 4): linear basis [1, (y - x)/h],
 * cubic-spline weight w(|x_i - x| / r_s) on the same support radius,
 *   phi_i(x) = w_i p_i^T A(x)^-1 p(x),  A(x) = sum_i w_i p_i p_i^T,
 * and its exact x-derivatives. RPIM_SHAPE_SHEPARD is the constant-basis
 * member of the same family (also named in Sec. 4): phi_i = w_i / sum_j w_j
 * with the same weights; it reproduces constants but not linear fields.
 * MLS and Shepard shape functions do not interpolate (phi_i(x_j) !=
 * delta_ij), so penalty values act on nodal parameters.
 * The kind is stored in the pattern; set it before the stage that should use
 * it. rpim_autotune_shape and rpim_autotune_buckets tune the RPIM kernel
 * only (the MLS and Shepard kernels have no launch shape to tune) and leave
 * such a pattern untouched.
 * Errors: RPIM_E_ARG (null pattern, unknown kind). MLS assembly reports
 * RPIM_E_SINGULAR when the 4x4 moment matrix has a pivot below
 * 1e-13 max|A| (fewer than four non-coplanar weighted nodes); Shepard when
 * no support node lies strictly inside the radius.
 */
typedef enum { RPIM_SHAPE_RPIM = 0, RPIM_SHAPE_MLS = 1, RPIM_SHAPE_SHEPARD = 2 } rpim_shape_kind;
rpim_status rpim_pattern_set_shape(rpim_pattern *pattern, int32_t kind);
rpim_status rpim_pattern_get_shape(const rpim_pattern *pattern, int32_t *kind);

/* Releases the pattern and all device memory it owns (stream-ordered on the
 * stream of the last call that used it). NULL is accepted. */
rpim_status rpim_pattern_free(rpim_pattern *pattern);

/* Sizes of a pattern (host struct). */
rpim_status rpim_pattern_get_info(const rpim_pattern *pattern, rpim_pattern_info *info);

/* Borrowed device pointers to the BSR structure of K (valid until free). */
rpim_status rpim_pattern_csr(const rpim_pattern *pattern, const int64_t **rowptr,
                             const int32_t **cols);

/* Borrowed device pointers to the integration points (n_points x 3, AoS),
 * their weights w|J| and the point supports (offsets int64 [n_points+1],
 * node ids int32 [n_entries], ascending within a point). */
rpim_status rpim_pattern_points(const rpim_pattern *pattern, const double **xyz,
                                const double **wj, const int64_t **support_offsets,
                                const int32_t **support_ids);

/*
 * Copies of the pattern's structure into caller-owned device buffers
 * (stream ordered, no synchronisation): rowptr [n_nodes+1] (int64),
 * cols [nnz_blocks] (int32); points [n_points*3], wj [n_points],
 * support_offsets [n_points+1] (int64), support_ids [n_entries] (int32).
 * Any output pointer may be NULL to skip it.
 */
rpim_status rpim_pattern_copy_csr(const rpim_pattern *pattern, int64_t *rowptr, int32_t *cols,
                                  rpim_stream_t stream);
rpim_status rpim_pattern_copy_points(const rpim_pattern *pattern, double *xyz, double *wj,
                                     int64_t *support_offsets, int32_t *support_ids,
                                     rpim_stream_t stream);

/*
 * Stage 1b (Sec. 2): assemble K and the body-force vector.
 * For every integration point g: RPIM shape functions phi and their
 * gradients at g from its support (multiquadric + linear polynomial moment
 * problem, FP64), then, per point, w|J| B_I^T D(E_g, nu_g) B_J for every
 * pair (I, J) of its support, and f_I = phi_I(g) b w|J|. K and f are sums
 * over points in ascending point order for every entry (deterministic, no
 * atomics); K is exactly symmetric.
 *   E, nu    [n_points]   Young's modulus and Poisson's ratio per point
 *   body     [3]          body force per unit volume (device), or NULL
 *   K_vals   [9*nnz_blocks] output, overwritten
 *   f        [3*n_nodes]  output, overwritten with the body-force vector
 * Synchronises `stream` to report per-point errors.
 * Errors: RPIM_E_ARG, RPIM_E_SINGULAR (point index in rpim_last_error),
 * RPIM_E_NONFINITE, RPIM_E_CUDA.
 */
rpim_status rpim_assemble(rpim_pattern *pattern, const double *E, const double *nu,
                          const double *body, double *K_vals, double *f, rpim_stream_t stream);

/*
 * rpim_assemble replayed from a CUDA graph (same arguments, same results,
 * bit for bit). The first call captures the assembly's launches (Lame
 * factors, the shape kernel, the row kernel, the mirror copy) on a stream
 * the pattern owns; capturing runs nothing. Later calls with the same
 * argument pointers, shape kind and launch plan (buckets, tuned shapes,
 * schedule) replay the graph with one launch; any change recaptures. The
 * caller may change the contents of E, nu and body between calls. With
 * per-kernel timing on (rpim_profile_enable) the launches are issued
 * directly. Synchronises `stream`. Errors as rpim_assemble.
 */
rpim_status rpim_assemble_graphed(rpim_pattern *pattern, const double *E, const double *nu,
                                  const double *body, double *K_vals, double *f, rpim_stream_t stream);

/*
 * Autotuner of the shape-function kernel's launch shape (points per block,
 * warps per point) for every support-size bucket of a pattern (the batched
 * workloads' tile and bucket choice): each admissible shape is timed on up
 * to max_points points of the bucket (CUDA events on `stream`), and the
 * fastest is used from then on, by every pattern of the process, for
 * supports of that bucket's size. The shape functions, hence K, are bitwise
 * the same for every launch shape, so tuning changes speed only.
 *   table   host int32 [3*16], optional: (largest support, warps per point,
 *           points per block) of each tuned bucket
 *   n_table host, optional: number of tuned buckets
 * Synchronises. Errors: RPIM_E_ARG, RPIM_E_CUDA.
 */
rpim_status rpim_autotune_shape(rpim_pattern *pattern, int64_t max_points, int32_t *table,
                                int32_t *n_table, rpim_stream_t stream);

/*
 * Support-size buckets of a pattern's integration points. The RPIM shape
 * kernel sizes each point's shared-memory buffers to the largest support of
 * its bucket, so the bounds trade buffer waste against the number of
 * distinct layouts. Bucket b holds the points with
 * bounds[b-1] < n <= bounds[b]; a final open-ended bucket is added.
 *   n_bounds 1..31, bounds host int32 [n_bounds], strictly increasing.
 * Re-groups on the device; synchronises. Results do not depend on the
 * bounds (every point's shape functions come from one group with a fixed
 * formula). Errors: RPIM_E_ARG.
 */
rpim_status rpim_pattern_set_buckets(rpim_pattern *pattern, int32_t n_bounds, const int32_t *bounds,
                                     rpim_stream_t stream);

/* Current buckets (host outputs, each optional, up to `capacity` entries):
 * upper bound, largest support and point count of every bucket. */
rpim_status rpim_pattern_get_buckets(const rpim_pattern *pattern, int32_t *n_buckets, int32_t *bounds,
                                     int32_t *max_support, int64_t *counts, int32_t capacity);

/*
 * Autotuner of the bucket bounds: applies each candidate set (the built-in
 * bounds 40/56/72/96/128/160 and uniform widths of 4, 8, 12, 16, 24 and 32
 * support sizes from the pattern's smallest to its largest support), times
 * the persistent shape pass on a sample of about max_points points spread
 * over the buckets (CUDA events on `stream`) and keeps the fastest set, for
 * this pattern and as the bounds every pattern built later in the process
 * starts with (like the launch shapes of rpim_autotune_shape).
 *   bounds host int32 [31], optional; n_bounds host, optional.
 * Synchronises. An MLS or Shepard pattern is left as it is (n_bounds = 0).
 */
rpim_status rpim_autotune_buckets(rpim_pattern *pattern, int64_t max_points, int32_t *bounds,
                                  int32_t *n_bounds, rpim_stream_t stream);

/*
 * Schedule of the RPIM shape kernel over the buckets, process-wide:
 * 1 (default) one persistent launch: the blocks walk the buckets, largest
 * supports first, and each point group takes the bucket's next point from a
 * device counter; 0 one launch per bucket. The shape functions are bitwise
 * the same either way. Errors: RPIM_E_ARG.
 */
rpim_status rpim_set_shape_schedule(int32_t persistent);

/*
 * Solver of the reduced moment system S a_r = rhs inside the RPIM shape
 * kernel (Sec. 1: the RPIM shape functions are the solution of the moment
 * problem), process-wide:
 *   RPIM_SOLVER_FP64 (0, default): S = L D L' factored in FP64.
 *   RPIM_SOLVER_REFINED (1): L D L' factored in float-float arithmetic
 *     (pairs of FP32 numbers, about 48 bits), then one step of iterative
 *     refinement whose residual rhs - S a_r is formed in FP64 from S in
 *     FP64, the correction solved with the same factors. The result has the
 *     accuracy of the FP64 factorisation (the refinement contracts the
 *     factorisation error by about cond(S) * 2^-46, cond(S) <= 1e7 here)
 *     with about half its FP64 work, but three triangular solves instead of
 *     one; the FP64 copy of S lives in a scratch array of the pattern
 *     (multiprocessors x 228 KB, allocated with the pattern).
 * The two solvers give different roundings, each deterministic and
 * independent of the launch shape. Changing the solver invalidates captured
 * assembly graphs (rpim_assemble_graphed recaptures). Errors: RPIM_E_ARG.
 */
#define RPIM_SOLVER_FP64 0
#define RPIM_SOLVER_REFINED 1
rpim_status rpim_set_shape_solver(int32_t solver);
rpim_status rpim_get_shape_solver(int32_t *solver);

/*
 * Order in which the row-owner kernels (the pattern build's two row passes
 * and the assembly's row kernel) take the rows of K, process-wide:
 * 1 (default) the Morton order of the nodes' grid cells (computed by every
 * rpim_build_pattern: Morton keys of the cell coordinates, instance first,
 * sorted by a stable radix sort), which keeps the rows that the GPU works on
 * at the same time spatially compact so that they share the integration
 * points they read; 0 node order. Every row is computed the same way in
 * either order, so K, f and the pattern are bitwise the same; the setting
 * changes speed only. Errors: RPIM_E_ARG.
 */
rpim_status rpim_set_row_order(int32_t morton);

/* Copy of a pattern's Morton row order (device int32 [n_nodes], a
 * permutation of the nodes), stream ordered. Errors: RPIM_E_ARG. */
rpim_status rpim_pattern_copy_row_order(const rpim_pattern *pattern, int32_t *order, rpim_stream_t stream);

/* Sets the launch shape for buckets whose largest support is max_support
 * (as rpim_autotune_shape would). Errors: RPIM_E_ARG when the shape is not
 * admissible (1-16 warps per point, 1-15 points per block, at most 768
 * threads, 512 with the refined solver, the points' shared memory within
 * 216 KB). */
rpim_status rpim_autotune_set(int32_t max_support, int32_t warps_per_point, int32_t points_per_block);

/* Forgets every tuned launch shape and the tuned bucket bounds (back to the
 * built-in rules for patterns built from now on). */
rpim_status rpim_autotune_reset(void);

/*
 * Shape functions only: writes, for every support entry e of every
 * integration point, phi[4e .. 4e+3] = (phi, dphi/dx, dphi/dy, dphi/dz)
 * in the order of rpim_pattern_points' support lists. Synchronises.
 */
rpim_status rpim_shape_functions(rpim_pattern *pattern, double *phi, rpim_stream_t stream);

/*
 * Loads at given points: f_I += sum_p phi_I(x_p) F_p (point forces, or
 * surface loads lumped at quadrature points chosen by the caller),
 * summed in ascending p for each node. Point supports use the pattern's
 * cell list and parameters.
 *   n_pts, xyz [n_pts*3], force [n_pts*3]; f [3*n_nodes] accumulated.
 * Synchronises. Errors as rpim_assemble.
 */
rpim_status rpim_add_point_loads(rpim_pattern *pattern, int64_t n_pts, const double *xyz,
                                 const double *force, double *f, rpim_stream_t stream);

/*
 * Surface tractions (Sec. 2, stage 1: the load side of the system; Sec. 3
 * examples: pressure on a face, parabolic shear on a beam end), integrated
 * by the library over axis-aligned face rectangles:
 *   face k lies in the plane x_a = face_lo[3k+a], a = face_axis[k] in {0,1,2}
 *   (face_hi[3k+a] must equal it), and spans [face_lo, face_hi] along its two
 *   tangent axes u < v (ascending axis order);
 *   coef [n_faces*18]: component c of the traction on face k is
 *   t_c(u, v) = sum_j coef[18k + 6c + j] m_j, m = (1, u, v, u^2, u v, v^2),
 *   in global coordinates (u, v of the point on the face).
 * Each face is integrated with the 2x2 Gauss-Legendre rule (points
 * mid +- half/sqrt(3) along u and v, weight half_u half_v):
 *   f_I += sum_k sum_p phi_I(x_kp) t(x_kp) w_kp,
 * summed for each node in ascending (face, point) order. Point supports use
 * the pattern's cell list and parameters; the points must have supports of
 * 4..RPIM_MAX_SUPPORT nodes.
 *   face_lo, face_hi [n_faces*3], face_axis [n_faces] (int8), coef: device;
 *   f [3*n_nodes] accumulated. n_faces = 0 is a no-op.
 * Synchronises. Errors: RPIM_E_ARG (a face that is not planar along its
 * axis, has lo > hi along a tangent axis or names no axis: face index in
 * rpim_last_error), RPIM_E_SUPPORT, RPIM_E_SINGULAR, RPIM_E_OOM, RPIM_E_CUDA.
 */
rpim_status rpim_add_traction(rpim_pattern *pattern, int64_t n_faces, const double *face_lo,
                              const double *face_hi, const int8_t *face_axis, const double *coef,
                              double *f, rpim_stream_t stream);

/* Batched tractions: as rpim_add_traction, with the instance of every face
 * (device int32 [n_faces]). Required for batched patterns. Errors: RPIM_E_ARG
 * also when an id is outside [0, n_inst) (checked on the device before any
 * use). */
rpim_status rpim_add_traction_batched(rpim_pattern *pattern, int64_t n_faces, const double *face_lo,
                                      const double *face_hi, const int8_t *face_axis, const double *coef,
                                      const int32_t *inst, double *f, rpim_stream_t stream);

/*
 * f += x over the 3*n_nodes entries of a load vector (device arrays), stream
 * ordered, no synchronisation: adds a material-independent load vector
 * assembled once (tractions, point loads) to the body-force vector that each
 * rpim_assemble writes, e.g. in every forward solve of a back-analysis.
 * Errors: RPIM_E_ARG (null pointer), RPIM_E_CUDA.
 */
rpim_status rpim_add_vector(rpim_pattern *pattern, const double *x, double *f, rpim_stream_t stream);

/*
 * Batched surface loads: as rpim_add_point_loads, with the instance of every
 * load point (device int32 [n_pts]). Required for batched patterns.
 * Errors: RPIM_E_ARG also when an id is outside [0, n_inst) (checked on the
 * device before any use; the load index is in rpim_last_error).
 */
rpim_status rpim_add_point_loads_batched(rpim_pattern *pattern, int64_t n_pts, const double *xyz,
                                         const double *force, const int32_t *inst, double *f,
                                         rpim_stream_t stream);

/*
 * Stage 2 (Sec. 2): penalty enforcement of prescribed displacements, one GPU
 * thread per constrained DOF as in the paper: alpha = penalty_scale *
 * max_i K_ii (over all scalar diagonal entries, computed on the device), then
 * K_dd += alpha and f_d += alpha * values[i] for d = dofs[i].
 *   m, dofs [m] (int64, unique), values [m]
 *   alpha_out host, optional: receives alpha (synchronises when given).
 * Errors: RPIM_E_ARG (DOF out of range or repeated).
 */
rpim_status rpim_apply_penalty_bc(rpim_pattern *pattern, double *K_vals, double *f, int64_t m,
                                  const int64_t *dofs, const double *values, double penalty_scale,
                                  double *alpha_out, rpim_stream_t stream);

/*
 * Batched stage 2: one alpha per instance (scale * the instance's largest
 * diagonal entry), each DOF penalised with its instance's alpha.
 *   alpha_out host [n_inst], optional. Synchronises.
 */
rpim_status rpim_apply_penalty_bc_batched(rpim_pattern *pattern, double *K_vals, double *f, int64_t m,
                                          const int64_t *dofs, const double *values,
                                          double penalty_scale, double *alpha_out,
                                          rpim_stream_t stream);

/*
 * Stage 2 with a given penalty: as rpim_apply_penalty_bc, but alpha is the
 * caller's value (for instance the one a previous call returned), so that K
 * depends on the material only through the stiffness: the frozen penalty of
 * a back-analysis. K_dd += alpha, f_d += alpha * values[i]. Synchronises.
 * Errors: RPIM_E_ARG (negative alpha, DOF out of range or repeated).
 */
rpim_status rpim_apply_penalty_alpha(rpim_pattern *pattern, double *K_vals, double *f, int64_t m,
                                     const int64_t *dofs, const double *values, double alpha,
                                     rpim_stream_t stream);

/*
 * Preconditioner of the PCG solves of a pattern (Sec. 2, stage 3: the paper
 * solves with library solvers; here K is symmetric positive definite after
 * the penalty, so conjugate gradients apply). RPIM_PRECOND_JACOBI (the
 * default): M = diag(K). RPIM_PRECOND_BLOCK_JACOBI: M = the 3x3 diagonal
 * blocks K_II (the three DOFs of a node), each inverted once per solve from
 * its L D L^T factors; a block that is not positive definite is reported as
 * RPIM_E_ARG (DOF index). Applies to rpim_solve_pcg and
 * rpim_solve_pcg_batched. Errors: RPIM_E_ARG (null pattern, unknown kind).
 */
typedef enum { RPIM_PRECOND_JACOBI = 0, RPIM_PRECOND_BLOCK_JACOBI = 1 } rpim_precond_kind;
rpim_status rpim_pattern_set_precond(rpim_pattern *pattern, int32_t kind);
rpim_status rpim_pattern_get_precond(const rpim_pattern *pattern, int32_t *kind);

/*
 * Stage 3 (Sec. 2): solve K u = f by preconditioned conjugate gradients
 * (rpim_pattern_set_precond; Jacobi by default) in FP64 with deterministic
 * reductions. u holds the initial guess on entry. Stops when
 * ||r||_2 <= rtol ||f||_2 or after max_iter iterations.
 *   iters, relres host, optional. Synchronises.
 * Errors: RPIM_E_NOCONV (u holds the last iterate), RPIM_E_NONFINITE.
 */
rpim_status rpim_solve_pcg(rpim_pattern *pattern, const double *K_vals, const double *f,
                           double *u, double rtol, int32_t max_iter, int32_t *iters,
                           double *relres, rpim_stream_t stream);

/*
 * Batched stage 3: the instances of a batched pattern are independent
 * systems (K is block diagonal by instance), each iterated with its own
 * PCG scalars and stopped on its own test ||r_i||_2 <= rtol ||f_i||_2 or
 * after max_iter iterations; finished instances drop out of the sweeps. All
 * instances advance in the same launches. Works on any pattern (one
 * instance: the same iteration as rpim_solve_pcg).
 *   iters host int32 [n_inst], relres host [n_inst], optional. Synchronises.
 * Errors: RPIM_E_NOCONV, RPIM_E_NONFINITE (the first failing instance in
 * rpim_last_error; u holds every instance's last iterate).
 */
rpim_status rpim_solve_pcg_batched(rpim_pattern *pattern, const double *K_vals, const double *f,
                                   double *u, double rtol, int32_t max_iter, int32_t *iters,
                                   double *relres, rpim_stream_t stream);

/*
 * Material gradient of a solved system, per integration point (the
 * back-analysis of the paper's geomechanics use, Sec. 1 and 4: the package
 * exists to model rock and soil masses whose properties are uncertain).
 * With K(E, nu) u = f, the penalty frozen, and the adjoint K lam = dL/du
 * (solve it with rpim_solve_pcg; K is symmetric),
 *   dE[g]  = dL/dE_g  = - w_g eps_g(lam)^T (dD/dE)  eps_g(u),
 *   dnu[g] = dL/dnu_g = - w_g eps_g(lam)^T (dD/dnu) eps_g(u),
 * eps_g(v) = sum_I B_I(x_g) v_I, D isotropic (Voigt, engineering shear).
 * Uses the shape functions of the last rpim_assemble of this pattern (they
 * do not depend on the material); computes them if none exist.
 *   u, lam [3*n_nodes]; E, nu [n_points]; dE, dnu [n_points] outputs.
 * Synchronises. Errors: RPIM_E_ARG (material out of range).
 */
rpim_status rpim_grad_material(rpim_pattern *pattern, const double *u, const double *lam,
                               const double *E, const double *nu, double *dE, double *dnu,
                               rpim_stream_t stream);

/*
 * Stresses at arbitrary points: sigma_p = D(E_p, nu_p) sum_I B_I(x_p) u_I,
 * Voigt order xx, yy, zz, yz, xz, xy (engineering shear strains in B).
 *   n_pts, xyz [n_pts*3], E [n_pts], nu [n_pts], u [3*n_nodes],
 *   sigma [n_pts*6] output. Synchronises.
 */
rpim_status rpim_stress(rpim_pattern *pattern, const double *u, int64_t n_pts,
                        const double *xyz, const double *E, const double *nu, double *sigma,
                        rpim_stream_t stream);

/*
 * rpim_stress without any device allocation, for callers that cannot allocate
 * device memory while they run: hosts that fix and account their device-memory
 * budget at start-up, or loops that keep other streams busy and cannot accept
 * the device synchronisation that cudaMalloc/cudaFree may imply. (The paper
 * has no counterpart; this is a deployment variant of rpim_stress.)
 * Same arguments and results as rpim_stress. The per-call scratch (support
 * lists and shape functions of the points) lives in one fixed array of
 * device memory owned by the library: 9.45 MB on every GPU that loads
 * the library, held until the process exits.
 *   Limits: at most RPIM_NOALLOC_MAX_POINTS points per call and at most
 *   RPIM_NOALLOC_MAX_ENTRIES support entries in total (sum of the points'
 *   support sizes); larger calls return RPIM_E_ARG and compute nothing.
 *   The first call on each device looks up the array's device address (no
 *   allocation); make that first call before any stream capture.
 *   Every call uses the same array: calls that may overlap on the GPU (other
 *   streams, other host threads) race and must be serialised by the caller.
 *   The refined shape solver (rpim_set_shape_solver) also uses the pattern's
 *   own solver scratch, allocated when the pattern was built; like every
 *   call on a pattern, the call must not overlap another call on the same
 *   pattern.
 * Synchronises `stream`.
 */
#define RPIM_NOALLOC_MAX_POINTS 2048
#define RPIM_NOALLOC_MAX_ENTRIES 262144
rpim_status rpim_stress_noalloc(rpim_pattern *pattern, const double *u, int64_t n_pts,
                                const double *xyz, const double *E, const double *nu,
                                double *sigma, rpim_stream_t stream);

/* Batched stresses: as rpim_stress, with the instance of every point
 * (device int32 [n_pts]). Required for batched patterns. Errors: RPIM_E_ARG
 * also when an id is outside [0, n_inst), checked on the device before any
 * use. */
rpim_status rpim_stress_batched(rpim_pattern *pattern, const double *u, int64_t n_pts,
                                const double *xyz, const int32_t *inst, const double *E,
                                const double *nu, double *sigma, rpim_stream_t stream);

/* Thread-local description of the last error returned on this thread. */
const char *rpim_last_error(void);

/* Library version string. */
const char *rpim_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RPIM_H */

/*
 * tursca.h -- C ABI of the GB300 scattering-graph radiative-transfer library
 * (libtursca_gb.so).
 *
 * The library computes the data-parallel hot path of the scattering graph
 * method (Mikkonen et al., "Scattering graph method for 3D radiative
 * transfer", Sec. 2 and Sec. 3) on a graph whose nodes are the voxels of a
 * regular 3D grid plus one Lambertian ground node per column:
 *
 *   1. assemble the flux matrix K (rows = receivers) whose entries are a
 *      Beer-Lambert transmittance of the edge (Eq. radiance_effectuality and
 *      the exponential of Eq. Fab) x a phase-function quadrature weight p'
 *      (Eq. F_term_phase, Fibonacci lattice of Sec. 3) x the normalised
 *      scattering coupling C(r, r') (Eq. scatt_coup), and the direct solar
 *      source s (S_a, Sec. 2);
 *   2. solve (I - K) x = s (Eq. flux_system, equivalently the series of
 *      Eq. fs_sum);
 *   3. sum the node radiances into detector pixels along the lines of sight
 *      (final radiance sum of Sec. 2, step 5 of the algorithm in Sec. 3).
 *
 * Conventions for every entry point:
 *   - Functions return tursca_status; no C++ exception crosses the ABI.
 *   - Array arguments are caller-owned and borrowed for the duration of the
 *     call; the library copies what it keeps.  They may be device pointers or
 *     host pointers (pageable or pinned): copies use cudaMemcpyDefault.
 *   - The element type of field and output arrays follows
 *     tursca_grid_desc.precision: double for TURSCA_FP64, float for
 *     TURSCA_FP32_REFINE.
 *   - Grid arrays are C order (z, y, x), x fastest.  Lengths in km,
 *     coefficients in km^-1, angles in degrees.
 *   - Work is enqueued on the stream given at creation.  Argument errors are
 *     returned synchronously; asynchronous CUDA errors and invalid field
 *     values found on the device are returned by the next call that
 *     synchronises (tursca_solve, tursca_render_radiance, tursca_get).
 *   - Calls out of order (e.g. solve before assemble_flux) return
 *     TURSCA_E_STATE.
 *   - A scene is not thread safe; distinct scenes may be used from distinct
 *     threads.
 */
#ifndef TURSCA_H
#define TURSCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tursca_scene tursca_scene; /* opaque; owns its device state */

typedef enum {
    TURSCA_OK = 0,
    TURSCA_E_INVALID = 1,       /* bad argument or invalid field value */
    TURSCA_E_NOMEM = 2,         /* device or host allocation failed */
    TURSCA_E_CUDA = 3,          /* CUDA runtime error (see tursca_last_error) */
    TURSCA_E_NOT_CONVERGED = 4, /* solver stopped at max_iter above rtol */
    TURSCA_E_TIMEOUT = 5,       /* a bounded device wait gave up */
    TURSCA_E_STATE = 6,         /* call out of order */
    TURSCA_E_UNSUPPORTED = 7    /* entry point declared but not available */
} tursca_status;

enum { TURSCA_FP64 = 0, TURSCA_FP32_REFINE = 1 };
enum { TURSCA_COUPLING_NONE = 0, TURSCA_COUPLING_WEIGHT = 1 };
enum { TURSCA_SOLVER_AUTO = 0, TURSCA_SOLVER_NEUMANN = 1, TURSCA_SOLVER_GMRES = 2, TURSCA_SOLVER_CHEBYSHEV = 3 };

/* Grid and method parameters (fixed for the life of a scene).
 *   nx, ny >= 2 R + 1 (x and y are periodic), nz >= R.
 *   stencil_radius R in {1, 2}: each voxel couples to the voxel centres
 *     j + k u, u a primitive integer vector with |u|_inf <= R,
 *     k = 1..floor(R / |u|_inf) (26 neighbours for R = 1, 124 for R = 2);
 *     the ground node of a column couples to the voxels (dx, dy, dz - 1/2)
 *     away, |dx|, |dy| <= R, 1 <= dz <= R.
 *   fib_points M (>= 64): points of the Fibonacci lattice used for the
 *     quadrature of Eq. F_term_phase (Sec. 3).
 *   n_species S in 1..4: scattering species, each with a Henyey-Greenstein
 *     phase function.
 *   coupling_mode: TURSCA_COUPLING_WEIGHT applies Eq. scatt_coup as a
 *     normalised routing weight; TURSCA_COUPLING_NONE uses weight 1.
 *   precision: TURSCA_FP64 (all FP64) or TURSCA_FP32_REFINE (FP32 edge march
 *     and SpMV, FP64 residual and refinement update). */
typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    int n_species;
    int stencil_radius;
    int fib_points;
    int coupling_mode;
    int precision;
} tursca_grid_desc;

/* Illumination and viewing geometry (Sec. 2: far-field source, instrument).
 *   sza < 90, vza < 90; f0 the solar irradiance normal to the beam.
 *   The sun's beam travels along -(sin sza cos saa, sin sza sin saa, cos sza);
 *   the instrument sees the scene along +(sin vza cos vaa, sin vza sin vaa,
 *   cos vza).  Pixel (a, b) of the npx x npy detector looks at the ground
 *   point ((a + 1/2) nx hx / npx, (b + 1/2) ny hy / npy, 0). */
typedef struct {
    double sza, saa, vza, vaa, f0;
    int npx, npy;
} tursca_geometry;

typedef struct {
    int iters;          /* matrix-vector products with K in the solve */
    int refinements;    /* outer FP64 residual evaluations */
    double rel_resid64; /* ||s - (I - K) x|| / ||s|| evaluated in FP64 */
    double rho_est;     /* estimate of the spectral radius of K */
    int solver;         /* TURSCA_SOLVER_* actually used */
} tursca_solve_info;

/* Counts of the graph for a grid (host only; no GPU needed). */
typedef struct {
    int n_atm, n_ground, n_nodes;
    int n_dirs, n_up_dirs, n_gdirs, n_gmembers;
    long long nnz;        /* stored slots including row padding */
    long long nnz_edges;  /* slots that carry a graph edge (no padding) */
    int n_classes;        /* distinct slot classes (translation-invariant) */
    int max_row;          /* longest row (slots) */
} tursca_graph_stats;

/* Internal arrays that tursca_get can copy out (for tests and tools). */
typedef enum {
    TURSCA_F_ROW_PTR = 0,  /* int32 [n_nodes + 1] */
    TURSCA_F_COL = 1,      /* int32 [nnz] source node of each slot */
    TURSCA_F_VAL = 2,      /* real  [nnz] K value of each slot */
    TURSCA_F_SLOT_DIR = 3, /* int16 [nnz] direction: atmospheric 0..n_dirs-1, ground n_dirs + g, -1 padding */
    TURSCA_F_SLOT_K = 4,   /* int8  [nnz] chain index; 0 self, 7 ground hit, -1 padding */
    TURSCA_F_TSUN = 5,     /* real  [n_nodes] sun transmittance (top-face centre / ground point) */
    TURSCA_F_E1 = 6,       /* real  [n_nodes] first-order scattered (reflected) power */
    TURSCA_F_S = 7,        /* real  [n_nodes] s = K^sun e1 */
    TURSCA_F_X = 8,        /* double [n_nodes] solution of (I - K) x = s */
    TURSCA_F_EMIS = 9,     /* real  [n_atm] emission toward the instrument E_i */
    TURSCA_F_GSUN = 10,    /* real  [n_atm] second-order part of E_i */
    TURSCA_F_Q_ISO = 11,   /* double [n_dirs] */
    TURSCA_F_Q_LAMB = 12,  /* double [n_gdirs] */
    TURSCA_F_Q_SUN = 13,   /* real  [n_species][n_dirs] */
    TURSCA_F_DIRS = 14,    /* int32 [n_dirs][3] lattice directions, in the library's order */
    TURSCA_F_ANISO_X = 15  /* double [n_dirs + n_gdirs][n_nodes] edge unknowns X(i, w) of the last
                              TURSCA_OPT_ANISO solve (TURSCA_E_STATE before one) */
} tursca_field;

/* Create a scene for grid *desc whose work runs on cuda_stream (a
 * cudaStream_t; NULL = the legacy default stream).  Allocates nothing on the
 * device until build_graph.  Errors: TURSCA_E_INVALID on a bad descriptor. */
tursca_status tursca_scene_create(const tursca_grid_desc *desc, void *cuda_stream, tursca_scene **out);

/* Free every resource of the scene (synchronises its stream).  NULL is a no-op. */
tursca_status tursca_scene_destroy(tursca_scene *scene);

/* Set the optical fields (Sec. 2: mu_a, mu_s, Theta).
 *   mu_abs [nz][ny][nx] absorption coefficient, >= 0;
 *   mu_sca [n_species][nz][ny][nx] scattering coefficient per species, >= 0;
 *   g [n_species] host array of HG asymmetry parameters, |g| < 1;
 *   albedo: Lambertian surface albedo in [0, 1].
 * The fields are copied; negative or non-finite values are reported as
 * TURSCA_E_INVALID by the next synchronising call. */
tursca_status tursca_set_medium(tursca_scene *scene, const void *mu_abs, const void *mu_sca, const double *g,
                                double albedo);

/* Build the graph for the scene's grid: direction sets, Fibonacci partition
 * (Sec. 3), translation-invariant tap tables of every edge segment, and the
 * CSR structure of K (rows = receivers).  Cached: a second call is a no-op. */
tursca_status tursca_build_graph(tursca_scene *scene);

/* Assemble K, the direct source e1 and s = K^sun e1 for the current medium
 * and geometry (Eqs. Fab, F_term_phase, scatt_coup; S_a of Sec. 2).
 * Requires build_graph and set_medium. */
tursca_status tursca_assemble_flux(tursca_scene *scene, const tursca_geometry *geom);

/* Solve (I - K) x = s (Eq. flux_system) to ||s - (I - K) x|| <= rtol ||s||
 * evaluated in FP64, with at most max_iter inner steps (a sweep, a Chebyshev
 * step, or a GMRES step, which applies K twice).  The outer loop is FP64
 * residual refinement; each refinement solves for the correction with inner
 * iterations in the scene's precision: FP32_REFINE scenes first run a few
 * Neumann sweeps (the series of Eq. fs_sum) that also estimate the largest
 * eigenvalue of K, then Chebyshev iterations on the interval that estimate
 * implies, or GMRES when the estimate is 0.85 or more or a Chebyshev
 * refinement under-delivers; FP64 scenes run GMRES.  GMRES(30) (FP64: 40)
 * is right-preconditioned with I + K, the first two terms of that series.
 * Synchronises once per refinement (GMRES: once per step).  info may be
 * NULL. */
tursca_status tursca_solve(tursca_scene *scene, double rtol, int max_iter, tursca_solve_info *info);

/* Same as tursca_solve with an explicit solver choice (TURSCA_SOLVER_*). */
tursca_status tursca_solve_with(tursca_scene *scene, int solver, double rtol, int max_iter,
                                tursca_solve_info *info);

/* Emission toward the instrument and detector radiance (final radiance sum of
 * Sec. 2, integrated over voxel segments): radiance [npy][npx] in units of
 * f0 per steradian; reflectance [npy][npx] = pi L / (cos(sza) f0), may be
 * NULL.  Requires solve.  Synchronises before returning. */
tursca_status tursca_render_radiance(tursca_scene *scene, void *radiance, void *reflectance);

/* The whole path for one medium in one call: tursca_set_medium,
 * tursca_assemble_flux, tursca_solve_with and tursca_render_radiance in that
 * order, with the arguments and the ownership rules of those calls (the
 * steps of the method's data flow, Sec. 3: medium, graph weights, solve,
 * detector).  Returns the first error (the later steps are then not run);
 * info may be NULL.  Requires build_graph.  Synchronises before returning,
 * as the render does; saves the caller's turnarounds between the four calls. */
tursca_status tursca_run(tursca_scene *scene, const void *mu_abs, const void *mu_sca, const double *g, double albedo,
                         const tursca_geometry *geom, int solver, double rtol, int max_iter, void *radiance,
                         void *reflectance, tursca_solve_info *info);

/* Gradient of a detector objective J with respect to the absorption
 * coefficient of every voxel, by the adjoint of the whole path (reverse-mode
 * differentiation written out by hand; the paper motivates the method with
 * retrievals, Sec. 3 and the conclusions).  mu_abs enters only through the
 * extinction mu_e = mu_abs + sum_s mu_sca,s, which enters the optical depths
 * of every edge, the direct beam and the lines of sight (Eq.
 * radiance_effectuality, Eq. Fab, the final radiance sum of Sec. 2) and the
 * scattering ratio and e1 of every node.  The adjoint runs: pixels -> emission
 * -> (I - K)^T lambda = x-bar (the transposed system of Eq. flux_system,
 * solved like the forward one) -> reverse edge march (segment-table, tau_inf,
 * tap and direct-beam adjoints) -> dJ/dmu_e.
 *   dJ_dL       [npy][npx] dJ/dL_p, compute type, host or device; borrowed.
 *   dJ_dmu_abs  [nz][ny][nx] output, compute type, host or device.
 * Requires render_radiance since the last solve (TURSCA_E_STATE otherwise);
 * uses the scene's resident state and does not change the forward results.
 * The first call allocates a transposed copy of K (4 bytes per edge in FP32)
 * and the adjoint accumulators.  Accumulations use atomic adds, so repeated
 * calls agree to rounding, not bit for bit.  Synchronises before returning. */
tursca_status tursca_adjoint(tursca_scene *scene, const void *dJ_dL, void *dJ_dmu_abs);

/* Copy an internal array out (device -> dst, host or device pointer) after the
 * stage that produces it; bytes must equal the array size.  Synchronises. */
tursca_status tursca_get(tursca_scene *scene, tursca_field which, void *dst, size_t bytes);

/* Scene options (tursca_set_option).
 *   TURSCA_OPT_RESIDUAL_FP64: 0 (default) evaluates the refinement residual of
 *     FP32_REFINE scenes in FP32-pair arithmetic (exact products by FMA and
 *     compensated sums, about 48 significant bits; FP64 arithmetic runs at a
 *     small fraction of the FP32 rate on GB300); 1 uses FP64 arithmetic.
 *   TURSCA_OPT_GROUP_WARPS: warps that share each group of 128 rows in the
 *     sweep, Chebyshev, residual and emission passes: 4, 6, 8 or 16 (the
 *     streamed passes take 4, 8 or 16), or 0 to let the library pick
 *     (default: 6, 16 for the streamed passes).
 *   TURSCA_OPT_STAGE_VALUES: 0 (default) runs one block per group of 128
 *     rows that reads the matrix values directly; 1 runs the FP32 sweep,
 *     Chebyshev, residual and emission passes as persistent kernels (one
 *     block per SM, each streaming an equal share of the values) in which
 *     one warp copies the values into a ring of shared-memory stages with
 *     bulk asynchronous copies while the other warps compute.  Both sum the
 *     same products in the same order for the same TURSCA_OPT_GROUP_WARPS.
 *     A copy that does not land within about a second makes the solve
 *     return TURSCA_E_TIMEOUT.
 *   TURSCA_OPT_L2_RESIDENT: 0 (default); 1 keeps the values of K in the
 *     persisting part of L2 while a solve runs (every pass of a solve streams
 *     the same values).  Setting 1 raises this CUDA context's persisting-L2
 *     set-aside to the device maximum for the rest of the process; each
 *     solve sets an access-policy window over the values on the scene
 *     stream, and on return removes it and resets every persisting line of
 *     the context to normal (which also affects other scenes running
 *     concurrently in the same context).  Pays only when the values fit in
 *     the set-aside; results are bit-identical either way.
 *   TURSCA_OPT_GATHER_TILE: 1 (default) lets the FP32 row-group passes
 *     (sweeps, Chebyshev steps, products with I - K, the FP32-pair residual
 *     and the emission pass, also over K^T in the adjoint) copy each group's
 *     source rows of the vectors they gather from into shared-memory tiles
 *     (at most 48 KB per block; larger groups gather from global memory);
 *     0 always gathers from global memory.  Results are bit-identical
 *     either way.
 *   TURSCA_OPT_SINGLE_SCATTER: 0 (default); 1 makes the following
 *     assemblies first-order only (single scattering, the branch of the data
 *     flow of Sec. 3 that stops after the direct beam): assemble_flux computes
 *     the phase tables, the extinction and e1 and forms neither K nor
 *     K^sun (s reads as 0); solve sets x = 0 without a product with K
 *     (iters = refinements = 0, rel_resid64 = 0); render_radiance takes
 *     E_i = e1_i Theta_i(s0 . v) and the ground's e1_c.  get(TURSCA_F_VAL)
 *     and tursca_adjoint return TURSCA_E_STATE after such an assembly.
 *     Changing the value invalidates the current assembly.
 *   TURSCA_OPT_COUPLING_MIN: c_min >= 0 of the scattering graph (Sec. 2: the
 *     graph keeps the couplings C of Eq. scatt_coup above c_min; default 0,
 *     the full stencil).  With c_min > 0 a chain whose first receiver has
 *     C <= c_min gets the weight 0 (its slots stay in K), chains without a
 *     receiver are always kept, and each source re-draws its quadrature cells
 *     (Eq. F_term_phase) among the directions it keeps: a lattice point joins
 *     the kept direction closest to it (exact ties to the lower index).  The
 *     decision is taken in FP64 in every precision.  The first assembly with
 *     c_min > 0 ranks the lattice (M x n_dirs bytes; M <= 2^20, else
 *     TURSCA_E_UNSUPPORTED) and allocates two weight planes per direction
 *     (2 x n_dirs x nodes of the haloed layout, compute type).  The
 *     weights depend on the scattering coefficients only, so tursca_adjoint
 *     (a gradient with respect to absorption) reads the same weights.
 *     Changing the value invalidates the current assembly.
 *   TURSCA_OPT_MAX_COUPLINGS: K >= 0, a whole number (default 0: off).  The
 *     preselected maximum number of couplings of Sec. 3: the graph keeps the
 *     chains whose coupling exceeds the (K + 1)-th largest coupling over
 *     every chain that has a receiver other than its source, found in FP64
 *     at every assembly (an exact radix select over the chains' couplings);
 *     then everything proceeds as TURSCA_OPT_COUPLING_MIN with that
 *     threshold (the smallest positive double when that coupling is 0, so
 *     zero couplings go first).  Exactly K chains are kept unless couplings
 *     tie at the boundary (a chain and its reverse share one coupling; a tied
 *     group at the boundary goes as a whole); K at or above the number of
 *     chains keeps the full stencil.  Excludes c_min > 0 (TURSCA_E_INVALID at
 *     assembly).  Memory: 8 bytes per chain (n_atm n_dirs + n_ground
 *     n_gdirs) for the keys, besides what TURSCA_OPT_COUPLING_MIN allocates.
 *     Changing the value invalidates the current assembly.
 *   TURSCA_OPT_ANISO: 0 (default); 1 (or 2) keeps the arrival direction of the
 *     light into every scattering (the edge unknowns of Eq. flux_system;
 *     the default node form re-emits isotropically after the first
 *     scattering).  The unknown is X(i, w), the power scattered at node i from
 *     light that arrived along w (the n_dirs atmospheric directions, then the
 *     n_gdirs ground chains' directions).  At every scattering the species' HG
 *     is integrated over the cell of each outgoing direction with the angle
 *     measured from w (Eq. F_term_phase).  assemble_flux stores each slot's
 *     deposit fraction in place of K (get(TURSCA_F_VAL) then returns
 *     TURSCA_E_STATE) and builds the quadrature by arrival direction.  solve
 *     sums the series of Eq. fs_sum until the relative change of X is at most
 *     rtol; FP32 scenes sum it in FP32 to a change of max(rtol, 1e-6), then
 *     refine: while the residual |F(X) - X| / |X| of the fixed point, with X
 *     in FP64 and double-single sums, is above rtol, an FP32 series for the
 *     correction, added in FP64.  iters counts the terms of all series,
 *     refinements the residual evaluations, and rel_resid64 holds the last
 *     residual (FP64 scenes: the last relative change).  FP32 scenes compute
 *     each term's dense per-node contraction on the tensor cores (tcgen05,
 *     TF32 operands split in high and low parts) with 1 and on the CUDA cores
 *     with 2; FP64 scenes on the CUDA cores.  Every term is deterministic (no
 *     atomics).  Combines with neither
 *     TURSCA_OPT_SINGLE_SCATTER nor coupling selection (TURSCA_E_INVALID at
 *     assembly); tursca_adjoint returns TURSCA_E_UNSUPPORTED.  Memory:
 *     3 (n_dirs + n_gdirs) + 2 n_dirs values per node plus n_dirs haloed
 *     planes, in the compute type; FP32 scenes add, at the first solve,
 *     (n_dirs + n_gdirs) (8 + 4 + 4) bytes per node and n_dirs haloed FP64
 *     planes.  Changing the value invalidates the current assembly.
 */
enum {
    TURSCA_OPT_RESIDUAL_FP64 = 1,
    TURSCA_OPT_GROUP_WARPS = 2,
    TURSCA_OPT_STAGE_VALUES = 3,
    TURSCA_OPT_L2_RESIDENT = 4,
    TURSCA_OPT_GATHER_TILE = 5,
    TURSCA_OPT_SINGLE_SCATTER = 6,
    TURSCA_OPT_COUPLING_MIN = 7,
    TURSCA_OPT_ANISO = 8,
    TURSCA_OPT_MAX_COUPLINGS = 9
};
tursca_status tursca_set_option(tursca_scene *scene, int option, double value);

/* The coupling selection of the current assembly: *threshold the c_min
 * applied (0: the full stencil); with TURSCA_OPT_MAX_COUPLINGS also
 * *n_couplings, the chains that carry a coupling, and *n_kept, those kept
 * (both -1 otherwise).  Any output may be NULL.  TURSCA_E_STATE before the
 * first assembly. */
tursca_status tursca_selection_info(const tursca_scene *scene, double *threshold, long long *n_couplings,
                                    long long *n_kept);

/* Number of kernel launches the scene has issued since creation. */
long long tursca_launch_count(const tursca_scene *scene);

/* Device memory the scene holds (bytes of its own allocations). */
size_t tursca_scene_device_bytes(const tursca_scene *scene);

/* Per-kernel device time measured with CUDA events recorded on the scene's
 * stream around each launch of the hot kernels (profiling only). */
typedef struct {
    char name[32];      /* "spmv", "resid64", "assemble_rows", "assemble_pre", "render", "cheb",
                           "gmres_orth" (both Gram-Schmidt passes of one Arnoldi step),
                           "select" (coupling selection), "gmres_prod" (the passes over K of
                           one Arnoldi step: preconditioner and product with I - K, each
                           counted as a launch), "set_medium" (its copies), "solve" (a whole
                           solve, from its first to its last operation on the stream,
                           host round trips included; the solve's other categories lie
                           inside it), and of the anisotropic mode "ani_leave" (one term's
                           contraction and ground leaving power), "ani_transport" (one
                           term's transport and stopping test; terms launched past
                           convergence return at once and count too), "ani_residual" (one
                           residual evaluation of the FP32 refinement) */
    long long launches; /* launches since the last read */
    double total_ms;    /* summed event time of those launches */
} tursca_kernel_stat;

/* Turn event timing on (1) or off (0).  While on, every launch of a profiled
 * kernel is bracketed by two events; the pool grows as needed. */
tursca_status tursca_profile_enable(tursca_scene *scene, int on);

/* Synchronise, fill out[0..n) with the per-kernel totals since the last read
 * (or enable), reset them, and set *n_out to the number of entries. */
tursca_status tursca_profile_read(tursca_scene *scene, tursca_kernel_stat *out, int n, int *n_out);

/* Host-only (no GPU): graph counts for a grid descriptor. */
tursca_status tursca_graph_info(const tursca_grid_desc *desc, tursca_graph_stats *out);

/* Host-only (no GPU): the CSR structure for a grid descriptor, into caller
 * host arrays sized by tursca_graph_info: row_ptr [n_nodes + 1], col [nnz],
 * dir [nnz], k [nnz] (same meaning as the TURSCA_F_* fields). */
tursca_status tursca_graph_structure(const tursca_grid_desc *desc, int32_t *row_ptr, int32_t *col, int16_t *dir,
                                     int8_t *k);

/* Host-only (no GPU): the Fibonacci-partition quadrature weights of the grid's
 * direction sets: q_iso [n_dirs] (cell fraction), q_lamb [n_gdirs]
 * (cosine-weighted fraction of the upper hemisphere). */
tursca_status tursca_quadrature(const tursca_grid_desc *desc, double *q_iso, double *q_lamb);

/* Allocation-free solve of (I - K) x = s for callers that may not allocate
 * device memory when they solve: programs whose device memory is owned by
 * their own allocator and fixed at start-up, or latency-critical loops where
 * cudaMalloc / cudaFree (which can synchronise the whole device) are not
 * allowed.  The paper has no counterpart; it is a deployment variant of the
 * refined solve that tursca_solve_with(..., TURSCA_SOLVER_NEUMANN, ...) runs.
 *
 * Computes, on cuda_stream, x = 0 then `refinements` times: sweeps of
 * d <- r + K d starting from d = r (FP32), x += d, r = s - (I - K) x (FP64).
 *   row_ptr [n_nodes + 1], col [nnz] (entries in [0, n_nodes)), val [nnz]:
 *     K in CSR, rows = receivers, any layout (e.g. TURSCA_F_ROW_PTR,
 *     TURSCA_F_COL, TURSCA_F_VAL of an FP32 scene); s [n_nodes] float;
 *     x [n_nodes] double (output); resid2: optional device double receiving
 *     ||r||^2 of the last refinement.  All are caller-owned device pointers.
 *   1 <= n_nodes <= 1048576, 0 <= sweeps <= 100000, 1 <= refinements <= 1000,
 *     and at most 10^6 launches ((sweeps + 2) * refinements + 2); larger sizes
 *     or null pointers return TURSCA_E_INVALID before any work.
 * Its work vectors live in one fixed device array of about 12 MiB that every
 * GPU loading the library holds until the process exits.  Every call looks up
 * that array's address in the current device's context (the first call in a
 * context loads the library's device code there; make that first call before
 * any stream capture).  Every call shares the array and finds the previous
 * call's contents in it, so calls whose work overlaps on the GPU (different
 * streams, or different host threads) race with each other.
 * Errors: TURSCA_E_CUDA, without launching anything, when a CUDA error is
 * already pending in the calling thread (it is left pending for its owner) or
 * the array's address cannot be found; TURSCA_E_CUDA when a launch fails (the
 * call stops at the first failed launch; later asynchronous faults surface at
 * the caller's next synchronisation).
 * The call allocates nothing and returns without synchronising. */
tursca_status tursca_csr_solve_noalloc(const int32_t *row_ptr, const int32_t *col, const float *val, int n_nodes,
                                       const float *s, double *x, int sweeps, int refinements, double *resid2,
                                       void *cuda_stream);

/* Self-test of the bounded device wait used by the pipelined passes
 * (TURSCA_OPT_STAGE_VALUES): one thread of one block waits, with those
 * passes' own wait (a bounded number of polls of an mbarrier phase), on a
 * barrier that receives its single expected arrival (arrive != 0) or none
 * (arrive == 0).  Returns TURSCA_OK when the wait completed and
 * TURSCA_E_TIMEOUT when it ran out (the kernel then returns normally and the
 * context stays usable); *seconds (may be NULL) receives the host time of the
 * call.  Allocates and frees 4 bytes of device memory and synchronises
 * cuda_stream.  TURSCA_E_CUDA on a CUDA error. */
tursca_status tursca_selftest_wait(void *cuda_stream, int arrive, double *seconds);

/* Static description of a status code. */
const char *tursca_status_string(tursca_status status);

/* Last error message recorded on the scene (or the last global error when
 * scene is NULL), NUL-terminated into buf[n]. */
tursca_status tursca_last_error(const tursca_scene *scene, char *buf, size_t n);

/* ---- Serving (continuous batching of scene solves).  The paper solves one
 * scene at a time (Sec. 3, step 4) and notes that the graph structure can be
 * reused across runs that change only the optical properties (Fig.
 * tursca-data); the server below is the deployment form of that: a pool of
 * resident scenes ("slots", one per grid shape and precision in use, each on
 * its own CUDA stream, keeping graph, tables and solver state between
 * requests) and worker threads that run each request's
 * set_medium -> assemble_flux -> solve -> render_radiance on a free slot.
 * Requests that arrive while others run are admitted as soon as a worker and
 * a slot are free; a request whose shape has no idle slot gets a new slot if
 * the slot's device memory fits the budget (idle slots of other shapes are
 * evicted, least recently used first, to make room) and otherwise waits.
 * Work of concurrent requests overlaps on the device.  Every request runs
 * the same deterministic kernels on its own scene, so its radiance does not
 * depend on what else runs (tested bit for bit). */
typedef struct tursca_server tursca_server;

typedef struct {
    double submit_ms;     /* times on the server's clock (ms since creation) */
    double start_ms;      /* a worker began the request */
    double end_ms;        /* the radiance was copied out */
    int slot_reused;      /* 1: ran on a resident slot, 0: a new slot was built */
    int iters;            /* solver products with K */
    double rel_resid64;   /* final relative residual */
    tursca_status status; /* the request's own status */
} tursca_request_info;

typedef struct {
    size_t budget_bytes, used_bytes, peak_bytes;
    int slots, busy_slots, pending, evictions, slots_built;
    /* batched Chebyshev refinements (see tursca_server_configure): launches,
     * refinements run in them, and the most in one launch */
    long long batches, batched_refinements;
    int max_batch;
} tursca_server_stats;

/* Server options (tursca_server_configure), to be set before the first
 * request:
 *   TURSCA_SERVER_BATCH_SOLVES: 0 (default) runs every request's passes on
 *     its own stream; 1 batches the Chebyshev refinements of the requests
 *     that run at the same time: a refinement handed over while others wait
 *     is launched together with them in one persistent kernel, which runs
 *     every request's row groups step after step with a grid-wide barrier
 *     between steps (every wait bounded); each request keeps its own step
 *     count and coefficients, and each group is computed by the same device
 *     code as the request's own Chebyshev pass, so a result does not depend
 *     on what it ran beside.  FP32 + refinement scenes whose pass has at most
 *     640 row groups (larger ones fill the GPU by themselves); two such
 *     launches may run at once, each on at most half the GPU. */
enum { TURSCA_SERVER_BATCH_SOLVES = 1 };
tursca_status tursca_server_configure(tursca_server *srv, int option, double value);

/* Self-test of the anisotropic mode's dense contractions (FP32 scenes with
 * a current assembly with TURSCA_OPT_ANISO): out[n][n_atm] (device, FP32)
 * gets the raw contraction of the current tables for every atmospheric
 * node, which = 0: sum_(w,sp) w_sp(j) zf(j,w) X(j,w) Q_sp(w -> n) with X a
 * device array [n_dirs + n_gdirs][n_nodes] (n < n_dirs); which = 1:
 * sum_(u,sp) w_sp(j) C(j,u) Q_sp(n -> u) (n < n_dirs + n_gdirs), the
 * denominators of the routing factors.  tensor_cores: 1 the tcgen05 kernel
 * (which = 0 only, TURSCA_E_UNSUPPORTED for 1; needs TURSCA_OPT_ANISO = 1 at
 * assembly), 0 the CUDA-core kernel.
 * Synchronises the scene's stream.  TURSCA_E_UNSUPPORTED for FP64 scenes,
 * TURSCA_E_STATE without such an assembly. */
tursca_status tursca_selftest_aniso_contract(tursca_scene *scene, int which, int tensor_cores, const void *X,
                                            void *out);

/* Self-test of the bounded grid barrier of the batched refinements: `blocks`
 * blocks of one cooperative launch wait at a barrier that expects all of
 * them (arrive != 0) or one more (arrive == 0, so it never completes).
 * TURSCA_OK when the barrier completed, TURSCA_E_TIMEOUT when every block
 * gave up (about a second; the kernel returns and the context stays
 * usable), TURSCA_E_CUDA on a CUDA error.  Synchronises cuda_stream. */
tursca_status tursca_selftest_barrier(void *cuda_stream, int blocks, int arrive);

/* hbm_budget_bytes: device memory the slots may hold together (>= the
 * largest single slot); max_concurrent: worker threads (1..64), i.e. requests
 * on the device at once.  Uses the current device. */
tursca_status tursca_server_create(size_t hbm_budget_bytes, int max_concurrent, tursca_server **out);

/* Queue one scene solve.  desc, geom: as for tursca_scene_create /
 * tursca_assemble_flux (copied).  mu_abs, mu_sca, g, albedo: as for
 * tursca_set_medium, host or device, borrowed until tursca_server_wait
 * returns for this ticket.  radiance: caller output [npy][npx] in the scene
 * precision, host or device.  rtol: as for tursca_solve.  Returns at once
 * with a ticket; invalid descriptors return TURSCA_E_INVALID. */
tursca_status tursca_server_submit(tursca_server *srv, const tursca_grid_desc *desc, const tursca_geometry *geom,
                                   const void *mu_abs, const void *mu_sca, const double *g, double albedo,
                                   double rtol, void *radiance, long long *ticket);

/* Block until the request completes; info may be NULL.  Returns the
 * request's status (the ticket is released). */
tursca_status tursca_server_wait(tursca_server *srv, long long ticket, tursca_request_info *info);

tursca_status tursca_server_stats_get(tursca_server *srv, tursca_server_stats *out);

/* Waits for all queued requests, then frees every slot. */
tursca_status tursca_server_destroy(tursca_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* TURSCA_H */

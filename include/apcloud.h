/*
 * apcloud.h -- C ABI of the GB300 AP-Cloud electrostatic solve.
 *
 * The library computes the electric potential and field of N charged
 * particles with the Adaptive Particle-in-Cloud method (Wang, Samulyak, Jiao,
 * Yu, arXiv 1603.04039): the Poisson equation  Lap phi = c rho  (Section 2,
 * Eq. Poisson) is discretised by second-order generalized finite differences
 * on the centres of an adaptive octree (Section 3), with E = grad phi.
 *
 * Call order for one solve (Section 3.2, "three steps", preceded by the tree
 * construction of Section 4):
 *     apcloud_build_octree -> apcloud_stencils -> apcloud_deposit
 *       -> apcloud_solve -> apcloud_gather_field
 * A call out of this order returns APCLOUD_E_STATE.  apcloud_field_host runs
 * the whole sequence on host arrays.
 *
 * Conventions shared by every entry point:
 *   - Pointers named d_* are device pointers (for example the data pointer of
 *     a CUDA tensor); pointers named h_* and the info/size out-parameters are
 *     host pointers.  The caller owns every array it passes.
 *   - All device work is ordered on the CUDA stream given to apcloud_create.
 *     Only apcloud_build_octree (node counts), apcloud_deposit and
 *     apcloud_solve (convergence checks) and the introspection getters
 *     synchronise that stream.
 *   - apcloud_build_octree keeps the position pointers; they must stay valid
 *     and unchanged until the next apcloud_build_octree (apcloud_gather_field
 *     reads them again).  No other input pointer is retained.
 *   - No exception or abort crosses the ABI.  Negative status = error (the
 *     outputs of that call are undefined, apcloud_last_error() explains);
 *     positive status = warning (outputs valid).
 *   - Node order: interior nodes (octree leaves) in Morton order of their
 *     lowest corner, then boundary nodes ordered by (face 0..5 = -x,+x,-y,+y,
 *     -z,+z, owner leaf).
 */
#ifndef APCLOUD_H
#define APCLOUD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    APCLOUD_OK = 0,
    APCLOUD_W_NOT_CONVERGED = 1, /* a Krylov solve reached max_iter first */
    APCLOUD_E_INVALID = -1,      /* bad argument or parameter */
    APCLOUD_E_DOMAIN = -2,       /* a particle lies outside the domain or is NaN */
    APCLOUD_E_STENCIL = -3,      /* a node has no full-rank stencil within ring_max */
    APCLOUD_E_CUDA = -4,         /* a CUDA call failed */
    APCLOUD_E_NOMEM = -5,        /* device allocation failed */
    APCLOUD_E_TIMEOUT = -6,      /* a bounded device wait gave up */
    APCLOUD_E_STATE = -7,        /* call out of order */
    APCLOUD_E_NUMERIC = -8       /* a factorisation met a zero pivot */
} apcloud_status;

/* Method parameters (defaults from apcloud_default_params). */
typedef struct {
    double lo[3], hi[3]; /* cubic domain Omega (Section 5: [-1,1]^3); hi-lo equal on all axes */
    int max_depth;       /* deepest octree level, 0..21 (64-bit Morton key, Section 4.3) */
    double c_refine;     /* tuning constant c of the error-balance criterion
                            h < c N'^(-1/2) (Section 4.3, k = 2) */
    int m_target;        /* GFD neighbours per node before distance ties, 9..32 (Section 3.1) */
    int ring_max;        /* widest k-ring searched for a stencil, 2..5 (Section 4.3) */
    double weight_c;     /* constant c of the normalized Gaussian weight, 4 (Section 3.1) */
    double poisson_c;    /* c in Lap phi = c rho (Eq. Poisson), 1 in Section 5 */
    int restart;         /* GMRES restart length, 1..64 */
    int precision;       /* 0 = FP64 throughout; 1 = mixed: FP32 WLS stencils with FP64
                            refactorisation of blocks the FP32 factorisation cannot certify
                            (fp32_rcond_min below),
                            FP32 GMRES iterations inside an FP64 iterative-refinement loop
                            (FP64 residual and solution), FP64 charge sums and gather */
    int poly_degree;     /* right preconditioner of GMRES: 1 = Jacobi; d > 1 = Jacobi-Neumann
                            polynomial omega sum_{i<d} (I - omega D^-1 A)^i, i.e. d damped
                            Jacobi sweeps per Arnoldi step (1..32) */
    double poly_omega;   /* damping omega of those sweeps, 0 < omega < 2 */
    double fp32_rcond_min; /* mixed form: a stencil block whose FP32 factorisation gives a
                              condition estimate min|R_ii| / max|R_ii| below this value (or
                              fails) is refactorised in FP64; 0..2, default 1e-3 (FP32
                              Cholesky QR squares the condition number).  apcloud_get_sizes
                              counts those blocks. */
    int stencil_slots;     /* k-ring candidates a node may gather in the first stencil pass,
                              16..128 (default 128); a node whose ring outgrows them is
                              redone in a second pass with 512 slots, with the same result
                              (launch mechanics, no counterpart in the paper) */
} apcloud_params;

/* Optional device allocator; NULL selects cudaMallocAsync/cudaFreeAsync on
 * the context stream.  alloc returns NULL on failure. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, void *stream, void *user);
    void *user;
} apcloud_allocator;

typedef struct {
    int iters;        /* Krylov iterations (matrix-vector products of the Arnoldi loop) */
    int restarts;     /* restart cycles */
    double relres;    /* final ||b - A x|| / ||b||, recomputed after the last cycle */
} apcloud_solve_info;

typedef struct apcloud_ctx apcloud_ctx;

/* Fills *p with the defaults: domain [-1,1]^3, max_depth 6, c_refine 1,
 * m_target 20, ring_max 5, weight_c 4, poisson_c 1, restart 30, FP64,
 * Jacobi preconditioning (poly_degree 1, poly_omega 0.7), fp32_rcond_min 1e-3,
 * stencil_slots 128. */
void apcloud_default_params(apcloud_params *p);

/* Creates a context bound to `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream) on the current device.  Validates *params. */
apcloud_status apcloud_create(const apcloud_params *params, const apcloud_allocator *alloc, void *cuda_stream,
                              apcloud_ctx **out);

/* Frees every buffer the context owns.  NULL is ignored. */
void apcloud_destroy(apcloud_ctx *ctx);

/* Message for the last non-OK status of this context (static storage of the context). */
const char *apcloud_last_error(const apcloud_ctx *ctx);

/* Section 4 (tree) and Sections 4.1-4.3 (node selection): Morton keys of the
 * n particles, key sort, error-balance refinement, minimal 2:1 face balance,
 * boundary nodes (one per leaf face on the domain boundary) and face
 * adjacency.  d_x, d_y, d_z: device FP64 arrays of n positions.  Writes the
 * interior (leaf) and boundary node counts.  Synchronises once.
 * Errors: APCLOUD_E_DOMAIN if a position is outside [lo, hi] or NaN. */
apcloud_status apcloud_build_octree(apcloud_ctx *ctx, const double *d_x, const double *d_y, const double *d_z,
                                    int64_t n, int64_t *n_interior, int64_t *n_boundary);

/* Batch of independent problems ("beams"): n_beams particle sets that share
 * the domain and the parameters, beam b holding particles
 * h_offsets[b] .. h_offsets[b+1]-1 of d_x, d_y, d_z (h_offsets: host array of
 * n_beams + 1 non-decreasing entries, h_offsets[0] = 0).  Each beam gets the
 * octree, node set, stencils and linear systems it would get alone (Sections
 * 3-4 per beam); the beams are laid out as one block-diagonal problem, so
 * every later call (stencils, deposit, solve, gather) processes all beams in
 * the same launches.  Interior nodes are ordered by beam, then Morton order;
 * boundary nodes by face, then owner leaf.  Leaf keys (apcloud_get_leaves)
 * carry the beam index above the 3*level Morton bits.  In a batch every
 * beam stops at its own ||r_b|| <= rtol ||b_b||.  With the polynomial
 * preconditioner (poly_degree > 1) every beam runs its own GMRES(restart) --
 * own Krylov space, Hessenberg matrix and stopping test -- inside the same
 * launches, and info.relres is the largest relative residual over the beams.
 * With Jacobi alone the batch shares one Krylov space and freezes the beams
 * that have converged at each restart (their residual rows are zeroed and
 * skipped); info.relres is then 0 once all have converged.  In both cases
 * info.iters counts the Arnoldi steps of the longest-running beam.  The
 * paper treats one problem at a time; the
 * batch is this library's.  Errors: APCLOUD_E_INVALID for bad offsets or
 * when 3*max_depth plus the bits of n_beams - 1 exceed 63. */
#define APCLOUD_MAX_BEAMS 65536
apcloud_status apcloud_build_octree_batched(apcloud_ctx *ctx, const double *d_x, const double *d_y,
                                            const double *d_z, const int64_t *h_offsets, int n_beams,
                                            int64_t *n_interior, int64_t *n_boundary);

/* Beam index of every node after an octree build (device int32, n_nodes
 * entries; boundary nodes take their owner leaf's beam).  Synchronises. */
apcloud_status apcloud_get_node_beams(apcloud_ctx *ctx, int32_t *d_beam);

/* Node geometry after apcloud_build_octree, device outputs of n_nodes =
 * n_interior + n_boundary entries (any may be NULL): d_xyz FP64 [n_nodes][3]
 * centres, d_level int8 (owner's level for boundary nodes), d_kind int8
 * (0 interior, 1 boundary). */
apcloud_status apcloud_get_nodes(apcloud_ctx *ctx, double *d_xyz, int8_t *d_level, int8_t *d_kind);

/* Leaf data after apcloud_build_octree (device, n_interior entries each, any
 * may be NULL): Morton key of the leaf at its own level, first particle in
 * key-sorted order and particle count N' (Section 4). */
apcloud_status apcloud_get_leaves(apcloud_ctx *ctx, uint64_t *d_key, int32_t *d_first, int32_t *d_count);

/* Section 3.1 with the neighbour search of Section 4.3: for every interior
 * node, grow k-rings (k = 2..ring_max) over face adjacency, pick two nearest
 * per octant then the nearest up to m_target plus every candidate tied at the
 * cut distance (at most 32), build the weighted scaled Vandermonde V0 with
 * the normalized Gaussian weight, factor it, and keep the pseudo-inverse
 * operator (gradient and Hessian weights) and the Laplacian row.  Assembles
 * the density matrix B and the Poisson matrix A (Section 3.2).
 * Errors: APCLOUD_E_STENCIL if some node has no full-rank stencil. */
apcloud_status apcloud_stencils(apcloud_ctx *ctx);

/* Stencils after apcloud_stencils (device, any may be NULL): d_nbr int32
 * [n_interior][32] neighbour node indices in increasing distance, -1 padded;
 * d_m int32 stencil sizes; d_lap FP64 [n_interior][32] Laplacian weights;
 * d_lapdiag FP64 diagonal (minus their sum); d_D FP64 [n_interior][9][32]
 * derivative operator, rows f_x f_y f_z f_xx f_xy f_xz f_yy f_yz f_zz. */
apcloud_status apcloud_get_stencils(apcloud_ctx *ctx, int32_t *d_nbr, int32_t *d_m, double *d_lap,
                                    double *d_lapdiag, double *d_D);

/* Step 1 of Section 3.2 (Eq. density_apcloud to Eq. density_linear_system)
 * with the cell-indicator kernel of Section 5: rho_M of every leaf = sum of
 * its particles' charges / h^3, then solve B rho~ = rho_M by GMRES to `rtol`.
 * d_q: device FP64 charges in the caller's particle order, or NULL for
 * q_uniform on every particle.  d_rho_out (optional, device, n_nodes):
 * rho~.  info (optional, host) receives the solve statistics.
 * Returns APCLOUD_W_NOT_CONVERGED if max_iter was reached. */
apcloud_status apcloud_deposit(apcloud_ctx *ctx, const double *d_q, double q_uniform, double rtol, int max_iter,
                               double *d_rho_out, apcloud_solve_info *info);

/* rho_M after apcloud_deposit (device, n_nodes; boundary entries are the
 * owner's value). */
apcloud_status apcloud_get_rho_m(apcloud_ctx *ctx, double *d_rho_m);

/* Step 2 of Section 3.2: A phi = poisson_c rho~ on interior rows and
 * phi_b = g_b on boundary rows (Dirichlet data).  d_g: device FP64
 * [n_boundary] or NULL for g = 0.  d_phi0: device initial guess [n_nodes] or
 * NULL for zero.  d_phi_out (optional, device, n_nodes).  GMRES(restart) with
 * right Jacobi preconditioning to ||b - A phi|| <= rtol ||b||.
 * Returns APCLOUD_W_NOT_CONVERGED if max_iter was reached. */
apcloud_status apcloud_solve(apcloud_ctx *ctx, const double *d_g, const double *d_phi0, double rtol, int max_iter,
                             double *d_phi_out, apcloud_solve_info *info);

/* Step 3 of Section 3.2: GFD gradient and Hessian of phi at every interior
 * node, then second-order Taylor expansion about the centre of each
 * particle's leaf: phi_p, and E_p = grad phi (Section 2).  Outputs are device
 * FP64 arrays of n particles in the caller's order (any may be NULL). */
apcloud_status apcloud_gather_field(apcloud_ctx *ctx, double *d_phi_p, double *d_ex, double *d_ey, double *d_ez);

/* Node derivatives after apcloud_gather_field: device FP64 [n_interior][9]. */
apcloud_status apcloud_get_derivatives(apcloud_ctx *ctx, double *d_dphi);

/* y = A x (which = 1) or y = B x (which = 0) with the assembled matrices;
 * device FP64 vectors of n_nodes entries. */
apcloud_status apcloud_matvec(apcloud_ctx *ctx, int which, const double *d_x, double *d_y);

/* Solves B x = b (which = 0) or A x = b (which = 1) for an arbitrary
 * right-hand side with the same GMRES; d_x holds the initial guess on entry. */
apcloud_status apcloud_solve_system(apcloud_ctx *ctx, int which, const double *d_b, double *d_x, double rtol,
                                    int max_iter, apcloud_solve_info *info);

/* Allocation-free GMRES solve, for callers that cannot allocate device
 * memory once their setup is done: a host whose device memory is all handed
 * out up front (a fixed budget, or a memory manager that owns every byte of
 * the device and rejects cudaMalloc), or a real-time loop where a pool
 * growing or a cudaMalloc stalling the device is not acceptable.  The paper
 * has no counterpart; this is a deployment convenience.
 * It solves B x = b (which = 0) or A x = b (which = 1) by FP64 GMRES(restart)
 * with Jacobi preconditioning, one Krylov space and one stopping test
 * ||b - A x|| <= rtol ||b||: the algorithm apcloud_solve_system runs in an
 * FP64 single-beam context with poly_degree 1, giving the same iterations and
 * results there.  Other contexts (precision 1, poly_degree > 1, or a batch of
 * beams) return APCLOUD_E_INVALID.  The Krylov basis, work vectors,
 * reduction partials and device state live in one file-scope device array
 * of 20 MiB, which every GPU that loads the library holds until the process
 * exits; the call allocates nothing and kernel timers are ignored during it.
 * Limits: at most 65536 nodes (interior + boundary) and restart <= 30;
 * larger problems return APCLOUD_E_INVALID.  The context's device must be
 * the current device (APCLOUD_E_INVALID otherwise).  The first call on a
 * device also looks up the array's device address (cudaGetSymbolAddress).
 * The call reads the residual back to the host once per restart cycle, so it
 * synchronises the context stream every cycle and must not be called while
 * that stream is being captured into a CUDA graph.  All calls share the one
 * array: two calls whose work overlaps on the GPU (other streams, other
 * contexts, other host threads) race and give undefined results; each call
 * clears the state it needs, since the array keeps the previous call's
 * contents. */
apcloud_status apcloud_solve_system_noalloc(apcloud_ctx *ctx, int which, const double *d_b, double *d_x,
                                            double rtol, int max_iter, apcloud_solve_info *info);

/* ILU(0)-preconditioned GMRES(restart) on the density (which = 0) or Poisson
 * (which = 1) system: the comparison baseline for the learned preconditioner
 * (besides Jacobi).  The paper has no counterpart.  ILU(0) is the incomplete
 * LU factorisation with no fill outside the pattern of the stored matrix
 * (Saad, Iterative Methods for Sparse Linear Systems, Algorithm 10.4, IKJ
 * order), taken of the stored column-scaled FP64 values; it is computed on
 * the host at every call, and every application (LU)^-1 v runs on the GPU as
 * a forward and a backward sweep of dependency levels: one launch for each
 * level wider than 4096 rows, one single-block launch for each run of
 * narrower levels between them (no CUDA graphs).  d_b, d_x and the result are as in apcloud_solve_system (x is the
 * start and the answer, n = interior + boundary nodes, device memory).  FP64
 * form (precision 0) and single-beam contexts only, else APCLOUD_E_INVALID;
 * APCLOUD_E_NUMERIC on a zero pivot.  h_stats (NULL or 4 doubles) receives the
 * host setup milliseconds (copy, factorisation, level schedule, upload), the
 * numbers of forward and backward levels, and the stored nonzeros.
 * Synchronises the context stream. */
apcloud_status apcloud_solve_system_ilu0(apcloud_ctx *ctx, int which, const double *d_b, double *d_x, double rtol,
                                         int max_iter, apcloud_solve_info *info, double *h_stats);

/* The ILU(0) factorisation of the comparison solve on a host CSR matrix, in
 * place: n rows, h_rowptr[n + 1], column indices h_col sorted and distinct in
 * every row, each row holding its diagonal; h_val is overwritten with the
 * strict lower part of L (unit diagonal implied) and U.  Host memory only; no
 * GPU is used.  APCLOUD_E_INVALID on a malformed pattern, APCLOUD_E_NUMERIC
 * on a zero pivot. */
apcloud_status apcloud_ilu0_factor_host(int64_t n, const int64_t *h_rowptr, const int32_t *h_col, double *h_val);

/* The whole solve on host arrays: copies positions and charges (h_q NULL =
 * q_uniform) to the device, runs the five steps with g = 0, and copies phi
 * and E at the particles back.  Host arrays may be pageable or pinned; pinned
 * memory makes the copies asynchronous, and the charges' copy then runs on a
 * second stream of the context while the tree and the stencils are built.
 * Returns with no copy from or to the host arrays in flight, on every path. */
apcloud_status apcloud_field_host(apcloud_ctx *ctx, const double *h_x, const double *h_y, const double *h_z,
                                  const double *h_q, double q_uniform, int64_t n, double rtol, int max_iter,
                                  double *h_phi, double *h_ex, double *h_ey, double *h_ez,
                                  apcloud_solve_info *info_rho, apcloud_solve_info *info_phi);

/* apcloud_field_host for a batch of beams (see apcloud_build_octree_batched):
 * h_offsets (host, n_beams + 1 entries) splits the h_offsets[n_beams]
 * particles into beams; outputs are in the input order. */
apcloud_status apcloud_field_host_batched(apcloud_ctx *ctx, const double *h_x, const double *h_y,
                                          const double *h_z, const double *h_q, double q_uniform,
                                          const int64_t *h_offsets, int n_beams, double rtol, int max_iter,
                                          double *h_phi, double *h_ex, double *h_ey, double *h_ez,
                                          apcloud_solve_info *info_rho, apcloud_solve_info *info_phi);

/* ---- time stepping (Vlasov-Poisson, the setting of the paper's title) ----
 * The paper gives no time integrator; these entry points support a leapfrog
 * in which every step rebuilds the tree, stencils and systems (Section 4
 * onward) for the moved particles. */

/* phi at n arbitrary points (device FP64 SoA x, y, z inside the domain) from
 * this context's last solution: second-order Taylor expansion about the
 * centre of the point's leaf, as apcloud_gather_field does for particles.
 * Used to warm-start the next step's solve on a new node set.  Requires
 * apcloud_gather_field on a single-beam context (APCLOUD_E_INVALID for a
 * batch). */
apcloud_status apcloud_interpolate_potential(apcloud_ctx *ctx, const double *d_x, const double *d_y,
                                             const double *d_z, int64_t n, double *d_phi);

/* One leapfrog half step on n particles (device FP64 arrays, updated in
 * place): v += qm_dt * E if the field arrays are given (all three or none),
 * then x += dt * v with specular reflection at the walls of the cubic domain.
 * E = grad phi as in Section 2.  Does not need a solved context. */
apcloud_status apcloud_push_particles(apcloud_ctx *ctx, double *d_x, double *d_y, double *d_z, double *d_vx,
                                      double *d_vy, double *d_vz, int64_t n, const double *d_ex,
                                      const double *d_ey, const double *d_ez, double qm_dt, double dt);

/* CUDA graphs: every full GMRES restart cycle (its Arnoldi steps,
 * Gram-Schmidt reductions, preconditioner sweeps, the update of the iterate
 * and the residual that opens the next cycle) is captured once per set of
 * buffers and sizes and replayed with one cudaGraphLaunch on the context
 * stream; the host synchronises once per cycle for the convergence test.
 * Arnoldi step j >= 1 of a captured cycle is the body of a conditional (IF)
 * node that the previous step sets while the cycle's stopping test has not
 * passed, so the steps after it are skipped on the device.  On by default;
 * enable = 0 launches every kernel directly and reads the stopping flag back
 * after every Arnoldi step (the same kernels in the same order, the same
 * results).  Kernel timers (apcloud_set_timing) also run cycles as direct
 * launches, stopped the same way.  Synchronises the context stream.  The
 * paper has no counterpart (launch mechanics). */
apcloud_status apcloud_set_graphs(apcloud_ctx *ctx, int enable);

/* Autotuner of the launch shapes (after apcloud_stencils): bit 0 of `what`
 * times a whole solve of the Poisson system A (configured solver, CUDA graphs
 * included; a synthetic right-hand side, relative residual 1e-10 or 1000
 * Arnoldi steps; one untimed solve first, then the best of two timed
 * ones) for every shape of the
 * row-parallel products: 64, 128, 256 and 512 threads per block, each with
 * the loads of 1 or 4 stencil entries issued ahead of their multiply-adds
 * (on the width-sorted copy: 1 or 2 chunks of 4 entries; the sum keeps its
 * order either way), and -- for the FP16 sweeps and FP32 Arnoldi products of
 * the mixed form -- on the sliced ELL and on its width-sorted copy (rows
 * ordered by stencil width inside 256-row windows, so 32-row slices carry
 * little padding; same entries in the same order per row).  The solves run on scratch vectors and the
 * graphs they capture are released; bit 1 times the stencil build (neighbour
 * search + WLS) at 2, 4 and 8 nodes (warps) per block on the current node
 * set.  The fastest shapes are kept for later calls and written to
 * *h_spmv_block, *h_spmv_unroll, *h_sweep_sorted and *h_wls_warps (any may be
 * NULL); h_ms (NULL or 19 doubles) receives the measured milliseconds: 16
 * solves (index = block-size index + 4 * unroll-4 + 8 * sorted; variants not
 * timed stay 0), then three stencil builds.  Results never depend on the
 * shapes.  Runs on the context stream and synchronises.  The paper has no
 * counterpart (launch mechanics). */
apcloud_status apcloud_autotune(apcloud_ctx *ctx, unsigned what, int *h_spmv_block, int *h_spmv_unroll,
                                int *h_sweep_sorted, int *h_wls_warps, double *h_ms);

/* Sets the launch shapes directly: spmv_block in {64, 128, 256, 512},
 * spmv_unroll in {1, 4}, sweep_sorted in {0, 1}, wls_warps in {2, 4, 8};
 * APCLOUD_E_INVALID otherwise. */
apcloud_status apcloud_set_launch_shape(apcloud_ctx *ctx, int spmv_block, int spmv_unroll, int sweep_sorted,
                                        int wls_warps);

/* L2 residency of the FP16 sweep matrix (width-sorted copy with packed
 * columns, the mixed form's polynomial preconditioner).  The sweeps of one
 * polynomial application read the whole matrix one after another; a sweep
 * loads its first keep_bytes of matrix bytes (5 per stored entry) as
 * ordinary loads and the rest as streaming loads (ld.global.cs: lines
 * allocated evict-first in L2), so that the streamed part replaces itself in
 * L2 and the kept part is still there for the next sweep.  keep_bytes = -1
 * (the default): 0.4 of the L2 when the matrix and the sweep's vectors (12
 * bytes per row) take between 3/4 of the L2 and twice the L2, else all of
 * the matrix (no streaming loads); 0: every matrix load streaming; larger
 * than the matrix: none.
 * Results are bit-identical for every value (the same loads in the same
 * order).  APCLOUD_E_INVALID for keep_bytes < -1.  The getter writes the
 * value in effect for the current node set (the automatic choice resolved;
 * INT64_MAX when no load is streaming).  The paper has no counterpart (cache
 * mechanics). */
/* Programmatic dependent launch of the polynomial's sweeps (on by default):
 * every sweep after the first of an application is launched so that its
 * blocks may start while the sweep before it drains; each row reads its
 * slice, b, the solver state and its first matrix chunks, then waits on the
 * device (griddepcontrol.wait) for the previous sweep to complete before it
 * reads x or writes y.  enable = 0 launches every sweep in plain stream
 * order.  Results are bit-identical either way.  The paper has no
 * counterpart (launch mechanics). */
apcloud_status apcloud_set_dependent_launch(apcloud_ctx *ctx, int enable);

apcloud_status apcloud_set_sweep_l2_keep(apcloud_ctx *ctx, int64_t keep_bytes);
apcloud_status apcloud_get_sweep_l2_keep(const apcloud_ctx *ctx, int64_t *h_keep_bytes);

/* Graph replays since the context was created and graphs currently cached. */
apcloud_status apcloud_graph_stats(const apcloud_ctx *ctx, int64_t *h_replays, int64_t *h_cached);

/* Field energy 1/2 sum_j |grad phi_j|^2 h_j^3 over the leaves (node gradients
 * from the last apcloud_gather_field times cell volumes), FP64, fixed order. */
apcloud_status apcloud_field_energy(apcloud_ctx *ctx, double *h_energy);

/* ---- learned preconditioner (no counterpart in the paper) ----
 * A message-passing network over the GFD stencil graph proposes, for the
 * Poisson system A phi = c rho of Section 3.2 step 2, a diagonal right
 * preconditioner and an initial guess.  With Ahat = A D^-1 (D = diag A):
 *   W = |Ahat_off| + |Ahat_off|^T, P = W normalised by its row sums;
 *   H_0 = 16 node features (row and column sums of the WLS weights through
 *   sign(f) log(1 + |f|), mean neighbour offset and level offset, b and P b
 *   scaled by max|b|, degree);
 *   H_{l+1} = relu([H_l | P H_l] W_l + b_l), l = 0, 1, 2, width 64;
 *   t = H_3 W_o + b_o; s = exp(ln 8 tanh t_0) on interior nodes, 1 on
 *   boundary nodes (identity rows); gamma = exp(tanh t_1).
 * The solve then runs GMRES on Ahat S (columns scaled by s) from the guess
 * x0 = gamma b / D.  Training minimises L = Lp + Lg with
 *   Lp = (1/n_int) sum over interior columns of ||e_j - Ahat S e_j||^2
 *   (approximate-inverse objective; its minimiser is s_j = 1/||Ahat e_j||^2),
 *   Lg = ||b - Ahat (gamma b)||^2 / ||b||^2 (initial residual of the guess).
 * Dense layers and their gradients run on the tensor cores in BF16 with FP32
 * accumulation; master weights are FP32.  Flat parameter layout (FP32):
 *   W0 [32][64], b0 [64], W1 [128][64], b1 [64], W2 [128][64], b2 [64],
 *   Wo [64][2], bo [2]  (apcloud_mpnn_num_params() values).
 * A network object lives on the device that was current at creation and
 * may be used with any context on that device. */
typedef struct apcloud_mpnn apcloud_mpnn;

int apcloud_mpnn_num_params(void);

/* Creates a network with the given host parameters, or (h_theta NULL)
 * Glorot-uniform layers drawn from SplitMix64(seed) with zero biases and a
 * zero head, which is exactly Jacobi (s = 1) with the guess gamma = 1.
 * Synchronises the device. */
apcloud_status apcloud_mpnn_create(const float *h_theta, uint64_t seed, apcloud_mpnn **out);
void apcloud_mpnn_destroy(apcloud_mpnn *net);

/* Host copies of the parameters and of the last gradient (either NULL),
 * and replacement of the parameters (which also clears the Adam moments).
 * Both synchronise the device. */
apcloud_status apcloud_mpnn_get_params(apcloud_mpnn *net, float *h_theta, float *h_grad);
apcloud_status apcloud_mpnn_set_params(apcloud_mpnn *net, const float *h_theta);

/* Loss of the network on ctx's current Poisson system (after
 * apcloud_deposit; boundary data g = 0): h_loss[3] = {L, Lp, Lg}.  With
 * backward != 0 also the gradient dL/dtheta (kept in the network for
 * apcloud_mpnn_adam).  Synchronises.  APCLOUD_E_TIMEOUT if a tensor-core
 * layer gave up waiting for its MMAs. */
apcloud_status apcloud_mpnn_loss(apcloud_ctx *ctx, apcloud_mpnn *net, int backward, double *h_loss);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr on the
 * last gradient, on ctx's stream. */
apcloud_status apcloud_mpnn_adam(apcloud_ctx *ctx, apcloud_mpnn *net, float lr);

/* Network outputs on ctx's current Poisson system (device FP32, n_nodes
 * entries each, any NULL): column scaling s, guess factor gamma, and the
 * n_nodes x 16 node features.  Synchronises. */
apcloud_status apcloud_mpnn_outputs(apcloud_ctx *ctx, apcloud_mpnn *net, float *d_s, float *d_gamma,
                                    float *d_features);

/* apcloud_solve (g = 0) with the network's proposals: bit 0 of `use` scales
 * the preconditioner columns by s, bit 1 starts from x0 = gamma b / D, bit 2
 * scales by the closed-form minimiser 1/||Ahat e_j||^2 of the same objective
 * instead of the network's s (the comparison baseline).  Without bit 1 the
 * start is d_phi0 (device, n_nodes values) or 0 when it is NULL; use = 0 is
 * plain apcloud_solve.  The scaled solve gets at most 1000 Arnoldi steps; if
 * it has not converged by then, the plain Jacobi-scaled solve runs from the
 * original start (the fallback; info counts both phases).  The stored
 * matrix is restored afterwards.  The residual test is the same FP64 true
 * residual, so the network can change the iteration count, never the
 * accuracy. */
apcloud_status apcloud_solve_learned(apcloud_ctx *ctx, apcloud_mpnn *net, unsigned use, const double *d_phi0,
                                     double rtol, int max_iter, double *d_phi_out, apcloud_solve_info *info);

/* Per-kernel device timing with CUDA events on the context stream.
 * apcloud_set_timing(ctx, mask) enables timing for the kernel kinds whose
 * bit is set in mask (bit k = kind k, see apcloud_kernel_name), 0 disables.
 * apcloud_get_timing synchronises and returns, for kind k (host arrays of
 * APCLOUD_NUM_KINDS entries, any may be NULL): summed milliseconds, launch
 * count, and the algorithmic bytes and floating-point operations of those
 * launches (what the kernel must move and compute, not what it did), since
 * the last reset (reset = 1 clears).  Consecutive launches of one timed kind
 * share one pair of events (before the first, after the last), so their time
 * includes the gaps between them; a launch of any other kind or a host
 * read-back closes the pair. */
#define APCLOUD_NUM_KINDS 19
apcloud_status apcloud_set_timing(apcloud_ctx *ctx, unsigned mask);
apcloud_status apcloud_get_timing(apcloud_ctx *ctx, double *h_ms, int64_t *h_launches, double *h_bytes,
                                  double *h_flops, int reset);
const char *apcloud_kernel_name(int kind);

/* Fused multiply-add throughput of the current device in TFLOP/s (2 flops per
 * FMA), FP64 and FP32, from independent FMA chains on every SM; allocates a
 * few MB temporarily and synchronises the device.  No paper counterpart: it
 * provides the ALU roofline of the FP64 kernels.  Either pointer may be NULL. */
apcloud_status apcloud_measure_fma_peak(double *h_fp64_tflops, double *h_fp32_tflops);

/* Problem sizes after the last completed step (host array of 9 int64):
 * particles, interior nodes, boundary nodes, matrix nonzeros (stencil
 * entries + diagonals + boundary rows), stored sliced-ELL entries (with
 * padding), sum of stencil sizes, ELL slices, octree depth, and (mixed form)
 * stencils refactored in FP64. */
apcloud_status apcloud_get_sizes(const apcloud_ctx *ctx, int64_t *h_sizes);

/* Total kernel launches issued by this context since creation. */
int64_t apcloud_launch_count(const apcloud_ctx *ctx);

/* Host read-backs since creation that waited for the context stream (tree
 * sizes, the convergence test of every restart cycle and refinement step,
 * introspection); each one idles the GPU between the work before and after
 * it.  No paper counterpart (launch mechanics). */
int64_t apcloud_host_sync_count(const apcloud_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* APCLOUD_H */

// internal.cuh -- shared declarations of the GB300 AP-Cloud library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "apcloud.h"

namespace apc {

constexpr int KEY_DEPTH = 21;   // 63-bit Morton keys (Section 4.3)
constexpr int NCOL = 9;         // unknowns of the 3-D second-order GFD system (Section 3.1)
constexpr int MMAX = 32;        // widest stencil, one warp lane per neighbour
constexpr int MAXC = 512;       // ring candidates held per node in shared memory
constexpr int MAXC_FAST = 128;  // the same in the stencil kernel over all nodes (overflow: redone with MAXC)
constexpr double RANK_TOL = 1e-6;
constexpr int MAX_RESTART = 64;

// kernel kinds for the event timers (bit k of the timing mask)
enum Kind {
    K_KEYS = 0, K_SORT, K_TREE, K_ADJ, K_STENCIL, K_ELL, K_DEPOSIT, K_SPMV,
    K_DOT, K_UPDDOT, K_UPDNORM, K_CYCLE, K_DERIV, K_GATHER, K_VEC, K_COPY, K_MPNN_TC, K_MPNN_GRAPH, K_SWEEP, NKIND
};
static_assert(NKIND == APCLOUD_NUM_KINDS, "kind count");

// device error word bits
enum : unsigned { ERR_DOMAIN = 1u, ERR_STENCIL = 2u, ERR_BALANCE = 4u, ERR_OVERFLOW = 8u, ERR_TIMEOUT = 16u };

struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Leaves are in Morton order and so are the particles, so the particle ranges
// [first_j, first_j + count_j) of consecutive leaves tile the key-sorted
// particles in order.  A warp can own 32 consecutive leaves (lane l holding
// leaf j0 + l's first particle, INT_MAX past the last leaf) and stream their
// particles coalesced.  The leaf of sorted particle i within such a group is
// the last lane whose first is <= i; an empty leaf shares its first with the
// next leaf and is never chosen.  All 32 lanes must call it.
__device__ __forceinline__ int group_leaf(int my_first, int i) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int f = __shfl_sync(0xffffffffu, my_first, lo + step);
        if (f <= i) lo += step;
    }
    return lo;
}

// GMRES bookkeeping kept on the device so that a whole restart cycle runs
// without host round trips.
struct GmresState {
    double H[(MAX_RESTART + 1) * MAX_RESTART];  // Hessenberg, row-major [i][j], rotated in place
    double cs[MAX_RESTART], sn[MAX_RESTART];
    double g[MAX_RESTART + 1];
    double y[MAX_RESTART];
    double h1[MAX_RESTART + 1];   // first Gram-Schmidt projection of the current column
    double h2[MAX_RESTART + 1];   // second projection
    // delayed reorthogonalisation (k_dcgs_dots): the tentative vector q_j of
    // slot j is w_{j-1} minus its first projection over an estimate nut of
    // its norm; its second projection s waits for step j
    double dq[MAX_RESTART + 1];   // s = V^T q_j
    double nu;                    // ||q_j - V s||
    double inu;                   // 1 / nu
    double nut;                   // the estimate that scaled q_j (then q_{j+1})
    double gpre;                  // g[j] before the tentative rotation of column j
    double bnorm;                 // ||b||
    double beta;                  // ||r|| at cycle start
    double inv_norm;              // 1 / ||w|| of the vector about to become V_{j+1}
    double rtol;
    double omega;                 // damping of the polynomial preconditioner sweeps
    int jend;                     // columns completed in this cycle
    int done;                     // 1 once the cycle must stop (converged or breakdown)
    unsigned ticket;              // grid-reduction ticket
    int jlast;                    // columns completed by the previous cycle
};

// A captured restart cycle (CUDA graph), keyed by everything its launches
// depend on: element size, sizes, timing mask and every buffer address.
struct GraphKey {
    int tsize, n, jmax, pdeg, nblk, spmv_bs, pdl;
    unsigned mask;
    int64_t ldv, skeep;
    const void *p[32];
};

// Arnoldi step j >= 1 of a captured cycle sits in an IF node whose condition
// (cond[j], reset to 0 at every replay) the last kernel of step j - 1 sets
// while the cycle's stopping test has not passed, so the steps after it are
// skipped on the device instead of launched.
struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;             // kernel nodes outside the step bodies (run at every replay)
    std::vector<int64_t> step_kernels;             // kernel nodes of the body of step j
    std::vector<cudaGraphConditionalHandle> cond;  // condition of step j's body (j >= 1)
    int cur_step = -1;               // body being captured (-1: none)
    bool broken = false;             // a capture step failed: the graph is discarded
    uint64_t last_use = 0;
};

// Per-kind kernel timers.  Consecutive launches of one timed kind share one
// event pair (one start before the first, one end after the last): any
// launch of another kind, timed or not, and any host read-back close it.
struct Timer {
    unsigned mask = 0;
    std::vector<cudaEvent_t> ev;   // pairs
    std::vector<int> kind;          // per pair
    std::vector<int> nl;            // launches per pair
    size_t used = 0;
    long open = -1;                 // pair still open (its end not recorded), or -1
    double ms[NKIND] = {0};
    int64_t launches[NKIND] = {0};
    double bytes[NKIND] = {0};   // algorithmic bytes of the timed launches
    double flops[NKIND] = {0};   // algorithmic floating-point operations
};

// ILU(0) factors on the device for the comparison solve: rows listed level by
// level (forward and backward), the strict lower / upper entries of each listed
// row, 1 / U_rr per backward position; level offsets on the host
// One launch of a triangular sweep: levels [l0, l1) either as one block that
// takes them in order (a run of small levels) or, for a single wide level, as
// a grid over its rows.
struct IluSeg {
    int l0, l1;
    bool wide;
};

struct IluDev {
    const int32_t *lrows = nullptr, *urows = nullptr, *lcol = nullptr, *ucol = nullptr;
    const int64_t *lrp = nullptr, *urp = nullptr;
    const double *lval = nullptr, *uval = nullptr, *udinv = nullptr;
    const int32_t *dloff = nullptr, *duoff = nullptr;   // loff, uoff on the device
    std::vector<int> loff, uoff;
    std::vector<IluSeg> lseg, useg;
};

}  // namespace apc

struct apcloud_ctx {
    apcloud_params P;
    apcloud_allocator A;
    bool default_alloc = true;
    cudaStream_t s = nullptr;
    int device = 0;  // device current at apcloud_create; the context's buffers live there
    int stage = 0;  // 0 created, 1 octree, 2 stencils, 3 deposit, 4 solved, 5 gathered
    char err[512] = {0};
    int64_t launches = 0;
    int64_t host_syncs = 0;   // read-backs that waited for the stream
    apc::Timer timer;
    // launch shapes chosen by apcloud_autotune
    int spmv_bs = 256;     // threads per block of the Arnoldi products and sweeps
    int spmv_unroll = 1;   // stencil entries whose loads a thread issues ahead (1 or 4)
    int sweep_sorted = 0;  // 1: FP16 sweeps on the width-sorted matrix (autotuner's choice)
    bool pdl_on = true;        // sweeps after the first of a polynomial application as programmatic dependents
    int64_t sweep_keep = -1;   // bytes of that matrix the sweeps read with ordinary loads, the rest streaming (-1: automatic)
    int jprev[2][2] = {{0, 0}, {0, 0}};   // Arnoldi steps of the last cycle, per system (B, A) and FP64/FP32
    int wls_warps = 4;     // nodes (warps) per block of the stencil build
    // CUDA graphs of GMRES restart cycles (captured on cap_stream, replayed on s)
    bool graphs_on = true;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t body_stream = nullptr;   // capture of conditional step bodies
    cudaStream_t copy_stream = nullptr;   // host copies that overlap the tree build (field_host)
    cudaEvent_t copy_done = nullptr;
    apc::GraphEntry *capturing = nullptr;
    apc::GraphEntry *last_stepped = nullptr;   // last replayed graph whose step kernels are not counted yet
    std::vector<apc::GraphEntry *> graphs;
    uint64_t graph_clock = 0;
    int64_t graph_replays = 0;
    bool stopped = false;   // timed direct launches: the cycle's stopping test passed

    // particles (caller's device arrays, kept until the next build)
    const double *px = nullptr, *py = nullptr, *pz = nullptr;
    int64_t N = 0;

    // batch of independent problems (beams) sharing the domain and parameters
    int nbeams = 1, beam_bits = 0;
    std::vector<int64_t> h_beam_off;
    // sizes
    int L = 0;
    int n_int = 0, n_bnd = 0, n_tot = 0;
    int n_slices = 0;
    int64_t ell_entries = 0;
    int64_t sum_m = 0;  // total stencil neighbours over interior nodes
    int64_t n_fp64_wls = 0;  // mixed form: stencils refactored in FP64

    // sorted particle keys and permutation (result in key[kbuf], val[kbuf])
    apc::DBuf key[2], val[2];
    int kbuf = 0;
    // tree temporaries
    apc::DBuf ucell[2], ustart[2], opened, cand[2], cval[2], flags, scan, scan_blk, lkey, lval;
    // nodes
    apc::DBuf leaf_anchor, leaf_level, leaf_first, leaf_count, node_ic, bowner, bface, bidx, adj;
    apc::DBuf pleaf;   // leaf of every particle, in the caller's particle order
    apc::DBuf spos;    // key-sorted position of every particle, in the caller's order
    apc::DBuf qsort;   // charges in key-sorted order (deposit)
    apc::DBuf beam_off, leaf_beam, beam_rng, beam_norm, beam_r2, beam_done, node_beam, tile_act;
    apc::DBuf bk_items, bk_ioff, bk_d, bk_i;   // per-beam Krylov spaces of a batch
    apc::DBuf mp[48];   // learned preconditioner: graph, activations, gradients (indices in mpnn.cu)
    int mp_graph_n = -1; // node count the graph in mp was built for (-1: none)
    // stencils
    apc::DBuf nbr, msz, ring, lap, lapd, D, rcond;
    // matrices (sliced ELL, 32-row slices, column-major inside a slice)
    apc::DBuf slice_w, slice_off, ell_col, ell_A, ell_B, dA, dB;
    apc::DBuf ell_A32, ell_B32;  // FP32 copies for the inner iterations of the mixed form
    apc::DBuf ell_A16, ell_B16;  // FP16 copies for the preconditioner sweeps of the mixed form
    // width-sorted copy of the FP16 sweep matrix: rows ordered by stencil width
    // inside windows of 256 rows, so 32-row slices pad little (see build_sorted_sweep)
    apc::DBuf ss_perm, ss_w, ss_o, ss_col, ss_A, ss_B;
    apc::DBuf ss_col24;                             // chunk columns of the sorted copy, 24 bits each
    apc::DBuf stencil_ovf;                          // nodes whose k-ring outgrew MAXC_FAST candidates
    bool ss_col24_ok = false;
    apc::DBuf ss_A32, ss_B32;   // FP32 values in the same layout (Arnoldi products of the mixed form)
    apc::DBuf beam_part;        // per-beam norms: partial sums, BSQ_CH per beam
    apc::DBuf tune_b, tune_x;   // autotuner: right-hand side and iterate of its timed restart cycles
    // ILU(0) comparison solve: factors of system ilu_which while it runs (-1: none)
    apc::IluDev ilu;
    int ilu_which = -1;
    apc::DBuf ilu_lrows, ilu_urows, ilu_lrp, ilu_urp, ilu_lcol, ilu_ucol, ilu_lval, ilu_uval, ilu_dinv;
    apc::DBuf ilu_loff, ilu_uoff;   // level offsets of the two sweeps, for the one-block runs of small levels
    bool ss_ok = false;
    int64_t ss_entries = 0;
    // solver
    apc::DBuf V, w0, w1, u, b, partial, gstate, rho_m, rho, phi, nodefield, tmp;
    apc::DBuf nodefield32;   // mixed form: compact node records of the particle pass
    apc::DBuf V32, w32a, w32b, r32, e32, gstate2;   // mixed form: FP32 Krylov scratch, outer state
    apc::DBuf pz0, pz1, pt;                         // polynomial preconditioner sweeps
    apc::DBuf zbasis;                               // preconditioned basis Z (flexible cycle end)
    apc::DBuf ell_rd;                               // reciprocal diagonals while the ELL is filled
    // device staging for apcloud_field_host
    apc::DBuf hx, hy, hz, hq, hphi, hex, hey, hez;
    // error word, small host-visible values
    apc::DBuf derr, dsmall;
    unsigned *h_pinned = nullptr;  // pinned staging for small reads
};

namespace apc {

// ---- context helpers (api.cu) ----
apcloud_status fail(apcloud_ctx *c, apcloud_status st, const char *fmt, ...);
apcloud_status cuda_check(apcloud_ctx *c, cudaError_t e, const char *what);
void *raw_alloc(apcloud_ctx *c, size_t bytes);
void count_captured(apcloud_ctx *c);
// inside a capture: the launches up to end_step form the body of an IF node on
// cond[j]; the condition of step j + 1 (0 when there is none) for the step's
// last kernel
void begin_step(apcloud_ctx *c, int j);
void end_step(apcloud_ctx *c);
cudaGraphConditionalHandle next_step_cond(const apcloud_ctx *c, int j);
// kernels of the first je steps' bodies of the last replayed graph, added to
// the launch count once the host knows je
void count_replayed_steps(apcloud_ctx *c, int je);
void raw_free(apcloud_ctx *c, void *p);
bool ensure_bytes(apcloud_ctx *c, DBuf &b, size_t bytes, bool keep = false);
template <class T>
inline T *ensure(apcloud_ctx *c, DBuf &b, size_t count, bool keep = false) {
    if (!ensure_bytes(c, b, count * sizeof(T) + 16, keep)) return nullptr;
    return static_cast<T *>(b.p);
}
template <class T>
inline T *ptr(DBuf &b) { return static_cast<T *>(b.p); }

// event timers around launches of one kind
void timer_begin(apcloud_ctx *c, int kind);
void timer_close(apcloud_ctx *c);
// add algorithmic traffic of launches of `kind` (only while that kind is timed)
inline void account(apcloud_ctx *c, int kind, double bytes, double flops) {
    if (c->timer.mask >> kind & 1u) { c->timer.bytes[kind] += bytes; c->timer.flops[kind] += flops; }
}

// read `bytes` from device to host on the context stream and synchronise
apcloud_status read_back(apcloud_ctx *c, void *host, const void *dev, size_t bytes);
apcloud_status check_device_errors(apcloud_ctx *c);

// ---- primitives (prims.cu) ----
// exclusive scan of n uint32 values; writes the total to *d_total if non-null
apcloud_status scan_u32(apcloud_ctx *c, const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total);
// stable LSD radix sort of (key, value) pairs on key bits [0, nbits); returns
// 0/1 = which of the two buffers holds the result
apcloud_status radix_sort(apcloud_ctx *c, uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n,
                          int nbits, int *which);

// ---- stages ----
apcloud_status build_octree(apcloud_ctx *c, const double *x, const double *y, const double *z, int64_t n,
                            const int64_t *h_offsets, int nbeams);
apcloud_status node_beams(apcloud_ctx *c, int32_t *out);
apcloud_status refresh_lowp(apcloud_ctx *c);          // FP32/FP16 matrix copies from the FP64 values
apcloud_status build_sorted_sweep(apcloud_ctx *c);    // width-sorted FP16 sweep matrix from the ELL
double *poisson_rhs(apcloud_ctx *c, const double *g);  // b of the Poisson system into c->b
apcloud_status tune_spmv(apcloud_ctx *c, double *ms_out);      // ms per sweep at 64/128/256/512 threads
int64_t sweep_keep_bytes(const apcloud_ctx *c);                 // sweep matrix bytes read with ordinary loads
apcloud_status tune_stencils(apcloud_ctx *c, double *ms_out);  // ms per build at 2/4/8 warps
// CUDA graphs of restart cycles
GraphEntry *find_graph(apcloud_ctx *c, const GraphKey &key);
GraphEntry *begin_capture(apcloud_ctx *c, const GraphKey &key);
GraphEntry *end_capture(apcloud_ctx *c, GraphEntry *g, apcloud_status st);
apcloud_status launch_graph(apcloud_ctx *c, GraphEntry *g);
void free_graphs(apcloud_ctx *c);
apcloud_status build_stencils(apcloud_ctx *c);
apcloud_status deposit(apcloud_ctx *c, const double *q, double q_uniform);
apcloud_status gmres_solve(apcloud_ctx *c, int which, const double *b, double *x_inout_scaled, double rtol,
                           int max_iter, apcloud_solve_info *info);
bool ilu0_factor(int64_t n, const int64_t *rp, const int32_t *cj, const int64_t *dg, double *a);
double *ilu_apply(apcloud_ctx *c, const IluDev &I, const double *v, double *z, const GmresState *st);
apcloud_status spmv(apcloud_ctx *c, int which, const double *x, double *y, double scale, double *copy_out);
apcloud_status gather_field(apcloud_ctx *c, double *phi_p, double *ex, double *ey, double *ez);
apcloud_status interpolate_phi(apcloud_ctx *c, const double *x, const double *y, const double *z, int64_t n,
                               double *phi);
apcloud_status push(apcloud_ctx *c, double *x, double *y, double *z, double *vx, double *vy, double *vz, int64_t n,
                    const double *ex, const double *ey, const double *ez, double qm_dt, double dt);
apcloud_status field_energy(apcloud_ctx *c, double *h_out);

// ---- device helpers ----
__host__ __device__ inline uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}
__host__ __device__ inline uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}
// Morton key with x most significant in every 3-bit group
__host__ __device__ inline uint64_t morton(uint32_t ix, uint32_t iy, uint32_t iz) {
    return (spread3(ix) << 2) | (spread3(iy) << 1) | spread3(iz);
}
__host__ __device__ inline void unmorton(uint64_t k, uint32_t &ix, uint32_t &iy, uint32_t &iz) {
    ix = compact3(k >> 2);
    iy = compact3(k >> 1);
    iz = compact3(k);
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

#define APC_LAUNCH(c, kind, grid, block, smem, kern, ...)                       \
    do {                                                                        \
        if ((grid) > 0) {                                                       \
            ::apc::timer_begin(c, kind);                                        \
            kern<<<(grid), (block), (smem), (c)->s>>>(__VA_ARGS__);             \
            if ((c)->capturing) ::apc::count_captured(c);                        \
            else (c)->launches++;                                               \
        }                                                                       \
    } while (0)

// The same launch as programmatic dependent launch: the kernel's blocks may
// start once every block of the kernel before it in the stream has executed
// griddepcontrol.launch_dependents (or exited); the kernel must execute
// griddepcontrol.wait, which returns once that kernel has completed and its
// writes are visible, before it reads anything that kernel writes or writes
// anything that kernel reads.  Captured into graphs as programmatic edges.
#define APC_LAUNCH_PDL(c, kind, grid, block, smem, kern, ...)                   \
    do {                                                                        \
        if ((grid) > 0) {                                                       \
            ::apc::timer_begin(c, kind);                                        \
            cudaLaunchAttribute _at[1];                                         \
            _at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;     \
            _at[0].val.programmaticStreamSerializationAllowed = 1;              \
            cudaLaunchConfig_t _cfg = {};                                       \
            _cfg.gridDim = dim3((unsigned)(grid));                              \
            _cfg.blockDim = dim3((unsigned)(block));                            \
            _cfg.dynamicSmemBytes = (smem);                                     \
            _cfg.stream = (c)->s;                                               \
            _cfg.attrs = _at;                                                   \
            _cfg.numAttrs = 1;                                                  \
            (void)cudaLaunchKernelEx(&_cfg, kern, __VA_ARGS__);                 \
            if ((c)->capturing) ::apc::count_captured(c);                        \
            else (c)->launches++;                                               \
        }                                                                       \
    } while (0)

#define APC_TRY(expr)                          \
    do {                                       \
        apcloud_status _st = (expr);           \
        if (_st < 0) return _st;               \
    } while (0)

#define APC_CUDA(c, expr) APC_TRY(::apc::cuda_check(c, (expr), #expr))

}  // namespace apc

/*
 * apcloud_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of the AP-Cloud electrostatic
 * solve (Wang, Samulyak, Jiao, Yu, "AP-Cloud: Adaptive Particle-in-Cloud
 * method", arXiv 1603.04039).  It exists to check the CUDA library; only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Steps, in the paper's order:
 *   Section 4        Morton keys, key sort, 2^D-tree cells (first particle, count)
 *   Section 4.1      error-balance criterion h < c N'^(-1/(2k-2)) with k = 2
 *   Section 4.3      queue-based node selection with the "open" operation,
 *                    face-neighbour definition, 2:1 balance pass (Section 4.2),
 *                    boundary nodes, k-ring neighbour search
 *   Section 3.1      quadrant (octant) criterion, generalized Vandermonde V,
 *                    scaled V0, normalized Gaussian weight, weighted least
 *                    squares by Householder QR, pseudo-inverse
 *   Section 3.2      step 1: density system B rho~ = rho_M (Eq. density_apcloud,
 *                    Eq. pseudoinverse, Eq. density_linear_system);
 *                    step 2: GFD Poisson system (Eq. Poisson, c = poisson_c);
 *                    step 3: GFD gradient and Taylor interpolation to particles
 *   (unnamed solver) restarted GMRES with right Jacobi preconditioning, MGS.
 *
 * Readings where the paper is silent or garbled (each also listed in the
 * design notes):
 *   R1  criterion compared squared: a cell at level l < max_depth opens iff
 *       N' > 0 and N' * h_l^2 >= c^2, h_l the cell edge (worked example, Sec. 4.3).
 *   R2  2:1 balance is across faces only (face-neighbour definition, Sec. 4.3).
 *   R3  boundary nodes: one at the centre of every leaf face lying on the
 *       domain boundary; it is joined to its owner leaf in the ring graph.
 *   R4  octant of a neighbour: the signs of (dx, dy, dz), zero counted as +;
 *       two nearest per octant, then the nearest remaining up to m_target,
 *       then every remaining candidate at the same distance as the last one
 *       filled (at most 32 in all), so that the cut never splits a shell of
 *       equidistant nodes and symmetric stencils stay symmetric (Sec. 3.3
 *       ties second-order accuracy to well-balanced stencils); order and
 *       ties by (exact integer squared distance, node index).
 *   R5  V0 row [xi_x, xi_y, xi_z, xi_x^2/2, xi_x xi_y, xi_x xi_z, xi_y^2/2,
 *       xi_y xi_z, xi_z^2/2] (the 2-D example of Sec. 3.1 extended to 3-D);
 *       rows are multiplied by W (not sqrt W).
 *   R6  density-system moments for the cell-indicator kernel with the Taylor
 *       1/l! factor: row j is rho~_j + (h_j^2/24) sum_i l_ji (rho~_i - rho~_j).
 *   R7  density-system boundary rows: rho~_b = rho_M of the owner leaf.
 *   R8  a ring is searched only once it has m_target candidates (or it is the
 *       last ring and has at least 9); a weighted Vandermonde with
 *       min |R_ii| < 1e-6 max |R_ii| is rank deficient and not used.
 *   R9  a stencil whose Laplacian diagonal (minus the sum of its weights) is
 *       not negative is not used either: that row would have the wrong sign
 *       and make the discrete Laplacian indefinite.  A node that gets an
 *       unusable stencil retries with target sizes m_target + 2, + 4, ... (at
 *       most 32) in the same ring, then widens the ring; after ring_max the
 *       build fails.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_KEY_DEPTH 21 /* 3 x 21 = 63 bits of a 64-bit Morton key (Sec. 4.3) */
#define OR_NCOL 9       /* unknowns of the second-order GFD system in 3-D */
#define OR_RANK_TOL 1e-6
#define OR_MMAX 32      /* largest stencil */

enum { OR_OK = 0, OR_E_INVALID = -1, OR_E_DOMAIN = -2, OR_E_STENCIL = -3, OR_E_NOMEM = -5 };

typedef struct {
    uint64_t key;   /* Morton index of the cell at its own level */
    int level;
    int first;      /* first particle in the key-sorted array (Section 4) */
    int count;      /* N', particles in the cell */
    int child;      /* index of the first of 8 children, -1 while not opened */
} or_cell;

typedef struct or_ctx {
    double lo[3], hi[3];
    int max_depth;
    double c_refine;
    int m_target, ring_max;
    double weight_c, poisson_c;

    /* particles */
    int64_t N;
    double *px, *py, *pz;
    uint64_t *skey;     /* keys in sorted order */
    int32_t *order;     /* sorted position -> caller index */

    /* tree: every cell ever created is in the queue Q, in creation order */
    or_cell *cell;
    int ncell, capcell;

    /* nodes: interior (leaves, Morton order) then boundary */
    int n_int, n_bnd;
    int32_t *leaf_cell;     /* interior node -> cell */
    int32_t *icoord;        /* 3 per node, units of (hi-lo) 2^-22 */
    int8_t *nlevel, *nkind; /* kind: 0 interior, 1 boundary */
    int32_t *bowner;        /* boundary node -> owner interior node */
    int8_t *bface;
    int32_t *bidx;          /* interior node * 6 + face -> boundary node or -1 */
    int32_t *adj_off, *adj; /* ring graph, CSR over all nodes */

    /* stencils */
    int32_t *nbr;   /* n_int x OR_MMAX, -1 padded */
    int32_t *msz;   /* stencil size */
    int32_t *ring;  /* ring the stencil was taken from */
    double *D;      /* n_int x 9 x OR_MMAX derivative operator */
    double *lap;    /* n_int x OR_MMAX Laplacian weights */
    double *lapd;   /* n_int diagonal */

    char err[256];
} or_ctx;

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

static double unit_len(const or_ctx *c) { return ldexp(c->hi[0] - c->lo[0], -22); }

/* Section 4: interleave 21 bits per coordinate, x most significant. */
static uint64_t interleave(uint32_t ix, uint32_t iy, uint32_t iz, int nbits) {
    uint64_t k = 0;
    for (int b = nbits - 1; b >= 0; --b) {
        k = (k << 3) | ((uint64_t)((ix >> b) & 1u) << 2) | ((uint64_t)((iy >> b) & 1u) << 1) |
            (uint64_t)((iz >> b) & 1u);
    }
    return k;
}

static void deinterleave(uint64_t k, int nbits, uint32_t *ix, uint32_t *iy, uint32_t *iz) {
    uint32_t x = 0, y = 0, z = 0;
    for (int b = 0; b < nbits; ++b) {
        z |= (uint32_t)((k >> (3 * b)) & 1u) << b;
        y |= (uint32_t)((k >> (3 * b + 1)) & 1u) << b;
        x |= (uint32_t)((k >> (3 * b + 2)) & 1u) << b;
    }
    *ix = x; *iy = y; *iz = z;
}

/* Integer cell coordinate along one axis at depth 21: floor((p-lo) 2^21/(hi-lo)),
 * a point on a face goes to the upper cell and p = hi is clamped into the last. */
static uint32_t cell_coord(double p, double lo, double hi) {
    double s = ldexp(1.0, OR_KEY_DEPTH) / (hi - lo);
    double t = (p - lo) * s;
    double f = floor(t);
    if (f < 0.0) f = 0.0;
    if (f > (double)((1u << OR_KEY_DEPTH) - 1u)) f = (double)((1u << OR_KEY_DEPTH) - 1u);
    return (uint32_t)f;
}

/* ------------------------------------------------------------------------ */
/* context                                                                   */
/* ------------------------------------------------------------------------ */

or_ctx *or_create(const double *lo, const double *hi, int max_depth, double c_refine, int m_target,
                  int ring_max, double weight_c, double poisson_c) {
    or_ctx *c = (or_ctx *)xcalloc(1, sizeof(or_ctx));
    for (int d = 0; d < 3; ++d) { c->lo[d] = lo[d]; c->hi[d] = hi[d]; }
    c->max_depth = max_depth;
    c->c_refine = c_refine;
    c->m_target = m_target;
    c->ring_max = ring_max;
    c->weight_c = weight_c;
    c->poisson_c = poisson_c;
    return c;
}

static void free_tree(or_ctx *c) {
    free(c->px); free(c->py); free(c->pz); free(c->skey); free(c->order); free(c->cell);
    free(c->leaf_cell); free(c->icoord); free(c->nlevel); free(c->nkind); free(c->bowner);
    free(c->bface); free(c->bidx); free(c->adj_off); free(c->adj);
    free(c->nbr); free(c->msz); free(c->ring); free(c->D); free(c->lap); free(c->lapd);
    c->px = c->py = c->pz = NULL; c->skey = NULL; c->order = NULL; c->cell = NULL;
    c->leaf_cell = c->icoord = NULL; c->nlevel = c->nkind = NULL; c->bowner = NULL;
    c->bface = NULL; c->bidx = NULL; c->adj_off = c->adj = NULL;
    c->nbr = c->msz = c->ring = NULL; c->D = c->lap = c->lapd = NULL;
    c->ncell = c->capcell = 0; c->n_int = c->n_bnd = 0;
}

void or_destroy(or_ctx *c) {
    if (!c) return;
    free_tree(c);
    free(c);
}

const char *or_last_error(const or_ctx *c) { return c->err; }

/* ------------------------------------------------------------------------ */
/* Section 4: key sort and 2^D-tree cells                                   */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t key; int32_t idx; } keyidx;

static int cmp_keyidx(const void *a, const void *b) {
    const keyidx *x = (const keyidx *)a, *y = (const keyidx *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static int lower_bound_key(const uint64_t *k, int n, uint64_t v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        if (k[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Particle range of a cell: all depth-21 keys with the cell's key as prefix. */
static void cell_range(const or_ctx *c, uint64_t key, int level, int *first, int *count) {
    int sh = 3 * (OR_KEY_DEPTH - level);
    uint64_t a = key << sh;
    uint64_t b = (level == 0) ? UINT64_MAX : ((key + 1) << sh);
    int f = lower_bound_key(c->skey, (int)c->N, a);
    int e = (level == 0) ? (int)c->N : lower_bound_key(c->skey, (int)c->N, b);
    *first = f;
    *count = e - f;
}

static int new_cell(or_ctx *c, uint64_t key, int level) {
    if (c->ncell == c->capcell) {
        int nc = c->capcell ? 2 * c->capcell : 1024;
        or_cell *p = (or_cell *)realloc(c->cell, (size_t)nc * sizeof(or_cell));
        if (!p) return -1;
        c->cell = p;
        c->capcell = nc;
    }
    or_cell *y = &c->cell[c->ncell];
    y->key = key;
    y->level = level;
    y->child = -1;
    cell_range(c, key, level, &y->first, &y->count);
    return c->ncell++;
}

/* The "open" operation of Section 4.3: the cell stops being a node candidate
 * and its 8 children join the end of the queue as node candidates.  Neighbour
 * lists are not stored; or_face_neighbour() evaluates the definition. */
static int open_cell(or_ctx *c, int y) {
    uint64_t k = c->cell[y].key;
    int l = c->cell[y].level;
    int first = -1;
    for (int o = 0; o < 8; ++o) {
        int id = new_cell(c, (k << 3) | (uint64_t)o, l + 1);
        if (id < 0) return -1;
        if (o == 0) first = id;
    }
    c->cell[y].child = first;
    return 0;
}

/* Error-balance criterion, Eq. errorbalance_implementation with k = 2:
 * the cell stays a node iff h < c N'^(-1/2); compared squared (reading R1). */
int or_criterion_opens(int64_t nprime, int level, int max_depth, double lo, double hi, double c_refine) {
    if (level >= max_depth || nprime <= 0) return 0;
    double h = ldexp(hi - lo, -level);
    double h2 = h * h;
    double lhs = (double)nprime * h2;
    double rhs = c_refine * c_refine;
    return lhs >= rhs;
}

/* Face neighbour of cell y (Section 4.3): the deepest cell in the tree whose
 * level is at most level(y) and that meets y across face f (0..5 = -x,+x,-y,
 * +y,-z,+z).  Returns -1 when the face lies on the domain boundary. */
static int face_neighbour(const or_ctx *c, int y, int f) {
    int l = c->cell[y].level;
    uint32_t x[3];
    deinterleave(c->cell[y].key, l, &x[0], &x[1], &x[2]);
    int d = f / 2;
    long t = (long)x[d] + ((f & 1) ? 1 : -1);
    if (t < 0 || t >= (1L << l)) return -1;
    x[d] = (uint32_t)t;
    int z = 0;
    while (c->cell[z].child >= 0 && c->cell[z].level < l) {
        int lz = c->cell[z].level + 1;
        int sh = l - lz;
        int o = (int)((((x[0] >> sh) & 1u) << 2) | (((x[1] >> sh) & 1u) << 1) | ((x[2] >> sh) & 1u));
        z = c->cell[z].child + o;
    }
    return z;
}

static int cmp_u64_pair(const void *a, const void *b) {
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

int or_build(or_ctx *c, const double *x, const double *y, const double *z, int64_t N) {
    free_tree(c);
    c->err[0] = 0;
    if (N < 0 || N > 2000000000LL || c->max_depth < 0 || c->max_depth > OR_KEY_DEPTH) {
        snprintf(c->err, sizeof c->err, "invalid size or depth");
        return OR_E_INVALID;
    }
    double ext = c->hi[0] - c->lo[0];
    if (!(ext > 0) || c->hi[1] - c->lo[1] != ext || c->hi[2] - c->lo[2] != ext) {
        snprintf(c->err, sizeof c->err, "domain must be a cube");
        return OR_E_INVALID;
    }
    c->N = N;
    c->px = (double *)xcalloc((size_t)N, sizeof(double));
    c->py = (double *)xcalloc((size_t)N, sizeof(double));
    c->pz = (double *)xcalloc((size_t)N, sizeof(double));
    keyidx *ki = (keyidx *)xcalloc((size_t)N, sizeof(keyidx));
    c->skey = (uint64_t *)xcalloc((size_t)N, sizeof(uint64_t));
    c->order = (int32_t *)xcalloc((size_t)N, sizeof(int32_t));
    if (!c->px || !c->py || !c->pz || !ki || !c->skey || !c->order) { free(ki); return OR_E_NOMEM; }
    memcpy(c->px, x, (size_t)N * sizeof(double));
    memcpy(c->py, y, (size_t)N * sizeof(double));
    memcpy(c->pz, z, (size_t)N * sizeof(double));

    /* Section 4: Morton keys, then sort so that every cell is contiguous. */
    for (int64_t i = 0; i < N; ++i) {
        double p[3] = {x[i], y[i], z[i]};
        for (int d = 0; d < 3; ++d) {
            if (!(p[d] >= c->lo[d] && p[d] <= c->hi[d])) {
                free(ki);
                snprintf(c->err, sizeof c->err, "particle %lld outside the domain", (long long)i);
                return OR_E_DOMAIN;
            }
        }
        ki[i].key = interleave(cell_coord(p[0], c->lo[0], c->hi[0]), cell_coord(p[1], c->lo[1], c->hi[1]),
                               cell_coord(p[2], c->lo[2], c->hi[2]), OR_KEY_DEPTH);
        ki[i].idx = (int32_t)i;
    }
    qsort(ki, (size_t)N, sizeof(keyidx), cmp_keyidx);
    for (int64_t i = 0; i < N; ++i) { c->skey[i] = ki[i].key; c->order[i] = ki[i].idx; }
    free(ki);

    /* Section 4.3, node selection.  Step 1: the queue holds the root. */
    if (new_cell(c, 0, 0) < 0) return OR_E_NOMEM;
    /* Step 2: traverse the queue (it grows as cells open), open every cell
     * that fails the error-balance criterion. */
    for (int q = 0; q < c->ncell; ++q) {
        or_cell *cy = &c->cell[q];
        if (or_criterion_opens(cy->count, cy->level, c->max_depth, c->lo[0], c->hi[0], c->c_refine)) {
            if (open_cell(c, q) < 0) return OR_E_NOMEM;
        }
    }
    int lmax = 0;
    for (int q = 0; q < c->ncell; ++q) if (c->cell[q].level > lmax) lmax = c->cell[q].level;
    /* Steps 3-4: from the deepest level up, every leaf at level l opens each
     * face neighbour that is more than one level coarser (Section 4.2). */
    for (int l = lmax; l > 0; --l) {
        int nq = c->ncell;
        for (int q = 0; q < nq; ++q) {
            if (c->cell[q].child >= 0 || c->cell[q].level != l) continue;
            for (int f = 0; f < 6; ++f) {
                for (;;) {
                    int nb = face_neighbour(c, q, f);
                    if (nb < 0 || c->cell[nb].level >= l - 1) break;
                    if (open_cell(c, nb) < 0) return OR_E_NOMEM;
                }
            }
        }
    }

    /* Step 4 output: the node candidates are the leaves; order them by the
     * depth-21 key of their lowest corner (Morton order of the leaves). */
    int nleaf = 0;
    for (int q = 0; q < c->ncell; ++q) if (c->cell[q].child < 0) ++nleaf;
    uint64_t *srt = (uint64_t *)xcalloc((size_t)nleaf * 2, sizeof(uint64_t));
    if (!srt) return OR_E_NOMEM;
    int t = 0;
    for (int q = 0; q < c->ncell; ++q) {
        if (c->cell[q].child >= 0) continue;
        srt[2 * t] = c->cell[q].key << (3 * (OR_KEY_DEPTH - c->cell[q].level));
        srt[2 * t + 1] = (uint64_t)q;
        ++t;
    }
    qsort(srt, (size_t)nleaf, 2 * sizeof(uint64_t), cmp_u64_pair);
    c->n_int = nleaf;
    c->leaf_cell = (int32_t *)xcalloc((size_t)nleaf, sizeof(int32_t));
    for (int j = 0; j < nleaf; ++j) c->leaf_cell[j] = (int32_t)srt[2 * j + 1];
    free(srt);

    /* Boundary nodes (reading R3): centre of every leaf face on the boundary,
     * ordered by (face, owner). */
    c->bidx = (int32_t *)xcalloc((size_t)nleaf * 6, sizeof(int32_t));
    int nb = 0;
    for (int f = 0; f < 6; ++f) {
        for (int j = 0; j < nleaf; ++j) {
            const or_cell *cy = &c->cell[c->leaf_cell[j]];
            uint32_t xx[3];
            deinterleave(cy->key, cy->level, &xx[0], &xx[1], &xx[2]);
            uint32_t edge = (f & 1) ? ((1u << cy->level) - 1u) : 0u;
            c->bidx[j * 6 + f] = (xx[f / 2] == edge) ? nb++ : -1;
        }
    }
    c->n_bnd = nb;
    int ntot = nleaf + nb;
    c->icoord = (int32_t *)xcalloc((size_t)ntot * 3, sizeof(int32_t));
    c->nlevel = (int8_t *)xcalloc((size_t)ntot, 1);
    c->nkind = (int8_t *)xcalloc((size_t)ntot, 1);
    c->bowner = (int32_t *)xcalloc((size_t)(nb ? nb : 1), sizeof(int32_t));
    c->bface = (int8_t *)xcalloc((size_t)(nb ? nb : 1), 1);
    for (int j = 0; j < nleaf; ++j) {
        const or_cell *cy = &c->cell[c->leaf_cell[j]];
        uint32_t xx[3];
        deinterleave(cy->key, cy->level, &xx[0], &xx[1], &xx[2]);
        int sh = OR_KEY_DEPTH - cy->level;
        int32_t ctr[3];
        for (int d = 0; d < 3; ++d) ctr[d] = (int32_t)((2u * xx[d] + 1u) << sh);
        for (int d = 0; d < 3; ++d) c->icoord[3 * j + d] = ctr[d];
        c->nlevel[j] = (int8_t)cy->level;
        c->nkind[j] = 0;
        for (int f = 0; f < 6; ++f) {
            int b = c->bidx[j * 6 + f];
            if (b < 0) continue;
            int g = nleaf + b;
            for (int d = 0; d < 3; ++d) c->icoord[3 * g + d] = ctr[d];
            c->icoord[3 * g + f / 2] = (f & 1) ? (1 << 22) : 0;
            c->nlevel[g] = (int8_t)cy->level;
            c->nkind[g] = 1;
            c->bowner[b] = j;
            c->bface[b] = (int8_t)f;
        }
    }

    /* Ring graph (Section 4.3): a leaf's 1-ring holds its face neighbours that
     * are nodes and, for a neighbour that is not a node, its 4 children that
     * share the face; boundary nodes hang off their owner (reading R3). */
    int32_t *cell2node = (int32_t *)xcalloc((size_t)c->ncell, sizeof(int32_t));
    for (int q = 0; q < c->ncell; ++q) cell2node[q] = -1;
    for (int j = 0; j < nleaf; ++j) cell2node[c->leaf_cell[j]] = j;
    c->adj_off = (int32_t *)xcalloc((size_t)ntot + 1, sizeof(int32_t));
    int cap = ntot * 8 + 64, na = 0;
    c->adj = (int32_t *)xcalloc((size_t)cap, sizeof(int32_t));
    for (int j = 0; j < ntot; ++j) {
        c->adj_off[j] = na;
        if (na + 32 > cap) {
            cap *= 2;
            c->adj = (int32_t *)realloc(c->adj, (size_t)cap * sizeof(int32_t));
        }
        if (j >= nleaf) { c->adj[na++] = c->bowner[j - nleaf]; continue; }
        int q = c->leaf_cell[j];
        for (int f = 0; f < 6; ++f) {
            int zc = face_neighbour(c, q, f);
            if (zc < 0) { c->adj[na++] = nleaf + c->bidx[j * 6 + f]; continue; }
            if (c->cell[zc].child < 0) { c->adj[na++] = cell2node[zc]; continue; }
            /* children of z touching y: bit of axis f/2 is 0 when z lies on
             * the + side of y, 1 when on the - side */
            int d = f / 2, want = (f & 1) ? 0 : 1;
            for (int o = 0; o < 8; ++o) {
                if (((o >> (2 - d)) & 1) != want) continue;
                int ch = c->cell[zc].child + o;
                if (c->cell[ch].child >= 0) {
                    free(cell2node);
                    snprintf(c->err, sizeof c->err, "2:1 balance violated at node %d", j);
                    return OR_E_INVALID;
                }
                c->adj[na++] = cell2node[ch];
            }
        }
    }
    c->adj_off[ntot] = na;
    free(cell2node);
    return OR_OK;
}

int64_t or_n_interior(const or_ctx *c) { return c->n_int; }
int64_t or_n_boundary(const or_ctx *c) { return c->n_bnd; }
int64_t or_n_cells(const or_ctx *c) { return c->ncell; }

void or_get_nodes(const or_ctx *c, int32_t *icoord, int8_t *level, int8_t *kind, double *xyz) {
    int nt = c->n_int + c->n_bnd;
    double u = unit_len(c);
    for (int j = 0; j < nt; ++j) {
        for (int d = 0; d < 3; ++d) {
            if (icoord) icoord[3 * j + d] = c->icoord[3 * j + d];
            if (xyz) xyz[3 * j + d] = c->lo[d] + (double)c->icoord[3 * j + d] * u;
        }
        if (level) level[j] = c->nlevel[j];
        if (kind) kind[j] = c->nkind[j];
    }
}

/* Leaf keys at their own level, particle range in sorted order. */
void or_get_leaves(const or_ctx *c, uint64_t *key, int32_t *first, int32_t *count) {
    for (int j = 0; j < c->n_int; ++j) {
        const or_cell *cy = &c->cell[c->leaf_cell[j]];
        if (key) key[j] = cy->key;
        if (first) first[j] = cy->first;
        if (count) count[j] = cy->count;
    }
}

void or_get_boundary(const or_ctx *c, int32_t *owner, int8_t *face) {
    for (int b = 0; b < c->n_bnd; ++b) { owner[b] = c->bowner[b]; face[b] = c->bface[b]; }
}

void or_get_order(const or_ctx *c, int32_t *order) { memcpy(order, c->order, (size_t)c->N * sizeof(int32_t)); }

/* Every cell of the tree: key, level, opened flag. */
void or_get_cells(const or_ctx *c, uint64_t *key, int8_t *level, int8_t *opened, int32_t *count) {
    for (int q = 0; q < c->ncell; ++q) {
        key[q] = c->cell[q].key;
        level[q] = (int8_t)c->cell[q].level;
        opened[q] = (int8_t)(c->cell[q].child >= 0);
        count[q] = c->cell[q].count;
    }
}

int64_t or_adjacency_size(const or_ctx *c) { return c->adj_off[c->n_int + c->n_bnd]; }

void or_get_adjacency(const or_ctx *c, int32_t *off, int32_t *adj) {
    int nt = c->n_int + c->n_bnd;
    memcpy(off, c->adj_off, (size_t)(nt + 1) * sizeof(int32_t));
    memcpy(adj, c->adj, (size_t)c->adj_off[nt] * sizeof(int32_t));
}

/* ------------------------------------------------------------------------ */
/* Section 3.1: weighted least squares GFD operator                          */
/* ------------------------------------------------------------------------ */

/* Householder QR of the m x 9 matrix a (row-major), Golub and Van Loan
 * Algorithm 5.2.1.  On return the upper triangle holds R, the reflector
 * vectors are kept in v (column k occupies rows k..m-1) with beta[k]. */
static void householder_qr(int m, double *a, double *v, double *beta) {
    for (int k = 0; k < OR_NCOL; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += a[i * OR_NCOL + k] * a[i * OR_NCOL + k];
        nrm = sqrt(nrm);
        double x0 = a[k * OR_NCOL + k];
        double alpha = (x0 >= 0.0) ? -nrm : nrm;
        for (int i = 0; i < m; ++i) v[i * OR_NCOL + k] = 0.0;
        for (int i = k; i < m; ++i) v[i * OR_NCOL + k] = a[i * OR_NCOL + k];
        v[k * OR_NCOL + k] = x0 - alpha;
        double vtv = 0.0;
        for (int i = k; i < m; ++i) vtv += v[i * OR_NCOL + k] * v[i * OR_NCOL + k];
        beta[k] = (vtv > 0.0) ? 2.0 / vtv : 0.0;
        for (int col = k; col < OR_NCOL; ++col) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i * OR_NCOL + k] * a[i * OR_NCOL + col];
            s *= beta[k];
            for (int i = k; i < m; ++i) a[i * OR_NCOL + col] -= s * v[i * OR_NCOL + k];
        }
    }
}

/* Weighted least-squares derivative operator of one stencil.
 *   dint   : m x 3 integer offsets y^j - y^0 in units of `unit`
 *   P      : out, 9 x m, with  [f_x f_y f_z f_xx f_xy f_xz f_yy f_yz f_zz]^T = P (f(y^j) - f(y^0))
 *   lap    : out, m Laplacian weights (rows xx + yy + zz of P); *lapd = -sum
 * Returns 0, or 1 when the weighted Vandermonde is rank deficient (reading R8).
 * Eq. gfd / regfd for V and V0 (reading R5), normalized Gaussian weight with
 * r_max the largest neighbour distance, pseudo-inverse of Eq. pseudoinverse. */
int or_wls(int m, const int64_t *dint, double unit, double weight_c, double *P, double *lap, double *lapd,
           double *rratio) {
    if (m < OR_NCOL || m > 64) return 1;
    double a[64 * OR_NCOL], v[64 * OR_NCOL], beta[OR_NCOL], w[64];
    /* h = max_{d,j} |dy_d^j| (Section 3.1) and xi = dy / h */
    int64_t hint = 0, r2max = 0;
    for (int j = 0; j < m; ++j) {
        int64_t r2 = 0;
        for (int d = 0; d < 3; ++d) {
            int64_t t = dint[3 * j + d] < 0 ? -dint[3 * j + d] : dint[3 * j + d];
            if (t > hint) hint = t;
            r2 += dint[3 * j + d] * dint[3 * j + d];
        }
        if (r2 > r2max) r2max = r2;
    }
    if (hint == 0) return 1;
    double h = (double)hint * unit;
    double ec = exp(-weight_c);
    for (int j = 0; j < m; ++j) {
        double xi[3];
        int64_t r2 = 0;
        for (int d = 0; d < 3; ++d) {
            xi[d] = (double)dint[3 * j + d] / (double)hint;
            r2 += dint[3 * j + d] * dint[3 * j + d];
        }
        double ratio = (double)r2 / (double)r2max;
        w[j] = (exp(-ratio) - ec) / (1.0 - ec);
        double row[OR_NCOL] = {xi[0], xi[1], xi[2], 0.5 * xi[0] * xi[0], xi[0] * xi[1], xi[0] * xi[2],
                               0.5 * xi[1] * xi[1], xi[1] * xi[2], 0.5 * xi[2] * xi[2]};
        for (int k = 0; k < OR_NCOL; ++k) a[j * OR_NCOL + k] = w[j] * row[k];
    }
    householder_qr(m, a, v, beta);
    double rmax = 0.0, rmin = INFINITY;
    for (int k = 0; k < OR_NCOL; ++k) {
        double r = fabs(a[k * OR_NCOL + k]);
        if (r > rmax) rmax = r;
        if (r < rmin) rmin = r;
    }
    if (rratio) *rratio = rmin / rmax;
    if (!(rmin >= OR_RANK_TOL * rmax)) return 1;
    /* column j of the pseudo-inverse applied to W: R^{-1} (Q^T e_j)[0:9] W_j */
    for (int j = 0; j < m; ++j) {
        double e[64];
        for (int i = 0; i < m; ++i) e[i] = (i == j) ? 1.0 : 0.0;
        for (int k = 0; k < OR_NCOL; ++k) {       /* Q^T = H_9 ... H_1 */
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i * OR_NCOL + k] * e[i];
            s *= beta[k];
            for (int i = k; i < m; ++i) e[i] -= s * v[i * OR_NCOL + k];
        }
        double sol[OR_NCOL];
        for (int k = OR_NCOL - 1; k >= 0; --k) {  /* back substitution with R */
            double s = e[k];
            for (int l = k + 1; l < OR_NCOL; ++l) s -= a[k * OR_NCOL + l] * sol[l];
            sol[k] = s / a[k * OR_NCOL + k];
        }
        for (int k = 0; k < OR_NCOL; ++k) {
            double sc = (k < 3) ? h : h * h;       /* undo the column scaling of V0 */
            P[k * m + j] = sol[k] * w[j] / sc;
        }
    }
    double s = 0.0;
    for (int j = 0; j < m; ++j) {
        lap[j] = P[3 * m + j] + P[6 * m + j] + P[8 * m + j];
        s += lap[j];
    }
    *lapd = -s;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 4.3 + Section 3.1: k-ring search, octant criterion, WLS stencils  */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t d2; int32_t idx; int32_t oct; } cand_t;

static int cmp_cand(const void *a, const void *b) {
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->d2 != y->d2) return (x->d2 > y->d2) - (x->d2 < y->d2);
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Section 3.1, "two nearest nodes from each quadrant", in 3-D (reading R4):
 * the stencil of one node chosen from nc ring candidates, given by their
 * integer offsets dint (nc x 3, from the node to the candidate) and node
 * indices idx.  Candidates are ranked by (squared distance, index).  The
 * octant of a candidate is the sign pattern of its offset, a zero component
 * counting as +.  Taken are: the two nearest candidates of every octant;
 * then the nearest remaining ones until mt are taken; then every remaining
 * candidate at the squared distance of the last one taken in that fill; at
 * most OR_MMAX in all.  Writes the chosen indices, in rank order, to sel
 * (room for OR_MMAX) and returns their number (-1 when out of memory). */
int or_select(int nc, const int64_t *dint, const int32_t *idx, int mt, int32_t *sel) {
    cand_t *cand = (cand_t *)xcalloc((size_t)nc, sizeof(cand_t));
    int8_t *pk = (int8_t *)xcalloc((size_t)nc, 1);
    if (!cand || !pk) { free(cand); free(pk); return -1; }
    for (int t = 0; t < nc; ++t) {
        const int64_t *d = dint + 3 * (size_t)t;
        cand[t].d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        cand[t].idx = idx[t];
        cand[t].oct = (int)((d[0] >= 0) << 2 | (d[1] >= 0) << 1 | (d[2] >= 0));
    }
    qsort(cand, (size_t)nc, sizeof(cand_t), cmp_cand);
    int taken[8] = {0}, m = 0;
    for (int t = 0; t < nc && m < OR_MMAX; ++t)
        if (taken[cand[t].oct] < 2) { taken[cand[t].oct]++; pk[t] = 1; m++; }
    int64_t cut = -1;
    for (int t = 0; t < nc && m < mt && m < OR_MMAX; ++t) if (!pk[t]) { pk[t] = 1; m++; cut = cand[t].d2; }
    for (int t = 0; t < nc && m < OR_MMAX; ++t) if (!pk[t] && cand[t].d2 == cut) { pk[t] = 1; m++; }
    int s = 0;
    for (int t = 0; t < nc && s < m; ++t) if (pk[t]) sel[s++] = cand[t].idx;
    free(cand);
    free(pk);
    return m;
}

int or_stencils(or_ctx *c) {
    int n = c->n_int, nt = c->n_int + c->n_bnd, M = c->m_target, W = OR_MMAX;
    if (M < OR_NCOL || M > OR_MMAX || c->ring_max < 2) return OR_E_INVALID;
    free(c->nbr); free(c->msz); free(c->ring); free(c->D); free(c->lap); free(c->lapd);
    c->nbr = (int32_t *)xcalloc((size_t)n * W, sizeof(int32_t));
    c->msz = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
    c->ring = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
    c->D = (double *)xcalloc((size_t)n * OR_NCOL * W, sizeof(double));
    c->lap = (double *)xcalloc((size_t)n * W, sizeof(double));
    c->lapd = (double *)xcalloc((size_t)n, sizeof(double));
    int32_t *mark = (int32_t *)xcalloc((size_t)nt, sizeof(int32_t));
    int32_t *list = (int32_t *)xcalloc((size_t)nt, sizeof(int32_t));
    int64_t *coff = (int64_t *)xcalloc((size_t)nt * 3, sizeof(int64_t));
    int32_t *cidx = (int32_t *)xcalloc((size_t)nt, sizeof(int32_t));
    if (!c->nbr || !mark || !list || !coff || !cidx) return OR_E_NOMEM;
    for (int i = 0; i < nt; ++i) mark[i] = -1;
    double unit = unit_len(c);
    int status = OR_OK;
    for (int y0 = 0; y0 < n && status == OR_OK; ++y0) {
        for (int i = 0; i < W; ++i) c->nbr[(size_t)y0 * W + i] = -1;
        int nl = 0, head = 0;
        mark[y0] = y0;
        list[nl++] = y0;
        int done = 0;
        for (int k = 1; k <= c->ring_max && !done; ++k) {
            /* (k)-ring = (k-1)-ring plus the ring-graph neighbours of its nodes */
            int tail = nl;
            for (int t = head; t < tail; ++t) {
                int u = list[t];
                for (int e = c->adj_off[u]; e < c->adj_off[u + 1]; ++e) {
                    int v = c->adj[e];
                    if (mark[v] != y0) { mark[v] = y0; list[nl++] = v; }
                }
            }
            head = tail;
            if (k < 2) continue;
            int nc = nl - 1;
            if (nc < M && k < c->ring_max) continue;
            if (nc < OR_NCOL) continue;
            for (int t = 1; t < nl; ++t) {
                int v = list[t];
                for (int d = 0; d < 3; ++d)
                    coff[3 * (size_t)(t - 1) + d] = (int64_t)c->icoord[3 * v + d] - (int64_t)c->icoord[3 * y0 + d];
                cidx[t - 1] = v;
            }
            /* target sizes m_target, m_target + 2, ... up to OR_MMAX (reading R9) */
            int last_k = (k == c->ring_max);
            for (int mt = M; mt <= OR_MMAX && !done; mt += 2) {
                int32_t ids[OR_MMAX];
                int m = or_select(nc, coff, cidx, mt, ids);
                if (m < 0) { status = OR_E_NOMEM; break; }
                int64_t dint[OR_MMAX * 3];
                for (int s = 0; s < m; ++s)
                    for (int d = 0; d < 3; ++d)
                        dint[3 * s + d] = (int64_t)c->icoord[3 * ids[s] + d] - (int64_t)c->icoord[3 * y0 + d];
                double P[OR_NCOL * OR_MMAX], lp[OR_MMAX], ld, rr;
                int bad = or_wls(m, dint, unit, c->weight_c, P, lp, &ld, &rr);
                /* R8: rank deficient, R9: Laplacian diagonal not negative */
                if (bad || !(ld < 0.0)) {
                    if (m >= nc) break;          /* no more candidates in this ring */
                    continue;
                }
                for (int i = 0; i < m; ++i) {
                    c->nbr[(size_t)y0 * W + i] = ids[i];
                    c->lap[(size_t)y0 * W + i] = lp[i];
                    for (int r = 0; r < OR_NCOL; ++r) c->D[((size_t)y0 * OR_NCOL + r) * W + i] = P[r * m + i];
                }
                c->lapd[y0] = ld;
                c->msz[y0] = m;
                c->ring[y0] = k;
                done = 1;
            }
            if (!done && last_k) {
                snprintf(c->err, sizeof c->err, "node %d: no usable stencil within ring %d", y0, c->ring_max);
                status = OR_E_STENCIL;
                break;
            }
        }
        if (!done && status == OR_OK) {
            snprintf(c->err, sizeof c->err, "node %d: fewer than 9 candidates within ring %d", y0, c->ring_max);
            status = OR_E_STENCIL;
        }
    }
    free(mark); free(list); free(coff); free(cidx);
    return status;
}

void or_get_stencils(const or_ctx *c, int32_t *nbr, int32_t *msz, int32_t *ring, double *lap, double *lapd, double *D) {
    size_t n = (size_t)c->n_int, M = OR_MMAX;
    if (nbr) memcpy(nbr, c->nbr, n * M * sizeof(int32_t));
    if (msz) memcpy(msz, c->msz, n * sizeof(int32_t));
    if (ring) memcpy(ring, c->ring, n * sizeof(int32_t));
    if (lap) memcpy(lap, c->lap, n * M * sizeof(double));
    if (lapd) memcpy(lapd, c->lapd, n * sizeof(double));
    if (D) memcpy(D, c->D, n * OR_NCOL * M * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* Section 3.2: the two linear systems                                       */
/* ------------------------------------------------------------------------ */

static double node_h(const or_ctx *c, int j) { return ldexp(c->hi[0] - c->lo[0], -(int)c->nlevel[j]); }

/* CSR of the density matrix B (which = 0) or the Poisson matrix A (which = 1).
 * Interior rows follow the stencil: A_jj = -sum l, A_ji = l_ji;
 * B_jj = 1 + (h_j^2/24) A_jj, B_ji = (h_j^2/24) l_ji (reading R6).
 * Boundary rows are identity rows.  Columns in stencil order after the diagonal. */
int64_t or_matrix_nnz(const or_ctx *c) {
    int64_t z = c->n_bnd;
    for (int j = 0; j < c->n_int; ++j) z += 1 + c->msz[j];
    return z;
}

void or_matrix(const or_ctx *c, int which, int64_t *rowptr, int32_t *col, double *val) {
    int M = OR_MMAX, t = 0;
    for (int j = 0; j < c->n_int + c->n_bnd; ++j) {
        rowptr[j] = t;
        if (j >= c->n_int) { col[t] = j; val[t] = 1.0; ++t; continue; }
        double s = 1.0;
        if (which == 0) { double h = node_h(c, j); s = h * h / 24.0; }
        col[t] = j;
        val[t] = (which == 0) ? 1.0 + s * c->lapd[j] : c->lapd[j];
        ++t;
        for (int i = 0; i < c->msz[j]; ++i) {
            col[t] = c->nbr[(size_t)j * M + i];
            val[t] = s * c->lap[(size_t)j * M + i];
            ++t;
        }
    }
    rowptr[c->n_int + c->n_bnd] = t;
}

/* Step 1 right-hand side, Eq. density_apcloud with Phi the indicator of the
 * node's own cell (Section 5): rho_M = (sum of charges in the cell) / h^3.
 * q == NULL means every particle carries q_uniform.  Boundary entries take the
 * owner's value (reading R7).  Also returns the total deposited charge. */
double or_density_rhs(const or_ctx *c, const double *q, double q_uniform, double *rhs, double *Qcell) {
    double total = 0.0;
    for (int j = 0; j < c->n_int; ++j) {
        const or_cell *cy = &c->cell[c->leaf_cell[j]];
        double Q = 0.0;
        if (q) { for (int i = cy->first; i < cy->first + cy->count; ++i) Q += q[c->order[i]]; }
        else Q = (double)cy->count * q_uniform;
        double h = node_h(c, j);
        rhs[j] = Q / (h * h * h);
        if (Qcell) Qcell[j] = Q;
        total += Q;
    }
    for (int b = 0; b < c->n_bnd; ++b) rhs[c->n_int + b] = rhs[c->bowner[b]];
    return total;
}

static void csr_mv(int n, const int64_t *rp, const int32_t *col, const double *val, const double *x, double *y) {
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += val[e] * x[col[e]];
        y[i] = s;
    }
}

static double nrm2(int n, const double *x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += x[i] * x[i];
    return sqrt(s);
}

/* Restarted GMRES(restart), right preconditioned with M = diag(A), modified
 * Gram-Schmidt Arnoldi and Givens rotations (Saad, Iterative Methods for
 * Sparse Linear Systems, 2nd ed., Algorithms 6.9 and 9.5).  Stops when the
 * recomputed ||b - A x|| / ||b|| <= rtol.  Returns 0, or 1 when max_iter is
 * reached first. */
int or_gmres(int n, const int64_t *rp, const int32_t *col, const double *val, const double *b, double *x,
             double rtol, int max_iter, int restart, int *iters_out, double *relres_out) {
    int mr = restart;
    double *dinv = (double *)xcalloc((size_t)n, sizeof(double));
    double *V = (double *)xcalloc((size_t)n * (mr + 1), sizeof(double));
    double *Hm = (double *)xcalloc((size_t)(mr + 1) * mr, sizeof(double));
    double *cs = (double *)xcalloc((size_t)mr, sizeof(double));
    double *sn = (double *)xcalloc((size_t)mr, sizeof(double));
    double *g = (double *)xcalloc((size_t)mr + 1, sizeof(double));
    double *yv = (double *)xcalloc((size_t)mr, sizeof(double));
    double *r = (double *)xcalloc((size_t)n, sizeof(double));
    double *zt = (double *)xcalloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) if (col[e] == i) d = val[e];
        dinv[i] = (d != 0.0) ? 1.0 / d : 1.0;
    }
    double bn = nrm2(n, b);
    int it = 0, status = 1;
    double rel = 0.0;
    if (bn == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        status = 0;
        goto done;
    }
    for (;;) {
        csr_mv(n, rp, col, val, x, r);
        for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double beta = nrm2(n, r);
        rel = beta / bn;
        if (rel <= rtol) { status = 0; break; }
        if (it >= max_iter) break;
        for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
        for (int i = 0; i <= mr; ++i) g[i] = 0.0;
        g[0] = beta;
        int j;
        for (j = 0; j < mr && it < max_iter; ++j) {
            ++it;
            for (int i = 0; i < n; ++i) zt[i] = dinv[i] * V[(size_t)j * n + i];
            double *w = V + (size_t)(j + 1) * n;
            csr_mv(n, rp, col, val, zt, w);
            for (int i = 0; i <= j; ++i) {                   /* MGS */
                double h = 0.0;
                const double *vi = V + (size_t)i * n;
                for (int t = 0; t < n; ++t) h += vi[t] * w[t];
                Hm[i * mr + j] = h;
                for (int t = 0; t < n; ++t) w[t] -= h * vi[t];
            }
            double hn = nrm2(n, w);
            Hm[(j + 1) * mr + j] = hn;
            if (hn != 0.0) for (int t = 0; t < n; ++t) w[t] /= hn;
            for (int i = 0; i < j; ++i) {                    /* apply old rotations */
                double a = Hm[i * mr + j], bb = Hm[(i + 1) * mr + j];
                Hm[i * mr + j] = cs[i] * a + sn[i] * bb;
                Hm[(i + 1) * mr + j] = -sn[i] * a + cs[i] * bb;
            }
            double a = Hm[j * mr + j], bb = Hm[(j + 1) * mr + j];
            double den = sqrt(a * a + bb * bb);
            cs[j] = (den != 0.0) ? a / den : 1.0;
            sn[j] = (den != 0.0) ? bb / den : 0.0;
            Hm[j * mr + j] = den;
            Hm[(j + 1) * mr + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (fabs(g[j + 1]) / bn <= rtol || hn == 0.0) { ++j; break; }
        }
        for (int k = j - 1; k >= 0; --k) {                   /* y = H^-1 g */
            double s = g[k];
            for (int l = k + 1; l < j; ++l) s -= Hm[k * mr + l] * yv[l];
            yv[k] = s / Hm[k * mr + k];
        }
        for (int i = 0; i < n; ++i) {                        /* x += M^-1 V y */
            double s = 0.0;
            for (int k = 0; k < j; ++k) s += V[(size_t)k * n + i] * yv[k];
            x[i] += dinv[i] * s;
        }
    }
done:
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = rel;
    free(dinv); free(V); free(Hm); free(cs); free(sn); free(g); free(yv); free(r); free(zt);
    return status;
}

static int solve_system(const or_ctx *c, int which, const double *rhs, double *x, double rtol, int max_iter,
                        int restart, int *iters, double *relres) {
    int nt = c->n_int + c->n_bnd;
    int64_t nnz = or_matrix_nnz(c);
    int64_t *rp = (int64_t *)xcalloc((size_t)nt + 1, sizeof(int64_t));
    int32_t *col = (int32_t *)xcalloc((size_t)nnz, sizeof(int32_t));
    double *val = (double *)xcalloc((size_t)nnz, sizeof(double));
    or_matrix(c, which, rp, col, val);
    int s = or_gmres(nt, rp, col, val, rhs, x, rtol, max_iter, restart, iters, relres);
    free(rp); free(col); free(val);
    return s;
}

/* Step 1: B rho~ = rhs (Eq. density_linear_system). x holds the initial guess. */
int or_solve_density(const or_ctx *c, const double *rhs, double *rho, double rtol, int max_iter, int restart,
                     int *iters, double *relres) {
    return solve_system(c, 0, rhs, rho, rtol, max_iter, restart, iters, relres);
}

/* Step 2: A phi = poisson_c rho~ on interior rows, phi_b = g_b on boundary
 * rows (Eq. Poisson with Dirichlet data).  g == NULL means g = 0. */
int or_solve_poisson(const or_ctx *c, const double *rho, const double *gb, double *phi, double rtol, int max_iter,
                     int restart, int *iters, double *relres) {
    int nt = c->n_int + c->n_bnd;
    double *rhs = (double *)xcalloc((size_t)nt, sizeof(double));
    for (int j = 0; j < c->n_int; ++j) rhs[j] = c->poisson_c * rho[j];
    for (int b = 0; b < c->n_bnd; ++b) rhs[c->n_int + b] = gb ? gb[b] : 0.0;
    int s = solve_system(c, 1, rhs, phi, rtol, max_iter, restart, iters, relres);
    free(rhs);
    return s;
}

void or_poisson_rhs(const or_ctx *c, const double *rho, const double *gb, double *rhs) {
    for (int j = 0; j < c->n_int; ++j) rhs[j] = c->poisson_c * rho[j];
    for (int b = 0; b < c->n_bnd; ++b) rhs[c->n_int + b] = gb ? gb[b] : 0.0;
}

/* Step 3: GFD derivatives at every interior node, dphi_j = P_j (phi_nbr - phi_j),
 * 9 per node in the order [x y z xx xy xz yy yz zz]. */
void or_derivatives(const or_ctx *c, const double *phi, double *dphi) {
    int M = OR_MMAX;
    for (int j = 0; j < c->n_int; ++j) {
        for (int r = 0; r < OR_NCOL; ++r) {
            double s = 0.0;
            for (int i = 0; i < c->msz[j]; ++i) {
                int v = c->nbr[(size_t)j * M + i];
                s += c->D[((size_t)j * OR_NCOL + r) * M + i] * (phi[v] - phi[j]);
            }
            dphi[(size_t)j * OR_NCOL + r] = s;
        }
    }
}

/* Step 3: second-order Taylor expansion about the centre of the particle's
 * own leaf: phi_p = phi + g.r + r^T H r / 2, E_p = g + H r, with E = grad phi
 * (Section 2).  Outputs are in the caller's particle order. */
void or_gather(const or_ctx *c, const double *phi, const double *dphi, double *phip, double *ex, double *ey,
               double *ez) {
    double u = unit_len(c);
    for (int j = 0; j < c->n_int; ++j) {
        const or_cell *cy = &c->cell[c->leaf_cell[j]];
        double y0[3];
        for (int d = 0; d < 3; ++d) y0[d] = c->lo[d] + (double)c->icoord[3 * j + d] * u;
        const double *g = dphi + (size_t)j * OR_NCOL;
        double H[3][3] = {{g[3], g[4], g[5]}, {g[4], g[6], g[7]}, {g[5], g[7], g[8]}};
        for (int i = cy->first; i < cy->first + cy->count; ++i) {
            int p = c->order[i];
            double r[3] = {c->px[p] - y0[0], c->py[p] - y0[1], c->pz[p] - y0[2]};
            double Hr[3];
            for (int a = 0; a < 3; ++a) Hr[a] = H[a][0] * r[0] + H[a][1] * r[1] + H[a][2] * r[2];
            phip[p] = phi[j] + (g[0] * r[0] + g[1] * r[1] + g[2] * r[2]) +
                      0.5 * (r[0] * Hr[0] + r[1] * Hr[1] + r[2] * Hr[2]);
            ex[p] = g[0] + Hr[0];
            ey[p] = g[1] + Hr[1];
            ez[p] = g[2] + Hr[2];
        }
    }
}

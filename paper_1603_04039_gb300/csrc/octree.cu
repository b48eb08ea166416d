// octree.cu -- Section 4: Morton keys, key sort, error-balance refinement,
// minimal 2:1 face balance, leaves, boundary nodes and face adjacency.
//
// GB300 design.  The paper builds the tree with a sequential queue and
// incremental neighbour lists (Section 4.3).  Here the node set is computed
// as a closure, one level at a time from the deepest up, with sorts and
// compactions only:
//   * every cell at level l < max_depth that holds N' > 0 particles with
//     N' h_l^2 >= c^2 opens (the criterion is monotone down the tree, so the
//     criterion tree is exactly this set);
//   * an opened cell at level l+1 forces its parent and the parents of its
//     six same-level face neighbours to open (this is the 2:1 face balance
//     rule: the children of the opened cell need face neighbours no more than
//     one level coarser);
// so O_l = Crit_l U parent(O_{l+1}) U parent(faces(O_{l+1})), a sort + unique
// per level.  The result is the unique minimal balanced refinement, the set
// the paper's deepest-level-first loop produces.
//
// Batches: several independent problems (beams) on the same cubic domain are
// one tree whose cell keys carry the beam index above the 3l Morton bits of
// level l, so one sort and one closure serve all beams and no neighbour
// relation crosses from one beam to another.
#include <cmath>

#include <climits>

#include "fpconv.cuh"
#include "internal.cuh"

namespace apc {

namespace {

constexpr int T = 256;

// beam of particle i from the batch offsets (nb + 1 entries, offs[0] = 0)
__device__ __forceinline__ uint64_t beam_of(const int64_t *offs, int nb, int64_t i) {
    int lo = 0, hi = nb;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (offs[mid] <= i) lo = mid; else hi = mid;
    }
    return (uint64_t)lo;
}

__global__ void k_keys(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                       int64_t n, double lo0, double lo1, double lo2, double hi0, double hi1, double hi2, double s,
                       int shift, const int64_t *__restrict__ offs, int nb, int L, uint64_t *__restrict__ key,
                       uint32_t *__restrict__ idx, unsigned *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double p[3] = {x[i], y[i], z[i]};
    double lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
    uint32_t cc[3];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        bad |= !f64_in_range(p[d], lo[d], hi[d]);
        // floor((p - lo) * 2^21 / (hi - lo)), no contraction, clamped into the
        // cube; the floor, the clamp and the range test on the integer pipe
        // (two FP64 operations per coordinate instead of eight)
        const double t = __dmul_rn(__dsub_rn(p[d], lo[d]), s);
        cc[d] = f64_floor_clamp_u32(t, (1u << KEY_DEPTH) - 1u) >> shift;
    }
    if (bad) atomicOr(err, ERR_DOMAIN);
    key[i] = (nb > 1 ? beam_of(offs, nb, i) << (3 * L) : 0ull) | morton(cc[0], cc[1], cc[2]);
    idx[i] = (uint32_t)i;
}

// run heads of keys >> sh
__global__ void k_run_flags(const uint64_t *__restrict__ keys, int64_t n, int sh, uint32_t *__restrict__ f) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    f[i] = (i == 0 || (keys[i] >> sh) != (keys[i - 1] >> sh)) ? 1u : 0u;
}

__global__ void k_run_scatter(const uint64_t *__restrict__ keys, int64_t n, int sh, const uint32_t *__restrict__ f,
                              const uint32_t *__restrict__ pos, const uint32_t *__restrict__ start_in,
                              uint64_t *__restrict__ okey, uint32_t *__restrict__ ostart) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !f[i]) return;
    uint32_t p = pos[i];
    okey[p] = keys[i] >> sh;
    ostart[p] = start_in ? start_in[i] : (uint32_t)i;
}

// error-balance criterion (Section 4.3, k = 2): open iff N' > 0 and N' h^2 >= c^2
__global__ void k_crit_flags(const uint32_t *__restrict__ start, int64_t u, int64_t npart, double h2, double c2,
                             uint32_t *__restrict__ f) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= u) return;
    uint32_t e = (r + 1 < u) ? start[r + 1] : (uint32_t)npart;
    uint32_t cnt = e - start[r];
    f[r] = (cnt > 0 && __dmul_rn((double)cnt, h2) >= c2) ? 1u : 0u;
}

__global__ void k_compact_u64(const uint64_t *__restrict__ in, int64_t n, const uint32_t *__restrict__ f,
                              const uint32_t *__restrict__ pos, uint64_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !f[i]) return;
    out[pos[i]] = in[i];
}

// for every opened cell at level l+1: its parent and the parents of its six
// face neighbours (the parent itself stands in for a neighbour outside the cube)
__global__ void k_balance_gen(const uint64_t *__restrict__ op, int64_t n, int lev1, uint64_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = op[i];
    uint64_t par = k >> 3;
    const uint64_t pre = (k >> (3 * lev1)) << (3 * lev1);   // beam index bits
    uint32_t c[3];
    unmorton(k ^ pre, c[0], c[1], c[2]);
    const uint32_t lim = 1u << lev1;
    out[i * 7] = par;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        uint32_t t[3] = {c[0], c[1], c[2]};
        int d = f >> 1;
        bool inside = (f & 1) ? (t[d] + 1 < lim) : (t[d] > 0);
        t[d] = (f & 1) ? t[d] + 1 : t[d] - 1;
        out[i * 7 + 1 + f] = inside ? ((pre | morton(t[0], t[1], t[2])) >> 3) : par;
    }
}

__device__ __forceinline__ bool contains_sorted(const uint64_t *a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < n && a[lo] == v;
}

// children of opened cells at level l-1 that are not opened at level l are leaves
__global__ void k_leaf_flags(const uint64_t *__restrict__ par, int64_t npar, const uint64_t *__restrict__ op,
                             int64_t nop, uint32_t *__restrict__ f) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npar * 8) return;
    uint64_t ch = (par[i >> 3] << 3) | (uint64_t)(i & 7);
    f[i] = contains_sorted(op, nop, ch) ? 0u : 1u;
}

// level-0 cells (one root per beam) that are not opened are leaves
__global__ void k_root_flags(int nb, const uint64_t *__restrict__ op, int64_t nop, uint32_t *__restrict__ f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb) f[i] = contains_sorted(op, nop, (uint64_t)i) ? 0u : 1u;
}

__global__ void k_root_emit(int nb, const uint32_t *__restrict__ f, const uint32_t *__restrict__ pos, int L,
                            uint64_t *__restrict__ anchor, uint32_t *__restrict__ level) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb || !f[i]) return;
    anchor[pos[i]] = (uint64_t)i << (3 * L);
    level[pos[i]] = 0u;
}

__global__ void k_leaf_emit(const uint64_t *__restrict__ par, int64_t npar, const uint32_t *__restrict__ f,
                            const uint32_t *__restrict__ pos, int lev, int L, uint64_t *__restrict__ anchor,
                            uint32_t *__restrict__ level) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npar * 8 || !f[i]) return;
    uint64_t ch = (par[i >> 3] << 3) | (uint64_t)(i & 7);
    uint32_t p = pos[i];
    anchor[p] = ch << (3 * (L - lev));
    level[p] = (uint32_t)lev;
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// index of the leaf whose anchor is the largest one <= v
__device__ __forceinline__ int64_t leaf_of(const uint64_t *anchor, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (anchor[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

__global__ void k_leaf_geom(const uint64_t *__restrict__ anchor, const uint32_t *__restrict__ lvl32, int64_t n,
                            int L, const uint64_t *__restrict__ skeys, int64_t npart, int8_t *__restrict__ level,
                            int32_t *__restrict__ first, int32_t *__restrict__ count, int4 *__restrict__ ic,
                            uint32_t *__restrict__ bflag, int32_t *__restrict__ beam) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int lev = (int)lvl32[j];
    uint64_t a = anchor[j];
    int64_t f0 = lower_bound_u64(skeys, npart, a);
    int64_t f1 = (j + 1 < n) ? lower_bound_u64(skeys, npart, anchor[j + 1]) : npart;
    first[j] = (int32_t)f0;
    count[j] = (int32_t)(f1 - f0);
    level[j] = (int8_t)lev;
    if (beam) beam[j] = (int32_t)(a >> (3 * L));
    uint32_t c[3];
    unmorton((a >> (3 * (L - lev))) & ((1ull << (3 * lev)) - 1ull), c[0], c[1], c[2]);
    int sh = KEY_DEPTH - lev;
    ic[j] = make_int4((int)((2u * c[0] + 1u) << sh), (int)((2u * c[1] + 1u) << sh), (int)((2u * c[2] + 1u) << sh),
                      lev);
    uint32_t edge = (1u << lev) - 1u;
#pragma unroll
    for (int f = 0; f < 6; ++f) bflag[f * n + j] = (c[f >> 1] == ((f & 1) ? edge : 0u)) ? 1u : 0u;
}

// Leaf and key-sorted position of every particle in the caller's order (read
// by the gather and the deposit, so that neither needs a search or a gather
// through the permutation): each warp owns 32 consecutive leaves and walks
// their key-sorted particle range, writing through the permutation.
__global__ void k_particle_leaf(const int32_t *__restrict__ first, const int32_t *__restrict__ count, int n_leaf,
                                const uint32_t *__restrict__ perm, int32_t *__restrict__ pleaf,
                                int32_t *__restrict__ spos) {
    const int lane = threadIdx.x & 31;
    const int64_t j0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
    if (j0 >= n_leaf) return;   // the whole warp
    const int64_t j = j0 + lane;
    const bool valid = j < n_leaf;
    const int f = valid ? first[j] : INT_MAX;
    int e = valid ? f + count[j] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    const int s = __shfl_sync(0xffffffffu, f, 0);
#pragma unroll 4
    for (int base = s; base < e; base += 32) {
        const int i = base + lane;
        const int k = group_leaf(f, i);
        if (i < e) {
            const uint32_t p = __ldcs(perm + i);
            pleaf[p] = (int32_t)(j0 + k);
            spos[p] = i;
        }
    }
}

__global__ void k_boundary(const uint32_t *__restrict__ bflag, const uint32_t *__restrict__ bpos, int64_t n,
                           int4 *__restrict__ ic, int32_t *__restrict__ owner, int8_t *__restrict__ face) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 6 * n || !bflag[t]) return;
    int f = (int)(t / n);
    int64_t j = t - (int64_t)f * n;
    uint32_t b = bpos[t];
    int4 q = ic[j];
    int v = (f & 1) ? (1 << (KEY_DEPTH + 1)) : 0;
    if ((f >> 1) == 0) q.x = v; else if ((f >> 1) == 1) q.y = v; else q.z = v;
    ic[n + b] = q;
    owner[b] = (int32_t)j;
    face[b] = (int8_t)f;
}

// Face adjacency (Section 4.3): per leaf and face, the face neighbour when it
// is a leaf, else its 4 children touching the face (leaves by 2:1 balance),
// or the boundary node of that face.
__global__ void k_adjacency(const uint64_t *__restrict__ anchor, const int8_t *__restrict__ level, int64_t n, int L,
                            const uint32_t *__restrict__ bflag, const uint32_t *__restrict__ bpos,
                            int32_t *__restrict__ adj, unsigned *err) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 6 * n) return;
    int64_t j = t / 6;
    int f = (int)(t - j * 6);
    int32_t *out = adj + j * 24 + f * 4;
    out[0] = out[1] = out[2] = out[3] = -1;
    if (bflag[(int64_t)f * n + j]) {
        out[0] = (int32_t)(n + bpos[(int64_t)f * n + j]);
        return;
    }
    int lev = level[j];
    const uint64_t pre = (anchor[j] >> (3 * L)) << (3 * L);   // beam index bits
    uint32_t c[3];
    unmorton((anchor[j] ^ pre) >> (3 * (L - lev)), c[0], c[1], c[2]);
    int d = f >> 1;
    c[d] = (f & 1) ? c[d] + 1 : c[d] - 1;
    uint64_t a = pre | (morton(c[0], c[1], c[2]) << (3 * (L - lev)));
    int64_t k = leaf_of(anchor, n, a);
    if (k < 0) { atomicOr(err, ERR_BALANCE); return; }
    if (level[k] <= lev) { out[0] = (int32_t)k; return; }
    int want = (f & 1) ? 0 : 1;
    int s = 0;
    for (int o = 0; o < 8; ++o) {
        if (((o >> (2 - d)) & 1) != want) continue;
        uint32_t cc[3] = {2u * c[0] + ((o >> 2) & 1u), 2u * c[1] + ((o >> 1) & 1u), 2u * c[2] + (o & 1u)};
        uint64_t ac = pre | (morton(cc[0], cc[1], cc[2]) << (3 * (L - lev - 1)));
        int64_t kk = leaf_of(anchor, n, ac);
        if (kk < 0 || anchor[kk] != ac || level[kk] != lev + 1) { atomicOr(err, ERR_BALANCE); return; }
        out[s++] = (int32_t)kk;
    }
}

// Node ranges of every beam: interior nodes [r[b], r[b+1]) (the leaves are
// beam-sorted) and, per face f, boundary nodes [r[(1+f)(nb+1)+b], ...+1) (the
// boundary nodes are face-major, leaf-ordered within a face).
__global__ void k_beam_ranges(const int32_t *__restrict__ beam, int64_t n, int nb, const uint32_t *__restrict__ bpos,
                              int64_t nbnd, int64_t *__restrict__ r) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nb) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (beam[mid] < b) lo = mid + 1; else hi = mid;
    }
    r[b] = lo;
    for (int f = 0; f < 6; ++f) {
        int64_t t = (int64_t)f * n + lo;
        r[(int64_t)(1 + f) * (nb + 1) + b] = n + (t < 6 * n ? (int64_t)bpos[t] : nbnd);
    }
}

// beam index of every node (boundary nodes take their owner leaf's)
__global__ void k_node_beam(const int32_t *__restrict__ leaf_beam, const int32_t *__restrict__ owner, int64_t n,
                            int64_t nt, int32_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    out[i] = i < n ? leaf_beam[i] : leaf_beam[owner[i - n]];
}

}  // namespace

apcloud_status node_beams(apcloud_ctx *c, int32_t *out) {
    APC_LAUNCH(c, K_COPY, div_up(c->n_tot, T), T, 0, k_node_beam, ptr<int32_t>(c->leaf_beam),
               ptr<int32_t>(c->bowner), (int64_t)c->n_int, (int64_t)c->n_tot, out);
    return cuda_check(c, cudaGetLastError(), "node_beams");
}

apcloud_status build_octree(apcloud_ctx *c, const double *x, const double *y, const double *z, int64_t n,
                            const int64_t *h_offsets, int nb) {
    const int L = c->P.max_depth;
    int bb = 0;  // bits of the beam index above the tree bits
    while ((1 << bb) < nb) ++bb;
    if (3 * L + bb > 63) return fail(c, APCLOUD_E_INVALID, "%d beams need %d key bits above depth %d", nb, bb, L);
    c->L = L;
    c->N = n;
    c->px = x; c->py = y; c->pz = z;
    c->nbeams = nb;
    c->beam_bits = bb;
    c->h_beam_off.assign(h_offsets, h_offsets + nb + 1);
    int64_t *doff = ensure<int64_t>(c, c->beam_off, nb + 1);
    if (!doff) return APCLOUD_E_NOMEM;
    APC_CUDA(c, cudaMemcpyAsync(doff, h_offsets, sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, c->s));
    unsigned *derr = ptr<unsigned>(c->derr);
    APC_CUDA(c, cudaMemsetAsync(derr, 0, 4 * sizeof(unsigned), c->s));
    uint32_t *small = ptr<uint32_t>(c->dsmall);

    // K1 keys at depth L, K2 sort on the 3L key bits
    int64_t nn = n > 0 ? n : 1;
    uint64_t *k0 = ensure<uint64_t>(c, c->key[0], nn), *k1 = ensure<uint64_t>(c, c->key[1], nn);
    uint32_t *v0 = ensure<uint32_t>(c, c->val[0], nn), *v1 = ensure<uint32_t>(c, c->val[1], nn);
    if (!k0 || !k1 || !v0 || !v1) return APCLOUD_E_NOMEM;
    const double ext = c->P.hi[0] - c->P.lo[0];
    const double s = ldexp(1.0, KEY_DEPTH) / ext;
    APC_LAUNCH(c, K_KEYS, div_up(n, T), T, 0, k_keys, x, y, z, n, c->P.lo[0], c->P.lo[1], c->P.lo[2], c->P.hi[0],
               c->P.hi[1], c->P.hi[2], s, KEY_DEPTH - L, (const int64_t *)doff, nb, L, k0, v0, derr);
    account(c, K_KEYS, 36.0 * n, 9.0 * n);   // 24 B positions in, 12 B key and index out
    int which = 0;
    APC_TRY(radix_sort(c, k0, v0, k1, v1, n, 3 * L + bb, &which));
    c->kbuf = which;
    uint64_t *skeys = which ? k1 : k0;

    // unique cells at level L
    uint32_t *fl = ensure<uint32_t>(c, c->tmp, nn), *pos = ensure<uint32_t>(c, c->b, nn);
    uint64_t *uk[2] = {ensure<uint64_t>(c, c->ucell[0], nn), ensure<uint64_t>(c, c->ucell[1], nn)};
    uint32_t *us[2] = {ensure<uint32_t>(c, c->ustart[0], nn), ensure<uint32_t>(c, c->ustart[1], nn)};
    if (!fl || !pos || !uk[0] || !uk[1] || !us[0] || !us[1]) return APCLOUD_E_NOMEM;
    int64_t U = 0;
    int cur = 0;
    if (n > 0) {
        APC_LAUNCH(c, K_TREE, div_up(n, T), T, 0, k_run_flags, skeys, n, 0, fl);
        APC_TRY(scan_u32(c, fl, pos, n, small));
        APC_LAUNCH(c, K_TREE, div_up(n, T), T, 0, k_run_scatter, skeys, n, 0, fl, pos, (const uint32_t *)nullptr,
                   uk[0], us[0]);
        uint32_t hu;
        APC_TRY(read_back(c, &hu, small, sizeof hu));
        U = hu;
    }

    // levels L-1 .. 0: unique cells, criterion, balance closure
    std::vector<int64_t> ocount(L + 1, 0);
    // opened cells of all levels live in `opened`, level l at open_off[l]; capacity grows with copy
    int64_t ocap = 1024;
    if (!ensure<uint64_t>(c, c->opened, ocap)) return APCLOUD_E_NOMEM;
    std::vector<int64_t> ooff(L + 1, 0);
    int64_t oused = 0;
    int64_t prev_open = 0;  // |O_{l+1}|, at ooff[l+1]
    for (int l = L - 1; l >= 0; --l) {
        // unique cells at level l from those at level l+1
        int nxt = cur ^ 1;
        int64_t Ul = 0;
        if (U > 0) {
            APC_LAUNCH(c, K_TREE, div_up(U, T), T, 0, k_run_flags, uk[cur], U, 3, fl);
            APC_TRY(scan_u32(c, fl, pos, U, small));
            APC_LAUNCH(c, K_TREE, div_up(U, T), T, 0, k_run_scatter, uk[cur], U, 3, fl, pos, us[cur], uk[nxt], us[nxt]);
        }
        // criterion flags on level-l cells
        double h = ldexp(ext, -l);
        double h2 = h * h;
        double c2 = c->P.c_refine * c->P.c_refine;
        uint32_t hv[2] = {0, 0};
        if (U > 0) {
            APC_TRY(read_back(c, hv, small, sizeof(uint32_t)));
            Ul = hv[0];
            APC_LAUNCH(c, K_TREE, div_up(Ul, T), T, 0, k_crit_flags, us[nxt], Ul, n, h2, c2, fl);
            APC_TRY(scan_u32(c, fl, pos, Ul, small + 1));
            APC_TRY(read_back(c, hv + 1, small + 1, sizeof(uint32_t)));
        }
        int64_t ncrit = hv[1];
        int64_t ncand = ncrit + 7 * prev_open;
        int64_t ccap = ncand > 0 ? ncand : 1;
        uint64_t *ca0 = ensure<uint64_t>(c, c->cand[0], ccap), *ca1 = ensure<uint64_t>(c, c->cand[1], ccap);
        uint32_t *cv0 = ensure<uint32_t>(c, c->cval[0], ccap), *cv1 = ensure<uint32_t>(c, c->cval[1], ccap);
        if (!ca0 || !ca1 || !cv0 || !cv1) return APCLOUD_E_NOMEM;
        if (ncrit > 0) APC_LAUNCH(c, K_TREE, div_up(Ul, T), T, 0, k_compact_u64, uk[nxt], Ul, fl, pos, ca0);
        if (prev_open > 0)
            APC_LAUNCH(c, K_TREE, div_up(prev_open, T), T, 0, k_balance_gen, ptr<uint64_t>(c->opened) + ooff[l + 1],
                       prev_open, l + 1, ca0 + ncrit);
        int64_t nol = 0;
        if (ncand > 0) {
            int w = 0;
            APC_TRY(radix_sort(c, ca0, cv0, ca1, cv1, ncand, 3 * l + bb, &w));
            uint64_t *sc = w ? ca1 : ca0;
            uint32_t *f2 = ensure<uint32_t>(c, c->lval, ncand), *p2 = ensure<uint32_t>(c, c->lkey, ncand);
            if (!f2 || !p2) return APCLOUD_E_NOMEM;
            APC_LAUNCH(c, K_TREE, div_up(ncand, T), T, 0, k_run_flags, sc, ncand, 0, f2);
            APC_TRY(scan_u32(c, f2, p2, ncand, small + 2));
            uint32_t hn;
            APC_TRY(read_back(c, &hn, small + 2, sizeof hn));
            nol = hn;
            if (oused + nol > ocap) {
                while (oused + nol > ocap) ocap *= 2;
                if (!ensure<uint64_t>(c, c->opened, ocap, true)) return APCLOUD_E_NOMEM;
            }
            APC_LAUNCH(c, K_TREE, div_up(ncand, T), T, 0, k_compact_u64, sc, ncand, f2, p2,
                       ptr<uint64_t>(c->opened) + oused);
        }
        ooff[l] = oused;
        ocount[l] = nol;
        oused += nol;
        prev_open = nol;
        if (U > 0) { cur = nxt; U = Ul; }
    }

    // leaves: the roots (one per beam) that are not opened, and for l = 1..L the
    // children of O_{l-1} not in O_l
    int64_t nseg = nb;
    std::vector<int64_t> segoff(L + 2, 0);
    for (int l = 1; l <= L; ++l) { segoff[l] = nseg; nseg += 8 * ocount[l - 1]; }
    uint32_t *f3 = ensure<uint32_t>(c, c->lval, nseg), *p3 = ensure<uint32_t>(c, c->lkey, nseg);
    if (!f3 || !p3) return APCLOUD_E_NOMEM;
    const uint64_t *ob = ptr<uint64_t>(c->opened);
    APC_LAUNCH(c, K_TREE, div_up(nb, T), T, 0, k_root_flags, nb, L > 0 ? ob + ooff[0] : ob, L > 0 ? ocount[0] : 0,
               f3);
    for (int l = 1; l <= L; ++l) {
        int64_t np = ocount[l - 1];
        if (np == 0) continue;
        APC_LAUNCH(c, K_TREE, div_up(8 * np, T), T, 0, k_leaf_flags, ob + ooff[l - 1], np,
                   l < L ? ob + ooff[l] : ob, l < L ? ocount[l] : 0, f3 + segoff[l]);
    }
    APC_TRY(scan_u32(c, f3, p3, nseg, small + 3));
    uint32_t hl;
    APC_TRY(read_back(c, &hl, small + 3, sizeof hl));
    const int64_t nleaf = hl;
    uint64_t *lk0 = ensure<uint64_t>(c, c->cand[0], nleaf), *lk1 = ensure<uint64_t>(c, c->cand[1], nleaf);
    uint32_t *lv0 = ensure<uint32_t>(c, c->cval[0], nleaf), *lv1 = ensure<uint32_t>(c, c->cval[1], nleaf);
    if (!lk0 || !lk1 || !lv0 || !lv1) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_TREE, div_up(nb, T), T, 0, k_root_emit, nb, f3, p3, L, lk0, lv0);
    for (int l = 1; l <= L; ++l) {
        int64_t np = ocount[l - 1];
        if (np == 0) continue;
        APC_LAUNCH(c, K_TREE, div_up(8 * np, T), T, 0, k_leaf_emit, ob + ooff[l - 1], np, f3 + segoff[l],
                   p3 + segoff[l], l, L, lk0, lv0);
    }
    int wl = 0;
    APC_TRY(radix_sort(c, lk0, lv0, lk1, lv1, nleaf, 3 * L + bb, &wl));
    uint64_t *anc = wl ? lk1 : lk0;
    uint32_t *alv = wl ? lv1 : lv0;
    c->n_int = (int)nleaf;

    // leaf geometry, particle ranges, boundary faces
    uint64_t *la = ensure<uint64_t>(c, c->leaf_anchor, nleaf);
    int8_t *ll = ensure<int8_t>(c, c->leaf_level, nleaf);
    int32_t *lb = ensure<int32_t>(c, c->leaf_beam, nleaf);
    int32_t *lf = ensure<int32_t>(c, c->leaf_first, nleaf);
    int32_t *lc = ensure<int32_t>(c, c->leaf_count, nleaf);
    uint32_t *bfl = ensure<uint32_t>(c, c->bidx, 12 * nleaf);  // flags then positions
    if (!la || !ll || !lf || !lc || !bfl || !lb) return APCLOUD_E_NOMEM;
    APC_CUDA(c, cudaMemcpyAsync(la, anc, nleaf * sizeof(uint64_t), cudaMemcpyDeviceToDevice, c->s));
    uint32_t *bpos = bfl + 6 * nleaf;
    // node coordinates need room for boundary nodes: at most 6 per leaf
    int4 *ic = ensure<int4>(c, c->node_ic, 7 * nleaf);
    if (!ic) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_TREE, div_up(nleaf, T), T, 0, k_leaf_geom, la, alv, nleaf, L, skeys, n, ll, lf, lc, ic, bfl, lb);
    int32_t *pl = ensure<int32_t>(c, c->pleaf, nn), *sp = ensure<int32_t>(c, c->spos, nn);
    if (!pl || !sp) return APCLOUD_E_NOMEM;
    if (n > 0)
        APC_LAUNCH(c, K_TREE, div_up(nleaf, 32 * (T / 32)), T, 0, k_particle_leaf, (const int32_t *)lf,
                   (const int32_t *)lc, (int)nleaf, (const uint32_t *)ptr<uint32_t>(c->val[c->kbuf]), pl, sp);
    APC_TRY(scan_u32(c, bfl, bpos, 6 * nleaf, small + 4));
    uint32_t hb;
    APC_TRY(read_back(c, &hb, small + 4, sizeof hb));
    c->n_bnd = (int)hb;
    c->n_tot = c->n_int + c->n_bnd;
    int32_t *bo = ensure<int32_t>(c, c->bowner, hb + 1);
    int8_t *bf = ensure<int8_t>(c, c->bface, hb + 1);
    int32_t *adj = ensure<int32_t>(c, c->adj, 24 * nleaf);
    if (!bo || !bf || !adj) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_TREE, div_up(6 * nleaf, T), T, 0, k_boundary, bfl, bpos, nleaf, ic, bo, bf);
    APC_LAUNCH(c, K_ADJ, div_up(6 * nleaf, T), T, 0, k_adjacency, la, ll, nleaf, L, bfl, bpos, adj, derr);
    int64_t *rng = ensure<int64_t>(c, c->beam_rng, 7 * (nb + 1));
    if (!rng) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_TREE, div_up(nb + 1, T), T, 0, k_beam_ranges, lb, nleaf, nb, bpos, (int64_t)hb, rng);
    APC_CUDA(c, cudaGetLastError());
    return check_device_errors(c);
}

}  // namespace apc

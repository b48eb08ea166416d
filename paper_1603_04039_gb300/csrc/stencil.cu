// stencil.cu -- Section 3.1 (WLS GFD operators) with the k-ring neighbour
// search of Section 4.3, and assembly of the density matrix B and the
// Poisson matrix A of Section 3.2 in sliced ELL.
//
// One warp per node.  The warp grows the k-ring (k = 2..ring_max) by BFS over
// the face adjacency with the candidate set in shared memory, sorts the
// candidates once by (exact integer squared distance, node index), takes the
// octant picks, the nearest fill and the ties as prefix counts (ballots) along
// that order, and builds the weighted scaled Vandermonde W V0 with one lane per
// neighbour (lane j = row j, m <= 32).  The least-squares operator
// P = (W V0)^+ W is formed by Cholesky QR applied twice (CholeskyQR2): the
// 9x9 Gram matrices come from shared memory and are factored by the whole
// warp, Q = A R^-1 is lane-local, and column j of P is R^-1 q_j^T W_j, again
// lane-local.  This replaces the column-by-column Householder reductions of a
// CPU QR (9 dependent cross-lane reductions) with two Gram products, two
// 9-step warp factorisations and lane-private triangular solves.
#include <cuda_fp16.h>

#include <cmath>

#include "fpconv.cuh"
#include "internal.cuh"

namespace apc {

namespace {

constexpr int ASTR = NCOL;      // row stride of the staged Vandermonde

// MC candidate slots: MAXC_FAST in the kernel over all nodes, MAXC in the one
// that redoes the nodes whose rings outgrew them
template <int MC>
struct __align__(16) WarpSmemT {
    int32_t cand[MC];   // read four at a time by the membership test
    long long d2[MC];
    uint16_t srt[MC];   // candidate slots in (d2, index) order
    uint8_t oct[MC];
    uint8_t pick[MC];   // octant picks, by sorted position
    int32_t sel[MMAX];
    long long seld2[MMAX];
    double A[MMAX * ASTR];
    double G[48];
    double R1[NCOL * NCOL];
    double R2[NCOL * NCOL];
    double Ri1[NCOL], Ri2[NCOL];   // reciprocal diagonals of R1, R2
};


__device__ __forceinline__ bool key_less(long long da, int ia, long long db, int ib) {
    return da < db || (da == db && ia < ib);
}

__device__ __forceinline__ long long warp_max_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t > v ? t : v;
    }
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Packed upper storage of the symmetric 9x9 Gram matrix: entry (a, b), a <= b,
// sits at a * 9 - a (a - 1) / 2 + (b - a), 45 entries in all.  Lane l owns
// entries l and l + 32 (the second only for l < 13).
__device__ __forceinline__ int pk_idx(int a, int b) { return a * NCOL - a * (a - 1) / 2 + (b - a); }

struct GramOwn {
    int a1, b1, a2, b2;
    bool two;
};

__device__ __forceinline__ void pk_rowcol(int e, int &a, int &b) {
    int e0 = 0;
    a = 0;
    while (e - e0 >= NCOL - a) { e0 += NCOL - a; ++a; }
    b = a + (e - e0);
}

__device__ __forceinline__ GramOwn gram_own(int lane) {
    GramOwn o;
    o.two = lane + 32 < NCOL * (NCOL + 1) / 2;
    pk_rowcol(lane, o.a1, o.b1);
    pk_rowcol(o.two ? lane + 32 : 0, o.a2, o.b2);
    return o;
}

// Cholesky G = R^T R of the packed Gram matrix by the whole warp: right-looking,
// each lane updating the trailing entries it owns after the pivot row k is
// scaled.  R is row-major upper (the strict lower part is not written), Ri the
// reciprocals of its diagonal.  G is overwritten.  Returns false on a
// non-positive pivot, the same decision in every lane.
template <class T>
__device__ bool cholesky_warp(T *G, T *R, T *Ri, const GramOwn &o, int lane) {
    for (int k = 0; k < NCOL; ++k) {
        const T gkk = G[pk_idx(k, k)];
        if (!(gkk > (T)0)) return false;
        const T d = sqrt(gkk), rd = (T)1 / d;
        if (o.a1 == k) R[k * NCOL + o.b1] = (o.b1 == k) ? d : G[lane] * rd;
        else if (o.a1 > k) G[lane] -= (G[pk_idx(k, o.a1)] * rd) * (G[pk_idx(k, o.b1)] * rd);
        if (o.two) {
            if (o.a2 == k) R[k * NCOL + o.b2] = (o.b2 == k) ? d : G[lane + 32] * rd;
            else if (o.a2 > k) G[lane + 32] -= (G[pk_idx(k, o.a2)] * rd) * (G[pk_idx(k, o.b2)] * rd);
        }
        if (lane == 0) Ri[k] = rd;
        __syncwarp();
    }
    return true;
}

// FP32 Cholesky of the packed Gram matrix computed by every lane at once in
// registers (the 45 entries are broadcast from shared memory, the nine pivot
// steps run without any exchange between lanes); lane 0 stores R and the
// reciprocal pivots for the triangular solves.  The reciprocal square root of
// each pivot gives both R_kk = g * rsqrt(g) and 1 / R_kk.  Returns false on a
// non-positive pivot, the same decision in every lane.
__device__ bool cholesky_regs(const float *G, float *R, float *Ri, int lane) {
    float g[45];
#pragma unroll
    for (int e = 0; e < 45; ++e) g[e] = G[e];
    float rd[NCOL];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < NCOL; ++k) {
        const float gkk = g[pk_idx(k, k)];
        ok = ok && gkk > 0.f;
        const float r = rsqrtf(ok ? gkk : 1.f);
        rd[k] = r;
        g[pk_idx(k, k)] = gkk * r;
#pragma unroll
        for (int j = k + 1; j < NCOL; ++j) g[pk_idx(k, j)] *= r;
#pragma unroll
        for (int i = k + 1; i < NCOL; ++i)
#pragma unroll
            for (int j = i; j < NCOL; ++j) g[pk_idx(i, j)] = fmaf(-g[pk_idx(k, i)], g[pk_idx(k, j)], g[pk_idx(i, j)]);
    }
    if (!ok) return false;
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < NCOL; ++a) {
            Ri[a] = rd[a];
#pragma unroll
            for (int b = a; b < NCOL; ++b) R[a * NCOL + b] = g[pk_idx(a, b)];
        }
    }
    __syncwarp();
    return true;
}

// the FP32 path factors in registers, the FP64 path with the warp
template <class T>
__device__ __forceinline__ bool cholesky(T *G, T *R, T *Ri, const GramOwn &o, int lane) {
    if constexpr (sizeof(T) == 4) return cholesky_regs(G, R, Ri, lane);
    else return cholesky_warp<T>(G, R, Ri, o, lane);
}

// solve q R = a for the row vector q (R upper), in place on v
template <class T>
__device__ __forceinline__ void row_solve_upper(const T *R, const T *Ri, T *v) {
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
        T s = v[c];
#pragma unroll
        for (int k = 0; k < c; ++k) s -= v[k] * R[k * NCOL + c];
        v[c] = s * Ri[c];
    }
}

// solve R z = v for the column vector z (R upper), in place
template <class T>
__device__ __forceinline__ void col_solve_upper(const T *R, const T *Ri, T *v) {
#pragma unroll
    for (int c = NCOL - 1; c >= 0; --c) {
        T s = v[c];
#pragma unroll
        for (int k = c + 1; k < NCOL; ++k) s -= R[c * NCOL + k] * v[k];
        v[c] = s * Ri[c];
    }
}

// Gram matrix of the m staged rows, the lane's two owned entries accumulated
// side by side
template <class T>
__device__ __forceinline__ void gram(const T *A, int m, T *G, const GramOwn &o, int lane) {
    T s1 = (T)0, s2 = (T)0;
    for (int j = 0; j < m; ++j) {
        const T *r = A + j * ASTR;
        s1 = fma(r[o.a1], r[o.b1], s1);
        s2 = fma(r[o.a2], r[o.b2], s2);
    }
    G[lane] = s1;
    if (o.two) G[lane + 32] = s2;
}

__device__ __forceinline__ double exp_t(double v) { return exp(v); }
__device__ __forceinline__ float exp_t(float v) { return expf(v); }

// Weighted least-squares operator (Section 3.1) of the stencil staged in
// W.sel / W.seld2, in arithmetic T: rows of W V0 (Eq. regfd with the
// normalized Gaussian weight), CholeskyQR2, and column `lane` of
// P = (W V0)^+ W unscaled by h and h^2, returned in FP64.  Returns false when
// a Cholesky pivot fails; rratio = min |R_ii| / max |R_ii|.
template <class T, class WS>
__device__ bool wls_column(WS &W, int m, int lane, const GramOwn &own, int4 c0, const int4 *__restrict__ ic,
                           double unit, double ec, double inv_1mec, double (&qout)[NCOL], double &lapj,
                           double &rratio) {
    T *A = reinterpret_cast<T *>(W.A);
    T *G = reinterpret_cast<T *>(W.G);
    T *R1 = reinterpret_cast<T *>(W.R1);
    T *R2 = reinterpret_cast<T *>(W.R2);
    T *Ri1 = reinterpret_cast<T *>(W.Ri1);
    T *Ri2 = reinterpret_cast<T *>(W.Ri2);
    long long off[3] = {0, 0, 0};
    long long mydist = 0, amax = 0;
    if (lane < m) {
        int4 q = ic[W.sel[lane]];
        off[0] = (long long)q.x - c0.x; off[1] = (long long)q.y - c0.y; off[2] = (long long)q.z - c0.z;
        mydist = W.seld2[lane];
        for (int d = 0; d < 3; ++d) { long long a = off[d] < 0 ? -off[d] : off[d]; amax = a > amax ? a : amax; }
    }
    const long long hint = warp_max_ll(amax);
    const long long r2max = W.seld2[m - 1];
    T wj = (T)0;
    {
        T row[NCOL];
#pragma unroll
        for (int e = 0; e < NCOL; ++e) row[e] = (T)0;
        if (lane < m) {
            // xi = dy / h with h = max |dy_d| (Section 3.1): exact integers, one rounding in T
            T xi0 = (T)off[0] / (T)hint, xi1 = (T)off[1] / (T)hint, xi2 = (T)off[2] / (T)hint;
            T ratio = (T)mydist / (T)r2max;
            wj = (exp_t(-ratio) - (T)ec) * (T)inv_1mec;
            const T half = (T)0.5;
            row[0] = xi0; row[1] = xi1; row[2] = xi2;
            row[3] = (half * xi0) * xi0;
            row[4] = xi0 * xi1;
            row[5] = xi0 * xi2;
            row[6] = (half * xi1) * xi1;
            row[7] = xi1 * xi2;
            row[8] = (half * xi2) * xi2;
#pragma unroll
            for (int e = 0; e < NCOL; ++e) row[e] = wj * row[e];
        }
#pragma unroll
        for (int e = 0; e < NCOL; ++e) A[lane * ASTR + e] = row[e];
    }
    __syncwarp();
    gram<T>(A, m, G, own, lane);
    __syncwarp();
    bool ok = cholesky<T>(G, R1, Ri1, own, lane);
    T q[NCOL];
    if (ok) {
        if (lane < m) {
#pragma unroll
            for (int e = 0; e < NCOL; ++e) q[e] = A[lane * ASTR + e];
            row_solve_upper<T>(R1, Ri1, q);
#pragma unroll
            for (int e = 0; e < NCOL; ++e) A[lane * ASTR + e] = q[e];
        }
        __syncwarp();
        gram<T>(A, m, G, own, lane);
        __syncwarp();
        ok = cholesky<T>(G, R2, Ri2, own, lane);
    }
    rratio = 0.0;
    lapj = 0.0;
    if (!ok) return false;
    T dmin = (T)1e30, dmax = (T)0;
#pragma unroll
    for (int e = 0; e < NCOL; ++e) {
        T r = fabs(R1[e * NCOL + e] * R2[e * NCOL + e]);
        dmin = fmin(dmin, r);
        dmax = fmax(dmax, r);
    }
    rratio = (double)(dmin / dmax);
    // unscale rows by 1/h and 1/h^2 (h = max |dy_d|), in T
    const T h = (T)((double)hint * unit);
    const T ih = (T)1 / h, ih2 = ih * ih;
    if (lane < m) {
#pragma unroll
        for (int e = 0; e < NCOL; ++e) q[e] = A[lane * ASTR + e];
        row_solve_upper<T>(R2, Ri2, q);
        col_solve_upper<T>(R2, Ri2, q);
        col_solve_upper<T>(R1, Ri1, q);
        T lj = (T)0;
#pragma unroll
        for (int e = 0; e < NCOL; ++e) {
            const T v = (q[e] * wj) * (e < 3 ? ih : ih2);
            qout[e] = (double)v;
            if (e == 3 || e == 6 || e == 8) lj += v;
        }
        lapj = (double)lj;
    } else {
#pragma unroll
        for (int e = 0; e < NCOL; ++e) qout[e] = 0.0;
    }
    return true;
}

// The rows of the derivative operator D (row-of-operator major, nodes
// fastest) of a block's SW nodes.  Each warp stages its node's 9 x MMAX block
// in its W.A as [e * MMAX + lane] (free once the WLS is done); the last warp
// of the block to finish writes every row as SW consecutive nodes, one
// 8 x SW-byte run per row, where each warp writing its own node would store
// 288 lone 8-byte words, each in a sector of its own.  Warps without a node
// (past n_int) only arrive.
template <int SW, class WS>
__device__ __forceinline__ void write_block_d(const unsigned char *smem_raw, unsigned *arrived, int lane, int y_base,
                                              int n_int, double *__restrict__ D_out, int64_t dstride) {
    __threadfence_block();
    __syncwarp();
    unsigned last = 0u;
    if (lane == 0) last = (atomicAdd(arrived, 1u) == SW - 1) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence_block();
    const WS *Ws = reinterpret_cast<const WS *>(smem_raw);
    for (int t = lane; t < NCOL * MMAX * SW; t += 32) {
        const int row = t / SW, w = t - row * SW;
        const int y = y_base + w;
        if (y < n_int) D_out[(int64_t)row * dstride + y] = Ws[w].A[row];
    }
}

// SW warps (nodes) per block, one WarpSmemT<MC> each (and the block's
// arrival count after them); the autotuner picks SW.  With MC = MAXC_FAST
// (LIST false, every node): 6.6 KB of shared memory per warp and 32 warps per
// SM at a register budget that spills part of the FP32 factorisation; a node
// whose ring outgrows MC candidates goes to ovf_list instead of failing.
// Against 512 slots at 16 warps: 7.1 -> 5.9 ms on a 1e7-particle beam and
// 31.6 -> 26.1 ms on a 64-beam batch (both passes).  With MC = MAXC and LIST: the nodes of that list
// (n_list of them), each warp writing its own D columns.  slots <= MC is the
// capacity in force (the context's stencil_slots in the first kernel).
template <int SW, int MC, bool LIST>
__global__ void __launch_bounds__(SW * 32, (MC < MAXC ? 32 : 16) / SW) k_stencil(
    const int4 *__restrict__ ic, const int32_t *__restrict__ adj, const int32_t *__restrict__ bowner, int n_int,
    int m_target, int ring_max, double unit, double ec, double inv_1mec, int32_t *__restrict__ nbr_out,
    int32_t *__restrict__ m_out, int32_t *__restrict__ ring_out, double *__restrict__ lap_out,
    double *__restrict__ lapd_out, double *__restrict__ D_out, int64_t dstride, double *__restrict__ rcond_out,
    int fp32_first, double fp32_rcond_min, int *__restrict__ fp64_count, unsigned *err,
    const int32_t *__restrict__ list, int n_list, unsigned *__restrict__ ovf_count, int32_t *__restrict__ ovf_list,
    int slots) {
    typedef WarpSmemT<MC> WarpSmem;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem &W = reinterpret_cast<WarpSmem *>(smem_raw)[wid];
    const int li = blockIdx.x * SW + wid;
    const int y0 = LIST ? (li < n_list ? list[li] : n_int) : li;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    unsigned *arrived = reinterpret_cast<unsigned *>(reinterpret_cast<WarpSmem *>(smem_raw) + SW);
    if (!LIST) {
        if (threadIdx.x == 0) *arrived = 0u;
        __syncthreads();
    }
    if (y0 >= n_int) {
        if (!LIST) write_block_d<SW, WarpSmem>(smem_raw, arrived, lane, blockIdx.x * SW, n_int, D_out, dstride);
        return;
    }

    const int4 c0 = ic[y0];
    int nc = 1;
    if (lane == 0) W.cand[0] = y0;
    __syncwarp();
    int head = 0, tail = 1;
    bool done = false, overflow = false;
    int m = 0, ring = 0;
    double rmin_over_rmax = 0.0;

    const GramOwn own = gram_own(lane);

    for (int k = 1; k <= ring_max && !done; ++k) {
        // ---- grow the ring by one layer (Section 4.3: (k+1)-ring = k-ring
        // plus the face neighbours of its nodes).  The frontier [head, tail)
        // does not change while the layer grows, so the adjacency of up to
        // eight 32-slot batches is loaded before any of them is merged; the
        // valid slots (about a quarter: a face with a same-size or coarser
        // neighbour fills one of its four) are packed densely in the d2 area,
        // which is free until the candidates are ranked.
        int32_t *stg = reinterpret_cast<int32_t *>(W.d2);
        const int nslots = (tail - head) * 24;
        for (int g0 = 0; g0 < nslots; g0 += 8 * 32) {
            int vb[8];
#pragma unroll
            for (int bt = 0; bt < 8; ++bt) {
                const int s = g0 + bt * 32 + lane;
                int v = -1;
                if (s < nslots) {
                    const int u = W.cand[head + s / 24];
                    const int slot = s % 24;
                    if (u < n_int) v = adj[(int64_t)u * 24 + slot];
                    else if (slot == 0) v = bowner[u - n_int];
                }
                vb[bt] = v;
            }
            int nv = 0;
#pragma unroll
            for (int bt = 0; bt < 8; ++bt) {
                const unsigned bv = __ballot_sync(FULL, vb[bt] >= 0);
                if (vb[bt] >= 0) stg[nv + __popc(bv & lt)] = vb[bt];
                nv += __popc(bv);
            }
            __syncwarp();
            for (int b0 = 0; b0 < nv; b0 += 32) {
                const int v = (b0 + lane < nv) ? stg[b0 + lane] : -1;
                bool fresh = v >= 0;
                for (int t = 0; fresh && t < nc; t += 4) {
                    const int4 c4 = *reinterpret_cast<const int4 *>(&W.cand[t]);
                    if (c4.x == v || (c4.y == v && t + 1 < nc) || (c4.z == v && t + 2 < nc) ||
                        (c4.w == v && t + 3 < nc))
                        fresh = false;
                }
                unsigned peers = __match_any_sync(FULL, fresh ? v : -2 - lane);
                if (fresh && lane != __ffs(peers) - 1) fresh = false;
                unsigned bal = __ballot_sync(FULL, fresh);
                int p = nc + __popc(bal & lt);
                if (fresh) {
                    if (p < slots) W.cand[p] = v;
                    else overflow = true;
                }
                nc += __popc(bal);
                if (nc > slots) nc = slots;
                __syncwarp();
            }
        }
        if (__any_sync(FULL, overflow)) break;
        head = tail;
        tail = nc;
        if (k < 2) continue;
        const int ncand = nc - 1;
        if (ncand < m_target && k < ring_max) continue;
        if (ncand < NCOL) continue;

        // ---- order the candidates by (exact integer squared distance, node
        // index): every later choice is a prefix of this order
        for (int t = 1 + lane; t < nc; t += 32) {
            int4 q = ic[W.cand[t]];
            long long dx = (long long)q.x - c0.x, dy = (long long)q.y - c0.y, dz = (long long)q.z - c0.z;
            W.d2[t] = dx * dx + dy * dy + dz * dz;
            W.oct[t] = (uint8_t)(((dx >= 0) << 2) | ((dy >= 0) << 1) | (dz >= 0));
        }
        __syncwarp();
        for (int t = 1 + lane; t < nc; t += 32) {
            const long long dt = W.d2[t];
            const int it = W.cand[t];
            int r = 0;
            for (int u = 1; u < nc; ++u) r += key_less(W.d2[u], W.cand[u], dt, it) ? 1 : 0;
            W.srt[r] = (uint16_t)t;
        }
        __syncwarp();
        // ---- Section 3.1 quadrant criterion, octants in 3-D: the two nearest
        // in each octant, counted along the order 32 positions at a time
        int nA = 0;
        {
            int cnt[8];
#pragma unroll
            for (int o = 0; o < 8; ++o) cnt[o] = 0;
            for (int p0 = 0; p0 < ncand; p0 += 32) {
                const int pos = p0 + lane;
                const int o = (pos < ncand) ? (int)W.oct[W.srt[pos]] : -1;
                int before = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const unsigned bq = __ballot_sync(FULL, o == q);
                    if (o == q) before = cnt[q] + __popc(bq & lt);
                    cnt[q] += __popc(bq);
                }
                const bool pk = o >= 0 && before < 2;
                if (pos < ncand) W.pick[pos] = pk ? 1 : 0;
                nA += __popc(__ballot_sync(FULL, pk));
            }
        }
        __syncwarp();
        // target sizes m_target, m_target + 2, ... (a rank-deficient stencil or
        // one whose Laplacian diagonal is not negative is not used).  One pass
        // along the order: the picks, then the nearest non-picked up to the
        // target (the last of them sets the cut distance), then every further
        // candidate tied at the cut while the stencil has room, in index order;
        // the stencil is written in (d2, index) order.
        for (int mt = m_target; mt <= MMAX && !done; mt += 2) {
        const int need = mt - nA;
        const int room = MMAX - nA - (need > 0 ? need : 0);
        int nsel = 0, nnp = 0, ntie = 0;
        bool cut_found = false;
        long long cut = 0;
        for (int p0 = 0; p0 < ncand; p0 += 32) {
            const int pos = p0 + lane;
            const bool valid = pos < ncand;
            int t = 0;
            long long d = 0;
            bool pk = false;
            if (valid) { t = W.srt[pos]; d = W.d2[t]; pk = W.pick[pos] != 0; }
            const bool np = valid && !pk;
            const unsigned bnp = __ballot_sync(FULL, np);
            const int npr = nnp + __popc(bnp & lt);
            const bool fill = np && npr < need;
            if (!cut_found) {
                const unsigned bc = __ballot_sync(FULL, np && npr == need - 1);
                if (bc) {
                    cut = __shfl_sync(FULL, d, __ffs(bc) - 1);
                    cut_found = true;
                }
            }
            const bool te = np && !fill && cut_found && d == cut;
            const unsigned bte = __ballot_sync(FULL, te);
            const bool tie = te && ntie + __popc(bte & lt) < room;
            ntie += __popc(__ballot_sync(FULL, tie));
            const bool sl = pk || fill || tie;
            const unsigned bs = __ballot_sync(FULL, sl);
            if (sl) {
                const int r = nsel + __popc(bs & lt);
                W.sel[r] = W.cand[t];
                W.seld2[r] = d;
            }
            nsel += __popc(bs);
            nnp += __popc(bnp);
        }
        __syncwarp();
        m = nsel;

        // ---- weighted least squares: FP32 first when asked, FP64 for blocks the
        // FP32 factorisation cannot certify (Cholesky failure or condition
        // estimate min|R_ii|/max|R_ii| below fp32_rcond_min, by default 1e-3,
        // where FP32 Cholesky QR loses its accuracy)
        double q[NCOL], lapj = 0.0;
        bool ok = false;
        if (fp32_first) {
            ok = wls_column<float>(W, m, lane, own, c0, ic, unit, ec, inv_1mec, q, lapj, rmin_over_rmax);
            if (ok && rmin_over_rmax < fp32_rcond_min) ok = false;
            if (!ok && lane == 0) atomicAdd(fp64_count, 1);
        }
        if (!ok) ok = wls_column<double>(W, m, lane, own, c0, ic, unit, ec, inv_1mec, q, lapj, rmin_over_rmax);
        if (ok) ok = rmin_over_rmax >= RANK_TOL;
        if (!ok) lapj = 0.0;
        const double lsum = warp_sum_d(lapj);
        if (!ok || !(-lsum < 0.0)) {       // unusable: more neighbours, then a wider ring
            if (m >= nc - 1) break;
            continue;
        }

        nbr_out[(int64_t)y0 * MMAX + lane] = (lane < m) ? W.sel[lane] : -1;
        lap_out[(int64_t)y0 * MMAX + lane] = lapj;
        if (lane == 0) {
            lapd_out[y0] = -lsum;
            m_out[y0] = m;
            ring_out[y0] = k;
            rcond_out[y0] = rmin_over_rmax;
        }
        __syncwarp();
        // derivative operator, staged for write_block_d (the list kernel's
        // nodes are not consecutive: each warp writes its own columns)
        __syncwarp();
        if (LIST) {
#pragma unroll
            for (int e = 0; e < NCOL; ++e) D_out[((int64_t)e * MMAX + lane) * dstride + y0] = (lane < m) ? q[e] : 0.0;
        } else {
#pragma unroll
            for (int e = 0; e < NCOL; ++e) W.A[e * MMAX + lane] = (lane < m) ? q[e] : 0.0;
        }
        ring = k;
        done = true;
        }   // target sizes
    }
    if (!done) {
        const bool ovf = __any_sync(FULL, overflow);
        if (lane == 0) {
            if (ovf && !LIST) ovf_list[atomicAdd(ovf_count, 1u)] = y0;   // redone with MAXC slots
            else atomicOr(err, ovf ? (ERR_STENCIL | ERR_OVERFLOW) : ERR_STENCIL);
            m_out[y0] = 0;
            ring_out[y0] = -1;
            lapd_out[y0] = 0.0;
            rcond_out[y0] = 0.0;
        }
        nbr_out[(int64_t)y0 * MMAX + lane] = -1;
        lap_out[(int64_t)y0 * MMAX + lane] = 0.0;
        __syncwarp();
        if (LIST) {
#pragma unroll
            for (int e = 0; e < NCOL; ++e) D_out[((int64_t)e * MMAX + lane) * dstride + y0] = 0.0;
        } else {
#pragma unroll
            for (int e = 0; e < NCOL; ++e) W.A[e * MMAX + lane] = 0.0;
        }
    }
    (void)ring;
    if (!LIST) write_block_d<SW, WarpSmem>(smem_raw, arrived, lane, blockIdx.x * SW, n_int, D_out, dstride);
}

// ---------------------------------------------------------------- matrices
// diagonals of A and B (the Jacobi scaling) and their reciprocals
__global__ void k_diag(const int32_t *__restrict__ msz, const double *__restrict__ lapd, const int4 *__restrict__ ic,
                       int n_int, int n_tot, double ext, double *__restrict__ dA, double *__restrict__ dB,
                       double *__restrict__ rA, double *__restrict__ rB) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_tot) return;
    double a = 1.0, b = 1.0;
    if (r < n_int) {
        double h = ldexp(ext, -ic[r].w);
        double s = h * h / 24.0;
        a = lapd[r];
        b = 1.0 + s * lapd[r];
    }
    dA[r] = a;
    dB[r] = b;
    rA[r] = 1.0 / a;
    rB[r] = 1.0 / b;
}

__global__ void k_slice_width(const int32_t *__restrict__ msz, int n_int, int n_tot, int nsl, uint32_t *__restrict__ w) {
    int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (s >= nsl) return;
    int r = s * 32 + lane;
    int v = 0;
    if (r < n_int) v = msz[r] + 1;
    else if (r < n_tot) v = 1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) { int t = __shfl_xor_sync(0xffffffffu, v, o); v = t > v ? t : v; }
    if (lane == 0) w[s] = (uint32_t)v;
}

// Row j of A: diag = -sum l, off-diagonals l_ji; row j of B: 1 + (h_j^2/24) A_jj
// and (h_j^2/24) l_ji (Section 3.2 with the cell-indicator moments); boundary
// rows are identity rows.  Values are stored right-scaled by the inverse
// diagonal of the column (Jacobi preconditioning folded into the matrix).
__global__ void k_ell_fill(const int32_t *__restrict__ msz, const int32_t *__restrict__ nbr,
                           const double *__restrict__ lap, const double *__restrict__ lapd, const int4 *__restrict__ ic,
                           const double *__restrict__ dA, const double *__restrict__ dB, const double *__restrict__ rA,
                           const double *__restrict__ rB, int n_int, int n_tot, double ext,
                           const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                           int32_t *__restrict__ col, double *__restrict__ vA, double *__restrict__ vB) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int s = r >> 5, lane = r & 31;
    if (s * 32 >= n_tot) return;
    int w = (int)sw[s];
    int64_t base = (int64_t)soff[s] * 32 + lane;
    if (r >= n_tot) {
        for (int k = 0; k < w; ++k) { col[base + k * 32] = 0; vA[base + k * 32] = 0.0; vB[base + k * 32] = 0.0; }
        return;
    }
    if (r >= n_int) {
        col[base] = r; vA[base] = 1.0 / dA[r]; vB[base] = 1.0 / dB[r];
        for (int k = 1; k < w; ++k) { col[base + k * 32] = r; vA[base + k * 32] = 0.0; vB[base + k * 32] = 0.0; }
        return;
    }
    int m = msz[r];
    double h = ldexp(ext, -ic[r].w);
    double sc = h * h / 24.0;
    col[base] = r;
    vA[base] = lapd[r] / dA[r];
    vB[base] = (1.0 + sc * lapd[r]) / dB[r];
    for (int k = 1; k < w; ++k) {
        int64_t e = base + (int64_t)k * 32;
        if (k <= m) {
            int cj = nbr[(int64_t)r * MMAX + k - 1];
            double l = lap[(int64_t)r * MMAX + k - 1];
            // off-diagonal entries times the column's reciprocal diagonal (an
            // FP64 division per entry would make this pass FP64-bound; the
            // diagonal entries above keep their exact division, so they stay 1)
            col[e] = cj;
            vA[e] = l * rA[cj];
            vB[e] = (sc * l) * rB[cj];
        } else {
            col[e] = r;
            vA[e] = 0.0;
            vB[e] = 0.0;
        }
    }
}

// FP32 copies of the stored (Jacobi-scaled) matrix values for the mixed form
__global__ void k_values_f32(const double *__restrict__ vA, const double *__restrict__ vB, int64_t n,
                             float *__restrict__ fA, float *__restrict__ fB, __half *__restrict__ hA,
                             __half *__restrict__ hB) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        // the FP32 copies on the integer pipe (bit-exact); the FP16 ones keep
        // the hardware conversion (a direct rounding from FP64)
        fA[i] = f64_to_f32_int(vA[i]);
        fB[i] = f64_to_f32_int(vB[i]);
        hA[i] = __double2half(vA[i]);
        hB[i] = __double2half(vB[i]);
    }
}

template <int SW>
apcloud_status launch_stencil(apcloud_ctx *c, int n, double unit, double ec, double inv_1mec, int32_t *nbr,
                              int32_t *msz, int32_t *ring, double *lap, double *lapd, double *D, int64_t dstride,
                              double *rc, unsigned *derr) {
    // every node with MAXC_FAST candidate slots, then (one read-back of the
    // count) the nodes whose rings outgrew them with MAXC
    int32_t *ovf = ensure<int32_t>(c, c->stencil_ovf, n + 1);
    if (!ovf) return APCLOUD_E_NOMEM;
    APC_CUDA(c, cudaMemsetAsync(derr + 2, 0, sizeof(unsigned), c->s));
    const size_t smem = SW * sizeof(WarpSmemT<MAXC_FAST>) + 16;   // the warps' areas, then the block's arrival count
    // the limit is a per-device property of the function: set on every build
    // (one host call each), so that contexts on other devices get it too
    APC_CUDA(c, cudaFuncSetAttribute(k_stencil<SW, MAXC_FAST, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    APC_CUDA(c, cudaFuncSetAttribute(k_stencil<4, MAXC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(4 * sizeof(WarpSmemT<MAXC>) + 16)));
    APC_LAUNCH(c, K_STENCIL, div_up(n, SW), SW * 32, smem, (k_stencil<SW, MAXC_FAST, false>), ptr<int4>(c->node_ic),
               ptr<int32_t>(c->adj), ptr<int32_t>(c->bowner), n, c->P.m_target, c->P.ring_max, unit, ec, inv_1mec,
               nbr, msz, ring, lap, lapd, D, dstride, rc, c->P.precision == 1 ? 1 : 0, c->P.fp32_rcond_min,
               reinterpret_cast<int *>(derr + 1), derr, (const int32_t *)nullptr, 0, derr + 2, ovf, c->P.stencil_slots);
    unsigned nov = 0;
    APC_TRY(read_back(c, &nov, derr + 2, sizeof nov));
    if (nov > 0)
        APC_LAUNCH(c, K_STENCIL, div_up(nov, 4), 4 * 32, 4 * sizeof(WarpSmemT<MAXC>) + 16, (k_stencil<4, MAXC, true>),
                   ptr<int4>(c->node_ic), ptr<int32_t>(c->adj), ptr<int32_t>(c->bowner), n, c->P.m_target,
                   c->P.ring_max, unit, ec, inv_1mec, nbr, msz, ring, lap, lapd, D, dstride, rc,
                   c->P.precision == 1 ? 1 : 0, c->P.fp32_rcond_min, reinterpret_cast<int *>(derr + 1), derr,
                   (const int32_t *)ovf, (int)nov, derr + 2, ovf, MAXC);
    return APCLOUD_OK;
}

}  // namespace

apcloud_status build_stencils(apcloud_ctx *c) {
    const int n = c->n_int, nt = c->n_tot;
    const int64_t dstride = ((int64_t)n + 31) / 32 * 32;
    int32_t *nbr = ensure<int32_t>(c, c->nbr, (int64_t)n * MMAX);
    int32_t *msz = ensure<int32_t>(c, c->msz, n + 1);
    int32_t *ring = ensure<int32_t>(c, c->ring, n + 1);
    double *lap = ensure<double>(c, c->lap, (int64_t)n * MMAX);
    double *lapd = ensure<double>(c, c->lapd, n + 1);
    double *D = ensure<double>(c, c->D, (int64_t)NCOL * MMAX * dstride);
    double *rc = ensure<double>(c, c->rcond, n + 1);
    if (!nbr || !msz || !ring || !lap || !lapd || !D || !rc) return APCLOUD_E_NOMEM;
    unsigned *derr = ptr<unsigned>(c->derr);
    APC_CUDA(c, cudaMemsetAsync(derr, 0, 4 * sizeof(unsigned), c->s));
    const double ext = c->P.hi[0] - c->P.lo[0];
    const double unit = ldexp(ext, -(KEY_DEPTH + 1));
    const double ec = exp(-c->P.weight_c);
    const double inv_1mec = 1.0 / (1.0 - ec);
    switch (c->wls_warps) {
    case 2:
        APC_TRY(launch_stencil<2>(c, n, unit, ec, inv_1mec, nbr, msz, ring, lap, lapd, D, dstride, rc, derr));
        break;
    case 8:
        APC_TRY(launch_stencil<8>(c, n, unit, ec, inv_1mec, nbr, msz, ring, lap, lapd, D, dstride, rc, derr));
        break;
    default:
        APC_TRY(launch_stencil<4>(c, n, unit, ec, inv_1mec, nbr, msz, ring, lap, lapd, D, dstride, rc, derr));
        break;
    }
    APC_CUDA(c, cudaGetLastError());
    APC_TRY(check_device_errors(c));
    {
        unsigned e[2];
        APC_TRY(read_back(c, e, derr, sizeof e));
        c->n_fp64_wls = e[1];
    }
    {   // total stencil size, for the algorithmic traffic of later kernels
        uint32_t *tmp = ensure<uint32_t>(c, c->tmp, n + 1);
        if (!tmp) return APCLOUD_E_NOMEM;
        uint32_t *small = ptr<uint32_t>(c->dsmall);
        APC_TRY(scan_u32(c, reinterpret_cast<const uint32_t *>(msz), tmp, n, small + 6));
        uint32_t sm;
        APC_TRY(read_back(c, &sm, small + 6, sizeof sm));
        c->sum_m = sm;
        // per node: offsets and weights in (28 B per neighbour), Laplacian row and
        // 9 x m operator out (80 B per neighbour); two 9-column Gram products,
        // three triangular solves per row and two 9x9 factorizations
        account(c, K_STENCIL, 108.0 * sm + 8.0 * n, 450.0 * sm + 660.0 * n);
    }

    // sliced ELL of A and B
    const int nsl = div_up(nt, 32);
    c->n_slices = nsl;
    uint32_t *sw = ensure<uint32_t>(c, c->slice_w, nsl + 1);
    uint32_t *so = ensure<uint32_t>(c, c->slice_off, nsl + 1);
    double *dA = ensure<double>(c, c->dA, nt + 1);
    double *dB = ensure<double>(c, c->dB, nt + 1);
    double *rd = ensure<double>(c, c->ell_rd, 2 * ((int64_t)nt + 1));   // reciprocals, for the fill only
    if (!sw || !so || !dA || !dB || !rd) return APCLOUD_E_NOMEM;
    double *rA = rd, *rB = rd + nt + 1;
    APC_LAUNCH(c, K_ELL, div_up(nt, 256), 256, 0, k_diag, msz, lapd, ptr<int4>(c->node_ic), n, nt, ext, dA, dB, rA,
               rB);
    APC_LAUNCH(c, K_ELL, div_up(nsl, 8), 256, 0, k_slice_width, msz, n, nt, nsl, sw);
    uint32_t *small = ptr<uint32_t>(c->dsmall);
    APC_TRY(scan_u32(c, sw, so, nsl, small + 5));
    uint32_t tot;
    APC_TRY(read_back(c, &tot, small + 5, sizeof tot));
    c->ell_entries = (int64_t)tot * 32;
    int32_t *col = ensure<int32_t>(c, c->ell_col, c->ell_entries);
    double *vA = ensure<double>(c, c->ell_A, c->ell_entries);
    double *vB = ensure<double>(c, c->ell_B, c->ell_entries);
    if (!col || !vA || !vB) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_ELL, div_up((int64_t)nsl * 32, 256), 256, 0, k_ell_fill, msz, nbr, lap, lapd,
               ptr<int4>(c->node_ic), dA, dB, (const double *)rA, (const double *)rB, n, nt, ext, sw, so, col, vA,
               vB);
    if (c->P.precision == 1) {
        float *fA = ensure<float>(c, c->ell_A32, c->ell_entries), *fB = ensure<float>(c, c->ell_B32, c->ell_entries);
        __half *hA = ensure<__half>(c, c->ell_A16, c->ell_entries), *hB = ensure<__half>(c, c->ell_B16, c->ell_entries);
        if (!fA || !fB || !hA || !hB) return APCLOUD_E_NOMEM;
        APC_LAUNCH(c, K_ELL, div_up(c->ell_entries, 256), 256, 0, k_values_f32, (const double *)vA,
                   (const double *)vB, c->ell_entries, fA, fB, hA, hB);
        APC_TRY(build_sorted_sweep(c));
    }
    return cuda_check(c, cudaGetLastError(), "ell");
}

}  // namespace apc

namespace apc {

// Times the stencil kernel at 2, 4 and 8 nodes per block on the current node
// set (after build_stencils) and keeps the fastest.  Every node's outputs are
// independent of the block shape, so the reruns rewrite identical values.
apcloud_status tune_stencils(apcloud_ctx *c, double *ms_out) {
    const int n = c->n_int;
    if (n == 0) return APCLOUD_OK;
    const int64_t dstride = ((int64_t)n + 31) / 32 * 32;
    int32_t *nbr = ptr<int32_t>(c->nbr), *msz = ptr<int32_t>(c->msz), *ring = ptr<int32_t>(c->ring);
    double *lap = ptr<double>(c->lap), *lapd = ptr<double>(c->lapd), *D = ptr<double>(c->D);
    double *rc = ptr<double>(c->rcond);
    unsigned *derr = ptr<unsigned>(c->derr);
    const double ext = c->P.hi[0] - c->P.lo[0];
    const double unit = ldexp(ext, -(KEY_DEPTH + 1));
    const double ec = exp(-c->P.weight_c);
    const double inv_1mec = 1.0 / (1.0 - ec);
    const int shapes[3] = {2, 4, 8};
    cudaEvent_t e0, e1;
    APC_CUDA(c, cudaEventCreate(&e0));
    APC_CUDA(c, cudaEventCreate(&e1));
    const unsigned mask = c->timer.mask;
    c->timer.mask = 0;
    double best = 1e30;
    int pick = c->wls_warps;
    apcloud_status st = APCLOUD_OK;
    for (int t = 0; t < 3 && st == APCLOUD_OK; ++t) {
        float ms = 0.f;
        for (int rep = 0; rep < 2 && st == APCLOUD_OK; ++rep) {
            st = cuda_check(c, cudaMemsetAsync(derr, 0, 4 * sizeof(unsigned), c->s), "autotune stencils");
            if (st != APCLOUD_OK) break;
            cudaEventRecord(e0, c->s);
            if (shapes[t] == 2)
                st = launch_stencil<2>(c, n, unit, ec, inv_1mec, nbr, msz, ring, lap, lapd, D, dstride, rc, derr);
            else if (shapes[t] == 4)
                st = launch_stencil<4>(c, n, unit, ec, inv_1mec, nbr, msz, ring, lap, lapd, D, dstride, rc, derr);
            else
                st = launch_stencil<8>(c, n, unit, ec, inv_1mec, nbr, msz, ring, lap, lapd, D, dstride, rc, derr);
            cudaEventRecord(e1, c->s);
            if (st == APCLOUD_OK) st = cuda_check(c, cudaEventSynchronize(e1), "autotune stencils");
            if (st == APCLOUD_OK) cudaEventElapsedTime(&ms, e0, e1);
        }
        if (st == APCLOUD_OK) st = check_device_errors(c);
        if (ms_out) ms_out[t] = ms;
        if (st == APCLOUD_OK && ms < best) { best = ms; pick = shapes[t]; }
    }
    c->timer.mask = mask;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == APCLOUD_OK) c->wls_warps = pick;
    return st;
}

}  // namespace apc

namespace apc {

// FP32/FP16 copies of the stored values again (after the FP64 values changed)
apcloud_status refresh_lowp(apcloud_ctx *c) {
    if (c->P.precision != 1 || c->ell_entries == 0) return APCLOUD_OK;
    APC_LAUNCH(c, K_ELL, div_up(c->ell_entries, 256), 256, 0, k_values_f32, (const double *)ptr<double>(c->ell_A),
               (const double *)ptr<double>(c->ell_B), c->ell_entries, ptr<float>(c->ell_A32), ptr<float>(c->ell_B32),
               ptr<__half>(c->ell_A16), ptr<__half>(c->ell_B16));
    APC_TRY(build_sorted_sweep(c));
    return cuda_check(c, cudaGetLastError(), "refresh_lowp");
}

namespace {

constexpr int SS_WIN = 256;   // rows per sorting window (8 slices)

// one block per window: rank the window's rows by stored width (descending,
// ties by row index), perm[slot] = row (-1 past the last row), and the width
// of each of the window's 8 slices
__global__ void __launch_bounds__(SS_WIN) k_ss_rank(const int32_t *__restrict__ msz, int n_int, int n_tot,
                                                  int32_t *__restrict__ perm, uint32_t *__restrict__ w) {
    __shared__ int wd[SS_WIN];
    __shared__ int sorted_w[SS_WIN];
    const int base = blockIdx.x * SS_WIN, t = threadIdx.x, r = base + t;
    const int my = r < n_int ? msz[r] + 1 : (r < n_tot ? 1 : -1);
    wd[t] = my;
    __syncthreads();
    int rank = 0;
    for (int k = 0; k < SS_WIN; ++k) {
        const int o = wd[k];
        rank += (o > my) || (o == my && k < t);
    }
    perm[base + rank] = my >= 0 ? r : -1;
    sorted_w[rank] = my > 0 ? my : 0;
    __syncthreads();
    if ((t & 31) == 0) w[blockIdx.x * (SS_WIN / 32) + (t >> 5)] = (uint32_t)sorted_w[t];   // max of the slice
}

// entry k of lane `lane` in a sorted slice of width w starting at entry sb:
// 4-entry chunks lane-major for the first 4 * floor(w / 4) columns, the rest
// slice-major
__device__ __forceinline__ int64_t ss_slot(int64_t sb, int w, int k, int lane) {
    const int kf = w & ~3;
    return (k < kf) ? sb + (int64_t)(k >> 2) * 128 + lane * 4 + (k & 3)
                    : sb + (int64_t)kf * 32 + (int64_t)(k - kf) * 32 + lane;
}

// copy every row's stored entries (in their order) into its slot of the sorted layout
__global__ void k_ss_fill(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                          const int32_t *__restrict__ col, const __half *__restrict__ hA, const __half *__restrict__ hB,
                          const float *__restrict__ fA, const float *__restrict__ fB,
                          const int32_t *__restrict__ perm, const uint32_t *__restrict__ w2,
                          const uint32_t *__restrict__ o2, int64_t nslot, int32_t *__restrict__ col2,
                          __half *__restrict__ A2, __half *__restrict__ B2, float *__restrict__ A4,
                          float *__restrict__ B4, uint32_t *__restrict__ col24) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslot) return;
    const int sl2 = (int)(s >> 5), lane2 = (int)(s & 31);
    const int64_t b2 = (int64_t)o2[sl2] * 32;
    const int wid2 = (int)w2[sl2];
    const int r = perm[s];
    int k = 0;
    if (r >= 0) {
        const int sl = r >> 5, lane = r & 31;
        const int w = (int)sw[sl];
        const int64_t base = (int64_t)soff[sl] * 32 + lane;
        for (; k < wid2 && k < w; ++k) {
            const int64_t e = base + (int64_t)k * 32, q = ss_slot(b2, wid2, k, lane2);
            col2[q] = col[e];
            A2[q] = hA[e];
            B2[q] = hB[e];
            A4[q] = fA[e];
            B4[q] = fB[e];
        }
    }
    for (; k < wid2; ++k) {   // padding: the row itself (or row 0) with value 0
        const int64_t q = ss_slot(b2, wid2, k, lane2);
        col2[q] = r >= 0 ? r : 0;
        A2[q] = __float2half(0.f);
        B2[q] = __float2half(0.f);
        A4[q] = 0.f;
        B4[q] = 0.f;
    }
    if (col24) {
        // the columns of the 4-entry chunks again, 24 bits each: a chunk's four
        // columns in three words, word p of lane l at 24 o + 96 j + 32 p + l
        const int64_t pw = (int64_t)o2[sl2] * 24 + lane2;
        for (int j = 0; j < (wid2 >> 2); ++j) {
            uint32_t cc[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) cc[t] = (uint32_t)col2[ss_slot(b2, wid2, 4 * j + t, lane2)];
            col24[pw + (int64_t)j * 96] = cc[0] | (cc[1] << 24);
            col24[pw + (int64_t)j * 96 + 32] = (cc[1] >> 8) | (cc[2] << 16);
            col24[pw + (int64_t)j * 96 + 64] = (cc[2] >> 16) | (cc[3] << 8);
        }
    }
}

}  // namespace

// The FP16 preconditioner sweeps stream the whole matrix 15 times per Arnoldi
// step; in 32-row slices of consecutive rows the slice width is that of its
// widest stencil and 14% of the stored entries are padding.  This copy orders
// the rows of every 256-row window by stored width (SELL-C-sigma, C = 32,
// sigma = 256): slices then hold rows of nearly equal width.  Within a slice
// the entries are grouped in 4-entry chunks per row (16-byte column loads),
// the last width % 4 columns as in the ELL.  Each row keeps its entries in
// their stored order, so a sweep on this copy gives the same bits as on the
// ELL.  The copy carries the FP16 values of the sweeps and the FP32 values of
// the Arnoldi products (also the same bits as the FP32 ELL product), and for
// the sweeps the chunks' columns packed to 24 bits (while n < 2^24): 20
// instead of 24 bytes per 4-entry chunk of a bandwidth-bound stream.
apcloud_status build_sorted_sweep(apcloud_ctx *c) {
    c->ss_ok = false;
    const int n = c->n_tot;
    if (n == 0) return APCLOUD_OK;
    const int nwin = div_up(n, SS_WIN);
    const int64_t nslot = (int64_t)nwin * SS_WIN;
    const int nsl2 = (int)(nslot / 32);
    int32_t *perm = ensure<int32_t>(c, c->ss_perm, nslot);
    uint32_t *w2 = ensure<uint32_t>(c, c->ss_w, nsl2 + 1), *o2 = ensure<uint32_t>(c, c->ss_o, nsl2 + 1);
    if (!perm || !w2 || !o2) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_ELL, nwin, SS_WIN, 0, k_ss_rank, (const int32_t *)ptr<int32_t>(c->msz), c->n_int, n, perm, w2);
    uint32_t *small = ptr<uint32_t>(c->dsmall);
    APC_TRY(scan_u32(c, w2, o2, nsl2, small + 13));
    uint32_t tot;
    APC_TRY(read_back(c, &tot, small + 13, sizeof tot));
    c->ss_entries = (int64_t)tot * 32;
    int32_t *col2 = ensure<int32_t>(c, c->ss_col, c->ss_entries + 1);
    __half *A2 = ensure<__half>(c, c->ss_A, c->ss_entries + 1), *B2 = ensure<__half>(c, c->ss_B, c->ss_entries + 1);
    float *A4 = ensure<float>(c, c->ss_A32, c->ss_entries + 1), *B4 = ensure<float>(c, c->ss_B32, c->ss_entries + 1);
    if (!col2 || !A2 || !B2 || !A4 || !B4) return APCLOUD_E_NOMEM;
    // 24-bit columns for the sweeps while every node index fits
    uint32_t *col24 = nullptr;
    c->ss_col24_ok = false;
    if (n < (1 << 24)) {
        col24 = ensure<uint32_t>(c, c->ss_col24, c->ss_entries / 4 * 3 + 1);
        if (!col24) return APCLOUD_E_NOMEM;
        c->ss_col24_ok = true;
    }
    APC_LAUNCH(c, K_ELL, div_up(nslot, 256), 256, 0, k_ss_fill, (const uint32_t *)ptr<uint32_t>(c->slice_w),
               (const uint32_t *)ptr<uint32_t>(c->slice_off), (const int32_t *)ptr<int32_t>(c->ell_col),
               (const __half *)ptr<__half>(c->ell_A16), (const __half *)ptr<__half>(c->ell_B16),
               (const float *)ptr<float>(c->ell_A32), (const float *)ptr<float>(c->ell_B32), (const int32_t *)perm,
               (const uint32_t *)w2, (const uint32_t *)o2, nslot, col2, A2, B2, A4, B4, col24);
    c->ss_ok = true;
    return cuda_check(c, cudaGetLastError(), "sorted sweep matrix");
}

}  // namespace apc

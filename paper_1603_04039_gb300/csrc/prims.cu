// prims.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// The tree construction of Section 4 sorts particles by Morton key; these are
// the primitives it (and the node ordering) is built from.  Both are written
// for determinism: the scan is a fixed two-phase tree (integer sums, exact in
// any order), the sort is stable.
#include "internal.cuh"

namespace apc {

namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_I = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_I;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive block scan of one value per thread; returns the block total in *total
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh, uint32_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = (lane < nw) ? sh[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (lane < nw) sh[lane] = wi - w;
        if (lane == nw - 1) sh[32] = wi;
    }
    __syncthreads();
    uint32_t r = inc - v + sh[wid];
    *total = sh[32];
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ blk) {
    __shared__ uint32_t sh[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        int64_t idx = base + (int64_t)i * SCAN_T + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    uint32_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

// Block b scans its tile and adds the sum of the block totals before it (it
// sums blk[0 .. b) itself, so no pass scans the block totals); the last
// block writes the grand total.  blk == null: a single block.
__global__ void k_scan_down(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
                            const uint32_t *__restrict__ blk, uint32_t *__restrict__ d_total) {
    __shared__ uint32_t sh[33];
    uint32_t pre = 0;
    if (blk) {
        uint32_t ps = 0;
        for (int i = threadIdx.x; i < (int)blockIdx.x; i += blockDim.x) ps += blk[i];
        block_excl_scan(ps, sh, &pre);
    }
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    uint32_t v[SCAN_I];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        int64_t idx = base + i;
        v[i] = (idx < n) ? in[idx] : 0u;
        s += v[i];
    }
    uint32_t tot;
    uint32_t e = block_excl_scan(s, sh, &tot) + pre;
    if (d_total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *d_total = pre + tot;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = e;
        e += v[i];
    }
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_T = 256;         // threads per block
constexpr int RS_I = 8;           // keys per thread
constexpr int RS_TILE = RS_T * RS_I;
constexpr int RS_BITS = 8;
constexpr int RS_BINS = 1 << RS_BITS;

__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, uint32_t mask,
                          uint32_t *__restrict__ hist, int nblk) {
    __shared__ uint32_t h[RS_BINS];
    for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int i = 0; i < RS_I; ++i) {
        int64_t idx = base + (int64_t)i * RS_T + threadIdx.x;
        if (idx < n) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += blockDim.x) hist[(int64_t)d * nblk + blockIdx.x] = h[d];
}

// Stable scatter: warp w of the block owns keys [w*256, w*256+256) of the
// tile and walks them 32 at a time in index order; equal digits inside a
// step are ranked by lane with __match_any_sync.  The tile is then ordered
// by digit in shared memory (same order inside a digit: warp, step, lane)
// and written out with consecutive threads on consecutive destinations, so
// the writes of a digit's run land together instead of one 8-byte key per
// lane in 32 places.
__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint64_t *__restrict__ kin,
                                                     const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                                                     uint32_t *__restrict__ vout, int64_t n, int shift, uint32_t mask,
                                                     const uint32_t *__restrict__ offs, int nblk) {
    static_assert(RS_T == RS_BINS, "one digit per thread in the block scan");
    __shared__ uint32_t cnt[RS_T / 32][RS_BINS];
    __shared__ uint32_t loc[RS_BINS], gof[RS_BINS], wtot[RS_T / 32];
    __shared__ uint64_t sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, tid = threadIdx.x;
    for (int i = tid; i < (RS_T / 32) * RS_BINS; i += blockDim.x) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    const int64_t base = tile0 + (int64_t)w * (32 * RS_I);
    const unsigned lt = (1u << lane) - 1u;
    uint64_t k[RS_I];
    uint32_t v[RS_I];
    uint32_t d[RS_I], r[RS_I];
#pragma unroll
    for (int i = 0; i < RS_I; ++i) {
        int64_t idx = base + i * 32 + lane;
        bool ok = idx < n;
        k[i] = ok ? kin[idx] : 0ull;
        v[i] = ok ? vin[idx] : 0u;
        d[i] = ok ? ((uint32_t)(k[i] >> shift) & mask) : RS_BINS;   // RS_BINS = not a key
        unsigned peers = __match_any_sync(0xffffffffu, d[i]);
        uint32_t before = 0;
        if (ok) before = cnt[w][d[i]];
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) cnt[w][d[i]] = before + __popc(peers);
        __syncwarp();
        r[i] = before + __popc(peers & lt);
    }
    __syncthreads();
    // digit tid: prefix over warps inside the block, the digit's total, and
    // the block's first destination for it
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < RS_T / 32; ++ww) {
        const uint32_t t = cnt[ww][tid];
        cnt[ww][tid] = tot;
        tot += t;
    }
    gof[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
    // exclusive scan of the digit totals over the block: where each digit's
    // run starts in the staged tile
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtot[w] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (int ww = 0; ww < w; ++ww) wbase += wtot[ww];
    loc[tid] = wbase + incl - tot;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_I; ++i) {
        if (d[i] < RS_BINS) {
            const uint32_t lp = loc[d[i]] + cnt[w][d[i]] + r[i];
            sk[lp] = k[i];
            sv[lp] = v[i];
        }
    }
    __syncthreads();
    const int m = (int)((n - tile0) < RS_TILE ? (n - tile0) : RS_TILE);
    for (int j = tid; j < m; j += RS_T) {
        const uint64_t kk = sk[j];
        const uint32_t dg = (uint32_t)(kk >> shift) & mask;
        const uint32_t dst = gof[dg] + (uint32_t)j - loc[dg];
        kout[dst] = kk;
        vout[dst] = sv[j];
    }
}

}  // namespace

apcloud_status scan_u32(apcloud_ctx *c, const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total) {
    if (n <= 0) {
        if (d_total) APC_CUDA(c, cudaMemsetAsync(d_total, 0, sizeof(uint32_t), c->s));
        return APCLOUD_OK;
    }
    int nb = div_up(n, SCAN_TILE);
    if (nb == 1) {
        APC_LAUNCH(c, K_TREE, 1, SCAN_T, 0, k_scan_down, in, out, n, (const uint32_t *)nullptr, d_total);
        return cuda_check(c, cudaGetLastError(), "scan");
    }
    uint32_t *blk = ensure<uint32_t>(c, c->scan_blk, nb);
    if (!blk) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_TREE, nb, SCAN_T, 0, k_scan_reduce, in, n, blk);
    APC_LAUNCH(c, K_TREE, nb, SCAN_T, 0, k_scan_down, in, out, n, (const uint32_t *)blk, d_total);
    return cuda_check(c, cudaGetLastError(), "scan");
}

apcloud_status radix_sort(apcloud_ctx *c, uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n,
                          int nbits, int *which) {
    *which = 0;
    if (n <= 1 || nbits <= 0) return APCLOUD_OK;
    int nblk = div_up(n, RS_TILE);
    int64_t nh = (int64_t)RS_BINS * nblk;
    uint32_t *hist = ensure<uint32_t>(c, c->flags, nh);
    uint32_t *offs = ensure<uint32_t>(c, c->scan, nh);
    if (!hist || !offs) return APCLOUD_E_NOMEM;
    uint64_t *ka = k0, *kb = k1;
    uint32_t *va = v0, *vb = v1;
    int cur = 0;
    for (int shift = 0; shift < nbits; shift += RS_BITS) {
        int bits = nbits - shift < RS_BITS ? nbits - shift : RS_BITS;
        uint32_t mask = (1u << bits) - 1u;
        APC_LAUNCH(c, K_SORT, nblk, RS_T, 0, k_rs_hist, ka, n, shift, mask, hist, nblk);
        APC_TRY(scan_u32(c, hist, offs, nh, nullptr));
        APC_LAUNCH(c, K_SORT, nblk, RS_T, 0, k_rs_scatter, ka, va, kb, vb, n, shift, mask, offs, nblk);
        account(c, K_SORT, 32.0 * n, 0.0);   // key read for the histogram, key+value read and write
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
        cur ^= 1;
    }
    *which = cur;
    return cuda_check(c, cudaGetLastError(), "radix_sort");
}

}  // namespace apc

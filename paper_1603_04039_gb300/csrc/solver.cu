// solver.cu -- Section 3.2 steps 1 and 2: charge deposit, sliced-ELL SpMV
// and restarted GMRES for the density system B rho~ = rho_M and the Poisson
// system A phi = c rho~.
//
// GMRES is right-preconditioned by Jacobi, M = diag(A), folded into the
// stored matrix values (column j scaled by 1/M_jj), so the Krylov iteration
// runs on Ahat u = b with x = M^-1 u and the residual of Ahat u is the
// residual of A x.  Each Arnoldi step is four kernels that keep all scalar
// bookkeeping on the device:
//   spmv      w = Ahat (wraw s), V_j = wraw s        (s = 1/||wraw||, normalisation fused)
//   dots      h1 = V_{0..j}^T w
//   upd_dots  w -= V h1 ; h2 = V^T w                 (classical Gram-Schmidt, second pass)
//   upd_norm  wraw = w - V h2 ; ||wraw|| ; Givens rotation and convergence test
// Grid reductions are finished by the last block to arrive (fixed summation
// order, so results are deterministic).  The host synchronises once per
// restart cycle.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include <climits>

#include "fpconv.cuh"
#include "internal.cuh"

namespace apc {

namespace {

constexpr int RT = 256;  // threads of the reduction kernels

// Block reduction of NJ per-thread values into sums held by threads 0..nj-1
// of the block (returned in `out`, valid for threadIdx.x < nj).
template <int NJ>
__device__ __forceinline__ void block_reduce_many(const double (&acc)[NJ], int nj, double *sm, double *out) {
    // sm: blockDim * NJ doubles laid out [k][t], then NJ * (blockDim / 32) segment sums
    const int t = threadIdx.x, B = blockDim.x;
#pragma unroll
    for (int k = 0; k < NJ; ++k)
        if (k < nj) sm[k * B + t] = acc[k];
    __syncthreads();
    // nj * (B / 32) threads each sum a segment of 32
    const int seg = B / 32;
    for (int q = t; q < nj * seg; q += B) {
        int k = q / seg, s = q % seg;
        const double *p = sm + k * B + s * 32;
        double v = 0.0;
#pragma unroll 8
        for (int i = 0; i < 32; ++i) v += p[i];
        sm[NJ * B + q] = v;
    }
    __syncthreads();
    if (t < nj) {
        double v = 0.0;
        for (int s = 0; s < seg; ++s) v += sm[NJ * B + t * seg + s];
        *out = v;
    }
    __syncthreads();
}

// Write the block partials, take a ticket; returns true in the last block.
__device__ __forceinline__ bool last_block(unsigned *ticket) {
    __shared__ bool amlast;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        amlast = (t == gridDim.x - 1);
    }
    __syncthreads();
    return amlast;
}

// Last block: deterministic sums over blocks of partial[b * 64 + k], k < nk.
// nk == 1 uses every thread on one value; otherwise each value gets a group
// of G = min(32, 2^floor(log2(blockDim / nk))) lanes of one warp, lane l of
// the group summing blocks l, l + G, ... (four chains in flight) before a
// shuffle tree over the group.  Result in out[k] (shared).
__device__ void final_sums(const double *partial, int nblk, int nk, double *sm, double *out) {
    const int t = threadIdx.x;
    if (nk == 1) {
        double v = 0.0;
        for (int b = t; b < nblk; b += blockDim.x) v += __ldcg(&partial[(int64_t)b * 64]);
        double a[1] = {v};
        double tot = 0.0;
        block_reduce_many<1>(a, 1, sm, &tot);
        if (t == 0) out[0] = tot;
    } else {
        int G = 32;
        while (G > 1 && G * nk > (int)blockDim.x) G >>= 1;
        const int k = t / G, l = t & (G - 1);
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        if (k < nk) {
            int b = l;
            for (; b + 3 * G < nblk; b += 4 * G) {
                v0 += __ldcg(&partial[(int64_t)b * 64 + k]);
                v1 += __ldcg(&partial[(int64_t)(b + G) * 64 + k]);
                v2 += __ldcg(&partial[(int64_t)(b + 2 * G) * 64 + k]);
                v3 += __ldcg(&partial[(int64_t)(b + 3 * G) * 64 + k]);
            }
            for (; b < nblk; b += G) v0 += __ldcg(&partial[(int64_t)b * 64 + k]);
        }
        double v = (v0 + v1) + (v2 + v3);
        for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
        if (k < nk && l == 0) out[k] = v;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- deposit
// Cell-indicator charge assignment (Section 5): Q_j = sum of the charges of
// the particles in leaf j, rho_M = Q_j / h_j^3; boundary rows copy the owner.
// Two passes, both coalesced on the particle side:
//  * k_charge_sort, four particles per thread in the caller's order: each
//    charge goes to its key-sorted position (recorded by the tree build); the
//    scattered stores land in an array that L2 keeps (evict-last hint) while
//    the caller's charges stream through (evict-first);
//  * k_deposit, one thread per leaf: the leaf's sorted charges (a contiguous
//    range) summed in order, one FP64 add per particle -- a warp-wide tree
//    reduction per leaf would cost 32 lanes of FP64 adds at every step on
//    this GPU's narrow FP64 pipe.
// The summation order is fixed, so the result does not depend on timing.
constexpr int CS_PER = 4;

__global__ void __launch_bounds__(256) k_charge_sort(const double *__restrict__ q, const int32_t *__restrict__ spos,
                                                     int64_t n, double *__restrict__ qs) {
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x) * CS_PER + threadIdx.x;
    uint64_t keep;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
    double v[CS_PER];
    int32_t p[CS_PER];
#pragma unroll
    for (int u = 0; u < CS_PER; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        if (i < n) {
            v[u] = __ldcs(q + i);
            p[u] = __ldcs(spos + i);
        }
    }
#pragma unroll
    for (int u = 0; u < CS_PER; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        if (i < n)
            asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(qs + p[u]), "d"(v[u]), "l"(keep)
                         : "memory");
    }
}

// rho_M = Q / h^3 with h = ext 2^-level: Q (1 / ext^3) 2^(3 level), the power
// of two built from its exponent bits (no FP64 division)
__global__ void __launch_bounds__(256) k_deposit(const double *__restrict__ qs, double qu,
                                                 const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                                                 const int4 *__restrict__ ic, int n_int, double inv_ext3,
                                                 double *__restrict__ rho_m) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_int) return;
    const int f = first[j], c = count[j];
    double Q;
    if (qs) {
        double s = 0.0;
        int i = f;
        const int e = f + c;
        for (; i + 4 <= e; i += 4) {
            const double a0 = __ldcs(qs + i), a1 = __ldcs(qs + i + 1), a2 = __ldcs(qs + i + 2),
                         a3 = __ldcs(qs + i + 3);
            s += a0;
            s += a1;
            s += a2;
            s += a3;
        }
        for (; i < e; ++i) s += __ldcs(qs + i);
        Q = s;
    } else {
        Q = (double)c * qu;
    }
    const double p3 = __longlong_as_double((long long)(1023 + 3 * ic[j].w) << 52);
    rho_m[j] = (Q * inv_ext3) * p3;
}

__global__ void k_bcopy(const int32_t *__restrict__ owner, int n_int, int n_bnd, double *__restrict__ v) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n_bnd) v[n_int + b] = v[owner[b]];
}

// ---------------------------------------------------------------- SpMV
// T is the value and vector type (double for the FP64 form and the outer
// residual of the mixed form, float for the inner iterations of the mixed
// form); per-thread sums run in T, every block or grid reduction in FP64.
// mode 0: y = Ahat x
// mode 1: y = Ahat x * s, vout[r] = x[r] * s, s = st->inv_norm (Arnoldi step)
// mode 2: y = b - Ahat x, ||y||^2 reduced into st (cycle start)
// mode 3: y = x + omega (b - Ahat x)   (damped Jacobi sweep of the polynomial
//         preconditioner, Ahat already carries the Jacobi scaling)
// mode 4: y = Ahat x, skipped once the cycle is done
// One row of the sliced ELL product, sum_k val[e_k] x[col[e_k]] in stored
// order.  U > 1 issues the column, value and gather loads of U entries
// before their multiply-adds (more bytes in flight per thread) while keeping
// the sequential summation order, so every U gives the same bits.
template <int U, class V, class X>
__device__ __forceinline__ X row_dot(const V *__restrict__ val, const int32_t *__restrict__ col,
                                     const X *__restrict__ x, int64_t base, int w) {
    X acc = (X)0;
    int k = 0;
    if (U > 1) {
        for (; k + U <= w; k += U) {
            int ci[U];
            X vv[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = base + (int64_t)(k + u) * 32;
                ci[u] = col[e];
                vv[u] = (X)val[e];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = x[ci[u]];
#pragma unroll
            for (int u = 0; u < U; ++u) acc = fma(vv[u], xv[u], acc);
        }
    }
    for (; k < w; ++k) {
        const int64_t e = base + (int64_t)k * 32;
        acc = fma((X)val[e], x[col[e]], acc);
    }
    return acc;
}

template <int U>
__device__ __forceinline__ float row_dot_h(const __half *__restrict__ val, const int32_t *__restrict__ col,
                                           const float *__restrict__ x, int64_t base, int w) {
    float acc = 0.f;
    int k = 0;
    if (U > 1) {
        for (; k + U <= w; k += U) {
            int ci[U];
            float vv[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = base + (int64_t)(k + u) * 32;
                ci[u] = col[e];
                vv[u] = __half2float(val[e]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = x[ci[u]];
#pragma unroll
            for (int u = 0; u < U; ++u) acc = fmaf(vv[u], xv[u], acc);
        }
    }
    for (; k < w; ++k) {
        const int64_t e = base + (int64_t)k * 32;
        acc = fmaf(__half2float(val[e]), x[col[e]], acc);
    }
    return acc;
}

// Resident blocks asked of the width-sorted row kernels: with two chunks in
// flight (U > 1) they fit 32 registers without spilling, so blocks of up to
// 256 threads fill the SM's 64 warps (left to itself the compiler takes more
// registers and fewer warps); the one-chunk form spills at 32 or 40
// registers and keeps the compiler's choice.  The FP32 product with packed
// columns needs 40 (48 warps).
#define SS_MINB(BS, U) (((U) > 1 && (BS) <= 256) ? 2048 / (BS) : 1)

// A row of the width-sorted sweep matrix.  A slice of width w stores its first
// 4 * floor(w / 4) columns lane-major in 4-entry chunks (chunk j of lane l at
// entries sbase + 128 j + 4 l .. + 3: one 16-byte column load and one 8-byte
// value load per chunk) and the last w % 4 columns slice-major as in the ELL.
// The entries are summed in the same order as row_dot_h.  The columns and
// values of the next chunk (U = 1) or the next two (U > 1) are in flight
// while a chunk's x entries are gathered.
template <int U>
__device__ __forceinline__ float row_dot_c(const __half *__restrict__ val, const int32_t *__restrict__ col,
                                           const float *__restrict__ x, int64_t sbase, int lane, int w) {
    constexpr int AH = (U > 1) ? 2 : 1;   // chunks whose loads are in flight
    const int4 z4 = make_int4(0, 0, 0, 0);
    const uint2 z2 = make_uint2(0u, 0u);
    float acc = 0.f;
    const int nch = w >> 2;
    const int4 *c4 = reinterpret_cast<const int4 *>(col + sbase) + lane;
    const uint2 *v4 = reinterpret_cast<const uint2 *>(val + sbase) + lane;
    int4 cq[AH];
    uint2 vq[AH];
#pragma unroll
    for (int a = 0; a < AH; ++a) {
        cq[a] = a < nch ? c4[(int64_t)a * 32] : z4;
        vq[a] = a < nch ? v4[(int64_t)a * 32] : z2;
    }
    for (int j = 0; j < nch; ++j) {
        const int4 c0 = cq[0];
        const uint2 v0 = vq[0];
#pragma unroll
        for (int a = 0; a + 1 < AH; ++a) {
            cq[a] = cq[a + 1];
            vq[a] = vq[a + 1];
        }
        cq[AH - 1] = (j + AH < nch) ? c4[(int64_t)(j + AH) * 32] : z4;
        vq[AH - 1] = (j + AH < nch) ? v4[(int64_t)(j + AH) * 32] : z2;
        const float x0 = x[c0.x], x1 = x[c0.y], x2 = x[c0.z], x3 = x[c0.w];
        const float2 f01 = __half22float2(*reinterpret_cast<const __half2 *>(&v0.x));
        const float2 f23 = __half22float2(*reinterpret_cast<const __half2 *>(&v0.y));
        acc = fmaf(f01.x, x0, acc);
        acc = fmaf(f01.y, x1, acc);
        acc = fmaf(f23.x, x2, acc);
        acc = fmaf(f23.y, x3, acc);
    }
    const int64_t tb = sbase + (int64_t)nch * 128 + lane;
    for (int k = 0; k < (w & 3); ++k) acc = fmaf(__half2float(val[tb + (int64_t)k * 32]), x[col[tb + (int64_t)k * 32]], acc);
    return acc;
}

// Programmatic dependent launch (APC_LAUNCH_PDL).  A kernel launched with the
// attribute may start while the kernel before it in the stream is running,
// once every block of that kernel has executed griddepcontrol.launch_dependents
// (or exited); griddepcontrol.wait returns once that kernel has completed and
// its writes are visible.  Without the attribute the wait returns at once.
// A sweep lets the next one start only after its own wait: so sweep i + 1
// never runs beside sweep i - 1, which read the buffer (through the SM's
// read-only cache) that sweep i rewrites and sweep i + 1 reads.  With the
// release at block start, small grids ran three sweeps side by side and
// sweep i + 1 read lines that sweep i - 1 had cached: wrong results.
__device__ __forceinline__ void grid_dep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// L2 eviction priority of the sweep's matrix loads.  The polynomial's sweeps
// follow one another, each reading the whole width-sorted matrix, so what
// the L2 still holds of one sweep's matrix the next one reads from there.
// A matrix larger than the L2 read as a plain cyclic stream leaves nothing
// to reuse (every line is evicted before its next read); with the slices
// past a threshold read as streaming data (ld.global.cs, __ldcs: lines
// allocated evict-first in L1 and L2), those lines replace one another and
// the slices below it stay resident.  The cache operator only steers the
// caches: the loads, and the results, are the same.

// row_dot_c with the chunks' columns packed to 24 bits: chunk j of lane l is
// three words at pbase + 96 j + 32 p + l (p = 0, 1, 2), read by three
// coalesced 4-byte loads; the last w % 4 columns stay in the 32-bit array.
// Same entries in the same order: the same bits as row_dot_c.  With EF the
// matrix loads are streaming loads; the two forms are separate
// instantiations, chosen per row, so each keeps the 32-register bound.  The
// grid-dependency wait (grid_dep_wait) comes after the first chunks' loads
// are issued and before any x is read; xr receives x[r].
template <int U, bool EF>
__device__ __forceinline__ float row_dot_c24(const __half *__restrict__ val, const int32_t *__restrict__ col,
                                             const uint32_t *__restrict__ col24, const float *__restrict__ x,
                                             int64_t sbase, int64_t pbase, int lane, int w, int r, float &xr) {
    constexpr int AH = (U > 1) ? 2 : 1;   // chunks whose loads are in flight
    float acc = 0.f;
    const int nch = w >> 2;
    const uint32_t *p0 = col24 + pbase + lane;
    const uint2 *v4 = reinterpret_cast<const uint2 *>(val + sbase) + lane;
    uint3 cq[AH];
    uint2 vq[AH];
    auto load = [&](int a, uint3 &c, uint2 &v) {
        if (a >= nch) {
            c = make_uint3(0u, 0u, 0u);
            v = make_uint2(0u, 0u);
        } else {
            const uint32_t *q = p0 + (int64_t)a * 96;
            const uint2 *u = v4 + (int64_t)a * 32;
            if (EF) {
                c = make_uint3(__ldcs(q), __ldcs(q + 32), __ldcs(q + 64));
                v = __ldcs(u);
            } else {
                c = make_uint3(q[0], q[32], q[64]);
                v = *u;
            }
        }
    };
#pragma unroll
    for (int a = 0; a < AH; ++a) load(a, cq[a], vq[a]);
    grid_dep_wait();
    xr = x[r];
    for (int j = 0; j < nch; ++j) {
        const uint3 c0 = cq[0];
        const uint2 v0 = vq[0];
#pragma unroll
        for (int a = 0; a + 1 < AH; ++a) {
            cq[a] = cq[a + 1];
            vq[a] = vq[a + 1];
        }
        load(j + AH, cq[AH - 1], vq[AH - 1]);
        const uint32_t i0 = c0.x & 0xFFFFFFu, i1 = (c0.x >> 24) | ((c0.y & 0xFFFFu) << 8),
                       i2 = (c0.y >> 16) | ((c0.z & 0xFFu) << 16), i3 = c0.z >> 8;
        const float x0 = x[i0], x1 = x[i1], x2 = x[i2], x3 = x[i3];
        const float2 f01 = __half22float2(*reinterpret_cast<const __half2 *>(&v0.x));
        const float2 f23 = __half22float2(*reinterpret_cast<const __half2 *>(&v0.y));
        acc = fmaf(f01.x, x0, acc);
        acc = fmaf(f01.y, x1, acc);
        acc = fmaf(f23.x, x2, acc);
        acc = fmaf(f23.y, x3, acc);
    }
    const int64_t tb = sbase + (int64_t)nch * 128 + lane;
    for (int k = 0; k < (w & 3); ++k) {
        const __half *hv = val + tb + (int64_t)k * 32;
        const int32_t *hc = col + tb + (int64_t)k * 32;
        const float fv = __half2float(EF ? __ldcs(hv) : *hv);
        acc = fmaf(fv, x[EF ? __ldcs(hc) : *hc], acc);
    }
    return acc;
}

// Rows of beams that have converged in a batch (both null outside batches):
// their Krylov vectors are zero, so the products skip them.
struct RowSkip {
    const int32_t *nbo;   // beam of every node
    const int *bdone;     // 1 once the beam has converged (or finished its cycle)
    const double *binv;   // per-beam Krylov spaces: 1 / ||w|| of each beam (null: st->inv_norm)
};

// BS: threads per block (one row each; mode 2 strides over the rows with a
// grid of resid_blocks(n) blocks of RT threads: one block per row block put
// 4118 same-address ticket atomics on the last-block test of a 1.05e6-row
// product).  U: loads issued ahead (row_dot).
template <int MODE, class T, int BS = RT, int U = 1>
__global__ void __launch_bounds__(BS) k_spmv(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                                             const int32_t *__restrict__ col, const T *__restrict__ val, int n,
                                             const T *__restrict__ x, T *__restrict__ y, T *__restrict__ vout,
                                             const T *__restrict__ b, GmresState *st, double *__restrict__ partial,
                                             RowSkip skip) {
    static_assert(MODE != 2 || BS == RT, "mode 2 partials are sized for RT-thread blocks");
    __shared__ double sm[MODE == 2 ? RT + RT / 32 + 8 : 1];
    if ((MODE == 1 || MODE == 3 || MODE == 4) && st->done) return;
    const int r = blockIdx.x * BS + threadIdx.x;
    if ((MODE == 1 || MODE == 3 || MODE == 4) && skip.nbo && r < n && skip.bdone[skip.nbo[r]]) {
        y[r] = (T)0;
        if (MODE == 1) vout[r] = (T)0;
        return;
    }
    T s = (T)1;
    if (MODE == 1) s = (skip.binv && r < n) ? (T)skip.binv[skip.nbo[r]] : (T)st->inv_norm;
    if (MODE == 3) s = (T)st->omega;
    T acc = (T)0;
    double yv = 0.0;
    if (MODE != 2 && r < n) {
        const int sl = r >> 5, lane = r & 31;
        const int w = (int)sw[sl];
        const int64_t base = (int64_t)soff[sl] * 32 + lane;
        acc = row_dot<U, T, T>(val, col, x, base, w);
        if (MODE == 0 || MODE == 4) y[r] = acc;
        if (MODE == 1) { y[r] = acc * s; vout[r] = x[r] * s; }
        if (MODE == 3) y[r] = fma(s, b[r] - acc, x[r]);
    }
    if (MODE == 2) {
        for (int rr = r; rr < n; rr += gridDim.x * BS) {
            const int sl = rr >> 5, lane = rr & 31;
            const int w = (int)sw[sl];
            const int64_t base = (int64_t)soff[sl] * 32 + lane;
            acc = row_dot<U, T, T>(val, col, x, base, w);
            const T t = b[rr] - acc;
            y[rr] = t;
            yv = fma((double)t, (double)t, yv);
        }
        double a[1] = {yv};
        double tot = 0.0;
        block_reduce_many<1>(a, 1, sm, &tot);
        if (threadIdx.x == 0) partial[blockIdx.x * 64] = tot;
        if (last_block(&st->ticket)) {
            __shared__ double fs[1];
            final_sums(partial, gridDim.x, 1, sm, fs);
            if (threadIdx.x == 0) {
                double beta = sqrt(fs[0]);
                st->beta = beta;
                st->g[0] = beta;
                for (int i = 1; i <= MAX_RESTART; ++i) st->g[i] = 0.0;
                st->jend = 0;
                st->done = (beta <= st->rtol * st->bnorm) ? 1 : 0;
                st->inv_norm = beta > 0.0 ? 1.0 / beta : 0.0;
                st->ticket = 0;
            }
        }
    }
}

// Damped Jacobi sweep of the polynomial preconditioner with FP16 matrix values
// and FP32 vectors: y = x + omega (b - Ahat x).  The preconditioner only
// steers the Krylov space (right preconditioning keeps the residual exact),
// so its 11-bit values cost convergence at most, never accuracy; they cut the
// sweep's traffic from 8 to 6 bytes per stored entry.
template <int BS, int U = 1>
__global__ void __launch_bounds__(BS) k_sweep_h(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                                                const int32_t *__restrict__ col, const __half *__restrict__ val,
                                                int n, const float *__restrict__ x, float *__restrict__ y,
                                                const float *__restrict__ b, const GmresState *__restrict__ st,
                                                RowSkip skip) {
    if (st->done) return;
    const int r = blockIdx.x * BS + threadIdx.x;
    if (r >= n) return;
    if (skip.nbo && skip.bdone[skip.nbo[r]]) {
        y[r] = 0.f;
        return;
    }
    const float om = (float)st->omega;
    const int sl = r >> 5, lane = r & 31;
    const int w = (int)sw[sl];
    const int64_t base = (int64_t)soff[sl] * 32 + lane;
    const float acc = row_dot_h<U>(val, col, x, base, w);
    y[r] = fmaf(om, b[r] - acc, x[r]);
}

// The same sweep on the width-sorted copy: thread = slot of a 32-slot slice,
// its row from the window's permutation (entries in the same order, so the
// same bits as k_sweep_h).  With packed columns and KS, slices stored from
// entry `keep` on are read as streaming (evict-first) loads; without KS
// (no threshold in effect) the kernel holds the ordinary form alone, whose
// code the branch slows by 5% (98 against 103 us per sweep of a 64-beam
// batch).
template <int BS, int U = 1, bool P24 = false, bool KS = false>
__global__ void __launch_bounds__(BS, SS_MINB(BS, U)) k_sweep_s(const int32_t *__restrict__ perm, const uint32_t *__restrict__ sw,
                                                const uint32_t *__restrict__ soff, const int32_t *__restrict__ col,
                                                const __half *__restrict__ val, int64_t nslot,
                                                const float *__restrict__ x, float *__restrict__ y,
                                                const float *__restrict__ b, const GmresState *__restrict__ st,
                                                RowSkip skip, const uint32_t *__restrict__ col24, int64_t keep) {
    // Sweeps after the first of a polynomial application are launched as
    // programmatic dependents of the sweep before them, whose y is their x:
    // a row reads its slice, b, the state and its first chunks before the
    // grid-dependency wait (none of them is written by a sweep), x and y only
    // after it.  The row's own loads are issued before the state is read (in
    // batches after the test for a converged beam, whose rows read nothing
    // more).
    const int64_t sl_ = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (sl_ >= nslot) return;
    const int r = perm[sl_];
    const int sl = (int)(sl_ >> 5), lane = (int)(sl_ & 31);
    const int w = (int)sw[sl];
    const int64_t sb = (int64_t)soff[sl] * 32;
    float br, xr;
    if (!skip.nbo) {
        br = b[r < 0 ? 0 : r];
        if (st->done || r < 0) return;
    } else {
        if (st->done || r < 0) return;
        if (skip.bdone[skip.nbo[r]]) {
            grid_dep_wait();
            y[r] = 0.f;
            return;
        }
        br = b[r];
    }
    const float om = (float)st->omega;
    float acc;
    if (!P24) {
        grid_dep_wait();
        xr = x[r];
        acc = row_dot_c<U>(val, col, x, sb, lane, w);
    } else if (KS && sb >= keep) {
        acc = row_dot_c24<U, true>(val, col, col24, x, sb, (int64_t)soff[sl] * 24, lane, w, r, xr);
    } else {
        acc = row_dot_c24<U, false>(val, col, col24, x, sb, (int64_t)soff[sl] * 24, lane, w, r, xr);
    }
    y[r] = fmaf(om, br - acc, xr);
}

// A row of the width-sorted copy with FP32 values: the same chunked layout as
// row_dot_c (one 16-byte column load and one 16-byte value load per 4-entry
// chunk, one or two chunks in flight), the entries in their stored order.
template <int U>
__device__ __forceinline__ float row_dot_cf(const float *__restrict__ val, const int32_t *__restrict__ col,
                                            const float *__restrict__ x, int64_t sbase, int lane, int w) {
    constexpr int AH = (U > 1) ? 2 : 1;
    const int4 z4 = make_int4(0, 0, 0, 0);
    const float4 zf = make_float4(0.f, 0.f, 0.f, 0.f);
    float acc = 0.f;
    const int nch = w >> 2;
    const int4 *c4 = reinterpret_cast<const int4 *>(col + sbase) + lane;
    const float4 *v4 = reinterpret_cast<const float4 *>(val + sbase) + lane;
    int4 cq[AH];
    float4 vq[AH];
#pragma unroll
    for (int a = 0; a < AH; ++a) {
        cq[a] = a < nch ? c4[(int64_t)a * 32] : z4;
        vq[a] = a < nch ? v4[(int64_t)a * 32] : zf;
    }
    for (int j = 0; j < nch; ++j) {
        const int4 c0 = cq[0];
        const float4 v0 = vq[0];
#pragma unroll
        for (int a = 0; a + 1 < AH; ++a) {
            cq[a] = cq[a + 1];
            vq[a] = vq[a + 1];
        }
        cq[AH - 1] = (j + AH < nch) ? c4[(int64_t)(j + AH) * 32] : z4;
        vq[AH - 1] = (j + AH < nch) ? v4[(int64_t)(j + AH) * 32] : zf;
        const float x0 = x[c0.x], x1 = x[c0.y], x2 = x[c0.z], x3 = x[c0.w];
        acc = fmaf(v0.x, x0, acc);
        acc = fmaf(v0.y, x1, acc);
        acc = fmaf(v0.z, x2, acc);
        acc = fmaf(v0.w, x3, acc);
    }
    const int64_t tb = sbase + (int64_t)nch * 128 + lane;
    for (int k = 0; k < (w & 3); ++k) acc = fmaf(val[tb + (int64_t)k * 32], x[col[tb + (int64_t)k * 32]], acc);
    return acc;
}

// row_dot_cf with the chunks' columns packed to 24 bits (see row_dot_c24):
// the same entries in the same order, the same bits
template <int U>
__device__ __forceinline__ float row_dot_cf24(const float *__restrict__ val, const int32_t *__restrict__ col,
                                              const uint32_t *__restrict__ col24, const float *__restrict__ x,
                                              int64_t sbase, int64_t pbase, int lane, int w) {
    constexpr int AH = (U > 1) ? 2 : 1;
    const uint3 z3 = make_uint3(0u, 0u, 0u);
    const float4 zf = make_float4(0.f, 0.f, 0.f, 0.f);
    float acc = 0.f;
    const int nch = w >> 2;
    const uint32_t *p0 = col24 + pbase + lane;
    const float4 *v4 = reinterpret_cast<const float4 *>(val + sbase) + lane;
    uint3 cq[AH];
    float4 vq[AH];
#pragma unroll
    for (int a = 0; a < AH; ++a) {
        cq[a] = a < nch ? make_uint3(p0[a * 96], p0[a * 96 + 32], p0[a * 96 + 64]) : z3;
        vq[a] = a < nch ? v4[(int64_t)a * 32] : zf;
    }
    for (int j = 0; j < nch; ++j) {
        const uint3 c0 = cq[0];
        const float4 v0 = vq[0];
#pragma unroll
        for (int a = 0; a + 1 < AH; ++a) {
            cq[a] = cq[a + 1];
            vq[a] = vq[a + 1];
        }
        const int64_t jn = (int64_t)(j + AH) * 96;
        cq[AH - 1] = (j + AH < nch) ? make_uint3(p0[jn], p0[jn + 32], p0[jn + 64]) : z3;
        vq[AH - 1] = (j + AH < nch) ? v4[(int64_t)(j + AH) * 32] : zf;
        const uint32_t i0 = c0.x & 0xFFFFFFu, i1 = (c0.x >> 24) | ((c0.y & 0xFFFFu) << 8),
                       i2 = (c0.y >> 16) | ((c0.z & 0xFFu) << 16), i3 = c0.z >> 8;
        const float x0 = x[i0], x1 = x[i1], x2 = x[i2], x3 = x[i3];
        acc = fmaf(v0.x, x0, acc);
        acc = fmaf(v0.y, x1, acc);
        acc = fmaf(v0.z, x2, acc);
        acc = fmaf(v0.w, x3, acc);
    }
    const int64_t tb = sbase + (int64_t)nch * 128 + lane;
    for (int k = 0; k < (w & 3); ++k) acc = fmaf(val[tb + (int64_t)k * 32], x[col[tb + (int64_t)k * 32]], acc);
    return acc;
}

// y = Ahat x on the width-sorted FP32 copy, skipped once the cycle is done
// (the Arnoldi product of k_spmv<4, float> with the same bits)
template <int BS, int U = 1, bool P24 = false>
__global__ void __launch_bounds__(BS, (P24 && SS_MINB(BS, U) > 1) ? 1536 / BS : SS_MINB(BS, U)) k_spmv_s(const int32_t *__restrict__ perm, const uint32_t *__restrict__ sw,
                                               const uint32_t *__restrict__ soff, const int32_t *__restrict__ col,
                                               const float *__restrict__ val, int64_t nslot,
                                               const float *__restrict__ x, float *__restrict__ y,
                                               const GmresState *__restrict__ st, RowSkip skip,
                                               const uint32_t *__restrict__ col24) {
    const int64_t sl_ = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (sl_ >= nslot) return;
    const int r = perm[sl_];
    const int sl = (int)(sl_ >> 5), lane = (int)(sl_ & 31);
    const int w = (int)sw[sl];
    const int64_t sb = (int64_t)soff[sl] * 32;
    if (st->done || r < 0) return;
    if (skip.nbo && skip.bdone[skip.nbo[r]]) {
        y[r] = 0.f;
        return;
    }
    y[r] = P24 ? row_dot_cf24<U>(val, col, col24, x, sb, (int64_t)soff[sl] * 24, lane, w)
               : row_dot_cf<U>(val, col, x, sb, lane, w);
}

// r = b - Ahat u and ||r||^2 (the restart residual, MODE 2 of k_spmv) on the
// width-sorted FP32 copy with 24-bit chunk columns: every row's entries in the
// same order as on the ELL (the same r), the norm summed over the sorted slots
// by a grid of resid_blocks blocks striding over them
template <int U>
__global__ void __launch_bounds__(RT) k_resid_s(const int32_t *__restrict__ perm, const uint32_t *__restrict__ sw,
                                                const uint32_t *__restrict__ soff, const int32_t *__restrict__ col,
                                                const float *__restrict__ val, const uint32_t *__restrict__ col24,
                                                int64_t nslot, const float *__restrict__ x, float *__restrict__ y,
                                                const float *__restrict__ b, GmresState *st,
                                                double *__restrict__ partial) {
    __shared__ double sm[RT + RT / 32 + 8];
    double yv = 0.0;
    for (int64_t sl_ = (int64_t)blockIdx.x * RT + threadIdx.x; sl_ < nslot; sl_ += (int64_t)gridDim.x * RT) {
        const int r = perm[sl_];
        if (r >= 0) {
            const int sl = (int)(sl_ >> 5), lane = (int)(sl_ & 31);
            const int w = (int)sw[sl];
            const int64_t sb = (int64_t)soff[sl] * 32;
            const float acc = row_dot_cf24<U>(val, col, col24, x, sb, (int64_t)soff[sl] * 24, lane, w);
            const float t = b[r] - acc;
            y[r] = t;
            yv = fma((double)t, (double)t, yv);
        }
    }
    double a[1] = {yv};
    double tot = 0.0;
    block_reduce_many<1>(a, 1, sm, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x * 64] = tot;
    if (last_block(&st->ticket)) {
        __shared__ double fs[1];
        final_sums(partial, gridDim.x, 1, sm, fs);
        if (threadIdx.x == 0) {
            const double beta = sqrt(fs[0]);
            st->beta = beta;
            st->g[0] = beta;
            for (int i = 1; i <= MAX_RESTART; ++i) st->g[i] = 0.0;
            st->jend = 0;
            st->done = (beta <= st->rtol * st->bnorm) ? 1 : 0;
            st->inv_norm = beta > 0.0 ? 1.0 / beta : 0.0;
            st->ticket = 0;
        }
    }
}

// Row-parallel products of the Arnoldi steps and sweeps at the block size the
// autotuner chose (64, 128, 256 or 512 threads).
#define APC_ROWS_BS_WITH(LAUNCH, c, kind, n, KERNEL_OF, ...)                                                \
    do {                                                                                                    \
        if ((c)->spmv_unroll == 4) {                                                                        \
            switch ((c)->spmv_bs) {                                                                         \
            case 64: LAUNCH(c, kind, div_up(n, 64), 64, 0, KERNEL_OF(64, 4), __VA_ARGS__); break;         \
            case 128: LAUNCH(c, kind, div_up(n, 128), 128, 0, KERNEL_OF(128, 4), __VA_ARGS__); break;     \
            case 512: LAUNCH(c, kind, div_up(n, 512), 512, 0, KERNEL_OF(512, 4), __VA_ARGS__); break;     \
            default: LAUNCH(c, kind, div_up(n, 256), 256, 0, KERNEL_OF(256, 4), __VA_ARGS__); break;      \
            }                                                                                               \
        } else {                                                                                            \
            switch ((c)->spmv_bs) {                                                                         \
            case 64: LAUNCH(c, kind, div_up(n, 64), 64, 0, KERNEL_OF(64, 1), __VA_ARGS__); break;         \
            case 128: LAUNCH(c, kind, div_up(n, 128), 128, 0, KERNEL_OF(128, 1), __VA_ARGS__); break;     \
            case 512: LAUNCH(c, kind, div_up(n, 512), 512, 0, KERNEL_OF(512, 1), __VA_ARGS__); break;     \
            default: LAUNCH(c, kind, div_up(n, 256), 256, 0, KERNEL_OF(256, 1), __VA_ARGS__); break;      \
            }                                                                                               \
        }                                                                                                   \
    } while (0)
#define APC_ROWS_BS(c, kind, n, KERNEL_OF, ...) APC_ROWS_BS_WITH(APC_LAUNCH, c, kind, n, KERNEL_OF, __VA_ARGS__)
#define APC_SPMV_BS(c, n, KERNEL_OF, ...) APC_ROWS_BS(c, K_SPMV, n, KERNEL_OF, __VA_ARGS__)
#define APC_SWEEP_BS(c, n, KERNEL_OF, ...) APC_ROWS_BS(c, K_SWEEP, n, KERNEL_OF, __VA_ARGS__)
#define APC_SWEEP_BS_PDL(c, n, KERNEL_OF, ...) APC_ROWS_BS_WITH(APC_LAUNCH_PDL, c, K_SWEEP, n, KERNEL_OF, __VA_ARGS__)
#define APC_SPMV1(B, U) (k_spmv<1, T, B, U>)
#define APC_SPMV3(B, U) (k_spmv<3, T, B, U>)
#define APC_SPMV4(B, U) (k_spmv<4, T, B, U>)
#define APC_SWEEPH(B, U) (k_sweep_h<B, U>)
#define APC_SWEEPS(B, U) (k_sweep_s<B, U, false>)
#define APC_SWEEPS24(B, U) (k_sweep_s<B, U, true>)
#define APC_SWEEPS24K(B, U) (k_sweep_s<B, U, true, true>)
#define APC_SPMVS(B, U) (k_spmv_s<B, U, false>)
#define APC_SPMVS24(B, U) (k_spmv_s<B, U, true>)


// ---------------------------------------------------------------- Gram-Schmidt passes
// Every arithmetic instruction does useful work on 32 lanes (GB300 runs FP64
// at 1/58 of FP32 and charges predicated-off lanes in full), and loads are
// 16-byte vectors so enough bytes are in flight to stream HBM in FP32:
//   * dot products V_k^T w: one warp per basis vector over a tile of w staged
//     in shared memory (lanes over 16-byte chunks of rows, coalesced);
//   * updates w -= V h: one thread per 16-byte chunk of rows, runtime loop
//     over k unrolled for independent loads.
// Work vectors are ldv long (a multiple of 32) with zero tails past n, so
// whole chunks are always in bounds and the tails add nothing.
constexpr int GT = 256;                    // threads per block of the row-parallel kernels
constexpr int DT = 512;                    // threads per block of the dot kernels (16 warps)
constexpr int GW = DT / 32;
constexpr int TILE = 2048;                 // rows staged per tile
constexpr int KPW = MAX_RESTART / GW;      // basis vectors per warp (<= 4)

template <class T> struct Vec;
template <> struct Vec<double> { typedef double2 type; static constexpr int n = 2; };
template <> struct Vec<float> { typedef float4 type; static constexpr int n = 4; };

__device__ __forceinline__ double dotv(double2 a, double2 b, double acc) { return fma(a.y, b.y, fma(a.x, b.x, acc)); }
__device__ __forceinline__ float dotv(float4 a, float4 b, float acc) {
    return fma(a.w, b.w, fma(a.z, b.z, fma(a.y, b.y, fma(a.x, b.x, acc))));
}
__device__ __forceinline__ double2 axpyv(double2 w, double2 v, double h) {
    return make_double2(fma(-v.x, h, w.x), fma(-v.y, h, w.y));
}
__device__ __forceinline__ float4 axpyv(float4 w, float4 v, float h) {
    return make_float4(fma(-v.x, h, w.x), fma(-v.y, h, w.y), fma(-v.z, h, w.z), fma(-v.w, h, w.w));
}
__device__ __forceinline__ double sumsq(double2 a, double acc) { return fma(a.y, a.y, fma(a.x, a.x, acc)); }
__device__ __forceinline__ float sumsq(float4 a, float acc) {
    return fma(a.w, a.w, fma(a.z, a.z, fma(a.y, a.y, fma(a.x, a.x, acc))));
}
__device__ __forceinline__ double2 fmav(double2 v, double y, double2 s) {
    return make_double2(fma(v.x, y, s.x), fma(v.y, y, s.y));
}
__device__ __forceinline__ float4 fmav(float4 v, float y, float4 s) {
    return make_float4(fma(v.x, y, s.x), fma(v.y, y, s.y), fma(v.z, y, s.z), fma(v.w, y, s.w));
}
__device__ __forceinline__ double2 addv(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float4 addv(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
template <class VT> __device__ __forceinline__ VT zerov();
template <> __device__ __forceinline__ double2 zerov<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float4 zerov<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// Dots of the staged tile ws with the basis vectors.  A basis of j1 <= GW / 2
// vectors splits the tile's chunks into GW / j1 parts, warp wid taking vector
// wid % j1 over part wid / j1 (every warp streams even for the first steps of
// a cycle); larger bases give warp wid the vectors wid, wid + GW, ...
template <class T>
__device__ __forceinline__ void tile_dots(const T *__restrict__ V, int64_t ldv, int64_t base, int lim, int j1,
                                          const T *ws, T (&acc)[KPW]) {
    typedef typename Vec<T>::type VT;
    constexpr int VN = Vec<T>::n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const VT *wv = reinterpret_cast<const VT *>(ws);
    const int parts = GW / j1;
    if (parts >= 2) {
        const int k = wid % j1, part = wid / j1;
        if (part < parts) {
            const VT *vk = reinterpret_cast<const VT *>(V + (int64_t)k * ldv + base);
            T a = acc[0];
#pragma unroll 8
            for (int c = lane + 32 * part; c < lim / VN; c += 32 * parts) a = dotv(__ldg(vk + c), wv[c], a);
            acc[0] = a;
        }
        return;
    }
#pragma unroll
    for (int kk = 0; kk < KPW; ++kk) {
        const int k = wid + GW * kk;
        if (k < j1) {   // uniform across the warp
            const VT *vk = reinterpret_cast<const VT *>(V + (int64_t)k * ldv + base);
            T a = acc[kk];
#pragma unroll 8
            for (int c = lane; c < lim / VN; c += 32) a = dotv(__ldg(vk + c), wv[c], a);
            acc[kk] = a;
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Hessenberg column j (h1 + h2 over its first j + 1 rows, h_{j+1,j} =
// sqrt(hn2)), its Givens rotations and the stopping test (Saad, Algorithms
// 6.9 / 6.10), run by the whole last block of a reduction: the inputs are
// loaded in parallel into shared memory, the serial part runs in thread 0
// (the only thread whose hn2 is read), the column is written back in
// parallel (dependent global round trips in one thread would dominate the
// kernel).  In a captured cycle it also sets the condition of the next
// step's body (set_next): 1 while the stopping test has not passed.
__device__ void arnoldi_tail(GmresState *st, int j, const double *h2s, double hn2, cudaGraphConditionalHandle next,
                             int set_next) {
    __shared__ double col[MAX_RESTART + 1], csj[MAX_RESTART], snj[MAX_RESTART];
    const int tid = threadIdx.x;
    if (tid <= j) col[tid] = __ldcg(&st->h1[tid]) + h2s[tid];
    if (tid < j) {
        csj[tid] = __ldcg(&st->cs[tid]);
        snj[tid] = __ldcg(&st->sn[tid]);
    }
    __syncthreads();
    if (tid == 0) {
        const double hn = sqrt(hn2 > 0.0 ? hn2 : 0.0);
        col[j + 1] = hn;
        for (int i = 0; i < j; ++i) {
            const double a = col[i], bb = col[i + 1];
            col[i] = csj[i] * a + snj[i] * bb;
            col[i + 1] = -snj[i] * a + csj[i] * bb;
        }
        const double a = col[j], bb = col[j + 1];
        const double den = sqrt(a * a + bb * bb);
        const double cj = den != 0.0 ? a / den : 1.0, sj = den != 0.0 ? bb / den : 0.0;
        st->cs[j] = cj;
        st->sn[j] = sj;
        col[j] = den;
        col[j + 1] = 0.0;
        const double gj = __ldcg(&st->g[j]);
        st->g[j + 1] = -sj * gj;
        st->g[j] = cj * gj;
        st->jend = j + 1;
        if (fabs(sj * gj) <= st->rtol * st->bnorm || hn == 0.0) st->done = 1;
        st->inv_norm = hn > 0.0 ? 1.0 / hn : 0.0;
        st->ticket = 0;
        if (set_next) cudaGraphSetConditional(next, st->done ? 0u : 1u);
    }
    __syncthreads();
    if (tid <= j + 1) st->H[tid * MAX_RESTART + j] = col[tid];
}

// PASS 0: h1 = V^T w.   PASS 1: w -= V h1, then h2 = V^T w.   (nrow = ldv)
// PASS 2: PASS 1 and ||w||^2 in the same sweep (j + 1 < 64); the last block
// closes the Arnoldi step with ||w - V h2||^2 = ||w||^2 - ||h2||^2 (V has
// orthonormal columns and h2 = V^T w), so that the second update and the
// normalisation can run as one pass at the start of the next step
// (k_gs_update_normalize).
template <int PASS, class T>
__global__ void __launch_bounds__(DT, 2) k_gs_dots(const T *__restrict__ V, int64_t ldv, int nrow, int j,
                                                T *__restrict__ w, GmresState *st, double *__restrict__ partial,
                                                const uint8_t *__restrict__ tact, cudaGraphConditionalHandle next,
                                                int set_next) {
    typedef typename Vec<T>::type VT;
    constexpr int VN = Vec<T>::n;
    __shared__ __align__(16) T ws[TILE];
    __shared__ T hs[MAX_RESTART];
    __shared__ double red[MAX_RESTART + 1];
    __shared__ double wsum[GW];
    __shared__ double sm[DT + DT / 32 + 8];
    __shared__ double fs[MAX_RESTART + 1];
    if (st->done) return;
    const int j1 = j + 1, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nk = j1 + (PASS == 2 ? 1 : 0);
    if (PASS >= 1 && tid < j1) hs[tid] = (T)st->h1[tid];
    __syncthreads();
    T acc[KPW];
#pragma unroll
    for (int kk = 0; kk < KPW; ++kk) acc[kk] = (T)0;
    T sq = (T)0;
    VT *wsv = reinterpret_cast<VT *>(ws);
    for (int64_t base = (int64_t)blockIdx.x * TILE; base < nrow; base += (int64_t)gridDim.x * TILE) {
        if (tact && !tact[base / TILE]) continue;   // every row of the tile is zero (converged beams)
        const int lim = (int)((nrow - base) < TILE ? (nrow - base) : TILE);
        VT *wg = reinterpret_cast<VT *>(w + base);
        if (PASS == 0) {
            for (int cix = tid; cix < lim / VN; cix += DT) wsv[cix] = wg[cix];
        } else {
            for (int cix = tid; cix < lim / VN; cix += DT) {
                VT wi = wg[cix];
                const T *vb = V + base;
#pragma unroll 8
                for (int k = 0; k < j1; ++k)
                    wi = axpyv(wi, __ldg(reinterpret_cast<const VT *>(vb + (int64_t)k * ldv) + cix), hs[k]);
                wg[cix] = wi;
                wsv[cix] = wi;
                if (PASS == 2) sq = sumsq(wi, sq);
            }
        }
        __syncthreads();
        tile_dots<T>(V, ldv, base, lim, j1, ws, acc);
        __syncthreads();
    }
    if (GW / j1 >= 2) {
        // one partial per warp; the parts of each vector summed in a fixed order
        const double v = warp_sum((double)acc[0]);
        if (lane == 0) wsum[wid] = v;
        __syncthreads();
        if (tid < j1) {
            double s = 0.0;
            for (int part = 0; part < GW / j1; ++part) s += wsum[tid + j1 * part];
            red[tid] = s;
        }
    } else {
#pragma unroll
        for (int kk = 0; kk < KPW; ++kk) {
            const int k = wid + GW * kk;
            if (k < j1) {
                double v = warp_sum((double)acc[kk]);
                if (lane == 0) red[k] = v;
            }
        }
    }
    if (PASS == 2) {
        __syncthreads();
        const double v = warp_sum((double)sq);
        if (lane == 0) wsum[wid] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < GW; ++q) s += wsum[q];
            red[j1] = s;
        }
    }
    __syncthreads();
    if (tid < nk) partial[(int64_t)blockIdx.x * 64 + tid] = red[tid];
    if (!last_block(&st->ticket)) return;
    final_sums(partial, gridDim.x, nk, sm, fs);
    if (PASS == 2) {
        if (tid < j1) st->h2[tid] = fs[tid];
        double hn2 = 0.0;
        if (tid == 0) {
            double h2sq = 0.0;
            for (int k = 0; k < j1; ++k) h2sq = fma(fs[k], fs[k], h2sq);
            hn2 = fs[j1] - h2sq;
        }
        arnoldi_tail(st, j, fs, hn2, next, set_next);
        return;
    }
    if (tid < j1) {
        if (PASS == 0) st->h1[tid] = fs[tid];
        else st->h2[tid] = fs[tid];
    }
    if (tid == 0) st->ticket = 0;
}

// wraw = w - V h2 ; ||wraw||^2 ; Hessenberg column, Givens rotation and
// convergence test in the last block (arnoldi_tail)
template <class T>
__global__ void __launch_bounds__(GT) k_gs_norm(const T *__restrict__ V, int64_t ldv, int nrow, int j,
                                                const T *__restrict__ w, T *__restrict__ wraw, GmresState *st,
                                                double *__restrict__ partial, const uint8_t *__restrict__ tact,
                                                cudaGraphConditionalHandle next, int set_next) {
    typedef typename Vec<T>::type VT;
    constexpr int VN = Vec<T>::n;
    __shared__ T hs[MAX_RESTART];
    __shared__ double sm[RT + RT / 32 + 8];
    __shared__ double fs[1];
    if (st->done) return;
    const int j1 = j + 1, tid = threadIdx.x;
    if (tid < j1) hs[tid] = (T)st->h2[tid];
    __syncthreads();
    T sq = (T)0;
    const int nch = nrow / VN;
    const VT *wv = reinterpret_cast<const VT *>(w);
    VT *ov = reinterpret_cast<VT *>(wraw);
    for (int cix = blockIdx.x * GT + tid; cix < nch; cix += gridDim.x * GT) {
        if (tact && !tact[(int64_t)cix * VN / TILE]) continue;
        VT wi = wv[cix];
#pragma unroll 8
        for (int k = 0; k < j1; ++k)
            wi = axpyv(wi, __ldg(reinterpret_cast<const VT *>(V + (int64_t)k * ldv) + cix), hs[k]);
        ov[cix] = wi;
        sq = sumsq(wi, sq);
    }
    double a1[1] = {(double)sq};
    double tot = 0.0;
    block_reduce_many<1>(a1, 1, sm, &tot);
    if (tid == 0) partial[(int64_t)blockIdx.x * 64] = tot;
    if (!last_block(&st->ticket)) return;
    final_sums(partial, gridDim.x, 1, sm, fs);
    __shared__ double h2s[MAX_RESTART];
    if (tid <= j) h2s[tid] = __ldcg(&st->h2[tid]);
    __syncthreads();
    arnoldi_tail(st, j, h2s, fs[0], next, set_next);
}

// u += V y with H y = g solved (upper triangular, jend x jend) in every block
template <class T>
__global__ void __launch_bounds__(GT) k_cycle_end(const T *__restrict__ V, int64_t ldv, int nrow, T *__restrict__ u,
                                                  const GmresState *__restrict__ st) {
    typedef typename Vec<T>::type VT;
    constexpr int VN = Vec<T>::n;
    __shared__ T ys[MAX_RESTART];
    const int je = st->jend;
    if (threadIdx.x == 0) {
        const int M = MAX_RESTART;
        double yd[MAX_RESTART];
        for (int k = je - 1; k >= 0; --k) {
            double s = st->g[k];
            for (int l = k + 1; l < je; ++l) s -= st->H[k * M + l] * yd[l];
            yd[k] = s / st->H[k * M + k];
            ys[k] = (T)yd[k];
        }
    }
    __syncthreads();
    if (je == 0) return;
    VT *uv = reinterpret_cast<VT *>(u);
    for (int cix = blockIdx.x * GT + threadIdx.x; cix < nrow / VN; cix += gridDim.x * GT) {
        VT s = zerov<VT>();
#pragma unroll 8
        for (int k = 0; k < je; ++k) s = fmav(__ldg(reinterpret_cast<const VT *>(V + (int64_t)k * ldv) + cix), ys[k], s);
        uv[cix] = addv(uv[cix], s);
    }
}

template <class T>
__global__ void __launch_bounds__(RT) k_norm2(const T *__restrict__ x, int n, GmresState *st,
                                              double *__restrict__ partial) {
    __shared__ double sm[RT + RT / 32 + 8];
    double s = 0.0;
    for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) s = fma((double)x[i], (double)x[i], s);
    double a[1] = {s};
    double tot = 0.0;
    block_reduce_many<1>(a, 1, sm, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x * 64] = tot;
    if (last_block(&st->ticket)) {
        __shared__ double fs[1];
        final_sums(partial, gridDim.x, 1, sm, fs);
        if (threadIdx.x == 0) {
            st->bnorm = sqrt(fs[0]);
            st->ticket = 0;
        }
    }
}

__global__ void k_mul(double *__restrict__ out, const double *__restrict__ a, const double *__restrict__ d, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a ? a[i] * d[i] : 0.0;
}

__global__ void k_div(double *__restrict__ out, const double *__restrict__ a, const double *__restrict__ d, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] / d[i];
}

// V_j = wraw / ||wraw||, z = omega V_j (first sweep of the polynomial from z = 0)
template <class T>
__global__ void k_normalize_first(const T *__restrict__ wraw, T *__restrict__ vj, T *__restrict__ z, int n,
                                  const GmresState *__restrict__ st) {
    if (st->done) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        T v = wraw[i] * (T)st->inv_norm;
        vj[i] = v;
        z[i] = (T)st->omega * v;
    }
}

// Start of Arnoldi step j >= 1 after a PASS 2 step: V_j = (w - V h2) / h_{j,j-1}
// over the j previous basis vectors, z = omega V_j (first sweep of the
// polynomial from z = 0)
template <class T>
__global__ void __launch_bounds__(GT) k_gs_update_normalize(const T *__restrict__ V, int64_t ldv, int nrow, int j,
                                                            const T *__restrict__ w, T *__restrict__ vj,
                                                            T *__restrict__ z, const GmresState *__restrict__ st) {
    typedef typename Vec<T>::type VT;
    constexpr int VN = Vec<T>::n;
    __shared__ T hs[MAX_RESTART];
    if (st->done) return;
    if (threadIdx.x < j) hs[threadIdx.x] = (T)st->h2[threadIdx.x];
    __syncthreads();
    const T inv = (T)st->inv_norm, om = (T)st->omega;
    const VT *wv = reinterpret_cast<const VT *>(w);
    VT *vv = reinterpret_cast<VT *>(vj), *zv = reinterpret_cast<VT *>(z);
    for (int cix = blockIdx.x * GT + threadIdx.x; cix < nrow / VN; cix += gridDim.x * GT) {
        VT wi = wv[cix];
#pragma unroll 8
        for (int k = 0; k < j; ++k)
            wi = axpyv(wi, __ldg(reinterpret_cast<const VT *>(V + (int64_t)k * ldv) + cix), hs[k]);
        const VT v = fmav(wi, inv, zerov<VT>());
        vv[cix] = v;
        zv[cix] = fmav(v, om, zerov<VT>());
    }
}

// ---------------------------------------------------------------- DCGS2
// Classical Gram-Schmidt with delayed reorthogonalisation (DCGS2: Bielich,
// Langou, Thomas, Swirydowicz, Yamazaki and Boman, Parallel Computing 112,
// 2022), one grid reduction and two passes over the basis per Arnoldi step
// where CGS2 takes two reductions and three passes.  Slot j of V holds the
// tentative vector q_j: w_{j-1} minus its first projection, scaled by an
// estimate nut_j of its norm.  Z_j = p(Ahat) q_j and w = Ahat Z_j, so the
// flexible relation Ahat Z = V H holds for whatever q_j is; the second
// projection of q_j (s = V^T q_j) is taken at step j together with the first
// projection of w, and finishes column j - 1 of H.

// tile_dots for two staged tiles at once: acq against qs, acw against ws
// (nv basis vectors, same work split as tile_dots)
template <class T>
__device__ __forceinline__ void tile_dots2(const T *__restrict__ V, int64_t ldv, int64_t base, int lim, int nv,
                                           const T *qs, const T *ws, T (&acq)[KPW], T (&acw)[KPW]) {
    typedef typename Vec<T>::type VT;
    constexpr int VN = Vec<T>::n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const VT *qv = reinterpret_cast<const VT *>(qs);
    const VT *wv = reinterpret_cast<const VT *>(ws);
    const int parts = GW / nv;
    if (parts >= 2) {
        const int k = wid % nv, part = wid / nv;
        if (part < parts) {
            const VT *vk = reinterpret_cast<const VT *>(V + (int64_t)k * ldv + base);
            T a = acq[0], b = acw[0];
#pragma unroll 4
            for (int c = lane + 32 * part; c < lim / VN; c += 32 * parts) {
                const VT x = __ldg(vk + c);
                a = dotv(x, qv[c], a);
                b = dotv(x, wv[c], b);
            }
            acq[0] = a;
            acw[0] = b;
        }
        return;
    }
#pragma unroll
    for (int kk = 0; kk < KPW; ++kk) {
        const int k = wid + GW * kk;
        if (k < nv) {   // uniform across the warp
            const VT *vk = reinterpret_cast<const VT *>(V + (int64_t)k * ldv + base);
            T a = acq[kk], b = acw[kk];
#pragma unroll 4
            for (int c = lane; c < lim / VN; c += 32) {
                const VT x = __ldg(vk + c);
                a = dotv(x, qv[c], a);
                b = dotv(x, wv[c], b);
            }
            acq[kk] = a;
            acw[kk] = b;
        }
    }
}

__device__ __forceinline__ void givens(double a, double b, double &c, double &s, double &r) {
    r = sqrt(a * a + b * b);
    c = r != 0.0 ? a / r : 1.0;
    s = r != 0.0 ? b / r : 0.0;
}

// Compensated FP32 sums for the reductions of k_dcgs_dots: a value is a pair
// (s, e) whose sum is the value; adding two pairs keeps the rounding error of
// s_a + s_b in e (TwoSum, Knuth, TAOCP vol. 2, 4.2.2), so the block and grid
// sums carry about twice the FP32 precision on the FP32 pipe.  GB300 issues
// one FP64 lane pair per clock and SM: the FP64 shuffle trees and block sums
// they replace cost ~15 us of a ~50 us kernel.
struct F2 {
    float s, e;
};
__device__ __forceinline__ F2 f2add(F2 a, F2 b) {
    const float s = a.s + b.s;
    const float bb = s - a.s;
    const float err = (a.s - (s - bb)) + (b.s - bb);
    return F2{s, (a.e + b.e) + err};
}
__device__ __forceinline__ F2 warp_sum_f2(F2 v, int width = 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        if (o < width) v = f2add(v, F2{__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.e, o)});
    return v;
}
__device__ __forceinline__ double f2_value(F2 v) { return f32_to_f64_int(v.s) + f32_to_f64_int(v.e); }

// final_sums for F2 partials (float2 in the 8-byte slots partial[b * 64 + k]):
// each value gets a group of G = min(32, 2^floor(log2(blockDim / nk))) lanes,
// lane l of the group adding blocks l, l + G, ... before a shuffle tree over
// the group; out[k] (shared) in FP64.
__device__ void final_sums_f2(const double *partial, int nblk, int nk, double *out) {
    const int t = threadIdx.x;
    int G = 32;
    while (G > 1 && G * nk > (int)blockDim.x) G >>= 1;
    const int k = t / G, l = t & (G - 1);
    F2 a{0.f, 0.f}, b{0.f, 0.f};
    if (k < nk) {
        const float2 *p2 = reinterpret_cast<const float2 *>(partial);
        int bl = l;
        for (; bl + G < nblk; bl += 2 * G) {
            const float2 x = __ldcg(&p2[(int64_t)bl * 64 + k]), y = __ldcg(&p2[(int64_t)(bl + G) * 64 + k]);
            a = f2add(a, F2{x.x, x.y});
            b = f2add(b, F2{y.x, y.y});
        }
        for (; bl < nblk; bl += G) {
            const float2 x = __ldcg(&p2[(int64_t)bl * 64 + k]);
            a = f2add(a, F2{x.x, x.y});
        }
    }
    F2 v = f2add(a, b);
    for (int o = G >> 1; o > 0; o >>= 1)
        v = f2add(v, F2{__shfl_xor_sync(0xffffffffu, v.s, o, G), __shfl_xor_sync(0xffffffffu, v.e, o, G)});
    if (k < nk && l == 0) out[k] = f2_value(v);
    __syncthreads();
}

// Last block of k_dcgs_dots.  fs holds s (j values), t (j values), alpha =
// q_j.q_j, beta = q_j.w, gamma = w.w.  With v_j = (q_j - V s) / nu:
//   nu = sqrt(alpha - s.s);
//   w_{j-1} = V (h_{j-1} + nut_j s) + nut_j nu v_j    (column j - 1, final);
//   tau = v_j.w = (beta - s.t) / nu, h_j = (t, tau)    (first projection of w);
//   nut_{j+1}^2 = ||w - V h_j||^2 = gamma - t.t - tau^2 (next estimate).
// Column j - 1 gets its rotation for good (its g[j - 1] comes back from
// gpre); column j enters with h_{j+1,j} = nut_{j+1} and a tentative rotation
// whose |g[j + 1]| is the stopping test (Saad, Algorithms 6.9 / 6.10); step
// j + 1 replaces both.  A cycle that stops here keeps the tentative column:
// the cycle end solves with it and the restart computes the true residual.
__device__ void dcgs_tail(GmresState *st, int j, const double *fs, cudaGraphConditionalHandle next,
                          int set_next) {
    __shared__ double colp[MAX_RESTART + 1], colc[MAX_RESTART + 2], csj[MAX_RESTART], snj[MAX_RESTART];
    __shared__ double hp[MAX_RESTART + 1];
    __shared__ double sums[3], gjs, taus;
    const int tid = threadIdx.x;
    const double *s = fs, *t = fs + j;
    if (tid < j) {
        csj[tid] = __ldcg(&st->cs[tid]);
        snj[tid] = __ldcg(&st->sn[tid]);
        hp[tid] = __ldcg(&st->h1[tid]);
    }
    if (tid < 32) {   // s.s, s.t, t.t over the lanes of warp 0 (j < 32)
        double a = 0.0, b = 0.0, c = 0.0;
        if (tid < j) {
            a = s[tid] * s[tid];
            b = s[tid] * t[tid];
            c = t[tid] * t[tid];
        }
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
        if (tid == 0) {
            sums[0] = a;
            sums[1] = b;
            sums[2] = c;
        }
    }
    __syncthreads();
    const double alpha = fs[2 * j], beta = fs[2 * j + 1], gamma = fs[2 * j + 2];
    // column j - 1 (thread 0) and the rotations of column j before the last
    // one (thread 32) side by side
    if ((tid == 0 && j > 0) || tid == 32) {
        const double nu = j > 0 ? sqrt(fmax(alpha - sums[0], 0.0)) : 1.0;
        if (tid == 0) {
            const double nut = __ldcg(&st->nut);
            for (int k = 0; k < j; ++k) colp[k] = fma(nut, s[k], hp[k]);
            colp[j] = nut * nu;
            for (int i = 0; i + 1 < j; ++i) {
                const double a = colp[i], b = colp[i + 1];
                colp[i] = csj[i] * a + snj[i] * b;
                colp[i + 1] = -snj[i] * a + csj[i] * b;
            }
            double c, sv, r;
            givens(colp[j - 1], colp[j], c, sv, r);
            csj[j - 1] = c;
            snj[j - 1] = sv;
            st->cs[j - 1] = c;
            st->sn[j - 1] = sv;
            colp[j - 1] = r;
            colp[j] = 0.0;
            const double gp = __ldcg(&st->gpre);
            st->g[j - 1] = c * gp;
            gjs = -sv * gp;
        } else {
            const double tau = nu > 0.0 ? (beta - sums[1]) / nu : 0.0;
            taus = tau;
            for (int k = 0; k < j; ++k) colc[k] = t[k];
            colc[j] = tau;
            colc[j + 1] = sqrt(fmax(gamma - sums[2] - tau * tau, 0.0));
            for (int i = 0; i + 1 < j; ++i) {
                const double a = colc[i], b = colc[i + 1];
                colc[i] = csj[i] * a + snj[i] * b;
                colc[i + 1] = -snj[i] * a + csj[i] * b;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        const double nu = j > 0 ? sqrt(fmax(alpha - sums[0], 0.0)) : 1.0;
        const double nut1 = colc[j + 1];
        if (j > 0) {   // the rotation of column j - 1, final now
            const double a = colc[j - 1], b = colc[j];
            colc[j - 1] = csj[j - 1] * a + snj[j - 1] * b;
            colc[j] = -snj[j - 1] * a + csj[j - 1] * b;
        }
        double c, sv, r;
        givens(colc[j], colc[j + 1], c, sv, r);
        st->cs[j] = c;
        st->sn[j] = sv;
        colc[j] = r;
        colc[j + 1] = 0.0;
        const double gj = j > 0 ? gjs : __ldcg(&st->g[0]);
        st->gpre = gj;
        st->g[j] = c * gj;
        st->g[j + 1] = -sv * gj;
        st->jend = j + 1;
        st->nu = nu;
        st->inu = nu > 0.0 ? 1.0 / nu : 0.0;
        st->nut = nut1;
        st->inv_norm = nut1 > 0.0 ? 1.0 / nut1 : 0.0;
        if (fabs(sv * gj) <= st->rtol * st->bnorm || nut1 == 0.0 || nu == 0.0) st->done = 1;
        st->ticket = 0;
        if (set_next) cudaGraphSetConditional(next, st->done ? 0u : 1u);
    }
    __syncthreads();
    constexpr int M = MAX_RESTART;
    if (j > 0 && tid <= j) st->H[tid * M + j - 1] = colp[tid];
    if (tid <= j + 1) st->H[tid * M + j] = colc[tid];
    if (tid < j) {
        st->h1[tid] = t[tid];
        st->dq[tid] = s[tid];
    }
    if (tid == j) st->h1[j] = taus;
}

// Step j's one reduction: s = V_{<j}^T q_j and t = V_{<j}^T w against the
// first j basis vectors, alpha, beta, gamma over q_j (slot j) and w; tiles of
// q_j and w staged in shared memory.  FP32 vectors (the form that keeps a
// flexible basis); warp, block and grid sums are compensated FP32 pairs (F2),
// FP64 from the last block on.  partial[b * 64 + i] holds pair i < 2 j + 3.
template <class T>
__global__ void __launch_bounds__(DT, 2) k_dcgs_dots(const T *__restrict__ V, int64_t ldv, int nrow, int j,
                                                   const T *__restrict__ w, GmresState *st,
                                                   double *__restrict__ partial, cudaGraphConditionalHandle next,
                                                   int set_next) {
    static_assert(sizeof(T) == 4, "DCGS2 runs on FP32 vectors");
    typedef typename Vec<T>::type VT;
    constexpr int VN = Vec<T>::n;
    __shared__ __align__(16) T qs[TILE];
    __shared__ __align__(16) T ws[TILE];
    __shared__ F2 red[2 * MAX_RESTART + 3];
    __shared__ F2 wsum[3 * GW];
    __shared__ double fs[64];
    if (st->done) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nk = 2 * j + 3;
    T aq[KPW], aw[KPW];
#pragma unroll
    for (int kk = 0; kk < KPW; ++kk) aq[kk] = aw[kk] = (T)0;
    T qq = (T)0, qw = (T)0, ww = (T)0;
    VT *qsv = reinterpret_cast<VT *>(qs), *wsv = reinterpret_cast<VT *>(ws);
    for (int64_t base = (int64_t)blockIdx.x * TILE; base < nrow; base += (int64_t)gridDim.x * TILE) {
        const int lim = (int)((nrow - base) < TILE ? (nrow - base) : TILE);
        const VT *qg = reinterpret_cast<const VT *>(V + (int64_t)j * ldv + base);
        const VT *wg = reinterpret_cast<const VT *>(w + base);
        for (int cix = tid; cix < lim / VN; cix += DT) {
            const VT qi = qg[cix], wi = wg[cix];
            qsv[cix] = qi;
            wsv[cix] = wi;
            qq = sumsq(qi, qq);
            qw = dotv(qi, wi, qw);
            ww = sumsq(wi, ww);
        }
        __syncthreads();
        if (j > 0) tile_dots2<T>(V, ldv, base, lim, j, qs, ws, aq, aw);
        __syncthreads();
    }
    // per basis vector, the block's parts summed in a fixed order
    if (j > 0) {
        if (GW / j >= 2) {
            const int parts = GW / j;
            const F2 vq = warp_sum_f2(F2{aq[0], 0.f}), vw = warp_sum_f2(F2{aw[0], 0.f});
            if (lane == 0) {
                wsum[wid] = vq;
                wsum[GW + wid] = vw;
            }
            __syncthreads();
            if (tid < j) {
                F2 a{0.f, 0.f}, b{0.f, 0.f};
                for (int part = 0; part < parts; ++part) {
                    a = f2add(a, wsum[tid + j * part]);
                    b = f2add(b, wsum[GW + tid + j * part]);
                }
                red[tid] = a;
                red[j + tid] = b;
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < KPW; ++kk) {
                const int k = wid + GW * kk;
                if (k < j) {
                    const F2 vq = warp_sum_f2(F2{aq[kk], 0.f}), vw = warp_sum_f2(F2{aw[kk], 0.f});
                    if (lane == 0) {
                        red[k] = vq;
                        red[j + k] = vw;
                    }
                }
            }
        }
    }
    __syncthreads();
    {
        const F2 a = warp_sum_f2(F2{qq, 0.f}), b = warp_sum_f2(F2{qw, 0.f}), c = warp_sum_f2(F2{ww, 0.f});
        if (lane == 0) {
            wsum[wid] = a;
            wsum[GW + wid] = b;
            wsum[2 * GW + wid] = c;
        }
        __syncthreads();
        if (tid < 3) {
            F2 v{0.f, 0.f};
            for (int q = 0; q < GW; ++q) v = f2add(v, wsum[tid * GW + q]);
            red[2 * j + tid] = v;
        }
    }
    __syncthreads();
    if (tid < nk)
        reinterpret_cast<float2 *>(partial)[(int64_t)blockIdx.x * 64 + tid] = make_float2(red[tid].s, red[tid].e);
    if (!last_block(&st->ticket)) return;
    final_sums_f2(partial, gridDim.x, nk, fs);
    dcgs_tail(st, j, fs, next, set_next);
}

// Start of DCGS2 step j >= 1: slot p = j - 1 finished, v_p = (q_p - V_{<p} s)
// / nu (slot 0 holds v_0 already), and the tentative q_j = (w - V_{<=p} h_p)
// / nut_j written to slot j, with z = omega q_j for the polynomial.
template <class T>
__global__ void __launch_bounds__(GT) k_dcgs_update(T *__restrict__ V, int64_t ldv, int nrow, int j,
                                                   const T *__restrict__ w, T *__restrict__ z,
                                                   const GmresState *__restrict__ st) {
    typedef typename Vec<T>::type VT;
    constexpr int VN = Vec<T>::n;
    __shared__ T sq[MAX_RESTART], th[MAX_RESTART + 1];
    if (st->done) return;
    const int p = j - 1;
    if (threadIdx.x < p) sq[threadIdx.x] = (T)st->dq[threadIdx.x];
    if (threadIdx.x <= p) th[threadIdx.x] = (T)st->h1[threadIdx.x];
    __syncthreads();
    const T inu = (T)st->inu, inut = (T)st->inv_norm, om = (T)st->omega;
    const VT *wv = reinterpret_cast<const VT *>(w);
    VT *vp = reinterpret_cast<VT *>(V + (int64_t)p * ldv), *vj = reinterpret_cast<VT *>(V + (int64_t)j * ldv);
    VT *zv = reinterpret_cast<VT *>(z);
    for (int cix = blockIdx.x * GT + threadIdx.x; cix < nrow / VN; cix += gridDim.x * GT) {
        VT a = vp[cix], b = wv[cix];
#pragma unroll 8
        for (int k = 0; k < p; ++k) {
            const VT x = __ldg(reinterpret_cast<const VT *>(V + (int64_t)k * ldv) + cix);
            a = axpyv(a, x, sq[k]);
            b = axpyv(b, x, th[k]);
        }
        if (p > 0) {
            a = fmav(a, inu, zerov<VT>());
            vp[cix] = a;
        }
        b = axpyv(b, a, th[p]);
        const VT q = fmav(b, inut, zerov<VT>());
        vj[cix] = q;
        zv[cix] = fmav(q, om, zerov<VT>());
    }
}

// t = V y with H y = g (the combination the cycle end adds, before preconditioning)
template <class T>
__global__ void __launch_bounds__(256) k_combine(const T *__restrict__ V, int64_t ldv, int nrow, T *__restrict__ t,
                                                 const GmresState *__restrict__ st) {
    __shared__ T ys[MAX_RESTART];
    const int je = st->jend;
    if (threadIdx.x == 0) {
        const int M = MAX_RESTART;
        double yd[MAX_RESTART];
        for (int k = je - 1; k >= 0; --k) {
            double s = st->g[k];
            for (int l = k + 1; l < je; ++l) s -= st->H[k * M + l] * yd[l];
            yd[k] = s / st->H[k * M + k];
            ys[k] = (T)yd[k];
        }
    }
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrow; i += gridDim.x * blockDim.x) {
        T s = (T)0;
        for (int k = 0; k < je; ++k) s = fma(V[(int64_t)k * ldv + i], ys[k], s);
        t[i] = s;
    }
}

template <class T>
__global__ void k_axpy_first(const T *__restrict__ t, T *__restrict__ z, int n, const GmresState *__restrict__ st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = (T)st->omega * t[i];
}

template <class T>
__global__ void k_add(T *__restrict__ u, const T *__restrict__ z, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] += z[i];
}

__global__ void k_to_f32(float *__restrict__ out, const double *__restrict__ a, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)a[i];
}

// u += e (FP32 correction into the FP64 iterate), e cleared for the next refinement
__global__ void k_add_f32(double *__restrict__ u, float *__restrict__ e, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { u[i] += (double)e[i]; e[i] = 0.f; }
}

int sm_count() {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 152;
}

int64_t l2_bytes() {
    int b = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b, cudaDevAttrL2CacheSize, dev);
    return b > 0 ? b : (int64_t)126 << 20;
}

// Bytes a sweep reads per stored entry of the packed width-sorted matrix (a
// 2-byte value and 3 bytes of packed column) and per row (x and b read, y
// written, FP32).
constexpr double SWEEP_ENTRY_BYTES = 5.0, SWEEP_ROW_BYTES = 12.0;

}  // namespace

// Matrix bytes the sweeps read with ordinary loads when left to the library:
// all of them when the matrix and the sweep's vectors fit in 3/4 of the L2;
// 0.4 of the L2 when they take up to twice the L2 (the rest of the L2 holds
// the vectors and the streamed lines; on the 1.05e6-row, 145 MB matrix of a
// 1e7-particle beam at depth 10 kept sizes of 0.2 to 0.5 of the L2 gave
// 30.5 to 31.2 us per sweep against 35.3 us with no streaming loads and
// 33.0 us with streaming loads only); all of them again beyond (a 650 MB
// matrix of a 64-beam batch gained nothing from the 8% that can stay and
// lost 2% to the streaming loads).
int64_t sweep_keep_bytes(const apcloud_ctx *c) {
    if (c->sweep_keep >= 0) return c->sweep_keep;
    const double l2 = (double)l2_bytes();
    const double tot = SWEEP_ENTRY_BYTES * (double)c->ss_entries + SWEEP_ROW_BYTES * (double)c->n_tot;
    return (tot <= 0.75 * l2 || tot > 2.0 * l2) ? INT64_MAX : (int64_t)(0.4 * l2);
}

namespace {

// the same as the entry of the sorted matrix from which slices are hinted
int64_t sweep_keep_entries(const apcloud_ctx *c) {
    const int64_t kb = sweep_keep_bytes(c);
    return kb == INT64_MAX ? INT64_MAX : (int64_t)((double)kb / SWEEP_ENTRY_BYTES);
}

// dot kernels: 2 fat blocks per SM (few partials for the last block to sum)
// grid of the restart residual: 4 blocks of RT threads per SM striding over
// the rows (few partials and few ticket atomics for the last block)
int resid_blocks(int64_t nrow) {
    const int nb = div_up(nrow, RT), cap = 4 * sm_count();
    return nb < 1 ? 1 : (nb > cap ? cap : nb);
}

int dot_blocks(int64_t ldv) {
    int nb = div_up(ldv, TILE), cap = 2 * sm_count();
    return nb < 1 ? 1 : (nb > cap ? cap : nb);
}

// row-parallel kernels: up to 8 blocks per SM for memory parallelism
int stream_blocks(int64_t nrow) {
    int nb = div_up(nrow / 2, GT), cap = 8 * sm_count();
    return nb < 1 ? 1 : (nb > cap ? cap : nb);
}

template <class T>
void gs_dispatch(apcloud_ctx *c, int pass, int nblk, const T *V, int64_t ldv, int j, T *w, T *wraw, GmresState *st,
                 double *partial, const uint8_t *tact, cudaGraphConditionalHandle next = {}, int set_next = 0) {
    (void)nblk;
    const int nrow = (int)ldv;
    if (pass == 0)
        APC_LAUNCH(c, K_DOT, dot_blocks(ldv), DT, 0, (k_gs_dots<0, T>), V, ldv, nrow, j, w, st, partial, tact,
                   next, 0);
    else if (pass == 1)
        APC_LAUNCH(c, K_UPDDOT, dot_blocks(ldv), DT, 0, (k_gs_dots<1, T>), V, ldv, nrow, j, w, st, partial, tact,
                   next, 0);
    else if (pass == 3)   // PASS 2 of k_gs_dots: the step's last kernel
        APC_LAUNCH(c, K_UPDDOT, dot_blocks(ldv), DT, 0, (k_gs_dots<2, T>), V, ldv, nrow, j, w, st, partial, tact,
                   next, set_next);
    else
        APC_LAUNCH(c, K_UPDNORM, stream_blocks(ldv), GT, 0, k_gs_norm<T>, V, ldv, nrow, j, (const T *)w, wraw, st,
                   partial, tact, next, set_next);
}

// grid of the streaming reductions (norms, cycle end); the partial buffer
// must hold (div_up(n, RT) + 2 * reduction_blocks) * 64 doubles
int reduction_blocks(apcloud_ctx *c, int n) {
    (void)c;
    int64_t ldv = ((int64_t)n + 31) / 32 * 32;
    int a = stream_blocks(ldv), b = dot_blocks(ldv);
    return a > b ? a : b;
}


// Per-beam convergence of a batch: at every restart the residual of each beam
// is compared with rtol ||b_b||; converged beams are frozen (their residual
// rows set to zero, so the block-diagonal Krylov vectors stay zero there and
// the products skip them) and the cycle continues on the others.
struct BeamMask {
    int nb;
    const int64_t *rng;   // 7 node ranges per beam
    const double *b2;     // ||b_b||^2
    double *r2;           // ||r_b||^2 scratch
    int *bdone;
    const int32_t *nbo;
    uint8_t *tact;
    int64_t ntile;
    double rtol;
};

// squared norm of r over the nodes of each beam, in fixed order: BSQ_CH
// blocks per beam each sum one part of every row segment of the beam, then
// the parts are added in order (one block per beam left the largest beam's
// ~4e5 rows to a single SM)
constexpr int BSQ_CH = 16;

template <class T>
__global__ void __launch_bounds__(256) k_beam_sq_part(const T *__restrict__ r, const int64_t *__restrict__ rng, int nb,
                                                      double *__restrict__ part) {
    __shared__ double sh[256];
    const int beam = blockIdx.x / BSQ_CH, ch = blockIdx.x % BSQ_CH;
    double s = 0.0;
    for (int seg = 0; seg < 7; ++seg) {
        const int64_t lo = rng[(int64_t)seg * (nb + 1) + beam], hi = rng[(int64_t)seg * (nb + 1) + beam + 1];
        const int64_t a = lo + (hi - lo) * ch / BSQ_CH, e = lo + (hi - lo) * (ch + 1) / BSQ_CH;
        for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) s = fma((double)r[i], (double)r[i], s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_beam_sq_sum(const double *__restrict__ part, int nb, double *__restrict__ out) {
    const int beam = blockIdx.x * blockDim.x + threadIdx.x;
    if (beam >= nb) return;
    double s = 0.0;
    for (int ch = 0; ch < BSQ_CH; ++ch) s += part[(int64_t)beam * BSQ_CH + ch];
    out[beam] = s;
}

// out[b] = sum of r^2 over the rows of beam b (its 7 row segments)
template <class T>
void beam_sq(apcloud_ctx *c, const T *r, const int64_t *rng, int nb, double *out) {
    double *part = ptr<double>(c->beam_part);
    APC_LAUNCH(c, K_VEC, nb * BSQ_CH, 256, 0, k_beam_sq_part<T>, r, rng, nb, part);
    APC_LAUNCH(c, K_VEC, div_up(nb, 64), 64, 0, k_beam_sq_sum, (const double *)part, nb, out);
}

// one block: mark converged beams, then restart the cycle on the others:
// beta = ||r|| over unconverged beams, the in-cycle stopping threshold
// rtol * min ||b_b|| over them (which implies every one of them converged)
__global__ void __launch_bounds__(256) k_beam_mask(const double *__restrict__ r2, const double *__restrict__ b2, int nb,
                                                   double rtol, int *__restrict__ bdone, GmresState *st) {
    __shared__ double ssum[256], smin[256];
    __shared__ int scnt[256];
    double sum = 0.0, mn = 1e300;
    int cnt = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int done = bdone[b] || b2[b] == 0.0 || r2[b] <= rtol * rtol * b2[b];
        bdone[b] = done;
        if (!done) {
            sum += r2[b];
            mn = fmin(mn, b2[b]);
            ++cnt;
        }
    }
    ssum[threadIdx.x] = sum;
    smin[threadIdx.x] = mn;
    scnt[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ssum[threadIdx.x] += ssum[threadIdx.x + o];
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
            scnt[threadIdx.x] += scnt[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double beta = sqrt(ssum[0]);
        st->beta = beta;
        st->g[0] = beta;
        st->inv_norm = beta > 0.0 ? 1.0 / beta : 0.0;
        st->bnorm = scnt[0] > 0 ? sqrt(smin[0]) : 1.0;
        st->done = scnt[0] == 0 ? 1 : 0;
        st->jend = 0;
    }
}

template <class T>
__global__ void k_mask_rows(T *__restrict__ r, int n, const int32_t *__restrict__ nbo, const int *__restrict__ bdone) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && bdone[nbo[i]]) r[i] = (T)0;
}

// tile t (TILE rows) is active if one of its rows belongs to an unconverged beam
__global__ void k_tile_active(const int32_t *__restrict__ nbo, const int *__restrict__ bdone, int n,
                              uint8_t *__restrict__ tact) {
    const int64_t lo = (int64_t)blockIdx.x * TILE;
    int any = 0;
    for (int64_t i = lo + threadIdx.x; i < lo + TILE && i < n; i += blockDim.x) any |= !bdone[nbo[i]];
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) tact[blockIdx.x] = (uint8_t)any;
}

// after a residual product: freeze converged beams, restart on the others
template <class T>
apcloud_status mask_residual(apcloud_ctx *c, const BeamMask &bm, T *r, GmresState *st) {
    const int n = c->n_tot;
    beam_sq<T>(c, (const T *)r, bm.rng, bm.nb, bm.r2);
    APC_LAUNCH(c, K_VEC, 1, 256, 0, k_beam_mask, (const double *)bm.r2, bm.b2, bm.nb, bm.rtol, bm.bdone, st);
    APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_mask_rows<T>, r, n, bm.nbo, (const int *)bm.bdone);
    APC_LAUNCH(c, K_VEC, (int)bm.ntile, 256, 0, k_tile_active, bm.nbo, (const int *)bm.bdone, n, bm.tact);
    return cuda_check(c, cudaGetLastError(), "beam mask");
}

// ---------------------------------------------------------------- per-beam Krylov spaces
// A batch of B independent beams is block-diagonal.  Instead of one Krylov
// space for the whole vector (whose iteration count is set by all beams at
// once), every beam runs its own GMRES(m): the row-parallel kernels (products,
// sweeps, normalisation) look up the row's beam, and the Gram-Schmidt
// reductions run over "items" -- chunks of at most BITEM rows inside one of a
// beam's 7 node ranges -- whose partial sums are added per beam in a fixed
// order.  Each beam has its own Hessenberg matrix, Givens rotations, residual
// estimate and stopping test; a beam that has finished its cycle (or
// converged) drops out of every later launch of the cycle.
constexpr int BITEM = 1024;   // rows per item
constexpr int BGT = 256;      // threads per item block (8 warps)

struct BKry {
    int nb, nitems, m;
    const int4 *items;        // (beam, lo, hi, 0)
    const int *item_off;      // items of beam b: item_off[b] .. item_off[b+1]-1
    const int32_t *nbo;       // beam of every node
    double *H, *cs, *sn, *g, *h1, *h2, *y;   // per beam: (m+1) x m, m, m, m+1, m+1, m+1, m
    double *bnorm, *binv, *r2, *relres;
    // per beam for DCGS2 (k_bdcgs_*): s = V^T q_j (m+1), nu, 1 / nu, nut, gpre,
    // and the step's 2 j + 3 sums (64)
    double *dq, *nu, *inu, *nut, *gpre, *fs;
    int *done;                // cycle finished (converged, breakdown or m steps)
    int *conv;                // converged: frozen for the rest of the solve
    int *jend;
};

template <class T>
__global__ void k_bnormalize_first(const T *__restrict__ wraw, T *__restrict__ vj, T *__restrict__ z, int n,
                                   const int32_t *__restrict__ nbo, const int *__restrict__ done,
                                   const double *__restrict__ binv, const GmresState *__restrict__ st) {
    if (st->done) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = nbo[i];
    if (done[b]) return;
    const T v = wraw[i] * (T)binv[b];
    vj[i] = v;
    z[i] = (T)st->omega * v;
}

// PASS 0: h1 = V^T w over the item's rows.  PASS 1: w -= V h1 there, then
// h2 = V^T w.  Partial sums per item (64 per item).
template <int PASS, class T>
__global__ void __launch_bounds__(BGT) k_bgs_dots(const T *__restrict__ V, int64_t ldv, int j, T *__restrict__ w,
                                                  BKry bk, const GmresState *__restrict__ st,
                                                  double *__restrict__ partial) {
    __shared__ T ws[BITEM];
    __shared__ T hs[MAX_RESTART + 1];
    if (st->done) return;
    const int4 it = bk.items[blockIdx.x];
    const int beam = it.x, lo = it.y, cnt = it.z - it.y;
    if (bk.done[beam]) return;
    const int j1 = j + 1, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (PASS == 1 && tid < j1) hs[tid] = (T)bk.h1[(int64_t)beam * (bk.m + 1) + tid];
    __syncthreads();
    for (int r = tid; r < cnt; r += BGT) {
        T wi = w[lo + r];
        if (PASS == 1) {
            for (int k = 0; k < j1; ++k) wi = fma(-V[(int64_t)k * ldv + lo + r], hs[k], wi);
            w[lo + r] = wi;
        }
        ws[r] = wi;
    }
    __syncthreads();
    for (int k = wid; k < j1; k += BGT / 32) {
        const T *vk = V + (int64_t)k * ldv + lo;
        T a = (T)0;
        for (int r = lane; r < cnt; r += 32) a = fma(vk[r], ws[r], a);
        if constexpr (sizeof(T) == 4) {   // compensated FP32 tree (F2) instead of FP64 shuffles
            const F2 sum = warp_sum_f2(F2{a, 0.f});
            if (lane == 0) partial[(int64_t)blockIdx.x * 64 + k] = f2_value(sum);
        } else {
            const double sum = warp_sum((double)a);
            if (lane == 0) partial[(int64_t)blockIdx.x * 64 + k] = sum;
        }
    }
}

// per beam: h = sum of its items' partials (fixed order)
template <int PASS>
__global__ void k_bfinal_h(int j, BKry bk, const GmresState *__restrict__ st, const double *__restrict__ partial) {
    if (st->done) return;
    const int beam = blockIdx.x, i = threadIdx.x;
    if (bk.done[beam] || i > j) return;
    double s = 0.0;
    for (int q = bk.item_off[beam]; q < bk.item_off[beam + 1]; ++q) s += partial[(int64_t)q * 64 + i];
    double *h = (PASS == 0 ? bk.h1 : bk.h2) + (int64_t)beam * (bk.m + 1);
    h[i] = s;
}

// wraw = w - V h2 over the item's rows; partial = ||wraw||^2 there
template <class T>
__global__ void __launch_bounds__(BGT) k_bgs_norm(const T *__restrict__ V, int64_t ldv, int j,
                                                  const T *__restrict__ w, T *__restrict__ wraw, BKry bk,
                                                  const GmresState *__restrict__ st, double *__restrict__ partial) {
    __shared__ T hs[MAX_RESTART + 1];
    __shared__ double red[BGT / 32];
    __shared__ F2 redf[BGT / 32];
    if (st->done) return;
    const int4 it = bk.items[blockIdx.x];
    const int beam = it.x, lo = it.y, cnt = it.z - it.y;
    if (bk.done[beam]) return;
    const int j1 = j + 1, tid = threadIdx.x;
    if (tid < j1) hs[tid] = (T)bk.h2[(int64_t)beam * (bk.m + 1) + tid];
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
        // ||wraw||^2 as a compensated FP32 sum: each square enters exactly
        // (p + fma(w, w, -p)); an FP64 product per row kept the FP64 pipe busy
        F2 sq{0.f, 0.f};
        for (int r = tid; r < cnt; r += BGT) {
            T wi = w[lo + r];
            for (int k = 0; k < j1; ++k) wi = fma(-V[(int64_t)k * ldv + lo + r], hs[k], wi);
            wraw[lo + r] = wi;
            const float p = wi * wi;
            sq = f2add(sq, F2{p, fmaf(wi, wi, -p)});
        }
        sq = warp_sum_f2(sq);
        if ((tid & 31) == 0) redf[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            F2 t{0.f, 0.f};
            for (int q = 0; q < BGT / 32; ++q) t = f2add(t, redf[q]);
            partial[(int64_t)blockIdx.x * 64] = f2_value(t);
        }
    } else {
        double sq = 0.0;
        for (int r = tid; r < cnt; r += BGT) {
            T wi = w[lo + r];
            for (int k = 0; k < j1; ++k) wi = fma(-V[(int64_t)k * ldv + lo + r], hs[k], wi);
            wraw[lo + r] = wi;
            sq = fma((double)wi, (double)wi, sq);
        }
        sq = warp_sum(sq);
        if ((tid & 31) == 0) red[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < BGT / 32; ++q) t += red[q];
            partial[(int64_t)blockIdx.x * 64] = t;
        }
    }
}

// per beam (one thread each): Hessenberg column j, Givens rotation, residual
// estimate, stopping test; then (block 0 of a single-block launch) the
// number of beams still in their cycle decides st->done
__global__ void __launch_bounds__(256) k_bfinal_norm(int j, BKry bk, GmresState *st,
                                                     const double *__restrict__ partial,
                                                     cudaGraphConditionalHandle next, int set_next) {
    __shared__ int act[256];
    int a = 0;
    if (!st->done) {
        const int M = bk.m;
        for (int beam = threadIdx.x; beam < bk.nb; beam += blockDim.x) {
            if (bk.done[beam]) continue;
            double s = 0.0;
            for (int q = bk.item_off[beam]; q < bk.item_off[beam + 1]; ++q) s += partial[(int64_t)q * 64];
            const double hn = sqrt(s);
            double *H = bk.H + (int64_t)beam * (M + 1) * M, *cs = bk.cs + (int64_t)beam * M,
                   *sn = bk.sn + (int64_t)beam * M, *g = bk.g + (int64_t)beam * (M + 1);
            const double *h1 = bk.h1 + (int64_t)beam * (M + 1), *h2 = bk.h2 + (int64_t)beam * (M + 1);
            // rotation i acts on entries i and i + 1 of column j: the entry it
            // carries to the next rotation stays in a register, the others are
            // the unrotated h1 + h2 (no store-then-load chain through memory)
            double carried = h1[0] + h2[0];
            for (int i = 0; i < j; ++i) {
                const double x0 = carried, x1 = h1[i + 1] + h2[i + 1];
                H[i * M + j] = cs[i] * x0 + sn[i] * x1;
                carried = -sn[i] * x0 + cs[i] * x1;
            }
            const double x0 = carried, x1 = hn;
            const double den = sqrt(x0 * x0 + x1 * x1);
            cs[j] = den != 0.0 ? x0 / den : 1.0;
            sn[j] = den != 0.0 ? x1 / den : 0.0;
            H[j * M + j] = den;
            H[(j + 1) * M + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            bk.jend[beam] = j + 1;
            const bool fin = fabs(g[j + 1]) <= st->rtol * bk.bnorm[beam] || hn == 0.0 || j + 1 >= M;
            bk.done[beam] = fin ? 1 : 0;
            bk.binv[beam] = hn > 0.0 ? 1.0 / hn : 0.0;
            if (!fin) ++a;
        }
    }
    act[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) act[threadIdx.x] += act[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && !st->done && act[0] == 0) st->done = 1;
    if (threadIdx.x == 0 && set_next) cudaGraphSetConditional(next, st->done ? 0u : 1u);
}

// per beam: y = H^-1 g (jend x jend, upper triangular after the rotations)
__global__ void k_bsolve_y(BKry bk) {
    const int beam = blockIdx.x * blockDim.x + threadIdx.x;
    if (beam >= bk.nb) return;
    const int M = bk.m, je = bk.jend[beam];
    const double *H = bk.H + (int64_t)beam * (M + 1) * M, *g = bk.g + (int64_t)beam * (M + 1);
    double *y = bk.y + (int64_t)beam * M;
    for (int k = je - 1; k >= 0; --k) {
        double t = g[k];
        for (int l = k + 1; l < je; ++l) t -= H[k * M + l] * y[l];
        y[k] = t / H[k * M + k];
    }
}

// ---- DCGS2 for per-beam Krylov spaces (the batch form of k_dcgs_dots,
// dcgs_tail and k_dcgs_update; FP32 vectors with a flexible basis).
// Step j's pass over one item: s = V_{<j}^T q_j and t = V_{<j}^T w over its
// rows (a warp per basis vector), q.q, q.w, w.w; compensated FP32 sums, the
// products entering exactly.  partial[item * 64 + i], i < 2 j + 3.
template <class T>
__global__ void __launch_bounds__(BGT) k_bdcgs_dots(const T *__restrict__ V, int64_t ldv, int j,
                                                    const T *__restrict__ w, BKry bk,
                                                    const GmresState *__restrict__ st, double *__restrict__ partial) {
    static_assert(sizeof(T) == 4, "DCGS2 runs on FP32 vectors");
    __shared__ T qs[BITEM], ws[BITEM];
    __shared__ F2 red[3][BGT / 32];
    if (st->done) return;
    const int4 it = bk.items[blockIdx.x];
    const int beam = it.x, lo = it.y, cnt = it.z - it.y;
    if (bk.done[beam]) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const T *q = V + (int64_t)j * ldv + lo;
    F2 aa{0.f, 0.f}, ab{0.f, 0.f}, ac{0.f, 0.f};
    for (int r = tid; r < cnt; r += BGT) {
        const T qi = q[r], wi = w[lo + r];
        qs[r] = qi;
        ws[r] = wi;
        const float p1 = qi * qi, p2 = qi * wi, p3 = wi * wi;
        aa = f2add(aa, F2{p1, fmaf(qi, qi, -p1)});
        ab = f2add(ab, F2{p2, fmaf(qi, wi, -p2)});
        ac = f2add(ac, F2{p3, fmaf(wi, wi, -p3)});
    }
    __syncthreads();
    for (int k = wid; k < j; k += BGT / 32) {
        const T *vk = V + (int64_t)k * ldv + lo;
        T a = (T)0, b = (T)0;
        for (int r = lane; r < cnt; r += 32) {
            const T x = vk[r];
            a = fma(x, qs[r], a);
            b = fma(x, ws[r], b);
        }
        const F2 sa = warp_sum_f2(F2{a, 0.f}), sb = warp_sum_f2(F2{b, 0.f});
        if (lane == 0) {
            partial[(int64_t)blockIdx.x * 64 + k] = f2_value(sa);
            partial[(int64_t)blockIdx.x * 64 + j + k] = f2_value(sb);
        }
    }
    aa = warp_sum_f2(aa);
    ab = warp_sum_f2(ab);
    ac = warp_sum_f2(ac);
    if (lane == 0) {
        red[0][wid] = aa;
        red[1][wid] = ab;
        red[2][wid] = ac;
    }
    __syncthreads();
    if (tid < 3) {
        F2 v{0.f, 0.f};
        for (int qd = 0; qd < BGT / 32; ++qd) v = f2add(v, red[tid][qd]);
        partial[(int64_t)blockIdx.x * 64 + 2 * j + tid] = f2_value(v);
    }
}

// per beam: its items' sums of step j (fixed order) into bk.fs
__global__ void k_bdcgs_sum(int j, BKry bk, const GmresState *__restrict__ st, const double *__restrict__ partial) {
    if (st->done) return;
    const int beam = blockIdx.x, i = threadIdx.x;
    if (bk.done[beam] || i >= 2 * j + 3) return;
    double s = 0.0;
    for (int qd = bk.item_off[beam]; qd < bk.item_off[beam + 1]; ++qd) s += partial[(int64_t)qd * 64 + i];
    bk.fs[(int64_t)beam * 64 + i] = s;
}

// per beam (one thread each): dcgs_tail's algebra on the beam's sums --
// column j - 1 finished, column j projected with a tentative rotation, the
// beam's stopping test; then (single-block launch) the number of beams still
// in their cycle decides st->done
__global__ void __launch_bounds__(256) k_bdcgs_tail(int j, BKry bk, GmresState *st, cudaGraphConditionalHandle next,
                                                    int set_next) {
    __shared__ int act[256];
    int a = 0;
    if (!st->done) {
        const int M = bk.m;
        for (int beam = threadIdx.x; beam < bk.nb; beam += blockDim.x) {
            if (bk.done[beam]) continue;
            const double *fs = bk.fs + (int64_t)beam * 64, *s = fs, *t = fs + j;
            const double alpha = fs[2 * j], beta = fs[2 * j + 1], gamma = fs[2 * j + 2];
            double *H = bk.H + (int64_t)beam * (M + 1) * M, *cs = bk.cs + (int64_t)beam * M,
                   *sn = bk.sn + (int64_t)beam * M, *g = bk.g + (int64_t)beam * (M + 1);
            double *h1 = bk.h1 + (int64_t)beam * (M + 1), *dq = bk.dq + (int64_t)beam * (M + 1);
            double nu = 1.0, gj = g[0], ss = 0.0, stt = 0.0, tt = 0.0;
            for (int k = 0; k < j; ++k) {
                ss = fma(s[k], s[k], ss);
                stt = fma(s[k], t[k], stt);
                tt = fma(t[k], t[k], tt);
            }
            if (j > 0) {
                nu = sqrt(fmax(alpha - ss, 0.0));
                const double nut = bk.nut[beam];
                // column j - 1: (h_{j-1} + nut s, nut nu), rotations 0 .. j - 2, then its own
                double carried = fma(nut, s[0], h1[0]);
                for (int i = 0; i + 1 < j; ++i) {
                    const double x0 = carried, x1 = fma(nut, s[i + 1], h1[i + 1]);
                    H[i * M + j - 1] = cs[i] * x0 + sn[i] * x1;
                    carried = -sn[i] * x0 + cs[i] * x1;
                }
                double c, sv, r;
                givens(carried, nut * nu, c, sv, r);
                cs[j - 1] = c;
                sn[j - 1] = sv;
                H[(j - 1) * M + j - 1] = r;
                H[j * M + j - 1] = 0.0;
                const double gp = bk.gpre[beam];
                g[j - 1] = c * gp;
                gj = -sv * gp;
            }
            const double tau = nu > 0.0 ? (beta - stt) / nu : 0.0;
            const double nut1 = sqrt(fmax(gamma - tt - tau * tau, 0.0));
            // column j: (t, tau, nut1), rotations 0 .. j - 1, then its tentative own
            double carried = j > 0 ? t[0] : tau;
            for (int i = 0; i < j; ++i) {
                const double x0 = carried, x1 = i + 1 < j ? t[i + 1] : tau;
                H[i * M + j] = cs[i] * x0 + sn[i] * x1;
                carried = -sn[i] * x0 + cs[i] * x1;
            }
            double c, sv, r;
            givens(carried, nut1, c, sv, r);
            cs[j] = c;
            sn[j] = sv;
            H[j * M + j] = r;
            H[(j + 1) * M + j] = 0.0;
            bk.gpre[beam] = gj;
            g[j] = c * gj;
            g[j + 1] = -sv * gj;
            for (int k = 0; k < j; ++k) {
                h1[k] = t[k];
                dq[k] = s[k];
            }
            h1[j] = tau;
            bk.nu[beam] = nu;
            bk.inu[beam] = nu > 0.0 ? 1.0 / nu : 0.0;
            bk.nut[beam] = nut1;
            bk.binv[beam] = nut1 > 0.0 ? 1.0 / nut1 : 0.0;
            bk.jend[beam] = j + 1;
            const bool fin = fabs(sv * gj) <= st->rtol * bk.bnorm[beam] || nut1 == 0.0 || nu == 0.0 || j + 1 >= M;
            bk.done[beam] = fin ? 1 : 0;
            if (!fin) ++a;
        }
    }
    act[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) act[threadIdx.x] += act[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && !st->done && act[0] == 0) st->done = 1;
    if (threadIdx.x == 0 && set_next) cudaGraphSetConditional(next, st->done ? 0u : 1u);
}

// start of step j >= 1 over one item: v_{j-1} = (q_{j-1} - V s) / nu (slot 0
// holds v_0 already), q_j = (w - V h_{j-1}) / nut_j, z = omega q_j
template <class T>
__global__ void __launch_bounds__(BGT) k_bdcgs_update(T *__restrict__ V, int64_t ldv, int j,
                                                      const T *__restrict__ w, T *__restrict__ z, BKry bk,
                                                      const GmresState *__restrict__ st) {
    __shared__ T sq[MAX_RESTART], th[MAX_RESTART + 1];
    __shared__ T sc[2];
    if (st->done) return;
    const int4 it = bk.items[blockIdx.x];
    const int beam = it.x, lo = it.y, cnt = it.z - it.y;
    if (bk.done[beam]) return;
    const int p = j - 1, tid = threadIdx.x;
    const int64_t bo = (int64_t)beam * (bk.m + 1);
    if (tid < p) sq[tid] = (T)bk.dq[bo + tid];
    if (tid <= p) th[tid] = (T)bk.h1[bo + tid];
    if (tid == 0) {
        sc[0] = (T)bk.inu[beam];
        sc[1] = (T)bk.binv[beam];
    }
    __syncthreads();
    const T inu = sc[0], inut = sc[1], om = (T)st->omega;
    T *vp = V + (int64_t)p * ldv + lo, *vj = V + (int64_t)j * ldv + lo;
    for (int r = tid; r < cnt; r += BGT) {
        T a = vp[r], b = w[lo + r];
        for (int k = 0; k < p; ++k) {
            const T x = V[(int64_t)k * ldv + lo + r];
            a = fma(-x, sq[k], a);
            b = fma(-x, th[k], b);
        }
        if (p > 0) {
            a *= inu;
            vp[r] = a;
        }
        b = fma(-a, th[p], b);
        const T qv = b * inut;
        vj[r] = qv;
        z[lo + r] = om * qv;
    }
}

// out (+)= V y over the item's rows (ADD: u += V y; else t = V y)
template <bool ADD, class T>
__global__ void __launch_bounds__(BGT) k_bcombine(const T *__restrict__ V, int64_t ldv, T *__restrict__ out,
                                                  BKry bk) {
    const int4 it = bk.items[blockIdx.x];
    const int beam = it.x, lo = it.y, cnt = it.z - it.y;
    const int je = bk.jend[beam];
    const double *y = bk.y + (int64_t)beam * bk.m;
    for (int r = threadIdx.x; r < cnt; r += BGT) {
        T sum = (T)0;
        for (int k = 0; k < je; ++k) sum = fma(V[(int64_t)k * ldv + lo + r], (T)y[k], sum);
        if (ADD) out[lo + r] += sum;
        else out[lo + r] = sum;
    }
}

// per beam after the residual b - Ahat u of a restart: beta_b, the stopping
// test against rtol ||b_b|| (converged beams stay frozen), the start of the
// beam's next cycle; st->done once every beam has converged
__global__ void __launch_bounds__(256) k_bstart(BKry bk, GmresState *st) {
    __shared__ int act[256];
    __shared__ double rmax[256];
    int a = 0;
    double rm = 0.0;
    const int M = bk.m;
    for (int beam = threadIdx.x; beam < bk.nb; beam += blockDim.x) {
        const double beta = sqrt(bk.r2[beam]), bn = bk.bnorm[beam];
        const bool conv = bk.conv[beam] || bn == 0.0 || beta <= st->rtol * bn;
        bk.conv[beam] = conv ? 1 : 0;
        bk.done[beam] = conv ? 1 : 0;
        bk.jend[beam] = 0;
        double *g = bk.g + (int64_t)beam * (M + 1);
        g[0] = beta;
        for (int i = 1; i <= M; ++i) g[i] = 0.0;
        bk.binv[beam] = beta > 0.0 ? 1.0 / beta : 0.0;
        if (bn > 0.0) rm = fmax(rm, beta / bn);
        if (!conv) ++a;
    }
    act[threadIdx.x] = a;
    rmax[threadIdx.x] = rm;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            act[threadIdx.x] += act[threadIdx.x + o];
            rmax[threadIdx.x] = fmax(rmax[threadIdx.x], rmax[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // the host's test beta <= rtol * bnorm holds exactly when every beam converged
        st->bnorm = 1.0;
        st->beta = act[0] > 0 ? 1.0 : 0.0;
        st->done = act[0] == 0 ? 1 : 0;
        st->jend = 0;
        *bk.relres = rmax[0];
    }
}

__global__ void k_bnorm_init(BKry bk) {
    const int beam = blockIdx.x * blockDim.x + threadIdx.x;
    if (beam < bk.nb) {
        bk.bnorm[beam] = sqrt(bk.r2[beam]);
        bk.conv[beam] = 0;
    }
}

// st->jlast = the longest cycle of any beam (for the host's step count)
__global__ void __launch_bounds__(256) k_bmax_jend(BKry bk, GmresState *st) {
    __shared__ int mx[256];
    int v = 0;
    for (int beam = threadIdx.x; beam < bk.nb; beam += blockDim.x) v = max(v, bk.jend[beam]);
    mx[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) mx[threadIdx.x] = max(mx[threadIdx.x], mx[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) st->jlast = mx[0];
}

// Krylov scratch of one GMRES of element type T
template <class T>
struct Krylov {
    T *V;
    int64_t ldv;
    T *w, *wraw;
    GmresState *st;
    double *partial;
    int nblk;
    int pdeg = 1;                   // degree of the Jacobi-Neumann polynomial (1 = Jacobi)
    double omega = 1.0;
    const __half *hval = nullptr;   // FP16 copy of the matrix for the sweeps (FP32 vectors only)
    // width-sorted FP16 sweep matrix (null: sweep on the ELL)
    const int32_t *sperm = nullptr, *scol = nullptr;
    const uint32_t *ssw = nullptr, *sso = nullptr;
    const __half *sval = nullptr;
    const float *sval32 = nullptr;  // FP32 values of the same copy (Arnoldi products)
    const uint32_t *scol24 = nullptr;   // its chunk columns packed to 24 bits (sweeps), or null
    int64_t skeep = INT64_MAX;          // sweeps: slices from this entry on are read with streaming loads
    int64_t nslot = 0;
    T *z0 = nullptr, *z1 = nullptr, *t = nullptr;   // sweep ping-pong and cycle-end combination
    // flexible basis: Z_j = p(Ahat) v_j kept from step j, so that the cycle ends
    // with u += Z y instead of applying the polynomial to V y once more
    T *Z = nullptr;
    bool graphs = true;             // replay full restart cycles as CUDA graphs
    int *jhint = nullptr;           // Arnoldi steps the last cycle of this system used (cycle cap)
    RowSkip skip{nullptr, nullptr};         // batches: rows of converged beams
    const uint8_t *tact = nullptr;          // batches: tiles holding a row of an unconverged beam
    const BeamMask *mask = nullptr;         // batches: per-beam convergence at every restart
    const BKry *bk = nullptr;               // batches: an independent Krylov space per beam
    const IluDev *ilu = nullptr;            // FP64 comparison solve: (LU)^-1 of ILU(0) instead of the polynomial
};


// z = p(Ahat) v with p(A) = omega sum_{i<d} (I - omega A)^i: d damped Jacobi
// sweeps from z = 0 (the first one is z = omega v).  Returns the buffer
// holding z.  v is read with a full row and the sweeps ping-pong z0/z1; the
// last sweep writes to `last` when it is given.
template <class T>
T *poly_apply(apcloud_ctx *c, const T *val, const T *v, T *z_first, const Krylov<T> &K, GmresState *st,
              RowSkip skip, T *last = nullptr) {
    const int n = c->n_tot;
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    if constexpr (sizeof(T) == 8) {
        if (K.ilu) return ilu_apply(c, *K.ilu, (const double *)v, (double *)z_first, (const GmresState *)st);
    }
    T *cur = z_first, *nxt = (z_first == K.z0) ? K.z1 : K.z0;
    for (int i = 1; i < K.pdeg; ++i) {
        if (last && i + 1 == K.pdeg) nxt = last;   // the last sweep writes where the caller keeps z
        if constexpr (sizeof(T) == 4) {
            if (K.hval && K.sperm) {
                // the first sweep follows the kernel that wrote v and the
                // state; each later one follows a sweep (APC_LAUNCH_PDL)
                const bool pdl = i > 1 && c->pdl_on;
                const float *xc = (const float *)cur;
                float *yn = (float *)nxt;
                const GmresState *sc = (const GmresState *)st;
                if (K.scol24 && K.skeep < c->ss_entries) {
                    if (pdl) APC_SWEEP_BS_PDL(c, K.nslot, APC_SWEEPS24K, K.sperm, K.ssw, K.sso, K.scol, K.sval,
                                              K.nslot, xc, yn, (const float *)v, sc, skip, K.scol24, K.skeep);
                    else APC_SWEEP_BS(c, K.nslot, APC_SWEEPS24K, K.sperm, K.ssw, K.sso, K.scol, K.sval, K.nslot,
                                      xc, yn, (const float *)v, sc, skip, K.scol24, K.skeep);
                } else if (K.scol24) {
                    if (pdl) APC_SWEEP_BS_PDL(c, K.nslot, APC_SWEEPS24, K.sperm, K.ssw, K.sso, K.scol, K.sval,
                                              K.nslot, xc, yn, (const float *)v, sc, skip, K.scol24, K.skeep);
                    else APC_SWEEP_BS(c, K.nslot, APC_SWEEPS24, K.sperm, K.ssw, K.sso, K.scol, K.sval, K.nslot,
                                      xc, yn, (const float *)v, sc, skip, K.scol24, K.skeep);
                } else {
                    if (pdl) APC_SWEEP_BS_PDL(c, K.nslot, APC_SWEEPS, K.sperm, K.ssw, K.sso, K.scol, K.sval,
                                              K.nslot, xc, yn, (const float *)v, sc, skip,
                                              (const uint32_t *)nullptr, (int64_t)0);
                    else APC_SWEEP_BS(c, K.nslot, APC_SWEEPS, K.sperm, K.ssw, K.sso, K.scol, K.sval, K.nslot,
                                      xc, yn, (const float *)v, sc, skip, (const uint32_t *)nullptr, (int64_t)0);
                }
                T *tmp = cur; cur = nxt; nxt = tmp;
                continue;
            }
            if (K.hval) {
                APC_SWEEP_BS(c, n, APC_SWEEPH, sw, so, col, K.hval, n, (const float *)cur,
                           (float *)nxt, (const float *)v, (const GmresState *)st, skip);
                T *tmp = cur; cur = nxt; nxt = tmp;
                continue;
            }
        }
        APC_SWEEP_BS(c, n, APC_SPMV3, sw, so, col, val, n, (const T *)cur, nxt, (T *)nullptr, v, st,
                     (double *)nullptr, skip);
        T *tmp = cur; cur = nxt; nxt = tmp;
    }
    return cur;
}

// the restart residual r = b - Ahat u into K.wraw with beta = ||r||: on the
// packed sorted FP32 copy when the cycle has it, else on the ELL
template <class T>
void residual_launch(apcloud_ctx *c, const T *val, const Krylov<T> &K, const T *u, const T *b, GmresState *st) {
    const int n = c->n_tot;
    if constexpr (sizeof(T) == 4) {
        if (K.pdeg > 1 && K.sval32 && K.sperm && K.scol24) {
            const int nb = resid_blocks(K.nslot);
            if (c->spmv_unroll == 4)
                APC_LAUNCH(c, K_SPMV, nb, RT, 0, k_resid_s<4>, K.sperm, K.ssw, K.sso, K.scol, K.sval32, K.scol24,
                           K.nslot, (const float *)u, (float *)K.wraw, (const float *)b, st, K.partial);
            else
                APC_LAUNCH(c, K_SPMV, nb, RT, 0, k_resid_s<1>, K.sperm, K.ssw, K.sso, K.scol, K.sval32, K.scol24,
                           K.nslot, (const float *)u, (float *)K.wraw, (const float *)b, st, K.partial);
            return;
        }
    }
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    APC_LAUNCH(c, K_SPMV, resid_blocks(n), RT, 0, (k_spmv<2, T>), sw, so, col, val, n, u, K.wraw, (T *)nullptr, b, st,
               K.partial, RowSkip{nullptr, nullptr});
}

// w = Ahat z of a polynomial-preconditioned Arnoldi step (skipped once the
// cycle is done): on the width-sorted FP32 copy when the sweeps use it, else
// on the ELL
template <class T>
void arnoldi_product(apcloud_ctx *c, const T *val, const Krylov<T> &K, const T *z, GmresState *st, RowSkip skip) {
    const int n = c->n_tot;
    if constexpr (sizeof(T) == 4) {
        if (K.sval32 && K.sperm && K.scol24) {
            APC_SPMV_BS(c, K.nslot, APC_SPMVS24, K.sperm, K.ssw, K.sso, K.scol, K.sval32, K.nslot, (const float *)z,
                        (float *)K.w, (const GmresState *)st, skip, K.scol24);
            return;
        }
        if (K.sval32 && K.sperm) {
            APC_SPMV_BS(c, K.nslot, APC_SPMVS, K.sperm, K.ssw, K.sso, K.scol, K.sval32, K.nslot, (const float *)z,
                        (float *)K.w, (const GmresState *)st, skip, (const uint32_t *)nullptr);
            return;
        }
    }
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    APC_SPMV_BS(c, n, APC_SPMV4, sw, so, col, val, n, z, K.w, (T *)nullptr, (const T *)nullptr, st,
                (double *)nullptr, skip);
}

// bnorm .. jlast of GmresState, read back once per restart cycle; jlast is the
// number of columns the cycle completed (the residual product that opens the
// next cycle resets jend)
struct StateTail {
    double bnorm, beta, inv_norm, rtol, omega;
    int jend, done;
    unsigned ticket;
    int jlast;
};
static_assert(sizeof(StateTail) == sizeof(GmresState) - offsetof(GmresState, bnorm), "GmresState tail layout");

__global__ void k_save_jend(GmresState *st) {
    if (threadIdx.x == 0) st->jlast = st->jend;
}

// Direct launches with kernel timers on (the roofline pass) or with graphs
// turned off by the caller (apcloud_set_graphs): the host reads the stopping
// flag after every Arnoldi step and ends the cycle there, so no launch after
// the test is issued or timed.  Captured cycles skip those steps on the
// device instead (IF nodes).  Solves that never use graphs (the ILU(0)
// comparison, the allocation-free solve) launch every step of a cycle.
apcloud_status stop_when_done(apcloud_ctx *c, GmresState *st) {
    c->stopped = false;
    if (c->capturing || (c->timer.mask == 0 && c->graphs_on)) return APCLOUD_OK;
    int done = 0;
    APC_TRY(read_back(c, &done, &st->done, sizeof done));
    c->stopped = done != 0;
    return APCLOUD_OK;
}

// Per-beam Krylov spaces: the residual that opens a cycle gives every beam its
// own beta and stopping test (k_bstart).
template <class T>
apcloud_status bstart_launches(apcloud_ctx *c, const Krylov<T> &K) {
    const BKry &bk = *K.bk;
    beam_sq<T>(c, (const T *)K.wraw, (const int64_t *)ptr<int64_t>(c->beam_rng), bk.nb, bk.r2);
    APC_LAUNCH(c, K_VEC, 1, 256, 0, k_bstart, bk, K.st);
    return cuda_check(c, cudaGetLastError(), "batched restart");
}

// One restart cycle with an independent Krylov space per beam (same launches
// for every beam), the update of u and the residual that opens the next cycle.
// DCGS2 on a batch's per-beam spaces (k_bdcgs_*): FP32 vectors with a
// flexible basis, while a cycle's 2 j + 3 sums per item fit its 64 slots
template <class T>
bool bdcgs_on(const Krylov<T> &K, int jmax) {
    return sizeof(T) == 4 && K.bk && K.pdeg > 1 && K.Z != nullptr && 2 * jmax + 1 <= 64;
}

template <class T>
apcloud_status bcycle_launches(apcloud_ctx *c, const T *val, const T *b, T *u, const Krylov<T> &K, int jmax) {
    const int n = c->n_tot;
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    GmresState *st = K.st;
    const BKry &bk = *K.bk;
    const RowSkip active{bk.nbo, bk.done, bk.binv};
    const bool dcgs = bdcgs_on(K, jmax);
    for (int j = 0; j < jmax; ++j) {
        begin_step(c, j);
        if (K.pdeg <= 1) {
            APC_SPMV_BS(c, n, APC_SPMV1, sw, so, col, val, n, (const T *)K.wraw, K.w, K.V + (int64_t)j * K.ldv,
                        (const T *)nullptr, st, (double *)nullptr, active);
        } else {
            T *vj = K.V + (int64_t)j * K.ldv;
            if (dcgs && j > 0)
                APC_LAUNCH(c, K_UPDNORM, bk.nitems, BGT, 0, k_bdcgs_update<T>, K.V, K.ldv, j, (const T *)K.w,
                           K.z0, bk, (const GmresState *)st);
            else
                APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_bnormalize_first<T>, (const T *)K.wraw, vj, K.z0, n,
                           bk.nbo, (const int *)bk.done, (const double *)bk.binv, (const GmresState *)st);
            T *z = poly_apply<T>(c, val, vj, K.z0, K, st, RowSkip{bk.nbo, bk.done, nullptr},
                                 K.Z ? K.Z + (int64_t)j * K.ldv : nullptr);
            arnoldi_product<T>(c, val, K, (const T *)z, st, RowSkip{bk.nbo, bk.done, nullptr});
        }
        if constexpr (sizeof(T) == 4) {
            if (dcgs) {   // one pass and one sum per step (k_bdcgs_*)
                APC_LAUNCH(c, K_DOT, bk.nitems, BGT, 0, k_bdcgs_dots<T>, (const T *)K.V, K.ldv, j, (const T *)K.w,
                           bk, (const GmresState *)st, K.partial);
                APC_LAUNCH(c, K_DOT, bk.nb, 64, 0, k_bdcgs_sum, j, bk, (const GmresState *)st,
                           (const double *)K.partial);
                APC_LAUNCH(c, K_DOT, 1, 256, 0, k_bdcgs_tail, j, bk, st, next_step_cond(c, j),
                           (c->capturing && j + 1 < jmax) ? 1 : 0);
                end_step(c);
                APC_TRY(stop_when_done(c, st));
                if (c->stopped) break;
                continue;
            }
        }
        APC_LAUNCH(c, K_DOT, bk.nitems, BGT, 0, (k_bgs_dots<0, T>), (const T *)K.V, K.ldv, j, K.w, bk,
                   (const GmresState *)st, K.partial);
        APC_LAUNCH(c, K_DOT, bk.nb, 64, 0, k_bfinal_h<0>, j, bk, (const GmresState *)st, (const double *)K.partial);
        APC_LAUNCH(c, K_UPDDOT, bk.nitems, BGT, 0, (k_bgs_dots<1, T>), (const T *)K.V, K.ldv, j, K.w, bk,
                   (const GmresState *)st, K.partial);
        APC_LAUNCH(c, K_UPDDOT, bk.nb, 64, 0, k_bfinal_h<1>, j, bk, (const GmresState *)st,
                   (const double *)K.partial);
        APC_LAUNCH(c, K_UPDNORM, bk.nitems, BGT, 0, k_bgs_norm<T>, (const T *)K.V, K.ldv, j, (const T *)K.w, K.wraw,
                   bk, (const GmresState *)st, K.partial);
        APC_LAUNCH(c, K_UPDNORM, 1, 256, 0, k_bfinal_norm, j, bk, st, (const double *)K.partial,
                   next_step_cond(c, j), (c->capturing && j + 1 < jmax) ? 1 : 0);
        end_step(c);
        APC_TRY(stop_when_done(c, st));
        if (c->stopped) break;
    }
    APC_LAUNCH(c, K_CYCLE, div_up(bk.nb, 64), 64, 0, k_bsolve_y, bk);
    if (K.pdeg <= 1 || K.Z) {
        APC_LAUNCH(c, K_CYCLE, bk.nitems, BGT, 0, (k_bcombine<true, T>), (const T *)(K.Z ? K.Z : K.V), K.ldv, u,
                   bk);
    } else {
        // u += p(Ahat) (V y), beam by beam; beams converged before this cycle are skipped
        APC_LAUNCH(c, K_CYCLE, bk.nitems, BGT, 0, (k_bcombine<false, T>), (const T *)K.V, K.ldv, K.t, bk);
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_axpy_first<T>, (const T *)K.t, K.z0, n,
                   (const GmresState *)st);
        GmresState *stp = st;
        APC_CUDA(c, cudaMemsetAsync(&stp->done, 0, sizeof(int), c->s));
        T *z = poly_apply<T>(c, val, K.t, K.z0, K, st, RowSkip{bk.nbo, bk.conv, nullptr});
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_add<T>, u, (const T *)z, n);
    }
    APC_LAUNCH(c, K_VEC, 1, 256, 0, k_bmax_jend, bk, st);
    residual_launch<T>(c, val, K, (const T *)u, b, st);
    APC_TRY(bstart_launches<T>(c, K));
    return cuda_check(c, cudaGetLastError(), "batched gmres cycle");
}

// A single-beam polynomial (or ILU) cycle closes each Arnoldi step with the
// second Gram-Schmidt pass and the norm in one sweep (k_gs_dots PASS 2) and
// opens the next with the second update and the normalisation in one
// (k_gs_update_normalize): two reductions and three passes over the basis
// per step.  Jacobi cycles normalise inside their product and batches skip
// converged tiles, so they keep the separate norm pass.
template <class T>
bool gs_fused(const Krylov<T> &K, int jmax) {
    return K.pdeg > 1 && !K.bk && !K.tact && !K.skip.nbo && jmax < MAX_RESTART;
}

// DCGS2 (k_dcgs_dots) on the same cycles when they keep the flexible basis
// (Z_j = p(Ahat) q_j of the tentative q_j; the cycle end without it applies
// the polynomial to V y, which needs Z = p(Ahat) V) and while its 2 j + 3
// sums per block fit the 64 partial slots of a block
template <class T>
bool gs_dcgs(const Krylov<T> &K, int jmax) {
    return sizeof(T) == 4 && gs_fused(K, jmax) && K.Z != nullptr && 2 * jmax + 1 <= 64;
}

// One restart cycle of jmax Arnoldi steps, the update of u, and the residual
// b - Ahat u that opens the next cycle (beta, g, done for it).
template <class T>
apcloud_status cycle_launches(apcloud_ctx *c, const T *val, const T *b, T *u, const Krylov<T> &K, int jmax) {
    const int n = c->n_tot;
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    GmresState *st = K.st;
    if (K.bk) return bcycle_launches<T>(c, val, b, u, K, jmax);
    const bool dcgs = gs_dcgs(K, jmax);
    const bool fused = gs_fused(K, jmax) && !dcgs;
    for (int j = 0; j < jmax; ++j) {
        begin_step(c, j);
        if (K.pdeg <= 1) {
            APC_SPMV_BS(c, n, APC_SPMV1, sw, so, col, val, n, (const T *)K.wraw, K.w, K.V + (int64_t)j * K.ldv,
                        (const T *)nullptr, st, (double *)nullptr, K.skip);
        } else {
            // w = Ahat p(Ahat) v_j (right preconditioning)
            T *vj = K.V + (int64_t)j * K.ldv;
            if (dcgs && j > 0)
                APC_LAUNCH(c, K_UPDNORM, stream_blocks(K.ldv), GT, 0, k_dcgs_update<T>, K.V, K.ldv, (int)K.ldv, j,
                           (const T *)K.w, K.z0, (const GmresState *)st);
            else if (fused && j > 0)
                APC_LAUNCH(c, K_UPDNORM, stream_blocks(K.ldv), GT, 0, k_gs_update_normalize<T>, (const T *)K.V,
                           K.ldv, (int)K.ldv, j, (const T *)K.w, vj, K.z0, (const GmresState *)st);
            else
                APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_normalize_first<T>, (const T *)K.wraw, vj, K.z0, n,
                           (const GmresState *)st);
            T *z = poly_apply<T>(c, val, vj, K.z0, K, st, K.skip, K.Z ? K.Z + (int64_t)j * K.ldv : nullptr);
            arnoldi_product<T>(c, val, K, (const T *)z, st, K.skip);
        }
        const int set_next = (c->capturing && j + 1 < jmax) ? 1 : 0;
        if constexpr (sizeof(T) == 4) {
            if (dcgs) {
                APC_LAUNCH(c, K_DOT, dot_blocks(K.ldv), DT, 0, k_dcgs_dots<T>, (const T *)K.V, K.ldv, (int)K.ldv, j,
                           (const T *)K.w, st, K.partial, next_step_cond(c, j), set_next);
                end_step(c);
                APC_TRY(stop_when_done(c, st));
                if (c->stopped) break;
                continue;
            }
        }
        gs_dispatch<T>(c, 0, K.nblk, K.V, K.ldv, j, K.w, K.wraw, st, K.partial, K.tact);
        if (fused) {
            gs_dispatch<T>(c, 3, K.nblk, K.V, K.ldv, j, K.w, K.wraw, st, K.partial, K.tact, next_step_cond(c, j),
                           set_next);
        } else {
            gs_dispatch<T>(c, 1, K.nblk, K.V, K.ldv, j, K.w, K.wraw, st, K.partial, K.tact);
            gs_dispatch<T>(c, 2, K.nblk, K.V, K.ldv, j, K.w, K.wraw, st, K.partial, K.tact, next_step_cond(c, j),
                           set_next);
        }
        end_step(c);
        APC_TRY(stop_when_done(c, st));
        if (c->stopped) break;
    }
    if (K.pdeg <= 1 || K.Z) {
        // u += V y (Jacobi: the preconditioner is in the stored matrix) or u += Z y
        APC_LAUNCH(c, K_CYCLE, stream_blocks(K.ldv), GT, 0, k_cycle_end<T>, (const T *)(K.Z ? K.Z : K.V), K.ldv,
                   (int)K.ldv, u, (const GmresState *)st);
    } else {
        // u += p(Ahat) (V y)
        APC_LAUNCH(c, K_CYCLE, stream_blocks(K.ldv), 256, 0, k_combine<T>, (const T *)K.V, K.ldv, n, K.t,
                   (const GmresState *)st);
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_axpy_first<T>, (const T *)K.t, K.z0, n,
                   (const GmresState *)st);
        // the sweeps must run even though the cycle is done: clear the flag for them
        GmresState *stp = st;
        APC_CUDA(c, cudaMemsetAsync(&stp->done, 0, sizeof(int), c->s));
        T *z = poly_apply<T>(c, val, K.t, K.z0, K, st, K.skip);
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_add<T>, u, (const T *)z, n);
    }
    // the next cycle's residual keeps this cycle's column count: save it first
    APC_LAUNCH(c, K_VEC, 1, 32, 0, k_save_jend, st);
    residual_launch<T>(c, val, K, (const T *)u, b, st);
    if (K.mask) APC_TRY(mask_residual<T>(c, *K.mask, K.wraw, st));
    return cuda_check(c, cudaGetLastError(), "gmres cycle");
}

template <class T>
apcloud_status run_cycle(apcloud_ctx *c, const T *val, const T *b, T *u, const Krylov<T> &K, int jmax, bool graph) {
    if (graph && c->graphs_on && c->timer.mask == 0) {
        GraphKey key;
        memset(&key, 0, sizeof key);
        key.tsize = (int)sizeof(T);
        key.n = c->n_tot;
        key.jmax = jmax;
        key.pdeg = K.pdeg;
        key.nblk = K.nblk;
        key.ldv = K.ldv;
        key.mask = c->timer.mask;
        key.spmv_bs = c->spmv_bs * 8 + c->spmv_unroll;
        key.skeep = K.skeep;
        key.pdl = c->pdl_on ? 1 : 0;
        const void *p[] = {val, b, u, K.V, K.w, K.wraw, K.st, K.partial, K.z0, K.z1, K.t, K.hval,
                           c->slice_w.p, c->slice_off.p, c->ell_col.p, K.skip.nbo, K.skip.bdone, K.tact,
                           K.mask ? K.mask->r2 : nullptr, K.bk ? K.bk->items : nullptr,
                           K.bk ? K.bk->H : nullptr, K.bk ? K.bk->done : nullptr,
                           K.bk ? (const void *)(intptr_t)K.bk->nitems : nullptr, K.sperm, K.sval, K.scol, K.ssw,
                           K.sso, K.Z, K.sval32, K.scol24};
        static_assert(sizeof p <= sizeof key.p, "graph key holds every buffer address");
        for (size_t i = 0; i < sizeof p / sizeof p[0]; ++i) key.p[i] = p[i];
        GraphEntry *g = find_graph(c, key);
        if (!g) {
            g = begin_capture(c, key);
            if (g) {
                apcloud_status st = cycle_launches<T>(c, val, b, u, K, jmax);
                g = end_capture(c, g, st);
            }
        }
        if (g) return launch_graph(c, g);
    }
    return cycle_launches<T>(c, val, b, u, K, jmax);
}

// Restarted GMRES(restart) on Ahat u = b, u in/out; no allocation.  Returns
// OK when ||b - Ahat u|| <= rtol ||b||, W_NOT_CONVERGED at max_iter.
template <class T>
apcloud_status gmres_core(apcloud_ctx *c, const T *val, const T *b, T *u, double rtol, int max_iter,
                          const Krylov<T> &K, int *iters_out, int *cycles_out, double *relres_out) {
    const int n = c->n_tot;
    const int m = c->P.restart;
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    GmresState *st = K.st;
    APC_CUDA(c, cudaMemsetAsync(st, 0, sizeof(GmresState), c->s));
    // basis and work vectors are processed in whole 16-byte chunks up to ldv: zero tails
    APC_CUDA(c, cudaMemsetAsync(K.V, 0, sizeof(T) * (size_t)(m + 1) * K.ldv, c->s));
    APC_CUDA(c, cudaMemsetAsync(K.w, 0, sizeof(T) * (size_t)K.ldv, c->s));
    APC_CUDA(c, cudaMemsetAsync(K.wraw, 0, sizeof(T) * (size_t)K.ldv, c->s));
    APC_CUDA(c, cudaMemcpyAsync(&st->rtol, &rtol, sizeof(double), cudaMemcpyHostToDevice, c->s));
    APC_CUDA(c, cudaMemcpyAsync(&st->omega, &K.omega, sizeof(double), cudaMemcpyHostToDevice, c->s));
    APC_LAUNCH(c, K_VEC, K.nblk, RT, 0, k_norm2<T>, b, n, st, K.partial);
    int iters = 0, cycles = 0;
    double relres = 0.0;
    apcloud_status status = APCLOUD_W_NOT_CONVERGED;
    const double vb = (double)sizeof(T), nnz = (double)c->sum_m + (double)c->n_int + (double)c->n_bnd, dn = n;
    residual_launch<T>(c, val, K, (const T *)u, b, st);
    if (K.mask) APC_TRY(mask_residual<T>(c, *K.mask, K.wraw, st));
    if (K.bk) {
        // per-beam ||b_b|| once, then every beam's first cycle
        beam_sq<T>(c, b, (const int64_t *)ptr<int64_t>(c->beam_rng), K.bk->nb, K.bk->r2);
        APC_LAUNCH(c, K_VEC, div_up(K.bk->nb, 64), 64, 0, k_bnorm_init, *K.bk);
        APC_TRY(bstart_launches<T>(c, K));
    }
    StateTail tail;
    APC_TRY(read_back(c, &tail, &st->bnorm, sizeof tail));
    for (;;) {
        relres = tail.bnorm > 0.0 ? tail.beta / tail.bnorm : 0.0;
        if (tail.bnorm == 0.0 || tail.beta <= rtol * tail.bnorm) { status = APCLOUD_OK; break; }
        if (iters >= max_iter) break;
        // A cycle ends at the stopping test or after m steps; its launches are
        // fixed in advance (graph), so steps past the test are empty launches.
        // Systems that converge in a few steps per cycle (the density system)
        // get a cycle of at most 2 j + 2 steps after one that needed j.
        int cap = m;
        if (K.jhint && *K.jhint > 0) cap = std::min(m, std::max(4, 2 * *K.jhint + 2));
        const int jmax = (cap < max_iter - iters) ? cap : (max_iter - iters);
        // one restart cycle and the next restart's residual: a CUDA graph replay
        // when the cycle is a full one, otherwise direct launches
        APC_TRY(run_cycle<T>(c, val, b, u, K, jmax, jmax == cap && K.graphs));
        APC_TRY(read_back(c, &tail, &st->bnorm, sizeof tail));
        const int je = tail.jlast;
        count_replayed_steps(c, je);
        // algorithmic traffic of the launches that did work (values + column index per entry)
        {
            // per Arnoldi step: one product with the full matrix, pdeg - 1 sweeps (FP16
            // values when available); the cycle end adds pdeg - 1 sweeps, the restart one product
            const double sweeps = (K.pdeg <= 1 || K.ilu) ? 0.0 : (double)(K.pdeg - 1) * (je + (K.Z ? 0 : 1));
            const double prods = je + 1.0;
            const double sb = K.hval ? 2.0 : vb;
            const double cb = K.scol24 ? 3.0 : 4.0;   // column bytes per entry read by a sweep
            // Arnoldi products and the restart residual (24-bit columns on the packed sorted copy)
            const double pcb = (K.pdeg > 1 && K.sval32 && K.scol24) ? 3.0 : 4.0;
            account(c, K_SPMV, ((vb + pcb) * nnz + 2.0 * vb * dn) * prods, 2.0 * nnz * prods);
            account(c, K_SWEEP, ((sb + cb) * nnz + 3.0 * vb * dn) * sweeps, 2.0 * nnz * sweeps);
        }
        const bool dcgs = gs_dcgs(K, jmax) || bdcgs_on(K, jmax), fused = gs_fused(K, jmax) && !dcgs;
        for (int j = 0; j < je; ++j) {
            if (dcgs) {
                // one pass over j basis vectors, q_j and w; step j >= 1 opened by one
                // pass over j - 1 basis vectors, q_{j-1} and w, writing v_{j-1}, q_j, z
                account(c, K_DOT, vb * dn * (j + 2), 4.0 * dn * j + 6.0 * dn);
                if (j > 0) account(c, K_UPDNORM, vb * dn * (j + 1 + 3), 4.0 * dn * (j - 1) + 4.0 * dn);
                continue;
            }
            account(c, K_DOT, vb * dn * (j + 2), 2.0 * dn * (j + 1));
            if (fused) {
                // PASS 2 with its sum of squares; step j >= 1 opened with w - V h2 over
                // its j predecessors, written to V_j and z
                account(c, K_UPDDOT, vb * dn * (j + 3), 4.0 * dn * (j + 1) + 2.0 * dn);
                if (j > 0) account(c, K_UPDNORM, vb * dn * (j + 3), 2.0 * dn * (j + 1));
            } else {
                account(c, K_UPDDOT, vb * dn * (j + 3), 4.0 * dn * (j + 1));
                account(c, K_UPDNORM, vb * dn * (j + 3), 2.0 * dn * (j + 2));
            }
        }
        account(c, K_CYCLE, vb * dn * (je + 2), 2.0 * dn * je);
        iters += je;
        if (K.jhint) *K.jhint = je;
        ++cycles;
        if (je == 0) {
            relres = tail.bnorm > 0.0 ? tail.beta / tail.bnorm : 0.0;
            if (tail.bnorm == 0.0 || tail.beta <= rtol * tail.bnorm) status = APCLOUD_OK;
            break;
        }
    }
    if (K.bk) {   // largest relative residual over the beams
        double rr;
        APC_TRY(read_back(c, &rr, K.bk->relres, sizeof rr));
        relres = rr;
    }
    *iters_out = iters;
    *cycles_out = cycles;
    *relres_out = relres;
    return status;
}

}  // namespace

apcloud_status deposit(apcloud_ctx *c, const double *q, double q_uniform) {
    const int n = c->n_int, nt = c->n_tot;
    double *rm = ensure<double>(c, c->rho_m, nt + 1);
    if (!rm) return APCLOUD_E_NOMEM;
    const double ext = c->P.hi[0] - c->P.lo[0];
    double *qs = nullptr;
    if (q && c->N > 0) {
        qs = ensure<double>(c, c->qsort, c->N);
        if (!qs) return APCLOUD_E_NOMEM;
        APC_LAUNCH(c, K_DEPOSIT, div_up(c->N, 256 * CS_PER), 256, 0, k_charge_sort, q,
                   (const int32_t *)ptr<int32_t>(c->spos), c->N, qs);
    }
    APC_LAUNCH(c, K_DEPOSIT, div_up(n, 256), 256, 0, k_deposit, (const double *)qs, q_uniform,
               ptr<int32_t>(c->leaf_first), ptr<int32_t>(c->leaf_count), ptr<int4>(c->node_ic), n,
               1.0 / (ext * ext * ext), rm);
    APC_LAUNCH(c, K_DEPOSIT, div_up(c->n_bnd, 256), 256, 0, k_bcopy, ptr<int32_t>(c->bowner), n, c->n_bnd, rm);
    // sorted position and charge per particle, rho_M per node
    account(c, K_DEPOSIT, (q ? 12.0 * c->N : 0.0) + 8.0 * nt, q ? (double)c->N : (double)n);
    return cuda_check(c, cudaGetLastError(), "deposit");
}

apcloud_status spmv(apcloud_ctx *c, int which, const double *x, double *y, double scale, double *copy_out) {
    (void)scale; (void)copy_out;
    const double *val = ptr<double>(which ? c->ell_A : c->ell_B);
    const int n = c->n_tot;
    APC_LAUNCH(c, K_SPMV, div_up(n, RT), RT, 0, (k_spmv<0, double>), ptr<uint32_t>(c->slice_w),
               ptr<uint32_t>(c->slice_off), ptr<int32_t>(c->ell_col), val, n, x, y, (double *)nullptr,
               (const double *)nullptr, (GmresState *)nullptr, (double *)nullptr, RowSkip{nullptr, nullptr});
    return cuda_check(c, cudaGetLastError(), "spmv");
}

// Solve (B or A) x = b.  On entry x holds the initial guess (unscaled); on
// exit the solution.  FP64 form: GMRES(restart) on Ahat u = b in FP64.
// Mixed form: iterative refinement -- the residual r = b - Ahat u is formed
// in FP64 with the FP64 matrix, the correction Ahat e = r gets one FP32
// GMRES(restart) cycle on the FP32 copy of the matrix (stopping early at a
// relative 1e-4 or what the outer tolerance still needs), and u += e in FP64:
// restarted GMRES whose restarts recompute the residual in FP64.
apcloud_status gmres_solve(apcloud_ctx *c, int which, const double *b, double *x, double rtol, int max_iter,
                           apcloud_solve_info *info) {
    const int n = c->n_tot;
    const int m = c->P.restart;
    const int64_t ldv = ((int64_t)n + 31) / 32 * 32;
    const int nblk = reduction_blocks(c, n);
    const int64_t npart = (int64_t)(div_up(n, RT) + 2 * nblk) * 64;
    double *u = ensure<double>(c, c->u, ldv + 1);
    double *partial = ensure<double>(c, c->partial, npart);
    if (!u || !partial) return APCLOUD_E_NOMEM;
    const double *val = ptr<double>(which ? c->ell_A : c->ell_B);
    const double *d = ptr<double>(which ? c->dA : c->dB);
    // batch: every beam has its own Krylov space and stops at its own
    // rtol ||b_b|| (BKry); the FP64 refinement loop of the mixed form freezes
    // converged beams (BeamMask)
    BeamMask bmv{};
    const BeamMask *bm = nullptr;
    BKry bkv{};
    const BKry *bk = nullptr;
    if (c->nbeams > 1) {
        const int nb = c->nbeams;
        const int64_t ntile = div_up(ldv, TILE);
        double *b2 = ensure<double>(c, c->beam_norm, nb), *r2 = ensure<double>(c, c->beam_r2, nb);
        int *bdone = ensure<int>(c, c->beam_done, nb);
        int32_t *nbo = ensure<int32_t>(c, c->node_beam, n);
        uint8_t *tact = ensure<uint8_t>(c, c->tile_act, ntile);
        double *bpart = ensure<double>(c, c->beam_part, (int64_t)nb * BSQ_CH);
        if (!b2 || !r2 || !bdone || !nbo || !tact || !bpart) return APCLOUD_E_NOMEM;
        APC_TRY(node_beams(c, nbo));
        APC_CUDA(c, cudaMemsetAsync(bdone, 0, sizeof(int) * nb, c->s));
        APC_CUDA(c, cudaMemsetAsync(tact, 1, ntile, c->s));
        const int64_t *rng = ptr<int64_t>(c->beam_rng);
        beam_sq<double>(c, b, rng, nb, b2);
        bmv = BeamMask{nb, rng, b2, r2, bdone, nbo, tact, ntile, rtol};
        bm = &bmv;
        // work items of the per-beam Krylov spaces: chunks of at most BITEM rows
        // inside each beam's 7 node ranges, grouped by beam
        std::vector<int64_t> hr(7 * (size_t)(nb + 1));
        APC_TRY(read_back(c, hr.data(), rng, sizeof(int64_t) * hr.size()));
        std::vector<int4> items;
        std::vector<int> ioff(nb + 1, 0);
        for (int bb = 0; bb < nb; ++bb) {
            ioff[bb] = (int)items.size();
            for (int seg = 0; seg < 7; ++seg) {
                const int64_t lo = hr[(size_t)seg * (nb + 1) + bb], hi = hr[(size_t)seg * (nb + 1) + bb + 1];
                for (int64_t a = lo; a < hi; a += BITEM)
                    items.push_back(make_int4(bb, (int)a, (int)(a + BITEM < hi ? a + BITEM : hi), 0));
            }
        }
        ioff[nb] = (int)items.size();
        const int ni = (int)items.size();
        int4 *ditems = ensure<int4>(c, c->bk_items, ni > 0 ? ni : 1);
        int *dioff = ensure<int>(c, c->bk_ioff, nb + 1);
        const int64_t per = (int64_t)(m + 1) * m + 2 * m + 3 * (m + 1) + m + 3 + (m + 1) + 4 + 64;
        double *dd = ensure<double>(c, c->bk_d, per * nb + 1);
        int *di = ensure<int>(c, c->bk_i, 3 * (int64_t)nb);
        double *part2 = ensure<double>(c, c->partial, std::max<int64_t>(npart, (int64_t)ni * 64), true);
        if (!ditems || !dioff || !dd || !di || !part2) return APCLOUD_E_NOMEM;
        partial = part2;
        if (ni > 0)
            APC_CUDA(c, cudaMemcpyAsync(ditems, items.data(), sizeof(int4) * ni, cudaMemcpyHostToDevice, c->s));
        APC_CUDA(c, cudaMemcpyAsync(dioff, ioff.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, c->s));
        APC_CUDA(c, cudaStreamSynchronize(c->s));   // the host vectors go out of scope
        double *q = dd;
        bkv.nb = nb; bkv.nitems = ni; bkv.m = m;
        bkv.items = ditems; bkv.item_off = dioff; bkv.nbo = nbo;
        bkv.H = q; q += (int64_t)(m + 1) * m * nb;
        bkv.cs = q; q += (int64_t)m * nb;
        bkv.sn = q; q += (int64_t)m * nb;
        bkv.g = q; q += (int64_t)(m + 1) * nb;
        bkv.h1 = q; q += (int64_t)(m + 1) * nb;
        bkv.h2 = q; q += (int64_t)(m + 1) * nb;
        bkv.y = q; q += (int64_t)m * nb;
        bkv.bnorm = q; q += nb;
        bkv.binv = q; q += nb;
        bkv.r2 = q; q += nb;
        bkv.relres = q; q += nb;
        bkv.dq = q; q += (int64_t)(m + 1) * nb;
        bkv.nu = q; q += nb;
        bkv.inu = q; q += nb;
        bkv.nut = q; q += nb;
        bkv.gpre = q; q += nb;
        bkv.fs = q;
        bkv.done = di; bkv.conv = di + nb; bkv.jend = di + 2 * nb;
        bk = &bkv;
    }
    APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_mul, u, (const double *)x, d, n);
    // cycle caps learn within this solve only: a solve does not depend on earlier ones
    c->jprev[which][0] = c->jprev[which][1] = 0;
    int iters = 0, cycles = 0;
    double relres = 0.0;
    apcloud_status status;
    if (c->P.precision == 0) {
        Krylov<double> K{ensure<double>(c, c->V, (int64_t)(m + 1) * ldv), ldv, ensure<double>(c, c->w0, ldv + 1),
                         ensure<double>(c, c->w1, ldv + 1), ptr<GmresState>(c->gstate), partial, nblk};
        if (!K.V || !K.w || !K.wraw) return APCLOUD_E_NOMEM;
        const bool ilu = c->ilu_which == which && !bm;
        if (c->P.poly_degree > 1 || ilu) {
            // the ILU(0) comparison takes the polynomial's place: one application per step
            K.pdeg = ilu ? 2 : c->P.poly_degree;
            K.omega = c->P.poly_omega;
            K.z0 = ensure<double>(c, c->pz0, ldv + 1);
            K.z1 = ensure<double>(c, c->pz1, ldv + 1);
            K.t = ensure<double>(c, c->pt, ldv + 1);
            if (!K.z0 || !K.z1 || !K.t) return APCLOUD_E_NOMEM;
            if (!ilu) {
                K.Z = ensure<double>(c, c->zbasis, (int64_t)m * ldv);
                if (!K.Z) return APCLOUD_E_NOMEM;
            }
            if (ilu) {
                K.ilu = &c->ilu;
                K.graphs = false;   // thousands of level launches per step
            }
        }
        if (bk && K.pdeg > 1) {
            K.bk = bk;
        } else if (bm) {
            // Jacobi alone: restarted GMRES(30) on a single small beam can stall where the
            // shared space of the whole batch does not, so the batch keeps one Krylov
            // space and freezes converged beams at restarts
            K.mask = bm;
            K.skip = RowSkip{bm->nbo, bm->bdone, nullptr};
            K.tact = bm->tact;
        }
        K.jhint = &c->jprev[which][0];
        status = gmres_core<double>(c, val, b, u, rtol, max_iter, K, &iters, &cycles, &relres);
        if (status < 0) return status;
    } else {
        Krylov<float> K{ensure<float>(c, c->V32, (int64_t)(m + 1) * ldv), ldv, ensure<float>(c, c->w32a, ldv + 1),
                        ensure<float>(c, c->w32b, ldv + 1), ptr<GmresState>(c->gstate), partial, nblk};
        float *r32 = ensure<float>(c, c->r32, n + 1), *e32 = ensure<float>(c, c->e32, ldv + 1);
        double *r64 = ensure<double>(c, c->w0, n + 1);
        GmresState *so = ensure<GmresState>(c, c->gstate2, 1);
        if (!K.V || !K.w || !K.wraw || !r32 || !e32 || !r64 || !so) return APCLOUD_E_NOMEM;
        if (c->P.poly_degree > 1) {
            K.pdeg = c->P.poly_degree;
            K.omega = c->P.poly_omega;
            K.hval = ptr<__half>(which ? c->ell_A16 : c->ell_B16);
            if (c->ss_ok && c->sweep_sorted) {
                K.sperm = ptr<int32_t>(c->ss_perm);
                K.ssw = ptr<uint32_t>(c->ss_w);
                K.sso = ptr<uint32_t>(c->ss_o);
                K.scol = ptr<int32_t>(c->ss_col);
                K.sval = ptr<__half>(which ? c->ss_A : c->ss_B);
                K.sval32 = ptr<float>(which ? c->ss_A32 : c->ss_B32);
                if (c->ss_col24_ok) K.scol24 = ptr<uint32_t>(c->ss_col24);
                K.skeep = sweep_keep_entries(c);
                K.nslot = (int64_t)div_up(c->n_tot, 256) * 256;
            }
            K.z0 = ensure<float>(c, c->pz0, ldv + 1);
            K.z1 = ensure<float>(c, c->pz1, ldv + 1);
            K.t = ensure<float>(c, c->pt, ldv + 1);
            K.Z = ensure<float>(c, c->zbasis, (int64_t)m * ldv);
            if (!K.z0 || !K.z1 || !K.t || !K.Z) return APCLOUD_E_NOMEM;
        }
        if (bk && K.pdeg > 1) {
            K.bk = bk;   // beams frozen by the outer loop have zero residual: their inner spaces stop at once
        } else if (bm) {
            K.skip = RowSkip{bm->nbo, bm->bdone, nullptr};
            K.tact = bm->tact;
        }
        K.jhint = &c->jprev[which][1];
        const float *val32 = ptr<float>(which ? c->ell_A32 : c->ell_B32);
        const uint32_t *sw = ptr<uint32_t>(c->slice_w), *sof = ptr<uint32_t>(c->slice_off);
        const int32_t *col = ptr<int32_t>(c->ell_col);
        APC_CUDA(c, cudaMemsetAsync(so, 0, sizeof(GmresState), c->s));
        APC_CUDA(c, cudaMemcpyAsync(&so->rtol, &rtol, sizeof(double), cudaMemcpyHostToDevice, c->s));
        APC_CUDA(c, cudaMemsetAsync(e32, 0, sizeof(float) * ldv, c->s));
        APC_LAUNCH(c, K_VEC, nblk, RT, 0, k_norm2<double>, b, n, so, partial);
        status = APCLOUD_W_NOT_CONVERGED;
        for (;;) {
            APC_LAUNCH(c, K_SPMV, resid_blocks(n), RT, 0, (k_spmv<2, double>), sw, sof, col, val, n,
                       (const double *)u, r64, (double *)nullptr, b, so, partial, RowSkip{nullptr, nullptr});
            if (bm) APC_TRY(mask_residual<double>(c, *bm, r64, so));
            double tmp[2];
            APC_TRY(read_back(c, tmp, &so->bnorm, 2 * sizeof(double)));
            relres = tmp[0] > 0.0 ? tmp[1] / tmp[0] : 0.0;
            if (tmp[0] == 0.0 || tmp[1] <= rtol * tmp[0]) { status = APCLOUD_OK; break; }
            if (iters >= max_iter) break;
            APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_to_f32, r32, (const double *)r64, n);
            // one FP32 restart cycle per refinement step: FP32 residuals bottom out
            // near kappa * 6e-8, so the FP64 residual takes over after each cycle
            double inner = 0.5 * rtol * tmp[0] / tmp[1];
            if (inner < 1e-4) inner = 1e-4;
            const int cap = (m < max_iter - iters) ? m : (max_iter - iters);
            int it = 0, cy = 0;
            double rr = 0.0;
            apcloud_status si = gmres_core<float>(c, val32, r32, e32, inner, cap, K, &it, &cy, &rr);
            if (si < 0) return si;
            APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_add_f32, u, e32, n);
            iters += it;
            cycles += cy;
            if (it == 0) break;
        }
    }
    APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_div, x, (const double *)u, d, n);
    APC_CUDA(c, cudaGetLastError());
    if (info) {
        info->iters = iters;
        info->restarts = cycles;
        info->relres = relres;
    }
    return status;
}

// Times the preconditioner sweep of the active form (FP16 values and FP32
// vectors in the mixed form, else the matrix's own type; the plain Arnoldi
// product when the preconditioner is Jacobi) at each block size and keeps the
// fastest.  Contents of the work vectors do not matter for the timing.
// right-hand side of the autotuner's solves: 1 + (i mod 7) / 10
__global__ void k_tune_rhs(double *b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = 1.0 + 0.1 * (double)(i % 7);
}

// The row-parallel products are timed where they run: for every launch
// shape, one untimed solve (it captures the cycle graphs) and one timed solve
// of the Poisson system with the configured solver, to a relative residual of
// 1e-10 or TUNE_STEPS Arnoldi steps.  Timed in isolation, or over a single
// restart cycle, the shapes rank differently from a whole solve (shorter
// capped cycles, and in a batch the beams converge one by one and their rows
// then return at once).  The graphs the solves capture are released.
constexpr int TUNE_STEPS = 1000;

apcloud_status tune_spmv(apcloud_ctx *c, double *ms_out) {
    const int n = c->n_tot;
    const bool mixed = c->P.precision == 1;
    double *tb = ensure<double>(c, c->tune_b, n + 1), *tx = ensure<double>(c, c->tune_x, n + 1);
    if (!tb || !tx) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_tune_rhs, tb, n);
    const int sizes[4] = {64, 128, 256, 512}, unrolls[2] = {1, 4};
    const int saved = c->spmv_bs, saved_u = c->spmv_unroll, saved_s = c->sweep_sorted;
    int pick = saved, pick_u = saved_u, pick_s = saved_s;
    // the width-sorted sweep matrix is a third dimension when it exists
    const int nvar = (mixed && c->P.poly_degree > 1 && c->ss_ok) ? 16 : 8;
    cudaEvent_t e0, e1;
    APC_CUDA(c, cudaEventCreate(&e0));
    APC_CUDA(c, cudaEventCreate(&e1));
    const unsigned mask = c->timer.mask;
    c->timer.mask = 0;
    double best = 1e30;
    apcloud_status rc = APCLOUD_OK;
    for (int tu = 0; tu < nvar && rc == APCLOUD_OK; ++tu) {
        const int t = tu & 3;
        c->spmv_bs = sizes[t];
        c->spmv_unroll = unrolls[(tu >> 2) & 1];
        c->sweep_sorted = tu >> 3;
        // a capture pass, then the best of two timed passes: shapes that differ by
        // ~1% of a solve were ranked by single timings at random
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && rc == APCLOUD_OK; ++rep) {
            apcloud_solve_info info{};
            rc = cuda_check(c, cudaMemsetAsync(tx, 0, sizeof(double) * n, c->s), "autotune");
            if (rc != APCLOUD_OK) break;
            cudaEventRecord(e0, c->s);
            rc = gmres_solve(c, 1, tb, tx, 1e-10, TUNE_STEPS, &info);
            if (rc < 0) break;
            rc = APCLOUD_OK;
            cudaEventRecord(e1, c->s);
            rc = cuda_check(c, cudaEventSynchronize(e1), "autotune solve");
            if (rc != APCLOUD_OK) break;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0 && t < ms) ms = t;
        }
        if (rc != APCLOUD_OK) break;
        if (ms_out) ms_out[tu] = ms;
        if (ms < best) { best = ms; pick = sizes[t]; pick_u = unrolls[(tu >> 2) & 1]; pick_s = tu >> 3; }
    }
    free_graphs(c);
    c->jprev[1][0] = c->jprev[1][1] = 0;
    c->timer.mask = mask;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->spmv_bs = (rc == APCLOUD_OK) ? pick : saved;
    c->spmv_unroll = (rc == APCLOUD_OK) ? pick_u : saved_u;
    c->sweep_sorted = (rc == APCLOUD_OK) ? pick_s : saved_s;
    return rc;
}

}  // namespace apc

// ---------------------------------------------------------------- allocation-free solve
// apcloud_solve_system_noalloc: the GMRES solve of apcloud_solve_system with
// every piece of Krylov scratch (basis, work vectors, block partials, device
// state) carved from one file-scope device array instead of context buffers,
// so a call allocates no device or host memory.  Sized for at most
// NOALLOC_MAX_NODES nodes and restart <= NOALLOC_MAX_RESTART.
#include <mutex>

namespace apc {

constexpr size_t NOALLOC_BYTES = (size_t)20 << 20;   // 20 MiB on every device that loads the library
constexpr int NOALLOC_MAX_NODES = 65536;
constexpr int NOALLOC_MAX_RESTART = 30;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_base[NOALLOC_MAX_DEVICES] = {};

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of the scratch array on the context's device (the host-side
// name of the array is only a stand-in); resolved once per device.  The
// context's device must be current: cudaGetSymbolAddress answers for the
// current device, and the scratch must sit on the device of the context's
// matrices and stream.
apcloud_status noalloc_base(apcloud_ctx *c, unsigned char **out) {
    int dev = 0;
    APC_CUDA(c, cudaGetDevice(&dev));
    if (dev != c->device)
        return fail(c, APCLOUD_E_INVALID, "current device %d is not the context's device %d", dev, c->device);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(c, APCLOUD_E_INVALID, "device index %d too large", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_check(c, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                      "cudaGetSymbolAddress(scratch)");
        g_noalloc_base[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_base[dev];
    return APCLOUD_OK;
}
}  // namespace
}  // namespace apc

extern "C" apcloud_status apcloud_solve_system_noalloc(apcloud_ctx *c, int which, const double *b, double *x,
                                                       double rtol, int max_iter, apcloud_solve_info *info) {
    using namespace apc;
    if (!c || !b || !x || (which != 0 && which != 1)) return APCLOUD_E_INVALID;
    if (c->stage < 2) return fail(c, APCLOUD_E_STATE, "matrices are available after apcloud_stencils");
    if (!(rtol > 0) || max_iter < 0) return fail(c, APCLOUD_E_INVALID, "rtol must be > 0 and max_iter >= 0");
    const int n = c->n_tot;
    const int m = c->P.restart;
    if (n > NOALLOC_MAX_NODES)
        return fail(c, APCLOUD_E_INVALID, "%d nodes exceed the %d-node limit of the allocation-free solve", n,
                    NOALLOC_MAX_NODES);
    if (m > NOALLOC_MAX_RESTART)
        return fail(c, APCLOUD_E_INVALID, "restart %d exceeds the limit %d of the allocation-free solve", m,
                    NOALLOC_MAX_RESTART);
    // it runs one algorithm only: FP64 GMRES with Jacobi on one Krylov space
    // and one global stopping test; other forms would silently change results
    if (c->P.precision != 0 || c->P.poly_degree > 1 || c->nbeams > 1)
        return fail(c, APCLOUD_E_INVALID,
                    "the allocation-free solve runs FP64 Jacobi GMRES on a single-beam context only "
                    "(precision %d, poly_degree %d, beams %d)", c->P.precision, c->P.poly_degree, c->nbeams);
    unsigned char *base = nullptr;
    APC_TRY(noalloc_base(c, &base));
    // carve: state | basis | w | wraw | u | partials
    const int64_t ldv = ((int64_t)n + 31) / 32 * 32;
    const int nblk = reduction_blocks(c, n);
    size_t off = 0;
    GmresState *st = reinterpret_cast<GmresState *>(base + off);
    off = align256(off + sizeof(GmresState));
    double *V = reinterpret_cast<double *>(base + off);
    off = align256(off + sizeof(double) * (size_t)(m + 1) * ldv);
    double *w = reinterpret_cast<double *>(base + off);
    off = align256(off + sizeof(double) * (size_t)ldv);
    double *wraw = reinterpret_cast<double *>(base + off);
    off = align256(off + sizeof(double) * (size_t)ldv);
    double *u = reinterpret_cast<double *>(base + off);
    off = align256(off + sizeof(double) * (size_t)ldv);
    double *partial = reinterpret_cast<double *>(base + off);
    off = align256(off + sizeof(double) * (size_t)(div_up(n, RT) + 2 * nblk) * 64);
    if (off > NOALLOC_BYTES) return fail(c, APCLOUD_E_INVALID, "allocation-free scratch too small");

    const unsigned saved_mask = c->timer.mask;   // event timers may allocate: off for this call
    c->timer.mask = 0;
    const double *val = ptr<double>(which ? c->ell_A : c->ell_B);
    const double *d = ptr<double>(which ? c->dA : c->dB);
    apcloud_status status = APCLOUD_W_NOT_CONVERGED;
    int iters = 0, cycles = 0;
    double relres = 0.0;
    do {
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_mul, u, (const double *)x, d, n);
        Krylov<double> K{V, ldv, w, wraw, st, partial, nblk};
        K.graphs = false;   // instantiating a graph allocates
        // gmres_core clears the device state itself (the array keeps the previous call's contents)
        status = gmres_core<double>(c, val, b, u, rtol, max_iter, K, &iters, &cycles, &relres);
        if (status < 0) break;
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_div, x, (const double *)u, d, n);
        apcloud_status r = cuda_check(c, cudaStreamSynchronize(c->s), "solve_system_noalloc");
        if (r < 0) status = r;
    } while (0);
    c->timer.mask = saved_mask;
    if (info && status >= 0) {
        info->iters = iters;
        info->restarts = cycles;
        info->relres = relres;
    }
    return status;
}

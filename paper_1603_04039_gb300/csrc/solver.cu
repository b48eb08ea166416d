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
#include <cmath>

#include "internal.cuh"

namespace apc {

namespace {

constexpr int RT = 256;  // threads of the reduction kernels

// Block reduction of NJ per-thread values into sums held by threads 0..nj-1
// of the block (returned in `out`, valid for threadIdx.x < nj).
template <int NJ>
__device__ __forceinline__ void block_reduce_many(const double (&acc)[NJ], int nj, double *sm, double *out) {
    // sm: RT * NJ doubles laid out [k][t]
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < NJ; ++k)
        if (k < nj) sm[k * RT + t] = acc[k];
    __syncthreads();
    // nj * 8 threads each sum a segment of 32
    const int seg = RT / 32;
    for (int q = t; q < nj * seg; q += RT) {
        int k = q / seg, s = q % seg;
        const double *p = sm + k * RT + s * 32;
        double v = 0.0;
#pragma unroll 8
        for (int i = 0; i < 32; ++i) v += p[i];
        sm[NJ * RT + q] = v;
    }
    __syncthreads();
    if (t < nj) {
        double v = 0.0;
#pragma unroll
        for (int s = 0; s < seg; ++s) v += sm[NJ * RT + t * seg + s];
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
// nk == 1 uses every thread on one value; otherwise thread t takes value
// t % 64 and every fourth block starting at t / 64.  Result in out[k] (shared).
__device__ void final_sums(const double *partial, int nblk, int nk, double *sm, double *out) {
    const int t = threadIdx.x;
    if (nk == 1) {
        double v = 0.0;
        for (int b = t; b < nblk; b += RT) v += __ldcg(&partial[(int64_t)b * 64]);
        double a[1] = {v};
        double tot = 0.0;
        block_reduce_many<1>(a, 1, sm, &tot);
        if (t == 0) out[0] = tot;
    } else {
        const int k = t & 63, part = t >> 6;
        double v = 0.0;
        if (k < nk)
            for (int b = part; b < nblk; b += RT / 64) v += __ldcg(&partial[(int64_t)b * 64 + k]);
        sm[t] = v;
        __syncthreads();
        if (t < nk) out[t] = (sm[t] + sm[t + 64]) + (sm[t + 128] + sm[t + 192]);
    }
    __syncthreads();
}

// ---------------------------------------------------------------- deposit
// Cell-indicator charge assignment (Section 5): Q_j = sum of the charges of
// the particles in leaf j, rho_M = Q_j / h_j^3; boundary rows copy the owner.
__global__ void k_deposit(const double *__restrict__ q, double qu, const uint32_t *__restrict__ perm,
                          const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                          const int4 *__restrict__ ic, int n_int, double ext, double *__restrict__ rho_m) {
    int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (j >= n_int) return;
    int f = first[j], c = count[j];
    double Q;
    if (q) {
        double s = 0.0;
        for (int i = f + lane; i < f + c; i += 32) s += q[perm[i]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        Q = s;
    } else {
        Q = (double)c * qu;
    }
    if (lane == 0) {
        double h = ldexp(ext, -ic[j].w);
        rho_m[j] = Q / (h * h * h);
    }
}

__global__ void k_bcopy(const int32_t *__restrict__ owner, int n_int, int n_bnd, double *__restrict__ v) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n_bnd) v[n_int + b] = v[owner[b]];
}

// ---------------------------------------------------------------- SpMV
// mode 0: y = Ahat x
// mode 1: y = Ahat x * s, vout[r] = x[r] * s, s = *sptr (Arnoldi step)
// mode 2: y = b - Ahat x, ||y||^2 reduced into st (cycle start)
template <int MODE>
__global__ void __launch_bounds__(RT) k_spmv(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                                             const int32_t *__restrict__ col, const double *__restrict__ val,
                                             int n, const double *__restrict__ x, double *__restrict__ y,
                                             double *__restrict__ vout, const double *__restrict__ b,
                                             GmresState *st, double *__restrict__ partial) {
    __shared__ double sm[RT + RT / 32 + 8];
    if (MODE == 1 && st->done) return;
    const int r = blockIdx.x * RT + threadIdx.x;
    double s = 1.0;
    if (MODE == 1) s = st->inv_norm;
    double acc = 0.0, yv = 0.0;
    if (r < n) {
        const int sl = r >> 5, lane = r & 31;
        const int w = (int)sw[sl];
        const int64_t base = (int64_t)soff[sl] * 32 + lane;
        for (int k = 0; k < w; ++k) {
            const int64_t e = base + (int64_t)k * 32;
            acc = fma(val[e], x[col[e]], acc);
        }
        if (MODE == 0) { yv = acc; y[r] = yv; }
        if (MODE == 1) { y[r] = acc * s; vout[r] = x[r] * s; }
        if (MODE == 2) { yv = b[r] - acc; y[r] = yv; }
    }
    if (MODE == 2) {
        double a[1] = {yv * yv};
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

// ---------------------------------------------------------------- Gram-Schmidt passes
// GB300 executes FP64 at 1/58 of its FP32 rate and charges a warp-wide FP64
// instruction in full even when lanes are predicated off, so every FP64
// instruction here does useful work on 32 lanes:
//   * dot products V_k^T w: one warp per basis vector over a tile of w staged
//     in shared memory (lanes over rows, coalesced, no padding terms);
//   * updates w -= V h: one thread per row with a runtime loop over k (four
//     rows per thread for independent FMA chains).
constexpr int GT = 256;                    // threads per block (8 warps)
constexpr int GW = GT / 32;
constexpr int TILE = 512;                  // rows staged per tile
constexpr int KPW = MAX_RESTART / GW;      // basis vectors per warp (<= 8)

__device__ __forceinline__ void tile_dots(const double *__restrict__ V, int64_t ldv, int base, int lim, int j1,
                                          const double *ws, double (&acc)[KPW]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int kk = 0; kk < KPW; ++kk) {
        const int k = wid + GW * kk;
        if (k < j1) {   // uniform across the warp
            const double *vk = V + (int64_t)k * ldv + base;
            double a = acc[kk];
#pragma unroll 4
            for (int i = lane; i < lim; i += 32) a = fma(vk[i], ws[i], a);
            acc[kk] = a;
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// PASS 0: h1 = V^T w.   PASS 1: w -= V h1, then h2 = V^T w.
template <int PASS>
__global__ void __launch_bounds__(GT) k_gs_dots(const double *__restrict__ V, int64_t ldv, int n, int j,
                                                double *__restrict__ w, GmresState *st, double *__restrict__ partial) {
    __shared__ double ws[TILE];
    __shared__ double hs[MAX_RESTART];
    __shared__ double red[MAX_RESTART];
    __shared__ double sm[RT + RT / 32 + 8];
    __shared__ double fs[64];
    if (st->done) return;
    const int j1 = j + 1, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (PASS == 1 && tid < j1) hs[tid] = st->h1[tid];
    __syncthreads();
    double acc[KPW];
#pragma unroll
    for (int kk = 0; kk < KPW; ++kk) acc[kk] = 0.0;
    for (int64_t base = (int64_t)blockIdx.x * TILE; base < n; base += (int64_t)gridDim.x * TILE) {
        const int lim = (int)((n - base) < TILE ? (n - base) : TILE);
        if (PASS == 0) {
            for (int t = tid; t < TILE; t += GT) ws[t] = (t < lim) ? w[base + t] : 0.0;
        } else {
            double wi[TILE / GT];
#pragma unroll
            for (int r = 0; r < TILE / GT; ++r) {
                int t = tid + GT * r;
                wi[r] = (t < lim) ? w[base + t] : 0.0;
            }
            for (int k = 0; k < j1; ++k) {
                const double hk = hs[k];
                const double *vk = V + (int64_t)k * ldv + base;
#pragma unroll
                for (int r = 0; r < TILE / GT; ++r) {
                    int t = tid + GT * r;
                    if (t < lim) wi[r] = fma(-vk[t], hk, wi[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < TILE / GT; ++r) {
                int t = tid + GT * r;
                if (t < lim) w[base + t] = wi[r];
                ws[t] = (t < lim) ? wi[r] : 0.0;
            }
        }
        __syncthreads();
        tile_dots(V, ldv, (int)base, lim, j1, ws, acc);
        __syncthreads();
    }
#pragma unroll
    for (int kk = 0; kk < KPW; ++kk) {
        const int k = wid + GW * kk;
        if (k < j1) {
            double v = warp_sum(acc[kk]);
            if (lane == 0) red[k] = v;
        }
    }
    __syncthreads();
    if (tid < j1) partial[(int64_t)blockIdx.x * 64 + tid] = red[tid];
    if (!last_block(&st->ticket)) return;
    final_sums(partial, gridDim.x, j1, sm, fs);
    if (tid < j1) {
        if (PASS == 0) st->h1[tid] = fs[tid];
        else st->h2[tid] = fs[tid];
    }
    if (tid == 0) st->ticket = 0;
}

// wraw = w - V h2 ; ||wraw||^2 ; Hessenberg column, Givens rotation and
// convergence test in the last block (Saad, Algorithms 6.9 / 6.10)
__global__ void __launch_bounds__(GT) k_gs_norm(const double *__restrict__ V, int64_t ldv, int n, int j,
                                                const double *__restrict__ w, double *__restrict__ wraw,
                                                GmresState *st, double *__restrict__ partial) {
    __shared__ double hs[MAX_RESTART];
    __shared__ double sm[RT + RT / 32 + 8];
    __shared__ double fs[1];
    if (st->done) return;
    const int j1 = j + 1, tid = threadIdx.x;
    if (tid < j1) hs[tid] = st->h2[tid];
    __syncthreads();
    double sq = 0.0;
    constexpr int R = 4;
    for (int64_t base = (int64_t)blockIdx.x * GT * R; base < n; base += (int64_t)gridDim.x * GT * R) {
        double wi[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t i = base + tid + GT * r;
            wi[r] = (i < n) ? w[i] : 0.0;
        }
        for (int k = 0; k < j1; ++k) {
            const double hk = hs[k];
            const double *vk = V + (int64_t)k * ldv + base + tid;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (base + tid + GT * r < n) wi[r] = fma(-vk[GT * r], hk, wi[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t i = base + tid + GT * r;
            if (i < n) {
                wraw[i] = wi[r];
                sq = fma(wi[r], wi[r], sq);
            }
        }
    }
    double a1[1] = {sq};
    double tot = 0.0;
    block_reduce_many<1>(a1, 1, sm, &tot);
    if (tid == 0) partial[(int64_t)blockIdx.x * 64] = tot;
    if (!last_block(&st->ticket)) return;
    final_sums(partial, gridDim.x, 1, sm, fs);
    if (tid == 0) {
        const int M = MAX_RESTART;
        double hn = sqrt(fs[0]);
        for (int i = 0; i <= j; ++i) st->H[i * M + j] = st->h1[i] + st->h2[i];
        st->H[(j + 1) * M + j] = hn;
        for (int i = 0; i < j; ++i) {
            double a = st->H[i * M + j], bb = st->H[(i + 1) * M + j];
            st->H[i * M + j] = st->cs[i] * a + st->sn[i] * bb;
            st->H[(i + 1) * M + j] = -st->sn[i] * a + st->cs[i] * bb;
        }
        double a = st->H[j * M + j], bb = st->H[(j + 1) * M + j];
        double den = sqrt(a * a + bb * bb);
        st->cs[j] = den != 0.0 ? a / den : 1.0;
        st->sn[j] = den != 0.0 ? bb / den : 0.0;
        st->H[j * M + j] = den;
        st->H[(j + 1) * M + j] = 0.0;
        st->g[j + 1] = -st->sn[j] * st->g[j];
        st->g[j] = st->cs[j] * st->g[j];
        st->jend = j + 1;
        if (fabs(st->g[j + 1]) <= st->rtol * st->bnorm || hn == 0.0) st->done = 1;
        st->inv_norm = hn > 0.0 ? 1.0 / hn : 0.0;
        st->ticket = 0;
    }
}

// u += V y with H y = g solved (upper triangular, jend x jend) in every block
__global__ void __launch_bounds__(GT) k_cycle_end(const double *__restrict__ V, int64_t ldv, int n,
                                                  double *__restrict__ u, const GmresState *__restrict__ st) {
    __shared__ double ys[MAX_RESTART];
    const int je = st->jend;
    if (threadIdx.x == 0) {
        const int M = MAX_RESTART;
        for (int k = je - 1; k >= 0; --k) {
            double s = st->g[k];
            for (int l = k + 1; l < je; ++l) s -= st->H[k * M + l] * ys[l];
            ys[k] = s / st->H[k * M + k];
        }
    }
    __syncthreads();
    if (je == 0) return;
    for (int64_t i = (int64_t)blockIdx.x * GT + threadIdx.x; i < n; i += (int64_t)gridDim.x * GT) {
        double s = 0.0;
        for (int k = 0; k < je; ++k) s = fma(V[(int64_t)k * ldv + i], ys[k], s);
        u[i] += s;
    }
}

__global__ void __launch_bounds__(RT) k_norm2(const double *__restrict__ x, int n, GmresState *st,
                                              double *__restrict__ partial) {
    __shared__ double sm[RT + RT / 32 + 8];
    double s = 0.0;
    for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) s = fma(x[i], x[i], s);
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

void gs_dispatch(apcloud_ctx *c, int pass, int nblk, const double *V, int64_t ldv, int n, int j, double *w,
                 double *wraw, GmresState *st, double *partial) {
    if (pass == 0) APC_LAUNCH(c, K_DOT, nblk, GT, 0, k_gs_dots<0>, V, ldv, n, j, w, st, partial);
    else if (pass == 1) APC_LAUNCH(c, K_UPDDOT, nblk, GT, 0, k_gs_dots<1>, V, ldv, n, j, w, st, partial);
    else APC_LAUNCH(c, K_UPDNORM, nblk, GT, 0, k_gs_norm, V, ldv, n, j, (const double *)w, wraw, st, partial);
}

void cycle_end_dispatch(apcloud_ctx *c, int nblk, int jmax, const double *V, int64_t ldv, int n, double *u,
                        GmresState *st) {
    (void)jmax;
    APC_LAUNCH(c, K_CYCLE, nblk, GT, 0, k_cycle_end, V, ldv, n, u, st);
}

int reduction_blocks(apcloud_ctx *c, int n) {
    (void)c;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    int nb = div_up(n, TILE);
    int cap = 2 * sms;
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    return nb;
}

}  // namespace

apcloud_status deposit(apcloud_ctx *c, const double *q, double q_uniform) {
    const int n = c->n_int, nt = c->n_tot;
    double *rm = ensure<double>(c, c->rho_m, nt + 1);
    if (!rm) return APCLOUD_E_NOMEM;
    const uint32_t *perm = ptr<uint32_t>(c->val[c->kbuf]);
    const double ext = c->P.hi[0] - c->P.lo[0];
    APC_LAUNCH(c, K_DEPOSIT, div_up(n, 8), 256, 0, k_deposit, q, q_uniform, perm, ptr<int32_t>(c->leaf_first),
               ptr<int32_t>(c->leaf_count), ptr<int4>(c->node_ic), n, ext, rm);
    APC_LAUNCH(c, K_DEPOSIT, div_up(c->n_bnd, 256), 256, 0, k_bcopy, ptr<int32_t>(c->bowner), n, c->n_bnd, rm);
    // permutation and charge per particle, rho_M per node
    account(c, K_DEPOSIT, (q ? 12.0 * c->N : 0.0) + 8.0 * nt, q ? (double)c->N : (double)n);
    return cuda_check(c, cudaGetLastError(), "deposit");
}

apcloud_status spmv(apcloud_ctx *c, int which, const double *x, double *y, double scale, double *copy_out) {
    (void)scale; (void)copy_out;
    const double *val = ptr<double>(which ? c->ell_A : c->ell_B);
    const int n = c->n_tot;
    APC_LAUNCH(c, K_SPMV, div_up(n, RT), RT, 0, k_spmv<0>, ptr<uint32_t>(c->slice_w), ptr<uint32_t>(c->slice_off),
               ptr<int32_t>(c->ell_col), val, n, x, y, (double *)nullptr, (const double *)nullptr,
               (GmresState *)nullptr, (double *)nullptr);
    return cuda_check(c, cudaGetLastError(), "spmv");
}

// Solve (B or A) x = b.  On entry x holds the initial guess (unscaled); on
// exit the solution.
apcloud_status gmres_solve(apcloud_ctx *c, int which, const double *b, double *x, double rtol, int max_iter,
                           apcloud_solve_info *info) {
    const int n = c->n_tot;
    const int m = c->P.restart;
    const int64_t ldv = ((int64_t)n + 31) / 32 * 32;
    double *V = ensure<double>(c, c->V, (int64_t)(m + 1) * ldv);
    double *w = ensure<double>(c, c->w0, n + 1);
    double *wraw = ensure<double>(c, c->w1, n + 1);
    double *u = ensure<double>(c, c->u, n + 1);
    const int nblk = reduction_blocks(c, n);
    double *partial = ensure<double>(c, c->partial, (int64_t)(div_up(n, RT) + 2 * nblk) * 64);
    GmresState *st = ptr<GmresState>(c->gstate);
    if (!V || !w || !wraw || !u || !partial) return APCLOUD_E_NOMEM;
    const double *val = ptr<double>(which ? c->ell_A : c->ell_B);
    const double *d = ptr<double>(which ? c->dA : c->dB);
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);

    APC_CUDA(c, cudaMemsetAsync(st, 0, sizeof(GmresState), c->s));
    APC_CUDA(c, cudaMemcpyAsync(&st->rtol, &rtol, sizeof(double), cudaMemcpyHostToDevice, c->s));
    APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_mul, u, (const double *)x, d, n);
    APC_LAUNCH(c, K_VEC, nblk, RT, 0, k_norm2, b, n, st, partial);

    struct { double beta, bnorm; int jend, done; } hs;
    int iters = 0, cycles = 0;
    double relres = 0.0;
    apcloud_status status = APCLOUD_W_NOT_CONVERGED;
    for (;;) {
        // r = b - Ahat u, into wraw; beta = ||r||
        APC_LAUNCH(c, K_SPMV, div_up(n, RT), RT, 0, k_spmv<2>, sw, so, col, val, n, (const double *)u, wraw,
                   (double *)nullptr, b, st, partial);
        double tmp[2];  // bnorm and beta are adjacent in GmresState
        APC_TRY(read_back(c, tmp, &st->bnorm, 2 * sizeof(double)));
        hs.bnorm = tmp[0];
        hs.beta = tmp[1];
        relres = hs.bnorm > 0.0 ? hs.beta / hs.bnorm : 0.0;
        if (hs.bnorm == 0.0 || hs.beta <= rtol * hs.bnorm) { status = APCLOUD_OK; break; }
        if (iters >= max_iter) break;
        const int jmax = (m < max_iter - iters) ? m : (max_iter - iters);
        for (int j = 0; j < jmax; ++j) {
            APC_LAUNCH(c, K_SPMV, div_up(n, RT), RT, 0, k_spmv<1>, sw, so, col, val, n, (const double *)wraw, w,
                       V + (int64_t)j * ldv, (const double *)nullptr, st, (double *)nullptr);
            gs_dispatch(c, 0, nblk, V, ldv, n, j, w, wraw, st, partial);
            gs_dispatch(c, 1, nblk, V, ldv, n, j, w, wraw, st, partial);
            gs_dispatch(c, 2, nblk, V, ldv, n, j, w, wraw, st, partial);
        }
        cycle_end_dispatch(c, nblk, jmax, V, ldv, n, u, st);
        APC_CUDA(c, cudaGetLastError());
        int je;
        APC_TRY(read_back(c, &je, &st->jend, sizeof(int)));
        {   // algorithmic traffic of the launches that did work
            const double nnz = (double)c->sum_m + (double)c->n_int + (double)c->n_bnd, dn = n;
            account(c, K_SPMV, (12.0 * nnz + 16.0 * dn) * (je + 1), 2.0 * nnz * (je + 1));
            for (int j = 0; j < je; ++j) {
                account(c, K_DOT, 8.0 * dn * (j + 2), 2.0 * dn * (j + 1));
                account(c, K_UPDDOT, 8.0 * dn * (j + 3), 4.0 * dn * (j + 1));
                account(c, K_UPDNORM, 8.0 * dn * (j + 3), 2.0 * dn * (j + 2));
            }
            account(c, K_CYCLE, 8.0 * dn * (je + 2), 2.0 * dn * je);
        }
        iters += je;
        ++cycles;
        if (je == 0) break;  // breakdown at the first column: nothing more to gain
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

// Device address of the scratch array for the current device (the host-side
// name of the array is only a stand-in); resolved once per device.
apcloud_status noalloc_base(apcloud_ctx *c, unsigned char **out) {
    int dev = 0;
    APC_CUDA(c, cudaGetDevice(&dev));
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
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    apcloud_status status = APCLOUD_W_NOT_CONVERGED;
    int iters = 0, cycles = 0;
    double relres = 0.0;
    do {
        // the array keeps the previous call's contents: the state must start from zero
        if (cuda_check(c, cudaMemsetAsync(st, 0, sizeof(GmresState), c->s), "memset") < 0) { status = APCLOUD_E_CUDA; break; }
        if (cuda_check(c, cudaMemcpyAsync(&st->rtol, &rtol, sizeof(double), cudaMemcpyHostToDevice, c->s), "rtol") < 0) {
            status = APCLOUD_E_CUDA;
            break;
        }
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_mul, u, (const double *)x, d, n);
        APC_LAUNCH(c, K_VEC, nblk, RT, 0, k_norm2, b, n, st, partial);
        for (;;) {
            APC_LAUNCH(c, K_SPMV, div_up(n, RT), RT, 0, k_spmv<2>, sw, so, col, val, n, (const double *)u, wraw,
                       (double *)nullptr, b, st, partial);
            double tmp[2];
            apcloud_status r = read_back(c, tmp, &st->bnorm, 2 * sizeof(double));
            if (r < 0) { status = r; break; }
            relres = tmp[0] > 0.0 ? tmp[1] / tmp[0] : 0.0;
            if (tmp[0] == 0.0 || tmp[1] <= rtol * tmp[0]) { status = APCLOUD_OK; break; }
            if (iters >= max_iter) break;
            const int jmax = (m < max_iter - iters) ? m : (max_iter - iters);
            for (int j = 0; j < jmax; ++j) {
                APC_LAUNCH(c, K_SPMV, div_up(n, RT), RT, 0, k_spmv<1>, sw, so, col, val, n, (const double *)wraw, w,
                           V + (int64_t)j * ldv, (const double *)nullptr, st, (double *)nullptr);
                gs_dispatch(c, 0, nblk, V, ldv, n, j, w, wraw, st, partial);
                gs_dispatch(c, 1, nblk, V, ldv, n, j, w, wraw, st, partial);
                gs_dispatch(c, 2, nblk, V, ldv, n, j, w, wraw, st, partial);
            }
            cycle_end_dispatch(c, nblk, jmax, V, ldv, n, u, st);
            int je = 0;
            r = read_back(c, &je, &st->jend, sizeof(int));
            if (r < 0) { status = r; break; }
            iters += je;
            ++cycles;
            if (je == 0) break;
        }
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

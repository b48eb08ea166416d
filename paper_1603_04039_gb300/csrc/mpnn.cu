// mpnn.cu -- the learned part of the solver: a message-passing network over
// the GFD stencil graph that proposes a diagonal right preconditioner (an
// approximate-inverse column scaling of Ahat = A D^-1) and an initial guess
// for the Poisson solve (Section 3.2 step 2 is the system it serves; the paper
// itself has no learned component).
//
// Network (width 64, 3 layers, BF16 weights and activations, FP32
// accumulation):
//   W = |Ahat_off| + |Ahat_off|^T (symmetric stencil graph), P = W / rowsum
//   H_0 = F (16 node features), H_{l+1} = relu([H_l | P H_l] W_l + b_l)
//   t = H_3 W_o + b_o;  s = exp(ln8 tanh t_0) (1 on boundary nodes);  gamma = exp(tanh t_1)
//   Lp = (1/n_int) sum over interior columns j of (1 - 2 s_j + s_j^2 c_j)
//   Lg = ||b - Ahat (gamma * b)||^2 / ||b||^2
// The dense layers, their data gradients and their weight gradients run on
// the 5th-generation tensor cores: tcgen05.mma (kind::f16, BF16 inputs, FP32
// accumulator in tensor memory) issued by one thread, operands staged in
// shared memory in the canonical no-swizzle K-major layout, completion
// signalled through an mbarrier, results read back with tcgen05.ld.  The
// graph products (P H, P^T G), features, head, loss and Adam run on the CUDA
// cores.  Every reduction has a fixed order, so a training run is repeatable.
#include <atomic>
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "internal.cuh"

struct apcloud_mpnn {
    // flat FP32 parameters, gradients and Adam moments (layout in apcloud.h)
    float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    // BF16 copies of W_l: row-major (K_l x 64) and transposed (64 x K_l)
    __nv_bfloat16 *w[3] = {nullptr, nullptr, nullptr}, *wt[3] = {nullptr, nullptr, nullptr};
    int64_t adam_steps = 0;
    unsigned *err = nullptr;   // device error word of the tensor-core kernels
};

namespace apc {

namespace {

constexpr int NF = 16, WD = 64;
constexpr float ALPHA = 2.0794415416798357f;   // ln 8: s in [1/8, 8]
constexpr int K_L[3] = {2 * NF, 2 * WD, 2 * WD};
// offsets into the flat parameter vector
constexpr int OFF_W0 = 0, OFF_B0 = OFF_W0 + 2 * NF * WD, OFF_W1 = OFF_B0 + WD, OFF_B1 = OFF_W1 + 2 * WD * WD,
              OFF_W2 = OFF_B1 + WD, OFF_B2 = OFF_W2 + 2 * WD * WD, OFF_WO = OFF_B2 + WD, OFF_BO = OFF_WO + 2 * WD,
              N_PARAMS = OFF_BO + 2;
constexpr int OFF_W[3] = {OFF_W0, OFF_W1, OFF_W2}, OFF_B[3] = {OFF_B0, OFF_B1, OFF_B2};
constexpr unsigned ERR_TC_TIMEOUT = 1u;
constexpr int LEARNED_STEPS = 1000;   // Arnoldi steps the scaled solve gets before the Jacobi fallback

// ---------------------------------------------------------------- tcgen05 helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major core matrices of
// 8 rows x 16 bytes; lbo = byte step between the two core matrices of a
// 16-element K block, sbo = byte step between 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor cores
    return d;                 // base offset 0, relative LBO, no swizzle
}

// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait on an mbarrier phase; false if it did not complete in time
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row, k) of an operand tile with `rows` rows inside
// its 16-wide K block kb (core matrices 8 x 8, two per K block)
__device__ __forceinline__ uint32_t tile_off(int row, int k, int rows) {
    return (uint32_t)((k >> 4) * rows * 32 + (row >> 3) * 256 + ((k >> 3) & 1) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// the 8 elements of v (row chunk cc of sample k) into column k of a K-major
// tile with `rows` rows, element i to row 8 cc + ((i + 2 q) & 7)
__device__ __forceinline__ void scatter_col(unsigned char *tile, uint4 v, int cc, int k, int rows, int q) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t rw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t a0 = w[j], a1 = w[(j + 1) & 3], a2 = w[(j + 2) & 3], a3 = w[(j + 3) & 3];
        rw[j] = q == 0 ? a0 : q == 1 ? a1 : q == 2 ? a2 : a3;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int e = (i + 2 * q) & 7;   // element index; rw[i >> 1] holds elements 2((i>>1)+q), +1
        const uint16_t h = (uint16_t)((i & 1) ? (rw[i >> 1] >> 16) : (rw[i >> 1] & 0xFFFFu));
        *reinterpret_cast<uint16_t *>(tile + tile_off(cc * 8 + e, k, rows)) = h;
    }
}

constexpr int TC_THREADS = 128;
constexpr int TC_COLS = 128;        // TMEM columns allocated (N <= 128)
constexpr int TC_SMEM = 64 * 1024;  // A (<= 32 KB) + B (<= 32 KB)

struct TcArgs {
    const __nv_bfloat16 *x0, *x1;   // A rows: [x0 | x1], each n x c (x1 null: x0 only, c = K)
    int c;
    const __nv_bfloat16 *bmat;      // B operand rows, N x K row-major (forward Wt, data-gradient W)
    const __nv_bfloat16 *g;         // weight gradient: dZ (n x 64)
    const float *bias;
    __nv_bfloat16 *out_bf;          // forward: relu(acc + bias) (n x 64)
    float *out_f;                   // data gradient: acc (n x N); weight gradient: partials
    int n, K, N, Kl;
    unsigned *err;
};

// MODE 0: forward layer, out_bf = relu([x0|x1] Wt^T + bias), N = 64
// MODE 1: data gradient, out_f = dZ W^T (A = x0 = dZ, K = 64, N = K_l)
// MODE 2: weight gradient, partial[cta] = X^T dZ over the CTA's row chunks
//         (M = K_l rows of X^T padded to 128, N = 64, K = rows)
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_dense_tc(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *sA = smem;
    unsigned char *sB = smem + 32 * 1024;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) { bar_init(&bar); failed = 0; }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int N = a.N;
    uint32_t phase = 0;

    if (MODE == 0 || MODE == 1) {
        const int K = a.K;
        const int row0 = blockIdx.x * 128;
        const int cpr = K / 8;   // 16-byte chunks per row (4, 8 or 16)
        const int cq = cpr >> 2;
        // each warp store covers 8 rows x 4 chunks: four whole core matrices,
        // one 128-byte wavefront each, and 64 contiguous bytes of every row
        // read; four chunks per thread are loaded before any is stored
        constexpr int NB = 4;
        for (int base = tid; base < 128 * cpr; base += NB * TC_THREADS) {
            uint4 v[NB];
            uint32_t off[NB];
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                const int idx = base + u * TC_THREADS;
                const int g = idx >> 5, l = idx & 31;
                const int r = (g / cq) * 8 + (l & 7), cc = (g % cq) * 4 + (l >> 3), row = row0 + r;
                v[u] = make_uint4(0u, 0u, 0u, 0u);
                off[u] = tile_off(r, cc * 8, 128);
                if (idx < 128 * cpr && row < a.n) {
                    const __nv_bfloat16 *src;
                    if (a.x1) {
                        const int ch = a.c / 8;
                        src = (cc < ch) ? a.x0 + (int64_t)row * a.c + cc * 8
                                        : a.x1 + (int64_t)row * a.c + (cc - ch) * 8;
                    } else {
                        src = a.x0 + (int64_t)row * K + cc * 8;
                    }
                    v[u] = *reinterpret_cast<const uint4 *>(src);
                }
            }
#pragma unroll
            for (int u = 0; u < NB; ++u)
                if (base + u * TC_THREADS < 128 * cpr) *reinterpret_cast<uint4 *>(sA + off[u]) = v[u];
        }
        for (int base = tid; base < N * cpr; base += NB * TC_THREADS) {
            uint4 v[NB];
            uint32_t off[NB];
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                const int idx = base + u * TC_THREADS;
                const int g = idx >> 5, l = idx & 31;
                const int r = (g / cq) * 8 + (l & 7), cc = (g % cq) * 4 + (l >> 3);
                off[u] = tile_off(r, cc * 8, N);
                v[u] = idx < N * cpr ? *reinterpret_cast<const uint4 *>(a.bmat + (int64_t)r * K + cc * 8)
                                     : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < NB; ++u)
                if (base + u * TC_THREADS < N * cpr) *reinterpret_cast<uint4 *>(sB + off[u]) = v[u];
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t idesc = idesc_bf16(128, N);
            for (int kb = 0; kb < K / 16; ++kb) {
                const uint64_t ad = smem_desc(smem_u32(sA) + kb * 128 * 32, 128, 256);
                const uint64_t bd = smem_desc(smem_u32(sB) + kb * N * 32, 128, 256);
                mma_bf16(tmem, ad, bd, idesc, kb > 0 ? 1u : 0u);
            }
            mma_commit(&bar);
        }
        if (!bar_wait(&bar, phase)) failed = 1;
        phase ^= 1u;
        __syncthreads();
        tc_fence_after();
        if (!failed) {
            const int row = row0 + warp * 32 + lane;
            const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tmem_ld16(tl + c0, v);
                if (row < a.n) {
                    if (MODE == 0) {
                        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) o[i] = __float2bfloat16_rn(fmaxf(v[i] + a.bias[c0 + i], 0.f));
                        uint4 *dst = reinterpret_cast<uint4 *>(a.out_bf + (int64_t)row * WD + c0);
                        dst[0] = reinterpret_cast<const uint4 *>(o)[0];
                        dst[1] = reinterpret_cast<const uint4 *>(o)[1];
                    } else {
                        float4 *dst = reinterpret_cast<float4 *>(a.out_f + (int64_t)row * N + c0);
#pragma unroll
                        for (int i = 0; i < 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    }
                }
            }
        }
    } else {
        // weight gradient: chunks of 128 rows (K) per MMA group
        const int nchunk = (a.n + 127) / 128;
        const int Kl = a.Kl, ch = a.c / 8;
        int first = 1;
        for (int chunk = blockIdx.x; chunk < nchunk && !failed; chunk += gridDim.x) {
            // zero both operand tiles (rows of X^T past K_l and rows past n stay zero)
            for (int idx = tid; idx < (32 * 1024 + 64 * 128 * 2) / 16; idx += TC_THREADS)
                reinterpret_cast<uint4 *>(smem)[idx] = make_uint4(0u, 0u, 0u, 0u);
            __syncthreads();
            const int k = tid, row = chunk * 128 + k;
            // thread k scatters its row into column k of the transposed tiles;
            // the four 8-lane groups of a warp start at rows 2q apart, so one
            // 2-byte store of the warp lands in 16 distinct banks
            const int q = (lane >> 3) & 3;
            if (row < a.n) {
                // Kl / 8 (4 or 16) chunks of X, 8 of dZ: loads of four chunks in flight
                for (int c0 = 0; c0 < Kl / 8; c0 += 4) {
                    uint4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int cc = c0 + u;
                        v[u] = *reinterpret_cast<const uint4 *>(
                            (cc < ch) ? a.x0 + (int64_t)row * a.c + cc * 8 : a.x1 + (int64_t)row * a.c + (cc - ch) * 8);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) scatter_col(sA, v[u], c0 + u, k, 128, q);
                }
                for (int c0 = 0; c0 < WD / 8; c0 += 4) {
                    uint4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v[u] = *reinterpret_cast<const uint4 *>(a.g + (int64_t)row * WD + (c0 + u) * 8);
#pragma unroll
                    for (int u = 0; u < 4; ++u) scatter_col(sB, v[u], c0 + u, k, WD, q);
                }
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t idesc = idesc_bf16(128, WD);
                for (int kb = 0; kb < 8; ++kb) {
                    const uint64_t ad = smem_desc(smem_u32(sA) + kb * 128 * 32, 128, 256);
                    const uint64_t bd = smem_desc(smem_u32(sB) + kb * WD * 32, 128, 256);
                    mma_bf16(tmem, ad, bd, idesc, (first && kb == 0) ? 0u : 1u);
                }
                mma_commit(&bar);
            }
            if (!bar_wait(&bar, phase)) failed = 1;
            phase ^= 1u;
            first = 0;
            __syncthreads();
        }
        tc_fence_after();
        if (!failed) {
            const int mm = warp * 32 + lane;
            const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
            float *dst = a.out_f + ((int64_t)blockIdx.x * 128 + mm) * WD;
            for (int c0 = 0; c0 < WD; c0 += 16) {
                float v[16];
                tmem_ld16(tl + c0, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) dst[c0 + i] = first ? 0.f : v[i];
            }
        }
    }
    if (failed && tid == 0) atomicOr(a.err, ERR_TC_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
    }
}

// dW (Kl x 64) = sum over CTAs of the partials, fixed order
__global__ void k_wgrad_reduce(const float *__restrict__ part, int nblk, int Kl, float *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Kl * WD) return;
    const int m = i / WD, c = i - m * WD;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[((int64_t)b * 128 + m) * WD + c];
    out[i] = s;
}

// ---------------------------------------------------------------- graph
// ELL entry e of row j with column i != j and a nonzero value: two records,
// (j, i) carrying Ahat_ji as the row's own entry and (i, j) carrying it as an
// entry of column i's transpose.  Record value: (ELL index << 1) | direction.
__global__ void k_edge_emit(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                            const int32_t *__restrict__ col, const double *__restrict__ val, int n,
                            const uint32_t *__restrict__ cnt_off, uint64_t *__restrict__ key,
                            uint32_t *__restrict__ rec) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int sl = r >> 5, lane = r & 31;
    const int w = (int)sw[sl];
    const int64_t base = (int64_t)soff[sl] * 32 + lane;
    uint32_t o = cnt_off[r];
    for (int k = 1; k < w; ++k) {
        const int64_t e = base + (int64_t)k * 32;
        const int i = col[e];
        if (i == r || val[e] == 0.0) continue;
        key[2 * o] = ((uint64_t)(uint32_t)r << 32) | (uint32_t)i;
        rec[2 * o] = (uint32_t)(e << 1);
        key[2 * o + 1] = ((uint64_t)(uint32_t)i << 32) | (uint32_t)r;
        rec[2 * o + 1] = (uint32_t)((e << 1) | 1);
        ++o;
    }
}

__global__ void k_edge_count(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                             const int32_t *__restrict__ col, const double *__restrict__ val, int n,
                             uint32_t *__restrict__ cnt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int sl = r >> 5, lane = r & 31;
    const int w = (int)sw[sl];
    const int64_t base = (int64_t)soff[sl] * 32 + lane;
    uint32_t c = 0;
    for (int k = 1; k < w; ++k) {
        const int64_t e = base + (int64_t)k * 32;
        if (col[e] != r && val[e] != 0.0) ++c;
    }
    cnt[r] = c;
}

__global__ void k_run_heads(const uint64_t *__restrict__ key, int64_t m, uint32_t *__restrict__ f) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) f[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

// unique (row, col) pairs: column, signed out value Ahat_row,col and in value Ahat_col,row
__global__ void k_edge_merge(const uint64_t *__restrict__ key, const uint32_t *__restrict__ rec, int64_t m,
                             const uint32_t *__restrict__ f, const uint32_t *__restrict__ pos,
                             const double *__restrict__ val, int32_t *__restrict__ ecol, float *__restrict__ aout,
                             float *__restrict__ ain, uint64_t *__restrict__ ukey) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || !f[i]) return;
    float o = 0.f, in = 0.f;
    for (int64_t t = i; t < m && t < i + 2 && key[t] == key[i]; ++t) {
        const uint32_t r = rec[t];
        const float v = (float)val[r >> 1];
        if (r & 1u) in = v; else o = v;
    }
    const uint32_t p = pos[i];
    ecol[p] = (int32_t)(uint32_t)(key[i] & 0xFFFFFFFFull);
    aout[p] = o;
    ain[p] = in;
    ukey[p] = key[i];
}

__global__ void k_rowptr(const uint64_t *__restrict__ ukey, int64_t m, int n, int32_t *__restrict__ rp) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n) return;
    const uint64_t v = (uint64_t)(uint32_t)j << 32;
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ukey[mid] < v) lo = mid + 1; else hi = mid;
    }
    rp[j] = (int32_t)lo;
}

// row sums of W = |a_out| + |a_in| and the two aggregation weights per edge:
// pf = W_ji / S_j (P), pb = W_ji / S_i (P^T applied by gathering over row j)
__global__ void k_row_sums(const int32_t *__restrict__ rp, const float *__restrict__ aout,
                           const float *__restrict__ ain, int n, float *__restrict__ S) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float s = 0.f;
    for (int e = rp[j]; e < rp[j + 1]; ++e) s += fabsf(aout[e]) + fabsf(ain[e]);
    S[j] = s;
}

__global__ void k_agg_weights(const int32_t *__restrict__ rp, const int32_t *__restrict__ ecol,
                              const float *__restrict__ aout, const float *__restrict__ ain,
                              const float *__restrict__ S, int n, float *__restrict__ pf, float *__restrict__ pb) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float sj = S[j];
    for (int e = rp[j]; e < rp[j + 1]; ++e) {
        const float w = fabsf(aout[e]) + fabsf(ain[e]);
        const float si = S[ecol[e]];
        pf[e] = sj > 0.f ? w / sj : 0.f;
        pb[e] = si > 0.f ? w / si : 0.f;
    }
}

// ---------------------------------------------------------------- features
__global__ void k_absmax(const double *__restrict__ b, int n, double *__restrict__ out, unsigned *ticket,
                         double *__restrict__ part) {
    __shared__ double sh[256];
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmax(m, fabs(b[i]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
    __threadfence();
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        double mm = 0.0;
        for (unsigned k = 0; k < gridDim.x; ++k) mm = fmax(mm, part[k]);
        *out = mm;
        *ticket = 0u;
    }
}

__global__ void k_features(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                           const int32_t *__restrict__ col, const double *__restrict__ val,
                           const int32_t *__restrict__ rp, const int32_t *__restrict__ ecol,
                           const float *__restrict__ aout, const float *__restrict__ ain,
                           const float *__restrict__ pf, const int4 *__restrict__ ic, int n, int n_int,
                           const double *__restrict__ b, const double *__restrict__ bmax, float *__restrict__ F,
                           __nv_bfloat16 *__restrict__ H0, float *__restrict__ c_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float f[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) f[i] = 0.f;
    f[0] = 1.f;
    f[1] = j >= n_int ? 1.f : 0.f;
    {   // row sums over the stencil entries of row j
        const int sl = j >> 5, lane = j & 31;
        const int w = (int)sw[sl];
        const int64_t base = (int64_t)soff[sl] * 32 + lane;
        for (int k = 1; k < w; ++k) {
            const int64_t e = base + (int64_t)k * 32;
            if (col[e] == j) continue;
            const float v = (float)val[e];
            f[2] += fabsf(v);
            f[3] += v;
            f[4] += v * v;
        }
    }
    const int4 cj = ic[j];
    const float inv_h = 1.0f / (float)(1 << (KEY_DEPTH + 1 - cj.w));   // h_j in integer units is 2^(22-l)
    const double B = *bmax;
    float pbsum = 0.f;
    for (int e = rp[j]; e < rp[j + 1]; ++e) {
        const float in = ain[e];
        f[5] += in * in;
        f[6] += fabsf(in);
        const float p = pf[e];
        const int i = ecol[e];
        const int4 ci = ic[i];
        const float dx = (float)(ci.x - cj.x) * inv_h, dy = (float)(ci.y - cj.y) * inv_h,
                    dz = (float)(ci.z - cj.z) * inv_h;
        f[7] += p * dx;
        f[8] += p * dy;
        f[9] += p * dz;
        f[10] += p * (dx * dx + dy * dy + dz * dz);
        f[11] += p * (float)(ci.w - cj.w);
        pbsum += p * (float)b[i];
    }
    if (B > 0.0) {
        f[12] = (float)(b[j] / B);
        f[13] = (float)((double)pbsum / B);
    }
    f[14] = (float)(rp[j + 1] - rp[j]) / 64.f;
    c_out[j] = 1.f + f[5];   // squared norm of column j of Ahat, for the loss
    // the sums of WLS weights are heavy-tailed: signed log1p keeps them O(1)
#pragma unroll
    for (int i = 2; i < 7; ++i) f[i] = copysignf(log1pf(fabsf(f[i])), f[i]);
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        F[(int64_t)j * NF + i] = f[i];
        H0[(int64_t)j * NF + i] = __float2bfloat16_rn(f[i]);
    }
}

// Y = P X (gather with weights w over the symmetric graph), X and Y n x C BF16,
// FP32 sums; one warp per row, lanes over channel pairs
template <int C>
__global__ void k_agg_bf16(const int32_t *__restrict__ rp, const int32_t *__restrict__ ecol,
                           const float *__restrict__ w, const __nv_bfloat16 *__restrict__ X, int n,
                           __nv_bfloat16 *__restrict__ Y) {
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= n || lane >= C / 2) return;
    float a0 = 0.f, a1 = 0.f;
    for (int e = rp[j]; e < rp[j + 1]; ++e) {
        const float p = w[e];
        const __nv_bfloat162 x = reinterpret_cast<const __nv_bfloat162 *>(X + (int64_t)ecol[e] * C)[lane];
        a0 = fmaf(p, __bfloat162float(x.x), a0);
        a1 = fmaf(p, __bfloat162float(x.y), a1);
    }
    reinterpret_cast<__nv_bfloat162 *>(Y + (int64_t)j * C)[lane] = __floats2bfloat162_rn(a0, a1);
}

// dH = dX[:, :C] + P^T dX[:, C:]  (FP32, dX is n x 2C), P^T gathered with pb
template <int C>
__global__ void k_agg_back(const int32_t *__restrict__ rp, const int32_t *__restrict__ ecol,
                           const float *__restrict__ pb, const float *__restrict__ dX, int n, float *__restrict__ dH) {
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= n) return;
    for (int c = lane; c < C; c += 32) {
        float a = dX[(int64_t)j * 2 * C + c];
        for (int e = rp[j]; e < rp[j + 1]; ++e) a = fmaf(pb[e], dX[(int64_t)ecol[e] * 2 * C + C + c], a);
        dH[(int64_t)j * C + c] = a;
    }
}

// ---------------------------------------------------------------- head, loss, backward of the head
__global__ void k_head(const __nv_bfloat16 *__restrict__ H3, const float *__restrict__ theta, int n, int n_int,
                       float *__restrict__ t, float *__restrict__ s, float *__restrict__ gamma) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float *Wo = theta + OFF_WO, *bo = theta + OFF_BO;
    float t0 = bo[0], t1 = bo[1];
    for (int k = 0; k < WD; ++k) {
        const float h = __bfloat162float(H3[(int64_t)j * WD + k]);
        t0 = fmaf(h, Wo[2 * k], t0);
        t1 = fmaf(h, Wo[2 * k + 1], t1);
    }
    t[2 * j] = t0;
    t[2 * j + 1] = t1;
    s[j] = j < n_int ? expf(ALPHA * tanhf(t0)) : 1.f;   // boundary rows are identity rows
    gamma[j] = expf(tanhf(t1));
}

// u0 = gamma * b, r = b - Ahat u0 (row by row over the ELL), per-block sums of
// r^2, b^2 and of the Lp terms 1 - 2 s + s^2 c, c_j the squared column norm
__global__ void k_loss_terms(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                             const int32_t *__restrict__ col, const double *__restrict__ val,
                             const double *__restrict__ b, const float *__restrict__ gamma,
                             const float *__restrict__ s, const float *__restrict__ ccol, int n, int n_int,
                             float *__restrict__ r, double *__restrict__ part) {
    __shared__ double sh[3][256];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0.0, bb = 0.0, lp = 0.0;
    if (j < n) {
        const int sl = j >> 5, lane = j & 31;
        const int w = (int)sw[sl];
        const int64_t base = (int64_t)soff[sl] * 32 + lane;
        double acc = 0.0;
        for (int k = 0; k < w; ++k) {
            const int64_t e = base + (int64_t)k * 32;
            const int i = col[e];
            acc = fma(val[e], (double)gamma[i] * b[i], acc);
        }
        const double rj = b[j] - acc;
        r[j] = (float)rj;
        rr = rj * rj;
        bb = b[j] * b[j];
        const double sj = s[j], cj = (double)ccol[j];
        lp = j < n_int ? 1.0 - 2.0 * sj + sj * sj * cj : 0.0;
    }
    sh[0][threadIdx.x] = rr;
    sh[1][threadIdx.x] = bb;
    sh[2][threadIdx.x] = lp;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) part[(int64_t)blockIdx.x * 3 + q] = sh[q][0];
}

__global__ void k_loss_final(const double *__restrict__ part, int nblk, int n_int, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double rr = 0.0, bb = 0.0, lp = 0.0;
    for (int k = 0; k < nblk; ++k) {
        rr += part[3 * k];
        bb += part[3 * k + 1];
        lp += part[3 * k + 2];
    }
    out[1] = n_int > 0 ? lp / n_int : 0.0;
    out[2] = bb > 0.0 ? rr / bb : 0.0;
    out[0] = out[1] + out[2];
    out[3] = bb;
}

// dt from dLp/ds = (2/n)(s c - 1) and dLg/dgamma = -2 b (Ahat^T r) / ||b||^2;
// (Ahat^T r)_j = r_j + sum over the graph row j of a_in * r_i
__global__ void k_head_back(const int32_t *__restrict__ rp, const int32_t *__restrict__ ecol,
                            const float *__restrict__ ain, const float *__restrict__ r, const double *__restrict__ b,
                            const float *__restrict__ s, const float *__restrict__ gamma, const float *__restrict__ t,
                            const float *__restrict__ ccol, const double *__restrict__ lossv, int n, int n_int,
                            float *__restrict__ dt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float atr = r[j];
    for (int e = rp[j]; e < rp[j + 1]; ++e) atr = fmaf(ain[e], r[ecol[e]], atr);
    const double bb = lossv[3];
    const float cj = ccol[j];
    const float ds = j < n_int ? (2.0f / n_int) * (s[j] * cj - 1.f) : 0.f;
    const float dg = bb > 0.0 ? (float)(-2.0 * b[j] * (double)atr / bb) : 0.f;
    const float th0 = tanhf(t[2 * j]), th1 = tanhf(t[2 * j + 1]);
    dt[2 * j] = ds * s[j] * ALPHA * (1.f - th0 * th0);
    dt[2 * j + 1] = dg * gamma[j] * (1.f - th1 * th1);
}

// head weight gradients: dWo = H3^T dt (64 x 2), dbo = sum dt; per-block
// partials then a fixed-order sum
__global__ void k_head_wgrad(const __nv_bfloat16 *__restrict__ H3, const float *__restrict__ dt, int n,
                             float *__restrict__ part) {
    __shared__ float sh[256];
    float acc[2 * WD + 2];
#pragma unroll 4
    for (int i = 0; i < 2 * WD + 2; ++i) acc[i] = 0.f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const float d0 = dt[2 * j], d1 = dt[2 * j + 1];
        for (int k = 0; k < WD; ++k) {
            const float h = __bfloat162float(H3[(int64_t)j * WD + k]);
            acc[2 * k] = fmaf(h, d0, acc[2 * k]);
            acc[2 * k + 1] = fmaf(h, d1, acc[2 * k + 1]);
        }
        acc[2 * WD] += d0;
        acc[2 * WD + 1] += d1;
    }
    for (int q = 0; q < 2 * WD + 2; ++q) {
        sh[threadIdx.x] = acc[q];
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * (2 * WD + 2) + q] = sh[0];
        __syncthreads();
    }
}

__global__ void k_sum_partials(const float *__restrict__ part, int nblk, int width, float *__restrict__ out) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= width) return;
    float s = 0.f;
    for (int k = 0; k < nblk; ++k) s += part[(int64_t)k * width + q];
    out[q] = s;
}

// dH3 = dt Wo^T, then dZ2 = dH3 * [H3 > 0] in BF16
__global__ void k_head_dH(const float *__restrict__ dt, const float *__restrict__ theta,
                          const __nv_bfloat16 *__restrict__ H3, int n, __nv_bfloat16 *__restrict__ dZ) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * WD) return;
    const int64_t j = i / WD;
    const int k = (int)(i - j * WD);
    const float *Wo = theta + OFF_WO;
    const float d = dt[2 * j] * Wo[2 * k] + dt[2 * j + 1] * Wo[2 * k + 1];
    dZ[i] = __float2bfloat16_rn(__bfloat162float(H3[i]) > 0.f ? d : 0.f);
}

// dZ = dH * [H > 0] in BF16
__global__ void k_relu_back(const float *__restrict__ dH, const __nv_bfloat16 *__restrict__ H, int64_t m,
                            __nv_bfloat16 *__restrict__ dZ) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) dZ[i] = __float2bfloat16_rn(__bfloat162float(H[i]) > 0.f ? dH[i] : 0.f);
}

// db = column sums of dZ (n x 64), per-block partials
__global__ void k_colsum(const __nv_bfloat16 *__restrict__ dZ, int n, float *__restrict__ part) {
    // blockDim 256 = 4 row groups x 64 columns
    __shared__ float sh[256];
    const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
    float s = 0.f;
    for (int j = blockIdx.x * 4 + g; j < n; j += gridDim.x * 4) s += __bfloat162float(dZ[(int64_t)j * WD + c]);
    sh[threadIdx.x] = s;
    __syncthreads();
    if (g == 0) part[(int64_t)blockIdx.x * WD + c] = sh[c] + sh[64 + c] + sh[128 + c] + sh[192 + c];
}

// ---------------------------------------------------------------- parameters
__global__ void k_refresh_bf16(const float *__restrict__ theta, __nv_bfloat16 *w0, __nv_bfloat16 *wt0,
                               __nv_bfloat16 *w1, __nv_bfloat16 *wt1, __nv_bfloat16 *w2, __nv_bfloat16 *wt2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    __nv_bfloat16 *w[3] = {w0, w1, w2}, *wt[3] = {wt0, wt1, wt2};
    const int kl[3] = {2 * NF, 2 * WD, 2 * WD}, offw[3] = {OFF_W0, OFF_W1, OFF_W2};
    int o = i;
    for (int l = 0; l < 3; ++l) {
        const int sz = kl[l] * WD;
        if (o < sz) {
            const int k = o / WD, c = o - k * WD;
            const __nv_bfloat16 v = __float2bfloat16_rn(theta[offw[l] + o]);
            w[l][o] = v;
            wt[l][c * kl[l] + k] = v;
            return;
        }
        o -= sz;
    }
}

__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, int np, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi, v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    theta[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace

int mpnn_num_params() { return N_PARAMS; }

}  // namespace apc

// ---------------------------------------------------------------- host side
namespace apc {
namespace {

// indices of the context buffers used by the network
enum MpBuf {
    MB_CNT = 0, MB_OFF, MB_KEY0, MB_KEY1, MB_REC0, MB_REC1, MB_FLAG, MB_POS, MB_ECOL, MB_AOUT, MB_AIN, MB_UKEY,
    MB_RP, MB_S, MB_PF, MB_PB, MB_F, MB_H0, MB_PH0, MB_H1, MB_PH1, MB_H2, MB_PH2, MB_H3, MB_T, MB_SV, MB_GAMMA,
    MB_R, MB_PART, MB_LOSS, MB_DT, MB_DZ, MB_DX, MB_DH, MB_WPART, MB_BMAX, MB_TICKET, MB_BACKUP, MB_DBACKUP,
    MB_PHI0, MB_CCOL, MB_X0, MB_COUNT
};
static_assert(MB_COUNT <= 48, "buffer slots");

template <class T>
T *mb(apcloud_ctx *c, int i, int64_t count) { return ensure<T>(c, c->mp[i], (size_t)(count > 0 ? count : 1)); }
template <class T>
T *mp(apcloud_ctx *c, int i) { return ptr<T>(c->mp[i]); }

constexpr int GT1 = 256;

// symmetric stencil graph of the current system (built once per matrix:
// apcloud_stencils clears mp_graph_n)
apcloud_status build_graph(apcloud_ctx *c) {
    const int n = c->n_tot;
    if (c->mp_graph_n == n) return APCLOUD_OK;
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    const double *val = ptr<double>(c->ell_A);
    uint32_t *cnt = mb<uint32_t>(c, MB_CNT, n + 1), *off = mb<uint32_t>(c, MB_OFF, n + 1);
    if (!cnt || !off) return APCLOUD_E_NOMEM;
    uint32_t *small = ptr<uint32_t>(c->dsmall);
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(n, GT1), GT1, 0, k_edge_count, sw, so, col, val, n, cnt);
    APC_TRY(scan_u32(c, cnt, off, n, small + 8));
    uint32_t ne;
    APC_TRY(read_back(c, &ne, small + 8, sizeof ne));
    const int64_t m = 2 * (int64_t)ne;
    uint64_t *k0 = mb<uint64_t>(c, MB_KEY0, m), *k1 = mb<uint64_t>(c, MB_KEY1, m);
    uint32_t *r0 = mb<uint32_t>(c, MB_REC0, m), *r1 = mb<uint32_t>(c, MB_REC1, m);
    uint32_t *fl = mb<uint32_t>(c, MB_FLAG, m), *pos = mb<uint32_t>(c, MB_POS, m);
    if (!k0 || !k1 || !r0 || !r1 || !fl || !pos) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(n, GT1), GT1, 0, k_edge_emit, sw, so, col, val, n, (const uint32_t *)off, k0,
               r0);
    int bits = 0;
    while ((1ll << bits) < n) ++bits;
    int which = 0;
    APC_TRY(radix_sort(c, k0, r0, k1, r1, m, 32 + bits, &which));
    const uint64_t *sk = which ? k1 : k0;
    const uint32_t *sr = which ? r1 : r0;
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(m, GT1), GT1, 0, k_run_heads, sk, m, fl);
    APC_TRY(scan_u32(c, fl, pos, m, small + 9));
    uint32_t nu;
    APC_TRY(read_back(c, &nu, small + 9, sizeof nu));
    int32_t *ecol = mb<int32_t>(c, MB_ECOL, nu);
    float *aout = mb<float>(c, MB_AOUT, nu), *ain = mb<float>(c, MB_AIN, nu);
    uint64_t *uk = mb<uint64_t>(c, MB_UKEY, nu);
    int32_t *rp = mb<int32_t>(c, MB_RP, n + 1);
    float *S = mb<float>(c, MB_S, n), *pf = mb<float>(c, MB_PF, nu), *pb = mb<float>(c, MB_PB, nu);
    if (!ecol || !aout || !ain || !uk || !rp || !S || !pf || !pb) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(m, GT1), GT1, 0, k_edge_merge, sk, sr, m, (const uint32_t *)fl,
               (const uint32_t *)pos, val, ecol, aout, ain, uk);
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(n + 1, GT1), GT1, 0, k_rowptr, (const uint64_t *)uk, (int64_t)nu, n, rp);
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(n, GT1), GT1, 0, k_row_sums, (const int32_t *)rp, (const float *)aout,
               (const float *)ain, n, S);
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(n, GT1), GT1, 0, k_agg_weights, (const int32_t *)rp, (const int32_t *)ecol,
               (const float *)aout, (const float *)ain, (const float *)S, n, pf, pb);
    APC_CUDA(c, cudaGetLastError());
    c->mp_graph_n = n;
    return APCLOUD_OK;
}

apcloud_status tc_launch(apcloud_ctx *c, int mode, const TcArgs &a, int grid) {
    // the shared-memory limit is a per-device property of the function: one
    // bit per (device, mode) once it is set there (devices past 63: every call)
    static std::atomic<uint64_t> attr_set[3];
    const uint64_t bit = c->device >= 0 && c->device < 64 ? uint64_t(1) << c->device : 0;
    if (!bit || !(attr_set[mode].load(std::memory_order_relaxed) & bit)) {
        cudaError_t e = mode == 0   ? cudaFuncSetAttribute(k_dense_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM)
                        : mode == 1 ? cudaFuncSetAttribute(k_dense_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM)
                                    : cudaFuncSetAttribute(k_dense_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        APC_CUDA(c, e);
        attr_set[mode].fetch_or(bit, std::memory_order_relaxed);
    }
    if (mode == 0) APC_LAUNCH(c, K_MPNN_TC, grid, TC_THREADS, TC_SMEM, k_dense_tc<0>, a);
    else if (mode == 1) APC_LAUNCH(c, K_MPNN_TC, grid, TC_THREADS, TC_SMEM, k_dense_tc<1>, a);
    else APC_LAUNCH(c, K_MPNN_TC, grid, TC_THREADS, TC_SMEM, k_dense_tc<2>, a);
    return cuda_check(c, cudaGetLastError(), "tensor-core layer");
}

// features, three layers and the head for the Poisson right-hand side b
apcloud_status forward(apcloud_ctx *c, apcloud_mpnn *m, const double *b) {
    APC_TRY(build_graph(c));
    const int n = c->n_tot;
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    const double *val = ptr<double>(c->ell_A);
    double *bmax = mb<double>(c, MB_BMAX, 1);
    unsigned *ticket = mb<unsigned>(c, MB_TICKET, 1);
    double *part = mb<double>(c, MB_PART, 3 * (int64_t)div_up(n, GT1) + 2048);
    float *F = mb<float>(c, MB_F, (int64_t)n * NF);
    __nv_bfloat16 *H[4] = {mb<__nv_bfloat16>(c, MB_H0, (int64_t)n * NF), mb<__nv_bfloat16>(c, MB_H1, (int64_t)n * WD),
                           mb<__nv_bfloat16>(c, MB_H2, (int64_t)n * WD), mb<__nv_bfloat16>(c, MB_H3, (int64_t)n * WD)};
    __nv_bfloat16 *PH[3] = {mb<__nv_bfloat16>(c, MB_PH0, (int64_t)n * NF), mb<__nv_bfloat16>(c, MB_PH1, (int64_t)n * WD),
                            mb<__nv_bfloat16>(c, MB_PH2, (int64_t)n * WD)};
    float *t = mb<float>(c, MB_T, 2 * (int64_t)n), *s = mb<float>(c, MB_SV, n), *gm = mb<float>(c, MB_GAMMA, n);
    float *cc = mb<float>(c, MB_CCOL, n);
    if (!bmax || !ticket || !part || !F || !H[0] || !H[1] || !H[2] || !H[3] || !PH[0] || !PH[1] || !PH[2] || !t ||
        !s || !gm || !cc)
        return APCLOUD_E_NOMEM;
    APC_CUDA(c, cudaMemsetAsync(ticket, 0, sizeof(unsigned), c->s));
    const int nb = div_up(n, GT1) < 1024 ? div_up(n, GT1) : 1024;
    APC_LAUNCH(c, K_MPNN_GRAPH, nb, GT1, 0, k_absmax, b, n, bmax, ticket, part);
    const int32_t *rp = mp<int32_t>(c, MB_RP), *ecol = mp<int32_t>(c, MB_ECOL);
    const float *aout = mp<float>(c, MB_AOUT), *ain = mp<float>(c, MB_AIN), *pf = mp<float>(c, MB_PF);
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(n, GT1), GT1, 0, k_features, sw, so, col, val, rp, ecol, aout, ain, pf,
               ptr<int4>(c->node_ic), n, c->n_int, b, (const double *)bmax, F, H[0], cc);
    for (int l = 0; l < 3; ++l) {
        const int C = l == 0 ? NF : WD;
        if (l == 0)
            APC_LAUNCH(c, K_MPNN_GRAPH, div_up((int64_t)n * 32, GT1), GT1, 0, k_agg_bf16<NF>, rp, ecol, pf,
                       (const __nv_bfloat16 *)H[0], n, PH[0]);
        else
            APC_LAUNCH(c, K_MPNN_GRAPH, div_up((int64_t)n * 32, GT1), GT1, 0, k_agg_bf16<WD>, rp, ecol, pf,
                       (const __nv_bfloat16 *)H[l], n, PH[l]);
        TcArgs a{};
        a.x0 = H[l]; a.x1 = PH[l]; a.c = C;
        a.bmat = m->wt[l];
        a.bias = m->theta + OFF_B[l];
        a.out_bf = H[l + 1];
        a.n = n; a.K = 2 * C; a.N = WD; a.Kl = 2 * C;
        a.err = m->err;
        APC_TRY(tc_launch(c, 0, a, div_up(n, 128)));
    }
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(n, GT1), GT1, 0, k_head, (const __nv_bfloat16 *)H[3],
               (const float *)m->theta, n, c->n_int, t, s, gm);
    return cuda_check(c, cudaGetLastError(), "mpnn forward");
}

apcloud_status check_tc(apcloud_ctx *c, apcloud_mpnn *m) {
    unsigned e;
    APC_TRY(read_back(c, &e, m->err, sizeof e));
    if (e) return fail(c, APCLOUD_E_TIMEOUT, "a tensor-core layer gave up waiting for its MMAs");
    return APCLOUD_OK;
}

// loss (and with backward, every gradient into m->grad)
apcloud_status loss_grad(apcloud_ctx *c, apcloud_mpnn *m, const double *b, bool backward, double *h_loss) {
    const int n = c->n_tot;
    APC_TRY(forward(c, m, b));
    const uint32_t *sw = ptr<uint32_t>(c->slice_w), *so = ptr<uint32_t>(c->slice_off);
    const int32_t *col = ptr<int32_t>(c->ell_col);
    const double *val = ptr<double>(c->ell_A);
    float *r = mb<float>(c, MB_R, n);
    double *lossv = mb<double>(c, MB_LOSS, 4);
    if (!r || !lossv) return APCLOUD_E_NOMEM;
    const int nb = div_up(n, GT1);
    double *part = mp<double>(c, MB_PART);
    APC_LAUNCH(c, K_MPNN_GRAPH, nb, GT1, 0, k_loss_terms, sw, so, col, val, b, (const float *)mp<float>(c, MB_GAMMA),
               (const float *)mp<float>(c, MB_SV), (const float *)mp<float>(c, MB_CCOL), n, c->n_int, r, part);
    APC_LAUNCH(c, K_MPNN_GRAPH, 1, 32, 0, k_loss_final, (const double *)part, nb, c->n_int, lossv);
    if (backward) {
        const int32_t *rp = mp<int32_t>(c, MB_RP), *ecol = mp<int32_t>(c, MB_ECOL);
        const float *ain = mp<float>(c, MB_AIN), *pb = mp<float>(c, MB_PB);
        float *dt = mb<float>(c, MB_DT, 2 * (int64_t)n);
        __nv_bfloat16 *dZ = mb<__nv_bfloat16>(c, MB_DZ, (int64_t)n * WD);
        float *dX = mb<float>(c, MB_DX, (int64_t)n * 2 * WD), *dH = mb<float>(c, MB_DH, (int64_t)n * WD);
        const int wblk = div_up(n, 128) < 2 * 152 ? div_up(n, 128) : 2 * 152;
        float *wpart = mb<float>(c, MB_WPART, (int64_t)wblk * 128 * WD + 1024 * (2 * WD + 2));
        if (!dt || !dZ || !dX || !dH || !wpart) return APCLOUD_E_NOMEM;
        APC_LAUNCH(c, K_MPNN_GRAPH, nb, GT1, 0, k_head_back, rp, ecol, ain, (const float *)r, b,
                   (const float *)mp<float>(c, MB_SV), (const float *)mp<float>(c, MB_GAMMA),
                   (const float *)mp<float>(c, MB_T), (const float *)mp<float>(c, MB_CCOL), (const double *)lossv, n,
                   c->n_int, dt);
        const __nv_bfloat16 *H3 = mp<__nv_bfloat16>(c, MB_H3);
        const int hb = nb < 1024 ? nb : 1024;
        APC_LAUNCH(c, K_MPNN_GRAPH, hb, GT1, 0, k_head_wgrad, H3, (const float *)dt, n, wpart);
        APC_LAUNCH(c, K_MPNN_GRAPH, 1, 2 * WD + 2, 0, k_sum_partials, (const float *)wpart, hb, 2 * WD + 2,
                   m->grad + OFF_WO);
        APC_LAUNCH(c, K_MPNN_GRAPH, div_up((int64_t)n * WD, GT1), GT1, 0, k_head_dH, (const float *)dt,
                   (const float *)m->theta, H3, n, dZ);
        const int HB[3] = {MB_H0, MB_H1, MB_H2}, PB[3] = {MB_PH0, MB_PH1, MB_PH2};
        for (int l = 2; l >= 0; --l) {
            const int C = l == 0 ? NF : WD, Kl = 2 * C;
            // dW_l = [H_l | P H_l]^T dZ on the tensor cores, then a fixed-order sum
            TcArgs a{};
            a.x0 = mp<__nv_bfloat16>(c, HB[l]); a.x1 = mp<__nv_bfloat16>(c, PB[l]); a.c = C;
            a.g = dZ; a.out_f = wpart; a.n = n; a.K = 128; a.N = WD; a.Kl = Kl; a.err = m->err;
            APC_TRY(tc_launch(c, 2, a, wblk));
            APC_LAUNCH(c, K_MPNN_GRAPH, div_up(Kl * WD, GT1), GT1, 0, k_wgrad_reduce, (const float *)wpart, wblk, Kl,
                       m->grad + OFF_W[l]);
            const int cb = div_up(n, 4) < 1024 ? div_up(n, 4) : 1024;
            APC_LAUNCH(c, K_MPNN_GRAPH, cb, 256, 0, k_colsum, (const __nv_bfloat16 *)dZ, n, wpart);
            APC_LAUNCH(c, K_MPNN_GRAPH, 1, WD, 0, k_sum_partials, (const float *)wpart, cb, WD, m->grad + OFF_B[l]);
            if (l == 0) break;
            // dX = dZ W_l^T (tensor cores), dH_l = dX[:, :C] + P^T dX[:, C:], dZ_{l-1} = dH_l * [H_l > 0]
            TcArgs d{};
            d.x0 = dZ; d.x1 = nullptr; d.c = WD; d.bmat = m->w[l]; d.out_f = dX;
            d.n = n; d.K = WD; d.N = Kl; d.Kl = Kl; d.err = m->err;
            APC_TRY(tc_launch(c, 1, d, div_up(n, 128)));
            APC_LAUNCH(c, K_MPNN_GRAPH, div_up((int64_t)n * 32, GT1), GT1, 0, k_agg_back<WD>, rp, ecol, pb,
                       (const float *)dX, n, dH);
            APC_LAUNCH(c, K_MPNN_GRAPH, div_up((int64_t)n * WD, GT1), GT1, 0, k_relu_back, (const float *)dH,
                       (const __nv_bfloat16 *)mp<__nv_bfloat16>(c, HB[l]), (int64_t)n * WD, dZ);
        }
    }
    APC_CUDA(c, cudaGetLastError());
    APC_TRY(check_tc(c, m));
    double h[4];
    APC_TRY(read_back(c, h, lossv, sizeof h));
    if (h_loss) { h_loss[0] = h[0]; h_loss[1] = h[1]; h_loss[2] = h[2]; }
    return APCLOUD_OK;
}

__global__ void k_scale_cols(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                             const int32_t *__restrict__ col, double *__restrict__ val, const float *__restrict__ s,
                             int n, double *__restrict__ d) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int sl = r >> 5, lane = r & 31;
    const int w = (int)sw[sl];
    const int64_t base = (int64_t)soff[sl] * 32 + lane;
    for (int k = 0; k < w; ++k) {
        const int64_t e = base + (int64_t)k * 32;
        val[e] *= (double)s[col[e]];
    }
    d[r] /= (double)s[r];
}

// closed-form minimiser of the approximate-inverse objective: s_j = 1 / c_j
// on interior columns, 1 on boundary ones
__global__ void k_spai_diag(const float *__restrict__ ccol, int n, int n_int, float *__restrict__ s) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) s[j] = (j < n_int && ccol[j] > 0.f) ? 1.f / ccol[j] : 1.f;
}

__global__ void k_guess(const float *__restrict__ gamma, const double *__restrict__ b, const double *__restrict__ d,
                        int n, double *__restrict__ x0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) x0[j] = (double)gamma[j] * b[j] / d[j];
}

}  // namespace
}  // namespace apc

// ---------------------------------------------------------------- C ABI
using namespace apc;

extern "C" int apcloud_mpnn_num_params(void) { return N_PARAMS; }

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), output k of a seeded stream
static uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" apcloud_status apcloud_mpnn_create(const float *h_theta, uint64_t seed, apcloud_mpnn **out) {
    if (!out) return APCLOUD_E_INVALID;
    *out = nullptr;
    std::vector<float> init;
    if (!h_theta) {
        // Glorot-uniform layers, zero biases and a zero head: the untrained
        // network is exactly Jacobi (s = 1) with the guess u0 = b
        init.assign(N_PARAMS, 0.f);
        uint64_t k = seed * 0x632BE59BD9B4E019ull;
        for (int l = 0; l < 3; ++l) {
            const double lim = std::sqrt(6.0 / (K_L[l] + WD));
            for (int i = 0; i < K_L[l] * WD; ++i) {
                const double u = (double)(splitmix64(k += 0x9E3779B97F4A7C15ull) >> 11) * (1.0 / 9007199254740992.0);
                init[OFF_W[l] + i] = (float)((2.0 * u - 1.0) * lim);
            }
        }
        h_theta = init.data();
    }
    apcloud_mpnn *m = new apcloud_mpnn;
    bool ok = cudaMalloc(&m->theta, 4 * N_PARAMS * sizeof(float)) == cudaSuccess;
    if (ok) {
        m->grad = m->theta + N_PARAMS;
        m->m1 = m->grad + N_PARAMS;
        m->m2 = m->m1 + N_PARAMS;
        ok = cudaMemset(m->theta, 0, 4 * N_PARAMS * sizeof(float)) == cudaSuccess;
    }
    int total = 0;
    for (int l = 0; l < 3; ++l) total += 2 * K_L[l] * WD;
    __nv_bfloat16 *wb = nullptr;
    if (ok) ok = cudaMalloc(&wb, total * sizeof(__nv_bfloat16)) == cudaSuccess;
    if (ok) {
        for (int l = 0; l < 3; ++l) {
            m->w[l] = wb;
            m->wt[l] = wb + K_L[l] * WD;
            wb += 2 * K_L[l] * WD;
        }
        ok = cudaMalloc(&m->err, sizeof(unsigned)) == cudaSuccess && cudaMemset(m->err, 0, sizeof(unsigned)) == cudaSuccess;
    }
    if (ok && h_theta) ok = cudaMemcpy(m->theta, h_theta, N_PARAMS * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) {
        k_refresh_bf16<<<div_up(2 * (2 * WD + 2 * NF) * WD, 256), 256>>>(m->theta, m->w[0], m->wt[0], m->w[1],
                                                                          m->wt[1], m->w[2], m->wt[2]);
        ok = cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        apcloud_mpnn_destroy(m);
        return APCLOUD_E_CUDA;
    }
    *out = m;
    return APCLOUD_OK;
}

extern "C" void apcloud_mpnn_destroy(apcloud_mpnn *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    if (m->theta) cudaFree(m->theta);
    if (m->w[0]) cudaFree(m->w[0]);
    if (m->err) cudaFree(m->err);
    delete m;
}

extern "C" apcloud_status apcloud_mpnn_get_params(apcloud_mpnn *m, float *h_theta, float *h_grad) {
    if (!m) return APCLOUD_E_INVALID;
    if (cudaDeviceSynchronize() != cudaSuccess) return APCLOUD_E_CUDA;
    if (h_theta && cudaMemcpy(h_theta, m->theta, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return APCLOUD_E_CUDA;
    if (h_grad && cudaMemcpy(h_grad, m->grad, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return APCLOUD_E_CUDA;
    return APCLOUD_OK;
}

extern "C" apcloud_status apcloud_mpnn_set_params(apcloud_mpnn *m, const float *h_theta) {
    if (!m || !h_theta) return APCLOUD_E_INVALID;
    if (cudaDeviceSynchronize() != cudaSuccess) return APCLOUD_E_CUDA;
    if (cudaMemcpy(m->theta, h_theta, N_PARAMS * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return APCLOUD_E_CUDA;
    cudaMemset(m->m1, 0, 2 * N_PARAMS * sizeof(float));
    m->adam_steps = 0;
    k_refresh_bf16<<<div_up(2 * (2 * WD + 2 * NF) * WD, 256), 256>>>(m->theta, m->w[0], m->wt[0], m->w[1], m->wt[1],
                                                                      m->w[2], m->wt[2]);
    return cudaDeviceSynchronize() == cudaSuccess ? APCLOUD_OK : APCLOUD_E_CUDA;
}

extern "C" apcloud_status apcloud_mpnn_loss(apcloud_ctx *c, apcloud_mpnn *m, int backward, double *h_loss) {
    if (!c || !m) return APCLOUD_E_INVALID;
    if (c->stage < 3) return fail(c, APCLOUD_E_STATE, "the network needs the Poisson right-hand side: deposit first");
    const double *b = poisson_rhs(c, nullptr);
    if (!b) return APCLOUD_E_NOMEM;
    return loss_grad(c, m, b, backward != 0, h_loss);
}

extern "C" apcloud_status apcloud_mpnn_adam(apcloud_ctx *c, apcloud_mpnn *m, float lr) {
    if (!c || !m || !(lr > 0.f)) return APCLOUD_E_INVALID;
    m->adam_steps++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->adam_steps), c2 = 1.f - powf(b2, (float)m->adam_steps);
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(N_PARAMS, 256), 256, 0, k_adam, m->theta, (const float *)m->grad, m->m1, m->m2,
               N_PARAMS, lr, b1, b2, 1e-8f, c1, c2);
    APC_LAUNCH(c, K_MPNN_GRAPH, div_up(2 * (2 * WD + 2 * NF) * WD, 256), 256, 0, k_refresh_bf16,
               (const float *)m->theta, m->w[0], m->wt[0], m->w[1], m->wt[1], m->w[2], m->wt[2]);
    return cuda_check(c, cudaGetLastError(), "adam");
}

extern "C" apcloud_status apcloud_mpnn_outputs(apcloud_ctx *c, apcloud_mpnn *m, float *d_s, float *d_gamma,
                                               float *d_features) {
    if (!c || !m) return APCLOUD_E_INVALID;
    if (c->stage < 3) return fail(c, APCLOUD_E_STATE, "the network needs the Poisson right-hand side: deposit first");
    const double *b = poisson_rhs(c, nullptr);
    if (!b) return APCLOUD_E_NOMEM;
    APC_TRY(forward(c, m, b));
    const int n = c->n_tot;
    if (d_s) APC_CUDA(c, cudaMemcpyAsync(d_s, mp<float>(c, MB_SV), n * sizeof(float), cudaMemcpyDeviceToDevice, c->s));
    if (d_gamma)
        APC_CUDA(c, cudaMemcpyAsync(d_gamma, mp<float>(c, MB_GAMMA), n * sizeof(float), cudaMemcpyDeviceToDevice, c->s));
    if (d_features)
        APC_CUDA(c, cudaMemcpyAsync(d_features, mp<float>(c, MB_F), (size_t)n * NF * sizeof(float),
                                    cudaMemcpyDeviceToDevice, c->s));
    APC_TRY(check_tc(c, m));
    return cuda_check(c, cudaStreamSynchronize(c->s), "mpnn outputs");
}

extern "C" apcloud_status apcloud_solve_learned(apcloud_ctx *c, apcloud_mpnn *m, unsigned use, const double *phi0,
                                                double rtol, int max_iter, double *d_phi_out,
                                                apcloud_solve_info *info) {
    if (!c || !m) return APCLOUD_E_INVALID;
    if (c->stage < 3) return fail(c, APCLOUD_E_STATE, "apcloud_solve_learned before apcloud_deposit");
    if (!(rtol > 0) || max_iter < 0) return fail(c, APCLOUD_E_INVALID, "rtol must be > 0 and max_iter >= 0");
    const int n = c->n_tot;
    double *b = poisson_rhs(c, nullptr);
    double *phi = ensure<double>(c, c->phi, n + 1);
    if (!b || !phi) return APCLOUD_E_NOMEM;
    APC_TRY(forward(c, m, b));
    APC_TRY(check_tc(c, m));
    double *dA = ptr<double>(c->dA);
    // initial guess from the original Jacobi scaling: x0 = gamma b / d
    if (use & 2u)
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_guess, (const float *)mp<float>(c, MB_GAMMA), (const double *)b,
                   (const double *)dA, n, phi);
    else if (phi0)
        APC_CUDA(c, cudaMemcpyAsync(phi, phi0, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    else
        APC_CUDA(c, cudaMemsetAsync(phi, 0, sizeof(double) * n, c->s));
    double *bk = nullptr, *dbk = nullptr;
    const float *scale = mp<float>(c, MB_SV);
    if (use & 4u) {
        // the closed-form diagonal instead of the network's (comparison baseline)
        float *sd = mb<float>(c, MB_PHI0, n);
        if (!sd) return APCLOUD_E_NOMEM;
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_spai_diag, (const float *)mp<float>(c, MB_CCOL), n, c->n_int,
                   sd);
        scale = sd;
        use |= 1u;
    }
    if (use & 1u) {
        // Ahat S: scale the stored columns by s and the diagonal by 1/s; keep the originals
        bk = mb<double>(c, MB_BACKUP, c->ell_entries);
        dbk = mb<double>(c, MB_DBACKUP, n);
        if (!bk || !dbk) return APCLOUD_E_NOMEM;
        APC_CUDA(c, cudaMemcpyAsync(bk, ptr<double>(c->ell_A), sizeof(double) * c->ell_entries, cudaMemcpyDeviceToDevice, c->s));
        APC_CUDA(c, cudaMemcpyAsync(dbk, dA, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
        APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_scale_cols, ptr<uint32_t>(c->slice_w),
                   ptr<uint32_t>(c->slice_off), ptr<int32_t>(c->ell_col), ptr<double>(c->ell_A), scale, n, dA);
        APC_TRY(refresh_lowp(c));
    }
    // the scaled phase gets at most LEARNED_STEPS Arnoldi steps; a solve it has
    // not finished continues with plain Jacobi from its iterate (the fallback)
    const int budget = (use & 1u) && max_iter > LEARNED_STEPS ? LEARNED_STEPS : max_iter;
    double *x0 = nullptr;
    if (budget < max_iter) {   // keep the start: the fallback begins from it, not from the scaled phase's iterate
        x0 = mb<double>(c, MB_X0, n);
        if (!x0) return APCLOUD_E_NOMEM;
        APC_CUDA(c, cudaMemcpyAsync(x0, phi, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    }
    apcloud_solve_info i1{};
    apcloud_status st = gmres_solve(c, 1, b, phi, rtol, budget, &i1);
    if (use & 1u) {
        APC_CUDA(c, cudaMemcpyAsync(ptr<double>(c->ell_A), bk, sizeof(double) * c->ell_entries, cudaMemcpyDeviceToDevice, c->s));
        APC_CUDA(c, cudaMemcpyAsync(dA, dbk, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
        APC_TRY(refresh_lowp(c));
    }
    if (st < 0) return st;
    if (st == APCLOUD_W_NOT_CONVERGED && budget < max_iter) {
        // restarted GMRES can stall on the rough residual a failed scaled phase
        // leaves, so the plain solve starts again from the original start
        APC_CUDA(c, cudaMemcpyAsync(phi, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
        apcloud_solve_info i2{};
        st = gmres_solve(c, 1, b, phi, rtol, max_iter - i1.iters, &i2);
        if (st < 0) return st;
        i1.iters += i2.iters;
        i1.restarts += i2.restarts;
        i1.relres = i2.relres;
    }
    if (info) *info = i1;
    if (d_phi_out) APC_CUDA(c, cudaMemcpyAsync(d_phi_out, phi, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    c->stage = 4;
    return st;
}

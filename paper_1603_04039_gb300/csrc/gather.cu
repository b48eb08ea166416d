// gather.cu -- Section 3.2 step 3: GFD gradient and Hessian of phi at every
// interior node, and second-order Taylor interpolation of phi and E = grad phi
// (Section 2) from the centre of each particle's own leaf.
//
// Node pass: one thread per node walks its ELL row (the stencil neighbours in
// order) and the derivative operator stored with nodes fastest, so the loads
// of a warp are contiguous.  Particle pass: one thread per particle in the
// caller's order reads the particle's leaf (recorded when the tree was
// built), its position, the leaf's centre and its record (potential and
// derivatives), and writes phi and E coalesced; the particle streams bypass L2
// retention so the node records stay cached.  Interpolation at arbitrary
// points (no recorded leaf) recomputes the point's Morton key and finds its
// leaf by binary search over the Morton-ordered leaf anchors (the leaves
// partition the key space).
#include <cmath>

#include "fpconv.cuh"
#include "internal.cuh"

namespace apc {

namespace {

constexpr int NF = 12;  // per-node record: phi, 9 derivatives, 2 pad
// compact per-node record of the mixed form's particle pass, 80 bytes in 4-byte
// words: phi and the node centre (FP64, words 0-7), gradient and Hessian
// fx fy fz fxx fxy fxz fyy fyz fzz (FP32, words 8-16), pad
constexpr int NF32 = 20;

__global__ void k_derivs(const uint32_t *__restrict__ sw, const uint32_t *__restrict__ soff,
                         const int32_t *__restrict__ col, const double *__restrict__ D, int64_t dstride,
                         const double *__restrict__ phi, int n_int, double *__restrict__ nf,
                         const int4 *__restrict__ ic, double lo0, double lo1, double lo2, double unit,
                         float *__restrict__ nf32) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_int) return;
    const int sl = j >> 5, lane = j & 31;
    const int w = (int)sw[sl];
    const int64_t base = (int64_t)soff[sl] * 32 + lane;
    const double p0 = phi[j];
    double acc[NCOL];
#pragma unroll
    for (int r = 0; r < NCOL; ++r) acc[r] = 0.0;
    for (int k = 1; k < w; ++k) {
        const int cj = col[base + (int64_t)k * 32];
        const double diff = phi[cj] - p0;
#pragma unroll
        for (int r = 0; r < NCOL; ++r) acc[r] = fma(D[((int64_t)r * MMAX + (k - 1)) * dstride + j], diff, acc[r]);
    }
    double *o = nf + (int64_t)j * NF;
    o[0] = p0;
#pragma unroll
    for (int r = 0; r < NCOL; ++r) o[1 + r] = acc[r];
    o[10] = 0.0;
    o[11] = 0.0;
    if (nf32) {
        const int4 q = ic[j];
        double2 *c2 = reinterpret_cast<double2 *>(nf32 + (int64_t)j * NF32);
        c2[0] = make_double2(p0, __dadd_rn(lo0, __dmul_rn((double)q.x, unit)));
        c2[1] = make_double2(__dadd_rn(lo1, __dmul_rn((double)q.y, unit)), __dadd_rn(lo2, __dmul_rn((double)q.z, unit)));
        float4 *f4 = reinterpret_cast<float4 *>(nf32 + (int64_t)j * NF32 + 8);
        f4[0] = make_float4((float)acc[0], (float)acc[1], (float)acc[2], (float)acc[3]);
        f4[1] = make_float4((float)acc[4], (float)acc[5], (float)acc[6], (float)acc[7]);
        f4[2] = make_float4((float)acc[8], 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ int leaf_of(const uint64_t *anchor, int n, uint64_t v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(anchor + mid) <= v) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

// Second-order Taylor expansion about the leaf centre (Section 3.2 step 3):
// phi_p = phi + g.r + r.H.r / 2, E_p = g + H r (E = grad phi, Section 2).
__device__ __forceinline__ void taylor(const double *__restrict__ nf, int j, double r0, double r1, double r2,
                                       double &php, double &ex, double &ey, double &ez) {
    const double2 *f2 = reinterpret_cast<const double2 *>(nf + (int64_t)j * NF);
    const double2 a = f2[0], b = f2[1], c = f2[2], d = f2[3], e = f2[4];
    // a = (phi, fx), b = (fy, fz), c = (fxx, fxy), d = (fxz, fyy), e = (fyz, fzz)
    const double hr0 = c.x * r0 + c.y * r1 + d.x * r2;
    const double hr1 = c.y * r0 + d.y * r1 + e.x * r2;
    const double hr2 = d.x * r0 + e.x * r1 + e.y * r2;
    const double g0 = a.y, g1 = b.x, g2 = b.y;
    php = a.x + (g0 * r0 + g1 * r1 + g2 * r2) + 0.5 * (r0 * hr0 + r1 * hr1 + r2 * hr2);
    ex = g0 + hr0;
    ey = g1 + hr1;
    ez = g2 + hr2;
}

template <bool F32>
__global__ void __launch_bounds__(256) k_gather_leaf(
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z, int64_t n,
    double lo0, double lo1, double lo2, double unit, const int32_t *__restrict__ pleaf, const int4 *__restrict__ ic,
    const double *__restrict__ nf, const float *__restrict__ nf32, double *__restrict__ php, double *__restrict__ ex,
    double *__restrict__ ey, double *__restrict__ ez) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = __ldcs(pleaf + i);
    const double p0 = __ldcs(x + i), p1 = __ldcs(y + i), p2 = __ldcs(z + i);
    double v, gx, gy, gz;
    if (F32) {
        // the mixed form: corrections (g.r, H r, r.H.r) in FP32 around the FP64
        // node potential, from the compact record; its node derivatives carry
        // FP32 accuracy already (FP32 stencils).  The pass stays off the slow
        // FP64 pipe but for the offsets from the centre and the potential's
        // add: the seven double/float conversions run on the integer pipe
        const double2 *c2 = reinterpret_cast<const double2 *>(nf32 + (int64_t)j * NF32);
        const float4 *f4 = reinterpret_cast<const float4 *>(nf32 + (int64_t)j * NF32 + 8);
        const double2 pc = c2[0], cc = c2[1];
        const float4 u = f4[0], w = f4[1], t = f4[2];
        const float r0 = f64_to_f32_int(p0 - pc.y), r1 = f64_to_f32_int(p1 - cc.x), r2 = f64_to_f32_int(p2 - cc.y);
        // u = (fx, fy, fz, fxx), w = (fxy, fxz, fyy, fyz), t.x = fzz
        const float hr0 = fmaf(w.y, r2, fmaf(w.x, r1, u.w * r0));
        const float hr1 = fmaf(w.w, r2, fmaf(w.z, r1, w.x * r0));
        const float hr2 = fmaf(t.x, r2, fmaf(w.w, r1, w.y * r0));
        const float corr = fmaf(u.z, r2, fmaf(u.y, r1, u.x * r0)) + 0.5f * fmaf(r2, hr2, fmaf(r1, hr1, r0 * hr0));
        v = pc.x + f32_to_f64_int(corr);
        gx = f32_to_f64_int(u.x + hr0);
        gy = f32_to_f64_int(u.y + hr1);
        gz = f32_to_f64_int(u.z + hr2);
    } else {
        const int4 q = ic[j];
        const double r0 = p0 - __dadd_rn(lo0, __dmul_rn((double)q.x, unit));
        const double r1 = p1 - __dadd_rn(lo1, __dmul_rn((double)q.y, unit));
        const double r2 = p2 - __dadd_rn(lo2, __dmul_rn((double)q.z, unit));
        taylor(nf, j, r0, r1, r2, v, gx, gy, gz);
    }
    if (php) __stcs(php + i, v);
    if (ex) __stcs(ex + i, gx);
    if (ey) __stcs(ey + i, gy);
    if (ez) __stcs(ez + i, gz);
}

__global__ void k_gather(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                         int64_t n, double lo0, double lo1, double lo2, double s, int shift, double unit,
                         const int64_t *__restrict__ offs, int nb, int L, const uint64_t *__restrict__ anchor, int n_int, const int4 *__restrict__ ic,
                         const double *__restrict__ nf, double *__restrict__ php, double *__restrict__ ex,
                         double *__restrict__ ey, double *__restrict__ ez) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p[3] = {x[i], y[i], z[i]};
    const double lo[3] = {lo0, lo1, lo2};
    uint32_t cc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double t = floor(__dmul_rn(__dsub_rn(p[d], lo[d]), s));
        t = fmin(fmax(t, 0.0), (double)((1u << KEY_DEPTH) - 1u));
        cc[d] = (uint32_t)t >> shift;
    }
    uint64_t pre = 0;
    if (nb > 1) {   // beam of particle i from the batch offsets
        int lo = 0, hi = nb;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (offs[mid] <= i) lo = mid; else hi = mid;
        }
        pre = (uint64_t)lo << (3 * L);
    }
    const int j = leaf_of(anchor, n_int, pre | morton(cc[0], cc[1], cc[2]));
    const int4 q = ic[j];
    const double r0 = p[0] - __dadd_rn(lo0, __dmul_rn((double)q.x, unit));
    const double r1 = p[1] - __dadd_rn(lo1, __dmul_rn((double)q.y, unit));
    const double r2 = p[2] - __dadd_rn(lo2, __dmul_rn((double)q.z, unit));
    double v, gx, gy, gz;
    taylor(nf, j, r0, r1, r2, v, gx, gy, gz);
    if (php) php[i] = v;
    if (ex) ex[i] = gx;
    if (ey) ey[i] = gy;
    if (ez) ez[i] = gz;
}

}  // namespace

apcloud_status gather_field(apcloud_ctx *c, double *phi_p, double *ex, double *ey, double *ez) {
    const int n = c->n_int;
    const bool mixed = c->P.precision == 1;
    double *nf = ensure<double>(c, c->nodefield, (int64_t)n * NF);
    float *nf32 = mixed ? ensure<float>(c, c->nodefield32, (int64_t)n * NF32 + 4) : nullptr;
    if (!nf || (mixed && !nf32)) return APCLOUD_E_NOMEM;
    const int64_t dstride = ((int64_t)n + 31) / 32 * 32;
    const double ext = c->P.hi[0] - c->P.lo[0];
    const double unit = ldexp(ext, -(KEY_DEPTH + 1));
    APC_LAUNCH(c, K_DERIV, div_up(n, 128), 128, 0, k_derivs, ptr<uint32_t>(c->slice_w), ptr<uint32_t>(c->slice_off),
               ptr<int32_t>(c->ell_col), ptr<double>(c->D), dstride, ptr<double>(c->phi), n, nf,
               ptr<int4>(c->node_ic), c->P.lo[0], c->P.lo[1], c->P.lo[2], unit, nf32);
    if (mixed)
        APC_LAUNCH(c, K_GATHER, div_up(c->N, 256), 256, 0, k_gather_leaf<true>, c->px, c->py, c->pz, c->N,
                   c->P.lo[0], c->P.lo[1], c->P.lo[2], unit, (const int32_t *)ptr<int32_t>(c->pleaf),
                   ptr<int4>(c->node_ic), (const double *)nf, (const float *)nf32, phi_p, ex, ey, ez);
    else
        APC_LAUNCH(c, K_GATHER, div_up(c->N, 256), 256, 0, k_gather_leaf<false>, c->px, c->py, c->pz, c->N,
                   c->P.lo[0], c->P.lo[1], c->P.lo[2], unit, (const int32_t *)ptr<int32_t>(c->pleaf),
                   ptr<int4>(c->node_ic), (const double *)nf, (const float *)nullptr, phi_p, ex, ey, ez);
    // node pass: operator (72 B), column (4 B) and neighbour value (8 B) per
    // stencil entry plus the 96 B record (and the 80 B compact record of the
    // mixed form); particle pass: leaf index and position in (28 B), phi and E
    // out (32 B), and each leaf's record once (FP64: 96 B and the 16 B centre;
    // mixed: the 80 B compact record)
    account(c, K_DERIV, 84.0 * c->sum_m + (mixed ? 200.0 : 104.0) * n, 19.0 * c->sum_m);
    account(c, K_GATHER, 60.0 * c->N + (mixed ? 80.0 : 112.0) * n, 38.0 * c->N);
    return cuda_check(c, cudaGetLastError(), "gather");
}

}  // namespace apc

// ---------------------------------------------------------------- time stepping support
namespace apc {
namespace {

// Leapfrog half steps for particles with charge-to-mass ratio qm in the field
// E = grad phi (Section 2): v += qm dt_kick E, then x += dt_drift v, with
// specular reflection at the walls of the cubic domain.
__global__ void k_push(double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                       double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz, int64_t n,
                       const double *__restrict__ ex, const double *__restrict__ ey, const double *__restrict__ ez,
                       double qm_dt, double dt, double lo, double hi) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double p[3] = {x[i], y[i], z[i]}, v[3] = {vx[i], vy[i], vz[i]};
    if (ex) { v[0] += qm_dt * ex[i]; v[1] += qm_dt * ey[i]; v[2] += qm_dt * ez[i]; }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p[d] += dt * v[d];
        if (p[d] > hi) { p[d] = 2.0 * hi - p[d]; v[d] = -v[d]; }
        if (p[d] < lo) { p[d] = 2.0 * lo - p[d]; v[d] = -v[d]; }
        p[d] = fmin(fmax(p[d], lo), hi);
    }
    x[i] = p[0]; y[i] = p[1]; z[i] = p[2];
    vx[i] = v[0]; vy[i] = v[1]; vz[i] = v[2];
}

// W = 1/2 sum over leaves of |grad phi|^2 h^3 (node derivatives times cell volume),
// one block, fixed summation order
__global__ void k_field_energy(const double *__restrict__ nf, const int4 *__restrict__ ic, int n, double ext,
                               double *__restrict__ out) {
    __shared__ double sh[1024];
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double *f = nf + (int64_t)j * NF;
        double h = ldexp(ext, -ic[j].w);
        s += (f[1] * f[1] + f[2] * f[2] + f[3] * f[3]) * (h * h * h);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 0.5 * sh[0];
}

}  // namespace

apcloud_status interpolate_phi(apcloud_ctx *c, const double *x, const double *y, const double *z, int64_t n,
                               double *phi) {
    const double ext = c->P.hi[0] - c->P.lo[0];
    const double s = ldexp(1.0, KEY_DEPTH) / ext;
    const double unit = ldexp(ext, -(KEY_DEPTH + 1));
    APC_LAUNCH(c, K_GATHER, div_up(n, 256), 256, 0, k_gather, x, y, z, n, c->P.lo[0], c->P.lo[1], c->P.lo[2], s,
               KEY_DEPTH - c->L, unit, (const int64_t *)nullptr, 1, c->L, ptr<uint64_t>(c->leaf_anchor), c->n_int,
               ptr<int4>(c->node_ic),
               ptr<double>(c->nodefield), phi, (double *)nullptr, (double *)nullptr, (double *)nullptr);
    return cuda_check(c, cudaGetLastError(), "interpolate");
}

apcloud_status push(apcloud_ctx *c, double *x, double *y, double *z, double *vx, double *vy, double *vz, int64_t n,
                    const double *ex, const double *ey, const double *ez, double qm_dt, double dt) {
    APC_LAUNCH(c, K_VEC, div_up(n, 256), 256, 0, k_push, x, y, z, vx, vy, vz, n, ex, ey, ez, qm_dt, dt, c->P.lo[0],
               c->P.hi[0]);
    return cuda_check(c, cudaGetLastError(), "push");
}

apcloud_status field_energy(apcloud_ctx *c, double *h_out) {
    double *tmp = ensure<double>(c, c->tmp, 2);
    if (!tmp) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_VEC, 1, 1024, 0, k_field_energy, ptr<double>(c->nodefield), ptr<int4>(c->node_ic), c->n_int,
               c->P.hi[0] - c->P.lo[0], tmp);
    return read_back(c, h_out, tmp, sizeof(double));
}

}  // namespace apc

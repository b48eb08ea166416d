// ilu.cu -- ILU(0)-preconditioned GMRES, the comparison baseline that the
// learned preconditioner is measured against (besides Jacobi).  The paper has
// no counterpart.  ILU(0) is the incomplete LU factorisation without fill
// outside the pattern of A, computed row by row in the IKJ order (Saad,
// Iterative Methods for Sparse Linear Systems, 2nd ed., Algorithm 10.4).
//
// The factors are computed once per call on the host from the stored FP64
// matrix (the same column-scaled values the Krylov loop multiplies); every
// application of the preconditioner, z = (LU)^-1 v, runs on the GPU as two
// level-scheduled triangular sweeps: the rows of a level depend only on rows of
// earlier levels.  A wide level is one launch over its rows; a run of
// consecutive narrow levels is one launch of a single block that takes them in
// order, with a block barrier between levels (the octree matrices have
// thousands of levels of a few hundred rows, where a launch per level costs
// more than the level's work).  Each row sums in the same order either way.
#include <algorithm>
#include <chrono>
#include <vector>

#include "internal.cuh"

namespace apc {

namespace {

constexpr int ILU_RUN_THREADS = 1024;   // threads of a one-block run of narrow levels
constexpr int ILU_WIDE_ROWS = 4096;     // wider levels get a launch of their own
static_assert(sizeof(int) == sizeof(int32_t), "level offsets are copied to the device as int32");

// s - sum_{e0 <= e < e1} a[e] z[cj[e]], subtracted in order of e.  The
// entries' columns and values are loaded 8 at a time ahead of the z loads
// they feed, so a row costs a few dependent loads rather than two per entry.
__device__ __forceinline__ double row_minus(double s, int64_t e0, int64_t e1, const int32_t *__restrict__ cj,
                                            const double *__restrict__ a, const double *z) {
    for (; e0 < e1; e0 += 8) {
        int j[8];
        double av[8], zv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            j[k] = e0 + k < e1 ? cj[e0 + k] : 0;
            av[k] = e0 + k < e1 ? a[e0 + k] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) zv[k] = e0 + k < e1 ? z[j[k]] : 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (e0 + k < e1) s -= av[k] * zv[k];
    }
    return s;
}

// forward sweep, one level: z[r] = v[r] - sum_{k < r} L_rk z[k] (L unit lower)
__global__ void k_ilu_lower(const int32_t *__restrict__ rows, int p0, int p1, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ cj, const double *__restrict__ lv,
                            const double *__restrict__ v, double *__restrict__ z, const GmresState *__restrict__ st) {
    if (st->done) return;
    const int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    const int r = rows[p];
    const double s = row_minus(v[r], rp[p], rp[p + 1], cj, lv, z);
    z[r] = s;
}

// backward sweep, one level: z[r] = (z[r] - sum_{j > r} U_rj z[j]) / U_rr
__global__ void k_ilu_upper(const int32_t *__restrict__ rows, int p0, int p1, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ cj, const double *__restrict__ uv,
                            const double *__restrict__ dinv, double *__restrict__ z,
                            const GmresState *__restrict__ st) {
    if (st->done) return;
    const int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    const int r = rows[p];
    const double s = row_minus(z[r], rp[p], rp[p + 1], cj, uv, z);
    z[r] = s * dinv[p];
}

// A run of narrow levels [l0, l1) of the forward sweep in one block.  The
// barrier after each level also makes that level's z values visible to the
// block's reads in the next, so z is read through the ordinary (coherent) path.
__global__ void __launch_bounds__(ILU_RUN_THREADS)
    k_ilu_lower_run(const int32_t *__restrict__ rows, const int32_t *__restrict__ off, int l0, int l1,
                    const int64_t *__restrict__ rp, const int32_t *__restrict__ cj, const double *__restrict__ lv,
                    const double *__restrict__ v, double *z, const GmresState *__restrict__ st) {
    if (st->done) return;
    for (int l = l0; l < l1; ++l) {
        const int p1 = off[l + 1];
        for (int p = off[l] + threadIdx.x; p < p1; p += ILU_RUN_THREADS) {
            const int r = rows[p];
            const double s = row_minus(v[r], rp[p], rp[p + 1], cj, lv, z);
            z[r] = s;
        }
        __syncthreads();
    }
}

// the backward sweep's run of narrow levels, as k_ilu_lower_run
__global__ void __launch_bounds__(ILU_RUN_THREADS)
    k_ilu_upper_run(const int32_t *__restrict__ rows, const int32_t *__restrict__ off, int l0, int l1,
                    const int64_t *__restrict__ rp, const int32_t *__restrict__ cj, const double *__restrict__ uv,
                    const double *__restrict__ dinv, double *z, const GmresState *__restrict__ st) {
    if (st->done) return;
    for (int l = l0; l < l1; ++l) {
        const int p1 = off[l + 1];
        for (int p = off[l] + threadIdx.x; p < p1; p += ILU_RUN_THREADS) {
            const int r = rows[p];
            const double s = row_minus(z[r], rp[p], rp[p + 1], cj, uv, z);
            z[r] = s * dinv[p];
        }
        __syncthreads();
    }
}

// The launches of one sweep: each level wider than ILU_WIDE_ROWS alone on a
// grid, the narrow levels between them in one-block runs.
std::vector<IluSeg> plan_sweep(const std::vector<int> &off) {
    std::vector<IluSeg> seg;
    const int nlev = (int)off.size() - 1;
    for (int l = 0; l < nlev;) {
        if (off[l + 1] - off[l] > ILU_WIDE_ROWS) {
            seg.push_back({l, l + 1, true});
            ++l;
            continue;
        }
        int e = l + 1;
        while (e < nlev && off[e + 1] - off[e] <= ILU_WIDE_ROWS) ++e;
        seg.push_back({l, e, false});
        l = e;
    }
    return seg;
}

// Host CSR of a stored matrix: columns sorted, duplicates merged (the ELL pads
// a row with zero-valued copies of its diagonal), dg = position of the diagonal.
struct HostCsr {
    std::vector<int64_t> rp, dg;
    std::vector<int32_t> cj;
    std::vector<double> v;
};

apcloud_status ell_to_csr(apcloud_ctx *c, const double *dval, HostCsr &A) {
    const int n = c->n_tot;
    const int ns = div_up(n, 32);
    std::vector<uint32_t> sw(ns), so(ns);
    APC_CUDA(c, cudaMemcpyAsync(sw.data(), c->slice_w.p, sizeof(uint32_t) * ns, cudaMemcpyDeviceToHost, c->s));
    APC_CUDA(c, cudaMemcpyAsync(so.data(), c->slice_off.p, sizeof(uint32_t) * ns, cudaMemcpyDeviceToHost, c->s));
    APC_CUDA(c, cudaStreamSynchronize(c->s));
    const int64_t ne = c->ell_entries;
    std::vector<int32_t> col(ne);
    std::vector<double> val(ne);
    APC_CUDA(c, cudaMemcpyAsync(col.data(), c->ell_col.p, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost, c->s));
    APC_CUDA(c, cudaMemcpyAsync(val.data(), dval, sizeof(double) * ne, cudaMemcpyDeviceToHost, c->s));
    APC_CUDA(c, cudaStreamSynchronize(c->s));
    A.rp.assign(n + 1, 0);
    A.dg.assign(n, -1);
    A.cj.clear();
    A.v.clear();
    std::vector<std::pair<int32_t, double>> row;
    for (int r = 0; r < n; ++r) {
        const int sl = r >> 5, lane = r & 31, w = (int)sw[sl];
        const int64_t base = (int64_t)so[sl] * 32 + lane;
        row.clear();
        for (int k = 0; k < w; ++k) row.emplace_back(col[base + (int64_t)k * 32], val[base + (int64_t)k * 32]);
        std::stable_sort(row.begin(), row.end(),
                         [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                             return a.first < b.first;
                         });
        for (size_t t = 0; t < row.size(); ++t) {
            if (!A.cj.empty() && (int64_t)A.cj.size() > A.rp[r] && A.cj.back() == row[t].first) {
                A.v.back() += row[t].second;
                continue;
            }
            if (row[t].first == r) A.dg[r] = (int64_t)A.cj.size();
            A.cj.push_back(row[t].first);
            A.v.push_back(row[t].second);
        }
        A.rp[r + 1] = (int64_t)A.cj.size();
        if (A.dg[r] < 0) return fail(c, APCLOUD_E_INVALID, "row %d of the stored matrix has no diagonal", r);
    }
    return APCLOUD_OK;
}

// level of every row: forward (a row after all rows k < r in its pattern) and
// backward (after all rows j > r); rows listed level by level, offsets per level
void levels(const HostCsr &A, bool lower, std::vector<int32_t> &rows, std::vector<int> &off) {
    const int64_t n = (int64_t)A.dg.size();
    std::vector<int> lev(n, 0);
    int nlev = 0;
    for (int64_t t = 0; t < n; ++t) {
        const int64_t i = lower ? t : n - 1 - t;
        int l = 0;
        for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
            const int64_t k = A.cj[e];
            if ((lower && k < i) || (!lower && k > i)) l = std::max(l, lev[k] + 1);
        }
        lev[i] = l;
        nlev = std::max(nlev, l + 1);
    }
    off.assign(nlev + 1, 0);
    for (int64_t i = 0; i < n; ++i) ++off[lev[i] + 1];
    for (int l = 0; l < nlev; ++l) off[l + 1] += off[l];
    rows.assign(n, 0);
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int64_t i = 0; i < n; ++i) rows[fill[lev[i]]++] = (int32_t)i;
}

}  // namespace

// ILU(0) in place on CSR values (columns sorted, the diagonal of row i at
// dg[i]); false on a zero pivot
bool ilu0_factor(int64_t n, const int64_t *rp, const int32_t *cj, const int64_t *dg, double *a) {
    std::vector<int64_t> iw(n, -1);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) iw[cj[e]] = e;
        bool ok = true;
        for (int64_t e = rp[i]; e < rp[i + 1] && cj[e] < i; ++e) {
            const int64_t k = cj[e];
            const double piv = a[dg[k]];
            if (piv == 0.0) { ok = false; break; }
            a[e] /= piv;
            const double lik = a[e];
            for (int64_t f = dg[k] + 1; f < rp[k + 1]; ++f) {   // entries (k, j), j > k
                const int64_t pos = iw[cj[f]];
                if (pos >= 0) a[pos] -= lik * a[f];
            }
        }
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) iw[cj[e]] = -1;
        if (!ok || a[dg[i]] == 0.0) return false;
    }
    return true;
}

// z = (LU)^-1 v: the forward levels, then the backward levels
double *ilu_apply(apcloud_ctx *c, const IluDev &I, const double *v, double *z, const GmresState *st) {
    for (const IluSeg &g : I.lseg) {
        if (g.wide) {
            const int p0 = I.loff[g.l0], p1 = I.loff[g.l1];
            APC_LAUNCH(c, K_SWEEP, div_up(p1 - p0, 128), 128, 0, k_ilu_lower, I.lrows, p0, p1, I.lrp, I.lcol, I.lval,
                       v, z, st);
        } else {
            APC_LAUNCH(c, K_SWEEP, 1, ILU_RUN_THREADS, 0, k_ilu_lower_run, I.lrows, I.dloff, g.l0, g.l1, I.lrp, I.lcol,
                       I.lval, v, z, st);
        }
    }
    for (const IluSeg &g : I.useg) {
        if (g.wide) {
            const int p0 = I.uoff[g.l0], p1 = I.uoff[g.l1];
            APC_LAUNCH(c, K_SWEEP, div_up(p1 - p0, 128), 128, 0, k_ilu_upper, I.urows, p0, p1, I.urp, I.ucol, I.uval,
                       I.udinv, z, st);
        } else {
            APC_LAUNCH(c, K_SWEEP, 1, ILU_RUN_THREADS, 0, k_ilu_upper_run, I.urows, I.duoff, g.l0, g.l1, I.urp, I.ucol,
                       I.uval, I.udinv, z, st);
        }
    }
    return z;
}

}  // namespace apc

using namespace apc;

apcloud_status apcloud_ilu0_factor_host(int64_t n, const int64_t *h_rowptr, const int32_t *h_col, double *h_val) {
    if (n < 0 || (n > 0 && (!h_rowptr || !h_col || !h_val))) return APCLOUD_E_INVALID;
    std::vector<int64_t> dg(n, -1);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = h_rowptr[i]; e < h_rowptr[i + 1]; ++e) {
            if (h_col[e] < 0 || h_col[e] >= n) return APCLOUD_E_INVALID;
            if (e > h_rowptr[i] && h_col[e] <= h_col[e - 1]) return APCLOUD_E_INVALID;   // sorted, no repeats
            if (h_col[e] == i) dg[i] = e;
        }
        if (dg[i] < 0) return APCLOUD_E_INVALID;
    }
    return ilu0_factor(n, h_rowptr, h_col, dg.data(), h_val) ? APCLOUD_OK : APCLOUD_E_NUMERIC;
}

apcloud_status apcloud_solve_system_ilu0(apcloud_ctx *c, int which, const double *b, double *x, double rtol,
                                         int max_iter, apcloud_solve_info *info, double *h_stats) {
    if (!c || !b || !x || (which != 0 && which != 1)) return APCLOUD_E_INVALID;
    if (c->stage < 2) return fail(c, APCLOUD_E_STATE, "matrices are available after apcloud_stencils");
    if (!(rtol > 0) || max_iter < 0) return fail(c, APCLOUD_E_INVALID, "rtol must be > 0 and max_iter >= 0");
    if (c->P.precision != 0) return fail(c, APCLOUD_E_INVALID, "the ILU(0) comparison runs in the FP64 form");
    if (c->nbeams > 1) return fail(c, APCLOUD_E_INVALID, "the ILU(0) comparison takes a single beam");
    const auto t0 = std::chrono::steady_clock::now();
    HostCsr A;
    APC_TRY(ell_to_csr(c, ptr<double>(which ? c->ell_A : c->ell_B), A));
    const int64_t n = (int64_t)A.dg.size();
    if (!ilu0_factor(n, A.rp.data(), A.cj.data(), A.dg.data(), A.v.data()))
        return fail(c, APCLOUD_E_NUMERIC, "ILU(0): zero pivot");
    IluDev &I = c->ilu;
    std::vector<int32_t> lrows, urows;
    levels(A, true, lrows, I.loff);
    levels(A, false, urows, I.uoff);
    // level-ordered strict lower and strict upper parts, and 1 / U_rr
    std::vector<int64_t> lrp(n + 1, 0), urp(n + 1, 0);
    std::vector<int32_t> lcol, ucol;
    std::vector<double> lval, uval, dinv(n);
    for (int64_t p = 0; p < n; ++p) {
        const int64_t i = lrows[p];
        for (int64_t e = A.rp[i]; e < A.dg[i]; ++e) { lcol.push_back(A.cj[e]); lval.push_back(A.v[e]); }
        lrp[p + 1] = (int64_t)lcol.size();
    }
    for (int64_t p = 0; p < n; ++p) {
        const int64_t i = urows[p];
        for (int64_t e = A.dg[i] + 1; e < A.rp[i + 1]; ++e) { ucol.push_back(A.cj[e]); uval.push_back(A.v[e]); }
        urp[p + 1] = (int64_t)ucol.size();
        dinv[p] = 1.0 / A.v[A.dg[i]];
    }
    const int64_t nl = std::max<int64_t>(1, (int64_t)lcol.size()), nu = std::max<int64_t>(1, (int64_t)ucol.size());
    int32_t *d_lrows = ensure<int32_t>(c, c->ilu_lrows, n), *d_urows = ensure<int32_t>(c, c->ilu_urows, n);
    int64_t *d_lrp = ensure<int64_t>(c, c->ilu_lrp, n + 1), *d_urp = ensure<int64_t>(c, c->ilu_urp, n + 1);
    int32_t *d_lcol = ensure<int32_t>(c, c->ilu_lcol, nl), *d_ucol = ensure<int32_t>(c, c->ilu_ucol, nu);
    double *d_lval = ensure<double>(c, c->ilu_lval, nl), *d_uval = ensure<double>(c, c->ilu_uval, nu);
    double *d_dinv = ensure<double>(c, c->ilu_dinv, n);
    int32_t *d_loff = ensure<int32_t>(c, c->ilu_loff, (int64_t)I.loff.size());
    int32_t *d_uoff = ensure<int32_t>(c, c->ilu_uoff, (int64_t)I.uoff.size());
    if (!d_lrows || !d_urows || !d_lrp || !d_urp || !d_lcol || !d_ucol || !d_lval || !d_uval || !d_dinv || !d_loff ||
        !d_uoff)
        return APCLOUD_E_NOMEM;
    APC_CUDA(c, cudaMemcpyAsync(d_lrows, lrows.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->s));
    APC_CUDA(c, cudaMemcpyAsync(d_urows, urows.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->s));
    APC_CUDA(c, cudaMemcpyAsync(d_lrp, lrp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->s));
    APC_CUDA(c, cudaMemcpyAsync(d_urp, urp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->s));
    if (!lcol.empty()) {
        APC_CUDA(c, cudaMemcpyAsync(d_lcol, lcol.data(), sizeof(int32_t) * lcol.size(), cudaMemcpyHostToDevice, c->s));
        APC_CUDA(c, cudaMemcpyAsync(d_lval, lval.data(), sizeof(double) * lval.size(), cudaMemcpyHostToDevice, c->s));
    }
    if (!ucol.empty()) {
        APC_CUDA(c, cudaMemcpyAsync(d_ucol, ucol.data(), sizeof(int32_t) * ucol.size(), cudaMemcpyHostToDevice, c->s));
        APC_CUDA(c, cudaMemcpyAsync(d_uval, uval.data(), sizeof(double) * uval.size(), cudaMemcpyHostToDevice, c->s));
    }
    APC_CUDA(c, cudaMemcpyAsync(d_dinv, dinv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->s));
    APC_CUDA(c, cudaMemcpyAsync(d_loff, I.loff.data(), sizeof(int32_t) * I.loff.size(), cudaMemcpyHostToDevice, c->s));
    APC_CUDA(c, cudaMemcpyAsync(d_uoff, I.uoff.data(), sizeof(int32_t) * I.uoff.size(), cudaMemcpyHostToDevice, c->s));
    APC_CUDA(c, cudaStreamSynchronize(c->s));   // the host vectors go out of scope
    I.lrows = d_lrows; I.urows = d_urows; I.lrp = d_lrp; I.urp = d_urp;
    I.lcol = d_lcol; I.ucol = d_ucol; I.lval = d_lval; I.uval = d_uval; I.udinv = d_dinv;
    I.dloff = d_loff; I.duoff = d_uoff;
    I.lseg = plan_sweep(I.loff);
    I.useg = plan_sweep(I.uoff);
    const double setup_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    c->ilu_which = which;
    apcloud_status st = gmres_solve(c, which, b, x, rtol, max_iter, info);
    c->ilu_which = -1;
    if (h_stats) {
        h_stats[0] = setup_ms;
        h_stats[1] = (double)(I.loff.size() - 1);
        h_stats[2] = (double)(I.uoff.size() - 1);
        h_stats[3] = (double)(A.cj.size());
    }
    return st;
}

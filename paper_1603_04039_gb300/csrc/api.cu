// api.cu -- the C ABI: context lifecycle, argument validation, call order,
// buffers, event timers and the entry points declared in apcloud.h.
#include <cmath>
#include <cstdarg>
#include <new>

#include "internal.cuh"

namespace apc {

apcloud_status fail(apcloud_ctx *c, apcloud_status st, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

apcloud_status cuda_check(apcloud_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return APCLOUD_OK;
    if (e == cudaErrorMemoryAllocation) return fail(c, APCLOUD_E_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(c, APCLOUD_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *raw_alloc(apcloud_ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (!c->default_alloc) return c->A.alloc(bytes, (void *)c->s, c->A.user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, c->s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void raw_free(apcloud_ctx *c, void *p) {
    if (!p) return;
    if (!c->default_alloc) c->A.free(p, (void *)c->s, c->A.user);
    else cudaFreeAsync(p, c->s);
}

bool ensure_bytes(apcloud_ctx *c, DBuf &b, size_t bytes, bool keep) {
    if (b.bytes >= bytes && b.p) return true;
    size_t nb = bytes + bytes / 4;
    void *p = raw_alloc(c, nb);
    if (!p) {
        fail(c, APCLOUD_E_NOMEM, "device allocation of %zu bytes failed", nb);
        return false;
    }
    if (keep && b.p && b.bytes) cudaMemcpyAsync(p, b.p, b.bytes, cudaMemcpyDeviceToDevice, c->s);
    raw_free(c, b.p);
    b.p = p;
    b.bytes = nb;
    return true;
}

static void free_buf(apcloud_ctx *c, DBuf &b) {
    raw_free(c, b.p);
    b.p = nullptr;
    b.bytes = 0;
}

void timer_close(apcloud_ctx *c) {
    Timer &t = c->timer;
    if (t.open < 0) return;
    cudaEventRecord(t.ev[t.open * 2 + 1], c->s);
    t.used++;
    t.open = -1;
}

void timer_begin(apcloud_ctx *c, int kind) {
    Timer &t = c->timer;
    // cycles are captured only with every timer off (event records cannot
    // sit in the conditional step bodies); timed cycles run as direct launches
    if (c->capturing) return;
    if (t.open >= 0 && (t.kind[t.open] != kind || !(t.mask >> kind & 1u))) timer_close(c);
    if (!(t.mask >> kind & 1u)) return;
    if (t.open >= 0) {   // the same kind again: the open pair covers this launch too
        t.nl[t.open]++;
        return;
    }
    if (t.used * 2 + 2 > t.ev.size()) {
        size_t old = t.ev.size();
        size_t nn = old ? old * 2 : 512;
        t.ev.resize(nn);
        for (size_t i = old; i < nn; ++i) cudaEventCreate(&t.ev[i]);
        t.kind.resize(nn / 2);
        t.nl.resize(nn / 2);
    }
    cudaEventRecord(t.ev[t.used * 2], c->s);
    t.kind[t.used] = kind;
    t.nl[t.used] = 1;
    t.open = (long)t.used;
}

static void timer_collect(apcloud_ctx *c) {
    Timer &t = c->timer;
    timer_close(c);
    if (!t.used) return;
    cudaStreamSynchronize(c->s);
    for (size_t i = 0; i < t.used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.ev[2 * i], t.ev[2 * i + 1]) == cudaSuccess) {
            t.ms[t.kind[i]] += ms;
            t.launches[t.kind[i]] += t.nl[i];
        }
    }
    t.used = 0;
}

// ---------------------------------------------------------------- CUDA graphs
static void destroy_entry(GraphEntry *g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
}

void free_graphs(apcloud_ctx *c) {
    for (GraphEntry *g : c->graphs) destroy_entry(g);
    c->graphs.clear();
    c->last_stepped = nullptr;
}

GraphEntry *find_graph(apcloud_ctx *c, const GraphKey &key) {
    for (GraphEntry *g : c->graphs)
        if (memcmp(&g->key, &key, sizeof key) == 0) return g;
    return nullptr;
}

GraphEntry *begin_capture(apcloud_ctx *c, const GraphKey &key) {
    for (cudaStream_t *ps : {&c->cap_stream, &c->body_stream}) {
        if (!*ps && cudaStreamCreateWithFlags(ps, cudaStreamNonBlocking) != cudaSuccess) {
            *ps = nullptr;
            cudaGetLastError();
            return nullptr;
        }
    }
    GraphEntry *g = new GraphEntry;
    g->key = key;
    // capture on the context's own capture stream (the caller's may be the legacy
    // default stream, which cannot be captured); replays run on the caller's stream
    std::swap(c->s, c->cap_stream);
    if (cudaStreamBeginCapture(c->s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        std::swap(c->s, c->cap_stream);
        cudaGetLastError();
        delete g;
        return nullptr;
    }
    // one condition per Arnoldi step, created on the graph being captured and
    // reset to 0 (skip) at every replay
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const int nstep = key.jmax > 0 ? key.jmax : 0;
    g->cond.assign(nstep, cudaGraphConditionalHandle{});
    g->step_kernels.assign(nstep, 0);
    if (cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &graph) != cudaSuccess || !graph) g->broken = true;
    for (int j = 1; j < nstep && !g->broken; ++j)
        if (cudaGraphConditionalHandleCreate(&g->cond[j], graph, 0, cudaGraphCondAssignDefault) != cudaSuccess)
            g->broken = true;
    c->capturing = g;
    return g;
}

void count_captured(apcloud_ctx *c) {
    GraphEntry *g = c->capturing;
    if (g->cur_step > 0) g->step_kernels[g->cur_step]++;
    else g->kernels++;
}

// IF node on cond[j] after everything captured so far; the launches that
// follow go to its body (captured on the body stream) until end_step
void begin_step(apcloud_ctx *c, int j) {
    GraphEntry *g = c->capturing;
    if (!g || j < 1 || j >= (int)g->cond.size() || g->broken) return;
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &graph, &deps, nullptr, &nd) != cudaSuccess || !graph) {
        g->broken = true;
        return;
    }
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = g->cond[j];
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, graph, deps, nullptr, nd, &p) != cudaSuccess ||
        cudaStreamUpdateCaptureDependencies(c->s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
            cudaSuccess ||
        cudaStreamBeginCaptureToGraph(c->body_stream, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        g->broken = true;
        return;
    }
    std::swap(c->s, c->body_stream);
    g->cur_step = j;
}

void end_step(apcloud_ctx *c) {
    GraphEntry *g = c->capturing;
    if (!g || g->cur_step < 1) return;
    cudaGraph_t body = nullptr;
    if (cudaStreamEndCapture(c->s, &body) != cudaSuccess) g->broken = true;
    std::swap(c->s, c->body_stream);
    g->cur_step = -1;
}

cudaGraphConditionalHandle next_step_cond(const apcloud_ctx *c, int j) {
    const GraphEntry *g = c->capturing;
    if (!g || j + 1 >= (int)g->cond.size()) return cudaGraphConditionalHandle{};
    return g->cond[j + 1];
}

void count_replayed_steps(apcloud_ctx *c, int je) {
    GraphEntry *g = c->last_stepped;
    c->last_stepped = nullptr;
    if (!g) return;
    for (int j = 1; j < je && j < (int)g->step_kernels.size(); ++j) c->launches += g->step_kernels[j];
}

GraphEntry *end_capture(apcloud_ctx *c, GraphEntry *g, apcloud_status st) {
    if (g->cur_step > 0) end_step(c);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->s, &graph);
    std::swap(c->s, c->cap_stream);
    c->capturing = nullptr;
    if (g->broken) e = cudaErrorStreamCaptureInvalidated;
    if (st >= 0 && e == cudaSuccess && graph) e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st < 0 || e != cudaSuccess || !g->exec) {
        cudaGetLastError();
        destroy_entry(g);
        c->err[0] = 0;
        return nullptr;
    }
    // keep the 8 most recently used cycles
    if (c->graphs.size() >= 8) {
        size_t old = 0;
        for (size_t i = 1; i < c->graphs.size(); ++i)
            if (c->graphs[i]->last_use < c->graphs[old]->last_use) old = i;
        if (c->last_stepped == c->graphs[old]) c->last_stepped = nullptr;
        destroy_entry(c->graphs[old]);
        c->graphs.erase(c->graphs.begin() + old);
    }
    c->graphs.push_back(g);
    return g;
}

apcloud_status launch_graph(apcloud_ctx *c, GraphEntry *g) {
    g->last_use = ++c->graph_clock;
    APC_CUDA(c, cudaGraphLaunch(g->exec, c->s));
    c->launches += g->kernels;
    c->last_stepped = g;
    c->graph_replays++;
    return APCLOUD_OK;
}


apcloud_status read_back(apcloud_ctx *c, void *host, const void *dev, size_t bytes) {
    timer_close(c);   // a timed pair must not span the host's wait
    c->host_syncs++;
    if (bytes > 256) {
        APC_CUDA(c, cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->s));
        return cuda_check(c, cudaStreamSynchronize(c->s), "synchronise");
    }
    APC_CUDA(c, cudaMemcpyAsync(c->h_pinned, dev, bytes, cudaMemcpyDeviceToHost, c->s));
    APC_CUDA(c, cudaStreamSynchronize(c->s));
    memcpy(host, c->h_pinned, bytes);
    return APCLOUD_OK;
}

apcloud_status check_device_errors(apcloud_ctx *c) {
    unsigned e[4];
    APC_TRY(read_back(c, e, c->derr.p, sizeof e));
    if (e[0] & ERR_DOMAIN) return fail(c, APCLOUD_E_DOMAIN, "a particle position is outside the domain or NaN");
    if (e[0] & ERR_OVERFLOW)
        return fail(c, APCLOUD_E_STENCIL, "a k-ring holds more than %d candidates", MAXC);
    if (e[0] & ERR_STENCIL)
        return fail(c, APCLOUD_E_STENCIL, "a node has no full-rank stencil within ring %d", c->P.ring_max);
    if (e[0] & ERR_BALANCE) return fail(c, APCLOUD_E_INVALID, "internal: 2:1 balance violated");
    if (e[0] & ERR_TIMEOUT) return fail(c, APCLOUD_E_TIMEOUT, "a kernel gave up waiting for its bulk copy");
    return APCLOUD_OK;
}

static apcloud_status validate(const apcloud_params *p, char *msg, size_t len) {
    double ext = p->hi[0] - p->lo[0];
    for (int d = 0; d < 3; ++d) {
        if (!std::isfinite(p->lo[d]) || !std::isfinite(p->hi[d]) || !(p->hi[d] > p->lo[d])) {
            snprintf(msg, len, "domain bounds must be finite with hi > lo");
            return APCLOUD_E_INVALID;
        }
        if (p->hi[d] - p->lo[d] != ext) {
            snprintf(msg, len, "domain must be a cube (equal extents)");
            return APCLOUD_E_INVALID;
        }
    }
    if (p->max_depth < 0 || p->max_depth > KEY_DEPTH) { snprintf(msg, len, "max_depth must be 0..21"); return APCLOUD_E_INVALID; }
    if (!(p->c_refine > 0) || !std::isfinite(p->c_refine)) { snprintf(msg, len, "c_refine must be > 0"); return APCLOUD_E_INVALID; }
    if (p->m_target < NCOL || p->m_target > MMAX) { snprintf(msg, len, "m_target must be 9..32"); return APCLOUD_E_INVALID; }
    if (p->ring_max < 2 || p->ring_max > 5) { snprintf(msg, len, "ring_max must be 2..5"); return APCLOUD_E_INVALID; }
    if (!(p->weight_c > 0) || !std::isfinite(p->weight_c)) { snprintf(msg, len, "weight_c must be > 0"); return APCLOUD_E_INVALID; }
    if (!std::isfinite(p->poisson_c)) { snprintf(msg, len, "poisson_c must be finite"); return APCLOUD_E_INVALID; }
    if (p->restart < 1 || p->restart > MAX_RESTART) { snprintf(msg, len, "restart must be 1..64"); return APCLOUD_E_INVALID; }
    if (p->poly_degree < 1 || p->poly_degree > 32) { snprintf(msg, len, "poly_degree must be 1..32"); return APCLOUD_E_INVALID; }
    if (!(p->poly_omega > 0 && p->poly_omega < 2)) { snprintf(msg, len, "poly_omega must be in (0, 2)"); return APCLOUD_E_INVALID; }
    if (p->stencil_slots < 16 || p->stencil_slots > MAXC_FAST) {
        snprintf(msg, len, "stencil_slots must be in [16, %d]", MAXC_FAST);
        return APCLOUD_E_INVALID;
    }
    if (!(p->fp32_rcond_min >= 0 && p->fp32_rcond_min <= 2)) {
        snprintf(msg, len, "fp32_rcond_min must be in [0, 2]");
        return APCLOUD_E_INVALID;
    }
    if (p->precision != 0 && p->precision != 1) {
        snprintf(msg, len, "precision must be 0 (FP64) or 1 (mixed)");
        return APCLOUD_E_INVALID;
    }
    return APCLOUD_OK;
}

}  // namespace apc

using namespace apc;

extern "C" {

void apcloud_default_params(apcloud_params *p) {
    if (!p) return;
    for (int d = 0; d < 3; ++d) { p->lo[d] = -1.0; p->hi[d] = 1.0; }
    p->max_depth = 6;
    p->c_refine = 1.0;
    p->m_target = 20;
    p->ring_max = 5;
    p->weight_c = 4.0;
    p->poisson_c = 1.0;
    p->restart = 30;
    p->precision = 0;
    p->poly_degree = 1;
    p->poly_omega = 0.7;
    p->fp32_rcond_min = 1e-3;
    p->stencil_slots = MAXC_FAST;
}

apcloud_status apcloud_create(const apcloud_params *params, const apcloud_allocator *alloc, void *stream,
                              apcloud_ctx **out) {
    if (!out) return APCLOUD_E_INVALID;
    *out = nullptr;
    if (!params) return APCLOUD_E_INVALID;
    char msg[256];
    apcloud_status st = validate(params, msg, sizeof msg);
    if (st != APCLOUD_OK) return st;
    if (alloc && (!alloc->alloc || !alloc->free)) return APCLOUD_E_INVALID;
    apcloud_ctx *c = new (std::nothrow) apcloud_ctx();
    if (!c) return APCLOUD_E_NOMEM;
    c->P = *params;
    if (alloc) { c->A = *alloc; c->default_alloc = false; }
    c->s = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return APCLOUD_E_CUDA;
    }
    if (cudaMallocHost(&c->h_pinned, 4096) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return APCLOUD_E_CUDA;
    }
    if (!ensure<unsigned>(c, c->derr, 4) || !ensure<uint32_t>(c, c->dsmall, 64) ||
        !ensure<GmresState>(c, c->gstate, 1)) {
        apcloud_destroy(c);
        return APCLOUD_E_NOMEM;
    }
    cudaMemsetAsync(c->derr.p, 0, 16, c->s);
    *out = c;
    return APCLOUD_OK;
}

void apcloud_destroy(apcloud_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->s);
    DBuf *bufs[] = {&c->key[0], &c->key[1], &c->val[0], &c->val[1], &c->ucell[0], &c->ucell[1], &c->ustart[0],
                    &c->ustart[1], &c->opened, &c->cand[0], &c->cand[1], &c->cval[0], &c->cval[1], &c->flags,
                    &c->scan, &c->scan_blk, &c->lkey, &c->lval, &c->leaf_anchor, &c->leaf_level, &c->leaf_first,
                    &c->leaf_count, &c->pleaf, &c->spos, &c->qsort, &c->node_ic, &c->bowner, &c->bface, &c->bidx, &c->adj, &c->nbr, &c->msz,
                    &c->ring, &c->lap, &c->lapd, &c->D, &c->rcond, &c->slice_w, &c->slice_off, &c->ell_col,
                    &c->ell_A, &c->ell_B, &c->dA, &c->dB, &c->V, &c->w0, &c->w1, &c->u, &c->b, &c->partial,
                    &c->gstate, &c->rho_m, &c->rho, &c->phi, &c->nodefield, &c->nodefield32, &c->tmp, &c->derr, &c->dsmall,
                    &c->hx, &c->hy, &c->hz, &c->hq, &c->hphi, &c->hex, &c->hey, &c->hez, &c->ell_A32,
                    &c->ell_B32, &c->V32, &c->w32a, &c->w32b, &c->r32, &c->e32, &c->gstate2,
                    &c->pz0, &c->pz1, &c->pt, &c->zbasis, &c->ell_rd, &c->ell_A16, &c->ell_B16, &c->beam_off, &c->leaf_beam,
                    &c->beam_rng, &c->beam_norm, &c->beam_r2, &c->beam_done, &c->node_beam, &c->tile_act,
                    &c->bk_items, &c->bk_ioff, &c->bk_d, &c->bk_i, &c->ss_perm, &c->ss_w, &c->ss_o, &c->ss_col, &c->ss_col24, &c->stencil_ovf,
                    &c->ss_A, &c->ss_B, &c->ss_A32, &c->ss_B32, &c->tune_b, &c->tune_x, &c->beam_part, &c->ilu_lrows, &c->ilu_urows, &c->ilu_lrp, &c->ilu_urp,
                    &c->ilu_lcol, &c->ilu_ucol, &c->ilu_lval, &c->ilu_uval, &c->ilu_dinv,
                    &c->ilu_loff, &c->ilu_uoff};
    for (DBuf *b : bufs) free_buf(c, *b);
    for (DBuf &b : c->mp) free_buf(c, b);
    cudaStreamSynchronize(c->s);
    free_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->body_stream) cudaStreamDestroy(c->body_stream);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->copy_done) cudaEventDestroy(c->copy_done);
    for (cudaEvent_t e : c->timer.ev) cudaEventDestroy(e);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
}

const char *apcloud_last_error(const apcloud_ctx *c) { return c ? c->err : "null context"; }

apcloud_status apcloud_build_octree(apcloud_ctx *c, const double *x, const double *y, const double *z, int64_t n,
                                    int64_t *n_interior, int64_t *n_boundary) {
    if (!c) return APCLOUD_E_INVALID;
    if (n < 0 || n > 2000000000LL) return fail(c, APCLOUD_E_INVALID, "particle count %lld out of range", (long long)n);
    if (n > 0 && (!x || !y || !z)) return fail(c, APCLOUD_E_INVALID, "null position array");
    c->stage = 0;
    const int64_t off[2] = {0, n};
    apcloud_status st = build_octree(c, x, y, z, n, off, 1);
    if (st < 0) return st;
    c->stage = 1;
    if (n_interior) *n_interior = c->n_int;
    if (n_boundary) *n_boundary = c->n_bnd;
    return APCLOUD_OK;
}

apcloud_status apcloud_build_octree_batched(apcloud_ctx *c, const double *x, const double *y, const double *z,
                                            const int64_t *offsets, int n_beams, int64_t *n_interior,
                                            int64_t *n_boundary) {
    if (!c) return APCLOUD_E_INVALID;
    if (n_beams < 1 || n_beams > APCLOUD_MAX_BEAMS || !offsets)
        return fail(c, APCLOUD_E_INVALID, "n_beams must be in 1..%d with an offsets array", APCLOUD_MAX_BEAMS);
    if (offsets[0] != 0) return fail(c, APCLOUD_E_INVALID, "offsets[0] must be 0");
    for (int b = 0; b < n_beams; ++b)
        if (offsets[b + 1] < offsets[b]) return fail(c, APCLOUD_E_INVALID, "offsets must not decrease (beam %d)", b);
    const int64_t n = offsets[n_beams];
    if (n > 2000000000LL) return fail(c, APCLOUD_E_INVALID, "particle count %lld out of range", (long long)n);
    if (n > 0 && (!x || !y || !z)) return fail(c, APCLOUD_E_INVALID, "null position array");
    c->stage = 0;
    apcloud_status st = build_octree(c, x, y, z, n, offsets, n_beams);
    if (st < 0) return st;
    c->stage = 1;
    if (n_interior) *n_interior = c->n_int;
    if (n_boundary) *n_boundary = c->n_bnd;
    return APCLOUD_OK;
}

apcloud_status apcloud_get_node_beams(apcloud_ctx *c, int32_t *beam) {
    if (!c || !beam) return APCLOUD_E_INVALID;
    if (c->stage < 1) return fail(c, APCLOUD_E_STATE, "node beams are available after apcloud_build_octree");
    APC_TRY(node_beams(c, beam));
    return cuda_check(c, cudaStreamSynchronize(c->s), "get_node_beams");
}

apcloud_status apcloud_get_nodes(apcloud_ctx *c, double *xyz, int8_t *level, int8_t *kind);
apcloud_status apcloud_get_leaves(apcloud_ctx *c, uint64_t *key, int32_t *first, int32_t *count);

apcloud_status apcloud_stencils(apcloud_ctx *c) {
    if (!c) return APCLOUD_E_INVALID;
    if (c->stage < 1) return fail(c, APCLOUD_E_STATE, "apcloud_stencils before apcloud_build_octree");
    c->mp_graph_n = -1;   // the learned preconditioner's graph belongs to the old matrix
    apcloud_status st = build_stencils(c);
    if (st < 0) { c->stage = 1; return st; }
    c->stage = 2;
    return APCLOUD_OK;
}

apcloud_status apcloud_deposit(apcloud_ctx *c, const double *q, double q_uniform, double rtol, int max_iter,
                               double *rho_out, apcloud_solve_info *info) {
    if (!c) return APCLOUD_E_INVALID;
    if (c->stage < 2) return fail(c, APCLOUD_E_STATE, "apcloud_deposit before apcloud_stencils");
    if (!(rtol > 0) || max_iter < 0) return fail(c, APCLOUD_E_INVALID, "rtol must be > 0 and max_iter >= 0");
    if (!q && !std::isfinite(q_uniform)) return fail(c, APCLOUD_E_INVALID, "q_uniform must be finite");
    APC_TRY(deposit(c, q, q_uniform));
    double *rho = ensure<double>(c, c->rho, c->n_tot + 1);
    if (!rho) return APCLOUD_E_NOMEM;
    APC_CUDA(c, cudaMemsetAsync(rho, 0, sizeof(double) * c->n_tot, c->s));
    apcloud_status st = gmres_solve(c, 0, ptr<double>(c->rho_m), rho, rtol, max_iter, info);
    if (st < 0) return st;
    if (rho_out) APC_CUDA(c, cudaMemcpyAsync(rho_out, rho, sizeof(double) * c->n_tot, cudaMemcpyDeviceToDevice, c->s));
    c->stage = 3;
    return st;
}

apcloud_status apcloud_get_rho_m(apcloud_ctx *c, double *d) {
    if (!c || !d) return APCLOUD_E_INVALID;
    if (c->stage < 3) return fail(c, APCLOUD_E_STATE, "rho_M is available after apcloud_deposit");
    APC_CUDA(c, cudaMemcpyAsync(d, c->rho_m.p, sizeof(double) * c->n_tot, cudaMemcpyDeviceToDevice, c->s));
    return cuda_check(c, cudaStreamSynchronize(c->s), "get_rho_m");
}

}  // extern "C"

namespace apc {
namespace {
__global__ void k_poisson_rhs(const double *__restrict__ rho, const double *__restrict__ g, int n_int, int n_tot,
                              double cp, double *__restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tot) return;
    b[i] = (i < n_int) ? cp * rho[i] : (g ? g[i - n_int] : 0.0);
}
__global__ void k_nodes_out(const int4 *__restrict__ ic, int n_int, int n_tot, double lo0, double lo1, double lo2,
                            double unit, double *__restrict__ xyz, int8_t *__restrict__ level,
                            int8_t *__restrict__ kind) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tot) return;
    int4 q = ic[i];
    if (xyz) {
        xyz[3 * i + 0] = __dadd_rn(lo0, __dmul_rn((double)q.x, unit));
        xyz[3 * i + 1] = __dadd_rn(lo1, __dmul_rn((double)q.y, unit));
        xyz[3 * i + 2] = __dadd_rn(lo2, __dmul_rn((double)q.z, unit));
    }
    if (level) level[i] = (int8_t)q.w;
    if (kind) kind[i] = (int8_t)(i >= n_int);
}
__global__ void k_leaves_out(const uint64_t *__restrict__ anchor, const int8_t *__restrict__ lev, int n, int L,
                             const int32_t *__restrict__ f, const int32_t *__restrict__ cnt, uint64_t *__restrict__ key,
                             int32_t *__restrict__ first, int32_t *__restrict__ count) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (key) key[j] = anchor[j] >> (3 * (L - lev[j]));
    if (first) first[j] = f[j];
    if (count) count[j] = cnt[j];
}
__global__ void k_stencils_out(const double *__restrict__ D, int64_t dstride, int n, double *__restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * NCOL * MMAX) return;
    int64_t j = t / (NCOL * MMAX);
    int ri = (int)(t % (NCOL * MMAX));
    out[t] = D[(int64_t)ri * dstride + j];
}
__global__ void k_scale_in(const double *__restrict__ x, const double *__restrict__ d, int n, double *__restrict__ o) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = x[i] * d[i];
}
__global__ void k_copy_nf(const double *__restrict__ nf, int n, double *__restrict__ o) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * NCOL) return;
    int64_t j = t / NCOL;
    int r = (int)(t % NCOL);
    o[t] = nf[j * 12 + 1 + r];
}
}  // namespace

double *poisson_rhs(apcloud_ctx *c, const double *g) {
    double *b = ensure<double>(c, c->b, c->n_tot + 1);
    if (!b) return nullptr;
    APC_LAUNCH(c, K_VEC, div_up(c->n_tot, 256), 256, 0, k_poisson_rhs, ptr<double>(c->rho), g, c->n_int, c->n_tot,
               c->P.poisson_c, b);
    return b;
}

}  // namespace apc

extern "C" {

apcloud_status apcloud_get_nodes(apcloud_ctx *c, double *xyz, int8_t *level, int8_t *kind) {
    if (!c) return APCLOUD_E_INVALID;
    if (c->stage < 1) return fail(c, APCLOUD_E_STATE, "nodes are available after apcloud_build_octree");
    double unit = ldexp(c->P.hi[0] - c->P.lo[0], -(KEY_DEPTH + 1));
    APC_LAUNCH(c, K_COPY, div_up(c->n_tot, 256), 256, 0, k_nodes_out, ptr<int4>(c->node_ic), c->n_int, c->n_tot,
               c->P.lo[0], c->P.lo[1], c->P.lo[2], unit, xyz, level, kind);
    return cuda_check(c, cudaStreamSynchronize(c->s), "get_nodes");
}

apcloud_status apcloud_get_leaves(apcloud_ctx *c, uint64_t *key, int32_t *first, int32_t *count) {
    if (!c) return APCLOUD_E_INVALID;
    if (c->stage < 1) return fail(c, APCLOUD_E_STATE, "leaves are available after apcloud_build_octree");
    APC_LAUNCH(c, K_COPY, div_up(c->n_int, 256), 256, 0, k_leaves_out, ptr<uint64_t>(c->leaf_anchor),
               ptr<int8_t>(c->leaf_level), c->n_int, c->L, ptr<int32_t>(c->leaf_first), ptr<int32_t>(c->leaf_count),
               key, first, count);
    return cuda_check(c, cudaStreamSynchronize(c->s), "get_leaves");
}

apcloud_status apcloud_get_stencils(apcloud_ctx *c, int32_t *nbr, int32_t *m, double *lap, double *lapd, double *D) {
    if (!c) return APCLOUD_E_INVALID;
    if (c->stage < 2) return fail(c, APCLOUD_E_STATE, "stencils are available after apcloud_stencils");
    size_t n = (size_t)c->n_int;
    if (nbr) APC_CUDA(c, cudaMemcpyAsync(nbr, c->nbr.p, n * MMAX * 4, cudaMemcpyDeviceToDevice, c->s));
    if (m) APC_CUDA(c, cudaMemcpyAsync(m, c->msz.p, n * 4, cudaMemcpyDeviceToDevice, c->s));
    if (lap) APC_CUDA(c, cudaMemcpyAsync(lap, c->lap.p, n * MMAX * 8, cudaMemcpyDeviceToDevice, c->s));
    if (lapd) APC_CUDA(c, cudaMemcpyAsync(lapd, c->lapd.p, n * 8, cudaMemcpyDeviceToDevice, c->s));
    if (D) {
        int64_t dstride = ((int64_t)n + 31) / 32 * 32;
        APC_LAUNCH(c, K_COPY, div_up((int64_t)n * NCOL * MMAX, 256), 256, 0, k_stencils_out, ptr<double>(c->D),
                   dstride, (int)n, D);
    }
    return cuda_check(c, cudaStreamSynchronize(c->s), "get_stencils");
}

apcloud_status apcloud_solve(apcloud_ctx *c, const double *g, const double *phi0, double rtol, int max_iter,
                             double *phi_out, apcloud_solve_info *info) {
    if (!c) return APCLOUD_E_INVALID;
    if (c->stage < 3) return fail(c, APCLOUD_E_STATE, "apcloud_solve before apcloud_deposit");
    if (!(rtol > 0) || max_iter < 0) return fail(c, APCLOUD_E_INVALID, "rtol must be > 0 and max_iter >= 0");
    double *b = ensure<double>(c, c->b, c->n_tot + 1);
    double *phi = ensure<double>(c, c->phi, c->n_tot + 1);
    if (!b || !phi) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_VEC, div_up(c->n_tot, 256), 256, 0, k_poisson_rhs, ptr<double>(c->rho), g, c->n_int, c->n_tot,
               c->P.poisson_c, b);
    if (phi0) APC_CUDA(c, cudaMemcpyAsync(phi, phi0, sizeof(double) * c->n_tot, cudaMemcpyDeviceToDevice, c->s));
    else APC_CUDA(c, cudaMemsetAsync(phi, 0, sizeof(double) * c->n_tot, c->s));
    apcloud_status st = gmres_solve(c, 1, b, phi, rtol, max_iter, info);
    if (st < 0) return st;
    if (phi_out) APC_CUDA(c, cudaMemcpyAsync(phi_out, phi, sizeof(double) * c->n_tot, cudaMemcpyDeviceToDevice, c->s));
    c->stage = 4;
    return st;
}

apcloud_status apcloud_gather_field(apcloud_ctx *c, double *phi_p, double *ex, double *ey, double *ez) {
    if (!c) return APCLOUD_E_INVALID;
    if (c->stage < 4) return fail(c, APCLOUD_E_STATE, "apcloud_gather_field before apcloud_solve");
    APC_TRY(gather_field(c, phi_p, ex, ey, ez));
    c->stage = 5;
    return APCLOUD_OK;
}

apcloud_status apcloud_get_derivatives(apcloud_ctx *c, double *d) {
    if (!c || !d) return APCLOUD_E_INVALID;
    if (c->stage < 5) return fail(c, APCLOUD_E_STATE, "derivatives are available after apcloud_gather_field");
    APC_LAUNCH(c, K_COPY, div_up((int64_t)c->n_int * NCOL, 256), 256, 0, k_copy_nf, ptr<double>(c->nodefield),
               c->n_int, d);
    return cuda_check(c, cudaStreamSynchronize(c->s), "get_derivatives");
}

apcloud_status apcloud_matvec(apcloud_ctx *c, int which, const double *x, double *y) {
    if (!c || !x || !y || (which != 0 && which != 1)) return APCLOUD_E_INVALID;
    if (c->stage < 2) return fail(c, APCLOUD_E_STATE, "matrices are available after apcloud_stencils");
    double *t = ensure<double>(c, c->w0, c->n_tot + 1);
    if (!t) return APCLOUD_E_NOMEM;
    APC_LAUNCH(c, K_VEC, div_up(c->n_tot, 256), 256, 0, k_scale_in, x, ptr<double>(which ? c->dA : c->dB), c->n_tot, t);
    APC_TRY(spmv(c, which, t, y, 1.0, nullptr));
    return cuda_check(c, cudaGetLastError(), "matvec");
}

apcloud_status apcloud_solve_system(apcloud_ctx *c, int which, const double *b, double *x, double rtol, int max_iter,
                                    apcloud_solve_info *info) {
    if (!c || !b || !x || (which != 0 && which != 1)) return APCLOUD_E_INVALID;
    if (c->stage < 2) return fail(c, APCLOUD_E_STATE, "matrices are available after apcloud_stencils");
    if (!(rtol > 0) || max_iter < 0) return fail(c, APCLOUD_E_INVALID, "rtol must be > 0 and max_iter >= 0");
    return gmres_solve(c, which, b, x, rtol, max_iter, info);
}

static apcloud_status field_host_run(apcloud_ctx *c, const double *hx, const double *hy, const double *hz,
                                     const double *hq, double q_uniform, int64_t n, const int64_t *offsets,
                                     int nbeams, double rtol, int max_iter, double *hphi, double *hex, double *hey,
                                     double *hez, apcloud_solve_info *ir, apcloud_solve_info *ip) {
    if (n < 0 || (n > 0 && (!hx || !hy || !hz))) return fail(c, APCLOUD_E_INVALID, "bad host particle arrays");
    size_t nb = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *dx = ensure<double>(c, c->hx, n + 1), *dy = ensure<double>(c, c->hy, n + 1),
           *dz = ensure<double>(c, c->hz, n + 1);
    double *dq = hq ? ensure<double>(c, c->hq, n + 1) : nullptr;
    double *dp = ensure<double>(c, c->hphi, n + 1), *de0 = ensure<double>(c, c->hex, n + 1),
           *de1 = ensure<double>(c, c->hey, n + 1), *de2 = ensure<double>(c, c->hez, n + 1);
    if (!dx || !dy || !dz || (hq && !dq) || !dp || !de0 || !de1 || !de2) return APCLOUD_E_NOMEM;
    // the charges are not needed before the deposit: their copy runs on a
    // second stream while the tree and the stencils are built
    bool q_side = false;
    if (n > 0) {
        APC_CUDA(c, cudaMemcpyAsync(dx, hx, nb, cudaMemcpyHostToDevice, c->s));
        APC_CUDA(c, cudaMemcpyAsync(dy, hy, nb, cudaMemcpyHostToDevice, c->s));
        APC_CUDA(c, cudaMemcpyAsync(dz, hz, nb, cudaMemcpyHostToDevice, c->s));
        if (hq) {
            if (!c->copy_stream) {
                if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&c->copy_done, cudaEventDisableTiming) != cudaSuccess) {
                    cudaGetLastError();
                    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
                    c->copy_stream = nullptr;
                }
            }
            if (c->copy_stream) {
                // the device buffer may still be read by earlier work on the context stream
                APC_CUDA(c, cudaEventRecord(c->copy_done, c->s));
                APC_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->copy_done, 0));
                APC_CUDA(c, cudaMemcpyAsync(dq, hq, nb, cudaMemcpyHostToDevice, c->copy_stream));
                APC_CUDA(c, cudaEventRecord(c->copy_done, c->copy_stream));
                q_side = true;
            } else {
                APC_CUDA(c, cudaMemcpyAsync(dq, hq, nb, cudaMemcpyHostToDevice, c->s));
            }
        }
    }
    int64_t ni, nbd;
    apcloud_status sb;
    if (offsets) sb = apcloud_build_octree_batched(c, dx, dy, dz, offsets, nbeams, &ni, &nbd);
    else sb = apcloud_build_octree(c, dx, dy, dz, n, &ni, &nbd);
    if (sb == APCLOUD_OK) sb = apcloud_stencils(c);
    if (q_side) {
        // joined on every path, so that no copy into dq is left running
        cudaError_t e = cudaStreamWaitEvent(c->s, c->copy_done, 0);
        if (sb == APCLOUD_OK && e != cudaSuccess) sb = cuda_check(c, e, "charge copy");
    }
    APC_TRY(sb);
    apcloud_status s1 = apcloud_deposit(c, dq, q_uniform, rtol, max_iter, nullptr, ir);
    if (s1 < 0) return s1;
    apcloud_status s2 = apcloud_solve(c, nullptr, nullptr, rtol, max_iter, nullptr, ip);
    if (s2 < 0) return s2;
    APC_TRY(apcloud_gather_field(c, dp, de0, de1, de2));
    if (n > 0) {
        if (hphi) APC_CUDA(c, cudaMemcpyAsync(hphi, dp, nb, cudaMemcpyDeviceToHost, c->s));
        if (hex) APC_CUDA(c, cudaMemcpyAsync(hex, de0, nb, cudaMemcpyDeviceToHost, c->s));
        if (hey) APC_CUDA(c, cudaMemcpyAsync(hey, de1, nb, cudaMemcpyDeviceToHost, c->s));
        if (hez) APC_CUDA(c, cudaMemcpyAsync(hez, de2, nb, cudaMemcpyDeviceToHost, c->s));
    }
    APC_CUDA(c, cudaStreamSynchronize(c->s));
    return (s1 > 0 || s2 > 0) ? APCLOUD_W_NOT_CONVERGED : APCLOUD_OK;
}

// every return leaves no copy from or to the caller's host arrays in flight
static apcloud_status field_host(apcloud_ctx *c, const double *hx, const double *hy, const double *hz,
                                 const double *hq, double q_uniform, int64_t n, const int64_t *offsets, int nbeams,
                                 double rtol, int max_iter, double *hphi, double *hex, double *hey, double *hez,
                                 apcloud_solve_info *ir, apcloud_solve_info *ip) {
    if (!c) return APCLOUD_E_INVALID;
    const apcloud_status st = field_host_run(c, hx, hy, hz, hq, q_uniform, n, offsets, nbeams, rtol, max_iter, hphi,
                                             hex, hey, hez, ir, ip);
    if (st < 0) {
        cudaStreamSynchronize(c->s);
        if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
        cudaGetLastError();
    }
    return st;
}

apcloud_status apcloud_field_host(apcloud_ctx *c, const double *hx, const double *hy, const double *hz,
                                  const double *hq, double q_uniform, int64_t n, double rtol, int max_iter,
                                  double *hphi, double *hex, double *hey, double *hez, apcloud_solve_info *ir,
                                  apcloud_solve_info *ip) {
    return field_host(c, hx, hy, hz, hq, q_uniform, n, nullptr, 1, rtol, max_iter, hphi, hex, hey, hez, ir, ip);
}

apcloud_status apcloud_field_host_batched(apcloud_ctx *c, const double *hx, const double *hy, const double *hz,
                                          const double *hq, double q_uniform, const int64_t *offsets, int n_beams,
                                          double rtol, int max_iter, double *hphi, double *hex, double *hey,
                                          double *hez, apcloud_solve_info *ir, apcloud_solve_info *ip) {
    if (!c) return APCLOUD_E_INVALID;
    if (!offsets || n_beams < 1) return fail(c, APCLOUD_E_INVALID, "a batch needs n_beams >= 1 and offsets");
    return field_host(c, hx, hy, hz, hq, q_uniform, offsets[n_beams], offsets, n_beams, rtol, max_iter, hphi, hex,
                      hey, hez, ir, ip);
}

apcloud_status apcloud_interpolate_potential(apcloud_ctx *c, const double *x, const double *y, const double *z,
                                             int64_t n, double *phi) {
    if (!c || n < 0 || (n > 0 && (!x || !y || !z || !phi))) return APCLOUD_E_INVALID;
    if (c->stage < 5) return fail(c, APCLOUD_E_STATE, "interpolation needs apcloud_gather_field first");
    if (c->nbeams > 1) return fail(c, APCLOUD_E_INVALID, "interpolation needs a single-beam context");
    if (n == 0) return APCLOUD_OK;
    return interpolate_phi(c, x, y, z, n, phi);
}

apcloud_status apcloud_push_particles(apcloud_ctx *c, double *x, double *y, double *z, double *vx, double *vy,
                                      double *vz, int64_t n, const double *ex, const double *ey, const double *ez,
                                      double qm_dt, double dt) {
    if (!c || n < 0 || (n > 0 && (!x || !y || !z || !vx || !vy || !vz))) return APCLOUD_E_INVALID;
    if ((ex || ey || ez) && !(ex && ey && ez)) return fail(c, APCLOUD_E_INVALID, "field components: all or none");
    if (!std::isfinite(qm_dt) || !std::isfinite(dt)) return fail(c, APCLOUD_E_INVALID, "non-finite step");
    if (n == 0) return APCLOUD_OK;
    return push(c, x, y, z, vx, vy, vz, n, ex, ey, ez, qm_dt, dt);
}

apcloud_status apcloud_field_energy(apcloud_ctx *c, double *h_energy) {
    if (!c || !h_energy) return APCLOUD_E_INVALID;
    if (c->stage < 5) return fail(c, APCLOUD_E_STATE, "field energy needs apcloud_gather_field first");
    return field_energy(c, h_energy);
}

apcloud_status apcloud_set_timing(apcloud_ctx *c, unsigned mask) {
    if (!c) return APCLOUD_E_INVALID;
    timer_collect(c);
    c->timer.mask = mask;
    return APCLOUD_OK;
}

apcloud_status apcloud_get_timing(apcloud_ctx *c, double *ms, int64_t *launches, double *bytes, double *flops,
                                  int reset) {
    if (!c) return APCLOUD_E_INVALID;
    timer_collect(c);
    for (int k = 0; k < NKIND; ++k) {
        if (ms) ms[k] = c->timer.ms[k];
        if (launches) launches[k] = c->timer.launches[k];
        if (bytes) bytes[k] = c->timer.bytes[k];
        if (flops) flops[k] = c->timer.flops[k];
        if (reset) { c->timer.ms[k] = 0; c->timer.launches[k] = 0; c->timer.bytes[k] = 0; c->timer.flops[k] = 0; }
    }
    return APCLOUD_OK;
}

const char *apcloud_kernel_name(int kind) {
    static const char *names[NKIND] = {"morton_keys", "radix_sort", "tree", "face_adjacency", "ring_select_wls",
                                       "assemble_ell", "deposit", "spmv", "gmres_dots", "gmres_update_dots",
                                       "gmres_update_norm", "gmres_cycle_end", "derivatives", "gather",
                                       "vector", "copy", "mpnn_dense_tc", "mpnn_graph", "precond_sweep"};
    return (kind >= 0 && kind < NKIND) ? names[kind] : "unknown";
}

int64_t apcloud_launch_count(const apcloud_ctx *c) { return c ? c->launches : 0; }

int64_t apcloud_host_sync_count(const apcloud_ctx *c) { return c ? c->host_syncs : 0; }

apcloud_status apcloud_autotune(apcloud_ctx *c, unsigned what, int *spmv_block, int *spmv_unroll,
                                int *sweep_sorted, int *wls_warps, double *ms) {
    if (!c) return APCLOUD_E_INVALID;
    if (c->stage < 2) return fail(c, APCLOUD_E_STATE, "apcloud_autotune needs apcloud_stencils first");
    if (ms)
        for (int i = 0; i < 19; ++i) ms[i] = 0.0;
    if (what & 1u) APC_TRY(tune_spmv(c, ms));
    if (what & 2u) APC_TRY(tune_stencils(c, ms ? ms + 16 : nullptr));
    if (spmv_block) *spmv_block = c->spmv_bs;
    if (spmv_unroll) *spmv_unroll = c->spmv_unroll;
    if (sweep_sorted) *sweep_sorted = c->sweep_sorted;
    if (wls_warps) *wls_warps = c->wls_warps;
    return APCLOUD_OK;
}

apcloud_status apcloud_set_launch_shape(apcloud_ctx *c, int spmv_block, int spmv_unroll, int sweep_sorted,
                                        int wls_warps) {
    if (!c) return APCLOUD_E_INVALID;
    if (spmv_block != 64 && spmv_block != 128 && spmv_block != 256 && spmv_block != 512)
        return fail(c, APCLOUD_E_INVALID, "spmv_block must be 64, 128, 256 or 512");
    if (spmv_unroll != 1 && spmv_unroll != 4) return fail(c, APCLOUD_E_INVALID, "spmv_unroll must be 1 or 4");
    if (sweep_sorted != 0 && sweep_sorted != 1) return fail(c, APCLOUD_E_INVALID, "sweep_sorted must be 0 or 1");
    if (wls_warps != 2 && wls_warps != 4 && wls_warps != 8)
        return fail(c, APCLOUD_E_INVALID, "wls_warps must be 2, 4 or 8");
    c->spmv_bs = spmv_block;
    c->spmv_unroll = spmv_unroll;
    c->sweep_sorted = sweep_sorted;
    c->wls_warps = wls_warps;
    return APCLOUD_OK;
}

apcloud_status apcloud_set_sweep_l2_keep(apcloud_ctx *c, int64_t keep_bytes) {
    if (!c) return APCLOUD_E_INVALID;
    if (keep_bytes < -1) return fail(c, APCLOUD_E_INVALID, "keep_bytes must be -1 (automatic) or >= 0");
    c->sweep_keep = keep_bytes;
    return APCLOUD_OK;
}

apcloud_status apcloud_get_sweep_l2_keep(const apcloud_ctx *c, int64_t *h_keep_bytes) {
    if (!c || !h_keep_bytes) return APCLOUD_E_INVALID;
    *h_keep_bytes = sweep_keep_bytes(c);
    return APCLOUD_OK;
}

apcloud_status apcloud_set_dependent_launch(apcloud_ctx *c, int enable) {
    if (!c) return APCLOUD_E_INVALID;
    c->pdl_on = enable != 0;
    return APCLOUD_OK;
}

apcloud_status apcloud_set_graphs(apcloud_ctx *c, int enable) {
    if (!c) return APCLOUD_E_INVALID;
    cudaStreamSynchronize(c->s);
    c->graphs_on = enable != 0;
    if (!c->graphs_on) free_graphs(c);
    return APCLOUD_OK;
}

apcloud_status apcloud_graph_stats(const apcloud_ctx *c, int64_t *replays, int64_t *cached) {
    if (!c) return APCLOUD_E_INVALID;
    if (replays) *replays = c->graph_replays;
    if (cached) *cached = (int64_t)c->graphs.size();
    return APCLOUD_OK;
}

apcloud_status apcloud_get_sizes(const apcloud_ctx *c, int64_t *h) {
    if (!c || !h) return APCLOUD_E_INVALID;
    h[0] = c->N;
    h[1] = c->n_int;
    h[2] = c->n_bnd;
    h[3] = c->sum_m + c->n_int + c->n_bnd;
    h[4] = c->ell_entries;
    h[5] = c->sum_m;
    h[6] = c->n_slices;
    h[7] = c->L;
    h[8] = c->n_fp64_wls;
    return APCLOUD_OK;
}

}  // extern "C"

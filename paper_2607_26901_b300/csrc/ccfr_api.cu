// C ABI of the CCFR library: context set-up, argument checks, launch
// orchestration and CUDA-graph capture of the substep.  See include/ccfr.h.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ccfr.h"
#include "ccfr_internal.h"

using namespace ccfr;

namespace {

struct GraphEntry {
    float* x;
    float* v;
    cudaGraphExec_t exec;
};

// Constraints beyond the collision edges (ccfr_create_ext), on the host.
struct Extras {
    std::vector<int> links;         // 2 per link
    std::vector<float> link_comp;   // per link
    std::vector<int> tets;          // 4 per tetrahedron
    float vol_comp = 0.f;
};

}  // namespace

struct ccfr_ctx {
    int device = 0;
    ccfr_params prm{};
    DevCtx dc{};
    int n_buckets_total = 0;
    unsigned* tile_sums = nullptr;
    std::vector<int> color_off;
    int n_colors = 0;
    std::vector<int> tcolor_off;    // colours of the tetrahedra
    int n_tcolors = 0;
    cudaStream_t cap_stream = nullptr;
    SideStream side;
    std::vector<GraphEntry> graphs;
    bool regions_valid = false;
    bool rest_pending = false;
    float4* hx = nullptr;
    float4* hv = nullptr;
    unsigned long long* pair_count = nullptr;
    std::vector<void*> allocs;
    int n_scenes = 1;
    unsigned char* active = nullptr;   // per-scene step mask of a batched context (all 1 between calls)
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

template <typename T>
cudaError_t dalloc(ccfr_ctx* c, T** p, size_t count) {
    *p = nullptr;
    size_t bytes = (count > 0 ? count : 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e == cudaSuccess) c->allocs.push_back((void*)*p);
    return e;
}

void free_ctx(ccfr_ctx* c) {
    if (!c) return;
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    for (void* p : c->allocs) cudaFree(p);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side.s) cudaStreamDestroy(c->side.s);
    if (c->side.fork) cudaEventDestroy(c->side.fork);
    if (c->side.join) cudaEventDestroy(c->side.join);
    delete c;
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

unsigned next_pow2(unsigned v) {
    unsigned p = 1;
    while (p < v) p <<= 1;
    return p;
}

ccfr_status check_params(const ccfr_params* p) {
    if (!p) return CCFR_ERR_INVALID_ARG;
    if (!(p->r > 0.f) || !(p->xi >= 0.f) || !(p->delta >= 0.f) || !(p->pad > 0.f)) return CCFR_ERR_INVALID_ARG;
    if (!(p->eps_retract >= 0.f) || !(p->eps_dep > 0.f) || !(p->tau_feas >= 0.f)) return CCFR_ERR_INVALID_ARG;
    if (p->max_passes < 0 || p->max_passes > 64 || p->solver_iters < 1 || p->solver_iters > 10000)
        return CCFR_ERR_INVALID_ARG;
    if (p->plane_capacity < 32 || p->plane_capacity % 32 != 0 || p->plane_capacity > 65536) return CCFR_ERR_INVALID_ARG;
    if (!(p->cell_size >= 0.f) || !(p->dt > 0.f) || !(p->compliance >= 0.f)) return CCFR_ERR_INVALID_ARG;
    if (!(p->cell_factor >= 0.f) || p->cell_factor > 64.f) return CCFR_ERR_INVALID_ARG;
    if (p->pair_capacity < 0 || p->pair_capacity > 1024) return CCFR_ERR_INVALID_ARG;
    if (!(p->response_stiffness >= 0.f) || !(p->mu_s >= 0.f) || !(p->mu_k >= 0.f) || !(p->delta_v >= 0.f))
        return CCFR_ERR_INVALID_ARG;
    if (p->delta > 0.f && !(p->delta_v > 0.f)) return CCFR_ERR_INVALID_ARG;
    return CCFR_OK;
}

ccfr_status from_cuda(cudaError_t e) { return e == cudaSuccess ? CCFR_OK : CCFR_ERR_CUDA; }

// Enqueue one full substep (Alg. 4) on stream st.
void enqueue_step(ccfr_ctx* c, float4* x, float4* v, cudaStream_t st, StageTimer* tm = nullptr) {
    if (tm) tm->mark(ST_MISC, st);
    launch_predict(c->dc, x, v, st);
    if (tm) tm->mark(ST_PREDICT, st);
    int early = (c->prm.flags & CCFR_FLAG_EARLY_EXIT) ? 1 : 0;
    for (int it = 0; it < c->prm.solver_iters; ++it)
        launch_iteration(c->dc, x, st, c->color_off.data(), c->n_colors, c->tile_sums, c->n_buckets_total, early, tm,
                         &c->side, c->tcolor_off.data(), c->n_tcolors);
    launch_update(c->dc, x, v, st);
    if (tm) tm->mark(ST_MISC, st);
}

const char* kStageNames[N_STAGES] = {"predict", "grid_extent", "grid_count", "grid_scan", "grid_scatter",
                                     "emit_vf", "emit_ee", "emit_pp", "xpbd", "project", "misc",
                                     "grid_units", "emit_vf_big", "emit_ee_big", "project_heavy",
                                     "project_short", "response"};

}  // namespace

extern "C" {

const char* ccfr_status_string(ccfr_status s) {
    switch (s) {
        case CCFR_OK: return "ok";
        case CCFR_ERR_INVALID_ARG: return "invalid argument";
        case CCFR_ERR_CAPACITY: return "output capacity exceeded";
        case CCFR_ERR_OOM: return "device allocation failed";
        case CCFR_ERR_CUDA: return "CUDA runtime error";
        case CCFR_ERR_TIMEOUT: return "bounded wait timed out";
        case CCFR_ERR_NONFINITE: return "non-finite input";
        case CCFR_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

// Build a context from host topology (validated, vertex ids in [0, N)).
// vscene / sparams: the scene of every vertex and each scene's (r, 2r, xi,
// pad), or empty for a single scene.
static ccfr_status create_impl(const std::vector<int>& he, const std::vector<int>& ht, int N,
                               const ccfr_params* params, const float* rest_x,
                               const std::vector<unsigned short>& vscene, const std::vector<float4>& sparams,
                               cudaStream_t st, ccfr_ctx** out, const Extras* ex = nullptr) {
    const int E = (int)(he.size() / 2), T = (int)(ht.size() / 3);
    const int L = ex ? (int)(ex->links.size() / 2) : 0, Q = ex ? (int)(ex->tets.size() / 4) : 0;
    // 1: in a collision edge; 2: only in links or tetrahedra (no collision)
    std::vector<char> used(N > 0 ? N : 1, 0);
    for (int e = 0; e < E; ++e) { used[he[2 * e]] = 1; used[he[2 * e + 1]] = 1; }
    for (int i = 0; i < L; ++i)
        for (int k = 0; k < 2; ++k) if (!used[ex->links[2 * i + k]]) used[ex->links[2 * i + k]] = 2;
    for (int q = 0; q < Q; ++q)
        for (int k = 0; k < 4; ++k) if (!used[ex->tets[4 * q + k]]) used[ex->tets[4 * q + k]] = 2;
    std::vector<int> pts;
    bool interior = false;
    for (int i = 0; i < N; ++i) {
        if (!used[i]) pts.push_back(i);
        if (used[i] == 2) interior = true;
    }
    // free edges (of no triangle) meet the isolated points
    std::vector<unsigned char> efree;
    if (!pts.empty() && E > 0) {
        efree.assign(E, 1);
        for (int t = 0; t < T; ++t)
            for (int k = 0; k < 3; ++k) {
                int a = ht[3 * t + k], b = ht[3 * t + (k + 1) % 3];
                if (a > b) std::swap(a, b);
                int lo = 0, hi = E;
                while (lo < hi) {
                    int mid = (lo + hi) / 2;
                    if (he[2 * mid] < a || (he[2 * mid] == a && he[2 * mid + 1] < b)) lo = mid + 1; else hi = mid;
                }
                if (lo < E && he[2 * lo] == a && he[2 * lo + 1] == b) efree[lo] = 0;
            }
        bool any = false;
        for (int e = 0; e < E; ++e) any |= efree[e] != 0;
        if (!any) efree.clear();
    }
    // distance constraints: the edges in canonical order, then the links;
    // greedy first-fit colouring in that order
    const int ND = E + L;
    auto dpair = [&](int i, int k) { return i < E ? he[2 * i + k] : ex->links[2 * (i - E) + k]; };
    std::vector<unsigned long long> vmask(N > 0 ? N : 1, 0ull);
    std::vector<int> col(ND > 0 ? ND : 1, 0);
    int ncol = 0;
    for (int e = 0; e < ND; ++e) {
        unsigned long long m = vmask[dpair(e, 0)] | vmask[dpair(e, 1)];
        int k = 0;
        while (k < 64 && ((m >> k) & 1ull)) ++k;
        if (k == 64) return CCFR_ERR_INVALID_ARG;
        col[e] = k;
        vmask[dpair(e, 0)] |= 1ull << k;
        vmask[dpair(e, 1)] |= 1ull << k;
        if (k + 1 > ncol) ncol = k + 1;
    }
    std::vector<int> coff(ncol + 1, 0);
    for (int e = 0; e < ND; ++e) coff[col[e] + 1]++;
    for (int k = 0; k < ncol; ++k) coff[k + 1] += coff[k];
    std::vector<int> ecol(2 * (size_t)ND);
    std::vector<float> acol(ND > 0 ? ND : 1);
    {
        std::vector<int> fill(coff.begin(), coff.end() - 1);
        for (int e = 0; e < ND; ++e) {
            int pos = fill[col[e]]++;
            ecol[2 * pos] = dpair(e, 0);
            ecol[2 * pos + 1] = dpair(e, 1);
            acol[pos] = (e < E ? params->compliance : ex->link_comp[e - E]) / (params->dt * params->dt);
        }
    }
    // tetrahedra: greedy first-fit colouring in their order
    std::vector<int> tcoff(1, 0), tcol4;
    int ntcol = 0;
    if (Q > 0) {
        std::fill(vmask.begin(), vmask.end(), 0ull);
        std::vector<int> tc(Q);
        for (int q = 0; q < Q; ++q) {
            const int* Tq = &ex->tets[4 * q];
            unsigned long long m = vmask[Tq[0]] | vmask[Tq[1]] | vmask[Tq[2]] | vmask[Tq[3]];
            int k = 0;
            while (k < 64 && ((m >> k) & 1ull)) ++k;
            if (k == 64) return CCFR_ERR_INVALID_ARG;
            tc[q] = k;
            for (int j = 0; j < 4; ++j) vmask[Tq[j]] |= 1ull << k;
            if (k + 1 > ntcol) ntcol = k + 1;
        }
        tcoff.assign(ntcol + 1, 0);
        for (int q = 0; q < Q; ++q) tcoff[tc[q] + 1]++;
        for (int k = 0; k < ntcol; ++k) tcoff[k + 1] += tcoff[k];
        tcol4.resize(4 * (size_t)Q);
        std::vector<int> fill(tcoff.begin(), tcoff.end() - 1);
        for (int q = 0; q < Q; ++q) {
            int pos = fill[tc[q]]++;
            for (int j = 0; j < 4; ++j) tcol4[4 * pos + j] = ex->tets[4 * q + j];
        }
    }

    ccfr_ctx* c = new (std::nothrow) ccfr_ctx();
    if (!c) return CCFR_ERR_OOM;
    cudaGetDevice(&c->device);
    c->prm = *params;
    c->color_off = coff;
    c->n_colors = ncol;
    c->tcolor_off = tcoff;
    c->n_tcolors = ntcol;
    DevCtx& d = c->dc;
    d.n_verts = N;
    d.n_edges = E;
    d.n_tris = T;
    d.n_pts = (int)pts.size();
    d.p.r = params->r;
    d.p.two_r = 2.f * params->r;
    d.p.xi = params->xi;
    d.p.pad = params->pad;
    d.p.eps = params->eps_retract;
    d.p.eps_dep = params->eps_dep;
    d.p.tau = params->tau_feas;
    d.p.dt = params->dt;
    d.p.gx = params->gravity[0];
    d.p.gy = params->gravity[1];
    d.p.gz = params->gravity[2];
    d.p.alpha_tilde = params->compliance / (params->dt * params->dt);
    d.n_dist = ND;
    d.n_tets = Q;
    d.alpha_vol = ex ? ex->vol_comp / (params->dt * params->dt) : 0.f;
    d.p.max_passes = params->max_passes;
    d.p.K = params->plane_capacity;
    d.p.short_max = short_list_max(d.p.K);
    d.p.cell_size = params->cell_size;
    d.p.delta = params->delta;
    d.p.k_resp = params->response_stiffness;
    d.p.delta_v = params->delta_v;
    d.p.mu_s = params->mu_s;
    d.p.mu_k = params->mu_k;
    // grid geometry: tables of triangles, edges, isolated points, vertices,
    // oversized edges and giant edges (items of the last two are the edges that
    // do not fit an edge cell, routed there by the edge items' own passes)
    int nk[N_TABLES] = {T, E, d.n_pts, N, E, E, E};
    d.n_items = T + E + d.n_pts + N;
    d.item_base[0] = 0;
    for (int k = 1; k < N_TABLES; ++k) d.item_base[k] = d.item_base[k - 1] + (k - 1 < KIND_BIGE ? nk[k - 1] : 0);
    int btot = 0;
    for (int k = 0; k < N_TABLES; ++k) {
        // the oversized-edge tables are sized for a quarter / a sixteenth of the edges
        int want = (k == KIND_BIGE || k == KIND_BIGS) ? nk[k] / 4 : (k == KIND_GIANT) ? nk[k] / 16 : nk[k];
        unsigned M = next_pow2((unsigned)(want > 64 ? want : 64));
        d.bucket_base[k] = btot;
        d.bucket_mask[k] = (int)(M - 1);
        btot += (int)M;
    }
    d.bucket_base[N_TABLES] = btot;
    c->n_buckets_total = btot;
    d.n_kind[0] = T;
    d.n_kind[1] = E;
    d.n_kind[2] = d.n_pts;
    d.cell_factor = params->cell_factor > 0.f ? params->cell_factor : 1.5f;
    d.emit_bps = 8;
    d.big_base[0] = 0;
    d.big_base[1] = T;
    d.unit_base[0] = 0;
    d.unit_base[1] = T + 1;
    d.unit_base[2] = T + 1 + E + 1;
    int n_units = T + E + d.n_pts + 3;
    {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
        d.n_sm = nsm;
    }
    const int SCAN_TILE = 4096;
    const int n_tiles = (btot + 1 + SCAN_TILE - 1) / SCAN_TILE;

    size_t NK = (size_t)N * params->plane_capacity;
    bool ok = true;
    ok &= dalloc(c, &d.planes, NK) == cudaSuccess;
    // the contact response reads each plane's gap phi (only stored when it is on)
    if (params->delta > 0.f) ok &= dalloc(c, &d.phi, NK) == cudaSuccess;
    if (params->flags & CCFR_FLAG_STORE_KEYS) ok &= dalloc(c, &d.keys, NK) == cudaSuccess;
    ok &= dalloc(c, &d.count, N) == cudaSuccess;
    ok &= dalloc(c, &d.dmin_drop, N) == cudaSuccess;
    ok &= dalloc(c, &d.x_tilde, N) == cudaSuccess;
    ok &= dalloc(c, &d.x_n, N) == cudaSuccess;
    ok &= dalloc(c, &d.x_s, N) == cudaSuccess;
    ok &= dalloc(c, &d.lambda, ND) == cudaSuccess;
    int2* edges = nullptr;
    int2* edges_col = nullptr;
    int3* tris = nullptr;
    int* dpts = nullptr;
    float* rest = nullptr;
    float* alpha = nullptr;
    int4* tets_col = nullptr;
    unsigned char* vcol = nullptr;
    ok &= dalloc(c, &edges, E) == cudaSuccess;
    ok &= dalloc(c, &edges_col, ND) == cudaSuccess;
    ok &= dalloc(c, &rest, ND) == cudaSuccess;
    ok &= dalloc(c, &alpha, ND) == cudaSuccess;
    if (Q > 0) {
        ok &= dalloc(c, &tets_col, Q) == cudaSuccess;
        ok &= dalloc(c, &d.vol6_col, Q) == cudaSuccess;
        ok &= dalloc(c, &d.tlambda, Q) == cudaSuccess;
    }
    if (interior) ok &= dalloc(c, &vcol, N) == cudaSuccess;
    std::vector<int> hfree;
    for (size_t e = 0; e < efree.size(); ++e) if (efree[e]) hfree.push_back((int)e);
    int* dflist = nullptr;
    if (!hfree.empty()) ok &= dalloc(c, &dflist, hfree.size()) == cudaSuccess;
    ok &= dalloc(c, &tris, T) == cudaSuccess;
    ok &= dalloc(c, &dpts, pts.size()) == cudaSuccess;
    ok &= dalloc(c, &d.ext_bits, 3) == cudaSuccess;
    ok &= dalloc(c, &d.bucket_count, (size_t)btot + 1) == cudaSuccess;
    ok &= dalloc(c, &d.bucket_fill, (size_t)btot) == cudaSuccess;
    ok &= dalloc(c, &d.item_bucket, d.n_items) == cudaSuccess;
    ok &= dalloc(c, &d.rec, 2 * (size_t)d.n_items) == cudaSuccess;
    ok &= dalloc(c, &d.units, (size_t)n_units) == cudaSuccess;
    ok &= dalloc(c, &d.ext_sum, 3) == cudaSuccess;
    ok &= dalloc(c, &d.big, (size_t)T + E) == cudaSuccess;
    ok &= dalloc(c, &d.big_box, 2 * ((size_t)T + E)) == cudaSuccess;
    ok &= dalloc(c, &d.work, (size_t)N) == cudaSuccess;
    ok &= dalloc(c, &d.work_count, 4) == cudaSuccess;
    ok &= dalloc(c, &d.big_count, 2) == cudaSuccess;
    const long pcap = params->pair_capacity > 0 ? params->pair_capacity : PAIR_CAP_DEFAULT;
    d.bq_cap = pcap * ((long)T + E) + 4096;
    ok &= dalloc(c, &d.bq, (size_t)d.bq_cap) == cudaSuccess;
    ok &= dalloc(c, &d.bq_count, 1) == cudaSuccess;
    d.eq_cap = 3 * pcap * (long)E + 4096;
    ok &= dalloc(c, &d.eq, (size_t)d.eq_cap) == cudaSuccess;
    ok &= dalloc(c, &d.eq_count, 1) == cudaSuccess;
    ok &= dalloc(c, &d.unit_count, 3) == cudaSuccess;
    ok &= dalloc(c, &d.sched, N_SCHED) == cudaSuccess;
    ok &= dalloc(c, &c->tile_sums, (size_t)n_tiles) == cudaSuccess;
    ok &= dalloc(c, &d.flags, 2) == cudaSuccess;
    ok &= dalloc(c, &d.stats, 1) == cudaSuccess;
    ok &= dalloc(c, &c->pair_count, 3) == cudaSuccess;
    ok &= dalloc(c, &c->hx, N) == cudaSuccess;
    ok &= dalloc(c, &c->hv, N) == cudaSuccess;
    unsigned short* dscene = nullptr;
    float4* dsp = nullptr;
    if (!vscene.empty()) {
        ok &= dalloc(c, &dscene, vscene.size()) == cudaSuccess;
        ok &= dalloc(c, &dsp, sparams.size()) == cudaSuccess;
        ok &= dalloc(c, &c->active, sparams.size()) == cudaSuccess;
    }
    if (!ok) { cudaGetLastError(); free_ctx(c); return CCFR_ERR_OOM; }
    d.vscene = dscene;
    d.sparams = dsp;
    d.active = c->active;
    c->n_scenes = vscene.empty() ? 1 : (int)sparams.size();
    d.edges = edges;
    d.edges_col = edges_col;
    d.rest_col = rest;
    d.alpha_col = alpha;
    d.tets_col = tets_col;
    d.vcollide = vcol;
    d.free_list = dflist;
    d.n_free = (int)hfree.size();
    d.tris = tris;
    d.pts = dpts;

    cudaError_t err = cudaSuccess;
    if (E) err = cudaMemcpyAsync(edges, he.data(), he.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess && ND) {
        err = cudaMemcpyAsync(edges_col, ecol.data(), ecol.size() * sizeof(int), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(alpha, acol.data(), (size_t)ND * sizeof(float), cudaMemcpyHostToDevice, st);
    }
    if (err == cudaSuccess && Q)
        err = cudaMemcpyAsync(tets_col, tcol4.data(), tcol4.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    std::vector<unsigned char> hvcol;
    if (err == cudaSuccess && vcol) {
        hvcol.resize(N);
        for (int i = 0; i < N; ++i) hvcol[i] = used[i] == 2 ? 0 : 1;
        err = cudaMemcpyAsync(vcol, hvcol.data(), (size_t)N, cudaMemcpyHostToDevice, st);
    }
    if (err == cudaSuccess && dflist)
        err = cudaMemcpyAsync(dflist, hfree.data(), hfree.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess && T) err = cudaMemcpyAsync(tris, ht.data(), ht.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess && !pts.empty())
        err = cudaMemcpyAsync(dpts, pts.data(), pts.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess && dscene) {
        err = cudaMemcpyAsync(dscene, vscene.data(), vscene.size() * sizeof(unsigned short), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(dsp, sparams.data(), sparams.size() * sizeof(float4), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess) err = cudaMemsetAsync(c->active, 1, sparams.size(), st);
    }
    if (err == cudaSuccess) err = cudaMemsetAsync(d.flags, 0, 2 * sizeof(int), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(d.stats, 0, sizeof(DevStats), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(d.count, 0, (size_t)(N > 0 ? N : 1) * sizeof(unsigned), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(d.dmin_drop, 0xFF, (size_t)(N > 0 ? N : 1) * sizeof(unsigned), st);
    if (err == cudaSuccess && (ND || Q)) {
        if (rest_x) launch_rest_state(d, (const float4*)rest_x, st);
        else c->rest_pending = true;
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = configure_kernels();
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&c->side.s, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&c->side.fork, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&c->side.join, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) { free_ctx(c); return CCFR_ERR_CUDA; }
    *out = c;
    return CCFR_OK;
}

static ccfr_status create_single(const ccfr_mesh* mesh, const ccfr_params* params, void* stream, ccfr_ctx** out,
                                 const Extras* ex) {
    if (!out) return CCFR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mesh || check_params(params) != CCFR_OK) return CCFR_ERR_INVALID_ARG;
    const int N = mesh->n_verts, E = mesh->n_edges, T = mesh->n_tris;
    if (N < 0 || E < 0 || T < 0 || N > (1 << 30) || E > (1 << 30) || T > (1 << 30)) return CCFR_ERR_INVALID_ARG;
    if ((E > 0 && !mesh->edges) || (T > 0 && !mesh->tris)) return CCFR_ERR_INVALID_ARG;
    if (mesh->rest_x && !aligned16(mesh->rest_x)) return CCFR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;

    // topology to the host: validation, isolated points, edge colours
    std::vector<int> he(2 * (size_t)E), ht(3 * (size_t)T);
    if (E && cudaMemcpy(he.data(), mesh->edges, he.size() * sizeof(int), cudaMemcpyDefault) != cudaSuccess)
        return CCFR_ERR_CUDA;
    if (T && cudaMemcpy(ht.data(), mesh->tris, ht.size() * sizeof(int), cudaMemcpyDefault) != cudaSuccess)
        return CCFR_ERR_CUDA;
    for (int e = 0; e < E; ++e) {
        int a = he[2 * e], b = he[2 * e + 1];
        if (a < 0 || b >= N || a >= b) return CCFR_ERR_INVALID_ARG;
        if (e > 0) {
            int pa = he[2 * e - 2], pb = he[2 * e - 1];
            if (!(pa < a || (pa == a && pb < b))) return CCFR_ERR_INVALID_ARG;
        }
    }
    for (int t = 0; t < T; ++t) {
        int a = ht[3 * t], b = ht[3 * t + 1], d = ht[3 * t + 2];
        if (a < 0 || b < 0 || d < 0 || a >= N || b >= N || d >= N || a == b || b == d || a == d)
            return CCFR_ERR_INVALID_ARG;
    }
    return create_impl(he, ht, N, params, mesh->rest_x, {}, {}, st, out, ex);
}

ccfr_status ccfr_create(const ccfr_mesh* mesh, const ccfr_params* params, void* stream, ccfr_ctx** out) {
    return create_single(mesh, params, stream, out, nullptr);
}

ccfr_status ccfr_create_ext(const ccfr_mesh_ext* mesh, const ccfr_params* params, void* stream, ccfr_ctx** out) {
    if (!out) return CCFR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mesh || check_params(params) != CCFR_OK) return CCFR_ERR_INVALID_ARG;
    const int N = mesh->mesh.n_verts, L = mesh->n_links, Q = mesh->n_tets;
    if (L < 0 || Q < 0 || L > (1 << 30) || Q > (1 << 28)) return CCFR_ERR_INVALID_ARG;
    if ((L > 0 && (!mesh->links || !mesh->link_compliance)) || (Q > 0 && !mesh->tets)) return CCFR_ERR_INVALID_ARG;
    if (!(mesh->volume_compliance >= 0.f)) return CCFR_ERR_INVALID_ARG;
    Extras ex;
    ex.links.resize(2 * (size_t)L);
    ex.link_comp.resize(L);
    ex.tets.resize(4 * (size_t)Q);
    ex.vol_comp = mesh->volume_compliance;
    if (L && (cudaMemcpy(ex.links.data(), mesh->links, ex.links.size() * sizeof(int), cudaMemcpyDefault) != cudaSuccess ||
              cudaMemcpy(ex.link_comp.data(), mesh->link_compliance, (size_t)L * sizeof(float), cudaMemcpyDefault) !=
                  cudaSuccess))
        return CCFR_ERR_CUDA;
    if (Q && cudaMemcpy(ex.tets.data(), mesh->tets, ex.tets.size() * sizeof(int), cudaMemcpyDefault) != cudaSuccess)
        return CCFR_ERR_CUDA;
    for (int i = 0; i < L; ++i) {
        int a = ex.links[2 * i], b = ex.links[2 * i + 1];
        if (a < 0 || b < 0 || a >= N || b >= N || a == b || !(ex.link_comp[i] >= 0.f)) return CCFR_ERR_INVALID_ARG;
    }
    for (int q = 0; q < Q; ++q) {
        const int* T = &ex.tets[4 * q];
        for (int j = 0; j < 4; ++j) {
            if (T[j] < 0 || T[j] >= N) return CCFR_ERR_INVALID_ARG;
            for (int k = j + 1; k < 4; ++k) if (T[j] == T[k]) return CCFR_ERR_INVALID_ARG;
        }
    }
    return create_single(&mesh->mesh, params, stream, out, &ex);
}

ccfr_status ccfr_create_batch(const ccfr_mesh* meshes, const ccfr_params* params, int n_scenes, void* stream,
                              ccfr_ctx** out) {
    if (!out) return CCFR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!meshes || !params || n_scenes < 1 || n_scenes > 2048) return CCFR_ERR_INVALID_ARG;
    for (int k = 0; k < n_scenes; ++k) {
        if (check_params(&params[k]) != CCFR_OK) return CCFR_ERR_INVALID_ARG;
        // what the scenes share: the time step, the loop and the projection settings
        if (params[k].dt != params[0].dt || params[k].solver_iters != params[0].solver_iters ||
            params[k].max_passes != params[0].max_passes || params[k].plane_capacity != params[0].plane_capacity ||
            params[k].eps_retract != params[0].eps_retract || params[k].eps_dep != params[0].eps_dep ||
            params[k].tau_feas != params[0].tau_feas || params[k].compliance != params[0].compliance ||
            params[k].gravity[0] != params[0].gravity[0] || params[k].gravity[1] != params[0].gravity[1] ||
            params[k].gravity[2] != params[0].gravity[2] || params[k].flags != params[0].flags ||
            params[k].delta != params[0].delta || params[k].response_stiffness != params[0].response_stiffness ||
            params[k].delta_v != params[0].delta_v || params[k].mu_s != params[0].mu_s ||
            params[k].mu_k != params[0].mu_k)
            return CCFR_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    long NL = 0, EL = 0, TL = 0;
    for (int k = 0; k < n_scenes; ++k) {
        const ccfr_mesh& m = meshes[k];
        if (m.n_verts < 0 || m.n_edges < 0 || m.n_tris < 0) return CCFR_ERR_INVALID_ARG;
        if ((m.n_edges > 0 && !m.edges) || (m.n_tris > 0 && !m.tris) || !m.rest_x || !aligned16(m.rest_x))
            return CCFR_ERR_INVALID_ARG;
        NL += m.n_verts; EL += m.n_edges; TL += m.n_tris;
    }
    if (NL > (1 << 30) || EL > (1 << 30) || TL > (1 << 30)) return CCFR_ERR_INVALID_ARG;
    const int N = (int)NL;
    std::vector<int> he(2 * (size_t)EL), ht(3 * (size_t)TL);
    std::vector<unsigned short> vscene((size_t)N);
    std::vector<float4> sparams((size_t)n_scenes);
    size_t eo = 0, to = 0;
    int vo = 0;
    for (int k = 0; k < n_scenes; ++k) {
        const ccfr_mesh& m = meshes[k];
        std::vector<int> le(2 * (size_t)m.n_edges), lt(3 * (size_t)m.n_tris);
        if (m.n_edges && cudaMemcpy(le.data(), m.edges, le.size() * sizeof(int), cudaMemcpyDefault) != cudaSuccess)
            return CCFR_ERR_CUDA;
        if (m.n_tris && cudaMemcpy(lt.data(), m.tris, lt.size() * sizeof(int), cudaMemcpyDefault) != cudaSuccess)
            return CCFR_ERR_CUDA;
        for (int e = 0; e < m.n_edges; ++e) {
            int a = le[2 * e], b = le[2 * e + 1];
            if (a < 0 || b >= m.n_verts || a >= b) return CCFR_ERR_INVALID_ARG;
            if (e > 0 && !(le[2 * e - 2] < a || (le[2 * e - 2] == a && le[2 * e - 1] < b))) return CCFR_ERR_INVALID_ARG;
            he[eo + 2 * e] = a + vo;
            he[eo + 2 * e + 1] = b + vo;
        }
        for (int t = 0; t < m.n_tris; ++t) {
            int a = lt[3 * t], b = lt[3 * t + 1], d = lt[3 * t + 2];
            if (a < 0 || b < 0 || d < 0 || a >= m.n_verts || b >= m.n_verts || d >= m.n_verts || a == b || b == d ||
                a == d)
                return CCFR_ERR_INVALID_ARG;
            ht[to + 3 * t] = a + vo;
            ht[to + 3 * t + 1] = b + vo;
            ht[to + 3 * t + 2] = d + vo;
        }
        for (int i = 0; i < m.n_verts; ++i) vscene[vo + i] = (unsigned short)k;
        sparams[k] = make_float4(params[k].r, 2.f * params[k].r, params[k].xi, params[k].pad);
        eo += 2 * (size_t)m.n_edges;
        to += 3 * (size_t)m.n_tris;
        vo += m.n_verts;
    }
    // rest shapes side by side in one device buffer (read once for the rest lengths)
    float4* rest = nullptr;
    if (cudaMalloc((void**)&rest, (size_t)(N > 0 ? N : 1) * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        return CCFR_ERR_OOM;
    }
    vo = 0;
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < n_scenes && err == cudaSuccess; ++k) {
        if (meshes[k].n_verts)
            err = cudaMemcpyAsync(rest + vo, meshes[k].rest_x, (size_t)meshes[k].n_verts * sizeof(float4),
                                  cudaMemcpyDefault, st);
        vo += meshes[k].n_verts;
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    ccfr_status s = (err == cudaSuccess)
                        ? create_impl(he, ht, N, &params[0], (const float*)rest, vscene, sparams, st, out)
                        : CCFR_ERR_CUDA;
    cudaStreamSynchronize(st);
    cudaFree(rest);
    return s;
}

ccfr_status ccfr_destroy(ccfr_ctx* c) {
    if (!c) return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    free_ctx(c);
    return CCFR_OK;
}

ccfr_status ccfr_build_regions(ccfr_ctx* c, const float* x, void* stream) {
    if (!c || !x || !aligned16(x)) return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    launch_clear_regions(c->dc, st);
    launch_build(c->dc, (const float4*)x, st, MODE_PLANES, nullptr, c->tile_sums, c->n_buckets_total, nullptr,
                 &c->side);
    c->regions_valid = true;
    return from_cuda(cudaGetLastError());
}

ccfr_status ccfr_project(ccfr_ctx* c, const float* x, float* x_io, unsigned char* halt_out, void* stream) {
    if (!c || !x || !x_io || !aligned16(x) || !aligned16(x_io)) return CCFR_ERR_INVALID_ARG;
    if (!c->regions_valid) return CCFR_ERR_STATE;
    DeviceGuard g(c->device);
    launch_project(c->dc, (const float4*)x, (float4*)x_io, halt_out, (cudaStream_t)stream);
    return from_cuda(cudaGetLastError());
}

ccfr_status ccfr_step(ccfr_ctx* c, float* x, float* v, void* stream) {
    if (!c || !x || !v || !aligned16(x) || !aligned16(v)) return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (c->rest_pending) {
        launch_rest_state(c->dc, (const float4*)x, st);
        c->rest_pending = false;
    }
    if (c->prm.flags & CCFR_FLAG_NO_GRAPH) {
        enqueue_step(c, (float4*)x, (float4*)v, st);
        c->regions_valid = true;
        return from_cuda(cudaGetLastError());
    }
    cudaGraphExec_t exec = nullptr;
    for (auto& e : c->graphs)
        if (e.x == x && e.v == v) { exec = e.exec; break; }
    if (!exec) {
        // record the substep once for this (x, v) pair and replay it afterwards
        cudaError_t err = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) return CCFR_ERR_CUDA;
        enqueue_step(c, (float4*)x, (float4*)v, c->cap_stream);
        cudaGraph_t graph = nullptr;
        err = cudaStreamEndCapture(c->cap_stream, &graph);
        if (err != cudaSuccess || !graph) { cudaGetLastError(); return CCFR_ERR_CUDA; }
        err = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (err != cudaSuccess) { cudaGetLastError(); return CCFR_ERR_CUDA; }
        if (c->graphs.size() >= 16) {
            cudaGraphExecDestroy(c->graphs.front().exec);
            c->graphs.erase(c->graphs.begin());
        }
        c->graphs.push_back(GraphEntry{x, v, exec});
    }
    cudaError_t err = cudaGraphLaunch(exec, st);
    c->regions_valid = true;
    return from_cuda(err);
}

ccfr_status ccfr_step_active(ccfr_ctx* c, float* x, float* v, const unsigned char* active, void* stream) {
    if (!c || !active) return CCFR_ERR_INVALID_ARG;
    if (!c->active) return CCFR_ERR_INVALID_ARG;           // not a batched context
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t err = cudaMemcpyAsync(c->active, active, (size_t)c->n_scenes, cudaMemcpyDeviceToDevice, st);
    if (err != cudaSuccess) return CCFR_ERR_CUDA;
    ccfr_status s = ccfr_step(c, x, v, stream);
    // back to "every scene" for the next ccfr_step
    err = cudaMemsetAsync(c->active, 1, (size_t)c->n_scenes, st);
    if (s != CCFR_OK) return s;
    return from_cuda(err);
}

ccfr_status ccfr_step_timed(ccfr_ctx* c, float* x, float* v, double* stage_ms, int n_stages, void* stream) {
    if (!c || !x || !v || !stage_ms || n_stages < N_STAGES || !aligned16(x) || !aligned16(v)) return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (c->rest_pending) {
        launch_rest_state(c->dc, (const float4*)x, st);
        c->rest_pending = false;
    }
    int cap = 16 + c->prm.solver_iters * 16;
    std::vector<cudaEvent_t> ev(cap);
    std::vector<int> stg(cap);
    for (int i = 0; i < cap; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
            return CCFR_ERR_CUDA;
        }
    StageTimer tm{ev.data(), stg.data(), 0, cap};
    enqueue_step(c, (float4*)x, (float4*)v, st, &tm);
    cudaError_t err = cudaStreamSynchronize(st);
    for (int i = 0; i < n_stages; ++i) stage_ms[i] = 0.0;
    for (int i = 1; i < tm.n && err == cudaSuccess; ++i) {
        float ms = 0.f;
        err = cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
        stage_ms[stg[i]] += ms;
    }
    for (int i = 0; i < cap; ++i) cudaEventDestroy(ev[i]);
    c->regions_valid = true;
    return from_cuda(err);
}

const char* ccfr_stage_name(int i) { return (i >= 0 && i < N_STAGES) ? kStageNames[i] : ""; }

ccfr_status ccfr_step_record(ccfr_ctx* c, float* x, float* v, float* x_tilde_out, float* iterates_out,
                             void* stream) {
    if (!c || !x || !v || !aligned16(x) || !aligned16(v)) return CCFR_ERR_INVALID_ARG;
    if ((x_tilde_out && !aligned16(x_tilde_out)) || (iterates_out && !aligned16(iterates_out)))
        return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (c->rest_pending) {
        launch_rest_state(c->dc, (const float4*)x, st);
        c->rest_pending = false;
    }
    const size_t bytes = (size_t)c->dc.n_verts * sizeof(float4);
    launch_predict(c->dc, (float4*)x, (float4*)v, st);
    cudaError_t err = cudaSuccess;
    if (x_tilde_out && bytes) err = cudaMemcpyAsync(x_tilde_out, c->dc.x_tilde, bytes, cudaMemcpyDeviceToDevice, st);
    const int early = (c->prm.flags & CCFR_FLAG_EARLY_EXIT) ? 1 : 0;
    for (int it = 0; it < c->prm.solver_iters && err == cudaSuccess; ++it) {
        launch_iteration(c->dc, (float4*)x, st, c->color_off.data(), c->n_colors, c->tile_sums, c->n_buckets_total,
                         early, nullptr, &c->side, c->tcolor_off.data(), c->n_tcolors);
        if (iterates_out && bytes)
            err = cudaMemcpyAsync((char*)iterates_out + (size_t)it * bytes, x, bytes, cudaMemcpyDeviceToDevice, st);
    }
    if (err != cudaSuccess) return CCFR_ERR_CUDA;
    launch_update(c->dc, (float4*)x, (float4*)v, st);
    c->regions_valid = true;
    return from_cuda(cudaGetLastError());
}

ccfr_status ccfr_step_host(ccfr_ctx* c, float* x_host, float* v_host, void* stream) {
    if (!c || !x_host || !v_host) return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = (size_t)c->dc.n_verts * sizeof(float4);
    cudaError_t err = cudaMemcpyAsync(c->hx, x_host, bytes, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaMemcpyAsync(c->hv, v_host, bytes, cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return CCFR_ERR_CUDA;
    ccfr_status s = ccfr_step(c, (float*)c->hx, (float*)c->hv, stream);
    if (s != CCFR_OK) return s;
    err = cudaMemcpyAsync(x_host, c->hx, bytes, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaMemcpyAsync(v_host, c->hv, bytes, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    return from_cuda(err);
}

ccfr_status ccfr_get_candidates(ccfr_ctx* c, const float* x, int* vf, long cap_vf, int* ee, long cap_ee, int* vv,
                                long cap_vv, long* counts, void* stream) {
    if (!c || !x || !aligned16(x) || !counts || cap_vf < 0 || cap_ee < 0 || cap_vv < 0) return CCFR_ERR_INVALID_ARG;
    if ((cap_vf > 0 && !vf) || (cap_ee > 0 && !ee) || (cap_vv > 0 && !vv)) return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    PairOutHost po;
    po.out[0] = vf; po.out[1] = ee; po.out[2] = vv;
    po.cap[0] = cap_vf; po.cap[1] = cap_ee; po.cap[2] = cap_vv;
    po.count = c->pair_count;
    cudaError_t err = cudaMemsetAsync(c->pair_count, 0, 3 * sizeof(unsigned long long), st);
    if (err != cudaSuccess) return CCFR_ERR_CUDA;
    launch_build(c->dc, (const float4*)x, st, MODE_PAIRS, &po, c->tile_sums, c->n_buckets_total);
    unsigned long long h[3];
    err = cudaMemcpyAsync(h, c->pair_count, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return CCFR_ERR_CUDA;
    for (int k = 0; k < 3; ++k) counts[k] = (long)h[k];
    if (counts[0] > cap_vf || counts[1] > cap_ee || counts[2] > cap_vv) return CCFR_ERR_CAPACITY;
    return CCFR_OK;
}

ccfr_status ccfr_copy_regions(ccfr_ctx* c, float* planes, unsigned long long* keys, int* count, float* dmin_drop,
                              void* stream) {
    if (!c) return CCFR_ERR_INVALID_ARG;
    if (!c->regions_valid) return CCFR_ERR_STATE;
    if (keys && !c->dc.keys) return CCFR_ERR_STATE;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    size_t NK = (size_t)c->dc.n_verts * c->dc.p.K;
    cudaError_t err = cudaSuccess;
    if (planes) err = cudaMemcpyAsync(planes, c->dc.planes, NK * sizeof(float4), cudaMemcpyDeviceToDevice, st);
    if (err == cudaSuccess && keys)
        err = cudaMemcpyAsync(keys, c->dc.keys, NK * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
    if (err == cudaSuccess && count)
        err = cudaMemcpyAsync(count, c->dc.count, (size_t)c->dc.n_verts * sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (err == cudaSuccess && dmin_drop) launch_dmin_export(c->dc, dmin_drop, st);
    if (err == cudaSuccess) err = cudaGetLastError();
    return from_cuda(err);
}

ccfr_status ccfr_load_regions(ccfr_ctx* c, const float* planes, const int* count, int capacity, void* stream) {
    if (!c || !planes || !count || capacity < 1 || capacity > c->dc.p.K || !aligned16(planes))
        return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    launch_load_regions(c->dc, (const float4*)planes, count, capacity, (cudaStream_t)stream);
    c->regions_valid = true;
    return from_cuda(cudaGetLastError());
}

ccfr_status ccfr_get_info(const ccfr_ctx* c, int* n_verts, int* capacity, int* n_colors) {
    if (!c) return CCFR_ERR_INVALID_ARG;
    if (n_verts) *n_verts = c->dc.n_verts;
    if (capacity) *capacity = c->dc.p.K;
    if (n_colors) *n_colors = c->n_colors;
    return CCFR_OK;
}

ccfr_status ccfr_set_tuning(ccfr_ctx* c, const ccfr_tuning* t) {
    if (!c || !t) return CCFR_ERR_INVALID_ARG;
    if (!(t->cell_factor >= 0.f) || t->cell_factor > 64.f || t->emit_blocks_per_sm < 0 || t->emit_blocks_per_sm > 64)
        return CCFR_ERR_INVALID_ARG;
    if (t->plane_capacity != 0 && (t->plane_capacity < 32 || t->plane_capacity % 32 || t->plane_capacity > 65536))
        return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return CCFR_ERR_CUDA;
    if (t->plane_capacity && t->plane_capacity != c->dc.p.K) {
        // the only call besides ccfr_create that allocates: new plane lists
        size_t NK = (size_t)c->dc.n_verts * t->plane_capacity;
        float4* planes = nullptr;
        unsigned long long* keys = nullptr;
        float* phi = nullptr;
        if (cudaMalloc((void**)&planes, (NK ? NK : 1) * sizeof(float4)) != cudaSuccess) {
            cudaGetLastError();
            return CCFR_ERR_OOM;
        }
        if ((c->dc.keys && cudaMalloc((void**)&keys, (NK ? NK : 1) * sizeof(unsigned long long)) != cudaSuccess) ||
            (c->dc.phi && cudaMalloc((void**)&phi, (NK ? NK : 1) * sizeof(float)) != cudaSuccess)) {
            cudaGetLastError();
            cudaFree(planes);
            if (keys) cudaFree(keys);
            return CCFR_ERR_OOM;
        }
        for (auto& p : c->allocs) {
            if (p == (void*)c->dc.planes) { cudaFree(p); p = planes; }
            else if (c->dc.keys && p == (void*)c->dc.keys) { cudaFree(p); p = keys; }
            else if (c->dc.phi && p == (void*)c->dc.phi) { cudaFree(p); p = phi; }
        }
        c->dc.planes = planes;
        if (c->dc.keys) c->dc.keys = keys;
        if (c->dc.phi) c->dc.phi = phi;
        c->dc.p.K = t->plane_capacity;
        c->dc.p.short_max = short_list_max(t->plane_capacity);
        c->prm.plane_capacity = t->plane_capacity;
        c->regions_valid = false;
    }
    if (t->cell_factor > 0.f) c->dc.cell_factor = t->cell_factor;
    if (t->emit_blocks_per_sm > 0) c->dc.emit_bps = t->emit_blocks_per_sm;
    // recorded graphs captured the old settings
    for (auto& e : c->graphs) cudaGraphExecDestroy(e.exec);
    c->graphs.clear();
    return CCFR_OK;
}

ccfr_status ccfr_get_tuning(const ccfr_ctx* c, ccfr_tuning* t) {
    if (!c || !t) return CCFR_ERR_INVALID_ARG;
    t->cell_factor = c->dc.cell_factor;
    t->emit_blocks_per_sm = c->dc.emit_bps;
    t->plane_capacity = c->dc.p.K;
    return CCFR_OK;
}

ccfr_status ccfr_autotune(ccfr_ctx* c, const float* x, const float* v, int steps, ccfr_tuning* best, double* best_ms,
                          void* stream) {
    if (!c || !x || !v || !best || steps < 1 || steps > 16 || !aligned16(x) || !aligned16(v)) return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int N = c->dc.n_verts;
    size_t bytes = (size_t)(N > 0 ? N : 1) * sizeof(float4);
    // 1. plane capacity: as given, or 1.5 x the largest per-vertex count at x
    //    (counts are exact beyond the capacity)
    int K = best->plane_capacity;
    ccfr_status s = CCFR_OK;
    if (K != 0 && (K < 32 || K % 32 || K > 65536)) return CCFR_ERR_INVALID_ARG;
    if (K == 0) {
        s = ccfr_build_regions(c, x, stream);
        if (s != CCFR_OK) return s;
        std::vector<unsigned> cnt((size_t)N);
        if (N && cudaMemcpyAsync(cnt.data(), c->dc.count, (size_t)N * sizeof(unsigned), cudaMemcpyDeviceToHost,
                                 st) != cudaSuccess)
            return CCFR_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return CCFR_ERR_CUDA;
        unsigned mx = 0;
        for (unsigned k : cnt) mx = k > mx ? k : mx;
        K = (int)((mx * 3u / 2u + 32u + 31u) / 32u * 32u);
        if (K < 64) K = 64;
        if (K > 65536) K = 65536;
    }
    ccfr_tuning t{};
    t.plane_capacity = K;
    s = ccfr_set_tuning(c, &t);
    if (s != CCFR_OK) return s;
    // 2. cell size and emission grid: time `steps` substeps from a scratch copy of (x, v)
    float4 *xs = nullptr, *vs = nullptr;
    if (cudaMalloc((void**)&xs, bytes) != cudaSuccess || cudaMalloc((void**)&vs, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(xs);
        return CCFR_ERR_OOM;
    }
    const float factors[4] = {1.0f, 1.5f, 2.0f, 3.0f};
    const int bps[3] = {4, 8, 16};
    double best_t = 1e300;
    ccfr_tuning bt{1.5f, 8, K};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t err = cudaSuccess;
    for (float f : factors) {
        for (int b : bps) {
            ccfr_tuning cand{f, b, 0};
            if ((s = ccfr_set_tuning(c, &cand)) != CCFR_OK) break;
            err = cudaMemcpyAsync(xs, x, bytes, cudaMemcpyDeviceToDevice, st);
            if (err == cudaSuccess) err = cudaMemcpyAsync(vs, v, bytes, cudaMemcpyDeviceToDevice, st);
            if (err != cudaSuccess) break;
            cudaEventRecord(e0, st);
            for (int k = 0; k < steps; ++k) enqueue_step(c, xs, vs, st);
            cudaEventRecord(e1, st);
            err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err != cudaSuccess) break;
            if (ms < best_t) { best_t = ms; bt = ccfr_tuning{f, b, K}; }
        }
        if (s != CCFR_OK || err != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(xs);
    cudaFree(vs);
    if (s != CCFR_OK) return s;
    if (err != cudaSuccess) return CCFR_ERR_CUDA;
    s = ccfr_set_tuning(c, &bt);
    if (s != CCFR_OK) return s;
    *best = bt;
    if (best_ms) *best_ms = best_t / steps;
    c->regions_valid = false;
    return CCFR_OK;
}

ccfr_status ccfr_get_stats(ccfr_ctx* c, ccfr_stats* out) {
    if (!c || !out) return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    DevStats s;
    cudaError_t err = cudaDeviceSynchronize();
    if (err == cudaSuccess) err = cudaMemcpy(&s, c->dc.stats, sizeof(s), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return CCFR_ERR_CUDA;
    out->cand_vf = s.cand[0]; out->cand_ee = s.cand[1]; out->cand_vv = s.cand[2];
    out->cand_ve = s.cand[PAIR_VE]; out->pairs_ve = s.pairs[PAIR_VE]; out->planes_ve = s.planes_kind[PAIR_VE];
    out->pairs_vf = s.pairs[0]; out->pairs_ee = s.pairs[1]; out->pairs_vv = s.pairs[2];
    out->planes_vf = s.planes_kind[0]; out->planes_ee = s.planes_kind[1]; out->planes_vv = s.planes_kind[2];
    out->planes = s.planes;
    out->overflow_verts = s.overflow_verts;
    out->violated_verts = s.violated_verts;
    out->halts = s.halts;
    out->ee_fp64 = s.ee_fp64;
    out->feas_fp64 = s.feas_fp64;
    out->feas_halts = s.feas_halts;
    out->iterations = s.iterations;
    out->steps = s.steps;
    for (int i = 0; i < 16; ++i) out->aux[i] = s.aux[i];
    out->max_planes = s.max_planes;
    out->error_flags = s.error_flags;
    return (s.error_flags & ERR_NONFINITE) ? CCFR_ERR_NONFINITE : CCFR_OK;
}

ccfr_status ccfr_reset_stats(ccfr_ctx* c, void* stream) {
    if (!c) return CCFR_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    return from_cuda(cudaMemsetAsync(c->dc.stats, 0, sizeof(DevStats), (cudaStream_t)stream));
}

}  // extern "C"

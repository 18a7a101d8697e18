// Serving loop for CCFR step requests (see include/ccfr.h, "Serving").
//
// Scenes are registered with their topology and state on the host.  A worker
// thread admits a scene to the device (context + state) when a request for it
// is due and the HBM budget allows, evicting idle resident scenes (least
// recently used, state copied back to the host) when it does not.  Up to
// n_slots steps run at once, each on its own stream, so requests that arrive
// while others are on the GPU start as soon as a slot and memory are free and
// their work overlaps on the device.  Requests of one scene run in arrival
// order, one at a time.  Every wait is bounded: a step that does not finish
// within the timeout is reported as timed out.
//
// Batching (ccfr_server_set_batching): small scenes with the same settings
// are grouped into pools, each resident as one batched context.  A pool's
// launch steps, in one graph-captured substep, every member scene that has a
// request due when the launch starts (ccfr_step_active masks the others);
// requests that arrive meanwhile join the pool's next launch.  Pools are
// admitted and evicted as units.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ccfr.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct SceneRec {
    int n_verts = 0, n_edges = 0, n_tris = 0;
    std::vector<int> edges, tris;
    std::vector<float> x, v;           // host state (authoritative while not resident)
    std::vector<float> rest;           // rest shape (edge rest lengths)
    ccfr_params params{};
    size_t bytes = 0;                  // device bytes while resident
    ccfr_ctx* ctx = nullptr;
    float* dx = nullptr;
    float* dv = nullptr;
    bool busy = false;
    bool stall = false;                // test hook: pretend the step never finishes
    double last_used = 0.0;
    long steps_done = 0;
    int pool = -1;                     // pool of the scene (batching), or -1
    int member = -1;                   // its index in the pool
};

// Scenes stepped together in one batched context.
struct Pool {
    std::vector<int> members;          // scene ids, in pool order
    std::vector<long> voff;            // first vertex of each member in the merged arrays (+ total)
    ccfr_ctx* ctx = nullptr;
    float* dx = nullptr;               // merged state (device) while resident
    float* dv = nullptr;
    unsigned char* dmask = nullptr;    // per-member step mask (device)
    std::vector<unsigned char> hmask;
    size_t bytes = 0;
    bool busy = false;
    double last_used = 0.0;
};

struct Req {
    int scene;
    double t_arrival, t_start = -1.0, t_done = -1.0;
    int status = -1;                   // -1 pending, else ccfr_status
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    long req = -1;                     // request of a scene stepped alone
    int pool = -1;                     // or: the pool launched here and its requests
    std::vector<long> preqs;
    double t_launch = 0.0;
    bool stalled = false;
    bool busy() const { return req >= 0 || pool >= 0; }
};

}  // namespace

struct ccfr_server {
    int device = 0;
    size_t budget = 0;
    size_t resident = 0, peak_resident = 0;
    double timeout = 30.0;
    std::vector<SceneRec> scenes;
    std::vector<Req> reqs;
    std::vector<Slot> slots;
    std::mutex mu;
    std::thread worker;
    std::atomic<bool> running{false};
    std::atomic<bool> stop{false};
    double t0 = 0.0;
    long n_done = 0, admissions = 0, evictions = 0, failed = 0;
    long scan_from = 0;
    // batching
    int pool_max_verts = 0, pool_scene_max = 0;
    bool pools_formed = false;
    long pool_launches = 0;
    std::vector<Pool> pools;
};

namespace {

// Device bytes of a context for n verts, e edges, t triangles and capacity k
// (the allocations of ccfr_create, isolated points bounded by the vertices),
// plus the resident state x, v.
size_t ctx_bytes(long n, long e, long t, long k, bool keys, bool phi = false, int pair_cap = 0) {
    auto pow2 = [](long v) { long p = 64; while (p < v) p <<= 1; return p; };
    long buckets = pow2(t) + pow2(e) + pow2(n) + pow2(n) + 2 * pow2(e / 4) + pow2(e / 16) + 1;
    long items = t + e + 2 * n;
    size_t b = 0;
    b += (size_t)n * k * 16 + (keys ? (size_t)n * k * 8 : 0) + (phi ? (size_t)n * k * 4 : 0);
    b += (size_t)n * (16 * 5 + 4 * 2 + 16 + 16 * 2 + 4);
    b += (size_t)e * (8 + 8 + 4 + 4);
    b += (size_t)t * 12;
    b += (size_t)buckets * 8 + (size_t)items * (4 + 32) + (size_t)(t + e + n + 3) * 8 + (size_t)(t + e) * 36;
    const size_t pc = pair_cap > 0 ? (size_t)pair_cap : 32;
    b += ((size_t)(t + e) * pc + (size_t)e * 3 * pc + 2 * 4096) * 8;   // candidate-pair buffers
    b += 2 * (size_t)n * 16;               // resident x, v
    return b + (1 << 20);
}

// Copy a resident pool's state back to its members and release its memory.
ccfr_status release_pool(ccfr_server* sv, Pool& P) {
    for (size_t m = 0; m < P.members.size(); ++m) {
        SceneRec& sc = sv->scenes[P.members[m]];
        size_t nb = (size_t)sc.n_verts * 4 * sizeof(float);
        if (cudaMemcpy(sc.x.data(), P.dx + 4 * P.voff[m], nb, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(sc.v.data(), P.dv + 4 * P.voff[m], nb, cudaMemcpyDeviceToHost) != cudaSuccess)
            return CCFR_ERR_CUDA;
    }
    ccfr_destroy(P.ctx);
    cudaFree(P.dx);
    cudaFree(P.dv);
    cudaFree(P.dmask);
    P.ctx = nullptr;
    P.dx = P.dv = nullptr;
    P.dmask = nullptr;
    sv->resident -= P.bytes;
    sv->evictions++;
    return CCFR_OK;
}

// Evict the least recently used idle resident unit (a scene served alone, or
// a pool), its state copied back to the host.  False when every resident unit
// is busy (the caller waits).
bool evict_one(ccfr_server* sv, ccfr_status* err) {
    *err = CCFR_OK;
    int vs = -1, vp = -1;
    double oldest = 1e300;
    for (int k = 0; k < (int)sv->scenes.size(); ++k) {
        SceneRec& o = sv->scenes[k];
        if (o.ctx && !o.busy && o.last_used < oldest) { oldest = o.last_used; vs = k; vp = -1; }
    }
    for (int p = 0; p < (int)sv->pools.size(); ++p) {
        Pool& P = sv->pools[p];
        if (P.ctx && !P.busy && P.last_used < oldest) { oldest = P.last_used; vp = p; vs = -1; }
    }
    if (vp >= 0) {
        *err = release_pool(sv, sv->pools[vp]);
        return true;
    }
    if (vs < 0) return false;
    SceneRec& o = sv->scenes[vs];
    size_t nb = (size_t)o.n_verts * 4 * sizeof(float);
    if (cudaMemcpy(o.x.data(), o.dx, nb, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(o.v.data(), o.dv, nb, cudaMemcpyDeviceToHost) != cudaSuccess) {
        *err = CCFR_ERR_CUDA;
        return true;
    }
    ccfr_destroy(o.ctx);
    cudaFree(o.dx);
    cudaFree(o.dv);
    o.ctx = nullptr;
    o.dx = o.dv = nullptr;
    sv->resident -= o.bytes;
    sv->evictions++;
    return true;
}

// Make room for `bytes` more resident bytes.
ccfr_status make_room(ccfr_server* sv, size_t bytes) {
    while (sv->resident + bytes > sv->budget) {
        ccfr_status e;
        if (!evict_one(sv, &e)) return CCFR_ERR_OOM;   // everything resident is busy: wait
        if (e != CCFR_OK) return e;
    }
    return CCFR_OK;
}

// Make pool p resident: one batched context over its members (scene-local
// topology, rest shapes at registration), their current states merged.
ccfr_status admit_pool(ccfr_server* sv, int p) {
    Pool& P = sv->pools[p];
    if (P.ctx) return CCFR_OK;
    ccfr_status rs = make_room(sv, P.bytes);
    if (rs != CCFR_OK) return rs;
    const int M = (int)P.members.size();
    const long nv = P.voff[M];
    size_t ne = 0, nt = 0;
    for (int m = 0; m < M; ++m) {
        ne += sv->scenes[P.members[m]].edges.size();
        nt += sv->scenes[P.members[m]].tris.size();
    }
    int *de = nullptr, *dt = nullptr;
    float* dr = nullptr;
    const size_t nb = (size_t)nv * 4 * sizeof(float);
    cudaError_t err = cudaMalloc((void**)&dr, nb ? nb : 16);
    if (err == cudaSuccess) err = cudaMalloc((void**)&de, (ne ? ne : 1) * sizeof(int));
    if (err == cudaSuccess) err = cudaMalloc((void**)&dt, (nt ? nt : 1) * sizeof(int));
    if (err == cudaSuccess) err = cudaMalloc((void**)&P.dx, nb ? nb : 16);
    if (err == cudaSuccess) err = cudaMalloc((void**)&P.dv, nb ? nb : 16);
    if (err == cudaSuccess) err = cudaMalloc((void**)&P.dmask, (size_t)M);
    std::vector<ccfr_mesh> meshes((size_t)M);
    std::vector<ccfr_params> prm((size_t)M);
    size_t eo = 0, to = 0;
    for (int m = 0; m < M && err == cudaSuccess; ++m) {
        const SceneRec& sc = sv->scenes[P.members[m]];
        const size_t vb = (size_t)sc.n_verts * 4 * sizeof(float), vo = (size_t)P.voff[m] * 4;
        err = cudaMemcpy(dr + vo, sc.rest.data(), vb, cudaMemcpyHostToDevice);
        if (err == cudaSuccess) err = cudaMemcpy(P.dx + vo, sc.x.data(), vb, cudaMemcpyHostToDevice);
        if (err == cudaSuccess) err = cudaMemcpy(P.dv + vo, sc.v.data(), vb, cudaMemcpyHostToDevice);
        if (err == cudaSuccess && !sc.edges.empty())
            err = cudaMemcpy(de + eo, sc.edges.data(), sc.edges.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (err == cudaSuccess && !sc.tris.empty())
            err = cudaMemcpy(dt + to, sc.tris.data(), sc.tris.size() * sizeof(int), cudaMemcpyHostToDevice);
        meshes[m] = ccfr_mesh{sc.n_verts, sc.n_edges, sc.n_tris, de + eo, dt + to, dr + vo};
        prm[m] = sc.params;
        eo += sc.edges.size();
        to += sc.tris.size();
    }
    ccfr_status st = CCFR_OK;
    if (err == cudaSuccess) st = ccfr_create_batch(meshes.data(), prm.data(), M, nullptr, &P.ctx);
    cudaFree(de);
    cudaFree(dt);
    cudaFree(dr);
    if (err != cudaSuccess || st != CCFR_OK) {
        cudaGetLastError();
        cudaFree(P.dx);
        cudaFree(P.dv);
        cudaFree(P.dmask);
        P.dx = P.dv = nullptr;
        P.dmask = nullptr;
        P.ctx = nullptr;
        return st != CCFR_OK ? st : CCFR_ERR_OOM;
    }
    sv->resident += P.bytes;
    sv->peak_resident = std::max(sv->peak_resident, sv->resident);
    sv->admissions++;
    return CCFR_OK;
}

// Group the scenes into pools (once, before serving): scenes of at most
// pool_scene_max vertices whose settings agree except for r, xi, delta and
// pad (what a batched context allows to differ), in registration order, up to
// pool_max_verts vertices and 2048 scenes per pool.
void form_pools(ccfr_server* sv) {
    if (sv->pools_formed || sv->pool_max_verts <= 0) return;
    sv->pools_formed = true;
    auto signature = [](ccfr_params q) {
        q.r = q.xi = q.delta = q.pad = 0.f;
        return q;
    };
    std::vector<int> open_pool;             // the pool taking members, per signature
    std::vector<ccfr_params> open_sig;
    for (int k = 0; k < (int)sv->scenes.size(); ++k) {
        SceneRec& sc = sv->scenes[k];
        if (sc.n_verts > sv->pool_scene_max || sc.n_verts > sv->pool_max_verts) continue;
        const ccfr_params sig = signature(sc.params);
        int i = 0;
        while (i < (int)open_sig.size() && std::memcmp(&open_sig[i], &sig, sizeof(sig)) != 0) ++i;
        if (i < (int)open_sig.size()) {
            const Pool& P = sv->pools[open_pool[i]];
            if (P.voff.back() + sc.n_verts > sv->pool_max_verts || P.members.size() >= 2048) {
                open_pool.erase(open_pool.begin() + i);
                open_sig.erase(open_sig.begin() + i);
                i = (int)open_sig.size();
            }
        }
        if (i == (int)open_sig.size()) {
            sv->pools.emplace_back();
            sv->pools.back().voff.push_back(0);
            open_pool.push_back((int)sv->pools.size() - 1);
            open_sig.push_back(sig);
        }
        const int p = open_pool[i];
        Pool& P = sv->pools[p];
        sc.pool = p;
        sc.member = (int)P.members.size();
        P.members.push_back(k);
        P.voff.push_back(P.voff.back() + sc.n_verts);
    }
    for (Pool& P : sv->pools) {
        long ne = 0, nt = 0;
        int K = 0, pc = 0;
        bool phi = false;
        for (int k : P.members) {
            const SceneRec& sc = sv->scenes[k];
            ne += sc.n_edges;
            nt += sc.n_tris;
            K = sc.params.plane_capacity;
            pc = sc.params.pair_capacity;
            phi = sc.params.delta > 0.f;
        }
        const long nv = P.voff.back();
        P.bytes = ctx_bytes(nv, ne, nt, K, false, phi, pc) + (size_t)nv * 2 + P.members.size() * 20;
        P.hmask.assign(P.members.size(), 0);
    }
}

// Make scene s resident (served alone); evict idle units if needed.  Called
// by the worker.
ccfr_status admit(ccfr_server* sv, int s) {
    SceneRec& sc = sv->scenes[s];
    if (sc.ctx) return CCFR_OK;
    ccfr_status rs = make_room(sv, sc.bytes);
    if (rs != CCFR_OK) return rs;
    int *de = nullptr, *dt = nullptr;
    float* dr = nullptr;
    size_t nb = (size_t)sc.n_verts * 4 * sizeof(float);
    cudaError_t err = cudaMalloc((void**)&dr, nb ? nb : 16);
    if (err == cudaSuccess) err = cudaMemcpy(dr, sc.rest.data(), nb, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && sc.n_edges) err = cudaMalloc((void**)&de, sc.edges.size() * sizeof(int));
    if (err == cudaSuccess && sc.n_tris) err = cudaMalloc((void**)&dt, sc.tris.size() * sizeof(int));
    if (err == cudaSuccess) err = cudaMalloc((void**)&sc.dx, nb ? nb : 16);
    if (err == cudaSuccess) err = cudaMalloc((void**)&sc.dv, nb ? nb : 16);
    if (err == cudaSuccess && sc.n_edges) err = cudaMemcpy(de, sc.edges.data(), sc.edges.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (err == cudaSuccess && sc.n_tris) err = cudaMemcpy(dt, sc.tris.data(), sc.tris.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(sc.dx, sc.x.data(), nb, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(sc.dv, sc.v.data(), nb, cudaMemcpyHostToDevice);
    ccfr_status st = CCFR_OK;
    if (err == cudaSuccess) {
        // rest lengths always from the rest shape given at registration
        ccfr_mesh m{sc.n_verts, sc.n_edges, sc.n_tris, de, dt, dr};
        st = ccfr_create(&m, &sc.params, nullptr, &sc.ctx);
    }
    cudaFree(de);
    cudaFree(dt);
    cudaFree(dr);
    if (err != cudaSuccess || st != CCFR_OK) {
        cudaGetLastError();
        cudaFree(sc.dx);
        cudaFree(sc.dv);
        sc.dx = sc.dv = nullptr;
        sc.ctx = nullptr;
        return st != CCFR_OK ? st : CCFR_ERR_OOM;
    }
    sv->resident += sc.bytes;
    sv->peak_resident = std::max(sv->peak_resident, sv->resident);
    sv->admissions++;
    return CCFR_OK;
}

void finish(ccfr_server* sv, Slot& sl, double t, int status) {
    Req& r = sv->reqs[sl.req];
    r.t_done = t - sv->t0;
    if (r.status != CCFR_ERR_TIMEOUT) r.status = status;
    else status = CCFR_ERR_TIMEOUT;
    SceneRec& sc = sv->scenes[r.scene];
    sc.busy = false;
    sc.last_used = t;
    if (status == CCFR_OK) sc.steps_done++;
    else sv->failed++;
    sv->n_done++;
    sl.req = -1;
    sl.stalled = false;
}

// All requests of a pool launch are done (or failed together).
void finish_pool(ccfr_server* sv, Slot& sl, double t, int status) {
    Pool& P = sv->pools[sl.pool];
    for (long i : sl.preqs) {
        Req& r = sv->reqs[i];
        r.t_done = t - sv->t0;
        const int st = (r.status == CCFR_ERR_TIMEOUT) ? CCFR_ERR_TIMEOUT : status;
        r.status = st;
        SceneRec& sc = sv->scenes[r.scene];
        sc.last_used = t;
        if (st == CCFR_OK) sc.steps_done++;
        else sv->failed++;
        sv->n_done++;
    }
    P.busy = false;
    P.last_used = t;
    sl.pool = -1;
    sl.preqs.clear();
    sl.stalled = false;
}

// Launch pool p on slot sl: every member with a request due now takes its
// oldest one (one step per scene and launch, in arrival order per scene).
void launch_pool(ccfr_server* sv, Slot& sl, int p, double rel, double t) {
    Pool& P = sv->pools[p];
    std::fill(P.hmask.begin(), P.hmask.end(), (unsigned char)0);
    sl.preqs.clear();
    for (long i = sv->scan_from; i < (long)sv->reqs.size(); ++i) {
        Req& q = sv->reqs[i];
        if (q.t_arrival > rel) break;
        if (q.t_start >= 0.0) continue;
        const SceneRec& sc = sv->scenes[q.scene];
        if (sc.pool != p || P.hmask[sc.member]) continue;
        P.hmask[sc.member] = 1;
        q.t_start = rel;
        sl.preqs.push_back(i);
    }
    P.busy = true;
    sl.pool = p;
    sl.t_launch = t;
    sv->pool_launches++;
    // (a copy from pageable memory returns once the bytes are staged)
    cudaError_t e = cudaMemcpyAsync(P.dmask, P.hmask.data(), P.hmask.size(), cudaMemcpyHostToDevice, sl.stream);
    ccfr_status st = (e == cudaSuccess) ? ccfr_step_active(P.ctx, P.dx, P.dv, P.dmask, sl.stream) : CCFR_ERR_CUDA;
    if (st != CCFR_OK || cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
        finish_pool(sv, sl, now_s(), st ? st : CCFR_ERR_CUDA);
}

void worker_loop(ccfr_server* sv) {
    cudaSetDevice(sv->device);
    while (!sv->stop.load()) {
        bool active = false;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            const double t = now_s();
            for (Slot& sl : sv->slots) {
                if (!sl.busy()) continue;
                active = true;
                if (sl.stalled) {
                    if (t - sl.t_launch > sv->timeout) finish(sv, sl, t, CCFR_ERR_TIMEOUT);
                    continue;
                }
                cudaError_t q = cudaEventQuery(sl.done);
                const bool pool = sl.pool >= 0;
                if (q == cudaSuccess) {
                    if (pool) finish_pool(sv, sl, t, CCFR_OK);
                    else finish(sv, sl, t, CCFR_OK);
                } else if (q != cudaErrorNotReady) {
                    cudaGetLastError();
                    if (pool) finish_pool(sv, sl, t, CCFR_ERR_CUDA);
                    else finish(sv, sl, t, CCFR_ERR_CUDA);
                } else if (t - sl.t_launch > sv->timeout) {
                    // bounded wait: report the request(s); the slot stays closed until its
                    // work drains, so no later work is queued behind it
                    if (pool) {
                        for (long i : sl.preqs) sv->reqs[i].status = CCFR_ERR_TIMEOUT;
                    } else {
                        sv->reqs[sl.req].status = CCFR_ERR_TIMEOUT;
                    }
                }
            }
            const double rel = t - sv->t0;
            for (Slot& sl : sv->slots) {
                if (sl.busy()) continue;
                // earliest due request whose scene (or pool) is idle (first hit per scene = its oldest)
                long pick = -1;
                while (sv->scan_from < (long)sv->reqs.size() && sv->reqs[sv->scan_from].t_start >= 0.0) sv->scan_from++;
                for (long i = sv->scan_from; i < (long)sv->reqs.size(); ++i) {
                    Req& r = sv->reqs[i];
                    if (r.t_arrival > rel) break;
                    if (r.t_start >= 0.0) continue;
                    SceneRec& sc = sv->scenes[r.scene];
                    if (sc.pool >= 0) {
                        if (sv->pools[sc.pool].busy) continue;
                        if (admit_pool(sv, sc.pool) != CCFR_OK) continue;
                        pick = i;
                        break;
                    }
                    if (sc.busy) continue;
                    if (admit(sv, r.scene) != CCFR_OK) continue;
                    pick = i;
                    break;
                }
                if (pick < 0) break;
                Req& r = sv->reqs[pick];
                SceneRec& sc = sv->scenes[r.scene];
                if (sc.pool >= 0) {
                    launch_pool(sv, sl, sc.pool, rel, t);
                    active = true;
                    continue;
                }
                sc.busy = true;
                r.t_start = rel;
                sl.req = pick;
                sl.t_launch = t;
                active = true;
                if (sc.stall) { sl.stalled = true; continue; }
                ccfr_status st = ccfr_step(sc.ctx, sc.dx, sc.dv, sl.stream);
                if (st != CCFR_OK || cudaEventRecord(sl.done, sl.stream) != cudaSuccess) finish(sv, sl, now_s(), st ? st : CCFR_ERR_CUDA);
            }
            // requests due but not started keep the loop busy
            if (!active && sv->scan_from < (long)sv->reqs.size() && sv->reqs[sv->scan_from].t_arrival <= rel) active = true;
        }
        if (!active) std::this_thread::sleep_for(std::chrono::microseconds(50));
        else std::this_thread::yield();
    }
}

}  // namespace

extern "C" {

ccfr_status ccfr_server_create(size_t hbm_budget_bytes, int n_slots, double timeout_s, ccfr_server** out) {
    if (!out || n_slots < 1 || n_slots > 64 || !(timeout_s > 0.0)) return CCFR_ERR_INVALID_ARG;
    *out = nullptr;
    ccfr_server* sv = new (std::nothrow) ccfr_server();
    if (!sv) return CCFR_ERR_OOM;
    cudaGetDevice(&sv->device);
    sv->budget = hbm_budget_bytes;
    sv->timeout = timeout_s;
    sv->slots.resize(n_slots);
    for (Slot& sl : sv->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ccfr_server_destroy(sv);
            return CCFR_ERR_CUDA;
        }
    }
    *out = sv;
    return CCFR_OK;
}

ccfr_status ccfr_server_add_scene(ccfr_server* sv, int n_verts, int n_edges, int n_tris, const int* edges,
                                  const int* tris, const float* x, const float* v, const ccfr_params* params,
                                  int* scene_id) {
    if (!sv || !params || !scene_id || n_verts < 1 || n_edges < 0 || n_tris < 0 || !x || !v) return CCFR_ERR_INVALID_ARG;
    if ((n_edges && !edges) || (n_tris && !tris)) return CCFR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->running.load()) return CCFR_ERR_STATE;
    SceneRec sc;
    sc.n_verts = n_verts;
    sc.n_edges = n_edges;
    sc.n_tris = n_tris;
    sc.edges.assign(edges, edges + 2 * (size_t)n_edges);
    sc.tris.assign(tris, tris + 3 * (size_t)n_tris);
    sc.x.assign(x, x + 4 * (size_t)n_verts);
    sc.v.assign(v, v + 4 * (size_t)n_verts);
    sc.rest = sc.x;
    sc.params = *params;
    sc.params.flags &= ~(unsigned)CCFR_FLAG_STORE_KEYS;
    sc.bytes = ctx_bytes(n_verts, n_edges, n_tris, params->plane_capacity, false, params->delta > 0.f,
                         params->pair_capacity);
    if (sc.bytes > sv->budget) return CCFR_ERR_OOM;
    sv->scenes.push_back(std::move(sc));
    *scene_id = (int)sv->scenes.size() - 1;
    return CCFR_OK;
}

ccfr_status ccfr_server_submit(ccfr_server* sv, int scene_id, double t_arrival, long* request_id) {
    if (!sv || t_arrival < 0.0) return CCFR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (scene_id < 0 || scene_id >= (int)sv->scenes.size()) return CCFR_ERR_INVALID_ARG;
    if (!sv->reqs.empty() && t_arrival < sv->reqs.back().t_arrival) return CCFR_ERR_INVALID_ARG;   // arrival order
    Req r;
    r.scene = scene_id;
    r.t_arrival = t_arrival;
    sv->reqs.push_back(r);
    if (request_id) *request_id = (long)sv->reqs.size() - 1;
    return CCFR_OK;
}

ccfr_status ccfr_server_preload(ccfr_server* sv, double fraction, int* n_admitted) {
    if (!sv || !(fraction > 0.0) || fraction > 1.0) return CCFR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->running.load()) return CCFR_ERR_STATE;
    form_pools(sv);
    int n = 0;
    for (int k = 0; k < (int)sv->scenes.size(); ++k) {
        SceneRec& sc = sv->scenes[k];
        if (sc.pool >= 0) {
            Pool& P = sv->pools[sc.pool];
            if (P.ctx || (double)(sv->resident + P.bytes) > fraction * (double)sv->budget) continue;
            ccfr_status st = admit_pool(sv, sc.pool);
            if (st != CCFR_OK) return st;
            n += (int)P.members.size();
            continue;
        }
        if (sc.ctx) continue;
        if ((double)(sv->resident + sc.bytes) > fraction * (double)sv->budget) continue;
        ccfr_status st = admit(sv, k);
        if (st != CCFR_OK) return st;
        ++n;
    }
    if (n_admitted) *n_admitted = n;
    return CCFR_OK;
}

ccfr_status ccfr_server_set_batching(ccfr_server* sv, int max_pool_verts, int max_scene_verts) {
    if (!sv || max_pool_verts < 0 || max_scene_verts < 0) return CCFR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->running.load() || sv->pools_formed) return CCFR_ERR_STATE;
    sv->pool_max_verts = max_pool_verts;
    sv->pool_scene_max = max_scene_verts;
    return CCFR_OK;
}

ccfr_status ccfr_server_start(ccfr_server* sv) {
    if (!sv) return CCFR_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        form_pools(sv);
    }
    if (sv->running.exchange(true)) return CCFR_ERR_STATE;
    sv->t0 = now_s();
    sv->stop = false;
    sv->worker = std::thread(worker_loop, sv);
    return CCFR_OK;
}

ccfr_status ccfr_server_wait(ccfr_server* sv, double timeout_s, long* n_done) {
    if (!sv) return CCFR_ERR_INVALID_ARG;
    const double t_end = now_s() + timeout_s;
    for (;;) {
        long done, total;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            done = sv->n_done;
            total = (long)sv->reqs.size();
        }
        if (n_done) *n_done = done;
        if (done >= total) return CCFR_OK;
        if (now_s() > t_end) return CCFR_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

ccfr_status ccfr_server_stop(ccfr_server* sv) {
    if (!sv) return CCFR_ERR_INVALID_ARG;
    if (sv->running.load()) {
        sv->stop = true;
        if (sv->worker.joinable()) sv->worker.join();
        sv->running = false;
    }
    return CCFR_OK;
}

ccfr_status ccfr_server_results(ccfr_server* sv, long n, double* t_arrival, double* t_start, double* t_done,
                                int* status) {
    if (!sv || n < 0) return CCFR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (n > (long)sv->reqs.size()) return CCFR_ERR_INVALID_ARG;
    for (long i = 0; i < n; ++i) {
        const Req& r = sv->reqs[i];
        if (t_arrival) t_arrival[i] = r.t_arrival;
        if (t_start) t_start[i] = r.t_start;
        if (t_done) t_done[i] = r.t_done;
        if (status) status[i] = r.status;
    }
    return CCFR_OK;
}

ccfr_status ccfr_server_get_state(ccfr_server* sv, int scene_id, float* x, float* v) {
    if (!sv || !x || !v) return CCFR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (scene_id < 0 || scene_id >= (int)sv->scenes.size()) return CCFR_ERR_INVALID_ARG;
    SceneRec& sc = sv->scenes[scene_id];
    if (sc.busy) return CCFR_ERR_STATE;
    size_t nb = (size_t)sc.n_verts * 4 * sizeof(float);
    if (sc.pool >= 0) {
        const Pool& P = sv->pools[sc.pool];
        if (P.busy) return CCFR_ERR_STATE;
        if (P.ctx) {
            const size_t vo = (size_t)P.voff[sc.member] * 4;
            if (cudaMemcpy(x, P.dx + vo, nb, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(v, P.dv + vo, nb, cudaMemcpyDeviceToHost) != cudaSuccess)
                return CCFR_ERR_CUDA;
            return CCFR_OK;
        }
    }
    if (sc.ctx) {
        if (cudaMemcpy(x, sc.dx, nb, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(v, sc.dv, nb, cudaMemcpyDeviceToHost) != cudaSuccess)
            return CCFR_ERR_CUDA;
    } else {
        std::memcpy(x, sc.x.data(), nb);
        std::memcpy(v, sc.v.data(), nb);
    }
    return CCFR_OK;
}

ccfr_status ccfr_server_get_info(ccfr_server* sv, ccfr_server_info* out) {
    if (!sv || !out) return CCFR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    out->scenes = (long)sv->scenes.size();
    out->requests = (long)sv->reqs.size();
    out->done = sv->n_done;
    out->failed = sv->failed;
    out->admissions = sv->admissions;
    out->evictions = sv->evictions;
    out->resident_bytes = sv->resident;
    out->peak_resident_bytes = sv->peak_resident;
    out->budget_bytes = sv->budget;
    out->pools = (long)sv->pools.size();
    out->pool_launches = sv->pool_launches;
    return CCFR_OK;
}

ccfr_status ccfr_estimate_bytes(int n_verts, int n_edges, int n_tris, int plane_capacity, size_t* bytes) {
    if (!bytes || n_verts < 0 || n_edges < 0 || n_tris < 0 || plane_capacity < 1) return CCFR_ERR_INVALID_ARG;
    *bytes = ctx_bytes(n_verts, n_edges, n_tris, plane_capacity, false);
    return CCFR_OK;
}

ccfr_status ccfr_server_set_stall(ccfr_server* sv, int scene_id, int stall) {
    if (!sv) return CCFR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (scene_id < 0 || scene_id >= (int)sv->scenes.size()) return CCFR_ERR_INVALID_ARG;
    sv->scenes[scene_id].stall = stall != 0;
    return CCFR_OK;
}

ccfr_status ccfr_server_destroy(ccfr_server* sv) {
    if (!sv) return CCFR_ERR_INVALID_ARG;
    ccfr_server_stop(sv);
    for (Slot& sl : sv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    }
    for (SceneRec& sc : sv->scenes) {
        if (sc.ctx) ccfr_destroy(sc.ctx);
        cudaFree(sc.dx);
        cudaFree(sc.dv);
    }
    for (Pool& P : sv->pools) {
        if (P.ctx) ccfr_destroy(P.ctx);
        cudaFree(P.dx);
        cudaFree(P.dv);
        cudaFree(P.dmask);
    }
    for (Slot& sl : sv->slots) {
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete sv;
    return CCFR_OK;
}

}  // extern "C"

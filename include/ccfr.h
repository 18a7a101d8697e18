/*
 * ccfr.h - C ABI of the B300 (sm_103a) implementation of Convex Collision-Free
 * Regions (CCFR): per-vertex convex regions built from nearby vertex-face,
 * edge-edge and point-point pairs (and point-edge pairs in mixed scenes, see
 * ccfr_mesh_ext), projection of XPBD iterates into them, and the XPBD substep
 * that runs both inside every solver iteration.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Positions are float4 records (x, y, z, w) laid out as 4 consecutive
 *    floats per vertex, 16-byte aligned; w is the vertex's inverse mass
 *    (0 = static obstacle vertex).  Velocities use the same layout (w unused).
 *  - Pointers documented as "device" must be CUDA device (or managed) memory of
 *    the device that was current at ccfr_create; "host" pointers are ordinary
 *    host memory.  The caller owns every buffer it passes in.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    enqueue work on it and return without synchronising, except where noted.
 *  - Host-detectable errors are returned at once and leave the context
 *    unchanged.  Conditions found on the device (non-finite input, plane-list
 *    overflow) are recorded in the context and reported by ccfr_get_stats.
 *  - Nothing in this library traps or aborts; no call waits without a bound.
 *  - A context is not thread-safe: calls on one context must be serialised by
 *    the caller.  Distinct contexts are independent.
 *
 * Citations refer to the paper "Convex Collision-Free Regions" (sections,
 * equations and algorithms).
 */
#ifndef CCFR_H
#define CCFR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CCFR_OK = 0,
    CCFR_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or parameter   */
    CCFR_ERR_CAPACITY = 2,      /* an output buffer given by the caller is too small */
    CCFR_ERR_OOM = 3,           /* device allocation failed in ccfr_create     */
    CCFR_ERR_CUDA = 4,          /* a CUDA runtime call failed                   */
    CCFR_ERR_TIMEOUT = 5,       /* a bounded wait gave up                       */
    CCFR_ERR_NONFINITE = 6,     /* a position or velocity was NaN or infinite   */
    CCFR_ERR_STATE = 7          /* call out of order (e.g. project before build) */
} ccfr_status;

/* Option bits of ccfr_params.flags. */
enum {
    CCFR_FLAG_STORE_KEYS = 1u << 0,  /* store each plane's pair key (tests, tooling) */
    CCFR_FLAG_EARLY_EXIT = 1u << 1,  /* stop the iteration loop once converged (Alg. 4) */
    CCFR_FLAG_NO_GRAPH = 1u << 2     /* launch ccfr_step kernel by kernel, no CUDA graph */
};

/* Parameters of one scene (paper Table 3 and Sec. 3.2, 4.1; Alg. 2, 4). */
typedef struct {
    float r;              /* search radius: pairs with gap phi < 2r form planes (Sec. 3.1), and
                             the max step per iteration (Alg. 4)                          */
    float xi;             /* offset / minimum separation (Eq. 2)                          */
    float delta;          /* repulsion range of the soft response; enlarges the AABB pad  */
    float pad;            /* AABB enlargement r + xi/2 + delta/2 (Sec. 4.1), binary32     */
    float eps_retract;    /* retraction margin eps (Sec. 3.2), scene units               */
    float eps_dep;        /* dependence tolerance of Alg. 1                               */
    float tau_feas;       /* tolerance of the final feasibility check                     */
    int max_passes;       /* n_maxIterations of Alg. 2; n_max + 1 passes are run          */
    int solver_iters;     /* solver iterations of Alg. 4                                  */
    int plane_capacity;   /* planes kept per vertex (K); must be a multiple of 32, >= 32  */
    float cell_size;      /* uniform-grid cell size; 0 = cell_factor x mean padded extent */
    float cell_factor;    /* cell size in mean padded primitive extents; 0 = 1.5          */
    float dt;             /* substep (Alg. 4)                                              */
    float gravity[3];
    float compliance;     /* XPBD compliance of the edge-distance constraints             */
    unsigned flags;       /* CCFR_FLAG_*                                                   */
    /* Contact response and friction (Sec. 3.3), active when delta > 0: the
     * energy (k/2) w_c max(0, delta - g_c)^2 per contact as an XPBD constraint
     * of compliance 1/(k w_c), w_c the smooth occlusion weight of transition
     * width delta_v, then position-based static / kinetic friction.  Needs 4
     * more bytes per plane slot (each plane's gap). */
    float response_stiffness;  /* k (>= 0)                                                */
    float delta_v;        /* occlusion transition width (> 0 when delta > 0)             */
    float mu_s, mu_k;     /* static and kinetic friction coefficients (>= 0)             */
    /* Candidate pairs buffered between the broad and the narrow kernels of
     * the region build (Alg. 3): the vertex-face and oversized-primitive
     * buffer holds pair_capacity x (triangles + edges) pairs, the edge-edge
     * buffer 3 x pair_capacity x edges (plus 4096 each); 8 bytes a pair.
     * 0 = 32.  A kind whose pairs overflow a buffer is redone by a fused
     * kernel: the result is the same, only slower (stats aux[15]). */
    int pair_capacity;
} ccfr_params;

/* Topology of one scene.  All arrays are device pointers, read at ccfr_create
 * only (copied into the context). */
typedef struct {
    int n_verts, n_edges, n_tris;
    const int* edges;      /* n_edges x 2, each (a, b) with a < b, sorted lexicographically,
                              unique: the unique edges of the triangles plus polyline edges */
    const int* tris;       /* n_tris x 3 vertex ids (may be NULL when n_tris == 0)         */
    const float* rest_x;   /* n_verts x 4 rest positions; edge rest lengths are taken from
                              them (may be NULL: rest lengths from the first step's x)      */
} ccfr_mesh;

/* A scene that mixes rods, cloth, volumes and particles in one simulation (the
 * coupled codimensional scene of Sec. 5): the collision topology of ccfr_mesh
 * plus XPBD constraints that are no collision primitives.  Alg. 4 solves "a
 * set of XPBD constraints" without naming them; this library takes
 *  - links: extra distance constraints (bending: the two vertices opposite an
 *    interior cloth edge, every second rod neighbour; the inner edges of
 *    tetrahedral volumes), each with its own compliance, rest lengths from
 *    rest_x;
 *  - tetrahedra: volume constraints C = 6 V - 6 V0, with 6 V = (x1 - x0) .
 *    ((x2 - x0) x (x3 - x0)) signed and V0 from rest_x, one compliance.
 * Each iteration sweeps the distance constraints (the edges in canonical
 * order, then the links, coloured together first-fit, colours ascending) and
 * then the tetrahedra (coloured first-fit in their order).  A vertex that
 * belongs to links or tetrahedra only (the inside of a volume) takes no part
 * in collision; the isolated points (no edge, link or tetrahedron) meet the
 * free edges (edges of no triangle, i.e. rods) through point-edge pairs, which
 * Alg. 3 lacks.  Arrays are device pointers (or host memory), read at
 * ccfr_create_ext only. */
typedef struct {
    ccfr_mesh mesh;                /* collision topology, as for ccfr_create          */
    int n_links;
    const int* links;              /* n_links x 2 vertex ids, a != b                   */
    const float* link_compliance;  /* n_links compliances (>= 0), XPBD alpha            */
    int n_tets;
    const int* tets;               /* n_tets x 4 distinct vertex ids                    */
    float volume_compliance;       /* compliance of every volume constraint (>= 0)      */
} ccfr_mesh_ext;

/* Counters accumulated since the last ccfr_reset_stats (device-side, read by
 * ccfr_get_stats).  Per-iteration quantities are summed over iterations. */
typedef struct {
    unsigned long long cand_vf, cand_ee, cand_vv;     /* broad-phase candidates         */
    unsigned long long pairs_vf, pairs_ee, pairs_vv;  /* accepted pairs (phi < 2r)      */
    unsigned long long planes_vf, planes_ee, planes_vv; /* planes emitted per pair kind  */
    unsigned long long planes;                        /* planes seen by the projection  */
    unsigned long long overflow_verts;                /* vertices over the capacity     */
    unsigned long long violated_verts;                /* vertices with a violated plane */
    unsigned long long halts;                         /* vertices reset to x (Alg. 2)   */
    unsigned long long ee_fp64;                       /* near-parallel EE solved in FP64 */
    unsigned long long feas_fp64;                     /* final checks decided in FP64   */
    unsigned long long feas_halts;                    /* halts caused by the final check */
    unsigned long long iterations;                    /* solver iterations executed     */
    unsigned long long steps;                         /* ccfr_step calls                */
    unsigned long long aux[16];                       /* diagnostics: [0] projection passes
                                                         of the group-per-vertex walk (long
                                                         lists), [1] passes of the thread-per-
                                                         vertex walk (short lists), [2]
                                                         violated planes visited until Alg. 1
                                                         holds three lines, [3] oversized
                                                         triangles, [4] oversized edges, [5]
                                                         zero, [6] planes of the violated
                                                         vertices with long lists, [7] zero, [8]
                                                         violated vertices with short lists,
                                                         [9] their planes, [10] grid cells
                                                         scanned for oversized primitives,
                                                         [11] their whole-table scans, [12]
                                                         items they tested, [13] oversized-
                                                         edge items tested by oversized
                                                         edges, [14] candidates found by
                                                         oversized primitives, [15] kinds
                                                         whose oversized pairs overflowed
                                                         the pair buffer (redone by the
                                                         fused pass; time only)           */
    unsigned int max_planes;                          /* largest per-vertex plane count */
    unsigned int error_flags;                         /* bit 0 non-finite input         */
    unsigned long long cand_ve, pairs_ve, planes_ve;  /* point-edge pairs (ccfr_mesh_ext):
                                                         candidates, accepted, planes   */
} ccfr_stats;

typedef struct ccfr_ctx ccfr_ctx;

/* Create a context for one scene: copies the topology, computes edge
 * colours and rest lengths, and allocates every workspace (grid, plane lists,
 * multipliers).  No later call allocates device memory.  `stream` orders the
 * set-up copies.  On failure *out is NULL. */
ccfr_status ccfr_create(const ccfr_mesh* mesh, const ccfr_params* params, void* stream, ccfr_ctx** out);

/* ccfr_create for a scene with links and tetrahedra (ccfr_mesh_ext above):
 * the same context, whose substep also sweeps those constraints and whose
 * region build adds the point-edge pairs.  Errors: CCFR_ERR_INVALID_ARG for a
 * vertex id out of range, a link with equal ends or a negative compliance, a
 * tetrahedron with a repeated vertex, more than 64 colours; otherwise as
 * ccfr_create. */
ccfr_status ccfr_create_ext(const ccfr_mesh_ext* mesh, const ccfr_params* params, void* stream, ccfr_ctx** out);

/* Release the context and all its device memory (synchronises the context's work). */
ccfr_status ccfr_destroy(ccfr_ctx* ctx);

/* Build every vertex's convex region at the collision-free configuration x
 * (device, n_verts x 4): broad phase (uniform-grid spatial hash), narrow phase
 * (Alg. 3 over all VF, EE and point-point pairs; contact normal Eq. 1,
 * half-space Eq. 2-3), compaction into per-vertex lists of at most
 * plane_capacity planes (n, d) with (x' - x) . n + d >= 0.  A vertex that
 * receives more planes than the capacity is marked overflowed: projection
 * then bounds its step by max(0, min d) instead.  The regions stay in the
 * context for ccfr_project and ccfr_copy_regions. */
ccfr_status ccfr_build_regions(ccfr_ctx* ctx, const float* x, void* stream);

/* Project candidate positions into the regions of the last build
 * (Alg. 2 calling Alg. 1, with the retraction and halt of Sec. 3.2, and a
 * final feasibility check).  x: device, the build positions; x_io: device,
 * in = candidates x', out = projected x* (w untouched).  halt_out: optional
 * device array of n_verts bytes, 1 where the vertex was reset to x.
 * Returns CCFR_ERR_STATE when no region has been built. */
ccfr_status ccfr_project(ccfr_ctx* ctx, const float* x, float* x_io, unsigned char* halt_out, void* stream);

/* One XPBD substep (Alg. 4): predict, then solver_iters iterations of
 * {build regions at x_c, restart from the prediction, XPBD edge sweep,
 * project, clamp the step to r, convergence test}, then the implicit-Euler
 * update.  x, v: device, n_verts x 4, updated in place.  The iteration loop is
 * recorded once per (x, v) pair as a CUDA graph and replayed (unless
 * CCFR_FLAG_NO_GRAPH). */
ccfr_status ccfr_step(ccfr_ctx* ctx, float* x, float* v, void* stream);

/* Number of stages reported by ccfr_step_timed. */
#define CCFR_N_STAGES 17

/* ccfr_step launched kernel by kernel with CUDA events between the stages
 * (prediction, grid extent, grid count, grid scan, grid scatter, vertex-face
 * narrow phase, edge-edge narrow phase, point-point narrow phase, XPBD sweep,
 * projection scan, bookkeeping, work units, oversized vertex-face and
 * edge-edge passes, projection of the violated vertices with long and with
 * short plane lists, contact response): the per-stage split of the paper's timing table
 * (Table 1: broad, narrow, resolution, XPBD).  stage_ms (host, n_stages >=
 * CCFR_N_STAGES doubles) receives milliseconds summed over the iterations.
 * Synchronises `stream`. */
ccfr_status ccfr_step_timed(ccfr_ctx* ctx, float* x, float* v, double* stage_ms, int n_stages, void* stream);

/* Name of stage i of ccfr_step_timed (static string; "" when out of range). */
const char* ccfr_stage_name(int i);

/* ccfr_step launched kernel by kernel (the same kernels in the same order),
 * recording the substep's intermediate states for tests and tooling: the
 * prediction x~ = x + dt v + dt^2 g of Alg. 4 into x_tilde_out (device,
 * n_verts x 4 floats, or NULL) and, after every solver iteration i, the
 * collision-free iterate x_c into iterates_out + i * n_verts * 4 (device,
 * solver_iters x n_verts x 4 floats, or NULL).  x and v are updated as by
 * ccfr_step.  Both outputs must be 16-byte aligned. */
ccfr_status ccfr_step_record(ccfr_ctx* ctx, float* x, float* v, float* x_tilde_out, float* iterates_out,
                             void* stream);

/* ccfr_step on host buffers: copies x and v (host, n_verts x 4 floats each,
 * preferably pinned) to the context's device buffers, steps, copies them back,
 * and synchronises `stream` before returning. */
ccfr_status ccfr_step_host(ccfr_ctx* ctx, float* x_host, float* v_host, void* stream);

/* Candidate pairs of the broad phase at x (device): vertex-face (v, t),
 * edge-edge (e, f) with e < f, and point-point (p, q) with p < q, written as
 * int pairs into the device arrays vf, ee, vv (capacities in pairs).  The
 * order inside each list is unspecified.  Counts are written to the host
 * array counts[3] after the call synchronises `stream`; if any count exceeds
 * its capacity, CCFR_ERR_CAPACITY is returned and the lists are truncated. */
ccfr_status ccfr_get_candidates(ccfr_ctx* ctx, const float* x, int* vf, long cap_vf, int* ee, long cap_ee,
                                int* vv, long cap_vv, long* counts, void* stream);

/* Copy the current regions out: planes (device, n_verts * capacity * 4 floats,
 * vertex-major: slot j of vertex v at [(v*capacity + j)*4]), keys (device,
 * n_verts * capacity u64, or NULL; valid only with CCFR_FLAG_STORE_KEYS),
 * count (device, n_verts ints: planes received, may exceed capacity),
 * dmin_drop (device, n_verts floats: smallest d among planes beyond the
 * capacity, +inf if none; or NULL). */
ccfr_status ccfr_copy_regions(ccfr_ctx* ctx, float* planes, unsigned long long* keys, int* count,
                              float* dmin_drop, void* stream);

/* Replace the current regions with caller-provided ones (same layout as
 * ccfr_copy_regions, `capacity` slots per vertex, capacity <= the context's).
 * Used to feed externally built regions to ccfr_project. */
ccfr_status ccfr_load_regions(ccfr_ctx* ctx, const float* planes, const int* count, int capacity, void* stream);

/* Projection that allocates nothing, for callers that cannot allocate device
 * memory: a caller whose memory is fully owned by another allocator or
 * budget (a host engine or plug-in that hands this library fixed buffers),
 * or a caller on a path where cudaMalloc is not permitted.  (The paper has no
 * counterpart; this is an interface of this library.)
 *
 * Same computation as ccfr_project (Alg. 2 with Alg. 1, retraction, halt,
 * final check) on regions the caller holds, in the layout of
 * ccfr_copy_regions: planes (device, n_verts * capacity float4, vertex-major),
 * count (device, n_verts ints), dmin_drop (device, n_verts floats, +inf =
 * none; or NULL when no vertex has more than `capacity` planes).  x: device,
 * build positions; x_io: device, candidates in, projected positions out;
 * halt_out: optional device bytes.  params: r, eps_retract, eps_dep, tau_feas
 * and max_passes are used.
 *
 * Scratch: a file-scope device array sized for n_verts <= 262,144 (about
 * 5 MB on every GPU that loads the library, held until the process exits).
 * Larger n_verts is rejected with CCFR_ERR_INVALID_ARG.  The first call on a
 * device, with that device current, looks up the array's device address and
 * sets the kernels' shared-memory limit; make that first call before any
 * stream capture.  Every call shares the one array and clears what must start
 * at zero, so calls that overlap on the GPU (other streams, other threads)
 * race: serialise them.  No call allocates or frees device memory. */
ccfr_status ccfr_project_static(const float* x, float* x_io, const float* planes, const int* count,
                                const float* dmin_drop, int n_verts, int capacity, const ccfr_params* params,
                                unsigned char* halt_out, void* stream);

/* A context for several independent scenes stepped together (batched step).
 * meshes[k] / params[k] describe scene k with scene-local vertex ids; the
 * context numbers the vertices of scene k after those of scenes 0..k-1, so x
 * and v passed to ccfr_step hold all scenes one after another.  rest_x is
 * required for every scene.  Pairs never cross scenes; r, xi, delta and pad
 * are per scene, everything else (dt, gravity, iterations, projection
 * settings, capacity, flags) must be equal across scenes.  At most 2048
 * scenes.  Each scene's result equals its result in a context of its own. */
ccfr_status ccfr_create_batch(const ccfr_mesh* meshes, const ccfr_params* params, int n_scenes, void* stream,
                              ccfr_ctx** out);

/* One substep of a batched context in which only the scenes whose byte in
 * `active` (device, n_scenes bytes, scene order of ccfr_create_batch) is
 * nonzero advance; the others keep their positions and velocities bitwise.
 * Each active scene's result equals ccfr_step of that scene alone.  (A serving
 * loop steps the scenes that have a request due in one launch.)  Returns
 * CCFR_ERR_INVALID_ARG for a context not made by ccfr_create_batch. */
ccfr_status ccfr_step_active(ccfr_ctx* ctx, float* x, float* v, const unsigned char* active, void* stream);

/* Performance knobs: grid cell size in mean padded primitive extents and
 * emission blocks per SM (no effect on results), and plane capacity (a
 * multiple of 32; changing it reallocates the plane lists; results change
 * only for vertices that receive more planes than the capacity, whose step
 * is then bounded by the overflow rule).  0 keeps a setting. */
typedef struct {
    float cell_factor;
    int emit_blocks_per_sm;
    int plane_capacity;
} ccfr_tuning;

/* Apply tuning (synchronises the device; drops recorded step graphs). */
ccfr_status ccfr_set_tuning(ccfr_ctx* ctx, const ccfr_tuning* t);
ccfr_status ccfr_get_tuning(const ccfr_ctx* ctx, ccfr_tuning* t);

/* Autotuner: sets the plane capacity (best->plane_capacity on input: 0 =
 * choose 1.5x the largest per-vertex plane count at x, +32; otherwise keep
 * that value), then times `steps` substeps from a scratch copy of
 * (x, v) for every cell factor in {1, 1.5, 2, 3} and emission grid in {4, 8,
 * 16} blocks per SM, and keeps the fastest.  x, v (device) are not modified.
 * Allocates two scratch vectors for the duration of the call.  best receives
 * the chosen tuning, best_ms (optional) its time per substep. */
ccfr_status ccfr_autotune(ccfr_ctx* ctx, const float* x, const float* v, int steps, ccfr_tuning* best,
                          double* best_ms, void* stream);

/* ---------------------------------------------------------------- Serving
 * A server takes step requests for registered scenes as they arrive, keeps
 * admitted scenes' state on the device, admits scenes within an HBM budget
 * (evicting idle scenes, least recently used first, to the host), and runs
 * up to n_slots steps of different scenes at once on separate streams, so
 * the work of requests that arrive while others run overlaps on the device.
 * Requests of one scene run in arrival order.  Each request is one
 * ccfr_step; a scene's results are the same whatever else is served.
 * Waits are bounded by timeout_s (a step that does not finish in time is
 * reported as CCFR_ERR_TIMEOUT).  The server allocates device memory when it
 * admits a scene.  Calls are thread-safe. */
typedef struct ccfr_server ccfr_server;

typedef struct {
    long scenes, requests, done, failed, admissions, evictions;
    size_t resident_bytes, peak_resident_bytes, budget_bytes;
    long pools, pool_launches;     /* batching: pools formed, batched launches issued */
} ccfr_server_info;

ccfr_status ccfr_server_create(size_t hbm_budget_bytes, int n_slots, double timeout_s, ccfr_server** out);
/* Register a scene (host arrays, copied; x is also the rest shape).  Only
 * before ccfr_server_start.  CCFR_ERR_OOM if the scene alone exceeds the budget. */
ccfr_status ccfr_server_add_scene(ccfr_server* sv, int n_verts, int n_edges, int n_tris, const int* edges,
                                  const int* tris, const float* x, const float* v, const ccfr_params* params,
                                  int* scene_id);
/* Queue one step of a scene, due t_arrival seconds after ccfr_server_start
 * (non-decreasing across calls).  May be called before or after start. */
ccfr_status ccfr_server_submit(ccfr_server* sv, int scene_id, double t_arrival, long* request_id);
/* Before start: admit registered scenes, in order, while the resident bytes
 * stay within `fraction` of the budget (first requests then skip admission). */
ccfr_status ccfr_server_preload(ccfr_server* sv, double fraction, int* n_admitted);
/* Continuous batching (before ccfr_server_start or _preload): scenes of at
 * most max_scene_verts vertices whose settings agree except for r, xi, delta
 * and pad are grouped, in registration order, into pools of at most
 * max_pool_verts vertices (and 2048 scenes), each resident as one batched
 * context (ccfr_create_batch) and admitted or evicted as a unit.  A pool's
 * launch steps, in one graph-captured substep (ccfr_step_active), every member
 * with a request due when the launch starts (its oldest one); requests that
 * arrive while the pool is on the GPU join its next launch.  Larger scenes are
 * served alone as before.  Results are those of ccfr_step alone.  The stall
 * test hook applies to scenes served alone.  0 vertices: no batching. */
ccfr_status ccfr_server_set_batching(ccfr_server* sv, int max_pool_verts, int max_scene_verts);
ccfr_status ccfr_server_start(ccfr_server* sv);
/* Wait (at most timeout_s) until every submitted request is done. */
ccfr_status ccfr_server_wait(ccfr_server* sv, double timeout_s, long* n_done);
/* Per request (first n): arrival, start and completion times (s, since
 * start; -1 if not reached) and status (-1 pending). */
ccfr_status ccfr_server_results(ccfr_server* sv, long n, double* t_arrival, double* t_start, double* t_done,
                                int* status);
/* Current state of a scene (host arrays, n_verts x 4 floats each). */
ccfr_status ccfr_server_get_state(ccfr_server* sv, int scene_id, float* x, float* v);
ccfr_status ccfr_server_get_info(ccfr_server* sv, ccfr_server_info* out);
/* Device bytes a resident scene takes (context, plane lists, candidate-pair
 * buffers at the default pair_capacity, state), the amount the server charges
 * against its budget for a scene with that capacity. */
ccfr_status ccfr_estimate_bytes(int n_verts, int n_edges, int n_tris, int plane_capacity, size_t* bytes);
/* Test hook: steps of the scene are treated as never finishing (no GPU work
 * is issued), to exercise the bounded wait. */
ccfr_status ccfr_server_set_stall(ccfr_server* sv, int scene_id, int stall);
ccfr_status ccfr_server_stop(ccfr_server* sv);
ccfr_status ccfr_server_destroy(ccfr_server* sv);

/* Context geometry: n_verts, plane capacity, number of edge colours. */
ccfr_status ccfr_get_info(const ccfr_ctx* ctx, int* n_verts, int* capacity, int* n_colors);

/* Synchronise the context's pending work and read the counters. */
ccfr_status ccfr_get_stats(ccfr_ctx* ctx, ccfr_stats* out);

/* Zero the counters (enqueued on `stream`). */
ccfr_status ccfr_reset_stats(ccfr_ctx* ctx, void* stream);

/* Human-readable name of a status code (static string). */
const char* ccfr_status_string(ccfr_status s);

#ifdef __cplusplus
}
#endif

#endif /* CCFR_H */

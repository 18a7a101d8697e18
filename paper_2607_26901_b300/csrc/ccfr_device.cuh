// Device-side data structures and helpers of the CCFR library (sm_103a).
//
// Layout in HBM (one scene per context):
//   x, v            float4 per vertex (xyz + inverse mass), caller-owned
//   x_tilde, x_n    float4 per vertex: prediction and step-start positions
//   x_s             float4 per vertex: XPBD iterate before projection
//   planes          float4 (n, d) per slot, vertex-major: [v * K + j]
//   keys            u64 per slot (optional)
//   count           u32 per vertex (planes received; may exceed K)
//   dmin_drop       u32 per vertex: order-preserving code of the smallest d
//                   among planes beyond K (0xFFFFFFFF = none)
//   grid            one counting-sorted spatial hash per table (triangles,
//                   edges, isolated points, vertices); buckets of all tables
//                   are concatenated so one scan serves the four; each item
//                   record is two float4: (lo.xyz, id), (hi.xyz, packed cell)
//   units           per query table, (bucket, offset) of every run of up to
//                   32 queries that share a bucket: one warp work unit
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ccfr {

typedef unsigned long long u64;

// Grid tables: triangles, edges and isolated points (queries and items of
// their own kind), and all vertices bucketed with the triangle cell size (the
// items of the vertex-face queries).
// A fifth table holds the oversized edges again, with a cell as large as the
// largest edge, so that oversized edge pairs are found by a local search.
// Grid tables: triangles, edges, isolated points, vertices (queried by
// triangles), oversized moving edges, oversized static edges (every vertex
// immobile), and giant edges.
enum { KIND_TRI = 0, KIND_EDGE = 1, KIND_PT = 2, KIND_VQ = 3, KIND_BIGE = 4, KIND_BIGS = 5, KIND_GIANT = 6,
       N_TABLES = 7 };
// MODE_BIGQ: the oversized pass's broad phase alone, its candidate pairs
// written to DevCtx::bq for the narrow kernel (k_big_narrow)
enum { MODE_PLANES = 0, MODE_PAIRS = 1, MODE_BIGQ = 2 };
enum { ERR_NONFINITE = 1u };

// Near-parallel edge pairs (a*e - b^2 <= NEAR_PARALLEL * a * e in binary32)
// are re-solved in FP64; below that ratio the binary32 closest points lose
// more than ~1e-5 of the contact normal.
constexpr float NEAR_PARALLEL = 1e-3f;
// The FP64 closest-point solve treats a*e - b^2 <= PARALLEL_EPS * a * e as
// parallel (textbook clamped rule: s = 0, then t, then s again).
constexpr double PARALLEL_EPS = 1e-12;

// Pair kinds of the counters: 0 vertex-face, 1 edge-edge, 2 point-point,
// 3 point-edge (isolated points against free edges).
constexpr int PAIR_VE = 3;
struct DevStats {
    u64 cand[4];
    u64 pairs[4];
    u64 planes_kind[4];
    u64 planes;
    u64 overflow_verts;
    u64 violated_verts;
    u64 halts;
    u64 ee_fp64;
    u64 feas_fp64;
    u64 feas_halts;
    u64 iterations;
    u64 steps;
    u64 aux[16];
    unsigned max_planes;
    unsigned error_flags;
};

struct DevParams {
    float r, two_r, xi, pad;
    float eps, eps_dep, tau;
    float dt, gx, gy, gz, alpha_tilde;
    int max_passes;
    int K;
    int short_max;              // plane lists up to this length are projected one thread per vertex
    float cell_size;
    float delta, k_resp, delta_v, mu_s, mu_k;   // contact response (Sec. 3.3); on when delta > 0
};

// Everything a kernel needs, passed by value.
struct DevCtx {
    DevParams p;
    int n_verts, n_edges, n_tris, n_pts;
    const int2* edges;          // canonical order
    const int3* tris;
    const int* pts;             // isolated vertices
    // XPBD (colour-sorted copies): distance constraints (the edges, then the
    // extra links) with their rest lengths and compliances / dt^2, then the
    // tetrahedra with their rest volumes (x 6)
    const int2* edges_col;
    const float* rest_col;
    const float* alpha_col;
    float* lambda;
    int n_dist;                 // edges + links
    int n_tets;
    const int4* tets_col;
    float* vol6_col;
    float* tlambda;
    float alpha_vol;
    // collision participation: a vertex of links or tetrahedra only (the
    // interior of a volume) is no collision query (null: every vertex is);
    // the free edges (of no triangle), which meet the isolated points
    const unsigned char* vcollide;
    const int* free_list;       // null: none
    int n_free;
    // grid
    int n_items;                // n_tris + 2 n_edges + n_pts + n_verts
    int item_base[N_TABLES];    // first item of each table in the item space
    int bucket_base[N_TABLES + 1];  // first bucket of each table (+ total)
    int bucket_mask[N_TABLES];  // M_table - 1
    unsigned* ext_bits;         // [3] largest padded extent per kind (float bits)
    u64* ext_sum;               // [3] sum of padded extents per kind, in nanometres
    int n_kind[3];              // primitives per kind (triangles, edges, points)
    float cell_factor;          // cell size = cell_factor x mean padded extent
    int* big;                   // [n_tris + n_edges] primitives larger than a cell
    float4* big_box;            // [2 (n_tris + n_edges)] their padded boxes (lo + id, hi)
    int big_base[2];            // first slot of the triangles / edges
    unsigned* big_count;        // [2]
    // candidate pairs between the broad and narrow kernels of the emission
    // (MODE_BIGQ): bq for the kinds on the main stream (vertex-face, oversized
    // primitives), eq for the edge-edge pairs of fitting edges (side stream)
    int2* bq;
    u64* bq_count;              // [1]
    long bq_cap;
    int2* eq;
    u64* eq_count;              // [1]
    long eq_cap;
    int2* units;                // [n_tris + n_edges + n_pts + 3] warp work units
    int unit_base[3];           // first unit slot of each query table
    unsigned* unit_count;       // [3]
    unsigned* sched;            // [N_SCHED] next-work counters of the emission launches of one
                                //   build (zeroed at its start), one per kernel instance
    unsigned* bucket_count;     // [Mtot + 1] counts, then exclusive scan (start)
    unsigned* bucket_fill;      // [Mtot]
    unsigned* item_bucket;      // [n_items]
    float4* rec;                // [2 * n_items]
    // regions
    float4* planes;
    float* phi;                 // [n_verts * K] gap phi of each plane's pair (contact response only)
    u64* keys;                  // may be null
    unsigned* count;
    unsigned* dmin_drop;
    // step state
    float4* x_tilde;
    float4* x_n;
    float4* x_s;
    int* flags;                 // [0] not converged, [1] done (early exit)
    int n_sm;                   // streaming multiprocessors (persistent grids)
    int emit_bps;               // emission blocks per SM
    // several independent scenes in one context (batched step): the scene of
    // every vertex and each scene's (r, 2r, xi, pad); null for a single scene
    const unsigned short* vscene;
    const float4* sparams;
    // per-scene step mask (ccfr_step_active): a scene whose byte is 0 is left
    // unchanged by the substep (positions and velocities); null: all scenes
    const unsigned char* active;
    int4* work;                 // [n_verts] vertices queued for the second projection kernels:
                                //   long plane lists from the front, short ones from the back
    unsigned* work_count;       // [4] queue lengths (long lists, short lists), the long-list
                                //   kernel's next queue entry, spare
    DevStats* stats;
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned f2ord(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned o) {
    unsigned u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    return __uint_as_float(u);
}

__device__ __forceinline__ u64 pair_key(int kind, int a, int b) {
    return ((u64)kind << 62) | ((u64)(unsigned)a << 31) | (u64)(unsigned)b;
}

// Cell size of a table: cell_factor x the mean padded extent of its
// primitives (or the user's cell size if larger), never below the padded
// vertex box, so vertex boxes always fit in one cell.  Primitives whose box
// spans more than a cell are handled by the oversized pass.
// Oversized edges (boxes larger than an edge cell) go to a table whose cell is
// BIGE_FACTOR edge cells; the few larger than that ("giants") to a table whose
// cell is the largest edge box.
constexpr float BIGE_FACTOR = 2.0f;
constexpr int N_SCHED = 24;

// The longest plane list the projection gives a thread of its own
// (k_project_short) rather than a warp (k_project_heavy): a warp spends its
// Alg. 1 steps on one lane (and on this part an FP64 warp instruction holds
// the FP64 pipe for the whole warp), a thread-per-vertex walk runs 32
// vertices' steps in double-float side by side but scans its list alone.
// Lists of contexts with a small capacity (<= 128: few planes per vertex)
// are short up to 64 planes (the 1.2 M-vertex wires: 15% faster per substep
// than at 32); otherwise up to 32 (the cloth stack's few lists of 33 to 64
// planes carry long walks, and 64 cost 1% there).
__host__ __device__ __forceinline__ int short_list_max(int K) { return K <= 128 ? 64 : 32; }

// Default capacity of the candidate-pair buffers (ccfr_params.pair_capacity):
// the main-stream buffer holds 32 pairs per triangle and edge, the edge-edge
// buffer 96 per edge.  The cloth stack at 262,144 vertices (520,200
// triangles, 782,340 edges) finds about 42 vertex-face pairs per triangle
// and 67 edge-edge pairs per edge in its initial layered state, and about 21
// and 42 once tangled.  An overflow only costs time: the fused pass redoes
// the kind.
constexpr long PAIR_CAP_DEFAULT = 32;

// One of the pair buffers, as a kernel argument.
struct PairBuf {
    int2* p;
    u64* count;                 // pairs found (64-bit: it runs on past cap)
    long cap;
};

__device__ __forceinline__ float cell_size_of(const DevCtx& c, int kind) {
    const bool big = kind == KIND_BIGE || kind == KIND_BIGS;
    if (kind == KIND_GIANT) {
        float h = __uint_as_float(c.ext_bits[KIND_EDGE]) * 1.0625f;
        return (h > 0.f) ? h : 1.f;
    }
    if (big) kind = KIND_EDGE;   // scaled by BIGE_FACTOR below
    float mean = (c.n_kind[kind] > 0) ? (float)((double)c.ext_sum[kind] * 1e-9 / (double)c.n_kind[kind]) : 0.f;
    float h = mean * c.cell_factor;
    float hmin = 2.f * c.p.pad * 1.0625f;
    if (h < hmin) h = hmin;
    if (c.p.cell_size > h) h = c.p.cell_size;
    if (!(h > 0.f)) h = 1.f;
    if (big) h *= BIGE_FACTOR;
    return h;
}

// A primitive fits the single-cell scheme when its box is at most h / 1.0625
// on every axis (the margin absorbs the rounding of the cell coordinates).
__device__ __forceinline__ bool fits_cell(const float lo[3], const float hi[3], float h) {
    float lim = h * (1.0f / 1.0625f);
    return (hi[0] - lo[0]) <= lim && (hi[1] - lo[1]) <= lim && (hi[2] - lo[2]) <= lim;
}

__device__ __forceinline__ int cell_coord(float v, float inv_h) {
    return (int)floorf(v * inv_h);
}

// Cells of different scenes are different cells: the scene enters the hash
// and the packed tag.  The tag keeps 7 bits per axis, enough to tell apart the
// cells one search visits (never more than 127 per axis), and 11 scene bits.
__device__ __forceinline__ unsigned cell_hash(int cx, int cy, int cz, unsigned scene) {
    return ((unsigned)cx * 73856093u) ^ ((unsigned)cy * 19349663u) ^ ((unsigned)cz * 83492791u) ^
           (scene * 2654435761u);
}

__device__ __forceinline__ unsigned cell_pack(int cx, int cy, int cz, unsigned scene) {
    return ((unsigned)cx & 127u) | (((unsigned)cy & 127u) << 7) | (((unsigned)cz & 127u) << 14) | (scene << 21);
}

__device__ __forceinline__ unsigned pack_scene(unsigned packed) { return packed >> 21; }

// Per-scene parameters of the narrow phase and the clamp.
struct SceneParams { float r, two_r, xi, pad; };
__device__ __forceinline__ unsigned scene_of(const DevCtx& c, int v) { return c.vscene ? c.vscene[v] : 0u; }
__device__ __forceinline__ bool vertex_active(const DevCtx& c, int v) {
    return !c.active || c.active[scene_of(c, v)] != 0;
}
__device__ __forceinline__ SceneParams scene_params(const DevCtx& c, unsigned s) {
    SceneParams q;
    if (c.sparams) {
        float4 t = c.sparams[s];
        q.r = t.x; q.two_r = t.y; q.xi = t.z; q.pad = t.w;
    } else {
        q.r = c.p.r; q.two_r = c.p.two_r; q.xi = c.p.xi; q.pad = c.p.pad;
    }
    return q;
}

__device__ __forceinline__ void warp_add_u64(u64* dst, u64 v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

}  // namespace ccfr

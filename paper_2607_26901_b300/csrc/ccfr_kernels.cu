// CUDA kernels of the CCFR hot path (sm_103a).  CUDA cores only: nothing on
// this path is a dense contraction, so no tensor-core path exists.
//
//   broad phase   k_extent, k_bucket_count, k_scan_*, k_bucket_scatter:
//                 padded AABBs (pad = r + xi/2 + delta/2, Sec. 4.1), one
//                 counting-sorted uniform-grid hash table per primitive kind
//   narrow phase  k_emit_vf, k_emit_ee, k_emit_pp: each query primitive scans
//                 its 3x3x3 cell neighbourhood, applies the exact binary32 box
//                 predicate and the exclusions of Alg. 3, and (fused) computes
//                 the closest points, the contact normal (Eq. 1) and the
//                 mass-weighted half-spaces (Eq. 2-3), appending them to the
//                 receiving vertices' fixed-capacity plane lists
//   resolution    k_project: Alg. 2 calling Alg. 1 per vertex, one warp per
//                 vertex streaming its plane list
//   XPBD          k_predict, k_xpbd_color, k_update (Alg. 4)
#include <atomic>

#include "ccfr_device.cuh"
#include "ccfr_internal.h"
#include "ccfr_df.cuh"

namespace ccfr {

// ------------------------------------------------------------ float3 math

struct f3 { float x, y, z; };
__device__ __forceinline__ f3 mk(float x, float y, float z) { f3 r; r.x = x; r.y = y; r.z = z; return r; }
__device__ __forceinline__ f3 sub(f3 a, f3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ f3 add(f3 a, f3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ f3 mul(f3 a, float s) { return mk(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ f3 axpy(float s, f3 a, f3 b) { return mk(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z)); }
__device__ __forceinline__ float dot(f3 a, f3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float len(f3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ f3 xyz(float4 a) { return mk(a.x, a.y, a.z); }

// ---------------------------------------------------------------- boxes

// Padded box of item i of the concatenated item space (triangles, edges,
// isolated points, vertices): lo = fl32(min - pad), hi = fl32(max + pad).
__device__ __forceinline__ int item_box(const DevCtx& c, const float4* __restrict__ x, int i,
                                        float lo[3], float hi[3], int& id, unsigned& scene, bool* immobile = nullptr) {
    int kind, v0;
    float4 a, b, d;
    if (i < c.item_base[KIND_EDGE]) {
        kind = KIND_TRI;
        id = i;
        int3 t = c.tris[id];
        v0 = t.x;
        a = x[t.x]; b = x[t.y]; d = x[t.z];
    } else if (i < c.item_base[KIND_PT]) {
        kind = KIND_EDGE;
        id = i - c.item_base[KIND_EDGE];
        int2 e = c.edges[id];
        v0 = e.x;
        a = x[e.x]; b = x[e.y]; d = b;
    } else if (i < c.item_base[KIND_VQ]) {
        kind = KIND_PT;
        id = c.pts[i - c.item_base[KIND_PT]];
        v0 = id;
        a = x[id]; b = a; d = a;
    } else {
        kind = KIND_VQ;
        id = i - c.item_base[KIND_VQ];
        v0 = id;
        a = x[id]; b = a; d = a;
    }
    scene = scene_of(c, v0);
    if (immobile) *immobile = !(a.w > 0.f || b.w > 0.f || d.w > 0.f);
    const float pad = scene_params(c, scene).pad;
    lo[0] = __fsub_rn(fminf(fminf(a.x, b.x), d.x), pad);
    lo[1] = __fsub_rn(fminf(fminf(a.y, b.y), d.y), pad);
    lo[2] = __fsub_rn(fminf(fminf(a.z, b.z), d.z), pad);
    hi[0] = __fadd_rn(fmaxf(fmaxf(a.x, b.x), d.x), pad);
    hi[1] = __fadd_rn(fmaxf(fmaxf(a.y, b.y), d.y), pad);
    hi[2] = __fadd_rn(fmaxf(fmaxf(a.z, b.z), d.z), pad);
    return kind;
}

// Cell size of a table: the vertex table shares the triangle cells so that a
// triangle's 27-cell neighbourhood holds every vertex whose box overlaps it.
__device__ __forceinline__ int cell_kind(int kind) { return kind == KIND_VQ ? KIND_TRI : kind; }

__global__ void k_extent(DevCtx c, const float4* __restrict__ x) {
    if (c.flags[1]) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned e[3] = {0u, 0u, 0u};
    u64 sum[3] = {0ull, 0ull, 0ull};
    if (i < c.n_items) {
        float lo[3], hi[3];
        int id;
        unsigned sc;
        int kind = item_box(c, x, i, lo, hi, id, sc);
        float m = fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
        if (c.active && !c.active[sc]) m = 0.f;   // paused scene (ccfr_step_active): not in the grid
        // positive floats order as integers; the sum is fixed-point (nm) so it is order-independent
        if (m == m && m > 0.f && m < 1e6f && kind < 3) {
            e[kind] = __float_as_uint(m);
            sum[kind] = (u64)(m * 1e9f + 0.5f);
        }
    }
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        unsigned v = __reduce_max_sync(0xffffffffu, e[k]);
        if ((threadIdx.x & 31) == 0 && v) atomicMax(&c.ext_bits[k], v);
        warp_add_u64(&c.ext_sum[k], sum[k]);
    }
}

__device__ __forceinline__ unsigned item_bucket_of(const DevCtx& c, int kind, const float lo[3], unsigned scene,
                                                   unsigned& packed) {
    float h = cell_size_of(c, cell_kind(kind));
    float inv = 1.0f / h;
    int cx = cell_coord(lo[0], inv), cy = cell_coord(lo[1], inv), cz = cell_coord(lo[2], inv);
    packed = cell_pack(cx, cy, cz, scene);
    return (unsigned)c.bucket_base[kind] + (cell_hash(cx, cy, cz, scene) & (unsigned)c.bucket_mask[kind]);
}

// Triangles and edges whose box spans more than a cell go to the oversized
// list instead of their grid table (the count pass decides).  An oversized
// edge is also an item of an oversized-edge table (cell = BIGE_FACTOR edge
// cells; one for moving and one for immobile edges) when it fits a cell
// there, else of the giant table.
__device__ __forceinline__ int table_of(const DevCtx& c, int kind, const float lo[3], const float hi[3],
                                        bool immobile) {
    if (kind != KIND_EDGE || fits_cell(lo, hi, cell_size_of(c, KIND_EDGE))) return kind;
    if (!fits_cell(lo, hi, cell_size_of(c, KIND_BIGE))) return KIND_GIANT;
    return immobile ? KIND_BIGS : KIND_BIGE;
}

__global__ void k_bucket_count(DevCtx c, const float4* __restrict__ x) {
    if (c.flags[1]) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n_items) return;
    float lo[3], hi[3];
    int id;
    unsigned sc;
    bool immobile;
    int kind = item_box(c, x, i, lo, hi, id, sc, &immobile);
    if (c.active && !c.active[sc]) return;   // paused scene (ccfr_step_active): not in the grid
    if (kind <= KIND_EDGE && !fits_cell(lo, hi, cell_size_of(c, kind))) {
        unsigned s = atomicAdd(&c.big_count[kind], 1u);
        unsigned o = c.big_base[kind] + s;
        c.big[o] = id;
        c.big_box[2 * o] = make_float4(lo[0], lo[1], lo[2], __int_as_float(id));
        c.big_box[2 * o + 1] = make_float4(hi[0], hi[1], hi[2], __uint_as_float(sc));
        if (kind == KIND_TRI) return;
        kind = table_of(c, kind, lo, hi, immobile);
    }
    unsigned packed;
    unsigned b = item_bucket_of(c, kind, lo, sc, packed);
    c.item_bucket[i] = b;
    atomicAdd(&c.bucket_count[b], 1u);
}

__global__ void k_bucket_scatter(DevCtx c, const float4* __restrict__ x) {
    if (c.flags[1]) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n_items) return;
    float lo[3], hi[3];
    int id;
    unsigned sc;
    bool immobile;
    int kind = item_box(c, x, i, lo, hi, id, sc, &immobile);
    if (c.active && !c.active[sc]) return;
    if (kind == KIND_TRI && !fits_cell(lo, hi, cell_size_of(c, kind))) return;
    kind = table_of(c, kind, lo, hi, immobile);
    unsigned packed;
    unsigned b = item_bucket_of(c, kind, lo, sc, packed);
    unsigned pos = c.bucket_count[b] + atomicAdd(&c.bucket_fill[b], 1u);
    // giant-table records carry the immobile flag in the id's top bit
    if (kind == KIND_GIANT && immobile) id |= (int)0x80000000u;
    c.rec[2 * pos] = make_float4(lo[0], lo[1], lo[2], __int_as_float(id));
    c.rec[2 * pos + 1] = make_float4(hi[0], hi[1], hi[2], __uint_as_float(packed));
}

// ------------------------------------------------------------------ scan
// Exclusive scan of n unsigned values in place: per-tile sums, a single-block
// scan of the tile sums, then per-tile scans with the tile offset.

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* smem, unsigned& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned incl = v;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) smem[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned s = (lane < (int)(blockDim.x >> 5)) ? smem[lane] : 0u;
        unsigned si = s;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        smem[lane] = si - s;
        if (lane == 31) smem[32] = si;
    }
    __syncthreads();
    unsigned r = smem[wid] + incl - v;
    total = smem[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(DevCtx c, unsigned* data, int n, unsigned* tile_sums) {
    if (c.flags[1]) return;
    __shared__ unsigned smem[33];
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned s = 0;
    #pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) s += (base + k < n) ? data[base + k] : 0u;
    unsigned total;
    block_exclusive_scan(s, smem, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Scan of the tile sums by one block, SCAN_TILE at a time with a running carry.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_top(DevCtx c, unsigned* tile_sums, int n_tiles) {
    if (c.flags[1]) return;
    __shared__ unsigned smem[33];
    unsigned carry = 0;
    for (int chunk = 0; chunk < n_tiles; chunk += SCAN_TILE) {
        int base = chunk + threadIdx.x * SCAN_ITEMS;
        unsigned vals[SCAN_ITEMS], s = 0;
        #pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) { vals[k] = (base + k < n_tiles) ? tile_sums[base + k] : 0u; s += vals[k]; }
        unsigned total;
        unsigned off = block_exclusive_scan(s, smem, total) + carry;
        #pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            if (base + k < n_tiles) tile_sums[base + k] = off;
            off += vals[k];
        }
        carry += total;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(DevCtx c, unsigned* data, int n, const unsigned* tile_sums) {
    if (c.flags[1]) return;
    __shared__ unsigned smem[33];
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned vals[SCAN_ITEMS], s = 0;
    #pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) { vals[k] = (base + k < n) ? data[base + k] : 0u; s += vals[k]; }
    unsigned total;
    unsigned off = block_exclusive_scan(s, smem, total) + tile_sums[blockIdx.x];
    #pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) data[base + k] = off;
        off += vals[k];
    }
}

// ------------------------------------------------------- plane emission

// A pair's planes are emitted in two steps: every plane first reserves its
// slot in its vertex's list (one count atomic each, all issued before any
// store, so that their round trips to L2 overlap), then the planes are stored.
// A plane beyond the list capacity only lowers the vertex's smallest dropped d.
__device__ __forceinline__ unsigned reserve_slot(const DevCtx& c, int v, bool on) {
    return on ? atomicAdd(&c.count[v], 1u) : 0u;
}
__device__ __forceinline__ void store_plane(const DevCtx& c, int v, bool on, unsigned slot, f3 n, float d, float phi,
                                            u64 key) {
    if (!on) return;
    if (slot < (unsigned)c.p.K) {
        size_t o = (size_t)v * c.p.K + slot;
        c.planes[o] = make_float4(n.x, n.y, n.z, d);
        if (c.keys) c.keys[o] = key;
        if (c.phi) c.phi[o] = phi;
    } else {
        atomicMin(&c.dmin_drop[v], f2ord(d));
    }
}

__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Closest point to the origin on triangle (a, b, c) by Voronoi-region
// classification: the vertex and edge regions are decided from the signs of
// first-order dot products (never by comparing squared distances, which
// differ only at second order near a vertex and would misplace the contact
// normal).  Returns true when the point is the foot of the perpendicular
// inside the face; wa, wb, wc are its barycentric weights.
__device__ bool closest_on_triangle(f3 a, f3 b, f3 cc, f3& q, float& wa, float& wb, float& wc) {
    f3 ab = sub(b, a), ac = sub(cc, a);
    f3 pa = mk(-a.x, -a.y, -a.z);                 // origin - a
    float d1 = dot(ab, pa), d2 = dot(ac, pa);
    if (d1 <= 0.f && d2 <= 0.f) { q = a; wa = 1.f; wb = 0.f; wc = 0.f; return false; }
    f3 pb = mk(-b.x, -b.y, -b.z);
    float d3 = dot(ab, pb), d4 = dot(ac, pb);
    if (d3 >= 0.f && d4 <= d3) { q = b; wa = 0.f; wb = 1.f; wc = 0.f; return false; }
    float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
        float t = d1 / (d1 - d3);
        q = axpy(t, ab, a); wa = 1.f - t; wb = t; wc = 0.f;
        return false;
    }
    f3 pc = mk(-cc.x, -cc.y, -cc.z);
    float d5 = dot(ab, pc), d6 = dot(ac, pc);
    if (d6 >= 0.f && d5 <= d6) { q = cc; wa = 0.f; wb = 0.f; wc = 1.f; return false; }
    float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        float t = d2 / (d2 - d6);
        q = axpy(t, ac, a); wa = 1.f - t; wb = 0.f; wc = t;
        return false;
    }
    float va = d3 * d6 - d5 * d4;
    float e43 = d4 - d3, e56 = d5 - d6;
    if (va <= 0.f && e43 >= 0.f && e56 >= 0.f) {
        float t = e43 / (e43 + e56);
        q = axpy(t, sub(cc, b), b); wa = 0.f; wb = 1.f - t; wc = t;
        return false;
    }
    float inv = 1.f / (va + vb + vc);
    float v = vb * inv, w = vc * inv;
    q = add(a, add(mul(ab, v), mul(ac, w)));
    wa = 1.f - v - w; wb = v; wc = w;
    return true;
}

// Vertex-face pair (Alg. 3): p against triangle t = (ta, tb, tc).  Local
// coordinates centred at p.  Returns 1 if the pair is accepted (phi < 2r).
__device__ int narrow_vf(const DevCtx& c, int p, float4 P, int t, int3 T, float4 A, float4 B, float4 C) {
    const SceneParams sp = scene_params(c, scene_of(c, p));
    f3 o = xyz(P);
    f3 a = sub(xyz(A), o), b = sub(xyz(B), o), cc = sub(xyz(C), o);
    f3 q;
    float wa, wb, wc;
    bool inside = closest_on_triangle(a, b, cc, q, wa, wb, wc);
    f3 diff = mk(-q.x, -q.y, -q.z);
    if (inside) {
        // foot of the perpendicular: the separation is along the face normal,
        // which the cross product gives to binary32 accuracy
        f3 N = cross(sub(b, a), sub(cc, a));
        float nl = len(N);
        if (nl > 0.f) {
            f3 nh = mk(N.x / nl, N.y / nl, N.z / nl);
            float h = -dot(a, nh);
            diff = mul(nh, h);
        }
    }
    float dist = len(diff);
    if (dist == 0.f) return 0;
    float phi = dist - sp.xi;
    if (!(phi < sp.two_r)) return 0;
    float wf = wa * A.w + wb * B.w + wc * C.w;
    float W = P.w + wf;
    if (W == 0.f) return 0;
    f3 n = mk(diff.x / dist, diff.y / dist, diff.z / dist);
    f3 mn = mk(-n.x, -n.y, -n.z);
    u64 key = pair_key(0, p, t);
    const bool op = P.w > 0.f, oa = A.w > 0.f, ob = B.w > 0.f, oc = C.w > 0.f;
    const unsigned sp_ = reserve_slot(c, p, op), sa = reserve_slot(c, T.x, oa), sb = reserve_slot(c, T.y, ob),
                   sc = reserve_slot(c, T.z, oc);
    const float df = (wf / W) * phi;
    store_plane(c, p, op, sp_, n, (P.w / W) * phi, phi, key);
    store_plane(c, T.x, oa, sa, mn, df, phi, key);
    store_plane(c, T.y, ob, sb, mn, df, phi, key);
    store_plane(c, T.z, oc, sc, mn, df, phi, key);
    return (int)op + (int)oa + (int)ob + (int)oc;
}

// Closest points of segments p1 + s d1 and p2 + t d2 in FP64 with the
// textbook clamped rule (parallel: s = 0 first).
__device__ void closest_segments_fp64(float4 P1, float4 Q1, float4 P2, float4 Q2, double& s, double& t) {
    double d1x = (double)Q1.x - P1.x, d1y = (double)Q1.y - P1.y, d1z = (double)Q1.z - P1.z;
    double d2x = (double)Q2.x - P2.x, d2y = (double)Q2.y - P2.y, d2z = (double)Q2.z - P2.z;
    double rx = (double)P1.x - P2.x, ry = (double)P1.y - P2.y, rz = (double)P1.z - P2.z;
    double a = d1x * d1x + d1y * d1y + d1z * d1z;
    double e = d2x * d2x + d2y * d2y + d2z * d2z;
    double f = d2x * rx + d2y * ry + d2z * rz;
    double cc = d1x * rx + d1y * ry + d1z * rz;
    double b = d1x * d2x + d1y * d2y + d1z * d2z;
    if (a <= 0.0 && e <= 0.0) { s = t = 0.0; return; }
    if (a <= 0.0) { s = 0.0; t = fmin(fmax(f / e, 0.0), 1.0); return; }
    if (e <= 0.0) { t = 0.0; s = fmin(fmax(-cc / a, 0.0), 1.0); return; }
    double den = a * e - b * b;
    s = (den > PARALLEL_EPS * a * e) ? fmin(fmax((b * f - cc * e) / den, 0.0), 1.0) : 0.0;
    t = (b * s + f) / e;
    if (t < 0.0) { t = 0.0; s = fmin(fmax(-cc / a, 0.0), 1.0); }
    else if (t > 1.0) { t = 1.0; s = fmin(fmax((b - cc) / a, 0.0), 1.0); }
}

// Near-parallel edges: closest points in FP64 and their separation rounded
// once to binary32.  Out of line: rare, and its FP64 registers would
// otherwise count against the occupancy of the whole emission kernel.
__device__ __noinline__ void near_parallel_fp64(const float4* __restrict__ x, int2 E, int2 F, f3& diff, float& s,
                                                float& t) {
    const float4 A0 = x[E.x], A1 = x[E.y], B0 = x[F.x], B1 = x[F.y];
    double sd, td;
    closest_segments_fp64(A0, A1, B0, B1, sd, td);
    double ax = (double)A0.x + sd * ((double)A1.x - A0.x), ay = (double)A0.y + sd * ((double)A1.y - A0.y),
           az = (double)A0.z + sd * ((double)A1.z - A0.z);
    double bx = (double)B0.x + td * ((double)B1.x - B0.x), by = (double)B0.y + td * ((double)B1.y - B0.y),
           bz = (double)B0.z + td * ((double)B1.z - B0.z);
    diff = mk((float)(ax - bx), (float)(ay - by), (float)(az - bz));
    s = (float)sd;
    t = (float)td;
}

// Edge-edge pair (Alg. 3): e = (e0, e1) against f = (f0, f1), local
// coordinates centred at e0.  Returns 1 if accepted; *fp64 is set when the
// near-parallel FP64 solve was used.
__device__ int narrow_ee(const DevCtx& c, const float4* __restrict__ x, int e, int2 E, int f, int2 F, float4 A0,
                         float4 A1, float4 B0, float4 B1, int& fp64) {
    const SceneParams sp = scene_params(c, scene_of(c, E.x));
    f3 o = xyz(A0);
    f3 d1 = sub(xyz(A1), o), p2 = sub(xyz(B0), o), d2 = sub(xyz(B1), xyz(B0));
    // r = p1 - p2 = -p2
    float a = dot(d1, d1), ee = dot(d2, d2);
    float f_ = -dot(d2, p2), cc = -dot(d1, p2), b = dot(d1, d2);
    // |d1 x d2|^2 = a e - b^2 (Lagrange), and the unclamped line parameter
    // s* = ((p2 - p1) x d2) . N / |N|^2 loses a factor 1/sin(theta) less than
    // the dot-product form
    f3 N = cross(d1, d2);
    float den = dot(N, N);
    float s, t;
    f3 diff;
    if (den > NEAR_PARALLEL * a * ee) {
        s = fminf(fmaxf(dot(cross(p2, d2), N) / den, 0.f), 1.f);
        t = (b * s + f_) / ee;
        if (t < 0.f) { t = 0.f; s = fminf(fmaxf(-cc / a, 0.f), 1.f); }
        else if (t > 1.f) { t = 1.f; s = fminf(fmaxf((b - cc) / a, 0.f), 1.f); }
        f3 pa = mul(d1, s);
        f3 pb = axpy(t, d2, p2);
        diff = sub(pa, pb);
        if (s > 0.f && s < 1.f && t > 0.f && t < 1.f) {
            // interior closest points: the separation is along d1 x d2
            float nl = sqrtf(den);
            if (nl > 0.f) {
                f3 nh = mk(N.x / nl, N.y / nl, N.z / nl);
                diff = mul(nh, -dot(p2, nh));
            }
        }
    } else {
        near_parallel_fp64(x, E, F, diff, s, t);
        fp64 = 1;
    }
    float dist = len(diff);
    if (dist == 0.f) return 0;
    float phi = dist - sp.xi;
    if (!(phi < sp.two_r)) return 0;
    float wa = (1.f - s) * A0.w + s * A1.w;
    float wb = (1.f - t) * B0.w + t * B1.w;
    float W = wa + wb;
    if (W == 0.f) return 0;
    f3 n = mk(diff.x / dist, diff.y / dist, diff.z / dist);
    f3 mn = mk(-n.x, -n.y, -n.z);
    u64 key = pair_key(1, e, f);
    float da = (wa / W) * phi, db = (wb / W) * phi;
    const bool o0 = A0.w > 0.f, o1 = A1.w > 0.f, o2 = B0.w > 0.f, o3 = B1.w > 0.f;
    const unsigned s0 = reserve_slot(c, E.x, o0), s1 = reserve_slot(c, E.y, o1), s2 = reserve_slot(c, F.x, o2),
                   s3 = reserve_slot(c, F.y, o3);
    store_plane(c, E.x, o0, s0, n, da, phi, key);
    store_plane(c, E.y, o1, s1, n, da, phi, key);
    store_plane(c, F.x, o2, s2, mn, db, phi, key);
    store_plane(c, F.y, o3, s3, mn, db, phi, key);
    return (int)o0 + (int)o1 + (int)o2 + (int)o3;
}

// Point-point pair (isolated particles).
__device__ int narrow_pp(const DevCtx& c, int p, int q, float4 P, float4 Q) {
    const SceneParams sp = scene_params(c, scene_of(c, p));
    f3 diff = sub(xyz(P), xyz(Q));
    float dist = len(diff);
    if (dist == 0.f) return 0;
    float phi = dist - sp.xi;
    if (!(phi < sp.two_r)) return 0;
    float W = P.w + Q.w;
    if (W == 0.f) return 0;
    f3 n = mk(diff.x / dist, diff.y / dist, diff.z / dist);
    u64 key = pair_key(2, p, q);
    const bool op = P.w > 0.f, oq = Q.w > 0.f;
    const unsigned sp_ = reserve_slot(c, p, op), sq = reserve_slot(c, q, oq);
    store_plane(c, p, op, sp_, n, (P.w / W) * phi, phi, key);
    store_plane(c, q, oq, sq, mk(-n.x, -n.y, -n.z), (Q.w / W) * phi, phi, key);
    return (int)op + (int)oq;
}

// Point-edge pair: isolated point p against free edge e = (a, b), a pair kind
// that Alg. 3 lacks (a particle meets a wire through no vertex-face or
// edge-edge pair).  Local coordinates centred at p; the closest point of the
// segment by the clamped parameter t = -a.(b - a) / |b - a|^2, and the plane of
// Alg. 3 with the segment point's inverse mass (1 - t) w_a + t w_b.
__device__ int narrow_pe(const DevCtx& c, int p, float4 P, int e, int2 E, float4 A, float4 B) {
    const SceneParams sp = scene_params(c, scene_of(c, p));
    const f3 o = xyz(P);
    const f3 a = sub(xyz(A), o), ab = sub(xyz(B), xyz(A));
    const float l2 = dot(ab, ab);
    const float t = l2 > 0.f ? fminf(fmaxf(-dot(a, ab) / l2, 0.f), 1.f) : 0.f;
    const f3 q = axpy(t, ab, a);
    const f3 diff = mk(-q.x, -q.y, -q.z);
    const float dist = len(diff);
    if (dist == 0.f) return 0;
    const float phi = dist - sp.xi;
    if (!(phi < sp.two_r)) return 0;
    const float wf = (1.f - t) * A.w + t * B.w;
    const float W = P.w + wf;
    if (W == 0.f) return 0;
    const f3 n = mk(diff.x / dist, diff.y / dist, diff.z / dist);
    const f3 mn = mk(-n.x, -n.y, -n.z);
    const u64 key = pair_key(PAIR_VE, p, e);
    const bool op = P.w > 0.f, oa = A.w > 0.f, ob = B.w > 0.f;
    const unsigned sp_ = reserve_slot(c, p, op), sa = reserve_slot(c, E.x, oa), sb = reserve_slot(c, E.y, ob);
    const float df = (wf / W) * phi;
    store_plane(c, p, op, sp_, n, (P.w / W) * phi, phi, key);
    store_plane(c, E.x, oa, sa, mn, df, phi, key);
    store_plane(c, E.y, ob, sb, mn, df, phi, key);
    return (int)op + (int)oa + (int)ob;
}

// ------------------------------------------------------ neighbourhood scan
//
// Work is organised by grid cell.  A work unit is a run of up to 32 query
// primitives that share a bucket of the query table; the lanes of a warp hold
// one query each, and the queries of one cell share one 3x3x3 neighbourhood
// in the item table.  The warp walks that neighbourhood item by item (every
// lane loads the same record: one broadcast transaction), tests its own query
// against the item with the exact binary32 box predicate, and appends the
// hits to a per-warp queue in shared memory.  Whenever 32 pairs are queued,
// every lane runs the narrow phase of one pair, so the closest-point work
// always runs on full warps.

struct PairOut {
    int* out[3];
    long cap[3];
    unsigned long long* count;   // [3]
};

__device__ __forceinline__ void write_pair(const PairOut& po, int kind, int a, int b) {
    unsigned long long s = atomicAdd(&po.count[kind], 1ull);
    if ((long)s < po.cap[kind]) {
        po.out[kind][2 * s] = a;
        po.out[kind][2 * s + 1] = b;
    }
}

constexpr int EMIT_WARPS = 8;     // warps per block
constexpr int QCAP = 64;          // pair queue per warp (two warps' worth of hits)
constexpr unsigned FULL = 0xffffffffu;

// Work units: one per run of up to 32 items of a non-empty bucket of the
// triangle, edge and point tables.
__global__ void k_make_units(DevCtx c) {
    if (c.flags[1]) return;
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) {
        c.stats->aux[3] += c.big_count[KIND_TRI];
        c.stats->aux[4] += c.big_count[KIND_EDGE];
    }
    if (b >= c.bucket_base[KIND_VQ]) return;
    int kind = (b < c.bucket_base[KIND_EDGE]) ? KIND_TRI : ((b < c.bucket_base[KIND_PT]) ? KIND_EDGE : KIND_PT);
    unsigned n = c.bucket_count[b + 1] - c.bucket_count[b];
    if (n == 0) return;
    unsigned nu = (n + 31u) / 32u;
    unsigned u0 = atomicAdd(&c.unit_count[kind], nu);
    for (unsigned k = 0; k < nu; ++k) c.units[c.unit_base[kind] + u0 + k] = make_int2(b, (int)(32u * k));
}

struct EmitCounters { u64 cand, acc, planes, fp64; };

// Append the n (<= 32) pairs the lanes hold to a candidate-pair buffer (one
// reservation per warp; the count runs on past the capacity, which tells the
// fused pass to redo the kind).
__device__ __forceinline__ void pb_put(const PairBuf& pb, int2 pr, int n, int lane) {
    u64 base = 0;
    if (lane == 0) base = atomicAdd(pb.count, (u64)n);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (lane < n && base + (u64)lane < (u64)pb.cap) pb.p[base + lane] = pr;
}

// Narrow phase of one queued pair (a = query id, b = item id).  VE: (isolated
// point, free edge) pairs.
template <int QK, int MODE, bool VE = false>
__device__ __forceinline__ void process_pair(const DevCtx& c, const float4* __restrict__ x, const PairOut& po,
                                             int2 pr, EmitCounters& k) {
    if (VE) {                                      // (point, edge)
        const int p = pr.x, e = pr.y;
        const int2 E = c.edges[e];
        const float4 P = x[p], A = x[E.x], B = x[E.y];
        if (!(P.w > 0.f || A.w > 0.f || B.w > 0.f)) return;
        ++k.cand;
        if (MODE == MODE_PAIRS) return;
        const int np = narrow_pe(c, p, P, e, E, A, B);
        k.acc += (np > 0);
        k.planes += np;
    } else if (QK == KIND_TRI) {                   // (triangle, vertex)
        int t = pr.x, v = pr.y;
        if (c.vcollide && !c.vcollide[v]) return;   // the interior of a volume: no collision query
        int3 T = c.tris[t];
        float4 P = x[v], A = x[T.x], B = x[T.y], C = x[T.z];
        if (!(P.w > 0.f || A.w > 0.f || B.w > 0.f || C.w > 0.f)) return;
        ++k.cand;
        if (MODE == MODE_PAIRS) { write_pair(po, 0, v, t); return; }
        int np = narrow_vf(c, v, P, t, T, A, B, C);
        k.acc += (np > 0);
        k.planes += np;
    } else if (QK == KIND_EDGE) {                  // (edge, edge), taken as e < f
        const int e = min(pr.x, pr.y), f = max(pr.x, pr.y);
        int2 E = c.edges[e], F = c.edges[f];
        if (F.x == E.x || F.x == E.y || F.y == E.x || F.y == E.y) return;
        float4 A0 = x[E.x], A1 = x[E.y], B0 = x[F.x], B1 = x[F.y];
        if (!(A0.w > 0.f || A1.w > 0.f || B0.w > 0.f || B1.w > 0.f)) return;
        ++k.cand;
        if (MODE == MODE_PAIRS) { write_pair(po, 1, e, f); return; }
        int fp64 = 0;
        int np = narrow_ee(c, x, e, E, f, F, A0, A1, B0, B1, fp64);
        k.acc += (np > 0);
        k.planes += np;
        k.fp64 += fp64;
    } else {                                       // (point, point), taken as p < q
        const int p = min(pr.x, pr.y), q = max(pr.x, pr.y);
        float4 P = x[p], Q = x[q];
        if (!(P.w > 0.f || Q.w > 0.f)) return;
        ++k.cand;
        if (MODE == MODE_PAIRS) { write_pair(po, 2, p, q); return; }
        int np = narrow_pp(c, p, q, P, Q);
        k.acc += (np > 0);
        k.planes += np;
    }
}

// The items of up to 32 cells of one table, gathered across the warp.  Lane j
// describes cell j (has: there is one; b: its bucket; pk: its tag).  The cells'
// item lists are concatenated and dealt out 32 per round, item k to lane
// k % 32, so that the loads of all cells are in flight together.  f(valid, i0,
// i1, j) runs once per round on every lane; valid lanes hold an item of cell j
// whose tag matches (other cells that share the bucket are skipped).  The
// cells with has must come first.
template <typename F>
__device__ __forceinline__ void warp_cell_items(const DevCtx& c, int lane, bool has, unsigned b, unsigned pk, F f) {
    unsigned t0 = 0, cnt = 0;
    if (has) {
        t0 = c.bucket_count[b];
        cnt = c.bucket_count[b + 1] - t0;
    }
    unsigned inc = cnt;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
    }
    const unsigned total = __shfl_sync(FULL, inc, 31);
    const unsigned excl = inc - cnt;
    for (unsigned base = 0; base < total; base += 32) {
        const unsigned k = base + (unsigned)lane;
        // owner: the last cell whose list starts at or before k
        int j = 0;
        #pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const unsigned e = __shfl_sync(FULL, excl, min(j + step, 31));
            if (j + step <= 31 && e <= k) j += step;
        }
        const unsigned tj = __shfl_sync(FULL, t0, j), ej = __shfl_sync(FULL, excl, j), pj = __shfl_sync(FULL, pk, j);
        bool valid = k < total;
        float4 i0 = make_float4(0.f, 0.f, 0.f, 0.f), i1 = i0;
        if (valid) {
            const unsigned s = tj + (k - ej);
            i0 = c.rec[2 * s];
            i1 = c.rec[2 * s + 1];
            valid = __float_as_uint(i1.w) == pj;
        }
        f(valid, i0, i1, j);
    }
}

// The same items as warp_cell_items, cell after cell: each non-empty cell's
// list is dealt out 32 items per round, item k of the cell to lane k % 32.
// No owner search per round, at the price of a partial round at the end of
// each cell; for the oversized primitives, which scan their cells with one
// query per warp, the search was a third of the loop.  Items come in the same
// order.
template <typename F>
__device__ __forceinline__ void warp_cell_items_seq(const DevCtx& c, int lane, bool has, unsigned b, unsigned pk, F f) {
    unsigned t0 = 0, cnt = 0;
    if (has) {
        t0 = c.bucket_count[b];
        cnt = c.bucket_count[b + 1] - t0;
    }
    unsigned nonempty = __ballot_sync(FULL, cnt > 0u);
    while (nonempty) {
        const int j = __ffs(nonempty) - 1;
        nonempty &= nonempty - 1u;
        const unsigned tj = __shfl_sync(FULL, t0, j), cj = __shfl_sync(FULL, cnt, j), pj = __shfl_sync(FULL, pk, j);
        for (unsigned base = 0; base < cj; base += 32) {
            const unsigned k = base + (unsigned)lane;
            bool valid = k < cj;
            float4 i0 = make_float4(0.f, 0.f, 0.f, 0.f), i1 = i0;
            if (valid) {
                const unsigned s = tj + k;
                i0 = c.rec[2 * s];
                i1 = c.rec[2 * s + 1];
                valid = __float_as_uint(i1.w) == pj;
            }
            f(valid, i0, i1, j);
        }
    }
}

// QK: query table (KIND_TRI: triangles against the vertex table, KIND_EDGE,
// KIND_PT: against their own table).  Persistent warps stride over the units.
// A table queried against itself needs only half of the neighbourhood: the
// query's own cell (pairs taken from the smaller id) and the 13 cells after it
// in (z, y, x) order find every pair of cells once.  The triangle queries scan
// all 27 cells of the vertex table.  The items of the scanned cells are
// gathered 32 at a time (warp_cell_items), compacted into shared memory and
// tested by every query lane against one broadcast item at a time.
// MODE_BIGQ: the scan alone, its pairs written to pb for k_pair_narrow (the
// scan then runs at the occupancy of its own small register set); FALLBACK:
// the fused scan and narrow phase, run only when pb overflowed.
template <int QK, int MODE, bool FALLBACK = false>
// three blocks per SM with the narrow phase (the edge-edge one would otherwise
// take enough registers to leave room for two), five for the scan alone
__global__ void __launch_bounds__(EMIT_WARPS * 32, MODE == MODE_BIGQ ? 5 : 3) k_emit(DevCtx c, const float4* __restrict__ x, PairOut po,
                                                             PairBuf pb) {
    if (c.flags[1]) return;
    if (FALLBACK && *pb.count <= (u64)pb.cap) return;
    __shared__ int2 queue[EMIT_WARPS][QCAP];
    __shared__ float4 items[EMIT_WARPS][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int2* q = queue[wib];
    float4* it = items[wib];
    int qn = 0;
    EmitCounters k{0, 0, 0, 0};
    constexpr bool HALF = QK != KIND_TRI;
    constexpr int NOFF = HALF ? 14 : 27;
    const int IK = (QK == KIND_TRI) ? KIND_VQ : QK;
    const float inv = 1.0f / cell_size_of(c, QK);
    const unsigned ibase = (unsigned)c.bucket_base[IK], imask = (unsigned)c.bucket_mask[IK];
    const unsigned nunits = c.unit_count[QK];
    // work units are taken one at a time from this launch's counter (their cells hold
    // very different numbers of items)
    unsigned* const ctr = c.sched + QK * 3 + (MODE == MODE_BIGQ ? 0 : MODE == MODE_PAIRS ? 1 : 2);
    auto next = [&]() {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(ctr, 1u);
        return __shfl_sync(FULL, w, 0);
    };
    // this lane's neighbour offset (cell order (z, y, x); index 13 is the cell itself)
    const int oi = HALF ? 13 + lane : lane;
    const int ox = oi % 3 - 1, oy = (oi / 3) % 3 - 1, oz = oi / 9 - 1;
    for (unsigned u = next(); u < nunits; u = next()) {
        int2 U = c.units[c.unit_base[QK] + u];
        unsigned s0 = c.bucket_count[U.x] + (unsigned)U.y, s1 = c.bucket_count[U.x + 1];
        unsigned n = min(32u, s1 - s0);
        bool act = (unsigned)lane < n;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        if (act) { r0 = c.rec[2 * (s0 + lane)]; r1 = c.rec[2 * (s0 + lane) + 1]; }
        const int qid = __float_as_int(r0.w);
        const unsigned qs = pack_scene(__float_as_uint(r1.w));
        int3 qt = make_int3(-1, -1, -1);
        if (QK == KIND_TRI && act) qt = c.tris[qid];
        const int mx = cell_coord(r0.x, inv), my = cell_coord(r0.y, inv), mz = cell_coord(r0.z, inv);
        unsigned pending = __ballot_sync(FULL, act);
        while (pending) {
            // the queries of one cell (of one scene) share its neighbourhood
            const int leader = __ffs(pending) - 1;
            const int cx = __shfl_sync(FULL, mx, leader), cy = __shfl_sync(FULL, my, leader),
                      cz = __shfl_sync(FULL, mz, leader);
            const unsigned cs = __shfl_sync(FULL, qs, leader);
            const bool in = ((pending >> lane) & 1u) && mx == cx && my == cy && mz == cz && qs == cs;
            pending &= ~__ballot_sync(FULL, in);
            const bool has = lane < NOFF;
            unsigned b = 0, pk = 0;
            if (has) {
                b = ibase + (cell_hash(cx + ox, cy + oy, cz + oz, cs) & imask);
                pk = cell_pack(cx + ox, cy + oy, cz + oz, cs);
            }
            warp_cell_items(c, lane, has, b, pk, [&](bool valid, float4 i0, float4 i1, int j) {
                // compact this round's items into shared memory; w = 1 marks the query's own cell
                const unsigned vb = __ballot_sync(FULL, valid);
                if (valid) {
                    const int pos = __popc(vb & ((1u << lane) - 1u));
                    i1.w = __int_as_float(HALF && j == 0 ? 1 : 0);
                    it[2 * pos] = i0;
                    it[2 * pos + 1] = i1;
                }
                __syncwarp();
                const int nv = __popc(vb);
                // the box test of one broadcast item against this lane's query
                auto test = [&](float4 a0, float4 a1) {
                    const int iid = __float_as_int(a0.w);
                    bool hit = in && r0.x <= a1.x && a0.x <= r1.x && r0.y <= a1.y && a0.y <= r1.y && r0.z <= a1.z &&
                               a0.z <= r1.z;
                    if (QK == KIND_TRI) hit = hit && iid != qt.x && iid != qt.y && iid != qt.z;
                    else hit = hit && (__float_as_int(a1.w) == 0 || iid > qid);
                    return hit;
                };
                // queue the lanes' hits on item iid; send 32 queued pairs on
                auto take = [&](bool hit, int iid) {
                    const unsigned hb = __ballot_sync(FULL, hit);
                    if (!hb) return;
                    if (hit) q[qn + __popc(hb & ((1u << lane) - 1u))] = make_int2(qid, iid);
                    qn += __popc(hb);
                    if (qn >= 32) {
                        __syncwarp();
                        if constexpr (MODE == MODE_BIGQ) pb_put(pb, q[lane], 32, lane);
                        else process_pair<QK, MODE>(c, x, po, q[lane], k);
                        int2 rest = (lane < qn - 32) ? q[32 + lane] : make_int2(0, 0);
                        __syncwarp();
                        if (lane < qn - 32) q[lane] = rest;
                        qn -= 32;
                        __syncwarp();
                    }
                };
                // two items per step: one vote for both when neither hits (most steps)
                int v = 0;
                for (; v + 1 < nv; v += 2) {
                    const float4 a0 = it[2 * v], a1 = it[2 * v + 1], b0 = it[2 * v + 2], b1 = it[2 * v + 3];
                    const bool ha = test(a0, a1), hb = test(b0, b1);
                    if (!__any_sync(FULL, ha || hb)) continue;
                    take(ha, __float_as_int(a0.w));
                    take(hb, __float_as_int(b0.w));
                }
                if (v < nv) {
                    const float4 a0 = it[2 * v], a1 = it[2 * v + 1];
                    take(test(a0, a1), __float_as_int(a0.w));
                }
                __syncwarp();
            });
        }
    }
    __syncwarp();
    if constexpr (MODE == MODE_BIGQ) {
        if (qn > 0) pb_put(pb, q[lane], qn, lane);
        return;                         // the narrow kernel counts the pairs
    } else {
        if (lane < qn) process_pair<QK, MODE>(c, x, po, q[lane], k);
    }
    warp_add_u64(&c.stats->cand[QK], k.cand);
    warp_add_u64(&c.stats->pairs[QK], k.acc);
    warp_add_u64(&c.stats->planes_kind[QK], k.planes);
    if (QK == KIND_EDGE) warp_add_u64(&c.stats->ee_fp64, k.fp64);
    if (FALLBACK && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&c.stats->aux[15], 1ull);
}

// Oversized primitives (box larger than a cell): one warp per primitive scans
// every cell its box can reach, lanes striding over the items of each cell;
// edges also test the other oversized edges with a larger id.  Together with
// the per-cell pass over the fitting primitives this visits every candidate
// pair exactly once.
__device__ __forceinline__ unsigned prim_box(const DevCtx& c, const float4* __restrict__ x, int kind, int id,
                                             float lo[3], float hi[3], bool& immobile) {
    float4 a, b, d;
    int v0;
    if (kind == KIND_TRI) {
        int3 t = c.tris[id];
        v0 = t.x;
        a = x[t.x]; b = x[t.y]; d = x[t.z];
    } else {
        int2 e = c.edges[id];
        v0 = e.x;
        a = x[e.x]; b = x[e.y]; d = b;
    }
    const unsigned scene = scene_of(c, v0);
    immobile = !(a.w > 0.f || b.w > 0.f || d.w > 0.f);
    const float pad = scene_params(c, scene).pad;
    lo[0] = __fsub_rn(fminf(fminf(a.x, b.x), d.x), pad);
    lo[1] = __fsub_rn(fminf(fminf(a.y, b.y), d.y), pad);
    lo[2] = __fsub_rn(fminf(fminf(a.z, b.z), d.z), pad);
    hi[0] = __fadd_rn(fmaxf(fmaxf(a.x, b.x), d.x), pad);
    hi[1] = __fadd_rn(fmaxf(fmaxf(a.y, b.y), d.y), pad);
    hi[2] = __fadd_rn(fmaxf(fmaxf(a.z, b.z), d.z), pad);
    return scene;
}


// VE (QK = KIND_EDGE): every free edge against the isolated points of the
// point-table cells its box reaches (pairs (point, edge)); one warp per free
// edge, as for the oversized primitives, so that no point scans the far more
// numerous edges of triangles.
// MODE_BIGQ: the scan alone; its pairs go to pb for k_pair_narrow, so that
// the scan runs at the occupancy of its own small register set.  FALLBACK:
// the fused scan and narrow phase, run only when the pair buffer of this kind
// overflowed (k_pair_narrow then left the kind untouched).
// five blocks per SM (48 registers, a few spilled; 64 and four blocks without the bound)
constexpr int BIG_MIN_BLOCKS = 5;
template <int QK, int MODE, bool VE = false, bool FALLBACK = false>
__global__ void __launch_bounds__(EMIT_WARPS * 32, BIG_MIN_BLOCKS) k_emit_big(DevCtx c, const float4* __restrict__ x, PairOut po,
                                                              PairBuf pb) {
    if (c.flags[1]) return;
    if (FALLBACK && *pb.count <= (u64)pb.cap) return;
    __shared__ int2 queue[EMIT_WARPS][QCAP];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int2* q = queue[wib];
    int qn = 0;
    EmitCounters k{0, 0, 0, 0};
    const int IK = (QK == KIND_TRI) ? KIND_VQ : KIND_EDGE;
    const unsigned nbig = VE ? (unsigned)c.n_free : c.big_count[QK];
    u64 big_cells = 0, big_scans = 0, big_items = 0, bige_items = 0;   // diagnostics
    // oversized primitives are taken one at a time from this launch's counter (the cells
    // their boxes reach vary by orders of magnitude)
    unsigned* const ctr = c.sched + 9 + (VE ? 6 : QK * 3) + (MODE == MODE_BIGQ ? 0 : MODE == MODE_PAIRS ? 1 : 2);
    auto next = [&]() {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(ctr, 1u);
        return __shfl_sync(FULL, w, 0);
    };
    // append a hit to the warp queue; process 32 queued pairs at a time
    auto push = [&](bool hit, int2 pr) {
        const unsigned hb = __ballot_sync(FULL, hit);
        if (!hb) return;
        if (hit) q[qn + __popc(hb & ((1u << lane) - 1u))] = pr;
        qn += __popc(hb);
        if (qn >= 32) {
            __syncwarp();
            if constexpr (MODE == MODE_BIGQ) pb_put(pb, q[lane], 32, lane);
            else process_pair<VE ? KIND_PT : QK, MODE, VE>(c, x, po, q[lane], k);
            int2 rest = (lane < qn - 32) ? q[32 + lane] : make_int2(0, 0);
            __syncwarp();
            if (lane < qn - 32) q[lane] = rest;
            qn -= 32;
            __syncwarp();
        }
    };
    for (unsigned u = next(); u < nbig; u = next()) {
        const int o = VE ? c.free_list[u] : c.big[c.big_base[QK] + u];
        float lo[3], hi[3];
        bool qimm;
        const unsigned qs = prim_box(c, x, QK, o, lo, hi, qimm);
        int3 ot = make_int3(-1, -1, -1);
        if (QK == KIND_TRI) ot = c.tris[o];
        bool fin = isfinite(lo[0]) && isfinite(lo[1]) && isfinite(lo[2]) && isfinite(hi[0]) && isfinite(hi[1]) &&
                   isfinite(hi[2]);
        if (!fin) {
            if (lane == 0) atomicOr(&c.stats->error_flags, ERR_NONFINITE);
            continue;
        }
        // every item of table TK whose box can reach this one: items sit in the cell
        // of their lower corner and fit a cell, so the cells from lo - 1 to hi
        auto scan_cells = [&](int TK, auto&& test, u64& items) {
            const float tinv = 1.0f / cell_size_of(c, cell_kind(TK));
            const unsigned tbase = (unsigned)c.bucket_base[TK], tmask = (unsigned)c.bucket_mask[TK];
            const float fx0 = floorf(lo[0] * tinv) - 1.f, fx1 = floorf(hi[0] * tinv);
            const float fy0 = floorf(lo[1] * tinv) - 1.f, fy1 = floorf(hi[1] * tinv);
            const float fz0 = floorf(lo[2] * tinv) - 1.f, fz1 = floorf(hi[2] * tinv);
            const double ncell = (double)(fx1 - fx0 + 1.f) * (double)(fy1 - fy0 + 1.f) * (double)(fz1 - fz0 + 1.f);
            const unsigned t_begin = c.bucket_count[tbase], t_end = c.bucket_count[c.bucket_base[TK + 1]];
            const float cmax = 1e9f;
            // the packed tag tells apart at most 127 cells per axis: wider ranges test the whole table
            const bool huge = fabsf(fx0) > cmax || fabsf(fx1) > cmax || fabsf(fy0) > cmax || fabsf(fy1) > cmax ||
                              fabsf(fz0) > cmax || fabsf(fz1) > cmax || fx1 - fx0 >= 127.f || fy1 - fy0 >= 127.f ||
                              fz1 - fz0 >= 127.f;
            const bool whole = huge || ncell * 8.0 > (double)(t_end - t_begin);
            if (lane == 0 && TK == IK) {
                big_cells += whole ? 0ull : (u64)ncell;
                big_scans += whole ? 1ull : 0ull;
            }
            if (whole) {
                // cheaper to test the whole table
                for (unsigned s0 = t_begin; s0 < t_end; s0 += 32) {
                    const unsigned s = s0 + lane;
                    int2 pr = make_int2(-1, -1);
                    if (s < t_end) pr = test(c.rec[2 * s], c.rec[2 * s + 1]);
                    items += (s < t_end) ? 1ull : 0ull;
                    push(pr.x >= 0, pr);
                }
                return;
            }
            // the reachable cells, 32 per round, their items gathered across the warp
            const int x0 = (int)fx0, y0 = (int)fy0, z0 = (int)fz0;
            const int nx = (int)fx1 - x0 + 1, ny = (int)fy1 - y0 + 1, nz = (int)fz1 - z0 + 1;
            const int nc = nx * ny * nz;
            for (int c0 = 0; c0 < nc; c0 += 32) {
                const int ci = c0 + lane;
                const bool has = ci < nc;
                unsigned b = 0, pk = 0;
                if (has) {
                    const int cx = x0 + ci % nx, cy = y0 + (ci / nx) % ny, cz = z0 + ci / (nx * ny);
                    b = tbase + (cell_hash(cx, cy, cz, qs) & tmask);
                    pk = cell_pack(cx, cy, cz, qs);
                }
                warp_cell_items_seq(c, lane, has, b, pk, [&](bool valid, float4 i0, float4 i1, int) {
                    int2 pr = make_int2(-1, -1);
                    if (valid) pr = test(i0, i1);
                    items += valid ? 1ull : 0ull;
                    push(pr.x >= 0, pr);
                });
            }
        };
        auto overlaps = [&](float4 i0, float4 i1) {
            return pack_scene(__float_as_uint(i1.w)) == qs && lo[0] <= i1.x && i0.x <= hi[0] && lo[1] <= i1.y &&
                   i0.y <= hi[1] && lo[2] <= i1.z && i0.z <= hi[2];
        };
        if (VE) {
            u64 pt_items = 0;
            scan_cells(KIND_PT, [&](float4 i0, float4 i1) -> int2 {
                return overlaps(i0, i1) ? make_int2(__float_as_int(i0.w), o) : make_int2(-1, -1);
            }, pt_items);
            continue;
        }
        // the fitting primitives of the item table
        scan_cells(IK, [&](float4 i0, float4 i1) -> int2 {
            const int iid = __float_as_int(i0.w);
            const bool hit = overlaps(i0, i1);
            if (QK == KIND_TRI) {
                if (!(hit && iid != ot.x && iid != ot.y && iid != ot.z)) return make_int2(-1, -1);
                return make_int2(o, iid);
            }
            if (!hit) return make_int2(-1, -1);
            return make_int2(min(o, iid), max(o, iid));
        }, big_items);
        if (QK == KIND_EDGE) {
            // Oversized-oversized pairs; a pair of two immobile edges is never a
            // candidate, so immobile edges only get found.  An edge that fits a
            // cell of the oversized tables (cell = BIGE_FACTOR edge cells) meets
            // the moving ones in their table: its own cell (pairs from the smaller
            // id) and the 13 cells after it in (z, y, x) order, which visit every
            // pair of cells once; and the immobile ones in theirs (27 cells).  A
            // giant (larger than that cell) finds the edges of those tables over
            // its whole range (an immobile giant only the moving ones), and a
            // moving giant the other giants in the giant table (cell = the largest
            // edge box: 27 cells): the immobile ones, and the moving ones from the
            // smaller id.
            auto cells27 = [&](int TK, auto&& accept) {
                const float tinv = 1.0f / cell_size_of(c, TK);
                const unsigned tb = (unsigned)c.bucket_base[TK], tm = (unsigned)c.bucket_mask[TK];
                const int bx = cell_coord(lo[0], tinv), by = cell_coord(lo[1], tinv), bz = cell_coord(lo[2], tinv);
                const bool has = lane < 27;
                unsigned b = 0, pk = 0;
                if (has) {
                    const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
                    b = tb + (cell_hash(bx + dx, by + dy, bz + dz, qs) & tm);
                    pk = cell_pack(bx + dx, by + dy, bz + dz, qs);
                }
                warp_cell_items_seq(c, lane, has, b, pk, [&](bool valid, float4 i0, float4 i1, int) {
                    int2 pr = make_int2(-1, -1);
                    bige_items += valid ? 1ull : 0ull;
                    if (valid && overlaps(i0, i1)) pr = accept((unsigned)__float_as_int(i0.w));
                    push(pr.x >= 0, pr);
                });
            };
            if (fits_cell(lo, hi, cell_size_of(c, KIND_BIGE))) {
                if (!qimm) {
                    const float binv = 1.0f / cell_size_of(c, KIND_BIGE);
                    const unsigned bb = (unsigned)c.bucket_base[KIND_BIGE], bm = (unsigned)c.bucket_mask[KIND_BIGE];
                    const int bx = cell_coord(lo[0], binv), by = cell_coord(lo[1], binv), bz = cell_coord(lo[2], binv);
                    const bool has = lane < 14;
                    const int oi = 13 + lane;
                    const int dx = oi % 3 - 1, dy = (oi / 3) % 3 - 1, dz = oi / 9 - 1;
                    unsigned b = 0, pk = 0;
                    if (has) {
                        b = bb + (cell_hash(bx + dx, by + dy, bz + dz, qs) & bm);
                        pk = cell_pack(bx + dx, by + dy, bz + dz, qs);
                    }
                    warp_cell_items_seq(c, lane, has, b, pk, [&](bool valid, float4 i0, float4 i1, int j) {
                        int2 pr = make_int2(-1, -1);
                        bige_items += valid ? 1ull : 0ull;
                        if (valid) {
                            const int o2 = __float_as_int(i0.w);
                            if ((j != 0 || o2 > o) && overlaps(i0, i1)) pr = make_int2(min(o, o2), max(o, o2));
                        }
                        push(pr.x >= 0, pr);
                    });
                    cells27(KIND_BIGS, [&](unsigned id2) { const int o2 = (int)id2; return make_int2(min(o, o2), max(o, o2)); });
                }
            } else {
                auto any_pair = [&](float4 i0, float4 i1) -> int2 {
                    const int o2 = __float_as_int(i0.w);
                    return overlaps(i0, i1) ? make_int2(min(o, o2), max(o, o2)) : make_int2(-1, -1);
                };
                scan_cells(KIND_BIGE, any_pair, bige_items);
                if (!qimm) {
                    scan_cells(KIND_BIGS, any_pair, bige_items);
                    cells27(KIND_GIANT, [&](unsigned id2) {
                        const int o2 = (int)(id2 & 0x7FFFFFFFu);
                        const bool imm2 = (id2 >> 31) != 0u;
                        return (imm2 || o2 > o) ? make_int2(min(o, o2), max(o, o2)) : make_int2(-1, -1);
                    });
                }
            }
        }
    }
    __syncwarp();
    if constexpr (MODE == MODE_BIGQ) {
        if (qn > 0) pb_put(pb, q[lane], qn, lane);
    } else {
        if (lane < qn) process_pair<VE ? KIND_PT : QK, MODE, VE>(c, x, po, q[lane], k);
    }
    constexpr int SK = VE ? PAIR_VE : QK;
    if (MODE != MODE_BIGQ) {
        warp_add_u64(&c.stats->cand[SK], k.cand);
        warp_add_u64(&c.stats->pairs[SK], k.acc);
        warp_add_u64(&c.stats->planes_kind[SK], k.planes);
    }
    if (VE) return;
    if (MODE != MODE_BIGQ && QK == KIND_EDGE) warp_add_u64(&c.stats->ee_fp64, k.fp64);
    if (MODE != MODE_BIGQ) warp_add_u64(&c.stats->aux[14], k.cand);
    if (FALLBACK) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&c.stats->aux[15], 1ull);
        return;                        // the scan diagnostics were counted by the MODE_BIGQ pass
    }
    warp_add_u64(&c.stats->aux[10], big_cells);
    warp_add_u64(&c.stats->aux[11], big_scans);
    warp_add_u64(&c.stats->aux[12], big_items);
    warp_add_u64(&c.stats->aux[13], bige_items);
}

// Narrow phase of the candidate pairs a MODE_BIGQ scan wrote to pb: one
// thread per pair, grid-strided, four blocks per SM (64 registers, a few
// spilled: 1.5% faster per stack substep than three at 80); nothing when the
// buffer overflowed.  BIG: the pairs of the oversized primitives.
template <int QK, bool BIG>
__global__ void __launch_bounds__(256, 4) k_pair_narrow(DevCtx c, const float4* __restrict__ x, PairOut po,
                                                        PairBuf pb) {
    if (c.flags[1]) return;
    const u64 n = *pb.count;
    EmitCounters k{0, 0, 0, 0};
    if (n <= (u64)pb.cap)
        for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
            process_pair<QK, MODE_PLANES>(c, x, po, pb.p[i], k);
    warp_add_u64(&c.stats->cand[QK], k.cand);
    warp_add_u64(&c.stats->pairs[QK], k.acc);
    warp_add_u64(&c.stats->planes_kind[QK], k.planes);
    if (QK == KIND_EDGE) warp_add_u64(&c.stats->ee_fp64, k.fp64);
    if (BIG) warp_add_u64(&c.stats->aux[14], k.cand);
}

// -------------------------------------------------------------- Alg. 1/2

// Plesnik's ERO-line state (Alg. 1), in coordinates centred at the pass
// start x^(0), so that the auxiliary point w starts at the normal itself.
// Alg. 1 divides by the dependence measures beta; with nearly dependent planes
// (beta ~ 1e-3, e.g. two normals 0.05 rad apart) binary32 would lose the
// result's accuracy, so the steps run in an extended precision R:
//   double: FP64, for the kernels where a group of lanes works on one vertex
//     (the step, a few dozen FP64 instructions, runs on the group's first
//     lane; in the heavy projection the four groups of a warp take theirs in
//     the same warp instructions, since the FP64 pipe, a small fraction of the
//     binary32 rate on this part, is charged per warp instruction);
//   dfl: double-float (two binary32 words, about 48 significant bits;
//     ccfr_df.cuh), for the one-thread-per-vertex kernel, where 32 steps run
//     side by side and FP64 would saturate its pipe.
// The stored normals A are binary32 values (the planes' own); V and B are R.
template <typename R> struct XP;
template <> struct XP<double> {
    static __device__ __forceinline__ double make(float a) { return (double)a; }
    static __device__ __forceinline__ double diff(float a, float b) { return (double)a - (double)b; }  // exact
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
    static __device__ __forceinline__ double neg(double a) { return -a; }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
    static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    // a / b for |b| >= eps_dep: a binary32 reciprocal estimate (relative error
    // below 2^-21) refined by one Newton-Raphson step r <- r + r (1 - b r),
    // which squares the relative error (< 2^-42); the quotient is then a r.
    // Far cheaper on the FP64 pipe than an IEEE division.
    static __device__ __forceinline__ double div(double a, double b) {
        double r = (double)__fdividef(1.f, (float)b);
        r = ::fma(r, ::fma(-b, r, 1.0), r);
        return a * r;
    }
    static __device__ __forceinline__ bool abs_lt(double a, float e) { return fabs(a) < (double)e; }
    static __device__ __forceinline__ bool abs_gt(double a, float e) { return fabs(a) > (double)e; }
    static __device__ __forceinline__ bool gt(double a, float e) { return a > (double)e; }
    static __device__ __forceinline__ float to_float(double a) { return (float)a; }
    // a - b from the binary32 values and their R conversions: exact, as diff
    static __device__ __forceinline__ double diff2(float, double ad, float, double bd) { return ad - bd; }
};
template <> struct XP<dfl> {
    static __device__ __forceinline__ dfl make(float a) { return df_make(a); }
    static __device__ __forceinline__ dfl diff(float a, float b) { return two_sum(a, -b); }  // exact
    static __device__ __forceinline__ dfl add(dfl a, dfl b) { return df_add(a, b); }
    static __device__ __forceinline__ dfl sub(dfl a, dfl b) { return df_sub(a, b); }
    static __device__ __forceinline__ dfl neg(dfl a) { return df_neg(a); }
    static __device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) { return df_fma(a, b, c); }
    static __device__ __forceinline__ dfl mul(dfl a, dfl b) { return df_mul(a, b); }
    static __device__ __forceinline__ dfl div(dfl a, dfl b) { return df_div(a, b); }
    static __device__ __forceinline__ bool abs_lt(dfl a, float e) { return fabsf(a.hi) < e; }
    static __device__ __forceinline__ bool abs_gt(dfl a, float e) { return fabsf(a.hi) > e; }
    static __device__ __forceinline__ bool gt(dfl a, float e) { return a.hi > e; }
    static __device__ __forceinline__ float to_float(dfl a) { return df_to_float(a); }
    static __device__ __forceinline__ dfl diff2(float a, dfl, float b, dfl) { return two_sum(a, -b); }
};

template <typename R> struct V3 { R x, y, z; };
template <typename R> __device__ __forceinline__ V3<R> v3(R x, R y, R z) { V3<R> r; r.x = x; r.y = y; r.z = z; return r; }
template <typename R> __device__ __forceinline__ V3<R> v3_of(f3 a) {
    return v3<R>(XP<R>::make(a.x), XP<R>::make(a.y), XP<R>::make(a.z));
}
// a - b of binary32 vectors, exact in R
template <typename R> __device__ __forceinline__ V3<R> v3_diff(f3 a, f3 b) {
    return v3<R>(XP<R>::diff(a.x, b.x), XP<R>::diff(a.y, b.y), XP<R>::diff(a.z, b.z));
}
template <typename R> __device__ __forceinline__ V3<R> v3_add(V3<R> a, V3<R> b) {
    return v3<R>(XP<R>::add(a.x, b.x), XP<R>::add(a.y, b.y), XP<R>::add(a.z, b.z));
}
template <typename R> __device__ __forceinline__ V3<R> v3_sub(V3<R> a, V3<R> b) {
    return v3<R>(XP<R>::sub(a.x, b.x), XP<R>::sub(a.y, b.y), XP<R>::sub(a.z, b.z));
}
template <typename R> __device__ __forceinline__ R v3_dot(V3<R> a, V3<R> b) {
    return XP<R>::fma(a.x, b.x, XP<R>::fma(a.y, b.y, XP<R>::mul(a.z, b.z)));
}
// s a + b
template <typename R> __device__ __forceinline__ V3<R> v3_axpy(R s, V3<R> a, V3<R> b) {
    return v3<R>(XP<R>::fma(s, a.x, b.x), XP<R>::fma(s, a.y, b.y), XP<R>::fma(s, a.z, b.z));
}

template <typename R> struct Ero {
    int m;
    V3<R> V[3];
    f3 A[3];
    R B[3];
    V3<R> D[3];   // A[j] - A[0] in R (exact: a difference of two binary32 values), j >= 1
};

// One Alg. 1 step with |V| >= 1 stored lines: project zt onto the
// intersection of the stored hyperplanes and n . z = b.  (The first step, onto
// a single plane, is taken in binary32 by the caller.)  The |v| > eps_dep
// test compares squares (no square root).
template <typename R>
__device__ __noinline__ void ortho_step(V3<R>& zt, f3 n, const V3<R>& nd, R b, Ero<R>& S, float eps) {
    using X = XP<R>;
    const int m = S.m;
    const f3 n0 = S.A[0];
    const R b0 = S.B[0];
    const V3<R> vm = S.V[m - 1];
    // (S.V[0] is the first line's normal n0 in R)
    const V3<R> dn = v3<R>(X::diff2(n.x, nd.x, n0.x, S.V[0].x), X::diff2(n.y, nd.y, n0.y, S.V[0].y),
                           X::diff2(n.z, nd.z, n0.z, S.V[0].z));
    const R beta_u = v3_dot(dn, vm);
    if (X::abs_lt(beta_u, eps)) return;
    const V3<R> u = v3_axpy(X::div(X::sub(b, v3_dot(nd, zt)), beta_u), vm, zt);
    V3<R> w = nd;
    #pragma unroll
    for (int j = 1; j <= 2; ++j) {
        if (j > m) break;
        const R bj = (j < m) ? S.B[j] : b;
        const V3<R> dnj = (j < m) ? S.D[j] : dn;
        const R beta_w = v3_dot(dnj, S.V[j - 1]);
        if (X::abs_gt(beta_w, eps))
            w = v3_axpy(X::div(X::sub(X::sub(bj, b0), v3_dot(dnj, w)), beta_w), S.V[j - 1], w);
    }
    const V3<R> vn = v3_sub(w, u);
    if (X::gt(v3_dot(vn, vn), eps * eps)) {
        const V3<R> n0d = S.V[0];   // the first line's vector is its normal, in R
        const R beta_new = v3_dot(n0d, vn);
        zt = X::abs_lt(beta_new, eps) ? u : v3_axpy(X::div(X::sub(b0, v3_dot(n0d, u)), beta_new), vn, u);
        if (S.m < 3) {
            S.V[S.m] = vn;
            S.A[S.m] = n;
            S.B[S.m] = b;
            S.D[S.m] = dn;
            S.m++;
        }
    }
}

__device__ __forceinline__ float rho_at(f3 y, float4 P) { return fmaf(y.x, P.x, fmaf(y.y, P.y, fmaf(y.z, P.z, P.w))); }

// Copies of one plane (one contact reached through several pairs): equal in
// value, bitwise or up to the sign of a zero component.  A copy of the plane
// just visited is a no-op for Alg. 1 (beta = 0: the iterate is already on it)
// and for the pass result (its violation was counted with the first copy), so
// the walks skip it.  Comparing values rather than bits also makes the visit
// count independent of the arrival order of copies that differ only in the
// sign of a zero (those can tie in the pass order up to their slots).
__device__ __forceinline__ bool same_plane(float4 a, float4 b) {
    return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
}

// One pass of Alg. 2 in progress: the pass input, the binary32 iterate y
// (offset from the build position) on which the planes are tested, the
// largest squared distance of y from the pass input so far, the number of
// violated planes met and the ERO state.  The first Alg. 1 step of a pass
// (|V| = 0) is a plain orthogonal projection onto one plane, with no division
// by a dependence measure: it runs in binary32, and its ERO entry (and its
// result in R) is formed from the stored plane P0 only when a second step
// needs it.  Later steps carry their iterate z = y - ypass in R from step to
// step (y is its binary32 rounding): Alg. 1 divides by dependence measures
// beta, and restarting each step from the rounded y would amplify that
// rounding by 1 / beta.
template <typename R> struct Walk {
    f3 ypass, y;
    float dmax2;
    int nv;
    bool lazy0;
    float4 P0;
    V3<R> yp;     // the pass input in R, formed with the first step in R
    V3<R> z;
    Ero<R> S;
};

template <typename R> __device__ __forceinline__ void walk_begin(Walk<R>& W, f3 ypass) {
    W.ypass = ypass;
    W.y = ypass;
    W.dmax2 = 0.f;
    W.nv = 0;
    W.lazy0 = false;
    W.S.m = 0;
}

// b = -d - n . ypass of the plane (n, d) as n . z = b in coordinates centred
// at ypass, from the normal already converted to R (nd)
template <typename R> __device__ __forceinline__ R plane_b_nd(float w, const V3<R>& nd, const V3<R>& yp) {
    return XP<R>::neg(XP<R>::add(XP<R>::make(w), v3_dot(nd, yp)));
}

// The first step's ERO entry and its iterate in R (z = (b0 / |n0|^2) n0 in
// coordinates centred at the pass input), formed when a second step needs them.
template <typename R> __device__ __forceinline__ void walk_lazy0(Walk<R>& W, const V3<R>& yp) {
    W.S.A[0] = xyz(W.P0);
    W.S.V[0] = v3_of<R>(xyz(W.P0));
    W.S.B[0] = plane_b_nd<R>(W.P0.w, W.S.V[0], yp);
    const R beta0 = v3_dot(W.S.V[0], W.S.V[0]);
    const R s0 = XP<R>::div(W.S.B[0], beta0);
    W.z = v3<R>(XP<R>::mul(s0, W.S.V[0].x), XP<R>::mul(s0, W.S.V[0].y), XP<R>::mul(s0, W.S.V[0].z));
}

// A plane violated at the current iterate: Alg. 1 (while |V| < 3; with
// |V| = 3 the plane is counted and the iterate stays).  Steps with |V| >= 1
// work in R on z (kept in R across steps) and round each result to binary32
// for the tests.  The retraction follows once, at the end of the pass
// (walk_end).
template <typename R> __device__ __forceinline__ void walk_visit(Walk<R>& W, float4 P, float eps, float eps_dep) {
    ++W.nv;
    if (W.S.m == 0) {
        const f3 n = xyz(P);
        const float beta0 = dot(n, n);
        if (!(fabsf(beta0) < eps_dep)) {
            W.y = sub(W.y, mul(n, rho_at(W.y, P) / beta0));
            W.P0 = P;
            W.lazy0 = true;
            W.S.m = 1;
        }
    } else if (W.S.m < 3 && !(P.x == W.P0.x && P.y == W.P0.y && P.z == W.P0.z)) {
        // (a normal equal to the first line's gives beta_u = (n - n0) . v = 0
        // exactly, and Alg. 1 leaves the iterate unchanged: skipped)
        if (W.lazy0) {
            W.yp = v3_of<R>(W.ypass);
            walk_lazy0(W, W.yp);
            W.lazy0 = false;
        }
        const V3<R> nd = v3_of<R>(xyz(P));
        ortho_step<R>(W.z, xyz(P), nd, plane_b_nd<R>(P.w, nd, W.yp), W.S, eps_dep);
        const V3<R> yn = v3_add(W.yp, W.z);
        W.y = mk(XP<R>::to_float(yn.x), XP<R>::to_float(yn.y), XP<R>::to_float(yn.z));
    }
    const f3 dz = sub(W.y, W.ypass);
    W.dmax2 = fmaxf(W.dmax2, dot(dz, dz));
}

// Lanes per vertex in k_project_heavy: a warp projects 32 / HEAVY_GROUP
// vertices side by side, each by a group of HEAVY_GROUP lanes (a power of two).
#ifndef CCFR_HEAVY_GROUP
#define CCFR_HEAVY_GROUP 8
#endif
constexpr int HEAVY_GROUP = CCFR_HEAVY_GROUP;
// Extended precision of the heavy projection's Alg. 1 steps (double-float in
// its place was 47% slower on the cloth stack: the steps then compete with the
// selection scans for issue slots) and its resident blocks per SM.
using HeavyR = double;
#ifndef CCFR_HEAVY_BPS
#define CCFR_HEAVY_BPS 8
#endif
static_assert(HEAVY_GROUP >= 2 && HEAVY_GROUP <= 32 && (HEAVY_GROUP & (HEAVY_GROUP - 1)) == 0,
              "HEAVY_GROUP must be a power of two in [2, 32]");

// walk_visit for a group of HEAVY_GROUP lanes that works on one vertex (every
// lane of the group holds the same walk), called by all 32 lanes of the warp;
// `on`: this group visits plane P.  The extended-precision Alg. 1 step runs on
// the group's first lane alone, and the new iterate and line count are
// broadcast to the group.  The leaders of all groups that take an FP64 step
// in the same call take it in the same warp instructions: on this part an
// FP64 warp instruction occupies the FP64 pipe as long with one active lane
// as with 32, so the groups share that cost.  The result is the one every
// lane would compute.
template <typename R>
__device__ __forceinline__ void walk_visit_group(Walk<R>& W, float4 P, bool on, float eps, float eps_dep, int lane) {
    const int gl = lane & (HEAVY_GROUP - 1), leader = lane & ~(HEAVY_GROUP - 1);
    if (on) {
        ++W.nv;
        if (W.S.m == 0) {
            const f3 n = xyz(P);
            const float beta0 = dot(n, n);
            if (!(fabsf(beta0) < eps_dep)) {
                W.y = sub(W.y, mul(n, rho_at(W.y, P) / beta0));
                W.P0 = P;
                W.lazy0 = true;
                W.S.m = 1;
            }
        } else if (W.S.m < 3 && !(P.x == W.P0.x && P.y == W.P0.y && P.z == W.P0.z)) {
            if (gl == 0) {
                if (W.lazy0) {
                    W.yp = v3_of<R>(W.ypass);
                    walk_lazy0(W, W.yp);
                }
                const V3<R> nd = v3_of<R>(xyz(P));
                ortho_step<R>(W.z, xyz(P), nd, plane_b_nd<R>(P.w, nd, W.yp), W.S, eps_dep);
                const V3<R> yn = v3_add(W.yp, W.z);
                W.y = mk(XP<R>::to_float(yn.x), XP<R>::to_float(yn.y), XP<R>::to_float(yn.z));
            }
            W.lazy0 = false;
        }
    }
    W.y = mk(__shfl_sync(FULL, W.y.x, leader), __shfl_sync(FULL, W.y.y, leader), __shfl_sync(FULL, W.y.z, leader));
    W.S.m = __shfl_sync(FULL, W.S.m, leader);
    if (on) {
        const f3 dz = sub(W.y, W.ypass);
        W.dmax2 = fmaxf(W.dmax2, dot(dz, dz));
    }
}

// End of a pass: the pass result (the projected boundary position) is
// shifted back by eps towards the build position, or reset to it when it is
// closer than eps (Sec. 3.2), once per pass that met a violated plane.
template <typename R> __device__ __forceinline__ void walk_end(Walk<R>& W, float eps) {
    if (W.nv == 0) return;
    const float L = len(W.y);
    W.y = (L > eps) ? mul(W.y, (L - eps) / L) : mk(0.f, 0.f, 0.f);
}

// 16-bit hash of a plane's bits: the second sort key, which splits runs of
// equal rho keys on distinct planes (near-duplicate contacts reached through
// several pairs) without a comparison sort.  Any fixed function of the bits
// gives a deterministic order; this one is a multiply-xorshift mix.
__device__ __forceinline__ unsigned plane_hash16(float4 P) {
    unsigned h = __float_as_uint(P.x) * 0x9E3779B1u + __float_as_uint(P.y) * 0x85EBCA77u +
                 __float_as_uint(P.z) * 0xC2B2AE3Du + __float_as_uint(P.w) * 0x27D4EB2Fu;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 13;
    return h & 0xFFFFu;
}

// Order of the planes in a pass of Alg. 2: the sort key (rho at the first
// pass input; Alg. 2 sorts once), then the plane hash, the plane's own bits
// (d, n) and its slot, so that equal keys break ties deterministically and
// independently of the order in which the planes were stored.
struct Tup { u64 a, b, c; unsigned d; };
__device__ __forceinline__ bool tless(const Tup& x, const Tup& y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    if (x.c != y.c) return x.c < y.c;
    return x.d < y.d;
}
__device__ __forceinline__ Tup make_tup_ord(unsigned key_ord, float4 P, int j) {
    Tup t;
    t.a = ((u64)key_ord << 32) | plane_hash16(P);
    t.b = ((u64)f2ord(P.w) << 32) | f2ord(P.x);
    t.c = ((u64)f2ord(P.y) << 32) | f2ord(P.z);
    t.d = (unsigned)j;
    return t;
}
__device__ __forceinline__ Tup make_tup(float key, float4 P, int j) { return make_tup_ord(f2ord(key), P, j); }
__device__ __forceinline__ float4 tup_plane(const Tup& t) {
    return make_float4(ord2f((unsigned)t.b), ord2f((unsigned)(t.c >> 32)), ord2f((unsigned)t.c),
                       ord2f((unsigned)(t.b >> 32)));
}
__device__ __forceinline__ Tup tup_none() {
    Tup t;
    t.a = t.b = t.c = ~0ull;
    t.d = ~0u;
    return t;
}

__device__ __forceinline__ f3 clamp_len(f3 y, float lim) {
    if (!(lim > 0.f)) return mk(0.f, 0.f, 0.f);
    float L = len(y);
    return (L > lim) ? mul(y, lim / L) : y;
}

struct BlockCounters {
    unsigned viol, halt, over, f64, fhalt, maxc, long_pass, short_pass, nviol;
    unsigned long long planes, heavy_planes, short_planes;
    unsigned short_verts;
};

constexpr int PROJ_WARPS = 4;

__device__ __forceinline__ Tup warp_min_tup(Tup best) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Tup t;
        t.a = __shfl_xor_sync(FULL, best.a, o);
        t.b = __shfl_xor_sync(FULL, best.b, o);
        t.c = __shfl_xor_sync(FULL, best.c, o);
        t.d = __shfl_xor_sync(FULL, best.d, o);
        if (tless(t, best)) best = t;
    }
    return best;
}

__device__ __forceinline__ float warp_min(float v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// Minimum of the pass order within each group of HEAVY_GROUP lanes.
__device__ __forceinline__ Tup group_min_tup(Tup best) {
    #pragma unroll
    for (int o = HEAVY_GROUP / 2; o > 0; o >>= 1) {
        Tup t;
        t.a = __shfl_xor_sync(FULL, best.a, o);
        t.b = __shfl_xor_sync(FULL, best.b, o);
        t.c = __shfl_xor_sync(FULL, best.c, o);
        t.d = __shfl_xor_sync(FULL, best.d, o);
        if (tless(t, best)) best = t;
    }
    return best;
}

// One visit of a pass of Alg. 2 over a vertex's np planes pl, by a group of
// HEAVY_GROUP lanes (called by all 32 lanes; `on`: this group selects).
// Alg. 2 sorts the planes once, by rho at the first pass input y0, and walks
// them in that order, handing each plane violated at the current iterate to
// Alg. 1.  Here each visit selects the next such plane directly: the minimum,
// in the pass order (key rho at y0, then plane hash, plane bits, slot), of
// the planes violated at the current iterate y that come after the last
// visited one, cur (a copy of the plane just visited skipped); `first`: no
// plane visited yet in this pass.  That is the plane the ordered walk would
// meet next, so the pass is the same.  Returns tup_none() when there is none.
// Four planes in flight per lane.
__device__ __forceinline__ Tup group_select(const float4* pl, int np, f3 y, f3 y0, const Tup& cur, bool first,
                                            bool on, int lane) {
    Tup best = tup_none();
    if (on) {
        const float4 Pc = tup_plane(cur);
        for (int j0 = lane & (HEAVY_GROUP - 1); j0 < np; j0 += 4 * HEAVY_GROUP) {
            float4 P[4];
            #pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = j0 + HEAVY_GROUP * k;
                P[k] = (j < np) ? pl[j] : make_float4(0.f, 0.f, 0.f, 3.4e38f);
            }
            #pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = j0 + HEAVY_GROUP * k;
                if (j < np && rho_at(y, P[k]) < 0.f && (first || !same_plane(P[k], Pc))) {
                    const Tup t = make_tup(rho_at(y0, P[k]), P[k], j);
                    if ((first || tless(cur, t)) && tless(t, best)) best = t;
                }
            }
        }
    }
    return group_min_tup(best);
}

// Minimum of rho over a vertex's planes at y, and the largest |d|; four
// independent loads in flight per lane.
__device__ __forceinline__ void scan_min_rho(const float4* pl, int np, f3 y, int lane, float& mn, float& dabs) {
    mn = 3.4e38f;
    dabs = 0.f;
    for (int j0 = lane; j0 < np; j0 += 128) {
        float4 P[4];
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            int j = j0 + 32 * k;
            P[k] = (j < np) ? pl[j] : make_float4(0.f, 0.f, 0.f, 3.4e38f);
        }
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            mn = fminf(mn, rho_at(y, P[k]));
            if (j0 + 32 * k < np) dabs = fmaxf(dabs, fabsf(P[k].w));
        }
    }
    mn = warp_min(mn);
    dabs = warp_max(dabs);
}

// Final feasibility check on the stored binary32 position xn: every plane
// must hold within tau plus the binary32 rounding of the position; a
// rounding-error filter decides most planes, FP64 the rest.  This part checks
// the planes j_start, j_start + j_step, ... and sets fail (a plane fails) and
// undecided (FP64 was needed).
__device__ __forceinline__ void final_check_planes(const DevCtx& c, const float4* pl, int np, float4 X, f3 xn,
                                                   int j_start, int j_step, bool& fail, bool& undecided) {
    const float U = 5.9604645e-8f;
    f3 dl = sub(xn, xyz(X));
    float tau = c.p.tau + 2.f * U * (fabsf(xn.x) + fabsf(xn.y) + fabsf(xn.z));
    for (int j0 = j_start; j0 < np; j0 += 4 * j_step) {
        float4 P[4];
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            int j = j0 + j_step * k;
            P[k] = (j < np) ? pl[j] : make_float4(0.f, 0.f, 0.f, 1.f);
        }
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            float rho = rho_at(dl, P[k]);
            float S = fabsf(dl.x * P[k].x) + fabsf(dl.y * P[k].y) + fabsf(dl.z * P[k].z) + fabsf(P[k].w);
            float err = 8.f * U * S;
            if (rho - err >= -tau) continue;
            if (rho + err < -tau) { fail = true; continue; }
            double rd = ((double)xn.x - X.x) * P[k].x + ((double)xn.y - X.y) * P[k].y + ((double)xn.z - X.z) * P[k].z +
                        (double)P[k].w;
            undecided = true;
            if (rd < -(double)tau) fail = true;
        }
    }
}

// The final check of one vertex.  Returns true when the position fails (the
// vertex then halts).  THREAD: one thread checks all planes; otherwise the
// warp's lanes share them.
template <bool THREAD>
__device__ __forceinline__ bool final_check_fails(const DevCtx& c, const float4* pl, int np, float4 X, f3 xn,
                                                  int lane, bool& used_fp64) {
    bool fail = false, undecided = false;
    final_check_planes(c, pl, np, X, xn, THREAD ? 0 : lane, THREAD ? 1 : 32, fail, undecided);
    if (THREAD) {
        used_fp64 = undecided;
        return fail;
    }
    used_fp64 = __any_sync(FULL, undecided);
    return __any_sync(FULL, fail);
}

// Common end of a vertex: max-step clamp (STEP), final check, write-back,
// convergence flag and counters.  THREAD: the vertex belongs to one thread;
// otherwise to the whole warp (lane 0 writes).
template <bool STEP, bool THREAD>
__device__ __forceinline__ void finish_vertex(const DevCtx& c, int lane, int v, float4 X, float4 XP, f3 y0, f3 y,
                                              bool halted, const float4* pl, int np, bool over, unsigned cnt,
                                              BlockCounters& bc, float4* x_out, unsigned char* halt_out) {
    const bool leader = THREAD || lane == 0;
    if (STEP && !halted) y = clamp_len(y, scene_params(c, scene_of(c, v)).r);
    f3 xn = add(xyz(X), y);
    bool changed = (y.x != y0.x || y.y != y0.y || y.z != y0.z);
    if (!halted && np > 0 && (changed || over)) {
        bool f64 = false;
        if (final_check_fails<THREAD>(c, pl, np, X, xn, lane, f64)) {
            halted = true;
            y = mk(0.f, 0.f, 0.f);
            xn = xyz(X);
            if (leader) atomicAdd(&bc.fhalt, 1u);
        }
        if (f64 && leader) atomicAdd(&bc.f64, 1u);
    }
    if (leader) {
        if (halted) atomicAdd(&bc.halt, 1u);
        if (cnt) { atomicMax(&bc.maxc, cnt); atomicAdd(&bc.planes, (unsigned long long)cnt); }
        if (STEP) {
            if (len(sub(y, y0)) > 2.f * c.p.eps) c.flags[0] = 1;
            x_out[v] = make_float4(xn.x, xn.y, xn.z, X.w);
        } else {
            x_out[v] = make_float4(xn.x, xn.y, xn.z, XP.w);
            if (halt_out) halt_out[v] = halted ? 1 : 0;
        }
    }
}

// finish_vertex for the groups of k_project_heavy, called by all 32 lanes;
// `on`: this group's vertex v ends here (its lanes share the final check, its
// first lane writes).  The same end as finish_vertex<STEP, false> for a vertex
// within its plane capacity.
template <bool STEP>
__device__ __forceinline__ void finish_vertex_group(const DevCtx& c, int lane, bool on, int v, float4 X, float4 XP,
                                                    f3 y0, f3 y, bool halted, const float4* pl, int np, unsigned cnt,
                                                    BlockCounters& bc, float4* x_out, unsigned char* halt_out) {
    const bool leader = on && (lane & (HEAVY_GROUP - 1)) == 0;
    if (on && STEP && !halted) y = clamp_len(y, scene_params(c, scene_of(c, v)).r);
    f3 xn = add(xyz(X), y);
    const bool changed = (y.x != y0.x || y.y != y0.y || y.z != y0.z);
    const bool check = on && !halted && np > 0 && changed;
    bool fail = false, undecided = false;
    if (check) final_check_planes(c, pl, np, X, xn, lane & (HEAVY_GROUP - 1), HEAVY_GROUP, fail, undecided);
    const unsigned gbits = (HEAVY_GROUP == 32) ? FULL : (((1u << HEAVY_GROUP) - 1u) << (lane & ~(HEAVY_GROUP - 1)));
    fail = (__ballot_sync(FULL, fail) & gbits) != 0u;
    undecided = (__ballot_sync(FULL, undecided) & gbits) != 0u;
    if (check && fail) {
        halted = true;
        y = mk(0.f, 0.f, 0.f);
        xn = xyz(X);
        if (leader) atomicAdd(&bc.fhalt, 1u);
    }
    if (check && undecided && leader) atomicAdd(&bc.f64, 1u);
    if (leader) {
        if (halted) atomicAdd(&bc.halt, 1u);
        if (cnt) { atomicMax(&bc.maxc, cnt); atomicAdd(&bc.planes, (unsigned long long)cnt); }
        if (STEP) {
            if (len(sub(y, y0)) > 2.f * c.p.eps) c.flags[0] = 1;
            x_out[v] = make_float4(xn.x, xn.y, xn.z, X.w);
        } else {
            x_out[v] = make_float4(xn.x, xn.y, xn.z, XP.w);
            if (halt_out) halt_out[v] = halted ? 1 : 0;
        }
    }
}

__device__ __forceinline__ void flush_block_counters(const DevCtx& c, BlockCounters& bc) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bc.viol) atomicAdd(&c.stats->violated_verts, (u64)bc.viol);
        if (bc.halt) atomicAdd(&c.stats->halts, (u64)bc.halt);
        if (bc.over) atomicAdd(&c.stats->overflow_verts, (u64)bc.over);
        if (bc.f64) atomicAdd(&c.stats->feas_fp64, (u64)bc.f64);
        if (bc.fhalt) atomicAdd(&c.stats->feas_halts, (u64)bc.fhalt);
        if (bc.maxc) atomicMax(&c.stats->max_planes, bc.maxc);
        if (bc.planes) atomicAdd(&c.stats->planes, bc.planes);
        if (bc.long_pass) atomicAdd(&c.stats->aux[0], (u64)bc.long_pass);
        if (bc.short_pass) atomicAdd(&c.stats->aux[1], (u64)bc.short_pass);
        if (bc.nviol) atomicAdd(&c.stats->aux[2], (u64)bc.nviol);
        if (bc.heavy_planes) atomicAdd(&c.stats->aux[6], bc.heavy_planes);
        if (bc.short_verts) atomicAdd(&c.stats->aux[8], (u64)bc.short_verts);
        if (bc.short_planes) atomicAdd(&c.stats->aux[9], bc.short_planes);
    }
}

__device__ __forceinline__ void zero_block_counters(BlockCounters& bc) {
    if (threadIdx.x == 0) {
        bc.viol = bc.halt = bc.over = bc.f64 = bc.fhalt = bc.maxc = bc.long_pass = bc.short_pass = bc.nviol = 0u;
        bc.planes = 0ull;
        bc.heavy_planes = 0ull;
        bc.short_planes = 0ull;
        bc.short_verts = 0u;
    }
    __syncthreads();
}

// The contact response's short lists (one thread per vertex; longer ones one
// warp per vertex).  The projection's bound is per context (DevParams::short_max).
constexpr int SHORT_LIST = 32;

// Projection, first kernel.  Vertices whose planes all hold at the candidate
// (rho_k(x') >= 0: Alg. 2 returns x' after its first pass), vertices without
// planes, and overflowed vertices are finished here; the others are queued
// for k_project_short or k_project_heavy by the length of their plane list.
// One thread per vertex: a short list is scanned by its own thread; long and
// overflowed lists are taken by the whole warp, one vertex after another.
// STEP = true: x_b is the collision-free iterate x_c (read and overwritten),
// candidates come from x_in (the XPBD iterate), and the step is clamped to r.
template <bool STEP>
__device__ __forceinline__ void queue_violated(const DevCtx& c, int v, int np, float mn, float dabs,
                                               BlockCounters& bc) {
    const int4 wk = make_int4(v, __float_as_int(mn), __float_as_int(dabs), 0);
    if (np <= c.p.short_max) {
        const unsigned w = atomicAdd(&c.work_count[1], 1u);
        c.work[c.n_verts - 1 - (int)w] = wk;
    } else {
        const unsigned w = atomicAdd(&c.work_count[0], 1u);
        c.work[w] = wk;
    }
    atomicAdd(&bc.viol, 1u);
}

template <bool STEP>
__global__ void __launch_bounds__(256) k_project(DevCtx c, const float4* x_b, const float4* x_in, float4* x_out,
                                                  unsigned char* halt_out) {
    if (STEP && c.flags[1]) return;
    __shared__ BlockCounters bc;
    zero_block_counters(bc);
    const int lane = threadIdx.x & 31;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    bool warp_job = false;
    if (v < c.n_verts) {
        const float4 X = x_b[v];
        const float4 XP = x_in[v];
        if (X.w > 0.f && (!STEP || vertex_active(c, v))) {
            const unsigned cnt = c.count[v];
            const int np = (int)min(cnt, (unsigned)c.p.K);
            if (cnt > (unsigned)c.p.K || np > c.p.short_max) {
                warp_job = true;
            } else {
                const f3 y0 = sub(xyz(XP), xyz(X));
                const float4* pl = c.planes + (size_t)v * c.p.K;
                float mn = 3.4e38f, dabs = 0.f;
                for (int j = 0; j < np; ++j) {
                    const float4 P = pl[j];
                    mn = fminf(mn, rho_at(y0, P));
                    dabs = fmaxf(dabs, fabsf(P.w));
                }
                if (np > 0 && mn < 0.f)
                    queue_violated<STEP>(c, v, np, mn, dabs, bc);
                else
                    finish_vertex<STEP, true>(c, 0, v, X, XP, y0, y0, false, pl, np, false, cnt, bc, x_out, halt_out);
            }
        } else if (!STEP && halt_out) {
            halt_out[v] = 0;
        }
    }
    // long and overflowed lists: the warp takes them one at a time
    unsigned pend = __ballot_sync(FULL, warp_job);
    while (pend) {
        const int l = __ffs(pend) - 1;
        pend &= pend - 1;
        const int u = v - lane + l;
        const float4 X = x_b[u];
        const float4 XP = x_in[u];
        const f3 y0 = sub(xyz(XP), xyz(X));
        const unsigned cnt = c.count[u];
        const int np = (int)min(cnt, (unsigned)c.p.K);
        const bool over = cnt > (unsigned)c.p.K;
        const float4* pl = c.planes + (size_t)u * c.p.K;
        f3 y = y0;
        bool queued = false;
        if (over) {
            // more planes than slots: bound the step by the smallest d of all planes
            unsigned code = c.dmin_drop[u];
            float dmin = (code == 0xFFFFFFFFu) ? 3.4e38f : ord2f(code);
            float mn, dabs;
            scan_min_rho(pl, np, mk(0.f, 0.f, 0.f), lane, mn, dabs);   // rho at x is d
            y = clamp_len(y0, fmaxf(fminf(dmin, mn), 0.f));
            if (lane == 0) atomicAdd(&bc.over, 1u);
        } else {
            float mn, dabs;
            scan_min_rho(pl, np, y0, lane, mn, dabs);
            if (mn < 0.f) {
                queued = true;
                if (lane == 0) queue_violated<STEP>(c, u, np, mn, dabs, bc);
            }
        }
        if (!queued) finish_vertex<STEP, false>(c, lane, u, X, XP, y0, y, false, pl, np, over, cnt, bc, x_out, halt_out);
    }
    flush_block_counters(c, bc);
}

// Projection, second kernel: the vertices with a violated plane and a long
// plane list.  Each warp projects 32 / HEAVY_GROUP vertices side by side, one
// per group of HEAVY_GROUP lanes, and a group takes the next queued vertex
// from a shared counter as soon as its vertex is done (a vertex costs from a
// few hundred to many thousands of instructions).  All groups advance in
// lockstep, one visit per round: each round every busy group selects the next
// plane of its pass (group_select) and hands it to Alg. 1, whose FP64 steps
// the groups' first lanes take together (walk_visit_group).  A pass of Alg. 2
// is the run of visits from its input; it ends when no violated plane is left
// after the last visited one or once Alg. 1 holds three lines (the iterate no
// longer moves), and its result is retracted once by eps.  The first
// selection of a pass also decides convergence: no plane violated at the pass
// input means Alg. 2 returns it; a violated plane at the input of pass
// max_passes means the vertex halts.  Eight blocks of four warps per SM (64
// registers, a few spilled: 4% faster than six blocks at 80).
template <bool STEP>
__global__ void __launch_bounds__(PROJ_WARPS * 32, CCFR_HEAVY_BPS) k_project_heavy(DevCtx c, const float4* x_b, const float4* x_in,
                                                                    float4* x_out, unsigned char* halt_out) {
    if (STEP && c.flags[1]) return;
    __shared__ BlockCounters bc;
    zero_block_counters(bc);
    const int lane = threadIdx.x & 31, gl = lane & (HEAVY_GROUP - 1), leader = lane & ~(HEAVY_GROUP - 1);
    const unsigned nwork = c.work_count[0];
    const float eps = c.p.eps, eps_dep = c.p.eps_dep;
    int v = -1;                          // the group's vertex; -1: take the next one; -2: queue drained
    float4 X = make_float4(0.f, 0.f, 0.f, 0.f), XP = X;
    f3 y0 = mk(0.f, 0.f, 0.f), ypass = y0;
    int np = 0, pass = 0;
    unsigned cnt = 0;
    const float4* pl = c.planes;
    bool first = true;
    Tup cur = tup_none();
    Walk<HeavyR> W;
    walk_begin(W, ypass);
    for (;;) {
        unsigned w = 0;
        if (v == -1 && gl == 0) w = atomicAdd(&c.work_count[2], 1u);
        w = __shfl_sync(FULL, w, leader);
        if (v == -1) {
            if (w < nwork) {
                v = c.work[w].x;
                X = x_b[v];
                XP = x_in[v];
                y0 = sub(xyz(XP), xyz(X));
                cnt = c.count[v];
                np = (int)min(cnt, (unsigned)c.p.K);
                pl = c.planes + (size_t)v * c.p.K;
                if (gl == 0) atomicAdd(&bc.heavy_planes, (unsigned long long)np);
                ypass = y0;
                pass = 0;
                first = true;
                cur = tup_none();
                walk_begin(W, ypass);
            } else {
                v = -2;
            }
        }
        if (__all_sync(FULL, v == -2)) break;
        const bool sel = v >= 0;
        const Tup best = group_select(pl, np, W.y, y0, cur, first, sel, lane);
        bool visit = false, end_pass = false, done = false, halted = false;
        if (sel) {
            if (best.d == ~0u) {
                if (first) done = true;            // converged: no plane violated at the pass input
                else end_pass = true;
            } else if (first && pass == c.p.max_passes) {
                done = halted = true;              // still violated after max_passes passes
            } else {
                visit = true;
                cur = best;
                first = false;
            }
        }
        walk_visit_group(W, tup_plane(best), visit, eps, eps_dep, lane);
        if (visit && W.S.m == 3) end_pass = true;
        if (end_pass) {
            walk_end(W, eps);
            if (gl == 0) { atomicAdd(&bc.long_pass, 1u); atomicAdd(&bc.nviol, (unsigned)W.nv); }
            ypass = W.y;
            ++pass;
            first = true;
            cur = tup_none();
            walk_begin(W, ypass);
        }
        finish_vertex_group<STEP>(c, lane, done, v, X, XP, y0, halted ? mk(0.f, 0.f, 0.f) : ypass, halted, pl, np, cnt,
                                  bc, x_out, halt_out);
        if (done) v = -1;
    }
    flush_block_counters(c, bc);
}

// Projection, second kernel for short plane lists: one thread per queued
// vertex (persistent threads over the back of the queue).  Each pass of Alg. 2
// visits, over and over, the first plane in the pass order (sort key rho at
// the first input, then hash, plane bits and slot: the order of the warp
// kernel) that comes after the last one visited and is violated at the
// current iterate: the same walk as over the sorted list, without storing it.
template <bool STEP>
__global__ void __launch_bounds__(128) k_project_short(DevCtx c, const float4* x_b, const float4* x_in,
                                                        float4* x_out, unsigned char* halt_out) {
    if (STEP && c.flags[1]) return;
    __shared__ BlockCounters bc;
    zero_block_counters(bc);
    const unsigned nwork = c.work_count[1];
    for (unsigned wi = blockIdx.x * blockDim.x + threadIdx.x; wi < nwork; wi += gridDim.x * blockDim.x) {
        const int4 wk = c.work[c.n_verts - 1 - (int)wi];
        const int v = wk.x;
        const float mn = __int_as_float(wk.y);
        const float4 X = x_b[v];
        const float4 XP = x_in[v];
        const f3 y0 = sub(xyz(XP), xyz(X));
        const unsigned cnt = c.count[v];
        const int np = (int)min(cnt, (unsigned)c.p.K);
        const float4* pl = c.planes + (size_t)v * c.p.K;
        atomicAdd(&bc.short_planes, (unsigned long long)np);
        atomicAdd(&bc.short_verts, 1u);
        f3 ypass = y0;
        bool conv = false;
        for (int pass = 0; pass <= c.p.max_passes; ++pass) {
            // converged when no plane is violated at the pass input (the scan stops at
            // the first violated one)
            bool viol = mn < 0.f;
            if (pass > 0) {
                viol = false;
                for (int j = 0; j < np && !viol; ++j) viol = rho_at(ypass, pl[j]) < 0.f;
            }
            if (!viol) { conv = true; break; }
            if (pass == c.p.max_passes) break;
            Walk<dfl> W;
            walk_begin(W, ypass);
            Tup cur = tup_none();
            bool first = true;
            for (;;) {
                Tup best = tup_none();
                const float4 Pcur = tup_plane(cur);
                for (int j = 0; j < np; ++j) {
                    const float4 P = pl[j];
                    if (rho_at(W.y, P) < 0.f && (first || !same_plane(P, Pcur))) {
                        const Tup t = make_tup(rho_at(y0, P), P, j);
                        if ((first || tless(cur, t)) && tless(t, best)) best = t;
                    }
                }
                if (best.d == ~0u) break;
                cur = best;
                first = false;
                walk_visit(W, tup_plane(best), c.p.eps, c.p.eps_dep);
                if (W.S.m == 3) break;   // the iterate no longer moves in this pass
            }
            walk_end(W, c.p.eps);
            atomicAdd(&bc.short_pass, 1u);
            atomicAdd(&bc.nviol, (unsigned)W.nv);
            ypass = W.y;
        }
        const bool halted = !conv;
        finish_vertex<STEP, true>(c, 0, v, X, XP, y0, halted ? mk(0.f, 0.f, 0.f) : ypass, halted, pl, np, false, cnt,
                                  bc, x_out, halt_out);
    }
    flush_block_counters(c, bc);
}

// ------------------------------------------------------------ response
//
// Contact response and friction (Sec. 3.3), after the XPBD sweep and before
// the projection (Alg. 4, applyResponse).  A contact is one of the vertex's
// planes: normal n_c and its pair's gap phi_c beyond xi at the build position x.
//  - signed distance along the normal at the iterate y, the other side at its
//    build position: g_c = phi_c + n_c . (y - x);
//  - active contacts: g_c < delta, the RESP_CAP innermost in the order of
//    Alg. 2's planes with g as the key (g, plane hash, plane bits, slot);
//  - visibility weight w_c = prod over the other active contacts j of
//    (1 - S((g_c - g_j) / delta_v)), S the cubic smoothstep clamped to [0, 1],
//    at the iterate before the response;
//  - in that order, each active contact once (Gauss-Seidel, fresh multiplier):
//    C = max(0, delta - g_c(y)), compliance 1 / (k w_c):
//    y += w C / (w + 1 / (k w_c dt^2)) n_c;
//  - friction, same order, for each contact that moved y by depth > 0: t = the
//    tangential part of the displacement since the substep start; removed if
//    |t| < mu_s depth, else shortened by min(mu_k depth, |t|).
// Vertices over the plane capacity get no response.  Short plane lists are
// handled one thread per vertex, long ones by the warp.
constexpr int RESP_CAP = 32;
constexpr int RESP_POOL = 256;   // active contacts of a long list held before the innermost are chosen
constexpr int RESP_WARPS = 4;

__device__ __forceinline__ float smoothstep01(float t) {
    t = fminf(fmaxf(t, 0.f), 1.f);
    return t * t * (3.f - 2.f * t);
}

// Visibility weight of contact a among the na active ones (gaps ag).
__device__ __forceinline__ float occlusion_weight(const DevCtx& c, const float* ag, int na, int a) {
    const float inv_dv = 1.f / c.p.delta_v;
    float w = 1.f;
    for (int b = 0; b < na; ++b)
        if (b != a) w *= 1.f - smoothstep01((ag[a] - ag[b]) * inv_dv);
    return w;
}

// The response of one vertex once its active contacts are known, in order,
// with their weights: Gauss-Seidel repulsion, then friction.
__device__ __forceinline__ f3 respond(const DevCtx& c, int v, f3 x, f3 y, float wv, const float4* pl,
                                      const float* ph, const int* aj, const float* wt, int na) {
    float depth[RESP_CAP];
    const float dt2 = c.p.dt * c.p.dt;
    for (int a = 0; a < na; ++a) {
        const f3 n = xyz(pl[aj[a]]);
        const float C = c.p.delta - (ph[aj[a]] + dot(n, sub(y, x)));
        depth[a] = 0.f;
        if (!(C > 0.f) || !(wt[a] > 0.f) || !(c.p.k_resp > 0.f)) continue;
        const float at = 1.f / (c.p.k_resp * wt[a] * dt2);
        const float corr = wv * C / (wv + at);
        y = add(y, mul(n, corr));
        depth[a] = corr;
    }
    if (c.p.mu_s > 0.f || c.p.mu_k > 0.f) {
        const f3 xn = xyz(c.x_n[v]);
        for (int a = 0; a < na; ++a) {
            if (!(depth[a] > 0.f)) continue;
            const f3 n = xyz(pl[aj[a]]);
            const f3 d = sub(y, xn);
            const f3 t = sub(d, mul(n, dot(d, n)));
            const float tl = len(t);
            if (!(tl > 0.f)) continue;
            const float f = (tl < c.p.mu_s * depth[a]) ? 1.f : fminf(c.p.mu_k * depth[a] / tl, 1.f);
            y = sub(y, mul(t, f));
        }
    }
    return y;
}

__global__ void __launch_bounds__(RESP_WARPS * 32) k_response(DevCtx c, const float4* __restrict__ x_b) {
    if (c.flags[1]) return;
    __shared__ float s_g[RESP_WARPS][RESP_POOL];
    __shared__ int s_j[RESP_WARPS][RESP_POOL];
    __shared__ float s_w[RESP_WARPS][RESP_CAP];
    __shared__ unsigned s_h[RESP_WARPS][256];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const float delta = c.p.delta;
    bool warp_job = false;
    if (v < c.n_verts) {
        const float4 X = x_b[v];
        const unsigned cnt = c.count[v];
        if (X.w > 0.f && cnt > 0u && cnt <= (unsigned)c.p.K && vertex_active(c, v)) {
            const int np = (int)cnt;
            if (np > SHORT_LIST) {
                warp_job = true;
            } else {
                // short list: this thread, the active contacts kept in order by insertion
                const float4* pl = c.planes + (size_t)v * c.p.K;
                const float* ph = c.phi + (size_t)v * c.p.K;
                const float4 Y0 = c.x_s[v];
                const f3 x = xyz(X), y = xyz(Y0), dy = sub(y, x);
                float ag[RESP_CAP];
                int aj[RESP_CAP];
                int na = 0;
                for (int j = 0; j < np; ++j) {
                    const float4 P = pl[j];
                    const float g = ph[j] + dot(xyz(P), dy);
                    if (!(g < delta)) continue;
                    int q = na++;
                    const Tup t = make_tup(g, P, j);
                    while (q > 0 && tless(t, make_tup(ag[q - 1], pl[aj[q - 1]], aj[q - 1]))) {
                        ag[q] = ag[q - 1];
                        aj[q] = aj[q - 1];
                        --q;
                    }
                    ag[q] = g;
                    aj[q] = j;
                }
                if (na > 0) {
                    float wt[RESP_CAP];
                    for (int a = 0; a < na; ++a) wt[a] = occlusion_weight(c, ag, na, a);
                    const f3 yn = respond(c, v, x, y, X.w, pl, ph, aj, wt, na);
                    c.x_s[v] = make_float4(yn.x, yn.y, yn.z, Y0.w);
                }
            }
        }
    }
    // long lists: the warp scans the planes, collects the active contacts and
    // picks the innermost, one per lane, in order
    unsigned pend = __ballot_sync(FULL, warp_job);
    float* pg = s_g[wib];
    int* pj = s_j[wib];
    while (pend) {
        const int l = __ffs(pend) - 1;
        pend &= pend - 1;
        const int u = v - lane + l;
        const float4 X = x_b[u];
        const float4 Y0 = c.x_s[u];
        const int np = (int)c.count[u];
        const float4* pl = c.planes + (size_t)u * c.p.K;
        const float* ph = c.phi + (size_t)u * c.p.K;
        const f3 x = xyz(X), y = xyz(Y0), dy = sub(y, x);
        int total = 0;
        for (int j0 = 0; j0 < np; j0 += 32) {
            const int j = j0 + lane;
            float g = 0.f;
            bool act = false;
            if (j < np) {
                g = ph[j] + dot(xyz(pl[j]), dy);
                act = g < delta;
            }
            const unsigned bal = __ballot_sync(FULL, act);
            const int pos = total + __popc(bal & ((1u << lane) - 1u));
            if (act && pos < RESP_POOL) {
                pg[pos] = g;
                pj[pos] = j;
            }
            total += __popc(bal);
        }
        __syncwarp();
        if (total == 0) continue;
        int sel = total;   // contacts in the pool's head to order (after the select below)
        if (total > 32 && total <= RESP_POOL) {
            // radix select on the ordered gap: the 32nd smallest key K, then the
            // contacts below K and, of those at K, the first in the full order
            unsigned* hist = s_h[wib];
            unsigned prefix = 0u, pmask = 0u;
            int need = RESP_CAP;
            for (int shift = 24; shift >= 0; shift -= 8) {
                for (int b = lane; b < 256; b += 32) hist[b] = 0u;
                __syncwarp();
                for (int i = lane; i < total; i += 32) {
                    const unsigned k = f2ord(pg[i]);
                    if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
                }
                __syncwarp();
                unsigned loc[8], tot = 0;
                #pragma unroll
                for (int q = 0; q < 8; ++q) { loc[q] = hist[lane * 8 + q]; tot += loc[q]; }
                unsigned inc = tot;
                #pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned t = __shfl_up_sync(FULL, inc, o);
                    if (lane >= o) inc += t;
                }
                const unsigned before = inc - tot;
                // the lane whose bins reach the need-th key holds the digit
                int digit = -1;
                unsigned below = 0u;
                if (before < (unsigned)need && inc >= (unsigned)need) {
                    unsigned acc = before;
                    for (int q = 0; q < 8; ++q) {
                        if (acc + loc[q] >= (unsigned)need) { digit = lane * 8 + q; below = acc; break; }
                        acc += loc[q];
                    }
                }
                const unsigned bd = __ballot_sync(FULL, digit >= 0);
                const int owner = __ffs(bd) - 1;
                digit = __shfl_sync(FULL, digit, owner);
                below = __shfl_sync(FULL, below, owner);
                prefix |= (unsigned)digit << shift;
                pmask |= 255u << shift;
                need -= (int)below;
                __syncwarp();
            }
            // compact: keys below K first (fewer than 32), then the ties at K
            int n_lt = 0;
            for (int i0 = 0; i0 < total; i0 += 32) {
                const int i = i0 + lane;
                const bool lt = i < total && f2ord(pg[i]) < prefix;
                const unsigned bal = __ballot_sync(FULL, lt);
                if (lt) hist[n_lt + __popc(bal & ((1u << lane) - 1u))] = (unsigned)i;
                n_lt += __popc(bal);
            }
            __syncwarp();
            int n_eq = 0;
            for (int i0 = 0; i0 < total; i0 += 32) {
                const int i = i0 + lane;
                const bool eq = i < total && f2ord(pg[i]) == prefix;
                const unsigned bal = __ballot_sync(FULL, eq);
                const int pos = n_lt + n_eq + __popc(bal & ((1u << lane) - 1u));
                if (eq && pos < 256) hist[pos] = (unsigned)i;
                n_eq += __popc(bal);
            }
            __syncwarp();
            if (n_lt + n_eq <= 32) {
                // gather the chosen (all of the ties fit) to the pool's head
                float gl = 0.f;
                int jl = -1;
                const bool mine = lane < n_lt + n_eq;
                if (mine) { gl = pg[hist[lane]]; jl = pj[hist[lane]]; }
                __syncwarp();
                if (mine) { pg[lane] = gl; pj[lane] = jl; }
                __syncwarp();
                sel = n_lt + n_eq;
            }
            // else: too many exact ties at K, the repeated minimum below decides
        }
        const int na = min(total, RESP_CAP);
        float mg = 0.f;
        int mj = -1;
        if (sel <= 32) {
            total = sel;
            // one contact per lane: rank by the full order
            Tup me = tup_none();
            if (lane < total) me = make_tup(pg[lane], pl[pj[lane]], pj[lane]);
            int rank = 0;
            for (int t = 0; t < total; ++t) {
                Tup o;
                o.a = __shfl_sync(FULL, me.a, t);
                o.b = __shfl_sync(FULL, me.b, t);
                o.c = __shfl_sync(FULL, me.c, t);
                o.d = __shfl_sync(FULL, me.d, t);
                rank += tless(o, me) ? 1 : 0;
            }
            const float gl = (lane < total) ? pg[lane] : 0.f;
            const int jl = (lane < total) ? pj[lane] : -1;
            __syncwarp();
            if (lane < total) {
                pg[rank] = gl;
                pj[rank] = jl;
            }
            __syncwarp();
            if (lane < na) {
                mg = pg[lane];
                mj = pj[lane];
            }
        } else {
            // repeated warp minimum, over the pool, or over the whole list when
            // more contacts are active than the pool holds
            Tup last = tup_none();
            bool first = true;
            for (int r = 0; r < na; ++r) {
                Tup best = tup_none();
                if (total <= RESP_POOL) {
                    for (int i = lane; i < total; i += 32) {
                        const Tup t = make_tup(pg[i], pl[pj[i]], pj[i]);
                        if ((first || tless(last, t)) && tless(t, best)) best = t;
                    }
                } else {
                    for (int j = lane; j < np; j += 32) {
                        const float4 P = pl[j];
                        const float g = ph[j] + dot(xyz(P), dy);
                        if (!(g < delta)) continue;
                        const Tup t = make_tup(g, P, j);
                        if ((first || tless(last, t)) && tless(t, best)) best = t;
                    }
                }
                best = warp_min_tup(best);
                if (lane == r) {
                    mj = (int)best.d;
                    mg = ord2f((unsigned)(best.a >> 32));
                }
                last = best;
                first = false;
            }
        }
        __syncwarp();
        // the chosen contacts in order at the pool's head; each lane weighs its
        // own contact, then lane 0 runs the sequential repulsion and friction
        if (lane < na) {
            pg[lane] = mg;
            pj[lane] = mj;
        }
        __syncwarp();
        if (lane < na) s_w[wib][lane] = occlusion_weight(c, pg, na, lane);
        __syncwarp();
        if (lane == 0) {
            const f3 yn = respond(c, u, x, y, X.w, pl, ph, pj, s_w[wib], na);
            c.x_s[u] = make_float4(yn.x, yn.y, yn.z, Y0.w);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ XPBD

// Alg. 4 prediction: x~ = x + dt v + dt^2 g for movable vertices; keeps x^n.
__global__ void k_predict(DevCtx c, const float4* __restrict__ x, const float4* __restrict__ vel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n_verts) return;
    float4 X = x[i], V = vel[i];
    bool fin = isfinite(X.x) && isfinite(X.y) && isfinite(X.z) && isfinite(X.w) &&
               isfinite(V.x) && isfinite(V.y) && isfinite(V.z);
    if (!fin) atomicOr(&c.stats->error_flags, ERR_NONFINITE);
    c.x_n[i] = X;
    float dt = c.p.dt;
    if (X.w > 0.f && vertex_active(c, i)) {
        X.x = X.x + dt * V.x + dt * dt * c.p.gx;
        X.y = X.y + dt * V.y + dt * dt * c.p.gy;
        X.z = X.z + dt * V.z + dt * dt * c.p.gz;
    }
    c.x_tilde[i] = X;
}

// Start of an iteration: x_s <- x~; clear the per-iteration region counters.
__global__ void k_iter_begin(DevCtx c) {
    if (c.flags[1]) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < c.n_verts) {
        c.x_s[i] = c.x_tilde[i];
        c.count[i] = 0u;
        c.dmin_drop[i] = 0xFFFFFFFFu;
    }
    if (i == 0) c.flags[0] = 0;
}

// One colour of the Gauss-Seidel sweep over edge-distance constraints:
// C = |xa - xb| - L0, dlambda = (-C - alpha~ lambda) / (wa + wb + alpha~).
__global__ void k_xpbd_color(DevCtx c, int e0, int e1) {
    if (c.flags[1]) return;
    int i = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= e1) return;
    int2 e = c.edges_col[i];
    if (!vertex_active(c, e.x)) return;
    float4 A = c.x_s[e.x], B = c.x_s[e.y];
    float at = c.alpha_col[i];
    float wsum = A.w + B.w + at;
    if (wsum == 0.f) return;
    f3 d = sub(xyz(A), xyz(B));
    float L = len(d);
    if (L == 0.f) return;
    float lam = c.lambda[i];
    float dl = (-(L - c.rest_col[i]) - at * lam) / wsum;
    f3 nd = mul(d, 1.f / L);
    float sa = A.w * dl, sb = B.w * dl;
    c.x_s[e.x] = make_float4(A.x + sa * nd.x, A.y + sa * nd.y, A.z + sa * nd.z, A.w);
    c.x_s[e.y] = make_float4(B.x - sb * nd.x, B.y - sb * nd.y, B.z - sb * nd.z, B.w);
    c.lambda[i] = lam + dl;
}

// One colour of the volume constraints: C = 6 V - 6 V0 per tetrahedron with
// 6 V = (x1 - x0) . ((x2 - x0) x (x3 - x0)), whose gradients are the three
// cross products and minus their sum; XPBD update with compliance alpha_vol.
__global__ void k_xpbd_tet_color(DevCtx c, int q0, int q1) {
    if (c.flags[1]) return;
    int i = q0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q1) return;
    const int4 T = c.tets_col[i];
    if (!vertex_active(c, T.x)) return;
    const float4 X0 = c.x_s[T.x], X1 = c.x_s[T.y], X2 = c.x_s[T.z], X3 = c.x_s[T.w];
    const f3 e1 = sub(xyz(X1), xyz(X0)), e2 = sub(xyz(X2), xyz(X0)), e3 = sub(xyz(X3), xyz(X0));
    const f3 g1 = cross(e2, e3), g2 = cross(e3, e1), g3 = cross(e1, e2);
    const f3 g0 = mk(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
    const float C = dot(e1, g1) - c.vol6_col[i];
    const float at = c.alpha_vol;
    const float den = at + X0.w * dot(g0, g0) + X1.w * dot(g1, g1) + X2.w * dot(g2, g2) + X3.w * dot(g3, g3);
    if (den == 0.f) return;
    const float lam = c.tlambda[i];
    const float dl = (-C - at * lam) / den;
    c.x_s[T.x] = make_float4(X0.x + X0.w * dl * g0.x, X0.y + X0.w * dl * g0.y, X0.z + X0.w * dl * g0.z, X0.w);
    c.x_s[T.y] = make_float4(X1.x + X1.w * dl * g1.x, X1.y + X1.w * dl * g1.y, X1.z + X1.w * dl * g1.z, X1.w);
    c.x_s[T.z] = make_float4(X2.x + X2.w * dl * g2.x, X2.y + X2.w * dl * g2.y, X2.z + X2.w * dl * g2.z, X2.w);
    c.x_s[T.w] = make_float4(X3.x + X3.w * dl * g3.x, X3.y + X3.w * dl * g3.y, X3.z + X3.w * dl * g3.z, X3.w);
    c.tlambda[i] = lam + dl;
}

// End of an iteration: count it, and with early exit stop once converged.
__global__ void k_iter_end(DevCtx c, int early_exit) {
    if (c.flags[1]) return;
    c.stats->iterations += 1ull;
    if (early_exit && c.flags[0] == 0) c.flags[1] = 1;
}

// Alg. 4 update: v = (x - x^n) / dt.
__global__ void k_update(DevCtx c, const float4* __restrict__ x, float4* vel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) { c.flags[1] = 0; c.stats->steps += 1ull; }
    if (i >= c.n_verts || !vertex_active(c, i)) return;
    float4 X = x[i], N = c.x_n[i];
    float inv = 1.f / c.p.dt;
    vel[i] = make_float4((X.x - N.x) * inv, (X.y - N.y) * inv, (X.z - N.z) * inv, vel[i].w);
}

__global__ void k_rest_lengths(const int2* edges_col, const float4* __restrict__ x, float* rest, int ne) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    int2 e = edges_col[i];
    rest[i] = len(sub(xyz(x[e.x]), xyz(x[e.y])));
}

__global__ void k_tet_vol6(const int4* tets_col, const float4* __restrict__ x, float* vol6, int nt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int4 T = tets_col[i];
    const f3 a = xyz(x[T.x]);
    vol6[i] = dot(sub(xyz(x[T.y]), a), cross(sub(xyz(x[T.z]), a), sub(xyz(x[T.w]), a)));
}

__global__ void k_load_regions(DevCtx c, const float4* planes, const int* count, int cap) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)c.n_verts * cap;
    if (idx >= total) return;
    int v = (int)(idx / cap), j = (int)(idx % cap);
    int n = count[v];
    if (j == 0) { c.count[v] = (unsigned)n; c.dmin_drop[v] = 0xFFFFFFFFu; }
    if (j < n && j < c.p.K) c.planes[(size_t)v * c.p.K + j] = planes[(size_t)v * cap + j];
}

__global__ void k_dmin_export(DevCtx c, float* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n_verts) return;
    unsigned code = c.dmin_drop[i];
    out[i] = (code == 0xFFFFFFFFu) ? __int_as_float(0x7f800000) : ord2f(code);
}

// ------------------------------------------------------------- launchers

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// The planes of one kind (BIG: of its oversized primitives): the scan into
// the pair buffer pb, the narrow phase over it, and the fused pass that runs
// only if pb overflowed.
template <int QK, bool BIG>
static void launch_emit(const DevCtx& c, const float4* x, const PairOut& po, const PairBuf& pb, int G,
                        cudaStream_t st) {
    cudaMemsetAsync(pb.count, 0, sizeof(u64), st);
    if (BIG) k_emit_big<QK, MODE_BIGQ><<<G, EMIT_WARPS * 32, 0, st>>>(c, x, po, pb);
    else k_emit<QK, MODE_BIGQ><<<G, EMIT_WARPS * 32, 0, st>>>(c, x, po, pb);
    k_pair_narrow<QK, BIG><<<G, 256, 0, st>>>(c, x, po, pb);
    if (BIG) k_emit_big<QK, MODE_PLANES, false, true><<<G, EMIT_WARPS * 32, 0, st>>>(c, x, po, pb);
    else k_emit<QK, MODE_PLANES, true><<<G, EMIT_WARPS * 32, 0, st>>>(c, x, po, pb);
}

void launch_build(const DevCtx& c, const float4* x, cudaStream_t st, int mode, const PairOutHost* poh,
                  unsigned* tile_sums, int n_buckets_total, StageTimer* tm, const SideStream* side) {
    PairOut po{};
    if (poh) {
        for (int k = 0; k < 3; ++k) { po.out[k] = poh->out[k]; po.cap[k] = poh->cap[k]; }
        po.count = poh->count;
    }
    cudaMemsetAsync(c.ext_bits, 0, 3 * sizeof(unsigned), st);
    cudaMemsetAsync(c.ext_sum, 0, 3 * sizeof(u64), st);
    cudaMemsetAsync(c.big_count, 0, 2 * sizeof(unsigned), st);
    cudaMemsetAsync(c.bucket_count, 0, (size_t)(n_buckets_total + 1) * sizeof(unsigned), st);
    cudaMemsetAsync(c.bucket_fill, 0, (size_t)n_buckets_total * sizeof(unsigned), st);
    cudaMemsetAsync(c.sched, 0, N_SCHED * sizeof(unsigned), st);
    if (tm) tm->mark(ST_MISC, st);
    if (c.n_items > 0) k_extent<<<nblk(c.n_items, 256), 256, 0, st>>>(c, x);
    if (tm) tm->mark(ST_GRID_EXTENT, st);
    if (c.n_items > 0) k_bucket_count<<<nblk(c.n_items, 256), 256, 0, st>>>(c, x);
    if (tm) tm->mark(ST_GRID_COUNT, st);
    int n = n_buckets_total + 1;
    int tiles = nblk(n, SCAN_TILE);
    k_scan_tiles<<<tiles, SCAN_THREADS, 0, st>>>(c, c.bucket_count, n, tile_sums);
    k_scan_top<<<1, SCAN_THREADS, 0, st>>>(c, tile_sums, tiles);
    k_scan_apply<<<tiles, SCAN_THREADS, 0, st>>>(c, c.bucket_count, n, tile_sums);
    if (tm) tm->mark(ST_GRID_SCAN, st);
    if (c.n_items > 0) k_bucket_scatter<<<nblk(c.n_items, 256), 256, 0, st>>>(c, x);
    if (tm) tm->mark(ST_GRID_SCATTER, st);
    cudaMemsetAsync(c.unit_count, 0, 3 * sizeof(unsigned), st);
    int nqb = c.bucket_base[KIND_VQ];
    k_make_units<<<nblk(nqb, 256), 256, 0, st>>>(c);
    if (tm) tm->mark(ST_GRID_UNITS, st);
    const int G = c.n_sm * (c.emit_bps > 0 ? c.emit_bps : 8);
    if (mode == MODE_PLANES) {
        // The emission kernels only add planes through count atomics, so they are
        // independent: with a side stream (and no per-stage timing) the edge-edge
        // and point-point ones run beside the vertex-face and oversized ones (two
        // branches of similar length that fill each other's tails).
        const bool fork = side && !tm;
        cudaStream_t sb = st;
        if (fork) {
            cudaEventRecord(side->fork, st);
            cudaStreamWaitEvent(side->s, side->fork, 0);
            sb = side->s;
        }
        const PairBuf bq{c.bq, c.bq_count, c.bq_cap}, eq{c.eq, c.eq_count, c.eq_cap}, none{nullptr, nullptr, 0};
        if (c.n_tris > 0) launch_emit<KIND_TRI, false>(c, x, po, bq, G, st);
        if (tm) tm->mark(ST_EMIT_VF, st);
        if (c.n_tris > 0) launch_emit<KIND_TRI, true>(c, x, po, bq, G, st);
        if (tm) tm->mark(ST_EMIT_VF_BIG, st);
        if (c.n_edges > 0) launch_emit<KIND_EDGE, false>(c, x, po, eq, G, sb);
        if (tm) tm->mark(ST_EMIT_EE, st);
        if (c.n_edges > 0) launch_emit<KIND_EDGE, true>(c, x, po, bq, G, st);
        if (tm) tm->mark(ST_EMIT_EE_BIG, st);
        if (c.n_pts > 1) k_emit<KIND_PT, MODE_PLANES><<<G, EMIT_WARPS * 32, 0, sb>>>(c, x, po, none);
        if (c.n_pts > 0 && c.n_free > 0)
            k_emit_big<KIND_EDGE, MODE_PLANES, true><<<G, EMIT_WARPS * 32, 0, sb>>>(c, x, po, none);
        if (tm) tm->mark(ST_EMIT_PP, st);
        if (fork) {
            cudaEventRecord(side->join, sb);
            cudaStreamWaitEvent(st, side->join, 0);
        }
    } else {
        const PairBuf none{nullptr, nullptr, 0};
        if (c.n_tris > 0) {
            k_emit<KIND_TRI, MODE_PAIRS><<<G, EMIT_WARPS * 32, 0, st>>>(c, x, po, none);
            k_emit_big<KIND_TRI, MODE_PAIRS><<<G, EMIT_WARPS * 32, 0, st>>>(c, x, po, none);
        }
        if (c.n_edges > 0) {
            k_emit<KIND_EDGE, MODE_PAIRS><<<G, EMIT_WARPS * 32, 0, st>>>(c, x, po, none);
            k_emit_big<KIND_EDGE, MODE_PAIRS><<<G, EMIT_WARPS * 32, 0, st>>>(c, x, po, none);
        }
        if (c.n_pts > 1) k_emit<KIND_PT, MODE_PAIRS><<<G, EMIT_WARPS * 32, 0, st>>>(c, x, po, none);
    }
}

// persistent blocks of k_project_short per SM (128 threads each): as many as
// are resident at once, found by configure_kernels
// (atomic: contexts may be created, and the static projection set up, on
// other threads while launches read them)
static std::atomic<int> g_short_blocks_per_sm{4};
#define SHORT_BLOCKS_PER_SM g_short_blocks_per_sm.load(std::memory_order_relaxed)
static std::atomic<int> g_heavy_blocks_per_sm{4};
#define HEAVY_BLOCKS_PER_SM g_heavy_blocks_per_sm.load(std::memory_order_relaxed)

cudaError_t configure_kernels() {
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_project_short<true>, 128, 0);
    if (e == cudaSuccess && nb > 0) g_short_blocks_per_sm.store(nb, std::memory_order_relaxed);
    nb = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_project_heavy<true>, PROJ_WARPS * 32, 0);
    if (e == cudaSuccess && nb > 0) g_heavy_blocks_per_sm.store(nb, std::memory_order_relaxed);
    return e;
}

void launch_clear_regions(const DevCtx& c, cudaStream_t st) {
    cudaMemsetAsync(c.count, 0, (size_t)c.n_verts * sizeof(unsigned), st);
    cudaMemsetAsync(c.dmin_drop, 0xFF, (size_t)c.n_verts * sizeof(unsigned), st);
}

void launch_project(const DevCtx& c, const float4* xb, float4* xio, unsigned char* halt, cudaStream_t st) {
    long threads = (long)c.n_verts * 32;
    cudaMemsetAsync(c.work_count, 0, 4 * sizeof(unsigned), st);
    if (threads > 0) {
        k_project<false><<<nblk(c.n_verts, 256), 256, 0, st>>>(c, xb, xio, xio, halt);
        k_project_heavy<false><<<c.n_sm * HEAVY_BLOCKS_PER_SM, PROJ_WARPS * 32, 0, st>>>(c, xb, xio, xio, halt);
        k_project_short<false><<<c.n_sm * SHORT_BLOCKS_PER_SM, 128, 0, st>>>(c, xb, xio, xio, halt);
    }
}

void launch_predict(const DevCtx& c, const float4* x, const float4* v, cudaStream_t st) {
    cudaMemsetAsync(c.lambda, 0, (size_t)(c.n_dist > 0 ? c.n_dist : 1) * sizeof(float), st);
    if (c.n_tets > 0) cudaMemsetAsync(c.tlambda, 0, (size_t)c.n_tets * sizeof(float), st);
    cudaMemsetAsync(c.flags, 0, 2 * sizeof(int), st);
    if (c.n_verts > 0) k_predict<<<nblk(c.n_verts, 256), 256, 0, st>>>(c, x, v);
}

void launch_iteration(const DevCtx& c, float4* x, cudaStream_t st, const int* color_off, int n_colors,
                      unsigned* tile_sums, int n_buckets_total, int early_exit, StageTimer* tm,
                      const SideStream* side, const int* tcolor_off, int n_tcolors) {
    if (c.n_verts > 0) k_iter_begin<<<nblk(c.n_verts, 256), 256, 0, st>>>(c);
    launch_build(c, x, st, MODE_PLANES, nullptr, tile_sums, n_buckets_total, tm, side);
    for (int k = 0; k < n_colors; ++k) {
        int e0 = color_off[k], e1 = color_off[k + 1];
        if (e1 > e0) k_xpbd_color<<<nblk(e1 - e0, 256), 256, 0, st>>>(c, e0, e1);
    }
    for (int k = 0; k < n_tcolors; ++k) {
        int q0 = tcolor_off[k], q1 = tcolor_off[k + 1];
        if (q1 > q0) k_xpbd_tet_color<<<nblk(q1 - q0, 256), 256, 0, st>>>(c, q0, q1);
    }
    if (tm) tm->mark(ST_XPBD, st);
    if (c.p.delta > 0.f && c.phi && c.n_verts > 0)
        k_response<<<nblk(c.n_verts, RESP_WARPS * 32), RESP_WARPS * 32, 0, st>>>(c, x);
    if (tm) tm->mark(ST_RESPONSE, st);
    long threads = (long)c.n_verts * 32;
    cudaMemsetAsync(c.work_count, 0, 4 * sizeof(unsigned), st);
    if (threads > 0) k_project<true><<<nblk(c.n_verts, 256), 256, 0, st>>>(c, x, c.x_s, x, nullptr);
    if (tm) tm->mark(ST_PROJECT, st);
    if (threads > 0) k_project_heavy<true><<<c.n_sm * HEAVY_BLOCKS_PER_SM, PROJ_WARPS * 32, 0, st>>>(c, x, c.x_s, x, nullptr);
    if (tm) tm->mark(ST_PROJECT_HEAVY, st);
    if (threads > 0) k_project_short<true><<<c.n_sm * SHORT_BLOCKS_PER_SM, 128, 0, st>>>(c, x, c.x_s, x, nullptr);
    if (tm) tm->mark(ST_PROJECT_SHORT, st);
    k_iter_end<<<1, 1, 0, st>>>(c, early_exit);
}

void launch_update(const DevCtx& c, const float4* x, float4* v, cudaStream_t st) {
    if (c.n_verts > 0) k_update<<<nblk(c.n_verts, 256), 256, 0, st>>>(c, x, v);
    else k_update<<<1, 32, 0, st>>>(c, x, v);
}

void launch_rest_state(const DevCtx& c, const float4* x, cudaStream_t st) {
    if (c.n_dist > 0) k_rest_lengths<<<nblk(c.n_dist, 256), 256, 0, st>>>(c.edges_col, x, (float*)c.rest_col, c.n_dist);
    if (c.n_tets > 0) k_tet_vol6<<<nblk(c.n_tets, 256), 256, 0, st>>>(c.tets_col, x, c.vol6_col, c.n_tets);
}

void launch_load_regions(const DevCtx& c, const float4* planes, const int* count, int cap, cudaStream_t st) {
    long total = (long)c.n_verts * cap;
    if (total > 0) k_load_regions<<<nblk(total, 256), 256, 0, st>>>(c, planes, count, cap);
}

void launch_dmin_export(const DevCtx& c, float* out, cudaStream_t st) {
    if (c.n_verts > 0) k_dmin_export<<<nblk(c.n_verts, 256), 256, 0, st>>>(c, out);
}

}  // namespace ccfr

// ------------------------------------------------ projection without allocation
//
// ccfr_project_static runs the projection (k_project + k_project_heavy) on
// regions the caller already holds, for callers that cannot allocate device
// memory at all.  Its scratch (queue of violated vertices, overflow codes,
// counters) is the file-scope array below: every GPU that loads the library
// holds it until the process exits, and every call shares it.

#include <cstddef>
#include <mutex>

#include "ccfr.h"

namespace ccfr {

constexpr int STATIC_MAX_VERTS = 1 << 18;   // 262,144 vertices

struct StaticScratch {
    DevStats stats;
    int flags[2];
    unsigned work_count[4];
    unsigned pad_[10];
    int4 work[STATIC_MAX_VERTS];
    unsigned dmin[STATIC_MAX_VERTS];
};

static __device__ __align__(256) StaticScratch g_static_scratch;

// Overflow codes for the projection: the caller's smallest dropped d (float,
// +inf = none) in the order-preserving encoding the kernels read.
__global__ void k_static_dmin(const float* dmin_drop, unsigned* out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d = dmin_drop ? dmin_drop[i] : __int_as_float(0x7f800000);
    out[i] = (d == __int_as_float(0x7f800000)) ? 0xFFFFFFFFu : f2ord(d);
}

namespace {

struct StaticSetup {
    StaticScratch* ptr = nullptr;
    int n_sm = 0;
    bool ready = false;
};
constexpr int MAX_DEVICES = 64;
StaticSetup g_setup[MAX_DEVICES];
std::mutex g_setup_mutex;

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in) and the kernels'
// shared-memory limit.
ccfr_status static_setup(int dev, StaticSetup** out) {
    if (dev < 0 || dev >= MAX_DEVICES) return CCFR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    StaticSetup& s = g_setup[dev];
    if (!s.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return CCFR_ERR_CUDA;
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) return CCFR_ERR_CUDA;
        if (configure_kernels() != cudaSuccess) return CCFR_ERR_CUDA;
        s.ptr = (StaticScratch*)p;
        s.n_sm = nsm;
        s.ready = true;
    }
    *out = &s;
    return CCFR_OK;
}

}  // namespace
}  // namespace ccfr

extern "C" ccfr_status ccfr_project_static(const float* x, float* x_io, const float* planes, const int* count,
                                          const float* dmin_drop, int n_verts, int capacity,
                                          const ccfr_params* params, unsigned char* halt_out, void* stream) {
    using namespace ccfr;
    if (!x || !x_io || !params || n_verts < 0 || capacity < 1 || capacity > 65535) return CCFR_ERR_INVALID_ARG;
    if (n_verts > STATIC_MAX_VERTS) return CCFR_ERR_INVALID_ARG;     // beyond the scratch array
    if (n_verts > 0 && (!planes || !count)) return CCFR_ERR_INVALID_ARG;
    if (((uintptr_t)x & 15u) || ((uintptr_t)x_io & 15u) || ((uintptr_t)planes & 15u)) return CCFR_ERR_INVALID_ARG;
    if (!(params->eps_retract >= 0.f) || !(params->eps_dep > 0.f) || !(params->tau_feas >= 0.f) ||
        params->max_passes < 0 || params->max_passes > 64 || !(params->r > 0.f))
        return CCFR_ERR_INVALID_ARG;
    if (n_verts == 0) return CCFR_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCFR_ERR_CUDA;
    StaticSetup* su = nullptr;
    ccfr_status st = static_setup(dev, &su);
    if (st != CCFR_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    StaticScratch* sc = su->ptr;
    // what must start at zero: the queue length, the flags and the counters
    cudaError_t e = cudaMemsetAsync(sc, 0, offsetof(StaticScratch, work), s);
    if (e != cudaSuccess) return CCFR_ERR_CUDA;
    DevCtx c{};
    c.p.r = params->r;
    c.p.two_r = 2.f * params->r;
    c.p.xi = params->xi;
    c.p.pad = params->pad;
    c.p.eps = params->eps_retract;
    c.p.eps_dep = params->eps_dep;
    c.p.tau = params->tau_feas;
    c.p.max_passes = params->max_passes;
    c.p.K = capacity;
    c.p.short_max = short_list_max(capacity);
    c.n_verts = n_verts;
    c.planes = const_cast<float4*>((const float4*)planes);
    c.count = const_cast<unsigned*>((const unsigned*)count);
    c.dmin_drop = sc->dmin;
    c.flags = sc->flags;
    c.stats = &sc->stats;
    c.work = sc->work;
    c.work_count = sc->work_count;
    c.n_sm = su->n_sm;
    k_static_dmin<<<nblk(n_verts, 256), 256, 0, s>>>(dmin_drop, sc->dmin, n_verts);
    k_project<false><<<nblk(n_verts, 256), 256, 0, s>>>(c, (const float4*)x, (float4*)x_io, (float4*)x_io, halt_out);
    k_project_heavy<false><<<c.n_sm * HEAVY_BLOCKS_PER_SM, PROJ_WARPS * 32, 0, s>>>(c, (const float4*)x, (float4*)x_io,
                                                                         (float4*)x_io, halt_out);
    k_project_short<false><<<c.n_sm * SHORT_BLOCKS_PER_SM, 128, 0, s>>>(c, (const float4*)x, (float4*)x_io,
                                                                       (float4*)x_io, halt_out);
    return (cudaGetLastError() == cudaSuccess) ? CCFR_OK : CCFR_ERR_CUDA;
}

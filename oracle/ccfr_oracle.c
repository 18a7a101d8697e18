/*
 * FP64 CPU oracle for Convex Collision-Free Regions (CCFR).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow restatement of the
 * method that the CUDA library is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load it; the library never
 * does, and the two share no source, header, table or helper.
 *
 * What it follows (paper sections, equations and algorithms):
 *   - candidate predicate: padded AABB overlap, pad = r + xi/2 + delta/2
 *     (Sec. 4.1), evaluated in binary32 with the topological exclusions of
 *     Alg. 3;
 *   - narrow phase: Alg. 3 (VF, EE, FV) with the contact normal of Eq. 1 and
 *     the mass-weighted half-space of Eq. 2-3, the point-point variant for
 *     isolated particles;
 *   - projection: Alg. 2 (projectOntoConvexRegion) calling Alg. 1
 *     (Plesnik's orthogonalProjection), with the retraction and the halt of
 *     Sec. 3.2;
 *   - step: Alg. 4 (prediction, per-iteration detection, XPBD sweep,
 *     projection, max-step clamp, convergence, implicit-Euler update).
 *
 * Readings of passages that are silent, garbled or inconsistent (each one is
 * named where it is used):
 *   R1  Eq. 2 sign: a plane stores d = s * (dist - xi) and the constraint is
 *       (x' - x) . n + d >= 0, the form Alg. 2 and Alg. 3 use.
 *   R2  FV normal points from the passive vertex towards the active face
 *       (the face side gets -n of the vertex-face pair).
 *   R3  FV share is w_face / (w_face + w_vertex), so the two shares sum to 1.
 *   R4  generalized inverse mass of a primitive point = sum(bary_i * w_i).
 *   R5  point-point pairs only between isolated vertices (point primitives).
 *   R6  Alg. 2 runs n_max + 1 passes; the extra pass is the check that returns
 *       x' once nothing is violated.
 *   R7  Alg. 1 uses the new (n, b) for j = m and appends the new (n, b).
 *   R8  one tolerance eps_dep for every test in Alg. 1, on absolute values;
 *       at most 3 ERO directions (a fourth normal in 3-D is dependent).
 *   R9  one retraction per pass: the pass's result (the projected boundary
 *       position x* of Sec. 3.2) is shifted back by eps towards the build
 *       position x (reset to x when closer than eps).  Alg. 2's listing places
 *       the retraction after every Alg. 1 call; but Alg. 1 assumes its iterate
 *       lies on the planes already taken, and a retraction between calls moves
 *       it off them, so the next call misses its own plane by about
 *       eps d / |y| and the final check halts the vertex.  Sec. 3.2 describes
 *       the retraction as a numerical margin applied to the projected position,
 *       which is what this reading does (see the halting study).
 *   R10 planes are sorted once by (rho, key) at the pass input.
 *   R11 final check rho_k >= -tau_feas on the result, else halt.
 *   R12 every iteration restarts the XPBD candidate from the prediction and
 *       builds regions at the current collision-free iterate x_c.
 *   R13 converged <=> no vertex was shortened by more than 2 eps.
 *   R14 the max-step clamp is relative to x_c.
 *   R15 internal model: edge-distance constraints with rest lengths from the
 *       rest shape, greedy first-fit edge colours in canonical edge order,
 *       colours swept in ascending order.
 *   R16 plane capacity K: a vertex with more than K planes is not projected;
 *       its step is clamped to max(0, min_k d_k) over all its planes, which
 *       satisfies every plane because |n . y| <= |y|.
 *
 * Scenes that mix rods, cloth, volumes and particles (the paper's coupled
 * codimensional scene, Sec. 5) use these further readings:
 *   X1  bending: extra distance constraints ("links") given by the scene (for
 *       cloth the two vertices opposite each interior edge, for rods every
 *       second neighbour), each with its own compliance; rest lengths from the
 *       rest shape.
 *   X2  volume: per tetrahedron (x0, x1, x2, x3) the constraint
 *       C = 6 V - 6 V0 with 6 V = (x1 - x0) . ((x2 - x0) x (x3 - x0)), signed,
 *       V0 from the rest shape, one compliance for all tetrahedra.
 *   X3  constraint order: the edges (canonical order) and then the links form
 *       one list coloured greedily first-fit; its colours are swept in
 *       ascending order, then the tetrahedra, coloured the same way.
 *   X4  vertex-edge pairs between isolated points and free edges (edges of no
 *       triangle, i.e. rods): a particle meets a wire through no pair of
 *       Alg. 3.  The plane is built as in Alg. 3 with the point on the segment
 *       and its barycentric inverse mass (R4); pair kind 3.
 *   X5  a vertex that belongs to links or tetrahedra but to no edge or triangle
 *       (the interior of a volume) takes no part in collision: it is neither an
 *       isolated point nor a vertex-face query.
 *
 * Parity pins: every function here is pinned by tests against closed forms,
 * brute force or invariants (see tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned long long u64;

typedef struct {
    double r, xi, delta;
    float pad;           /* binary32 AABB enlargement */
    double eps;          /* retraction margin (Sec. 3.2) */
    double eps_dep;      /* Alg. 1 dependence tolerance */
    double tau_feas;     /* final feasibility tolerance */
    double band;         /* width of the decision bands reported to tests */
    double dep_band;     /* factor of the dependence-test band: |beta| in [eps_dep / f, eps_dep f]
                            is reported (f > 1; 0 = 10) */
    double cond_band;    /* an Alg. 1 division by beta with |beta| / |direction| below this is
                            reported (an ill-conditioned step; 0 = none) */
    int n_max;           /* Alg. 2 n_maxIterations */
    int iters;           /* Alg. 4 solver iterations */
    int capacity;        /* plane capacity K per vertex, 0 = unbounded */
    int early_exit;      /* stop iterating once converged (R13) */
    double dt, g[3], compliance;
    double k_resp;       /* response stiffness k (Sec. 3.3) */
    double delta_v;      /* smooth transition width of the occlusion factor */
    double mu_s, mu_k;   /* static and kinetic friction coefficients */
} orc_params;

/* ---------------------------------------------------------------- helpers */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double norm3(const double *a) { return sqrt(dot3(a, a)); }
static double clamp01(double s) { return s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s); }

/* plane key: kind (0 VF, 1 EE, 2 VV) in the top bits, then the two primitive ids */
static u64 make_key(int kind, int a, int b) {
    return ((u64)kind << 62) | ((u64)(unsigned)a << 31) | (u64)(unsigned)b;
}

/* ------------------------------------------------- candidate predicate */

/* Padded box of a primitive in binary32: lo = fl32(min - pad), hi = fl32(max + pad)
 * (Sec. 4.1 enlarges every AABB by r + xi/2 + delta/2). */
typedef struct { float lo[3], hi[3]; } fbox;

static fbox box_of(const float *x4, const int *vid, int nv, float pad) {
    fbox b;
    for (int a = 0; a < 3; ++a) {
        float mn = x4[4 * vid[0] + a], mx = mn;
        for (int i = 1; i < nv; ++i) {
            float c = x4[4 * vid[i] + a];
            if (c < mn) mn = c;
            if (c > mx) mx = c;
        }
        volatile float lo = mn - pad, hi = mx + pad;
        b.lo[a] = lo;
        b.hi[a] = hi;
    }
    return b;
}

static int overlap(const fbox *p, const fbox *q) {
    for (int a = 0; a < 3; ++a)
        if (!(p->lo[a] <= q->hi[a] && q->lo[a] <= p->hi[a])) return 0;
    return 1;
}

typedef struct { int a, b; } ipair;
typedef struct { ipair *v; long n, cap; } pairvec;

static void pv_push(pairvec *pv, int a, int b) {
    if (pv->n == pv->cap) {
        pv->cap = pv->cap ? 2 * pv->cap : 1024;
        pv->v = (ipair *)realloc(pv->v, sizeof(ipair) * pv->cap);
    }
    pv->v[pv->n].a = a;
    pv->v[pv->n].b = b;
    pv->n++;
}

static int cmp_int(const void *x, const void *y) {
    int a = *(const int *)x, b = *(const int *)y;
    return (a > b) - (a < b);
}

/* Sort pairs lexicographically: a counting sort on the first element (range
 * [0, na)), then each run sorted by the second element (runs in parallel).
 * The same order as one lexicographic sort of the pairs. */
static void sort_pairs(pairvec *pv, int na) {
    long n = pv->n;
    if (n <= 1) return;
    long *start = (long *)calloc((size_t)na + 1, sizeof(long));
    for (long i = 0; i < n; ++i) start[pv->v[i].a + 1]++;
    for (int a = 0; a < na; ++a) start[a + 1] += start[a];
    long *fill = (long *)malloc(sizeof(long) * (size_t)(na > 0 ? na : 1));
    memcpy(fill, start, sizeof(long) * (size_t)na);
    int *b = (int *)malloc(sizeof(int) * (size_t)n);
    for (long i = 0; i < n; ++i) b[fill[pv->v[i].a]++] = pv->v[i].b;
#pragma omp parallel for schedule(dynamic, 256)
    for (int a = 0; a < na; ++a) {
        if (start[a + 1] - start[a] > 1) qsort(b + start[a], (size_t)(start[a + 1] - start[a]), sizeof(int), cmp_int);
        for (long i = start[a]; i < start[a + 1]; ++i) { pv->v[i].a = a; pv->v[i].b = b[i]; }
    }
    free(b);
    free(fill);
    free(start);
}

/* Append b's pairs to a (b is left untouched). */
static void pv_append(pairvec *a, const pairvec *b) {
    for (long i = 0; i < b->n; ++i) pv_push(a, b->v[i].a, b->v[i].b);
}

/* Constraints beyond the collision edges (readings X1-X3): distance links
 * with their compliances, rest lengths and tetrahedra with their rest volumes
 * (6 V0).  A null pointer means none. */
typedef struct {
    int nl;
    const int *links;              /* nl x 2 */
    const double *link_compliance; /* nl */
    const double *link_rest;       /* nl */
    int ntet;
    const int *tets;               /* ntet x 4 */
    const double *vol6_rest;       /* ntet */
    double volume_compliance;
} orc_extra;

typedef struct {
    int n, ne, nt;
    const int *edges, *tris;
    const float *w;      /* inverse masses (as stored in binary32) */
    int *iso;            /* isolated vertices */
    int niso;
    unsigned char *collides;   /* per vertex: takes part in collision (X5) */
    unsigned char *free_edge;  /* per edge: belongs to no triangle (X4) */
} topo;

static long find_edge(const int *edges, int ne, int a, int b) {
    long lo = 0, hi = ne;
    while (lo < hi) {
        long mid = (lo + hi) / 2;
        const int *e = edges + 2 * mid;
        if (e[0] < a || (e[0] == a && e[1] < b)) lo = mid + 1; else hi = mid;
    }
    return (lo < ne && edges[2 * lo] == a && edges[2 * lo + 1] == b) ? lo : -1;
}

static void topo_init_ext(topo *t, int n, const int *edges, int ne, const int *tris, int nt, const float *x4,
                          const orc_extra *ex) {
    t->n = n; t->ne = ne; t->nt = nt; t->edges = edges; t->tris = tris;
    float *w = (float *)malloc(sizeof(float) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) w[i] = x4[4 * i + 3];
    t->w = w;
    char *used = (char *)calloc(n > 0 ? n : 1, 1);   /* 1: collision edge, 2: link or tetrahedron only */
    for (int e = 0; e < ne; ++e) { used[edges[2 * e]] = 1; used[edges[2 * e + 1]] = 1; }
    for (int f = 0; f < nt; ++f)
        for (int k = 0; k < 3; ++k) used[tris[3 * f + k]] = 1;
    if (ex) {
        for (int l = 0; l < ex->nl; ++l)
            for (int k = 0; k < 2; ++k) if (!used[ex->links[2 * l + k]]) used[ex->links[2 * l + k]] = 2;
        for (int q = 0; q < ex->ntet; ++q)
            for (int k = 0; k < 4; ++k) if (!used[ex->tets[4 * q + k]]) used[ex->tets[4 * q + k]] = 2;
    }
    t->iso = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    t->collides = (unsigned char *)malloc(n > 0 ? n : 1);
    t->niso = 0;
    for (int i = 0; i < n; ++i) {
        if (!used[i]) t->iso[t->niso++] = i;
        t->collides[i] = used[i] != 2;
    }
    free(used);
    t->free_edge = (unsigned char *)malloc(ne > 0 ? ne : 1);
    for (int e = 0; e < ne; ++e) t->free_edge[e] = 1;
    for (int f = 0; f < nt; ++f)
        for (int k = 0; k < 3; ++k) {
            int a = tris[3 * f + k], b = tris[3 * f + (k + 1) % 3];
            long e = find_edge(edges, ne, a < b ? a : b, a < b ? b : a);
            if (e >= 0) t->free_edge[e] = 0;
        }
}

static void topo_init(topo *t, int n, const int *edges, int ne, const int *tris, int nt, const float *x4) {
    topo_init_ext(t, n, edges, ne, tris, nt, x4, NULL);
}

static void topo_free(topo *t) { free((void *)t->w); free(t->iso); free(t->collides); free(t->free_edge); }

/* Pair filters (Alg. 3 exclusions): a VF pair needs the vertex outside the
 * triangle, an EE pair needs e < e' and no shared vertex, a VV pair needs two
 * isolated points p < q; every pair needs one movable vertex. */
static int vf_ok(const topo *t, int v, int f) {
    const int *T = t->tris + 3 * f;
    if (!t->collides[v]) return 0;   /* X5 */
    if (v == T[0] || v == T[1] || v == T[2]) return 0;
    return (t->w[v] > 0 || t->w[T[0]] > 0 || t->w[T[1]] > 0 || t->w[T[2]] > 0);
}

static int ee_ok(const topo *t, int e, int f) {
    if (!(e < f)) return 0;
    const int *A = t->edges + 2 * e, *B = t->edges + 2 * f;
    if (A[0] == B[0] || A[0] == B[1] || A[1] == B[0] || A[1] == B[1]) return 0;
    return (t->w[A[0]] > 0 || t->w[A[1]] > 0 || t->w[B[0]] > 0 || t->w[B[1]] > 0);
}

static int vv_ok(const topo *t, int p, int q) {
    if (!(p < q)) return 0;
    return (t->w[p] > 0 || t->w[q] > 0);
}

/* X4: an isolated point against a free edge (a point is never an endpoint). */
static int ve_ok(const topo *t, int p, int e) {
    if (!t->free_edge[e]) return 0;
    const int *E = t->edges + 2 * e;
    return (t->w[p] > 0 || t->w[E[0]] > 0 || t->w[E[1]] > 0);
}

/* Sort-and-sweep over x of the item boxes; returns all (query, item) pairs
 * whose binary32 boxes overlap.  kind 0 = VF (queries vertices, items tris),
 * 1 = EE (edges, edges), 2 = VV (isolated points, isolated points),
 * 3 = VE (isolated points, edges; X4). */
typedef struct { float lo; int idx; } sortkey;
static int cmp_sk(const void *x, const void *y) {
    const sortkey *p = (const sortkey *)x, *q = (const sortkey *)y;
    if (p->lo < q->lo) return -1;
    if (p->lo > q->lo) return 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

static fbox kind_query_box(const topo *t, const float *x4, int kind, int i, float pad) {
    int vid[2];
    if (kind == 0) { vid[0] = i; return box_of(x4, vid, 1, pad); }
    if (kind == 1) return box_of(x4, t->edges + 2 * i, 2, pad);
    vid[0] = t->iso[i];
    return box_of(x4, vid, 1, pad);
}

static fbox kind_item_box(const topo *t, const float *x4, int kind, int j, float pad) {
    int vid[1];
    if (kind == 0) return box_of(x4, t->tris + 3 * j, 3, pad);
    if (kind == 1 || kind == 3) return box_of(x4, t->edges + 2 * j, 2, pad);
    vid[0] = t->iso[j];
    return box_of(x4, vid, 1, pad);
}

static int kind_ok(const topo *t, int kind, int i, int j) {
    if (kind == 0) return vf_ok(t, i, j);
    if (kind == 1) return ee_ok(t, i, j);
    if (kind == 3) return ve_ok(t, t->iso[i], j);
    return vv_ok(t, t->iso[i], t->iso[j]);
}

#define N_PAIR_KINDS 4

static void broad_kind(const topo *t, const float *x4, float pad, int kind, int brute, pairvec *out) {
    int nq = kind == 0 ? t->n : (kind == 1 ? t->ne : t->niso);
    int ni = kind == 0 ? t->nt : ((kind == 1 || kind == 3) ? t->ne : t->niso);
    if (nq <= 0 || ni <= 0) return;
    fbox *ib = (fbox *)malloc(sizeof(fbox) * ni);
    for (int j = 0; j < ni; ++j) ib[j] = kind_item_box(t, x4, kind, j, pad);
    if (brute) {
        for (int i = 0; i < nq; ++i) {
            fbox q = kind_query_box(t, x4, kind, i, pad);
            for (int j = 0; j < ni; ++j)
                if (overlap(&q, &ib[j]) && kind_ok(t, kind, i, j))
                    pv_push(out, kind >= 2 ? t->iso[i] : i, kind == 2 ? t->iso[j] : j);
        }
    } else {
        sortkey *sk = (sortkey *)malloc(sizeof(sortkey) * ni);
        double maxext = 0.0;
        for (int j = 0; j < ni; ++j) {
            sk[j].lo = ib[j].lo[0];
            sk[j].idx = j;
            double e = (double)ib[j].hi[0] - (double)ib[j].lo[0];
            if (e > maxext) maxext = e;
        }
        qsort(sk, ni, sizeof(sortkey), cmp_sk);
        /* queries are independent: each thread collects its own pairs; the
         * result is sorted below, so it does not depend on the threads */
#pragma omp parallel
        {
            pairvec mine = {0, 0, 0};
#pragma omp for schedule(dynamic, 256)
            for (int i = 0; i < nq; ++i) {
                fbox q = kind_query_box(t, x4, kind, i, pad);
                double from = (double)q.lo[0] - maxext;
                int lo = 0, hi = ni;  /* first index with sk.lo >= from */
                while (lo < hi) {
                    int mid = (lo + hi) / 2;
                    if ((double)sk[mid].lo < from) lo = mid + 1; else hi = mid;
                }
                for (int s = lo; s < ni && sk[s].lo <= q.hi[0]; ++s) {
                    int j = sk[s].idx;
                    if (overlap(&q, &ib[j]) && kind_ok(t, kind, i, j))
                        pv_push(&mine, kind >= 2 ? t->iso[i] : i, kind == 2 ? t->iso[j] : j);
                }
            }
#pragma omp critical
            pv_append(out, &mine);
            free(mine.v);
        }
        free(sk);
    }
    free(ib);
    sort_pairs(out, kind == 0 ? t->n : (kind == 1 ? t->ne : t->n));
}

/* Candidate sets C_VF, C_EE, C_VV, C_VE.  Two-call protocol: with out == NULL
 * only the counts are written.  out receives VF pairs, then EE, VV and VE
 * (point, edge), each sorted lexicographically. */
long orc_candidates_ext(const float *x4, int n, const int *edges, int ne, const int *tris, int nt,
                        const orc_extra *ex, float pad, int brute, int *out, long counts[N_PAIR_KINDS]) {
    topo t;
    topo_init_ext(&t, n, edges, ne, tris, nt, x4, ex);
    long total = 0;
    for (int k = 0; k < N_PAIR_KINDS; ++k) {
        pairvec pv = {0, 0, 0};
        broad_kind(&t, x4, pad, k, brute, &pv);
        counts[k] = pv.n;
        if (out) {
            for (long i = 0; i < pv.n; ++i) {
                out[2 * (total + i)] = pv.v[i].a;
                out[2 * (total + i) + 1] = pv.v[i].b;
            }
        }
        total += pv.n;
        free(pv.v);
    }
    topo_free(&t);
    return total;
}

long orc_candidates(const float *x4, int n, const int *edges, int ne, const int *tris, int nt,
                    float pad, int brute, int *out, long counts[N_PAIR_KINDS]) {
    return orc_candidates_ext(x4, n, edges, ne, tris, nt, NULL, pad, brute, out, counts);
}

/* ------------------------------------------------------- closest points */

/* Closest point on triangle abc to p by Voronoi-region classification
 * (Ericson, Real-Time Collision Detection, Sec. 5.1.5).  bary holds the
 * weights of a, b, c. */
void orc_closest_point_triangle(const double *p, const double *a, const double *b, const double *c,
                                double *q, double *bary) {
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    sub3(b, a, ab); sub3(c, a, ac); sub3(p, a, ap);
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    double u, v, w;
    if (d1 <= 0.0 && d2 <= 0.0) { u = 1; v = 0; w = 0; goto done; }
    sub3(p, b, bp);
    double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) { u = 0; v = 1; w = 0; goto done; }
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        double s = d1 / (d1 - d3);
        u = 1 - s; v = s; w = 0; goto done;
    }
    sub3(p, c, cp);
    double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { u = 0; v = 0; w = 1; goto done; }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double s = d2 / (d2 - d6);
        u = 1 - s; v = 0; w = s; goto done;
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
        double s = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        u = 0; v = 1 - s; w = s; goto done;
    }
    {
        double den = 1.0 / (va + vb + vc);
        v = vb * den; w = vc * den; u = 1.0 - v - w;
    }
done:
    bary[0] = u; bary[1] = v; bary[2] = w;
    for (int i = 0; i < 3; ++i) q[i] = u * a[i] + v * b[i] + w * c[i];
}

/* Closest points of segments p1q1 and p2q2 with clamping (Ericson,
 * Sec. 5.1.9).  Parallel segments (a*e - b*b <= 1e-12 * a * e) take s = 0 on
 * the first segment, then t from it, then re-clamp s. */
void orc_closest_segments(const double *p1, const double *q1, const double *p2, const double *q2,
                          double *s_out, double *t_out) {
    double d1[3], d2[3], r[3];
    sub3(q1, p1, d1); sub3(q2, p2, d2); sub3(p1, p2, r);
    double a = dot3(d1, d1), e = dot3(d2, d2), f = dot3(d2, r);
    double s, t;
    if (a <= 0.0 && e <= 0.0) { s = t = 0.0; }
    else if (a <= 0.0) { s = 0.0; t = clamp01(f / e); }
    else {
        double c = dot3(d1, r);
        if (e <= 0.0) { t = 0.0; s = clamp01(-c / a); }
        else {
            double b = dot3(d1, d2);
            double den = a * e - b * b;
            s = (den > 1e-12 * a * e) ? clamp01((b * f - c * e) / den) : 0.0;
            t = (b * s + f) / e;
            if (t < 0.0) { t = 0.0; s = clamp01(-c / a); }
            else if (t > 1.0) { t = 1.0; s = clamp01((b - c) / a); }
        }
    }
    *s_out = s; *t_out = t;
}

/* Closest point of segment ab to p: parameter t = (p - a).(b - a) / |b - a|^2
 * clamped to [0, 1] (t = 0 for a degenerate segment). */
double orc_closest_point_segment(const double *p, const double *a, const double *b) {
    double ab[3], ap[3];
    sub3(b, a, ab); sub3(p, a, ap);
    double l2 = dot3(ab, ab);
    return l2 > 0.0 ? clamp01(dot3(ap, ab) / l2) : 0.0;
}

/* ---------------------------------------------------------- narrow phase */

typedef struct {
    int v;               /* receiving vertex */
    double n[3], d, phi;
    u64 key;
} plane_rec;

typedef struct { plane_rec *p; long n, cap; } planevec;

static void plv_push(planevec *pv, int v, const double *n, double d, double phi, u64 key);

/* Append b's planes to a. */
static void plv_append(planevec *a, const planevec *b) {
    if (a->n + b->n > a->cap) {
        a->cap = a->n + b->n;
        a->p = (plane_rec *)realloc(a->p, sizeof(plane_rec) * (a->cap > 0 ? a->cap : 1));
    }
    if (b->n) memcpy(a->p + a->n, b->p, sizeof(plane_rec) * b->n);
    a->n += b->n;
}

static void plv_push(planevec *pv, int v, const double *n, double d, double phi, u64 key) {
    if (pv->n == pv->cap) {
        pv->cap = pv->cap ? 2 * pv->cap : 4096;
        pv->p = (plane_rec *)realloc(pv->p, sizeof(plane_rec) * pv->cap);
    }
    plane_rec *r = &pv->p[pv->n++];
    r->v = v; r->n[0] = n[0]; r->n[1] = n[1]; r->n[2] = n[2]; r->d = d; r->phi = phi; r->key = key;
}

/* One accepted pair: emit (n, s_A * phi) to every movable vertex of side A and
 * (-n, s_B * phi) to every movable vertex of side B (Alg. 3; Eq. 2-3; R1-R4).
 * Returns 1 when the pair is accepted (phi < 2r). */
static int emit_pair(planevec *out, const double *w, const double *A, const double *B,
                     const int *va, const double *ba, int na, const int *vb, const double *bb, int nb,
                     const orc_params *P, u64 key, unsigned char *vflag) {
    double diff[3];
    sub3(A, B, diff);
    double dist = norm3(diff);
    double phi = dist - P->xi;
    if (vflag && fabs(phi - 2.0 * P->r) <= P->band) {
        for (int i = 0; i < na; ++i) {
#pragma omp atomic
            vflag[va[i]] |= 2;
        }
        for (int i = 0; i < nb; ++i) {
#pragma omp atomic
            vflag[vb[i]] |= 2;
        }
    }
    if (dist == 0.0) return 0;            /* touching at build time: skipped (Sec. 4.1) */
    if (!(phi < 2.0 * P->r)) return 0;
    double wa = 0.0, wb = 0.0;
    for (int i = 0; i < na; ++i) wa += ba[i] * w[va[i]];
    for (int i = 0; i < nb; ++i) wb += bb[i] * w[vb[i]];
    double W = wa + wb;
    if (W == 0.0) return 0;
    double n[3] = {diff[0] / dist, diff[1] / dist, diff[2] / dist};
    double mn[3] = {-n[0], -n[1], -n[2]};
    for (int i = 0; i < na; ++i)
        if (w[va[i]] > 0) plv_push(out, va[i], n, (wa / W) * phi, phi, key);
    for (int i = 0; i < nb; ++i)
        if (w[vb[i]] > 0) plv_push(out, vb[i], mn, (wb / W) * phi, phi, key);
    return 1;
}

static int narrow_vf(planevec *out, const double *x3, const double *w, const topo *t, int v, int f,
                      const orc_params *P, unsigned char *vflag) {
    const int *T = t->tris + 3 * f;
    double q[3], bary[3];
    orc_closest_point_triangle(x3 + 3 * v, x3 + 3 * T[0], x3 + 3 * T[1], x3 + 3 * T[2], q, bary);
    double one = 1.0;
    return emit_pair(out, w, x3 + 3 * v, q, &v, &one, 1, T, bary, 3, P, make_key(0, v, f), vflag);
}

static int narrow_ee(planevec *out, const double *x3, const double *w, const topo *t, int e, int f,
                      const orc_params *P, unsigned char *vflag) {
    const int *A = t->edges + 2 * e, *B = t->edges + 2 * f;
    double s, u;
    orc_closest_segments(x3 + 3 * A[0], x3 + 3 * A[1], x3 + 3 * B[0], x3 + 3 * B[1], &s, &u);
    double pa[3], pb[3];
    for (int i = 0; i < 3; ++i) {
        pa[i] = (1 - s) * x3[3 * A[0] + i] + s * x3[3 * A[1] + i];
        pb[i] = (1 - u) * x3[3 * B[0] + i] + u * x3[3 * B[1] + i];
    }
    double ba[2] = {1 - s, s}, bb[2] = {1 - u, u};
    return emit_pair(out, w, pa, pb, A, ba, 2, B, bb, 2, P, make_key(1, e, f), vflag);
}

static int narrow_vv(planevec *out, const double *x3, const double *w, int p, int q,
                      const orc_params *P, unsigned char *vflag) {
    double one = 1.0;
    return emit_pair(out, w, x3 + 3 * p, x3 + 3 * q, &p, &one, 1, &q, &one, 1, P, make_key(2, p, q), vflag);
}

/* X4: isolated point p against free edge e; side A is the point. */
static int narrow_ve(planevec *out, const double *x3, const double *w, const topo *t, int p, int e,
                      const orc_params *P, unsigned char *vflag) {
    const int *E = t->edges + 2 * e;
    double u = orc_closest_point_segment(x3 + 3 * p, x3 + 3 * E[0], x3 + 3 * E[1]);
    double q[3];
    for (int i = 0; i < 3; ++i) q[i] = (1 - u) * x3[3 * E[0] + i] + u * x3[3 * E[1] + i];
    double one = 1.0, bb[2] = {1 - u, u};
    return emit_pair(out, w, x3 + 3 * p, q, &p, &one, 1, E, bb, 2, P, make_key(3, p, e), vflag);
}

/* Per-vertex region = CSR list of planes sorted by key. */
typedef struct {
    int n;
    long *offs;          /* n + 1 */
    plane_rec *p;
    long total;
    double *dlimit;      /* +inf, or the step bound of an overflowing vertex (R16) */
    unsigned char *vflag;/* bit0 overflow, bit1 band pair */
    long cand[N_PAIR_KINDS], acc[N_PAIR_KINDS];
} orc_regions;

static int cmp_plane(const void *x, const void *y) {
    const plane_rec *p = (const plane_rec *)x, *q = (const plane_rec *)y;
    if (p->v != q->v) return p->v < q->v ? -1 : 1;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return 0;
}

static orc_regions *build_regions(const double *x3, const double *w, const topo *t, const orc_params *P) {
    int n = t->n;
    /* the candidate predicate reads binary32 positions */
    float *x4 = (float *)malloc(sizeof(float) * 4 * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) x4[4 * i + a] = (float)x3[3 * i + a];
        x4[4 * i + 3] = (float)w[i];
    }
    orc_regions *R = (orc_regions *)calloc(1, sizeof(orc_regions));
    R->n = n;
    R->vflag = (unsigned char *)calloc(n > 0 ? n : 1, 1);
    planevec pv = {0, 0, 0};
    for (int kind = 0; kind < N_PAIR_KINDS; ++kind) {
        pairvec c = {0, 0, 0};
        broad_kind(t, x4, P->pad, kind, 0, &c);
        R->cand[kind] = c.n;
        long acc_k = 0;
        /* pairs are independent; the planes are sorted by (vertex, key) below */
#pragma omp parallel reduction(+ : acc_k)
        {
            planevec mine = {0, 0, 0};
#pragma omp for schedule(dynamic, 1024)
            for (long i = 0; i < c.n; ++i) {
                int acc;
                if (kind == 0) acc = narrow_vf(&mine, x3, w, t, c.v[i].a, c.v[i].b, P, R->vflag);
                else if (kind == 1) acc = narrow_ee(&mine, x3, w, t, c.v[i].a, c.v[i].b, P, R->vflag);
                else if (kind == 2) acc = narrow_vv(&mine, x3, w, c.v[i].a, c.v[i].b, P, R->vflag);
                else acc = narrow_ve(&mine, x3, w, t, c.v[i].a, c.v[i].b, P, R->vflag);
                acc_k += acc;
            }
#pragma omp critical
            plv_append(&pv, &mine);
            free(mine.p);
        }
        R->acc[kind] += acc_k;
        free(c.v);
    }
    free(x4);
    /* CSR by receiving vertex (a counting sort), each vertex's planes sorted
     * by key: the order of one sort by (vertex, key), which is unique */
    R->total = pv.n;
    R->offs = (long *)calloc(n + 1, sizeof(long));
    for (long i = 0; i < pv.n; ++i) R->offs[pv.p[i].v + 1]++;
    for (int i = 0; i < n; ++i) R->offs[i + 1] += R->offs[i];
    R->p = (plane_rec *)malloc(sizeof(plane_rec) * (pv.n > 0 ? pv.n : 1));
    {
        long *fill = (long *)malloc(sizeof(long) * (n > 0 ? n : 1));
        memcpy(fill, R->offs, sizeof(long) * (size_t)n);
        for (long i = 0; i < pv.n; ++i) R->p[fill[pv.p[i].v]++] = pv.p[i];
        free(fill);
    }
    free(pv.p);
#pragma omp parallel for schedule(dynamic, 256)
    for (int i = 0; i < n; ++i)
        if (R->offs[i + 1] - R->offs[i] > 1)
            qsort(R->p + R->offs[i], (size_t)(R->offs[i + 1] - R->offs[i]), sizeof(plane_rec), cmp_plane);
    R->dlimit = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        R->dlimit[i] = INFINITY;
        long cnt = R->offs[i + 1] - R->offs[i];
        if (P->capacity > 0 && cnt > P->capacity) {
            double m = INFINITY;
            for (long k = R->offs[i]; k < R->offs[i + 1]; ++k) if (R->p[k].d < m) m = R->p[k].d;
            R->dlimit[i] = m;
            R->vflag[i] |= 1;
        }
    }
    return R;
}

void orc_regions_free(orc_regions *R) {
    if (!R) return;
    free(R->offs); free(R->p); free(R->dlimit); free(R->vflag); free(R);
}

orc_regions *orc_build_ext(const double *x3, const float *x4w, int n, const int *edges, int ne,
                           const int *tris, int nt, const orc_extra *ex, const orc_params *P) {
    topo t;
    topo_init_ext(&t, n, edges, ne, tris, nt, x4w, ex);
    double *w = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) w[i] = (double)x4w[4 * i + 3];
    orc_regions *R = build_regions(x3, w, &t, P);
    free(w);
    topo_free(&t);
    return R;
}

orc_regions *orc_build(const double *x3, const float *x4w, int n, const int *edges, int ne,
                       const int *tris, int nt, const orc_params *P) {
    return orc_build_ext(x3, x4w, n, edges, ne, tris, nt, NULL, P);
}

long orc_regions_total(const orc_regions *R) { return R->total; }

/* Planes per vertex and the band flags of a region build, without exporting
 * the planes (for scenes whose plane lists are large). */
void orc_region_counts(const double *x3, const float *x4w, int n, const int *edges, int ne, const int *tris,
                       int nt, const orc_params *P, long *count, unsigned char *vflag) {
    orc_regions *R = orc_build_ext(x3, x4w, n, edges, ne, tris, nt, NULL, P);
    for (int i = 0; i < n; ++i) {
        count[i] = R->offs[i + 1] - R->offs[i];
        vflag[i] = R->vflag[i];
    }
    orc_regions_free(R);
}

void orc_regions_export(const orc_regions *R, long *offs, double *planes4, double *phi, u64 *key,
                        double *dlimit, unsigned char *vflag, long *cand_acc) {
    for (int i = 0; i <= R->n; ++i) offs[i] = R->offs[i];
    for (long k = 0; k < R->total; ++k) {
        planes4[4 * k + 0] = R->p[k].n[0];
        planes4[4 * k + 1] = R->p[k].n[1];
        planes4[4 * k + 2] = R->p[k].n[2];
        planes4[4 * k + 3] = R->p[k].d;
        phi[k] = R->p[k].phi;
        key[k] = R->p[k].key;
    }
    for (int i = 0; i < R->n; ++i) { dlimit[i] = R->dlimit[i]; vflag[i] = R->vflag[i]; }
    for (int k = 0; k < N_PAIR_KINDS; ++k) { cand_acc[k] = R->cand[k]; cand_acc[N_PAIR_KINDS + k] = R->acc[k]; }
}

/* Threads of the parallel loops (<= 0: all host cores); returns the count
 * in use.  Results do not depend on it: every loop is over independent
 * queries, pairs or vertices, and every output is sorted or per vertex. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n <= 0) n = omp_get_num_procs();
    omp_set_num_threads(n);
    return n;
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------- Alg. 1 */

typedef struct {
    int m;               /* |V| */
    double V[3][3], A[3][3], B[3];
} ero_state;

static int near_eps(double v, double eps, double f) {
    if (!(f > 1.0)) f = 10.0;
    v = fabs(v);
    return v >= eps / f && v <= eps * f;
}

/* Plesnik's orthogonal projection step (Alg. 1; R7, R8).  xt is updated in
 * place; x0 is the pass's starting point.  *band is set when a dependence
 * test falls within a factor 10 of eps_dep. */
/* An Alg. 1 step moving along `dir` by (numerator / beta): its result
 * changes by |dir| / |beta| times any error of the numerator (the planes' and
 * the iterate's rounding), so a small |beta| / |dir| is an ill-conditioned
 * step, reported as a band. */
static int ill_conditioned(double beta, const double *dir, double cond_band) {
    return cond_band > 0.0 && fabs(beta) < cond_band * norm3(dir);
}

static void ortho_projection(double *xt, const double *x0, const double *n, double b, ero_state *S,
                             double eps_dep, double dep_band, double cond_band, int *band) {
    if (S->m == 0) {
        double beta0 = dot3(n, n);
        if (near_eps(beta0, eps_dep, dep_band)) *band = 1;
        if (fabs(beta0) < eps_dep) return;
        double a = (b - dot3(n, xt)) / beta0;
        for (int i = 0; i < 3; ++i) xt[i] += a * n[i];
        for (int i = 0; i < 3; ++i) { S->V[0][i] = n[i]; S->A[0][i] = n[i]; }
        S->B[0] = b;
        S->m = 1;
        return;
    }
    int m = S->m;
    const double *n0 = S->A[0];
    double b0 = S->B[0];
    double dn[3];
    sub3(n, n0, dn);
    double beta_u = dot3(dn, S->V[m - 1]);
    double alpha_u = b - dot3(n, xt);
    if (near_eps(beta_u, eps_dep, dep_band)) *band = 1;
    if (fabs(beta_u) < eps_dep) return;
    double u[3], wv[3];
    if (ill_conditioned(beta_u, S->V[m - 1], cond_band)) *band = 1;
    for (int i = 0; i < 3; ++i) u[i] = xt[i] + (alpha_u / beta_u) * S->V[m - 1][i];
    for (int i = 0; i < 3; ++i) wv[i] = x0[i] + n[i];
    for (int j = 1; j <= m; ++j) {
        const double *nj = (j < m) ? S->A[j] : n;
        double bj = (j < m) ? S->B[j] : b;
        double dnj[3];
        sub3(nj, n0, dnj);
        double beta_w = dot3(dnj, S->V[j - 1]);
        if (near_eps(beta_w, eps_dep, dep_band)) *band = 1;
        if (fabs(beta_w) > eps_dep) {
            double alpha_w = bj - b0 - dot3(dnj, wv);
            if (ill_conditioned(beta_w, S->V[j - 1], cond_band)) *band = 1;
            for (int i = 0; i < 3; ++i) wv[i] += (alpha_w / beta_w) * S->V[j - 1][i];
        }
    }
    double vnew[3];
    sub3(wv, u, vnew);
    double vn = norm3(vnew);
    if (near_eps(vn, eps_dep, dep_band)) *band = 1;
    if (vn > eps_dep) {
        double beta_new = dot3(n0, vnew);
        if (near_eps(beta_new, eps_dep, dep_band)) *band = 1;
        if (fabs(beta_new) < eps_dep) {
            for (int i = 0; i < 3; ++i) xt[i] = u[i];
        } else {
            double alpha_new = b0 - dot3(n0, u);
            if (ill_conditioned(beta_new, vnew, cond_band)) *band = 1;
            for (int i = 0; i < 3; ++i) xt[i] = u[i] + (alpha_new / beta_new) * vnew[i];
        }
        if (m < 3) {
            for (int i = 0; i < 3; ++i) { S->V[m][i] = vnew[i]; S->A[m][i] = n[i]; }
            S->B[m] = b;
            S->m = m + 1;
        }
    }
}

/* Alg. 1 applied to k planes n_i . x = b_i in order, from x0, with no
 * retraction: the pure Plesnik recursion (for the closed-form pin). */
void orc_ortho_sequence(const double *x0, const double *normals, const double *b, int k,
                        double eps_dep, double *out) {
    ero_state S;
    S.m = 0;
    double xt[3] = {x0[0], x0[1], x0[2]};
    int band = 0;
    for (int i = 0; i < k; ++i) {
        if (S.m >= 3) break;
        ortho_projection(xt, x0, normals + 3 * i, b[i], &S, eps_dep, 0.0, 0.0, &band);
    }
    out[0] = xt[0]; out[1] = xt[1]; out[2] = xt[2];
}

/* ------------------------------------------------------------- Alg. 2 */

typedef struct { double rho; u64 key; long idx; } ord_rec;
static int cmp_ord(const void *x, const void *y) {
    const ord_rec *p = (const ord_rec *)x, *q = (const ord_rec *)y;
    if (p->rho < q->rho) return -1;
    if (p->rho > q->rho) return 1;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return 0;
}

/* Whether the decision "plane pl violated or not" at the iterate xt can
 * change the pass's result (used only to report band decisions): the plane
 * would be the pass's first violation (which decides between returning x'
 * and retracting the pass result), or Alg. 1 would store it or move the
 * iterate.  A plane identical to one already taken, met with rho = 0 up to
 * rounding right after the iterate was projected onto that plane, is a no-op
 * either way. */
static int decision_matters(const double *xt, const double *x0, const double *pl, double b, const ero_state *S,
                            int nv, const orc_params *P) {
    if (nv == 0) return 1;
    if (S->m >= 3) return 0;
    double xc[3] = {xt[0], xt[1], xt[2]};
    ero_state Sc = *S;
    int unused = 0;
    ortho_projection(xc, x0, pl, b, &Sc, P->eps_dep, P->dep_band, 0.0, &unused);
    if (Sc.m != S->m) return 1;
    double d[3];
    sub3(xc, xt, d);
    return norm3(d) > P->band;
}

/* projectOntoConvexRegion for one vertex (Alg. 2; R6, R9, R10, R11).
 * planes4[k] = (n_k, d_k).  Returns 1 on halt.  nviol receives the number of
 * violated planes seen in the first pass.  *band is set when a decision of
 * the algorithm falls inside a band (rho near 0 where the decision can change
 * the result, near-tied sort keys of distinct planes, dependence tests within
 * a factor dep_band of eps_dep, ill-conditioned Alg. 1 steps (cond_band),
 * |dx| near eps). */
static int project_vertex(const double *x, double *xp, const double *planes4, const u64 *keys, long np,
                          const orc_params *P, int *nviol, int *band) {
    *nviol = 0;
    if (np == 0) return 0;
    ord_rec *ord = (ord_rec *)malloc(sizeof(ord_rec) * np);
    double y[3];
    sub3(xp, x, y);
    for (long k = 0; k < np; ++k) {
        ord[k].rho = dot3(y, planes4 + 4 * k) + planes4[4 * k + 3];
        ord[k].key = keys[k];
        ord[k].idx = k;
    }
    qsort(ord, np, sizeof(ord_rec), cmp_ord);
    int halted = 1;
    for (int pass = 0; pass < P->n_max + 1; ++pass) {
        double xt[3] = {xp[0], xp[1], xp[2]}, x0[3] = {xp[0], xp[1], xp[2]};
        ero_state S;
        S.m = 0;
        int nv = 0;
        for (long s = 0; s < np; ++s) {
            const double *pl = planes4 + 4 * ord[s].idx;
            double dx[3];
            sub3(xt, x, dx);
            double rho = dot3(dx, pl) + pl[3];
            if (fabs(rho) <= P->band && decision_matters(xt, x0, pl, dot3(pl, x) - pl[3], &S, nv, P)) *band = 1;
            if (rho >= 0.0) continue;
            /* a near-tie in the sort order between distinct planes changes the
             * visiting order on a lower-precision replay */
            if (pass == 0) {
                for (long o = 0; o < np; ++o) {
                    if (o == s) continue;
                    const double *q = planes4 + 4 * ord[o].idx;
                    if (fabs(ord[o].rho - ord[s].rho) <= P->band) {
                        double dn = fabs(q[0] - pl[0]) + fabs(q[1] - pl[1]) + fabs(q[2] - pl[2]);
                        if (dn > 1e-5 || fabs(q[3] - pl[3]) > P->band) *band = 1;
                    }
                }
            }
            double b = dot3(pl, x) - pl[3];
            nv++;
            if (S.m < 3) ortho_projection(xt, x0, pl, b, &S, P->eps_dep, P->dep_band, P->cond_band, band);
        }
        /* R9: the pass result (the projected boundary position) is retracted
         * once by eps towards the build position x, or reset to x when it is
         * closer to x than eps (Sec. 3.2) */
        if (nv > 0) {
            double dn[3];
            sub3(xt, x, dn);
            double L = norm3(dn);
            if (fabs(L - P->eps) <= P->band) *band = 1;
            if (L > P->eps) {
                for (int i = 0; i < 3; ++i) xt[i] = x[i] + (L - P->eps) * dn[i] / L;
            } else {
                for (int i = 0; i < 3; ++i) xt[i] = x[i];
            }
        }
        if (pass == 0) *nviol = nv;
        if (nv == 0) { halted = 0; break; }
        xp[0] = xt[0]; xp[1] = xt[1]; xp[2] = xt[2];
    }
    if (halted) { xp[0] = x[0]; xp[1] = x[1]; xp[2] = x[2]; }
    free(ord);
    return halted;
}

/* Final feasibility check (R11): every plane holds within tau at y. */
static int feasible(const double *x, const double *y, const double *planes4, long np, double tau) {
    double dx[3];
    sub3(y, x, dx);
    for (long k = 0; k < np; ++k)
        if (dot3(dx, planes4 + 4 * k) + planes4[4 * k + 3] < -tau) return 0;
    return 1;
}

/* Step bound of an overflowing vertex (R16). */
static void clamp_len(const double *x, double *y, double lim) {
    double dx[3];
    sub3(y, x, dx);
    double L = norm3(dx);
    if (lim <= 0.0) { y[0] = x[0]; y[1] = x[1]; y[2] = x[2]; return; }
    if (L > lim) for (int i = 0; i < 3; ++i) y[i] = x[i] + dx[i] * (lim / L);
}

/* Alg. 2 over all vertices with given CSR planes.  x3: build positions;
 * xp3: in = candidate x', out = x*.  w: inverse masses (static vertices are
 * left untouched).  dlimit: per-vertex overflow bound (+inf = none).
 * halt/band/nviol: per-vertex outputs (may be NULL).  Returns #halts. */
long orc_project(const double *x3, double *xp3, const double *w, int n, const long *offs,
                 const double *planes4, const u64 *keys, const double *dlimit, const orc_params *P,
                 unsigned char *halt, unsigned char *band, int *nviol) {
    long halts = 0;
#pragma omp parallel for reduction(+ : halts) schedule(dynamic, 64)
    for (int v = 0; v < n; ++v) {
        int h = 0, bd = 0, nv = 0;
        if (w[v] > 0) {
            long o = offs[v], np = offs[v + 1] - offs[v];
            if (dlimit && isfinite(dlimit[v])) {
                clamp_len(x3 + 3 * v, xp3 + 3 * v, dlimit[v]);
            } else {
                h = project_vertex(x3 + 3 * v, xp3 + 3 * v, planes4 + 4 * o, keys + o, np, P, &nv, &bd);
                if (!h && !feasible(x3 + 3 * v, xp3 + 3 * v, planes4 + 4 * o, np, P->tau_feas)) {
                    h = 1;
                    for (int i = 0; i < 3; ++i) xp3[3 * v + i] = x3[3 * v + i];
                }
            }
        }
        halts += h;
        if (halt) halt[v] = (unsigned char)h;
        if (band) band[v] = (unsigned char)bd;
        if (nviol) nviol[v] = nv;
    }
    return halts;
}

/* -------------------------------------------------------------- Alg. 4 */

/* Greedy first-fit edge colouring in canonical edge order (R15). */
int orc_edge_colors(const int *edges, int ne, int n, int *color) {
    u64 *used = (u64 *)calloc(n > 0 ? n : 1, sizeof(u64));
    int ncol = 0;
    for (int e = 0; e < ne; ++e) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        u64 m = used[a] | used[b];
        int c = 0;
        while (c < 64 && (m >> c & 1ull)) ++c;
        if (c == 64) { free(used); return -1; }
        color[e] = c;
        used[a] |= 1ull << c;
        used[b] |= 1ull << c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(used);
    return ncol;
}

/* Greedy first-fit colouring of tetrahedra (no two of a colour share a vertex),
 * in tetrahedron order (X3). */
int orc_tet_colors(const int *tets, int ntet, int n, int *color) {
    u64 *used = (u64 *)calloc(n > 0 ? n : 1, sizeof(u64));
    int ncol = 0;
    for (int q = 0; q < ntet; ++q) {
        const int *T = tets + 4 * q;
        u64 m = used[T[0]] | used[T[1]] | used[T[2]] | used[T[3]];
        int c = 0;
        while (c < 64 && (m >> c & 1ull)) ++c;
        if (c == 64) { free(used); return -1; }
        color[q] = c;
        for (int k = 0; k < 4; ++k) used[T[k]] |= 1ull << c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(used);
    return ncol;
}

static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Six times the signed volume of each tetrahedron (X2). */
void orc_tet_volumes6(const double *x3, const int *tets, int ntet, double *out) {
    for (int q = 0; q < ntet; ++q) {
        const int *T = tets + 4 * q;
        double e1[3], e2[3], e3[3], c[3];
        sub3(x3 + 3 * T[1], x3 + 3 * T[0], e1);
        sub3(x3 + 3 * T[2], x3 + 3 * T[0], e2);
        sub3(x3 + 3 * T[3], x3 + 3 * T[0], e3);
        cross3(e2, e3, c);
        out[q] = dot3(e1, c);
    }
}

typedef struct {
    int iters_run;
    long planes, violated, halts, overflow, shortened;
    int any_band;
} orc_step_info;

/* ------------------------------------------------------ response (Sec. 3.3)
 *
 * Soft repulsion and friction on a vertex's contacts, applied after the XPBD
 * sweep and before the projection (Alg. 4, applyResponse; readings F1-F7).
 * A contact c of vertex v is one of its planes: normal n_c and the pair's gap
 * phi_c = dist - xi at the build position x.
 *  F1  the signed distance along the contact normal at the iterate y, with
 *      the other side held at its build position: g_c(y) = phi_c + n_c.(y - x);
 *  F7  active contacts: g_c < delta, at most RESP_CAP of them, the innermost
 *      by (g, pair key);
 *  F2  visibility weight w_c = prod over the other active contacts j of
 *      (1 - S((g_c - g_j) / delta_v)), S the cubic smoothstep 3t^2 - 2t^3
 *      clamped to [0, 1]; gaps and weights at the iterate before the response;
 *  F3  the energy (k/2) w_c max(0, delta - g_c)^2 as the XPBD constraint
 *      C = max(0, delta - g_c(y)) with compliance 1/(k w_c), a fresh
 *      multiplier every iteration (the contacts are rebuilt every iteration):
 *      y += w C / (w + 1/(k w_c dt^2)) n_c, w the vertex's inverse mass;
 *  F4  Gauss-Seidel over the active contacts in ascending (g, key) order;
 *  F5  friction (position-based, after the repulsion): for each contact in
 *      the same order whose repulsion moved y by depth > 0, t = the tangential
 *      part of the vertex's displacement since the substep start; |t| <
 *      mu_s depth: t is removed (static), else it is shortened by
 *      min(mu_k depth, |t|) (kinetic);
 *  F6  overflowed vertices (R16) get no response.
 * *band is set when a decision falls within `band` of its threshold (an
 * activation, a friction mode, the order of two distinct contacts). */
#define RESP_CAP 32

typedef struct { double g; u64 key; long k; } resp_entry;

static int cmp_resp(const void *a, const void *b) {
    const resp_entry *p = (const resp_entry *)a, *q = (const resp_entry *)b;
    if (p->g != q->g) return p->g < q->g ? -1 : 1;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return 0;
}

static double smoothstep01(double t) {
    if (t <= 0.0) return 0.0;
    if (t >= 1.0) return 1.0;
    return t * t * (3.0 - 2.0 * t);
}

void orc_response(double *y, const double *x, const double *xn, const double *planes4, const double *phi,
                  const u64 *keys, long np, double w, const orc_params *P, int *band) {
    if (!(P->delta > 0.0) || !(w > 0.0) || np <= 0) return;
    resp_entry *all = (resp_entry *)malloc(sizeof(resp_entry) * np);
    long nall = 0;
    for (long k = 0; k < np; ++k) {
        double d[3];
        sub3(y, x, d);
        double g = phi[k] + dot3(planes4 + 4 * k, d);
        if (band && fabs(g - P->delta) <= P->band) *band = 1;
        if (g < P->delta) { all[nall].g = g; all[nall].key = keys[k]; all[nall].k = k; nall++; }
    }
    qsort(all, nall, sizeof(resp_entry), cmp_resp);
    int na = nall < RESP_CAP ? (int)nall : RESP_CAP;
    /* near-tied gaps decide an order; two contacts whose normals agree to
     * 1e-4 commute to within 1e-4 of a correction (<= delta), far below any
     * tolerance, so only near-ties of distinctly oriented contacts are bands */
    for (int a = 1; a < (nall > RESP_CAP ? RESP_CAP + 1 : na); ++a) {
        const double *p0 = planes4 + 4 * all[a - 1].k, *p1 = planes4 + 4 * all[a].k;
        double dn = fmax(fabs(p0[0] - p1[0]), fmax(fabs(p0[1] - p1[1]), fabs(p0[2] - p1[2])));
        if (band && dn > 1e-4 && all[a].g - all[a - 1].g <= P->band) *band = 1;
    }
    double wt[RESP_CAP], depth[RESP_CAP];
    for (int a = 0; a < na; ++a) {
        double v = 1.0;
        for (int b = 0; b < na; ++b)
            if (b != a) v *= 1.0 - smoothstep01((all[a].g - all[b].g) / P->delta_v);
        wt[a] = v;
    }
    for (int a = 0; a < na; ++a) {
        const double *n = planes4 + 4 * all[a].k;
        double d[3];
        sub3(y, x, d);
        double C = P->delta - (phi[all[a].k] + dot3(n, d));
        depth[a] = 0.0;
        if (!(C > 0.0) || !(wt[a] > 0.0)) continue;
        double at = 1.0 / (P->k_resp * wt[a] * P->dt * P->dt);
        double corr = w * C / (w + at);
        for (int i = 0; i < 3; ++i) y[i] += corr * n[i];
        depth[a] = corr;
    }
    if (P->mu_s > 0.0 || P->mu_k > 0.0) {
        for (int a = 0; a < na; ++a) {
            if (!(depth[a] > 0.0)) continue;
            const double *n = planes4 + 4 * all[a].k;
            double d[3], t[3];
            sub3(y, xn, d);
            double dn = dot3(d, n);
            for (int i = 0; i < 3; ++i) t[i] = d[i] - dn * n[i];
            double tl = norm3(t);
            if (!(tl > 0.0)) continue;
            if (band && fabs(tl - P->mu_s * depth[a]) <= P->band) *band = 1;
            double f = (tl < P->mu_s * depth[a]) ? 1.0 : (P->mu_k * depth[a] / tl < 1.0 ? P->mu_k * depth[a] / tl : 1.0);
            for (int i = 0; i < 3; ++i) y[i] -= f * t[i];
        }
    }
    free(all);
}

/* One substep of Alg. 4 with the readings R12-R16 (and X1-X5 for the
 * constraints in ex).  x3, v3 are updated in place (FP64).  x4w supplies
 * inverse masses; rest[e] the edges' rest lengths.  vband (optional, per
 * vertex) collects band flags over all iterations. */
static int step_impl(double *x3, double *v3, const float *x4w, int n, const int *edges, int ne,
                     const int *tris, int nt, const double *rest, const orc_extra *ex, const orc_params *P,
                     unsigned char *vband, orc_step_info *info, unsigned char *halt_iter) {
    topo t;
    topo_init_ext(&t, n, edges, ne, tris, nt, x4w, ex);
    double *w = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) w[i] = (double)x4w[4 * i + 3];
    /* distance constraints: the edges, then the links (X1, X3) */
    const int nl = ex ? ex->nl : 0, ntet = ex ? ex->ntet : 0;
    const int nd = ne + nl;
    int *dpair = (int *)malloc(sizeof(int) * 2 * (nd > 0 ? nd : 1));
    double *drest = (double *)malloc(sizeof(double) * (nd > 0 ? nd : 1));
    double *dcomp = (double *)malloc(sizeof(double) * (nd > 0 ? nd : 1));
    for (int e = 0; e < ne; ++e) {
        dpair[2 * e] = edges[2 * e]; dpair[2 * e + 1] = edges[2 * e + 1];
        drest[e] = rest[e]; dcomp[e] = P->compliance;
    }
    for (int l = 0; l < nl; ++l) {
        dpair[2 * (ne + l)] = ex->links[2 * l]; dpair[2 * (ne + l) + 1] = ex->links[2 * l + 1];
        drest[ne + l] = ex->link_rest[l]; dcomp[ne + l] = ex->link_compliance[l];
    }
    int *color = (int *)malloc(sizeof(int) * (nd > 0 ? nd : 1));
    int ncol = orc_edge_colors(dpair, nd, n, color);
    int *tcolor = (int *)malloc(sizeof(int) * (ntet > 0 ? ntet : 1));
    int ntcol = ntet > 0 ? orc_tet_colors(ex->tets, ntet, n, tcolor) : 0;
    if (ncol < 0 || ntcol < 0) {
        free(w); free(color); free(tcolor); free(dpair); free(drest); free(dcomp); topo_free(&t);
        return -1;
    }
    size_t N3 = sizeof(double) * 3 * (n > 0 ? n : 1);
    double *xn = (double *)malloc(N3), *xt = (double *)malloc(N3), *xc = (double *)malloc(N3);
    double *xs = (double *)malloc(N3), *pre = (double *)malloc(N3);
    double *lambda = (double *)calloc(nd > 0 ? nd : 1, sizeof(double));
    double *tlambda = (double *)calloc(ntet > 0 ? ntet : 1, sizeof(double));
    memcpy(xn, x3, N3);
    memcpy(xc, x3, N3);
    double dt = P->dt;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a)
            xt[3 * i + a] = w[i] > 0 ? x3[3 * i + a] + dt * v3[3 * i + a] + dt * dt * P->g[a] : x3[3 * i + a];
    memset(info, 0, sizeof(*info));
    double atv = ex ? ex->volume_compliance / (dt * dt) : 0.0;
    unsigned char *bflag = (unsigned char *)calloc(n > 0 ? n : 1, 1);
    for (int it = 0; it < P->iters; ++it) {
        orc_regions *R = build_regions(xc, w, &t, P);
        info->planes += R->total;
        memcpy(xs, xt, N3);
        /* XPBD sweep of the distance constraints, colours ascending (R15, X3) */
        for (int c = 0; c < ncol; ++c) {
            /* constraints of one colour share no vertex */
#pragma omp parallel for schedule(static)
            for (int e = 0; e < nd; ++e) {
                if (color[e] != c) continue;
                int a = dpair[2 * e], b = dpair[2 * e + 1];
                double at = dcomp[e] / (dt * dt);
                double wsum = w[a] + w[b] + at;
                if (wsum == 0.0) continue;
                double dd[3];
                sub3(xs + 3 * a, xs + 3 * b, dd);
                double L = norm3(dd);
                if (L == 0.0) continue;
                double C = L - drest[e];
                double dl = (-C - at * lambda[e]) / wsum;
                for (int k = 0; k < 3; ++k) {
                    xs[3 * a + k] += w[a] * dl * dd[k] / L;
                    xs[3 * b + k] -= w[b] * dl * dd[k] / L;
                }
                lambda[e] += dl;
            }
        }
        /* then the volume constraints of the tetrahedra, colours ascending (X2, X3) */
        for (int c = 0; c < ntcol; ++c) {
#pragma omp parallel for schedule(static)
            for (int q = 0; q < ntet; ++q) {
                if (tcolor[q] != c) continue;
                const int *T = ex->tets + 4 * q;
                double e1[3], e2[3], e3[3], g[4][3];
                sub3(xs + 3 * T[1], xs + 3 * T[0], e1);
                sub3(xs + 3 * T[2], xs + 3 * T[0], e2);
                sub3(xs + 3 * T[3], xs + 3 * T[0], e3);
                cross3(e2, e3, g[1]);
                cross3(e3, e1, g[2]);
                cross3(e1, e2, g[3]);
                for (int k = 0; k < 3; ++k) g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);
                double C = dot3(e1, g[1]) - ex->vol6_rest[q];
                double den = atv;
                for (int i = 0; i < 4; ++i) den += w[T[i]] * dot3(g[i], g[i]);
                if (den == 0.0) continue;
                double dl = (-C - atv * tlambda[q]) / den;
                for (int i = 0; i < 4; ++i)
                    for (int k = 0; k < 3; ++k) xs[3 * T[i] + k] += w[T[i]] * dl * g[i][k];
                tlambda[q] += dl;
            }
        }
        /* contact response on every movable vertex, then the projection */
        if (P->delta > 0.0) {
#pragma omp parallel for schedule(dynamic, 64)
            for (int v = 0; v < n; ++v) {
                if (!(w[v] > 0) || isfinite(R->dlimit[v])) continue;
                long o = R->offs[v], np = R->offs[v + 1] - R->offs[v];
                if (np <= 0) continue;
                double *planes4 = (double *)malloc(sizeof(double) * 4 * np);
                double *phi = (double *)malloc(sizeof(double) * np);
                u64 *keys = (u64 *)malloc(sizeof(u64) * np);
                for (long k = 0; k < np; ++k) {
                    for (int a = 0; a < 3; ++a) planes4[4 * k + a] = R->p[o + k].n[a];
                    planes4[4 * k + 3] = R->p[o + k].d;
                    phi[k] = R->p[o + k].phi;
                    keys[k] = R->p[o + k].key;
                }
                int bd = 0;
                orc_response(xs + 3 * v, xc + 3 * v, xn + 3 * v, planes4, phi, keys, np, w[v], P, &bd);
                if (bd) bflag[v] = 1;
                free(planes4); free(phi); free(keys);
            }
        }
        memcpy(pre, xs, N3);
        int shortened = 0;
        long n_over = 0, n_viol = 0, n_halt = 0, n_short = 0;
        /* vertices are independent (each reads its own planes and iterate) */
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : n_over, n_viol, n_halt, n_short) \
    reduction(| : shortened)
        for (int v = 0; v < n; ++v) {
            double *y = xs + 3 * v;
            const double *x = xc + 3 * v;
            if (!(w[v] > 0)) { y[0] = x[0]; y[1] = x[1]; y[2] = x[2]; continue; }
            long o = R->offs[v], np = R->offs[v + 1] - R->offs[v];
            double *planes4 = (double *)malloc(sizeof(double) * 4 * (np > 0 ? np : 1));
            u64 *keys = (u64 *)malloc(sizeof(u64) * (np > 0 ? np : 1));
            for (long k = 0; k < np; ++k) {
                planes4[4 * k + 0] = R->p[o + k].n[0];
                planes4[4 * k + 1] = R->p[o + k].n[1];
                planes4[4 * k + 2] = R->p[o + k].n[2];
                planes4[4 * k + 3] = R->p[o + k].d;
                keys[k] = R->p[o + k].key;
            }
            int h = 0, nv = 0, bd = 0;
            if (isfinite(R->dlimit[v])) {
                clamp_len(x, y, R->dlimit[v]);
                n_over++;
            } else {
                h = project_vertex(x, y, planes4, keys, np, P, &nv, &bd);
            }
            clamp_len(x, y, P->r);   /* max-step clamp relative to x_c (R14) */
            if (!h && !feasible(x, y, planes4, np, P->tau_feas)) {
                h = 1;
                y[0] = x[0]; y[1] = x[1]; y[2] = x[2];
            }
            if (nv) n_viol++;
            n_halt += h;
            if (halt_iter) halt_iter[(size_t)it * n + v] = (unsigned char)h;
            double dd[3];
            sub3(y, pre + 3 * v, dd);
            if (norm3(dd) > 2.0 * P->eps) { shortened = 1; n_short++; }
            if (bd || (R->vflag[v] & 2)) bflag[v] = 1;
            free(planes4);
            free(keys);
        }
        info->overflow += n_over;
        info->violated += n_viol;
        info->halts += n_halt;
        info->shortened += n_short;
        orc_regions_free(R);
        memcpy(xc, xs, N3);
        info->iters_run = it + 1;
        if (P->early_exit && !shortened) break;
    }
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            v3[3 * i + a] = (xc[3 * i + a] - xn[3 * i + a]) / dt;
            x3[3 * i + a] = xc[3 * i + a];
        }
        if (bflag[i]) info->any_band = 1;
        if (vband) vband[i] |= bflag[i];
    }
    free(bflag);
    free(xn); free(xt); free(xc); free(xs); free(pre); free(lambda); free(w); free(color);
    free(tlambda); free(tcolor); free(dpair); free(drest); free(dcomp);
    topo_free(&t);
    return 0;
}

int orc_step_ext(double *x3, double *v3, const float *x4w, int n, const int *edges, int ne,
                 const int *tris, int nt, const double *rest, const orc_extra *ex, const orc_params *P,
                 unsigned char *vband, orc_step_info *info) {
    return step_impl(x3, v3, x4w, n, edges, ne, tris, nt, rest, ex, P, vband, info, NULL);
}

/* orc_step_ext that also records, per iteration and vertex, whether the
 * vertex halted (halt_iter[it * n + v], iters x n bytes; observability only). */
int orc_step_hist(double *x3, double *v3, const float *x4w, int n, const int *edges, int ne,
                  const int *tris, int nt, const double *rest, const orc_extra *ex, const orc_params *P,
                  unsigned char *vband, orc_step_info *info, unsigned char *halt_iter) {
    return step_impl(x3, v3, x4w, n, edges, ne, tris, nt, rest, ex, P, vband, info, halt_iter);
}

int orc_step(double *x3, double *v3, const float *x4w, int n, const int *edges, int ne,
             const int *tris, int nt, const double *rest, const orc_params *P,
             unsigned char *vband, orc_step_info *info) {
    return orc_step_ext(x3, v3, x4w, n, edges, ne, tris, nt, rest, NULL, P, vband, info);
}

void orc_rest_lengths(const double *x3, const int *edges, int ne, double *rest) {
    for (int e = 0; e < ne; ++e) {
        double d[3];
        sub3(x3 + 3 * edges[2 * e], x3 + 3 * edges[2 * e + 1], d);
        rest[e] = norm3(d);
    }
}

/* ------------------------------------------------------- invariant checks */

/* Distance from p to triangle abc and between two segments, FP64. */
double orc_point_triangle_distance(const double *p, const double *a, const double *b, const double *c) {
    double q[3], bary[3], d[3];
    orc_closest_point_triangle(p, a, b, c, q, bary);
    sub3(p, q, d);
    return norm3(d);
}

double orc_segment_distance(const double *p1, const double *q1, const double *p2, const double *q2) {
    double s, t, a[3], b[3], d[3];
    orc_closest_segments(p1, q1, p2, q2, &s, &t);
    for (int i = 0; i < 3; ++i) {
        a[i] = (1 - s) * p1[i] + s * q1[i];
        b[i] = (1 - t) * p2[i] + t * q2[i];
    }
    sub3(a, b, d);
    return norm3(d);
}

/* Minimum distance over non-adjacent VF, EE and VV pairs whose binary32 boxes
 * (enlarged by cutoff/2) overlap; pairs farther than cutoff are ignored and
 * the result is capped at cutoff.  The static-static pairs are skipped like
 * in the candidate predicate.  out3 = (min VF, min EE, min VV). */
void orc_min_distances(const double *x3, const float *x4w, int n, const int *edges, int ne,
                       const int *tris, int nt, double cutoff, double *out3) {
    topo t;
    topo_init(&t, n, edges, ne, tris, nt, x4w);
    float *x4 = (float *)malloc(sizeof(float) * 4 * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) x4[4 * i + a] = (float)x3[3 * i + a];
        x4[4 * i + 3] = x4w[4 * i + 3];
    }
    float pad = (float)(0.5 * cutoff) * 1.0001f;
    for (int kind = 0; kind < 3; ++kind) {
        double m = cutoff;
        pairvec c = {0, 0, 0};
        broad_kind(&t, x4, pad, kind, 0, &c);
        for (long i = 0; i < c.n; ++i) {
            double d;
            if (kind == 0) {
                const int *T = tris + 3 * c.v[i].b;
                d = orc_point_triangle_distance(x3 + 3 * c.v[i].a, x3 + 3 * T[0], x3 + 3 * T[1], x3 + 3 * T[2]);
            } else if (kind == 1) {
                const int *A = edges + 2 * c.v[i].a, *B = edges + 2 * c.v[i].b;
                d = orc_segment_distance(x3 + 3 * A[0], x3 + 3 * A[1], x3 + 3 * B[0], x3 + 3 * B[1]);
            } else {
                double dd[3];
                sub3(x3 + 3 * c.v[i].a, x3 + 3 * c.v[i].b, dd);
                d = norm3(dd);
            }
            if (d < m) m = d;
        }
        free(c.v);
        out3[kind] = m;
    }
    free(x4);
    topo_free(&t);
}

/* Segment-triangle intersection test (Moller-Trumbore style with the
 * segment parameter restricted to [0, 1]); 1 if they intersect. */
static int seg_tri_intersect(const double *p, const double *q, const double *a, const double *b, const double *c) {
    double e1[3], e2[3], dir[3], h[3], s[3], qv[3];
    sub3(b, a, e1); sub3(c, a, e2); sub3(q, p, dir);
    h[0] = dir[1] * e2[2] - dir[2] * e2[1];
    h[1] = dir[2] * e2[0] - dir[0] * e2[2];
    h[2] = dir[0] * e2[1] - dir[1] * e2[0];
    double det = dot3(e1, h);
    if (fabs(det) < 1e-300) return 0;
    double inv = 1.0 / det;
    sub3(p, a, s);
    double u = inv * dot3(s, h);
    if (u < 0.0 || u > 1.0) return 0;
    qv[0] = s[1] * e1[2] - s[2] * e1[1];
    qv[1] = s[2] * e1[0] - s[0] * e1[2];
    qv[2] = s[0] * e1[1] - s[1] * e1[0];
    double v = inv * dot3(dir, qv);
    if (v < 0.0 || u + v > 1.0) return 0;
    double tt = inv * dot3(e2, qv);
    return tt >= 0.0 && tt <= 1.0;
}

/* Number of (edge, triangle) pairs that intersect, over pairs sharing no
 * vertex.  A penetrating triangle pair always has such an edge. */
long orc_count_edge_triangle_intersections(const double *x3, int n, const int *edges, int ne,
                                           const int *tris, int nt) {
    long cnt = 0;
    if (ne == 0 || nt == 0) return 0;
    /* boxes in double, sweep over x */
    double *tlo = (double *)malloc(sizeof(double) * 3 * nt), *thi = (double *)malloc(sizeof(double) * 3 * nt);
    sortkey *sk = (sortkey *)malloc(sizeof(sortkey) * nt);
    double maxext = 0.0;
    for (int f = 0; f < nt; ++f) {
        for (int a = 0; a < 3; ++a) {
            double mn = x3[3 * tris[3 * f] + a], mx = mn;
            for (int i = 1; i < 3; ++i) {
                double c = x3[3 * tris[3 * f + i] + a];
                if (c < mn) mn = c;
                if (c > mx) mx = c;
            }
            tlo[3 * f + a] = mn; thi[3 * f + a] = mx;
        }
        sk[f].lo = (float)tlo[3 * f];
        sk[f].idx = f;
        if (thi[3 * f] - tlo[3 * f] > maxext) maxext = thi[3 * f] - tlo[3 * f];
    }
    qsort(sk, nt, sizeof(sortkey), cmp_sk);
    for (int e = 0; e < ne; ++e) {
        int a0 = edges[2 * e], a1 = edges[2 * e + 1];
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(x3[3 * a0 + a], x3[3 * a1 + a]);
            hi[a] = fmax(x3[3 * a0 + a], x3[3 * a1 + a]);
        }
        double from = lo[0] - maxext - 1e-6;
        int l = 0, h = nt;
        while (l < h) { int mid = (l + h) / 2; if ((double)sk[mid].lo < from) l = mid + 1; else h = mid; }
        for (int s = l; s < nt && (double)sk[s].lo <= hi[0] + 1e-6; ++s) {
            int f = sk[s].idx;
            int ok = 1;
            for (int a = 0; a < 3; ++a) if (tlo[3 * f + a] > hi[a] || thi[3 * f + a] < lo[a]) ok = 0;
            if (!ok) continue;
            const int *T = tris + 3 * f;
            if (T[0] == a0 || T[1] == a0 || T[2] == a0 || T[0] == a1 || T[1] == a1 || T[2] == a1) continue;
            cnt += seg_tri_intersect(x3 + 3 * a0, x3 + 3 * a1, x3 + 3 * T[0], x3 + 3 * T[1], x3 + 3 * T[2]);
        }
    }
    free(tlo); free(thi); free(sk);
    (void)n;
    return cnt;
}

/* geodesic.c -- part of the CPU oracle: TEST INFRASTRUCTURE ONLY (only the
 * test suite, the smoke check and the benchmark's CPU legs call it).
 *
 * Reference distances of a shell whose rest shape is not cut from a flat
 * pattern (doubly curved), taken as geodesic distances on its rest mesh.
 * Sec. 3.2 measures a shell stencil pair's reference distance in the shell's
 * 2D rest domain; the paper names non-flat rest shapes as future work.  Here
 * the rest domain is the rest mesh itself:
 *
 *   dbar(P, Q) = min over p in P, q in Q of g(p, q),
 *
 * g the length of the shortest path between p and q on the polyhedral rest
 * surface.  For a flat convex sheet, and for a developable sheet isometric to
 * a convex pattern, this is the pattern distance.
 *
 * Facts used (polyhedral geodesics):
 *  (i)   a shortest path is straight inside every face and straight across
 *        every edge it crosses -- a straight segment once the faces it crosses
 *        are unfolded into one plane -- and bends only at vertices;
 *  (ii)  hence for a vertex v and an edge e, g(v, e) is the minimum, over the
 *        vertices u a path may bend at (u = v included), of g(v, u) plus the
 *        length of a straight unfolded segment from u to a point of e;
 *  (iii) point-triangle (p; t), p not in t: a path from p reaches t on its
 *        boundary first, so dbar = min over the three edges e of t of g(p, e);
 *  (iv)  edge-edge (A, B): at a minimizing pair of interior points with no
 *        bend between them the path is perpendicular to both edges, so the
 *        edges are parallel in the unfolding and sliding the path along them
 *        keeps its length until it meets an end point or a vertex; a bend is
 *        at a vertex too.  Hence dbar = min over vertices w of
 *        g(w, A) + g(w, B)  (w an end point of A gives g(w, A) = 0).
 *
 * Computation, per source vertex v, for distances below a (only those decide
 * the filter), by Dijkstra over the vertices: the unsettled vertex u of
 * smallest distance du is settled and expanded by enumerating every strip of
 * faces that a straight segment from u can cross within length a - du.  Each
 * face around u is laid flat with u at the origin; the face beyond an edge
 * already crossed is unfolded across that edge (to the side away from the
 * face before it).  A point X of the plane is reached straight iff the
 * segment from the origin to X crosses every edge of the strip so far; that
 * is tested edge by edge (X on the far side of the edge's line, and X inside
 * the cone the edge spans from the origin).  Every vertex so reached is
 * relaxed with du + |X|; every edge whose reachable part has positive length
 * records du plus the distance from the origin to that part, and the strip
 * continues across it (a path reaching an edge in a single point runs
 * through a vertex and is the one that bends there).  Bends are allowed at every vertex:
 * at a vertex whose angle sum is at most 2 pi they never shorten a path, so
 * allowing them changes only the work.
 *
 * Arithmetic: FP64, compiled without contraction.  parity pinned:
 * tests/test_oracle_geodesic.py (flat and rolled sheets against the pattern
 * distance, cone surfaces against closed forms, a Steiner-point graph on
 * random bumpy meshes as a bound from above).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* the topology struct passed from Python (same layout as in oracle.c) */
typedef struct {
    int kind;
    int n;
    int n_edges;
    const int32_t* edges;  /* [2][E], e0 < e1, sorted lexicographically */
    int n_tris;
    const int32_t* tris;   /* [3][T] */
    const int32_t* comp;
} geo_topo;

int64_t orc_broad(const geo_topo* tp, const double* x, const double* p, double h, uint64_t** out);
int orc_stencil(const geo_topo* tp, uint64_t key, int32_t* v4);

#define GEO_MAX_DEPTH 512

typedef struct { double x, y; } p2;
static inline double cr2(p2 a, p2 b) { return a.x * b.y - a.y * b.x; }
static inline double dt2(p2 a, p2 b) { return a.x * b.x + a.y * b.y; }
static inline p2 sb2(p2 a, p2 b) { p2 r = {a.x - b.x, a.y - b.y}; return r; }

/* ---- mesh adjacency ------------------------------------------------------ */
typedef struct {
    int n, E, T;
    const int32_t* e0; const int32_t* e1;   /* edge end points */
    const int32_t* tv;                      /* [3][T] */
    int32_t* te;                            /* [T][3]: edge of (t_k, t_k+1) */
    int32_t* ef;                            /* [E][2]: faces of an edge, -1 if none */
    int32_t* vf_ptr; int32_t* vf;           /* faces around each vertex (CSR) */
    double* len;                            /* [E] rest length */
} geo_mesh;

static int edge_id(const geo_mesh* m, int a, int b) {
    int lo = a < b ? a : b, hi = a < b ? b : a;
    int l = 0, r = m->E;
    while (l < r) {
        int mid = (l + r) >> 1;
        if (m->e0[mid] < lo || (m->e0[mid] == lo && m->e1[mid] < hi)) l = mid + 1;
        else r = mid;
    }
    return (l < m->E && m->e0[l] == lo && m->e1[l] == hi) ? l : -1;
}

static void mesh_free(geo_mesh* m) {
    free(m->te); free(m->ef); free(m->vf_ptr); free(m->vf); free(m->len);
}

/* returns 0, or -1 if an edge has more than two faces (not a manifold) */
static int mesh_build(const geo_topo* tp, const double* rest, geo_mesh* m) {
    m->n = tp->n; m->E = tp->n_edges; m->T = tp->n_tris;
    m->e0 = tp->edges; m->e1 = tp->edges + tp->n_edges; m->tv = tp->tris;
    const int n = m->n, E = m->E, T = m->T;
    m->te = (int32_t*)malloc(sizeof(int32_t) * 3 * (T > 0 ? T : 1));
    m->ef = (int32_t*)malloc(sizeof(int32_t) * 2 * (E > 0 ? E : 1));
    m->vf_ptr = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    m->vf = (int32_t*)malloc(sizeof(int32_t) * 3 * (T > 0 ? T : 1));
    m->len = (double*)malloc(sizeof(double) * (E > 0 ? E : 1));
    for (int e = 0; e < E; ++e) {
        m->ef[2 * e] = m->ef[2 * e + 1] = -1;
        double dx = rest[(size_t)0 * n + m->e1[e]] - rest[(size_t)0 * n + m->e0[e]];
        double dy = rest[(size_t)1 * n + m->e1[e]] - rest[(size_t)1 * n + m->e0[e]];
        double dz = rest[(size_t)2 * n + m->e1[e]] - rest[(size_t)2 * n + m->e0[e]];
        m->len[e] = sqrt((dx * dx + dy * dy) + dz * dz);
    }
    int bad = 0;
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) {
            int e = edge_id(m, m->tv[(size_t)k * T + t], m->tv[(size_t)((k + 1) % 3) * T + t]);
            m->te[3 * t + k] = e;
            if (m->ef[2 * e] < 0) m->ef[2 * e] = t;
            else if (m->ef[2 * e + 1] < 0) m->ef[2 * e + 1] = t;
            else bad = 1;
        }
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) m->vf_ptr[m->tv[(size_t)k * T + t] + 1]++;
    for (int v = 0; v < n; ++v) m->vf_ptr[v + 1] += m->vf_ptr[v];
    int32_t* fill = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) {
            int v = m->tv[(size_t)k * T + t];
            m->vf[m->vf_ptr[v] + fill[v]++] = t;
        }
    free(fill);
    return bad ? -1 : 0;
}

static inline double elen(const geo_mesh* m, int a, int b) { return m->len[edge_id(m, a, b)]; }

/* ---- one source ---------------------------------------------------------- */
typedef struct {
    const geo_mesh* m;
    double a;
    double* dist; char* done; int32_t* vt; int nvt;   /* vertex distances, touched list */
    double* eb; int32_t* et; int net;                 /* edge distances, touched list */
    double du, R;                                     /* expanding vertex: distance, remaining length */
    p2 PA[GEO_MAX_DEPTH], PB[GEO_MAX_DEPTH];          /* unfolded strip edges, origin at the expanding vertex */
    int err;
} geo_src;

static void relax_vertex(geo_src* s, int w, double d) {
    if (!(d < s->a)) return;
    if (isinf(s->dist[w])) s->vt[s->nvt++] = w;
    if (d < s->dist[w]) s->dist[w] = d;
}

static void record_edge(geo_src* s, int e, double d) {
    if (!(d < s->a)) return;
    if (isinf(s->eb[e])) s->et[s->net++] = e;
    if (d < s->eb[e]) s->eb[e] = d;
}

/* s in [lo, hi] with al + be * s >= 0 */
static void clip(double al, double be, double* lo, double* hi) {
    if (be > 0.0) { double t = -al / be; if (t > *lo) *lo = t; }
    else if (be < 0.0) { double t = -al / be; if (t < *hi) *hi = t; }
    else if (al < 0.0) { *lo = 1.0; *hi = 0.0; }
}

/* the part s in [lo, hi] of X0 + s D whose segments from the origin cross
 * strip edge (A, B): X on the far side of the line AB (or on it) and inside
 * the cone spanned by A and B.  An edge whose line passes through the
 * origin is crossed by no such segment. */
static void clip_by_edge(p2 A, p2 B, p2 X0, p2 D, double* lo, double* hi) {
    double c = cr2(A, B);
    if (c == 0.0) { *lo = 1.0; *hi = 0.0; return; }
    if (c < 0.0) { p2 t = A; A = B; B = t; }
    p2 AB = sb2(B, A);
    /* cross(A, X) >= 0, cross(X, B) >= 0 */
    clip(cr2(A, X0), cr2(A, D), lo, hi);
    clip(cr2(X0, B), cr2(D, B), lo, hi);
    /* far side: cross(AB, X - A) <= 0  (the origin has cross(AB, -A) = cross(A, B) > 0) */
    clip(-cr2(AB, sb2(X0, A)), -cr2(AB, D), lo, hi);
}

static int point_reached(const geo_src* s, int depth, p2 X) {
    p2 Z = {0.0, 0.0};
    for (int i = 0; i <= depth; ++i) {
        double lo = 0.0, hi = 0.0;
        clip_by_edge(s->PA[i], s->PB[i], X, Z, &lo, &hi);
        if (lo > hi) return 0;
    }
    return 1;
}

/* unfold the vertex at distances la from A and lb from B (|AB| = lab), on
 * the side of line AB away from C */
static p2 unfold(p2 A, p2 B, p2 C, double la, double lb, double lab) {
    p2 AB = sb2(B, A);
    double nab = sqrt(dt2(AB, AB));
    p2 u = {AB.x / nab, AB.y / nab};
    p2 nrm = {-u.y, u.x};
    double x = (la * la - lb * lb + lab * lab) / (2.0 * lab);
    double y2 = la * la - x * x;
    double y = y2 > 0.0 ? sqrt(y2) : 0.0;
    if (cr2(AB, sb2(C, A)) > 0.0) y = -y;
    p2 W = {A.x + x * u.x + y * nrm.x, A.y + x * u.y + y * nrm.y};
    return W;
}

/* the strip's edges 0..depth are in PA/PB; the last one, between mesh
 * vertices ia (at PA[depth]) and ib (at PB[depth]), is an edge of face f_from,
 * whose third vertex lies at C */
static void strip(geo_src* s, int depth, int f_from, int ia, int ib, p2 C) {
    const geo_mesh* m = s->m;
    p2 A = s->PA[depth], B = s->PB[depth];
    p2 D = sb2(B, A);
    double lo = 0.0, hi = 1.0;
    for (int i = 0; i <= depth && lo < hi; ++i) clip_by_edge(s->PA[i], s->PB[i], A, D, &lo, &hi);
    /* a single reached point is an end point of the edge or lies on a ray
     * through a vertex: those paths are the ones that bend at that vertex */
    if (!(lo < hi)) return;
    double dd = dt2(D, D);
    double sf = dd > 0.0 ? -dt2(A, D) / dd : lo;
    if (sf < lo) sf = lo;
    if (sf > hi) sf = hi;
    p2 F = {A.x + sf * D.x, A.y + sf * D.y};
    double dmin = sqrt(dt2(F, F));
    const int e = edge_id(m, ia, ib);
    record_edge(s, e, s->du + dmin);
    if (!(dmin < s->R)) return;
    int f = m->ef[2 * e] == f_from ? m->ef[2 * e + 1] : m->ef[2 * e];
    if (f < 0) return;
    if (depth + 1 >= GEO_MAX_DEPTH) { s->err = 1; return; }
    int w = -1;
    for (int k = 0; k < 3; ++k) {
        int c = m->tv[(size_t)k * m->T + f];
        if (c != ia && c != ib) w = c;
    }
    p2 W = unfold(A, B, C, elen(m, ia, w), elen(m, ib, w), m->len[e]);
    if (point_reached(s, depth, W)) relax_vertex(s, w, s->du + sqrt(dt2(W, W)));
    s->PA[depth + 1] = A; s->PB[depth + 1] = W;
    strip(s, depth + 1, f, ia, w, B);
    s->PA[depth + 1] = W; s->PB[depth + 1] = B;
    strip(s, depth + 1, f, w, ib, A);
}

static void expand(geo_src* s, int u) {
    const geo_mesh* m = s->m;
    for (int q = m->vf_ptr[u]; q < m->vf_ptr[u + 1]; ++q) {
        int f = m->vf[q];
        int k = 0;
        while (m->tv[(size_t)k * m->T + f] != u) ++k;
        int p = m->tv[(size_t)((k + 1) % 3) * m->T + f], r = m->tv[(size_t)((k + 2) % 3) * m->T + f];
        double lup = elen(m, u, p), lur = elen(m, u, r), lpr = elen(m, p, r);
        relax_vertex(s, p, s->du + lup);
        relax_vertex(s, r, s->du + lur);
        record_edge(s, edge_id(m, u, p), s->du);
        record_edge(s, edge_id(m, u, r), s->du);
        double x = (lup * lup + lur * lur - lpr * lpr) / (2.0 * lup);
        double y2 = lur * lur - x * x;
        p2 P = {lup, 0.0}, Rr = {x, y2 > 0.0 ? sqrt(y2) : 0.0}, O = {0.0, 0.0};
        s->PA[0] = P; s->PB[0] = Rr;
        strip(s, 0, f, p, r, O);
    }
}

static void source_run(geo_src* s, int v) {
    s->nvt = 0; s->net = 0;
    relax_vertex(s, v, 0.0);
    for (;;) {
        int u = -1;
        for (int i = 0; i < s->nvt; ++i) {
            int c = s->vt[i];
            if (!s->done[c] && (u < 0 || s->dist[c] < s->dist[u])) u = c;
        }
        if (u < 0) break;
        s->done[u] = 1;
        s->du = s->dist[u];
        s->R = s->a - s->du;
        expand(s, u);
    }
}

static void source_reset(geo_src* s) {
    for (int i = 0; i < s->nvt; ++i) { s->dist[s->vt[i]] = INFINITY; s->done[s->vt[i]] = 0; }
    for (int i = 0; i < s->net; ++i) s->eb[s->et[i]] = INFINITY;
    s->nvt = s->net = 0;
}

static geo_src* source_new(const geo_mesh* m, double a) {
    geo_src* s = (geo_src*)calloc(1, sizeof(geo_src));
    s->m = m; s->a = a;
    s->dist = (double*)malloc(sizeof(double) * (m->n > 0 ? m->n : 1));
    s->done = (char*)calloc(m->n > 0 ? m->n : 1, 1);
    s->vt = (int32_t*)malloc(sizeof(int32_t) * (m->n > 0 ? m->n : 1));
    s->eb = (double*)malloc(sizeof(double) * (m->E > 0 ? m->E : 1));
    s->et = (int32_t*)malloc(sizeof(int32_t) * (m->E > 0 ? m->E : 1));
    for (int i = 0; i < m->n; ++i) s->dist[i] = INFINITY;
    for (int i = 0; i < m->E; ++i) s->eb[i] = INFINITY;
    return s;
}

static void source_free(geo_src* s) {
    free(s->dist); free(s->done); free(s->vt); free(s->eb); free(s->et); free(s);
}

/* ---- exported ------------------------------------------------------------ */

/* geodesic distances from vertex src, below a (INFINITY elsewhere): to every
 * vertex (dist_out[n], may be NULL) and to every edge (edge_out[E], may be
 * NULL).  Returns 0, -1 for a non-manifold mesh, -2 if a strip grew too long. */
int orc_geo_source(const geo_topo* tp, const double* rest, double a, int src, double* dist_out,
                   double* edge_out) {
    geo_mesh m;
    int rc = mesh_build(tp, rest, &m);
    if (rc == 0) {
        geo_src* s = source_new(&m, a);
        source_run(s, src);
        if (dist_out)
            for (int i = 0; i < m.n; ++i) dist_out[i] = s->dist[i];
        if (edge_out)
            for (int i = 0; i < m.E; ++i) edge_out[i] = s->eb[i];
        rc = s->err ? -2 : 0;
        source_free(s);
    }
    mesh_free(&m);
    return rc;
}

typedef struct { int32_t e, w; double g; } geo_triple;

static int triple_cmp(const void* x, const void* y) {
    const geo_triple* p = (const geo_triple*)x;
    const geo_triple* q = (const geo_triple*)y;
    if (p->e != q->e) return p->e < q->e ? -1 : 1;
    if (p->w != q->w) return p->w < q->w ? -1 : 1;
    return 0;
}

/* g(w, e) for one edge e and vertex w from the table sorted by (e, w) */
static double lookup(const geo_triple* tb, const int64_t* row, int e, int w) {
    int64_t l = row[e], r = row[e + 1];
    while (l < r) {
        int64_t mid = (l + r) >> 1;
        if (tb[mid].w < w) l = mid + 1;
        else r = mid;
    }
    return (l < row[e + 1] && tb[l].w == w) ? tb[l].g : INFINITY;
}

/* Rest filter of a shell with geodesic reference distances: the stencil
 * pairs of one component with dbar < a and their dbar, keys sorted.  The
 * candidates are the rest broad phase at activation a (a geodesic distance is
 * at least the 3D distance, so no pair with dbar < a is missed).  Returns the
 * count, or -1 (non-manifold mesh) / -2 (a strip grew too long). */
int64_t orc_geo_rest_filter(const geo_topo* tp, const double* rest, double a, uint64_t** out_keys,
                            double** out_dbar) {
    geo_mesh m;
    *out_keys = NULL;
    *out_dbar = NULL;
    if (mesh_build(tp, rest, &m) != 0) { mesh_free(&m); return -1; }
    const int n = m.n, E = m.E;
    /* g(w, e) < a for every vertex w and edge e */
    int64_t cap = 1024, cnt = 0;
    geo_triple* tb = (geo_triple*)malloc(sizeof(geo_triple) * cap);
    int err = 0;
    #pragma omp parallel
    {
        geo_src* s = source_new(&m, a);
        #pragma omp for schedule(dynamic, 16)
        for (int v = 0; v < n; ++v) {
            source_run(s, v);
            #pragma omp critical(geo_out)
            {
                for (int i = 0; i < s->net; ++i) {
                    if (cnt == cap) { cap *= 2; tb = (geo_triple*)realloc(tb, sizeof(geo_triple) * cap); }
                    geo_triple t = {s->et[i], v, s->eb[s->et[i]]};
                    tb[cnt++] = t;
                }
                if (s->err) err = 1;
            }
            s->err = 0;
            source_reset(s);
        }
        source_free(s);
    }
    if (err) { free(tb); mesh_free(&m); return -2; }
    qsort(tb, (size_t)cnt, sizeof(geo_triple), triple_cmp);
    int64_t* row = (int64_t*)calloc((size_t)E + 1, sizeof(int64_t));
    for (int64_t i = 0; i < cnt; ++i) row[tb[i].e + 1]++;
    for (int e = 0; e < E; ++e) row[e + 1] += row[e];
    /* candidates and their reference distances */
    uint64_t* cand;
    int64_t nc = orc_broad(tp, rest, NULL, 0.5 * a, &cand);
    double* db = (double*)malloc(sizeof(double) * (nc > 0 ? nc : 1));
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t c = 0; c < nc; ++c) {
        int32_t v[4];
        int ee = orc_stencil(tp, cand[c], v);
        double d = INFINITY;
        if (tp->comp[v[0]] == tp->comp[v[2]]) {
            if (!ee) {
                int ta[3] = {v[1], v[2], v[3]};
                for (int k = 0; k < 3; ++k) {
                    double g = lookup(tb, row, edge_id(&m, ta[k], ta[(k + 1) % 3]), v[0]);
                    if (g < d) d = g;
                }
            } else {
                int ea = (int)((cand[c] >> 31) & 0x7FFFFFFFu), eb = (int)(cand[c] & 0x7FFFFFFFu);
                int64_t i = row[ea], j = row[eb];
                while (i < row[ea + 1] && j < row[eb + 1]) {
                    if (tb[i].w < tb[j].w) ++i;
                    else if (tb[j].w < tb[i].w) ++j;
                    else {
                        double g = tb[i].g + tb[j].g;
                        if (g < d) d = g;
                        ++i; ++j;
                    }
                }
            }
        }
        db[c] = d;
    }
    int64_t nf = 0;
    for (int64_t c = 0; c < nc; ++c) if (db[c] < a) ++nf;
    uint64_t* ok = (uint64_t*)malloc(sizeof(uint64_t) * (nf > 0 ? nf : 1));
    double* od = (double*)malloc(sizeof(double) * (nf > 0 ? nf : 1));
    int64_t w = 0;
    for (int64_t c = 0; c < nc; ++c)
        if (db[c] < a) { ok[w] = cand[c]; od[w] = db[c]; ++w; }
    free(db); free(cand); free(row); free(tb);
    mesh_free(&m);
    *out_keys = ok;
    *out_dbar = od;
    return nf;
}

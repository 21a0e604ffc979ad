/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, brute-force FP64 CPU reference of the barrier-filtered contact
 * pass (Li-style IPC barrier with thickness offsets, filtered as in Sec. 3.2-3.4
 * of "Unlocking Thickness Modeling for Codimensional Contact Simulation").
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may load
 * this library; the product path never does.  It shares no code with the CUDA
 * library.
 *
 * Everything is O(n^2) over all primitive pairs.  Derivatives of the distance
 * come from hyper-dual numbers (exact first and second derivatives up to
 * rounding), not from hand-derived formulas.  PSD projection is cyclic Jacobi on
 * the full 12x12 matrix run to convergence.  Build with -ffp-contract=off: no
 * fused multiply-adds, so every rounding is the written one.
 *
 * Pair keys: bits 63..62 type (0 rod edge-edge, 1 shell point-triangle,
 * 2 shell edge-edge), bits 61..31 first index, bits 30..0 second index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ROD_EE 0
#define ORC_PT 1
#define ORC_EE 2

static inline uint64_t mk_key(int type, int64_t i, int64_t j) {
    return ((uint64_t)type << 62) | ((uint64_t)i << 31) | (uint64_t)j;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the oracle's parallel loops use from now on (timing only; the
 * results do not depend on it: every loop writes per-pair outputs). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

void orc_free(void* p) { free(p); }

/* ------------------------------------------------------------------------- */
/* Hyper-dual numbers: v + e1*E1 + e2*E2 + e12*E1E2 with E1^2 = E2^2 = 0.      */
/* The value part of every operation is exactly the plain double operation.    */
/* ------------------------------------------------------------------------- */
typedef struct { double v, e1, e2, e12; } hd;

static inline hd hc(double v) { hd r = {v, 0.0, 0.0, 0.0}; return r; }
static inline hd hadd(hd a, hd b) { hd r = {a.v + b.v, a.e1 + b.e1, a.e2 + b.e2, a.e12 + b.e12}; return r; }
static inline hd hsub(hd a, hd b) { hd r = {a.v - b.v, a.e1 - b.e1, a.e2 - b.e2, a.e12 - b.e12}; return r; }
static inline hd hmul(hd a, hd b) {
    hd r;
    r.v = a.v * b.v;
    r.e1 = a.v * b.e1 + a.e1 * b.v;
    r.e2 = a.v * b.e2 + a.e2 * b.v;
    r.e12 = a.v * b.e12 + a.e1 * b.e2 + a.e2 * b.e1 + a.e12 * b.v;
    return r;
}
static inline hd hdiv(hd a, hd b) {
    /* q = a/b ; from a = q*b differentiate once and twice */
    hd q;
    q.v = a.v / b.v;
    q.e1 = (a.e1 - q.v * b.e1) / b.v;
    q.e2 = (a.e2 - q.v * b.e2) / b.v;
    q.e12 = (a.e12 - q.e1 * b.e2 - q.e2 * b.e1 - q.v * b.e12) / b.v;
    return q;
}
static inline hd hsqrt(hd a) {
    /* s = sqrt(a) ; from a = s*s */
    hd s;
    s.v = sqrt(a.v);
    s.e1 = a.e1 / (2.0 * s.v);
    s.e2 = a.e2 / (2.0 * s.v);
    s.e12 = (a.e12 - 2.0 * s.e1 * s.e2) / (2.0 * s.v);
    return s;
}

typedef struct { hd c[3]; } hv3;
static inline hv3 vsub(hv3 a, hv3 b) { hv3 r; for (int k = 0; k < 3; ++k) r.c[k] = hsub(a.c[k], b.c[k]); return r; }
static inline hd vdot(hv3 a, hv3 b) {
    return hadd(hadd(hmul(a.c[0], b.c[0]), hmul(a.c[1], b.c[1])), hmul(a.c[2], b.c[2]));
}
static inline hv3 vcross(hv3 a, hv3 b) {
    hv3 r;
    r.c[0] = hsub(hmul(a.c[1], b.c[2]), hmul(a.c[2], b.c[1]));
    r.c[1] = hsub(hmul(a.c[2], b.c[0]), hmul(a.c[0], b.c[2]));
    r.c[2] = hsub(hmul(a.c[0], b.c[1]), hmul(a.c[1], b.c[0]));
    return r;
}

/* plain-double views of the same operations (used by the type classification) */
static inline void dsub3(const double* a, const double* b, double* r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static inline double ddot3(const double* a, const double* b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }
static inline void dcross3(const double* a, const double* b, double* r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------- */
/* Distance types.                                                            */
/*  point-triangle (p; t0,t1,t2):                                             */
/*    0 PP(p,t0) 1 PP(p,t1) 2 PP(p,t2) 3 PE(p,t0t1) 4 PE(p,t1t2) 5 PE(p,t2t0)  */
/*    6 face                                                                  */
/*  edge-edge (a0,a1; b0,b1):                                                 */
/*    0 PP(a0,b0) 1 PP(a0,b1) 2 PP(a1,b0) 3 PP(a1,b1)                         */
/*    4 PE(a0,b) 5 PE(a1,b) 6 PE(b0,a) 7 PE(b1,a) 8 line-line interior        */
/* All computations use coordinates relative to the pair's first vertex       */
/* (p for point-triangle, a0 for edge-edge).                                  */
/* ------------------------------------------------------------------------- */

/* squared point-point distance |b - a|^2 */
static hd d2_pp(hv3 a, hv3 b) { hv3 d = vsub(b, a); return vdot(d, d); }
/* squared point-line distance |(q-e0) x (e1-e0)|^2 / |e1-e0|^2 */
static hd d2_pe(hv3 q, hv3 e0, hv3 e1) {
    hv3 u = vsub(e1, e0), w = vsub(q, e0);
    hv3 c = vcross(w, u);
    return hdiv(vdot(c, c), vdot(u, u));
}
/* squared point-plane distance ((q-t0).n)^2 / |n|^2, n = (t1-t0) x (t2-t0) */
static hd d2_pf(hv3 q, hv3 t0, hv3 t1, hv3 t2) {
    hv3 u = vsub(t1, t0), v = vsub(t2, t0);
    hv3 n = vcross(u, v);
    hv3 w = vsub(q, t0);
    hd g = vdot(w, n);
    return hdiv(hmul(g, g), vdot(n, n));
}
/* squared line-line distance ((b0-a0).n)^2/|n|^2, n = (a1-a0) x (b1-b0) */
static hd d2_ll(hv3 a0, hv3 a1, hv3 b0, hv3 b1) {
    hv3 u = vsub(a1, a0), v = vsub(b1, b0);
    hv3 n = vcross(u, v);
    hv3 w = vsub(b0, a0);
    hd g = vdot(w, n);
    return hdiv(hmul(g, g), vdot(n, n));
}

/* squared distance of a PT stencil for a fixed type; X are the 4 global points */
static hd pt_d2_typed(const hv3 X[4], int type) {
    hv3 Q, T[3];
    /* local frame: subtract the point */
    for (int k = 0; k < 3; ++k) Q.c[k] = hsub(X[0].c[k], X[0].c[k]);
    for (int i = 0; i < 3; ++i) T[i] = vsub(X[i + 1], X[0]);
    switch (type) {
    case 0: return d2_pp(Q, T[0]);
    case 1: return d2_pp(Q, T[1]);
    case 2: return d2_pp(Q, T[2]);
    case 3: return d2_pe(Q, T[0], T[1]);
    case 4: return d2_pe(Q, T[1], T[2]);
    case 5: return d2_pe(Q, T[2], T[0]);
    default: return d2_pf(Q, T[0], T[1], T[2]);
    }
}

static hd ee_d2_typed(const hv3 X[4], int type) {
    hv3 A0, A1, B0, B1;
    for (int k = 0; k < 3; ++k) A0.c[k] = hsub(X[0].c[k], X[0].c[k]);
    A1 = vsub(X[1], X[0]);
    B0 = vsub(X[2], X[0]);
    B1 = vsub(X[3], X[0]);
    switch (type) {
    case 0: return d2_pp(A0, B0);
    case 1: return d2_pp(A0, B1);
    case 2: return d2_pp(A1, B0);
    case 3: return d2_pp(A1, B1);
    case 4: return d2_pe(A0, B0, B1);
    case 5: return d2_pe(A1, B0, B1);
    case 6: return d2_pe(B0, A0, A1);
    case 7: return d2_pe(B1, A0, A1);
    default: return d2_ll(A0, A1, B0, B1);
    }
}

static hd d2_typed(int is_ee, const hv3 X[4], int type) {
    return is_ee ? ee_d2_typed(X, type) : pt_d2_typed(X, type);
}

static void to_hv(const double* x12, hv3 X[4]) {
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) X[i].c[k] = hc(x12[3 * i + k]);
}

static double d2_typed_value(int is_ee, const double* x12, int type) {
    hv3 X[4];
    to_hv(x12, X);
    return d2_typed(is_ee, X, type).v;
}

/* point-segment sub-classification: 0 -> nearest is e0, 1 -> e1, 2 -> interior */
static int seg_region(const double* q, const double* e0, const double* e1) {
    double u[3], w[3];
    dsub3(e1, e0, u);
    dsub3(q, e0, w);
    double lam = ddot3(w, u);
    if (lam <= 0.0) return 0;
    if (lam >= ddot3(u, u)) return 1;
    return 2;
}

typedef struct { int type; double d2; } cand_t;

static void take_min(cand_t* best, int type, double d2) {
    if (d2 < best->d2 || (d2 == best->d2 && type < best->type)) { best->type = type; best->d2 = d2; }
}

/* Point-triangle type: face if the projection of p falls strictly inside the
 * (non-degenerate) triangle, else the nearest of the three point-segment
 * distances (each PP or PE).  Ties go to the lowest type id. */
int orc_pt_type(const double* x12, double* d2_out) {
    const double* p = x12;
    double T[3][3], n[3], e1[3], e2[3];
    for (int i = 0; i < 3; ++i) dsub3(x12 + 3 * (i + 1), p, T[i]);
    dsub3(T[1], T[0], e1);
    dsub3(T[2], T[0], e2);
    dcross3(e1, e2, n);
    double nn = ddot3(n, n);
    if (nn > 0.0) {
        /* sign of each barycentric coordinate of the projection of q = 0:
         * ((t_{i+1}-q) x (t_{i+2}-q)) . n  */
        double c[3], s0, s1, s2;
        dcross3(T[1], T[2], c); s0 = ddot3(c, n);
        dcross3(T[2], T[0], c); s1 = ddot3(c, n);
        dcross3(T[0], T[1], c); s2 = ddot3(c, n);
        if (s0 > 0.0 && s1 > 0.0 && s2 > 0.0) {
            if (d2_out) *d2_out = d2_typed_value(0, x12, 6);
            return 6;
        }
    }
    double Q[3] = {0.0, 0.0, 0.0};
    cand_t best = {99, INFINITY};
    static const int ea[3] = {0, 1, 2}, eb[3] = {1, 2, 0}, pe_type[3] = {3, 4, 5};
    for (int e = 0; e < 3; ++e) {
        int r = seg_region(Q, T[ea[e]], T[eb[e]]);
        int type = (r == 0) ? ea[e] : (r == 1) ? eb[e] : pe_type[e];
        take_min(&best, type, d2_typed_value(0, x12, type));
    }
    if (d2_out) *d2_out = best.d2;
    return best.type;
}

/* Edge-edge type: line-line interior if the unconstrained closest-point
 * parameters lie strictly inside (0,1)^2 and the edges are not parallel
 * (|u x v|^2 > 1e-20 |u|^2 |v|^2); otherwise the nearest of the four
 * point-segment distances.  Ties go to the lowest type id. */
int orc_ee_type(const double* x12, double* d2_out) {
    double A0[3] = {0.0, 0.0, 0.0}, A1[3], B0[3], B1[3];
    dsub3(x12 + 3, x12, A1);
    dsub3(x12 + 6, x12, B0);
    dsub3(x12 + 9, x12, B1);
    double u[3], v[3], w[3], cr[3];
    dsub3(A1, A0, u);
    dsub3(B1, B0, v);
    dsub3(A0, B0, w);
    dcross3(u, v, cr);
    double cc = ddot3(cr, cr), uu = ddot3(u, u), vv = ddot3(v, v);
    if (cc > (1e-20 * uu) * vv) {
        double B = ddot3(u, v), D = ddot3(u, w), E = ddot3(v, w);
        double sN = B * E - vv * D;
        double tN = uu * E - B * D;
        if (sN > 0.0 && sN < cc && tN > 0.0 && tN < cc) {
            if (d2_out) *d2_out = d2_typed_value(1, x12, 8);
            return 8;
        }
    }
    cand_t best = {99, INFINITY};
    int r, type;
    r = seg_region(A0, B0, B1); type = (r == 0) ? 0 : (r == 1) ? 1 : 4; take_min(&best, type, d2_typed_value(1, x12, type));
    r = seg_region(A1, B0, B1); type = (r == 0) ? 2 : (r == 1) ? 3 : 5; take_min(&best, type, d2_typed_value(1, x12, type));
    r = seg_region(B0, A0, A1); type = (r == 0) ? 0 : (r == 1) ? 2 : 6; take_min(&best, type, d2_typed_value(1, x12, type));
    r = seg_region(B1, A0, A1); type = (r == 0) ? 1 : (r == 1) ? 3 : 7; take_min(&best, type, d2_typed_value(1, x12, type));
    if (d2_out) *d2_out = best.d2;
    return best.type;
}

/* distance d = sqrt(d^2) of a stencil; returns the type */
int orc_distance(int is_ee, const double* x12, double* d_out) {
    double d2;
    int t = is_ee ? orc_ee_type(x12, &d2) : orc_pt_type(x12, &d2);
    *d_out = sqrt(d2);
    return t;
}

/* gradient (12) and Hessian (144, row-major) of d for a fixed type, by
 * hyper-dual evaluation of d = sqrt(d^2) for every coordinate pair (i <= j) */
void orc_distance_derivs(int is_ee, const double* x12, int type, double* grad, double* hess) {
    for (int i = 0; i < 12; ++i) {
        for (int j = i; j < 12; ++j) {
            hv3 X[4];
            to_hv(x12, X);
            X[i / 3].c[i % 3].e1 = 1.0;
            X[j / 3].c[j % 3].e2 = 1.0;
            hd d = hsqrt(d2_typed(is_ee, X, type));
            hess[12 * i + j] = d.e12;
            hess[12 * j + i] = d.e12;
            if (i == j) grad[i] = d.e1;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* IPC log barrier (Eq. 2) with the offset of Eq. 3: y = d - xi, width dhat.   */
/*   b   = -(y - dh)^2 ln(y/dh)                                              */
/*   b'  = -2 (y - dh) ln(y/dh) - (y - dh)^2 / y                              */
/*   b'' = -2 ln(y/dh) - 4 (y - dh)/y + (y - dh)^2 / y^2                      */
/* valid for 0 < y < dh; zero for y >= dh.                                    */
/* ------------------------------------------------------------------------- */
void orc_barrier(double y, double dh, double* b, double* b1, double* b2) {
    if (y >= dh) { *b = 0.0; *b1 = 0.0; *b2 = 0.0; return; }
    double r = y - dh, l = log(y / dh);
    *b = -(r * r) * l;
    *b1 = -2.0 * r * l - (r * r) / y;
    *b2 = -2.0 * l - 4.0 * r / y + (r * r) / (y * y);
}

/* ------------------------------------------------------------------------- */
/* Cyclic Jacobi on a symmetric n x n matrix (Golub & Van Loan, Sec. 8.5),    */
/* run until the off-diagonal norm is below 1e-15 of the Frobenius norm or 50 */
/* sweeps.  Then clamp negative eigenvalues to zero and rebuild Q L+ Q^T.     */
/* ------------------------------------------------------------------------- */
int orc_psd_project(int n, const double* A_in, double* A_out, double* evals) {
    double A[144], V[144];
    memcpy(A, A_in, sizeof(double) * n * n);
    for (int i = 0; i < n * n; ++i) V[i] = 0.0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    int sweep;
    for (sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0, fro = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                fro += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (fro == 0.0 || sqrt(off) <= 1e-15 * sqrt(fro)) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) { /* columns p, q */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* rows p, q */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) if (evals) evals[i] = A[i * n + i];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) {
                double lk = A[k * n + k];
                if (lk > 0.0) s += V[i * n + k] * lk * V[j * n + k];
            }
            A_out[i * n + j] = s;
        }
    return sweep;
}

/* ------------------------------------------------------------------------- */
/* Topology passed from Python.                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int kind;              /* 0 rods, 1 shells */
    int n;                 /* vertices */
    int n_edges;           /* E */
    const int32_t* edges;  /* [2][E] SoA */
    int n_tris;            /* T (shells) */
    const int32_t* tris;   /* [3][T] SoA */
    const int32_t* comp;   /* component id per vertex */
} orc_topo;

/* the 4 vertex ids of a pair key */
static void stencil(const orc_topo* tp, uint64_t key, int v[4], int* is_ee) {
    int type = (int)(key >> 62);
    int64_t i = (int64_t)((key >> 31) & 0x7FFFFFFFu), j = (int64_t)(key & 0x7FFFFFFFu);
    if (type == ORC_PT) {
        v[0] = (int)i;
        v[1] = tp->tris[j];
        v[2] = tp->tris[tp->n_tris + j];
        v[3] = tp->tris[2 * tp->n_tris + j];
        *is_ee = 0;
    } else {
        v[0] = tp->edges[i];
        v[1] = tp->edges[tp->n_edges + i];
        v[2] = tp->edges[j];
        v[3] = tp->edges[tp->n_edges + j];
        *is_ee = 1;
    }
}

int orc_stencil(const orc_topo* tp, uint64_t key, int32_t* v4) {
    int v[4], e;
    stencil(tp, key, v, &e);
    for (int k = 0; k < 4; ++k) v4[k] = v[k];
    return e;
}

static void gather12(const double* x, int n, const int v[4], double* x12) {
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) x12[3 * i + k] = x[(size_t)k * n + v[i]];
}

/* ------------------------------------------------------------------------- */
/* Brute-force broad phase over ALL non-incident primitive pairs.             */
/* Box of a primitive: per axis [fl(min - h), fl(max + h)] over its vertices, */
/* where the coordinates are x (static) or both x and x + p (swept).          */
/* Two boxes overlap iff lo_P <= hi_Q and lo_Q <= hi_P on all three axes.     */
/* Output is sorted: pairs are emitted row by row in index order.             */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t* k; int64_t n, cap; } kvec;
static void kpush(kvec* v, uint64_t k) {
    if (v->n == v->cap) { v->cap = v->cap ? 2 * v->cap : 16; v->k = (uint64_t*)realloc(v->k, v->cap * sizeof(uint64_t)); }
    v->k[v->n++] = k;
}

static void prim_box(const double* x, const double* p, int n, const int* vs, int nv, double h, double lo[3], double hi[3]) {
    for (int k = 0; k < 3; ++k) {
        double mn = INFINITY, mx = -INFINITY;
        for (int a = 0; a < nv; ++a) {
            double c = x[(size_t)k * n + vs[a]];
            if (c < mn) mn = c;
            if (c > mx) mx = c;
            if (p) {
                double c2 = c + p[(size_t)k * n + vs[a]];
                if (c2 < mn) mn = c2;
                if (c2 > mx) mx = c2;
            }
        }
        lo[k] = mn - h;
        hi[k] = mx + h;
    }
}

static inline int box_overlap(const double* l1, const double* h1, const double* l2, const double* h2) {
    for (int k = 0; k < 3; ++k)
        if (!(l1[k] <= h2[k] && l2[k] <= h1[k])) return 0;
    return 1;
}

/* p may be NULL (static boxes).  Returns count; *out is malloc'd. */
int64_t orc_broad(const orc_topo* tp, const double* x, const double* p, double h, uint64_t** out) {
    const int n = tp->n, E = tp->n_edges, T = tp->n_tris;
    double* elo = (double*)malloc(sizeof(double) * 3 * (E > 0 ? E : 1));
    double* ehi = (double*)malloc(sizeof(double) * 3 * (E > 0 ? E : 1));
    for (int e = 0; e < E; ++e) {
        int vs[2] = {tp->edges[e], tp->edges[E + e]};
        prim_box(x, p, n, vs, 2, h, elo + 3 * e, ehi + 3 * e);
    }
    int rows = E + (tp->kind == 1 ? n : 0);
    kvec* per = (kvec*)calloc(rows > 0 ? rows : 1, sizeof(kvec));
    if (tp->kind == 1) {
        double* tlo = (double*)malloc(sizeof(double) * 3 * (T > 0 ? T : 1));
        double* thi = (double*)malloc(sizeof(double) * 3 * (T > 0 ? T : 1));
        double* vlo = (double*)malloc(sizeof(double) * 3 * n);
        double* vhi = (double*)malloc(sizeof(double) * 3 * n);
        for (int t = 0; t < T; ++t) {
            int vs[3] = {tp->tris[t], tp->tris[T + t], tp->tris[2 * T + t]};
            prim_box(x, p, n, vs, 3, h, tlo + 3 * t, thi + 3 * t);
        }
        for (int v = 0; v < n; ++v) { int vs[1] = {v}; prim_box(x, p, n, vs, 1, h, vlo + 3 * v, vhi + 3 * v); }
        #pragma omp parallel for schedule(dynamic, 64)
        for (int v = 0; v < n; ++v) {
            for (int t = 0; t < T; ++t) {
                if (tp->tris[t] == v || tp->tris[T + t] == v || tp->tris[2 * T + t] == v) continue;
                if (box_overlap(vlo + 3 * v, vhi + 3 * v, tlo + 3 * t, thi + 3 * t)) kpush(&per[v], mk_key(ORC_PT, v, t));
            }
        }
        free(tlo); free(thi); free(vlo); free(vhi);
    }
    const int base = (tp->kind == 1) ? n : 0;
    const int etype = (tp->kind == 1) ? ORC_EE : ORC_ROD_EE;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int e = 0; e < E; ++e) {
        int a0 = tp->edges[e], a1 = tp->edges[E + e];
        for (int f = e + 1; f < E; ++f) {
            int b0 = tp->edges[f], b1 = tp->edges[E + f];
            if (a0 == b0 || a0 == b1 || a1 == b0 || a1 == b1) continue;
            if (box_overlap(elo + 3 * e, ehi + 3 * e, elo + 3 * f, ehi + 3 * f)) kpush(&per[base + e], mk_key(etype, e, f));
        }
    }
    int64_t total = 0;
    for (int r = 0; r < rows; ++r) total += per[r].n;
    uint64_t* o = (uint64_t*)malloc(sizeof(uint64_t) * (total > 0 ? total : 1));
    int64_t w = 0;
    for (int r = 0; r < rows; ++r) {
        if (per[r].n) memcpy(o + w, per[r].k, per[r].n * sizeof(uint64_t));
        w += per[r].n;
        free(per[r].k);
    }
    free(per); free(elo); free(ehi);
    *out = o;
    return total;
}

/* ------------------------------------------------------------------------- */
/* Rest filter, Sec. 3.2: among same-component stencil pairs of K, those whose */
/* reference distance dbar is below the activation a.                          */
/* Rods: dbar(k,l) = S[l] - S[k+1] for edges k < l of one polyline, S the     */
/*   arc length at each vertex summed sequentially from the polyline start.  */
/* Shells: dbar = Euclidean PT/EE distance at the rest positions; pairs whose */
/*   rest boxes inflated by a/2 do not overlap have dbar >= a and are skipped. */
/* Outputs sorted keys and their dbar.                                         */
/* ------------------------------------------------------------------------- */
void orc_arclength(int n, const double* rest, int n_rods, const int32_t* rod_ptr, double* S) {
    for (int r = 0; r < n_rods; ++r) {
        int s = rod_ptr[r], e = rod_ptr[r + 1];
        if (e <= s) continue;
        S[s] = 0.0;
        for (int v = s + 1; v < e; ++v) {
            double dx = rest[v] - rest[v - 1];
            double dy = rest[(size_t)n + v] - rest[(size_t)n + v - 1];
            double dz = rest[2 * (size_t)n + v] - rest[2 * (size_t)n + v - 1];
            S[v] = S[v - 1] + sqrt((dx * dx + dy * dy) + dz * dz);
        }
    }
}

int64_t orc_rest_filter(const orc_topo* tp, const double* rest, double a, const double* S,
                        uint64_t** out_keys, double** out_dbar) {
    kvec* per = NULL;
    int rows = 0;
    if (tp->kind == 0) {
        const int E = tp->n_edges;
        rows = E;
        per = (kvec*)calloc(rows > 0 ? rows : 1, sizeof(kvec));
        #pragma omp parallel for schedule(dynamic, 64)
        for (int k = 0; k < E; ++k) {
            int k1 = tp->edges[E + k];          /* end vertex of edge k = k+1 on its rod */
            /* the edges of one polyline are contiguous: stop at the next polyline */
            for (int l = k + 1; l < E; ++l) {
                int l0 = tp->edges[l];
                if (tp->comp[l0] != tp->comp[k1]) break;      /* other polyline */
                if (l0 <= k1) continue;                        /* incident */
                double dbar = S[l0] - S[k1];
                if (dbar < a) kpush(&per[k], mk_key(ORC_ROD_EE, k, l));
            }
        }
    } else {
        uint64_t* cand;
        int64_t nc = orc_broad(tp, rest, NULL, 0.5 * a, &cand);
        kvec keep = {0, 0, 0};
        char* ok = (char*)calloc(nc > 0 ? nc : 1, 1);
        #pragma omp parallel for schedule(dynamic, 256)
        for (int64_t c = 0; c < nc; ++c) {
            int v[4], ee;
            stencil(tp, cand[c], v, &ee);
            if (tp->comp[v[0]] != tp->comp[v[2]]) continue;
            double x12[12], d;
            gather12(rest, tp->n, v, x12);
            orc_distance(ee, x12, &d);
            if (d < a) ok[c] = 1;
        }
        for (int64_t c = 0; c < nc; ++c) if (ok[c]) kpush(&keep, cand[c]);
        free(ok); free(cand);
        rows = 1;
        per = (kvec*)calloc(1, sizeof(kvec));
        per[0] = keep;
    }
    int64_t total = 0;
    for (int r = 0; r < rows; ++r) total += per[r].n;
    uint64_t* o = (uint64_t*)malloc(sizeof(uint64_t) * (total > 0 ? total : 1));
    double* db = (double*)malloc(sizeof(double) * (total > 0 ? total : 1));
    int64_t w = 0;
    for (int r = 0; r < rows; ++r) {
        if (per[r].n) memcpy(o + w, per[r].k, per[r].n * sizeof(uint64_t));
        w += per[r].n;
        free(per[r].k);
    }
    free(per);
    #pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < total; ++c) {
        int v[4], ee;
        stencil(tp, o[c], v, &ee);
        if (tp->kind == 0) {
            db[c] = S[v[2]] - S[v[1]];
        } else {
            double x12[12];
            gather12(rest, tp->n, v, x12);
            orc_distance(ee, x12, &db[c]);
        }
    }
    *out_keys = o;
    *out_dbar = db;
    return total;
}

/* ------------------------------------------------------------------------- */
/* Narrow phase for candidate pairs (Sec. 3.3, Eq. 2-4; Sec. 3.4 for class C). */
/* klass_in: 0 = U (unfiltered), 1 = F (filtered).                             */
/* Per-pair parameters (offset xi_p, width dhat_p):                            */
/*   double-filtered (Eq. 4): U -> (xi, dhat); F -> (0, dbar_min);             */
/*   C (U with d <= xi, core_temp on) -> (0, xi + dhat)                        */
/*   single-filtered (Eq. 1, single=1): U -> (0, xi + dhat); F -> (0, dbar_min) */
/* y = d - xi_p; active iff y < dhat_p; y <= 0 is a penetration.               */
/* Outputs per candidate: d, type, final class (0 U, 1 F, 2 C), active flag.  */
/* For active pairs (in candidate order): energy kappa*b, gradient (12) and   */
/* PSD-projected Hessian (144) of kappa*b(d - xi_p, dhat_p).                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    double xi, dhat, kappa, dbar_min;
    int single;      /* 1: Eq. 1 (single-phase) */
    int core_temp;   /* 1: class C on */
    int project;     /* 1: PSD-project the Hessian (0 only for derivative checks) */
    const double* dbar_comp;  /* per-component dbar_min by component label, or NULL (one scalar) */
    const double* moll_eps;   /* per active pair (orc_barrier_pairs order): the edge-edge mollifier's
                                 threshold eps_x, <= 0 for none; NULL: no mollifier */
} orc_params;

/* comp: the component label of the pair's first vertex */
static void pair_params(const orc_params* P, int klass, int comp, double* xi_p, double* dh_p) {
    double a = P->xi + P->dhat;
    if (klass == 1) { *xi_p = 0.0; *dh_p = P->dbar_comp ? P->dbar_comp[comp] : P->dbar_min; return; }
    if (klass == 2) { *xi_p = 0.0; *dh_p = a; return; }
    if (P->single) { *xi_p = 0.0; *dh_p = a; return; }
    *xi_p = P->xi; *dh_p = P->dhat;
}

int64_t orc_narrow(const orc_topo* tp, const double* x, const orc_params* P, int64_t nc,
                   const uint64_t* keys, const uint8_t* klass_in,
                   double* d_out, int8_t* type_out, uint8_t* klass_out, uint8_t* active_out,
                   int* penetration) {
    int pen = 0;
    int64_t nact = 0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(+ : nact) reduction(| : pen)
    for (int64_t c = 0; c < nc; ++c) {
        int v[4], ee;
        stencil(tp, keys[c], v, &ee);
        double x12[12], d;
        gather12(x, tp->n, v, x12);
        int type = orc_distance(ee, x12, &d);
        int k = klass_in[c];
        if (k == 0 && P->core_temp && !P->single && d <= P->xi) k = 2;
        double xi_p, dh_p;
        pair_params(P, k, tp->comp[v[0]], &xi_p, &dh_p);
        double y = d - xi_p;
        /* class 3: culled (Kaldor et al.'s index-radius culling, the paper's
         * comparison): no barrier */
        int act = (k != 3) && (y < dh_p);
        if (act && y <= 0.0) pen = 1;
        d_out[c] = d;
        type_out[c] = (int8_t)type;
        klass_out[c] = (uint8_t)k;
        active_out[c] = (uint8_t)act;
        nact += act;
    }
    *penetration = pen;
    return nact;
}

/* ------------------------------------------------------------------------- */
/* IPC's edge-edge mollifier (Li et al. 2020), which the paper's solver takes   */
/* with the IPC contact energy (App. A): with c = |e0 x e1|^2 (e0 = a1 - a0,    */
/* e1 = b1 - b0) and the threshold eps_x = 1e-3 |rest e0|^2 |rest e1|^2,        */
/*   m(c) = -c^2 / eps_x^2 + 2 c / eps_x  for c < eps_x,  1 otherwise,          */
/* and the pair's energy is m kappa b.  m vanishes for parallel edges, where    */
/* the edge-edge distance type is ambiguous, and is C^1 at eps_x.               */
/* ------------------------------------------------------------------------- */
void orc_mollifier(double c, double eps, double* m, double* m1, double* m2) {
    if (!(c < eps)) { *m = 1.0; *m1 = 0.0; *m2 = 0.0; return; }
    *m = -(c * c) / (eps * eps) + 2.0 * c / eps;
    *m1 = -2.0 * c / (eps * eps) + 2.0 / eps;
    *m2 = -2.0 / (eps * eps);
}

/* c = |(a1 - a0) x (b1 - b0)|^2 of an edge-edge stencil with its gradient (12)
 * and Hessian (144, row-major), by hyper-dual evaluation per coordinate pair */
void orc_ee_cross2_derivs(const double* x12, double* c, double* grad, double* hess) {
    for (int i = 0; i < 12; ++i) {
        for (int j = i; j < 12; ++j) {
            hv3 X[4];
            to_hv(x12, X);
            X[i / 3].c[i % 3].e1 = 1.0;
            X[j / 3].c[j % 3].e2 = 1.0;
            hv3 n = vcross(vsub(X[1], X[0]), vsub(X[3], X[2]));
            hd v = vdot(n, n);
            hess[12 * i + j] = v.e12;
            hess[12 * j + i] = v.e12;
            if (i == j) grad[i] = v.e1;
            if (i == 0 && j == 0) *c = v.v;
        }
    }
}

/* Energy and derivatives of the active pairs listed in idx[] (indices into the
 * candidate arrays).  grad: [na][12]; hess: [na][144].  Edge-edge pairs with
 * a mollifier threshold (P->moll_eps[a] > 0) take m kappa b and its
 * derivatives by the product rule. */
void orc_barrier_pairs(const orc_topo* tp, const double* x, const orc_params* P, int64_t na,
                       const uint64_t* keys, const uint8_t* klass, const double* d,
                       const int8_t* type, double* energy, double* grad, double* hess, double* hmax) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < na; ++a) {
        int v[4], ee;
        stencil(tp, keys[a], v, &ee);
        double x12[12], gd[12], Hd[144], H[144];
        gather12(x, tp->n, v, x12);
        double xi_p, dh_p, b, b1, b2;
        pair_params(P, klass[a], tp->comp[v[0]], &xi_p, &dh_p);
        double y = d[a] - xi_p;
        if (y <= 0.0) {
            energy[a] = INFINITY;
            for (int i = 0; i < 12; ++i) grad[12 * a + i] = NAN;
            for (int i = 0; i < 144; ++i) hess[144 * a + i] = NAN;
            if (hmax) hmax[a] = NAN;
            continue;
        }
        orc_barrier(y, dh_p, &b, &b1, &b2);
        orc_distance_derivs(ee, x12, type[a], gd, Hd);
        energy[a] = P->kappa * b;
        for (int i = 0; i < 12; ++i) grad[12 * a + i] = P->kappa * b1 * gd[i];
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j)
                H[12 * i + j] = P->kappa * (b2 * gd[i] * gd[j] + b1 * Hd[12 * i + j]);
        const double eps = (ee && P->moll_eps) ? P->moll_eps[a] : 0.0;
        if (eps > 0.0) {
            double c, gc[12], Hc[144], m, m1, m2;
            orc_ee_cross2_derivs(x12, &c, gc, Hc);
            orc_mollifier(c, eps, &m, &m1, &m2);
            if (c < eps) {
                const double k = P->kappa;
                energy[a] = k * m * b;
                for (int i = 0; i < 12; ++i) grad[12 * a + i] = k * (m * b1 * gd[i] + b * m1 * gc[i]);
                for (int i = 0; i < 12; ++i)
                    for (int j = 0; j < 12; ++j)
                        H[12 * i + j] = k * (m * (b2 * gd[i] * gd[j] + b1 * Hd[12 * i + j]) +
                                             b1 * m1 * (gc[i] * gd[j] + gd[i] * gc[j]) +
                                             b * (m2 * gc[i] * gc[j] + m1 * Hc[12 * i + j]));
            }
        }
        double mx = 0.0;
        for (int i = 0; i < 144; ++i) mx = fmax(mx, fabs(H[i]));
        if (hmax) hmax[a] = mx;   /* largest entry before projection */
        if (P->project) orc_psd_project(12, H, hess + 144 * a, NULL);
        else memcpy(hess + 144 * a, H, sizeof(H));
    }
}

/* ------------------------------------------------------------------------- */
/* Additive CCD (C-IPC, Li et al. 2021) for one stencil.                        */
/* x12, p12: positions and displacements of the 4 stencil vertices.            */
/* Local frame: positions relative to the first vertex; displacements minus  */
/* their mean.  l_p bounds the relative speed of the closest points:           */
/*   PT: |p0| + max(|p1|,|p2|,|p3|);  EE: max(|p0|,|p1|) + max(|p2|,|p3|).     */
/* Starting from g0 = d - offset, the first step (1-s) g0 / l_p, then steps    */
/* c (d - offset) / l_p, each cannot close the current gap; the loop stops    */
/* before the gap would fall below s*g0 and returns the last safe t, or t_c   */
/* when t passes t_c.  Returns the number of iterations (capped by max_iter). */
/* ------------------------------------------------------------------------- */
static double norm3(const double* a) { return sqrt(ddot3(a, a)); }

int orc_accd(int is_ee, const double* x12, const double* p12, double offset, double s, double c_inner,
             double t_c, int max_iter, double* t_out, int* status) {
    double X[12], Pm[12], pbar[3];
    for (int k = 0; k < 3; ++k) pbar[k] = (((p12[k] + p12[3 + k]) + p12[6 + k]) + p12[9 + k]) * 0.25;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) {
            X[3 * i + k] = x12[3 * i + k] - x12[k];
            Pm[3 * i + k] = p12[3 * i + k] - pbar[k];
        }
    double n0 = norm3(Pm), n1 = norm3(Pm + 3), n2 = norm3(Pm + 6), n3 = norm3(Pm + 9);
    double lp;
    if (is_ee) lp = fmax(n0, n1) + fmax(n2, n3);
    else lp = n0 + fmax(fmax(n1, n2), n3);
    *status = 0;
    if (lp == 0.0) { *t_out = t_c; return 0; }
    double d;
    orc_distance(is_ee, X, &d);
    double g0 = d - offset;
    if (g0 <= 0.0) { *t_out = 0.0; *status = 1; return 0; }
    double g = s * g0;
    double t = 0.0;
    double tl = (1.0 - s) * g0 / lp;
    int it;
    for (it = 0; it < max_iter; ++it) {
        for (int i = 0; i < 12; ++i) X[i] = X[i] + tl * Pm[i];
        orc_distance(is_ee, X, &d);
        if (t > 0.0 && (d - offset) < g) break;
        t = t + tl;
        if (t > t_c) { *t_out = t_c; return it + 1; }
        tl = c_inner * (d - offset) / lp;
    }
    if (it == max_iter) *status = 2;
    *t_out = t;
    return it + 1;
}

/* ACCD over a list of pairs.  klass: 0 U (offset xi), 1 F / 2 C (offset 0). */
void orc_ccd_pairs(const orc_topo* tp, const double* x, const double* p, int64_t np,
                   const uint64_t* keys, const uint8_t* klass, double xi, double s, double c_inner,
                   double t_c, int max_iter, double* t_out, int32_t* status, int32_t* iters) {
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < np; ++q) {
        int v[4], ee, st;
        stencil(tp, keys[q], v, &ee);
        double x12[12], p12[12];
        gather12(x, tp->n, v, x12);
        gather12(p, tp->n, v, p12);
        if (klass[q] == 3) {  /* culled: no constraint on the step */
            t_out[q] = t_c;
            iters[q] = 0;
            status[q] = 0;
            continue;
        }
        double off = klass[q] == 0 ? xi : 0.0;
        iters[q] = orc_accd(ee, x12, p12, off, s, c_inner, t_c, max_iter, &t_out[q], &st);
        status[q] = st;
    }
}

/*
 * ORACLE -- test infrastructure only.  Plain, slow, obviously-correct CPU
 * code that the tests, the smoke check and the benchmark's CPU baseline use
 * to check the CUDA library.  Nothing in the product links or calls it.
 * It shares no code with the CUDA library.
 *
 * Scope: mesh snapping and geometry (Section 3, midpoint collocation: A_i,
 * x_i, n_i), pair visibility with back-face culling (Section 3.2),
 * point-sun visibility and insolation (Eq. for the point-sun insolation,
 * Section 2), view-factor entries F_ij (Eq. FF-def, Section 3).
 *
 * Exact predicates.  Vertices are snapped to an integer grid whose unit is
 * the power of two 2^e with extent/2^e <= 2^18 (extent = largest bounding-box
 * side).  Points are carried at scale 3 (3 x centroid = a + b + c is an
 * integer vector), so every orientation determinant below fits in int64
 * (|det| < 2^61.8) and every visibility decision is exact.
 *
 * Occlusion reading (the paper's open segment, Section 3.2): the open segment
 * (x_i, x_j) is blocked by triangle k (k != i, j) iff its endpoints lie
 * strictly on opposite sides of k's plane and the line through them meets the
 * closed triangle (edge and vertex touches block).  A segment in k's plane is
 * not blocked by k.  The pair test runs on (min(i,j), max(i,j)).
 *
 * Sun ray: from x_i along s_q = round(2^20 s) (componentwise), t > 0; blocked
 * by any triangle k != i met with the same rules.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;

/* ---------------------------------------------------------------- snap */
/* Returns 0 on success, -1 for a degenerate (zero-extent) vertex set. */
int or_snap(const double* v, i64 nv, i64* q, double* unit_out, i64* base_out)
{
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = v[a]; hi[a] = v[a]; }
    for (i64 i = 1; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            double x = v[3 * i + a];
            if (x < lo[a]) lo[a] = x;
            if (x > hi[a]) hi[a] = x;
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) if (hi[a] - lo[a] > ext) ext = hi[a] - lo[a];
    if (!(ext > 0.0)) return -1;
    int ex;
    frexp(ext, &ex);                /* ext <= 2^ex */
    double unit = ldexp(1.0, ex - 18);
    i64 base[3];
    for (int a = 0; a < 3; ++a) base[a] = llround(lo[a] / unit);
    for (i64 i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) q[3 * i + a] = llround(v[3 * i + a] / unit) - base[a];
    *unit_out = unit;
    for (int a = 0; a < 3; ++a) base_out[a] = base[a];
    return 0;
}

/* ------------------------------------------------------------ geometry */
/* Per facet: area, centroid (relative to the grid origin), unit normal
 * (right-hand rule), scale-3 integer centroid and integer normal
 * (b-a)x(c-a) in grid units. */
void or_geometry(const i64* q, double unit, const int32_t* f, i64 nf,
                 double* area, double* cent, double* nrm, i64* c3, i64* nint)
{
    for (i64 t = 0; t < nf; ++t) {
        const i64* A = q + 3 * (i64)f[3 * t];
        const i64* B = q + 3 * (i64)f[3 * t + 1];
        const i64* C = q + 3 * (i64)f[3 * t + 2];
        double a[3], b[3], c[3];
        for (int k = 0; k < 3; ++k) { a[k] = (double)A[k] * unit; b[k] = (double)B[k] * unit; c[k] = (double)C[k] * unit; }
        double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        area[t] = 0.5 * len;
        for (int k = 0; k < 3; ++k) {
            cent[3 * t + k] = (a[k] + b[k] + c[k]) / 3.0;
            nrm[3 * t + k] = len > 0 ? cr[k] / len : 0.0;
            c3[3 * t + k] = A[k] + B[k] + C[k];
        }
        i64 iu[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        i64 iw[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        nint[3 * t + 0] = iu[1] * iw[2] - iu[2] * iw[1];
        nint[3 * t + 1] = iu[2] * iw[0] - iu[0] * iw[2];
        nint[3 * t + 2] = iu[0] * iw[1] - iu[1] * iw[0];
    }
}

/* ----------------------------------------------------- exact predicates */
static i64 orient3(const i64* a, const i64* b, const i64* c, const i64* d)
{
    i64 u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
    i64 v0 = c[0] - a[0], v1 = c[1] - a[1], v2 = c[2] - a[2];
    i64 w0 = d[0] - a[0], w1 = d[1] - a[1], w2 = d[2] - a[2];
    i64 x0 = v1 * w2 - v2 * w1, x1 = v2 * w0 - v0 * w2, x2 = v0 * w1 - v1 * w0;
    return u0 * x0 + u1 * x1 + u2 * x2;
}

static int sgn(i64 x) { return (x > 0) - (x < 0); }

/* scale-3 triangle vertices of facet k */
static void tri3(const i64* q, const int32_t* f, i64 k, i64 A[3], i64 B[3], i64 C[3])
{
    for (int a = 0; a < 3; ++a) {
        A[a] = 3 * q[3 * (i64)f[3 * k] + a];
        B[a] = 3 * q[3 * (i64)f[3 * k + 1] + a];
        C[a] = 3 * q[3 * (i64)f[3 * k + 2] + a];
    }
}

/* open segment P-Q (scale 3) against closed triangle A,B,C (scale 3) */
static int seg_blocked(const i64* P, const i64* Q, const i64* A, const i64* B, const i64* C)
{
    int s1 = sgn(orient3(A, B, C, P));
    int s2 = sgn(orient3(A, B, C, Q));
    if (s1 == 0 || s2 == 0 || s1 == s2) return 0;
    int e1 = sgn(orient3(P, Q, A, B));
    int e2 = sgn(orient3(P, Q, B, C));
    int e3 = sgn(orient3(P, Q, C, A));
    return (e1 >= 0 && e2 >= 0 && e3 >= 0) || (e1 <= 0 && e2 <= 0 && e3 <= 0);
}

/* ray P + t D (t > 0) against closed triangle A,B,C */
static int ray_blocked(const i64* P, const i64* D, const i64* A, const i64* B, const i64* C)
{
    i64 u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    i64 w[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    i64 n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    int s1 = sgn(orient3(A, B, C, P));
    int sd = sgn(n[0] * D[0] + n[1] * D[1] + n[2] * D[2]);
    if (s1 == 0 || sd == 0 || s1 == sd) return 0;
    i64 a[3] = {A[0] - P[0], A[1] - P[1], A[2] - P[2]};
    i64 b[3] = {B[0] - P[0], B[1] - P[1], B[2] - P[2]};
    i64 c[3] = {C[0] - P[0], C[1] - P[1], C[2] - P[2]};
    /* e = D . (a x b) etc. */
#define TRIPLE(x, y) (D[0] * (x[1] * y[2] - x[2] * y[1]) + D[1] * (x[2] * y[0] - x[0] * y[2]) + D[2] * (x[0] * y[1] - x[1] * y[0]))
    int e1 = sgn(TRIPLE(a, b));
    int e2 = sgn(TRIPLE(b, c));
    int e3 = sgn(TRIPLE(c, a));
#undef TRIPLE
    return (e1 >= 0 && e2 >= 0 && e3 >= 0) || (e1 <= 0 && e2 <= 0 && e3 <= 0);
}

static int cull_pass(const i64* c3, const i64* nint, i64 i, i64 j)
{
    i64 d0 = c3[3 * j] - c3[3 * i], d1 = c3[3 * j + 1] - c3[3 * i + 1], d2 = c3[3 * j + 2] - c3[3 * i + 2];
    i64 a = nint[3 * i] * d0 + nint[3 * i + 1] * d1 + nint[3 * i + 2] * d2;
    i64 b = -(nint[3 * j] * d0 + nint[3 * j + 1] * d1 + nint[3 * j + 2] * d2);
    return a > 0 && b > 0;
}

/* ------------------------------------------------ brute-force visibility */
/* V (nf x nf, row-major bytes): V_ij = 1 iff the cull passes both ways and no
 * other facet blocks the open segment.  O(N^3). */
void or_visibility_brute(const i64* q, const int32_t* f, i64 nf, const i64* c3, const i64* nint,
                         uint8_t* V)
{
    memset(V, 0, (size_t)(nf * nf));
    for (i64 i = 0; i < nf; ++i)
        for (i64 j = i + 1; j < nf; ++j) {
            if (!cull_pass(c3, nint, i, j)) continue;
            int vis = 1;
            for (i64 k = 0; k < nf && vis; ++k) {
                if (k == i || k == j) continue;
                i64 A[3], B[3], C[3];
                tri3(q, f, k, A, B, C);
                if (seg_blocked(c3 + 3 * i, c3 + 3 * j, A, B, C)) vis = 0;
            }
            V[i * nf + j] = (uint8_t)vis;
            V[j * nf + i] = (uint8_t)vis;
        }
}

/* ------------------------------------------------------- the oracle BVH */
typedef struct { i64 lo[3], hi[3]; i64 left, right, first, count; } obvh_node;
typedef struct { obvh_node* nodes; i64 nnodes; i64* idx; } obvh;

static i64 g_axis;
static const i64* g_c3;
static int cmp_axis(const void* x, const void* y)
{
    i64 a = *(const i64*)x, b = *(const i64*)y;
    i64 ka = g_c3[3 * a + g_axis], kb = g_c3[3 * b + g_axis];
    if (ka != kb) return ka < kb ? -1 : 1;
    return a < b ? -1 : (a > b);
}

static i64 obvh_build_rec(obvh* T, const i64* q, const int32_t* f, const i64* c3, i64 first, i64 count)
{
    i64 id = T->nnodes++;
    obvh_node* nd = &T->nodes[id];
    for (int a = 0; a < 3; ++a) { nd->lo[a] = INT64_MAX; nd->hi[a] = INT64_MIN; }
    i64 clo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, chi[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
    for (i64 s = first; s < first + count; ++s) {
        i64 k = T->idx[s];
        for (int v = 0; v < 3; ++v)
            for (int a = 0; a < 3; ++a) {
                i64 x = 3 * q[3 * (i64)f[3 * k + v] + a];
                if (x < nd->lo[a]) nd->lo[a] = x;
                if (x > nd->hi[a]) nd->hi[a] = x;
            }
        for (int a = 0; a < 3; ++a) {
            if (c3[3 * k + a] < clo[a]) clo[a] = c3[3 * k + a];
            if (c3[3 * k + a] > chi[a]) chi[a] = c3[3 * k + a];
        }
    }
    if (count <= 4) { nd->left = nd->right = -1; nd->first = first; nd->count = count; return id; }
    int ax = 0;
    for (int a = 1; a < 3; ++a) if (chi[a] - clo[a] > chi[ax] - clo[ax]) ax = a;
    g_axis = ax; g_c3 = c3;
    qsort(T->idx + first, (size_t)count, sizeof(i64), cmp_axis);
    i64 half = count / 2;
    i64 l = obvh_build_rec(T, q, f, c3, first, half);
    i64 r = obvh_build_rec(T, q, f, c3, first + half, count - half);
    nd = &T->nodes[id];
    nd->left = l; nd->right = r; nd->first = -1; nd->count = 0;
    return id;
}

void* or_bvh_build(const i64* q, const int32_t* f, i64 nf, const i64* c3)
{
    obvh* T = (obvh*)calloc(1, sizeof(obvh));
    T->nodes = (obvh_node*)calloc((size_t)(2 * nf + 1), sizeof(obvh_node));
    T->idx = (i64*)malloc(sizeof(i64) * (size_t)nf);
    for (i64 k = 0; k < nf; ++k) T->idx[k] = k;
    obvh_build_rec(T, q, f, c3, 0, nf);
    return T;
}

void or_bvh_free(void* p)
{
    obvh* T = (obvh*)p;
    if (!T) return;
    free(T->nodes); free(T->idx); free(T);
}

/* Conservative box test for the parametric set P + t D, t in (t0, t1):
 * the box is widened by 2 units so double rounding can only add boxes. */
static int box_hit(const obvh_node* nd, const i64* P, const double* D, double t0, double t1)
{
    for (int a = 0; a < 3; ++a) {
        double lo = (double)(nd->lo[a] - 2), hi = (double)(nd->hi[a] + 2);
        double p = (double)P[a];
        if (D[a] == 0.0) {
            if (p < lo || p > hi) return 0;
            continue;
        }
        double ta = (lo - p) / D[a], tb = (hi - p) / D[a];
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1 * (1.0 + 1e-12) + 1e-12) return 0;
    }
    return 1;
}

/* any-hit query; mode 0: segment P->Q (excluding facets i, j); mode 1: ray
 * from P along D (excluding facet i) */
static int bvh_blocked(const obvh* T, const i64* q, const int32_t* f, const i64* P, const i64* QD,
                       int mode, i64 i, i64 j)
{
    i64 stack[128];
    int sp = 0;
    stack[sp++] = 0;
    double D[3];
    for (int a = 0; a < 3; ++a) D[a] = mode == 0 ? (double)(QD[a] - P[a]) : (double)QD[a];
    double t1 = mode == 0 ? 1.0 : 1e300;
    while (sp) {
        const obvh_node* nd = &T->nodes[stack[--sp]];
        if (!box_hit(nd, P, D, 0.0, t1)) continue;
        if (nd->left < 0) {
            for (i64 s = nd->first; s < nd->first + nd->count; ++s) {
                i64 k = T->idx[s];
                if (k == i || k == j) continue;
                i64 A[3], B[3], C[3];
                tri3(q, f, k, A, B, C);
                if (mode == 0 ? seg_blocked(P, QD, A, B, C) : ray_blocked(P, QD, A, B, C)) return 1;
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    return 0;
}

/* V rows for the given facets (nrows x nf bytes), BVH-accelerated; identical
 * decisions to or_visibility_brute. */
void or_visibility_rows_bvh(void* bvh, const i64* q, const int32_t* f, i64 nf, const i64* c3,
                            const i64* nint, const i64* rows, i64 nrows, uint8_t* V)
{
    const obvh* T = (const obvh*)bvh;
    for (i64 r = 0; r < nrows; ++r) {
        i64 i = rows[r];
        for (i64 j = 0; j < nf; ++j) {
            uint8_t vis = 0;
            if (j != i && cull_pass(c3, nint, i, j)) {
                i64 a = i < j ? i : j, b = i < j ? j : i;
                vis = !bvh_blocked(T, q, f, c3 + 3 * a, c3 + 3 * b, 0, a, b);
            }
            V[r * nf + j] = vis;
        }
    }
}

/* --------------------------------------------------------- sun visibility */
void or_quantize_dir(const double* s, i64* sq)
{
    for (int a = 0; a < 3; ++a) sq[a] = llround(ldexp(s[a], 20));
}

/* vis[i] = 1 iff nint_i . s_q > 0 and the ray from x_i along s_q is not
 * blocked; brute force over all facets when bvh == NULL. */
void or_sun_visibility(void* bvh, const i64* q, const int32_t* f, i64 nf, const i64* c3,
                       const i64* nint, const double* s, uint8_t* vis)
{
    i64 D[3];
    or_quantize_dir(s, D);
    for (i64 i = 0; i < nf; ++i) {
        i64 nd = nint[3 * i] * D[0] + nint[3 * i + 1] * D[1] + nint[3 * i + 2] * D[2];
        if (nd <= 0) { vis[i] = 0; continue; }
        int blocked = 0;
        if (bvh) {
            blocked = bvh_blocked((const obvh*)bvh, q, f, c3 + 3 * i, D, 1, i, -1);
        } else {
            for (i64 k = 0; k < nf && !blocked; ++k) {
                if (k == i) continue;
                i64 A[3], B[3], C[3];
                tri3(q, f, k, A, B, C);
                blocked = ray_blocked(c3 + 3 * i, D, A, B, C);
            }
        }
        vis[i] = (uint8_t)!blocked;
    }
}

/* ------------------------------------------------------------ F entries */
/* Rows of F (Eq. FF-def): F_ij = [n_i.(x_j-x_i)][n_j.(x_i-x_j)] V_ij A_j /
 * (pi |x_i-x_j|^4), F_ii = 0.  Vrows is nrows x nf (bytes). */
void or_F_rows(const double* area, const double* cent, const double* nrm, i64 nf,
               const i64* rows, i64 nrows, const uint8_t* Vrows, double* Frows)
{
    const double pi = 3.14159265358979323846;
    for (i64 r = 0; r < nrows; ++r) {
        i64 i = rows[r];
        for (i64 j = 0; j < nf; ++j) {
            double val = 0.0;
            if (j != i && Vrows[r * nf + j]) {
                double d[3] = {cent[3 * j] - cent[3 * i], cent[3 * j + 1] - cent[3 * i + 1], cent[3 * j + 2] - cent[3 * i + 2]};
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double ci = nrm[3 * i] * d[0] + nrm[3 * i + 1] * d[1] + nrm[3 * i + 2] * d[2];
                double cj = -(nrm[3 * j] * d[0] + nrm[3 * j + 1] * d[1] + nrm[3 * j + 2] * d[2]);
                val = ci * cj * area[j] / (pi * r2 * r2);
            }
            Frows[r * nf + j] = val;
        }
    }
}

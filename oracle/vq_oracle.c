/*
 * vq_oracle.c -- CPU oracle for the planar Quickhull of the VQhull paper
 * (arxiv 2510.09417).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code
 * with the CUDA path, and the CUDA path never calls it.
 *
 * Plain, sequential, slow on purpose.  Every predicate is exact:
 *   - orient(a,b,c): the paper's left-of test, Sec. 2.1 (first display),
 *     (px-ux)(qy-uy) > (py-uy)(qx-ux), i.e. orient(p,q,u) > 0;
 *   - the paper's farther-than test, Sec. 2.1 (second display),
 *     (qy-py)(ux-u'x) < (qx-px)(uy-u'y), i.e. the sign of (q-p) x (u-u');
 *   - a dot product sign used by the tie rule below.
 * Each is first tried with the FP64 error-bound filter of Shewchuk,
 * "Adaptive Precision Floating-Point Arithmetic and Fast Robust Geometric
 * Predicates" (1997), Sec. 4 (bound (3 + 16 eps) eps * detsum for a
 * two-product determinant of rounded differences), then settled exactly by
 * summing the products of the raw coordinates as big integers.  Build with
 * -ffp-contract=off so the filter's products and sums are rounded one by one.
 *
 * The hull follows Algorithm 1 (Sec. 2.1) step by step with an explicit
 * stack instead of recursion.  Readings where the paper is silent:
 *   - leftmost / rightmost: lexicographic (x, then y) min / max; among
 *     coincident points the lowest index;
 *   - "to the left of" is strict: orient = 0 is discarded, so the output
 *     holds strict vertices only, each coordinate pair once;
 *   - farthest point: max orient(a,b,u); ties broken by the smaller
 *     projection (b-a).u (the tied point nearest a), then the lowest index;
 *   - clockwise with the y axis up, starting at the lexicographic minimum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_NONFINITE (-2)
#define ORC_ERR_NOMEM (-4)

/* ------------------------------------------------------------------ */
/* Exact sign of a sum of signed products of doubles (big integers).   */
/* ------------------------------------------------------------------ */

/* Exponents of products of two finite doubles lie in [-2252, 1942] after
 * scaling each mantissa to a 53-bit integer, so a product shifted to the
 * smallest exponent needs < 4200 + 106 bits.  140 limbs of 32 bits hold
 * that with room for the carries of up to 16 terms. */
#define ORC_LIMBS 140

typedef struct {
    uint32_t w[ORC_LIMBS];
} orc_big;

static long long orc_exact_calls = 0;

/* v = m * 2^e with m an integer of at most 53 bits (sign kept separately). */
static void orc_split(double v, uint64_t *m, int *e, int *s)
{
    int ex;
    double f = frexp(fabs(v), &ex); /* |v| = f * 2^ex, f in [0.5, 1) */
    *m = (uint64_t)ldexp(f, 53);    /* exact: f has at most 53 bits  */
    *e = ex - 53;
    *s = v < 0 ? -1 : 1;
}

static void orc_big_add_shifted(orc_big *acc, unsigned __int128 mag, int shift)
{
    int limb = shift / 32;
    int bit = shift % 32;
    /* mag < 2^106; shifted by < 32 bits it fits in 138 bits = 5 limbs. */
    uint32_t part[6];
    unsigned __int128 lo = mag << bit; /* low 128 bits */
    unsigned __int128 hi = bit ? (mag >> (128 - bit)) : 0;
    for (int i = 0; i < 4; i++) part[i] = (uint32_t)(lo >> (32 * i));
    part[4] = (uint32_t)hi;
    part[5] = (uint32_t)(hi >> 32);
    uint64_t carry = 0;
    for (int i = 0; limb + i < ORC_LIMBS; i++) {
        uint64_t add = (i < 6) ? part[i] : 0;
        if (i >= 6 && carry == 0) break;
        uint64_t t = (uint64_t)acc->w[limb + i] + add + carry;
        acc->w[limb + i] = (uint32_t)t;
        carry = t >> 32;
    }
}

/* sign( sum_k sg[k] * a[k] * b[k] ), exactly. */
static int orc_sum_products_sign(int nterm, const double *a, const double *b, const int *sg)
{
    uint64_t ma[16], mb[16];
    int ea[16], eb[16], sa[16], sb[16];
    int emin = 1 << 30;
    int live = 0;
    orc_exact_calls++;
    for (int k = 0; k < nterm; k++) {
        if (a[k] == 0.0 || b[k] == 0.0) {
            ma[k] = 0;
            continue;
        }
        orc_split(a[k], &ma[k], &ea[k], &sa[k]);
        orc_split(b[k], &mb[k], &eb[k], &sb[k]);
        if (ea[k] + eb[k] < emin) emin = ea[k] + eb[k];
        live++;
    }
    if (!live) return 0;
    orc_big pos, neg;
    memset(&pos, 0, sizeof pos);
    memset(&neg, 0, sizeof neg);
    for (int k = 0; k < nterm; k++) {
        if (ma[k] == 0) continue;
        unsigned __int128 mag = (unsigned __int128)ma[k] * mb[k];
        int sign = sg[k] * sa[k] * sb[k];
        orc_big_add_shifted(sign > 0 ? &pos : &neg, mag, ea[k] + eb[k] - emin);
    }
    for (int i = ORC_LIMBS - 1; i >= 0; i--) {
        if (pos.w[i] != neg.w[i]) return pos.w[i] > neg.w[i] ? 1 : -1;
    }
    return 0;
}

/* Shewchuk (1997), Sec. 4: with eps = 2^-53, a determinant t1 - t2 (or sum
 * t1 + t2) of products of rounded differences has the sign of its rounded
 * value whenever |value| >= (3 + 16 eps) eps (|t1| + |t2|). */
static int orc_use_filter = 1;
static const double ORC_EPS = 1.1102230246251565404e-16; /* 2^-53 */

static int orc_filter(double t1, double t2, double det, int *sign)
{
    if (!orc_use_filter) return 0;
    double bound = (3.0 + 16.0 * ORC_EPS) * ORC_EPS * (fabs(t1) + fabs(t2));
    if (det > bound || -det > bound) {
        *sign = det > 0 ? 1 : -1;
        return 1;
    }
    if (bound == 0.0 && det == 0.0) { /* both products exactly zero */
        *sign = 0;
        return 1;
    }
    return 0;
}

/* orient(a,b,c) = (bx-ax)(cy-ay) - (by-ay)(cx-ax); > 0 iff c is to the
 * left of a->b.  Sec. 2.1 writes the same determinant as
 * (ax-cx)(by-cy) - (ay-cy)(bx-cx). */
int orc_orient_sign(double ax, double ay, double bx, double by, double cx, double cy)
{
    double t1 = (bx - ax) * (cy - ay);
    double t2 = (by - ay) * (cx - ax);
    int s;
    if (orc_filter(t1, t2, t1 - t2, &s)) return s;
    /* expand: bx*cy - bx*ay - ax*cy - by*cx + by*ax + ay*cx (ax*ay cancels) */
    const double a[6] = {bx, bx, ax, by, by, ay};
    const double b[6] = {cy, ay, cy, cx, ax, cx};
    const int sg[6] = {+1, -1, -1, -1, +1, +1};
    return orc_sum_products_sign(6, a, b, sg);
}

/* sign of (p1 - p0) x (q1 - q0).  With p0 = a, p1 = b, q1 = u, q0 = u' this
 * is the farther-than test of Sec. 2.1: > 0 iff u is farther to the left of
 * a->b than u'. */
int orc_cross_sign(double p0x, double p0y, double p1x, double p1y,
                   double q0x, double q0y, double q1x, double q1y)
{
    double t1 = (p1x - p0x) * (q1y - q0y);
    double t2 = (p1y - p0y) * (q1x - q0x);
    int s;
    if (orc_filter(t1, t2, t1 - t2, &s)) return s;
    const double a[8] = {p1x, p1x, p0x, p0x, p1y, p1y, p0y, p0y};
    const double b[8] = {q1y, q0y, q1y, q0y, q1x, q0x, q1x, q0x};
    const int sg[8] = {+1, -1, -1, +1, -1, +1, +1, -1};
    return orc_sum_products_sign(8, a, b, sg);
}

/* sign of (p1 - p0) . (q1 - q0) */
int orc_dot_sign(double p0x, double p0y, double p1x, double p1y,
                 double q0x, double q0y, double q1x, double q1y)
{
    double t1 = (p1x - p0x) * (q1x - q0x);
    double t2 = (p1y - p0y) * (q1y - q0y);
    int s;
    if (orc_filter(t1, -t2, t1 + t2, &s)) return s;
    const double a[8] = {p1x, p1x, p0x, p0x, p1y, p1y, p0y, p0y};
    const double b[8] = {q1x, q0x, q1x, q0x, q1y, q0y, q1y, q0y};
    const int sg[8] = {+1, -1, -1, +1, +1, -1, -1, +1};
    return orc_sum_products_sign(8, a, b, sg);
}

/* Checker of an approximate orient with an error bound (used by the tests
 * of the device's FP32 tier): for m triples tri[6k .. 6k+5] = (ax, ay, bx,
 * by, cx, cy), counts the k whose exact orient(a,b,c) (the left-of test of
 * Sec. 2.1) lies outside [d[k] - e[k], d[k] + e[k]], and in *sign_bad the k
 * with |d[k]| > e[k] whose sign differs from the exact sign.  Both tests
 * are exact sums of products: orient - d + e >= 0 and d + e - orient >= 0. */
int64_t orc_orient_bound_check(const double *tri, int64_t m, const float *d, const float *e, int64_t *sign_bad)
{
    int64_t out = 0, bad = 0;
    for (int64_t k = 0; k < m; k++) {
        const double *t = tri + 6 * k;
        const double ax = t[0], ay = t[1], bx = t[2], by = t[3], cx = t[4], cy = t[5];
        const double dk = d[k], ek = e[k];
        /* orient = bx*cy - bx*ay - ax*cy - by*cx + by*ax + ay*cx */
        const double a[8] = {bx, bx, ax, by, by, ay, dk, ek};
        const double b[8] = {cy, ay, cy, cx, ax, cx, 1.0, 1.0};
        const int lo[8] = {+1, -1, -1, -1, +1, +1, -1, +1}; /* orient - d + e */
        const int hi[8] = {-1, +1, +1, +1, -1, -1, +1, +1}; /* d + e - orient */
        if (orc_sum_products_sign(8, a, b, lo) < 0 || orc_sum_products_sign(8, a, b, hi) < 0) out++;
        if (fabs(dk) > ek) {
            const int s = orc_sum_products_sign(6, a, b, lo);
            const int want = dk > 0 ? 1 : -1;
            if (s != want) bad++;
        }
    }
    if (sign_bad) *sign_bad = bad;
    return out;
}

void orc_set_filter(int on) { orc_use_filter = on ? 1 : 0; }
long long orc_exact_count(void) { return orc_exact_calls; }

/* ------------------------------------------------------------------ */
/* Quickhull, Algorithm 1, with an explicit stack                       */
/* ------------------------------------------------------------------ */

#define ORC_MAX_LEVELS 512

typedef struct {
    int64_t levels;                        /* deepest partition level + 1      */
    int64_t read[ORC_MAX_LEVELS];          /* points read by partitions        */
    int64_t written[ORC_MAX_LEVELS];       /* points kept (|S1| + |S2|)        */
    int64_t segments[ORC_MAX_LEVELS];      /* partition calls                  */
    int64_t exact_calls;                   /* exact (non-filtered) evaluations */
    double paper_bytes;                    /* byte model of Sec. 5.2 / 5.3     */
} orc_stats;

/* Does u beat v as the farthest point from a->b?  (max orient, then min
 * projection on b - a, then lowest index) */
static int orc_farther(const double *x, const double *y, int32_t a, int32_t b,
                       int32_t u, int32_t v)
{
    int c = orc_cross_sign(x[a], y[a], x[b], y[b], x[v], y[v], x[u], y[u]);
    if (c != 0) return c > 0;
    int d = orc_dot_sign(x[a], y[a], x[b], y[b], x[v], y[v], x[u], y[u]);
    if (d != 0) return d < 0;
    return u < v;
}

/* Index of the farthest point to the left of a->b among cand[0..m), by the
 * rule above; -1 when m = 0.  Exposed so the tie rule can be pinned alone. */
int32_t orc_farthest(const double *x, const double *y, int32_t a, int32_t b,
                     const int32_t *cand, int64_t m)
{
    int32_t best = -1;
    for (int64_t k = 0; k < m; k++)
        if (best < 0 || orc_farther(x, y, a, b, cand[k], best)) best = cand[k];
    return best;
}

typedef struct {
    int64_t lo, hi;   /* range of the index array holding P (r included) */
    int32_t a, r, b;  /* Hull(P, a, r, b); r < 0 marks an "emit a" task   */
    int32_t level;
} orc_task;

static void orc_level_add(orc_stats *st, int level, int64_t rd, int64_t wr)
{
    int l = level < ORC_MAX_LEVELS ? level : ORC_MAX_LEVELS - 1;
    st->read[l] += rd;
    st->written[l] += wr;
    st->segments[l] += 1;
    if (level + 1 > st->levels) st->levels = level + 1;
}

/*
 * Convex hull of (x[i], y[i]), i < n.  Writes the hull's vertex indices,
 * clockwise from the lexicographic minimum, to out (capacity n) and returns
 * their count h, or ORC_ERR_NONFINITE / ORC_ERR_NOMEM.
 */
int64_t orc_hull(const double *x, const double *y, int64_t n, int32_t *out, orc_stats *st)
{
    orc_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof *st);
    long long exact0 = orc_exact_calls;
    if (n <= 0) return 0;
    for (int64_t i = 0; i < n; i++)
        if (!isfinite(x[i]) || !isfinite(y[i])) return ORC_ERR_NONFINITE;

    /* Alg. 1, first two steps: leftmost p and rightmost q. */
    int32_t p = 0, q = 0;
    for (int64_t i = 1; i < n; i++) {
        if (x[i] < x[p] || (x[i] == x[p] && y[i] < y[p])) p = (int32_t)i;
        if (x[i] > x[q] || (x[i] == x[q] && y[i] > y[q])) q = (int32_t)i;
    }
    st->paper_bytes = 8.0 * (double)n;
    int64_t h = 0;
    if (p == q) { /* every point coincides with p */
        out[h++] = p;
        return h;
    }

    int32_t *idx = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *tmp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t cap = 2 * n + 16;
    orc_task *stack = (orc_task *)malloc((size_t)cap * sizeof(orc_task));
    if (!idx || !tmp || !stack) {
        free(idx); free(tmp); free(stack);
        return ORC_ERR_NOMEM;
    }

    /* Alg. 1, S1 / S2 around p->q and their farthest points r1 / r2.
     * S1 goes to the front of idx, S2 to the back. */
    int64_t n1 = 0, n2 = 0;
    int32_t r1 = -1, r2 = -1;
    for (int64_t i = 0; i < n; i++) {
        int32_t u = (int32_t)i;
        int s = orc_orient_sign(x[p], y[p], x[q], y[q], x[u], y[u]);
        if (s > 0) {
            idx[n1++] = u;
            if (r1 < 0 || orc_farther(x, y, p, q, u, r1)) r1 = u;
        } else if (s < 0) {
            idx[n - 1 - n2++] = u;
            if (r2 < 0 || orc_farther(x, y, q, p, u, r2)) r2 = u;
        }
    }
    orc_level_add(st, 0, n, n1 + n2);

    /* H = {p} u Hull(S1, p, r1, q) u {q} u Hull(S2, q, r2, p), in order.
     * Tasks pop in LIFO order, so push the last part first. */
    int64_t top = 0;
    if (n2 > 0) stack[top++] = (orc_task){n - n2, n, q, r2, p, 1};
    stack[top++] = (orc_task){0, 0, q, -1, -1, 0}; /* emit q */
    if (n1 > 0) stack[top++] = (orc_task){0, n1, p, r1, q, 1};
    out[h++] = p;

    while (top > 0) {
        orc_task t = stack[--top];
        if (t.r < 0) { /* emit vertex t.a */
            out[h++] = t.a;
            continue;
        }
        int64_t m = t.hi - t.lo;
        if (m <= 1) { /* Alg. 1: |P| <= 1 -> P, which is {r} */
            out[h++] = t.r;
            continue;
        }
        /* S1 left of a->r with farthest r1; S2 left of r->b with farthest r2 */
        int32_t a = t.a, r = t.r, b = t.b;
        int64_t k1 = 0, k2 = 0;
        int32_t s1r = -1, s2r = -1;
        for (int64_t i = t.lo; i < t.hi; i++) {
            int32_t u = idx[i];
            if (orc_orient_sign(x[a], y[a], x[r], y[r], x[u], y[u]) > 0) {
                tmp[t.lo + k1++] = u;
                if (s1r < 0 || orc_farther(x, y, a, r, u, s1r)) s1r = u;
            } else if (orc_orient_sign(x[r], y[r], x[b], y[b], x[u], y[u]) > 0) {
                tmp[t.hi - 1 - k2++] = u;
                if (s2r < 0 || orc_farther(x, y, r, b, u, s2r)) s2r = u;
            }
        }
        for (int64_t i = 0; i < k1; i++) idx[t.lo + i] = tmp[t.lo + i];
        for (int64_t i = 0; i < k2; i++) idx[t.hi - 1 - i] = tmp[t.hi - 1 - i];
        orc_level_add(st, t.level, m, k1 + k2);
        /* Return Hull(S1, a, r1, r) ++ [r] ++ Hull(S2, r, r2, b). */
        if (top + 3 > cap) break; /* cannot happen: depth <= n */
        if (k2 > 0) stack[top++] = (orc_task){t.hi - k2, t.hi, r, s2r, b, t.level + 1};
        stack[top++] = (orc_task){0, 0, r, -1, -1, t.level};
        if (k1 > 0) stack[top++] = (orc_task){t.lo, t.lo + k1, a, s1r, r, t.level + 1};
    }
    free(idx);
    free(tmp);
    free(stack);

    /* Byte model of Sec. 5.2: 16 bytes (x and y) per point read or kept by
     * each partition, on top of the 8n of the extreme search. */
    for (int l = 0; l < ORC_MAX_LEVELS; l++)
        st->paper_bytes += 16.0 * (double)(st->read[l] + st->written[l]);
    st->exact_calls = (int64_t)(orc_exact_calls - exact0);
    return h;
}

/* ------------------------------------------------------------------ */
/* Verifier: the invariants that determine the hull uniquely            */
/* ------------------------------------------------------------------ */

#define ORC_V_OK 0
#define ORC_V_COUNT 1       /* h = 0 with n > 0, or h > n               */
#define ORC_V_RANGE 2       /* index outside [0, n)                       */
#define ORC_V_START 3       /* H[0] is not the lowest-index lex minimum   */
#define ORC_V_CONVEX 4      /* a turn that is not strictly clockwise      */
#define ORC_V_MONOTONE 5    /* chains not x-monotone around the lex max   */
#define ORC_V_OUTSIDE 6     /* an input point strictly outside the hull   */
#define ORC_V_DUPINDEX 7    /* a vertex not the lowest index at its spot  */
#define ORC_V_DEGENERATE 8  /* 1- or 2-vertex hull that does not hold     */

static int orc_lex_less(double ax, double ay, double bx, double by)
{
    return ax < bx || (ax == bx && ay < by);
}

typedef struct {
    double x, y;
    int32_t i;
} orc_vtx;

static int orc_vtx_cmp(const void *pa, const void *pb)
{
    const orc_vtx *a = (const orc_vtx *)pa, *b = (const orc_vtx *)pb;
    if (orc_lex_less(a->x, a->y, b->x, b->y)) return -1;
    if (orc_lex_less(b->x, b->y, a->x, a->y)) return 1;
    return 0;
}

/*
 * Checks hull H (h indices) of the n points against the definition: H is a
 * strictly convex polygon, clockwise from the lowest-index lexicographic
 * minimum, made of input points, each the lowest index at its coordinates,
 * and no input point lies outside it.  Only points lo <= i < hi are tested
 * for containment and for lower duplicate indices (so callers may split the
 * O(n log h) scan); the polygon itself is checked in every call.  Returns
 * ORC_V_OK or the first failed invariant, and its point in *bad.
 */
int orc_verify(const double *x, const double *y, int64_t n, const int32_t *H, int64_t h,
               int64_t lo, int64_t hi, int64_t *bad)
{
    int64_t dummy;
    if (!bad) bad = &dummy;
    *bad = -1;
    if (n == 0) return h == 0 ? ORC_V_OK : ORC_V_COUNT;
    if (h <= 0 || h > n) return ORC_V_COUNT;
    for (int64_t k = 0; k < h; k++)
        if (H[k] < 0 || H[k] >= n) { *bad = k; return ORC_V_RANGE; }
    if (lo < 0) lo = 0;
    if (hi > n) hi = n;
    const int32_t s = H[0];

    /* start vertex: lexicographic minimum; lowest index checked below */
    for (int64_t i = lo; i < hi; i++)
        if (orc_lex_less(x[i], y[i], x[s], y[s])) { *bad = i; return ORC_V_START; }

    if (h == 1) {
        for (int64_t i = lo; i < hi; i++) {
            if (x[i] != x[s] || y[i] != y[s]) { *bad = i; return ORC_V_DEGENERATE; }
            if (i < s) { *bad = i; return ORC_V_DUPINDEX; }
        }
        return ORC_V_OK;
    }
    if (h == 2) {
        const int32_t e = H[1];
        if (!orc_lex_less(x[s], y[s], x[e], y[e])) return ORC_V_DEGENERATE;
        for (int64_t i = lo; i < hi; i++) {
            if (orc_orient_sign(x[s], y[s], x[e], y[e], x[i], y[i]) != 0 ||
                orc_lex_less(x[e], y[e], x[i], y[i])) { *bad = i; return ORC_V_OUTSIDE; }
            if ((x[i] == x[s] && y[i] == y[s] && i < s) ||
                (x[i] == x[e] && y[i] == y[e] && i < e)) { *bad = i; return ORC_V_DUPINDEX; }
        }
        return ORC_V_OK;
    }

    /* strictly clockwise turns everywhere */
    for (int64_t k = 0; k < h; k++) {
        int32_t a = H[k], b = H[(k + 1) % h], c = H[(k + 2) % h];
        if (orc_orient_sign(x[a], y[a], x[b], y[b], x[c], y[c]) >= 0) { *bad = k; return ORC_V_CONVEX; }
    }
    /* one upper chain H[0..m] with non-decreasing x ending at the lex max H[m],
     * then a lower chain H[m..h-1], H[0] with non-increasing x: with the
     * strict turns this makes a simple convex polygon */
    int64_t m = 0;
    for (int64_t k = 1; k < h; k++)
        if (orc_lex_less(x[H[m]], y[H[m]], x[H[k]], y[H[k]])) m = k;
    for (int64_t k = 0; k < m; k++)
        if (x[H[k + 1]] < x[H[k]]) { *bad = k; return ORC_V_MONOTONE; }
    for (int64_t k = m; k < h; k++)
        if (x[H[(k + 1) % h]] > x[H[k]]) { *bad = k; return ORC_V_MONOTONE; }
    for (int64_t i = lo; i < hi; i++)
        if (orc_lex_less(x[H[m]], y[H[m]], x[i], y[i])) { *bad = i; return ORC_V_OUTSIDE; }

    /* sorted vertex coordinates for the lowest-index test */
    orc_vtx *vs = (orc_vtx *)malloc((size_t)h * sizeof(orc_vtx));
    if (!vs) return ORC_ERR_NOMEM;
    for (int64_t k = 0; k < h; k++) vs[k] = (orc_vtx){x[H[k]], y[H[k]], H[k]};
    qsort(vs, (size_t)h, sizeof(orc_vtx), orc_vtx_cmp);

    int rc = ORC_V_OK;
    for (int64_t i = lo; i < hi && rc == ORC_V_OK; i++) {
        const double ux = x[i], uy = y[i];
        /* upper chain: last k < m with x[H[k]] <= ux < x[H[k+1]] (or the
         * final edge when ux equals the lex max's x) */
        int64_t l0 = 0, h0 = m - 1;
        while (l0 < h0) {
            int64_t mid = (l0 + h0 + 1) / 2;
            if (x[H[mid]] <= ux) l0 = mid; else h0 = mid - 1;
        }
        while (l0 < m - 1 && x[H[l0 + 1]] == x[H[l0]]) l0++; /* skip a vertical edge */
        {
            int32_t a = H[l0], b = H[l0 + 1];
            if (orc_orient_sign(x[a], y[a], x[b], y[b], ux, uy) > 0) { *bad = i; rc = ORC_V_OUTSIDE; break; }
        }
        /* lower chain H[m], ..., H[h-1], H[0]: x non-increasing */
        int64_t cnt = h - m; /* number of lower edges */
        int64_t l1 = 0, h1 = cnt - 1;
        while (l1 < h1) {
            int64_t mid = (l1 + h1 + 1) / 2;
            if (x[H[(m + mid) % h]] >= ux) l1 = mid; else h1 = mid - 1;
        }
        while (l1 < cnt - 1 && x[H[(m + l1 + 1) % h]] == x[H[(m + l1) % h]]) l1++;
        {
            int32_t a = H[(m + l1) % h], b = H[(m + l1 + 1) % h];
            if (orc_orient_sign(x[a], y[a], x[b], y[b], ux, uy) > 0) { *bad = i; rc = ORC_V_OUTSIDE; break; }
        }
        /* a point at a vertex's coordinates must not have a lower index */
        int64_t a0 = 0, a1 = h;
        while (a0 < a1) {
            int64_t mid = (a0 + a1) / 2;
            if (orc_lex_less(vs[mid].x, vs[mid].y, ux, uy)) a0 = mid + 1; else a1 = mid;
        }
        if (a0 < h && vs[a0].x == ux && vs[a0].y == uy && i < vs[a0].i) { *bad = i; rc = ORC_V_DUPINDEX; }
    }
    free(vs);
    return rc;
}

/* Number of struct bytes, so the Python side can check its mirror. */
int64_t orc_stats_size(void) { return (int64_t)sizeof(orc_stats); }
int64_t orc_max_levels(void) { return ORC_MAX_LEVELS; }

/*
 * AD-LBR reference oracle in plain C, FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is not part of the product: only the
 * test suite, __graft_entry__.smoke() and the CPU-baseline / reference legs of
 * bench.py may load it.  It shares no code, header or table with the CUDA
 * library; the two are written independently and compared in the tests.
 *
 * It follows Fehrenbach & Mirebeau, "Sparse Non-Negative Stencils for
 * Anisotropic Diffusion":
 *   - Sec. 1, Eqs. def:M and eq:DM: in 2D, <e^perp, D f^perp> = <e, adj(D) f>
 *     and M = adj(D) / sqrt(det D).  Every decision below only needs the SIGN
 *     of a scalar product <e, M f> (or of a difference of two squared
 *     M-norms), and M is a positive multiple of S := adj(D), so the oracle
 *     works with S and takes no square root.
 *   - Sec. 2, Eq. GaussAlgo: Lagrange's reduction, Do (e,f) := (f, e -
 *     Round(<e,Mf>/|f|_M^2) f) while |e|_M > |f|_M, from the canonical basis.
 *   - Sec. 2, the three-step 2D construction that follows Corollary
 *     ObtuseSuperBaseFromReducedBasis2: reduce, flip f so that <e,Mf> <= 0,
 *     superbase (e, f, -e-f); stencil Eq. def:Vz and weights Eq. def:GammaZ.
 *   - Sec. 2, Def. ReducedBasis and the greedy reduction it cites (Nguyen and
 *     Stehle) for the 3D D-reduced basis; Prop. MakeObtuse, Eqs.
 *     SignedOrderedIneq and 3DSuperBase; Selling's stencil (Lemma Selling,
 *     Eq. DSum3D): offsets e_k x e_l, weights -<e_i, D e_j>/2.
 *   - Sec. 1, Eq. def:E*: the operator is A = (1/2) grad E_h with h = 1, and
 *     the Neumann rule V(z;h) = {e in V(z): z + h e in Omega_h}.
 *
 * Exactness.  Every decision (loop test, sign flip, permutation, signs,
 * zero weight) is the sign of sum_k n_k x_k with small integers n_k and the
 * FP64 entries x_k of D.  It is evaluated exactly: each product n_k * x_k is
 * split into two doubles with an fma (the "TwoProduct" error-free
 * transformation of Ogita, Rump and Oishi), and the sum is accumulated as a
 * non-overlapping floating-point expansion with Shewchuk's Grow-Expansion
 * (Shewchuk 1997, "Adaptive precision floating-point arithmetic and fast
 * robust geometric predicates").  The sign of an expansion is the sign of its
 * largest component.  This file must be compiled with -ffp-contract=off so
 * that the compiler does not fuse the error-free transformations.
 *
 * Canonical output (the paper leaves order and sign free): an offset whose
 * weight is exactly zero is stored as the zero vector with weight +0; every
 * other offset is negated if needed so that its first non-zero coordinate
 * (x, then y, then z) is positive; the (offset, weight) pairs are then sorted
 * lexicographically on (x, y[, z]).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    OR_OK = 0,
    OR_E_NOT_SPD = 3,
    OR_E_NONFINITE = 4,
    OR_E_NOT_CONVERGED = 5,
    OR_E_RANGE = 8,
    OR_E_INTERNAL = 9
};

/* ------------------------------------------------------------------------- */
/* Exact sign / accurate value of sum_k n_k x_k                              */
/* ------------------------------------------------------------------------- */

#define OR_MAXTERMS 12

/* Knuth's TwoSum: a + b = s + e exactly. */
static void or_two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

/* Shewchuk's Grow-Expansion with zero elimination: adds b to the
 * non-overlapping expansion h[0..m) (increasing magnitude) in place. */
static int or_grow(double *h, int m, double b)
{
    double q = b;
    int mm = 0;
    for (int i = 0; i < m; i++) {
        double s, e;
        or_two_sum(q, h[i], &s, &e);
        q = s;
        if (e != 0.0)
            h[mm++] = e;
    }
    if (q != 0.0)
        h[mm++] = q;
    return mm;
}

/* Builds the exact expansion of sum_k n[k] * x[k]; returns its length. */
static int or_expansion(int K, const double *x, const long *n, double *h)
{
    int m = 0;
    for (int k = 0; k < K; k++) {
        double nk = (double)n[k];
        double p = nk * x[k];
        double pe = fma(nk, x[k], -p); /* exact low part of the product */
        m = or_grow(h, m, pe);
        m = or_grow(h, m, p);
    }
    return m;
}

static int or_sign_sum(int K, const double *x, const long *n)
{
    double h[2 * OR_MAXTERMS + 2];
    int m = or_expansion(K, x, n, h);
    if (m == 0)
        return 0;
    return h[m - 1] > 0.0 ? 1 : -1;
}

static double or_value_sum(int K, const double *x, const long *n)
{
    double h[2 * OR_MAXTERMS + 2];
    int m = or_expansion(K, x, n, h);
    double v = 0.0;
    for (int i = 0; i < m; i++) /* smallest components first */
        v += h[i];
    return v;
}

/* Exported for the tests that pin the predicate against exact rationals. */
int or_exact_sign(int K, const double *x, const long *n)
{
    if (K < 0 || K > OR_MAXTERMS)
        return -2;
    return or_sign_sum(K, x, n);
}

double or_exact_value(int K, const double *x, const long *n)
{
    if (K < 0 || K > OR_MAXTERMS)
        return NAN;
    return or_value_sum(K, x, n);
}

/* ------------------------------------------------------------------------- */
/* 2D: scalar products <u, S v> with S = adj(D) = [[c, -b], [-b, a]]         */
/* ------------------------------------------------------------------------- */

typedef struct {
    long x, y;
} v2;

/* D = [[a, b], [b, c]] given as (a, b, c).
 * <u, adj(D) v> = c ux vx - b (ux vy + uy vx) + a uy vy = <u^perp, D v^perp>. */
static void or_terms2(const double D[3], v2 u, v2 v, double x[3], long n[3])
{
    x[0] = D[2];
    n[0] = u.x * v.x;
    x[1] = D[1];
    n[1] = -(u.x * v.y + u.y * v.x);
    x[2] = D[0];
    n[2] = u.y * v.y;
}

static int or_sgnS(const double D[3], v2 u, v2 v)
{
    double x[3];
    long n[3];
    or_terms2(D, u, v, x, n);
    return or_sign_sum(3, x, n);
}

static double or_valS(const double D[3], v2 u, v2 v)
{
    double x[3];
    long n[3];
    or_terms2(D, u, v, x, n);
    return or_value_sum(3, x, n);
}

static v2 v2_sub(v2 a, v2 b) { v2 r = {a.x - b.x, a.y - b.y}; return r; }
static v2 v2_add(v2 a, v2 b) { v2 r = {a.x + b.x, a.y + b.y}; return r; }
static v2 v2_neg(v2 a) { v2 r = {-a.x, -a.y}; return r; }

/* sign(|u|_M^2 - |v|_M^2) = sign(<u - v, M (u + v)>). */
static int or_cmp_norm2(const double D[3], v2 u, v2 v)
{
    return or_sgnS(D, v2_sub(u, v), v2_add(u, v));
}

static int or_check_spd2(const double D[3])
{
    for (int i = 0; i < 3; i++)
        if (!isfinite(D[i]))
            return OR_E_NONFINITE;
    if (!(D[0] > 0.0) || !(D[2] > 0.0))
        return OR_E_NOT_SPD;
    /* det D = a c - b^2 > 0, exactly */
    double h[8];
    int m = 0;
    double p = D[0] * D[2], pe = fma(D[0], D[2], -p);
    double q = -D[1] * D[1], qe = fma(-D[1], D[1], -q);
    m = or_grow(h, m, pe);
    m = or_grow(h, m, p);
    m = or_grow(h, m, qe);
    m = or_grow(h, m, q);
    if (m == 0 || h[m - 1] <= 0.0)
        return OR_E_NOT_SPD;
    return OR_OK;
}

static int or_canon_less2(const long *a, const long *b)
{
    if (a[0] != b[0])
        return a[0] < b[0];
    return a[1] < b[1];
}

/* One point of the 2D construction (Sec. 2).  offs[3][2], w[3]. */
static int or_stencil2(const double D[3], int32_t *offs, double *w, int *iters)
{
    int st = or_check_spd2(D);
    if (st != OR_OK)
        return st;

    /* (i) Lagrange's algorithm, Eq. GaussAlgo, from the canonical basis. */
    v2 e = {1, 0}, f = {0, 1};
    int it = 0;
    for (;;) {
        if (++it > 400)
            return OR_E_NOT_CONVERGED;
        /* Round(<e,Mf> / |f|_M^2): the ratio of two accurately evaluated
         * values, rounded half to even.  In a near-tie either neighbouring
         * integer leaves |<e',Mf>| <= (1/2 + tiny) |f|_M^2, which is all the
         * obtuse-superbase argument below needs. */
        double num = or_valS(D, e, f);
        double den = or_valS(D, f, f);
        double r = rint(num / den);
        if (!(fabs(r) < 1e15))
            return OR_E_RANGE;
        long q = (long)r;
        v2 ne = f;
        v2 nf = {e.x - q * f.x, e.y - q * f.y};
        e = ne;
        f = nf;
        if (labs(e.x) > 32767 || labs(e.y) > 32767 || labs(f.x) > 32767 || labs(f.y) > 32767)
            return OR_E_RANGE;
        /* while |e|_M > |f|_M */
        if (!(or_cmp_norm2(D, e, f) > 0))
            break;
    }
    if (iters)
        *iters = it;

    /* (ii) replace f with -f if needed so that <e, M f> <= 0. */
    if (or_sgnS(D, e, f) > 0)
        f = v2_neg(f);

    /* (iii) superbase (e0, e1, e2) = (e, f, -e-f), Eqs. def:Vz, def:GammaZ:
     * gamma(+-e_i) = -1/2 <e_{i+1}^perp, D e_{i+2}^perp>
     *             = -1/2 <e_{i+1}, adj(D) e_{i+2}>. */
    v2 sb[3];
    sb[0] = e;
    sb[1] = f;
    sb[2] = v2_neg(v2_add(e, f));
    if (labs(sb[2].x) > 32767 || labs(sb[2].y) > 32767)
        return OR_E_RANGE;

    long co[3][2];
    double cw[3];
    for (int i = 0; i < 3; i++) {
        v2 a = sb[(i + 1) % 3], b = sb[(i + 2) % 3];
        int s = or_sgnS(D, a, b);
        if (s > 0)
            return OR_E_INTERNAL; /* not obtuse: cannot happen */
        if (s == 0) {
            co[i][0] = 0;
            co[i][1] = 0;
            cw[i] = 0.0;
        } else {
            long x = sb[i].x, y = sb[i].y;
            if (x < 0 || (x == 0 && y < 0)) {
                x = -x;
                y = -y;
            }
            co[i][0] = x;
            co[i][1] = y;
            cw[i] = -0.5 * or_valS(D, a, b);
            if (!(cw[i] > 0.0))
                cw[i] = 0.0; /* only if the value underflows */
        }
    }
    /* sort the three (offset, weight) pairs */
    int idx[3] = {0, 1, 2};
    for (int i = 1; i < 3; i++)
        for (int j = i; j > 0 && or_canon_less2(co[idx[j]], co[idx[j - 1]]); j--) {
            int t = idx[j];
            idx[j] = idx[j - 1];
            idx[j - 1] = t;
        }
    for (int i = 0; i < 3; i++) {
        offs[2 * i + 0] = (int32_t)co[idx[i]][0];
        offs[2 * i + 1] = (int32_t)co[idx[i]][1];
        w[i] = cw[idx[i]];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* 3D: <u, D v>, D given as (xx, yy, zz, xy, xz, yz)                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    long c[3];
} v3;

static void or_terms3(const double D[6], v3 u, v3 v, double x[6], long n[6])
{
    const long *a = u.c, *b = v.c;
    x[0] = D[0];
    n[0] = a[0] * b[0];
    x[1] = D[1];
    n[1] = a[1] * b[1];
    x[2] = D[2];
    n[2] = a[2] * b[2];
    x[3] = D[3];
    n[3] = a[0] * b[1] + a[1] * b[0];
    x[4] = D[4];
    n[4] = a[0] * b[2] + a[2] * b[0];
    x[5] = D[5];
    n[5] = a[1] * b[2] + a[2] * b[1];
}

static int or_sgnD3(const double D[6], v3 u, v3 v)
{
    double x[6];
    long n[6];
    or_terms3(D, u, v, x, n);
    return or_sign_sum(6, x, n);
}

static double or_valD3(const double D[6], v3 u, v3 v)
{
    double x[6];
    long n[6];
    or_terms3(D, u, v, x, n);
    return or_value_sum(6, x, n);
}

static v3 v3_add(v3 a, v3 b) { v3 r = {{a.c[0] + b.c[0], a.c[1] + b.c[1], a.c[2] + b.c[2]}}; return r; }
static v3 v3_sub(v3 a, v3 b) { v3 r = {{a.c[0] - b.c[0], a.c[1] - b.c[1], a.c[2] - b.c[2]}}; return r; }
static v3 v3_neg(v3 a) { v3 r = {{-a.c[0], -a.c[1], -a.c[2]}}; return r; }
static v3 v3_scale(long k, v3 a) { v3 r = {{k * a.c[0], k * a.c[1], k * a.c[2]}}; return r; }
static v3 v3_cross(v3 a, v3 b)
{
    v3 r = {{a.c[1] * b.c[2] - a.c[2] * b.c[1], a.c[2] * b.c[0] - a.c[0] * b.c[2],
             a.c[0] * b.c[1] - a.c[1] * b.c[0]}};
    return r;
}
static int v3_big(v3 a)
{
    return labs(a.c[0]) > 32767 || labs(a.c[1]) > 32767 || labs(a.c[2]) > 32767;
}

/* sign(|u|_D^2 - |v|_D^2) */
static int or_cmp_norm3(const double D[6], v3 u, v3 v)
{
    return or_sgnD3(D, v3_sub(u, v), v3_add(u, v));
}

/* sign(|x| - |y|) for x = <a, D b>, y = <c, D d>: (|x| - |y|)(|x| + |y|) =
 * x^2 - y^2 = (x - y)(x + y), and x - y, x + y are again sums of integer
 * multiples of the entries of D. */
static int or_cmp_abs3(const double D[6], v3 a, v3 b, v3 c, v3 d)
{
    double xs[12];
    long ns[12];
    double x1[6], x2[6];
    long n1[6], n2[6];
    or_terms3(D, a, b, x1, n1);
    or_terms3(D, c, d, x2, n2);
    for (int k = 0; k < 6; k++) {
        xs[k] = x1[k];
        ns[k] = n1[k] - n2[k];
        xs[6 + k] = 0.0;
        ns[6 + k] = 0;
    }
    int sdiff = or_sign_sum(6, xs, ns);
    for (int k = 0; k < 6; k++)
        ns[k] = n1[k] + n2[k];
    int ssum = or_sign_sum(6, xs, ns);
    return sdiff * ssum;
}

static int or_check_spd3(const double D[6])
{
    for (int i = 0; i < 6; i++)
        if (!isfinite(D[i]))
            return OR_E_NONFINITE;
    /* Leading principal minors, evaluated in FP64 with a relative margin;
     * the exact construction below fails loudly on anything borderline. */
    double a = D[0], b = D[1], c = D[2], xy = D[3], xz = D[4], yz = D[5];
    if (!(a > 0.0) || !(b > 0.0) || !(c > 0.0))
        return OR_E_NOT_SPD;
    double m2 = a * b - xy * xy;
    if (!(m2 > 1e-14 * a * b))
        return OR_E_NOT_SPD;
    double det = a * (b * c - yz * yz) - xy * (xy * c - yz * xz) + xz * (xy * yz - b * xz);
    double scale = a * b * c;
    if (!(det > 1e-13 * scale))
        return OR_E_NOT_SPD;
    return OR_OK;
}

/* Lagrange's algorithm (Eq. GaussAlgo) on the pair (e, f) of 3D integer
 * vectors, for the scalar product of D.  On return |e|_D <= |f|_D and
 * (e, f) is a D-reduced basis of the 2D sub-lattice it spans. */
static int or_lagrange3(const double D[6], v3 *pe, v3 *pf)
{
    v3 e = *pe, f = *pf;
    for (int it = 0;; it++) {
        if (it > 400)
            return OR_E_NOT_CONVERGED;
        double num = or_valD3(D, e, f);
        double den = or_valD3(D, f, f);
        double r = rint(num / den);
        if (!(fabs(r) < 1e15))
            return OR_E_RANGE;
        v3 ne = f;
        v3 nf = v3_sub(e, v3_scale((long)r, f));
        e = ne;
        f = nf;
        if (v3_big(e) || v3_big(f))
            return OR_E_RANGE;
        if (!(or_cmp_norm3(D, e, f) > 0))
            break;
    }
    *pe = e;
    *pf = f;
    return OR_OK;
}

/* Greedy reduction (Nguyen-Stehle) for d = 3: keep the basis sorted by
 * D-norm, Lagrange-reduce the two shortest vectors, subtract from the third
 * its closest vector in their lattice, and repeat until the third vector is
 * no shorter than the second.  The output is a D-reduced basis in the sense
 * of Def. ReducedBasis (Minkowski reduction, d <= 4). */
static int or_greedy3(const double D[6], v3 b[3], int *iters)
{
    for (int it = 0;; it++) {
        if (it > 200)
            return OR_E_NOT_CONVERGED;
        /* sort by D-norm (insertion sort, exact comparisons) */
        for (int i = 1; i < 3; i++)
            for (int j = i; j > 0 && or_cmp_norm3(D, b[j], b[j - 1]) < 0; j--) {
                v3 t = b[j];
                b[j] = b[j - 1];
                b[j - 1] = t;
            }
        /* reduce (b0, b1), starting from (longer, shorter) */
        v3 e = b[1], f = b[0];
        int st = or_lagrange3(D, &e, &f);
        if (st != OR_OK)
            return st;
        b[0] = e;
        b[1] = f;
        /* closest vector to b2 in b0 Z + b1 Z: real coordinates of the
         * D-orthogonal projection, then an exact search over the integer
         * points within distance 1 of them (for a reduced pair the closest
         * vector's coordinates differ from the real ones by at most 1). */
        double g00 = or_valD3(D, b[0], b[0]), g01 = or_valD3(D, b[0], b[1]);
        double g11 = or_valD3(D, b[1], b[1]);
        double r0 = or_valD3(D, b[0], b[2]), r1 = or_valD3(D, b[1], b[2]);
        double det = g00 * g11 - g01 * g01;
        double y0 = (g11 * r0 - g01 * r1) / det;
        double y1 = (g00 * r1 - g01 * r0) / det;
        if (!(fabs(y0) < 1e12) || !(fabs(y1) < 1e12))
            return OR_E_RANGE;
        long f0 = (long)floor(y0), f1 = (long)floor(y1);
        v3 best = {{0, 0, 0}};
        int have = 0;
        for (long k0 = f0 - 1; k0 <= f0 + 2; k0++)
            for (long k1 = f1 - 1; k1 <= f1 + 2; k1++) {
                v3 c = v3_add(v3_scale(k0, b[0]), v3_scale(k1, b[1]));
                if (!have) {
                    best = c;
                    have = 1;
                    continue;
                }
                /* |t - c|^2 < |t - best|^2  <=>  <best - c, D (2t - c - best)> < 0 */
                v3 two_t = v3_add(b[2], b[2]);
                v3 w = v3_sub(v3_sub(two_t, c), best);
                if (or_sgnD3(D, v3_sub(best, c), w) < 0)
                    best = c;
            }
        b[2] = v3_sub(b[2], best);
        if (v3_big(b[2]))
            return OR_E_RANGE;
        if (or_cmp_norm3(D, b[2], b[1]) >= 0) {
            if (iters)
                *iters = it + 1;
            return OR_OK;
        }
    }
}

static int or_canon_less3(const long *a, const long *b)
{
    for (int k = 0; k < 3; k++)
        if (a[k] != b[k])
            return a[k] < b[k];
    return 0;
}

/* One point of the 3D construction (Sec. 2).  offs[6][3], w[6]. */
static int or_stencil3(const double D[6], int32_t *offs, double *w, int *iters)
{
    int st = or_check_spd3(D);
    if (st != OR_OK)
        return st;
    v3 b[3] = {{{1, 0, 0}}, {{0, 1, 0}}, {{0, 0, 1}}};
    st = or_greedy3(D, b, iters);
    if (st != OR_OK)
        return st;

    /* Prop. MakeObtuse: permutation sigma with
     * |<b'1,Db'2>| <= |<b'1,Db'3>| <= |<b'2,Db'3>|, enumerated in a fixed
     * order, the first that satisfies both inequalities is taken. */
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int p = -1;
    for (int k = 0; k < 6 && p < 0; k++) {
        v3 x1 = b[perms[k][0]], x2 = b[perms[k][1]], x3 = b[perms[k][2]];
        if (or_cmp_abs3(D, x1, x2, x1, x3) <= 0 && or_cmp_abs3(D, x1, x3, x2, x3) <= 0)
            p = k;
    }
    if (p < 0)
        return OR_E_INTERNAL;
    v3 b1 = b[perms[p][0]], b2 = b[perms[p][1]], b3 = b[perms[p][2]];
    /* signs: <b1, D b3> <= 0 and <b2, D b3> <= 0 */
    if (or_sgnD3(D, b1, b3) > 0)
        b1 = v3_neg(b1);
    if (or_sgnD3(D, b2, b3) > 0)
        b2 = v3_neg(b2);
    /* Eq. 3DSuperBase */
    v3 e[4];
    if (or_sgnD3(D, b1, b2) <= 0) {
        e[1] = b1;
        e[2] = b2;
        e[3] = b3;
        e[0] = v3_neg(v3_add(v3_add(b1, b2), b3));
    } else {
        e[1] = v3_neg(b1);
        e[2] = b2;
        e[3] = v3_add(b1, b3);
        e[0] = v3_neg(v3_add(b2, b3));
    }
    for (int i = 0; i < 4; i++)
        if (v3_big(e[i]))
            return OR_E_RANGE;

    /* Selling (Lemma Selling, Eq. DSum3D): for {i,j,k,l} = {0,1,2,3}, i < j,
     * k < l: offset c_ij = e_k x e_l, weight -<e_i, D e_j>/2. */
    static const int pairs[6][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2},
                                    {1, 2, 0, 3}, {1, 3, 0, 2}, {2, 3, 0, 1}};
    long co[6][3];
    double cw[6];
    for (int q = 0; q < 6; q++) {
        v3 ei = e[pairs[q][0]], ej = e[pairs[q][1]];
        int s = or_sgnD3(D, ei, ej);
        if (s > 0)
            return OR_E_INTERNAL; /* not D-obtuse: cannot happen */
        if (s == 0) {
            co[q][0] = co[q][1] = co[q][2] = 0;
            cw[q] = 0.0;
            continue;
        }
        v3 c = v3_cross(e[pairs[q][2]], e[pairs[q][3]]);
        if (v3_big(c))
            return OR_E_RANGE;
        int flip = 0;
        for (int k = 0; k < 3; k++)
            if (c.c[k] != 0) {
                flip = c.c[k] < 0;
                break;
            }
        if (flip)
            c = v3_neg(c);
        for (int k = 0; k < 3; k++)
            co[q][k] = c.c[k];
        cw[q] = -0.5 * or_valD3(D, ei, ej);
        if (!(cw[q] > 0.0))
            cw[q] = 0.0;
    }
    int idx[6] = {0, 1, 2, 3, 4, 5};
    for (int i = 1; i < 6; i++)
        for (int j = i; j > 0 && or_canon_less3(co[idx[j]], co[idx[j - 1]]); j--) {
            int t = idx[j];
            idx[j] = idx[j - 1];
            idx[j - 1] = t;
        }
    for (int i = 0; i < 6; i++) {
        for (int k = 0; k < 3; k++)
            offs[3 * i + k] = (int32_t)co[idx[i]][k];
        w[i] = cw[idx[i]];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Batch entry points                                                         */
/* ------------------------------------------------------------------------- */

/* D: 3 planes (xx, xy, yy) of n doubles.  offs: n*3*2 int32, w: n*3.
 * status: n ints (per-point status, may be NULL).  Returns the first
 * non-zero per-point status, or 0. */
int or_build2d(int64_t n, const double *Dxx, const double *Dxy, const double *Dyy,
               int32_t *offs, double *w, int32_t *status, int32_t *iters)
{
    int first = OR_OK;
    for (int64_t i = 0; i < n; i++) {
        double D[3] = {Dxx[i], Dxy[i], Dyy[i]};
        int it = 0;
        int st = or_stencil2(D, offs + 6 * i, w + 3 * i, &it);
        if (st != OR_OK) {
            memset(offs + 6 * i, 0, 6 * sizeof(int32_t));
            w[3 * i] = w[3 * i + 1] = w[3 * i + 2] = 0.0;
            if (first == OR_OK)
                first = st;
        }
        if (status)
            status[i] = st;
        if (iters)
            iters[i] = it;
    }
    return first;
}

/* D: 6 planes (xx, yy, zz, xy, xz, yz) of n doubles, plane-major.
 * offs: n*6*3 int32, w: n*6. */
int or_build3d(int64_t n, const double *D6, int32_t *offs, double *w, int32_t *status,
               int32_t *iters)
{
    int first = OR_OK;
    for (int64_t i = 0; i < n; i++) {
        double D[6];
        for (int k = 0; k < 6; k++)
            D[k] = D6[(int64_t)k * n + i];
        int it = 0;
        int st = or_stencil3(D, offs + 18 * i, w + 6 * i, &it);
        if (st != OR_OK) {
            memset(offs + 18 * i, 0, 18 * sizeof(int32_t));
            for (int k = 0; k < 6; k++)
                w[6 * i + k] = 0.0;
            if (first == OR_OK)
                first = st;
        }
        if (status)
            status[i] = st;
        if (iters)
            iters[i] = it;
    }
    return first;
}

/* ------------------------------------------------------------------------- */
/* Operator A = (1/2) grad E_h, Eq. def:E* with h = 1                        */
/* ------------------------------------------------------------------------- */

/* Neighbour index of point (x, y, z) + s*o, or -1 if it leaves the grid and
 * the boundary is Neumann (pair dropped, Sec. 1).  bc: 0 Neumann, 1 periodic. */
static int64_t or_neighbour(int dim, const int64_t *nn, int bc, const int64_t *p, const int32_t *o,
                            int s)
{
    int64_t q[3] = {0, 0, 0};
    for (int k = 0; k < dim; k++) {
        int64_t c = p[k] + (int64_t)s * o[k];
        if (bc == 1) {
            c %= nn[k];
            if (c < 0)
                c += nn[k];
        } else if (c < 0 || c >= nn[k]) {
            return -1;
        }
        q[k] = c;
    }
    if (dim == 2)
        return q[0] + nn[0] * q[1];
    return q[0] + nn[0] * (q[1] + nn[1] * q[2]);
}

/* E_h(u) = sum_z sum_{e in V(z)} gamma_z(e) |u(z+e) - u(z)|^2, V(z) symmetric.
 * Each (z, e) term contributes gamma (u(z) - u(z+e)) to (1/2) dE/du(z) and the
 * opposite to (1/2) dE/du(z+e).  offs: [N][K][dim], w: [N][K], K half-stencil
 * offsets per point, both signs taken. */
int or_apply(int dim, const int64_t *nn, int bc, int K, const int32_t *offs, const double *w,
             const double *u, double *Au)
{
    int64_t N = nn[0] * nn[1] * (dim == 3 ? nn[2] : 1);
    memset(Au, 0, (size_t)N * sizeof(double));
    int64_t p[3];
    for (int64_t z = 0; z < N; z++) {
        p[0] = z % nn[0];
        p[1] = (z / nn[0]) % nn[1];
        p[2] = dim == 3 ? z / (nn[0] * nn[1]) : 0;
        for (int k = 0; k < K; k++) {
            double g = w[z * K + k];
            const int32_t *o = offs + (z * K + k) * dim;
            for (int s = -1; s <= 1; s += 2) {
                int64_t y = or_neighbour(dim, nn, bc, p, o, s);
                if (y < 0)
                    continue;
                double flux = g * (u[z] - u[y]);
                Au[z] += flux;
                Au[y] -= flux;
            }
        }
    }
    return OR_OK;
}

/* Diagonal of A: A_zz = sum of the weights of the in-grid pairs touching z. */
int or_diag(int dim, const int64_t *nn, int bc, int K, const int32_t *offs, const double *w,
            double *diag)
{
    int64_t N = nn[0] * nn[1] * (dim == 3 ? nn[2] : 1);
    memset(diag, 0, (size_t)N * sizeof(double));
    int64_t p[3];
    for (int64_t z = 0; z < N; z++) {
        p[0] = z % nn[0];
        p[1] = (z / nn[0]) % nn[1];
        p[2] = dim == 3 ? z / (nn[0] * nn[1]) : 0;
        for (int k = 0; k < K; k++) {
            double g = w[z * K + k];
            const int32_t *o = offs + (z * K + k) * dim;
            for (int s = -1; s <= 1; s += 2) {
                int64_t y = or_neighbour(dim, nn, bc, p, o, s);
                if (y < 0 || y == z)
                    continue;
                diag[z] += g;
                diag[y] += g;
            }
        }
    }
    return OR_OK;
}

/* E_h(u) itself (for the tests that rebuild A from the energy). */
double or_energy(int dim, const int64_t *nn, int bc, int K, const int32_t *offs, const double *w,
                 const double *u)
{
    int64_t N = nn[0] * nn[1] * (dim == 3 ? nn[2] : 1);
    int64_t p[3];
    double E = 0.0;
    for (int64_t z = 0; z < N; z++) {
        p[0] = z % nn[0];
        p[1] = (z / nn[0]) % nn[1];
        p[2] = dim == 3 ? z / (nn[0] * nn[1]) : 0;
        for (int k = 0; k < K; k++) {
            double g = w[z * K + k];
            const int32_t *o = offs + (z * K + k) * dim;
            for (int s = -1; s <= 1; s += 2) {
                int64_t y = or_neighbour(dim, nn, bc, p, o, s);
                if (y < 0)
                    continue;
                double d = u[y] - u[z];
                E += g * d * d;
            }
        }
    }
    return E;
}

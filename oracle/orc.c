/*
 * FP64 CPU oracle for lattice spline evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load this file or
 * the library built from it; only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py do.  It shares no code with the CUDA path.
 *
 * What it computes (Horacsek & Alim, "Automatic Generation of Interpolants for
 * Lattice Samplings, Part II", Eq. 1, Sec. 1):
 *
 *     f(x) = sum_{n in L Z^s} c_n phi(x - n)
 *
 * evaluated NAIVELY, exactly as Eq. 1 is written: every stored lattice site n
 * whose basis function support contains x contributes c_n * phi(x - n).  No
 * region of evaluation, no sub-regions, no symmetry, no unrolling.  Sites that
 * are not stored contribute nothing (zero extension beyond the coefficient
 * arrays; the paper does not discuss boundaries).
 *
 * The basis functions are the box splines the paper benchmarks (Sec. 5.1) and
 * its worked example (Fig. 1, the ZP element).  A box spline with direction
 * matrix Xi (s x m, spanning R^s) is the function M_Xi defined by
 *
 *     integral M_Xi(x) g(x) dx = integral_{[0,1)^m} g(Xi t) dt   for all g.
 *
 * The paper takes it from its references and does not restate it.  The basis
 * function is the centred, lattice-normalised box spline
 *
 *     phi(x) = |det L| * M_Xi(x + Xi * (1/2, ..., 1/2)),
 *
 * centred on the origin like the region of evaluation of Fig. 1 and scaled so
 * that sum_n phi(x - n) = 1 (the constant terms of Fig. 1 sum to one).
 *
 * M_Xi is evaluated by the de Boor-Hoellig recurrence with two rules for
 * degenerate direction sets (repeated and coplanar directions):
 *   R1  Xi does not span R^k                  -> 0
 *   R2  |Xi| = k                              -> 1[0 <= Xi^-1 x < 1] / |det Xi|
 *   R3  some xi is essential (Xi\xi spans only a hyperplane H): with U a basis
 *       of H taken from Xi\xi and [U xi](y, tau) = x,
 *           M_Xi(x) = M^{(k-1)}_{U^-1 (Xi\xi)}(y) * 1[0 <= tau < 1] / |det [U xi]|
 *   R4  otherwise, with x = Xi t (t = B^-1 x on a basis B, zero elsewhere),
 *           (|Xi| - k) M_Xi(x) = sum_xi [ t_xi M_{Xi\xi}(x) + (1 - t_xi) M_{Xi\xi}(x - xi) ]
 * The recurrence over the top-level direction multiset is memoised on the
 * state (copies left, copies shifted) of each distinct direction.  The tensor
 * product cubic B-spline (the tricubic of Sec. 5.1) is also provided in closed
 * form, phi(x) = prod_i beta3(x_i).
 *
 * Gradients use the box spline derivative identity
 *     D_xi M_Xi(x) = M_{Xi\xi}(x) - M_{Xi\xi}(x - xi)
 * along s independent directions whose removal keeps Xi spanning.  Applied
 * twice it gives, for two columns i != j of Xi (possibly equal directions),
 *     D_xi_i D_xi_j M_Xi(x) = sum_{a,b in {0,1}} (-1)^(a+b) M_{Xi\{i,j}}(x - a xi_i - b xi_j),
 * which is 0 off the knot planes when Xi\{i,j} does not span (rule R1); the
 * Hessian H is the symmetric matrix with xi_i^T H xi_j equal to these values
 * for every pair, solved by least squares over all pairs.
 *
 * Everything is plain FP64 with round-to-nearest; no fast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXDIR 16   /* columns of Xi */
#define ORC_MAXCOSET 8

typedef struct {
    int32_t dim;                    /* s: 1, 2 or 3 */
    int32_t kind;                   /* 0: box spline from dirs; 1: closed-form tensor cubic B-spline */
    int32_t ndir;                   /* m = |Xi| */
    int32_t pad0;
    double  dirs[ORC_MAXDIR * 3];   /* column j of Xi at dirs[3*j .. 3*j+dim-1] */
    double  detL;                   /* |det L|, lattice density normalisation */
    int32_t scale;                  /* storage grid spacing a: site = a*i + l_j */
    int32_t ncoset;                 /* number of Cartesian cosets l_j */
    int32_t coset[ORC_MAXCOSET * 3];/* l_j at coset[3*j ..] */
    int64_t ext[3];                 /* extent of every coset array, axis 0 fastest */
} orc_spec;

/* ------------------------------------------------------------------------- */
/* small dense linear algebra (k <= 3)                                         */
/* ------------------------------------------------------------------------- */

/* Solve A z = b for a k x k matrix given by columns cols[j][i].  Returns the
 * determinant (0 if singular).  Gaussian elimination with partial pivoting. */
static double solve_cols(int k, const double cols[][3], const double *b, double *z)
{
    double a[3][4];
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) a[i][j] = cols[j][i];
        a[i][k] = b ? b[i] : 0.0;
    }
    double det = 1.0;
    for (int c = 0; c < k; ++c) {
        int p = c;
        for (int r = c + 1; r < k; ++r)
            if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
        if (fabs(a[p][c]) < 1e-12) return 0.0;
        if (p != c) {
            for (int j = 0; j <= k; ++j) { double t = a[c][j]; a[c][j] = a[p][j]; a[p][j] = t; }
            det = -det;
        }
        det *= a[c][c];
        for (int r = c + 1; r < k; ++r) {
            double f = a[r][c] / a[c][c];
            for (int j = c; j <= k; ++j) a[r][j] -= f * a[c][j];
        }
    }
    if (z) {
        for (int r = k - 1; r >= 0; --r) {
            double s = a[r][k];
            for (int j = r + 1; j < k; ++j) s -= a[r][j] * z[j];
            z[r] = s / a[r][r];
        }
    }
    return det;
}

/* Rank of a set of m vectors in R^k. */
static int rank_of(int k, int m, const double cols[][3])
{
    double a[ORC_MAXDIR][3];
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < k; ++i) a[j][i] = cols[j][i];
    int rank = 0;
    for (int c = 0; c < k && rank < m; ++c) {
        int p = -1;
        double best = 1e-9;
        for (int r = rank; r < m; ++r)
            if (fabs(a[r][c]) > best) { best = fabs(a[r][c]); p = r; }
        if (p < 0) continue;
        for (int i = 0; i < k; ++i) { double t = a[rank][i]; a[rank][i] = a[p][i]; a[p][i] = t; }
        for (int r = 0; r < m; ++r) {
            if (r == rank) continue;
            double f = a[r][c] / a[rank][c];
            for (int i = 0; i < k; ++i) a[r][i] -= f * a[rank][i];
        }
        ++rank;
    }
    return rank;
}

/* Pick k linearly independent columns (greedy, in order).  Returns 1 on success. */
static int pick_basis(int k, int m, const double cols[][3], int *idx)
{
    double sel[3][3];
    int n = 0;
    for (int j = 0; j < m && n < k; ++j) {
        for (int i = 0; i < k; ++i) sel[n][i] = cols[j][i];
        if (rank_of(k, n + 1, sel) == n + 1) idx[n++] = j;
    }
    return n == k;
}

/* ------------------------------------------------------------------------- */
/* generic recurrence (no memo), used below the top level after rule R3        */
/* ------------------------------------------------------------------------- */

static double box_generic(int k, int m, const double cols[][3], const double *x);

/* Rule R3 for column `e` of cols (essential).  */
static double box_factor(int k, int m, const double cols[][3], int e, const double *x)
{
    double rest[ORC_MAXDIR][3];
    int mr = 0;
    for (int j = 0; j < m; ++j)
        if (j != e) { for (int i = 0; i < 3; ++i) rest[mr][i] = cols[j][i]; ++mr; }
    double uc[3][3];
    int nu = 0;
    {   /* k-1 independent columns of rest */
        double sel[3][3];
        for (int j = 0; j < mr && nu < k - 1; ++j) {
            for (int i = 0; i < k; ++i) sel[nu][i] = rest[j][i];
            if (rank_of(k, nu + 1, sel) == nu + 1) {
                for (int i = 0; i < 3; ++i) uc[nu][i] = rest[j][i];
                ++nu;
            }
        }
    }
    if (nu != k - 1) return 0.0;
    for (int i = 0; i < 3; ++i) uc[k - 1][i] = cols[e][i];
    double z[3];
    double det = solve_cols(k, uc, x, z);
    if (det == 0.0) return 0.0;
    double tau = z[k - 1];
    if (!(tau >= 0.0 && tau < 1.0)) return 0.0;
    /* coordinates of the remaining directions in the basis U of H */
    double proj[ORC_MAXDIR][3];
    for (int j = 0; j < mr; ++j) {
        double w[3];
        solve_cols(k, uc, rest[j], w);
        for (int i = 0; i < k - 1; ++i) proj[j][i] = w[i];
        for (int i = k - 1; i < 3; ++i) proj[j][i] = 0.0;
    }
    double y[3] = {0, 0, 0};
    for (int i = 0; i < k - 1; ++i) y[i] = z[i];
    if (k - 1 == 0) return (mr == 0 ? 1.0 : 0.0) / fabs(det);
    return box_generic(k - 1, mr, proj, y) / fabs(det);
}

static double box_generic(int k, int m, const double cols[][3], const double *x)
{
    if (m < k || rank_of(k, m, cols) < k) return 0.0;                    /* R1 */
    if (m == k) {                                                         /* R2 */
        double t[3];
        double det = solve_cols(k, cols, x, t);
        if (det == 0.0) return 0.0;
        for (int i = 0; i < k; ++i)
            if (!(t[i] >= 0.0 && t[i] < 1.0)) return 0.0;
        return 1.0 / fabs(det);
    }
    double rest[ORC_MAXDIR][3];
    for (int e = 0; e < m; ++e) {                                         /* R3 */
        int mr = 0;
        for (int j = 0; j < m; ++j)
            if (j != e) { for (int i = 0; i < 3; ++i) rest[mr][i] = cols[j][i]; ++mr; }
        if (rank_of(k, mr, rest) < k) return box_factor(k, m, cols, e, x);
    }
    int b[3];                                                             /* R4 */
    pick_basis(k, m, cols, b);
    double bc[3][3], tb[3];
    for (int n = 0; n < k; ++n)
        for (int i = 0; i < 3; ++i) bc[n][i] = cols[b[n]][i];
    solve_cols(k, bc, x, tb);
    double sum = 0.0;
    for (int e = 0; e < m; ++e) {
        double te = 0.0;
        for (int n = 0; n < k; ++n)
            if (b[n] == e) te = tb[n];
        int mr = 0;
        for (int j = 0; j < m; ++j)
            if (j != e) { for (int i = 0; i < 3; ++i) rest[mr][i] = cols[j][i]; ++mr; }
        double xs[3];
        for (int i = 0; i < 3; ++i) xs[i] = x[i] - (i < k ? cols[e][i] : 0.0);
        double a0 = (te != 0.0) ? box_generic(k, mr, rest, x) : 0.0;
        double a1 = (te != 1.0) ? box_generic(k, mr, rest, xs) : 0.0;
        sum += te * a0 + (1.0 - te) * a1;
    }
    return sum / (double)(m - k);
}

/* ------------------------------------------------------------------------- */
/* memoised recurrence over the top-level multiset                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    int k;
    int D;                         /* distinct directions */
    double dir[ORC_MAXDIR][3];
    int mult[ORC_MAXDIR];
    int stride[ORC_MAXDIR];
    int nstate;
    double x0[3];
    double *val;
    uint32_t *stamp;
    uint32_t cur;
} box_memo;

static int memo_init(box_memo *c, int k, int m, const double *cols)
{
    memset(c, 0, sizeof(*c));
    c->k = k;
    for (int j = 0; j < m; ++j) {
        int found = -1;
        for (int d = 0; d < c->D; ++d) {
            int same = 1;
            for (int i = 0; i < k; ++i)
                if (c->dir[d][i] != cols[3 * j + i]) same = 0;
            if (same) { found = d; break; }
        }
        if (found >= 0) { c->mult[found]++; continue; }
        for (int i = 0; i < 3; ++i) c->dir[c->D][i] = (i < k) ? cols[3 * j + i] : 0.0;
        c->mult[c->D] = 1;
        c->D++;
    }
    long n = 1;
    for (int d = 0; d < c->D; ++d) {
        c->stride[d] = (int)n;
        n *= (long)(c->mult[d] + 1) * (c->mult[d] + 1);
        if (n > (1L << 22)) return -1;
    }
    c->nstate = (int)n;
    c->val = (double *)malloc(sizeof(double) * n);
    c->stamp = (uint32_t *)calloc(n, sizeof(uint32_t));
    c->cur = 0;
    return (c->val && c->stamp) ? 0 : -1;
}

static void memo_free(box_memo *c)
{
    free(c->val);
    free(c->stamp);
    c->val = NULL;
    c->stamp = NULL;
}

/* r[d]: copies of direction d still in the set; s[d]: copies removed with a shift. */
static double memo_state(box_memo *c, int *r, int *s)
{
    const int k = c->k;
    int index = 0;
    for (int d = 0; d < c->D; ++d) index += (r[d] * (c->mult[d] + 1) + s[d]) * c->stride[d];
    if (c->stamp[index] == c->cur) return c->val[index];

    double x[3];
    for (int i = 0; i < 3; ++i) {
        x[i] = c->x0[i];
        for (int d = 0; d < c->D; ++d) x[i] -= s[d] * c->dir[d][i];
    }
    double cols[ORC_MAXDIR][3];
    int m = 0;
    for (int d = 0; d < c->D; ++d)
        for (int q = 0; q < r[d]; ++q) { for (int i = 0; i < 3; ++i) cols[m][i] = c->dir[d][i]; ++m; }

    double res;
    if (m < k || rank_of(k, m, cols) < k) {
        res = 0.0;                                                        /* R1 */
    } else if (m == k) {
        res = box_generic(k, m, cols, x);                                 /* R2 */
    } else {
        int essential = -1;                                               /* R3 */
        for (int d = 0; d < c->D && essential < 0; ++d) {
            if (r[d] != 1) continue;
            double rest[ORC_MAXDIR][3];
            int mr = 0;
            for (int e = 0; e < c->D; ++e)
                for (int q = 0; q < r[e] - (e == d); ++q) {
                    for (int i = 0; i < 3; ++i) rest[mr][i] = c->dir[e][i];
                    ++mr;
                }
            if (rank_of(k, mr, rest) < k) essential = d;
        }
        if (essential >= 0) {
            int e = 0;
            for (int d = 0; d < essential; ++d) e += r[d];
            res = box_factor(k, m, cols, e, x);
        } else {                                                          /* R4 */
            /* basis from distinct directions, one copy each */
            double dcols[ORC_MAXDIR][3];
            int dmap[ORC_MAXDIR], nd = 0;
            for (int d = 0; d < c->D; ++d)
                if (r[d] > 0) {
                    for (int i = 0; i < 3; ++i) dcols[nd][i] = c->dir[d][i];
                    dmap[nd++] = d;
                }
            int b[3];
            pick_basis(k, nd, dcols, b);
            double bc[3][3], tb[3];
            for (int n = 0; n < k; ++n)
                for (int i = 0; i < 3; ++i) bc[n][i] = dcols[b[n]][i];
            solve_cols(k, bc, x, tb);
            double sum = 0.0;
            for (int n = 0; n < nd; ++n) {
                int d = dmap[n];
                /* sum of t over the r[d] copies of direction d */
                double T = 0.0;
                for (int q = 0; q < k; ++q)
                    if (b[q] == n) T = tb[q];
                r[d]--;
                double a0 = memo_state(c, r, s);
                s[d]++;
                double a1 = memo_state(c, r, s);
                s[d]--;
                r[d]++;
                sum += T * a0 + ((double)r[d] - T) * a1;
            }
            res = sum / (double)(m - k);
        }
    }
    c->stamp[index] = c->cur;
    c->val[index] = res;
    return res;
}

static double memo_eval(box_memo *c, const double *x)
{
    int r[ORC_MAXDIR], s[ORC_MAXDIR];
    for (int d = 0; d < c->D; ++d) { r[d] = c->mult[d]; s[d] = 0; }
    for (int i = 0; i < 3; ++i) c->x0[i] = (i < c->k) ? x[i] : 0.0;
    c->cur++;
    if (c->cur == 0) { memset(c->stamp, 0, sizeof(uint32_t) * c->nstate); c->cur = 1; }
    return memo_state(c, r, s);
}

/* ------------------------------------------------------------------------- */
/* the centred basis function and its support                                  */
/* ------------------------------------------------------------------------- */

/* centred cubic B-spline, beta3(t) = (M_{1,1,1,1} shifted by 2) */
static double beta3(double t)
{
    double a = fabs(t);
    if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    if (a < 2.0) { double u = 2.0 - a; return u * u * u / 6.0; }
    return 0.0;
}

static double d2beta3(double t)
{
    double a = fabs(t);
    if (a < 1.0) return -2.0 + 3.0 * a;
    if (a < 2.0) return 2.0 - a;
    return 0.0;
}

static double dbeta3(double t)
{
    double a = fabs(t), sg = (t < 0.0) ? -1.0 : 1.0;
    if (a < 1.0) return -2.0 * t + 1.5 * t * a;
    if (a < 2.0) { double u = 2.0 - a; return -0.5 * sg * u * u; }
    return 0.0;
}

typedef struct {
    const orc_spec *sp;
    box_memo full;                 /* M_Xi */
    box_memo part[3];              /* M_{Xi \ xi_b} for the gradient basis */
    int gbasis[3];                 /* column indices used for the gradient */
    double gbinv[3][3];            /* (B^T)^{-1} */
    double half[3];                /* Xi * 1/2 */
    int nfacet;
    double facet[64][3];           /* support facet normals */
    double fbound[64];             /* support half-widths along the normals */
    int noff[64];                  /* knot plane offsets per normal */
    double *off[64];               /* nu . (sum of a subset of Xi), sorted */
    int ready_grad;
} phi_ctx;

/* Normals of the support zonotope: vectors orthogonal to k-1 independent columns. */
static void support_facets(phi_ctx *p)
{
    const orc_spec *sp = p->sp;
    const int k = sp->dim, m = sp->ndir;
    p->nfacet = 0;
    if (k == 1) {
        p->facet[0][0] = 1.0; p->facet[0][1] = 0.0; p->facet[0][2] = 0.0;
        p->nfacet = 1;
    } else {
        for (int a = 0; a < m; ++a)
            for (int b = (k == 2 ? a : a + 1); b < m; ++b) {
                const double *u = sp->dirs + 3 * a, *v = sp->dirs + 3 * b;
                double nrm[3];
                if (k == 2) { nrm[0] = -u[1]; nrm[1] = u[0]; nrm[2] = 0.0; }
                else {
                    nrm[0] = u[1] * v[2] - u[2] * v[1];
                    nrm[1] = u[2] * v[0] - u[0] * v[2];
                    nrm[2] = u[0] * v[1] - u[1] * v[0];
                }
                double len = fabs(nrm[0]) + fabs(nrm[1]) + fabs(nrm[2]);
                if (len < 1e-12) continue;
                int dup = 0;
                for (int f = 0; f < p->nfacet && !dup; ++f) {
                    double cx = p->facet[f][1] * nrm[2] - p->facet[f][2] * nrm[1];
                    double cy = p->facet[f][2] * nrm[0] - p->facet[f][0] * nrm[2];
                    double cz = p->facet[f][0] * nrm[1] - p->facet[f][1] * nrm[0];
                    if (fabs(cx) + fabs(cy) + fabs(cz) < 1e-12) dup = 1;
                }
                if (!dup && p->nfacet < 64) {
                    for (int i = 0; i < 3; ++i) p->facet[p->nfacet][i] = nrm[i];
                    p->nfacet++;
                }
            }
    }
    for (int f = 0; f < p->nfacet; ++f) {
        double b = 0.0;
        for (int j = 0; j < m; ++j) {
            double d = 0.0;
            for (int i = 0; i < k; ++i) d += p->facet[f][i] * sp->dirs[3 * j + i];
            b += fabs(d);
        }
        p->fbound[f] = 0.5 * b;
    }
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Knot planes of M_Xi: nu . x = nu . (sum over a subset S of Xi), for every
 * normal nu orthogonal to s-1 independent columns.  M_Xi is a polynomial on
 * each cell of this arrangement. */
static int knot_planes(phi_ctx *p)
{
    const orc_spec *sp = p->sp;
    const int k = sp->dim, m = sp->ndir;
    for (int f = 0; f < p->nfacet; ++f) {
        double dots[ORC_MAXDIR];
        for (int j = 0; j < m; ++j) {
            dots[j] = 0.0;
            for (int i = 0; i < k; ++i) dots[j] += p->facet[f][i] * sp->dirs[3 * j + i];
        }
        long nsub = 1L << m;
        double *v = (double *)malloc(sizeof(double) * nsub);
        if (!v) return -1;
        for (long S = 0; S < nsub; ++S) {
            double s = 0.0;
            for (int j = 0; j < m; ++j)
                if (S & (1L << j)) s += dots[j];
            v[S] = s;
        }
        qsort(v, nsub, sizeof(double), cmp_double);
        int n = 0;
        for (long S = 0; S < nsub; ++S)
            if (n == 0 || v[S] - v[n - 1] > 1e-12) v[n++] = v[S];
        p->off[f] = v;
        p->noff[f] = n;
    }
    return 0;
}

/* Is x within tol of a knot plane? */
static int on_knot_plane(const phi_ctx *p, const double *x)
{
    const int k = p->sp->dim;
    for (int f = 0; f < p->nfacet; ++f) {
        double d = 0.0, len = 0.0;
        for (int i = 0; i < k; ++i) { d += p->facet[f][i] * x[i]; len += fabs(p->facet[f][i]); }
        for (int o = 0; o < p->noff[f]; ++o)
            if (fabs(d - p->off[f][o]) <= 1e-10 * len) return 1;
    }
    return 0;
}

static int phi_init(phi_ctx *p, const orc_spec *sp, int want_grad)
{
    memset(p, 0, sizeof(*p));
    p->sp = sp;
    if (sp->kind == 1) return 0;
    const int k = sp->dim, m = sp->ndir;
    for (int i = 0; i < 3; ++i) {
        p->half[i] = 0.0;
        for (int j = 0; j < m; ++j) p->half[i] += (i < k) ? 0.5 * sp->dirs[3 * j + i] : 0.0;
    }
    if (memo_init(&p->full, k, m, sp->dirs)) return -1;
    support_facets(p);
    if (knot_planes(p)) return -1;
    if (want_grad) {
        /* gradient basis: k independent columns whose removal keeps Xi spanning */
        double cols[ORC_MAXDIR][3];
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < 3; ++i) cols[j][i] = sp->dirs[3 * j + i];
        double sel[3][3];
        int n = 0;
        for (int j = 0; j < m && n < k; ++j) {
            double rest[ORC_MAXDIR][3];
            int mr = 0;
            for (int q = 0; q < m; ++q)
                if (q != j) { for (int i = 0; i < 3; ++i) rest[mr][i] = cols[q][i]; ++mr; }
            if (rank_of(k, mr, rest) < k) continue;
            for (int i = 0; i < 3; ++i) sel[n][i] = cols[j][i];
            if (rank_of(k, n + 1, sel) != n + 1) continue;
            p->gbasis[n] = j;
            double restflat[ORC_MAXDIR * 3];
            for (int q = 0; q < mr; ++q)
                for (int i = 0; i < 3; ++i) restflat[3 * q + i] = rest[q][i];
            if (memo_init(&p->part[n], k, mr, restflat)) return -1;
            ++n;
        }
        if (n != k) return -2;
        /* rows of B^T are the basis columns; invert B^T */
        double bt[3][3];   /* columns of B^T = rows of B */
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b) bt[a][b] = sel[b][a];
        for (int e = 0; e < k; ++e) {
            double rhs[3] = {0, 0, 0}, z[3];
            rhs[e] = 1.0;
            solve_cols(k, bt, rhs, z);
            for (int i = 0; i < k; ++i) p->gbinv[i][e] = z[i];
        }
        p->ready_grad = 1;
    }
    return 0;
}

static void phi_free(phi_ctx *p)
{
    if (p->sp->kind == 1) return;
    for (int f = 0; f < p->nfacet; ++f) free(p->off[f]);
    memo_free(&p->full);
    if (p->ready_grad)
        for (int n = 0; n < p->sp->dim; ++n) memo_free(&p->part[n]);
}

static int outside_support(const phi_ctx *p, const double *y)
{
    const int k = p->sp->dim;
    for (int f = 0; f < p->nfacet; ++f) {
        double d = 0.0;
        for (int i = 0; i < k; ++i) d += p->facet[f][i] * y[i];
        if (fabs(d) >= p->fbound[f]) return 1;
    }
    return 0;
}

static double phi_generic(phi_ctx *p, const double *y, double *g);

/* phi(y) and, if g != NULL, grad phi(y) */
static double phi_eval(phi_ctx *p, const double *y, double *g)
{
    const orc_spec *sp = p->sp;
    const int k = sp->dim;
    if (sp->kind == 1) {
        double b[3], db[3], v = 1.0;
        for (int i = 0; i < k; ++i) { b[i] = beta3(y[i]); db[i] = dbeta3(y[i]); v *= b[i]; }
        if (g)
            for (int i = 0; i < k; ++i) {
                double t = db[i];
                for (int j = 0; j < k; ++j)
                    if (j != i) t *= b[j];
                g[i] = t;
            }
        return v;
    }
    if (outside_support(p, y)) {
        if (g) for (int i = 0; i < k; ++i) g[i] = 0.0;
        return 0.0;
    }
    double x[3] = {0, 0, 0};
    for (int i = 0; i < k; ++i) x[i] = y[i] + p->half[i];
    if (on_knot_plane(p, x)) {
        /* The recurrence's half-open base cases are only consistent off the
         * knot planes.  phi is continuous for every direction set used here,
         * so its value on a plane is the limit along a fixed generic
         * direction v; two points on that ray (all within one polynomial
         * piece) extrapolate linearly to the plane: error O(delta^2). */
        static const double vdir[3] = {0.5377451, 0.3141593, 0.7993603};
        const double delta = 1e-7;
        double y1[3] = {0, 0, 0}, y2[3] = {0, 0, 0}, g1[3], g2[3];
        for (int i = 0; i < k; ++i) { y1[i] = y[i] + delta * vdir[i]; y2[i] = y[i] + 2 * delta * vdir[i]; }
        double v1 = phi_generic(p, y1, g ? g1 : NULL);
        double v2 = phi_generic(p, y2, g ? g2 : NULL);
        if (g) for (int i = 0; i < k; ++i) g[i] = 2.0 * g1[i] - g2[i];
        return 2.0 * v1 - v2;
    }
    return phi_generic(p, y, g);
}

/* phi and grad phi at a point off every knot plane (y inside the support). */
static double phi_generic(phi_ctx *p, const double *y, double *g)
{
    const orc_spec *sp = p->sp;
    const int k = sp->dim;
    if (outside_support(p, y)) {
        if (g) for (int i = 0; i < k; ++i) g[i] = 0.0;
        return 0.0;
    }
    double x[3] = {0, 0, 0};
    for (int i = 0; i < k; ++i) x[i] = y[i] + p->half[i];
    double v = sp->detL * memo_eval(&p->full, x);
    if (g) {
        /* D_xi phi(y) = |det L| [M_{Xi\xi}(x) - M_{Xi\xi}(x - xi)], x = y + Xi/2 */
        double dd[3];
        for (int n = 0; n < k; ++n) {
            const double *xi = sp->dirs + 3 * p->gbasis[n];
            double xs[3] = {0, 0, 0};
            for (int i = 0; i < k; ++i) xs[i] = x[i] - xi[i];
            dd[n] = sp->detL * (memo_eval(&p->part[n], x) - memo_eval(&p->part[n], xs));
        }
        for (int i = 0; i < k; ++i) {
            g[i] = 0.0;
            for (int n = 0; n < k; ++n) g[i] += p->gbinv[i][n] * dd[n];
        }
    }
    return v;
}

/* ------------------------------------------------------------------------- */
/* Hessian                                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    phi_ctx *p;
    int npair;
    int pi[ORC_MAXDIR * (ORC_MAXDIR - 1) / 2], pj[ORC_MAXDIR * (ORC_MAXDIR - 1) / 2];
    box_memo *pm;                  /* M_{Xi \ {i, j}} per pair */
    double ninv[6][6];             /* inverse of the normal matrix of the pair equations */
    double rows[ORC_MAXDIR * (ORC_MAXDIR - 1) / 2][6];
    int nh;                        /* unknowns: 6 (3D: 00 11 22 01 02 12) or 3 (2D: 00 11 01) */
} hess_ctx;

static const int HA[6] = {0, 1, 2, 0, 0, 1}, HB[6] = {0, 1, 2, 1, 2, 2};
static const int HA2[3] = {0, 1, 0}, HB2[3] = {0, 1, 1};

/* Invert an n x n matrix (n <= 6) by Gauss-Jordan with partial pivoting. */
static int invert_small(int n, double a[6][6], double inv[6][6])
{
    double m[6][12];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c) m[r][c] = c < n ? a[r][c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(m[r][c]) > fabs(m[piv][c])) piv = r;
        if (fabs(m[piv][c]) < 1e-12) return -1;
        if (piv != c)
            for (int q = 0; q < 2 * n; ++q) { double t = m[c][q]; m[c][q] = m[piv][q]; m[piv][q] = t; }
        double d = m[c][c];
        for (int q = 0; q < 2 * n; ++q) m[c][q] /= d;
        for (int r = 0; r < n; ++r)
            if (r != c) {
                double f = m[r][c];
                for (int q = 0; q < 2 * n; ++q) m[r][q] -= f * m[c][q];
            }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r][c] = m[r][c + n];
    return 0;
}

static int hess_init(hess_ctx *h, phi_ctx *p)
{
    memset(h, 0, sizeof(*h));
    h->p = p;
    const orc_spec *sp = p->sp;
    const int k = sp->dim, m = sp->ndir;
    h->nh = k == 3 ? 6 : 3;
    if (sp->kind == 1) return 0;
    h->npair = m * (m - 1) / 2;
    h->pm = (box_memo *)calloc((size_t)h->npair, sizeof(box_memo));
    if (!h->pm) return -1;
    double ata[6][6];
    memset(ata, 0, sizeof(ata));
    int q = 0;
    for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j, ++q) {
            h->pi[q] = i;
            h->pj[q] = j;
            double rest[ORC_MAXDIR * 3];
            int mr = 0;
            for (int c = 0; c < m; ++c)
                if (c != i && c != j) { for (int t = 0; t < 3; ++t) rest[3 * mr + t] = sp->dirs[3 * c + t]; ++mr; }
            if (memo_init(&h->pm[q], k, mr, rest)) return -1;
            /* xi_i^T H xi_j in the unknowns */
            const double *u = sp->dirs + 3 * i, *v = sp->dirs + 3 * j;
            for (int e = 0; e < h->nh; ++e) {
                int a = k == 3 ? HA[e] : HA2[e], b = k == 3 ? HB[e] : HB2[e];
                h->rows[q][e] = a == b ? u[a] * v[a] : u[a] * v[b] + u[b] * v[a];
            }
            for (int r = 0; r < h->nh; ++r)
                for (int c = 0; c < h->nh; ++c) ata[r][c] += h->rows[q][r] * h->rows[q][c];
        }
    return invert_small(h->nh, ata, h->ninv);
}

static void hess_free(hess_ctx *h)
{
    if (h->pm) {
        for (int q = 0; q < h->npair; ++q) memo_free(&h->pm[q]);
        free(h->pm);
    }
}

/* Hessian of phi at y off every knot plane (out: nh values). */
static void hess_generic(hess_ctx *h, const double *y, double *out)
{
    const orc_spec *sp = h->p->sp;
    const int k = sp->dim;
    for (int e = 0; e < h->nh; ++e) out[e] = 0.0;
    if (outside_support(h->p, y)) return;
    double x[3] = {0, 0, 0};
    for (int i = 0; i < k; ++i) x[i] = y[i] + h->p->half[i];
    double atb[6] = {0, 0, 0, 0, 0, 0};
    for (int q = 0; q < h->npair; ++q) {
        const double *u = sp->dirs + 3 * h->pi[q], *v = sp->dirs + 3 * h->pj[q];
        double d = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double xs[3] = {0, 0, 0};
                for (int i = 0; i < k; ++i) xs[i] = x[i] - a * u[i] - b * v[i];
                d += ((a + b) & 1 ? -1.0 : 1.0) * memo_eval(&h->pm[q], xs);
            }
        d *= sp->detL;
        for (int e = 0; e < h->nh; ++e) atb[e] += h->rows[q][e] * d;
    }
    for (int r = 0; r < h->nh; ++r)
        for (int c = 0; c < h->nh; ++c) out[r] += h->ninv[r][c] * atb[c];
}

/* Hessian of phi at y; on a knot plane the limit from the side of a fixed
 * generic direction (as for the value and the gradient). */
static void hess_eval(hess_ctx *h, const double *y, double *out)
{
    const orc_spec *sp = h->p->sp;
    const int k = sp->dim;
    if (sp->kind == 1) {
        double b[3], db[3], d2[3];
        for (int i = 0; i < 3; ++i) { b[i] = beta3(y[i]); db[i] = dbeta3(y[i]); d2[i] = d2beta3(y[i]); }
        for (int e = 0; e < h->nh; ++e) {
            int a = k == 3 ? HA[e] : HA2[e], c = k == 3 ? HB[e] : HB2[e];
            double t = 1.0;
            for (int i = 0; i < k; ++i) {
                if (a == c) t *= (i == a) ? d2[i] : b[i];
                else t *= (i == a || i == c) ? db[i] : b[i];
            }
            out[e] = t;
        }
        return;
    }
    double x[3] = {0, 0, 0};
    for (int i = 0; i < k; ++i) x[i] = y[i] + h->p->half[i];
    if (on_knot_plane(h->p, x)) {
        static const double vdir[3] = {0.5377451, 0.3141593, 0.7993603};
        const double delta = 1e-7;
        double y1[3] = {0, 0, 0}, y2[3] = {0, 0, 0}, o1[6], o2[6];
        for (int i = 0; i < k; ++i) { y1[i] = y[i] + delta * vdir[i]; y2[i] = y[i] + 2 * delta * vdir[i]; }
        hess_generic(h, y1, o1);
        hess_generic(h, y2, o2);
        for (int e = 0; e < h->nh; ++e) out[e] = 2.0 * o1[e] - o2[e];
        return;
    }
    hess_generic(h, y, out);
}

/* ------------------------------------------------------------------------- */
/* exported entry points                                                       */
/* ------------------------------------------------------------------------- */

/* M_Xi(x) for k <= 3 and m <= 16 columns (not centred, not normalised). */
double orc_box(int32_t k, int32_t m, const double *cols, const double *x)
{
    box_memo c;
    if (k < 1 || k > 3 || m < 0 || m > ORC_MAXDIR) return NAN;
    if (memo_init(&c, k, m, cols)) return NAN;
    double v = memo_eval(&c, x);
    memo_free(&c);
    return v;
}

/* phi at n points y (n*dim), optional gradient (n*dim). Returns 0 or <0 on error. */
int32_t orc_phi(const orc_spec *sp, const double *y, int64_t n, double *val, double *grad)
{
    phi_ctx p;
    if (phi_init(&p, sp, grad != NULL)) return -1;
    const int k = sp->dim;
    for (int64_t q = 0; q < n; ++q) {
        double v = phi_eval(&p, y + k * q, grad ? grad + k * q : NULL);
        if (val) val[q] = v;
    }
    phi_free(&p);
    return 0;
}

/* Half-width of the support bounding box along each axis: 1/2 sum_xi |xi_i|. */
static void support_halfwidth(const orc_spec *sp, double *h)
{
    for (int i = 0; i < 3; ++i) h[i] = 0.0;
    if (sp->kind == 1) { for (int i = 0; i < sp->dim; ++i) h[i] = 2.0; return; }
    for (int j = 0; j < sp->ndir; ++j)
        for (int i = 0; i < sp->dim; ++i) h[i] += 0.5 * fabs(sp->dirs[3 * j + i]);
}

/* Enumerate the stored sites whose support bounding box contains x. */
typedef void (*site_fn)(void *ctx, int64_t lin, const double *y);

static void for_each_site(const orc_spec *sp, const double *x, site_fn fn, void *ctx)
{
    const int k = sp->dim;
    const int64_t a = sp->scale;
    double h[3];
    support_halfwidth(sp, h);
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    const int64_t per = sp->ext[0] * (k > 1 ? sp->ext[1] : 1) * (k > 2 ? sp->ext[2] : 1);
    for (int j = 0; j < sp->ncoset; ++j) {
        int ok = 1;
        for (int i = 0; i < k; ++i) {
            /* sites n = a*idx + l with |x - n| < h  ->  idx in (x - h - l)/a .. (x + h - l)/a */
            double lof = ceil((x[i] - h[i] - sp->coset[3 * j + i]) / (double)a);
            double hif = floor((x[i] + h[i] - sp->coset[3 * j + i]) / (double)a);
            lo[i] = (int64_t)lof;
            hi[i] = (int64_t)hif;
            if (lo[i] < 0) lo[i] = 0;
            if (hi[i] > sp->ext[i] - 1) hi[i] = sp->ext[i] - 1;
            if (lo[i] > hi[i]) ok = 0;
        }
        if (!ok) continue;
        for (int i = k; i < 3; ++i) { lo[i] = 0; hi[i] = 0; }
        for (int64_t i2 = lo[2]; i2 <= hi[2]; ++i2)
            for (int64_t i1 = lo[1]; i1 <= hi[1]; ++i1)
                for (int64_t i0 = lo[0]; i0 <= hi[0]; ++i0) {
                    int64_t idx[3] = {i0, i1, i2};
                    double y[3] = {0, 0, 0};
                    for (int i = 0; i < k; ++i)
                        y[i] = x[i] - (double)(a * idx[i] + sp->coset[3 * j + i]);
                    int64_t lin = j * per + i0 + sp->ext[0] * (i1 + (k > 1 ? sp->ext[1] : 1) * i2);
                    fn(ctx, lin, y);
                }
    }
}

typedef struct {
    phi_ctx *p;
    const double *coef;
    double f;
    double g[3];
    int want_grad;
} eval_acc;

static void eval_site(void *vctx, int64_t lin, const double *y)
{
    eval_acc *e = (eval_acc *)vctx;
    double c = e->coef[lin];
    double g[3];
    double v = phi_eval(e->p, y, e->want_grad ? g : NULL);
    e->f += c * v;
    if (e->want_grad)
        for (int i = 0; i < e->p->sp->dim; ++i) e->g[i] += c * g[i];
}

static int nthreads_or_default(int32_t nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/*
 * Naive convolution sum (Eq. 1) at n points x (n*dim, FP64).
 * coef: ncoset * ext0*ext1*ext2 values, coset-major, axis 0 fastest.
 * out: n values; grad (nullable): n*dim values of grad f.
 */
int32_t orc_eval(const orc_spec *sp, const double *coef, const double *pts, int64_t n,
                 double *out, double *grad, int32_t nthreads)
{
    int err = 0;
    const int k = sp->dim;
#pragma omp parallel num_threads(nthreads_or_default(nthreads)) reduction(| : err)
    {
        phi_ctx p;
        if (phi_init(&p, sp, grad != NULL)) {
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t q = 0; q < n; ++q) {
                eval_acc e;
                memset(&e, 0, sizeof(e));
                e.p = &p;
                e.coef = coef;
                e.want_grad = grad != NULL;
                for_each_site(sp, pts + k * q, eval_site, &e);
                out[q] = e.f;
                if (grad)
                    for (int i = 0; i < k; ++i) grad[k * q + i] = e.g[i];
            }
            phi_free(&p);
        }
    }
    return err ? -1 : 0;
}

typedef struct {
    phi_ctx *p;
    double gp;
    double *dc;
} adj_acc;

static void adj_site(void *vctx, int64_t lin, const double *y)
{
    adj_acc *a = (adj_acc *)vctx;
    double v = phi_eval(a->p, y, NULL);
    if (v != 0.0) a->dc[lin] += a->gp * v;
}

/*
 * Adjoint of Eq. 1 with respect to the coefficients:
 *     dc_n += sum_p g_p phi(x_p - n)
 * dc has the layout of coef and is accumulated into (serial, point order).
 */
int32_t orc_adjoint(const orc_spec *sp, const double *pts, const double *g, int64_t n, double *dc)
{
    phi_ctx p;
    if (phi_init(&p, sp, 0)) return -1;
    const int k = sp->dim;
    for (int64_t q = 0; q < n; ++q) {
        adj_acc a = {&p, g[q], dc};
        for_each_site(sp, pts + k * q, adj_site, &a);
    }
    phi_free(&p);
    return 0;
}

typedef struct {
    phi_ctx *p;
    int64_t row;
    int64_t *rows, *cols;
    double *vals;
    int64_t cap, cnt;
} trip_acc;

static void trip_site(void *vctx, int64_t lin, const double *y)
{
    trip_acc *t = (trip_acc *)vctx;
    double v = phi_eval(t->p, y, NULL);
    if (v == 0.0) return;
    if (t->cnt < t->cap) {
        t->rows[t->cnt] = t->row;
        t->cols[t->cnt] = lin;
        t->vals[t->cnt] = v;
    }
    t->cnt++;
}

/*
 * Entries A[p, n] = phi(x_p - n) of the linear map c -> f(x_p) (Eq. 1), as
 * (row, col, value) triplets.  Returns the number of nonzeros; if it exceeds
 * cap, nothing beyond cap is written and the caller retries with more room.
 */
int64_t orc_design_triplets(const orc_spec *sp, const double *pts, int64_t n,
                            int64_t *rows, int64_t *cols, double *vals, int64_t cap)
{
    phi_ctx p;
    if (phi_init(&p, sp, 0)) return -1;
    trip_acc t = {&p, 0, rows, cols, vals, cap, 0};
    for (int64_t q = 0; q < n; ++q) {
        t.row = q;
        for_each_site(sp, pts + sp->dim * q, trip_site, &t);
    }
    phi_free(&p);
    return t.cnt;
}

/*
 * 3D Morton code: bit b of coordinate i goes to bit 3*b + i of the key
 * (coordinate 0 in the lowest bit), 10 bits per coordinate.
 */
uint32_t orc_morton3(uint32_t c0, uint32_t c1, uint32_t c2)
{
    uint32_t key = 0;
    const uint32_t c[3] = {c0, c1, c2};
    for (int b = 0; b < 10; ++b)
        for (int i = 0; i < 3; ++i)
            key |= ((c[i] >> b) & 1u) << (3 * b + i);
    return key;
}

/* Hessian of phi at n points y (n*dim): hess n*6 (3D: xx yy zz xy xz yz) or n*3 (2D: xx yy xy). */
int32_t orc_phi_hess(const orc_spec *sp, const double *y, int64_t n, double *hess)
{
    phi_ctx p;
    hess_ctx h;
    if (phi_init(&p, sp, 0)) return -1;
    if (hess_init(&h, &p)) { hess_free(&h); phi_free(&p); return -1; }
    const int k = sp->dim;
    for (int64_t q = 0; q < n; ++q) hess_eval(&h, y + k * q, hess + h.nh * q);
    hess_free(&h);
    phi_free(&p);
    return 0;
}

typedef struct {
    hess_ctx *h;
    const double *coef;
    double hs[6];
} hess_acc;

static void hess_site(void *vctx, int64_t lin, const double *y)
{
    hess_acc *e = (hess_acc *)vctx;
    double c = e->coef[lin];
    if (c == 0.0) return;
    double o[6];
    hess_eval(e->h, y, o);
    for (int t = 0; t < e->h->nh; ++t) e->hs[t] += c * o[t];
}

/* Hessian of the naive sum (Eq. 1) at n points: hess n*6 (3D) or n*3 (2D). */
int32_t orc_eval_hess(const orc_spec *sp, const double *coef, const double *pts, int64_t n, double *hess,
                      int32_t nthreads)
{
    int err = 0;
    const int k = sp->dim;
#pragma omp parallel num_threads(nthreads_or_default(nthreads)) reduction(| : err)
    {
        phi_ctx p;
        hess_ctx h;
        if (phi_init(&p, sp, 0)) {
            err = 1;
        } else if (hess_init(&h, &p)) {
            hess_free(&h);
            phi_free(&p);
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t q = 0; q < n; ++q) {
                hess_acc e;
                memset(&e, 0, sizeof(e));
                e.h = &h;
                e.coef = coef;
                for_each_site(sp, pts + k * q, hess_site, &e);
                for (int t = 0; t < h.nh; ++t) hess[h.nh * q + t] = e.hs[t];
            }
            hess_free(&h);
            phi_free(&p);
        }
    }
    return err ? -1 : 0;
}

int32_t orc_abi_version(void) { return 1; }

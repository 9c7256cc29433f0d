/*
 * dg_oracle.c -- plain, slow, FP64 CPU reference of the modal discontinuous
 * Galerkin method for 2D nonlinear conservation laws of Fuhry, Giuliani and
 * Krivodonova (arXiv:1601.07944), applied to the compressible Euler equations.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the package's smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, table or helper with the CUDA path.
 *
 * What it follows, section by section of the paper:
 *   - weak form and reference map (Section 2, Eqs. 2ddg, weak2dsys, 2dmap);
 *   - edge map and edge Jacobian l = |edge|/2 (Eqs. 1dmap, len, surfaceintegral);
 *   - orthonormal basis on the reference triangle, N_p = (p+1)(p+2)/2 (Eq. np);
 *   - semi-discrete system dc/dt = (volume - surface)/det J (Eq. 2ddg0);
 *   - the three kernels of Section 4.3 in their order: the per-element volume
 *     integral (Algorithm 1), the per-edge surface integral with left/right
 *     temporaries and reversed point order on the right element (Algorithm 2,
 *     Eq. edgeint), and the per-element combination (Algorithm 3);
 *   - Euler flux and equation of state, gamma = 1.4 (Eq. euler, Section 5).
 *
 * Readings where the paper is silent or garbled (each one is listed in the
 * design notes of the repository):
 *   - basis: the Dubiner product basis in collapsed coordinates, ordered by
 *     total degree and, within a degree, by the second index ascending; each
 *     function is expanded here exactly into monomials r^x s^y and normalised
 *     with the exact monomial integrals int r^x s^y = x! y! / (x+y+2)!;
 *   - volume rule: collapsed Gauss-Jacobi (Stroud) rule with n = p+1 points per
 *     direction, exact to degree 2p+1 (the paper's degree-2p tables are not
 *     reproduced);  edge rule: Gauss-Legendre with p+1 points;
 *   - the volume term is F . (det J J^{-T} grad_r phi), i.e. the physical
 *     gradient of the test function (the paper's printed transpose is garbled);
 *   - numerical flux: local Lax-Friedrichs with alpha = max(|v.n| + c) of the
 *     two traces at each quadrature point;
 *   - the surface temporaries are per edge (one left and one right block).
 *   - time integration: the three-stage SSP Runge-Kutta method in Shu-Osher
 *     form, and the paper's own classic RK2 (read as Heun's method) and RK4;
 *   - the Barth-Jespersen limiter (p = 1) with the standard per-point ratio;
 *   - boundary faces (Algorithm 2's ghost state): a solid wall mirrors the
 *     momentum, U_g = (rho, m - 2 (m.n) n, E); a prescribed boundary takes a
 *     state the caller gives at each boundary quadrature point.
 *
 * Layout of every coefficient array: c[e][m][j], element e, variable m (M=4),
 * mode j (N_p), float64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OM 4           /* number of conserved variables */
#define OPMAX 12       /* highest polynomial degree handled by the monomial tables */

/* ------------------------------------------------------------------------- */
/* Quadrature: Gauss-Jacobi nodes by Newton iteration on the three-term      */
/* recurrence, with deflation against the roots already found.               */
/* ------------------------------------------------------------------------- */

/* P_n^{(a,b)}(x) and its derivative, from the standard three-term recurrence
 * (normalisation P_n(1) = binom(n+a, n)), in extended precision. */
static void jacobi_eval(int n, long double a, long double b, long double x, long double *P, long double *dP)
{
    long double p0 = 1.0L, p1 = 0.5L * (a - b + (a + b + 2.0L) * x);
    long double d0 = 0.0L, d1 = 0.5L * (a + b + 2.0L);
    if (n == 0) { *P = 1.0L; *dP = 0.0L; return; }
    for (int k = 2; k <= n; ++k) {
        long double kk = (long double)k;
        long double c1 = 2.0L * kk * (kk + a + b) * (2.0L * kk + a + b - 2.0L);
        long double c2 = (2.0L * kk + a + b - 1.0L) * (a * a - b * b);
        long double c3 = (2.0L * kk + a + b - 2.0L) * (2.0L * kk + a + b - 1.0L) * (2.0L * kk + a + b);
        long double c4 = 2.0L * (kk + a - 1.0L) * (kk + b - 1.0L) * (2.0L * kk + a + b);
        long double p2 = ((c2 + c3 * x) * p1 - c4 * p0) / c1;
        long double d2 = ((c2 + c3 * x) * d1 + c3 * p1 - c4 * d0) / c1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    *P = p1; *dP = d1;
}

/* n-point Gauss-Jacobi rule for the weight (1-x)^a (1+x)^b on [-1, 1], nodes
 * ascending, computed in extended precision (Newton iteration with deflation)
 * and rounded once to double.  xl, wl (optional) receive the extended values. */
static int gauss_jacobi_l(int n, double a_, double b_, long double *xl, long double *wl)
{
    if (n < 1 || n > 64) return 1;
    long double a = a_, b = b_;
    const long double pi = 3.14159265358979323846264338327950288L;
    for (int k = 0; k < n; ++k) {
        /* Chebyshev-Gauss guess, then Newton with deflation */
        long double r = -cosl((2.0L * k + 1.0L) * pi / (2.0L * n));
        for (int it = 0; it < 200; ++it) {
            long double P, dP;
            jacobi_eval(n, a, b, r, &P, &dP);
            long double s = 0.0L;
            for (int i = 0; i < k; ++i) s += 1.0L / (r - xl[i]);
            long double delta = -P / (dP - s * P);
            r += delta;
            if (fabsl(delta) <= 1e-30L * (1.0L + fabsl(r)) || (it > 8 && fabsl(delta) < 1e-17L)) break;
        }
        xl[k] = r;
    }
    /* sort ascending (deflation keeps them distinct but not necessarily ordered) */
    for (int i = 1; i < n; ++i) {
        long double t = xl[i]; int j = i - 1;
        while (j >= 0 && xl[j] > t) { xl[j + 1] = xl[j]; --j; }
        xl[j + 1] = t;
    }
    long double lg = lgammal(n + a + 1.0L) + lgammal(n + b + 1.0L) - lgammal(n + a + b + 1.0L) - lgammal(n + 1.0L);
    long double cst = powl(2.0L, a + b + 1.0L) * expl(lg);
    for (int k = 0; k < n; ++k) {
        long double P, dP;
        jacobi_eval(n, a, b, xl[k], &P, &dP);
        wl[k] = cst / ((1.0L - xl[k] * xl[k]) * dP * dP);
    }
    return 0;
}

int or_gauss_jacobi(int n, double a, double b, double *x, double *w)
{
    long double xl[64], wl[64];
    if (gauss_jacobi_l(n, a, b, xl, wl)) return 1;
    for (int k = 0; k < n; ++k) { x[k] = (double)xl[k]; w[k] = (double)wl[k]; }
    return 0;
}

int or_gauss_legendre(int n, double *x, double *w) { return or_gauss_jacobi(n, 0.0, 0.0, x, w); }

/* Collapsed (Stroud conical product) rule on the reference triangle
 * {(0,0),(1,0),(0,1)}: Gauss-Legendre in a, Gauss-Jacobi(1,0) in b,
 * r = (1+a)(1-b)/4, s = (1+b)/2, weight w_a w_b / 8.  n^2 points, exact for
 * polynomials of degree 2n-1; the weights sum to 1/2 (the triangle's area).
 * Point order: b-index outer, a-index inner.  The 1D nodes are rounded to
 * double; the points are the exact (extended-precision) images of those rounded
 * nodes, which is where the basis tables are evaluated, and they are stored
 * rounded to double.  rl, sl (optional) receive the extended points. */
static int stroud_l(int n, double *r, double *s, double *w, long double *rl, long double *sl)
{
    long double xa[64], wa[64], xb[64], wb[64];
    if (gauss_jacobi_l(n, 0.0, 0.0, xa, wa)) return 1;
    if (gauss_jacobi_l(n, 1.0, 0.0, xb, wb)) return 1;
    for (int ib = 0; ib < n; ++ib)
        for (int ia = 0; ia < n; ++ia) {
            int k = ib * n + ia;
            long double a = (double)xa[ia], b = (double)xb[ib];
            long double rr = 0.25L * (1.0L + a) * (1.0L - b), ss = 0.5L * (1.0L + b);
            r[k] = (double)rr;
            s[k] = (double)ss;
            w[k] = (double)(0.125L * wa[ia] * wb[ib]);
            if (rl) rl[k] = rr;
            if (sl) sl[k] = ss;
        }
    return 0;
}

int or_stroud(int n, double *r, double *s, double *w) { return stroud_l(n, r, s, w, NULL, NULL); }

/* ------------------------------------------------------------------------- */
/* Orthonormal Dubiner basis on the reference triangle.                      */
/* In collapsed coordinates alpha = 2r/(1-s) - 1, beta = 2s - 1              */
/*   psi_ab = P_a(alpha) (1-s)^a P_b^{(2a+1,0)}(beta),   a + b <= p.         */
/* With the explicit sum                                                      */
/*   P_n^{(u,v)}(x) = sum_m C(n+u, n-m) C(n+v, m) ((x-1)/2)^m ((x+1)/2)^(n-m) */
/* and ((alpha-1)/2)(1-s) = r+s-1, ((alpha+1)/2)(1-s) = r, this is           */
/*   psi_ab = A_a(r,s) B_ab(s),                                              */
/*   A_a  = sum_m C(a,m)^2 (r+s-1)^m r^(a-m),                                */
/*   B_ab = sum_m C(b+2a+1, b-m) C(b,m) (s-1)^m s^(b-m),                     */
/* a polynomial with integer coefficients.  The normalisation int psi^2 = 1  */
/* is computed exactly from those integer coefficients and the monomial      */
/* integrals int r^x s^y = x! y! / (x+y+2)!; point values and gradients are  */
/* evaluated from the two sums above in extended precision.                  */
/* Order: total degree d = a+b ascending, then b ascending.                  */
/* ------------------------------------------------------------------------- */

typedef __int128 i128;
typedef struct { i128 c[OPMAX + 1][OPMAX + 1]; } ipoly;   /* c[x][y] * r^x s^y */

static int64_t ibinom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    int64_t v = 1;
    for (int i = 1; i <= k; ++i) v = v * (n - k + i) / i;
    return v;
}

static void ip_zero(ipoly *p) { memset(p, 0, sizeof *p); }

static void ip_mul(const ipoly *a, const ipoly *b, ipoly *out)
{
    ipoly t; ip_zero(&t);
    for (int x1 = 0; x1 <= OPMAX; ++x1)
        for (int y1 = 0; x1 + y1 <= OPMAX; ++y1) {
            if (a->c[x1][y1] == 0) continue;
            for (int x2 = 0; x1 + x2 <= OPMAX; ++x2)
                for (int y2 = 0; x1 + y1 + x2 + y2 <= OPMAX; ++y2)
                    t.c[x1 + x2][y1 + y2] += a->c[x1][y1] * b->c[x2][y2];
        }
    *out = t;
}

static void ip_pow(const ipoly *a, int k, ipoly *out)
{
    ipoly t; ip_zero(&t); t.c[0][0] = 1;
    for (int i = 0; i < k; ++i) ip_mul(&t, a, &t);
    *out = t;
}

static void ip_axpy(i128 f, const ipoly *x, ipoly *y)
{
    for (int i = 0; i <= OPMAX; ++i)
        for (int j = 0; i + j <= OPMAX; ++j) y->c[i][j] += f * x->c[i][j];
}

/* integer monomial coefficients of the unnormalised psi_ab */
static void psi_int(int a, int b, ipoly *out)
{
    ipoly rs1, r1, s1, s0, A, B, t1, t2;
    ip_zero(&rs1); rs1.c[1][0] = 1; rs1.c[0][1] = 1; rs1.c[0][0] = -1;   /* r+s-1 */
    ip_zero(&r1); r1.c[1][0] = 1;                                        /* r */
    ip_zero(&s1); s1.c[0][1] = 1; s1.c[0][0] = -1;                       /* s-1 */
    ip_zero(&s0); s0.c[0][1] = 1;                                        /* s */
    ip_zero(&A);
    for (int m = 0; m <= a; ++m) {
        ip_pow(&rs1, m, &t1); ip_pow(&r1, a - m, &t2); ip_mul(&t1, &t2, &t1);
        ip_axpy((i128)(ibinom(a, m) * ibinom(a, m)), &t1, &A);
    }
    ip_zero(&B);
    for (int m = 0; m <= b; ++m) {
        ip_pow(&s1, m, &t1); ip_pow(&s0, b - m, &t2); ip_mul(&t1, &t2, &t1);
        ip_axpy((i128)(ibinom(b + 2 * a + 1, b - m) * ibinom(b, m)), &t1, &B);
    }
    ip_mul(&A, &B, out);
}

/* exact integral over the reference triangle of an integer polynomial of degree
 * <= dmax, returned as (numerator, denominator = (dmax+2)!) in long double */
static long double ip_integral(const ipoly *a, int dmax)
{
    i128 D = 1;
    for (int i = 2; i <= dmax + 2; ++i) D *= i;
    i128 num = 0;
    for (int x = 0; x <= dmax; ++x)
        for (int y = 0; x + y <= dmax; ++y) {
            if (a->c[x][y] == 0) continue;
            /* x! y! D / (x+y+2)! is an integer */
            i128 f;
            i128 w = 1;
            for (int i = 2; i <= x; ++i) w *= i;
            for (int i = 2; i <= y; ++i) w *= i;
            i128 den = 1;
            for (int i = 2; i <= x + y + 2; ++i) den *= i;
            f = (D / den) * w;
            num += a->c[x][y] * f;
        }
    return (long double)num / (long double)D;
}

/* 1/sqrt(int psi_ab^2), exact up to the final rounding */
static long double psi_norm(int a, int b)
{
    ipoly psi, sq;
    psi_int(a, b, &psi);
    ip_mul(&psi, &psi, &sq);
    return 1.0L / sqrtl(ip_integral(&sq, 2 * (a + b)));
}

static long double powli(long double x, int k)
{
    long double v = 1.0L;
    for (int i = 0; i < k; ++i) v *= x;
    return v;
}

/* value and gradient of the normalised psi_ab at (r, s) from the two sums */
static void psi_eval(int a, int b, long double nrm, long double r, long double s,
                     double *v, double *dr, double *ds)
{
    long double t = r + s - 1.0L, u = s - 1.0L;
    long double A = 0, Ar = 0, As = 0;
    for (int m = 0; m <= a; ++m) {
        long double cf = (long double)(ibinom(a, m) * ibinom(a, m));
        long double tm = powli(t, m), rm = powli(r, a - m);
        A += cf * tm * rm;
        long double dtm = m > 0 ? m * powli(t, m - 1) : 0.0L;          /* d t^m / dt */
        long double drm = (a - m) > 0 ? (a - m) * powli(r, a - m - 1) : 0.0L;
        Ar += cf * (dtm * rm + tm * drm);                               /* dt/dr = 1 */
        As += cf * (dtm * rm);                                          /* dt/ds = 1 */
    }
    long double B = 0, Bs = 0;
    for (int m = 0; m <= b; ++m) {
        long double cf = (long double)(ibinom(b + 2 * a + 1, b - m) * ibinom(b, m));
        long double um = powli(u, m), sm = powli(s, b - m);
        B += cf * um * sm;
        long double dum = m > 0 ? m * powli(u, m - 1) : 0.0L;
        long double dsm = (b - m) > 0 ? (b - m) * powli(s, b - m - 1) : 0.0L;
        Bs += cf * (dum * sm + um * dsm);
    }
    *v = (double)(nrm * A * B);
    if (dr) *dr = (double)(nrm * Ar * B);
    if (ds) *ds = (double)(nrm * (As * B + A * Bs));
}

static int mode_ab(int p, int j, int *a, int *b)
{
    int k = 0;
    for (int d = 0; d <= p; ++d)
        for (int bb = 0; bb <= d; ++bb, ++k)
            if (k == j) { *a = d - bb; *b = bb; return 0; }
    return 1;
}

/* Values and reference gradients of the N_p basis functions at npts points:
 * out arrays are [npts][Np].  Any of dphir, dphis may be NULL. */
int or_dubiner_eval(int p, int npts, const double *r, const double *s,
                    double *phi, double *dphir, double *dphis)
{
    if (p < 0 || 2 * p > OPMAX) return 1;
    int np = (p + 1) * (p + 2) / 2;
    for (int j = 0; j < np; ++j) {
        int a = 0, b = 0;
        mode_ab(p, j, &a, &b);
        long double nrm = psi_norm(a, b);
        for (int k = 0; k < npts; ++k)
            psi_eval(a, b, nrm, r[k], s[k], &phi[k * np + j],
                     dphir ? &dphir[k * np + j] : NULL, dphis ? &dphis[k * np + j] : NULL);
    }
    return 0;
}

/* the same at extended-precision points */
static int dubiner_eval_l(int p, int npts, const long double *r, const long double *s,
                          double *phi, double *dphir, double *dphis)
{
    if (p < 0 || 2 * p > OPMAX) return 1;
    int np = (p + 1) * (p + 2) / 2;
    for (int j = 0; j < np; ++j) {
        int a = 0, b = 0;
        mode_ab(p, j, &a, &b);
        long double nrm = psi_norm(a, b);
        for (int k = 0; k < npts; ++k)
            psi_eval(a, b, nrm, r[k], s[k], &phi[k * np + j],
                     dphir ? &dphir[k * np + j] : NULL, dphis ? &dphis[k * np + j] : NULL);
    }
    return 0;
}

/* exact integrals int phi_j over the reference triangle */
int or_dubiner_integrals(int p, double *out)
{
    if (p < 0 || 2 * p > OPMAX) return 1;
    int np = (p + 1) * (p + 2) / 2;
    for (int j = 0; j < np; ++j) {
        int a = 0, b = 0; ipoly psi;
        mode_ab(p, j, &a, &b);
        psi_int(a, b, &psi);
        out[j] = (double)(psi_norm(a, b) * ip_integral(&psi, a + b));
    }
    return 0;
}

/* exact Gram matrix int phi_i phi_j from the integer expansions */
int or_dubiner_gram_exact(int p, double *G)
{
    if (p < 0 || 2 * p > OPMAX) return 1;
    int np = (p + 1) * (p + 2) / 2;
    for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
            int ai = 0, bi = 0, aj = 0, bj = 0; ipoly pi, pj, t;
            mode_ab(p, i, &ai, &bi); mode_ab(p, j, &aj, &bj);
            psi_int(ai, bi, &pi); psi_int(aj, bj, &pj);
            ip_mul(&pi, &pj, &t);
            G[i * np + j] = (double)(psi_norm(ai, bi) * psi_norm(aj, bj) * ip_integral(&t, ai + bi + aj + bj));
        }
    return 0;
}

/* normalised monomial coefficients of phi_j, [Np][OPMAX+1][OPMAX+1] (rank tests) */
int or_dubiner_monomials(int p, double *out)
{
    if (p < 0 || 2 * p > OPMAX) return 1;
    int np = (p + 1) * (p + 2) / 2, K = OPMAX + 1;
    for (int j = 0; j < np; ++j) {
        int a = 0, b = 0; ipoly psi;
        mode_ab(p, j, &a, &b);
        psi_int(a, b, &psi);
        long double nrm = psi_norm(a, b);
        for (int x = 0; x < K; ++x)
            for (int y = 0; y < K; ++y)
                out[((size_t)j * K + x) * K + y] = (double)(nrm * (long double)psi.c[x][y]);
    }
    return 0;
}

int or_opmax(void) { return OPMAX; }

/* ------------------------------------------------------------------------- */
/* Solver state                                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    int p, np, nq, ne;
    double gamma;
    /* volume rule and tables, [nq] and [nq][np] */
    double *vr, *vs, *vw, *phi, *phir, *phis;
    /* edge rule on [-1,1], [ne]; face tables phif[q][k][np] */
    double *ex, *ew, *phif;
    double phi_int[64];                       /* int phi_j over the reference triangle */
    /* mesh */
    int64_t N, Ns;
    double *xy;                               /* [N][3][2] */
    double *detJ;                             /* [N] */
    double *JT;                               /* [N][4]: det J * J^{-T}, row-major */
    int64_t *el, *er;                         /* [Ns] left/right element */
    int *eL, *eR;                             /* [Ns] side maps (0-based local face) */
    double *enx, *eny, *elen;                 /* [Ns] unit normal l->r, full length */
    int64_t *elem_edge;                       /* [N][3] edge of each local face */
    /* temporaries of Algorithms 1-3 */
    double *rhs_volume;                       /* [N][M][Np] */
    double *rhs_surface_left, *rhs_surface_right;   /* [Ns][M][Np] */
    int limit;                                /* limit every stage value (p = 1) */
    /* boundary faces (Algorithm 2: the right state is a ghost state): er[s] is the
     * boundary code (-1 solid wall, -2 prescribed state), bidx[s] the face's index
     * among the boundary faces (-1 for interior faces); bstate [Nb][ne][M] */
    int64_t Nb, *bidx;
    double *bstate;
} oracle_dg;

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

void or_destroy(oracle_dg *o)
{
    if (!o) return;
    free(o->vr); free(o->vs); free(o->vw); free(o->phi); free(o->phir); free(o->phis);
    free(o->ex); free(o->ew); free(o->phif);
    free(o->xy); free(o->detJ); free(o->JT); free(o->el); free(o->er); free(o->eL); free(o->eR);
    free(o->enx); free(o->eny); free(o->elen); free(o->elem_edge);
    free(o->rhs_volume); free(o->rhs_surface_left); free(o->rhs_surface_right);
    free(o->bidx); free(o->bstate);
    free(o);
}

/* reference coordinates of point k (0-based, xi ascending) of local face q:
 * face q runs from reference vertex q to vertex q+1 (mod 3), counter-clockwise */
static void face_point(int q, double xi, double *r, double *s)
{
    static const double V[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
    int q1 = (q + 1) % 3;
    *r = 0.5 * (1.0 - xi) * V[q][0] + 0.5 * (1.0 + xi) * V[q1][0];
    *s = 0.5 * (1.0 - xi) * V[q][1] + 0.5 * (1.0 + xi) * V[q1][1];
}

/*
 * Creates the oracle for a mesh of N counter-clockwise triangles.
 *   xy[N][3][2]      vertex coordinates (unwrapped per element);
 *   nbr[N][3]        element across local face q, or a boundary code: -1 for a
 *                    solid wall, -2 for a state prescribed at the face's points;
 *   nbr_face[N][3]   the neighbour's local face index of that edge (-1 on a
 *                    boundary).
 * nvol = points per direction of the collapsed volume rule (0: p+1);
 * ne = edge points (0: p+1).  Returns NULL on invalid input.
 */
oracle_dg *or_create(int p, int ne, int nvol, double gamma, int64_t N, const double *xy,
                     const int64_t *nbr, const int8_t *nbr_face)
{
    if (p < 0 || 2 * p > OPMAX || N < 1) return NULL;
    oracle_dg *o = (oracle_dg *)calloc(1, sizeof *o);
    if (!o) return NULL;
    o->p = p; o->np = (p + 1) * (p + 2) / 2;
    o->ne = ne > 0 ? ne : p + 1;
    int nd = nvol > 0 ? nvol : p + 1;
    o->nq = nd * nd;
    o->gamma = gamma;
    o->N = N;
    int np = o->np, nq = o->nq;

    o->vr = xcalloc(nq, sizeof(double)); o->vs = xcalloc(nq, sizeof(double)); o->vw = xcalloc(nq, sizeof(double));
    o->phi = xcalloc((size_t)nq * np, sizeof(double));
    o->phir = xcalloc((size_t)nq * np, sizeof(double));
    o->phis = xcalloc((size_t)nq * np, sizeof(double));
    {
        long double rl[4096], sl[4096];
        if (nq > 4096) { or_destroy(o); return NULL; }
        stroud_l(nd, o->vr, o->vs, o->vw, rl, sl);
        dubiner_eval_l(p, nq, rl, sl, o->phi, o->phir, o->phis);
    }
    or_dubiner_integrals(p, o->phi_int);

    o->ex = xcalloc(o->ne, sizeof(double)); o->ew = xcalloc(o->ne, sizeof(double));
    or_gauss_legendre(o->ne, o->ex, o->ew);
    o->phif = xcalloc((size_t)3 * o->ne * np, sizeof(double));
    for (int q = 0; q < 3; ++q)
        for (int k = 0; k < o->ne; ++k) {
            double r, s;
            face_point(q, o->ex[k], &r, &s);
            or_dubiner_eval(p, 1, &r, &s, o->phif + ((size_t)q * o->ne + k) * np, NULL, NULL);
        }

    /* element geometry (Eq. 2dmap): J = [[x2-x1, x3-x1], [y2-y1, y3-y1]] */
    o->xy = xcalloc((size_t)N * 6, sizeof(double));
    memcpy(o->xy, xy, sizeof(double) * 6 * (size_t)N);
    o->detJ = xcalloc(N, sizeof(double));
    o->JT = xcalloc((size_t)N * 4, sizeof(double));
    for (int64_t e = 0; e < N; ++e) {
        const double *v = xy + 6 * e;
        double a = v[2] - v[0], b = v[4] - v[0], c = v[3] - v[1], d = v[5] - v[1];
        double det = a * d - b * c;
        if (!(det > 0.0)) { or_destroy(o); return NULL; }
        o->detJ[e] = det;
        /* det J * J^{-T} = [[d, -c], [-b, a]] */
        o->JT[4 * e + 0] = d;  o->JT[4 * e + 1] = -c;
        o->JT[4 * e + 2] = -b; o->JT[4 * e + 3] = a;
    }

    /* edge list: the pair (e,q) that sorts first is the left element */
    o->elem_edge = xcalloc((size_t)N * 3, sizeof(int64_t));
    int64_t Ns = 0, Nb = 0;
    for (int64_t e = 0; e < N; ++e)
        for (int q = 0; q < 3; ++q) {
            int64_t f = nbr[3 * e + q]; int qf = nbr_face[3 * e + q];
            if (f == -1 || f == -2) { ++Ns; ++Nb; continue; }
            if (f < 0 || f >= N || qf < 0 || qf > 2) { or_destroy(o); return NULL; }
            if (nbr[3 * f + qf] != e || nbr_face[3 * f + qf] != q) { or_destroy(o); return NULL; }
            if (e < f || (e == f && q < qf)) ++Ns;
        }
    o->Ns = Ns;
    o->Nb = Nb;
    o->bidx = xcalloc(Ns, sizeof(int64_t));
    o->bstate = xcalloc((size_t)Nb * o->ne * OM, sizeof(double));
    o->el = xcalloc(Ns, sizeof(int64_t)); o->er = xcalloc(Ns, sizeof(int64_t));
    o->eL = xcalloc(Ns, sizeof(int)); o->eR = xcalloc(Ns, sizeof(int));
    o->enx = xcalloc(Ns, sizeof(double)); o->eny = xcalloc(Ns, sizeof(double));
    o->elen = xcalloc(Ns, sizeof(double));
    int64_t s = 0, b = 0;
    for (int64_t e = 0; e < N; ++e)
        for (int q = 0; q < 3; ++q) {
            int64_t f = nbr[3 * e + q]; int qf = nbr_face[3 * e + q];
            if (f < 0) {
                /* boundary face: the element is its left side, the code its right */
                const double *v = xy + 6 * e;
                int q1 = (q + 1) % 3;
                double dx = v[2 * q1] - v[2 * q], dy = v[2 * q1 + 1] - v[2 * q + 1];
                double len = sqrt(dx * dx + dy * dy);
                o->el[s] = e; o->er[s] = f; o->eL[s] = q; o->eR[s] = -1;
                o->enx[s] = dy / len; o->eny[s] = -dx / len;
                o->elen[s] = len;
                o->elem_edge[3 * e + q] = s;
                o->bidx[s] = b++;
                ++s;
                continue;
            }
            if (!(e < f || (e == f && q < qf))) continue;
            o->bidx[s] = -1;
            const double *v = xy + 6 * e;
            int q1 = (q + 1) % 3;
            double dx = v[2 * q1] - v[2 * q], dy = v[2 * q1 + 1] - v[2 * q + 1];
            double len = sqrt(dx * dx + dy * dy);
            o->el[s] = e; o->er[s] = f; o->eL[s] = q; o->eR[s] = qf;
            o->enx[s] = dy / len; o->eny[s] = -dx / len;   /* outward for the left element */
            o->elen[s] = len;
            o->elem_edge[3 * e + q] = s;
            o->elem_edge[3 * f + qf] = s;
            ++s;
        }
    o->rhs_volume = xcalloc((size_t)N * OM * np, sizeof(double));
    o->rhs_surface_left = xcalloc((size_t)Ns * OM * np, sizeof(double));
    o->rhs_surface_right = xcalloc((size_t)Ns * OM * np, sizeof(double));
    return o;
}

/* Number of boundary faces. */
int64_t or_n_boundary(const oracle_dg *o) { return o->Nb; }

/* Physical points of the boundary faces (Eq. 1dmap): out[Nb][ne][2], faces in
 * element order (element, then local face), points at the edge nodes in the
 * element's counter-clockwise direction. */
int or_boundary_points(const oracle_dg *o, double *out)
{
    for (int64_t s = 0; s < o->Ns; ++s) {
        if (o->bidx[s] < 0) continue;
        const double *v = o->xy + 6 * o->el[s];
        int q = o->eL[s], q1 = (q + 1) % 3;
        for (int k = 0; k < o->ne; ++k) {
            double t = o->ex[k];
            double *p = out + ((size_t)o->bidx[s] * o->ne + k) * 2;
            p[0] = 0.5 * (1.0 - t) * v[2 * q] + 0.5 * (1.0 + t) * v[2 * q1];
            p[1] = 0.5 * (1.0 - t) * v[2 * q + 1] + 0.5 * (1.0 + t) * v[2 * q1 + 1];
        }
    }
    return 0;
}

/* The state prescribed at the boundary points (faces with code -2; the entries
 * of wall faces are not read): u[Nb][ne][M], in or_boundary_points' order. */
int or_set_boundary_state(oracle_dg *o, const double *u)
{
    memcpy(o->bstate, u, sizeof(double) * (size_t)o->Nb * o->ne * OM);
    return 0;
}

int or_info(const oracle_dg *o, int64_t *out)
{
    out[0] = o->N; out[1] = o->np; out[2] = o->nq; out[3] = o->ne; out[4] = o->Ns;
    return 0;
}

/* the volume rule: r, s, w [nq] */
int or_volume_rule(const oracle_dg *o, double *r, double *s, double *w)
{
    memcpy(r, o->vr, sizeof(double) * o->nq);
    memcpy(s, o->vs, sizeof(double) * o->nq);
    memcpy(w, o->vw, sizeof(double) * o->nq);
    return 0;
}

/* Replaces the volume rule by nq points (r, s) with weights w, and the volume
 * tables by the basis evaluated at those points: the symmetric rules of degree
 * 2p of Section 4.3.2 (point counts in Section 6.1) in place of the collapsed
 * grid.  Every volume sum of the solver runs over whatever rule is installed.
 * Returns 0, or 1 on invalid input. */
int or_set_volume_rule(oracle_dg *o, int nq, const double *r, const double *s, const double *w)
{
    if (nq < 1 || nq > 4096) return 1;
    int np = o->np;
    double *vr = xcalloc(nq, sizeof(double)), *vs = xcalloc(nq, sizeof(double)), *vw = xcalloc(nq, sizeof(double));
    double *phi = xcalloc((size_t)nq * np, sizeof(double));
    double *phir = xcalloc((size_t)nq * np, sizeof(double));
    double *phis = xcalloc((size_t)nq * np, sizeof(double));
    long double *rl = xcalloc(nq, sizeof(long double)), *sl = xcalloc(nq, sizeof(long double));
    if (!vr || !vs || !vw || !phi || !phir || !phis || !rl || !sl) {
        free(vr); free(vs); free(vw); free(phi); free(phir); free(phis); free(rl); free(sl);
        return 1;
    }
    for (int k = 0; k < nq; ++k) {
        vr[k] = r[k]; vs[k] = s[k]; vw[k] = w[k];
        rl[k] = r[k]; sl[k] = s[k];
    }
    dubiner_eval_l(o->p, nq, rl, sl, phi, phir, phis);
    free(rl); free(sl);
    free(o->vr); free(o->vs); free(o->vw); free(o->phi); free(o->phir); free(o->phis);
    o->vr = vr; o->vs = vs; o->vw = vw; o->phi = phi; o->phir = phir; o->phis = phis;
    o->nq = nq;
    return 0;
}

/* the volume tables phi, dphi/dr, dphi/ds at the volume points, [nq][np] each */
int or_volume_tables(const oracle_dg *o, double *phi, double *dr, double *ds)
{
    size_t n = (size_t)o->nq * o->np;
    memcpy(phi, o->phi, sizeof(double) * n);
    memcpy(dr, o->phir, sizeof(double) * n);
    memcpy(ds, o->phis, sizeof(double) * n);
    return 0;
}

/* the edge rule: xi, w [ne] */
int or_edge_rule(const oracle_dg *o, double *x, double *w)
{
    memcpy(x, o->ex, sizeof(double) * o->ne);
    memcpy(w, o->ew, sizeof(double) * o->ne);
    return 0;
}

/* edge data: el, er [Ns], eL, eR [Ns], normal nx, ny and full length [Ns] */
int or_edges(const oracle_dg *o, int64_t *el, int64_t *er, int32_t *eL, int32_t *eR,
             double *nx, double *ny, double *len)
{
    for (int64_t s = 0; s < o->Ns; ++s) {
        el[s] = o->el[s]; er[s] = o->er[s]; eL[s] = o->eL[s]; eR[s] = o->eR[s];
        nx[s] = o->enx[s]; ny[s] = o->eny[s]; len[s] = o->elen[s];
    }
    return 0;
}

int or_det_j(const oracle_dg *o, double *out)
{
    memcpy(out, o->detJ, sizeof(double) * o->N);
    return 0;
}

/* physical coordinates of npts reference points on every element: out[N][npts][2] */
int or_map_points(const oracle_dg *o, int npts, const double *r, const double *s, double *out)
{
    for (int64_t e = 0; e < o->N; ++e) {
        const double *v = o->xy + 6 * e;
        for (int k = 0; k < npts; ++k) {
            double l0 = 1.0 - r[k] - s[k];
            out[(e * npts + k) * 2 + 0] = v[0] * l0 + v[2] * r[k] + v[4] * s[k];
            out[(e * npts + k) * 2 + 1] = v[1] * l0 + v[3] * r[k] + v[5] * s[k];
        }
    }
    return 0;
}

int or_volume_points(const oracle_dg *o, double *out)
{
    return or_map_points(o, o->nq, o->vr, o->vs, out);
}

/* U at npts reference points on every element: out[N][npts][M] */
int or_eval_points(const oracle_dg *o, const double *c, int npts, const double *r,
                   const double *s, double *out)
{
    int np = o->np;
    double *phi = (double *)malloc(sizeof(double) * (size_t)npts * np);
    if (!phi || or_dubiner_eval(o->p, npts, r, s, phi, NULL, NULL)) { free(phi); return 1; }
    for (int64_t e = 0; e < o->N; ++e)
        for (int k = 0; k < npts; ++k)
            for (int m = 0; m < OM; ++m) {
                double u = 0.0;
                for (int j = 0; j < np; ++j) u += c[(e * OM + m) * np + j] * phi[k * np + j];
                out[(e * npts + k) * OM + m] = u;
            }
    free(phi);
    return 0;
}

/* L2 projection of point values u[N][nq][M] given at the volume points:
 * c_j = sum_k w_k u(x_k) phi_j(r_k) (orthonormal basis on the reference triangle) */
int or_project(const oracle_dg *o, const double *u, double *c)
{
    int np = o->np, nq = o->nq;
    for (int64_t e = 0; e < o->N; ++e)
        for (int m = 0; m < OM; ++m)
            for (int j = 0; j < np; ++j) {
                double acc = 0.0;
                for (int k = 0; k < nq; ++k)
                    acc += o->vw[k] * u[(e * nq + k) * OM + m] * o->phi[k * np + j];
                c[(e * OM + m) * np + j] = acc;
            }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Euler flux, equation of state, Lax-Friedrichs numerical flux (Eq. euler)  */
/* ------------------------------------------------------------------------- */

static void euler_flux(double g, const double *U, double *F1, double *F2)
{
    double rho = U[0], u = U[1] / rho, v = U[2] / rho, E = U[3];
    double p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    F1[0] = rho * u; F1[1] = rho * u * u + p; F1[2] = rho * u * v; F1[3] = u * (E + p);
    F2[0] = rho * v; F2[1] = rho * u * v; F2[2] = rho * v * v + p; F2[3] = v * (E + p);
}

static double normal_speed(double g, const double *U, double nx, double ny)
{
    double rho = U[0], u = U[1] / rho, v = U[2] / rho, E = U[3];
    double p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    return fabs(u * nx + v * ny) + sqrt(g * p / rho);
}

/* F_n(Ul, Ur) = (F(Ul).n + F(Ur).n)/2 - alpha (Ur - Ul)/2 */
static void lax_friedrichs(double g, const double *Ul, const double *Ur, double nx, double ny, double *Fn)
{
    double F1l[OM], F2l[OM], F1r[OM], F2r[OM];
    euler_flux(g, Ul, F1l, F2l);
    euler_flux(g, Ur, F1r, F2r);
    double al = normal_speed(g, Ul, nx, ny), ar = normal_speed(g, Ur, nx, ny);
    double alpha = al > ar ? al : ar;
    for (int m = 0; m < OM; ++m)
        Fn[m] = 0.5 * ((F1l[m] * nx + F2l[m] * ny) + (F1r[m] * nx + F2r[m] * ny)) - 0.5 * alpha * (Ur[m] - Ul[m]);
}

int or_lax_friedrichs(double g, const double *Ul, const double *Ur, double nx, double ny, double *Fn)
{
    lax_friedrichs(g, Ul, Ur, nx, ny, Fn);
    return 0;
}

int or_euler_flux(double g, const double *U, double *F1, double *F2)
{
    euler_flux(g, U, F1, F2);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Right-hand side of Eq. 2ddg0 in the order of Algorithms 1, 2 and 3        */
/* ------------------------------------------------------------------------- */

/* Algorithm 1: volume integral, one element at a time */
static void eval_volume(oracle_dg *o, const double *C)
{
    int np = o->np, nq = o->nq;
    for (int64_t i = 0; i < o->N; ++i) {
        double *rv = o->rhs_volume + (size_t)i * OM * np;
        for (int t = 0; t < OM * np; ++t) rv[t] = 0.0;
        const double *c = C + (size_t)i * OM * np;
        const double *T = o->JT + 4 * i;
        for (int k = 0; k < nq; ++k) {
            double u[OM], F1[OM], F2[OM];
            for (int m = 0; m < OM; ++m) {
                u[m] = 0.0;
                for (int j = 0; j < np; ++j) u[m] += c[m * np + j] * o->phi[k * np + j];
            }
            euler_flux(o->gamma, u, F1, F2);
            for (int j = 0; j < np; ++j) {
                double dr = o->phir[k * np + j], ds = o->phis[k * np + j];
                /* (det J) times the physical gradient of phi_j */
                double gx = T[0] * dr + T[1] * ds;
                double gy = T[2] * dr + T[3] * ds;
                for (int m = 0; m < OM; ++m)
                    rv[m * np + j] += o->vw[k] * (F1[m] * gx + F2[m] * gy);
            }
        }
    }
}

/* Algorithm 2: surface integral, one edge at a time, with the right element's
 * points traversed in reverse (Eq. edgeint and the reversal k -> ne+1-k) */
/* Ghost state at point k of boundary edge s from the interior trace ul (the
 * paper's eval_boundary, Algorithm 2): a solid wall mirrors the momentum in the
 * wall, U_g = (rho, m - 2 (m.n) n, E); a prescribed boundary takes the caller's
 * state at that point. */
static void ghost_state(const oracle_dg *o, int64_t s, int k, const double *ul, double *ug)
{
    if (o->er[s] == -1) {
        double nx = o->enx[s], ny = o->eny[s];
        double mn = ul[1] * nx + ul[2] * ny;
        ug[0] = ul[0];
        ug[1] = ul[1] - 2.0 * mn * nx;
        ug[2] = ul[2] - 2.0 * mn * ny;
        ug[3] = ul[3];
    } else {
        const double *u = o->bstate + ((size_t)o->bidx[s] * o->ne + k) * OM;
        for (int m = 0; m < OM; ++m) ug[m] = u[m];
    }
}

static void eval_surface(oracle_dg *o, const double *C)
{
    int np = o->np, ne = o->ne;
    for (int64_t s = 0; s < o->Ns; ++s) {
        double *sl = o->rhs_surface_left + (size_t)s * OM * np;
        double *sr = o->rhs_surface_right + (size_t)s * OM * np;
        for (int t = 0; t < OM * np; ++t) { sl[t] = 0.0; sr[t] = 0.0; }
        if (o->er[s] < 0) {
            /* boundary edge: the ghost state takes the right trace's place */
            const double *cl = C + (size_t)o->el[s] * OM * np;
            int L = o->eL[s];
            double len = o->elen[s];
            for (int k = 0; k < ne; ++k) {
                const double *phiL = o->phif + ((size_t)L * ne + k) * np;
                double ul[OM], ug[OM], Fn[OM];
                for (int m = 0; m < OM; ++m) {
                    ul[m] = 0.0;
                    for (int j = 0; j < np; ++j) ul[m] += cl[m * np + j] * phiL[j];
                }
                ghost_state(o, s, k, ul, ug);
                lax_friedrichs(o->gamma, ul, ug, o->enx[s], o->eny[s], Fn);
                for (int m = 0; m < OM; ++m)
                    for (int j = 0; j < np; ++j)
                        sl[m * np + j] -= len * o->ew[k] * Fn[m] * phiL[j] / 2.0;
            }
            continue;
        }
        const double *cl = C + (size_t)o->el[s] * OM * np;
        const double *cr = C + (size_t)o->er[s] * OM * np;
        int L = o->eL[s], R = o->eR[s];
        double len = o->elen[s];
        for (int k = 0; k < ne; ++k) {
            int kr = ne - 1 - k;
            const double *phiL = o->phif + ((size_t)L * ne + k) * np;
            const double *phiR = o->phif + ((size_t)R * ne + kr) * np;
            double ul[OM], ur[OM], Fn[OM];
            for (int m = 0; m < OM; ++m) {
                ul[m] = 0.0; ur[m] = 0.0;
                for (int j = 0; j < np; ++j) {
                    ul[m] += cl[m * np + j] * phiL[j];
                    ur[m] += cr[m * np + j] * phiR[j];
                }
            }
            lax_friedrichs(o->gamma, ul, ur, o->enx[s], o->eny[s], Fn);
            for (int m = 0; m < OM; ++m)
                for (int j = 0; j < np; ++j) {
                    sl[m * np + j] -= len * o->ew[k] * Fn[m] * phiL[j] / 2.0;
                    sr[m * np + j] += len * o->ew[k] * Fn[m] * phiR[j] / 2.0;
                }
        }
    }
}

/* Algorithm 3: combine the volume and the three surface contributions */
static void eval_rhs(oracle_dg *o, double *R)
{
    int np = o->np;
    for (int64_t i = 0; i < o->N; ++i) {
        double *r = R + (size_t)i * OM * np;
        const double *rv = o->rhs_volume + (size_t)i * OM * np;
        double dJ = o->detJ[i];
        for (int t = 0; t < OM * np; ++t) r[t] = rv[t] / dJ;
        for (int q = 0; q < 3; ++q) {
            int64_t s = o->elem_edge[3 * i + q];
            const double *src;
            if (o->el[s] == i && o->eL[s] == q) src = o->rhs_surface_left + (size_t)s * OM * np;
            else src = o->rhs_surface_right + (size_t)s * OM * np;
            for (int t = 0; t < OM * np; ++t) r[t] += src[t] / dJ;
        }
    }
}

int or_rhs(oracle_dg *o, const double *C, double *R)
{
    eval_volume(o, C);
    eval_surface(o, C);
    eval_rhs(o, R);
    return 0;
}

/* The volume part (rhs_volume / det J) of the last or_rhs call: the size of the
 * terms whose difference is the RHS, which sets the RHS's rounding error. */
int or_last_volume_term(const oracle_dg *o, double *out)
{
    int np = o->np;
    for (int64_t i = 0; i < o->N; ++i)
        for (int t = 0; t < OM * np; ++t)
            out[(size_t)i * OM * np + t] = o->rhs_volume[(size_t)i * OM * np + t] / o->detJ[i];
    return 0;
}

/* Barth-Jespersen limiter for p = 1 (Section 4.3.5, Eqs. limit, limitmax,
 * limitmin), variable by variable, in place on C.  The linear approximation is
 * written U_i(r) = Ubar_i + alpha_i grad U_i . (r - r_i) with Ubar_i = U_i(r_i), the
 * value at the centroid r_i.  U^max and U^min are the largest and smallest
 * centroid values of element i and its three neighbours.  At every edge
 * integration point r_{q,k} of element i, with d = U_i(r_{q,k}) - Ubar_i,
 *   alpha_{i,k} = min(1, (U^max - Ubar_i) / d)   if d > 0,
 *               = min(1, (U^min - Ubar_i) / d)   if d < 0,   1 if d = 0,
 * (reading: the paper names the limiter and its bounds; this per-point ratio is
 * the standard Barth-Jespersen one), alpha_i = min_k alpha_{i,k}, and the two
 * linear modes of U_i are multiplied by alpha_i.  Centroid values are taken from
 * the input state; the limiter does not change them (the linear modes vanish
 * at the centroid).  Returns 2 unless p = 1. */
int or_limit_bj(oracle_dg *o, double *C)
{
    if (o->p != 1) return 2;
    const int np = o->np, ne = o->ne;
    const int64_t N = o->N;
    double rc = 1.0 / 3.0, sc = 1.0 / 3.0, cphi[3];
    or_dubiner_eval(1, 1, &rc, &sc, cphi, NULL, NULL);
    double *ubar = malloc(sizeof(double) * (size_t)N * OM);
    if (!ubar) return 1;
    for (int64_t e = 0; e < N; ++e)
        for (int m = 0; m < OM; ++m) {
            const double *c = C + ((size_t)e * OM + m) * np;
            double u = 0.0;
            for (int j = 0; j < np; ++j) u += c[j] * cphi[j];
            ubar[e * OM + m] = u;
        }
    for (int64_t e = 0; e < N; ++e) {
        int64_t nb[3];
        for (int q = 0; q < 3; ++q) {
            int64_t s = o->elem_edge[3 * e + q];
            nb[q] = (o->el[s] == e && o->eL[s] == q) ? o->er[s] : o->el[s];
            if (nb[q] < 0) nb[q] = e;                 /* a boundary face adds no neighbour */
        }
        for (int m = 0; m < OM; ++m) {
            double *c = C + ((size_t)e * OM + m) * np;
            const double ub = ubar[e * OM + m];
            double umax = ub, umin = ub;
            for (int q = 0; q < 3; ++q) {
                double v = ubar[nb[q] * OM + m];
                if (v > umax) umax = v;
                if (v < umin) umin = v;
            }
            double alpha = 1.0;
            for (int q = 0; q < 3; ++q)
                for (int k = 0; k < ne; ++k) {
                    const double *ph = o->phif + ((size_t)q * ne + k) * np;
                    double u = 0.0;
                    for (int j = 0; j < np; ++j) u += c[j] * ph[j];
                    double d = u - ub, a = 1.0;
                    if (d > 0.0) a = fmin(1.0, (umax - ub) / d);
                    else if (d < 0.0) a = fmin(1.0, (umin - ub) / d);
                    if (a < alpha) alpha = a;
                }
            c[1] *= alpha;
            c[2] *= alpha;
        }
    }
    free(ubar);
    return 0;
}

/* Limit every intermediate stage value and the new state of the time steppers
 * below (Section 4.3.1), p = 1 only. */
int or_set_limiter(oracle_dg *o, int on)
{
    if (on && o->p != 1) return 2;
    o->limit = on != 0;
    return 0;
}

static void stage_limit(oracle_dg *o, double *C)
{
    if (o->limit) or_limit_bj(o, C);
}

/* Three-stage SSP Runge-Kutta (Shu-Osher form), nsteps steps in place:
 *   u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1)); u <- 1/3 u + 2/3 (u2 + dt L(u2)) */
int or_ssp_rk3(oracle_dg *o, double *C, double dt, int nsteps)
{
    size_t n = (size_t)o->N * OM * o->np;
    double *u1 = malloc(sizeof(double) * n), *u2 = malloc(sizeof(double) * n), *L = malloc(sizeof(double) * n);
    if (!u1 || !u2 || !L) { free(u1); free(u2); free(L); return 1; }
    for (int it = 0; it < nsteps; ++it) {
        or_rhs(o, C, L);
        for (size_t t = 0; t < n; ++t) u1[t] = C[t] + dt * L[t];
        stage_limit(o, u1);
        or_rhs(o, u1, L);
        for (size_t t = 0; t < n; ++t) u2[t] = 0.75 * C[t] + 0.25 * (u1[t] + dt * L[t]);
        stage_limit(o, u2);
        or_rhs(o, u2, L);
        for (size_t t = 0; t < n; ++t) C[t] = C[t] / 3.0 + 2.0 / 3.0 * (u2[t] + dt * L[t]);
        stage_limit(o, C);
    }
    free(u1); free(u2); free(L);
    return 0;
}

/* The paper's own time integrators (Section 4.3.1, classic explicit Runge-Kutta
 * methods of order two and four), in Butcher form with every stage derivative
 * k_i = L(u + dt sum_j a_ij k_j) kept, nsteps steps in place.
 *   RK2 (reading: Heun's method, c = (0, 1), b = (1/2, 1/2)), taken in its
 *     Shu-Osher form, the convex combination the stage limiting of Section
 *     4.3.1 is applied to (the same method, u + dt/2 (k1 + k2), when nothing
 *     is limited):  u1 = u + dt L(u),  u <- 1/2 u + 1/2 (u1 + dt L(u1))
 *   RK4 (the classical method, c = (0, 1/2, 1/2, 1), b = (1, 2, 2, 1)/6):
 *     k1 = L(u), k2 = L(u + dt/2 k1), k3 = L(u + dt/2 k2), k4 = L(u + dt k3),
 *     u <- u + dt/6 (k1 + 2 k2 + 2 k3 + k4) */
int or_rk2(oracle_dg *o, double *C, double dt, int nsteps)
{
    size_t n = (size_t)o->N * OM * o->np;
    double *u1 = malloc(sizeof(double) * n), *L = malloc(sizeof(double) * n);
    if (!u1 || !L) { free(u1); free(L); return 1; }
    for (int it = 0; it < nsteps; ++it) {
        or_rhs(o, C, L);
        for (size_t t = 0; t < n; ++t) u1[t] = C[t] + dt * L[t];
        stage_limit(o, u1);
        or_rhs(o, u1, L);
        for (size_t t = 0; t < n; ++t) C[t] = 0.5 * C[t] + 0.5 * (u1[t] + dt * L[t]);
        stage_limit(o, C);
    }
    free(u1); free(L);
    return 0;
}

int or_rk4(oracle_dg *o, double *C, double dt, int nsteps)
{
    size_t n = (size_t)o->N * OM * o->np;
    double *y = malloc(sizeof(double) * n), *k[4];
    for (int i = 0; i < 4; ++i) k[i] = malloc(sizeof(double) * n);
    if (!y || !k[0] || !k[1] || !k[2] || !k[3]) {
        free(y); for (int i = 0; i < 4; ++i) free(k[i]);
        return 1;
    }
    static const double a[4] = {0.0, 0.5, 0.5, 1.0};   /* a_{i,i-1}; every other a_ij is 0 */
    for (int it = 0; it < nsteps; ++it) {
        or_rhs(o, C, k[0]);
        for (int i = 1; i < 4; ++i) {
            for (size_t t = 0; t < n; ++t) y[t] = C[t] + a[i] * dt * k[i - 1][t];
            stage_limit(o, y);
            or_rhs(o, y, k[i]);
        }
        for (size_t t = 0; t < n; ++t)
            C[t] = C[t] + dt / 6.0 * (k[0][t] + 2.0 * k[1][t] + 2.0 * k[2][t] + k[3][t]);
        stage_limit(o, C);
    }
    free(y); for (int i = 0; i < 4; ++i) free(k[i]);
    return 0;
}

/* Domain integrals of the conserved variables: sum_i det J_i sum_j c_ijm int phi_j */
int or_totals(const oracle_dg *o, const double *C, double *out)
{
    int np = o->np;
    for (int m = 0; m < OM; ++m) out[m] = 0.0;
    for (int64_t i = 0; i < o->N; ++i)
        for (int m = 0; m < OM; ++m) {
            double s = 0.0;
            for (int j = 0; j < np; ++j) s += C[((size_t)i * OM + m) * np + j] * o->phi_int[j];
            out[m] += o->detJ[i] * s;
        }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Discrete adjoint: transposed Jacobian-vector products of the RHS and of   */
/* one SSP-RK3 step, taken through the forward steps in reverse order.       */
/* Derivative conventions at the kinks of the Lax-Friedrichs flux:           */
/*   d|x|/dx = sign(x) with sign(0) = 0;  d max(a, b) follows a when a >= b  */
/*   (a tie goes to the left trace).                                         */
/* ------------------------------------------------------------------------- */

/* gradients of the pressure and of the sound speed with respect to U */
static void pressure_grad(double g, const double *U, double *p, double *dp)
{
    double rho = U[0], u = U[1] / rho, v = U[2] / rho;
    *p = (g - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v));
    dp[0] = (g - 1.0) * 0.5 * (u * u + v * v);
    dp[1] = -(g - 1.0) * u;
    dp[2] = -(g - 1.0) * v;
    dp[3] = (g - 1.0);
}

/* J[a][b] = d (F(U).n)_a / d U_b for F.n = (rho vn, mx vn + p nx, my vn + p ny, (E+p) vn) */
static void flux_n_jacobian(double g, const double *U, double nx, double ny, double J[OM][OM])
{
    double rho = U[0], vn = (U[1] * nx + U[2] * ny) / rho;
    double dvn[OM] = {-vn / rho, nx / rho, ny / rho, 0.0};
    double p, dp[OM];
    pressure_grad(g, U, &p, dp);
    for (int b = 0; b < OM; ++b) {
        double e0 = b == 0, e1 = b == 1, e2 = b == 2, e3 = b == 3;
        J[0][b] = e0 * vn + rho * dvn[b];
        J[1][b] = e1 * vn + U[1] * dvn[b] + nx * dp[b];
        J[2][b] = e2 * vn + U[2] * dvn[b] + ny * dp[b];
        J[3][b] = (e3 + dp[b]) * vn + (U[3] + p) * dvn[b];
    }
}

/* s(U) = |v.n| + c and its gradient */
static double wave_speed_grad(double g, const double *U, double nx, double ny, double *ds)
{
    double rho = U[0], vn = (U[1] * nx + U[2] * ny) / rho;
    double dvn[OM] = {-vn / rho, nx / rho, ny / rho, 0.0};
    double p, dp[OM];
    pressure_grad(g, U, &p, dp);
    double c = sqrt(g * p / rho);
    double sg = vn > 0.0 ? 1.0 : (vn < 0.0 ? -1.0 : 0.0);
    for (int b = 0; b < OM; ++b) {
        double dc = g / (2.0 * c) * (dp[b] / rho - (b == 0 ? p / (rho * rho) : 0.0));
        ds[b] = sg * dvn[b] + dc;
    }
    return fabs(vn) + c;
}

/* Jacobians of the Lax-Friedrichs flux with respect to its two arguments */
static void lax_friedrichs_jacobians(double g, const double *Ul, const double *Ur, double nx, double ny,
                                     double Jl[OM][OM], double Jr[OM][OM])
{
    double Al[OM][OM], Ar[OM][OM], dsl[OM], dsr[OM];
    flux_n_jacobian(g, Ul, nx, ny, Al);
    flux_n_jacobian(g, Ur, nx, ny, Ar);
    double sl = wave_speed_grad(g, Ul, nx, ny, dsl);
    double sr = wave_speed_grad(g, Ur, nx, ny, dsr);
    double alpha = sl >= sr ? sl : sr;
    int left = sl >= sr;
    for (int a = 0; a < OM; ++a)
        for (int b = 0; b < OM; ++b) {
            double jump = Ur[a] - Ul[a];
            double dal = left ? dsl[b] : 0.0, dar = left ? 0.0 : dsr[b];
            Jl[a][b] = 0.5 * Al[a][b] + (a == b ? 0.5 * alpha : 0.0) - 0.5 * jump * dal;
            Jr[a][b] = 0.5 * Ar[a][b] - (a == b ? 0.5 * alpha : 0.0) - 0.5 * jump * dar;
        }
}

int or_lax_friedrichs_jacobians(double g, const double *Ul, const double *Ur, double nx, double ny,
                                double *Jl, double *Jr)
{
    double A[OM][OM], B[OM][OM];
    lax_friedrichs_jacobians(g, Ul, Ur, nx, ny, A, B);
    memcpy(Jl, A, sizeof A);
    memcpy(Jr, B, sizeof B);
    return 0;
}

int or_flux_jacobian(double g, const double *U, double nx, double ny, double *J)
{
    double A[OM][OM];
    flux_n_jacobian(g, U, nx, ny, A);
    memcpy(J, A, sizeof A);
    return 0;
}

/* out = (dR/dC)^T lam, following Algorithms 3, 2 and 1 backwards */
int or_rhs_vjp(oracle_dg *o, const double *C, const double *lam, double *out)
{
    int np = o->np, nq = o->nq, ne = o->ne;
    size_t n = (size_t)o->N * OM * np;
    for (size_t t = 0; t < n; ++t) out[t] = 0.0;
    /* Algorithm 3 backwards: every contribution to R_i is divided by det J_i */
    double *lb = malloc(sizeof(double) * n);
    if (!lb) return 1;
    for (int64_t i = 0; i < o->N; ++i)
        for (int t = 0; t < OM * np; ++t) lb[(size_t)i * OM * np + t] = lam[(size_t)i * OM * np + t] / o->detJ[i];

    /* Algorithm 2 backwards, edge by edge */
    for (int64_t s = 0; s < o->Ns; ++s) {
        if (o->er[s] < 0) {
            /* boundary edge: F_hat(U_l, U_g(U_l)); a wall's ghost is the reflection
             * U_g = Rf U_l, Rf = diag(1, I - 2 n n^T, 1) (symmetric), so the left
             * trace's cotangent is Jl^T fb + Rf Jr^T fb; a prescribed ghost does not
             * depend on U_l */
            int64_t l = o->el[s];
            const double *cl = C + (size_t)l * OM * np, *bl = lb + (size_t)l * OM * np;
            double *ol = out + (size_t)l * OM * np;
            int L = o->eL[s];
            double len = o->elen[s], nx = o->enx[s], ny = o->eny[s];
            for (int k = 0; k < ne; ++k) {
                const double *phiL = o->phif + ((size_t)L * ne + k) * np;
                double ul[OM], ug[OM], fb[OM];
                for (int m = 0; m < OM; ++m) {
                    ul[m] = 0.0;
                    for (int j = 0; j < np; ++j) ul[m] += cl[m * np + j] * phiL[j];
                }
                ghost_state(o, s, k, ul, ug);
                for (int m = 0; m < OM; ++m) {
                    double a = 0.0;
                    for (int j = 0; j < np; ++j) a += -bl[m * np + j] * len * o->ew[k] * phiL[j] / 2.0;
                    fb[m] = a;
                }
                double Jl[OM][OM], Jr[OM][OM], gl[OM], gr[OM];
                lax_friedrichs_jacobians(o->gamma, ul, ug, nx, ny, Jl, Jr);
                for (int b = 0; b < OM; ++b) {
                    gl[b] = 0.0; gr[b] = 0.0;
                    for (int a = 0; a < OM; ++a) { gl[b] += Jl[a][b] * fb[a]; gr[b] += Jr[a][b] * fb[a]; }
                }
                if (o->er[s] == -1) {
                    double gn = gr[1] * nx + gr[2] * ny;
                    gl[0] += gr[0];
                    gl[1] += gr[1] - 2.0 * gn * nx;
                    gl[2] += gr[2] - 2.0 * gn * ny;
                    gl[3] += gr[3];
                }
                for (int b = 0; b < OM; ++b)
                    for (int j = 0; j < np; ++j) ol[b * np + j] += gl[b] * phiL[j];
            }
            continue;
        }
        int64_t l = o->el[s], r = o->er[s];
        const double *cl = C + (size_t)l * OM * np, *cr = C + (size_t)r * OM * np;
        const double *bl = lb + (size_t)l * OM * np, *br = lb + (size_t)r * OM * np;
        double *ol = out + (size_t)l * OM * np, *orr = out + (size_t)r * OM * np;
        int L = o->eL[s], R = o->eR[s];
        double len = o->elen[s];
        for (int k = 0; k < ne; ++k) {
            int kr = ne - 1 - k;
            const double *phiL = o->phif + ((size_t)L * ne + k) * np;
            const double *phiR = o->phif + ((size_t)R * ne + kr) * np;
            double ul[OM], ur[OM];
            for (int m = 0; m < OM; ++m) {
                ul[m] = 0.0; ur[m] = 0.0;
                for (int j = 0; j < np; ++j) { ul[m] += cl[m * np + j] * phiL[j]; ur[m] += cr[m * np + j] * phiR[j]; }
            }
            /* cotangent of F_n at this point */
            double fb[OM];
            for (int m = 0; m < OM; ++m) {
                double a = 0.0;
                for (int j = 0; j < np; ++j)
                    a += -bl[m * np + j] * len * o->ew[k] * phiL[j] / 2.0 + br[m * np + j] * len * o->ew[k] * phiR[j] / 2.0;
                fb[m] = a;
            }
            double Jl[OM][OM], Jr[OM][OM];
            lax_friedrichs_jacobians(o->gamma, ul, ur, o->enx[s], o->eny[s], Jl, Jr);
            for (int b = 0; b < OM; ++b) {
                double gl = 0.0, gr = 0.0;
                for (int a = 0; a < OM; ++a) { gl += Jl[a][b] * fb[a]; gr += Jr[a][b] * fb[a]; }
                for (int j = 0; j < np; ++j) { ol[b * np + j] += gl * phiL[j]; orr[b * np + j] += gr * phiR[j]; }
            }
        }
    }

    /* Algorithm 1 backwards, element by element */
    for (int64_t i = 0; i < o->N; ++i) {
        const double *c = C + (size_t)i * OM * np;
        const double *bi = lb + (size_t)i * OM * np;
        double *oi = out + (size_t)i * OM * np;
        const double *T = o->JT + 4 * i;
        for (int k = 0; k < nq; ++k) {
            double u[OM];
            for (int m = 0; m < OM; ++m) {
                u[m] = 0.0;
                for (int j = 0; j < np; ++j) u[m] += c[m * np + j] * o->phi[k * np + j];
            }
            double a1[OM] = {0}, a2[OM] = {0};
            for (int j = 0; j < np; ++j) {
                double dr = o->phir[k * np + j], ds = o->phis[k * np + j];
                double gx = T[0] * dr + T[1] * ds, gy = T[2] * dr + T[3] * ds;
                for (int m = 0; m < OM; ++m) { a1[m] += bi[m * np + j] * gx; a2[m] += bi[m * np + j] * gy; }
            }
            double A1[OM][OM], A2[OM][OM];
            flux_n_jacobian(o->gamma, u, 1.0, 0.0, A1);
            flux_n_jacobian(o->gamma, u, 0.0, 1.0, A2);
            for (int b = 0; b < OM; ++b) {
                double ub = 0.0;
                for (int a = 0; a < OM; ++a) ub += A1[a][b] * a1[a] + A2[a][b] * a2[a];
                ub *= o->vw[k];
                for (int j = 0; j < np; ++j) oi[b * np + j] += ub * o->phi[k * np + j];
            }
        }
    }
    free(lb);
    return 0;
}

/* lam_n = (d C_{n+1} / d C_n)^T lam_np1 for one SSP-RK3 step from C_n */
int or_ssp_rk3_vjp(oracle_dg *o, const double *Cn, double dt, const double *lam_np1, double *lam_n)
{
    size_t n = (size_t)o->N * OM * o->np;
    double *u1 = malloc(sizeof(double) * n), *u2 = malloc(sizeof(double) * n);
    double *L = malloc(sizeof(double) * n), *b2 = malloc(sizeof(double) * n);
    double *b1 = malloc(sizeof(double) * n), *t = malloc(sizeof(double) * n);
    if (!u1 || !u2 || !L || !b2 || !b1 || !t) { free(u1); free(u2); free(L); free(b2); free(b1); free(t); return 1; }
    /* forward stages */
    or_rhs(o, Cn, L);
    for (size_t i = 0; i < n; ++i) u1[i] = Cn[i] + dt * L[i];
    or_rhs(o, u1, L);
    for (size_t i = 0; i < n; ++i) u2[i] = 0.75 * Cn[i] + 0.25 * (u1[i] + dt * L[i]);
    /* C_{n+1} = 1/3 C_n + 2/3 (u2 + dt R(u2)) */
    or_rhs_vjp(o, u2, lam_np1, t);
    for (size_t i = 0; i < n; ++i) b2[i] = 2.0 / 3.0 * (lam_np1[i] + dt * t[i]);
    /* u2 = 3/4 C_n + 1/4 (u1 + dt R(u1)) */
    or_rhs_vjp(o, u1, b2, t);
    for (size_t i = 0; i < n; ++i) b1[i] = 0.25 * (b2[i] + dt * t[i]);
    /* u1 = C_n + dt R(C_n) */
    or_rhs_vjp(o, Cn, b1, t);
    for (size_t i = 0; i < n; ++i) lam_n[i] = lam_np1[i] / 3.0 + 0.75 * b2[i] + b1[i] + dt * t[i];
    free(u1); free(u2); free(L); free(b2); free(b1); free(t);
    return 0;
}

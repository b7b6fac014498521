/*
 * bcmg_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU reference ("the oracle") of the
 * ghost-point Boundary Condition MultiGrid (BCMG) method of Coco, Mazza and
 * Semplice, "A ghost-point smoothing strategy for geometric multigrid on
 * curved boundaries" (arXiv 2207.14208).  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline / reference legs may load it.  It
 * shares no code, header, table or helper with the CUDA library: every rule
 * below is written out here from the paper (and from the readings of the
 * places where the paper is silent, which are listed next to each rule).
 *
 * Grid (Sec. 2 / Sec. 3 set-up): D = [-1,1]^d, N cells per axis, n = N+1
 * nodes per axis, x_i = -1 + i h, h = 2/N, arrays x-fastest with n^d entries,
 * linear index i + n*j + n*n*k.  d = 1, 2 or 3.
 *
 * Node classes (Sec. 3.3): Omega = {phi < 0}.
 *   INTERIOR : phi < 0 and not on the box boundary (an unknown of -Lap u = f)
 *   BOXDIR   : phi < 0 on the box boundary; an eliminated Dirichlet node whose
 *              value is carried in u (Sec. 3, problem mainProblem2D, Gamma_B)
 *   GHOST    : phi >= 0 with at least one of its 2d axis neighbours INTERIOR
 *   INACTIVE : everything else
 *
 * Boundary condition on Gamma (Sec. 3, operator B of the problem statement):
 *   Dirichlet (bc = 0): B u = u(Q), the tensor Lagrange interpolant of u on
 *              the ghost stencil evaluated at Q (eq. BCh);
 *   Neumann   (bc = 1): B u = grad u(Q) . n, the normal derivative of the same
 *              interpolant at Q (Sec. 3.2.2 in 1D/2D, Sec. 4.1 in 3D), with n
 *              the unit normal computed at G; its relaxation step is
 *              Delta tau = h * (Delta tau / h)_OPT (eqs. dtauoptLFA_Neumann,
 *              dtauoptLFA3D_Neumann).
 * Interior equation: c u - Lap_h u = f with reaction coefficient c >= 0
 * (c = 0: Poisson; c = 1: the reaction-diffusion problem of Test2N, Sec. 4.2).
 *
 * Parity unpinned (no printed value in the paper fixes them; they are pinned
 * only by the convergence and accuracy tests): the band extension (number of
 * sweeps, upwind form), the coarse-level stencil fall-backs and the root
 * finder that places the projection point Q.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXL 24

enum { CL_INACTIVE = 0, CL_INTERIOR = 1, CL_GHOST = 2, CL_BOXDIR = 3 };
enum { ORD_RB = 0, ORD_LEX = 1, ORD_BLOCK = 2 };
enum { DT_EXP = 0, DT_POLY = 1, DT_CONST = 2 };
enum { CYC_V = 0, CYC_TGCS = 1, CYC_W = 2 };

typedef struct {
    int d, N, n;
    long nn, st[3];
    double h;
    int bc;       /* 0 Dirichlet, 1 Neumann on Gamma */
    double react; /* reaction coefficient c of c u - Lap u = f */
    double *phi;
    unsigned char *cls;
    long nint, nbox;
    /* ghost points */
    long ng, nclamp, nfall;
    long *gidx;
    double *geta, *gn, *gxi, *gdt, *gQ; /* gn, gxi, gQ: 3 per ghost */
    int *gs, *gq;                       /* 3 per ghost */
    /* inactive band that receives the normal extension */
    long nb;
    long *bidx, *bup; /* bup: 3 per band node, -1 = no upwind source on axis */
    double *bw;       /* 3 per band node: |d phi / d x_a| */
    int *bpos;        /* nn entries: band position or -1 */
    /* per-level arrays (u is the correction e on coarse levels) */
    double *u, *F, *r, *tmp;
    /* dense direct solver (coarsest level only) */
    long nact;
    long *act;
    int *apos;
    double *LU;
    long *piv;
    int direct_ok;
} olevel;

typedef struct {
    int d, N, L;
    int nu1, nu2, ordering, dtau_mode, ext_sweeps, cycle, min_coarse, max_levels;
    int tgcs_maxit, rmode, ext_mode;
    int bc;
    int band_width;  /* Chebyshev radius of the extension band (default 2) */
    int gfam;        /* coarse-ghost family: 0 ghost + inactive, 1 ghost only */
    int cg_rhs;      /* coarse-ghost right-hand side: 0 family restriction,
                        1 the (extended) fine residual at the coincident node */
    double react;
    double ext_cfl;
    double dtau_const, tgcs_tol;
    long block_sweeps_last;
    olevel lv[ORC_MAXL];
} oracle_t;

/* ------------------------------------------------------------------ */
/* small helpers                                                        */
/* ------------------------------------------------------------------ */

static void decode(const olevel *L, long lin, int ix[3]) {
    ix[0] = ix[1] = ix[2] = 0;
    for (int a = 0; a < L->d; ++a) {
        ix[a] = (int)(lin % L->n);
        lin /= L->n;
    }
}

static int in_grid(const olevel *L, const int ix[3]) {
    for (int a = 0; a < L->d; ++a)
        if (ix[a] < 0 || ix[a] > L->N) return 0;
    return 1;
}

static long lin_of(const olevel *L, const int ix[3]) {
    long s = 0;
    for (int a = 0; a < L->d; ++a) s += (long)ix[a] * L->st[a];
    return s;
}

/* 1D Lagrange basis on the local nodes 0, 1, .., q evaluated at xi
 * (Sec. 2, BC1D: the Dirichlet coefficients (c_0, c_-1, c_-2) for s = 3 are
 * these values at xi = theta).  q = 2: quadratic, q = 1: linear, q = 0: 1. */
static void lagrange(int q, double xi, double w[3]) {
    w[0] = w[1] = w[2] = 0.0;
    if (q == 2) {
        w[0] = (1.0 - xi) * (2.0 - xi) / 2.0;
        w[1] = xi * (2.0 - xi);
        w[2] = xi * (xi - 1.0) / 2.0;
    } else if (q == 1) {
        w[0] = 1.0 - xi;
        w[1] = xi;
    } else {
        w[0] = 1.0;
    }
}

/* derivatives d/dxi of the same basis (the Neumann rows of Sec. 3.2.2: at
 * xi = theta they give -(c_0, c_-1, c_-2) of eq. coeffN) */
static void lagrange_d(int q, double xi, double w[3]) {
    w[0] = w[1] = w[2] = 0.0;
    if (q == 2) {
        w[0] = xi - 1.5;
        w[1] = 2.0 - 2.0 * xi;
        w[2] = xi - 0.5;
    } else if (q == 1) {
        w[0] = -1.0;
        w[1] = 1.0;
    }
}

/* ------------------------------------------------------------------ */
/* BLFA closed forms (Sec. 3.2.1, 3.2.2, 4.1 and Remark exptheta2D)     */
/* ------------------------------------------------------------------ */

/* p(alpha_1..alpha_{d-1}) = acosh(d - sum cos alpha_i)  (eqs. alphaNalpha,
 * alphaNalpha3D and the d-dimensional remark of Sec. 4.1). */
double orc_blfa_p(int d, const double *alpha) {
    double s = (double)d;
    for (int i = 0; i < d - 1; ++i) s -= cos(alpha[i]);
    return acosh(s);
}

/* G0 for a given p and theta.
 * bc = 0 Dirichlet: poly form eq. G with coefficients eq. coeff,
 *                   exp form exp(-p theta)          (Remark exptheta2D)
 * bc = 1 Neumann:   poly form eq. GN with coefficients eq. coeffN,
 *                   exp form p exp(-p theta)        (Remark exptheta2D)
 * form = 0 exp, 1 poly.  Neumann values are G0 without the 1/h factor. */
double orc_blfa_G0(int bc, int form, double p, double theta) {
    double e1 = exp(-p), e2 = exp(-2.0 * p);
    if (bc == 0) {
        if (form == 0) return exp(-p * theta);
        double cm2 = theta * (theta - 1.0) / 2.0;
        double cm1 = theta * (2.0 - theta);
        double c0 = (1.0 - theta) * (2.0 - theta) / 2.0;
        return cm2 * e2 + cm1 * e1 + c0;
    }
    if (form == 0) return p * exp(-p * theta);
    {
        double cm2 = 0.5 - theta;
        double cm1 = 2.0 * (theta - 1.0);
        double c0 = 1.5 - theta;
        return cm2 * e2 + cm1 * e1 + c0;
    }
}

/* Delta tau_OPT(theta) = 2 / (G0min + G0max) over the corner frequencies
 * A_1 = (pi/2, 0, .., 0), .., A_{d-1} = (pi/2, .., pi/2), A_d = (pi, .., pi)
 * (Prop. 1 eq. dtauoptLFA for d = 2, Prop. 3 eqs. dtauoptLFA3D/G0minmax for
 * d = 3, eq. G0minmax_dD in general; Neumann Props. 2 and 4 give Dtau/h).
 * mode: 0 exp form of G0, 1 poly form, 2 constant.  For d = 1 there is no
 * tangential frequency; the single point has p = acosh(1) = 0. */
double orc_dtau(int d, int bc, int mode, double cst, double theta) {
    if (mode == DT_CONST) return cst;
    double gmin = INFINITY, gmax = 0.0;
    for (int m = 1; m <= d; ++m) {
        double al[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < d - 1; ++i) {
            if (m == d) al[i] = M_PI;
            else if (i < m) al[i] = M_PI / 2.0;
            else al[i] = 0.0;
        }
        double p = orc_blfa_p(d, al);
        double g = fabs(orc_blfa_G0(bc, mode == DT_EXP ? 0 : 1, p, theta));
        if (g < gmin) gmin = g;
        if (g > gmax) gmax = g;
    }
    return 2.0 / (gmin + gmax);
}

/* ------------------------------------------------------------------ */
/* geometry: classification, ghost projection, stencil, band (Sec. 3.3)  */
/* ------------------------------------------------------------------ */

static void classify(olevel *L) {
    L->nint = L->nbox = 0;
    for (long lin = 0; lin < L->nn; ++lin) {
        int ix[3];
        decode(L, lin, ix);
        int edge = 0;
        for (int a = 0; a < L->d; ++a)
            if (ix[a] == 0 || ix[a] == L->N) edge = 1;
        if (L->phi[lin] < 0.0) {
            L->cls[lin] = edge ? CL_BOXDIR : CL_INTERIOR;
            if (edge) L->nbox++;
            else L->nint++;
        } else {
            L->cls[lin] = CL_INACTIVE;
        }
    }
    /* Gamma_h: outside nodes with an interior 2d-neighbour */
    for (long lin = 0; lin < L->nn; ++lin) {
        if (L->phi[lin] < 0.0) continue;
        int ix[3];
        decode(L, lin, ix);
        int ghost = 0;
        for (int a = 0; a < L->d && !ghost; ++a)
            for (int dir = -1; dir <= 1; dir += 2) {
                int iy[3] = {ix[0], ix[1], ix[2]};
                iy[a] += dir;
                if (!in_grid(L, iy)) continue;
                if (L->cls[lin_of(L, iy)] == CL_INTERIOR) ghost = 1;
            }
        if (ghost) L->cls[lin] = CL_GHOST;
    }
}

/* phi gradient component in index units: central difference, one-sided on
 * the box boundary ("finite-difference discretization centered at the ghost
 * point", Sec. 3.3). */
static double grad_a(const olevel *L, long lin, const int ix[3], int a) {
    long s = L->st[a];
    if (ix[a] == 0) return L->phi[lin + s] - L->phi[lin];
    if (ix[a] == L->N) return L->phi[lin] - L->phi[lin - s];
    return 0.5 * (L->phi[lin + s] - L->phi[lin - s]);
}

/* multilinear interpolation of grid phi at index-space point p */
static double interp_phi(const olevel *L, const double p[3]) {
    long c[3] = {0, 0, 0};
    double t[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < L->d; ++a) {
        double f = floor(p[a]);
        long ci = (long)f;
        if (ci < 0) ci = 0;
        if (ci > L->N - 1) ci = L->N - 1;
        c[a] = ci;
        t[a] = p[a] - (double)ci;
    }
    double val = 0.0;
    for (int corner = 0; corner < (1 << L->d); ++corner) {
        double w = 1.0;
        long idx = 0;
        for (int a = 0; a < L->d; ++a) {
            int b = (corner >> a) & 1;
            w *= b ? t[a] : (1.0 - t[a]);
            idx += (c[a] + b) * L->st[a];
        }
        val += w * L->phi[idx];
    }
    return val;
}

/* Is every node of the tensor stencil {X - sum_a s_a o_a e_a, 0<=o_a<=q_a}
 * usable (i.e. not INACTIVE)? */
static int stencil_ok(const olevel *L, const int ix[3], const int s[3], const int q[3]) {
    int o[3];
    for (o[2] = 0; o[2] <= (L->d > 2 ? q[2] : 0); ++o[2])
        for (o[1] = 0; o[1] <= (L->d > 1 ? q[1] : 0); ++o[1])
            for (o[0] = 0; o[0] <= q[0]; ++o[0]) {
                int iy[3];
                for (int a = 0; a < 3; ++a) iy[a] = ix[a] - (a < L->d ? s[a] * o[a] : 0);
                if (!in_grid(L, iy)) return 0;
                if (L->cls[lin_of(L, iy)] == CL_INACTIVE) return 0;
            }
    return 1;
}

static void setup_ghosts(oracle_t *O, olevel *L) {
    int d = L->d;
    L->ng = 0;
    for (long lin = 0; lin < L->nn; ++lin)
        if (L->cls[lin] == CL_GHOST) L->ng++;
    long ng = L->ng;
    L->gidx = (long *)calloc(ng + 1, sizeof(long));
    L->geta = (double *)calloc(ng + 1, sizeof(double));
    L->gdt = (double *)calloc(ng + 1, sizeof(double));
    L->gn = (double *)calloc(3 * ng + 3, sizeof(double));
    L->gxi = (double *)calloc(3 * ng + 3, sizeof(double));
    L->gQ = (double *)calloc(3 * ng + 3, sizeof(double));
    L->gs = (int *)calloc(3 * ng + 3, sizeof(int));
    L->gq = (int *)calloc(3 * ng + 3, sizeof(int));
    L->nclamp = L->nfall = 0;
    long g = 0;
    for (long lin = 0; lin < L->nn; ++lin) {
        if (L->cls[lin] != CL_GHOST) continue;
        int ix[3];
        decode(L, lin, ix);
        /* outward normal n = grad phi / |grad phi| */
        double gr[3] = {0.0, 0.0, 0.0}, n[3] = {0.0, 0.0, 0.0}, key[3] = {0.0, 0.0, 0.0};
        double gn2 = 0.0;
        for (int a = 0; a < d; ++a) {
            gr[a] = grad_a(L, lin, ix, a);
            gn2 += gr[a] * gr[a];
        }
        if (gn2 > 0.0) {
            double gnorm = sqrt(gn2);
            for (int a = 0; a < d; ++a) {
                n[a] = gr[a] / gnorm;
                key[a] = fabs(gr[a]);
            }
        } else {
            /* flat phi: point away from the first interior axis neighbour */
            int done = 0;
            for (int a = 0; a < d && !done; ++a)
                for (int dir = -1; dir <= 1 && !done; dir += 2) {
                    int iy[3] = {ix[0], ix[1], ix[2]};
                    iy[a] += dir;
                    if (in_grid(L, iy) && L->cls[lin_of(L, iy)] == CL_INTERIOR) {
                        n[a] = (double)(-dir);
                        done = 1;
                    }
                }
            for (int a = 0; a < d; ++a) key[a] = fabs(n[a]);
        }
        /* projection Q = G - eta h n with phi(Q) = 0, eta in [0, 1]: bisection
         * on the multilinear interpolant of grid phi (Sec. 3.3). */
        double eta;
        if (L->phi[lin] == 0.0) {
            eta = 0.0;
        } else {
            double p1[3];
            for (int a = 0; a < 3; ++a) p1[a] = (double)ix[a] - (a < d ? n[a] : 0.0);
            if (interp_phi(L, p1) >= 0.0) {
                eta = 1.0;
                L->nclamp++;
            } else {
                double lo = 0.0, hi = 1.0;
                for (int it = 0; it < 64; ++it) {
                    double mid = 0.5 * (lo + hi), pm[3];
                    for (int a = 0; a < 3; ++a) pm[a] = (double)ix[a] - (a < d ? mid * n[a] : 0.0);
                    if (interp_phi(L, pm) >= 0.0) lo = mid;
                    else hi = mid;
                }
                eta = 0.5 * (lo + hi);
            }
        }
        /* upwind 3^d stencil with G at a corner (Sec. 3.3): along axis a the
         * nodes G, G - s_a e_a, G - 2 s_a e_a with s_a = sign(n_a) (+1 for
         * n_a = 0), reversed if it would leave the grid. */
        int s[3] = {1, 1, 1}, q[3] = {0, 0, 0};
        double xi[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < d; ++a) {
            s[a] = (n[a] >= 0.0) ? 1 : -1;
            int far = ix[a] - 2 * s[a];
            if (far < 0 || far > L->N) s[a] = -s[a];
            xi[a] = (double)s[a] * eta * n[a];
            q[a] = 2;
        }
        /* fall-back when the stencil meets an inactive node (thin features,
         * coarse levels; the paper assumes a fine enough grid).  Axes are
         * visited by increasing |n_a| (ties by axis index); each axis steps
         * through (reversed direction, degree 2), (upwind, 1), (reversed, 1),
         * (upwind, 0), keeping the last option if the stencil still fails,
         * until the stencil has no inactive node.  A reversed direction is
         * skipped if it would leave the grid. */
        if (!stencil_ok(L, ix, s, q)) {
            int order[3] = {0, 1, 2};
            for (int i = 1; i < d; ++i) /* stable insertion sort by key */
                for (int j = i; j > 0 && key[order[j]] < key[order[j - 1]]; --j) {
                    int t = order[j];
                    order[j] = order[j - 1];
                    order[j - 1] = t;
                }
            static const int opt_flip[4] = {1, 0, 1, 0};
            static const int opt_deg[4] = {2, 1, 1, 0};
            int ok = 0;
            for (int m = 0; m < d && !ok; ++m) {
                int a = order[m];
                int s0 = s[a];
                for (int o = 0; o < 4 && !ok; ++o) {
                    int sa = opt_flip[o] ? -s0 : s0;
                    int far = ix[a] - sa * opt_deg[o];
                    if (far < 0 || far > L->N) continue;
                    s[a] = sa;
                    q[a] = opt_deg[o];
                    ok = stencil_ok(L, ix, s, q);
                }
                if (!ok) {
                    s[a] = s0;
                    q[a] = 0;
                }
            }
            for (int a = 0; a < d; ++a) xi[a] = (double)s[a] * eta * n[a];
            L->nfall++;
        }
        L->gidx[g] = lin;
        L->geta[g] = eta;
        for (int a = 0; a < d; ++a) {
            L->gn[3 * g + a] = n[a];
            L->gxi[3 * g + a] = xi[a];
            L->gs[3 * g + a] = s[a];
            L->gq[3 * g + a] = q[a];
            L->gQ[3 * g + a] = (-1.0 + ix[a] * L->h) - eta * L->h * n[a];
        }
        /* Delta tau = Delta tau_OPT(theta~), theta~ = |G - Q| / h = eta
         * (eq. DtauOptTheta; exp form of G0 by Remark exptheta2D). */
        L->gdt[g] = orc_dtau(d, O->bc, O->dtau_mode, O->dtau_const, eta);
        if (O->bc == 1) L->gdt[g] *= L->h; /* Neumann: the formulas give Dtau / h */
        ++g;
    }
}

/* inactive nodes within Chebyshev distance rad (2 by default: exactly the
 * inactive points a coarse-ghost restriction can read) of a ghost receive the
 * normal extension of ghost quantities (Sec. 3.3.2, transfer operators). */
static void setup_band(olevel *L, int rad) {
    int d = L->d;
    L->bpos = (int *)malloc(sizeof(int) * (size_t)L->nn);
    for (long i = 0; i < L->nn; ++i) L->bpos[i] = -1;
    unsigned char *mark = (unsigned char *)calloc((size_t)L->nn, 1);
    for (long g = 0; g < L->ng; ++g) {
        int ix[3];
        decode(L, L->gidx[g], ix);
        int o[3];
        for (o[2] = (d > 2 ? -rad : 0); o[2] <= (d > 2 ? rad : 0); ++o[2])
            for (o[1] = (d > 1 ? -rad : 0); o[1] <= (d > 1 ? rad : 0); ++o[1])
                for (o[0] = -rad; o[0] <= rad; ++o[0]) {
                    int iy[3] = {ix[0] + o[0], ix[1] + o[1], ix[2] + o[2]};
                    if (!in_grid(L, iy)) continue;
                    long y = lin_of(L, iy);
                    if (L->cls[y] == CL_INACTIVE) mark[y] = 1;
                }
    }
    L->nb = 0;
    for (long i = 0; i < L->nn; ++i)
        if (mark[i]) L->nb++;
    L->bidx = (long *)calloc(L->nb + 1, sizeof(long));
    L->bup = (long *)calloc(3 * L->nb + 3, sizeof(long));
    L->bw = (double *)calloc(3 * L->nb + 3, sizeof(double));
    long b = 0;
    for (long i = 0; i < L->nn; ++i)
        if (mark[i]) {
            L->bidx[b] = i;
            L->bpos[i] = (int)b;
            ++b;
        }
    for (b = 0; b < L->nb; ++b) {
        long lin = L->bidx[b];
        int ix[3];
        decode(L, lin, ix);
        for (int a = 0; a < 3; ++a) {
            L->bup[3 * b + a] = -1;
            L->bw[3 * b + a] = 0.0;
        }
        for (int a = 0; a < d; ++a) {
            double ga = grad_a(L, lin, ix, a);
            if (ga == 0.0) continue;
            int s = ga > 0.0 ? 1 : -1;
            int iy[3] = {ix[0], ix[1], ix[2]};
            iy[a] -= s; /* upwind = towards the domain */
            if (!in_grid(L, iy)) continue;
            long y = lin_of(L, iy);
            if (L->cls[y] == CL_GHOST || mark[y]) {
                L->bup[3 * b + a] = y;
                L->bw[3 * b + a] = fabs(ga);
            }
        }
    }
    free(mark);
}

/* ------------------------------------------------------------------ */
/* operators                                                            */
/* ------------------------------------------------------------------ */

/* Per-ghost basis values w[a][o] = L_o(xi_a) and derivatives dw[a][o] =
 * L_o'(xi_a) on the stencil ST_G = {X - sum_a s_a o_a e_a, 0 <= o_a <= q_a}. */
typedef struct {
    int q[3], s[3];
    double w[3][3], dw[3][3], n[3];
} gstencil;

static void ghost_stencil(const olevel *L, long g, gstencil *S) {
    for (int a = 0; a < 3; ++a) {
        S->q[a] = 0;
        S->s[a] = 0;
        S->n[a] = 0.0;
        S->w[a][0] = 1.0;
        S->w[a][1] = S->w[a][2] = 0.0;
        S->dw[a][0] = S->dw[a][1] = S->dw[a][2] = 0.0;
    }
    for (int a = 0; a < L->d; ++a) {
        S->q[a] = L->gq[3 * g + a];
        S->s[a] = L->gs[3 * g + a];
        S->n[a] = L->gn[3 * g + a];
        lagrange(S->q[a], L->gxi[3 * g + a], S->w[a]);
        lagrange_d(S->q[a], L->gxi[3 * g + a], S->dw[a]);
    }
}

/* weight of stencil node (o0, o1, o2) in the ghost row.  Dirichlet: the
 * tensor Lagrange weight.  Neumann: sum_a n_a d/dx_a of it; with the local
 * coordinate t_a = -s_a (x_a - x_G,a) / h of the stencil axis, d/dx_a =
 * (-s_a / h) d/dt_a, evaluated at t = xi (the position of Q). */
static double ghost_weight(const olevel *L, const gstencil *S, int o0, int o1, int o2) {
    const int o[3] = {o0, o1, o2};
    if (L->bc == 0) return S->w[0][o0] * S->w[1][o1] * S->w[2][o2];
    double v = 0.0;
    for (int a = 0; a < L->d; ++a) {
        double t = S->n[a] * (-(double)S->s[a] / L->h) * S->dw[a][o[a]];
        for (int b = 0; b < L->d; ++b)
            if (b != a) t *= S->w[b][o[b]];
        v += t;
    }
    return v;
}

/* B u~ at ghost g: the boundary operator of the ghost row applied to the
 * (tri/bi)quadratic interpolant of u on ST_G at Q (eq. BCh), i.e.
 * sum_k w_k u_k with the row's weights. */
static double ghost_apply(const olevel *L, long g, const double *u) {
    gstencil S;
    ghost_stencil(L, g, &S);
    long X = L->gidx[g];
    double B = 0.0;
    for (int o2 = 0; o2 <= S.q[2]; ++o2)
        for (int o1 = 0; o1 <= S.q[1]; ++o1)
            for (int o0 = 0; o0 <= S.q[0]; ++o0) {
                long Y = X - (long)S.s[0] * o0 * L->st[0] - (long)S.s[1] * o1 * L->st[1] -
                         (long)S.s[2] * o2 * L->st[2];
                B += ghost_weight(L, &S, o0, o1, o2) * u[Y];
            }
    return B;
}

/* sum of the 2d axis neighbours */
static double nbr_sum(const olevel *L, long lin, const double *u) {
    double s = 0.0;
    for (int a = 0; a < L->d; ++a) s += u[lin - L->st[a]] + u[lin + L->st[a]];
    return s;
}

/* Fictitious-time relaxation of every ghost (eqs. relghostdt, relax2DV, rel):
 * u_G <- u_G + dtau_G (F_G - B u~), all ghosts from the same u (the ghost
 * block of P is diag(1/dtau), eq. 2Ddiri:P, so ghosts do not see each
 * other's new values within a sweep). */
static void ghost_relax(olevel *L, double *u, const double *F) {
    for (long g = 0; g < L->ng; ++g) {
        long X = L->gidx[g];
        L->tmp[g] = u[X] + L->gdt[g] * (F[X] - ghost_apply(L, g, u));
    }
    for (long g = 0; g < L->ng; ++g) u[L->gidx[g]] = L->tmp[g];
}

static int parity(const olevel *L, long lin) {
    int ix[3];
    decode(L, lin, ix);
    return (ix[0] + ix[1] + ix[2]) & 1;
}

/* Gauss-Seidel on the 5/7-point equations (eq. GSLEX_2D, eq. Laph) of
 * c u - Lap_h u = f: u_X = (sum nbrs + h^2 F_X) / (2d + c h^2); ghost
 * neighbours hold their old values. */
static void interior_update(olevel *L, long lin, double *u, const double *F) {
    u[lin] = (nbr_sum(L, lin, u) + L->h * L->h * F[lin]) / (2.0 * L->d + L->react * L->h * L->h);
}

static void interior_lex(olevel *L, double *u, const double *F) {
    for (long lin = 0; lin < L->nn; ++lin)
        if (L->cls[lin] == CL_INTERIOR) interior_update(L, lin, u, F);
}

static void interior_rb(olevel *L, double *u, const double *F) {
    for (int c = 0; c < 2; ++c)
        for (long lin = 0; lin < L->nn; ++lin)
            if (L->cls[lin] == CL_INTERIOR && parity(L, lin) == c) interior_update(L, lin, u, F);
}

/* REL-BC (eq. 2Ddiri:Pbc): the interior block solved exactly for the current
 * ghost values, here by GS-LEX sweeps run to convergence. */
static long interior_block(olevel *L, double *u, const double *F) {
    long sweeps = 0;
    for (; sweeps < 200000; ++sweeps) {
        double dmax = 0.0, umax = 0.0;
        for (long lin = 0; lin < L->nn; ++lin) {
            if (L->cls[lin] != CL_INTERIOR) continue;
            double old = u[lin];
            interior_update(L, lin, u, F);
            double dd = fabs(u[lin] - old);
            if (dd > dmax) dmax = dd;
            if (fabs(u[lin]) > umax) umax = fabs(u[lin]);
        }
        if (dmax <= 1e-17 * (umax > 1e-300 ? umax : 1e-300) || dmax == 0.0) break;
    }
    return sweeps + 1;
}

/* one smoothing step: interior sweep(s) then the ghost relaxation (block
 * lower-triangular P of eq. 2Ddiri:P). */
static void smooth_step(oracle_t *O, olevel *L, double *u, const double *F) {
    if (O->ordering == ORD_RB) interior_rb(L, u, F);
    else if (O->ordering == ORD_LEX) interior_lex(L, u, F);
    else O->block_sweeps_last = interior_block(L, u, F);
    ghost_relax(L, u, F);
}

/* residual r = F - A u on interior (eq. Laph) and ghost (eq. BCh) rows; zero
 * on every other node. */
static void residual(const olevel *L, const double *u, const double *F, double *r) {
    double h2 = L->h * L->h;
    for (long lin = 0; lin < L->nn; ++lin) r[lin] = 0.0;
    for (long lin = 0; lin < L->nn; ++lin)
        if (L->cls[lin] == CL_INTERIOR)
            r[lin] = F[lin] - ((2.0 * L->d + L->react * h2) * u[lin] - nbr_sum(L, lin, u)) / h2;
    for (long g = 0; g < L->ng; ++g) {
        long X = L->gidx[g];
        r[X] = F[X] - ghost_apply(L, g, u);
    }
}

/* The paper's own scheme for the extension (Sec. 3.3.2): explicit Euler in
 * the pseudo-time sigma for dr/dsigma + dr/dn = 0 with the normal derivative
 * dr/dn = sum_a n_a (r(X + e_a) - r(X - e_a)) / 2 taken by central differences
 * (index units), step ext_cfl, over the band nodes only; ghost and interior
 * values act as fixed data, the band starts from zero.  Kept as an option
 * (ext_mode = 1): forward Euler with central differences is not stable for
 * pure advection, so the default is the upwind scheme below. */
static void extend_central(const oracle_t *O, olevel *L, double *arr) {
    long nb = L->nb;
    double *old = L->tmp, *nw = L->tmp + nb;
    for (long b = 0; b < nb; ++b) old[b] = 0.0;
    for (long b = 0; b < nb; ++b) arr[L->bidx[b]] = 0.0;
    for (int k = 0; k < O->ext_sweeps; ++k) {
        for (long b = 0; b < nb; ++b) {
            long X = L->bidx[b];
            int ix[3];
            decode(L, X, ix);
            double gr[3] = {0, 0, 0}, g2 = 0.0;
            for (int a = 0; a < L->d; ++a) {
                gr[a] = grad_a(L, X, ix, a);
                g2 += gr[a] * gr[a];
            }
            double dn = 0.0;
            if (g2 > 0.0) {
                double gn = sqrt(g2);
                for (int a = 0; a < L->d; ++a) {
                    double vp = 0.0, vm = 0.0;
                    int iy[3] = {ix[0], ix[1], ix[2]};
                    iy[a] += 1;
                    if (in_grid(L, iy)) vp = arr[lin_of(L, iy)];
                    iy[a] -= 2;
                    if (in_grid(L, iy)) vm = arr[lin_of(L, iy)];
                    dn += (gr[a] / gn) * 0.5 * (vp - vm);
                }
            }
            nw[b] = old[b] - O->ext_cfl * dn;
        }
        for (long b = 0; b < nb; ++b) {
            old[b] = nw[b];
            arr[L->bidx[b]] = nw[b];
        }
    }
}

/* Default extension (reading of Sec. 3.3.2): a fixed number of explicit
 * pseudo-time sweeps of dr/dsigma + dr/dn = 0 with upwind differences at the
 * largest stable step, which makes each sweep the |n_a|-weighted mean of the
 * upwind neighbours; sources are ghosts and band nodes; the band starts from
 * zero. */
static void extend(const oracle_t *O, olevel *L, double *arr) {
    long nb = L->nb;
    if (nb == 0) return;
    if (O->ext_mode == 1) {
        extend_central(O, L, arr);
        return;
    }
    double *old = L->tmp, *nw = L->tmp + nb;
    for (long b = 0; b < nb; ++b) old[b] = 0.0;
    for (int k = 0; k < O->ext_sweeps; ++k) {
        for (long b = 0; b < nb; ++b) {
            double num = 0.0, den = 0.0;
            for (int a = 0; a < L->d; ++a) {
                long y = L->bup[3 * b + a];
                if (y < 0) continue;
                double v = (L->cls[y] == CL_GHOST) ? arr[y] : old[L->bpos[y]];
                num += L->bw[3 * b + a] * v;
                den += L->bw[3 * b + a];
            }
            nw[b] = den > 0.0 ? num / den : 0.0;
        }
        double *t = old;
        old = nw;
        nw = t;
    }
    for (long b = 0; b < nb; ++b) arr[L->bidx[b]] = old[b];
}

/* Restriction (Sec. 2.1 eq. coarseFW and the mean next to the boundary;
 * Sec. 3.3.2): coarse interior nodes take FW of the fine interior residual
 * if all 3^d fine neighbours are interior, else the plain mean of the
 * interior ones; coarse ghosts take FW of the (extended) exterior residual
 * if all 3^d are ghost/inactive, else the mean of the ghost/inactive ones. */
static void restrict_op(const olevel *Lf, const olevel *Lc, const double *rf, double *Fc, int rmode,
                        int gfam, int cg_rhs) {
    int d = Lf->d;
    for (long c = 0; c < Lc->nn; ++c) {
        Fc[c] = 0.0;
        unsigned char pc = Lc->cls[c];
        if (pc != CL_INTERIOR && pc != CL_GHOST) continue;
        int ic[3];
        decode(Lc, c, ic);
        double sum = 0.0, fw = 0.0, wsum = 0.0;
        long cnt = 0;
        int all = 1;
        int o[3];
        for (o[2] = (d > 2 ? -1 : 0); o[2] <= (d > 2 ? 1 : 0); ++o[2])
            for (o[1] = (d > 1 ? -1 : 0); o[1] <= (d > 1 ? 1 : 0); ++o[1])
                for (o[0] = -1; o[0] <= 1; ++o[0]) {
                    int iy[3] = {0, 0, 0};
                    double wfw = 1.0;
                    for (int a = 0; a < d; ++a) {
                        iy[a] = 2 * ic[a] + o[a];
                        wfw *= (o[a] == 0) ? 0.5 : 0.25;
                    }
                    if (!in_grid(Lf, iy)) {
                        all = 0;
                        continue;
                    }
                    long y = lin_of(Lf, iy);
                    unsigned char cy = Lf->cls[y];
                    int fam = (pc == CL_INTERIOR) ? (cy == CL_INTERIOR)
                                                  : (cy == CL_GHOST || (cy == CL_INACTIVE && gfam == 0));
                    if (!fam) {
                        all = 0;
                        continue;
                    }
                    sum += rf[y];
                    fw += wfw * rf[y];
                    wsum += wfw;
                    cnt++;
                }
        int weighted = (pc == CL_INTERIOR) ? (rmode & 1) : ((rmode >> 1) & 1);
        if (pc == CL_GHOST && cg_rhs == 1) {
            /* injection: the fine node at the coarse ghost's position (a
             * ghost or an extended band node, never interior since phi is
             * injected) */
            int iy[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) iy[a] = 2 * ic[a];
            Fc[c] = rf[lin_of(Lf, iy)];
            continue;
        }
        if (all) Fc[c] = fw;
        else if (weighted) Fc[c] = wsum > 0.0 ? fw / wsum : 0.0;
        else Fc[c] = cnt > 0 ? sum / (double)cnt : 0.0;
    }
}

/* Prolongation (Sec. 2.1 linear interpolation, Sec. 3.2 bilinear, Sec. 3.3.2):
 * u_f += multilinear interpolation of e_c on interior and ghost fine nodes. */
static void prolong_op(const olevel *Lf, const olevel *Lc, const double *ec, double *uf) {
    int d = Lf->d;
    for (long y = 0; y < Lf->nn; ++y) {
        unsigned char cy = Lf->cls[y];
        if (cy != CL_INTERIOR && cy != CL_GHOST) continue;
        int iy[3];
        decode(Lf, y, iy);
        int lo[3] = {0, 0, 0}, cnt[3] = {1, 1, 1};
        for (int a = 0; a < d; ++a) {
            if (iy[a] % 2 == 0) {
                lo[a] = iy[a] / 2;
                cnt[a] = 1;
            } else {
                lo[a] = (iy[a] - 1) / 2;
                cnt[a] = 2;
            }
        }
        double v = 0.0;
        for (int b2 = 0; b2 < cnt[2]; ++b2)
            for (int b1 = 0; b1 < cnt[1]; ++b1)
                for (int b0 = 0; b0 < cnt[0]; ++b0) {
                    int ic[3] = {lo[0] + b0, lo[1] + b1, lo[2] + b2};
                    double w = (cnt[0] == 2 ? 0.5 : 1.0) * (cnt[1] == 2 ? 0.5 : 1.0) *
                               (cnt[2] == 2 ? 0.5 : 1.0);
                    v += w * ec[lin_of(Lc, ic)];
                }
        uf[y] += v;
    }
}

/* ------------------------------------------------------------------ */
/* dense system (interior + ghost unknowns), direct solve                */
/* ------------------------------------------------------------------ */

/* Assemble A (nact x nact, row-major) of the level's equations over the
 * active unknowns (interior and ghost nodes in index order).  Eliminated
 * BOXDIR nodes are not unknowns. */
static void assemble(const olevel *L, const long *act, const int *apos, long nact, double *A) {
    int d = L->d;
    double ih2 = 1.0 / (L->h * L->h);
    memset(A, 0, sizeof(double) * (size_t)nact * (size_t)nact);
    for (long r = 0; r < nact; ++r) {
        long X = act[r];
        if (L->cls[X] == CL_INTERIOR) {
            A[r * nact + r] += 2.0 * d * ih2 + L->react;
            for (int a = 0; a < d; ++a)
                for (int dir = -1; dir <= 1; dir += 2) {
                    long Y = X + dir * L->st[a];
                    if (apos[Y] >= 0) A[r * nact + apos[Y]] -= ih2;
                }
        }
    }
    for (long g = 0; g < L->ng; ++g) {
        long X = L->gidx[g];
        long r = apos[X];
        gstencil S;
        ghost_stencil(L, g, &S);
        for (int o2 = 0; o2 <= S.q[2]; ++o2)
            for (int o1 = 0; o1 <= S.q[1]; ++o1)
                for (int o0 = 0; o0 <= S.q[0]; ++o0) {
                    long Y = X - (long)S.s[0] * o0 * L->st[0] - (long)S.s[1] * o1 * L->st[1] -
                             (long)S.s[2] * o2 * L->st[2];
                    if (apos[Y] >= 0) A[r * nact + apos[Y]] += ghost_weight(L, &S, o0, o1, o2);
                }
    }
}

static void build_active(olevel *L) {
    L->apos = (int *)malloc(sizeof(int) * (size_t)L->nn);
    L->nact = 0;
    for (long i = 0; i < L->nn; ++i) {
        L->apos[i] = -1;
        if (L->cls[i] == CL_INTERIOR || L->cls[i] == CL_GHOST) L->nact++;
    }
    L->act = (long *)calloc(L->nact + 1, sizeof(long));
    long k = 0;
    for (long i = 0; i < L->nn; ++i)
        if (L->cls[i] == CL_INTERIOR || L->cls[i] == CL_GHOST) {
            L->act[k] = i;
            L->apos[i] = (int)k;
            ++k;
        }
}

/* Gaussian elimination with partial pivoting, LU in place (row swaps in piv) */
static int lu_factor(double *A, long n, long *piv) {
    for (long k = 0; k < n; ++k) {
        long p = k;
        double best = fabs(A[k * n + k]);
        for (long i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > best) {
                best = fabs(A[i * n + k]);
                p = i;
            }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k)
            for (long j = 0; j < n; ++j) {
                double t = A[k * n + j];
                A[k * n + j] = A[p * n + j];
                A[p * n + j] = t;
            }
        for (long i = k + 1; i < n; ++i) {
            double m = A[i * n + k] / A[k * n + k];
            A[i * n + k] = m;
            for (long j = k + 1; j < n; ++j) A[i * n + j] -= m * A[k * n + j];
        }
    }
    return 0;
}

static void lu_solve(const double *LU, long n, const long *piv, double *b) {
    for (long k = 0; k < n; ++k) {
        long p = piv[k];
        if (p != k) {
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
    }
    for (long i = 0; i < n; ++i)
        for (long j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];
    for (long i = n - 1; i >= 0; --i) {
        for (long j = i + 1; j < n; ++j) b[i] -= LU[i * n + j] * b[j];
        b[i] /= LU[i * n + i];
    }
}

/* ------------------------------------------------------------------ */
/* hierarchy                                                            */
/* ------------------------------------------------------------------ */

static void level_init(olevel *L, int d, int N) {
    memset(L, 0, sizeof(*L));
    L->d = d;
    L->N = N;
    L->n = N + 1;
    L->h = 2.0 / N;
    L->nn = 1;
    for (int a = 0; a < 3; ++a) L->st[a] = 0;
    for (int a = 0; a < d; ++a) {
        L->st[a] = L->nn;
        L->nn *= L->n;
    }
    L->phi = (double *)calloc((size_t)L->nn, sizeof(double));
    L->cls = (unsigned char *)calloc((size_t)L->nn, 1);
}

static void level_free(olevel *L) {
    free(L->phi);
    free(L->cls);
    free(L->gidx);
    free(L->geta);
    free(L->gn);
    free(L->gxi);
    free(L->gdt);
    free(L->gQ);
    free(L->gs);
    free(L->gq);
    free(L->bidx);
    free(L->bup);
    free(L->bw);
    free(L->bpos);
    free(L->u);
    free(L->F);
    free(L->r);
    free(L->tmp);
    free(L->act);
    free(L->apos);
    free(L->LU);
    free(L->piv);
    memset(L, 0, sizeof(*L));
}

static void level_finish(oracle_t *O, olevel *L) {
    L->bc = O->bc;
    L->react = O->react;
    setup_ghosts(O, L);
    setup_band(L, O->band_width);
    L->u = (double *)calloc((size_t)L->nn, sizeof(double));
    L->F = (double *)calloc((size_t)L->nn, sizeof(double));
    L->r = (double *)calloc((size_t)L->nn, sizeof(double));
    long t = L->ng > L->nb ? L->ng : L->nb;
    L->tmp = (double *)calloc((size_t)(2 * t + 2), sizeof(double));
}

void orc_destroy(void *hp) {
    oracle_t *O = (oracle_t *)hp;
    if (!O) return;
    for (int l = 0; l < O->L; ++l) level_free(&O->lv[l]);
    free(O);
}

/* iopts: nu1, nu2, ordering, dtau_mode, ext_sweeps, cycle, min_coarse,
 *        max_levels, tgcs_maxit, rmode, ext_mode, bc (0 Dirichlet,
 *        1 Neumann on Gamma), band_width (Chebyshev radius of the
 *        extension band, 2), gfam (coarse-ghost restriction family: 0 ghost
 *        and inactive points, 1 ghost points only), cg_rhs (coarse-ghost
 *        right-hand side: 0 the family restriction, 1 injection)
 * dopts: dtau_const (Dtau, or Dtau / h for Neumann), tgcs_tol, ext_cfl,
 *        reaction coefficient c
 * Coarsening (geometric re-discretisation, Sec. 2.1): N_{l+1} = N_l / 2
 * while N_l is even, N_l / 2 >= min_coarse and the coarse level still has
 * interior nodes.  Returns NULL if the finest level has no interior node or
 * the coarsest system is singular / too large for the dense solve. */
void *orc_create(int d, int N, const double *phi, const int *iopts, const double *dopts) {
    if (d < 1 || d > 3 || N < 4) return NULL;
    oracle_t *O = (oracle_t *)calloc(1, sizeof(oracle_t));
    O->d = d;
    O->N = N;
    O->nu1 = iopts[0];
    O->nu2 = iopts[1];
    O->ordering = iopts[2];
    O->dtau_mode = iopts[3];
    O->ext_sweeps = iopts[4];
    O->cycle = iopts[5];
    O->min_coarse = iopts[6];
    O->max_levels = iopts[7];
    O->tgcs_maxit = iopts[8];
    O->rmode = iopts[9];
    O->ext_mode = iopts[10];
    O->bc = iopts[11];
    O->band_width = iopts[12];
    O->gfam = iopts[13];
    O->cg_rhs = iopts[14];
    if (O->band_width < 1 || O->band_width > 4) O->band_width = 2;
    O->react = dopts[3];
    O->ext_cfl = dopts[2];
    O->dtau_const = dopts[0];
    O->tgcs_tol = dopts[1];
    if (O->max_levels < 1 || O->max_levels > ORC_MAXL) O->max_levels = ORC_MAXL;
    level_init(&O->lv[0], d, N);
    memcpy(O->lv[0].phi, phi, sizeof(double) * (size_t)O->lv[0].nn);
    classify(&O->lv[0]);
    if (O->lv[0].nint == 0) {
        level_free(&O->lv[0]);
        free(O);
        return NULL;
    }
    level_finish(O, &O->lv[0]);
    O->L = 1;
    while (O->L < O->max_levels) {
        olevel *Lf = &O->lv[O->L - 1];
        if (Lf->N % 2 != 0 || Lf->N / 2 < O->min_coarse) break;
        olevel *Lc = &O->lv[O->L];
        level_init(Lc, d, Lf->N / 2);
        for (long c = 0; c < Lc->nn; ++c) {
            int ic[3], iy[3];
            decode(Lc, c, ic);
            for (int a = 0; a < 3; ++a) iy[a] = 2 * ic[a];
            Lc->phi[c] = Lf->phi[lin_of(Lf, iy)]; /* injection */
        }
        classify(Lc);
        if (Lc->nint == 0) {
            level_free(Lc);
            break;
        }
        level_finish(O, Lc);
        O->L++;
    }
    olevel *Lc = &O->lv[O->L - 1];
    build_active(Lc);
    Lc->direct_ok = -1; /* factored on first use */
    /* a hierarchy whose coarsest system cannot be factored is still usable
     * for the geometry and the stage operators; cycles refuse to run */
    return O;
}

/* ------------------------------------------------------------------ */
/* cycles (Sec. 2.1: TGCS, V-cycle gamma = 1, W-cycle gamma = 2)          */
/* ------------------------------------------------------------------ */

static double l2_active(const olevel *L, const double *r) {
    double s = 0.0;
    for (long i = 0; i < L->nn; ++i)
        if (L->cls[i] == CL_INTERIOR || L->cls[i] == CL_GHOST) s += r[i] * r[i];
    return sqrt(s);
}

/* Factor the coarsest dense system on first use (Gaussian elimination with
 * partial pivoting); 1 if it could be factored, 0 if singular or too big. */
static int ensure_direct(oracle_t *O) {
    olevel *Lc = &O->lv[O->L - 1];
    if (Lc->direct_ok >= 0) return Lc->direct_ok;
    Lc->direct_ok = 0;
    if (Lc->nact <= 12000) {
        Lc->LU = (double *)malloc(sizeof(double) * (size_t)Lc->nact * (size_t)Lc->nact);
        Lc->piv = (long *)calloc(Lc->nact + 1, sizeof(long));
        assemble(Lc, Lc->act, Lc->apos, Lc->nact, Lc->LU);
        if (lu_factor(Lc->LU, Lc->nact, Lc->piv) == 0) Lc->direct_ok = 1;
    }
    return Lc->direct_ok;
}

static void coarsest_solve(oracle_t *O, int l, double *u, const double *F) {
    olevel *L = &O->lv[l];
    if (ensure_direct(O) != 1) return;
    residual(L, u, F, L->r);
    double *b = (double *)malloc(sizeof(double) * (size_t)(L->nact + 1));
    for (long k = 0; k < L->nact; ++k) b[k] = L->r[L->act[k]];
    lu_solve(L->LU, L->nact, L->piv, b);
    for (long k = 0; k < L->nact; ++k) u[L->act[k]] += b[k];
    free(b);
}

static void cycle_rec(oracle_t *O, int l, double *u, const double *F, int gamma);

static void coarse_exact(oracle_t *O, int l) {
    olevel *L = &O->lv[l];
    double f0 = l2_active(L, L->F);
    for (int it = 0; it < O->tgcs_maxit; ++it) {
        cycle_rec(O, l, L->u, L->F, 1);
        residual(L, L->u, L->F, L->r);
        double rn = l2_active(L, L->r);
        if (rn <= O->tgcs_tol * f0 || rn == 0.0) break;
    }
}

static void cycle_rec(oracle_t *O, int l, double *u, const double *F, int gamma) {
    olevel *L = &O->lv[l];
    if (l == O->L - 1) {
        coarsest_solve(O, l, u, F);
        return;
    }
    olevel *Lc = &O->lv[l + 1];
    for (int s = 0; s < O->nu1; ++s) smooth_step(O, L, u, F);
    residual(L, u, F, L->r);
    extend(O, L, L->r);
    restrict_op(L, Lc, L->r, Lc->F, O->rmode, O->gfam, O->cg_rhs);
    memset(Lc->u, 0, sizeof(double) * (size_t)Lc->nn);
    if (O->cycle == CYC_TGCS && l == 0 && O->L > 2) {
        coarse_exact(O, 1);
    } else {
        for (int gi = 0; gi < gamma; ++gi) cycle_rec(O, l + 1, Lc->u, Lc->F, gamma);
    }
    extend(O, Lc, Lc->u);
    prolong_op(L, Lc, Lc->u, u);
    for (int s = 0; s < O->nu2; ++s) smooth_step(O, L, u, F);
}

/* ------------------------------------------------------------------ */
/* exported entry points                                                */
/* ------------------------------------------------------------------ */

int orc_num_levels(void *hp) { return ((oracle_t *)hp)->L; }

int orc_direct_ok(void *hp) { return ensure_direct((oracle_t *)hp); }

/* out: N, n, nn, n_interior, n_ghost, n_band, n_boxdir, n_clamped,
 *      n_fallback, n_active(coarsest only, else 0) */
void orc_level_info(void *hp, int l, long *out) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    out[0] = L->N;
    out[1] = L->n;
    out[2] = L->nn;
    out[3] = L->nint;
    out[4] = L->ng;
    out[5] = L->nb;
    out[6] = L->nbox;
    out[7] = L->nclamp;
    out[8] = L->nfall;
    out[9] = L->nact;
}

void orc_get_class(void *hp, int l, unsigned char *out) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    memcpy(out, L->cls, (size_t)L->nn);
}

void orc_get_phi(void *hp, int l, double *out) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    memcpy(out, L->phi, sizeof(double) * (size_t)L->nn);
}

/* ghost data, 3 entries per ghost for the vector fields */
void orc_get_ghosts(void *hp, int l, long *idx, double *eta, double *n, double *xi, int *s,
                    int *q, double *dtau, double *Q) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    memcpy(idx, L->gidx, sizeof(long) * (size_t)L->ng);
    memcpy(eta, L->geta, sizeof(double) * (size_t)L->ng);
    memcpy(n, L->gn, sizeof(double) * 3 * (size_t)L->ng);
    memcpy(xi, L->gxi, sizeof(double) * 3 * (size_t)L->ng);
    memcpy(s, L->gs, sizeof(int) * 3 * (size_t)L->ng);
    memcpy(q, L->gq, sizeof(int) * 3 * (size_t)L->ng);
    memcpy(dtau, L->gdt, sizeof(double) * (size_t)L->ng);
    memcpy(Q, L->gQ, sizeof(double) * 3 * (size_t)L->ng);
}

void orc_get_band(void *hp, int l, long *idx) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    memcpy(idx, L->bidx, sizeof(long) * (size_t)L->nb);
}

/* F_0: f at interior nodes (eq. Laph), g(Q_G) at ghosts (eq. BCh), zero
 * elsewhere. */
void orc_set_rhs(void *hp, const double *f, const double *gQ) {
    olevel *L = &((oracle_t *)hp)->lv[0];
    for (long i = 0; i < L->nn; ++i) L->F[i] = (L->cls[i] == CL_INTERIOR) ? f[i] : 0.0;
    for (long g = 0; g < L->ng; ++g) L->F[L->gidx[g]] = gQ[g];
}

void orc_get_F(void *hp, int l, double *out) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    memcpy(out, L->F, sizeof(double) * (size_t)L->nn);
}

void orc_set_F(void *hp, int l, const double *in) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    memcpy(L->F, in, sizeof(double) * (size_t)L->nn);
}

/* stage operators on caller arrays of level l */
void orc_smooth(void *hp, int l, double *u, const double *F, int nsteps) {
    oracle_t *O = (oracle_t *)hp;
    for (int s = 0; s < nsteps; ++s) smooth_step(O, &O->lv[l], u, F);
}

void orc_interior_sweep(void *hp, int l, double *u, const double *F) {
    oracle_t *O = (oracle_t *)hp;
    olevel *L = &O->lv[l];
    if (O->ordering == ORD_RB) interior_rb(L, u, F);
    else if (O->ordering == ORD_LEX) interior_lex(L, u, F);
    else O->block_sweeps_last = interior_block(L, u, F);
}

long orc_interior_block(void *hp, int l, double *u, const double *F) {
    oracle_t *O = (oracle_t *)hp;
    return interior_block(&O->lv[l], u, F);
}

void orc_ghost_relax(void *hp, int l, double *u, const double *F) {
    oracle_t *O = (oracle_t *)hp;
    ghost_relax(&O->lv[l], u, F);
}

void orc_ghost_apply(void *hp, int l, const double *u, double *out) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    for (long g = 0; g < L->ng; ++g) out[g] = ghost_apply(L, g, u);
}

void orc_residual(void *hp, int l, const double *u, const double *F, double *r) {
    residual(&((oracle_t *)hp)->lv[l], u, F, r);
}

void orc_extend(void *hp, int l, double *a) {
    oracle_t *O = (oracle_t *)hp;
    extend(O, &O->lv[l], a);
}

void orc_restrict(void *hp, int l, const double *rf, double *Fc) {
    oracle_t *O = (oracle_t *)hp;
    restrict_op(&O->lv[l], &O->lv[l + 1], rf, Fc, O->rmode, O->gfam, O->cg_rhs);
}

void orc_prolong(void *hp, int l, const double *ec, double *uf) {
    oracle_t *O = (oracle_t *)hp;
    prolong_op(&O->lv[l], &O->lv[l + 1], ec, uf);
}

/* exact correction solve on the coarsest level: u += A^-1 (F - A u) */
void orc_coarsest_solve(void *hp, double *u, const double *F) {
    oracle_t *O = (oracle_t *)hp;
    coarsest_solve(O, O->L - 1, u, F);
}

/* ncycles cycles on the finest level with its stored F */
void orc_vcycle(void *hp, double *u, int ncycles) {
    oracle_t *O = (oracle_t *)hp;
    int gamma = (O->cycle == CYC_W) ? 2 : 1;
    for (int c = 0; c < ncycles; ++c) cycle_rec(O, 0, u, O->lv[0].F, gamma);
}

/* residual norms on the finest level: ||r_I||_2, ||r_G||_2, ||r_I||_inf,
 * ||r_G||_inf (unscaled residuals, the paper's ||r_h||_p of Sec. 2.2). */
void orc_norms(void *hp, const double *u, double *out) {
    olevel *L = &((oracle_t *)hp)->lv[0];
    residual(L, u, L->F, L->r);
    double s2i = 0.0, s2g = 0.0, mi = 0.0, mg = 0.0;
    for (long i = 0; i < L->nn; ++i) {
        double v = L->r[i];
        if (L->cls[i] == CL_INTERIOR) {
            s2i += v * v;
            if (fabs(v) > mi) mi = fabs(v);
        } else if (L->cls[i] == CL_GHOST) {
            s2g += v * v;
            if (fabs(v) > mg) mg = fabs(v);
        }
    }
    out[0] = sqrt(s2i);
    out[1] = sqrt(s2g);
    out[2] = mi;
    out[3] = mg;
}

/* cycles until ||r||_2 <= rtol ||r0||_2; hist[0..] receives ||r||_2 after each
 * cycle (hist[0] = initial).  Returns the number of cycles done. */
int orc_solve(void *hp, double *u, double rtol, int maxc, double *hist) {
    double nr[4];
    orc_norms(hp, u, nr);
    double r0 = sqrt(nr[0] * nr[0] + nr[1] * nr[1]);
    if (hist) hist[0] = r0;
    if (r0 == 0.0) return 0;
    for (int c = 1; c <= maxc; ++c) {
        orc_vcycle(hp, u, 1);
        orc_norms(hp, u, nr);
        double rn = sqrt(nr[0] * nr[0] + nr[1] * nr[1]);
        if (hist) hist[c] = rn;
        if (rn <= rtol * r0) return c;
    }
    return maxc;
}

/* Dense system of level l over interior + ghost unknowns (index order) with
 * the eliminated BOXDIR values of u moved to the right-hand side. */
long orc_active_count(void *hp, int l) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    long c = 0;
    for (long i = 0; i < L->nn; ++i)
        if (L->cls[i] == CL_INTERIOR || L->cls[i] == CL_GHOST) c++;
    return c;
}

void orc_assemble(void *hp, int l, const double *u, const double *F, long *act, double *A,
                  double *rhs) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    int d = L->d;
    int *apos = (int *)malloc(sizeof(int) * (size_t)L->nn);
    long nact = 0;
    for (long i = 0; i < L->nn; ++i) {
        apos[i] = -1;
        if (L->cls[i] == CL_INTERIOR || L->cls[i] == CL_GHOST) {
            act[nact] = i;
            apos[i] = (int)nact;
            nact++;
        }
    }
    assemble(L, act, apos, nact, A);
    double ih2 = 1.0 / (L->h * L->h);
    for (long r = 0; r < nact; ++r) {
        long X = act[r];
        rhs[r] = F[X];
        if (L->cls[X] == CL_INTERIOR) {
            for (int a = 0; a < d; ++a)
                for (int dir = -1; dir <= 1; dir += 2) {
                    long Y = X + dir * L->st[a];
                    if (L->cls[Y] == CL_BOXDIR) rhs[r] += u[Y] * ih2;
                }
        }
    }
    for (long g = 0; g < L->ng; ++g) {
        long X = L->gidx[g];
        long r = apos[X];
        gstencil S;
        ghost_stencil(L, g, &S);
        for (int o2 = 0; o2 <= S.q[2]; ++o2)
            for (int o1 = 0; o1 <= S.q[1]; ++o1)
                for (int o0 = 0; o0 <= S.q[0]; ++o0) {
                    long Y = X - (long)S.s[0] * o0 * L->st[0] - (long)S.s[1] * o1 * L->st[1] -
                             (long)S.s[2] * o2 * L->st[2];
                    if (L->cls[Y] == CL_BOXDIR) rhs[r] -= ghost_weight(L, &S, o0, o1, o2) * u[Y];
                }
    }
    free(apos);
}

/* Oracle's own dense direct solve of the full discrete problem on level l
 * (tiny grids): u at interior and ghost nodes <- A^-1 rhs.  0 on success. */
int orc_direct_solve(void *hp, int l, double *u, const double *F) {
    olevel *L = &((oracle_t *)hp)->lv[l];
    long nact = orc_active_count(hp, l);
    long *act = (long *)calloc(nact + 1, sizeof(long));
    double *A = (double *)malloc(sizeof(double) * (size_t)nact * (size_t)nact);
    double *b = (double *)malloc(sizeof(double) * (size_t)(nact + 1));
    long *piv = (long *)calloc(nact + 1, sizeof(long));
    orc_assemble(hp, l, u, F, act, A, b);
    int rc = lu_factor(A, nact, piv);
    if (rc == 0) {
        lu_solve(A, nact, piv, b);
        for (long k = 0; k < nact; ++k) u[act[k]] = b[k];
    }
    (void)L;
    free(act);
    free(A);
    free(b);
    free(piv);
    return rc;
}

long orc_block_sweeps_last(void *hp) { return ((oracle_t *)hp)->block_sweeps_last; }

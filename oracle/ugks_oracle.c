/*
 * ugks_oracle.c -- plain FP64 CPU oracle of one explicit UGKS time step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  Built with -O2 -ffp-contract=off so that every
 * product and sum is rounded as written.
 *
 * The step follows Algorithm 1 of the paper (Sec. 3.2) literally:
 *   1. time step (CFL) and cell heat flux from f^n;
 *   2. macroscopic reconstruction;
 *   3. interface equilibrium and time coefficients for every face;
 *   4. for every discrete velocity k: reconstruct f_k, evolve the face flux
 *      F_k (Eq. microscopicFlux with Eq. fullSolution) and its macroscopic
 *      contribution (Eq. macroscopicFlux), interpolate f_k and its gradient at
 *      the wall, and update f_k^n -> f~_k^{n+1} in place (Eq. microS1);
 *   5. evolve the wall flux (Sec. 2.5, Eq. maxWalldes);
 *   6. update W (Eq. macroscopicUpdata);
 *   7. update f (Eq. microS2).
 * Readings of points the paper leaves open are marked "READING" below.
 */
#include "ugks_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXD 3
#define MAXM 5 /* D + 2 conserved variables */

struct or_case {
    int D, nc;      /* dimension, stored components (h,b in 2D; h in 3D) */
    double nxi;     /* internal translational degrees of freedom 3 - D (K = 0) */
    int64_t C, F, Nv;
    double *cell_xc, *cell_vol, *face_n, *face_S, *face_xc, *face_shift;
    int64_t *face_cells;
    int32_t *face_type, *face_tag;
    double *u, *w;
    or_params p;
    double *wall_T, *wall_U;
    double dt, mu_ref;
    /* faces of each cell: face id, side (0 owner, 1 neighbour), offset r = x_f - x_i */
    int64_t *cf_ptr, *cf_face;
    int32_t *cf_side;
    double *cf_r;
    /* least-squares neighbours: id >= 0 cell, id < 0 far-field ghost of face -id-1 */
    int64_t *nb_ptr, *nb_id;
    double *nb_a;
    double *eps2;
    /* wall faces */
    int64_t n_wall, *wall_face, *wall_slot_of_face;
    /* state */
    double *f, *W;
    /* per-step work arrays */
    double *Wold, *q, *rho, *U, *lam, *tau, *gradW, *Wghost, *W0, *fa, *fA, *q0, *qs, *grad_k,
        *Fk, *Fm, *fin, *gfin, *rho_w, *ghost_k, res[MAXM], *P, *Pg, *gradP;
    /* face states W_L, W_R of the last step (conserved; W_R = ghost state at far field) */
    double *WLs, *WRs;
};

/* ------------------------------------------------------------------------ */
/* gas model (Sec. 2.1-2.2)                                                  */
/* ------------------------------------------------------------------------ */

/* primitive variables from W = (rho, rho U, rho E); T = (2/3)(E - |U|^2/2)
 * for a monatomic gas (three translational degrees of freedom), lambda = 1/(2T) */
static void prim_of(int D, const double *W, double *rho, double *U, double *lam)
{
    double ke = 0.0;
    *rho = W[0];
    for (int d = 0; d < D; ++d) {
        U[d] = W[1 + d] / W[0];
        ke += U[d] * U[d];
    }
    double E = W[D + 1] / W[0];
    double T = (2.0 / 3.0) * (E - 0.5 * ke);
    *lam = 1.0 / (2.0 * T);
}

/* H = rho (lam/pi)^{D/2} exp(-lam |u-U|^2); B = (3-D+K)/(2 lam) H with K = 0 */
static void maxwell1(int D, double rho, const double *U, double lam, const double *uk,
                     double *H, double *B)
{
    double c2 = 0.0;
    for (int d = 0; d < D; ++d) {
        double c = uk[d] - U[d];
        c2 += c * c;
    }
    double h = rho * pow(lam / M_PI, 0.5 * D) * exp(-lam * c2);
    *H = h;
    *B = (3.0 - D) / (2.0 * lam) * h;
}

/* H+ = 4(1-Pr) lam^2/(5 rho) (c.q)(2 lam c^2 - 2 - D) H,
 * B+ = 4(1-Pr) lam^2/(5 rho) (c.q){[2 lam c^2 - D](3-D+K) - 2K} H/(2 lam), K = 0 */
static void shakhov1(int D, double Pr, double rho, const double *U, double lam, const double *q,
                     const double *uk, double H, double *Hp, double *Bp)
{
    double c2 = 0.0, cq = 0.0;
    for (int d = 0; d < D; ++d) {
        double c = uk[d] - U[d];
        c2 += c * c;
        cq += c * q[d];
    }
    double pre = 4.0 * (1.0 - Pr) * lam * lam / (5.0 * rho) * cq;
    *Hp = pre * (2.0 * lam * c2 - 2.0 - D) * H;
    *Bp = pre * ((2.0 * lam * c2 - D) * (3.0 - D)) * H / (2.0 * lam);
}

/* moments of phi(u, xi) = alpha_0 + alpha_u.u + alpha_E (|u|^2+xi^2)/2 against g
 * integrated over xi:  out_h = int phi g dxi,  out_b = int xi^2 phi g dxi.
 * Uses int g = H, int xi^2 g = B, int xi^4 g = X = N(N+2)/(4 lam^2) H. */
static void psi_moment(int D, const double *uk, const double *alpha, double H, double B,
                       double X, double *out_h, double *out_b)
{
    double u2 = 0.0, lin = alpha[0];
    for (int d = 0; d < D; ++d) {
        u2 += uk[d] * uk[d];
        lin += alpha[1 + d] * uk[d];
    }
    double poly = lin + alpha[D + 1] * 0.5 * u2;
    *out_h = poly * H + alpha[D + 1] * 0.5 * B;
    *out_b = poly * B + alpha[D + 1] * 0.5 * X;
}

/* P(u) = int psi psi^T g dxi at one velocity (psi = (1, u, (u^2+xi^2)/2)) */
static void psi_outer(int D, const double *uk, double H, double B, double X, double *P)
{
    int M = D + 2;
    double u2 = 0.0;
    for (int d = 0; d < D; ++d) u2 += uk[d] * uk[d];
    double e_h = 0.5 * (u2 * H + B); /* int psi_E g */
    P[0] = H;
    for (int d = 0; d < D; ++d) {
        P[1 + d] = uk[d] * H;
        P[(1 + d) * M] = uk[d] * H;
        for (int e = 0; e < D; ++e) P[(1 + d) * M + 1 + e] = uk[d] * uk[e] * H;
        P[(1 + d) * M + D + 1] = uk[d] * e_h;
        P[(D + 1) * M + 1 + d] = uk[d] * e_h;
    }
    P[D + 1] = e_h;
    P[(D + 1) * M] = e_h;
    P[(D + 1) * M + D + 1] = 0.25 * (u2 * u2 * H + 2.0 * u2 * B + X);
}

/* Gaussian elimination with partial pivoting; A is n x n row-major, b overwritten */
static int solve(int n, double *A, double *b)
{
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
        if (A[piv * n + col] == 0.0) return -1;
        if (piv != col) {
            for (int k = 0; k < n; ++k) {
                double t = A[col * n + k];
                A[col * n + k] = A[piv * n + k];
                A[piv * n + k] = t;
            }
            double t = b[col];
            b[col] = b[piv];
            b[piv] = t;
        }
        for (int r = col + 1; r < n; ++r) {
            double m = A[r * n + col] / A[col * n + col];
            for (int k = col; k < n; ++k) A[r * n + k] -= m * A[col * n + k];
            b[r] -= m * b[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* exported building blocks                                                  */
/* ------------------------------------------------------------------------ */

void or_maxwellian(int32_t D, double rho, const double *U, double lam, int64_t nv,
                   const double *u, double *H, double *B)
{
    for (int64_t k = 0; k < nv; ++k) {
        double b;
        maxwell1(D, rho, U, lam, u + k * D, &H[k], &b);
        if (B) B[k] = b;
    }
}

void or_shakhov(int32_t D, double Pr, double rho, const double *U, double lam, const double *q,
                int64_t nv, const double *u, double *Hp, double *Bp)
{
    for (int64_t k = 0; k < nv; ++k) {
        double H, B, hp, bp;
        maxwell1(D, rho, U, lam, u + k * D, &H, &B);
        shakhov1(D, Pr, rho, U, lam, q, u + k * D, H, &hp, &bp);
        Hp[k] = hp;
        if (Bp) Bp[k] = bp;
    }
}

/* q = 1/2 int c (|c|^2 + xi^2) f  ->  1/2 sum_k w_k c_k (|c_k|^2 h_k + b_k) (Sec. 2.1) */
void or_heat_flux(int32_t D, int64_t nv, const double *u, const double *w, const double *h,
                  const double *b, const double *U, double *q)
{
    for (int d = 0; d < D; ++d) q[d] = 0.0;
    for (int64_t k = 0; k < nv; ++k) {
        double c[MAXD], c2 = 0.0;
        for (int d = 0; d < D; ++d) {
            c[d] = u[k * D + d] - U[d];
            c2 += c[d] * c[d];
        }
        double e = c2 * h[k] + (b ? b[k] : 0.0);
        for (int d = 0; d < D; ++d) q[d] += 0.5 * w[k] * c[d] * e;
    }
}

/* time integrals of c1..c5 (Sec. 2.4) over [0, dt]:
 *   q1 = int e^{-t/tau}                 = tau (1-e)
 *   q2 = int -t e^{-t/tau}              = tau dt e - tau^2 (1-e)
 *   q3 = int 1 - e^{-t/tau}             = dt - tau (1-e)
 *   q4 = int t e^{-t/tau} - tau(1-e^{-t/tau}) = 2 tau^2 (1-e) - tau dt (1+e)
 *   q5 = int t - tau(1-e^{-t/tau})      = dt^2/2 - tau dt + tau^2 (1-e)
 * with e = exp(-dt/tau).  For x = dt/tau < 1/2 the same functions are summed
 * from their power series in x (no cancellation); tau = +inf gives x = 0. */
void or_time_integrals(double dt, double tau, double q[5])
{
    double x = dt / tau;
    if (x < 0.5) {
        double s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
        double xj = 1.0, fact1 = 1.0, fact2 = 2.0; /* x^j, (j+1)!, (j+2)! */
        for (int j = 0; j < 30; ++j) {
            double sg = (j % 2 == 0) ? 1.0 : -1.0; /* (-1)^j */
            s1 += sg * xj / fact1;
            s2 += -sg * (j + 1) * xj / fact2;
            if (j >= 1) {
                s3 += -sg * xj / fact1;
                s4 += sg * j * xj / fact2;
                s5 += -sg * xj / fact2;
            }
            xj *= x;
            fact1 *= (j + 2);
            fact2 *= (j + 3);
        }
        q[0] = dt * s1;
        q[1] = dt * dt * s2;
        q[2] = dt * s3;
        q[3] = dt * dt * s4;
        q[4] = dt * dt * s5;
    } else {
        double e = exp(-x);
        double om = -expm1(-x); /* 1 - e */
        q[0] = tau * om;
        q[1] = tau * dt * e - tau * tau * om;
        q[2] = dt - tau * om;
        q[3] = 2.0 * tau * tau * om - tau * dt * (1.0 + e);
        q[4] = 0.5 * dt * dt - tau * dt + tau * tau * om;
    }
}

/* Venkatakrishnan's limiter function (as published):
 *   phi = [(D1^2 + eps^2) D2 + 2 D2^2 D1] / [D2 (D1^2 + 2 D2^2 + D1 D2 + eps^2)],
 * phi = 1 when D2 = 0. */
double or_venkat(double d1, double d2, double eps2)
{
    if (d2 == 0.0) return 1.0;
    double num = (d1 * d1 + eps2) * d2 + 2.0 * d2 * d2 * d1;
    double den = d2 * (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2);
    return num / den;
}

void or_moment_matrix(int32_t D, int64_t nv, const double *u, const double *w, const double *W0,
                      double *M0)
{
    int M = D + 2;
    double rho, U[MAXD], lam;
    prim_of(D, W0, &rho, U, &lam);
    double nxi = 3.0 - D;
    for (int i = 0; i < M * M; ++i) M0[i] = 0.0;
    for (int64_t k = 0; k < nv; ++k) {
        double H, B, P[MAXM * MAXM];
        maxwell1(D, rho, U, lam, u + k * D, &H, &B);
        double X = nxi * (nxi + 2.0) / (4.0 * lam * lam) * H;
        psi_outer(D, u + k * D, H, B, X, P);
        for (int i = 0; i < M * M; ++i) M0[i] += w[k] * P[i];
    }
}

/* Interface equilibrium (Sec. 2.4; the equilibrium step of Algorithm 1).
 * READING: g0 is the Maxwellian of W0, the conservative moments of the
 * particles arriving from both sides, computed before the velocity loop from
 * the macroscopic reconstruction: W0 = sum_k w_k psi_k [H(u_n) g_L + (1-H(u_n)) g_R]
 * with g_L,R = Maxwellians of the face states, H the Heaviside function
 * (H(0) = 1/2).  The spatial slope a^(d) solves M0 a^(d) = dW0/dx_d, and the
 * time slope A follows from the compatibility condition
 * int psi (u.a + A) g0 = 0, i.e. M0 A = -sum_d sum_k w_k u_d (a^(d).psi) psi g0. */
/* Half-range moments of the Maxwellian (rho, U, lam), over u.n > 0 (sigma =
 * +1) or u.n < 0 (sigma = -1), added into W0.  The velocity splits into u_n
 * along the unit normal n and a tangential part; with U_n = U.n the normal
 * moments over the half line are
 *   <1>     = erfc(-sigma sqrt(lam) U_n) / 2,
 *   <u_n>   = U_n <1> + e,   e = sigma exp(-lam U_n^2) / (2 sqrt(pi lam)),
 *   <u_n^2> = (U_n^2 + 1/(2 lam)) <1> + U_n e,
 * while the D-1 tangential components (mean U - U_n n) and the 3-D internal
 * ones take full Gaussian moments (variance 1/(2 lam) each). */
static void half_range_moments(int D, double rho, const double *U, double lam, const double *n, double sigma,
                               double *W0)
{
    double Un = 0.0;
    for (int d = 0; d < D; ++d) Un += U[d] * n[d];
    const double m0 = 0.5 * erfc(-sigma * sqrt(lam) * Un);
    const double e = sigma * exp(-lam * Un * Un) / (2.0 * sqrt(M_PI * lam));
    const double m1 = Un * m0 + e;
    const double m2 = (Un * Un + 0.5 / lam) * m0 + Un * e;
    double Ut2 = 0.0;
    W0[0] += rho * m0;
    for (int d = 0; d < D; ++d) {
        const double Ut = U[d] - Un * n[d];
        Ut2 += Ut * Ut;
        W0[1 + d] += rho * (m1 * n[d] + Ut * m0);
    }
    /* (D - 1) tangential + (3 - D) internal components: 2 of variance 1/(2 lam) */
    W0[D + 1] += 0.5 * rho * (m2 + (Ut2 + 2.0 * 0.5 / lam) * m0);
}

void or_face_equilibrium(int32_t D, int64_t nv, const double *u, const double *w, const double *n,
                         const double *WL, const double *WR, const double *gradW0, double *W0,
                         double *a, double *A)
{
    or_face_equilibrium_ex(D, nv, u, w, n, WL, WR, gradW0, W0, a, A, 0);
}

void or_face_equilibrium_ex(int32_t D, int64_t nv, const double *u, const double *w, const double *n,
                            const double *WL, const double *WR, const double *gradW0, double *W0,
                            double *a, double *A, int analytic)
{
    int M = D + 2;
    double rL, UL[MAXD], lL, rR, UR[MAXD], lR;
    prim_of(D, WL, &rL, UL, &lL);
    prim_of(D, WR, &rR, UR, &lR);
    for (int m = 0; m < M; ++m) W0[m] = 0.0;
    if (analytic) {
        half_range_moments(D, rL, UL, lL, n, +1.0, W0);
        half_range_moments(D, rR, UR, lR, n, -1.0, W0);
    }
    for (int64_t k = 0; k < (analytic ? 0 : nv); ++k) {
        const double *uk = u + k * D;
        double un = 0.0, u2 = 0.0;
        for (int d = 0; d < D; ++d) {
            un += uk[d] * n[d];
            u2 += uk[d] * uk[d];
        }
        double HL, BL, HR, BR;
        maxwell1(D, rL, UL, lL, uk, &HL, &BL);
        maxwell1(D, rR, UR, lR, uk, &HR, &BR);
        double sL = un > 0.0 ? 1.0 : (un < 0.0 ? 0.0 : 0.5);
        double sR = 1.0 - sL;
        double h = sL * HL + sR * HR;
        double b = sL * BL + sR * BR;
        W0[0] += w[k] * h;
        for (int d = 0; d < D; ++d) W0[1 + d] += w[k] * uk[d] * h;
        W0[D + 1] += w[k] * 0.5 * (u2 * h + b);
    }
    double M0[MAXM * MAXM], Mt[MAXM * MAXM];
    or_moment_matrix(D, nv, u, w, W0, M0);
    for (int d = 0; d < D; ++d) {
        memcpy(Mt, M0, sizeof(double) * M * M);
        for (int m = 0; m < M; ++m) a[d * M + m] = gradW0[d * M + m];
        solve(M, Mt, a + d * M);
    }
    /* right-hand side of the compatibility condition */
    double rho0, U0[MAXD], lam0;
    prim_of(D, W0, &rho0, U0, &lam0);
    double nxi = 3.0 - D;
    double rhs[MAXM] = {0, 0, 0, 0, 0};
    for (int64_t k = 0; k < nv; ++k) {
        const double *uk = u + k * D;
        double H, B, P[MAXM * MAXM];
        maxwell1(D, rho0, U0, lam0, uk, &H, &B);
        double X = nxi * (nxi + 2.0) / (4.0 * lam0 * lam0) * H;
        psi_outer(D, uk, H, B, X, P);
        for (int d = 0; d < D; ++d)
            for (int i = 0; i < M; ++i) {
                double s = 0.0;
                for (int j = 0; j < M; ++j) s += P[i * M + j] * a[d * M + j];
                rhs[i] -= w[k] * uk[d] * s;
            }
    }
    memcpy(Mt, M0, sizeof(double) * M * M);
    for (int m = 0; m < M; ++m) A[m] = rhs[m];
    solve(M, Mt, A);
}

/* ------------------------------------------------------------------------ */
/* case set-up                                                               */
/* ------------------------------------------------------------------------ */

static void *dupa(const void *src, size_t bytes)
{
    void *p = malloc(bytes ? bytes : 1);
    if (src && bytes) memcpy(p, src, bytes);
    return p;
}

static double tau_of(const or_case *c, double rho, double lam)
{
    /* READING: VHS viscosity mu = mu_ref T^omega with
     * mu_ref = 15 sqrt(2 pi) Kn L_ref / (2 (5-2w)(7-2w)) (Bird's mean free path
     * at the reference state rho = T = 1); tau = mu / p, p = rho T. */
    double T = 1.0 / (2.0 * lam);
    return c->mu_ref * pow(T, c->p.omega) / (rho * T);
}

double or_mu_ref(const or_case *c) { return c->mu_ref; }

or_case *or_create(const or_mesh *m, const or_vgrid *v, const or_params *p,
                   const double *prim_init)
{
    or_case *c = (or_case *)calloc(1, sizeof(or_case));
    int D = m->dim;
    c->D = D;
    c->nc = (D == 2) ? 2 : 1;
    c->nxi = 3.0 - D;
    c->C = m->n_cells;
    c->F = m->n_faces;
    c->Nv = v->nv;
    int64_t C = c->C, F = c->F, Nv = c->Nv;
    c->cell_xc = dupa(m->cell_xc, sizeof(double) * C * D);
    c->cell_vol = dupa(m->cell_vol, sizeof(double) * C);
    c->face_cells = dupa(m->face_cells, sizeof(int64_t) * F * 2);
    c->face_n = dupa(m->face_n, sizeof(double) * F * D);
    c->face_S = dupa(m->face_S, sizeof(double) * F);
    c->face_xc = dupa(m->face_xc, sizeof(double) * F * D);
    c->face_type = dupa(m->face_type, sizeof(int32_t) * F);
    c->face_tag = dupa(m->face_tag, sizeof(int32_t) * F);
    c->face_shift = (double *)calloc((size_t)F * D, sizeof(double));
    if (m->face_shift) memcpy(c->face_shift, m->face_shift, sizeof(double) * F * D);
    c->u = dupa(v->u, sizeof(double) * Nv * D);
    c->w = dupa(v->w, sizeof(double) * Nv);
    c->p = *p;
    c->wall_T = dupa(p->wall_T, sizeof(double) * (p->n_walls > 0 ? p->n_walls : 0));
    c->wall_U = dupa(p->wall_U, sizeof(double) * 3 * (p->n_walls > 0 ? p->n_walls : 0));
    c->p.wall_T = c->wall_T;
    c->p.wall_U = c->wall_U;
    if (isinf(p->Kn))
        c->mu_ref = INFINITY;
    else
        c->mu_ref = 15.0 * sqrt(2.0 * M_PI) * p->Kn * p->L_ref /
                    (2.0 * (5.0 - 2.0 * p->omega) * (7.0 - 2.0 * p->omega));

    /* faces of each cell */
    c->cf_ptr = (int64_t *)calloc(C + 1, sizeof(int64_t));
    for (int64_t f = 0; f < F; ++f) {
        c->cf_ptr[c->face_cells[2 * f] + 1]++;
        if (c->face_cells[2 * f + 1] >= 0) c->cf_ptr[c->face_cells[2 * f + 1] + 1]++;
    }
    for (int64_t i = 0; i < C; ++i) c->cf_ptr[i + 1] += c->cf_ptr[i];
    int64_t ncf = c->cf_ptr[C];
    c->cf_face = (int64_t *)malloc(sizeof(int64_t) * ncf);
    c->cf_side = (int32_t *)malloc(sizeof(int32_t) * ncf);
    c->cf_r = (double *)malloc(sizeof(double) * ncf * D);
    int64_t *fill = (int64_t *)calloc(C, sizeof(int64_t));
    for (int64_t f = 0; f < F; ++f)
        for (int s = 0; s < 2; ++s) {
            int64_t i = c->face_cells[2 * f + s];
            if (i < 0) continue;
            int64_t slot = c->cf_ptr[i] + fill[i]++;
            c->cf_face[slot] = f;
            c->cf_side[slot] = s;
            for (int d = 0; d < D; ++d) {
                double xf = c->face_xc[f * D + d] - (s == 1 ? c->face_shift[f * D + d] : 0.0);
                c->cf_r[slot * D + d] = xf - c->cell_xc[i * D + d];
            }
        }
    free(fill);

    /* least-squares neighbours and coefficients (READING: weights 1/|d|^2,
     * a_ij = w_ij M_i^{-1} d_ij, walls excluded, far-field ghosts mirrored) */
    c->nb_ptr = (int64_t *)calloc(C + 1, sizeof(int64_t));
    for (int64_t i = 0; i < C; ++i) {
        int64_t cnt = 0;
        for (int64_t s = c->cf_ptr[i]; s < c->cf_ptr[i + 1]; ++s)
            if (c->face_type[c->cf_face[s]] != OR_WALL) ++cnt;
        c->nb_ptr[i + 1] = c->nb_ptr[i] + cnt;
    }
    int64_t nnb = c->nb_ptr[C];
    c->nb_id = (int64_t *)malloc(sizeof(int64_t) * (nnb ? nnb : 1));
    c->nb_a = (double *)malloc(sizeof(double) * (nnb ? nnb : 1) * D);
    double *dvec = (double *)malloc(sizeof(double) * (nnb ? nnb : 1) * D);
    c->eps2 = (double *)malloc(sizeof(double) * C);
    double hmin = INFINITY;
    for (int64_t i = 0; i < C; ++i) {
        int64_t n = c->nb_ptr[i];
        double sumS = 0.0;
        for (int64_t s = c->cf_ptr[i]; s < c->cf_ptr[i + 1]; ++s) {
            int64_t f = c->cf_face[s];
            int side = c->cf_side[s];
            sumS += c->face_S[f];
            int t = c->face_type[f];
            if (t == OR_WALL) continue;
            double d[MAXD];
            if (t == OR_FARFIELD) {
                double rn = 0.0;
                for (int e = 0; e < D; ++e) rn += c->cf_r[s * D + e] * c->face_n[f * D + e];
                for (int e = 0; e < D; ++e) d[e] = 2.0 * rn * c->face_n[f * D + e];
                c->nb_id[n] = -(f + 1);
            } else {
                int64_t j = c->face_cells[2 * f + (1 - side)];
                for (int e = 0; e < D; ++e) {
                    double sh = c->face_shift[f * D + e];
                    double xj = c->cell_xc[j * D + e] + (side == 0 ? sh : -sh);
                    d[e] = xj - c->cell_xc[i * D + e];
                }
                c->nb_id[n] = j;
            }
            for (int e = 0; e < D; ++e) dvec[n * D + e] = d[e];
            ++n;
        }
        /* normal matrix */
        double Mx[MAXD * MAXD] = {0};
        for (int64_t q = c->nb_ptr[i]; q < c->nb_ptr[i + 1]; ++q) {
            double dd = 0.0;
            for (int e = 0; e < D; ++e) dd += dvec[q * D + e] * dvec[q * D + e];
            double wq = 1.0 / dd;
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) Mx[a * D + b] += wq * dvec[q * D + a] * dvec[q * D + b];
        }
        double tr = 0.0;
        for (int a = 0; a < D; ++a) tr += Mx[a * D + a];
        double det = (D == 2) ? Mx[0] * Mx[3] - Mx[1] * Mx[2]
                              : Mx[0] * (Mx[4] * Mx[8] - Mx[5] * Mx[7]) -
                                    Mx[1] * (Mx[3] * Mx[8] - Mx[5] * Mx[6]) +
                                    Mx[2] * (Mx[3] * Mx[7] - Mx[4] * Mx[6]);
        int singular = !(fabs(det) > 1e-12 * pow(tr / D, D));
        for (int64_t q = c->nb_ptr[i]; q < c->nb_ptr[i + 1]; ++q) {
            if (singular) {
                for (int e = 0; e < D; ++e) c->nb_a[q * D + e] = 0.0;
                continue;
            }
            double dd = 0.0;
            for (int e = 0; e < D; ++e) dd += dvec[q * D + e] * dvec[q * D + e];
            double Mt[MAXD * MAXD], rhs[MAXD];
            memcpy(Mt, Mx, sizeof(Mt));
            for (int e = 0; e < D; ++e) rhs[e] = dvec[q * D + e] / dd;
            solve(D, Mt, rhs);
            for (int e = 0; e < D; ++e) c->nb_a[q * D + e] = rhs[e];
        }
        /* READING: h_i = 2 D |Omega_i| / sum_f S_f (edge length of a square or
         * cube, twice the inradius of a simplex); Venkatakrishnan eps^2 = (K h)^3 */
        double hi = 2.0 * D * c->cell_vol[i] / sumS;
        double hcfl = 2.0 * c->cell_vol[i] / sumS;
        if (hcfl < hmin) hmin = hcfl;
        double Kh = p->venkat_K * hi;
        c->eps2[i] = Kh * Kh * Kh;
    }
    free(dvec);

    /* READING (the CFL condition of Algorithm 1): the stability bound of the upwind finite-volume
     * update, dt <= |Omega_i| / sum_f S_f (u_k . n_f)^+; since the positive
     * part is at most |u_k| sum_f S_f / 2, dt = CFL min_i (2 |Omega_i| /
     * sum_f S_f) / max_k |u_k| (= CFL h_i / (D max|u|)), fixed for a fixed
     * velocity grid */
    double umax = 0.0;
    for (int64_t k = 0; k < Nv; ++k) {
        double s = 0.0;
        for (int d = 0; d < D; ++d) s += c->u[k * D + d] * c->u[k * D + d];
        if (sqrt(s) > umax) umax = sqrt(s);
    }
    c->dt = (p->dt > 0.0) ? p->dt : p->cfl * hmin / umax;

    /* wall faces */
    c->wall_slot_of_face = (int64_t *)malloc(sizeof(int64_t) * (F ? F : 1));
    c->n_wall = 0;
    for (int64_t f = 0; f < F; ++f) c->wall_slot_of_face[f] = (c->face_type[f] == OR_WALL) ? c->n_wall++ : -1;
    c->wall_face = (int64_t *)malloc(sizeof(int64_t) * (c->n_wall ? c->n_wall : 1));
    for (int64_t f = 0; f < F; ++f)
        if (c->wall_slot_of_face[f] >= 0) c->wall_face[c->wall_slot_of_face[f]] = f;

    /* state and work arrays */
    int M = D + 2, nc = c->nc;
    c->f = (double *)malloc(sizeof(double) * C * nc * Nv);
    c->W = (double *)malloc(sizeof(double) * C * M);
    c->Wold = (double *)malloc(sizeof(double) * C * M);
    c->q = (double *)calloc((size_t)C * D, sizeof(double));
    c->rho = (double *)malloc(sizeof(double) * C);
    c->U = (double *)malloc(sizeof(double) * C * D);
    c->lam = (double *)malloc(sizeof(double) * C);
    c->tau = (double *)malloc(sizeof(double) * C);
    c->gradW = (double *)malloc(sizeof(double) * C * D * M);
    c->gradP = (double *)malloc(sizeof(double) * C * D * M);
    c->P = (double *)malloc(sizeof(double) * C * M);
    c->Pg = (double *)malloc(sizeof(double) * (F ? F : 1) * M);
    c->Wghost = (double *)malloc(sizeof(double) * (F ? F : 1) * M);
    c->W0 = (double *)malloc(sizeof(double) * (F ? F : 1) * M);
    c->fa = (double *)malloc(sizeof(double) * (F ? F : 1) * D * M);
    c->fA = (double *)malloc(sizeof(double) * (F ? F : 1) * M);
    c->q0 = (double *)malloc(sizeof(double) * (F ? F : 1) * D);
    c->qs = (double *)malloc(sizeof(double) * (F ? F : 1) * 5);
    c->grad_k = (double *)malloc(sizeof(double) * C * nc * D);
    c->Fk = (double *)malloc(sizeof(double) * (F ? F : 1) * nc);
    c->Fm = (double *)calloc((size_t)(F ? F : 1) * M, sizeof(double));
    c->ghost_k = (double *)malloc(sizeof(double) * (F ? F : 1) * nc);
    size_t nwk = (size_t)(c->n_wall ? c->n_wall : 1) * Nv * nc;
    c->fin = (double *)malloc(sizeof(double) * nwk);
    c->gfin = (double *)malloc(sizeof(double) * nwk * D);
    c->rho_w = (double *)calloc((size_t)(c->n_wall ? c->n_wall : 1), sizeof(double));
    c->WLs = (double *)calloc((size_t)(F ? F : 1) * M, sizeof(double));
    c->WRs = (double *)calloc((size_t)(F ? F : 1) * M, sizeof(double));
    memset(c->res, 0, sizeof(c->res));

    /* initial condition: W^0 from the primitive state, f^0 = Maxwellian(W^0) */
    for (int64_t i = 0; i < C; ++i) {
        double pr[MAXM];
        if (prim_init) {
            for (int m2 = 0; m2 < M; ++m2) pr[m2] = prim_init[i * M + m2];
        } else {
            pr[0] = p->inf_rho;
            for (int d = 0; d < D; ++d) pr[1 + d] = p->inf_U[d];
            pr[D + 1] = p->inf_T;
        }
        double *Wi = c->W + i * M;
        double ke = 0.0;
        Wi[0] = pr[0];
        for (int d = 0; d < D; ++d) {
            Wi[1 + d] = pr[0] * pr[1 + d];
            ke += pr[1 + d] * pr[1 + d];
        }
        Wi[D + 1] = pr[0] * (0.5 * ke + 1.5 * pr[D + 1]);
        double rho, U[MAXD], lam;
        prim_of(D, Wi, &rho, U, &lam);
        for (int64_t k = 0; k < Nv; ++k) {
            double H, B;
            maxwell1(D, rho, U, lam, c->u + k * D, &H, &B);
            c->f[(i * nc + 0) * Nv + k] = H;
            if (nc == 2) c->f[(i * nc + 1) * Nv + k] = B;
        }
    }
    return c;
}

void or_destroy(or_case *c)
{
    if (!c) return;
    void *ptrs[] = {c->cell_xc, c->cell_vol, c->face_n, c->face_S, c->face_xc, c->face_shift,
                    c->face_cells, c->face_type, c->face_tag, c->u, c->w, c->wall_T, c->wall_U,
                    c->cf_ptr, c->cf_face, c->cf_side, c->cf_r, c->nb_ptr, c->nb_id, c->nb_a,
                    c->eps2, c->wall_face, c->wall_slot_of_face, c->f, c->W, c->Wold, c->q,
                    c->rho, c->U, c->lam, c->tau, c->gradW, c->Wghost, c->W0, c->fa, c->fA,
                    c->q0, c->qs, c->grad_k, c->Fk, c->Fm, c->fin, c->gfin, c->rho_w,
                    c->ghost_k, c->P, c->Pg, c->gradP, c->WLs, c->WRs};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(c);
}

double or_dt(const or_case *c) { return c->dt; }
int32_t or_ncomp(const or_case *c) { return c->nc; }

/* ------------------------------------------------------------------------ */
/* reconstruction (Sec. 3.1 Step 2)                                          */
/* ------------------------------------------------------------------------ */

/* Least-squares gradient of one scalar quantity at cell i.  val[j * stride] is
 * the value in cell j, gval[f] the value in the far-field ghost of face f.
 * With the limiter, the gradient is scaled by phi = min over all faces of i of
 * Venkatakrishnan's phi(D1, D2), D2 = grad.(x_f - x_i), D1 = max_j v_j - v_i
 * (D2 > 0) or min_j v_j - v_i (D2 < 0), the extrema taken over i and its
 * least-squares neighbours. */
static void lsq_gradient(const or_case *c, int64_t i, const double *val, int64_t stride,
                         const double *gval, int64_t gstride, int limited, double *g)
{
    int D = c->D;
    double vi = val[i * stride];
    double vmax = vi, vmin = vi;
    for (int d = 0; d < D; ++d) g[d] = 0.0;
    for (int64_t q = c->nb_ptr[i]; q < c->nb_ptr[i + 1]; ++q) {
        int64_t id = c->nb_id[q];
        double vj = (id >= 0) ? val[id * stride] : gval[(-id - 1) * gstride];
        for (int d = 0; d < D; ++d) g[d] += c->nb_a[q * D + d] * (vj - vi);
        if (vj > vmax) vmax = vj;
        if (vj < vmin) vmin = vj;
    }
    if (!limited) return;
    double phi = 1.0;
    for (int64_t s = c->cf_ptr[i]; s < c->cf_ptr[i + 1]; ++s) {
        double d2 = 0.0;
        for (int d = 0; d < D; ++d) d2 += g[d] * c->cf_r[s * D + d];
        double d1 = (d2 > 0.0) ? vmax - vi : vmin - vi;
        double ph = or_venkat(d1, d2, c->eps2[i]);
        if (ph < phi) phi = ph;
    }
    for (int d = 0; d < D; ++d) g[d] *= phi;
}

/* Micro reconstruction of f_k at cell i (Sec. 3.1 Step 2): the limited
 * least-squares slope, then scaled by theta in [0, 1] so that the linear
 * reconstruction is non-negative wherever the step evaluates it.
 * READING: f is a density; the free-transport part of the flux is a
 * positively weighted time average of f_i + grad f . (x_f - x_i - t u_k),
 * 0 <= t <= dt, so the reconstruction is required to be >= 0 at every face
 * centre (t = 0) and at the foot of the characteristic (t = dt).  If the
 * smallest of these values v is negative, theta = f_i / (f_i - v) (0 if
 * f_i <= 0); otherwise theta = 1 (a positivity-preserving scaling in the
 * manner of Zhang and Shu).  Venkatakrishnan's eps^2 = (K h)^3 is
 * dimensional and leaves small f (velocity tails, near-vacuum wakes)
 * unlimited, which is where the scaling acts. */
static void micro_gradient(const or_case *c, int64_t i, const double *val, int64_t stride,
                           const double *gval, int64_t gstride, const double *uk, double *g)
{
    int D = c->D;
    lsq_gradient(c, i, val, stride, gval, gstride, c->p.limiter, g);
    double vi = val[i * stride];
    double vmin = vi;
    for (int64_t s = c->cf_ptr[i]; s < c->cf_ptr[i + 1]; ++s) {
        double v0 = vi, v1 = vi;
        for (int d = 0; d < D; ++d) {
            v0 += g[d] * c->cf_r[s * D + d];
            v1 += g[d] * (c->cf_r[s * D + d] - c->dt * uk[d]);
        }
        if (v0 < vmin) vmin = v0;
        if (v1 < vmin) vmin = v1;
    }
    if (vmin < 0.0) {
        double theta = vi > 0.0 ? vi / (vi - vmin) : 0.0;
        for (int d = 0; d < D; ++d) g[d] *= theta;
    }
}

void or_micro_gradient(or_case *c, const double *phi, const double *phi_ghost, const double *uk,
                       double *grad)
{
    double *gv = (double *)malloc(sizeof(double) * (c->F ? c->F : 1));
    for (int64_t f = 0; f < c->F; ++f)
        gv[f] = phi_ghost ? phi_ghost[f] : phi[c->face_cells[2 * f]];
    for (int64_t i = 0; i < c->C; ++i) micro_gradient(c, i, phi, 1, gv, 1, uk, grad + i * c->D);
    free(gv);
}

void or_scalar_gradient(or_case *c, const double *phi, const double *phi_ghost, int32_t limited,
                        double *grad)
{
    double *gv = (double *)malloc(sizeof(double) * (c->F ? c->F : 1));
    for (int64_t f = 0; f < c->F; ++f)
        gv[f] = phi_ghost ? phi_ghost[f] : phi[c->face_cells[2 * f]];
    for (int64_t i = 0; i < c->C; ++i) lsq_gradient(c, i, phi, 1, gv, 1, limited, grad + i * c->D);
    free(gv);
}

/* face state from the primitive reconstruction P_i + grad P_i . r, returned
 * as conserved variables, with a positivity fallback (READING: if rho or T of
 * the extrapolated state is not positive, the cell average is used). */
static void face_state(const or_case *c, int64_t i, const double *r, double *Ws)
{
    int D = c->D, M = D + 2;
    double pf[MAXM];
    for (int m = 0; m < M; ++m) {
        double s = c->P[i * M + m];
        for (int d = 0; d < D; ++d) s += c->gradP[(i * D + d) * M + m] * r[d];
        pf[m] = s;
    }
    if (!(pf[0] > 0.0) || !(pf[D + 1] > 0.0))
        for (int m = 0; m < M; ++m) pf[m] = c->P[i * M + m];
    double ke = 0.0;
    Ws[0] = pf[0];
    for (int d = 0; d < D; ++d) {
        Ws[1 + d] = pf[0] * pf[1 + d];
        ke += pf[1 + d] * pf[1 + d];
    }
    Ws[D + 1] = pf[0] * (0.5 * ke + 1.5 * pf[D + 1]);
}

/* primitive variables (rho, U, T) of a conserved state */
static void to_primitive(int D, const double *W, double *P)
{
    double rho, U[MAXD], lam;
    prim_of(D, W, &rho, U, &lam);
    P[0] = rho;
    for (int d = 0; d < D; ++d) P[1 + d] = U[d];
    P[D + 1] = 1.0 / (2.0 * lam);
}

/* ------------------------------------------------------------------------ */
/* one time step (Algorithm 1)                                               */
/* ------------------------------------------------------------------------ */

static int nthreads(const or_case *c)
{
#ifdef _OPENMP
    return c->p.n_threads > 0 ? c->p.n_threads : omp_get_max_threads();
#else
    (void)c;
    return 1;
#endif
}

static void one_step(or_case *c)
{
    const int D = c->D, M = D + 2, nc = c->nc;
    const int64_t C = c->C, F = c->F, Nv = c->Nv;
    const double dt = c->dt, Pr = c->p.Pr, nxi = c->nxi;
    const int nt = nthreads(c);
    (void)nt;

    memcpy(c->Wold, c->W, sizeof(double) * C * M);

    /* ---- Algorithm 1: heat flux of each cell from f^n ---- */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < C; ++i) {
        prim_of(D, c->W + i * M, &c->rho[i], c->U + i * D, &c->lam[i]);
        c->tau[i] = tau_of(c, c->rho[i], c->lam[i]);
        const double *h = c->f + (i * nc) * Nv;
        const double *b = (nc == 2) ? c->f + (i * nc + 1) * Nv : NULL;
        or_heat_flux(D, Nv, c->u, c->w, h, b, c->U + i * D, c->q + i * D);
    }

    /* far-field ghost states (Sec. 2.5, READING: the free stream on faces where
     * it enters the domain, U_inf . n < 0; zero-gradient extrapolation elsewhere) */
    for (int64_t f = 0; f < F; ++f) {
        if (c->face_type[f] != OR_FARFIELD) continue;
        int64_t i = c->face_cells[2 * f];
        double un = 0.0;
        for (int d = 0; d < D; ++d) un += c->p.inf_U[d] * c->face_n[f * D + d];
        double *Wg = c->Wghost + f * M;
        if (un < 0.0) {
            double ke = 0.0;
            Wg[0] = c->p.inf_rho;
            for (int d = 0; d < D; ++d) {
                Wg[1 + d] = c->p.inf_rho * c->p.inf_U[d];
                ke += c->p.inf_U[d] * c->p.inf_U[d];
            }
            Wg[D + 1] = c->p.inf_rho * (0.5 * ke + 1.5 * c->p.inf_T);
        } else {
            for (int m = 0; m < M; ++m) Wg[m] = c->W[i * M + m];
        }
    }

    /* ---- Algorithm 1: macroscopic reconstruction ----
     * READING: the "gradients of macroscopic values" are least-squares
     * gradients of the primitive variables (rho, U, T), and the "gradient
     * compressor factors" of the cited sliding-mesh paper are taken as
     * Venkatakrishnan factors on each of them (the limiter of the micro
     * slopes).  Face states are reconstructed from these, so the face
     * temperature stays within the range of the neighbours'; limiting the
     * conserved components separately can leave a face temperature far below
     * every neighbour's, whose Maxwellian the velocity grid cannot resolve.
     * The conserved-variable gradient used for the slopes of g0 is the chain
     * rule of the limited primitive gradient at the cell state. */
    for (int64_t i = 0; i < C; ++i) to_primitive(D, c->W + i * M, c->P + i * M);
    for (int64_t f = 0; f < F; ++f)
        if (c->face_type[f] == OR_FARFIELD) to_primitive(D, c->Wghost + f * M, c->Pg + f * M);
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < C; ++i) {
        const double *Pi = c->P + i * M;
        for (int m = 0; m < M; ++m) {
            double g[MAXD];
            lsq_gradient(c, i, c->P + m, M, c->Pg + m, M, c->p.limiter, g);
            for (int d = 0; d < D; ++d) c->gradP[(i * D + d) * M + m] = g[d];
        }
        double uu = 0.0;
        for (int e = 0; e < D; ++e) uu += Pi[1 + e] * Pi[1 + e];
        for (int d = 0; d < D; ++d) {
            const double *gp = c->gradP + (i * D + d) * M;
            double *gw = c->gradW + (i * D + d) * M;
            double udu = 0.0;
            gw[0] = gp[0];
            for (int e = 0; e < D; ++e) {
                gw[1 + e] = Pi[1 + e] * gp[0] + Pi[0] * gp[1 + e];
                udu += Pi[1 + e] * gp[1 + e];
            }
            gw[D + 1] = gp[0] * (0.5 * uu + 1.5 * Pi[D + 1]) + Pi[0] * (udu + 1.5 * gp[D + 1]);
        }
    }

    /* ---- Algorithm 1: interface equilibrium and time coefficients ---- */
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
    for (int64_t f = 0; f < F; ++f) {
        int t = c->face_type[f];
        if (t == OR_WALL) continue;
        int64_t i = c->face_cells[2 * f], j = c->face_cells[2 * f + 1];
        double WL[MAXM], WR[MAXM], g0[MAXD * MAXM], rL[MAXD], rR[MAXD];
        for (int d = 0; d < D; ++d) rL[d] = c->face_xc[f * D + d] - c->cell_xc[i * D + d];
        face_state(c, i, rL, WL);
        if (t == OR_FARFIELD) {
            for (int m = 0; m < M; ++m) WR[m] = c->Wghost[f * M + m];
            for (int d = 0; d < D; ++d)
                for (int m = 0; m < M; ++m) g0[d * M + m] = 0.5 * c->gradW[(i * D + d) * M + m];
            for (int d = 0; d < D; ++d) c->q0[f * D + d] = 0.5 * c->q[i * D + d];
        } else {
            for (int d = 0; d < D; ++d)
                rR[d] = c->face_xc[f * D + d] - c->face_shift[f * D + d] - c->cell_xc[j * D + d];
            face_state(c, j, rR, WR);
            for (int d = 0; d < D; ++d)
                for (int m = 0; m < M; ++m)
                    g0[d * M + m] =
                        0.5 * (c->gradW[(i * D + d) * M + m] + c->gradW[(j * D + d) * M + m]);
            /* Sec. 3.2: interface heat flux = average of the two cells */
            for (int d = 0; d < D; ++d) c->q0[f * D + d] = 0.5 * (c->q[i * D + d] + c->q[j * D + d]);
        }
        for (int m = 0; m < M; ++m) {
            c->WLs[f * M + m] = WL[m];
            c->WRs[f * M + m] = WR[m];
        }
        or_face_equilibrium_ex(D, Nv, c->u, c->w, c->face_n + f * D, WL, WR, g0, c->W0 + f * M,
                               c->fa + f * D * M, c->fA + f * M, c->p.w0_analytic);
        double rho0, U0[MAXD], lam0;
        prim_of(D, c->W0 + f * M, &rho0, U0, &lam0);
        or_time_integrals(dt, tau_of(c, rho0, lam0), c->qs + f * 5);
        for (int m = 0; m < M; ++m) c->Fm[f * M + m] = 0.0;
    }

    /* ---- Algorithm 1: the velocity loop ---- */
    for (int64_t k = 0; k < Nv; ++k) {
        const double *uk = c->u + k * D;
        double u2 = 0.0;
        for (int d = 0; d < D; ++d) u2 += uk[d] * uk[d];

        /* ghost values of f_k: Maxwellian of the ghost state */
        for (int64_t f = 0; f < F; ++f) {
            if (c->face_type[f] != OR_FARFIELD) continue;
            double rg, Ug[MAXD], lg, H, B;
            prim_of(D, c->Wghost + f * M, &rg, Ug, &lg);
            maxwell1(D, rg, Ug, lg, uk, &H, &B);
            c->ghost_k[f * nc] = H;
            if (nc == 2) c->ghost_k[f * nc + 1] = B;
        }

        /* reconstruct f_k (limited, positivity-scaled slope per component) */
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int64_t i = 0; i < C; ++i)
            for (int cc = 0; cc < nc; ++cc)
                micro_gradient(c, i, c->f + cc * Nv + k, (int64_t)nc * Nv, c->ghost_k + cc, nc, uk,
                               c->grad_k + (i * nc + cc) * D);

        /* flux F_k through every non-wall face (Eq. microscopicFlux,
         * Eq. fullSolution) and its macroscopic contribution (Eq. macroscopicFlux) */
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int64_t f = 0; f < F; ++f) {
            int t = c->face_type[f];
            if (t == OR_WALL) continue;
            int64_t i = c->face_cells[2 * f], j = c->face_cells[2 * f + 1];
            const double *n = c->face_n + f * D;
            double un = 0.0;
            for (int d = 0; d < D; ++d) un += uk[d] * n[d];
            double Fh = 0.0, Fb = 0.0;
            if (un != 0.0) {
                double fup[2] = {0, 0}, ugf[2] = {0, 0};
                if (un > 0.0) {
                    for (int cc = 0; cc < nc; ++cc) {
                        const double *g = c->grad_k + (i * nc + cc) * D;
                        double v = c->f[(i * nc + cc) * Nv + k], ug = 0.0;
                        for (int d = 0; d < D; ++d) {
                            v += g[d] * (c->face_xc[f * D + d] - c->cell_xc[i * D + d]);
                            ug += uk[d] * g[d];
                        }
                        fup[cc] = v;
                        ugf[cc] = ug;
                    }
                } else if (t == OR_FARFIELD) {
                    for (int cc = 0; cc < nc; ++cc) fup[cc] = c->ghost_k[f * nc + cc];
                } else {
                    for (int cc = 0; cc < nc; ++cc) {
                        const double *g = c->grad_k + (j * nc + cc) * D;
                        double v = c->f[(j * nc + cc) * Nv + k], ug = 0.0;
                        for (int d = 0; d < D; ++d) {
                            double r = c->face_xc[f * D + d] - c->face_shift[f * D + d] -
                                       c->cell_xc[j * D + d];
                            v += g[d] * r;
                            ug += uk[d] * g[d];
                        }
                        fup[cc] = v;
                        ugf[cc] = ug;
                    }
                }
                /* equilibrium part g0 + g0+ and its slopes */
                double rho0, U0[MAXD], lam0, H0, B0, H0p, B0p;
                prim_of(D, c->W0 + f * M, &rho0, U0, &lam0);
                maxwell1(D, rho0, U0, lam0, uk, &H0, &B0);
                shakhov1(D, Pr, rho0, U0, lam0, c->q0 + f * D, uk, H0, &H0p, &B0p);
                double X0 = nxi * (nxi + 2.0) / (4.0 * lam0 * lam0) * H0;
                double ua_h = 0.0, ua_b = 0.0, At_h, At_b;
                for (int d = 0; d < D; ++d) {
                    double mh, mb;
                    psi_moment(D, uk, c->fa + (f * D + d) * M, H0, B0, X0, &mh, &mb);
                    ua_h += uk[d] * mh;
                    ua_b += uk[d] * mb;
                }
                psi_moment(D, uk, c->fA + f * M, H0, B0, X0, &At_h, &At_b);
                const double *qs = c->qs + f * 5;
                Fh = un * (qs[0] * fup[0] + qs[1] * ugf[0] + qs[2] * (H0 + H0p) + qs[3] * ua_h +
                           qs[4] * At_h);
                if (nc == 2)
                    Fb = un * (qs[0] * fup[1] + qs[1] * ugf[1] + qs[2] * (B0 + B0p) +
                               qs[3] * ua_b + qs[4] * At_b);
            }
            c->Fk[f * nc] = Fh;
            if (nc == 2) c->Fk[f * nc + 1] = Fb;
            double *Fm = c->Fm + f * M;
            Fm[0] += c->w[k] * Fh;
            for (int d = 0; d < D; ++d) Fm[1 + d] += c->w[k] * uk[d] * Fh;
            Fm[D + 1] += c->w[k] * 0.5 * (u2 * Fh + Fb);
        }

        /* interpolate f_k and its gradient to the wall faces */
        for (int64_t s = 0; s < c->n_wall; ++s) {
            int64_t f = c->wall_face[s];
            int64_t i = c->face_cells[2 * f];
            for (int cc = 0; cc < nc; ++cc) {
                const double *g = c->grad_k + (i * nc + cc) * D;
                double v = c->f[(i * nc + cc) * Nv + k];
                for (int d = 0; d < D; ++d) v += g[d] * (c->face_xc[f * D + d] - c->cell_xc[i * D + d]);
                size_t o = ((size_t)s * Nv + k) * nc + cc;
                c->fin[o] = v;
                for (int d = 0; d < D; ++d) c->gfin[o * D + d] = g[d];
            }
        }

        /* stage 1 (Eq. microS1) over non-wall faces, in place */
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int64_t i = 0; i < C; ++i) {
            double H, B, Hp, Bp;
            maxwell1(D, c->rho[i], c->U + i * D, c->lam[i], uk, &H, &B);
            shakhov1(D, Pr, c->rho[i], c->U + i * D, c->lam[i], c->q + i * D, uk, H, &Hp, &Bp);
            double fplus[2] = {H + Hp, B + Bp};
            for (int cc = 0; cc < nc; ++cc) {
                double sum = 0.0;
                for (int64_t s = c->cf_ptr[i]; s < c->cf_ptr[i + 1]; ++s) {
                    int64_t f = c->cf_face[s];
                    if (c->face_type[f] == OR_WALL) continue;
                    double sig = (c->cf_side[s] == 0) ? 1.0 : -1.0;
                    sum += sig * c->face_S[f] * c->Fk[f * nc + cc];
                }
                double *fi = c->f + (i * nc + cc) * Nv + k;
                double fn = *fi;
                *fi = fn - sum / c->cell_vol[i] + 0.5 * dt * (fplus[cc] - fn) / c->tau[i];
            }
        }
    }

    /* ---- Algorithm 1: flux at the walls (Sec. 2.5) ----
     * READING: outgoing particles (u_n > 0, n pointing into the wall) are
     * transported freely, f_in(-u t) = f_in - t u.grad f_in; incoming particles
     * carry g_w with rho_w from zero net mass flux (Eq. maxWalldes). */
    for (int64_t s = 0; s < c->n_wall; ++s) {
        int64_t f = c->wall_face[s];
        int64_t i = c->face_cells[2 * f];
        const double *n = c->face_n + f * D;
        int tag = c->face_tag[f];
        double Tw = c->wall_T[tag], lw = 1.0 / (2.0 * Tw), Uw[MAXD];
        for (int d = 0; d < D; ++d) Uw[d] = c->wall_U[3 * tag + d];
        double num = 0.0, den = 0.0;
        for (int64_t k = 0; k < Nv; ++k) {
            const double *uk = c->u + k * D;
            double un = 0.0, ug = 0.0;
            for (int d = 0; d < D; ++d) un += uk[d] * n[d];
            size_t o = ((size_t)s * Nv + k) * nc;
            for (int d = 0; d < D; ++d) ug += uk[d] * c->gfin[o * D + d];
            if (un > 0.0) {
                num += c->w[k] * un * (dt * c->fin[o] - 0.5 * dt * dt * ug);
            } else if (un < 0.0) {
                double H, B;
                maxwell1(D, 1.0, Uw, lw, uk, &H, &B);
                den += c->w[k] * un * dt * H;
            }
        }
        double rw = -num / den;
        c->rho_w[s] = rw;
        double *Fm = c->Fm + f * M;
        for (int m = 0; m < M; ++m) Fm[m] = 0.0;
        for (int64_t k = 0; k < Nv; ++k) {
            const double *uk = c->u + k * D;
            double un = 0.0, u2 = 0.0;
            for (int d = 0; d < D; ++d) {
                un += uk[d] * n[d];
                u2 += uk[d] * uk[d];
            }
            double Fw[2] = {0.0, 0.0};
            if (un > 0.0) {
                for (int cc = 0; cc < nc; ++cc) {
                    size_t o = ((size_t)s * Nv + k) * nc + cc;
                    double ug = 0.0;
                    for (int d = 0; d < D; ++d) ug += uk[d] * c->gfin[o * D + d];
                    Fw[cc] = un * (dt * c->fin[o] - 0.5 * dt * dt * ug);
                }
            } else if (un < 0.0) {
                double H, B;
                maxwell1(D, rw, Uw, lw, uk, &H, &B);
                Fw[0] = un * dt * H;
                Fw[1] = un * dt * B;
            }
            for (int cc = 0; cc < nc; ++cc)
                c->f[(i * nc + cc) * Nv + k] -= c->face_S[f] * Fw[cc] / c->cell_vol[i];
            Fm[0] += c->w[k] * Fw[0];
            for (int d = 0; d < D; ++d) Fm[1 + d] += c->w[k] * uk[d] * Fw[0];
            Fm[D + 1] += c->w[k] * 0.5 * (u2 * Fw[0] + (nc == 2 ? Fw[1] : 0.0));
        }
    }

    /* ---- Algorithm 1: W update (Eq. macroscopicUpdata) ---- */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < C; ++i) {
        for (int m = 0; m < M; ++m) {
            double sum = 0.0;
            for (int64_t s = c->cf_ptr[i]; s < c->cf_ptr[i + 1]; ++s) {
                int64_t f = c->cf_face[s];
                double sig = (c->cf_side[s] == 0) ? 1.0 : -1.0;
                sum += sig * c->face_S[f] * c->Fm[f * M + m];
            }
            c->W[i * M + m] = c->Wold[i * M + m] - sum / c->cell_vol[i];
        }
    }

    /* ---- Algorithm 1: stage 2 (Eq. microS2) with f+^{(n+1)} from W^{n+1}
     * READING: the Shakhov heat flux of f+^{(n+1)} is the lagged q^n ---- */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < C; ++i) {
        double rho, U[MAXD], lam;
        prim_of(D, c->W + i * M, &rho, U, &lam);
        double tau1 = tau_of(c, rho, lam);
        for (int64_t k = 0; k < Nv; ++k) {
            const double *uk = c->u + k * D;
            double H, B, Hp, Bp;
            maxwell1(D, rho, U, lam, uk, &H, &B);
            shakhov1(D, Pr, rho, U, lam, c->q + i * D, uk, H, &Hp, &Bp);
            double fplus[2] = {H + Hp, B + Bp};
            for (int cc = 0; cc < nc; ++cc) {
                double *fi = c->f + (i * nc + cc) * Nv + k;
                *fi = (*fi + 0.5 * dt * fplus[cc] / tau1) / (1.0 + dt / (2.0 * tau1));
            }
        }
    }

    /* residual per conserved component */
    for (int m = 0; m < M; ++m) {
        double a = 0.0, b = 0.0;
        for (int64_t i = 0; i < C; ++i) {
            double d = c->W[i * M + m] - c->Wold[i * M + m];
            a += d * d;
            b += c->Wold[i * M + m] * c->Wold[i * M + m];
        }
        c->res[m] = (b > 0.0) ? sqrt(a) / sqrt(b) : sqrt(a);
    }
}

void or_step(or_case *c, int32_t nsteps)
{
    for (int32_t s = 0; s < nsteps; ++s) one_step(c);
}

void or_get_state(or_case *c, double *f, double *W, double *q)
{
    int D = c->D, M = D + 2, nc = c->nc;
    if (f) memcpy(f, c->f, sizeof(double) * c->C * nc * c->Nv);
    if (W) memcpy(W, c->W, sizeof(double) * c->C * M);
    if (q) {
        for (int64_t i = 0; i < c->C; ++i) {
            double rho, U[MAXD], lam;
            prim_of(D, c->W + i * M, &rho, U, &lam);
            const double *h = c->f + (i * nc) * c->Nv;
            const double *b = (nc == 2) ? c->f + (i * nc + 1) * c->Nv : NULL;
            or_heat_flux(D, c->Nv, c->u, c->w, h, b, U, q + i * D);
        }
    }
}

void or_set_state(or_case *c, const double *f, const double *W)
{
    if (f) memcpy(c->f, f, sizeof(double) * c->C * c->nc * c->Nv);
    if (W) memcpy(c->W, W, sizeof(double) * c->C * (c->D + 2));
}

void or_residual(const or_case *c, double *res)
{
    for (int m = 0; m < c->D + 2; ++m) res[m] = c->res[m];
}

void or_wall_rho(const or_case *c, double *rho_w)
{
    for (int64_t s = 0; s < c->n_wall; ++s) rho_w[s] = c->rho_w[s];
}

/* Surface quantities at every wall face, in face order (Sec. 2.5): with F_w
 * the macroscopic wall flux of Eq. macroscopicFlux over the last step,
 * F_mw its momentum part and n_w the face normal (out of the fluid cell,
 * into the wall), p_w = F_mw . n_w, sigma_w = |F_mw - p_w n_w|, q_w = F_w4
 * (the energy component).  READING: F_w is integrated over the step, so the
 * surface quantities are taken as its time average F_w / dt.  Zero before
 * the first step. */
void or_wall_quantities(const or_case *c, double *p, double *sigma, double *q)
{
    const int D = c->D, M = D + 2;
    for (int64_t s = 0; s < c->n_wall; ++s) {
        const int64_t f = c->wall_face[s];
        const double *Fm = c->Fm + f * M;
        const double *n = c->face_n + f * D;
        double pn = 0.0;
        for (int d = 0; d < D; ++d) pn += Fm[1 + d] * n[d];
        double t2 = 0.0;
        for (int d = 0; d < D; ++d) {
            const double t = Fm[1 + d] - pn * n[d];
            t2 += t * t;
        }
        p[s] = pn / c->dt;
        sigma[s] = sqrt(t2) / c->dt;
        q[s] = Fm[D + 1] / c->dt;
    }
}

/* face states of the last step: the reconstructed W_L (owner side) and W_R
 * (neighbour side, or the far-field ghost state) of every non-wall face, as
 * conserved variables [F][D+2]; zero at wall faces and before the first step */
void or_face_states(const or_case *c, double *WL, double *WR)
{
    const size_t n = (size_t)c->F * (c->D + 2);
    if (WL) memcpy(WL, c->WLs, sizeof(double) * n);
    if (WR) memcpy(WR, c->WRs, sizeof(double) * n);
}

void or_face_macro_flux(const or_case *c, double *F)
{
    memcpy(F, c->Fm, sizeof(double) * c->F * (c->D + 2));
}

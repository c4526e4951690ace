/*
 * ugks_oracle.h -- plain FP64 CPU oracle of one explicit UGKS time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA library under paper_2412_06546_gb300/.
 *
 * It follows the paper "An efficiency and memory-saving programming paradigm
 * for the unified gas-kinetic scheme" (Zhang, Wei, Long, Xu, arXiv:2412.06546):
 * the BGK-Shakhov model and reduced distributions (Sec. 2.1-2.2), the finite
 * volume update (Sec. 2.3, Eq. microscopicFlux / macroscopicUpdata /
 * macroscopicFlux), the interface solution with c1..c5 (Sec. 2.4, Eq.
 * fullSolution), ghost far field and Maxwell walls (Sec. 2.5, Eq. maxWalldes),
 * the trapezoid source term (Sec. 2.6) and the two-stage update in the order of
 * Algorithm 1 (Sec. 3.2, Eq. microS1 / microS2).
 *
 * Units: R = 1, reference density and temperature 1; lambda = 1/(2T).
 * Layout: f[cell][comp][k], comp 0 = h, comp 1 = b (2D only; b == 0 in 3D).
 */
#ifndef UGKS_ORACLE_H
#define UGKS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_INTERIOR = 0, OR_WALL = 1, OR_FARFIELD = 2, OR_PERIODIC = 3 };

typedef struct {
    int32_t dim;
    int64_t n_cells, n_faces;
    const double *cell_xc, *cell_vol;
    const int64_t *face_cells;
    const double *face_n, *face_S, *face_xc;
    const int32_t *face_type, *face_tag;
    const double *face_shift; /* may be NULL */
} or_mesh;

typedef struct {
    int32_t dim;
    int64_t nv;
    const double *u, *w;
} or_vgrid;

typedef struct {
    double Kn, L_ref, Pr, omega, cfl, dt; /* dt <= 0: from the CFL number */
    int32_t limiter;                      /* Venkatakrishnan on (1) / off (0) */
    double venkat_K;
    int32_t n_walls;
    const double *wall_T;   /* [n_walls] */
    const double *wall_U;   /* [n_walls][3] */
    double inf_rho, inf_U[3], inf_T;
    int32_t n_threads;      /* OpenMP threads, <= 0: library default */
    int32_t w0_analytic;    /* 1: W0 from the analytic half-range moments (continuous velocity
                               space) instead of the discrete sums over the velocity set */
} or_params;

typedef struct or_case or_case;

/* prim_init[C][D+2] = (rho, U_1..U_D, T); NULL -> the far-field state. */
or_case *or_create(const or_mesh *m, const or_vgrid *v, const or_params *p,
                   const double *prim_init);
void or_destroy(or_case *c);
void or_step(or_case *c, int32_t nsteps);
double or_dt(const or_case *c);
int32_t or_ncomp(const or_case *c);
/* f[C][ncomp][Nv], W[C][D+2], q[C][D] (heat flux of the current f; any may be NULL) */
void or_get_state(or_case *c, double *f, double *W, double *q);
void or_set_state(or_case *c, const double *f, const double *W);
/* residual of the last step: |W^{n+1}_m - W^n_m|_2 / |W^n_m|_2 per component */
void or_residual(const or_case *c, double *res);
/* wall density of each wall face in the last step (face order), may be NULL-safe */
void or_wall_rho(const or_case *c, double *rho_w);
/* face states W_L, W_R[F][D+2] (conserved) of the last step: the primitive
 * reconstruction of each side at the face centre; at far-field faces W_R is the
 * ghost state (W_inf on inflow faces, the owner's state elsewhere); zero at walls */
void or_face_states(const or_case *c, double *WL, double *WR);
/* macroscopic flux of every face in the last step, F[F][D+2] */
void or_face_macro_flux(const or_case *c, double *F);
/* p_w, sigma_w, q_w of the last step at every wall face (face order), Sec. 2.5 */
void or_wall_quantities(const or_case *c, double *p, double *sigma, double *q);

/* ---- building blocks, exported for the pin tests ---- */
/* Eq. c1..c5 integrated over [0, dt]; tau may be +inf */
void or_time_integrals(double dt, double tau, double q[5]);
/* reduced Maxwellian H, B at velocities u[nv][D] */
void or_maxwellian(int32_t D, double rho, const double *U, double lam, int64_t nv,
                   const double *u, double *H, double *B);
/* reduced Shakhov corrections H+, B+ (Sec. 2.2) */
void or_shakhov(int32_t D, double Pr, double rho, const double *U, double lam,
                const double *q, int64_t nv, const double *u, double *Hp, double *Bp);
/* heat flux 1/2 sum_k w c (|c|^2 h + b) of one cell row */
void or_heat_flux(int32_t D, int64_t nv, const double *u, const double *w,
                  const double *h, const double *b, const double *U, double *q);
/* Venkatakrishnan limiter function phi(D1, D2, eps^2) */
double or_venkat(double d1, double d2, double eps2);
/* interface equilibrium of Sec. 2.4: from the face states W_L, W_R (normal n),
 * the interface macro gradient gradW0[D][D+2] -> W0[D+2], a[D][D+2], A[D+2] */
void or_face_equilibrium(int32_t D, int64_t nv, const double *u, const double *w,
                         const double *n, const double *WL, const double *WR,
                         const double *gradW0, double *W0, double *a, double *A);
/* the same, with W0 from the analytic half-range moments when analytic != 0 */
void or_face_equilibrium_ex(int32_t D, int64_t nv, const double *u, const double *w, const double *n,
                            const double *WL, const double *WR, const double *gradW0, double *W0,
                            double *a, double *A, int analytic);
/* moment matrix M0[(D+2)^2] of the Maxwellian of W0 on the discrete grid */
void or_moment_matrix(int32_t D, int64_t nv, const double *u, const double *w,
                      const double *W0, double *M0);
/* least-squares (optionally limited) gradient of a scalar cell field; ghost
 * values per face (far-field faces only; NULL -> owner value) */
void or_scalar_gradient(or_case *c, const double *phi, const double *phi_ghost,
                        int32_t limited, double *grad);
/* micro reconstruction of a scalar field at velocity u (limited least-squares
 * slope with the positivity scaling of the oracle's step) */
void or_micro_gradient(or_case *c, const double *phi, const double *phi_ghost, const double *uk,
                       double *grad);
/* mu_ref and tau of the VHS viscosity law used by the case */
double or_mu_ref(const or_case *c);

#ifdef __cplusplus
}
#endif
#endif

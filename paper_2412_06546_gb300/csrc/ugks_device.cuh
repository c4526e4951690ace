// ugks_device.cuh -- device-side data layout and per-velocity building blocks
// of the GB300 UGKS library (internal; not part of the C ABI).
//
// Layout in HBM (internal cell order = Morton order of the centroids):
//   f      [C][NC][nvp]  T   distribution, NC = 2 (h, b) in 2D, 1 (h) in 3D,
//                            velocity contiguous, padded to a multiple of the
//                            velocity tile (padded velocities have u = 0, w = 0)
//   W      [C][D+2]      f64 conserved variables
//   q      [C][D]        f64 heat flux of f^n
//   cell records [C][CREC] T   Maxwellian / Shakhov / collision coefficients
//   face records [F][FREC] T   interface equilibrium g0, its slopes, q1..q5
// T is the per-velocity arithmetic type (double or float).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ugks {

constexpr int MAXD = 3;
constexpr int MAXM = 5;

// cell record: Maxwellian of the cell state plus Shakhov and collision factors
enum { CR_U = 0, CR_LAM = 3, CR_PREF = 4, CR_KQ = 5, CR_C = 8, CR_NB = 9, CREC = 12 };
// ghost / side / wall record: a Maxwellian
enum { GR_U = 0, GR_LAM = 3, GR_PREF = 4, GR_NB = 5, GREC = 8 };
// face record: g0 of the interface, Shakhov factor, time integrals, slopes in
// the basis centred at U0: psi_c = (1, c, (|c|^2 + xi^2)/2), c = u - U0
enum { FR_U = 0, FR_LAM = 3, FR_PREF = 4, FR_KQ = 5, FR_QS = 8, FR_NB = 13, FR_XB = 14,
       FR_BETA = 15, FREC = 40 };

enum { FT_INTERIOR = 0, FT_WALL = 1, FT_FARFIELD = 2, FT_PERIODIC = 3 };

// Everything a kernel needs, by value.  Geometry used inside velocity loops is
// held in the arithmetic type T; macroscopic data is FP64.
template <typename T>
struct DevCase {
    int D, NC;
    int C, F, G, NW;         // cells, faces, far-field ghosts, wall faces
    int nv, nvp;             // velocities, padded count
    double dt, Pr, omega, mu_ref, nxi;
    int limiter;
    // velocity grid (padded), FP64 and T copies
    const double *ud[3], *wd;
    const T *u[3], *w;
    // distribution: f_cur = f^n, f_nxt = f~ written by the gather pass
    T *f_cur, *f_nxt;
    // macroscopic state
    double *W, *q, *gradW, *vol;
    double *prim, *primg, *gradprim;  // primitive (rho, U, T) of cells / ghosts, limited gradient
    // least squares (CSR over cells)
    const int *nb_ptr, *nb_id;    // id >= 0: cell, id < 0: ghost -(id+1)
    const double *nb_a_d;
    const T *nb_a;
    // faces of each cell (CSR): limiter offsets and gather entries
    const int *cf_ptr, *cf_face;
    const signed char *cf_side;   // 0 owner, 1 neighbour
    const double *cf_r_d;
    const T *cf_r;                // x_f - x_c (periodic image on the neighbour side)
    const T *cf_coef;             // -sigma S_f / |Omega_c|
    const short *cf_sL, *cf_sR;   // local slope slot of the owner / neighbour in the patch
    const double *eps2_d;
    const T *eps2;
    // faces
    const int *fL, *fR, *faux;    // owner, neighbour (-1 at boundaries), ghost or wall slot
    const signed char *ftype;
    const double *fn_d, *frL_d, *frR_d;
    const T *fn;
    // ghosts (one per far-field face)
    const int *gface;
    double *Wg;                   // [G][D+2]
    T *grec;                      // [G][GREC]
    // walls
    const int *wface;             // [NW] face id
    const double *wallT, *wallU;  // per wall tag
    const int *ftag;
    double inf_W[MAXM];
    double *rho_w;                // [NW]
    T *wrec;                      // [NW][GREC]
    // per-step work
    T *crec;                      // [C][CREC] stage-1 record (W^n, q^n)
    T *krec;                      // [C][CREC] stage-2 record (W^{n+1}, q^n)
    T *frec;                      // [F][FREC]
    T *fside;                     // [F][2][GREC] Maxwellians of the face states
    double *fdW0;                 // [F][D][D+2] interface macro gradient
    double *fq0;                  // [F][D]
    double *fUref;                // [F][D]
    double *fsum1, *fsum2;        // [F][S1], [F][S2]
    double *fprim0;               // [F][D+2] rho0, U0, lam0
    double *dW_part;              // [C][n_vt][D+2]
    double *res_part;             // [n_res_blocks][2(D+2)]
    int *flags;                   // [1] numeric failure flag
    // gather tiling
    int P, n_patches, n_vt, vtile;
    const int *ring_ptr, *ring_cells;
};

// ------------------------------------------------------------------ math
template <typename T> __device__ __forceinline__ T dexp(T x);
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }

template <typename T> __device__ __forceinline__ T mul_rn(T a, T b);
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T add_rn(T a, T b);
template <> __device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }

// u . n without contraction: the upwind and half-range decisions are taken
// from exactly the same rounded value as the oracle computes
template <typename T, int D>
__device__ __forceinline__ T normal_velocity(const T u[3], const T *n)
{
    T s = mul_rn(u[0], n[0]);
    s = add_rn(s, mul_rn(u[1], n[1]));
    if (D == 3) s = add_rn(s, mul_rn(u[2], n[2]));
    return s;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Maxwellian H and the b-factor of a record (cell / ghost / side / wall)
template <typename T, int D>
__device__ __forceinline__ T maxwell_h(const T *rec, const T u[3])
{
    T c2 = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        T c = u[d] - rec[GR_U + d];
        c2 += c * c;
    }
    return rec[GR_PREF] * dexp(-rec[GR_LAM] * c2);
}

// Shakhov equilibrium f+ = (H + H+, B + B+) of a cell record at velocity u:
// H+ = kappa (c.q)(2 lam c^2 - D - 2) H,  B+ = kappa (c.q)(2 lam c^2 - D) nb H
template <typename T, int D, int NC>
__device__ __forceinline__ void shakhov_fplus(const T *rec, const T u[3], T fp[NC])
{
    T c[D], c2 = 0, kqc = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        c[d] = u[d] - rec[CR_U + d];
        c2 += c[d] * c[d];
        kqc += rec[CR_KQ + d] * c[d];
    }
    T H = rec[CR_PREF] * dexp(-rec[CR_LAM] * c2);
    T l2c2 = T(2) * rec[CR_LAM] * c2;
    fp[0] = H * (T(1) + kqc * (l2c2 - T(D + 2)));
    if (NC == 2) fp[NC - 1] = H * rec[CR_NB] * (T(1) + kqc * (l2c2 - T(D)));
}

// Micro reconstruction of cell c at velocity index k (Sec. 3.1 Step 2):
// least-squares slope grad = sum_j a_cj (f_j - f_c), Venkatakrishnan factor
// phi = min over the faces of c of (D1^2 + eps^2 + 2 D1 D2) / (D1^2 + 2 D2^2 +
// D1 D2 + eps^2), then a positivity scaling theta so that the reconstruction is
// non-negative at every face centre and at the foot of the characteristic
// after one step: with dmin = min(0, min_f D2_f),
// v = f_c + phi (dmin + min(0, -dt u.grad)); theta = f_c / (f_c - v) if v < 0.
template <typename T, int D, int NC>
__device__ __forceinline__ void cell_slope(const DevCase<T> &dc, const T *__restrict__ f, int c, int k,
                                           const T u[3], T g[NC][D])
{
    const size_t rs = (size_t)NC * dc.nvp;
    T fi[NC], vmax[NC], vmin[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        fi[m] = f[(size_t)c * rs + (size_t)m * dc.nvp + k];
        vmax[m] = vmin[m] = fi[m];
#pragma unroll
        for (int d = 0; d < D; ++d) g[m][d] = 0;
    }
    const int q0 = dc.nb_ptr[c], q1 = dc.nb_ptr[c + 1];
    for (int q = q0; q < q1; ++q) {
        const int id = dc.nb_id[q];
        T fj[NC];
        if (id >= 0) {
#pragma unroll
            for (int m = 0; m < NC; ++m) fj[m] = f[(size_t)id * rs + (size_t)m * dc.nvp + k];
        } else {
            const T *gr = dc.grec + (size_t)(-id - 1) * GREC;
            T H = maxwell_h<T, D>(gr, u);
            fj[0] = H;
            if (NC == 2) fj[NC - 1] = gr[GR_NB] * H;
        }
        T a[D];
#pragma unroll
        for (int d = 0; d < D; ++d) a[d] = dc.nb_a[(size_t)q * D + d];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            T df = fj[m] - fi[m];
#pragma unroll
            for (int d = 0; d < D; ++d) g[m][d] += a[d] * df;
            vmax[m] = fj[m] > vmax[m] ? fj[m] : vmax[m];
            vmin[m] = fj[m] < vmin[m] ? fj[m] : vmin[m];
        }
    }
    const T e2 = dc.eps2[c];
    T phi[NC], dmin[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        phi[m] = T(1);
        dmin[m] = T(0);
    }
    const int s0 = dc.cf_ptr[c], s1 = dc.cf_ptr[c + 1];
    for (int s = s0; s < s1; ++s) {
        T r[D];
#pragma unroll
        for (int d = 0; d < D; ++d) r[d] = dc.cf_r[(size_t)s * D + d];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            T d2 = 0;
#pragma unroll
            for (int d = 0; d < D; ++d) d2 += g[m][d] * r[d];
            dmin[m] = d2 < dmin[m] ? d2 : dmin[m];
            if (dc.limiter) {
                T d1 = d2 > T(0) ? vmax[m] - fi[m] : vmin[m] - fi[m];
                T a2 = d1 * d1 + e2;
                T num = a2 + T(2) * d1 * d2;
                T den = a2 + d2 * (T(2) * d2 + d1);
                T ph = den > T(0) ? num / den : T(1);
                phi[m] = ph < phi[m] ? ph : phi[m];
            }
        }
    }
    const T dt = (T)dc.dt;
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        T ug = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) ug += u[d] * g[m][d];
        const T foot = -dt * ug;
        const T v = fi[m] + phi[m] * (dmin[m] + (foot < T(0) ? foot : T(0)));
        T s = phi[m];
        if (v < T(0)) s *= fi[m] > T(0) ? fi[m] / (fi[m] - v) : T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) g[m][d] *= s;
    }
}

// Interface flux of Eq. microscopicFlux with the distribution of Eq.
// fullSolution integrated over the step (time integrals q1..q5 in the record):
// F = u_n [q1 f_up + q2 u.grad f_up + q3 (g0 + g0+) + q4 u.grad g0 + q5 dg0/dt]
template <typename T, int D, int NC>
__device__ __forceinline__ void interface_flux(const T *__restrict__ fr, const T u[3], T un,
                                               const T fup[NC], const T ugf[NC], T F[NC])
{
    T c[D], c2 = 0, kqc = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        c[d] = u[d] - fr[FR_U + d];
        c2 += c[d] * c[d];
        kqc += fr[FR_KQ + d] * c[d];
    }
    const T lam = fr[FR_LAM];
    const T H0 = fr[FR_PREF] * dexp(-lam * c2);
    const T nb = fr[FR_NB], xb = fr[FR_XB];
    const T l2c2 = T(2) * lam * c2;
    const T hc2 = T(0.5) * c2;
    T ua_h = 0, ua_b = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const T *b = fr + FR_BETA + d * (D + 2);
        T phi = b[0] + b[D + 1] * hc2;
#pragma unroll
        for (int e = 0; e < D; ++e) phi += b[1 + e] * c[e];
        ua_h += u[d] * (phi + T(0.5) * b[D + 1] * nb);
        if (NC == 2) ua_b += u[d] * (phi * nb + T(0.5) * b[D + 1] * xb);
    }
    const T *bA = fr + FR_BETA + D * (D + 2);
    T phiA = bA[0] + bA[D + 1] * hc2;
#pragma unroll
    for (int e = 0; e < D; ++e) phiA += bA[1 + e] * c[e];
    const T *qs = fr + FR_QS;
    T sh_h = T(1) + kqc * (l2c2 - T(D + 2));
    T At_h = phiA + T(0.5) * bA[D + 1] * nb;
    F[0] = un * (qs[0] * fup[0] + qs[1] * ugf[0] + H0 * (qs[2] * sh_h + qs[3] * ua_h + qs[4] * At_h));
    if (NC == 2) {
        T sh_b = nb * (T(1) + kqc * (l2c2 - T(D)));
        T At_b = phiA * nb + T(0.5) * bA[D + 1] * xb;
        F[NC - 1] = un * (qs[0] * fup[NC - 1] + qs[1] * ugf[NC - 1] +
                          H0 * (qs[2] * sh_b + qs[3] * ua_b + qs[4] * At_b));
    }
}

}  // namespace ugks

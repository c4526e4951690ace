// ugks_kernels.cu -- the CUDA kernels of one UGKS time step (sm_103a).
//
// One step (Algorithm 1 of arXiv:2412.06546, reorganised for the GPU):
//   k_prep        cell records from W^n, q^n; far-field ghost states     (CFL and heat-flux step, Sec. 2.5)
//   k_macro_grad  limited least-squares gradient of W                    (macroscopic reconstruction)
//   k_face_pre    face states W_L, W_R, interface macro gradient, q0     (interface equilibrium)
//   k_face_sum1   half-range moments over the velocity grid -> W0        (Sec. 2.4)
//   k_face_fin1   g0 parameters, tau0, time integrals q1..q5             (Sec. 2.4)
//   k_face_sum2   moments of g0 for the slope systems                    (Sec. 2.4)
//   k_face_fin2   spatial and time slopes of g0                          (Sec. 2.4)
//   k_wall_sum    wall density from zero net mass flux                   (Eq. maxWalldes)
//   k_gather      per (cell patch, velocity tile): micro slopes, face fluxes, stage 1,
//                 moments of the flux residual                           (velocity loop, Eq. microS1)
//   k_update_W    W^{n+1} and stage-2 coefficients                       (Eq. macroscopicUpdata)
//   k_collide     stage 2 and the heat flux of f^{n+1}                   (Eq. microS2)
// All per-velocity arithmetic is in T (double or float).  Velocity-moment sums
// are FP64 in the FP64 form.  In the FP32 form the products are FP32 and the
// sums are accumulated in FP64: the face sums from FP32 block partials of at
// most SUM_BLOCK terms per lane (see block_to_fp64), the wall density and the
// heat flux from Kahan-compensated lane sums, the moments of the flux residual
// from double-float lane and warp sums.  Macroscopic scalars (W, the
// equilibrium parameters, the heat flux, the collision coefficients) are
// formed in FP64.
#include "ugks_device.cuh"
#include "ugks_kernels.h"

#include <algorithm>
#include <type_traits>
#include <cmath>

namespace ugks {

// ------------------------------------------------------------ FP64 helpers
struct Prim {
    double rho, U[MAXD], lam, T;
};

__device__ __forceinline__ Prim prim_of(const double *W, int D)
{
    Prim p;
    p.rho = W[0];
    double ke = 0.0;
    for (int d = 0; d < MAXD; ++d) p.U[d] = 0.0;
    for (int d = 0; d < D; ++d) {
        p.U[d] = W[1 + d] / W[0];
        ke += p.U[d] * p.U[d];
    }
    double E = W[D + 1] / W[0];
    p.T = (2.0 / 3.0) * (E - 0.5 * ke);
    p.lam = 1.0 / (2.0 * p.T);
    return p;
}

constexpr double LOG2E = 1.4426950408889634073599246810018921;

__device__ __forceinline__ double pref_of(double rho, double lam, int D)
{
    double a = lam / 3.141592653589793238462643383279502884;
    return D == 2 ? rho * a : rho * a * sqrt(a);
}

// collision time tau = mu_ref T^omega / (rho T)  (VHS viscosity, p = rho T)
template <typename T>
__device__ __forceinline__ double tau_of(const DevCase<T> &dc, double rho, double Tmp)
{
    return dc.mu_ref * pow(Tmp, dc.omega) / (rho * Tmp);
}

// Time integrals of c1..c5 over [0, dt] (Sec. 2.4), written with x = dt/tau,
// E = 1 - e^{-x}:  q1 = dt E/x, q2 = dt^2 (x e^{-x} - E)/x^2, q3 = dt (x - E)/x,
// q4 = dt^2 (2E - x(1 + e^{-x}))/x^2, q5 = dt^2 (x^2/2 - x + E)/x^2.
// Below x = 1/2 each bracket is summed from its Taylor series.
__device__ void time_integrals(double dt, double tau, double q[5])
{
    const double x = dt / tau;
    if (x < 0.5) {
        double s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
        double xp = 1.0;       // x^{j-2} for j >= 2
        double inv_fact = 1.0; // 1/j!
        double xm1 = 1.0;      // x^{j-1}
        for (int j = 1; j <= 22; ++j) {
            inv_fact /= (double)j;
            const double sg = (j & 1) ? 1.0 : -1.0;   // (-1)^{j+1}
            s1 += sg * xm1 * inv_fact;                  // E/x
            if (j >= 2) {
                const double xm2 = xp;                  // x^{j-2}
                s2 += sg * (1.0 - (double)j) * xm2 * inv_fact;   // (E - x e)/x^2
                s3 += -sg * xm1 * inv_fact;                      // (x - E)/x
                if (j >= 3) {
                    s4 += sg * (2.0 - (double)j) * xm2 * inv_fact;   // (2E - x(1+e))/x^2
                    s5 += sg * xm2 * inv_fact;                        // (x^2/2 - x + E)/x^2
                }
                xp *= x;
            }
            xm1 *= x;
        }
        q[0] = dt * s1;
        q[1] = -dt * dt * s2;
        q[2] = dt * s3;
        q[3] = dt * dt * s4;
        q[4] = dt * dt * s5;
    } else {
        const double e = exp(-x);
        const double E = -expm1(-x);
        const double ix = 1.0 / x, ix2 = ix * ix;
        q[0] = dt * E * ix;
        q[1] = dt * dt * (x * e - E) * ix2;
        q[2] = dt * (x - E) * ix;
        q[3] = dt * dt * (2.0 * E - x * (1.0 + e)) * ix2;
        q[4] = dt * dt * (0.5 * x * x - x + E) * ix2;
    }
}

// Venkatakrishnan factor on FP64 data (macro reconstruction)
__device__ __forceinline__ double venkat_d(double d1, double d2, double e2)
{
    double a2 = d1 * d1 + e2;
    double num = a2 + 2.0 * d1 * d2;
    double den = a2 + d2 * (2.0 * d2 + d1);
    return den > 0.0 ? num / den : 1.0;
}

// ------------------------------------------------------------ batched launches
// The per-case kernels of a step (all but the gather) are written as bodies of
// a block index.  k_X runs them for one case (block index = blockIdx.x);
// k_X_batch runs them for many cases of a batch in one launch.  Its block b
// belongs to the last case i with off[i] <= b (off[] holds the prefix sums of
// the cases' block counts, so a case without blocks is never chosen) and runs
// that case's local block b - off[i]: the same arithmetic as the single-case
// launch.  The case's DevCase is copied into shared memory, where its fields
// are read without aliasing the arrays the kernel writes.
template <typename T>
__device__ __forceinline__ const DevCase<T> &batch_case(const DevCase<T> *__restrict__ cases,
                                                       const int *__restrict__ off, int n, int &bx)
{
    __shared__ __align__(16) unsigned char raw[sizeof(DevCase<T>)];
    static_assert(sizeof(DevCase<T>) % sizeof(int) == 0, "DevCase is copied in 4-byte words");
    const int b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    bx = b - __ldg(off + lo);
    const int *src = reinterpret_cast<const int *>(cases + lo);
    int *dst = reinterpret_cast<int *>(raw);
    for (int w = threadIdx.x; w < (int)(sizeof(DevCase<T>) / sizeof(int)); w += blockDim.x) dst[w] = __ldg(src + w);
    __syncthreads();
    return *reinterpret_cast<const DevCase<T> *>(raw);
}

// ------------------------------------------------------------ init / moments
template <typename T, int D, int NC>
__global__ void k_init_f(DevCase<T> dc)
{
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= dc.C) return;
    Prim p = prim_of(dc.W + (size_t)c * (D + 2), D);
    T rec[GREC];
    for (int d = 0; d < 3; ++d) rec[GR_U + d] = (T)p.U[d];
    rec[GR_LAM] = (T)p.lam;
    rec[GR_PREF] = (T)pref_of(p.rho, p.lam, D);
    rec[GR_NB] = (T)(dc.nxi / (2.0 * p.lam));
    rec[GR_NL2] = (T)(-p.lam * LOG2E);
    const size_t rs = (size_t)NC * dc.nvp;
    for (int k = lane; k < dc.nvp; k += 32) {
        T u[3] = {dc.u[0][k], dc.u[1][k], D == 3 ? dc.u[2][k] : T(0)};
        T H = maxwell_h<T, D>(rec, u);
        dc.f_cur[(size_t)c * rs + k] = H;
        if (NC == 2) dc.f_cur[(size_t)c * rs + dc.nvp + k] = rec[GR_NB] * H;
    }
}

// heat flux q = 1/2 sum_k w c (|c|^2 h + b), c = u - U(W)  (Sec. 2.1)
template <typename T, int D, int NC>
__global__ void k_heatflux(DevCase<T> dc)
{
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= dc.C) return;
    Prim p = prim_of(dc.W + (size_t)c * (D + 2), D);
    T U[3] = {(T)p.U[0], (T)p.U[1], (T)p.U[2]};
    const size_t rs = (size_t)NC * dc.nvp;
    CSum<T> acc[D];
    for (int k = lane; k < dc.nvp; k += 32) {
        T cc[D], c2 = 0;
        for (int d = 0; d < D; ++d) {
            cc[d] = dc.u[d][k] - U[d];
            c2 += cc[d] * cc[d];
        }
        T h = dc.f_cur[(size_t)c * rs + k];
        T e = c2 * h + (NC == 2 ? dc.f_cur[(size_t)c * rs + dc.nvp + k] : T(0));
        T we = dc.w[k] * e;
        for (int d = 0; d < D; ++d) acc[d].add(cc[d] * we);
    }
    for (int d = 0; d < D; ++d) {
        const double s = warp_sum(acc[d].value());
        if (lane == 0) dc.q[(size_t)c * D + d] = 0.5 * s;
    }
}

// ------------------------------------------------------------ k_prep
template <typename T, int D, int NC>
__device__ __forceinline__ void prep_body(const DevCase<T> &dc, const int bx)
{
    const int t = bx * blockDim.x + threadIdx.x;
    constexpr int M = D + 2;
    if (t < dc.C) {
        const int c = t;
        Prim p = prim_of(dc.W + (size_t)c * M, D);
        if (!(p.rho > 0.0) || !(p.T > 0.0)) atomicOr(dc.flags, 1);
        double *Pc = dc.prim + (size_t)c * M;
        Pc[0] = p.rho;
        for (int d = 0; d < D; ++d) Pc[1 + d] = p.U[d];
        Pc[D + 1] = p.T;
        double tau = tau_of(dc, p.rho, p.T);
        double kappa = 4.0 * (1.0 - dc.Pr) * p.lam * p.lam / (5.0 * p.rho);
        T *r = dc.crec + (size_t)c * CREC;
        for (int d = 0; d < 3; ++d) r[CR_U + d] = (T)p.U[d];
        r[CR_LAM] = (T)p.lam;
        r[CR_PREF] = (T)pref_of(p.rho, p.lam, D);
        for (int d = 0; d < 3; ++d) r[CR_KQ + d] = d < D ? (T)(kappa * dc.q[(size_t)c * D + d]) : T(0);
        const double cc = 0.5 * dc.dt / tau;
        r[CR_C] = (T)cc;
        r[CR_INV] = (T)(1.0 / (1.0 + cc));
        r[CR_NB] = (T)(dc.nxi / (2.0 * p.lam));
        r[CR_NL2] = (T)(-p.lam * LOG2E);
        return;
    }
    const int g = t - dc.C;
    if (g >= dc.G) return;
    // far-field ghost (Sec. 2.5): free stream where it enters (U_inf . n < 0),
    // zero-gradient extrapolation of the cell state elsewhere
    const int f = dc.gface[g];
    const int own = dc.fL[f];
    double un = __dmul_rn(dc.inf_W[1] / dc.inf_W[0], dc.fn_d[(size_t)f * D]);
    un = __dadd_rn(un, __dmul_rn(dc.inf_W[2] / dc.inf_W[0], dc.fn_d[(size_t)f * D + 1]));
    if (D == 3) un = __dadd_rn(un, __dmul_rn(dc.inf_W[3] / dc.inf_W[0], dc.fn_d[(size_t)f * D + 2]));
    double *Wg = dc.Wg + (size_t)g * M;
    for (int m = 0; m < M; ++m) Wg[m] = un < 0.0 ? dc.inf_W[m] : dc.W[(size_t)own * M + m];
    Prim p = prim_of(Wg, D);
    double *Pg = dc.primg + (size_t)g * M;
    Pg[0] = p.rho;
    for (int d = 0; d < D; ++d) Pg[1 + d] = p.U[d];
    Pg[D + 1] = p.T;
    T *r = dc.grec + (size_t)g * GREC;
    for (int d = 0; d < 3; ++d) r[GR_U + d] = (T)p.U[d];
    r[GR_LAM] = (T)p.lam;
    r[GR_PREF] = (T)pref_of(p.rho, p.lam, D);
    r[GR_NB] = (T)(dc.nxi / (2.0 * p.lam));
    r[GR_NL2] = (T)(-p.lam * LOG2E);
}

template <typename T, int D, int NC>
__global__ void k_prep(DevCase<T> dc)
{
    prep_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void k_prep_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    prep_body<T, D, NC>(dc, bx);
}

// ------------------------------------------------------------ k_macro_grad
// limited least-squares gradients of the primitive variables (rho, U, T) and
// the conserved-variable gradient obtained from them by the chain rule
template <typename T, int D, int NC>
__device__ __forceinline__ void macro_grad_body(const DevCase<T> &dc, const int bx)
{
    const int c = bx * blockDim.x + threadIdx.x;
    constexpr int M = D + 2;
    if (c >= dc.C) return;
    const double *Pc = dc.prim + (size_t)c * M;
    const int q0 = dc.nb_ptr[c], q1 = dc.nb_ptr[c + 1];
    const int s0 = dc.cf_ptr[c], s1 = dc.cf_ptr[c + 1];
    const double e2 = dc.eps2_d[c];
    double gp[D][M];
    for (int m = 0; m < M; ++m) {
        const double vi = Pc[m];
        double g[D], vmax = vi, vmin = vi;
        for (int d = 0; d < D; ++d) g[d] = 0.0;
        for (int q = q0; q < q1; ++q) {
            const int id = dc.nb_id[q];
            const double vj = id >= 0 ? dc.prim[(size_t)id * M + m] : dc.primg[(size_t)(-id - 1) * M + m];
            for (int d = 0; d < D; ++d) g[d] += dc.nb_a_d[(size_t)q * D + d] * (vj - vi);
            vmax = fmax(vmax, vj);
            vmin = fmin(vmin, vj);
        }
        if (dc.limiter) {
            double phi = 1.0;
            for (int s = s0; s < s1; ++s) {
                double d2 = 0.0;
                for (int d = 0; d < D; ++d) d2 += g[d] * dc.cf_r_d[(size_t)s * D + d];
                double d1 = d2 > 0.0 ? vmax - vi : vmin - vi;
                phi = fmin(phi, venkat_d(d1, d2, e2));
            }
            for (int d = 0; d < D; ++d) g[d] *= phi;
        }
        for (int d = 0; d < D; ++d) {
            gp[d][m] = g[d];
            dc.gradprim[((size_t)c * D + d) * M + m] = g[d];
        }
    }
    double uu = 0.0;
    for (int e = 0; e < D; ++e) uu += Pc[1 + e] * Pc[1 + e];
    for (int d = 0; d < D; ++d) {
        double *gw = dc.gradW + ((size_t)c * D + d) * M;
        double udu = 0.0;
        gw[0] = gp[d][0];
        for (int e = 0; e < D; ++e) {
            gw[1 + e] = Pc[1 + e] * gp[d][0] + Pc[0] * gp[d][1 + e];
            udu += Pc[1 + e] * gp[d][1 + e];
        }
        gw[D + 1] = gp[d][0] * (0.5 * uu + 1.5 * Pc[D + 1]) + Pc[0] * (udu + 1.5 * gp[d][D + 1]);
    }
}

template <typename T, int D, int NC>
__global__ void k_macro_grad(DevCase<T> dc)
{
    macro_grad_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void k_macro_grad_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    macro_grad_body<T, D, NC>(dc, bx);
}

// ------------------------------------------------------------ face pass
// face state reconstructed in primitive variables, P_c + gradP_c . r, returned
// as conserved variables; the cell average is used if rho or T would not be
// positive
template <int D>
__device__ __forceinline__ void face_state(const double *P, const double *gradP, int c, const double *r,
                                           double *Ws)
{
    constexpr int M = D + 2;
    double pf[M];
    for (int m = 0; m < M; ++m) {
        double s = P[(size_t)c * M + m];
        for (int d = 0; d < D; ++d) s += gradP[((size_t)c * D + d) * M + m] * r[d];
        pf[m] = s;
    }
    if (!(pf[0] > 0.0) || !(pf[D + 1] > 0.0))
        for (int m = 0; m < M; ++m) pf[m] = P[(size_t)c * M + m];
    double ke = 0.0;
    Ws[0] = pf[0];
    for (int d = 0; d < D; ++d) {
        Ws[1 + d] = pf[0] * pf[1 + d];
        ke += pf[1 + d] * pf[1 + d];
    }
    Ws[D + 1] = pf[0] * (0.5 * ke + 1.5 * pf[D + 1]);
}

template <typename T, int D>
__device__ __forceinline__ void side_record(const double *Ws, double nxi, T *rec)
{
    Prim p = prim_of(Ws, D);
    for (int d = 0; d < 3; ++d) rec[GR_U + d] = (T)p.U[d];
    rec[GR_LAM] = (T)p.lam;
    rec[GR_PREF] = (T)pref_of(p.rho, p.lam, D);
    rec[GR_NB] = (T)(nxi / (2.0 * p.lam));
    rec[GR_NL2] = (T)(-p.lam * LOG2E);
}

// Analytic half-range moments of the Maxwellian p over u.n > 0 (sigma = +1)
// or u.n < 0 (sigma = -1), added into the conserved components W.  Along the
// unit normal, with U_n = U.n and e = sigma exp(-lam U_n^2) / (2 sqrt(pi lam)):
// <1> = erfc(-sigma sqrt(lam) U_n) / 2, <u_n> = U_n <1> + e and
// <u_n^2> = (U_n^2 + 1/(2 lam)) <1> + U_n e; the D-1 tangential components
// (mean U - U_n n) and the 3-D internal ones are full Gaussians of variance
// 1/(2 lam) each, two components in all.
template <int D>
__device__ void add_half_range(const Prim &p, const double n[D], double sigma, double *W)
{
    double Un = 0.0;
    for (int d = 0; d < D; ++d) Un += p.U[d] * n[d];
    const double m0 = 0.5 * erfc(-sigma * sqrt(p.lam) * Un);
    const double e = sigma * exp(-p.lam * Un * Un) / (2.0 * sqrt(3.14159265358979323846 * p.lam));
    const double m1 = Un * m0 + e;
    const double m2 = (Un * Un + 0.5 / p.lam) * m0 + Un * e;
    double Ut2 = 0.0;
    W[0] += p.rho * m0;
    for (int d = 0; d < D; ++d) {
        const double Ut = p.U[d] - Un * n[d];
        Ut2 += Ut * Ut;
        W[1 + d] += p.rho * (m1 * n[d] + Ut * m0);
    }
    W[D + 1] += 0.5 * p.rho * (m2 + (Ut2 + 1.0 / p.lam) * m0);
}

template <typename T, int D, int NC>
__device__ __forceinline__ void face_pre_body(const DevCase<T> &dc, const int bx)
{
    const int f = bx * blockDim.x + threadIdx.x;
    constexpr int M = D + 2;
    if (f >= dc.F) return;
    const int typ = dc.ftype[f];
    if (typ == FT_WALL) return;
    const int L = dc.fL[f];
    double WL[M], WR[M], rL[D], rR[D];
    for (int d = 0; d < D; ++d) rL[d] = dc.frL_d[(size_t)f * D + d];
    face_state<D>(dc.prim, dc.gradprim, L, rL, WL);
    double *dW0 = dc.fdW0 + (size_t)f * D * M;
    double *q0 = dc.fq0 + (size_t)f * D;
    if (typ == FT_FARFIELD) {
        const int g = dc.faux[f];
        for (int m = 0; m < M; ++m) WR[m] = dc.Wg[(size_t)g * M + m];
        for (int d = 0; d < D; ++d) {
            for (int m = 0; m < M; ++m) dW0[d * M + m] = 0.5 * dc.gradW[((size_t)L * D + d) * M + m];
            q0[d] = 0.5 * dc.q[(size_t)L * D + d];
        }
    } else {
        const int R = dc.fR[f];
        for (int d = 0; d < D; ++d) rR[d] = dc.frR_d[(size_t)f * D + d];
        face_state<D>(dc.prim, dc.gradprim, R, rR, WR);
        for (int d = 0; d < D; ++d) {
            for (int m = 0; m < M; ++m)
                dW0[d * M + m] = 0.5 * (dc.gradW[((size_t)L * D + d) * M + m] + dc.gradW[((size_t)R * D + d) * M + m]);
            q0[d] = 0.5 * (dc.q[(size_t)L * D + d] + dc.q[(size_t)R * D + d]);
        }
    }
    side_record<T, D>(WL, dc.nxi, dc.fside + (size_t)f * 2 * GREC);
    side_record<T, D>(WR, dc.nxi, dc.fside + (size_t)f * 2 * GREC + GREC);
    Prim pL = prim_of(WL, D), pR = prim_of(WR, D);
    for (int d = 0; d < D; ++d) dc.fUref[(size_t)f * D + d] = 0.5 * (pL.U[d] + pR.U[d]);
    if (dc.w0_analytic) {
        // W0 from the analytic half-range moments (continuous velocity space),
        // stored centred at U_ref as the discrete sums of k_face_sum1 are
        double n[D], W0[M];
        for (int d = 0; d < D; ++d) n[d] = dc.fn_d[(size_t)f * D + d];
        for (int m = 0; m < M; ++m) W0[m] = 0.0;
        add_half_range<D>(pL, n, 1.0, W0);
        add_half_range<D>(pR, n, -1.0, W0);
        double *S = dc.fsum1 + (size_t)f * M;
        double uS = 0.0, uu = 0.0;
        S[0] = W0[0];
        for (int d = 0; d < D; ++d) {
            const double Ur = dc.fUref[(size_t)f * D + d];
            S[1 + d] = W0[1 + d] - Ur * W0[0];
            uS += Ur * W0[1 + d];
            uu += Ur * Ur;
        }
        S[D + 1] = W0[D + 1] - uS + 0.5 * uu * W0[0];
    }
}

template <typename T, int D, int NC>
__global__ void k_face_pre(DevCase<T> dc)
{
    face_pre_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void k_face_pre_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    face_pre_body<T, D, NC>(dc, bx);
}

// half-range moments: sum_k w psi_c [H(u_n) g_L + (1 - H(u_n)) g_R], centred at U_ref
template <typename T, int D, int NC>
__device__ __forceinline__ void face_sum1_body(const DevCase<T> &dc, const int bx)
{
    const int f = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    constexpr int M = D + 2;
    if (f >= dc.F || dc.ftype[f] == FT_WALL) return;
    // both side records in registers; a velocity selects its upwind side's
    // values instead of loading them through a selected pointer
    T sL[GREC], sR[GREC];
#pragma unroll
    for (int i = 0; i < GREC; ++i) {
        sL[i] = __ldg(dc.fside + (size_t)f * 2 * GREC + i);
        sR[i] = __ldg(dc.fside + (size_t)f * 2 * GREC + GREC + i);
    }
    T n[D], Ur[D];
    for (int d = 0; d < D; ++d) {
        n[d] = dc.fn[(size_t)f * D + d];
        Ur[d] = (T)dc.fUref[(size_t)f * D + d];
    }
    // the terms of velocity k, added into a[0..M)
    auto terms = [&](int k, T *a) {
        T u[3], wk;
        load_uw(dc.uw, k, u, wk);
        T un = normal_velocity<T, D>(u, n);
        T h, b;
        if (un != T(0)) {
            T s[GREC];
#pragma unroll
            for (int i = 0; i < GREC; ++i) s[i] = un > T(0) ? sL[i] : sR[i];
            h = maxwell_h<T, D>(s, u);
            b = s[GR_NB] * h;
        } else {
            T hl = maxwell_h<T, D>(sL, u), hr = maxwell_h<T, D>(sR, u);
            h = T(0.5) * hl + T(0.5) * hr;
            b = T(0.5) * sL[GR_NB] * hl + T(0.5) * sR[GR_NB] * hr;
        }
        T c2 = 0;
        T wh = wk * h;
        a[0] += wh;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            T c = u[d] - Ur[d];
            c2 += c * c;
            a[1 + d] += c * wh;
        }
        a[D + 1] += T(0.5) * wk * (c2 * h + b);
    };
    if constexpr (std::is_same<T, float>::value) {
        // blocked sums accumulated in FP64 (SUM_BLOCK terms per lane per block)
        constexpr int NP = M <= 4 ? 4 : 8;
        double acc = 0.0;
        for (int k0 = lane; k0 < dc.nvp; k0 += 32 * SUM_BLOCK) {
            float blk[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) blk[i] = 0.f;
#pragma unroll 4
            for (int j = 0; j < SUM_BLOCK; ++j) {
                const int k = k0 + 32 * j;
                if (k >= dc.nvp) break;              // uniform: nvp is a multiple of 32
                terms(k, blk);
            }
            acc += block_to_fp64<NP>(blk);
        }
        const int vi = lane >> (NP == 4 ? 3 : 2);
        if ((lane & (NP == 4 ? 7 : 3)) == 0 && vi < M) dc.fsum1[(size_t)f * M + vi] = acc;
    } else {
        T acc[M];
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] = 0;
        for (int k = lane; k < dc.nvp; k += 32) terms(k, acc);
        for (int m = 0; m < M; ++m) {
            const double sm = warp_sum(acc[m]);
            if (lane == 0) dc.fsum1[(size_t)f * M + m] = sm;
        }
    }
}

template <typename T, int D, int NC>
__global__ void k_face_sum1(DevCase<T> dc)
{
    face_sum1_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void k_face_sum1_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    face_sum1_body<T, D, NC>(dc, bx);
}

// k_face_sum1 on a tensor-product velocity grid.  With the face-state
// Maxwellians factored by axis, the half-range sums become, for every point of
// the outer axes, sums over a contiguous range of the last axis: u.n, rounded
// as everywhere (no contraction, last term added last), is monotone along that
// axis when its nodes ascend.  Prefix sums of the last axis' 1-D moments give
// every range in O(1); the range ends come from binary searches on the exact
// u.n, and nodes with u.n = 0 keep their half weight on both sides.  One warp
// per face; the prefix sums live in shared memory, 2 sides x 3 powers x
// (NL + 1) doubles per warp.
constexpr int SUM1_SEP_WARPS = 4;

template <typename T, int D, int NC>
__device__ __forceinline__ void face_sum1_sep_body(const DevCase<T> &dc, const int bx)
{
    extern __shared__ __align__(16) unsigned char psum_raw[];
    T *psum = reinterpret_cast<T *>(psum_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = bx * SUM1_SEP_WARPS + warp;
    constexpr int M = D + 2;
    constexpr int L = D - 1;                 // the prefix-sum axis
    const int NL = dc.cart_n[L];
    if (f >= dc.F || dc.ftype[f] == FT_WALL) return;
    T *P = psum + (size_t)warp * 6 * (NL + 1);
    const T *side[2] = {dc.fside + (size_t)f * 2 * GREC, dc.fside + (size_t)f * 2 * GREC + GREC};
    T n[D], Ur[D];
    for (int d = 0; d < D; ++d) {
        n[d] = dc.fn[(size_t)f * D + d];
        Ur[d] = (T)dc.fUref[(size_t)f * D + d];
    }
    // prefix sums over the last axis of w g (u - Ur)^p, p = 0, 1, 2, per side
    // (at most SUM1_SEP_MAX_NL = 512 terms each: one block of the FP32 form's
    // blocked sums)
    for (int s = 0; s < 2; ++s) {
        const T *r = side[s];
        T *Ps = P + s * 3 * (NL + 1);
        if (lane == 0) Ps[0] = Ps[NL + 1] = Ps[2 * (NL + 1)] = T(0);
        T carry[3] = {0, 0, 0};
        for (int j0 = 0; j0 < NL; j0 += 32) {
            const int j = j0 + lane;
            T v[3] = {0, 0, 0};
            if (j < NL) {
                const T a = dc.axis[L][j];
                const T dv = a - r[GR_U + L];
                const T g = dc.axw[L][j] * gauss<T>(r[GR_LAM], r[GR_NL2], dv * dv);
                const T c = a - Ur[L];
                v[0] = g;
                v[1] = g * c;
                v[2] = g * c * c;
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) {
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const T t = __shfl_up_sync(0xffffffffu, v[p], o);
                    if (lane >= o) v[p] += t;
                }
                if (j < NL) Ps[p * (NL + 1) + j + 1] = carry[p] + v[p];
                carry[p] += __shfl_sync(0xffffffffu, v[p], 31);
            }
        }
    }
    __syncwarp();
    const T nl = n[L];
    const T *aL = dc.axis[L];
    int nouter = dc.cart_n[0];
    if (D == 3) nouter *= dc.cart_n[1];
    // the terms of outer node o (both sides), added into acc[0..M)
    auto terms = [&](int o, T *acc) {
        int idx[2] = {o % dc.cart_n[0], D == 3 ? o / dc.cart_n[0] : 0};
        T uo[2];
        uo[0] = dc.axis[0][idx[0]];
        uo[1] = D == 3 ? dc.axis[1][idx[1]] : T(0);
        T sp = mul_rn(uo[0], n[0]);
        if (D == 3) sp = add_rn(sp, mul_rn(uo[1], n[1]));
        // [ja, jb): u.n = 0; ascending u.n (nl >= 0): u.n < 0 on [0, ja), > 0 on [jb, NL);
        // descending (nl < 0): u.n > 0 on [0, ja), < 0 on [jb, NL)
        auto first = [&](int mode) {
            int lo = 0, hi = NL;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const T v = add_rn(sp, mul_rn(aL[mid], nl));
                const bool t = mode == 0 ? v >= T(0) : mode == 1 ? v > T(0) : mode == 2 ? v <= T(0) : v < T(0);
                if (t) hi = mid;
                else lo = mid + 1;
            }
            return lo;
        };
        const bool asc = nl >= T(0);
        const int ja = first(asc ? 0 : 2), jb = first(asc ? 1 : 3);
        T co2 = 0, co[2];
#pragma unroll
        for (int e = 0; e < D - 1; ++e) {
            co[e] = uo[e] - Ur[e];
            co2 += co[e] * co[e];
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const T *r = side[s];
            const T *Ps = P + s * 3 * (NL + 1);
            const bool lo_side = (s == 0) != asc;        // the full range starts at 0
            const int f0 = lo_side ? 0 : jb, f1 = lo_side ? ja : NL;
            T Y[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const T *Pp = Ps + p * (NL + 1);
                Y[p] = (Pp[f1] - Pp[f0]) + T(0.5) * (Pp[jb] - Pp[ja]);
            }
            T go = r[GR_PREF];
#pragma unroll
            for (int e = 0; e < D - 1; ++e) {
                const T dv = uo[e] - r[GR_U + e];
                go *= dc.axw[e][idx[e]] * gauss<T>(r[GR_LAM], r[GR_NL2], dv * dv);
            }
            const T g = go;
            acc[0] += g * Y[0];
#pragma unroll
            for (int e = 0; e < D - 1; ++e) acc[1 + e] += g * co[e] * Y[0];
            acc[1 + L] += g * Y[1];
            acc[D + 1] += T(0.5) * g * (co2 * Y[0] + Y[2] + r[GR_NB] * Y[0]);
        }
    };
    if constexpr (std::is_same<T, float>::value) {
        // blocked sums accumulated in FP64 (SUM_BLOCK outer nodes per lane per block)
        constexpr int NP = M <= 4 ? 4 : 8;
        double acc = 0.0;
        for (int o0 = 0; o0 < nouter; o0 += 32 * SUM_BLOCK) {
            float blk[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) blk[i] = 0.f;
            for (int j = 0; j < SUM_BLOCK; ++j) {
                const int o = o0 + 32 * j + lane;
                if (o >= nouter) break;
                terms(o, blk);
            }
            acc += block_to_fp64<NP>(blk);
        }
        const int vi = lane >> (NP == 4 ? 3 : 2);
        if ((lane & (NP == 4 ? 7 : 3)) == 0 && vi < M) dc.fsum1[(size_t)f * M + vi] = acc;
    } else {
        T acc[M];
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] = 0;
        for (int o = lane; o < nouter; o += 32) terms(o, acc);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const double sm = warp_sum(acc[m]);
            if (lane == 0) dc.fsum1[(size_t)f * M + m] = sm;
        }
    }
}

template <typename T, int D, int NC>
__global__ void __launch_bounds__(32 * SUM1_SEP_WARPS) k_face_sum1_sep(DevCase<T> dc)
{
    face_sum1_sep_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void __launch_bounds__(32 * SUM1_SEP_WARPS) k_face_sum1_sep_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    face_sum1_sep_body<T, D, NC>(dc, bx);
}

template <typename T, int D, int NC>
__device__ __forceinline__ void face_fin1_body(const DevCase<T> &dc, const int bx)
{
    const int f = bx * blockDim.x + threadIdx.x;
    constexpr int M = D + 2;
    if (f >= dc.F || dc.ftype[f] == FT_WALL) return;
    const double *S = dc.fsum1 + (size_t)f * M;
    const double *Ur = dc.fUref + (size_t)f * D;
    // shift the centred sums back: psi = L psi_c with c = u - U_ref
    double W0[M];
    W0[0] = S[0];
    double uS = 0.0, uu = 0.0;
    for (int d = 0; d < D; ++d) {
        W0[1 + d] = S[1 + d] + Ur[d] * S[0];
        uS += Ur[d] * S[1 + d];
        uu += Ur[d] * Ur[d];
    }
    W0[D + 1] = S[D + 1] + uS + 0.5 * uu * S[0];
    Prim p = prim_of(W0, D);
    double *pp = dc.fprim0 + (size_t)f * M;
    pp[0] = p.rho;
    for (int d = 0; d < D; ++d) pp[1 + d] = p.U[d];
    pp[D + 1] = p.lam;
    T *r = dc.frec + (size_t)f * FREC;
    for (int d = 0; d < 3; ++d) r[FR_U + d] = (T)p.U[d];
    r[FR_LAM] = (T)p.lam;
    r[FR_PREF] = (T)pref_of(p.rho, p.lam, D);
    const double kappa = 4.0 * (1.0 - dc.Pr) * p.lam * p.lam / (5.0 * p.rho);
    for (int d = 0; d < 3; ++d) r[FR_KQ + d] = d < D ? (T)(kappa * dc.fq0[(size_t)f * D + d]) : T(0);
    double *qs = dc.fqs + (size_t)f * 5;         // kept in FP64 for k_face_fin2
    time_integrals(dc.dt, tau_of(dc, p.rho, p.T), qs);
    for (int i = 0; i < 5; ++i) r[FR_QS + i] = (T)qs[i];
    r[FR_NB] = (T)(dc.nxi / (2.0 * p.lam));
    r[FR_XB] = (T)(dc.nxi * (dc.nxi + 2.0) / (4.0 * p.lam * p.lam));
    r[FR_NL2] = (T)(-p.lam * LOG2E);
}

template <typename T, int D, int NC>
__global__ void k_face_fin1(DevCase<T> dc)
{
    face_fin1_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void k_face_fin1_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    face_fin1_body<T, D, NC>(dc, bx);
}

// number of unique entries of a symmetric (D+2)x(D+2) matrix
template <int D> struct Sym { static constexpr int N = (D + 2) * (D + 3) / 2; };

// The sums the slope systems need on an unstructured velocity set are the
// entries of sum_k w_k H0 psi_c psi_c^T and of the same with a factor c_d, with
// psi_c = (1, c, psi_E) and, after integrating the internal degrees of freedom,
// psi_E = (|c|^2 + nb) / 2 and psi_E^2 = (|c|^4 + 2 nb |c|^2 + xb) / 4.  Every
// one of them is a combination of fewer distinct moments R of w H0:
//   c^a for |a| <= 3 (1, c_d, pairs d <= e, triples d <= e <= g),
//   |c|^2 c_d c_e (d <= e), |c|^4 and |c|^4 c_d,
// 30 in 3D against 60 entries (16 against 30 in 2D).  k_face_sum2 reduces R;
// k_face_fin2 forms the entries in FP64 (mono_moments).
template <int D> struct Mono {
    static constexpr int N2 = D * (D + 1) / 2;                // pairs d <= e
    static constexpr int N3 = D * (D + 1) * (D + 2) / 6;      // triples d <= e <= g
    static constexpr int O1 = 1, O2 = O1 + D, O3 = O2 + N2, OQ2 = O3 + N3, OQ4 = OQ2 + N2, N = OQ4 + 1 + D;
};

// position of the pair d <= e (row-major upper triangle) and of the triple
// d <= e <= g (lexicographic), the order in which k_face_sum2 stores them
__host__ __device__ constexpr int pair_index(int D, int d, int e) { return d * D - d * (d - 1) / 2 + (e - d); }

__host__ __device__ constexpr int triple_index(int D, int d, int e, int g)
{
    // triples with a first index below d, then with (d, b < e), then (d, e, c < g)
    return (D * (D + 1) * (D + 2) - (D - d) * (D - d + 1) * (D - d + 2)) / 6 +
           ((D - d) * (D - d + 1) - (D - e) * (D - e + 1)) / 2 + (g - e);
}

// sum w H0 c_a c_b (c_g) from R, indices in any order
template <int D> __device__ __forceinline__ double mono2(const double *R, int a, int b)
{
    return R[Mono<D>::O2 + (a <= b ? pair_index(D, a, b) : pair_index(D, b, a))];
}

template <int D> __device__ __forceinline__ double mono3(const double *R, int a, int b, int g)
{
    int x = a, y = b, z = g, t;
    if (x > y) { t = x; x = y; y = t; }
    if (y > z) { t = y; y = z; z = t; }
    if (x > y) { t = x; x = y; y = t; }
    return R[Mono<D>::O3 + triple_index(D, x, y, z)];
}

// the k_face_sum2 entries (layout of sep_moments) from the distinct moments R
template <int D>
__device__ void mono_moments(const double *R, double nb, double xb, double *S)
{
    using Mo = Mono<D>;
    constexpr int NS = Sym<D>::N;
    constexpr int M = D + 2;
    double s2 = 0.0, s2c[D];                        // sum |c|^2 and sum |c|^2 c_d
#pragma unroll
    for (int e = 0; e < D; ++e) s2 += mono2<D>(R, e, e);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        s2c[d] = 0.0;
#pragma unroll
        for (int e = 0; e < D; ++e) s2c[d] += mono3<D>(R, d, e, e);
    }
    int t = 0;
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int j = i; j < M; ++j) {
            double base, bc[D];
            if (j < M - 1) {                        // psi_i psi_j: a monomial of degree <= 2
                if (i == 0 && j == 0) {
                    base = R[0];
#pragma unroll
                    for (int d = 0; d < D; ++d) bc[d] = R[Mo::O1 + d];
                } else if (i == 0) {
                    base = R[Mo::O1 + j - 1];
#pragma unroll
                    for (int d = 0; d < D; ++d) bc[d] = mono2<D>(R, j - 1, d);
                } else {
                    base = mono2<D>(R, i - 1, j - 1);
#pragma unroll
                    for (int d = 0; d < D; ++d) bc[d] = mono3<D>(R, i - 1, j - 1, d);
                }
            } else if (i < M - 1) {                 // psi_i psi_E
                if (i == 0) {
                    base = 0.5 * (s2 + nb * R[0]);
#pragma unroll
                    for (int d = 0; d < D; ++d) bc[d] = 0.5 * (s2c[d] + nb * R[Mo::O1 + d]);
                } else {
                    const int a = i - 1;
                    base = 0.5 * (s2c[a] + nb * R[Mo::O1 + a]);
#pragma unroll
                    for (int d = 0; d < D; ++d)
                        bc[d] = 0.5 * (R[Mo::OQ2 + (a <= d ? pair_index(D, a, d) : pair_index(D, d, a))] +
                                       nb * mono2<D>(R, a, d));
                }
            } else {                                // psi_E^2
                base = 0.25 * (R[Mo::OQ4] + 2.0 * nb * s2 + xb * R[0]);
#pragma unroll
                for (int d = 0; d < D; ++d) bc[d] = 0.25 * (R[Mo::OQ4 + 1 + d] + 2.0 * nb * s2c[d] + xb * R[Mo::O1 + d]);
            }
            S[t] = base;
#pragma unroll
            for (int d = 0; d < D; ++d) S[NS * (1 + d) + t] = bc[d];
            ++t;
        }
}

template <typename T, int D, int NC>
__device__ __forceinline__ void face_sum2_body(const DevCase<T> &dc, const int bx)
{
    const int f = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    constexpr int NS = Sym<D>::N;
    constexpr int S2 = NS * (D + 1);
    if (f >= dc.F || dc.ftype[f] == FT_WALL) return;
    const T *fr = dc.frec + (size_t)f * FREC;
    T U0[D];
#pragma unroll
    for (int d = 0; d < D; ++d) U0[d] = fr[FR_U + d];
    const T lam = fr[FR_LAM], pref = fr[FR_PREF], nl2 = fr[FR_NL2];
    using Mo = Mono<D>;
    // the distinct monomial moments of velocity k, added into r[0..Mo::N)
    auto terms = [&](int k, T *r) {
        T uk[3], wk, c[D], c2 = 0;
        load_uw(dc.uw, k, uk, wk);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            c[d] = uk[d] - U0[d];
            c2 += c[d] * c[d];
        }
        const T a = wk * pref * gauss<T>(lam, nl2, c2);
        r[0] += a;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const T a1 = a * c[d];
            r[Mo::O1 + d] += a1;
#pragma unroll
            for (int e = d; e < D; ++e) {
                const T a2 = a1 * c[e];
                r[Mo::O2 + pair_index(D, d, e)] += a2;
                r[Mo::OQ2 + pair_index(D, d, e)] += a2 * c2;
#pragma unroll
                for (int g = e; g < D; ++g) r[Mo::O3 + triple_index(D, d, e, g)] += a2 * c[g];
            }
        }
        const T a4 = a * c2 * c2;
        r[Mo::OQ4] += a4;
#pragma unroll
        for (int d = 0; d < D; ++d) r[Mo::OQ4 + 1 + d] += a4 * c[d];
    };
    if constexpr (std::is_same<T, float>::value) {
        // blocked sums accumulated in FP64 (SUM_BLOCK terms per lane per block)
        constexpr int NP = Mo::N <= 16 ? 16 : 32;
        double acc = 0.0;
        for (int k0 = lane; k0 < dc.nvp; k0 += 32 * SUM_BLOCK) {
            float blk[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) blk[i] = 0.f;
#pragma unroll 2
            for (int j = 0; j < SUM_BLOCK; ++j) {
                const int k = k0 + 32 * j;
                if (k >= dc.nvp) break;              // uniform: nvp is a multiple of 32
                terms(k, blk);
            }
            acc += block_to_fp64<NP>(blk);
        }
        const int vi = lane >> (NP == 16 ? 1 : 0);
        if ((lane & (NP == 16 ? 1 : 0)) == 0 && vi < Mo::N) dc.fsum2[(size_t)f * S2 + vi] = acc;
    } else {
        T r[Mo::N];
#pragma unroll
        for (int i = 0; i < Mo::N; ++i) r[i] = 0;
        for (int k = lane; k < dc.nvp; k += 32) terms(k, r);
#pragma unroll
        for (int i = 0; i < Mo::N; ++i) {
            const double sm = warp_sum(r[i]);
            if (lane == 0) dc.fsum2[(size_t)f * S2 + i] = sm;
        }
    }
}

template <typename T, int D, int NC>
__global__ void k_face_sum2(DevCase<T> dc)
{
    face_sum2_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void k_face_sum2_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    face_sum2_body<T, D, NC>(dc, bx);
}

// The same sums as k_face_sum2 on a tensor-product velocity grid, where
// u_k = (x_i, y_j[, z_l]) and w_k = wx_i wy_j [wz_l]: every moment of g0 the slope
// systems need is sum_k w_k H0(u_k) c^alpha = pref0 prod_d m_d[alpha_d] with the
// 1-D moments m_d[p] = sum_i w_{d,i} exp(-lam0 c_{d,i}^2) c_{d,i}^p, p <= 5.
// This kernel reduces the 1-D moments (warp per face); k_face_fin2 forms the
// products (thread per face, FP64).
template <typename T, int D, int NC>
__device__ __forceinline__ void face_sum2_sep_body(const DevCase<T> &dc, const int bx)
{
    const int f = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    constexpr int NS = Sym<D>::N;
    if (f >= dc.F || dc.ftype[f] == FT_WALL) return;
    const T *fr = dc.frec + (size_t)f * FREC;
    const T lam = fr[FR_LAM], nl2 = fr[FR_NL2];
    double *out = dc.fsum2 + (size_t)f * NS * (D + 1);
    for (int d = 0; d < D; ++d) {
        const T U0 = fr[FR_U + d];
        if constexpr (std::is_same<T, float>::value) {
            // blocked sums accumulated in FP64 (SUM_BLOCK nodes per lane per block)
            double acc = 0.0;
            for (int i0 = 0; i0 < dc.cart_n[d]; i0 += 32 * SUM_BLOCK) {
                float blk[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int j = 0; j < SUM_BLOCK; ++j) {
                    const int i = i0 + 32 * j + lane;
                    if (i >= dc.cart_n[d]) break;
                    const float c = dc.axis[d][i] - U0;
                    float v = dc.axw[d][i] * gauss<float>(lam, nl2, c * c);
#pragma unroll
                    for (int pw = 0; pw < 6; ++pw) {
                        blk[pw] += v;
                        v *= c;
                    }
                }
                acc += block_to_fp64<8>(blk);
            }
            if ((lane & 3) == 0 && (lane >> 2) < 6) out[d * 6 + (lane >> 2)] = acc;
        } else {
            T acc[6] = {0, 0, 0, 0, 0, 0};
            for (int i = lane; i < dc.cart_n[d]; i += 32) {
                const T c = dc.axis[d][i] - U0;
                T v = dc.axw[d][i] * gauss<T>(lam, nl2, c * c);
#pragma unroll
                for (int pw = 0; pw < 6; ++pw) {
                    acc[pw] += v;
                    v *= c;
                }
            }
#pragma unroll
            for (int pw = 0; pw < 6; ++pw) {
                const double sm = warp_sum(acc[pw]);
                if (lane == pw) out[d * 6 + pw] = sm;
            }
        }
    }
}

template <typename T, int D, int NC>
__global__ void k_face_sum2_sep(DevCase<T> dc)
{
    face_sum2_sep_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void k_face_sum2_sep_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    face_sum2_sep_body<T, D, NC>(dc, bx);
}

// M_c and T_c,d of k_face_sum2 from the 1-D moments m[d][0..5] (tensor grids)
template <int D>
__device__ void sep_moments(const double m[D][6], double pref, double nb, double xb, double *S)
{
    constexpr int NS = Sym<D>::N;
    constexpr int M = D + 2;
    auto Q = [&](const int *a) {
        double r = pref;
        for (int d = 0; d < D; ++d) r *= m[d][a[d]];
        return r;
    };
    for (int t = -1; t < D; ++t) {          // t = -1: M_c; t = d: T_c,d (extra factor c_d)
        int base[3] = {0, 0, 0};
        if (t >= 0) base[t] = 1;
        int idx = 0;
        for (int i = 0; i < M; ++i)
            for (int j = i; j < M; ++j) {
                double val;
                int a[3] = {base[0], base[1], base[2]};
                const bool iE = i == M - 1, jE = j == M - 1;
                if (!iE && !jE) {
                    if (i > 0) a[i - 1]++;
                    if (j > 0) a[j - 1]++;
                    val = Q(a);
                } else if (!iE || !jE) {
                    // psi_o (|c|^2 + xi^2)/2 with psi_o = 1 or c_(o-1)
                    const int o = iE ? j : i;
                    if (o > 0) a[o - 1]++;
                    double s2 = 0.0;
                    for (int e = 0; e < D; ++e) {
                        int b[3] = {a[0], a[1], a[2]};
                        b[e] += 2;
                        s2 += Q(b);
                    }
                    val = 0.5 * (s2 + nb * Q(a));
                } else {
                    double s4 = 0.0, s2 = 0.0;
                    for (int e = 0; e < D; ++e) {
                        int b[3] = {a[0], a[1], a[2]};
                        b[e] += 2;
                        s2 += Q(b);
                        for (int g = 0; g < D; ++g) {
                            int c4[3] = {b[0], b[1], b[2]};
                            c4[g] += 2;
                            s4 += Q(c4);
                        }
                    }
                    val = 0.25 * (s4 + 2.0 * nb * s2 + xb * Q(a));
                }
                S[NS * (t + 1) + idx] = val;
                ++idx;
            }
    }
}

// Cholesky solve of the SPD system A x = b (n <= 5), A overwritten
__device__ void chol_solve(int n, double *A, double *b, int nrhs, int ldb)
{
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        const double Ljj = sqrt(s);
        A[j * n + j] = Ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / Ljj;
        }
    }
    for (int r = 0; r < nrhs; ++r) {
        double *x = b + r * ldb;
        for (int i = 0; i < n; ++i) {
            double t = x[i];
            for (int k = 0; k < i; ++k) t -= A[i * n + k] * x[k];
            x[i] = t / A[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double t = x[i];
            for (int k = i + 1; k < n; ++k) t -= A[k * n + i] * x[k];
            x[i] = t / A[i * n + i];
        }
    }
}

// slopes of g0 in the centred basis: M0 = L Mc L^T, sum_k w u_d psi psi^T g0 =
// L (Tc_d + U0_d Mc) L^T with psi = L psi_c.  Then beta_d = L^T a_d solves
// Mc beta_d = L^{-1} dW0/dx_d, and the compatibility condition gives
// beta_A = L^T A = -Mc^{-1} sum_d Tc_d beta_d - sum_d U0_d beta_d.
template <typename T, int D, int NC>
__device__ __forceinline__ void face_fin2_body(const DevCase<T> &dc, const int bx)
{
    const int f = bx * blockDim.x + threadIdx.x;
    constexpr int M = D + 2, NS = Sym<D>::N, S2 = NS * (D + 1);
    if (f >= dc.F || dc.ftype[f] == FT_WALL) return;
    double Ssep[S2];
    const double *S = dc.fsum2 + (size_t)f * S2;
    if (dc.sep) {
        double m1[D][6];
        for (int d = 0; d < D; ++d)
            for (int pw = 0; pw < 6; ++pw) m1[d][pw] = S[d * 6 + pw];
        const double *pq = dc.fprim0 + (size_t)f * M;
        const double lam0 = pq[D + 1];
        sep_moments<D>(m1, pref_of(pq[0], lam0, D), dc.nxi / (2.0 * lam0),
                       dc.nxi * (dc.nxi + 2.0) / (4.0 * lam0 * lam0), Ssep);
        S = Ssep;
    } else {
        const double lam0 = dc.fprim0[(size_t)f * M + D + 1];
        mono_moments<D>(S, dc.nxi / (2.0 * lam0), dc.nxi * (dc.nxi + 2.0) / (4.0 * lam0 * lam0), Ssep);
        S = Ssep;
    }
    double Mc[M * M], Tc[D][M * M];
    {
        int t = 0;
        for (int i = 0; i < M; ++i)
            for (int j = i; j < M; ++j) {
                Mc[i * M + j] = Mc[j * M + i] = S[t];
                for (int d = 0; d < D; ++d) Tc[d][i * M + j] = Tc[d][j * M + i] = S[NS * (1 + d) + t];
                ++t;
            }
    }
    const double *pp = dc.fprim0 + (size_t)f * M;
    double U0[D], uu = 0.0;
    for (int d = 0; d < D; ++d) {
        U0[d] = pp[1 + d];
        uu += U0[d] * U0[d];
    }
    // right-hand sides L^{-1} dW0_d
    double B[(D + 1) * M];
    const double *dW = dc.fdW0 + (size_t)f * D * M;
    for (int d = 0; d < D; ++d) {
        const double *g = dW + d * M;
        double *x = B + d * M;
        x[0] = g[0];
        double um = 0.0;
        for (int e = 0; e < D; ++e) {
            x[1 + e] = g[1 + e] - U0[e] * g[0];
            um += U0[e] * g[1 + e];
        }
        x[D + 1] = g[D + 1] - um + 0.5 * uu * g[0];
    }
    double A[M * M];
    for (int i = 0; i < M * M; ++i) A[i] = Mc[i];
    chol_solve(M, A, B, D, M);              // B[d] = beta_d ; A holds the factor
    double *xa = B + D * M;
    for (int i = 0; i < M; ++i) {
        double s = 0.0;
        for (int d = 0; d < D; ++d)
            for (int j = 0; j < M; ++j) s += Tc[d][i * M + j] * B[d * M + j];
        xa[i] = -s;
    }
    // solve with the stored factor
    for (int i = 0; i < M; ++i) {
        double t = xa[i];
        for (int k = 0; k < i; ++k) t -= A[i * M + k] * xa[k];
        xa[i] = t / A[i * M + i];
    }
    for (int i = M - 1; i >= 0; --i) {
        double t = xa[i];
        for (int k = i + 1; k < M; ++k) t -= A[k * M + i] * xa[k];
        xa[i] = t / A[i * M + i];
    }
    for (int i = 0; i < M; ++i)
        for (int d = 0; d < D; ++d) xa[i] -= U0[d] * B[d * M + i];
    T *r = dc.frec + (size_t)f * FREC;
    for (int i = 0; i < (D + 1) * M; ++i) r[FR_BETA + i] = (T)B[i];

    // Expand the equilibrium part of the interface distribution,
    // q3 (g0 + g0+) + q4 u.grad g0 + q5 dg0/dt, into H0(c) P_m(c), c = u - U0:
    //   h: sh = 1 + (kq.c)(2 lam |c|^2 - D - 2), slope terms of int (beta.psi_c) g0 dxi
    //   b: sh = nb [1 + (kq.c)(2 lam |c|^2 - D)], slope terms of int xi^2 (beta.psi_c) g0 dxi
    // with u_d = c_d + U0_d.
    const double rho0 = pp[0], lam0 = pp[D + 1];
    const double nb = dc.nxi / (2.0 * lam0), xb = dc.nxi * (dc.nxi + 2.0) / (4.0 * lam0 * lam0);
    const double kappa = 4.0 * (1.0 - dc.Pr) * lam0 * lam0 / (5.0 * rho0);
    double kq[D];
    for (int d = 0; d < D; ++d) kq[d] = kappa * dc.fq0[(size_t)f * D + d];
    const double *qs = dc.fqs + (size_t)f * 5;   // time integrals of k_face_fin1
    T *x = dc.xrec + (size_t)f * XREC;
    for (int d = 0; d < 3; ++d) x[XR_U + d] = d < D ? (T)U0[d] : T(0);
    x[XR_PREF] = (T)pref_of(rho0, lam0, D);
    x[XR_NL2] = (T)(-lam0 * LOG2E);
    x[XR_LAM] = (T)lam0;
    x[XR_Q1] = (T)qs[0];
    x[XR_Q2] = (T)qs[1];
    constexpr int NB = Poly<D>::NB, NP = Poly<D>::N;
    for (int m = 0; m < NC; ++m) {
        const double sm = m == 0 ? 1.0 : nb;            // scale of the b moments
        const double xm = m == 0 ? nb : xb;             // xi^2 (resp. xi^4) factor of beta_E / 2
        const double sh0 = m == 0 ? 1.0 : nb;
        const double shl = m == 0 ? -(double)(D + 2) : -(double)D;
        double a0 = qs[2] * sh0, a[D], Bq[D][D], gam[D];
        for (int e = 0; e < D; ++e) {
            a[e] = qs[2] * sh0 * shl * kq[e];
            gam[e] = qs[2] * sh0 * 2.0 * lam0 * kq[e];
            for (int g = 0; g < D; ++g) Bq[e][g] = 0.0;
        }
        double diag = 0.0;
        for (int d = 0; d < D; ++d) {
            const double *bd = B + d * M;                // beta^(d) in the psi_c basis
            const double alpha = sm * bd[0] + 0.5 * bd[D + 1] * xm;
            a0 += qs[3] * U0[d] * alpha;
            a[d] += qs[3] * alpha;
            for (int e = 0; e < D; ++e) {
                a[e] += qs[3] * U0[d] * sm * bd[1 + e];
                Bq[d][e] += qs[3] * sm * bd[1 + e];
            }
            diag += qs[3] * U0[d] * 0.5 * sm * bd[D + 1];
            gam[d] += qs[3] * 0.5 * sm * bd[D + 1];
        }
        const double alphaA = sm * xa[0] + 0.5 * xa[D + 1] * xm;
        a0 += qs[4] * alphaA;
        for (int e = 0; e < D; ++e) a[e] += qs[4] * sm * xa[1 + e];
        diag += qs[4] * 0.5 * sm * xa[D + 1];
        T *pm = x + XR_POLY + m * NP;
        pm[0] = (T)a0;
        for (int e = 0; e < D; ++e) pm[1 + e] = (T)a[e];
        int t = 1 + D;
        for (int e = 0; e < D; ++e)
            for (int g = e; g < D; ++g)
                pm[t++] = (T)(e == g ? Bq[e][e] + diag : Bq[e][g] + Bq[g][e]);
        for (int e = 0; e < D; ++e) pm[1 + D + NB + e] = (T)gam[e];
    }
}

template <typename T, int D, int NC>
__global__ void k_face_fin2(DevCase<T> dc)
{
    face_fin2_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void k_face_fin2_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    face_fin2_body<T, D, NC>(dc, bx);
}

// ------------------------------------------------------------ walls
// rho_w from zero net mass flux (Eq. maxWalldes): outgoing particles (u_n > 0)
// carry the interior reconstruction transported freely over the step,
// incoming ones the wall Maxwellian.
template <typename T, int D, int NC>
__device__ __forceinline__ void wall_sum_body(const DevCase<T> &dc, const int bx)
{
    constexpr int M = D + 2;
    constexpr int NR = 2 + 2 * M;               // num, den, outgoing moments A, incoming moments B
    __shared__ double red[NR][8];
    const int s = bx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (s >= dc.NW) return;
    const int f = dc.wface[s];
    const int c = dc.fL[f];
    const int tag = dc.ftag[f];
    const double Tw = dc.wallT[tag];
    const double lw = 1.0 / (2.0 * Tw);
    T wr[GREC];
    for (int d = 0; d < 3; ++d) wr[GR_U + d] = (T)dc.wallU[tag * 3 + d];
    wr[GR_LAM] = (T)lw;
    wr[GR_PREF] = (T)pref_of(1.0, lw, D);
    wr[GR_NB] = (T)(dc.nxi / (2.0 * lw));
    wr[GR_NL2] = (T)(-lw * LOG2E);
    wr[GREC - 1] = T(0);
    T n[D], r[D];
    for (int d = 0; d < D; ++d) {
        n[d] = dc.fn[(size_t)f * D + d];
        r[d] = dc.frL[(size_t)f * D + d];
    }
    const T dt = dc.dtT;
    const T hdt = T(0.5) * dc.dtT;
    const size_t rs = (size_t)NC * dc.nvp;
    // num / den: zero net mass flux (Eq. maxWalldes); A / B: moments (Eq.
    // macroscopicFlux) of the outgoing flux and of the incoming flux of the
    // unit-density wall Maxwellian over the step, so that F_w = A + rho_w B
    CSum<T> v[NR];
    // TW consecutive velocities per thread: the wall cell's limited slope
    // (the gather's slope routine) reads each face entry once for all of them
    constexpr int TW = 4;
    for (int k0 = TW * threadIdx.x; k0 < dc.nvp; k0 += TW * blockDim.x) {
        T u[3][TW], wk[TW], un[TW];
        ldv<T, TW>(dc.u[0] + k0, u[0]);
        ldv<T, TW>(dc.u[1] + k0, u[1]);
        if (D == 3) ldv<T, TW>(dc.u[2] + k0, u[2]);
        else
#pragma unroll
            for (int j = 0; j < TW; ++j) u[2][j] = T(0);
        ldv<T, TW>(dc.w + k0, wk);
        bool out = false;
#pragma unroll
        for (int j = 0; j < TW; ++j) {
            const T uj[3] = {u[0][j], u[1][j], u[2][j]};
            un[j] = normal_velocity<T, D>(uj, n);
            out = out || un[j] > T(0);
        }
        T g[NC][D][TW], fi[NC][TW];
        if (out) cell_slope_tv<T, D, NC, TW>(dc, dc.f_cur + k0, c, u, g, fi);
#pragma unroll
        for (int j = 0; j < TW; ++j) {
            const T uj[3] = {u[0][j], u[1][j], u[2][j]};
            T Fh = 0, Fb = 0;
            int off = -1;
            if (un[j] > T(0)) {
                T hin = fi[0][j], ug = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    hin += g[0][d][j] * r[d];
                    ug += uj[d] * g[0][d][j];
                }
                v[0].add(wk[j] * un[j] * (hin - hdt * ug));
                Fh = dt * un[j] * (hin - hdt * ug);
                if (NC == 2) {
                    T bin = fi[NC - 1][j], ugb = 0;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        bin += g[NC - 1][d][j] * r[d];
                        ugb += uj[d] * g[NC - 1][d][j];
                    }
                    Fb = dt * un[j] * (bin - hdt * ugb);
                }
                off = 2;
            } else if (un[j] < T(0)) {
                const T H = maxwell_h<T, D>(wr, uj);
                v[1].add(wk[j] * un[j] * H);
                Fh = dt * un[j] * H;
                Fb = wr[GR_NB] * Fh;
                off = 2 + M;
            }
            if (off >= 0) {
                T u2 = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) u2 += uj[d] * uj[d];
                T mom[M];
                mom[0] = wk[j] * Fh;
#pragma unroll
                for (int d = 0; d < D; ++d) mom[1 + d] = wk[j] * uj[d] * Fh;
                mom[D + 1] = T(0.5) * wk[j] * (u2 * Fh + (NC == 2 ? Fb : T(0)));
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    if (off == 2) v[2 + i].add(mom[i]);
                    else v[2 + M + i].add(mom[i]);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const double t = warp_sum(v[i].value());
        if (lane == 0) red[i][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a[NR];
        for (int i = 0; i < NR; ++i) {
            a[i] = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a[i] += red[i][w];
        }
        const double rw = -a[0] / a[1];
        dc.rho_w[s] = rw;
        T *w = dc.wrec + (size_t)s * GREC;
        for (int i = 0; i < GREC; ++i) w[i] = wr[i];
        w[GR_PREF] = (T)pref_of(rw, lw, D);
        for (int m = 0; m < M; ++m) dc.wall_F[(size_t)s * M + m] = a[2 + m] + rw * a[2 + M + m];
    }
}

template <typename T, int D, int NC>
__global__ void __launch_bounds__(256) k_wall_sum(DevCase<T> dc)
{
    wall_sum_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void __launch_bounds__(256) k_wall_sum_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    wall_sum_body<T, D, NC>(dc, bx);
}

// ------------------------------------------------------------ gather pass
// One CTA per (patch of P consecutive cells, group of G = vt_group consecutive
// velocity tiles of V = 32*TV velocities); the CTA takes the group's tiles one
// after the other, and in a tile lane l handles the TV consecutive velocities
// V*tile + TV*l + j.  Per tile:
// Phase A: limited slopes of the patch cells and their face neighbours (ring)
//          into shared memory, each computed once.
// Phase B: per patch cell, the flux of every face (Eq. microscopicFlux with
//          Eq. fullSolution; walls per Sec. 2.5) in the cell's own
//          orientation, stage 1 (Eq. microS1) written to f_nxt, and the moments
//          sum_k w psi_k R_k of the flux residual for the W update (Eq.
//          macroscopicUpdata / macroscopicFlux).  The cell's own f and slopes
//          stay in registers; every face entry is read once for all TV
//          velocities of the lane.
// The moments of a cell accumulate over the group's tiles in shared memory
// (the warp that owns a cell is the same for every tile) and are written once
// per (cell, group).  Consecutive tiles of a patch re-read its face entries
// and records from the SM's cache.
//
// Shared memory: the moment accumulators, P x 16 values of T (FP32: the
// double-float pair of each of up to 8 moments; FP64: the moments), then the
// slope buffer, (patch + ring) x NC x D x V values of T.
template <typename T>
__host__ __device__ constexpr int gather_acc_values(int P) { return P * 16; }

template <typename T, int D, int NC, int TV>
__device__ __forceinline__ void gather_item(const DevCase<T> &dc, const int p, const int grp, T *sg)
{
    constexpr int V = 32 * TV;
    constexpr int M = D + 2;
    // velocities per lane of the slope pass: twice TV in the FP32 form with one
    // stored component (a half-warp per slope cell), else TV (registers)
    constexpr int TVA = std::is_same<T, float>::value && NC == 1 && TV <= 2 ? 2 * TV : TV;
    using E = GEnt<D>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int cb = p * dc.P;
    const int npc = min(dc.P, dc.C - cb);
    const int rb = dc.ring_ptr[p], re = dc.ring_ptr[p + 1];
    const int nslope = npc + (re - rb);
    const int nvp = dc.nvp;
    const size_t rs = (size_t)NC * nvp;
    T *const sacc = sg;                         // moment accumulators [P][16]
    T *const sl = sg + gather_acc_values<T>(dc.P) + TV * lane;   // this lane's column of the slope buffer
    for (int i = threadIdx.x; i < gather_acc_values<T>(dc.P); i += blockDim.x) sacc[i] = T(0);
    const int vt0 = grp * dc.vt_group, vt1 = min(dc.n_vt, vt0 + dc.vt_group);
    for (int vt = vt0; vt < vt1; ++vt) {
        const int kl = vt * V + TV * lane;
        const T *__restrict__ fl = dc.f_cur + kl;

        T u[3][TV];
        auto load_u = [&](int k, auto &uu) {
            constexpr int N = sizeof(uu[0]) / sizeof(T);
            ldv<T, N>(dc.u[0] + k, uu[0]);
            ldv<T, N>(dc.u[1] + k, uu[1]);
            if (D == 3) ldv<T, N>(dc.u[2] + k, uu[2]);
            else
#pragma unroll
                for (int j = 0; j < N; ++j) uu[2][j] = T(0);
        };

        // ---- phase A: slopes (micro reconstruction of the velocity loop, Algorithm 1)
        if constexpr (TVA == TV) {
            load_u(kl, u);
            for (int s = warp; s < nslope; s += nwarps) {
                const int c = s < npc ? cb + s : dc.ring_cells[rb + s - npc];
                T g[NC][D][TV], fi[NC][TV];
                cell_slope_tv<T, D, NC, TV>(dc, fl, c, u, g, fi);
#pragma unroll
                for (int m = 0; m < NC; ++m)
#pragma unroll
                    for (int d = 0; d < D; ++d) stv<T, TV>(sl + ((s * NC + m) * D + d) * V, g[m][d]);
            }
        } else {
            // each half-warp takes a slope cell, TVA velocities per lane: the
            // face entries are read once for twice the velocities
            const int hl = lane & 15;
            const int klA = vt * V + TVA * hl;
            T ua[3][TVA];
            load_u(klA, ua);
            const T *__restrict__ fla = dc.f_cur + klA;
            T *const sla = sg + gather_acc_values<T>(dc.P) + TVA * hl;
            for (int s = 2 * warp + (lane >> 4); s < nslope; s += 2 * nwarps) {
                const int c = s < npc ? cb + s : dc.ring_cells[rb + s - npc];
                T g[NC][D][TVA], fi[NC][TVA];
                cell_slope_tv<T, D, NC, TVA>(dc, fla, c, ua, g, fi);
#pragma unroll
                for (int m = 0; m < NC; ++m)
#pragma unroll
                    for (int d = 0; d < D; ++d) stv<T, TVA>(sla + ((s * NC + m) * D + d) * V, g[m][d]);
            }
            load_u(kl, u);
        }
        __syncthreads();

        // ---- phase B: fluxes, stage 1, moments (velocity loop and wall flux, Algorithm 1)
        const T dt = dc.dtT;
        const T hdt2 = T(0.5) * dc.dtT * dc.dtT;
        for (int s = warp; s < npc; s += nwarps) {
            const int c = cb + s;
            T fs[NC][TV], gs[NC][D][TV], R[NC][TV];
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                ldv<T, TV>(fl + (size_t)c * rs + (size_t)m * nvp, fs[m]);
#pragma unroll
                for (int d = 0; d < D; ++d) ldv_s<T, TV>(sl + ((s * NC + m) * D + d) * V, gs[m][d]);
#pragma unroll
                for (int j = 0; j < TV; ++j) R[m][j] = 0;
            }
            const int e0 = __ldg(dc.cf_ptr + c), e1 = __ldg(dc.cf_ptr + c + 1);
#pragma unroll 4
            for (int e = e0; e < e1; ++e) {
                const int4 gi = __ldg(dc.gi + e);
                T ge[E::LEN];
                if constexpr (E::SKIP1 > E::SKIP0) {
                    load_rec<E::SKIP0>(dc.gf + (size_t)e * E::LEN, *reinterpret_cast<T (*)[E::SKIP0]>(ge));
                    load_rec<E::LEN - E::SKIP1>(dc.gf + (size_t)e * E::LEN + E::SKIP1,
                                                *reinterpret_cast<T (*)[E::LEN - E::SKIP1]>(ge + E::SKIP1));
                } else {
                    load_rec<E::LEN>(dc.gf + (size_t)e * E::LEN, ge);
                }
                const T cs = ge[E::CS];
                T un[TV];
#pragma unroll
                for (int j = 0; j < TV; ++j) {
                    const T uj[3] = {u[0][j], u[1][j], u[2][j]};
                    un[j] = normal_velocity<T, D>(uj, ge + E::N);
                }
                if (gi.z == FT_WALL) {
                    T wr[GREC];
                    load_rec<GREC>(dc.wrec + (size_t)gi.x * GREC, wr);
#pragma unroll
                    for (int j = 0; j < TV; ++j) {
                        const T uj[3] = {u[0][j], u[1][j], u[2][j]};
                        T F[NC];
                        if (un[j] > T(0)) {
#pragma unroll
                            for (int m = 0; m < NC; ++m) {
                                T fin = fs[m][j], ug = 0;
#pragma unroll
                                for (int d = 0; d < D; ++d) {
                                    fin += gs[m][d][j] * ge[E::RS + d];
                                    ug += uj[d] * gs[m][d][j];
                                }
                                F[m] = un[j] * (dt * fin - hdt2 * ug);
                            }
                        } else {
                            const T H = maxwell_h<T, D>(wr, uj);
                            F[0] = un[j] * dt * H;
                            if (NC == 2) F[NC - 1] = un[j] * dt * wr[GR_NB] * H;
                        }
#pragma unroll
                        for (int m = 0; m < NC; ++m) R[m][j] += cs * F[m];
                    }
                    continue;
                }
                T fr[XREC];
                load_rec<XREC>(dc.xrec + (size_t)gi.y * XREC, fr);
                if (gi.z == FT_FARFIELD) {
                    T gr[GREC];
                    load_rec<GREC>(dc.grec + (size_t)gi.x * GREC, gr);
#pragma unroll
                    for (int j = 0; j < TV; ++j) {
                        const T uj[3] = {u[0][j], u[1][j], u[2][j]};
                        T fup[NC], ugf[NC], F[NC];
                        if (un[j] > T(0)) {
#pragma unroll
                            for (int m = 0; m < NC; ++m) {
                                T v = fs[m][j], ug = 0;
#pragma unroll
                                for (int d = 0; d < D; ++d) {
                                    v += gs[m][d][j] * ge[E::RS + d];
                                    ug += uj[d] * gs[m][d][j];
                                }
                                fup[m] = v;
                                ugf[m] = ug;
                            }
                        } else {
                            const T H = maxwell_h<T, D>(gr, uj);
                            fup[0] = H;
                            if (NC == 2) fup[NC - 1] = gr[GR_NB] * H;
#pragma unroll
                            for (int m = 0; m < NC; ++m) ugf[m] = 0;
                        }
                        interface_flux<T, D, NC>(fr, uj, un[j], fup, ugf, F);
#pragma unroll
                        for (int m = 0; m < NC; ++m) R[m][j] += cs * F[m];
                    }
                    continue;
                }
                // interior or periodic: the neighbour's f and slopes
                T fo[NC][TV], go[NC][D][TV];
                const T *so = sl + (size_t)gi.w * NC * D * V;
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    ldv<T, TV>(fl + (size_t)gi.x * rs + (size_t)m * nvp, fo[m]);
#pragma unroll
                    for (int d = 0; d < D; ++d) ldv_s<T, TV>(so + (m * D + d) * V, go[m][d]);
                }
#pragma unroll
                for (int j = 0; j < TV; ++j) {
                    const T uj[3] = {u[0][j], u[1][j], u[2][j]};
                    const bool self = un[j] > T(0);
                    T fup[NC], ugf[NC], F[NC];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        T v = self ? fs[m][j] : fo[m][j], ug = 0;
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            const T gd = self ? gs[m][d][j] : go[m][d][j];
                            v += gd * (self ? ge[E::RS + d] : ge[E::RO + d]);
                            ug += uj[d] * gd;
                        }
                        fup[m] = v;
                        ugf[m] = ug;
                    }
                    interface_flux<T, D, NC>(fr, uj, un[j], fup, ugf, F);
#pragma unroll
                    for (int m = 0; m < NC; ++m) R[m][j] += cs * F[m];
                }
            }
            // stage 1 and the moments of R
            T cr[CREC];
            load_rec<CREC>(dc.crec + (size_t)c * CREC, cr);
            const T cc = cr[CR_C];
            T wk[TV];
            ldv<T, TV>(dc.w + kl, wk);
            // moments sum_k w psi_k R_k of this tile: FP64 sums in the FP64 form;
            // in the FP32 form each term is an FP32 product, and the sums over the
            // lane's velocities and across the warp are double-float (error-free
            // additions), widened to FP64 for the W update
            constexpr int NR = M <= 4 ? 4 : 8;
            T mh[NR], ml[NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) mh[i] = ml[i] = T(0);
            T out[NC][TV];
#pragma unroll
            for (int j = 0; j < TV; ++j) {
                const T uj[3] = {u[0][j], u[1][j], u[2][j]};
                T fp[NC];
                shakhov_fplus<T, D, NC>(cr, uj, fp);
#pragma unroll
                for (int m = 0; m < NC; ++m) out[m][j] = fs[m][j] + R[m][j] + cc * (fp[m] - fs[m][j]);
                T u2 = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) u2 += uj[d] * uj[d];
                const T wr0 = wk[j] * R[0][j];
                T x[M];
                x[0] = wr0;
#pragma unroll
                for (int d = 0; d < D; ++d) x[1 + d] = uj[d] * wr0;
                x[D + 1] = T(0.5) * (u2 * wr0 + (NC == 2 ? wk[j] * R[NC - 1][j] : T(0)));
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    if constexpr (std::is_same<T, float>::value) {
                        if (j == 0) mh[i] = x[i];
                        else ff_add(mh[i], ml[i], x[i], 0.f);
                    } else {
                        mh[i] += x[i];
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < NC; ++m) stv<T, TV>(dc.f_nxt + kl + (size_t)c * rs + (size_t)m * nvp, out[m]);
            const int vi = lane >> (NR == 4 ? 3 : 2);
            const bool holder = (lane & (NR == 4 ? 7 : 3)) == 0 && vi < M;
            if constexpr (std::is_same<T, float>::value) {
                float oh, ol;
                warp_transpose_sum_ff2<NR>(mh, ml, oh, ol);
                if (holder) ff_add(sacc[s * 16 + vi], sacc[s * 16 + 8 + vi], oh, ol);
            } else {
                const T sm = warp_transpose_sum<T, NR>(mh);
                if (holder) sacc[s * 16 + vi] += sm;
            }
        }
        __syncthreads();                        // the next tile's slopes overwrite the buffer
    }
    // the moments of the group, once per (cell, group), by the warp that owns the cell
    for (int s = warp; s < npc; s += nwarps) {
        const int vi = lane >> (M <= 4 ? 3 : 2);
        if ((lane & (M <= 4 ? 7 : 3)) == 0 && vi < M) {
            double v = (double)sacc[s * 16 + vi];
            if constexpr (std::is_same<T, float>::value) v += (double)sacc[s * 16 + 8 + vi];
            dc.dW_part[((size_t)(cb + s) * dc.n_groups + grp) * M + vi] = v;
        }
    }
}

// NTH threads per CTA; 512-thread CTAs are held to 64 registers so that two
// fit an SM (32 resident warps, against 24 for 256-thread CTAs at 80).  A
// minimum of 0 blocks leaves 256-thread CTAs to ptxas's own register choice:
// an explicit 1 lets it take 113 registers in the 2D FP32 kernel, which
// drops the SM to two CTAs and costs about 20 %.
template <typename T, int D, int NC, int TV, int NTH>
__global__ void __launch_bounds__(NTH, NTH >= 512 ? 2 : 0) k_gather(DevCase<T> dc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // One-dimensional grid of n_patches x n_groups blocks, patches fastest:
    // the CTAs in flight cover neighbouring patches in the same tile group,
    // so the rows of f they share (ring cells) are read from L2.
    const int grp = blockIdx.x / dc.n_patches;
    gather_item<T, D, NC, TV>(dc, blockIdx.x - grp * dc.n_patches, grp, reinterpret_cast<T *>(smem_raw));
}

// Persistent gather over many cases: a fixed grid of CTAs walks a work list of
// (case, patch, tile group) items; each item is exactly the CTA of k_gather
// for that case, so every case gets bit-identical results alone or batched.
template <typename T, int D, int NC, int TV, int NTH>
__global__ void __launch_bounds__(NTH, NTH >= 512 ? 2 : 0) k_gather_batch(const DevCase<T> *__restrict__ cases,
                                                                          const int4 *__restrict__ work, int nwork)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int4 it = work[w];
        gather_item<T, D, NC, TV>(cases[it.x], it.y, it.z, reinterpret_cast<T *>(smem_raw));
        __syncthreads();
    }
}

// ------------------------------------------------------------ W update
template <typename T, int D, int NC>
__device__ __forceinline__ void update_W_body(const DevCase<T> &dc, const int bx)
{
    constexpr int M = D + 2;
    __shared__ double red[2 * M][8];
    const int c = bx * blockDim.x + threadIdx.x;
    double dsq[M], wsq[M];
    for (int m = 0; m < M; ++m) dsq[m] = wsq[m] = 0.0;
    if (c < dc.C) {
        double *Wc = dc.W + (size_t)c * M;
        const bool counts = !dc.owned || dc.owned[c];      // halo cells of a subdomain do not count
        for (int m = 0; m < M; ++m) {
            double s = 0.0;
            for (int t = 0; t < dc.n_groups; ++t) s += dc.dW_part[((size_t)c * dc.n_groups + t) * M + m];
            if (counts) {
                wsq[m] = Wc[m] * Wc[m];
                dsq[m] = s * s;
            }
            Wc[m] += s;
        }
        Prim p = prim_of(Wc, D);
        if (!(p.rho > 0.0) || !(p.T > 0.0) || !isfinite(p.rho) || !isfinite(p.T)) atomicOr(dc.flags, 1);
        const double tau = tau_of(dc, p.rho, p.T);
        const double kappa = 4.0 * (1.0 - dc.Pr) * p.lam * p.lam / (5.0 * p.rho);
        T *r = dc.krec + (size_t)c * CREC;
        for (int d = 0; d < 3; ++d) r[CR_U + d] = (T)p.U[d];
        r[CR_LAM] = (T)p.lam;
        r[CR_PREF] = (T)pref_of(p.rho, p.lam, D);
        for (int d = 0; d < 3; ++d) r[CR_KQ + d] = d < D ? (T)(kappa * dc.q[(size_t)c * D + d]) : T(0);
        const double cc = 0.5 * dc.dt / tau;
        r[CR_C] = (T)cc;
        r[CR_INV] = (T)(1.0 / (1.0 + cc));
        r[CR_NB] = (T)(dc.nxi / (2.0 * p.lam));
        r[CR_NL2] = (T)(-p.lam * LOG2E);
    }
    // deterministic block partials of the residual
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int m = 0; m < M; ++m) {
        double a = warp_sum(dsq[m]), b = warp_sum(wsq[m]);
        if (lane == 0) {
            red[m][warp] = a;
            red[M + m][warp] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * M) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
        dc.res_part[(size_t)bx * 2 * M + threadIdx.x] = s;
    }
}

template <typename T, int D, int NC>
__global__ void __launch_bounds__(256) k_update_W(DevCase<T> dc)
{
    update_W_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void __launch_bounds__(256) k_update_W_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off, int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    update_W_body<T, D, NC>(dc, bx);
}

template <int M>
__global__ void k_residual(const double *res_part, int nblocks, double *res)
{
    __shared__ double acc[2 * M][32];
    const int t = threadIdx.x;
    for (int i = 0; i < 2 * M; ++i) {
        double s = 0.0;
        for (int b = t; b < nblocks; b += 32) s += res_part[(size_t)b * 2 * M + i];
        acc[i][t] = s;
    }
    __syncwarp();
    if (t < M) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 32; ++w) {
            a += acc[t][w];
            b += acc[M + t][w];
        }
        res[t] = b > 0.0 ? sqrt(a) / sqrt(b) : sqrt(a);
    }
}

// ------------------------------------------------------------ stage 2
template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

// 4 consecutive velocities per lane (rows are padded to a multiple of 32, so
// every row start is 16-byte aligned for FP32 and 32-byte aligned for FP64)
template <typename T, int D, int NC>
__device__ __forceinline__ void collide_body(const DevCase<T> &dc, const int bx)
{
    using V4 = typename Vec4<T>::type;
    const int c = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= dc.C) return;
    // the cell's record in registers: read once, not again after every store of f
    T kr[CREC];
#pragma unroll
    for (int i = 0; i < CREC; ++i) kr[i] = __ldg(dc.krec + (size_t)c * CREC + i);
    const T cc = kr[CR_C];
    const T inv = kr[CR_INV];
    T U[D];
#pragma unroll
    for (int d = 0; d < D; ++d) U[d] = kr[CR_U + d];
    const size_t rs = (size_t)NC * dc.nvp;
    // heat-flux terms: FP64 sums in the FP64 form; blocked sums accumulated in
    // FP64 in the FP32 form (16 terms per lane per block)
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int NP = D == 2 ? 2 : 4;
    T blk[NP];
#pragma unroll
    for (int d = 0; d < NP; ++d) blk[d] = 0;
    double acc = 0.0;
    int nblk = 0;
    // the f~ vectors of the next iteration are loaded before this one's
    // arithmetic, so that a warp keeps a load in flight while it computes
    const T *frow = dc.f_nxt + (size_t)c * rs;
    V4 nxt[NC];
    if (4 * lane < dc.nvp)
#pragma unroll
        for (int m = 0; m < NC; ++m) nxt[m] = *reinterpret_cast<const V4 *>(frow + (size_t)m * dc.nvp + 4 * lane);
    for (int k00 = 0; k00 < dc.nvp; k00 += 128) {          // uniform over the warp
        const int k0 = k00 + 4 * lane;
        if (k0 < dc.nvp) {
            T ft[NC][4], fn[NC][4];
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                const V4 v = nxt[m];
                ft[m][0] = v.x;
                ft[m][1] = v.y;
                ft[m][2] = v.z;
                ft[m][3] = v.w;
            }
            if (k0 + 128 < dc.nvp)
#pragma unroll
                for (int m = 0; m < NC; ++m)
                    nxt[m] = *reinterpret_cast<const V4 *>(frow + (size_t)m * dc.nvp + k0 + 128);
            // the lane's four velocities from the per-component arrays: each load
            // of the warp covers one contiguous span (the packed [k][4] records
            // of four consecutive velocities per lane would touch four times the
            // cache lines per load)
            T uv[3][4], wv[4];
            ldv<T, 4>(dc.u[0] + k0, uv[0]);
            ldv<T, 4>(dc.u[1] + k0, uv[1]);
            if (D == 3) ldv<T, 4>(dc.u[2] + k0, uv[2]);
            else
#pragma unroll
                for (int j = 0; j < 4; ++j) uv[2][j] = T(0);
            ldv<T, 4>(dc.w + k0, wv);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const T u[3] = {uv[0][j], uv[1][j], uv[2][j]};
                const T wk = wv[j];
                T fp[NC];
                shakhov_fplus<T, D, NC>(kr, u, fp);
#pragma unroll
                for (int m = 0; m < NC; ++m) fn[m][j] = (ft[m][j] + cc * fp[m]) * inv;
                T cv[D], c2 = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    cv[d] = u[d] - U[d];
                    c2 += cv[d] * cv[d];
                }
                const T we = wk * (c2 * fn[0][j] + (NC == 2 ? fn[NC - 1][j] : T(0)));
#pragma unroll
                for (int d = 0; d < D; ++d) blk[d] += cv[d] * we;
            }
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                V4 v;
                v.x = fn[m][0];
                v.y = fn[m][1];
                v.z = fn[m][2];
                v.w = fn[m][3];
                *reinterpret_cast<V4 *>(dc.f_cur + (size_t)c * rs + (size_t)m * dc.nvp + k0) = v;
            }
        }
        if constexpr (F32) {
            if (++nblk == SUM_BLOCK / 4 || k00 + 128 >= dc.nvp) {
                acc += block_to_fp64<NP>(blk);
#pragma unroll
                for (int d = 0; d < NP; ++d) blk[d] = 0;
                nblk = 0;
            }
        }
    }
    if constexpr (F32) {
        // lanes 16j.. (D = 2) or 8j.. (D = 3) hold component j
        const int vi = lane >> (NP == 2 ? 4 : 3);
        if ((lane & (NP == 2 ? 15 : 7)) == 0 && vi < D) dc.q[(size_t)c * D + vi] = 0.5 * acc;
    } else {
        for (int d = 0; d < D; ++d) {
            const double sm = warp_sum(blk[d]);
            if (lane == 0) dc.q[(size_t)c * D + d] = 0.5 * sm;
        }
    }
}

// five 256-thread blocks per SM in the 2D FP32 form (48 registers); the 3D
// FP32 form and the batched kernels would spill at that bound
template <typename T, int D, int NC>
__global__ void __launch_bounds__(256, sizeof(T) == 4 && D == 2 ? 5 : 0) k_collide(DevCase<T> dc)
{
    collide_body<T, D, NC>(dc, blockIdx.x);
}

template <typename T, int D, int NC>
__global__ void __launch_bounds__(256) k_collide_batch(const DevCase<T> *__restrict__ cases, const int *__restrict__ off,
                                                       int n)
{
    int bx;
    const DevCase<T> &dc = batch_case(cases, off, n, bx);
    collide_body<T, D, NC>(dc, bx);
}

// ------------------------------------------------------------ state I/O
// Host-layout element type S: double, or float for callers that hold the
// distribution in single precision (exact for FP32 storage).
template <typename T, int D, int NC, typename S>
__global__ void k_f_export(DevCase<T> dc, const long long *perm, int c0, int nc, S *out)
{
    // out[(i - c0)][m][k] (caller cell order i) from internal cell perm[i]
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long per = (long long)NC * dc.nv;
    if (idx >= (long long)nc * per) return;
    const int i = c0 + (int)(idx / per);
    const long long r = idx % per;
    const int m = (int)(r / dc.nv), k = (int)(r % dc.nv);
    const long long ci = perm[i];
    out[idx] = (S)dc.f_cur[(size_t)ci * NC * dc.nvp + (size_t)m * dc.nvp + k];
}

template <typename T, int D, int NC, typename S>
__global__ void k_f_import(DevCase<T> dc, const long long *perm, int c0, int nc, const S *in)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long per = (long long)NC * dc.nvp;
    if (idx >= (long long)nc * per) return;
    const int i = c0 + (int)(idx / per);
    const long long r = idx % per;
    const int m = (int)(r / dc.nvp), k = (int)(r % dc.nvp);
    const long long ci = perm[i];
    dc.f_cur[(size_t)ci * NC * dc.nvp + (size_t)m * dc.nvp + k] =
        k < dc.nv ? (T)in[((long long)(i - c0) * NC + m) * dc.nv + k] : T(0);
}

template <int D>
__global__ void k_moments_out(const double *W, const double *q, const long long *perm, int C, double *out)
{
    // out[i][0..]: rho, U[D], T, q[D] in caller order
    constexpr int M = D + 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const long long c = perm[i];
    Prim p = prim_of(W + (size_t)c * M, D);
    double *o = out + (size_t)i * (2 * D + 2);
    o[0] = p.rho;
    for (int d = 0; d < D; ++d) o[1 + d] = p.U[d];
    o[D + 1] = p.T;
    for (int d = 0; d < D; ++d) o[D + 2 + d] = q[(size_t)c * D + d];
}

template <int D>
__global__ void k_W_permute(const double *src, const long long *perm, int C, double *dst, int to_internal)
{
    constexpr int M = D + 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const long long c = perm[i];
    for (int m = 0; m < M; ++m) {
        if (to_internal) dst[(size_t)c * M + m] = src[(size_t)i * M + m];
        else dst[(size_t)i * M + m] = src[(size_t)c * M + m];
    }
}

__global__ void k_check(const double *W, int n, int M, int *flags)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const double *w = W + (size_t)c * M;
    double ke = 0.0;
    for (int d = 1; d < M - 1; ++d) ke += w[d] * w[d];
    const double e = w[M - 1] - 0.5 * ke / w[0];
    bool bad = !(w[0] > 0.0) || !(e > 0.0);
    for (int m = 0; m < M; ++m) bad |= !isfinite(w[m]);
    if (bad) atomicOr(flags, 1);
}

// Smallest and largest density over the own cells (owned == NULL: all cells).
// Densities are positive doubles, whose bit patterns order as the values do;
// a non-positive or non-finite density enters as +0.  range[0] starts at all
// ones (atomicMin), range[1] at zero (atomicMax).
__global__ void k_density_range(const double *W, int n, int M, const unsigned char *owned,
                                unsigned long long *range)
{
    unsigned long long lo = ~0ull, hi = 0ull;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        if (owned && !owned[c]) continue;
        const double r = W[(size_t)c * M];
        const unsigned long long b = (r > 0.0 && isfinite(r)) ? (unsigned long long)__double_as_longlong(r) : 0ull;
        lo = b < lo ? b : lo;
        hi = b > hi ? b : hi;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&range[0], lo);
        atomicMax(&range[1], hi);
    }
}

// ------------------------------------------------------------ halo exchange
// Rows of the halo buffer: f of the cell in the storage type [NC][nv], padded
// to 8 bytes, then W [D+2] and q [D] in FP64.  One block per listed cell.
template <typename T, int D, int NC>
__global__ void k_halo_pack(DevCase<T> dc, const int *cells, int n, size_t row, unsigned char *buf)
{
    constexpr int M = D + 2;
    const int i = blockIdx.x;
    if (i >= n) return;
    const int c = cells[i];
    unsigned char *r = buf + (size_t)i * row;
    T *fo = reinterpret_cast<T *>(r);
    const T *fc = dc.f_cur + (size_t)c * NC * dc.nvp;
    for (int j = threadIdx.x; j < NC * dc.nv; j += blockDim.x) fo[j] = fc[(size_t)(j / dc.nv) * dc.nvp + j % dc.nv];
    double *tail = reinterpret_cast<double *>(r + row - (size_t)(M + D) * sizeof(double));
    if (threadIdx.x < M) tail[threadIdx.x] = dc.W[(size_t)c * M + threadIdx.x];
    else if (threadIdx.x < M + D) tail[threadIdx.x] = dc.q[(size_t)c * D + threadIdx.x - M];
}

template <typename T, int D, int NC>
__global__ void k_halo_unpack(DevCase<T> dc, const int *cells, int n, size_t row, const unsigned char *buf)
{
    constexpr int M = D + 2;
    const int i = blockIdx.x;
    if (i >= n) return;
    const int c = cells[i];
    const unsigned char *r = buf + (size_t)i * row;
    const T *fi = reinterpret_cast<const T *>(r);
    T *fc = dc.f_cur + (size_t)c * NC * dc.nvp;
    for (int j = threadIdx.x; j < NC * dc.nv; j += blockDim.x) fc[(size_t)(j / dc.nv) * dc.nvp + j % dc.nv] = fi[j];
    const double *tail = reinterpret_cast<const double *>(r + row - (size_t)(M + D) * sizeof(double));
    if (threadIdx.x < M) dc.W[(size_t)c * M + threadIdx.x] = tail[threadIdx.x];
    else if (threadIdx.x < M + D) dc.q[(size_t)c * D + threadIdx.x - M] = tail[threadIdx.x];
}

// ------------------------------------------------------------ launchers
static inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

template <typename T, int D, int NC, int TV, int NTH>
static cudaError_t gather_launch(const DevCase<T> &dc, size_t smem, cudaStream_t st)
{
    auto kern = k_gather<T, D, NC, TV, NTH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = dc.n_patches * dc.n_groups;
    kern<<<grid, NTH, smem, st>>>(dc);
    return cudaGetLastError();
}

// the gather kernel of a case: velocities per lane TV = vtile / 32 and
// threads per CTA (256, or 512 for FP32 at TV <= 2)
template <typename T, int D, int NC>
static cudaError_t gather_dispatch(const DevCase<T> &dc, size_t smem, cudaStream_t st)
{
    const int tv = dc.vtile / 32;
    if (dc.nth == 512) {
        if constexpr (std::is_same<T, float>::value) {
            if (tv == 1) return gather_launch<T, D, NC, 1, 512>(dc, smem, st);
            if (tv == 2) return gather_launch<T, D, NC, 2, 512>(dc, smem, st);
        }
        return cudaErrorInvalidValue;
    }
    if (dc.nth != 256) return cudaErrorInvalidValue;
    if (tv == 1) return gather_launch<T, D, NC, 1, 256>(dc, smem, st);
    if (tv == 2) return gather_launch<T, D, NC, 2, 256>(dc, smem, st);
    if (tv == 4) return gather_launch<T, D, NC, 4, 256>(dc, smem, st);
    return cudaErrorInvalidValue;
}

// Blocks, threads and dynamic shared memory of the per-case kernels of a step
// (SmallKernel order); 0 blocks: the case does not run that kernel.
template <typename T, int D>
static int sk_blocks(const DevCase<T> &dc, int k)
{
    const int C = dc.C, F = dc.F;
    const bool faces = F > 0, sums1 = faces && !dc.w0_analytic;
    switch (k) {
    case SK_PREP: return cdiv(C + dc.G, 128);
    case SK_MACRO_GRAD: return cdiv(C, 128);
    case SK_FACE_PRE: return faces ? cdiv(F, 128) : 0;
    case SK_FACE_SUM1_SEP: return sums1 && dc.sep1 ? cdiv(F, SUM1_SEP_WARPS) : 0;
    case SK_FACE_SUM1: return sums1 && !dc.sep1 ? cdiv(F, 8) : 0;
    case SK_FACE_FIN1: return faces ? cdiv(F, 128) : 0;
    case SK_FACE_SUM2_SEP: return faces && dc.sep ? cdiv(F, 8) : 0;
    case SK_FACE_SUM2: return faces && !dc.sep ? cdiv(F, 8) : 0;
    case SK_FACE_FIN2: return faces ? cdiv(F, 64) : 0;
    case SK_WALL_SUM: return dc.NW;
    case SK_UPDATE_W: return cdiv(C, 256);
    case SK_COLLIDE: return cdiv(C, 8);
    default: return 0;
    }
}

constexpr int kSkThreads[SK_COUNT] = {128, 128, 128, 32 * SUM1_SEP_WARPS, 256, 128, 256, 256, 64, 256, 256, 256};

template <typename T, int D>
static size_t sk_smem(const DevCase<T> &dc, int k)
{
    // k_face_sum1_sep: prefix sums of the last axis, 2 sides x 3 powers per warp
    return k == SK_FACE_SUM1_SEP ? (size_t)SUM1_SEP_WARPS * 6 * (dc.cart_n[D - 1] + 1) * sizeof(T) : 0;
}

// one per-case kernel, for one case (cases == nullptr) or for the cases of a
// batch (block offsets off[0..n])
template <typename T, int D, int NC>
static cudaError_t sk_launch(int k, int blocks, size_t smem, cudaStream_t st, const DevCase<T> *dc,
                             const DevCase<T> *cases, const int *off, int n)
{
    if (blocks <= 0) return cudaSuccess;
    const int nt = kSkThreads[k];
#define UGKS_SK(ID, K)                                                                                  \
    case ID:                                                                                            \
        if (cases) K##_batch<T, D, NC><<<blocks, nt, smem, st>>>(cases, off, n);                        \
        else K<T, D, NC><<<blocks, nt, smem, st>>>(*dc);                                                \
        break;
    if (k == SK_FACE_SUM1_SEP && smem > 48 * 1024) {
        cudaError_t e = cases ? cudaFuncSetAttribute(k_face_sum1_sep_batch<T, D, NC>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                              : cudaFuncSetAttribute(k_face_sum1_sep<T, D, NC>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    switch (k) {
        UGKS_SK(SK_PREP, k_prep)
        UGKS_SK(SK_MACRO_GRAD, k_macro_grad)
        UGKS_SK(SK_FACE_PRE, k_face_pre)
        UGKS_SK(SK_FACE_SUM1_SEP, k_face_sum1_sep)
        UGKS_SK(SK_FACE_SUM1, k_face_sum1)
        UGKS_SK(SK_FACE_FIN1, k_face_fin1)
        UGKS_SK(SK_FACE_SUM2_SEP, k_face_sum2_sep)
        UGKS_SK(SK_FACE_SUM2, k_face_sum2)
        UGKS_SK(SK_FACE_FIN2, k_face_fin2)
        UGKS_SK(SK_WALL_SUM, k_wall_sum)
        UGKS_SK(SK_UPDATE_W, k_update_W)
        UGKS_SK(SK_COLLIDE, k_collide)
    default: return cudaErrorInvalidValue;
    }
#undef UGKS_SK
    return cudaGetLastError();
}

template <typename T, int D, int NC>
static void sk_case(const DevCase<T> &dc, int k, cudaStream_t st)
{
    sk_launch<T, D, NC>(k, sk_blocks<T, D>(dc, k), sk_smem<T, D>(dc, k), st, &dc, nullptr, nullptr, 0);
}

template <typename T, int D, int NC>
static void pre_gather(const DevCase<T> &dc, cudaStream_t st, cudaEvent_t *ev)
{
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev[i], st);
    };
    mark(0);
    sk_case<T, D, NC>(dc, SK_PREP, st);
    sk_case<T, D, NC>(dc, SK_MACRO_GRAD, st);
    mark(1);
    for (int k = SK_FACE_PRE; k <= SK_FACE_FIN2; ++k) sk_case<T, D, NC>(dc, k, st);
    mark(2);
    sk_case<T, D, NC>(dc, SK_WALL_SUM, st);
    mark(3);
}

template <typename T, int D, int NC>
static void post_gather(const DevCase<T> &dc, const StepConfig &, cudaStream_t st, cudaEvent_t *ev)
{
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev[i], st);
    };
    mark(4);
    sk_case<T, D, NC>(dc, SK_UPDATE_W, st);
    mark(5);
    sk_case<T, D, NC>(dc, SK_COLLIDE, st);
    mark(6);
}

template <typename T, int D, int NC>
static cudaError_t step_dn(const DevCase<T> &dc, const StepConfig &cfg, cudaStream_t st, cudaEvent_t *ev)
{
    pre_gather<T, D, NC>(dc, st, ev);
    cudaError_t e = gather_dispatch<T, D, NC>(dc, cfg.smem, st);
    if (e != cudaSuccess) return e;
    post_gather<T, D, NC>(dc, cfg, st, ev);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pre_gather(const DevCase<T> &dc, cudaStream_t st)
{
    if (dc.D == 2) pre_gather<T, 2, 2>(dc, st, nullptr);
    else pre_gather<T, 3, 1>(dc, st, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_post_gather(const DevCase<T> &dc, const StepConfig &cfg, cudaStream_t st)
{
    if (dc.D == 2) post_gather<T, 2, 2>(dc, cfg, st, nullptr);
    else post_gather<T, 3, 1>(dc, cfg, st, nullptr);
    return cudaGetLastError();
}

template <typename T>
int small_kernel_blocks(const DevCase<T> &dc, int k)
{
    return dc.D == 2 ? sk_blocks<T, 2>(dc, k) : sk_blocks<T, 3>(dc, k);
}

template <typename T>
size_t small_kernel_smem(const DevCase<T> &dc, int k)
{
    return dc.D == 2 ? sk_smem<T, 2>(dc, k) : sk_smem<T, 3>(dc, k);
}

template <typename T>
cudaError_t launch_small_batch(int D, int k, const DevCase<T> *cases, const int *off, int n, int blocks, size_t smem,
                               cudaStream_t st)
{
    if (D == 2) return sk_launch<T, 2, 2>(k, blocks, smem, st, nullptr, cases, off, n);
    return sk_launch<T, 3, 1>(k, blocks, smem, st, nullptr, cases, off, n);
}

template <typename T>
cudaError_t launch_gather(const DevCase<T> &dc, size_t smem, cudaStream_t st)
{
    if (dc.D == 2) return gather_dispatch<T, 2, 2>(dc, smem, st);
    return gather_dispatch<T, 3, 1>(dc, smem, st);
}

template <typename T, int D, int NC, int TV, int NTH>
static cudaError_t gather_batch_launch(const DevCase<T> *cases, const int4 *work, int nwork, int grid, size_t smem,
                                       cudaStream_t st)
{
    auto kern = k_gather_batch<T, D, NC, TV, NTH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NTH, smem, st>>>(cases, work, nwork);
    return cudaGetLastError();
}

template <typename T, int D, int NC>
static cudaError_t gather_batch_dispatch(int vtile, int nth, const DevCase<T> *cases, const int4 *work, int nwork,
                                         int grid, size_t smem, cudaStream_t st)
{
    const int tv = vtile / 32;
    if (nth == 512) {
        if constexpr (std::is_same<T, float>::value) {
            if (tv == 1) return gather_batch_launch<T, D, NC, 1, 512>(cases, work, nwork, grid, smem, st);
            if (tv == 2) return gather_batch_launch<T, D, NC, 2, 512>(cases, work, nwork, grid, smem, st);
        }
        return cudaErrorInvalidValue;
    }
    if (nth != 256) return cudaErrorInvalidValue;
    if (tv == 1) return gather_batch_launch<T, D, NC, 1, 256>(cases, work, nwork, grid, smem, st);
    if (tv == 2) return gather_batch_launch<T, D, NC, 2, 256>(cases, work, nwork, grid, smem, st);
    if (tv == 4) return gather_batch_launch<T, D, NC, 4, 256>(cases, work, nwork, grid, smem, st);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_gather_batch(int D, int vtile, int nth, const DevCase<T> *cases, const int4 *work, int nwork,
                                int grid, size_t smem, cudaStream_t st)
{
    if (D == 2) return gather_batch_dispatch<T, 2, 2>(vtile, nth, cases, work, nwork, grid, smem, st);
    return gather_batch_dispatch<T, 3, 1>(vtile, nth, cases, work, nwork, grid, smem, st);
}

// CTAs of the gather kernel that fit on the device at once (persistent grid)
template <typename T>
int gather_resident_ctas(int D, int vtile, int nth, size_t smem)
{
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int tv = vtile / 32;
    const void *fn = nullptr;
    if (nth == 512 && std::is_same<T, float>::value) {
        if (D == 2) fn = tv == 1 ? (const void *)k_gather_batch<T, 2, 2, 1, 512> : (const void *)k_gather_batch<T, 2, 2, 2, 512>;
        else fn = tv == 1 ? (const void *)k_gather_batch<T, 3, 1, 1, 512> : (const void *)k_gather_batch<T, 3, 1, 2, 512>;
    } else {
        if (D == 2)
            fn = tv == 1   ? (const void *)k_gather_batch<T, 2, 2, 1, 256>
                 : tv == 2 ? (const void *)k_gather_batch<T, 2, 2, 2, 256>
                           : (const void *)k_gather_batch<T, 2, 2, 4, 256>;
        else
            fn = tv == 1   ? (const void *)k_gather_batch<T, 3, 1, 1, 256>
                 : tv == 2 ? (const void *)k_gather_batch<T, 3, 1, 2, 256>
                           : (const void *)k_gather_batch<T, 3, 1, 4, 256>;
    }
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, nth, smem);
    return std::max(1, per) * std::max(1, nsm);
}

template <typename T>
cudaError_t launch_step(const DevCase<T> &dc, const StepConfig &cfg, cudaStream_t st, cudaEvent_t *ev)
{
    return dc.D == 2 ? step_dn<T, 2, 2>(dc, cfg, st, ev) : step_dn<T, 3, 1>(dc, cfg, st, ev);
}

template <typename T>
cudaError_t launch_init(const DevCase<T> &dc, cudaStream_t st)
{
    if (dc.D == 2) {
        k_init_f<T, 2, 2><<<cdiv(dc.C, 8), 256, 0, st>>>(dc);
        k_heatflux<T, 2, 2><<<cdiv(dc.C, 8), 256, 0, st>>>(dc);
    } else {
        k_init_f<T, 3, 1><<<cdiv(dc.C, 8), 256, 0, st>>>(dc);
        k_heatflux<T, 3, 1><<<cdiv(dc.C, 8), 256, 0, st>>>(dc);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_heatflux(const DevCase<T> &dc, cudaStream_t st)
{
    if (dc.D == 2) k_heatflux<T, 2, 2><<<cdiv(dc.C, 8), 256, 0, st>>>(dc);
    else k_heatflux<T, 3, 1><<<cdiv(dc.C, 8), 256, 0, st>>>(dc);
    return cudaGetLastError();
}

template <typename T, typename S>
cudaError_t launch_f_export(const DevCase<T> &dc, const long long *perm, int c0, int nc, S *out, cudaStream_t st)
{
    long long n = (long long)nc * (dc.D == 2 ? 2 : 1) * dc.nv;
    if (n == 0) return cudaSuccess;
    if (dc.D == 2) k_f_export<T, 2, 2, S><<<cdiv(n, 256), 256, 0, st>>>(dc, perm, c0, nc, out);
    else k_f_export<T, 3, 1, S><<<cdiv(n, 256), 256, 0, st>>>(dc, perm, c0, nc, out);
    return cudaGetLastError();
}

template <typename T, typename S>
cudaError_t launch_f_import(const DevCase<T> &dc, const long long *perm, int c0, int nc, const S *in,
                            cudaStream_t st)
{
    long long n = (long long)nc * (dc.D == 2 ? 2 : 1) * dc.nvp;
    if (n == 0) return cudaSuccess;
    if (dc.D == 2) k_f_import<T, 2, 2, S><<<cdiv(n, 256), 256, 0, st>>>(dc, perm, c0, nc, in);
    else k_f_import<T, 3, 1, S><<<cdiv(n, 256), 256, 0, st>>>(dc, perm, c0, nc, in);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_halo(const DevCase<T> &dc, const int *cells, int n, size_t row, void *buf, int unpack,
                        cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    if (dc.D == 2) {
        if (unpack) k_halo_unpack<T, 2, 2><<<n, 128, 0, st>>>(dc, cells, n, row, (const unsigned char *)buf);
        else k_halo_pack<T, 2, 2><<<n, 128, 0, st>>>(dc, cells, n, row, (unsigned char *)buf);
    } else {
        if (unpack) k_halo_unpack<T, 3, 1><<<n, 128, 0, st>>>(dc, cells, n, row, (const unsigned char *)buf);
        else k_halo_pack<T, 3, 1><<<n, 128, 0, st>>>(dc, cells, n, row, (unsigned char *)buf);
    }
    return cudaGetLastError();
}
template cudaError_t launch_halo<double>(const DevCase<double> &, const int *, int, size_t, void *, int,
                                         cudaStream_t);
template cudaError_t launch_halo<float>(const DevCase<float> &, const int *, int, size_t, void *, int,
                                        cudaStream_t);

cudaError_t launch_residual(const double *res_part, int nblocks, int D, double *res, cudaStream_t st)
{
    if (D == 2) k_residual<4><<<1, 32, 0, st>>>(res_part, nblocks, res);
    else k_residual<5><<<1, 32, 0, st>>>(res_part, nblocks, res);
    return cudaGetLastError();
}

cudaError_t launch_moments_out(const double *W, const double *q, const long long *perm, int C, int D,
                               double *out, cudaStream_t st)
{
    if (C == 0) return cudaSuccess;
    if (D == 2) k_moments_out<2><<<cdiv(C, 128), 128, 0, st>>>(W, q, perm, C, out);
    else k_moments_out<3><<<cdiv(C, 128), 128, 0, st>>>(W, q, perm, C, out);
    return cudaGetLastError();
}

cudaError_t launch_W_permute(const double *src, const long long *perm, int C, int D, double *dst,
                             int to_internal, cudaStream_t st)
{
    if (C == 0) return cudaSuccess;
    if (D == 2) k_W_permute<2><<<cdiv(C, 128), 128, 0, st>>>(src, perm, C, dst, to_internal);
    else k_W_permute<3><<<cdiv(C, 128), 128, 0, st>>>(src, perm, C, dst, to_internal);
    return cudaGetLastError();
}

cudaError_t launch_check(const double *W, int C, int M, int *flags, cudaStream_t st)
{
    if (C == 0) return cudaSuccess;
    k_check<<<cdiv(C, 128), 128, 0, st>>>(W, C, M, flags);
    return cudaGetLastError();
}

cudaError_t launch_density_range(const double *W, int C, int M, const unsigned char *owned,
                                 unsigned long long *range, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(&range[0], 0xff, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&range[1], 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || C == 0) return e;
    k_density_range<<<std::min(cdiv(C, 256), 1024), 256, 0, st>>>(W, C, M, owned, range);
    return cudaGetLastError();
}

template cudaError_t launch_pre_gather<double>(const DevCase<double> &, cudaStream_t);
template cudaError_t launch_pre_gather<float>(const DevCase<float> &, cudaStream_t);
template cudaError_t launch_post_gather<double>(const DevCase<double> &, const StepConfig &, cudaStream_t);
template cudaError_t launch_post_gather<float>(const DevCase<float> &, const StepConfig &, cudaStream_t);
template int small_kernel_blocks<double>(const DevCase<double> &, int);
template int small_kernel_blocks<float>(const DevCase<float> &, int);
template size_t small_kernel_smem<double>(const DevCase<double> &, int);
template size_t small_kernel_smem<float>(const DevCase<float> &, int);
template cudaError_t launch_small_batch<double>(int, int, const DevCase<double> *, const int *, int, int, size_t,
                                                cudaStream_t);
template cudaError_t launch_small_batch<float>(int, int, const DevCase<float> *, const int *, int, int, size_t,
                                               cudaStream_t);
template cudaError_t launch_gather<double>(const DevCase<double> &, size_t, cudaStream_t);
template cudaError_t launch_gather<float>(const DevCase<float> &, size_t, cudaStream_t);
template cudaError_t launch_gather_batch<double>(int, int, int, const DevCase<double> *, const int4 *, int, int, size_t,
                                                 cudaStream_t);
template cudaError_t launch_gather_batch<float>(int, int, int, const DevCase<float> *, const int4 *, int, int, size_t,
                                                cudaStream_t);
template int gather_resident_ctas<double>(int, int, int, size_t);
template int gather_resident_ctas<float>(int, int, int, size_t);
template cudaError_t launch_step<double>(const DevCase<double> &, const StepConfig &, cudaStream_t, cudaEvent_t *);
template cudaError_t launch_step<float>(const DevCase<float> &, const StepConfig &, cudaStream_t, cudaEvent_t *);
template cudaError_t launch_init<double>(const DevCase<double> &, cudaStream_t);
template cudaError_t launch_init<float>(const DevCase<float> &, cudaStream_t);
template cudaError_t launch_heatflux<double>(const DevCase<double> &, cudaStream_t);
template cudaError_t launch_heatflux<float>(const DevCase<float> &, cudaStream_t);
#define UGKS_STATE_IO(T, S)                                                                                   \
    template cudaError_t launch_f_export<T, S>(const DevCase<T> &, const long long *, int, int, S *, cudaStream_t); \
    template cudaError_t launch_f_import<T, S>(const DevCase<T> &, const long long *, int, int, const S *,          \
                                               cudaStream_t);
UGKS_STATE_IO(double, double)
UGKS_STATE_IO(double, float)
UGKS_STATE_IO(float, double)
UGKS_STATE_IO(float, float)
#undef UGKS_STATE_IO

}  // namespace ugks

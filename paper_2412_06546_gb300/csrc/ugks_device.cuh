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
// (CR_C = dt / (2 tau) and CR_INV = 1 / (1 + dt / (2 tau)), both formed in FP64)
enum { CR_U = 0, CR_LAM = 3, CR_PREF = 4, CR_KQ = 5, CR_C = 8, CR_NB = 9, CR_NL2 = 10, CR_INV = 11, CREC = 12 };
// ghost / side / wall record: a Maxwellian
enum { GR_U = 0, GR_LAM = 3, GR_PREF = 4, GR_NB = 5, GR_NL2 = 6, GREC = 8 };
// face record: g0 of the interface, Shakhov factor, time integrals, slopes in
// the basis centred at U0: psi_c = (1, c, (|c|^2 + xi^2)/2), c = u - U0
enum { FR_U = 0, FR_LAM = 3, FR_PREF = 4, FR_KQ = 5, FR_QS = 8, FR_NB = 13, FR_XB = 14,
       FR_BETA = 15, FR_NL2 = 39, FREC = 40 };

// flux record read by the gather pass: the equilibrium part of the
// time-integrated interface distribution, q3 (g0 + g0+) + q4 u.grad g0 +
// q5 dg0/dt, is H0(c) P_m(c) with c = u - U0 and, per stored component m,
// P_m(c) = a0 + a.c + sum_{e<=f} B_ef c_e c_f + (gamma.c)|c|^2
enum { XR_U = 0, XR_PREF = 3, XR_NL2 = 4, XR_LAM = 5, XR_Q1 = 6, XR_Q2 = 7, XR_POLY = 8, XREC = 24 };
template <int D> struct Poly {
    static constexpr int NB = D * (D + 1) / 2;
    static constexpr int N = 1 + D + NB + D;   // a0, a, B (packed upper, off-diagonal doubled), gamma
};

enum { FT_INTERIOR = 0, FT_WALL = 1, FT_FARFIELD = 2, FT_PERIODIC = 3 };

// nodes of the last velocity axis the separable half-range sums hold in shared memory
constexpr int SUM1_SEP_MAX_NL = 512;

// layout of the values of one gather entry (cell c, face f): a = LSQ
// coefficient of the neighbour across f (0 for a wall), rs = x_f - x_c,
// n = unit normal of f pointing out of c, ro = x_f - x_other (periodic image;
// 0 for far-field ghosts), cs = -S_f / |Omega_c|.  Grouped in 16-byte vectors
// so that each pass loads only the vectors it reads: the slopes' first face
// loop the first SLOPE1 values (a, rs), their limiter loop the first vector
// (rs), the flux loop everything but the vectors in [SKIP0, SKIP1) (a, in 3D).
template <int D> struct GEnt;
template <> struct GEnt<2> {
    static constexpr int A = 0, RS = 2, N = 4, RO = 6, CS = 8, LEN = 12;
    static constexpr int SLOPE1 = 4, LIMIT = 4, SKIP0 = 0, SKIP1 = 0;
};
template <> struct GEnt<3> {
    static constexpr int RS = 0, CS = 3, A = 4, N = 8, RO = 12, LEN = 16;
    static constexpr int SLOPE1 = 8, LIMIT = 4, SKIP0 = 4, SKIP1 = 8;
};

// Everything a kernel needs, by value.  Geometry used inside velocity loops is
// held in the arithmetic type T; macroscopic data is FP64.
template <typename T>
struct DevCase {
    int D, NC;
    int C, F, G, NW;         // cells, faces, far-field ghosts, wall faces
    int nv, nvp;             // velocities, padded count
    double dt, Pr, omega, mu_ref, nxi;
    int limiter;
    int w0_analytic;              // 1: W0 from the analytic half-range moments
    // velocity grid (padded), FP64 and T copies
    const double *ud[3], *wd;
    const T *u[3], *w;
    const T *uw;                  // [nvp][4] (u_x, u_y, u_z or 0, w) packed for one vector load
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
    // gather entries, one per (cell, face) in cf order, in the cell's own
    // orientation: gi = {other, face, type, patch slot of other}, where other
    // is the neighbour cell (interior, periodic), the ghost slot (far field) or
    // the wall slot (wall); gf = GEnt<D> values (LSQ coefficient, offsets,
    // outward normal, -S_f/|Omega_c|)
    const int4 *gi;
    const T *gf;
    const double *eps2_d;
    const T *eps2;
    // faces
    const int *fL, *fR, *faux;    // owner, neighbour (-1 at boundaries), ghost or wall slot
    const signed char *ftype;
    const double *fn_d, *frL_d, *frR_d;
    const T *fn, *frL, *frR;      // T copies used inside velocity loops
    T dtT;                        // dt in the arithmetic type
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
    double *wall_F;               // [NW][D+2] macroscopic wall flux over the last step (Eq. macroscopicFlux)
    T *wrec;                      // [NW][GREC]
    // per-step work
    T *crec;                      // [C][CREC] stage-1 record (W^n, q^n)
    T *krec;                      // [C][CREC] stage-2 record (W^{n+1}, q^n)
    T *frec;                      // [F][FREC] face-pass work record
    T *xrec;                      // [F][XREC] flux record of the gather pass
    T *fside;                     // [F][2][GREC] Maxwellians of the face states
    double *fdW0;                 // [F][D][D+2] interface macro gradient
    double *fq0;                  // [F][D]
    double *fUref;                // [F][D]
    double *fsum1, *fsum2;        // [F][S1], [F][S2]
    double *fprim0;               // [F][D+2] rho0, U0, lam0
    double *fqs;                  // [F][5] time integrals q1..q5 of the interface
    double *dW_part;              // [C][n_groups][D+2] moments of the flux residual over a tile group
    double *res_part;             // [n_res_blocks][2(D+2)]
    const unsigned char *owned;   // [C] 1 for cells whose residual counts (a subdomain's own cells),
                                  // nullptr: every cell
    int *flags;                   // [1] numeric failure flag
    // tensor-product velocity grid (sep = 1): axes and 1-D weights per dimension
    int sep, cart_n[3];
    int sep1;                     // sep with the last axis strictly ascending and at most
                                  // SUM1_SEP_MAX_NL nodes (separable half-range sums)
    const T *axis[3], *axw[3];
    // gather tiling
    int P, n_patches, n_vt, vtile;
    int nth;                      // threads per gather CTA (256, or 512 for FP32 at TV <= 2)
    int vt_group;                 // velocity tiles per gather CTA (see k_gather)
    int n_groups;                 // tile groups: ceil(n_vt / vt_group)
    const int *ring_ptr, *ring_cells;
};

// ------------------------------------------------------------------ math
template <typename T> __device__ __forceinline__ T dexp(T x);
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }

// 2^x with the hardware approximation (relative error ~2^-22); FP32 only
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// exp(-lambda c2) of a record: FP64 through exp(), FP32 through 2^(nl2 c2)
// with nl2 = -lambda log2(e) precomputed in the record
template <typename T> __device__ __forceinline__ T gauss(T lam, T nl2, T c2);
template <> __device__ __forceinline__ double gauss<double>(double lam, double, double c2) { return exp(-lam * c2); }
template <> __device__ __forceinline__ float gauss<float>(float, float nl2, float c2) { return ex2_approx(nl2 * c2); }

// a / b: IEEE in FP64, the fast reciprocal-based quotient in FP32
template <typename T> __device__ __forceinline__ T fdiv(T a, T b);
template <> __device__ __forceinline__ double fdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }

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

// ------------------------------------------------------------ moment sums
// Velocity-moment sums of the FP32 form are compensated: a lane accumulates
// its FP32 terms with Kahan's correction (the running sum s and the rounding
// error c lost so far; the sum is s - c, returned in FP64), and the lanes'
// sums are combined in FP64.  The FP64 form sums plainly in FP64.  The
// corrections rely on IEEE rounding of every addition: nothing here may be
// reassociated or contracted (no fast-math flags).
template <typename T> struct CSum;
template <> struct CSum<double> {
    double s;
    __device__ __forceinline__ CSum() : s(0.0) {}
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct CSum<float> {
    float s, c;
    __device__ __forceinline__ CSum() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float x)
    {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Blocked accumulation in FP64 for sums with many terms per lane and many
// values (the face sums): every lane adds at most SUM_BLOCK of its FP32 terms
// per value into blk[] (a block of 32 x SUM_BLOCK terms per warp), the warp
// combines each block value across lanes (warp_transpose_sum, FP32), and the
// block totals are accumulated in FP64, lane j holding value j >> (5 - log2 N).
// The FP32 part of every sum spans one block, so its rounding error is bounded
// by about (SUM_BLOCK + 5) units in the last place of the block's absolute sum
// whatever the number of terms.
constexpr int SUM_BLOCK = 16;

// Error-free sum of two FP32 values (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// Double-float addition (hi, lo) += (bh, bl): about 44 significant bits, with
// FP32 instructions only (FP64 arithmetic is scarce on this part).
__device__ __forceinline__ void ff_add(float &hi, float &lo, float bh, float bl)
{
    float s, e;
    two_sum(hi, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// warp_transpose_sum on double-float pairs (h, l): the same exchange pattern,
// with every addition a double-float addition.  On return (oh, ol) is the
// full sum of value index lane >> (5 - log2 N).
template <int N>
__device__ __forceinline__ void warp_transpose_sum_ff2(float (&h)[N], float (&l)[N], float &oh, float &ol)
{
    const int lane = threadIdx.x & 31;
    int n = N;
#pragma unroll
    for (int bit = 16; n > 1; bit >>= 1) {
        n >>= 1;
        const bool upper = (lane & bit) != 0;
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            if (i >= n) break;
            const float sh = upper ? h[i] : h[i + n], sl = upper ? l[i] : l[i + n];
            const float kh = upper ? h[i + n] : h[i], kl = upper ? l[i + n] : l[i];
            const float rh = __shfl_xor_sync(0xffffffffu, sh, bit), rl = __shfl_xor_sync(0xffffffffu, sl, bit);
            h[i] = kh;
            l[i] = kl;
            ff_add(h[i], l[i], rh, rl);
        }
    }
    constexpr int used = (N == 32) ? 5 : (N == 16) ? 4 : (N == 8) ? 3 : (N == 4 ? 2 : (N == 2 ? 1 : 0));
    float rh = h[0], rl = l[0];
#pragma unroll
    for (int bit = 16 >> used; bit > 0; bit >>= 1) {
        const float qh = __shfl_xor_sync(0xffffffffu, rh, bit), ql = __shfl_xor_sync(0xffffffffu, rl, bit);
        ff_add(rh, rl, qh, ql);
    }
    oh = rh;
    ol = rl;
}

// Sum of N (a power of two up to 32) values over the 32 lanes of a warp by
// recursive halving: at every exchange a lane keeps half of its values and
// receives the partner's partial sums of that half.  On return lane l holds
// the full sum of value index l >> (5 - log2 N) (lanes 8j..8j+7 for N = 4,
// lane j for N = 32).
template <typename T, int N>
__device__ __forceinline__ T warp_transpose_sum(T (&v)[N])
{
    const int lane = threadIdx.x & 31;
    int n = N;
#pragma unroll
    for (int bit = 16; n > 1; bit >>= 1) {
        n >>= 1;
        const bool upper = (lane & bit) != 0;
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            if (i >= n) break;
            const T send = upper ? v[i] : v[i + n];
            const T keep = upper ? v[i + n] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
    }
    constexpr int used = (N == 32) ? 5 : (N == 16) ? 4 : (N == 8) ? 3 : (N == 4 ? 2 : (N == 2 ? 1 : 0));
    static_assert((1 << used) == N, "N must be a power of two up to 32");
    T r = v[0];
#pragma unroll
    for (int bit = 16 >> used; bit > 0; bit >>= 1) r += __shfl_xor_sync(0xffffffffu, r, bit);
    return r;
}

// the block step of the blocked FP64 accumulation (see SUM_BLOCK)
template <int N>
__device__ __forceinline__ double block_to_fp64(float (&blk)[N])
{
    return (double)warp_transpose_sum<float, N>(blk);
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
    return rec[GR_PREF] * gauss<T>(rec[GR_LAM], rec[GR_NL2], c2);
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
    T H = rec[CR_PREF] * gauss<T>(rec[CR_LAM], rec[CR_NL2], c2);
    T l2c2 = T(2) * rec[CR_LAM] * c2;
    fp[0] = H * (T(1) + kqc * (l2c2 - T(D + 2)));
    if (NC == 2) fp[NC - 1] = H * rec[CR_NB] * (T(1) + kqc * (l2c2 - T(D)));
}

// TV consecutive values at a TV*sizeof(T)-aligned address, moved in chunks
// of at most 16 bytes (read-only data through the non-coherent path)
template <typename T, int N> struct VecOf;
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<float, 4> { using type = float4; };
template <> struct VecOf<double, 1> { using type = double; };
template <> struct VecOf<double, 2> { using type = double2; };
template <typename T, int TV> constexpr int vec_chunk() { return TV * (int)sizeof(T) <= 16 ? TV : 16 / (int)sizeof(T); }

template <typename T, int TV>
__device__ __forceinline__ void ldv(const T *__restrict__ p, T (&x)[TV])
{
    constexpr int CH = vec_chunk<T, TV>();
    using V = typename VecOf<T, CH>::type;
#pragma unroll
    for (int i = 0; i < TV / CH; ++i) {
        const V v = __ldg(reinterpret_cast<const V *>(p) + i);
        const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
        for (int j = 0; j < CH; ++j) x[i * CH + j] = e[j];
    }
}
// the same from and to shared memory
template <typename T, int TV>
__device__ __forceinline__ void ldv_s(const T *p, T (&x)[TV])
{
    constexpr int CH = vec_chunk<T, TV>();
    using V = typename VecOf<T, CH>::type;
#pragma unroll
    for (int i = 0; i < TV / CH; ++i) {
        const V v = reinterpret_cast<const V *>(p)[i];
        const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
        for (int j = 0; j < CH; ++j) x[i * CH + j] = e[j];
    }
}
template <typename T, int TV>
__device__ __forceinline__ void stv(T *p, const T (&x)[TV])
{
    constexpr int CH = vec_chunk<T, TV>();
    using V = typename VecOf<T, CH>::type;
#pragma unroll
    for (int i = 0; i < TV / CH; ++i) {
        V v;
        T *e = reinterpret_cast<T *>(&v);
#pragma unroll
        for (int j = 0; j < CH; ++j) e[j] = x[i * CH + j];
        reinterpret_cast<V *>(p)[i] = v;
    }
}

// copy a 16-byte aligned record of N values into registers with vector loads
template <int N>
__device__ __forceinline__ void load_rec(const float *__restrict__ p, float (&r)[N])
{
    static_assert(N % 4 == 0, "record length");
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + i);
        r[4 * i] = v.x;
        r[4 * i + 1] = v.y;
        r[4 * i + 2] = v.z;
        r[4 * i + 3] = v.w;
    }
}
template <int N>
__device__ __forceinline__ void load_rec(const double *__restrict__ p, double (&r)[N])
{
    static_assert(N % 2 == 0, "record length");
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + i);
        r[2 * i] = v.x;
        r[2 * i + 1] = v.y;
    }
}

// velocity k and its weight from the packed array, one 16-byte (FP32) or two
// 16-byte (FP64) loads
__device__ __forceinline__ void load_uw(const float *__restrict__ uw, int k, float u[3], float &w)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(uw) + k);
    u[0] = v.x;
    u[1] = v.y;
    u[2] = v.z;
    w = v.w;
}
__device__ __forceinline__ void load_uw(const double *__restrict__ uw, int k, double u[3], double &w)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(uw) + 2 * k);
    const double2 b = __ldg(reinterpret_cast<const double2 *>(uw) + 2 * k + 1);
    u[0] = a.x;
    u[1] = a.y;
    u[2] = b.x;
    w = b.y;
}

// Micro reconstruction of cell c (Sec. 3.1 Step 2) for the TV consecutive
// velocities of this lane: least-squares slope grad = sum_j a_cj (f_j - f_c),
// Venkatakrishnan factor phi = min over the faces of c of (D1^2 + eps^2 +
// 2 D1 D2) / (D1^2 + 2 D2^2 + D1 D2 + eps^2), then a positivity scaling theta
// so that the reconstruction is non-negative at every face centre and at the
// foot of the characteristic after one step: with dmin = min(0, min_f D2_f),
// v = f_c + phi (dmin + min(0, -dt u.grad)); theta = f_c / (f_c - v) if v < 0.
// Every face entry is read once for all TV velocities.  fl points at f_cur +
// the lane's first velocity; fi returns f_c.  The face loops are unrolled so
// that the entry and neighbour loads of several faces are in flight together
// (the pass is bound by their latency).
template <typename T, int D, int NC, int TV>
__device__ __forceinline__ void cell_slope_tv(const DevCase<T> &dc, const T *__restrict__ fl, int c,
                                              const T (&u)[3][TV], T (&g)[NC][D][TV], T (&fi)[NC][TV])
{
    using E = GEnt<D>;
    constexpr int HA = E::SLOPE1;                 // a and rs, in whole vector loads
    const int nvp = dc.nvp;
    const size_t rs = (size_t)NC * nvp;
    T vmax[NC][TV], vmin[NC][TV];
    const T *fc = fl + (size_t)c * rs;
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        ldv<T, TV>(fc + (size_t)m * nvp, fi[m]);
#pragma unroll
        for (int j = 0; j < TV; ++j) {
            vmax[m][j] = vmin[m][j] = fi[m][j];
#pragma unroll
            for (int d = 0; d < D; ++d) g[m][d][j] = 0;
        }
    }
    const int e0 = __ldg(dc.cf_ptr + c), e1 = __ldg(dc.cf_ptr + c + 1);
#pragma unroll 4
    for (int e = e0; e < e1; ++e) {
        const int4 gi = __ldg(dc.gi + e);
        if (gi.z == FT_WALL) continue;
        T ge[HA];
        load_rec<HA>(dc.gf + (size_t)e * E::LEN, ge);
        T fj[NC][TV];
        if (gi.z == FT_FARFIELD) {
            T gr[GREC];
            load_rec<GREC>(dc.grec + (size_t)gi.x * GREC, gr);
#pragma unroll
            for (int j = 0; j < TV; ++j) {
                const T uj[3] = {u[0][j], u[1][j], u[2][j]};
                const T H = maxwell_h<T, D>(gr, uj);
                fj[0][j] = H;
                if (NC == 2) fj[NC - 1][j] = gr[GR_NB] * H;
            }
        } else {
            const T *fo = fl + (size_t)gi.x * rs;
#pragma unroll
            for (int m = 0; m < NC; ++m) ldv<T, TV>(fo + (size_t)m * nvp, fj[m]);
        }
#pragma unroll
        for (int m = 0; m < NC; ++m)
#pragma unroll
            for (int j = 0; j < TV; ++j) {
                const T df = fj[m][j] - fi[m][j];
#pragma unroll
                for (int d = 0; d < D; ++d) g[m][d][j] += ge[E::A + d] * df;
                vmax[m][j] = fj[m][j] > vmax[m][j] ? fj[m][j] : vmax[m][j];
                vmin[m][j] = fj[m][j] < vmin[m][j] ? fj[m][j] : vmin[m][j];
            }
    }
    const T e2 = __ldg(dc.eps2 + c);
    // Venkatakrishnan's factor at a face, phi(d2) = (a2 + 2 d1 d2) / (a2 + d2 (2 d2 + d1))
    // with a2 = d1^2 + eps^2 and d1 of the sign of d2, is at least 1 for
    // 0 <= d2/d1 <= 1/2 and strictly decreasing in |d2| beyond.  Its minimum over
    // the faces (clipped at 1) is therefore taken at the largest and at the most
    // negative d2, so the face loop only tracks those two, and phi is evaluated
    // twice per velocity instead of once per face.
    T dmax[NC][TV], dmin[NC][TV];
#pragma unroll
    for (int m = 0; m < NC; ++m)
#pragma unroll
        for (int j = 0; j < TV; ++j) dmax[m][j] = dmin[m][j] = T(0);
#pragma unroll 4
    for (int e = e0; e < e1; ++e) {
        T ge[E::LIMIT];
        load_rec<E::LIMIT>(dc.gf + (size_t)e * E::LEN, ge);
#pragma unroll
        for (int m = 0; m < NC; ++m)
#pragma unroll
            for (int j = 0; j < TV; ++j) {
                T d2 = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) d2 += g[m][d][j] * ge[E::RS + d];
                dmin[m][j] = d2 < dmin[m][j] ? d2 : dmin[m][j];
                dmax[m][j] = d2 > dmax[m][j] ? d2 : dmax[m][j];
            }
    }
    T phi[NC][TV];
#pragma unroll
    for (int m = 0; m < NC; ++m)
#pragma unroll
        for (int j = 0; j < TV; ++j) {
            phi[m][j] = T(1);
            if (dc.limiter) {
                auto venk = [&](T d1, T d2) {
                    const T a2 = d1 * d1 + e2;
                    const T num = a2 + T(2) * d1 * d2;
                    const T den = a2 + d2 * (T(2) * d2 + d1);
                    return den > T(0) ? fdiv(num, den) : T(1);
                };
                if (dmax[m][j] > T(0)) {
                    const T ph = venk(vmax[m][j] - fi[m][j], dmax[m][j]);
                    phi[m][j] = ph < phi[m][j] ? ph : phi[m][j];
                }
                if (dmin[m][j] < T(0)) {
                    const T ph = venk(vmin[m][j] - fi[m][j], dmin[m][j]);
                    phi[m][j] = ph < phi[m][j] ? ph : phi[m][j];
                }
            }
        }
    const T dt = dc.dtT;
#pragma unroll
    for (int m = 0; m < NC; ++m)
#pragma unroll
        for (int j = 0; j < TV; ++j) {
            T ug = 0;
#pragma unroll
            for (int d = 0; d < D; ++d) ug += u[d][j] * g[m][d][j];
            const T foot = -dt * ug;
            const T v = fi[m][j] + phi[m][j] * (dmin[m][j] + (foot < T(0) ? foot : T(0)));
            T sc = phi[m][j];
            if (v < T(0)) sc *= fi[m][j] > T(0) ? fdiv(fi[m][j], fi[m][j] - v) : T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) g[m][d][j] *= sc;
        }
}

// Interface flux of Eq. microscopicFlux with the distribution of Eq.
// fullSolution integrated over the step (q1..q5):
// F = u_n [q1 f_up + q2 u.grad f_up + H0(c) P(c)], the equilibrium part
// q3 (g0 + g0+) + q4 u.grad g0 + q5 dg0/dt expanded into P (see XR_POLY).
template <typename T, int D>
__device__ __forceinline__ T poly_eval(const T *__restrict__ a, const T c[D], T c2)
{
    constexpr int NB = Poly<D>::NB;
    T p = a[0];
#pragma unroll
    for (int e = 0; e < D; ++e) p += a[1 + e] * c[e];
    int t = 1 + D;
    T q = 0;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        T r = 0;
#pragma unroll
        for (int f = e; f < D; ++f) r += a[t + (e * (2 * D - e + 1)) / 2 + (f - e)] * c[f];
        q += r * c[e];
    }
    p += q;
    T g = 0;
#pragma unroll
    for (int e = 0; e < D; ++e) g += a[t + NB + e] * c[e];
    return p + g * c2;
}

template <typename T, int D, int NC>
__device__ __forceinline__ void interface_flux(const T *__restrict__ xr, const T u[3], T un,
                                               const T fup[NC], const T ugf[NC], T F[NC])
{
    T c[D], c2 = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        c[d] = u[d] - xr[XR_U + d];
        c2 += c[d] * c[d];
    }
    const T H0 = xr[XR_PREF] * gauss<T>(xr[XR_LAM], xr[XR_NL2], c2);
    const T q1 = xr[XR_Q1], q2 = xr[XR_Q2];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const T P = poly_eval<T, D>(xr + XR_POLY + m * Poly<D>::N, c, c2);
        F[m] = un * (q1 * fup[m] + q2 * ugf[m] + H0 * P);
    }
}

}  // namespace ugks

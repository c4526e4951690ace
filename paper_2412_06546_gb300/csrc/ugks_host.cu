// ugks_host.cu -- C ABI of the UGKS library: validation, host preprocessing
// (cell ordering, least-squares coefficients, gather patches), device state and
// the launch sequence of a time step.  The numerics live in ugks_kernels.cu.
#include "../../include/ugks.h"
#include "ugks_device.cuh"
#include "ugks_kernels.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

namespace {

thread_local std::string g_err;

struct Fail {
    ugks_status code;
    std::string msg;
};

[[noreturn]] void fail(ugks_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw Fail{code, buf};
}

void cuda_ok(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) fail(UGKS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

struct ugks_case {
    int D = 0, NC = 0, prec = UGKS_FP64;
    int64_t C = 0, F = 0, Nv = 0, nvp = 0;
    int G = 0, NW = 0;
    double dt = 0.0;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    ugks_alloc alloc{};
    bool user_alloc = false;
    std::vector<std::pair<void *, size_t>> blocks;
    size_t device_bytes = 0, f_bytes = 0;
    size_t stage_bytes = 0;        // bytes of f_nxt, the staging area of state I/O (>= f_bytes)
    ugks::DevCase<double> d64{};
    ugks::DevCase<float> d32{};
    ugks::StepConfig cfg{};
    int P = 0, vtile = 0, nth = 256, n_patches = 0, n_vt = 0, vt_group = 1, n_groups = 1;
    long long *perm_d = nullptr;   // caller cell i -> internal cell
    std::vector<long long> perm_h; // the same on the host
    std::vector<long long> wall_face_h;   // face id of every wall slot
    std::vector<double> wall_n_h;         // [NW][D] its normal
    double *res_d = nullptr;       // [M]
    int *flags_d = nullptr;
    unsigned long long *range_d = nullptr;   // [2] bit patterns of the min and max density
    int n_res_blocks = 0;
    bool stepped = false;
    // kernel-group profiling
    std::vector<cudaEvent_t> prof_ev;
    int prof_max = 0, prof_used = 0;
    // host -> device copies of ugks_set_state (created on first use): the copy
    // stream and its events (ready, copied[2], consumed[2])
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t io_ev[5] = {};
    // domain decomposition: owned-cell mask (internal order) and the halo
    // lists registered by ugks_halo_set (internal cell ids on the device)
    unsigned char *owned_d = nullptr;
    struct HaloList {
        int *ids = nullptr;
        int n = 0;
    };
    std::vector<HaloList> halo;

    void *dalloc(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~size_t(255);
        void *p = nullptr;
        if (user_alloc) {
            p = alloc.alloc(alloc.ctx, bytes, (void *)stream);
            if (!p) fail(UGKS_ENOMEM, "device allocation of %zu bytes failed", bytes);
            if ((uintptr_t)p & 255) {       // the vector loads and stores rely on it
                alloc.free(alloc.ctx, p, bytes, (void *)stream);
                fail(UGKS_EINVAL, "the allocator returned a pointer that is not 256-byte aligned");
            }
        } else {
            cudaError_t e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                fail(UGKS_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
            }
        }
        blocks.push_back({p, bytes});
        device_bytes += bytes;
        return p;
    }

    // frees one block of dalloc (the patch arrays of a tiling that is replaced)
    void dfree(const void *p)
    {
        if (!p) return;
        for (size_t i = 0; i < blocks.size(); ++i)
            if (blocks[i].first == p) {
                if (user_alloc) alloc.free(alloc.ctx, blocks[i].first, blocks[i].second, (void *)stream);
                else cudaFree(blocks[i].first);
                device_bytes -= blocks[i].second;
                blocks.erase(blocks.begin() + (long)i);
                return;
            }
    }

    template <typename V>
    V *upload(const std::vector<V> &h)
    {
        V *d = (V *)dalloc(h.size() * sizeof(V));
        if (!h.empty()) cuda_ok(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, stream),
                                "upload");
        return d;
    }

    void release()
    {
        if (stream) cudaStreamSynchronize(stream);
        else cudaDeviceSynchronize();
        if (copy_stream) {
            cudaStreamSynchronize(copy_stream);
            for (auto &e : io_ev) {
                if (e) cudaEventDestroy(e);
                e = nullptr;
            }
            cudaStreamDestroy(copy_stream);
            copy_stream = nullptr;
        }
        for (auto &b : blocks) {
            if (user_alloc) alloc.free(alloc.ctx, b.first, b.second, (void *)stream);
            else cudaFree(b.first);
        }
        blocks.clear();
    }
};

namespace {

// 2D / 3D Morton key of quantised centroids
uint64_t spread2(uint64_t x)
{
    x &= 0xffffffffULL;
    x = (x | (x << 16)) & 0x0000ffff0000ffffULL;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffULL;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0fULL;
    x = (x | (x << 2)) & 0x3333333333333333ULL;
    x = (x | (x << 1)) & 0x5555555555555555ULL;
    return x;
}

uint64_t spread3(uint64_t x)
{
    x &= 0x1fffffULL;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

struct Host {
    // internal-order geometry produced by preprocessing
    std::vector<int> perm_i2u, perm_u2i;
    std::vector<int> cf_ptr, cf_face;
    std::vector<signed char> cf_side;
    std::vector<double> cf_r, cf_coef;
    std::vector<double> gf;          // gather entry values [ncf][GEnt<D>::LEN]
    std::vector<int> gi;             // gather entry ids [ncf][4] (patch slots: build_patches)
    std::vector<int> nb_ptr, nb_id;
    std::vector<double> nb_a, eps2, vol;
    std::vector<int> fL, fR, faux, ftag, gface, wface;
    std::vector<signed char> ftype;
    std::vector<double> fn, frL, frR;
    std::vector<int> ring_ptr, ring_cells;
    int max_slope = 0;
};

// CFL time step of Algorithm 1 over the first n cells of the mesh:
// dt = cfl * min_i (2 |Omega_i| / sum_f S_f) / max_k |u_k|.  Each cell's face
// areas are summed in ascending face order, so a cell gives the same value in
// any mesh that holds all of its faces in the same relative order (a
// subdomain's own cells).
double cfl_dt_of(const ugks_mesh *m, const ugks_vgrid *v, double cfl, int64_t n)
{
    const int D = m->dim;
    std::vector<double> sumS((size_t)m->n_cells, 0.0);
    for (int64_t f = 0; f < m->n_faces; ++f) {
        sumS[(size_t)m->face_cells[2 * f]] += m->face_S[f];
        const int64_t b = m->face_cells[2 * f + 1];
        if (b >= 0) sumS[(size_t)b] += m->face_S[f];
    }
    double hmin = INFINITY;
    for (int64_t i = 0; i < n; ++i) hmin = std::min(hmin, 2.0 * m->cell_vol[i] / sumS[(size_t)i]);
    double umax = 0.0;
    for (int64_t k = 0; k < v->nv; ++k) {
        double s = 0.0;
        for (int d = 0; d < D; ++d) s += v->u[k * D + d] * v->u[k * D + d];
        umax = std::max(umax, std::sqrt(s));
    }
    return cfl * hmin / umax;
}

void validate(const ugks_mesh *m, const ugks_vgrid *v, const ugks_params *p)
{
    if (!m || !v || !p) fail(UGKS_EINVAL, "mesh, vgrid and params must not be NULL");
    if (m->dim != 2 && m->dim != 3) fail(UGKS_EINVAL, "mesh dim must be 2 or 3 (got %d)", m->dim);
    if (v->dim != m->dim) fail(UGKS_EINVAL, "velocity grid dim %d != mesh dim %d", v->dim, m->dim);
    if (m->n_cells <= 0 || m->n_faces < 0) fail(UGKS_EINVAL, "mesh needs n_cells > 0, n_faces >= 0");
    if (m->n_cells > (1LL << 30) || m->n_faces > (1LL << 30)) fail(UGKS_EINVAL, "mesh too large for 32-bit indexing");
    if (v->nv <= 0 || v->nv > (1 << 24)) fail(UGKS_EINVAL, "velocity count %lld out of range", (long long)v->nv);
    if (!m->cell_xc || !m->cell_vol || !m->face_cells || !m->face_n || !m->face_S || !m->face_xc ||
        !m->face_type || !m->face_tag)
        fail(UGKS_EINVAL, "mesh arrays must not be NULL");
    if (!v->u || !v->w) fail(UGKS_EINVAL, "velocity arrays must not be NULL");
    if (p->precision != UGKS_FP64 && p->precision != UGKS_FP32) fail(UGKS_EINVAL, "unknown precision %d", p->precision);
    if (!(p->Pr > 0.0) || !(p->omega >= 0.0) || !(p->L_ref > 0.0) || !(p->Kn > 0.0))
        fail(UGKS_EINVAL, "need Kn > 0, L_ref > 0, Pr > 0, omega >= 0");
    if (!(p->dt > 0.0) && !(p->cfl > 0.0)) fail(UGKS_EINVAL, "need cfl > 0 or dt > 0");
    if (p->limiter && !(p->venkat_K > 0.0)) fail(UGKS_EINVAL, "venkat_K must be > 0 with the limiter on");
    if (p->n_walls < 0 || (p->n_walls > 0 && (!p->wall_T || !p->wall_U))) fail(UGKS_EINVAL, "wall arrays missing");
    for (int i = 0; i < p->n_walls; ++i)
        if (!(p->wall_T[i] > 0.0)) fail(UGKS_EINVAL, "wall %d temperature must be > 0", i);
    const int D = m->dim;
    for (int64_t i = 0; i < m->n_cells; ++i)
        if (!(m->cell_vol[i] > 0.0)) fail(UGKS_EINVAL, "cell %lld has non-positive volume", (long long)i);
    bool farfield = false;
    for (int64_t f = 0; f < m->n_faces; ++f) {
        const int64_t a = m->face_cells[2 * f], b = m->face_cells[2 * f + 1];
        const int t = m->face_type[f];
        if (a < 0 || a >= m->n_cells) fail(UGKS_EINVAL, "face %lld: owner out of range", (long long)f);
        if (t == UGKS_FACE_INTERIOR || t == UGKS_FACE_PERIODIC) {
            if (b < 0 || b >= m->n_cells) fail(UGKS_EINVAL, "face %lld: neighbour out of range", (long long)f);
            if (t == UGKS_FACE_PERIODIC && !m->face_shift) fail(UGKS_EINVAL, "periodic faces need face_shift");
        } else if (t == UGKS_FACE_WALL || t == UGKS_FACE_FARFIELD) {
            if (b != -1) fail(UGKS_EINVAL, "face %lld: boundary face must have neighbour -1", (long long)f);
            if (t == UGKS_FACE_WALL && (m->face_tag[f] < 0 || m->face_tag[f] >= p->n_walls))
                fail(UGKS_EINVAL, "face %lld: wall tag %d out of range", (long long)f, m->face_tag[f]);
            if (t == UGKS_FACE_FARFIELD) farfield = true;
        } else {
            fail(UGKS_EINVAL, "face %lld: unknown type %d", (long long)f, t);
        }
        if (!(m->face_S[f] > 0.0)) fail(UGKS_EINVAL, "face %lld: area must be > 0", (long long)f);
        double nn = 0.0;
        for (int d = 0; d < D; ++d) nn += m->face_n[f * D + d] * m->face_n[f * D + d];
        if (std::fabs(nn - 1.0) > 1e-8) fail(UGKS_EINVAL, "face %lld: normal is not unit length", (long long)f);
    }
    if (farfield && (!(p->inf_rho > 0.0) || !(p->inf_T > 0.0)))
        fail(UGKS_EINVAL, "far-field faces need inf_rho > 0 and inf_T > 0");
    for (int64_t k = 0; k < v->nv; ++k)
        if (!(v->w[k] >= 0.0) || !std::isfinite(v->w[k])) fail(UGKS_EINVAL, "velocity weight %lld invalid", (long long)k);
    if (p->prim_init)
        for (int64_t i = 0; i < m->n_cells; ++i)
            if (!(p->prim_init[i * (D + 2)] > 0.0) || !(p->prim_init[i * (D + 2) + D + 1] > 0.0))
                fail(UGKS_EINVAL, "initial state of cell %lld needs rho > 0 and T > 0", (long long)i);
    if (p->vtile != 0 && p->vtile != 32 && p->vtile != 64 && p->vtile != 128)
        fail(UGKS_EINVAL, "vtile must be 0, 32, 64 or 128");
    if (p->patch_cells < 0 || p->patch_cells > 4096) fail(UGKS_EINVAL, "patch_cells out of range");
    if (p->w0_analytic != 0 && p->w0_analytic != 1) fail(UGKS_EINVAL, "w0_analytic must be 0 or 1");
    if (p->gather_threads != 0 && p->gather_threads != 256 && p->gather_threads != 512)
        fail(UGKS_EINVAL, "gather_threads must be 0, 256 or 512");
    if (p->gather_threads == 512 && (p->precision != UGKS_FP32 || p->vtile > 64))
        fail(UGKS_EINVAL, "gather_threads = 512 needs UGKS_FP32 and vtile <= 64");
    if (p->gather_tile_group < 0 || p->gather_tile_group > 1024)
        fail(UGKS_EINVAL, "gather_tile_group must be in [0, 1024]");
}

// invert the DxD normal matrix by its adjugate
bool invert_small(int D, const double *A, double *Ainv)
{
    double tr = 0.0;
    for (int a = 0; a < D; ++a) tr += A[a * D + a];
    double det;
    if (D == 2) {
        det = A[0] * A[3] - A[1] * A[2];
        if (!(std::fabs(det) > 1e-12 * std::pow(tr / D, D))) return false;
        Ainv[0] = A[3] / det;
        Ainv[1] = -A[1] / det;
        Ainv[2] = -A[2] / det;
        Ainv[3] = A[0] / det;
        return true;
    }
    const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(std::fabs(det) > 1e-12 * std::pow(tr / D, D))) return false;
    Ainv[0] = c00 / det;
    Ainv[3] = c01 / det;
    Ainv[6] = c02 / det;
    Ainv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    Ainv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    Ainv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    Ainv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    Ainv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    Ainv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    return true;
}

void build_patches(Host &h, int C, int P);

void preprocess(const ugks_mesh *m, const ugks_params *p, int P, Host &h)
{
    const int D = m->dim;
    const int C = (int)m->n_cells, F = (int)m->n_faces;
    // ---- cell order: Morton order of the centroids (spatially compact patches)
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < C; ++i)
        for (int d = 0; d < D; ++d) {
            lo[d] = std::min(lo[d], m->cell_xc[(size_t)i * D + d]);
            hi[d] = std::max(hi[d], m->cell_xc[(size_t)i * D + d]);
        }
    std::vector<uint64_t> key(C);
    const double bits = D == 2 ? 4294967295.0 : 2097151.0;
    for (int i = 0; i < C; ++i) {
        uint64_t k = 0;
        for (int d = 0; d < D; ++d) {
            double span = hi[d] - lo[d];
            double t = span > 0 ? (m->cell_xc[(size_t)i * D + d] - lo[d]) / span : 0.0;
            uint64_t qv = (uint64_t)std::llround(t * bits);
            k |= (D == 2 ? spread2(qv) : spread3(qv)) << d;
        }
        key[i] = k;
    }
    h.perm_i2u.resize(C);
    std::iota(h.perm_i2u.begin(), h.perm_i2u.end(), 0);
    std::stable_sort(h.perm_i2u.begin(), h.perm_i2u.end(), [&](int a, int b) { return key[a] < key[b]; });
    h.perm_u2i.resize(C);
    for (int i = 0; i < C; ++i) h.perm_u2i[h.perm_i2u[i]] = i;
    auto X = [&](int ci, int d) { return m->cell_xc[(size_t)h.perm_i2u[ci] * D + d]; };
    h.vol.resize(C);
    for (int i = 0; i < C; ++i) h.vol[i] = m->cell_vol[h.perm_i2u[i]];

    // ---- faces
    h.fL.assign(F, -1);
    h.fR.assign(F, -1);
    h.faux.assign(F, -1);
    h.ftag.assign(F, 0);
    h.ftype.assign(F, 0);
    h.fn.assign((size_t)F * D, 0.0);
    h.frL.assign((size_t)F * D, 0.0);
    h.frR.assign((size_t)F * D, 0.0);
    for (int f = 0; f < F; ++f) {
        const int t = m->face_type[f];
        h.ftype[f] = (signed char)t;
        h.ftag[f] = m->face_tag[f];
        h.fL[f] = h.perm_u2i[m->face_cells[2 * f]];
        if (t == UGKS_FACE_INTERIOR || t == UGKS_FACE_PERIODIC) h.fR[f] = h.perm_u2i[m->face_cells[2 * f + 1]];
        for (int d = 0; d < D; ++d) {
            h.fn[(size_t)f * D + d] = m->face_n[(size_t)f * D + d];
            const double xf = m->face_xc[(size_t)f * D + d];
            h.frL[(size_t)f * D + d] = xf - X(h.fL[f], d);
            if (h.fR[f] >= 0) {
                const double sh = (t == UGKS_FACE_PERIODIC) ? m->face_shift[(size_t)f * D + d] : 0.0;
                h.frR[(size_t)f * D + d] = xf - sh - X(h.fR[f], d);
            }
        }
        if (t == UGKS_FACE_FARFIELD) {
            h.faux[f] = (int)h.gface.size();
            h.gface.push_back(f);
        } else if (t == UGKS_FACE_WALL) {
            h.faux[f] = (int)h.wface.size();
            h.wface.push_back(f);
        }
    }

    // ---- faces of each cell (CSR, face order within a cell)
    h.cf_ptr.assign(C + 1, 0);
    for (int f = 0; f < F; ++f) {
        h.cf_ptr[h.fL[f] + 1]++;
        if (h.fR[f] >= 0) h.cf_ptr[h.fR[f] + 1]++;
    }
    for (int i = 0; i < C; ++i) h.cf_ptr[i + 1] += h.cf_ptr[i];
    const int ncf = h.cf_ptr[C];
    h.cf_face.resize(ncf);
    h.cf_side.resize(ncf);
    h.cf_r.resize((size_t)ncf * D);
    h.cf_coef.resize(ncf);
    std::vector<int> fill(C, 0);
    for (int f = 0; f < F; ++f)
        for (int s = 0; s < 2; ++s) {
            const int c = s == 0 ? h.fL[f] : h.fR[f];
            if (c < 0) continue;
            const int e = h.cf_ptr[c] + fill[c]++;
            h.cf_face[e] = f;
            h.cf_side[e] = (signed char)s;
            for (int d = 0; d < D; ++d) h.cf_r[(size_t)e * D + d] = s == 0 ? h.frL[(size_t)f * D + d] : h.frR[(size_t)f * D + d];
            h.cf_coef[e] = (s == 0 ? -1.0 : 1.0) * m->face_S[f] / h.vol[c];
        }

    // ---- least squares: neighbours across non-wall faces, far-field ghosts
    //      mirrored across the face; weights 1/|d|^2; a = w M^{-1} d
    h.nb_ptr.assign(C + 1, 0);
    h.eps2.resize(C);
    std::vector<double> dvec;
    for (int c = 0; c < C; ++c) {
        double sumS = 0.0;
        const int n0 = (int)h.nb_id.size();
        for (int e = h.cf_ptr[c]; e < h.cf_ptr[c + 1]; ++e) {
            const int f = h.cf_face[e];
            sumS += m->face_S[f];
            const int t = h.ftype[f];
            if (t == UGKS_FACE_WALL) continue;
            double d[3];
            if (t == UGKS_FACE_FARFIELD) {
                double rn = 0.0;
                for (int k = 0; k < D; ++k) rn += h.frL[(size_t)f * D + k] * h.fn[(size_t)f * D + k];
                for (int k = 0; k < D; ++k) d[k] = 2.0 * rn * h.fn[(size_t)f * D + k];
                h.nb_id.push_back(-(h.faux[f] + 1));
            } else {
                // vector from this cell to the other one through the face
                const bool own = h.cf_side[e] == 0;
                const int o = own ? h.fR[f] : h.fL[f];
                for (int k = 0; k < D; ++k) {
                    const double ro = own ? h.frR[(size_t)f * D + k] : h.frL[(size_t)f * D + k];
                    d[k] = h.cf_r[(size_t)e * D + k] - ro;
                }
                h.nb_id.push_back(o);
            }
            for (int k = 0; k < D; ++k) dvec.push_back(d[k]);
        }
        const int n1 = (int)h.nb_id.size();
        h.nb_ptr[c + 1] = n1;
        double A[9] = {0}, Ai[9];
        for (int q = n0; q < n1; ++q) {
            const double *d = &dvec[(size_t)q * D];
            double dd = 0.0;
            for (int k = 0; k < D; ++k) dd += d[k] * d[k];
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) A[a * D + b] += d[a] * d[b] / dd;
        }
        const bool ok = n1 > n0 && invert_small(D, A, Ai);
        for (int q = n0; q < n1; ++q) {
            const double *d = &dvec[(size_t)q * D];
            double dd = 0.0;
            for (int k = 0; k < D; ++k) dd += d[k] * d[k];
            for (int a = 0; a < D; ++a) {
                double s = 0.0;
                if (ok)
                    for (int b = 0; b < D; ++b) s += Ai[a * D + b] * d[b];
                h.nb_a.push_back(s / dd);
            }
        }
        // limiter scale h_c = 2 D |Omega_c| / sum S (the time-step scale is cfl_dt_of's)
        const double hc = 2.0 * D * h.vol[c] / sumS;
        const double Kh = p->venkat_K * hc;
        h.eps2[c] = Kh * Kh * Kh;
    }

    // ---- gather entry values of every (cell, face), in the cell's own
    //      orientation: LSQ coefficient, x_f - x_c, outward normal,
    //      x_f - x_other, -S_f / |Omega_c|
    const int GL = D == 2 ? ugks::GEnt<2>::LEN : ugks::GEnt<3>::LEN;
    h.gf.assign((size_t)ncf * GL, 0.0);
    for (int c = 0; c < C; ++c) {
        int q = h.nb_ptr[c];
        for (int e = h.cf_ptr[c]; e < h.cf_ptr[c + 1]; ++e) {
            const int f = h.cf_face[e], t = h.ftype[f];
            const bool own = h.cf_side[e] == 0;
            double *g = &h.gf[(size_t)e * GL];
            const int oA = D == 2 ? ugks::GEnt<2>::A : ugks::GEnt<3>::A;
            const int oRS = D == 2 ? ugks::GEnt<2>::RS : ugks::GEnt<3>::RS;
            const int oN = D == 2 ? ugks::GEnt<2>::N : ugks::GEnt<3>::N;
            const int oRO = D == 2 ? ugks::GEnt<2>::RO : ugks::GEnt<3>::RO;
            const int oCS = D == 2 ? ugks::GEnt<2>::CS : ugks::GEnt<3>::CS;
            if (t != UGKS_FACE_WALL) {
                for (int d = 0; d < D; ++d) g[oA + d] = h.nb_a[(size_t)q * D + d];
                ++q;
            }
            for (int d = 0; d < D; ++d) {
                g[oRS + d] = h.cf_r[(size_t)e * D + d];
                g[oN + d] = own ? h.fn[(size_t)f * D + d] : -h.fn[(size_t)f * D + d];
                if (t == UGKS_FACE_INTERIOR || t == UGKS_FACE_PERIODIC)
                    g[oRO + d] = own ? h.frR[(size_t)f * D + d] : h.frL[(size_t)f * D + d];
            }
            g[oCS] = -m->face_S[f] / h.vol[c];
        }
    }

    build_patches(h, C, P);
}

// gather patches: P consecutive cells (Morton order) and their face neighbours
// (ring); slot indices of every face entry's owner / neighbour in its patch
void build_patches(Host &h, int C, int P)
{
    const int ncf = h.cf_ptr[C];
    h.ring_ptr.clear();
    h.ring_cells.clear();
    h.max_slope = 0;
    const int np = (C + P - 1) / P;
    h.ring_ptr.assign(np + 1, 0);
    h.gi.assign((size_t)ncf * 4, -1);
    std::vector<int> slot_of(C, -1);
    for (int pi = 0; pi < np; ++pi) {
        const int cb = pi * P, ce = std::min(C, cb + P);
        for (int c = cb; c < ce; ++c) slot_of[c] = c - cb;
        int ns = ce - cb;
        std::vector<int> ring;
        for (int c = cb; c < ce; ++c)
            for (int e = h.cf_ptr[c]; e < h.cf_ptr[c + 1]; ++e) {
                const int f = h.cf_face[e];
                for (int o : {h.fL[f], h.fR[f]})
                    if (o >= 0 && slot_of[o] < 0) {
                        slot_of[o] = ns++;
                        ring.push_back(o);
                    }
            }
        // gather entries of the patch cells: {other, face, type, slot of other}
        for (int c = cb; c < ce; ++c)
            for (int e = h.cf_ptr[c]; e < h.cf_ptr[c + 1]; ++e) {
                const int f = h.cf_face[e], t = h.ftype[f];
                int *g = &h.gi[(size_t)e * 4];
                if (t == UGKS_FACE_INTERIOR || t == UGKS_FACE_PERIODIC) {
                    const int o = h.cf_side[e] == 0 ? h.fR[f] : h.fL[f];
                    g[0] = o;
                    g[3] = slot_of[o];
                } else {
                    g[0] = h.faux[f];
                }
                g[1] = f;
                g[2] = t;
            }
        h.max_slope = std::max(h.max_slope, ns);
        h.ring_cells.insert(h.ring_cells.end(), ring.begin(), ring.end());
        h.ring_ptr[pi + 1] = (int)h.ring_cells.size();
        for (int c = cb; c < ce; ++c) slot_of[c] = -1;
        for (int o : ring) slot_of[o] = -1;
    }
    if (h.max_slope > 32767) fail(UGKS_EINVAL, "patch too large");
}

template <typename T>
std::vector<T> cast(const std::vector<double> &v)
{
    return std::vector<T>(v.begin(), v.end());
}

template <typename T>
void fill_case(ugks_case *c, ugks::DevCase<T> &dc, const ugks_mesh *m, const ugks_vgrid *v, const ugks_params *p,
               const Host &h)
{
    const int D = c->D, M = D + 2;
    dc.D = D;
    dc.NC = c->NC;
    dc.C = (int)c->C;
    dc.F = (int)c->F;
    dc.G = c->G;
    dc.NW = c->NW;
    dc.nv = (int)c->Nv;
    dc.nvp = (int)c->nvp;
    dc.dt = c->dt;
    dc.Pr = p->Pr;
    dc.omega = p->omega;
    dc.nxi = 3.0 - D;
    dc.mu_ref = std::isinf(p->Kn) ? INFINITY
                                  : 15.0 * std::sqrt(2.0 * M_PI) * p->Kn * p->L_ref /
                                        (2.0 * (5.0 - 2.0 * p->omega) * (7.0 - 2.0 * p->omega));
    dc.limiter = p->limiter ? 1 : 0;
    dc.w0_analytic = p->w0_analytic ? 1 : 0;
    // velocities, padded with u = 0, w = 0
    for (int d = 0; d < 3; ++d) {
        dc.ud[d] = nullptr;
        dc.u[d] = nullptr;
    }
    for (int d = 0; d < D; ++d) {
        std::vector<double> ud(c->nvp, 0.0);
        for (int64_t k = 0; k < c->Nv; ++k) ud[k] = v->u[k * D + d];
        dc.ud[d] = c->upload(ud);
        dc.u[d] = c->upload(cast<T>(ud));
    }
    // tensor-product grid: u_k = (x_i, y_j[, z_l]), k = i + nx (j + ny l), and
    // w_k = wx_i wy_j [wz_l]; verified exactly for the axes and to 1e-14 for the
    // weights, else the general per-velocity face sums are used
    dc.sep = 0;
    dc.sep1 = 0;
    for (int d = 0; d < 3; ++d) {
        dc.cart_n[d] = 0;
        dc.axis[d] = dc.axw[d] = nullptr;
    }
    {
        int64_t prod = 1;
        bool ok = true;
        for (int d = 0; d < D; ++d) {
            ok = ok && v->cart_n[d] > 1;
            prod *= std::max(v->cart_n[d], 1);
        }
        ok = ok && prod == c->Nv;
        if (ok) {
            const int nx = v->cart_n[0], ny = v->cart_n[1], nz = D == 3 ? v->cart_n[2] : 1;
            std::vector<std::vector<double>> ax(D), aw(D);
            auto kidx = [&](int i, int j, int l) { return (int64_t)i + (int64_t)nx * (j + (int64_t)ny * l); };
            const int nn[3] = {nx, ny, nz};
            for (int d = 0; d < D; ++d) {
                for (int i = 0; i < nn[d]; ++i) {
                    int ijk[3] = {0, 0, 0};
                    ijk[d] = i;
                    const int64_t k = kidx(ijk[0], ijk[1], ijk[2]);
                    ax[d].push_back(v->u[k * D + d]);
                    aw[d].push_back(d == 0 ? v->w[k] : v->w[k] / v->w[0]);
                }
            }
            for (int l = 0; l < nz && ok; ++l)
                for (int j = 0; j < ny && ok; ++j)
                    for (int i = 0; i < nx && ok; ++i) {
                        const int64_t k = kidx(i, j, l);
                        const int ijk[3] = {i, j, l};
                        double wp = 1.0;
                        for (int d = 0; d < D; ++d) {
                            ok = ok && v->u[k * D + d] == ax[d][ijk[d]];
                            wp *= aw[d][ijk[d]];
                        }
                        ok = ok && std::fabs(wp - v->w[k]) <= 1e-14 * std::fabs(v->w[k]) + 1e-300;
                    }
            if (ok) {
                dc.sep = 1;
                for (int d = 0; d < D; ++d) {
                    dc.cart_n[d] = nn[d];
                    dc.axis[d] = c->upload(cast<T>(ax[d]));
                    dc.axw[d] = c->upload(cast<T>(aw[d]));
                }
                // the separable half-range sums search the last axis for the
                // sign changes of u.n, so its nodes must ascend (also in T)
                const std::vector<T> last = cast<T>(ax[D - 1]);
                bool asc = last.size() <= (size_t)ugks::SUM1_SEP_MAX_NL;
                for (size_t i = 1; i < last.size(); ++i) asc = asc && last[i - 1] < last[i];
                dc.sep1 = asc ? 1 : 0;
            }
        }
    }
    std::vector<double> wd(c->nvp, 0.0);
    for (int64_t k = 0; k < c->Nv; ++k) wd[k] = v->w[k];
    dc.wd = c->upload(wd);
    dc.w = c->upload(cast<T>(wd));
    {
        std::vector<T> uw((size_t)c->nvp * 4, T(0));
        for (int64_t k = 0; k < c->Nv; ++k) {
            for (int d = 0; d < D; ++d) uw[(size_t)k * 4 + d] = (T)v->u[k * D + d];
            uw[(size_t)k * 4 + 3] = (T)v->w[k];
        }
        dc.uw = c->upload(uw);
    }
    // state
    const size_t fcount = (size_t)c->C * c->NC * c->nvp;
    dc.f_cur = (T *)c->dalloc(fcount * sizeof(T));
    // f_nxt also stages state I/O, in host rows of up to FP64: room for at
    // least two cells' FP64 rows (one per upload slot), even on tiny meshes
    c->stage_bytes = std::max(fcount * sizeof(T), (size_t)2 * c->NC * c->nvp * sizeof(double));
    dc.f_nxt = (T *)c->dalloc(c->stage_bytes);
    c->f_bytes = fcount * sizeof(T);
    std::vector<double> W((size_t)c->C * M);
    for (int64_t i = 0; i < c->C; ++i) {
        const int ci = h.perm_u2i[i];
        double pr[5];
        if (p->prim_init) {
            for (int k = 0; k < M; ++k) pr[k] = p->prim_init[i * M + k];
        } else {
            pr[0] = p->inf_rho;
            for (int d = 0; d < D; ++d) pr[1 + d] = p->inf_U[d];
            pr[D + 1] = p->inf_T;
        }
        double ke = 0.0;
        W[(size_t)ci * M] = pr[0];
        for (int d = 0; d < D; ++d) {
            W[(size_t)ci * M + 1 + d] = pr[0] * pr[1 + d];
            ke += pr[1 + d] * pr[1 + d];
        }
        W[(size_t)ci * M + D + 1] = pr[0] * (0.5 * ke + 1.5 * pr[D + 1]);
    }
    dc.W = c->upload(W);
    dc.q = (double *)c->dalloc((size_t)c->C * D * sizeof(double));
    dc.gradW = (double *)c->dalloc((size_t)c->C * D * M * sizeof(double));
    dc.gradprim = (double *)c->dalloc((size_t)c->C * D * M * sizeof(double));
    dc.prim = (double *)c->dalloc((size_t)c->C * M * sizeof(double));
    dc.primg = (double *)c->dalloc((size_t)std::max(c->G, 1) * M * sizeof(double));
    dc.vol = c->upload(h.vol);
    dc.nb_ptr = c->upload(h.nb_ptr);
    dc.nb_id = c->upload(h.nb_id);
    dc.nb_a_d = c->upload(h.nb_a);
    dc.nb_a = c->upload(cast<T>(h.nb_a));
    dc.cf_ptr = c->upload(h.cf_ptr);
    dc.cf_face = c->upload(h.cf_face);
    dc.cf_side = c->upload(h.cf_side);
    dc.cf_r_d = c->upload(h.cf_r);
    dc.cf_r = c->upload(cast<T>(h.cf_r));
    dc.cf_coef = c->upload(cast<T>(h.cf_coef));
    dc.gi = reinterpret_cast<const int4 *>(c->upload(h.gi));
    dc.gf = c->upload(cast<T>(h.gf));
    dc.eps2_d = c->upload(h.eps2);
    dc.eps2 = c->upload(cast<T>(h.eps2));
    dc.fL = c->upload(h.fL);
    dc.fR = c->upload(h.fR);
    dc.faux = c->upload(h.faux);
    dc.ftype = c->upload(h.ftype);
    dc.ftag = c->upload(h.ftag);
    dc.fn_d = c->upload(h.fn);
    dc.frL_d = c->upload(h.frL);
    dc.frR_d = c->upload(h.frR);
    dc.fn = c->upload(cast<T>(h.fn));
    dc.frL = c->upload(cast<T>(h.frL));
    dc.frR = c->upload(cast<T>(h.frR));
    dc.dtT = (T)c->dt;
    dc.gface = c->upload(h.gface);
    dc.Wg = (double *)c->dalloc((size_t)std::max(c->G, 1) * M * sizeof(double));
    dc.grec = (T *)c->dalloc((size_t)std::max(c->G, 1) * ugks::GREC * sizeof(T));
    dc.wface = c->upload(h.wface);
    std::vector<double> wT(std::max(p->n_walls, 1), 1.0), wU(3 * std::max(p->n_walls, 1), 0.0);
    for (int i = 0; i < p->n_walls; ++i) {
        wT[i] = p->wall_T[i];
        for (int d = 0; d < 3; ++d) wU[3 * i + d] = p->wall_U[3 * i + d];
    }
    dc.wallT = c->upload(wT);
    dc.wallU = c->upload(wU);
    {
        double ke = 0.0;
        dc.inf_W[0] = p->inf_rho;
        for (int d = 0; d < D; ++d) {
            dc.inf_W[1 + d] = p->inf_rho * p->inf_U[d];
            ke += p->inf_U[d] * p->inf_U[d];
        }
        dc.inf_W[D + 1] = p->inf_rho * (0.5 * ke + 1.5 * p->inf_T);
    }
    dc.rho_w = (double *)c->dalloc((size_t)std::max(c->NW, 1) * sizeof(double));
    dc.wall_F = (double *)c->dalloc((size_t)std::max(c->NW, 1) * M * sizeof(double));
    cuda_ok(cudaMemsetAsync(dc.wall_F, 0, (size_t)std::max(c->NW, 1) * M * sizeof(double), c->stream), "memset");
    c->wall_face_h.assign(h.wface.begin(), h.wface.end());
    c->wall_n_h.resize((size_t)c->NW * D);
    for (int s = 0; s < c->NW; ++s)
        for (int d = 0; d < D; ++d) c->wall_n_h[(size_t)s * D + d] = m->face_n[(size_t)h.wface[s] * D + d];
    dc.wrec = (T *)c->dalloc((size_t)std::max(c->NW, 1) * ugks::GREC * sizeof(T));
    dc.crec = (T *)c->dalloc((size_t)c->C * ugks::CREC * sizeof(T));
    dc.krec = (T *)c->dalloc((size_t)c->C * ugks::CREC * sizeof(T));
    const size_t Fm = (size_t)std::max<int64_t>(c->F, 1);
    dc.frec = (T *)c->dalloc(Fm * ugks::FREC * sizeof(T));
    dc.xrec = (T *)c->dalloc(Fm * ugks::XREC * sizeof(T));
    dc.fside = (T *)c->dalloc(Fm * 2 * ugks::GREC * sizeof(T));
    dc.fdW0 = (double *)c->dalloc(Fm * D * M * sizeof(double));
    dc.fq0 = (double *)c->dalloc(Fm * D * sizeof(double));
    dc.fUref = (double *)c->dalloc(Fm * D * sizeof(double));
    dc.fsum1 = (double *)c->dalloc(Fm * M * sizeof(double));
    const int NS = M * (M + 1) / 2;
    dc.fsum2 = (double *)c->dalloc(Fm * NS * (D + 1) * sizeof(double));
    dc.fprim0 = (double *)c->dalloc(Fm * M * sizeof(double));
    dc.fqs = (double *)c->dalloc(Fm * 5 * sizeof(double));
    // sized for the smallest velocity tile, so that the autotuner may retile
    dc.dW_part = (double *)c->dalloc((size_t)c->C * (c->nvp / 32) * M * sizeof(double));
    dc.res_part = (double *)c->dalloc((size_t)c->n_res_blocks * 2 * M * sizeof(double));
    dc.flags = c->flags_d;
    dc.owned = nullptr;
    dc.P = c->P;
    dc.nth = c->nth;
    dc.vt_group = c->vt_group;
    dc.n_groups = c->n_groups;
    dc.n_patches = c->n_patches;
    dc.n_vt = c->n_vt;
    dc.vtile = c->vtile;
    dc.ring_ptr = c->upload(h.ring_ptr);
    dc.ring_cells = c->upload(h.ring_cells);
}

}  // namespace

namespace {

// Autotuner of the gather tiling: the patch size, the velocity tile and the
// threads per CTA are chosen by timing the gather kernel itself on this case (it writes only f~
// and scratch, so the state is untouched), and the choice is cached per
// (dimension, precision, velocity count, mesh-size bucket) for later cases of
// the same shape.
struct Tiling {
    int P = 0, vtile = 0, nth = 256, G = 1;
};
std::mutex g_tune_mutex;
std::map<std::string, Tiling> g_tune_cache;

// dynamic shared memory of the gather: the moment accumulators (P x 16
// values) and the slope buffer ((patch + ring) x NC x D x vtile values)
size_t gather_smem(int max_slope, int NC, int D, int vtile, int P, size_t esz)
{
    return ((size_t)P * 16 + (size_t)max_slope * NC * D * vtile) * esz;
}

// velocity tile used when neither the caller nor the autotuner sets one
int kDefaultVtile(int prec) { return prec == UGKS_FP64 ? 32 : 64; }

template <typename T>
void set_tiling(ugks_case *c, ugks::DevCase<T> &dc, const Host &h, int P, int vtile, int nth, int G, size_t smem)
{
    c->P = P;
    c->n_patches = (int)((c->C + P - 1) / P);
    c->vtile = vtile;
    c->nth = nth;
    c->n_vt = (int)(c->nvp / vtile);
    c->vt_group = std::max(1, std::min(G, c->n_vt));
    c->n_groups = (c->n_vt + c->vt_group - 1) / c->vt_group;
    c->cfg.smem = smem;
    dc.P = P;
    dc.n_patches = c->n_patches;
    dc.vtile = vtile;
    dc.nth = nth;
    dc.n_vt = c->n_vt;
    dc.vt_group = c->vt_group;
    dc.n_groups = c->n_groups;
    // the old patch arrays may still be read by queued kernels: drain the
    // stream first, so that any allocator may reuse them at once
    if (dc.ring_ptr || dc.ring_cells || dc.gi)
        cuda_ok(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize(), "retile sync");
    c->dfree(dc.ring_ptr);
    c->dfree(dc.ring_cells);
    c->dfree(dc.gi);
    dc.ring_ptr = c->upload(h.ring_ptr);
    dc.ring_cells = c->upload(h.ring_cells);
    dc.gi = reinterpret_cast<const int4 *>(c->upload(h.gi));
}

template <typename T>
void autotune(ugks_case *c, ugks::DevCase<T> &dc, Host &h, int smem_max, bool tune_vtile, bool tune_threads,
              bool tune_group)
{
    const size_t esz = sizeof(T);
    char key[160];
    snprintf(key, sizeof(key), "D%d_nc%d_p%d_vt%d_t%d_g%d_nv%lld_c%d", c->D, c->NC, c->prec,
             tune_vtile ? 0 : c->vtile, tune_threads ? 0 : c->nth, tune_group ? 0 : c->vt_group, (long long)c->Nv,
             (int)std::lround(std::log2((double)c->C)));
    Tiling best;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) best = it->second;
    }
    const int C = (int)c->C;
    auto smem_of = [&](const Host &hh, int vt, int P) { return gather_smem(hh.max_slope, c->NC, c->D, vt, P, esz); };
    if (best.P == 0) {
        // tetrahedra have more faces and larger rings than triangles, and one
        // stored component per velocity: smaller patches and wider velocity tiles
        const std::vector<int> pc = c->prec == UGKS_FP64 ? std::vector<int>{16, 24, 32, 48}
                                    : c->D == 3          ? std::vector<int>{16, 24, 32, 48, 64, 96}
                                                         : std::vector<int>{24, 32, 48, 64, 96};
        std::vector<int> vc = {c->vtile};
        if (tune_vtile) vc = c->D == 3 ? std::vector<int>{32, 64, 128} : std::vector<int>{32, 64};
        // 512-thread CTAs (64 registers, two per SM) for FP32 at up to 64 velocities
        std::vector<int> tc = {c->nth};
        if (tune_threads) tc = c->prec == UGKS_FP32 ? std::vector<int>{256, 512} : std::vector<int>{256};
        cuda_ok(ugks::launch_pre_gather(dc, c->stream), "autotune prep");
        cudaEvent_t e0, e1;
        cuda_ok(cudaEventCreate(&e0), "event");
        cuda_ok(cudaEventCreate(&e1), "event");
        auto time_gather = [&](size_t smem) {
            cuda_ok(ugks::launch_gather(dc, smem, c->stream), "autotune gather");
            cuda_ok(cudaEventRecord(e0, c->stream), "event");
            for (int r = 0; r < 2; ++r) cuda_ok(ugks::launch_gather(dc, smem, c->stream), "autotune gather");
            cuda_ok(cudaEventRecord(e1, c->stream), "event");
            cuda_ok(cudaEventSynchronize(e1), "event");
            float ms = 0.f;
            cuda_ok(cudaEventElapsedTime(&ms, e0, e1), "event");
            return ms;
        };
        const int G0 = c->vt_group;
        float best_ms = 0.f;
        for (int nth : tc)
            for (int vt : vc) {
                if (c->nvp % vt || (nth == 512 && vt > 64)) continue;
                for (int P : pc) {
                    if (P > C && P != pc.front()) continue;
                    if (nth == 512 && P < 32) continue;          // 16 warps need work
                    build_patches(h, C, P);
                    const size_t smem = smem_of(h, vt, P);
                    if (smem > (size_t)smem_max) continue;
                    set_tiling(c, dc, h, P, vt, nth, G0, smem);
                    const float ms = time_gather(smem);
                    if (best.P == 0 || ms < best_ms) {
                        best = {P, vt, nth, G0};
                        best_ms = ms;
                    }
                }
            }
        // then the grid order at the chosen tiling: groups of G velocity tiles
        if (best.P != 0 && tune_group) {
            build_patches(h, C, best.P);
            const size_t smem = smem_of(h, best.vtile, best.P);
            set_tiling(c, dc, h, best.P, best.vtile, best.nth, G0, smem);
            for (int G : {1, 2, 4, 8, 16, 32, 64}) {
                if (G == G0 || G > c->n_vt) continue;
                dc.vt_group = G;
                dc.n_groups = (c->n_vt + G - 1) / G;
                const float ms = time_gather(smem);
                if (ms < best_ms) {
                    best.G = G;
                    best_ms = ms;
                }
            }
            dc.vt_group = c->vt_group;
            dc.n_groups = c->n_groups;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (best.P == 0) return;                 // keep the default tiling
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best;
    }
    if (best.P != c->P || best.vtile != c->vtile || best.nth != c->nth) {
        build_patches(h, C, best.P);
        const size_t smem = smem_of(h, best.vtile, best.P);
        if (smem <= (size_t)smem_max) set_tiling(c, dc, h, best.P, best.vtile, best.nth, best.G, smem);
    } else if (best.G != c->vt_group) {
        c->vt_group = dc.vt_group = best.G;
        c->n_groups = dc.n_groups = (c->n_vt + best.G - 1) / best.G;
    }
}

ugks_status guard(const std::function<void()> &fn)
{
    try {
        g_err.clear();
        fn();
        return UGKS_OK;
    } catch (const Fail &e) {
        g_err = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        return UGKS_ENOMEM;
    } catch (const std::exception &e) {
        g_err = e.what();
        return UGKS_EINVAL;
    } catch (...) {
        g_err = "unknown error";
        return UGKS_EINVAL;
    }
}

template <typename Fn>
auto with_dc(ugks_case *c, Fn &&fn)
{
    if (c->prec == UGKS_FP64) return fn(c->d64);
    return fn(c->d32);
}

// f of the case into host memory, f[C][ncomp][nv] of element type S in caller
// cell order, staged through the f_nxt buffer in chunks of cells
template <typename S>
void export_f(ugks_case *c, S *f)
{
    const size_t per = (size_t)c->NC * c->Nv;
    const size_t cap = c->stage_bytes / sizeof(S);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(cap / per, (size_t)c->C));
    for (int c0 = 0; c0 < (int)c->C; c0 += chunk) {
        const int nc = (int)std::min<int64_t>(chunk, c->C - c0);
        with_dc(c, [&](auto &dc) {
            S *stg = (S *)dc.f_nxt;
            cuda_ok(ugks::launch_f_export(dc, c->perm_d, c0, nc, stg, c->stream), "f export");
            cuda_ok(cudaMemcpyAsync(f + (size_t)c0 * per, stg, (size_t)nc * per * sizeof(S), cudaMemcpyDeviceToHost,
                                    c->stream),
                    "f copy");
            cuda_ok(cudaStreamSynchronize(c->stream), "sync");
        });
    }
}

// f from host memory (layout of export_f) into the case.  The f_nxt buffer is
// split into two staging slots; chunks of cells alternate between them.  The
// copy of a chunk runs on the case's copy stream while the case stream imports
// (reorders and converts) the chunk before it; a slot is refilled only after
// its previous import.  The first copy waits for the work already queued on
// the case stream, which may still use f_nxt.
template <typename S>
void import_f(ugks_case *c, const S *f)
{
    const size_t per = (size_t)c->NC * c->Nv;
    const size_t slot = c->stage_bytes / 2 / sizeof(S);            // >= one cell's row
    int chunk = (int)std::max<size_t>(1, std::min<size_t>(slot / per, (size_t)c->C));
    chunk = std::min(chunk, (int)std::max<int64_t>(1, (c->C + 3) / 4));   // at least four chunks in flight
    if (!c->copy_stream) {
        cuda_ok(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "copy stream");
        for (auto &e : c->io_ev) cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create");
    }
    cudaEvent_t ready = c->io_ev[0], *copied = c->io_ev + 1, *consumed = c->io_ev + 3;
    cuda_ok(cudaEventRecord(ready, c->stream), "event");
    cuda_ok(cudaStreamWaitEvent(c->copy_stream, ready, 0), "event wait");
    int k = 0;
    for (int c0 = 0; c0 < (int)c->C; c0 += chunk, ++k) {
        const int nc = (int)std::min<int64_t>(chunk, c->C - c0);
        const int sl = k & 1;
        if (k >= 2) cuda_ok(cudaStreamWaitEvent(c->copy_stream, consumed[sl], 0), "event wait");
        with_dc(c, [&](auto &dc) {
            S *stg = (S *)dc.f_nxt + (size_t)sl * slot;
            cuda_ok(cudaMemcpyAsync(stg, f + (size_t)c0 * per, (size_t)nc * per * sizeof(S), cudaMemcpyHostToDevice,
                                    c->copy_stream),
                    "f upload");
            cuda_ok(cudaEventRecord(copied[sl], c->copy_stream), "event");
            cuda_ok(cudaStreamWaitEvent(c->stream, copied[sl], 0), "event wait");
            cuda_ok(ugks::launch_f_import(dc, c->perm_d, c0, nc, stg, c->stream), "f import");
            cuda_ok(cudaEventRecord(consumed[sl], c->stream), "event");
        });
    }
}

// W[C][dim+2] (caller cell order) into the case through the gradW scratch
void import_W(ugks_case *c, const double *W)
{
    const int D = c->D, M = D + 2;
    double *Wd = c->prec == UGKS_FP64 ? c->d64.W : c->d32.W;
    double *stg = c->prec == UGKS_FP64 ? c->d64.gradW : c->d32.gradW;
    cuda_ok(cudaMemcpyAsync(stg, W, (size_t)c->C * M * sizeof(double), cudaMemcpyHostToDevice, c->stream),
            "W upload");
    cuda_ok(ugks::launch_W_permute(stg, c->perm_d, (int)c->C, D, Wd, 1, c->stream), "W import");
}

void export_W(ugks_case *c, double *W)
{
    const int D = c->D, M = D + 2;
    double *Wd = c->prec == UGKS_FP64 ? c->d64.W : c->d32.W;
    double *stg = c->prec == UGKS_FP64 ? c->d64.gradW : c->d32.gradW;
    cuda_ok(ugks::launch_W_permute(Wd, c->perm_d, (int)c->C, D, stg, 0, c->stream), "W export");
    cuda_ok(cudaMemcpyAsync(W, stg, (size_t)c->C * M * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "W copy");
    cuda_ok(cudaStreamSynchronize(c->stream), "sync");
}

template <typename S>
ugks_status get_state(ugks_case *c, S *f, double *W)
{
    return guard([&] {
        if (!c) fail(UGKS_EINVAL, "case is NULL");
        if (W) export_W(c, W);
        if (f) export_f(c, f);
    });
}

template <typename S>
ugks_status set_state(ugks_case *c, const S *f, const double *W)
{
    return guard([&] {
        if (!c) fail(UGKS_EINVAL, "case is NULL");
        if (W) import_W(c, W);
        if (f) import_f(c, f);
        if (f || W) with_dc(c, [&](auto &dc) { cuda_ok(ugks::launch_heatflux(dc, c->stream), "heat flux"); });
    });
}
}  // namespace

namespace ugks {
// lets other translation units of the library report through ugks_last_error()
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace ugks

extern "C" {

const char *ugks_last_error(void) { return g_err.c_str(); }

ugks_status ugks_create(const ugks_mesh *mesh, const ugks_vgrid *vgrid, const ugks_params *params,
                        const ugks_alloc *alloc, void *stream, ugks_case **out)
{
    if (!out) {
        g_err = "out must not be NULL";
        return UGKS_EINVAL;
    }
    *out = nullptr;
    std::unique_ptr<ugks_case> c(new ugks_case());
    ugks_status st = guard([&] {
        validate(mesh, vgrid, params);
        if (alloc && (!alloc->alloc || !alloc->free)) fail(UGKS_EINVAL, "allocator callbacks missing");
        c->D = mesh->dim;
        c->NC = mesh->dim == 2 ? 2 : 1;
        c->prec = params->precision;
        c->C = mesh->n_cells;
        c->F = mesh->n_faces;
        c->Nv = vgrid->nv;
        c->stream = (cudaStream_t)stream;
        if (alloc) {
            c->alloc = *alloc;
            c->user_alloc = true;
        }
        const size_t esz = c->prec == UGKS_FP64 ? 8 : 4;
        // tiling: velocity tile of 32*TV, patch of P cells sized to shared memory
        // velocity rows are padded to a multiple of the widest tile the autotuner
        // may choose (64 in 2D, 128 in 3D) unless the tile is fixed
        c->vtile = params->vtile > 0 ? params->vtile : kDefaultVtile(c->prec);
        c->nth = params->gather_threads > 0 ? params->gather_threads : 256;
        const int vpad = params->vtile > 0 ? params->vtile : (c->D == 3 ? 128 : 64);
        int P = params->patch_cells > 0 ? params->patch_cells : (c->prec == UGKS_FP64 ? 32 : 48);
        Host h;
        int dev = 0;
        cuda_ok(cudaGetDevice(&dev), "cudaGetDevice");
        int smem_max = 0;
        cuda_ok(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "smem attr");
        for (;;) {
            h = Host();
            preprocess(mesh, params, P, h);
            const size_t smem = gather_smem(h.max_slope, c->NC, c->D, c->vtile, P, esz);
            if (smem <= (size_t)smem_max || P <= 4) {
                if (smem > (size_t)smem_max) fail(UGKS_EINVAL, "mesh stencil too large for shared memory");
                c->cfg.smem = smem;
                break;
            }
            P = std::max(4, P / 2);
        }
        c->P = P;
        c->n_patches = (int)((c->C + P - 1) / P);
        c->nvp = (c->Nv + vpad - 1) / vpad * vpad;
        c->n_vt = (int)(c->nvp / c->vtile);
        c->vt_group = std::max(1, std::min(params->gather_tile_group > 0 ? params->gather_tile_group : 1, c->n_vt));
        c->n_groups = (c->n_vt + c->vt_group - 1) / c->vt_group;
        c->G = (int)h.gface.size();
        c->NW = (int)h.wface.size();
        // upwind CFL bound (the CFL step of Algorithm 1)
        c->dt = params->dt > 0.0 ? params->dt : cfl_dt_of(mesh, vgrid, params->cfl, mesh->n_cells);
        c->n_res_blocks = (int)((c->C + 255) / 256);
        c->cfg.n_res_blocks = c->n_res_blocks;
        c->flags_d = (int *)c->dalloc(sizeof(int));
        cuda_ok(cudaMemsetAsync(c->flags_d, 0, sizeof(int), c->stream), "memset");
        c->range_d = (unsigned long long *)c->dalloc(2 * sizeof(unsigned long long));
        c->res_d = (double *)c->dalloc(8 * sizeof(double));
        cuda_ok(cudaMemsetAsync(c->res_d, 0, 8 * sizeof(double), c->stream), "memset");
        c->perm_h.assign(h.perm_u2i.begin(), h.perm_u2i.end());
        c->perm_d = c->upload(c->perm_h);
        if (c->prec == UGKS_FP64) {
            fill_case<double>(c.get(), c->d64, mesh, vgrid, params, h);
            cuda_ok(ugks::launch_init(c->d64, c->stream), "init");
            if (params->patch_cells == 0)
                autotune<double>(c.get(), c->d64, h, smem_max, params->vtile == 0, params->gather_threads == 0,
                                 params->gather_tile_group == 0);
        } else {
            fill_case<float>(c.get(), c->d32, mesh, vgrid, params, h);
            cuda_ok(ugks::launch_init(c->d32, c->stream), "init");
            if (params->patch_cells == 0)
                autotune<float>(c.get(), c->d32, h, smem_max, params->vtile == 0, params->gather_threads == 0,
                                params->gather_tile_group == 0);
        }
        cuda_ok(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize(), "create sync");
    });
    if (st != UGKS_OK) {
        std::string keep = g_err;
        c->release();
        g_err = keep;
        return st;
    }
    *out = c.release();
    return UGKS_OK;
}

ugks_status ugks_step(ugks_case *c, int32_t nsteps)
{
    return guard([&] {
        if (!c) fail(UGKS_EINVAL, "case is NULL");
        if (nsteps < 0) fail(UGKS_EINVAL, "nsteps must be >= 0");
        for (int32_t s = 0; s < nsteps; ++s) {
            cudaEvent_t *ev = nullptr;
            if (c->prof_used < c->prof_max) ev = &c->prof_ev[(size_t)c->prof_used++ * (ugks::N_GROUPS + 1)];
            with_dc(c, [&](auto &dc) { cuda_ok(ugks::launch_step(dc, c->cfg, c->stream, ev), "step launch"); });
            ++c->step;
            c->stepped = true;
        }
    });
}

ugks_status ugks_check(ugks_case *c)
{
    return guard([&] {
        if (!c) fail(UGKS_EINVAL, "case is NULL");
        const int M = c->D + 2;
        double *W = c->prec == UGKS_FP64 ? c->d64.W : c->d32.W;
        cuda_ok(ugks::launch_check(W, (int)c->C, M, c->flags_d, c->stream), "check launch");
        int flag = 0;
        cuda_ok(cudaMemcpyAsync(&flag, c->flags_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "check copy");
        cuda_ok(cudaStreamSynchronize(c->stream), "check sync");
        if (flag) fail(UGKS_ENUMERIC, "non-finite or non-positive density / temperature in the state");
    });
}

ugks_status ugks_density_range(ugks_case *c, double *range)
{
    return guard([&] {
        if (!c || !range) fail(UGKS_EINVAL, "case and range must not be NULL");
        const int M = c->D + 2;
        const double *W = c->prec == UGKS_FP64 ? c->d64.W : c->d32.W;
        cuda_ok(ugks::launch_density_range(W, (int)c->C, M, c->owned_d, c->range_d, c->stream), "range launch");
        unsigned long long b[2];
        cuda_ok(cudaMemcpyAsync(b, c->range_d, sizeof(b), cudaMemcpyDeviceToHost, c->stream), "range copy");
        cuda_ok(cudaStreamSynchronize(c->stream), "range sync");
        if (b[0] == ~0ull) b[0] = 0ull;          // no own cell
        std::memcpy(&range[0], &b[0], sizeof(double));
        std::memcpy(&range[1], &b[1], sizeof(double));
    });
}

ugks_status ugks_moments(ugks_case *c, double *rho, double *U, double *T, double *q)
{
    return guard([&] {
        if (!c) fail(UGKS_EINVAL, "case is NULL");
        const int D = c->D;
        const size_t per = 2 * D + 2;
        double *Wd = c->prec == UGKS_FP64 ? c->d64.W : c->d32.W;
        double *qd = c->prec == UGKS_FP64 ? c->d64.q : c->d32.q;
        // reuse the gradient buffer as staging ([C][D][D+2] >= [C][2D+2])
        double *out = c->prec == UGKS_FP64 ? c->d64.gradW : c->d32.gradW;
        cuda_ok(ugks::launch_moments_out(Wd, qd, c->perm_d, (int)c->C, D, out, c->stream), "moments launch");
        std::vector<double> hbuf((size_t)c->C * per);
        cuda_ok(cudaMemcpyAsync(hbuf.data(), out, hbuf.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                "moments copy");
        cuda_ok(cudaStreamSynchronize(c->stream), "moments sync");
        for (int64_t i = 0; i < c->C; ++i) {
            const double *o = &hbuf[(size_t)i * per];
            if (rho) rho[i] = o[0];
            for (int d = 0; d < D; ++d) {
                if (U) U[i * D + d] = o[1 + d];
                if (q) q[i * D + d] = o[D + 2 + d];
            }
            if (T) T[i] = o[D + 1];
        }
    });
}

ugks_status ugks_residual(ugks_case *c, double *res)
{
    return guard([&] {
        if (!c || !res) fail(UGKS_EINVAL, "case and res must not be NULL");
        const int M = c->D + 2;
        if (!c->stepped) {
            for (int m = 0; m < M; ++m) res[m] = 0.0;
            return;
        }
        const double *rp = c->prec == UGKS_FP64 ? c->d64.res_part : c->d32.res_part;
        cuda_ok(ugks::launch_residual(rp, c->n_res_blocks, c->D, c->res_d, c->stream), "residual launch");
        cuda_ok(cudaMemcpyAsync(res, c->res_d, M * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "residual copy");
        cuda_ok(cudaStreamSynchronize(c->stream), "residual sync");
    });
}

ugks_status ugks_get_state(ugks_case *c, double *f, double *W) { return get_state(c, f, W); }

ugks_status ugks_get_state_f32(ugks_case *c, float *f, double *W) { return get_state(c, f, W); }

ugks_status ugks_wall_quantities(ugks_case *c, int64_t *face, double *p, double *sigma, double *q)
{
    return guard([&] {
        if (!c) fail(UGKS_EINVAL, "case is NULL");
        const int D = c->D, M = D + 2, NW = c->NW;
        if (NW == 0) return;
        std::vector<double> F((size_t)NW * M);
        const double *Fd = c->prec == UGKS_FP64 ? c->d64.wall_F : c->d32.wall_F;
        cuda_ok(cudaMemcpyAsync(F.data(), Fd, F.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                "wall flux copy");
        cuda_ok(cudaStreamSynchronize(c->stream), "sync");
        for (int s = 0; s < NW; ++s) {
            const double *Fs = &F[(size_t)s * M];
            const double *n = &c->wall_n_h[(size_t)s * D];
            double pn = 0.0, t2 = 0.0;
            for (int d = 0; d < D; ++d) pn += Fs[1 + d] * n[d];
            for (int d = 0; d < D; ++d) {
                const double t = Fs[1 + d] - pn * n[d];
                t2 += t * t;
            }
            if (face) face[s] = c->wall_face_h[s];
            if (p) p[s] = pn / c->dt;
            if (sigma) sigma[s] = std::sqrt(t2) / c->dt;
            if (q) q[s] = Fs[D + 1] / c->dt;
        }
    });
}

ugks_status ugks_get_cells(ugks_case *c, const int64_t *cells, int64_t n, double *f, double *W)
{
    return guard([&] {
        if (!c || !cells) fail(UGKS_EINVAL, "case and cells must not be NULL");
        if (n < 0 || n > c->C) fail(UGKS_EINVAL, "n = %lld outside [0, n_cells]", (long long)n);
        if (n == 0) return;
        const int D = c->D, M = D + 2;
        std::vector<long long> ids((size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            if (cells[i] < 0 || cells[i] >= c->C) fail(UGKS_EINVAL, "cell id %lld out of range", (long long)cells[i]);
            ids[(size_t)i] = c->perm_h[(size_t)cells[i]];
        }
        // staging in the gradient scratch (C*D*M doubles >= n*(1 + M)): the
        // internal ids, then W; f goes through the f~ buffer in chunks
        double *gW = c->prec == UGKS_FP64 ? c->d64.gradW : c->d32.gradW;
        long long *ids_d = reinterpret_cast<long long *>(gW);
        double *wst = gW + n;
        cuda_ok(cudaMemcpyAsync(ids_d, ids.data(), (size_t)n * sizeof(long long), cudaMemcpyHostToDevice, c->stream),
                "ids upload");
        if (W) {
            double *Wd = c->prec == UGKS_FP64 ? c->d64.W : c->d32.W;
            cuda_ok(ugks::launch_W_permute(Wd, ids_d, (int)n, D, wst, 0, c->stream), "W gather");
            cuda_ok(cudaMemcpyAsync(W, wst, (size_t)n * M * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                    "W copy");
        }
        if (f) {
            const size_t per = (size_t)c->NC * c->Nv;
            const size_t cap = c->stage_bytes / sizeof(double);
            const int chunk = (int)std::max<size_t>(1, std::min<size_t>(cap / per, (size_t)n));
            for (int c0 = 0; c0 < (int)n; c0 += chunk) {
                const int nc = (int)std::min<int64_t>(chunk, n - c0);
                with_dc(c, [&](auto &dc) {
                    double *stg = (double *)dc.f_nxt;
                    cuda_ok(ugks::launch_f_export(dc, ids_d, c0, nc, stg, c->stream), "f gather");
                    cuda_ok(cudaMemcpyAsync(f + (size_t)c0 * per, stg, (size_t)nc * per * sizeof(double),
                                            cudaMemcpyDeviceToHost, c->stream),
                            "f copy");
                });
                cuda_ok(cudaStreamSynchronize(c->stream), "sync");
            }
        }
        cuda_ok(cudaStreamSynchronize(c->stream), "sync");
    });
}

ugks_status ugks_set_state(ugks_case *c, const double *f, const double *W) { return set_state(c, f, W); }

ugks_status ugks_set_state_f32(ugks_case *c, const float *f, const double *W) { return set_state(c, f, W); }

ugks_status ugks_profile_begin(ugks_case *c, int32_t max_steps)
{
    return guard([&] {
        if (!c || max_steps < 0) fail(UGKS_EINVAL, "invalid profile request");
        for (auto e : c->prof_ev) cudaEventDestroy(e);
        c->prof_ev.assign((size_t)max_steps * (ugks::N_GROUPS + 1), nullptr);
        for (auto &e : c->prof_ev) cuda_ok(cudaEventCreate(&e), "event create");
        c->prof_max = max_steps;
        c->prof_used = 0;
    });
}

ugks_status ugks_profile_end(ugks_case *c, double *ms, int32_t n, int32_t *steps)
{
    return guard([&] {
        if (!c || !ms) fail(UGKS_EINVAL, "invalid profile request");
        cuda_ok(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize(), "profile sync");
        for (int i = 0; i < n; ++i) ms[i] = 0.0;
        for (int s = 0; s < c->prof_used; ++s)
            for (int g = 0; g < ugks::N_GROUPS && g < n; ++g) {
                float t = 0.f;
                cudaEvent_t *e = &c->prof_ev[(size_t)s * (ugks::N_GROUPS + 1)];
                cuda_ok(cudaEventElapsedTime(&t, e[g], e[g + 1]), "event time");
                ms[g] += t;
            }
        if (steps) *steps = c->prof_used;
        for (auto e : c->prof_ev) cudaEventDestroy(e);
        c->prof_ev.clear();
        c->prof_max = c->prof_used = 0;
    });
}

ugks_status ugks_info(const ugks_case *c, ugks_info_t *info)
{
    return guard([&] {
        if (!c || !info) fail(UGKS_EINVAL, "case and info must not be NULL");
        info->dim = c->D;
        info->ncomp = c->NC;
        info->precision = c->prec;
        info->n_cells = c->C;
        info->n_faces = c->F;
        info->nv = c->Nv;
        info->nv_pad = c->nvp;
        info->dt = c->dt;
        info->step = c->step;
        info->device_bytes = c->device_bytes;
        info->f_bytes = c->f_bytes;
        info->n_patches = c->n_patches;
        info->patch_cells = c->P;
        info->vtile = c->vtile;
        info->gather_threads = c->nth;
        info->gather_tile_group = c->vt_group;
        info->kernel_launches_per_step = 5 + (c->F > 0 ? 5 : 0) + (c->NW > 0 ? 1 : 0);
        info->n_wall_faces = c->NW;
    });
}

ugks_status ugks_cfl_dt(const ugks_mesh *mesh, const ugks_vgrid *vgrid, double cfl, int64_t n_cells, double *dt)
{
    return guard([&] {
        if (!mesh || !vgrid || !dt) fail(UGKS_EINVAL, "mesh, vgrid and dt must not be NULL");
        if (!(cfl > 0.0)) fail(UGKS_EINVAL, "cfl must be > 0");
        if (n_cells < 1 || n_cells > mesh->n_cells) fail(UGKS_EINVAL, "n_cells outside [1, mesh n_cells]");
        if (!mesh->cell_vol || !mesh->face_cells || !mesh->face_S || !vgrid->u || vgrid->nv < 1 ||
            vgrid->dim != mesh->dim)
            fail(UGKS_EINVAL, "incomplete mesh or velocity grid");
        for (int64_t f = 0; f < mesh->n_faces; ++f) {
            const int64_t a = mesh->face_cells[2 * f], b = mesh->face_cells[2 * f + 1];
            if (a < 0 || a >= mesh->n_cells || b >= mesh->n_cells) fail(UGKS_EINVAL, "face %lld: cell out of range",
                                                                       (long long)f);
        }
        *dt = cfl_dt_of(mesh, vgrid, cfl, n_cells);
    });
}

ugks_status ugks_set_owned(ugks_case *c, int64_t n_owned)
{
    return guard([&] {
        if (!c) fail(UGKS_EINVAL, "case is NULL");
        if (n_owned < 0 || n_owned > c->C) fail(UGKS_EINVAL, "n_owned outside [0, n_cells]");
        std::vector<unsigned char> mask((size_t)c->C, 0);
        for (int64_t i = 0; i < n_owned; ++i) mask[(size_t)c->perm_h[(size_t)i]] = 1;
        if (!c->owned_d) c->owned_d = (unsigned char *)c->dalloc((size_t)c->C);
        cuda_ok(cudaMemcpyAsync(c->owned_d, mask.data(), mask.size(), cudaMemcpyHostToDevice, c->stream), "upload");
        cuda_ok(cudaStreamSynchronize(c->stream), "sync");
        c->d64.owned = c->owned_d;
        c->d32.owned = c->owned_d;
    });
}

ugks_status ugks_residual_sums(ugks_case *c, double *sums)
{
    return guard([&] {
        if (!c || !sums) fail(UGKS_EINVAL, "case and sums must not be NULL");
        const int M = c->D + 2;
        for (int i = 0; i < 2 * M; ++i) sums[i] = 0.0;
        if (!c->stepped) return;
        std::vector<double> part((size_t)c->n_res_blocks * 2 * M);
        const double *rp = c->prec == UGKS_FP64 ? c->d64.res_part : c->d32.res_part;
        cuda_ok(cudaMemcpyAsync(part.data(), rp, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                "residual copy");
        cuda_ok(cudaStreamSynchronize(c->stream), "residual sync");
        for (int b = 0; b < c->n_res_blocks; ++b)
            for (int i = 0; i < 2 * M; ++i) sums[i] += part[(size_t)b * 2 * M + i];
    });
}

ugks_status ugks_halo_row_bytes(const ugks_case *c, size_t *bytes)
{
    return guard([&] {
        if (!c || !bytes) fail(UGKS_EINVAL, "case and bytes must not be NULL");
        const size_t esz = c->prec == UGKS_FP64 ? 8 : 4;
        const size_t fbytes = ((size_t)c->NC * c->Nv * esz + 7) / 8 * 8;
        *bytes = fbytes + (size_t)(2 * c->D + 2) * sizeof(double);
    });
}

ugks_status ugks_halo_set(ugks_case *c, int32_t slot, const int64_t *cells, int64_t n)
{
    return guard([&] {
        if (!c) fail(UGKS_EINVAL, "case is NULL");
        if (slot < 0 || slot >= 4096) fail(UGKS_EINVAL, "slot outside [0, 4096)");
        if (n < 0 || n > c->C || (n > 0 && !cells)) fail(UGKS_EINVAL, "invalid cell list");
        std::vector<int> ids((size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            if (cells[i] < 0 || cells[i] >= c->C) fail(UGKS_EINVAL, "cell id %lld out of range", (long long)cells[i]);
            ids[(size_t)i] = (int)c->perm_h[(size_t)cells[i]];
        }
        if ((size_t)slot >= c->halo.size()) c->halo.resize((size_t)slot + 1);
        auto &h = c->halo[(size_t)slot];
        if (h.ids) {
            cuda_ok(cudaStreamSynchronize(c->stream), "sync");   // queued packs may still read the old list
            c->dfree(h.ids);
            h.ids = nullptr;
        }
        h.n = (int)n;
        if (n > 0) h.ids = c->upload(ids);
        cuda_ok(cudaStreamSynchronize(c->stream), "sync");
    });
}

static ugks_status halo_move(ugks_case *c, int32_t slot, void *buf, int unpack)
{
    return guard([&] {
        if (!c) fail(UGKS_EINVAL, "case is NULL");
        if (slot < 0 || (size_t)slot >= c->halo.size()) fail(UGKS_EINVAL, "halo slot %d is not set", slot);
        const auto &h = c->halo[(size_t)slot];
        if (h.n > 0 && !buf) fail(UGKS_EINVAL, "buffer must not be NULL");
        size_t row = 0;
        ugks_halo_row_bytes(c, &row);
        with_dc(c, [&](auto &dc) {
            cuda_ok(ugks::launch_halo(dc, h.ids, h.n, row, buf, unpack, c->stream), unpack ? "halo unpack" : "halo pack");
        });
    });
}

ugks_status ugks_halo_pack(ugks_case *c, int32_t slot, void *device_buf) { return halo_move(c, slot, device_buf, 0); }

ugks_status ugks_halo_unpack(ugks_case *c, int32_t slot, const void *device_buf)
{
    return halo_move(c, slot, const_cast<void *>(device_buf), 1);
}

}  // extern "C"

struct ugks_batch {
    std::vector<ugks_case *> cases;
    int D = 0, prec = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *dcases = nullptr;         // device array of DevCase<T>
    // one persistent gather launch per (velocity tile, threads per CTA) in the batch
    struct Group {
        int vtile = 0, nth = 256, nwork = 0, grid = 0;
        int4 *work = nullptr;
        size_t smem = 0;
    };
    std::vector<Group> groups;
    // the other kernels of a step, one launch each over all cases: block offsets
    // off[k][0..n] (device, prefix sums of the cases' block counts), total
    // blocks and dynamic shared memory per kernel
    int *small_off = nullptr;
    int small_blocks[ugks::SK_COUNT] = {};
    size_t small_smem[ugks::SK_COUNT] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> case_ev;   // orders each case's stream with the batch stream
    cudaEvent_t done = nullptr;
};

namespace {

template <typename T>
ugks::DevCase<T> &dc_of(ugks_case *c);
template <>
ugks::DevCase<double> &dc_of<double>(ugks_case *c) { return c->d64; }
template <>
ugks::DevCase<float> &dc_of<float>(ugks_case *c) { return c->d32; }

template <typename T>
void batch_build(ugks_batch *b)
{
    const int n = (int)b->cases.size();
    std::vector<ugks::DevCase<T>> h(n);
    for (int i = 0; i < n; ++i) h[i] = dc_of<T>(b->cases[i]);
    cuda_ok(cudaMalloc(&b->dcases, sizeof(ugks::DevCase<T>) * n), "batch alloc");
    cuda_ok(cudaMemcpy(b->dcases, h.data(), sizeof(ugks::DevCase<T>) * n, cudaMemcpyHostToDevice), "batch upload");
    // offsets of the batched per-case kernels
    std::vector<int> off((size_t)ugks::SK_COUNT * (n + 1), 0);
    for (int k = 0; k < ugks::SK_COUNT; ++k) {
        int *o = &off[(size_t)k * (n + 1)];
        for (int i = 0; i < n; ++i) {
            const long long nb = (long long)o[i] + ugks::small_kernel_blocks<T>(h[i], k);
            if (nb > INT32_MAX) fail(UGKS_EINVAL, "batch too large for one launch of kernel %d", k);
            o[i + 1] = (int)nb;
            b->small_smem[k] = std::max(b->small_smem[k], ugks::small_kernel_smem<T>(h[i], k));
        }
        b->small_blocks[k] = o[n];
    }
    cuda_ok(cudaMalloc((void **)&b->small_off, off.size() * sizeof(int)), "batch alloc");
    cuda_ok(cudaMemcpy(b->small_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice), "batch upload");
    // one persistent launch per (velocity tile, threads per CTA) in the batch
    std::vector<std::pair<int, int>> tiles;
    for (auto *c : b->cases)
        if (std::find(tiles.begin(), tiles.end(), std::make_pair(c->vtile, c->nth)) == tiles.end())
            tiles.push_back({c->vtile, c->nth});
    for (const auto &tt : tiles) {
        const int vtile = tt.first, nth = tt.second;
        auto in_group = [&](const ugks_case *c) { return c->vtile == vtile && c->nth == nth; };
        ugks_batch::Group g;
        g.vtile = vtile;
        g.nth = nth;
        std::vector<int4> work;
        int max_grp = 0;
        for (int i = 0; i < n; ++i)
            if (in_group(b->cases[i])) {
                g.smem = std::max(g.smem, b->cases[i]->cfg.smem);
                max_grp = std::max(max_grp, b->cases[i]->n_groups);
            }
        // tile group outer, case, then patch innermost: consecutive CTAs work
        // on neighbouring patches of one case and group, as in the single-case grid
        for (int gr = 0; gr < max_grp; ++gr)
            for (int i = 0; i < n; ++i) {
                if (!in_group(b->cases[i]) || gr >= b->cases[i]->n_groups) continue;
                for (int pi = 0; pi < b->cases[i]->n_patches; ++pi) work.push_back(make_int4(i, pi, gr, 0));
            }
        cuda_ok(cudaMalloc((void **)&g.work, sizeof(int4) * std::max<size_t>(1, work.size())), "batch alloc");
        b->groups.push_back(g);      // owned by the batch from here on
        cuda_ok(cudaMemcpy(g.work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice), "batch upload");
        b->groups.back().nwork = (int)work.size();
        b->groups.back().grid = std::min((int)work.size(), ugks::gather_resident_ctas<T>(b->D, vtile, nth, g.smem));
    }
}

template <typename T>
void batch_capture(ugks_batch *b)
{
    cudaStream_t st = b->stream;
    const int n = (int)b->cases.size();
    const auto *dcs = (const ugks::DevCase<T> *)b->dcases;
    auto small = [&](int k) {
        cuda_ok(ugks::launch_small_batch<T>(b->D, k, dcs, b->small_off + (size_t)k * (n + 1), n, b->small_blocks[k],
                                            b->small_smem[k], st),
                "batched step kernel");
    };
    cuda_ok(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    for (int k = ugks::SK_PREP; k <= ugks::SK_WALL_SUM; ++k) small(k);
    for (const auto &g : b->groups)
        cuda_ok(ugks::launch_gather_batch<T>(b->D, g.vtile, g.nth, (const ugks::DevCase<T> *)b->dcases, g.work,
                                             g.nwork, g.grid, g.smem, st),
                "batched gather");
    small(ugks::SK_UPDATE_W);
    small(ugks::SK_COLLIDE);
    cuda_ok(cudaStreamEndCapture(st, &b->graph), "end capture");
    cuda_ok(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
}

void batch_free(ugks_batch *b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->dcases) cudaFree(b->dcases);
    for (auto &g : b->groups)
        if (g.work) cudaFree(g.work);
    if (b->small_off) cudaFree(b->small_off);
    for (auto e : b->case_ev)
        if (e) cudaEventDestroy(e);
    if (b->done) cudaEventDestroy(b->done);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

}  // namespace

extern "C" {

ugks_status ugks_batch_create(ugks_case *const *cases, int32_t n, void *stream, ugks_batch **out)
{
    if (!out) {
        g_err = "out must not be NULL";
        return UGKS_EINVAL;
    }
    *out = nullptr;
    std::unique_ptr<ugks_batch> b(new ugks_batch());
    ugks_status st = guard([&] {
        if (!cases || n <= 0) fail(UGKS_EINVAL, "a batch needs at least one case");
        for (int i = 0; i < n; ++i) {
            if (!cases[i]) fail(UGKS_EINVAL, "case %d is NULL", i);
            if (cases[i]->D != cases[0]->D || cases[i]->prec != cases[0]->prec)
                fail(UGKS_EINVAL, "case %d differs from case 0 in dimension or precision", i);
            for (int j = 0; j < i; ++j)
                if (cases[j] == cases[i]) fail(UGKS_EINVAL, "case %d appears twice", i);
            b->cases.push_back(cases[i]);
        }
        b->D = cases[0]->D;
        b->prec = cases[0]->prec;
        if (stream) {
            b->stream = (cudaStream_t)stream;
        } else {
            cuda_ok(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "stream");
            b->own_stream = true;
        }
        cuda_ok(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming), "event");
        b->case_ev.assign(b->cases.size(), nullptr);
        for (auto &e : b->case_ev) cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        // the cases' own streams must have finished their queued work
        for (auto *c : b->cases) cuda_ok(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize(), "sync");
        if (b->prec == UGKS_FP64) batch_build<double>(b.get());
        else batch_build<float>(b.get());
    });
    if (st != UGKS_OK) {
        std::string keep = g_err;
        batch_free(b.get());
        g_err = keep;
        return st;
    }
    *out = b.release();
    return UGKS_OK;
}

ugks_status ugks_batch_step(ugks_batch *b, int32_t nsteps)
{
    return guard([&] {
        if (!b) fail(UGKS_EINVAL, "batch is NULL");
        if (nsteps < 0) fail(UGKS_EINVAL, "nsteps must be >= 0");
        if (nsteps == 0) return;
        if (!b->exec) {
            if (b->prec == UGKS_FP64) batch_capture<double>(b);
            else batch_capture<float>(b);
        }
        // work queued on the cases' own streams comes first, and later calls
        // on a case (moments, state I/O, ugks_step) wait for the batch
        for (size_t i = 0; i < b->cases.size(); ++i) {
            cuda_ok(cudaEventRecord(b->case_ev[i], b->cases[i]->stream), "order");
            cuda_ok(cudaStreamWaitEvent(b->stream, b->case_ev[i], 0), "order");
        }
        for (int32_t s = 0; s < nsteps; ++s) cuda_ok(cudaGraphLaunch(b->exec, b->stream), "graph launch");
        cuda_ok(cudaEventRecord(b->done, b->stream), "order");
        for (auto *c : b->cases) {
            cuda_ok(cudaStreamWaitEvent(c->stream, b->done, 0), "order");
            c->step += nsteps;
            c->stepped = true;
        }
    });
}

void ugks_batch_destroy(ugks_batch *b)
{
    if (!b) return;
    batch_free(b);
    delete b;
}

void ugks_destroy(ugks_case *c)
{
    if (!c) return;
    for (auto e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->release();
    delete c;
}

}  // extern "C"

// ugks_server.cu -- continuous-batching serving loop over UGKS cases.
//
// Requests (a mesh, velocity grid and parameters with a residual tolerance
// and a step limit) arrive at given times.  Every tick the server
//   1. admits arrived requests, first fit in arrival order, while a slot is
//      free and the request's device footprint fits the remaining budget;
//   2. steps all running cases together: cases are grouped by (dimension,
//      precision) into ugks_batch objects (each kernel of a step launched once
//      for all cases of a group, CUDA-graph replay), rebuilt when the running
//      set changes;
//   3. reads every running case's residual and retires the converged ones
//      (max_m r_m < tol), those at their step limit and those with a numeric
//      failure, copying their macroscopic fields to host memory and freeing
//      their device memory.
// Latency of a request = completion time - arrival time on the server clock.
#include "../../include/ugks.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

namespace ugks {
void set_last_error(const std::string &msg);
}

namespace {

struct Request {
    uint64_t ticket = 0;
    // owned copies of the inputs
    int D = 0;
    int64_t C = 0, F = 0, Nv = 0;
    std::vector<double> cell_xc, cell_vol, face_n, face_S, face_xc, face_shift, u, w, wall_T, wall_U, prim_init;
    std::vector<int64_t> face_cells;
    std::vector<int32_t> face_type, face_tag;
    int32_t cart_n[3] = {0, 0, 0};
    ugks_params params{};
    bool has_shift = false, has_init = false;
    double tol = 0.0;
    int64_t max_steps = 0;
    size_t footprint = 0, device_bytes = 0;
    // progress
    int32_t state = UGKS_REQ_QUEUED;
    int32_t status = UGKS_OK;
    ugks_case *c = nullptr;
    int64_t steps = 0;
    double res[5] = {0, 0, 0, 0, 0};
    double t_arrive = 0, t_admit = -1, t_done = -1;
    std::vector<double> rho, U, T, q;   // results of a finished request
};

// Device bytes a case will hold, from its sizes (an upper bound of what
// ugks_create allocates: two copies of f, FP64 cell / face arrays and records).
size_t footprint_estimate(const Request &r)
{
    const int D = r.D, M = D + 2, NC = D == 2 ? 2 : 1;
    const size_t s = r.params.precision == UGKS_FP64 ? 8 : 4;
    const size_t nvp = (size_t)((r.Nv + 127) / 128 * 128);
    const size_t C = (size_t)r.C, F = (size_t)std::max<int64_t>(r.F, 1);
    size_t b = 2 * C * NC * nvp * s;                                   // f_cur, f_nxt
    b += C * (size_t)(M * 2 + D + D * M * 2 + 8) * 8;                  // W, q, prim, gradients, vol
    b += C * 2 * 12 * s + C * (nvp / 32 + 1) * M * s;                  // records, residual partials
    b += F * (size_t)(40 * s + 24 * s + 16 * s + (D * M + D + D + M + M + 5) * 8 + 60 * 8 + 64);
    b += 2 * F * (size_t)(8 * D + 24) + C * 64 + nvp * 64;             // geometry, LSQ, patches
    b += 2 * F * (size_t)(16 + 16 * s);                                // gather entries
    b += (size_t)64 * 256 * 40;                                        // allocation rounding
    return b + b / 8;
}

}  // namespace

struct ugks_server {
    std::mutex mu;
    size_t budget = 0, used = 0;
    int32_t max_slots = 0, steps_per_tick = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::chrono::steady_clock::time_point t0;
    uint64_t next_ticket = 1;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<Request *> queue, running;
    std::vector<ugks_batch *> batches;
    bool batches_stale = true;
    int64_t total_cvu = 0;      // cell-velocity updates executed

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

ugks_status set_err(ugks_status code, const std::string &m)
{
    ugks::set_last_error(m);
    return code;
}

void free_batches(ugks_server *s)
{
    for (auto *b : s->batches) ugks_batch_destroy(b);
    s->batches.clear();
    s->batches_stale = true;
}

ugks_status create_case(ugks_server *s, Request *r)
{
    ugks_mesh m{};
    m.dim = r->D;
    m.n_cells = r->C;
    m.n_faces = r->F;
    m.cell_xc = r->cell_xc.data();
    m.cell_vol = r->cell_vol.data();
    m.face_cells = r->face_cells.data();
    m.face_n = r->face_n.data();
    m.face_S = r->face_S.data();
    m.face_xc = r->face_xc.data();
    m.face_type = r->face_type.data();
    m.face_tag = r->face_tag.data();
    m.face_shift = r->has_shift ? r->face_shift.data() : nullptr;
    ugks_vgrid v{};
    v.dim = r->D;
    v.nv = r->Nv;
    v.u = r->u.data();
    v.w = r->w.data();
    for (int d = 0; d < 3; ++d) v.cart_n[d] = r->cart_n[d];
    ugks_params p = r->params;
    p.wall_T = r->wall_T.empty() ? nullptr : r->wall_T.data();
    p.wall_U = r->wall_U.empty() ? nullptr : r->wall_U.data();
    p.prim_init = r->has_init ? r->prim_init.data() : nullptr;
    // one velocity tile and one block size for every case of a precision, so
    // that all of them share one batched gather launch
    if (p.vtile == 0) p.vtile = p.precision == UGKS_FP64 ? 32 : 64;
    if (p.gather_threads == 0) p.gather_threads = 256;
    return ugks_create(&m, &v, &p, nullptr, (void *)s->stream, &r->c);
}

void retire(ugks_server *s, Request *r, int32_t state, ugks_status status)
{
    r->state = state;
    r->status = status;
    r->t_done = s->now();
    if (r->c) {
        r->rho.resize(r->C);
        r->U.resize(r->C * r->D);
        r->T.resize(r->C);
        r->q.resize(r->C * r->D);
        if (ugks_moments(r->c, r->rho.data(), r->U.data(), r->T.data(), r->q.data()) != UGKS_OK) {
            r->state = UGKS_REQ_FAILED;
            r->status = UGKS_ECUDA;
        }
        ugks_destroy(r->c);
        r->c = nullptr;
    }
    s->used -= std::min(s->used, r->footprint);
    s->running.erase(std::find(s->running.begin(), s->running.end(), r));
    s->batches_stale = true;
}

}  // namespace

extern "C" {

ugks_status ugks_server_create(size_t device_budget_bytes, int32_t max_slots, int32_t steps_per_tick, void *stream,
                               ugks_server **out)
{
    if (!out) return set_err(UGKS_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (device_budget_bytes == 0 || max_slots <= 0 || steps_per_tick <= 0)
        return set_err(UGKS_EINVAL, "server needs a positive budget, slot count and steps per tick");
    std::unique_ptr<ugks_server> s(new ugks_server());
    s->budget = device_budget_bytes;
    s->max_slots = max_slots;
    s->steps_per_tick = steps_per_tick;
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return set_err(UGKS_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
        s->own_stream = true;
    }
    s->t0 = std::chrono::steady_clock::now();
    *out = s.release();
    ugks::set_last_error("");
    return UGKS_OK;
}

ugks_status ugks_server_submit(ugks_server *s, const ugks_mesh *mesh, const ugks_vgrid *vgrid,
                               const ugks_params *params, double tol, int64_t max_steps, double t_arrive,
                               uint64_t *ticket)
{
    if (!s || !mesh || !vgrid || !params || !ticket) return set_err(UGKS_EINVAL, "NULL argument");
    if (!(tol > 0.0) || max_steps <= 0) return set_err(UGKS_EINVAL, "need tol > 0 and max_steps > 0");
    if (mesh->dim != 2 && mesh->dim != 3) return set_err(UGKS_EINVAL, "mesh dim must be 2 or 3");
    if (mesh->n_cells <= 0 || mesh->n_faces < 0 || vgrid->nv <= 0) return set_err(UGKS_EINVAL, "empty case");
    std::unique_ptr<Request> r(new Request());
    const int D = mesh->dim;
    const int64_t C = mesh->n_cells, F = mesh->n_faces, Nv = vgrid->nv;
    r->D = D;
    r->C = C;
    r->F = F;
    r->Nv = Nv;
    auto cp = [](auto &dst, const auto *src, size_t n) {
        if (src) dst.assign(src, src + n);
    };
    cp(r->cell_xc, mesh->cell_xc, C * D);
    cp(r->cell_vol, mesh->cell_vol, C);
    cp(r->face_cells, mesh->face_cells, 2 * F);
    cp(r->face_n, mesh->face_n, F * D);
    cp(r->face_S, mesh->face_S, F);
    cp(r->face_xc, mesh->face_xc, F * D);
    cp(r->face_type, mesh->face_type, F);
    cp(r->face_tag, mesh->face_tag, F);
    r->has_shift = mesh->face_shift != nullptr;
    cp(r->face_shift, mesh->face_shift, F * D);
    cp(r->u, vgrid->u, Nv * D);
    cp(r->w, vgrid->w, Nv);
    for (int d = 0; d < 3; ++d) r->cart_n[d] = vgrid->cart_n[d];
    r->params = *params;
    if (params->n_walls > 0) {
        cp(r->wall_T, params->wall_T, params->n_walls);
        cp(r->wall_U, params->wall_U, 3 * params->n_walls);
    }
    r->has_init = params->prim_init != nullptr;
    cp(r->prim_init, params->prim_init, C * (D + 2));
    if (r->cell_xc.size() != (size_t)(C * D) || r->face_cells.size() != (size_t)(2 * F) || r->u.size() != (size_t)(Nv * D))
        return set_err(UGKS_EINVAL, "mesh or velocity arrays missing");
    r->tol = tol;
    r->max_steps = max_steps;
    r->footprint = footprint_estimate(*r);
    std::lock_guard<std::mutex> lock(s->mu);
    if (r->footprint > s->budget) return set_err(UGKS_EINVAL, "request footprint exceeds the whole device budget");
    r->t_arrive = t_arrive >= 0.0 ? t_arrive : s->now();
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    std::stable_sort(s->queue.begin(), s->queue.end(),
                     [](const Request *a, const Request *b) { return a->t_arrive < b->t_arrive; });
    s->reqs[r->ticket] = std::move(r);
    ugks::set_last_error("");
    return UGKS_OK;
}

ugks_status ugks_server_tick(ugks_server *s, int32_t *n_running, int32_t *n_queued)
{
    if (!s) return set_err(UGKS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    const double t = s->now();
    // 1. admission: first fit in arrival order among arrived requests
    for (size_t i = 0; i < s->queue.size();) {
        Request *r = s->queue[i];
        if (r->t_arrive > t) break;
        if ((int)s->running.size() >= s->max_slots) break;
        if (s->used + r->footprint > s->budget) {
            ++i;
            continue;
        }
        s->queue.erase(s->queue.begin() + i);
        r->t_admit = s->now();
        ugks_status st = create_case(s, r);
        if (st != UGKS_OK) {
            r->state = UGKS_REQ_FAILED;
            r->status = st;
            r->t_done = s->now();
            continue;
        }
        r->state = UGKS_REQ_RUNNING;
        {
            ugks_info_t inf;
            if (ugks_info(r->c, &inf) == UGKS_OK) r->device_bytes = inf.device_bytes;
        }
        s->used += r->footprint;
        s->running.push_back(r);
        s->batches_stale = true;
    }
    // 2. batched steps of every running case
    if (!s->running.empty()) {
        if (s->batches_stale) {
            free_batches(s);
            std::map<std::string, std::vector<ugks_case *>> groups;
            for (Request *r : s->running) {
                ugks_info_t inf;
                ugks_info(r->c, &inf);
                groups[std::to_string(inf.dim) + "/" + std::to_string(inf.precision)].push_back(r->c);
            }
            for (auto &g : groups) {
                ugks_batch *b = nullptr;
                ugks_status st = ugks_batch_create(g.second.data(), (int32_t)g.second.size(), (void *)s->stream, &b);
                if (st != UGKS_OK) return st;
                s->batches.push_back(b);
            }
            s->batches_stale = false;
        }
        for (auto *b : s->batches) {
            ugks_status st = ugks_batch_step(b, s->steps_per_tick);
            if (st != UGKS_OK) return st;
        }
        // 3. residuals and retirement
        std::vector<Request *> done;
        for (Request *r : s->running) {
            r->steps += s->steps_per_tick;
            s->total_cvu += (int64_t)s->steps_per_tick * r->C * r->Nv;
            const int M = r->D + 2;
            ugks_status st = ugks_residual(r->c, r->res);
            if (st == UGKS_OK) st = ugks_check(r->c);
            double worst = 0.0;
            for (int m = 0; m < M; ++m) worst = std::max(worst, std::isfinite(r->res[m]) ? r->res[m] : INFINITY);
            if (st != UGKS_OK) {
                r->state = UGKS_REQ_FAILED;
                r->status = st;
                done.push_back(r);
            } else if (worst < r->tol) {
                r->state = UGKS_REQ_DONE;
                done.push_back(r);
            } else if (r->steps >= r->max_steps) {
                r->state = UGKS_REQ_DONE;
                r->status = UGKS_ENOTCONVERGED;
                done.push_back(r);
            }
        }
        if (!done.empty()) free_batches(s);
        for (Request *r : done) retire(s, r, r->state, (ugks_status)r->status);
    }
    if (n_running) *n_running = (int32_t)s->running.size();
    if (n_queued) *n_queued = (int32_t)s->queue.size();
    ugks::set_last_error("");
    return UGKS_OK;
}

ugks_status ugks_server_poll(ugks_server *s, uint64_t ticket, ugks_result *out)
{
    if (!s || !out) return set_err(UGKS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_err(UGKS_ENOTFOUND, "unknown ticket");
    const Request *r = it->second.get();
    out->state = r->state;
    out->status = r->status;
    out->steps = r->steps;
    for (int m = 0; m < 5; ++m) out->residual[m] = r->res[m];
    out->t_arrive = r->t_arrive;
    out->t_admit = r->t_admit;
    out->t_done = r->t_done;
    out->footprint_bytes = r->footprint;
    out->device_bytes = r->device_bytes;
    out->n_cells = r->C;
    out->nv = r->Nv;
    return UGKS_OK;
}

ugks_status ugks_server_moments(ugks_server *s, uint64_t ticket, double *rho, double *U, double *T, double *q)
{
    if (!s) return set_err(UGKS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_err(UGKS_ENOTFOUND, "unknown ticket");
    const Request *r = it->second.get();
    if (r->rho.empty()) return set_err(UGKS_EBUSY, "request has not finished");
    if (rho) std::memcpy(rho, r->rho.data(), r->rho.size() * sizeof(double));
    if (U) std::memcpy(U, r->U.data(), r->U.size() * sizeof(double));
    if (T) std::memcpy(T, r->T.data(), r->T.size() * sizeof(double));
    if (q) std::memcpy(q, r->q.data(), r->q.size() * sizeof(double));
    return UGKS_OK;
}

ugks_status ugks_server_stats(ugks_server *s, ugks_server_stats_t *out)
{
    if (!s || !out) return set_err(UGKS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out->device_budget = s->budget;
    out->device_used = s->used;
    out->n_running = (int32_t)s->running.size();
    out->n_queued = (int32_t)s->queue.size();
    out->total_cvu = s->total_cvu;
    out->clock = s->now();
    return UGKS_OK;
}

void ugks_server_destroy(ugks_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        free_batches(s);
        for (Request *r : s->running)
            if (r->c) ugks_destroy(r->c);
        s->running.clear();
    }
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"

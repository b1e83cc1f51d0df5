// Interactive re-filter service over a resident batch: continuous batching at
// iteration granularity (the serving line; the paper's goal of interactive,
// real-time inspection of faint structure, Sec. 1 and Sec. 6).
//
// Requests (cube, K, dt, n_iter, conductance) are queued by afd_serve_submit.
// afd_serve_step
//   * retires finished rounds (their CUDA events), timestamping requests whose
//     last iteration ran in them,
//   * admits queued requests while a descriptor slot and slot memory for their
//     output and scratch cubes fit the service's HBM budget,
//   * launches the next round: ONE launch of the batched streaming kernel per
//     conductance kind over the tiles of every active request, each request
//     advancing one iteration with its own coefficients and buffer roles.
// Requests that arrive while others are on the GPU join at the next round
// boundary; at most two rounds are in flight, so the host builds round k+1
// while the GPU runs round k (a request's last round is known when it is
// launched; only its completion time needs the GPU).  Every request runs the
// same per-voxel code on its own buffers, so its result is bit-identical to
// afd_filter_ex with t_block 1 on that cube alone.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <vector>

#include "afd_batch.h"
#include "afd_trace.h"
#include "afd_store.cuh"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum { REQ_QUEUED = 0, REQ_ACTIVE = 1, REQ_DONE = 2 };

struct Req {
    uint64_t ticket = 0;
    int cube = 0;
    int kind = 0;
    afd::Coef coef{};
    int n_iter = 0;
    int issued = 0;    // iterations launched
    int finished = 0;  // iterations whose round has completed
    int slot = -1;
    size_t off = 0, bytes = 0;  // slot memory: result at off, scratch at off + bytes/2
    double t_submit = 0.0, t_admit = 0.0, t_launch = 0.0, t_done = 0.0;
    int state = REQ_QUEUED;
};

struct Round {
    cudaEvent_t ev = nullptr;
    std::vector<uint64_t> tickets;
};

// First-fit allocator over [0, capacity).
struct Pool {
    std::map<size_t, size_t> free_;  // offset -> size
    void init(size_t cap)
    {
        free_.clear();
        if (cap)
            free_[0] = cap;
    }
    bool alloc(size_t n, size_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t at = it->first + n;
                free_.erase(it);
                if (rest)
                    free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

}  // namespace

struct afd_serve {
    afd_ctx *ctx = nullptr;
    afd_batch *cubes = nullptr;
    int cap = 0;  // descriptor slots (concurrently active requests)
    afd::BatchDesc *d_desc = nullptr;
    afd::BatchDesc *h_desc = nullptr;  // pinned
    int2 *d_roles[2] = {nullptr, nullptr};
    int2 *h_roles[2] = {nullptr, nullptr};
    int2 *d_list[2] = {nullptr, nullptr};
    int2 *h_list[2] = {nullptr, nullptr};
    size_t list_cap = 0;
    void *mem = nullptr;
    size_t mem_bytes = 0;
    Pool pool;
    std::vector<int> free_slots;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Req> reqs;
    std::deque<Round> inflight;
    cudaEvent_t evs[2] = {nullptr, nullptr};
    uint64_t next_ticket = 1;
    uint64_t round_no = 0;
};

namespace {

using namespace afd_host;

void free_serve(afd_serve *s)
{
    if (!s)
        return;
    for (int i = 0; i < 2; ++i) {
        if (s->evs[i])
            cudaEventDestroy(s->evs[i]);
        if (s->h_roles[i])
            cudaFreeHost(s->h_roles[i]);
        if (s->h_list[i])
            cudaFreeHost(s->h_list[i]);
    }
    if (s->h_desc)
        cudaFreeHost(s->h_desc);
    if (s->d_desc)
        cudaFree(s->d_desc);  // roles and lists live in the same allocation
    if (s->mem)
        cudaFree(s->mem);
    delete s;
}

size_t cube_bytes(const afd_batch *b, int c)
{
    const size_t es = static_cast<size_t>(afd::store_bytes(b->S));
    const size_t n = static_cast<size_t>(b->px[c] * b->ny[c] * b->nz[c]) * es;
    return (n + 255) / 256 * 256;
}

int64_t cube_tiles(const afd_batch *b, int c)
{
    const afd::BatchDesc &d = b->h_desc[c];
    return batch_cube_txy(b, c) * ((d.nz + d.zc - 1) / d.zc);
}

// Retire rounds whose event has completed (all of them, waiting, if `all`).
afd_status retire(afd_serve *s, bool wait_front)
{
    while (!s->inflight.empty()) {
        Round &r = s->inflight.front();
        cudaError_t e = wait_front ? cudaEventSynchronize(r.ev) : cudaEventQuery(r.ev);
        if (e == cudaErrorNotReady)
            break;
        if (e != cudaSuccess)
            return cuda_fail(s->ctx, e);
        wait_front = false;
        const double t = now_s();
        for (uint64_t tk : r.tickets) {
            auto it = s->reqs.find(tk);
            if (it == s->reqs.end())
                continue;
            Req &q = it->second;
            if (++q.finished == q.n_iter) {
                q.state = REQ_DONE;
                q.t_done = t;
            }
        }
        s->inflight.pop_front();
    }
    return AFD_OK;
}

afd_status admit(afd_serve *s)
{
    afd_batch *b = s->cubes;
    int box_w = 0, box_h = 0, hx = 0;
    afd::pm_stream_box(b->S, &box_w, &box_h, &hx);
    while (!s->queue.empty() && !s->free_slots.empty()) {
        Req &q = s->reqs[s->queue.front()];
        const size_t half = cube_bytes(b, q.cube);
        size_t off = 0;
        if (!s->pool.alloc(2 * half, &off))
            break;  // wait for memory: admission by free HBM
        const int slot = s->free_slots.back();
        s->free_slots.pop_back();
        q.slot = slot;
        q.off = off;
        q.bytes = 2 * half;
        afd::BatchDesc &d = s->h_desc[slot];
        d = b->h_desc[q.cube];  // role 0: the resident cube
        d.buf[1] = static_cast<char *>(s->mem) + off;
        d.buf[2] = static_cast<char *>(s->mem) + off + half;
        const int hxw = 16 / afd::store_bytes(b->S);
        for (int r = 1; r <= 2; ++r) {
            afd_status st = encode_pitched_map(s->ctx, &d.map[r], d.buf[r], b->S, box_w, box_h,
                                               d.nx, d.ny, d.nz, d.px);
            if (st == AFD_OK)
                st = encode_pitched_map(s->ctx, &d.mapw[r], d.buf[r], b->S, d.wtx + 2 * hxw,
                                        d.wty + 2, d.nx, d.ny, d.nz, d.px);
            if (st != AFD_OK)
                return st;
        }
        d.coef = q.coef;
        cudaError_t e = cudaMemcpyAsync(&s->d_desc[slot], &s->h_desc[slot], sizeof(d),
                                        cudaMemcpyHostToDevice, s->ctx->stream);
        if (e != cudaSuccess)
            return cuda_fail(s->ctx, e);
        q.state = REQ_ACTIVE;
        q.t_admit = now_s();
        s->queue.pop_front();
    }
    return AFD_OK;
}

afd_status launch_round(afd_serve *s, bool *launched)
{
    *launched = false;
    afd_batch *b = s->cubes;
    const int p = static_cast<int>(s->round_no & 1);
    int2 *list = s->h_list[p];
    int2 *roles = s->h_roles[p];
    // tiles grouped by conductance kind: [kind][...]
    std::vector<int2> by_kind[3];
    Round r;
    for (auto &kv : s->reqs) {
        Req &q = kv.second;
        if (q.state != REQ_ACTIVE || q.issued >= q.n_iter)
            continue;
        const int i = q.issued;
        if (i == 0)
            q.t_launch = now_s();
        const int dst = ((q.n_iter - 1 - i) & 1) ? 2 : 1;
        const int src = i == 0 ? 0 : (((q.n_iter - i) & 1) ? 2 : 1);
        roles[q.slot] = make_int2(src, dst);
        const int64_t nt = cube_tiles(b, q.cube);
        for (int64_t t = 0; t < nt; ++t)
            by_kind[q.kind].push_back(make_int2(q.slot, static_cast<int>(t)));
        q.issued++;
        r.tickets.push_back(q.ticket);
    }
    if (r.tickets.empty())
        return AFD_OK;
    size_t n = 0;
    size_t seg[3][2];
    for (int k = 0; k < 3; ++k) {
        seg[k][0] = n;
        seg[k][1] = by_kind[k].size();
        if (n + by_kind[k].size() > s->list_cap)
            return AFD_ENOMEM;  // cannot happen: sized for cap requests of the largest cube
        std::memcpy(list + n, by_kind[k].data(), by_kind[k].size() * sizeof(int2));
        n += by_kind[k].size();
    }
    cudaStream_t st = s->ctx->stream;
    cudaError_t e = cudaMemcpyAsync(s->d_roles[p], roles, s->cap * sizeof(int2),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_list[p], list, n * sizeof(int2), cudaMemcpyHostToDevice, st);
    const int64_t gmax = static_cast<int64_t>(s->ctx->sm_count) * batch_bps(b);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        if (!seg[k][1])
            continue;
        const int64_t nt = static_cast<int64_t>(seg[k][1]);
        const int64_t rounds = (nt + gmax - 1) / gmax;
        const int grid = static_cast<int>((nt + rounds - 1) / rounds);
        e = batch_launch(b, k, s->d_desc, s->d_list[p] + seg[k][0], s->d_roles[p], nt, 0, 1,
                         grid, nullptr, 0, false, s->ctx->d_err, st);
        s->ctx->launches++;
    }
    if (e == cudaSuccess) {
        r.ev = s->evs[p];
        e = cudaEventRecord(r.ev, st);
    }
    if (e != cudaSuccess)
        return cuda_fail(s->ctx, e);
    s->inflight.push_back(r);
    s->round_no++;
    *launched = true;
    return AFD_OK;
}

}  // namespace

extern "C" {

afd_status afd_serve_create(afd_ctx *ctx, afd_batch *cubes, size_t mem_bytes, int max_active,
                            afd_serve **out)
{
    if (!ctx || !cubes || !out || max_active < 1 || cubes->ctx != ctx)
        return AFD_EINVAL;
    *out = nullptr;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    afd_serve *s = new (std::nothrow) afd_serve();
    if (!s)
        return AFD_ENOMEM;
    s->ctx = ctx;
    s->cubes = cubes;
    s->cap = max_active;
    // room for either tile kind (the batch's kind may change later)
    int64_t maxt = 0;
    for (int c = 0; c < cubes->count; ++c) {
        const afd::BatchDesc &d = cubes->h_desc[c];
        const int64_t chunks = (d.nz + d.zc - 1) / d.zc;
        maxt = std::max(maxt, static_cast<int64_t>(d.tiles_x) * d.tiles_y * chunks);
        maxt = std::max(maxt, static_cast<int64_t>(d.wtiles_x) * d.wtiles_y * chunks);
    }
    s->list_cap = static_cast<size_t>(maxt) * max_active;
    const size_t dbytes = max_active * sizeof(afd::BatchDesc);
    const size_t rbytes = max_active * sizeof(int2);
    const size_t lbytes = s->list_cap * sizeof(int2);
    void *p = nullptr;
    if ((st = device_alloc(ctx, &p, dbytes + 2 * rbytes + 2 * lbytes + 1024)) != AFD_OK) {
        free_serve(s);
        return st;
    }
    s->d_desc = static_cast<afd::BatchDesc *>(p);
    char *q = static_cast<char *>(p) + (dbytes + 255) / 256 * 256;
    for (int i = 0; i < 2; ++i) {
        s->d_roles[i] = reinterpret_cast<int2 *>(q);
        q += (rbytes + 255) / 256 * 256;
        s->d_list[i] = reinterpret_cast<int2 *>(q);
        q += (lbytes + 255) / 256 * 256;
    }
    cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(&s->h_desc), dbytes);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMallocHost(reinterpret_cast<void **>(&s->h_roles[i]), rbytes);
        if (e == cudaSuccess)
            e = cudaMallocHost(reinterpret_cast<void **>(&s->h_list[i]), lbytes);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&s->evs[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        st = cuda_fail(ctx, e);
        free_serve(s);
        return st;
    }
    std::memset(static_cast<void *>(s->h_desc), 0, dbytes);
    for (int i = 0; i < 2; ++i)
        std::memset(s->h_roles[i], 0, rbytes);
    if (mem_bytes) {
        if ((st = device_alloc(ctx, &s->mem, mem_bytes)) != AFD_OK) {
            free_serve(s);
            return st;
        }
    }
    s->mem_bytes = mem_bytes;
    s->pool.init(mem_bytes);
    for (int i = max_active - 1; i >= 0; --i)
        s->free_slots.push_back(i);
    *out = s;
    return AFD_OK;
}

afd_status afd_serve_destroy(afd_serve *s)
{
    if (!s)
        return AFD_OK;
    set_device(s->ctx);
    cudaStreamSynchronize(s->ctx->stream);
    free_serve(s);
    return AFD_OK;
}

afd_status afd_serve_submit(afd_serve *s, int cube, float K, float dt, int n_iter,
                            afd_conductance cond, uint64_t *ticket)
{
    if (!s || !ticket || cube < 0 || cube >= s->cubes->count || n_iter < 1 ||
        !params_ok(nullptr, K, dt, n_iter, cond) || K == 0.0f)
        return AFD_EINVAL;
    const afd_batch *b = s->cubes;
    if (2 * cube_bytes(b, cube) > s->mem_bytes)
        return AFD_ENOMEM;  // could never be admitted
    Req q;
    q.ticket = s->next_ticket++;
    q.cube = cube;
    q.n_iter = n_iter;
    const float Ks = std::isinf(K) ? K : static_cast<float>(static_cast<double>(K) * b->units);
    q.coef = afd::make_coef(nullptr, Ks, dt, cond == AFD_COND_EXPONENTIAL, &q.kind);
    q.t_submit = now_s();
    s->reqs[q.ticket] = q;
    s->queue.push_back(q.ticket);
    *ticket = q.ticket;
    return AFD_OK;
}

afd_status afd_serve_step(afd_serve *s, int wait, int *active, int *queued)
{
    const afd_host::TraceRange trace_("afd_serve_step");
    if (!s)
        return AFD_EINVAL;
    afd_status st = set_device(s->ctx);
    if (st == AFD_OK)
        st = retire(s, false);
    if (st == AFD_OK)
        st = admit(s);
    bool launched = false;
    if (st == AFD_OK && s->inflight.size() < 2)
        st = launch_round(s, &launched);
    if (st == AFD_OK && wait && !launched && !s->inflight.empty())
        st = retire(s, true);
    if (st != AFD_OK)
        return st;
    int a = 0;
    for (auto &kv : s->reqs)
        a += kv.second.state == REQ_ACTIVE;
    if (active)
        *active = a;
    if (queued)
        *queued = static_cast<int>(s->queue.size());
    return AFD_OK;
}

afd_status afd_serve_poll(afd_serve *s, uint64_t ticket, int *state, double *latency_s)
{
    if (!s || !state)
        return AFD_EINVAL;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return AFD_EINVAL;
    *state = it->second.state;
    if (latency_s)
        *latency_s = it->second.state == REQ_DONE ? it->second.t_done - it->second.t_submit : -1.0;
    return AFD_OK;
}

afd_status afd_serve_times(afd_serve *s, uint64_t ticket, double *out4)
{
    if (!s || !out4)
        return AFD_EINVAL;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return AFD_EINVAL;
    const Req &q = it->second;
    out4[0] = q.t_submit;
    out4[1] = q.state >= REQ_ACTIVE ? q.t_admit : -1.0;
    out4[2] = q.issued > 0 ? q.t_launch : -1.0;
    out4[3] = q.state == REQ_DONE ? q.t_done : -1.0;
    return AFD_OK;
}

afd_status afd_serve_result(afd_serve *s, uint64_t ticket, void *dst)
{
    if (!s || !dst)
        return AFD_EINVAL;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return AFD_EINVAL;
    const Req &q = it->second;
    if (q.state != REQ_DONE)
        return AFD_EBUSY;
    afd_status st = set_device(s->ctx);
    if (st != AFD_OK)
        return st;
    const afd_batch *b = s->cubes;
    const size_t es = static_cast<size_t>(afd::store_bytes(b->S));
    const size_t width = static_cast<size_t>(b->nx[q.cube]) * es;
    const size_t pitch = static_cast<size_t>(b->px[q.cube]) * es;
    const size_t rows = static_cast<size_t>(b->ny[q.cube] * b->nz[q.cube]);
    cudaError_t e = cudaMemcpy2DAsync(dst, width, static_cast<char *>(s->mem) + q.off, pitch,
                                      width, rows, cudaMemcpyDefault, s->ctx->stream);
    return e == cudaSuccess ? AFD_OK : cuda_fail(s->ctx, e);
}

afd_status afd_serve_release(afd_serve *s, uint64_t ticket)
{
    if (!s)
        return AFD_EINVAL;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return AFD_EINVAL;
    Req &q = it->second;
    if (q.state != REQ_DONE)
        return AFD_EBUSY;
    s->pool.release(q.off, q.bytes);
    s->free_slots.push_back(q.slot);
    s->reqs.erase(it);
    return AFD_OK;
}

afd_status afd_serve_free_bytes(afd_serve *s, size_t *out)
{
    if (!s || !out)
        return AFD_EINVAL;
    size_t f = 0;
    for (auto &kv : s->pool.free_)
        f += kv.second;
    *out = f;
    return AFD_OK;
}

}  // extern "C"

// vp_server.cu -- continuous-batching request loop over the public C ABI.
//
// Host code only: a FIFO admission queue, a first-fit allocator over the
// caller's device arena (the HBM budget), and scheduling rounds that advance
// every admitted request together through one vp_batch. Each round takes a
// slice of steps; vp_batch_step_each lets every member stop at its own step
// count inside the slice (its tiles are skipped afterwards), so a nearly
// finished request does not shorten the others' slice. A request that
// finishes is retired at once (its moments and kept weights go to the caller)
// but its simulation stays a member of the batch, taking no steps, until the
// batch is rebuilt: rebuilds (and their graph capture) happen only when queued
// requests are admitted, not whenever a member leaves.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <vector>

#include "vlasov.h"

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

double now_s()
{
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

// first-fit allocator over [0, size)
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        free_[0] = size;
        used_ = 0;
        size_ = size;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = align_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = align_up(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
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
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, size_ = 0;
};

struct Req {
    vp_request r;
    std::vector<char> f0;
    vp_sim *sim = nullptr;
    size_t off = 0, bytes = 0;
    int done = 0;
    double t_submit = 0, t_admit = 0, t_finish = 0;
    bool batched = false;
    bool cancelled = false;   // retire at the start of the next round
    bool retired = false;     // result handed out; the simulation waits for the next rebuild
};

}  // namespace

struct vp_server {
    vp_server_opts o;
    char *arena;
    size_t arena_bytes;
    Arena alloc;
    std::deque<Req *> queue;
    std::vector<Req *> active;
    std::vector<vp_result> finished;
    std::map<uint64_t, std::vector<char>> kept_f;   // final weights (FP32 or FP64 bytes)
    std::map<uint64_t, int> kept_dtype;
    vp_batch *batch = nullptr;
    size_t batch_off = 0, batch_bytes = 0;
    bool dirty = true;
    char msg[512];
};

namespace {

vp_status sfail(vp_server *s, vp_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s->msg, sizeof(s->msg), fmt, ap);
    va_end(ap);
    return st;
}

void drop_batch(vp_server *s)
{
    if (s->batch) {
        vp_batch_sync(s->batch);
        vp_batch_destroy(s->batch);
        s->batch = nullptr;
        s->alloc.release(s->batch_off, s->batch_bytes);
    }
}

vp_status admit(vp_server *s)
{
    while (!s->queue.empty() && (int)s->active.size() < s->o.max_active) {   // (after reap)
        Req *q = s->queue.front();
        vp_opts o{q->r.precision, q->r.projection, VP_KERNEL_AUTO, 0, 0, 0, s->o.stream};
        size_t bytes = 0;
        vp_status st = vp_workspace_size(&q->r.grid, q->r.basis, &q->r.pusher, &o, &bytes);
        if (st != VP_OK) {
            // an invalid request finishes at once with its status
            vp_result res{};
            res.id = q->r.id;
            res.status = st;
            res.t_submit = q->t_submit;
            res.t_admit = res.t_finish = now_s();
            s->finished.push_back(res);
            s->queue.pop_front();
            delete q;
            continue;
        }
        if (s->alloc.used() + align_up(bytes) > s->o.budget_bytes) break;
        size_t off = 0;
        if (!s->alloc.alloc(bytes, &off)) break;   // first fit failed: wait for memory
        vp_sim *sim = nullptr;
        st = vp_create(&q->r.grid, q->r.basis, &q->r.pusher, &o, s->arena + off, bytes, &sim);
        if (st == VP_OK) st = vp_set_f(sim, q->f0.data(), q->r.f0_dtype,
                                       (size_t)q->r.grid.nx * q->r.grid.np);
        if (st != VP_OK) {
            if (sim) vp_destroy(sim);
            s->alloc.release(off, bytes);
            vp_result res{};
            res.id = q->r.id;
            res.status = st;
            res.t_submit = q->t_submit;
            res.t_admit = res.t_finish = now_s();
            s->finished.push_back(res);
            s->queue.pop_front();
            delete q;
            continue;
        }
        q->sim = sim;
        q->off = off;
        q->bytes = bytes;
        q->t_admit = now_s();
        std::vector<char>().swap(q->f0);   // the weights live on the device now
        s->queue.pop_front();
        s->active.push_back(q);
        s->dirty = true;
    }
    return VP_OK;
}

vp_status rebuild_batch(vp_server *s)
{
    drop_batch(s);
    std::vector<vp_sim *> sims;
    for (Req *q : s->active) {
        size_t b = 0;
        vp_sim *one = q->sim;
        q->batched = vp_batch_workspace_size(&one, 1, &b) == VP_OK;
        if (q->batched) sims.push_back(q->sim);
    }
    s->dirty = false;
    if (sims.empty()) return VP_OK;
    size_t bytes = 0;
    vp_status st = vp_batch_workspace_size(sims.data(), (int)sims.size(), &bytes);
    if (st != VP_OK) {
        // mixed basis/projection: step individually
        for (Req *q : s->active) q->batched = false;
        return VP_OK;
    }
    size_t off = 0;
    if (!s->alloc.alloc(bytes, &off)) {
        for (Req *q : s->active) q->batched = false;
        return VP_OK;
    }
    st = vp_batch_create(sims.data(), (int)sims.size(), s->o.stream, s->arena + off, bytes, &s->batch);
    if (st != VP_OK) {
        s->alloc.release(off, bytes);
        s->batch = nullptr;
        for (Req *q : s->active) q->batched = false;
        return VP_OK;
    }
    s->batch_off = off;
    s->batch_bytes = bytes;
    return VP_OK;
}

// Hand out the result of a finished or cancelled request (moments, and the final weights if
// kept). The simulation itself stays until reap() frees it.
void retire(vp_server *s, Req *q, bool cancelled)
{
    vp_result res{};
    res.id = q->r.id;
    res.batched = q->batched ? 1 : 0;
    res.status = vp_moments(q->sim, &res.moments);
    if (cancelled && res.status == VP_OK) res.status = VP_ERR_CANCELLED;
    if (!cancelled && q->r.keep_f && res.status == VP_OK) {
        const int dt = q->r.precision == VP_FP64 ? VP_FP64 : VP_FP32;
        const size_t n = (size_t)q->r.grid.nx * q->r.grid.np;
        std::vector<char> buf(n * (dt == VP_FP64 ? 8 : 4));
        res.status = vp_get_f(q->sim, buf.data(), dt, n);
        s->kept_f[q->r.id].swap(buf);
        s->kept_dtype[q->r.id] = dt;
    }
    res.t_submit = q->t_submit;
    res.t_admit = q->t_admit;
    res.t_finish = q->t_finish = now_s();
    s->finished.push_back(res);
    q->retired = true;
}

// Free the simulations of retired requests (the batch that holds them goes first).
void reap(vp_server *s)
{
    bool any = false;
    for (Req *q : s->active) any |= q->retired;
    if (!any) return;
    drop_batch(s);
    std::vector<Req *> keep;
    for (Req *q : s->active) {
        if (!q->retired) {
            keep.push_back(q);
            continue;
        }
        vp_destroy(q->sim);
        s->alloc.release(q->off, q->bytes);
        delete q;
    }
    s->active.swap(keep);
    s->dirty = true;
}

// requests cancelled while running leave before the round steps anything
void retire_cancelled(vp_server *s)
{
    for (Req *q : s->active)
        if (q->cancelled && !q->retired) retire(s, q, true);
}

int live_count(const vp_server *s)
{
    int n = 0;
    for (const Req *q : s->active) n += q->retired ? 0 : 1;
    return n;
}

// Whether the retired members hold most of the batch's nodes: their tiles are skipped in every
// launch, which costs a work-queue pass per tile; below half the nodes live, rebuild.
bool mostly_retired(const vp_server *s)
{
    if (!s->batch) return false;
    size_t live = 0, all = 0;
    for (const Req *q : s->active) {
        if (!q->batched) continue;
        const size_t n = (size_t)q->r.grid.nx * q->r.grid.np;
        all += n;
        if (!q->retired) live += n;
    }
    return all > 0 && 2 * live < all;
}

// Whether freeing the retired members would let the head of the queue in (by the budget and
// the active limit; an invalid head request is admitted, i.e. failed, at once).
bool head_would_fit(vp_server *s)
{
    if (s->queue.empty()) return false;
    const Req *q = s->queue.front();
    size_t freed = 0;
    int retired = 0;
    for (const Req *a : s->active)
        if (a->retired) {
            freed += align_up(a->bytes);
            ++retired;
        }
    if ((int)s->active.size() - retired >= s->o.max_active) return false;
    vp_opts o{q->r.precision, q->r.projection, VP_KERNEL_AUTO, 0, 0, 0, s->o.stream};
    size_t bytes = 0;
    if (vp_workspace_size(&q->r.grid, q->r.basis, &q->r.pusher, &o, &bytes) != VP_OK) return true;
    const size_t batch = s->batch ? align_up(s->batch_bytes) : 0;
    return s->alloc.used() - freed - batch + align_up(bytes) <= s->o.budget_bytes;
}

}  // namespace

extern "C" {

double vp_server_clock(void) { return now_s(); }

vp_status vp_server_create(const vp_server_opts *opts, void *arena, size_t arena_bytes,
                           vp_server **out)
{
    if (!opts || !out) return VP_ERR_ARG;
    *out = nullptr;
    if (!arena || (reinterpret_cast<uintptr_t>(arena) % kAlign)) return VP_ERR_WORKSPACE;
    vp_server *s = new (std::nothrow) vp_server();
    if (!s) return VP_ERR_ARG;
    s->o = *opts;
    if (s->o.slice_steps <= 0) s->o.slice_steps = 50;
    if (s->o.max_active <= 0) s->o.max_active = 4096;
    if (s->o.budget_bytes == 0 || s->o.budget_bytes > arena_bytes) s->o.budget_bytes = arena_bytes;
    s->arena = static_cast<char *>(arena);
    s->arena_bytes = arena_bytes;
    s->alloc.reset(arena_bytes);
    s->msg[0] = 0;
    *out = s;
    return VP_OK;
}

vp_status vp_server_submit(vp_server *s, const vp_request *req)
{
    if (!s || !req) return VP_ERR_ARG;
    if (!req->f0 || req->steps < 0 || req->grid.nx < 1 || req->grid.np < 1 ||
        (req->f0_dtype != VP_FP32 && req->f0_dtype != VP_FP64))
        return sfail(s, VP_ERR_ARG, "request %llu: bad weights, dtype or step count",
                     (unsigned long long)req->id);
    if ((req->pusher.kind == VP_PUSH_FEL_DKD && req->pusher.sigma2 != 0.0) ||
        req->pusher.kind == VP_PUSH_FEL_RK4)
        return sfail(s, VP_ERR_UNSUPPORTED,
                     "request %llu: FEL space charge and the RK4 integrator are not served in batches",
                     (unsigned long long)req->id);
    Req *q = new (std::nothrow) Req();
    if (!q) return VP_ERR_ARG;
    q->r = *req;
    const size_t n = (size_t)req->grid.nx * req->grid.np * (req->f0_dtype == VP_FP64 ? 8 : 4);
    q->f0.assign(static_cast<const char *>(req->f0), static_cast<const char *>(req->f0) + n);
    q->r.f0 = nullptr;
    q->t_submit = now_s();
    s->queue.push_back(q);
    return VP_OK;
}

vp_status vp_server_run(vp_server *s, int32_t rounds, int32_t *queued, int32_t *active)
{
    if (!s) return VP_ERR_ARG;
    std::vector<int32_t> limits;
    for (int r = 0; r < rounds; ++r) {
        retire_cancelled(s);
        // admission rebuilds the batch: free the retired members first, so that their memory
        // can take queued requests; with nothing queued they stay and the batch is kept
        if (live_count(s) == 0 || head_would_fit(s) || mostly_retired(s)) {
            reap(s);
            admit(s);
        }
        if (live_count(s) == 0) {
            reap(s);
            break;
        }
        if (s->dirty) rebuild_batch(s);
        const int slice = s->o.slice_steps;
        if (s->batch) {
            limits.clear();
            for (Req *q : s->active)
                if (q->batched) limits.push_back(q->retired ? 0 : q->r.steps - q->done);
            vp_status st = vp_batch_step_each(s->batch, slice, limits.data(), 1);
            if (st != VP_OK) return sfail(s, st, "batch step: %s", vp_batch_last_error(s->batch));
        }
        for (Req *q : s->active)
            if (!q->batched && !q->retired) {
                vp_status st = vp_step(q->sim, std::min(slice, q->r.steps - q->done));
                if (st != VP_OK) return sfail(s, st, "step: %s", vp_last_error(q->sim));
            }
        for (Req *q : s->active)
            if (!q->retired) q->done += std::min(slice, q->r.steps - q->done);
        // retire requests that reached their step count (their simulations stay until a reap)
        for (Req *q : s->active)
            if (!q->retired && q->done >= q->r.steps) retire(s, q, false);
    }
    if (queued) *queued = (int32_t)s->queue.size();
    if (active) *active = (int32_t)live_count(s);
    return VP_OK;
}

vp_status vp_server_cancel(vp_server *s, uint64_t id)
{
    if (!s) return VP_ERR_ARG;
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Req *q = *it;
        if (q->r.id != id) continue;
        vp_result res{};
        res.id = id;
        res.status = VP_ERR_CANCELLED;
        res.t_submit = q->t_submit;
        res.t_admit = res.t_finish = now_s();
        s->finished.push_back(res);
        s->queue.erase(it);
        delete q;
        return VP_OK;
    }
    for (Req *q : s->active)
        if (q->r.id == id && !q->cancelled && !q->retired) {
            q->cancelled = true;
            return VP_OK;
        }
    return sfail(s, VP_ERR_STATE, "request %llu is neither queued nor running",
                 (unsigned long long)id);
}

vp_status vp_server_poll(vp_server *s, vp_result *out, int32_t max, int32_t *count)
{
    if (!s || !count || (max > 0 && !out)) return VP_ERR_ARG;
    const int n = std::min<int>(max, (int)s->finished.size());
    for (int k = 0; k < n; ++k) out[k] = s->finished[k];
    s->finished.erase(s->finished.begin(), s->finished.begin() + n);
    *count = n;
    return VP_OK;
}

vp_status vp_server_take_f(vp_server *s, uint64_t id, void *host, int32_t dtype, size_t n)
{
    if (!s || !host) return VP_ERR_ARG;
    auto it = s->kept_f.find(id);
    if (it == s->kept_f.end()) return sfail(s, VP_ERR_STATE, "no kept weights for %llu",
                                            (unsigned long long)id);
    const int kd = s->kept_dtype[id];
    const size_t have = it->second.size() / (kd == VP_FP64 ? 8 : 4);
    if (n != have || (dtype != VP_FP32 && dtype != VP_FP64)) return VP_ERR_ARG;
    if (dtype == kd) {
        memcpy(host, it->second.data(), it->second.size());
    } else if (kd == VP_FP32) {
        const float *in = reinterpret_cast<const float *>(it->second.data());
        for (size_t k = 0; k < n; ++k) static_cast<double *>(host)[k] = in[k];
    } else {
        const double *in = reinterpret_cast<const double *>(it->second.data());
        for (size_t k = 0; k < n; ++k) static_cast<float *>(host)[k] = (float)in[k];
    }
    s->kept_f.erase(it);
    s->kept_dtype.erase(id);
    return VP_OK;
}

void vp_server_destroy(vp_server *s)
{
    if (!s) return;
    drop_batch(s);
    for (Req *q : s->active) {
        vp_destroy(q->sim);
        delete q;
    }
    for (Req *q : s->queue) delete q;
    delete s;
}

const char *vp_server_last_error(const vp_server *s) { return s ? s->msg : "NULL server"; }

}  // extern "C"

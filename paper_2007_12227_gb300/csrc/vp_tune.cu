// vp_tune.cu -- tile-shape autotuner of the C ABI (vlasov.h, "autotuning").
//
// The destination tile of the step kernel trades the redundant halo work of
// small tiles (the Lambda_x halo on both sides, the warm-up rows of the p solve,
// the guard bands) against the parallelism and shared-memory occupancy of large
// ones; which side wins depends on the mesh, the displacement per step (window
// height) and, in a batch, on the other simulations sharing the launch. The
// tuner therefore measures: it creates each candidate plan in the caller's
// workspace through the public calls, fills the density with a constant, and
// times steps with CUDA events on the caller's stream. The shape changes only
// which CTA computes a node, not the node's arithmetic, so any candidate gives
// the same step.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "vp_internal.h"

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxTimedSteps = 4096;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Shape {
    int tx, tp;
    int kernel;   // -1: the caller's opts.kernel
};

// the planner's default first, then widths x heights; batched runs use a shorter list. xpass:
// also the one-pass tiles with a separate x pass (no x halo, so a tile of width w walks about
// w + 12 source columns: widths up to 288 keep two CTAs per SM)
std::vector<Shape> candidate_shapes(int precision, bool batched, bool xpass = false)
{
    std::vector<Shape> c{{0, 0, -1}};
    static const int w32[] = {96, 128, 160, 192, 224, 256, 320, 384, 448};
    // heights include multiples of the warp counts of the common widths (60 = 6 x 10, 63 = 9 x 7),
    // which give each warp of the x solve the same number of window rows; which height wins
    // depends mostly on how the tile count fills the waves of 2 CTAs per SM, so it is measured
    static const int h32[] = {16, 32, 60, 63, 64, 128};
    static const int w64[] = {64, 96, 128, 192, 256};
    static const int h64[] = {16, 32, 64};
    static const int wb[] = {128, 160, 224, 320};
    static const int hb[] = {16, 32, 63, 64};
    static const int wx32[] = {128, 192, 224, 256, 288};
    static const int hx32[] = {32, 60, 63, 64, 128};
    static const int wx64[] = {64, 96, 128, 192, 256};
    static const int hx64[] = {16, 32, 64};
    if (batched) {
        for (int w : wb)
            for (int h : hb) c.push_back({w, h, -1});
    } else if (precision == VP_FP64) {
        for (int w : w64)
            for (int h : h64) c.push_back({w, h, -1});
    } else {
        for (int w : w32)
            for (int h : h32) c.push_back({w, h, -1});
    }
    if (xpass && !batched) {
        c.push_back({0, 0, VP_KERNEL_FUSED_XPASS});
        if (precision == VP_FP64) {
            for (int w : wx64)
                for (int h : hx64) c.push_back({w, h, VP_KERNEL_FUSED_XPASS});
        } else {
            for (int w : wx32)
                for (int h : hx32) c.push_back({w, h, VP_KERNEL_FUSED_XPASS});
        }
    }
    return c;
}

template <typename T>
__global__ void fill_kernel(T *f, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        f[i] = T(1);
}

std::mutex g_mu;
std::map<std::string, std::vector<vp_tune_result>> g_cache;

void put_bytes(std::string &k, const void *p, size_t n) { k.append(static_cast<const char *>(p), n); }

std::string cache_key(const vp_tune_config *cfgs, int count, const vp_opts *o, const vp_tune_opts &t)
{
    std::string k;
    for (int i = 0; i < count; ++i) {
        vp_tune_config c = cfgs[i];
        c.pad = 0;
        c.pusher.a0_re = 0.0;   // A0 only sets where the FEL field starts
        c.pusher.a0_im = 0.0;
        put_bytes(k, &c, sizeof(c));
    }
    const int32_t f[5] = {o->precision, o->projection, o->kernel, o->history_cap, t.batched};
    put_bytes(k, f, sizeof(f));
    return k;
}

size_t nodes_of(const vp_grid &g) { return (size_t)g.nx * (size_t)g.np; }

// a single configuration tuned for the planner's choice also times the separate-x-pass plan
// (batches take the one-pass kernel only)
bool tunes_xpass(const vp_opts *o, const vp_tune_opts &t) { return !t.batched && o->kernel == VP_KERNEL_AUTO; }

// Device time of one step: warm-up, then the better of two runs of k steps, k grown until a run
// lasts min_ms.
vp_status time_steps(const std::function<vp_status(int)> &step, cudaStream_t st, int min_steps,
                     double min_ms, double *ms_per_step)
{
    vp_status r = step(2);
    if (r != VP_OK) return r;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return VP_ERR_CUDA;
    }
    double best = INFINITY;
    int k = std::max(1, min_steps);
    for (int rep = 0; rep < 2 && r == VP_OK; ++rep) {
        for (;;) {
            float ms = 0.f;
            if (cudaEventRecord(e0, st) != cudaSuccess) { r = VP_ERR_CUDA; break; }
            r = step(k);
            if (r != VP_OK) break;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                r = VP_ERR_CUDA;
                break;
            }
            if (ms >= min_ms || k >= kMaxTimedSteps) {
                best = std::min(best, (double)ms / k);
                break;
            }
            const double grow = min_ms / std::max((double)ms, 1e-3);
            k = (int)std::min<double>(kMaxTimedSteps, std::max(2.0 * k, ceil(k * grow * 1.1)));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r == VP_OK) *ms_per_step = best;
    return r;
}

struct Need {
    std::vector<size_t> sim;   // per configuration: largest workspace over the candidates
    size_t batch = 0, fill = 0, total = 0;
};

vp_status workspace_need(const vp_tune_config *cfgs, int count, const vp_opts *opts,
                         const vp_tune_opts &t, Need *need)
{
    const std::vector<Shape> shapes = candidate_shapes(opts->precision, t.batched != 0, tunes_xpass(opts, t));
    const size_t sz = opts->precision == VP_FP64 ? 8 : 4;
    need->sim.assign(count, 0);
    size_t off = 0, maxn = 0;
    long long items = 0;
    for (int i = 0; i < count; ++i) {
        const vp_tune_config &c = cfgs[i];
        for (const Shape &s : shapes) {
            vp_opts o = *opts;
            o.tile_x = s.tx;
            o.tile_p = s.tp;
            if (s.kernel >= 0) o.kernel = s.kernel;
            size_t b = 0;
            if (vp_workspace_size(&c.grid, c.basis, &c.pusher, &o, &b) == VP_OK)
                need->sim[i] = std::max(need->sim[i], b);
        }
        if (need->sim[i] == 0) return VP_ERR_ARG;   // no candidate plans this configuration
        maxn = std::max(maxn, nodes_of(c.grid));
        // tiles are at least 64 wide (or the whole period) and 8 high
        items += (long long)((c.grid.nx + 63) / 64) * ((c.grid.np + 7) / 8);
        off += t.batched ? align_up(need->sim[i]) : 0;
    }
    if (!t.batched) off = align_up(need->sim[0]);
    if (t.batched) {
        if (items > (1LL << 30)) return VP_ERR_UNSUPPORTED;
        need->batch = vp::batch_workspace_bytes(count, (int)items);
        off += align_up(need->batch);
    }
    need->fill = maxn * sz;
    need->total = off + align_up(need->fill);
    return VP_OK;
}

}  // namespace

extern "C" {

vp_status vp_autotune_workspace_size(const vp_tune_config *cfgs, int32_t count, const vp_opts *opts,
                                     const vp_tune_opts *topts, size_t *bytes)
{
    if (!cfgs || count < 1 || !opts || !bytes) return VP_ERR_ARG;
    vp_tune_opts t{};
    if (topts) t = *topts;
    if (!t.batched && count != 1) return VP_ERR_ARG;
    if (t.batched && opts->precision != VP_FP32) return VP_ERR_UNSUPPORTED;
    Need need;
    vp_status st = workspace_need(cfgs, count, opts, t, &need);
    if (st == VP_OK) *bytes = need.total;
    return st;
}

void vp_autotune_clear_cache(void)
{
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache.clear();
}

vp_status vp_autotune(const vp_tune_config *cfgs, int32_t count, const vp_opts *opts,
                      const vp_tune_opts *topts, void *workspace, size_t workspace_bytes,
                      vp_tune_result *out)
{
    if (!cfgs || count < 1 || !opts || !out) return VP_ERR_ARG;
    vp_tune_opts t{};
    if (topts) t = *topts;
    if (!t.batched && count != 1) return VP_ERR_ARG;
    if (t.batched && opts->precision != VP_FP32) return VP_ERR_UNSUPPORTED;
    const int min_steps = t.min_steps > 0 ? t.min_steps : 3;
    const double min_ms = t.min_ms > 0.0 ? t.min_ms : 2.0;
    const std::string key = cache_key(cfgs, count, opts, t);
    if (t.use_cache) {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            for (int i = 0; i < count; ++i) {
                out[i] = it->second[i];
                out[i].from_cache = 1;
            }
            return VP_OK;
        }
    }
    Need need;
    vp_status st = workspace_need(cfgs, count, opts, t, &need);
    if (st != VP_OK) return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) || workspace_bytes < need.total)
        return VP_ERR_WORKSPACE;
    char *ws = static_cast<char *>(workspace);
    const cudaStream_t stream = static_cast<cudaStream_t>(opts->stream);

    // sim workspaces, then the batch tables, then the constant density
    std::vector<char *> sim_ws(count);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        sim_ws[i] = ws + off;
        off += align_up(t.batched ? need.sim[i] : need.sim[0]);
        if (!t.batched) break;
    }
    char *batch_ws = ws + off;
    if (t.batched) off += align_up(need.batch);
    void *fill = ws + off;
    {
        const size_t n = need.fill / (opts->precision == VP_FP64 ? 8 : 4);
        const int blocks = (int)std::min<size_t>(4096, (n + 255) / 256);
        if (opts->precision == VP_FP64)
            fill_kernel<double><<<std::max(blocks, 1), 256, 0, stream>>>(static_cast<double *>(fill), n);
        else
            fill_kernel<float><<<std::max(blocks, 1), 256, 0, stream>>>(static_cast<float *>(fill), n);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(stream) != cudaSuccess)
            return VP_ERR_CUDA;
    }

    const std::vector<Shape> shapes = candidate_shapes(opts->precision, t.batched != 0, tunes_xpass(opts, t));
    std::set<std::vector<int>> seen;
    std::vector<vp_tune_result> best(count);
    double best_ms = INFINITY, default_ms = NAN;
    int timed = 0, default_kernel = -1;
    for (const Shape &shape : shapes) {
        const bool is_default = shape.tx == 0 && shape.tp == 0 && shape.kernel < 0;
        std::vector<vp_sim *> sims;
        std::vector<vp_plan_info> info;
        bool ok = true;
        for (int i = 0; i < count && ok; ++i) {
            vp_opts o = *opts;
            o.tile_x = shape.tx;
            o.tile_p = shape.tp;
            if (shape.kernel >= 0) o.kernel = shape.kernel;
            vp_sim *s = nullptr;
            const size_t cap = t.batched ? need.sim[i] : need.sim[0];
            if (vp_create(&cfgs[i].grid, cfgs[i].basis, &cfgs[i].pusher, &o, sim_ws[i], cap, &s) != VP_OK) {
                ok = false;
                break;
            }
            sims.push_back(s);
            vp_plan_info pi;
            vp_plan(s, &pi);
            info.push_back(pi);
            if (t.batched && pi.kernel != VP_KERNEL_FUSED) ok = false;
        }
        if (ok && is_default) default_kernel = info[0].kernel;
        // only shapes of the default plan's kernel compete (and, next to the one-pass kernel, its
        // separate-x-pass form)
        if (ok && !t.batched && info[0].kernel != default_kernel &&
            !(default_kernel == VP_KERNEL_FUSED && info[0].kernel == VP_KERNEL_FUSED_XPASS))
            ok = false;
        std::vector<int> sig;
        for (const vp_plan_info &pi : info) {
            sig.push_back(pi.kernel);
            sig.push_back(pi.tile_x);
            sig.push_back(pi.tile_p);
            sig.push_back(pi.threads);
        }
        if (ok && !seen.insert(sig).second) ok = false;
        for (int i = 0; i < (int)sims.size() && ok; ++i)
            if (vp_set_f_device(sims[i], fill, opts->precision, nodes_of(cfgs[i].grid)) != VP_OK) ok = false;
        vp_batch *b = nullptr;
        if (ok && t.batched) {
            size_t bb = 0;
            if (vp_batch_workspace_size(sims.data(), count, &bb) != VP_OK || bb > need.batch ||
                vp_batch_create(sims.data(), count, opts->stream, batch_ws, need.batch, &b) != VP_OK)
                ok = false;
        }
        double ms = INFINITY;
        if (ok) {
            std::function<vp_status(int)> step;
            if (t.batched)
                step = [&](int n) { return vp_batch_step(b, n, 1); };
            else
                step = [&](int n) { return vp_step(sims[0], n); };
            if (time_steps(step, stream, min_steps, min_ms, &ms) != VP_OK) ms = INFINITY;
            else ++timed;
        }
        if (b) vp_batch_destroy(b);
        for (vp_sim *s : sims) vp_destroy(s);
        if (cudaStreamSynchronize(stream) != cudaSuccess) return VP_ERR_CUDA;
        if (!isfinite(ms)) continue;
        if (is_default) default_ms = ms;
        if (ms < best_ms) {
            best_ms = ms;
            for (int i = 0; i < count; ++i) {
                memset(&best[i], 0, sizeof(best[i]));
                best[i].tile_x = info[i].tile_x;
                best[i].tile_p = info[i].tile_p;
                best[i].kernel = info[i].kernel;
            }
        }
    }
    if (!isfinite(best_ms)) return VP_ERR_UNSUPPORTED;
    for (int i = 0; i < count; ++i) {
        best[i].candidates = timed;
        best[i].ms_per_step = best_ms;
        best[i].default_ms_per_step = default_ms;
        best[i].from_cache = 0;
        out[i] = best[i];
    }
    if (t.use_cache) {
        std::lock_guard<std::mutex> lock(g_mu);
        g_cache[key] = best;
    }
    return VP_OK;
}

}  // extern "C"

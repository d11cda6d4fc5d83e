// serve.cu -- the serving loop: continuous batching of IK requests.
//
// hjcd_submit copies a request (targets, seed counts, inline obstacles) into
// the server and returns at once.  One scheduler thread forms batches from
// the pending requests in arrival order and launches each batch as a packed
// solve (wave.cu) on one of max_inflight slots -- a stream with its own device
// workspace and pinned buffers -- as soon as a slot is free, so requests that
// arrive while others run are admitted as slots free up and their work
// overlaps on the device.  A batch is bounded by max_batch_requests, by
// max_batch_seeds and by the slot's share of the memory budget (admission by
// device memory); a request that cannot fit a slot alone fails with
// HJCD_ENOMEM.  When a batch's copies back to pinned memory complete, a host
// callback wakes the scheduler, which copies each request's results into its
// caller's buffers and marks it done.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <unordered_map>

#include "host.h"

namespace hjcd {

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Req {
    int64_t id = 0;
    int32_t robot_id = 0, scene_id = -1;
    std::vector<float> targets, sph, box, q_ref;
    std::vector<int32_t> spt;
    hjcd_solve_opts opts{};
    int cd_iters = -1, lm_iters = -1;
    int n = 0;  // robot DoF
    int64_t seeds = 0;
    float* out_q = nullptr;
    float* out_err = nullptr;
    int32_t* out_count = nullptr;
    hjcd_status status = HJCD_OK;
    bool done = false;
    int32_t batch_requests = 0;
    Clock::time_point t_submit, t_launch, t_done;
};

struct Slot {
    cudaStream_t s = nullptr;
    char* ws = nullptr;
    size_t ws_cap = 0;
    char* pin = nullptr;  // head image
    size_t pin_cap = 0;
    char* pout = nullptr;  // results
    size_t pout_cap = 0;
    std::vector<Req*> reqs;
    std::vector<WaveItem> items;
    WavePlan plan;
    bool busy = false;
    bool completed = false;  // set by the host callback (under the server mutex)
};

}  // namespace

struct Server {
    hjcd_ctx* ctx = nullptr;
    hjcd_params P{};
    int max_inflight = 2, max_requests = 256;
    int64_t max_seeds = 1 << 20;
    size_t slot_budget = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;       // scheduler: submit, completion, stop
    std::condition_variable cv_done;  // callers waiting for results
    std::deque<Req*> pending;
    std::unordered_map<int64_t, std::unique_ptr<Req>> reqs;
    int64_t next_id = 1;
    bool stopping = false;
    std::vector<Slot> slots;
    std::string fatal;  // first CUDA failure of the scheduler

    void run();
    void finish(Slot& sl);
    bool launch(Slot& sl, std::vector<Req*>& take);
};

namespace {

struct CbArg {
    Server* sv;
    Slot* sl;
};

void CUDART_CB on_batch_done(void* p) {
    CbArg* a = static_cast<CbArg*>(p);
    {
        std::lock_guard<std::mutex> lock(a->sv->mu);
        a->sl->completed = true;
    }
    a->sv->cv.notify_all();
    delete a;
}

// Capacities double when a batch outgrows them (each regrowth frees and allocates while other
// streams run, so it should be rare).
size_t grow(size_t need) { return align_up(2 * need, 1 << 20); }

// Initial capacities of a slot, allocated when the server starts so that the first requests do
// not pay for allocation: 256 MB of device workspace (or the slot's budget), 4 MB of pinned
// head image and of pinned results.
constexpr size_t kSlotWs0 = size_t(256) << 20;
constexpr size_t kSlotPin0 = size_t(4) << 20;

}  // namespace

// Copy a finished batch's results to the callers' buffers.
void Server::finish(Slot& sl) {
    int32_t flag = 0;
    const WavePlan& W = sl.plan;
    // the flag travels with the results (last 4 bytes of the result image)
    std::memcpy(&flag, sl.pout + W.q_total * 4 + W.e_total * 4 + (size_t)W.T * 4, sizeof flag);
    const auto now = Clock::now();
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        Req* r = sl.reqs[i];
        const int T = (int)(r->targets.size() / 7);
        const size_t nq = (size_t)T * r->opts.top_k * r->n, ne = (size_t)T * r->opts.top_k * 2;
        std::memcpy(r->out_q, sl.pout + 4 * (W.item_q0[i]), 4 * nq);
        std::memcpy(r->out_err, sl.pout + 4 * (W.q_total + W.item_e0[i]), 4 * ne);
        std::memcpy(r->out_count, sl.pout + 4 * (W.q_total + W.e_total + W.item_t0[i]), 4 * (size_t)T);
        r->status = flag ? HJCD_ETIMEOUT : HJCD_OK;
        r->t_done = now;
        r->batch_requests = (int32_t)sl.reqs.size();
    }
    std::lock_guard<std::mutex> lock(mu);
    for (Req* r : sl.reqs) r->done = true;
    sl.reqs.clear();
    sl.busy = false;
    sl.completed = false;
    cv_done.notify_all();
}

// Plan and launch a batch of `take` on slot sl; false (requests failed or
// returned to the queue) when it cannot be launched.
bool Server::launch(Slot& sl, std::vector<Req*>& take) {
    hjcd_ctx* c = ctx;
    std::vector<WaveItem> items(take.size());
    {
        std::lock_guard<std::mutex> api(c->api_mu);
        for (size_t i = 0; i < take.size(); ++i) {
            Req* r = take[i];
            WaveItem& it = items[i];
            it.rob = &c->robots[r->robot_id];
            it.scene = r->scene_id >= 0 ? &c->scenes[r->scene_id] : nullptr;
            it.inl_nsph = (int)(r->sph.size() / 4);
            it.inl_sph = r->sph.empty() ? nullptr : r->sph.data();
            it.inl_nbox = (int)(r->box.size() / 6);
            it.inl_box = r->box.empty() ? nullptr : r->box.data();
            it.T = (int)(r->targets.size() / 7);
            it.targets = r->targets.data();
            it.spt = r->spt.empty() ? nullptr : r->spt.data();
            it.n_samples = r->opts.n_samples;
            it.eps_pos = r->opts.eps_pos;
            it.eps_ori = r->opts.eps_ori;
            it.seed = r->opts.seed;
            it.top_k = r->opts.top_k;
            it.cd_iters = r->cd_iters;
            it.lm_iters = r->lm_iters;
            it.q_ref = r->q_ref.empty() ? nullptr : r->q_ref.data();
        }
        // a first plan (without outputs) sizes the batch
        for (auto& it : items) {
            static float dummy_f[1];
            static int32_t dummy_i[1];
            it.out_q = it.out_err = dummy_f;
            it.out_count = dummy_i;
        }
        WavePlan W;
        hjcd_status st = plan_wave(c, items.data(), (int)items.size(), P, &W);
        while (st == HJCD_OK && W.bytes > slot_budget && items.size() > 1) {
            // admission by memory: hand the last request back
            {
                std::lock_guard<std::mutex> lock(mu);
                pending.push_front(take.back());
            }
            take.pop_back();
            items.pop_back();
            st = plan_wave(c, items.data(), (int)items.size(), P, &W);
        }
        if (st == HJCD_OK && W.bytes > slot_budget) st = HJCD_ENOMEM;
        const size_t res_bytes = 4 * (size_t)(W.q_total + W.e_total + W.T) + 16;
        if (st == HJCD_OK && W.bytes > sl.ws_cap) {
            // stream-ordered: freeing the old workspace does not wait for the other streams
            if (sl.ws) cudaFreeAsync(sl.ws, sl.s);
            sl.ws = nullptr;
            sl.ws_cap = 0;
            const size_t cap = std::min(grow(W.bytes), std::max(slot_budget, W.bytes));
            if (cudaMallocAsync(reinterpret_cast<void**>(&sl.ws), cap, sl.s) != cudaSuccess) {
                cudaGetLastError();
                st = HJCD_ENOMEM;
            } else {
                sl.ws_cap = cap;
            }
        }
        if (st == HJCD_OK && W.head > sl.pin_cap) {
            if (sl.pin) cudaFreeHost(sl.pin);
            sl.pin = nullptr;
            sl.pin_cap = 0;
            if (cudaMallocHost(&sl.pin, grow(W.head)) != cudaSuccess) {
                cudaGetLastError();
                st = HJCD_ENOMEM;
            } else {
                sl.pin_cap = grow(W.head);
            }
        }
        if (st == HJCD_OK && res_bytes > sl.pout_cap) {
            if (sl.pout) cudaFreeHost(sl.pout);
            sl.pout = nullptr;
            sl.pout_cap = 0;
            if (cudaMallocHost(&sl.pout, grow(res_bytes)) != cudaSuccess) {
                cudaGetLastError();
                st = HJCD_ENOMEM;
            } else {
                sl.pout_cap = grow(res_bytes);
            }
        }
        if (st == HJCD_OK) {
            // results land in the slot's pinned buffer: q | err | count | flag
            for (size_t i = 0; i < items.size(); ++i) {
                items[i].out_q = reinterpret_cast<float*>(sl.pout) + W.item_q0[i];
                items[i].out_err = reinterpret_cast<float*>(sl.pout) + W.q_total + W.item_e0[i];
                items[i].out_count = reinterpret_cast<int32_t*>(sl.pout) + W.q_total + W.e_total + W.item_t0[i];
            }
            st = plan_wave(c, items.data(), (int)items.size(), P, &W);
        }
        const auto now = Clock::now();
        if (st == HJCD_OK) st = run_wave(c, W, items.data(), P, sl.ws, sl.pin, sl.s, nullptr);
        if (st == HJCD_OK) {
            cudaError_t e = cudaMemcpyAsync(sl.pout + 4 * (size_t)(W.q_total + W.e_total + W.T), wave_flag(W, sl.ws), 4,
                                            cudaMemcpyDeviceToHost, sl.s);
            if (e == cudaSuccess) e = cudaLaunchHostFunc(sl.s, on_batch_done, new CbArg{this, &sl});
            if (e != cudaSuccess) {
                fatal = cudaGetErrorString(e);
                st = HJCD_ECUDA;
            }
        }
        if (st != HJCD_OK) {
            std::lock_guard<std::mutex> lock(mu);
            for (Req* r : take) {
                r->status = st;
                r->t_launch = r->t_done = now;
                r->done = true;
            }
            cv_done.notify_all();
            return false;
        }
        for (Req* r : take) r->t_launch = now;
        sl.plan = std::move(W);
        sl.items = std::move(items);
    }
    sl.reqs = take;
    sl.busy = true;
    return true;
}

void Server::run() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
        // completed batches
        bool progressed = false;
        for (Slot& sl : slots) {
            if (sl.busy && sl.completed) {
                lock.unlock();
                finish(sl);
                lock.lock();
                progressed = true;
            }
        }
        // new batches on free slots
        for (Slot& sl : slots) {
            if (sl.busy || pending.empty()) continue;
            std::vector<Req*> take;
            int64_t seeds = 0;
            std::vector<int32_t> robots;
            while (!pending.empty() && (int)take.size() < max_requests) {
                Req* r = pending.front();
                if (!take.empty() && seeds + r->seeds > max_seeds) break;
                if (std::find(robots.begin(), robots.end(), r->robot_id) == robots.end()) {
                    if ((int)robots.size() == kMaxLaunchRobots) break;
                    robots.push_back(r->robot_id);
                }
                pending.pop_front();
                take.push_back(r);
                seeds += r->seeds;
            }
            lock.unlock();
            launch(sl, take);
            lock.lock();
            progressed = true;
        }
        if (progressed) continue;
        bool busy = false;
        for (Slot& sl : slots) busy = busy || sl.busy;
        if (stopping && pending.empty() && !busy) break;
        cv.wait(lock);
    }
}

void server_stop(hjcd_ctx* ctx) {
    Server* sv = ctx->server;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stopping = true;
    }
    sv->cv.notify_all();
    if (sv->th.joinable()) sv->th.join();
    for (Slot& sl : sv->slots) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        if (sl.ws) cudaFreeAsync(sl.ws, sl.s);
        if (sl.s) cudaStreamSynchronize(sl.s);
        if (sl.pin) cudaFreeHost(sl.pin);
        if (sl.pout) cudaFreeHost(sl.pout);
        if (sl.s) cudaStreamDestroy(sl.s);
    }
    cudaGetLastError();
    delete sv;
    ctx->server = nullptr;
}

}  // namespace hjcd

using namespace hjcd;

extern "C" {

hjcd_status hjcd_server_start(hjcd_ctx* ctx, const hjcd_server_opts* opts) {
    if (!ctx) return HJCD_EINVAL;
    if (ctx->server) return fail(ctx, HJCD_EINVAL, "a server is already running on this context");
    hjcd_server_opts o{};
    if (opts) o = *opts;
    if (o.max_inflight < 0 || o.max_inflight > 8) return fail(ctx, HJCD_EINVAL, "max_inflight outside [0, 8]");
    if (o.max_batch_requests < 0 || o.max_batch_requests > 4096)
        return fail(ctx, HJCD_EINVAL, "max_batch_requests outside [0, 4096]");
    if (o.max_batch_seeds < 0) return fail(ctx, HJCD_EINVAL, "max_batch_seeds < 0");
    hjcd_status st;
    if ((st = make_current(ctx))) return st;
    auto sv = std::make_unique<Server>();
    sv->ctx = ctx;
    if (o.params) sv->P = *o.params;
    else hjcd_default_params(&sv->P);
    if ((st = check_params(ctx, sv->P))) return st;
    sv->max_inflight = o.max_inflight ? o.max_inflight : 2;
    sv->max_requests = o.max_batch_requests ? o.max_batch_requests : 256;
    sv->max_seeds = o.max_batch_seeds ? o.max_batch_seeds : (int64_t)1 << 20;
    size_t budget = (size_t)o.memory_budget;
    if (!budget) {
        size_t fr = 0, tot = 0;
        HJCD_CUDA(ctx, cudaMemGetInfo(&fr, &tot));
        budget = fr / 4;
    }
    sv->slot_budget = budget / (size_t)sv->max_inflight;
    sv->slots.resize(sv->max_inflight);
    for (Slot& sl : sv->slots) {
        HJCD_CUDA(ctx, cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking));
        const size_t ws0 = std::min(kSlotWs0, sv->slot_budget);
        if (cudaMallocAsync(reinterpret_cast<void**>(&sl.ws), ws0, sl.s) == cudaSuccess) sl.ws_cap = ws0;
        if (cudaMallocHost(&sl.pin, kSlotPin0) == cudaSuccess) sl.pin_cap = kSlotPin0;
        if (cudaMallocHost(&sl.pout, kSlotPin0) == cudaSuccess) sl.pout_cap = kSlotPin0;
        cudaGetLastError();  // a failed reservation is retried, sized to the batch, when one needs it
    }
    Server* raw = sv.release();
    ctx->server = raw;
    raw->th = std::thread([raw] { raw->run(); });
    return HJCD_OK;
}

hjcd_status hjcd_server_stop(hjcd_ctx* ctx) {
    if (!ctx) return HJCD_EINVAL;
    if (!ctx->server) return fail(ctx, HJCD_EINVAL, "no server running");
    server_stop(ctx);
    return HJCD_OK;
}

hjcd_status hjcd_submit(hjcd_ctx* ctx, const hjcd_batch_item* req, int64_t* request_id) {
    if (!ctx || !req || !request_id) return HJCD_EINVAL;
    Server* sv = ctx->server;
    if (!sv) return fail(ctx, HJCD_EINVAL, "no server running");
    auto r = std::make_unique<Req>();
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> api(ctx->api_mu);
        if (req->robot_id < 0 || req->robot_id >= (int32_t)ctx->robots.size())
            return fail(ctx, HJCD_ENOTFOUND, "unknown robot id %d", req->robot_id);
        if (req->scene_id >= 0 && (req->scene_id >= (int32_t)ctx->scenes.size() || !ctx->scenes[req->scene_id].live))
            return fail(ctx, HJCD_ENOTFOUND, "unknown scene id %d", req->scene_id);
        r->n = ctx->robots[req->robot_id].P.n;
    }
    const int T = req->n_targets;
    const hjcd_solve_opts& o = req->opts;
    if (T < 1) return fail(ctx, HJCD_EINVAL, "a request needs n_targets >= 1");
    if (!req->targets_pq || !req->out_q || !req->out_err || !req->out_count)
        return fail(ctx, HJCD_EINVAL, "null buffer");
    if (pointer_kind(req->targets_pq) == 1 || pointer_kind(req->out_q) == 1 || pointer_kind(req->out_err) == 1 ||
        pointer_kind(req->out_count) == 1)
        return fail(ctx, HJCD_EINVAL, "served requests take host buffers");
    if (!(o.eps_pos > 0.0f) || !(o.eps_ori > 0.0f)) return fail(ctx, HJCD_EINVAL, "tolerances must be > 0");
    if (o.top_k < 1 || o.top_k > HJCD_MAX_TOPK) return fail(ctx, HJCD_EINVAL, "top_k outside [1, %d]", HJCD_MAX_TOPK);
    r->robot_id = req->robot_id;
    r->scene_id = req->scene_id;
    r->opts = o;
    r->opts.params = nullptr;
    r->opts.samples_per_target = nullptr;
    if (o.params) {
        hjcd_status st;
        if ((st = check_params(ctx, *o.params))) return st;
        r->cd_iters = o.params->cd_max_iters;
        r->lm_iters = o.params->lm_max_iters;
    }
    r->targets.assign(req->targets_pq, req->targets_pq + 7 * (size_t)T);
    if (req->q_current) {
        if (pointer_kind(req->q_current) == 1) return fail(ctx, HJCD_EINVAL, "served requests take host buffers");
        r->q_ref.assign(req->q_current, req->q_current + (size_t)T * r->n);
    }
    for (int t = 0; t < T; ++t) {
        const int m = o.samples_per_target ? o.samples_per_target[t] : o.n_samples;
        if (m < 1 || m > HJCD_MAX_SAMPLES) return fail(ctx, HJCD_EINVAL, "target %d: seed count %d outside [1, %d]", t, m, HJCD_MAX_SAMPLES);
        r->seeds += m;
    }
    if (o.samples_per_target) r->spt.assign(o.samples_per_target, o.samples_per_target + T);
    if (req->scene_id < 0) {
        if (req->n_inline_spheres < 0 || req->n_inline_boxes < 0 ||
            (req->n_inline_spheres > 0 && !req->inline_spheres) || (req->n_inline_boxes > 0 && !req->inline_boxes))
            return fail(ctx, HJCD_EINVAL, "bad inline scene");
        if (req->n_inline_spheres > 0)
            r->sph.assign(req->inline_spheres, req->inline_spheres + 4 * (size_t)req->n_inline_spheres);
        if (req->n_inline_boxes > 0) r->box.assign(req->inline_boxes, req->inline_boxes + 6 * (size_t)req->n_inline_boxes);
    }
    r->out_q = req->out_q;
    r->out_err = req->out_err;
    r->out_count = req->out_count;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        if (sv->stopping) return fail(ctx, HJCD_EINVAL, "the server is stopping");
        r->id = sv->next_id++;
        *request_id = r->id;
        sv->pending.push_back(r.get());
        sv->reqs.emplace(r->id, std::move(r));
    }
    sv->cv.notify_all();
    return HJCD_OK;
}

static void fill_info(const Req& r, hjcd_request_info* info) {
    if (!info) return;
    info->status = r.status;
    info->batch_requests = r.batch_requests;
    info->queued_ms = r.done ? ms_between(r.t_submit, r.t_launch) : 0.0;
    info->total_ms = r.done ? ms_between(r.t_submit, r.t_done) : 0.0;
}

hjcd_status hjcd_poll(hjcd_ctx* ctx, int64_t request_id, int32_t* done, hjcd_request_info* info) {
    if (!ctx || !done) return HJCD_EINVAL;
    Server* sv = ctx->server;
    if (!sv) return fail(ctx, HJCD_EINVAL, "no server running");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto f = sv->reqs.find(request_id);
    if (f == sv->reqs.end()) return fail(ctx, HJCD_ENOTFOUND, "unknown request %lld", (long long)request_id);
    Req& r = *f->second;
    *done = r.done ? 1 : 0;
    if (r.done) {
        fill_info(r, info);
        sv->reqs.erase(f);  // a finished request is reported once
    }
    return HJCD_OK;
}

hjcd_status hjcd_wait(hjcd_ctx* ctx, int64_t request_id, double timeout_s, hjcd_request_info* info) {
    if (!ctx) return HJCD_EINVAL;
    Server* sv = ctx->server;
    if (!sv) return fail(ctx, HJCD_EINVAL, "no server running");
    std::unique_lock<std::mutex> lock(sv->mu);
    auto f = sv->reqs.find(request_id);
    if (f == sv->reqs.end()) return fail(ctx, HJCD_ENOTFOUND, "unknown request %lld", (long long)request_id);
    Req* r = f->second.get();
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (!r->done) {
        if (sv->cv_done.wait_until(lock, until) == std::cv_status::timeout && !r->done)
            return fail(ctx, HJCD_ETIMEOUT, "request %lld not finished within %.3f s", (long long)request_id, timeout_s);
    }
    fill_info(*r, info);
    sv->reqs.erase(f);
    return HJCD_OK;
}

}  // extern "C"

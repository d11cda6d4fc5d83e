// graph.cu -- a packed batch captured once as a CUDA graph and replayed.
//
// The batch is planned and given its own device workspace and pinned image;
// one ordinary run (which also sets the kernels' attributes) precedes the
// capture of the same launch sequence on a private stream.  A replay copies
// the pinned image (robot and scene tables, target rows, offsets) and the
// targets from the callers' device buffers, runs every phase and copies each
// request's results to its device buffers, so changing the targets between
// replays re-solves the new poses with everything else fixed.
#include "host.h"

struct hjcd_graph {
    hjcd_ctx* ctx = nullptr;
    hjcd::WavePlan plan;
    std::vector<hjcd::WaveItem> items;
    hjcd_params P{};
    char* ws = nullptr;
    char* pin = nullptr;
    cudaStream_t s = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    cudaEvent_t done = nullptr;
    int64_t kernels = 0;  // kernel launches of one replay
};

using namespace hjcd;

namespace {

void release(hjcd_graph* G) {
    if (!G) return;
    if (G->s) cudaStreamSynchronize(G->s);
    if (G->x) cudaGraphExecDestroy(G->x);
    if (G->g) cudaGraphDestroy(G->g);
    if (G->done) cudaEventDestroy(G->done);
    if (G->s) cudaStreamDestroy(G->s);
    if (G->ws) cudaFree(G->ws);
    if (G->pin) cudaFreeHost(G->pin);
    cudaGetLastError();
    delete G;
}

}  // namespace

extern "C" {

hjcd_status hjcd_graph_create(hjcd_ctx* ctx, int n_items, const hjcd_batch_item* items, const hjcd_params* params,
                              hjcd_graph** out) {
    if (!ctx || !out) return HJCD_EINVAL;
    *out = nullptr;
    if (n_items < 1 || !items) return fail(ctx, HJCD_EINVAL, "a graph needs at least one item");
    hjcd_status st;
    hjcd_params P;
    if (params) P = *params;
    else hjcd_default_params(&P);
    if ((st = check_params(ctx, P))) return st;
    if ((st = make_current(ctx))) return st;
    auto* G = new hjcd_graph();
    G->ctx = ctx;
    G->P = P;
    G->items.resize(n_items);
    for (int i = 0; i < n_items; ++i) {
        const hjcd_batch_item& b = items[i];
        RobotRec* rob;
        SceneRec* sc;
        if ((st = check_robot(ctx, b.robot_id, &rob)) || (st = check_scene(ctx, b.scene_id, &sc))) {
            release(G);
            return st;
        }
        if (b.n_targets < 1 || pointer_kind(b.targets_pq) != 1 || pointer_kind(b.out_q) != 1 ||
            pointer_kind(b.out_err) != 1 || pointer_kind(b.out_count) != 1) {
            release(G);
            return fail(ctx, HJCD_EINVAL, "item %d: a graph takes n_targets >= 1 and device targets and outputs", i);
        }
        WaveItem& it = G->items[i];
        it.rob = rob;
        it.scene = sc;
        if (b.scene_id < 0) {
            it.inl_nsph = b.n_inline_spheres;
            it.inl_sph = b.inline_spheres;
            it.inl_nbox = b.n_inline_boxes;
            it.inl_box = b.inline_boxes;
        }
        it.T = b.n_targets;
        it.targets = b.targets_pq;
        it.spt = b.opts.samples_per_target;
        it.n_samples = b.opts.n_samples;
        it.eps_pos = b.opts.eps_pos;
        it.eps_ori = b.opts.eps_ori;
        it.seed = b.opts.seed;
        it.top_k = b.opts.top_k;
        it.cd_iters = b.opts.params ? b.opts.params->cd_max_iters : -1;
        it.lm_iters = b.opts.params ? b.opts.params->lm_max_iters : -1;
        it.out_q = b.out_q;
        it.out_err = b.out_err;
        it.out_count = b.out_count;
        if (b.q_current && pointer_kind(b.q_current) != 1) {
            release(G);
            return fail(ctx, HJCD_EINVAL, "item %d: a graph takes q_current in device memory", i);
        }
        it.q_ref = b.q_current;
    }
    if ((st = plan_wave(ctx, G->items.data(), n_items, P, &G->plan))) {
        release(G);
        return st;
    }
    // the inline obstacles and seed counts are read while the image is filled, here; the
    // image itself stays in the graph's pinned buffer for every replay
    const WavePlan& W = G->plan;
    cudaError_t e = cudaMalloc(&G->ws, W.bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&G->pin, W.head);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G->s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(G);
        return fail(ctx, e == cudaErrorMemoryAllocation ? HJCD_ENOMEM : HJCD_ECUDA, "graph buffers: %s",
                    cudaGetErrorString(e));
    }
    // one ordinary run, then the capture of the same sequence
    if ((st = run_wave(ctx, W, G->items.data(), P, G->ws, G->pin, G->s, nullptr))) {
        release(G);
        return st;
    }
    e = cudaStreamSynchronize(G->s);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(G->s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        release(G);
        return fail(ctx, HJCD_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    const int64_t k0 = ctx->launches.load();
    st = run_wave(ctx, W, G->items.data(), P, G->ws, G->pin, G->s, nullptr);
    G->kernels = ctx->launches.load() - k0;
    ctx->launches -= G->kernels;  // captured, not launched
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(G->s, &g);
    G->g = g;
    if (st == HJCD_OK && e == cudaSuccess) e = cudaGraphInstantiate(&G->x, g, 0);
    if (st != HJCD_OK || e != cudaSuccess) {
        cudaGetLastError();
        release(G);
        return st != HJCD_OK ? st : fail(ctx, HJCD_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    // the inline arrays and seed counts were copied into the image: the items must not point at them any more
    for (auto& it : G->items) {
        it.inl_sph = it.inl_box = nullptr;
        it.spt = nullptr;
    }
    *out = G;
    return HJCD_OK;
}

hjcd_status hjcd_graph_launch(hjcd_graph* G, void* stream) {
    if (!G) return HJCD_EINVAL;
    hjcd_ctx* ctx = G->ctx;
    hjcd_status st;
    if ((st = make_current(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    HJCD_CUDA(ctx, cudaGraphLaunch(G->x, s));
    HJCD_CUDA(ctx, cudaEventRecord(G->done, s));
    ctx->launches += G->kernels;
    return HJCD_OK;
}

hjcd_status hjcd_graph_check(hjcd_graph* G) {
    if (!G) return HJCD_EINVAL;
    hjcd_ctx* ctx = G->ctx;
    HJCD_CUDA(ctx, cudaEventSynchronize(G->done));
    int32_t flag = 0;
    HJCD_CUDA(ctx, cudaMemcpy(&flag, wave_flag(G->plan, G->ws), sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) return fail(ctx, HJCD_ETIMEOUT, "collision kernel: staging wait ran out");
    return HJCD_OK;
}

void hjcd_graph_destroy(hjcd_graph* G) {
    if (!G) return;
    cudaSetDevice(G->ctx->device);
    release(G);
}

}  // extern "C"

// tune.cu -- the autotuner: launch configuration and iteration caps from
// timed solves of a calibration batch.
//
// Step 1 times the batch under every launch configuration (PO-CCD candidates
// per CTA x PJ-IK warps per CTA; results do not depend on it) and keeps the
// fastest.  Step 2 sweeps the PO-CCD sweep count and the PJ-IK iteration cap
// and keeps the fastest pair whose success rate (a collision-free solution
// within the request's tolerances) is within success_tol of the best rate
// seen.  Each configuration: one warm-up solve, then the median of `repeats`
// solves timed with events on a private stream.
#include <algorithm>
#include <cstring>

#include "host.h"

using namespace hjcd;

namespace {

struct Trial {
    double ms = 0.0;
    double success = 0.0;
};

}  // namespace

extern "C" {

hjcd_status hjcd_set_launch_config(hjcd_ctx* ctx, int32_t ccd_block, int32_t lm_warps) {
    if (!ctx) return HJCD_EINVAL;
    if (ccd_block != 64 && ccd_block != 128 && ccd_block != 256)
        return fail(ctx, HJCD_EINVAL, "ccd_block must be 64, 128 or 256");
    if (lm_warps != 2 && lm_warps != 4 && lm_warps != 8) return fail(ctx, HJCD_EINVAL, "lm_warps must be 2, 4 or 8");
    ctx->ccd_block = ccd_block;
    ctx->lm_warps = lm_warps;
    return HJCD_OK;
}

hjcd_status hjcd_autotune(hjcd_ctx* ctx, int n_items, const hjcd_batch_item* items, const hjcd_params* base,
                          float success_tol, int32_t repeats, hjcd_params* tuned, hjcd_tune_report* report) {
    if (!ctx || !tuned) return HJCD_EINVAL;
    if (n_items < 1 || !items) return fail(ctx, HJCD_EINVAL, "the calibration batch needs at least one item");
    if (!(success_tol >= 0.0f)) return fail(ctx, HJCD_EINVAL, "success_tol must be >= 0");
    if (repeats < 1) repeats = 3;
    hjcd_status st;
    hjcd_params P0;
    if (base) P0 = *base;
    else hjcd_default_params(&P0);
    if ((st = check_params(ctx, P0))) return st;
    if ((st = make_current(ctx))) return st;

    // the calibration batch with outputs in one device buffer of the tuner
    std::vector<WaveItem> w(n_items);
    int64_t nq = 0, ne = 0, nc = 0;
    for (int i = 0; i < n_items; ++i) {
        const hjcd_batch_item& b = items[i];
        RobotRec* rob;
        SceneRec* sc;
        if ((st = check_robot(ctx, b.robot_id, &rob)) || (st = check_scene(ctx, b.scene_id, &sc))) return st;
        if (b.n_targets < 1 || !b.targets_pq) return fail(ctx, HJCD_EINVAL, "item %d: no targets", i);
        WaveItem& it = w[i];
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
        it.top_k = 1;
        nq += (int64_t)it.T * rob->P.n;
        ne += (int64_t)it.T * 2;
        nc += it.T;
    }
    char* dout = nullptr;
    const size_t bytes = 4 * (size_t)(nq + ne + nc);
    HJCD_CUDA(ctx, cudaMalloc(&dout, bytes));
    std::vector<float> h_err(ne);
    std::vector<int32_t> h_cnt(nc);
    int64_t oq = 0, oe = 0, oc = 0;
    for (auto& it : w) {
        it.out_q = reinterpret_cast<float*>(dout) + oq;
        it.out_err = reinterpret_cast<float*>(dout) + nq + oe;
        it.out_count = reinterpret_cast<int32_t*>(dout) + nq + ne + oc;
        oq += (int64_t)it.T * it.rob->P.n;
        oe += (int64_t)it.T * 2;
        oc += it.T;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int32_t blk0 = ctx->ccd_block, warps0 = ctx->lm_warps;
    auto cleanup = [&]() {
        if (s) cudaStreamSynchronize(s);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        cudaFree(dout);
        cudaGetLastError();
    };
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return fail(ctx, HJCD_ECUDA, "autotune: stream or event creation failed");
    }
    int trials = 0;
    // one configuration: warm-up, `repeats` timed solves (median), success of the last
    auto run = [&](const hjcd_params& P, Trial* out) -> hjcd_status {
        WavePlan W;
        hjcd_status r;
        if ((r = plan_wave(ctx, w.data(), n_items, P, &W))) return r;
        if ((r = ensure_ws(ctx, W.bytes))) return r;
        if ((r = ensure_pin(ctx, W.head))) return r;
        std::vector<double> ms;
        for (int k = 0; k <= repeats; ++k) {
            HJCD_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ws_free, 0));
            HJCD_CUDA(ctx, cudaEventRecord(e0, s));
            if ((r = run_wave(ctx, W, w.data(), P, ctx->ws, ctx->pin, s, nullptr))) return r;
            HJCD_CUDA(ctx, cudaEventRecord(e1, s));
            HJCD_CUDA(ctx, cudaEventRecord(ctx->pin_free, s));
            HJCD_CUDA(ctx, cudaEventRecord(ctx->ws_free, s));
            HJCD_CUDA(ctx, cudaEventSynchronize(e1));
            float t = 0.0f;
            HJCD_CUDA(ctx, cudaEventElapsedTime(&t, e0, e1));
            if (k > 0) ms.push_back(t);
        }
        std::sort(ms.begin(), ms.end());
        out->ms = ms[ms.size() / 2];
        HJCD_CUDA(ctx, cudaMemcpy(h_err.data(), dout + 4 * nq, 4 * ne, cudaMemcpyDeviceToHost));
        HJCD_CUDA(ctx, cudaMemcpy(h_cnt.data(), dout + 4 * (nq + ne), 4 * nc, cudaMemcpyDeviceToHost));
        int64_t ok = 0, t0 = 0;
        for (const auto& it : w) {
            for (int t = 0; t < it.T; ++t) {
                const int64_t g = t0 + t;
                ok += h_cnt[g] > 0 && h_err[2 * g] <= it.eps_pos && h_err[2 * g + 1] <= it.eps_ori;
            }
            t0 += it.T;
        }
        out->success = (double)ok / (double)nc;
        ++trials;
        return HJCD_OK;
    };

    // step 1: launch configuration
    static const int blocks[3] = {64, 128, 256}, warps[3] = {2, 4, 8};
    int best_b = blk0, best_w = warps0;
    double best_ms = 1e300;
    for (int b : blocks)
        for (int wp : warps) {
            ctx->ccd_block = b;
            ctx->lm_warps = wp;
            Trial tr;
            if ((st = run(P0, &tr))) {
                ctx->ccd_block = blk0;
                ctx->lm_warps = warps0;
                cleanup();
                return st;
            }
            if (tr.ms < best_ms) {
                best_ms = tr.ms;
                best_b = b;
                best_w = wp;
            }
        }
    ctx->ccd_block = best_b;
    ctx->lm_warps = best_w;

    // step 2: iteration caps
    static const int cds[6] = {8, 12, 16, 24, 32, 48}, lms[5] = {8, 12, 16, 20, 30};
    std::vector<std::pair<hjcd_params, Trial>> res;
    double best_succ = 0.0;
    for (int cd : cds)
        for (int lm : lms) {
            hjcd_params P = P0;
            P.cd_max_iters = cd;
            P.lm_max_iters = lm;
            Trial tr;
            if ((st = run(P, &tr))) {
                cleanup();
                return st;
            }
            res.emplace_back(P, tr);
            best_succ = std::max(best_succ, tr.success);
        }
    const std::pair<hjcd_params, Trial>* pick = nullptr;
    for (const auto& r : res)
        if (r.second.success >= best_succ - success_tol && (!pick || r.second.ms < pick->second.ms)) pick = &r;
    *tuned = pick->first;
    if (report) {
        report->ccd_block = best_b;
        report->lm_warps = best_w;
        report->cd_max_iters = pick->first.cd_max_iters;
        report->lm_max_iters = pick->first.lm_max_iters;
        report->success_rate = (float)pick->second.success;
        report->best_success_rate = (float)best_succ;
        report->ms = pick->second.ms;
        report->trials = trials;
    }
    cleanup();
    return HJCD_OK;
}

}  // extern "C"

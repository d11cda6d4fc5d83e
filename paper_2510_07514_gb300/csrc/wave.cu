// wave.cu -- one packed solve over several requests (robots, scenes, seed
// counts and tolerances may all differ): Alg. 2 as one launch per phase over
// every target of the wave.
//
// Every target row carries its robot and scene (rows of the wave's tables),
// its request's tolerances, random-stream key and target index inside the
// request, so a request's results do not depend on what it is packed with.
//
// Device layout of a wave (one workspace):
//   head  robot kinematic tables | robot collision descriptors | scene
//         descriptors | target rows | seed offsets m_off | candidate offsets
//         b_off | output offsets | target poses [T][7] | inline obstacles
//         (written in pinned host memory, copied with one transfer)
//   PO-CCD joint vectors [n_max][CM] and scores [CM]
//   PJ-IK joint vectors [n_max][CB], scores, errors, collision verdicts [CB]
//   outputs (each request's block as it wants it), queue head, error flag
#include <algorithm>
#include <cmath>
#include <cstring>

#include "host.h"

namespace hjcd {

hjcd_status plan_wave(hjcd_ctx* ctx, const WaveItem* items, int n_items, const hjcd_params& P, WavePlan* out) {
    WavePlan& W = *out;
    W = WavePlan{};
    W.n_items = n_items;
    W.item_robot.resize(n_items);
    W.item_scene.resize(n_items);
    W.item_t0.resize(n_items);
    W.item_q0.resize(n_items);
    W.item_e0.resize(n_items);
    W.dev_tgt.resize(n_items);
    W.dev_q.resize(n_items);
    W.dev_e.resize(n_items);
    W.dev_c.resize(n_items);
    W.dev_ref.resize(n_items);
    size_t inl_bytes = 0;
    for (int i = 0; i < n_items; ++i) {
        const WaveItem& it = items[i];
        if (!it.rob) return fail(ctx, HJCD_EINVAL, "item %d: no robot", i);
        if (it.T < 0) return fail(ctx, HJCD_EINVAL, "item %d: n_targets < 0", i);
        if (it.T > 0 && (!it.targets || !it.out_q || !it.out_err || !it.out_count))
            return fail(ctx, HJCD_EINVAL, "item %d: null buffer", i);
        if (!(it.eps_pos > 0.0f) || !(it.eps_ori > 0.0f)) return fail(ctx, HJCD_EINVAL, "item %d: tolerances must be > 0", i);
        if (it.top_k < 1 || it.top_k > HJCD_MAX_TOPK) return fail(ctx, HJCD_EINVAL, "item %d: top_k outside [1, %d]", i, HJCD_MAX_TOPK);
        if (it.inl_nsph < 0 || it.inl_nbox < 0 || (it.inl_nsph > 0 && !it.inl_sph) || (it.inl_nbox > 0 && !it.inl_box))
            return fail(ctx, HJCD_EINVAL, "item %d: bad inline scene", i);
        if (it.cd_iters > 32767 || it.lm_iters > 32767) return fail(ctx, HJCD_EINVAL, "item %d: iteration caps above 32767", i);
        // robot table of the wave
        int r = -1;
        for (int k = 0; k < (int)W.robots.size(); ++k)
            if (W.robots[k] == it.rob) r = k;
        if (r < 0) {
            if ((int)W.robots.size() == kMaxLaunchRobots)
                return fail(ctx, HJCD_EINVAL, "more than %d distinct robots in one batch", kMaxLaunchRobots);
            r = (int)W.robots.size();
            W.robots.push_back(it.rob);
        }
        W.item_robot[i] = r;
        // scene table: resident scenes once each, inline scenes one per item
        int sidx = -1;
        if (it.scene) {
            for (int k = 0; k < (int)W.scenes.size(); ++k)
                if (W.scenes[k].res == it.scene) sidx = k;
            if (sidx < 0) {
                sidx = (int)W.scenes.size();
                W.scenes.push_back({it.scene, i, 0, it.scene->dev.n_sph, it.scene->dev.n_box});
            }
        } else if (it.inl_nsph + it.inl_nbox > 0) {
            for (int k = 0; k < it.inl_nsph; ++k)
                if (!(it.inl_sph[4 * k + 3] > 0.0f)) return fail(ctx, HJCD_EINVAL, "item %d: obstacle sphere %d radius must be > 0", i, k);
            for (int k = 0; k < it.inl_nbox; ++k) {
                const float* b = it.inl_box + 6 * k;
                if (!(b[0] <= b[3] && b[1] <= b[4] && b[2] <= b[5])) return fail(ctx, HJCD_EINVAL, "item %d: box %d lo > hi", i, k);
            }
            sidx = (int)W.scenes.size();
            W.scenes.push_back({nullptr, i, inl_bytes, it.inl_nsph, it.inl_nbox});
            inl_bytes += align_up(16 * (size_t)(it.inl_nsph + 2 * it.inl_nbox), 16);
        }
        W.item_scene[i] = sidx;
        W.dev_tgt[i] = it.T > 0 && pointer_kind(it.targets) == 1;
        W.dev_q[i] = it.T > 0 && pointer_kind(it.out_q) == 1;
        W.dev_e[i] = it.T > 0 && pointer_kind(it.out_err) == 1;
        W.dev_c[i] = it.T > 0 && pointer_kind(it.out_count) == 1;
        W.dev_ref[i] = it.T > 0 && it.q_ref && pointer_kind(it.q_ref) == 1;
        W.has_ref = W.has_ref || (it.T > 0 && it.q_ref);
        W.host_out = W.host_out || (it.T > 0 && (!W.dev_q[i] || !W.dev_e[i] || !W.dev_c[i]));
        if (it.T > 0 && !W.dev_tgt[i]) {
            for (int t = 0; t < it.T; ++t) {
                const float* q = it.targets + 7 * (size_t)t + 3;
                const float nn = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
                if (!(nn > 0.0f) || !std::isfinite(nn)) return fail(ctx, HJCD_EINVAL, "item %d target %d: zero quaternion", i, t);
            }
        }
        // seeds and candidates
        W.item_t0[i] = W.T;
        W.item_q0[i] = W.q_total;
        W.item_e0[i] = W.e_total;
        for (int t = 0; t < it.T; ++t) {
            const int m = it.spt ? it.spt[t] : it.n_samples;
            if (m < 1 || m > HJCD_MAX_SAMPLES)
                return fail(ctx, HJCD_EINVAL, "item %d target %d: seed count %d outside [1, %d]", i, t, m, HJCD_MAX_SAMPLES);
            const int64_t b = dup_count(m, P.dup_ratio);
            W.CM += m;
            W.CB += b;
            W.min_m = W.CM == m ? m : std::min(W.min_m, m);
            W.max_m = std::max(W.max_m, m);
            W.max_b = std::max(W.max_b, (int)b);
        }
        if ((int64_t)W.T + it.T > (int64_t)(1 << 30)) return fail(ctx, HJCD_EINVAL, "too many targets in one batch");
        W.T += it.T;
        W.q_total += (int64_t)it.T * it.top_k * it.rob->P.n;
        W.e_total += (int64_t)it.T * it.top_k * 2;
    }
    W.NR = (int)W.robots.size();
    W.NS = (int)W.scenes.size();
    for (const RobotRec* r : W.robots) {
        W.n_max = std::max(W.n_max, r->P.n);
        W.ns_max = std::max(W.ns_max, r->P.n_sph);
        W.pairs_max = std::max(W.pairs_max, r->n_pairs);
    }
    for (const auto& e : W.scenes) W.obj4_max = std::max(W.obj4_max, e.nsph + 2 * e.nbox);

    Carve cv;
    W.o_rp = cv.take<RobotParams>(std::max(W.NR, 1));
    W.o_rd = cv.take<RobotDev>(std::max(W.NR, 1));
    W.o_sd = cv.take<SceneDev>(std::max(W.NS, 1));
    W.o_tg = cv.take<TargetDesc>(W.T);
    W.o_moff = cv.take<int64_t>((size_t)W.T + 1);
    W.o_boff = cv.take<int64_t>((size_t)W.T + 1);
    W.o_qe = cv.take<int64_t>(2 * (size_t)W.T);
    W.o_pq7 = cv.take<float>(7 * (size_t)W.T);
    W.o_ref = cv.take<float>(W.has_ref ? (size_t)W.T * W.n_max : 0);
    W.o_inl = cv.take<char>(inl_bytes);
    W.head = cv.off;
    W.o_thM = cv.take<float>((size_t)W.n_max * W.CM);
    W.o_thM2 = cv.take<float>(P.cd_variant == 2 ? (size_t)W.n_max * W.CM : 0);  // lock-step PO-CCD's second buffer
    W.o_sM = cv.take<float>(W.CM);
    W.o_thB = cv.take<float>((size_t)W.n_max * W.CB);
    W.o_sB = cv.take<float>(W.CB);
    W.o_pB = cv.take<float>(W.CB);
    W.o_oB = cv.take<float>(W.CB);
    W.o_hB = cv.take<uint8_t>(W.CB);
    W.o_q = cv.take<float>(W.q_total);
    W.o_e = cv.take<float>(W.e_total);
    W.o_c = cv.take<int32_t>(W.T);
    W.o_ul = cv.take<int32_t>(W.T);           // targets left to the second collision pass
    W.o_sg = cv.take<int32_t>(2 * (size_t)W.CM);  // PO-CCD candidates handed between segments
    // queue head, error flag, count of o_ul, counts of o_sg; the PO-CCD segments' queue heads
    W.o_qf = cv.take<unsigned long long>(6);
    W.bytes = cv.off;
    return HJCD_OK;
}

hjcd_status run_wave(hjcd_ctx* ctx, const WavePlan& W, const WaveItem* items, const hjcd_params& P, char* ws,
                     char* pin, cudaStream_t s, cudaEvent_t* ev) {
    if (W.T == 0) return HJCD_OK;
    hjcd_status st;
    // ---- pinned image of the head ----
    RobotParams* h_rp = reinterpret_cast<RobotParams*>(pin + W.o_rp);
    RobotDev* h_rd = reinterpret_cast<RobotDev*>(pin + W.o_rd);
    SceneDev* h_sd = reinterpret_cast<SceneDev*>(pin + W.o_sd);
    TargetDesc* h_tg = reinterpret_cast<TargetDesc*>(pin + W.o_tg);
    int64_t* h_moff = reinterpret_cast<int64_t*>(pin + W.o_moff);
    int64_t* h_boff = reinterpret_cast<int64_t*>(pin + W.o_boff);
    int64_t* h_qe = reinterpret_cast<int64_t*>(pin + W.o_qe);
    float* h_pq7 = reinterpret_cast<float*>(pin + W.o_pq7);
    for (int r = 0; r < W.NR; ++r) {
        h_rp[r] = W.robots[r]->P;
        h_rd[r] = W.robots[r]->dev;
    }
    for (int k = 0; k < W.NS; ++k) {
        const auto& e = W.scenes[k];
        if (e.res) {
            h_sd[k] = e.res->dev;
        } else {
            const WaveItem& it = items[e.item];
            float4* o = reinterpret_cast<float4*>(pin + W.o_inl + e.off);
            for (int q = 0; q < it.inl_nsph; ++q)
                o[q] = make_float4(it.inl_sph[4 * q], it.inl_sph[4 * q + 1], it.inl_sph[4 * q + 2], it.inl_sph[4 * q + 3]);
            for (int q = 0; q < it.inl_nbox; ++q) {
                const float* b = it.inl_box + 6 * q;
                o[it.inl_nsph + 2 * q] = make_float4(b[0], b[1], b[2], 0.0f);
                o[it.inl_nsph + 2 * q + 1] = make_float4(b[3], b[4], b[5], 0.0f);
            }
            h_sd[k] = SceneDev{reinterpret_cast<const float4*>(ws + W.o_inl + e.off), e.nsph, e.nbox};
        }
    }
    h_moff[0] = h_boff[0] = 0;
    for (int i = 0; i < W.n_items; ++i) {
        const WaveItem& it = items[i];
        const int n = it.rob->P.n;
        const int cd = it.cd_iters >= 0 ? it.cd_iters : P.cd_max_iters;
        const int lm = it.lm_iters >= 0 ? it.lm_iters : P.lm_max_iters;
        for (int t = 0; t < it.T; ++t) {
            const int g = W.item_t0[i] + t;
            TargetDesc d{};
            d.eps_pos = it.eps_pos;
            d.eps_ori = it.eps_ori;
            d.key[0] = (uint32_t)(it.seed & 0xffffffffu);
            d.key[1] = (uint32_t)(it.seed >> 32);
            d.t_local = it.t_base + t;
            d.robot = W.item_robot[i];
            d.scene = W.item_scene[i];
            d.cd_iters = (int16_t)cd;
            d.lm_iters = (int16_t)lm;
            d.top_k = it.top_k | (it.q_ref ? kNearestFlag : 0);
            h_tg[g] = d;
            const int m = it.spt ? it.spt[t] : it.n_samples;
            h_moff[g + 1] = h_moff[g] + m;
            h_boff[g + 1] = h_boff[g] + dup_count(m, P.dup_ratio);
            h_qe[2 * g] = W.item_q0[i] + (int64_t)t * it.top_k * n;
            h_qe[2 * g + 1] = W.item_e0[i] + (int64_t)t * it.top_k * 2;
        }
        if (!W.dev_tgt[i] && it.T > 0)
            std::memcpy(h_pq7 + 7 * (size_t)W.item_t0[i], it.targets, sizeof(float) * 7 * (size_t)it.T);
        if (W.has_ref && it.T > 0) {
            // reference rows at stride n_max (rows of requests without references are not read)
            float* h_ref = reinterpret_cast<float*>(pin + W.o_ref) + (size_t)W.item_t0[i] * W.n_max;
            for (int t = 0; t < it.T; ++t)
                for (int j = 0; j < W.n_max; ++j)
                    h_ref[(size_t)t * W.n_max + j] =
                        (it.q_ref && !W.dev_ref[i] && j < n) ? it.q_ref[(size_t)t * n + j] : 0.0f;
        }
    }

    // ---- host -> device ----
    HJCD_CUDA(ctx, cudaMemcpyAsync(ws, pin, W.head, cudaMemcpyHostToDevice, s));
    for (int i = 0; i < W.n_items; ++i)
        if (W.dev_tgt[i] && items[i].T > 0)
            HJCD_CUDA(ctx, cudaMemcpyAsync(ws + W.o_pq7 + sizeof(float) * 7 * (size_t)W.item_t0[i], items[i].targets,
                                           sizeof(float) * 7 * (size_t)items[i].T, cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < W.n_items; ++i)
        if (W.dev_ref[i])
            HJCD_CUDA(ctx, cudaMemcpy2DAsync(ws + W.o_ref + sizeof(float) * (size_t)W.item_t0[i] * W.n_max,
                                             sizeof(float) * W.n_max, items[i].q_ref,
                                             sizeof(float) * items[i].rob->P.n, sizeof(float) * items[i].rob->P.n,
                                             (size_t)items[i].T, cudaMemcpyDeviceToDevice, s));
    HJCD_CUDA(ctx, cudaMemsetAsync(ws + W.o_qf, 0, 48, s));
    HJCD_CUDA(ctx, cudaMemsetAsync(ws + W.o_q, 0xff, sizeof(float) * (size_t)W.q_total, s));  // unfilled rows: NaN
    HJCD_CUDA(ctx, cudaMemsetAsync(ws + W.o_e, 0xff, sizeof(float) * (size_t)W.e_total, s));

    TargetDesc* d_tg = reinterpret_cast<TargetDesc*>(ws + W.o_tg);
    const int64_t* d_moff = reinterpret_cast<const int64_t*>(ws + W.o_moff);
    const int64_t* d_boff = reinterpret_cast<const int64_t*>(ws + W.o_boff);
    float* thM = reinterpret_cast<float*>(ws + W.o_thM);
    float* sM = reinterpret_cast<float*>(ws + W.o_sM);
    float* thB = reinterpret_cast<float*>(ws + W.o_thB);
    float* sB = reinterpret_cast<float*>(ws + W.o_sB);
    float* pB = reinterpret_cast<float*>(ws + W.o_pB);
    float* oB = reinterpret_cast<float*>(ws + W.o_oB);
    uint8_t* hB = reinterpret_cast<uint8_t*>(ws + W.o_hB);
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(ws + W.o_qf);
    RobotSet rs{reinterpret_cast<const RobotParams*>(ws + W.o_rp), reinterpret_cast<const RobotDev*>(ws + W.o_rd),
                W.NR, W.n_max, W.ns_max, W.pairs_max};
    rs.plain = 1;
    for (int r = 0; r < W.NR; ++r) rs.plain &= W.robots[r]->P.plain;

    if (ev) HJCD_CUDA(ctx, cudaEventRecord(ev[0], s));
    launch_pack_targets(reinterpret_cast<const float*>(ws + W.o_pq7), W.T, d_tg, TargetDesc{}, d_tg, s);
    if ((st = after_launch(ctx, 1, "k_pack_targets"))) return st;

    // Alg. 2: PO-CCD from uniform seeds
    CcdArgs ca{};
    ca.rs = rs;
    ca.tg = d_tg;
    const bool uni_m = W.T > 0 && W.min_m == W.max_m;  // offsets t * max_b for PJ-IK and the filter
    ca.map = CandMap{nullptr, nullptr, d_moff, W.T, 0};
    ca.C = W.CM;
    ca.ld = W.CM;
    ca.th_out = thM;
    ca.th_tmp = reinterpret_cast<float*>(ws + W.o_thM2);
    ca.score = sM;
    ca.n_iters = -1;
    ca.P = P;
    ca.cnt = ctx->cnt;
    ca.block = ctx->ccd_block;
    ca.in_limits = 1;  // seeds sampled inside the limits, every update clamped to them
    // Iteration segments: a lane whose candidate meets the coarse tolerance waits for the rest of
    // its warp, so the iterations run in three launches ([0, cap/2), [cap/2, 3 cap/4), the rest)
    // and the candidates still iterating are packed afresh into full warps for the next (the same
    // results: each candidate's state, iteration index and random streams carry over).  Only for
    // waves that fill the GPU many times over with equal seed counts: a small wave pays the extra
    // launches in latency, and the mixed eight-chain batch (unequal counts) measured slower.
    int cap_max = 0;
    for (int i = 0; i < W.n_items; ++i) cap_max = std::max(cap_max, items[i].cd_iters >= 0 ? items[i].cd_iters : P.cd_max_iters);
    const bool segments = P.cd_variant != 2 && cap_max >= 8 && W.min_m == W.max_m && W.CM >= (int64_t)sm_count() * 2048;
    if (segments) {
        int32_t* lists = reinterpret_cast<int32_t*>(ws + W.o_sg);
        int32_t* counts = reinterpret_cast<int32_t*>(ws + W.o_qf + 16);
        const int seg[3] = {0, cap_max / 2, (3 * cap_max) / 4};
        for (int g = 0; g < 3; ++g) {
            CcdArgs cg = ca;
            cg.seg_begin = seg[g];
            cg.seg_end = g < 2 ? seg[g + 1] : 0;
            cg.list_in = g > 0 ? lists + (size_t)((g - 1) & 1) * W.CM : nullptr;
            cg.n_in = g > 0 ? counts + ((g - 1) & 1) : nullptr;
            cg.list_out = g < 2 ? lists + (size_t)(g & 1) * W.CM : nullptr;
            cg.n_out = g < 2 ? counts + (g & 1) : nullptr;
            cg.queue = reinterpret_cast<unsigned long long*>(ws + W.o_qf + 24) + g;
            launch_ccd(cg, false, s);
            if ((st = after_launch(ctx, 1, "k_ccd"))) return st;
        }
    } else {
        CcdArgs c1 = ca;
        c1.queue = reinterpret_cast<unsigned long long*>(ws + W.o_qf + 24);
        launch_ccd(c1, false, s);
        if ((st = after_launch(ctx, 1, "k_ccd"))) return st;
    }
    if (ev) HJCD_CUDA(ctx, cudaEventRecord(ev[1], s));

    // top-K and perturbed duplication
    DupArgs da{rs, d_tg, W.T, d_moff, sM, thM, W.CM, d_boff, thB, W.CB, nullptr, P.dup_ratio, P.dup_sigma};
    launch_topk_dup(da, W.max_m, s);
    if ((st = after_launch(ctx, 1, "k_topk_dup"))) return st;
    if (ev) HJCD_CUDA(ctx, cudaEventRecord(ev[2], s));

    // PJ-IK
    LmArgs la{};
    la.rs = rs;
    la.tg = d_tg;
    la.map = CandMap{nullptr, nullptr, d_boff, W.T, uni_m ? W.max_b : 0};
    la.C = W.CB;
    la.ld = W.CB;
    la.th = thB;
    la.score = sB;
    la.perr = pB;
    la.oerr = oB;
    la.n_iters = -1;
    la.P = P;
    la.cnt = ctx->cnt;
    la.queue = queue;
    la.warps = ctx->lm_warps;
    la.in_limits = 1;  // PO-CCD's joint vectors and their clamped duplicates
    launch_lm(la, false, s);
    if ((st = after_launch(ctx, 1, "k_lm"))) return st;
    if (ev) HJCD_CUDA(ctx, cudaEventRecord(ev[3], s));

    // collision filter and ranking
    const bool collide = W.ns_max > 0;
    float* q_out = reinterpret_cast<float*>(ws + W.o_q);
    float* e_out = reinterpret_cast<float*>(ws + W.o_e);
    int32_t* c_out = reinterpret_cast<int32_t*>(ws + W.o_c);
    RankArgs ra{rs, d_tg, W.T, d_boff, thB, W.CB, sB, pB, oB, collide ? hB : nullptr, 0,
                reinterpret_cast<const int64_t*>(ws + W.o_qe), q_out, e_out, c_out,
                W.has_ref ? reinterpret_cast<const float*>(ws + W.o_ref) : nullptr, W.n_max};
    CollideArgs cl{};
    if (collide) {
        cl.rs = rs;
        cl.scenes = reinterpret_cast<const SceneDev*>(ws + W.o_sd);
        cl.n_scenes = W.NS;
        cl.max_obj4 = W.obj4_max;
        bool same_scene = true;  // one robot and the same scene for every request
        for (int i = 1; i < W.n_items; ++i) same_scene = same_scene && W.item_scene[i] == W.item_scene[0];
        cl.uniform = W.NR == 1 && same_scene && (W.NS == 0 || W.item_scene[0] == 0);
        if (cl.uniform) {
            cl.u_n = W.robots[0]->P.n;
            cl.u_pairs = W.robots[0]->n_pairs;
            cl.u_osph = W.NS ? W.scenes[0].nsph : 0;
            cl.u_obox = W.NS ? W.scenes[0].nbox : 0;
        }
        for (const auto& e : W.scenes) cl.has_grid = cl.has_grid || (e.res && e.res->dev.cell);
        cl.tg = d_tg;
        cl.map = CandMap{nullptr, nullptr, d_boff, W.T, uni_m ? W.max_b : 0};
        cl.C = W.CB;
        cl.ld = W.CB;
        cl.th = thB;
        cl.hit = hB;
        cl.cnt = ctx->cnt;
        cl.err_flag = wave_flag(W, ws);
        cl.first_wait_polls = ctx->first_wait_polls.load();
    }
    // the top_k collision-free candidates by score are the first top_k collision-free ones in score
    // order: check candidates in that order until they are found (same output as filtering all)
    // A target whose first kLazyDepth ranked candidates hold fewer than top_k collision-free ones
    // (a cluttered scene) would keep one CTA busy for its whole list while the other SMs idle: it
    // is listed instead, and the filter over the listed targets' candidates and their ranking
    // follow as two grid-wide launches.
    bool lazy = false;
    if (collide && ctx->collide_lazy) {
        if (ev) HJCD_CUDA(ctx, cudaEventRecord(ev[4], s));
        RankArgs rl = ra;
        rl.list = reinterpret_cast<int32_t*>(ws + W.o_ul);
        rl.n_list = reinterpret_cast<int32_t*>(ws + W.o_qf + 12);
        lazy = launch_rank_lazy(cl, rl, W.max_b, kLazyDepth, s);
        if (lazy) {
            if ((st = after_launch(ctx, 1, "k_rank_lazy"))) return st;
            CollideArgs c2 = cl;
            c2.list = rl.list;
            c2.n_list = rl.n_list;
            c2.b_off = d_boff;
            c2.list_bmax = std::max(W.max_b, 1);
            launch_collide(c2, s);
            if ((st = after_launch(ctx, 1, "k_collide (list)"))) return st;
            launch_rank(rl, W.max_b, s);
            if ((st = after_launch(ctx, 1, "k_rank (list)"))) return st;
        }
    }
    if (!lazy) {
        if (collide) {
            launch_collide(cl, s);
            if ((st = after_launch(ctx, 1, "k_collide"))) return st;
        }
        if (ev) HJCD_CUDA(ctx, cudaEventRecord(ev[4], s));
        launch_rank(ra, W.max_b, s);
        if ((st = after_launch(ctx, 1, "k_rank"))) return st;
    }
    if (ev) HJCD_CUDA(ctx, cudaEventRecord(ev[5], s));

    // each request's results to its own buffers
    for (int i = 0; i < W.n_items; ++i) {
        const WaveItem& it = items[i];
        if (it.T == 0) continue;
        const size_t nq = (size_t)it.T * it.top_k * it.rob->P.n, ne = (size_t)it.T * it.top_k * 2;
        HJCD_CUDA(ctx, cudaMemcpyAsync(it.out_q, q_out + W.item_q0[i], sizeof(float) * nq,
                                       W.dev_q[i] ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        HJCD_CUDA(ctx, cudaMemcpyAsync(it.out_err, e_out + W.item_e0[i], sizeof(float) * ne,
                                       W.dev_e[i] ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        HJCD_CUDA(ctx, cudaMemcpyAsync(it.out_count, c_out + W.item_t0[i], sizeof(int32_t) * (size_t)it.T,
                                       W.dev_c[i] ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    }
    return HJCD_OK;
}

}  // namespace hjcd

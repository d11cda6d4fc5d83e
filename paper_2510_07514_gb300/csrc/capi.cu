// capi.cu -- the C ABI of include/hjcd.h: context, resident robot and scene
// tables, pointer-kind detection, the whole-method entry points (one request,
// or a batch packed into one launch per phase; wave.cu) and the stage entry
// points.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "host.h"

using namespace hjcd;

namespace hjcd {

hjcd_status fail(hjcd_ctx* ctx, hjcd_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

hjcd_status after_launch(hjcd_ctx* ctx, int kernels, const char* what) {
    ctx->launches += kernels;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, HJCD_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return HJCD_OK;
}

// 1 = device-accessible (device or managed), 0 = host, -1 = null
int pointer_kind(const void* p) {
    if (!p) return -1;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 1;
    return 0;
}

bool pinned_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

hjcd_status make_current(hjcd_ctx* ctx) {
    HJCD_CUDA(ctx, cudaSetDevice(ctx->device));
    return HJCD_OK;
}

hjcd_status ensure_ws(hjcd_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_cap) return HJCD_OK;
    HJCD_CUDA(ctx, cudaEventSynchronize(ctx->ws_free));
    if (ctx->ws) HJCD_CUDA(ctx, cudaFree(ctx->ws));
    ctx->ws = nullptr;
    ctx->ws_cap = 0;
    const size_t cap = align_up(bytes + bytes / 4, 1 << 20);
    HJCD_CUDA(ctx, cudaMalloc(&ctx->ws, cap));
    ctx->ws_cap = cap;
    return HJCD_OK;
}

hjcd_status ensure_pin(hjcd_ctx* ctx, size_t bytes) {
    HJCD_CUDA(ctx, cudaEventSynchronize(ctx->pin_free));
    if (bytes <= ctx->pin_cap) return HJCD_OK;
    if (ctx->pin) HJCD_CUDA(ctx, cudaFreeHost(ctx->pin));
    ctx->pin = nullptr;
    ctx->pin_cap = 0;
    const size_t cap = align_up(bytes + bytes / 4, 1 << 16);
    HJCD_CUDA(ctx, cudaMallocHost(&ctx->pin, cap));
    ctx->pin_cap = cap;
    return HJCD_OK;
}

hjcd_status check_robot(hjcd_ctx* ctx, int32_t id, RobotRec** out) {
    if (id < 0 || id >= (int32_t)ctx->robots.size()) return fail(ctx, HJCD_ENOTFOUND, "unknown robot id %d", id);
    *out = &ctx->robots[id];
    return HJCD_OK;
}

hjcd_status check_scene(hjcd_ctx* ctx, int32_t id, SceneRec** out) {
    *out = nullptr;
    if (id < 0) return HJCD_OK;
    if (id >= (int32_t)ctx->scenes.size() || !ctx->scenes[id].live)
        return fail(ctx, HJCD_ENOTFOUND, "unknown scene id %d", id);
    *out = &ctx->scenes[id];
    return HJCD_OK;
}

hjcd_status check_params(hjcd_ctx* ctx, const hjcd_params& P) {
    if (P.cd_max_iters < 0 || P.lm_max_iters < 0 || P.cd_max_iters > 32767 || P.lm_max_iters > 32767)
        return fail(ctx, HJCD_EINVAL, "iteration caps must be in [0, 32767]");
    if (P.dup_ratio < 1) return fail(ctx, HJCD_EINVAL, "dup_ratio must be >= 1");
    if (P.lm_A < 0 || P.lm_A > 31) return fail(ctx, HJCD_EINVAL, "lm_A must be in [0, 31]");
    if (!(P.lm_beta > 1.0f)) return fail(ctx, HJCD_EINVAL, "lm_beta must be > 1");
    if (!(P.lm_lambda > 0.0f) || !(P.lm_trust_R > 0.0f) || !(P.lm_gn_reg > 0.0f))
        return fail(ctx, HJCD_EINVAL, "lm_lambda, lm_trust_R and lm_gn_reg must be > 0");
    if (!(P.cd_sigma >= 0.0f) || !(P.dup_sigma >= 0.0f) || !(P.lm_sigma >= 0.0f))
        return fail(ctx, HJCD_EINVAL, "perturbation scales must be >= 0");
    if (!(P.proj_eps >= 0.0f)) return fail(ctx, HJCD_EINVAL, "proj_eps must be >= 0");
    if (!(P.cd_tie >= 0.0f && P.cd_tie < 1.0f)) return fail(ctx, HJCD_EINVAL, "cd_tie must be in [0, 1)");
    if (P.cd_variant < 0 || P.cd_variant > 2) return fail(ctx, HJCD_EINVAL, "cd_variant must be 0, 1 or 2");
    return HJCD_OK;
}

int64_t dup_count(int64_t M, int ratio) {
    if (M <= 0) return 0;
    const int64_t K = std::max<int64_t>(1, M / ratio);
    return K * (M / K);
}

RobotSet single_robot_set(const RobotRec& r) {
    return RobotSet{r.d_params, r.d_dev, 1, r.P.n, r.P.n_sph, r.n_pairs, r.P.plain};
}

void collide_uniform(CollideArgs& a, const RobotRec& r, const SceneRec* sc) {
    a.rs = single_robot_set(r);
    a.scenes = sc ? sc->d_dev : nullptr;
    a.n_scenes = sc ? 1 : 0;
    a.max_obj4 = sc ? sc->dev.n_sph + 2 * sc->dev.n_box : 0;
    a.uniform = 1;
    a.u_n = r.P.n;
    a.u_pairs = r.n_pairs;
    a.u_osph = sc ? sc->dev.n_sph : 0;
    a.u_obox = sc ? sc->dev.n_box : 0;
    a.has_grid = sc && sc->dev.cell ? 1 : 0;
}

}  // namespace hjcd

namespace {

// a target-row template for the stage entry points: robot 0, no scene
TargetDesc stage_template(float eps_pos, float eps_ori, uint64_t seed, int cd_iters, int lm_iters, int top_k,
                          int scene) {
    TargetDesc d{};
    d.q[0] = 1.0f;
    d.eps_pos = eps_pos;
    d.eps_ori = eps_ori;
    d.key[0] = (uint32_t)(seed & 0xffffffffu);
    d.key[1] = (uint32_t)(seed >> 32);
    d.robot = 0;
    d.scene = scene;
    d.cd_iters = (int16_t)cd_iters;
    d.lm_iters = (int16_t)lm_iters;
    d.top_k = top_k;
    return d;
}

}  // namespace

extern "C" {

const char* hjcd_status_string(hjcd_status s) {
    switch (s) {
        case HJCD_OK: return "ok";
        case HJCD_EINVAL: return "invalid argument";
        case HJCD_ENOMEM: return "out of memory";
        case HJCD_ECUDA: return "CUDA error";
        case HJCD_ETIMEOUT: return "bounded device wait ran out";
        case HJCD_ENOTFOUND: return "unknown id";
        default: return "unknown status";
    }
}

void hjcd_default_params(hjcd_params* o) {
    if (!o) return;
    o->cd_max_iters = 32;
    o->cd_eps_pos2 = 0.01f * 0.01f;
    o->cd_eps_ori2 = 0.1f * 0.1f;
    o->cd_gamma_pos = 1e-4f;
    o->cd_gamma_ori = 1e-3f;
    o->cd_sigma = 0.05f;
    o->cd_delta0 = 0.5f;
    o->cd_rho = 0.97f;
    o->proj_eps = 1e-4f;
    o->dup_ratio = 4;
    o->dup_sigma = 0.02f;
    o->lm_max_iters = 20;
    o->lm_lambda = 1e-3f;
    o->lm_trust_R = 0.3f;
    o->lm_beta = 2.0f;
    o->lm_A = 4;
    o->lm_sigma = 0.01f;
    o->lm_gn_reg = 1e-6f;
    o->cd_tie = 1e-4f;
    o->cd_variant = 0;
}

hjcd_status hjcd_init(int device, hjcd_ctx** out) {
    if (!out) return HJCD_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HJCD_EINVAL;
    }
    hjcd_ctx* ctx = new hjcd_ctx();
    ctx->device = device;
    hjcd_status s = make_current(ctx);
    if (s == HJCD_OK && (cudaEventCreateWithFlags(&ctx->ws_free, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&ctx->pin_free, cudaEventDisableTiming) != cudaSuccess))
        s = HJCD_ECUDA;
    for (int i = 0; s == HJCD_OK && i < 6; ++i)
        if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) s = HJCD_ECUDA;
    if (s == HJCD_OK && (cudaMalloc(&ctx->cnt, sizeof(Counters)) != cudaSuccess ||
                         cudaMalloc(&ctx->err_flag, sizeof(int32_t)) != cudaSuccess ||
                         cudaMalloc(&ctx->queue, 8 * sizeof(unsigned long long)) != cudaSuccess ||
                         cudaMalloc(&ctx->sink, 4096 * sizeof(float)) != cudaSuccess))
        s = HJCD_ENOMEM;
    if (s == HJCD_OK && (cudaMemset(ctx->cnt, 0, sizeof(Counters)) != cudaSuccess ||
                         cudaMemset(ctx->err_flag, 0, sizeof(int32_t)) != cudaSuccess))
        s = HJCD_ECUDA;
    if (s != HJCD_OK) {
        cudaGetLastError();
        hjcd_destroy(ctx);
        return s;
    }
    *out = ctx;
    return HJCD_OK;
}

void hjcd_destroy(hjcd_ctx* ctx) {
    if (!ctx) return;
    server_stop(ctx);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& r : ctx->robots)
        if (r.dbuf) cudaFree(r.dbuf);
    for (auto& sc : ctx->scenes)
        if (sc.buf) cudaFree(sc.buf);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->pin) cudaFreeHost(ctx->pin);
    if (ctx->cnt) cudaFree(ctx->cnt);
    if (ctx->err_flag) cudaFree(ctx->err_flag);
    if (ctx->queue) cudaFree(ctx->queue);
    if (ctx->sink) cudaFree(ctx->sink);
    if (ctx->ws_free) cudaEventDestroy(ctx->ws_free);
    if (ctx->pin_free) cudaEventDestroy(ctx->pin_free);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    cudaGetLastError();
    delete ctx;
}

const char* hjcd_last_error(const hjcd_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

hjcd_status hjcd_create_robot(hjcd_ctx* ctx, int n, const float* dh_a, const float* dh_alpha, const float* dh_d,
                              const float* dh_theta_off, const float flange[16], const float* q_lo,
                              const float* q_hi, int n_spheres, const int32_t* sph_link, const float* sph_xyzr,
                              const uint8_t* ignore_pairs, int32_t* robot_id) {
    if (!ctx) return HJCD_EINVAL;
    if (n < 1 || n > HJCD_MAX_DOF) return fail(ctx, HJCD_EINVAL, "n_dof %d outside [1, %d]", n, HJCD_MAX_DOF);
    if (!dh_a || !dh_alpha || !dh_d || !flange || !q_lo || !q_hi || !robot_id)
        return fail(ctx, HJCD_EINVAL, "null robot table");
    if (n_spheres < 0 || n_spheres > HJCD_MAX_SPHERES)
        return fail(ctx, HJCD_EINVAL, "n_spheres %d outside [0, %d]", n_spheres, HJCD_MAX_SPHERES);
    if (n_spheres > 0 && (!sph_link || !sph_xyzr)) return fail(ctx, HJCD_EINVAL, "null sphere table");
    if (pointer_kind(dh_a) == 1) return fail(ctx, HJCD_EINVAL, "robot tables must be host memory");
    RobotRec rec;
    RobotParams& P = rec.P;
    P.n = n;
    P.n_sph = n_spheres;
    for (int i = 0; i < n; ++i) {
        if (!(q_lo[i] < q_hi[i])) return fail(ctx, HJCD_EINVAL, "joint %d: q_lo must be < q_hi", i);
        if (!std::isfinite(dh_a[i]) || !std::isfinite(dh_alpha[i]) || !std::isfinite(dh_d[i]))
            return fail(ctx, HJCD_EINVAL, "joint %d: non-finite DH entry", i);
        P.dh[i] = make_float4((float)std::cos((double)dh_alpha[i]), (float)std::sin((double)dh_alpha[i]), dh_a[i],
                              dh_d[i]);
        P.off[i] = dh_theta_off ? dh_theta_off[i] : 0.0f;
        P.lim[i].x = q_lo[i];
        P.lim[i].y = q_hi[i];
    }
    P.fl_eye = flange[0] == 1.0f && flange[5] == 1.0f && flange[10] == 1.0f && flange[1] == 0.0f && flange[2] == 0.0f &&
               flange[4] == 0.0f && flange[6] == 0.0f && flange[8] == 0.0f && flange[9] == 0.0f;
    // plain: no joint offsets, and theta within (-pi, pi) over the limits with a margin far above
    // binary32 rounding; the kinematics then need neither the offset nor a range reduction
    P.plain = 1;
    for (int i = 0; i < n; ++i)
        if (!(P.off[i] == 0.0f && std::fabs((double)P.lim[i].x) <= 3.1415 && std::fabs((double)P.lim[i].y) <= 3.1415))
            P.plain = 0;
    // flange: rigid transform check
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += (double)flange[4 * k + i] * flange[4 * k + j];
            if (std::fabs(s - (i == j ? 1.0 : 0.0)) > 1e-4) return fail(ctx, HJCD_EINVAL, "flange rotation not orthonormal");
        }
    if (flange[12] != 0.0f || flange[13] != 0.0f || flange[14] != 0.0f || flange[15] != 1.0f)
        return fail(ctx, HJCD_EINVAL, "flange last row must be 0 0 0 1");
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) P.fl_r[3 * i + j] = flange[4 * i + j];
        P.fl_p[i] = flange[4 * i + 3];
    }
    const int nb = n + 2;
    for (int s = 0; s < n_spheres; ++s) {
        if (sph_link[s] < 0 || sph_link[s] > n + 1) return fail(ctx, HJCD_EINVAL, "sphere %d: body outside [0, n+1]", s);
        if (!(sph_xyzr[4 * s + 3] > 0.0f)) return fail(ctx, HJCD_EINVAL, "sphere %d: radius must be > 0", s);
    }
    // spheres grouped by body (stable), per-body ranges
    std::vector<float4> sph;
    std::vector<int32_t> body;
    std::vector<int2> range(nb, make_int2(0, 0));
    for (int b = 0; b < nb; ++b) {
        range[b].x = (int)sph.size();
        for (int s = 0; s < n_spheres; ++s)
            if (sph_link[s] == b) {
                sph.push_back(make_float4(sph_xyzr[4 * s], sph_xyzr[4 * s + 1], sph_xyzr[4 * s + 2], sph_xyzr[4 * s + 3]));
                body.push_back(b);
            }
        range[b].y = (int)sph.size() - range[b].x;
    }
    // Bounding sphere of each body's spheres (centre of their bounding box, radius padded by
    // 1e-5 m + 1e-6 relative so binary32 rounding of the transforms cannot hide a fine overlap):
    // a fine sphere overlaps an obstacle only if its body's bounding sphere does.
    std::vector<float4> coarse(nb, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int b = 0; b < nb; ++b) {
        if (!range[b].y) continue;
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int i = range[b].x; i < range[b].x + range[b].y; ++i) {
            const double c[3] = {sph[i].x, sph[i].y, sph[i].z};
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], c[k]);
                hi[k] = std::max(hi[k], c[k]);
            }
        }
        const double m[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
        double r = 0.0;
        for (int i = range[b].x; i < range[b].x + range[b].y; ++i) {
            const double dx = sph[i].x - m[0], dy = sph[i].y - m[1], dz = sph[i].z - m[2];
            r = std::max(r, std::sqrt(dx * dx + dy * dy + dz * dz) + (double)sph[i].w);
        }
        coarse[b] = make_float4((float)m[0], (float)m[1], (float)m[2], (float)(r * (1.0 + 1e-6) + 1e-5));
    }
    // body pairs checked for self-collision: not ignored, spheres on both
    std::vector<int2> pairs;
    for (int i = 0; i < nb; ++i)
        for (int j = i + 1; j < nb; ++j) {
            const bool ign = ignore_pairs ? (ignore_pairs[i * nb + j] != 0 || ignore_pairs[j * nb + i] != 0)
                                          : std::abs(i - j) <= 1;
            if (!ign && range[i].y && range[j].y) pairs.push_back(make_int2(i, j));
        }
    rec.n_pairs = (int)pairs.size();
    hjcd_status st = make_current(ctx);
    if (st) return st;
    const size_t ns1 = std::max<size_t>(sph.size(), 1), np1 = std::max<size_t>(pairs.size(), 1);
    const size_t o_dev = align_up(sizeof(RobotParams)), o_sph = o_dev + align_up(sizeof(RobotDev)),
                 o_body = o_sph + align_up(16 * ns1), o_range = o_body + align_up(4 * ns1),
                 o_coarse = o_range + align_up(8 * (size_t)nb), o_pairs = o_coarse + align_up(16 * (size_t)nb),
                 bytes = o_pairs + align_up(8 * np1);
    HJCD_CUDA(ctx, cudaMalloc(&rec.dbuf, bytes));
    char* base = static_cast<char*>(rec.dbuf);
    rec.d_params = reinterpret_cast<RobotParams*>(base);
    rec.d_dev = reinterpret_cast<RobotDev*>(base + o_dev);
    rec.dev.sph = reinterpret_cast<const float4*>(base + o_sph);
    rec.dev.body = reinterpret_cast<const int32_t*>(base + o_body);
    rec.dev.range = reinterpret_cast<const int2*>(base + o_range);
    rec.dev.coarse = reinterpret_cast<const float4*>(base + o_coarse);
    rec.dev.pairs = reinterpret_cast<const int2*>(base + o_pairs);
    rec.dev.n_pairs = rec.n_pairs;
    rec.dev.n_sph = n_spheres;
    HJCD_CUDA(ctx, cudaMemcpy(rec.d_params, &rec.P, sizeof(RobotParams), cudaMemcpyHostToDevice));
    HJCD_CUDA(ctx, cudaMemcpy(rec.d_dev, &rec.dev, sizeof(RobotDev), cudaMemcpyHostToDevice));
    if (!sph.empty()) {
        HJCD_CUDA(ctx, cudaMemcpy(base + o_sph, sph.data(), 16 * sph.size(), cudaMemcpyHostToDevice));
        HJCD_CUDA(ctx, cudaMemcpy(base + o_body, body.data(), 4 * body.size(), cudaMemcpyHostToDevice));
    }
    HJCD_CUDA(ctx, cudaMemcpy(base + o_range, range.data(), 8 * (size_t)nb, cudaMemcpyHostToDevice));
    HJCD_CUDA(ctx, cudaMemcpy(base + o_coarse, coarse.data(), 16 * (size_t)nb, cudaMemcpyHostToDevice));
    if (!pairs.empty()) HJCD_CUDA(ctx, cudaMemcpy(base + o_pairs, pairs.data(), 8 * pairs.size(), cudaMemcpyHostToDevice));
    std::lock_guard<std::mutex> lock(ctx->api_mu);
    ctx->robots.push_back(rec);
    *robot_id = (int32_t)ctx->robots.size() - 1;
    return HJCD_OK;
}

hjcd_status hjcd_set_scene(hjcd_ctx* ctx, int32_t scene_id_or_new, int n_sph, const float* sph_xyzr, int n_box,
                           const float* box_lohi, int32_t* scene_id) {
    if (!ctx) return HJCD_EINVAL;
    if (!scene_id || n_sph < 0 || n_box < 0 || (n_sph > 0 && !sph_xyzr) || (n_box > 0 && !box_lohi))
        return fail(ctx, HJCD_EINVAL, "bad scene arguments");
    const int nf4 = n_sph + 2 * n_box;
    if (nf4 > kMaxSceneFloat4)
        return fail(ctx, HJCD_EINVAL, "scene too large: spheres + 2*boxes = %d > %d", nf4, kMaxSceneFloat4);
    if (scene_id_or_new >= (int32_t)ctx->scenes.size()) return fail(ctx, HJCD_ENOTFOUND, "unknown scene id %d", scene_id_or_new);
    if ((n_sph > 0 && pointer_kind(sph_xyzr) == 1) || (n_box > 0 && pointer_kind(box_lohi) == 1))
        return fail(ctx, HJCD_EINVAL, "scene tables must be host memory");
    std::vector<float4> buf(std::max(nf4, 1));
    for (int i = 0; i < n_sph; ++i) {
        if (!(sph_xyzr[4 * i + 3] > 0.0f)) return fail(ctx, HJCD_EINVAL, "obstacle sphere %d: radius must be > 0", i);
        if (!std::isfinite(sph_xyzr[4 * i]) || !std::isfinite(sph_xyzr[4 * i + 1]) || !std::isfinite(sph_xyzr[4 * i + 2]))
            return fail(ctx, HJCD_EINVAL, "obstacle sphere %d: non-finite centre", i);
        buf[i] = make_float4(sph_xyzr[4 * i], sph_xyzr[4 * i + 1], sph_xyzr[4 * i + 2], sph_xyzr[4 * i + 3]);
    }
    for (int i = 0; i < n_box; ++i) {
        const float* b = box_lohi + 6 * i;
        if (!(b[0] <= b[3] && b[1] <= b[4] && b[2] <= b[5])) return fail(ctx, HJCD_EINVAL, "box %d: lo > hi", i);
        buf[n_sph + 2 * i] = make_float4(b[0], b[1], b[2], 0.0f);
        buf[n_sph + 2 * i + 1] = make_float4(b[3], b[4], b[5], 0.0f);
    }
    // a large scene gets a uniform grid over its sphere centres, the spheres sorted by cell
    SceneDev d{};
    d.n_sph = n_sph;
    d.n_box = n_box;
    std::vector<int32_t> cell, perm(std::max(n_sph, 1));
    for (int i = 0; i < n_sph; ++i) perm[i] = i;
    if (n_sph >= kGridMinSpheres) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, rmax = 0.0;
        for (int i = 0; i < n_sph; ++i) {
            const double c[3] = {buf[i].x, buf[i].y, buf[i].z};
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], c[k]);
                hi[k] = std::max(hi[k], c[k]);
            }
            rmax = std::max(rmax, (double)buf[i].w);
        }
        double vol = 1.0;
        for (int k = 0; k < 3; ++k) vol *= std::max(hi[k] - lo[k], 1e-3);
        const double h = std::max({std::cbrt(vol / n_sph), 2.0 * rmax, 1e-3});
        int64_t ncell = 1;
        for (int k = 0; k < 3; ++k) {
            d.dim[k] = (int32_t)std::min<double>(std::floor((hi[k] - lo[k]) / h) + 1.0, 1024.0);
            d.lo[k] = (float)lo[k];
            ncell *= d.dim[k];
        }
        d.inv_h = (float)(1.0 / h);
        d.reach = (float)(rmax + 1e-4);
        auto cell_of = [&](const float4& c) {
            int idx[3];
            const float q[3] = {c.x, c.y, c.z};
            for (int k = 0; k < 3; ++k) {
                const int v = (int)std::floor(((double)q[k] - (double)d.lo[k]) * (double)d.inv_h);
                idx[k] = std::min(std::max(v, 0), d.dim[k] - 1);
            }
            return (int64_t)idx[0] + (int64_t)d.dim[0] * ((int64_t)idx[1] + (int64_t)d.dim[1] * idx[2]);
        };
        cell.assign(ncell + 1, 0);
        std::vector<int64_t> key(n_sph);
        for (int i = 0; i < n_sph; ++i) {
            key[i] = cell_of(buf[i]);
            ++cell[key[i] + 1];
        }
        for (int64_t k = 0; k < ncell; ++k) cell[k + 1] += cell[k];
        std::vector<int32_t> fill(cell.begin(), cell.end() - 1);
        std::vector<float4> sorted(n_sph);
        for (int i = 0; i < n_sph; ++i) {
            const int32_t at = fill[key[i]]++;
            sorted[at] = buf[i];
            perm[at] = i;
        }
        std::copy(sorted.begin(), sorted.end(), buf.begin());
    }
    hjcd_status st = make_current(ctx);
    if (st) return st;
    std::lock_guard<std::mutex> lock(ctx->api_mu);
    int32_t id = scene_id_or_new;
    if (id < 0) {
        ctx->scenes.push_back(SceneRec{});
        id = (int32_t)ctx->scenes.size() - 1;
    }
    SceneRec& S = ctx->scenes[id];
    // descriptor slot, obstacles, cell starts, the original index of each sorted sphere
    const size_t o_obj = 64, o_cell = o_obj + align_up(16 * (size_t)std::max(nf4, 1)),
                 o_perm = o_cell + align_up(4 * std::max<size_t>(cell.size(), 1)),
                 bytes = o_perm + align_up(4 * perm.size());
    // an earlier solve may still read the old table
    HJCD_CUDA(ctx, cudaDeviceSynchronize());
    if (bytes > S.cap) {
        if (S.buf) HJCD_CUDA(ctx, cudaFree(S.buf));
        S.buf = nullptr;
        S.cap = 0;
        HJCD_CUDA(ctx, cudaMalloc(&S.buf, bytes));
        S.cap = bytes;
    }
    static_assert(sizeof(SceneDev) <= 64, "scene descriptor fits its slot");
    char* base = static_cast<char*>(S.buf);
    S.d_dev = reinterpret_cast<SceneDev*>(base);
    d.obj = reinterpret_cast<const float4*>(base + o_obj);
    d.cell = cell.empty() ? nullptr : reinterpret_cast<const int32_t*>(base + o_cell);
    S.dev = d;
    S.perm = reinterpret_cast<const int32_t*>(base + o_perm);
    HJCD_CUDA(ctx, cudaMemcpy(base, &S.dev, sizeof(SceneDev), cudaMemcpyHostToDevice));
    HJCD_CUDA(ctx, cudaMemcpy(base + o_obj, buf.data(), 16 * (size_t)std::max(nf4, 1), cudaMemcpyHostToDevice));
    if (!cell.empty()) HJCD_CUDA(ctx, cudaMemcpy(base + o_cell, cell.data(), 4 * cell.size(), cudaMemcpyHostToDevice));
    HJCD_CUDA(ctx, cudaMemcpy(base + o_perm, perm.data(), 4 * perm.size(), cudaMemcpyHostToDevice));
    S.live = true;
    *scene_id = id;
    return HJCD_OK;
}

// one request (or a batch) through the context's own workspace; synchronises
// when an output is host memory
static hjcd_status run_waves(hjcd_ctx* ctx, const WaveItem* items, int n_items, const hjcd_params& P,
                             cudaStream_t s, const WavePlan& whole);

static hjcd_status solve_items(hjcd_ctx* ctx, const WaveItem* items, int n_items, const hjcd_params& P,
                               cudaStream_t s) {
    hjcd_status st;
    WavePlan W;
    if ((st = plan_wave(ctx, items, n_items, P, &W))) return st;
    if (W.T == 0) return HJCD_OK;
    if (ctx->ws_budget && W.bytes > ctx->ws_budget) return run_waves(ctx, items, n_items, P, s, W);
    if ((st = ensure_ws(ctx, W.bytes))) return st;
    if ((st = ensure_pin(ctx, W.head))) return st;
    HJCD_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ws_free, 0));
    const bool prof = ctx->profile;
    if ((st = run_wave(ctx, W, items, P, ctx->ws, ctx->pin, s, prof ? ctx->ev : nullptr))) return st;
    HJCD_CUDA(ctx, cudaEventRecord(ctx->pin_free, s));
    HJCD_CUDA(ctx, cudaEventRecord(ctx->ws_free, s));
    if (prof) ctx->ev_valid = true;
    if (W.host_out) {
        HJCD_CUDA(ctx, cudaStreamSynchronize(s));
        int32_t flag = 0;
        HJCD_CUDA(ctx, cudaMemcpy(&flag, wave_flag(W, ctx->ws), sizeof flag, cudaMemcpyDeviceToHost));
        if (flag) return fail(ctx, HJCD_ETIMEOUT, "collision kernel: staging wait ran out");
    }
    return HJCD_OK;
}

// A solve larger than the workspace budget, in waves: each item's targets are
// cut into consecutive chunks whose seeds fit the budget (estimated from the
// whole plan's bytes per seed), and the chunks run one after another on the
// stream through the same workspace.  Each chunk keeps its targets' indices
// inside the request, so the results equal one whole solve.
static hjcd_status run_waves(hjcd_ctx* ctx, const WaveItem* items, int n_items, const hjcd_params& P,
                             cudaStream_t s, const WavePlan& whole) {
    hjcd_status st;
    const double per_seed = (double)whole.bytes / (double)std::max<int64_t>(whole.CM, 1);
    const int64_t cap_seeds = std::max<int64_t>(1, (int64_t)(0.9 * (double)ctx->ws_budget / per_seed));
    bool host_out = false;
    WavePlan last;
    for (int i = 0; i < n_items; ++i) {
        const WaveItem& it = items[i];
        const int n = it.rob->P.n;
        for (int t0 = 0; t0 < it.T;) {
            int64_t seeds = 0;
            int t1 = t0;
            while (t1 < it.T) {
                const int m = it.spt ? it.spt[t1] : it.n_samples;
                if (t1 > t0 && seeds + m > cap_seeds) break;
                seeds += m;
                ++t1;
            }
            WaveItem sub = it;
            sub.T = t1 - t0;
            sub.t_base = it.t_base + t0;
            sub.targets = it.targets + 7 * (size_t)t0;
            if (it.spt) sub.spt = it.spt + t0;
            if (it.q_ref) sub.q_ref = it.q_ref + (size_t)t0 * n;
            sub.out_q = it.out_q + (size_t)t0 * it.top_k * n;
            sub.out_err = it.out_err + (size_t)t0 * it.top_k * 2;
            sub.out_count = it.out_count + t0;
            WavePlan W;
            if ((st = plan_wave(ctx, &sub, 1, P, &W))) return st;
            if ((st = ensure_ws(ctx, W.bytes))) return st;
            if ((st = ensure_pin(ctx, W.head))) return st;  // waits until the previous chunk's image was copied
            HJCD_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ws_free, 0));
            if ((st = run_wave(ctx, W, &sub, P, ctx->ws, ctx->pin, s, nullptr))) return st;
            HJCD_CUDA(ctx, cudaEventRecord(ctx->pin_free, s));
            HJCD_CUDA(ctx, cudaEventRecord(ctx->ws_free, s));
            host_out = host_out || W.host_out;
            last = std::move(W);
            t0 = t1;
        }
    }
    if (host_out) {
        HJCD_CUDA(ctx, cudaStreamSynchronize(s));
        int32_t flag = 0;
        HJCD_CUDA(ctx, cudaMemcpy(&flag, wave_flag(last, ctx->ws), sizeof flag, cudaMemcpyDeviceToHost));
        if (flag) return fail(ctx, HJCD_ETIMEOUT, "collision kernel: staging wait ran out");
    }
    return HJCD_OK;
}

static hjcd_status item_from(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int n_targets, const float* targets_pq,
                             const hjcd_solve_opts* opts, float* out_q, float* out_err, int32_t* out_count,
                             WaveItem* it) {
    RobotRec* rob;
    SceneRec* sc;
    hjcd_status st;
    if ((st = check_robot(ctx, robot_id, &rob))) return st;
    if ((st = check_scene(ctx, scene_id, &sc))) return st;
    if (!opts) return fail(ctx, HJCD_EINVAL, "null opts");
    if (n_targets < 0) return fail(ctx, HJCD_EINVAL, "n_targets < 0");
    *it = WaveItem{};
    it->rob = rob;
    it->scene = sc;
    it->T = n_targets;
    it->targets = targets_pq;
    it->spt = opts->samples_per_target;
    it->n_samples = opts->n_samples;
    it->eps_pos = opts->eps_pos;
    it->eps_ori = opts->eps_ori;
    it->seed = opts->seed;
    it->top_k = opts->top_k;
    it->cd_iters = -1;
    it->lm_iters = -1;
    it->out_q = out_q;
    it->out_err = out_err;
    it->out_count = out_count;
    return HJCD_OK;
}

hjcd_status hjcd_solve(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int n_targets, const float* targets_pq,
                       const hjcd_solve_opts* opts, float* out_q, float* out_err, int32_t* out_count,
                       void* stream) {
    if (!ctx) return HJCD_EINVAL;
    hjcd_status st;
    WaveItem it;
    if ((st = item_from(ctx, robot_id, scene_id, n_targets, targets_pq, opts, out_q, out_err, out_count, &it)))
        return st;
    if (n_targets == 0) return HJCD_OK;
    hjcd_params P;
    if (opts->params) P = *opts->params;
    else hjcd_default_params(&P);
    if ((st = check_params(ctx, P))) return st;
    if ((st = make_current(ctx))) return st;
    return solve_items(ctx, &it, 1, P, (cudaStream_t)stream);
}

hjcd_status hjcd_solve_nearest(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int n_targets,
                               const float* targets_pq, const float* q_current, const hjcd_solve_opts* opts,
                               float* out_q, float* out_err, int32_t* out_count, void* stream) {
    if (!ctx) return HJCD_EINVAL;
    hjcd_status st;
    WaveItem it;
    if ((st = item_from(ctx, robot_id, scene_id, n_targets, targets_pq, opts, out_q, out_err, out_count, &it)))
        return st;
    if (n_targets == 0) return HJCD_OK;
    if (!q_current) return fail(ctx, HJCD_EINVAL, "null q_current");
    it.q_ref = q_current;
    hjcd_params P;
    if (opts->params) P = *opts->params;
    else hjcd_default_params(&P);
    if ((st = check_params(ctx, P))) return st;
    if ((st = make_current(ctx))) return st;
    return solve_items(ctx, &it, 1, P, (cudaStream_t)stream);
}

hjcd_status hjcd_solve_batch(hjcd_ctx* ctx, int n_items, const hjcd_batch_item* items, const hjcd_params* params,
                             void* stream) {
    if (!ctx) return HJCD_EINVAL;
    if (n_items < 0 || (n_items > 0 && !items)) return fail(ctx, HJCD_EINVAL, "bad item list");
    if (n_items == 0) return HJCD_OK;
    hjcd_status st;
    hjcd_params P;
    if (params) P = *params;
    else hjcd_default_params(&P);
    if ((st = check_params(ctx, P))) return st;
    std::vector<WaveItem> w(n_items);
    for (int i = 0; i < n_items; ++i) {
        const hjcd_batch_item& b = items[i];
        if ((st = item_from(ctx, b.robot_id, b.scene_id, b.n_targets, b.targets_pq, &b.opts, b.out_q, b.out_err,
                            b.out_count, &w[i])))
            return st;
        if (b.scene_id < 0) {
            w[i].inl_nsph = b.n_inline_spheres;
            w[i].inl_sph = b.inline_spheres;
            w[i].inl_nbox = b.n_inline_boxes;
            w[i].inl_box = b.inline_boxes;
            if ((b.n_inline_spheres > 0 && pointer_kind(b.inline_spheres) == 1) ||
                (b.n_inline_boxes > 0 && pointer_kind(b.inline_boxes) == 1))
                return fail(ctx, HJCD_EINVAL, "item %d: inline obstacles must be host memory", i);
        }
        if (b.opts.params) {
            if ((st = check_params(ctx, *b.opts.params))) return st;
            w[i].cd_iters = b.opts.params->cd_max_iters;
            w[i].lm_iters = b.opts.params->lm_max_iters;
        }
        w[i].q_ref = b.q_current;
    }
    if ((st = make_current(ctx))) return st;
    return solve_items(ctx, w.data(), n_items, P, (cudaStream_t)stream);
}

// ---- stages ----------------------------------------------------------------

static hjcd_status stage_prologue(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const float* targets_pq,
                                  float eps_pos, float eps_ori, uint64_t seed, const hjcd_params* params,
                                  int64_t n_cand, const int32_t* tgt, const int32_t* cand, cudaStream_t s,
                                  RobotRec** rob, hjcd_params* P, TargetDesc** d_tg) {
    hjcd_status st;
    if (!ctx) return HJCD_EINVAL;
    if ((st = check_robot(ctx, robot_id, rob))) return st;
    if (n_targets < 1 || !targets_pq || pointer_kind(targets_pq) != 1)
        return fail(ctx, HJCD_EINVAL, "targets must be a device array of n_targets >= 1 poses");
    if (n_cand < 0) return fail(ctx, HJCD_EINVAL, "n_cand < 0");
    if (n_cand > 0 && (pointer_kind(tgt) != 1 || pointer_kind(cand) != 1))
        return fail(ctx, HJCD_EINVAL, "tgt and cand must be device arrays");
    if (!(eps_pos > 0.0f) || !(eps_ori > 0.0f)) return fail(ctx, HJCD_EINVAL, "tolerances must be > 0");
    if (params) *P = *params;
    else hjcd_default_params(P);
    if ((st = check_params(ctx, *P))) return st;
    if ((st = make_current(ctx))) return st;
    if ((st = ensure_ws(ctx, align_up(sizeof(TargetDesc) * (size_t)n_targets)))) return st;
    HJCD_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ws_free, 0));
    *d_tg = reinterpret_cast<TargetDesc*>(ctx->ws);
    launch_pack_targets(targets_pq, n_targets, nullptr, stage_template(eps_pos, eps_ori, seed, 0, 0, 1, -1), *d_tg, s);
    return after_launch(ctx, 1);
}

static hjcd_status check_theta(hjcd_ctx* ctx, const void* p, int64_t n_cand, int64_t ld, const char* what) {
    if (n_cand == 0) return HJCD_OK;
    if (!p || pointer_kind(p) != 1) return fail(ctx, HJCD_EINVAL, "%s must be a device array", what);
    if (ld < n_cand) return fail(ctx, HJCD_EINVAL, "%s: ld %lld < n_cand %lld", what, (long long)ld, (long long)n_cand);
    return HJCD_OK;
}

hjcd_status hjcd_fk(hjcd_ctx* ctx, int32_t robot_id, int64_t n_cand, const float* theta, int64_t ld, float* out_pq,
                    void* stream) {
    if (!ctx) return HJCD_EINVAL;
    RobotRec* rob;
    hjcd_status st;
    if ((st = check_robot(ctx, robot_id, &rob))) return st;
    if ((st = check_theta(ctx, theta, n_cand, ld, "theta"))) return st;
    if (n_cand > 0 && pointer_kind(out_pq) != 1) return fail(ctx, HJCD_EINVAL, "out_pq must be a device array");
    if ((st = make_current(ctx))) return st;
    launch_fk(rob->P, n_cand, theta, ld, out_pq, (cudaStream_t)stream);
    return n_cand > 0 ? after_launch(ctx, 1) : HJCD_OK;
}

hjcd_status hjcd_sample_seeds(hjcd_ctx* ctx, int32_t robot_id, int64_t n_cand, const int32_t* tgt,
                              const int32_t* cand, uint64_t seed, float* theta, int64_t ld, void* stream) {
    if (!ctx) return HJCD_EINVAL;
    RobotRec* rob;
    hjcd_status st;
    if ((st = check_robot(ctx, robot_id, &rob))) return st;
    if ((st = check_theta(ctx, theta, n_cand, ld, "theta"))) return st;
    if (n_cand == 0) return HJCD_OK;
    if (pointer_kind(tgt) != 1 || pointer_kind(cand) != 1) return fail(ctx, HJCD_EINVAL, "tgt and cand must be device arrays");
    if ((st = make_current(ctx))) return st;
    launch_sample(rob->P, seed, CandMap{tgt, cand, nullptr, 0}, n_cand, theta, ld, (cudaStream_t)stream);
    return after_launch(ctx, 1);
}

hjcd_status hjcd_po_ccd(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const float* targets_pq, float eps_pos,
                        float eps_ori, uint64_t seed, const hjcd_params* params, int64_t n_cand, const int32_t* tgt,
                        const int32_t* cand, const float* theta_in, float* theta_out, int64_t ld, int k0,
                        int n_iters, float* score, float* perr, float* oerr, int32_t* iters,
                        const hjcd_ccd_trace* trace, void* stream) {
    RobotRec* rob;
    hjcd_params P;
    TargetDesc* d_tg;
    cudaStream_t s = (cudaStream_t)stream;
    hjcd_status st = stage_prologue(ctx, robot_id, n_targets, targets_pq, eps_pos, eps_ori, seed, params, n_cand,
                                    tgt, cand, s, &rob, &P, &d_tg);
    if (st) return st;
    if (theta_in && (st = check_theta(ctx, theta_in, n_cand, ld, "theta_in"))) return st;
    if ((st = check_theta(ctx, theta_out, n_cand, ld, "theta_out"))) return st;
    if (k0 < 0 || n_iters < 0) return fail(ctx, HJCD_EINVAL, "k0 and n_iters must be >= 0");
    if (trace && n_iters != 1) return fail(ctx, HJCD_EINVAL, "a trace needs n_iters == 1");
    if (P.cd_variant == 2)
        return fail(ctx, HJCD_EINVAL, "cd_variant 2 (target-wide break) runs whole targets: use hjcd_solve");
    CcdArgs a{};
    a.rs = single_robot_set(*rob);
    a.tg = d_tg;
    a.map = CandMap{tgt, cand, nullptr, n_targets};
    a.C = n_cand;
    a.ld = ld;
    a.th_in = theta_in;
    a.th_out = theta_out;
    a.score = score;
    a.perr = perr;
    a.oerr = oerr;
    a.iters = iters;
    a.k0 = k0;
    a.n_iters = n_iters;
    a.P = P;
    if (trace) a.tr = *trace;
    a.cnt = ctx->cnt;
    launch_ccd(a, trace != nullptr, s);
    if ((st = after_launch(ctx, n_cand > 0 ? 1 : 0))) return st;
    HJCD_CUDA(ctx, cudaEventRecord(ctx->ws_free, s));
    return HJCD_OK;
}

hjcd_status hjcd_topk_dup(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const int64_t* m_off, const float* score_M,
                          const float* theta_M, int64_t ld_M, const int64_t* b_off, float* theta_B, int64_t ld_B,
                          int32_t* src_B, uint64_t seed, const hjcd_params* params, void* stream) {
    if (!ctx) return HJCD_EINVAL;
    RobotRec* rob;
    hjcd_status st;
    if ((st = check_robot(ctx, robot_id, &rob))) return st;
    if (n_targets < 1) return fail(ctx, HJCD_EINVAL, "n_targets must be >= 1");
    if (pointer_kind(m_off) != 1 || pointer_kind(b_off) != 1 || pointer_kind(score_M) != 1 ||
        pointer_kind(theta_M) != 1 || pointer_kind(theta_B) != 1)
        return fail(ctx, HJCD_EINVAL, "m_off, b_off, score_M, theta_M, theta_B must be device arrays");
    hjcd_params P;
    if (params) P = *params;
    else hjcd_default_params(&P);
    if ((st = check_params(ctx, P))) return st;
    if ((st = make_current(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // read the offsets back once to size the sort and validate the layout
    std::vector<int64_t> mo(n_targets + 1), bo(n_targets + 1);
    HJCD_CUDA(ctx, cudaMemcpyAsync(mo.data(), m_off, sizeof(int64_t) * mo.size(), cudaMemcpyDeviceToHost, s));
    HJCD_CUDA(ctx, cudaMemcpyAsync(bo.data(), b_off, sizeof(int64_t) * bo.size(), cudaMemcpyDeviceToHost, s));
    HJCD_CUDA(ctx, cudaStreamSynchronize(s));
    int max_m = 0;
    for (int t = 0; t < n_targets; ++t) {
        const int64_t m = mo[t + 1] - mo[t];
        if (m < 0 || m > HJCD_MAX_SAMPLES) return fail(ctx, HJCD_EINVAL, "target %d: seed count outside [0, %d]", t, HJCD_MAX_SAMPLES);
        if (bo[t + 1] - bo[t] != dup_count(m, P.dup_ratio)) return fail(ctx, HJCD_EINVAL, "target %d: b_off does not match the duplication layout", t);
        max_m = std::max(max_m, (int)m);
    }
    if (mo[n_targets] > ld_M || bo[n_targets] > ld_B) return fail(ctx, HJCD_EINVAL, "ld smaller than the candidate count");
    // a TargetDesc per target carrying only the key, the target index and robot 0
    if ((st = ensure_ws(ctx, align_up(sizeof(TargetDesc) * (size_t)n_targets)))) return st;
    HJCD_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ws_free, 0));
    TargetDesc* d_tg = reinterpret_cast<TargetDesc*>(ctx->ws);
    std::vector<TargetDesc> h(n_targets);
    for (int t = 0; t < n_targets; ++t) {
        h[t] = stage_template(1.0f, 1.0f, seed, 0, 0, 1, -1);
        h[t].t_local = t;
    }
    HJCD_CUDA(ctx, cudaMemcpyAsync(d_tg, h.data(), sizeof(TargetDesc) * h.size(), cudaMemcpyHostToDevice, s));
    DupArgs a{single_robot_set(*rob), d_tg, n_targets, m_off, score_M, theta_M, ld_M, b_off, theta_B, ld_B, src_B,
              P.dup_ratio, P.dup_sigma};
    launch_topk_dup(a, max_m, s);
    if ((st = after_launch(ctx, 1))) return st;
    HJCD_CUDA(ctx, cudaStreamSynchronize(s));  // the host staging of the key table must outlive the copy
    HJCD_CUDA(ctx, cudaEventRecord(ctx->ws_free, s));
    return HJCD_OK;
}

hjcd_status hjcd_pjik(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const float* targets_pq, float eps_pos,
                      float eps_ori, uint64_t seed, const hjcd_params* params, int64_t n_cand, const int32_t* tgt,
                      const int32_t* cand, float* theta, int64_t ld, int k0, int n_iters, float* score, float* perr,
                      float* oerr, int32_t* iters, const hjcd_lm_trace* trace, void* stream) {
    RobotRec* rob;
    hjcd_params P;
    TargetDesc* d_tg;
    cudaStream_t s = (cudaStream_t)stream;
    hjcd_status st = stage_prologue(ctx, robot_id, n_targets, targets_pq, eps_pos, eps_ori, seed, params, n_cand,
                                    tgt, cand, s, &rob, &P, &d_tg);
    if (st) return st;
    if ((st = check_theta(ctx, theta, n_cand, ld, "theta"))) return st;
    if (k0 < 0 || n_iters < 0) return fail(ctx, HJCD_EINVAL, "k0 and n_iters must be >= 0");
    if (trace && n_iters != 1) return fail(ctx, HJCD_EINVAL, "a trace needs n_iters == 1");
    LmArgs a{};
    a.rs = single_robot_set(*rob);
    a.tg = d_tg;
    a.map = CandMap{tgt, cand, nullptr, n_targets};
    a.C = n_cand;
    a.ld = ld;
    a.th = theta;
    a.score = score;
    a.perr = perr;
    a.oerr = oerr;
    a.iters = iters;
    a.k0 = k0;
    a.n_iters = n_iters;
    a.P = P;
    if (trace) a.tr = *trace;
    a.cnt = ctx->cnt;
    a.queue = ctx->queue;
    HJCD_CUDA(ctx, cudaMemsetAsync(ctx->queue, 0, sizeof(unsigned long long), s));
    launch_lm(a, trace != nullptr, s);
    if ((st = after_launch(ctx, n_cand > 0 ? 1 : 0))) return st;
    HJCD_CUDA(ctx, cudaEventRecord(ctx->ws_free, s));
    return HJCD_OK;
}

hjcd_status hjcd_collide(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int64_t n_cand, const float* theta,
                         int64_t ld, uint8_t* hit, void* stream) {
    if (!ctx) return HJCD_EINVAL;
    RobotRec* rob;
    SceneRec* sc;
    hjcd_status st;
    if ((st = check_robot(ctx, robot_id, &rob))) return st;
    if ((st = check_scene(ctx, scene_id, &sc))) return st;
    if ((st = check_theta(ctx, theta, n_cand, ld, "theta"))) return st;
    if (n_cand == 0) return HJCD_OK;
    if (pointer_kind(hit) != 1) return fail(ctx, HJCD_EINVAL, "hit must be a device array");
    if ((st = make_current(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (rob->P.n_sph == 0) {
        HJCD_CUDA(ctx, cudaMemsetAsync(hit, 0, (size_t)n_cand, s));
        return HJCD_OK;
    }
    HJCD_CUDA(ctx, cudaMemsetAsync(ctx->err_flag, 0, sizeof(int32_t), s));
    CollideArgs a{};
    collide_uniform(a, *rob, sc);
    a.C = n_cand;
    a.ld = ld;
    a.th = theta;
    a.hit = hit;
    a.cnt = ctx->cnt;
    a.err_flag = ctx->err_flag;
    a.first_wait_polls = ctx->first_wait_polls.load();
    launch_collide(a, s);
    return after_launch(ctx, 1);
}

hjcd_status hjcd_scene_contacts(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int64_t n_cand, const float* theta,
                                int64_t ld, uint8_t* touched, void* stream) {
    if (!ctx) return HJCD_EINVAL;
    RobotRec* rob;
    SceneRec* sc;
    hjcd_status st;
    if ((st = check_robot(ctx, robot_id, &rob))) return st;
    if ((st = check_scene(ctx, scene_id, &sc))) return st;
    if (!sc) return fail(ctx, HJCD_EINVAL, "hjcd_scene_contacts needs a scene");
    if ((st = check_theta(ctx, theta, n_cand, ld, "theta"))) return st;
    const int n_obj = sc->dev.n_sph + sc->dev.n_box;
    if (n_obj > 0 && pointer_kind(touched) != 1) return fail(ctx, HJCD_EINVAL, "touched must be a device array");
    if ((st = make_current(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_obj == 0) return HJCD_OK;
    HJCD_CUDA(ctx, cudaMemsetAsync(touched, 0, (size_t)n_obj, s));
    launch_contacts(rob->P, rob->dev, sc->dev, sc->perm, n_cand, theta, ld, touched, s);
    return after_launch(ctx, n_cand > 0 && rob->P.n_sph > 0 ? 1 : 0);
}

hjcd_status hjcd_rank(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const int64_t* b_off, const float* theta_B,
                      int64_t ld, const float* score, const float* perr, const float* oerr, const uint8_t* hit,
                      float eps_pos, float eps_ori, const float* q_ref, int top_k, float* out_q, float* out_err,
                      int32_t* out_count, void* stream) {
    if (!ctx) return HJCD_EINVAL;
    RobotRec* rob;
    hjcd_status st;
    if ((st = check_robot(ctx, robot_id, &rob))) return st;
    if (n_targets < 1 || top_k < 1 || top_k > HJCD_MAX_TOPK) return fail(ctx, HJCD_EINVAL, "bad n_targets or top_k");
    if (!(eps_pos > 0.0f) || !(eps_ori > 0.0f)) return fail(ctx, HJCD_EINVAL, "tolerances must be > 0");
    if (pointer_kind(b_off) != 1 || pointer_kind(theta_B) != 1 || pointer_kind(score) != 1 ||
        pointer_kind(perr) != 1 || pointer_kind(oerr) != 1 || (hit && pointer_kind(hit) != 1) ||
        (q_ref && pointer_kind(q_ref) != 1) || pointer_kind(out_q) != 1 || pointer_kind(out_err) != 1 ||
        pointer_kind(out_count) != 1)
        return fail(ctx, HJCD_EINVAL, "rank buffers must be device arrays");
    if ((st = make_current(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> bo(n_targets + 1);
    HJCD_CUDA(ctx, cudaMemcpyAsync(bo.data(), b_off, sizeof(int64_t) * bo.size(), cudaMemcpyDeviceToHost, s));
    HJCD_CUDA(ctx, cudaStreamSynchronize(s));
    int max_b = 0;
    for (int t = 0; t < n_targets; ++t) {
        const int64_t b = bo[t + 1] - bo[t];
        if (b < 0 || b > HJCD_MAX_SAMPLES) return fail(ctx, HJCD_EINVAL, "target %d: candidate count outside [0, %d]", t, HJCD_MAX_SAMPLES);
        max_b = std::max(max_b, (int)b);
    }
    if (bo[n_targets] > ld) return fail(ctx, HJCD_EINVAL, "ld smaller than the candidate count");
    RankArgs a{single_robot_set(*rob), nullptr, n_targets, b_off, theta_B, ld, score, perr, oerr, hit, top_k,
               nullptr, out_q, out_err, out_count, q_ref, rob->P.n};
    a.eps_pos = eps_pos;
    a.eps_ori = eps_ori;
    // rows past a target's count read NaN, as hjcd_solve leaves them
    HJCD_CUDA(ctx, cudaMemsetAsync(out_q, 0xff, sizeof(float) * (size_t)n_targets * top_k * rob->P.n, s));
    HJCD_CUDA(ctx, cudaMemsetAsync(out_err, 0xff, sizeof(float) * (size_t)n_targets * top_k * 2, s));
    launch_rank(a, max_b, s);
    return after_launch(ctx, 1);
}

hjcd_status hjcd_philox(hjcd_ctx* ctx, int64_t n_blocks, const uint32_t* ctr, uint64_t key, uint32_t* out,
                        void* stream) {
    if (!ctx) return HJCD_EINVAL;
    if (n_blocks < 0) return fail(ctx, HJCD_EINVAL, "n_blocks < 0");
    if (n_blocks == 0) return HJCD_OK;
    if (pointer_kind(ctr) != 1 || pointer_kind(out) != 1) return fail(ctx, HJCD_EINVAL, "ctr and out must be device arrays");
    if ((reinterpret_cast<uintptr_t>(ctr) | reinterpret_cast<uintptr_t>(out)) & 15u)
        return fail(ctx, HJCD_EINVAL, "ctr and out must be 16-byte aligned");
    hjcd_status st;
    if ((st = make_current(ctx))) return st;
    launch_philox(n_blocks, ctr, key, out, (cudaStream_t)stream);
    return after_launch(ctx, 1, "k_philox");
}

// ---- instrumentation -----------------------------------------------------

hjcd_status hjcd_set_collision_mode(hjcd_ctx* ctx, int32_t mode) {
    if (!ctx) return HJCD_EINVAL;
    if (mode != 0 && mode != 1) return fail(ctx, HJCD_EINVAL, "collision mode must be 0 (all candidates) or 1 (ranked)");
    ctx->collide_lazy = mode == 1;
    return HJCD_OK;
}

hjcd_status hjcd_set_wait_limit(hjcd_ctx* ctx, int64_t polls) {
    if (!ctx) return HJCD_EINVAL;
    ctx->first_wait_polls = polls < 0 ? -1 : polls;
    return HJCD_OK;
}

hjcd_status hjcd_set_memory_budget(hjcd_ctx* ctx, uint64_t bytes) {
    if (!ctx) return HJCD_EINVAL;
    if (bytes && bytes < (1u << 20)) return fail(ctx, HJCD_EINVAL, "a memory budget below 1 MiB cannot hold a wave");
    ctx->ws_budget = (size_t)bytes;
    return HJCD_OK;
}

hjcd_status hjcd_set_profiling(hjcd_ctx* ctx, int on) {
    if (!ctx) return HJCD_EINVAL;
    ctx->profile = on != 0;
    ctx->ev_valid = false;
    return HJCD_OK;
}

hjcd_status hjcd_phase_times(hjcd_ctx* ctx, float ms[6]) {
    if (!ctx || !ms) return HJCD_EINVAL;
    if (!ctx->ev_valid) return fail(ctx, HJCD_EINVAL, "no profiled solve recorded");
    HJCD_CUDA(ctx, cudaEventSynchronize(ctx->ev[5]));
    for (int i = 0; i < 5; ++i) HJCD_CUDA(ctx, cudaEventElapsedTime(&ms[i], ctx->ev[i], ctx->ev[i + 1]));
    HJCD_CUDA(ctx, cudaEventElapsedTime(&ms[5], ctx->ev[0], ctx->ev[5]));
    return HJCD_OK;
}

hjcd_status hjcd_counters(hjcd_ctx* ctx, uint64_t out[8], int reset) {
    if (!ctx || !out) return HJCD_EINVAL;
    hjcd_status st;
    if ((st = make_current(ctx))) return st;
    HJCD_CUDA(ctx, cudaDeviceSynchronize());
    Counters c;
    HJCD_CUDA(ctx, cudaMemcpy(&c, ctx->cnt, sizeof c, cudaMemcpyDeviceToHost));
    for (int i = 0; i < 8; ++i) out[i] = c.v[i];
    if (reset) HJCD_CUDA(ctx, cudaMemset(ctx->cnt, 0, sizeof(Counters)));
    int32_t flag = 0;
    HJCD_CUDA(ctx, cudaMemcpy(&flag, ctx->err_flag, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) return fail(ctx, HJCD_ETIMEOUT, "a bounded device wait ran out");
    return HJCD_OK;
}

int64_t hjcd_launch_count(const hjcd_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

hjcd_status hjcd_ffma_probe(hjcd_ctx* ctx, int iters, double* tflops, void* stream) {
    if (!ctx || !tflops || iters < 1) return HJCD_EINVAL;
    hjcd_status st;
    if ((st = make_current(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = sm_count() * 8;
    cudaEvent_t a, b;
    HJCD_CUDA(ctx, cudaEventCreate(&a));
    HJCD_CUDA(ctx, cudaEventCreate(&b));
    launch_ffma(ctx->sink, iters, blocks, s);  // warm-up
    HJCD_CUDA(ctx, cudaEventRecord(a, s));
    launch_ffma(ctx->sink, iters, blocks, s);
    HJCD_CUDA(ctx, cudaEventRecord(b, s));
    if ((st = after_launch(ctx, 2))) return st;
    HJCD_CUDA(ctx, cudaEventSynchronize(b));
    float ms = 0.0f;
    HJCD_CUDA(ctx, cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double flops = (double)blocks * 256.0 * (double)iters * (double)ffma_flops_per_thread_iter();
    *tflops = flops / ((double)ms * 1e-3) / 1e12;
    return HJCD_OK;
}

}  // extern "C"

// ---- allocation-free solve ----------------------------------------------------
//
// hjcd_solve_noalloc keeps all of its scratch in the file-scope device array
// below.  Host code cannot use the array's name as an address (there it
// denotes a host-side stand-in), so the device address is looked up once per
// device with cudaGetSymbolAddress and passed to the kernels.

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[HJCD_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoallocMaxDevices] = {};

// device address of g_noalloc_scratch on `device` (current), looked up on first use
hjcd_status noalloc_scratch(hjcd_ctx* ctx, int device, char** out) {
    if (device < 0 || device >= kNoallocMaxDevices) return fail(ctx, HJCD_EINVAL, "device ordinal %d unsupported", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(ctx, HJCD_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
        g_noalloc_addr[device] = p;
    }
    *out = static_cast<char*>(g_noalloc_addr[device]);
    return HJCD_OK;
}

// per-target seed and candidate offsets for a uniform seed count
__global__ void k_uniform_offsets(int64_t* m_off, int64_t* b_off, int T, int64_t M, int64_t B) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= T; t += gridDim.x * blockDim.x) {
        m_off[t] = (int64_t)t * M;
        b_off[t] = (int64_t)t * B;
    }
}

}  // namespace

extern "C" hjcd_status hjcd_solve_noalloc(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int n_targets,
                                          const float* targets_pq, const hjcd_solve_opts* opts, float* out_q,
                                          float* out_err, int32_t* out_count, void* stream) {
    if (!ctx) return HJCD_EINVAL;
    RobotRec* rob;
    SceneRec* sc;
    hjcd_status st;
    if ((st = check_robot(ctx, robot_id, &rob))) return st;
    if ((st = check_scene(ctx, scene_id, &sc))) return st;
    if (!opts) return fail(ctx, HJCD_EINVAL, "null opts");
    if (n_targets < 0) return fail(ctx, HJCD_EINVAL, "n_targets < 0");
    if (n_targets == 0) return HJCD_OK;
    if (opts->samples_per_target)
        return fail(ctx, HJCD_EINVAL, "hjcd_solve_noalloc takes a uniform n_samples (samples_per_target must be NULL)");
    if (pointer_kind(targets_pq) != 1 || pointer_kind(out_q) != 1 || pointer_kind(out_err) != 1 ||
        pointer_kind(out_count) != 1)
        return fail(ctx, HJCD_EINVAL, "hjcd_solve_noalloc needs device pointers for targets and outputs");
    if (!(opts->eps_pos > 0.0f) || !(opts->eps_ori > 0.0f)) return fail(ctx, HJCD_EINVAL, "tolerances must be > 0");
    if (opts->top_k < 1 || opts->top_k > HJCD_MAX_TOPK) return fail(ctx, HJCD_EINVAL, "top_k outside [1, %d]", HJCD_MAX_TOPK);
    if (opts->n_samples < 1 || opts->n_samples > HJCD_MAX_SAMPLES)
        return fail(ctx, HJCD_EINVAL, "n_samples outside [1, %d]", HJCD_MAX_SAMPLES);
    hjcd_params P;
    if (opts->params) P = *opts->params;
    else hjcd_default_params(&P);
    if ((st = check_params(ctx, P))) return st;
    if (P.cd_variant == 2) return fail(ctx, HJCD_EINVAL, "hjcd_solve_noalloc does not run cd_variant 2");
    if ((st = make_current(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const RobotParams& R = rob->P;
    const int n = R.n, T = n_targets, top_k = opts->top_k, M = opts->n_samples;
    const int64_t B = dup_count(M, P.dup_ratio);
    const int64_t CM = (int64_t)T * M, CB = (int64_t)T * B;

    // layout inside the static scratch
    Carve cv;
    const size_t o_tg = cv.take<TargetDesc>(T);
    const size_t o_off = cv.take<int64_t>(2 * (size_t)(T + 1));
    const size_t o_thM = cv.take<float>((size_t)n * CM);
    const size_t o_sM = cv.take<float>(CM);
    const size_t o_thB = cv.take<float>((size_t)n * CB);
    const size_t o_sB = cv.take<float>(CB);
    const size_t o_pB = cv.take<float>(CB);
    const size_t o_oB = cv.take<float>(CB);
    const size_t o_hB = cv.take<uint8_t>(CB);
    const size_t o_q = cv.take<unsigned long long>(1);
    const size_t o_f = cv.take<int32_t>(1);
    if (cv.off > HJCD_NOALLOC_SCRATCH_BYTES)
        return fail(ctx, HJCD_EINVAL, "hjcd_solve_noalloc: %d targets x %d seeds need %zu bytes of scratch, "
                    "the static scratch holds %u", T, M, cv.off, (unsigned)HJCD_NOALLOC_SCRATCH_BYTES);
    char* W = nullptr;
    if ((st = noalloc_scratch(ctx, ctx->device, &W))) return st;
    TargetDesc* d_tg = reinterpret_cast<TargetDesc*>(W + o_tg);
    int64_t* d_moff = reinterpret_cast<int64_t*>(W + o_off);
    int64_t* d_boff = d_moff + T + 1;
    float* thM = reinterpret_cast<float*>(W + o_thM);
    float* sM = reinterpret_cast<float*>(W + o_sM);
    float* thB = reinterpret_cast<float*>(W + o_thB);
    float* sB = reinterpret_cast<float*>(W + o_sB);
    float* pB = reinterpret_cast<float*>(W + o_pB);
    float* oB = reinterpret_cast<float*>(W + o_oB);
    uint8_t* hB = reinterpret_cast<uint8_t*>(W + o_hB);
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(W + o_q);
    int32_t* flag = reinterpret_cast<int32_t*>(W + o_f);

    // the previous call's contents are still there: clear what must start at zero
    HJCD_CUDA(ctx, cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s));
    HJCD_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    k_uniform_offsets<<<(T + 256) / 256, 256, 0, s>>>(d_moff, d_boff, T, M, B);
    launch_pack_targets(targets_pq, T, nullptr,
                        stage_template(opts->eps_pos, opts->eps_ori, opts->seed, P.cd_max_iters, P.lm_max_iters, top_k,
                                       sc ? 0 : -1),
                        d_tg, s);
    if ((st = after_launch(ctx, 2))) return st;

    const RobotSet rs = single_robot_set(*rob);
    CcdArgs ca{};
    ca.rs = rs;
    ca.tg = d_tg;
    ca.map = CandMap{nullptr, nullptr, d_moff, T, M};  // every target has M seeds: no search
    ca.C = CM;
    ca.ld = CM;
    ca.th_out = thM;
    ca.score = sM;
    ca.n_iters = P.cd_max_iters;
    ca.P = P;
    ca.block = ctx->ccd_block;
    ca.in_limits = 1;  // sampled seeds
    launch_ccd(ca, false, s);
    DupArgs da{rs, d_tg, T, d_moff, sM, thM, CM, d_boff, thB, CB, nullptr, P.dup_ratio, P.dup_sigma};
    launch_topk_dup(da, M, s);
    LmArgs la{};
    la.rs = rs;
    la.tg = d_tg;
    la.map = CandMap{nullptr, nullptr, d_boff, T, (int32_t)B};
    la.C = CB;
    la.ld = CB;
    la.th = thB;
    la.score = sB;
    la.perr = pB;
    la.oerr = oB;
    la.n_iters = P.lm_max_iters;
    la.P = P;
    la.queue = queue;
    la.warps = ctx->lm_warps;
    la.in_limits = 1;  // PO-CCD's joint vectors and their clamped duplicates
    launch_lm(la, false, s);
    const bool collide = R.n_sph > 0;
    if (collide) {
        // a collision CTA whose staging wait runs out returns without verdicts: its candidates
        // must then count as colliding, not keep the previous call's verdicts
        HJCD_CUDA(ctx, cudaMemsetAsync(hB, 1, (size_t)CB, s));
        CollideArgs cl{};
        collide_uniform(cl, *rob, sc);
        cl.tg = d_tg;
        cl.map = CandMap{nullptr, nullptr, d_boff, T, (int32_t)B};
        cl.C = CB;
        cl.ld = CB;
        cl.th = thB;
        cl.hit = hB;
        cl.err_flag = flag;
        launch_collide(cl, s);
    }
    RankArgs ra{rs, d_tg, T, d_boff, thB, CB, sB, pB, oB, collide ? hB : nullptr, top_k, nullptr,
                out_q, out_err, out_count};
    // rows past a target's count are NaN, as hjcd_solve leaves them (stream-ordered, no allocation)
    HJCD_CUDA(ctx, cudaMemsetAsync(out_q, 0xff, sizeof(float) * (size_t)T * top_k * n, s));
    HJCD_CUDA(ctx, cudaMemsetAsync(out_err, 0xff, sizeof(float) * (size_t)T * top_k * 2, s));
    launch_rank(ra, (int)B, s);
    return after_launch(ctx, collide ? 5 : 4);
}

// ---- seeds of a target sharded across devices -----------------------------------

namespace {

hjcd_status shard_common(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const float* targets_pq,
                         const hjcd_solve_opts* opts, RobotRec** rob, hjcd_params* P, int64_t* K) {
    hjcd_status st;
    if ((st = check_robot(ctx, robot_id, rob))) return st;
    if (!opts || n_targets < 1 || pointer_kind(targets_pq) != 1)
        return fail(ctx, HJCD_EINVAL, "need opts and n_targets >= 1 device target poses");
    if (opts->samples_per_target) return fail(ctx, HJCD_EINVAL, "sharded solves take a uniform n_samples");
    if (opts->n_samples < 1 || opts->n_samples > HJCD_MAX_SAMPLES)
        return fail(ctx, HJCD_EINVAL, "n_samples outside [1, %d]", HJCD_MAX_SAMPLES);
    if (!(opts->eps_pos > 0.0f) || !(opts->eps_ori > 0.0f)) return fail(ctx, HJCD_EINVAL, "tolerances must be > 0");
    if (opts->params) *P = *opts->params;
    else hjcd_default_params(P);
    if ((st = check_params(ctx, *P))) return st;
    if (P->cd_variant == 2) return fail(ctx, HJCD_EINVAL, "sharded seeds cannot take the target-wide break");
    *K = std::max<int64_t>(1, opts->n_samples / P->dup_ratio);
    return make_current(ctx);
}

}  // namespace

extern "C" {

hjcd_status hjcd_shard_topk(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const float* targets_pq,
                            const hjcd_solve_opts* opts, int32_t seed_begin, int32_t seed_end, float* out_score,
                            int32_t* out_index, float* out_theta, void* stream) {
    if (!ctx) return HJCD_EINVAL;
    RobotRec* rob;
    hjcd_params P;
    int64_t K;
    hjcd_status st;
    if ((st = shard_common(ctx, robot_id, n_targets, targets_pq, opts, &rob, &P, &K))) return st;
    if (seed_begin < 0 || seed_end <= seed_begin || seed_end > opts->n_samples)
        return fail(ctx, HJCD_EINVAL, "seed range [%d, %d) outside [0, %d)", seed_begin, seed_end, opts->n_samples);
    if (pointer_kind(out_score) != 1 || pointer_kind(out_index) != 1 || pointer_kind(out_theta) != 1)
        return fail(ctx, HJCD_EINVAL, "outputs must be device arrays");
    const int T = n_targets, n = rob->P.n, Ms = seed_end - seed_begin;
    const int64_t C = (int64_t)T * Ms;
    Carve cv;
    const size_t o_tg = cv.take<TargetDesc>(T), o_off = cv.take<int64_t>(2 * (size_t)(T + 1)),
                 o_th = cv.take<float>((size_t)n * C), o_s = cv.take<float>(C);
    if ((st = ensure_ws(ctx, cv.off))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    HJCD_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ws_free, 0));
    char* W = ctx->ws;
    TargetDesc* d_tg = reinterpret_cast<TargetDesc*>(W + o_tg);
    int64_t* d_off = reinterpret_cast<int64_t*>(W + o_off);
    k_uniform_offsets<<<(T + 256) / 256, 256, 0, s>>>(d_off, d_off + T + 1, T, Ms, Ms);
    launch_pack_targets(targets_pq, T, nullptr,
                        stage_template(opts->eps_pos, opts->eps_ori, opts->seed, P.cd_max_iters, P.lm_max_iters, 1, -1),
                        d_tg, s);
    CcdArgs ca{};
    ca.rs = single_robot_set(*rob);
    ca.tg = d_tg;
    ca.map = CandMap{nullptr, nullptr, d_off, T};
    ca.C = C;
    ca.ld = C;
    ca.th_out = reinterpret_cast<float*>(W + o_th);
    ca.score = reinterpret_cast<float*>(W + o_s);
    ca.n_iters = P.cd_max_iters;
    ca.P = P;
    ca.cnt = ctx->cnt;
    ca.block = ctx->ccd_block;
    ca.seed_base = seed_begin;
    ca.in_limits = 1;  // sampled seeds
    launch_ccd(ca, false, s);
    ShardTopkArgs ta{single_robot_set(*rob), d_tg, T, (int32_t)K, seed_begin, d_off, ca.score, ca.th_out, C,
                     out_score, out_index, out_theta, n};
    launch_shard_topk(ta, Ms, s);
    HJCD_CUDA(ctx, cudaEventRecord(ctx->ws_free, s));
    return after_launch(ctx, 4);
}

hjcd_status hjcd_topk_merge(hjcd_ctx* ctx, int n_targets, int n_lists, int K, int n, const float* in_score,
                            const int32_t* in_index, const float* in_theta, float* out_score, int32_t* out_index,
                            float* out_theta, void* stream) {
    if (!ctx) return HJCD_EINVAL;
    if (n_targets < 1 || n_lists < 1 || K < 1 || n < 1 || n > HJCD_MAX_DOF || (int64_t)n_lists * K > HJCD_MAX_SAMPLES)
        return fail(ctx, HJCD_EINVAL, "bad merge sizes");
    if (pointer_kind(in_score) != 1 || pointer_kind(in_index) != 1 || pointer_kind(in_theta) != 1 ||
        pointer_kind(out_score) != 1 || pointer_kind(out_index) != 1 || pointer_kind(out_theta) != 1)
        return fail(ctx, HJCD_EINVAL, "merge buffers must be device arrays");
    hjcd_status st;
    if ((st = make_current(ctx))) return st;
    MergeArgs a{n_targets, n_lists, K, n, in_score, in_index, in_theta, out_score, out_index, out_theta};
    launch_topk_merge(a, (cudaStream_t)stream);
    return after_launch(ctx, 1);
}

hjcd_status hjcd_solve_from_topk(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int n_targets,
                                 const float* targets_pq, int32_t first_target, const hjcd_solve_opts* opts,
                                 const float* kept_theta, float* out_q, float* out_err, int32_t* out_count,
                                 void* stream) {
    if (!ctx) return HJCD_EINVAL;
    RobotRec* rob;
    SceneRec* sc;
    hjcd_params P;
    int64_t K;
    hjcd_status st;
    if ((st = shard_common(ctx, robot_id, n_targets, targets_pq, opts, &rob, &P, &K))) return st;
    if ((st = check_scene(ctx, scene_id, &sc))) return st;
    if (opts->top_k < 1 || opts->top_k > HJCD_MAX_TOPK) return fail(ctx, HJCD_EINVAL, "top_k outside [1, %d]", HJCD_MAX_TOPK);
    if (first_target < 0) return fail(ctx, HJCD_EINVAL, "first_target < 0");
    if (pointer_kind(kept_theta) != 1 || pointer_kind(out_q) != 1 || pointer_kind(out_err) != 1 ||
        pointer_kind(out_count) != 1)
        return fail(ctx, HJCD_EINVAL, "kept_theta and the outputs must be device arrays");
    const int T = n_targets, top_k = opts->top_k;
    const int64_t B = dup_count(opts->n_samples, P.dup_ratio), CB = (int64_t)T * B;
    Carve cv;
    const size_t o_tg = cv.take<TargetDesc>(T), o_off = cv.take<int64_t>(2 * (size_t)(T + 1)),
                 o_th = cv.take<float>((size_t)rob->P.n * CB), o_sB = cv.take<float>(CB), o_pB = cv.take<float>(CB),
                 o_oB = cv.take<float>(CB), o_hB = cv.take<uint8_t>(CB), o_q = cv.take<unsigned long long>(2);
    if ((st = ensure_ws(ctx, cv.off))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    HJCD_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ws_free, 0));
    char* W = ctx->ws;
    TargetDesc* d_tg = reinterpret_cast<TargetDesc*>(W + o_tg);
    int64_t* d_boff = reinterpret_cast<int64_t*>(W + o_off);
    float* thB = reinterpret_cast<float*>(W + o_th);
    float* sB = reinterpret_cast<float*>(W + o_sB);
    float* pB = reinterpret_cast<float*>(W + o_pB);
    float* oB = reinterpret_cast<float*>(W + o_oB);
    uint8_t* hB = reinterpret_cast<uint8_t*>(W + o_hB);
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(W + o_q);
    HJCD_CUDA(ctx, cudaMemsetAsync(queue, 0, 16, s));
    HJCD_CUDA(ctx, cudaMemsetAsync(out_q, 0xff, sizeof(float) * (size_t)T * top_k * rob->P.n, s));
    HJCD_CUDA(ctx, cudaMemsetAsync(out_err, 0xff, sizeof(float) * (size_t)T * top_k * 2, s));
    k_uniform_offsets<<<(T + 256) / 256, 256, 0, s>>>(d_boff + T + 1, d_boff, T, B, B);
    // each target keeps its index inside the whole request, which keys its random streams
    TargetDesc tmpl = stage_template(opts->eps_pos, opts->eps_ori, opts->seed, P.cd_max_iters, P.lm_max_iters, top_k,
                                     sc ? 0 : -1);
    tmpl.t_local = first_target;
    launch_pack_targets(targets_pq, T, nullptr, tmpl, d_tg, s);
    const RobotSet rs = single_robot_set(*rob);
    KeptDupArgs da{rs, d_tg, T, (int32_t)K, kept_theta, d_boff, thB, CB, P.dup_sigma};
    launch_dup_kept(da, s);
    LmArgs la{};
    la.rs = rs;
    la.tg = d_tg;
    la.map = CandMap{nullptr, nullptr, d_boff, T};
    la.C = CB;
    la.ld = CB;
    la.th = thB;
    la.score = sB;
    la.perr = pB;
    la.oerr = oB;
    la.n_iters = -1;
    la.P = P;
    la.cnt = ctx->cnt;
    la.queue = queue;
    la.warps = ctx->lm_warps;
    launch_lm(la, false, s);
    const bool collide = rob->P.n_sph > 0;
    if (collide) {
        // a collision CTA whose staging wait runs out returns without verdicts (this call does not
        // report it): its candidates then count as colliding instead of keeping stale verdicts
        HJCD_CUDA(ctx, cudaMemsetAsync(hB, 1, (size_t)CB, s));
        CollideArgs cl{};
        collide_uniform(cl, *rob, sc);
        cl.tg = d_tg;
        cl.map = CandMap{nullptr, nullptr, d_boff, T};
        cl.C = CB;
        cl.ld = CB;
        cl.th = thB;
        cl.hit = hB;
        cl.cnt = ctx->cnt;
        cl.err_flag = reinterpret_cast<int32_t*>(queue + 1);
        launch_collide(cl, s);
    }
    RankArgs ra{rs, d_tg, T, d_boff, thB, CB, sB, pB, oB, collide ? hB : nullptr, top_k, nullptr,
                out_q, out_err, out_count};
    launch_rank(ra, (int)B, s);
    HJCD_CUDA(ctx, cudaEventRecord(ctx->ws_free, s));
    return after_launch(ctx, collide ? 6 : 5);
}

}  // extern "C"

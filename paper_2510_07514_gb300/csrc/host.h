// host.h -- host-side state of a context (resident robots and scenes, the
// solve workspace, the serving loop) and the helpers the C-ABI translation
// units share.  Not part of the public interface.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdarg>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hjcd_internal.cuh"

namespace hjcd {

constexpr int kMaxSceneFloat4 = 1 << 20;  // resident scene: obstacle spheres + 2 * boxes
constexpr int kGridMinSpheres = 512;      // resident scenes with this many spheres get a uniform grid
constexpr int kLazyDepth = 64;            // ranked candidates a target's CTA checks before it hands over

// Resident robot: the kinematic table (host copy) and one device buffer with
// the kinematic table, the collision-table descriptor and the collision
// tables themselves (spheres sorted by body, bodies, per-body ranges and
// bounding spheres, self-collision body pairs).
struct RobotRec {
    RobotParams P{};
    RobotDev dev{};  // device pointers into dbuf
    void* dbuf = nullptr;
    RobotParams* d_params = nullptr;
    RobotDev* d_dev = nullptr;
    int n_pairs = 0;
};

// Resident scene: one device buffer holding its descriptor, then the obstacles.
struct SceneRec {
    void* buf = nullptr;
    SceneDev* d_dev = nullptr;
    SceneDev dev{};  // host copy (device pointers to the obstacles and grid)
    const int32_t* perm = nullptr;  // device: original index of each stored sphere
    size_t cap = 0;
    bool live = false;
};

struct Server;  // serving loop (serve.cu)

}  // namespace hjcd

struct hjcd_ctx {
    int device = 0;
    std::vector<hjcd::RobotRec> robots;
    std::vector<hjcd::SceneRec> scenes;
    std::string err;
    char* ws = nullptr;  // device workspace of the synchronous entry points
    size_t ws_cap = 0;
    char* pin = nullptr;  // pinned host staging
    size_t pin_cap = 0;
    cudaEvent_t ws_free = nullptr;   // recorded when the last call's device work on the workspace ends
    cudaEvent_t pin_free = nullptr;  // recorded after the last copy out of the pinned staging
    hjcd::Counters* cnt = nullptr;
    int32_t* err_flag = nullptr;
    unsigned long long* queue = nullptr;  // work-queue heads of the persistent kernels (stage entry points)
    float* sink = nullptr;
    bool profile = false;
    cudaEvent_t ev[6] = {};
    bool ev_valid = false;
    std::atomic<int64_t> launches{0};
    size_t ws_budget = 0;     // workspace bytes one solve may use before it splits into waves (0: unlimited)
    // settings read by the serving thread's launches while a caller may change them
    std::atomic<bool> collide_lazy{true};  // rank first, collision-check in rank order (hjcd_set_collision_mode)
    std::atomic<int32_t> ccd_block{64};    // launch configuration (hjcd_set_launch_config, hjcd_autotune)
    std::atomic<int32_t> lm_warps{8};
    std::atomic<int64_t> first_wait_polls{-1};  // collision kernels' first staging wait (hjcd_set_wait_limit)
    std::mutex api_mu;  // robots/scenes tables against the serving thread
    hjcd::Server* server = nullptr;  // owned; freed by server_stop
};

namespace hjcd {

hjcd_status fail(hjcd_ctx* ctx, hjcd_status code, const char* fmt, ...);

#define HJCD_CUDA(ctx, call)                                                                         \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return ::hjcd::fail(ctx, e_ == cudaErrorMemoryAllocation ? HJCD_ENOMEM : HJCD_ECUDA,      \
                                "%s: %s (%s)", #call, cudaGetErrorString(e_), cudaGetErrorName(e_)); \
    } while (0)

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

struct Carve {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        const size_t o = off;
        off = align_up(off + count * sizeof(T));
        return o;
    }
};

hjcd_status after_launch(hjcd_ctx* ctx, int kernels, const char* what = "kernel");
int pointer_kind(const void* p);  // 1 device/managed, 0 host, -1 null
bool pinned_host(const void* p);
hjcd_status make_current(hjcd_ctx* ctx);
hjcd_status ensure_ws(hjcd_ctx* ctx, size_t bytes);
hjcd_status ensure_pin(hjcd_ctx* ctx, size_t bytes);
hjcd_status check_robot(hjcd_ctx* ctx, int32_t id, RobotRec** out);
hjcd_status check_scene(hjcd_ctx* ctx, int32_t id, SceneRec** out);
hjcd_status check_params(hjcd_ctx* ctx, const hjcd_params& P);
int64_t dup_count(int64_t M, int ratio);
RobotSet single_robot_set(const RobotRec& r);
// collision arguments of a launch where every candidate is robot r against scene sc (or none)
void collide_uniform(CollideArgs& a, const RobotRec& r, const SceneRec* sc);

// ---- packed solve of several requests ("wave") ---------------------------------

// One request inside a wave.
struct WaveItem {
    const RobotRec* rob = nullptr;
    const SceneRec* scene = nullptr;  // resident scene, or
    int inl_nsph = 0, inl_nbox = 0;   // an inline scene (host arrays, copied with the wave)
    const float* inl_sph = nullptr;
    const float* inl_box = nullptr;
    int T = 0;
    const float* targets = nullptr;  // [T][7] px py pz qw qx qy qz, host or device
    const int32_t* spt = nullptr;    // seeds per target (host), or null for n_samples each
    int n_samples = 0;
    float eps_pos = 0.0f, eps_ori = 0.0f;
    uint64_t seed = 0;
    int top_k = 1;
    int cd_iters = -1, lm_iters = -1;  // < 0: the batch parameters' caps
    int t_base = 0;  // index of targets[0] inside its request (keys the random streams)
    const float* q_ref = nullptr;  // [T][n] reference configurations (nearest-first ranking), host or device
    float* out_q = nullptr;  // [T][top_k][n], host or device
    float* out_err = nullptr;  // [T][top_k][2]
    int32_t* out_count = nullptr;  // [T]
};

struct WavePlan {
    int n_items = 0, T = 0, NR = 0, NS = 0;
    int64_t CM = 0, CB = 0;
    int max_m = 0, max_b = 0, min_m = 0;  // min_m == max_m: every target has max_m seeds
    int n_max = 0, ns_max = 0, pairs_max = 0, obj4_max = 0;
    std::vector<const RobotRec*> robots;  // the wave's robot table
    std::vector<int> item_robot, item_scene;
    struct SceneEnt {
        const SceneRec* res;  // resident scene, or null for item `item`'s inline scene
        int item;
        size_t off;  // inline: byte offset of its obstacles in the head
        int nsph, nbox;
    };
    std::vector<SceneEnt> scenes;
    std::vector<int> item_t0;
    std::vector<int64_t> item_q0, item_e0;
    std::vector<char> dev_tgt, dev_q, dev_e, dev_c, dev_ref;
    bool has_ref = false;
    int64_t q_total = 0, e_total = 0;
    // head: copied from the pinned image to the start of the workspace in one copy
    size_t o_rp = 0, o_rd = 0, o_sd = 0, o_tg = 0, o_moff = 0, o_boff = 0, o_qe = 0, o_pq7 = 0, o_ref = 0, o_inl = 0,
           head = 0;
    // the rest of the workspace
    size_t o_thM = 0, o_thM2 = 0, o_sM = 0, o_thB = 0, o_sB = 0, o_pB = 0, o_oB = 0, o_hB = 0, o_q = 0, o_e = 0, o_c = 0,
           o_ul = 0, o_sg = 0, o_qf = 0, bytes = 0;
    bool host_out = false;  // some output goes to host memory
};

// Validate the items and lay out the wave.  Caps from P unless an item sets
// its own (cd_iters / lm_iters >= 0).
hjcd_status plan_wave(hjcd_ctx* ctx, const WaveItem* items, int n_items, const hjcd_params& P, WavePlan* out);

// Fill the pinned image (plan.head bytes at `pin`), copy it to `ws`, run the
// launch sequence of Alg. 2 over the whole wave and copy each item's results
// out, all on stream s.  Nothing is synchronised.  ev (6 events or null) is
// recorded around the phases.
hjcd_status run_wave(hjcd_ctx* ctx, const WavePlan& W, const WaveItem* items, const hjcd_params& P, char* ws,
                     char* pin, cudaStream_t s, cudaEvent_t* ev);

// The wave's error flag (int32, nonzero: a bounded device wait ran out).
inline int32_t* wave_flag(const WavePlan& W, char* ws) { return reinterpret_cast<int32_t*>(ws + W.o_qf + 8); }

// ---- serving loop --------------------------------------------------------------

void server_stop(hjcd_ctx* ctx);

}  // namespace hjcd

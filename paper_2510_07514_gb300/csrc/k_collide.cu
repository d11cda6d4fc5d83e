// k_collide.cu -- sphere collision filter (Sec. V-C), one warp per candidate.
//
// Two levels, as in the paper's coarse-then-fine check: every body carries a
// bounding sphere of its link spheres, and a body's fine spheres are tested
// against an obstacle (or another body's spheres) only when the bounding
// spheres overlap.  The bounding radii are padded beyond binary32 rounding, so
// the verdict is the brute-force verdict over all fine pairs.
//
// Per candidate: every lane walks the kinematic chain and moves its own fine
// spheres (sphere lane + 32 q of the body-grouped table) and, on lane b, the
// bounding sphere of body b into the world frame; the warp publishes them to
// shared memory.  Self pairs: lanes over the checked body pairs for the
// bounding test; the fine sphere pairs of each overlapping body pair are
// spread over the warp.  Obstacles: lanes over obstacles (32 at a time) for
// the bounding test of one body; the overlapping obstacles are compacted into
// a list and their fine tests (list x the body's spheres) spread over the
// warp.  The warp stops at the first overlap.  When the launch has a single
// scene, its obstacles (spheres, then boxes) are staged once per CTA into
// shared memory by one bulk asynchronous copy (TMA, cp.async.bulk) completing
// on an mbarrier; a launch mixing scenes reads each candidate's obstacles from
// its scene table.  Each candidate uses its target's robot: the kinematic
// tables of the launch's robots sit in shared memory, a warp reloads its
// lanes' link spheres when its candidate's robot changes.
//
// Overlap: |c1 - c2|^2 < (r1 + r2)^2 for spheres; for a box, the squared
// distance from the centre to its clamp into the box below r^2.
#include "hjcd_internal.cuh"

namespace hjcd {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kMaxStagedObj4 = 10240;  // obstacle float4s staged in shared memory (160 KB)
constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait polls before the staged tables are given up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bulk global -> shared copy; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// an obstacle: from shared memory (staged scene) or through the read-only cache
template <bool STAGED>
__device__ __forceinline__ float4 ld_obj(const float4* p, int i) {
    if (STAGED) return p[i];
    return __ldg(p + i);
}

__device__ __forceinline__ float4 to_world(const Frame& F, float4 s) {
    const V3 w = fma3(s.z, F.c2, fma3(s.y, F.c1, fma3(s.x, F.c0, F.p)));
    return make_float4(w.x, w.y, w.z, s.w);
}

__device__ __forceinline__ bool sph_sph(float4 a, float4 b) {
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, rr = a.w + b.w;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
}

__device__ __forceinline__ bool sph_box(float4 a, float4 lo, float4 hi) {
    const float dx = a.x - clampf(a.x, lo.x, hi.x);
    const float dy = a.y - clampf(a.y, lo.y, hi.y);
    const float dz = a.z - clampf(a.z, lo.z, hi.z);
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < a.w * a.w;
}

// shared-memory layout of a CTA: staged obstacles, mbarrier, robot tables,
// then per warp the world-frame fine spheres, bounding spheres and a list
struct CollideLayout {
    uint32_t bar, robots, warp, warp_bytes, total;
};

// per warp: world fine spheres [ns], world bounding spheres [nb], the robot's
// body ranges [nb] and checked body pairs [n_pairs], a list of 32 indices
__host__ __device__ __forceinline__ CollideLayout collide_smem_layout(int n_obj4, int n_robots, int nb, int ns,
                                                                      int n_pairs) {
    CollideLayout L;
    L.bar = 16u * (uint32_t)n_obj4;
    L.robots = L.bar + 16u;
    L.warp = L.robots + (uint32_t)robots_smem_bytes(n_robots);
    L.warp_bytes = (16u * (uint32_t)(ns + nb) + 8u * (uint32_t)(nb + n_pairs) + 4u * 32u + 15u) / 16u * 16u;
    L.total = L.warp + kWarpsPerBlock * L.warp_bytes;
    return L;
}


// The warp's current robot: its lanes' link spheres (body frame) and bodies, the
// bounding sphere of body `lane`, DoF, checked pairs and the bodies that carry spheres.
template <int SPL>
struct WarpRobot {
    float4 ls[SPL];
    int lb[SPL];
    float4 lco;
    int cur, n_m, pairs_m;
    unsigned bmask;
};

// The warp's shared-memory buffers: world fine spheres, world bounding spheres,
// the robot's body ranges and checked pairs, a list of 32 indices.
struct WarpBufs {
    float4* wsph;
    float4* wco;
    int2* wrange;
    int2* wpairs;
    int* list;
};

// Collision verdict of candidate c (robot row rid, scene row sid, -1: none),
// warp-uniform; t_s / t_b accumulate the sphere and box tests.
template <int SPL, bool UNIFORM, bool GRID>
__device__ __forceinline__ bool warp_collides(const CollideArgs& A, const RobotParams* rob, const SceneDev& sc0,
                                              const float4* s_scene, WarpRobot<SPL>& W, const WarpBufs& Bf, int64_t c,
                                              int rid, int sid, unsigned long long& t_s, unsigned long long& t_b) {
    constexpr bool STAGED = UNIFORM;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    float4* const wsph = Bf.wsph;
    float4* const wco = Bf.wco;
    int2* const wrange = Bf.wrange;
    int2* const wpairs = Bf.wpairs;
    int* const list = Bf.list;
    if (rid != W.cur) {
        W.cur = rid;
        const RobotDev rd = A.rs.rd[rid];
        W.n_m = rob[rid].n;
        W.pairs_m = rd.n_pairs;
        const int ns = rd.n_sph, nbr = W.n_m + 2;
#pragma unroll
        for (int q = 0; q < SPL; ++q) {
            const int i = lane + 32 * q;
            W.lb[q] = i < ns ? __ldg(rd.body + i) : -1;
            W.ls[q] = i < ns ? __ldg(rd.sph + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        W.lco = lane < nbr ? __ldg(rd.coarse + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        for (int i = lane; i < nbr; i += 32) wrange[i] = __ldg(rd.range + i);
        for (int i = lane; i < W.pairs_m; i += 32) wpairs[i] = __ldg(rd.pairs + i);
        __syncwarp();
        W.bmask = __ballot_sync(0xffffffffu, lane < nbr && wrange[lane].y > 0);  // bodies with spheres
    }
    const RobotParams& R = rob[rid];
    const int n = UNIFORM ? A.u_n : W.n_m, nb = n + 2, n_pairs = UNIFORM ? A.u_pairs : W.pairs_m;
    // obstacles: the staged copy (shared memory) or the scene's table (global, read-only path)
    const float4* obj = s_scene;
    int n_osph = 0, n_obox = 0;
    if (UNIFORM) {
        n_osph = A.u_osph;
        n_obox = A.u_obox;
    } else if (sid >= 0) {
        const SceneDev sd = A.scenes[sid];
        obj = sd.obj;
        n_osph = sd.n_sph;
        n_obox = sd.n_box;
    }

    // world frame: body 0 is the base (identity)
    float4 ws[SPL];
#pragma unroll
    for (int q = 0; q < SPL; ++q) ws[q] = W.ls[q];
    float4 wc = W.lco;
    Frame F = frame_identity();
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
        fk_step(R, j, A.th[j * A.ld + c], F);
#pragma unroll
        for (int q = 0; q < SPL; ++q)
            if (W.lb[q] == j + 1) ws[q] = to_world(F, W.ls[q]);
        if (lane == j + 1) wc = to_world(F, W.lco);
    }
    const Frame E = fk_flange(R, F);
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
        if (W.lb[q] == n + 1) ws[q] = to_world(E, W.ls[q]);
        if (W.lb[q] >= 0) wsph[lane + 32 * q] = ws[q];
    }
    if (lane == n + 1) wc = to_world(E, W.lco);
    if (lane < nb) wco[lane] = wc;
    __syncwarp();

    bool hit = false;

    // self-collision: bounding test per checked body pair, fine pairs spread over the warp
    for (int p0 = 0; p0 < n_pairs && !hit; p0 += 32) {
        const int p = p0 + lane;
        int2 pr = make_int2(0, 0);
        bool ch = false;
        if (p < n_pairs) {
            pr = wpairs[p];
            ch = sph_sph(wco[pr.x], wco[pr.y]);
        }
        t_s += (unsigned long long)min(32, n_pairs - p0);
        unsigned m = __ballot_sync(0xffffffffu, ch);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1u;
            const int ba = __shfl_sync(0xffffffffu, pr.x, src), bb = __shfl_sync(0xffffffffu, pr.y, src);
            const int2 ra = wrange[ba], rb = wrange[bb];
            const int items = ra.y * rb.y;
            bool h = false;
            for (int w = lane; w < items; w += 32) {
                const int i = w / rb.y;
                h |= sph_sph(wsph[ra.x + i], wsph[rb.x + (w - i * rb.y)]);
            }
            t_s += (unsigned long long)items;
            if (__any_sync(0xffffffffu, h)) {
                hit = true;
                break;
            }
        }
    }

    // obstacle spheres of a gridded scene: per body, the lanes walk the cells within the
    // bounding sphere's radius plus the largest obstacle radius; each obstacle that
    // overlaps the bounding sphere is tested against the body's fine spheres
    const int32_t* gcell = nullptr;
    if (GRID && n_osph > 0) gcell = (UNIFORM ? sc0 : A.scenes[sid]).cell;
    if (GRID && gcell) {
        const SceneDev& G = A.scenes[UNIFORM ? 0 : sid];
        for (int b = 0; b < nb && !hit; ++b) {
            const int2 rg = wrange[b];
            if (rg.y == 0) continue;
            const float4 co = wco[b];
            const float ext = co.w + G.reach;
            const float cc[3] = {co.x, co.y, co.z};
            int i0[3], i1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int dmax = G.dim[k] - 1;
                i0[k] = min(max((int)floorf((cc[k] - ext - G.lo[k]) * G.inv_h), 0), dmax);
                i1[k] = min(max((int)floorf((cc[k] + ext - G.lo[k]) * G.inv_h), 0), dmax);
            }
            const int nx = i1[0] - i0[0] + 1, ny = i1[1] - i0[1] + 1, nxy = nx * ny;
            const int ncell = nxy * (i1[2] - i0[2] + 1);
            bool h = false;
            unsigned tl = 0;
            for (int q = lane; q < ncell && !h; q += 32) {
                const int z = q / nxy, r = q - z * nxy, y = r / nx, x = r - y * nx;
                const int k = (i0[0] + x) + G.dim[0] * ((i0[1] + y) + G.dim[1] * (i0[2] + z));
                const int a = __ldg(gcell + k), e = __ldg(gcell + k + 1);
                for (int o = a; o < e && !h; ++o) {
                    const float4 sp = ld_obj<STAGED>(obj, o);
                    ++tl;
                    if (sph_sph(co, sp)) {
                        for (int i = 0; i < rg.y && !h; ++i) h = sph_sph(wsph[rg.x + i], sp);
                        tl += rg.y;
                    }
                }
            }
            t_s += __reduce_add_sync(0xffffffffu, tl);
            hit = __any_sync(0xffffffffu, h);
        }
    }

    // obstacle spheres, 32 at a time: each lane tests its obstacle against every body's
    // bounding sphere (a bit per body); only bodies some obstacle overlaps are visited, their
    // overlapping obstacles compacted and the fine tests spread over the warp
    const int nbs = __popc(W.bmask);
    for (int o0 = 0; o0 < n_osph && !hit && !(GRID && gcell); o0 += 32) {
        const int o = o0 + lane;
        const bool valid = o < n_osph;
        const float4 s = valid ? ld_obj<STAGED>(obj, o) : make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned bm = 0;
        if (valid)
            for (unsigned bb = W.bmask; bb; bb &= bb - 1u) {
                const int b = __ffs(bb) - 1;
                if (sph_sph(wco[b], s)) bm |= 1u << b;
            }
        t_s += (unsigned long long)min(32, n_osph - o0) * nbs;
        for (unsigned todo = __reduce_or_sync(0xffffffffu, bm); todo && !hit; todo &= todo - 1u) {
            const int b = __ffs(todo) - 1;
            const int2 rg = wrange[b];
            const bool ch = (bm >> b) & 1u;
            const unsigned m = __ballot_sync(0xffffffffu, ch);
            if (ch) list[__popc(m & lt)] = o;
            __syncwarp();
            const int items = __popc(m) * rg.y;
            bool h = false;
            for (int w = lane; w < items; w += 32) {
                const int k = w / rg.y;
                h |= sph_sph(wsph[rg.x + (w - k * rg.y)], ld_obj<STAGED>(obj, list[k]));
            }
            t_s += (unsigned long long)items;
            hit = __any_sync(0xffffffffu, h);
            __syncwarp();
        }
    }

    // obstacle boxes, the same way
    const float4* box = obj + n_osph;
    for (int o0 = 0; o0 < n_obox && !hit; o0 += 32) {
        const int o = o0 + lane;
        const bool valid = o < n_obox;
        const float4 lo = valid ? ld_obj<STAGED>(box, 2 * o) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 hi = valid ? ld_obj<STAGED>(box, 2 * o + 1) : lo;
        unsigned bm = 0;
        if (valid)
            for (unsigned bb = W.bmask; bb; bb &= bb - 1u) {
                const int b = __ffs(bb) - 1;
                if (sph_box(wco[b], lo, hi)) bm |= 1u << b;
            }
        t_b += (unsigned long long)min(32, n_obox - o0) * nbs;
        for (unsigned todo = __reduce_or_sync(0xffffffffu, bm); todo && !hit; todo &= todo - 1u) {
            const int b = __ffs(todo) - 1;
            const int2 rg = wrange[b];
            const bool ch = (bm >> b) & 1u;
            const unsigned m = __ballot_sync(0xffffffffu, ch);
            if (ch) list[__popc(m & lt)] = o;
            __syncwarp();
            const int items = __popc(m) * rg.y;
            bool h = false;
            for (int w = lane; w < items; w += 32) {
                const int k = w / rg.y, bo = list[k];
                h |= sph_box(wsph[rg.x + (w - k * rg.y)], ld_obj<STAGED>(box, 2 * bo), ld_obj<STAGED>(box, 2 * bo + 1));
            }
            t_b += (unsigned long long)items;
            hit = __any_sync(0xffffffffu, h);
            __syncwarp();
        }
    }

    return hit;
}

// CTA prologue of the collision kernels: the obstacles of a single scene
// staged by one bulk copy (UNIFORM), the robots' kinematic tables with plain
// loads.  False (error flag set) when the staging wait ran out or the scene
// outgrew the shared memory the host sized; the CTA must return.
template <bool UNIFORM>
__device__ __forceinline__ bool collide_prologue(const CollideArgs& A, unsigned char* smem, const CollideLayout& L,
                                                 const SceneDev& sc0, int n_obj4, const RobotParams** rob) {
    float4* s_scene = reinterpret_cast<float4*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    const uint32_t bytes = 16u * (uint32_t)n_obj4;
    if (UNIFORM) {
        if (threadIdx.x == 0) mbar_init(bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (bytes > 0) {
                mbar_arrive_expect_tx(bar, bytes);
                bulk_g2s(s_scene, sc0.obj, bytes, bar);
            } else {
                mbar_arrive(bar);
            }
        }
    }
    *rob = stage_robots(smem + L.robots, A.rs);
    if (UNIFORM) {
        const uint32_t polls = A.first_wait_polls < 0 ? kWaitLimit
                               : (uint32_t)(A.first_wait_polls < (int64_t)kWaitLimit ? A.first_wait_polls : kWaitLimit);
        const bool staged = mbar_wait_bounded(bar, 0, polls);
        if (__syncthreads_or(!staged)) {
            // give up: flag the error, give the copy one more bounded wait (the full limit: the
            // copy must land before the CTA's shared memory is released)
            if (threadIdx.x == 0) {
                atomicExch(A.err_flag, 1);
                mbar_wait_bounded(bar, 0);
            }
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ WarpBufs warp_bufs(unsigned char* smem, const CollideLayout& L, const CollideArgs& A) {
    const int nb_max = A.rs.n_max + 2;
    unsigned char* wb = smem + L.warp + (threadIdx.x >> 5) * L.warp_bytes;
    WarpBufs B;
    B.wsph = reinterpret_cast<float4*>(wb);
    B.wco = B.wsph + A.rs.ns_max;
    B.wrange = reinterpret_cast<int2*>(B.wco + nb_max);
    B.wpairs = B.wrange + nb_max;
    B.list = reinterpret_cast<int*>(B.wpairs + A.rs.pairs_max);
    return B;
}

template <int SPL, bool UNIFORM, bool GRID>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_collide(const CollideArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SceneDev sc0 = A.n_scenes > 0 ? A.scenes[0] : SceneDev{nullptr, 0, 0};
    const int n_obj4 = UNIFORM ? sc0.n_sph + 2 * sc0.n_box : 0;
    if (n_obj4 > (UNIFORM ? A.max_obj4 : 0)) {  // the scene outgrew the shared memory the host sized
        if (threadIdx.x == 0) atomicExch(A.err_flag, 2);
        return;
    }
    // list mode: the candidates of the listed targets only (none listed: nothing to stage)
    const int64_t items = A.list ? (int64_t)*A.n_list * A.list_bmax : A.C;
    if (items == 0) return;
    const CollideLayout L = collide_smem_layout(n_obj4, A.rs.n, A.rs.n_max + 2, A.rs.ns_max, A.rs.pairs_max);
    const RobotParams* rob;
    if (!collide_prologue<UNIFORM>(A, smem, L, sc0, n_obj4, &rob)) return;
    const WarpBufs Bf = warp_bufs(smem, L, A);
    const float4* s_scene = reinterpret_cast<const float4*>(smem);

    WarpRobot<SPL> W;
    W.cur = -1;
    W.n_m = W.pairs_m = 0;
    W.bmask = 0;
    unsigned long long tests = 0, btests = 0, ncand = 0;
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    int rid = 0, sid = 0;
    bool tvalid = true;
    for (int64_t it = (int64_t)blockIdx.x * kWarpsPerBlock + warp; it < items; it += nwarps) {
        int64_t c = it;
        if (A.list) {
            const int t = A.list[it / A.list_bmax];
            const int j = (int)(it % A.list_bmax);
            const int64_t b0 = A.b_off[t];
            if (j >= A.b_off[t + 1] - b0 || A.hit[b0 + j] != 2) continue;  // not ranked, or checked
            c = b0 + j;
        }
        if (!UNIFORM && A.tg) {
            int32_t t, s;
            tvalid = A.map.lookup(c, t, s);
            if (tvalid) {
                const TargetDesc& Td = A.tg[t];
                rid = Td.robot;
                sid = Td.scene;
                tvalid = Td.eps_pos > 0.0f;
            }
        } else if (!UNIFORM) {
            sid = A.n_scenes > 0 ? 0 : -1;
        }
        if (!tvalid) {  // no such target, or an invalid one: never ranked
            if (lane == 0) A.hit[c] = 1;
            continue;
        }
        unsigned long long t_s = 0, t_b = 0;  // tests of this candidate (uniform over the warp)
        const bool hit = warp_collides<SPL, UNIFORM, GRID>(A, rob, sc0, s_scene, W, Bf, c, rid, sid, t_s, t_b);
        if (lane == 0) {
            A.hit[c] = hit ? 1 : 0;
            tests += t_s;
            btests += t_b;
            ++ncand;
        }
        __syncwarp();
    }
    if (A.cnt && lane == 0) {
        atomicAdd(&A.cnt->v[3], tests);
        atomicAdd(&A.cnt->v[6], btests);
        atomicAdd(&A.cnt->v[4], ncand);
    }
}

// Ranking with the collision filter applied lazily (the top_k collision-free
// candidates by score are the first top_k collision-free ones in score
// order): one CTA per target sorts its candidates' keys, then its warps check
// candidates in rank order, one candidate per warp and kWarpsPerBlock at a
// time, until top_k collision-free ones are found or the ranked candidates
// run out.  Same output as the collision filter over all candidates followed
// by k_rank.
template <int SPL, bool UNIFORM, bool GRID>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_rank_lazy(const CollideArgs A, const RankArgs R,
                                                                  uint32_t keys_off, int depth) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int verdict[kWarpsPerBlock];
    __shared__ int picks[HJCD_MAX_TOPK];
    __shared__ int n_found;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x;
    const SceneDev sc0 = A.n_scenes > 0 ? A.scenes[0] : SceneDev{nullptr, 0, 0};
    const int n_obj4 = UNIFORM ? sc0.n_sph + 2 * sc0.n_box : 0;
    if (n_obj4 > (UNIFORM ? A.max_obj4 : 0)) {
        if (threadIdx.x == 0) atomicExch(A.err_flag, 2);
        return;
    }
    const CollideLayout L = collide_smem_layout(n_obj4, A.rs.n, A.rs.n_max + 2, A.rs.ns_max, A.rs.pairs_max);
    const RobotParams* rob;
    if (!collide_prologue<UNIFORM>(A, smem, L, sc0, n_obj4, &rob)) return;
    const WarpBufs Bf = warp_bufs(smem, L, A);
    const float4* s_scene = reinterpret_cast<const float4*>(smem);
    uint64_t* keys = reinterpret_cast<uint64_t*>(smem + keys_off);

    const TargetDesc& T = R.tg[t];
    const int rid = T.robot, sid = UNIFORM ? 0 : T.scene;
    const int n = rob[rid].n;
    const int64_t b0 = R.b_off[t];
    const int B = (int)(R.b_off[t + 1] - b0);
    const int N = pow2_at_least(B > 0 ? B : 1);
    for (int i = threadIdx.x; i < N; i += blockDim.x) keys[i] = rank_key(R, t, b0, B, n, i, false);
    __syncthreads();
    bitonic_sort(keys, N);
    int ranked = 0;  // candidates with a key (finite score)
    for (int base = 0; base < N; base += blockDim.x)
        ranked += __syncthreads_count(base + (int)threadIdx.x < N && keys[base + threadIdx.x] != kNoKey);
    const int top_k = T.top_k & ~kNearestFlag;

    WarpRobot<SPL> W;
    W.cur = -1;
    W.n_m = W.pairs_m = 0;
    W.bmask = 0;
    unsigned long long tests = 0, btests = 0, ncand = 0;
    if (threadIdx.x == 0) n_found = 0;
    __syncthreads();
    int p0 = 0;
    for (; p0 < ranked && n_found < top_k && (!R.list || p0 < depth); p0 += kWarpsPerBlock) {
        const int p = p0 + warp;
        bool hit = true;
        if (p < ranked) {
            const int64_t c = b0 + (int64_t)(keys[p] & 0xffffffffu);
            unsigned long long t_s = 0, t_b = 0;
            hit = warp_collides<SPL, UNIFORM, GRID>(A, rob, sc0, s_scene, W, Bf, c, rid, sid, t_s, t_b);
            if (lane == 0) {
                tests += t_s;
                btests += t_b;
                ++ncand;
            }
        }
        if (lane == 0) verdict[warp] = hit ? 1 : 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            int f = n_found;
            for (int w = 0; w < kWarpsPerBlock && f < top_k; ++w)
                if (p0 + w < ranked && !verdict[w]) picks[f++] = p0 + w;
            n_found = f;
        }
        __syncthreads();
    }
    const int count = n_found;
    if (A.cnt && lane == 0) {
        atomicAdd(&A.cnt->v[3], tests);
        atomicAdd(&A.cnt->v[6], btests);
        atomicAdd(&A.cnt->v[4], ncand);
    }
    if (R.list && count < top_k && p0 < ranked) {
        // deeper than the bound: the verdicts taken so far are kept (0 free, 1 colliding), the
        // unchecked ranked candidates marked 2 for the collision filter over the listed targets,
        // which spreads them over every SM; the ranking of the listed targets follows it
        for (int q = threadIdx.x; q < ranked; q += blockDim.x) {
            uint8_t v = 2;
            if (q < p0) {
                v = 1;
                for (int r = 0; r < count; ++r) v = picks[r] == q ? 0 : v;
            }
            A.hit[b0 + (int64_t)(keys[q] & 0xffffffffu)] = v;
        }
        if (threadIdx.x == 0) R.list[atomicAdd(R.n_list, 1)] = t;
        return;
    }
    float* oq = R.out_q + R.qe_off[2 * t];
    float* oe = R.out_err + R.qe_off[2 * t + 1];
    for (int q = threadIdx.x; q < count * (n + 2); q += blockDim.x) {
        const int r = q / (n + 2), j = q % (n + 2);
        const int64_t g = b0 + (int64_t)(keys[picks[r]] & 0xffffffffu);
        if (j < n) oq[r * n + j] = R.th[j * R.ld + g];
        else if (j == n) oe[r * 2] = R.perr[g];
        else oe[r * 2 + 1] = R.oerr[g];
    }
    if (threadIdx.x == 0) R.out_count[t] = count;
}

template <int SPL, bool UNIFORM, bool GRID>
bool launch_rank_lazy_t(const CollideArgs& A, const RankArgs& R, int n_obj4, int max_b, int depth, cudaStream_t st) {
    const CollideLayout L =
        collide_smem_layout(UNIFORM ? n_obj4 : 0, A.rs.n, A.rs.n_max + 2, A.rs.ns_max, A.rs.pairs_max);
    const uint32_t keys_off = (L.total + 15u) / 16u * 16u;
    int N = 1;
    while (N < max_b) N <<= 1;
    const size_t smem = keys_off + 8 * (size_t)N;
    if (smem > 220 * 1024) return false;
    static SmemLimit lim;
    allow_dyn_smem(k_rank_lazy<SPL, UNIFORM, GRID>, lim, 220 * 1024);
    k_rank_lazy<SPL, UNIFORM, GRID><<<R.T, kWarpsPerBlock * 32, smem, st>>>(A, R, keys_off, depth);
    return true;
}

template <bool UNIFORM, bool GRID>
bool launch_rank_lazy_s(const CollideArgs& A, const RankArgs& R, int n_obj4, int max_b, int depth, cudaStream_t st) {
    const int ns = A.rs.ns_max;
    if (ns <= 32) return launch_rank_lazy_t<1, UNIFORM, GRID>(A, R, n_obj4, max_b, depth, st);
    if (ns <= 64) return launch_rank_lazy_t<2, UNIFORM, GRID>(A, R, n_obj4, max_b, depth, st);
    if (ns <= 128) return launch_rank_lazy_t<4, UNIFORM, GRID>(A, R, n_obj4, max_b, depth, st);
    return launch_rank_lazy_t<8, UNIFORM, GRID>(A, R, n_obj4, max_b, depth, st);
}

template <int SPL, bool UNIFORM, bool GRID>
void launch_collide_t(const CollideArgs& A, int n_obj4, cudaStream_t st) {
    const size_t smem =
        collide_smem_layout(UNIFORM ? n_obj4 : 0, A.rs.n, A.rs.n_max + 2, A.rs.ns_max, A.rs.pairs_max).total;
    static SmemLimit lim;
    allow_dyn_smem(k_collide<SPL, UNIFORM, GRID>, lim, 227 * 1024);
    const int g = grid_for(A.C, kWarpsPerBlock, 8);
    k_collide<SPL, UNIFORM, GRID><<<g, kWarpsPerBlock * 32, smem, st>>>(A);
}

template <bool UNIFORM, bool GRID>
void launch_collide_s(const CollideArgs& A, int n_obj4, cudaStream_t st) {
    const int ns = A.rs.ns_max;
    if (ns <= 32) launch_collide_t<1, UNIFORM, GRID>(A, n_obj4, st);
    else if (ns <= 64) launch_collide_t<2, UNIFORM, GRID>(A, n_obj4, st);
    else if (ns <= 128) launch_collide_t<4, UNIFORM, GRID>(A, n_obj4, st);
    else launch_collide_t<8, UNIFORM, GRID>(A, n_obj4, st);
}

constexpr int kContactTile = 8;  // configurations per CTA of the contact kernel

// touched[o] = 1 for every obstacle o (spheres in the caller's order, then
// boxes) that overlaps a link sphere of one of the C configurations; the
// world spheres of kContactTile configurations sit in shared memory and each
// thread tests its obstacles against all of them.
__global__ void __launch_bounds__(256) k_contacts(const RobotParams R, const RobotDev rd, const SceneDev sc,
                                                 const int32_t* perm, int64_t C, const float* th, int64_t ld,
                                                 uint8_t* touched) {
    extern __shared__ float4 wsp[];  // [kContactTile][n_sph]
    const int ns = rd.n_sph;
    const int64_t c0 = (int64_t)blockIdx.x * kContactTile;
    const int nc = (int)min((int64_t)kContactTile, C - c0);
    if (threadIdx.x < nc) {
        const int64_t c = c0 + threadIdx.x;
        float4* w = wsp + threadIdx.x * ns;
        Frame F = frame_identity();
        for (int b = 0; b <= R.n + 1; ++b) {
            if (b >= 1 && b <= R.n) fk_step(R, b - 1, th[(b - 1) * ld + c], F);
            const Frame E = b == R.n + 1 ? fk_flange(R, F) : F;
            const int2 rg = rd.range[b];
            for (int i = rg.x; i < rg.x + rg.y; ++i) w[i] = to_world(E, rd.sph[i]);
        }
    }
    __syncthreads();
    const int n_obj = sc.n_sph + sc.n_box;
    for (int o = threadIdx.x; o < n_obj; o += blockDim.x) {
        bool hit = false;
        if (o < sc.n_sph) {
            const float4 s = sc.obj[o];
            for (int i = 0; i < nc * ns && !hit; ++i) hit = sph_sph(wsp[i], s);
            if (hit) touched[perm[o]] = 1;
        } else {
            const int k = o - sc.n_sph;
            const float4 lo = sc.obj[sc.n_sph + 2 * k], hi = sc.obj[sc.n_sph + 2 * k + 1];
            for (int i = 0; i < nc * ns && !hit; ++i) hit = sph_box(wsp[i], lo, hi);
            if (hit) touched[o] = 1;
        }
    }
}

}  // namespace

void launch_contacts(const RobotParams& R, const RobotDev& rd, const SceneDev& sc, const int32_t* perm, int64_t C,
                     const float* th, int64_t ld, uint8_t* touched, cudaStream_t st) {
    if (C <= 0 || rd.n_sph <= 0 || sc.n_sph + sc.n_box <= 0) return;
    const size_t smem = sizeof(float4) * kContactTile * (size_t)rd.n_sph;
    static SmemLimit lim;
    allow_dyn_smem(k_contacts, lim, sizeof(float4) * kContactTile * (size_t)HJCD_MAX_SPHERES);
    const int64_t blocks = (C + kContactTile - 1) / kContactTile;
    k_contacts<<<(unsigned)blocks, 256, smem, st>>>(R, rd, sc, perm, C, th, ld, touched);
}

bool launch_rank_lazy(const CollideArgs& A, const RankArgs& R, int max_b, int depth, cudaStream_t st) {
    if (R.T <= 0 || A.rs.ns_max <= 0 || !R.tg || !R.qe_off) return false;
    const bool uni = A.uniform && A.rs.n == 1 && A.n_scenes <= 1 && A.max_obj4 <= kMaxStagedObj4;
    const int n4 = A.n_scenes == 1 ? A.max_obj4 : 0;
    if (uni && A.has_grid) return launch_rank_lazy_s<true, true>(A, R, n4, max_b, depth, st);
    if (uni) return launch_rank_lazy_s<true, false>(A, R, n4, max_b, depth, st);
    if (A.has_grid) return launch_rank_lazy_s<false, true>(A, R, 0, max_b, depth, st);
    return launch_rank_lazy_s<false, false>(A, R, 0, max_b, depth, st);
}

// One robot and one scene (or none) for every candidate, with the scene small
// enough to stage: the uniform kernel (scene staged into shared memory, counts
// as launch parameters); otherwise the mixed kernel.  Launches with a gridded
// scene take the variants with the grid query.
void launch_collide(const CollideArgs& A, cudaStream_t st) {
    if (A.C <= 0 || A.rs.ns_max <= 0) return;
    const bool uni = A.uniform && A.rs.n == 1 && A.n_scenes <= 1 && A.max_obj4 <= kMaxStagedObj4;
    const int n4 = A.n_scenes == 1 ? A.max_obj4 : 0;
    if (uni && A.has_grid) launch_collide_s<true, true>(A, n4, st);
    else if (uni) launch_collide_s<true, false>(A, n4, st);
    else if (A.has_grid) launch_collide_s<false, true>(A, 0, st);
    else launch_collide_s<false, false>(A, 0, st);
}

}  // namespace hjcd

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

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i)
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


template <int SPL, bool UNIFORM, bool GRID>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_collide(const CollideArgs A) {
    constexpr bool STAGED = UNIFORM;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const SceneDev sc0 = A.n_scenes > 0 ? A.scenes[0] : SceneDev{nullptr, 0, 0};
    const int n_obj4 = STAGED ? sc0.n_sph + 2 * sc0.n_box : 0;
    if (n_obj4 > (STAGED ? A.max_obj4 : 0)) {  // the scene outgrew the shared memory the host sized
        if (threadIdx.x == 0) atomicExch(A.err_flag, 2);
        return;
    }
    const int nb_max = A.rs.n_max + 2;
    const CollideLayout L = collide_smem_layout(n_obj4, A.rs.n, nb_max, A.rs.ns_max, A.rs.pairs_max);
    float4* s_scene = reinterpret_cast<float4*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    unsigned char* wb = smem + L.warp + warp * L.warp_bytes;
    float4* wsph = reinterpret_cast<float4*>(wb);
    float4* wco = wsph + A.rs.ns_max;
    int2* wrange = reinterpret_cast<int2*>(wco + nb_max);
    int2* wpairs = wrange + nb_max;
    int* list = reinterpret_cast<int*>(wpairs + A.rs.pairs_max);

    // stage the obstacles with one bulk copy, the robots' kinematic tables with plain loads
    const uint32_t bytes = 16u * (uint32_t)n_obj4;
    if (STAGED) {
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
    const RobotParams* rob = stage_robots(smem + L.robots, A.rs);
    if (STAGED) {
        const bool staged = mbar_wait_bounded(bar, 0);
        if (__syncthreads_or(!staged)) {
            // give up: flag the error, give the copy one more bounded wait, return
            if (threadIdx.x == 0) {
                atomicExch(A.err_flag, 1);
                mbar_wait_bounded(bar, 0);
            }
            return;
        }
    }

    // this lane's fine spheres (body frame) and bodies, its bounding sphere
    // (body lane), for the robot of the warp's current candidate
    float4 ls[SPL];
    int lb[SPL];
    float4 lco = make_float4(0.f, 0.f, 0.f, 0.f);
    int cur = -1, n_m = 0, pairs_m = 0;  // robot of a mixed launch: DoF, checked pairs
    unsigned bmask = 0;                  // its bodies that carry spheres (bit per body, n + 2 <= 26)

    unsigned long long tests = 0, btests = 0, ncand = 0;
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    int rid = 0, sid = 0;
    bool tvalid = true;
    for (int64_t c = (int64_t)blockIdx.x * kWarpsPerBlock + warp; c < A.C; c += nwarps) {
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
        if (rid != cur) {
            cur = rid;
            const RobotDev rd = A.rs.rd[rid];
            n_m = rob[rid].n;
            pairs_m = rd.n_pairs;
            const int ns = rd.n_sph, nbr = n_m + 2;
#pragma unroll
            for (int q = 0; q < SPL; ++q) {
                const int i = lane + 32 * q;
                lb[q] = i < ns ? __ldg(rd.body + i) : -1;
                ls[q] = i < ns ? __ldg(rd.sph + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            lco = lane < nbr ? __ldg(rd.coarse + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();
            for (int i = lane; i < nbr; i += 32) wrange[i] = __ldg(rd.range + i);
            for (int i = lane; i < pairs_m; i += 32) wpairs[i] = __ldg(rd.pairs + i);
            __syncwarp();
            bmask = __ballot_sync(0xffffffffu, lane < nbr && wrange[lane].y > 0);  // bodies with spheres
        }
        const RobotParams& R = rob[rid];
        const int n = UNIFORM ? A.u_n : n_m, nb = n + 2, n_pairs = UNIFORM ? A.u_pairs : pairs_m;
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
        for (int q = 0; q < SPL; ++q) ws[q] = ls[q];
        float4 wc = lco;
        Frame F = frame_identity();
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            fk_step(R, j, A.th[j * A.ld + c], F);
#pragma unroll
            for (int q = 0; q < SPL; ++q)
                if (lb[q] == j + 1) ws[q] = to_world(F, ls[q]);
            if (lane == j + 1) wc = to_world(F, lco);
        }
        const Frame E = fk_flange(R, F);
#pragma unroll
        for (int q = 0; q < SPL; ++q) {
            if (lb[q] == n + 1) ws[q] = to_world(E, ls[q]);
            if (lb[q] >= 0) wsph[lane + 32 * q] = ws[q];
        }
        if (lane == n + 1) wc = to_world(E, lco);
        if (lane < nb) wco[lane] = wc;
        __syncwarp();

        bool hit = false;
        unsigned long long t_s = 0, t_b = 0;  // tests of this candidate (uniform over the warp)

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
        const int nbs = __popc(bmask);
        for (int o0 = 0; o0 < n_osph && !hit && !(GRID && gcell); o0 += 32) {
            const int o = o0 + lane;
            const bool valid = o < n_osph;
            const float4 s = valid ? ld_obj<STAGED>(obj, o) : make_float4(0.f, 0.f, 0.f, 0.f);
            unsigned bm = 0;
            if (valid)
                for (unsigned bb = bmask; bb; bb &= bb - 1u) {
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
                for (unsigned bb = bmask; bb; bb &= bb - 1u) {
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

template <int SPL, bool UNIFORM, bool GRID>
void launch_collide_t(const CollideArgs& A, int n_obj4, cudaStream_t st) {
    const size_t smem =
        collide_smem_layout(UNIFORM ? n_obj4 : 0, A.rs.n, A.rs.n_max + 2, A.rs.ns_max, A.rs.pairs_max).total;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_collide<SPL, UNIFORM, GRID>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_set = true;
    }
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
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_contacts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t blocks = (C + kContactTile - 1) / kContactTile;
    k_contacts<<<(unsigned)blocks, 256, smem, st>>>(R, rd, sc, perm, C, th, ld, touched);
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

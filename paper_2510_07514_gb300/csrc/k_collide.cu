// k_collide.cu -- sphere collision filter (Sec. V-C), one warp per candidate.
//
// Each lane owns up to SPL of the robot's link spheres (sphere lane + 32 q).
// Every lane walks the kinematic chain for the candidate and moves its own
// spheres into the world frame; the warp publishes them to shared memory for
// the self-collision pairs.  Obstacles (spheres, then boxes) are staged once
// per CTA into shared memory by a single bulk asynchronous copy (TMA,
// cp.async.bulk) completing on an mbarrier, and are read by the whole warp
// as broadcasts.  The warp votes after every few obstacles and stops at the
// first overlap -- a candidate is discarded as soon as any pair overlaps.
//
// Overlap: |c1 - c2|^2 < (r1 + r2)^2 for spheres; for a box, the squared
// distance from the centre to its clamp into the box below r^2.
#include "hjcd_internal.cuh"

namespace hjcd {

namespace {

constexpr int kWarpsPerBlock = 8;
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

__device__ __forceinline__ float4 to_world(const Frame& F, float4 s) {
    const V3 w = fma3(s.z, F.c2, fma3(s.y, F.c1, fma3(s.x, F.c0, F.p)));
    return make_float4(w.x, w.y, w.z, s.w);
}

template <int SPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_collide(const RobotParams R, const CollideArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int n_obj4 = A.n_osph + 2 * A.n_obox;
    const int ns = R.n_sph;
    float4* scene = reinterpret_cast<float4*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 16 * (size_t)n_obj4);
    float4* wall = reinterpret_cast<float4*>(smem + 16 * (size_t)n_obj4 + 16);
    int32_t* sbody = reinterpret_cast<int32_t*>(wall + kWarpsPerBlock * ns);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* wsph = wall + warp * ns;

    // stage the obstacles with one bulk copy; the sphere-to-body table with plain loads
    const uint32_t bytes = 16u * (uint32_t)n_obj4;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bytes > 0) {
            mbar_arrive_expect_tx(bar, bytes);
            bulk_g2s(scene, A.scene, bytes, bar);
        } else {
            mbar_arrive(bar);
        }
    }
    for (int i = threadIdx.x; i < ns; i += blockDim.x) sbody[i] = A.rsph_body[i];
    bool staged = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!staged)) {
        // give up: flag the error, give the copy one more bounded wait, return
        if (threadIdx.x == 0) {
            atomicExch(A.err_flag, 1);
            mbar_wait_bounded(bar, 0);
        }
        return;
    }

    // this lane's spheres (body frame), bodies and self-collision masks
    float4 ls[SPL];
    int lb[SPL];
    uint32_t pm[SPL];
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
        const int i = lane + 32 * q;
        if (i < ns) {
            ls[q] = A.rsph[i];
            lb[q] = sbody[i];
            pm[q] = A.pair_mask[lb[q]];
        } else {
            ls[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            lb[q] = -1;
            pm[q] = 0u;
        }
    }

    unsigned long long tests = 0, btests = 0, ncand = 0;
    const int n = R.n;
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t c = (int64_t)blockIdx.x * kWarpsPerBlock + warp; c < A.C; c += nwarps) {
        // world positions of this lane's spheres
        float4 ws[SPL];
#pragma unroll
        for (int q = 0; q < SPL; ++q) ws[q] = ls[q];  // body 0: the base frame is the world frame
        Frame F = frame_identity();
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            fk_step(R, j, A.th[j * A.ld + c], F);
#pragma unroll
            for (int q = 0; q < SPL; ++q)
                if (lb[q] == j + 1) ws[q] = to_world(F, ls[q]);
        }
        const Frame E = fk_flange(R, F);
#pragma unroll
        for (int q = 0; q < SPL; ++q) {
            if (lb[q] == n + 1) ws[q] = to_world(E, ls[q]);
            if (lb[q] >= 0) wsph[lane + 32 * q] = ws[q];
        }
        __syncwarp();

        bool hit = false;
        unsigned long long my_tests = 0;
        // self-collision: each unordered pair (i < j) of spheres on bodies not ignored
        for (int j = 0; j < ns; ++j) {
            const float4 o = wsph[j];
            const int bj = sbody[j];
#pragma unroll
            for (int q = 0; q < SPL; ++q) {
                if (lane + 32 * q < j && ((pm[q] >> bj) & 1u)) {
                    const float dx = ws[q].x - o.x, dy = ws[q].y - o.y, dz = ws[q].z - o.z;
                    const float rr = ws[q].w + o.w;
                    hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
                    ++my_tests;
                }
            }
        }
        hit = __any_sync(0xffffffffu, hit);
        int o_sph = 0, o_box = 0;
        if (!hit) {
            for (int o = 0; o < A.n_osph; ++o) {
                const float4 s = scene[o];
#pragma unroll
                for (int q = 0; q < SPL; ++q) {
                    if (lb[q] >= 0) {
                        const float dx = ws[q].x - s.x, dy = ws[q].y - s.y, dz = ws[q].z - s.z;
                        const float rr = ws[q].w + s.w;
                        hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
                    }
                }
                ++o_sph;
                if ((o & 7) == 7 && __any_sync(0xffffffffu, hit)) break;
            }
            hit = __any_sync(0xffffffffu, hit);
        }
        if (!hit) {
            const float4* box = scene + A.n_osph;
            for (int o = 0; o < A.n_obox; ++o) {
                const float4 lo = box[2 * o], hi = box[2 * o + 1];
#pragma unroll
                for (int q = 0; q < SPL; ++q) {
                    if (lb[q] >= 0) {
                        const float dx = ws[q].x - clampf(ws[q].x, lo.x, hi.x);
                        const float dy = ws[q].y - clampf(ws[q].y, lo.y, hi.y);
                        const float dz = ws[q].z - clampf(ws[q].z, lo.z, hi.z);
                        hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < ws[q].w * ws[q].w;
                    }
                }
                ++o_box;
                if ((o & 7) == 7 && __any_sync(0xffffffffu, hit)) break;
            }
            hit = __any_sync(0xffffffffu, hit);
        }
        if (lane == 0) {
            A.hit[c] = hit ? 1 : 0;
            tests += (unsigned long long)o_sph * (unsigned long long)ns;
            btests += (unsigned long long)o_box * (unsigned long long)ns;
            ++ncand;
        }
        tests += my_tests;
        __syncwarp();
    }
    if (A.cnt) {
        tests = warp_sum(tests);
        btests = warp_sum(btests);
        ncand = warp_sum(ncand);
        if (lane == 0) {
            atomicAdd(&A.cnt->v[3], tests);
            atomicAdd(&A.cnt->v[6], btests);
            atomicAdd(&A.cnt->v[4], ncand);
        }
    }
}

template <int SPL>
void launch_collide_t(const RobotParams& R, const CollideArgs& A, cudaStream_t st) {
    const size_t smem = 16 * (size_t)(A.n_osph + 2 * A.n_obox) + 16 + (size_t)kWarpsPerBlock * R.n_sph * 16 +
                        (size_t)R.n_sph * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_collide<SPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_set = true;
    }
    const int g = grid_for(A.C, kWarpsPerBlock, 8);
    k_collide<SPL><<<g, kWarpsPerBlock * 32, smem, st>>>(R, A);
}

}  // namespace

size_t collide_smem_bytes(int n_sph, int n_osph, int n_obox) {
    return 16 * (size_t)(n_osph + 2 * n_obox) + 16 + (size_t)kWarpsPerBlock * n_sph * 16 + (size_t)n_sph * 4;
}

void launch_collide(const RobotParams& R, const CollideArgs& A, cudaStream_t st) {
    if (A.C <= 0 || R.n_sph <= 0) return;
    if (R.n_sph <= 32) launch_collide_t<1>(R, A, st);
    else if (R.n_sph <= 64) launch_collide_t<2>(R, A, st);
    else if (R.n_sph <= 128) launch_collide_t<4>(R, A, st);
    else launch_collide_t<8>(R, A, st);
}

}  // namespace hjcd

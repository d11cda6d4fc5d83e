// k_misc.cu -- forward-kinematics stage kernel (Eq. fk), raw blocks of the
// kernels' Philox generator, and the FP32 FMA throughput probe used as the
// CUDA-core roofline denominator.
#include "hjcd_internal.cuh"

namespace hjcd {

namespace {

__global__ void __launch_bounds__(128) k_fk(const RobotParams R, int64_t C, const float* th_in, int64_t ld,
                                            float* out) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        Frame F = frame_identity();
#pragma unroll 1
        for (int j = 0; j < R.n; ++j) fk_step(R, j, th_in[j * ld + c], F);
        const Frame E = fk_flange(R, F);
        const Q4 q = quat_from_frame(E);
        float* o = out + 7 * c;
        o[0] = E.p.x;
        o[1] = E.p.y;
        o[2] = E.p.z;
        o[3] = q.w;
        o[4] = q.v.x;
        o[5] = q.v.y;
        o[6] = q.v.z;
    }
}

// out[i] = Philox4x32-10 block at counter ctr[i] under (k0, k1): the generator every kernel draws from
__global__ void __launch_bounds__(256) k_philox(int64_t n, const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = philox(ctr[i], k0, k1);
}

constexpr int kChains = 8, kUnroll = 16;

// kChains independent FMA chains per thread, kUnroll steps per iteration
__global__ void __launch_bounds__(256) k_ffma(float* sink, int iters) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-7f;
    const float m = 0.9999999f, b = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == 1234.5f) sink[blockIdx.x] = s;  // never true; keeps the chains alive
}

}  // namespace

void launch_fk(const RobotParams& R, int64_t C, const float* th, int64_t ld, float* out, cudaStream_t st) {
    if (C <= 0) return;
    k_fk<<<grid_for(C, 128), 128, 0, st>>>(R, C, th, ld, out);
}

void launch_philox(int64_t n, const uint32_t* ctr, uint64_t key, uint32_t* out, cudaStream_t st) {
    if (n <= 0) return;
    k_philox<<<grid_for(n, 256), 256, 0, st>>>(n, reinterpret_cast<const uint4*>(ctr), (uint32_t)key,
                                               (uint32_t)(key >> 32), reinterpret_cast<uint4*>(out));
}

void launch_ffma(float* sink, int iters, int blocks, cudaStream_t st) { k_ffma<<<blocks, 256, 0, st>>>(sink, iters); }

int ffma_flops_per_thread_iter() { return 2 * kChains * kUnroll; }

}  // namespace hjcd

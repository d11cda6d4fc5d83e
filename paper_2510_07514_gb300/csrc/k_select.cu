// k_select.cu -- per-target selection: top-K and perturbed duplication
// (Alg. 2), ranking of the collision-free candidates (Alg. 2, final
// step), and packing of target poses.
//
// One CTA per target sorts 64-bit keys (score bits << 32 | index) in shared
// memory with a bitonic network; scores are non-negative, so their IEEE bit
// patterns order like the values, and the index in the low word breaks ties
// toward the lower candidate.  Invalid entries (padding, collisions, NaN)
// get the all-ones key and sort last.
#include "hjcd_internal.cuh"

namespace hjcd {

namespace {

constexpr int kSelThreads = 512;

__global__ void __launch_bounds__(kSelThreads) k_topk_dup(const DupArgs A) {
    extern __shared__ uint64_t keys[];
    const int t = blockIdx.x;
    const int64_t m0 = A.m_off[t];
    const int M = (int)(A.m_off[t + 1] - m0);
    if (M <= 0) return;
    const int N = pow2_at_least(M);
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        keys[i] = i < M ? score_key(A.score_M[m0 + i], (uint32_t)i) : kNoKey;
    __syncthreads();
    bitonic_sort(keys, N);

    const int K = max(1, M / A.ratio), copies = M / K, B = K * copies;
    const int64_t b0 = A.b_off[t];
    const TargetDesc T = A.tg[t];
    const RobotParams& R = A.rs.rp[T.robot];
    const int n = R.n;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const int i = b % K;  // copy r = b / K of kept seed i
        const uint32_t src = (uint32_t)(keys[i] & 0xffffffffu);
#pragma unroll 1
        for (int q = 0; 2 * q < n; ++q) {
            const float2 z = normal_pair(T, (uint32_t)b, kPhaseDup, 0, q);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = 2 * q + h;
                if (j < n)
                    A.th_B[j * A.ld_B + b0 + b] =
                        clampf(fmaf(A.sigma, h ? z.y : z.x, A.th_M[j * A.ld_M + m0 + src]), R.lim[j].x, R.lim[j].y);
            }
        }
        if (A.src_B) A.src_B[b0 + b] = (int32_t)src;
    }
}

__global__ void __launch_bounds__(kSelThreads) k_rank(const RankArgs A) {
    extern __shared__ uint64_t keys[];
    int t = blockIdx.x;
    if (A.list) {  // the targets the bounded lazy pass left unfinished
        if (t >= *A.n_list) return;
        t = A.list[t];
    }
    const int64_t b0 = A.b_off[t];
    const int B = (int)(A.b_off[t + 1] - b0);
    int count = 0;
    if (B > 0) {
        const int N = pow2_at_least(B);
        const int n = A.rs.rp[A.tg ? A.tg[t].robot : 0].n;
        const int tk = A.tg ? A.tg[t].top_k : A.top_k;
        for (int i = threadIdx.x; i < N; i += blockDim.x) keys[i] = rank_key(A, t, b0, B, n, i, true);
        __syncthreads();
        bitonic_sort(keys, N);
        const int top_k = tk & ~kNearestFlag;
        const int lim = min(top_k, B);
        for (int r = 0; r < lim; ++r) count += keys[r] != kNoKey;
        float* oq = A.out_q + (A.qe_off ? A.qe_off[2 * t] : (int64_t)t * top_k * n);
        float* oe = A.out_err + (A.qe_off ? A.qe_off[2 * t + 1] : (int64_t)t * top_k * 2);
        for (int q = threadIdx.x; q < count * (n + 2); q += blockDim.x) {
            const int r = q / (n + 2), j = q % (n + 2);
            const int64_t g = b0 + (int64_t)(keys[r] & 0xffffffffu);
            if (j < n) oq[r * n + j] = A.th[j * A.ld + g];
            else if (j == n) oe[r * 2] = A.perr[g];
            else oe[r * 2 + 1] = A.oerr[g];
        }
    }
    if (threadIdx.x == 0) A.out_count[t] = count;
}

__global__ void __launch_bounds__(kSelThreads) k_shard_topk(const ShardTopkArgs A) {
    extern __shared__ uint64_t keys[];
    const int t = blockIdx.x;
    const int64_t m0 = A.off[t];
    const int M = (int)(A.off[t + 1] - m0);
    const int N = pow2_at_least(M > 0 ? M : 1);
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        keys[i] = i < M ? score_key(A.score[m0 + i], (uint32_t)i) : kNoKey;
    __syncthreads();
    bitonic_sort(keys, N);
    const int n = A.rs.rp[A.tg[t].robot].n;
    for (int q = threadIdx.x; q < A.K * (n + 2); q += blockDim.x) {
        const int r = q / (n + 2), j = q % (n + 2);
        const uint64_t key = r < N ? keys[r] : kNoKey;
        const bool ok = r < M && key != kNoKey;
        const uint32_t src = (uint32_t)(key & 0xffffffffu);
        const int64_t o = (int64_t)t * A.K + r;
        if (j < n) A.out_th[o * A.ld_n + j] = ok ? A.th[j * A.ld + m0 + src] : 0.0f;
        else if (j == n) A.out_s[o] = ok ? A.score[m0 + src] : __int_as_float(0x7f800000);
        else A.out_i[o] = ok ? A.seed_base + (int32_t)src : -1;
    }
}

__global__ void __launch_bounds__(kSelThreads) k_topk_merge(const MergeArgs A) {
    extern __shared__ uint64_t keys[];
    const int t = blockIdx.x;
    const int LK = A.L * A.K;
    const int N = pow2_at_least(LK);
    // key: score bits, then the seed index (ties to the lower index); the list slot is found again below
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        uint64_t k = kNoKey;
        if (i < LK) {
            const int l = i / A.K, r = i % A.K;
            const int64_t e = ((int64_t)l * A.T + t) * A.K + r;
            const int32_t idx = A.in_i[e];
            if (idx >= 0) k = score_key(A.in_s[e], (uint32_t)idx);
        }
        keys[i] = k;
    }
    __syncthreads();
    bitonic_sort(keys, N);
    // the i-th best: locate its list entry (seed indices are unique within a target)
    for (int r = threadIdx.x; r < A.K; r += blockDim.x) {
        const uint64_t key = keys[r];
        const int64_t o = (int64_t)t * A.K + r;
        if (key == kNoKey) {
            A.out_s[o] = __int_as_float(0x7f800000);
            A.out_i[o] = -1;
            for (int j = 0; j < A.n; ++j) A.out_th[o * A.n + j] = 0.0f;
            continue;
        }
        const int32_t idx = (int32_t)(key & 0xffffffffu);
        int64_t e = -1;
        for (int l = 0; l < A.L && e < 0; ++l)
            for (int q = 0; q < A.K; ++q) {
                const int64_t f = ((int64_t)l * A.T + t) * A.K + q;
                if (A.in_i[f] == idx) {
                    e = f;
                    break;
                }
            }
        A.out_s[o] = A.in_s[e];
        A.out_i[o] = idx;
        for (int j = 0; j < A.n; ++j) A.out_th[o * A.n + j] = A.in_th[e * A.n + j];
    }
}

__global__ void __launch_bounds__(kSelThreads) k_dup_kept(const KeptDupArgs A) {
    const int t = blockIdx.x;
    const int64_t b0 = A.b_off[t];
    const int B = (int)(A.b_off[t + 1] - b0);
    const TargetDesc T = A.tg[t];
    const RobotParams& R = A.rs.rp[T.robot];
    const int n = R.n;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const int i = b % A.K;  // copy r = b / K of kept seed i
        const float* src = A.kept + ((int64_t)t * A.K + i) * n;
#pragma unroll 1
        for (int q = 0; 2 * q < n; ++q) {
            const float2 z = normal_pair(T, (uint32_t)b, kPhaseDup, 0, q);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = 2 * q + h;
                if (j < n) A.th_B[j * A.ld_B + b0 + b] = clampf(fmaf(A.sigma, h ? z.y : z.x, src[j]), R.lim[j].x, R.lim[j].y);
            }
        }
    }
}

__global__ void k_pack_targets(const float* pq7, int T, const TargetDesc* meta, const TargetDesc tmpl,
                               TargetDesc* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const float* s = pq7 + 7 * (int64_t)t;
    const float qw = s[3], qx = s[4], qy = s[5], qz = s[6];
    const float nn = qw * qw + qx * qx + qy * qy + qz * qz;
    const bool ok = nn > 0.0f && isfinite(nn);
    const float r = ok ? rsqrtf(nn) : 0.0f;
    TargetDesc d;
    if (meta) {
        d = meta[t];
    } else {
        d = tmpl;
        d.t_local = tmpl.t_local + t;  // the template holds the index of the first target
    }
    d.p[0] = s[0];
    d.p[1] = s[1];
    d.p[2] = s[2];
    d.q[0] = ok ? qw * r : 1.0f;
    d.q[1] = qx * r;
    d.q[2] = qy * r;
    d.q[3] = qz * r;
    if (!ok) d.eps_pos = -1.0f;  // a zero quaternion marks the target invalid
    out[t] = d;
}

int smem_for(int m) {
    int N = 1;
    while (N < m) N <<= 1;
    return N * (int)sizeof(uint64_t);
}


}  // namespace

void launch_topk_dup(const DupArgs& A, int max_m, cudaStream_t st) {
    if (A.T <= 0 || max_m <= 0) return;
    const int sm = smem_for(max_m);
    static SmemLimit lim;
    allow_dyn_smem(k_topk_dup, lim, smem_for(HJCD_MAX_SAMPLES));
    k_topk_dup<<<A.T, kSelThreads, sm, st>>>(A);
}

void launch_rank(const RankArgs& A, int max_b, cudaStream_t st) {
    if (A.T <= 0) return;
    const int sm = smem_for(max_b > 0 ? max_b : 1);
    static SmemLimit lim;
    allow_dyn_smem(k_rank, lim, smem_for(HJCD_MAX_SAMPLES));
    k_rank<<<A.T, kSelThreads, sm, st>>>(A);
}

void launch_shard_topk(const ShardTopkArgs& A, int max_m, cudaStream_t st) {
    if (A.T <= 0) return;
    const int sm = smem_for(max_m > 0 ? max_m : 1);
    static SmemLimit lim;
    allow_dyn_smem(k_shard_topk, lim, smem_for(HJCD_MAX_SAMPLES));
    k_shard_topk<<<A.T, kSelThreads, sm, st>>>(A);
}

void launch_topk_merge(const MergeArgs& A, cudaStream_t st) {
    if (A.T <= 0 || A.L <= 0 || A.K <= 0) return;
    const int sm = smem_for(A.L * A.K);
    static SmemLimit lim;
    allow_dyn_smem(k_topk_merge, lim, 227 * 1024);
    k_topk_merge<<<A.T, kSelThreads, sm, st>>>(A);
}

void launch_dup_kept(const KeptDupArgs& A, cudaStream_t st) {
    if (A.T <= 0) return;
    k_dup_kept<<<A.T, kSelThreads, 0, st>>>(A);
}

void launch_pack_targets(const float* pq7, int T, const TargetDesc* meta, const TargetDesc& tmpl, TargetDesc* out,
                         cudaStream_t st) {
    if (T <= 0) return;
    k_pack_targets<<<(T + 127) / 128, 128, 0, st>>>(pq7, T, meta, tmpl, out);
}

}  // namespace hjcd

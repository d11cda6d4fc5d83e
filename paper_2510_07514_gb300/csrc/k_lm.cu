// k_lm.cu -- PJ-IK (Sec. V-B, Alg. 4): persistent, warp-cooperative.
//
// Per iteration and candidate: one kinematics pass with frames gives the
// 6 x n geometric Jacobian (Eq. jacobian) and the residual; W normalises the
// Jacobian's rows (orientation rows also scaled by eps_pos / eps_ori).  The
// damped normal equations of Eq. normal-eqs, ((WJ)^T (WJ) + lambda D) d =
// (WJ)^T W r with D = diag((WJ)^T (WJ)), are solved in their 6 x 6
// push-through form
//     d = S Ah^T (Ah Ah^T + lambda I)^-1 W r,   Ah = WJ S,  S = D^(-1/2),
// an exact identity for lambda > 0, so one 6 x 6 Cholesky factorisation runs
// per candidate whatever n is.  The step is clamped to the trust region and
// validated by the backtracking line search of Eq. line-search; failing that,
// the dogleg step (Eq. dogleg), then the single-coordinate step
// (Eq. single-coord) with the same line search, and finally a random
// perturbation.
//
// Mapping.  Each lane of a warp owns one candidate at a time and takes the
// next one from a global queue when its candidate finishes, so lanes never
// idle while work remains.  Line-search trials are where candidates diverge
// (a failing candidate needs up to 2(A+1)+1 extra kinematics passes), so only
// the full-step trial is evaluated by its owner; the remaining trials of all
// failing lanes of the warp are spread over the 32 lanes (each trial is an
// independent kinematics pass), and each owner then takes the first trial
// that lowered its cost -- the same step the sequential search accepts.
// Per-lane state (joint vector, trial direction, weighted Jacobian, W, W r,
// cost, target row, trial outcomes) lives in shared memory as structure of
// arrays over the lanes, laid out for the largest chain of the launch; joint
// loops are not unrolled, which keeps the kernel small enough for the
// instruction cache at any n.  Each candidate uses its target's robot (the
// launch's robot tables sit in shared memory), also when another lane
// evaluates one of its trials.
#include <algorithm>

#include "hjcd_internal.cuh"

namespace hjcd {

namespace {

constexpr int kLmWarps = 4;  // default warps per CTA; 2 and 8 also built
constexpr int kMaxTrials = 32;  // A + 1 <= 32 (validated by the host)

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

// words of per-warp shared state for an n-joint chain
__host__ __device__ constexpr int lm_warp_words(int n) { return (8 * n + 14) * 32 + kMaxTrials * 32 / 4 + 32; }

// Per-warp state, field[...][lane] (each lane's own accesses conflict-free);
// n is the layout's chain length (the launch's largest).
struct LmW {
    float* f;
    int n;
    __device__ __forceinline__ float& th(int j, int l) const { return f[j * 32 + l]; }
    __device__ __forceinline__ float& d(int j, int l) const { return f[(n + j) * 32 + l]; }
    __device__ __forceinline__ float& jw(int r, int i, int l) const { return f[(2 * n + r * n + i) * 32 + l]; }
    __device__ __forceinline__ float& W(int r, int l) const { return f[(8 * n + r) * 32 + l]; }
    __device__ __forceinline__ float& b(int r, int l) const { return f[(8 * n + 6 + r) * 32 + l]; }
    __device__ __forceinline__ float& cost0(int l) const { return f[(8 * n + 12) * 32 + l]; }
    __device__ __forceinline__ int& t(int l) const { return reinterpret_cast<int*>(f)[(8 * n + 13) * 32 + l]; }
    __device__ __forceinline__ uint8_t& ok(int i, int l) const {
        return reinterpret_cast<uint8_t*>(f + (8 * n + 14) * 32)[i * 32 + l];
    }
    __device__ __forceinline__ int& list(int l) const {
        return reinterpret_cast<int*>(f + (8 * n + 14) * 32 + kMaxTrials * 32 / 4)[l];
    }
};

// In-place Cholesky of a packed 6 x 6 symmetric positive-definite matrix
// (lower triangle, row by row); inv receives the reciprocal pivots.  One
// template instance per column keeps every index a compile-time constant, so
// the matrix stays in registers.
template <int J>
__device__ __forceinline__ void chol_col(float (&a)[21], float (&inv)[6]) {
    float s = a[tri(J, J)];
#pragma unroll
    for (int k = 0; k < J; ++k) s = fmaf(-a[tri(J, k)], a[tri(J, k)], s);
    const float r = rsqrtf(fmaxf(s, 1e-30f));
    a[tri(J, J)] = s * r;
    inv[J] = r;
#pragma unroll
    for (int i = J + 1; i < 6; ++i) {
        float t = a[tri(i, J)];
#pragma unroll
        for (int k = 0; k < J; ++k) t = fmaf(-a[tri(i, k)], a[tri(J, k)], t);
        a[tri(i, J)] = t * r;
    }
}

__device__ __forceinline__ void chol6(float (&a)[21], float (&inv)[6]) {
    chol_col<0>(a, inv);
    chol_col<1>(a, inv);
    chol_col<2>(a, inv);
    chol_col<3>(a, inv);
    chol_col<4>(a, inv);
    chol_col<5>(a, inv);
}

__device__ __forceinline__ void chol6_solve(const float (&L)[21], const float (&inv)[6], const float (&b)[6],
                                            float (&x)[6]) {
    float y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float t = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t = fmaf(-L[tri(i, k)], y[k], t);
        y[i] = t * inv[i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        float t = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) t = fmaf(-L[tri(k, i)], x[k], t);
        x[i] = t * inv[i];
    }
}

struct Y6 {
    float v[6];
};

// Solve M y = b with M the 6 x 6 sum over the joints of col col^T plus reg I,
// for lane l's weighted Jacobian columns.  lm: the columns are first weighted
// by the rows' W (and stored back, so the smem Jacobian becomes W J) and then
// scaled to unit length (S = D^-1/2 of the push-through LM step); otherwise
// they are used as stored (the dogleg's Gauss-Newton system on W J).
__device__ __noinline__ Y6 normal_solve(const LmW S, int l, int n, bool lm, float reg, Y6 w, Y6 b) {
    float M[21], inv[6];
#pragma unroll
    for (int q = 0; q < 21; ++q) M[q] = 0.0f;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        float col[6], dd = 1e-9f;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            col[r] = S.jw(r, i, l);
            if (lm) {
                col[r] *= w.v[r];
                S.jw(r, i, l) = col[r];
                dd = fmaf(col[r], col[r], dd);
            }
        }
        if (lm) {
            const float rs = rsqrtf(dd);
#pragma unroll
            for (int r = 0; r < 6; ++r) col[r] *= rs;
        }
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int q = 0; q <= r; ++q) M[tri(r, q)] = fmaf(col[r], col[q], M[tri(r, q)]);
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) M[tri(r, r)] += reg;
    chol6(M, inv);
    Y6 y;
    chol6_solve(M, inv, b.v, y.v);
    return y;
}

// alpha_i = 1 / beta^i by repeated division (the same bits on every lane)
__device__ __forceinline__ float ls_alpha(int i, float beta) {
    float a = 1.0f;
    for (int q = 0; q < i; ++q) a = a / beta;
    return a;
}

// weighted cost 1/2 |W r|^2 at the trial point clamp(theta + alpha d) of lane s
// (the kinematics passes, the 6 x 6 solve and the trial spreading each exist
// once in the kernel, called from every branch that needs them, which keeps
// the per-iteration body inside the instruction cache)
__device__ __noinline__ float trial_cost(const RobotParams* rob, const TargetDesc* tg, int row, const LmW S, int s,
                                        float alpha) {
    const TargetDesc T = tg[row];
    const RobotParams& R = rob[T.robot];
    Frame F = frame_identity();
#pragma unroll 1
    for (int j = 0; j < R.n; ++j)
        fk_step(R, j, clampf(fmaf(alpha, S.d(j, s), S.th(j, s)), R.lo[j], R.hi[j]), F);
    const Frame E = fk_flange(R, F);
    const V3 w = quat_log(quat_error(T, quat_from_frame(E)));
    const float e0 = S.W(0, s) * (T.p[0] - E.p.x), e1 = S.W(1, s) * (T.p[1] - E.p.y);
    const float e2 = S.W(2, s) * (T.p[2] - E.p.z), e3 = S.W(3, s) * w.x, e4 = S.W(4, s) * w.y;
    const float e5 = S.W(5, s) * w.z;
    return 0.5f * fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, fmaf(e4, e4, e5 * e5)))));
}

// theta <- clamp(theta + alpha d) for lane s (the trial point the cost was taken at)
__device__ __noinline__ void take_step(const RobotParams& R, const LmW S, int s, float alpha) {
#pragma unroll 1
    for (int j = 0; j < R.n; ++j) S.th(j, s) = clampf(fmaf(alpha, S.d(j, s), S.th(j, s)), R.lo[j], R.hi[j]);
}

// Trials i = i0 .. A of every lane in `mask`, spread over the warp; results in S.ok(i, lane).
__device__ __noinline__ unsigned long long warp_trials(const RobotParams* rob, const TargetDesc* tg, const LmW S,
                                                          unsigned mask, int lane, int i0, int A, float beta) {
    const int per = A + 1 - i0;
    if (!mask || per <= 0) return 0;
    if ((mask >> lane) & 1u) S.list(__popc(mask & ((1u << lane) - 1u))) = lane;
    __syncwarp();
    const int items = __popc(mask) * per;
    unsigned long long cnt = 0;
    for (int w = lane; w < items; w += 32) {
        const int s = S.list(w / per), i = i0 + w % per;
        S.ok(i, s) = trial_cost(rob, tg, S.t(s), S, s, ls_alpha(i, beta)) < S.cost0(s) ? 1 : 0;
        ++cnt;
    }
    __syncwarp();
    return cnt;
}

template <bool TRACE, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 16 / WARPS) k_lm(const LmArgs A) {
    extern __shared__ __align__(16) float smem_f[];
    const RobotParams* rob = stage_robots(smem_f, A.rs);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const LmW S{smem_f + robots_smem_bytes(A.rs.n) / sizeof(float) + warp * lm_warp_words(A.rs.n_max), A.rs.n_max};

    const hjcd_params& P = A.P;
    const float Rt = P.lm_trust_R;
    unsigned long long n_it = 0, n_fk = 0;

    bool has = false;
    int64_t c = 0;
    int32_t t = 0, s = 0, kk = 0, cap = 0;
    TargetDesc T{};

    for (;;) {
        // refill idle lanes from the global queue (one atomic per warp)
        const unsigned need = __ballot_sync(0xffffffffu, !has);
        if (need) {
            const int leader = __ffs(need) - 1;
            long long base = 0;
            if (lane == leader) base = (long long)atomicAdd(A.queue, (unsigned long long)__popc(need));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (!has) {
                c = base + __popc(need & ((1u << lane) - 1u));
                if (c < A.C && A.map.lookup(c, t, s)) {
                    T = A.tg[t];
                    kk = 0;
                    cap = A.n_iters >= 0 ? A.n_iters : T.lm_iters;
                    if (T.eps_pos > 0.0f) {
                        has = true;
                        const int nl = rob[T.robot].n;
#pragma unroll 1
                        for (int j = 0; j < nl; ++j) S.th(j, lane) = A.th[j * A.ld + c];
                    } else {  // invalid target: no iterations, infinite score
                        if (A.score) A.score[c] = __int_as_float(0x7f800000);
                        if (A.perr) A.perr[c] = 0.0f;
                        if (A.oerr) A.oerr[c] = 0.0f;
                        if (A.iters) A.iters[c] = cap;
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, has)) {
            // every lane asked for work: stop once the queue is drained, else ask again
            if (!__any_sync(0xffffffffu, c < A.C)) break;
            continue;
        }

        // ---- phase A: kinematics with frames, residual, LM step (owner) ----
        const RobotParams& R = rob[T.robot];
        const int n = R.n;
        bool act = false;
        if (has) {
            // joint origins and axes are parked in the lane's J slots
            Frame F = frame_identity();
#pragma unroll 1
            for (int j = 0; j < n; ++j) {
                fk_step(R, j, S.th(j, lane), F);
                S.jw(0, j, lane) = F.p.x;
                S.jw(1, j, lane) = F.p.y;
                S.jw(2, j, lane) = F.p.z;
                S.jw(3, j, lane) = F.c2.x;
                S.jw(4, j, lane) = F.c2.y;
                S.jw(5, j, lane) = F.c2.z;
            }
            const Frame E = fk_flange(R, F);
            ++n_fk;
            const V3 pt = v3(T.p[0], T.p[1], T.p[2]);
            const V3 om = quat_log(quat_error(T, quat_from_frame(E)));
            const V3 epv = pt - E.p;
            const float ep = sqrtf(dot(epv, epv)), eo = sqrtf(dot(om, om));
            if ((kk > 0 && ep < T.eps_pos && eo < T.eps_ori) || kk == cap) {
                // Alg. 4 break (checked after each update) or the iteration cap
#pragma unroll 1
                for (int j = 0; j < n; ++j) A.th[j * A.ld + c] = S.th(j, lane);
                if (A.score) {
                    const float a = ep / T.eps_pos, bb = eo / T.eps_ori;
                    A.score[c] = fmaf(a, a, bb * bb);
                }
                if (A.perr) A.perr[c] = ep;
                if (A.oerr) A.oerr[c] = eo;
                if (A.iters) A.iters[c] = kk;
                has = false;
            } else {
                act = true;
                // Jacobian columns z_i x (P_ee - P_i), z_i (in place), and the row norms
                float rn[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
                for (int i = 0; i < n; ++i) {
                    const V3 Pi = v3(S.jw(0, i, lane), S.jw(1, i, lane), S.jw(2, i, lane));
                    const V3 Zi = v3(S.jw(3, i, lane), S.jw(4, i, lane), S.jw(5, i, lane));
                    const V3 jp = cross(Zi, E.p - Pi);
                    S.jw(0, i, lane) = jp.x;
                    S.jw(1, i, lane) = jp.y;
                    S.jw(2, i, lane) = jp.z;
                    const float col[6] = {jp.x, jp.y, jp.z, Zi.x, Zi.y, Zi.z};
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
                        rn[r] = fmaf(col[r], col[r], rn[r]);
                        if (TRACE && kk == 0 && A.tr.J) A.tr.J[(r * n + i) * A.ld + c] = col[r];
                    }
                }
                const float e[6] = {epv.x, epv.y, epv.z, om.x, om.y, om.z};
                const float wo = T.eps_pos / T.eps_ori;
                float W[6], b[6], cost0 = 0.0f;
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    W[r] = (r < 3 ? 1.0f : wo) / fmaxf(sqrtf(rn[r]), 1e-6f);
                    b[r] = W[r] * e[r];
                    cost0 = fmaf(b[r], b[r], cost0);
                    S.W(r, lane) = W[r];
                    S.b(r, lane) = b[r];
                    if (TRACE && kk == 0 && A.tr.W) A.tr.W[r * A.ld + c] = W[r];
                }
                S.cost0(lane) = 0.5f * cost0;
                S.t(lane) = t;
                // the push-through LM step on the weighted Jacobian
                Y6 wv, bv;
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    wv.v[r] = W[r];
                    bv.v[r] = b[r];
                }
                const Y6 yy = normal_solve(S, lane, n, true, P.lm_lambda, wv, bv);
                float y[6];
#pragma unroll
                for (int r = 0; r < 6; ++r) y[r] = yy.v[r];
#pragma unroll 1
                for (int i = 0; i < n; ++i) {
                    float a = 0.0f, dd = 1e-9f;
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
                        const float v = S.jw(r, i, lane);
                        a = fmaf(v, y[r], a);
                        dd = fmaf(v, v, dd);
                    }
                    const float st = clampf(a / dd, -Rt, Rt);  // trust region
                    S.d(i, lane) = st;
                    if (TRACE && kk == 0 && A.tr.d_lm) A.tr.d_lm[i * A.ld + c] = st;
                }
            }
        }

        // ---- line search; the full step by its owner, the rest spread ----
        int branch = 3;
        float alpha_acc = 0.0f;
        if (act) {
            ++n_fk;
            if (trial_cost(rob, A.tg, t, S, lane, 1.0f) < S.cost0(lane)) {
                take_step(R, S, lane, 1.0f);
                branch = 0;
                alpha_acc = 1.0f;
            }
        }
        unsigned fail = __ballot_sync(0xffffffffu, act && branch != 0);
        n_fk += warp_trials(rob, A.tg, S, fail, lane, 1, P.lm_A, P.lm_beta);
        if (act && branch != 0) {
            for (int i = 1; i <= P.lm_A; ++i) {
                if (S.ok(i, lane)) {
                    alpha_acc = ls_alpha(i, P.lm_beta);
                    take_step(R, S, lane, alpha_acc);
                    branch = 0;
                    break;
                }
            }
        }

        // ---- dogleg (owner) ----
        if (act && branch != 0) {
            float b[6];
            Y6 bv, wv;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                b[r] = S.b(r, lane);
                bv.v[r] = b[r];
                wv.v[r] = 1.0f;
            }
            float Jg[6];
#pragma unroll
            for (int r = 0; r < 6; ++r) Jg[r] = 0.0f;
            float gg = 0.0f;
#pragma unroll 1
            for (int i = 0; i < n; ++i) {
                float col[6], g = 0.0f;
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    col[r] = S.jw(r, i, lane);
                    g = fmaf(col[r], b[r], g);
                }
                gg = fmaf(g, g, gg);
#pragma unroll
                for (int r = 0; r < 6; ++r) Jg[r] = fmaf(col[r], g, Jg[r]);
            }
            const Y6 yy2 = normal_solve(S, lane, n, false, P.lm_gn_reg, wv, bv);
            float y2[6];
#pragma unroll
            for (int r = 0; r < 6; ++r) y2[r] = yy2.v[r];
            float jgjg = 0.0f;
#pragma unroll
            for (int r = 0; r < 6; ++r) jgjg = fmaf(Jg[r], Jg[r], jgjg);
            const float ac = jgjg > 0.0f ? gg / jgjg : 0.0f;
            // g_i = (WJ)_i . W r and dgn_i = (WJ)_i . y2 are recomputed where needed
            float ngn2 = 0.0f;
#pragma unroll 1
            for (int i = 0; i < n; ++i) {
                float a = 0.0f;
#pragma unroll
                for (int r = 0; r < 6; ++r) a = fmaf(S.jw(r, i, lane), y2[r], a);
                ngn2 = fmaf(a, a, ngn2);
            }
            const float ngd2 = ac * ac * gg, R2 = Rt * Rt;
            float wgn = 1.0f, wgd = 0.0f;  // step = wgn * dgn + wgd * g
            if (ngn2 <= R2) {
                wgn = 1.0f;
                wgd = 0.0f;
            } else if (ngd2 >= R2) {
                wgn = 0.0f;
                wgd = ngd2 > 0.0f ? Rt * rsqrtf(ngd2) * ac : 0.0f;
            } else {
                float qa = 0.0f, qb = 0.0f;
#pragma unroll 1
                for (int i = 0; i < n; ++i) {
                    float dgn = 0.0f, g = 0.0f;
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
                        dgn = fmaf(S.jw(r, i, lane), y2[r], dgn);
                        g = fmaf(S.jw(r, i, lane), b[r], g);
                    }
                    const float di = fmaf(ac, g, -dgn);
                    qa = fmaf(di, di, qa);
                    qb = fmaf(2.0f * dgn, di, qb);
                }
                const float qc = ngn2 - R2;
                const float disc = fmaxf(fmaf(qb, qb, -4.0f * qa * qc), 0.0f);
                const float tau = (2.0f * qc) / (sqrtf(disc) - qb);  // smaller root, stable form
                wgn = 1.0f - tau;
                wgd = tau * ac;
            }
            // dogleg step as the trial direction, evaluated at alpha = 1
            int is = 0;
            float gbest = -1.0f, cn = 0.0f, gsel = 0.0f;
#pragma unroll 1
            for (int i = 0; i < n; ++i) {
                float dgn = 0.0f, g = 0.0f, q2 = 0.0f;
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    const float v = S.jw(r, i, lane);
                    dgn = fmaf(v, y2[r], dgn);
                    g = fmaf(v, b[r], g);
                    q2 = fmaf(v, v, q2);
                }
                S.d(i, lane) = fmaf(wgn, dgn, wgd * g);
                if (fabsf(g) > gbest) {  // single-coordinate choice
                    gbest = fabsf(g);
                    is = i;
                    gsel = g;
                    cn = q2;
                }
            }
            ++n_fk;
            if (trial_cost(rob, A.tg, t, S, lane, 1.0f) < S.cost0(lane)) {
                take_step(R, S, lane, 1.0f);
                branch = 1;
            } else {
                // single coordinate: the joint with the largest |g_i|, a 1-D Gauss-Newton step on
                // it clamped to R; its line-search trials are spread over the warp below
                const float sstep = cn > 0.0f ? clampf(gsel / cn, -Rt, Rt) : 0.0f;
#pragma unroll 1
                for (int j = 0; j < n; ++j) S.d(j, lane) = (j == is) ? sstep : 0.0f;
            }
        }
        fail = __ballot_sync(0xffffffffu, act && branch == 3);
        n_fk += warp_trials(rob, A.tg, S, fail, lane, 0, P.lm_A, P.lm_beta);
        if (act && branch == 3) {
            for (int i = 0; i <= P.lm_A; ++i) {
                if (S.ok(i, lane)) {
                    alpha_acc = ls_alpha(i, P.lm_beta);
                    take_step(R, S, lane, alpha_acc);
                    branch = 2;
                    break;
                }
            }
        }
        if (act && branch == 3) {
            // random perturbation when every update fails
            const uint32_t k = (uint32_t)(A.k0 + kk);
#pragma unroll 1
            for (int q = 0; 2 * q < n; ++q) {
                const float2 z = normal_pair(T, (uint32_t)s, kPhaseLm, k, q);
                const int j0 = 2 * q, j1 = 2 * q + 1;
                S.th(j0, lane) = clampf(fmaf(P.lm_sigma, z.x, S.th(j0, lane)), R.lo[j0], R.hi[j0]);
                if (j1 < n) S.th(j1, lane) = clampf(fmaf(P.lm_sigma, z.y, S.th(j1, lane)), R.lo[j1], R.hi[j1]);
            }
        }
        if (act) {
            if (TRACE && kk == 0) {
                if (A.tr.branch) A.tr.branch[c] = branch;
                if (A.tr.alpha) A.tr.alpha[c] = alpha_acc;
            }
            ++kk;
            ++n_it;
        }
        __syncwarp();
    }
    if (A.cnt) {
        n_it = warp_sum(n_it);
        n_fk = warp_sum(n_fk);
        if (lane == 0) {
            atomicAdd(&A.cnt->v[1], n_it);
            atomicAdd(&A.cnt->v[2], n_fk);
        }
    }
}

template <bool TRACE, int WARPS>
void launch_lm_t(const LmArgs& A, cudaStream_t st) {
    const size_t smem = robots_smem_bytes(A.rs.n) + sizeof(float) * (size_t)lm_warp_words(A.rs.n_max) * WARPS;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_lm<TRACE, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(robots_smem_bytes(kMaxLaunchRobots) +
                                   sizeof(float) * lm_warp_words(kMaxDof) * WARPS));
        attr = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lm<TRACE, WARPS>, WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t want = (A.C + 32 * WARPS - 1) / (32 * WARPS);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * per_sm));
    k_lm<TRACE, WARPS><<<g, WARPS * 32, smem, st>>>(A);
}

template <bool TRACE>
void launch_lm_w(const LmArgs& A, cudaStream_t st) {
    if (A.warps == 2) launch_lm_t<TRACE, 2>(A, st);
    else if (A.warps == 8) launch_lm_t<TRACE, 8>(A, st);
    else launch_lm_t<TRACE, kLmWarps>(A, st);
}

}  // namespace

void launch_lm(const LmArgs& A, bool trace, cudaStream_t st) {
    if (A.C <= 0) return;
    if (trace) launch_lm_w<true>(A, st);
    else launch_lm_w<false>(A, st);
}

}  // namespace hjcd

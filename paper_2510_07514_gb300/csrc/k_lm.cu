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
// Mapping.  Each lane of a warp owns one candidate (a slot of per-lane state)
// at a time and takes the next one from a global queue when its candidate
// finishes, so lanes never idle while work remains.  The full-step trial is
// evaluated by each owner.  The failure path is where candidates diverge (a
// third or more of the iterations fail the full step, and such a candidate
// needs up to 2(A+1) more trials), so the warps of a CTA iterate in lock step
// and the failing slots of all of them are compacted into one list that all
// the CTA's threads work through: each failing slot's dogleg and
// single-coordinate steps (whether or not a shorter step will succeed), then
// its remaining line-search trials and the dogleg trial as independent
// kinematics passes, and the trials of its single-coordinate line search, one
// per thread, then per slot the first of them, in the order of Alg. 4, that
// lowered its cost -- the step the sequential method accepts.  The
// single-coordinate trials run in closed form: turning one joint by x about
// its axis z moves the end effector by (1 - cos x) (v x z) + sin x v, with
// v = z x (p_ee - p_j) the joint's Jacobian column, and composes the
// orientation error with the half-angle quaternion [cos x/2, -sin x/2 z], so
// each costs a handful of operations instead of a kinematics pass, and they
// fill the threads the kinematics passes leave idle.  The perturbation's normal pairs of
// the slots that found no step are spread over the CTA as well.
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

constexpr int kLmWarps = 8;  // default warps per CTA; 2 and 4 also built
constexpr int kMaxLsDepth = 31;  // A (validated by the host)

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

// words of per-warp shared state for an n-joint chain and line-search depth A
// W[6], b[6], cost0, t, s, kk, sc_j, sc_step, e[3], q_err[4], sc_z[3], sc_v[3], branch, alpha;
// then one byte per lane and trial: the A + 1 kinematics trials, the A + 1 single-coordinate trials
constexpr int kLmScalars = 33;
__host__ __device__ constexpr int lm_warp_words(int n, int A) { return (8 * n + kLmScalars) * 32 + (A + 1) * 16; }

// trial directions: the LM (or line-search) direction d, the dogleg step d2,
// the single coordinate (joint sc_j by sc_step)
enum TrialKind { kDirLm = 0, kDirDogleg = 1 };

// Per-warp state, field[...][lane] (each lane's own accesses conflict-free);
// n is the layout's chain length (the launch's largest).  A joint's angle and
// trial direction, and rows 2q and 2q + 1 of a Jacobian column, are pairs
// [...][lane][2] that move as one 64-bit access.  The dogleg step d2
// shares its words with row 0 of the weighted Jacobian: it is written column
// by column after that column's last read, and the Jacobian is not read again
// before the next iteration rebuilds it.
struct LmW {
    float* f;
    int n;
    // joint j's angle and LM (or line-search) direction as one pair (one 64-bit access)
    __device__ __forceinline__ float2& thd(int j, int l) const { return reinterpret_cast<float2*>(f)[j * 32 + l]; }
    __device__ __forceinline__ float& th(int j, int l) const { return thd(j, l).x; }
    __device__ __forceinline__ float& d(int j, int l) const { return thd(j, l).y; }
    // rows 2q and 2q + 1 of column i of the weighted Jacobian as one pair (one 64-bit access)
    __device__ __forceinline__ float2& jw2(int q, int i, int l) const {
        return reinterpret_cast<float2*>(f + 2 * n * 32)[(q * n + i) * 32 + l];
    }
    __device__ __forceinline__ float& jw(int r, int i, int l) const {
        return reinterpret_cast<float*>(&jw2(r >> 1, i, l))[r & 1];
    }
    // column i's six rows
    __device__ __forceinline__ void col6(int i, int l, float (&c)[6]) const {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float2 v = jw2(q, i, l);
            c[2 * q] = v.x;
            c[2 * q + 1] = v.y;
        }
    }
    __device__ __forceinline__ void set_col6(int i, int l, const float (&c)[6]) const {
#pragma unroll
        for (int q = 0; q < 3; ++q) jw2(q, i, l) = make_float2(c[2 * q], c[2 * q + 1]);
    }
    __device__ __forceinline__ float& d2(int j, int l) const { return jw(0, j, l); }
    __device__ __forceinline__ float& W(int r, int l) const { return f[(8 * n + r) * 32 + l]; }
    __device__ __forceinline__ float& b(int r, int l) const { return f[(8 * n + 6 + r) * 32 + l]; }
    __device__ __forceinline__ float& cost0(int l) const { return f[(8 * n + 12) * 32 + l]; }
    __device__ __forceinline__ int& t(int l) const { return reinterpret_cast<int*>(f)[(8 * n + 13) * 32 + l]; }
    __device__ __forceinline__ int& s(int l) const { return reinterpret_cast<int*>(f)[(8 * n + 14) * 32 + l]; }
    __device__ __forceinline__ int& kk(int l) const { return reinterpret_cast<int*>(f)[(8 * n + 15) * 32 + l]; }
    __device__ __forceinline__ int& sc_j(int l) const { return reinterpret_cast<int*>(f)[(8 * n + 16) * 32 + l]; }
    __device__ __forceinline__ float& sc_step(int l) const { return f[(8 * n + 17) * 32 + l]; }
    // position error and error quaternion at the iteration's configuration; the single
    // coordinate's axis and position Jacobian column (unweighted)
    __device__ __forceinline__ float& e(int r, int l) const { return f[(8 * n + 18 + r) * 32 + l]; }
    __device__ __forceinline__ float& qe(int r, int l) const { return f[(8 * n + 21 + r) * 32 + l]; }
    __device__ __forceinline__ float& sc_z(int r, int l) const { return f[(8 * n + 25 + r) * 32 + l]; }
    __device__ __forceinline__ float& sc_v(int r, int l) const { return f[(8 * n + 28 + r) * 32 + l]; }
    // the failure path's outcome for the owner: Alg. 4 branch and accepted alpha
    __device__ __forceinline__ int& br(int l) const { return reinterpret_cast<int*>(f)[(8 * n + 31) * 32 + l]; }
    __device__ __forceinline__ float& al(int l) const { return f[(8 * n + 32) * 32 + l]; }
    // trial i lowered the cost (i < A + 1: kinematics trial i; else single-coordinate trial i - A - 1)
    __device__ __forceinline__ uint8_t& ok(int i, int l) const {
        return reinterpret_cast<uint8_t*>(f + (8 * n + kLmScalars) * 32)[i * 32 + l];
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
// for lane l's Jacobian columns, each first weighted by the rows' W (and
// stored back, so the smem Jacobian becomes W J) and then scaled to unit
// length (S = D^-1/2 of the push-through LM step).
__device__ __noinline__ Y6 normal_solve(const LmW S, int l, int n, float reg, Y6 w, Y6 b) {
    float M[21], inv[6];
#pragma unroll
    for (int q = 0; q < 21; ++q) M[q] = 0.0f;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        float col[6], dd = 1e-9f;
        S.col6(i, l, col);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            col[r] *= w.v[r];
            dd = fmaf(col[r], col[r], dd);
        }
        S.set_col6(i, l, col);
        const float rs = rsqrtf(dd);
#pragma unroll
        for (int r = 0; r < 6; ++r) col[r] *= rs;
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

// alpha_i = 1 / beta^i by repeated division, i = 0 .. A, into a table of the CTA (one set of bits
// for every thread)
__device__ __forceinline__ void ls_alphas(float* tab, int A, float beta) {
    float a = 1.0f;
    for (int i = 0; i <= A; ++i) {
        tab[i] = a;
        a = a / beta;
    }
}

// CTA-wide lists of the failure path (after the warps' state): per warp its mask of failing
// lanes, the failing slots compacted, the slots left to the perturbation and their count.
template <int WARPS>
struct LmCta {
    unsigned* wm;
    int* fl;
    int* pl;
    int* np;
};
template <int WARPS>
__host__ __device__ constexpr int lm_cta_words() { return WARPS + 2 * WARPS * 32 + 1; }
template <int WARPS>
__device__ __forceinline__ LmCta<WARPS> lm_cta(float* f) {
    int* b = reinterpret_cast<int*>(f);
    return LmCta<WARPS>{reinterpret_cast<unsigned*>(b), b + WARPS, b + WARPS + WARPS * 32, b + WARPS + 2 * WARPS * 32};
}

// weighted cost 1/2 |W r|^2 at the trial point clamp(theta + alpha dir) of lane s
// (the kinematics passes, the 6 x 6 solve and the trial spreading each exist
// once in the kernel, called from every branch that needs them, which keeps
// the per-iteration body inside the instruction cache)
template <bool RED>
__device__ __noinline__ float trial_cost(const RobotParams* rob, const TargetDesc* tg, int row, const LmW S, int s,
                                        float alpha, int kind) {
    const TargetDesc T = tg[row];
    const RobotParams& R = rob[T.robot];
    Frame F = frame_identity();
#pragma unroll 1
    for (int j = 0; j < R.n; ++j) {
        const float2 td = S.thd(j, s);
        const float dir = kind == kDirDogleg ? S.d2(j, s) : td.y;
        fk_step<RED>(R, j, clampf(fmaf(alpha, dir, td.x), R.lim[j].x, R.lim[j].y), F);
    }
    const Frame E = fk_flange(R, F);
    const V3 w = quat_log(quat_error(T, quat_from_frame(E)));
    const float e0 = S.W(0, s) * (T.p[0] - E.p.x), e1 = S.W(1, s) * (T.p[1] - E.p.y);
    const float e2 = S.W(2, s) * (T.p[2] - E.p.z), e3 = S.W(3, s) * w.x, e4 = S.W(4, s) * w.y;
    const float e5 = S.W(5, s) * w.z;
    return 0.5f * fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, fmaf(e4, e4, e5 * e5)))));
}

// theta <- clamp(theta + alpha dir) for lane s (the trial point the cost was taken at)
__device__ __noinline__ void take_step(const RobotParams& R, const LmW S, int s, float alpha, int kind) {
#pragma unroll 1
    for (int j = 0; j < R.n; ++j) {
        const float2 td = S.thd(j, s);
        const float dir = kind == kDirDogleg ? S.d2(j, s) : td.y;
        S.th(j, s) = clampf(fmaf(alpha, dir, td.x), R.lim[j].x, R.lim[j].y);
    }
}

// The kinematics-pass trials that follow a failed full step, in the order Alg. 4
// takes them: item i < A is the line-search trial alpha = 1/beta^(i+1) along d,
// item A the dogleg step.
__device__ __forceinline__ void trial_item(int i, int A, const float* alphas, int* kind, float* alpha) {
    *kind = i < A ? kDirLm : kDirDogleg;
    *alpha = i < A ? alphas[i + 1] : 1.0f;
}

// Weighted cost of lane l's configuration with its single coordinate turned by x (the end
// effector rotated by x about the joint's axis; see the mapping notes above).
__device__ __noinline__ float coord_cost(const LmW S, int l, float x) {
    float sh, ch;
    sincos_red(0.5f * x, &sh, &ch);
    const V3 z = v3(S.sc_z(0, l), S.sc_z(1, l), S.sc_z(2, l));
    const V3 v = v3(S.sc_v(0, l), S.sc_v(1, l), S.sc_v(2, l));
    const V3 up = cross(v, z);  // component of p_ee - p_j normal to the axis
    const float a = 2.0f * sh * sh, b = 2.0f * sh * ch;  // 1 - cos x, sin x
    const V3 e = fma3(a, up, fma3(-b, v, v3(S.e(0, l), S.e(1, l), S.e(2, l))));
    const Q4 q{S.qe(0, l), v3(S.qe(1, l), S.qe(2, l), S.qe(3, l))};
    Q4 q2{fmaf(q.w, ch, sh * dot(q.v, z)), fma3(ch, q.v, (-sh) * fma3(q.w, z, cross(q.v, z)))};
    if (q2.w < 0.0f) {
        q2.w = -q2.w;
        q2.v = (-1.0f) * q2.v;
    }
    const V3 w = quat_log(q2);
    const float e0 = S.W(0, l) * e.x, e1 = S.W(1, l) * e.y, e2 = S.W(2, l) * e.z;
    const float e3 = S.W(3, l) * w.x, e4 = S.W(4, l) * w.y, e5 = S.W(5, l) * w.z;
    return 0.5f * fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, fmaf(e4, e4, e5 * e5)))));
}

// The dogleg step of Eq. dogleg and the single-coordinate step of Eq. single-coord for lane l,
// from its weighted Jacobian W J (columns in shared memory) and W r: into S.d2, S.sc_j,
// S.sc_step.  With M0 = (WJ)(WJ)^T the Gauss-Newton step is (WJ)^T y2, y2 = (M0 + reg I)^-1 W r,
// and the Cauchy point's quantities reduce to 6 x 6 forms: J g = M0 W r, |g|^2 = (W r).M0 W r.
// |d_gn|^2 is summed over the step's components instead of as y2.M0 y2: when M0 is nearly
// singular y2 is large and that form cancels catastrophically (its binary32 value could fall
// inside the trust region while the step is far outside).  The first pass over the columns
// gives |d_gn|^2 and the coefficients of the segment's crossing of the boundary, the second
// forms the step.
__device__ __noinline__ void dogleg_prepare(const LmW S, int l, int n, float Rt, float gn_reg) {
    float M0[21], M[21], inv[6], b[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) b[r] = S.b(r, l);
#pragma unroll
    for (int q = 0; q < 21; ++q) M0[q] = 0.0f;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        float col[6];
        S.col6(i, l, col);
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int q = 0; q <= r; ++q) M0[tri(r, q)] = fmaf(col[r], col[q], M0[tri(r, q)]);
    }
#pragma unroll
    for (int q = 0; q < 21; ++q) M[q] = M0[q];
#pragma unroll
    for (int r = 0; r < 6; ++r) M[tri(r, r)] += gn_reg;
    chol6(M, inv);
    float y2[6];
    chol6_solve(M, inv, b, y2);
    // J g = M0 W r
    float Jg[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        float a = 0.0f;
#pragma unroll
        for (int q = 0; q < 6; ++q) a = fmaf(r >= q ? M0[tri(r, q)] : M0[tri(q, r)], b[q], a);
        Jg[r] = a;
    }
    float gg = 0.0f, jgjg = 0.0f;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        gg = fmaf(b[r], Jg[r], gg);
        jgjg = fmaf(Jg[r], Jg[r], jgjg);
    }
    const float ac = jgjg > 0.0f ? __fdividef(gg, jgjg) : 0.0f;
    const float ngd2 = ac * ac * gg, R2 = Rt * Rt;
    // |d_gn|^2 and, for the segment from d_gn to the Cauchy point, |d_cp - d_gn|^2 and 2 d_gn.(d_cp - d_gn)
    float ngn2 = 0.0f, qa = 0.0f, qb = 0.0f;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        float dgn = 0.0f, g = 0.0f, col[6];
        S.col6(i, l, col);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            dgn = fmaf(col[r], y2[r], dgn);
            g = fmaf(col[r], b[r], g);
        }
        const float di = fmaf(ac, g, -dgn);
        ngn2 = fmaf(dgn, dgn, ngn2);
        qa = fmaf(di, di, qa);
        qb = fmaf(2.0f * dgn, di, qb);
    }
    float wgn = 1.0f, wgd = 0.0f;  // step = wgn * dgn + wgd * g
    if (ngn2 <= R2) {
        wgn = 1.0f;
        wgd = 0.0f;
    } else if (ngd2 >= R2) {
        wgn = 0.0f;
        wgd = ngd2 > 0.0f ? Rt * rsqrtf(ngd2) * ac : 0.0f;
    } else {
        // the point of the segment from the Gauss-Newton step to the Cauchy point on the boundary
        const float qc = ngn2 - R2;
        const float disc = fmaxf(fmaf(qb, qb, -4.0f * qa * qc), 0.0f);
        const float tau = (2.0f * qc) / (sqrtf(disc) - qb);  // smaller root, stable form (qb < 0 here)
        wgn = 1.0f - tau;
        wgd = tau * ac;
    }
    // the step, and the single coordinate: the joint with the largest |g_i| (the first of
    // equals), a 1-D Gauss-Newton step on it clamped to R
    int is = 0;
    float gbest = -1.0f, cn = 0.0f, gsel = 0.0f, csel[6];
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        float dgn = 0.0f, g = 0.0f, q2 = 0.0f, col[6];
        S.col6(i, l, col);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            dgn = fmaf(col[r], y2[r], dgn);
            g = fmaf(col[r], b[r], g);
            q2 = fmaf(col[r], col[r], q2);
        }
        S.d2(i, l) = fmaf(wgn, dgn, wgd * g);
        if (fabsf(g) > gbest) {
            gbest = fabsf(g);
            is = i;
            gsel = g;
            cn = q2;
#pragma unroll
            for (int r = 0; r < 6; ++r) csel[r] = col[r];
        }
    }
    S.sc_j(l) = is;
    S.sc_step(l) = cn > 0.0f ? clampf(__fdividef(gsel, cn), -Rt, Rt) : 0.0f;
    // the chosen joint's position column and axis without the row weights
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        S.sc_v(r, l) = __fdividef(csel[r], S.W(r, l));
        S.sc_z(r, l) = __fdividef(csel[3 + r], S.W(3 + r, l));
    }
}

// RED = false: the launch's joint vectors lie within the limits of plain robots (no offsets and
// no range reduction in the kinematics steps; the same bits)
template <bool TRACE, int WARPS, bool RED>
__global__ void __launch_bounds__(WARPS * 32, 16 / WARPS) k_lm(const LmArgs A) {
    extern __shared__ __align__(16) float smem_f[];
    __shared__ float alphas[kMaxLsDepth + 1];
    if (threadIdx.x == 0) ls_alphas(alphas, A.P.lm_A, A.P.lm_beta);  // visible after the staging barrier
    const RobotParams* rob = stage_robots(smem_f, A.rs);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* const warps_f = smem_f + robots_smem_bytes(A.rs.n) / sizeof(float);
    const int words = lm_warp_words(A.rs.n_max, A.P.lm_A);
    const LmW S{warps_f + warp * words, A.rs.n_max};
    // the state of slot sl = warp * 32 + lane, whichever thread works on it
    auto slot_state = [&](int sl) { return LmW{warps_f + (sl >> 5) * words, A.rs.n_max}; };
    const LmCta<WARPS> CL = lm_cta<WARPS>(warps_f + WARPS * words);

    const hjcd_params& P = A.P;
    const float Rt = P.lm_trust_R;
    unsigned long long n_it = 0, n_fk = 0, n_sc = 0;

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
                        load_joints<8>(A.th, A.ld, c, rob[T.robot].n, [&](int j, float v) { S.th(j, lane) = v; });
                    } else {  // invalid target: no iterations, infinite score
                        if (A.score) A.score[c] = __int_as_float(0x7f800000);
                        if (A.perr) A.perr[c] = 0.0f;
                        if (A.oerr) A.oerr[c] = 0.0f;
                        if (A.iters) A.iters[c] = cap;
                    }
                }
            }
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
                fk_step<RED>(R, j, S.th(j, lane), F);
                S.jw2(0, j, lane) = make_float2(F.p.x, F.p.y);
                S.jw2(1, j, lane) = make_float2(F.p.z, F.c2.x);
                S.jw2(2, j, lane) = make_float2(F.c2.y, F.c2.z);
            }
            const Frame E = fk_flange(R, F);
            ++n_fk;
            const V3 pt = v3(T.p[0], T.p[1], T.p[2]);
            const Q4 qerr = quat_error(T, quat_from_frame(E));
            const V3 om = quat_log(qerr);
            const V3 epv = pt - E.p;
            const float ep = sqrt_approx(dot(epv, epv)), eo = sqrt_approx(dot(om, om));
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
                    float fr[6];
                    S.col6(i, lane, fr);
                    const V3 Pi = v3(fr[0], fr[1], fr[2]);
                    const V3 Zi = v3(fr[3], fr[4], fr[5]);
                    const V3 jp = cross(Zi, E.p - Pi);
                    S.jw2(0, i, lane) = make_float2(jp.x, jp.y);
                    S.jw2(1, i, lane) = make_float2(jp.z, Zi.x);
                    const float col[6] = {jp.x, jp.y, jp.z, Zi.x, Zi.y, Zi.z};
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
                        rn[r] = fmaf(col[r], col[r], rn[r]);
                        if (TRACE && kk == 0 && A.tr.J) A.tr.J[(r * n + i) * A.ld + c] = col[r];
                    }
                }
                const float e[6] = {epv.x, epv.y, epv.z, om.x, om.y, om.z};
                const float wo = __fdividef(T.eps_pos, T.eps_ori);
                float W[6], b[6], cost0 = 0.0f;
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    W[r] = (r < 3 ? 1.0f : wo) * rsqrtf(fmaxf(rn[r], 1e-12f));  // c / max(|row|, 1e-6)
                    b[r] = W[r] * e[r];
                    cost0 = fmaf(b[r], b[r], cost0);
                    S.W(r, lane) = W[r];
                    S.b(r, lane) = b[r];
                    if (TRACE && kk == 0 && A.tr.W) A.tr.W[r * A.ld + c] = W[r];
                }
                S.cost0(lane) = 0.5f * cost0;
                S.t(lane) = t;
                S.e(0, lane) = epv.x;
                S.e(1, lane) = epv.y;
                S.e(2, lane) = epv.z;
                S.qe(0, lane) = qerr.w;
                S.qe(1, lane) = qerr.v.x;
                S.qe(2, lane) = qerr.v.y;
                S.qe(3, lane) = qerr.v.z;
                // the push-through LM step on the weighted Jacobian
                Y6 wv, bv;
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    wv.v[r] = W[r];
                    bv.v[r] = b[r];
                }
                const Y6 yy = normal_solve(S, lane, n, P.lm_lambda, wv, bv);
                float y[6];
#pragma unroll
                for (int r = 0; r < 6; ++r) y[r] = yy.v[r];
#pragma unroll 1
                for (int i = 0; i < n; ++i) {
                    float a = 0.0f, dd = 1e-9f, cl[6];
                    S.col6(i, lane, cl);
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
                        a = fmaf(cl[r], y[r], a);
                        dd = fmaf(cl[r], cl[r], dd);
                    }
                    const float st = clampf(__fdividef(a, dd), -Rt, Rt);  // trust region
                    S.d(i, lane) = st;
                    if (TRACE && kk == 0 && A.tr.d_lm) A.tr.d_lm[i * A.ld + c] = st;
                }
            }
        }

        // ---- the full step by its owner ----
        int branch = 3;
        float alpha_acc = 0.0f;
        if (act) {
            ++n_fk;
            if (trial_cost<RED>(rob, A.tg, t, S, lane, 1.0f, kDirLm) < S.cost0(lane)) {
                take_step(R, S, lane, 1.0f, kDirLm);
                branch = 0;
                alpha_acc = 1.0f;
            }
        }
        const bool failed = act && branch != 0;
        if (failed) {
            S.s(lane) = s;
            S.kk(lane) = kk;
        }

        // ---- the failure path over the CTA: the failing slots of all warps, compacted ----
        // (the same barrier ends the loop once no lane holds a candidate and the queue is drained:
        // a lane whose candidate just finished still holds an index below C and asks again)
        const unsigned fail = __ballot_sync(0xffffffffu, failed);
        if (lane == 0) CL.wm[warp] = fail;
        if (!__syncthreads_or(has || c < A.C)) break;
        int nf = 0, before = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const int k = __popc(CL.wm[w]);
            before += w < warp ? k : 0;
            nf += k;
        }
        if (failed) CL.fl[before + __popc(fail & ((1u << lane) - 1u))] = threadIdx.x;
        if (threadIdx.x == 0) CL.np[0] = 0;
        __syncthreads();
        if (nf > 0) {
            // dogleg and single-coordinate steps of each failing slot
            for (int i = threadIdx.x; i < nf; i += blockDim.x) {
                const int sl = CL.fl[i], l = sl & 31;
                const LmW Sx = slot_state(sl);
                dogleg_prepare(Sx, l, rob[A.tg[Sx.t(l)].robot].n, Rt, P.lm_gn_reg);
            }
            __syncthreads();
            // the remaining line-search trials and the dogleg trial, one kinematics pass each, then
            // the single-coordinate line search's trials in closed form (each slot's A + 1 of
            // them, whether or not the sequential method gets that far: they take the threads the
            // kinematics passes leave idle)
            const int per = P.lm_A + 1;
            const int nk = nf * per;
            for (int w = threadIdx.x; w < 2 * nk; w += blockDim.x) {
                const int wi = w < nk ? w : w - nk;
                const int sl = CL.fl[wi / per], l = sl & 31, i = wi % per;
                const LmW Sx = slot_state(sl);
                if (w < nk) {
                    int kind;
                    float alpha;
                    trial_item(i, P.lm_A, alphas, &kind, &alpha);
                    Sx.ok(i, l) = trial_cost<RED>(rob, A.tg, Sx.t(l), Sx, l, alpha, kind) < Sx.cost0(l) ? 1 : 0;
                } else {
                    const RobotParams& Rx = rob[A.tg[Sx.t(l)].robot];
                    const int j = Sx.sc_j(l);
                    const float th0 = Sx.th(j, l);
                    const float thj = clampf(fmaf(alphas[i], Sx.sc_step(l), th0), Rx.lim[j].x, Rx.lim[j].y);
                    Sx.ok(per + i, l) = coord_cost(Sx, l, thj - th0) < Sx.cost0(l) ? 1 : 0;
                }
            }
            __syncthreads();
            // each slot's first successful trial in the order of Alg. 4, else the first successful
            // trial of its single-coordinate line search, else the perturbation
            for (int i = threadIdx.x; i < nf; i += blockDim.x) {
                const int sl = CL.fl[i], l = sl & 31;
                const LmW Sx = slot_state(sl);
                const RobotParams& Rx = rob[A.tg[Sx.t(l)].robot];
                int pick = per;
                for (int q = 0; q < per; ++q)
                    if (Sx.ok(q, l)) {
                        pick = q;
                        break;
                    }
                n_fk += pick < per ? pick + 1 : per;  // the passes the sequential method evaluates
                int br = 3;
                float al = 0.0f;
                if (pick < per) {
                    int kind;
                    trial_item(pick, P.lm_A, alphas, &kind, &al);
                    take_step(Rx, Sx, l, al, kind);
                    br = kind == kDirLm ? 0 : 1;
                    if (kind == kDirDogleg) al = 0.0f;  // no line-search alpha (as traced)
                } else {
                    int qc = per;
                    for (int q = 0; q < per; ++q)
                        if (Sx.ok(per + q, l)) {
                            qc = q;
                            break;
                        }
                    n_sc += qc < per ? qc + 1 : per;  // the trials the sequential method evaluates
                    if (qc < per) {
                        const int j = Sx.sc_j(l);
                        const float th0 = Sx.th(j, l);
                        Sx.th(j, l) = clampf(fmaf(alphas[qc], Sx.sc_step(l), th0), Rx.lim[j].x, Rx.lim[j].y);
                        br = 2;
                        al = alphas[qc];
                    } else {
                        CL.pl[atomicAdd(CL.np, 1)] = sl;
                    }
                }
                Sx.br(l) = br;
                Sx.al(l) = al;
            }
            __syncthreads();
            // the perturbation of Alg. 4: normal pairs of every slot that found no step
            const int np = CL.np[0];
            if (np > 0) {
                const int pp = (A.rs.n_max + 1) / 2;
                for (int w = threadIdx.x; w < np * pp; w += blockDim.x) {
                    const int sl = CL.pl[w / pp], l = sl & 31, q = w % pp;
                    const LmW Sx = slot_state(sl);
                    const TargetDesc& Tx = A.tg[Sx.t(l)];
                    const RobotParams& Rx = rob[Tx.robot];
                    const int j0 = 2 * q, j1 = 2 * q + 1;
                    if (j0 >= Rx.n) continue;
                    const float2 z = normal_pair(Tx, (uint32_t)Sx.s(l), kPhaseLm, (uint32_t)A.k0 + (uint32_t)Sx.kk(l), q);
                    Sx.th(j0, l) = clampf(fmaf(P.lm_sigma, z.x, Sx.th(j0, l)), Rx.lim[j0].x, Rx.lim[j0].y);
                    if (j1 < Rx.n) Sx.th(j1, l) = clampf(fmaf(P.lm_sigma, z.y, Sx.th(j1, l)), Rx.lim[j1].x, Rx.lim[j1].y);
                }
                __syncthreads();
            }
            if (failed) {
                branch = S.br(lane);
                alpha_acc = S.al(lane);
            }
        }
        if (act) {
            if (TRACE && kk == 0) {
                if (A.tr.branch) A.tr.branch[c] = branch;
                if (A.tr.alpha) A.tr.alpha[c] = alpha_acc;
                if (failed) {  // the fallback steps exist for the slots whose full step failed
                    if (A.tr.d_dog)
#pragma unroll 1
                        for (int j = 0; j < n; ++j) A.tr.d_dog[j * A.ld + c] = S.d2(j, lane);
                    if (A.tr.sc_joint) A.tr.sc_joint[c] = S.sc_j(lane);
                    if (A.tr.sc_step) A.tr.sc_step[c] = S.sc_step(lane);
                }
            }
            ++kk;
            ++n_it;
        }
        __syncwarp();
    }
    if (A.cnt) {
        n_it = warp_sum(n_it);
        n_fk = warp_sum(n_fk);
        n_sc = warp_sum(n_sc);
        if (lane == 0) {
            atomicAdd(&A.cnt->v[1], n_it);
            atomicAdd(&A.cnt->v[2], n_fk);
            atomicAdd(&A.cnt->v[7], n_sc);
        }
    }
}

template <bool TRACE, int WARPS, bool RED>
void launch_lm_t(const LmArgs& A, cudaStream_t st) {
    const size_t smem = robots_smem_bytes(A.rs.n) +
                        sizeof(float) * ((size_t)lm_warp_words(A.rs.n_max, A.P.lm_A) * WARPS + lm_cta_words<WARPS>());
    static SmemLimit lim;
    allow_dyn_smem(k_lm<TRACE, WARPS, RED>, lim,
                   robots_smem_bytes(kMaxLaunchRobots) +
                       sizeof(float) * ((size_t)lm_warp_words(kMaxDof, kMaxLsDepth) * WARPS + lm_cta_words<WARPS>()));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lm<TRACE, WARPS, RED>, WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t want = (A.C + 32 * WARPS - 1) / (32 * WARPS);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * per_sm));
    k_lm<TRACE, WARPS, RED><<<g, WARPS * 32, smem, st>>>(A);
}

template <bool TRACE, bool RED>
void launch_lm_w(const LmArgs& A, cudaStream_t st) {
    // fewer warps per CTA when the requested count's state does not fit in shared memory
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, current_device());
    const size_t per_warp = sizeof(float) * (size_t)lm_warp_words(A.rs.n_max, A.P.lm_A);
    int warps = A.warps == 2 || A.warps == 4 || A.warps == 8 ? A.warps : kLmWarps;
    // a batch too small to give every SM a CTA of two warps (a single target, say): two-warp CTAs,
    // spread over more SMs with shorter lock-step stages (latency, not throughput, is at stake)
    if (A.C <= (int64_t)sm_count() * 64) warps = 2;
    // (the CTA lists: 65 words per warp and one; 256 bytes kept for the kernel's static arrays)
    while (warps > 2 && robots_smem_bytes(A.rs.n) + (per_warp + sizeof(float) * 65) * warps + 4 + 256 > (size_t)optin)
        warps /= 2;
    if (warps == 2) launch_lm_t<TRACE, 2, RED>(A, st);
    else if (warps == 4) launch_lm_t<TRACE, 4, RED>(A, st);
    else launch_lm_t<TRACE, 8, RED>(A, st);
}

}  // namespace

void launch_lm(const LmArgs& A, bool trace, cudaStream_t st) {
    if (A.C <= 0) return;
    if (trace) launch_lm_w<true, true>(A, st);
    else if (A.in_limits && A.rs.plain) launch_lm_w<false, false>(A, st);
    else launch_lm_w<false, true>(A, st);
}

}  // namespace hjcd

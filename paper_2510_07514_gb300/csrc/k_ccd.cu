// k_ccd.cu -- seed sampling (Alg. 3) and PO-CCD iterations (Sec. IV,
// Alg. 3), one candidate per thread.
//
// Per iteration one forward-kinematics pass gives every joint's origin and
// axis.  The 2n trial updates are evaluated in O(1) each: rotating joint j by
// d moves the end effector about the axis (Rodrigues) and composes the error
// quaternion with the joint rotation, so both parts of each trial's task
// residual follow from the projected vectors of Eq. vec_proj and one half-angle
// sine/cosine.  The proposed theta_hat changes at most two joints; its
// residual is the composition of the two joint rotations applied to the
// current end-effector pose (the more distal joint first), so acceptance
// needs no second kinematics pass.
//
// Each thread keeps its joint vector and the joint origins/axes of the last
// kinematics pass in a column of shared memory ([quantity][thread], so the
// accesses of a warp hit 32 different banks); joint loops are not unrolled,
// which keeps the kernel small enough for the instruction cache at any n.
// The robot tables of the launch sit in shared memory in front of the
// columns; each candidate uses its target's robot.
#include <algorithm>

#include "hjcd_internal.cuh"

namespace hjcd {

namespace {

// CTA size of the seed-sampling kernel, and of the PO-CCD kernel when the launch names none of
// 64, 128, 256 (a context starts at 64 candidates per CTA: hjcd_set_launch_config)
constexpr int kCcdThreads = 128;

// shared-memory column of a thread in a CTA of TH threads, laid out [quantity][thread] (a warp's
// accesses hit 32 different banks): per joint j the pairs (px, py), (pz, theta_j), (zx, zy),
// (zz, -) of joint j's frame after its kinematics step, 8 n words in all; each pair moves as one
// 64-bit access
template <int TH>
struct ColT {
    float2* base;  // this thread's first pair
    __device__ __forceinline__ float2& a(int j) const { return base[4 * j * TH]; }
    __device__ __forceinline__ float2& b(int j) const { return base[(4 * j + 1) * TH]; }
    __device__ __forceinline__ float2& c(int j) const { return base[(4 * j + 2) * TH]; }
    __device__ __forceinline__ float& zz(int j) const { return base[(4 * j + 3) * TH].x; }
    __device__ __forceinline__ float& th(int j) const { return b(j).y; }
    // joint j's origin and axis
    __device__ __forceinline__ void frame(int j, V3& p, V3& z) const {
        const float2 pa = a(j), pb = b(j), za = c(j);
        p = v3(pa.x, pa.y, pb.x);
        z = v3(za.x, za.y, zz(j));
    }
    __device__ __forceinline__ void set_frame(int j, const Frame& F, float theta) const {
        a(j) = make_float2(F.p.x, F.p.y);
        b(j) = make_float2(F.p.z, theta);
        c(j) = make_float2(F.c2.x, F.c2.y);
        zz(j) = F.c2.z;
    }
};
constexpr int kColWordsPerJoint = 8;

// the joint vector alone, theta[n] (the seed-sampling kernel)
template <int TH>
struct ThetaCol {
    float* base;
    __device__ __forceinline__ float& th(int j) const { return base[j * TH]; }
};

template <class Col>
__device__ __forceinline__ void sample_seed(const RobotParams& R, const TargetDesc& T, uint32_t s, const Col& col) {
#pragma unroll 1
    for (int b = 0; 4 * b < R.n; ++b) {
        const uint4 w = rnd_block(T, s, kPhaseSeed, 0, (uint32_t)b);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = 4 * b + q;
            if (j < R.n) col.th(j) = fmaf(u01(word(w, q)), R.lim[j].y - R.lim[j].x, R.lim[j].x);
        }
    }
}

// Both trials of joint j (origin pj, unit axis z, angle thj in [lo, hi]) against the end
// effector at Ep and the error quaternion qerr (angle phi): the position step d of Eq.
// theta_proj and the orientation step dq of Eq. ori_update, each clamped to the limits, with the
// task residual each leaves (position error squared, orientation angle) and its score.  Rotating
// joint j by x moves the end effector to pj + uz z + cos x up + sin x (z x up) and turns the error
// quaternion into qerr [cos(x/2), -sin(x/2) z].
struct CcdTrials {
    float d, rp2, op, sp;   // position trial
    float dq, pq2, rq, so;  // orientation trial
};

// The two trials of a joint share their arithmetic once the steps are known, so from there on
// they run as pairs (.x the position trial, .y the orientation trial) on the packed FP32
// instructions of sm_100+ (two IEEE operations per instruction, each half rounded on its own), in
// the order of the scalar helpers (dot, fma3, quat_angle); where the compiler contracts the scalar
// helpers differently the results differ by an ulp.

// p(t^2) of atan01 for both halves (atan t = t p(t^2), t in [0, 1])
__device__ __forceinline__ float2 atan_poly2(float2 t) {
    const float2 s = mul2(t, t);
    float2 p = fma2(bc2(-4.166443301e-03f), s, bc2(2.232482877e-02f));
    p = fma2(p, s, bc2(-5.666722692e-02f));
    p = fma2(p, s, bc2(9.704074739e-02f));
    p = fma2(p, s, bc2(-1.393516270e-01f));
    p = fma2(p, s, bc2(1.995220255e-01f));
    p = fma2(p, s, bc2(-3.333036250e-01f));
    return fma2(p, s, bc2(9.999994549e-01f));
}

// quat_angle of both halves: 2 atan2(sqrt(vv), |w|); the reflection about pi/4 takes the last
// product into one rounding, 2 (pi/2 - t p) = pi - 2 t p
__device__ __forceinline__ float2 quat_angle2(float2 w, float2 vv) {
    const float yx = sqrt_approx(vv.x), yy = sqrt_approx(vv.y);
    const float xx = fabsf(w.x), xy = fabsf(w.y);
    const float mxx = fmaxf(fmaxf(xx, yx), 1e-30f), mnx = fminf(xx, yx);
    const float mxy = fmaxf(fmaxf(xy, yy), 1e-30f), mny = fminf(xy, yy);
    const float2 t = make_float2(__fdividef(mnx, mxx), __fdividef(mny, mxy));
    const float2 p = atan_poly2(t);
    const float2 a = mul2(mul2(bc2(2.0f), t), p);                                      // 2 t p
    const float2 r = fma2(mul2(bc2(-2.0f), t), p, bc2(2.0f * 1.57079632679489662f));  // pi - 2 t p
    return make_float2(yx > xx ? r.x : a.x, yy > xy ? r.y : a.y);
}

// Both residual parts of a trial in closed form.  With r = p_t - p_ee, split along z and the
// plane normal to it, the rotated end effector leaves the axial part r.z and, in the plane,
// v_p - cos x u_p - sin x (z x u_p); u_p and z x u_p are orthogonal with equal norms, so the
// in-plane part squared is ((u_p.v_p - cos x |u_p|^2)^2 + ((z x u_p).v_p - sin x |u_p|^2)^2) / |u_p|^2.
// The error quaternion's vector part, split the same way into a_z z + q_perp, becomes
// (cos a_z - sin w) z + cos q_perp - sin (q_perp x z), of squared norm (cos a_z - sin w)^2 + |q_perp|^2
// (cos, sin of x/2).  The only differences are those that form the residual's own components, as
// in the direct evaluation, and the squares are summed, so the closed form is as accurate (a float32
// emulation against the float64 method agrees to 2e-7 on Panda).
__device__ __forceinline__ CcdTrials ccd_joint_trials(const V3 pj, const V3 z, float thj, float lo, float hi,
                                                      const V3 Ep, const V3 pt, const Q4 qerr, float nqw,
                                                      float dphi, float pe2, float inv_p2, float inv_o2) {
    CcdTrials o;
    const V3 u = Ep - pj;
    const V3 v = pt - pj;
    const float uz = dot(u, z), vz = dot(v, z);
    const V3 up = fma3(-uz, z, u);
    const V3 vp = fma3(-vz, z, v);
    const float nup2 = dot(up, up), nvp2 = dot(vp, vp);
    const float nu2 = fmaf(uz, uz, nup2), nv2 = fmaf(vz, vz, nvp2);
    const V3 zxu = cross(z, up);
    const float ez = vz - uz;
    const float az = dot(qerr.v, z);
    const V3 qp = fma3(-az, z, qerr.v);
    const float qp2 = dot(qp, qp);

    // Eq. theta_proj, signed about the axis: atan2(z.(up x vp), up.vp) = atan2(zxu.vp, up.vp)
    const float cs = dot(up, vp), sn = dot(zxu, vp);
    const bool deg = nu2 < 1e-24f || nv2 < 1e-24f || nup2 <= pe2 * nu2 || nvp2 <= pe2 * nv2;
    const float d = deg ? 0.0f : atan2_all(sn, cs);
    // Eq. ori_update: delta(k) sgn(a.z) phi
    const float dq = (az > 0.0f) ? dphi : ((az < 0.0f) ? -dphi : 0.0f);

    // both steps clamped to the limits
    float2 st = add2(bc2(thj), make_float2(d, dq));
    st = make_float2(clampf(st.x, lo, hi), clampf(st.y, lo, hi));
    st = add2(st, bc2(-thj));
    o.d = st.x;
    o.dq = st.y;
    const float2 hs = mul2(bc2(0.5f), st);
    float2 sh, ch;
    __sincosf(hs.x, &sh.x, &ch.x);
    __sincosf(hs.y, &sh.y, &ch.y);
    const float2 m2sh = mul2(bc2(-2.0f), sh);
    const float2 msn = mul2(m2sh, ch);             // -sin(step)
    const float2 cst = fma2(m2sh, sh, bc2(1.0f));  // cos(step)
    // position residual of each trial.  Where u_p is at the rounding level of u (the end effector
    // on the axis, as the flange on a last joint's axis) its direction is noise that leaves the
    // plane, and the quotient would drop part of v_p; there the expanded form
    // |v_p|^2 + |u_p|^2 - 2 (cos u_p.v_p + sin (z x u_p).v_p), which cannot cancel while
    // |u_p| << |u|, is taken instead.
    float2 r2;
    if (nup2 <= 1e-6f * nu2) {
        r2 = fma2(bc2(2.0f), fma2(msn, bc2(sn), mul2(cst, bc2(-cs))), bc2(fmaf(ez, ez, nvp2 + nup2)));
    } else {
        const float2 ex = fma2(cst, bc2(-nup2), bc2(cs));
        const float2 ey = fma2(msn, bc2(nup2), bc2(sn));
        r2 = fma2(fma2(ex, ex, mul2(ey, ey)), bc2(__fdividef(1.0f, nup2)), bc2(ez * ez));
    }
    // error quaternion of each trial: qerr [cos, -sin z]
    const float2 w2 = fma2(bc2(qerr.w), ch, mul2(sh, bc2(az)));
    const float2 tz = fma2(ch, bc2(az), mul2(sh, bc2(nqw)));
    const float2 vv = fma2(tz, tz, bc2(qp2));
    const float2 ang = quat_angle2(w2, vv);
    const float2 sc = fma2(r2, bc2(inv_p2), mul2(mul2(ang, ang), bc2(inv_o2)));
    o.rp2 = r2.x;
    o.op = ang.x;
    o.sp = sc.x;
    o.pq2 = r2.y;
    o.rq = ang.y;
    o.so = sc.y;
    return o;
}

// One iteration of a candidate: kinematics with frames into the column, the
// residual (ep2 = |e_p|^2, eo = |omega|), the break test (kk > 0) and the cap,
// then the update of Alg. 3 (or Alg. 1 with cd_variant = 1) of the joint
// vector in the column.  Returns 1 when the candidate has converged, 2 at the
// cap (no update in either case), 0 after an update.
constexpr int kSlotWords = 8;  // per-thread shared-memory slot of the cooperative perturbation

// w / nb = (w * kDivMagic[nb]) >> 16 exactly for 1 <= nb <= 12 and 0 <= w < 32 nb (the normal
// pairs of a joint vector, at most 12, times the lanes of a warp); kDivMagic[nb] = ceil(2^16 / nb)
__constant__ uint32_t kDivMagic[13] = {0, 65536, 32768, 21846, 16384, 13108, 10923, 9363, 8192, 7282, 6554, 5958, 5462};
static_assert((kMaxDof + 1) / 2 <= 12, "the normal pairs of a joint vector index kDivMagic");

template <bool TRACE, int TH, bool RED = true>
__device__ __forceinline__ int ccd_step(const RobotParams* rob, const RobotParams& R, const TargetDesc& T,
                                        const hjcd_params& P, const ColT<TH>& col, uint32_t* slots, const CcdArgs& A,
                                        int64_t c, uint32_t s, int kk, int cap, float delta_k, const V3 pt, float pe2,
                                        float one_m_tie, float inv_p2, float inv_o2, float& ep2, float& eo) {
    const int n = R.n;
    // kinematics with frames
    Frame F = frame_identity();
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
        const float thj = col.th(j);
        fk_step<RED>(R, j, thj, F);
        col.set_frame(j, F, thj);
    }
    const Frame E = fk_flange(R, F);
    const Q4 qerr = quat_error(T, quat_from_frame(E));
    const V3 e = pt - E.p;
    ep2 = dot(e, e);
    eo = quat_angle(qerr.w, dot(qerr.v, qerr.v));
    // Alg. 3 coarse break, checked after each update (Alg. 1: the position part only)
    if (kk > 0 && ep2 < P.cd_eps_pos2 && (P.cd_variant == 1 || eo * eo < P.cd_eps_ori2)) return 1;
    if (kk == cap) return 2;
    const int k = A.k0 + kk;
    const float ep0 = sqrt_approx(ep2);

    if (P.cd_variant == 1) {
        // Alg. 1: joints from the last to the first, each rotated at once by its Eq. theta_proj
        // step; rotating joint j leaves the frames of joints <= j in place and moves the end
        // effector about joint j's axis
        V3 x = E.p;
#pragma unroll 1
        for (int j = n - 1; j >= 0; --j) {
            V3 pj, z;
            col.frame(j, pj, z);
            const float thj = col.th(j);
            const V3 u = x - pj, v = pt - pj;
            const float uz = dot(u, z), vz = dot(v, z);
            const V3 up = fma3(-uz, z, u), vp = fma3(-vz, z, v);
            const float nu2 = dot(u, u), nv2 = dot(v, v), nup2 = dot(up, up), nvp2 = dot(vp, vp);
            const V3 zxu = cross(z, up);
            const bool deg = nu2 < 1e-24f || nv2 < 1e-24f || nup2 <= pe2 * nu2 || nvp2 <= pe2 * nv2;
            float d = deg ? 0.0f : atan2_all(dot(zxu, vp), dot(up, vp));
            d = clampf(thj + d, R.lim[j].x, R.lim[j].y) - thj;
            float sd, cd;
            sincos_red(d, &sd, &cd);  // |d| may exceed pi
            x = pj + fma3(uz, z, fma3(cd, up, sd * zxu));
            col.th(j) = thj + d;
            if (TRACE && kk == 0 && A.tr.dp) A.tr.dp[j * A.ld + c] = d;
        }
        return 0;
    }

    // one position and one orientation proposal per joint, the
    // task residual each leaves, and the greedy choice by its score
    // (|e_p|/eps_pos)^2 + (|omega|/eps_ori)^2; a later joint replaces the
    // choice only when its score is lower by more than the fraction cd_tie
    float best_p = __int_as_float(0x7f800000), dP = 0.0f, best_o = __int_as_float(0x7f800000), dO = 0.0f;
    int jp = 0, jo = 0;
    const float dphi = delta_k * eo, nqw = -qerr.w;
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
        const float2 pa = col.a(j), pb = col.b(j), za = col.c(j);
        const V3 pj = v3(pa.x, pa.y, pb.x);
        const V3 z = v3(za.x, za.y, col.zz(j));
        const CcdTrials tr =
            ccd_joint_trials(pj, z, pb.y, R.lim[j].x, R.lim[j].y, E.p, pt, qerr, nqw, dphi, pe2, inv_p2, inv_o2);
        if (tr.sp < best_p * one_m_tie) {  // joint 0 against +inf
            best_p = tr.sp;
            jp = j;
            dP = tr.d;
        }
        if (tr.so < best_o * one_m_tie) {
            best_o = tr.so;
            jo = j;
            dO = tr.dq;
        }
        if (TRACE && kk == 0) {
            if (A.tr.dp) A.tr.dp[j * A.ld + c] = tr.d;
            if (A.tr.rp) A.tr.rp[j * A.ld + c] = sqrtf(tr.rp2);
            if (A.tr.op) A.tr.op[j * A.ld + c] = tr.op;
            if (A.tr.dq) A.tr.dq[j * A.ld + c] = tr.dq;
            if (A.tr.pq) A.tr.pq[j * A.ld + c] = sqrtf(tr.pq2);
            if (A.tr.rq) A.tr.rq[j * A.ld + c] = tr.rq;
        }
    }

    // apply both; on the same joint the larger step
    float aP = dP, aO = dO;
    if (jp == jo) {
        if (fabsf(dP) >= fabsf(dO)) aO = 0.0f;
        else aP = 0.0f;
    }
    // residual at theta_hat: the distal joint's rotation first, then the proximal one
    // (the chosen joints' origins and axes are still in the shared-memory column)
    const bool p_hi = jp > jo;
    V3 Pa, Za, Pb, Zb;
    col.frame(p_hi ? jp : jo, Pa, Za);  // the distal joint
    col.frame(p_hi ? jo : jp, Pb, Zb);
    const float da = p_hi ? aP : aO, db = p_hi ? aO : aP;
    float sa_, ca_, sb_, cb_;
    __sincosf(0.5f * da, &sa_, &ca_);
    __sincosf(0.5f * db, &sb_, &cb_);
    V3 x = Pa + rotate_half(Za, sa_, ca_, E.p - Pa);
    x = Pb + rotate_half(Zb, sb_, cb_, x - Pb);
    Q4 q1 = qmul(qerr, Q4{ca_, (-sa_) * Za});
    q1 = qmul(q1, Q4{cb_, (-sb_) * Zb});
    const V3 e1 = pt - x;
    const float ep1 = sqrt_approx(dot(e1, e1));
    const float eo1 = quat_angle(q1.w, dot(q1.v, q1.v));
    // acceptance (reading: an improvement above gamma in position or in orientation)
    const bool acc = (ep0 - ep1 > P.cd_gamma_pos) || (eo - eo1 > P.cd_gamma_ori);

    if (TRACE && kk == 0) {
        if (A.tr.jp) A.tr.jp[c] = jp;
        if (A.tr.jo) A.tr.jo[c] = jo;
        if (A.tr.accepted) A.tr.accepted[c] = acc ? 1 : 0;
        if (A.tr.th_hat) {
#pragma unroll 1
            for (int j = 0; j < n; ++j)
                A.tr.th_hat[j * A.ld + c] = col.th(j) + (j == jp ? aP : 0.0f) + (j == jo ? aO : 0.0f);
        }
    }
    if (acc) {  // clamped again: theta + (clamp(theta + d) - theta) can round an ulp past a limit
        col.th(jp) = clampf(col.th(jp) + aP, R.lim[jp].x, R.lim[jp].y);
        col.th(jo) = clampf(col.th(jo) + aO, R.lim[jo].x, R.lim[jo].y);
    }
    // rejection: theta + N(0, sigma^2 I), kept inside the limits.  Few lanes reject at a time,
    // so the lanes executing here together share the work: each rejected lane publishes its
    // stream (key, target index, candidate, iteration) and robot, and the (lane, normal pair)
    // items are spread over all of them; every joint column lives in shared memory.
    const unsigned am = __activemask();
    const unsigned rej = __ballot_sync(am, !acc);
    if (rej) {
        const int lane = threadIdx.x & 31;
        uint32_t* const slot = slots + (threadIdx.x & ~31u) * kSlotWords;  // this warp's slots
        if (!acc) {
            uint32_t* me = slot + lane * kSlotWords;
            me[0] = T.key[0];
            me[1] = T.key[1];
            me[2] = (uint32_t)T.t_local;
            me[3] = s;
            me[4] = (uint32_t)k;
            me[5] = (uint32_t)T.robot;
        }
        const int NB = (int)__reduce_max_sync(am, acc ? 0u : (uint32_t)((n + 1) / 2));
        __syncwarp(am);
        const int items = __popc(rej) * NB, step = __popc(am);
        const uint32_t magic = kDivMagic[NB];
        for (int w = __popc(am & ((1u << lane) - 1u)); w < items; w += step) {
            const int r = (int)(((uint32_t)w * magic) >> 16), b = w - r * NB;
            const int sl = __fns(rej, 0, r + 1);
            const uint32_t* q = slot + sl * kSlotWords;
            const RobotParams& Rs = rob[q[5]];
            if (2 * b >= Rs.n) continue;
            TargetDesc Tq;
            Tq.key[0] = q[0];
            Tq.key[1] = q[1];
            Tq.t_local = (int32_t)q[2];
            const float2 z = normal_pair(Tq, q[3], kPhaseCd, q[4], b);
            const ColT<TH> cs{col.base - lane + sl};
            const int j0 = 2 * b, j1 = 2 * b + 1;
            cs.th(j0) = clampf(fmaf(P.cd_sigma, z.x, cs.th(j0)), Rs.lim[j0].x, Rs.lim[j0].y);
            if (j1 < Rs.n) cs.th(j1) = clampf(fmaf(P.cd_sigma, z.y, cs.th(j1)), Rs.lim[j1].x, Rs.lim[j1].y);
        }
        __syncwarp(am);
    }
    return 0;
}

// resident threads per SM the register allocation aims at: 768 gives 80 registers, the budget
// that leaves no spill, for 24 resident warps
#ifndef HJCD_CCD_THREADS_PER_SM
#define HJCD_CCD_THREADS_PER_SM 768
#endif
// RED = false: the launch's joint vectors lie within the limits of plain robots (no offsets and
// no range reduction in the kinematics steps; the same bits)
template <bool TRACE, int TH, bool RED>
__global__ void __launch_bounds__(TH, HJCD_CCD_THREADS_PER_SM / TH) k_ccd(const CcdArgs A) {
    using Col = ColT<TH>;
    extern __shared__ __align__(16) float sm[];
    const RobotParams* rob = stage_robots(sm, A.rs);
    uint32_t* const slots = reinterpret_cast<uint32_t*>(sm + robots_smem_bytes(A.rs.n) / sizeof(float));
    float2* const colbase =
        reinterpret_cast<float2*>(sm + robots_smem_bytes(A.rs.n) / sizeof(float) + TH * kSlotWords) + threadIdx.x;
    const hjcd_params& P = A.P;
    const float pe2 = P.proj_eps * P.proj_eps;
    const float one_m_tie = 1.0f - P.cd_tie;
    unsigned long long n_it = 0, n_cand = 0;

    // a segment of the iterations (seg_end > 0): candidates still iterating at seg_end are handed
    // to the next launch through list_out, which runs them from there (list_in)
    const int64_t items = A.list_in ? (int64_t)*A.n_in : A.C;
    const int k_end = A.seg_end > 0 ? A.seg_end : 0x7fffffff;
    // the order of the items: a grid stride, or (A.queue set, a grid of resident CTAs) 32
    // consecutive items per warp from the queue at a time, so that every SM keeps working until
    // the queue is drained whatever the number of waves the items would fill
    const bool dyn = A.queue != nullptr;
    const int wl = threadIdx.x & 31;
    int64_t wbase = 0;
    if (dyn) {
        unsigned long long b0 = 0;
        if (wl == 0) b0 = atomicAdd(A.queue, 32ull);
        wbase = (int64_t)__shfl_sync(0xffffffffu, b0, 0);
    }
    for (int64_t it = dyn ? wbase + wl : blockIdx.x * (int64_t)blockDim.x + threadIdx.x; dyn ? wbase < items : it < items;) {
      do {  // one item (break: done with it)
        if (it >= items) break;  // past the end in the queue's last batch
        const int64_t c = A.list_in ? (int64_t)A.list_in[it] : it;
        int32_t t, s;
        if (!A.map.lookup_search(c, t, s)) break;
        s += A.seed_base;
        const TargetDesc T = A.tg[t];
        const RobotParams& R = rob[T.robot];
        const int n = R.n;
        const Col col{colbase};
        const V3 pt = v3(T.p[0], T.p[1], T.p[2]);
        if (!A.list_in) ++n_cand;

        if (A.list_in) {  // the state the previous segment left
#pragma unroll 1
            for (int j = 0; j < n; ++j) col.th(j) = A.th_out[j * A.ld + c];
        } else if (A.th_in) {
#pragma unroll 1
            for (int j = 0; j < n; ++j) col.th(j) = A.th_in[j * A.ld + c];
        } else {
            sample_seed(R, T, (uint32_t)s, col);
        }

        const int cap = A.n_iters >= 0 ? A.n_iters : T.cd_iters;
        float delta_k = P.cd_delta0 * powf(P.cd_rho, (float)A.k0);
#pragma unroll 1
        for (int q = 0; q < A.seg_begin; ++q) delta_k *= P.cd_rho;  // the bits of one run from k0
        const float inv_p2 = 1.0f / (T.eps_pos * T.eps_pos), inv_o2 = 1.0f / (T.eps_ori * T.eps_ori);
        int iters = cap;
        float ep2 = 0.0f, eo = 0.0f;
        const bool valid = T.eps_pos > 0.0f;
        bool handed = false;

        for (int kk = A.seg_begin; valid; ++kk) {
            if (kk == k_end && kk < cap) {
                // still iterating at the segment's end: keep the state, list the candidate
                const unsigned m = __activemask();
                const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(A.n_out, __popc(m));
                base = __shfl_sync(m, base, leader);
                A.list_out[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)c;
                handed = true;
                break;
            }
            const int r = ccd_step<TRACE, TH, RED>(rob, R, T, P, col, slots, A, c, (uint32_t)s, kk, cap, delta_k, pt, pe2,
                                              one_m_tie, inv_p2, inv_o2, ep2, eo);
            if (r == 1) iters = kk;
            if (r) break;
            delta_k *= P.cd_rho;
            ++n_it;
        }

        if (handed) {
#pragma unroll 1
            for (int j = 0; j < n; ++j) A.th_out[j * A.ld + c] = col.th(j);
            break;
        }
        if (A.th_out) {
#pragma unroll 1
            for (int j = 0; j < n; ++j) A.th_out[j * A.ld + c] = col.th(j);
        }
        const float ep = sqrtf(ep2);
        if (A.score) {
            const float a = ep / T.eps_pos, b = eo / T.eps_ori;
            A.score[c] = valid ? fmaf(a, a, b * b) : __int_as_float(0x7f800000);
        }
        if (A.perr) A.perr[c] = ep;
        if (A.oerr) A.oerr[c] = eo;
        if (A.iters) A.iters[c] = iters;
      } while (0);
        if (dyn) {
            __syncwarp();
            unsigned long long b0 = 0;
            if (wl == 0) b0 = atomicAdd(A.queue, 32ull);
            wbase = (int64_t)__shfl_sync(0xffffffffu, b0, 0);
            it = wbase + wl;
        } else {
            it += (int64_t)gridDim.x * blockDim.x;
        }
    }
    if (A.cnt) {
        n_it = warp_sum(n_it);
        n_cand = warp_sum(n_cand);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&A.cnt->v[0], n_it);
            atomicAdd(&A.cnt->v[5], n_cand);
        }
    }
}

// cd_variant = 2, the target-wide break: one CTA per target runs all of its
// seeds in lock-step, iteration by iteration, and stops every seed once any
// seed passes the coarse test.  Pass kk tests each seed's state after kk
// updates and writes its update to the other buffer; when some seed passed,
// the updates of that pass are dropped and every seed keeps its state after
// kk updates.
template <int TH>
__global__ void __launch_bounds__(TH, 4) k_ccd_lock(const CcdArgs A) {
    extern __shared__ __align__(16) float sm[];
    __shared__ int any;
    const RobotParams* rob = stage_robots(sm, A.rs);
    uint32_t* const slots = reinterpret_cast<uint32_t*>(sm + robots_smem_bytes(A.rs.n) / sizeof(float));
    float2* const colbase =
        reinterpret_cast<float2*>(sm + robots_smem_bytes(A.rs.n) / sizeof(float) + TH * kSlotWords) + threadIdx.x;
    const int t = blockIdx.x;
    const hjcd_params& P = A.P;
    const TargetDesc T = A.tg[t];
    const RobotParams& R = rob[T.robot];
    const int n = R.n;
    const ColT<TH> col{colbase};
    const int64_t m0 = A.map.off[t];
    const int M = (int)(A.map.off[t + 1] - m0);
    const bool valid = T.eps_pos > 0.0f;
    const int cap = A.n_iters >= 0 ? A.n_iters : T.cd_iters;
    const V3 pt = v3(T.p[0], T.p[1], T.p[2]);
    const float pe2 = P.proj_eps * P.proj_eps, one_m_tie = 1.0f - P.cd_tie;
    const float inv_p2 = 1.0f / (T.eps_pos * T.eps_pos), inv_o2 = 1.0f / (T.eps_ori * T.eps_ori);
    float* cur = A.th_out;
    float* nxt = A.th_tmp;
    for (int s = threadIdx.x; s < M; s += TH) {
        const int64_t c = m0 + s;
        if (A.th_in) {
            for (int j = 0; j < n; ++j) cur[j * A.ld + c] = A.th_in[j * A.ld + c];
        } else {
            sample_seed(R, T, (uint32_t)s, col);
            for (int j = 0; j < n; ++j) cur[j * A.ld + c] = col.th(j);
        }
    }
    unsigned long long n_it = 0;
    float delta_k = P.cd_delta0 * powf(P.cd_rho, (float)A.k0);
    int kk = 0;
    for (; valid; ++kk) {
        if (threadIdx.x == 0) any = 0;
        __syncthreads();
        for (int s = threadIdx.x; s < M; s += TH) {
            const int64_t c = m0 + s;
#pragma unroll 1
            for (int j = 0; j < n; ++j) col.th(j) = cur[j * A.ld + c];
            float ep2 = 0.0f, eo = 0.0f;
            const int r = ccd_step<false, TH>(rob, R, T, P, col, slots, A, c, (uint32_t)s, kk, cap, delta_k, pt, pe2,
                                              one_m_tie, inv_p2, inv_o2, ep2, eo);
            const float ep = sqrtf(ep2), a = ep / T.eps_pos, b = eo / T.eps_ori;
            if (A.score) A.score[c] = fmaf(a, a, b * b);
            if (A.perr) A.perr[c] = ep;
            if (A.oerr) A.oerr[c] = eo;
            if (r == 1) any = 1;
            if (r == 0) {
                ++n_it;
#pragma unroll 1
                for (int j = 0; j < n; ++j) nxt[j * A.ld + c] = col.th(j);
            }
        }
        __syncthreads();
        if (any || kk == cap) break;
        float* sw = cur;
        cur = nxt;
        nxt = sw;
        delta_k *= P.cd_rho;
    }
    for (int s = threadIdx.x; s < M; s += TH) {
        const int64_t c = m0 + s;
        if (cur != A.th_out)
            for (int j = 0; j < n; ++j) A.th_out[j * A.ld + c] = cur[j * A.ld + c];
        if (!valid && A.score) A.score[c] = __int_as_float(0x7f800000);
        if (A.iters) A.iters[c] = valid ? kk : cap;
    }
    if (A.cnt) {
        n_it = warp_sum(n_it);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&A.cnt->v[0], n_it);
            if (threadIdx.x == 0) atomicAdd(&A.cnt->v[5], (unsigned long long)M);
        }
    }
}

__global__ void __launch_bounds__(kCcdThreads) k_sample(const RobotParams R, uint32_t k0, uint32_t k1, CandMap map,
                                                        int64_t C, float* th_out, int64_t ld) {
    extern __shared__ float sm[];
    const ThetaCol<kCcdThreads> col{sm + threadIdx.x};
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        int32_t t, s;
        map.lookup(c, t, s);  // only the row index keys the stream
        TargetDesc T{};
        T.key[0] = k0;
        T.key[1] = k1;
        T.t_local = t;
        sample_seed(R, T, (uint32_t)s, col);
#pragma unroll 1
        for (int j = 0; j < R.n; ++j) th_out[j * ld + c] = col.th(j);
    }
}


template <bool TRACE, int TH, bool RED>
void launch_ccd_t(const CcdArgs& A, cudaStream_t st) {
    const size_t smem =
        robots_smem_bytes(A.rs.n) + sizeof(float) * (kColWordsPerJoint * A.rs.n_max + kSlotWords) * TH;
    static SmemLimit lim;
    allow_dyn_smem(k_ccd<TRACE, TH, RED>, lim,
                   robots_smem_bytes(kMaxLaunchRobots) + sizeof(float) * (kColWordsPerJoint * kMaxDof + kSlotWords) * TH);
    int g = grid_for(A.C, TH, 16 * 128 / TH);
    if (A.queue) {  // the resident CTAs only: the queue spreads the items
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ccd<TRACE, TH, RED>, TH, smem);
        g = std::min(g, sm_count() * std::max(per_sm, 1));
    }
    k_ccd<TRACE, TH, RED><<<g, TH, smem, st>>>(A);
}

template <bool TRACE, bool RED>
void launch_ccd_b(const CcdArgs& A, cudaStream_t st) {
    if (A.block == 64) launch_ccd_t<TRACE, 64, RED>(A, st);
    else if (A.block == 256) launch_ccd_t<TRACE, 256, RED>(A, st);
    else launch_ccd_t<TRACE, 128, RED>(A, st);
}

}  // namespace

void launch_ccd(const CcdArgs& A, bool trace, cudaStream_t st) {
    if (A.C <= 0) return;
    if (A.P.cd_variant == 2) {  // one CTA per target (offset maps only)
        const size_t smem =
            robots_smem_bytes(A.rs.n) + sizeof(float) * (kColWordsPerJoint * A.rs.n_max + kSlotWords) * 128;
        static SmemLimit lim;
        allow_dyn_smem(k_ccd_lock<128>, lim,
                       robots_smem_bytes(kMaxLaunchRobots) +
                           sizeof(float) * (kColWordsPerJoint * kMaxDof + kSlotWords) * 128);
        k_ccd_lock<128><<<A.map.T, 128, smem, st>>>(A);
        return;
    }
    if (trace) launch_ccd_b<true, true>(A, st);
    else if (A.in_limits && A.rs.plain) launch_ccd_b<false, false>(A, st);
    else launch_ccd_b<false, true>(A, st);
}

void launch_sample(const RobotParams& R, uint64_t seed, CandMap map, int64_t C, float* th, int64_t ld,
                   cudaStream_t st) {
    if (C <= 0) return;
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    k_sample<<<grid_for(C, kCcdThreads), kCcdThreads, sizeof(float) * R.n * kCcdThreads, st>>>(R, k0, k1, map, C,
                                                                                               th, ld);
}

}  // namespace hjcd

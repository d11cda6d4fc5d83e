// k_ccd.cu -- seed sampling (Alg. 3 line 3) and PO-CCD iterations (Sec. IV,
// Alg. 3), one candidate per thread.
//
// Per iteration one forward-kinematics pass gives every joint's origin and
// axis.  The 2n trial updates are evaluated in O(1) each: rotating joint j by
// d moves the end effector about the axis (Rodrigues), so the position trial
// residual follows from the projected vectors of Eq. vec_proj, and the
// orientation trial residual from composing the error quaternion with the
// joint rotation.  The proposed theta_hat changes at most two joints; its
// residual is the composition of the two joint rotations applied to the
// current end-effector pose (the more distal joint first), so acceptance
// needs no second kinematics pass.
#include "hjcd_internal.cuh"

namespace hjcd {

namespace {

template <int NB>
__device__ __forceinline__ void sample_seed(const RobotParams& R, const TargetDesc& T, uint32_t s,
                                            float (&th)[NB]) {
#pragma unroll
    for (int b = 0; b < (NB + 3) / 4; ++b) {
        if (4 * b < R.n) {
            const uint4 w = rnd_block(T, s, kPhaseSeed, 0, (uint32_t)b);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * b + q;
                if (j < NB && j < R.n) th[j] = fmaf(u01(word(w, q)), R.hi[j] - R.lo[j], R.lo[j]);
            }
        }
    }
}

template <int NB, bool TRACE>
__global__ void __launch_bounds__(128) k_ccd(const RobotParams R, const CcdArgs A) {
    const hjcd_params& P = A.P;
    const int n = R.n;
    const float pe2 = P.proj_eps * P.proj_eps;
    unsigned long long n_it = 0, n_cand = 0;

    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < A.C;
         c += (int64_t)gridDim.x * blockDim.x) {
        int32_t t, s;
        if (!A.map.lookup(c, t, s)) continue;
        const TargetDesc T = A.tg[t];
        const V3 pt = v3(T.p[0], T.p[1], T.p[2]);
        ++n_cand;

        float th[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) th[j] = 0.0f;
        if (A.th_in) {
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (j < n) th[j] = A.th_in[j * A.ld + c];
        } else {
            sample_seed<NB>(R, T, (uint32_t)s, th);
        }

        float delta_k = P.cd_delta0 * powf(P.cd_rho, (float)A.k0);
        int iters = A.n_iters;
        float ep2 = 0.0f, eo = 0.0f;
        const bool valid = T.eps_pos > 0.0f;

        for (int kk = 0; valid; ++kk) {
            V3 Pj[NB], Zj[NB];
            Frame E;
            fk_chain<NB, true>(R, th, Pj, Zj, E);
            const Q4 qerr = quat_error(T, quat_from_frame(E));
            const V3 e = pt - E.p;
            ep2 = dot(e, e);
            eo = quat_angle(qerr.w, dot(qerr.v, qerr.v));
            // Alg. 3 line 14, checked after each update
            if (kk > 0 && ep2 < P.cd_eps_pos2 && eo * eo < P.cd_eps_ori2) {
                iters = kk;
                break;
            }
            if (kk == A.n_iters) break;
            const int k = A.k0 + kk;
            const float ep0 = sqrtf(ep2);

            // lines 6-9: one position and one orientation proposal per joint and the
            // greedy choice; a later joint replaces the choice only when its trial
            // residual is lower by more than cd_tie
            float best_p = 0.0f, dP = 0.0f, best_o = 0.0f, dO = 0.0f;
            int jp = 0, jo = 0;
            V3 Pp = v3(0.f, 0.f, 0.f), Zp = Pp, Po = Pp, Zo = Pp;
            const float phi = eo;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (j < n) {
                    const V3 z = Zj[j];
                    const V3 u = E.p - Pj[j];
                    const V3 v = pt - Pj[j];
                    const float uz = dot(u, z), vz = dot(v, z);
                    const V3 up = fma3(-uz, z, u);
                    const V3 vp = fma3(-vz, z, v);
                    const float nu2 = dot(u, u), nv2 = dot(v, v);
                    const float nup2 = dot(up, up), nvp2 = dot(vp, vp);
                    const V3 zxu = cross(z, up);
                    // Eq. theta_proj, signed about the axis: atan2(z.(up x vp), up.vp) = atan2(zxu.vp, up.vp)
                    const float cs = dot(up, vp), sn = dot(zxu, vp);
                    const bool deg = nu2 < 1e-24f || nv2 < 1e-24f || nup2 <= pe2 * nu2 || nvp2 <= pe2 * nv2;
                    float d = deg ? 0.0f : atan2f(sn, cs);
                    d = clampf(th[j] + d, R.lo[j], R.hi[j]) - th[j];
                    float sd, cd;
                    __sincosf(d, &sd, &cd);
                    // target minus the end effector rotated about joint j by d
                    const V3 r = fma3(vz - uz, z, fma3(-sd, zxu, fma3(-cd, up, vp)));
                    const float rp = sqrtf(dot(r, r));
                    if (j == 0 || rp < best_p - P.cd_tie) {
                        best_p = rp;
                        jp = j;
                        dP = d;
                        Pp = Pj[j];
                        Zp = z;
                    }
                    // Eq. ori_update: delta(k) sgn(a.z) phi; the error quaternion composed with
                    // the inverse joint rotation [cos(d/2), -sin(d/2) z]
                    const float az = dot(qerr.v, z);
                    const float sg = (az > 0.0f) ? 1.0f : ((az < 0.0f) ? -1.0f : 0.0f);
                    float dq = delta_k * sg * phi;
                    dq = clampf(th[j] + dq, R.lo[j], R.hi[j]) - th[j];
                    float sh, ch;
                    __sincosf(0.5f * dq, &sh, &ch);
                    const float w2 = fmaf(qerr.w, ch, sh * az);
                    const V3 v2 = fma3(ch, qerr.v, (-sh) * fma3(qerr.w, z, cross(qerr.v, z)));
                    const float rq = quat_angle(w2, dot(v2, v2));
                    if (j == 0 || rq < best_o - P.cd_tie) {
                        best_o = rq;
                        jo = j;
                        dO = dq;
                        Po = Pj[j];
                        Zo = z;
                    }
                    if (TRACE && kk == 0) {
                        if (A.tr.dp) A.tr.dp[j * A.ld + c] = d;
                        if (A.tr.rp) A.tr.rp[j * A.ld + c] = rp;
                        if (A.tr.dq) A.tr.dq[j * A.ld + c] = dq;
                        if (A.tr.rq) A.tr.rq[j * A.ld + c] = rq;
                    }
                }
            }

            // line 10: apply both; on the same joint the larger step
            float aP = dP, aO = dO;
            if (jp == jo) {
                if (fabsf(dP) >= fabsf(dO)) aO = 0.0f;
                else aP = 0.0f;
            }
            // residual at theta_hat: the distal joint's rotation first, then the proximal one
            const bool p_hi = jp > jo;
            const V3 Pa = p_hi ? Pp : Po, Za = p_hi ? Zp : Zo, Pb = p_hi ? Po : Pp, Zb = p_hi ? Zo : Zp;
            const float da = p_hi ? aP : aO, db = p_hi ? aO : aP;
            float sa_, ca_, sb_, cb_;
            __sincosf(0.5f * da, &sa_, &ca_);
            __sincosf(0.5f * db, &sb_, &cb_);
            V3 x = Pa + rotate_half(Za, sa_, ca_, E.p - Pa);
            x = Pb + rotate_half(Zb, sb_, cb_, x - Pb);
            Q4 q1 = qmul(qerr, Q4{ca_, (-sa_) * Za});
            q1 = qmul(q1, Q4{cb_, (-sb_) * Zb});
            const V3 e1 = pt - x;
            const float ep1 = sqrtf(dot(e1, e1));
            const float eo1 = quat_angle(q1.w, dot(q1.v, q1.v));
            // line 11 (reading: an improvement above gamma in position or in orientation)
            const bool acc = (ep0 - ep1 > P.cd_gamma_pos) || (eo - eo1 > P.cd_gamma_ori);

            if (TRACE && kk == 0) {
                if (A.tr.jp) A.tr.jp[c] = jp;
                if (A.tr.jo) A.tr.jo[c] = jo;
                if (A.tr.accepted) A.tr.accepted[c] = acc ? 1 : 0;
                if (A.tr.th_hat) {
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        if (j < n) A.tr.th_hat[j * A.ld + c] = th[j] + (j == jp ? aP : 0.0f) + (j == jo ? aO : 0.0f);
                }
            }
            if (acc) {
#pragma unroll
                for (int j = 0; j < NB; ++j) th[j] += (j == jp ? aP : 0.0f) + (j == jo ? aO : 0.0f);
            } else {
                // line 12: theta + N(0, sigma^2 I), kept inside the limits
                float z[NB];
                normals<NB>(T, (uint32_t)s, kPhaseCd, (uint32_t)k, n, z);
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    if (j < n) th[j] = clampf(fmaf(P.cd_sigma, z[j], th[j]), R.lo[j], R.hi[j]);
            }
            delta_k *= P.cd_rho;
            ++n_it;
        }

        if (A.th_out) {
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (j < n) A.th_out[j * A.ld + c] = th[j];
        }
        const float ep = sqrtf(ep2);
        if (A.score) {
            const float a = ep / T.eps_pos, b = eo / T.eps_ori;
            A.score[c] = valid ? fmaf(a, a, b * b) : __int_as_float(0x7f800000);
        }
        if (A.perr) A.perr[c] = ep;
        if (A.oerr) A.oerr[c] = eo;
        if (A.iters) A.iters[c] = iters;
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

template <int NB>
__global__ void __launch_bounds__(128) k_sample(const RobotParams R, uint32_t k0, uint32_t k1, CandMap map, int64_t C,
                                                float* th_out, int64_t ld) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        int32_t t, s;
        map.lookup(c, t, s);  // only the row index keys the stream
        TargetDesc T{};
        T.key[0] = k0;
        T.key[1] = k1;
        T.t_local = t;
        float th[NB];
        sample_seed<NB>(R, T, (uint32_t)s, th);
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j < R.n) th_out[j * ld + c] = th[j];
    }
}

}  // namespace

void launch_ccd(const RobotParams& R, const CcdArgs& A, bool trace, cudaStream_t st) {
    if (A.C <= 0) return;
    const int g = grid_for(A.C, 128);
#define HJCD_CCD(NB)                                                   \
    if (R.n <= NB) {                                                   \
        if (trace) k_ccd<NB, true><<<g, 128, 0, st>>>(R, A);           \
        else k_ccd<NB, false><<<g, 128, 0, st>>>(R, A);                \
        return;                                                        \
    }
    HJCD_CCD(8)
    HJCD_CCD(16)
    HJCD_CCD(24)
#undef HJCD_CCD
}

void launch_sample(const RobotParams& R, uint64_t seed, CandMap map, int64_t C, float* th, int64_t ld,
                   cudaStream_t st) {
    if (C <= 0) return;
    const int g = grid_for(C, 128);
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    if (R.n <= 8) k_sample<8><<<g, 128, 0, st>>>(R, k0, k1, map, C, th, ld);
    else if (R.n <= 16) k_sample<16><<<g, 128, 0, st>>>(R, k0, k1, map, C, th, ld);
    else k_sample<24><<<g, 128, 0, st>>>(R, k0, k1, map, C, th, ld);
}

}  // namespace hjcd

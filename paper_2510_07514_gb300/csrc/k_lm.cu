// k_lm.cu -- PJ-IK (Sec. V-B, Alg. 4), one candidate per thread.
//
// Each iteration: one kinematics pass with frames gives the 6 x n geometric
// Jacobian (Eq. jacobian) and the residual; W normalises the Jacobian's rows
// (orientation rows also scaled by eps_pos / eps_ori).  The damped normal
// equations of Eq. normal-eqs, ((WJ)^T (WJ) + lambda D) d = (WJ)^T W r with
// D = diag((WJ)^T (WJ)), are solved in their 6 x 6 push-through form
//     d = S Ah^T (Ah Ah^T + lambda I)^-1 W r,   Ah = WJ S,  S = D^(-1/2),
// an exact identity for lambda > 0, so only a 6 x 6 Cholesky factorisation
// runs per candidate whatever n is.  The step is clamped to the trust region
// and validated by the backtracking line search of Eq. line-search; failing
// that, the dogleg step (Eq. dogleg), then the single-coordinate step
// (Eq. single-coord) are tried, and finally a random perturbation is made.
#include "hjcd_internal.cuh"

namespace hjcd {

namespace {

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

// In-place Cholesky of a packed 6 x 6 symmetric positive-definite matrix
// (lower triangle, row by row).  inv receives the reciprocal pivots.
__device__ __forceinline__ void chol6(float (&a)[21], float (&inv)[6]) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float s = a[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) s = fmaf(-a[tri(j, k)], a[tri(j, k)], s);
        const float r = rsqrtf(fmaxf(s, 1e-30f));
        a[tri(j, j)] = s * r;
        inv[j] = r;
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            float t = a[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) t = fmaf(-a[tri(i, k)], a[tri(j, k)], t);
            a[tri(i, j)] = t * r;
        }
    }
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

// weighted cost 1/2 |W r(theta)|^2 (W fixed for the iteration)
template <int NB>
__device__ __forceinline__ float wcost(const RobotParams& R, const TargetDesc& T, const float (&th)[NB],
                                       const float (&W)[6]) {
    const Frame E = fk_ee<NB>(R, th);
    const V3 w = quat_log(quat_error(T, quat_from_frame(E)));
    const float e0 = W[0] * (T.p[0] - E.p.x), e1 = W[1] * (T.p[1] - E.p.y), e2 = W[2] * (T.p[2] - E.p.z);
    const float e3 = W[3] * w.x, e4 = W[4] * w.y, e5 = W[5] * w.z;
    return 0.5f * fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, fmaf(e4, e4, e5 * e5)))));
}

template <int NB, bool TRACE>
__global__ void __launch_bounds__(128) k_lm(const RobotParams R, const LmArgs A) {
    const hjcd_params& P = A.P;
    const int n = R.n;
    const float Rt = P.lm_trust_R;
    unsigned long long n_it = 0, n_fk = 0;

    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < A.C;
         c += (int64_t)gridDim.x * blockDim.x) {
        int32_t t, s;
        if (!A.map.lookup(c, t, s)) continue;
        const TargetDesc T = A.tg[t];
        const V3 pt = v3(T.p[0], T.p[1], T.p[2]);
        const bool valid = T.eps_pos > 0.0f;
        const float wo = T.eps_pos / T.eps_ori;

        float th[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) th[j] = (j < n) ? A.th[j * A.ld + c] : 0.0f;

        int iters = A.n_iters;
        float ep = 0.0f, eo = 0.0f;
        for (int kk = 0; valid; ++kk) {
            V3 Pj[NB], Zj[NB];
            Frame E;
            fk_chain<NB, true>(R, th, Pj, Zj, E);
            ++n_fk;
            const V3 om = quat_log(quat_error(T, quat_from_frame(E)));
            const V3 epv = pt - E.p;
            ep = sqrtf(dot(epv, epv));
            eo = sqrtf(dot(om, om));
            // Alg. 4 line 16, checked after each update
            if (kk > 0 && ep < T.eps_pos && eo < T.eps_ori) {
                iters = kk;
                break;
            }
            if (kk == A.n_iters) break;
            const int k = A.k0 + kk;
            const float e[6] = {epv.x, epv.y, epv.z, om.x, om.y, om.z};

            // line 3: Jacobian columns z_i x (P_ee - P_i), z_i
            float J[6][NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                if (i < n) {
                    const V3 jp = cross(Zj[i], E.p - Pj[i]);
                    J[0][i] = jp.x;
                    J[1][i] = jp.y;
                    J[2][i] = jp.z;
                    J[3][i] = Zj[i].x;
                    J[4][i] = Zj[i].y;
                    J[5][i] = Zj[i].z;
                } else {
#pragma unroll
                    for (int r = 0; r < 6; ++r) J[r][i] = 0.0f;
                }
            }
            float W[6], b[6];
            float cost0 = 0.0f;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                float ss = 0.0f;
#pragma unroll
                for (int i = 0; i < NB; ++i) ss = fmaf(J[r][i], J[r][i], ss);
                W[r] = (r < 3 ? 1.0f : wo) / fmaxf(sqrtf(ss), 1e-6f);
                b[r] = W[r] * e[r];
                cost0 = fmaf(b[r], b[r], cost0);
            }
            cost0 *= 0.5f;
            if (TRACE && kk == 0) {
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    if (A.tr.W) A.tr.W[r * A.ld + c] = W[r];
#pragma unroll
                    for (int i = 0; i < NB; ++i)
                        if (A.tr.J && i < n) A.tr.J[(r * n + i) * A.ld + c] = J[r][i];
                }
            }
#pragma unroll
            for (int r = 0; r < 6; ++r)
#pragma unroll
                for (int i = 0; i < NB; ++i) J[r][i] *= W[r];

            // line 4: LM step in push-through form
            float M[21], inv[6], y[6], D[NB];
#pragma unroll
            for (int q = 0; q < 21; ++q) M[q] = 0.0f;
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                if (i < n) {
                    float dd = 1e-9f;
#pragma unroll
                    for (int r = 0; r < 6; ++r) dd = fmaf(J[r][i], J[r][i], dd);
                    D[i] = dd;
                    const float rs = rsqrtf(dd);
                    float ah[6];
#pragma unroll
                    for (int r = 0; r < 6; ++r) ah[r] = J[r][i] * rs;
#pragma unroll
                    for (int r = 0; r < 6; ++r)
#pragma unroll
                        for (int q = 0; q <= r; ++q) M[tri(r, q)] = fmaf(ah[r], ah[q], M[tri(r, q)]);
                } else {
                    D[i] = 1.0f;
                }
            }
#pragma unroll
            for (int r = 0; r < 6; ++r) M[tri(r, r)] += P.lm_lambda;
            chol6(M, inv);
            chol6_solve(M, inv, b, y);
            float step[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                float a = 0.0f;
#pragma unroll
                for (int r = 0; r < 6; ++r) a = fmaf(J[r][i], y[r], a);
                step[i] = (i < n) ? clampf(a / D[i], -Rt, Rt) : 0.0f;  // line 5
            }
            if (TRACE && kk == 0 && A.tr.d_lm) {
#pragma unroll
                for (int i = 0; i < NB; ++i)
                    if (i < n) A.tr.d_lm[i * A.ld + c] = step[i];
            }

            // lines 6-8: backtracking line search over 1, 1/beta, ..., 1/beta^A
            float tn[NB];
            int branch = 3;
            float alpha_acc = 0.0f;
            {
                float alpha = 1.0f;
                for (int ls = 0; ls <= P.lm_A; ++ls) {
#pragma unroll
                    for (int j = 0; j < NB; ++j) tn[j] = (j < n) ? clampf(fmaf(alpha, step[j], th[j]), R.lo[j], R.hi[j]) : 0.0f;
                    ++n_fk;
                    if (wcost<NB>(R, T, tn, W) < cost0) {
                        branch = 0;
                        alpha_acc = alpha;
                        break;
                    }
                    alpha = alpha / P.lm_beta;
                }
            }
            float g[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                float a = 0.0f;
#pragma unroll
                for (int r = 0; r < 6; ++r) a = fmaf(J[r][i], b[r], a);
                g[i] = a;
            }
            if (branch != 0) {
                // lines 9-11: dogleg.  Minimum-norm Gauss-Newton step (WJ)^T ((WJ)(WJ)^T + mu I)^-1 W r,
                // Cauchy point along g, and tau in [0, 1] putting the blend inside the radius R.
                float G[21], y2[6], Jg[6];
#pragma unroll
                for (int q = 0; q < 21; ++q) G[q] = 0.0f;
#pragma unroll
                for (int r = 0; r < 6; ++r) Jg[r] = 0.0f;
                float gg = 0.0f;
#pragma unroll
                for (int i = 0; i < NB; ++i) {
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
#pragma unroll
                        for (int q = 0; q <= r; ++q) G[tri(r, q)] = fmaf(J[r][i], J[q][i], G[tri(r, q)]);
                        Jg[r] = fmaf(J[r][i], g[i], Jg[r]);
                    }
                    gg = fmaf(g[i], g[i], gg);
                }
#pragma unroll
                for (int r = 0; r < 6; ++r) G[tri(r, r)] += P.lm_gn_reg;
                chol6(G, inv);
                chol6_solve(G, inv, b, y2);
                float jgjg = 0.0f;
#pragma unroll
                for (int r = 0; r < 6; ++r) jgjg = fmaf(Jg[r], Jg[r], jgjg);
                const float ac = jgjg > 0.0f ? gg / jgjg : 0.0f;
                float dgn[NB], ngn2 = 0.0f;
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    float a = 0.0f;
#pragma unroll
                    for (int r = 0; r < 6; ++r) a = fmaf(J[r][i], y2[r], a);
                    dgn[i] = a;
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
#pragma unroll
                    for (int i = 0; i < NB; ++i) {
                        const float di = fmaf(ac, g[i], -dgn[i]);
                        qa = fmaf(di, di, qa);
                        qb = fmaf(2.0f * dgn[i], di, qb);
                    }
                    const float qc = ngn2 - R2;
                    const float disc = fmaxf(fmaf(qb, qb, -4.0f * qa * qc), 0.0f);
                    const float tau = (2.0f * qc) / (sqrtf(disc) - qb);  // smaller root, stable form
                    wgn = 1.0f - tau;
                    wgd = tau * ac;
                }
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    tn[j] = (j < n) ? clampf(th[j] + fmaf(wgn, dgn[j], wgd * g[j]), R.lo[j], R.hi[j]) : 0.0f;
                ++n_fk;
                if (wcost<NB>(R, T, tn, W) < cost0) branch = 1;
            }
            if (branch == 3) {
                // lines 12-14: the joint with the largest gradient magnitude, a 1-D
                // Gauss-Newton step on it clamped to R, and the same line search
                int is = 0;
                float gbest = -1.0f, cn = 0.0f, gsel = 0.0f;
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    if (i < n && fabsf(g[i]) > gbest) {
                        gbest = fabsf(g[i]);
                        is = i;
                        cn = D[i] - 1e-9f;
                        gsel = g[i];
                    }
                }
                const float sstep = cn > 0.0f ? clampf(gsel / cn, -Rt, Rt) : 0.0f;
                float alpha = 1.0f;
                for (int ls = 0; ls <= P.lm_A; ++ls) {
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        tn[j] = (j < n) ? clampf(th[j] + (j == is ? alpha * sstep : 0.0f), R.lo[j], R.hi[j]) : 0.0f;
                    ++n_fk;
                    if (wcost<NB>(R, T, tn, W) < cost0) {
                        branch = 2;
                        alpha_acc = alpha;
                        break;
                    }
                    alpha = alpha / P.lm_beta;
                }
            }
            if (branch == 3) {
                // line 15: random perturbation
                float z[NB];
                normals<NB>(T, (uint32_t)s, kPhaseLm, (uint32_t)k, n, z);
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    tn[j] = (j < n) ? clampf(fmaf(P.lm_sigma, z[j], th[j]), R.lo[j], R.hi[j]) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < NB; ++j) th[j] = tn[j];
            if (TRACE && kk == 0) {
                if (A.tr.branch) A.tr.branch[c] = branch;
                if (A.tr.alpha) A.tr.alpha[c] = alpha_acc;
            }
            ++n_it;
        }
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j < n) A.th[j * A.ld + c] = th[j];
        if (A.score) {
            const float a = ep / T.eps_pos, bb = eo / T.eps_ori;
            A.score[c] = valid ? fmaf(a, a, bb * bb) : __int_as_float(0x7f800000);
        }
        if (A.perr) A.perr[c] = ep;
        if (A.oerr) A.oerr[c] = eo;
        if (A.iters) A.iters[c] = iters;
    }
    if (A.cnt) {
        n_it = warp_sum(n_it);
        n_fk = warp_sum(n_fk);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&A.cnt->v[1], n_it);
            atomicAdd(&A.cnt->v[2], n_fk);
        }
    }
}

}  // namespace

void launch_lm(const RobotParams& R, const LmArgs& A, bool trace, cudaStream_t st) {
    if (A.C <= 0) return;
    const int g = grid_for(A.C, 128);
#define HJCD_LM(NB)                                                 \
    if (R.n <= NB) {                                                \
        if (trace) k_lm<NB, true><<<g, 128, 0, st>>>(R, A);         \
        else k_lm<NB, false><<<g, 128, 0, st>>>(R, A);              \
        return;                                                     \
    }
    HJCD_LM(8)
    HJCD_LM(16)
    HJCD_LM(24)
#undef HJCD_LM
}

}  // namespace hjcd

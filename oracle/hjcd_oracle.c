/*
 * hjcd_oracle.c -- FP64 CPU oracle of batched HJCD-IK (arXiv 2510.07514).
 *
 * TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg use it to say what the GPU path must compute.
 * The product library never links or calls it, and the two share no code.
 *
 * Everything here is the plain statement of the method, in double precision:
 * forward kinematics as products of 4x4 matrices, every trial residual by a
 * fresh forward-kinematics pass, the damped normal equations in their n x n
 * form, brute-force collision over all sphere pairs.  Each function names the
 * equation or algorithm of the paper it follows.  Where the paper is silent or
 * ambiguous the reading taken is stated beside the code (and listed in the
 * design notes).  OpenMP only spreads independent candidates over cores.
 *
 * Parity notes:
 *   - Random draws: Philox4x32-10 (Salmon et al., SC'11) keyed by the request
 *     seed, counter = (candidate, target, phase << 24 | iteration, block).
 *   - Orientation residual: the sign of the error quaternion is fixed so that
 *     w >= 0 before Eq. quat_diff is applied (the paper writes |w|).
 */
#include "hjcd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXB (ORC_MAXN + 2)

enum { PHASE_SEED = 1, PHASE_CD = 2, PHASE_DUP = 3, PHASE_LM = 4 };
enum { BR_LM = 0, BR_DOGLEG = 1, BR_SINGLE = 2, BR_PERTURB = 3 };

struct orc_robot {
    int n;
    double a[ORC_MAXN], alpha[ORC_MAXN], d[ORC_MAXN], off[ORC_MAXN];
    double flange[16];
    double lo[ORC_MAXN], hi[ORC_MAXN];
    int n_sph;
    int32_t* sph_body;
    double* sph; /* x y z r in the body frame */
    uint8_t ignore[MAXB * MAXB];
};

struct orc_scene {
    int n_sph, n_box;
    double* sph; /* x y z r */
    double* box; /* lo xyz, hi xyz */
};

/* ------------------------------------------------------------------------ */
/* construction                                                             */

orc_robot* orc_robot_new(int n, const double* a, const double* alpha, const double* d,
                         const double* theta_off, const double* flange16,
                         const double* lo, const double* hi,
                         int n_sph, const int32_t* sph_body, const double* sph_xyzr,
                         const uint8_t* ignore) {
    if (n < 1 || n > ORC_MAXN) return NULL;
    orc_robot* R = (orc_robot*)calloc(1, sizeof(orc_robot));
    R->n = n;
    for (int i = 0; i < n; ++i) {
        R->a[i] = a[i];
        R->alpha[i] = alpha[i];
        R->d[i] = d[i];
        R->off[i] = theta_off ? theta_off[i] : 0.0;
        R->lo[i] = lo[i];
        R->hi[i] = hi[i];
    }
    memcpy(R->flange, flange16, 16 * sizeof(double));
    R->n_sph = n_sph;
    R->sph_body = (int32_t*)malloc((size_t)(n_sph > 0 ? n_sph : 1) * sizeof(int32_t));
    R->sph = (double*)malloc((size_t)(n_sph > 0 ? n_sph : 1) * 4 * sizeof(double));
    if (n_sph > 0) {
        memcpy(R->sph_body, sph_body, (size_t)n_sph * sizeof(int32_t));
        memcpy(R->sph, sph_xyzr, (size_t)n_sph * 4 * sizeof(double));
    }
    int nb = n + 2;
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) {
            int v;
            /* either entry of the matrix marks the pair; default: adjacent bodies are never checked */
            if (ignore) v = ignore[i * nb + j] != 0 || ignore[j * nb + i] != 0;
            else v = abs(i - j) <= 1;
            R->ignore[i * MAXB + j] = (uint8_t)v;
        }
    return R;
}

void orc_robot_free(orc_robot* R) {
    if (!R) return;
    free(R->sph_body);
    free(R->sph);
    free(R);
}

orc_scene* orc_scene_new(int n_sph, const double* sph_xyzr, int n_box, const double* box_lohi) {
    orc_scene* S = (orc_scene*)calloc(1, sizeof(orc_scene));
    S->n_sph = n_sph;
    S->n_box = n_box;
    S->sph = (double*)malloc((size_t)(n_sph > 0 ? n_sph : 1) * 4 * sizeof(double));
    S->box = (double*)malloc((size_t)(n_box > 0 ? n_box : 1) * 6 * sizeof(double));
    if (n_sph > 0) memcpy(S->sph, sph_xyzr, (size_t)n_sph * 4 * sizeof(double));
    if (n_box > 0) memcpy(S->box, box_lohi, (size_t)n_box * 6 * sizeof(double));
    return S;
}

void orc_scene_free(orc_scene* S) {
    if (!S) return;
    free(S->sph);
    free(S->box);
    free(S);
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* random numbers                                                           */

/* Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64-bit
 * multiplications with the round multipliers, the key bumped by the Weyl
 * constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Top 23 bits, centred in their cell: ((x >> 9) + 1/2) * 2^-23, in (0, 1).
 * The value is exact in binary32 as well as binary64. */
double orc_u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Box-Muller, cosine branch: sqrt(-2 ln u0) cos(2 pi u1). */
double orc_normal(uint32_t x0, uint32_t x1) {
    double u0 = orc_u01(x0), u1 = orc_u01(x1);
    return sqrt(-2.0 * log(u0)) * cos(2.0 * M_PI * u1);
}

static void rnd_block(const orc_params* P, uint32_t cand, uint32_t tgt, uint32_t phase,
                      uint32_t iter, uint32_t block, uint32_t out[4]) {
    uint32_t ctr[4] = {cand, tgt, (phase << 24) | (iter & 0xFFFFFFu), block};
    orc_philox4x32_10(ctr, P->key, out);
}

/* j-th uniform of a stream: word j%4 of block j/4 */
static double rnd_uniform(const orc_params* P, uint32_t cand, uint32_t tgt, uint32_t phase,
                          uint32_t iter, int j) {
    uint32_t w[4];
    rnd_block(P, cand, tgt, phase, iter, (uint32_t)(j / 4), w);
    return orc_u01(w[j % 4]);
}

/* j-th standard normal of a stream: words 2(j%2), 2(j%2)+1 of block j/2 */
static double rnd_normal(const orc_params* P, uint32_t cand, uint32_t tgt, uint32_t phase,
                         uint32_t iter, int j) {
    uint32_t w[4];
    rnd_block(P, cand, tgt, phase, iter, (uint32_t)(j / 2), w);
    int h = 2 * (j % 2);
    return orc_normal(w[h], w[h + 1]);
}

/* ------------------------------------------------------------------------ */
/* small linear algebra                                                     */

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void cross3(const double a[3], const double b[3], double o[3]) {
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x;
    o[1] = y;
    o[2] = z;
}

static void m4_eye(double T[16]) {
    memset(T, 0, 16 * sizeof(double));
    T[0] = T[5] = T[10] = T[15] = 1.0;
}

static void m4_mul(const double A[16], const double B[16], double C[16]) {
    double tmp[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[4 * i + k] * B[4 * k + j];
            tmp[4 * i + j] = s;
        }
    memcpy(C, tmp, sizeof tmp);
}

static void m4_rotx(double t, double T[16]) {
    m4_eye(T);
    double c = cos(t), s = sin(t);
    T[5] = c;
    T[6] = -s;
    T[9] = s;
    T[10] = c;
}

static void m4_rotz(double t, double T[16]) {
    m4_eye(T);
    double c = cos(t), s = sin(t);
    T[0] = c;
    T[1] = -s;
    T[4] = s;
    T[5] = c;
}

static void m4_trans(double x, double y, double z, double T[16]) {
    m4_eye(T);
    T[3] = x;
    T[7] = y;
    T[11] = z;
}

static void frame_pos(const double T[16], double p[3]) {
    p[0] = T[3];
    p[1] = T[7];
    p[2] = T[11];
}

static void frame_col(const double T[16], int c, double v[3]) {
    v[0] = T[c];
    v[1] = T[4 + c];
    v[2] = T[8 + c];
}

static void frame_rot(const double T[16], double Rm[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rm[3 * i + j] = T[4 * i + j];
}

static void frame_apply(const double T[16], const double x[3], double y[3]) {
    for (int i = 0; i < 3; ++i) y[i] = T[4 * i] * x[0] + T[4 * i + 1] * x[1] + T[4 * i + 2] * x[2] + T[4 * i + 3];
}

/* Cholesky solve of the SPD system A x = b (A is m x m, row-major, overwritten). */
static int chol_solve(int m, double* A, const double* b, double* x) {
    for (int j = 0; j < m; ++j) {
        double s = A[j * m + j];
        for (int k = 0; k < j; ++k) s -= A[j * m + k] * A[j * m + k];
        if (!(s > 0.0)) return -1;
        double l = sqrt(s);
        A[j * m + j] = l;
        for (int i = j + 1; i < m; ++i) {
            double t = A[i * m + j];
            for (int k = 0; k < j; ++k) t -= A[i * m + k] * A[j * m + k];
            A[i * m + j] = t / l;
        }
    }
    double y[ORC_MAXN];
    for (int i = 0; i < m; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= A[i * m + k] * y[k];
        y[i] = t / A[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < m; ++k) t -= A[k * m + i] * x[k];
        x[i] = t / A[i * m + i];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* quaternions                                                              */

static void q_mul(const double a[4], const double b[4], double o[4]) {
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = w;
    o[1] = x;
    o[2] = y;
    o[3] = z;
}

static void q_normalize(const double a[4], double o[4]) {
    double s = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
    for (int i = 0; i < 4; ++i) o[i] = a[i] / s;
}

/* Unit quaternion of a rotation matrix (Shepperd's method: the largest of
 * w, x, y, z is taken from the diagonal, the others from off-diagonal sums),
 * returned with w >= 0. */
void orc_quat_from_rot(const double m[9], double q[4]) {
    double tr = m[0] + m[4] + m[8];
    double w, x, y, z;
    if (tr >= m[0] && tr >= m[4] && tr >= m[8]) {
        double s = 2.0 * sqrt(1.0 + tr);
        w = 0.25 * s;
        x = (m[7] - m[5]) / s;
        y = (m[2] - m[6]) / s;
        z = (m[3] - m[1]) / s;
    } else if (m[0] >= m[4] && m[0] >= m[8]) {
        double s = 2.0 * sqrt(1.0 + m[0] - m[4] - m[8]);
        w = (m[7] - m[5]) / s;
        x = 0.25 * s;
        y = (m[1] + m[3]) / s;
        z = (m[2] + m[6]) / s;
    } else if (m[4] >= m[8]) {
        double s = 2.0 * sqrt(1.0 + m[4] - m[0] - m[8]);
        w = (m[2] - m[6]) / s;
        x = (m[1] + m[3]) / s;
        y = 0.25 * s;
        z = (m[5] + m[7]) / s;
    } else {
        double s = 2.0 * sqrt(1.0 + m[8] - m[0] - m[4]);
        w = (m[3] - m[1]) / s;
        x = (m[2] + m[6]) / s;
        y = (m[5] + m[7]) / s;
        z = 0.25 * s;
    }
    double sg = (w < 0.0) ? -1.0 : 1.0;
    q[0] = sg * w;
    q[1] = sg * x;
    q[2] = sg * y;
    q[3] = sg * z;
}

/* Error quaternion q_err = q_t (x) q_e^-1 = [w, v], sign fixed so w >= 0. */
static void quat_error(const double qt[4], const double qe[4], double qerr[4]) {
    double qi[4] = {qe[0], -qe[1], -qe[2], -qe[3]};
    q_mul(qt, qi, qerr);
    if (qerr[0] < 0.0)
        for (int i = 0; i < 4; ++i) qerr[i] = -qerr[i];
}

/* Eq. quat_diff: omega = 2 atan2(|v|, |w|) / |v| * v. */
void orc_omega(const double qt[4], const double qe[4], double w[3]) {
    double qerr[4];
    quat_error(qt, qe, qerr);
    double nv = sqrt(qerr[1] * qerr[1] + qerr[2] * qerr[2] + qerr[3] * qerr[3]);
    double f = (nv > 1e-15) ? 2.0 * atan2(nv, fabs(qerr[0])) / nv : 2.0 / qerr[0];
    w[0] = f * qerr[1];
    w[1] = f * qerr[2];
    w[2] = f * qerr[3];
}

/* ------------------------------------------------------------------------ */
/* kinematics                                                               */

/* Eq. fk for a modified-DH (Craig) serial revolute chain: joint i contributes
 * Rx(alpha_i) Tx(a_i) Rz(theta_i + off_i) Tz(d_i); the flange transform
 * follows joint n.  frames[0] is the base, frames[i] = T_{0,i}. */
void orc_fk_frames(const orc_robot* R, const double* th, double* F) {
    m4_eye(F);
    for (int i = 0; i < R->n; ++i) {
        double A[16], B[16], Cz[16], D[16], L[16];
        m4_rotx(R->alpha[i], A);
        m4_trans(R->a[i], 0.0, 0.0, B);
        m4_rotz(th[i] + R->off[i], Cz);
        m4_trans(0.0, 0.0, R->d[i], D);
        m4_mul(A, B, L);
        m4_mul(L, Cz, L);
        m4_mul(L, D, L);
        m4_mul(F + 16 * i, L, F + 16 * (i + 1));
    }
    m4_mul(F + 16 * R->n, R->flange, F + 16 * (R->n + 1));
}

void orc_pose(const orc_robot* R, const double* th, double pq[7]) {
    double F[MAXB * 16], Rm[9];
    orc_fk_frames(R, th, F);
    const double* T = F + 16 * (R->n + 1);
    frame_pos(T, pq);
    frame_rot(T, Rm);
    orc_quat_from_rot(Rm, pq + 3);
}

/* Eq. task_residual: r = [P_t - P_ee; omega]. */
void orc_residual(const orc_robot* R, const double* th, const double tgt[7], double e[6]) {
    double pq[7], qt[4];
    orc_pose(R, th, pq);
    for (int i = 0; i < 3; ++i) e[i] = tgt[i] - pq[i];
    q_normalize(tgt + 3, qt);
    orc_omega(qt, pq + 3, e + 3);
}

static void pos_ori_err(const orc_robot* R, const double* th, const double tgt[7], double* ep, double* eo) {
    double e[6];
    orc_residual(R, th, tgt, e);
    *ep = norm3(e);
    *eo = norm3(e + 3);
}

/* Eq. jacobian: column i = [z_i x (P_ee - P_i); z_i] with the world-frame
 * axis z_i and a point P_i on it (the origin of frame i). */
void orc_jacobian(const orc_robot* R, const double* th, double* J) {
    int n = R->n;
    double F[MAXB * 16], pee[3];
    orc_fk_frames(R, th, F);
    frame_pos(F + 16 * (n + 1), pee);
    for (int i = 0; i < n; ++i) {
        double z[3], p[3], r[3], c[3];
        frame_col(F + 16 * (i + 1), 2, z);
        frame_pos(F + 16 * (i + 1), p);
        for (int k = 0; k < 3; ++k) r[k] = pee[k] - p[k];
        cross3(z, r, c);
        for (int k = 0; k < 3; ++k) {
            J[k * n + i] = c[k];
            J[(3 + k) * n + i] = z[k];
        }
    }
}

void orc_fk_batch(const orc_robot* R, int64_t C, const double* th, double* pq) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < C; ++c) orc_pose(R, th + c * R->n, pq + 7 * c);
}

/* ------------------------------------------------------------------------ */
/* Alg. 3, seeding: seeds uniform inside the joint limits                  */

static void sample_seed(const orc_robot* R, const orc_params* P, uint32_t t, uint32_t c, double* th) {
    for (int j = 0; j < R->n; ++j) {
        double u = rnd_uniform(P, c, t, PHASE_SEED, 0, j);
        th[j] = R->lo[j] + u * (R->hi[j] - R->lo[j]);
    }
}

void orc_sample_seeds(const orc_robot* R, const orc_params* P, int64_t C, const int32_t* tgt,
                      const int32_t* cand, double* th) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < C; ++c) sample_seed(R, P, (uint32_t)tgt[c], (uint32_t)cand[c], th + c * R->n);
}

/* ------------------------------------------------------------------------ */
/* PO-CCD (Sec. IV, Alg. 3)                                                 */

/* Eq. vec_proj and theta_proj: normalised joint-to-EE and joint-to-target
 * vectors, projected onto the plane normal to the joint axis; the update is
 * the angle between the projections.  Reading: the angle is signed about the
 * axis (the printed arccos gives only its magnitude). */
static double ccd_position_delta(const double pee[3], const double pt[3], const double pj[3],
                                 const double rj[3], double proj_eps) {
    double u[3], v[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = pee[k] - pj[k];
        v[k] = pt[k] - pj[k];
    }
    double nu = norm3(u), nv = norm3(v);
    if (nu < 1e-12 || nv < 1e-12) return 0.0;
    for (int k = 0; k < 3; ++k) {
        u[k] /= nu;
        v[k] /= nv;
    }
    double rr = dot3(rj, rj);
    double su = dot3(u, rj) / rr, sv = dot3(v, rj) / rr;
    double up[3], vp[3];
    for (int k = 0; k < 3; ++k) {
        up[k] = u[k] - su * rj[k];
        vp[k] = v[k] - sv * rj[k];
    }
    double nup = norm3(up), nvp = norm3(vp);
    if (nup < proj_eps || nvp < proj_eps) return 0.0;
    for (int k = 0; k < 3; ++k) {
        up[k] /= nup;
        vp[k] /= nvp;
    }
    double cr[3], rhat[3];
    cross3(up, vp, cr);
    double nr = sqrt(rr);
    for (int k = 0; k < 3; ++k) rhat[k] = rj[k] / nr;
    return atan2(dot3(rhat, cr), dot3(up, vp));
}

/* One iteration k of Alg. 3 for one candidate (theta updated in place).
 * Returns 1 when the coarse tolerance of Alg. 3 holds after the update. */
static double score_of(const orc_params* P, double ep, double eo);
static int ccd_classic_iteration(const orc_robot* R, const orc_params* P, const double tgt[7], double* th,
                                 double* dp);

static int ccd_iteration(const orc_robot* R, const orc_params* P, const double tgt[7], uint32_t t,
                         uint32_t c, int k, double* th, double* dp, double* ep_p, double* eo_p, double* dq,
                         double* ep_q, double* eo_q, int32_t* jp_out, int32_t* jo_out, uint8_t* acc_out,
                         double* th_hat_out, double* mp_out, double* mo_out, double* ma_out) {
    const int n = R->n;
    double F[MAXB * 16], pee[3], Rm[9], qe[4], qt[4], pt[3] = {tgt[0], tgt[1], tgt[2]};
    orc_fk_frames(R, th, F);
    frame_pos(F + 16 * (n + 1), pee);
    frame_rot(F + 16 * (n + 1), Rm);
    orc_quat_from_rot(Rm, qe);
    q_normalize(tgt + 3, qt);
    double ep0, eo0;
    pos_ori_err(R, th, tgt, &ep0, &eo0);

    /* Eq. angle_axis on the error quaternion */
    double qerr[4];
    quat_error(qt, qe, qerr);
    double phi = 2.0 * acos(clampd(qerr[0], -1.0, 1.0));
    double sh = sin(phi / 2.0);
    double ahat[3] = {0.0, 0.0, 0.0};
    if (sh > 1e-12)
        for (int i = 0; i < 3; ++i) ahat[i] = qerr[1 + i] / sh;
    double delta_k = P->cd_delta0 * pow(P->cd_rho, (double)k);

    /* Alg. 3: per joint, a position update and an orientation update, and the
     * task residual r (position and orientation error) after each of them */
    double Dp[ORC_MAXN], Pp[ORC_MAXN], Op[ORC_MAXN], Dq[ORC_MAXN], Pq[ORC_MAXN], Oq[ORC_MAXN], trial[ORC_MAXN];
    for (int j = 0; j < n; ++j) {
        double pj[3], rj[3];
        frame_pos(F + 16 * (j + 1), pj);
        frame_col(F + 16 * (j + 1), 2, rj);

        /* position update (Eq. vec_proj, theta_proj), kept inside the limits */
        double dpos = ccd_position_delta(pee, pt, pj, rj, P->proj_eps);
        Dp[j] = clampd(th[j] + dpos, R->lo[j], R->hi[j]) - th[j];
        memcpy(trial, th, (size_t)n * sizeof(double));
        trial[j] += Dp[j];
        pos_ori_err(R, trial, tgt, &Pp[j], &Op[j]);

        /* orientation update (Eq. ori_update), sgn(0) = 0 */
        double s = dot3(ahat, rj);
        double sg = (s > 0.0) ? 1.0 : ((s < 0.0) ? -1.0 : 0.0);
        double dori = delta_k * sg * phi;
        Dq[j] = clampd(th[j] + dori, R->lo[j], R->hi[j]) - th[j];
        memcpy(trial, th, (size_t)n * sizeof(double));
        trial[j] += Dq[j];
        pos_ori_err(R, trial, tgt, &Pq[j], &Oq[j]);
    }

    /* Alg. 3, greedy choice of the best position update and the best
     * orientation update.  Reading: each trial is judged by the task residual it
     * leaves (Alg. 3 computes the full r of each trial), through its scalar form, the score
     * (|e_p|/eps_pos)^2 + (|omega|/eps_ori)^2 used for every ranking.  Ties: joints
     * are scanned from the base and a later joint replaces the current choice
     * only when its score is lower by more than the relative tolerance cd_tie,
     * so updates equal up to rounding (joints sharing axis and origin) go to the
     * lower joint index.  The margins record, relative to the score, how close
     * each of these comparisons came to flipping. */
    int jp = 0, jo = 0;
    double gp = INFINITY, go = INFINITY;
    double sp_best = score_of(P, Pp[0], Op[0]), so_best = score_of(P, Pq[0], Oq[0]);
    for (int j = 1; j < n; ++j) {
        double sp = score_of(P, Pp[j], Op[j]), so = score_of(P, Pq[j], Oq[j]);
        double mp = sp - sp_best * (1.0 - P->cd_tie), mo = so - so_best * (1.0 - P->cd_tie);
        gp = fmin(gp, fabs(mp) / fmax(sp_best, 1e-300));
        go = fmin(go, fabs(mo) / fmax(so_best, 1e-300));
        if (mp < 0.0) {
            jp = j;
            sp_best = sp;
        }
        if (mo < 0.0) {
            jo = j;
            so_best = so;
        }
    }

    /* Alg. 3: apply both; on the same joint keep the larger step */
    double th_hat[ORC_MAXN];
    memcpy(th_hat, th, (size_t)n * sizeof(double));
    if (jp != jo) {
        th_hat[jp] += Dp[jp];
        th_hat[jo] += Dq[jo];
    } else {
        gp = fmin(gp, fabs(fabs(Dp[jp]) - fabs(Dq[jo])));
        if (fabs(Dp[jp]) >= fabs(Dq[jo])) th_hat[jp] += Dp[jp];
        else th_hat[jo] += Dq[jo];
    }

    /* Alg. 3 acceptance, read as: accept when the position error or the
     * orientation error drops by more than its threshold gamma */
    double ep1, eo1;
    pos_ori_err(R, th_hat, tgt, &ep1, &eo1);
    double mA = (ep0 - ep1) - P->cd_gamma_pos, mB = (eo0 - eo1) - P->cd_gamma_ori;
    int acc = (mA > 0.0) || (mB > 0.0);

    if (dp) memcpy(dp, Dp, (size_t)n * sizeof(double));
    if (ep_p) memcpy(ep_p, Pp, (size_t)n * sizeof(double));
    if (eo_p) memcpy(eo_p, Op, (size_t)n * sizeof(double));
    if (dq) memcpy(dq, Dq, (size_t)n * sizeof(double));
    if (ep_q) memcpy(ep_q, Pq, (size_t)n * sizeof(double));
    if (eo_q) memcpy(eo_q, Oq, (size_t)n * sizeof(double));
    if (jp_out) *jp_out = jp;
    if (jo_out) *jo_out = jo;
    if (acc_out) *acc_out = (uint8_t)acc;
    if (th_hat_out) memcpy(th_hat_out, th_hat, (size_t)n * sizeof(double));
    if (mp_out) *mp_out = gp;
    if (mo_out) *mo_out = go;
    if (ma_out) *ma_out = fabs(fmax(mA, mB));

    if (acc) {
        memcpy(th, th_hat, (size_t)n * sizeof(double));
    } else {
        /* Alg. 3 rejection: random perturbation N(0, sigma^2 I), kept in the limits */
        for (int j = 0; j < n; ++j)
            th[j] = clampd(th[j] + P->cd_sigma * rnd_normal(P, c, t, PHASE_CD, (uint32_t)k, j),
                           R->lo[j], R->hi[j]);
    }

    /* Alg. 3 break: coarse tolerance on the squared norms */
    double ep2, eo2;
    pos_ori_err(R, th, tgt, &ep2, &eo2);
    return (ep2 * ep2 < P->cd_eps_pos2) && (eo2 * eo2 < P->cd_eps_ori2);
}

void orc_ccd_iteration_batch(const orc_robot* R, const orc_params* P, const double* targets,
                             int64_t C, const int32_t* tgt, const int32_t* cand, int k,
                             const double* th_in, double* th_out,
                             double* dp, double* ep_p, double* eo_p, double* dq, double* ep_q, double* eo_q,
                             int32_t* jp, int32_t* jo, uint8_t* accepted, double* th_hat,
                             double* margin_p, double* margin_o, double* margin_acc,
                             uint8_t* converged) {
    const int n = R->n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < C; ++c) {
        double th[ORC_MAXN];
        memcpy(th, th_in + c * n, (size_t)n * sizeof(double));
        if (P->cd_variant == 1) {
            const int cv = ccd_classic_iteration(R, P, targets + 7 * (int64_t)tgt[c], th, dp ? dp + c * n : NULL);
            memcpy(th_out + c * n, th, (size_t)n * sizeof(double));
            if (converged) converged[c] = (uint8_t)cv;
            continue;
        }
        int conv = ccd_iteration(R, P, targets + 7 * (int64_t)tgt[c], (uint32_t)tgt[c], (uint32_t)cand[c], k, th,
                                 dp ? dp + c * n : NULL, ep_p ? ep_p + c * n : NULL, eo_p ? eo_p + c * n : NULL,
                                 dq ? dq + c * n : NULL, ep_q ? ep_q + c * n : NULL, eo_q ? eo_q + c * n : NULL,
                                 jp ? jp + c : NULL, jo ? jo + c : NULL,
                                 accepted ? accepted + c : NULL, th_hat ? th_hat + c * n : NULL,
                                 margin_p ? margin_p + c : NULL, margin_o ? margin_o + c : NULL,
                                 margin_acc ? margin_acc + c : NULL);
        memcpy(th_out + c * n, th, (size_t)n * sizeof(double));
        if (converged) converged[c] = (uint8_t)conv;
    }
}

static double score_of(const orc_params* P, double ep, double eo) {
    double a = ep / P->eps_pos, b = eo / P->eps_ori;
    return a * a + b * b;
}

/* Alg. 1, one iteration: joints from the last to the first, each rotated at
 * once by its Eq. theta_proj step (kept inside the limits, reading c18), with a
 * fresh kinematics pass before every joint; then the break test on the squared
 * position error.  dp (may be NULL) receives the step applied to each joint.
 * Returns 1 when the break test holds. */
static int ccd_classic_iteration(const orc_robot* R, const orc_params* P, const double tgt[7], double* th,
                                 double* dp) {
    const int n = R->n;
    const double pt[3] = {tgt[0], tgt[1], tgt[2]};
    double F[MAXB * 16], pee[3], pj[3], rj[3];
    for (int j = n - 1; j >= 0; --j) {
        orc_fk_frames(R, th, F);
        frame_pos(F + 16 * (n + 1), pee);
        frame_pos(F + 16 * (j + 1), pj);
        frame_col(F + 16 * (j + 1), 2, rj);
        const double d = clampd(th[j] + ccd_position_delta(pee, pt, pj, rj, P->proj_eps), R->lo[j], R->hi[j]) - th[j];
        th[j] += d;
        if (dp) dp[j] = d;
    }
    double ep, eo;
    pos_ori_err(R, th, tgt, &ep, &eo);
    return ep * ep < P->cd_eps_pos2;
}

/* cd_variant 2, reading of Sec. IV ("once a seed satisfies the thresholds the
 * parallel loop is broken and all samples are returned"): the seeds of a
 * target (the candidates with that target row, in input order) take
 * iterations together; after the first iteration that leaves any of them
 * inside the coarse tolerance, every seed of the target stops. */
static void po_ccd_target_break(const orc_robot* R, const orc_params* P, const double* targets, int64_t C,
                                const int32_t* tgt, const int32_t* cand, double* th_out, double* score,
                                double* perr, double* oerr, int32_t* iters) {
    const int n = R->n;
    int32_t tmax = -1;
    for (int64_t c = 0; c < C; ++c)
        if (tgt[c] > tmax) tmax = tgt[c];
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t t = 0; t <= tmax; ++t) {
        const double* T = targets + 7 * (int64_t)t;
        for (int64_t c = 0; c < C; ++c)
            if (tgt[c] == t) sample_seed(R, P, (uint32_t)t, (uint32_t)cand[c], th_out + c * n);
        int stop = P->cd_max_iters;
        for (int k = 0; k < P->cd_max_iters; ++k) {
            int any = 0;
            for (int64_t c = 0; c < C; ++c)
                if (tgt[c] == t)
                    any |= ccd_iteration(R, P, T, (uint32_t)t, (uint32_t)cand[c], k, th_out + c * n, NULL, NULL, NULL,
                                         NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
            if (any) {
                stop = k + 1;
                break;
            }
        }
        for (int64_t c = 0; c < C; ++c) {
            if (tgt[c] != t) continue;
            double ep, eo;
            pos_ori_err(R, th_out + c * n, T, &ep, &eo);
            if (score) score[c] = score_of(P, ep, eo);
            if (perr) perr[c] = ep;
            if (oerr) oerr[c] = eo;
            if (iters) iters[c] = stop;
        }
    }
}

/* Alg. 3 for one candidate: seed, then at most max_iters iterations. */
void orc_po_ccd_batch(const orc_robot* R, const orc_params* P, const double* targets,
                      int64_t C, const int32_t* tgt, const int32_t* cand,
                      double* th_out, double* score, double* perr, double* oerr, int32_t* iters) {
    const int n = R->n;
    if (P->cd_variant == 2) {
        po_ccd_target_break(R, P, targets, C, tgt, cand, th_out, score, perr, oerr, iters);
        return;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < C; ++c) {
        const double* T = targets + 7 * (int64_t)tgt[c];
        double th[ORC_MAXN];
        sample_seed(R, P, (uint32_t)tgt[c], (uint32_t)cand[c], th);
        int it = P->cd_max_iters;
        for (int k = 0; k < P->cd_max_iters; ++k) {
            const int cv = P->cd_variant == 1
                               ? ccd_classic_iteration(R, P, T, th, NULL)
                               : ccd_iteration(R, P, T, (uint32_t)tgt[c], (uint32_t)cand[c], k, th, NULL, NULL, NULL,
                                               NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
            if (cv) {
                it = k + 1;
                break;
            }
        }
        double ep, eo;
        pos_ori_err(R, th, T, &ep, &eo);
        memcpy(th_out + c * n, th, (size_t)n * sizeof(double));
        if (score) score[c] = score_of(P, ep, eo);
        if (perr) perr[c] = ep;
        if (oerr) oerr[c] = eo;
        if (iters) iters[c] = it;
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: top-K by residual score and perturbed duplication               */

/* K = max(1, floor(M / ratio)) seeds kept, each copied floor(M / K) times. */
int64_t orc_dup_layout(int64_t M, int32_t ratio, int64_t* K, int64_t* copies) {
    if (M <= 0) {
        if (K) *K = 0;
        if (copies) *copies = 0;
        return 0;
    }
    int64_t k = M / ratio;
    if (k < 1) k = 1;
    int64_t cp = M / k;
    if (K) *K = k;
    if (copies) *copies = cp;
    return k * cp;
}

void orc_topk_dup(const orc_robot* R, const orc_params* P, int64_t T, const int64_t* m_off,
                  const double* score_M, const double* th_M, const int64_t* b_off,
                  double* th_B, int32_t* src_B) {
    const int n = R->n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < T; ++t) {
        int64_t M = m_off[t + 1] - m_off[t], K, copies;
        orc_dup_layout(M, P->dup_ratio, &K, &copies);
        uint8_t* taken = (uint8_t*)calloc((size_t)(M > 0 ? M : 1), 1);
        int64_t* sel = (int64_t*)malloc((size_t)(K > 0 ? K : 1) * sizeof(int64_t));
        /* K successive argmins, each removed from the set */
        for (int64_t i = 0; i < K; ++i) {
            int64_t best = -1;
            for (int64_t m = 0; m < M; ++m) {
                if (taken[m]) continue;
                if (best < 0 || score_M[m_off[t] + m] < score_M[m_off[t] + best]) best = m;
            }
            sel[i] = best;
            taken[best] = 1;
        }
        /* floor(B/K) perturbed copies of the K kept seeds */
        for (int64_t r = 0; r < copies; ++r)
            for (int64_t i = 0; i < K; ++i) {
                int64_t b = r * K + i;
                const double* src = th_M + (m_off[t] + sel[i]) * n;
                double* dst = th_B + (b_off[t] + b) * n;
                for (int j = 0; j < n; ++j)
                    dst[j] = clampd(src[j] + P->dup_sigma * rnd_normal(P, (uint32_t)b, (uint32_t)t, PHASE_DUP, 0, j),
                                    R->lo[j], R->hi[j]);
                if (src_B) src_B[b_off[t] + b] = (int32_t)sel[i];
            }
        free(taken);
        free(sel);
    }
}

/* ------------------------------------------------------------------------ */
/* PJ-IK (Sec. V-B, Alg. 4)                                                 */

/* Eq. normal-eqs, read as ((WJ)^T (WJ) + lambda D) step = (WJ)^T W r with
 * D = diag((WJ)^T (WJ)) (+1e-9) and r = target - current (the printed minus
 * sign belongs to the opposite residual convention), followed by the
 * elementwise trust region of Alg. 4.  Jw = W J is 6 x n, b = W r. */
void orc_lm_step(int n, const double* Jw, const double* b, double lambda, double R, double* step) {
    double A[ORC_MAXN * ORC_MAXN], g[ORC_MAXN];
    for (int i = 0; i < n; ++i) {
        g[i] = 0.0;
        for (int r = 0; r < 6; ++r) g[i] += Jw[r * n + i] * b[r];
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int r = 0; r < 6; ++r) s += Jw[r * n + i] * Jw[r * n + j];
            A[i * n + j] = s;
        }
    }
    for (int i = 0; i < n; ++i) A[i * n + i] += lambda * (A[i * n + i] + 1e-9);
    if (chol_solve(n, A, g, step) != 0)
        for (int i = 0; i < n; ++i) step[i] = 0.0;
    for (int i = 0; i < n; ++i) step[i] = clampd(step[i], -R, R);
}

/* Eq. dogleg.  The Gauss-Newton step is taken in its minimum-norm form
 * (WJ)^T ((WJ)(WJ)^T + mu I)^-1 W r, since J^T J is singular when n > 6; the
 * gradient step is the Cauchy point along g = (WJ)^T W r; tau is the smallest
 * value in [0, 1] that puts tau*GD + (1-tau)*GN inside the ball of radius R,
 * and when even tau = 1 lies outside, the gradient step is scaled to the
 * boundary. */
void orc_dogleg_step(int n, const double* Jw, const double* b, double R, double gn_reg, double* step) {
    double G[36], y[6], g[ORC_MAXN], dgn[ORC_MAXN], dgd[ORC_MAXN];
    for (int r = 0; r < 6; ++r)
        for (int q = 0; q < 6; ++q) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += Jw[r * n + i] * Jw[q * n + i];
            G[r * 6 + q] = s + (r == q ? gn_reg : 0.0);
        }
    if (chol_solve(6, G, b, y) != 0)
        for (int r = 0; r < 6; ++r) y[r] = 0.0;
    double Jg[6] = {0}, gg = 0.0;
    for (int i = 0; i < n; ++i) {
        dgn[i] = 0.0;
        g[i] = 0.0;
        for (int r = 0; r < 6; ++r) {
            dgn[i] += Jw[r * n + i] * y[r];
            g[i] += Jw[r * n + i] * b[r];
        }
        gg += g[i] * g[i];
    }
    for (int r = 0; r < 6; ++r)
        for (int i = 0; i < n; ++i) Jg[r] += Jw[r * n + i] * g[i];
    double jgjg = Jg[0] * Jg[0] + Jg[1] * Jg[1] + Jg[2] * Jg[2] + Jg[3] * Jg[3] + Jg[4] * Jg[4] + Jg[5] * Jg[5];
    double ac = (jgjg > 0.0) ? gg / jgjg : 0.0;
    double ngn2 = 0.0, ngd2 = 0.0;
    for (int i = 0; i < n; ++i) {
        dgd[i] = ac * g[i];
        ngn2 += dgn[i] * dgn[i];
        ngd2 += dgd[i] * dgd[i];
    }
    if (ngn2 <= R * R) {
        for (int i = 0; i < n; ++i) step[i] = dgn[i]; /* tau = 0 */
    } else if (ngd2 >= R * R) {
        double f = (ngd2 > 0.0) ? R / sqrt(ngd2) : 0.0;
        for (int i = 0; i < n; ++i) step[i] = f * dgd[i];
    } else {
        double qa = 0.0, qb = 0.0, qc = ngn2 - R * R;
        for (int i = 0; i < n; ++i) {
            double di = dgd[i] - dgn[i];
            qa += di * di;
            qb += 2.0 * dgn[i] * di;
        }
        double tau = (-qb - sqrt(qb * qb - 4.0 * qa * qc)) / (2.0 * qa);
        for (int i = 0; i < n; ++i) step[i] = dgn[i] + tau * (dgd[i] - dgn[i]);
    }
}

/* Eq. single-coord.  The paper moves the one joint with the largest gradient
 * component; read here as i* = argmax_i |g_i| of g = (WJ)^T W r, the gradient
 * of -1/2 |W r|^2 (ties to the lower joint), and on that joint the
 * one-dimensional Gauss-Newton step g_i* / |(WJ)_{:,i*}|^2 -- the minimiser of
 * the linearised cost 1/2 |W r - x (WJ)_{:,i*}|^2 -- clamped to the trust
 * region.  step receives the n-vector (zero except at i*). */
void orc_single_coord_step(int n, const double* Jw, const double* b, double R, int* i_star, double* step) {
    double g[ORC_MAXN];
    for (int i = 0; i < n; ++i) {
        g[i] = 0.0;
        for (int r = 0; r < 6; ++r) g[i] += Jw[r * n + i] * b[r];
    }
    int is = 0;
    for (int i = 1; i < n; ++i)
        if (fabs(g[i]) > fabs(g[is])) is = i;
    double cn = 0.0;
    for (int r = 0; r < 6; ++r) cn += Jw[r * n + is] * Jw[r * n + is];
    for (int i = 0; i < n; ++i) step[i] = 0.0;
    step[is] = (cn > 0.0) ? clampd(g[is] / cn, -R, R) : 0.0;
    *i_star = is;
}

typedef struct {
    const orc_robot* R;
    const orc_params* P;
    const double* tgt;
    double W[6];
} lm_ctx;

/* weighted cost 1/2 |W r(theta)|^2 with W held fixed for the iteration */
static double lm_cost(const lm_ctx* L, const double* th) {
    double e[6], s = 0.0;
    orc_residual(L->R, th, L->tgt, e);
    for (int r = 0; r < 6; ++r) s += (L->W[r] * e[r]) * (L->W[r] * e[r]);
    return 0.5 * s;
}

static void clamp_limits(const orc_robot* R, double* th) {
    for (int j = 0; j < R->n; ++j) th[j] = clampd(th[j], R->lo[j], R->hi[j]);
}

/* Eq. line-search: the first alpha of 1, 1/beta, ..., 1/beta^A whose step
 * lowers the cost (reading: "first iterate that reduces" the residual);
 * returns 0 when none does. */
static double line_search(const lm_ctx* L, const double* th, const double* step, double cost0,
                          double* th_new, double* margin) {
    const int n = L->R->n;
    for (int i = 0; i <= L->P->lm_A; ++i) {
        double alpha = 1.0 / pow(L->P->lm_beta, (double)i);
        double trial[ORC_MAXN];
        for (int j = 0; j < n; ++j) trial[j] = th[j] + alpha * step[j];
        clamp_limits(L->R, trial);
        double c = lm_cost(L, trial);
        double rel = fabs(c - cost0) / fmax(cost0, 1e-300);
        if (rel < *margin) *margin = rel;
        if (c < cost0) {
            memcpy(th_new, trial, (size_t)n * sizeof(double));
            return alpha;
        }
    }
    return 0.0;
}

/* One iteration k of Alg. 4 (theta updated in place).  Returns 1 when the
 * tolerance of Alg. 4 holds after the update. */
static int lm_iteration(const orc_robot* R, const orc_params* P, const double tgt[7], uint32_t t,
                        uint32_t c, int k, double* th, double* J_out, double* W_out, double* dlm_out,
                        int32_t* branch_out, double* alpha_out, double* margin_out, double* ddog_out,
                        int32_t* scj_out, double* scs_out) {
    const int n = R->n;
    lm_ctx L = {R, P, tgt, {0}};
    double e[6], J[6 * ORC_MAXN];
    orc_residual(R, th, tgt, e);
    orc_jacobian(R, th, J);

    /* W: diagonal, each row of J normalised; orientation rows additionally
     * scaled by eps_pos / eps_ori (reading of "adaptively scales") */
    for (int r = 0; r < 6; ++r) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += J[r * n + i] * J[r * n + i];
        double wc = (r < 3) ? 1.0 : P->eps_pos / P->eps_ori;
        L.W[r] = wc / fmax(sqrt(s), 1e-6);
    }
    double Jw[6 * ORC_MAXN], b[6];
    for (int r = 0; r < 6; ++r) {
        b[r] = L.W[r] * e[r];
        for (int i = 0; i < n; ++i) Jw[r * n + i] = L.W[r] * J[r * n + i];
    }
    double cost0 = 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3] + b[4] * b[4] + b[5] * b[5]);

    /* Eq. normal-eqs (see orc_lm_step), then the trust region of Alg. 4 */
    double step[ORC_MAXN];
    orc_lm_step(n, Jw, b, P->lm_lambda, P->lm_trust_R, step);

    /* the fallback steps of Alg. 4, taken below in its order when the LM step fails
     * (computed here in any case so that a trace can show them) */
    double dd[ORC_MAXN], sstep[ORC_MAXN];
    int is = 0;
    orc_dogleg_step(n, Jw, b, P->lm_trust_R, P->lm_gn_reg, dd);
    orc_single_coord_step(n, Jw, b, P->lm_trust_R, &is, sstep);

    double margin = INFINITY, th_new[ORC_MAXN];
    int branch;
    double alpha = line_search(&L, th, step, cost0, th_new, &margin);
    if (alpha > 0.0) {
        memcpy(th, th_new, (size_t)n * sizeof(double));
        branch = BR_LM;
    } else {
        double trial[ORC_MAXN];
        for (int i = 0; i < n; ++i) trial[i] = th[i] + dd[i];
        clamp_limits(R, trial);
        double cd = lm_cost(&L, trial);
        double rel = fabs(cd - cost0) / fmax(cost0, 1e-300);
        if (rel < margin) margin = rel;
        if (cd < cost0) {
            memcpy(th, trial, (size_t)n * sizeof(double));
            branch = BR_DOGLEG;
        } else {
            /* Eq. single-coord (step from orc_single_coord_step), then the same line search */
            double a2 = line_search(&L, th, sstep, cost0, th_new, &margin);
            if (a2 > 0.0) {
                memcpy(th, th_new, (size_t)n * sizeof(double));
                branch = BR_SINGLE;
                alpha = a2;
            } else {
                /* Alg. 4: random perturbation when every update fails */
                for (int j = 0; j < n; ++j)
                    th[j] = clampd(th[j] + P->lm_sigma * rnd_normal(P, c, t, PHASE_LM, (uint32_t)k, j),
                                   R->lo[j], R->hi[j]);
                branch = BR_PERTURB;
            }
        }
    }
    if (J_out) memcpy(J_out, J, (size_t)(6 * n) * sizeof(double));
    if (W_out) memcpy(W_out, L.W, 6 * sizeof(double));
    if (dlm_out) memcpy(dlm_out, step, (size_t)n * sizeof(double));
    if (branch_out) *branch_out = branch;
    if (alpha_out) *alpha_out = alpha;
    if (margin_out) *margin_out = margin;
    if (ddog_out) memcpy(ddog_out, dd, (size_t)n * sizeof(double));
    if (scj_out) *scj_out = is;
    if (scs_out) *scs_out = sstep[is];

    /* Alg. 4 break */
    double ep, eo;
    pos_ori_err(R, th, tgt, &ep, &eo);
    return (ep < P->eps_pos) && (eo < P->eps_ori);
}

void orc_lm_iteration_batch(const orc_robot* R, const orc_params* P, const double* targets,
                            int64_t C, const int32_t* tgt, const int32_t* cand, int k,
                            const double* th_in, double* th_out,
                            double* J, double* W, double* d_lm, int32_t* branch,
                            double* alpha, double* ls_margin, uint8_t* converged,
                            double* d_dog, int32_t* sc_joint, double* sc_step) {
    const int n = R->n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < C; ++c) {
        double th[ORC_MAXN];
        memcpy(th, th_in + c * n, (size_t)n * sizeof(double));
        int conv = lm_iteration(R, P, targets + 7 * (int64_t)tgt[c], (uint32_t)tgt[c], (uint32_t)cand[c], k, th,
                                J ? J + c * 6 * n : NULL, W ? W + c * 6 : NULL,
                                d_lm ? d_lm + c * n : NULL, branch ? branch + c : NULL,
                                alpha ? alpha + c : NULL, ls_margin ? ls_margin + c : NULL,
                                d_dog ? d_dog + c * n : NULL, sc_joint ? sc_joint + c : NULL,
                                sc_step ? sc_step + c : NULL);
        memcpy(th_out + c * n, th, (size_t)n * sizeof(double));
        if (converged) converged[c] = (uint8_t)conv;
    }
}

/* Alg. 4 for one candidate: at most lm_max_iters iterations. */
void orc_pjik_batch(const orc_robot* R, const orc_params* P, const double* targets,
                    int64_t C, const int32_t* tgt, const int32_t* cand, double* theta,
                    double* score, double* perr, double* oerr, int32_t* iters) {
    const int n = R->n;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < C; ++c) {
        const double* T = targets + 7 * (int64_t)tgt[c];
        double* th = theta + c * n;
        int it = P->lm_max_iters;
        for (int k = 0; k < P->lm_max_iters; ++k) {
            if (lm_iteration(R, P, T, (uint32_t)tgt[c], (uint32_t)cand[c], k, th, NULL, NULL, NULL, NULL,
                             NULL, NULL, NULL, NULL, NULL)) {
                it = k + 1;
                break;
            }
        }
        double ep, eo;
        pos_ori_err(R, th, T, &ep, &eo);
        if (score) score[c] = score_of(P, ep, eo);
        if (perr) perr[c] = ep;
        if (oerr) oerr[c] = eo;
        if (iters) iters[c] = it;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. V-C: collision filter, brute force over every sphere pair            */

/* Overlap iff |c1 - c2|^2 < (r1 + r2)^2 (sphere-sphere) or, for a box, iff
 * the squared distance from the centre to its closest point of the box is
 * below r^2.  The verdict margin is the depth of the deepest overlap when the
 * configuration collides, else the smallest clearance. */
static int collide_one(const orc_robot* R, const orc_scene* S, const double* th, double* vmargin) {
    const int n = R->n, ns = R->n_sph;
    double F[MAXB * 16];
    orc_fk_frames(R, th, F);
    double* W = (double*)malloc((size_t)(ns > 0 ? ns : 1) * 4 * sizeof(double));
    for (int s = 0; s < ns; ++s) {
        frame_apply(F + 16 * R->sph_body[s], R->sph + 4 * s, W + 4 * s);
        W[4 * s + 3] = R->sph[4 * s + 3];
    }
    int hit = 0;
    double deepest = 0.0, clearest = INFINITY;
#define ACCOUNT(d2, rr)                                          \
    do {                                                         \
        double cl_ = sqrt(d2) - (rr);                            \
        if ((d2) < (rr) * (rr)) {                                \
            hit = 1;                                             \
            if (-cl_ > deepest) deepest = -cl_;                  \
        } else if (cl_ < clearest) {                             \
            clearest = cl_;                                      \
        }                                                        \
    } while (0)
    for (int i = 0; i < ns; ++i)
        for (int j = i + 1; j < ns; ++j) {
            int bi = R->sph_body[i], bj = R->sph_body[j];
            if (bi == bj || R->ignore[bi * MAXB + bj]) continue;
            double dx = W[4 * i] - W[4 * j], dy = W[4 * i + 1] - W[4 * j + 1], dz = W[4 * i + 2] - W[4 * j + 2];
            ACCOUNT(dx * dx + dy * dy + dz * dz, W[4 * i + 3] + W[4 * j + 3]);
        }
    if (S) {
        for (int i = 0; i < ns; ++i) {
            for (int o = 0; o < S->n_sph; ++o) {
                const double* q = S->sph + 4 * o;
                double dx = W[4 * i] - q[0], dy = W[4 * i + 1] - q[1], dz = W[4 * i + 2] - q[2];
                ACCOUNT(dx * dx + dy * dy + dz * dz, W[4 * i + 3] + q[3]);
            }
            for (int o = 0; o < S->n_box; ++o) {
                const double* bx = S->box + 6 * o;
                double d2 = 0.0;
                for (int k = 0; k < 3; ++k) {
                    double cl = clampd(W[4 * i + k], bx[k], bx[3 + k]);
                    double dk = W[4 * i + k] - cl;
                    d2 += dk * dk;
                }
                ACCOUNT(d2, W[4 * i + 3]);
            }
        }
    }
#undef ACCOUNT
    free(W);
    (void)n;
    if (vmargin) *vmargin = hit ? deepest : clearest;
    return hit;
}

void orc_collide_batch(const orc_robot* R, const orc_scene* S, int64_t C, const double* theta,
                       uint8_t* hit, double* vmargin) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < C; ++c)
        hit[c] = (uint8_t)collide_one(R, S, theta + c * R->n, vmargin ? vmargin + c : NULL);
}

/* ------------------------------------------------------------------------ */
/* Alg. 2, final step: collision-free candidates ranked                      */

/* Alg. 2 returns the best collision-free candidates of each target.  Reading
 * (c20): the candidates inside the request's tolerances (|e_p| <= eps_pos and
 * |omega| <= eps_ori) come before the others, each group by the score of
 * reading c4, ties to the lower candidate index.  Reading (c24, the tracking
 * use of Sec. VI-D): with q_ref ([T][n]) the group inside the tolerances is
 * ordered by squared joint-space distance to q_ref[t] instead of the score.
 * Selection by repeated minimum over the untaken candidates. */
static int rank_before(int conv_a, double key_a, int64_t ia, int conv_b, double key_b, int64_t ib) {
    if (conv_a != conv_b) return conv_a > conv_b;
    if (key_a != key_b) return key_a < key_b;
    return ia < ib;
}

void orc_rank(const orc_robot* R, int64_t T, const int64_t* b_off, const double* th_B,
              const double* score, const double* perr, const double* oerr, const uint8_t* hit,
              double eps_pos, double eps_ori, const double* q_ref,
              int top_k, double* out_q, double* out_err, int32_t* out_count) {
    const int n = R->n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < T; ++t) {
        int64_t B = b_off[t + 1] - b_off[t];
        uint8_t* taken = (uint8_t*)calloc((size_t)(B > 0 ? B : 1), 1);
        int* conv = (int*)malloc((size_t)(B > 0 ? B : 1) * sizeof(int));
        double* key = (double*)malloc((size_t)(B > 0 ? B : 1) * sizeof(double));
        for (int64_t b = 0; b < B; ++b) {
            int64_t g = b_off[t] + b;
            conv[b] = perr[g] <= eps_pos && oerr[g] <= eps_ori;
            key[b] = score[g];
            if (q_ref && conv[b]) {
                double d2 = 0.0;
                for (int j = 0; j < n; ++j) {
                    double dj = th_B[g * n + j] - q_ref[t * n + j];
                    d2 += dj * dj;
                }
                key[b] = d2;
            }
        }
        int cnt = 0;
        for (int r = 0; r < top_k; ++r) {
            int64_t best = -1;
            for (int64_t b = 0; b < B; ++b) {
                int64_t g = b_off[t] + b;
                if (taken[b] || (hit && hit[g])) continue;
                if (best < 0 || rank_before(conv[b], key[b], b, conv[best], key[best], best)) best = b;
            }
            if (best < 0) break;
            taken[best] = 1;
            int64_t g = b_off[t] + best;
            memcpy(out_q + ((t * top_k) + r) * n, th_B + g * n, (size_t)n * sizeof(double));
            out_err[((t * top_k) + r) * 2] = perr[g];
            out_err[((t * top_k) + r) * 2 + 1] = oerr[g];
            ++cnt;
        }
        out_count[t] = cnt;
        free(taken);
        free(conv);
        free(key);
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: the whole method                                                 */

void orc_solve(const orc_robot* R, const orc_scene* S, const orc_params* P, int64_t T,
               const double* targets, const int64_t* samples, const double* q_ref, int top_k,
               double* out_q, double* out_err, int32_t* out_count) {
    const int n = R->n;
    int64_t* m_off = (int64_t*)malloc((size_t)(T + 1) * sizeof(int64_t));
    int64_t* b_off = (int64_t*)malloc((size_t)(T + 1) * sizeof(int64_t));
    m_off[0] = b_off[0] = 0;
    for (int64_t t = 0; t < T; ++t) {
        m_off[t + 1] = m_off[t] + samples[t];
        b_off[t + 1] = b_off[t] + orc_dup_layout(samples[t], P->dup_ratio, NULL, NULL);
    }
    int64_t CM = m_off[T], CB = b_off[T];
    int32_t* tg = (int32_t*)malloc((size_t)(CM > CB ? CM : CB) * sizeof(int32_t) + 4);
    int32_t* cd = (int32_t*)malloc((size_t)(CM > CB ? CM : CB) * sizeof(int32_t) + 4);
    double* thM = (double*)malloc((size_t)CM * n * sizeof(double) + 8);
    double* sM = (double*)malloc((size_t)CM * sizeof(double) + 8);
    double* thB = (double*)malloc((size_t)CB * n * sizeof(double) + 8);
    double* sB = (double*)malloc((size_t)CB * sizeof(double) + 8);
    double* pB = (double*)malloc((size_t)CB * sizeof(double) + 8);
    double* oB = (double*)malloc((size_t)CB * sizeof(double) + 8);
    uint8_t* hB = (uint8_t*)calloc((size_t)CB + 1, 1);

    for (int64_t t = 0; t < T; ++t)
        for (int64_t m = m_off[t]; m < m_off[t + 1]; ++m) {
            tg[m] = (int32_t)t;
            cd[m] = (int32_t)(m - m_off[t]);
        }
    orc_po_ccd_batch(R, P, targets, CM, tg, cd, thM, sM, NULL, NULL, NULL);  /* PO-CCD */
    orc_topk_dup(R, P, T, m_off, sM, thM, b_off, thB, NULL);                   /* top-K, duplication */
    for (int64_t t = 0; t < T; ++t)
        for (int64_t b = b_off[t]; b < b_off[t + 1]; ++b) {
            tg[b] = (int32_t)t;
            cd[b] = (int32_t)(b - b_off[t]);
        }
    orc_pjik_batch(R, P, targets, CB, tg, cd, thB, sB, pB, oB, NULL);         /* PJ-IK */
    if (R->n_sph > 0) orc_collide_batch(R, S, CB, thB, hB, NULL);              /* collision filter */
    orc_rank(R, T, b_off, thB, sB, pB, oB, hB, P->eps_pos, P->eps_ori, q_ref, top_k, out_q, out_err,
             out_count);                                                          /* ranking */

    free(m_off);
    free(b_off);
    free(tg);
    free(cd);
    free(thM);
    free(sM);
    free(thB);
    free(sB);
    free(pB);
    free(oB);
    free(hB);
}

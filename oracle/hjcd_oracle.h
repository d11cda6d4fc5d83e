/*
 * hjcd_oracle.h -- FP64 CPU oracle of batched HJCD-IK (arXiv 2510.07514).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, double-precision
 * statement of what the GPU path computes, used by the test-suite, by the
 * smoke check and by the benchmark's CPU-baseline leg.  The product library
 * never links, loads or calls it, and it shares no code with the product.
 *
 * Layout conventions (all row-major, double):
 *   joint vectors  theta[c*n + j]
 *   poses          pq[7] = px, py, pz, qw, qx, qy, qz   (unit quaternion)
 *   frames         (n+2) 4x4 matrices: body 0 = base (identity),
 *                  body i = T_{0,i} (i = 1..n), body n+1 = T_{0,n} * flange
 *   Jacobian       J[r*n + i], r = 0..5 (position rows, then orientation rows)
 */
#ifndef HJCD_ORACLE_H
#define HJCD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXN 32

typedef struct orc_robot orc_robot;
typedef struct orc_scene orc_scene;

/* Parameter table; the values are the readings of the paper stated in hjcd_oracle.c. */
typedef struct {
    double eps_pos, eps_ori;            /* request tolerances: PJ-IK break and score scale */
    int32_t cd_max_iters;
    double cd_eps_pos2, cd_eps_ori2;    /* PO-CCD coarse break on squared norms (epsilon, nu) */
    double cd_gamma_pos, cd_gamma_ori;  /* improvement thresholds gamma */
    double cd_sigma;                    /* PO-CCD rejection perturbation std (rad) */
    double cd_delta0, cd_rho;           /* delta(k) = delta0 * rho^k */
    double proj_eps;                    /* relative projected length below which Eq. theta_proj gives 0 */
    int32_t dup_ratio;                  /* K = max(1, floor(B / dup_ratio)) */
    double dup_sigma;
    int32_t lm_max_iters;
    double lm_lambda, lm_trust_R, lm_beta;
    int32_t lm_A;
    double lm_sigma, lm_gn_reg;
    double cd_tie;                      /* relative tie tolerance of the greedy joint choice */
    int32_t cd_variant;                 /* 0: PO-CCD (Alg. 3); 1: position-only CCD (Alg. 1);
                                           2: PO-CCD with the target-wide break */
    uint32_t key[2];                    /* Philox key = request seed (lo, hi) */
} orc_params;

orc_robot* orc_robot_new(int n, const double* a, const double* alpha, const double* d,
                         const double* theta_off, const double* flange16,
                         const double* lo, const double* hi,
                         int n_sph, const int32_t* sph_body, const double* sph_xyzr,
                         const uint8_t* ignore /* (n+2)^2 or NULL */);
void orc_robot_free(orc_robot*);
orc_scene* orc_scene_new(int n_sph, const double* sph_xyzr, int n_box, const double* box_lohi);
void orc_scene_free(orc_scene*);

void orc_set_threads(int n);
int orc_get_threads(void);

/* Random numbers: Philox4x32-10 and the maps to (0,1) and N(0,1). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t x);
double orc_normal(uint32_t x0, uint32_t x1);

/* Kinematics and residual (Eq. fk, task_residual, quat_diff, jacobian). */
void orc_fk_frames(const orc_robot* R, const double* theta, double* frames);
void orc_pose(const orc_robot* R, const double* theta, double pq[7]);
void orc_quat_from_rot(const double Rm[9], double q[4]);
void orc_omega(const double qt[4], const double qe[4], double w[3]);
void orc_residual(const orc_robot* R, const double* theta, const double tgt[7], double e[6]);
void orc_jacobian(const orc_robot* R, const double* theta, double* J);

/* Batched stages.  tgt[c] indexes `targets` (7 doubles each); cand[c] is the
 * candidate's index inside its target, which keys its random streams. */
void orc_fk_batch(const orc_robot* R, int64_t C, const double* theta, double* pq);
void orc_sample_seeds(const orc_robot* R, const orc_params* P, int64_t C,
                      const int32_t* tgt, const int32_t* cand, double* theta);
void orc_ccd_iteration_batch(const orc_robot* R, const orc_params* P, const double* targets,
                             int64_t C, const int32_t* tgt, const int32_t* cand, int k,
                             const double* th_in, double* th_out,
                             double* dp, double* ep_p, double* eo_p, double* dq, double* ep_q, double* eo_q,
                             int32_t* jp, int32_t* jo, uint8_t* accepted, double* th_hat,
                             double* margin_p, double* margin_o, double* margin_acc,
                             uint8_t* converged);
void orc_po_ccd_batch(const orc_robot* R, const orc_params* P, const double* targets,
                      int64_t C, const int32_t* tgt, const int32_t* cand,
                      double* th_out, double* score, double* perr, double* oerr, int32_t* iters);
int64_t orc_dup_layout(int64_t M, int32_t ratio, int64_t* K, int64_t* copies);
void orc_topk_dup(const orc_robot* R, const orc_params* P, int64_t T, const int64_t* m_off,
                  const double* score_M, const double* th_M, const int64_t* b_off,
                  double* th_B, int32_t* src_B);
void orc_lm_iteration_batch(const orc_robot* R, const orc_params* P, const double* targets,
                            int64_t C, const int32_t* tgt, const int32_t* cand, int k,
                            const double* th_in, double* th_out,
                            double* J, double* W, double* d_lm, int32_t* branch,
                            double* alpha, double* ls_margin, uint8_t* converged,
                            double* d_dog, int32_t* sc_joint, double* sc_step);
void orc_lm_step(int n, const double* Jw, const double* b, double lambda, double R, double* step);
void orc_dogleg_step(int n, const double* Jw, const double* b, double R, double gn_reg, double* step);
void orc_single_coord_step(int n, const double* Jw, const double* b, double R, int* i_star, double* step);
void orc_pjik_batch(const orc_robot* R, const orc_params* P, const double* targets,
                    int64_t C, const int32_t* tgt, const int32_t* cand, double* theta,
                    double* score, double* perr, double* oerr, int32_t* iters);
void orc_collide_batch(const orc_robot* R, const orc_scene* S, int64_t C, const double* theta,
                       uint8_t* hit, double* min_abs_margin);
void orc_rank(const orc_robot* R, int64_t T, const int64_t* b_off, const double* th_B,
              const double* score, const double* perr, const double* oerr, const uint8_t* hit,
              double eps_pos, double eps_ori, const double* q_ref /* [T][n] or NULL */,
              int top_k, double* out_q, double* out_err, int32_t* out_count);

/* Whole method (Alg. 2) for T targets; samples[t] = M = B seeds of target t. */
void orc_solve(const orc_robot* R, const orc_scene* S, const orc_params* P, int64_t T,
               const double* targets, const int64_t* samples, const double* q_ref /* [T][n] or NULL */,
               int top_k, double* out_q, double* out_err, int32_t* out_count);

#ifdef __cplusplus
}
#endif
#endif

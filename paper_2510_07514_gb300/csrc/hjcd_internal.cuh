// hjcd_internal.cuh -- types and device math shared by the HJCD-IK kernels.
//
// All arithmetic is binary32.  Joint vectors are structure-of-arrays
// (theta[j * ld + c]).  One launch may mix robots and scenes: every target
// row names its robot and scene in the launch's tables, and the kernels copy
// the (small) kinematic tables of the launch's robots into shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "hjcd.h"

namespace hjcd {

constexpr int kMaxDof = HJCD_MAX_DOF;
constexpr int kMaxBodies = HJCD_MAX_DOF + 2;
constexpr int kMaxLaunchRobots = HJCD_MAX_BATCH_ROBOTS;  // robots one launch can mix

// Philox stream phases (third counter word, high byte).
enum : uint32_t { kPhaseSeed = 1, kPhaseCd = 2, kPhaseDup = 3, kPhaseLm = 4 };

// Robot as seen by the kernels: modified-DH table, limits, flange transform
// (736 bytes).  A joint's cos alpha, sin alpha, a and d sit together, so one
// 16-byte load per kinematics step fetches them.
struct __align__(16) RobotParams {
    int32_t n;
    int32_t n_sph;
    int32_t plain;  // 1: every joint offset is 0 and every theta within the limits lies inside (-pi, pi)
    int32_t fl_eye; // 1: the flange rotation is the identity (the flange frame's axes are the last joint's)
    float4 dh[kMaxDof];  // cos alpha, sin alpha, a, d
    float off[kMaxDof];
    float2 lim[kMaxDof];  // joint limits lo, hi
    float fl_r[9];  // flange rotation, row-major
    float fl_p[3];  // flange translation
};
static_assert(sizeof(RobotParams) % 16 == 0, "RobotParams tables are 16-byte aligned in shared memory");

// Collision tables of a robot in device memory: spheres grouped by body
// (float4 x y z r in the body frame) with their bodies, per-body
// [first, count) ranges and bounding spheres, the body pairs checked for
// self-collision.
struct RobotDev {
    const float4* sph;    // [n_sph], grouped by body
    const int32_t* body;  // [n_sph]
    const int2* range;    // [n + 2]: first sphere, count
    const float4* coarse; // [n + 2]: bounding sphere in the body frame (r = 0: no spheres)
    const int2* pairs;    // [n_pairs]
    int32_t n_pairs;
    int32_t n_sph;
};

// Obstacles of a scene in device memory: spheres (float4) followed by boxes
// (two float4: lo.xyz, hi.xyz); 16-byte aligned.  A large scene also carries
// a uniform grid over its sphere centres: the spheres are sorted by cell and
// cell[k] .. cell[k+1] are the spheres whose centre lies in cell k (cells
// numbered x fastest); a query for a ball of radius R searches the cells
// within R + reach of its centre.
struct SceneDev {
    const float4* obj;
    int32_t n_sph, n_box;
    const int32_t* cell;  // [dim.x * dim.y * dim.z + 1], or null: no grid
    float lo[3];          // grid origin
    float inv_h;          // 1 / cell edge
    int32_t dim[3];       // cells per axis
    float reach;          // largest obstacle radius, plus a margin beyond binary32 rounding
};

// The robots of one launch and the maxima the kernels size shared memory by.
struct RobotSet {
    const RobotParams* rp;  // [n] (device)
    const RobotDev* rd;     // [n] (device; read by the collision kernel only)
    int32_t n;
    int32_t n_max;          // largest DoF
    int32_t ns_max;         // most link spheres
    int32_t pairs_max;      // most self-collision body pairs
    int32_t plain = 0;      // 1: every robot of the set is plain (see RobotParams)
};

// One target pose with its request's tolerances, random-stream key, robot,
// scene and iteration caps (64 bytes).
struct __align__(16) TargetDesc {
    float p[3];
    float eps_pos;
    float q[4];  // w x y z, unit
    uint32_t key[2];
    int32_t t_local;  // target index inside its request (keys the streams)
    float eps_ori;
    int32_t robot;     // row of the launch's RobotSet
    int32_t scene;     // row of the launch's scene table, -1: no obstacles
    int16_t cd_iters;  // PO-CCD iteration cap
    int16_t lm_iters;  // PJ-IK iteration cap
    int32_t top_k;     // solutions returned; kNearestFlag set: ranked nearest-first (RankArgs::q_ref)
};
constexpr int32_t kNearestFlag = 1 << 30;
static_assert(sizeof(TargetDesc) == 64, "TargetDesc layout");

// Copy the launch's robot tables into shared memory (all threads of the CTA
// take part; ends with a barrier).
__device__ __forceinline__ const RobotParams* stage_robots(void* smem, const RobotSet& rs) {
    const uint4* src = reinterpret_cast<const uint4*>(rs.rp);
    uint4* dst = reinterpret_cast<uint4*>(smem);
    const int words = rs.n * (int)(sizeof(RobotParams) / 16);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    return reinterpret_cast<const RobotParams*>(smem);
}

__host__ __device__ constexpr size_t robots_smem_bytes(int n) { return (sizeof(RobotParams) * (size_t)n + 15) / 16 * 16; }

// Candidate -> (target row, candidate index inside the target).
struct CandMap {
    const int32_t* tgt;   // explicit [C], or null
    const int32_t* cand;  // explicit [C]
    const int64_t* off;   // [T+1] prefix offsets, used when tgt is null
    int32_t T;
    int32_t stride;       // > 0: every target has this many candidates (off[t] = t * stride)

    // false when an explicit target row is outside [0, T): the candidate is skipped
    __device__ __forceinline__ bool lookup(int64_t c, int32_t& t, int32_t& s) const {
        if (!tgt && stride > 0) {  // no search: a division
            if (c < 0x7fffffff) {
                const uint32_t q = (uint32_t)c / (uint32_t)stride;
                t = (int32_t)q;
                s = (int32_t)((uint32_t)c - q * (uint32_t)stride);
            } else {
                t = (int32_t)(c / stride);
                s = (int32_t)(c - (int64_t)t * stride);
            }
            return true;
        }
        return lookup_search(c, t, s);
    }

    // the same without the stride (kernels that look a candidate up once)
    __device__ __forceinline__ bool lookup_search(int64_t c, int32_t& t, int32_t& s) const {
        if (tgt) {
            t = tgt[c];
            s = cand[c];
            return (uint32_t)t < (uint32_t)T;
        }
        int lo = 0, hi = T - 1;  // largest t with off[t] <= c
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (__ldg(off + mid) <= c) lo = mid;
            else hi = mid - 1;
        }
        t = lo;
        s = (int32_t)(c - __ldg(off + lo));
        return true;
    }
};

// Copy joint vector c (structure of arrays, src[j * ld + c], j < n) into dst(j), K loads in
// flight at a time: a rolled loop would wait out one global-memory latency per joint.
template <int K, class Dst>
__device__ __forceinline__ void load_joints(const float* src, int64_t ld, int64_t c, int n, Dst dst) {
#pragma unroll 1
    for (int j0 = 0; j0 < n; j0 += K) {
        float v[K];
#pragma unroll
        for (int q = 0; q < K; ++q) v[q] = j0 + q < n ? src[(int64_t)(j0 + q) * ld + c] : 0.0f;
#pragma unroll
        for (int q = 0; q < K; ++q)
            if (j0 + q < n) dst(j0 + q, v[q]);
    }
}

// Device work counters (see hjcd_counters).
struct Counters {
    unsigned long long v[8];
};

// ----------------------------------------------------------------------------
// small vector algebra

struct V3 {
    float x, y, z;
};

__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
// s * a + b with fused multiply-adds
__device__ __forceinline__ V3 fma3(float s, V3 a, V3 b) {
    return V3{fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z)};
}
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return V3{fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x)};
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

// sin and cos after reducing x to [-pi, pi] (Cody-Waite, 2*pi split into a
// binary32 head and its residual), where the hardware approximation is
// accurate to ~4e-7 absolute.
__device__ __forceinline__ void sincos_red(float x, float* s, float* c) {
    const float k = rintf(x * 0.159154943091895336f);
    float r = fmaf(-k, 6.28318548202514648f, x);
    r = fmaf(-k, -1.74845553e-07f, r);
    __sincosf(r, s, c);
}

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and the maps to (0,1) and N(0,1)

__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 rnd_block(const TargetDesc& T, uint32_t cand, uint32_t phase, uint32_t iter,
                                           uint32_t block) {
    return philox(make_uint4(cand, (uint32_t)T.t_local, (phase << 24) | (iter & 0xFFFFFFu), block), T.key[0],
                  T.key[1]);
}

// ((x >> 9) + 1/2) * 2^-23: exact in binary32, inside (0, 1)
__device__ __forceinline__ float u01(uint32_t x) { return ((float)(x >> 9) + 0.5f) * 1.1920928955078125e-07f; }

// Square root by the hardware approximation (PTX sqrt.approx.f32, a few ulp):
// for the angles and norms that rank trials and test tolerances, where the
// IEEE-rounded sqrtf's correction steps cost issue slots of issue-bound
// kernels and buy no decision the binary32 kinematics can resolve.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ln u of u = u01(x) in (0, 1).  The hardware logarithm's absolute error (at most 2^-21.4) would
// dominate ln u near 1, so below v = 1 - u = 2^-8 (v exact for u >= 1/2) three terms of
// -ln(1 - v) = v + v^2/2 + v^3/3 + ... take over (truncation below 2e-8 of ln u).
__device__ __forceinline__ float ln_u01(uint32_t x) {
    const float u = u01(x);
    const float v = 1.0f - u;
    return v < 0.00390625f ? -v * fmaf(v, fmaf(v, 0.333333343f, 0.5f), 1.0f) : __logf(u);
}

// N(0, 1) by Box-Muller, cosine branch: sqrt(-2 ln u0) cos(2 pi u1), with the hardware
// approximations (the angle taken as 2 pi (u1 - 1/2) in [-pi, pi), whose cosine is the negated
// one); the absolute error stays below 5e-6 against the exact mapping.
__device__ __forceinline__ float normal01(uint32_t a, uint32_t b) {
    return sqrt_approx(-2.0f * ln_u01(a)) * -__cosf(6.28318530718f * (u01(b) - 0.5f));
}

__device__ __forceinline__ uint32_t word(uint4 w, int i) { return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w)); }

// the pair of normals of block b of a stream: normal 2b from words (x, y),
// normal 2b+1 from words (z, w)
__device__ __forceinline__ float2 normal_pair(const TargetDesc& T, uint32_t cand, uint32_t phase, uint32_t iter,
                                              int b) {
    const uint4 w = rnd_block(T, cand, phase, iter, (uint32_t)b);
    return make_float2(normal01(w.x, w.y), normal01(w.z, w.w));
}

// ----------------------------------------------------------------------------
// forward kinematics (Eq. fk), modified DH in column form
//
// With C0 C1 C2 the columns of R_{0,i-1}: R_{0,i-1} Rx(alpha) has columns
// C0, B1 = ca C1 + sa C2, B2 = ca C2 - sa C1; the origin moves by a C0 + d B2;
// Rz(theta) then gives C0' = c C0 + s B1, C1' = c B1 - s C0, C2' = B2.  The
// joint axis is B2 and the new origin lies on it.

struct Frame {
    V3 c0, c1, c2, p;
};

__device__ __forceinline__ Frame frame_identity() {
    return Frame{v3(1.f, 0.f, 0.f), v3(0.f, 1.f, 0.f), v3(0.f, 0.f, 1.f), v3(0.f, 0.f, 0.f)};
}

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 xy(V3 a) { return make_float2(a.x, a.y); }

// The x and y components run as packed FP32 pairs, the operations of the scalar form in its order.
// RED = false leaves out the offset and the range reduction of theta + offset: the caller
// guarantees theta within the limits of a plain robot, whose offsets are 0 and where the
// reduction's multiple of 2 pi is 0, so both return their argument unchanged (the same bits either
// way, up to the sign of an exact zero).
template <bool RED = true>
__device__ __forceinline__ void fk_step(const RobotParams& R, int j, float theta, Frame& F) {
    const float4 g = R.dh[j];
    const float ca = g.x, sa = g.y;
    const float2 b1 = fma2(bc2(ca), xy(F.c1), mul2(bc2(sa), xy(F.c2)));
    const float b1z = fmaf(ca, F.c1.z, sa * F.c2.z);
    const float2 b2 = fma2(bc2(ca), xy(F.c2), mul2(bc2(-sa), xy(F.c1)));
    const float b2z = fmaf(ca, F.c2.z, (-sa) * F.c1.z);
    const float2 p = fma2(bc2(g.w), b2, fma2(bc2(g.z), xy(F.c0), xy(F.p)));
    F.p = v3(p.x, p.y, fmaf(g.w, b2z, fmaf(g.z, F.c0.z, F.p.z)));
    float s, c;
    if (RED) sincos_red(theta + R.off[j], &s, &c);
    else __sincosf(theta, &s, &c);
    const float2 n0 = fma2(bc2(c), xy(F.c0), mul2(bc2(s), b1));
    const float2 n1 = fma2(bc2(c), b1, mul2(bc2(-s), xy(F.c0)));
    const float n0z = fmaf(c, F.c0.z, s * b1z), n1z = fmaf(c, b1z, (-s) * F.c0.z);
    F.c0 = v3(n0.x, n0.y, n0z);
    F.c1 = v3(n1.x, n1.y, n1z);
    F.c2 = v3(b2.x, b2.y, b2z);
}

// flange frame from the last joint frame
__device__ __forceinline__ Frame fk_flange(const RobotParams& R, const Frame& F) {
    Frame E;
    if (R.fl_eye) {  // the general form's products with 1 and 0 (up to the sign of an exact zero)
        E.c0 = F.c0;
        E.c1 = F.c1;
        E.c2 = F.c2;
        E.p = fma3(R.fl_p[2], F.c2, fma3(R.fl_p[1], F.c1, fma3(R.fl_p[0], F.c0, F.p)));
        return E;
    }
    E.c0 = fma3(R.fl_r[6], F.c2, fma3(R.fl_r[3], F.c1, R.fl_r[0] * F.c0));
    E.c1 = fma3(R.fl_r[7], F.c2, fma3(R.fl_r[4], F.c1, R.fl_r[1] * F.c0));
    E.c2 = fma3(R.fl_r[8], F.c2, fma3(R.fl_r[5], F.c1, R.fl_r[2] * F.c0));
    E.p = fma3(R.fl_p[2], F.c2, fma3(R.fl_p[1], F.c1, fma3(R.fl_p[0], F.c0, F.p)));
    return E;
}

// Flange frame of the joint vector theta[j * stride] (joint loop not
// unrolled: the kernels keep their code small enough for the instruction
// cache, with per-joint state in shared memory).
__device__ __forceinline__ Frame fk_ee_col(const RobotParams& R, const float* th, int stride) {
    Frame F = frame_identity();
#pragma unroll 1
    for (int j = 0; j < R.n; ++j) fk_step(R, j, th[j * stride], F);
    return fk_flange(R, F);
}

// ----------------------------------------------------------------------------
// quaternions (w, x, y, z)

struct Q4 {
    float w;
    V3 v;
};

// Unit quaternion of the rotation with columns c0 c1 c2 (Shepperd's method:
// the largest of 4w^2, 4x^2, 4y^2, 4z^2 from the diagonal, the rest from the
// off-diagonal sums), returned with w >= 0.  The pivot is chosen first and one
// square root serves every case, so lanes with different pivots do not
// diverge; the pivot t = 4 max(w^2, x^2, y^2, z^2) is at least 1, and with
// rs = 1/sqrt(t) the pivot component is t rs / 2 and the others are sums
// times rs / 2.
__device__ __forceinline__ Q4 quat_from_frame(const Frame& E) {
    const float m00 = E.c0.x, m10 = E.c0.y, m20 = E.c0.z;
    const float m01 = E.c1.x, m11 = E.c1.y, m21 = E.c1.z;
    const float m02 = E.c2.x, m12 = E.c2.y, m22 = E.c2.z;
    const float tr = m00 + m11 + m22;
    const bool b0 = tr >= m00 && tr >= m11 && tr >= m22;
    const bool b1 = !b0 && m00 >= m11 && m00 >= m22;
    const bool b2 = !b0 && !b1 && m11 >= m22;
    const float t = b0 ? 1.0f + tr : (b1 ? 1.0f + m00 - m11 - m22 : (b2 ? 1.0f + m11 - m00 - m22 : 1.0f + m22 - m00 - m11));
    const float rs = rsqrtf(t);
    const float h = 0.5f * t * rs, r = 0.5f * rs;
    const float a = (m21 - m12) * r, bq = (m02 - m20) * r, c = (m10 - m01) * r;
    const float d = (m01 + m10) * r, e = (m02 + m20) * r, f = (m12 + m21) * r;
    const float w = b0 ? h : (b1 ? a : (b2 ? bq : c));
    const float x = b0 ? a : (b1 ? h : (b2 ? d : e));
    const float y = b0 ? bq : (b1 ? d : (b2 ? h : f));
    const float z = b0 ? c : (b1 ? e : (b2 ? f : h));
    const float sg = (w < 0.0f) ? -1.0f : 1.0f;
    return Q4{sg * w, v3(sg * x, sg * y, sg * z)};
}

__device__ __forceinline__ Q4 qmul(Q4 a, Q4 b) {
    return Q4{a.w * b.w - dot(a.v, b.v), fma3(a.w, b.v, fma3(b.w, a.v, cross(a.v, b.v)))};
}

// q_err = q_t (x) q_e^-1 with the sign chosen so that w >= 0
__device__ __forceinline__ Q4 quat_error(const TargetDesc& T, Q4 qe) {
    const Q4 qt{T.q[0], v3(T.q[1], T.q[2], T.q[3])};
    Q4 e = qmul(qt, Q4{qe.w, (-1.0f) * qe.v});
    if (e.w < 0.0f) {
        e.w = -e.w;
        e.v = (-1.0f) * e.v;
    }
    return e;
}


// Arctangent of t in [0, 1] as t P(t^2), P of degree 7: the coefficients
// minimise the largest absolute error on a dense grid of [0, 1] (a linear
// program; fit_atan.py beside this file regenerates them); |error| < 3e-8 rad
// in exact arithmetic and < 1.5e-7 rad evaluated in binary32 (checked against
// float64 over [0, 1] by the test suite, which reads these coefficients from
// this file and compares them with the script's output).
__device__ __forceinline__ float atan01(float t) {
    const float s = t * t;
    float p = -4.166443301e-03f;
    p = fmaf(p, s, 2.232482877e-02f);
    p = fmaf(p, s, -5.666722692e-02f);
    p = fmaf(p, s, 9.704074739e-02f);
    p = fmaf(p, s, -1.393516270e-01f);
    p = fmaf(p, s, 1.995220255e-01f);
    p = fmaf(p, s, -3.333036250e-01f);
    p = fmaf(p, s, 9.999994549e-01f);
    return t * p;
}

// atan2(y, x) for y >= 0, x >= 0: the ratio of the smaller to the larger
// argument in [0, 1], reflected about pi/4 when y > x
__device__ __forceinline__ float atan2_q1(float y, float x) {
    const float mx = fmaxf(x, y), mn = fminf(x, y);
    const float a = atan01(__fdividef(mn, fmaxf(mx, 1e-30f)));  // 0 at the origin
    return y > x ? 1.57079632679489662f - a : a;
}

// atan2(y, x) over all four quadrants (atan2(+-0, x < 0) = +-pi)
__device__ __forceinline__ float atan2_all(float y, float x) {
    float a = atan2_q1(fabsf(y), fabsf(x));
    if (x < 0.0f) a = 3.14159265358979324f - a;
    return copysignf(a, y);
}

// rotation angle of a (not necessarily unit-normalised) error quaternion,
// 2 atan2(|v|, |w|): the norm of omega in Eq. quat_diff
__device__ __forceinline__ float quat_angle(float w, float vv) { return 2.0f * atan2_q1(sqrt_approx(vv), fabsf(w)); }

// omega of Eq. quat_diff
__device__ __forceinline__ V3 quat_log(Q4 e) {
    const float vv = dot(e.v, e.v);
    const float rs = rsqrtf(vv);  // |v| = vv rs
    const float f = (vv > 1e-30f) ? 2.0f * atan2_q1(vv * rs, e.w) * rs : __fdividef(2.0f, e.w);  // e.w >= 0
    return f * e.v;
}

// rotate x by the unit quaternion (ch, sh * z) (rotation about unit z by 2 atan2(sh, ch))
__device__ __forceinline__ V3 rotate_half(V3 z, float sh, float ch, V3 x) {
    const V3 u = sh * z;
    const V3 t = 2.0f * cross(u, x);
    return x + fma3(ch, t, cross(u, t));
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-device values looked up once (host threads may launch concurrently: the
// serving scheduler and callers; a process may drive several devices).
constexpr int kMaxDevices = 64;

inline int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev;
}

// SM count of the current device.
inline int sm_count() {
    static std::atomic<int> sms[kMaxDevices];
    const int dev = current_device();
    const int i = dev >= 0 && dev < kMaxDevices ? dev : 0;
    int v = sms[i].load(std::memory_order_relaxed);
    if (v <= 0) {
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v <= 0) v = 1;
        sms[i].store(v, std::memory_order_relaxed);
    }
    return v;
}

// A kernel's dynamic shared-memory limit, raised once per device, at the kernel's first launch
// there, to the most any launch of it takes (clamped to what the device allows beside the
// kernel's static shared memory).  Raising it later, when a launch first needed more than 48 KB,
// made that launch fail ("invalid argument") while smaller launches of the kernel were running
// on other streams.  Under a lock: host threads may launch concurrently.
struct SmemLimit {
    std::mutex mu;
    bool set[kMaxDevices] = {};
};

template <typename K>
inline void allow_dyn_smem(K kernel, SmemLimit& lim, size_t most) {
    const int dev = current_device();
    const int i = dev >= 0 && dev < kMaxDevices ? dev : 0;
    std::lock_guard<std::mutex> g(lim.mu);
    if (lim.set[i] && i == dev) return;
    lim.set[i] = true;
    if (most <= 48 * 1024) return;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kernel);
    const size_t cap = optin > (int)fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : most;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(most < cap ? most : cap));
}

// Grid for a grid-stride kernel: one thread (or warp) per item, capped at
// `per_sm` blocks per SM.

inline int grid_for(int64_t items, int per_block, int per_sm = 64) {
    int64_t b = (items + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// ----------------------------------------------------------------------------
// per-target selection: 64-bit keys (score bits << 32 | index) sorted in
// shared memory by a bitonic network; non-negative scores order like their
// IEEE bit patterns, the index in the low word breaks ties toward the lower
// candidate, and invalid entries get the all-ones key and sort last.

constexpr uint64_t kNoKey = ~0ull;

__device__ __forceinline__ uint64_t score_key(float s, uint32_t idx) {
    if (!(s == s)) return kNoKey;  // NaN
    const uint32_t bits = __float_as_uint(s + 0.0f);  // -0 -> +0
    return ((uint64_t)bits << 32) | idx;
}

__device__ __forceinline__ void bitonic_sort(uint64_t* keys, int N) {
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (N >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t a = keys[lo], b = keys[hi];
                if ((a > b) == up) {
                    keys[lo] = b;
                    keys[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ int pow2_at_least(int m) {
    int N = 1;
    while (N < m) N <<= 1;
    return N;
}

// ----------------------------------------------------------------------------
// host-side launch entry points (defined in the kernel translation units)

struct CcdArgs {
    RobotSet rs;
    const TargetDesc* tg;
    CandMap map;
    int64_t C, ld;
    const float* th_in;  // null: sample seeds
    float* th_out;
    float* th_tmp;       // cd_variant = 2: a second [n][ld] buffer
    float *score, *perr, *oerr;
    int32_t* iters;
    int k0, n_iters;  // n_iters < 0: each target's cd_iters
    hjcd_params P;
    hjcd_ccd_trace tr;
    Counters* cnt;
    int32_t block;  // threads (candidates) per CTA: 64, 128 or 256 (anything else: 128; contexts pass 64 by default)
    int32_t seed_base;  // added to each candidate's index inside its target (a shard of the seeds)
    // Iteration segments (no trace, th_out set): this launch runs iterations [seg_begin, seg_end)
    // (seg_end 0: to the cap) of every candidate, or of the candidates list_in[0 .. *n_in) whose
    // state th_out holds; a candidate still iterating at seg_end keeps its state in th_out and is
    // appended to list_out (count *n_out) instead of writing its results.
    int32_t seg_begin, seg_end;
    int32_t in_limits;  // 1: every joint vector the launch reads lies within its robot's limits
    const int32_t* list_in;
    const int32_t* n_in;
    int32_t* list_out;
    int32_t* n_out;
    // null: the items in a grid stride; else a zeroed queue head the warps take items from
    // (cd_variant 0 and 1)
    unsigned long long* queue;
};

struct LmArgs {
    RobotSet rs;
    const TargetDesc* tg;
    CandMap map;
    int64_t C, ld;
    float* th;
    float *score, *perr, *oerr;
    int32_t* iters;
    int k0, n_iters;  // n_iters < 0: each target's lm_iters
    hjcd_params P;
    hjcd_lm_trace tr;
    Counters* cnt;
    unsigned long long* queue;  // candidate queue head, zero at launch
    int32_t warps;  // warps per CTA: 2, 4 or 8 (anything else: 8, the contexts' default)
    int32_t in_limits;  // 1: every joint vector the launch reads lies within its robot's limits
};

struct DupArgs {
    RobotSet rs;
    const TargetDesc* tg;
    int32_t T;
    const int64_t* m_off;
    const float* score_M;
    const float* th_M;
    int64_t ld_M;
    const int64_t* b_off;
    float* th_B;
    int64_t ld_B;
    int32_t* src_B;
    int32_t ratio;
    float sigma;
};

// Output of target t: solutions at out_q + qe_off[2t] (top_k rows of its
// robot's n), errors at out_err + qe_off[2t+1] (top_k pairs).  With tg null
// every target takes top_k and robot 0; with qe_off null the blocks are
// contiguous in target order.
struct RankArgs {
    RobotSet rs;
    const TargetDesc* tg;
    int32_t T;
    const int64_t* b_off;
    const float* th;
    int64_t ld;
    const float *score, *perr, *oerr;
    const uint8_t* hit;
    int top_k;
    const int64_t* qe_off;
    float* out_q;
    float* out_err;
    int32_t* out_count;
    // with q_ref set ([T][ld_ref], target t's reference configuration in row t): the candidates
    // within the target's tolerances come first, nearest to the reference (squared joint
    // distance), then the others by score
    const float* q_ref;
    int32_t ld_ref;
    // with list set: block b ranks target list[b] when b < *n_list, else nothing (the targets
    // that the bounded lazy pass left unfinished); k_rank_lazy appends those targets here
    int32_t* list;
    int32_t* n_list;
    // tolerances of every target when tg is null (with tg: each target row's own)
    float eps_pos, eps_ori;
};

// Ranking key of candidate i of target t (candidates [b0, b0 + B), robot DoF
// n), never for a colliding candidate (with use_hit) or a non-finite score.
// Reading c20 of Alg. 2's final step: the candidates within the target's
// tolerances (|e_p| <= eps_pos and |omega| <= eps_ori) form class 0, the rest
// class 1 (the top key bit), each class ordered by score and then index.  With
// the target's nearest flag (with tg null: whenever q_ref is set), class 0 is
// ordered by squared joint distance to the reference q_ref[t] instead
// (reading c24).  kNoKey past B.
__device__ __forceinline__ uint64_t rank_key(const RankArgs& A, int t, int64_t b0, int B, int n, int i, bool use_hit) {
    if (i >= B || (use_hit && A.hit && A.hit[b0 + i])) return kNoKey;
    const int64_t g = b0 + i;
    const float sc = A.score[g];
    if (!(sc < __int_as_float(0x7f800000))) return kNoKey;  // finite only
    const float ep = A.tg ? A.tg[t].eps_pos : A.eps_pos, eo = A.tg ? A.tg[t].eps_ori : A.eps_ori;
    const bool conv = A.perr[g] <= ep && A.oerr[g] <= eo;
    const bool nearest = A.q_ref && (!A.tg || (A.tg[t].top_k & kNearestFlag));
    if (conv && nearest) {
        float d2 = 0.0f;
        for (int j = 0; j < n; ++j) {
            const float dj = A.th[j * A.ld + g] - A.q_ref[(int64_t)t * A.ld_ref + j];
            d2 = fmaf(dj, dj, d2);
        }
        return score_key(d2, (uint32_t)i);
    }
    const uint64_t k = score_key(sc, (uint32_t)i);
    return conv ? k : (k | (1ull << 63));
}

// Collision filter of C candidates.  With tg null or uniform set every
// candidate is robot 0 against scene 0 (if any); otherwise candidate c belongs
// to target row map(c), whose robot and scene it uses (an invalid row: hit).  A launch with a single scene
// stages it into shared memory; with several, obstacles are read from the
// scene tables directly.
struct CollideArgs {
    RobotSet rs;
    const SceneDev* scenes;   // [n_scenes] (device)
    int32_t n_scenes;
    int32_t max_obj4;         // largest n_sph + 2 n_box over the scenes
    int32_t uniform;          // every candidate: robot 0 and scene 0 (if any) -- no per-candidate lookup
    int32_t has_grid;         // some scene of the launch carries a uniform grid
    // with uniform set: robot 0's DoF and checked body pairs, scene 0's obstacle counts (0 without a scene)
    int32_t u_n, u_pairs, u_osph, u_obox;
    const TargetDesc* tg;
    CandMap map;
    int64_t C, ld;
    const float* th;
    uint8_t* hit;
    Counters* cnt;
    int32_t* err_flag;        // set when the bounded wait for the staged tables runs out
    // polls of the first wait for the staged tables (< 0: the kernels' default limit); 0 makes
    // that wait run out at once, which only tests of the timeout path ask for
    int64_t first_wait_polls = -1;
    // with list set: only the candidates of the targets list[0 .. *n_list) whose hit entry is 2
    // are checked, item i = (list entry i / list_bmax, candidate i % list_bmax of that target's
    // b_off range)
    const int32_t* list;
    const int32_t* n_list;
    const int64_t* b_off;
    int32_t list_bmax;
};

// Fill p and q of the target rows from [T][7] poses (quaternion normalised; a
// zero or non-finite one marks the row invalid with eps_pos = -1).  With meta
// non-null the other fields come from meta[t], else from tmpl with t_local = t.
// Per target t: the K = max(1, floor(M_full / ratio)) lowest scores of its
// candidates [off[t], off[t+1]) (ties to the lower index), written as score,
// seed index (seed_base + index in the target) and joint vector; +inf / -1
// past the candidates.  out_th [T][K][ld_n], out_s / out_i [T][K].
struct ShardTopkArgs {
    RobotSet rs;
    const TargetDesc* tg;
    int32_t T, K, seed_base;
    const int64_t* off;
    const float* score;
    const float* th;
    int64_t ld;
    float* out_s;
    int32_t* out_i;
    float* out_th;
    int32_t ld_n;
};
void launch_shard_topk(const ShardTopkArgs& A, int max_m, cudaStream_t st);

// Per target: the K best of L lists of K (score, seed index, joint vector),
// ties to the lower seed index.
struct MergeArgs {
    int32_t T, L, K, n;
    const float* in_s;   // [L][T][K]
    const int32_t* in_i; // [L][T][K]
    const float* in_th;  // [L][T][K][n]
    float* out_s;
    int32_t* out_i;
    float* out_th;       // [T][K][n]
};
void launch_topk_merge(const MergeArgs& A, cudaStream_t st);

// Alg. 2's duplication from kept seeds given per target ([T][K][n], best first):
// copy r of seed i at index r K + i, perturbed as in k_topk_dup.
struct KeptDupArgs {
    RobotSet rs;
    const TargetDesc* tg;
    int32_t T, K;
    const float* kept;   // [T][K][n]
    const int64_t* b_off;
    float* th_B;
    int64_t ld_B;
    float sigma;
};
void launch_dup_kept(const KeptDupArgs& A, cudaStream_t st);

void launch_pack_targets(const float* pq7, int T, const TargetDesc* meta, const TargetDesc& tmpl, TargetDesc* out,
                         cudaStream_t st);
void launch_fk(const RobotParams& R, int64_t C, const float* th, int64_t ld, float* out, cudaStream_t st);
void launch_sample(const RobotParams& R, uint64_t seed, CandMap map, int64_t C, float* th, int64_t ld,
                   cudaStream_t st);
void launch_ccd(const CcdArgs& A, bool trace, cudaStream_t st);
void launch_lm(const LmArgs& A, bool trace, cudaStream_t st);
void launch_topk_dup(const DupArgs& A, int max_m, cudaStream_t st);
void launch_rank(const RankArgs& A, int max_b, cudaStream_t st);
void launch_collide(const CollideArgs& A, cudaStream_t st);
// The ranking with the collision filter applied lazily (k_rank_lazy); false
// when it does not apply (no spheres, no target rows, or too large for shared
// memory): use launch_collide + launch_rank.  With R.list set, a target whose
// first `depth` ranked candidates hold fewer than top_k collision-free ones is
// appended to R.list instead of ranked; launch_collide and launch_rank with
// that list finish those targets.
bool launch_rank_lazy(const CollideArgs& A, const RankArgs& R, int max_b, int depth, cudaStream_t st);
void launch_contacts(const RobotParams& R, const RobotDev& rd, const SceneDev& sc, const int32_t* perm, int64_t C,
                     const float* th, int64_t ld, uint8_t* touched, cudaStream_t st);
void launch_ffma(float* sink, int iters, int blocks, cudaStream_t st);
void launch_philox(int64_t n, const uint32_t* ctr, uint64_t key, uint32_t* out, cudaStream_t st);
int ffma_flops_per_thread_iter();

}  // namespace hjcd

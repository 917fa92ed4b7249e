// Quadrotor dynamics and its adjoint, one thread per agent (sm_103a, FP32).
//
// Forward step (Sec. III-A): body-rate (CTBR) controller -> rotor first-order
// lag (Eq. 4, exact over the sub-step) -> rotor thrusts, collective thrust and
// moment (Eq. 3, 4) held over the sub-step -> RK4 (or Euler) on Eq. 1 with
// body-frame quadratic drag (Eq. 2) -> quaternion normalisation.
//
// Adjoint: hand-derived reverse mode of the same map.  Each thread recomputes
// its agent's forward internals (stage states, clamp flags) and sweeps them
// backwards; the rollout adjoint re-runs K steps from a checkpoint, keeps them
// in thread-local memory and walks them in reverse.
//
// Layout: state SoA float32 [17][n], commands [4][n]; loads and stores are
// coalesced across the agents of a warp.
#include "common.cuh"
#include "launch.h"

namespace vf {
namespace {

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Body-to-world rotation of q / |q| (q = w, x, y, z); also returns 1/|q|^2.
__device__ __forceinline__ void rotation(const float q[4], float R[3][3], float& inv_n) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    inv_n = 1.0f / (w * w + x * x + y * y + z * z);
    R[0][0] = (w * w + x * x - y * y - z * z) * inv_n;
    R[0][1] = 2.0f * (x * y - w * z) * inv_n;
    R[0][2] = 2.0f * (x * z + w * y) * inv_n;
    R[1][0] = 2.0f * (x * y + w * z) * inv_n;
    R[1][1] = (w * w - x * x + y * y - z * z) * inv_n;
    R[1][2] = 2.0f * (y * z - w * x) * inv_n;
    R[2][0] = 2.0f * (x * z - w * y) * inv_n;
    R[2][1] = 2.0f * (y * z + w * x) * inv_n;
    R[2][2] = (w * w - x * x - y * y + z * z) * inv_n;
}

// Controller internals kept for the adjoint.
struct CtrlTape {
    float fc[4];      // clamped rotor thrust requests
    float dw_df[4];   // slope of the thrust inverse at fc
    bool in_f[4];     // thrust request inside [f_lo, f_hi]
    bool in_w[4];     // rotor speed inside [omega_min, omega_max]
};

// ---------------------------------------------------------------- double-float
// A value as the unevaluated sum hi + lo of two floats (about 48 significant
// bits), built from exact products (FMA) and exact sums (Knuth's two-sum).
// This GPU runs FP64 at a small fraction of its FP32 rate, so the controller's
// cancellation-prone steps use these pairs on the FP32 pipes instead.
struct dfl {
    float hi, lo;
};
// The additions and products below are written with the _rn intrinsics: the
// compiler never fuses those into FMAs, which would break the exact
// transformations.
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfl df_norm(float hi, float lo) {  // |hi| >= |lo|
    const float s = __fadd_rn(hi, lo);
    return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
__device__ __forceinline__ dfl df_of(float2 c) { return {c.x, c.y}; }
__device__ __forceinline__ dfl df_of(float a) { return {a, 0.0f}; }
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const dfl s = df_two_sum(a.hi, b.hi), t = df_two_sum(a.lo, b.lo);
    const dfl u = df_norm(s.hi, __fadd_rn(s.lo, t.hi));
    return df_norm(u.hi, __fadd_rn(u.lo, t.lo));
}
// a + b with one two-sum on the high parts: error about 2^-44 relative to
// the operands (not to the result), for sums whose result need not keep full
// precision under cancellation
__device__ __forceinline__ dfl df_add_fast(dfl a, dfl b) {
    const dfl s = df_two_sum(a.hi, b.hi);
    return df_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_sub_fast(dfl a, dfl b) { return df_add_fast(a, df_neg(b)); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return df_norm(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
__device__ __forceinline__ bool df_lt(dfl a, dfl b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ float df_float(dfl a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ dfl df_twice(dfl a) { return {__fmul_rn(2.0f, a.hi), __fmul_rn(2.0f, a.lo)}; }
// a / b: an FP32 quotient, then one correction from the double-float
// remainder a - q b (relative error about 1e-14).
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
    const float r = __frcp_rn(b.hi);
    const float q = __fmul_rn(a.hi, r);
    const dfl rem = df_sub(a, df_mul(b, df_of(q)));
    return df_norm(q, __fmul_rn(rem.hi, r));
}
// sqrt(a) for a >= 0: the FP32 root s, then one Newton correction
// (a - s^2) / (2 s) with s^2 formed exactly.
__device__ __forceinline__ dfl df_sqrt(dfl a) {
    const float s = __fsqrt_rn(a.hi);
    if (!(s > 0.0f)) return {s, 0.0f};
    const float p = __fmul_rn(s, s);
    const dfl rem = df_sub(a, dfl{p, __fmaf_rn(s, s, -p)});
    return df_norm(s, __fmul_rn(rem.hi, __frcp_rn(__fmul_rn(2.0f, s))));
}
// 1/n! as double-float pairs, n = 0 .. 17
__constant__ float2 kInvFact[18] = {
    {0x1p+0f, 0.0f}, {0x1p+0f, 0.0f}, {0x1p-1f, 0.0f}, {0x1.555556p-3f, -0x1.555556p-28f},
    {0x1.555556p-5f, -0x1.555556p-30f}, {0x1.111112p-7f, -0x1.dddddep-32f}, {0x1.6c16c2p-10f, -0x1.27d27ep-35f},
    {0x1.a01a02p-13f, -0x1.7f97fap-39f}, {0x1.a01a02p-16f, -0x1.7f97fap-42f}, {0x1.71de3ap-19f, 0x1.55b1ccp-45f},
    {0x1.27e4fcp-22f, -0x1.10ec14p-47f}, {0x1.ae6456p-26f, 0x1.fd5138p-52f}, {0x1.1eed8ep-29f, 0x1.ff1b12p-54f},
    {0x1.612462p-33f, -0x1.8af25ep-58f}, {0x1.93974ap-37f, 0x1.180f94p-62f}, {0x1.ae7f3ep-41f, 0x1.ccee08p-67f},
    {0x1.ae7f3ep-45f, 0x1.ccee08p-71f}, {0x1.952c78p-49f, -0x1.f9ea56p-74f}};
// sin a and cos a of a float angle as double-float pairs.  Cody-Waite
// reduction r = a - k pi/2 with pi/2 = P1 + P2 + P3 in three floats (each
// product k Pi is exact as an FMA pair), then the Taylor series of sin and
// cos on |r| <= pi/4, Horner in r^2 up to r^17 / 17!, and the quadrant of k.
// Absolute error below 1e-14 for |a| < 1e6 against FP64 sin and cos.
__device__ __forceinline__ void df_sincos(float a, dfl& sa, dfl& ca) {
    const float k = rintf(a * 0x1.45f306p-1f);
    dfl r = df_sub(df_of(a), df_mul(df_of(k), df_of(0x1.921fb6p+0f)));
    r = df_sub(r, df_mul(df_of(k), df_of(-0x1.777a5cp-25f)));
    r = df_sub(r, df_mul(df_of(k), df_of(-0x1.ee59dap-50f)));
    const dfl x = df_mul(r, r);
    dfl ps = df_of(kInvFact[17]), pc = df_of(kInvFact[16]);
#pragma unroll
    for (int j = 7; j >= 0; --j) {
        const dfl fs = df_of(kInvFact[2 * j + 1]), fc = df_of(kInvFact[2 * j]);
        ps = df_add_fast(df_mul(ps, x), (j & 1) ? df_neg(fs) : fs);
        pc = df_add_fast(df_mul(pc, x), (j & 1) ? df_neg(fc) : fc);
    }
    const dfl sr = df_mul(r, ps);
    const int q = (int)k & 3;
    sa = q == 0 ? sr : q == 1 ? pc : q == 2 ? df_neg(sr) : df_neg(pc);
    ca = q == 0 ? pc : q == 1 ? df_neg(sr) : q == 2 ? df_neg(pc) : sr;
}
__device__ __forceinline__ dfl df_dot3(const dfl a[3], const dfl b[3]) {
    return df_add_fast(df_add_fast(df_mul(a[0], b[0]), df_mul(a[1], b[1])), df_mul(a[2], b[2]));
}
// a x b
__device__ __forceinline__ void df_cross(const dfl a[3], const dfl b[3], dfl r[3]) {
    r[0] = df_sub_fast(df_mul(a[1], b[2]), df_mul(a[2], b[1]));
    r[1] = df_sub_fast(df_mul(a[2], b[0]), df_mul(a[0], b[2]));
    r[2] = df_sub_fast(df_mul(a[0], b[1]), df_mul(a[1], b[0]));
}

// ---------------------------------------------------------------- thrust allocation
// Shared by the controllers: rotor thrusts f = Ainv (collective thrust,
// moment), clamped to the reachable range, and the desired rotor speeds from
// the thrust polynomial's positive root.

// Rotor speed of thrust fc, the positive root of k2 w^2 + k1 w + k0 = fc
// (Eq. 4 inverted); dw = dw/dfc.  The discriminant k1^2 - 4 k2 (k0 - fc) is a
// small difference of larger terms near zero thrust and is formed in double
// precision; the root is then taken in FP32 in the cancellation-free form
// w = 2 (fc - k0) / (sqrt(disc) + k1), which equals (sqrt(disc) - k1) / (2 k2).
__device__ __forceinline__ float rotor_speed(const DynConsts& c, dfl fc, float& dw) {
    const dfl f0 = df_sub(fc, df_of(c.xk0));
    if (c.k2 != 0.0f) {
        const dfl disc = df_add(df_of(c.xk1sq), df_mul(df_of(c.x4k2), f0));
        const float sq = sqrtf(fmaxf(df_float(disc), 0.0f));
        const float den = sq + c.k1;
        dw = sq > 0.0f ? 1.0f / sq : 0.0f;
        return den > 0.0f ? 2.0f * df_float(f0) / den : 0.0f;
    }
    dw = 1.0f / c.k1;
    return df_float(f0) / c.k1;
}

// Clamp rotor thrust i to the reachable range, invert it to a rotor speed and
// clamp that; record what the adjoint needs.
__device__ __forceinline__ void rotor_command(const DynConsts& c, int i, dfl f, float omega_des[4], CtrlTape* tape) {
    const dfl lo = df_of(c.xf_lo), hi = df_of(c.xf_hi);
    const bool in_f = !df_lt(f, lo) && !df_lt(hi, f);
    const dfl fc = df_lt(f, lo) ? lo : (df_lt(hi, f) ? hi : f);
    float dw;
    const float w = rotor_speed(c, fc, dw);
    const bool in_w = w >= c.omega_min && w <= c.omega_max;
    omega_des[i] = fminf(fmaxf(w, c.omega_min), c.omega_max);
    if (tape) {
        tape->fc[i] = df_float(fc);
        tape->dw_df[i] = dw;
        tape->in_f[i] = in_f;
        tape->in_w[i] = in_w;
    }
}

// Mixer: rotor thrusts from (collective thrust, moment), f = A^-1 rhs.
__device__ __forceinline__ void allocate(const DynConsts& c, const dfl rhs[4], float omega_des[4], CtrlTape* tape) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        dfl f = df_mul(df_of(c.xAinv[i][0]), rhs[0]);
#pragma unroll
        for (int k = 1; k < 4; ++k) f = df_add(f, df_mul(df_of(c.xAinv[i][k]), rhs[k]));
        rotor_command(c, i, f, omega_des, tape);
    }
}

// CTBR: u0 -> collective thrust m a, u1..3 -> desired rates; P rate loop with
// gyroscopic feed-forward -> desired moment (Sec. III-A; the action type of the
// paper's examples, Sec. IV).
__device__ __forceinline__ void ctbr_rhs(const DynConsts& c, const float Om[3], const float u[4], dfl rhs[4]) {
    dfl L[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) L[j] = df_mul(df_of(c.xJ[j]), df_of(Om[j]));
    // gyroscopic feed-forward Omega x (J Omega)
    const dfl gyro[3] = {df_sub(df_mul(df_of(Om[1]), L[2]), df_mul(df_of(Om[2]), L[1])),
                         df_sub(df_mul(df_of(Om[2]), L[0]), df_mul(df_of(Om[0]), L[2])),
                         df_sub(df_mul(df_of(Om[0]), L[1]), df_mul(df_of(Om[1]), L[0]))};
    rhs[0] = df_mul(df_two_sum(u[0], 1.0f), df_of(c.xhalf_a_max_m));
#pragma unroll
    for (int j = 0; j < 3; ++j)
        rhs[j + 1] = df_add(df_mul(df_of(c.xJK[j]),
                                   df_sub(df_mul(df_of(u[j + 1]), df_of(c.xrate_max[j])), df_of(Om[j]))),
                            gyro[j]);
}

// LV / PS (geometric control with yaw, after Lee et al. 2010): desired force
// from the velocity (LV) or position and velocity (PS) errors plus gravity;
// collective thrust = its projection on body z; desired attitude from the
// force direction and the yaw command; moment from the attitude and rate
// errors plus the gyroscopic term.  u = (target, yaw) in m or m/s and rad.
// On double-float pairs like the CTBR law, the yaw's sine and cosine
// included.  R is used unnormalised (Rr = |q|^2 R): the collective thrust
// and the attitude error are linear in it and take the 1/|q|^2 at the end.
__device__ void geometric_rhs(const DynConsts& c, const float y[17], const float u[4], bool position, dfl rhs[4]) {
    dfl sy, cy;
    df_sincos(u[3], sy, cy);
    const float w = y[6], x = y[7], yq = y[8], z = y[9];
    auto pr = [](float a, float b) { return df_mul(df_of(a), df_of(b)); };  // exact
    const dfl ww = pr(w, w), xx = pr(x, x), yy = pr(yq, yq), zz = pr(z, z);
    const dfl xy = pr(x, yq), wz = pr(w, z), xz = pr(x, z), wy = pr(w, yq), yz = pr(yq, z), wx = pr(w, x);
    const dfl inv_n = df_div(df_of(1.0f), df_add_fast(df_add_fast(ww, xx), df_add_fast(yy, zz)));
    dfl Rr[3][3];
    Rr[0][0] = df_sub_fast(df_add_fast(ww, xx), df_add_fast(yy, zz));
    Rr[0][1] = df_twice(df_sub_fast(xy, wz));
    Rr[0][2] = df_twice(df_add_fast(xz, wy));
    Rr[1][0] = df_twice(df_add_fast(xy, wz));
    Rr[1][1] = df_sub_fast(df_add_fast(ww, yy), df_add_fast(xx, zz));
    Rr[1][2] = df_twice(df_sub_fast(yz, wx));
    Rr[2][0] = df_twice(df_sub_fast(xz, wy));
    Rr[2][1] = df_twice(df_add_fast(yz, wx));
    Rr[2][2] = df_sub_fast(df_add_fast(ww, zz), df_add_fast(xx, yy));
    dfl F[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (position)
            F[j] = df_neg(df_add_fast(df_mul(df_of(c.xmKpos[j]), df_two_sum(y[j], -u[j])),
                                 df_mul(df_of(c.xmKvel[j]), df_of(y[3 + j]))));
        else
            F[j] = df_neg(df_mul(df_of(c.xmKvel[j]), df_two_sum(y[3 + j], -u[j])));
    }
    F[2] = df_add_fast(F[2], df_of(c.xmg));
    const dfl col2[3] = {Rr[0][2], Rr[1][2], Rr[2][2]};
    rhs[0] = df_mul(df_dot3(F, col2), inv_n);
    dfl b3[3] = {df_of(0.0f), df_of(0.0f), df_of(1.0f)};
    const dfl nF = df_sqrt(df_dot3(F, F));
    if (nF.hi >= 1e-9f) {
        const dfl r = df_div(df_of(1.0f), nF);
#pragma unroll
        for (int k = 0; k < 3; ++k) b3[k] = df_mul(F[k], r);
    }
    const dfl zero = df_of(0.0f);
    const dfl c1[3] = {cy, sy, zero};
    dfl b2[3];
    df_cross(b3, c1, b2);
    dfl n2 = df_sqrt(df_dot3(b2, b2));
    if (n2.hi < 1e-6f) {
        const dfl c1b[3] = {df_neg(sy), cy, zero};
        df_cross(b3, c1b, b2);
        n2 = df_sqrt(df_dot3(b2, b2));
    }
    const dfl r2 = df_div(df_of(1.0f), n2);
#pragma unroll
    for (int k = 0; k < 3; ++k) b2[k] = df_mul(b2[k], r2);
    dfl b1[3];
    df_cross(b2, b3, b1);
    // vee of M = Rd^T R - R^T Rd with Rd = [b1 b2 b3]: the entries (2,1),
    // (0,2), (1,0), i.e. sum_k Rd[k][i] R[k][j] - R[k][i] Rd[k][j]
    const dfl* bcol[3] = {b1, b2, b3};
    const int I[3] = {2, 0, 1}, J[3] = {1, 2, 0};
    dfl eR[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int i = I[e], j = J[e];
        dfl m = df_sub_fast(df_mul(bcol[i][0], Rr[0][j]), df_mul(Rr[0][i], bcol[j][0]));
#pragma unroll
        for (int k = 1; k < 3; ++k)
            m = df_add_fast(m, df_sub_fast(df_mul(bcol[i][k], Rr[k][j]), df_mul(Rr[k][i], bcol[j][k])));
        const dfl mn = df_mul(m, inv_n);
        eR[e] = {__fmul_rn(0.5f, mn.hi), __fmul_rn(0.5f, mn.lo)};
    }
    const dfl Om[3] = {df_of(y[10]), df_of(y[11]), df_of(y[12])};
    const dfl L[3] = {df_mul(df_of(c.xJ[0]), Om[0]), df_mul(df_of(c.xJ[1]), Om[1]), df_mul(df_of(c.xJ[2]), Om[2])};
    dfl gyro[3];
    df_cross(Om, L, gyro);
#pragma unroll
    for (int j = 0; j < 3; ++j)
        rhs[j + 1] = df_sub_fast(gyro[j], df_add_fast(df_mul(df_of(c.xJKatt[j]), eR[j]), df_mul(df_of(c.xJKom[j]), Om[j])));
}

// Desired rotor speeds from the selected controller.  GEO = false leaves the
// geometric controllers (LV, PS) out at compile time: their law is several
// times the size of the CTBR and SRT paths, and each launch fetches its code
// from a cold instruction cache.
template <bool GEO>
__device__ __forceinline__ void controller(const DynConsts& c, const float y[17], const float u[4],
                                           float omega_des[4], CtrlTape* tape) {
    if (c.controller == 1) {
        // SRT: u_i in [-1, 1] -> rotor i's thrust (u_i + 1) / 2 * f(omega_max)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            rotor_command(c, i, df_mul(df_two_sum(u[i], 1.0f), df_of(c.xhalf_f_hi)), omega_des, tape);
        return;
    }
    dfl rhs[4];
    if (GEO && (c.controller == 2 || c.controller == 3))
        geometric_rhs(c, y, u, c.controller == 3, rhs);
    else
        ctbr_rhs(c, y + 10, u, rhs);
    allocate(c, rhs, omega_des, tape);
}

// Eq. 1 right-hand side for y = (x, v, q, Omega) with body thrust (0,0,Fz) and
// moment eta fixed; drag d = -rho Cd s / 2 * v_B |v_B| per body axis (Eq. 2).
__device__ __forceinline__ void rhs(const DynConsts& c, const float y[13], float Fz, const float eta[3],
                                    float dy[13]) {
    const float* v = y + 3;
    const float* q = y + 6;
    const float* Om = y + 10;
    float R[3][3], inv_n;
    rotation(q, R, inv_n);
    float fB[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float vb = R[0][j] * v[0] + R[1][j] * v[1] + R[2][j] * v[2];
        fB[j] = -c.drag[j] * vb * fabsf(vb);
    }
    fB[2] += Fz;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        dy[j] = v[j];
        dy[3 + j] = (R[j][0] * fB[0] + R[j][1] * fB[1] + R[j][2] * fB[2]) * c.inv_mass;
    }
    dy[5] -= c.g;
    dy[6] = 0.5f * (-q[1] * Om[0] - q[2] * Om[1] - q[3] * Om[2]);
    dy[7] = 0.5f * (q[0] * Om[0] + q[2] * Om[2] - q[3] * Om[1]);
    dy[8] = 0.5f * (q[0] * Om[1] - q[1] * Om[2] + q[3] * Om[0]);
    dy[9] = 0.5f * (q[0] * Om[2] + q[1] * Om[1] - q[2] * Om[0]);
    float L[3] = {c.J[0] * Om[0], c.J[1] * Om[1], c.J[2] * Om[2]};
    float cr[3];
    cross3(Om, L, cr);
#pragma unroll
    for (int j = 0; j < 3; ++j) dy[10 + j] = (eta[j] - cr[j]) * c.invJ[j];
}

// Controller, rotor lag and thrust/moment of one sub-step.
template <bool GEO>
__device__ __forceinline__ void rotors(const DynConsts& c, float y[17], const float u[4], float& Fz, float eta[3],
                                       CtrlTape* tape) {
    float wd[4];
    controller<GEO>(c, y, u, wd, tape);
    Fz = 0.0f;
    eta[0] = eta[1] = eta[2] = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float w = wd[i] + (y[13 + i] - wd[i]) * c.decay;
        y[13 + i] = w;
        const float f = (c.k2 * w + c.k1) * w + c.k0;
        Fz += f;
        eta[0] += c.mix[0][i] * f;
        eta[1] += c.mix[1][i] * f;
        eta[2] += c.mix[2][i] * f;
    }
}

template <bool GEO = false>
__device__ __forceinline__ void substep(const DynConsts& c, float y[17], const float u[4]) {
    float Fz, eta[3];
    rotors<GEO>(c, y, u, Fz, eta, nullptr);
    const float h = c.h;
    if (c.integrator == 1) {
        float k1[13];
        rhs(c, y, Fz, eta, k1);
#pragma unroll
        for (int j = 0; j < 13; ++j) y[j] += h * k1[j];
    } else {
        float k[13], acc[13], yt[13];
        rhs(c, y, Fz, eta, k);
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            acc[j] = k[j];
            yt[j] = y[j] + 0.5f * h * k[j];
        }
        rhs(c, yt, Fz, eta, k);
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            acc[j] += 2.0f * k[j];
            yt[j] = y[j] + 0.5f * h * k[j];
        }
        rhs(c, yt, Fz, eta, k);
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            acc[j] += 2.0f * k[j];
            yt[j] = y[j] + h * k[j];
        }
        rhs(c, yt, Fz, eta, k);
#pragma unroll
        for (int j = 0; j < 13; ++j) y[j] += (h / 6.0f) * (acc[j] + k[j]);
    }
    const float qn = rsqrtf(y[6] * y[6] + y[7] * y[7] + y[8] * y[8] + y[9] * y[9]);
#pragma unroll
    for (int j = 6; j < 10; ++j) y[j] *= qn;
}

template <bool GEO = false>
__device__ __forceinline__ void control_step(const DynConsts& c, float y[17], const float u[4]) {
    for (int s = 0; s < c.n_sub; ++s) substep<GEO>(c, y, u);
}

// ---------------------------------------------------------------- adjoint
// Reverse mode of rhs(): accumulate the cotangents of y, Fz and eta from the
// cotangent kb of dy.
__device__ void rhs_vjp(const DynConsts& c, const float y[13], float Fz, const float kb[13], float yb[13],
                        float& Fzb, float etab[3]) {
    const float* v = y + 3;
    const float* q = y + 6;
    const float* Om = y + 10;
    float R[3][3], inv_n;
    rotation(q, R, inv_n);
    float vB[3], fB[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        vB[j] = R[0][j] * v[0] + R[1][j] * v[1] + R[2][j] * v[2];
        fB[j] = -c.drag[j] * vB[j] * fabsf(vB[j]);
    }
    fB[2] += Fz;
    // dx = v
#pragma unroll
    for (int j = 0; j < 3; ++j) yb[3 + j] += kb[j];
    // dv = R fB / m - g z
    const float* kv = kb + 3;
    float Rb[3][3];
    float fBb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        fBb[j] = (R[0][j] * kv[0] + R[1][j] * kv[1] + R[2][j] * kv[2]) * c.inv_mass;
#pragma unroll
        for (int i = 0; i < 3; ++i) Rb[i][j] = kv[i] * fB[j] * c.inv_mass;
    }
    Fzb += fBb[2];
    float vBb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) vBb[j] = fBb[j] * (-2.0f * c.drag[j] * fabsf(vB[j]));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        yb[3 + i] += R[i][0] * vBb[0] + R[i][1] * vBb[1] + R[i][2] * vBb[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) Rb[i][j] += v[i] * vBb[j];
    }
    // dq = 1/2 q (x) (0, Omega)
    const float h0 = 0.5f * kb[6], h1 = 0.5f * kb[7], h2 = 0.5f * kb[8], h3 = 0.5f * kb[9];
    float qb[4];
    qb[0] = h1 * Om[0] + h2 * Om[1] + h3 * Om[2];
    qb[1] = -h0 * Om[0] - h2 * Om[2] + h3 * Om[1];
    qb[2] = -h0 * Om[1] + h1 * Om[2] - h3 * Om[0];
    qb[3] = -h0 * Om[2] - h1 * Om[1] + h2 * Om[0];
    yb[10] += -h0 * q[1] + h1 * q[0] + h2 * q[3] - h3 * q[2];
    yb[11] += -h0 * q[2] - h1 * q[3] + h2 * q[0] + h3 * q[1];
    yb[12] += -h0 * q[3] + h1 * q[2] - h2 * q[1] + h3 * q[0];
    // dOmega = (eta - Omega x J Omega) / J
    float cb[3], L[3] = {c.J[0] * Om[0], c.J[1] * Om[1], c.J[2] * Om[2]};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        etab[j] += kb[10 + j] * c.invJ[j];
        cb[j] = -kb[10 + j] * c.invJ[j];
    }
    float t[3], Lb[3];
    cross3(L, cb, t);   // Omega-bar from Omega in (Omega x L)
    cross3(cb, Om, Lb); // L-bar
#pragma unroll
    for (int j = 0; j < 3; ++j) yb[10 + j] += t[j] + c.J[j] * Lb[j];
    // R(q) = M(q) / |q|^2
    const float w = q[0], x = q[1], yy = q[2], z = q[3];
    float dot = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dot += Rb[i][j] * R[i][j];
    const float gw = 2.0f * (w * (Rb[0][0] + Rb[1][1] + Rb[2][2]) + z * (Rb[1][0] - Rb[0][1]) +
                             yy * (Rb[0][2] - Rb[2][0]) + x * (Rb[2][1] - Rb[1][2]));
    const float gx = 2.0f * (x * (Rb[0][0] - Rb[1][1] - Rb[2][2]) + yy * (Rb[0][1] + Rb[1][0]) +
                             z * (Rb[0][2] + Rb[2][0]) + w * (Rb[2][1] - Rb[1][2]));
    const float gy = 2.0f * (yy * (-Rb[0][0] + Rb[1][1] - Rb[2][2]) + x * (Rb[0][1] + Rb[1][0]) +
                             w * (Rb[0][2] - Rb[2][0]) + z * (Rb[1][2] + Rb[2][1]));
    const float gz = 2.0f * (z * (-Rb[0][0] - Rb[1][1] + Rb[2][2]) + w * (Rb[1][0] - Rb[0][1]) +
                             x * (Rb[0][2] + Rb[2][0]) + yy * (Rb[1][2] + Rb[2][1]));
    yb[6] += qb[0] + gw * inv_n - 2.0f * w * inv_n * dot;
    yb[7] += qb[1] + gx * inv_n - 2.0f * x * inv_n * dot;
    yb[8] += qb[2] + gy * inv_n - 2.0f * yy * inv_n * dot;
    yb[9] += qb[3] + gz * inv_n - 2.0f * z * inv_n * dot;
}

// Reverse mode of one sub-step: y_in (pre), u, cotangent gout of the post-sub-
// step state -> gin (cotangent of y_in) and accumulated gu.
// What the reverse sweep of one sub-step needs from its forward pass: the
// controller's tape, the held collective thrust, the lagged rotor speeds, the
// inputs of RK4 stages 2-4 (stage 1 starts from the sub-step's own input) and
// the un-normalised result.
struct StepTape {
    CtrlTape ctrl;
    float Fz, w[4];
    float ys[3][13];
    float yn[13];
};
constexpr int kTapeWords = 4 + 4 + 1 + 1 + 4 + 3 * 13 + 13;  // fc, dw_df, flag bits, Fz, w, ys, yn

// Forward pass of one sub-step from y_in, recording the tape (the same
// arithmetic as substep()).
__device__ void substep_record(const DynConsts& c, const float y_in[17], const float u[4], StepTape& T) {
    float y[17];
#pragma unroll
    for (int j = 0; j < 17; ++j) y[j] = y_in[j];
    float eta[3];
    rotors<false>(c, y, u, T.Fz, eta, &T.ctrl);
#pragma unroll
    for (int i = 0; i < 4; ++i) T.w[i] = y[13 + i];
    const float h = c.h;
    if (c.integrator == 1) {
        float k1[13];
        rhs(c, y, T.Fz, eta, k1);
#pragma unroll
        for (int j = 0; j < 13; ++j) T.yn[j] = y[j] + h * k1[j];
    } else {
        float k[13], acc[13];
        rhs(c, y, T.Fz, eta, k);
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            acc[j] = k[j];
            T.ys[0][j] = y[j] + 0.5f * h * k[j];
        }
        rhs(c, T.ys[0], T.Fz, eta, k);
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            acc[j] += 2.0f * k[j];
            T.ys[1][j] = y[j] + 0.5f * h * k[j];
        }
        rhs(c, T.ys[1], T.Fz, eta, k);
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            acc[j] += 2.0f * k[j];
            T.ys[2][j] = y[j] + h * k[j];
        }
        rhs(c, T.ys[2], T.Fz, eta, k);
#pragma unroll
        for (int j = 0; j < 13; ++j) T.yn[j] = y[j] + (h / 6.0f) * (acc[j] + k[j]);
    }
}

// A tape as kTapeWords columns of n agents (word f of agent a at f * n + a),
// so that a warp's stores and loads of one word are coalesced.
__device__ void tape_store(const StepTape& T, float* __restrict__ base, int n, int a) {
    unsigned bits = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        base[(size_t)i * n + a] = T.ctrl.fc[i];
        base[(size_t)(4 + i) * n + a] = T.ctrl.dw_df[i];
        bits |= (T.ctrl.in_f[i] ? 1u : 0u) << i;
        bits |= (T.ctrl.in_w[i] ? 1u : 0u) << (4 + i);
    }
    base[(size_t)8 * n + a] = __uint_as_float(bits);
    base[(size_t)9 * n + a] = T.Fz;
#pragma unroll
    for (int i = 0; i < 4; ++i) base[(size_t)(10 + i) * n + a] = T.w[i];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int j = 0; j < 13; ++j) base[(size_t)(14 + 13 * s + j) * n + a] = T.ys[s][j];
#pragma unroll
    for (int j = 0; j < 13; ++j) base[(size_t)(53 + j) * n + a] = T.yn[j];
}
__device__ void tape_load(StepTape& T, const float* __restrict__ base, int n, int a) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        T.ctrl.fc[i] = base[(size_t)i * n + a];
        T.ctrl.dw_df[i] = base[(size_t)(4 + i) * n + a];
    }
    const unsigned bits = __float_as_uint(base[(size_t)8 * n + a]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        T.ctrl.in_f[i] = (bits >> i) & 1u;
        T.ctrl.in_w[i] = (bits >> (4 + i)) & 1u;
    }
    T.Fz = base[(size_t)9 * n + a];
#pragma unroll
    for (int i = 0; i < 4; ++i) T.w[i] = base[(size_t)(10 + i) * n + a];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int j = 0; j < 13; ++j) T.ys[s][j] = base[(size_t)(14 + 13 * s + j) * n + a];
#pragma unroll
    for (int j = 0; j < 13; ++j) T.yn[j] = base[(size_t)(53 + j) * n + a];
}

// The state after the recorded sub-step, exactly as substep() leaves it.
__device__ __forceinline__ void substep_result(const StepTape& T, float y[17]) {
#pragma unroll
    for (int j = 0; j < 13; ++j) y[j] = T.yn[j];
    const float qn = rsqrtf(y[6] * y[6] + y[7] * y[7] + y[8] * y[8] + y[9] * y[9]);
#pragma unroll
    for (int j = 6; j < 10; ++j) y[j] *= qn;
#pragma unroll
    for (int i = 0; i < 4; ++i) y[13 + i] = T.w[i];
}

// Reverse sweep of one sub-step from its recorded forward pass.
__device__ void substep_reverse(const DynConsts& c, const float y_in[17], const float u[4], const StepTape& T,
                                const float gout[17], float gin[17], float gu[4]) {
    const CtrlTape& tape = T.ctrl;
    const float Fz = T.Fz;
    const float h = c.h;
    const float* ys[4] = {y_in, T.ys[0], T.ys[1], T.ys[2]};
    const float (&yn)[13] = T.yn;
    // normalisation q <- q / |q|
    float ybn[13];
#pragma unroll
    for (int j = 0; j < 13; ++j) ybn[j] = gout[j];
    {
        const float nq = sqrtf(yn[6] * yn[6] + yn[7] * yn[7] + yn[8] * yn[8] + yn[9] * yn[9]);
        const float inv = 1.0f / nq;
        float d = 0.0f;
#pragma unroll
        for (int j = 6; j < 10; ++j) d += yn[j] * inv * gout[j];
#pragma unroll
        for (int j = 6; j < 10; ++j) ybn[j] = (gout[j] - yn[j] * inv * d) * inv;
    }
    // integrator
    float yb[13];
    float Fzb = 0.0f, etab[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < 13; ++j) yb[j] = ybn[j];
    if (c.integrator == 1) {
        float kb[13], t[13];
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            kb[j] = h * ybn[j];
            t[j] = 0.0f;
        }
        rhs_vjp(c, ys[0], Fz, kb, t, Fzb, etab);
#pragma unroll
        for (int j = 0; j < 13; ++j) yb[j] += t[j];
    } else {
        float kb[13], t[13];
        // stage 4
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            kb[j] = (h / 6.0f) * ybn[j];
            t[j] = 0.0f;
        }
        rhs_vjp(c, ys[3], Fz, kb, t, Fzb, etab);
        // stage 3: kb3 = h/3 ybn + h * t4
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            yb[j] += t[j];
            kb[j] = (h / 3.0f) * ybn[j] + h * t[j];
            t[j] = 0.0f;
        }
        rhs_vjp(c, ys[2], Fz, kb, t, Fzb, etab);
        // stage 2: kb2 = h/3 ybn + h/2 * t3
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            yb[j] += t[j];
            kb[j] = (h / 3.0f) * ybn[j] + 0.5f * h * t[j];
            t[j] = 0.0f;
        }
        rhs_vjp(c, ys[1], Fz, kb, t, Fzb, etab);
        // stage 1: kb1 = h/6 ybn + h/2 * t2
#pragma unroll
        for (int j = 0; j < 13; ++j) {
            yb[j] += t[j];
            kb[j] = (h / 6.0f) * ybn[j] + 0.5f * h * t[j];
            t[j] = 0.0f;
        }
        rhs_vjp(c, ys[0], Fz, kb, t, Fzb, etab);
#pragma unroll
        for (int j = 0; j < 13; ++j) yb[j] += t[j];
    }
    // thrust and rotor lag
    float fb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float w = T.w[i];  // lagged rotor speed
        const float fbi = Fzb + c.mix[0][i] * etab[0] + c.mix[1][i] * etab[1] + c.mix[2][i] * etab[2];
        const float wb = gout[13 + i] + fbi * (2.0f * c.k2 * w + c.k1);
        gin[13 + i] = wb * c.decay;
        const float wdb = tape.in_w[i] ? wb * (1.0f - c.decay) : 0.0f;
        fb[i] = tape.in_f[i] ? wdb * tape.dw_df[i] : 0.0f;
    }
    if (c.controller == 1) {
        // SRT: f_i = (u_i + 1) / 2 * f(omega_max)
#pragma unroll
        for (int i = 0; i < 4; ++i) gu[i] += fb[i] * 0.5f * c.f_hi;
#pragma unroll
        for (int j = 0; j < 13; ++j) gin[j] = yb[j];
        return;
    }
    // controller: f = Ainv * rhs
    float rb[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) rb[r] = c.Ainv[0][r] * fb[0] + c.Ainv[1][r] * fb[1] + c.Ainv[2][r] * fb[2] + c.Ainv[3][r] * fb[3];
    gu[0] += rb[0] * c.half_a_max_m;
    const float* Om = y_in + 10;
    float L[3] = {c.J[0] * Om[0], c.J[1] * Om[1], c.J[2] * Om[2]};
    float cb[3] = {rb[1], rb[2], rb[3]};
    float t1[3], Lb[3];
    cross3(L, cb, t1);
    cross3(cb, Om, Lb);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        gu[j + 1] += cb[j] * c.JK[j] * c.rate_max[j];
        yb[10 + j] += -cb[j] * c.JK[j] + t1[j] + c.J[j] * Lb[j];
    }
#pragma unroll
    for (int j = 0; j < 13; ++j) gin[j] = yb[j];
}

// Reverse mode of one sub-step: its forward pass, then its reverse sweep.
__device__ void substep_vjp(const DynConsts& c, const float y_in[17], const float u[4], const float gout[17],
                            float gin[17], float gu[4]) {
    StepTape T;
    substep_record(c, y_in, u, T);
    substep_reverse(c, y_in, u, T, gout, gin, gu);
}

// Reverse mode of a full control step (n_sub sub-steps): the sub-step start
// states are recomputed into local memory first.
__device__ void control_step_vjp(const DynConsts& c, const float y_in[17], const float u[4], const float gout[17],
                                 float gin[17], float gu[4]) {
    float g[17];
#pragma unroll
    for (int j = 0; j < 17; ++j) g[j] = gout[j];
    if (c.n_sub == 1) {
        substep_vjp(c, y_in, u, g, gin, gu);
        return;
    }
    float ys[kMaxSub][17];
#pragma unroll
    for (int j = 0; j < 17; ++j) ys[0][j] = y_in[j];
    for (int s = 1; s < c.n_sub; ++s) {
#pragma unroll
        for (int j = 0; j < 17; ++j) ys[s][j] = ys[s - 1][j];
        substep(c, ys[s], u);
    }
    for (int s = c.n_sub - 1; s >= 0; --s) {
        float gi[17];
        substep_vjp(c, ys[s], u, g, gi, gu);
#pragma unroll
        for (int j = 0; j < 17; ++j) g[j] = gi[j];
    }
#pragma unroll
    for (int j = 0; j < 17; ++j) gin[j] = g[j];
}

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ void load_state(const float* __restrict__ s, int n, int a, float y[17]) {
#pragma unroll
    for (int j = 0; j < 17; ++j) y[j] = s[(size_t)j * n + a];
}
__device__ __forceinline__ void store_state(float* __restrict__ s, int n, int a, const float y[17]) {
#pragma unroll
    for (int j = 0; j < 17; ++j) s[(size_t)j * n + a] = y[j];
}
__device__ __forceinline__ void load_cmd(const float* __restrict__ u_, int n, int a, float u[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = u_[(size_t)j * n + a];
}

template <bool GEO>
__global__ void __launch_bounds__(128) step_kernel(DynConsts c, int n, float* state, const float* __restrict__ cmd,
                                                   float* __restrict__ ckpt) {
    // a render launched next as a programmatic dependent may start its
    // prologue now; it waits for this grid to finish before reading the state
    asm volatile("griddepcontrol.launch_dependents;");
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    float y[17], u[4];
    load_state(state, n, a, y);
    load_cmd(cmd, n, a, u);
    if (ckpt) store_state(ckpt, n, a, y);
    control_step<GEO>(c, y, u);
    store_state(state, n, a, y);
}

__global__ void __launch_bounds__(128) step_backward_kernel(DynConsts c, int n, const float* __restrict__ state_in,
                                                            const float* __restrict__ cmd,
                                                            const float* __restrict__ g_out,
                                                            float* __restrict__ g_in, float* __restrict__ g_cmd) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    float y[17], u[4], go[17], gi[17], gu[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    load_state(state_in, n, a, y);
    load_cmd(cmd, n, a, u);
    load_state(g_out, n, a, go);
    control_step_vjp(c, y, u, go, gi, gu);
    store_state(g_in, n, a, gi);
#pragma unroll
    for (int j = 0; j < 4; ++j) g_cmd[(size_t)j * n + a] = gu[j];
}

template <bool GEO>
__global__ void __launch_bounds__(128) rollout_kernel(DynConsts c, int n, int T, int K,
                                                      const float* __restrict__ state0,
                                                      const float* __restrict__ cmds, float* __restrict__ states_out,
                                                      float* __restrict__ ckpt, float* __restrict__ state_final) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    float y[17], u[4];
    load_state(state0, n, a, y);
    if (states_out) store_state(states_out, n, a, y);
    for (int t = 0; t < T; ++t) {
        if (ckpt && t % K == 0) store_state(ckpt + (size_t)(t / K) * 17 * n, n, a, y);
        load_cmd(cmds + (size_t)t * 4 * n, n, a, u);
        control_step<GEO>(c, y, u);
        if (states_out) store_state(states_out + (size_t)(t + 1) * 17 * n, n, a, y);
    }
    if (state_final) store_state(state_final, n, a, y);
}

// Rollout adjoint with recompute from checkpoints: segment s covers steps
// [sK, min(sK+K, T)); its states are re-run from ckpt[s] into local memory and
// swept backwards.  g_states[t] is added to the running cotangent of state t.
__global__ void __launch_bounds__(64) rollout_backward_kernel(DynConsts c, int n, int T, int K,
                                                              const float* __restrict__ ckpt,
                                                              const float* __restrict__ cmds,
                                                              const float* __restrict__ g_states,
                                                              float* __restrict__ g_state0,
                                                              float* __restrict__ g_cmds, float* __restrict__ tape) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    float seg[kMaxCkptK][17];
    // with one sub-step per control step, and tape memory given, the
    // segment's forward passes are recorded while the segment is recomputed,
    // so the reverse sweep does not run them a second time
    const bool taped = tape != nullptr && c.n_sub == 1;
    float g[17];
    load_state(g_states + (size_t)T * 17 * n, n, a, g);
    const int nseg = (T + K - 1) / K;
    for (int s = nseg - 1; s >= 0; --s) {
        const int t0 = s * K;
        const int t1 = min(t0 + K, T);
        load_state(ckpt + (size_t)s * 17 * n, n, a, seg[0]);
        for (int t = t0 + 1; t < (taped ? t1 + 1 : t1); ++t) {
            float u[4];
            load_cmd(cmds + (size_t)(t - 1) * 4 * n, n, a, u);
            if (taped) {
                StepTape rec;
                substep_record(c, seg[t - 1 - t0], u, rec);
                tape_store(rec, tape + (size_t)(t - 1 - t0) * kTapeWords * n, n, a);
                if (t < t1) substep_result(rec, seg[t - t0]);
            } else {
#pragma unroll
                for (int j = 0; j < 17; ++j) seg[t - t0][j] = seg[t - t0 - 1][j];
                control_step(c, seg[t - t0], u);
            }
        }
        for (int t = t1 - 1; t >= t0; --t) {
            float u[4], gi[17], gu[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            load_cmd(cmds + (size_t)t * 4 * n, n, a, u);
            if (taped) {
                StepTape rec;
                tape_load(rec, tape + (size_t)(t - t0) * kTapeWords * n, n, a);
                substep_reverse(c, seg[t - t0], u, rec, g, gi, gu);
            } else {
                control_step_vjp(c, seg[t - t0], u, g, gi, gu);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) g_cmds[((size_t)t * 4 + j) * n + a] = gu[j];
            float gs[17];
            load_state(g_states + (size_t)t * 17 * n, n, a, gs);
#pragma unroll
            for (int j = 0; j < 17; ++j) g[j] = gi[j] + gs[j];
        }
    }
    store_state(g_state0, n, a, g);
}

inline unsigned blocks_for(int n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_step(const DynConsts& c, int n, float* state, const float* cmd, float* ckpt, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (c.controller >= 2) step_kernel<true><<<blocks_for(n, 128), 128, 0, s>>>(c, n, state, cmd, ckpt);
    else step_kernel<false><<<blocks_for(n, 128), 128, 0, s>>>(c, n, state, cmd, ckpt);
    return cudaGetLastError();
}

cudaError_t launch_step_backward(const DynConsts& c, int n, const float* state_in, const float* cmd,
                                 const float* g_out, float* g_in, float* g_cmd, cudaStream_t s) {
    if (c.controller >= 2) return cudaErrorInvalidValue;  // the adjoint kernels carry the CTBR and SRT laws only
    if (n == 0) return cudaSuccess;
    step_backward_kernel<<<blocks_for(n, 128), 128, 0, s>>>(c, n, state_in, cmd, g_out, g_in, g_cmd);
    return cudaGetLastError();
}

cudaError_t launch_rollout(const DynConsts& c, int n, int T, int K, const float* state0, const float* cmds,
                           float* states_out, float* ckpt, float* state_final, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (c.controller >= 2)
        rollout_kernel<true><<<blocks_for(n, 128), 128, 0, s>>>(c, n, T, K, state0, cmds, states_out, ckpt, state_final);
    else
        rollout_kernel<false><<<blocks_for(n, 128), 128, 0, s>>>(c, n, T, K, state0, cmds, states_out, ckpt,
                                                                 state_final);
    return cudaGetLastError();
}

size_t rollout_tape_bytes(int n, int K) { return sizeof(float) * kTapeWords * (size_t)K * (size_t)n; }

cudaError_t launch_rollout_backward(const DynConsts& c, int n, int T, int K, const float* ckpt, const float* cmds,
                                    const float* g_states, float* g_state0, float* g_cmds, float* tape,
                                    cudaStream_t s) {
    if (c.controller >= 2) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    rollout_backward_kernel<<<blocks_for(n, 64), 64, 0, s>>>(c, n, T, K, ckpt, cmds, g_states, g_state0, g_cmds,
                                                             tape);
    return cudaGetLastError();
}

}  // namespace vf

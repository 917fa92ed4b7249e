// FP64 CPU oracle for the VisFly rollout-step hot path.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
// CUDA path is checked against.  Only the test suite, the package smoke check
// and the benchmark's CPU-baseline leg may load it; the product library never
// links or calls it, and it shares no code, header or constant with the CUDA
// sources.  Every value it needs arrives as an argument.
//
// What it computes (paper sections and equations in brackets):
//   * one control step of N quadrotors [Sec. III-A, Eq. 1-4]:
//       controller (body rate CTBR, single-rotor thrust SRT, or geometric
//       linear-velocity LV / position PS control after Lee et al.) ->
//       rotor first-order lag [Eq. 4] -> thrust and moment [Eq. 3] -> RK4 (or
//       Euler) on the rigid body [Eq. 1] with quadratic body-frame drag
//       [Eq. 2] -> quaternion normalisation;
//   * the closest-hit depth / colour / triangle-id image of every agent's
//     pinhole camera over a triangle mesh [Sec. III-B] (Moller-Trumbore,
//     brute force or a median-split BVH of its own);
//   * exact forward-mode (dual number) derivatives of the step map and of a
//     rollout loss, for checking the hand-written adjoint [Sec. III-A: the
//     dynamics are differentiable];
//   * the nearest point of a scene's mesh to each agent [Sec. III-B, the
//     obstacle-distance module], by brute force over every triangle with
//     Ericson's closest point on a triangle (Voronoi regions).
//
// Readings of points the paper leaves open (drag sign, moment-arm meaning,
// frame layout, constants, camera convention, ties) are the ones listed in the
// design notes; they are implemented here literally and commented in place.
//
// Parity: every function below is pinned by closed-form tests (hover
// equilibrium, free fall, drag terminal velocity, rate-loop response, rotor
// lag, constant-rate rotation, torque-free symmetric top, RK4 order, analytic
// plane / box / sphere depths, brute force vs BVH, finite differences,
// controller equilibria and step responses, rotation equivariance, box and
// room distances).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
// Field order is mirrored by the ctypes structure in oracle/__init__.py.
struct OracleParams {
    double mass;
    double J[3];
    double arm;
    double k[3];          // thrust polynomial k0, k1, k2
    double c_lag;         // rotor time-decay constant c
    double kappa;         // rotor torque / thrust ratio
    double rho;
    double Cd[3];
    double area[3];
    double omega_min, omega_max;
    double a_max;
    double rate_max[3];
    double K_rate[3];
    double g;
    double dt;
    int32_t n_sub;
    int32_t integrator;   // 0 = RK4, 1 = explicit Euler
    int32_t width, height;
    double fov_deg;
    double max_depth;
    double cam_off[3];
    int32_t controller;   // 0 CTBR, 1 SRT, 2 LV, 3 PS
    double K_pos[3], K_vel[3], K_att[3], K_omega[3];
};
}

namespace {

// ---------------------------------------------------------------- dual numbers
struct Dual {
    double v, d;
    Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
inline Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
inline Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
inline Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
inline Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
inline Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
inline Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double s_sqrt(double x) { return std::sqrt(x); }
inline Dual s_sqrt(const Dual& x) {
    const double r = std::sqrt(x.v);
    if (r == 0.0) return {0.0, x.d == 0.0 ? 0.0 : std::numeric_limits<double>::infinity()};
    return {r, x.d / (2.0 * r)};
}
inline double s_cos(double x) { return std::cos(x); }
inline double s_sin(double x) { return std::sin(x); }
inline Dual s_cos(const Dual& x) { return {std::cos(x.v), -std::sin(x.v) * x.d}; }
inline Dual s_sin(const Dual& x) { return {std::sin(x.v), std::cos(x.v) * x.d}; }
inline double s_abs(double x) { return std::fabs(x); }
inline Dual s_abs(const Dual& x) { return x.v < 0.0 ? -x : x; }

// clamp with unit slope inside [lo, hi] (boundaries count as inside) and zero
// slope outside.
template <class S>
inline S s_clamp(const S& x, double lo, double hi) {
    if (val(x) < lo) return S(lo);
    if (val(x) > hi) return S(hi);
    return x;
}

// ------------------------------------------------------------- quad geometry
// X layout: rotor i at azimuth 45 + 90 i degrees in the body x-y plane, spin
// directions +1, -1, +1, -1 (diagonal pairs turn the same way).
inline void rotor_arm(const OracleParams& p, int i, double& rx, double& ry) {
    const double th = (45.0 + 90.0 * i) * M_PI / 180.0;
    rx = p.arm * std::cos(th);
    ry = p.arm * std::sin(th);
}
inline double rotor_spin(int i) { return (i % 2 == 0) ? 1.0 : -1.0; }

// Rotor thrust along body z [Eq. 4, first part].
template <class S>
inline S rotor_thrust(const OracleParams& p, const S& w) {
    return p.k[2] * w * w + p.k[1] * w + p.k[0];
}

// Rotor speed that produces thrust f: the non-negative root of the Eq. 4
// polynomial (linear case when k2 = 0).
template <class S>
inline S rotor_speed_for_thrust(const OracleParams& p, const S& f) {
    if (p.k[2] == 0.0) return (f - p.k[0]) / p.k[1];
    S disc = p.k[1] * p.k[1] - 4.0 * p.k[2] * (p.k[0] - f);
    if (val(disc) < 0.0) disc = S(0.0);
    return (-p.k[1] + s_sqrt(disc)) / (2.0 * p.k[2]);
}

// Mixer matrix A mapping the four rotor thrusts to (collective thrust,
// body moment) [Eq. 3]: the moment of rotor i is the arm cross product
// r_i x (0, 0, f_i) = (r_iy f_i, -r_ix f_i, 0) plus the rotor reaction torque
// s_i kappa f_i about body z.
inline void mixer_matrix(const OracleParams& p, double A[4][4]) {
    for (int i = 0; i < 4; ++i) {
        double rx, ry;
        rotor_arm(p, i, rx, ry);
        A[0][i] = 1.0;
        A[1][i] = ry;
        A[2][i] = -rx;
        A[3][i] = rotor_spin(i) * p.kappa;
    }
}

// Solve A f = b by Gaussian elimination with partial pivoting (A is constant).
template <class S>
void solve4(const double Ain[4][4], const S bin[4], S f[4]) {
    double A[4][4];
    S b[4];
    for (int r = 0; r < 4; ++r) {
        for (int c = 0; c < 4; ++c) A[r][c] = Ain[r][c];
        b[r] = bin[r];
    }
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
        if (piv != col) {
            for (int c = 0; c < 4; ++c) std::swap(A[col][c], A[piv][c]);
            std::swap(b[col], b[piv]);
        }
        for (int r = col + 1; r < 4; ++r) {
            const double m = A[r][col] / A[col][col];
            for (int c = col; c < 4; ++c) A[r][c] -= m * A[col][c];
            b[r] = b[r] - m * b[col];
        }
    }
    for (int r = 3; r >= 0; --r) {
        S acc = b[r];
        for (int c = r + 1; c < 4; ++c) acc = acc - A[r][c] * f[c];
        f[r] = acc / A[r][r];
    }
}

// Thrust allocation shared by the controllers: solve A f = (collective
// thrust, body moment) for the four rotor thrusts, clamp each to the
// reachable range and convert to desired rotor speeds.
template <class S>
void allocate(const OracleParams& p, const S rhs[4], S omega_des[4]) {
    double A[4][4];
    mixer_matrix(p, A);
    S f[4];
    solve4(A, rhs, f);
    const double f_lo = rotor_thrust(p, p.omega_min);
    const double f_hi = rotor_thrust(p, p.omega_max);
    for (int i = 0; i < 4; ++i) {
        const S fi = s_clamp(f[i], f_lo, f_hi);
        omega_des[i] = s_clamp(rotor_speed_for_thrust(p, fi), p.omega_min, p.omega_max);
    }
}

// Body-rate (CTBR) controller [Sec. III-A, controllers; Sec. IV: CTBR is the
// action type of all examples].  u[0] in [-1, 1] maps to a mass-normalised
// collective thrust (u0 + 1) / 2 * a_max; u[1..3] scale to desired body rates.
// A proportional rate loop with gyroscopic feed-forward gives the desired
// moment; the allocation gives desired rotor speeds.
template <class S>
void controller_ctbr(const OracleParams& p, const S Om[3], const S u[4], S omega_des[4]) {
    const S a = (u[0] + 1.0) * 0.5 * p.a_max;
    S JOm[3], gyro[3], rhs[4];
    for (int j = 0; j < 3; ++j) JOm[j] = p.J[j] * Om[j];
    gyro[0] = Om[1] * JOm[2] - Om[2] * JOm[1];
    gyro[1] = Om[2] * JOm[0] - Om[0] * JOm[2];
    gyro[2] = Om[0] * JOm[1] - Om[1] * JOm[0];
    rhs[0] = p.mass * a;
    for (int j = 0; j < 3; ++j) {
        const S om_des = u[j + 1] * p.rate_max[j];
        rhs[j + 1] = p.J[j] * p.K_rate[j] * (om_des - Om[j]) + gyro[j];
    }
    allocate(p, rhs, omega_des);
}

// Single-rotor thrusts (SRT) [Sec. III-A]: u_i in [-1, 1] maps to rotor i's
// thrust (u_i + 1) / 2 * f(omega_max), clamped, converted to a rotor speed.
template <class S>
void controller_srt(const OracleParams& p, const S u[4], S omega_des[4]) {
    const double f_lo = rotor_thrust(p, p.omega_min);
    const double f_hi = rotor_thrust(p, p.omega_max);
    for (int i = 0; i < 4; ++i) {
        const S fi = s_clamp((u[i] + 1.0) * 0.5 * f_hi, f_lo, f_hi);
        omega_des[i] = s_clamp(rotor_speed_for_thrust(p, fi), p.omega_min, p.omega_max);
    }
}

template <class S>
void rotation_matrix(const S q[4], S R[3][3]);

// Linear-velocity (LV) and position (PS) commands with yaw [Sec. III-A, after
// the geometric controller of Lee et al. 2010], world z up:
//   desired acceleration  a_d = -K_pos (x - x_d) - K_vel v           (PS)
//                         a_d = -K_vel (v - v_d)                     (LV)
//   desired force F_d = m (a_d + g z); collective thrust = F_d . (R z_B);
//   desired attitude R_d = [b1 b2 b3]: b3 = F_d / |F_d| (z when |F_d| = 0),
//   b2 = b3 x c1 / |b3 x c1| with c1 = (cos yaw_d, sin yaw_d, 0) (or
//   (-sin, cos, 0) when b3 x c1 vanishes), b1 = b2 x b3;
//   attitude error e_R = vee(R_d^T R - R^T R_d) / 2, rate error e_W = Omega;
//   moment = J (-K_att e_R - K_omega e_W) + Omega x J Omega;
// then the same allocation as CTBR.  u = (x_d or v_d, yaw_d) in m, m/s, rad.
template <class S>
void controller_geometric(const OracleParams& p, const S y[17], const S u[4], bool position, S omega_des[4]) {
    const S* x = y;
    const S* v = y + 3;
    const S* Om = y + 10;
    S R[3][3];
    rotation_matrix(y + 6, R);
    S F[3];
    for (int j = 0; j < 3; ++j) {
        const S acc = position ? (-p.K_pos[j] * (x[j] - u[j]) - p.K_vel[j] * v[j]) : (-p.K_vel[j] * (v[j] - u[j]));
        F[j] = p.mass * acc;
    }
    F[2] = F[2] + p.mass * p.g;
    const S f_coll = F[0] * R[0][2] + F[1] * R[1][2] + F[2] * R[2][2];
    const S nF = s_sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    S b3[3];
    if (val(nF) < 1e-9) {
        b3[0] = S(0.0);
        b3[1] = S(0.0);
        b3[2] = S(1.0);
    } else {
        for (int j = 0; j < 3; ++j) b3[j] = F[j] / nF;
    }
    S c1[3] = {s_cos(u[3]), s_sin(u[3]), S(0.0)};
    auto cross = [](const S a[3], const S b[3], S c[3]) {
        c[0] = a[1] * b[2] - a[2] * b[1];
        c[1] = a[2] * b[0] - a[0] * b[2];
        c[2] = a[0] * b[1] - a[1] * b[0];
    };
    S b2[3];
    cross(b3, c1, b2);
    S n2 = s_sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
    if (val(n2) < 1e-6) {
        S c1b[3] = {-s_sin(u[3]), s_cos(u[3]), S(0.0)};
        cross(b3, c1b, b2);
        n2 = s_sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
    }
    for (int j = 0; j < 3; ++j) b2[j] = b2[j] / n2;
    S b1[3];
    cross(b2, b3, b1);
    S Rd[3][3];
    for (int i = 0; i < 3; ++i) {
        Rd[i][0] = b1[i];
        Rd[i][1] = b2[i];
        Rd[i][2] = b3[i];
    }
    // M = Rd^T R - R^T Rd (skew-symmetric); e_R = vee(M) / 2
    S M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            S a(0.0), b(0.0);
            for (int k = 0; k < 3; ++k) {
                a = a + Rd[k][i] * R[k][j];
                b = b + R[k][i] * Rd[k][j];
            }
            M[i][j] = a - b;
        }
    const S eR[3] = {0.5 * M[2][1], 0.5 * M[0][2], 0.5 * M[1][0]};
    S JOm[3], gyro[3], rhs[4];
    for (int j = 0; j < 3; ++j) JOm[j] = p.J[j] * Om[j];
    cross(Om, JOm, gyro);
    rhs[0] = f_coll;
    for (int j = 0; j < 3; ++j) rhs[j + 1] = p.J[j] * (-p.K_att[j] * eR[j] - p.K_omega[j] * Om[j]) + gyro[j];
    allocate(p, rhs, omega_des);
}

template <class S>
void controller(const OracleParams& p, const S y[17], const S u[4], S omega_des[4]) {
    switch (p.controller) {
        case 1: controller_srt(p, u, omega_des); break;
        case 2: controller_geometric(p, y, u, false, omega_des); break;
        case 3: controller_geometric(p, y, u, true, omega_des); break;
        default: controller_ctbr(p, y + 10, u, omega_des); break;
    }
}

// Rotation body -> world of the unit quaternion q / |q|, q = (w, x, y, z).
template <class S>
void rotation_matrix(const S q[4], S R[3][3]) {
    const S w = q[0], x = q[1], y = q[2], z = q[3];
    const S n = w * w + x * x + y * y + z * z;
    R[0][0] = (w * w + x * x - y * y - z * z) / n;
    R[0][1] = 2.0 * (x * y - w * z) / n;
    R[0][2] = 2.0 * (x * z + w * y) / n;
    R[1][0] = 2.0 * (x * y + w * z) / n;
    R[1][1] = (w * w - x * x + y * y - z * z) / n;
    R[1][2] = 2.0 * (y * z - w * x) / n;
    R[2][0] = 2.0 * (x * z - w * y) / n;
    R[2][1] = 2.0 * (y * z + w * x) / n;
    R[2][2] = (w * w - x * x - y * y + z * z) / n;
}

// Right-hand side of Eq. 1 for y = (x, v, q, Omega) with the body thrust
// (0, 0, Fz) and moment eta held fixed.  Drag [Eq. 2] opposes the body-frame
// velocity: d = -1/2 rho Cd * s * v_B * |v_B| component-wise.
template <class S>
void rigid_body_rhs(const OracleParams& p, const S y[13], const S& Fz, const S eta[3], S dy[13]) {
    const S* v = y + 3;
    const S* q = y + 6;
    const S* Om = y + 10;
    S R[3][3];
    rotation_matrix(q, R);
    S vB[3], fB[3];
    for (int j = 0; j < 3; ++j) vB[j] = R[0][j] * v[0] + R[1][j] * v[1] + R[2][j] * v[2];
    for (int j = 0; j < 3; ++j) fB[j] = -0.5 * p.rho * p.Cd[j] * p.area[j] * vB[j] * s_abs(vB[j]);
    fB[2] = fB[2] + Fz;
    for (int j = 0; j < 3; ++j) dy[j] = v[j];
    for (int j = 0; j < 3; ++j) dy[3 + j] = (R[j][0] * fB[0] + R[j][1] * fB[1] + R[j][2] * fB[2]) / p.mass;
    dy[5] = dy[5] - p.g;
    // 1/2 q (x) (0, Omega), Hamilton product
    dy[6] = 0.5 * (-q[1] * Om[0] - q[2] * Om[1] - q[3] * Om[2]);
    dy[7] = 0.5 * (q[0] * Om[0] + q[2] * Om[2] - q[3] * Om[1]);
    dy[8] = 0.5 * (q[0] * Om[1] - q[1] * Om[2] + q[3] * Om[0]);
    dy[9] = 0.5 * (q[0] * Om[2] + q[1] * Om[1] - q[2] * Om[0]);
    S JOm[3];
    for (int j = 0; j < 3; ++j) JOm[j] = p.J[j] * Om[j];
    const S c0 = Om[1] * JOm[2] - Om[2] * JOm[1];
    const S c1 = Om[2] * JOm[0] - Om[0] * JOm[2];
    const S c2 = Om[0] * JOm[1] - Om[1] * JOm[0];
    dy[10] = (eta[0] - c0) / p.J[0];
    dy[11] = (eta[1] - c1) / p.J[1];
    dy[12] = (eta[2] - c2) / p.J[2];
}

// One control step of one agent, state y = (x, v, q, Omega, omega_1..4).
// Each of n_sub physics sub-steps of length h = dt / n_sub: controller ->
// rotor lag over h (exact solution of the first-order lag, Eq. 4 with t = h)
// -> thrust and moment from the lagged rotor speeds, held over the sub-step
// -> RK4 (or Euler) on (x, v, q, Omega) -> q normalised.
template <class S>
void step_agent(const OracleParams& p, S y[17], const S u[4]) {
    const double h = p.dt / p.n_sub;
    const double decay = std::exp(-p.c_lag * h);
    double rx[4], ry[4];
    for (int i = 0; i < 4; ++i) rotor_arm(p, i, rx[i], ry[i]);
    for (int sub = 0; sub < p.n_sub; ++sub) {
        S omega_des[4];
        controller(p, y, u, omega_des);
        for (int i = 0; i < 4; ++i) y[13 + i] = omega_des[i] + (y[13 + i] - omega_des[i]) * decay;
        S Fz(0.0), eta[3] = {S(0.0), S(0.0), S(0.0)};
        for (int i = 0; i < 4; ++i) {
            const S fi = rotor_thrust(p, y[13 + i]);
            Fz = Fz + fi;
            eta[0] = eta[0] + ry[i] * fi;
            eta[1] = eta[1] - rx[i] * fi;
            eta[2] = eta[2] + rotor_spin(i) * p.kappa * fi;
        }
        if (p.integrator == 1) {
            S k1[13];
            rigid_body_rhs(p, y, Fz, eta, k1);
            for (int j = 0; j < 13; ++j) y[j] = y[j] + h * k1[j];
        } else {
            S k1[13], k2[13], k3[13], k4[13], yt[13];
            rigid_body_rhs(p, y, Fz, eta, k1);
            for (int j = 0; j < 13; ++j) yt[j] = y[j] + 0.5 * h * k1[j];
            rigid_body_rhs(p, yt, Fz, eta, k2);
            for (int j = 0; j < 13; ++j) yt[j] = y[j] + 0.5 * h * k2[j];
            rigid_body_rhs(p, yt, Fz, eta, k3);
            for (int j = 0; j < 13; ++j) yt[j] = y[j] + h * k3[j];
            rigid_body_rhs(p, yt, Fz, eta, k4);
            for (int j = 0; j < 13; ++j)
                y[j] = y[j] + (h / 6.0) * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
        }
        const S qn = s_sqrt(y[6] * y[6] + y[7] * y[7] + y[8] * y[8] + y[9] * y[9]);
        for (int j = 6; j < 10; ++j) y[j] = y[j] / qn;
    }
}

// ------------------------------------------------------------------- scenes
struct Tri {
    double v0[3], v1[3], v2[3];
    double lo[3], hi[3];
};

struct BvhNode {
    double lo[3], hi[3];
    int32_t left, right;   // children; -1 for a leaf
    int32_t first, count;  // leaf range into OracleScene::order
};

struct OracleScene {
    std::vector<Tri> tris;
    std::vector<uint8_t> rgb;
    std::vector<BvhNode> nodes;
    std::vector<int32_t> order;
};

void bvh_build(OracleScene& s, int32_t first, int32_t count, int depth) {
    BvhNode node;
    for (int j = 0; j < 3; ++j) {
        node.lo[j] = std::numeric_limits<double>::infinity();
        node.hi[j] = -std::numeric_limits<double>::infinity();
    }
    double clo[3], chi[3];
    for (int j = 0; j < 3; ++j) {
        clo[j] = std::numeric_limits<double>::infinity();
        chi[j] = -std::numeric_limits<double>::infinity();
    }
    for (int32_t i = first; i < first + count; ++i) {
        const Tri& t = s.tris[s.order[i]];
        for (int j = 0; j < 3; ++j) {
            node.lo[j] = std::min(node.lo[j], t.lo[j]);
            node.hi[j] = std::max(node.hi[j], t.hi[j]);
            const double c = 0.5 * (t.lo[j] + t.hi[j]);
            clo[j] = std::min(clo[j], c);
            chi[j] = std::max(chi[j], c);
        }
    }
    node.left = node.right = -1;
    node.first = first;
    node.count = count;
    const int32_t me = (int32_t)s.nodes.size();
    s.nodes.push_back(node);
    if (count <= 4 || depth > 60) return;
    int axis = 0;
    for (int j = 1; j < 3; ++j)
        if (chi[j] - clo[j] > chi[axis] - clo[axis]) axis = j;
    const int32_t mid = first + count / 2;
    std::nth_element(s.order.begin() + first, s.order.begin() + mid, s.order.begin() + first + count,
                     [&](int32_t a, int32_t b) {
                         const double ca = s.tris[a].lo[axis] + s.tris[a].hi[axis];
                         const double cb = s.tris[b].lo[axis] + s.tris[b].hi[axis];
                         return ca < cb || (ca == cb && a < b);
                     });
    const int32_t l = (int32_t)s.nodes.size();
    bvh_build(s, first, mid - first, depth + 1);
    const int32_t r = (int32_t)s.nodes.size();
    bvh_build(s, mid, first + count - mid, depth + 1);
    s.nodes[me].left = l;
    s.nodes[me].right = r;
    s.nodes[me].count = 0;
}

// Candidate filter: a triangle can matter for a ray only if the ray enters its
// AABB grown by kGrow metres before t_lim.  The same test runs in the brute
// force and in the BVH walk, so both see identical candidate sets.
constexpr double kGrow = 1e-3;
// Relative band used to call a pixel ambiguous (see classify()).  FP32
// Moller-Trumbore errors in u, v are a few eps_f32 (6e-8) times sigma; the
// band is about 50 eps_f32 * sigma, ten times that estimate.
constexpr double kTau = 3e-6;
// Closest accepted hit distance (rays start at the camera centre).
constexpr double kTmin = 1e-6;

inline bool ray_box(const double o[3], const double inv[3], const double lo[3], const double hi[3],
                    double t_lim) {
    double t0 = 0.0, t1 = t_lim;
    for (int j = 0; j < 3; ++j) {
        double a = (lo[j] - kGrow - o[j]) * inv[j];
        double b = (hi[j] + kGrow - o[j]) * inv[j];
        if (std::isnan(a) || std::isnan(b)) {  // direction component zero, origin on the slab plane
            if (o[j] < lo[j] - kGrow || o[j] > hi[j] + kGrow) return false;
            continue;
        }
        if (a > b) std::swap(a, b);
        t0 = std::max(t0, a);
        t1 = std::min(t1, b);
        if (t0 > t1) return false;
    }
    return true;
}

// Moller-Trumbore ray / triangle evaluation (two-sided).  Returns false when
// the ray is parallel to the plane.  Otherwise t, the barycentric margin
// m = min(u, v, 1 - u - v) (m >= 0 means inside, edges inclusive) and sigma,
// a dimensionless conditioning scale of the intersection: the reciprocal of
// (sin of the corner angle * |cos| of the incidence angle), times
// (1 + |o - v0| / shortest edge).  FP32 evaluations of u, v carry errors of
// order eps_f32 * sigma, which is what the ambiguity band is scaled by.
struct Hit {
    double t, m, sigma;
};
inline bool moller_trumbore(const double o[3], const double d[3], const Tri& tr, Hit& h) {
    double e1[3], e2[3], pv[3], sv[3], qv[3];
    for (int j = 0; j < 3; ++j) {
        e1[j] = tr.v1[j] - tr.v0[j];
        e2[j] = tr.v2[j] - tr.v0[j];
        sv[j] = o[j] - tr.v0[j];
    }
    pv[0] = d[1] * e2[2] - d[2] * e2[1];
    pv[1] = d[2] * e2[0] - d[0] * e2[2];
    pv[2] = d[0] * e2[1] - d[1] * e2[0];
    const double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
    if (det == 0.0) return false;
    const double inv = 1.0 / det;
    const double u = (sv[0] * pv[0] + sv[1] * pv[1] + sv[2] * pv[2]) * inv;
    qv[0] = sv[1] * e1[2] - sv[2] * e1[1];
    qv[1] = sv[2] * e1[0] - sv[0] * e1[2];
    qv[2] = sv[0] * e1[1] - sv[1] * e1[0];
    const double v = (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]) * inv;
    h.t = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
    h.m = std::min(std::min(u, v), 1.0 - u - v);
    auto norm = [](const double a[3]) { return std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); };
    double e3[3] = {e2[0] - e1[0], e2[1] - e1[1], e2[2] - e1[2]};
    const double l1 = norm(e1), l2 = norm(e2), l3 = norm(e3);
    const double kappa = norm(d) * l1 * l2 / std::fabs(det);
    h.sigma = kappa * (1.0 + norm(sv) / std::min(l1, std::min(l2, l3)));
    return true;
}

struct Cand {
    int32_t id;
    Hit h;
};

void collect_candidates(const OracleScene& s, const double o[3], const double d[3], double t_lim, bool use_bvh,
                        std::vector<Cand>& out) {
    out.clear();
    double inv[3];
    for (int j = 0; j < 3; ++j) inv[j] = 1.0 / d[j];
    auto consider = [&](int32_t id) {
        const Tri& t = s.tris[id];
        if (!ray_box(o, inv, t.lo, t.hi, t_lim)) return;
        Cand c;
        c.id = id;
        if (moller_trumbore(o, d, t, c.h)) out.push_back(c);
    };
    if (!use_bvh) {
        for (int32_t id = 0; id < (int32_t)s.tris.size(); ++id) consider(id);
        return;
    }
    if (s.nodes.empty()) return;
    std::vector<int32_t> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        const BvhNode& n = s.nodes[stack.back()];
        stack.pop_back();
        if (!ray_box(o, inv, n.lo, n.hi, t_lim)) continue;
        if (n.left < 0) {
            for (int32_t i = n.first; i < n.first + n.count; ++i) consider(s.order[i]);
        } else {
            stack.push_back(n.left);
            stack.push_back(n.right);
        }
    }
}

// Camera convention: camera at body-frame offset cam_off looking along body
// +x; image right is body -y and image down is body -z.  Pixel (r, c) has its
// centre at (c + 0.5, r + 0.5); the body-frame direction is
// (1, -(2c + 1 - W) / W * tan(fov/2), -(2r + 1 - H) / W * tan(fov/2)), not
// normalised, so the hit distance t along it is the planar depth along the
// optical axis.
void camera_ray(const OracleParams& p, const double* st, int r, int c, double o[3], double d[3]) {
    double q[4] = {st[6], st[7], st[8], st[9]};
    double R[3][3];
    rotation_matrix(q, R);
    const double th = std::tan(0.5 * p.fov_deg * M_PI / 180.0);
    const double dB[3] = {1.0, -(2.0 * c + 1.0 - p.width) / p.width * th,
                          -(2.0 * r + 1.0 - p.height) / p.width * th};
    for (int j = 0; j < 3; ++j) {
        o[j] = st[j] + R[j][0] * p.cam_off[0] + R[j][1] * p.cam_off[1] + R[j][2] * p.cam_off[2];
        d[j] = R[j][0] * dB[0] + R[j][1] * dB[1] + R[j][2] * dB[2];
    }
}

// Per-pixel result and ambiguity classification.
//   hit: candidates with m >= 0 and kTmin < t <= max_depth; the closest t wins,
//        equal t broken by the lowest triangle id.
//   ambiguous (a "stated tie") when any of:
//     (a) the winning hit lies within the band of an edge: m < kTau * sigma;
//     (b) another candidate that is hit or nearly hit (m > -kTau * sigma) lies
//         no farther than t_hit * (1 + kTau) (or anywhere up to the range end
//         when nothing is hit);
//     (c) the winning hit, or any nearly hit candidate, lies within
//         kTau * max_depth of the range end.
struct PixelResult {
    int32_t id;
    double t;
    uint8_t tie;
};

PixelResult classify(const std::vector<Cand>& cands, double max_depth) {
    PixelResult r{-1, max_depth, 0};
    int best = -1;
    for (int i = 0; i < (int)cands.size(); ++i) {
        const Cand& c = cands[i];
        if (c.h.m >= 0.0 && c.h.t > kTmin && c.h.t <= max_depth) {
            if (best < 0 || c.h.t < cands[best].h.t || (c.h.t == cands[best].h.t && c.id < cands[best].id))
                best = i;
        }
    }
    const double t_ref = best >= 0 ? cands[best].h.t * (1.0 + kTau) : max_depth * (1.0 + kTau);
    if (best >= 0) {
        r.id = cands[best].id;
        r.t = cands[best].h.t;
        if (cands[best].h.m < kTau * cands[best].h.sigma) r.tie = 1;
        if (std::fabs(r.t - max_depth) <= kTau * max_depth) r.tie = 1;
    }
    for (int i = 0; i < (int)cands.size(); ++i) {
        if (i == best) continue;
        const Cand& c = cands[i];
        const bool near = c.h.m > -kTau * c.h.sigma && c.h.t > kTmin;
        if (!near) continue;
        if (c.h.t <= t_ref) r.tie = 1;
        if (std::fabs(c.h.t - max_depth) <= kTau * max_depth) r.tie = 1;
    }
    return r;
}

inline double t_limit(const OracleParams& p) { return p.max_depth * (1.0 + kTau); }

// ------------------------------------------------------------ swarm drones
// Multi-agent mode [Sec. III-B]: the drones of one scene see each other (the
// parallel-agents mode omits them).  Reading: each drone is a box of half
// extents h about its body origin, aligned with its body axes, and a camera
// never sees its own drone.  Drone j enters a pixel's candidate list with id
// INT32_MIN + j, so the closest-hit rule and the ambiguity classification of
// triangles apply unchanged:
//   * definite hit (m = 1): the ray hits the box shrunk by delta on every axis;
//   * hit near the silhouette (m = 0, ambiguous): hits the box, not the shrunk one;
//   * near miss (m = -kTau / 2): only the box grown by delta is hit;
// delta = kTau * (|o - centre| + |h|), the FP32 error scale of moving the ray
// into the drone's frame, times the same 50 eps_f32 band as the triangles.
struct Swarm {
    const double* states;  // [n][17], the swarm's agents
    int64_t n;
    double half[3];
    uint8_t rgb[3];
    // the swarm index of each rendered view (its own drone is never seen), or
    // null when the views are the swarm's agents in order
    const int64_t* self = nullptr;
};

// Ray (o, d) against the box of half extents h + g (every axis) of the drone
// with state st.  Hit at t > kTmin: the entry distance, or the exit distance
// when the ray starts inside (boxes are seen from inside, like two-sided
// triangles of a closed mesh).
bool ray_drone(const double* st, const double h[3], double g, const double o[3], const double d[3], double& t) {
    const double q[4] = {st[6], st[7], st[8], st[9]};
    double R[3][3];
    rotation_matrix(q, R);
    double tn = -std::numeric_limits<double>::infinity(), tf = std::numeric_limits<double>::infinity();
    for (int k = 0; k < 3; ++k) {
        // coordinates along the drone's body axis k (column k of R)
        const double ol = R[0][k] * (o[0] - st[0]) + R[1][k] * (o[1] - st[1]) + R[2][k] * (o[2] - st[2]);
        const double dl = R[0][k] * d[0] + R[1][k] * d[1] + R[2][k] * d[2];
        const double hk = h[k] + g;
        if (!(hk > 0.0)) return false;
        if (dl == 0.0) {
            if (std::fabs(ol) > hk) return false;
            continue;
        }
        double a = (-hk - ol) / dl, b = (hk - ol) / dl;
        if (a > b) std::swap(a, b);
        tn = std::max(tn, a);
        tf = std::min(tf, b);
    }
    if (tn > tf) return false;
    if (tn > kTmin) {
        t = tn;
        return true;
    }
    if (tf > kTmin) {
        t = tf;
        return true;
    }
    return false;
}

void collect_drones(const Swarm& sw, int64_t self, const double o[3], const double d[3], std::vector<Cand>& out) {
    const double hn = std::sqrt(sw.half[0] * sw.half[0] + sw.half[1] * sw.half[1] + sw.half[2] * sw.half[2]);
    for (int64_t j = 0; j < sw.n; ++j) {
        if (j == self) continue;
        const double* st = sw.states + 17 * j;
        const double dx = o[0] - st[0], dy = o[1] - st[1], dz = o[2] - st[2];
        const double delta = kTau * (std::sqrt(dx * dx + dy * dy + dz * dz) + hn);
        double t_in = 0.0, t_ex = 0.0, t_out = 0.0;
        const bool in = ray_drone(st, sw.half, -delta, o, d, t_in);
        const bool ex = ray_drone(st, sw.half, 0.0, o, d, t_ex);
        const bool grown = ray_drone(st, sw.half, delta, o, d, t_out);
        if (!ex && !grown) continue;
        Cand c;
        c.id = std::numeric_limits<int32_t>::min() + (int32_t)j;
        c.h.sigma = 1.0;
        if (ex) {
            c.h.t = t_ex;
            c.h.m = in ? 1.0 : 0.0;
        } else {
            c.h.t = t_out;
            c.h.m = -0.5 * kTau;
        }
        out.push_back(c);
    }
}

// Output id of a candidate id: triangles as they are, drone j as -2 - j.
inline int32_t output_id(int32_t id) {
    return id >= -1 ? id : -2 - (int32_t)((int64_t)id - std::numeric_limits<int32_t>::min());
}
inline int32_t candidate_id(int32_t out) {
    return out >= -1 ? out : (int32_t)((int64_t)std::numeric_limits<int32_t>::min() + (-2 - (int64_t)out));
}

int render_impl(const OracleScene* s, const OracleParams* p, int64_t n, const double* states, int use_bvh,
                const Swarm* sw, double* depth, uint8_t* rgb, int32_t* hit_id, uint8_t* tie) {
    if (!s || !p || n < 0) return -1;
    if (use_bvh && s->nodes.empty() && !s->tris.empty()) return -2;
    const int W = p->width, H = p->height;
    const int64_t npix = n * (int64_t)W * H;
#pragma omp parallel
    {
        std::vector<Cand> cands;
#pragma omp for schedule(dynamic, 64)
        for (int64_t k = 0; k < npix; ++k) {
            const int64_t a = k / ((int64_t)W * H);
            const int r = (int)((k / W) % H), c = (int)(k % W);
            double o[3], d[3];
            camera_ray(*p, states + a * 17, r, c, o, d);
            collect_candidates(*s, o, d, t_limit(*p), use_bvh != 0, cands);
            if (sw) collect_drones(*sw, sw->self ? sw->self[a] : a, o, d, cands);
            const PixelResult pr = classify(cands, p->max_depth);
            if (depth) depth[k] = pr.t;
            if (hit_id) hit_id[k] = output_id(pr.id);
            if (tie) tie[k] = pr.tie;
            if (rgb) {
                for (int j = 0; j < 3; ++j)
                    rgb[3 * k + j] = pr.id >= 0 ? s->rgb[3 * (int64_t)pr.id + j] : pr.id < -1 ? sw->rgb[j] : 0;
            }
        }
    }
    return 0;
}

// Entry distance of the ray into a box no farther than t_lim, or -1 when it
// misses (exact slab test; a zero direction component keeps the slab open
// when the origin lies inside it).
double box_entry(const double o[3], const double inv[3], const double lo[3], const double hi[3], double t_lim) {
    double t0 = 0.0, t1 = t_lim;
    for (int j = 0; j < 3; ++j) {
        double a = (lo[j] - o[j]) * inv[j], b = (hi[j] - o[j]) * inv[j];
        if (std::isnan(a) || std::isnan(b)) {
            if (o[j] < lo[j] || o[j] > hi[j]) return -1.0;
            continue;
        }
        if (a > b) std::swap(a, b);
        t0 = std::max(t0, a);
        t1 = std::min(t1, b);
        if (t0 > t1) return -1.0;
    }
    return t0;
}

// Work of one ray's closest-hit walk over the oracle's median-split BVH: the
// internal nodes it visits (the root, then every child whose box it enters
// before its current closest hit, nearer child first) and the triangles of the
// leaves it reaches.  A statistic to set beside the GPU's counted walks, not a
// parity quantity.
void walk_counts(const OracleScene& s, const double o[3], const double d[3], double t_max, int64_t& nodes,
                 int64_t& tests) {
    if (s.nodes.empty()) return;
    double inv[3];
    for (int j = 0; j < 3; ++j) inv[j] = 1.0 / d[j];
    double best = t_max;
    std::vector<std::pair<int32_t, double>> stack;
    stack.push_back({0, 0.0});
    while (!stack.empty()) {
        const auto top = stack.back();
        stack.pop_back();
        if (top.second > best) continue;
        const BvhNode& n = s.nodes[top.first];
        if (n.left < 0) {
            for (int32_t i = n.first; i < n.first + n.count; ++i) {
                ++tests;
                Hit h;
                if (moller_trumbore(o, d, s.tris[s.order[i]], h) && h.m >= 0.0 && h.t > kTmin && h.t <= best)
                    best = h.t;
            }
            continue;
        }
        ++nodes;
        const double tl = box_entry(o, inv, s.nodes[n.left].lo, s.nodes[n.left].hi, best);
        const double tr = box_entry(o, inv, s.nodes[n.right].lo, s.nodes[n.right].hi, best);
        const bool l_first = tl >= 0.0 && (tr < 0.0 || tl <= tr);
        // the farther child goes on the stack first
        if (l_first) {
            if (tr >= 0.0) stack.push_back({n.right, tr});
            stack.push_back({n.left, tl});
        } else {
            if (tl >= 0.0) stack.push_back({n.left, tl});
            if (tr >= 0.0) stack.push_back({n.right, tr});
        }
    }
}

int validate_impl(const OracleScene* s, const OracleParams* p, int64_t n, const double* states, const Swarm* sw,
                  int64_t npix, const int64_t* pix, const int32_t* id, const float* depth, uint8_t* valid) {
    if (!s || !p || n < 0) return -1;
    const int W = p->width, H = p->height;
    const bool use_bvh = !s->nodes.empty();
#pragma omp parallel
    {
        std::vector<Cand> cands;
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < npix; ++k) {
            const int64_t q = pix[k];
            const int64_t a = q / ((int64_t)W * H);
            const int r = (int)((q / W) % H), c = (int)(q % W);
            valid[k] = 0;
            if (a < 0 || a >= n) continue;
            double o[3], d[3];
            camera_ray(*p, states + a * 17, r, c, o, d);
            collect_candidates(*s, o, d, t_limit(*p), use_bvh, cands);
            if (sw) collect_drones(*sw, sw->self ? sw->self[a] : a, o, d, cands);
            double t_def = std::numeric_limits<double>::infinity();
            for (const Cand& cd : cands)
                if (cd.h.m > kTau * cd.h.sigma && cd.h.t > kTmin && cd.h.t <= p->max_depth * (1.0 - kTau))
                    t_def = std::min(t_def, cd.h.t);
            if (id[k] == -1) {
                valid[k] = (std::isinf(t_def) && depth[k] == (float)p->max_depth) ? 1 : 0;
                continue;
            }
            const int32_t want = candidate_id(id[k]);
            for (const Cand& cd : cands) {
                if (cd.id != want) continue;
                const bool ok = cd.h.m > -kTau * cd.h.sigma && cd.h.t > kTmin &&
                                cd.h.t <= p->max_depth * (1.0 + kTau) && cd.h.t <= t_def * (1.0 + kTau) &&
                                std::fabs((double)depth[k] - cd.h.t) <= 1e-4 * cd.h.t;
                valid[k] = ok ? 1 : 0;
            }
        }
    }
    return 0;
}

}  // namespace

extern "C" {

// ----------------------------------------------------------------- dynamics
// state_in / state_out: [n][17] (x, v, q(w,x,y,z), Omega, omega_1..4); cmd: [n][4].
int oracle_step(const OracleParams* p, int64_t n, const double* state_in, const double* cmd, double* state_out) {
    if (!p || n < 0 || p->n_sub < 1) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n; ++a) {
        double y[17], u[4];
        for (int j = 0; j < 17; ++j) y[j] = state_in[a * 17 + j];
        for (int j = 0; j < 4; ++j) u[j] = cmd[a * 4 + j];
        step_agent(*p, y, u);
        for (int j = 0; j < 17; ++j) state_out[a * 17 + j] = y[j];
    }
    return 0;
}

// states: [T+1][n][17] with states[0] = state0; cmds: [T][n][4].
int oracle_rollout(const OracleParams* p, int64_t n, int64_t T, const double* state0, const double* cmds,
                   double* states) {
    if (!p || n < 0 || T < 0 || p->n_sub < 1) return -1;
    std::memcpy(states, state0, sizeof(double) * n * 17);
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n; ++a) {
        double y[17], u[4];
        for (int j = 0; j < 17; ++j) y[j] = state0[a * 17 + j];
        for (int64_t t = 0; t < T; ++t) {
            for (int j = 0; j < 4; ++j) u[j] = cmds[(t * n + a) * 4 + j];
            step_agent(*p, y, u);
            for (int j = 0; j < 17; ++j) states[((t + 1) * n + a) * 17 + j] = y[j];
        }
    }
    return 0;
}

// Vector-Jacobian product of one step, column by column with dual numbers:
// g_state_in[a][j] = sum_i g_out[a][i] d out_i / d state_j, likewise g_cmd.
int oracle_step_vjp(const OracleParams* p, int64_t n, const double* state_in, const double* cmd,
                    const double* g_out, double* g_state_in, double* g_cmd) {
    if (!p || n < 0 || p->n_sub < 1) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n; ++a) {
        for (int dir = 0; dir < 21; ++dir) {
            Dual y[17], u[4];
            for (int j = 0; j < 17; ++j) y[j] = Dual(state_in[a * 17 + j], dir == j ? 1.0 : 0.0);
            for (int j = 0; j < 4; ++j) u[j] = Dual(cmd[a * 4 + j], dir == 17 + j ? 1.0 : 0.0);
            step_agent(*p, y, u);
            double acc = 0.0;
            for (int i = 0; i < 17; ++i) acc += g_out[a * 17 + i] * y[i].d;
            if (dir < 17)
                g_state_in[a * 17 + dir] = acc;
            else
                g_cmd[a * 4 + dir - 17] = acc;
        }
    }
    return 0;
}

// Rollout loss per agent a (goal g_a, horizon T, weight lam):
//   L_a = 1/T sum_{t=1..T} |x_t - g_a|^2 + lam/T sum_{t=0..T-1} |u_t|^2
// and its exact gradient w.r.t. state0 [n][17] and cmds [T][n][4], one
// forward-mode pass per input component.
int oracle_rollout_loss_grad(const OracleParams* p, int64_t n, int64_t T, const double* state0,
                             const double* cmds, const double* goals, double lam, double* loss,
                             double* g_state0, double* g_cmds) {
    if (!p || n < 0 || T < 1 || p->n_sub < 1) return -1;
    const int64_t ndir = 17 + 4 * T;
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int64_t a = 0; a < n; ++a) {
        for (int64_t dir = 0; dir < ndir; ++dir) {
            Dual y[17];
            for (int j = 0; j < 17; ++j) y[j] = Dual(state0[a * 17 + j], dir == j ? 1.0 : 0.0);
            Dual L(0.0);
            for (int64_t t = 0; t < T; ++t) {
                Dual u[4];
                for (int j = 0; j < 4; ++j)
                    u[j] = Dual(cmds[(t * n + a) * 4 + j], dir == 17 + 4 * t + j ? 1.0 : 0.0);
                for (int j = 0; j < 4; ++j) L = L + (lam / T) * u[j] * u[j];
                step_agent(*p, y, u);
                for (int j = 0; j < 3; ++j) {
                    const Dual e = y[j] - goals[a * 3 + j];
                    L = L + (1.0 / T) * e * e;
                }
            }
            if (dir == 0) loss[a] = L.v;
            if (dir < 17)
                g_state0[a * 17 + dir] = L.d;
            else {
                const int64_t t = (dir - 17) / 4, j = (dir - 17) % 4;
                g_cmds[(t * n + a) * 4 + j] = L.d;
            }
        }
    }
    return 0;
}

// ------------------------------------------------------------------- render
// verts: [nv][3] (float32 values promoted), tris: [nt][3] int32, rgb: [nt][3].
void* oracle_scene_create(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, const uint8_t* rgb,
                          int build_bvh) {
    if (nv < 0 || nt < 0) return nullptr;
    OracleScene* s = new OracleScene();
    s->tris.resize(nt);
    s->rgb.assign(rgb, rgb + nt * 3);
    for (int64_t i = 0; i < nt; ++i) {
        Tri& t = s->tris[i];
        const double* a = verts + 3 * (int64_t)tris[3 * i];
        const double* b = verts + 3 * (int64_t)tris[3 * i + 1];
        const double* c = verts + 3 * (int64_t)tris[3 * i + 2];
        for (int j = 0; j < 3; ++j) {
            t.v0[j] = a[j];
            t.v1[j] = b[j];
            t.v2[j] = c[j];
            t.lo[j] = std::min(a[j], std::min(b[j], c[j]));
            t.hi[j] = std::max(a[j], std::max(b[j], c[j]));
        }
    }
    if (build_bvh && nt > 0) {
        s->order.resize(nt);
        for (int64_t i = 0; i < nt; ++i) s->order[i] = (int32_t)i;
        bvh_build(*s, 0, (int32_t)nt, 0);
    }
    return s;
}

void oracle_scene_destroy(void* scene) { delete static_cast<OracleScene*>(scene); }

int64_t oracle_scene_bvh_nodes(const void* scene) {
    return (int64_t) static_cast<const OracleScene*>(scene)->nodes.size();
}

// states: [n][17]; outputs [n][H][W] (rgb [n][H][W][3]).  Any output may be null.
int oracle_render(const void* scene, const OracleParams* p, int64_t n, const double* states, int use_bvh,
                  double* depth, uint8_t* rgb, int32_t* hit_id, uint8_t* tie) {
    return render_impl(static_cast<const OracleScene*>(scene), p, n, states, use_bvh, nullptr, depth, rgb, hit_id,
                       tie);
}

// Mean per ray of the internal nodes visited and the triangles tested by
// closest-hit walks over the oracle's median-split BVH (walk_counts), for every
// pixel of the n agents' images.  states [n][17]; out[0] nodes, out[1] triangles.
int oracle_traversal_counts(const void* scene, const OracleParams* p, int64_t n, const double* states,
                            double* out) {
    const OracleScene* s = static_cast<const OracleScene*>(scene);
    if (!s || !p || n < 0 || !out) return -1;
    if (s->nodes.empty() && !s->tris.empty()) return -2;
    const int W = p->width, H = p->height;
    const int64_t npix = n * (int64_t)W * H;
    int64_t nodes = 0, tests = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : nodes, tests)
    for (int64_t k = 0; k < npix; ++k) {
        const int64_t a = k / ((int64_t)W * H);
        const int r = (int)((k / W) % H), c = (int)(k % W);
        double o[3], d[3];
        camera_ray(*p, states + a * 17, r, c, o, d);
        walk_counts(*s, o, d, p->max_depth, nodes, tests);
    }
    out[0] = npix ? (double)nodes / (double)npix : 0.0;
    out[1] = npix ? (double)tests / (double)npix : 0.0;
    return 0;
}

// As oracle_render, with the n agents forming one swarm [Sec. III-B]: every
// other agent's drone (box of half extents half[3] about its body origin,
// colour drone_rgb) is visible.  A drone hit reports id -2 - j.
int oracle_render_swarm(const void* scene, const OracleParams* p, int64_t n, const double* states, int use_bvh,
                        const double* half, const uint8_t* drone_rgb, double* depth, uint8_t* rgb, int32_t* hit_id,
                        uint8_t* tie) {
    if (!half || !drone_rgb) return -1;
    Swarm sw{states, n, {half[0], half[1], half[2]}, {drone_rgb[0], drone_rgb[1], drone_rgb[2]}};
    return render_impl(static_cast<const OracleScene*>(scene), p, n, states, use_bvh, &sw, depth, rgb, hit_id, tie);
}

// Check answers given for ambiguous pixels.  For pixel k = (agent, row, col)
// (pix[k] = agent * H * W + row * W + col) with claimed id[k] (a triangle, -1
// for a miss, or -2 - j for drone j in the swarm form) and depth[k],
// valid[k] = 1 when the claim is one of the answers the ambiguity admits:
//   * "definite" hits are candidates with m > kTau * sigma and
//     kTmin < t <= max_depth * (1 - kTau); t_def is the closest of them;
//   * a miss (id = -1, depth = max_depth) is valid when no definite hit exists;
//   * a candidate j is valid when it is nearly hit (m > -kTau * sigma),
//     t_j <= max_depth * (1 + kTau), t_j <= t_def * (1 + kTau), and the claimed
//     depth is within 1e-4 * t_j of t_j.
int oracle_validate(const void* scene, const OracleParams* p, int64_t n, const double* states, int64_t npix,
                    const int64_t* pix, const int32_t* id, const float* depth, uint8_t* valid) {
    return validate_impl(static_cast<const OracleScene*>(scene), p, n, states, nullptr, npix, pix, id, depth, valid);
}

int oracle_validate_swarm(const void* scene, const OracleParams* p, int64_t n, const double* states,
                          const double* half, int64_t npix, const int64_t* pix, const int32_t* id, const float* depth,
                          uint8_t* valid) {
    if (!half) return -1;
    Swarm sw{states, n, {half[0], half[1], half[2]}, {0, 0, 0}};
    return validate_impl(static_cast<const OracleScene*>(scene), p, n, states, &sw, npix, pix, id, depth, valid);
}

// As oracle_render_swarm / oracle_validate_swarm for a chosen set of views:
// view k has the state views[k] ([n_views][17]) and is agent self[k] of the
// swarm (swarm [n_swarm][17]), whose other drones it sees.  Lets a test check a
// few cameras of a large swarm without rendering every camera.
int oracle_render_swarm_views(const void* scene, const OracleParams* p, int64_t n_views, const double* views,
                              const int64_t* self, int64_t n_swarm, const double* swarm, int use_bvh,
                              const double* half, const uint8_t* drone_rgb, double* depth, uint8_t* rgb,
                              int32_t* hit_id, uint8_t* tie) {
    if (!half || !drone_rgb || !self || !swarm) return -1;
    for (int64_t k = 0; k < n_views; ++k)
        if (self[k] < 0 || self[k] >= n_swarm) return -1;
    Swarm sw{swarm, n_swarm, {half[0], half[1], half[2]}, {drone_rgb[0], drone_rgb[1], drone_rgb[2]}, self};
    return render_impl(static_cast<const OracleScene*>(scene), p, n_views, views, use_bvh, &sw, depth, rgb, hit_id,
                       tie);
}

int oracle_validate_swarm_views(const void* scene, const OracleParams* p, int64_t n_views, const double* views,
                                const int64_t* self, int64_t n_swarm, const double* swarm, const double* half,
                                int64_t npix, const int64_t* pix, const int32_t* id, const float* depth,
                                uint8_t* valid) {
    if (!half || !self || !swarm) return -1;
    for (int64_t k = 0; k < n_views; ++k)
        if (self[k] < 0 || self[k] >= n_swarm) return -1;
    Swarm sw{swarm, n_swarm, {half[0], half[1], half[2]}, {0, 0, 0}, self};
    return validate_impl(static_cast<const OracleScene*>(scene), p, n_views, views, &sw, npix, pix, id, depth, valid);
}

// Pairwise proximity of a swarm [Sec. III-B: collisions among the drones of
// the multi-agent mode], brute force over all pairs.  Reading: drones collide
// as spheres of the given radius.  pos [n][3]; outputs per agent: the centre
// distance to the nearest other agent (+inf when alone), that agent (lowest
// index among equal distances, -1 when alone), and how many others lie closer
// than 2 * radius.
int oracle_swarm_proximity(int64_t n, const double* pos, double radius, double* dist, int32_t* other,
                           int32_t* n_collide) {
    if (n < 0 || (n > 0 && !pos)) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double best = std::numeric_limits<double>::infinity();
        int32_t who = -1, hits = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                         dz = pos[3 * i + 2] - pos[3 * j + 2];
            const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
            if (r < best) {
                best = r;
                who = (int32_t)j;
            }
            if (r < 2.0 * radius) ++hits;
        }
        if (dist) dist[i] = best;
        if (other) other[i] = who;
        if (n_collide) n_collide[i] = hits;
    }
    return 0;
}

// ------------------------------------------------------- nearest obstacle
// Closest point of triangle (a, b, c) to point p, by the Voronoi regions of
// the triangle: the three vertex regions, the three edge regions, and the
// face region (projection onto the plane).  Barycentric-style parameters are
// computed from dot products of the edge vectors with the point's offsets.
static void closest_on_triangle(const double p[3], const double a[3], const double b[3], const double c[3],
                                double out[3]) {
    auto sub = [](const double* x, const double* y, double* r) {
        for (int j = 0; j < 3; ++j) r[j] = x[j] - y[j];
    };
    auto dot = [](const double* x, const double* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    sub(b, a, ab);
    sub(c, a, ac);
    sub(p, a, ap);
    const double d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) {  // vertex a
        for (int j = 0; j < 3; ++j) out[j] = a[j];
        return;
    }
    sub(p, b, bp);
    const double d3 = dot(ab, bp), d4 = dot(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) {  // vertex b
        for (int j = 0; j < 3; ++j) out[j] = b[j];
        return;
    }
    const double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {  // edge ab
        const double v = d1 / (d1 - d3);
        for (int j = 0; j < 3; ++j) out[j] = a[j] + v * ab[j];
        return;
    }
    sub(p, c, cp);
    const double d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) {  // vertex c
        for (int j = 0; j < 3; ++j) out[j] = c[j];
        return;
    }
    const double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {  // edge ac
        const double w = d2 / (d2 - d6);
        for (int j = 0; j < 3; ++j) out[j] = a[j] + w * ac[j];
        return;
    }
    const double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {  // edge bc
        const double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int j = 0; j < 3; ++j) out[j] = b[j] + w * (c[j] - b[j]);
        return;
    }
    const double den = 1.0 / (va + vb + vc);  // face
    const double v = vb * den, w = vc * den;
    for (int j = 0; j < 3; ++j) out[j] = a[j] + ab[j] * v + ac[j] * w;
}

// For every query point (positions [n][3]): the distance to the closest point
// of the mesh (brute force over all triangles), that point, and the lowest id
// among triangles within 1e-12 of the minimum; distances above max_dist give
// max_dist, id -1 and the query point itself.
int oracle_nearest(const void* scene, int64_t n, const double* pos, double max_dist, double* dist, double* point,
                   int32_t* tri) {
    const OracleScene* s = static_cast<const OracleScene*>(scene);
    if (!s || n < 0) return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < n; ++a) {
        const double* p = pos + 3 * a;
        double best = std::numeric_limits<double>::infinity(), bp[3] = {p[0], p[1], p[2]};
        int32_t bid = -1;
        for (int32_t id = 0; id < (int32_t)s->tris.size(); ++id) {
            const Tri& t = s->tris[id];
            double q[3];
            closest_on_triangle(p, t.v0, t.v1, t.v2, q);
            const double d = std::sqrt((q[0] - p[0]) * (q[0] - p[0]) + (q[1] - p[1]) * (q[1] - p[1]) +
                                       (q[2] - p[2]) * (q[2] - p[2]));
            if (d < best - 1e-12 || (std::fabs(d - best) <= 1e-12 && id < bid)) {
                best = d;
                bid = id;
                for (int j = 0; j < 3; ++j) bp[j] = q[j];
            }
        }
        if (!(best <= max_dist)) {
            best = max_dist;
            bid = -1;
            for (int j = 0; j < 3; ++j) bp[j] = p[j];
        }
        dist[a] = best;
        tri[a] = bid;
        for (int j = 0; j < 3; ++j) point[3 * a + j] = bp[j];
    }
    return 0;
}

// Distance from p to triangle id (for validating a claimed nearest triangle).
int oracle_point_triangle(const void* scene, int64_t n, const double* pos, const int32_t* ids, double* dist) {
    const OracleScene* s = static_cast<const OracleScene*>(scene);
    if (!s || n < 0) return -1;
    for (int64_t a = 0; a < n; ++a) {
        if (ids[a] < 0 || ids[a] >= (int32_t)s->tris.size()) {
            dist[a] = std::numeric_limits<double>::infinity();
            continue;
        }
        const Tri& t = s->tris[ids[a]];
        double q[3];
        closest_on_triangle(pos + 3 * a, t.v0, t.v1, t.v2, q);
        const double* p = pos + 3 * a;
        dist[a] = std::sqrt((q[0] - p[0]) * (q[0] - p[0]) + (q[1] - p[1]) * (q[1] - p[1]) + (q[2] - p[2]) * (q[2] - p[2]));
    }
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"

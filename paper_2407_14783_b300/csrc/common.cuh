// Shared device-side definitions of the rollout-step library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "visfly_b300.h"

namespace vf {

constexpr int kStateDim = 17;
constexpr int kCmdDim = 4;
constexpr int kMaxSub = 8;      // physics sub-steps per control step
constexpr int kLeafMax = 3;     // triangles per BVH leaf after collapsing
constexpr int kMaxCkptK = 32;   // steps between checkpoints in the rollout adjoint
constexpr int kEmptyRoot = INT32_MIN;

// Device error codes written into the context's error word (first one wins).
constexpr int kDevErrTraversal = 1;
constexpr int kDevErrNotFound = 2;

// Constants of the dynamics derived once on the host from sim_params.
struct DynConsts {
    float mass, inv_mass;
    float J[3], invJ[3], JK[3];     // J, 1/J, J * K_rate
    float rate_max[3];
    float half_a_max_m;             // mass * a_max / 2: collective thrust per unit of (u0 + 1)
    float Ainv[4][4];               // inverse of the mixer (collective thrust, moment) <- rotor thrusts
    float mix[3][4];                // rows: r_y, -r_x, spin * kappa (moment per unit rotor thrust)
    float k0, k1, k2;
    float f_lo, f_hi;               // reachable rotor thrust range
    float omega_min, omega_max;
    // Near zero rotor thrust the square-root inverse of the thrust polynomial
    // turns FP32 rounding of the mixer solve (about 1e-6 N) into rotor-speed
    // errors of order 1 rad/s, so the controller carries its cancellation-prone
    // quantities in double precision, as double-float pairs (hi + lo floats,
    // about 48 bits, on the FP32 pipes) formed on the host from FP64 values.
    float2 xJ[3], xJK[3], xrate_max[3], xhalf_a_max_m, xAinv[4][4], xf_lo, xf_hi, xk0, xk1sq, x4k2, xhalf_f_hi;
    int controller;                 // 0 CTBR, 1 SRT, 2 LV, 3 PS
    // geometric controllers: m K_pos, m K_vel, m g, J K_att, J K_omega
    float2 xmKpos[3], xmKvel[3], xmg, xJKatt[3], xJKom[3];
    float decay;                    // exp(-c h)
    float drag[3];                  // rho Cd s / 2
    float g;
    float h;                        // physics sub-step
    int n_sub, integrator;
};

// Camera constants for the ray generator.
struct CamConsts {
    int W, H;
    float pix;          // 2 tan(fov/2) / W: body-frame direction change per pixel
    float max_depth;
    float cam_off[3];
};

// One row of the segmented scene table: everything a ray needs about its
// agent's scene.  Child / root encoding: >= 0 internal node index; < 0 a leaf
// range (see leaf_code); kEmptyRoot when the BVH holds no triangle.
struct SceneRow {
    const float4* nodes;     // 4 float4 per internal node
    const float4* wide;      // 8 float4 per internal node: 4-wide layout of the even-depth ones
    const float4* tris;      // 3 float4 per triangle, leaf order
    const float4* large;     // 3 float4 per large triangle (tested by every ray)
    const uint32_t* colors;  // RGB8 per original triangle id
    const int32_t* labels;   // segmentation label per original triangle id (null: the id itself)
    int32_t root;
    int32_t n_large;
    int32_t depth;
    int32_t live;
    int32_t n_nodes;         // internal nodes (binary layout)
    int32_t n_tree_tris;     // triangles in the tree (leaf order)
};

__host__ __device__ inline int32_t leaf_code(int32_t first, int32_t count) {
    return -1 - ((first << 3) | (count - 1));
}
__host__ __device__ inline void leaf_decode(int32_t code, int32_t& first, int32_t& count) {
    const int32_t v = -1 - code;
    first = v >> 3;
    count = (v & 7) + 1;
}

__device__ inline void set_error(int* err, int code) { atomicCAS(err, 0, code); }

// Sensor noise of the rendered images (Table II models), drawn from the
// counter-based SplitMix64 generator: output number i of the stream `seed`.
struct NoiseParams {
    int enabled;
    unsigned long long seed;
    float d_gauss, d_speckle, d_shot, d_sp;   // depth: additive N(0,s^2) m, multiplicative, shot scale, salt&pepper
    float c_gauss, c_speckle, c_shot, c_sp;   // colour channels (0-255 units)
    float s_drop;                             // segmentation: probability of an unlabelled pixel
    float s_gauss, s_speckle, s_shot, s_sp;   // segmentation label noise (label units)
    float s_max;                              // largest label after noise
    int s_models;                             // any label-noise model on
};

__host__ __device__ inline unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace vf

// Multi-agent (swarm) mode [Sec. III-B]: the drones of one scene see each
// other and can collide; the parallel-agents mode omits them.  Before a swarm
// render the agents of a launch are bucketed by scene and every drone's pose
// is packed for the ray cast:
//   drones[3 j + k] = (body axis k of drone j in world coordinates, centre_k)
// so a ray moves into drone j's frame with three dot products per axis.  The
// member lists also serve the pairwise proximity query.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "launch.h"

namespace vf {
namespace {

// One CTA buckets the launch's agents by scene and packs every drone's pose:
// zero the counts, count (shared-memory atomics when the table is small),
// scan, scatter.  A single launch with no host-side clears: the per-launch
// preparation costs one small kernel, whatever the number of scenes.
constexpr int kPrepThreads = 1024;
constexpr int kPrepSmemScenes = 4096;

__global__ void __launch_bounds__(kPrepThreads) swarm_prep_kernel(int n, const int* __restrict__ scene_of_agent,
                                                                  const float* __restrict__ state, int n_scenes,
                                                                  int* __restrict__ off, int* __restrict__ cursor,
                                                                  int* __restrict__ members,
                                                                  float4* __restrict__ spheres,
                                                                  float4* __restrict__ drones) {
    __shared__ int cnt[kPrepSmemScenes];
    __shared__ int part[kPrepThreads];
    __shared__ int carry;
    const bool small = n_scenes <= kPrepSmemScenes;
    const int tid = threadIdx.x;
    for (int k = tid; k <= n_scenes; k += kPrepThreads) {
        off[k] = 0;
        if (small && k < n_scenes) cnt[k] = 0;
    }
    if (tid == 0) carry = 0;
    __syncthreads();
    // counts (into off[sid + 1]) and drone poses
    for (int i = tid; i < n; i += kPrepThreads) {
        const float qw = state[6 * n + i], qx = state[7 * n + i], qy = state[8 * n + i], qz = state[9 * n + i];
        const float inv_n = 1.0f / (qw * qw + qx * qx + qy * qy + qz * qz);
        // columns of R(q / |q|): the drone's body axes in world coordinates
        drones[3 * (size_t)i] = make_float4((qw * qw + qx * qx - qy * qy - qz * qz) * inv_n,
                                            2.0f * (qx * qy + qw * qz) * inv_n, 2.0f * (qx * qz - qw * qy) * inv_n,
                                            state[i]);
        drones[3 * (size_t)i + 1] = make_float4(2.0f * (qx * qy - qw * qz) * inv_n,
                                                (qw * qw - qx * qx + qy * qy - qz * qz) * inv_n,
                                                2.0f * (qy * qz + qw * qx) * inv_n, state[n + i]);
        drones[3 * (size_t)i + 2] = make_float4(2.0f * (qx * qz + qw * qy) * inv_n, 2.0f * (qy * qz - qw * qx) * inv_n,
                                                (qw * qw - qx * qx - qy * qy + qz * qz) * inv_n, state[2 * n + i]);
        const int sid = scene_of_agent[i];
        if (sid >= 0 && sid < n_scenes) {
            if (small) atomicAdd(cnt + sid, 1);
            else atomicAdd(off + sid + 1, 1);
        }
    }
    __syncthreads();
    // inclusive scan of the counts into off[1 .. n_scenes]
    for (int base = 0; base < n_scenes; base += kPrepThreads) {
        const int k = base + tid;
        part[tid] = k < n_scenes ? (small ? cnt[k] : off[k + 1]) : 0;
        __syncthreads();
        for (int st = 1; st < kPrepThreads; st <<= 1) {
            const int v = tid >= st ? part[tid - st] : 0;
            __syncthreads();
            part[tid] += v;
            __syncthreads();
        }
        if (k < n_scenes) off[k + 1] = part[tid] + carry;
        __syncthreads();
        if (tid == kPrepThreads - 1) carry += part[tid];
        __syncthreads();
    }
    // scatter (order within a scene is arbitrary: the ray cast's closest-hit
    // rule does not depend on it); cursors count from zero again
    for (int k = tid; k < n_scenes; k += kPrepThreads) {
        if (small) cnt[k] = 0;
        else cursor[k] = 0;
    }
    __syncthreads();
    for (int i = tid; i < n; i += kPrepThreads) {
        const int sid = scene_of_agent[i];
        if (sid < 0 || sid >= n_scenes) continue;
        const int slot = small ? atomicAdd(cnt + sid, 1) : atomicAdd(cursor + sid, 1);
        members[off[sid] + slot] = i;
        spheres[off[sid] + slot] = make_float4(state[i], state[n + i], state[2 * n + i], __int_as_float(i));
    }
}

// Per agent (one warp each, the lanes splitting the scene's members): the
// nearest other agent of its scene (centre distance; lowest index among equal
// squared distances) and how many lie closer than 2 radius.
__global__ void swarm_proximity_kernel(int n, const int* __restrict__ scene_of_agent, const float* __restrict__ state,
                                       int n_scenes, const int* __restrict__ off, const float4* __restrict__ spheres,
                                       float radius, float* __restrict__ dist, int* __restrict__ other,
                                       int* __restrict__ n_collide) {
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;  // whole warps leave together
    const int sid = __ldg(scene_of_agent + i);
    float best = INFINITY;
    int who = -1, hits = 0;
    if (sid >= 0 && sid < n_scenes) {
        const float x = __ldg(state + i), y = __ldg(state + n + i), z = __ldg(state + 2 * n + i);
        const float lim = 4.0f * radius * radius;
        const int hi = __ldg(off + sid + 1);
#pragma unroll 4
        for (int k = __ldg(off + sid) + lane; k < hi; k += 32) {
            const float4 m = __ldg(spheres + k);
            const int j = __float_as_int(m.w);
            if (j == i) continue;
            const float dx = x - m.x, dy = y - m.y, dz = z - m.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < best || (d2 == best && j < who)) {
                best = d2;
                who = j;
            }
            if (d2 < lim) ++hits;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int w2 = __shfl_xor_sync(0xffffffffu, who, o);
        if (b2 < best || (b2 == best && w2 >= 0 && (who < 0 || w2 < who))) {
            best = b2;
            who = w2;
        }
        hits += __shfl_xor_sync(0xffffffffu, hits, o);
    }
    if (lane == 0) {
        if (dist) dist[i] = sqrtf(best);
        if (other) other[i] = who;
        if (n_collide) n_collide[i] = hits;
    }
}

}  // namespace

cudaError_t launch_swarm_prep(int n, const int* scene_of_agent, const float* state, int n_scenes, SwarmScratch& s,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    swarm_prep_kernel<<<1, kPrepThreads, 0, st>>>(n, scene_of_agent, state, n_scenes, s.off, s.cursor, s.members,
                                                  s.spheres, s.drones);
    return cudaGetLastError();
}

cudaError_t launch_swarm_proximity(int n, const int* scene_of_agent, const float* state, int n_scenes,
                                   const SwarmScratch& s, float radius, float* dist, int* other, int* n_collide,
                                   cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int b = 128, g = (int)(((long long)n * 32 + b - 1) / b);
    swarm_proximity_kernel<<<g, b, 0, st>>>(n, scene_of_agent, state, n_scenes, s.off, s.spheres, radius, dist, other,
                                            n_collide);
    return cudaGetLastError();
}

}  // namespace vf

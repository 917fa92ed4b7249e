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

// 10 bits of v spread three apart (bit i to bit 3 i).
__device__ __forceinline__ unsigned spread3(unsigned v) {
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ float block_reduce(float v, bool take_max, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, v, o);
        v = take_max ? fmaxf(v, w) : fminf(v, w);
    }
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float r = red[0];
    for (int k = 1; k < nw; ++k) r = take_max ? fmaxf(r, red[k]) : fminf(r, red[k]);
    return r;
}

// One CTA per scene: a scene with more than kSwarmGroupMin members (and at
// most kSwarmSortMax) has them ordered along the Morton curve of their
// centres (bitonic sort of (code, position) in shared memory, then an
// in-place permutation of the member and sphere lists), so that 32
// consecutive members lie close together; then every group of 32 gets the
// bounds of its members' centres.  Larger swarms keep the bucket order (their
// groups are looser, the result is the same).  Only the order of members
// within a scene changes, which neither the ray cast's closest-hit rule nor
// the proximity query depends on.
constexpr int kGroupThreads = 512;
__global__ void __launch_bounds__(kGroupThreads) swarm_group_kernel(const int* __restrict__ off,
                                                                    int* __restrict__ members,
                                                                    float4* __restrict__ spheres,
                                                                    float4* __restrict__ groups) {
    __shared__ unsigned long long key[kSwarmSortMax];
    __shared__ float red[kGroupThreads / 32];
    const int sid = blockIdx.x, tid = threadIdx.x;
    const int lo = off[sid], m = off[sid + 1] - lo;
    if (m <= kSwarmGroupMin) return;
    if (m <= kSwarmSortMax) {
        float bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int k = tid; k < m; k += kGroupThreads) {
            const float4 c = spheres[lo + k];
            bl[0] = fminf(bl[0], c.x), bl[1] = fminf(bl[1], c.y), bl[2] = fminf(bl[2], c.z);
            bh[0] = fmaxf(bh[0], c.x), bh[1] = fmaxf(bh[1], c.y), bh[2] = fmaxf(bh[2], c.z);
        }
        float L[3], S[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            L[j] = block_reduce(bl[j], false, red);
            const float h = block_reduce(bh[j], true, red);
            S[j] = h > L[j] ? 1023.0f / (h - L[j]) : 0.0f;
        }
        int p2 = 1;
        while (p2 < m) p2 <<= 1;
        for (int k = tid; k < p2; k += kGroupThreads) {
            unsigned long long v = ~0ull;  // padding sorts last
            if (k < m) {
                const float4 c = spheres[lo + k];
                const unsigned code = (spread3((unsigned)((c.x - L[0]) * S[0])) << 2) |
                                      (spread3((unsigned)((c.y - L[1]) * S[1])) << 1) |
                                      spread3((unsigned)((c.z - L[2]) * S[2]));
                v = ((unsigned long long)code << 32) | (unsigned)k;
            }
            key[k] = v;
        }
        __syncthreads();
        for (int size = 2; size <= p2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int k = tid; k < p2; k += kGroupThreads) {
                    const int partner = k ^ stride;
                    if (partner > k) {
                        const bool up = (k & size) == 0;
                        const unsigned long long a = key[k], b = key[partner];
                        if ((a > b) == up) {
                            key[k] = b;
                            key[partner] = a;
                        }
                    }
                }
                __syncthreads();
            }
        // permute in place: everything is read before anything is written
        constexpr int kPer = kSwarmSortMax / kGroupThreads;
        float4 sv[kPer];
        int mv[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int k = tid + r * kGroupThreads;
            if (k < m) {
                const int src = (int)(key[k] & 0xFFFFFFFFu);
                sv[r] = spheres[lo + src];
                mv[r] = members[lo + src];
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int k = tid + r * kGroupThreads;
            if (k < m) {
                spheres[lo + k] = sv[r];
                members[lo + k] = mv[r];
            }
        }
        __syncthreads();
    }
    // group boxes, one warp per group of 32 consecutive members
    const int lane = tid & 31, warp = tid >> 5, n_g = (m + 31) / 32;
    float4* gb = groups + 2 * ((size_t)lo / 32 + sid);
    for (int g = warp; g < n_g; g += kGroupThreads / 32) {
        const int k = g * 32 + lane;
        float4 c = k < m ? spheres[lo + k] : spheres[lo + g * 32];
        float l0 = c.x, l1 = c.y, l2 = c.z, h0 = c.x, h1 = c.y, h2 = c.z;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            l0 = fminf(l0, __shfl_xor_sync(0xffffffffu, l0, o));
            l1 = fminf(l1, __shfl_xor_sync(0xffffffffu, l1, o));
            l2 = fminf(l2, __shfl_xor_sync(0xffffffffu, l2, o));
            h0 = fmaxf(h0, __shfl_xor_sync(0xffffffffu, h0, o));
            h1 = fmaxf(h1, __shfl_xor_sync(0xffffffffu, h1, o));
            h2 = fmaxf(h2, __shfl_xor_sync(0xffffffffu, h2, o));
        }
        if (lane == 0) {
            gb[2 * g] = make_float4(l0, l1, l2, 0.0f);
            gb[2 * g + 1] = make_float4(h0, h1, h2, 0.0f);
        }
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

cudaError_t launch_swarm_groups(int n, int n_scenes, SwarmScratch& s, cudaStream_t st) {
    if (n <= kSwarmGroupMin || n_scenes <= 0) return cudaSuccess;
    swarm_group_kernel<<<n_scenes, kGroupThreads, 0, st>>>(s.off, s.members, s.spheres, s.groups);
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

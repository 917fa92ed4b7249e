// Persistent ray-cast renderer: 64x64 FP32 depth + uint8 RGB per agent
// (the depth and colour sensors of Sec. III-B), sm_103a.
//
// One warp renders one image tile of 32 * RPL pixels (one or two rays per
// lane) and pulls the next (agent, tile) item from a global counter, so scenes
// of very different size load-balance inside one launch.  The warp walks its
// agent's scene BVH as a packet: a node's 64 bytes are either fetched by four
// lanes with coalesced float4 loads into the warp's shared-memory slot and read
// back by every lane (STAGE), or loaded by every lane from the same address (a
// broadcast through L1).  Each lane slab-tests both child boxes against its own
// rays and a warp vote (__ballot_sync) decides which children any ray needs;
// the near one along the tile's central ray (by the node's stored split axis)
// is walked first, the other pushed on the warp's stack (shared memory or a
// stack spread over the lanes' registers).  Leaves (up to 3 triangles, 9
// float4, contiguous in leaf order) are fetched the same way and every lane runs
// Moller-Trumbore on them.  The walk ends when the stack is empty; the votes
// skip every subtree that no ray of the tile can reach before its current
// closest hit.  The scene's few large triangles (walls, floors) are kept out of
// the tree; each tile first culls them against the bounding box of its ray
// segments and tests the rest, which also seeds every ray's closest hit.
//
// Result per ray: the closest hit with max_depth >= t > 1e-6 and, among equal
// FP32 t, the lowest triangle id (order-independent, so every configuration
// gives identical images).  Stores are packed: depth as one float per lane,
// colour bytes gathered in shared memory and written as 32-bit words.
#include "common.cuh"
#include "launch.h"

namespace vf {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kTmin = 1e-6f;
constexpr int kIterCap = 1 << 18;  // node + leaf visits per work item
constexpr int kStack = 64;  // traversal stack entries of the counted, streamed, multi-agent and 4-wide builds
constexpr int kWarpsPerCta = 4;
constexpr int kSplit = 4;  // sub-packets (quarter tiles) of a very heavy tile

struct Ray {
    float o[3], d[3], inv[3], ood[3];
    float best_t;
    int best_id;
    bool live;
};

__device__ __forceinline__ void mt_test(Ray& r, const float4 a, const float4 b, const float4 c) {
    // a = (v0, id), b = e1, c = e2; two-sided Moller-Trumbore
    const float px = r.d[1] * c.z - r.d[2] * c.y;
    const float py = r.d[2] * c.x - r.d[0] * c.z;
    const float pz = r.d[0] * c.y - r.d[1] * c.x;
    const float det = b.x * px + b.y * py + b.z * pz;
    // approximate reciprocal (about 1 ulp): t, u, v move by ~1e-7 relative,
    // far inside the depth tolerance and the 1e-5 edge band of stated ties
    const float inv = __fdividef(1.0f, det);
    const float sx = r.o[0] - a.x, sy = r.o[1] - a.y, sz = r.o[2] - a.z;
    const float u = (sx * px + sy * py + sz * pz) * inv;
    const float qx = sy * b.z - sz * b.y;
    const float qy = sz * b.x - sx * b.z;
    const float qz = sx * b.y - sy * b.x;
    const float v = (r.d[0] * qx + r.d[1] * qy + r.d[2] * qz) * inv;
    const float t = (c.x * qx + c.y * qy + c.z * qz) * inv;
    const int id = __float_as_int(a.w);
    const bool hit = det != 0.0f && u >= 0.0f && v >= 0.0f && u + v <= 1.0f && t > kTmin &&
                     (t < r.best_t || (t == r.best_t && (unsigned)id < (unsigned)r.best_id));
    if (hit) {
        r.best_t = t;
        r.best_id = id;
    }
}

// Ray against drone j's box (multi-agent mode): move the ray into the drone's
// frame (c_k = body axis k with the centre's k-th world coordinate in w) and
// slab-test the half extents h.  The hit is the entry distance, or the exit
// distance when the ray starts inside; it competes with the triangles under
// the same (t, unsigned id) order with id = INT_MIN + j.
__device__ __forceinline__ void drone_test(Ray& r, const float4 c0, const float4 c1, const float4 c2, const float h[3],
                                           int code) {
    const float dx = r.o[0] - c0.w, dy = r.o[1] - c1.w, dz = r.o[2] - c2.w;
    const float4 c[3] = {c0, c1, c2};
    float tn = -INFINITY, tf = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ol = c[k].x * dx + c[k].y * dy + c[k].z * dz;
        const float dl = c[k].x * r.d[0] + c[k].y * r.d[1] + c[k].z * r.d[2];
        const float inv = 1.0f / (fabsf(dl) > 1e-20f ? dl : copysignf(1e-20f, dl));
        const float t0 = (-h[k] - ol) * inv, t1 = (h[k] - ol) * inv;
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
    const float t = tn > kTmin ? tn : tf;
    const bool hit = tn <= tf && t > kTmin && (t < r.best_t || (t == r.best_t && (unsigned)code < (unsigned)r.best_id));
    if (hit && r.live) {
        r.best_t = t;
        r.best_id = code;
    }
}

// Slab test of one child box against a ray; entry distance in tn.
__device__ __forceinline__ bool slab(const Ray& r, float lx, float ly, float lz, float hx, float hy, float hz,
                                     float& tn) {
    const float x0 = fmaf(lx, r.inv[0], -r.ood[0]), x1 = fmaf(hx, r.inv[0], -r.ood[0]);
    const float y0 = fmaf(ly, r.inv[1], -r.ood[1]), y1 = fmaf(hy, r.inv[1], -r.ood[1]);
    const float z0 = fmaf(lz, r.inv[2], -r.ood[2]), z1 = fmaf(hz, r.inv[2], -r.ood[2]);
    tn = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), 0.0f));
    const float tf = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), r.best_t));
    return tn <= tf;  // a dead ray has best_t < 0, so it passes no box
}

// 32 bytes in one read-only load (sm_100 and later): half a binary node, whose
// records are 64-byte aligned.
__device__ __forceinline__ void ld_nc_v8(const float4* p, float4& a, float4& b) {
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}

// Fetch `count` (<= 4) consecutive triangle records and test every ray.
template <int RPL, bool STAGE>
__device__ __forceinline__ void test_leaf(Ray (&ray)[RPL], const float4* __restrict__ src, int count, float4* stage,
                                          int lane) {
    if (STAGE) {
        __syncwarp();
        if (lane < 3 * count) stage[lane] = __ldg(src + lane);
        __syncwarp();
        for (int k = 0; k < count; ++k) {
            const float4 a = stage[3 * k], b = stage[3 * k + 1], c = stage[3 * k + 2];
#pragma unroll
            for (int q = 0; q < RPL; ++q) mt_test(ray[q], a, b, c);
        }
    } else {
        for (int k = 0; k < count; ++k) {
            const float4 a = __ldg(src + 3 * k), b = __ldg(src + 3 * k + 1), c = __ldg(src + 3 * k + 2);
#pragma unroll
            for (int q = 0; q < RPL; ++q) mt_test(ray[q], a, b, c);
        }
    }
}

// Minimum / maximum over the full warp in one instruction (sm_100 and later:
// redux.sync on f32); exact, so the same as a shuffle ladder.
__device__ __forceinline__ float warp_min(float v) {
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float warp_max(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// Noise draws of one pixel: 64 consecutive outputs of the generator starting
// at ((frame * n_agents + agent) * H * W + pixel) * 64 (mod 2^64).  Slots: depth
// 0-7, colour channel c 8 + 8c .. 15 + 8c, segmentation labels 32-39,
// segmentation dropout 40.  Within a block of 8: Gaussian 0-1, speckle 2-3,
// shot 4-5, salt & pepper 6-7.
__device__ __forceinline__ float unit_open(unsigned long long x) {
    return ((float)(x >> 40) + 0.5f) * (1.0f / 16777216.0f);
}
__device__ __forceinline__ float unit_half_open(unsigned long long x) { return (float)(x >> 40) * (1.0f / 16777216.0f); }
// Box-Muller with the hardware logarithm and cosine (__logf, __cosf).  The
// hardware logarithm's error is absolute (a few 1e-7), so near u1 = 1, where
// -log u1 itself is small, -log u1 comes from the Mercator series of
// -log(1 - v) in v = 1 - u1 (exact in FP32 for these uniforms) instead: five
// terms for v < 1/16 keep it within 2e-7 relative, and the logarithm's
// relative error elsewhere stays below 6e-6, so a draw moves by under 2e-5
// absolute, far inside the depth tolerance and the rounding band of colour
// and labels.  cos(2 pi u2) is taken as -cos(2 pi (u2 - 1/2)), whose argument
// lies in [-pi, pi), the range the hardware cosine is accurate on.  With every
// noise model on the render is 9% faster than with logf / cospif.
__device__ __forceinline__ float gauss_at(unsigned long long seed, unsigned long long i) {
    const float u1 = unit_open(splitmix64_at(seed, i)), u2 = unit_half_open(splitmix64_at(seed, i + 1));
    const float v = 1.0f - u1;
    const float series = v * (1.0f + v * (0.5f + v * (1.0f / 3.0f + v * (0.25f + v * 0.2f))));
    const float nl = v < 0.0625f ? series : -__logf(u1);
    return -sqrtf(2.0f * nl) * __cosf(6.2831853f * (u2 - 0.5f));
}
// shot (Gaussian form: mean k x, variance k x, scaled back), additive, speckle,
// salt & pepper, then clamp to [0, hi]
__device__ float noisy(float x, float hi, float gs, float sp, float shot, float sandp, unsigned long long seed,
                       unsigned long long b) {
    if (shot > 0.0f) {
        const float lam = shot * x;
        x = (lam + sqrtf(fmaxf(lam, 0.0f)) * gauss_at(seed, b + 4)) / shot;
    }
    if (gs > 0.0f) x += gs * gauss_at(seed, b);
    if (sp > 0.0f) x *= 1.0f + sp * gauss_at(seed, b + 2);
    if (sandp > 0.0f && unit_half_open(splitmix64_at(seed, b + 6)) < sandp)
        x = unit_half_open(splitmix64_at(seed, b + 7)) < 0.5f ? 0.0f : hi;
    return fminf(fmaxf(x, 0.0f), hi);
}

// Warp-wide copy of `bytes` from device memory (read through L2, where other
// warps' stores are visible after their fence) to host memory.
__device__ __noinline__ void copy_out(const uint8_t* src, uint8_t* dst, size_t bytes, int lane) {
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) | bytes) & 15) == 0) {
        const uint4* s = reinterpret_cast<const uint4*>(src);
        uint4* d = reinterpret_cast<uint4*>(dst);
        for (size_t i = lane; i < bytes / 16; i += 32) d[i] = __ldcg(s + i);
    } else {
        for (size_t i = lane; i < bytes; i += 32) dst[i] = __ldcg(src + i);
    }
}

// Bounds of a tile's ray segments (per-lane bounds reduced over the warp), padded.
__device__ __forceinline__ void tile_bounds(const float flo[3], const float fhi[3], float blo[3], float bhi[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float lo = warp_min(flo[j]), hi = warp_max(fhi[j]);
        const float pad = 1e-3f * (hi - lo) + 1e-4f;
        blo[j] = lo - pad;
        bhi[j] = hi + pad;
    }
}

__device__ __forceinline__ float comp4(const float4& v, int s) { return s == 0 ? v.x : s == 1 ? v.y : s == 2 ? v.z : v.w; }

// Identity of a launch's item layout: item ids are (rank * n + agent), so the
// costs of one launch describe the next only when both agree on all three.
__host__ __device__ __forceinline__ unsigned long long sched_shape(int tiles_x, int tiles_y, int n) {
    return (unsigned long long)tiles_x | ((unsigned long long)tiles_y << 16) | ((unsigned long long)(unsigned)n << 32);
}

// Tile rows are ranked from the image centre outwards (rank row 0 is row
// tiles_y / 2, then the rows above and below it in turn): tile row of a rank
// row, and back.
__device__ __forceinline__ int tile_row_of(int rr, int tiles_y) {
    const int mid = tiles_y >> 1;
    return (rr & 1) ? mid - 1 - (rr >> 1) : mid + (rr >> 1);
}
__device__ __forceinline__ int rank_row_of(int ty, int tiles_y) {
    const int mid = tiles_y >> 1;
    return ty >= mid ? 2 * (ty - mid) : 2 * (mid - 1 - ty) + 1;
}

__device__ __forceinline__ void quat_rotation(float w, float x, float y, float z, float R[3][3]) {
    R[0][0] = w * w + x * x - y * y - z * z;
    R[0][1] = 2.0f * (x * y - w * z);
    R[0][2] = 2.0f * (x * z + w * y);
    R[1][0] = 2.0f * (x * y + w * z);
    R[1][1] = w * w - x * x + y * y - z * z;
    R[1][2] = 2.0f * (y * z - w * x);
    R[2][0] = 2.0f * (x * z - w * y);
    R[2][1] = 2.0f * (y * z + w * x);
    R[2][2] = w * w - x * x - y * y + z * z;
}

// Files the coming launch's work items into the cost buckets, one thread per
// tile (a warp holds 32 tiles of one agent when the agent has that many).  A
// tile's estimate is the previous launch's cost of the image region its rays
// looked at then: the tile's centre direction is carried from the agent's
// current camera attitude into the previous one (in one control step an agent
// turns by up to a few pixels but moves a centimetre or so, so the rotation
// alone moves the image), and the previous tiles that the moved tile overlaps
// contribute by overlap area; parts outside the previous image count at the
// mean cost.  The launch's order only changes which warp renders which tile
// when, never a pixel's value.
__global__ void __launch_bounds__(256) sched_estimate_kernel(RenderArgs A, int TW, int TH, float split) {
    // the ray cast that follows may start its prologue now; everything this
    // kernel reads was written by earlier stream work, so wait for it first
    // (every thread, before any early exit: the ray cast's own wait relies on
    // this kernel finishing only after that work)
    asm volatile("griddepcontrol.launch_dependents;");
    const int lane = threadIdx.x & 31;
    const int n = A.n_agents;
    const int W = A.cam.W, H = A.cam.H;
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH, tiles = tiles_x * tiles_y;
    const long long total = (long long)n * tiles;
    {
        // while the previous kernel (the dynamics step) finishes: pull the last
        // launch's costs and attitudes into L2 (a hint, no data is read yet)
        const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        if (t * 32 < total && total <= A.sched_cap) asm volatile("prefetch.global.L2 [%0];" ::"l"(A.cost + t * 32));
        if (t * 8 < n && n <= A.sched_cap) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(A.pose + t * 8));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(A.pose + (size_t)A.sched_cap + t * 8));
        }
        if (t == 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(A.sched));
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (total > A.sched_cap) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // agent-major: t = agent * tiles + p
    const bool act = t < total;
    const unsigned ua = act ? (unsigned)t / (unsigned)tiles : 0u;  // total < 2^31
    const int agent = (int)ua, p = act ? (int)((unsigned)t - ua * (unsigned)tiles) : 0;
    unsigned long long* S = A.sched;
    const unsigned long long ep = S[kSchedEpoch];
    const bool valid = S[kSchedTotal] == (unsigned long long)total && S[kSchedShape] == sched_shape(tiles_x, tiles_y, n);
    const float mean = valid ? (float)S[(ep + 1) & 1] / (float)total : 0.0f;
    int b = -1;
    unsigned item = 0;
    if (act) {
        const float* st = A.state;
        float qw = __ldg(st + 6 * n + agent), qx = __ldg(st + 7 * n + agent), qy = __ldg(st + 8 * n + agent),
              qz = __ldg(st + 9 * n + agent);
        const float q2 = qw * qw + qx * qx + qy * qy + qz * qz;
        const float qi = q2 > 0.0f ? rsqrtf(q2) : 0.0f;
        qw *= qi;
        qx *= qi;
        qy *= qi;
        qz *= qi;
        const int tx = p % tiles_x, ty = p / tiles_x;
        item = (unsigned)((long long)(rank_row_of(ty, tiles_y) * tiles_x + tx) * n + agent);
        // attitudes are double-buffered by epoch: this launch reads the
        // previous launch's slot and records its own in the other
        if (p == 0) A.pose[(size_t)(ep & 1) * A.sched_cap + agent] = make_float4(qw, qx, qy, qz);
        if (mean > 0.0f && q2 > 0.0f) {
            const float4 qo = A.pose[(size_t)((ep + 1) & 1) * A.sched_cap + agent];
            float Rn[3][3], Ro[3][3];
            quat_rotation(qw, qx, qy, qz, Rn);
            quat_rotation(qo.x, qo.y, qo.z, qo.w, Ro);
            const float pix = A.cam.pix, area = (float)(TW * TH);
            // tile centre in continuous pixel coordinates, its body-frame direction
            const float u = (tx + 0.5f) * TW, v = (ty + 0.5f) * TH;
            const float d[3] = {1.0f, -(2.0f * u - W) * 0.5f * pix, -(2.0f * v - H) * 0.5f * pix};
            // world direction, then the previous body frame's
            float w[3], e[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) w[i] = Rn[i][0] * d[0] + Rn[i][1] * d[1] + Rn[i][2] * d[2];
#pragma unroll
            for (int i = 0; i < 3; ++i) e[i] = Ro[0][i] * w[0] + Ro[1][i] * w[1] + Ro[2][i] * w[2];
            float est = mean;
            if (e[0] > 1e-3f) {
                // the moved tile's corner in the previous image
                const float x0 = 0.5f * W - e[1] / (e[0] * pix) - 0.5f * TW;
                const float y0 = 0.5f * H - e[2] / (e[0] * pix) - 0.5f * TH;
                if (fabsf(x0) < 4.0f * W && fabsf(y0) < 4.0f * H) {
                    const int ox0 = (int)floorf(x0 / TW), oy0 = (int)floorf(y0 / TH);
                    float acc = 0.0f, cov = 0.0f;
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            const int ox = ox0 + dx, oy = oy0 + dy;
                            if (ox < 0 || oy < 0 || ox >= tiles_x || oy >= tiles_y) continue;
                            const float wx = fminf(x0 + TW, (float)((ox + 1) * TW)) - fmaxf(x0, (float)(ox * TW));
                            const float wy = fminf(y0 + TH, (float)((oy + 1) * TH)) - fmaxf(y0, (float)(oy * TH));
                            if (wx <= 0.0f || wy <= 0.0f) continue;
                            const long long it = (long long)(rank_row_of(oy, tiles_y) * tiles_x + ox) * n + agent;
                            acc += wx * wy * (float)A.cost[it];
                            cov += wx * wy;
                        }
                    est = (acc + fmaxf(area - cov, 0.0f) * mean) / area;
                }
            }
            b = est > split * mean   ? 0
                : est > 2.0f * mean  ? 1
                : est > 1.25f * mean ? 2
                : est > 0.8f * mean  ? 3
                : est > 0.5f * mean  ? 4
                : est > 0.25f * mean ? 5
                                     : 6;
        }
    }
    // warp-aggregated filing: lane k reserves the warp's slots in bucket k,
    // all buckets' atomics in flight at once
    unsigned mine = 0u, cnt_k = 0u;
#pragma unroll
    for (int k = 0; k < kBuckets; ++k) {
        const unsigned m = __ballot_sync(kFull, b == k);
        if (b == k) mine = m;
        if (lane == k) cnt_k = (unsigned)__popc(m);
    }
    unsigned long long base = 0;
    if (lane < kBuckets && cnt_k > 0) base = atomicAdd(&S[kSchedLen + lane], (unsigned long long)cnt_k);
    const unsigned long long my_base = __shfl_sync(kFull, base, b < 0 ? 0 : b);
    if (b >= 0) {
        const unsigned long long slot = my_base + (unsigned long long)__popc(mine & ((1u << lane) - 1u));
        if (slot < (unsigned long long)A.sched_cap) A.heavy[(size_t)b * A.sched_cap + slot] = item;
    }
}

// STACK: the warp's traversal stack entries.  In registers a stack of 32 takes
// one register per lane (entry k in lane k), 64 take two; in shared memory it
// is STACK ints per warp.  A scene deeper than the stack is refused on the host.
// Resident CTAs per SM the register budget is set for: 8 (64 registers) for
// one ray per lane, 9 (56) for the streamed build, whose host stores and
// completion fences gain from the extra warps (environment step +1.5%, while
// the device-only render loses 2% at 9), 6 for two rays per lane or 4-wide nodes.
template <int TW, int TH, int RPL, bool SMEM_STACK, bool STAGE, bool COUNT, bool WIDE, int EXTRA, int STACK>
__global__ void __launch_bounds__(32 * kWarpsPerCta, (RPL == 1 && !WIDE) ? (EXTRA == 1 ? 9 : 8) : 6)
    raycast_kernel(RenderArgs A) {
    static_assert(STACK > 0 && STACK <= 64 && (SMEM_STACK || STACK % 32 == 0), "stack depth");
    static_assert(TW * TH == 32 * RPL, "tile must hold 32 * RPL pixels");
    extern __shared__ float4 smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* stage = smem + warp * 12;
    int* sstack = reinterpret_cast<int*>(smem + kWarpsPerCta * 12) + warp * STACK;
    uint8_t* rgbstage = reinterpret_cast<uint8_t*>(reinterpret_cast<int*>(smem + kWarpsPerCta * 12) +
                                                   kWarpsPerCta * STACK) + warp * (32 * RPL * 3);

    const int W = A.cam.W, H = A.cam.H;
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    const int tiles = tiles_x * tiles_y;
    const long long total = (long long)A.n_agents * tiles;
    // COUNT statistics: per work item (warp) and per ray (what each ray's own walk needs)
    long long c_nodes = 0, c_tris = 0, c_large = 0, c_items = 0, c_need_nodes = 0, c_need_tris = 0;

    if (A.prefetch_l2) {
        // After an L2 flush the first walks would pay DRAM latency on every node of
        // their dependent chains; the whole grid streams the scenes into L2 at
        // once instead (one 128-byte line per prefetch, many in flight).
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)gridDim.x * blockDim.x;
        for (int sc = 0; sc < A.n_scenes; ++sc) {
            const SceneRow& r = A.table[sc];
            if (!r.live) continue;
            const char* bases[3] = {(const char*)r.nodes, (const char*)r.tris, (const char*)r.large};
            const long long lens[3] = {(long long)r.n_nodes * 64, (long long)r.n_tree_tris * 48,
                                       (long long)r.n_large * 48};
#pragma unroll
            for (int k = 0; k < 3; ++k)
                for (long long off = tid * 128; off < lens[k]; off += nthreads * 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(bases[k] + off));
        }
    }
    // launched as a programmatic dependent of the estimate kernel when
    // scheduled: the prefetch above overlaps it, nothing produced by earlier
    // stream work is read before this point
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const unsigned long long noise_frame = A.noise.enabled ? *A.noise_frame : 0ull;
    // Longest-first order: sched_estimate_kernel, launched just before, filed
    // every tile of this launch into a cost bucket (kBuckets) by the previous
    // launch's tile costs moved to the current camera poses; this launch hands
    // out bucket 0 first, each tile as kSplit quarter-tile sub-packets on
    // separate warps (a quarter walks only its own rays' paths, which shortens
    // the longest dependent chain of node fetches), then the other buckets
    // whole, costliest first.  A last sweep renders whatever no bucket held
    // (entries of a concurrent launch sharing the buffers, or no estimate at
    // all): by chunks of 32 items checked against this launch's done marks
    // when the buckets held every item, else item by item in natural order
    // (centre rows first without hints, edge rows first with partial ones).
    const bool sched = A.sched != nullptr && total <= A.sched_cap;
    // A launch that streams its bands to the host interleaves buckets 1-3 with
    // natural-order items one for one: a band is complete only when all its
    // tiles are, so taking every bucket first would hold back the download
    // until late in the launch.  Both sides claim a tile by exchanging its
    // done mark, so no tile is rendered twice.
    const bool weave = EXTRA >= 1 && sched && A.band_done != nullptr;
    // Splitting pays only when the launch is short enough for its longest tile
    // to matter: at most 12 tiles per resident warp.
    const bool allow_split = total <= 12ll * gridDim.x * kWarpsPerCta;
    // Claim arithmetic is 32-bit: the host admits fewer than 2^31 items counted
    // with 4 x 2-pixel tiles, so a launch has total < 2^29 items (its tiles hold
    // 32 pixels or more); bucket ends are clamped below 2^31, and the counter
    // (at most the bucket ends + total + one overshoot per warp) stays below 2^32.
    __shared__ unsigned s_end[kBuckets];  // cumulative ends of the buckets in the counter's range
    __shared__ unsigned s_entries;        // bucket entries (a split tile counts once)
    const unsigned utotal = (unsigned)total;
    unsigned long long mark = 0;
    unsigned ep = 0;
    if (sched) {
        ep = (unsigned)A.sched[kSchedEpoch];
        mark = ((unsigned long long)A.launch_id << 32) | ep;
        if (threadIdx.x == 0) {
            long long end = 0, entries = 0;
            for (int b = 0; b < kBuckets; ++b) {
                const long long len = (long long)min(A.sched[kSchedLen + b], (unsigned long long)total);
                end += (b == 0 && allow_split) ? len * kSplit : len;
                entries += len;
                s_end[b] = (unsigned)min(end, 0x7FFFFFFFll);
            }
            s_entries = (unsigned)min(entries, 0x7FFFFFFFll);
        }
    } else if (threadIdx.x == 0) {
        for (int b = 0; b < kBuckets; ++b) s_end[b] = 0;
        s_entries = 0;
    }
    __syncthreads();
    const bool hinted = s_end[kBuckets - 1] > 0;
    // the buckets held as many entries as the launch has items: the sweep only
    // checks done marks, 32 items per claim
    const bool sweep = !weave && s_entries >= utotal;
    unsigned pend = 0u;  // sweep: items of the warp's chunk that are still to render
    unsigned pend_base = 0;
    for (;;) {
        int item = 0;  // -1: nothing to render this round; utotal: no work left
        int sub = -1;
        int chunk = -1;
        if (pend) {
            item = (int)(pend_base + (unsigned)(__ffs(pend) - 1));
            pend &= pend - 1;
        } else {
            if (lane == 0) {
                const unsigned k = atomicAdd(A.counter, 1u);
                // position kb in the bucket lists, or a natural-order item at nat
                bool in_buckets = false;
                unsigned kb = 0, nat = 0;
                if (!weave) {
                    in_buckets = k < s_end[kBuckets - 1];
                    if (in_buckets) kb = k;
                    else nat = k - s_end[kBuckets - 1];
                } else if (k < s_end[0]) {
                    in_buckets = true;
                    kb = k;
                } else {
                    // a streamed launch interleaves the heavy buckets 1.. with the
                    // natural order, which also covers the cheap buckets' tiles
                    const unsigned r = k - s_end[0], pair = s_end[kHeavyBuckets - 1] - s_end[0];
                    if ((r >> 1) < pair) {
                        in_buckets = (r & 1) == 0;
                        if (in_buckets) kb = s_end[0] + (r >> 1);
                        else nat = r >> 1;
                    } else {
                        nat = r - pair;
                    }
                }
                if (!in_buckets && sweep) {
                    chunk = (int)min(nat, 0x7FFFFFFFu);
                } else if (in_buckets) {
                    int b = 0;
                    while (kb >= s_end[b]) ++b;
                    const unsigned j = kb - (b == 0 ? 0u : s_end[b - 1]);
                    const unsigned* list = A.heavy + (size_t)b * A.sched_cap;
                    unsigned it;
                    if (b == 0 && allow_split) {
                        it = list[j / kSplit];
                        sub = (int)(j % kSplit);
                    } else {
                        it = list[j];
                    }
                    // an entry from a concurrent launch of another size may not fit this one
                    item = it < utotal ? (int)it : -1;
                    if (item >= 0) {
                        if (b == 0 || !weave) __stcg(A.done + it, mark);
                        else if (atomicExch(A.done + it, mark) == mark) item = -1;  // taken in natural order
                    }
                } else {
                    // with hints the natural phase holds only tiles the last launch
                    // found cheap, and taking the edge rows first measured faster
                    // (0.8% with moving poses at 4x8 tiles); without hints the
                    // centre rows, where most costly tiles lie, go first
                    const unsigned v = (hinted && !weave && nat < utotal) ? utotal - 1 - nat : nat;
                    item = (int)min(v, utotal);  // utotal: no work left
                    if (v < utotal) {
                        if (weave) {
                            if (atomicExch(A.done + v, mark) == mark) item = -1;  // taken from a bucket
                        } else if (sched && __ldcg(A.done + v) == mark) {
                            item = -1;  // done from a bucket
                        }
                    }
                }
            }
            item = __shfl_sync(kFull, item, 0);
            sub = __shfl_sync(kFull, sub, 0);
            chunk = __shfl_sync(kFull, chunk, 0);
            if (chunk >= 0) {
                if ((unsigned)chunk >= (utotal + 31u) / 32u) break;
                const unsigned it = (unsigned)chunk * 32u + (unsigned)lane;
                pend = __ballot_sync(kFull, it < utotal && __ldcg(A.done + it) != mark);
                pend_base = (unsigned)chunk * 32u;
                continue;
            }
        }
        if (item < 0) continue;
        if ((unsigned)item >= utotal) break;
        // after a device-detected fault every warp stops taking work: the error
        // word is read here and tested when the item is done, so the read's
        // latency overlaps the item
        int err_seen = 0;
        if (lane == 0) asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(err_seen) : "l"(A.err));
        // Item ids run tile position by tile position across all agents, tile
        // rows from the image centre outwards: rows near the horizon (long rays
        // through clutter) are the costly ones, floor and ceiling rows the cheap
        // ones.
        // item < total < 2^31 (the host refuses larger launches): 32-bit divisions
        const unsigned uitem = (unsigned)item, un = (unsigned)A.n_agents, utx = (unsigned)tiles_x;
        const unsigned urank = uitem / un;
        const int agent = (int)(uitem - urank * un);
        const unsigned urow = urank / utx;
        const int ty = tile_row_of((int)urow, tiles_y);
        const int tx0 = (int)(urank - urow * utx) * TW, ty0 = ty * TH;
        const int sid = __ldg(A.scene_of_agent + agent);
        const bool scene_ok = sid >= 0 && sid < A.n_scenes && A.table[sid].live;
        if (!scene_ok && lane == 0) set_error(A.err, kDevErrNotFound);
        SceneRow row = {};
        if (scene_ok) row = A.table[sid];

        // camera pose of this agent (uniform loads)
        const float* st = A.state;
        const int n = A.n_agents;
        const float px = __ldg(st + agent), py = __ldg(st + n + agent), pz = __ldg(st + 2 * n + agent);
        const float qw = __ldg(st + 6 * n + agent), qx = __ldg(st + 7 * n + agent), qy = __ldg(st + 8 * n + agent),
                    qz = __ldg(st + 9 * n + agent);
        const float inv_n = 1.0f / (qw * qw + qx * qx + qy * qy + qz * qz);
        float R[3][3];
        R[0][0] = (qw * qw + qx * qx - qy * qy - qz * qz) * inv_n;
        R[0][1] = 2.0f * (qx * qy - qw * qz) * inv_n;
        R[0][2] = 2.0f * (qx * qz + qw * qy) * inv_n;
        R[1][0] = 2.0f * (qx * qy + qw * qz) * inv_n;
        R[1][1] = (qw * qw - qx * qx + qy * qy - qz * qz) * inv_n;
        R[1][2] = 2.0f * (qy * qz - qw * qx) * inv_n;
        R[2][0] = 2.0f * (qx * qz - qw * qy) * inv_n;
        R[2][1] = 2.0f * (qy * qz + qw * qx) * inv_n;
        R[2][2] = (qw * qw - qx * qx - qy * qy + qz * qz) * inv_n;
        const float o[3] = {
            px + R[0][0] * A.cam.cam_off[0] + R[0][1] * A.cam.cam_off[1] + R[0][2] * A.cam.cam_off[2],
            py + R[1][0] * A.cam.cam_off[0] + R[1][1] * A.cam.cam_off[1] + R[1][2] * A.cam.cam_off[2],
            pz + R[2][0] * A.cam.cam_off[0] + R[2][1] * A.cam.cam_off[1] + R[2][2] * A.cam.cam_off[2]};

        Ray ray[RPL];
        int pix_r[RPL], pix_c[RPL];
        bool mine_q[RPL];
        float flo[3] = {o[0], o[1], o[2]}, fhi[3] = {o[0], o[1], o[2]};  // ray-segment bounds
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int p = lane + 32 * q;
            const int c = tx0 + p % TW, r = ty0 + p / TW;
            pix_r[q] = r;
            pix_c[q] = c;
            const float dB[3] = {1.0f, -(float)(2 * c + 1 - W) * 0.5f * A.cam.pix,
                                 -(float)(2 * r + 1 - H) * 0.5f * A.cam.pix};
            Ray& ry = ray[q];
            const bool mine = sub < 0 || ((p % TW) / (TW / 2) == (sub & 1) && (p / TW) / (TH / 2) == (sub >> 1));
            mine_q[q] = mine;
            ry.live = scene_ok && r < H && c < W && mine;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                ry.o[j] = o[j];
                ry.d[j] = R[j][0] * dB[0] + R[j][1] * dB[1] + R[j][2] * dB[2];
                const float dd = fabsf(ry.d[j]) > 1e-20f ? ry.d[j] : copysignf(1e-20f, ry.d[j]);
                ry.inv[j] = 1.0f / dd;
                ry.ood[j] = ry.o[j] * ry.inv[j];
                if (ry.live) {
                    const float e = o[j] + ry.d[j] * A.cam.max_depth;
                    flo[j] = fminf(flo[j], e);
                    fhi[j] = fmaxf(fhi[j], e);
                }
            }
            // a dead ray (outside the image, another quarter, no scene) starts
            // behind its origin and so passes no box and no triangle test
            ry.best_t = ry.live ? A.cam.max_depth : -1.0f;
            ry.best_id = -1;
        }

        // Front-to-back order of a binary node's children: each node stores the
        // axis along which its children's centres lie farthest apart and which
        // child is the lower one there (its order word, 2 * axis + s); the tile's
        // central ray direction decides, per axis, whether the lower child comes
        // first.  Bit 2 * axis + s of near_bits is set when child 1 is the near
        // one.  The order changes which nodes the packet skips, never a result.
        unsigned near_bits;
        {
            const float cB[3] = {1.0f, -(float)(2 * tx0 + TW - W) * 0.5f * A.cam.pix,
                                 -(float)(2 * ty0 + TH - H) * 0.5f * A.cam.pix};
            near_bits = 0u;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float dj = R[j][0] * cB[0] + R[j][1] * cB[1] + R[j][2] * cB[2];
                near_bits |= (dj < 0.0f ? 1u : 2u) << (2 * j);
            }
        }
        int item_cost = 0;
        if (scene_ok) {
            // other drones of the scene (multi-agent mode): cull their bounding
            // spheres against the bounds of the tile's ray segments, then test
            // each survivor's box
            if (EXTRA == 2 && A.drones) {
                float blo[3], bhi[3];
                tile_bounds(flo, fhi, blo, bhi);
                const int m_lo = __ldg(A.swarm_off + sid), m_hi = __ldg(A.swarm_off + sid + 1);
                const float rad = A.swarm_radius;
                const float4 none = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(agent));
                // Side planes of the tile's frustum: through the camera origin and
                // the rays of two neighbouring corner pixels, normals (unit length)
                // pointing inward.  Every ray of the tile (or of a quarter of it) lies
                // in the cone of its corner pixels' rays.  An edge between two
                // corners that are the same pixel (a one-pixel-wide or -high tile)
                // gets a zero normal, which culls nothing: the cross product of a
                // ray with itself is not zero once the compiler fuses its products,
                // so the test is on the pixel indices.  Used for the larger
                // swarms (the grouped ones): 4,096 drones 6.08 -> 3.59 ms per step,
                // 1,024 0.94 -> 0.84 ms; at 256 the planes cost more than they save.
                const bool grouped = A.swarm_groups && m_hi - m_lo > kSwarmGroupMin;
                float fn[4][3] = {};
                if (grouped) {
                    const int cx[4] = {tx0, min(tx0 + TW, W) - 1, min(tx0 + TW, W) - 1, tx0};
                    const int cy[4] = {ty0, ty0, min(ty0 + TH, H) - 1, min(ty0 + TH, H) - 1};
                    float cd[4][3];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float b1 = -(float)(2 * cx[k] + 1 - W) * 0.5f * A.cam.pix;
                        const float b2 = -(float)(2 * cy[k] + 1 - H) * 0.5f * A.cam.pix;
#pragma unroll
                        for (int j = 0; j < 3; ++j) cd[k][j] = R[j][0] + R[j][1] * b1 + R[j][2] * b2;
                    }
                    const float mid[3] = {cd[0][0] + cd[2][0], cd[0][1] + cd[2][1], cd[0][2] + cd[2][2]};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float* u = cd[k];
                        const float* w = cd[(k + 1) & 3];
                        float nx = u[1] * w[2] - u[2] * w[1], ny = u[2] * w[0] - u[0] * w[2], nz = u[0] * w[1] - u[1] * w[0];
                        const float l2 = nx * nx + ny * ny + nz * nz;
                        const float sgn = nx * mid[0] + ny * mid[1] + nz * mid[2] < 0.0f ? -1.0f : 1.0f;
                        const bool same = cx[k] == cx[(k + 1) & 3] && cy[k] == cy[(k + 1) & 3];
                        const float inv = !same && l2 > 0.0f ? sgn * rsqrtf(l2) : 0.0f;
                        fn[k][0] = nx * inv;
                        fn[k][1] = ny * inv;
                        fn[k][2] = nz * inv;
                    }
                }
                // a sphere that lies wholly outside one side plane misses every
                // ray of the tile; the slack covers the planes' rounding
                auto in_frustum = [&](float x, float y, float z, float r) {
                    const float dx = x - o[0], dy = y - o[1], dz = z - o[2];
                    const float slack = 1.01f * r + 1e-3f * (1.0f + fabsf(dx) + fabsf(dy) + fabsf(dz));
                    bool in = true;
#pragma unroll
                    for (int k = 0; k < 4; ++k) in = in && fn[k][0] * dx + fn[k][1] * dy + fn[k][2] * dz >= -slack;
                    return in;
                };
                // members k0 .. k1 - 1 (at most 64): cull their bounding spheres
                // against the tile's bounds and frustum, test each survivor's box
                auto members = [&](int k0, int k1) {
                    float4 sph[2];
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        const int k = k0 + 32 * g + lane;
                        sph[g] = k < k1 ? __ldg(A.swarm_spheres + k) : none;
                    }
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        const int j = __float_as_int(sph[g].w);
                        const bool keep = j != agent && sph[g].x - rad <= bhi[0] && sph[g].x + rad >= blo[0] &&
                                          sph[g].y - rad <= bhi[1] && sph[g].y + rad >= blo[1] &&
                                          sph[g].z - rad <= bhi[2] && sph[g].z + rad >= blo[2] &&
                                          (!grouped || in_frustum(sph[g].x, sph[g].y, sph[g].z, rad));
                        unsigned mask = __ballot_sync(kFull, keep);
                        while (mask) {
                            const int src = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const int jj = __shfl_sync(kFull, j, src);
                            const float4 c0 = __ldg(A.drones + 3 * (size_t)jj), c1 = __ldg(A.drones + 3 * (size_t)jj + 1),
                                         c2 = __ldg(A.drones + 3 * (size_t)jj + 2);
#pragma unroll
                            for (int q = 0; q < RPL; ++q) drone_test(ray[q], c0, c1, c2, A.swarm_half, INT_MIN + jj);
                        }
                    }
                };
                if (grouped) {
                    // a larger swarm: cull its groups of 32 first (their centre
                    // bounds grown by the drones' radius)
                    const int n_g = (m_hi - m_lo + 31) / 32;
                    const float4* gb = A.swarm_groups + 2 * ((size_t)m_lo / 32 + sid);
                    for (int g0 = 0; g0 < n_g; g0 += 32) {
                        const int g = g0 + lane;
                        bool keep = false;
                        if (g < n_g) {
                            const float4 l = __ldg(gb + 2 * g), h = __ldg(gb + 2 * g + 1);
                            keep = l.x - rad <= bhi[0] && h.x + rad >= blo[0] && l.y - rad <= bhi[1] &&
                                   h.y + rad >= blo[1] && l.z - rad <= bhi[2] && h.z + rad >= blo[2];
                            // the group's sphere: its centre box's half diagonal plus the radius
                            const float ex = 0.5f * (h.x - l.x), ey = 0.5f * (h.y - l.y), ez = 0.5f * (h.z - l.z);
                            keep = keep && in_frustum(l.x + ex, l.y + ey, l.z + ez, sqrtf(ex * ex + ey * ey + ez * ez) + rad);
                        }
                        unsigned gm = __ballot_sync(kFull, keep);
                        while (gm) {
                            const int gg = g0 + __ffs(gm) - 1;
                            gm &= gm - 1;
                            const int k0 = m_lo + 32 * gg;
                            members(k0, min(k0 + 32, m_hi));
                        }
                    }
                } else {
                    for (int k0 = m_lo; k0 < m_hi; k0 += 64) members(k0, min(k0 + 64, m_hi));
                }
            }
            // large triangles: cull against the tile's ray-segment bounds, test the rest
            if (row.n_large > 0) {
                float blo[3], bhi[3];
                tile_bounds(flo, fhi, blo, bhi);
                for (int k0 = 0; k0 < row.n_large; k0 += 32) {
                    const int k = k0 + lane;
                    bool keep = false;
                    if (k < row.n_large) {
                        const float4 a = __ldg(row.large + 3 * k), b = __ldg(row.large + 3 * k + 1),
                                     c = __ldg(row.large + 3 * k + 2);
                        const float tl[3] = {fminf(a.x, fminf(a.x + b.x, a.x + c.x)),
                                             fminf(a.y, fminf(a.y + b.y, a.y + c.y)),
                                             fminf(a.z, fminf(a.z + b.z, a.z + c.z))};
                        const float th[3] = {fmaxf(a.x, fmaxf(a.x + b.x, a.x + c.x)),
                                             fmaxf(a.y, fmaxf(a.y + b.y, a.y + c.y)),
                                             fmaxf(a.z, fmaxf(a.z + b.z, a.z + c.z))};
                        keep = tl[0] <= bhi[0] && th[0] >= blo[0] && tl[1] <= bhi[1] && th[1] >= blo[1] &&
                               tl[2] <= bhi[2] && th[2] >= blo[2];
                    }
                    unsigned mask = __ballot_sync(kFull, keep);
                    while (mask) {
                        const int kk = k0 + __ffs(mask) - 1;
                        mask &= mask - 1;
                        test_leaf<RPL, false>(ray, row.large + 3 * (size_t)kk, 1, stage, lane);
                        if (COUNT) ++c_large;
                    }
                }
            }
            // BVH walk
            int cur = row.root;
            int sp = 0;
            int reg0 = 0, reg1 = 0;  // register stack: entry k in lane k % 32 of reg[k / 32]
            bool need[RPL];
            unsigned long long needmask[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                need[q] = ray[q].live;
                needmask[q] = 0ull;
            }
            int& iters = item_cost;
            while (cur != kEmptyRoot) {
                ++iters;
                int next = kEmptyRoot;
                if (WIDE && cur >= 0) {
                    // 4-wide node: SoA child boxes, codes in w[6]
                    const float4* wp = row.wide + 8 * (size_t)cur;
                    float4 w[7];
                    if (STAGE) {
                        __syncwarp();
                        if (lane < 7) stage[lane] = __ldg(wp + lane);
                        __syncwarp();
#pragma unroll
                        for (int k = 0; k < 7; ++k) w[k] = stage[k];
                    } else {
#pragma unroll
                        for (int k = 0; k < 7; ++k) w[k] = __ldg(wp + k);
                    }
                    float key[4];
                    int code[4], slot[4];
                    bool hq[RPL][4];
#pragma unroll
                    for (int c4 = 0; c4 < 4; ++c4) {
                        code[c4] = __float_as_int(comp4(w[6], c4));
                        slot[c4] = c4;
                        bool any = false;
#pragma unroll
                        for (int q = 0; q < RPL; ++q) {
                            float tn;
                            hq[q][c4] = code[c4] != kEmptyRoot &&
                                        slab(ray[q], comp4(w[0], c4), comp4(w[1], c4), comp4(w[2], c4),
                                             comp4(w[3], c4), comp4(w[4], c4), comp4(w[5], c4), tn);
                            any |= hq[q][c4];
                        }
                        const unsigned b = __ballot_sync(kFull, any);
                        // order key: distance from the common camera origin to the box centre
                        const float cx = 0.5f * (comp4(w[0], c4) + comp4(w[3], c4)) - o[0];
                        const float cy = 0.5f * (comp4(w[1], c4) + comp4(w[4], c4)) - o[1];
                        const float cz = 0.5f * (comp4(w[2], c4) + comp4(w[5], c4)) - o[2];
                        key[c4] = b ? cx * cx + cy * cy + cz * cz : 3.0e38f;
                    }
                    // sort the four (key, code, slot) triples ascending: 5 compare-exchanges
#define VF_CX(a, b)                                                                            \
    if (key[b] < key[a]) {                                                                     \
        const float tk = key[a]; key[a] = key[b]; key[b] = tk;                                 \
        const int tc = code[a]; code[a] = code[b]; code[b] = tc;                               \
        const int ts = slot[a]; slot[a] = slot[b]; slot[b] = ts;                               \
    }
                    VF_CX(0, 1) VF_CX(2, 3) VF_CX(0, 2) VF_CX(1, 3) VF_CX(1, 2)
#undef VF_CX
                    const int cnt = (key[0] < 3.0e38f) + (key[1] < 3.0e38f) + (key[2] < 3.0e38f) + (key[3] < 3.0e38f);
                    if (COUNT) {
                        ++c_nodes;
#pragma unroll
                        for (int q = 0; q < RPL; ++q) c_need_nodes += need[q] ? 1 : 0;
                    }
                    if (cnt > 0) {
                        if (sp + cnt - 1 > STACK) {
                            if (lane == 0) set_error(A.err, kDevErrTraversal);
                            break;
                        }
                        // push the farther hit children, farthest first
                        for (int j = cnt - 1; j >= 1; --j) {
                            const int far = j == 3 ? code[3] : j == 2 ? code[2] : code[1];
                            if (SMEM_STACK) {
                                if (lane == 0) sstack[sp] = far;
                            } else if (lane == (sp & 31)) {
                                if (STACK <= 32 || sp < 32) reg0 = far; else reg1 = far;
                            }
                            if (COUNT) {
                                const int sl = j == 3 ? slot[3] : j == 2 ? slot[2] : slot[1];
#pragma unroll
                                for (int q = 0; q < RPL; ++q) {
                                    const bool nf = need[q] && (sl == 0 ? hq[q][0] : sl == 1 ? hq[q][1] : sl == 2 ? hq[q][2] : hq[q][3]);
                                    needmask[q] = (needmask[q] & ~(1ull << sp)) | ((unsigned long long)nf << sp);
                                }
                            }
                            ++sp;
                        }
                        next = code[0];
                        if (COUNT) {
                            const int sl = slot[0];
#pragma unroll
                            for (int q = 0; q < RPL; ++q)
                                need[q] = need[q] && (sl == 0 ? hq[q][0] : sl == 1 ? hq[q][1] : sl == 2 ? hq[q][2] : hq[q][3]);
                        }
                    }
                } else if (cur >= 0) {
                    const float4* np = row.nodes + 4 * (size_t)cur;
                    float4 n0, n1, n2, n3;
                    if (STAGE) {
                        __syncwarp();
                        if (lane < 4) stage[lane] = __ldg(np + lane);
                        __syncwarp();
                        n0 = stage[0];
                        n1 = stage[1];
                        n2 = stage[2];
                        n3 = stage[3];
                    } else {
                        ld_nc_v8(np, n0, n1);
                        ld_nc_v8(np + 2, n2, n3);
                    }
                    bool h0 = false, h1 = false;
                    bool ha[RPL], hb[RPL];
#pragma unroll
                    for (int q = 0; q < RPL; ++q) {
                        float t0, t1;
                        ha[q] = slab(ray[q], n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, t0);
                        hb[q] = slab(ray[q], n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, t1);
                        h0 |= ha[q];
                        h1 |= hb[q];
                    }
                    const unsigned b0 = __ballot_sync(kFull, h0), b1 = __ballot_sync(kFull, h1);
                    const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
                    if (COUNT) {
                        ++c_nodes;
#pragma unroll
                        for (int q = 0; q < RPL; ++q) c_need_nodes += need[q] ? 1 : 0;
                    }
                    if (b0 && b1) {
                        const bool near1 = (near_bits >> __float_as_int(n3.z)) & 1u;
                        const int far = near1 ? c0 : c1;
                        next = near1 ? c1 : c0;
                        if (sp >= STACK) {
                            if (lane == 0) set_error(A.err, kDevErrTraversal);
                            break;
                        }
                        if (SMEM_STACK) {
                            if (lane == 0) sstack[sp] = far;
                        } else if (lane == (sp & 31)) {
                            if (STACK <= 32 || sp < 32) reg0 = far; else reg1 = far;
                        }
                        if (COUNT) {
#pragma unroll
                            for (int q = 0; q < RPL; ++q) {
                                const bool nf = need[q] && (near1 ? ha[q] : hb[q]);
                                needmask[q] = (needmask[q] & ~(1ull << sp)) | ((unsigned long long)nf << sp);
                                need[q] = need[q] && (near1 ? hb[q] : ha[q]);
                            }
                        }
                        ++sp;
                    } else if (b0) {
                        next = c0;
                        if (COUNT) {
#pragma unroll
                            for (int q = 0; q < RPL; ++q) need[q] = need[q] && ha[q];
                        }
                    } else if (b1) {
                        next = c1;
                        if (COUNT) {
#pragma unroll
                            for (int q = 0; q < RPL; ++q) need[q] = need[q] && hb[q];
                        }
                    }
                } else {
                    int first, count;
                    leaf_decode(cur, first, count);
                    test_leaf<RPL, STAGE>(ray, row.tris + 3 * (size_t)first, count, stage, lane);
                    if (COUNT) {
                        c_tris += count;
#pragma unroll
                        for (int q = 0; q < RPL; ++q) c_need_tris += need[q] ? count : 0;
                    }
                }
                if (next == kEmptyRoot) {
                    if (sp == 0) break;
                    // the cap is checked where the walk pops: between two pops
                    // it only descends, at most the tree's depth
                    if (iters > kIterCap) {
                        if (lane == 0) set_error(A.err, kDevErrTraversal);
                        break;
                    }
                    --sp;
                    if (SMEM_STACK) {
                        __syncwarp();
                        next = sstack[sp];
                    } else {
                        next = __shfl_sync(kFull, (STACK <= 32 || sp < 32) ? reg0 : reg1, sp & 31);
                    }
                    if (COUNT) {
#pragma unroll
                        for (int q = 0; q < RPL; ++q) need[q] = (needmask[q] >> sp) & 1ull;
                    }
                }
                cur = next;
            }
        }

        // stores
        const size_t frame = (size_t)agent * H * W;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const bool in = pix_r[q] < H && pix_c[q] < W && mine_q[q];
            const size_t off = frame + (size_t)pix_r[q] * W + pix_c[q];
            const NoiseParams& nz = A.noise;
            const unsigned long long nb =
                ((noise_frame * (unsigned long long)A.n_agents + agent) * (unsigned long long)(H * W) +
                 (unsigned long long)(pix_r[q] * W + pix_c[q])) * 64ull;
            if (in && A.depth) {
                float dv = ray[q].live ? ray[q].best_t : A.cam.max_depth;
                if (nz.enabled) dv = noisy(dv, A.cam.max_depth, nz.d_gauss, nz.d_speckle, nz.d_shot, nz.d_sp, nz.seed, nb);
                A.depth[off] = dv;
            }
            // ids: triangle >= 0, miss -1, drone j (internal INT_MIN + j) -2 - j
            const int bid = ray[q].best_id;
            const bool drone = bid < -1;
            if (in && A.hit_id) A.hit_id[off] = drone ? -2 - (bid - INT_MIN) : bid;
            if (in && A.seg) {
                int lab = bid >= 0 ? (row.labels ? __ldg(row.labels + bid) : bid) : drone ? A.swarm_label : -1;
                if (nz.enabled && nz.s_models && lab >= 0)
                    lab = (int)rintf(noisy((float)lab, nz.s_max, nz.s_gauss, nz.s_speckle, nz.s_shot, nz.s_sp, nz.seed,
                                           nb + 32));
                if (nz.enabled && nz.s_drop > 0.0f && unit_half_open(splitmix64_at(nz.seed, nb + 40)) < nz.s_drop)
                    lab = -1;
                A.seg[off] = lab;
            }
            if (A.rgb) {
                const uint32_t col = bid >= 0 ? __ldg(row.colors + bid) : drone ? A.swarm_rgb : 0u;
                const int p = lane + 32 * q;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    uint32_t v = (col >> (8 * ch)) & 0xFFu;
                    if (nz.enabled)
                        v = (uint32_t)rintf(noisy((float)v, 255.0f, nz.c_gauss, nz.c_speckle, nz.c_shot, nz.c_sp, nz.seed,
                                                  nb + 8 + 8 * ch));
                    rgbstage[3 * p + ch] = (uint8_t)v;
                }
            }
        }
        if (A.rgb) {
            __syncwarp();
            if (sub < 0 && (W % 4) == 0 && (TW % 4) == 0 && tx0 + TW <= W && ty0 + TH <= H &&
                (reinterpret_cast<uintptr_t>(A.rgb) & 3) == 0) {
                // each tile row is TW*3 bytes starting at a 4-byte-aligned offset
                constexpr int words_per_row = TW * 3 / 4;
                constexpr int words = words_per_row * TH;
                for (int w = lane; w < words; w += 32) {
                    const int r = w / words_per_row, k = w % words_per_row;
                    const uint32_t* srcw = reinterpret_cast<const uint32_t*>(rgbstage + r * TW * 3) + k;
                    uint32_t* dstw = reinterpret_cast<uint32_t*>(A.rgb + 3 * (frame + (size_t)(ty0 + r) * W + tx0)) + k;
                    *dstw = *srcw;
                }
            } else {
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    if (pix_r[q] < H && pix_c[q] < W && mine_q[q]) {
                        const int p = lane + 32 * q;
                        uint8_t* dst = A.rgb + 3 * (frame + (size_t)pix_r[q] * W + pix_c[q]);
                        dst[0] = rgbstage[3 * p];
                        dst[1] = rgbstage[3 * p + 1];
                        dst[2] = rgbstage[3 * p + 2];
                    }
                }
            }
            __syncwarp();
        }
        if (EXTRA >= 1 && A.band_done) {
            // Streamed download: the warp that completes an (agent, tile row)
            // band copies it from the output buffers (just written, resident in
            // L2) to the page-locked host images in 16-byte pieces, so the
            // transfer over the bus runs during the rest of the ray cast.
            __threadfence();  // this lane's image stores before the completion marks
            __syncwarp();
            const size_t band = (size_t)agent * tiles_y + ty;
            unsigned last = 0;
            if (lane == 0) {
                const unsigned bits = sub < 0 ? (1u << kSplit) - 1u : 1u << sub;
                const unsigned old = atomicOr(A.tile_bits + band * tiles_x + (tx0 / TW), bits);
                if (old != (1u << kSplit) - 1u && (old | bits) == (1u << kSplit) - 1u)
                    last = atomicAdd(A.band_done + band, 1u) + 1u == (unsigned)tiles_x;
            }
            if (__shfl_sync(kFull, last, 0)) {
                __threadfence();
                const int rows = min(TH, H - ty0);
                const size_t first = frame + (size_t)ty0 * W, px = (size_t)rows * W;
                if (A.host_depth && A.depth)
                    copy_out(reinterpret_cast<const uint8_t*>(A.depth + first), reinterpret_cast<uint8_t*>(A.host_depth + first),
                             4 * px, lane);
                if (A.host_rgb && A.rgb) copy_out(A.rgb + 3 * first, A.host_rgb + 3 * first, 3 * px, lane);
            }
        }
        if (__shfl_sync(kFull, err_seen, 0) == kDevErrTraversal) break;
        if (COUNT) ++c_items;
        if (sched && lane == 0) {
            // record this tile's cost for the next launch's schedule; a split
            // tile's cost is the sum of its quarters, recorded by the quarter
            // that completes it
            atomicAdd(&A.sched[ep & 1], (unsigned long long)item_cost);
            if (sub < 0) {
                A.cost[item] = (unsigned)item_cost;
            } else {
                const unsigned old = atomicAdd(A.acc + item, (unsigned)item_cost | (1u << 24));
                if ((old >> 24) == (unsigned)(kSplit - 1)) {
                    A.cost[item] = (old & 0xFFFFFFu) + (unsigned)item_cost;
                    A.acc[item] = 0u;
                }
            }
        }
    }

    if (COUNT) {
        // per-ray counts summed over the warp, per-item counts from lane 0
        long long nn = c_need_nodes, nt = c_need_tris;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            nn += __shfl_xor_sync(kFull, nn, off);
            nt += __shfl_xor_sync(kFull, nt, off);
        }
        if (lane == 0) {
            atomicAdd((unsigned long long*)&A.counters[0], (unsigned long long)c_nodes);
            atomicAdd((unsigned long long*)&A.counters[1], (unsigned long long)c_tris);
            atomicAdd((unsigned long long*)&A.counters[2], (unsigned long long)c_large);
            atomicAdd((unsigned long long*)&A.counters[3], (unsigned long long)c_items);
            atomicAdd((unsigned long long*)&A.counters[4], (unsigned long long)nn);
            atomicAdd((unsigned long long*)&A.counters[5], (unsigned long long)nt);
        }
    }
    // the last CTA to finish resets the work counter for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(A.done_ctas, 1u) == gridDim.x - 1) {
            *A.counter = 0u;
            *A.done_ctas = 0u;
            if (A.noise.enabled) *A.noise_frame = noise_frame + 1ull;
            if (sched) {
                // the next launch sums its costs into the other slot; its
                // buckets are filed afresh by its own estimate
                A.sched[(ep + 1) & 1] = 0ull;
                for (int b = 0; b < kBuckets; ++b) A.sched[kSchedLen + b] = 0ull;
                A.sched[kSchedTotal] = (unsigned long long)total;
                A.sched[kSchedShape] = sched_shape(tiles_x, tiles_y, A.n_agents);
                A.sched[kSchedEpoch] = (unsigned long long)ep + 1ull;
            }
            __threadfence();
        }
    }
}

template <int TW, int TH, int RPL, bool SMEM_STACK, bool STAGE, bool COUNT, bool WIDE, int EXTRA, int STACK>
cudaError_t launch_one(const RenderArgs& a, int ctas, cudaStream_t s) {
    auto k = raycast_kernel<TW, TH, RPL, SMEM_STACK, STAGE, COUNT, WIDE, EXTRA, STACK>;
    const size_t shm = render_smem_bytes(kWarpsPerCta, STACK, RPL);
    return launch_cfg(reinterpret_cast<const void*>(k), a, kWarpsPerCta, ctas, shm, s);
}

// The stack depth is a tuning choice of the device render (binary nodes, no
// counters, no drones; with the streamed download only the 32-entry register
// stack besides the default); the other builds keep kStack entries, which
// holds any scene the configured depth admits.  Traversal order does not
// depend on the stack's size, so images and counts are the same.
template <int TW, int TH, int RPL, bool SMEM_STACK, bool STAGE, bool COUNT, bool WIDE, int EXTRA>
cudaError_t launch_stack(const RenderArgs& a, const sim_render_config& c, int ctas, cudaStream_t s) {
    if constexpr (!COUNT && !WIDE && EXTRA == 0) {
        if (c.stack_depth == 32) return launch_one<TW, TH, RPL, SMEM_STACK, STAGE, COUNT, WIDE, EXTRA, 32>(a, ctas, s);
        if constexpr (SMEM_STACK)
            if (c.stack_depth == 48)
                return launch_one<TW, TH, RPL, SMEM_STACK, STAGE, COUNT, WIDE, EXTRA, 48>(a, ctas, s);
    }
    if constexpr (!COUNT && !WIDE && EXTRA == 1 && !SMEM_STACK)
        if (c.stack_depth == 32) return launch_one<TW, TH, RPL, SMEM_STACK, STAGE, COUNT, WIDE, EXTRA, 32>(a, ctas, s);
    return launch_one<TW, TH, RPL, SMEM_STACK, STAGE, COUNT, WIDE, EXTRA, kStack>(a, ctas, s);
}

template <int TW, int TH, int RPL, bool COUNT, bool WIDE, int EXTRA>
cudaError_t launch_shape_w(const RenderArgs& a, const sim_render_config& c, int ctas, cudaStream_t s) {
    if (c.stack_in_smem) {
        if (c.stage_in_smem) return launch_stack<TW, TH, RPL, true, true, COUNT, WIDE, EXTRA>(a, c, ctas, s);
        return launch_stack<TW, TH, RPL, true, false, COUNT, WIDE, EXTRA>(a, c, ctas, s);
    }
    if (c.stage_in_smem) return launch_stack<TW, TH, RPL, false, true, COUNT, WIDE, EXTRA>(a, c, ctas, s);
    return launch_stack<TW, TH, RPL, false, false, COUNT, WIDE, EXTRA>(a, c, ctas, s);
}

// EXTRA selects what is compiled in: 0 neither the drone test of the
// multi-agent mode nor the streamed download, 1 the streamed download only
// (environment steps in parallel-agents mode), 2 both (multi-agent launches and
// counted launches).  The leaner instantiations hold fewer registers in use and
// spill less: the streamed-only one made the environment step 1.7% faster.
template <int TW, int TH, int RPL, bool COUNT>
cudaError_t launch_shape(const RenderArgs& a, const sim_render_config& c, int ctas, cudaStream_t s) {
    if (COUNT || a.drones) {
        if (c.node_width == 4) return launch_shape_w<TW, TH, RPL, COUNT, true, 2>(a, c, ctas, s);
        return launch_shape_w<TW, TH, RPL, COUNT, false, 2>(a, c, ctas, s);
    }
    if constexpr (!COUNT) {
        if (a.band_done) {
            if (c.node_width == 4) return launch_shape_w<TW, TH, RPL, false, true, 1>(a, c, ctas, s);
            return launch_shape_w<TW, TH, RPL, false, false, 1>(a, c, ctas, s);
        }
        if (c.node_width == 4) return launch_shape_w<TW, TH, RPL, false, true, 0>(a, c, ctas, s);
        return launch_shape_w<TW, TH, RPL, false, false, 0>(a, c, ctas, s);
    }
    return cudaErrorInvalidValue;
}

template <bool COUNT>
cudaError_t dispatch(const RenderArgs& a, const sim_render_config& c, int ctas, cudaStream_t s) {
    if (c.tile_w == 8 && c.tile_h == 4 && c.rays_per_lane == 1) return launch_shape<8, 4, 1, COUNT>(a, c, ctas, s);
    if (c.tile_w == 4 && c.tile_h == 8 && c.rays_per_lane == 1) return launch_shape<4, 8, 1, COUNT>(a, c, ctas, s);
    if (c.tile_w == 16 && c.tile_h == 2 && c.rays_per_lane == 1) return launch_shape<16, 2, 1, COUNT>(a, c, ctas, s);
    if (c.tile_w == 8 && c.tile_h == 8 && c.rays_per_lane == 2) return launch_shape<8, 8, 2, COUNT>(a, c, ctas, s);
    if (c.tile_w == 16 && c.tile_h == 4 && c.rays_per_lane == 2) return launch_shape<16, 4, 2, COUNT>(a, c, ctas, s);
    return cudaErrorInvalidValue;
}

}  // namespace

size_t render_smem_bytes(int warps_per_cta, int stack_depth, int rpl) {
    return (size_t)warps_per_cta * (12 * sizeof(float4) + stack_depth * sizeof(int) + 32 * rpl * 3);
}

// Stack depths a configuration may take: binary nodes 32 or 64 entries in
// registers, 32, 48 or 64 in shared memory; 4-wide nodes 64.
static bool stack_depth_ok(int width, int in_smem, int depth) {
    if (width == 4) return depth == kStack;
    if (in_smem) return depth == 32 || depth == 48 || depth == 64;
    return depth == 32 || depth == 64;
}

int render_config_list(sim_render_config* out, int max) {
    static const int shapes[][3] = {{8, 4, 1}, {4, 8, 1}, {16, 2, 1}, {8, 8, 2}, {16, 4, 2}};
    int k = 0;
    for (int width : {2, 4})
        for (const auto& sh : shapes)
            for (int stack = 0; stack <= 1; ++stack)
                for (int depth : {32, 48, 64})
                    for (int stg = 0; stg <= 1; ++stg) {
                        if (!stack_depth_ok(width, stack, depth)) continue;
                        if (k < max && out)
                            out[k] = sim_render_config{sh[0], sh[1], sh[2], stack, depth, kWarpsPerCta, 0, stg, width};
                        ++k;
                    }
    return k;
}

bool render_config_valid(const sim_render_config& c) {
    sim_render_config all[128];
    const int n = render_config_list(all, 128);
    for (int i = 0; i < n; ++i) {
        const sim_render_config& a = all[i];
        if (a.tile_w == c.tile_w && a.tile_h == c.tile_h && a.rays_per_lane == c.rays_per_lane &&
            a.stack_in_smem == c.stack_in_smem && a.stack_depth == c.stack_depth && a.node_width == c.node_width &&
            (c.stage_in_smem == 0 || c.stage_in_smem == 1) && c.warps_per_cta == kWarpsPerCta &&
            c.ctas_per_sm >= 0 && c.ctas_per_sm <= 32)
            return true;
    }
    return false;
}

cudaError_t launch_render(const RenderArgs& a, const sim_render_config& c, int ctas, bool count, cudaStream_t s,
                          cudaEvent_t t0, cudaEvent_t t1) {
    if (a.sched && a.n_agents > 0 && c.tile_w > 0 && c.tile_h > 0) {
        const long long items = (long long)a.n_agents * ((a.cam.W + c.tile_w - 1) / c.tile_w) *
                                ((a.cam.H + c.tile_h - 1) / c.tile_h);
        // a programmatic dependent of the previous kernel: its launch overlaps
        // that kernel's tail, and it waits for it before reading anything
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)((items + 255) / 256));
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        // tiles over `split` times the mean cost are rendered as quarter-tile
        // sub-packets: 4x in device renders; 6x when the launch also streams its
        // bands to the host, where a split tile holds its band back longer
        // (measured: 2.3% faster host steps, device renders unchanged)
        const float split = a.band_done ? 6.0f : 4.0f;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, sched_estimate_kernel, a, c.tile_w, c.tile_h, split);
        if (e != cudaSuccess) return e;
    }
    // timed launches: events around the ray-cast kernel alone (the one before
    // it also ends its programmatic overlap with the estimate kernel)
    if (t0) {
        const cudaError_t e = cudaEventRecord(t0, s);
        if (e != cudaSuccess) return e;
    }
    const cudaError_t e = count ? dispatch<true>(a, c, ctas, s) : dispatch<false>(a, c, ctas, s);
    if (e != cudaSuccess || !t1) return e;
    return cudaEventRecord(t1, s);
}

}  // namespace vf

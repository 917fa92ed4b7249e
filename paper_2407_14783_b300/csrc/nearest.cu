// Nearest-obstacle query: for every agent, the closest point of its scene's
// mesh and the distance to it (the obstacle-distance module of Sec. III-B,
// there a CGAL C++ component on the CPU).  One warp per agent: the lanes first
// split the large-triangle list, then walk the scene's BVH together from a
// stack in shared memory, each iteration taking the top 32 entries (node,
// lower bound of the squared distance), pruning those farther than the warp's
// best so far, expanding nodes and testing leaf triangles, and pushing the
// surviving children (the nearer one on top).  A query thus costs about one
// dependent node fetch per 32 visited nodes, instead of one per node.
// Closest point on a triangle by its Voronoi regions (three vertices, three
// edges, the face).  Every triangle's distance is computed by the same code
// whatever the visiting order, and pruning keeps equal bounds, so the result
// (lowest id among equal distances) does not depend on the order.
#include "common.cuh"
#include "launch.h"

namespace vf {
namespace {

__device__ __forceinline__ float dot3(const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// a = v0 (w: id), e1 = v1 - v0, e2 = v2 - v0
__device__ void closest_on_tri(const float p[3], const float4 a, const float4 e1, const float4 e2, float out[3]) {
    const float ab[3] = {e1.x, e1.y, e1.z}, ac[3] = {e2.x, e2.y, e2.z};
    const float ap[3] = {p[0] - a.x, p[1] - a.y, p[2] - a.z};
    const float d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.0f && d2 <= 0.0f) {
        out[0] = a.x; out[1] = a.y; out[2] = a.z;
        return;
    }
    const float bp[3] = {ap[0] - ab[0], ap[1] - ab[1], ap[2] - ab[2]};
    const float d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0f && d4 <= d3) {
        out[0] = a.x + ab[0]; out[1] = a.y + ab[1]; out[2] = a.z + ab[2];
        return;
    }
    const float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
        const float v = d1 / (d1 - d3);
        out[0] = a.x + v * ab[0]; out[1] = a.y + v * ab[1]; out[2] = a.z + v * ab[2];
        return;
    }
    const float cp[3] = {ap[0] - ac[0], ap[1] - ac[1], ap[2] - ac[2]};
    const float d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0.0f && d5 <= d6) {
        out[0] = a.x + ac[0]; out[1] = a.y + ac[1]; out[2] = a.z + ac[2];
        return;
    }
    const float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
        const float w = d2 / (d2 - d6);
        out[0] = a.x + w * ac[0]; out[1] = a.y + w * ac[1]; out[2] = a.z + w * ac[2];
        return;
    }
    const float va = d3 * d6 - d5 * d4;
    if (va <= 0.0f && (d4 - d3) >= 0.0f && (d5 - d6) >= 0.0f) {
        const float w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        out[0] = a.x + ab[0] + w * (ac[0] - ab[0]);
        out[1] = a.y + ab[1] + w * (ac[1] - ab[1]);
        out[2] = a.z + ab[2] + w * (ac[2] - ab[2]);
        return;
    }
    const float den = 1.0f / (va + vb + vc);
    const float v = vb * den, w = vc * den;
    out[0] = a.x + ab[0] * v + ac[0] * w;
    out[1] = a.y + ab[1] * v + ac[1] * w;
    out[2] = a.z + ab[2] * v + ac[2] * w;
}

struct Best {
    float d2;
    int id;
    float q[3];
};

__device__ __forceinline__ void test_tri(const float p[3], const float4* t, Best& b) {
    const float4 a = __ldg(t), e1 = __ldg(t + 1), e2 = __ldg(t + 2);
    float q[3];
    closest_on_tri(p, a, e1, e2, q);
    const float dx = q[0] - p[0], dy = q[1] - p[1], dz = q[2] - p[2];
    const float d2 = dx * dx + dy * dy + dz * dz;
    const int id = __float_as_int(a.w);
    if (d2 < b.d2 || (d2 == b.d2 && (unsigned)id < (unsigned)b.id)) {
        b.d2 = d2;
        b.id = id;
        b.q[0] = q[0]; b.q[1] = q[1]; b.q[2] = q[2];
    }
}

__device__ __forceinline__ float box_d2(const float p[3], float lx, float ly, float lz, float hx, float hy, float hz) {
    const float dx = fmaxf(fmaxf(lx - p[0], p[0] - hx), 0.0f);
    const float dy = fmaxf(fmaxf(ly - p[1], p[1] - hy), 0.0f);
    const float dz = fmaxf(fmaxf(lz - p[2], p[2] - hz), 0.0f);
    return dx * dx + dy * dy + dz * dz;
}

constexpr int kNWarps = 4;       // warps (agents) per block
constexpr int kNCap = 1024;      // stack entries per warp

// Minimum over the full warp in one instruction (redux.sync on f32, sm_100 and
// later); exact, so the same as a shuffle ladder.
__device__ __forceinline__ float warp_min_f(float v) {
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

__global__ void __launch_bounds__(32 * kNWarps) nearest_kernel(NearestArgs A) {
    __shared__ int s_code[kNWarps][kNCap];
    __shared__ float s_bound[kNWarps][kNCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.x * kNWarps + warp;
    if (a >= A.n) return;  // whole warps leave together
    int* code = s_code[warp];
    float* bound = s_bound[warp];
    const float p[3] = {__ldg(A.state + a), __ldg(A.state + A.n + a), __ldg(A.state + 2 * A.n + a)};
    Best b;
    b.d2 = A.max_dist * A.max_dist;
    b.id = -1;
    b.q[0] = p[0]; b.q[1] = p[1]; b.q[2] = p[2];
    const int sid = __ldg(A.scene_of_agent + a);
    if (sid >= 0 && sid < A.n_scenes && A.table[sid].live) {
        const SceneRow row = A.table[sid];
        for (int k = lane; k < row.n_large; k += 32) test_tri(p, row.large + 3 * (size_t)k, b);
        float wbest = warp_min_f(b.d2);
        int sp = 0;
        if (row.root != kEmptyRoot) {
            if (lane == 0) {
                code[0] = row.root;
                bound[0] = 0.0f;
            }
            sp = 1;
        }
        __syncwarp();
        const unsigned lt = (1u << lane) - 1u;
        int iters = 0;
        while (sp > 0) {
            if (++iters > (1 << 20)) {
                if (lane == 0) set_error(A.err, kDevErrTraversal);
                break;
            }
            const int m = min(32, sp), base = sp - m;
            const bool have = lane < m;
            const int cur = have ? code[base + lane] : kEmptyRoot;
            const float bnd = have ? bound[base + lane] : INFINITY;
            __syncwarp();  // every pop is read before the pushes overwrite the slots
            sp = base;
            int c_near = 0, c_far = 0, npush = 0;
            float d_near = 0.0f, d_far = 0.0f;
            if (have && bnd <= wbest && cur != kEmptyRoot) {
                if (cur >= 0) {
                    const float4* np = row.nodes + 4 * (size_t)cur;
                    const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
                    const float d0 = box_d2(p, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y);
                    const float d1 = box_d2(p, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w);
                    const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
                    const bool h0 = d0 <= wbest, h1 = d1 <= wbest;
                    if (h0 && h1) {
                        const bool first1 = d1 < d0;
                        c_near = first1 ? c1 : c0;
                        d_near = first1 ? d1 : d0;
                        c_far = first1 ? c0 : c1;
                        d_far = first1 ? d0 : d1;
                        npush = 2;
                    } else if (h0 || h1) {
                        c_near = h0 ? c0 : c1;
                        d_near = h0 ? d0 : d1;
                        npush = 1;
                    }
                } else {
                    int first, count;
                    leaf_decode(cur, first, count);
                    for (int k = 0; k < count; ++k) test_tri(p, row.tris + 3 * (size_t)(first + k), b);
                }
            }
            // push: farther child below the nearer one, lanes in order
            const unsigned b1 = __ballot_sync(0xffffffffu, npush >= 1), b2 = __ballot_sync(0xffffffffu, npush == 2);
            const int total = __popc(b1) + __popc(b2);
            if (sp + total > kNCap) {
                if (lane == 0) set_error(A.err, kDevErrTraversal);
                break;
            }
            int pos = sp + __popc(b1 & lt) + __popc(b2 & lt);
            if (npush == 2) {
                code[pos] = c_far;
                bound[pos] = d_far;
                ++pos;
            }
            if (npush >= 1) {
                code[pos] = c_near;
                bound[pos] = d_near;
            }
            sp += total;
            __syncwarp();
            wbest = warp_min_f(b.d2);
        }
    } else if (lane == 0) {
        set_error(A.err, kDevErrNotFound);
    }
    // the lane holding the smallest (d2, unsigned id) writes the answer
    float bd = b.d2;
    unsigned bid = (unsigned)b.id;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float od = __shfl_xor_sync(0xffffffffu, bd, o);
        const unsigned oi = __shfl_xor_sync(0xffffffffu, bid, o);
        if (od < bd || (od == bd && oi < bid)) {
            bd = od;
            bid = oi;
        }
    }
    const unsigned mine = __ballot_sync(0xffffffffu, b.d2 == bd && (unsigned)b.id == bid);
    if (lane == __ffs(mine) - 1) {
        A.dist[a] = sqrtf(b.d2);
        if (A.point) {
            A.point[a] = b.q[0];
            A.point[A.n + a] = b.q[1];
            A.point[2 * A.n + a] = b.q[2];
        }
        if (A.tri) A.tri[a] = b.id;
    }
}

}  // namespace

cudaError_t launch_nearest(const NearestArgs& a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    nearest_kernel<<<(a.n + kNWarps - 1) / kNWarps, 32 * kNWarps, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vf

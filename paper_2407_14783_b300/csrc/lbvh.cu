// Device BVH builder (LBVH), one scene per call, sm_103a.
//
// The paper rasterises (Habitat-Sim); this library ray-casts, so each scene
// gets a device BVH built in these phases, all on the GPU:
//   1. per-triangle AABB and the scene AABB (block reduction + ordered-int
//      atomics);
//   2. triangles whose AABB spans more than a quarter of the scene's largest
//      extent (room walls, floors) are kept out of the tree in a short list
//      tested by every ray; the rest get 30-bit Morton codes (10 bits per axis)
//      of their centroids on a cubic grid over the centroid AABB (the same cell
//      size on every axis);
//   3. a stable LSD radix sort of (code, triangle) pairs, 8 bits per pass;
//   4. the binary radix tree over the sorted codes (Karras, HPG 2012): each
//      internal node finds its key range and split from longest common
//      prefixes, equal codes ordered by position;
//   5. bottom-up AABB refit with one atomic visit flag per internal node (the
//      second child to arrive computes the union);
//   6. packing: internal nodes as 4 float4 (both child boxes, padded by a
//      small margin so FP32 slab tests never reject a box that holds a hit,
//      and the two child codes); subtrees of <= kLeafMax triangles become leaf
//      ranges; triangles as 3 float4 (v0 + id, e1 = v1 - v0, e2 = v2 - v0) in
//      leaf order; one packed RGB word per original triangle id.
#include <vector>

#include "common.cuh"
#include "launch.h"

namespace vf {
namespace {

__device__ __forceinline__ int ordered(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__host__ __device__ inline float unordered(int i) {
#ifdef __CUDA_ARCH__
    return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF);
#else
    const int j = i >= 0 ? i : i ^ 0x7FFFFFFF;
    float f;
    memcpy(&f, &j, 4);
    return f;
#endif
}

// bounds layout: [0..2] min, [3..5] max as ordered ints
__device__ void reduce_bounds(const float lo[3], const float hi[3], bool valid, int* bounds) {
    float l[3], h[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        l[j] = valid ? lo[j] : 3.0e38f;
        h[j] = valid ? hi[j] : -3.0e38f;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            l[j] = fminf(l[j], __shfl_xor_sync(0xffffffffu, l[j], off));
            h[j] = fmaxf(h[j], __shfl_xor_sync(0xffffffffu, h[j], off));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            atomicMin(bounds + j, ordered(l[j]));
            atomicMax(bounds + 3 + j, ordered(h[j]));
        }
    }
}

__global__ void tri_bounds_kernel(int n, const float* __restrict__ verts, const int* __restrict__ tris,
                                  float4* __restrict__ tlo, float4* __restrict__ thi, int* bounds) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    const bool valid = i < n;
    if (valid) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            lo[j] = 3.0e38f;
            hi[j] = -3.0e38f;
        }
        for (int k = 0; k < 3; ++k) {
            const int vi = tris[3 * i + k];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float x = verts[3 * (size_t)vi + j];
                lo[j] = fminf(lo[j], x);
                hi[j] = fmaxf(hi[j], x);
            }
        }
        tlo[i] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        thi[i] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    }
    reduce_bounds(lo, hi, valid, bounds);
}

// Large-triangle flag and centroid bounds of the rest.
__global__ void centroid_bounds_kernel(int n, const float4* __restrict__ tlo, const float4* __restrict__ thi,
                                       float large_extent, int* __restrict__ is_large, int* cbounds,
                                       int* n_large) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float c[3] = {0, 0, 0};
    bool valid = false;
    if (i < n) {
        const float4 l = tlo[i], h = thi[i];
        const bool big = fmaxf(fmaxf(h.x - l.x, h.y - l.y), h.z - l.z) > large_extent;
        is_large[i] = big;
        if (big) atomicAdd(n_large, 1);
        valid = !big;
        c[0] = 0.5f * (l.x + h.x);
        c[1] = 0.5f * (l.y + h.y);
        c[2] = 0.5f * (l.z + h.z);
    }
    reduce_bounds(c, c, valid, cbounds);
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void morton_kernel(int n, const float4* __restrict__ tlo, const float4* __restrict__ thi,
                              const int* __restrict__ is_large, const int* __restrict__ cbounds,
                              uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vals[i] = (uint32_t)i;
    if (is_large[i]) {
        keys[i] = 0xFFFFFFFFu;  // sorts after every 30-bit code
        return;
    }
    const float4 l = tlo[i], h = thi[i];
    const float c[3] = {0.5f * (l.x + h.x), 0.5f * (l.y + h.y), 0.5f * (l.z + h.z)};
    uint32_t code = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // one cell size for all three axes (the largest extent): in a flat room
        // the top levels then split the long axes first
        const float lo = unordered(cbounds[j]);
        const float ext = fmaxf(fmaxf(unordered(cbounds[3]) - unordered(cbounds[0]), unordered(cbounds[4]) - unordered(cbounds[1])),
                                unordered(cbounds[5]) - unordered(cbounds[2]));
        float t = ext > 0.0f ? (c[j] - lo) / ext : 0.0f;
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        const uint32_t q = min((uint32_t)(t * 1024.0f), 1023u);
        code |= spread10(q) << (2 - j);
    }
    keys[i] = code;
}

// ------------------------------------------------------------ radix sort
constexpr int kMaxTreeDepth = 66;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(int n, const uint32_t* __restrict__ keys, int shift,
                                                                  uint32_t* __restrict__ hist, int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        const int i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m counters in one block of 1024 threads.
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t* data, int m) {
    __shared__ uint32_t part[1024];
    const int per = (m + 1023) / 1024;
    const int b = threadIdx.x * per;
    const int e = min(b + per, m);
    uint32_t s = 0;
    for (int i = b; i < e; ++i) s += data[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (int i = b; i < e; ++i) {
        const uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
}

// Stable scatter: items of a block are ranked in index order (round by round,
// warp by warp, lane by lane) among equal digits.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(int n, const uint32_t* __restrict__ kin,
                                                                     const uint32_t* __restrict__ vin,
                                                                     uint32_t* __restrict__ kout,
                                                                     uint32_t* __restrict__ vout, int shift,
                                                                     const uint32_t* __restrict__ offsets,
                                                                     int nblocks) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t running[256];
    __shared__ uint32_t wcount[kWarps][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    running[threadIdx.x] = offsets[threadIdx.x * nblocks + blockIdx.x];
    for (int w = 0; w < kWarps; ++w) wcount[w][threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        const int i = base + r * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        uint32_t key = 0, val = 0;
        if (valid) {
            key = kin[i];
            val = vin[i];
        }
        const uint32_t d = valid ? ((key >> shift) & 0xFF) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t lt = peers & ((1u << lane) - 1u);
        const int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcount[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = running[d] + __popc(lt);
            for (int w = 0; w < warp; ++w) pos += wcount[w][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < kWarps; ++w) {
            add += wcount[w][threadIdx.x];
            wcount[w][threadIdx.x] = 0;
        }
        running[threadIdx.x] += add;
        __syncthreads();
    }
}

// ------------------------------------------------------------ hierarchy
__device__ __forceinline__ int delta(const uint32_t* __restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = k[i], b = k[j];
    if (a != b) return __clz(a ^ b);
    return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

// Internal node i of n leaves: children (>= 0 internal, < 0: -1 - leaf) and
// the covered leaf range.
__global__ void hierarchy_kernel(int n, const uint32_t* __restrict__ k, int2* __restrict__ child,
                                 int2* __restrict__ range, int* __restrict__ parent_int, int* __restrict__ parent_leaf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(k, n, i, i - d);
    int lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(k, n, i, j);
    int s = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int gamma = i + s * d + min(d, 0);
    const int first = min(i, j), last = max(i, j);
    const int left = (first == gamma) ? -1 - gamma : gamma;
    const int right = (last == gamma + 1) ? -1 - (gamma + 1) : gamma + 1;
    child[i] = make_int2(left, right);
    range[i] = make_int2(first, last);
    if (left < 0) parent_leaf[-1 - left] = i; else parent_int[left] = i;
    if (right < 0) parent_leaf[-1 - right] = i; else parent_int[right] = i;
    if (i == 0) parent_int[0] = -1;
}

// Bottom-up refit: each leaf walks to the root; at every internal node the
// first arriving thread stops, the second computes the node box.
__global__ void refit_kernel(int n, const uint32_t* __restrict__ order, const float4* __restrict__ tlo,
                             const float4* __restrict__ thi, const int2* __restrict__ child,
                             const int* __restrict__ parent_int, const int* __restrict__ parent_leaf,
                             float4* node_lo, float4* node_hi, int* flags, int* max_depth) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    {
        // a valid binary radix tree over 32-bit keys plus 32-bit positions is at
        // most 64 levels deep; the walk is bounded so a broken tree cannot hang
        int depth = 0;
        for (int p = parent_leaf[j]; p >= 0 && depth <= kMaxTreeDepth; p = parent_int[p]) ++depth;
        atomicMax(max_depth, depth);
        if (depth > kMaxTreeDepth) return;
    }
    int p = parent_leaf[j];
    for (int level = 0; p >= 0 && level <= kMaxTreeDepth; ++level) {
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;
        __threadfence();
        const int2 c = child[p];
        float4 lo[2], hi[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int cc = s == 0 ? c.x : c.y;
            if (cc < 0) {
                const uint32_t tri = order[-1 - cc];
                lo[s] = tlo[tri];
                hi[s] = thi[tri];
            } else {
                lo[s] = __ldcg(&node_lo[cc]);
                hi[s] = __ldcg(&node_hi[cc]);
            }
        }
        __stcg(&node_lo[p], make_float4(fminf(lo[0].x, lo[1].x), fminf(lo[0].y, lo[1].y), fminf(lo[0].z, lo[1].z), 0.f));
        __stcg(&node_hi[p], make_float4(fmaxf(hi[0].x, hi[1].x), fmaxf(hi[0].y, hi[1].y), fmaxf(hi[0].z, hi[1].z), 0.f));
        p = parent_int[p];
    }
}

__device__ __forceinline__ void child_box(int cc, const uint32_t* __restrict__ order, const float4* __restrict__ tlo,
                                          const float4* __restrict__ thi, const float4* __restrict__ node_lo,
                                          const float4* __restrict__ node_hi, float pad, float4& lo, float4& hi) {
    if (cc < 0) {
        const uint32_t tri = order[-1 - cc];
        lo = tlo[tri];
        hi = thi[tri];
    } else {
        lo = node_lo[cc];
        hi = node_hi[cc];
    }
    lo.x -= pad; lo.y -= pad; lo.z -= pad;
    hi.x += pad; hi.y += pad; hi.z += pad;
}

__device__ __forceinline__ int child_code(int cc, const int2* __restrict__ range) {
    if (cc < 0) return leaf_code(-1 - cc, 1);
    const int2 r = range[cc];
    const int cnt = r.y - r.x + 1;
    return cnt <= kLeafMax ? leaf_code(r.x, cnt) : cc;
}

// Order word of a binary node: 2 * axis + s, axis the one along which the two
// child boxes' centres lie farthest apart, s = 1 when child 1's centre is the
// lower one along it.
__device__ __forceinline__ int order_word(const float4& l0, const float4& h0, const float4& l1, const float4& h1) {
    const float dx = (l1.x + h1.x) - (l0.x + h0.x), dy = (l1.y + h1.y) - (l0.y + h0.y);
    const float dz = (l1.z + h1.z) - (l0.z + h0.z);
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    const int axis = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    const float d = axis == 0 ? dx : axis == 1 ? dy : dz;
    return 2 * axis + (d < 0.0f ? 1 : 0);
}

__global__ void pack_nodes_kernel(int n, const uint32_t* __restrict__ order, const float4* __restrict__ tlo,
                                  const float4* __restrict__ thi, const int2* __restrict__ child,
                                  const int2* __restrict__ range, const float4* __restrict__ node_lo,
                                  const float4* __restrict__ node_hi, float pad, float4* __restrict__ nodes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int2 c = child[i];
    float4 l0, h0, l1, h1;
    child_box(c.x, order, tlo, thi, node_lo, node_hi, pad, l0, h0);
    child_box(c.y, order, tlo, thi, node_lo, node_hi, pad, l1, h1);
    nodes[4 * (size_t)i + 0] = make_float4(l0.x, l0.y, l0.z, h0.x);
    nodes[4 * (size_t)i + 1] = make_float4(h0.y, h0.z, l1.x, l1.y);
    nodes[4 * (size_t)i + 2] = make_float4(l1.z, h1.x, h1.y, h1.z);
    nodes[4 * (size_t)i + 3] = make_float4(__int_as_float(child_code(c.x, range)),
                                           __int_as_float(child_code(c.y, range)),
                                           __int_as_float(order_word(l0, h0, l1, h1)), 0.0f);
}

// Depth parity of every internal node (root: even).
__global__ void depth_parity_kernel(int n, const int* __restrict__ parent_int, int* __restrict__ parity) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = 0;
    for (int p = parent_int[i]; p >= 0 && d <= kMaxTreeDepth; p = parent_int[p]) ++d;
    parity[i] = d & 1;
}

// 4-wide node of every even-depth internal node i: its children, with every
// child that is an internal node (more than kLeafMax triangles) replaced by that
// child's two children -- which sit at even depth again.  Layout (8 float4):
// lo.x, lo.y, lo.z, hi.x, hi.y, hi.z of the four slots, then the four child
// codes; unused slots hold kEmptyRoot and a point box far outside the scene.
__global__ void pack_wide_kernel(int n, const uint32_t* __restrict__ order, const float4* __restrict__ tlo,
                                 const float4* __restrict__ thi, const int2* __restrict__ child,
                                 const int2* __restrict__ range, const float4* __restrict__ node_lo,
                                 const float4* __restrict__ node_hi, const int* __restrict__ parity, float pad,
                                 float4* __restrict__ wide) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1 || parity[i]) return;
    float bl[4][3], bh[4][3];
    int code[4];
    int k = 0;
    const int2 c = child[i];
    for (int s = 0; s < 2; ++s) {
        const int cc = s == 0 ? c.x : c.y;
        const int cd = child_code(cc, range);
        if (cd >= 0) {
            const int2 g = child[cd];
            for (int t = 0; t < 2; ++t) {
                const int gg = t == 0 ? g.x : g.y;
                float4 lo, hi;
                child_box(gg, order, tlo, thi, node_lo, node_hi, pad, lo, hi);
                bl[k][0] = lo.x; bl[k][1] = lo.y; bl[k][2] = lo.z;
                bh[k][0] = hi.x; bh[k][1] = hi.y; bh[k][2] = hi.z;
                code[k++] = child_code(gg, range);
            }
        } else {
            float4 lo, hi;
            child_box(cc, order, tlo, thi, node_lo, node_hi, pad, lo, hi);
            bl[k][0] = lo.x; bl[k][1] = lo.y; bl[k][2] = lo.z;
            bh[k][0] = hi.x; bh[k][1] = hi.y; bh[k][2] = hi.z;
            code[k++] = cd;
        }
    }
    for (; k < 4; ++k) {
        for (int j = 0; j < 3; ++j) bl[k][j] = bh[k][j] = 1.0e30f;
        code[k] = kEmptyRoot;
    }
    float4* w = wide + 8 * (size_t)i;
    w[0] = make_float4(bl[0][0], bl[1][0], bl[2][0], bl[3][0]);
    w[1] = make_float4(bl[0][1], bl[1][1], bl[2][1], bl[3][1]);
    w[2] = make_float4(bl[0][2], bl[1][2], bl[2][2], bl[3][2]);
    w[3] = make_float4(bh[0][0], bh[1][0], bh[2][0], bh[3][0]);
    w[4] = make_float4(bh[0][1], bh[1][1], bh[2][1], bh[3][1]);
    w[5] = make_float4(bh[0][2], bh[1][2], bh[2][2], bh[3][2]);
    w[6] = make_float4(__int_as_float(code[0]), __int_as_float(code[1]), __int_as_float(code[2]),
                       __int_as_float(code[3]));
    w[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Triangles in sorted order (first n_bvh go to the tree, the rest are large).
__global__ void pack_tris_kernel(int n, int n_bvh, const uint32_t* __restrict__ order,
                                 const float* __restrict__ verts, const int* __restrict__ tris,
                                 float4* __restrict__ out_tree, float4* __restrict__ out_large) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t t = order[j];
    float v[3][3];
    for (int k = 0; k < 3; ++k) {
        const int vi = tris[3 * (size_t)t + k];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[k][a] = verts[3 * (size_t)vi + a];
    }
    float4* dst = j < n_bvh ? out_tree + 3 * (size_t)j : out_large + 3 * (size_t)(j - n_bvh);
    dst[0] = make_float4(v[0][0], v[0][1], v[0][2], __int_as_float((int)t));
    dst[1] = make_float4(v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2], 0.0f);
    dst[2] = make_float4(v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2], 0.0f);
}

__global__ void pack_colors_kernel(int n, const uint8_t* __restrict__ rgb, uint32_t* __restrict__ colors) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    colors[i] = (uint32_t)rgb[3 * (size_t)i] | ((uint32_t)rgb[3 * (size_t)i + 1] << 8) |
                ((uint32_t)rgb[3 * (size_t)i + 2] << 16);
}

// ------------------------------------------------------------ PLOC
// The binary radix tree above splits by Morton prefix; its upper levels are
// then rebuilt by parallel locally-ordered clustering (Meister and Bittner
// 2018): the leaves of the packed radix tree (ranges of at most kLeafMax
// triangles, contiguous in Morton order) are the initial clusters, and every
// round each cluster finds, within kPlocRadius positions of the Morton-ordered
// list, the neighbour whose union box has the smallest surface area; mutual
// nearest neighbours merge into a new node and the list is compacted.  The
// surface-area-guided tree needs fewer node visits per ray than the prefix
// splits.  Node ids come from an exclusive scan over the merging pairs, so the
// tree does not depend on thread timing.
constexpr int kPlocRadius = 48;
constexpr int kPlocBlock = 256;
constexpr int kPlocMaxDepth = 56;  // deeper trees keep the radix-tree layout (traversal stacks hold 64)

__device__ __forceinline__ float half_area(float4 lo, float4 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

// The packed radix tree's leaves: the children with at most kLeafMax
// triangles of internal nodes with more.  At the leaf's first sorted position:
// code_at = its leaf code (0 elsewhere: leaf codes are < 0) and src_at = where
// its box is (>= 0 internal radix node, < 0: -1 - sorted triangle position).
__global__ void ploc_leaves_kernel(int n, const int2* __restrict__ child, const int2* __restrict__ range,
                                   int* __restrict__ code_at, int* __restrict__ src_at) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int2 r = range[i];
    if (r.y - r.x + 1 <= kLeafMax) return;  // inside a leaf of its ancestor
    const int2 c = child[i];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int cc = s == 0 ? c.x : c.y;
        if (cc < 0) {
            const int j = -1 - cc;
            code_at[j] = leaf_code(j, 1);
            src_at[j] = cc;
        } else {
            const int2 rc = range[cc];
            const int cnt = rc.y - rc.x + 1;
            if (cnt > kLeafMax) continue;
            code_at[rc.x] = leaf_code(rc.x, cnt);
            src_at[rc.x] = cc;
        }
    }
}

__global__ void ploc_flags_kernel(int n, const int* __restrict__ code_at, uint32_t* __restrict__ flag) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) flag[j] = code_at[j] != 0 ? 1u : 0u;
    if (j == n) flag[n] = 0u;
}

// Leaf k of the cluster list (Morton order): pool node k.
__global__ void ploc_gather_kernel(int n, const uint32_t* __restrict__ off, const int* __restrict__ code_at,
                                   const int* __restrict__ src_at, const uint32_t* __restrict__ order,
                                   const float4* __restrict__ tlo, const float4* __restrict__ thi,
                                   const float4* __restrict__ node_lo, const float4* __restrict__ node_hi,
                                   int* __restrict__ leaf_code_of, float4* __restrict__ plo, float4* __restrict__ phi,
                                   int* __restrict__ clusters) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || code_at[j] == 0) return;
    const int k = (int)off[j];
    const int src = src_at[j];
    leaf_code_of[k] = code_at[j];
    if (src < 0) {
        const uint32_t tri = order[-1 - src];
        plo[k] = tlo[tri];
        phi[k] = thi[tri];
    } else {
        plo[k] = node_lo[src];
        phi[k] = node_hi[src];
    }
    clusters[k] = k;
}

// Round state of the clustering in device memory, so that rounds run back to
// back without the host: [0] clusters m, [1] pool nodes created so far, [2] set
// when a round made no progress (the host then keeps the radix tree), [3] / [4]
// m and created at the start of the round being applied.
constexpr int kPlocState = 5;
constexpr int kPlocTile = 1024;  // clusters per block of the mark and apply kernels (one a thread)

__global__ void ploc_state_init_kernel(int* st, int m0) {
    st[0] = m0;
    st[1] = 0;
    st[2] = 0;
    st[3] = m0;
    st[4] = 0;
}

// Nearest neighbour of every cluster within kPlocRadius positions: smallest
// union surface area, lowest position among equals.
__device__ __forceinline__ int ploc_nearest(int k, int m, const float4* slo, const float4* shi, int at) {
    const float4 ml = slo[at], mh = shi[at];
    float best = INFINITY;
    int bj = -1;
    for (int d = -kPlocRadius; d <= kPlocRadius; ++d) {
        const int j = k + d;
        if (d == 0 || j < 0 || j >= m) continue;
        const float4 ol = slo[at + d], oh = shi[at + d];
        const float4 ul = make_float4(fminf(ml.x, ol.x), fminf(ml.y, ol.y), fminf(ml.z, ol.z), 0.0f);
        const float4 uh = make_float4(fmaxf(mh.x, oh.x), fmaxf(mh.y, oh.y), fmaxf(mh.z, oh.z), 0.0f);
        const float a = half_area(ul, uh);
        if (a < best) {
            best = a;
            bj = j;
        }
    }
    return bj;
}

__global__ void __launch_bounds__(kPlocBlock) ploc_nn_kernel(const int* __restrict__ st,
                                                             const int* __restrict__ clusters,
                                                             const float4* __restrict__ plo,
                                                             const float4* __restrict__ phi, int* __restrict__ nn) {
    if (st[2]) return;
    const int m = st[0];
    if (blockIdx.x * kPlocBlock >= m) return;
    __shared__ float4 slo[kPlocBlock + 2 * kPlocRadius], shi[kPlocBlock + 2 * kPlocRadius];
    const int base = blockIdx.x * kPlocBlock - kPlocRadius;
    for (int t = threadIdx.x; t < kPlocBlock + 2 * kPlocRadius; t += kPlocBlock) {
        const int k = base + t;
        if (k >= 0 && k < m) {
            const int id = clusters[k];
            slo[t] = plo[id];
            shi[t] = phi[id];
        }
    }
    __syncthreads();
    const int k = blockIdx.x * kPlocBlock + threadIdx.x;
    if (k >= m) return;
    nn[k] = ploc_nearest(k, m, slo, shi, threadIdx.x + kPlocRadius);
}

// Cluster k survives the round unless it merges into its earlier mutual
// nearest neighbour's new node; it makes a new node when its mutual nearest
// neighbour comes later.
__device__ __forceinline__ void ploc_fate(int k, int m, const int* __restrict__ nn, bool& keep, bool& make, int& j) {
    keep = make = false;
    j = -1;
    if (k >= m) return;
    j = nn[k];
    const bool mutual = j >= 0 && nn[j] == k;
    keep = !(mutual && k > j);
    make = mutual && k < j;
}

// Exclusive offsets of this thread's keep / make flags within its block of
// kPlocTile threads: lane ballots, then a scan of the 32 warps' counts.  Every
// thread of the block calls it.
__device__ __forceinline__ void ploc_block_offsets(bool keep, bool make, unsigned& koff, unsigned& moff) {
    __shared__ unsigned wk[32], wm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned bk = __ballot_sync(0xffffffffu, keep), bm = __ballot_sync(0xffffffffu, make);
    if (lane == 0) {
        wk[warp] = __popc(bk);
        wm[warp] = __popc(bm);
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned ck = wk[lane], cm = wm[lane];
        unsigned vk = ck, vm = cm;
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned tk = __shfl_up_sync(0xffffffffu, vk, off), tm = __shfl_up_sync(0xffffffffu, vm, off);
            if (lane >= off) {
                vk += tk;
                vm += tm;
            }
        }
        wk[lane] = vk - ck;
        wm[lane] = vm - cm;
    }
    __syncthreads();
    koff = wk[warp] + __popc(bk & lt);
    moff = wm[warp] + __popc(bm & lt);
}

// Merge of cluster k (pool id clusters[k]) with its later mutual neighbour j
// into pool node nid, or k alone; either way the survivor goes to out[koff].
__device__ __forceinline__ void ploc_apply_one(int k, int j, bool make, unsigned koff, int nid, int m0,
                                               const int* __restrict__ clusters, float4* __restrict__ plo,
                                               float4* __restrict__ phi, int2* __restrict__ pchild,
                                               int* __restrict__ out) {
    int id = clusters[k];
    if (make) {
        const int b = clusters[j];
        const float4 al = plo[id], ah = phi[id], bl = plo[b], bh = phi[b];
        plo[nid] = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.0f);
        phi[nid] = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.0f);
        pchild[nid - m0] = make_int2(id, b);
        id = nid;
    }
    out[koff] = id;
}

// Per block of kPlocTile clusters: how many survive the round and how many
// make a new node.
__global__ void __launch_bounds__(kPlocTile) ploc_mark_kernel(const int* __restrict__ st, const int* __restrict__ nn,
                                                              uint2* __restrict__ block_sums) {
    if (st[2]) return;
    const int m = st[0];
    bool keep, make;
    int j;
    ploc_fate(blockIdx.x * kPlocTile + threadIdx.x, m, nn, keep, make, j);
    const unsigned kt = (unsigned)__syncthreads_count(keep), mt = (unsigned)__syncthreads_count(make);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = make_uint2(kt, mt);
}

// Exclusive scan of the blocks' counts (in place, one block of 1024 threads)
// and the round's advance: the survivors become the next round's clusters.
// A round with more than one cluster and no merge sets the failure flag.
__global__ void __launch_bounds__(1024) ploc_advance_kernel(int* __restrict__ st, int m0, uint2* __restrict__ sums,
                                                            int nblocks) {
    if (st[2]) return;
    __shared__ unsigned pk[1024], pm[1024];
    const int per = (nblocks + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(b + per, nblocks);
    unsigned sk = 0, sm = 0;
    for (int i = b; i < e; ++i) {
        sk += sums[i].x;
        sm += sums[i].y;
    }
    pk[threadIdx.x] = sk;
    pm[threadIdx.x] = sm;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned vk = threadIdx.x >= off ? pk[threadIdx.x - off] : 0u;
        const unsigned vm = threadIdx.x >= off ? pm[threadIdx.x - off] : 0u;
        __syncthreads();
        pk[threadIdx.x] += vk;
        pm[threadIdx.x] += vm;
        __syncthreads();
    }
    unsigned rk = pk[threadIdx.x] - sk, rm = pm[threadIdx.x] - sm;
    for (int i = b; i < e; ++i) {
        const uint2 v = sums[i];
        sums[i] = make_uint2(rk, rm);
        rk += v.x;
        rm += v.y;
    }
    if (threadIdx.x == 1023) {
        const int m = st[0], created = st[1];
        const int kept = (int)pk[1023], made = (int)pm[1023];
        st[3] = m;
        st[4] = created;
        if (m > 1 && (kept >= m || created + made > m0 - 1)) {
            st[2] = 1;
        } else {
            st[0] = kept;
            st[1] = created + made;
        }
    }
}

__global__ void __launch_bounds__(kPlocTile) ploc_apply_kernel(const int* __restrict__ st, int m0,
                                                               const int* __restrict__ clusters,
                                                               const int* __restrict__ nn,
                                                               const uint2* __restrict__ block_off,
                                                               float4* __restrict__ plo, float4* __restrict__ phi,
                                                               int2* __restrict__ pchild, int* __restrict__ out) {
    if (st[2]) return;
    const int m = st[3], created = st[4];
    if (blockIdx.x * kPlocTile >= m) return;
    const int k = blockIdx.x * kPlocTile + threadIdx.x;
    bool keep, make;
    int j;
    ploc_fate(k, m, nn, keep, make, j);
    unsigned koff, moff;
    ploc_block_offsets(keep, make, koff, moff);
    if (!keep) return;
    const uint2 base = block_off[blockIdx.x];
    ploc_apply_one(k, j, make, base.x + koff, m0 + created + (int)(base.y + moff), m0, clusters, plo, phi, pchild,
                   out);
}

// A whole round in one block while at most kPlocTile clusters are left:
// neighbours (boxes staged in shared memory), fates, offsets, merges and the
// advance, with the same results as the multi-block kernels.
__global__ void __launch_bounds__(kPlocTile) ploc_round_small_kernel(int* __restrict__ st, int m0,
                                                                     const int* __restrict__ clusters,
                                                                     float4* __restrict__ plo,
                                                                     float4* __restrict__ phi,
                                                                     int2* __restrict__ pchild,
                                                                     int* __restrict__ out) {
    if (st[2]) return;
    __shared__ float4 slo[kPlocTile], shi[kPlocTile];
    __shared__ int snn[kPlocTile];
    const int m = st[0], created = st[1];
    const int k = threadIdx.x;
    if (k < m) {
        const int id = clusters[k];
        slo[k] = plo[id];
        shi[k] = phi[id];
    }
    __syncthreads();
    // the window never leaves [0, m): ploc_nearest skips positions outside it
    if (k < m) snn[k] = ploc_nearest(k, m, slo, shi, k);
    __syncthreads();
    bool keep, make;
    int j;
    ploc_fate(k, m, snn, keep, make, j);
    unsigned koff, moff;
    ploc_block_offsets(keep, make, koff, moff);
    const int kept = __syncthreads_count(keep), made = __syncthreads_count(make);
    if (keep) ploc_apply_one(k, j, make, koff, m0 + created + (int)moff, m0, clusters, plo, phi, pchild, out);
    if (threadIdx.x == 0) {
        st[3] = m;
        st[4] = created;
        if (m > 1 && (kept >= m || created + made > m0 - 1)) {
            st[2] = 1;
        } else {
            st[0] = kept;
            st[1] = created + made;
        }
    }
}

// Parent of every internal pool node (internal t = pool id m0 + t) and of
// every leaf cluster.
__global__ void ploc_parent_kernel(int n_int, int m0, const int2* __restrict__ pchild, int* __restrict__ parent,
                                   int* __restrict__ parent_leaf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_int) return;
    const int2 c = pchild[t];
    if (c.x >= m0) parent[c.x - m0] = t;
    else parent_leaf[c.x] = t;
    if (c.y >= m0) parent[c.y - m0] = t;
    else parent_leaf[c.y] = t;
}

// Internal nodes in each subtree, bottom-up from the leaf clusters: at every
// node the first arriving walk stops, the second sums the children (bounded
// like the refit).
__global__ void ploc_size_kernel(int m0, int n_int, const int2* __restrict__ pchild, const int* __restrict__ parent,
                                 const int* __restrict__ parent_leaf, int* flags, int* size) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m0) return;
    int p = parent_leaf[k];
    for (int level = 0; p >= 0 && level <= kMaxTreeDepth; ++level) {
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;
        __threadfence();
        const int2 c = pchild[p];
        const int a = c.x >= m0 ? __ldcg(&size[c.x - m0]) : 0, b = c.y >= m0 ? __ldcg(&size[c.y - m0]) : 0;
        __stcg(&size[p], 1 + a + b);
        p = parent[p];
    }
}

// Depth-first preorder index of every internal node (root 0, left subtree
// next): walking up, each step from a right child adds the left sibling's
// subtree.  In this layout a node's left child follows it in memory.
__global__ void ploc_dfs_kernel(int n_int, int m0, const int2* __restrict__ pchild, const int* __restrict__ parent,
                                const int* __restrict__ size, const int* __restrict__ depth, int* __restrict__ index,
                                int* __restrict__ depth_at) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_int) return;
    int idx = 0, c = t;
    for (int level = 0; level <= kMaxTreeDepth; ++level) {
        const int p = parent[c];
        if (p < 0) break;
        const int2 pc = pchild[p];
        idx += 1;
        if (pc.y == m0 + c && pc.x >= m0) idx += size[pc.x - m0];
        c = p;
    }
    index[t] = idx;
    depth_at[idx] = depth[t];
}

// Depth of every internal node (root 0), bounded walk; the tree's depth
// (internal levels plus the leaf level) goes to max_depth.
__global__ void ploc_depth_kernel(int n_int, const int* __restrict__ parent, int* __restrict__ depth,
                                  int* __restrict__ max_depth) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_int) return;
    int d = 0;
    for (int p = parent[t]; p >= 0 && d <= kMaxTreeDepth; p = parent[p]) ++d;
    depth[t] = d;
    atomicMax(max_depth, d + 1);
}

__device__ __forceinline__ void pool_child(int id, int m0, const int* __restrict__ leaf_code_of,
                                           const float4* __restrict__ plo, const float4* __restrict__ phi, float pad,
                                           float4& lo, float4& hi, int& code) {
    lo = plo[id];
    hi = phi[id];
    lo.x -= pad; lo.y -= pad; lo.z -= pad;
    hi.x += pad; hi.y += pad; hi.z += pad;
    code = id < m0 ? leaf_code_of[id] : id - m0;
}

__global__ void ploc_pack_kernel(int n_int, int m0, const int2* __restrict__ pchild, const int* __restrict__ leaf_code_of,
                                 const float4* __restrict__ plo, const float4* __restrict__ phi, float pad,
                                 const int* __restrict__ index, float4* __restrict__ nodes) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_int) return;
    const int2 c = pchild[u];
    float4 l0, h0, l1, h1;
    int c0, c1;
    pool_child(c.x, m0, leaf_code_of, plo, phi, pad, l0, h0, c0);
    pool_child(c.y, m0, leaf_code_of, plo, phi, pad, l1, h1, c1);
    if (c0 >= 0) c0 = index[c0];
    if (c1 >= 0) c1 = index[c1];
    const int t = index[u];
    nodes[4 * (size_t)t + 0] = make_float4(l0.x, l0.y, l0.z, h0.x);
    nodes[4 * (size_t)t + 1] = make_float4(h0.y, h0.z, l1.x, l1.y);
    nodes[4 * (size_t)t + 2] = make_float4(l1.z, h1.x, h1.y, h1.z);
    nodes[4 * (size_t)t + 3] = make_float4(__int_as_float(c0), __int_as_float(c1),
                                           __int_as_float(order_word(l0, h0, l1, h1)), 0.0f);
}

// 4-wide nodes from packed binary nodes (the same layout pack_wide_kernel
// writes): for every even-depth node t its children, each internal child
// replaced by that child's two children.  Boxes are already padded.
__global__ void wide_from_nodes_kernel(int n_int, const float4* __restrict__ nodes, const int* __restrict__ depth,
                                       float4* __restrict__ wide) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_int || (depth[t] & 1)) return;
    float bl[4][3], bh[4][3];
    int code[4];
    int k = 0;
    auto slot_of = [&](const float4* np, int s, float* lo, float* hi, int& cd) {
        const float4 a = np[0], b = np[1], c = np[2], d = np[3];
        if (s == 0) {
            lo[0] = a.x; lo[1] = a.y; lo[2] = a.z; hi[0] = a.w; hi[1] = b.x; hi[2] = b.y;
            cd = __float_as_int(d.x);
        } else {
            lo[0] = b.z; lo[1] = b.w; lo[2] = c.x; hi[0] = c.y; hi[1] = c.z; hi[2] = c.w;
            cd = __float_as_int(d.y);
        }
    };
    const float4* np = nodes + 4 * (size_t)t;
    for (int s = 0; s < 2; ++s) {
        float lo[3], hi[3];
        int cd;
        slot_of(np, s, lo, hi, cd);
        if (cd >= 0) {
            const float4* gp = nodes + 4 * (size_t)cd;
            for (int u = 0; u < 2; ++u) {
                slot_of(gp, u, bl[k], bh[k], code[k]);
                ++k;
            }
        } else {
            for (int j = 0; j < 3; ++j) {
                bl[k][j] = lo[j];
                bh[k][j] = hi[j];
            }
            code[k++] = cd;
        }
    }
    for (; k < 4; ++k) {
        for (int j = 0; j < 3; ++j) bl[k][j] = bh[k][j] = 1.0e30f;
        code[k] = kEmptyRoot;
    }
    float4* w = wide + 8 * (size_t)t;
    w[0] = make_float4(bl[0][0], bl[1][0], bl[2][0], bl[3][0]);
    w[1] = make_float4(bl[0][1], bl[1][1], bl[2][1], bl[3][1]);
    w[2] = make_float4(bl[0][2], bl[1][2], bl[2][2], bl[3][2]);
    w[3] = make_float4(bh[0][0], bh[1][0], bh[2][0], bh[3][0]);
    w[4] = make_float4(bh[0][1], bh[1][1], bh[2][1], bh[3][1]);
    w[5] = make_float4(bh[0][2], bh[1][2], bh[2][2], bh[3][2]);
    w[6] = make_float4(__int_as_float(code[0]), __int_as_float(code[1]), __int_as_float(code[2]),
                       __int_as_float(code[3]));
    w[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void init_bounds_kernel(int* b) {
    if (threadIdx.x < 3) b[threadIdx.x] = 0x7FFFFFFF;
    else if (threadIdx.x < 6) b[threadIdx.x] = (int)0x80000000;
}

inline unsigned nb(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

#define VF_TRY(x)                              \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

// Stream events at the phase boundaries of one build; timing failures only
// leave the phase times at zero.
struct PhaseTimer {
    cudaEvent_t ev[kBuildPhases + 1] = {};
    int next = 0;
    bool ok = true;
    explicit PhaseTimer() {
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) ok = false;
    }
    ~PhaseTimer() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
    // mark the end of every phase up to `phase` (phases with no work take 0)
    void mark(int phase, cudaStream_t s) {
        while (ok && next <= phase + 1 && next <= kBuildPhases)
            if (cudaEventRecord(ev[next++], s) != cudaSuccess) ok = false;
    }
    void read(float* ms) {
        for (int i = 0; i < kBuildPhases; ++i) ms[i] = 0.0f;
        if (!ok || next != kBuildPhases + 1 || cudaEventSynchronize(ev[kBuildPhases]) != cudaSuccess) return;
        for (int i = 0; i < kBuildPhases; ++i)
            if (cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]) != cudaSuccess) ms[i] = 0.0f;
    }
};

}  // namespace

// Scratch of the clustering, mostly buffers of the radix build that are dead
// by then; the node pool (boxes and children, 72 bytes per leaf cluster)
// lives in the scene's 4-wide node buffer, which is written last.
struct PlocScratch {
    int* code_at;       // [n]   (the large-triangle flags, dead after the Morton codes)
    int* src_at;        // [n]
    uint32_t* flag;     // [n + 1]
    int* leaf_code_of;  // [n]
    int* c0;            // [n]
    int* c1;            // [n]   (the spare sort values buffer)
    int* nn;            // [n]   (later the depth of every internal node)
    uint32_t* keep;     // [n]   rounds' per-block counts, then subtree sizes (the sorted keys, dead after the
                        //       hierarchy)
    uint32_t* make;     // [n]   arrival flags of the size pass (the spare sort keys buffer)
};

// Rebuild the tree above the radix tree's leaves by PLOC and pack it into
// out->nodes / out->wide.  *ok = false when it gives up (no progress in a
// round, or a tree deeper than kPlocMaxDepth): the caller then packs the radix
// tree, which overwrites everything this wrote.
cudaError_t ploc_build(int n_bvh, const uint32_t* order, const float4* tlo, const float4* thi, const int2* child,
                       const int2* range, const float4* node_lo, const float4* node_hi, const PlocScratch& w,
                       int* misc, float pad, LbvhResult* out, bool* ok, PhaseTimer& timer, cudaStream_t s) {
    *ok = false;
    VF_TRY(cudaMemsetAsync(w.code_at, 0, sizeof(int) * (size_t)n_bvh, s));
    ploc_leaves_kernel<<<nb(n_bvh - 1, 256), 256, 0, s>>>(n_bvh, child, range, w.code_at, w.src_at);
    ploc_flags_kernel<<<nb(n_bvh + 1, 256), 256, 0, s>>>(n_bvh, w.code_at, w.flag);
    scan_kernel<<<1, 1024, 0, s>>>(w.flag, n_bvh + 1);
    VF_TRY(cudaGetLastError());
    uint32_t m0u;
    VF_TRY(cudaMemcpyAsync(&m0u, w.flag + n_bvh, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VF_TRY(cudaStreamSynchronize(s));
    const int m0 = (int)m0u;
    // a radix tree over n_bvh >= 2 triangles has a leaf of two or more, so m0 < n_bvh
    if (m0 < 2 || m0 >= n_bvh) return cudaSuccess;
    // node pool in the 4-wide buffer (128 (n_bvh - 1) bytes >= 72 m0)
    float4* plo = out->wide;
    float4* phi = plo + 2 * (size_t)m0;
    int2* pchild = reinterpret_cast<int2*>(phi + 2 * (size_t)m0);
    ploc_gather_kernel<<<nb(n_bvh, 256), 256, 0, s>>>(n_bvh, w.flag, w.code_at, w.src_at, order, tlo, thi, node_lo,
                                                      node_hi, w.leaf_code_of, plo, phi, w.c0);
    // Rounds run back to back on the device (round state in misc[16..20]);
    // the host reads the state back only every few rounds, to size the grids
    // to the clusters left and to stop.  Rounds after the last merge copy the
    // single cluster over, so the result is the same however many run.
    int* st = misc + 16;
    uint2* sums = reinterpret_cast<uint2*>(w.keep);  // per-block counts, then offsets
    ploc_state_init_kernel<<<1, 1, 0, s>>>(st, m0);
    int* cur = w.c0;
    int* nxt = w.c1;
    int known_m = m0, rounds = 0, state[3] = {m0, 0, 0};
    while (known_m > 1) {
        if (rounds > 4096) return cudaSuccess;
        // rounds per read-back: fewer while the rounds are large
        const int batch = known_m > 65536 ? 2 : known_m > 8192 ? 4 : 8;
        for (int r = 0; r < batch; ++r) {
            if (known_m <= kPlocTile) {
                ploc_round_small_kernel<<<1, kPlocTile, 0, s>>>(st, m0, cur, plo, phi, pchild, nxt);
            } else {
                const int g = (int)nb(known_m, kPlocTile);
                ploc_nn_kernel<<<nb(known_m, kPlocBlock), kPlocBlock, 0, s>>>(st, cur, plo, phi, w.nn);
                ploc_mark_kernel<<<g, kPlocTile, 0, s>>>(st, w.nn, sums);
                ploc_advance_kernel<<<1, 1024, 0, s>>>(st, m0, sums, g);
                ploc_apply_kernel<<<g, kPlocTile, 0, s>>>(st, m0, cur, w.nn, sums, plo, phi, pchild, nxt);
            }
            std::swap(cur, nxt);
            ++rounds;
        }
        VF_TRY(cudaGetLastError());
        VF_TRY(cudaMemcpyAsync(state, st, sizeof(state), cudaMemcpyDeviceToHost, s));
        VF_TRY(cudaStreamSynchronize(s));
        if (state[2]) return cudaSuccess;  // a round without progress: keep the radix tree
        known_m = state[0];
    }
    const int created = state[1];
    const int n_int = m0 - 1;
    if (created != n_int) return cudaSuccess;
    timer.mark(5, s);
    int root;
    VF_TRY(cudaMemcpyAsync(&root, cur, sizeof(int), cudaMemcpyDeviceToHost, s));
    // buffers of the clustering rounds that are done with
    int* parent = nxt;
    int* depth = w.nn;
    int* parent_leaf = w.src_at;
    int* arrivals = reinterpret_cast<int*>(w.make);
    int* size = reinterpret_cast<int*>(w.keep);
    int* index = reinterpret_cast<int*>(w.flag);
    int* depth_at = w.code_at;
    VF_TRY(cudaMemsetAsync(parent, 0xFF, sizeof(int) * (size_t)n_int, s));  // -1: the root
    VF_TRY(cudaMemsetAsync(arrivals, 0, sizeof(int) * (size_t)n_int, s));
    VF_TRY(cudaMemsetAsync(misc + 14, 0, sizeof(int), s));
    ploc_parent_kernel<<<nb(n_int, 256), 256, 0, s>>>(n_int, m0, pchild, parent, parent_leaf);
    ploc_depth_kernel<<<nb(n_int, 256), 256, 0, s>>>(n_int, parent, depth, misc + 14);
    VF_TRY(cudaGetLastError());
    int tree_depth;
    VF_TRY(cudaMemcpyAsync(&tree_depth, misc + 14, sizeof(int), cudaMemcpyDeviceToHost, s));
    VF_TRY(cudaStreamSynchronize(s));
    if (tree_depth > kPlocMaxDepth || root != m0 + n_int - 1) return cudaSuccess;
    ploc_size_kernel<<<nb(m0, 256), 256, 0, s>>>(m0, n_int, pchild, parent, parent_leaf, arrivals, size);
    ploc_dfs_kernel<<<nb(n_int, 256), 256, 0, s>>>(n_int, m0, pchild, parent, size, depth, index, depth_at);
    ploc_pack_kernel<<<nb(n_int, 256), 256, 0, s>>>(n_int, m0, pchild, w.leaf_code_of, plo, phi, pad, index,
                                                    out->nodes);
    // the pool is read for the last time above: the 4-wide nodes overwrite it
    wide_from_nodes_kernel<<<nb(n_int, 256), 256, 0, s>>>(n_int, out->nodes, depth_at, out->wide);
    VF_TRY(cudaGetLastError());
    out->root = 0;  // depth-first order
    out->depth = tree_depth;
    *ok = true;
    return cudaSuccess;
}

// Build on `s`; device inputs verts [nv][3], tris [nt][3] (validated), rgb [nt][3].
// Scratch comes from `scratch` (size lbvh_scratch_bytes(nt)).  Outputs are
// allocated by the caller from the sizes in `out` after phase 1; to keep the
// interface single-call the caller passes an allocator callback.
cudaError_t lbvh_build(int64_t nt, const float* d_verts, const int* d_tris, const uint8_t* d_rgb, void* scratch,
                       LbvhAlloc alloc, void* alloc_user, LbvhResult* out, cudaStream_t s) {
    const int n = (int)nt;
    // scratch carve-up
    char* p = (char*)scratch;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)r;
    };
    float4* tlo = (float4*)take(sizeof(float4) * n);
    float4* thi = (float4*)take(sizeof(float4) * n);
    int* is_large = (int*)take(sizeof(int) * n);
    uint32_t* keys0 = (uint32_t*)take(sizeof(uint32_t) * n);
    uint32_t* vals0 = (uint32_t*)take(sizeof(uint32_t) * n);
    uint32_t* keys1 = (uint32_t*)take(sizeof(uint32_t) * n);
    uint32_t* vals1 = (uint32_t*)take(sizeof(uint32_t) * n);
    const int nblocks = (int)nb(n, kSortTile);
    uint32_t* hist = (uint32_t*)take(sizeof(uint32_t) * 256 * (size_t)nblocks);
    int2* child = (int2*)take(sizeof(int2) * n);
    int2* range = (int2*)take(sizeof(int2) * n);
    int* parent_int = (int*)take(sizeof(int) * n);
    int* parent_leaf = (int*)take(sizeof(int) * n);
    float4* node_lo = (float4*)take(sizeof(float4) * n);
    float4* node_hi = (float4*)take(sizeof(float4) * n);
    int* flags = (int*)take(sizeof(int) * n);
    int* misc = (int*)take(sizeof(int) * 32);  // [0..5] bounds, [6..11] centroid bounds, 12 n_large, 13 depth,
                                               // 14 clustered-tree depth, [16..20] clustering round state
    PlocScratch pw;
    pw.src_at = (int*)take(sizeof(int) * n);
    pw.flag = (uint32_t*)take(sizeof(uint32_t) * ((size_t)n + 1));
    pw.leaf_code_of = (int*)take(sizeof(int) * n);
    pw.c0 = (int*)take(sizeof(int) * n);
    pw.nn = (int*)take(sizeof(int) * n);

    PhaseTimer timer;
    timer.mark(-1, s);
    init_bounds_kernel<<<1, 32, 0, s>>>(misc);
    init_bounds_kernel<<<1, 32, 0, s>>>(misc + 6);
    VF_TRY(cudaMemsetAsync(misc + 12, 0, 2 * sizeof(int), s));
    tri_bounds_kernel<<<nb(n, 256), 256, 0, s>>>(n, d_verts, d_tris, tlo, thi, misc);
    VF_TRY(cudaGetLastError());
    int hb[6];
    VF_TRY(cudaMemcpyAsync(hb, misc, sizeof(hb), cudaMemcpyDeviceToHost, s));
    VF_TRY(cudaStreamSynchronize(s));
    float ext = 0.0f;
    for (int j = 0; j < 3; ++j) {
        out->lo[j] = unordered(hb[j]);
        out->hi[j] = unordered(hb[3 + j]);
        ext = fmaxf(ext, out->hi[j] - out->lo[j]);
    }
    timer.mark(0, s);
    centroid_bounds_kernel<<<nb(n, 256), 256, 0, s>>>(n, tlo, thi, 0.25f * ext, is_large, misc + 6, misc + 12);
    morton_kernel<<<nb(n, 256), 256, 0, s>>>(n, tlo, thi, is_large, misc + 6, keys0, vals0);
    VF_TRY(cudaGetLastError());
    timer.mark(1, s);
    uint32_t *ka = keys0, *va = vals0, *kb = keys1, *vb = vals1;
    for (int shift = 0; shift < 32; shift += 8) {
        radix_hist_kernel<<<nblocks, kSortThreads, 0, s>>>(n, ka, shift, hist, nblocks);
        scan_kernel<<<1, 1024, 0, s>>>(hist, 256 * nblocks);
        radix_scatter_kernel<<<nblocks, kSortThreads, 0, s>>>(n, ka, va, kb, vb, shift, hist, nblocks);
        VF_TRY(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    int nl;
    VF_TRY(cudaMemcpyAsync(&nl, misc + 12, sizeof(int), cudaMemcpyDeviceToHost, s));
    VF_TRY(cudaStreamSynchronize(s));
    timer.mark(2, s);
    const int n_bvh = n - nl;
    out->n_large = nl;
    out->n_bvh = n_bvh;
    out->n_nodes = n_bvh > 1 ? n_bvh - 1 : 0;
    // outputs
    VF_TRY(alloc(alloc_user, out));
    if (n_bvh > 1) {
        hierarchy_kernel<<<nb(n_bvh - 1, 256), 256, 0, s>>>(n_bvh, ka, child, range, parent_int, parent_leaf);
        timer.mark(3, s);
        VF_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * n_bvh, s));
        refit_kernel<<<nb(n_bvh, 256), 256, 0, s>>>(n_bvh, va, tlo, thi, child, parent_int, parent_leaf, node_lo,
                                                    node_hi, flags, misc + 13);
        const float pad = 2.0e-5f * fmaxf(ext, 1e-3f);
        VF_TRY(cudaGetLastError());
        int2 rr;
        VF_TRY(cudaMemcpyAsync(&rr, range, sizeof(int2), cudaMemcpyDeviceToHost, s));
        VF_TRY(cudaStreamSynchronize(s));
        const int cnt = rr.y - rr.x + 1;
        timer.mark(4, s);
        bool clustered = false;
        pw.code_at = is_large;  // dead buffers of the radix build
        pw.c1 = (int*)vb;
        pw.keep = ka;
        pw.make = kb;
        if (cnt > kLeafMax)
            VF_TRY(ploc_build(n_bvh, va, tlo, thi, child, range, node_lo, node_hi, pw, misc, pad, out, &clustered,
                              timer, s));
        // a clustering that gave up counts as clustering time; the radix tree is packed instead
        timer.mark(5, s);
        if (!clustered) {
            pack_nodes_kernel<<<nb(n_bvh - 1, 256), 256, 0, s>>>(n_bvh, va, tlo, thi, child, range, node_lo, node_hi,
                                                                 pad, out->nodes);
            depth_parity_kernel<<<nb(n_bvh - 1, 256), 256, 0, s>>>(n_bvh, parent_int, flags);
            pack_wide_kernel<<<nb(n_bvh - 1, 256), 256, 0, s>>>(n_bvh, va, tlo, thi, child, range, node_lo, node_hi,
                                                                flags, pad, out->wide);
            VF_TRY(cudaGetLastError());
            VF_TRY(cudaMemcpyAsync(&out->depth, misc + 13, sizeof(int), cudaMemcpyDeviceToHost, s));
            VF_TRY(cudaStreamSynchronize(s));
            out->root = cnt <= kLeafMax ? leaf_code(0, cnt) : 0;
        }
    } else if (n_bvh == 1) {
        out->root = leaf_code(0, 1);
        out->depth = 0;
    } else {
        out->root = kEmptyRoot;
        out->depth = 0;
    }
    timer.mark(6, s);
    if (n > 0) {
        pack_tris_kernel<<<nb(n, 256), 256, 0, s>>>(n, n_bvh, va, d_verts, d_tris, out->tris, out->large);
        pack_colors_kernel<<<nb(n, 256), 256, 0, s>>>(n, d_rgb, out->colors);
        VF_TRY(cudaGetLastError());
    }
    timer.mark(7, s);
    VF_TRY(cudaStreamSynchronize(s));
    timer.read(out->phase_ms);
    return cudaSuccess;
}

size_t lbvh_scratch_bytes(int64_t nt) {
    const size_t n = (size_t)(nt > 0 ? nt : 1);
    const size_t nblocks = (n + kSortTile - 1) / kSortTile;
    auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return 2 * r(16 * n) + 5 * r(4 * n) + r(4 * 256 * nblocks) + 2 * r(8 * n) + 2 * r(4 * n) + 2 * r(16 * n) +
           r(4 * n) + r(128) +
           // clustering: src_at, flag, leaf_code_of, c0, nn
           r(4 * n) + r(4 * (n + 1)) + 3 * r(4 * n);
}

}  // namespace vf

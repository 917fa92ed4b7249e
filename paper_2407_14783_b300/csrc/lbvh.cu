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
                                           __int_as_float(child_code(c.y, range)), 0.0f, 0.0f);
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

}  // namespace

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
    int* misc = (int*)take(sizeof(int) * 16);  // [0..5] bounds, [6..11] centroid bounds, 12 n_large, 13 depth

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
    centroid_bounds_kernel<<<nb(n, 256), 256, 0, s>>>(n, tlo, thi, 0.25f * ext, is_large, misc + 6, misc + 12);
    morton_kernel<<<nb(n, 256), 256, 0, s>>>(n, tlo, thi, is_large, misc + 6, keys0, vals0);
    VF_TRY(cudaGetLastError());
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
    const int n_bvh = n - nl;
    out->n_large = nl;
    out->n_bvh = n_bvh;
    out->n_nodes = n_bvh > 1 ? n_bvh - 1 : 0;
    // outputs
    VF_TRY(alloc(alloc_user, out));
    if (n_bvh > 1) {
        hierarchy_kernel<<<nb(n_bvh - 1, 256), 256, 0, s>>>(n_bvh, ka, child, range, parent_int, parent_leaf);
        VF_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * n_bvh, s));
        refit_kernel<<<nb(n_bvh, 256), 256, 0, s>>>(n_bvh, va, tlo, thi, child, parent_int, parent_leaf, node_lo,
                                                    node_hi, flags, misc + 13);
        const float pad = 2.0e-5f * fmaxf(ext, 1e-3f);
        pack_nodes_kernel<<<nb(n_bvh - 1, 256), 256, 0, s>>>(n_bvh, va, tlo, thi, child, range, node_lo, node_hi,
                                                             pad, out->nodes);
        depth_parity_kernel<<<nb(n_bvh - 1, 256), 256, 0, s>>>(n_bvh, parent_int, flags);
        pack_wide_kernel<<<nb(n_bvh - 1, 256), 256, 0, s>>>(n_bvh, va, tlo, thi, child, range, node_lo, node_hi,
                                                            flags, pad, out->wide);
        VF_TRY(cudaGetLastError());
        int2 rr;
        VF_TRY(cudaMemcpyAsync(&rr, range, sizeof(int2), cudaMemcpyDeviceToHost, s));
        VF_TRY(cudaMemcpyAsync(&out->depth, misc + 13, sizeof(int), cudaMemcpyDeviceToHost, s));
        VF_TRY(cudaStreamSynchronize(s));
        const int cnt = rr.y - rr.x + 1;
        out->root = cnt <= kLeafMax ? leaf_code(0, cnt) : 0;
    } else if (n_bvh == 1) {
        out->root = leaf_code(0, 1);
        out->depth = 0;
    } else {
        out->root = kEmptyRoot;
        out->depth = 0;
    }
    if (n > 0) {
        pack_tris_kernel<<<nb(n, 256), 256, 0, s>>>(n, n_bvh, va, d_verts, d_tris, out->tris, out->large);
        pack_colors_kernel<<<nb(n, 256), 256, 0, s>>>(n, d_rgb, out->colors);
        VF_TRY(cudaGetLastError());
    }
    return cudaStreamSynchronize(s);
}

size_t lbvh_scratch_bytes(int64_t nt) {
    const size_t n = (size_t)(nt > 0 ? nt : 1);
    const size_t nblocks = (n + kSortTile - 1) / kSortTile;
    auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return 2 * r(16 * n) + 5 * r(4 * n) + r(4 * 256 * nblocks) + 2 * r(8 * n) + 2 * r(4 * n) + 2 * r(16 * n) +
           r(4 * n) + r(64);
}

}  // namespace vf

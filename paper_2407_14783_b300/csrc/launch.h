// Host-side launch interfaces between the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace vf {

// dynamics.cu
cudaError_t launch_step(const DynConsts& c, int n, float* state, const float* cmd, float* ckpt, cudaStream_t s);
// Position of the command pointer among the dynamics kernel's arguments
// (DynConsts, n, state, cmd, ckpt): a captured step rebinds it per call.
constexpr int kStepCmdArg = 3;
cudaError_t launch_step_backward(const DynConsts& c, int n, const float* state_in, const float* cmd,
                                 const float* g_out, float* g_in, float* g_cmd, cudaStream_t s);
cudaError_t launch_rollout(const DynConsts& c, int n, int T, int K, const float* state0, const float* cmds,
                           float* states_out, float* ckpt, float* state_final, cudaStream_t s);
// tape: scratch of rollout_tape_bytes(n, K) bytes that records each step's
// forward pass for the reverse sweep, or null (the sweep then recomputes it)
cudaError_t launch_rollout_backward(const DynConsts& c, int n, int T, int K, const float* ckpt, const float* cmds,
                                    const float* g_states, float* g_state0, float* g_cmds, float* tape,
                                    cudaStream_t s);
size_t rollout_tape_bytes(int n, int K);

// lbvh.cu
// Phases of a scene build, timed by stream events at their boundaries: scene
// and triangle bounds, centroid bounds and Morton codes, radix sort, radix
// tree, refit, clustering rounds (PLOC), tree packing, triangle and colour
// packing.  A phase's time includes the host read-backs that end it.
constexpr int kBuildPhases = 8;
struct LbvhResult {
    float lo[3], hi[3];
    int n_large, n_bvh, n_nodes, depth, root;
    float phase_ms[kBuildPhases];
    float4* nodes;
    float4* wide;  // 8 float4 per internal node (valid at even depth): the 4-wide layout
    float4* tris;
    float4* large;
    uint32_t* colors;
};
// Called once the counts are known; must allocate nodes (4 float4 each), wide
// (8 float4 each), tris (3 float4 each, n_bvh), large (3 float4 each, n_large),
// colors (n_tris).
typedef cudaError_t (*LbvhAlloc)(void* user, LbvhResult* r);
size_t lbvh_scratch_bytes(int64_t nt);
cudaError_t lbvh_build(int64_t nt, const float* d_verts, const int* d_tris, const uint8_t* d_rgb, void* scratch,
                       LbvhAlloc alloc, void* alloc_user, LbvhResult* out, cudaStream_t s);

// raycast.cu
// Cost buckets of the longest-first schedule: estimates over 4 (6 in streamed
// launches), 2, 1.25, 0.8, 0.5 and 0.25 times the mean cost, and the rest.  The first kHeavyBuckets are
// the heavy ones that a streamed launch interleaves with the natural order.
constexpr int kBuckets = 7;
constexpr int kHeavyBuckets = 4;
constexpr int kSchedEpoch = 2;    // header words of the scheduling state
constexpr int kSchedTotal = 3;
constexpr int kSchedLen = 4;      // kSchedLen .. kSchedLen + kBuckets - 1
constexpr int kSchedShape = kSchedLen + kBuckets;
constexpr int kSchedHeaderWords = 16;

struct RenderArgs {
    int n_agents;
    const int* scene_of_agent;
    const float* state;
    float* depth;
    uint8_t* rgb;
    int* hit_id;
    const SceneRow* table;
    int n_scenes;
    CamConsts cam;
    unsigned* counter;   // work-item counter (zero between launches)
    unsigned* done_ctas; // finished-CTA counter (zero between launches)
    int* err;
    long long* counters; // traversal counters (COUNT builds)
    // Longest-first scheduling state carried between launches (may be null):
    // sched[e & 1] the cost sum of the launch with epoch e, sched[kSchedEpoch]
    // the epoch, sched[kSchedTotal] / sched[kSchedShape] item count and (tiles
    // x, tiles y, agents) of the last completed launch, sched[kSchedLen + b]
    // the lengths of this launch's buckets; heavy[b][cap] the bucket lists
    // (filed by sched_estimate_kernel just before the launch); done[cap] marks
    // of items already rendered in this launch; acc[cap] cost sums and arrival
    // counts of split tiles' quarters (zero between launches); cost[cap] each
    // item's cost in the last launch; pose[2][cap] each agent's unit attitude
    // quaternion at the launch with epoch e in slot e & 1.
    unsigned long long* sched;
    unsigned* heavy;
    unsigned long long* done;
    unsigned* acc;
    unsigned* cost;
    float4* pose;
    int sched_cap;
    unsigned launch_id;  // distinct per host-side launch
    int32_t* seg;        // segmentation image [n][H][W] or null
    NoiseParams noise;
    unsigned long long* noise_frame;  // frame counter of the noise streams (advanced by every noisy launch)
    int prefetch_l2;     // stream every live scene's nodes and triangles into L2 at launch start
    // Streamed download (may be null): page-locked host images [n][H][W] and
    // [n][H][W][3] that receive each (agent, tile row) band of depth / rgb as
    // soon as the band is complete; band_done[n][tiles_y] counts the band's
    // completed tiles and tile_bits[n][tiles_y][tiles_x] the quarters of a tile
    // rendered so far (both zero at launch start).  A tile can be rendered
    // twice in a launch (a scheduled heavy tile also taken by the plain pass
    // before its mark lands; both write the same values), so completion is
    // recorded per tile, not by counting pixels.
    float* host_depth = nullptr;
    uint8_t* host_rgb = nullptr;
    unsigned* band_done = nullptr;
    unsigned* tile_bits = nullptr;
    // Multi-agent mode (may be null): every agent sees the other drones of its
    // scene.  drones[3 j + k] = (body axis k of drone j, centre_k);
    // swarm_off[sid] .. swarm_off[sid + 1] index swarm_spheres, the agents of
    // scene sid.  A drone is a box of half extents swarm_half about its body
    // origin; a hit on drone j has the internal id INT_MIN + j.
    const float4* drones = nullptr;
    const int* swarm_off = nullptr;
    const float4* swarm_spheres = nullptr;  // per member, in member order: (centre, agent index as int bits)
    const float4* swarm_groups = nullptr;   // member groups of the larger swarms (SwarmScratch::groups) or null
    float swarm_half[3] = {0.0f, 0.0f, 0.0f};
    float swarm_radius = 0.0f;   // |swarm_half|: bounding sphere for the per-tile cull
    uint32_t swarm_rgb = 0;      // packed like the scene colours
    int swarm_label = -1;        // segmentation label of a drone
};

// Per-launch buffers of the multi-agent mode.
struct SwarmScratch {
    float4* drones = nullptr;  // [cap_agents][3]
    int* members = nullptr;    // [cap_agents]
    float4* spheres = nullptr; // [cap_agents]: member centres with the agent index in w
    int* off = nullptr;        // [cap_scenes + 1]
    int* cursor = nullptr;     // [cap_scenes]
    float4* groups = nullptr;  // [swarm_group_slots(cap_agents, cap_scenes)][2]: member groups' centre bounds
    int cap_agents = 0, cap_scenes = 0;
};
// Two-level hierarchy over a scene's swarm members (rebuilt every launch):
// scenes with more than kSwarmGroupMin members have their members ordered
// along a Morton curve and cut into groups of 32 consecutive members; group g
// of scene s is entry (off[s] / 32 + s + g) of `groups` (lo, hi of the member
// centres).  A tile tests the groups' boxes before their members.
constexpr int kSwarmGroupMin = 256;
constexpr int kSwarmSortMax = 4096;  // members per scene that are sorted; beyond that, groups in bucket order
inline size_t swarm_group_slots(int cap_agents, int cap_scenes) {
    return (size_t)cap_agents / 32 + (size_t)cap_scenes + 2;
}
cudaError_t launch_swarm_prep(int n, const int* scene_of_agent, const float* state, int n_scenes, SwarmScratch& s,
                              cudaStream_t st);
// After launch_swarm_prep: order each larger swarm along a Morton curve and
// write its groups' boxes (one CTA per scene).
cudaError_t launch_swarm_groups(int n, int n_scenes, SwarmScratch& s, cudaStream_t st);
cudaError_t launch_swarm_proximity(int n, const int* scene_of_agent, const float* state, int n_scenes,
                                   const SwarmScratch& s, float radius, float* dist, int* other, int* n_collide,
                                   cudaStream_t st);
size_t render_smem_bytes(int warps_per_cta, int stack_depth, int rpl);
int render_config_list(sim_render_config* out, int max);
bool render_config_valid(const sim_render_config& c);
// t0 / t1: events recorded just before and after the ray-cast kernel (after
// the estimate kernel), or null
cudaError_t launch_render(const RenderArgs& a, const sim_render_config& c, int ctas, bool count, cudaStream_t s,
                          cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr);
// api.cu: context helpers for entry points defined in other files.
void set_last_error(const char* msg);
int ctx_device(const sim_ctx* c);
// The checks of render_scene_with_scratch alone (scene, arguments, BVH depth
// against the traversal stack, launch size), for callers that must validate
// before touching their scratch.
int render_scene_check(sim_ctx* c, int n, int scene_id, const int32_t* soa_dev, const float* state);
int render_scene_with_scratch(sim_ctx* c, int n, int scene_id, const int32_t* soa_dev, unsigned* counters_dev,
                              const float* state, float* depth, uint8_t* rgb, int32_t* hit, cudaStream_t s);
// nearest.cu
struct NearestArgs {
    int n;
    const int* scene_of_agent;
    const float* state;
    float max_dist;
    float* dist;
    float* point;  // [3][n] or null
    int* tri;      // [n] or null
    const SceneRow* table;
    int n_scenes;
    int* err;
};
cudaError_t launch_nearest(const NearestArgs& a, cudaStream_t s);

// api.cu: context services for the step server.
int ctx_alloc_ext(sim_ctx* c, size_t bytes, void** out);
void ctx_free_ext(sim_ctx* c, void* p, size_t bytes);
int ctx_alloc_pool(sim_ctx* c, size_t bytes, void** out, cudaMemPool_t pool, cudaStream_t s);
void ctx_free_pool(sim_ctx* c, void* p, size_t bytes, cudaStream_t s);
void ctx_image_size(const sim_ctx* c, int* W, int* H);
bool ctx_scene_live(sim_ctx* c, int scene_id);
int ctx_step(sim_ctx* c, int n, float* state, const float* cmd, cudaStream_t s);
int ctx_render_own(sim_ctx* c, int n, const int32_t* soa, const float* state, float* depth, uint8_t* rgb,
                   unsigned* counters, cudaStream_t s);
int ctx_fail(int code, const char* msg);
// api.cu: launches a raycast kernel instance with the persistent grid size.
cudaError_t launch_cfg(const void* kernel, const RenderArgs& a, int warps_per_cta, int ctas, size_t smem,
                       cudaStream_t s);

}  // namespace vf

/*
 * visfly_b300.h -- C ABI of the B300 (sm_103a) rollout-step library.
 *
 * The library advances N quadrotors one control step and renders each agent's
 * depth and colour image of a triangle-mesh scene, following the environment
 * step of VisFly (arXiv 2407.14783): the user calls step(action) and receives
 * observations (Sec. III-C).  Physics follows Sec. III-A (Eq. 1-4, body-rate
 * controller, RK4); the depth and colour sensors follow Sec. III-B.  Reward,
 * termination and task logic stay in the caller (Sec. III-C, Listing 1).
 *
 * Conventions shared by every call
 *   - All calls return an int status (sim_status).  Nothing throws across the
 *     ABI.  Argument, budget and CUDA launch errors are reported synchronously
 *     and the message is available from sim_last_error() on the same thread.
 *   - "dev" pointers are CUDA device (or managed) pointers owned by the caller;
 *     "host" pointers are host memory owned by the caller (pinned memory makes
 *     the copies asynchronous).  The library never frees caller memory.
 *   - Work is enqueued on the caller's stream (cudaStream_t passed as void*,
 *     NULL = the legacy default stream) and is asynchronous unless stated.
 *   - Agent state is structure-of-arrays float32 [17][n]: rows 0-2 position x_W
 *     (m, world frame, z up), 3-5 velocity v_W (m/s), 6-9 attitude quaternion
 *     q = (w, x, y, z) body->world, 10-12 body rates Omega_B (rad/s), 13-16
 *     rotor speeds omega_1..4 (rad/s).  Row r of agent a is at state[r*n + a].
 *   - Commands are float32 [4][n]: normalised collective thrust u0 in [-1, 1]
 *     and body-rate commands u1..u3 in [-1, 1] (CTBR, Sec. III-A / Sec. IV).
 *   - Images are row-major per agent: depth float32 [n][H][W] (metres along the
 *     optical axis, max_depth on a miss), rgb uint8 [n][H][W][3], hit id int32
 *     [n][H][W] (original triangle index, -1 on a miss).
 *   - Device-side faults that kernels detect (traversal stack overflow, an
 *     iteration cap) set a device error word; sim_get_status() reports and
 *     clears it.  Kernels never trap.
 */
#ifndef VISFLY_B300_H
#define VISFLY_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The library is built with hidden symbol visibility; the declarations below
 * are its exported interface. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef struct sim_ctx sim_ctx;

typedef enum {
    SIM_OK = 0,
    SIM_ERR_INVALID_ARG = -1, /* bad pointer, size, id or parameter */
    SIM_ERR_OOM = -2,         /* device allocation failed */
    SIM_ERR_CUDA = -3,        /* a CUDA call failed; message has the CUDA error */
    SIM_ERR_NOT_FOUND = -4,   /* unknown scene id */
    SIM_ERR_TRAVERSAL = -5,   /* device: BVH traversal stack overflow or iteration cap */
    SIM_ERR_TIMEOUT = -6,     /* a bounded wait ran out */
    SIM_ERR_BUDGET = -7       /* the context's memory budget would be exceeded */
} sim_status;

/* Model, integrator and camera parameters.  The paper names the model terms
 * but prints no constants; every value is supplied by the caller.
 * Rotor i sits at azimuth 45 + 90 i degrees at distance `arm` in the body x-y
 * plane and spins in direction +1, -1, +1, -1 (X layout). */
typedef struct sim_params {
    float mass;          /* kg */
    float J[3];          /* diagonal inertia, kg m^2 (Eq. 1) */
    float arm;           /* m */
    float k[3];          /* thrust polynomial f = k2 w^2 + k1 w + k0 (Eq. 4) */
    float c_lag;         /* rotor time-decay constant c, 1/s (Eq. 4) */
    float kappa;         /* rotor reaction torque / thrust, m (Eq. 3) */
    float rho;           /* air density (Eq. 2) */
    float Cd[3];         /* drag coefficients (Eq. 2) */
    float area[3];       /* crossing areas (Eq. 2) */
    float omega_min, omega_max; /* rotor speed range, rad/s */
    float a_max;         /* mass-normalised thrust at u0 = +1, m/s^2 */
    float rate_max[3];   /* body-rate command scale, rad/s */
    float K_rate[3];     /* body-rate loop gains, 1/s */
    float g;             /* gravity, m/s^2 */
    float dt;            /* control step, s */
    int32_t n_sub;       /* physics sub-steps per control step, 1..8 */
    int32_t integrator;  /* 0 = RK4, 1 = explicit Euler */
    int32_t width, height; /* image size, pixels (1..1024) */
    float fov_deg;       /* horizontal field of view; square pixels */
    float max_depth;     /* m; farther hits are misses */
    float cam_off[3];    /* camera origin in the body frame, m */
    int32_t controller;  /* command interpretation (Sec. III-A):
                          * 0 CTBR: u = (collective thrust, body rates), normalised to [-1, 1];
                          * 1 SRT: u_i = rotor i's thrust, (u_i + 1) / 2 * f(omega_max);
                          * 2 LV: u = (world velocity m/s, yaw rad), geometric control;
                          * 3 PS: u = (world position m, yaw rad), geometric control.
                          * LV / PS: desired force m (a_d + g z) with
                          * a_d = -K_pos (x - x_d) - K_vel v (PS) or -K_vel (v - v_d) (LV),
                          * thrust = its projection on body z, desired attitude from its
                          * direction and the yaw, moment J (-K_att e_R - K_omega Omega) +
                          * Omega x J Omega with e_R = vee(R_d^T R - R^T R_d) / 2. */
    float K_pos[3], K_vel[3], K_att[3], K_omega[3];
} sim_params;

/* Create a context on CUDA device `device`.  The context owns scenes, BVHs, the
 * scene table, staging buffers and the device error word; all of them count
 * against mem_budget_bytes (0 = no limit).  *out is NULL on failure. */
int sim_create_ctx(sim_ctx** out, int device, const sim_params* p, size_t mem_budget_bytes);

/* Synchronise the device and free everything the context owns. */
int sim_destroy_ctx(sim_ctx* ctx);

/* Replace the context's parameters (affects calls enqueued afterwards). */
int sim_set_params(sim_ctx* ctx, const sim_params* p);

/* Upload a mesh and build its device BVH (Sec. III-B scenes).  The build
 * sorts the triangle centroids' 30-bit Morton codes (radix sort), builds the
 * binary radix tree by longest common prefix (Karras 2012) and refits its boxes
 * bottom-up, then rebuilds the tree above the radix tree's leaves of at most 3
 * triangles by PLOC clustering (Meister and Bittner 2018) and packs it in
 * depth-first order; triangles larger than a quarter of the scene extent stay
 * outside the tree.
 *   verts host float32 [n_verts][3]; tris host int32 [n_tris][3] (vertex
 *   indices, validated); rgb host uint8 [n_tris][3] (flat colour per triangle).
 * On success *scene_id_out receives the id used by sim_render.  The host
 * arrays may be freed when the call returns (it synchronises `stream`).
 * Errors: INVALID_ARG (bad sizes or index out of range), BUDGET, OOM, CUDA. */
int sim_create_scene(sim_ctx* ctx, const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                     const uint8_t* rgb, int32_t* scene_id_out, void* stream);

/* Free a scene's device memory (after synchronising the device).  The id may
 * be reused by a later sim_create_scene. */
int sim_destroy_scene(sim_ctx* ctx, int32_t scene_id);

/* Scene statistics: triangles, BVH nodes, triangles kept outside the BVH
 * (large ones, tested by every ray), BVH depth, resident bytes. */
typedef struct sim_scene_info {
    int64_t n_tris, n_nodes, n_large;
    int32_t depth, leaf_max;
    int64_t bytes;
} sim_scene_info;
int sim_scene_info_get(const sim_ctx* ctx, int32_t scene_id, sim_scene_info* info);

/* Where a scene's build spent its time (Sec. III-B scene set-up; no timing is
 * printed in the paper).  phase_ms host float [SIM_BUILD_PHASES] receives the
 * device time between stream events at the phase boundaries, in order:
 * 0 triangle and scene bounds, 1 centroid bounds and 30-bit Morton codes,
 * 2 radix sort, 3 radix tree (Karras 2012), 4 bottom-up refit, 5 clustering
 * rounds (PLOC, Meister and Bittner 2018), 6 tree packing (binary and 4-wide
 * nodes), 7 triangle and colour packing.  A phase's time includes the host
 * read-back that ends it; phases a scene skips read 0.  wall_ms (host float,
 * nullable) receives the host time of the whole sim_create_scene call.
 * Errors: INVALID_ARG (null context or phase_ms), NOT_FOUND. */
#define SIM_BUILD_PHASES 8
int sim_scene_build_times(const sim_ctx* ctx, int32_t scene_id, float* phase_ms, float* wall_ms);

/* One control step of n agents (Sec. III-A): for each of n_sub sub-steps,
 * body-rate controller -> rotor lag (Eq. 4) -> thrust and moment (Eq. 3) ->
 * RK4 or Euler on Eq. 1 with drag (Eq. 2) -> quaternion normalisation.
 *   state dev float32 [17][n], updated in place; cmd dev float32 [4][n];
 *   ckpt dev float32 [17][n] or NULL: receives the pre-step state. */
int sim_step(sim_ctx* ctx, int32_t n_agents, float* state, const float* cmd, float* ckpt, void* stream);

/* Render every agent's depth / colour / hit-id image (Sec. III-B sensors):
 * one primary ray per pixel centre from the camera at body offset cam_off
 * looking along body +x (image right = body -y, image down = body -z); the
 * closest Moller-Trumbore hit with max_depth >= t > 1e-6, equal t broken by the
 * lowest triangle id; colour is the hit triangle's flat colour, (0,0,0) on a
 * miss.  scene_of_agent dev int32 [n]: the scene id of each agent (ids are
 * checked on the device; an unknown id sets SIM_ERR_NOT_FOUND in the error word
 * and renders that agent as all misses).  Scenes of uneven size are rendered
 * in the same launch through the context's scene table.
 *   state dev [17][n]; depth dev float32 [n][H][W] or NULL; rgb dev uint8
 *   [n][H][W][3] or NULL; hit_id dev int32 [n][H][W] or NULL. */
int sim_render(sim_ctx* ctx, int32_t n_agents, const int32_t* scene_of_agent, const float* state, float* depth,
               uint8_t* rgb, int32_t* hit_id, void* stream);

/* Load analysis of the context's last sim_render launch (no counterpart in
 * the paper): the traversal cost of every image tile -- the node and leaf
 * visits of the warp that rendered it, summed over a split tile's quarters --
 * which is what the next launch's longest-first order is estimated from.
 * costs host uint32 [n][tiles_y][tiles_x] (tiles of the context's render
 * configuration, sim_get_render_config) or NULL to ask for the size only;
 * *n_items receives n * tiles_y * tiles_x.  Synchronises the device.
 * Errors: INVALID_ARG (null n_items, or max_items below the size), NOT_FOUND
 * (no sim_render launch recorded). */
int sim_render_tile_costs(sim_ctx* ctx, uint32_t* costs, int64_t max_items, int64_t* n_items);

/* Device time of the ray-cast kernel alone, per launch (no counterpart in the
 * paper; a measurement aid).  With timing on, every ray-cast launch of the
 * context that is not being captured into a graph -- up to
 * SIM_KERNEL_TIMING_MAX launches after sim_kernel_timing(ctx, 1) -- records one
 * CUDA event just before the kernel (after its estimate kernel) and one just
 * after it, on the launch's stream; the event before it also ends the
 * kernel's overlap with the estimate kernel, so a timed launch is, if
 * anything, slower.  Enabling (again) or disabling clears the record; the
 * first enable creates 2 * SIM_KERNEL_TIMING_MAX events.
 * sim_kernel_times waits for the recorded launches and writes the first
 * min(max, recorded) times in launch order to ms (host float, milliseconds);
 * *count receives the number recorded, and the record is cleared.
 * Errors: INVALID_ARG (null ctx or count, ms NULL with max > 0, negative max),
 * CUDA (event creation or read-back). */
#define SIM_KERNEL_TIMING_MAX 1024
int sim_kernel_timing(sim_ctx* ctx, int32_t enable);
int sim_kernel_times(sim_ctx* ctx, float* ms, int32_t max, int32_t* count);

/* As sim_render with every agent in one scene. */
int sim_render_scene(sim_ctx* ctx, int32_t n_agents, int32_t scene_id, const float* state, float* depth,
                     uint8_t* rgb, int32_t* hit_id, void* stream);

/* As sim_render_scene, but allocates no device memory (no cudaMalloc, no
 * cudaFree, no allocating library call).  The paper has no counterpart: this
 * is for callers that cannot allocate device memory while they run -- a control
 * loop that must not touch the allocator after set-up, or a process whose
 * device memory is handed in full to another framework's pool -- whereas
 * sim_render_scene allocates its agent -> scene id array on every call.
 * Scratch (that id array and the ray-cast kernel's two work counters) lives in
 * one file-scope device array of 256 B + 4 B * SIM_RENDER_STATIC_MAX_AGENTS
 * (256.25 KiB) that every GPU which loads the library holds until the process
 * exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the context's device current; make that first
 * call before any stream capture.  Every call shares the one array and clears
 * its counters before rendering, so calls whose work overlaps on the GPU (other
 * streams, other contexts on the same device) race: serialise them.
 * Errors: INVALID_ARG when n_agents > SIM_RENDER_STATIC_MAX_AGENTS or < 0,
 * or when sim_render_scene would reject the call (null pointers, a BVH deeper
 * than the traversal stack); NOT_FOUND for an unknown scene, also with
 * n_agents = 0; CUDA for a launch failure.  Every check runs before the shared
 * array is written, so a rejected call leaves it as it was. */
#define SIM_RENDER_STATIC_MAX_AGENTS 65536
int sim_render_scene_static(sim_ctx* ctx, int32_t n_agents, int32_t scene_id, const float* state, float* depth,
                            uint8_t* rgb, int32_t* hit_id, void* stream);

/* Nearest obstacle (Sec. III-B: the obstacle-distance module that reports the
 * nearest point of the obstacles without a collision happening): for every
 * agent, the closest point of its scene's mesh to the agent's position.
 *   scene_of_agent dev int32 [n]; state dev [17][n] (rows 0-2 used);
 *   dist dev float32 [n]: distance, or max_dist when nothing is closer;
 *   point dev float32 [3][n] or NULL: the closest point (the agent's position
 *   when nothing is within max_dist); tri dev int32 [n] or NULL: its triangle
 *   (lowest id among equal distances, -1 when nothing is within max_dist). */
int sim_nearest_obstacle(sim_ctx* ctx, int32_t n_agents, const int32_t* scene_of_agent, const float* state,
                         float max_dist, float* dist, float* point, int32_t* tri, void* stream);

/* As sim_render, with a segmentation image as well: seg dev int32 [n][H][W]
 * (or NULL) receives the hit triangle's label (sim_scene_set_labels; the
 * triangle id when the scene has none) and -1 on a miss (the segmentation
 * sensor of Sec. III-B, Fig. 3). */
int sim_render_ex(sim_ctx* ctx, int32_t n_agents, const int32_t* scene_of_agent, const float* state, float* depth,
                  uint8_t* rgb, int32_t* hit_id, int32_t* seg, void* stream);

/* Per-triangle segmentation labels of a scene (host int32 [n_tris], e.g. object
 * ids), or labels = NULL to drop them.  Synchronises the device. */
int sim_scene_set_labels(sim_ctx* ctx, int32_t scene_id, const int32_t* labels, int64_t n_tris);

/* Sensor noise of every later render on this context (domain randomisation of
 * the vision sensors, Sec. III-D, Table II), or cfg = NULL for clean images.
 * Per pixel, in this order: shot noise (Gaussian form: x' = (L + sqrt(L) z) / k
 * with L = k x, k = *_shot, skipped when 0), additive Gaussian (sigma *_gauss),
 * speckle (x' = x (1 + sigma z), sigma *_speckle), salt and pepper (probability
 * *_salt_pepper, then 0 or the maximum with equal chance), clamp to [0, max]
 * (max = max_depth for depth, 255 for colour and seg_max for segmentation labels;
 * colour and labels are then rounded half to even).  Label noise touches only
 * labelled pixels (a miss stays -1) and needs seg_max > 0 and labels below 2^24;
 * afterwards the segmentation image loses a pixel's label (-1) with probability
 * seg_dropout.  Hit ids are never noisy.  Draws come from SplitMix64 (Steele,
 * Lea, Flood 2014) as output number i of the stream `seed`, with
 * i = ((frame * n_agents + agent) * H * W + pixel) * 64 + slot (mod 2^64); slots:
 * depth 0-7, colour channel c 8+8c..15+8c, segmentation 32-39, segmentation
 * dropout 40; within a block of 8: Gaussian 0-1, speckle 2-3, shot 4-5, salt
 * and pepper 6-7 (decision, value).
 * A standard normal from slots (s, s+1): sqrt(-2 ln u1) cos(2 pi u2) with
 * u1 = (x1 >> 40 + 0.5) / 2^24 and u2 = (x2 >> 40) / 2^24; a uniform for a decision
 * is (x >> 40) / 2^24.  `frame` starts at first_frame and advances by one with
 * every render launch.  Synchronises the device. */
typedef struct sim_noise {
    uint64_t seed;
    uint64_t first_frame;
    float depth_gauss, depth_speckle, depth_shot, depth_salt_pepper;
    float rgb_gauss, rgb_speckle, rgb_shot, rgb_salt_pepper;
    float seg_dropout;
    float seg_gauss, seg_speckle, seg_shot, seg_salt_pepper;
    float seg_max;
} sim_noise;
int sim_set_noise(sim_ctx* ctx, const sim_noise* cfg);

/* Multi-agent mode (Sec. III-B: the drones of a multi-agent environment see
 * each other and collide; parallel agents omit each other).  With cfg set,
 * every later render on this context through sim_render, sim_render_ex,
 * sim_render_counted, sim_env_step and loops created afterwards treats the
 * agents of one launch that share a scene as one swarm: each camera also sees
 * the other drones, boxes of half extents `half` (m, body frame, about the
 * body origin), never its own.  A drone hit on agent j (its index in the
 * launch) gives depth as usual, hit id -2 - j, colour `rgb` and segmentation
 * label `label`; exact ties of depth go to the triangle, then to the lower
 * agent index.  cfg = NULL returns to the parallel-agents mode (the default).
 * The server and sim_render_scene_static always render in the
 * parallel-agents mode.  The mode's per-launch buffers belong to the context:
 * swarm renders on one context must not overlap on different streams.
 * INVALID_ARG for non-positive or non-finite extents.  Synchronises the device. */
typedef struct sim_swarm {
    float half[3];
    uint8_t rgb[3];
    int32_t label;
} sim_swarm;
int sim_set_swarm(sim_ctx* ctx, const sim_swarm* cfg);

/* Pairwise proximity of the swarms (Sec. III-B: collisions among the drones
 * of the multi-agent mode), whatever the render mode: for every agent, over
 * the other agents of the launch in its scene, the nearest centre distance
 * (dist, +inf when alone), that agent (other, the lowest index among equal
 * squared distances, -1 when alone) and how many lie closer than 2 * radius
 * (n_collide: drones collide as spheres of `radius`).
 *   scene_of_agent dev int32 [n]; state dev [17][n] (rows 0-2 used); dist dev
 *   float32 [n], other dev int32 [n], n_collide dev int32 [n], each may be NULL.
 * All pairs of a scene are visited (cost proportional to the sum of squared
 * swarm sizes).  Asynchronous on `stream`. */
int sim_swarm_proximity(sim_ctx* ctx, int32_t n_agents, const int32_t* scene_of_agent, const float* state,
                        float radius, float* dist, int32_t* other, int32_t* n_collide, void* stream);

/* Reverse-mode derivative of one sim_step (the dynamics are differentiable,
 * Sec. III-A): given the pre-step state, the command and the cotangent of the
 * post-step state, write the cotangents of the pre-step state and the command.
 * Implemented for the CTBR and SRT controllers (INVALID_ARG for LV / PS).
 * Clamps in the controller pass the gradient inside their range (boundary
 * included) and block it outside.  All dev float32: state_in [17][n], cmd
 * [4][n], g_state_out [17][n] (read), g_state_in [17][n] and g_cmd [4][n]
 * (written; they may not alias the inputs). */
int sim_step_backward(sim_ctx* ctx, int32_t n_agents, const float* state_in, const float* cmd,
                      const float* g_state_out, float* g_state_in, float* g_cmd, void* stream);

/* T steps in one launch (one thread per agent walks the whole horizon).
 *   state0 dev [17][n]; cmds dev [T][4][n]; states_out dev [T+1][17][n] or NULL
 *   (all states, states_out[0] = state0); ckpt dev [ceil(T/K)][17][n] or NULL
 *   (state at steps 0, K, 2K, ...); state_final dev [17][n] or NULL. */
int sim_rollout(sim_ctx* ctx, int32_t n_agents, int32_t T, int32_t K, const float* state0, const float* cmds,
                float* states_out, float* ckpt, float* state_final, void* stream);

/* Reverse sweep over a rollout with recompute from checkpoints every K steps:
 * each agent's thread re-runs K steps from a checkpoint, keeps them locally,
 * and walks them backwards.  g_states dev [T+1][17][n] is the cotangent of
 * every state of the trajectory (e.g. dLoss/dstate_t); outputs g_state0 dev
 * [17][n] and g_cmds dev [T][4][n].  K must be 1..32.
 * With one sub-step per control step the re-run records each step's forward
 * pass (264 B per agent and step) in a context-owned buffer of n * K entries,
 * so the backwards walk does not repeat it.  The buffer is allocated on first
 * need against the memory budget; where the budget refuses it the walk
 * recomputes the forward passes instead (same results, slower). */
int sim_rollout_backward(sim_ctx* ctx, int32_t n_agents, int32_t T, int32_t K, const float* ckpt,
                         const float* cmds, const float* g_states, float* g_state0, float* g_cmds, void* stream);

/* The environment step as a user calls it, with host buffers: commands in,
 * step, render, images (and optionally the state) out.
 *   cmd_host float32 [4][n]; depth_host float32 [n][H][W] or NULL; rgb_host
 *   uint8 [n][H][W][3] or NULL; state_host float32 [17][n] or NULL (post-step
 *   state).  The device state (state dev [17][n]) stays resident and is
 *   updated in place.  Page-locked host buffers (cudaHostAlloc, cudaMallocHost,
 *   cudaHostRegister) are accessed in place by the kernels: the step kernel
 *   reads the commands from host memory and the render writes the images into
 *   host memory as tiles finish, so the download overlaps the ray cast.
 *   Pageable buffers go through device staging and copies after the render.
 *   Asynchronous on `stream`; host buffers must stay valid and untouched until
 *   the stream reaches this point. */
int sim_env_step(sim_ctx* ctx, int32_t n_agents, const int32_t* scene_of_agent, float* state,
                 const float* cmd_host, float* depth_host, uint8_t* rgb_host, float* state_host, void* stream);

/* A prepared environment step: sim_env_step for a fixed set of agents and
 * fixed output buffers, validated once and then run as one captured CUDA graph
 * per call (band-word reset, dynamics, render with the streamed download,
 * optional state download), so a control loop pays one graph launch of host
 * work per step instead of a series of launches and checks.
 *   scene_of_agent dev int32 [n]; state dev [17][n] (updated in place by every
 *   run); depth_host float32 [n][H][W], rgb_host uint8 [n][H][W][3] and
 *   state_host float32 [17][n] are host buffers (at least one image buffer),
 *   each NULL or page-locked (cudaHostAlloc, cudaMallocHost, cudaHostRegister);
 *   INVALID_ARG otherwise.  All of them must stay allocated until
 *   sim_env_destroy.
 * sim_env_run: one step with commands cmd_host float32 [4][n] (page-locked:
 *   read in place; pageable: copied first), asynchronous on `stream`; the host
 *   buffers are complete when the stream reaches this point.  A later change of
 *   the context's parameters, scenes, labels, render configuration, noise or
 *   multi-agent mode is picked up by the next run (it synchronises `stream`
 *   and captures anew).  The prepared step owns its staging, scheduling hints
 *   and work counters, so it does not share them with other launches. */
typedef struct sim_env sim_env;
int sim_env_create(sim_ctx* ctx, sim_env** out, int32_t n_agents, const int32_t* scene_of_agent, float* state,
                   float* depth_host, uint8_t* rgb_host, float* state_host);
int sim_env_run(sim_env* env, const float* cmd_host, void* stream);
int sim_env_destroy(sim_env* env);

/* A captured step loop: T environment steps (sim_step then sim_render per
 * step, commands cmds[t]) recorded once into a CUDA graph and replayed with one
 * launch (the batched-multi-scene pattern: many scenes, one persistent render
 * per step, no per-step host work).
 *   scene_of_agent dev int32 [n]; state dev [17][n] (updated in place by every
 *   replay); cmds dev [T][4][n]; depth dev float32 [F][n][H][W] or NULL, rgb dev
 *   uint8 [F][n][H][W][3] or NULL: step t writes frame slot t % F (F >= 1).
 * The pointers are baked into the graph: the buffers must stay allocated and
 * at the same addresses until sim_loop_destroy.  The loop owns its own work
 * counters, so its replays do not share them with other renders.  The render
 * configuration current at creation is used.  Creation synchronises `stream`. */
typedef struct sim_loop sim_loop;
int sim_loop_create(sim_ctx* ctx, sim_loop** out, int32_t n_agents, int32_t T, const int32_t* scene_of_agent,
                    float* state, const float* cmds, float* depth, uint8_t* rgb, int32_t n_frames, void* stream);
/* Replay the whole loop on `stream` (asynchronous). */
int sim_loop_launch(sim_loop* loop, void* stream);
int sim_loop_destroy(sim_loop* loop);

/* ---------------------------------------------------------------- serving
 * A continuous-batching step server on one context.  Clients submit requests
 * ("advance these n agents of scene s by k steps with these commands and give
 * me the observations"); a server thread keeps scene BVHs and agent states on
 * the device, admits queued requests between device iterations as agent slots
 * and memory free up, packs every active request into one batch, and runs one
 * dynamics launch and one persistent render launch per iteration, so requests
 * of uneven size that arrive while others run share the GPU.  The environment
 * step of Sec. III-C, served.  Results do not depend on what else is in the
 * batch (agents never interact in this mode, Sec. III-B). */
typedef struct sim_server sim_server;

typedef struct sim_request {
    int32_t scene_id;     /* resident scene */
    int32_t n_agents;     /* 1 .. server capacity */
    int32_t n_steps;      /* >= 1 */
    int32_t frames;       /* 0: no images, 1: images of the last step, 2: images of every step */
    const float* state0;  /* [17][n] host or device; read when the request is admitted */
    const float* cmds;    /* [n_steps][4][n] host or device; read when the request is admitted */
    float* state_out;     /* [17][n] final state, or NULL */
    float* depth_out;     /* [n][H][W] (frames = 1) or [n_steps][n][H][W] (frames = 2), or NULL */
    uint8_t* rgb_out;     /* same with a trailing [3], or NULL */
} sim_request;

/* capacity: most agents in one batch (1 .. 1<<20).  The server's batch buffers
 * (two state buffers, commands, scene ids, one frame per agent slot) and each
 * admitted request's device copy of its inputs come from the context's memory
 * budget; a request that does not fit waits in the queue (memory admission). */
int sim_server_create(sim_ctx* ctx, sim_server** out, int32_t capacity);
/* Enqueue a request; *ticket identifies it.  The request's buffers must stay
 * valid until sim_server_wait reports it finished.  INVALID_ARG when n_agents
 * exceeds the capacity or the scene is not resident. */
int sim_server_submit(sim_server* srv, const sim_request* req, int64_t* ticket);
/* Wait up to timeout_ms (< 0: unbounded) for a request to finish.  SIM_OK with
 * *latency_ms = completion - submission time; SIM_ERR_TIMEOUT if still running;
 * SIM_ERR_NOT_FOUND for an unknown (or already collected) ticket; the
 * request's own failure code otherwise (a cancelled request reports
 * SIM_ERR_INVALID_ARG).  Collecting a finished request forgets the ticket. */
int sim_server_wait(sim_server* srv, int64_t ticket, int32_t timeout_ms, double* latency_ms);
/* Cancel a request that has not finished: queued requests are dropped, active
 * ones leave the batch at the next iteration without writing outputs. */
int sim_server_cancel(sim_server* srv, int64_t ticket);
typedef struct sim_server_stats {
    int64_t submitted, completed, cancelled, failed, iterations, agent_frames;
    int64_t queued, active_requests, active_agents;
    double mean_batch_agents;
} sim_server_stats;
int sim_server_stats_get(sim_server* srv, sim_server_stats* stats);
/* Stop the server thread (pending requests are cancelled) and free its memory. */
int sim_server_destroy(sim_server* srv);

/* Ray-cast kernel configuration (the autotuner's search space).
 *   tile_w x tile_h pixels per warp work item, rays_per_lane in {1, 2}
 *   (tile_w * tile_h = 32 * rays_per_lane); stack_in_smem (1: per-warp stack in
 *   shared memory, 0: stack spread over the warp's registers); stack_depth, the
 *   traversal stack's entries: 32 or 64 in registers (one or two registers a
 *   lane), 32, 48 or 64 in shared memory, 64 with 4-wide nodes -- a scene whose
 *   BVH is deeper than a binary stack (as deep as a 4-wide one) is refused
 *   (INVALID_ARG), and the autotuner skips such configurations; warps_per_cta must be 4; ctas_per_sm (persistent grid =
 *   ctas_per_sm * SM count; 0 = as many as fit); stage_in_smem (1: node and
 *   triangle records are fetched by a few lanes with coalesced float4 loads
 *   into shared memory and read back by all lanes; 0: every lane loads the
 *   same address, a broadcast through L1). */
typedef struct sim_render_config {
    int32_t tile_w, tile_h, rays_per_lane, stack_in_smem, stack_depth, warps_per_cta, ctas_per_sm, stage_in_smem;
    int32_t node_width;  /* 2: binary BVH nodes; 4: 4-wide nodes (two binary levels per fetch) */
} sim_render_config;
int sim_get_render_config(const sim_ctx* ctx, sim_render_config* cfg);
int sim_set_render_config(sim_ctx* ctx, const sim_render_config* cfg);

/* Time every supported configuration on the given workload (each `iters`
 * launches, CUDA events on `stream`), select the fastest and return it in
 * *best.  times_ms (may be NULL) receives up to max_times per-config averages
 * in the order of sim_render_config_list; a configuration whose stack is too
 * shallow for the context's deepest scene is not timed and keeps its entry.
 * Synchronises `stream`. */
int sim_autotune_render(sim_ctx* ctx, int32_t n_agents, const int32_t* scene_of_agent, const float* state,
                        float* depth, uint8_t* rgb, int32_t iters, sim_render_config* best, float* times_ms,
                        int32_t max_times, void* stream);
/* The supported configurations (returns how many; fills up to max of them). */
int sim_render_config_list(sim_render_config* out, int32_t max);

/* Traversal counters of one sim_render_counted call.  node_visits and
 * tri_tests count per warp work item (the packet walk); large_tests the large
 * triangles tested per item; need_node_visits and need_tri_tests sum over rays
 * the nodes and triangles that ray's own walk needs (its ray entered the box);
 * items the work items, rays the primary rays. */
typedef struct sim_render_counters {
    int64_t node_visits, tri_tests, large_tests, items, rays, need_node_visits, need_tri_tests;
} sim_render_counters;
int sim_render_counted(sim_ctx* ctx, int32_t n_agents, const int32_t* scene_of_agent, const float* state,
                       float* depth, uint8_t* rgb, int32_t* hit_id, sim_render_counters* counters, void* stream);

/* Wait for `stream` (polling, at most timeout_ms; <0 = unbounded), then read
 * and clear the device error word.  Returns SIM_OK, SIM_ERR_TIMEOUT (work still
 * running), SIM_ERR_CUDA, or the device-reported error. */
int sim_get_status(sim_ctx* ctx, void* stream, int32_t timeout_ms);

/* Message of the last failed call on this thread ("" if none). */
const char* sim_last_error(const sim_ctx* ctx);

/* Bytes currently allocated by the context, and its budget. */
int sim_mem_usage(const sim_ctx* ctx, size_t* used, size_t* budget);

/* Read-bandwidth probe: stream a device buffer of `bytes` (resident in L2 when
 * it fits) `iters` times with float4 loads and report GB/s.  Synchronises. */
int sim_probe_read_bandwidth(sim_ctx* ctx, size_t bytes, int32_t iters, double* gbs, void* stream);

/* Library version string. */
const char* sim_version(void);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* VISFLY_B300_H */

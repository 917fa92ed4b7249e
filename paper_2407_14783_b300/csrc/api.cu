// C ABI of the rollout-step library: contexts, budgeted device memory, the
// segmented scene table, argument checking and kernel launches.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "launch.h"
#include "visfly_b300.h"

using namespace vf;

namespace {
// NVTX range over one entry point (header-only NVTX: a no-op unless a
// profiler is attached), so timelines show which library call ran when.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};
}  // namespace

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA;
}

constexpr int kRing = 64;  // work-counter slots, so renders on different streams do not share one

struct SceneRec {
    bool live = false;
    int32_t* labels = nullptr;  // segmentation labels per triangle (owned), or null
    void* mem[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t bytes = 0;
    int64_t n_tris = 0;
    float build_wall_ms = 0.0f;  // host time of sim_create_scene, upload to table update
    LbvhResult r{};
};

}  // namespace

struct sim_loop {
    sim_ctx* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned* counters = nullptr;
    void* sched_mem = nullptr;
    int sched_cap = 0;
    vf::SwarmScratch swarm;  // the loop's own multi-agent buffers (baked into the graph)
};

// A prepared environment step (sim_env_create): its own buffers and one
// captured graph of band-word reset, dynamics and render.
struct sim_env {
    sim_ctx* ctx = nullptr;
    int n = 0;
    const int32_t* soa = nullptr;
    float* state = nullptr;
    float* h_depth = nullptr;  // device addresses of the page-locked host images
    uint8_t* h_rgb = nullptr;
    float* h_state = nullptr;
    float* d_depth = nullptr;  // render targets (device staging of the streamed download)
    uint8_t* d_rgb = nullptr;
    float* d_cmd = nullptr;    // commands from pageable host memory
    unsigned* band = nullptr;
    size_t band_words = 0, rows_max = 0;
    unsigned* counters = nullptr;
    void* sched_mem = nullptr;
    int sched_cap = 0;
    vf::SwarmScratch swarm;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t step_node = nullptr;
    unsigned long long gen = 0;
    const float* cmd_in_graph = nullptr;
};

struct sim_ctx {
    int device = 0;
    int num_sms = 0;
    sim_params params{};
    DynConsts dyn{};
    CamConsts cam{};
    size_t budget = 0;
    size_t used = 0;
    std::mutex mu;        // scene table
    std::mutex alloc_mu;  // budget accounting
    std::vector<SceneRec> scenes;
    SceneRow* d_table = nullptr;
    int table_cap = 0;
    int* d_err = nullptr;
    unsigned* d_ring = nullptr;  // [kRing][2]
    std::atomic<unsigned> ring_next{0};
    std::atomic<unsigned> launch_id{0};
    NoiseParams noise{};
    unsigned long long* d_noise_frame = nullptr;
    // longest-first scheduling hints shared by sim_render calls (see SchedBuf)
    void* sched_mem = nullptr;
    size_t sched_bytes = 0;
    int sched_cap = 0;
    long long* d_stats = nullptr;
    sim_render_config rcfg{8, 4, 1, 0, 64, 4, 0, 0, 2};  // fastest measured on the large scene
    // staging for sim_env_step
    float* d_cmd = nullptr;
    float* d_depth = nullptr;
    uint8_t* d_rgb = nullptr;
    unsigned* d_band = nullptr;  // completion words of the streamed download
    size_t band_words = 0;
    // tape of the rollout adjoint's forward passes (sim_rollout_backward)
    float* d_tape = nullptr;
    size_t tape_bytes = 0;
    // bumped by every call that changes what a captured environment step
    // launches (parameters, scenes, labels, render config, noise, swarm)
    std::atomic<unsigned long long> generation{1};
    // multi-agent mode (sim_set_swarm) and its per-launch buffers
    bool swarm_on = false;
    sim_swarm swarm_cfg{};
    vf::SwarmScratch swarm;
    int stage_n = 0;
    size_t stage_bytes = 0;
    // device time of each ray-cast launch alone (sim_kernel_timing): event
    // pairs recorded around the kernel, one pair per launch, in launch order
    struct {
        std::mutex mu;
        std::atomic<bool> on{false};
        std::vector<cudaEvent_t> t0, t1;
        int used = 0;
    } ktime;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int ctx_alloc(sim_ctx* c, size_t bytes, void** out) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    if (c->budget && c->used + bytes > c->budget)
        return fail(SIM_ERR_BUDGET, "memory budget exceeded: need " + std::to_string(bytes) + " B, used " +
                                        std::to_string(c->used) + " of " + std::to_string(c->budget));
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    c->used += bytes;
    return SIM_OK;
}
void ctx_free(sim_ctx* c, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    if (bytes == 0) bytes = 16;
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    c->used -= bytes;
}

bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

// Derived constants of the dynamics and the camera, in double then rounded.
int derive(const sim_params& p, DynConsts& d, CamConsts& cam) {
    if (!(p.mass > 0) || !(p.J[0] > 0 && p.J[1] > 0 && p.J[2] > 0) || !(p.arm > 0) || !(p.dt > 0) ||
        p.n_sub < 1 || p.n_sub > kMaxSub || (p.integrator != 0 && p.integrator != 1) || p.width < 1 ||
        p.height < 1 || p.width > 1024 || p.height > 1024 || !(p.fov_deg > 0 && p.fov_deg < 180) ||
        !(p.max_depth > 0) || !(p.omega_max >= p.omega_min) || !(p.c_lag >= 0) || !finite3(p.cam_off) ||
        (p.k[2] == 0 && p.k[1] == 0) || p.k[2] < 0 || p.k[1] < 0 || p.controller < 0 || p.controller > 3)
        return fail(SIM_ERR_INVALID_ARG, "invalid sim_params");
    memset(&d, 0, sizeof(d));
    // FP64 values of the controller constants; the kernels get them as
    // double-float pairs (the x* fields)
    struct {
        double dJ[3], dJK[3], drate_max[3], dhalf_a_max_m, dAinv[4][4], df_lo, df_hi, dk[3], domega_min, domega_max;
        double dmass, dg, dKpos[3], dKvel[3], dKatt[3], dKom[3];
    } w{};
    d.mass = p.mass;
    d.inv_mass = (float)(1.0 / p.mass);
    for (int j = 0; j < 3; ++j) {
        d.J[j] = p.J[j];
        d.invJ[j] = (float)(1.0 / p.J[j]);
        d.JK[j] = (float)((double)p.J[j] * p.K_rate[j]);
        d.rate_max[j] = p.rate_max[j];
        d.drag[j] = (float)(0.5 * p.rho * p.Cd[j] * p.area[j]);
    }
    d.half_a_max_m = (float)(0.5 * (double)p.a_max * p.mass);
    double A[4][4], rx[4], ry[4], sp[4];
    for (int i = 0; i < 4; ++i) {
        const double th = (45.0 + 90.0 * i) * M_PI / 180.0;
        rx[i] = p.arm * std::cos(th);
        ry[i] = p.arm * std::sin(th);
        sp[i] = (i % 2 == 0) ? 1.0 : -1.0;
        A[0][i] = 1.0;
        A[1][i] = ry[i];
        A[2][i] = -rx[i];
        A[3][i] = sp[i] * p.kappa;
        d.mix[0][i] = (float)ry[i];
        d.mix[1][i] = (float)(-rx[i]);
        d.mix[2][i] = (float)(sp[i] * p.kappa);
    }
    // inverse by Gauss-Jordan with partial pivoting
    double M[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 8; ++c) M[r][c] = c < 4 ? A[r][c] : (c - 4 == r ? 1.0 : 0.0);
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
        if (std::fabs(M[piv][col]) < 1e-12) return fail(SIM_ERR_INVALID_ARG, "singular mixer (kappa = 0?)");
        if (piv != col)
            for (int c = 0; c < 8; ++c) std::swap(M[col][c], M[piv][c]);
        const double inv = 1.0 / M[col][col];
        for (int c = 0; c < 8; ++c) M[col][c] *= inv;
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            const double f = M[r][col];
            for (int c = 0; c < 8; ++c) M[r][c] -= f * M[col][c];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            d.Ainv[r][c] = (float)M[r][4 + c];
            w.dAinv[r][c] = M[r][4 + c];
        }
    for (int j = 0; j < 3; ++j) {
        w.dJ[j] = p.J[j];
        w.dJK[j] = (double)p.J[j] * p.K_rate[j];
        w.drate_max[j] = p.rate_max[j];
        w.dk[j] = p.k[j];
    }
    w.dhalf_a_max_m = 0.5 * (double)p.a_max * p.mass;
    d.controller = p.controller;
    w.dmass = p.mass;
    w.dg = p.g;
    for (int j = 0; j < 3; ++j) {
        w.dKpos[j] = p.K_pos[j];
        w.dKvel[j] = p.K_vel[j];
        w.dKatt[j] = p.K_att[j];
        w.dKom[j] = p.K_omega[j];
    }
    w.domega_min = p.omega_min;
    w.domega_max = p.omega_max;
    d.k0 = p.k[0];
    d.k1 = p.k[1];
    d.k2 = p.k[2];
    auto thrust = [&](double w) { return (double)p.k[2] * w * w + (double)p.k[1] * w + (double)p.k[0]; };
    d.f_lo = (float)thrust(p.omega_min);
    d.f_hi = (float)thrust(p.omega_max);
    w.df_lo = thrust(p.omega_min);
    w.df_hi = thrust(p.omega_max);
    // double-float pairs of the controller constants (hi + lo == the double to ~48 bits)
    auto pair = [](double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    for (int j = 0; j < 3; ++j) {
        d.xJ[j] = pair(w.dJ[j]);
        d.xJK[j] = pair(w.dJK[j]);
        d.xrate_max[j] = pair(w.drate_max[j]);
    }
    for (int r = 0; r < 4; ++r)
        for (int k = 0; k < 4; ++k) d.xAinv[r][k] = pair(w.dAinv[r][k]);
    d.xhalf_a_max_m = pair(w.dhalf_a_max_m);
    d.xf_lo = pair(w.df_lo);
    d.xf_hi = pair(w.df_hi);
    d.xk0 = pair(w.dk[0]);
    d.xk1sq = pair(w.dk[1] * w.dk[1]);
    d.x4k2 = pair(4.0 * w.dk[2]);
    d.xhalf_f_hi = pair(0.5 * w.df_hi);
    for (int j = 0; j < 3; ++j) {
        d.xmKpos[j] = pair(w.dmass * w.dKpos[j]);
        d.xmKvel[j] = pair(w.dmass * w.dKvel[j]);
        d.xJKatt[j] = pair(w.dJ[j] * w.dKatt[j]);
        d.xJKom[j] = pair(w.dJ[j] * w.dKom[j]);
    }
    d.xmg = pair(w.dmass * w.dg);
    d.omega_min = p.omega_min;
    d.omega_max = p.omega_max;
    const double h = (double)p.dt / p.n_sub;
    d.h = (float)h;
    d.decay = (float)std::exp(-(double)p.c_lag * h);
    d.g = p.g;
    d.n_sub = p.n_sub;
    d.integrator = p.integrator;
    cam.W = p.width;
    cam.H = p.height;
    cam.pix = (float)(2.0 * std::tan(0.5 * (double)p.fov_deg * M_PI / 180.0) / p.width);
    cam.max_depth = p.max_depth;
    for (int j = 0; j < 3; ++j) cam.cam_off[j] = p.cam_off[j];
    return SIM_OK;
}

int upload_table(sim_ctx* c) {
    const int n = (int)c->scenes.size();
    if (n > c->table_cap) {
        int cap = c->table_cap ? c->table_cap : 16;
        while (cap < n) cap *= 2;
        void* p;
        int rc = ctx_alloc(c, sizeof(SceneRow) * cap, &p);
        if (rc) return rc;
        ctx_free(c, c->d_table, sizeof(SceneRow) * c->table_cap);
        c->d_table = (SceneRow*)p;
        c->table_cap = cap;
    }
    std::vector<SceneRow> rows(n);
    for (int i = 0; i < n; ++i) {
        const SceneRec& s = c->scenes[i];
        SceneRow& r = rows[i];
        memset(&r, 0, sizeof(r));
        r.live = s.live ? 1 : 0;
        if (!s.live) {
            r.root = kEmptyRoot;
            continue;
        }
        r.nodes = s.r.nodes;
        r.wide = s.r.wide;
        r.tris = s.r.tris;
        r.large = s.r.large;
        r.colors = s.r.colors;
        r.labels = s.labels;
        r.root = s.r.root;
        r.n_large = s.r.n_large;
        r.depth = s.r.depth;
        r.n_nodes = s.r.n_nodes;
        r.n_tree_tris = s.r.n_bvh;
    }
    if (n) {
        cudaError_t e = cudaMemcpy(c->d_table, rows.data(), sizeof(SceneRow) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "scene table upload");
    }
    return SIM_OK;
}

// Whether a configuration's traversal stack holds every walk of scenes up to
// `depth` levels (internal levels plus the leaf level).  A binary walk pushes
// at most one entry per internal node on its current root path, and such a
// path holds at most `depth` internal nodes (the deepest internal node's
// children are leaves), so depth <= stack_depth suffices.  A 4-wide node
// pushes up to three; its rule keeps one entry of slack and the kernel's own
// overflow check reports the rest.
bool stack_fits(const sim_render_config& cf, int depth) {
    return cf.node_width == 2 ? depth <= cf.stack_depth : depth < cf.stack_depth;
}

int max_scene_depth(const sim_ctx* c) {
    std::lock_guard<std::mutex> lk(const_cast<sim_ctx*>(c)->mu);
    int d = 0;
    for (const auto& s : c->scenes)
        if (s.live) d = std::max(d, s.r.depth);
    return d;
}

struct AllocCtx {
    sim_ctx* c;
    SceneRec* rec;
    int64_t n_tris;
    int status;
};

// Device buffers of a scene: binary nodes, 4-wide nodes, triangles, large triangles, colours.
void scene_sizes(const LbvhResult& r, int64_t n_tris, size_t sz[5]) {
    sz[0] = (size_t)r.n_nodes * 64;
    sz[1] = (size_t)r.n_bvh * 48;
    sz[2] = (size_t)r.n_large * 48;
    sz[3] = (size_t)n_tris * 4;
    sz[4] = (size_t)r.n_nodes * 128;
}

cudaError_t scene_alloc(void* user, LbvhResult* r) {
    AllocCtx* a = (AllocCtx*)user;
    size_t sz[5];
    scene_sizes(*r, a->n_tris, sz);
    for (int i = 0; i < 5; ++i) {
        int rc = ctx_alloc(a->c, sz[i], &a->rec->mem[i]);
        if (rc) {
            a->status = rc;
            return cudaErrorMemoryAllocation;
        }
        a->rec->bytes += sz[i] ? sz[i] : 16;
    }
    r->nodes = (float4*)a->rec->mem[0];
    r->tris = (float4*)a->rec->mem[1];
    r->large = (float4*)a->rec->mem[2];
    r->colors = (uint32_t*)a->rec->mem[3];
    r->wide = (float4*)a->rec->mem[4];
    return cudaSuccess;
}

void free_scene(sim_ctx* c, SceneRec& s) {
    if (s.labels) ctx_free(c, s.labels, sizeof(int32_t) * (size_t)std::max<int64_t>(s.n_tris, 1));
    s.labels = nullptr;
    size_t sz[5];
    scene_sizes(s.r, s.n_tris, sz);
    for (int i = 0; i < 5; ++i) {
        if (s.mem[i]) ctx_free(c, s.mem[i], sz[i]);
        s.mem[i] = nullptr;
    }
    s.live = false;
    s.bytes = 0;
}

RenderArgs render_args(sim_ctx* c, int n, const int32_t* soa, const float* state, float* depth, uint8_t* rgb,
                       int32_t* hit) {
    std::lock_guard<std::mutex> lk(c->mu);  // scene table pointer and size
    RenderArgs a{};
    a.n_agents = n;
    a.scene_of_agent = soa;
    a.state = state;
    a.depth = depth;
    a.rgb = rgb;
    a.hit_id = hit;
    a.table = c->d_table;
    a.n_scenes = (int)c->scenes.size();
    a.cam = c->cam;
    const unsigned slot = c->ring_next.fetch_add(1) % kRing;
    a.counter = c->d_ring + 2 * slot;
    a.done_ctas = c->d_ring + 2 * slot + 1;
    a.sched = nullptr;
    a.heavy = nullptr;
    a.done = nullptr;
    a.acc = nullptr;
    a.cost = nullptr;
    a.pose = nullptr;
    a.sched_cap = 0;
    a.launch_id = c->launch_id.fetch_add(1) + 1;
    a.seg = nullptr;
    a.noise = c->noise;
    a.noise_frame = c->d_noise_frame;
    // stream the resident scenes into L2 at launch start when they fit in it
    size_t scene_bytes = 0;
    for (const auto& sc : c->scenes)
        if (sc.live) scene_bytes += (size_t)sc.r.n_nodes * 64 + (size_t)sc.r.n_bvh * 48 + (size_t)sc.r.n_large * 48;
    a.prefetch_l2 = scene_bytes <= ((size_t)64 << 20) ? 1 : 0;
    a.err = c->d_err;
    a.counters = c->d_stats;
    return a;
}

int check_render_args(sim_ctx* c, int n, const void* soa, const void* state) {
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    if (n < 0) return fail(SIM_ERR_INVALID_ARG, "negative agent count");
    if (n > 0 && (!soa || !state)) return fail(SIM_ERR_INVALID_ARG, "null scene_of_agent or state");
    // items counted with 4 x 2-pixel tiles: a launch of any supported shape
    // (tiles of 32 pixels or more) then holds fewer than 2^29 items, which the
    // ray cast's 32-bit work-claim arithmetic relies on
    const long long tiles = (long long)((c->cam.W + 7) / 4) * ((c->cam.H + 7) / 2);
    if ((long long)n * tiles >= (1ll << 31)) return fail(SIM_ERR_INVALID_ARG, "too many agents for one launch");
    if (!stack_fits(c->rcfg, max_scene_depth(c)))
        return fail(SIM_ERR_INVALID_ARG, "a scene BVH is deeper than the traversal stack");
    return SIM_OK;
}

// Scheduling hints: a header (kSchedHeaderWords words), kBuckets item lists of
// cap entries, then per item a done mark, a quarter accumulator and the last
// launch's cost, and per agent (at most cap agents) the camera attitudes of the
// last two launches.  Zeroed at allocation.
size_t sched_bytes_for(int cap) {
    return sizeof(unsigned long long) * kSchedHeaderWords + kBuckets * sizeof(unsigned) * (size_t)cap +
           sizeof(unsigned long long) * cap + 2 * sizeof(unsigned) * (size_t)cap + 2 * sizeof(float4) * (size_t)cap;
}

int sched_alloc(sim_ctx* c, int cap, void** mem, cudaStream_t s) {
    int rc = ctx_alloc(c, sched_bytes_for(cap), mem);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(*mem, 0, sched_bytes_for(cap), s);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "schedule reset");
}

void sched_attach(RenderArgs& a, void* mem, int cap) {
    char* p = (char*)mem;
    a.sched = (unsigned long long*)p;
    p += sizeof(unsigned long long) * kSchedHeaderWords;
    a.heavy = (unsigned*)p;
    p += kBuckets * sizeof(unsigned) * (size_t)cap;
    a.done = (unsigned long long*)p;
    p += sizeof(unsigned long long) * (size_t)cap;
    a.acc = (unsigned*)p;
    p += sizeof(unsigned) * (size_t)cap;
    a.cost = (unsigned*)p;
    p += sizeof(unsigned) * (size_t)cap;
    a.pose = (float4*)p;
    a.sched_cap = cap;
}

// The context's shared hint buffer, grown (and reset) when a launch has more
// work items than it holds.
int ctx_sched(sim_ctx* c, long long items, cudaStream_t s) {
    if (items <= c->sched_cap) return SIM_OK;
    int cap = 1 << 16;
    while (cap < items) cap <<= 1;
    void* mem;
    int rc = sched_alloc(c, cap, &mem, s);
    if (rc) return rc;
    if (c->sched_mem) {
        cudaStreamSynchronize(s);
        ctx_free(c, c->sched_mem, c->sched_bytes);
    }
    c->sched_mem = mem;
    c->sched_bytes = sched_bytes_for(cap);
    c->sched_cap = cap;
    return SIM_OK;
}

long long render_items(const sim_ctx* c, int n, const sim_render_config& cfg) {
    const long long tx = (c->cam.W + cfg.tile_w - 1) / cfg.tile_w, ty = (c->cam.H + cfg.tile_h - 1) / cfg.tile_h;
    return (long long)n * tx * ty;
}

void swarm_free(sim_ctx* c, SwarmScratch& w) {
    ctx_free(c, w.drones, (size_t)w.cap_agents * 3 * sizeof(float4));
    ctx_free(c, w.members, (size_t)w.cap_agents * sizeof(int));
    ctx_free(c, w.spheres, (size_t)w.cap_agents * sizeof(float4));
    ctx_free(c, w.off, sizeof(int) * ((size_t)w.cap_scenes + 1));
    ctx_free(c, w.cursor, sizeof(int) * ((size_t)w.cap_scenes + 1));
    ctx_free(c, w.groups, 2 * sizeof(float4) * swarm_group_slots(w.cap_agents, w.cap_scenes));
    w = SwarmScratch{};
}
// Grow w to n agents and `rows` scene rows.  Growing synchronises the device
// (earlier launches may still read the old buffers).
int swarm_reserve(sim_ctx* c, SwarmScratch& w, int n, int rows) {
    if (n <= w.cap_agents && rows <= w.cap_scenes && w.off) return SIM_OK;
    const int na = std::max(std::max(n, w.cap_agents), 1), ns = std::max(std::max(rows, w.cap_scenes), 1);
    cudaDeviceSynchronize();
    swarm_free(c, w);
    void *a = nullptr, *b = nullptr, *o = nullptr, *u = nullptr, *sp = nullptr, *gr = nullptr;
    const size_t gbytes = 2 * sizeof(float4) * swarm_group_slots(na, ns);
    int rc;
    if ((rc = ctx_alloc(c, (size_t)na * 3 * sizeof(float4), &a)) || (rc = ctx_alloc(c, (size_t)na * sizeof(int), &b)) ||
        (rc = ctx_alloc(c, sizeof(int) * ((size_t)ns + 1), &o)) || (rc = ctx_alloc(c, sizeof(int) * ((size_t)ns + 1), &u)) ||
        (rc = ctx_alloc(c, (size_t)na * sizeof(float4), &sp)) || (rc = ctx_alloc(c, gbytes, &gr))) {
        ctx_free(c, a, (size_t)na * 3 * sizeof(float4));
        ctx_free(c, b, (size_t)na * sizeof(int));
        ctx_free(c, o, sizeof(int) * ((size_t)ns + 1));
        ctx_free(c, u, sizeof(int) * ((size_t)ns + 1));
        ctx_free(c, sp, (size_t)na * sizeof(float4));
        return rc;
    }
    w.groups = (float4*)gr;
    w.spheres = (float4*)sp;
    w.drones = (float4*)a;
    w.members = (int*)b;
    w.off = (int*)o;
    w.cursor = (int*)u;
    w.cap_agents = na;
    w.cap_scenes = ns;
    return SIM_OK;
}

// Which multi-agent buffers a render uses: the context's (when the mode is
// on; grown on demand), none (parallel-agents mode), or the caller's own,
// already sized (a captured loop, whose buffer addresses are baked in).
enum class SwarmUse { ctx, none, own };

int do_render(sim_ctx* c, int n, const int32_t* soa, const float* state, float* depth, uint8_t* rgb, int32_t* hit,
              bool count, const sim_render_config& cfg, cudaStream_t s, unsigned* own_counters = nullptr,
              void* sched_mem = nullptr, int sched_cap = 0, int32_t* seg = nullptr, float* host_depth = nullptr,
              uint8_t* host_rgb = nullptr, unsigned* band_done = nullptr, unsigned* tile_bits = nullptr,
              SwarmUse su = SwarmUse::ctx, SwarmScratch* own_swarm = nullptr) {
    if (n == 0) return SIM_OK;
    RenderArgs a = render_args(c, n, soa, state, depth, rgb, hit);
    if (c->swarm_on && su != SwarmUse::none) {
        SwarmScratch* w = su == SwarmUse::own ? own_swarm : &c->swarm;
        if (su == SwarmUse::ctx) {
            const int rc = swarm_reserve(c, *w, n, a.n_scenes);
            if (rc) return rc;
        }
        if (!w || !w->off || n > w->cap_agents || a.n_scenes > w->cap_scenes)
            return fail(SIM_ERR_INVALID_ARG, "multi-agent buffers too small for this launch");
        cudaError_t e = launch_swarm_prep(n, soa, state, a.n_scenes, *w, s);
        if (e == cudaSuccess && n > kSwarmGroupMin) e = launch_swarm_groups(n, a.n_scenes, *w, s);
        if (e != cudaSuccess) return cuda_fail(e, "swarm preparation");
        a.swarm_groups = n > kSwarmGroupMin ? w->groups : nullptr;
        const sim_swarm& sc = c->swarm_cfg;
        a.drones = w->drones;
        a.swarm_off = w->off;
        a.swarm_spheres = w->spheres;
        for (int k = 0; k < 3; ++k) a.swarm_half[k] = sc.half[k];
        a.swarm_radius = std::sqrt(sc.half[0] * sc.half[0] + sc.half[1] * sc.half[1] + sc.half[2] * sc.half[2]);
        a.swarm_rgb = (uint32_t)sc.rgb[0] | ((uint32_t)sc.rgb[1] << 8) | ((uint32_t)sc.rgb[2] << 16);
        a.swarm_label = sc.label;
    }
    a.seg = seg;
    a.host_depth = host_depth;
    a.host_rgb = host_rgb;
    a.band_done = band_done;
    a.tile_bits = tile_bits;
    if (own_counters) {
        a.counter = own_counters;
        a.done_ctas = own_counters + 1;
    }
    if (sched_mem) sched_attach(a, sched_mem, sched_cap);
    int ctas = 0;
    if (cfg.ctas_per_sm > 0) ctas = cfg.ctas_per_sm * c->num_sms;
    cudaEvent_t k0 = nullptr, k1 = nullptr;
    if (c->ktime.on) {
        // not inside a stream capture: there an event would time the capture
        std::lock_guard<std::mutex> lk(c->ktime.mu);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (c->ktime.on && c->ktime.used < (int)c->ktime.t0.size() && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
            cs == cudaStreamCaptureStatusNone) {
            k0 = c->ktime.t0[c->ktime.used];
            k1 = c->ktime.t1[c->ktime.used];
            ++c->ktime.used;
        }
    }
    cudaError_t e = launch_render(a, cfg, ctas, count, s, k0, k1);
    if (e != cudaSuccess) return cuda_fail(e, "ray-cast launch");
    return SIM_OK;
}

}  // namespace

namespace vf {
cudaError_t launch_cfg(const void* kernel, const RenderArgs& a, int warps_per_cta, int ctas, size_t smem,
                       cudaStream_t s) {
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (ctas <= 0) {
        // resident CTAs of a (kernel, block, shared memory) on this device:
        // queried once, then looked up (the query costs microseconds per launch)
        static std::mutex mu;
        static std::map<std::tuple<const void*, int, size_t, int>, int> resident;
        const auto key = std::make_tuple(kernel, warps_per_cta, smem, dev);
        int grid = 0;
        {
            std::lock_guard<std::mutex> lk(mu);
            const auto it = resident.find(key);
            if (it != resident.end()) grid = it->second;
        }
        if (grid == 0) {
            int sms = 0, per_sm = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * warps_per_cta, smem);
            if (e != cudaSuccess) return e;
            grid = std::max(1, per_sm) * sms;
            std::lock_guard<std::mutex> lk(mu);
            resident[key] = grid;
        }
        ctas = grid;
    }
    // never more CTAs than work items need
    const int tiles = ((a.cam.W + 3) / 4) * ((a.cam.H + 1) / 2);  // upper bound over tile shapes
    const long long items = (long long)a.n_agents * tiles;
    const long long need = (items + warps_per_cta - 1) / warps_per_cta;
    if (need < ctas) ctas = (int)std::max(1ll, need);
    void* args[] = {(void*)&a};
    if (!a.sched) return cudaLaunchKernel(kernel, dim3(ctas), dim3(32 * warps_per_cta), args, smem, s);
    // after the schedule's estimate kernel: programmatic dependent launch, so
    // the ray cast's CTAs start (and prefetch the scenes into L2) while the
    // estimate runs; the kernel waits for it before reading the schedule
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(32 * warps_per_cta);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kernel, args);
}
}  // namespace vf

extern "C" {

const char* sim_version(void) { return "visfly_b300 0.1 (sm_103a)"; }

const char* sim_last_error(const sim_ctx*) { return g_err.c_str(); }

int sim_create_ctx(sim_ctx** out, int device, const sim_params* p, size_t mem_budget_bytes) {
    if (!out || !p) return fail(SIM_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(SIM_ERR_INVALID_ARG, "no such device");
    sim_ctx* c = new sim_ctx();
    c->device = device;
    c->budget = mem_budget_bytes;
    int rc = derive(*p, c->dyn, c->cam);
    if (rc) {
        delete c;
        return rc;
    }
    c->params = *p;
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    void *err, *ring, *stats, *nf;
    if ((rc = ctx_alloc(c, sizeof(int), &err)) || (rc = ctx_alloc(c, sizeof(unsigned) * 2 * kRing, &ring)) ||
        (rc = ctx_alloc(c, sizeof(long long) * 8, &stats)) || (rc = ctx_alloc(c, sizeof(unsigned long long), &nf))) {
        sim_destroy_ctx(c);
        return rc;
    }
    c->d_noise_frame = (unsigned long long*)nf;
    cudaMemset(c->d_noise_frame, 0, sizeof(unsigned long long));
    c->d_err = (int*)err;
    c->d_ring = (unsigned*)ring;
    c->d_stats = (long long*)stats;
    cudaMemset(c->d_err, 0, sizeof(int));
    cudaMemset(c->d_ring, 0, sizeof(unsigned) * 2 * kRing);
    cudaMemset(c->d_stats, 0, sizeof(long long) * 8);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        sim_destroy_ctx(c);
        return cuda_fail(e, "context set-up");
    }
    *out = c;
    return SIM_OK;
}

int sim_destroy_ctx(sim_ctx* c) {
    if (!c) return SIM_OK;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    for (auto& s : c->scenes)
        if (s.live) free_scene(c, s);
    ctx_free(c, c->d_table, sizeof(SceneRow) * c->table_cap);
    ctx_free(c, c->d_err, sizeof(int));
    ctx_free(c, c->d_ring, sizeof(unsigned) * 2 * kRing);
    ctx_free(c, c->d_stats, sizeof(long long) * 8);
    ctx_free(c, c->d_noise_frame, sizeof(unsigned long long));
    if (c->sched_mem) ctx_free(c, c->sched_mem, c->sched_bytes);
    if (c->d_tape) ctx_free(c, c->d_tape, c->tape_bytes);
    ctx_free(c, c->d_cmd, 0);
    ctx_free(c, c->d_depth, 0);
    ctx_free(c, c->d_rgb, 0);
    ctx_free(c, c->d_band, 0);
    swarm_free(c, c->swarm);
    for (size_t i = 0; i < c->ktime.t0.size(); ++i) {
        cudaEventDestroy(c->ktime.t0[i]);
        cudaEventDestroy(c->ktime.t1[i]);
    }
    delete c;
    return SIM_OK;
}

int sim_set_params(sim_ctx* c, const sim_params* p) {
    if (!c || !p) return fail(SIM_ERR_INVALID_ARG, "null argument");
    ++c->generation;
    DynConsts d;
    CamConsts cam;
    int rc = derive(*p, d, cam);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    c->params = *p;
    c->dyn = d;
    c->cam = cam;
    return SIM_OK;
}

int sim_create_scene(sim_ctx* c, const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                     const uint8_t* rgb, int32_t* scene_id_out, void* stream) {
    Range nvtx_range("sim_create_scene");
    if (!c || !scene_id_out) return fail(SIM_ERR_INVALID_ARG, "null argument");
    ++c->generation;
    *scene_id_out = -1;
    if (n_verts < 0 || n_tris < 0 || n_tris > (1ll << 27) || n_verts > (1ll << 31))
        return fail(SIM_ERR_INVALID_ARG, "bad mesh size");
    if ((n_verts > 0 && !verts) || (n_tris > 0 && (!tris || !rgb)))
        return fail(SIM_ERR_INVALID_ARG, "null mesh array");
    for (int64_t i = 0; i < 3 * n_tris; ++i)
        if (tris[i] < 0 || tris[i] >= n_verts) return fail(SIM_ERR_INVALID_ARG, "triangle index out of range");
    for (int64_t i = 0; i < 3 * n_verts; ++i)
        if (!std::isfinite(verts[i])) return fail(SIM_ERR_INVALID_ARG, "non-finite vertex");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const auto t_start = std::chrono::steady_clock::now();
    SceneRec rec;
    rec.n_tris = n_tris;
    const size_t vb = sizeof(float) * 3 * std::max<int64_t>(n_verts, 1);
    const size_t tb = sizeof(int32_t) * 3 * std::max<int64_t>(n_tris, 1);
    const size_t cb = 3 * std::max<int64_t>(n_tris, 1);
    const size_t sb = lbvh_scratch_bytes(n_tris);
    void *dv = nullptr, *dt = nullptr, *dc = nullptr, *ds = nullptr;
    int rc;
    if ((rc = ctx_alloc(c, vb, &dv)) || (rc = ctx_alloc(c, tb, &dt)) || (rc = ctx_alloc(c, cb, &dc)) ||
        (rc = ctx_alloc(c, sb, &ds))) {
        ctx_free(c, dv, vb);
        ctx_free(c, dt, tb);
        ctx_free(c, dc, cb);
        ctx_free(c, ds, sb);
        return rc;
    }
    auto cleanup = [&]() {
        ctx_free(c, dv, vb);
        ctx_free(c, dt, tb);
        ctx_free(c, dc, cb);
        ctx_free(c, ds, sb);
    };
    cudaError_t e = cudaSuccess;
    if (n_verts) e = cudaMemcpyAsync(dv, verts, sizeof(float) * 3 * n_verts, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_tris) e = cudaMemcpyAsync(dt, tris, sizeof(int32_t) * 3 * n_tris, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_tris) e = cudaMemcpyAsync(dc, rgb, 3 * n_tris, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "mesh upload");
    }
    AllocCtx ac{c, &rec, n_tris, SIM_OK};
    if (n_tris == 0) {
        rec.r = LbvhResult{};
        rec.r.root = kEmptyRoot;
        e = scene_alloc(&ac, &rec.r);
    } else {
        e = lbvh_build(n_tris, (const float*)dv, (const int*)dt, (const uint8_t*)dc, ds, scene_alloc, &ac, &rec.r, s);
    }
    cleanup();
    if (e != cudaSuccess) {
        size_t sz[5];
        scene_sizes(rec.r, n_tris, sz);
        for (int i = 0; i < 5; ++i) {
            if (rec.mem[i]) ctx_free(c, rec.mem[i], sz[i]);
        }
        if (ac.status) return ac.status;
        return cuda_fail(e, "BVH build");
    }
    rec.live = true;
    int id = -1;
    for (int i = 0; i < (int)c->scenes.size(); ++i)
        if (!c->scenes[i].live) {
            id = i;
            break;
        }
    if (id < 0) {
        id = (int)c->scenes.size();
        c->scenes.push_back(rec);
    } else {
        c->scenes[id] = rec;
    }
    rc = upload_table(c);
    if (rc) {
        free_scene(c, c->scenes[id]);
        return rc;
    }
    c->scenes[id].build_wall_ms =
        std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    *scene_id_out = id;
    return SIM_OK;
}

int sim_destroy_scene(sim_ctx* c, int32_t id) {
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    ++c->generation;
    std::lock_guard<std::mutex> lk(c->mu);
    if (id < 0 || id >= (int)c->scenes.size() || !c->scenes[id].live) return fail(SIM_ERR_NOT_FOUND, "no such scene");
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    free_scene(c, c->scenes[id]);
    return upload_table(c);
}

int sim_scene_info_get(const sim_ctx* c, int32_t id, sim_scene_info* info) {
    if (!c || !info) return fail(SIM_ERR_INVALID_ARG, "null argument");
    if (id < 0 || id >= (int)c->scenes.size() || !c->scenes[id].live) return fail(SIM_ERR_NOT_FOUND, "no such scene");
    const SceneRec& s = c->scenes[id];
    info->n_tris = s.n_tris;
    info->n_nodes = s.r.n_nodes;
    info->n_large = s.r.n_large;
    info->depth = s.r.depth;
    info->leaf_max = kLeafMax;
    info->bytes = (int64_t)s.bytes;
    return SIM_OK;
}

int sim_scene_build_times(const sim_ctx* c, int32_t id, float* phase_ms, float* wall_ms) {
    if (!c || !phase_ms) return fail(SIM_ERR_INVALID_ARG, "null argument");
    if (id < 0 || id >= (int)c->scenes.size() || !c->scenes[id].live) return fail(SIM_ERR_NOT_FOUND, "no such scene");
    static_assert(kBuildPhases == SIM_BUILD_PHASES, "phase count of the ABI");
    const SceneRec& s = c->scenes[id];
    for (int i = 0; i < kBuildPhases; ++i) phase_ms[i] = s.r.phase_ms[i];
    if (wall_ms) *wall_ms = s.build_wall_ms;
    return SIM_OK;
}

int sim_step(sim_ctx* c, int32_t n, float* state, const float* cmd, float* ckpt, void* stream) {
    Range nvtx_range("sim_step");
    if (!c || n < 0 || (n > 0 && (!state || !cmd))) return fail(SIM_ERR_INVALID_ARG, "bad sim_step arguments");
    DeviceGuard g(c->device);
    cudaError_t e = launch_step(c->dyn, n, state, cmd, ckpt, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "sim_step launch");
}

int sim_step_backward(sim_ctx* c, int32_t n, const float* state_in, const float* cmd, const float* g_out,
                      float* g_in, float* g_cmd, void* stream) {
    Range nvtx_range("sim_step_backward");
    if (!c || n < 0 || (n > 0 && (!state_in || !cmd || !g_out || !g_in || !g_cmd)))
        return fail(SIM_ERR_INVALID_ARG, "bad sim_step_backward arguments");
    if (c->dyn.controller > 1) return fail(SIM_ERR_INVALID_ARG, "the adjoint covers the CTBR and SRT controllers");
    DeviceGuard g(c->device);
    cudaError_t e = launch_step_backward(c->dyn, n, state_in, cmd, g_out, g_in, g_cmd, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "sim_step_backward launch");
}

int sim_rollout(sim_ctx* c, int32_t n, int32_t T, int32_t K, const float* state0, const float* cmds, float* states_out,
                float* ckpt, float* state_final, void* stream) {
    Range nvtx_range("sim_rollout");
    if (!c || n < 0 || T < 0 || K < 1 || (n > 0 && (!state0 || (T > 0 && !cmds))))
        return fail(SIM_ERR_INVALID_ARG, "bad sim_rollout arguments");
    DeviceGuard g(c->device);
    cudaError_t e = launch_rollout(c->dyn, n, T, K, state0, cmds, states_out, ckpt, state_final, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "sim_rollout launch");
}

int sim_rollout_backward(sim_ctx* c, int32_t n, int32_t T, int32_t K, const float* ckpt, const float* cmds,
                         const float* g_states, float* g_state0, float* g_cmds, void* stream) {
    Range nvtx_range("sim_rollout_backward");
    if (!c || n < 0 || T < 1 || K < 1 || K > kMaxCkptK ||
        (n > 0 && (!ckpt || !cmds || !g_states || !g_state0 || !g_cmds)))
        return fail(SIM_ERR_INVALID_ARG, "bad sim_rollout_backward arguments");
    if (c->dyn.controller > 1) return fail(SIM_ERR_INVALID_ARG, "the adjoint covers the CTBR and SRT controllers");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    // With one sub-step per control step the adjoint records each step's
    // forward pass instead of running it twice; the tape is grown on demand
    // and, where the memory budget refuses it, the sweep recomputes instead.
    float* tape = nullptr;
    if (c->dyn.n_sub == 1 && n > 0) {
        const size_t need = rollout_tape_bytes(n, K);
        if (need > c->tape_bytes) {
            cudaStreamSynchronize(s);
            if (c->d_tape) ctx_free(c, c->d_tape, c->tape_bytes);
            c->d_tape = nullptr;
            c->tape_bytes = 0;
            void* p = nullptr;
            const std::string before = g_err;
            if (ctx_alloc(c, need, &p) == SIM_OK) {
                c->d_tape = (float*)p;
                c->tape_bytes = need;
            } else {
                g_err = before;  // not an error of this call: it recomputes instead
            }
        }
        tape = c->d_tape;
    }
    cudaError_t e = launch_rollout_backward(c->dyn, n, T, K, ckpt, cmds, g_states, g_state0, g_cmds, tape, s);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "sim_rollout_backward launch");
}

int sim_render_ex(sim_ctx* c, int32_t n, const int32_t* soa, const float* state, float* depth, uint8_t* rgb,
                  int32_t* hit, int32_t* seg, void* stream) {
    Range nvtx_range("sim_render_ex");
    int rc = check_render_args(c, n, soa, state);
    if (rc) return rc;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const sim_render_config cfg = c->rcfg;
    if ((rc = ctx_sched(c, render_items(c, n, cfg), s))) return rc;
    return do_render(c, n, soa, state, depth, rgb, hit, false, cfg, s, nullptr, c->sched_mem, c->sched_cap, seg);
}

int sim_kernel_timing(sim_ctx* c, int32_t enable) {
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    std::lock_guard<std::mutex> lk(c->ktime.mu);
    if (enable && c->ktime.t0.empty()) {
        DeviceGuard g(c->device);
        for (int i = 0; i < SIM_KERNEL_TIMING_MAX; ++i) {
            cudaEvent_t a = nullptr, b = nullptr;
            cudaError_t e = cudaEventCreate(&a);
            if (e == cudaSuccess) e = cudaEventCreate(&b);
            if (e != cudaSuccess) {
                if (a) cudaEventDestroy(a);
                return cuda_fail(e, "timing events");
            }
            c->ktime.t0.push_back(a);
            c->ktime.t1.push_back(b);
        }
    }
    c->ktime.on = enable != 0;
    c->ktime.used = 0;
    return SIM_OK;
}

int sim_kernel_times(sim_ctx* c, float* ms, int32_t max, int32_t* count) {
    if (!c || !count || (max > 0 && !ms) || max < 0) return fail(SIM_ERR_INVALID_ARG, "null or negative argument");
    std::lock_guard<std::mutex> lk(c->ktime.mu);
    DeviceGuard g(c->device);
    const int n = c->ktime.used;
    *count = n;
    c->ktime.used = 0;
    for (int i = 0; i < n && i < max; ++i) {
        cudaError_t e = cudaEventSynchronize(c->ktime.t1[i]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms + i, c->ktime.t0[i], c->ktime.t1[i]);
        if (e != cudaSuccess) return cuda_fail(e, "kernel timing read-back");
    }
    return SIM_OK;
}

int sim_render_tile_costs(sim_ctx* c, uint32_t* costs, int64_t max_items, int64_t* n_items) {
    if (!c || !n_items) return fail(SIM_ERR_INVALID_ARG, "null argument");
    *n_items = 0;
    if (!c->sched_mem) return fail(SIM_ERR_NOT_FOUND, "no render launch recorded yet");
    DeviceGuard g(c->device);
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long hdr[kSchedHeaderWords];
    if (e == cudaSuccess) e = cudaMemcpy(hdr, c->sched_mem, sizeof(hdr), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "schedule read-back");
    const long long total = (long long)hdr[kSchedTotal];
    const int tiles_x = (int)(hdr[kSchedShape] & 0xFFFFu), tiles_y = (int)((hdr[kSchedShape] >> 16) & 0xFFFFu);
    const long long n = (long long)(hdr[kSchedShape] >> 32);
    if (total <= 0 || total > c->sched_cap || total != n * tiles_x * tiles_y)
        return fail(SIM_ERR_NOT_FOUND, "no render launch recorded yet");
    *n_items = total;
    if (!costs) return SIM_OK;
    if (max_items < total) return fail(SIM_ERR_INVALID_ARG, "cost buffer smaller than the launch's tile count");
    RenderArgs a{};
    sched_attach(a, c->sched_mem, c->sched_cap);
    std::vector<uint32_t> by_item((size_t)total);
    e = cudaMemcpy(by_item.data(), a.cost, sizeof(uint32_t) * (size_t)total, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "schedule read-back");
    // item = (rank row * tiles_x + tx) * n + agent; rank rows run from the image centre outwards
    const int mid = tiles_y >> 1;
    for (int rr = 0; rr < tiles_y; ++rr) {
        const int ty = (rr & 1) ? mid - 1 - (rr >> 1) : mid + (rr >> 1);
        for (int tx = 0; tx < tiles_x; ++tx)
            for (long long ag = 0; ag < n; ++ag)
                costs[(ag * tiles_y + ty) * tiles_x + tx] = by_item[(size_t)(((long long)rr * tiles_x + tx) * n + ag)];
    }
    return SIM_OK;
}

int sim_render(sim_ctx* c, int32_t n, const int32_t* soa, const float* state, float* depth, uint8_t* rgb,
               int32_t* hit, void* stream) {
    return sim_render_ex(c, n, soa, state, depth, rgb, hit, nullptr, stream);
}

int sim_set_swarm(sim_ctx* c, const sim_swarm* cfg) {
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    ++c->generation;
    if (cfg) {
        for (int k = 0; k < 3; ++k)
            if (!(cfg->half[k] > 0.0f) || !std::isfinite(cfg->half[k]))
                return fail(SIM_ERR_INVALID_ARG, "drone half extents must be finite and > 0");
    }
    DeviceGuard g(c->device);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "swarm set-up");
    c->swarm_on = cfg != nullptr;
    if (cfg) c->swarm_cfg = *cfg;
    return SIM_OK;
}

int sim_swarm_proximity(sim_ctx* c, int32_t n, const int32_t* soa, const float* state, float radius, float* dist,
                        int32_t* other, int32_t* n_collide, void* stream) {
    Range nvtx_range("sim_swarm_proximity");
    int rc = check_render_args(c, n, soa, state);
    if (rc) return rc;
    if (!(radius >= 0.0f) || !std::isfinite(radius)) return fail(SIM_ERR_INVALID_ARG, "radius must be finite and >= 0");
    if (n == 0) return SIM_OK;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rows;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        rows = (int)c->scenes.size();
    }
    if ((rc = swarm_reserve(c, c->swarm, n, rows))) return rc;
    cudaError_t e = launch_swarm_prep(n, soa, state, rows, c->swarm, s);
    if (e == cudaSuccess) e = launch_swarm_proximity(n, soa, state, rows, c->swarm, radius, dist, other, n_collide, s);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "swarm proximity");
}

int sim_set_noise(sim_ctx* c, const sim_noise* cfg) {
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    ++c->generation;
    NoiseParams np{};
    unsigned long long frame = 0;
    if (cfg) {
        const float v[14] = {cfg->depth_gauss, cfg->depth_speckle, cfg->depth_shot, cfg->depth_salt_pepper,
                             cfg->rgb_gauss,   cfg->rgb_speckle,   cfg->rgb_shot,   cfg->rgb_salt_pepper,
                             cfg->seg_dropout, cfg->seg_gauss,     cfg->seg_speckle, cfg->seg_shot,
                             cfg->seg_salt_pepper, cfg->seg_max};
        for (float x : v)
            if (!(x >= 0.0f) || !std::isfinite(x)) return fail(SIM_ERR_INVALID_ARG, "noise parameters must be >= 0");
        if (cfg->depth_salt_pepper > 1 || cfg->rgb_salt_pepper > 1 || cfg->seg_dropout > 1 ||
            cfg->seg_salt_pepper > 1)
            return fail(SIM_ERR_INVALID_ARG, "probabilities must be <= 1");
        const bool seg_models =
            cfg->seg_gauss > 0 || cfg->seg_speckle > 0 || cfg->seg_shot > 0 || cfg->seg_salt_pepper > 0;
        if (seg_models && !(cfg->seg_max > 0 && cfg->seg_max < 16777216.0f))
            return fail(SIM_ERR_INVALID_ARG, "segmentation label noise needs 0 < seg_max < 2^24");
        np.enabled = 1;
        np.seed = cfg->seed;
        np.d_gauss = cfg->depth_gauss;
        np.d_speckle = cfg->depth_speckle;
        np.d_shot = cfg->depth_shot;
        np.d_sp = cfg->depth_salt_pepper;
        np.c_gauss = cfg->rgb_gauss;
        np.c_speckle = cfg->rgb_speckle;
        np.c_shot = cfg->rgb_shot;
        np.c_sp = cfg->rgb_salt_pepper;
        np.s_drop = cfg->seg_dropout;
        np.s_gauss = cfg->seg_gauss;
        np.s_speckle = cfg->seg_speckle;
        np.s_shot = cfg->seg_shot;
        np.s_sp = cfg->seg_salt_pepper;
        np.s_max = cfg->seg_max;
        np.s_models = seg_models ? 1 : 0;
        frame = cfg->first_frame;
    }
    DeviceGuard g(c->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c->d_noise_frame, &frame, sizeof(frame), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "noise set-up");
    c->noise = np;
    return SIM_OK;
}

int sim_scene_set_labels(sim_ctx* c, int32_t id, const int32_t* labels, int64_t n) {
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    ++c->generation;
    std::lock_guard<std::mutex> lk(c->mu);
    if (id < 0 || id >= (int)c->scenes.size() || !c->scenes[id].live) return fail(SIM_ERR_NOT_FOUND, "no such scene");
    SceneRec& r = c->scenes[id];
    if (labels && n != r.n_tris) return fail(SIM_ERR_INVALID_ARG, "need one label per triangle");
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    if (r.labels) ctx_free(c, r.labels, sizeof(int32_t) * (size_t)std::max<int64_t>(r.n_tris, 1));
    r.labels = nullptr;
    if (labels && n > 0) {
        void* p;
        int rc = ctx_alloc(c, sizeof(int32_t) * n, &p);
        if (rc) return rc;
        cudaError_t e = cudaMemcpy(p, labels, sizeof(int32_t) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            ctx_free(c, p, sizeof(int32_t) * n);
            return cuda_fail(e, "label upload");
        }
        r.labels = (int32_t*)p;
    }
    return upload_table(c);
}

int sim_render_counted(sim_ctx* c, int32_t n, const int32_t* soa, const float* state, float* depth, uint8_t* rgb,
                       int32_t* hit, sim_render_counters* out, void* stream) {
    Range nvtx_range("sim_render_counted");
    int rc = check_render_args(c, n, soa, state);
    if (rc) return rc;
    if (!out) return fail(SIM_ERR_INVALID_ARG, "null counters");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(c->d_stats, 0, sizeof(long long) * 8, s);
    if (e != cudaSuccess) return cuda_fail(e, "counter reset");
    rc = do_render(c, n, soa, state, depth, rgb, hit, true, c->rcfg, s);
    if (rc) return rc;
    long long h[8];
    e = cudaMemcpyAsync(h, c->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "counter read");
    out->node_visits = h[0];
    out->tri_tests = h[1];
    out->large_tests = h[2];
    out->items = h[3];
    out->rays = (int64_t)n * c->cam.W * c->cam.H;
    out->need_node_visits = h[4];
    out->need_tri_tests = h[5];
    return SIM_OK;
}

int sim_render_scene(sim_ctx* c, int32_t n, int32_t scene_id, const float* state, float* depth, uint8_t* rgb,
                     int32_t* hit, void* stream) {
    Range nvtx_range("sim_render_scene");
    // a device array of n copies of scene_id is needed; keep a small cache in the context staging area
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    if (scene_id < 0 || scene_id >= (int)c->scenes.size() || !c->scenes[scene_id].live)
        return fail(SIM_ERR_NOT_FOUND, "no such scene");
    if (n <= 0) return n == 0 ? SIM_OK : fail(SIM_ERR_INVALID_ARG, "negative agent count");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    void* p;
    int rc = ctx_alloc(c, sizeof(int32_t) * n, &p);
    if (rc) return rc;
    std::vector<int32_t> ids(n, scene_id);
    cudaError_t e = cudaMemcpyAsync(p, ids.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ctx_free(c, p, sizeof(int32_t) * n);
        return cuda_fail(e, "scene id upload");
    }
    rc = sim_render(c, n, (const int32_t*)p, state, depth, rgb, hit, stream);
    cudaStreamSynchronize(s);
    ctx_free(c, p, sizeof(int32_t) * n);
    return rc;
}

// Device address of a host buffer that kernels can reach directly (page-locked
// host memory under unified addressing: cudaHostAlloc, cudaMallocHost or
// cudaHostRegister), else null (pageable memory goes through staging copies).
static void* direct_host_address(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int sim_env_step(sim_ctx* c, int32_t n, const int32_t* soa, float* state, const float* cmd_host, float* depth_host,
                 uint8_t* rgb_host, float* state_host, void* stream) {
    Range nvtx_range("sim_env_step");
    if (!c || n < 0 || (n > 0 && (!soa || !state || !cmd_host)))
        return fail(SIM_ERR_INVALID_ARG, "bad sim_env_step arguments");
    if (n == 0) return SIM_OK;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t px = (size_t)n * c->cam.W * c->cam.H;
    // Page-locked buffers are used in place: the step kernel reads the commands
    // from host memory (no upload), and the render streams the images out band
    // by band while it runs.  The images are still rendered into device staging
    // first: storing each tile's rows straight into host memory was measured
    // slower (0.67 vs 0.44 ms per 256-agent step), because the short row
    // segments of a tile cross the bus as separate writes and stall the warps;
    // a completed band is one contiguous span copied in 16-byte pieces.
    const float* cmd_dev = (const float*)direct_host_address(cmd_host);
    float* hd = (float*)direct_host_address(depth_host);
    uint8_t* hr = (uint8_t*)direct_host_address(rgb_host);
    const bool need_cmd = !cmd_dev, need_depth = depth_host != nullptr, need_rgb = rgb_host != nullptr;
    const bool streamed = (need_depth || need_rgb) && (!need_depth || hd) && (!need_rgb || hr);
    // capacity in agents and in pixels: the image size can change with sim_set_params
    if ((need_cmd || need_depth || need_rgb) && (n > c->stage_n || px > c->stage_bytes)) {
        cudaStreamSynchronize(s);
        ctx_free(c, c->d_cmd, sizeof(float) * 4 * c->stage_n);
        ctx_free(c, c->d_depth, sizeof(float) * c->stage_bytes);
        ctx_free(c, c->d_rgb, 3 * c->stage_bytes);
        c->d_cmd = nullptr;
        c->d_depth = nullptr;
        c->d_rgb = nullptr;
        c->stage_n = 0;
        c->stage_bytes = 0;
        void *a, *b, *d;
        int rc;
        if ((rc = ctx_alloc(c, sizeof(float) * 4 * n, &a))) return rc;
        if ((rc = ctx_alloc(c, sizeof(float) * px, &b))) {
            ctx_free(c, a, sizeof(float) * 4 * n);
            return rc;
        }
        if ((rc = ctx_alloc(c, 3 * px, &d))) {
            ctx_free(c, a, sizeof(float) * 4 * n);
            ctx_free(c, b, sizeof(float) * px);
            return rc;
        }
        c->d_cmd = (float*)a;
        c->d_depth = (float*)b;
        c->d_rgb = (uint8_t*)d;
        c->stage_n = n;
        c->stage_bytes = px;  // pixels
    }
    // per agent: one counter per tile row and one word per tile, sized for the
    // smallest tiles (4 x 2 pixels bound every configuration from below)
    const size_t rows_max = (size_t)c->cam.H, tiles_max = (size_t)((c->cam.W + 3) / 4) * ((c->cam.H + 1) / 2);
    const size_t bands = (size_t)n * (rows_max + tiles_max);
    if (streamed && bands > c->band_words) {
        cudaStreamSynchronize(s);
        ctx_free(c, c->d_band, sizeof(unsigned) * c->band_words);
        c->d_band = nullptr;
        c->band_words = 0;
        void* a;
        int rc;
        if ((rc = ctx_alloc(c, sizeof(unsigned) * bands, &a))) return rc;
        c->d_band = (unsigned*)a;
        c->band_words = bands;
    }
    cudaError_t e = cudaSuccess;
    if (need_cmd) {
        e = cudaMemcpyAsync(c->d_cmd, cmd_host, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "command upload");
        cmd_dev = c->d_cmd;
    }
    int rc = sim_step(c, n, state, cmd_dev, nullptr, stream);
    if (rc) return rc;
    if (streamed) {
        // counters start from zero every call, so a launch that stopped early
        // (a device-detected fault) cannot leave the next one miscounting
        e = cudaMemsetAsync(c->d_band, 0, sizeof(unsigned) * bands, s);
        if (e != cudaSuccess) return cuda_fail(e, "band counters");
        if ((rc = check_render_args(c, n, soa, state))) return rc;
        const sim_render_config cfg = c->rcfg;
        if ((rc = ctx_sched(c, render_items(c, n, cfg), s))) return rc;
        rc = do_render(c, n, soa, state, need_depth ? c->d_depth : nullptr, need_rgb ? c->d_rgb : nullptr, nullptr,
                       false, cfg, s, nullptr, c->sched_mem, c->sched_cap, nullptr, hd, hr, c->d_band,
                       c->d_band + (size_t)n * rows_max);
        if (rc) return rc;
    } else if (need_depth || need_rgb) {
        rc = sim_render(c, n, soa, state, need_depth ? c->d_depth : nullptr, need_rgb ? c->d_rgb : nullptr, nullptr,
                        stream);
        if (rc) return rc;
        if (need_depth) e = cudaMemcpyAsync(depth_host, c->d_depth, sizeof(float) * px, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && need_rgb) e = cudaMemcpyAsync(rgb_host, c->d_rgb, 3 * px, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess && state_host)
        e = cudaMemcpyAsync(state_host, state, sizeof(float) * 17 * n, cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "observation download");
}

// ------------------------------------------------------------ prepared step
namespace {

void env_free(sim_env* E) {
    sim_ctx* c = E->ctx;
    if (E->exec) cudaGraphExecDestroy(E->exec);
    if (E->graph) cudaGraphDestroy(E->graph);
    E->exec = nullptr;
    E->graph = nullptr;
    const size_t px = (size_t)E->n * c->cam.W * c->cam.H;
    ctx_free(c, E->d_depth, sizeof(float) * px);
    ctx_free(c, E->d_rgb, 3 * px);
    ctx_free(c, E->d_cmd, sizeof(float) * 4 * (size_t)E->n);
    ctx_free(c, E->band, sizeof(unsigned) * E->band_words);
    ctx_free(c, E->counters, 2 * sizeof(unsigned));
    if (E->sched_mem) ctx_free(c, E->sched_mem, sched_bytes_for(E->sched_cap));
    swarm_free(c, E->swarm);
    if (E->cap) cudaStreamDestroy(E->cap);
}

// (Re)capture the step graph: band-word reset, dynamics, render with the
// streamed download, and the optional state download.  The caller has made
// sure nothing of an earlier capture is still running.
int env_capture(sim_env* E, const float* cmd) {
    sim_ctx* c = E->ctx;
    if (E->exec) cudaGraphExecDestroy(E->exec);
    if (E->graph) cudaGraphDestroy(E->graph);
    E->exec = nullptr;
    E->graph = nullptr;
    const unsigned long long gen = c->generation.load();
    int rc = check_render_args(c, E->n, E->soa, E->state);
    if (rc) return rc;
    const sim_render_config cfg = c->rcfg;
    const long long items = render_items(c, E->n, cfg);
    if (items > E->sched_cap) {
        if (E->sched_mem) ctx_free(c, E->sched_mem, sched_bytes_for(E->sched_cap));
        E->sched_mem = nullptr;
        E->sched_cap = 0;
        if ((rc = sched_alloc(c, (int)items, &E->sched_mem, E->cap))) return rc;
        E->sched_cap = (int)items;
    }
    if (c->swarm_on) {
        int rows;
        {
            std::lock_guard<std::mutex> lk(c->mu);
            rows = (int)c->scenes.size();
        }
        if ((rc = swarm_reserve(c, E->swarm, E->n, rows))) return rc;
    }
    cudaError_t e = cudaStreamSynchronize(E->cap);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(E->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "environment capture");
    e = cudaMemsetAsync(E->band, 0, sizeof(unsigned) * E->band_words, E->cap);
    if (e == cudaSuccess) e = launch_step(c->dyn, E->n, E->state, cmd, nullptr, E->cap);
    if (e == cudaSuccess) {
        // the node just added is the dynamics kernel: its command argument is
        // rebound per call without a new capture
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(E->cap, &st, nullptr, nullptr, &deps, nullptr, &nd);
        E->step_node = (e == cudaSuccess && nd == 1) ? deps[0] : nullptr;
        if (e == cudaSuccess && !E->step_node) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess)
        rc = do_render(c, E->n, E->soa, E->state, E->d_depth, E->d_rgb, nullptr, false, cfg, E->cap, E->counters,
                       E->sched_mem, E->sched_cap, nullptr, E->h_depth, E->h_rgb, E->band,
                       E->band + (size_t)E->n * E->rows_max, c->swarm_on ? SwarmUse::own : SwarmUse::none,
                       &E->swarm);
    if (e == cudaSuccess && rc == SIM_OK && E->h_state)
        e = cudaMemcpyAsync(E->h_state, E->state, sizeof(float) * vf::kStateDim * E->n, cudaMemcpyDeviceToHost,
                            E->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(E->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && rc == SIM_OK) e = cudaGraphInstantiate(&E->exec, g, 0);
    E->graph = g;
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "environment capture");
    E->gen = gen;
    E->cmd_in_graph = cmd;
    return SIM_OK;
}

}  // namespace

int sim_env_create(sim_ctx* c, sim_env** out, int32_t n, const int32_t* soa, float* state, float* depth_host,
                   uint8_t* rgb_host, float* state_host) {
    Range nvtx_range("sim_env_create");
    if (!out) return fail(SIM_ERR_INVALID_ARG, "null output");
    *out = nullptr;
    int rc = check_render_args(c, n, soa, state);
    if (rc) return rc;
    if (n < 1 || (!depth_host && !rgb_host)) return fail(SIM_ERR_INVALID_ARG, "need agents and an image buffer");
    float* hd = depth_host ? (float*)direct_host_address(depth_host) : nullptr;
    uint8_t* hr = rgb_host ? (uint8_t*)direct_host_address(rgb_host) : nullptr;
    if ((depth_host && !hd) || (rgb_host && !hr) || (state_host && !direct_host_address(state_host)))
        return fail(SIM_ERR_INVALID_ARG, "the host buffers of a prepared step must be page-locked");
    DeviceGuard g(c->device);
    sim_env* E = new sim_env();
    E->ctx = c;
    E->n = n;
    E->soa = soa;
    E->state = state;
    E->h_depth = hd;
    E->h_rgb = hr;
    E->h_state = state_host;
    const size_t px = (size_t)n * c->cam.W * c->cam.H;
    E->rows_max = (size_t)c->cam.H;
    E->band_words = (size_t)n * (E->rows_max + (size_t)((c->cam.W + 3) / 4) * ((c->cam.H + 1) / 2));
    void* p = nullptr;
    if ((depth_host && (rc = ctx_alloc(c, sizeof(float) * px, &p)) == SIM_OK)) E->d_depth = (float*)p;
    if (!rc && rgb_host && (rc = ctx_alloc(c, 3 * px, &p)) == SIM_OK) E->d_rgb = (uint8_t*)p;
    if (!rc && (rc = ctx_alloc(c, sizeof(float) * 4 * (size_t)n, &p)) == SIM_OK) E->d_cmd = (float*)p;
    if (!rc && (rc = ctx_alloc(c, sizeof(unsigned) * E->band_words, &p)) == SIM_OK) E->band = (unsigned*)p;
    if (!rc && (rc = ctx_alloc(c, 2 * sizeof(unsigned), &p)) == SIM_OK) E->counters = (unsigned*)p;
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaStreamCreateWithFlags(&E->cap, cudaStreamNonBlocking);
    if (!rc && e == cudaSuccess) e = cudaMemsetAsync(E->counters, 0, 2 * sizeof(unsigned), E->cap);
    if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(E->cap);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "environment set-up");
    if (rc) {
        env_free(E);
        delete E;
        return rc;
    }
    *out = E;
    return SIM_OK;
}

int sim_env_run(sim_env* E, const float* cmd_host, void* stream) {
    Range nvtx_range("sim_env_run");
    if (!E || !cmd_host) return fail(SIM_ERR_INVALID_ARG, "null argument");
    sim_ctx* c = E->ctx;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const float* cmd = (const float*)direct_host_address(cmd_host);
    cudaError_t e = cudaSuccess;
    if (!cmd) {
        e = cudaMemcpyAsync(E->d_cmd, cmd_host, sizeof(float) * 4 * (size_t)E->n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "command upload");
        cmd = E->d_cmd;
    }
    if (!E->exec || E->gen != c->generation.load()) {
        // the previous graph and the env's buffers must be idle before a new capture
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "environment step");
        const int rc = env_capture(E, cmd);
        if (rc) return rc;
    } else if (cmd != E->cmd_in_graph) {
        cudaKernelNodeParams kp;
        e = cudaGraphKernelNodeGetParams(E->step_node, &kp);
        if (e == cudaSuccess) {
            void* args[5];
            for (int k = 0; k < 5; ++k) args[k] = kp.kernelParams[k];
            args[vf::kStepCmdArg] = &cmd;
            kp.kernelParams = args;
            e = cudaGraphExecKernelNodeSetParams(E->exec, E->step_node, &kp);
        }
        if (e != cudaSuccess) return cuda_fail(e, "command rebind");
        E->cmd_in_graph = cmd;
    }
    e = cudaGraphLaunch(E->exec, s);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "environment step");
}

int sim_env_destroy(sim_env* E) {
    if (!E) return SIM_OK;
    DeviceGuard g(E->ctx->device);
    cudaDeviceSynchronize();
    env_free(E);
    delete E;
    return SIM_OK;
}

int sim_loop_create(sim_ctx* c, sim_loop** out, int32_t n, int32_t T, const int32_t* soa, float* state,
                    const float* cmds, float* depth, uint8_t* rgb, int32_t n_frames, void* stream) {
    if (!out) return fail(SIM_ERR_INVALID_ARG, "null output");
    *out = nullptr;
    if (T < 1 || n_frames < 1 || !cmds) return fail(SIM_ERR_INVALID_ARG, "bad loop arguments");
    int rc = check_render_args(c, n, soa, state);
    if (rc) return rc;
    DeviceGuard g(c->device);
    sim_loop* L = new sim_loop();
    L->ctx = c;
    void* cnt;
    if ((rc = ctx_alloc(c, 2 * sizeof(unsigned), &cnt))) {
        delete L;
        return rc;
    }
    L->counters = (unsigned*)cnt;
    cudaStream_t s = (cudaStream_t)stream;
    L->sched_cap = (int)std::max<long long>(1, render_items(c, n, c->rcfg));
    if ((rc = sched_alloc(c, L->sched_cap, &L->sched_mem, s))) {
        ctx_free(c, L->counters, 2 * sizeof(unsigned));
        delete L;
        return rc;
    }
    if (c->swarm_on) {
        int rows;
        {
            std::lock_guard<std::mutex> lk(c->mu);
            rows = (int)c->scenes.size();
        }
        if ((rc = swarm_reserve(c, L->swarm, n, rows))) {
            sim_loop_destroy(L);
            return rc;
        }
    }
    cudaStream_t cap;
    cudaError_t e = cudaMemsetAsync(L->counters, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        ctx_free(c, L->counters, 2 * sizeof(unsigned));
        delete L;
        return cuda_fail(e, "loop set-up");
    }
    const size_t frame = (size_t)n * c->cam.W * c->cam.H;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    for (int t = 0; t < T && e == cudaSuccess && rc == SIM_OK; ++t) {
        e = launch_step(c->dyn, n, state, cmds + (size_t)t * 4 * n, nullptr, cap);
        if (e != cudaSuccess) break;
        const size_t slot = (size_t)(t % n_frames);
        rc = do_render(c, n, soa, state, depth ? depth + slot * frame : nullptr, rgb ? rgb + slot * frame * 3 : nullptr,
                       nullptr, false, c->rcfg, cap, L->counters, L->sched_mem, L->sched_cap, nullptr, nullptr,
                       nullptr, nullptr, nullptr, c->swarm_on ? SwarmUse::own : SwarmUse::none, &L->swarm);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && rc == SIM_OK) e = cudaGraphInstantiate(&L->exec, graph, 0);
    cudaStreamDestroy(cap);
    L->graph = graph;
    if (e != cudaSuccess || rc != SIM_OK) {
        sim_loop_destroy(L);
        return rc ? rc : cuda_fail(e, "loop capture");
    }
    *out = L;
    return SIM_OK;
}

int sim_loop_launch(sim_loop* L, void* stream) {
    Range nvtx_range("sim_loop_launch");
    if (!L || !L->exec) return fail(SIM_ERR_INVALID_ARG, "null loop");
    DeviceGuard g(L->ctx->device);
    cudaError_t e = cudaGraphLaunch(L->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "loop launch");
}

int sim_loop_destroy(sim_loop* L) {
    if (!L) return SIM_OK;
    DeviceGuard g(L->ctx->device);
    cudaDeviceSynchronize();
    if (L->exec) cudaGraphExecDestroy(L->exec);
    if (L->graph) cudaGraphDestroy(L->graph);
    ctx_free(L->ctx, L->counters, 2 * sizeof(unsigned));
    if (L->sched_mem) ctx_free(L->ctx, L->sched_mem, sched_bytes_for(L->sched_cap));
    swarm_free(L->ctx, L->swarm);
    delete L;
    return SIM_OK;
}

int sim_get_render_config(const sim_ctx* c, sim_render_config* cfg) {
    if (!c || !cfg) return fail(SIM_ERR_INVALID_ARG, "null argument");
    *cfg = c->rcfg;
    return SIM_OK;
}

int sim_set_render_config(sim_ctx* c, const sim_render_config* cfg) {
    if (!c || !cfg) return fail(SIM_ERR_INVALID_ARG, "null argument");
    if (!render_config_valid(*cfg)) return fail(SIM_ERR_INVALID_ARG, "unsupported render configuration");
    c->rcfg = *cfg;
    ++c->generation;
    return SIM_OK;
}

int sim_render_config_list(sim_render_config* out, int32_t max) { return render_config_list(out, max); }

int sim_autotune_render(sim_ctx* c, int32_t n, const int32_t* soa, const float* state, float* depth, uint8_t* rgb,
                        int32_t iters, sim_render_config* best, float* times_ms, int32_t max_times, void* stream) {
    Range nvtx_range("sim_autotune_render");
    int rc = check_render_args(c, n, soa, state);
    if (rc) return rc;
    ++c->generation;
    if (iters < 1 || !best) return fail(SIM_ERR_INVALID_ARG, "bad autotune arguments");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    sim_render_config cfgs[128];
    const int nc = render_config_list(cfgs, 128);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    int best_i = -1;
    const int need_depth = max_scene_depth(c);
    // every configuration is timed as sim_render runs it: with scheduling hints,
    // from its own fresh hint buffer (two warm-up launches build the hints)
    long long max_items = 0;
    for (int i = 0; i < nc; ++i) max_items = std::max(max_items, render_items(c, n, cfgs[i]));
    const int scap = (int)std::max<long long>(1, max_items);
    void* smem = nullptr;
    if ((rc = sched_alloc(c, scap, &smem, s))) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
    }
    for (int i = 0; i < nc; ++i) {
        sim_render_config cf = cfgs[i];
        if (!stack_fits(cf, need_depth)) continue;
        cudaError_t me = cudaMemsetAsync(smem, 0, sched_bytes_for(scap), s);
        if (me != cudaSuccess) {
            rc = cuda_fail(me, "autotune reset");
            break;
        }
        for (int w = 0; w < 2 && !rc; ++w)
            rc = do_render(c, n, soa, state, depth, rgb, nullptr, false, cf, s, nullptr, smem, scap);  // warm-up
        if (rc) break;
        cudaEventRecord(e0, s);
        for (int k = 0; k < iters && !rc; ++k)
            rc = do_render(c, n, soa, state, depth, rgb, nullptr, false, cf, s, nullptr, smem, scap);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (rc) break;
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune timing");
            break;
        }
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= iters;
        if (times_ms && i < max_times) times_ms[i] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best_i = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    ctx_free(c, smem, sched_bytes_for(scap));
    if (rc) return rc;
    if (best_i < 0) return fail(SIM_ERR_INVALID_ARG, "no configuration fits the scene depth");
    c->rcfg = cfgs[best_i];
    *best = cfgs[best_i];
    return SIM_OK;
}

int sim_nearest_obstacle(sim_ctx* c, int32_t n, const int32_t* soa, const float* state, float max_dist, float* dist,
                         float* point, int32_t* tri, void* stream) {
    Range nvtx_range("sim_nearest_obstacle");
    if (!c || n < 0 || (n > 0 && (!soa || !state || !dist)) || !(max_dist > 0.0f))
        return fail(SIM_ERR_INVALID_ARG, "bad sim_nearest_obstacle arguments");
    if (n == 0) return SIM_OK;
    DeviceGuard g(c->device);
    NearestArgs a;
    a.n = n;
    a.scene_of_agent = soa;
    a.state = state;
    a.max_dist = max_dist;
    a.dist = dist;
    a.point = point;
    a.tri = tri;
    a.err = c->d_err;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        a.table = c->d_table;
        a.n_scenes = (int)c->scenes.size();
    }
    cudaError_t e = launch_nearest(a, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "nearest-obstacle launch");
}

int sim_get_status(sim_ctx* c, void* stream, int32_t timeout_ms) {
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(s);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_fail(q, "stream");
        if (timeout_ms >= 0 &&
            std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
            return fail(SIM_ERR_TIMEOUT, "stream still busy after timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "error word");
    if (h == kDevErrTraversal) return fail(SIM_ERR_TRAVERSAL, "device: traversal stack overflow or iteration cap");
    if (h == kDevErrNotFound) return fail(SIM_ERR_NOT_FOUND, "device: agent refers to an unknown scene");
    if (h != 0) return fail(SIM_ERR_CUDA, "device error word " + std::to_string(h));
    return SIM_OK;
}

int sim_mem_usage(const sim_ctx* c, size_t* used, size_t* budget) {
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    if (used) *used = c->used;
    if (budget) *budget = c->budget;
    return SIM_OK;
}

}  // extern "C"

namespace {
__global__ void probe_read_kernel(const float4* __restrict__ buf, size_t n4, int iters, float* sink) {
    float acc = 0.0f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int it = 0; it < iters; ++it)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += v.x + v.y + v.z + v.w;
        }
    if (acc == 1234.5678f) *sink = acc;
}
}  // namespace

extern "C" int sim_probe_read_bandwidth(sim_ctx* c, size_t bytes, int32_t iters, double* gbs, void* stream) {
    if (!c || !gbs || bytes < 4096 || iters < 1) return fail(SIM_ERR_INVALID_ARG, "bad probe arguments");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    void* buf;
    int rc = ctx_alloc(c, bytes + 256, &buf);
    if (rc) return rc;
    const size_t n4 = bytes / 16;
    cudaMemsetAsync(buf, 0, bytes + 256, s);
    const int grid = c->num_sms * 8;
    probe_read_kernel<<<grid, 512, 0, s>>>((const float4*)buf, n4, 1, (float*)((char*)buf + bytes));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    probe_read_kernel<<<grid, 512, 0, s>>>((const float4*)buf, n4, iters, (float*)((char*)buf + bytes));
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx_free(c, buf, bytes + 256);
    if (e != cudaSuccess) return cuda_fail(e, "probe");
    *gbs = (double)n4 * 16.0 * iters / (ms * 1e-3) / 1e9;
    return SIM_OK;
}

namespace vf {

void set_last_error(const char* msg) { g_err = msg; }

int ctx_device(const sim_ctx* c) { return c ? c->device : -1; }

// Render n agents of one scene with caller-supplied scratch: soa_dev holds the
// scene id of every agent and counters_dev the two work counters, already
// zero.  Same checks and kernel as sim_render.
int render_scene_check(sim_ctx* c, int n, int scene_id, const int32_t* soa_dev, const float* state) {
    if (!c) return fail(SIM_ERR_INVALID_ARG, "null context");
    if (!ctx_scene_live(c, scene_id)) return fail(SIM_ERR_NOT_FOUND, "no such scene");
    return check_render_args(c, n, soa_dev, state);
}

int render_scene_with_scratch(sim_ctx* c, int n, int scene_id, const int32_t* soa_dev, unsigned* counters_dev,
                              const float* state, float* depth, uint8_t* rgb, int32_t* hit, cudaStream_t s) {
    int rc = render_scene_check(c, n, scene_id, soa_dev, state);
    if (rc) return rc;
    if (n == 0) return SIM_OK;
    DeviceGuard g(c->device);
    RenderArgs a = render_args(c, n, soa_dev, state, depth, rgb, hit);
    a.counter = counters_dev;
    a.done_ctas = counters_dev + 1;
    int ctas = c->rcfg.ctas_per_sm > 0 ? c->rcfg.ctas_per_sm * c->num_sms : 0;
    cudaError_t e = launch_render(a, c->rcfg, ctas, false, s);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "ray-cast launch");
}

}  // namespace vf

namespace vf {

int ctx_alloc_ext(sim_ctx* c, size_t bytes, void** out) { return ctx_alloc(c, bytes, out); }
void ctx_free_ext(sim_ctx* c, void* p, size_t bytes) { ctx_free(c, p, bytes); }

// Stream-ordered allocation from `pool` on stream s, counted against the
// context's budget like ctx_alloc.  Unlike cudaFree, returning a block does
// not synchronise the device: the pool reuses it once s has passed the free.
int ctx_alloc_pool(sim_ctx* c, size_t bytes, void** out, cudaMemPool_t pool, cudaStream_t s) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    if (c->budget && c->used + bytes > c->budget)
        return fail(SIM_ERR_BUDGET, "memory budget exceeded: need " + std::to_string(bytes) + " B, used " +
                                        std::to_string(c->used) + " of " + std::to_string(c->budget));
    cudaError_t e = cudaMallocFromPoolAsync(out, bytes, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return cuda_fail(e, "cudaMallocFromPoolAsync");
    }
    c->used += bytes;
    return SIM_OK;
}
void ctx_free_pool(sim_ctx* c, void* p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    cudaFreeAsync(p, s);
    if (bytes == 0) bytes = 16;
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    c->used -= bytes;
}
void ctx_image_size(const sim_ctx* c, int* W, int* H) {
    *W = c->cam.W;
    *H = c->cam.H;
}
bool ctx_scene_live(sim_ctx* c, int scene_id) {
    std::lock_guard<std::mutex> lk(c->mu);
    return scene_id >= 0 && scene_id < (int)c->scenes.size() && c->scenes[scene_id].live;
}
int ctx_step(sim_ctx* c, int n, float* state, const float* cmd, cudaStream_t s) {
    cudaError_t e = launch_step(c->dyn, n, state, cmd, nullptr, s);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e, "step launch");
}
int ctx_render_own(sim_ctx* c, int n, const int32_t* soa, const float* state, float* depth, uint8_t* rgb,
                   unsigned* counters, cudaStream_t s) {
    int rc = check_render_args(c, n, soa, state);
    if (rc) return rc;
    // requests are independent: the server always renders in the parallel-agents mode
    return do_render(c, n, soa, state, depth, rgb, nullptr, false, c->rcfg, s, counters, nullptr, 0, nullptr, nullptr,
                     nullptr, nullptr, nullptr, SwarmUse::none);
}
int ctx_fail(int code, const char* msg) { return fail(code, msg); }

}  // namespace vf

// sim_render_scene_static: render every agent of one scene without allocating
// device memory.
//
// sim_render_scene needs an agent -> scene id array on the device and
// allocates it on every call.  Some callers cannot allocate device memory once
// they are running: a control loop that must not touch the allocator after
// set-up, or a process whose device memory is handed in full to another
// framework's memory pool.  This entry point keeps its scratch -- the id array
// and the ray-cast kernel's two work counters -- in one file-scope device array
// that exists on every GPU that loads the library until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "launch.h"
#include "visfly_b300.h"

constexpr size_t kCounterBytes = 256;
constexpr size_t kScratchBytes = kCounterBytes + sizeof(int32_t) * SIM_RENDER_STATIC_MAX_AGENTS;

// [0, 8): work-item counter and finished-CTA counter; [256, ...): scene ids.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};  // device address of g_scratch, per device

// Clear the counters (they must start at zero) and write the scene id of the
// first n agents; the array keeps whatever a previous call left beyond n.
__global__ void fill_static_scratch(int n, int scene_id) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        unsigned* counters = reinterpret_cast<unsigned*>(g_scratch);
        counters[0] = 0u;
        counters[1] = 0u;
    }
    if (i < n) reinterpret_cast<int32_t*>(g_scratch + kCounterBytes)[i] = scene_id;
}

// In host code g_scratch names a host-side stand-in, not device memory: the
// kernel must be given the address cudaGetSymbolAddress reports for the
// current device.  Looked up once per device, on the first call there.
int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) {
        vf::set_last_error("device index out of range for the static scratch table");
        return SIM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            vf::set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
            return SIM_ERR_CUDA;
        }
        g_scratch_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[device];
    return SIM_OK;
}

}  // namespace

extern "C" int sim_render_scene_static(sim_ctx* ctx, int32_t n_agents, int32_t scene_id, const float* state,
                                       float* depth, uint8_t* rgb, int32_t* hit_id, void* stream) {
    if (!ctx) {
        vf::set_last_error("null context");
        return SIM_ERR_INVALID_ARG;
    }
    if (n_agents < 0 || n_agents > SIM_RENDER_STATIC_MAX_AGENTS) {
        vf::set_last_error("sim_render_scene_static: n_agents must be in [0, SIM_RENDER_STATIC_MAX_AGENTS]");
        return SIM_ERR_INVALID_ARG;
    }
    if (!vf::ctx_scene_live(ctx, scene_id)) {
        vf::set_last_error("no such scene");
        return SIM_ERR_NOT_FOUND;
    }
    if (n_agents == 0) return SIM_OK;
    const int device = vf::ctx_device(ctx);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device) {
        const cudaError_t e = cudaSetDevice(device);
        if (e != cudaSuccess) {
            vf::set_last_error(cudaGetErrorString(e));
            return SIM_ERR_CUDA;
        }
    }
    unsigned char* base = nullptr;
    int rc = scratch_address(device, &base);
    const int32_t* ids = rc == SIM_OK ? reinterpret_cast<const int32_t*>(base + kCounterBytes) : nullptr;
    unsigned* counters = reinterpret_cast<unsigned*>(base);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // every check the render makes runs before the scratch is touched, so a
    // rejected call leaves the shared array as it was
    if (rc == SIM_OK) rc = vf::render_scene_check(ctx, n_agents, scene_id, ids, state);
    if (rc == SIM_OK) {
        fill_static_scratch<<<(n_agents + 255) / 256, 256, 0, s>>>(n_agents, scene_id);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            vf::set_last_error(cudaGetErrorString(e));
            rc = SIM_ERR_CUDA;
        } else {
            rc = vf::render_scene_with_scratch(ctx, n_agents, scene_id, ids, counters, state, depth, rgb, hit_id, s);
        }
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}

// rtsdf_build_bvh_noalloc: the BVH build with its scratch memory in a fixed
// device array instead of a caller-provided workspace.
//
// Who needs it: hosts that cannot call cudaMalloc on the library's behalf, or
// cannot give it a workspace, for example a renderer or game engine that owns
// all GPU memory through its own budgeted pool and forbids allocation inside
// the frame loop (cudaMalloc can synchronise the device and stall the frame),
// or a plugin whose host process hands it only the input and output buffers.
// The caller still provides the mesh and the output BVH buffer.
//
// The scratch is one file-scope __device__ array.  Every GPU that loads this
// library holds it (RTSDF_NOALLOC_SCRATCH_BYTES) until the process exits.
#include <mutex>

#include "rtsdf_device.cuh"
#include "rtsdf_launch.cuh"

namespace {

static __device__ __align__(256) unsigned char g_bvh_scratch[RTSDF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  Host code only
// sees a host-side stand-in under the array's name, so the address must be
// queried once per device, with that device current.
rtsdf_status scratch_on_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RTSDF_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bvh_scratch) != cudaSuccess || p == nullptr) return RTSDF_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RTSDF_OK;
}

}  // namespace

extern "C" rtsdf_status rtsdf_build_bvh_noalloc(const float* verts, int32_t V, const int32_t* tris, int32_t T,
                                                const rtsdf_grid* g, void* bvh, size_t bvh_bytes,
                                                rtsdf_counters* counters, rtsdf_stream stream) {
    if (T > RTSDF_NOALLOC_MAX_TRIS) return RTSDF_ENOMEM;  // the fixed scratch is sized for this many triangles
    if (rtsdf_bvh_workspace(T) > sizeof(g_bvh_scratch)) return RTSDF_ENOMEM;
    void* scratch = nullptr;
    rtsdf_status st = scratch_on_current_device(&scratch);
    if (st != RTSDF_OK) return st;
    // Same validation and kernels as rtsdf_build_bvh; only the workspace differs.
    // The build clears what it needs zeroed (header, visit counters) on every call.
    return rtsdf_build_bvh(verts, V, tris, T, g, bvh, bvh_bytes, scratch, sizeof(g_bvh_scratch), counters, stream);
}

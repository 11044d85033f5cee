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
struct ScratchAddr {
    void* ptr = nullptr;
    unsigned long long ctx = 0;  // id of the context the address belongs to
};
ScratchAddr g_scratch[kMaxDevices];

// Id of the calling thread's current CUDA context (0 when there is none or the
// driver cannot tell), through the driver's cuCtxGetCurrent and cuCtxGetId, found
// at run time so that the library needs no link against the driver.
unsigned long long current_context_id() {
    using GetCurrent = int (*)(void**);
    using GetId = int (*)(void*, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(a);
            get_id = reinterpret_cast<GetId>(b);
        }
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || ctx == nullptr || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array in the current device's context.  Host code
// only sees a host-side stand-in under the array's name, so the address is looked
// up with the device current: once per device, and again whenever that device's
// context has changed since (a cudaDeviceReset makes a new context, into which the
// module, and so the array, is loaded anew).
rtsdf_status scratch_on_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RTSDF_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    ScratchAddr& c = g_scratch[dev];
    if (c.ptr == nullptr || ctx == 0 || c.ctx != ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bvh_scratch) != cudaSuccess || p == nullptr) return RTSDF_ECUDA;
        c.ptr = p;
        c.ctx = current_context_id();  // the lookup made the context current if there was none
    }
    *out = c.ptr;
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

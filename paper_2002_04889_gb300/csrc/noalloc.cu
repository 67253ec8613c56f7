// vg_step_noalloc: one time step that allocates no memory.
//
// Some callers cannot call cudaMalloc when they need to advance the solver:
// code that runs while a memory pool is fully reserved, a caller inside a
// real-time loop that must not touch the allocator, or a host framework that
// forbids device allocations after its set-up phase.  For them this file keeps
// the step's scratch memory -- the stage-1 residual R0 [3][nc] and the step's
// device scalars -- in one file-scope __device__ array of fixed size, and runs
// the library's ordinary stage kernels on it.  The caller passes the input and
// output states; nothing here calls cudaMalloc, cudaFree or any allocating
// library routine.
//
// Limits and caveats (also in include/volna_gb.h):
//  * at most VG_NOALLOC_MAX_CELLS cells (larger meshes: VG_EINVAL);
//  * the array (about 6 MiB) is committed on a device when a context first
//    uploads a mesh there (vg_mesh_upload calls noalloc_prepare: it looks up the
//    array's address and loads this file's kernels, without launching one), and
//    is held until the process exits;
//  * all calls share the array, which keeps the last call's contents; each call
//    clears what must start fresh (the step scalars) before its kernels run, and
//    calls that overlap on the GPU (other streams, other threads) race on it;
//  * the device address of the array is looked up once per device (with that
//    device current) at that set-up and cached, so a step loads nothing.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <mutex>

#include "../../include/volna_gb.h"
#include "vg_internal.h"

namespace vg {

namespace {

constexpr size_t kScalarBytes = 256;
constexpr size_t kScratchBytes = kScalarBytes + sizeof(double) * 3 * (size_t)VG_NOALLOC_MAX_CELLS;

// The scratch: step scalars in the first 256 bytes, then R0 (sized for FP64).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Clear the step scalars at the start of every call: time t, empty CFL minimum
// (+inf in the context's precision), no flags, no records.
__global__ void noalloc_init_kernel(DevScalars *sc, double t, int precision)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc->t = t;
        sc->dt = 0.0;
        if (precision == 64) {
            sc->dtmin_bits = (unsigned long long)__double_as_longlong(CUDART_INF);
        } else {
            sc->dtmin_bits = (unsigned long long)__float_as_uint(CUDART_INF_F);
        }
        sc->steps = 0;
        sc->n_rec = 0;
        sc->neg_count = 0;
        sc->flags = 0u;
        sc->pad = 0;
    }
}

}  // namespace

// Device address of the scratch array on `device` (set-up on first use, with
// that device current).  Returns a cudaError_t as int.
int noalloc_scratch(int device, void **addr, size_t *bytes)
{
    if (device < 0 || device >= kMaxDevices) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaError_t e = cudaSetDevice(device);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&g_addr[device], g_noalloc_scratch);
        if (prev >= 0) cudaSetDevice(prev);
        if (e != cudaSuccess) {
            g_addr[device] = nullptr;
            return (int)e;
        }
    }
    *addr = g_addr[device];
    *bytes = kScratchBytes;
    return 0;
}

// Set-up at mesh upload: the array's address on `device` (committing the array
// under lazy module loading) and this file's kernel, loaded without a launch.
int noalloc_prepare(int device)
{
    void *addr = nullptr;
    size_t bytes = 0;
    int e = noalloc_scratch(device, &addr, &bytes);
    if (e) return e;
    cudaFuncAttributes fa;
    return (int)cudaFuncGetAttributes(&fa, (const void *)noalloc_init_kernel);
}

int noalloc_launch_init(void *scalars, double t, int precision, void *stream)
{
    noalloc_init_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<DevScalars *>(scalars), t,
                                                                         precision);
    return (int)cudaGetLastError();
}

}  // namespace vg

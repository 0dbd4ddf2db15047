// vof_reconstruct_static: the reconstruction of vof_reconstruct run over a
// compacted list of interface cells, with that list kept in a file-scope
// device array instead of memory the caller or the context allocates.
//
// It exists for callers that cannot allocate device memory at the point where
// they reconstruct: for example code running inside a host framework that owns
// every device allocation, or a real-time loop that forbids cudaMalloc after
// start-up.  The context itself must still have been created (vof_create
// allocates) by someone who could.
#include <cuda_runtime.h>

#include <mutex>

#include "vof_internal.h"

namespace {

// maximum number of cells this entry point handles: the list needs one int
// per cell in the worst case (16 MiB), plus a counter in the first 256 bytes
constexpr int STATIC_MAX_CELLS = VOF_STATIC_MAX_CELLS;
constexpr int STATIC_HEAD = 64;  // ints before the list: [0] = list length

// shared by every call on a device; held by every GPU that loads the library
static __device__ __align__(256) int g_static_scratch[STATIC_HEAD + STATIC_MAX_CELLS];

constexpr int MAX_DEVICES = 64;
static int *g_static_ptr[MAX_DEVICES];
static std::mutex g_static_mutex;

// default outputs for every cell, and the interface cells appended to the list
__global__ void k_static_fill(int nc, double eps, const double *__restrict__ alpha, double *n, double *d,
                              uint8_t *flags, int *scratch)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    bool isint = false;
    if (c < nc) {
        double a = alpha[c];
        flags[c] = a >= 1.0 - eps ? VOF_FULL : 0;
        n[c] = 0.0; n[nc + c] = 0.0; n[2 * nc + c] = 0.0;
        d[c] = 0.0;
        isint = a > eps && a < 1.0 - eps;
    }
    unsigned mask = __ballot_sync(0xffffffffu, isint);
    if (!mask) return;
    int lane = threadIdx.x & 31, leader = __ffs(mask) - 1, base = 0;
    if (lane == leader) base = atomicAdd(scratch, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (isint) scratch[STATIC_HEAD + base + __popc(mask & ((1u << lane) - 1u))] = c;
}

// device address of the static array on `device` (looked up once per device,
// with that device current)
int static_scratch(int device, int **out)
{
    if (device < 0 || device >= MAX_DEVICES) return VOF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return VOF_ERR_CUDA;
        g_static_ptr[device] = (int *)p;
    }
    *out = g_static_ptr[device];
    return VOF_OK;
}

}  // namespace

extern "C" int vof_reconstruct_static(vof_ctx *c, const double *alpha, double *n, double *d, uint8_t *flags,
                                      void *stream)
{
    if (!c || !alpha || !n || !d || !flags) return VOF_ERR_INVALID_ARG;
    if (c->nc > STATIC_MAX_CELLS) return VOF_ERR_INVALID_ARG;  // beyond the static list
    if (c->nc == 0) return VOF_OK;                               // nothing to reconstruct
    if (cudaSetDevice(c->device) != cudaSuccess) return VOF_ERR_CUDA;
    int *scratch = nullptr;
    int r = static_scratch(c->device, &scratch);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;
    // the list length starts at zero on every call (the array keeps the last
    // call's contents otherwise)
    if (cudaMemsetAsync(scratch, 0, sizeof(int), s) != cudaSuccess) return VOF_ERR_CUDA;
    // launched through cudaLaunchKernelEx, whose return code is this launch's
    // own (an error left by earlier, unrelated work is not blamed on it)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((c->nc + 255) / 256);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    if (cudaLaunchKernelEx(&cfg, k_static_fill, c->nc, c->eps, alpha, n, d, flags, scratch) != cudaSuccess)
        return VOF_ERR_CUDA;
    return launch_reconstruct(c, alpha, n, d, flags, nullptr, scratch + STATIC_HEAD, scratch, s);
}

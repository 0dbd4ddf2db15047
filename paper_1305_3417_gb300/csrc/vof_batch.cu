// Batched form: many independent cases advanced as one mesh.
//
// The cases' meshes are joined into one (disjoint union: each case's cells,
// points and faces after the previous case's, internal faces of every case
// first), so a step over the batch is a step over that mesh: the band lists,
// the per-warp load balancing of the narrow-band kernels and every launch cover
// all cases at once.  The method uses a velocity field only through F dt and
// U dt, so each case's own time step is folded into its F and U and the batch
// steps with dt = 1.  A step is captured once into a CUDA graph (all its
// kernels) and replayed as one graph launch; the phase-flux launch shape is
// chosen by timing the candidates on the batch itself.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "vof_device.cuh"
#include "vof_internal.h"

struct vof_batch {
    vof_ctx *ctx;
    int ncases;
    int *case_ptr;            // device [ncases + 1] cell offsets
    cudaStream_t gs;          // capture / replay stream
    cudaEvent_t ev_in, ev_out;
    cudaGraphExec_t exec;
    const void *key[5];       // arrays baked into the graph
    int key_cfg;              // launch configuration baked into the graph
};

namespace {

// per case (one block each): sum of V_c alpha_c over the case's cells, in a
// fixed order (thread-strided partial sums, then a fixed tree)
__global__ void k_case_mass(const double *__restrict__ alpha, const double *__restrict__ vc, const int *case_ptr,
                            double *out)
{
    const int cs = blockIdx.x, c0 = case_ptr[cs], c1 = case_ptr[cs + 1];
    double v = 0.0;
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) v += vc[c] * alpha[c];
    v = vofd::warp_sum(v);
    __shared__ double sh[4];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) out[cs] = (sh[0] + sh[1]) + (sh[2] + sh[3]);
}

int cfg_code(const vof_ctx *c) { return c->pf_stack * 256 + c->pf_warps * 16 + c->pf_mult; }

void drop_graph(vof_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// one step of the batch (dt = 1) plus the per-case masses, on stream s
int enqueue_step(vof_batch *b, double *alpha, const double *U, const double *F, double *stats, double *case_mass,
                 cudaStream_t s)
{
    int r = launch_advect(b->ctx, alpha, U, F, 1.0, stats, s);
    if (r) return r;
    if (case_mass) {
        k_case_mass<<<b->ncases, 128, 0, s>>>(alpha, b->ctx->m.vc, b->case_ptr, case_mass);
        if (cudaGetLastError() != cudaSuccess) return VOF_ERR_CUDA;
    }
    return VOF_OK;
}

}  // namespace

extern "C" {

int vof_batch_create(const vof_mesh *mesh, const int32_t *case_cell_ptr, int ncases, const vof_options *opt,
                     vof_batch **out)
{
    if (!mesh || !case_cell_ptr || ncases < 1 || !out) return VOF_ERR_INVALID_ARG;
    *out = nullptr;
    if (mesh->point_master) return VOF_ERR_INVALID_ARG;  // one set of periods cannot serve cases of any size
    if (case_cell_ptr[0] != 0 || case_cell_ptr[ncases] != mesh->n_cells) return VOF_ERR_INVALID_ARG;
    for (int i = 0; i < ncases; ++i)
        if (case_cell_ptr[i + 1] <= case_cell_ptr[i]) return VOF_ERR_INVALID_ARG;
    vof_ctx *ctx = nullptr;
    int r = vof_create(mesh, opt, &ctx);
    if (r) return r;
    // the global bounding step works per case
    r = set_bound_regions(ctx, case_cell_ptr, ncases);
    if (r) { vof_destroy(ctx); return r; }
    vof_batch *b = new (std::nothrow) vof_batch();
    if (!b) { vof_destroy(ctx); return VOF_ERR_CUDA; }
    std::memset(b, 0, sizeof(*b));
    b->ctx = ctx;
    b->ncases = ncases;
    bool ok = cudaMalloc(&b->case_ptr, sizeof(int) * (ncases + 1)) == cudaSuccess &&
              cudaMemcpy(b->case_ptr, case_cell_ptr, sizeof(int) * (ncases + 1), cudaMemcpyHostToDevice) ==
                  cudaSuccess &&
              cudaStreamCreateWithFlags(&b->gs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { vof_batch_destroy(b); return VOF_ERR_CUDA; }
    *out = b;
    return VOF_OK;
}

void vof_batch_destroy(vof_batch *b)
{
    if (!b) return;
    if (b->ctx) cudaSetDevice(b->ctx->device);
    drop_graph(b);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->gs) cudaStreamDestroy(b->gs);
    if (b->case_ptr) cudaFree(b->case_ptr);
    if (b->ctx) vof_destroy(b->ctx);
    delete b;
}

vof_ctx *vof_batch_context(vof_batch *b) { return b ? b->ctx : nullptr; }

int vof_batch_advect(vof_batch *b, double *alpha, const double *U_dt, const double *F_dt, double *stats,
                     double *case_mass, void *stream)
{
    if (!b || !alpha || !U_dt || !F_dt) return VOF_ERR_INVALID_ARG;
    vof_ctx *c = b->ctx;
    if (cudaSetDevice(c->device) != cudaSuccess) return VOF_ERR_CUDA;
    if (!stats) stats = c->stats_dev;
    const void *key[5] = {alpha, U_dt, F_dt, stats, case_mass};
    if (b->exec && (std::memcmp(key, b->key, sizeof(key)) != 0 || b->key_cfg != cfg_code(c))) drop_graph(b);
    if (!b->exec) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return VOF_ERR_CUDA;
        int r = enqueue_step(b, alpha, U_dt, F_dt, stats, case_mass, b->gs);
        cudaError_t e = cudaStreamEndCapture(b->gs, &g);
        if (r || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return r ? r : VOF_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { b->exec = nullptr; return VOF_ERR_CUDA; }
        std::memcpy(b->key, key, sizeof(key));
        b->key_cfg = cfg_code(c);
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaEventRecord(b->ev_in, s) != cudaSuccess || cudaStreamWaitEvent(b->gs, b->ev_in, 0) != cudaSuccess ||
        cudaGraphLaunch(b->exec, b->gs) != cudaSuccess || cudaEventRecord(b->ev_out, b->gs) != cudaSuccess ||
        cudaStreamWaitEvent(s, b->ev_out, 0) != cudaSuccess)
        return VOF_ERR_CUDA;
    return VOF_OK;
}

// Times one step (vof_advect's launch sequence, from the state alpha copied
// into the context's staging buffer: no allocation) for every launch
// configuration of the mixed phase flux -- clip-piece stack depth 92 or 56,
// 1, 2 or 3 warps (faces) per block, grid multipliers 1, 2, 4 over the
// resident blocks -- and keeps the fastest; an FP64 context keeps its launch
static int tune_launch(vof_ctx *c, const double *alpha, const double *U, const double *F, double dt, cudaStream_t s,
                       int *best_out, float *ms_out)
{
    int best = -1;
    float tbest = 0.0f;
    if (c->precision == VOF_MIXED) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return VOF_ERR_CUDA;
        if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return VOF_ERR_CUDA; }
        int err = VOF_OK;
        // every candidate steps from the same state: one untimed step, the
        // state restored, one timed step
        for (int st = 0; st <= 1 && !err; ++st)
            for (int w = 1; w <= 3 && !err; ++w)
                for (int mult = 1; mult <= 4 && !err; mult *= 2) {
                    c->pf_stack = st;
                    c->pf_warps = w;
                    c->pf_mult = mult;
                    float ms = 0.0f;
                    for (int rep = 0; rep < 2 && !err; ++rep) {
                        if (cudaMemcpyAsync(c->h_alpha, alpha, sizeof(double) * c->nc, cudaMemcpyDeviceToDevice, s) !=
                            cudaSuccess) { err = VOF_ERR_CUDA; break; }
                        if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) { err = VOF_ERR_CUDA; break; }
                        err = launch_advect(c, c->h_alpha, U, F, dt, c->stats_dev, s);
                        if (err) break;
                        if (rep == 1 &&
                            (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                            err = VOF_ERR_CUDA;
                    }
                    if (!err && (best < 0 || ms < tbest)) {
                        best = st * 256 + w * 16 + mult;
                        tbest = ms;
                    }
                }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (err) return err;
        c->pf_stack = best / 256;
        c->pf_warps = (best / 16) % 16;
        c->pf_mult = best % 16;
    }
    *best_out = best < 0 ? 0 : best;
    *ms_out = tbest;
    return VOF_OK;
}

int vof_batch_tune(vof_batch *b, const double *alpha, const double *U_dt, const double *F_dt, int *config,
                   float *best_ms, void *stream)
{
    if (!b || !alpha || !U_dt || !F_dt) return VOF_ERR_INVALID_ARG;
    vof_ctx *c = b->ctx;
    if (cudaSetDevice(c->device) != cudaSuccess) return VOF_ERR_CUDA;
    int best = 0;
    float tbest = 0.0f;
    int r = tune_launch(c, alpha, U_dt, F_dt, 1.0, (cudaStream_t)stream, &best, &tbest);
    if (r) return r;
    drop_graph(b);
    if (config) *config = best;
    if (best_ms) *best_ms = tbest;
    return VOF_OK;
}

int vof_tune(vof_ctx *c, const double *alpha, const double *Uc, const double *F, double dt, int *config,
             float *best_ms, void *stream)
{
    if (!c || !alpha || !Uc || !F || !(dt > 0.0)) return VOF_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return VOF_ERR_CUDA;
    int best = 0;
    float tbest = 0.0f;
    int r = tune_launch(c, alpha, Uc, F, dt, (cudaStream_t)stream, &best, &tbest);
    if (r) return r;
    if (config) *config = best;
    if (best_ms) *best_ms = tbest;
    return VOF_OK;
}

}  // extern "C"

// The initial-guess network: 33 features of an interface cell -> 64 -> 64 ->
// 4 (a unit normal and the plane offset s = (d - d_min) / (d_max - d_min)),
// ReLU hidden layers, BF16 weights and activations, FP32 accumulation on the
// tensor cores (mma.sync m16n8k16; the layers are 48-64 wide, far below the
// tile sizes where tcgen05 and TMEM would pay), trained by Adam on the mean
// squared error with the forward and backward kernels here.  The paper has no
// learned part: the network only moves the start of the plane positioning,
// whose root and stop are unchanged.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "vof_device.cuh"
#include "vof_internal.h"

namespace {

constexpr int IN = VOF_MLP_IN, K0 = 48, HID = VOF_MLP_HID, OUT = VOF_MLP_OUT, OUTP = 16;
// flat FP32 parameter layout: W1 [IN x HID], b1, W2 [HID x HID], b2, W3 [HID x OUT], b3
constexpr int OW1 = 0, OB1 = OW1 + IN * HID, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + HID * OUT, NPARAM = OB3 + OUT;
static_assert(NPARAM == VOF_MLP_NPARAM, "parameter count");
constexpr int CHUNK = 512;  // samples per weight-gradient partial

using bf = unsigned short;

__device__ __forceinline__ bf to_bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pk(bf lo, bf hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ void mma16816(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------- features
// Per interface cell: the volume fractions of its 3x3x3 lattice neighbourhood
// (the cells sharing a point with it, placed by the sign of their centre
// offset beyond half the cell size; missing slots take the cell's own value)
// and six scale-free shape numbers: box extents / V^(1/3) (3), V / box volume,
// faces / 24, points / 8.
__device__ void mlp_features_one(const DevMesh &m, const double *__restrict__ alpha, int c, float *f)
{
    const double ac = alpha[c];
    for (int k = 0; k < 27; ++k) f[k] = (float)ac;
    const double V = m.vc[c], h = cbrt(V);
    const vofd::V3 cc = vofd::ld3(m.cc, m.nc, c);
    for (int j = m.cpptr[c]; j < m.cpptr[c + 1]; ++j) {
        const int p = m.cpts[j];
        for (int q = m.pptr[p]; q < m.pptr[p + 1]; ++q) {
            const int nb = m.pcell[q];
            vofd::V3 d = vofd::ld3(m.cc, m.nc, nb) - cc;
            if (m.pcode) d = d + vofd::tshift(m, m.pcode[q]);  // periodic: the cell next to c
            const int sx = (d.x > 0.5 * h) - (d.x < -0.5 * h), sy = (d.y > 0.5 * h) - (d.y < -0.5 * h),
                      sz = (d.z > 0.5 * h) - (d.z < -0.5 * h);
            f[(sx + 1) + 3 * (sy + 1) + 9 * (sz + 1)] = (float)alpha[nb];
        }
    }
    const double *bx = m.cbox + 6 * (size_t)c;
    const double ex = bx[3] - bx[0], ey = bx[4] - bx[1], ez = bx[5] - bx[2];
    f[27] = (float)(ex / h);
    f[28] = (float)(ey / h);
    f[29] = (float)(ez / h);
    f[30] = (float)(V / (ex * ey * ez));
    f[31] = (float)((m.cptr[c + 1] - m.cptr[c]) / 24.0);
    f[32] = (float)((m.cpptr[c + 1] - m.cpptr[c]) / 8.0);
}

__global__ void k_mlp_features(DevMesh m, const double *__restrict__ alpha, const int *cells, int ncells,
                               const int *ndev, float *feat)
{
    const int nn = ndev ? min(*ndev, ncells) : ncells;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
        mlp_features_one(m, alpha, cells ? cells[i] : i, feat + (size_t)i * IN);
}

// ---------------------------------------------------------------- weights
// BF16 copies of the FP32 master weights, zero padded: W1 [K0 x HID] and its
// transpose, W2 [HID x HID] and transpose, W3 [HID x OUTP] and transpose
__global__ void k_mlp_pack(const float *p, bf *W1, bf *W1t, bf *W2, bf *W2t, bf *W3, bf *W3t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < K0 * HID) {
        const int k = i / HID, j = i % HID;
        const bf v = k < IN ? to_bf(p[OW1 + k * HID + j]) : (bf)0;
        W1[k * HID + j] = v;
        W1t[j * K0 + k] = v;
    }
    if (i < HID * HID) {
        const int k = i / HID, j = i % HID;
        const bf v = to_bf(p[OW2 + k * HID + j]);
        W2[k * HID + j] = v;
        W2t[j * HID + k] = v;
    }
    if (i < HID * OUTP) {
        const int k = i / OUTP, j = i % OUTP;
        const bf v = j < OUT ? to_bf(p[OW3 + k * OUT + j]) : (bf)0;
        W3[k * OUTP + j] = v;
        W3t[j * HID + k] = v;
    }
}

__global__ void k_mlp_input(const float *feat, int ncap, const int *ndev, bf *X0)
{
    const int n = ndev ? min(*ndev, ncap) : ncap;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * K0; i += gridDim.x * blockDim.x) {
        const int r = i / K0, k = i % K0;
        X0[i] = k < IN ? to_bf(feat[(size_t)r * IN + k]) : (bf)0;
    }
}

// ---------------------------------------------------------------- layers
// C [n x M] = A [n x K] . B [K x M] with A row-major BF16 (rows >= n read as
// 0) and B given as Bt [M x K] row-major.  One warp per 16 rows.  mode 0:
// Z = C + bias (FP32) and H = BF16(ReLU(Z)); mode 1: Y = C + bias (FP32);
// mode 2 (backward through a hidden layer): G = C * (Zf > 0) written as BF16.
template <int K, int M, int MODE>
__device__ __forceinline__ void mlp_gemm_tile(const bf *A, const bf *Bt, const float *bias, int n, int r0, int g, int t,
                                              float *Zout, bf *Hout, const float *Zf)
{
    float acc[M / 8][4];
#pragma unroll
    for (int j = 0; j < M / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
    auto ld = [&](int r, int k) -> bf { return r < n ? A[(size_t)r * K + k] : (bf)0; };
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) {
        const uint32_t a0 = pk(ld(r0 + g, k0 + 2 * t), ld(r0 + g, k0 + 2 * t + 1));
        const uint32_t a1 = pk(ld(r0 + g + 8, k0 + 2 * t), ld(r0 + g + 8, k0 + 2 * t + 1));
        const uint32_t a2 = pk(ld(r0 + g, k0 + 2 * t + 8), ld(r0 + g, k0 + 2 * t + 9));
        const uint32_t a3 = pk(ld(r0 + g + 8, k0 + 2 * t + 8), ld(r0 + g + 8, k0 + 2 * t + 9));
#pragma unroll
        for (int j = 0; j < M / 8; ++j) {
            const bf *bt = Bt + (size_t)(8 * j + g) * K + k0 + 2 * t;
            mma16816(acc[j], a0, a1, a2, a3, pk(bt[0], bt[1]), pk(bt[8], bt[9]));
        }
    }
#pragma unroll
    for (int j = 0; j < M / 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = r0 + g + (e >= 2 ? 8 : 0), col = 8 * j + 2 * t + (e & 1);
            if (r >= n) continue;
            const size_t o = (size_t)r * M + col;
            if (MODE == 0) {
                const float z = acc[j][e] + bias[col];
                Zout[o] = z;
                Hout[o] = to_bf(fmaxf(z, 0.0f));
            } else if (MODE == 1) {
                Zout[o] = acc[j][e] + (col < OUT ? bias[col] : 0.0f);
            } else {
                const float gz = Zf[o] > 0.0f ? acc[j][e] : 0.0f;
                Zout[o] = gz;
                Hout[o] = to_bf(gz);
            }
        }
}

template <int K, int M, int MODE>
__global__ void k_mlp_gemm(const bf *A, const bf *Bt, const float *bias, int ncap, const int *ndev, float *Zout,
                           bf *Hout, const float *Zf)
{
    const int n = ndev ? min(*ndev, ncap) : ncap;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int r0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 16; r0 < n; r0 += ((gridDim.x * blockDim.x) >> 5) * 16)
        mlp_gemm_tile<K, M, MODE>(A, Bt, bias, n, r0, g, t, Zout, Hout, Zf);
}

// output gradient of the mean squared error: dY = 2 (Y - T) / n (FP32 and
// BF16, padded columns 0) and per-block partial losses
__global__ void k_mlp_dy(const float *Y, const float *T, int n, float *dYf, bf *dYb, float *lpart)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < n * OUTP) {
        const int r = i / OUTP, j = i % OUTP;
        float d = 0.0f;
        if (j < OUT) {
            const float e = Y[i] - T[(size_t)r * OUT + j];
            l = e * e;
            d = 2.0f * e / (float)n;
        }
        dYf[i] = d;
        dYb[i] = to_bf(d);
    }
    l = vofd::warp_sum((double)l);
    __shared__ float sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        lpart[blockIdx.x] = s;
    }
}

// weight gradient partials: P[chunk] [K x M] = A[chunk]^T . D[chunk] over CHUNK
// samples (A [n x K], D [n x M], both BF16 row-major); one warp per 16 x 8
// output tile and chunk
template <int K, int M>
__global__ void k_mlp_wgrad(const bf *A, const bf *D, int n, float *P)
{
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    constexpr int TM = M / 8, NT = (K / 16) * TM;
    if (tile >= NT) return;
    const int k0 = (tile / TM) * 16, m0 = (tile % TM) * 8, ch = blockIdx.y;
    const int g = lane >> 2, t = lane & 3;
    const int s0 = ch * CHUNK, s1 = min(n, s0 + CHUNK);
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    auto la = [&](int r, int s) -> bf { return s < s1 ? A[(size_t)s * K + k0 + r] : (bf)0; };  // A^T (r, s)
    auto ld = [&](int s, int c) -> bf { return s < s1 ? D[(size_t)s * M + m0 + c] : (bf)0; };
    for (int sb = s0; sb < s1; sb += 16) {
        const uint32_t a0 = pk(la(g, sb + 2 * t), la(g, sb + 2 * t + 1));
        const uint32_t a1 = pk(la(g + 8, sb + 2 * t), la(g + 8, sb + 2 * t + 1));
        const uint32_t a2 = pk(la(g, sb + 2 * t + 8), la(g, sb + 2 * t + 9));
        const uint32_t a3 = pk(la(g + 8, sb + 2 * t + 8), la(g + 8, sb + 2 * t + 9));
        const uint32_t b0 = pk(ld(sb + 2 * t, g), ld(sb + 2 * t + 1, g));
        const uint32_t b1 = pk(ld(sb + 2 * t + 8, g), ld(sb + 2 * t + 9, g));
        mma16816(acc, a0, a1, a2, a3, b0, b1);
    }
    float *o = P + (size_t)ch * K * M;
    o[(k0 + g) * M + m0 + 2 * t] = acc[0];
    o[(k0 + g) * M + m0 + 2 * t + 1] = acc[1];
    o[(k0 + g + 8) * M + m0 + 2 * t] = acc[2];
    o[(k0 + g + 8) * M + m0 + 2 * t + 1] = acc[3];
}

// bias gradient partials: per chunk, column sums of the FP32 upstream gradient
__global__ void k_mlp_bgrad(const float *G, int n, int M, float *P)
{
    const int ch = blockIdx.x, col = threadIdx.x;
    if (col >= M) return;
    const int s0 = ch * CHUNK, s1 = min(n, s0 + CHUNK);
    float s = 0.0f;
    for (int r = s0; r < s1; ++r) s += G[(size_t)r * M + col];
    P[(size_t)ch * M + col] = s;
}

// sums the chunk partials in chunk order into the flat gradient, then Adam
struct GradPtrs {
    const float *pw1, *pw2, *pw3, *pb1, *pb2, *pb3, *lpart;
    int nch, nlb;
};

__global__ void k_mlp_reduce(GradPtrs q, float *grad, float *loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPARAM) {
        float s = 0.0f;
        if (i < OB1) {
            const int k = i / HID, j = i % HID;
            for (int c = 0; c < q.nch; ++c) s += q.pw1[(size_t)c * K0 * HID + k * HID + j];
        } else if (i < OW2) {
            for (int c = 0; c < q.nch; ++c) s += q.pb1[(size_t)c * HID + (i - OB1)];
        } else if (i < OB2) {
            const int k = (i - OW2) / HID, j = (i - OW2) % HID;
            for (int c = 0; c < q.nch; ++c) s += q.pw2[(size_t)c * HID * HID + k * HID + j];
        } else if (i < OW3) {
            for (int c = 0; c < q.nch; ++c) s += q.pb2[(size_t)c * HID + (i - OB2)];
        } else if (i < OB3) {
            const int k = (i - OW3) / OUT, j = (i - OW3) % OUT;
            for (int c = 0; c < q.nch; ++c) s += q.pw3[(size_t)c * HID * OUTP + k * OUTP + j];
        } else {
            for (int c = 0; c < q.nch; ++c) s += q.pb3[(size_t)c * OUTP + (i - OB3)];
        }
        grad[i] = s;
    }
    if (i == 0 && loss) {
        float s = 0.0f;
        for (int b = 0; b < q.nlb; ++b) s += q.lpart[b];
        *loss = s;  // sum of squared errors; the host divides by n
    }
}

__global__ void k_mlp_adam(float *p, const float *g, float *m1, float *m2, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float b1 = 0.9f, b2 = 0.999f;
    const float m = b1 * m1[i] + (1.0f - b1) * g[i], v = b2 * m2[i] + (1.0f - b2) * g[i] * g[i];
    m1[i] = m;
    m2[i] = v;
    p[i] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
}



// Per cell, once (vof_set_guess): the 27 lattice slots as cell indices (-1:
// the cell itself) and the 6 shape numbers, as vof_mlp_features places them
__global__ void k_mlp_tables(DevMesh m, int *nbr, float *geo)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    int *t = nbr + 27 * (size_t)c;
    for (int k = 0; k < 27; ++k) t[k] = -1;
    const double V = m.vc[c], h = cbrt(V);
    const vofd::V3 cc = vofd::ld3(m.cc, m.nc, c);
    for (int j = m.cpptr[c]; j < m.cpptr[c + 1]; ++j) {
        const int p = m.cpts[j];
        for (int q = m.pptr[p]; q < m.pptr[p + 1]; ++q) {
            const int nb = m.pcell[q];
            vofd::V3 d = vofd::ld3(m.cc, m.nc, nb) - cc;
            if (m.pcode) d = d + vofd::tshift(m, m.pcode[q]);  // periodic: the cell next to c
            const int sx = (d.x > 0.5 * h) - (d.x < -0.5 * h), sy = (d.y > 0.5 * h) - (d.y < -0.5 * h),
                      sz = (d.z > 0.5 * h) - (d.z < -0.5 * h);
            t[(sx + 1) + 3 * (sy + 1) + 9 * (sz + 1)] = nb;
        }
    }
    const double *bx = m.cbox + 6 * (size_t)c;
    const double ex = bx[3] - bx[0], ey = bx[4] - bx[1], ez = bx[5] - bx[2];
    float *g = geo + 6 * (size_t)c;
    g[0] = (float)(ex / h);
    g[1] = (float)(ey / h);
    g[2] = (float)(ez / h);
    g[3] = (float)(V / (ex * ey * ez));
    g[4] = (float)((m.cptr[c + 1] - m.cptr[c]) / 24.0);
    g[5] = (float)((m.cpptr[c + 1] - m.cpptr[c]) / 8.0);
}

// The guess of a step in one kernel: one warp per 16 listed cells gathers
// their features straight into the tensor-core operand layout (from the
// tables), runs the three layers chaining each layer's accumulators into the
// next layer's operands in registers, and writes the clamped offsets.
__global__ void __launch_bounds__(128) k_mlp_guess_fused(const int *nbr, const float *geo,
                                                          const double *__restrict__ alpha, const int *list,
                                                          const int *count, int cap, const bf *W1t, const bf *W2t,
                                                          const bf *W3t, const float *p, float *s0)
{
    const int n = min(*count, cap);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int wstride = (gridDim.x * blockDim.x) >> 5;
    for (int r0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 16; r0 < n; r0 += wstride * 16) {
        // feature (row r, column k) of the tile
        const int ra = r0 + g, rb = r0 + g + 8;
        const int ca = ra < n ? list[ra] : -1, cb = rb < n ? list[rb] : -1;
        auto feat = [&](int c, int k) -> bf {
            if (c < 0 || k >= IN) return (bf)0;
            if (k < 27) {
                const int q = nbr[27 * (size_t)c + k];
                return to_bf((float)alpha[q < 0 ? c : q]);
            }
            return to_bf(geo[6 * (size_t)c + (k - 27)]);
        };
        // layer 1: [16 x 48] . [48 x 64]
        float h1[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) h1[j][0] = h1[j][1] = h1[j][2] = h1[j][3] = 0.0f;
#pragma unroll
        for (int k0 = 0; k0 < K0; k0 += 16) {
            const uint32_t a0 = pk(feat(ca, k0 + 2 * t), feat(ca, k0 + 2 * t + 1));
            const uint32_t a1 = pk(feat(cb, k0 + 2 * t), feat(cb, k0 + 2 * t + 1));
            const uint32_t a2 = pk(feat(ca, k0 + 2 * t + 8), feat(ca, k0 + 2 * t + 9));
            const uint32_t a3 = pk(feat(cb, k0 + 2 * t + 8), feat(cb, k0 + 2 * t + 9));
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const bf *bt = W1t + (size_t)(8 * j + g) * K0 + k0 + 2 * t;
                mma16816(h1[j], a0, a1, a2, a3, pk(bt[0], bt[1]), pk(bt[8], bt[9]));
            }
        }
        // bias, ReLU, BF16: the accumulators of two n-tiles form one k-step of
        // the next layer's operand
        auto act = [&](float (*h)[4], const float *bias, int kk, uint32_t &a0, uint32_t &a1, uint32_t &a2,
                       uint32_t &a3) {
            const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
            a0 = pk(to_bf(fmaxf(h[2 * kk][0] + bias[c0], 0.f)), to_bf(fmaxf(h[2 * kk][1] + bias[c0 + 1], 0.f)));
            a1 = pk(to_bf(fmaxf(h[2 * kk][2] + bias[c0], 0.f)), to_bf(fmaxf(h[2 * kk][3] + bias[c0 + 1], 0.f)));
            a2 = pk(to_bf(fmaxf(h[2 * kk + 1][0] + bias[c1], 0.f)),
                    to_bf(fmaxf(h[2 * kk + 1][1] + bias[c1 + 1], 0.f)));
            a3 = pk(to_bf(fmaxf(h[2 * kk + 1][2] + bias[c1], 0.f)),
                    to_bf(fmaxf(h[2 * kk + 1][3] + bias[c1 + 1], 0.f)));
        };
        float h2[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) h2[j][0] = h2[j][1] = h2[j][2] = h2[j][3] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < HID / 16; ++kk) {
            uint32_t a0, a1, a2, a3;
            act(h1, p + OB1, kk, a0, a1, a2, a3);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const bf *bt = W2t + (size_t)(8 * j + g) * HID + 16 * kk + 2 * t;
                mma16816(h2[j], a0, a1, a2, a3, pk(bt[0], bt[1]), pk(bt[8], bt[9]));
            }
        }
        float y[4] = {0.f, 0.f, 0.f, 0.f};  // output columns 0..7 (the offset is column 3)
#pragma unroll
        for (int kk = 0; kk < HID / 16; ++kk) {
            uint32_t a0, a1, a2, a3;
            act(h2, p + OB2, kk, a0, a1, a2, a3);
            const bf *bt = W3t + (size_t)g * HID + 16 * kk + 2 * t;
            mma16816(y, a0, a1, a2, a3, pk(bt[0], bt[1]), pk(bt[8], bt[9]));
        }
        if (t == 1) {  // column 2t + 1 = 3
            const float b3 = p[OB3 + 3];
            if (ra < n) s0[ra] = fminf(fmaxf(y[1] + b3, 0.02f), 0.98f);
            if (rb < n) s0[rb] = fminf(fmaxf(y[3] + b3, 0.02f), 0.98f);
        }
    }
}

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

}  // namespace

struct vof_mlp {
    int device, max_batch, nch, adam_t;
    float *p, *grad, *m1, *m2;
    bf *W1, *W1t, *W2, *W2t, *W3, *W3t;
    bf *X0, *H1, *H2, *dYb, *dZ2b, *dZ1b;
    float *Z1, *Z2, *Y, *dYf, *dZ2f, *dZ1f, *lpart, *loss;
    float *pw1, *pw2, *pw3, *pb1, *pb2, *pb3;
    std::vector<void *> bufs;
};

namespace {

template <class T>
T *mlp_alloc(vof_mlp *q, size_t n, bool *ok)
{
    void *p = nullptr;
    if (*ok && cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess) {
        q->bufs.push_back(p);
        return (T *)p;
    }
    *ok = false;
    return nullptr;
}

// rows: n, or min(*ndev, n) when ndev is given (a device-side count)
int mlp_forward(vof_mlp *q, const float *feat, int n, const int *ndev, cudaStream_t s)
{
    const int blocks = std::min(cdiv(n, 64), 1024);
    k_mlp_input<<<std::min(cdiv((long)n * K0, 256), 2048), 256, 0, s>>>(feat, n, ndev, q->X0);
    k_mlp_gemm<K0, HID, 0><<<blocks, 128, 0, s>>>(q->X0, q->W1t, q->p + OB1, n, ndev, q->Z1, q->H1, nullptr);
    k_mlp_gemm<HID, HID, 0><<<blocks, 128, 0, s>>>(q->H1, q->W2t, q->p + OB2, n, ndev, q->Z2, q->H2, nullptr);
    k_mlp_gemm<HID, OUTP, 1><<<blocks, 128, 0, s>>>(q->H2, q->W3t, q->p + OB3, n, ndev, q->Y, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

int mlp_backward(vof_mlp *q, const float *target, int n, cudaStream_t s)
{
    const int nlb = cdiv((long)n * OUTP, 256), nch = cdiv(n, CHUNK), blocks = std::min(cdiv(n, 64), 1024);
    k_mlp_dy<<<nlb, 256, 0, s>>>(q->Y, target, n, q->dYf, q->dYb, q->lpart);
    // through layer 3 and 2: dZ = (dY . W^T) masked by the pre-activation
    k_mlp_gemm<OUTP, HID, 2><<<blocks, 128, 0, s>>>(q->dYb, q->W3, nullptr, n, nullptr, q->dZ2f, q->dZ2b, q->Z2);
    k_mlp_gemm<HID, HID, 2><<<blocks, 128, 0, s>>>(q->dZ2b, q->W2, nullptr, n, nullptr, q->dZ1f, q->dZ1b, q->Z1);
    // weight and bias gradients per chunk
    k_mlp_wgrad<HID, OUTP><<<dim3(cdiv((HID / 16) * (OUTP / 8), 4), nch), 128, 0, s>>>(q->H2, q->dYb, n, q->pw3);
    k_mlp_wgrad<HID, HID><<<dim3(cdiv((HID / 16) * (HID / 8), 4), nch), 128, 0, s>>>(q->H1, q->dZ2b, n, q->pw2);
    k_mlp_wgrad<K0, HID><<<dim3(cdiv((K0 / 16) * (HID / 8), 4), nch), 128, 0, s>>>(q->X0, q->dZ1b, n, q->pw1);
    k_mlp_bgrad<<<nch, 64, 0, s>>>(q->dYf, n, OUTP, q->pb3);
    k_mlp_bgrad<<<nch, 64, 0, s>>>(q->dZ2f, n, HID, q->pb2);
    k_mlp_bgrad<<<nch, 64, 0, s>>>(q->dZ1f, n, HID, q->pb1);
    GradPtrs g{q->pw1, q->pw2, q->pw3, q->pb1, q->pb2, q->pb3, q->lpart, nch, nlb};
    k_mlp_reduce<<<cdiv(NPARAM, 256), 256, 0, s>>>(g, q->grad, q->loss);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

int mlp_pack(vof_mlp *q, cudaStream_t s)
{
    k_mlp_pack<<<cdiv(HID * HID, 256), 256, 0, s>>>(q->p, q->W1, q->W1t, q->W2, q->W2t, q->W3, q->W3t);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

}  // namespace

// the reconstruction guess of a step: for the first max_batch listed
// interface cells (device count), the clamped offsets by list position in
// c->mlp_s0 (one fused kernel)
int launch_mlp_guess(vof_ctx *c, const double *alpha, const int *cells, const int *count, int nmax, cudaStream_t s)
{
    vof_mlp *q = c->mlp;
    if (!q) return VOF_OK;
    const int cap = std::min(q->max_batch, nmax);
    if (!cells || !count) return VOF_ERR_INVALID_ARG;
    k_mlp_guess_fused<<<std::min(cdiv(cap, 64), 1024), 128, 0, s>>>(c->mlp_nbr, c->mlp_geo, alpha, cells, count,
                                                                     cap, q->W1t, q->W2t, q->W3t, q->p, c->mlp_s0);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

int mlp_cap(const vof_ctx *c) { return c->mlp ? c->mlp->max_batch : 0; }

extern "C" {

int vof_mlp_create(int max_batch, const float *params, int device, vof_mlp **out)
{
    if (max_batch < 16 || !params || !out) return VOF_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return VOF_ERR_CUDA;
    vof_mlp *q = new (std::nothrow) vof_mlp();
    if (!q) return VOF_ERR_CUDA;
    q->device = device;
    q->max_batch = max_batch;
    q->nch = cdiv(max_batch, CHUNK);
    bool ok = true;
    const size_t B = max_batch;
    q->p = mlp_alloc<float>(q, NPARAM, &ok);
    q->grad = mlp_alloc<float>(q, NPARAM, &ok);
    q->m1 = mlp_alloc<float>(q, NPARAM, &ok);
    q->m2 = mlp_alloc<float>(q, NPARAM, &ok);
    q->W1 = mlp_alloc<bf>(q, K0 * HID, &ok);
    q->W1t = mlp_alloc<bf>(q, K0 * HID, &ok);
    q->W2 = mlp_alloc<bf>(q, HID * HID, &ok);
    q->W2t = mlp_alloc<bf>(q, HID * HID, &ok);
    q->W3 = mlp_alloc<bf>(q, HID * OUTP, &ok);
    q->W3t = mlp_alloc<bf>(q, HID * OUTP, &ok);
    q->X0 = mlp_alloc<bf>(q, B * K0, &ok);
    q->H1 = mlp_alloc<bf>(q, B * HID, &ok);
    q->H2 = mlp_alloc<bf>(q, B * HID, &ok);
    q->dYb = mlp_alloc<bf>(q, B * OUTP, &ok);
    q->dZ2b = mlp_alloc<bf>(q, B * HID, &ok);
    q->dZ1b = mlp_alloc<bf>(q, B * HID, &ok);
    q->Z1 = mlp_alloc<float>(q, B * HID, &ok);
    q->Z2 = mlp_alloc<float>(q, B * HID, &ok);
    q->Y = mlp_alloc<float>(q, B * OUTP, &ok);
    q->dYf = mlp_alloc<float>(q, B * OUTP, &ok);
    q->dZ2f = mlp_alloc<float>(q, B * HID, &ok);
    q->dZ1f = mlp_alloc<float>(q, B * HID, &ok);
    q->lpart = mlp_alloc<float>(q, cdiv((long)B * OUTP, 256), &ok);
    q->loss = mlp_alloc<float>(q, 1, &ok);
    q->pw1 = mlp_alloc<float>(q, (size_t)q->nch * K0 * HID, &ok);
    q->pw2 = mlp_alloc<float>(q, (size_t)q->nch * HID * HID, &ok);
    q->pw3 = mlp_alloc<float>(q, (size_t)q->nch * HID * OUTP, &ok);
    q->pb1 = mlp_alloc<float>(q, (size_t)q->nch * HID, &ok);
    q->pb2 = mlp_alloc<float>(q, (size_t)q->nch * HID, &ok);
    q->pb3 = mlp_alloc<float>(q, (size_t)q->nch * OUTP, &ok);
    ok = ok && cudaMemcpy(q->p, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(q->m1, 0, sizeof(float) * NPARAM) == cudaSuccess &&
         cudaMemset(q->m2, 0, sizeof(float) * NPARAM) == cudaSuccess && mlp_pack(q, 0) == VOF_OK &&
         cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) { vof_mlp_destroy(q); return VOF_ERR_CUDA; }
    *out = q;
    return VOF_OK;
}

void vof_mlp_destroy(vof_mlp *q)
{
    if (!q) return;
    cudaSetDevice(q->device);
    for (void *p : q->bufs) cudaFree(p);
    delete q;
}

int vof_mlp_params(vof_mlp *q, float *params)
{
    if (!q || !params) return VOF_ERR_INVALID_ARG;
    if (cudaSetDevice(q->device) != cudaSuccess) return VOF_ERR_CUDA;
    return cudaMemcpy(params, q->p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) == cudaSuccess ? VOF_OK
                                                                                                   : VOF_ERR_CUDA;
}

int vof_mlp_features(vof_ctx *c, const double *alpha, const int32_t *cells, int ncells, float *feat, void *stream)
{
    if (!c || !alpha || !feat || ncells < 0) return VOF_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return VOF_ERR_CUDA;
    if (ncells == 0) return VOF_OK;
    k_mlp_features<<<std::min(cdiv(ncells, 128), 4096), 128, 0, (cudaStream_t)stream>>>(c->m, alpha, cells, ncells,
                                                                                         nullptr, feat);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

int vof_mlp_forward(vof_mlp *q, const float *feat, int n, float *out, void *stream)
{
    if (!q || !feat || !out || n < 1 || n > q->max_batch) return VOF_ERR_INVALID_ARG;
    if (cudaSetDevice(q->device) != cudaSuccess) return VOF_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int r = mlp_forward(q, feat, n, nullptr, s);
    if (r) return r;
    return cudaMemcpy2DAsync(out, OUT * sizeof(float), q->Y, OUTP * sizeof(float), OUT * sizeof(float), n,
                             cudaMemcpyDeviceToDevice, s) == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

int vof_mlp_gradient(vof_mlp *q, const float *feat, const float *target, int n, float *grad, float *loss,
                     void *stream)
{
    if (!q || !feat || !target || n < 1 || n > q->max_batch) return VOF_ERR_INVALID_ARG;
    if (cudaSetDevice(q->device) != cudaSuccess) return VOF_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int r = mlp_forward(q, feat, n, nullptr, s);
    if (!r) r = mlp_backward(q, target, n, s);
    if (r) return r;
    if (grad && cudaMemcpyAsync(grad, q->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return VOF_ERR_CUDA;
    if (loss) {
        float l = 0.0f;
        if (cudaMemcpyAsync(&l, q->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return VOF_ERR_CUDA;
        *loss = l / (float)n;
    }
    return VOF_OK;
}

int vof_mlp_train_step(vof_mlp *q, const float *feat, const float *target, int n, float lr, float *loss,
                       void *stream)
{
    int r = vof_mlp_gradient(q, feat, target, n, nullptr, loss, stream);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;
    ++q->adam_t;
    const float c1 = 1.0f - powf(0.9f, (float)q->adam_t), c2 = 1.0f - powf(0.999f, (float)q->adam_t);
    k_mlp_adam<<<cdiv(NPARAM, 256), 256, 0, s>>>(q->p, q->grad, q->m1, q->m2, lr, c1, c2);
    return mlp_pack(q, s);
}

int vof_set_guess(vof_ctx *c, vof_mlp *q)
{
    if (!c) return VOF_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return VOF_ERR_CUDA;
    if (q && q->device != c->device) return VOF_ERR_INVALID_ARG;
    if (q && !c->mlp_nbr) {
        if (cudaMalloc(&c->mlp_nbr, sizeof(int) * 27 * (size_t)c->nc) != cudaSuccess ||
            cudaMalloc(&c->mlp_geo, sizeof(float) * 6 * (size_t)c->nc) != cudaSuccess)
            return VOF_ERR_CUDA;
        k_mlp_tables<<<cdiv(c->nc, 128), 128>>>(c->m, c->mlp_nbr, c->mlp_geo);
        if (cudaDeviceSynchronize() != cudaSuccess) return VOF_ERR_CUDA;
    }
    if (q && c->mlp_feat_cap < q->max_batch) {
        // guess and feature buffers for the network's batch (kept until vof_destroy)
        cudaFree(c->mlp_s0);
        cudaFree(c->mlp_feat);
        c->mlp_s0 = nullptr;
        c->mlp_feat = nullptr;
        c->mlp_feat_cap = 0;
        if (cudaMalloc(&c->mlp_s0, sizeof(float) * (size_t)q->max_batch) != cudaSuccess ||
            cudaMalloc(&c->mlp_feat, sizeof(float) * IN * (size_t)q->max_batch) != cudaSuccess)
            return VOF_ERR_CUDA;
        c->mlp_feat_cap = q->max_batch;
    }
    c->mlp = q;
    return VOF_OK;
}

}  // extern "C"

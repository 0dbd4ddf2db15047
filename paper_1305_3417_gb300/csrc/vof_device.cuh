// Device helpers shared by the libvof kernel translation units: double and
// float 3-vectors, warp reductions, list appends, the closed-form cut fraction
// of a tetrahedron, and face triangles.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "vof_internal.h"

namespace vofd {


constexpr int POS_MAXIT = 100;
constexpr double POS_TOL = 1e-13;
// Alg. 1's secant is taken as divergent after this many steps without meeting
// POS_TOL (a stall deep in the cubic corner of the fill near alpha = 0 or 1;
// a converging secant needs about a dozen): bisection from then on
constexpr int POS_SECANT_MAX = 20;
constexpr int CORR_MAXIT = 100;
constexpr double CORR_TOL = 1e-14;
constexpr double CORR_LMAX = 2.0;
constexpr int CORR_NSAMP = 16;
constexpr double BOUND_TOL = 1e-13;
constexpr double BOUND_FLAG = 1e-12;
// local redistribution passes run until no source has both something left
// and a receiver with room; this caps them (each pass finishes a source or
// fills at least one of its receivers)
constexpr int BOUND_PASSES_MAX = 32;
constexpr int CLIP_STACK = 12;
constexpr int DISP_STRIDE = (VOF_MAXFP + 1) * 3;

// Per-lane phase-flux work counters of the instrumented kernel variants
// (WkOn; WkOff compiles to nothing), added to the context's counters at a
// warp's end: one atomic per counter and warp
struct WkOn {
    unsigned v[WK_N] = {};
    unsigned faces = 0;
    __device__ __forceinline__ void add(int i, unsigned x) { v[i] += x; }
    __device__ __forceinline__ void face() { ++faces; }
    __device__ __forceinline__ void flush(unsigned long long *work, int lane)
    {
        if (!work) return;
#pragma unroll
        for (int i = 0; i < WK_N; ++i) {
            const unsigned r = __reduce_add_sync(0xffffffffu, v[i]);
            if (lane == 0 && r) atomicAdd(work + i, (unsigned long long)r);
        }
        if (lane == 0 && faces) atomicAdd(work + WK_FACES, (unsigned long long)faces);
    }
};
struct WkOff {
    __device__ __forceinline__ void add(int, unsigned) {}
    __device__ __forceinline__ void face() {}
    __device__ __forceinline__ void flush(unsigned long long *, int) {}
};
// one lane's count added to counter i (a few per thread)
__device__ __forceinline__ void work_add1(unsigned long long *work, int i, unsigned long long v)
{
    if (work && v) atomicAdd(work + i, v);
}

// ------------------------------------------------------------------ vectors
struct V3 { double x, y, z; };
__device__ __forceinline__ V3 mk(double x, double y, double z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(V3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b)
{
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double det3(V3 a, V3 b, V3 c) { return dot(a, cross(b, c)); }
__device__ __forceinline__ double norm3(V3 a) { return sqrt(dot(a, a)); }
// signed volume of tetrahedron (a,b,c,d)
__device__ __forceinline__ double tvol(V3 a, V3 b, V3 c, V3 d) { return det3(b - a, c - a, d - a) / 6.0; }

__device__ __forceinline__ V3 ldP(const DevMesh &m, int p)
{
    return mk(__ldg(m.px + p), __ldg(m.py + p), __ldg(m.pz + p));
}
__device__ __forceinline__ V3 ld3(const double *a, int n, int i)
{
    return mk(__ldg(a + i), __ldg(a + n + i), __ldg(a + 2 * n + i));
}
__device__ __forceinline__ void st3(double *a, int n, int i, V3 v)
{
    a[i] = v.x; a[n + i] = v.y; a[2 * n + i] = v.z;
}
// the translation of a periodic code, (i L0 + j L1) + k L2 (exact products)
constexpr int T_NONE = 13;
__device__ __forceinline__ V3 tshift(const DevMesh &m, int code)
{
    const double i = code % 3 - 1, j = (code / 3) % 3 - 1, k = code / 9 - 1;
    return mk(i * m.L[0], i * m.L[1], i * m.L[2]) + mk(j * m.L[3], j * m.L[4], j * m.L[5]) +
           mk(k * m.L[6], k * m.L[7], k * m.L[8]);
}

// Comparisons of a double with a threshold t > 0 through the order of the bit
// patterns as signed 64-bit integers: monotone on the non-negative doubles, and
// every negative double (-0 included) orders below t.  The same decision as the
// FP64 compare for every value that is not NaN, taken in 32-bit integer
// instructions on the two halves (the FP64 pipe of this part runs at 1/64 of
// the FP32 rate).  The halves come out of an opaque register move, so that the
// compiler cannot fold the tests back into FP64 compares.
struct DBits { int hi; unsigned lo; };
__device__ __forceinline__ DBits dbits(double x)
{
    DBits r;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(r.lo), "=r"(r.hi) : "d"(x));
    return r;
}
__device__ __forceinline__ bool bits_le(DBits a, DBits b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ bool le_pos(double a, double t) { return bits_le(dbits(a), dbits(t)); }
__device__ __forceinline__ bool lt_pos(double a, double t) { return !bits_le(dbits(t), dbits(a)); }
__device__ __forceinline__ bool ge_pos(double a, double t) { return bits_le(dbits(t), dbits(a)); }
__device__ __forceinline__ bool gt_pos(double a, double t) { return !bits_le(dbits(a), dbits(t)); }
// a < -t (t > 0): negative, with a magnitude above t
__device__ __forceinline__ bool lt_neg(double a, double t)
{
    DBits x = dbits(a);
    const bool neg = x.hi < 0;
    x.hi &= 0x7fffffff;
    return neg && !bits_le(x, dbits(t));
}
// a is +0 or -0
__device__ __forceinline__ bool is_zero(double a)
{
    const DBits x = dbits(a);
    return ((x.hi & 0x7fffffff) | x.lo) == 0;
}
// a is +0
__device__ __forceinline__ bool is_pzero(double a)
{
    const DBits x = dbits(a);
    return (x.hi | x.lo) == 0;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// append with one atomic per warp
__device__ __forceinline__ void warp_append(bool pred, int val, int *list, int *count, int cap,
                                            unsigned *status)
{
    unsigned mask = __ballot_sync(0xffffffffu, pred);
    if (!mask) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) {
        int pos = base + __popc(mask & ((1u << lane) - 1u));
        if (pos < cap) list[pos] = val;
        else atomicOr(status, VOF_ST_CAPACITY);
    }
}

// fraction of a tetrahedron below the level d of a linear function whose sorted
// vertex values are h0 <= h1 <= h2 <= h3.  One/three vertices below: product of
// edge fractions; two below: the wedge split into three tetrahedra, whose
// barycentric volumes are ab, a(1-b)e and (1-a)ce -- all terms non-negative.
__device__ __forceinline__ double frac_below(double h0, double h1, double h2, double h3, double d)
{
    if (d <= h0) return 0.0;
    if (d >= h3) return 1.0;
    if (d <= h1) {
        double x = d - h0;
        return (x / (h1 - h0)) * (x / (h2 - h0)) * (x / (h3 - h0));
    }
    if (d >= h2) {
        double y = h3 - d;
        return 1.0 - (y / (h3 - h0)) * (y / (h3 - h1)) * (y / (h3 - h2));
    }
    double a = (d - h0) / (h2 - h0), b = (d - h0) / (h3 - h0);
    double c = (d - h1) / (h2 - h1), e = (d - h1) / (h3 - h1);
    return a * b + a * (1.0 - b) * e + (1.0 - a) * c * e;
}

__device__ __forceinline__ void sort4(double &a, double &b, double &c, double &d)
{
    double t;
#define CS(p, q) if (p > q) { t = p; p = q; q = t; }
    CS(a, b) CS(c, d) CS(a, c) CS(b, d) CS(b, c)
#undef CS
}

// i-th triangle of face f oriented along S_f (flip for the neighbour side)
__device__ __forceinline__ void face_tri(const DevMesh &m, int f, int t, bool flip, V3 &t0, V3 &t1,
                                         V3 &t2)
{
    int b = __ldg(m.fptr + f), n = __ldg(m.fptr + f + 1) - b;
    if (n == 3) {
        t0 = ldP(m, __ldg(m.fpts + b)); t1 = ldP(m, __ldg(m.fpts + b + 1)); t2 = ldP(m, __ldg(m.fpts + b + 2));
    } else {
        t0 = ld3(m.cf, m.nf, f);
        t1 = ldP(m, __ldg(m.fpts + b + t));
        t2 = ldP(m, __ldg(m.fpts + b + (t + 1 == n ? 0 : t + 1)));
    }
    if (flip) { V3 s = t1; t1 = t2; t2 = s; }
}


}  // namespace vofd

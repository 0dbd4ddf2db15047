// FP64 kernels of libvof: geometry set-up, reconstruction (NAG gradient + Alg. 1
// positioning), point velocities, flux-polyhedron construction and correction,
// phase fluxes by tetrahedral clipping, the conservative update and the
// bounding pass.  Every kernel bounds its loops and reports problems through
// the context status word; none traps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "vof_internal.h"
#include "vof_device.cuh"

namespace {
using namespace vofd;

// =========================================================== set-up kernels
__global__ void k_face_geom(DevMesh m, double *cf, double *sf, double *nagc)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.nf) return;
    int b = m.fptr[f], n = m.fptr[f + 1] - b;
    V3 c = mk(0, 0, 0);
    for (int i = 0; i < n; ++i) c = c + ldP(m, m.fpts[b + i]);
    c = c * (1.0 / n);
    V3 S = mk(0, 0, 0);
    if (n == 3) {
        V3 p0 = ldP(m, m.fpts[b]), p1 = ldP(m, m.fpts[b + 1]), p2 = ldP(m, m.fpts[b + 2]);
        S = cross(p1 - p0, p2 - p0) * 0.5;
    } else {
        for (int t = 0; t < n; ++t) {
            V3 a = ldP(m, m.fpts[b + t]) - c, e = ldP(m, m.fpts[b + (t + 1) % n]) - c;
            S = S + cross(a, e) * 0.5;
        }
    }
    // NAG face value (Sec. 2.2.1) as a weighted sum of the point values:
    // phi_f = sum_t w_t (phi' + phi_t + phi_t+1)/3, phi' the point mean, w_t the
    // area share of fan triangle t, so point k weighs (1/n + w_k + w_k-1)/3.
    double A[VOF_MAXFP], sa = 0.0;
    for (int t = 0; t < n; ++t) {
        V3 a = ldP(m, m.fpts[b + t]) - c, e = ldP(m, m.fpts[b + (t + 1) % n]) - c;
        A[t] = 0.5 * norm3(cross(a, e));
        sa += A[t];
    }
    for (int k = 0; k < n; ++k)
        nagc[b + k] = (1.0 / n + A[k] / sa + A[(k + n - 1) % n] / sa) / 3.0;
    st3(cf, m.nf, f, c);
    st3(sf, m.nf, f, S);
}

__global__ void k_cell_geom(DevMesh m, double *cc, double *vc, double *cbox, unsigned *bad)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    int p0 = m.cpptr[c], p1 = m.cpptr[c + 1];
    V3 s = mk(0, 0, 0), lo = mk(1e300, 1e300, 1e300), hi = mk(-1e300, -1e300, -1e300);
    for (int i = p0; i < p1; ++i) {
        V3 p = ldP(m, m.cpts[i]);
        s = s + p;
        lo = mk(fmin(lo.x, p.x), fmin(lo.y, p.y), fmin(lo.z, p.z));
        hi = mk(fmax(hi.x, p.x), fmax(hi.y, p.y), fmax(hi.z, p.z));
    }
    V3 ctr = s * (1.0 / (p1 - p0));
    double V = 0.0;
    for (int k = m.cptr[c]; k < m.cptr[c + 1]; ++k) {
        int code = m.cface[k], f = code >> 1;
        int n = m.fptr[f + 1] - m.fptr[f], nt = n == 3 ? 1 : n;
        for (int t = 0; t < nt; ++t) {
            V3 a, b, e;
            face_tri(m, f, t, code & 1, a, b, e);
            double v = tvol(ctr, a, b, e);
            if (!(v > 0.0)) atomicOr(bad, 1u);
            V += v;
        }
    }
    st3(cc, m.nc, c, ctr);
    vc[c] = V;
    cbox[6 * c + 0] = lo.x; cbox[6 * c + 1] = lo.y; cbox[6 * c + 2] = lo.z;
    cbox[6 * c + 3] = hi.x; cbox[6 * c + 4] = hi.y; cbox[6 * c + 5] = hi.z;
}

// Eq. w_pc: inverse distance from the point to each point-cell centre (on a
// periodic mesh the cell moved next to the point), normalised
__global__ void k_point_weights(DevMesh m, double *pw)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m.np) return;
    V3 x = ldP(m, p);
    auto centre = [&](int j) {
        V3 c = ld3(m.cc, m.nc, m.pcell[j]);
        return m.pcode ? c + tshift(m, m.pcode[j]) : c;
    };
    double s = 0.0;
    for (int j = m.pptr[p]; j < m.pptr[p + 1]; ++j) s += 1.0 / norm3(x - centre(j));
    for (int j = m.pptr[p]; j < m.pptr[p + 1]; ++j) pw[j] = (1.0 / norm3(x - centre(j))) / s;
}

// wall table: distinct unit normals of the wall faces through each wall point
__global__ void k_wall_table(DevMesh m, const int *wptr, const int *wface, int nrows, double *wallt)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int cnt = 0;
    V3 v[2] = {mk(0, 0, 0), mk(0, 0, 0)};
    for (int j = wptr[r]; j < wptr[r + 1]; ++j) {
        int f = wface[j];
        V3 S = ld3(m.sf, m.nf, f);
        V3 u = S * (1.0 / norm3(S));
        bool dup = false;
        for (int k = 0; k < cnt && k < 2; ++k)
            if (fabs(dot(u, v[k])) > 1.0 - 1e-12) dup = true;
        if (dup || cnt >= 3) continue;
        if (cnt < 2) v[cnt] = u;
        ++cnt;
    }
    double *o = wallt + 7 * r;
    o[0] = cnt;
    o[1] = v[0].x; o[2] = v[0].y; o[3] = v[0].z;
    o[4] = v[1].x; o[5] = v[1].y; o[6] = v[1].z;
}

// ====================================================== point velocity (A4)
__device__ __forceinline__ V3 point_velocity(const DevMesh &m, int p, const double *__restrict__ Uc)
{
    V3 u = mk(0, 0, 0);
    for (int j = __ldg(m.pptr + p); j < __ldg(m.pptr + p + 1); ++j) {
        int c = __ldg(m.pcell + j);
        u = u + ld3(Uc, m.nc, c) * __ldg(m.pw + j);
    }
    int r = __ldg(m.pwall + p);
    if (r >= 0) {
        const double *w = m.wallt + 7 * r;
        int cnt = (int)w[0];
        V3 n1 = mk(w[1], w[2], w[3]), n2 = mk(w[4], w[5], w[6]);
        if (cnt == 1) u = u - n1 * dot(u, n1);
        else if (cnt == 2) {
            V3 t = cross(n1, n2);
            t = t * (1.0 / norm3(t));
            u = t * dot(u, t);
        } else if (cnt >= 3) u = mk(0, 0, 0);
    }
    return u;
}

__global__ void k_point_velocity(DevMesh m, const double *__restrict__ Uc, double *Up)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m.np) return;
    st3(Up, m.np, p, point_velocity(m, p, Uc));
}

// ===================================================== reconstruction (A1-A3)
// one warp per cell: NAG gradient over the (face, point) entries of the cell,
// then Alg. 1 with the fill function summed over the cell tetrahedra, one or
// two per lane, each a closed-form cut fraction of its sorted projections.

// Reciprocal for the fill of the mixed positioning: the correctly rounded FP32
// reciprocal for R = float (the FP32 stage only brings the residual to 1e-5);
// for R = double the FP32 reciprocal refined by one Newton-Raphson step
// r <- r + r (1 - x r) in FP64, whose relative error is about the square of
// the FP32 one (~4e-15), with exact division where x is outside the FP32
// range.  The FP64 pipe of this part runs at 1/64 of the FP32 rate: this is a
// conversion pair and two FMAs in place of a full FP64 division.
__device__ __noinline__ double exact_rcp(double x) { return 1.0 / x; }
template <class R> __device__ __forceinline__ R mx_rcp(R x);
template <> __device__ __forceinline__ float mx_rcp<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double mx_rcp<double>(double x)
{
    const float r0 = __frcp_rn((float)x);
    if (!isfinite(r0) || r0 == 0.0f) return exact_rcp(x);
    const double r = (double)r0;
    return fma(r, fma(-x, r, 1.0), r);
}

// Cut fraction of a tetrahedron with sorted projections h0..h3 below level d,
// and its derivative in d (the cut area over the volume): the same closed form
// as frac_below, differentiated piece by piece.
template <class R>
__device__ __forceinline__ R frac_below_dd(R h0, R h1, R h2, R h3, R d, R &df)
{
    df = R(0);
    if (d <= h0) return R(0);
    if (d >= h3) return R(1);
    if (d <= h1) {
        const R x = d - h0, p = mx_rcp<R>((h1 - h0) * (h2 - h0) * (h3 - h0));
        df = R(3) * x * x * p;
        return x * x * x * p;
    }
    if (d >= h2) {
        const R y = h3 - d, q = mx_rcp<R>((h3 - h0) * (h3 - h1) * (h3 - h2));
        df = R(3) * y * y * q;
        return R(1) - y * y * y * q;
    }
    const R ra = mx_rcp<R>(h2 - h0), rb = mx_rcp<R>(h3 - h0), rc = mx_rcp<R>(h2 - h1), re = mx_rcp<R>(h3 - h1);
    const R a = (d - h0) * ra, b = (d - h0) * rb, c = (d - h1) * rc, e = (d - h1) * re;
    df = ra * b + a * rb + ra * (R(1) - b) * e - a * rb * e + a * (R(1) - b) * re - ra * c * e +
         (R(1) - a) * rc * e + (R(1) - a) * c * re;
    return a * b + a * (R(1) - b) * e + (R(1) - a) * c * e;
}

// MIXED: cells with 1e-4 < alpha < 1 - 1e-4 are positioned by safeguarded
// Newton steps on the fill, whose derivative is the cut area: first in FP32
// on projections relative to the cell centre while the residual is above 1e-5
// (FP32 rounding of the fill is ~1e-7), then in FP64 to the 1e-13 stop; a
// step that leaves the bracket is replaced by bisection.  Cells within 1e-4
// of 0 or 1 take FP64 Newton from the corner estimate.  The plain FP64 form
// follows Alg. 1 (secant; bisection once the secant leaves the bracket or
// has not converged in POS_SECANT_MAX steps).
// G lanes per cell: 32, or 8 where every cell has at most 16 tetrahedra (a
// tetrahedral mesh: four cells per warp); reductions over the cell's lanes
template <bool LIST, bool MIXED, int G, int KL, bool COUNT>
__global__ void __launch_bounds__(128, KL == 3 ? 4 : 5) k_reconstruct(DevMesh m, const double *__restrict__ alpha,
                                                     const double *__restrict__ palpha, const int *list,
                                                     const int *count, double *nout, double *dout,
                                                     uint8_t *fout, int *itout, int *maxit, unsigned *status,
                                                     const float *__restrict__ s0, int s0cap, int *next,
                                                     unsigned long long *work, const double *__restrict__ gin)
{
    // fill evaluations per cell tetrahedron (FP64, FP32), counted by the
    // cell's first lane and added once per thread at the end
    unsigned long long nf64 = 0, nf32 = 0;
    const int lane = threadIdx.x & (G - 1);
    const unsigned tm = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (threadIdx.x & 31 & ~(G - 1));
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int nwarps = (gridDim.x * blockDim.x) / G;
    auto tsum = [&](double v) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(tm, v, o);
        return v;
    };
    auto tmin = [&](double v) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(tm, v, o));
        return v;
    };
    auto tmax = [&](double v) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(tm, v, o));
        return v;
    };
    const int total = LIST ? *count : m.nc;
    const double eps = m.eps;
    // LIST with a counter: a lane group takes its next cell as it finishes one
    // (cells differ in positioning iterations); else static striding
    const bool dyn = LIST && next != nullptr;
    auto take = [&]() {
        int v = 0;
        if (lane == 0) v = atomicAdd(next, 1);
        return __shfl_sync(tm, v, 0, G);
    };
    for (int item = dyn ? take() : warp; item < total; item = dyn ? take() : item + nwarps) {
        const int c = LIST ? list[item] : item;
        const double a = alpha[c];
        uint8_t fl = 0;
        V3 nn = mk(0, 0, 0);
        double dd = 0.0;
        int it = 0;
        if (a >= 1.0 - eps) fl = VOF_FULL;
        else if (a > eps) {
            fl = VOF_INTERFACE;
            const double V = m.vc[c];
            // ---- NAG gradient: lane j handles the j-th (face, point) entry
            // (a given gradient instead, times V: the generalised LSQ one)
            V3 g = mk(0, 0, 0);
            if (gin) {
                if (lane == 0) g = ld3(gin, m.nc, c) * V;
            } else
            for (int j = __ldg(m.ceptr + c) + lane, e1 = __ldg(m.ceptr + c + 1); j < e1; j += G) {
                const int2 en = __ldg(m.cent + j);  // {fpts slot, face code}
                const int f = en.y >> 1, p = __ldg(m.fpts + en.x);
                double ap = 0.0;  // Eq. idwpointphi (precomputed per point when palpha is given)
                if (palpha) ap = __ldg(palpha + p);
                else
                    for (int q = __ldg(m.pptr + p); q < __ldg(m.pptr + p + 1); ++q)
                        ap += __ldg(m.pw + q) * __ldg(alpha + __ldg(m.pcell + q));
                double w = __ldg(m.nagc + en.x) * ap;
                if (en.y & 1) w = -w;  // Eq. own-nei: the neighbour sees -S_f
                g = g + ld3(m.sf, m.nf, f) * w;
            }
            // g = G / V; the cell is oriented where |g| V^(1/3) > 1e-12, taken
            // as |G|^6 > 1e-72 V^4 (no cube root, square root or division)
            g = mk(tsum(g.x), tsum(g.y), tsum(g.z));
            const double g2 = dot(g, g);
            if (g2 * g2 * g2 > 1e-72 * (V * V) * (V * V)) {
                nn = g * -rsqrt(g2);  // points out of the phase
                fl |= VOF_ORIENTED;
                // ---- cell tetrahedra (c_c, outward face triangle), lanes j, j+32
                const V3 ctr = ld3(m.cc, m.nc, c);
                double h[KL][4], vk[KL];
                float hf[KL][4], vkf[KL];
                const double href = dot(nn, ctr);
                double lo = 1e300, hi = -1e300;
#pragma unroll
                for (int s = 0; s < KL; ++s) {
                    vk[s] = 0.0;
                    h[s][0] = h[s][1] = h[s][2] = h[s][3] = 0.0;
                    vkf[s] = 0.0f;
                    hf[s][0] = hf[s][1] = hf[s][2] = hf[s][3] = 0.0f;
                    const int tj = __ldg(m.ctptr + c) + lane + G * s;
                    if (tj >= __ldg(m.ctptr + c + 1)) continue;
                    const int4 te = __ldg(m.ctet + tj);  // {face code, slot a, slot b, slot c or -1}
                    V3 t0, t1, t2;
                    if (te.w >= 0) {
                        t0 = ldP(m, __ldg(m.fpts + te.y)); t1 = ldP(m, __ldg(m.fpts + te.z)); t2 = ldP(m, __ldg(m.fpts + te.w));
                    } else {
                        t0 = ld3(m.cf, m.nf, te.x >> 1); t1 = ldP(m, __ldg(m.fpts + te.y)); t2 = ldP(m, __ldg(m.fpts + te.z));
                    }
                    if (te.x & 1) { V3 q = t1; t1 = t2; t2 = q; }
                    vk[s] = fabs(tvol(ctr, t0, t1, t2));
                    double e0 = dot(nn, ctr), e1 = dot(nn, t0), e2 = dot(nn, t1), e3 = dot(nn, t2);
                    sort4(e0, e1, e2, e3);
                    h[s][0] = e0; h[s][1] = e1; h[s][2] = e2; h[s][3] = e3;
                    if (MIXED) {
                        hf[s][0] = (float)(e0 - href); hf[s][1] = (float)(e1 - href);
                        hf[s][2] = (float)(e2 - href); hf[s][3] = (float)(e3 - href);
                        vkf[s] = (float)vk[s];
                    }
                    lo = fmin(lo, e0);
                    hi = fmax(hi, e3);
                }
                const double dmin = tmin(lo), dmax = tmax(hi);
                double x = 0.0;
                int it32 = 0;
                if (MIXED && a > 1e-4 && a < 1.0 - 1e-4) {
                    // ---- FP32 Newton, relative to the cell centre's projection
                    const float Vf = (float)V, af = (float)a, rVf = __frcp_rn(Vf);
                    float Ar = (float)(dmin - href), Br = (float)(dmax - href);
                    // start: the learned offset where one is given, else alpha
                    const float sg = (s0 && item < s0cap) ? s0[item] : af;
                    float xr = Ar + sg * (Br - Ar);
                    int near = 0;
                    while (it < POS_MAXIT) {
                        float part = 0.0f, dpart = 0.0f;
#pragma unroll
                        for (int s = 0; s < KL; ++s)
                            if (vkf[s] > 0.0f) {
                                float df;
                                part += vkf[s] * frac_below_dd(hf[s][0], hf[s][1], hf[s][2], hf[s][3], xr, df);
                                dpart += vkf[s] * df;
                            }
#pragma unroll
                        for (int o = G / 2; o > 0; o >>= 1) {
                            part += __shfl_xor_sync(tm, part, o);
                            dpart += __shfl_xor_sync(tm, dpart, o);
                        }
                        ++it;
                        const float gf = part * rVf - af;
                        // below 1e-5 the FP32 sign is not reliable: the bracket takes
                        // no update from it, and after two more Newton steps (down to
                        // the FP32 rounding of the fill) FP64 takes over
                        const bool sure = fabsf(gf) > 1e-5f;
                        if (sure) {
                            if (gf < 0.0f) Ar = xr; else Br = xr;
                        }
                        float xn = xr - gf * Vf * __frcp_rn(dpart);
                        if (!(xn > Ar && xn < Br)) xn = 0.5f * (Ar + Br);
                        if (!(xn > Ar && xn < Br)) break;  // bracket at FP32 resolution
                        xr = xn;
                        if (!sure && ++near >= 2) break;
                    }
                    // ---- FP64 Newton from there
                    it32 = it;
                    const double rV = 1.0 / V;
                    double A = href + (double)Ar, B = href + (double)Br;
                    x = href + (double)xr;
                    while (it < POS_MAXIT) {
                        double part = 0.0, dpart = 0.0;
#pragma unroll
                        for (int s = 0; s < KL; ++s)
                            if (vk[s] > 0.0) {
                                double df;
                                part += vk[s] * frac_below_dd(h[s][0], h[s][1], h[s][2], h[s][3], x, df);
                                dpart += vk[s] * df;
                            }
                        const double gx = tsum(part) * rV - a;
                        dpart = tsum(dpart);
                        ++it;
                        if (fabs(gx) <= POS_TOL) break;
                        if (gx < 0) A = x; else B = x;
                        if (B - A <= 1e-15 * (dmax - dmin)) break;
                        // the slope only sets the rate, not the root: an FP32
                        // reciprocal of it (a step that leaves the bracket, or is
                        // NaN, is replaced by bisection)
                        double xn = x - gx * V * (double)__frcp_rn((float)dpart);
                        if (!(xn > A && xn < B)) xn = 0.5 * (A + B);
                        x = xn;
                    }
                } else if (MIXED) {
                    // ---- alpha within 1e-4 of 0 or 1: FP64 Newton from the corner
                    // estimate (near an end the fill grows like the cube of the
                    // distance from the extreme vertex)
                    double A = dmin, B = dmax;
                    const double rV = 1.0 / V;
                    x = a < 0.5 ? dmin + (dmax - dmin) * cbrt(a) : dmax - (dmax - dmin) * cbrt(1.0 - a);
                    while (it < POS_MAXIT) {
                        double part = 0.0, dpart = 0.0;
#pragma unroll
                        for (int s = 0; s < KL; ++s)
                            if (vk[s] > 0.0) {
                                double df;
                                part += vk[s] * frac_below_dd(h[s][0], h[s][1], h[s][2], h[s][3], x, df);
                                dpart += vk[s] * df;
                            }
                        const double gx = tsum(part) * rV - a;
                        dpart = tsum(dpart);
                        ++it;
                        if (fabs(gx) <= POS_TOL) break;
                        if (gx < 0) A = x; else B = x;
                        if (B - A <= 1e-15 * (dmax - dmin)) break;
                        // the slope only sets the rate, not the root: an FP32
                        // reciprocal of it (a step that leaves the bracket, or is
                        // NaN, is replaced by bisection)
                        double xn = x - gx * V * (double)__frcp_rn((float)dpart);
                        if (!(xn > A && xn < B)) xn = 0.5 * (A + B);
                        x = xn;
                    }
                } else {
                    // ---- Alg. 1: secant, bisection once the secant leaves the
                    // bracket or has stalled for POS_SECANT_MAX steps
                    double A = dmin, B = dmax, x0 = A, g0 = -a, x1 = B, g1 = 1.0 - a, gx = 0.0;
                    bool bisect = false;
                    while (it < POS_MAXIT) {
                        if (it >= POS_SECANT_MAX) bisect = true;
                        if (!bisect) {
                            x = x1 - g1 * (x1 - x0) / (g1 - g0);
                            if (!(x > A && x < B)) bisect = true;
                        }
                        if (bisect) x = 0.5 * (A + B);
                        double part = 0.0;
#pragma unroll
                        for (int s = 0; s < KL; ++s)
                            if (vk[s] > 0.0) part += vk[s] * frac_below(h[s][0], h[s][1], h[s][2], h[s][3], x);
                        gx = tsum(part) / V - a;
                        ++it;
                        if (gx < 0) A = x; else B = x;
                        x0 = x1; g0 = g1; x1 = x; g1 = gx;
                        if (fabs(gx) <= POS_TOL) break;
                        if (B - A <= 1e-15 * (dmax - dmin)) break;
                    }
                }
                if (it >= POS_MAXIT && lane == 0) atomicOr(status, VOF_ST_POS_NOT_CONVERGED);
                if (COUNT && lane == 0) {
                    const unsigned nte = __ldg(m.ctptr + c + 1) - __ldg(m.ctptr + c);
                    nf32 += (unsigned long long)it32 * nte;
                    nf64 += (unsigned long long)(it - it32) * nte;
                }
                dd = x;
            }
        }
        if (lane == 0) {
            if (nout) st3(nout, m.nc, c, nn);
            if (dout) dout[c] = dd;
            if (fout) fout[c] = fl;
            if (itout) itout[c] = it;
            if (maxit && it > 0) atomicMax(maxit, it);
        }
    }
    if (!COUNT) return;
    const unsigned r64 = __reduce_add_sync(0xffffffffu, (unsigned)nf64);
    const unsigned r32 = __reduce_add_sync(0xffffffffu, (unsigned)nf32);
    if ((threadIdx.x & 31) == 0) {
        work_add1(work, WK_FILL64, r64);
        work_add1(work, WK_FILL32, r32);
    }
}

// ======================================== flux polyhedra and correction (A5)
// Cubic V(lambda) = C1 lambda + C2 lambda^2 + C3 lambda^3 of the signed swept
// volume.  Each face triangle (a0,a1,a2), ordered by key (face centre first,
// then global point index, parity par), sweeps to b_k = a_k - lambda w_k and is
// split into the tetrahedra (a0,a1,a2,b2), (a0,a1,b2,b1), (a0,b0,b1,b2), whose
// signed volumes -par*det/6 expand, with E1 = a1-a0, E2 = a2-a0, into
//   k1 = -det(E1,E2,w0+w1+w2),  k2 = det(E1,w2,w1)+det(w0,w1,E2)+det(w0,E1,w2),
//   k3 = -det(w0,w1,w2).
struct Cubic { double c1, c2, c3, s1, s2, s3; };

__device__ __forceinline__ void prism_cubic(V3 a0, V3 a1, V3 a2, V3 w0, V3 w1, V3 w2, long k0,
                                            long k1, long k2, Cubic &q)
{
    int par = 1;
    // sort (a,w,k) triples by key, tracking permutation parity
    if (k1 < k0) { V3 t = a0; a0 = a1; a1 = t; t = w0; w0 = w1; w1 = t; long u = k0; k0 = k1; k1 = u; par = -par; }
    if (k2 < k1) { V3 t = a1; a1 = a2; a2 = t; t = w1; w1 = w2; w2 = t; long u = k1; k1 = k2; k2 = u; par = -par; }
    if (k1 < k0) { V3 t = a0; a0 = a1; a1 = t; t = w0; w0 = w1; w1 = t; long u = k0; k0 = k1; k1 = u; par = -par; }
    V3 E1 = a1 - a0, E2 = a2 - a0;
    const double f = par > 0 ? -1.0 / 6.0 : 1.0 / 6.0;
    double t1 = -det3(E1, E2, w0 + w1 + w2) * f;
    double t2 = (det3(E1, w2, w1) + det3(w0, w1, E2) + det3(w0, E1, w2)) * f;
    double t3 = -det3(w0, w1, w2) * f;
    q.c1 += t1; q.c2 += t2; q.c3 += t3;
    q.s1 += fabs(t1); q.s2 += fabs(t2); q.s3 += fabs(t3);
}

// loads the face's points and per-point displacements w = U_p dt
template <bool IDW>
__device__ __forceinline__ int face_points(const DevMesh &m, int f, const double *__restrict__ U,
                                           double dt, V3 *A, V3 *W, int *id)
{
    int b = __ldg(m.fptr + f), n = __ldg(m.fptr + f + 1) - b;
    for (int i = 0; i < n; ++i) {
        int p = __ldg(m.fpts + b + i);
        id[i] = __ldg(m.fkey + b + i);  // the point's index (its master's on a periodic mesh)
        A[i] = ldP(m, p);
        V3 u = IDW ? point_velocity(m, p, U) : ld3(U, m.np, p);
        W[i] = u * dt;
    }
    return n;
}

// 1/n for the face-centre average (a table: no FP64 division)
__device__ __forceinline__ double inv_n(int n)
{
    return n == 4 ? 0.25 : n == 3 ? 1.0 / 3.0 : n == 5 ? 0.2 : n == 6 ? 1.0 / 6.0 : n == 7 ? 1.0 / 7.0 : 0.125;
}

// face-centre displacement: the mean of the point displacements
__device__ __forceinline__ V3 centre_disp(int n, const V3 *W)
{
    V3 wc = mk(0, 0, 0);
    for (int i = 0; i < n; ++i) wc = wc + W[i];
    return wc * inv_n(n);
}

__device__ __forceinline__ Cubic face_cubic(const DevMesh &m, int f, int n, const V3 *A, const V3 *W,
                                            const int *id)
{
    Cubic q = {0, 0, 0, 0, 0, 0};
    if (n == 3) {
        prism_cubic(A[0], A[1], A[2], W[0], W[1], W[2], id[0], id[1], id[2], q);
    } else {
        V3 c = ld3(m.cf, m.nf, f), wc = centre_disp(n, W);
        for (int t = 0; t < n; ++t) {
            int u = t + 1 == n ? 0 : t + 1;
            prism_cubic(c, A[t], A[u], wc, W[t], W[u], -1, id[t], id[u], q);
        }
    }
    return q;
}

__device__ __forceinline__ double cubic_at(const Cubic &q, double x) { return ((q.c3 * x + q.c2) * x + q.c1) * x; }

// Root of V(lambda) = tau in the first sign-changing interval of the grid
// k*LMAX/NSAMP (the bracket is the same one the secant oracle uses), refined by
// Newton steps that fall back to bisection when they leave the bracket.
// Returns lambda, or -1 (normal-sweep fallback) when no interval brackets a root.
// A flux below 1e-12 of |S_f| max|w| (noise = the rounding of a zero flux, e.g.
// on a wall) gives lambda = 0: no sweep.  The test is taken on squares,
// tau^2 <= 1e-24 |S_f|^2 max|w|^2 (noise2), which needs no square root.
// The sign of V(lambda_k) - tau at a grid point is read from an FP32
// evaluation where that is clearly away from zero (the FP32 conversion of the
// four coefficients and Horner's rounding stay below about 7 units of 2^-24,
// 4.2e-7, of the terms' magnitude B; the test asks for 1e-6 B),
// else from the FP64 one: the same signs, so the same bracket, as FP64
// throughout.  The bracket's end values are FP64.  The Newton step divides by
// the slope through an FP32 reciprocal (the slope sets the rate, not the root).
__device__ double solve_lambda(const Cubic &q, double tau, double noise2, int &its, unsigned &nev)
{
    its = 0;
    if (tau == 0.0) return 0.0;
    if (tau * tau <= 1e-24 * noise2) return 0.0;
    const float c1 = (float)q.c1, c2 = (float)q.c2, c3 = (float)q.c3, tf = (float)tau;
    const float a1 = fabsf(c1), a2 = fabsf(c2), a3 = fabsf(c3), at = fabsf(tf);
    constexpr double STEP = CORR_LMAX / CORR_NSAMP;
    const bool pos0 = -tau > 0.0;
    int klo = 0, khi = 0;
    double rhi = 0.0;
    bool have_rhi = false;
    for (int k = 1; k <= CORR_NSAMP; ++k) {
        const float L = (float)(k * STEP);
        const float r32 = ((c3 * L + c2) * L + c1) * L - tf;
        const float B = ((a3 * L + a2) * L + a1) * L + at;
        bool pos;
        double rk = 0.0;
        const bool sure = fabsf(r32) > 1e-6f * B;
        if (sure) {
            pos = r32 > 0.0f;
        } else {
            rk = cubic_at(q, k * STEP) - tau;
            ++nev;
            if (rk == 0.0) return k * STEP;
            pos = rk > 0.0;
        }
        if (pos != pos0) {
            khi = k;
            rhi = rk;
            have_rhi = !sure;
            break;
        }
        klo = k;
    }
    if (khi == 0) return -1.0;
    double lo = klo * STEP, hi = khi * STEP;
    double rlo = klo == 0 ? -tau : cubic_at(q, lo) - tau;
    nev += klo != 0;
    if (!have_rhi) {
        rhi = cubic_at(q, hi) - tau;
        ++nev;
        if (rhi == 0.0) return hi;
    }
    double x = lo - rlo * (hi - lo) / (rhi - rlo);
    if (!(x > lo && x < hi)) x = 0.5 * (lo + hi);
    while (its < CORR_MAXIT) {
        double r = cubic_at(q, x) - tau;
        ++nev;
        double ax = fabs(x);
        double scale = fmax(fabs(tau), ((q.s3 * ax + q.s2) * ax + q.s1) * ax);
        ++its;
        if ((r > 0) == (rhi > 0)) { hi = x; rhi = r; } else { lo = x; rlo = r; }
        if (fabs(r) <= CORR_TOL * scale) break;
        if (hi - lo <= 1e-15 * hi) break;
        double dr = (3.0 * q.c3 * x + 2.0 * q.c2) * x + q.c1;
        double xn = x - r * (double)__frcp_rn((float)dr);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        x = xn;
    }
    return x;
}

__global__ void k_flux_polyhedra(DevMesh m, const double *__restrict__ Up, const double *F,
                                 const double *lambda, double dt, double *V)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.nf) return;
    V3 A[VOF_MAXFP], W[VOF_MAXFP];
    int id[VOF_MAXFP];
    int n = face_points<false>(m, f, Up, dt, A, W, id);
    double lam = lambda ? lambda[f] : 1.0;
    if (lam < 0.0) {  // normal sweep: uniform translation along S_f
        V3 S = ld3(m.sf, m.nf, f);
        V3 wn = S * (-lam * F[f] * dt / dot(S, S));
        for (int i = 0; i < n; ++i) W[i] = wn;
        lam = 1.0;
    }
    Cubic q = face_cubic(m, f, n, A, W, id);
    V[f] = cubic_at(q, lam);
}

// The correction of one face with points b .. b+n-1 of m.fpts.  N = 3 or 4:
// the face has exactly N points and every array index is static after
// unrolling (registers); N = VOF_MAXFP: any n (local arrays).
template <int N>
__device__ __forceinline__ void correct_face(const DevMesh &m, int f, int b, int n, const double *__restrict__ U,
                                             const double *__restrict__ F, double dt, int item, double *lam_out,
                                             int *it_out, double *disp_out, int *maxit, int *nfallback,
                                             unsigned &ntri, unsigned &nev)
{
    constexpr bool FIXED = N <= 4;
    const int nn = FIXED ? N : n;
    V3 A[N], W[N];
    int id[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i < nn) {
            int p = __ldg(m.fpts + b + i);
            id[i] = __ldg(m.fkey + b + i);  // the point's index (its master's on a periodic mesh)
            A[i] = ldP(m, p);
            W[i] = ld3(U, m.np, p) * dt;
        }
    }
    const double tau = F[f] * dt;
    Cubic q = {0, 0, 0, 0, 0, 0};
    if (nn == 3) {
        prism_cubic(A[0], A[1], A[2], W[0], W[1], W[2], id[0], id[1], id[2], q);
    } else {
        V3 c = ld3(m.cf, m.nf, f), wc = mk(0, 0, 0);
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < nn) wc = wc + W[i];
        wc = wc * inv_n(nn);
#pragma unroll
        for (int t = 0; t < N; ++t) {
            if (t < nn) {
                int u = t + 1 == nn ? 0 : t + 1;
                prism_cubic(c, A[t], A[u], wc, W[t], W[u], -1, id[t], id[u], q);
            }
        }
    }
    double w2 = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i < nn) w2 = fmax(w2, dot(W[i], W[i]));
    const V3 S = ld3(m.sf, m.nf, f);
    int its = 0;
    ntri += nn == 3 ? 1 : nn;
    const double lam = solve_lambda(q, tau, dot(S, S) * w2, its, nev);
    lam_out[item] = lam;
    if (it_out) it_out[item] = its;
    if (maxit && its > 0) atomicMax(maxit, its);
    if (lam < 0.0 && nfallback) atomicAdd(nfallback, 1);
    if (disp_out) {
        double *o = disp_out + (size_t)item * DISP_STRIDE;
        V3 wc = mk(0, 0, 0);
        if (lam < 0.0) {
            wc = S * (-lam * F[f] * dt / dot(S, S));
#pragma unroll
            for (int i = 0; i < N; ++i) W[i] = wc;
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i)
                if (i < nn) { W[i] = W[i] * lam; wc = wc + W[i]; }
            wc = wc * inv_n(nn);
        }
        o[0] = wc.x; o[1] = wc.y; o[2] = wc.z;
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < nn) { o[3 + 3 * i] = W[i].x; o[4 + 3 * i] = W[i].y; o[5 + 3 * i] = W[i].z; }
    }
}

// One thread per face (LIST: per band slot).  U holds the point velocities.
template <bool LIST>
__global__ void k_correct(DevMesh m, const double *__restrict__ U, const double *__restrict__ F,
                          double dt, const int *list, const int *count, double *lam_out,
                          int *it_out, double *disp_out, int *maxit, int *nfallback, unsigned long long *work)
{
    const int total = LIST ? *count : m.nf;
    unsigned ntri = 0, nev = 0;  // FP64 work: cubic coefficient triangles, cubic evaluations
    for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < total; item += gridDim.x * blockDim.x) {
        const int f = LIST ? list[item] : item;
        const int b = __ldg(m.fptr + f), n = __ldg(m.fptr + f + 1) - b;
        if (n == 4)
            correct_face<4>(m, f, b, n, U, F, dt, item, lam_out, it_out, disp_out, maxit, nfallback, ntri, nev);
        else if (n == 3)
            correct_face<3>(m, f, b, n, U, F, dt, item, lam_out, it_out, disp_out, maxit, nfallback, ntri, nev);
        else
            correct_face<VOF_MAXFP>(m, f, b, n, U, F, dt, item, lam_out, it_out, disp_out, maxit, nfallback, ntri,
                                    nev);
    }
    ntri = __reduce_add_sync(0xffffffffu, ntri);
    nev = __reduce_add_sync(0xffffffffu, nev);
    if ((threadIdx.x & 31) == 0) {
        work_add1(work, WK_CTRI, ntri);
        work_add1(work, WK_CEVAL, nev);
    }
}

// Point velocities (Eq. 4 weights, wall projection) of the points of this
// step's band faces, flagged by the classification; each point once, and the
// flag cleared for the next step.
__global__ void k_band_point_velocity(DevMesh m, const double *__restrict__ Uc, uint8_t *flag, double *Up)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m.np; p += gridDim.x * blockDim.x) {
        if (!flag[p]) continue;
        flag[p] = 0;
        st3(Up, m.np, p, point_velocity(m, p, Uc));
    }
}

// ========================================================= phase flux (A6)
struct Tet { V3 v[4]; };

// |T ^ {n_k.x <= d_k, k < np}| by depth-first splitting of T into the
// tetrahedra of its inside parts (1 or 3 per plane); the last plane is applied
// with the closed-form cut fraction.  Bounded stack: 1 + 2(np-1) entries.
__device__ double clip_tet(const Tet &T, const V3 *pn, const double *pd, int np, unsigned *status, WkOn &wk)
{
    wk.add(WK_VOL, 1);
    if (np == 0) return fabs(tvol(T.v[0], T.v[1], T.v[2], T.v[3]));
    Tet st[CLIP_STACK];
    unsigned char lv[CLIP_STACK];
    int sp = 1;
    st[0] = T;
    lv[0] = 0;
    double vol = 0.0;
    while (sp > 0) {
        --sp;
        Tet t = st[sp];
        int k = lv[sp];
        double s[4];
        int nin = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) { s[i] = dot(pn[k], t.v[i]) - pd[k]; nin += s[i] <= 0.0; }
        wk.add(WK_TEST, 1);
        if (nin == 0) continue;
        if (nin == 4) {
            if (k + 1 == np) { vol += fabs(tvol(t.v[0], t.v[1], t.v[2], t.v[3])); wk.add(WK_VOL, 1); }
            else if (sp < CLIP_STACK) { st[sp] = t; lv[sp] = k + 1; ++sp; }
            else atomicOr(status, VOF_ST_CLIP_OVERFLOW);
            continue;
        }
        if (k + 1 == np) {
            wk.add(WK_VOL, 1);
            wk.add(WK_FRAC, 1);
            double h0 = s[0], h1 = s[1], h2 = s[2], h3 = s[3];
            sort4(h0, h1, h2, h3);
            vol += fabs(tvol(t.v[0], t.v[1], t.v[2], t.v[3])) * frac_below(h0, h1, h2, h3, 0.0);
            continue;
        }
        // order vertices: inside ones first
        int ord[4], a = 0, b = 3;
#pragma unroll
        for (int i = 0; i < 4; ++i) { if (s[i] <= 0.0) ord[a++] = i; else ord[b--] = i; }
        V3 P[4];
        double S[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { P[i] = t.v[ord[i]]; S[i] = s[ord[i]]; }
        // point on edge (inside i, outside o), interpolated from the inside end
        auto ep = [&](int i, int o) { return P[i] + (P[o] - P[i]) * (S[i] / (S[i] - S[o])); };
        Tet out[3];
        int nout;
        if (nin == 1) {
            out[0] = Tet{{P[0], ep(0, 1), ep(0, 2), ep(0, 3)}};
            nout = 1;
        } else if (nin == 2) {
            // wedge (P0, p02, p03) -> (P1, p12, p13)
            V3 a0 = P[0], a1 = ep(0, 2), a2 = ep(0, 3), b0 = P[1], b1 = ep(1, 2), b2 = ep(1, 3);
            out[0] = Tet{{a0, a1, a2, b2}};
            out[1] = Tet{{a0, a1, b2, b1}};
            out[2] = Tet{{a0, b0, b1, b2}};
            nout = 3;
        } else {
            // prism (P0, P1, P2) -> (p03, p13, p23)
            V3 a0 = P[0], a1 = P[1], a2 = P[2], b0 = ep(0, 3), b1 = ep(1, 3), b2 = ep(2, 3);
            out[0] = Tet{{a0, a1, a2, b2}};
            out[1] = Tet{{a0, a1, b2, b1}};
            out[2] = Tet{{a0, b0, b1, b2}};
            nout = 3;
        }
        wk.add(WK_EDGE, nin == 2 ? 4 : 3);
        for (int i = 0; i < nout; ++i) {
            if (sp < CLIP_STACK) { st[sp] = out[i]; lv[sp] = k + 1; ++sp; }
            else atomicOr(status, VOF_ST_CLIP_OVERFLOW);
        }
    }
    return vol;
}

// ============================================================ update (A7)
constexpr int UPD_THREADS = 256;
constexpr int UPD_BLOCKS = 1024;
// partial layout per block: [mass_before, mass_after, min, max, boundary_out]

__device__ __forceinline__ void block_reduce5(double v[5], double *out)
{
    __shared__ double sh[5][UPD_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        v[1] += __shfl_xor_sync(0xffffffffu, v[1], o);
        v[2] = fmin(v[2], __shfl_xor_sync(0xffffffffu, v[2], o));
        v[3] = fmax(v[3], __shfl_xor_sync(0xffffffffu, v[3], o));
        v[4] += __shfl_xor_sync(0xffffffffu, v[4], o);
    }
    if (lane == 0) for (int i = 0; i < 5; ++i) sh[i][w] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[5] = {0.0, 0.0, 1e300, -1e300, 0.0};
        for (int k = 0; k < UPD_THREADS / 32; ++k) {
            r[0] += sh[0][k]; r[1] += sh[1][k];
            r[2] = fmin(r[2], sh[2][k]); r[3] = fmax(r[3], sh[3][k]);
            r[4] += sh[4][k];
        }
        for (int i = 0; i < 5; ++i) out[i] = r[i];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(UPD_THREADS) k_update(DevMesh m, double *alpha, const double *__restrict__ Va,
                                                        double *partial, int *viol, int *nviol, int cap,
                                                        unsigned *status)
{
    double v[5] = {0.0, 0.0, 1e300, -1e300, 0.0};
    bool zero = false;
    const int nb = m.nf - m.ni;
    const int stride = gridDim.x * blockDim.x;
    const int lim = m.nc > nb ? m.nc : nb;
    for (int i0 = blockIdx.x * blockDim.x; i0 < lim; i0 += stride) {
        int c = i0 + threadIdx.x;
        bool bad = false;
        if (c < m.nc) {
            // A cell whose face fluxes are all zero (the bulk of either phase
            // away from the band) has s = +0; the FP64 sum runs only where some
            // flux is not zero, so warps of such cells issue no FP64 adds.
            const int k0 = m.cptr[c], k1 = m.cptr[c + 1];
            unsigned nz = 0;
            // (cflux: the cell's faces, a periodic copy read as its face seen
            // from the neighbour; the cell's own faces on other meshes)
#pragma unroll 4
            for (int k = k0; k < k1; ++k) {
                DBits b = dbits(Va[m.cflux[k] >> 1]);
                nz |= (unsigned)(b.hi & 0x7fffffff) | b.lo;
            }
            double s = 0.0;
            if (nz)
                for (int k = k0; k < k1; ++k) {
                    int code = m.cflux[k];
                    double x = Va[code >> 1];
                    s += (code & 1) ? -x : x;
                }
            double a0 = alpha[c];
            if (is_zero(s) && is_pzero(a0)) {
                zero = true;  // an empty cell with no flux: alpha stays +0
            } else {
                double V = m.vc[c];
                double a1 = a0 - s / V;
                alpha[c] = a1;
                v[0] += V * a0;
                v[1] += V * a1;
                v[2] = fmin(v[2], a1);
                v[3] = fmax(v[3], a1);
                bad = gt_pos(a1, 1.0 + BOUND_TOL) || lt_neg(a1, BOUND_TOL);
            }
        }
        if (c < nb) v[4] += Va[m.ni + c];
        if (viol) warp_append(bad, c, viol, nviol, cap, status);
    }
    if (zero) {
        v[2] = fmin(v[2], 0.0);
        v[3] = fmax(v[3], 0.0);
    }
    block_reduce5(v, partial + 5 * blockIdx.x);
}

// final reduction of the per-block partials into stats: one block, each thread
// folds a fixed strided subset, then a fixed tree (deterministic)
constexpr int ST_THREADS = 256;

__device__ __forceinline__ void fold5(double *r, const double *p)
{
    r[0] += p[0]; r[1] += p[1]; r[2] = fmin(r[2], p[2]); r[3] = fmax(r[3], p[3]); r[4] += p[4];
}

// called by every thread of a block of ST_THREADS threads
__device__ void stats_block(const double *partial, int nblk, const int *counters, double *stats, int post,
                            const double *bound_partial, int nblk_post)
{
    __shared__ double sh[2][5][ST_THREADS];
    double r[5] = {0.0, 0.0, 1e300, -1e300, 0.0}, q[5] = {0.0, 0.0, 1e300, -1e300, 0.0};
    for (int k = threadIdx.x; k < nblk; k += ST_THREADS) fold5(r, partial + 5 * k);
    if (post)
        for (int k = threadIdx.x; k < nblk_post; k += ST_THREADS) fold5(q, bound_partial + 5 * k);
    for (int i = 0; i < 5; ++i) { sh[0][i][threadIdx.x] = r[i]; sh[1][i][threadIdx.x] = q[i]; }
    __syncthreads();
    for (int w = ST_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            for (int t = 0; t < 2; ++t) {
                double a[5], b2[5];
                for (int i = 0; i < 5; ++i) { a[i] = sh[t][i][threadIdx.x]; b2[i] = sh[t][i][threadIdx.x + w]; }
                fold5(a, b2);
                for (int i = 0; i < 5; ++i) sh[t][i][threadIdx.x] = a[i];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    stats[VOF_S_MASS_BEFORE] = sh[0][0][0];
    stats[VOF_S_MIN_PRE] = sh[0][2][0];
    stats[VOF_S_MAX_PRE] = sh[0][3][0];
    stats[VOF_S_BOUNDARY_OUT] = sh[0][4][0];
    const int t = post ? 1 : 0;
    stats[VOF_S_MASS_AFTER] = sh[t][1][0];
    stats[VOF_S_MIN_POST] = sh[t][2][0];
    stats[VOF_S_MAX_POST] = sh[t][3][0];
    if (counters) {
        stats[VOF_S_N_INTERFACE] = counters[CNT_ICELL];
        stats[VOF_S_N_BAND] = counters[CNT_BAND];
        stats[VOF_S_MAX_POS_IT] = counters[CNT_MAXPOS];
        stats[VOF_S_MAX_CORR_IT] = counters[CNT_MAXCORR];
        stats[VOF_S_N_FALLBACK] = counters[CNT_FALLBACK];
        stats[VOF_S_N_BOUND_SOURCES] = counters[CNT_VIOL0];
        stats[VOF_S_N_BOUND_LEFT] = counters[CNT_VIOL1];
    }
    if (!post) stats[VOF_S_BOUND_PASSES] = stats[VOF_S_BOUND_GLOBAL] = 0.0;
}

__global__ void __launch_bounds__(ST_THREADS) k_stats(const double *partial, int nblk, const int *counters,
                                                      double *stats, int post, const double *bound_partial,
                                                      int nblk_post)
{
    stats_block(partial, nblk, counters, stats, post, bound_partial, nblk_post);
}

// ------------------------------------------ redistribution passes (reading R10)
// Sec. 2.3's wisp redistribution, read as passes of a local redistribution:
// a source (alpha > 1 + tol: excess e = (alpha - 1) V; alpha < -tol: deficit
// u = -alpha V) asks each face neighbour r for e w_r / W, where the receiver
// weight w = alpha (1 - alpha) V of an interface cell (tol < alpha < 1 - tol;
// 0 elsewhere, so no bulk cell receives and no wisp is made) and W the sum
// over the source's neighbours; a receiver takes at most its room, (1 - alpha)
// V for excess and alpha V for deficit, and scales all requests to fit, so it
// never leaves [0, 1]; what a source could not place stays with it for the
// next pass.  Passes run while some source has both something left and a
// receiver with room.  Every touched cell's new value is a gather over its
// face neighbours in face order.
// Face neighbours of x in face order, handed to fn(s, k) (s the neighbour, k
// its cface slot).  The indices of a chunk of up to BP_CHUNK neighbours are
// loaded together, and fn's own loads across the unrolled chunk can issue
// together too: a few dependent load rounds per chunk instead of a chain per
// neighbour.
constexpr int BP_CHUNK = 8;
template <class Fn>
__device__ __forceinline__ void for_nbrs(const DevMesh &m, int x, Fn fn)
{
    const int k0 = m.cptr[x], k1 = m.cptr[x + 1];
    for (int kb = k0; kb < k1; kb += BP_CHUNK) {
        int nb[BP_CHUNK];
#pragma unroll
        for (int j = 0; j < BP_CHUNK; ++j) nb[j] = kb + j < k1 ? m.cnb[kb + j] : -1;
#pragma unroll
        for (int j = 0; j < BP_CHUNK; ++j)
            if (nb[j] >= 0) fn(nb[j], kb + j);
    }
}
__device__ __forceinline__ bool is_exc(double a) { return a > 1.0 + BOUND_TOL; }
__device__ __forceinline__ bool is_def(double a) { return a < -BOUND_TOL; }
__device__ __forceinline__ double recv_w(double a, double V)
{
    return (a > BOUND_TOL && a < 1.0 - BOUND_TOL) ? a * (1.0 - a) * V : 0.0;
}

// scratch per cell: [1/W (0 where the source has no receiver), receiver
// scales sp, sm]
enum { BS_RW = 0, BS_SP, BS_SM, BS_N = 3 };

struct BoundBufs {
    int *la;             // source list (from the update kernel), capacity nc
    const int *n0;       // its count
    int *pc;             // pending cells, capacity cap_pend
    double *pa;          // pending values
    double *bs;          // BS_N doubles per cell
    int *npass;          // out: passes that moved something
    int *act;            // two counters of active sources (pass parity)
    int cap, cap_pend;
};


// lowest-index source among x's face neighbours (and x itself if self)
__device__ __forceinline__ int first_source(const DevMesh &m, const double *alpha, int x, bool self)
{
    int first = 0x7fffffff;
    if (self) {
        double ax = alpha[x];
        if (is_exc(ax) || is_def(ax)) first = x;
    }
    for_nbrs(m, x, [&](int s, int) {
        double as = alpha[s];
        if ((is_exc(as) || is_def(as)) && s < first) first = s;
    });
    return first;
}

// One pass as three phases over the source list (count on the device): the
// receiver weight around each source, receiver scales, new values (a source's
// own placement summed where its new value is formed), then apply; t0 / nt:
// this thread's index and the thread count of the grid.
// A source with something left and a receiver is counted in *act.
__device__ __forceinline__ void bp_room(const DevMesh &m, const double *alpha, const BoundBufs &b, int *act, long t0, long nt)
{
    const int n = min(*b.n0, b.cap);
    int active = 0;
    for (long i = t0; i < n; i += nt) {
        int c = b.la[i];
        const double a = alpha[c];
        double W = 0.0;
        if (is_exc(a) || is_def(a))
            for_nbrs(m, c, [&](int nb, int) { W += recv_w(alpha[nb], m.vc[nb]); });
        b.bs[BS_N * (size_t)c + BS_RW] = W > 0.0 ? 1.0 / W : 0.0;
        active += W > 0.0;
    }
    if (active) atomicAdd(act, active);
}

// one thread per (source, face slot): slot j takes the faces j, j + BP_SLOTS, ...
constexpr int BP_SLOTS = 8;

__device__ __forceinline__ void bp_scale(const DevMesh &m, const double *alpha, const BoundBufs &b, long t0, long nt)
{
    const long n = min(*b.n0, b.cap);
    double *bs = b.bs;
    for (long t = t0; t < n * BP_SLOTS; t += nt) {
        int c = b.la[t / BP_SLOTS];
        for (int k = m.cptr[c] + (int)(t % BP_SLOTS); k < m.cptr[c + 1]; k += BP_SLOTS) {
            int r = m.cnb[k];
            if (r < 0 || first_source(m, alpha, r, false) != c) continue;
            const double ar = alpha[r], Vr = m.vc[r], wr = recv_w(ar, Vr);
            const double Rp = wr > 0.0 ? (1.0 - ar) * Vr : 0.0, Rm = wr > 0.0 ? ar * Vr : 0.0;
            double Qp = 0.0, Qm = 0.0;
            if (wr > 0.0)
                for_nbrs(m, r, [&](int s, int) {
                    const double as = alpha[s], rW = bs[BS_N * (size_t)s + BS_RW];
                    if (rW > 0.0) {
                        if (is_exc(as)) Qp += (as - 1.0) * m.vc[s] * (wr * rW);
                        else if (is_def(as)) Qm += -as * m.vc[s] * (wr * rW);
                    }
                });
            bs[BS_N * (size_t)r + BS_SP] = Qp > Rp ? Rp / Qp : 1.0;
            bs[BS_N * (size_t)r + BS_SM] = Qm > Rm ? Rm / Qm : 1.0;
        }
    }
}

// new values of the sources and their neighbours, each cell once: by the
// lowest-index source in its closed face neighbourhood
__device__ __forceinline__ void bp_new(const DevMesh &m, const double *alpha, const BoundBufs &b, int *npend, unsigned *status,
                       long t0, long nt)
{
    const long n = min(*b.n0, b.cap);
    const double *bs = b.bs;
    for (long t = t0; t < n * BP_SLOTS; t += nt) {
        int c = b.la[t / BP_SLOTS];
        // slot 0 takes the source itself (k = cptr[c] - 1)
        for (int k = m.cptr[c] - 1 + (int)(t % BP_SLOTS); k < m.cptr[c + 1]; k += BP_SLOTS) {
            int x = k < m.cptr[c] ? c : m.cnb[k];
            if (x < 0 || first_source(m, alpha, x, true) != c) continue;
            const double ax = alpha[x], V = m.vc[x], wx = recv_w(ax, V);
            double dV = 0.0;
            const bool xe = is_exc(ax);
            if (xe || is_def(ax)) {
                // a source: what it places in its receivers (each scaled to fit)
                const double rWx = bs[BS_N * (size_t)x + BS_RW];
                if (rWx > 0.0) {
                    const double e = xe ? (ax - 1.0) * V : -ax * V;
                    double g = 0.0;
                    for_nbrs(m, x, [&](int nb, int) {
                        const double w = recv_w(alpha[nb], m.vc[nb]);
                        if (w > 0.0) g += e * (w * rWx) * bs[BS_N * (size_t)nb + (xe ? BS_SP : BS_SM)];
                    });
                    dV += xe ? -g : g;
                }
            } else if (wx > 0.0) {
                // a receiver: what its source neighbours place in it
                const double SPx = bs[BS_N * (size_t)x + BS_SP], SMx = bs[BS_N * (size_t)x + BS_SM];
                for_nbrs(m, x, [&](int s, int) {
                    const double as = alpha[s], rW = bs[BS_N * (size_t)s + BS_RW];
                    if (rW > 0.0) {
                        if (is_exc(as)) dV += (as - 1.0) * m.vc[s] * (wx * rW) * SPx;
                        else if (is_def(as)) dV -= -as * m.vc[s] * (wx * rW) * SMx;
                    }
                });
            }
            if (dV != 0.0) {
                int pos = atomicAdd(npend, 1);
                if (pos < b.cap_pend) { b.pc[pos] = x; b.pa[pos] = (ax * V + dV) / V; }
                else atomicOr(status, VOF_ST_CAPACITY);
            }
        }
    }
}

__device__ __forceinline__ void bp_apply(double *alpha, const int *pc, const double *pa, const int *npend, int cap, long t0, long nt)
{
    const int n = min(*npend, cap);
    for (long i = t0; i < n; i += nt) alpha[pc[i]] = pa[i];
}

// Global fallback for what the local passes leave (a source none of whose face
// neighbours is an interface cell with room): the total excess (deficit) of a
// region (the whole mesh, or one case of a batch) goes to every cell of that
// region strictly inside (tol, 1-tol) in proportion to its free (phase)
// volume; sources are set to 1 (0).  A region's cells are contiguous and cut
// into segments; one block sums a segment, then one warp per region sums its
// segments in order (deterministic).
constexpr int GB_THREADS = 256;

// one segment, by a whole block of GB_THREADS threads
// A thread takes the cells c, c + blockDim.x, ... of the segment in order; the
// loads of SEG_UNROLL consecutive ones of its cells are issued together.
constexpr int SEG_UNROLL = 4;
__device__ void seg_reduce(const DevMesh &m, const double *alpha, int4 sg, double *spartial, int *nleft)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};  // Ep, Em, Sp, Sm
    int left = 0;
    auto cell = [&](int c, double a) {
        if (gt_pos(a, 1.0 + BOUND_TOL)) { v[0] += (a - 1.0) * m.vc[c]; ++left; }
        else if (lt_neg(a, BOUND_TOL)) { v[1] += -a * m.vc[c]; ++left; }
        else if (gt_pos(a, BOUND_TOL) && lt_pos(a, 1.0 - BOUND_TOL)) {
            double V = m.vc[c];
            v[2] += (1.0 - a) * V;
            v[3] += a * V;
        }
    };
    const int step = blockDim.x;
    int c = sg.y + threadIdx.x;
    for (; c + (SEG_UNROLL - 1) * step < sg.z; c += SEG_UNROLL * step) {
        double a[SEG_UNROLL];
#pragma unroll
        for (int u = 0; u < SEG_UNROLL; ++u) a[u] = alpha[c + u * step];
#pragma unroll
        for (int u = 0; u < SEG_UNROLL; ++u) cell(c + u * step, a[u]);
    }
    for (; c < sg.z; c += step) cell(c, alpha[c]);
    left = __reduce_add_sync(0xffffffffu, left);
    if ((threadIdx.x & 31) == 0 && left) atomicAdd(nleft, left);
    __shared__ double sh[4][GB_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = 0; i < 4; ++i) {
        double x = warp_sum(v[i]);
        if (lane == 0) sh[i][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 0; i < 4; ++i) {
            double r = 0.0;
            for (int k = 0; k < GB_THREADS / 32; ++k) r += sh[i][k];
            spartial[i] = r;
        }
    __syncthreads();
}

// region r, by a whole warp: totals[REG_TOT * r + 0..3] = Ep, Em, Sp, Sm and
// [4], [5] the shares Ep / Sp, Em / Sm of the global step (0 where none)
constexpr int REG_TOT = 6;
__device__ void region_totals(const int *reg_seg, int r, const double *spartial, double *totals)
{
    const int lane = threadIdx.x & 31;
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = reg_seg[r] + lane; k < reg_seg[r + 1]; k += 32)
        for (int i = 0; i < 4; ++i) t[i] += spartial[4 * k + i];
    for (int i = 0; i < 4; ++i) t[i] = warp_sum(t[i]);
    if (lane == 0) {
        double *o = totals + REG_TOT * (size_t)r;
        for (int i = 0; i < 4; ++i) o[i] = t[i];
        o[4] = t[0] > 0.0 && t[2] > 0.0 ? t[0] / t[2] : 0.0;
        o[5] = t[1] > 0.0 && t[3] > 0.0 ? t[1] / t[3] : 0.0;
    }
}

// one segment, by a whole block: the global step where its region needs one,
// then the segment's share of the post-bounding mass and extrema (v as in the
// update partials; +0 cells add nothing to the mass and set 'zero')
__device__ void seg_apply(const DevMesh &m, double *alpha, int4 sg, const double *totals, double v[5], bool &zero,
                          bool &bad)
{
    const double *tt = totals + REG_TOT * (size_t)sg.x;
    const double Ep = tt[0], Em = tt[1], Sp = tt[2], Sm = tt[3], sp = tt[4], sm = tt[5];
    const bool apply = !((Ep == 0.0 && Em == 0.0) || Ep > Sp || Em > Sm);
    auto cell = [&](int c, double a) {
        if (apply) {
            // a cell strictly inside takes Ep (1 - a) V / Sp and gives Em a V / Sm:
            // a + (Ep / Sp)(1 - a) - (Em / Sm) a, no division per cell
            if (gt_pos(a, 1.0 + BOUND_TOL)) alpha[c] = a = 1.0;
            else if (lt_neg(a, BOUND_TOL)) alpha[c] = a = 0.0;
            else if (gt_pos(a, BOUND_TOL) && lt_pos(a, 1.0 - BOUND_TOL)) alpha[c] = a = a + sp * (1.0 - a) - sm * a;
        }
        if (is_pzero(a)) { zero = true; return; }
        v[1] += m.vc[c] * a;
        v[2] = fmin(v[2], a);
        v[3] = fmax(v[3], a);
        bad |= gt_pos(a, 1.0 + BOUND_FLAG) || lt_neg(a, BOUND_FLAG);
    };
    const int step = blockDim.x;
    int c = sg.y + threadIdx.x;
    for (; c + (SEG_UNROLL - 1) * step < sg.z; c += SEG_UNROLL * step) {
        double a[SEG_UNROLL];
#pragma unroll
        for (int u = 0; u < SEG_UNROLL; ++u) a[u] = alpha[c + u * step];
#pragma unroll
        for (int u = 0; u < SEG_UNROLL; ++u) cell(c + u * step, a[u]);
    }
    for (; c < sg.z; c += step) cell(c, alpha[c]);
}

// Grid-wide barrier of a cooperative launch (every block resident): a block
// arrives on the count; the last to arrive resets it and advances the generation
// gen, which the others poll with a growing pause (count and generation sit
// on separate cache lines, so the polls do not hold up the arrivals).  A wait
// gives up after `limit` polls (BAR_SPIN_LIMIT: seconds) and flags VOF_ST_TIMEOUT;
// grid_sync then returns false in every thread of the block, which leaves the
// kernel (the blocks still waiting give up the same way: every wait ends).
constexpr long BAR_SPIN_LIMIT = 4000000;
__device__ bool grid_sync(unsigned *count, unsigned *generation, unsigned *status, long limit = BAR_SPIN_LIMIT)
{
    __shared__ int gave_up;
    __syncthreads();
    if (threadIdx.x == 0) {
        gave_up = 0;
        volatile unsigned *gen = generation;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(generation, 1u);
        } else {
            long it = 0;
            unsigned pause = 32;
            while (*gen == g) {
                if (++it > limit) {
                    atomicOr(status, VOF_ST_TIMEOUT);
                    gave_up = 1;
                    break;
                }
                __nanosleep(pause);
                if (pause < 1024) pause <<= 1;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return !gave_up;
}

// The whole redistribution, the post-bounding mass and the step statistics in
// one cooperative launch, a grid barrier between the phases: passes of the
// local redistribution (weights, scales, new values, apply) while
// some source has something left and a receiver, segment sums, region totals,
// global fallback with the mass partials, statistics (block 0).
struct BoundStep {
    double *alpha;
    BoundBufs b;
    int *npend;
    const int4 *seg;
    int nseg;
    double *gpartial;            // 4 per segment
    int *nleft;
    const int *reg_seg;
    int nreg;
    double *reg_tot;
    double *mpartial;            // 5 per block: post-bounding mass, extrema
    const double *upartial;      // the update kernel's partials
    int nupd;
    const int *counters;         // or null: no counter statistics
    double *stats;
    unsigned *bar_count;         // grid barrier: arrivals (zero before the launch)
    unsigned *bar_gen;           // and generation (any value)
    unsigned *status;
};

constexpr int BA_THREADS = 256;
static_assert(BA_THREADS == GB_THREADS && BA_THREADS == UPD_THREADS && BA_THREADS == ST_THREADS,
              "the phases share one block shape");

__global__ void __launch_bounds__(BA_THREADS, 4) k_bound_step(DevMesh m, BoundStep a)
{
    const long t0 = blockIdx.x * (long)blockDim.x + threadIdx.x, nt = (long)gridDim.x * blockDim.x;
    // the passes have few items (sources x slots): item i goes to block
    // i mod gridDim.x, so that they spread over every SM rather than fill the
    // first few blocks (the FP64 divisions of a phase run on all SMs' units)
    const long tl = threadIdx.x * (long)gridDim.x + blockIdx.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    // act[p & 1] counts pass p's active sources; it was zeroed by the pass
    // before (act[0] before the launch), after every block had read it
#pragma unroll 1
    for (int p = 0; p < BOUND_PASSES_MAX; ++p) {
        int *act = a.b.act + (p & 1);
        if (lead) {
            a.b.act[(p + 1) & 1] = 0;
            *a.npend = 0;  // the previous pass's apply phase is behind a barrier
        }
        bp_room(m, a.alpha, a.b, act, tl, nt);
        if (!grid_sync(a.bar_count, a.bar_gen, a.status)) return;
        if (*(volatile int *)act == 0) break;
        if (lead) *a.b.npass = p + 1;
        bp_scale(m, a.alpha, a.b, tl, nt);
        if (!grid_sync(a.bar_count, a.bar_gen, a.status)) return;
        bp_new(m, a.alpha, a.b, a.npend, a.status, tl, nt);
        if (!grid_sync(a.bar_count, a.bar_gen, a.status)) return;
        bp_apply(a.alpha, a.b.pc, a.b.pa, a.npend, a.b.cap_pend, tl, nt);
        if (!grid_sync(a.bar_count, a.bar_gen, a.status)) return;
    }
    for (int sgi = blockIdx.x; sgi < a.nseg; sgi += gridDim.x)
        seg_reduce(m, a.alpha, a.seg[sgi], a.gpartial + 4 * (size_t)sgi, a.nleft);
    if (!grid_sync(a.bar_count, a.bar_gen, a.status)) return;
    for (int r = (int)(t0 >> 5); r < a.nreg; r += (int)(nt >> 5)) region_totals(a.reg_seg, r, a.gpartial, a.reg_tot);
    if (!grid_sync(a.bar_count, a.bar_gen, a.status)) return;
    double v[5] = {0.0, 0.0, 1e300, -1e300, 0.0};
    bool zero = false, bad = false;
    for (int sgi = blockIdx.x; sgi < a.nseg; sgi += gridDim.x) seg_apply(m, a.alpha, a.seg[sgi], a.reg_tot, v, zero, bad);
    if (zero) {
        v[2] = fmin(v[2], 0.0);
        v[3] = fmax(v[3], 0.0);
    }
    if (bad) atomicOr(a.status, VOF_ST_BOUND_RESIDUAL);
    block_reduce5(v, a.mpartial + 5 * blockIdx.x);
    if (!grid_sync(a.bar_count, a.bar_gen, a.status)) return;
    if (blockIdx.x == 0) {
        stats_block(a.upartial, a.nupd, a.counters, a.stats, 1, a.mpartial, gridDim.x);
        if (threadIdx.x == 0) {
            // volume the global fallback moved (regions where it applied)
            double gv = 0.0;
            for (int r = 0; r < a.nreg; ++r) {
                const double *tt = a.reg_tot + REG_TOT * (size_t)r;
                if (!((tt[0] == 0.0 && tt[1] == 0.0) || tt[0] > tt[2] || tt[1] > tt[3])) gv += tt[0] + tt[1];
            }
            a.stats[VOF_S_BOUND_PASSES] = *(volatile int *)a.b.npass;
            a.stats[VOF_S_BOUND_GLOBAL] = gv;
        }
    }
}

// The barrier's own check (a cooperative launch): every block passes `rounds`
// barriers, except block `skip`, which leaves at once, so that the others'
// waits run out after `limit` polls and flag VOF_ST_TIMEOUT (skip < 0: none
// leaves and nothing is flagged).
__global__ void k_barrier_probe(unsigned *count, unsigned *generation, unsigned *status, int skip, int rounds,
                                long limit)
{
    if ((int)blockIdx.x == skip) return;
    for (int r = 0; r < rounds; ++r)
        if (!grid_sync(count, generation, status, limit)) return;
}

__global__ void k_zero_int(int *p, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0;
}

// the update group's counters: violations before / after the local passes,
// pending cells, passes, the first pass's active sources, and the grid
// barrier's arrival count
__global__ void k_zero_update(int *cnt)
{
    const int i = threadIdx.x;
    if (i < 3) cnt[CNT_VIOL0 + i] = 0;
    if (i == 3) cnt[CNT_BAR] = 0;
    if (i == 4) cnt[CNT_BPASS] = 0;
    if (i == 5) cnt[CNT_BACT0] = 0;
}

// ============================================== band classification (A2, R9)
// per point: all cells empty (bit 0) / all full (bit 1); for the other points
// (every point of an interface cell is one) the IDW point value of Eq.
// idwpointphi, in the order the reconstruction would sum it
__global__ void k_point_state(DevMesh m, const double *__restrict__ alpha, uint8_t *state, double *palpha)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m.np) return;
    bool all_e = true, all_f = true;
    const double full = 1.0 - m.eps;
    const int j0 = m.pptr[p], j1 = m.pptr[p + 1];
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        double a = __ldg(alpha + m.pcell[j]);
        all_e &= le_pos(a, m.eps);
        all_f &= ge_pos(a, full);
    }
    state[p] = (all_e ? 1 : 0) | (all_f ? 2 : 0);
    if (!all_e && !all_f) {
        double ap = 0.0;
        for (int j = j0; j < j1; ++j) ap += __ldg(m.pw + j) * __ldg(alpha + m.pcell[j]);
        palpha[p] = ap;
    }
}

__global__ void k_classify(DevMesh m, const double *__restrict__ alpha, const double *__restrict__ F,
                           double dt, const uint8_t *__restrict__ state, double *Va, int *band, int *nband,
                           int *icell, int *nicell, uint8_t *bpflag, unsigned *status)
{
    const int lim = m.nf > m.nc ? m.nf : m.nc;
    for (int i0 = blockIdx.x * blockDim.x; i0 < lim; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + threadIdx.x;
        bool isband = false, isint = false;
        if (i < m.nf) {
            double Ff = F[i];
            double v = 0.0;
            // (a periodic face's copy carries no flux)
            if (!is_zero(Ff) && !(i >= m.ni && (dbits(Ff).hi < 0 || (m.fimg && m.fimg[i - m.ni] >= 0)))) {
                unsigned st = 3u;
#pragma unroll 4
                for (int k = m.fptr[i]; k < m.fptr[i + 1]; ++k) st &= state[m.fpts[k]];
                if (st & 1u) v = 0.0;
                else if (st & 2u) v = Ff * dt;
                else {
                    isband = true;
                    for (int k = m.fptr[i]; k < m.fptr[i + 1]; ++k) bpflag[m.fpts[k]] = 1;
                }
            }
            Va[i] = v;
        }
        if (i < m.nc) {
            double a = alpha[i];
            isint = gt_pos(a, m.eps) && lt_pos(a, 1.0 - m.eps);
        }
        warp_append(isband, i, band, nband, m.nf, status);
        warp_append(isint, i, icell, nicell, m.nc, status);
    }
}

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// Grid of the update kernel: the blocks resident at once (at most
// UPD_BLOCKS), so that no block of the grid-stride loop waits for a second wave.
template <class K>
int resident_blocks(K kernel, int sms)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, UPD_THREADS, 0) != cudaSuccess || occ < 1) occ = 1;
    return sms * occ < UPD_BLOCKS ? sms * occ : UPD_BLOCKS;
}

}  // namespace

// ================================================================ launchers
#define LAUNCH_CHECK()                                            \
    do {                                                          \
        cudaError_t e_ = cudaGetLastError();                      \
        if (e_ != cudaSuccess) return VOF_ERR_CUDA;               \
    } while (0)

static int g_sms = 0;
static int num_sms(int dev)
{
    if (g_sms == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_sms = v > 0 ? v : 148;
    }
    return g_sms;
}
static int g_upd_blocks = 0;
static int upd_blocks(int dev)
{
    if (g_upd_blocks == 0) g_upd_blocks = resident_blocks(k_update, num_sms(dev));
    return g_upd_blocks;
}

int launch_setup_geometry(vof_ctx *c, cudaStream_t s)
{
    DevMesh &m = c->m;
    k_face_geom<<<cdiv(m.nf, 256), 256, 0, s>>>(m, (double *)m.cf, (double *)m.sf, (double *)m.nagc);
    LAUNCH_CHECK();
    unsigned *bad = c->status;
    k_cell_geom<<<cdiv(m.nc, 256), 256, 0, s>>>(m, (double *)m.cc, (double *)m.vc, (double *)m.cbox, bad);
    LAUNCH_CHECK();
    k_point_weights<<<cdiv(m.np, 256), 256, 0, s>>>(m, (double *)m.pw);
    LAUNCH_CHECK();
    return VOF_OK;
}

int launch_wall_table(vof_ctx *c, const int *wptr, const int *wface, int nrows, cudaStream_t s)
{
    if (nrows == 0) return VOF_OK;
    k_wall_table<<<cdiv(nrows, 256), 256, 0, s>>>(c->m, wptr, wface, nrows, (double *)c->m.wallt);
    LAUNCH_CHECK();
    return VOF_OK;
}

int launch_point_velocity(vof_ctx *c, const double *Uc, double *Up, cudaStream_t s)
{
    k_point_velocity<<<cdiv(c->np, 256), 256, 0, s>>>(c->m, Uc, Up);
    LAUNCH_CHECK();
    return VOF_OK;
}

// reconstruction launch with the context's lanes per cell (8 or 32)
// ===================================== generalised LSQ gradient (Sec. 2.2.1)
// Per cell the gradient minimising sum_k w^2 (phi_k - phi_c - g.d)^2 over the
// cells k sharing a point with c (d = x_k - x_c, w = 1/|d|, the inverse
// distance of Eq. generalizedLSQminimize): the 3x3 normal equations solved by
// the adjugate of their symmetric matrix (g = 0 where it is singular).
template <bool LIST>
__global__ void k_lsq_gradient(DevMesh m, const double *__restrict__ alpha, const int *list, const int *count,
                               const int *__restrict__ lptr, const int *__restrict__ lcell,
                               const uint8_t *__restrict__ lcode, double *grad)
{
    const int total = LIST ? *count : m.nc;
    for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < total; item += gridDim.x * blockDim.x) {
        const int c = LIST ? list[item] : item;
        const V3 xc = ld3(m.cc, m.nc, c);
        const double pc = alpha[c];
        double a00 = 0, a01 = 0, a02 = 0, a11 = 0, a12 = 0, a22 = 0, b0 = 0, b1 = 0, b2 = 0;
        for (int k = __ldg(lptr + c), k1 = __ldg(lptr + c + 1); k < k1; ++k) {
            const int q = __ldg(lcell + k);
            const V3 dd = (lcode ? ld3(m.cc, m.nc, q) + tshift(m, __ldg(lcode + k)) : ld3(m.cc, m.nc, q)) - xc;
            const double w2 = 1.0 / dot(dd, dd), dp = (alpha[q] - pc) * w2;
            const V3 wd = dd * w2;
            a00 += wd.x * dd.x; a01 += wd.x * dd.y; a02 += wd.x * dd.z;
            a11 += wd.y * dd.y; a12 += wd.y * dd.z; a22 += wd.z * dd.z;
            b0 += dp * dd.x; b1 += dp * dd.y; b2 += dp * dd.z;
        }
        const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
        const double c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
        const double det = a00 * c00 + a01 * c01 + a02 * c02;
        V3 g = mk(0, 0, 0);
        if (det != 0.0) {
            const double r = 1.0 / det;
            g = mk((c00 * b0 + c01 * b1 + c02 * b2) * r, (c01 * b0 + c11 * b1 + c12 * b2) * r,
                   (c02 * b0 + c12 * b1 + c22 * b2) * r);
        }
        st3(grad, m.nc, c, g);
    }
}

int launch_lsq_gradient(vof_ctx *c, const double *alpha, const int *list, const int *count, double *grad,
                        cudaStream_t s)
{
    if (list)
        k_lsq_gradient<true><<<num_sms(c->device) * 8, 128, 0, s>>>(c->m, alpha, list, count, c->lptr, c->lcell,
                                                                    c->lcode, grad);
    else
        k_lsq_gradient<false><<<cdiv(c->nc, 128), 128, 0, s>>>(c->m, alpha, nullptr, nullptr, c->lptr, c->lcell,
                                                                c->lcode, grad);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

// ======================================= reconstruction error E_vsd (Sec. 4.1)
// The true phase is a ball (centre bc, radius R), resolved as the paper's tool
// mesh resolves a geometry: each cell tetrahedron is split into eight (edge
// midpoints; the inner octahedron about the diagonal joining the midpoints of
// edges ab and cd) down to `levels`; a piece is wholly in the ball (its four
// vertices in the closed ball), wholly outside (centroid distance less the
// largest vertex distance to the centroid at least R), or, undecided at the
// last level, cut by the plane tangent to the sphere at the point nearest its
// centroid.  A piece S with true phase P and reconstructed phase H adds
// |P| + |S ^ H| - 2 |P ^ H| (E_vsd^- + E_vsd^+).  The decisions use
// round-to-nearest operations without contraction, so that every piece is
// decided as the plain definition decides it.
constexpr int EVSD_MAX_LEVELS = 6;
constexpr int EVSD_STACK = 7 * EVSD_MAX_LEVELS + 1;

__device__ __forceinline__ V3 ev_sub(V3 a, V3 b) { return mk(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)); }
__device__ __forceinline__ double ev_d2(V3 a, V3 b)
{
    const V3 t = ev_sub(a, b);
    return __dadd_rn(__dadd_rn(__dmul_rn(t.x, t.x), __dmul_rn(t.y, t.y)), __dmul_rn(t.z, t.z));
}
__device__ __forceinline__ V3 ev_mid(V3 a, V3 b)
{
    return mk(__dmul_rn(__dadd_rn(a.x, b.x), 0.5), __dmul_rn(__dadd_rn(a.y, b.y), 0.5), __dmul_rn(__dadd_rn(a.z, b.z), 0.5));
}

struct EvPiece { V3 v[4]; int lev; };

__device__ double evsd_tet(const Tet &T0, int levels, V3 bc, double R, int hmode, V3 hn, double hd, unsigned *status)
{
    WkOn wk;  // counts nothing here; clip_tet's bookkeeping
    EvPiece st[EVSD_STACK];
    int sp = 0;
    st[sp++] = EvPiece{{T0.v[0], T0.v[1], T0.v[2], T0.v[3]}, 0};
    const double R2 = __dmul_rn(R, R);
    double e = 0.0;
    while (sp > 0) {
        const EvPiece q = st[--sp];
        const V3 a = q.v[0], b = q.v[1], c = q.v[2], d = q.v[3];
        const V3 g = mk(__dmul_rn(__dadd_rn(__dadd_rn(a.x, b.x), __dadd_rn(c.x, d.x)), 0.25),
                        __dmul_rn(__dadd_rn(__dadd_rn(a.y, b.y), __dadd_rn(c.y, d.y)), 0.25),
                        __dmul_rn(__dadd_rn(__dadd_rn(a.z, b.z), __dadd_rn(c.z, d.z)), 0.25));
        const bool inside = ev_d2(a, bc) <= R2 && ev_d2(b, bc) <= R2 && ev_d2(c, bc) <= R2 && ev_d2(d, bc) <= R2;
        double rt = sqrt(ev_d2(a, g));
        rt = fmax(rt, sqrt(ev_d2(b, g)));
        rt = fmax(rt, sqrt(ev_d2(c, g)));
        rt = fmax(rt, sqrt(ev_d2(d, g)));
        const double dist = sqrt(ev_d2(g, bc));
        const Tet S{{a, b, c, d}};
        const bool outside = !inside && __dsub_rn(dist, rt) >= R;
        if (inside || outside || q.lev >= levels) {
            const double vS = fabs(tvol(a, b, c, d));
            const double SH = hmode == 0 ? 0.0 : hmode == 1 ? vS : clip_tet(S, &hn, &hd, 1, status, wk);
            if (inside) { e += vS - SH; continue; }
            if (outside) { e += SH; continue; }
            V3 pn[2];
            double pd[2];
            const V3 u = dist > 0.0 ? (g - bc) * (1.0 / dist) : mk(1, 0, 0);
            pn[0] = u; pd[0] = dot(u, bc) + R;
            const double P = clip_tet(S, pn, pd, 1, status, wk);
            double PH = 0.0;
            if (hmode == 1) PH = P;
            else if (hmode == 2) { pn[1] = hn; pd[1] = hd; PH = clip_tet(S, pn, pd, 2, status, wk); }
            e += P + SH - 2.0 * PH;
            continue;
        }
        if (sp + 8 > EVSD_STACK) { atomicOr(status, VOF_ST_CAPACITY); continue; }
        const V3 ab = ev_mid(a, b), ac = ev_mid(a, c), ad = ev_mid(a, d), bm = ev_mid(b, c), bd = ev_mid(b, d),
                 cd = ev_mid(c, d);
        const int l = q.lev + 1;
        st[sp++] = EvPiece{{a, ab, ac, ad}, l};
        st[sp++] = EvPiece{{b, ab, bm, bd}, l};
        st[sp++] = EvPiece{{c, ac, bm, cd}, l};
        st[sp++] = EvPiece{{d, ad, bd, cd}, l};
        st[sp++] = EvPiece{{ab, cd, ac, ad}, l};
        st[sp++] = EvPiece{{ab, cd, ad, bd}, l};
        st[sp++] = EvPiece{{ab, cd, bd, bm}, l};
        st[sp++] = EvPiece{{ab, cd, bm, ac}, l};
    }
    return e;
}

// one warp per cell, a lane per cell tetrahedron; the lanes' sums in a fixed order
__global__ void k_evsd(DevMesh m, const uint8_t *flags, const double *n, const double *d, double bx, double by,
                       double bz, double R, int levels, double *out, unsigned *status)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const V3 bc = mk(bx, by, bz);
    for (int c = warp; c < m.nc; c += nw) {
        int hmode = 0;
        V3 hn = mk(0, 0, 0);
        double hd = 0.0;
        if (flags) {
            const uint8_t f = flags[c];
            if (f & VOF_FULL) hmode = 1;
            else if ((f & VOF_INTERFACE) && (f & VOF_ORIENTED)) { hmode = 2; hn = ld3(n, m.nc, c); hd = d[c]; }
        }
        const V3 ctr = ld3(m.cc, m.nc, c);
        double e = 0.0;
        for (int tj = __ldg(m.ctptr + c) + lane; tj < __ldg(m.ctptr + c + 1); tj += 32) {
            const int4 te = __ldg(m.ctet + tj);
            V3 t0, t1, t2;
            if (te.w >= 0) {
                t0 = ldP(m, __ldg(m.fpts + te.y)); t1 = ldP(m, __ldg(m.fpts + te.z)); t2 = ldP(m, __ldg(m.fpts + te.w));
            } else {
                t0 = ld3(m.cf, m.nf, te.x >> 1); t1 = ldP(m, __ldg(m.fpts + te.y)); t2 = ldP(m, __ldg(m.fpts + te.z));
            }
            e += evsd_tet(Tet{{ctr, t0, t1, t2}}, levels, bc, R, hmode, hn, hd, status);
        }
        e = warp_sum(e);
        if (lane == 0) out[c] = e;
    }
}

int launch_evsd(vof_ctx *c, const uint8_t *flags, const double *n, const double *d, const double ball[4],
                int levels, double *out, cudaStream_t s)
{
    if (levels < 0 || levels > EVSD_MAX_LEVELS) return VOF_ERR_INVALID_ARG;
    k_evsd<<<num_sms(c->device) * 16, 128, 0, s>>>(c->m, flags, n, d, ball[0], ball[1], ball[2], ball[3], levels,
                                                   out, c->status);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

// ============================= geometric mapping for AMR (Sec. 3, Alg. 2)
// Per destination cell (one warp) the phase volume over its cell pairs
// (source cells sharing volume with it; nested cells): the same cell carries
// alpha_s V; a destination inside an oriented interface source takes its
// cell tetrahedra below the source's plane (lane per tetrahedron, closed-form
// cut fraction); inside any other source alpha_s V_dst; a source inside the
// destination adds alpha_s V_s.  Cells count as the same where their volumes
// agree to 1e-9.
__global__ void k_remap(DevMesh dm, const double *__restrict__ svc, int snc, const double *__restrict__ as,
                        const double *__restrict__ ns, const double *__restrict__ ds, const uint8_t *__restrict__ fs,
                        const int *__restrict__ pptr, const int *__restrict__ psrc, double *ad)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < dm.nc; c += nw) {
        const double Vc = dm.vc[c];
        const int q0 = __ldg(pptr + c), q1 = __ldg(pptr + c + 1);
        double acc = 0.0;
        if (q1 - q0 == 1) {
            const int s = __ldg(psrc + q0);
            const double Vs = svc[s], a = as[s];
            const uint8_t f = fs[s];
            if (fabs(Vc - Vs) <= 1e-9 * Vs) acc = lane == 0 ? a * Vc : 0.0;
            else if (Vc < Vs && (f & VOF_INTERFACE) && (f & VOF_ORIENTED)) {
                const V3 n = ld3(ns, snc, s);
                const double d = ds[s];
                const V3 ctr = ld3(dm.cc, dm.nc, c);
                for (int tj = __ldg(dm.ctptr + c) + lane; tj < __ldg(dm.ctptr + c + 1); tj += 32) {
                    const int4 te = __ldg(dm.ctet + tj);
                    V3 t0, t1, t2;
                    if (te.w >= 0) {
                        t0 = ldP(dm, __ldg(dm.fpts + te.y)); t1 = ldP(dm, __ldg(dm.fpts + te.z));
                        t2 = ldP(dm, __ldg(dm.fpts + te.w));
                    } else {
                        t0 = ld3(dm.cf, dm.nf, te.x >> 1); t1 = ldP(dm, __ldg(dm.fpts + te.y));
                        t2 = ldP(dm, __ldg(dm.fpts + te.z));
                    }
                    double h0 = dot(n, ctr), h1 = dot(n, t0), h2 = dot(n, t1), h3 = dot(n, t2);
                    sort4(h0, h1, h2, h3);
                    acc += fabs(tvol(ctr, t0, t1, t2)) * frac_below(h0, h1, h2, h3, d);
                }
            } else if (Vc < Vs) acc = lane == 0 ? a * Vc : 0.0;
            else acc = lane == 0 ? a * Vs : 0.0;
        } else {
            // several sources: each inside the destination (un-refined)
            for (int q = q0 + lane; q < q1; q += 32) {
                const int s = __ldg(psrc + q);
                acc += as[s] * svc[s];
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) ad[c] = acc / Vc;
    }
}

int launch_remap(vof_ctx *dst, const vof_ctx *src, const double *alpha_src, const double *n_src,
                 const double *d_src, const uint8_t *flags_src, const int *pair_ptr, const int *pair_src,
                 double *alpha_dst, cudaStream_t s)
{
    k_remap<<<num_sms(dst->device) * 16, 128, 0, s>>>(dst->m, src->m.vc, src->nc, alpha_src, n_src, d_src,
                                                       flags_src, pair_ptr, pair_src, alpha_dst);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

template <bool LIST, bool MIXED>
static void rc_launch(vof_ctx *c, int list_blocks, const double *alpha, const double *palpha, const int *list,
                      const int *count, double *n, double *d, uint8_t *flags, int *iters, int *maxit,
                      cudaStream_t s, int *next = nullptr)
{
    // the generalised LSQ gradient of the cells first, where selected
    const double *gin = nullptr;
    if (c->grad_kind == VOF_GRAD_LSQ) {
        launch_lsq_gradient(c, alpha, list, count, c->grad, s);
        gin = c->grad;
    }
    // lanes per cell and tetrahedra per lane: 4 x 1 (tetrahedral cells, eight
    // per warp), 8 x 2 (cells of <= 16 tetrahedra),
    // 8 x 3 (<= 24: hexahedra, four cells per warp), 32 x 2 (<= 64), 32 x 3
    // (<= 96: octree cells next to finer ones); the instrumented variant while
    // work counting is on (vof_count_work)
#define RC_GO(G_, K_, BL)                                                                                    \
    do {                                                                                                     \
        if (c->work_on)                                                                                      \
            k_reconstruct<LIST, MIXED, G_, K_, true><<<BL, 128, 0, s>>>(c->m, alpha, palpha, list, count, n, d, \
                flags, iters, maxit, c->status, c->mlp_s0, mlp_cap(c), next, c->work, gin);                  \
        else                                                                                                 \
            k_reconstruct<LIST, MIXED, G_, K_, false><<<BL, 128, 0, s>>>(c->m, alpha, palpha, list, count, n,   \
                d, flags, iters, maxit, c->status, c->mlp_s0, mlp_cap(c), next, nullptr, gin);                \
    } while (0)
    if (c->rc_g == 4) {
        const int blocks = LIST ? list_blocks : cdiv((long)c->nc * 4, 128);
        RC_GO(4, 1, blocks);
    } else if (c->rc_g == 8 && c->rc_k <= 2) {
        const int blocks = LIST ? list_blocks : cdiv((long)c->nc * 8, 128);
        RC_GO(8, 2, blocks);
    } else if (c->rc_g == 8) {
        const int blocks = LIST ? list_blocks : cdiv((long)c->nc * 8, 128);
        RC_GO(8, 3, blocks);
    } else if (c->rc_k <= 2) {
        const int blocks = LIST ? list_blocks : cdiv((long)c->nc * 32, 128);
        RC_GO(32, 2, blocks);
    } else {
        const int blocks = LIST ? list_blocks : cdiv((long)c->nc * 32, 128);
        RC_GO(32, 3, blocks);
    }
#undef RC_GO
}

// defaults of every cell (n = 0, d = 0, flags FULL or 0, iterations 0), and
// the interface cells appended to a list
__global__ void k_fill_list(int nc, double eps, const double *__restrict__ alpha, double *n, double *d,
                            uint8_t *flags, int *iters, int *list, int *count, unsigned *status)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    bool isint = false;
    if (c < nc) {
        const double a = alpha[c];
        flags[c] = a >= 1.0 - eps ? VOF_FULL : 0;
        n[c] = 0.0; n[nc + c] = 0.0; n[2 * nc + c] = 0.0;
        d[c] = 0.0;
        if (iters) iters[c] = 0;
        isint = a > eps && a < 1.0 - eps;
    }
    warp_append(isint, c, list, count, nc, status);
}

int launch_reconstruct(vof_ctx *c, const double *alpha, double *n, double *d, uint8_t *flags, int *iters,
                       const int *list, const int *count, cudaStream_t s)
{
    int sms = num_sms(c->device);
    const bool mx = c->precision == VOF_MIXED;
    if (mx && c->mlp && !list) {
        // the guess is indexed by list position: list the interface cells first
        k_zero_int<<<1, 32, 0, s>>>(c->counters + CNT_ICELL, 1);
        k_fill_list<<<cdiv(c->nc, 256), 256, 0, s>>>(c->nc, c->eps, alpha, n, d, flags, iters, c->icell,
                                                     c->counters + CNT_ICELL, c->status);
        list = c->icell;
        count = c->counters + CNT_ICELL;
    }
    if (mx && c->mlp) {
        int r = launch_mlp_guess(c, alpha, list, count, c->nc, s);
        if (r) return r;
    }
    if (list) {
        if (mx)
            rc_launch<true, true>(c, sms * 16, alpha, nullptr, list, count, n, d, flags, iters,
                                  c->counters + CNT_MAXPOS, s);
        else
            rc_launch<true, false>(c, sms * 16, alpha, nullptr, list, count, n, d, flags, iters,
                                   c->counters + CNT_MAXPOS, s);
    } else {
        if (mx)
            rc_launch<false, true>(c, 0, alpha, nullptr, nullptr, nullptr, n, d, flags, iters, nullptr, s);
        else
            rc_launch<false, false>(c, 0, alpha, nullptr, nullptr, nullptr, n, d, flags, iters, nullptr, s);
    }
    LAUNCH_CHECK();
    return VOF_OK;
}

int launch_flux_polyhedra(vof_ctx *c, const double *Up, const double *F, const double *lambda, double dt,
                          double *V, cudaStream_t s)
{
    k_flux_polyhedra<<<cdiv(c->nf, 128), 128, 0, s>>>(c->m, Up, F, lambda, dt, V);
    LAUNCH_CHECK();
    return VOF_OK;
}

int launch_correct_all(vof_ctx *c, const double *Up, const double *F, double dt, double *lambda, int *iters,
                       cudaStream_t s)
{
    k_correct<false><<<cdiv(c->nf, 128), 128, 0, s>>>(c->m, Up, F, dt, nullptr, nullptr, lambda, iters,
                                                             nullptr, nullptr, nullptr, c->work_on ? c->work : nullptr);
    LAUNCH_CHECK();
    return VOF_OK;
}

int launch_phase_flux_all(vof_ctx *c, const double *alpha, const double *n, const double *d, const uint8_t *flags,
                          const double *Up, const double *F, const double *lambda, double dt, double *Va, cudaStream_t s)
{
    return launch_pf_all(c, alpha, n, d, flags, Up, F, lambda, dt, Va, s);
}

// The bounding pass, post-bounding mass and statistics: one cooperative
// launch of k_bound_step, as many blocks as are resident at once (at most
// UPD_BLOCKS: the mass partials' room).
static int g_bound_blocks = 0;
static int launch_bound_step(vof_ctx *c, double *alpha, int nupd, const int *counters, double *stats,
                             cudaStream_t s)
{
    if (g_bound_blocks == 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bound_step, BA_THREADS, 0) != cudaSuccess || occ < 1)
            return VOF_ERR_CUDA;
        g_bound_blocks = std::min(num_sms(c->device) * occ, UPD_BLOCKS);
    }
    int *cnt = c->counters;
    BoundStep a{alpha,
                BoundBufs{c->viol[0], cnt + CNT_VIOL0, c->pend_c, c->pend_a, c->bscr, cnt + CNT_BPASS,
                          cnt + CNT_BACT0, c->nc, 8 * c->nc},
                cnt + CNT_PEND, c->seg, c->nseg, c->gpartial, cnt + CNT_VIOL1, c->reg_seg, c->nreg, c->reg_tot,
                c->partial + 5 * UPD_BLOCKS, c->partial, nupd, counters, stats,
                reinterpret_cast<unsigned *>(cnt + CNT_BAR), reinterpret_cast<unsigned *>(cnt + CNT_BARGEN), c->status};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g_bound_blocks);
    cfg.blockDim = dim3(BA_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_bound_step, c->m, a) != cudaSuccess) return VOF_ERR_CUDA;
    return VOF_OK;
}

int launch_barrier_probe(vof_ctx *c, int skip, cudaStream_t s)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_barrier_probe, 128, 0) != cudaSuccess || occ < 1)
        return VOF_ERR_CUDA;
    const int blocks = num_sms(c->device) * std::min(occ, 2);
    if (skip >= blocks) return VOF_ERR_INVALID_ARG;
    unsigned *cnt = reinterpret_cast<unsigned *>(c->counters + CNT_BAR);
    unsigned *gen = reinterpret_cast<unsigned *>(c->counters + CNT_BARGEN);
    if (cudaMemsetAsync(cnt, 0, sizeof(unsigned), s) != cudaSuccess) return VOF_ERR_CUDA;
    int rounds = 4;
    long limit = 2000;  // with the pauses (up to ~1 us) a few milliseconds
    void *args[] = {&cnt, &gen, &c->status, &skip, &rounds, &limit};
    if (cudaLaunchCooperativeKernel((const void *)k_barrier_probe, dim3(blocks), dim3(128), args, 0, s) != cudaSuccess)
        return VOF_ERR_CUDA;
    return VOF_OK;
}

// Courant number: the largest (1/2) sum |F_f| dt / V_c over the cells, the
// block maxima combined by an atomic max on the bit patterns (non-negative
// doubles order as their 64-bit integers)
__global__ void k_courant(DevMesh m, const double *__restrict__ F, double dt, unsigned long long *co)
{
    __shared__ double red[8];
    double v = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m.nc; c += gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int k = m.cptr[c]; k < m.cptr[c + 1]; ++k) sum += fabs(F[m.cflux[k] >> 1]);
        v = fmax(v, 0.5 * sum * dt / m.vc[c]);
    }
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
        atomicMax(co, (unsigned long long)__double_as_longlong(v));
    }
}

int launch_courant(vof_ctx *c, const double *F, double dt, double *co, cudaStream_t s)
{
    if (cudaMemsetAsync(co, 0, sizeof(double), s) != cudaSuccess) return VOF_ERR_CUDA;
    k_courant<<<num_sms(c->device) * 4, 256, 0, s>>>(c->m, F, dt, reinterpret_cast<unsigned long long *>(co));
    LAUNCH_CHECK();
    return VOF_OK;
}

int launch_update(vof_ctx *c, double *alpha, const double *Va, double *stats, cudaStream_t s)
{
    int *cnt = c->counters;
    int launches = 0;
    k_zero_update<<<1, 32, 0, s>>>(cnt);
    const int nu = upd_blocks(c->device);
    k_update<<<nu, UPD_THREADS, 0, s>>>(c->m, alpha, Va, c->partial, c->bound ? c->viol[0] : nullptr,
                                        cnt + CNT_VIOL0, c->nc, c->status);
    LAUNCH_CHECK();
    launches += 3;
    if (c->bound) {
        int r = launch_bound_step(c, alpha, nu, nullptr, stats ? stats : c->stats_dev, s);
        if (r) return r;
    } else {
        k_stats<<<1, ST_THREADS, 0, s>>>(c->partial, nu, nullptr, stats ? stats : c->stats_dev, 0, nullptr, 0);
        LAUNCH_CHECK();
    }
    c->launches = launches;
    return VOF_OK;
}

int launch_advect(vof_ctx *c, double *alpha, const double *Uc, const double *F, double dt, double *stats,
                  cudaStream_t s, cudaEvent_t wait_before_correct)
{
    DevMesh &m = c->m;
    int sms = num_sms(c->device);
    int *cnt = c->counters;
    int launches = 0;
    cudaEvent_t *ev = nullptr;
    if (c->prof_ev && c->prof_steps < c->prof_max) ev = c->prof_ev + (size_t)c->prof_steps++ * (VOF_PROF_GROUPS + 1);
#define MARK(i) do { if (ev) cudaEventRecord(ev[i], s); } while (0)
    MARK(0);
    k_zero_int<<<1, 32, 0, s>>>(cnt, CNT_LEN);
    k_point_state<<<cdiv(m.np, 256), 256, 0, s>>>(m, alpha, c->pstate, c->palpha);
    k_classify<<<sms * 16, 256, 0, s>>>(m, alpha, F, dt, c->pstate, c->Va, c->band, cnt + CNT_BAND, c->icell,
                                        cnt + CNT_ICELL, c->bpflag, c->status);
    launches += 3;
    LAUNCH_CHECK();
    MARK(1);
    // The correction (band point velocities, then lambda per band face) needs
    // the band list and the velocities, the reconstruction the interface list:
    // the two run side by side, the correction on the context's second stream,
    // joined before the phase flux.  The first use of Uc is there, so a
    // velocity copy still in flight on another stream is waited for there.
    if (cudaEventRecord(c->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(c->s_aux, c->ev_fork, 0) != cudaSuccess)
        return VOF_ERR_CUDA;
    if (wait_before_correct && cudaStreamWaitEvent(c->s_aux, wait_before_correct, 0) != cudaSuccess)
        return VOF_ERR_CUDA;
    k_band_point_velocity<<<cdiv(m.np, 256), 256, 0, c->s_aux>>>(m, Uc, c->bpflag, c->upb);
    k_correct<true><<<sms * 8, 128, 0, c->s_aux>>>(m, c->upb, F, dt, c->band, cnt + CNT_BAND, c->lam_b, c->it_b,
                                                   c->disp_b, cnt + CNT_MAXCORR, cnt + CNT_FALLBACK,
                                                   c->work_on ? c->work : nullptr);
    LAUNCH_CHECK();
    if (cudaEventRecord(c->ev_join, c->s_aux) != cudaSuccess) return VOF_ERR_CUDA;
    if (c->precision == VOF_MIXED && c->mlp) {
        int r = launch_mlp_guess(c, alpha, c->icell, cnt + CNT_ICELL, c->nc, s);
        if (r) return r;
        ++launches;
    }
    if (c->precision == VOF_MIXED)
        rc_launch<true, true>(c, sms * 16, alpha, c->palpha, c->icell, cnt + CNT_ICELL, c->n, c->d, c->flags, nullptr,
                              cnt + CNT_MAXPOS, s, cnt + CNT_RCNEXT);
    else
        rc_launch<true, false>(c, sms * 16, alpha, c->palpha, c->icell, cnt + CNT_ICELL, c->n, c->d, c->flags, nullptr,
                               cnt + CNT_MAXPOS, s, cnt + CNT_RCNEXT);
    MARK(2);
    if (cudaStreamWaitEvent(s, c->ev_join, 0) != cudaSuccess) return VOF_ERR_CUDA;
    MARK(3);
    {
        int r = launch_pf_list(c, alpha, F, dt, sms, s);
        if (r) return r;
    }
    launches += 4;  // reconstruct, band point velocities, correct, phase flux
    LAUNCH_CHECK();
    MARK(4);
    // update + bounding + stats
    k_zero_update<<<1, 32, 0, s>>>(cnt);
    const int nu = upd_blocks(c->device);
    k_update<<<nu, UPD_THREADS, 0, s>>>(m, alpha, c->Va, c->partial, c->bound ? c->viol[0] : nullptr,
                                        cnt + CNT_VIOL0, c->nc, c->status);
    launches += 3;
    LAUNCH_CHECK();
    if (c->bound) {
        int r = launch_bound_step(c, alpha, nu, cnt, stats ? stats : c->stats_dev, s);
        if (r) return r;
    } else {
        k_stats<<<1, ST_THREADS, 0, s>>>(c->partial, nu, cnt, stats ? stats : c->stats_dev, 0, nullptr, 0);
        LAUNCH_CHECK();
    }
    MARK(5);
#undef MARK
    c->launches = launches;
    return VOF_OK;
}

int launch_validate(vof_ctx *c, cudaStream_t s, unsigned *bad)
{
    (void)c; (void)s; (void)bad;
    return VOF_OK;
}

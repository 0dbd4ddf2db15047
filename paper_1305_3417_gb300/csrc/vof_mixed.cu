// Mixed-precision phase flux (A6): the flux-polyhedron tetrahedra T, the cell
// tetrahedra K and the PLIC planes are taken to a frame centred on the face
// centre and clipped in FP32; the pieces are summed per lane with TwoSum
// compensation and finished in FP64.
//
// Only the frame shift of a stencil cell (its centre minus the face centre) and
// of its plane offset are formed in FP64; the cell's own geometry comes from
// FP32 offsets to the cell centre computed once at context creation, so the
// rounding of a coordinate is relative to the cell size, not to its position.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "vof_device.cuh"
#include "vof_internal.h"

namespace {
using namespace vofd;

struct F3 { float x, y, z; };
__device__ __forceinline__ F3 f3(float x, float y, float z) { return F3{x, y, z}; }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ F3 operator*(F3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float fdot(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ F3 fcross(F3 a, F3 b)
{
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float fvol6(F3 a, F3 b, F3 c, F3 d) { return fdot(b - a, fcross(c - a, d - a)); }
__device__ __forceinline__ F3 ld4(const float4 *p, long i)
{
    float4 v = __ldg(p + i);
    return f3(v.x, v.y, v.z);
}

// fraction of a tetrahedron below level 0 for sorted vertex values h0..h3
__device__ __forceinline__ float ffrac_below(float h0, float h1, float h2, float h3)
{
    if (0.0f <= h0) return 0.0f;
    if (0.0f >= h3) return 1.0f;
    if (0.0f <= h1) {
        float x = -h0;
        return (x / (h1 - h0)) * (x / (h2 - h0)) * (x / (h3 - h0));
    }
    if (0.0f >= h2) {
        float y = h3;
        return 1.0f - (y / (h3 - h0)) * (y / (h3 - h1)) * (y / (h3 - h2));
    }
    float a = -h0 / (h2 - h0), b = -h0 / (h3 - h0), c = -h1 / (h2 - h1), e = -h1 / (h3 - h1);
    return a * b + a * (1.0f - b) * e + (1.0f - a) * c * e;
}

__device__ __forceinline__ void fsort4(float &a, float &b, float &c, float &d)
{
    float t;
#define CS(p, q) if (p > q) { t = p; p = q; q = t; }
    CS(a, b) CS(c, d) CS(a, c) CS(b, d) CS(b, c)
#undef CS
}

struct FTet { F3 v[4]; };

// |T ^ {n_k.x <= d_k}| in FP32: depth-first split into the tetrahedra of the
// inside parts, the last plane by the closed-form cut fraction (6x volume)
__device__ float fclip6(const FTet &T, const float4 *pl, int np, float tol, unsigned *status, unsigned &cuts)
{
    if (np == 0) return fabsf(fvol6(T.v[0], T.v[1], T.v[2], T.v[3]));
    FTet st[CLIP_STACK];
    unsigned char lv[CLIP_STACK];
    int sp = 1;
    st[0] = T;
    lv[0] = 0;
    float vol = 0.0f;
    while (sp > 0) {
        --sp;
        FTet t = st[sp];
        int k = lv[sp];
        float4 p = pl[k];
        F3 n = f3(p.x, p.y, p.z);
        float s[4];
        int nin = 0, nup = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            s[i] = fdot(n, t.v[i]) - p.w;
            if (fabsf(s[i]) <= tol) s[i] = 0.0f;  // on the plane (FP32 rounding of shared points)
            nin += s[i] < 0.0f;
            nup += s[i] > 0.0f;
        }
        if (nin == 0) continue;  // nothing strictly inside: no volume
        if (nup == 0) {
            if (k + 1 == np) vol += fabsf(fvol6(t.v[0], t.v[1], t.v[2], t.v[3]));
            else if (sp < CLIP_STACK) { st[sp] = t; lv[sp] = k + 1; ++sp; }
            else atomicOr(status, VOF_ST_CLIP_OVERFLOW);
            continue;
        }
        ++cuts;
        if (k + 1 == np) {
            float h0 = s[0], h1 = s[1], h2 = s[2], h3 = s[3];
            fsort4(h0, h1, h2, h3);
            vol += fabsf(fvol6(t.v[0], t.v[1], t.v[2], t.v[3])) * ffrac_below(h0, h1, h2, h3);
            continue;
        }
        int ord[4], a = 0, b = 3;
#pragma unroll
        for (int i = 0; i < 4; ++i) { if (s[i] < 0.0f) ord[a++] = i; else ord[b--] = i; }
        F3 P[4];
        float S[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { P[i] = t.v[ord[i]]; S[i] = s[ord[i]]; }
        auto ep = [&](int i, int o) { return P[i] + (P[o] - P[i]) * (S[i] / (S[i] - S[o])); };
        FTet out[3];
        int nout;
        if (nin == 1) {
            out[0] = FTet{{P[0], ep(0, 1), ep(0, 2), ep(0, 3)}};
            nout = 1;
        } else if (nin == 2) {
            F3 a0 = P[0], a1 = ep(0, 2), a2 = ep(0, 3), b0 = P[1], b1 = ep(1, 2), b2 = ep(1, 3);
            out[0] = FTet{{a0, a1, a2, b2}};
            out[1] = FTet{{a0, a1, b2, b1}};
            out[2] = FTet{{a0, b0, b1, b2}};
            nout = 3;
        } else {
            F3 a0 = P[0], a1 = P[1], a2 = P[2], b0 = ep(0, 3), b1 = ep(1, 3), b2 = ep(2, 3);
            out[0] = FTet{{a0, a1, a2, b2}};
            out[1] = FTet{{a0, a1, b2, b1}};
            out[2] = FTet{{a0, b0, b1, b2}};
            nout = 3;
        }
        for (int i = 0; i < nout; ++i) {
            if (sp < CLIP_STACK) { st[sp] = out[i]; lv[sp] = k + 1; ++sp; }
            else atomicOr(status, VOF_ST_CLIP_OVERFLOW);
        }
    }
    return vol;
}

// TwoSum (Knuth): s + c carries the running sum exactly up to the last addend's
// rounding; no multiplications, so no fused operation can change it
__device__ __forceinline__ void two_sum(float &s, float &c, float x)
{
    float t = s + x;
    float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

constexpr int MX_WARPS = 4;
constexpr int MX_MAXT = 3 * VOF_MAXFP;

struct MXArgs {
    const double *alpha, *n, *d;
    const uint8_t *flags;
    const double *Up, *F, *lambda;
    double dt;
    double *Va;
    const int *list, *count;
    const double *disp, *lam_b;
    unsigned *status;
    unsigned long long *work;
    const float4 *cfl, *cfpl, *fpl, *cbl;  // FP32 local geometry
    const int *cfpptr;
};

constexpr int MX_CAND = 32;                 // candidate cell tetrahedra buffered per warp
constexpr int MX_QUEUE = MX_MAXT * MX_CAND;  // clip jobs: one per (T, K) pair at most

struct MXShared {
    FTet T[MX_MAXT];
    float Tb[MX_MAXT][6];
    float Tv6[MX_MAXT];      // |6 vol(T)|
    float Tsg[MX_MAXT];      // sign of T in the flux polyhedron
    float4 Kp[MX_CAND][4];   // outward planes of the candidate cell tetrahedra
    float Kb[MX_CAND][6];
    float4 KH[MX_CAND];      // the cell's phase (or void) half-space
    float Kw[MX_CAND];       // weight: 1, or alpha (1-alpha) of an unoriented cell
    unsigned char KuseH[MX_CAND];
    unsigned Q[MX_QUEUE];    // clip jobs: t | k << 5 | plane mask << 10
};

// all (T, K) pairs of the buffered candidates: boxes and planes first; a pair
// inside every plane adds |T| at once, a pair that must be cut goes to the
// queue; then the lanes take the queued cuts
__device__ __forceinline__ void mx_flush(MXShared &sh, int nt, int ncand, float tol, float &accs, float &accc,
                                         unsigned &npairs, unsigned &ncuts, unsigned *status)
{
    const int lane = threadIdx.x & 31;
    const int npr = nt * ncand;
    int nq = 0;
    for (int base = 0; base < npr; base += 32) {
        const int w = base + lane;
        bool job = false;
        unsigned code = 0;
        if (w < npr) {
            const int t = w % nt, k = w / nt;
            const float sg = sh.Tsg[t];
            const float *tb = sh.Tb[t], *kb = sh.Kb[k];
            if (sg != 0.0f && !(tb[3] < kb[0] || kb[3] < tb[0] || tb[4] < kb[1] || kb[4] < tb[1] ||
                                tb[5] < kb[2] || kb[5] < tb[2])) {
                ++npairs;
                const FTet &T = sh.T[t];
                unsigned mask = 0;
                bool outside = false;
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    float4 p;
                    if (q < 4) p = sh.Kp[k][q];
                    else if (sh.KuseH[k]) p = sh.KH[k];
                    else break;
                    // a vertex within tol of the plane is on it: the pair is outside
                    // when no vertex is clearly inside, the plane cuts only when
                    // vertices lie clearly on both sides
                    int nneg = 0, npos = 0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float sd = p.x * T.v[i].x + p.y * T.v[i].y + p.z * T.v[i].z - p.w;
                        nneg += sd < -tol;
                        npos += sd > tol;
                    }
                    if (nneg == 0) { outside = true; break; }
                    if (npos > 0) mask |= 1u << q;
                }
                if (!outside) {
                    if (mask == 0) two_sum(accs, accc, sg * sh.Kw[k] * sh.Tv6[t]);
                    else { job = true; code = (unsigned)t | ((unsigned)k << 5) | (mask << 10); }
                }
            }
        }
        const unsigned bm = __ballot_sync(0xffffffffu, job);
        if (job) sh.Q[nq + __popc(bm & ((1u << lane) - 1u))] = code;
        nq += __popc(bm);
    }
    __syncwarp();
    for (int q = lane; q < nq; q += 32) {
        const unsigned code = sh.Q[q];
        const int t = code & 31, k = (code >> 5) & 31;
        const unsigned mask = code >> 10;
        float4 act[5];
        int np = 0;
#pragma unroll
        for (int j = 0; j < 5; ++j)
            if (mask & (1u << j)) act[np++] = j < 4 ? sh.Kp[k][j] : sh.KH[k];
        float v6 = fclip6(sh.T[t], act, np, tol, status, ncuts);
        two_sum(accs, accc, sh.Tsg[t] * sh.Kw[k] * v6);
    }
    __syncwarp();
}

template <bool LIST>
__global__ void __launch_bounds__(MX_WARPS * 32) k_phase_flux_mixed(DevMesh m, MXArgs a)
{
    __shared__ MXShared shm[MX_WARPS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    MXShared &sh = shm[wib];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int total = LIST ? *a.count : m.nf;
    const double eps = m.eps;
    for (int item = warp; item < total; item += nwarps) {
        const int f = LIST ? a.list[item] : item;
        const int s0 = __ldg(m.sptr + f), s1 = __ldg(m.sptr + f + 1);
        if (!LIST) {
            double Ff = a.F[f];
            bool all_e = true, all_f = true;
            for (int s = s0 + lane; s < s1; s += 32) {
                double al = a.alpha[__ldg(m.scell + s)];
                all_e &= al <= eps;
                all_f &= al >= 1.0 - eps;
            }
            all_e = __all_sync(0xffffffffu, all_e);
            all_f = __all_sync(0xffffffffu, all_f);
            double triv = 0.0;
            bool done = true;
            if (Ff == 0.0 || (f >= m.ni && Ff < 0.0) || all_e) triv = 0.0;
            else if (all_f) triv = Ff * a.dt;
            else done = false;
            if (done) {
                if (lane == 0) a.Va[f] = triv;
                continue;
            }
        }
        const V3 o = ld3(m.cf, m.nf, f);
        const int b = __ldg(m.fptr + f), n = __ldg(m.fptr + f + 1) - b;
        // Complement form: when the upwind cell is mostly phase, sum the void
        // pieces and take V_alpha = F dt - void (equal in exact arithmetic since
        // the corrected polyhedron holds F dt and the stencil covers it); a
        // polyhedron inside full cells then carries exactly F dt, one inside
        // empty cells exactly 0, and FP32 rounding stays with mixed cells
        // (not for the normal-sweep fallback, which can leave the domain at walls).
        const double Ff = a.F[f];
        const int up = Ff > 0.0 ? __ldg(m.own + f) : (f < m.ni ? __ldg(m.nei + f) : __ldg(m.own + f));
        const double lamf = LIST ? a.lam_b[item] : a.lambda[f];
        const bool comp = a.alpha[up] >= 0.5 && lamf >= 0.0;
        const int nt = n == 3 ? 3 : 3 * n;
        // signed distances (to unit-normal planes) within 2e-6 of the face size are
        // taken as zero: points shared by the polyhedron and the cell tetrahedra
        // come out of different FP32 roundings and would otherwise look like cuts
        const float tol = 2e-6f * (float)sqrt(sqrt(dot(ld3(m.sf, m.nf, f), ld3(m.sf, m.nf, f))));
        // ---- flux polyhedron tetrahedra in the face frame
        float bx[6] = {3e38f, 3e38f, 3e38f, -3e38f, -3e38f, -3e38f};
        if (lane < nt) {
            int pr = lane / 3, j = lane % 3;
            auto disp = [&](int i) -> F3 {  // i < 0: face centre
                V3 w;
                if (LIST) {
                    const double *q = a.disp + (size_t)item * DISP_STRIDE + (i < 0 ? 0 : 3 + 3 * i);
                    w = mk(q[0], q[1], q[2]);
                } else {
                    double lam = a.lambda[f];
                    if (lam < 0.0) {
                        V3 S = ld3(m.sf, m.nf, f);
                        w = S * (-lam * a.F[f] * a.dt / dot(S, S));
                    } else if (i >= 0) {
                        w = ld3(a.Up, m.np, __ldg(m.fpts + b + i)) * (a.dt * lam);
                    } else {
                        w = mk(0, 0, 0);
                        for (int q = 0; q < n; ++q) w = w + ld3(a.Up, m.np, __ldg(m.fpts + b + q)) * (a.dt * lam);
                        w = w * (1.0 / n);
                    }
                }
                return f3((float)w.x, (float)w.y, (float)w.z);
            };
            F3 a0, a1, a2, w0, w1, w2;
            long k0, k1, k2;
            if (n == 3) {
                k0 = __ldg(m.fpts + b); k1 = __ldg(m.fpts + b + 1); k2 = __ldg(m.fpts + b + 2);
                a0 = ld4(a.fpl, b); a1 = ld4(a.fpl, b + 1); a2 = ld4(a.fpl, b + 2);
                w0 = disp(0); w1 = disp(1); w2 = disp(2);
            } else {
                int u = pr + 1 == n ? 0 : pr + 1;
                k0 = -1; k1 = __ldg(m.fpts + b + pr); k2 = __ldg(m.fpts + b + u);
                a0 = f3(0.f, 0.f, 0.f); a1 = ld4(a.fpl, b + pr); a2 = ld4(a.fpl, b + u);
                w0 = disp(-1); w1 = disp(pr); w2 = disp(u);
            }
            int par = 1;
            if (k1 < k0) { F3 t = a0; a0 = a1; a1 = t; t = w0; w0 = w1; w1 = t; long q = k0; k0 = k1; k1 = q; par = -par; }
            if (k2 < k1) { F3 t = a1; a1 = a2; a2 = t; t = w1; w1 = w2; w2 = t; long q = k1; k1 = k2; k2 = q; par = -par; }
            if (k1 < k0) { F3 t = a0; a0 = a1; a1 = t; t = w0; w0 = w1; w1 = t; long q = k0; k0 = k1; k1 = q; par = -par; }
            F3 b0 = a0 - w0, b1 = a1 - w1, b2 = a2 - w2;
            FTet T;
            if (j == 0) T = FTet{{a0, a1, a2, b2}};
            else if (j == 1) T = FTet{{a0, a1, b2, b1}};
            else T = FTet{{a0, b0, b1, b2}};
            float v6 = fvol6(T.v[0], T.v[1], T.v[2], T.v[3]);
            float sv = -par * v6;
            sh.T[lane] = T;
            sh.Tsg[lane] = sv > 0.0f ? 1.0f : (sv < 0.0f ? -1.0f : 0.0f);
            sh.Tv6[lane] = fabsf(v6);
            bx[0] = fminf(fminf(T.v[0].x, T.v[1].x), fminf(T.v[2].x, T.v[3].x));
            bx[1] = fminf(fminf(T.v[0].y, T.v[1].y), fminf(T.v[2].y, T.v[3].y));
            bx[2] = fminf(fminf(T.v[0].z, T.v[1].z), fminf(T.v[2].z, T.v[3].z));
            bx[3] = fmaxf(fmaxf(T.v[0].x, T.v[1].x), fmaxf(T.v[2].x, T.v[3].x));
            bx[4] = fmaxf(fmaxf(T.v[0].y, T.v[1].y), fmaxf(T.v[2].y, T.v[3].y));
            bx[5] = fmaxf(fmaxf(T.v[0].z, T.v[1].z), fmaxf(T.v[2].z, T.v[3].z));
            for (int i = 0; i < 6; ++i) sh.Tb[lane][i] = bx[i];
        }
        // bounding box of the whole polyhedron
        float pb[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            float v = bx[i];
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) {
                float w = __shfl_xor_sync(0xffffffffu, v, o2);
                v = i < 3 ? fminf(v, w) : fmaxf(v, w);
            }
            pb[i] = v;
        }
        __syncwarp();
        float accs = 0.0f, accc = 0.0f;
        unsigned npairs = 0, ncuts = 0;
        int ncand = 0;
        for (int s = s0; s < s1; ++s) {
            const int c = __ldg(m.scell + s);
            const double al = a.alpha[c];
            if (!comp && al <= eps) continue;       // empty cell carries no phase
            if (comp && al >= 1.0 - eps) continue;  // full cell carries no void
            const V3 cc = ld3(m.cc, m.nc, c);
            const F3 dc = f3((float)(cc.x - o.x), (float)(cc.y - o.y), (float)(cc.z - o.z));
            const float4 cb0 = __ldg(a.cbl + 2 * (size_t)c), cb1 = __ldg(a.cbl + 2 * (size_t)c + 1);
            if (cb1.x + dc.x < pb[0] || pb[3] < cb0.x + dc.x || cb1.y + dc.y < pb[1] || pb[4] < cb0.y + dc.y ||
                cb1.z + dc.z < pb[2] || pb[5] < cb0.z + dc.z)
                continue;
            float wgt = 1.0f;
            bool useH = false;
            float4 H = make_float4(0.f, 0.f, 0.f, 0.f);
            if (al > eps && al < 1.0 - eps) {
                if (a.flags[c] & VOF_ORIENTED) {
                    V3 hn = ld3(a.n, m.nc, c);
                    double hd = a.d[c] - dot(hn, o);
                    // phase side n.x <= d; the void side is -n.x <= -d
                    float sg = comp ? -1.0f : 1.0f;
                    H = make_float4(sg * (float)hn.x, sg * (float)hn.y, sg * (float)hn.z, sg * (float)hd);
                    useH = true;
                } else wgt = comp ? (float)(1.0 - al) : (float)al;
            }
            // ---- this cell's tetrahedra, 32 at a time, into the candidate buffer
            const int f0 = __ldg(m.cptr + c), f1 = __ldg(m.cptr + c + 1);
            const int cpb = __ldg(a.cfpptr + c);
            for (int kb = 0;; kb += 32) {
                int off = kb + lane, k = f0, code = 0, gn = 0, pofs = cpb;
                bool found = false;
                for (; k < f1; ++k) {
                    code = __ldg(m.cface + k);
                    int g = code >> 1;
                    gn = __ldg(m.fptr + g + 1) - __ldg(m.fptr + g);
                    int gt = gn == 3 ? 1 : gn;
                    if (off < gt) { found = true; break; }
                    off -= gt;
                    pofs += gn;
                }
                if (!__any_sync(0xffffffffu, found)) break;
                bool cand = false;
                float4 kp[4];
                float kbx[6];
                if (found) {
                    F3 k0 = dc, k1, k2, k3;
                    if (gn == 3) {
                        k1 = ld4(a.cfpl, pofs) + dc; k2 = ld4(a.cfpl, pofs + 1) + dc; k3 = ld4(a.cfpl, pofs + 2) + dc;
                    } else {
                        k1 = ld4(a.cfl, k) + dc;
                        k2 = ld4(a.cfpl, pofs + off) + dc;
                        k3 = ld4(a.cfpl, pofs + (off + 1 == gn ? 0 : off + 1)) + dc;
                    }
                    if (code & 1) { F3 t = k2; k2 = k3; k3 = t; }
                    kbx[0] = fminf(fminf(k0.x, k1.x), fminf(k2.x, k3.x)); kbx[3] = fmaxf(fmaxf(k0.x, k1.x), fmaxf(k2.x, k3.x));
                    kbx[1] = fminf(fminf(k0.y, k1.y), fminf(k2.y, k3.y)); kbx[4] = fmaxf(fmaxf(k0.y, k1.y), fmaxf(k2.y, k3.y));
                    kbx[2] = fminf(fminf(k0.z, k1.z), fminf(k2.z, k3.z)); kbx[5] = fmaxf(fmaxf(k0.z, k1.z), fmaxf(k2.z, k3.z));
                    cand = !(kbx[3] < pb[0] || pb[3] < kbx[0] || kbx[4] < pb[1] || pb[4] < kbx[1] ||
                             kbx[5] < pb[2] || pb[5] < kbx[2]);
                    if (cand) {
                        F3 n0 = fcross(k2 - k0, k1 - k0), n1 = fcross(k1 - k0, k3 - k0);
                        F3 n2 = fcross(k3 - k0, k2 - k0), n3 = fcross(k2 - k1, k3 - k1);
                        n0 = n0 * rsqrtf(fdot(n0, n0) + 1e-37f); n1 = n1 * rsqrtf(fdot(n1, n1) + 1e-37f);
                        n2 = n2 * rsqrtf(fdot(n2, n2) + 1e-37f); n3 = n3 * rsqrtf(fdot(n3, n3) + 1e-37f);
                        kp[0] = make_float4(n0.x, n0.y, n0.z, fdot(n0, k0));
                        kp[1] = make_float4(n1.x, n1.y, n1.z, fdot(n1, k0));
                        kp[2] = make_float4(n2.x, n2.y, n2.z, fdot(n2, k0));
                        kp[3] = make_float4(n3.x, n3.y, n3.z, fdot(n3, k1));
                    }
                }
                const unsigned cmask = __ballot_sync(0xffffffffu, cand);
                if (ncand + __popc(cmask) > MX_CAND) {  // buffer full: process it first
                    mx_flush(sh, nt, ncand, tol, accs, accc, npairs, ncuts, a.status);
                    ncand = 0;
                }
                if (cand) {
                    int r = ncand + __popc(cmask & ((1u << lane) - 1u));
                    for (int q = 0; q < 4; ++q) sh.Kp[r][q] = kp[q];
                    for (int q = 0; q < 6; ++q) sh.Kb[r][q] = kbx[q];
                    sh.KH[r] = H;
                    sh.Kw[r] = wgt;
                    sh.KuseH[r] = useH;
                }
                ncand += __popc(cmask);
                __syncwarp();
            }
        }
        if (ncand > 0) mx_flush(sh, nt, ncand, tol, accs, accc, npairs, ncuts, a.status);
        // finish in FP64: lane sums and compensations, then the 1/6 of the volumes
        double acc = warp_sum((double)accs + (double)accc) / 6.0;
        if (comp) acc = Ff * a.dt - acc;
        if (a.work) {
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) {
                npairs += __shfl_xor_sync(0xffffffffu, npairs, o2);
                ncuts += __shfl_xor_sync(0xffffffffu, ncuts, o2);
            }
            if (lane == 0) {
                atomicAdd(a.work, (unsigned long long)npairs);
                atomicAdd(a.work + 1, (unsigned long long)ncuts);
                atomicAdd(a.work + 2, 1ull);
            }
        }
        if (lane == 0) a.Va[f] = acc;
        __syncwarp();
    }
}

// FP32 geometry of every cell relative to its centre (context creation)
__global__ void k_local_geom(DevMesh m, const int *cfpptr, float4 *cfl, float4 *cfpl, float4 *cbl)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    V3 cc = ld3(m.cc, m.nc, c);
    int o = cfpptr[c];
    for (int k = m.cptr[c]; k < m.cptr[c + 1]; ++k) {
        int g = m.cface[k] >> 1;
        V3 q = ld3(m.cf, m.nf, g) - cc;
        cfl[k] = make_float4((float)q.x, (float)q.y, (float)q.z, 0.f);
        for (int j = m.fptr[g]; j < m.fptr[g + 1]; ++j) {
            V3 p = ldP(m, m.fpts[j]) - cc;
            cfpl[o++] = make_float4((float)p.x, (float)p.y, (float)p.z, 0.f);
        }
    }
    const double *b = m.cbox + 6 * (size_t)c;
    // widened by one FP32 rounding so that FP32 boxes stay conservative
    auto lo = [](double v) { float f = (float)v; return f > v ? nextafterf(f, -3e38f) : f; };
    auto hi = [](double v) { float f = (float)v; return f < v ? nextafterf(f, 3e38f) : f; };
    cbl[2 * c] = make_float4(lo(b[0] - cc.x), lo(b[1] - cc.y), lo(b[2] - cc.z), 0.f);
    cbl[2 * c + 1] = make_float4(hi(b[3] - cc.x), hi(b[4] - cc.y), hi(b[5] - cc.z), 0.f);
}

__global__ void k_face_local(DevMesh m, float4 *fpl)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.nf) return;
    V3 c = ld3(m.cf, m.nf, f);
    for (int j = m.fptr[f]; j < m.fptr[f + 1]; ++j) {
        V3 p = ldP(m, m.fpts[j]) - c;
        fpl[j] = make_float4((float)p.x, (float)p.y, (float)p.z, 0.f);
    }
}

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

}  // namespace

int launch_setup_mixed(vof_ctx *c, cudaStream_t s)
{
    k_local_geom<<<cdiv(c->nc, 256), 256, 0, s>>>(c->m, c->cfpptr, c->cfl, c->cfpl, c->cbl);
    k_face_local<<<cdiv(c->nf, 256), 256, 0, s>>>(c->m, c->fpl);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

static MXArgs mx_args(vof_ctx *c, const double *alpha, const double *n, const double *d, const uint8_t *flags,
                      const double *Up, const double *F, const double *lambda, double dt, double *Va,
                      const int *list, const int *count, const double *disp, unsigned long long *work)
{
    return MXArgs{alpha, n, d, flags, Up, F, lambda, dt, Va, list, count, disp, c->lam_b, c->status, work,
                  c->cfl, c->cfpl, c->fpl, c->cbl, c->cfpptr};
}

int launch_phase_flux_mixed_all(vof_ctx *c, const double *alpha, const double *n, const double *d,
                                const uint8_t *flags, const double *Up, const double *F, const double *lambda,
                                double dt, double *Va, cudaStream_t s)
{
    MXArgs a = mx_args(c, alpha, n, d, flags, Up, F, lambda, dt, Va, nullptr, nullptr, nullptr, nullptr);
    k_phase_flux_mixed<false><<<cdiv((long)c->nf * 32, MX_WARPS * 32), MX_WARPS * 32, 0, s>>>(c->m, a);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

int launch_phase_flux_mixed_list(vof_ctx *c, const double *alpha, const double *F, double dt, int sms,
                                 cudaStream_t s)
{
    MXArgs a = mx_args(c, alpha, c->n, c->d, c->flags, nullptr, F, nullptr, dt, c->Va, c->band,
                       c->counters + CNT_BAND, c->disp_b, c->work);
    k_phase_flux_mixed<true><<<sms * 16, MX_WARPS * 32, 0, s>>>(c->m, a);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

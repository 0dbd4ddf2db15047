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
// (fast reciprocal divisions: 2 ulp, far inside the form's FP32 rounding)
__device__ __forceinline__ float ffrac_below(float h0, float h1, float h2, float h3)
{
    if (0.0f <= h0) return 0.0f;
    if (0.0f >= h3) return 1.0f;
    if (0.0f <= h1) {
        float x = -h0;
        return __fdividef(x, h1 - h0) * __fdividef(x, h2 - h0) * __fdividef(x, h3 - h0);
    }
    if (0.0f >= h2) {
        float y = h3;
        return 1.0f - __fdividef(y, h3 - h0) * __fdividef(y, h3 - h1) * __fdividef(y, h3 - h2);
    }
    float a = __fdividef(-h0, h2 - h0), b = __fdividef(-h0, h3 - h0);
    float c = __fdividef(-h1, h2 - h1), e = __fdividef(-h1, h3 - h1);
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

// TwoSum (Knuth): s + c carries the running sum exactly up to the last addend's
// rounding; no multiplications, so no fused operation can change it
__device__ __forceinline__ void two_sum(float &s, float &c, float x)
{
    float t = s + x;
    float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

constexpr int MX_MAXT = 3 * VOF_MAXFP;
static_assert(MX_MAXT <= 32, "one flux-polyhedron tetrahedron per lane");

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
    const float4 *fpl, *cbl;  // FP32 face points (face frame), cell boxes (cell frame)
    const float4 *ktl;        // cell tetrahedra: planes and box (cell frame)
    const int *ctptr;
    int *next;                // list form: next band slot to take (zero before the launch), or null
};

constexpr int MX_CAND = 32;    // candidate cell tetrahedra buffered per warp: one per lane
constexpr int MX_QUEUE = MX_MAXT * MX_CAND;  // clip jobs: one per (T, K) pair at most
constexpr int MX_STACK = 92;                 // pieces of clip jobs waiting for their next plane

// per warp; the 48-byte tetrahedra are moved as three float4 (conflict-free
// across a warp)
struct __align__(16) MXShared {
    FTet S[MX_STACK];        // pieces
    FTet T[MX_MAXT];         // flux-polyhedron tetrahedra
    float4 Kp[MX_CAND][5];   // outward unit-normal planes of the candidate cell tetrahedra, then
                             // the cell's phase (or void) half-space; 80-byte rows: a warp's
                             // float4 reads of different rows are conflict-free
    float4 P6[VOF_MAXFP][5]; // per prism (face triangle swept): a0 a1 a2 b0 b1 b2, 18 floats in 80 bytes
    float Pb[VOF_MAXFP][6];  // prism box
    float Kb[MX_CAND][6];
    float Tv6[MX_MAXT];      // |6 vol(T)|
    float Tsg[MX_MAXT];      // sign of T in the flux polyhedron
    float Kw[MX_CAND];       // weight: 1, or alpha (1-alpha) of an unoriented cell
    // stencil cells of the current chunk that reach the polyhedron's box
    float4 CH[32];           // phase (or void) half-space
    float Cdc[32][3];        // cell centre - face centre
    float Cw[32];
    int Ct0[32];             // first tetrahedron
    int Cend[32];            // running count of tetrahedra, inclusive
    unsigned short Sm[MX_STACK];  // piece: t | k << 5 | planes still to clip << 10
    unsigned short Q[MX_QUEUE];   // clip job: t | k << 5 | plane mask << 10
    unsigned short PQ[VOF_MAXFP * MX_CAND];  // (prism, candidate) pairs with overlapping boxes
    unsigned char KuseH[MX_CAND];
    unsigned char CuseH[32];
};

__device__ __forceinline__ FTet ldT(const FTet &t)
{
    const float4 *p = reinterpret_cast<const float4 *>(&t);
    const float4 a = p[0], b = p[1], c = p[2];
    return FTet{{f3(a.x, a.y, a.z), f3(a.w, b.x, b.y), f3(b.z, b.w, c.x), f3(c.y, c.z, c.w)}};
}

__device__ __forceinline__ void stT(FTet &t, const FTet &v)
{
    float4 *p = reinterpret_cast<float4 *>(&t);
    p[0] = make_float4(v.v[0].x, v.v[0].y, v.v[0].z, v.v[1].x);
    p[1] = make_float4(v.v[1].y, v.v[1].z, v.v[2].x, v.v[2].y);
    p[2] = make_float4(v.v[2].z, v.v[3].x, v.v[3].y, v.v[3].z);
}

// signed distances of the vertices to plane p, those within tol taken as 0;
// nin / nup count the vertices strictly below / above
__device__ __forceinline__ void fdist(const FTet &t, float4 p, float tol, float s[4], int &nin, int &nup)
{
    nin = 0;
    nup = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float v = p.x * t.v[i].x + p.y * t.v[i].y + p.z * t.v[i].z - p.w;
        if (fabsf(v) <= tol) v = 0.0f;
        s[i] = v;
        nin += v < 0.0f;
        nup += v > 0.0f;
    }
}

// the part of t below the plane (distances s, 1 <= nin <= 3 vertices strictly
// below, at least one strictly above) as one tetrahedron (nin == 1) or three,
// each handed to put(tet, i); vertices are ordered below-first by a
// compare-exchange network so that every index stays static
template <class Put>
__device__ __forceinline__ void fsplit(const FTet &t, const float s[4], int nin, Put put)
{
    F3 P0 = t.v[0], P1 = t.v[1], P2 = t.v[2], P3 = t.v[3];
    float S0 = s[0], S1 = s[1], S2 = s[2], S3 = s[3];
#define MX_CX(a, b)                                                   \
    if (!(S##a < 0.0f) && S##b < 0.0f) {                              \
        F3 tp = P##a; P##a = P##b; P##b = tp;                         \
        float ts = S##a; S##a = S##b; S##b = ts;                      \
    }
    MX_CX(0, 1) MX_CX(2, 3) MX_CX(0, 2) MX_CX(1, 3) MX_CX(1, 2)
#undef MX_CX
    auto ep = [](F3 a, float sa, F3 b, float sb) { return a + (b - a) * __fdividef(sa, sa - sb); };
    if (nin == 1) {
        put(FTet{{P0, ep(P0, S0, P1, S1), ep(P0, S0, P2, S2), ep(P0, S0, P3, S3)}}, 0);
        return;
    }
    F3 a0, a1, a2, b0, b1, b2;
    if (nin == 2) {
        a0 = P0; a1 = ep(P0, S0, P2, S2); a2 = ep(P0, S0, P3, S3);
        b0 = P1; b1 = ep(P1, S1, P2, S2); b2 = ep(P1, S1, P3, S3);
    } else {
        a0 = P0; a1 = P1; a2 = P2;
        b0 = ep(P0, S0, P3, S3); b1 = ep(P1, S1, P3, S3); b2 = ep(P2, S2, P3, S3);
    }
    put(FTet{{a0, a1, a2, b2}}, 0);
    put(FTet{{a0, a1, b2, b1}}, 1);
    put(FTet{{a0, b0, b1, b2}}, 2);
}

// The queued clip jobs, worked through by the whole warp, one piece per lane
// and step.  Pieces with one plane left (leaves) stack up from the bottom of S,
// the others down from its top, and a step works on one kind only, so that the
// lanes run the same code:
//  - leaf step: a piece adds its volume below its last plane (closed-form cut
//    fraction);
//  - split step: a piece from the other stack (else a new job) is cut by its
//    next plane and the parts below are pushed, to the leaves if one plane is
//    left.
// A split step commits the longest prefix of lanes that leaves the two stacks
// at most MX_STACK - 6 full; if none does, the top piece alone when it fits,
// else a leaf step runs first (leaves need no room).  Every part of a split
// piece has at most 4 planes to go, so the split pieces keep i + 1 + 2 (r - 1)
// <= MX_STACK for depth i and r planes to go: the top one alone always fits
// once the leaves are gone, and the stacks cannot overflow.
template <class Wk>
__device__ __forceinline__ void mx_clip(MXShared &sh, int nq, float tol, float &accs, float &accc, Wk &wk)
{
    const int lane = threadIdx.x & 31;
    const unsigned le = ((1u << lane) << 1) - 1u;
    __syncwarp();
    int nl = 0, nn = 0, qn = 0;
    bool force_leaf = false;
    for (;;) {
        const bool more = nn > 0 || qn < nq;
        if (!more && nl == 0) break;
        if (force_leaf || nl >= 32 || !more) {
            // ---- leaf step
            force_leaf = false;
            const int p = min(nl, 32);
            if (lane < p) {
                const FTet t = ldT(sh.S[nl - 1 - lane]);
                const unsigned meta = sh.Sm[nl - 1 - lane];
                const int ti = meta & 31, k = (meta >> 5) & 31, j = __ffs(meta >> 10) - 1;
                float sd[4];
                int nin, nup;
                fdist(t, sh.Kp[k][j], tol, sd, nin, nup);
                wk.add(WK_TEST, 1);
                float v6 = 0.0f;
                if (nin > 0) {
                    v6 = fabsf(fvol6(t.v[0], t.v[1], t.v[2], t.v[3]));
                    wk.add(WK_VOL, 1);
                    if (nup > 0) {
                        wk.add(WK_FRAC, 1);
                        float h0 = sd[0], h1 = sd[1], h2 = sd[2], h3 = sd[3];
                        fsort4(h0, h1, h2, h3);
                        v6 *= ffrac_below(h0, h1, h2, h3);
                    }
                }
                if (v6 != 0.0f) two_sum(accs, accc, sh.Tsg[ti] * sh.Kw[k] * v6);
            }
            nl -= p;
            __syncwarp();
            continue;
        }
        // ---- split step
        const int p = min(nn, 32), r = min(32 - p, nq - qn);
        const bool act = lane < p + r;
        FTet t;
        unsigned meta = 0;
        if (lane < p) {
            t = ldT(sh.S[MX_STACK - nn + lane]);
            meta = sh.Sm[MX_STACK - nn + lane];
        } else if (act) {
            meta = sh.Q[qn + lane - p];
            t = ldT(sh.T[meta & 31]);
        }
        __syncwarp();  // every piece read before the pushes reuse the slots
        int nch = 0, nin = 0, nup = 0, ti = 0, k = 0;
        unsigned rem = 0;
        float sd[4], v6 = 0.0f;
        bool cut = false;
        unsigned lw = 0;  // this lane's leaf work: 1 volume, 2 cut fraction
        if (act) {
            ti = meta & 31;
            k = (meta >> 5) & 31;
            rem = meta >> 10;
            const int j = __ffs(rem) - 1;
            rem &= rem - 1;
            fdist(t, sh.Kp[k][j], tol, sd, nin, nup);
            if (nin > 0) {
                if (nup > 0) cut = true;
                if (rem != 0) nch = nup == 0 || nin == 1 ? 1 : 3;
                else {  // a job with one plane: its leaf here
                    v6 = fabsf(fvol6(t.v[0], t.v[1], t.v[2], t.v[3]));
                    lw = 1;
                    if (nup > 0) {
                        lw = 3;
                        float h0 = sd[0], h1 = sd[1], h2 = sd[2], h3 = sd[3];
                        fsort4(h0, h1, h2, h3);
                        v6 *= ffrac_below(h0, h1, h2, h3);
                    }
                }
            }
        }
        const bool toleaf = (rem & (rem - 1)) == 0;  // one plane left after this one
        const unsigned b0 = __ballot_sync(0xffffffffu, nch & 1), b1 = __ballot_sync(0xffffffffu, nch & 2);
        const unsigned bl = __ballot_sync(0xffffffffu, toleaf);
        const int inc = __popc(b0 & le) + 2 * __popc(b1 & le);
        const bool fits = act && nl + nn - min(lane + 1, p) + inc <= MX_STACK - 6;
        const unsigned fm = __ballot_sync(0xffffffffu, fits);
        int L = fm ? 32 - __clz(fm) : 0;
        if (L == 0) {
            const int nch0 = __shfl_sync(0xffffffffu, nch, 0);
            if (nl + nn - (p > 0 ? 1 : 0) + nch0 <= MX_STACK) L = 1;
            else { force_leaf = true; continue; }  // nothing written: the leaves first
        }
        const unsigned lm = L >= 32 ? 0xffffffffu : (1u << L) - 1u;
        const int top = MX_STACK - nn + min(L, p);  // the split stack's top after the pops
        if (lane < L) {
            // work of the committed lanes (the others redo theirs later)
            wk.add(WK_TEST, 1);
            wk.add(WK_VOL, lw & 1);
            wk.add(WK_FRAC, lw >> 1);
            if (cut && nch > 0) wk.add(WK_EDGE, nin == 2 ? 4 : 3);
            if (v6 != 0.0f) two_sum(accs, accc, sh.Tsg[ti] * sh.Kw[k] * v6);
            if (nch > 0) {
                const unsigned cm = (unsigned)ti | ((unsigned)k << 5) | (rem << 10);
                // parts of the lanes before this one that go the same way
                const unsigned same = (toleaf ? bl : ~bl) & ((1u << lane) - 1u);
                const int before = __popc(b0 & same) + 2 * __popc(b1 & same);
                auto put = [&](const FTet &c, int i) {
                    const int at = toleaf ? nl + before + i : top - 1 - before - i;
                    stT(sh.S[at], c);
                    sh.Sm[at] = (unsigned short)cm;
                };
                if (nup == 0) put(t, 0);
                else fsplit(t, sd, nin, put);
            }
        }
        nl += __popc(b0 & bl & lm) + 2 * __popc(b1 & bl & lm);
        nn = MX_STACK - top + __popc(b0 & ~bl & lm) + 2 * __popc(b1 & ~bl & lm);
        qn += max(0, L - p);
        __syncwarp();
    }
}

// All (T, K) pairs of the buffered candidates, taken a prism (the three
// tetrahedra of one swept face triangle) at a time.  First lane k tests
// candidate k's box against each prism's box and the overlapping (prism, K)
// pairs are listed; then each listed pair, one per lane, gets the signed
// distances of the prism's six points to K's planes, from which each of its
// three tetrahedra is classified: outside a plane, inside every plane (adds
// |T| at once), or a clip job.
template <class Wk>
__device__ __forceinline__ void mx_flush(MXShared &sh, int nt, int ncand, float tol, float &accs, float &accc,
                                         Wk &wk)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int nprism = nt / 3;
    int total = 0;
    {
        float kb[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) kb[q] = lane < ncand ? sh.Kb[lane][q] : 0.0f;
        for (int pr = 0; pr < nprism; ++pr) {
            const float *tb = sh.Pb[pr];
            const bool live = sh.Tsg[3 * pr] != 0.0f || sh.Tsg[3 * pr + 1] != 0.0f || sh.Tsg[3 * pr + 2] != 0.0f;
            const bool ov = lane < ncand && live &&
                            !(tb[3] < kb[0] || kb[3] < tb[0] || tb[4] < kb[1] || kb[4] < tb[1] || tb[5] < kb[2] ||
                              kb[5] < tb[2]);
            const unsigned bm = __ballot_sync(0xffffffffu, ov);
            if (ov) sh.PQ[total + __popc(bm & lt)] = (unsigned short)(pr | lane << 3);
            total += __popc(bm);
        }
    }
    __syncwarp();
    int nq = 0;
    for (int pb = 0; pb < total; pb += 32) {
        const int pi = pb + lane;
        unsigned code[3] = {0u, 0u, 0u};
        bool job[3] = {false, false, false};
        if (pi < total) {
            const unsigned pc = sh.PQ[pi];
            const int pr = pc & 7, k = pc >> 3;
            float v[20];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const float4 q = sh.P6[pr][i];
                v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
            }
            const int npl = sh.KuseH[k] ? 5 : 4;
            wk.add(WK_PRISM, npl);
            unsigned mask[3] = {0u, 0u, 0u};
            bool outside[3] = {false, false, false};
            // a point within tol of a plane is on it: a tetrahedron is outside
            // when none of its points is clearly inside a plane, and a plane cuts
            // it only when its points lie clearly on both sides
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const float4 pl = sh.Kp[k][q];
                float d[6];
#pragma unroll
                for (int i = 0; i < 6; ++i)
                    d[i] = fmaf(pl.x, v[3 * i], fmaf(pl.y, v[3 * i + 1], fmaf(pl.z, v[3 * i + 2], -pl.w)));
                // T0 = a0 a1 a2 b2, T1 = a0 a1 b2 b1, T2 = a0 b0 b1 b2
                const float l01 = fminf(d[0], d[1]), h01 = fmaxf(d[0], d[1]);
                const float lo0 = fminf(l01, fminf(d[2], d[5])), hi0 = fmaxf(h01, fmaxf(d[2], d[5]));
                const float lo1 = fminf(l01, fminf(d[5], d[4])), hi1 = fmaxf(h01, fmaxf(d[5], d[4]));
                const float lo2 = fminf(fminf(d[0], d[3]), fminf(d[4], d[5])), hi2 = fmaxf(fmaxf(d[0], d[3]), fmaxf(d[4], d[5]));
                if (q < npl) {
                    outside[0] |= lo0 >= -tol; outside[1] |= lo1 >= -tol; outside[2] |= lo2 >= -tol;
                    if (hi0 > tol) mask[0] |= 1u << q;
                    if (hi1 > tol) mask[1] |= 1u << q;
                    if (hi2 > tol) mask[2] |= 1u << q;
                }
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int t = 3 * pr + j;
                const float sg = sh.Tsg[t];
                if (sg != 0.0f && !outside[j]) {
                    if (mask[j] == 0) two_sum(accs, accc, sg * sh.Kw[k] * sh.Tv6[t]);
                    else { job[j] = true; code[j] = (unsigned)t | ((unsigned)k << 5) | (mask[j] << 10); }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const unsigned bm = __ballot_sync(0xffffffffu, job[j]);
            if (job[j]) sh.Q[nq + __popc(bm & lt)] = (unsigned short)code[j];
            nq += __popc(bm);
        }
    }
    if (nq > 0) mx_clip(sh, nq, tol, accs, accc, wk);
    __syncwarp();
}

// W warps (faces) per block; blocks per SM as shared memory allows
constexpr int mx_resident(int w) { return w == 1 ? 15 : w == 2 ? 8 : 5; }

template <bool LIST, int W, class Wk>
__global__ void __launch_bounds__(W * 32, mx_resident(W)) k_phase_flux_mixed(DevMesh m, MXArgs a)
{
    __shared__ MXShared shm[W];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    MXShared &sh = shm[wib];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int total = LIST ? *a.count : m.nf;
    const double eps = m.eps;
    // Band faces differ in cost by an order of magnitude (a face whose
    // polyhedron cuts interface cells clips, one among uniform cells hardly
    // does): in the list form a warp takes its next face from a counter as it
    // finishes one, so that no warp ends long after the others; a face's flux
    // is one warp's work either way.
    const bool dyn = LIST && a.next != nullptr;
    auto take = [&]() {
        int v = 0;
        if (lane == 0) v = atomicAdd(a.next, 1);
        return __shfl_sync(0xffffffffu, v, 0);
    };
    Wk wk;
    for (int item = dyn ? take() : warp; item < total; item = dyn ? take() : item + nwarps) {
        const int f = LIST ? a.list[item] : item;
        const long long s0 = __ldg(m.sptr + f), s1 = __ldg(m.sptr + f + 1);
        if (!LIST) {
            double Ff = a.F[f];
            bool all_e = true, all_f = true;
            for (long long s = s0 + lane; s < s1; s += 32) {
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
        // empty cells exactly 0, and FP32 rounding stays with mixed cells.  Not
        // where the polyhedron can leave the domain (the normal-sweep fallback at
        // walls; a face touching an open boundary), since the part outside is
        // empty and the stencil does not cover it.
        const double Ff = a.F[f];
        const int up = Ff > 0.0 ? __ldg(m.own + f) : (f < m.ni ? __ldg(m.nei + f) : __ldg(m.own + f));
        const double lamf = LIST ? a.lam_b[item] : a.lambda[f];
        const bool comp = a.alpha[up] >= 0.5 && lamf >= 0.0 && !__ldg(m.fopen + f);
        const int nt = n == 3 ? 3 : 3 * n;
        // signed distances (to unit-normal planes) within 2e-6 of the face size are
        // taken as zero: points shared by the polyhedron and the cell tetrahedra
        // come out of different FP32 roundings and would otherwise look like cuts
        const float tol = __ldg(a.fpl + b).w;
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
            stT(sh.T[lane], T);
            sh.Tsg[lane] = sv > 0.0f ? 1.0f : (sv < 0.0f ? -1.0f : 0.0f);
            sh.Tv6[lane] = fabsf(v6);
            bx[0] = fminf(fminf(T.v[0].x, T.v[1].x), fminf(T.v[2].x, T.v[3].x));
            bx[1] = fminf(fminf(T.v[0].y, T.v[1].y), fminf(T.v[2].y, T.v[3].y));
            bx[2] = fminf(fminf(T.v[0].z, T.v[1].z), fminf(T.v[2].z, T.v[3].z));
            bx[3] = fmaxf(fmaxf(T.v[0].x, T.v[1].x), fmaxf(T.v[2].x, T.v[3].x));
            bx[4] = fmaxf(fmaxf(T.v[0].y, T.v[1].y), fmaxf(T.v[2].y, T.v[3].y));
            bx[5] = fmaxf(fmaxf(T.v[0].z, T.v[1].z), fmaxf(T.v[2].z, T.v[3].z));
            if (j == 0) {
                float *q = reinterpret_cast<float *>(sh.P6[pr]);
                const F3 pv[6] = {a0, a1, a2, b0, b1, b2};
#pragma unroll
                for (int i = 0; i < 6; ++i) { q[3 * i] = pv[i].x; q[3 * i + 1] = pv[i].y; q[3 * i + 2] = pv[i].z; }
                float lo3[3] = {3e38f, 3e38f, 3e38f}, hi3[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    lo3[0] = fminf(lo3[0], pv[i].x); lo3[1] = fminf(lo3[1], pv[i].y); lo3[2] = fminf(lo3[2], pv[i].z);
                    hi3[0] = fmaxf(hi3[0], pv[i].x); hi3[1] = fmaxf(hi3[1], pv[i].y); hi3[2] = fmaxf(hi3[2], pv[i].z);
                }
                for (int i = 0; i < 3; ++i) { sh.Pb[pr][i] = lo3[i]; sh.Pb[pr][3 + i] = hi3[i]; }
            }
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
        wk.add(WK_VOL, lane < nt);  // the flux polyhedron's tetrahedra
        wk.face();
        int ncand = 0;
        // The stencil is taken 32 cells at a time, one per lane: the cells that
        // reach the polyhedron's box are kept (with their half-space) in shared
        // memory, then their tetrahedra come 32 at a time into the candidate
        // buffer. A batch that does not fit is produced again after the buffer
        // has been processed, so that the buffer is processed at one place and
        // no candidate is held across it.
        long long sc = s0 - 32;
        int tb = 0, ntot = 0, ncell = 0;
        for (;;) {
            if (tb >= ntot) {  // the chunk's tetrahedra are done: next chunk
                sc += 32;
                tb = 0;
                ntot = 0;
                if (sc < s1) {
                    const long long s = sc + lane;
                    bool pass = false;
                    int c = 0;
                    double al = 0.0;
                    F3 dc = f3(0.f, 0.f, 0.f);
                    if (s < s1) {
                        c = __ldg(m.scell + s);
                        al = a.alpha[c];
                        // an empty cell carries no phase, a full cell no void
                        if (!((!comp && al <= eps) || (comp && al >= 1.0 - eps))) {
                            const V3 cc = ld3(m.cc, m.nc, c);
                            dc = f3((float)(cc.x - o.x), (float)(cc.y - o.y), (float)(cc.z - o.z));
                            const float4 cb0 = __ldg(a.cbl + 2 * (size_t)c), cb1 = __ldg(a.cbl + 2 * (size_t)c + 1);
                            pass = !(cb1.x + dc.x < pb[0] || pb[3] < cb0.x + dc.x || cb1.y + dc.y < pb[1] ||
                                     pb[4] < cb0.y + dc.y || cb1.z + dc.z < pb[2] || pb[5] < cb0.z + dc.z);
                        }
                    }
                    int nkt = 0, t0 = 0;
                    float wgt = 1.0f;
                    bool useH = false;
                    float4 H = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (pass) {
                        t0 = __ldg(a.ctptr + c);
                        nkt = __ldg(a.ctptr + c + 1) - t0;
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
                    }
                    int inc = nkt;
#pragma unroll
                    for (int o2 = 1; o2 < 32; o2 <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, inc, o2);
                        if (lane >= o2) inc += v;
                    }
                    const unsigned pm = __ballot_sync(0xffffffffu, pass);
                    if (pass) {
                        const int r = __popc(pm & ((1u << lane) - 1u));
                        sh.CH[r] = H;
                        sh.Cdc[r][0] = dc.x; sh.Cdc[r][1] = dc.y; sh.Cdc[r][2] = dc.z;
                        sh.Cw[r] = wgt;
                        sh.CuseH[r] = useH;
                        sh.Ct0[r] = t0;
                        sh.Cend[r] = inc;
                    }
                    ntot = __shfl_sync(0xffffffffu, inc, 31);
                    ncell = __popc(pm);
                    __syncwarp();
                    continue;
                }
            }
            const bool fin = sc >= s1;
            bool cand = false;
            int ci = 0;
            float4 kp[4];
            float kbx[6];
            if (!fin) {
                // the cell of tetrahedron tb + lane: the cells that end at or
                // before tb, plus one for each cell that ends inside the batch at
                // or before this lane (cell 'lane' ends rel tetrahedra after tb)
                const int rel = lane < ncell ? sh.Cend[lane] - tb : 0x7fffffff;
                const unsigned ends = __reduce_or_sync(0xffffffffu, rel > 0 && rel < 32 ? 1u << rel : 0u);
                ci = __popc(__ballot_sync(0xffffffffu, rel <= 0)) + __popc(ends & (((1u << lane) << 1) - 1u));
            }
            if (!fin && tb + lane < ntot) {
                // this lane's tetrahedron: planes and box move from the cell frame
                // to the face frame by the shift dc
                const int g = tb + lane;
                const int j = sh.Ct0[ci] + g - (ci ? sh.Cend[ci - 1] : 0);
                const F3 dc = f3(sh.Cdc[ci][0], sh.Cdc[ci][1], sh.Cdc[ci][2]);
                const float4 *q = a.ktl + 6 * (size_t)j;
                const float4 b0 = __ldg(q + 4), b1 = __ldg(q + 5);
                kbx[0] = b0.x + dc.x; kbx[1] = b0.y + dc.y; kbx[2] = b0.z + dc.z;
                kbx[3] = b1.x + dc.x; kbx[4] = b1.y + dc.y; kbx[5] = b1.z + dc.z;
                cand = !(kbx[3] < pb[0] || pb[3] < kbx[0] || kbx[4] < pb[1] || pb[4] < kbx[1] ||
                         kbx[5] < pb[2] || pb[5] < kbx[2]);
                if (cand) {
                    wk.add(WK_SHIFT, 4);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 pl = __ldg(q + i);
                        kp[i] = make_float4(pl.x, pl.y, pl.z, pl.w + (pl.x * dc.x + pl.y * dc.y + pl.z * dc.z));
                    }
                }
            }
            const unsigned cmask = __ballot_sync(0xffffffffu, cand);
            if (fin ? ncand > 0 : ncand + __popc(cmask) > MX_CAND) {
                mx_flush(sh, nt, ncand, tol, accs, accc, wk);
                ncand = 0;
                continue;  // the batch again (or the end)
            }
            if (fin) break;
            if (cand) {
                int r = ncand + __popc(cmask & ((1u << lane) - 1u));
                for (int q = 0; q < 4; ++q) sh.Kp[r][q] = kp[q];
                for (int q = 0; q < 6; ++q) sh.Kb[r][q] = kbx[q];
                sh.Kp[r][4] = sh.CH[ci];
                sh.Kw[r] = sh.Cw[ci];
                sh.KuseH[r] = sh.CuseH[ci];
            }
            ncand += __popc(cmask);
            tb += 32;
            __syncwarp();
        }
        // lane sums and compensations merged across the warp by TwoSum, then the
        // 1/6 of the volumes in FP64
        float rs = accs, rc = accc;
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            const float xs = __shfl_xor_sync(0xffffffffu, rs, o2), xc = __shfl_xor_sync(0xffffffffu, rc, o2);
            two_sum(rs, rc, xs);
            rc += xc;
        }
        double acc = ((double)rs + (double)rc) / 6.0;
        if (comp) acc = Ff * a.dt - acc;
        if (lane == 0) a.Va[f] = acc;
        __syncwarp();
    }
    wk.flush(a.work, lane);
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

// the tetrahedra of every cell (cell centre + fan triangle of a face, in the
// order of the cell's faces and of the face's points) as 4 outward unit-normal
// planes and a box, in the cell frame (context creation)
__global__ void k_cell_tets(DevMesh m, const int *cfpptr, const float4 *cfl, const float4 *cfpl, const int *ctptr,
                            float4 *ktl)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    int o = cfpptr[c], j = ctptr[c];
    for (int k = m.cptr[c]; k < m.cptr[c + 1]; ++k) {
        const int code = m.cface[k], g = code >> 1, gn = m.fptr[g + 1] - m.fptr[g];
        for (int i = 0; i < (gn == 3 ? 1 : gn); ++i, ++j) {
            F3 k0 = f3(0.f, 0.f, 0.f), k1, k2, k3;
            if (gn == 3) {
                k1 = ld4(cfpl, o); k2 = ld4(cfpl, o + 1); k3 = ld4(cfpl, o + 2);
            } else {
                k1 = ld4(cfl, k); k2 = ld4(cfpl, o + i); k3 = ld4(cfpl, o + (i + 1 == gn ? 0 : i + 1));
            }
            if (code & 1) { F3 t = k2; k2 = k3; k3 = t; }
            F3 n0 = fcross(k2 - k0, k1 - k0), n1 = fcross(k1 - k0, k3 - k0);
            F3 n2 = fcross(k3 - k0, k2 - k0), n3 = fcross(k2 - k1, k3 - k1);
            n0 = n0 * rsqrtf(fdot(n0, n0) + 1e-37f); n1 = n1 * rsqrtf(fdot(n1, n1) + 1e-37f);
            n2 = n2 * rsqrtf(fdot(n2, n2) + 1e-37f); n3 = n3 * rsqrtf(fdot(n3, n3) + 1e-37f);
            float4 *q = ktl + 6 * (size_t)j;
            q[0] = make_float4(n0.x, n0.y, n0.z, 0.f);
            q[1] = make_float4(n1.x, n1.y, n1.z, 0.f);
            q[2] = make_float4(n2.x, n2.y, n2.z, 0.f);
            q[3] = make_float4(n3.x, n3.y, n3.z, fdot(n3, k1));
            q[4] = make_float4(fminf(fminf(k0.x, k1.x), fminf(k2.x, k3.x)), fminf(fminf(k0.y, k1.y), fminf(k2.y, k3.y)),
                               fminf(fminf(k0.z, k1.z), fminf(k2.z, k3.z)), 0.f);
            q[5] = make_float4(fmaxf(fmaxf(k0.x, k1.x), fmaxf(k2.x, k3.x)), fmaxf(fmaxf(k0.y, k1.y), fmaxf(k2.y, k3.y)),
                               fmaxf(fmaxf(k0.z, k1.z), fmaxf(k2.z, k3.z)), 0.f);
        }
        o += gn;
    }
}

__global__ void k_face_local(DevMesh m, float4 *fpl)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.nf) return;
    V3 c = ld3(m.cf, m.nf, f), S = ld3(m.sf, m.nf, f);
    // w of the face's first point: the on-plane band of the clipping, 2e-6 of
    // the face size
    const float tol = (float)(2e-6 * sqrt(sqrt(dot(S, S))));
    for (int j = m.fptr[f]; j < m.fptr[f + 1]; ++j) {
        V3 p = ldP(m, m.fpts[j]) - c;
        fpl[j] = make_float4((float)p.x, (float)p.y, (float)p.z, j == m.fptr[f] ? tol : 0.f);
    }
}

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

}  // namespace

int launch_setup_mixed(vof_ctx *c, cudaStream_t s)
{
    k_local_geom<<<cdiv(c->nc, 256), 256, 0, s>>>(c->m, c->cfpptr, c->cfl, c->cfpl, c->cbl);
    k_face_local<<<cdiv(c->nf, 256), 256, 0, s>>>(c->m, c->fpl);
    if (c->ktl)
        k_cell_tets<<<cdiv(c->nc, 256), 256, 0, s>>>(c->m, c->cfpptr, c->cfl, c->cfpl, c->m.ctptr, c->ktl);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

static MXArgs mx_args(vof_ctx *c, const double *alpha, const double *n, const double *d, const uint8_t *flags,
                      const double *Up, const double *F, const double *lambda, double dt, double *Va,
                      const int *list, const int *count, const double *disp, unsigned long long *work)
{
    return MXArgs{alpha, n, d, flags, Up, F, lambda, dt, Va, list, count, disp, c->lam_b, c->status, work,
                  c->fpl, c->cbl, c->ktl, c->m.ctptr, nullptr};
}

int launch_phase_flux_mixed_all(vof_ctx *c, const double *alpha, const double *n, const double *d,
                                const uint8_t *flags, const double *Up, const double *F, const double *lambda,
                                double dt, double *Va, cudaStream_t s)
{
    MXArgs a = mx_args(c, alpha, n, d, flags, Up, F, lambda, dt, Va, nullptr, nullptr, nullptr, nullptr);
    if (c->work_on) k_phase_flux_mixed<false, 2, WkOn><<<cdiv((long)c->nf * 32, 64), 64, 0, s>>>(c->m, a);
    else k_phase_flux_mixed<false, 2, WkOff><<<cdiv((long)c->nf * 32, 64), 64, 0, s>>>(c->m, a);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

int launch_phase_flux_mixed_list(vof_ctx *c, const double *alpha, const double *F, double dt, int sms,
                                 cudaStream_t s)
{
    MXArgs a = mx_args(c, alpha, c->n, c->d, c->flags, nullptr, F, nullptr, dt, c->Va, c->band,
                       c->counters + CNT_BAND, c->disp_b, c->work);
    a.next = c->counters + CNT_PFNEXT;  // zeroed with the step's counters
    // launch configuration (vof_batch_tune): warps per block, and grid = SMs x
    // resident blocks x multiplier
    const int w = c->pf_warps >= 1 && c->pf_warps <= 3 ? c->pf_warps : 2;
    const int mult = c->pf_mult >= 1 ? c->pf_mult : 1;
    if (c->work_on)  // instrumented variant (vof_count_work), the 2-warp shape
        k_phase_flux_mixed<true, 2, WkOn><<<sms * mx_resident(2) * mult, 64, 0, s>>>(c->m, a);
    else if (w == 1)
        k_phase_flux_mixed<true, 1, WkOff><<<sms * mx_resident(1) * mult, 32, 0, s>>>(c->m, a);
    else if (w == 2)
        k_phase_flux_mixed<true, 2, WkOff><<<sms * mx_resident(2) * mult, 64, 0, s>>>(c->m, a);
    else
        k_phase_flux_mixed<true, 3, WkOff><<<sms * mx_resident(3) * mult, 96, 0, s>>>(c->m, a);
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

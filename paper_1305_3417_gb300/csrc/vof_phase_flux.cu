// Phase flux (A6, Eqs. S'_f, S''_f): the flux-polyhedron tetrahedra T of a
// band face, the cell tetrahedra K of its stencil cells and their PLIC planes
// are taken to a frame centred on the face centre and intersected there, one
// warp per face.  One source for both forms:
//  - mixed (R = float): FP32 clipping, pieces summed per lane with TwoSum
//    compensation and finished in FP64 (reading R13 on the on-plane band);
//  - plain (R = double): the same structure in FP64 throughout.
//
// Only the frame shift of a stencil cell (its centre minus the face centre) and
// of its plane offset are formed in FP64; the cell's own geometry comes from
// offsets to the cell centre computed once at context creation, so the
// rounding of a coordinate is relative to the cell size, not to its position.
#include <cuda_runtime.h>

#include <type_traits>
#include <math.h>
#include <stdint.h>

#include "vof_device.cuh"
#include "vof_internal.h"

namespace {
using namespace vofd;

// ------------------------------------------------------------ real types
template <class R>
struct R3 { R x, y, z; };
struct __align__(16) D4 { double x, y, z, w; };
template <class R> struct Q4;
template <> struct Q4<float> { using T = float4; };
template <> struct Q4<double> { using T = D4; };
template <class R> using R4 = typename Q4<R>::T;

template <class R> __device__ __forceinline__ R3<R> r3(R x, R y, R z) { return R3<R>{x, y, z}; }
template <class R> __device__ __forceinline__ R3<R> operator+(R3<R> a, R3<R> b) { return r3(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class R> __device__ __forceinline__ R3<R> operator-(R3<R> a, R3<R> b) { return r3(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class R> __device__ __forceinline__ R3<R> operator*(R3<R> a, R s) { return r3(a.x * s, a.y * s, a.z * s); }
template <class R> __device__ __forceinline__ R rdot(R3<R> a, R3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class R> __device__ __forceinline__ R3<R> rcross(R3<R> a, R3<R> b)
{
    return r3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <class R> __device__ __forceinline__ R rvol6(R3<R> a, R3<R> b, R3<R> c, R3<R> d)
{
    return rdot(b - a, rcross(c - a, d - a));
}
__device__ __forceinline__ float rmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double rmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float rmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float rabs(float a) { return fabsf(a); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rnext(float a, float b) { return nextafterf(a, b); }
__device__ __forceinline__ double rnext(double a, double b) { return nextafter(a, b); }
__device__ __forceinline__ double rabs(double a) { return fabs(a); }
// divisions of the clip: the fast FP32 reciprocal-multiply (2 ulp, far inside
// the mixed form's rounding) or a correctly rounded FP64 division
__device__ __forceinline__ float rdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return a / b; }

template <class R> __device__ __forceinline__ R4<R> mk4(R x, R y, R z, R w);
template <> __device__ __forceinline__ float4 mk4<float>(float x, float y, float z, float w) { return make_float4(x, y, z, w); }
template <> __device__ __forceinline__ D4 mk4<double>(double x, double y, double z, double w) { return D4{x, y, z, w}; }
__device__ __forceinline__ float4 ldg4(const float4 *p, long i) { return __ldg(p + i); }
__device__ __forceinline__ D4 ldg4(const D4 *p, long i)
{
    const double2 *q = reinterpret_cast<const double2 *>(p + i);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    return D4{a.x, a.y, b.x, b.y};
}
template <class R> __device__ __forceinline__ R3<R> ld43(const R4<R> *p, long i)
{
    const R4<R> v = ldg4(p, i);
    return r3<R>(v.x, v.y, v.z);
}

// Threshold, sign and order tests of distances (tol >= 0).  FP32: the native
// compares.  FP64: integer compares of the bit patterns (dbits), the same
// decisions for every value that is not NaN: this part's FP64 pipe runs at
// 1/64 of the FP32 rate, and an FP64 compare or min/max holds it as long as
// an FMA.
__device__ __forceinline__ bool rpos(float v) { return v > 0.0f; }
__device__ __forceinline__ bool rneg(float v) { return v < 0.0f; }
__device__ __forceinline__ bool rgt(float a, float b) { return a > b; }
__device__ __forceinline__ bool rabove(double v, double t) { return gt_pos(v, t); }   // v > t
__device__ __forceinline__ bool rbelow(double v, double t) { return lt_neg(v, t); }   // v < -t
__device__ __forceinline__ bool rpos(double v) { return gt_pos(v, 0.0); }
__device__ __forceinline__ bool rneg(double v) { return lt_neg(v, 0.0); }
// a > b for any signs: the bit patterns made monotone by flipping the
// magnitude bits of negative values (-0 then orders just below +0)
__device__ __forceinline__ bool rgt(double a, double b)
{
    DBits x = dbits(a), y = dbits(b);
    const int sx = x.hi >> 31, sy = y.hi >> 31;
    x.hi ^= sx & 0x7fffffff; x.lo ^= (unsigned)sx;
    y.hi ^= sy & 0x7fffffff; y.lo ^= (unsigned)sy;
    return !bits_le(x, y);
}

// fraction of a tetrahedron below level 0 for sorted vertex values h0..h3
template <class R>
__device__ __forceinline__ R rfrac_below(R h0, R h1, R h2, R h3)
{
    if (!rneg(h0)) return R(0);
    if (!rpos(h3)) return R(1);
    // one division per case
    if (!rneg(h1)) {
        const R x = -h0;
        return rdiv(x * x * x, (h1 - h0) * (h2 - h0) * (h3 - h0));
    }
    if (!rpos(h2)) {
        const R y = h3;
        return R(1) - rdiv(y * y * y, (h3 - h0) * (h3 - h1) * (h3 - h2));
    }
    const R d1 = h2 - h0, d2 = h3 - h0, d3 = h2 - h1, d4 = h3 - h1;
    const R p12 = d1 * d2, p123 = p12 * d3, q = rdiv(R(1), p123 * d4);
    const R r4 = q * p123, q3 = q * d4, r3 = q3 * p12, q2 = q3 * d3, r1 = q2 * d2, r2 = q2 * d1;
    const R a = -h0 * r1, b = -h0 * r2, c = -h1 * r3, e = -h1 * r4;
    return a * b + a * (R(1) - b) * e + (R(1) - a) * c * e;
}

template <class R>
__device__ __forceinline__ void rsort4(R &a, R &b, R &c, R &d)
{
    R t;
#define CS(p, q) if (rgt(p, q)) { t = p; p = q; q = t; }
    CS(a, b) CS(c, d) CS(a, c) CS(b, d) CS(b, c)
#undef CS
}

template <class R> struct RTet { R3<R> v[4]; };

// Running sum of the pieces (6 |volume| times sign and weight): FP32 with
// TwoSum (Knuth) compensation, s + c carrying the sum up to the rounding of
// the compensation (no multiplications, so no fused operation can change it);
// FP64 plainly.  (A 64-bit fixed-point sum, exact and order-independent, cost
// 6 % of the kernel's time in its conversions.)
template <class R> struct Acc { R s = R(0), c = R(0); };
__device__ __forceinline__ void acc_add(Acc<float> &a, float x)
{
    const float t = a.s + x;
    const float bp = t - a.s;
    a.c += (a.s - (t - bp)) + (x - bp);
    a.s = t;
}
__device__ __forceinline__ void acc_add(Acc<double> &a, double x) { a.s += x; }

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
    const void *fpl, *cbl, *ktl;  // the context's tables (R4 of the form's type)
    const int *ctptr;
    int *next;                // list form: next band slot to take (zero before the launch), or null
};

constexpr int MX_CAND = 32;    // candidate cell tetrahedra buffered per warp: one per lane
constexpr int MX_QUEUE = MX_MAXT * MX_CAND;  // clip jobs: one per (T, K) pair at most
// pieces of clip jobs waiting for their next plane, per warp (the stack depth
// S is a launch choice: 92 commits more lanes per split step, 56 leaves room
// for more resident warps)
constexpr int MX_STACK_WIDE = 92, MX_STACK_SLIM = 56;

// per warp; in FP32 the 48-byte tetrahedra are moved as three float4
// (conflict-free across a warp)
template <class R, int MX_STACK>
struct __align__(16) MXShared {
    RTet<R> S[MX_STACK];     // pieces
    RTet<R> T[MX_MAXT];      // flux-polyhedron tetrahedra
    R4<R> Kp[MX_CAND][5];    // outward unit-normal planes of the candidate cell tetrahedra, then
                             // the cell's phase (or void) half-space; 80-byte rows (FP32): a warp's
                             // float4 reads of different rows are conflict-free
    R4<R> P6[VOF_MAXFP][5];  // per prism (face triangle swept): a0 a1 a2 b0 b1 b2, 18 values in 20
    R Pb[VOF_MAXFP][6];      // prism box
    R Kb[MX_CAND][6];
    R Tv6[MX_MAXT];          // |6 vol(T)|
    R Tsg[MX_MAXT];          // sign of T in the flux polyhedron
    R Kw[MX_CAND];           // weight: 1, or alpha (1-alpha) of an unoriented cell
    // stencil cells of the current chunk that reach the polyhedron's box
    R4<R> CH[32];            // phase (or void) half-space
    R Cdc[32][3];            // cell centre - face centre
    R Cw[32];
    int Ct0[32];             // first tetrahedron
    int Cend[32];            // running count of tetrahedra, inclusive
    unsigned short Sm[MX_STACK];  // piece: t | k << 5 | planes still to clip << 10
    unsigned short Q[MX_QUEUE];   // clip job: t | k << 5 | plane mask << 10
    unsigned short PQ[VOF_MAXFP * MX_CAND];  // (prism, candidate) pairs with overlapping boxes
    unsigned char KuseH[MX_CAND];
    unsigned char CuseH[32];
};

__device__ __forceinline__ RTet<float> ldT(const RTet<float> &t)
{
    const float4 *p = reinterpret_cast<const float4 *>(&t);
    const float4 a = p[0], b = p[1], c = p[2];
    return RTet<float>{{r3(a.x, a.y, a.z), r3(a.w, b.x, b.y), r3(b.z, b.w, c.x), r3(c.y, c.z, c.w)}};
}
__device__ __forceinline__ RTet<double> ldT(const RTet<double> &t) { return t; }

__device__ __forceinline__ void stT(RTet<float> &t, const RTet<float> &v)
{
    float4 *p = reinterpret_cast<float4 *>(&t);
    p[0] = make_float4(v.v[0].x, v.v[0].y, v.v[0].z, v.v[1].x);
    p[1] = make_float4(v.v[1].y, v.v[1].z, v.v[2].x, v.v[2].y);
    p[2] = make_float4(v.v[2].z, v.v[3].x, v.v[3].y, v.v[3].z);
}
__device__ __forceinline__ void stT(RTet<double> &t, const RTet<double> &v) { t = v; }

// signed distances of the vertices to plane p, those within tol taken as 0;
// nin / nup count the vertices strictly below / above
template <class R>
__device__ __forceinline__ void fdist(const RTet<R> &t, R4<R> p, R tol, R s[4], int &nin, int &nup)
{
    nin = 0;
    nup = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        R v = p.x * t.v[i].x + p.y * t.v[i].y + p.z * t.v[i].z - p.w;
        if constexpr (std::is_same<R, double>::value) {  // integer tests
            const bool up = rabove(v, tol), dn = rbelow(v, tol);
            s[i] = (up || dn) ? v : R(0);
            nin += dn;
            nup += up;
        } else {
            if (rabs(v) <= tol) v = R(0);
            s[i] = v;
            nin += v < R(0);
            nup += v > R(0);
        }
    }
}

// the part of t below the plane (distances s, 1 <= nin <= 3 vertices strictly
// below, at least one strictly above) as one tetrahedron (nin == 1) or three,
// each handed to put(tet, i); vertices are ordered below-first by a
// compare-exchange network so that every index stays static
template <class R, class Put>
__device__ __forceinline__ void fsplit(const RTet<R> &t, const R s[4], int nin, Put put)
{
    using V = R3<R>;
    V P0 = t.v[0], P1 = t.v[1], P2 = t.v[2], P3 = t.v[3];
    R S0 = s[0], S1 = s[1], S2 = s[2], S3 = s[3];
#define MX_CX(a, b)                                                   \
    if (!rneg(S##a) && rneg(S##b)) {                                  \
        V tp = P##a; P##a = P##b; P##b = tp;                          \
        R ts = S##a; S##a = S##b; S##b = ts;                          \
    }
    MX_CX(0, 1) MX_CX(2, 3) MX_CX(0, 2) MX_CX(1, 3) MX_CX(1, 2)
#undef MX_CX
    // the three or four edge parameters sa / (sa - sb) from one division
    // (the reciprocal of the denominators' product, then products): the
    // divisions hold the FP64 pipe longest, and FP32 saves issue slots
    auto ept = [](V a, V b, R t) { return a + (b - a) * t; };
    if (nin == 1) {
        const R d1 = S0 - S1, d2 = S0 - S2, d3 = S0 - S3, p12 = d1 * d2, q = rdiv(R(1), p12 * d3);
        const R r3 = q * p12, q3 = q * d3, r1 = q3 * d2, r2 = q3 * d1;
        put(RTet<R>{{P0, ept(P0, P1, S0 * r1), ept(P0, P2, S0 * r2), ept(P0, P3, S0 * r3)}}, 0);
        return;
    }
    V a0, a1, a2, b0, b1, b2;
    if (nin == 2) {
        const R d1 = S0 - S2, d2 = S0 - S3, d3 = S1 - S2, d4 = S1 - S3;
        const R p12 = d1 * d2, p123 = p12 * d3, q = rdiv(R(1), p123 * d4);
        const R r4 = q * p123, q3 = q * d4, r3 = q3 * p12, q2 = q3 * d3, r1 = q2 * d2, r2 = q2 * d1;
        a0 = P0; a1 = ept(P0, P2, S0 * r1); a2 = ept(P0, P3, S0 * r2);
        b0 = P1; b1 = ept(P1, P2, S1 * r3); b2 = ept(P1, P3, S1 * r4);
    } else {
        const R d1 = S0 - S3, d2 = S1 - S3, d3 = S2 - S3, p12 = d1 * d2, q = rdiv(R(1), p12 * d3);
        const R r3 = q * p12, q3 = q * d3, r1 = q3 * d2, r2 = q3 * d1;
        a0 = P0; a1 = P1; a2 = P2;
        b0 = ept(P0, P3, S0 * r1); b1 = ept(P1, P3, S1 * r2); b2 = ept(P2, P3, S2 * r3);
    }
    put(RTet<R>{{a0, a1, a2, b2}}, 0);
    put(RTet<R>{{a0, a1, b2, b1}}, 1);
    put(RTet<R>{{a0, b0, b1, b2}}, 2);
}

// The queued clip jobs, worked through by the whole warp, one piece per lane
// and step.  Pieces with one plane left (leaves) stack up from the bottom of S,
// the others down from its top, and a step works on one kind only, so that the
// lanes run the same code:
//  - leaf step: a piece adds its volume below its last plane (closed-form cut
//    fraction);
//  - split step: a piece from the other stack (else a new job) is cut by its
//    next plane and the parts below are pushed, to the leaves if one plane is
//    left; a new job with one plane goes to the leaves whole (no leaf work in
//    a split step: a step's lanes never mix the two kinds of work).
// A split step commits the longest prefix of lanes that leaves the two stacks
// at most MX_STACK - 6 full; if none does, the top piece alone when it fits,
// else a leaf step runs first (leaves need no room).  Every part of a split
// piece has at most 4 planes to go, so the split pieces keep i + 1 + 2 (r - 1)
// <= MX_STACK for depth i and r planes to go: the top one alone always fits
// once the leaves are gone, and the stacks cannot overflow.
template <class R, int MX_STACK, class Wk>
__device__ __forceinline__ void mx_clip(MXShared<R, MX_STACK> &sh, int nq, R tol, Acc<R> &acc, Wk &wk)
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
                const RTet<R> t = ldT(sh.S[nl - 1 - lane]);
                const unsigned meta = sh.Sm[nl - 1 - lane];
                const int ti = meta & 31, k = (meta >> 5) & 31, j = __ffs(meta >> 10) - 1;
                R sd[4];
                int nin, nup;
                fdist(t, sh.Kp[k][j], tol, sd, nin, nup);
                wk.add(WK_TEST, 1);
                R v6 = R(0);
                if (nin > 0) {
                    v6 = rabs(rvol6(t.v[0], t.v[1], t.v[2], t.v[3]));
                    wk.add(WK_VOL, 1);
                    if (nup > 0) {
                        wk.add(WK_FRAC, 1);
                        R h0 = sd[0], h1 = sd[1], h2 = sd[2], h3 = sd[3];
                        rsort4(h0, h1, h2, h3);
                        v6 *= rfrac_below(h0, h1, h2, h3);
                    }
                }
                if (rpos(v6)) acc_add(acc, sh.Tsg[ti] * sh.Kw[k] * v6);  // (v6 >= 0)
            }
            nl -= p;
            __syncwarp();
            continue;
        }
        // ---- split step
        const int p = min(nn, 32), r = min(32 - p, nq - qn);
        const bool act = lane < p + r;
        RTet<R> t;
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
        R sd[4];
        bool cut = false, single = false;
        if (act) {
            ti = meta & 31;
            k = (meta >> 5) & 31;
            rem = meta >> 10;
            single = (rem & (rem - 1)) == 0;
            if (single) nch = 1;  // a job with one plane goes to the leaves whole
            else {
                const int j = __ffs(rem) - 1;
                rem &= rem - 1;
                fdist(t, sh.Kp[k][j], tol, sd, nin, nup);
                if (nin > 0) {
                    if (nup > 0) cut = true;
                    nch = nup == 0 || nin == 1 ? 1 : 3;
                }
            }
        }
        const bool toleaf = single || (rem & (rem - 1)) == 0;  // one plane left after this one
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
            wk.add(WK_TEST, !single);
            if (cut && nch > 0) wk.add(WK_EDGE, nin == 2 ? 4 : 3);
            if (nch > 0) {
                const unsigned cm = (unsigned)ti | ((unsigned)k << 5) | (rem << 10);
                // parts of the lanes before this one that go the same way
                const unsigned same = (toleaf ? bl : ~bl) & ((1u << lane) - 1u);
                const int before = __popc(b0 & same) + 2 * __popc(b1 & same);
                auto put = [&](const RTet<R> &c, int i) {
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
template <class R, int MX_STACK, class Wk>
__device__ __forceinline__ void mx_flush(MXShared<R, MX_STACK> &sh, int nt, int ncand, R tol, Acc<R> &acc,
                                         Wk &wk)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int nprism = nt / 3;
    int total = 0;
    {
        R kb[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) kb[q] = lane < ncand ? sh.Kb[lane][q] : R(0);
        for (int pr = 0; pr < nprism; ++pr) {
            const R *tb = sh.Pb[pr];
            const bool live = sh.Tsg[3 * pr] != R(0) || sh.Tsg[3 * pr + 1] != R(0) || sh.Tsg[3 * pr + 2] != R(0);
            const bool ov = lane < ncand && live &&
                            !(rgt(kb[0], tb[3]) || rgt(tb[0], kb[3]) || rgt(kb[1], tb[4]) || rgt(tb[1], kb[4]) ||
                              rgt(kb[2], tb[5]) || rgt(tb[2], kb[5]));
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
            R v[20];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const R4<R> q = sh.P6[pr][i];
                v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
            }
            const int npl = sh.KuseH[k] ? 5 : 4;
            wk.add(WK_PRISM, npl);
            unsigned mask[3] = {0u, 0u, 0u};
            bool outside[3] = {false, false, false};
            // a point within tol of a plane is on it: a tetrahedron is outside
            // when none of its points is clearly inside a plane, and a plane cuts
            // it only when its points lie clearly on both sides.  FP64: a rolled
            // loop over the pair's planes (the unrolled body's instruction
            // footprint cost 13 % of the launch); FP32: unrolled over five
            constexpr bool F64 = std::is_same<R, double>::value;
#pragma unroll(F64 ? 1 : 5)
            for (int q = 0; q < (F64 ? npl : 5); ++q) {
                const R4<R> pl = sh.Kp[k][q];
                R d[6];
#pragma unroll
                for (int i = 0; i < 6; ++i)
                    d[i] = rfma(pl.x, v[3 * i], rfma(pl.y, v[3 * i + 1], rfma(pl.z, v[3 * i + 2], -pl.w)));
                // T0 = a0 a1 a2 b2, T1 = a0 a1 b2 b1, T2 = a0 b0 b1 b2
                if constexpr (std::is_same<R, double>::value) {
                    // the points not clearly inside the plane (ge) and those
                    // clearly outside it (gt) as bits 0..5 = a0 a1 a2 b0 b1 b2,
                    // from integer tests (no FP64 compare or min/max)
                    unsigned ge = 0u, gt = 0u;
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        ge |= (unsigned)!rbelow(d[i], tol) << i;
                        gt |= (unsigned)rabove(d[i], tol) << i;
                    }
                    constexpr unsigned M0 = 0x27u, M1 = 0x33u, M2 = 0x39u;
                    if (q < npl) {
                        outside[0] |= (ge & M0) == M0; outside[1] |= (ge & M1) == M1; outside[2] |= (ge & M2) == M2;
                        if (gt & M0) mask[0] |= 1u << q;
                        if (gt & M1) mask[1] |= 1u << q;
                        if (gt & M2) mask[2] |= 1u << q;
                    }
                } else {
                    const R l01 = rmin(d[0], d[1]), h01 = rmax(d[0], d[1]);
                    const R lo0 = rmin(l01, rmin(d[2], d[5])), hi0 = rmax(h01, rmax(d[2], d[5]));
                    const R lo1 = rmin(l01, rmin(d[5], d[4])), hi1 = rmax(h01, rmax(d[5], d[4]));
                    const R lo2 = rmin(rmin(d[0], d[3]), rmin(d[4], d[5])), hi2 = rmax(rmax(d[0], d[3]), rmax(d[4], d[5]));
                    if (q < npl) {
                        outside[0] |= lo0 >= -tol; outside[1] |= lo1 >= -tol; outside[2] |= lo2 >= -tol;
                        if (hi0 > tol) mask[0] |= 1u << q;
                        if (hi1 > tol) mask[1] |= 1u << q;
                        if (hi2 > tol) mask[2] |= 1u << q;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int t = 3 * pr + j;
                const R sg = sh.Tsg[t];
                if (sg != R(0) && !outside[j]) {
                    if (mask[j] == 0) acc_add(acc, sg * sh.Kw[k] * sh.Tv6[t]);
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
    if (nq > 0) mx_clip(sh, nq, tol, acc, wk);
    __syncwarp();
}

// W warps (faces) per block; blocks per SM as shared memory allows (the FP64
// form's per-warp buffers are twice as large)
template <class R> constexpr int mx_resident(int w, int st)
{
    return st == MX_STACK_WIDE ? (w == 1 ? 15 : w == 2 ? 8 : 5) : (w == 1 ? 18 : w == 2 ? 9 : 6);
}
template <> constexpr int mx_resident<double>(int w, int) { return w == 1 ? 8 : 4; }

template <class R> __device__ __forceinline__ R rconv(double v) { return (R)v; }

template <class R, int MX_STACK, bool LIST, class Wk>
__device__ __forceinline__ void phase_flux_body(const DevMesh &m, const MXArgs &a, MXShared<R, MX_STACK> &sh)
{
    using V = R3<R>;
    const R4<R> *fpl = static_cast<const R4<R> *>(a.fpl), *cbl = static_cast<const R4<R> *>(a.cbl);
    const R4<R> *ktl = static_cast<const R4<R> *>(a.ktl);
    const int lane = threadIdx.x & 31;
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
            // (inflow through a boundary face brings nothing; a periodic face's
            // copy carries no flux)
            if (Ff == 0.0 || (f >= m.ni && (Ff < 0.0 || (m.fimg && m.fimg[f - m.ni] >= 0))) || all_e) triv = 0.0;
            else if (all_f) triv = Ff * a.dt;
            else done = false;
            if (done) {
                if (lane == 0) a.Va[f] = triv;
                continue;
            }
        }
        const V3 o = ld3(m.cf, m.nf, f);
        const int b = __ldg(m.fptr + f), n = __ldg(m.fptr + f + 1) - b;
        // Complement form: sum the void pieces and take V_alpha = F dt - void
        // (equal in exact arithmetic since the corrected polyhedron holds F dt
        // and the stencil covers it).  Full cells then need no clipping, where
        // the plain form clips them and skips empty ones; the form is chosen by
        // which of the two leaves fewer cells reaching the polyhedron's box
        // (stencils of one chunk; ties, and longer stencils, by whether the
        // upwind cell is mostly phase).  A polyhedron inside full cells carries
        // exactly F dt, one inside empty cells exactly 0, and the rounding of
        // the clipping stays with mixed cells.  Not where the polyhedron can
        // leave the domain (the normal-sweep fallback at walls; a face touching
        // an open boundary), since the part outside is empty and the stencil
        // does not cover it.
        const double Ff = a.F[f];
        const int up = Ff > 0.0 ? __ldg(m.own + f) : (f < m.ni ? __ldg(m.nei + f) : __ldg(m.own + f));
        const double lamf = LIST ? a.lam_b[item] : a.lambda[f];
        const bool comp_ok = lamf >= 0.0 && !__ldg(m.fopen + f);
        const bool decide = comp_ok && s1 - s0 <= 32;  // warp-uniform
        bool comp = comp_ok && ge_pos(a.alpha[up], 0.5);
        const int nt = n == 3 ? 3 : 3 * n;
        // signed distances (to unit-normal planes) within the on-plane band of
        // the face (FP32: 2e-6 of the face size, FP64: 1e-14) are taken as zero:
        // points shared by the polyhedron and the cell tetrahedra come out of
        // different roundings and would otherwise look like cuts
        const R tol = ldg4(fpl, b).w;
        // ---- flux polyhedron tetrahedra in the face frame
        R bx[6] = {R(3e38), R(3e38), R(3e38), R(-3e38), R(-3e38), R(-3e38)};
        if (lane < nt) {
            int pr = lane / 3, j = lane % 3;
            auto disp = [&](int i) -> V {  // i < 0: face centre
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
                return r3(rconv<R>(w.x), rconv<R>(w.y), rconv<R>(w.z));
            };
            V a0, a1, a2, w0, w1, w2;
            long k0, k1, k2;
            if (n == 3) {
                k0 = __ldg(m.fkey + b); k1 = __ldg(m.fkey + b + 1); k2 = __ldg(m.fkey + b + 2);
                a0 = ld43<R>(fpl, b); a1 = ld43<R>(fpl, b + 1); a2 = ld43<R>(fpl, b + 2);
                w0 = disp(0); w1 = disp(1); w2 = disp(2);
            } else {
                int u = pr + 1 == n ? 0 : pr + 1;
                k0 = -1; k1 = __ldg(m.fkey + b + pr); k2 = __ldg(m.fkey + b + u);
                a0 = r3(R(0), R(0), R(0)); a1 = ld43<R>(fpl, b + pr); a2 = ld43<R>(fpl, b + u);
                w0 = disp(-1); w1 = disp(pr); w2 = disp(u);
            }
            int par = 1;
            if (k1 < k0) { V t = a0; a0 = a1; a1 = t; t = w0; w0 = w1; w1 = t; long q = k0; k0 = k1; k1 = q; par = -par; }
            if (k2 < k1) { V t = a1; a1 = a2; a2 = t; t = w1; w1 = w2; w2 = t; long q = k1; k1 = k2; k2 = q; par = -par; }
            if (k1 < k0) { V t = a0; a0 = a1; a1 = t; t = w0; w0 = w1; w1 = t; long q = k0; k0 = k1; k1 = q; par = -par; }
            V b0 = a0 - w0, b1 = a1 - w1, b2 = a2 - w2;
            RTet<R> T;
            if (j == 0) T = RTet<R>{{a0, a1, a2, b2}};
            else if (j == 1) T = RTet<R>{{a0, a1, b2, b1}};
            else T = RTet<R>{{a0, b0, b1, b2}};
            R v6 = rvol6(T.v[0], T.v[1], T.v[2], T.v[3]);
            R sv = R(-par) * v6;
            stT(sh.T[lane], T);
            sh.Tsg[lane] = sv > R(0) ? R(1) : (sv < R(0) ? R(-1) : R(0));
            sh.Tv6[lane] = rabs(v6);
            bx[0] = rmin(rmin(T.v[0].x, T.v[1].x), rmin(T.v[2].x, T.v[3].x));
            bx[1] = rmin(rmin(T.v[0].y, T.v[1].y), rmin(T.v[2].y, T.v[3].y));
            bx[2] = rmin(rmin(T.v[0].z, T.v[1].z), rmin(T.v[2].z, T.v[3].z));
            bx[3] = rmax(rmax(T.v[0].x, T.v[1].x), rmax(T.v[2].x, T.v[3].x));
            bx[4] = rmax(rmax(T.v[0].y, T.v[1].y), rmax(T.v[2].y, T.v[3].y));
            bx[5] = rmax(rmax(T.v[0].z, T.v[1].z), rmax(T.v[2].z, T.v[3].z));
            if (j == 0) {
                R *q = reinterpret_cast<R *>(sh.P6[pr]);
                const V pv[6] = {a0, a1, a2, b0, b1, b2};
#pragma unroll
                for (int i = 0; i < 6; ++i) { q[3 * i] = pv[i].x; q[3 * i + 1] = pv[i].y; q[3 * i + 2] = pv[i].z; }
                R lo3[3] = {R(3e38), R(3e38), R(3e38)}, hi3[3] = {R(-3e38), R(-3e38), R(-3e38)};
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    lo3[0] = rmin(lo3[0], pv[i].x); lo3[1] = rmin(lo3[1], pv[i].y); lo3[2] = rmin(lo3[2], pv[i].z);
                    hi3[0] = rmax(hi3[0], pv[i].x); hi3[1] = rmax(hi3[1], pv[i].y); hi3[2] = rmax(hi3[2], pv[i].z);
                }
                for (int i = 0; i < 3; ++i) { sh.Pb[pr][i] = lo3[i]; sh.Pb[pr][3 + i] = hi3[i]; }
            }
        }
        // bounding box of the whole polyhedron
        R pb[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            R v = bx[i];
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) {
                R w = __shfl_xor_sync(0xffffffffu, v, o2);
                v = i < 3 ? rmin(v, w) : rmax(v, w);
            }
            pb[i] = v;
        }
        __syncwarp();
        Acc<R> acc;
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
                    V dc = r3(R(0), R(0), R(0));
                    // the face centre in the cell's frame: on a periodic mesh
                    // the cell sits next to the face moved by its stencil
                    // translation t, and the cell, its tetrahedra and its
                    // plane are taken relative to o - t
                    V3 oc = o;
                    bool emp = false, ful = false;
                    if (s < s1) {
                        c = __ldg(m.scell + s);
                        al = a.alpha[c];
                        if (m.scode) oc = o - tshift(m, __ldg(m.scode + s));
                        // an empty cell carries no phase, a full cell no void
                        // thresholds on the integer pipe (bit-pattern order of doubles)
                        emp = le_pos(al, eps);
                        ful = ge_pos(al, 1.0 - eps);
                        if (decide || !(comp ? ful : emp)) {
                            const V3 cc = ld3(m.cc, m.nc, c);
                            dc = r3(rconv<R>(cc.x - oc.x), rconv<R>(cc.y - oc.y), rconv<R>(cc.z - oc.z));
                            const R4<R> cb0 = ldg4(cbl, 2 * (long)c), cb1 = ldg4(cbl, 2 * (long)c + 1);
                            pass = !(rgt(pb[0], cb1.x + dc.x) || rgt(cb0.x + dc.x, pb[3]) || rgt(pb[1], cb1.y + dc.y) ||
                                     rgt(cb0.y + dc.y, pb[4]) || rgt(pb[2], cb1.z + dc.z) || rgt(cb0.z + dc.z, pb[5]));
                        }
                    }
                    if (decide) {  // the whole stencil is this chunk
                        const int nful = __popc(__ballot_sync(0xffffffffu, pass && ful));
                        const int nemp = __popc(__ballot_sync(0xffffffffu, pass && emp));
                        if (nful != nemp) comp = nful > nemp;
                    }
                    pass = pass && !(comp ? ful : emp);
                    int nkt = 0, t0 = 0;
                    R wgt = R(1);
                    bool useH = false;
                    R4<R> H = mk4<R>(R(0), R(0), R(0), R(0));
                    if (pass) {
                        t0 = __ldg(a.ctptr + c);
                        nkt = __ldg(a.ctptr + c + 1) - t0;
                        if (gt_pos(al, eps) && lt_pos(al, 1.0 - eps)) {
                            if (a.flags[c] & VOF_ORIENTED) {
                                V3 hn = ld3(a.n, m.nc, c);
                                double hd = a.d[c] - dot(hn, oc);
                                // phase side n.x <= d; the void side is -n.x <= -d
                                R sg = comp ? R(-1) : R(1);
                                H = mk4<R>(sg * rconv<R>(hn.x), sg * rconv<R>(hn.y), sg * rconv<R>(hn.z),
                                           sg * rconv<R>(hd));
                                useH = true;
                            } else wgt = comp ? rconv<R>(1.0 - al) : rconv<R>(al);
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
            R4<R> kp[4];
            R kbx[6];
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
                const V dc = r3(sh.Cdc[ci][0], sh.Cdc[ci][1], sh.Cdc[ci][2]);
                const R4<R> *q = ktl + 6 * (size_t)j;
                // box and planes in one round trip to L2 (the planes of the
                // tetrahedra the box test drops are read for nothing)
                const R4<R> b0 = ldg4(q, 4), b1 = ldg4(q, 5);
#pragma unroll
                for (int i = 0; i < 4; ++i) kp[i] = ldg4(q, i);
                kbx[0] = b0.x + dc.x; kbx[1] = b0.y + dc.y; kbx[2] = b0.z + dc.z;
                kbx[3] = b1.x + dc.x; kbx[4] = b1.y + dc.y; kbx[5] = b1.z + dc.z;
                cand = !(rgt(pb[0], kbx[3]) || rgt(kbx[0], pb[3]) || rgt(pb[1], kbx[4]) || rgt(kbx[1], pb[4]) ||
                         rgt(pb[2], kbx[5]) || rgt(kbx[2], pb[5]));
                if (cand) {
                    wk.add(WK_SHIFT, 4);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const R4<R> pl = kp[i];
                        kp[i] = mk4<R>(pl.x, pl.y, pl.z, pl.w + (pl.x * dc.x + pl.y * dc.y + pl.z * dc.z));
                    }
                }
            }
            const unsigned cmask = __ballot_sync(0xffffffffu, cand);
            if (fin ? ncand > 0 : ncand + __popc(cmask) > MX_CAND) {
                mx_flush(sh, nt, ncand, tol, acc, wk);
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
        // lane sums (and their compensations) merged across the warp, then the
        // 1/6 of the volumes in FP64
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            const R xs = __shfl_xor_sync(0xffffffffu, acc.s, o2), xc = __shfl_xor_sync(0xffffffffu, acc.c, o2);
            acc_add(acc, xs);
            acc.c += xc;
        }
        double va = ((double)acc.s + (double)acc.c) * (1.0 / 6.0);
        if (comp) va = Ff * a.dt - va;
        if (lane == 0) a.Va[f] = va;
        __syncwarp();
    }
    wk.flush(a.work, lane);
}

template <bool LIST, int W, int ST, class Wk>
__global__ void __launch_bounds__(W * 32, mx_resident<float>(W, ST)) k_phase_flux_mixed(DevMesh m, MXArgs a)
{
    __shared__ MXShared<float, ST> shm[W];
    phase_flux_body<float, ST, LIST, Wk>(m, a, shm[threadIdx.x >> 5]);
}

template <bool LIST, int W, class Wk>
__global__ void __launch_bounds__(W * 32, mx_resident<double>(W, MX_STACK_WIDE)) k_phase_flux(DevMesh m, MXArgs a)
{
    __shared__ MXShared<double, MX_STACK_WIDE> shm[W];
    phase_flux_body<double, MX_STACK_WIDE, LIST, Wk>(m, a, shm[threadIdx.x >> 5]);
}

// geometry of every cell relative to its centre (context creation): face
// centres and face points, and the cell's box widened by one rounding of R so
// that the boxes stay conservative
template <class R>
__global__ void k_local_geom(DevMesh m, const int *cfpptr, R4<R> *cfl, R4<R> *cfpl, R4<R> *cbl)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    V3 cc = ld3(m.cc, m.nc, c);
    int o = cfpptr[c];
    for (int k = m.cptr[c]; k < m.cptr[c + 1]; ++k) {
        int g = m.cface[k] >> 1;
        V3 q = ld3(m.cf, m.nf, g) - cc;
        cfl[k] = mk4<R>((R)q.x, (R)q.y, (R)q.z, R(0));
        for (int j = m.fptr[g]; j < m.fptr[g + 1]; ++j) {
            V3 p = ldP(m, m.fpts[j]) - cc;
            cfpl[o++] = mk4<R>((R)p.x, (R)p.y, (R)p.z, R(0));
        }
    }
    const double *b = m.cbox + 6 * (size_t)c;
    auto lo = [](double v) {
        R f = (R)v;
        return (double)f > v ? rnext(f, R(-3e38)) : f;
    };
    auto hi = [](double v) {
        R f = (R)v;
        return (double)f < v ? rnext(f, R(3e38)) : f;
    };
    cbl[2 * c] = mk4<R>(lo(b[0] - cc.x), lo(b[1] - cc.y), lo(b[2] - cc.z), R(0));
    cbl[2 * c + 1] = mk4<R>(hi(b[3] - cc.x), hi(b[4] - cc.y), hi(b[5] - cc.z), R(0));
}

__device__ __forceinline__ float rrsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rrsqrt(double x) { return rsqrt(x); }

// the tetrahedra of every cell (cell centre + fan triangle of a face, in the
// order of the cell's faces and of the face's points) as 4 outward unit-normal
// planes and a box, in the cell frame (context creation)
template <class R>
__global__ void k_cell_tets(DevMesh m, const int *cfpptr, const R4<R> *cfl, const R4<R> *cfpl, const int *ctptr,
                            R4<R> *ktl)
{
    using V = R3<R>;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    int o = cfpptr[c], j = ctptr[c];
    for (int k = m.cptr[c]; k < m.cptr[c + 1]; ++k) {
        const int code = m.cface[k], g = code >> 1, gn = m.fptr[g + 1] - m.fptr[g];
        for (int i = 0; i < (gn == 3 ? 1 : gn); ++i, ++j) {
            V k0 = r3(R(0), R(0), R(0)), k1, k2, k3;
            if (gn == 3) {
                k1 = ld43<R>(cfpl, o); k2 = ld43<R>(cfpl, o + 1); k3 = ld43<R>(cfpl, o + 2);
            } else {
                k1 = ld43<R>(cfl, k); k2 = ld43<R>(cfpl, o + i); k3 = ld43<R>(cfpl, o + (i + 1 == gn ? 0 : i + 1));
            }
            if (code & 1) { V t = k2; k2 = k3; k3 = t; }
            V n0 = rcross(k2 - k0, k1 - k0), n1 = rcross(k1 - k0, k3 - k0);
            V n2 = rcross(k3 - k0, k2 - k0), n3 = rcross(k2 - k1, k3 - k1);
            const R tiny = sizeof(R) == 4 ? R(1e-37) : R(1e-300);
            n0 = n0 * rrsqrt(rdot(n0, n0) + tiny); n1 = n1 * rrsqrt(rdot(n1, n1) + tiny);
            n2 = n2 * rrsqrt(rdot(n2, n2) + tiny); n3 = n3 * rrsqrt(rdot(n3, n3) + tiny);
            R4<R> *q = ktl + 6 * (size_t)j;
            q[0] = mk4<R>(n0.x, n0.y, n0.z, R(0));
            q[1] = mk4<R>(n1.x, n1.y, n1.z, R(0));
            q[2] = mk4<R>(n2.x, n2.y, n2.z, R(0));
            q[3] = mk4<R>(n3.x, n3.y, n3.z, rdot(n3, k1));
            q[4] = mk4<R>(rmin(rmin(k0.x, k1.x), rmin(k2.x, k3.x)), rmin(rmin(k0.y, k1.y), rmin(k2.y, k3.y)),
                          rmin(rmin(k0.z, k1.z), rmin(k2.z, k3.z)), R(0));
            q[5] = mk4<R>(rmax(rmax(k0.x, k1.x), rmax(k2.x, k3.x)), rmax(rmax(k0.y, k1.y), rmax(k2.y, k3.y)),
                          rmax(rmax(k0.z, k1.z), rmax(k2.z, k3.z)), R(0));
        }
        o += gn;
    }
}

// face points relative to the face centre; the w of the face's first point
// holds the on-plane band of the clipping: 2e-6 of the face size in FP32
// (reading R13), 1e-14 of it in FP64
template <class R>
__global__ void k_face_local(DevMesh m, R4<R> *fpl)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.nf) return;
    V3 c = ld3(m.cf, m.nf, f), S = ld3(m.sf, m.nf, f);
    const double band = sizeof(R) == 4 ? 2e-6 : 1e-14;
    const R tol = (R)(band * sqrt(sqrt(dot(S, S))));
    for (int j = m.fptr[f]; j < m.fptr[f + 1]; ++j) {
        V3 p = ldP(m, m.fpts[j]) - c;
        fpl[j] = mk4<R>((R)p.x, (R)p.y, (R)p.z, j == m.fptr[f] ? tol : R(0));
    }
}

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

template <class R>
int setup_tables(vof_ctx *c, cudaStream_t s)
{
    R4<R> *cfl = static_cast<R4<R> *>(c->cfl), *cfpl = static_cast<R4<R> *>(c->cfpl);
    k_local_geom<R><<<cdiv(c->nc, 256), 256, 0, s>>>(c->m, c->cfpptr, cfl, cfpl, static_cast<R4<R> *>(c->cbl));
    k_face_local<R><<<cdiv(c->nf, 256), 256, 0, s>>>(c->m, static_cast<R4<R> *>(c->fpl));
    k_cell_tets<R><<<cdiv(c->nc, 256), 256, 0, s>>>(c->m, c->cfpptr, cfl, cfpl, c->m.ctptr,
                                                    static_cast<R4<R> *>(c->ktl));
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

}  // namespace

size_t phase_flux_table_entry_bytes(int precision)
{
    return precision == VOF_MIXED ? sizeof(float4) : sizeof(D4);
}

int launch_setup_mixed(vof_ctx *c, cudaStream_t s)
{
    return c->precision == VOF_MIXED ? setup_tables<float>(c, s) : setup_tables<double>(c, s);
}

static MXArgs mx_args(vof_ctx *c, const double *alpha, const double *n, const double *d, const uint8_t *flags,
                      const double *Up, const double *F, const double *lambda, double dt, double *Va,
                      const int *list, const int *count, const double *disp, unsigned long long *work)
{
    return MXArgs{alpha, n, d, flags, Up, F, lambda, dt, Va, list, count, disp, c->lam_b, c->status, work,
                  c->fpl, c->cbl, c->ktl, c->m.ctptr, nullptr};
}

int launch_pf_all(vof_ctx *c, const double *alpha, const double *n, const double *d,
                                const uint8_t *flags, const double *Up, const double *F, const double *lambda,
                                double dt, double *Va, cudaStream_t s)
{
    MXArgs a = mx_args(c, alpha, n, d, flags, Up, F, lambda, dt, Va, nullptr, nullptr, nullptr,
                       c->work_on ? c->work : nullptr);
    if (c->precision == VOF_MIXED) {
        if (c->work_on) k_phase_flux_mixed<false, 2, MX_STACK_WIDE, WkOn><<<cdiv((long)c->nf * 32, 64), 64, 0, s>>>(c->m, a);
        else k_phase_flux_mixed<false, 2, MX_STACK_WIDE, WkOff><<<cdiv((long)c->nf * 32, 64), 64, 0, s>>>(c->m, a);
    } else {
        if (c->work_on) k_phase_flux<false, 1, WkOn><<<cdiv((long)c->nf * 32, 32), 32, 0, s>>>(c->m, a);
        else k_phase_flux<false, 1, WkOff><<<cdiv((long)c->nf * 32, 32), 32, 0, s>>>(c->m, a);
    }
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

int launch_pf_list(vof_ctx *c, const double *alpha, const double *F, double dt, int sms,
                                 cudaStream_t s)
{
    MXArgs a = mx_args(c, alpha, c->n, c->d, c->flags, nullptr, F, nullptr, dt, c->Va, c->band,
                       c->counters + CNT_BAND, c->disp_b, c->work_on ? c->work : nullptr);
    a.next = c->counters + CNT_PFNEXT;  // zeroed with the step's counters
    if (c->precision != VOF_MIXED) {
        // the FP64 form: one warp per block, as many blocks as shared memory allows
        if (c->work_on) k_phase_flux<true, 1, WkOn><<<sms * mx_resident<double>(1, MX_STACK_WIDE), 32, 0, s>>>(c->m, a);
        else k_phase_flux<true, 1, WkOff><<<sms * mx_resident<double>(1, MX_STACK_WIDE), 32, 0, s>>>(c->m, a);
        return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
    }
    // launch configuration (vof_batch_tune): warps per block, stack depth, and
    // grid = SMs x resident blocks x multiplier
    const int w = c->pf_warps >= 1 && c->pf_warps <= 3 ? c->pf_warps : 2;
    const int mult = c->pf_mult >= 1 ? c->pf_mult : 1;
    const bool slim = c->pf_stack == 1;
#define PF_GO(W_, ST_, WK_)                                                                                  \
    k_phase_flux_mixed<true, W_, ST_, WK_><<<sms * mx_resident<float>(W_, ST_) * mult, 32 * W_, 0, s>>>(c->m, a)
    if (c->work_on) {  // instrumented variant (vof_count_work), two warps per block
        if (slim) PF_GO(2, MX_STACK_SLIM, WkOn);
        else PF_GO(2, MX_STACK_WIDE, WkOn);
    } else if (slim) {
        if (w == 1) PF_GO(1, MX_STACK_SLIM, WkOff);
        else if (w == 2) PF_GO(2, MX_STACK_SLIM, WkOff);
        else PF_GO(3, MX_STACK_SLIM, WkOff);
    } else {
        if (w == 1) PF_GO(1, MX_STACK_WIDE, WkOff);
        else if (w == 2) PF_GO(2, MX_STACK_WIDE, WkOff);
        else PF_GO(3, MX_STACK_WIDE, WkOff);
    }
#undef PF_GO
    return cudaGetLastError() == cudaSuccess ? VOF_OK : VOF_ERR_CUDA;
}

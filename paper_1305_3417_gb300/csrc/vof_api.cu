// C-ABI entry points of libvof and the host-side topology builder.
//
// vof_create derives the integer topology on the host (cell->face,
// cell->point, point->cell, face stencils, wall-point lists), copies it to the
// device, and computes every geometric quantity in kernels.  Per-step entry
// points only validate arguments and enqueue kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "vof_internal.h"

int launch_wall_table(vof_ctx *c, const int *wptr, const int *wface, int nrows, cudaStream_t s);

namespace {

template <class F>
void parallel_for(long n, F fn)
{
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < 4096) nt = 1;
    std::vector<std::thread> th;
    long chunk = (n + nt - 1) / nt;
    for (unsigned t = 0; t < nt; ++t) {
        long a = t * chunk, b = std::min(n, a + chunk);
        if (a >= b) break;
        th.emplace_back([=, &fn] { for (long i = a; i < b; ++i) fn(i); });
    }
    for (auto &x : th) x.join();
}

template <class T>
T *dev_alloc(vof_ctx *c, size_t n, int *err)
{
    if (*err) return nullptr;
    if (c->nbufs >= (int)(sizeof(c->bufs) / sizeof(c->bufs[0]))) { *err = VOF_ERR_CUDA; return nullptr; }
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) { *err = VOF_ERR_CUDA; return nullptr; }
    c->bufs[c->nbufs++] = p;
    return (T *)p;
}

template <class T>
T *dev_copy(vof_ctx *c, const T *h, size_t n, int *err)
{
    T *d = dev_alloc<T>(c, n, err);
    if (*err) return nullptr;
    if (n && cudaMemcpy(d, h, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) *err = VOF_ERR_CUDA;
    return d;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

// regions of the global bounding step, cut into segments of at most 4096
// cells; replaces any earlier regions (buffers of earlier calls stay owned by
// the context until vof_destroy)
int set_bound_regions(vof_ctx *c, const int *reg_cell, int nreg)
{
    constexpr int SEG = 4096;
    std::vector<int4> seg;
    std::vector<int> rs(1, 0);
    for (int r = 0; r < nreg; ++r) {
        for (int a = reg_cell[r]; a < reg_cell[r + 1]; a += SEG)
            seg.push_back(make_int4(r, a, std::min(a + SEG, reg_cell[r + 1]), 0));
        rs.push_back((int)seg.size());
    }
    if (seg.empty()) seg.push_back(make_int4(0, 0, 0, 0));
    int err = 0;
    c->seg = dev_copy(c, seg.data(), seg.size(), &err);
    c->reg_seg = dev_copy(c, rs.data(), rs.size(), &err);
    c->gpartial = dev_alloc<double>(c, 4 * seg.size(), &err);
    c->reg_tot = dev_alloc<double>(c, 6 * (size_t)nreg, &err);  // per region: Ep, Em, Sp, Sm, Ep/Sp, Em/Sm
    if (err) return err;
    c->nseg = (int)seg.size();
    c->nreg = nreg;
    return VOF_OK;
}

extern "C" {

// the reason of the last VOF_ERR_BAD_MESH of vof_create on this thread
static thread_local const char *g_bad_mesh = "";
static int bad_mesh(const char *why)
{
    g_bad_mesh = why;
    return VOF_ERR_BAD_MESH;
}

const char *vof_create_error(void) { return g_bad_mesh; }

const char *vof_error_string(int code)
{
    switch (code) {
    case VOF_OK: return "ok";
    case VOF_ERR_INVALID_ARG: return "invalid argument";
    case VOF_ERR_CUDA: return "CUDA runtime error";
    case VOF_ERR_BAD_MESH: return "bad mesh (index out of range or non-positive cell volume)";
    case VOF_ERR_NOT_CONVERGED: return "iteration did not converge";
    case VOF_ERR_STENCIL: return "flux stencil does not cover the flux polyhedron";
    case VOF_ERR_TIMEOUT: return "device wait timed out";
    case VOF_ERR_NO_DEVICE: return "no compute capability 10.3 CUDA device";
    default: return "unknown error";
    }
}

static void free_profile(vof_ctx *c)
{
    if (!c->prof_ev) return;
    for (int i = 0; i < c->prof_max * (VOF_PROF_GROUPS + 1); ++i) cudaEventDestroy(c->prof_ev[i]);
    delete[] c->prof_ev;
    c->prof_ev = nullptr;
    c->prof_max = c->prof_steps = 0;
}

void vof_destroy(vof_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    free_profile(c);
    for (int i = 0; i < c->nbufs; ++i) cudaFree(c->bufs[i]);
    cudaFree(c->mlp_s0);
    cudaFree(c->mlp_feat);
    cudaFree(c->mlp_nbr);
    cudaFree(c->mlp_geo);
    if (c->s_copy) cudaStreamDestroy(c->s_copy);
    if (c->ev_f) cudaEventDestroy(c->ev_f);
    if (c->ev_u) cudaEventDestroy(c->ev_u);
    if (c->ev_ain) cudaEventDestroy(c->ev_ain);
    for (int i = 0; i < 2; ++i)
        if (c->ev_free[i]) cudaEventDestroy(c->ev_free[i]);
    if (c->s_aux) cudaStreamDestroy(c->s_aux);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
}

int vof_create(const vof_mesh *mesh, const vof_options *opt, vof_ctx **out)
{
    g_bad_mesh = "";
    if (!mesh || !out) return VOF_ERR_INVALID_ARG;
    *out = nullptr;
    const int np = mesh->n_points, nf = mesh->n_faces, ni = mesh->n_internal, nc = mesh->n_cells;
    if (np <= 0 || nf <= 0 || nc <= 0 || ni < 0 || ni > nf) return VOF_ERR_INVALID_ARG;
    if (!mesh->px || !mesh->py || !mesh->pz || !mesh->face_ptr || !mesh->face_pts || !mesh->owner ||
        (ni > 0 && !mesh->neighbour))
        return VOF_ERR_INVALID_ARG;
    int device = opt ? opt->device : 0;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return VOF_ERR_NO_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return VOF_ERR_NO_DEVICE;
    if (!(prop.major == 10 && prop.minor == 3)) return VOF_ERR_NO_DEVICE;
    if (cudaSetDevice(device) != cudaSuccess) return VOF_ERR_NO_DEVICE;

    // ---------------------------------------------------------- validation
    const int *fptr = mesh->face_ptr, *fpts = mesh->face_pts, *own = mesh->owner, *nei = mesh->neighbour;
    if (fptr[0] != 0) return bad_mesh("face_ptr[0] is not 0");
    for (int f = 0; f < nf; ++f) {
        int n = fptr[f + 1] - fptr[f];
        if (n < 3 || n > VOF_MAXFP) return bad_mesh("a face has fewer than 3 or more than 8 points");
        if (own[f] < 0 || own[f] >= nc) return bad_mesh("an owner index is out of range");
        if (f < ni && (nei[f] < 0 || nei[f] >= nc || nei[f] == own[f])) return bad_mesh("a neighbour index is out of range or equals the owner");
    }
    const long nfp = fptr[nf];
    for (long k = 0; k < nfp; ++k)
        if (fpts[k] < 0 || fpts[k] >= np) return bad_mesh("a face point index is out of range");
    // periodic data: each copy is owned by its face's neighbour and lists the
    // same points (by master) one translation away
    const bool periodic = mesh->point_master != nullptr;
    const int *pmas = mesh->point_master, *fimg = mesh->face_image;
    const int8_t *pimg = mesh->point_image;
    if (periodic && (!pimg || !mesh->period || !fimg)) return VOF_ERR_INVALID_ARG;
    std::vector<uint8_t> imaged(std::max(ni, 1), 0);
    if (periodic) {
        for (int p = 0; p < np; ++p) {
            if (pmas[p] < 0 || pmas[p] >= np || pmas[pmas[p]] != pmas[p]) return bad_mesh("a point master is out of range or not its own master");
            for (int e = 0; e < 3; ++e)
                if (pimg[3 * p + e] < -1 || pimg[3 * p + e] > 1) return bad_mesh("a point image is not in {-1, 0, 1}");
        }
        for (int b = ni; b < nf; ++b) {
            const int a = fimg[b - ni];
            if (a < 0) continue;
            if (a >= ni || imaged[a] || nei[a] != own[b] || fptr[a + 1] - fptr[a] != fptr[b + 1] - fptr[b])
                return bad_mesh("a periodic copy is not owned by its face's neighbour, copies an internal face twice, or differs in point count");
            int d0[3] = {0, 0, 0};
            for (int j = fptr[a]; j < fptr[a + 1]; ++j) {
                int pb = -1;
                for (int k = fptr[b]; k < fptr[b + 1]; ++k)
                    if (pmas[fpts[k]] == pmas[fpts[j]]) pb = fpts[k];
                if (pb < 0) return bad_mesh("a periodic copy lacks an image of one of its face's points");
                for (int e = 0; e < 3; ++e) {
                    const int d = pimg[3 * fpts[j] + e] - pimg[3 * pb + e];
                    if (j == fptr[a]) d0[e] = d;
                    else if (d != d0[e]) return bad_mesh("a periodic copy is not one translation away from its face");
                }
            }
            imaged[a] = 1;
        }
    }

    // ------------------------------------------------------ host topology
    // cell -> faces: a cell's own faces (a periodic face belongs to its owner;
    // its neighbour has the copy)
    std::vector<int> cptr(nc + 1, 0), cface;
    for (int f = 0; f < nf; ++f) {
        cptr[own[f] + 1]++;
        if (f < ni && !imaged[f]) cptr[nei[f] + 1]++;
    }
    for (int c = 0; c < nc; ++c) cptr[c + 1] += cptr[c];
    cface.resize(cptr[nc]);
    {
        std::vector<int> fill(nc, 0);
        for (int f = 0; f < nf; ++f) {
            cface[cptr[own[f]] + fill[own[f]]++] = 2 * f;
            if (f < ni && !imaged[f]) cface[cptr[nei[f]] + fill[nei[f]]++] = 2 * f + 1;
        }
    }
    std::vector<int> cnb(cface.size()), cflux;
    for (size_t k = 0; k < cface.size(); ++k) {
        const int f = cface[k] >> 1;
        if (f >= ni) cnb[k] = (periodic && fimg[f - ni] >= 0) ? own[fimg[f - ni]] : -1;
        else cnb[k] = (cface[k] & 1) ? own[f] : nei[f];
    }
    if (periodic) {  // the update reads a copy's entry as its periodic face, seen from the neighbour
        cflux = cface;
        for (size_t k = 0; k < cface.size(); ++k) {
            const int f = cface[k] >> 1;
            if (f >= ni && fimg[f - ni] >= 0) cflux[k] = 2 * fimg[f - ni] + 1;
        }
    }
    // cell -> distinct points, and the tetrahedron count per cell
    std::vector<int> cpcount(nc);
    std::vector<int> ktet(nc);
    parallel_for(nc, [&](long c) {
        int k = 0, kt = 0;
        for (int i = cptr[c]; i < cptr[c + 1]; ++i) {
            int f = cface[i] >> 1, n = fptr[f + 1] - fptr[f];
            k += n;
            kt += n == 3 ? 1 : n;
        }
        cpcount[c] = k;
        ktet[c] = kt;
    });
    for (int c = 0; c < nc; ++c)
        if (ktet[c] > 32 * VOF_MAXK_LANE || ktet[c] < 4) return bad_mesh("a cell has fewer than 4 or more than 96 tetrahedra");
    std::vector<int> cpptr(nc + 1, 0);
    {
        std::vector<int> uniq(nc);
        std::vector<long> off(nc + 1, 0);
        for (int c = 0; c < nc; ++c) off[c + 1] = off[c] + cpcount[c];
        std::vector<int> tmp(off[nc]);
        parallel_for(nc, [&](long c) {
            long o = off[c];
            int k = 0;
            for (int i = cptr[c]; i < cptr[c + 1]; ++i) {
                int f = cface[i] >> 1;
                for (int j = fptr[f]; j < fptr[f + 1]; ++j) tmp[o + k++] = fpts[j];
            }
            std::sort(tmp.begin() + o, tmp.begin() + o + k);
            uniq[c] = (int)(std::unique(tmp.begin() + o, tmp.begin() + o + k) - (tmp.begin() + o));
        });
        for (int c = 0; c < nc; ++c) cpptr[c + 1] = cpptr[c] + uniq[c];
        std::vector<int> cpts(cpptr[nc]);
        parallel_for(nc, [&](long c) {
            std::copy(tmp.begin() + off[c], tmp.begin() + off[c] + uniq[c], cpts.begin() + cpptr[c]);
        });
        tmp.clear();
        tmp.shrink_to_fit();
        cpcount.swap(cpts);  // reuse: cpcount now holds the flattened cell points
    }
    const std::vector<int> &cpts = cpcount;
    // point -> cells (ascending cell index)
    std::vector<int> pptr(np + 1, 0), pcell(cpptr[nc]);
    for (int c = 0; c < nc; ++c)
        for (int i = cpptr[c]; i < cpptr[c + 1]; ++i) pptr[cpts[i] + 1]++;
    for (int p = 0; p < np; ++p) pptr[p + 1] += pptr[p];
    {
        std::vector<int> fill(np, 0);
        for (int c = 0; c < nc; ++c)
            for (int i = cpptr[c]; i < cpptr[c + 1]; ++i) {
                int p = cpts[i];
                pcell[pptr[p] + fill[p]++] = c;
            }
    }
    for (int p = 0; p < np; ++p)
        if (pptr[p + 1] == pptr[p]) return bad_mesh("a point is used by no cell");  // point used by no cell
    // periodic: the cells around every image of a point, moved next to it
    // (code k(p) - k(q), q the image the cell lists), sorted by (cell, code)
    std::vector<uint8_t> pcode;
    if (periodic) {
        std::vector<int> mptr(np + 1, 0), mem(np);
        for (int p = 0; p < np; ++p) mptr[pmas[p] + 1]++;
        for (int p = 0; p < np; ++p) mptr[p + 1] += mptr[p];
        {
            std::vector<int> fill(np, 0);
            for (int p = 0; p < np; ++p) mem[mptr[pmas[p]] + fill[pmas[p]]++] = p;
        }
        std::vector<int> pptr2(np + 1, 0);
        for (int p = 0; p < np; ++p) {
            long k = 0;
            for (int j = mptr[pmas[p]]; j < mptr[pmas[p] + 1]; ++j) k += pptr[mem[j] + 1] - pptr[mem[j]];
            if (pptr2[p] + k > 0x7fffffffL) return bad_mesh("too many (point, cell) entries");
            pptr2[p + 1] = pptr2[p] + (int)k;
        }
        std::vector<long long> key(pptr2[np]);
        std::atomic<int> bad{0};
        parallel_for(np, [&](long p) {
            long o = pptr2[p];
            for (int j = mptr[pmas[p]]; j < mptr[pmas[p] + 1]; ++j) {
                const int q = mem[j];
                int code = 0;
                for (int e = 2; e >= 0; --e) {
                    const int d = pimg[3 * p + e] - pimg[3 * q + e];
                    if (d < -1 || d > 1) bad = 1;
                    code = 3 * code + (d + 1);
                }
                for (int i = pptr[q]; i < pptr[q + 1]; ++i) key[o++] = (long long)pcell[i] * 32 + code;
            }
            std::sort(key.begin() + pptr2[p], key.begin() + pptr2[p + 1]);
            for (long i = pptr2[p] + 1; i < pptr2[p + 1]; ++i)
                if (key[i] / 32 == key[i - 1] / 32) bad = 1;  // a cell at two images of one point
        });
        if (bad) return bad_mesh("periodic images more than one period apart, or a cell touching two images of one point");
        pcell.resize(key.size());
        pcode.resize(key.size());
        for (size_t i = 0; i < key.size(); ++i) {
            pcell[i] = (int)(key[i] / 32);
            pcode[i] = (uint8_t)(key[i] % 32);
        }
        pptr.swap(pptr2);
    }
    // face stencils: every cell sharing a point with the face, ascending
    std::vector<int> scount(nf);
    std::vector<long> soff(nf + 1, 0);
    for (int f = 0; f < nf; ++f) {
        long k = 0;
        for (int j = fptr[f]; j < fptr[f + 1]; ++j) k += pptr[fpts[j] + 1] - pptr[fpts[j]];
        soff[f + 1] = soff[f] + k;
    }
    std::vector<int> stmp(soff[nf]);
    std::vector<uint8_t> sctmp(periodic ? soff[nf] : 0);
    parallel_for(nf, [&](long f) {
        long o = soff[f];
        int k = 0;
        if (!periodic) {
            for (int j = fptr[f]; j < fptr[f + 1]; ++j)
                for (int q = pptr[fpts[j]]; q < pptr[fpts[j] + 1]; ++q) stmp[o + k++] = pcell[q];
            std::sort(stmp.begin() + o, stmp.begin() + o + k);
            scount[f] = (int)(std::unique(stmp.begin() + o, stmp.begin() + o + k) - (stmp.begin() + o));
        } else {  // (cell, code) pairs: a cell may sit next to the face at two translations
            std::vector<long long> kk;
            for (int j = fptr[f]; j < fptr[f + 1]; ++j)
                for (int q = pptr[fpts[j]]; q < pptr[fpts[j] + 1]; ++q) kk.push_back((long long)pcell[q] * 32 + pcode[q]);
            std::sort(kk.begin(), kk.end());
            kk.erase(std::unique(kk.begin(), kk.end()), kk.end());
            for (long long v : kk) {
                stmp[o + k] = (int)(v / 32);
                sctmp[o + k] = (uint8_t)(v % 32);
                ++k;
            }
            scount[f] = k;
        }
    });
    // 64-bit offsets: a large batch of tetrahedral cases holds billions of entries
    std::vector<long long> sptr(nf + 1, 0);
    for (int f = 0; f < nf; ++f) sptr[f + 1] = sptr[f] + scount[f];
    std::vector<int> scell(sptr[nf]);
    std::vector<uint8_t> scode(periodic ? sptr[nf] : 0);
    parallel_for(nf, [&](long f) {
        std::copy(stmp.begin() + soff[f], stmp.begin() + soff[f] + scount[f], scell.begin() + sptr[f]);
        if (periodic)
            std::copy(sctmp.begin() + soff[f], sctmp.begin() + soff[f] + scount[f], scode.begin() + sptr[f]);
    });
    stmp.clear();
    stmp.shrink_to_fit();
    sctmp.clear();
    sctmp.shrink_to_fit();
    // wall points and the wall faces through them (reading R2)
    std::vector<int> pwall(np, -1), wptr(1, 0), wface;
    {
        std::vector<std::vector<int>> lists;
        for (int f = ni; f < nf; ++f) {
            bool w = mesh->wall ? mesh->wall[f - ni] != 0 : true;
            if (!w || (periodic && fimg[f - ni] >= 0)) continue;  // a copy is no wall
            for (int j = fptr[f]; j < fptr[f + 1]; ++j) {
                int p = fpts[j];
                if (pwall[p] < 0) { pwall[p] = (int)lists.size(); lists.emplace_back(); }
                lists[pwall[p]].push_back(f);
            }
        }
        for (auto &l : lists) {
            wface.insert(wface.end(), l.begin(), l.end());
            wptr.push_back((int)wface.size());
        }
    }
    const int nwrows = (int)wptr.size() - 1;
    // faces with a point on an open boundary face: their flux polyhedra can
    // reach outside the domain, where the stencil does not cover them
    std::vector<uint8_t> popen(np, 0), fopen(nf, 0);
    for (int f = ni; f < nf; ++f)
        if (mesh->wall && mesh->wall[f - ni] == 0 && !(periodic && fimg[f - ni] >= 0))
            for (int j = fptr[f]; j < fptr[f + 1]; ++j) popen[fpts[j]] = 1;
    parallel_for(nf, [&](long f) {
        for (int j = fptr[f]; j < fptr[f + 1]; ++j)
            if (popen[fpts[j]]) { fopen[f] = 1; break; }
    });
    // per cell: offset of its (face, point) entries in face order
    std::vector<int> cfpptr(nc + 1, 0);
    for (int c = 0; c < nc; ++c) {
        long v = cfpptr[c];
        for (int i = cptr[c]; i < cptr[c + 1]; ++i) {
            int f = cface[i] >> 1;
            v += fptr[f + 1] - fptr[f];
        }
        if (v > 0x7fffffffL) return bad_mesh("too many (face, point) entries");
        cfpptr[c + 1] = (int)v;
    }
    std::vector<int> ctptr(nc + 1, 0);
    for (int c = 0; c < nc; ++c) ctptr[c + 1] = ctptr[c] + ktet[c];
    // (face, point) entries and tetrahedra of every cell, in face order
    std::vector<int2> cent(cfpptr[nc]);
    std::vector<int4> ctet(ctptr[nc]);
    parallel_for(nc, [&](long c) {
        int e = cfpptr[c], t = ctptr[c];
        for (int i = cptr[c]; i < cptr[c + 1]; ++i) {
            const int code = cface[i], f = code >> 1, b = fptr[f], n = fptr[f + 1] - b;
            for (int j = 0; j < n; ++j) cent[e++] = make_int2(b + j, code);
            if (n == 3) ctet[t++] = make_int4(code, b, b + 1, b + 2);
            else
                for (int j = 0; j < n; ++j) ctet[t++] = make_int4(code, b + j, b + (j + 1 == n ? 0 : j + 1), -1);
        }
    });

    // ------------------------------------------------------------- device
    vof_ctx *c = new vof_ctx();
    std::memset(c->bufs, 0, sizeof(c->bufs));
    c->nbufs = 0;
    c->device = device;
    c->np = np; c->nf = nf; c->ni = ni; c->nc = nc;
    c->eps = (opt && opt->eps > 0.0) ? opt->eps : 1e-9;
    c->precision = opt ? opt->precision : VOF_FP64;
    {
        const int kmax = *std::max_element(ktet.begin(), ktet.end());
        // lanes per cell in the reconstruction: narrow groups (several cells
        // a warp) for the mixed form's few, short FP32 iterations; in the FP64
        // form the groups of a warp would run their long Alg. 1 iterations
        // one after another, so hexahedra keep a warp each there
        if (c->precision == VOF_MIXED) {
            c->rc_g = kmax <= 4 ? 4 : kmax <= 24 ? 8 : 32;
            c->rc_k = kmax <= 4 ? 1 : kmax <= 16 ? 2 : kmax <= 24 ? 3 : kmax <= 64 ? 2 : 3;
        } else {
            c->rc_g = kmax <= 16 ? 8 : 32;
            c->rc_k = kmax <= 64 ? 2 : 3;
        }
    }
    c->bound = opt ? (opt->bound != 0) : 1;
    int err = 0;
    DevMesh &m = c->m;
    m.np = np; m.nf = nf; m.ni = ni; m.nc = nc; m.eps = c->eps;
    m.px = dev_copy(c, mesh->px, np, &err);
    m.py = dev_copy(c, mesh->py, np, &err);
    m.pz = dev_copy(c, mesh->pz, np, &err);
    m.fptr = dev_copy(c, fptr, nf + 1, &err);
    m.fpts = dev_copy(c, fpts, nfp, &err);
    m.own = dev_copy(c, own, nf, &err);
    m.nei = dev_copy(c, ni > 0 ? nei : own, std::max(ni, 1), &err);
    m.cptr = dev_copy(c, cptr.data(), cptr.size(), &err);
    m.cface = dev_copy(c, cface.data(), cface.size(), &err);
    m.cnb = dev_copy(c, cnb.data(), cnb.size(), &err);
    m.cpptr = dev_copy(c, cpptr.data(), cpptr.size(), &err);
    m.cpts = dev_copy(c, cpts.data(), cpts.size(), &err);
    m.pptr = dev_copy(c, pptr.data(), pptr.size(), &err);
    m.pcell = dev_copy(c, pcell.data(), pcell.size(), &err);
    m.pw = dev_alloc<double>(c, pcell.size(), &err);
    m.sptr = dev_copy(c, sptr.data(), sptr.size(), &err);
    m.scell = dev_copy(c, scell.data(), scell.size(), &err);
    m.pwall = dev_copy(c, pwall.data(), pwall.size(), &err);
    m.fopen = dev_copy(c, fopen.data(), fopen.size(), &err);
    m.wallt = dev_alloc<double>(c, 7 * (size_t)std::max(nwrows, 1), &err);
    int *d_wptr = dev_copy(c, wptr.data(), wptr.size(), &err);
    int *d_wface = dev_copy(c, wface.empty() ? wptr.data() : wface.data(), std::max<size_t>(wface.size(), 1), &err);
    m.cf = dev_alloc<double>(c, 3 * (size_t)nf, &err);
    m.sf = dev_alloc<double>(c, 3 * (size_t)nf, &err);
    m.cc = dev_alloc<double>(c, 3 * (size_t)nc, &err);
    m.vc = dev_alloc<double>(c, nc, &err);
    m.cbox = dev_alloc<double>(c, 6 * (size_t)nc, &err);
    m.nagc = dev_alloc<double>(c, nfp, &err);
    m.ceptr = dev_copy(c, cfpptr.data(), cfpptr.size(), &err);
    m.cent = dev_copy(c, cent.data(), cent.size(), &err);
    m.ctptr = dev_copy(c, ctptr.data(), ctptr.size(), &err);
    m.ctet = dev_copy(c, ctet.data(), ctet.size(), &err);
    m.pcode = nullptr; m.scode = nullptr; m.fimg = nullptr;
    m.fkey = m.fpts;
    m.cflux = m.cface;
    for (int i = 0; i < 9; ++i) m.L[i] = periodic ? mesh->period[i] : 0.0;
    if (periodic) {
        std::vector<int> fkey(nfp);
        for (long k = 0; k < nfp; ++k) fkey[k] = pmas[fpts[k]];
        m.pcode = dev_copy(c, pcode.data(), pcode.size(), &err);
        m.scode = dev_copy(c, scode.data(), scode.size(), &err);
        m.fkey = dev_copy(c, fkey.data(), fkey.size(), &err);
        m.cflux = dev_copy(c, cflux.data(), cflux.size(), &err);
        std::vector<int> fi(fimg, fimg + (nf - ni));
        fi.push_back(-1);  // (never empty)
        m.fimg = dev_copy(c, fi.data(), fi.size(), &err);
    }
    // per-step scratch
    c->pstate = dev_alloc<uint8_t>(c, np, &err);
    c->band = dev_alloc<int>(c, nf, &err);
    c->icell = dev_alloc<int>(c, nc, &err);
    c->viol[0] = dev_alloc<int>(c, nc, &err);
    c->pend_c = dev_alloc<int>(c, 8 * (size_t)nc, &err);
    c->pend_a = dev_alloc<double>(c, 8 * (size_t)nc, &err);
    c->counters = dev_alloc<int>(c, CNT_ALLOC, &err);
    c->lam_b = dev_alloc<double>(c, nf, &err);
    c->disp_b = dev_alloc<double>(c, (size_t)nf * (VOF_MAXFP + 1) * 3, &err);
    c->it_b = dev_alloc<int>(c, nf, &err);
    c->n = dev_alloc<double>(c, 3 * (size_t)nc, &err);
    c->d = dev_alloc<double>(c, nc, &err);
    c->flags = dev_alloc<uint8_t>(c, nc, &err);
    c->pit = dev_alloc<int>(c, nc, &err);
    c->Va = dev_alloc<double>(c, nf, &err);
    c->bscr = dev_alloc<double>(c, 3 * (size_t)nc, &err);
    c->partial = dev_alloc<double>(c, 10 * 1024, &err);
    c->stats_dev = dev_alloc<double>(c, VOF_S_LEN, &err);
    c->status = dev_alloc<unsigned>(c, 1, &err);
    c->h_alpha = dev_alloc<double>(c, nc, &err);
    for (int i = 0; i < 2; ++i) {
        c->h_Uc[i] = dev_alloc<double>(c, 3 * (size_t)nc, &err);
        c->h_F[i] = dev_alloc<double>(c, nf, &err);
    }
    c->work = dev_alloc<unsigned long long>(c, WK_LEN, &err);
    c->cfpptr = dev_copy(c, cfpptr.data(), cfpptr.size(), &err);
    // the phase-flux kernels' tables, 4-vectors of the context's form
    const size_t e4 = phase_flux_table_entry_bytes(c->precision);
    c->cfl = dev_alloc<unsigned char>(c, e4 * cface.size(), &err);
    c->cfpl = dev_alloc<unsigned char>(c, e4 * cfpptr[nc], &err);
    c->fpl = dev_alloc<unsigned char>(c, e4 * nfp, &err);
    c->cbl = dev_alloc<unsigned char>(c, e4 * 2 * (size_t)nc, &err);
    c->palpha = dev_alloc<double>(c, np, &err);
    c->bpflag = dev_alloc<uint8_t>(c, np, &err);
    c->upb = dev_alloc<double>(c, 3 * (size_t)np, &err);
    c->ktl = dev_alloc<unsigned char>(c, e4 * 6 * (size_t)ctptr[nc], &err);
    if (err) { vof_destroy(c); return err; }
    cudaMemset(c->work, 0, WK_LEN * sizeof(unsigned long long));
    cudaMemset(c->bscr, 0, sizeof(double) * 3 * nc);
    cudaMemset(c->counters, 0, sizeof(int) * CNT_ALLOC);
    cudaMemset(c->status, 0, sizeof(unsigned));
    cudaMemset(c->n, 0, sizeof(double) * 3 * nc);
    cudaMemset(c->d, 0, sizeof(double) * nc);
    cudaMemset(c->flags, 0, nc);
    cudaMemset(c->bpflag, 0, np);
    if (!err && (cudaStreamCreateWithFlags(&c->s_aux, cudaStreamNonBlocking) != cudaSuccess ||
                 cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                 cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess))
        err = VOF_ERR_CUDA;
    {
        const int whole[2] = {0, nc};
        if (!err) err = set_bound_regions(c, whole, 1);
        if (err) { vof_destroy(c); return err; }
    }
    int r = launch_setup_geometry(c, 0);
    if (!r) r = launch_wall_table(c, d_wptr, d_wface, nwrows, 0);
    if (!r) r = launch_setup_mixed(c, 0);
    if (r) { vof_destroy(c); return r; }
    unsigned bad = 0;
    if (cudaMemcpy(&bad, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        vof_destroy(c);
        return VOF_ERR_CUDA;
    }
    if (bad) { vof_destroy(c); return bad_mesh("a cell tetrahedron of non-positive volume"); }
    *out = c;
    return VOF_OK;
}

int vof_geometry(vof_ctx *c, double *cc, double *vc, double *cf, double *sf, void *stream)
{
    if (!c) return VOF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    if (cc && cudaMemcpyAsync(cc, c->m.cc, 3 * sizeof(double) * c->nc, cudaMemcpyDeviceToDevice, s)) return VOF_ERR_CUDA;
    if (vc && cudaMemcpyAsync(vc, c->m.vc, sizeof(double) * c->nc, cudaMemcpyDeviceToDevice, s)) return VOF_ERR_CUDA;
    if (cf && cudaMemcpyAsync(cf, c->m.cf, 3 * sizeof(double) * c->nf, cudaMemcpyDeviceToDevice, s)) return VOF_ERR_CUDA;
    if (sf && cudaMemcpyAsync(sf, c->m.sf, 3 * sizeof(double) * c->nf, cudaMemcpyDeviceToDevice, s)) return VOF_ERR_CUDA;
    return VOF_OK;
}

int vof_point_velocity(vof_ctx *c, const double *Uc, double *Up, void *stream)
{
    if (!c || !Uc || !Up) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_point_velocity(c, Uc, Up, (cudaStream_t)stream);
}

int vof_reconstruct(vof_ctx *c, const double *alpha, double *n, double *d, uint8_t *flags, int32_t *iters,
                    void *stream)
{
    if (!c || !alpha || !n || !d || !flags) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_reconstruct(c, alpha, n, d, flags, iters, nullptr, nullptr, (cudaStream_t)stream);
}

// the LSQ stencil: every other cell sharing a point with each cell (host, from
// the device copies of cell->point and point->cell), and the gradient buffer
static int build_lsq(vof_ctx *c)
{
    if (c->lptr) return VOF_OK;
    const int nc = c->nc, np = c->np;
    const bool periodic = c->m.pcode != nullptr;
    std::vector<int> cpptr(nc + 1), pptr(np + 1);
    if (cudaMemcpy(cpptr.data(), c->m.cpptr, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(pptr.data(), c->m.pptr, sizeof(int) * (np + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
        return VOF_ERR_CUDA;
    std::vector<int> cpts(cpptr[nc]), pcell(pptr[np]);
    std::vector<uint8_t> pcode(periodic ? pptr[np] : 0);
    if (cudaMemcpy(cpts.data(), c->m.cpts, sizeof(int) * cpts.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(pcell.data(), c->m.pcell, sizeof(int) * pcell.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (periodic && cudaMemcpy(pcode.data(), c->m.pcode, pcode.size(), cudaMemcpyDeviceToHost) != cudaSuccess))
        return VOF_ERR_CUDA;
    std::vector<long> off(nc + 1, 0);
    for (int x = 0; x < nc; ++x) {
        long k = 0;
        for (int i = cpptr[x]; i < cpptr[x + 1]; ++i) k += pptr[cpts[i] + 1] - pptr[cpts[i]];
        off[x + 1] = off[x] + k;
    }
    // (cell, translation code) keys; without periods every code is 13, so the
    // keys sort as the cells do; the cell itself unmoved is not its neighbour
    std::vector<long long> tmp(off[nc]);
    std::vector<int> cnt(nc);
    parallel_for(nc, [&](long x) {
        long o = off[x];
        int k = 0;
        for (int i = cpptr[x]; i < cpptr[x + 1]; ++i)
            for (int q = pptr[cpts[i]]; q < pptr[cpts[i] + 1]; ++q) {
                const int code = periodic ? pcode[q] : 13;
                if (pcell[q] != x || code != 13) tmp[o + k++] = (long long)pcell[q] * 32 + code;
            }
        std::sort(tmp.begin() + o, tmp.begin() + o + k);
        cnt[x] = (int)(std::unique(tmp.begin() + o, tmp.begin() + o + k) - (tmp.begin() + o));
    });
    std::vector<int> lptr(nc + 1, 0);
    for (int x = 0; x < nc; ++x) {
        if ((long)lptr[x] + cnt[x] > 0x7fffffffL) return VOF_ERR_INVALID_ARG;
        lptr[x + 1] = lptr[x] + cnt[x];
    }
    std::vector<int> lcell(lptr[nc]);
    std::vector<uint8_t> lcode(periodic ? lptr[nc] : 0);
    parallel_for(nc, [&](long x) {
        for (int i = 0; i < cnt[x]; ++i) {
            lcell[lptr[x] + i] = (int)(tmp[off[x] + i] / 32);
            if (periodic) lcode[lptr[x] + i] = (uint8_t)(tmp[off[x] + i] % 32);
        }
    });
    int err = 0;
    int *dp = dev_copy(c, lptr.data(), lptr.size(), &err);
    int *dc = dev_copy(c, lcell.data(), lcell.size(), &err);
    uint8_t *dk = periodic ? dev_copy(c, lcode.data(), lcode.size(), &err) : nullptr;
    double *g = dev_alloc<double>(c, 3 * (size_t)nc, &err);
    if (err) return err;
    c->lptr = dp;
    c->lcell = dc;
    c->lcode = dk;
    c->grad = g;
    return VOF_OK;
}

int vof_set_gradient(vof_ctx *c, int kind)
{
    if (!c || (kind != VOF_GRAD_NAG && kind != VOF_GRAD_LSQ)) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (kind == VOF_GRAD_LSQ) {
        int r = build_lsq(c);
        if (r) return r;
    }
    c->grad_kind = kind;
    return VOF_OK;
}

int vof_lsq_gradient(vof_ctx *c, const double *alpha, double *grad, void *stream)
{
    if (!c || !alpha || !grad) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    int r = build_lsq(c);
    if (r) return r;
    return launch_lsq_gradient(c, alpha, nullptr, nullptr, grad, (cudaStream_t)stream);
}

int vof_evsd(vof_ctx *c, const uint8_t *flags, const double *n, const double *d, const double ball[4], int levels,
             double *evsd, void *stream)
{
    if (!c || !ball || !evsd || (flags && (!n || !d))) return VOF_ERR_INVALID_ARG;
    if (!(ball[3] > 0.0) || !std::isfinite(ball[0]) || !std::isfinite(ball[1]) || !std::isfinite(ball[2]))
        return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_evsd(c, flags, n, d, ball, levels, evsd, (cudaStream_t)stream);
}

int vof_remap(vof_ctx *dst, const vof_ctx *src, const double *alpha_src, const double *n_src, const double *d_src,
              const uint8_t *flags_src, const int32_t *pair_ptr, const int32_t *pair_src, double *alpha_dst,
              void *stream)
{
    if (!dst || !src || !alpha_src || !n_src || !d_src || !flags_src || !pair_ptr || !pair_src || !alpha_dst)
        return VOF_ERR_INVALID_ARG;
    if (dst->device != src->device) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(dst->device);
    return launch_remap(dst, src, alpha_src, n_src, d_src, flags_src, pair_ptr, pair_src, alpha_dst,
                        (cudaStream_t)stream);
}

int vof_flux_polyhedra(vof_ctx *c, const double *Up, const double *F, const double *lambda, double dt,
                       double *V, void *stream)
{
    if (!c || !Up || !V || !finite_pos(dt)) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_flux_polyhedra(c, Up, F, lambda, dt, V, (cudaStream_t)stream);
}

int vof_correct_flux(vof_ctx *c, const double *Up, const double *F, double dt, double *lambda, int32_t *iters,
                     void *stream)
{
    if (!c || !Up || !F || !lambda || !finite_pos(dt)) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_correct_all(c, Up, F, dt, lambda, iters, (cudaStream_t)stream);
}

int vof_phase_flux(vof_ctx *c, const double *alpha, const double *n, const double *d, const uint8_t *flags,
                   const double *Up, const double *F, const double *lambda, double dt, double *Va, void *stream)
{
    if (!c || !alpha || !n || !d || !flags || !Up || !F || !lambda || !Va || !finite_pos(dt))
        return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_phase_flux_all(c, alpha, n, d, flags, Up, F, lambda, dt, Va, (cudaStream_t)stream);
}

int vof_update(vof_ctx *c, double *alpha, const double *Va, double *stats, void *stream)
{
    if (!c || !alpha || !Va) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_update(c, alpha, Va, stats, (cudaStream_t)stream);
}

int vof_courant(vof_ctx *c, const double *F, double dt, double *co, void *stream)
{
    if (!c || !F || !co || !finite_pos(dt)) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_courant(c, F, dt, co, (cudaStream_t)stream);
}

int vof_advect(vof_ctx *c, double *alpha, const double *Uc, const double *F, double dt, double *stats,
               void *stream)
{
    if (!c || !alpha || !Uc || !F || !finite_pos(dt)) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_advect(c, alpha, Uc, F, dt, stats, (cudaStream_t)stream);
}

int vof_advect_host(vof_ctx *c, double *alpha, const double *Uc, const double *F, double dt, double *stats,
                    void *stream)
{
    if (!c || !alpha || !Uc || !F || !finite_pos(dt)) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    // Uc in host memory the device can address (pinned: the driver gives a
    // device pointer for it) is read in place by the step: only the band
    // kernels read it, at the cells around band points, so the link carries
    // a small part of it.  F, which the classification reads in full, and
    // pageable Uc go to the staging pair of this call's parity on the copy
    // stream, once the step that last read that pair (two calls back) is done
    // and the previous call's alpha is in: they overlap the previous step's
    // kernels.  alpha (in place, so ordered after the previous step's
    // read-back) goes on `stream`; the classification waits for F, the flux
    // correction (inside the step) for a copied Uc.
    const double *dU = nullptr;
    {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, Uc) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
            dU = static_cast<const double *>(pa.devicePointer);
        cudaGetLastError();  // (an unknown pointer leaves an error behind)
    }
    if (!c->s_copy && (cudaStreamCreateWithFlags(&c->s_copy, cudaStreamNonBlocking) ||
                       cudaEventCreateWithFlags(&c->ev_f, cudaEventDisableTiming) ||
                       cudaEventCreateWithFlags(&c->ev_u, cudaEventDisableTiming) ||
                       cudaEventCreateWithFlags(&c->ev_free[0], cudaEventDisableTiming) ||
                       cudaEventCreateWithFlags(&c->ev_free[1], cudaEventDisableTiming) ||
                       cudaEventCreateWithFlags(&c->ev_ain, cudaEventDisableTiming)))
        return VOF_ERR_CUDA;
    const int p = c->h_par;
    // ev_ain: the previous call's alpha copy, which must not queue in the copy
    // engine behind this call's larger copies (it is on the step's critical path)
    if (cudaStreamWaitEvent(c->s_copy, c->ev_free[p], 0) || cudaStreamWaitEvent(c->s_copy, c->ev_ain, 0) ||
        cudaMemcpyAsync(c->h_F[p], F, sizeof(double) * c->nf, cudaMemcpyHostToDevice, c->s_copy) ||
        cudaEventRecord(c->ev_f, c->s_copy) ||
        (!dU && (cudaMemcpyAsync(c->h_Uc[p], Uc, 3 * sizeof(double) * c->nc, cudaMemcpyHostToDevice, c->s_copy) ||
                 cudaEventRecord(c->ev_u, c->s_copy))) ||
        cudaMemcpyAsync(c->h_alpha, alpha, sizeof(double) * c->nc, cudaMemcpyHostToDevice, s) ||
        cudaEventRecord(c->ev_ain, s) || cudaStreamWaitEvent(s, c->ev_f, 0))
        return VOF_ERR_CUDA;
    c->h_par ^= 1;
    int r = dU ? launch_advect(c, c->h_alpha, dU, c->h_F[p], dt, c->stats_dev, s)
               : launch_advect(c, c->h_alpha, c->h_Uc[p], c->h_F[p], dt, c->stats_dev, s, c->ev_u);
    if (r) return r;
    if (cudaEventRecord(c->ev_free[p], s)) return VOF_ERR_CUDA;
    if (cudaMemcpyAsync(alpha, c->h_alpha, sizeof(double) * c->nc, cudaMemcpyDeviceToHost, s)) return VOF_ERR_CUDA;
    if (stats && cudaMemcpyAsync(stats, c->stats_dev, sizeof(double) * VOF_S_LEN, cudaMemcpyDeviceToHost, s))
        return VOF_ERR_CUDA;
    return VOF_OK;
}

int vof_status(vof_ctx *c, uint32_t *bits, void *stream)
{
    if (!c || !bits) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned v = 0;
    if (cudaMemcpyAsync(&v, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VOF_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VOF_ERR_CUDA;
    if (cudaMemsetAsync(c->status, 0, sizeof(unsigned), s) != cudaSuccess) return VOF_ERR_CUDA;
    *bits = v;
    return VOF_OK;
}

int vof_last_launch_count(vof_ctx *c) { return c ? c->launches : 0; }

int vof_profile_begin(vof_ctx *c, int max_steps)
{
    if (!c || max_steps <= 0) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    free_profile(c);
    int n = max_steps * (VOF_PROF_GROUPS + 1);
    c->prof_ev = new cudaEvent_t[n];
    for (int i = 0; i < n; ++i)
        if (cudaEventCreate(&c->prof_ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(c->prof_ev[j]);
            delete[] c->prof_ev;
            c->prof_ev = nullptr;
            return VOF_ERR_CUDA;
        }
    c->prof_max = max_steps;
    c->prof_steps = 0;
    return VOF_OK;
}

int vof_profile_end(vof_ctx *c, double *group_ms, int *steps)
{
    if (!c || !group_ms) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    for (int g = 0; g < VOF_PROF_GROUPS; ++g) group_ms[g] = 0.0;
    int ns = c->prof_ev ? c->prof_steps : 0;
    if (ns > 0 && cudaEventSynchronize(c->prof_ev[(size_t)(ns - 1) * (VOF_PROF_GROUPS + 1) + VOF_PROF_GROUPS]) != cudaSuccess)
        return VOF_ERR_CUDA;
    for (int k = 0; k < ns; ++k)
        for (int g = 0; g < VOF_PROF_GROUPS; ++g) {
            float ms = 0.f;
            cudaEvent_t *e = c->prof_ev + (size_t)k * (VOF_PROF_GROUPS + 1);
            if (cudaEventElapsedTime(&ms, e[g], e[g + 1]) != cudaSuccess) return VOF_ERR_CUDA;
            group_ms[g] += ms;
        }
    if (steps) *steps = ns;
    free_profile(c);
    return VOF_OK;
}

int vof_probe_barrier(vof_ctx *c, int skip_block, void *stream)
{
    if (!c || skip_block < -1) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launch_barrier_probe(c, skip_block, (cudaStream_t)stream);
}

int vof_count_work(vof_ctx *c, int on)
{
    if (!c) return VOF_ERR_INVALID_ARG;
    c->work_on = on ? 1 : 0;
    return VOF_OK;
}

int vof_work_counts(vof_ctx *c, unsigned long long counts[VOF_WORK_LEN], int reset, void *stream)
{
    static_assert(VOF_WORK_LEN == WK_LEN, "work counter layout");
    if (!c || !counts) return VOF_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long v[WK_LEN] = {};
    if (cudaMemcpyAsync(v, c->work, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VOF_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VOF_ERR_CUDA;
    if (reset && cudaMemsetAsync(c->work, 0, sizeof(v), s) != cudaSuccess) return VOF_ERR_CUDA;
    for (int i = 0; i < WK_LEN; ++i) counts[i] = v[i];
    return VOF_OK;
}

}  // extern "C"

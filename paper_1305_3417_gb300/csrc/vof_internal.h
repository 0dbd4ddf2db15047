// Internal declarations of libvof: the context, the device-side mesh view
// passed by value to kernels, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vof.h"

#define VOF_MAXFP 8       // points per face handled by the per-face kernels
#define VOF_MAXK_LANE 3   // cell tetrahedra per lane in the reconstruction warp at most (96 per cell)

// Device view of the mesh, its derived topology and its geometry.  All
// pointers are device pointers owned by the context.
struct DevMesh {
    int np, nf, ni, nc;
    double eps;
    const double *px, *py, *pz;
    const int *fptr, *fpts, *own, *nei;
    const int *cptr, *cface;     // cell -> face codes, code = 2*f + (cell is neighbour)
    const int *cnb;              // per cface entry: the cell across that face, -1 on a boundary face
    const int *cpptr, *cpts;     // cell -> distinct points (ascending)
    const int *pptr, *pcell;     // point -> cells (ascending)
    const double *pw;            // inverse-distance weight per (point, cell) entry
    const long long *sptr;       // face stencil: cells sharing a point with the face
    const int *scell;
    const int *pwall;            // per point: wall-table row or -1
    const uint8_t *fopen;        // per face: 1 if a point lies on an open boundary face
    const double *wallt;         // wall table rows: count, n1 (3), n2 (3)
    const double *cf, *sf;       // face centre, area vector [3*nf]
    const double *cc, *vc, *cbox;  // cell centre [3*nc], volume [nc], box [6*nc]
    const double *nagc;          // NAG face-value weight per face-point entry
    // per cell, in face order then point order: the (face, point) entries
    // {fpts slot, face code} and the tetrahedra (c_c, outward face triangle)
    // {face code, slot a, slot b, slot c or -1 for the face centre}
    const int *ceptr;
    const int2 *cent;
    const int *ctptr;
    const int4 *ctet;
    // Periodic meshes (null otherwise, with fkey == fpts and cflux == cface):
    // translation code per (point, cell) entry and per stencil entry, (i+1) +
    // 3(j+1) + 9(k+1) for i L0 + j L1 + k L2 (13: none); the period vectors; the
    // sweep key of each face-point slot (its point's master); the flux code of
    // each cell-face entry (a copy's entry is its periodic face's, as
    // neighbour); the periodic face each boundary face copies (-1: none)
    const uint8_t *pcode, *scode;
    double L[9];
    const int *fkey;
    const int *cflux;
    const int *fimg;
};

// the context's counter buffer: per-step counters (the first CNT_LEN ints),
// then the two words of the grid barrier, each on its own 128-byte line
enum { CNT_BAND = 0, CNT_ICELL, CNT_MAXPOS, CNT_MAXCORR, CNT_FALLBACK, CNT_VIOL0, CNT_VIOL1, CNT_PEND, CNT_PFNEXT,
       CNT_RCNEXT, CNT_BPASS, CNT_BACT0, CNT_BACT1, CNT_LEN = 16 };
enum { CNT_BAR = 32, CNT_BARGEN = 64, CNT_ALLOC = 96 };
// algorithmic work counted by the step kernels (vof_work_counts): the phase
// flux's primitives (FP32 in the mixed form, FP64 in the plain one) -- signed
// distances of a prism's six points to a plane, of a piece's four points to a
// plane, edge intersections, tetrahedron volumes, closed-form cut fractions,
// plane shifts to the face frame -- and band faces; the reconstruction's fill
// evaluations per cell tetrahedron (FP64, FP32); the correction's cubic
// coefficient triangles and cubic evaluations (FP64)
enum { WK_PRISM = 0, WK_TEST, WK_EDGE, WK_VOL, WK_FRAC, WK_SHIFT, WK_N, WK_FACES = WK_N, WK_FILL64, WK_FILL32,
       WK_CTRI, WK_CEVAL, WK_LEN = 12 };

struct vof_ctx {
    int device;
    int np, nf, ni, nc;
    double eps;
    int precision, bound;
    DevMesh m;
    // owned device buffers (freed in vof_destroy)
    void *bufs[128];
    int nbufs;
    // per-step scratch
    uint8_t *pstate;
    int *band, *icell, *viol[2], *pend_c;
    double *pend_a;
    int *counters;               // CNT_ALLOC ints, laid out as CNT_* above
    double *lam_b, *disp_b;      // per band slot
    int *it_b;
    double *n, *d;
    uint8_t *flags;
    int *pit;
    double *Va;
    double *bscr;                // redistribution scratch, 3 doubles per cell
    double *gpartial;            // global bounding partial sums, 4 per segment
    // regions of the global bounding step (whole mesh, or the cases of a
    // batch): segments {region, first cell, end cell, -} and, per region, its
    // segment range and totals
    int nseg, nreg;
    int4 *seg;
    int *reg_seg;
    double *reg_tot;
    double *partial;             // reduction partials
    double *stats_dev;           // internal stats buffer
    unsigned *status;
    double *h_alpha;               // device staging for vof_advect_host; U and F double-buffered
    double *h_Uc[2], *h_F[2];      // by call parity, so that a call's copies overlap the previous step
    int h_par;
    cudaStream_t s_copy;           // vof_advect_host: the velocity copy overlaps the first kernels
    cudaEvent_t ev_f, ev_u, ev_free[2], ev_ain;
    cudaStream_t s_aux;            // the correction runs here, beside the reconstruction
    cudaEvent_t ev_fork, ev_join;
    int launches;
    unsigned long long *work;    // WK_LEN work counters
    int work_on;                 // 1: the step kernels count their work (instrumented variants)
    // geometry of the phase-flux kernels, 4-vectors of the context's form (float4
    // in a mixed context, four doubles in an FP64 one): face centres and face
    // points relative to each cell centre (cfl, cfpl), face points relative to
    // the face centre (fpl), cell boxes relative to the cell centre (cbl)
    void *cfl, *cfpl, *fpl, *cbl;
    int *cfpptr;
    // per cell tetrahedron: 4 outward unit-normal planes and the box, 6
    // 4-vectors, relative to the cell centre (first of each cell: m.ctptr)
    void *ktl;
    double *palpha;              // IDW point values of the points that are not all-empty / all-full
    uint8_t *bpflag;             // per point: a point of a band face this step (cleared by its reader)
    double *upb;                 // point velocities of the flagged points
    // mixed phase-flux launch configuration (0: defaults): warps per block 1-3,
    // grid multiplier over the resident blocks
    int pf_warps, pf_mult;
    int pf_stack;                // clip-piece stack per warp: 0 = 92 pieces, 1 = 56 (more resident warps)
    int rc_g;                    // reconstruction lanes per cell (4, 8 or 32; by form and cell size)
    int rc_k;                    // tetrahedra per lane (1, 2 or 3)
    // gradient of the reconstruction (vof_set_gradient): VOF_GRAD_NAG or
    // VOF_GRAD_LSQ; the LSQ stencil (cells sharing a point with each cell, CSR)
    // and the gradient buffer are made at the first selection of LSQ
    int grad_kind;
    int *lptr, *lcell;
    uint8_t *lcode;  // periodic meshes: translation code of each LSQ neighbour (else null)
    double *grad;
    // learned guess of the positioning (vof_set_guess): the network, offsets by
    // interface-list position, features
    struct vof_mlp *mlp;
    float *mlp_s0, *mlp_feat;
    int mlp_feat_cap;
    int *mlp_nbr;                // per cell: 27 lattice-slot cell indices (-1: itself)
    float *mlp_geo;              // per cell: 6 shape numbers
    // kernel-group timing (vof_profile_begin / _end)
    cudaEvent_t *prof_ev;
    int prof_max, prof_steps;
};

// ---- launchers (vof_kernels.cu) ----
int launch_lsq_gradient(vof_ctx *c, const double *alpha, const int *list, const int *count, double *grad,
                        cudaStream_t s);
int launch_evsd(vof_ctx *c, const uint8_t *flags, const double *n, const double *d, const double ball[4],
                int levels, double *out, cudaStream_t s);
int launch_remap(vof_ctx *dst, const vof_ctx *src, const double *alpha_src, const double *n_src,
                 const double *d_src, const uint8_t *flags_src, const int *pair_ptr, const int *pair_src,
                 double *alpha_dst, cudaStream_t s);
int launch_setup_geometry(vof_ctx *c, cudaStream_t s);
int launch_point_velocity(vof_ctx *c, const double *Uc, double *Up, cudaStream_t s);
int launch_reconstruct(vof_ctx *c, const double *alpha, double *n, double *d, uint8_t *flags,
                       int *iters, const int *list, const int *count, cudaStream_t s);
int launch_flux_polyhedra(vof_ctx *c, const double *Up, const double *F, const double *lambda,
                          double dt, double *V, cudaStream_t s);
int launch_correct_all(vof_ctx *c, const double *Up, const double *F, double dt, double *lambda,
                       int *iters, cudaStream_t s);
int launch_phase_flux_all(vof_ctx *c, const double *alpha, const double *n, const double *d,
                          const uint8_t *flags, const double *Up, const double *F,
                          const double *lambda, double dt, double *Va, cudaStream_t s);
int launch_update(vof_ctx *c, double *alpha, const double *Va, double *stats, cudaStream_t s);
int launch_courant(vof_ctx *c, const double *F, double dt, double *co, cudaStream_t s);
int launch_advect(vof_ctx *c, double *alpha, const double *Uc, const double *F, double dt,
                  double *stats, cudaStream_t s,
                  cudaEvent_t wait_before_correct = nullptr);
int launch_validate(vof_ctx *c, cudaStream_t s, unsigned *bad);
// ---- phase-flux tables (vof_phase_flux.cu) ----
int launch_setup_mixed(vof_ctx *c, cudaStream_t s);
// regions of the global bounding step: region r = cells [reg_cell[r], reg_cell[r+1]) (host array)
int set_bound_regions(vof_ctx *c, const int *reg_cell, int nreg);
// learned guess (vof_mlp.cu): offsets of the first min(nmax, batch) listed cells
// (count on the device, or all nmax when count is NULL) into c->mlp_s0
// the grid barrier's check: a cooperative launch in which block `skip` (if >= 0)
// leaves at once, so that the other blocks' waits run out (VOF_ST_TIMEOUT)
int launch_barrier_probe(vof_ctx *c, int skip, cudaStream_t s);
int launch_mlp_guess(vof_ctx *c, const double *alpha, const int *cells, const int *count, int nmax,
                     cudaStream_t s);
int mlp_cap(const vof_ctx *c);
// phase flux (vof_phase_flux.cu): every face (the standalone call) or the band
// list of a step, in the context's form (mixed FP32 or plain FP64)
int launch_pf_all(vof_ctx *c, const double *alpha, const double *n, const double *d, const uint8_t *flags,
                  const double *Up, const double *F, const double *lambda, double dt, double *Va, cudaStream_t s);
int launch_pf_list(vof_ctx *c, const double *alpha, const double *F, double dt, int sms, cudaStream_t s);
size_t phase_flux_table_entry_bytes(int precision);

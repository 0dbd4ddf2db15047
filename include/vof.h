/*
 * vof.h -- C ABI of libvof, the GB300 (sm_103a) implementation of the unsplit
 * geometric Volume-of-Fluid advection step of Maric, Marschall & Bothe (2013):
 * PLIC reconstruction, flux polyhedra, flux correction, phase fluxes and the
 * conservative volume-fraction update.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Return value: VOF_OK (0) or a negative VOF_ERR_* code; vof_error_string()
 *   names it.  Argument errors are detected on the host before anything is
 *   enqueued.  Conditions found on the device (an iteration cap reached, a
 *   clip buffer exhausted, a bounding residual) set bits of a per-context
 *   status word and never trap; vof_status() reads and clears it.
 * - Per-step arrays are DEVICE pointers owned by the caller (for example
 *   PyTorch tensors).  They must stay valid until `stream` reaches the call.
 *   Every per-step call is asynchronous on `stream` (a cudaStream_t; NULL is
 *   the legacy default stream) and allocates no memory: the context allocates
 *   all of its scratch in vof_create.
 * - Vectors are structure-of-arrays: x block, then y block, then z block.
 * - Face f of the mesh has points face_pts[face_ptr[f] .. face_ptr[f+1]),
 *   ordered so that the right-hand area vector S_f points from owner[f] to
 *   neighbour[f] (internal faces 0 .. n_internal-1) or out of the domain
 *   (boundary faces n_internal .. n_faces-1).  This is the owner/neighbour
 *   addressing of Sec. 2 (Eq. own-nei).  A volumetric flux F_f is positive
 *   from owner to neighbour; phase volumes V_alpha are signed the same way.
 * - Cell solids (reading of Sec. 2.1 for non-planar faces): a face with more
 *   than three points is the fan of triangles (c_f, p_i, p_i+1) about the mean
 *   of its points c_f; a cell is the union of the tetrahedra (c_c, outward face
 *   triangle), c_c the mean of the cell's points.
 */
#ifndef VOF_H
#define VOF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    VOF_OK = 0,
    VOF_ERR_INVALID_ARG = -1, /* NULL or inconsistent argument */
    VOF_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    VOF_ERR_BAD_MESH = -3,    /* index out of range, cell of non-positive volume, ... */
    VOF_ERR_NOT_CONVERGED = -4,
    VOF_ERR_STENCIL = -5,
    VOF_ERR_TIMEOUT = -6,
    VOF_ERR_NO_DEVICE = -7,   /* no CUDA device, or not a compute capability 10.3 part */
};

/* status bits accumulated on the device (vof_status) */
enum {
    VOF_ST_POS_NOT_CONVERGED = 1u << 0,  /* plane positioning hit its iteration cap */
    VOF_ST_CORR_NOT_CONVERGED = 1u << 1, /* flux correction hit its iteration cap */
    VOF_ST_CLIP_OVERFLOW = 1u << 2,      /* clipping stack exhausted (volume dropped) */
    VOF_ST_BOUND_RESIDUAL = 1u << 3,     /* |alpha - clamp(alpha)| > 1e-12 after bounding */
    VOF_ST_INDEX = 1u << 4,              /* an index check failed inside a kernel */
    VOF_ST_CAPACITY = 1u << 5,           /* a per-step list exceeded its capacity */
    VOF_ST_TIMEOUT = 1u << 6,            /* a grid barrier inside a kernel gave up waiting */
};

/* precision of the geometric kernels */
enum { VOF_FP64 = 0, VOF_MIXED = 1 };

/* cell flags written by vof_reconstruct */
enum { VOF_INTERFACE = 1, VOF_ORIENTED = 2, VOF_FULL = 4 };

/* Mesh description.  All pointers are HOST pointers, read during vof_create
 * only (the context keeps device copies). */
typedef struct {
    int32_t n_points, n_faces, n_internal, n_cells;
    const double *px, *py, *pz;  /* [n_points] point coordinates */
    const int32_t *face_ptr;     /* [n_faces + 1] CSR offsets into face_pts */
    const int32_t *face_pts;     /* [face_ptr[n_faces]] ordered point indices */
    const int32_t *owner;        /* [n_faces] */
    const int32_t *neighbour;    /* [n_internal] */
    const uint8_t *wall;         /* [n_faces - n_internal]: 1 = wall (no normal
                                    flow), 0 = open; NULL makes all walls */
    /* Periodic meshes (the paper's translation case runs on a periodic box,
     * Sec. 4.2); all NULL for other meshes.
     *   period       [9]: period vectors L0, L1, L2 as rows (unused rows zero);
     *   point_master [n_points]: the master point each point is an image of
     *                (itself for a master); the images of one master are one
     *                point of the periodic domain;
     *   point_image  [3*n_points], each in {-1, 0, 1}: P = P_master + sum_i k_i L_i;
     *   face_image   [n_faces - n_internal]: for the boundary face that is a
     *                periodic internal face's copy on its neighbour's side, that
     *                internal face; -1 for other boundary faces.
     * A periodic internal face is listed with its points on its owner's side;
     * its neighbour is built from the copy (same points, one translation
     * away), which carries no flux: the internal face's phase flux leaves the
     * owner and enters the neighbour.  The cells around a point are those
     * around all its images, each moved next to it; face stencils and
     * inverse-distance weights use the moved cells.  Flux polyhedra order
     * their points by master index. */
    const double *period;
    const int32_t *point_master;
    const int8_t *point_image;
    const int32_t *face_image;
} vof_mesh;

typedef struct {
    double eps;     /* interface tolerance: eps < alpha < 1-eps is an interface
                       cell (reading of Sec. 5.2's reconstruction tolerance);
                       <= 0 selects 1e-9 */
    int precision;  /* VOF_FP64 or VOF_MIXED */
    int bound;      /* 1: conservative bounding pass after the update */
    int device;     /* CUDA device ordinal */
} vof_options;

/* stats[] layout (doubles, device memory) written by vof_update / vof_advect */
enum {
    VOF_S_MASS_BEFORE = 0, VOF_S_MASS_AFTER, VOF_S_MIN_PRE, VOF_S_MAX_PRE, VOF_S_MIN_POST,
    VOF_S_MAX_POST, VOF_S_N_INTERFACE, VOF_S_N_BAND, VOF_S_MAX_POS_IT, VOF_S_MAX_CORR_IT,
    VOF_S_BOUNDARY_OUT, VOF_S_N_FALLBACK, VOF_S_N_BOUND_SOURCES,
    VOF_S_N_BOUND_LEFT,   /* sources left after the local redistribution passes */
    VOF_S_BOUND_PASSES,   /* local redistribution passes that moved something */
    VOF_S_BOUND_GLOBAL,   /* volume the global fallback moved after them */
    VOF_S_LEN = 16
};

typedef struct vof_ctx vof_ctx;

/* Builds the derived topology (cell->face, cell->point, point->cell, face
 * stencils: every cell sharing a point with the face, Sec. 2.3) on the host,
 * copies it to the device, computes the geometry (face centres and area
 * vectors, cell centres, volumes and bounding boxes, inverse-distance weights
 * of Eq. w_pc, NAG face weights of Sec. 2.2.1) in kernels, and allocates all
 * per-step scratch.  Synchronous.  Fails with VOF_ERR_BAD_MESH on an index out
 * of range, a cell tetrahedron of non-positive volume, a face of fewer than 3
 * or more than 8 points, a cell of more than 96 tetrahedra (a face of n > 3
 * points gives n; 2:1 octree cells have up to 78), or periodic data that do
 * not fit together (a copy not owned by its face's neighbour or not the same
 * points one translation away, images more than one period apart, a cell
 * touching two images of one point).  *out receives a context the caller
 * releases with vof_destroy. */
int vof_create(const vof_mesh *mesh, const vof_options *opt, vof_ctx **out);
void vof_destroy(vof_ctx *ctx);

/* Geometry computed by vof_create, copied to caller DEVICE arrays (any may be
 * NULL): cell centres [3*n_cells], volumes [n_cells], face centres and area
 * vectors [3*n_faces]. */
int vof_geometry(vof_ctx *ctx, double *cell_centre, double *cell_vol, double *face_centre,
                 double *face_area, void *stream);

/* Gradient of the reconstruction (Sec. 2.2.1): VOF_GRAD_NAG (the default, the
 * node-averaged gradient) or VOF_GRAD_LSQ (the generalised least-squares
 * gradient over the cells sharing a point with each cell, Eq.
 * generalizedLSQminimize with inverse-distance weights).  Selecting LSQ the
 * first time builds its stencil (host, then device) and a gradient buffer:
 * synchronous, allocates.  Later reconstructions (vof_reconstruct,
 * vof_advect, ...) take the normal -grad/|grad| of the selected gradient.
 * VOF_ERR_INVALID_ARG for another kind. */
enum { VOF_GRAD_NAG = 0, VOF_GRAD_LSQ = 1 };
int vof_set_gradient(vof_ctx *ctx, int kind);

/* The generalised LSQ gradient (Sec. 2.2.1) of alpha for every cell, grad
 * [3*n_cells] SoA (device).  Builds the LSQ stencil first if no earlier call
 * did (synchronous then, and allocating). */
int vof_lsq_gradient(vof_ctx *ctx, const double *alpha, double *grad, void *stream);

/* Reconstruction error of Sec. 4.1 against a ball (ball[0..2] its centre,
 * ball[3] its radius; host array): per cell the volume of the symmetric
 * difference between the reconstructed phase (the PLIC polyhedron of an
 * oriented interface cell, the whole cell for a full one, nothing for any
 * other; flags, n [3*n_cells], d [n_cells] as vof_reconstruct writes them) and
 * the ball, E_vsd = E_vsd^- + E_vsd^+, into evsd [n_cells] (device).  The ball
 * is resolved like the paper's tool mesh: each cell tetrahedron split into
 * eight, `levels` times (0..6), pieces wholly in or out of the ball kept
 * whole, the undecided ones of the last level cut by the sphere's tangent
 * plane at the point nearest their centroid.  With flags NULL it gives the
 * ball's volume in each cell (exact volume fractions of that description).
 * VOF_ERR_INVALID_ARG for levels outside 0..6 or R <= 0. */
int vof_evsd(vof_ctx *ctx, const uint8_t *flags, const double *n, const double *d, const double ball[4],
             int levels, double *evsd, void *stream);

/* Geometric mapping of the volume fraction for adaptive refinement (Sec. 3,
 * Alg. 2): the volume fractions alpha_dst [dst n_cells] of a new mesh (dst)
 * from an old mesh of the same domain (src: alpha_src and its reconstruction
 * n_src [3*src n_cells], d_src, flags_src as vof_reconstruct on src writes
 * them).  pair_ptr [dst n_cells + 1] and pair_src (device, int32, caller-owned)
 * are Alg. 2's cell map: per destination cell the source cells sharing volume
 * with it, which must be nested with it -- the same cell, a cell containing it
 * (refinement) or cells inside it (un-refinement), as one octree lattice
 * gives.  A destination cell inside an oriented interface source takes the
 * part of the source's PLIC polyhedron it holds (its cell tetrahedra clipped
 * by the source plane); inside any other source it takes the source's
 * fraction; a source inside it adds its whole phase volume; cells count as
 * the same where their volumes agree to 1e-9.  The phase volume is conserved
 * to the positioning tolerance.  Both contexts on one device (else
 * VOF_ERR_INVALID_ARG); asynchronous on `stream`. */
int vof_remap(vof_ctx *dst, const vof_ctx *src, const double *alpha_src, const double *n_src, const double *d_src,
              const uint8_t *flags_src, const int32_t *pair_ptr, const int32_t *pair_src, double *alpha_dst,
              void *stream);

/* A4, Eq. idwpointphi: point velocity Up [3*n_points] from the cell velocity
 * Uc [3*n_cells] by inverse-distance weighting over the point's cells; at a
 * point on wall faces only the component tangent to the walls is kept. */
int vof_point_velocity(vof_ctx *ctx, const double *Uc, double *Up, void *stream);

/* A1-A3, Alg. 1 and Sec. 2.2: for every cell with eps < alpha < 1-eps, the NAG
 * gradient (Sec. 2.2.1), the unit normal n = -grad/|grad| (pointing out of the
 * phase), and the plane offset d with |C ^ {x : n.x <= d}| = alpha |C| found by
 * the secant iteration with bisection fallback (Sec. 2.2.2; stops at a fill
 * residual of 1e-13 or a bracket of 1e-15 of the cell's extent, at most 100
 * iterations).  A VOF_MIXED context finds the same plane by safeguarded Newton
 * steps on the fill (the cut area is its derivative), FP32 then FP64, with the
 * same stop.  Outputs (device): n [3*n_cells], d [n_cells], flags [n_cells]
 * (VOF_INTERFACE / VOF_ORIENTED / VOF_FULL), iters [n_cells] or NULL.  Cells
 * that are not oriented interface cells get n = 0, d = 0. */
int vof_reconstruct(vof_ctx *ctx, const double *alpha, double *n, double *d, uint8_t *flags,
                    int32_t *iters, void *stream);

/* A4-A5, Eqs. sweep and V_fS: signed volume Vswept [n_faces] of the flux
 * polyhedron of every face, each face triangle swept to b = a - lambda*Up*dt
 * and split into three tetrahedra (positive for a sweep against S_f).  lambda
 * [n_faces] may be NULL (lambda = 1); a negative lambda selects the normal
 * sweep -lambda*(F_f/|S_f|^2) S_f dt, which needs F (else F may be NULL). */
int vof_flux_polyhedra(vof_ctx *ctx, const double *Up, const double *F, const double *lambda,
                       double dt, double *Vswept, void *stream);

/* A5, Eq. VF: per face the sweep factor lambda with V_f(lambda) = F_f dt, the
 * root in the first of the sixteen intervals of (0, 2] across which
 * V_f - F_f dt changes sign (V_f is a cubic in lambda, solved by a bracketed
 * Newton iteration); lambda = -1 where no interval brackets a root (normal-sweep
 * fallback), 0 where F_f = 0.  iters [n_faces] or NULL. */
int vof_correct_flux(vof_ctx *ctx, const double *Up, const double *F, double dt, double *lambda,
                     int32_t *iters, void *stream);

/* A6, Eqs. S'_f, S''_f and vol-phase-flux: fluxed phase volume Valpha
 * [n_faces].  A face whose stencil cells all have alpha <= eps carries 0, all
 * >= 1-eps carries F_f dt; a boundary face with inflow carries 0 (empty
 * exterior); every other face sums, over its stencil cells s and the
 * tetrahedra T of its flux polyhedron and K of cell s, sign(T) |T ^ K ^ H_s|,
 * H_s the phase half-space {n_s.x <= d_s} of an oriented interface cell, all
 * of K for a full cell, alpha_s |T ^ K| for an unoriented one. */
int vof_phase_flux(vof_ctx *ctx, const double *alpha, const double *n, const double *d,
                   const uint8_t *flags, const double *Up, const double *F, const double *lambda,
                   double dt, double *Valpha, void *stream);

/* A7, Eq. alpha-discrete with Eq. own-nei: alpha_c -= (sum over owner faces of
 * Valpha - sum over neighbour faces) / |C_c|, in place, then the optional
 * conservative bounding pass; stats (device, VOF_S_LEN doubles) or NULL. */
int vof_update(vof_ctx *ctx, double *alpha, const double *Valpha, double *stats, void *stream);

/* Courant number of a step (the paper sets each time step from the Courant
 * number of the current velocity, Sec. 4.2): Co = max over cells of
 * (1/2) sum over the cell's faces |F_f| dt / |C_c|, which is (|u|+|v|+|w|)
 * dt / h for a uniform velocity on a uniform hexahedral mesh.  F [n_faces]
 * (device) as for vof_advect (a periodic face counts for both its cells, its
 * copy for none); co: one double (device), written.  Asynchronous on
 * `stream`.  A caller keeping a target Courant number takes the next
 * dt = dt * Co_target / Co.  VOF_ERR_INVALID_ARG for a null pointer or a
 * dt that is not finite and positive. */
int vof_courant(vof_ctx *ctx, const double *F, double dt, double *co, void *stream);

/* One full advection step A1-A7 over the narrow band: band classification,
 * reconstruction of interface cells, point velocities and flux correction of
 * band faces, phase fluxes, update.  alpha [n_cells] in/out, Uc [3*n_cells]
 * cell velocity at the step midpoint, F [n_faces] volumetric flux averaged over
 * the step (discretely divergence-free, Eq. discretedivergence), dt > 0.
 * The flux correction runs on a second stream of the context, beside the
 * reconstruction, forked from and joined back into `stream` (also under CUDA
 * graph capture); `stream` orders the whole step as one unit. */
int vof_advect(vof_ctx *ctx, double *alpha, const double *Uc, const double *F, double dt,
               double *stats, void *stream);

/* vof_advect with HOST arrays: alpha is copied to the context's device buffer
 * in order on `stream`, the step runs, alpha (and stats, VOF_S_LEN doubles, if
 * not NULL) is copied back.  Asynchronous on `stream`; the host arrays must
 * stay valid, and Uc and F hold this step's values, from the call until the
 * stream reaches the end of it.
 * Uc in pinned host memory that the device can address (the driver reports a
 * device pointer for it: cudaHostAlloc or cudaHostRegister memory on this
 * system) is read in place by the step's kernels over the CPU-GPU link: only
 * the band kernels read it, at the cells around band points.  F (read in full
 * by the classification) and pageable Uc are copied on an internal stream
 * (created, with its events, at the first call) into one of two device buffer
 * pairs, alternating by call, as soon as the step two calls back is done and
 * the previous call's alpha copy is in, so that those copies overlap the
 * previous step's kernels; they are not ordered after earlier work on
 * `stream`. */
int vof_advect_host(vof_ctx *ctx, double *alpha, const double *Uc, const double *F, double dt,
                    double *stats, void *stream);

/* ---- Batched form --------------------------------------------------------
 * Many independent cases of uneven size advanced together; the paper advances
 * one case and has no counterpart.  The cases' meshes are joined into one mesh
 * (disjoint union: concatenated points, cells and faces, the internal faces of
 * every case first), described by `mesh` as for vof_create, with
 * case_cell_ptr[ncases + 1] (host) the first cell of each case (0 first,
 * n_cells last, strictly increasing).  Synchronous; *out receives a batch the
 * caller releases with vof_batch_destroy.  Errors as vof_create, and
 * VOF_ERR_INVALID_ARG for bad case offsets or a periodic mesh. */
typedef struct vof_batch vof_batch;
int vof_batch_create(const vof_mesh *mesh, const int32_t *case_cell_ptr, int ncases, const vof_options *opt,
                     vof_batch **out);
void vof_batch_destroy(vof_batch *batch);

/* The batch's context (owned by the batch), for the other entry points. */
vof_ctx *vof_batch_context(vof_batch *batch);

/* One step of every case (A1-A7, as vof_advect) with each case's own time step
 * folded into its inputs: U_dt [3*n_cells] = U_c dt_case and F_dt [n_faces] =
 * F_f dt_case (the method uses the field only through these products), so the
 * step runs with dt = 1.  The step's kernels are captured into a CUDA graph at
 * the first call (again when an array pointer or the launch configuration
 * changes) and replayed as one graph launch on an internal stream that is
 * ordered after, and before, `stream` by events.  stats (device, VOF_S_LEN)
 * and case_mass (device [ncases]: sum of V alpha per case after the step, in a
 * fixed order) may be NULL.  Errors: VOF_ERR_INVALID_ARG, VOF_ERR_CUDA. */
int vof_batch_advect(vof_batch *batch, double *alpha, const double *U_dt, const double *F_dt, double *stats,
                     double *case_mass, void *stream);

/* Autotuner for the phase-flux launch of a mixed batch: times one step from
 * the state alpha (left unchanged: the steps run on a copy in the context's
 * staging buffer) for every launch configuration -- the per-warp staging of
 * clip pieces in shared memory (a stack of 92 pieces, or of 56 for more
 * resident warps), 1, 2 or 3 warps (faces) per block, and grid multipliers
 * 1, 2 and 4 over the resident blocks -- keeps the fastest for later steps,
 * and returns it as config = 256 * stack + 16 * warps + multiplier (stack 0:
 * 92 pieces, 1: 56) with its step time in ms (either pointer may be NULL).
 * An FP64 batch keeps its launch (config 0).  Synchronous on `stream`. */
int vof_batch_tune(vof_batch *batch, const double *alpha, const double *U_dt, const double *F_dt, int *config,
                   float *best_ms, void *stream);

/* The same autotuner for one context's vof_advect (inputs as vof_advect); the
 * choice holds for the context's later steps.  The paper has no counterpart. */
int vof_tune(vof_ctx *ctx, const double *alpha, const double *Uc, const double *F, double dt, int *config,
             float *best_ms, void *stream);

/* ---- Learned initial guess of the plane positioning ----------------------
 * The paper has no learned part.  A small network (VOF_MLP_IN features of an
 * interface cell -> two ReLU layers of VOF_MLP_HID -> VOF_MLP_OUT outputs: a
 * unit normal and the offset s = (d - d_min)/(d_max - d_min) of the plane in
 * the cell's projection range) with BF16 weights and activations and FP32
 * accumulation on the tensor cores, trained by Adam on the mean squared
 * error.  In a VOF_MIXED context with a network attached (vof_set_guess) the
 * Newton positioning of a cell starts from the network's offset (clamped to
 * [0.02, 0.98]) instead of the linear guess alpha; the root, the stop and the
 * normal (NAG's) are unchanged, so the plane is the same to the 1e-13 stop.
 * Parameters: one float array of VOF_MLP_NPARAM values, W1 [IN x HID]
 * (input-major), b1 [HID], W2 [HID x HID], b2 [HID], W3 [HID x OUT], b3 [OUT].
 * Features (vof_mlp_features): the volume fractions of the cell's 3x3x3
 * lattice neighbourhood (cells sharing a point with it, placed by the sign of
 * their centre offset beyond half the cell size; missing slots take the
 * cell's own value), then box extents / V^(1/3) (3), V / box volume,
 * faces / 24, points / 8. */
#define VOF_MLP_IN 33
#define VOF_MLP_HID 64
#define VOF_MLP_OUT 4
#define VOF_MLP_NPARAM (VOF_MLP_IN * VOF_MLP_HID + VOF_MLP_HID + VOF_MLP_HID * VOF_MLP_HID + VOF_MLP_HID + \
                        VOF_MLP_HID * VOF_MLP_OUT + VOF_MLP_OUT)
typedef struct vof_mlp vof_mlp;
/* A network on `device` with room for batches of up to max_batch (>= 16)
 * samples, initialised from params (host, VOF_MLP_NPARAM floats).
 * Synchronous; release with vof_mlp_destroy. */
int vof_mlp_create(int max_batch, const float *params, int device, vof_mlp **out);
void vof_mlp_destroy(vof_mlp *mlp);
/* Copies the current FP32 parameters to params (host).  Synchronous. */
int vof_mlp_params(vof_mlp *mlp, float *params);
/* Features of ncells cells (device list `cells`, or cells 0..ncells-1 when
 * NULL) from alpha (device) into feat (device, [ncells x VOF_MLP_IN]). */
int vof_mlp_features(vof_ctx *ctx, const double *alpha, const int32_t *cells, int ncells, float *feat,
                     void *stream);
/* Forward pass of n (<= max_batch) samples: feat (device [n x IN]) -> out
 * (device [n x OUT]). */
int vof_mlp_forward(vof_mlp *mlp, const float *feat, int n, float *out, void *stream);
/* Forward and backward pass of the mean squared error against target (device
 * [n x OUT]): gradient (device [VOF_MLP_NPARAM], or NULL) and the loss (host,
 * or NULL; reading it synchronises `stream`). */
int vof_mlp_gradient(vof_mlp *mlp, const float *feat, const float *target, int n, float *grad, float *loss,
                     void *stream);
/* One Adam step (beta 0.9, 0.999) with learning rate lr on a batch; loss as
 * vof_mlp_gradient. */
int vof_mlp_train_step(vof_mlp *mlp, const float *feat, const float *target, int n, float lr, float *loss,
                       void *stream);
/* Attaches (mlp) or detaches (NULL) the network whose offsets start the
 * positioning of vof_advect and vof_reconstruct in a VOF_MIXED context; the
 * network must live on the context's device and outlive its use.  Allocates
 * the context's guess buffers the first time (outside any capture). */
int vof_set_guess(vof_ctx *ctx, vof_mlp *mlp);

/* Kernel-group timing with CUDA events recorded on the launching stream.
 * vof_profile_begin arms recording for up to max_steps subsequent vof_advect
 * calls (creating events, no device memory); vof_profile_end synchronises on
 * the last event and returns, per group, the summed milliseconds over the
 * recorded steps: [0] band classification, [1] reconstruction, [2] flux
 * correction (the time it adds after the reconstruction, beside which it
 * runs), [3] phase flux, [4] update, bounding and statistics; *steps
 * receives the number of steps recorded.  Recording stops at max_steps. */
enum { VOF_PROF_GROUPS = 5 };
int vof_profile_begin(vof_ctx *ctx, int max_steps);
int vof_profile_end(vof_ctx *ctx, double *group_ms, int *steps);

/* Algorithmic work counted by the step kernels since the last reset, as
 * counts of primitives (a measurement helper; the paper gives no costs):
 *  [0] prism-plane distance sets (six signed point-plane distances: the flux
 *      polyhedron prism of one face triangle against one plane of a cell
 *      tetrahedron or a PLIC plane),
 *  [1] piece-plane tests (four signed distances),
 *  [2] edge intersections,
 *  [3] tetrahedron volumes,
 *  [4] closed-form cut fractions of a tetrahedron below a plane,
 *  [5] plane shifts into a face's frame (one dot product each),
 *  [6] band faces fluxed geometrically,
 *  [7] FP64 fill evaluations of the positioning, per cell tetrahedron,
 *  [8] FP32 fill evaluations of the positioning, per cell tetrahedron,
 *  [9] face triangles whose swept prism enters the correction's cubic,
 *  [10] cubic evaluations of the correction,
 *  [11] reserved (0).
 * [0]-[5] are FP32 work in a VOF_MIXED context and FP64 in a VOF_FP64 one;
 * [7], [9], [10] are FP64.  Reading synchronises `stream`; reset zeroes the
 * counters. */
enum { VOF_WORK_LEN = 12 };
/* Work counting on (1) or off (0, the default): while on, later steps run
 * instrumented variants of the reconstruction, correction and phase-flux
 * kernels that add to the counters read by vof_work_counts; while off, the
 * uninstrumented ones run and the counters stay as they are.  A host-side
 * setting, effective for calls made after it. */
int vof_count_work(vof_ctx *ctx, int on);
int vof_work_counts(vof_ctx *ctx, unsigned long long counts[VOF_WORK_LEN], int reset, void *stream);

/* Measurement helper with no counterpart in the paper: sustained fused
 * multiply-add rate (FLOP/s, 2 per FMA) of the plain FP64 (VOF_FP64) or FP32
 * (VOF_MIXED) pipes of `device`, the roofline peak of arithmetic-bound kernels.
 * Synchronous; allocates and frees one scalar of device memory. */
int vof_probe_fma(int device, int precision, double *flops_per_s, void *stream);

/* Check of the grid barrier inside the cooperative bounding kernel (no paper
 * counterpart): a cooperative launch of two blocks per SM that pass four
 * barriers, with a wait limit of 2000 polls (milliseconds).  skip_block >= 0
 * makes that block leave at once, so that the others' waits run out: they set
 * VOF_ST_TIMEOUT in the status word (vof_status) and leave; no wait is
 * unbounded and the context stays usable.  skip_block = -1: every block
 * arrives and nothing is flagged.  Asynchronous on `stream`; skip_block beyond
 * the launch's blocks, or below -1: VOF_ERR_INVALID_ARG. */
int vof_probe_barrier(vof_ctx *ctx, int skip_block, void *stream);

/* Reconstruction for callers that cannot allocate device memory when they
 * call it -- code inside a host framework that owns every device allocation,
 * or a real-time loop that forbids cudaMalloc after start-up.  The paper has
 * no counterpart: it is vof_reconstruct's computation (same outputs, same
 * arrays, same errors) run over a compacted list of the interface cells that
 * is kept in a file-scope device array of VOF_STATIC_MAX_CELLS ints (16 MiB,
 * held by every GPU that loads the library until the process exits), not in
 * memory the caller or the context allocates.  It calls no allocating routine.
 * - The context must exist (vof_create allocates; someone who can must call it).
 * - n_cells > VOF_STATIC_MAX_CELLS is rejected with VOF_ERR_INVALID_ARG.
 * - The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any
 *   stream capture.
 * - Every call on a device shares the one array: the list length is cleared
 *   at the start of each call, and calls that overlap on the GPU (different
 *   streams, or different contexts on the same device) race.
 * - Iteration counts are not returned. */
#define VOF_STATIC_MAX_CELLS (1 << 22)
int vof_reconstruct_static(vof_ctx *ctx, const double *alpha, double *n, double *d, uint8_t *flags,
                           void *stream);

/* Reads (synchronising `stream`) and clears the device status word. */
int vof_status(vof_ctx *ctx, uint32_t *bits, void *stream);

/* Number of kernel launches the last vof_advect enqueued. */
int vof_last_launch_count(vof_ctx *ctx);

const char *vof_error_string(int code);
/* Why the last vof_create (or vof_batch_create) on the calling thread returned
 * VOF_ERR_BAD_MESH: a static string naming the failed check ("" when the last
 * call did not fail that way).  Owned by the library. */
const char *vof_create_error(void);

#ifdef __cplusplus
}
#endif
#endif

/*
 * vof_oracle.h -- plain FP64 CPU oracle of the unsplit geometric VoF step of
 * Maric, Marschall & Bothe (2013).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the reference that the CUDA path
 * is checked against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it; the product library never does, and
 * the two share no source, header or helper.
 *
 * Conventions (all arrays caller-owned, host memory):
 *   mesh   : points px/py/pz[n_points]; face f has points
 *            face_pts[face_ptr[f] .. face_ptr[f+1]) ordered so that the
 *            right-hand normal S_f points from owner[f] to neighbour[f]
 *            (internal faces 0..n_internal-1) or out of the domain (boundary
 *            faces).  Sec. 2, Eq. own-nei.
 *   vectors: structure of arrays, x block then y block then z block.
 *   flags  : per cell, VO_INTERFACE (eps < alpha < 1-eps), VO_ORIENTED
 *            (interface cell with a usable normal), VO_FULL (alpha >= 1-eps).
 * Every loop runs item by item in a fixed order per item, so results do not
 * depend on the thread count.
 */
#ifndef VOF_ORACLE_H
#define VOF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { VO_INTERFACE = 1, VO_ORIENTED = 2, VO_FULL = 4 };
enum { VO_ST_POS_NOT_CONVERGED = 1, VO_ST_CORR_NOT_CONVERGED = 2, VO_ST_BAD_VOLUME = 4,
       VO_ST_CLIP_OVERFLOW = 8, VO_ST_BOUNDARY_INFLOW_PHASE = 16, VO_ST_BOUND_RESIDUAL = 32 };

/* stats[] layout written by vo_update / vo_advect */
enum { VO_S_MASS_BEFORE = 0, VO_S_MASS_AFTER, VO_S_MIN_PRE, VO_S_MAX_PRE, VO_S_MIN_POST,
       VO_S_MAX_POST, VO_S_N_INTERFACE, VO_S_N_BAND, VO_S_MAX_POS_IT, VO_S_MAX_CORR_IT,
       VO_S_BOUNDARY_OUT, VO_S_STATUS,
       VO_S_BOUND_PASSES,   /* local redistribution passes that moved something */
       VO_S_BOUND_GLOBAL,   /* volume left to the global fallback after them */
       VO_S_LEN };

typedef struct vo_mesh vo_mesh;

/* wall[n_faces - n_internal]: 1 marks a wall boundary face (no normal flow);
 * NULL makes every boundary face a wall */
vo_mesh *vo_mesh_create(int n_points, int n_faces, int n_internal, int n_cells,
                        const double *px, const double *py, const double *pz,
                        const int *face_ptr, const int *face_pts, const int *owner,
                        const int *neighbour, const unsigned char *wall);
/* Periodic meshes (reading R21): period[9] holds the period vectors L0, L1,
 * L2 (rows); point_master[p] is the point p is an image of and
 * point_image[3p..3p+2] in {-1, 0, 1} the periods between them,
 * P[p] = P[master] + sum_i k_i L_i; face_image[b - n_internal] is, for a
 * boundary face that is the neighbour's copy of a periodic internal face, that
 * internal face (else -1).  NULL on failure (malformed periodic data, a cell
 * touching two images of one point). */
vo_mesh *vo_mesh_create_periodic(int n_points, int n_faces, int n_internal, int n_cells,
                                 const double *px, const double *py, const double *pz,
                                 const int *face_ptr, const int *face_pts, const int *owner,
                                 const int *neighbour, const unsigned char *wall, const double *period,
                                 const int *point_master, const signed char *point_image,
                                 const int *face_image);
void vo_mesh_destroy(vo_mesh *m);
int vo_set_threads(int n);

/* R1 geometry: face centre (point mean), fan area vector, cell centre (mean of
 * the cell's points), cell volume (sum of its centre-apex tetrahedra). */
void vo_geometry(const vo_mesh *m, double *cell_centre, double *cell_vol,
                 double *face_centre, double *face_area);
/* Courant number: max over cells of (1/2) sum_f |F_f| dt / V_c */
double vo_courant(const vo_mesh *m, const double *F, double dt);
/* number of cells in the face stencil (cells sharing a point with the face) */
int vo_stencil(const vo_mesh *m, int face, int *out, int cap);
/* the same with each cell's translation code (i+1) + 3(j+1) + 9(k+1) for
 * i L0 + j L1 + k L2 (13: none) */
int vo_stencil_codes(const vo_mesh *m, int face, int *out, int *codes, int cap);

/* Eq. idwpointphi: cell -> point inverse-distance interpolation of one scalar */
void vo_point_interp(const vo_mesh *m, const double *phi_c, double *phi_p);
/* NAG gradient (Sec. 2.2.1) for the selected cells (all when sel == NULL) */
void vo_nag_gradient(const vo_mesh *m, const double *alpha, int n_sel, const int *sel,
                     double *grad);

/* |C_c ^ {x : n.x <= d}| by clipping and capping every centre-apex tetrahedron */
double vo_cut_volume(const vo_mesh *m, int cell, const double n[3], double d);
/* Alg. 1 for one cell with a given unit normal: d with |C ^ {n.x <= d}| = alpha V;
 * returns the iterations taken (POS_MAXIT = 100 means not converged) */
int vo_position(const vo_mesh *m, int cell, double alpha, const double n[3], double *d);
/* Alg. 1 for the selected cells (all when sel == NULL); n (3*nc SoA), d, flags,
 * iters are indexed by cell.  Returns status bits. */
int vo_reconstruct(const vo_mesh *m, const double *alpha, double eps, int n_sel,
                   const int *sel, double *n, double *d, unsigned char *flags, int *iters);

/* Alg. 1 with the normal -grad/|grad| of a given gradient (3*nc SoA; NULL: NAG) */
int vo_reconstruct_grad(const vo_mesh *m, const double *alpha, const double *grad, double eps, int n_sel,
                        const int *sel, double *n, double *d, unsigned char *flags, int *iters);
/* generalised least-squares gradient (Sec. 2.2.1, Eq. generalizedLSQminimize)
 * over the cells sharing a point with each selected cell */
void vo_lsq_gradient(const vo_mesh *m, const double *phi, int n_sel, const int *sel, double *grad);
/* reconstruction error E_vsd (Sec. 4.1) per selected cell against the ball
 * ball[0..2] centre, ball[3] radius, resolved to `levels` splits of the cell
 * tetrahedra; flags NULL: no reconstruction (gives |C ^ ball|) */
void vo_evsd(const vo_mesh *m, const unsigned char *flags, const double *n, const double *d,
             const double ball[4], int levels, int n_sel, const int *sel, double *out);

/* geometric mapping of the volume fraction (Sec. 3, Alg. 2) from a source
 * mesh (alpha, its reconstruction n, d, flags) onto a destination mesh of the
 * same domain; pair_ptr [dst n_cells + 1] / pair_src list, per destination
 * cell, the source cells sharing volume with it (nested cells) */
int vo_remap(const vo_mesh *dst, const vo_mesh *src, const double *alpha_src, const double *n_src,
             const double *d_src, const unsigned char *flags_src, const int *pair_ptr, const int *pair_src,
             double *alpha_dst);

/* Eq. idwpointphi applied to the cell velocity (3*nc SoA) -> point velocity; at
 * wall points only the component tangent to the walls is kept */
void vo_point_velocity(const vo_mesh *m, const double *Uc, double *Up);
/* signed volume of the flux polyhedron of face f swept by lambda*Up*dt (Eq. sweep);
 * lambda < 0 selects the normal sweep -lambda*(F_f/|S_f|^2) S_f dt */
double vo_swept_volume(const vo_mesh *m, int face, const double *Up, double F, double dt,
                       double lambda);
/* secant correction of the sweep parameter so that V_f(lambda) = F_f dt (Eq. VF);
 * lambda = -1 marks faces that take the normal-sweep fallback */
int vo_correct_flux(const vo_mesh *m, const double *Up, const double *F, double dt, int n_sel,
                    const int *sel, double *lambda, int *iters);
/* fluxed phase volume per face (Eqs. S'_f, S''_f); returns status bits */
int vo_phase_flux(const vo_mesh *m, const double *alpha, double eps, const double *n,
                  const double *d, const unsigned char *flags, const double *Up,
                  const double *F, const double *lambda, double dt, int n_sel, const int *sel,
                  double *Valpha);
/* sum over stencil cells of |S_f ^ C_s| with the polyhedron's signs (coverage) */
double vo_stencil_coverage(const vo_mesh *m, int face, const double *Up, double F, double dt,
                           double lambda);
/* Eq. alpha-discrete with Eq. own-nei; optional conservative redistribution of
 * over/undershoots (reading R10 of Sec. 2.3's wisp redistribution) */
int vo_update(const vo_mesh *m, double *alpha, const double *Valpha, int bound, double *stats);
/* full step: classify, reconstruct, point velocity, correct, phase flux, update */
int vo_advect(const vo_mesh *m, double *alpha, const double *Uc, const double *F, double dt,
              double eps, int bound, double *stats);
/* one-time band classification used by vo_advect: 0 empty-trivial, 1 full-trivial,
 * 2 geometric, per face */
void vo_classify_faces(const vo_mesh *m, const double *alpha, double eps, unsigned char *cls);

/* primitives, exported for the pin tests */
double vo_tet_clip_volume(const double *tet12, int n_planes, const double *planes4);
double vo_signed_tet_volume(const double *tet12);

#ifdef __cplusplus
}
#endif
#endif

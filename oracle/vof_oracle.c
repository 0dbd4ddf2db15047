/*
 * vof_oracle.c -- plain FP64 CPU oracle of the unsplit geometric VoF advection
 * step of Maric, Marschall & Bothe (2013).  TEST INFRASTRUCTURE ONLY: it is the
 * reference that the CUDA path is checked against and is never called by it.
 *
 * Slow on purpose.  Geometry is done the way the paper describes it:
 *  - convex polyhedra are clipped face by face and capped with a cap polygon
 *    whose points are ordered by an angle insertion sort (Sec. 2.1);
 *  - intersections of two convex polyhedra are repeated plane clips (Sec. 2.1);
 *  - the NAG gradient follows Sec. 2.2.1 step by step;
 *  - interface positioning is the secant iteration with a bisection fallback
 *    of Alg. 1 (Sec. 2.2.2);
 *  - flux polyhedra come from the face sweep of Eq. sweep, their volume from a
 *    tetrahedral decomposition (Eq. V_fS), and the sweep is corrected by a
 *    secant iteration until Eq. VF holds (Sec. 2.3);
 *  - phase volumes are the intersections of Eqs. S'_f and S''_f, and the update
 *    is Eq. alpha-discrete in the owner/neighbour form of Eq. own-nei.
 * Readings where the paper is silent (cell solids, stencil, tolerances, the
 * narrow band, the bounding pass) are stated where they are used.
 * Compiled with -ffp-contract=off so no fused multiply-add changes rounding.
 */
#include "vof_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- vectors */
typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r; r.x = x; r.y = y; r.z = z; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b)
{
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double norm(v3 a) { return sqrt(dot(a, a)); }
/* signed volume of tetrahedron (a,b,c,d): (b-a).((c-a)x(d-a))/6 */
static double tetvol(v3 a, v3 b, v3 c, v3 d)
{
    return dot(sub(b, a), cross(sub(c, a), sub(d, a))) / 6.0;
}

/* ------------------------------------------------------------------ mesh */
struct vo_mesh {
    int np, nf, ni, nc;
    v3 *P;
    int *fptr, *fpts, *own, *nei;
    int *cptr, *cface;   /* cell -> faces, ascending face index */
    int *cpptr, *cpt;    /* cell -> its distinct points, ascending */
    int *pptr, *pcell;   /* point -> cells, ascending */
    double *w;           /* inverse-distance weight of each (point, cell) entry */
    v3 *cf, *sf, *cc;
    double *vc;
    unsigned char *wall; /* per boundary face: 1 = wall */
    int *pwn;            /* per point: number of distinct wall normals (0..3) */
    v3 *pwv;             /* per point: up to two wall normals */
    /* periodic meshes (R21); for others pmaster[p] = p and every code is T0 */
    v3 L[3];             /* period vectors */
    int *pmaster;        /* per point: the master point it is an image of */
    int *fimg;           /* per boundary face: the internal face it copies, or -1 */
    unsigned char *pcode;/* per (point, cell) entry: translation of the cell to the point */
};

/* A translation by i L0 + j L1 + k L2, i, j, k in {-1, 0, 1}, is coded
 * (i+1) + 3 (j+1) + 9 (k+1); T0 is no translation. */
#define T0 13
static v3 tvec(const vo_mesh *m, int code);

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}
static int cmp_long(const void *a, const void *b)
{
    long long x = *(const long long *)a, y = *(const long long *)b;
    return (x > y) - (x < y);
}

int vo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static int fn(const vo_mesh *m, int f) { return m->fptr[f + 1] - m->fptr[f]; }
static v3 fp(const vo_mesh *m, int f, int i) { return m->P[m->fpts[m->fptr[f] + i]]; }
/* R1: a face with three points is its own triangle; a face with more points is
 * the fan of triangles (c_f, p_i, p_i+1) about the mean point c_f, the
 * triangulation the paper uses for the NAG face values (Sec. 2.2.1). */
static int ntri(const vo_mesh *m, int f) { int n = fn(m, f); return n == 3 ? 1 : n; }
static void face_tri(const vo_mesh *m, int f, int t, v3 o[3])
{
    int n = fn(m, f);
    if (n == 3) { o[0] = fp(m, f, 0); o[1] = fp(m, f, 1); o[2] = fp(m, f, 2); }
    else { o[0] = m->cf[f]; o[1] = fp(m, f, t); o[2] = fp(m, f, (t + 1) % n); }
}

static v3 tvec(const vo_mesh *m, int code)
{
    int i = code % 3 - 1, j = (code / 3) % 3 - 1, k = code / 9 - 1;
    return add(add(scl(m->L[0], (double)i), scl(m->L[1], (double)j)), scl(m->L[2], (double)k));
}

/* R21: the cells around every image of each point, translated to it: per
 * point the union of its images' cells with code k(p) - k(q) (q the image that
 * lists the cell), sorted by (cell, code).  Fails when images differ by more
 * than one period or a cell lists two images of one point. */
static int periodic_rings(vo_mesh *m, const int *pm, const signed char *pimg)
{
    const int np = m->np;
    int i, total = 0, rc = 0;
    int *mptr = (int *)calloc((size_t)np + 1, sizeof(int));
    int *mem = (int *)malloc(sizeof(int) * (size_t)(np > 0 ? np : 1));
    int *fill = (int *)calloc((size_t)(np > 0 ? np : 1), sizeof(int));
    int *pptr2 = (int *)calloc((size_t)np + 1, sizeof(int)), *pcell2 = NULL;
    unsigned char *pcode2 = NULL;
    for (i = 0; i < np; i++) {
        if (pm[i] < 0 || pm[i] >= np || pm[pm[i]] != pm[i]) { rc = -1; goto out; }
        mptr[pm[i] + 1]++;
    }
    for (i = 0; i < np; i++) mptr[i + 1] += mptr[i];
    for (i = 0; i < np; i++) mem[mptr[pm[i]] + fill[pm[i]]++] = i;
    for (i = 0; i < np; i++) {
        int j, k = 0;
        for (j = mptr[pm[i]]; j < mptr[pm[i] + 1]; j++) k += m->pptr[mem[j] + 1] - m->pptr[mem[j]];
        pptr2[i + 1] = pptr2[i] + k;
    }
    total = pptr2[np];
    pcell2 = (int *)malloc(sizeof(int) * (size_t)(total > 0 ? total : 1));
    pcode2 = (unsigned char *)malloc((size_t)(total > 0 ? total : 1));
    for (i = 0; i < np; i++) {
        int j, k = pptr2[i], a, b;
        for (j = mptr[pm[i]]; j < mptr[pm[i] + 1]; j++) {
            int r = mem[j], e, d[3];
            for (e = 0; e < 3; e++) {
                d[e] = pimg[3 * i + e] - pimg[3 * r + e];
                if (d[e] < -1 || d[e] > 1) { rc = -1; goto out; }
            }
            for (e = m->pptr[r]; e < m->pptr[r + 1]; e++, k++) {
                pcell2[k] = m->pcell[e];
                pcode2[k] = (unsigned char)((d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1));
            }
        }
        for (a = pptr2[i] + 1; a < pptr2[i + 1]; a++) /* insertion sort by (cell, code) */
            for (b = a; b > pptr2[i] && (pcell2[b] < pcell2[b - 1] ||
                                         (pcell2[b] == pcell2[b - 1] && pcode2[b] < pcode2[b - 1])); b--) {
                int t = pcell2[b];
                unsigned char u = pcode2[b];
                pcell2[b] = pcell2[b - 1]; pcode2[b] = pcode2[b - 1];
                pcell2[b - 1] = t; pcode2[b - 1] = u;
            }
        for (a = pptr2[i] + 1; a < pptr2[i + 1]; a++)
            if (pcell2[a] == pcell2[a - 1]) { rc = -1; goto out; }
    }
    free(m->pptr); free(m->pcell); free(m->pcode);
    m->pptr = pptr2; m->pcell = pcell2; m->pcode = pcode2;
    pptr2 = NULL; pcell2 = NULL; pcode2 = NULL;
out:
    free(mptr); free(mem); free(fill); free(pptr2); free(pcell2); free(pcode2);
    return rc;
}

vo_mesh *vo_mesh_create(int n_points, int n_faces, int n_internal, int n_cells,
                        const double *px, const double *py, const double *pz,
                        const int *face_ptr, const int *face_pts, const int *owner,
                        const int *neighbour, const unsigned char *wall)
{
    return vo_mesh_create_periodic(n_points, n_faces, n_internal, n_cells, px, py, pz, face_ptr, face_pts,
                                   owner, neighbour, wall, NULL, NULL, NULL, NULL);
}

/* Reading R21, periodic meshes (the paper's translation case runs on a
 * periodic box, Sec. 4.2; the paper does not say how the sides are joined).
 * Every point is an image of a master point, P[p] = P[m] + sum_i k_i L_i with
 * m = point_master[p], k = point_image[3p..3p+2] in {-1, 0, 1}; the images of
 * one master are one point of the periodic domain.  A face of a periodic side,
 * given with its points on its owner's side, is an internal face whose
 * neighbour lies across the period; the neighbour's own copy of the face (its
 * points on the other side) is a boundary face with face_image[b - n_internal]
 * = that internal face.  A cell is built from its own faces: the neighbour
 * takes the copy, not the internal face.  The copy carries no flux: the
 * internal face's phase flux leaves its owner and enters the copy's owner,
 * who is the face's neighbour.  The cells around a point are the cells around
 * every image of it, each translated to this image; face stencils, inverse-
 * distance weights and the LSQ stencil take the translated cells.  Sweep keys
 * (R5) are master indices, so that a side quad of two prisms across the
 * period is split the same way in both. */
vo_mesh *vo_mesh_create_periodic(int n_points, int n_faces, int n_internal, int n_cells,
                                 const double *px, const double *py, const double *pz,
                                 const int *face_ptr, const int *face_pts, const int *owner,
                                 const int *neighbour, const unsigned char *wall, const double *period,
                                 const int *point_master, const signed char *point_image,
                                 const int *face_image)
{
    vo_mesh *m = (vo_mesh *)calloc(1, sizeof(vo_mesh));
    int i, f, c;
    const int nb = n_faces - n_internal;
    int *imaged = (int *)calloc((size_t)(n_internal > 0 ? n_internal : 1), sizeof(int));
    m->np = n_points; m->nf = n_faces; m->ni = n_internal; m->nc = n_cells;
    m->P = (v3 *)malloc(sizeof(v3) * (size_t)n_points);
    for (i = 0; i < n_points; i++) m->P[i] = mk(px[i], py[i], pz[i]);
    m->fptr = (int *)malloc(sizeof(int) * (size_t)(n_faces + 1));
    memcpy(m->fptr, face_ptr, sizeof(int) * (size_t)(n_faces + 1));
    m->fpts = (int *)malloc(sizeof(int) * (size_t)face_ptr[n_faces]);
    memcpy(m->fpts, face_pts, sizeof(int) * (size_t)face_ptr[n_faces]);
    m->own = (int *)malloc(sizeof(int) * (size_t)n_faces);
    memcpy(m->own, owner, sizeof(int) * (size_t)n_faces);
    m->nei = (int *)malloc(sizeof(int) * (size_t)(n_internal > 0 ? n_internal : 1));
    if (n_internal > 0) memcpy(m->nei, neighbour, sizeof(int) * (size_t)n_internal);

    /* R21 data */
    m->pmaster = (int *)malloc(sizeof(int) * (size_t)(n_points > 0 ? n_points : 1));
    m->fimg = (int *)malloc(sizeof(int) * (size_t)(nb > 0 ? nb : 1));
    for (i = 0; i < n_points; i++) m->pmaster[i] = point_master ? point_master[i] : i;
    for (i = 0; i < nb; i++) m->fimg[i] = face_image ? face_image[i] : -1;
    for (i = 0; i < 3; i++) m->L[i] = period ? mk(period[3 * i], period[3 * i + 1], period[3 * i + 2]) : mk(0, 0, 0);
    if (point_master && !point_image) goto bad;
    for (i = 0; i < nb; i++)
        if (m->fimg[i] >= 0) {
            /* the copy: owned by the internal face's neighbour, the same points
             * up to one translation */
            int a = m->fimg[i], b = n_internal + i, j, k, e, d0[3] = {0, 0, 0};
            if (a >= n_internal || imaged[a] || neighbour[a] != owner[b] || !point_master) goto bad;
            if (face_ptr[a + 1] - face_ptr[a] != face_ptr[b + 1] - face_ptr[b]) goto bad;
            for (j = face_ptr[a]; j < face_ptr[a + 1]; j++) {
                int pa = face_pts[j], pb = -1;
                for (k = face_ptr[b]; k < face_ptr[b + 1]; k++)
                    if (point_master[face_pts[k]] == point_master[pa]) pb = face_pts[k];
                if (pb < 0) goto bad;
                for (e = 0; e < 3; e++) {
                    int d = point_image[3 * pa + e] - point_image[3 * pb + e];
                    if (j == face_ptr[a]) d0[e] = d;
                    else if (d != d0[e]) goto bad;
                }
            }
            imaged[a] = 1;
        }

    /* cell -> faces (its own faces: an imaged internal face belongs to its owner
     * only, its neighbour has the copy) */
    m->cptr = (int *)calloc((size_t)n_cells + 1, sizeof(int));
    for (f = 0; f < n_faces; f++) {
        m->cptr[owner[f] + 1]++;
        if (f < n_internal && !imaged[f]) m->cptr[neighbour[f] + 1]++;
    }
    for (c = 0; c < n_cells; c++) m->cptr[c + 1] += m->cptr[c];
    m->cface = (int *)malloc(sizeof(int) * (size_t)m->cptr[n_cells]);
    {
        int *fill = (int *)calloc((size_t)n_cells, sizeof(int));
        for (f = 0; f < n_faces; f++) {
            c = owner[f]; m->cface[m->cptr[c] + fill[c]++] = f;
            if (f < n_internal && !imaged[f]) { c = neighbour[f]; m->cface[m->cptr[c] + fill[c]++] = f; }
        }
        free(fill);
    }
    /* cell -> distinct points */
    {
        int total = 0, *tmp, cap = 0;
        m->cpptr = (int *)calloc((size_t)n_cells + 1, sizeof(int));
        for (c = 0; c < n_cells; c++) {
            int k = 0;
            for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) k += fn(m, m->cface[i]);
            if (k > cap) cap = k;
            total += k;
        }
        m->cpt = (int *)malloc(sizeof(int) * (size_t)total);
        tmp = (int *)malloc(sizeof(int) * (size_t)(cap > 0 ? cap : 1));
        total = 0;
        for (c = 0; c < n_cells; c++) {
            int k = 0, u = 0, j;
            for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) {
                int g = m->cface[i];
                for (j = m->fptr[g]; j < m->fptr[g + 1]; j++) tmp[k++] = m->fpts[j];
            }
            qsort(tmp, (size_t)k, sizeof(int), cmp_int);
            for (j = 0; j < k; j++)
                if (j == 0 || tmp[j] != tmp[j - 1]) m->cpt[total + u++] = tmp[j];
            total += u;
            m->cpptr[c + 1] = total;
        }
        free(tmp);
    }
    /* point -> cells: the cells that list the point */
    m->pptr = (int *)calloc((size_t)n_points + 1, sizeof(int));
    for (i = 0; i < m->cpptr[n_cells]; i++) m->pptr[m->cpt[i] + 1]++;
    for (i = 0; i < n_points; i++) m->pptr[i + 1] += m->pptr[i];
    m->pcell = (int *)malloc(sizeof(int) * (size_t)(m->pptr[n_points] > 0 ? m->pptr[n_points] : 1));
    {
        int *fill = (int *)calloc((size_t)n_points, sizeof(int));
        for (c = 0; c < n_cells; c++)
            for (i = m->cpptr[c]; i < m->cpptr[c + 1]; i++) {
                int p = m->cpt[i];
                m->pcell[m->pptr[p] + fill[p]++] = c;
            }
        free(fill);
    }
    m->pcode = (unsigned char *)malloc((size_t)(m->pptr[n_points] > 0 ? m->pptr[n_points] : 1));
    memset(m->pcode, T0, (size_t)(m->pptr[n_points] > 0 ? m->pptr[n_points] : 1));
    if (point_master && periodic_rings(m, point_master, point_image)) goto bad;
    /* R1 geometry */
    m->cf = (v3 *)malloc(sizeof(v3) * (size_t)n_faces);
    m->sf = (v3 *)malloc(sizeof(v3) * (size_t)n_faces);
    for (f = 0; f < n_faces; f++) {
        int n = fn(m, f), t;
        v3 s = mk(0, 0, 0);
        for (i = 0; i < n; i++) s = add(s, fp(m, f, i));
        m->cf[f] = scl(s, 1.0 / n);
        s = mk(0, 0, 0);
        for (t = 0; t < ntri(m, f); t++) {
            v3 T[3];
            face_tri(m, f, t, T);
            s = add(s, scl(cross(sub(T[1], T[0]), sub(T[2], T[0])), 0.5));
        }
        m->sf[f] = s;
    }
    m->cc = (v3 *)malloc(sizeof(v3) * (size_t)n_cells);
    m->vc = (double *)malloc(sizeof(double) * (size_t)n_cells);
    for (c = 0; c < n_cells; c++) {
        v3 s = mk(0, 0, 0);
        double V = 0.0;
        int k = m->cpptr[c + 1] - m->cpptr[c];
        for (i = m->cpptr[c]; i < m->cpptr[c + 1]; i++) s = add(s, m->P[m->cpt[i]]);
        m->cc[c] = scl(s, 1.0 / k);
        for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) {
            int g = m->cface[i], t;
            for (t = 0; t < ntri(m, g); t++) {
                v3 T[3];
                face_tri(m, g, t, T);
                if (m->own[g] == c) V += tetvol(m->cc[c], T[0], T[1], T[2]);
                else V += tetvol(m->cc[c], T[0], T[2], T[1]);
            }
        }
        m->vc[c] = V;
    }
    /* reading R2: wall faces allow no normal flow, so the point velocity at a wall
     * point keeps only its component tangent to every wall through the point */
    m->wall = (unsigned char *)malloc((size_t)(n_faces - n_internal > 0 ? n_faces - n_internal : 1));
    for (f = n_internal; f < n_faces; f++) m->wall[f - n_internal] = wall ? wall[f - n_internal] : 1;
    m->pwn = (int *)calloc((size_t)n_points, sizeof(int));
    m->pwv = (v3 *)calloc(2 * (size_t)n_points, sizeof(v3));
    for (f = n_internal; f < n_faces; f++) {
        v3 u;
        if (!m->wall[f - n_internal] || m->fimg[f - n_internal] >= 0) continue; /* a copy is no wall */
        u = scl(m->sf[f], 1.0 / norm(m->sf[f]));
        for (i = m->fptr[f]; i < m->fptr[f + 1]; i++) {
            int p = m->fpts[i], k, dup = 0;
            for (k = 0; k < m->pwn[p] && k < 2; k++)
                if (fabs(dot(u, m->pwv[2 * p + k])) > 1.0 - 1e-12) dup = 1;
            if (dup || m->pwn[p] >= 3) continue;
            if (m->pwn[p] < 2) m->pwv[2 * p + m->pwn[p]] = u;
            m->pwn[p]++;
        }
    }
    /* Eq. w_pc: inverse distance between the point and the point-cell centre */
    m->w = (double *)malloc(sizeof(double) * (size_t)(m->pptr[n_points] > 0 ? m->pptr[n_points] : 1));
    for (i = 0; i < n_points; i++) {
        double s = 0.0;
        int j;
        for (j = m->pptr[i]; j < m->pptr[i + 1]; j++)
            s += 1.0 / norm(sub(m->P[i], add(m->cc[m->pcell[j]], tvec(m, m->pcode[j]))));
        for (j = m->pptr[i]; j < m->pptr[i + 1]; j++)
            m->w[j] = (1.0 / norm(sub(m->P[i], add(m->cc[m->pcell[j]], tvec(m, m->pcode[j]))))) / s;
    }
    free(imaged);
    return m;
bad:
    free(imaged);
    vo_mesh_destroy(m);
    return NULL;
}

void vo_mesh_destroy(vo_mesh *m)
{
    if (!m) return;
    free(m->P); free(m->fptr); free(m->fpts); free(m->own); free(m->nei);
    free(m->cptr); free(m->cface); free(m->cpptr); free(m->cpt); free(m->pptr);
    free(m->pcell); free(m->w); free(m->cf); free(m->sf); free(m->cc); free(m->vc);
    free(m->wall); free(m->pwn); free(m->pwv); free(m->pmaster); free(m->fimg); free(m->pcode);
    free(m);
}

void vo_geometry(const vo_mesh *m, double *cc, double *vc, double *cf, double *sf)
{
    int i;
    for (i = 0; i < m->nc; i++) {
        if (cc) { cc[i] = m->cc[i].x; cc[m->nc + i] = m->cc[i].y; cc[2 * m->nc + i] = m->cc[i].z; }
        if (vc) vc[i] = m->vc[i];
    }
    for (i = 0; i < m->nf; i++) {
        if (cf) { cf[i] = m->cf[i].x; cf[m->nf + i] = m->cf[i].y; cf[2 * m->nf + i] = m->cf[i].z; }
        if (sf) { sf[i] = m->sf[i].x; sf[m->nf + i] = m->sf[i].y; sf[2 * m->nf + i] = m->sf[i].z; }
    }
}

/* R7: the flux stencil of a face is every cell that shares a point with it
 * (point and edge neighbours, Sec. 2.3), listed in ascending order; on a
 * periodic mesh (R21) each with the translation that brings it next to the
 * face (a cell can appear at two translations), ordered by (cell, code). */
int vo_stencil_codes(const vo_mesh *m, int f, int *out, int *codes, int cap)
{
    int k = 0, i, j, u = 0;
    long long buf[1024];
    for (i = m->fptr[f]; i < m->fptr[f + 1]; i++) {
        int p = m->fpts[i];
        for (j = m->pptr[p]; j < m->pptr[p + 1]; j++)
            if (k < 1024) buf[k++] = (long long)m->pcell[j] * 32 + m->pcode[j];
    }
    qsort(buf, (size_t)k, sizeof(long long), cmp_long);
    for (i = 0; i < k; i++)
        if (i == 0 || buf[i] != buf[i - 1]) {
            if (u < cap) {
                out[u] = (int)(buf[i] / 32);
                if (codes) codes[u] = (int)(buf[i] % 32);
            }
            u++;
        }
    return u;
}

int vo_stencil(const vo_mesh *m, int f, int *out, int cap) { return vo_stencil_codes(m, f, out, NULL, cap); }

/* ---------------------------------------------------- A1: NAG gradient */
static double point_value(const vo_mesh *m, int p, const double *phi_c)
{
    double s = 0.0;
    int j;
    for (j = m->pptr[p]; j < m->pptr[p + 1]; j++) s += m->w[j] * phi_c[m->pcell[j]];
    return s; /* Eq. idwpointphi */
}

void vo_point_interp(const vo_mesh *m, const double *phi_c, double *phi_p)
{
    int p;
#pragma omp parallel for schedule(static)
    for (p = 0; p < m->np; p++) phi_p[p] = point_value(m, p, phi_c);
}

static v3 nag_gradient_cell(const vo_mesh *m, int c, const double *alpha)
{
    v3 g = mk(0, 0, 0);
    int i;
    for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) {
        int f = m->cface[i], n = fn(m, f), k;
        double phi1 = 0.0, sa = 0.0, sp = 0.0;
        double val[64];
        for (k = 0; k < n; k++) val[k] = point_value(m, m->fpts[m->fptr[f] + k], alpha);
        for (k = 0; k < n; k++) phi1 += val[k];
        phi1 /= n; /* initial face value: algebraic mean of the face points */
        for (k = 0; k < n; k++) {
            /* triangle (c_f, p_k, p_k+1): area weight and averaged value */
            v3 a = sub(fp(m, f, k), m->cf[f]), b = sub(fp(m, f, (k + 1) % n), m->cf[f]);
            double At = 0.5 * norm(cross(a, b));
            double pt = (phi1 + val[k] + val[(k + 1) % n]) / 3.0;
            sa += At;
            sp += At * pt;
        }
        /* Gauss theorem: owner faces add, neighbour faces subtract (Eq. own-nei) */
        if (m->own[f] == c) g = add(g, scl(m->sf[f], sp / sa));
        else g = sub(g, scl(m->sf[f], sp / sa));
    }
    return scl(g, 1.0 / m->vc[c]);
}

void vo_nag_gradient(const vo_mesh *m, const double *alpha, int n_sel, const int *sel, double *grad)
{
    int k, nn = sel ? n_sel : m->nc;
#pragma omp parallel for schedule(dynamic, 256)
    for (k = 0; k < nn; k++) {
        int c = sel ? sel[k] : k;
        v3 g = nag_gradient_cell(m, c, alpha);
        grad[c] = g.x; grad[m->nc + c] = g.y; grad[2 * m->nc + c] = g.z;
    }
}

/* ---------------------------------------- clipping and capping (Sec. 2.1) */
#define MAXF 12
#define MAXV 16
typedef struct {
    int nf;
    int nv[MAXF];
    v3 v[MAXF][MAXV];
} poly;

static void poly_tet(poly *P, v3 a, v3 b, v3 c, v3 d)
{
    if (tetvol(a, b, c, d) < 0) { v3 t = b; b = c; c = t; }
    /* faces oriented counter-clockwise seen from outside */
    P->nf = 4;
    P->nv[0] = 3; P->v[0][0] = a; P->v[0][1] = c; P->v[0][2] = b;
    P->nv[1] = 3; P->v[1][0] = a; P->v[1][1] = b; P->v[1][2] = d;
    P->nv[2] = 3; P->v[2][0] = a; P->v[2][1] = d; P->v[2][2] = c;
    P->nv[3] = 3; P->v[3][0] = b; P->v[3][1] = c; P->v[3][2] = d;
}

static double poly_volume(const poly *P)
{
    double V = 0.0;
    int f, i;
    v3 o;
    if (P->nf == 0) return 0.0;
    o = P->v[0][0];
    for (f = 0; f < P->nf; f++)
        for (i = 1; i + 1 < P->nv[f]; i++) V += tetvol(o, P->v[f][0], P->v[f][i], P->v[f][i + 1]);
    return V;
}

static int same(v3 a, v3 b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

/* Keep the part of P with n.x <= d.  Each face is clipped; the cut points
 * (edge crossings and vertices lying on the plane) are gathered, duplicates
 * dropped, and the cap face is added with its points ordered by the angle they
 * make about the cap centre (insertion sort).  Returns 0 with the result in Q,
 * 1 when no point of P is outside (P is the result), -1 on overflow. */
static int poly_clip(const poly *P, poly *Q, v3 n, double d)
{
    v3 cap[4 * MAXV];
    double sv[MAXF][MAXV], vmax = 0.0, tol;
    int ncap = 0, f, i, any_out = 0, any_in = 0;
    /* special cases (Sec. 2.1): a signed distance within a few rounding units of
     * zero is taken as exactly zero, so that faces lying in the clipping plane
     * are recognised as such instead of being cut into slivers */
    for (f = 0; f < P->nf; f++)
        for (i = 0; i < P->nv[f]; i++) {
            v3 v = P->v[f][i];
            if (fabs(v.x) > vmax) vmax = fabs(v.x);
            if (fabs(v.y) > vmax) vmax = fabs(v.y);
            if (fabs(v.z) > vmax) vmax = fabs(v.z);
        }
    tol = 1e-14 * (2.0 * norm(n) * vmax + fabs(d));
    for (f = 0; f < P->nf; f++)
        for (i = 0; i < P->nv[f]; i++) {
            double s = dot(n, P->v[f][i]) - d;
            if (fabs(s) <= tol) s = 0.0;
            sv[f][i] = s;
            if (s > 0) any_out = 1; else any_in = 1;
        }
    if (!any_out) return 1; /* nothing outside: P is unchanged */
    Q->nf = 0;
    if (!any_in) return 0;
    for (f = 0; f < P->nf; f++) {
        int k = P->nv[f], o = 0;
        v3 buf[MAXV];
        for (i = 0; i < k; i++) {
            v3 a = P->v[f][i], b = P->v[f][(i + 1) % k];
            double sa = sv[f][i], sb = sv[f][(i + 1) % k];
            if (sa <= 0) {
                if (o >= MAXV) return -1;
                buf[o++] = a;
                if (sa == 0) { if (ncap >= 4 * MAXV) return -1; cap[ncap++] = a; }
            }
            if ((sa < 0 && sb > 0) || (sa > 0 && sb < 0)) {
                /* interpolate from the inside end so both faces of an edge agree */
                v3 pi = sa < 0 ? a : b, po = sa < 0 ? b : a;
                double si = sa < 0 ? sa : sb, so = sa < 0 ? sb : sa;
                v3 x = add(pi, scl(sub(po, pi), si / (si - so)));
                if (o >= MAXV || ncap >= 4 * MAXV) return -1;
                buf[o++] = x;
                cap[ncap++] = x;
            }
        }
        if (o >= 3) {
            if (Q->nf >= MAXF) return -1;
            Q->nv[Q->nf] = o;
            for (i = 0; i < o; i++) Q->v[Q->nf][i] = buf[i];
            Q->nf++;
        }
    }
    {
        v3 u[4 * MAXV], c = mk(0, 0, 0), e1, e2;
        double ang[4 * MAXV];
        int nu = 0, j;
        for (i = 0; i < ncap; i++) {
            int dup = 0;
            for (j = 0; j < nu; j++) if (same(u[j], cap[i])) { dup = 1; break; }
            if (!dup) u[nu++] = cap[i];
        }
        if (nu >= 3) {
            for (i = 0; i < nu; i++) c = add(c, u[i]);
            c = scl(c, 1.0 / nu);
            e1 = sub(u[0], c);
            if (norm(e1) == 0.0) e1 = sub(u[1], c);
            e2 = cross(n, e1);
            for (i = 0; i < nu; i++) {
                v3 r = sub(u[i], c);
                ang[i] = atan2(dot(r, e2), dot(r, e1));
            }
            for (i = 1; i < nu; i++) { /* insertion sort by angle */
                double a = ang[i];
                v3 p = u[i];
                j = i - 1;
                while (j >= 0 && ang[j] > a) { ang[j + 1] = ang[j]; u[j + 1] = u[j]; j--; }
                ang[j + 1] = a; u[j + 1] = p;
            }
            if (Q->nf >= MAXF || nu > MAXV) return -1;
            Q->nv[Q->nf] = nu;
            for (i = 0; i < nu; i++) Q->v[Q->nf][i] = u[i];
            Q->nf++;
        }
    }
    return 0;
}

/* |tet ^ {x : n_k.x <= d_k, k < n_planes}| by repeated clipping (Sec. 2.1) */
static double tet_clip(v3 a, v3 b, v3 c, v3 d, int np, const v3 *n, const double *dd, int *st)
{
    poly A, B;
    poly *src = &A, *dst = &B, *t;
    int k;
    poly_tet(&A, a, b, c, d);
    for (k = 0; k < np; k++) {
        int r = poly_clip(src, dst, n[k], dd[k]);
        if (r < 0) { if (st) *st |= VO_ST_CLIP_OVERFLOW; return 0.0; }
        if (r == 1) continue;
        t = src; src = dst; dst = t;
        if (src->nf == 0) return 0.0;
    }
    return poly_volume(src);
}

double vo_tet_clip_volume(const double *t, int n_planes, const double *pl)
{
    v3 n[16];
    double dd[16];
    int k;
    for (k = 0; k < n_planes && k < 16; k++) { n[k] = mk(pl[4 * k], pl[4 * k + 1], pl[4 * k + 2]); dd[k] = pl[4 * k + 3]; }
    return tet_clip(mk(t[0], t[1], t[2]), mk(t[3], t[4], t[5]), mk(t[6], t[7], t[8]),
                    mk(t[9], t[10], t[11]), n_planes, n, dd, NULL);
}

double vo_signed_tet_volume(const double *t)
{
    return tetvol(mk(t[0], t[1], t[2]), mk(t[3], t[4], t[5]), mk(t[6], t[7], t[8]), mk(t[9], t[10], t[11]));
}

/* R1: cell c is the union of the tetrahedra (c_c, outward face triangle). */
static int cell_tets(const vo_mesh *m, int c, v3 (*K)[4], int cap)
{
    int i, k = 0;
    for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) {
        int f = m->cface[i], t;
        for (t = 0; t < ntri(m, f); t++) {
            v3 T[3];
            face_tri(m, f, t, T);
            if (k >= cap) return -1;
            K[k][0] = m->cc[c];
            K[k][1] = T[0];
            if (m->own[f] == c) { K[k][2] = T[1]; K[k][3] = T[2]; }
            else { K[k][2] = T[2]; K[k][3] = T[1]; }
            k++;
        }
    }
    return k;
}

/* outward face planes of a positively oriented tetrahedron: n.x <= d inside */
static void tet_planes(v3 *K, v3 *n, double *d)
{
    v3 a = K[0], b = K[1], c = K[2], e = K[3];
    if (tetvol(a, b, c, e) < 0) { v3 t = b; b = c; c = t; }
    n[0] = cross(sub(c, a), sub(b, a)); d[0] = dot(n[0], a);
    n[1] = cross(sub(b, a), sub(e, a)); d[1] = dot(n[1], a);
    n[2] = cross(sub(e, a), sub(c, a)); d[2] = dot(n[2], a);
    n[3] = cross(sub(c, b), sub(e, b)); d[3] = dot(n[3], b);
}

#define MAXK 256

double vo_cut_volume(const vo_mesh *m, int c, const double nn[3], double d)
{
    v3 K[MAXK][4], n = mk(nn[0], nn[1], nn[2]);
    int nk = cell_tets(m, c, K, MAXK), k;
    double V = 0.0;
    for (k = 0; k < nk; k++) V += tet_clip(K[k][0], K[k][1], K[k][2], K[k][3], 1, &n, &d, NULL);
    return V;
}

/* ------------------------------------ A2 + A3: reconstruction (Alg. 1) */
#define POS_TOL 1e-13
#define POS_MAXIT 100

#define POS_SECANT_MAX 20

static int position_cell(const vo_mesh *m, int c, double alpha, v3 n, double *dout)
{
    /* fill level g(d) = |C ^ {n.x <= d}|/V - alpha rises monotonically from -alpha
     * at d_min to 1-alpha at d_max (Sec. 2.2.2).  Alg. 1: secant steps through the
     * last two arguments until the secant diverges, then bisection.  Reading R3 of
     * "diverges": the new argument leaves the current bracket [a, b], or the
     * secant has taken POS_SECANT_MAX steps without meeting the tolerance (a
     * stall: deep in the cubic corner of the fill, near alpha = 0 or 1, each
     * secant step advances by about alpha times the cell extent, while a secant
     * that converges does so within a dozen steps). */
    double dmin = 1e300, dmax = -1e300, a, b, x0, g0, x1, g1, x = 0.0, gx = 0.0;
    double nn[3] = {n.x, n.y, n.z};
    int i, it = 0, bisect = 0;
    for (i = m->cpptr[c]; i < m->cpptr[c + 1]; i++) {
        double s = dot(n, m->P[m->cpt[i]]);
        if (s < dmin) dmin = s;
        if (s > dmax) dmax = s;
    }
    a = dmin; b = dmax;
    x0 = a; g0 = -alpha; x1 = b; g1 = 1.0 - alpha;
    while (it < POS_MAXIT) {
        if (!bisect && it >= POS_SECANT_MAX) bisect = 1;
        if (!bisect) {
            /* secant through the last two arguments */
            x = x1 - g1 * (x1 - x0) / (g1 - g0);
            if (!(x > a && x < b)) bisect = 1;
        }
        if (bisect) x = 0.5 * (a + b);
        gx = vo_cut_volume(m, c, nn, x) / m->vc[c] - alpha;
        it++;
        if (gx < 0) a = x; else b = x;
        x0 = x1; g0 = g1; x1 = x; g1 = gx;
        if (fabs(gx) <= POS_TOL) break;
        if (b - a <= 1e-15 * (dmax - dmin)) break;
    }
    *dout = x;
    return it;
}

int vo_position(const vo_mesh *m, int c, double alpha, const double nn[3], double *d)
{
    return position_cell(m, c, alpha, mk(nn[0], nn[1], nn[2]), d);
}

int vo_reconstruct(const vo_mesh *m, const double *alpha, double eps, int n_sel, const int *sel,
                   double *nout, double *dout, unsigned char *flags, int *iters)
{
    return vo_reconstruct_grad(m, alpha, NULL, eps, n_sel, sel, nout, dout, flags, iters);
}

/* as vo_reconstruct, the normal from a given gradient (3*nc SoA; NULL: NAG) */
int vo_reconstruct_grad(const vo_mesh *m, const double *alpha, const double *grad, double eps, int n_sel,
                        const int *sel, double *nout, double *dout, unsigned char *flags, int *iters)
{
    int k, nn = sel ? n_sel : m->nc, st = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : st)
    for (k = 0; k < nn; k++) {
        int c = sel ? sel[k] : k, it = 0;
        double a = alpha[c], d = 0.0;
        unsigned char fl = 0;
        v3 n = mk(0, 0, 0);
        if (a >= 1.0 - eps) fl = VO_FULL;
        else if (a > eps) {
            v3 g = grad ? mk(grad[c], grad[m->nc + c], grad[2 * m->nc + c]) : nag_gradient_cell(m, c, alpha);
            double gm = norm(g), hc = cbrt(m->vc[c]);
            fl = VO_INTERFACE;
            /* R4: a vanishing gradient leaves the cell unoriented */
            if (gm * hc > 1e-12) {
                n = scl(g, -1.0 / gm); /* R11: points out of the phase */
                fl |= VO_ORIENTED;
                it = position_cell(m, c, a, n, &d);
                if (it >= POS_MAXIT) st |= VO_ST_POS_NOT_CONVERGED;
            }
        }
        if (nout) { nout[c] = n.x; nout[m->nc + c] = n.y; nout[2 * m->nc + c] = n.z; }
        if (dout) dout[c] = d;
        if (flags) flags[c] = fl;
        if (iters) iters[c] = it;
    }
    return st;
}

/* ------------------------------ generalised LSQ gradient (Sec. 2.2.1) */
/* The cell's stencil: every other cell that shares a point with it. */
/* (On a periodic mesh, R21: each with the translation that brings it next to
 * the cell, coded as in the face stencils; the cell's own images other than
 * itself count as neighbours.) */
static int point_nbrs(const vo_mesh *m, int c, int *out, int *codes, int cap)
{
    int k = 0, i, j, u = 0;
    long long buf[4096];
    for (i = m->cpptr[c]; i < m->cpptr[c + 1]; i++) {
        int p = m->cpt[i];
        for (j = m->pptr[p]; j < m->pptr[p + 1]; j++)
            if ((m->pcell[j] != c || m->pcode[j] != T0) && k < 4096) buf[k++] = (long long)m->pcell[j] * 32 + m->pcode[j];
    }
    qsort(buf, (size_t)k, sizeof(long long), cmp_long);
    for (i = 0; i < k; i++)
        if (i == 0 || buf[i] != buf[i - 1]) {
            if (u < cap) { out[u] = (int)(buf[i] / 32); codes[u] = buf[i] % 32; }
            u++;
        }
    return u;
}

/* The gradient minimising E_c = sum_k w_ck^2 E_ck^2 (Eq. generalizedLSQminimize),
 * E_ck = -(phi_c - phi_k) + grad.(x_c - x_k), w_ck the inverse distance of the
 * two cell centres: the normal equations (sum w^2 d d^T) g = sum w^2 d (phi_k -
 * phi_c), d = x_k - x_c, solved by Cramer's rule (g = 0 for a singular system). */
static v3 lsq_gradient_cell(const vo_mesh *m, int c, const double *phi)
{
    int nb[1024], code[1024], k, nk = point_nbrs(m, c, nb, code, 1024);
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0}, det, x[3];
    int i, j, col;
    for (k = 0; k < nk && k < 1024; k++) {
        v3 d = sub(add(m->cc[nb[k]], tvec(m, code[k])), m->cc[c]);
        double dv[3] = {d.x, d.y, d.z}, w2 = 1.0 / dot(d, d), dphi = phi[nb[k]] - phi[c];
        for (i = 0; i < 3; i++) {
            b[i] += w2 * dv[i] * dphi;
            for (j = 0; j < 3; j++) A[i][j] += w2 * dv[i] * dv[j];
        }
    }
    det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
          A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (det == 0.0) return mk(0, 0, 0);
    for (col = 0; col < 3; col++) { /* replace column col by b */
        double M[3][3];
        for (i = 0; i < 3; i++)
            for (j = 0; j < 3; j++) M[i][j] = j == col ? b[i] : A[i][j];
        x[col] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                  M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
    }
    return mk(x[0], x[1], x[2]);
}

void vo_lsq_gradient(const vo_mesh *m, const double *phi, int n_sel, const int *sel, double *grad)
{
    int k, nn = sel ? n_sel : m->nc;
#pragma omp parallel for schedule(dynamic, 256)
    for (k = 0; k < nn; k++) {
        int c = sel ? sel[k] : k;
        v3 g = lsq_gradient_cell(m, c, phi);
        grad[c] = g.x; grad[m->nc + c] = g.y; grad[2 * m->nc + c] = g.z;
    }
}

/* ---------------------- reconstruction error E_vsd (Sec. 4.1, Eqs. E_vsd) */
/* The true phase is a ball B (centre bc, radius R), described the way the
 * paper's tool mesh describes a geometry: every cell tetrahedron is split
 * into eight (edge midpoints; the inner octahedron about the diagonal joining
 * the midpoints of edges ab and cd) down to `levels`, where a piece is taken
 * as wholly in B (all four vertices in the closed ball), wholly outside (its
 * centroid's distance to bc less its largest vertex distance to the centroid
 * is at least R), or, still undecided at the last level, cut by the plane
 * tangent to the sphere at the point nearest its centroid.  With P the true
 * phase in a piece S and H the cell's reconstructed phase (PLIC half-space of
 * an oriented interface cell, all of S for a full cell, none for any other),
 * the piece contributes |P \ H| + |(S ^ H) \ P| = |P| + |S ^ H| - 2 |P ^ H|:
 * E_vsd^- and E_vsd^+ of the paper summed.  With no H this is |P|, so the
 * same routine gives the ball's volume in the cell. */
static double d2(v3 a, v3 b) { v3 t = sub(a, b); return dot(t, t); }

static double tet_abs(v3 a, v3 b, v3 c, v3 d) { return fabs(tetvol(a, b, c, d)); }

static double evsd_piece(v3 a, v3 b, v3 c, v3 d, int level, int levels, v3 bc, double R, int hmode, v3 hn,
                         double hd)
{
    double R2 = R * R, S, SH, P, PH;
    v3 g = scl(add(add(a, b), add(c, d)), 0.25);
    double rt = sqrt(d2(a, g)), dist;
    int inside = d2(a, bc) <= R2 && d2(b, bc) <= R2 && d2(c, bc) <= R2 && d2(d, bc) <= R2;
    if (sqrt(d2(b, g)) > rt) rt = sqrt(d2(b, g));
    if (sqrt(d2(c, g)) > rt) rt = sqrt(d2(c, g));
    if (sqrt(d2(d, g)) > rt) rt = sqrt(d2(d, g));
    dist = sqrt(d2(g, bc));
    S = tet_abs(a, b, c, d);
    SH = hmode == 0 ? 0.0 : hmode == 1 ? S : tet_clip(a, b, c, d, 1, &hn, &hd, NULL);
    if (inside) return S + SH - 2.0 * SH;
    if (dist - rt >= R) return SH;
    if (level < levels) {
        v3 ab = scl(add(a, b), 0.5), ac = scl(add(a, c), 0.5), ad = scl(add(a, d), 0.5);
        v3 bcm = scl(add(b, c), 0.5), bd = scl(add(b, d), 0.5), cd = scl(add(c, d), 0.5);
        int l = level + 1;
        return evsd_piece(a, ab, ac, ad, l, levels, bc, R, hmode, hn, hd) +
               evsd_piece(b, ab, bcm, bd, l, levels, bc, R, hmode, hn, hd) +
               evsd_piece(c, ac, bcm, cd, l, levels, bc, R, hmode, hn, hd) +
               evsd_piece(d, ad, bd, cd, l, levels, bc, R, hmode, hn, hd) +
               evsd_piece(ab, cd, ac, ad, l, levels, bc, R, hmode, hn, hd) +
               evsd_piece(ab, cd, ad, bd, l, levels, bc, R, hmode, hn, hd) +
               evsd_piece(ab, cd, bd, bcm, l, levels, bc, R, hmode, hn, hd) +
               evsd_piece(ab, cd, bcm, ac, l, levels, bc, R, hmode, hn, hd);
    }
    {
        v3 pn[2], u = dist > 0.0 ? scl(sub(g, bc), 1.0 / dist) : mk(1, 0, 0);
        double pd[2];
        pn[0] = u; pd[0] = dot(u, bc) + R;
        P = tet_clip(a, b, c, d, 1, pn, pd, NULL);
        if (hmode == 0) PH = 0.0;
        else if (hmode == 1) PH = P;
        else { pn[1] = hn; pd[1] = hd; PH = tet_clip(a, b, c, d, 2, pn, pd, NULL); }
        return P + SH - 2.0 * PH;
    }
}

void vo_evsd(const vo_mesh *m, const unsigned char *flags, const double *n, const double *d,
             const double ball[4], int levels, int n_sel, const int *sel, double *out)
{
    int k, nn = sel ? n_sel : m->nc;
    v3 bc = mk(ball[0], ball[1], ball[2]);
#pragma omp parallel for schedule(dynamic, 16)
    for (k = 0; k < nn; k++) {
        int c = sel ? sel[k] : k, nk, t, hmode = 0;
        v3 K[MAXK][4], hn = mk(0, 0, 0);
        double hd = 0.0, e = 0.0;
        if (flags) {
            if (flags[c] & VO_FULL) hmode = 1;
            else if ((flags[c] & VO_INTERFACE) && (flags[c] & VO_ORIENTED)) {
                hmode = 2;
                hn = mk(n[c], n[m->nc + c], n[2 * m->nc + c]);
                hd = d[c];
            }
        }
        nk = cell_tets(m, c, K, MAXK);
        for (t = 0; t < nk; t++) e += evsd_piece(K[t][0], K[t][1], K[t][2], K[t][3], 0, levels, bc, ball[3], hmode, hn, hd);
        out[c] = e;
    }
}

/* ------------------------- geometric mapping for AMR (Sec. 3, Alg. 2) */
/* The volume fraction of each destination cell from the interface planes of
 * the source cells its cell map lists (pairs, CSR over destination cells).
 * The cells of a pair are nested: the destination cell is the source cell,
 * lies inside it (refined), or contains it (un-refined).  Its phase volume is
 * the sum over its pairs of |PLIC polyhedron of the source ^ destination|:
 *  - same cell: alpha_s V;
 *  - destination inside an oriented interface source: the destination
 *    cell's tetrahedra clipped by the source's plane n_s.x <= d_s;
 *  - destination inside any other source (empty, full, unoriented): the
 *    source's phase spread evenly, alpha_s V_dst (so no volume is lost to the
 *    eps thresholds);
 *  - source inside the destination: the source's whole phase, alpha_s V_s.
 * Cells count as the same where their volumes agree to 1e-9. */
int vo_remap(const vo_mesh *dst, const vo_mesh *src, const double *alpha_src, const double *n_src,
             const double *d_src, const unsigned char *flags_src, const int *pair_ptr, const int *pair_src,
             double *alpha_dst)
{
    int c;
#pragma omp parallel for schedule(dynamic, 64)
    for (c = 0; c < dst->nc; c++) {
        double Vc = dst->vc[c], acc = 0.0;
        int q;
        for (q = pair_ptr[c]; q < pair_ptr[c + 1]; q++) {
            int s = pair_src[q];
            double Vs = src->vc[s], as = alpha_src[s];
            if (fabs(Vc - Vs) <= 1e-9 * Vs) acc += as * Vc;
            else if (Vc < Vs) {
                if ((flags_src[s] & VO_INTERFACE) && (flags_src[s] & VO_ORIENTED)) {
                    v3 K[MAXK][4], n = mk(n_src[s], n_src[src->nc + s], n_src[2 * src->nc + s]);
                    double dd = d_src[s];
                    int nk = cell_tets(dst, c, K, MAXK), k;
                    for (k = 0; k < nk; k++) acc += tet_clip(K[k][0], K[k][1], K[k][2], K[k][3], 1, &n, &dd, NULL);
                } else acc += as * Vc;
            } else acc += as * Vs;
        }
        alpha_dst[c] = acc / Vc;
    }
    return 0;
}

/* ------------------------------------------- A4: point velocity + sweep */
void vo_point_velocity(const vo_mesh *m, const double *Uc, double *Up)
{
    int p;
#pragma omp parallel for schedule(static)
    for (p = 0; p < m->np; p++) {
        v3 u = mk(point_value(m, p, Uc), point_value(m, p, Uc + m->nc),
                  point_value(m, p, Uc + 2 * m->nc));
        if (m->pwn[p] == 1) {
            v3 n = m->pwv[2 * p];
            u = sub(u, scl(n, dot(u, n)));
        } else if (m->pwn[p] == 2) {
            v3 t = cross(m->pwv[2 * p], m->pwv[2 * p + 1]);
            t = scl(t, 1.0 / norm(t));
            u = scl(t, dot(u, t));
        } else if (m->pwn[p] >= 3) {
            u = mk(0, 0, 0);
        }
        Up[p] = u.x; Up[m->np + p] = u.y; Up[2 * m->np + p] = u.z;
    }
}

/* ----------------------------------------------- A5: flux polyhedra */
/* Tetrahedral decomposition of the flux polyhedron (reading R5): every face
 * triangle (a0,a1,a2) is swept to (b0,b1,b2), b = a - w (Eq. sweep).  With a
 * sweep factor lambda >= 0 the displacement is w = lambda*U_p*dt, the swept face
 * centre moving with the mean of the point displacements.  lambda < 0 marks the
 * normal-sweep fallback: every point moves by w = -lambda*(F_f/|S_f|^2) S_f dt,
 * a uniform translation whose swept volume is exactly -lambda*F_f*dt.
 * The triangular prism is split into three tetrahedra after ordering its
 * vertices by key (face centre first, then global point index; its master on
 * a periodic mesh, R21), so that a side
 * quad shared by two prisms is split along the same diagonal in both.  Each
 * tetrahedron carries the sign that makes the sum the signed swept volume,
 * positive for a sweep against S_f (flux from owner to neighbour). */
typedef struct { v3 v[4]; double s; } stet;

static v3 point_disp(const vo_mesh *m, int p, const double *Up, double dt, double lambda, v3 wn)
{
    if (lambda < 0) return wn;
    return scl(mk(Up[p], Up[m->np + p], Up[2 * m->np + p]), dt * lambda);
}

static int face_prism_tets(const vo_mesh *m, int f, const double *Up, double F, double dt,
                           double lambda, stet *out)
{
    int n = fn(m, f), t, q = 0, i;
    v3 wc = mk(0, 0, 0), wn = mk(0, 0, 0);
    const int *p = m->fpts + m->fptr[f];
    if (lambda < 0) wn = scl(m->sf[f], -lambda * F * dt / dot(m->sf[f], m->sf[f]));
    for (i = 0; i < n; i++) wc = add(wc, point_disp(m, p[i], Up, dt, lambda, wn));
    wc = scl(wc, 1.0 / n);
    for (t = 0; t < ntri(m, f); t++) {
        v3 a[3], w[3], b[3];
        long key[3];
        int id[3] = {0, 1, 2}, parity = 1, j, k;
        if (n == 3) {
            for (j = 0; j < 3; j++) {
                a[j] = m->P[p[j]];
                w[j] = point_disp(m, p[j], Up, dt, lambda, wn);
                key[j] = m->pmaster[p[j]];
            }
        } else {
            int j0 = p[t], j1 = p[(t + 1) % n];
            a[0] = m->cf[f]; w[0] = wc; key[0] = -1;
            a[1] = m->P[j0]; w[1] = point_disp(m, j0, Up, dt, lambda, wn); key[1] = m->pmaster[j0];
            a[2] = m->P[j1]; w[2] = point_disp(m, j1, Up, dt, lambda, wn); key[2] = m->pmaster[j1];
        }
        for (j = 0; j < 3; j++) b[j] = sub(a[j], w[j]);
        for (j = 1; j < 3; j++) /* sort vertex ids by key, tracking permutation parity */
            for (k = j; k > 0 && key[id[k]] < key[id[k - 1]]; k--) {
                int tmp = id[k]; id[k] = id[k - 1]; id[k - 1] = tmp; parity = -parity;
            }
        {
            v3 A0 = a[id[0]], A1 = a[id[1]], A2 = a[id[2]];
            v3 B0 = b[id[0]], B1 = b[id[1]], B2 = b[id[2]];
            stet *o = out + q;
            o[0].v[0] = A0; o[0].v[1] = A1; o[0].v[2] = A2; o[0].v[3] = B2;
            o[1].v[0] = A0; o[1].v[1] = A1; o[1].v[2] = B2; o[1].v[3] = B1;
            o[2].v[0] = A0; o[2].v[1] = B0; o[2].v[2] = B1; o[2].v[3] = B2;
            for (j = 0; j < 3; j++) o[j].s = -parity * tetvol(o[j].v[0], o[j].v[1], o[j].v[2], o[j].v[3]);
            q += 3;
        }
    }
    return q;
}

double vo_swept_volume(const vo_mesh *m, int f, const double *Up, double F, double dt, double lambda)
{
    stet T[3 * 64];
    int q = face_prism_tets(m, f, Up, F, dt, lambda, T), i;
    double V = 0.0;
    for (i = 0; i < q; i++) V += T[i].s; /* Eq. V_fS */
    return V;
}

static double swept_abs(const vo_mesh *m, int f, const double *Up, double dt, double lambda)
{
    stet T[3 * 64];
    int q = face_prism_tets(m, f, Up, 0.0, dt, lambda, T), i;
    double V = 0.0;
    for (i = 0; i < q; i++) V += fabs(T[i].s);
    return V;
}

#define CORR_TOL 1e-14
#define CORR_MAXIT 100
#define CORR_LMAX 2.0
#define CORR_NSAMP 16

/* Reading R5: the swept end points move along their stream vectors by a common
 * factor lambda, and the secant method drives r(lambda) = V_f(lambda) - F_f dt
 * to zero (Eq. VF, Sec. 2.3).  A flux below 1e-12 of |S_f| max_p |U_p| dt is
 * rounding noise of the field (a wall face, for instance): lambda = 0, no sweep.  The root taken is the one in the first of the
 * intervals [k, k+1]*LMAX/NSAMP (k = 0..NSAMP-1) at whose ends r changes sign;
 * inside it the secant starts from the interval ends, and an iterate that
 * leaves the current bracket is replaced by bisection (the safeguard of
 * Alg. 1).  When no interval brackets a root (point velocities nearly
 * tangential to the face disagree with F_f) the face takes the normal-sweep
 * fallback, returned as lambda = -1.  Returns the secant iterations. */
static int correct_face(const vo_mesh *m, int f, const double *Up, double F, double dt, double *lam)
{
    double tau = F * dt, lo = 0.0, hi = 0.0, rlo = -tau, rhi = 0.0, x0, r0, x1, r1, x, r, scale;
    int it = 0, k, bisect = 0, found = 0;
    double umax = 0.0;
    if (tau == 0.0) { *lam = 0.0; return 0; }
    for (k = m->fptr[f]; k < m->fptr[f + 1]; k++) {
        int p = m->fpts[k];
        double u = norm(mk(Up[p], Up[m->np + p], Up[2 * m->np + p]));
        if (u > umax) umax = u;
    }
    if (fabs(tau) <= 1e-12 * norm(m->sf[f]) * umax * dt) { *lam = 0.0; return 0; }
    for (k = 1; k <= CORR_NSAMP; k++) {
        double lk = k * (CORR_LMAX / CORR_NSAMP);
        double rk = vo_swept_volume(m, f, Up, F, dt, lk) - tau;
        if (rk == 0.0) { *lam = lk; return 0; }
        if ((rk > 0) != (rlo > 0)) { hi = lk; rhi = rk; found = 1; break; }
        lo = lk; rlo = rk;
    }
    if (!found) { *lam = -1.0; return 0; }
    x0 = lo; r0 = rlo; x1 = hi; r1 = rhi; x = hi;
    while (it < CORR_MAXIT) {
        if (!bisect) {
            x = x1 - r1 * (x1 - x0) / (r1 - r0);
            if (!(x > lo && x < hi)) bisect = 1;
        }
        if (bisect) x = 0.5 * (lo + hi);
        r = vo_swept_volume(m, f, Up, F, dt, x) - tau;
        scale = swept_abs(m, f, Up, dt, x);
        if (fabs(tau) > scale) scale = fabs(tau);
        it++;
        if ((r > 0) == (rhi > 0)) { hi = x; rhi = r; } else { lo = x; rlo = r; }
        x0 = x1; r0 = r1; x1 = x; r1 = r;
        if (fabs(r) <= CORR_TOL * scale) break;
        if (hi - lo <= 1e-15 * hi) break;
    }
    *lam = x;
    return it;
}

int vo_correct_flux(const vo_mesh *m, const double *Up, const double *F, double dt, int n_sel,
                    const int *sel, double *lambda, int *iters)
{
    int k, nn = sel ? n_sel : m->nf, st = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : st)
    for (k = 0; k < nn; k++) {
        int f = sel ? sel[k] : k;
        double l = 0.0;
        int it = correct_face(m, f, Up, F[f], dt, &l);
        if (it >= CORR_MAXIT) st |= VO_ST_CORR_NOT_CONVERGED;
        lambda[f] = l;
        if (iters) iters[f] = it;
    }
    return st;
}

/* ---------------------------------------------------- A6: phase flux */
static void aabb_tet(v3 *v, v3 *lo, v3 *hi)
{
    int i;
    *lo = v[0]; *hi = v[0];
    for (i = 1; i < 4; i++) {
        if (v[i].x < lo->x) lo->x = v[i].x;
        if (v[i].y < lo->y) lo->y = v[i].y;
        if (v[i].z < lo->z) lo->z = v[i].z;
        if (v[i].x > hi->x) hi->x = v[i].x;
        if (v[i].y > hi->y) hi->y = v[i].y;
        if (v[i].z > hi->z) hi->z = v[i].z;
    }
}
static int disjoint(v3 alo, v3 ahi, v3 blo, v3 bhi)
{
    return ahi.x < blo.x || bhi.x < alo.x || ahi.y < blo.y || bhi.y < alo.y || ahi.z < blo.z || bhi.z < alo.z;
}

/* R9: a face is trivial when every stencil cell is empty (alpha <= eps) or
 * every stencil cell is full (alpha >= 1-eps). */
void vo_classify_faces(const vo_mesh *m, const double *alpha, double eps, unsigned char *cls)
{
    int f;
#pragma omp parallel for schedule(dynamic, 1024)
    for (f = 0; f < m->nf; f++) {
        int all_e = 1, all_f = 1, i, j;
        if (f >= m->ni && m->fimg[f - m->ni] >= 0) { cls[f] = 0; continue; } /* R21: a copy carries no flux */
        for (i = m->fptr[f]; i < m->fptr[f + 1]; i++) {
            int p = m->fpts[i];
            for (j = m->pptr[p]; j < m->pptr[p + 1]; j++) {
                double a = alpha[m->pcell[j]];
                if (!(a <= eps)) all_e = 0;
                if (!(a >= 1.0 - eps)) all_f = 0;
            }
        }
        cls[f] = all_e ? 0 : (all_f ? 1 : 2);
    }
}

/* sum over the stencil of the signed |T ^ K ^ H| pieces (Eqs. S'_f, S''_f) */
static double face_phase_volume(const vo_mesh *m, int f, const double *alpha, double eps,
                                const double *nrm, const double *dd, const unsigned char *flags,
                                const double *Up, double F, double dt, double lambda, int coverage,
                                int *st)
{
    stet T[3 * 64];
    int sten[1024], code[1024];
    v3 K[MAXK][4];
    int q = face_prism_tets(m, f, Up, F, dt, lambda, T);
    int ns = vo_stencil_codes(m, f, sten, code, 1024), t, s, k;
    double acc = 0.0;
    for (t = 0; t < q; t++) {
        v3 tlo, thi;
        double sg;
        if (T[t].s == 0.0) continue;
        sg = T[t].s > 0 ? 1.0 : -1.0;
        aabb_tet(T[t].v, &tlo, &thi);
        for (s = 0; s < ns; s++) {
            int c = sten[s], nk, j;
            double a = coverage ? 1.0 : alpha[c], wgt = 1.0;
            int use_h = 0;
            v3 hn = mk(0, 0, 0), tr = tvec(m, code[s]);
            double hd = 0.0;
            if (!coverage) {
                if (a <= eps) continue; /* empty cell carries no phase */
                if (flags[c] & VO_INTERFACE) {
                    if (flags[c] & VO_ORIENTED) {
                        use_h = 1;
                        hn = mk(nrm[c], nrm[m->nc + c], nrm[2 * m->nc + c]);
                        hd = dd[c] + dot(hn, tr); /* the plane moves with the cell (R21) */
                    } else wgt = a; /* R4: unoriented mixed cell is homogeneous */
                }
            }
            nk = cell_tets(m, c, K, MAXK);
            if (code[s] != T0)
                for (k = 0; k < nk; k++)
                    for (j = 0; j < 4; j++) K[k][j] = add(K[k][j], tr);
            for (k = 0; k < nk; k++) {
                v3 klo, khi, pn[5];
                double pd[5], v;
                aabb_tet(K[k], &klo, &khi);
                if (disjoint(tlo, thi, klo, khi)) continue;
                tet_planes(K[k], pn, pd);
                if (use_h) { pn[4] = hn; pd[4] = hd; }
                v = tet_clip(T[t].v[0], T[t].v[1], T[t].v[2], T[t].v[3], use_h ? 5 : 4, pn, pd, st);
                acc += sg * wgt * v;
            }
        }
    }
    return acc;
}

double vo_stencil_coverage(const vo_mesh *m, int f, const double *Up, double F, double dt,
                           double lambda)
{
    int st = 0;
    return face_phase_volume(m, f, NULL, 0.0, NULL, NULL, NULL, Up, F, dt, lambda, 1, &st);
}

static double phase_flux_face(const vo_mesh *m, int f, const unsigned char *cls, const double *alpha,
                              double eps, const double *n, const double *d,
                              const unsigned char *flags, const double *Up, const double *F,
                              const double *lambda, double dt, int *st)
{
    if (F[f] == 0.0) return 0.0;
    /* R2: a boundary face with inflow brings in the empty exterior */
    if (f >= m->ni && F[f] < 0.0) return 0.0;
    if (cls[f] == 0) return 0.0;
    if (cls[f] == 1) return F[f] * dt; /* Eq. vol-phase-flux with alpha_f = 1 */
    return face_phase_volume(m, f, alpha, eps, n, d, flags, Up, F[f], dt, lambda[f], 0, st);
}

int vo_phase_flux(const vo_mesh *m, const double *alpha, double eps, const double *n,
                  const double *d, const unsigned char *flags, const double *Up, const double *F,
                  const double *lambda, double dt, int n_sel, const int *sel, double *Valpha)
{
    int k, nn = sel ? n_sel : m->nf, st = 0;
    unsigned char *cls = (unsigned char *)malloc((size_t)m->nf);
    vo_classify_faces(m, alpha, eps, cls);
#pragma omp parallel for schedule(dynamic, 16) reduction(| : st)
    for (k = 0; k < nn; k++) {
        int f = sel ? sel[k] : k, s1 = 0;
        Valpha[f] = phase_flux_face(m, f, cls, alpha, eps, n, d, flags, Up, F, lambda, dt, &s1);
        st |= s1;
    }
    free(cls);
    return st;
}

/* ---------------------------------------------------------- A7: update */
#define BOUND_PASSES_MAX 32
#define BOUND_TOL 1e-13   /* excursions this small (round-off) are left alone and never
                           * decide a redistribution; the target is 1e-12 */
#define BOUND_FLAG 1e-12  /* a violation above this after the passes is flagged */

/* Reading R10 of the wisp redistribution of Sec. 2.3: over- and undershoots
 * are redistributed conservatively to the surrounding interface cells, and
 * neither the removal nor the addition may create new over/undershoots or
 * wisps.  Read as passes of a local redistribution among face neighbours:
 *  - a source is a cell with alpha > 1 + BOUND_TOL (excess e = (alpha-1) V) or
 *    alpha < -BOUND_TOL (deficit u = -alpha V);
 *  - a receiver is an interface cell, BOUND_TOL < alpha < 1 - BOUND_TOL; its
 *    weight w = alpha (1 - alpha) V vanishes at both ends, so that no bulk cell
 *    receives (no wisp is made) and the amounts vary continuously with alpha;
 *  - a source asks each face neighbour r for e w_r / W, W the sum of its
 *    neighbours' weights; a receiver takes at most its room, (1 - alpha) V for
 *    excess and alpha V for deficit, and scales all requests down to fit, so
 *    it never leaves [0, 1] (no new over/undershoot);
 *  - what a source could not place stays with it for the next pass.
 * Each pass either finishes a source or fills (empties) at least one of its
 * receivers, whose weight is then zero; passes run until no source has both
 * something left and a receiver with room (BOUND_PASSES_MAX is a safety cap).
 * Every cell's new value is a gather over its face neighbours, so the result
 * does not depend on visiting order. */
static int face_nbr(const vo_mesh *m, int c, int i)
{
    int f = m->cface[i];
    if (f >= m->ni) return m->fimg[f - m->ni] >= 0 ? m->own[m->fimg[f - m->ni]] : -1; /* R21 copy */
    return m->own[f] == c ? m->nei[f] : m->own[f];
}

static double recv_w(double a, double V) { return (a > BOUND_TOL && a < 1.0 - BOUND_TOL) ? a * (1.0 - a) * V : 0.0; }
static double room_exc(double a, double V) { return recv_w(a, V) > 0.0 ? (1.0 - a) * V : 0.0; }
static double room_def(double a, double V) { return recv_w(a, V) > 0.0 ? a * V : 0.0; }

/* one pass; returns the number of sources that had a receiver */
static int bound_pass(const vo_mesh *m, double *alpha)
{
    int nc = m->nc, c, active = 0;
    size_t n1 = (size_t)(nc > 0 ? nc : 1);
    double *e = (double *)calloc(n1, sizeof(double)), *u = (double *)calloc(n1, sizeof(double));
    double *W = (double *)calloc(n1, sizeof(double));
    double *sp = (double *)malloc(n1 * sizeof(double)), *sm = (double *)malloc(n1 * sizeof(double));
    double *na = (double *)malloc(n1 * sizeof(double));
    for (c = 0; c < nc; c++) {
        double a = alpha[c];
        if (a > 1.0 + BOUND_TOL) e[c] = (a - 1.0) * m->vc[c];
        if (a < -BOUND_TOL) u[c] = -a * m->vc[c];
    }
    /* (1) total receiver weight around each source */
    for (c = 0; c < nc; c++) {
        int i;
        if (e[c] == 0.0 && u[c] == 0.0) continue;
        for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) {
            int nb = face_nbr(m, c, i);
            if (nb >= 0) W[c] += recv_w(alpha[nb], m->vc[nb]);
        }
        if (W[c] > 0.0) active++;
    }
    if (active) {
        /* (2) scale of each receiver: requests beyond its room are cut to fit */
#pragma omp parallel for schedule(static)
        for (c = 0; c < nc; c++) {
            int i;
            double Qp = 0.0, Qm = 0.0, wc = recv_w(alpha[c], m->vc[c]);
            double Rp = room_exc(alpha[c], m->vc[c]), Rm = room_def(alpha[c], m->vc[c]);
            for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) {
                int nb = face_nbr(m, c, i);
                if (nb < 0 || W[nb] == 0.0) continue;
                if (e[nb] > 0.0) Qp += e[nb] * (wc / W[nb]);
                if (u[nb] > 0.0) Qm += u[nb] * (wc / W[nb]);
            }
            sp[c] = Qp > Rp ? Rp / Qp : 1.0;
            sm[c] = Qm > Rm ? Rm / Qm : 1.0;
        }
        /* (3) new value of every cell: what it placed (a source), what its
         * source neighbours placed in it (a receiver) */
#pragma omp parallel for schedule(static)
        for (c = 0; c < nc; c++) {
            int i;
            double dV = 0.0, V = m->vc[c], wc = recv_w(alpha[c], V);
            for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) {
                int nb = face_nbr(m, c, i);
                if (nb < 0) continue;
                if (W[c] > 0.0) { /* c is a source: what it placed in nb */
                    double wn = recv_w(alpha[nb], m->vc[nb]);
                    if (e[c] > 0.0) dV -= e[c] * (wn / W[c]) * sp[nb];
                    if (u[c] > 0.0) dV += u[c] * (wn / W[c]) * sm[nb];
                }
                if (W[nb] > 0.0) { /* nb is a source: what it placed in c */
                    if (e[nb] > 0.0) dV += e[nb] * (wc / W[nb]) * sp[c];
                    if (u[nb] > 0.0) dV -= u[nb] * (wc / W[nb]) * sm[c];
                }
            }
            na[c] = dV != 0.0 ? (alpha[c] * V + dV) / V : alpha[c];
        }
        memcpy(alpha, na, sizeof(double) * (size_t)nc);
    }
    free(e); free(u); free(W); free(sp); free(sm); free(na);
    return active;
}

/* Fallback for what the local passes leave (a source none of whose face
 * neighbours is an interface cell with room): the total excess (deficit) goes
 * to every cell strictly inside (BOUND_TOL, 1-BOUND_TOL) in proportion to its
 * free (phase) volume, and the sources are set to 1 (0).  Skipped when the
 * receivers cannot hold it.  Returns the volume moved (0 if none). */
static double bound_global(const vo_mesh *m, double *alpha)
{
    double Ep = 0.0, Em = 0.0, Sp = 0.0, Sm = 0.0;
    int c;
    for (c = 0; c < m->nc; c++) {
        double a = alpha[c], V = m->vc[c];
        if (a > 1.0 + BOUND_TOL) Ep += (a - 1.0) * V;
        else if (a < -BOUND_TOL) Em += -a * V;
        else if (a > BOUND_TOL && a < 1.0 - BOUND_TOL) { Sp += (1.0 - a) * V; Sm += a * V; }
    }
    if ((Ep == 0.0 && Em == 0.0) || Ep > Sp || Em > Sm) return 0.0;
    for (c = 0; c < m->nc; c++) {
        double a = alpha[c], V = m->vc[c];
        if (a > 1.0 + BOUND_TOL) alpha[c] = 1.0;
        else if (a < -BOUND_TOL) alpha[c] = 0.0;
        else if (a > BOUND_TOL && a < 1.0 - BOUND_TOL) {
            double dV = 0.0;
            if (Ep > 0.0) dV += Ep * ((1.0 - a) * V / Sp);
            if (Em > 0.0) dV -= Em * (a * V / Sm);
            alpha[c] = (a * V + dV) / V;
        }
    }
    return Ep + Em;
}

/* The Courant number of a step (Sec. 4.2 sets the time step from it): the
 * largest (1/2) sum over a cell's faces |F_f| dt / V_c; a cell takes a
 * periodic face through its copy (R21). */
double vo_courant(const vo_mesh *m, const double *F, double dt)
{
    double co = 0.0;
    int c, i;
    for (c = 0; c < m->nc; c++) {
        double s = 0.0;
        for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) {
            int g = m->cface[i];
            if (g >= m->ni && m->fimg[g - m->ni] >= 0) g = m->fimg[g - m->ni];
            s += fabs(F[g]);
        }
        s = 0.5 * s * dt / m->vc[c];
        if (s > co) co = s;
    }
    return co;
}

int vo_update(const vo_mesh *m, double *alpha, const double *Va, int bound, double *stats)
{
    int c, st = 0, f;
    double mb = 0.0, ma = 0.0, mn = 1e300, mx = -1e300, bo = 0.0;
    for (c = 0; c < m->nc; c++) mb += m->vc[c] * alpha[c];
#pragma omp parallel for schedule(static)
    for (c = 0; c < m->nc; c++) {
        double s = 0.0;
        int i;
        for (i = m->cptr[c]; i < m->cptr[c + 1]; i++) {
            int g = m->cface[i];
            if (g >= m->ni && m->fimg[g - m->ni] >= 0) s -= Va[m->fimg[g - m->ni]]; /* R21: c is its neighbour */
            else if (m->own[g] == c) s += Va[g];
            else s -= Va[g];
        }
        alpha[c] = alpha[c] - s / m->vc[c];
    }
    for (c = 0; c < m->nc; c++) {
        if (alpha[c] < mn) mn = alpha[c];
        if (alpha[c] > mx) mx = alpha[c];
    }
    if (stats) { stats[VO_S_MIN_PRE] = mn; stats[VO_S_MAX_PRE] = mx; }
    if (bound) {
        int p;
        double gv;
        for (p = 0; p < BOUND_PASSES_MAX; p++)
            if (!bound_pass(m, alpha)) break;
        gv = bound_global(m, alpha);
        if (stats) { stats[VO_S_BOUND_PASSES] = p; stats[VO_S_BOUND_GLOBAL] = gv; }
        if (p == BOUND_PASSES_MAX) st |= VO_ST_BOUND_RESIDUAL;
        for (c = 0; c < m->nc; c++)
            if (alpha[c] < -BOUND_FLAG || alpha[c] > 1.0 + BOUND_FLAG) { st |= VO_ST_BOUND_RESIDUAL; break; }
    }
    mn = 1e300; mx = -1e300;
    for (c = 0; c < m->nc; c++) {
        ma += m->vc[c] * alpha[c];
        if (alpha[c] < mn) mn = alpha[c];
        if (alpha[c] > mx) mx = alpha[c];
    }
    for (f = m->ni; f < m->nf; f++) bo += Va[f];
    if (stats) {
        stats[VO_S_MASS_BEFORE] = mb; stats[VO_S_MASS_AFTER] = ma;
        stats[VO_S_MIN_POST] = mn; stats[VO_S_MAX_POST] = mx; stats[VO_S_BOUNDARY_OUT] = bo;
    }
    return st;
}

int vo_advect(const vo_mesh *m, double *alpha, const double *Uc, const double *F, double dt,
              double eps, int bound, double *stats)
{
    int nc = m->nc, nf = m->nf, st = 0, f, c, nb = 0, ni = 0, *band, *it, maxit = 0;
    unsigned char *cls = (unsigned char *)malloc((size_t)nf), *flags = (unsigned char *)malloc((size_t)nc);
    double *n = (double *)calloc(3 * (size_t)nc, sizeof(double)), *d = (double *)calloc((size_t)nc, sizeof(double));
    double *Up = (double *)malloc(sizeof(double) * 3 * (size_t)m->np);
    double *lam = (double *)calloc((size_t)nf, sizeof(double)), *Va = (double *)calloc((size_t)nf, sizeof(double));
    int *pit = (int *)calloc((size_t)nc, sizeof(int));
    band = (int *)malloc(sizeof(int) * (size_t)(nf > 0 ? nf : 1));
    it = (int *)calloc((size_t)(nf > 0 ? nf : 1), sizeof(int));
    vo_classify_faces(m, alpha, eps, cls);
    for (f = 0; f < nf; f++)
        if (cls[f] == 2 && F[f] != 0.0 && !(f >= m->ni && F[f] < 0.0)) band[nb++] = f;
    st |= vo_reconstruct(m, alpha, eps, 0, NULL, n, d, flags, pit);
    vo_point_velocity(m, Uc, Up);
    st |= vo_correct_flux(m, Up, F, dt, nb, band, lam, it);
    st |= vo_phase_flux(m, alpha, eps, n, d, flags, Up, F, lam, dt, 0, NULL, Va);
    st |= vo_update(m, alpha, Va, bound, stats);
    if (stats) {
        int mp = 0;
        for (c = 0; c < nc; c++) {
            if (flags[c] & VO_INTERFACE) ni++;
            if (pit[c] > mp) mp = pit[c];
        }
        for (f = 0; f < nb; f++) if (it[band[f]] > maxit) maxit = it[band[f]];
        stats[VO_S_N_INTERFACE] = ni;
        stats[VO_S_N_BAND] = nb;
        stats[VO_S_MAX_POS_IT] = mp;
        stats[VO_S_MAX_CORR_IT] = maxit;
        stats[VO_S_STATUS] = st;
    }
    free(cls); free(flags); free(n); free(d); free(Up); free(lam); free(Va); free(pit); free(band); free(it);
    return st;
}

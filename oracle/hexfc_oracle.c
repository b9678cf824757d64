/*
 * hexfc_oracle.c -- plain, slow CPU oracle for the focus+context hex-mesh
 * renderer of "Interactive Focus+Context Rendering for Hexahedral Mesh
 * Inspection" (Neuhauser, Wang, Westermann).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code,
 * header, table or helper with the CUDA library; both are written from the
 * paper and from the readings listed below.
 *
 * What it computes (brute force, in the paper's order):
 *   1. unique faces of the mesh, each rendered as two triangles (Section
 *      "Method Overview"; Section "GPU Implementation": two triangles per face),
 *      per-vertex and per-edge importance = max over incident cells;
 *   2. for every requested pixel, every triangle of every face is tested for
 *      coverage of the pixel centre with exact integer edge functions on
 *      16.8 fixed-point window coordinates (top-left tie rule);
 *   3. every covered sample becomes a fragment, shaded in double precision
 *      with Eq. 1 (edge classification), Eq. 2 (accentuation), Eq. 3 (face
 *      opacity) and Eq. 4 (per-fragment blend), focus from the lens
 *      (Section "Focus+Context");
 *   4. each pixel's list is sorted by (depth, face, triangle) ascending with
 *      an insertion sort and blended front to back over the background
 *      (Section "Method Overview": sorted by increasing distance, alpha
 *      blending in visibility order).
 *
 * Readings of passages the paper leaves open (all shared with the CUDA path
 * by specification only):
 *   R1 pixel centre (x+.5, y+.5), row 0 at the top; vertices rounded to 1/256
 *      px with rint; a pixel is covered iff all three edge functions are > 0,
 *      or == 0 on a top-left edge after normalising each triangle to positive
 *      area; zero-area triangles and triangles with a vertex outside
 *      (znear, zfar) or the +-16384 px guard band produce nothing.
 *   R2 faces are the unique geometric faces; corner 0 is the smallest vertex
 *      id, corner 1 the smaller of its two neighbours; triangle 0 = (c0,c1,c2),
 *      triangle 1 = (c0,c2,c3); face id = rank of the sorted 4-id tuple.
 *   R3 the camera basis, projection and snapping are evaluated in double in
 *      one fixed order with no fused multiply-add.
 *   R4 window depth is quantised per vertex to 24 bits and interpolated per
 *      sample with exact integer arithmetic; key = z24 << 32 | (2 face + tri).
 *   R5 every covered sample is stored, including fully transparent ones.
 *   R6 lens distance: SCREEN |p - c| / r in pixels, SPHERE |P - c| / r with
 *      P the perspective-correct world position; focus = 1 - smoothstep(0.7,
 *      1, dist).
 *   R7 Eq. 3 is used as printed, with dist clamped to 1.
 *   R8 edge distances are pixel-space distances to the four projected edge
 *      segments of the face; d_f over edges visible in focus (level >= lod or
 *      attr >= delta), d_c over edges visible in context (level >= lod), d_a
 *      over all four; Eq. 1 as e_focus = d_f <= w, e_context = d_c <= w;
 *      Eq. 2 with d_a.
 *   R9 depth-dependent width w = (1 + 0.3 focus) w_base g with g = clamp(
 *      z_ref / z_eye, g_min, g_max), z_ref = |target - eye| (g = 1 for
 *      orthographic views); white halo band w < d_f <= w + h, h = halo_scale
 *      w_base focus g, with alpha_e = focus; focus edges darkened by
 *      (1 - darken focus).
 *   R10 colour table t -> (t, 0, 1 - t) (blue to red), face opacity
 *      alpha_min + (alpha_max - alpha_min) t, t from the perspective-correct
 *      vertex importance mapped through [tf_lo, tf_hi]; an accentuated
 *      fragment (s_e > 1) brightens its face colour by accent_beta.
 *   R11 s_e alpha_f is clamped to 1 in Eq. 4; colours are premultiplied.
 *   R12 output = C + (1 - A) bg, alpha = A.
 *   R16 depth cue (Section "Evaluation": fragments in the focus region that
 *      lie further from the camera are slightly desaturated): with strength
 *      desat (0 = off, the default), k = desat focus clamp(1 - g, 0, 1) and
 *      the Eq. 4 colour moves towards its luma y = 0.299 R + 0.587 G +
 *      0.114 B by k; opacity unchanged.
 *
 *   R17 silhouettes (Section "Blending Focus and Context": white exterior and
 *      interior screen-space silhouettes; the boundary surface is rendered and
 *      fragments along sharp edges of its depth buffer are emphasised): D(p)
 *      = 24-bit depth of the nearest fragment of a boundary face (a face of
 *      one cell) at pixel p. p is a silhouette pixel iff D(p) exists and a
 *      4-neighbour inside the frame has none (exterior), or for a neighbour q
 *      and the opposite neighbour q' (both with D), D(q) - D(p) > T and
 *      |D(q) - 2 D(p) + D(q')| > T (interior: the near side of a jump in
 *      depth; a plane, however steep, has no second difference), T =
 *      sil_threshold. A silhouette pixel's image moves towards white by
 *      sil_alpha: RGB' = RGB + a (1 - RGB), A' = A + a (1 - A).
 *
 * Near-tie bookkeeping: a discrete decision of R8/R9 whose two sides differ by
 * less than ORC_TIE_MARGIN pixels is reported in a per-fragment bit mask, and
 * orc_shade() can evaluate a fragment with any of those decisions flipped, so
 * that a test can accept either outcome for such a fragment and nothing else.
 *
 * Build: cc -O2 -std=c11 -fPIC -shared -ffp-contract=off -fopenmp
 *        hexfc_oracle.c -lm  (no fused multiply-add anywhere).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TIE_MARGIN 2e-4
#define ORC_GUARD_PX 16384.0
#define ORC_Z24_MAX 16777215.0

/* ----------------------------------------------------------------- inputs */

typedef struct {
    double eye[3], target[3], up[3];
    double fovy_deg;      /* 0: orthographic */
    double ortho_half_h;  /* orthographic half height, world units */
    double znear, zfar;
    int32_t width, height;
} orc_view;

typedef struct {
    int32_t mode; /* 0 screen, 1 sphere */
    int32_t pad;
    double center[3];
    double radius;
} orc_lens;

typedef struct {
    float w_base;
    int32_t lod;
    float delta, s;
    float alpha_min, alpha_max, tf_lo, tf_hi;
    float bg[3];
    float accent_beta, halo_scale, darken, g_min, g_max;
    float desat;          /* depth cue strength (R16), 0 = off */
    float sil_alpha;      /* silhouette opacity (R17), 0 = off */
    float sil_threshold;  /* silhouette depth threshold T, 24-bit depth units (R17) */
} orc_style;

/* ----------------------------------------------------------------- quality */

/* Corner k of a VTK hexahedron and its three neighbours, ordered so that the
 * unit cube gives det = +1 at every corner. */
static const int ORC_CORNER_NB[8][3] = {
    {1, 3, 4}, {2, 0, 5}, {3, 1, 6}, {0, 2, 7},
    {7, 5, 0}, {4, 6, 1}, {5, 7, 2}, {6, 4, 3}};

static double det3(const double a[3], const double b[3], const double c[3])
{
    /* a . (b x c) */
    double cx = b[1] * c[2] - b[2] * c[1];
    double cy = b[2] * c[0] - b[0] * c[2];
    double cz = b[0] * c[1] - b[1] * c[0];
    return a[0] * cx + a[1] * cy + a[2] * cz;
}

static double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/*
 * Per-cell deformation from the Jacobian of the map from the unit cube to the
 * cell (Section "Introduction": quality from the Jacobian matrix; Section
 * "Results and Analysis": per-cell scaled Jacobian ratio). The paper names the
 * measure but prints no formula; the definitions used are the standard ones:
 *   scaled Jacobian = min over the 8 corners (and the centre, with_centre) of
 *                     det of the unit-length edge vectors at that point;
 *   Jacobian ratio  = min det / max det over the same points (unnormalised);
 *   importance      = clamp(1 - scaled Jacobian, 0, 1).
 * At the centre the edge vectors are the three principal axes (sums of the
 * four parallel edges), i.e. 4x the trilinear map's derivatives.
 * A zero-length edge gives a normalised determinant of 0.
 * metric: 0 scaled Jacobian, 1 Jacobian ratio, 2 importance.
 */
void orc_cell_quality(const float* verts, const int32_t* cells, int64_t n_cells, int metric,
                      int with_centre, double* out)
{
    for (int64_t c = 0; c < n_cells; ++c) {
        double p[8][3];
        for (int k = 0; k < 8; ++k)
            for (int d = 0; d < 3; ++d) p[k][d] = (double)verts[3 * (int64_t)cells[8 * c + k] + d];
        double dets[9], ndets[9];
        int npts = 0;
        for (int k = 0; k < 8; ++k) {
            double e[3][3];
            for (int m = 0; m < 3; ++m)
                for (int d = 0; d < 3; ++d) e[m][d] = p[ORC_CORNER_NB[k][m]][d] - p[k][d];
            dets[npts] = det3(e[0], e[1], e[2]);
            double l0 = norm3(e[0]), l1 = norm3(e[1]), l2 = norm3(e[2]);
            ndets[npts] = (l0 > 0 && l1 > 0 && l2 > 0) ? dets[npts] / (l0 * l1 * l2) : 0.0;
            ++npts;
        }
        if (with_centre) {
            double X[3][3];
            for (int d = 0; d < 3; ++d) {
                X[0][d] = (p[1][d] - p[0][d]) + (p[2][d] - p[3][d]) + (p[5][d] - p[4][d]) + (p[6][d] - p[7][d]);
                X[1][d] = (p[3][d] - p[0][d]) + (p[2][d] - p[1][d]) + (p[7][d] - p[4][d]) + (p[6][d] - p[5][d]);
                X[2][d] = (p[4][d] - p[0][d]) + (p[5][d] - p[1][d]) + (p[6][d] - p[2][d]) + (p[7][d] - p[3][d]);
            }
            /* derivative of the trilinear map at the centre is X / 4 */
            dets[npts] = det3(X[0], X[1], X[2]) / 64.0;
            double l0 = norm3(X[0]), l1 = norm3(X[1]), l2 = norm3(X[2]);
            ndets[npts] = (l0 > 0 && l1 > 0 && l2 > 0) ? det3(X[0], X[1], X[2]) / (l0 * l1 * l2) : 0.0;
            ++npts;
        }
        double sj = ndets[0], dmin = dets[0], dmax = dets[0];
        for (int i = 1; i < npts; ++i) {
            if (ndets[i] < sj) sj = ndets[i];
            if (dets[i] < dmin) dmin = dets[i];
            if (dets[i] > dmax) dmax = dets[i];
        }
        double v;
        if (metric == 0) v = sj;
        else if (metric == 1) v = (dmax > 0.0) ? dmin / dmax : -1.0;
        else v = fmin(fmax(1.0 - sj, 0.0), 1.0);
        out[c] = v;
    }
}

/* ----------------------------------------------------------------- mesh */

typedef struct {
    int32_t c[4];  /* canonical cyclic corners */
    int32_t s[4];  /* sorted ids: the identity of the face */
    int32_t ncell; /* cells sharing the face: 1 on the boundary surface */
} orc_face;

typedef struct {
    int32_t a, b;  /* a < b */
    int32_t level;
    float attr;
} orc_edge;

typedef struct {
    int64_t n_verts, n_cells, n_faces, n_edges;
    float* verts;        /* n_verts*3 */
    float* vimp;         /* per-vertex importance */
    orc_face* faces;     /* unique faces sorted by s */
    orc_edge* edges;     /* unique edges sorted by (a,b) */
    int32_t* face_edge;  /* n_faces*4: edge index of local edge k = (c_k, c_k+1) */
    int64_t* bfaces;     /* ids of the boundary faces (R17) */
    int64_t n_bfaces;
    double bbox_c[3];
} orc_mesh;

/* cyclic corner orders of the six faces of a VTK hexahedron */
static const int ORC_HEX_FACES[6][4] = {
    {0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
/* the twelve edges, in the order of the per-cell-edge level input */
static const int ORC_HEX_EDGES[12][2] = {
    {0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6}, {6, 7}, {7, 4},
    {0, 4}, {1, 5}, {2, 6}, {3, 7}};

static int cmp_face(const void* x, const void* y)
{
    const orc_face* a = (const orc_face*)x;
    const orc_face* b = (const orc_face*)y;
    for (int k = 0; k < 4; ++k) {
        if (a->s[k] != b->s[k]) return a->s[k] < b->s[k] ? -1 : 1;
    }
    return 0;
}

static int cmp_edge(const void* x, const void* y)
{
    const orc_edge* a = (const orc_edge*)x;
    const orc_edge* b = (const orc_edge*)y;
    if (a->a != b->a) return a->a < b->a ? -1 : 1;
    if (a->b != b->b) return a->b < b->b ? -1 : 1;
    return 0;
}

static int64_t find_edge(const orc_mesh* m, int32_t u, int32_t v)
{
    int32_t a = u < v ? u : v, b = u < v ? v : u;
    int64_t lo = 0, hi = m->n_edges - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        const orc_edge* e = &m->edges[mid];
        if (e->a == a && e->b == b) return mid;
        if (e->a < a || (e->a == a && e->b < b)) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/*
 * Build the oracle's mesh. Importance per vertex and per edge is the maximum
 * over the incident cells (Section "Method Overview"). An edge's LoD level is
 * the maximum over the per-cell-edge entries that name it (they agree for a
 * consistent input). Returns NULL on an invalid mesh.
 */
orc_mesh* orc_mesh_build(const float* verts, int64_t n_verts, const int32_t* cells, int64_t n_cells,
                         const float* cell_importance, const uint8_t* cell_edge_level)
{
    for (int64_t i = 0; i < 8 * n_cells; ++i)
        if (cells[i] < 0 || cells[i] >= n_verts) return NULL;
    orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
    m->n_verts = n_verts;
    m->n_cells = n_cells;
    m->verts = (float*)malloc(sizeof(float) * 3 * (size_t)n_verts);
    memcpy(m->verts, verts, sizeof(float) * 3 * (size_t)n_verts);

    /* per-vertex importance */
    m->vimp = (float*)malloc(sizeof(float) * (size_t)n_verts);
    for (int64_t v = 0; v < n_verts; ++v) m->vimp[v] = -INFINITY;
    for (int64_t c = 0; c < n_cells; ++c)
        for (int k = 0; k < 8; ++k) {
            int32_t v = cells[8 * c + k];
            if (cell_importance[c] > m->vimp[v]) m->vimp[v] = cell_importance[c];
        }
    for (int64_t v = 0; v < n_verts; ++v)
        if (m->vimp[v] == -INFINITY) m->vimp[v] = 0.0f;

    /* unique faces */
    orc_face* all = (orc_face*)malloc(sizeof(orc_face) * 6 * (size_t)n_cells);
    for (int64_t c = 0; c < n_cells; ++c)
        for (int f = 0; f < 6; ++f) {
            int32_t cyc[4];
            for (int k = 0; k < 4; ++k) cyc[k] = cells[8 * c + ORC_HEX_FACES[f][k]];
            int mi = 0;
            for (int k = 1; k < 4; ++k)
                if (cyc[k] < cyc[mi]) mi = k;
            int32_t nxt = cyc[(mi + 1) % 4], prv = cyc[(mi + 3) % 4];
            orc_face* F = &all[6 * c + f];
            for (int k = 0; k < 4; ++k)
                F->c[k] = (nxt < prv) ? cyc[(mi + k) % 4] : cyc[(mi + 4 - k) % 4];
            int32_t s[4] = {cyc[0], cyc[1], cyc[2], cyc[3]};
            for (int i = 1; i < 4; ++i)
                for (int j = i; j > 0 && s[j - 1] > s[j]; --j) {
                    int32_t t = s[j];
                    s[j] = s[j - 1];
                    s[j - 1] = t;
                }
            memcpy(F->s, s, sizeof(s));
        }
    qsort(all, 6 * (size_t)n_cells, sizeof(orc_face), cmp_face);
    int64_t nf = 0;
    for (int64_t i = 0; i < 6 * n_cells; ++i) {
        if (nf == 0 || cmp_face(&all[nf - 1], &all[i]) != 0) {
            all[nf] = all[i];
            all[nf].ncell = 1;
            ++nf;
        } else {
            all[nf - 1].ncell += 1;
        }
    }
    m->faces = all;
    m->n_faces = nf;
    m->bfaces = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nf + 1));
    m->n_bfaces = 0;
    for (int64_t f = 0; f < nf; ++f)
        if (all[f].ncell == 1) m->bfaces[m->n_bfaces++] = f;

    /* unique edges with level and importance */
    orc_edge* E = (orc_edge*)malloc(sizeof(orc_edge) * 12 * (size_t)n_cells);
    for (int64_t c = 0; c < n_cells; ++c)
        for (int k = 0; k < 12; ++k) {
            int32_t u = cells[8 * c + ORC_HEX_EDGES[k][0]], v = cells[8 * c + ORC_HEX_EDGES[k][1]];
            orc_edge* e = &E[12 * c + k];
            e->a = u < v ? u : v;
            e->b = u < v ? v : u;
            e->level = cell_edge_level ? cell_edge_level[12 * c + k] : 0;
            e->attr = cell_importance[c];
        }
    qsort(E, 12 * (size_t)n_cells, sizeof(orc_edge), cmp_edge);
    int64_t ne = 0;
    for (int64_t i = 0; i < 12 * n_cells; ++i) {
        if (ne > 0 && E[ne - 1].a == E[i].a && E[ne - 1].b == E[i].b) {
            if (E[i].level > E[ne - 1].level) E[ne - 1].level = E[i].level;
            if (E[i].attr > E[ne - 1].attr) E[ne - 1].attr = E[i].attr;
        } else {
            E[ne++] = E[i];
        }
    }
    m->edges = E;
    m->n_edges = ne;

    m->face_edge = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)nf);
    for (int64_t f = 0; f < nf; ++f)
        for (int k = 0; k < 4; ++k)
            m->face_edge[4 * f + k] = (int32_t)find_edge(m, m->faces[f].c[k], m->faces[f].c[(k + 1) % 4]);

    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t v = 0; v < n_verts; ++v)
        for (int d = 0; d < 3; ++d) {
            double x = verts[3 * v + d];
            if (x < lo[d]) lo[d] = x;
            if (x > hi[d]) hi[d] = x;
        }
    for (int d = 0; d < 3; ++d) m->bbox_c[d] = (lo[d] + hi[d]) * 0.5;
    return m;
}

void orc_mesh_free(orc_mesh* m)
{
    if (!m) return;
    free(m->verts);
    free(m->vimp);
    free(m->faces);
    free(m->edges);
    free(m->face_edge);
    free(m->bfaces);
    free(m);
}

int64_t orc_mesh_n_faces(const orc_mesh* m) { return m->n_faces; }
int64_t orc_mesh_n_edges(const orc_mesh* m) { return m->n_edges; }

/* canonical corners (n_faces*4) and per-face edge levels / attrs (n_faces*4) */
void orc_mesh_faces(const orc_mesh* m, int32_t* corners, int32_t* levels, float* attrs)
{
    for (int64_t f = 0; f < m->n_faces; ++f)
        for (int k = 0; k < 4; ++k) {
            corners[4 * f + k] = m->faces[f].c[k];
            const orc_edge* e = &m->edges[m->face_edge[4 * f + k]];
            if (levels) levels[4 * f + k] = e->level;
            if (attrs) attrs[4 * f + k] = e->attr;
        }
}

void orc_mesh_vertex_importance(const orc_mesh* m, float* out)
{
    memcpy(out, m->vimp, sizeof(float) * (size_t)m->n_verts);
}

/* ----------------------------------------------------------------- camera */

typedef struct {
    int ortho;
    double eye[3], R[3], U[3], F[3];
    double focal;   /* perspective: pixels per unit of (x / depth) */
    double scale;   /* orthographic: pixels per world unit */
    double cx, cy, znear, zfar, zf_over;
    double zref;    /* |target - eye| */
    int W, H;
} orc_cam;

/* Camera basis and projection constants (reading R3: double, fixed order). */
static void orc_camera(const orc_view* v, orc_cam* c)
{
    double f[3] = {v->target[0] - v->eye[0], v->target[1] - v->eye[1], v->target[2] - v->eye[2]};
    double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int d = 0; d < 3; ++d) c->F[d] = f[d] / fl;
    double r[3] = {c->F[1] * v->up[2] - c->F[2] * v->up[1],
                   c->F[2] * v->up[0] - c->F[0] * v->up[2],
                   c->F[0] * v->up[1] - c->F[1] * v->up[0]};
    double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int d = 0; d < 3; ++d) c->R[d] = r[d] / rl;
    c->U[0] = c->R[1] * c->F[2] - c->R[2] * c->F[1];
    c->U[1] = c->R[2] * c->F[0] - c->R[0] * c->F[2];
    c->U[2] = c->R[0] * c->F[1] - c->R[1] * c->F[0];
    for (int d = 0; d < 3; ++d) c->eye[d] = v->eye[d];
    c->W = v->width;
    c->H = v->height;
    c->cx = (double)v->width * 0.5;
    c->cy = (double)v->height * 0.5;
    c->znear = v->znear;
    c->zfar = v->zfar;
    c->ortho = !(v->fovy_deg > 0.0);
    if (c->ortho) {
        c->scale = ((double)v->height * 0.5) / v->ortho_half_h;
        c->focal = 0.0;
    } else {
        c->focal = ((double)v->height * 0.5) / tan(v->fovy_deg * (3.14159265358979323846 / 180.0) * 0.5);
        c->scale = 0.0;
    }
    c->zf_over = v->zfar / (v->zfar - v->znear);
    c->zref = fl;
}

typedef struct {
    int valid;
    int32_t X, Y;    /* 16.8 fixed point window position */
    uint32_t z24;    /* quantised window depth */
    double ed;       /* eye-space depth along the view direction */
} orc_pv;

/* Vertex stage (reading R3 and R4). */
static void orc_project(const orc_cam* c, const float* p, orc_pv* o)
{
    double dx = (double)p[0] - c->eye[0];
    double dy = (double)p[1] - c->eye[1];
    double dz = (double)p[2] - c->eye[2];
    double ex = dx * c->R[0] + dy * c->R[1] + dz * c->R[2];
    double ey = dx * c->U[0] + dy * c->U[1] + dz * c->U[2];
    double ed = dx * c->F[0] + dy * c->F[1] + dz * c->F[2];
    double xw, yw, z;
    if (c->ortho) {
        xw = c->cx + ex * c->scale;
        yw = c->cy - ey * c->scale;
        z = (ed - c->znear) / (c->zfar - c->znear);
    } else {
        xw = c->cx + (ex / ed) * c->focal;
        yw = c->cy - (ey / ed) * c->focal;
        z = c->zf_over * (1.0 - c->znear / ed);
    }
    o->valid = (ed > c->znear) && (ed < c->zfar) && (fabs(xw) <= ORC_GUARD_PX) && (fabs(yw) <= ORC_GUARD_PX);
    o->ed = ed;
    if (o->valid) {
        o->X = (int32_t)rint(xw * 256.0);
        o->Y = (int32_t)rint(yw * 256.0);
        if (z < 0.0) z = 0.0;
        if (z > 1.0) z = 1.0;
        o->z24 = (uint32_t)rint(z * ORC_Z24_MAX);
    } else {
        o->X = o->Y = 0;
        o->z24 = 0;
    }
}

/* ----------------------------------------------------------------- coverage */

typedef struct {
    int valid;
    int32_t X[3], Y[3];   /* winding normalised to positive area */
    int vi[3];            /* face corner index of each vertex */
    int64_t area;         /* twice the signed area, > 0 */
    int32_t bx0, by0, bx1, by1;  /* pixel bounding box (centres), clamped */
} orc_tri;

static int64_t edge_fn(int32_t xa, int32_t ya, int32_t xb, int32_t yb, int64_t px, int64_t py)
{
    return (int64_t)(xb - xa) * (py - ya) - (int64_t)(yb - ya) * (px - xa);
}

static int top_left(int32_t xa, int32_t ya, int32_t xb, int32_t yb)
{
    int32_t dx = xb - xa, dy = yb - ya;
    return (dy < 0) || (dy == 0 && dx > 0);
}

static int64_t floor_div64(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) --q;
    return q;
}

/* Triangle setup (reading R1, R2): tri 0 = corners (0,1,2), tri 1 = (0,2,3). */
static void orc_setup_tri(const orc_pv pv[4], int tri, int W, int H, orc_tri* t)
{
    int ids[3] = {0, tri == 0 ? 1 : 2, tri == 0 ? 2 : 3};
    t->valid = 0;
    for (int k = 0; k < 3; ++k)
        if (!pv[ids[k]].valid) return;
    for (int k = 0; k < 3; ++k) {
        t->X[k] = pv[ids[k]].X;
        t->Y[k] = pv[ids[k]].Y;
        t->vi[k] = ids[k];
    }
    int64_t a = edge_fn(t->X[0], t->Y[0], t->X[1], t->Y[1], t->X[2], t->Y[2]);
    if (a == 0) return;
    if (a < 0) { /* swap vertices 1 and 2 */
        int32_t tx = t->X[1], ty = t->Y[1];
        int tv = t->vi[1];
        t->X[1] = t->X[2]; t->Y[1] = t->Y[2]; t->vi[1] = t->vi[2];
        t->X[2] = tx; t->Y[2] = ty; t->vi[2] = tv;
        a = -a;
    }
    t->area = a;
    int32_t xmin = t->X[0], xmax = t->X[0], ymin = t->Y[0], ymax = t->Y[0];
    for (int k = 1; k < 3; ++k) {
        if (t->X[k] < xmin) xmin = t->X[k];
        if (t->X[k] > xmax) xmax = t->X[k];
        if (t->Y[k] < ymin) ymin = t->Y[k];
        if (t->Y[k] > ymax) ymax = t->Y[k];
    }
    /* pixel p has centre 256 p + 128: smallest p with centre >= min, largest with centre <= max */
    int64_t bx0 = -floor_div64(-((int64_t)xmin - 128), 256);
    int64_t by0 = -floor_div64(-((int64_t)ymin - 128), 256);
    int64_t bx1 = floor_div64((int64_t)xmax - 128, 256);
    int64_t by1 = floor_div64((int64_t)ymax - 128, 256);
    if (bx0 < 0) bx0 = 0;
    if (by0 < 0) by0 = 0;
    if (bx1 > W - 1) bx1 = W - 1;
    if (by1 > H - 1) by1 = H - 1;
    if (bx0 > bx1 || by0 > by1) return;
    t->bx0 = (int32_t)bx0; t->by0 = (int32_t)by0; t->bx1 = (int32_t)bx1; t->by1 = (int32_t)by1;
    t->valid = 1;
}

/* Coverage of pixel (px,py) with exact edge functions; on success the three
 * barycentric weights (l[k] for vertex k, summing to area) are returned. */
static int orc_covers(const orc_tri* t, int32_t px, int32_t py, int64_t l[3])
{
    if (!t->valid || px < t->bx0 || px > t->bx1 || py < t->by0 || py > t->by1) return 0;
    int64_t sx = 256 * (int64_t)px + 128, sy = 256 * (int64_t)py + 128;
    for (int k = 0; k < 3; ++k) {
        int a = (k + 1) % 3, b = (k + 2) % 3; /* edge opposite vertex k */
        int64_t e = edge_fn(t->X[a], t->Y[a], t->X[b], t->Y[b], sx, sy);
        if (e < 0) return 0;
        if (e == 0 && !top_left(t->X[a], t->Y[a], t->X[b], t->Y[b])) return 0;
        l[k] = e;
    }
    return 1;
}

/* Exact per-sample depth (reading R4): z0 + floor((l1 (z1-z0) + l2 (z2-z0)) / area). */
static uint32_t orc_depth(const orc_tri* t, const orc_pv pv[4], const int64_t l[3])
{
    int64_t z0 = pv[t->vi[0]].z24, z1 = pv[t->vi[1]].z24, z2 = pv[t->vi[2]].z24;
    __int128 n = (__int128)l[1] * (z1 - z0) + (__int128)l[2] * (z2 - z0);
    __int128 q = n / t->area;
    if ((n % t->area != 0) && (n < 0)) --q;
    return (uint32_t)(z0 + (int64_t)q);
}

/* ----------------------------------------------------------------- shading */

static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/* GLSL smoothstep */
double orc_smoothstep(double e0, double e1, double x)
{
    double t = clamp01((x - e0) / (e1 - e0));
    return t * t * (3.0 - 2.0 * t);
}

/* distance (pixels) from sample s to segment a-b; all in 1/256 pixel units */
static double seg_dist(int64_t sx, int64_t sy, int32_t ax, int32_t ay, int32_t bx, int32_t by)
{
    int64_t px = sx - ax, py = sy - ay;
    int64_t ex = (int64_t)bx - ax, ey = (int64_t)by - ay;
    int64_t len2 = ex * ex + ey * ey;
    int64_t dot = px * ex + py * ey;
    double d;
    if (len2 == 0 || dot <= 0) {
        d = sqrt((double)(px * px + py * py));
    } else if (dot >= len2) {
        int64_t qx = sx - bx, qy = sy - by;
        d = sqrt((double)(qx * qx + qy * qy));
    } else {
        double cr = (double)(px * ey - py * ex);
        d = fabs(cr) / sqrt((double)len2);
    }
    return d / 256.0;
}

/*
 * The focus+context formulas of Section "Focus+Context", given the per-
 * fragment geometric quantities. Inputs:
 *   dist   normalised lens distance (R6)
 *   d_f, d_c, d_a  edge distances in pixels (R8; INFINITY if no such edge)
 *   g      depth factor of R9 (1 for orthographic)
 *   t_imp  interpolated vertex importance
 * flip: bit 0 flips e_focus, bit 1 e_context, bit 2 the halo test, bit 3 the
 * Eq. 2 test. tie (optional) receives the bits of decisions within the margin.
 * Output: premultiplied colour and opacity of Eq. 4 (rgba[0..3]).
 */
void orc_fc_shade(const orc_style* st, double dist, double d_f, double d_c, double d_a, double g,
                  double t_imp, int flip, double rgba[4], int* tie)
{
    double w_base = st->w_base;
    double focus = 1.0 - orc_smoothstep(0.7, 1.0, dist);
    /* Eq. 1 */
    double w = (1.0 + 0.3 * focus) * w_base * g;
    int e_focus = d_f <= w;
    int e_context = d_c <= w;
    double h = (double)st->halo_scale * w_base * focus * g;
    int in_halo = d_f <= w + h;
    int accent = d_a <= (2.0 / 3.0) * w_base;
    int tb = 0;
    if (fabs(d_f - w) < ORC_TIE_MARGIN) tb |= 1;
    if (fabs(d_c - w) < ORC_TIE_MARGIN) tb |= 2;
    if (h > 0.0 && fabs(d_f - (w + h)) < ORC_TIE_MARGIN) tb |= 4;
    if (fabs(d_a - (2.0 / 3.0) * w_base) < ORC_TIE_MARGIN) tb |= 8;
    if (tie) *tie = tb;
    if (flip & 1) e_focus = !e_focus;
    if (flip & 2) e_context = !e_context;
    if (flip & 4) in_halo = !in_halo;
    if (flip & 8) accent = !accent;

    double alpha_e = (double)e_context + focus * ((double)e_focus - (double)e_context);
    int halo = (!e_focus) && in_halo && focus > 0.0;
    if (halo) alpha_e = focus; /* e_context = 0 in the band: d_c >= d_f > w */

    /* colour table (R10) */
    double t = clamp01((t_imp - st->tf_lo) / ((double)st->tf_hi - st->tf_lo));
    double ctf[3] = {t, 0.0, 1.0 - t};
    double ce[3], cf[3];
    for (int k = 0; k < 3; ++k) {
        ce[k] = halo ? 1.0 : ctf[k] * (1.0 - (double)st->darken * focus);
        cf[k] = ctf[k];
    }
    /* Eq. 2 */
    double s_e = accent ? (double)st->s : 1.0;
    if (s_e > 1.0)
        for (int k = 0; k < 3; ++k) cf[k] = cf[k] + (double)st->accent_beta * (1.0 - cf[k]);
    /* Eq. 3 */
    double ahat = st->alpha_min + ((double)st->alpha_max - st->alpha_min) * t;
    double dc = dist < 1.0 ? dist : 1.0;
    double alpha_f = ahat * dc * dc * dc * dc;
    /* Eq. 4 */
    double af = s_e * alpha_f;
    if (af > 1.0) af = 1.0;
    for (int k = 0; k < 3; ++k) rgba[k] = alpha_e * ce[k] + (1.0 - alpha_e) * af * cf[k];
    rgba[3] = alpha_e + (1.0 - alpha_e) * af;
    /* depth cue of Section "Evaluation" (R16): fragments in focus and beyond
     * the reference depth (g < 1) lose part of their saturation; the colour
     * moves towards its Rec. 601 luma, opacity unchanged */
    double kd = (double)st->desat * focus * clamp01(1.0 - g);
    if (kd > 0.0) {
        double y = 0.299 * rgba[0] + 0.587 * rgba[1] + 0.114 * rgba[2];
        for (int k = 0; k < 3; ++k) rgba[k] = rgba[k] + kd * (y - rgba[k]);
    }
}

typedef struct {
    orc_cam cam;
    orc_pv* pv;      /* per vertex */
    orc_tri* tri;    /* 2 per face */
} orc_frame;

static void orc_frame_setup(const orc_mesh* m, const orc_view* v, orc_frame* fr)
{
    orc_camera(v, &fr->cam);
    fr->pv = (orc_pv*)malloc(sizeof(orc_pv) * (size_t)m->n_verts);
    for (int64_t i = 0; i < m->n_verts; ++i) orc_project(&fr->cam, &m->verts[3 * i], &fr->pv[i]);
    fr->tri = (orc_tri*)malloc(sizeof(orc_tri) * 2 * (size_t)m->n_faces);
    for (int64_t f = 0; f < m->n_faces; ++f) {
        orc_pv pv[4];
        for (int k = 0; k < 4; ++k) pv[k] = fr->pv[m->faces[f].c[k]];
        orc_setup_tri(pv, 0, v->width, v->height, &fr->tri[2 * f]);
        orc_setup_tri(pv, 1, v->width, v->height, &fr->tri[2 * f + 1]);
    }
}

static void orc_frame_free(orc_frame* fr)
{
    free(fr->pv);
    free(fr->tri);
}

/* Geometric quantities of one fragment, the inputs of the focus+context
 * formulas (Section "Focus+Context", readings R6, R8, R9, R10). */
typedef struct {
    double dist;           /* normalised lens distance (R6) */
    double d_f, d_c, d_a;  /* edge distances per visibility class, pixels (R8) */
    double g;              /* depth factor of the edge width (R9) */
    double z_eye;          /* eye-space depth of the sample */
    double t_imp;          /* interpolated vertex importance (R10) */
    double P[3];           /* interpolated world position */
    double b[3];           /* interpolation weights of the triangle's vertices */
} orc_geom;

/* Fragment geometry of face f, triangle tri at pixel (px,py), whose exact
 * barycentric weights are l: perspective-correct weights, importance, world
 * position and eye depth, lens distance, edge distances and depth factor. */
static void orc_frag_geometry(const orc_mesh* m, const orc_frame* fr, const orc_lens* lens,
                              const orc_style* st, int64_t f, int tri, int32_t px, int32_t py,
                              const int64_t l[3], orc_geom* G)
{
    const orc_tri* t = &fr->tri[2 * f + tri];
    const orc_face* F = &m->faces[f];
    const orc_cam* c = &fr->cam;
    double lam[3], b[3];
    for (int k = 0; k < 3; ++k) lam[k] = (double)l[k] / (double)t->area;
    double z_eye;
    if (c->ortho) {
        for (int k = 0; k < 3; ++k) b[k] = lam[k];
        z_eye = 0.0;
        for (int k = 0; k < 3; ++k) z_eye += lam[k] * fr->pv[F->c[t->vi[k]]].ed;
    } else { /* perspective-correct interpolation */
        double q[3], Q = 0.0;
        for (int k = 0; k < 3; ++k) {
            q[k] = lam[k] / fr->pv[F->c[t->vi[k]]].ed;
            Q += q[k];
        }
        for (int k = 0; k < 3; ++k) b[k] = q[k] / Q;
        z_eye = 1.0 / Q;
    }
    double t_imp = 0.0, P[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
        int32_t vid = F->c[t->vi[k]];
        t_imp += b[k] * (double)m->vimp[vid];
        for (int d = 0; d < 3; ++d) P[d] += b[k] * (double)m->verts[3 * (int64_t)vid + d];
    }
    /* lens distance (R6) */
    double dist;
    if (lens->mode == 0) {
        double dx = ((double)px + 0.5) - lens->center[0], dy = ((double)py + 0.5) - lens->center[1];
        dist = sqrt(dx * dx + dy * dy) / lens->radius;
    } else {
        double dx = P[0] - lens->center[0], dy = P[1] - lens->center[1], dz = P[2] - lens->center[2];
        dist = sqrt(dx * dx + dy * dy + dz * dz) / lens->radius;
    }
    /* edge distances (R8) */
    int64_t sx = 256 * (int64_t)px + 128, sy = 256 * (int64_t)py + 128;
    double d_f = INFINITY, d_c = INFINITY, d_a = INFINITY;
    for (int k = 0; k < 4; ++k) {
        const orc_pv* A = &fr->pv[F->c[k]];
        const orc_pv* B = &fr->pv[F->c[(k + 1) % 4]];
        double d = seg_dist(sx, sy, A->X, A->Y, B->X, B->Y);
        const orc_edge* e = &m->edges[m->face_edge[4 * f + k]];
        int vis_c = e->level >= st->lod;
        int vis_f = vis_c || e->attr >= st->delta;
        if (d < d_a) d_a = d;
        if (vis_f && d < d_f) d_f = d;
        if (vis_c && d < d_c) d_c = d;
    }
    /* depth factor (R9) */
    double g = 1.0;
    if (!c->ortho) {
        g = c->zref / z_eye;
        if (g < st->g_min) g = st->g_min;
        if (g > st->g_max) g = st->g_max;
    }
    G->dist = dist;
    G->d_f = d_f;
    G->d_c = d_c;
    G->d_a = d_a;
    G->g = g;
    G->z_eye = z_eye;
    G->t_imp = t_imp;
    for (int k = 0; k < 3; ++k) {
        G->P[k] = P[k];
        G->b[k] = b[k];
    }
}

/* Shade the fragment of face f, triangle tri at pixel (px,py), whose exact
 * barycentric weights are l (Section "Focus+Context", readings R6-R11). */
static void orc_shade_frag(const orc_mesh* m, const orc_frame* fr, const orc_lens* lens,
                           const orc_style* st, int64_t f, int tri, int32_t px, int32_t py,
                           const int64_t l[3], int flip, double rgba[4], int* tie)
{
    orc_geom G;
    orc_frag_geometry(m, fr, lens, st, f, tri, px, py, l, &G);
    orc_fc_shade(st, G.dist, G.d_f, G.d_c, G.d_a, G.g, G.t_imp, flip, rgba, tie);
}

typedef struct {
    uint64_t key;
    double rgba[4];
    int tie;
} orc_frag;

/* Depth (24-bit) of the nearest fragment of a boundary face at pixel (px,py);
 * 0 if no boundary face covers it (reading R17). */
static int orc_boundary_depth(const orc_mesh* m, const orc_frame* fr, int32_t px, int32_t py, uint32_t* z)
{
    int found = 0;
    uint32_t best = 0;
    for (int64_t b = 0; b < m->n_bfaces; ++b) {
        const int64_t f = m->bfaces[b];
        for (int tri = 0; tri < 2; ++tri) {
            const orc_tri* t = &fr->tri[2 * f + tri];
            int64_t l[3];
            if (!orc_covers(t, px, py, l)) continue;
            orc_pv pv[4];
            for (int k = 0; k < 4; ++k) pv[k] = fr->pv[m->faces[f].c[k]];
            const uint32_t d = orc_depth(t, pv, l);
            if (!found || d < best) best = d;
            found = 1;
        }
    }
    *z = best;
    return found;
}

/* Is (px,py) a silhouette pixel of the boundary surface's depth image (R17)? */
static int orc_silhouette(const orc_mesh* m, const orc_frame* fr, const orc_style* st, int32_t px, int32_t py,
                          int W, int H)
{
    uint32_t zp;
    if (!orc_boundary_depth(m, fr, px, py, &zp)) return 0;
    static const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1};   /* k ^ 1 is the opposite side */
    int inside[4], has[4];
    uint32_t zq[4];
    for (int k = 0; k < 4; ++k) {
        const int32_t qx = px + dx[k], qy = py + dy[k];
        inside[k] = qx >= 0 && qy >= 0 && qx < W && qy < H;
        has[k] = inside[k] && orc_boundary_depth(m, fr, qx, qy, &zq[k]);
        if (inside[k] && !has[k]) return 1;   /* exterior: the surface ends here */
    }
    const int64_t T = (int64_t)st->sil_threshold;
    for (int k = 0; k < 4; ++k) {
        const int o = k ^ 1;
        if (!has[k] || !has[o]) continue;
        const int64_t d1 = (int64_t)zq[k] - (int64_t)zp;
        const int64_t d2 = (int64_t)zq[k] - 2 * (int64_t)zp + (int64_t)zq[o];
        if (d1 > T && (d2 > T || -d2 > T)) return 1;   /* interior: the near side of a depth jump */
    }
    return 0;
}

/*
 * Render the listed pixels. For pixel i: counts[i] fragments, written in
 * sorted order at the running offset into keys (uint64), frag_rgba (4 doubles
 * each) and frag_tie (bit mask of near-tie decisions); image[4 i..] gets the
 * composited RGBA (with the silhouette overlay of R17) and sil[i] 1 if the
 * pixel is a silhouette pixel (computed only if st->sil_alpha > 0). Any output
 * pointer may be NULL. Returns the total number of fragments, or -1 if it
 * exceeds cap (counts and image are still complete).
 */
int64_t orc_render(const orc_mesh* m, const orc_view* v, const orc_lens* lens, const orc_style* st,
                   const int32_t* pxs, const int32_t* pys, int64_t npix, int64_t cap,
                   uint32_t* counts, uint64_t* keys, double* frag_rgba, uint8_t* frag_tie,
                   double* image, uint8_t* sil)
{
    orc_frame fr;
    orc_frame_setup(m, v, &fr);
    int64_t n2 = 2 * m->n_faces;
    /* pass 1: counts per pixel (parallel over pixels) */
    uint32_t* cnt = (uint32_t*)calloc((size_t)npix + 1, sizeof(uint32_t));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < npix; ++i) {
        uint32_t n = 0;
        int64_t l[3];
        for (int64_t j = 0; j < n2; ++j) n += (uint32_t)orc_covers(&fr.tri[j], pxs[i], pys[i], l);
        cnt[i] = n;
    }
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)npix + 1));
    off[0] = 0;
    for (int64_t i = 0; i < npix; ++i) off[i + 1] = off[i] + cnt[i];
    int64_t total = off[npix];
    int fits = total <= cap;
    /* pass 2: fragments, sort, blend */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < npix; ++i) {
        orc_frag* L = (orc_frag*)malloc(sizeof(orc_frag) * (cnt[i] + 1));
        uint32_t n = 0;
        int64_t l[3];
        for (int64_t j = 0; j < n2; ++j) {
            if (!orc_covers(&fr.tri[j], pxs[i], pys[i], l)) continue;
            int64_t f = j / 2;
            int tri = (int)(j % 2);
            orc_pv pv[4];
            for (int k = 0; k < 4; ++k) pv[k] = fr.pv[m->faces[f].c[k]];
            uint32_t z = orc_depth(&fr.tri[j], pv, l);
            orc_frag* fg = &L[n++];
            fg->key = ((uint64_t)z << 32) | (uint64_t)(2 * f + tri);
            orc_shade_frag(m, &fr, lens, st, f, tri, pxs[i], pys[i], l, 0, fg->rgba, &fg->tie);
        }
        /* stable insertion sort by key, ascending = front to back */
        for (uint32_t a = 1; a < n; ++a) {
            orc_frag x = L[a];
            uint32_t b = a;
            while (b > 0 && L[b - 1].key > x.key) {
                L[b] = L[b - 1];
                --b;
            }
            L[b] = x;
        }
        /* front-to-back alpha compositing over the background */
        double C[3] = {0.0, 0.0, 0.0}, A = 0.0;
        for (uint32_t a = 0; a < n; ++a) {
            double tr = 1.0 - A;
            for (int k = 0; k < 3; ++k) C[k] += tr * L[a].rgba[k];
            A += tr * L[a].rgba[3];
        }
        if (counts) counts[i] = n;
        const int is_sil = st->sil_alpha > 0.0f &&
                           orc_silhouette(m, &fr, st, pxs[i], pys[i], v->width, v->height);
        if (sil) sil[i] = (uint8_t)is_sil;
        if (image) {
            for (int k = 0; k < 3; ++k) image[4 * i + k] = C[k] + (1.0 - A) * (double)st->bg[k];
            image[4 * i + 3] = A;
            if (is_sil) { /* white silhouette over the pixel (R17) */
                const double a = st->sil_alpha;
                for (int k = 0; k < 4; ++k) image[4 * i + k] = image[4 * i + k] + a * (1.0 - image[4 * i + k]);
            }
        }
        if (fits) {
            for (uint32_t a = 0; a < n; ++a) {
                int64_t o = off[i] + a;
                if (keys) keys[o] = L[a].key;
                if (frag_rgba)
                    for (int k = 0; k < 4; ++k) frag_rgba[4 * o + k] = L[a].rgba[k];
                if (frag_tie) frag_tie[o] = (uint8_t)L[a].tie;
            }
        }
        free(L);
    }
    free(cnt);
    free(off);
    orc_frame_free(&fr);
    return fits ? total : -1;
}

/* A frame holding only the four corners of face f and its triangle tri:
 * enough to shade that face's fragments. */
static int orc_face_frame(const orc_mesh* m, const orc_view* v, int64_t f, int tri, orc_frame* fr)
{
    if (f < 0 || f >= m->n_faces) return 0;
    orc_camera(v, &fr->cam);
    fr->pv = (orc_pv*)calloc((size_t)m->n_verts, sizeof(orc_pv));
    for (int k = 0; k < 4; ++k) {
        int32_t vid = m->faces[f].c[k];
        orc_project(&fr->cam, &m->verts[3 * (int64_t)vid], &fr->pv[vid]);
    }
    fr->tri = (orc_tri*)calloc(2 * (size_t)m->n_faces, sizeof(orc_tri));
    orc_pv pv[4];
    for (int k = 0; k < 4; ++k) pv[k] = fr->pv[m->faces[f].c[k]];
    orc_setup_tri(pv, tri, v->width, v->height, &fr->tri[2 * f + tri]);
    return 1;
}

/*
 * Shade one fragment (face2tri = 2 face + tri at pixel px,py) with the
 * decisions in flip inverted. Returns 1 and fills rgba/tie if the triangle
 * covers the pixel, 0 otherwise.
 */
int orc_shade(const orc_mesh* m, const orc_view* v, const orc_lens* lens, const orc_style* st,
              int32_t px, int32_t py, uint32_t face2tri, int flip, double rgba[4], int* tie)
{
    int64_t f = face2tri / 2;
    int tri = (int)(face2tri % 2);
    orc_frame fr;
    if (!orc_face_frame(m, v, f, tri, &fr)) return 0;
    int64_t l[3];
    int ok = orc_covers(&fr.tri[2 * f + tri], px, py, l);
    if (ok) orc_shade_frag(m, &fr, lens, st, f, tri, px, py, l, flip, rgba, tie);
    orc_frame_free(&fr);
    return ok;
}

/*
 * Test hook: the geometric inputs of the focus+context formulas for one
 * fragment (face2tri at pixel px,py). out[0..13] = dist, d_f, d_c, d_a, g,
 * z_eye, t_imp, P[3], b[3] (the weights of the triangle's vertices in the
 * winding order of the coverage setup), and vi[0..2] = the face corner index
 * (0..3) of each of those vertices. Returns 1 if the triangle covers the
 * pixel, 0 otherwise.
 */
int orc_fragment_geometry(const orc_mesh* m, const orc_view* v, const orc_lens* lens,
                          const orc_style* st, int32_t px, int32_t py, uint32_t face2tri,
                          double out[13], int32_t vi[3])
{
    int64_t f = face2tri / 2;
    int tri = (int)(face2tri % 2);
    orc_frame fr;
    if (!orc_face_frame(m, v, f, tri, &fr)) return 0;
    int64_t l[3];
    int ok = orc_covers(&fr.tri[2 * f + tri], px, py, l);
    if (ok) {
        orc_geom G;
        orc_frag_geometry(m, &fr, lens, st, f, tri, px, py, l, &G);
        double vals[13] = {G.dist, G.d_f, G.d_c, G.d_a, G.g, G.z_eye, G.t_imp,
                           G.P[0], G.P[1], G.P[2], G.b[0], G.b[1], G.b[2]};
        memcpy(out, vals, sizeof(vals));
        for (int k = 0; k < 3; ++k) vi[k] = fr.tri[2 * f + tri].vi[k];
    }
    orc_frame_free(&fr);
    return ok;
}

/* Test hook: the boundary surface's depth at pixel (px,py) (reading R17):
 * returns 1 and *z (24-bit depth of the nearest boundary-face fragment), or 0
 * if no boundary face covers the pixel. */
int orc_boundary_depth_at(const orc_mesh* m, const orc_view* v, int32_t px, int32_t py, uint32_t* z)
{
    orc_frame fr;
    orc_frame_setup(m, v, &fr);
    const int ok = orc_boundary_depth(m, &fr, px, py, z);
    orc_frame_free(&fr);
    return ok;
}

/* Test hook: pixel distance from sample (sx,sy) to the segment a-b, all in
 * 1/256 pixel units (reading R8). */
double orc_segment_distance(int64_t sx, int64_t sy, int32_t ax, int32_t ay, int32_t bx, int32_t by)
{
    return seg_dist(sx, sy, ax, ay, bx, by);
}

/* Front-to-back compositing of n premultiplied fragments (already sorted). */
void orc_composite(const double* rgba, int64_t n, const float bg[3], double out[4])
{
    double C[3] = {0.0, 0.0, 0.0}, A = 0.0;
    for (int64_t a = 0; a < n; ++a) {
        double tr = 1.0 - A;
        for (int k = 0; k < 3; ++k) C[k] += tr * rgba[4 * a + k];
        A += tr * rgba[4 * a + 3];
    }
    for (int k = 0; k < 3; ++k) out[k] = C[k] + (1.0 - A) * (double)bg[k];
    out[3] = A;
}

/* Projected vertices (for tests): valid, X, Y, z24 per vertex. */
void orc_project_vertices(const orc_mesh* m, const orc_view* v, int32_t* valid, int32_t* X,
                          int32_t* Y, uint32_t* z24)
{
    orc_cam c;
    orc_camera(v, &c);
    for (int64_t i = 0; i < m->n_verts; ++i) {
        orc_pv p;
        orc_project(&c, &m->verts[3 * i], &p);
        valid[i] = p.valid;
        X[i] = p.X;
        Y[i] = p.Y;
        z24[i] = p.z24;
    }
}

/* Coverage of one pixel by one raw triangle in 16.8 fixed point (for tests of
 * the fill rule): 1 if covered. */
int orc_cover_raw(const int32_t X[3], const int32_t Y[3], int32_t px, int32_t py, int W, int H)
{
    orc_pv pv[4];
    for (int k = 0; k < 3; ++k) {
        pv[k].valid = 1;
        pv[k].X = X[k];
        pv[k].Y = Y[k];
        pv[k].z24 = 0;
        pv[k].ed = 1.0;
    }
    pv[3] = pv[2];
    orc_tri t;
    orc_setup_tri(pv, 0, W, H, &t);
    int64_t l[3];
    return orc_covers(&t, px, py, l);
}

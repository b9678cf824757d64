/*
 * hexfc.h -- C ABI of the GB300 focus+context hex-mesh renderer.
 *
 * The library renders every face of a hexahedral mesh into per-pixel fragment
 * lists, shades each fragment in the focus+context edge/face style, sorts
 * each list by depth and blends it front to back ("Interactive Focus+Context
 * Rendering for Hexahedral Mesh Inspection", Neuhauser, Wang, Westermann:
 * Section "Method Overview", Section "Focus+Context" Eqs. 1-4, Section
 * "GPU Implementation").
 *
 * Conventions for every entry point
 *   - Host pointers are read during the call only; the caller keeps ownership.
 *   - Device pointers (marked "device") are caller-owned CUDA allocations on
 *     the context's device; the library writes them on the given stream.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - The library owns the resident mesh buffers and the fragment buffers; they
 *     live until hexfc_destroy.
 *   - No C++ exception crosses this boundary; every failure is a status < 0.
 *   - A context is not thread-safe: calls on one context must be serialised.
 */
#ifndef HEXFC_H
#define HEXFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hexfc_status;

enum {
    HEXFC_OK = 0,
    HEXFC_ERR_ARG = -1,       /* a pointer, size or parameter is invalid */
    HEXFC_ERR_OOM = -2,       /* device allocation failed, or the fragment total exceeds the budget */
    HEXFC_ERR_OVERFLOW = -3,  /* a per-pixel list exceeds HEXFC_MAX_LIST */
    HEXFC_ERR_CUDA = -4,      /* a CUDA runtime call or kernel launch failed */
    HEXFC_ERR_TIMEOUT = -5,   /* a bounded device-side wait ran out */
    HEXFC_ERR_MESH = -6,      /* the mesh is malformed (index out of range, non-finite vertex) */
    HEXFC_ERR_STATE = -7,     /* call out of order (no mesh, no view, no previous render) */
    HEXFC_ERR_CHECK = -8      /* a device-side consistency check failed (list sizes of the count and
                                 fill passes disagree, or an exact depth could not be confirmed) */
};

/* Longest per-pixel fragment list the sort/composite pass accepts. */
#define HEXFC_MAX_LIST 8192

typedef struct hexfc_ctx hexfc_ctx;

/*
 * Camera (Section "Results and Analysis": timings along camera paths).
 * eye/target/up in world units; fovy_deg > 0 selects a perspective camera with
 * that vertical field of view, fovy_deg == 0 an orthographic camera whose view
 * height is 2*ortho_half_h world units. Fragments are kept for
 * znear < depth < zfar (depth along the view direction); triangles with a
 * vertex outside that range, or outside +-16384 px, are not drawn.
 * width x height pixels, row 0 at the top, pixel centres at (x+.5, y+.5).
 */
typedef struct hexfc_view {
    double eye[3];
    double target[3];
    double up[3];
    double fovy_deg;
    double ortho_half_h;
    double znear, zfar;
    int32_t width, height;
} hexfc_view;

enum { HEXFC_LENS_SCREEN = 0, HEXFC_LENS_SPHERE = 1 };

/*
 * Focus lens (Section "Focus+Context": circular screen-space lens with centre
 * and radius, focus = 1 - smoothstep(0.7, 1, dist); Section "Evaluation":
 * object-space lens). SCREEN: center[0..1] in pixels, radius in pixels.
 * SPHERE: center in world units, radius in world units, dist measured from the
 * fragment's world position.
 */
typedef struct hexfc_lens {
    int32_t mode;
    int32_t pad;
    double center[3];
    double radius;
} hexfc_lens;

/*
 * Style constants (Section "GPU Implementation": all constants of Eqs. 1-3
 * are shader parameters). w_base: minimum edge width in pixels (Eq. 1);
 * lod, delta: LoD level and importance threshold of Eq. 1; s: accentuation
 * of Eq. 2; alpha_min..alpha_max: face opacity transfer function (Eq. 3's
 * alpha_hat); tf_lo..tf_hi: importance range mapped to the blue-to-red colour
 * table; bg: background colour (Section "Contextual Volume Rendering");
 * accent_beta: brightening of accentuated edges (Section "Blending Focus and
 * Context"); halo_scale, darken: halo width and edge darkening of the focus
 * edges; g_min, g_max: clamp of the depth-dependent width factor; desat:
 * strength of the depth cue of Section "Evaluation" (fragments in focus
 * beyond the reference depth are desaturated by desat * focus * clamp(1 - g,
 * 0, 1) towards their luma; 0 = off, the default).
 */
typedef struct hexfc_style {
    float w_base;
    int32_t lod;
    float delta;
    float s;
    float alpha_min, alpha_max;
    float tf_lo, tf_hi;
    float bg[3];
    float accent_beta;
    float halo_scale;
    float darken;
    float g_min, g_max;
    float desat;
    float sil_alpha;       /* opacity of the white silhouettes of the boundary surface, 0 = off */
    float sil_threshold;   /* depth jump (24-bit window depth units) of an interior silhouette */
} hexfc_style;

/* Per-frame statistics of the last hexfc_render* call. */
typedef struct hexfc_frame_stats {
    uint64_t fragments;      /* fragments generated (sum of list lengths) */
    uint64_t bin_entries;    /* (triangle, tile) pairs after binning */
    uint32_t max_list;       /* longest per-pixel list */
    uint32_t long_lists;     /* pixels handled by the long-list path */
    uint32_t width, height;
    uint32_t kernel_launches;  /* kernels this call launched */
    uint32_t covered_pixels;   /* reserved (0) */
    uint32_t predicted;        /* 1: drawn with chosen tile capacities (no pixel scan, no host wait
                                  after the count pass) */
    uint32_t overflow_tiles;   /* tiles above their chosen capacity (their lists in the pool) */
    uint64_t capacity;         /* sum of the chosen tile capacities (fragments), 0 if none */
    uint32_t pending;          /* 1: a frame with chosen capacities whose device statistics (fragments,
                                  max_list, long_lists, overflow_tiles, capacity) are not known yet:
                                  hexfc_finish or hexfc_completed_stats give them once it is verified */
    uint32_t redrawn;          /* 1: its chosen capacities ran out and it was drawn again exactly */
    uint64_t frame;            /* sequence number of the frame in its context (1, 2, ...) */
} hexfc_frame_stats;

/* Stages timed by HEXFC_OPT_STAGE_TIMING (CUDA events on the render stream).
 * GAP stages are the host round trips that read the bin and fragment totals. */
enum {
    HEXFC_STAGE_VERTEX = 0,   /* vertex projection */
    HEXFC_STAGE_FACE = 1,     /* face setup and tile counts */
    HEXFC_STAGE_TILE_SCAN = 2,
    HEXFC_STAGE_GAP1 = 3,
    HEXFC_STAGE_BIN = 4,      /* bin fill */
    HEXFC_STAGE_COUNT = 5,    /* per-pixel fragment count */
    HEXFC_STAGE_SCAN = 6,     /* pixel prefix scan */
    HEXFC_STAGE_GAP2 = 7,
    HEXFC_STAGE_FILL = 8,     /* fragment fill and shading */
    HEXFC_STAGE_COMPOSITE = 9,/* sort and composite (both list paths) */
    HEXFC_N_STAGES = 10
};

enum {
    HEXFC_METRIC_SCALED_JACOBIAN = 0,
    HEXFC_METRIC_JACOBIAN_RATIO = 1,
    HEXFC_METRIC_IMPORTANCE = 2   /* clamp(1 - scaled Jacobian, 0, 1) */
};

/* Fills *style with the defaults (w_base 2, lod 1, delta 0.5, s 1.5, alpha
 * 0.1..0.6, tf 0..1, black background, accent 0.2, halo 0.5, darken 0.25,
 * g 0.5..2). Never fails. */
void hexfc_style_default(hexfc_style* style);

/* Create a context on CUDA device `device`. frag_budget_bytes caps the device
 * memory of the context's frame buffers (hexfc_frame_memory), fragment arrays
 * (24 bytes per fragment) included: a count-then-fill frame that would need
 * more is refused with OOM before its fragment arrays grow; 0 means no cap
 * beyond free memory. HEXFC_OPT_FRAG_BUDGET changes it between frames.
 * Errors: ARG (out == NULL), CUDA (bad device). */
hexfc_status hexfc_create(hexfc_ctx** out, int device, uint64_t frag_budget_bytes);

/* Free everything the context owns. Accepts NULL. */
void hexfc_destroy(hexfc_ctx* ctx);

/*
 * Upload a hexahedral mesh and keep it resident on the device (Section "GPU
 * Implementation": all data required for rendering is kept on the GPU).
 *   verts            host, n_verts*3 float, xyz
 *   cells            host, n_cells*8 int32, VTK hexahedron corner order
 *   cell_scalar      host, n_cells float per-cell importance, or NULL: the
 *                    importance is computed on the device as
 *                    HEXFC_METRIC_IMPORTANCE (Section "Introduction")
 *   cell_edge_level  host, n_cells*12 uint8 LoD level per cell edge, edge order
 *                    01 12 23 30 45 56 67 74 04 15 26 37 (Section "Level of
 *                    Detail Structure": each edge carries the highest level
 *                    at which it still exists), or NULL for level 0
 * Builds the unique faces (each geometric face once, canonical corner order,
 * face id = rank of its sorted vertex ids) and unique edges on the host, and
 * the per-vertex / per-edge importance (max over incident cells, Section
 * "Method Overview") on the device. *mesh_id_out receives the mesh handle.
 * Errors: ARG, MESH (index out of range, non-finite vertex, n_cells == 0),
 * OOM, CUDA. Synchronous.
 */
hexfc_status hexfc_upload_mesh(hexfc_ctx* ctx, const float* verts, int64_t n_verts,
                               const int32_t* cells, int64_t n_cells, const float* cell_scalar,
                               const uint8_t* cell_edge_level, int32_t* mesh_id_out);

/*
 * Serving support (no counterpart in the paper; used to render many requests
 * at once on one GPU with one context per concurrent frame).
 *
 * hexfc_share_mesh: make mesh `mesh` of context src available in context dst
 * (same device) without a copy; *mesh_id_out receives its handle in dst. A
 * mesh stays resident until every context holding it is destroyed. Rendering
 * and quality evaluation only read a resident mesh, so contexts may render a
 * shared mesh at the same time from different host threads;
 * hexfc_set_cell_importance rewrites it for every holder and must not overlap
 * a render of it. Errors: ARG (NULL pointer, different devices), STATE (no
 * such mesh in src), OOM.
 *
 * hexfc_frame_memory: *bytes = device memory held by the context's per-frame
 * buffers (they grow to the largest frame rendered and are reused).
 * Errors: ARG.
 *
 * hexfc_trim: free the context's per-frame buffers (the next render allocates
 * them again). Call only when no render of this context is in flight.
 * Errors: ARG.
 */
hexfc_status hexfc_share_mesh(hexfc_ctx* dst, const hexfc_ctx* src, int32_t mesh, int32_t* mesh_id_out);

/*
 * Batched frames (no counterpart in the paper): many views of one or several
 * resident meshes, each with its own camera, lens, style and output, in one
 * call. The frame's three phases (geometry up to the bin total; binning,
 * depth order and coverage count up to the fragment total; fill and
 * composite) run for all items at once: each phase is captured as one CUDA
 * graph with the items on their own streams, and the executable graph of a
 * phase is reused (updated in place) when only parameters changed; with
 * HEXFC_OPT_BATCH_LAUNCH 1 the coverage count, the fill and the main resolve
 * pass of all items are instead each one launch over the tiles of every item.
 * The host waits twice per batch instead of twice per frame.
 *   items[i].mesh      mesh handle of ctx
 *   items[i].view, .lens, .style   as for hexfc_set_view / _lens / _style
 *                      (the context's own view, lens and style are unchanged)
 *   items[i].out_rgba  device, height*width*4 float, row-major (as hexfc_render)
 *   stats, item_status host arrays of n, or NULL: per-item statistics and status
 * The context owns one set of frame buffers per item position (grown and
 * reused). Work is ordered after earlier work on `stream`, and later work on
 * `stream` sees the images. Errors: ARG (a NULL output or an invalid view,
 * lens or style), STATE (unknown mesh) before anything runs; OOM, CUDA; the
 * first failing item's status (OVERFLOW, OOM, TIMEOUT) otherwise, the other
 * items drawn.
 */
typedef struct hexfc_batch_item {
    int32_t mesh;
    int32_t pad;
    hexfc_view view;
    hexfc_lens lens;
    hexfc_style style;
    float* out_rgba;
} hexfc_batch_item;

hexfc_status hexfc_render_batch(hexfc_ctx* ctx, int32_t n, const hexfc_batch_item* items,
                                hexfc_frame_stats* stats, hexfc_status* item_status, void* stream);
hexfc_status hexfc_frame_memory(const hexfc_ctx* ctx, uint64_t* bytes);
hexfc_status hexfc_trim(hexfc_ctx* ctx);

/*
 * Per-cell quality from the Jacobian of the cube-to-cell map (Section
 * "Introduction"; Section "Results and Analysis": per-cell scaled Jacobian
 * ratio). metric: HEXFC_METRIC_*; the 8 corners and the cell centre are
 * sampled. out: device, n_cells float. Errors: ARG, STATE (bad mesh), CUDA.
 */
hexfc_status hexfc_cell_quality(hexfc_ctx* ctx, int32_t mesh, int32_t metric, float* out,
                                void* stream);

/*
 * Replace the mesh's per-cell importance with `cell_importance` (device,
 * n_cells float) and recompute the per-vertex and per-edge maxima on the
 * device (Section "Method Overview"). Errors: ARG, STATE, CUDA.
 */
hexfc_status hexfc_set_cell_importance(hexfc_ctx* ctx, int32_t mesh, const float* cell_importance,
                                       void* stream);

/* Number of unique faces / edges of a mesh (for sizing and statistics). */
hexfc_status hexfc_mesh_info(hexfc_ctx* ctx, int32_t mesh, int64_t* n_faces, int64_t* n_edges);

/* Set the camera. Errors: ARG (NULL, width/height outside 1..16384,
 * znear >= zfar, degenerate basis). Draws the whole frame (see
 * hexfc_set_subrect). */
hexfc_status hexfc_set_view(hexfc_ctx* ctx, const hexfc_view* view);

/*
 * Draw only the rectangle [x0, x0 + w) x [y0, y0 + h) of the view's
 * width x height frame: the next frames' outputs are w x h images (row-major,
 * row 0 = frame row y0) equal, bit for bit, to those pixels of the whole frame
 * (vertices are snapped in frame coordinates, then moved by whole pixels; the
 * screen lens is placed in frame pixels). A frame whose fragment lists do not
 * fit the memory budget is drawn in parts this way (Section "Results and
 * Analysis": subdividing the screen and rendering each part separately).
 * (0, 0, 0, 0) selects the whole frame again; hexfc_set_view does too.
 * Errors: ARG (rectangle not inside the frame, w or h < 1), STATE (no view).
 */
hexfc_status hexfc_set_subrect(hexfc_ctx* ctx, int32_t x0, int32_t y0, int32_t w, int32_t h);

/* Set the focus lens (radius > 0). Errors: ARG. */
hexfc_status hexfc_set_lens(hexfc_ctx* ctx, const hexfc_lens* lens);

/* Set the style constants. Errors: ARG (w_base < 0, tf_hi == tf_lo, g_min < 0, g_min > g_max,
 * halo_scale < 0, desat outside [0, 1]). */
hexfc_status hexfc_set_style(hexfc_ctx* ctx, const hexfc_style* style);

/*
 * Render one frame of `mesh` with the current view, lens and style into
 * out_rgba (device, height*width*4 float, row-major, row 0 at the top,
 * straight RGB over the background plus accumulated alpha).
 * Steps, all on `stream`: vertex projection to 16.8 fixed point and 24-bit
 * depth; triangle setup and tile binning; per-pixel fragment count; prefix
 * scan; fragment fill with Eqs. 1-4; per-pixel depth sort and front-to-back
 * composite. The call waits once for the fragment total (to size the buffers);
 * the image is complete when `stream` reaches the end of the call.
 * stats (host, nullable) receives the frame statistics.
 * Errors: ARG, STATE (no view), OOM (the frame's buffers would exceed the
 * budget; stats still filled: fragments tells how far), OVERFLOW (a list longer than HEXFC_MAX_LIST), CUDA, and TIMEOUT or
 * CHECK from the device-side checks of the fill and composite passes: those
 * passes run after the call returns, so hexfc_render reports their failure
 * on the context's next call (hexfc_render_host at the end of its own frame).
 */
hexfc_status hexfc_render(hexfc_ctx* ctx, int32_t mesh, float* out_rgba, hexfc_frame_stats* stats,
                          void* stream);

/* As hexfc_render, with the image in out_rgba_host (host, height*width*4
 * float) when the call returns, and the device-side checks of this frame
 * reported by this call. If out_rgba_host is page-locked memory of the
 * context's device (cudaHostAlloc, cudaHostRegister) and 16-byte aligned, the
 * resolve kernels write the image into it directly through its device
 * mapping; otherwise the image is rendered into a device buffer of the
 * context and copied. On an error the buffer's contents are unspecified. */
hexfc_status hexfc_render_host(hexfc_ctx* ctx, int32_t mesh, float* out_rgba_host,
                               hexfc_frame_stats* stats, void* stream);

/*
 * Parity hook: the fragment lists of the last render for `n` listed pixels
 * (px[i], py[i], host). counts (host, n) receives each list length; keys
 * (host, cap) and rgba (host, cap*4 float) receive the lists concatenated in
 * the order of the pixel list, each sorted ascending by key =
 * (z24 << 32) | (2*face_id + triangle), rgba premultiplied (Eq. 4).
 * keys/rgba may be NULL. Errors: ARG, STATE (no previous render),
 * OVERFLOW (total > cap; counts still filled), CUDA. Synchronous.
 */
hexfc_status hexfc_debug_pixels(hexfc_ctx* ctx, const int32_t* px, const int32_t* py, int64_t n,
                                uint32_t* counts, uint64_t* keys, float* rgba, uint64_t cap);

/* Tuning and test options. */
enum {
    HEXFC_OPT_REVERSE_BIN_ORDER = 1, /* 1: process faces in reverse id order when binning (test hook) */
    HEXFC_OPT_STAGE_TIMING = 2,      /* 1: record CUDA events around every stage of hexfc_render* */
    HEXFC_OPT_DEPTH_BUCKETS = 3,     /* buckets of the per-tile depth order of the triangles: a power of
                                        two in 256..4096 (default 2048), or 0 for no depth order (lists
                                        in the faces' order: a test hook for the sorting passes) */
    HEXFC_OPT_COMPOSITE_WINDOW = 4,  /* sorted window of the per-pixel resolve: 2 (default), 4 or 8; the
                                        image does not depend on it, bit for bit */
    HEXFC_OPT_PREDICTED_CAPACITY = 5, /* 0: count-then-fill (default); 1: capacities from the previous
                                        frame's tile counts; 2: from the capacity network; 3: the previous
                                        frame's total spread evenly over the tiles (the baseline without
                                        any per-tile knowledge). See below. */
    HEXFC_OPT_DEBUG_ERROR_BITS = 6,  /* test hook, bits 0..7: after the last kernel of the next
                                        hexfc_render or hexfc_render_noalloc frame, these bits are set
                                        in the device error word as a kernel of that frame would set
                                        them (4: a bounded wait ran out, 1: a failed check); no wait
                                        runs out and nothing faults. One frame only. */
    HEXFC_OPT_FRAG_BUDGET = 7,       /* bytes: the cap of hexfc_create's frag_budget_bytes, per frame
                                        (0: none); a serving loop sets it to what the other frames in
                                        flight leave */
    HEXFC_OPT_BATCH_LAUNCH = 8       /* hexfc_render_batch: 0 (default): every item its own launches,
                                        the items as parallel branches of each phase's graph; 1: the
                                        coverage count, the fill and the main resolve pass of all items
                                        each one kernel launch over every item's tiles (groups of 64
                                        items). The images do not depend on it, bit for bit */
};
hexfc_status hexfc_set_option(hexfc_ctx* ctx, int32_t option, int64_t value);

/*
 * Complete the context's last frame. With predicted capacities
 * (HEXFC_OPT_PREDICTED_CAPACITY != 0) hexfc_render returns without waiting
 * for its frame, which is verified by the next call on the context (at that
 * call's first host wait, when the frame has completed) or by this one: if the
 * frame needed more room than its chosen capacities and the pool left, it is
 * drawn again exactly (count-then-fill) into its own output with the camera,
 * lens and style it was drawn with, so that no frame keeps an overflow error.
 * A predicted frame's image is final once the next hexfc_render* call or
 * hexfc_finish on its context has returned (and the stream work it issued has
 * run); its output buffer must stay valid until then. Waits for the last
 * frame's stream. stats (host, nullable): the final statistics of the last
 * frame (pending = 0; redrawn = 1 if it was drawn again). Errors: ARG,
 * TIMEOUT/CHECK (device error bits of the verified frame), CUDA. Not in the
 * paper, which sizes its fragment buffer once (Section "GPU Implementation").
 */
hexfc_status hexfc_finish(hexfc_ctx* ctx, hexfc_frame_stats* stats);

/* Final statistics of frame `frame` of the context (its sequence number,
 * hexfc_frame_stats.frame), or of the most recently verified frame if frame
 * is 0, without waiting (host `stats`). After hexfc_render of frame n with
 * predicted capacities returns, frame n-1 is verified. The last 16 frames are
 * kept. Errors: ARG, STATE (that frame is not verified yet or no longer kept). */
hexfc_status hexfc_completed_stats(const hexfc_ctx* ctx, uint64_t frame, hexfc_frame_stats* stats);

/*
 * Predicted capacities (HEXFC_OPT_PREDICTED_CAPACITY != 0; no counterpart in
 * the paper, which sizes its buffers once): the fragment arrays are divided
 * into per-16x16-tile regions of a chosen capacity before the frame,
 * followed by a pool; after the count pass, the fill lays out each tile's
 * lists in the tile's region itself (in the pool if they do not fit), so
 * there is no pixel scan and no host wait between counting and drawing; the
 * host waits once, at the end of the frame. Capacities come from the
 * previous frame's exact tile counts (mode 1: count * 1.15 + 256) or from the
 * capacity network (mode 2, see hexfc_capacity_*); the pool holds 35% of the
 * previous frame's fragments. stats.overflow_tiles counts the tiles above
 * their capacity. Only if the pool runs out is the frame drawn again by the
 * exact count-then-fill path, so the image is always exact. The first frame
 * at a resolution, with no previous counts, is drawn exactly.
 */

/*
 * Tile-capacity network (no counterpart in the paper): per 16x16 tile, a
 * 4 -> 64 -> 64 -> 1 ReLU network predicts y ~ log(1 + fragments) from the
 * tile's previous-frame count, the depth range of its triangles, its screen
 * distance to the lens and the camera's motion since the previous frame;
 * the capacity is expm1(y) * 1.15 + 256. Weights are used in FP16 with FP32
 * sums; training keeps FP32 master weights and Adam moments on the device.
 * Every frame leaves its features and exact tile counts (from the count pass
 * or the fused pass) for training. Parameters: HEXFC_CAPACITY_PARAMS floats,
 * in the order W1 (64 x 4, row-major), b1 (64), W2 (64 x 64, row-major,
 * W2[j][i] from hidden unit i of the first layer to unit j of the second),
 * b2 (64), w3 (64), b3 (1).
 *
 * hexfc_capacity_reset: set weights from seed (scaled normal, biases 0,
 *   b3 = 5) and clear the Adam state. Errors: ARG, OOM, CUDA.
 * hexfc_capacity_set_weights / _get_weights: host array of n ==
 *   HEXFC_CAPACITY_PARAMS floats (set also clears the Adam state).
 *   Errors: ARG (n, non-finite), STATE (get before any weights), CUDA.
 * hexfc_capacity_grad: loss (mean over the n rows of (y - log(1 + count))^2)
 *   and its gradient for host features x (n x 4) and counts (n), with the
 *   current weights (test hook). grad: host, HEXFC_CAPACITY_PARAMS floats.
 *   Errors: ARG, STATE (no weights), OOM, CUDA. Synchronous.
 * hexfc_capacity_train: `steps` Adam steps (rate lr) on the last frame's
 *   features and exact tile counts, on `stream`; *loss (nullable) receives
 *   the loss before the last step (the host waits when loss != NULL).
 *   Errors: ARG, STATE (no weights or no frame yet), OOM, CUDA.
 */
#define HEXFC_CAPACITY_PARAMS 4545
hexfc_status hexfc_capacity_reset(hexfc_ctx* ctx, uint64_t seed);
hexfc_status hexfc_capacity_set_weights(hexfc_ctx* ctx, const float* w, int64_t n);
hexfc_status hexfc_capacity_get_weights(hexfc_ctx* ctx, float* w, int64_t n);
hexfc_status hexfc_capacity_grad(hexfc_ctx* ctx, const float* x, const uint32_t* counts, int64_t n, float* grad,
                                 float* loss);
hexfc_status hexfc_capacity_train(hexfc_ctx* ctx, int32_t steps, float lr, float* loss, void* stream);

/*
 * Accumulated stage times (milliseconds, summed over frames) since the last
 * reset, for frames rendered with HEXFC_OPT_STAGE_TIMING on. ms: host array of
 * HEXFC_N_STAGES doubles; *frames: number of frames summed. Waits for the last
 * timed frame to finish. reset != 0 clears the sums afterwards. Errors: ARG, CUDA.
 */
hexfc_status hexfc_stage_times(hexfc_ctx* ctx, double* ms, uint64_t* frames, int32_t reset);

/* Static string for a status code. Never NULL. */
const char* hexfc_status_string(hexfc_status s);

/*
 * The CUDA runtime error code (cudaError_t) of the last CUDA call or kernel
 * launch of the library that failed on the calling host thread, 0 if none
 * has; a call that returns HEXFC_ERR_CUDA (or HEXFC_ERR_OOM from a failed
 * allocation) sets it. Not reset by later successful calls.
 */
int32_t hexfc_last_cuda_error(void);

/* Static name of a CUDA runtime error code (e.g. "cudaErrorIllegalAddress"). Never NULL. */
const char* hexfc_cuda_error_name(int32_t code);

/*
 * The raster tile of this build, in pixels: 16 x 16 by default, 32 x 8 or
 * 8 x 32 in a library built for those (always 256 pixels). Tiles are the
 * units of binning (Section "GPU Implementation" draws the faces into
 * per-pixel lists; the tiling is this implementation's). width, height: host
 * pointers, each may be NULL.
 */
void hexfc_raster_tile(int32_t* width, int32_t* height);

/* Size of the fixed device scratch array used by hexfc_render_noalloc. */
#define HEXFC_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * hexfc_render without any memory allocation. The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate, for
 * example an application that reserves all device memory for its own
 * allocator or a fixed budget up front, or a frame loop that must not stall
 * on cudaMalloc/cudaFree, which can synchronise the device.
 *
 * Same inputs, output and result as hexfc_render (the same kernels), but every
 * per-frame buffer (projected vertices, face records, tile bins, counts,
 * offsets, fragment lists) is carved from one file-scope device array of
 * HEXFC_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading the library holds
 * until the process exits. The call makes no cudaMalloc, cudaFree or
 * cudaMallocHost; the mesh must already be uploaded, and out_rgba (device,
 * height*width*4 float) is the caller's.
 *
 * - Every call looks up the array's device address on the current device
 *   (ctx's device). The first call on a device loads the library's module
 *   there, which creates the array: make that first call before any stream
 *   capture on that device.
 * - All calls share the one array and it keeps the last call's contents (the
 *   counters that must start at zero are cleared on the stream). Calls whose
 *   work overlaps on the GPU (other streams, other threads, other contexts of
 *   the same process on the same device) race on it: serialise them.
 * - It waits on `stream` twice, like hexfc_render, and returns with the fill
 *   and the composite still running. Their device error bits (a bounded wait
 *   that ran out, a failed exactness check) stay in the array and are
 *   reported, as TIMEOUT or CHECK, by the next hexfc_render_noalloc call on
 *   the same device, as hexfc_render reports its previous frame's.
 * - Stage timing is not recorded and hexfc_debug_pixels keeps referring to the
 *   last hexfc_render* frame.
 * Errors: ARG, STATE (no view or bad mesh), OVERFLOW (the frame needs more
 * than HEXFC_NOALLOC_SCRATCH_BYTES, or a list longer than HEXFC_MAX_LIST;
 * nothing is drawn, stats is filled as far as known), TIMEOUT, CHECK, CUDA.
 */
hexfc_status hexfc_render_noalloc(hexfc_ctx* ctx, int32_t mesh, float* out_rgba, hexfc_frame_stats* stats,
                                  void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HEXFC_H */

// C ABI of the hexfc library: context, resident meshes, camera/lens/style,
// and the per-frame orchestration of the kernels on the caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "hexfc_internal.cuh"
#include "mesh_host.h"

using namespace hexfc;

struct hexfc_ctx {
    int device = 0;
    uint64_t budget = 0;
    std::vector<std::shared_ptr<DevMesh>> meshes;   // resident meshes, possibly shared with other contexts
    bool have_view = false;
    hexfc_view view{};
    CamParams cam{};
    double zref = 1.0;
    hexfc_lens lens{};
    hexfc_style style{};
    FrameBufs fb;
    int reverse_bins = 0;
    int depth_buckets = 2048;   // HEXFC_OPT_DEPTH_BUCKETS
    int window = 2;             // HEXFC_OPT_COMPOSITE_WINDOW
    bool batch_launch = false;  // HEXFC_OPT_BATCH_LAUNCH
    int predicted = 0;          // HEXFC_OPT_PREDICTED_CAPACITY
    int sub_x0 = 0, sub_y0 = 0, sub_w = 0, sub_h = 0;   // hexfc_set_subrect (sub_w 0: the whole frame)
    OutWin last_win{};          // output window of the last frame, in its drawn rectangle
    uint64_t inject_bits = 0;   // HEXFC_OPT_DEBUG_ERROR_BITS: ORed into the error word after the next frame
    // A frame drawn with chosen capacities is verified by the next call on the
    // context (or hexfc_finish), once it has completed: what is needed to draw
    // it again exactly if its capacities ran out, and its device scalars and
    // count statistics, copied into h_pend at its end.
    struct Pending {
        bool active = false;
        std::shared_ptr<DevMesh> mesh;
        float* out = nullptr;
        cudaStream_t stream = nullptr;
        hexfc_view view{};
        CamParams cam{};
        double zref = 1.0;
        hexfc_lens lens{};
        hexfc_style style{};
        hexfc_frame_stats fs{};   // what was known when its call returned
    } pend;
    uint64_t* h_pend = nullptr;        // pinned [kScal + 4 kStatCopies]
    hexfc_frame_stats completed{};     // final statistics of the last verified frame
    hexfc_frame_stats history[16]{};   // final statistics of recent frames, at frame % 16
    uint64_t frame_seq = 0;            // frames drawn by this context
    // exact tile counts of the last frame (fb.tile_frag) are valid for this size
    int counts_W = 0, counts_H = 0;
    uint64_t counts_total = 0;
    // tile-capacity network and the camera of the previous frame (its motion is a feature)
    CapNet cap;
    bool have_prev_cam = false;
    double prev_eye[3] = {0, 0, 0}, prev_F[3] = {0, 0, 1};
    int64_t feat_tiles = 0;   // tiles whose features and exact counts the last frame left for training
    // last render
    bool have_frame = false;
    int last_W = 0, last_H = 0, last_tiles_x = 0, last_tiles_y = 0;
    hexfc_frame_stats last{};
    float* d_out = nullptr;   // image buffer of hexfc_render_host
    int64_t d_out_cap = 0;
    // stage timing: events of the frame in flight, sums over completed frames
    bool timing = false;
    cudaEvent_t ev[2][HEXFC_N_STAGES + 1] = {};   // two frames: the one in flight and the previous one
    bool ev_pending[2] = {false, false};
    int ev_cur = 0;
    double stage_ms[HEXFC_N_STAGES] = {};
    uint64_t timed_frames = 0;
    // batched frames (hexfc_render_batch): buffers and stream per item, an
    // origin stream for the captures, and one executable graph per phase
    struct BatchSlot {
        FrameBufs fb;
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
    };
    std::vector<std::unique_ptr<BatchSlot>> batch;
    cudaStream_t origin = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_p1 = nullptr;   // a single frame's phase 1: bin total copied (FrameJob::p1_done)
    cudaGraphExec_t graph_exec[3] = {nullptr, nullptr, nullptr};
    uint64_t graph_instantiations = 0, graph_updates = 0;
};

namespace {

// The CUDA error of the last failed runtime call or launch made by the library
// on this host thread (hexfc_last_cuda_error).
thread_local int32_t t_last_cuda = 0;

// Record a failed call's error and clear the runtime's (non-sticky) last error.
inline void note_cuda(cudaError_t e)
{
    t_last_cuda = (int32_t)e;
    (void)cudaGetLastError();
}

// Status for the device error bits of scal[5]: a bounded wait that ran out
// (bits 1, 2), else a failed exactness or consistency check (bit 0).
inline hexfc_status device_error_status(uint64_t bits)
{
    return (bits & 6ull) ? HEXFC_ERR_TIMEOUT : HEXFC_ERR_CHECK;
}

// Test hook (HEXFC_OPT_DEBUG_ERROR_BITS): set error bits in the device word
// as a kernel of the frame would, so that the host's reporting of them can be
// tested without making any device wait run out.
__global__ void k_or_error_bits(unsigned long long* word, unsigned long long bits)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(word, bits);
}

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) {                \
            note_cuda(e_);                      \
            return HEXFC_ERR_CUDA;              \
        }                                       \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename T>
hexfc_status dalloc(T** p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        note_cuda(e);
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? HEXFC_ERR_OOM : HEXFC_ERR_CUDA;
    }
    return HEXFC_OK;
}

template <typename T>
void dfree(T*& p)
{
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// Grow a device array to hold at least n elements (contents are not kept).
template <typename T>
hexfc_status ensure(T** p, int64_t* cap, int64_t n)
{
    if (*p && *cap >= n) return HEXFC_OK;
    dfree(*p);
    int64_t want = n + n / 4 + 1024;
    hexfc_status st = dalloc(p, (size_t)want);
    *cap = st == HEXFC_OK ? want : 0;
    return st;
}

void free_mesh(DevMesh* m)
{
    if (!m) return;
    dfree(m->verts); dfree(m->cells); dfree(m->cell_edges); dfree(m->cell_imp);
    dfree(m->vkey); dfree(m->ekey); dfree(m->vimp); dfree(m->eattr); dfree(m->elevel);
    dfree(m->fverts); dfree(m->fedges); dfree(m->fstat); dfree(m->fbound);
    delete m;
}

void free_frame(FrameBufs& f)
{
    dfree(f.vproj); dfree(f.ved); dfree(f.fframe); dfree(f.tzsum);
    dfree(f.tile_cnt); dfree(f.tile_off); dfree(f.tile_cur); dfree(f.tile_order); dfree(f.tile_frag); dfree(f.tile_cap); dfree(f.cap_off); dfree(f.tile_zr); dfree(f.cap_x);
    dfree(f.bins); dfree(f.bins_tmp); dfree(f.masks); dfree(f.seg); dfree(f.cnt);
    dfree(f.off); dfree(f.zsil);
    dfree(f.part); dfree(f.part_max); dfree(f.long_q); dfree(f.fix_q); dfree(f.key); dfree(f.rgba); dfree(f.scal);
    dfree(f.cstat);
    if (f.h_scal) cudaFreeHost(f.h_scal);
    f = FrameBufs{};
}

DevMesh* get_mesh(hexfc_ctx* ctx, int32_t id)
{
    if (!ctx || id < 0 || id >= (int32_t)ctx->meshes.size()) return nullptr;
    return ctx->meshes[(size_t)id].get();
}

// Stage events: record boundary k of the current frame (no-op without timing).
void mark(hexfc_ctx* ctx, int k, cudaStream_t s)
{
    if (ctx->timing) cudaEventRecord(ctx->ev[ctx->ev_cur][k], s);
}

// Add the stage times of event set `set` if it holds a recorded frame.
void collect_set(hexfc_ctx* ctx, int set)
{
    if (!ctx->ev_pending[set]) return;
    ctx->ev_pending[set] = false;
    if (cudaEventSynchronize(ctx->ev[set][HEXFC_N_STAGES]) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    for (int k = 0; k < HEXFC_N_STAGES; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev[set][k], ctx->ev[set][k + 1]) == cudaSuccess) ctx->stage_ms[k] += ms;
        else (void)cudaGetLastError();
    }
    ++ctx->timed_frames;
}

// The previous frame's events are complete once the stream has passed any later point.
void collect(hexfc_ctx* ctx) { collect_set(ctx, ctx->ev_cur ^ 1); }

// Camera basis and projection constants, evaluated in double in a fixed order
// (the host compiler is run without floating-point contraction).
bool make_camera(const hexfc_view* v, CamParams& c, double& zref)
{
    double f[3] = {v->target[0] - v->eye[0], v->target[1] - v->eye[1], v->target[2] - v->eye[2]};
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0.0)) return false;
    for (int d = 0; d < 3; ++d) c.F[d] = f[d] / fl;
    double r[3] = {c.F[1] * v->up[2] - c.F[2] * v->up[1], c.F[2] * v->up[0] - c.F[0] * v->up[2],
                   c.F[0] * v->up[1] - c.F[1] * v->up[0]};
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rl > 0.0)) return false;
    for (int d = 0; d < 3; ++d) c.R[d] = r[d] / rl;
    c.U[0] = c.R[1] * c.F[2] - c.R[2] * c.F[1];
    c.U[1] = c.R[2] * c.F[0] - c.R[0] * c.F[2];
    c.U[2] = c.R[0] * c.F[1] - c.R[1] * c.F[0];
    for (int d = 0; d < 3; ++d) c.eye[d] = v->eye[d];
    c.W = v->width;
    c.H = v->height;
    c.cx = (double)v->width * 0.5;
    c.cy = (double)v->height * 0.5;
    c.znear = v->znear;
    c.zfar = v->zfar;
    c.ortho = !(v->fovy_deg > 0.0);
    if (c.ortho) {
        if (!(v->ortho_half_h > 0.0)) return false;
        c.scale = ((double)v->height * 0.5) / v->ortho_half_h;
        c.focal = 0.0;
    } else {
        if (!(v->fovy_deg < 180.0)) return false;
        c.focal = ((double)v->height * 0.5) / std::tan(v->fovy_deg * (3.14159265358979323846 / 180.0) * 0.5);
        c.scale = 0.0;
    }
    c.zf_over = v->zfar / (v->zfar - v->znear);
    zref = fl;
    return true;
}

ShadeParams make_shade_params(const hexfc_lens& lens, const hexfc_style& s, double zref, int ortho)
{
    ShadeParams sp{};
    sp.lens_mode = lens.mode;
    for (int d = 0; d < 3; ++d) sp.lens_c[d] = (float)lens.center[d];
    sp.lens_inv_r = (float)(1.0 / lens.radius);
    sp.w_base = s.w_base;
    sp.lod = s.lod;
    sp.delta = s.delta;
    sp.s = s.s;
    sp.alpha_min = s.alpha_min;
    sp.alpha_span = s.alpha_max - s.alpha_min;
    sp.tf_lo = s.tf_lo;
    sp.tf_inv = (float)(1.0 / ((double)s.tf_hi - (double)s.tf_lo));
    for (int d = 0; d < 3; ++d) sp.bg[d] = s.bg[d];
    sp.accent_beta = s.accent_beta;
    sp.halo_scale = s.halo_scale;
    sp.darken = s.darken;
    sp.g_min = s.g_min;
    sp.g_max = s.g_max;
    sp.zref = (float)zref;
    sp.ortho = ortho;
    sp.desat = s.desat;
    const float acc = 256.f * (2.f / 3.f) * s.w_base;
    sp.accent_r2 = acc * acc;
    return sp;
}

ShadeParams make_shade(const hexfc_ctx* ctx)
{
    ShadeParams sp = make_shade_params(ctx->lens, ctx->style, ctx->zref, ctx->cam.ortho);
    sp.px_off = ctx->cam.ox;
    sp.py_off = ctx->cam.oy;
    return sp;
}

// Size of the output image (the whole frame unless hexfc_set_subrect chose a
// rectangle of it).
inline int draw_w(const hexfc_ctx* ctx) { return ctx->sub_w ? ctx->sub_w : ctx->view.width; }
inline int draw_h(const hexfc_ctx* ctx) { return ctx->sub_w ? ctx->sub_h : ctx->view.height; }

// A sub-rectangle is drawn with an apron of one pixel (inside the frame): the
// silhouettes of its border pixels read their neighbours' depths, as in the
// whole frame. The camera's rectangle (cam.ox, cam.oy, cam.W, cam.H) is the
// one drawn; the window selects the output pixels in it.
OutWin output_window(const hexfc_ctx* ctx)
{
    return OutWin{ctx->sub_x0 - ctx->cam.ox, ctx->sub_y0 - ctx->cam.oy, draw_w(ctx), draw_h(ctx)};
}

bool valid_view(const hexfc_view* v, CamParams& c, double& zref)
{
    if (v->width < 1 || v->height < 1 || v->width > 16384 || v->height > 16384) return false;
    if (!(v->znear < v->zfar) || !std::isfinite(v->znear) || !std::isfinite(v->zfar)) return false;
    if (!(v->fovy_deg >= 0.0)) return false;
    c.ox = c.oy = 0;
    return make_camera(v, c, zref);
}

bool valid_lens(const hexfc_lens* l)
{
    if (l->mode != HEXFC_LENS_SCREEN && l->mode != HEXFC_LENS_SPHERE) return false;
    return l->radius > 0.0 && std::isfinite(l->radius);
}

bool valid_style(const hexfc_style* s)
{
    if (!(s->w_base >= 0.f) || s->tf_hi == s->tf_lo || !(s->g_min >= 0.f) || !(s->g_min <= s->g_max)) return false;
    if (!(s->halo_scale >= 0.f)) return false;
    if (!(s->sil_alpha >= 0.f && s->sil_alpha <= 1.f) || !(s->sil_threshold >= 0.f)) return false;
    return s->desat >= 0.f && s->desat <= 1.f;
}

// One frame: its mesh, camera and style constants, its buffers, and what the
// host learns between the three phases. Phase 1 (geometry: vertices, face
// records, per-tile triangle counts and their scan) ends with the bin total;
// phase 2 (binning, depth order, tile order, coverage count, pixel scan) ends
// with the fragment total; phase 3 draws (fill and composite). The host reads
// the totals between phases to size the next phase's buffers.
struct FrameJob {
    FrameBufs* fb = nullptr;
    DevMesh* m = nullptr;
    CamParams cam{};
    ShadeParams sp{};
    int lod = 0;
    float delta = 0.f;
    int W = 0, H = 0, tiles_x = 0, tiles_y = 0;
    int64_t n_tiles = 0, n_pix = 0;
    int reverse = 0;
    int buckets = 2048, window = 2;
    float lens_x = 0.f, lens_y = 0.f, inv_diag = 0.f, motion = 0.f;   // capacity-network features
    bool prev_counts = false;   // fb.tile_frag holds the previous frame's counts for this tile grid
    uint64_t budget = 0;
    float* out = nullptr;
    OutWin win{};                  // output pixels of the drawn rectangle (the rest: the apron)
    float sil_alpha = 0.f, sil_threshold = 0.f;   // silhouettes (off at alpha 0)
    int frame_w = 0, frame_h = 0;  // the view's frame, which the drawn rectangle is a part of
    hexfc_ctx* timing = nullptr;   // stage events of the single-frame path
    // single-frame path: phase 1 records this event once its bin total is on the
    // way to the host and then orders the tiles (which needs only the tile
    // offsets), so that the tile order runs while the host waits and allocates
    cudaEvent_t p1_done = nullptr;
    bool order_done = false;
    uint32_t launches = 0;
    uint64_t n_bins = 0, total = 0;
    uint32_t max_list = 0, n_long = 0;
    hexfc_frame_stats fs{};
};

void job_mark(const FrameJob& j, int k, cudaStream_t s)
{
    if (j.timing) mark(j.timing, k, s);
}

// Per-frame constants of the capacity features: the lens centre on screen,
// 1 / screen diagonal, and the camera's motion since the previous frame
// (eye displacement / reference depth + angle between view directions).
void feature_constants(const hexfc_ctx* ctx, const hexfc_view& v, const hexfc_lens& lens, const CamParams& c,
                       double zref, FrameJob& j)
{
    double lx = lens.center[0], ly = lens.center[1];
    if (lens.mode == HEXFC_LENS_SPHERE) {
        const double dx = lens.center[0] - c.eye[0], dy = lens.center[1] - c.eye[1], dz = lens.center[2] - c.eye[2];
        const double ex = dx * c.R[0] + dy * c.R[1] + dz * c.R[2], ey = dx * c.U[0] + dy * c.U[1] + dz * c.U[2];
        const double ed = dx * c.F[0] + dy * c.F[1] + dz * c.F[2];
        if (c.ortho) {
            lx = c.cx + ex * c.scale;
            ly = c.cy - ey * c.scale;
        } else if (ed > c.znear) {
            lx = c.cx + ex / ed * c.focal;
            ly = c.cy - ey / ed * c.focal;
        } else {
            lx = ly = 1e9;   // behind the camera: far from every tile
        }
    }
    j.lens_x = (float)(lx - c.ox);   // tiles are placed in the drawn rectangle
    j.lens_y = (float)(ly - c.oy);
    j.inv_diag = (float)(1.0 / std::sqrt((double)v.width * v.width + (double)v.height * v.height));
    double motion = 0.0;
    if (ctx->have_prev_cam) {
        double d2 = 0.0, dot = 0.0;
        for (int k = 0; k < 3; ++k) {
            d2 += (c.eye[k] - ctx->prev_eye[k]) * (c.eye[k] - ctx->prev_eye[k]);
            dot += c.F[k] * ctx->prev_F[k];
        }
        motion = std::sqrt(d2) / (zref > 0 ? zref : 1.0) + std::acos(std::fmin(1.0, std::fmax(-1.0, dot)));
    }
    j.motion = (float)motion;
}

void remember_camera(hexfc_ctx* ctx, const CamParams& c)
{
    for (int k = 0; k < 3; ++k) {
        ctx->prev_eye[k] = c.eye[k];
        ctx->prev_F[k] = c.F[k];
    }
    ctx->have_prev_cam = true;
}

FrameJob make_job(hexfc_ctx* ctx, FrameBufs* fb, DevMesh* m, float* out)
{
    FrameJob j;
    j.fb = fb;
    j.m = m;
    j.cam = ctx->cam;
    j.sp = make_shade(ctx);
    j.lod = ctx->style.lod;
    j.delta = ctx->style.delta;
    j.W = ctx->cam.W;   // the drawn rectangle (the frame, or a sub-rectangle and its apron)
    j.H = ctx->cam.H;
    j.win = output_window(ctx);
    j.sil_alpha = ctx->style.sil_alpha;
    j.sil_threshold = ctx->style.sil_threshold;
    j.frame_w = ctx->view.width;
    j.frame_h = ctx->view.height;
    j.tiles_x = (j.W + kTileW - 1) / kTileW;
    j.tiles_y = (j.H + kTileH - 1) / kTileH;
    j.n_tiles = (int64_t)j.tiles_x * j.tiles_y;
    j.n_pix = j.n_tiles * kTilePix;
    j.reverse = ctx->reverse_bins;
    j.buckets = ctx->depth_buckets;
    j.window = ctx->window;
    j.budget = ctx->budget;
    j.out = out;
    feature_constants(ctx, ctx->view, ctx->lens, ctx->cam, ctx->zref, j);
    j.prev_counts = fb == &ctx->fb && ctx->counts_W == j.W && ctx->counts_H == j.H;
    return j;
}

// Capacity features of the frame (before its count overwrites the previous counts).
hexfc_status job_features(FrameJob& j, cudaStream_t s)
{
    FrameBufs& fb = *j.fb;
    if (!j.prev_counts) CK(cudaMemsetAsync(fb.tile_frag, 0, sizeof(uint32_t) * (size_t)j.n_tiles, s));
    CK(launch_cap_features(fb, j.n_tiles, j.tiles_x, j.lens_x, j.lens_y, j.inv_diag, j.motion, s));
    j.launches += 1;
    return HEXFC_OK;
}

// Buffers whose size follows from the mesh and the view.
hexfc_status job_alloc(FrameJob& j)
{
    FrameBufs& fb = *j.fb;
    const DevMesh* m = j.m;
    hexfc_status st;
    if (!fb.vproj || fb.v_cap < m->n_verts) {
        int64_t c1 = 0;
        dfree(fb.ved);
        if ((st = ensure(&fb.vproj, &fb.v_cap, m->n_verts)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.ved, &c1, fb.v_cap)) != HEXFC_OK) return st;
    }
    if (!fb.fframe || fb.f_cap < m->n_faces) {
        int64_t c1 = 0;
        dfree(fb.tzsum);
        if ((st = ensure(&fb.fframe, &fb.f_cap, m->n_faces)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.tzsum, &c1, 2 * fb.f_cap)) != HEXFC_OK) return st;
    }
    if (!fb.tile_cnt || fb.t_cap < j.n_tiles + 1) {
        int64_t c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0, c6 = 0;
        dfree(fb.tile_off); dfree(fb.tile_cur); dfree(fb.tile_order); dfree(fb.tile_frag); dfree(fb.tile_zr);
        dfree(fb.cap_x);
        if ((st = ensure(&fb.tile_cnt, &fb.t_cap, j.n_tiles + 1)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.tile_off, &c1, fb.t_cap)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.tile_cur, &c2, fb.t_cap)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.tile_order, &c3, fb.t_cap)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.tile_frag, &c4, fb.t_cap)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.tile_zr, &c5, fb.t_cap)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.cap_x, &c6, 4 * fb.t_cap)) != HEXFC_OK) return st;
    }
    if (!fb.cnt || fb.p_cap < j.n_pix + 1) {
        int64_t c1 = 0, c2 = 0, c3 = 0;
        dfree(fb.off); dfree(fb.long_q); dfree(fb.fix_q); dfree(fb.zsil);
        if ((st = ensure(&fb.cnt, &fb.p_cap, j.n_pix + 1)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.off, &c1, fb.p_cap)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.long_q, &c2, fb.p_cap)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.fix_q, &c3, fb.p_cap)) != HEXFC_OK) return st;
        int64_t c4 = 0;
        if ((st = ensure(&fb.zsil, &c4, fb.p_cap)) != HEXFC_OK) return st;
    }
    const int64_t nparts = scan_partials_needed(std::max<int64_t>(j.n_pix, j.n_tiles)) + 1;
    if (!fb.part || fb.part_cap < 2 * nparts) {
        int64_t c1 = 0;
        dfree(fb.part_max);
        if ((st = ensure(&fb.part, &fb.part_cap, 2 * nparts)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.part_max, &c1, fb.part_cap)) != HEXFC_OK) return st;
    }
    if (!fb.scal) {
        if ((st = dalloc(&fb.scal, kScal)) != HEXFC_OK) return st;
        CK(cudaMallocHost((void**)&fb.h_scal, kScal * sizeof(uint64_t)));
        fb.scal_fresh = true;   // contents undefined: phase 1 clears all of it
    }
    return HEXFC_OK;
}

hexfc_status job_phase1(FrameJob& j, cudaStream_t s)
{
    FrameBufs& fb = *j.fb;
    job_mark(j, 0, s);
    CK(cudaMemsetAsync(fb.tile_cnt, 0, sizeof(uint32_t) * (size_t)j.n_tiles, s));
    CK(cudaMemsetAsync(fb.tile_cur, 0, sizeof(uint32_t) * (size_t)j.n_tiles, s));
    // scal[5] (device error bits) is kept across frames so that errors of the
    // last passes of a frame are reported by the next call (hexfc_render_host
    // reads them at the end of its own frame)
    if (fb.scal_fresh) {
        CK(cudaMemsetAsync(fb.scal, 0, sizeof(uint64_t) * kScal, s));
        fb.scal_fresh = false;
    } else {
        CK(cudaMemsetAsync(fb.scal, 0, sizeof(uint64_t) * 5, s));
        CK(cudaMemsetAsync(fb.scal + 6, 0, sizeof(uint64_t) * (kScal - 6), s));
    }
    CK(launch_vertex_setup(*j.m, j.cam, fb, s));
    job_mark(j, 1, s);
    CK(launch_face_setup(*j.m, j.cam, j.lod, j.delta, fb, j.tiles_x, j.tiles_y, s));
    job_mark(j, 2, s);
    CK(scan_u32_to_u64(fb.tile_cnt, fb.tile_off, j.n_tiles, fb.part, fb.part_max, fb.scal + 8, 0xFFFFFFFFu, s,
                       (uint32_t)kChunk));
    job_mark(j, 3, s);
    j.launches = 5;
    CK(cudaMemcpyAsync(fb.h_scal + 8, fb.scal + 8, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    j.order_done = false;
    if (j.p1_done) {
        CK(cudaEventRecord(j.p1_done, s));
        CK(launch_tile_order(fb, j.n_tiles, s));
        j.order_done = true;
        j.launches += 1;
    }
    return HEXFC_OK;
}

// The host's wait for phase 1: for its bin total only (the tile order may
// still run), unless a pending frame is to be verified and perhaps drawn again
// in the same buffers first.
hexfc_status job_wait1(const hexfc_ctx* ctx, const FrameJob& j, cudaStream_t s)
{
    if (j.p1_done && !ctx->pend.active) CK(cudaEventSynchronize(j.p1_done));
    else CK(cudaStreamSynchronize(s));
    return HEXFC_OK;
}

// After phase 1 has completed: bins and masks for the bin total.
hexfc_status job_read1(FrameJob& j)
{
    FrameBufs& fb = *j.fb;
    hexfc_status st;
    j.n_bins = fb.h_scal[8];   // padded to whole chunks per tile
    if (!fb.bins || fb.bin_cap < (int64_t)j.n_bins) {
        int64_t c1 = 0;
        dfree(fb.bins_tmp);
        if ((st = ensure(&fb.bins, &fb.bin_cap, (int64_t)j.n_bins)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.bins_tmp, &c1, fb.bin_cap)) != HEXFC_OK) return st;
    }
    if ((st = ensure(&fb.masks, &fb.mask_cap, (int64_t)j.n_bins * (kTilePix / kChunk))) != HEXFC_OK) return st;
    if ((st = ensure(&fb.seg, &fb.seg_cap, (int64_t)(j.n_bins / kChunk) * (kTilePix / 32))) != HEXFC_OK) return st;
    return HEXFC_OK;
}

// Phase 2 up to the count: the bins in depth order, the tile order, the capacity features.
hexfc_status job_phase2_bins(FrameJob& j, cudaStream_t s)
{
    FrameBufs& fb = *j.fb;
    job_mark(j, 4, s);
    CK(cudaMemsetAsync(fb.bins, 0xFF, sizeof(uint32_t) * (size_t)j.n_bins, s));   // padding slots = kPadBin
    CK(launch_bin_fill(*j.m, fb, j.tiles_x, j.W, j.H, j.reverse, s));
    CK(launch_bin_sort(*j.m, fb, j.tiles_x, j.tiles_y, j.buckets, s));
    if (!j.order_done) {
        CK(launch_tile_order(fb, j.n_tiles, s));
        j.launches += 1;
    }
    j.launches += 2;
    hexfc_status fst = job_features(j, s);
    if (fst != HEXFC_OK) return fst;
    job_mark(j, 5, s);
    return HEXFC_OK;
}

// Phase 2 after the count: the pixel scan, its totals to the host.
hexfc_status job_phase2_scan(FrameJob& j, cudaStream_t s)
{
    FrameBufs& fb = *j.fb;
    job_mark(j, 6, s);
    CK(scan_u32_to_u64(fb.cnt, fb.off, j.n_pix, fb.part, fb.part_max, fb.scal, (uint32_t)kWarpSortMax, s));
    job_mark(j, 7, s);
    j.launches += 4;   // the count and the three scan passes
    CK(cudaMemcpyAsync(fb.h_scal, fb.scal, 6 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    return HEXFC_OK;
}

hexfc_status job_phase2(FrameJob& j, cudaStream_t s)
{
    hexfc_status st;
    if ((st = job_phase2_bins(j, s)) != HEXFC_OK) return st;
    CK(launch_count(*j.m, *j.fb, j.tiles_x, j.tiles_y, j.W, j.H, false, s));
    return job_phase2_scan(j, s);
}

// After phase 2 has completed: device error bits, totals, limits, fragment buffers.
// Device memory of a context's frame buffers, with fragment arrays of `frags` records.
uint64_t frame_bytes(const FrameBufs& f, int64_t frags)
{
    uint64_t b = 0;
    b += (uint64_t)f.v_cap * (sizeof(int4) + sizeof(float));
    b += (uint64_t)f.f_cap * (sizeof(FaceFrame) + 2 * sizeof(uint32_t));
    b += (uint64_t)f.t_cap * (9 * sizeof(uint32_t) + sizeof(uint64_t) + sizeof(uint32_t));
    b += (uint64_t)f.bin_cap * 2 * sizeof(uint32_t) + (uint64_t)f.mask_cap * sizeof(uint32_t) +
         (uint64_t)f.seg_cap * sizeof(uint64_t);
    b += (uint64_t)f.p_cap * (4 * sizeof(uint32_t) + sizeof(uint64_t));
    b += (uint64_t)f.part_cap * (sizeof(uint64_t) + sizeof(uint32_t));
    b += (uint64_t)frags * (sizeof(uint64_t) + sizeof(float4));
    return b;
}

hexfc_status job_read2(FrameJob& j, cudaStream_t s)
{
    FrameBufs& fb = *j.fb;
    hexfc_status st;
    if (fb.h_scal[5] != 0) {  // a bounded device wait ran out, or an exactness check failed
        const uint64_t bits = fb.h_scal[5];
        CK(cudaMemsetAsync(fb.scal + 5, 0, sizeof(uint64_t), s));
        return device_error_status(bits);
    }
    j.total = fb.h_scal[0];
    j.max_list = (uint32_t)fb.h_scal[1];
    j.n_long = (uint32_t)fb.h_scal[2];
    hexfc_frame_stats& fs = j.fs;
    fs = hexfc_frame_stats{};
    fs.fragments = j.total;
    fs.bin_entries = j.n_bins;
    fs.max_list = j.max_list;
    fs.long_lists = j.n_long;
    fs.width = (uint32_t)j.W;
    fs.height = (uint32_t)j.H;
    fs.kernel_launches = j.launches;
    if (j.max_list > HEXFC_MAX_LIST) return HEXFC_ERR_OVERFLOW;
    if (!fb.key || fb.frag_cap < (int64_t)j.total) {
        // the fragment arrays must grow: with a budget, the frame's buffers once
        // they hold it must fit (refused before anything grows), and their
        // headroom is what the budget leaves
        int64_t want = (int64_t)j.total + (int64_t)j.total / 4 + 1024;
        if (j.budget) {
            const uint64_t per = sizeof(uint64_t) + sizeof(float4);
            const uint64_t base = frame_bytes(fb, 0);
            if (base + j.total * per > j.budget) return HEXFC_ERR_OOM;
            want = std::min<int64_t>(want, (int64_t)((j.budget - base) / per));
        }
        dfree(fb.key);
        dfree(fb.rgba);
        fb.frag_cap = 0;
        if ((st = dalloc(&fb.key, (size_t)want)) != HEXFC_OK) return st;
        if ((st = dalloc(&fb.rgba, (size_t)want)) != HEXFC_OK) return st;
        fb.frag_cap = want;
    }
    return HEXFC_OK;
}

// With silhouettes: the depth image of the boundary surface starts empty.
hexfc_status job_sil_clear(const FrameJob& j, cudaStream_t s)
{
    if (j.sil_alpha > 0.f) CK(cudaMemsetAsync(j.fb->zsil, 0xFF, sizeof(uint32_t) * (size_t)j.n_pix, s));
    return HEXFC_OK;
}

// After the composite: the white silhouettes over the output window.
hexfc_status job_silhouette(FrameJob& j, float* out, cudaStream_t s)
{
    if (j.sil_alpha <= 0.f) return HEXFC_OK;
    CK(launch_silhouette(*j.fb, j.tiles_x, j.cam.ox, j.cam.oy, j.frame_w, j.frame_h, j.sil_alpha, j.sil_threshold,
                         out, j.win, s));
    j.launches += 2;
    return HEXFC_OK;
}

hexfc_status job_phase3(FrameJob& j, cudaStream_t s)
{
    FrameBufs& fb = *j.fb;
    job_mark(j, 8, s);
    hexfc_status st;
    if ((st = job_sil_clear(j, s)) != HEXFC_OK) return st;
    CK(launch_fill(*j.m, fb, j.sp, j.tiles_x, j.tiles_y, j.W, j.H, false, j.sil_alpha > 0.f, s));
    job_mark(j, 9, s);
    CK(launch_composite(fb, j.sp, j.tiles_x, j.tiles_y, j.W, j.H, j.out, j.n_long, j.window, j.win, s));
    if ((st = job_silhouette(j, j.out, s)) != HEXFC_OK) return st;
    job_mark(j, 10, s);
    j.launches += 3 + (j.n_long > 0 ? 1 : 0);
    j.fs.kernel_launches = j.launches;
    return HEXFC_OK;
}

// A frame's entries in the batched count, fill and main resolve launches.
CountItem count_item(const FrameJob& j)
{
    const FrameBufs& fb = *j.fb;
    return CountItem{fb.tile_off, fb.bins, fb.fframe, fb.tile_order, fb.cnt, fb.masks, fb.tile_frag,
                     j.tiles_x,   j.W,     j.H};
}

FillItem fill_item(const FrameJob& j)
{
    const FrameBufs& fb = *j.fb;
    FillItem it{};
    it.tile_off = fb.tile_off;
    it.bins = fb.bins;
    it.masks = fb.masks;
    it.fframe = fb.fframe;
    it.fstat = j.m->fstat;
    it.order = fb.tile_order;
    it.off = fb.off;
    it.cnt = fb.cnt;
    it.key = fb.key;
    it.rgba = fb.rgba;
    it.seg = fb.seg;
    it.err = reinterpret_cast<unsigned long long*>(fb.scal + 5);
    it.zsil = j.sil_alpha > 0.f ? fb.zsil : nullptr;
    it.sp = j.sp;
    it.tiles_x = j.tiles_x;
    it.W = j.W;
    it.H = j.H;
    return it;
}

CompositeItem composite_item(const FrameJob& j)
{
    const FrameBufs& fb = *j.fb;
    CompositeItem it{};
    it.cnt = fb.cnt;
    it.seg = fb.seg;
    it.tile_off = fb.tile_off;
    it.masks = fb.masks;
    it.key = fb.key;
    it.rgba = fb.rgba;
    it.out = reinterpret_cast<float4*>(j.out);
    it.long_q = fb.long_q;
    it.long_cursor = reinterpret_cast<unsigned long long*>(fb.scal + 3);
    it.fix_q = fb.fix_q;
    it.fix_cursor = reinterpret_cast<unsigned long long*>(fb.scal + 4);
    it.frag_cap = (uint64_t)fb.frag_cap;
    for (int c = 0; c < 3; ++c) it.bg[c] = j.sp.bg[c];
    it.win = j.win;
    it.tiles_x = j.tiles_x;
    it.W = j.W;
    it.H = j.H;
    return it;
}

// One batched launch per group of at most kBatchLaunchMax frames: `add` puts
// frame i in the batch, `go` launches it.
template <typename B, typename Add, typename Go>
hexfc_status batched(B& b, const std::vector<int>& items, Add&& add, Go&& go)
{
    b.n = 0;
    b.tile_begin[0] = 0;
    for (size_t k = 0; k < items.size(); ++k) {
        add(b, items[k]);   // sets b.it[b.n] and b.tile_begin[b.n + 1], advances b.n
        if (b.n == kBatchLaunchMax || k + 1 == items.size()) {
            CK(go(b));
            b.n = 0;
        }
    }
    return HEXFC_OK;
}

inline uint64_t* fb_of(FrameJob& j) { return j.fb->scal; }

hexfc_status settle_pending(hexfc_ctx* ctx, cudaStream_t s, bool* redrawn);

// A frame's final statistics: the latest verified, and kept by sequence number.
inline void record_final(hexfc_ctx* ctx, const hexfc_frame_stats& fs)
{
    ctx->completed = fs;
    ctx->history[fs.frame % 16] = fs;
}

// HEXFC_OPT_DEBUG_ERROR_BITS: after the frame's last kernel, set the requested
// bits in the device error word (one frame only).
hexfc_status inject_error_bits(hexfc_ctx* ctx, uint64_t* scal, cudaStream_t s)
{
    if (!ctx->inject_bits) return HEXFC_OK;
    k_or_error_bits<<<1, 32, 0, s>>>(reinterpret_cast<unsigned long long*>(scal + 5),
                                     (unsigned long long)ctx->inject_bits);
    ctx->inject_bits = 0;
    CK(cudaGetLastError());
    return HEXFC_OK;
}

// Bins, counts, scan, fill and composite of one frame (everything but the output copy).
hexfc_status render_frame(hexfc_ctx* ctx, DevMesh* m, float* out, hexfc_frame_stats* stats, cudaStream_t s)
{
    FrameJob j = make_job(ctx, &ctx->fb, m, out);
    hexfc_status st;
    if ((st = job_alloc(j)) != HEXFC_OK) return st;
    if (ctx->timing && !ctx->ev[0][0])
        for (auto& set : ctx->ev)
            for (auto& e : set) CK(cudaEventCreate(&e));
    ctx->ev_cur ^= 1;
    j.timing = ctx;
    if (!ctx->ev_p1) CK(cudaEventCreateWithFlags(&ctx->ev_p1, cudaEventDisableTiming));
    j.p1_done = ctx->ev_p1;
    if ((st = job_phase1(j, s)) != HEXFC_OK) return st;
    if ((st = job_wait1(ctx, j, s)) != HEXFC_OK) return st;
    collect(ctx);
    if (ctx->pend.active) {   // the previous frame (chosen capacities) has completed: verify it
        bool redrawn = false;
        if ((st = settle_pending(ctx, s, &redrawn)) != HEXFC_OK) return st;
        if (redrawn) {   // it was drawn again in these buffers: this frame's first passes once more
            if ((st = job_phase1(j, s)) != HEXFC_OK) return st;
            if ((st = job_wait1(ctx, j, s)) != HEXFC_OK) return st;
        }
    }
    if ((st = job_read1(j)) != HEXFC_OK) return st;
    if ((st = job_phase2(j, s)) != HEXFC_OK) return st;
    CK(cudaStreamSynchronize(s));
    ctx->have_frame = false;
    st = job_read2(j, s);
    j.fs.frame = ++ctx->frame_seq;
    ctx->last = j.fs;
    if (stats) *stats = j.fs;
    if (st != HEXFC_OK) return st;
    record_final(ctx, j.fs);
    if ((st = job_phase3(j, s)) != HEXFC_OK) return st;
    if ((st = inject_error_bits(ctx, fb_of(j), s)) != HEXFC_OK) return st;
    ctx->ev_pending[ctx->ev_cur] = ctx->timing;
    ctx->last.kernel_launches = j.launches;
    if (stats) stats->kernel_launches = j.launches;
    ctx->have_frame = true;
    ctx->last_W = j.W;
    ctx->last_win = j.win;
    ctx->last_H = j.H;
    ctx->last_tiles_x = j.tiles_x;
    ctx->last_tiles_y = j.tiles_y;
    ctx->counts_W = j.W;   // k_count left the exact tile counts in fb.tile_frag
    ctx->counts_H = j.H;
    ctx->counts_total = j.total;
    ctx->feat_tiles = j.n_tiles;
    remember_camera(ctx, j.cam);
    return HEXFC_OK;
}

constexpr float kCapMargin = 0.15f;   // capacity = predicted count * (1 + margin) + pad
constexpr uint32_t kCapPad = 256;
constexpr double kCapPool = 0.35;        // pool after the regions, in previous-frame fragments
constexpr uint64_t kErrPoolBit = 16;     // device error bit: no room for a tile's lists in the pool
constexpr uint32_t kLongListsUnknown = 1u << 30;   // the long-list pass reads the queue length on the device

// A frame with chosen tile capacities: capacities from the previous frame's
// exact tile counts or from the capacity network, the count pass, then the fill
// lays out each tile's lists in the tile's region (or the pool) itself, so
// there is no pixel scan and no host wait after the count; and the call does
// not wait at the end either. The frame is verified by the next call on the
// context, at that call's first host wait (it has completed by then), or by
// hexfc_finish: if its capacities ran out, it is drawn again exactly by
// count-then-fill into its own output, before anything else.
hexfc_status render_frame_predicted(hexfc_ctx* ctx, DevMesh* m, float* out, hexfc_frame_stats* stats,
                                    cudaStream_t s)
{
    if (ctx->predicted == 2 && !ctx->cap.ready) return HEXFC_ERR_STATE;   // no network weights
    // previous-frame capacities need the tile counts of a frame of this size; the
    // network (that feature is then 0) and the uniform capacity need only some
    // earlier frame, for the size of the pool
    const bool same_size = ctx->counts_W == draw_w(ctx) && ctx->counts_H == draw_h(ctx);
    if (ctx->counts_W == 0 || (ctx->predicted == 1 && !same_size))
        return render_frame(ctx, m, out, stats, s);
    FrameJob j = make_job(ctx, &ctx->fb, m, out);
    FrameBufs& fb = ctx->fb;
    hexfc_status st;
    if ((st = job_alloc(j)) != HEXFC_OK) return st;
    if (!fb.tile_cap || fb.cap_cap < fb.t_cap) {   // capacity arrays follow the tile arrays
        int64_t c1 = 0;
        dfree(fb.cap_off);
        if ((st = ensure(&fb.tile_cap, &fb.cap_cap, fb.t_cap)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.cap_off, &c1, fb.cap_cap)) != HEXFC_OK) return st;
    }
    if (!fb.cstat && (st = dalloc(&fb.cstat, 4 * kStatCopies)) != HEXFC_OK) return st;
    if (!ctx->h_pend) CK(cudaMallocHost((void**)&ctx->h_pend, (kScal + 4 * kStatCopies) * sizeof(uint64_t)));
    if (ctx->timing && !ctx->ev[0][0])
        for (auto& set : ctx->ev)
            for (auto& e : set) CK(cudaEventCreate(&e));
    ctx->ev_cur ^= 1;
    j.timing = ctx;
    if (!ctx->ev_p1) CK(cudaEventCreateWithFlags(&ctx->ev_p1, cudaEventDisableTiming));
    j.p1_done = ctx->ev_p1;
    if ((st = job_phase1(j, s)) != HEXFC_OK) return st;
    if ((st = job_wait1(ctx, j, s)) != HEXFC_OK) return st;
    collect(ctx);
    if (ctx->pend.active) {   // the previous frame has completed: verify it
        bool redrawn = false;
        if ((st = settle_pending(ctx, s, &redrawn)) != HEXFC_OK) return st;
        if (redrawn) {   // its exact redraw reused these buffers: this frame's first passes once more
            if (ctx->predicted == 1 && (ctx->counts_W != j.W || ctx->counts_H != j.H))
                return render_frame(ctx, m, out, stats, s);
            if ((st = job_phase1(j, s)) != HEXFC_OK) return st;
            if ((st = job_wait1(ctx, j, s)) != HEXFC_OK) return st;
        }
    }
    if ((st = job_read1(j)) != HEXFC_OK) return st;
    // fragment arrays for the regions of this frame (previous counts * margin + pad) and a pool
    // after them for the tiles above their capacity
    // (the previous frame's fragment total, now verified, scaled to this frame's pixels)
    const double prev_total = (double)ctx->counts_total * ((double)j.W * j.H) /
                              ((double)ctx->counts_W * (double)ctx->counts_H);
    const uint64_t want = (uint64_t)(prev_total * (1.0 + kCapMargin + kCapPool)) + (uint64_t)j.n_tiles * kCapPad;
    if (!fb.key || fb.frag_cap < (int64_t)want) {
        int64_t c1 = 0;
        dfree(fb.rgba);
        if ((st = ensure(&fb.key, &fb.frag_cap, (int64_t)want)) != HEXFC_OK) return st;
        if ((st = ensure(&fb.rgba, &c1, fb.frag_cap)) != HEXFC_OK) return st;
    }
    job_mark(j, 4, s);
    CK(cudaMemsetAsync(fb.bins, 0xFF, sizeof(uint32_t) * (size_t)j.n_bins, s));   // padding slots = kPadBin
    CK(launch_bin_fill(*m, fb, j.tiles_x, j.W, j.H, j.reverse, s));
    CK(launch_bin_sort(*m, fb, j.tiles_x, j.tiles_y, j.buckets, s));
    if (!j.order_done) CK(launch_tile_order(fb, j.n_tiles, s));
    if ((st = job_features(j, s)) != HEXFC_OK) return st;
    // stages: bin (with the features, the capacities and their scan), count,
    // then no pixel scan and no host wait, fill, composite
    if (ctx->predicted == 2) {
        CK(launch_cap_forward(ctx->cap, fb, j.n_tiles, kCapMargin, kCapPad, s));
    } else {   // previous-frame counts, or (mode 3) the previous total spread evenly over the tiles
        const uint32_t uniform =
            ctx->predicted == 3 ? (uint32_t)std::max(1.0, std::ceil(prev_total / (double)j.n_tiles)) : 0u;
        CK(launch_capacity_from_previous(fb, j.n_tiles, kCapMargin, kCapPad, uniform, s));
    }
    CK(scan_u32_to_u64(fb.tile_cap, fb.cap_off, j.n_tiles, fb.part, fb.part_max, fb.scal + 11, 0xFFFFFFFFu, s));
    CK(cudaMemsetAsync(fb.cstat, 0, sizeof(uint64_t) * 4 * kStatCopies, s));
    job_mark(j, 5, s);
    CK(launch_count(*m, fb, j.tiles_x, j.tiles_y, j.W, j.H, true, s));
    job_mark(j, 6, s);
    job_mark(j, 7, s);
    job_mark(j, 8, s);
    if ((st = job_sil_clear(j, s)) != HEXFC_OK) return st;
    CK(launch_fill(*m, fb, j.sp, j.tiles_x, j.tiles_y, j.W, j.H, true, j.sil_alpha > 0.f, s));
    job_mark(j, 9, s);
    CK(launch_composite(fb, j.sp, j.tiles_x, j.tiles_y, j.W, j.H, out, kLongListsUnknown, j.window, j.win, s));
    if ((st = job_silhouette(j, out, s)) != HEXFC_OK) return st;
    job_mark(j, 10, s);
    j.launches += (j.order_done ? 3 : 4) + 1 + 3 + 1 + 1 + 3;   // (the tile order counted by phase 1)
    // the frame's scalars and count statistics for its verification; no wait here
    CK(cudaMemcpyAsync(ctx->h_pend, fb.scal, kScal * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_pend + kScal, fb.cstat, 4 * kStatCopies * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                       s));
    ctx->ev_pending[ctx->ev_cur] = ctx->timing;
    hexfc_frame_stats& fs = j.fs;
    fs = hexfc_frame_stats{};
    fs.bin_entries = j.n_bins;
    fs.width = (uint32_t)j.W;
    fs.height = (uint32_t)j.H;
    fs.kernel_launches = j.launches;
    fs.predicted = 1;
    fs.pending = 1;   // fragments, longest list, tiles over capacity: known once verified
    fs.frame = ++ctx->frame_seq;
    hexfc_ctx::Pending& p = ctx->pend;
    p.active = true;
    p.mesh.reset();
    for (const auto& sp_m : ctx->meshes)
        if (sp_m.get() == m) p.mesh = sp_m;
    p.out = out;
    p.stream = s;
    p.view = ctx->view;
    p.cam = ctx->cam;
    p.zref = ctx->zref;
    p.lens = ctx->lens;
    p.style = ctx->style;
    p.fs = fs;
    ctx->last = fs;
    if (stats) *stats = fs;
    ctx->have_frame = true;
    ctx->last_W = j.W;
    ctx->last_win = j.win;
    ctx->last_H = j.H;
    ctx->last_tiles_x = j.tiles_x;
    ctx->last_tiles_y = j.tiles_y;
    ctx->counts_W = j.W;   // k_count leaves the exact tile counts in fb.tile_frag
    ctx->counts_H = j.H;
    ctx->feat_tiles = j.n_tiles;
    remember_camera(ctx, j.cam);
    return HEXFC_OK;
}

// Verify the pending frame (drawn with chosen capacities), which must have
// completed or be about to (its stream is waited for): its device scalars give
// its statistics; device error bits are reported; if its pool ran out or a list
// is too long for the resolve, it is drawn again exactly (count-then-fill) into
// its output with its own camera, lens and style. s: the stream of the caller's
// frame, on which the consumed error bits are cleared.
hexfc_status settle_pending(hexfc_ctx* ctx, cudaStream_t s, bool* redrawn)
{
    *redrawn = false;
    if (!ctx->pend.active) return HEXFC_OK;
    hexfc_ctx::Pending p = ctx->pend;
    ctx->pend.active = false;
    ctx->pend.mesh.reset();
    CK(cudaStreamSynchronize(p.stream));
    const uint64_t* h = ctx->h_pend;
    const uint64_t bits = h[5];
    hexfc_frame_stats fs = p.fs;
    fs.pending = 0;
    fs.overflow_tiles = (uint32_t)h[6];
    fs.capacity = h[11];
    fs.fragments = 0;   // from the count pass (no pixel scan): the sums over its counter copies
    fs.max_list = 0;
    fs.long_lists = 0;
    for (int c = 0; c < kStatCopies; ++c) {
        const uint64_t* cs = h + kScal + 4 * c;
        fs.fragments += cs[0];
        fs.max_list = std::max(fs.max_list, (uint32_t)cs[1]);
        fs.long_lists += (uint32_t)cs[2];
    }
    if (bits) CK(cudaMemsetAsync(ctx->fb.scal + 5, 0, sizeof(uint64_t), s));
    if (bits & ~kErrPoolBit) {   // a bounded wait ran out or a check failed
        record_final(ctx, fs);
        return device_error_status(bits);
    }
    if ((bits & kErrPoolBit) || fs.max_list > HEXFC_MAX_LIST) {
        if (!p.mesh) return HEXFC_ERR_STATE;
        // the pool after the regions ran out, or a list is too long: draw it
        // again exactly, with the camera, lens and style it was drawn with
        const hexfc_view v = ctx->view;
        const CamParams cam = ctx->cam;
        const double zref = ctx->zref;
        const hexfc_lens lens = ctx->lens;
        const hexfc_style style = ctx->style;
        ctx->view = p.view;
        ctx->cam = p.cam;
        ctx->zref = p.zref;
        ctx->lens = p.lens;
        ctx->style = p.style;
        hexfc_frame_stats ex{};
        hexfc_status st = render_frame(ctx, p.mesh.get(), p.out, &ex, p.stream);
        ctx->view = v;
        ctx->cam = cam;
        ctx->zref = zref;
        ctx->lens = lens;
        ctx->style = style;
        CK(cudaStreamSynchronize(p.stream));   // its buffers are this context's: done before the next frame
        ex.frame = fs.frame;
        ex.redrawn = 1;
        ex.overflow_tiles = fs.overflow_tiles;
        ex.capacity = fs.capacity;
        record_final(ctx, ex);
        *redrawn = true;
        return st;
    }
    ctx->counts_total = fs.fragments;
    record_final(ctx, fs);
    return HEXFC_OK;
}

// Wait for the context's last frame and verify it if it is pending.
hexfc_status finish_pending(hexfc_ctx* ctx)
{
    if (!ctx->pend.active) return HEXFC_OK;
    bool redrawn = false;
    return settle_pending(ctx, ctx->pend.stream, &redrawn);
}

// Capture `body(i, stream_i)` for the listed items, each on its own stream
// forked from the context's origin stream and joined back, as one graph;
// reuse the phase's executable graph when only parameters changed.
// Weights, moments and gradient of the capacity network (once).
hexfc_status cap_alloc(CapNet& n)
{
    hexfc_status st = HEXFC_OK;
    if (!n.w) {
        if ((st = dalloc(&n.w, kCapParams)) != HEXFC_OK) return st;
        if ((st = dalloc(&n.w16, kCapParams)) != HEXFC_OK) return st;
        if ((st = dalloc(&n.m, kCapParams)) != HEXFC_OK) return st;
        if ((st = dalloc(&n.v, kCapParams)) != HEXFC_OK) return st;
        if ((st = dalloc(&n.grad, kCapParams + 1)) != HEXFC_OK) return st;
    }
    return st;
}

// Per-tile training buffers for n tiles.
hexfc_status cap_train_buffers(CapNet& c, int64_t n)
{
    if (c.h1 && c.tiles >= n) return HEXFC_OK;
    dfree(c.h1); dfree(c.h2); dfree(c.da1); dfree(c.da2); dfree(c.dy); dfree(c.x); dfree(c.t);
    c.tiles = 0;
    hexfc_status st;
    const int64_t m = n + n / 4 + 256;
    if ((st = dalloc(&c.h1, (size_t)(m * kCapHid))) != HEXFC_OK) return st;
    if ((st = dalloc(&c.h2, (size_t)(m * kCapHid))) != HEXFC_OK) return st;
    if ((st = dalloc(&c.da1, (size_t)(m * kCapHid))) != HEXFC_OK) return st;
    if ((st = dalloc(&c.da2, (size_t)(m * kCapHid))) != HEXFC_OK) return st;
    if ((st = dalloc(&c.dy, (size_t)m)) != HEXFC_OK) return st;
    if ((st = dalloc(&c.x, (size_t)(4 * m))) != HEXFC_OK) return st;
    if ((st = dalloc(&c.t, (size_t)m)) != HEXFC_OK) return st;
    c.tiles = m;
    return HEXFC_OK;
}

// Standard normal values from a splitmix64 stream (Box-Muller).
struct NormalStream {
    uint64_t s;
    double next_u()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);   // (0, 1)
    }
    double next()
    {
        const double u1 = next_u(), u2 = next_u();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

// One phase of a batch as one graph: `pre` of every frame on the frame's own
// stream (branches that run side by side), then `mid` on the origin stream
// after all of them (the batched launches over every frame's tiles), then
// `post` of every frame on its stream again; `mid` and `post` may be empty.
template <typename Pre, typename Mid, typename Post>
hexfc_status batch_graph(hexfc_ctx* ctx, int phase, const std::vector<int>& items, Pre&& pre, Mid&& mid,
                         Post&& post, bool has_mid)
{
    cudaStream_t o = ctx->origin;
    if (const cudaError_t e = cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal); e != cudaSuccess) {
        note_cuda(e);
        return HEXFC_ERR_CUDA;
    }
    hexfc_status st = HEXFC_OK;
    bool ok = true;
    auto branches = [&](auto&& body) {   // fork from the origin stream, run body per frame, join
        ok = ok && cudaEventRecord(ctx->ev_in, o) == cudaSuccess;
        for (int i : items) {
            auto& b = *ctx->batch[(size_t)i];
            ok = ok && cudaStreamWaitEvent(b.stream, ctx->ev_in, 0) == cudaSuccess;
            if (ok && st == HEXFC_OK) st = body(i, b.stream);
            ok = ok && cudaEventRecord(b.done, b.stream) == cudaSuccess;   // join, also after a failure
            ok = ok && cudaStreamWaitEvent(o, b.done, 0) == cudaSuccess;
        }
    };
    branches(pre);
    if (has_mid) {
        if (ok && st == HEXFC_OK) st = mid(o);
        branches(post);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(o, &g);
    if (!ok || ec != cudaSuccess || st != HEXFC_OK || !g) {
        if (ec != cudaSuccess) note_cuda(ec);
        else (void)cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return st != HEXFC_OK ? st : HEXFC_ERR_CUDA;
    }
    cudaGraphExec_t& ex = ctx->graph_exec[phase];
    if (ex) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(ex, g, &info) == cudaSuccess) {
            ++ctx->graph_updates;
        } else {   // another shape of graph: build it anew
            (void)cudaGetLastError();
            cudaGraphExecDestroy(ex);
            ex = nullptr;
        }
    }
    if (!ex) {
        if (const cudaError_t e = cudaGraphInstantiate(&ex, g, 0); e != cudaSuccess) {
            note_cuda(e);
            ex = nullptr;
            cudaGraphDestroy(g);
            return HEXFC_ERR_CUDA;
        }
        ++ctx->graph_instantiations;
    }
    cudaGraphDestroy(g);
    if (const cudaError_t e = cudaGraphLaunch(ex, o); e != cudaSuccess) {
        note_cuda(e);
        return HEXFC_ERR_CUDA;
    }
    return HEXFC_OK;
}

}  // namespace

extern "C" {

void hexfc_style_default(hexfc_style* s)
{
    if (!s) return;
    s->w_base = 2.f;
    s->lod = 1;
    s->delta = 0.5f;
    s->s = 1.5f;
    s->alpha_min = 0.1f;
    s->alpha_max = 0.6f;
    s->tf_lo = 0.f;
    s->tf_hi = 1.f;
    s->bg[0] = s->bg[1] = s->bg[2] = 0.f;
    s->accent_beta = 0.2f;
    s->halo_scale = 0.5f;
    s->darken = 0.25f;
    s->g_min = 0.5f;
    s->g_max = 2.f;
    s->desat = 0.35f;          // the depth cue and the silhouettes of the paper's final look
    s->sil_alpha = 1.f;
    s->sil_threshold = 32768.f;
}

hexfc_status hexfc_create(hexfc_ctx** out, int device, uint64_t frag_budget_bytes)
{
    if (!out) return HEXFC_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (const cudaError_t e = cudaGetDeviceCount(&n); e != cudaSuccess || device < 0 || device >= n) {
        note_cuda(e != cudaSuccess ? e : cudaErrorInvalidDevice);
        return HEXFC_ERR_CUDA;
    }
    hexfc_ctx* c = new (std::nothrow) hexfc_ctx();
    if (!c) return HEXFC_ERR_OOM;
    c->device = device;
    c->budget = frag_budget_bytes;
    hexfc_style_default(&c->style);
    c->lens.mode = HEXFC_LENS_SCREEN;
    c->lens.radius = 1.0;
    {
        DeviceGuard g(device);
        if (prepare_raster_kernels() != cudaSuccess || prepare_fill_kernels() != cudaSuccess ||
            prepare_composite_kernels() != cudaSuccess) {
            (void)cudaGetLastError();
            delete c;
            return HEXFC_ERR_CUDA;
        }
    }
    *out = c;
    return HEXFC_OK;
}

void hexfc_destroy(hexfc_ctx* ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    ctx->pend.active = false;
    ctx->pend.mesh.reset();
    if (ctx->h_pend) cudaFreeHost(ctx->h_pend);
    ctx->h_pend = nullptr;
    ctx->meshes.clear();   // a mesh is freed with its last holder
    free_frame(ctx->fb);
    for (auto& b : ctx->batch) {
        free_frame(b->fb);
        if (b->stream) cudaStreamDestroy(b->stream);
        if (b->done) cudaEventDestroy(b->done);
    }
    for (auto& g : ctx->graph_exec)
        if (g) cudaGraphExecDestroy(g);
    {
        CapNet& n = ctx->cap;
        dfree(n.w); dfree(n.w16); dfree(n.m); dfree(n.v); dfree(n.grad);
        dfree(n.h1); dfree(n.h2); dfree(n.da1); dfree(n.da2); dfree(n.dy); dfree(n.x); dfree(n.t);
    }
    if (ctx->origin) cudaStreamDestroy(ctx->origin);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->ev_p1) cudaEventDestroy(ctx->ev_p1);
    dfree(ctx->d_out);
    for (auto& set : ctx->ev)
        for (auto& e : set)
            if (e) cudaEventDestroy(e);
    delete ctx;
}

hexfc_status hexfc_upload_mesh(hexfc_ctx* ctx, const float* verts, int64_t n_verts, const int32_t* cells,
                               int64_t n_cells, const float* cell_scalar, const uint8_t* cell_edge_level,
                               int32_t* mesh_id_out)
{
    if (!ctx || !verts || !cells || !mesh_id_out || n_verts <= 0) return HEXFC_ERR_ARG;
    if (n_cells <= 0) return HEXFC_ERR_MESH;
    if (n_verts >= (1ll << 31) || n_cells >= (1ll << 27)) return HEXFC_ERR_ARG;
    DeviceGuard g(ctx->device);
    HostTables t;
    if (build_host_tables(verts, n_verts, cells, n_cells, cell_edge_level, t) != 0) return HEXFC_ERR_MESH;
    if (2 * t.n_faces >= (1ll << 32)) return HEXFC_ERR_ARG;
    DevMesh* m = new (std::nothrow) DevMesh();
    if (!m) return HEXFC_ERR_OOM;
    m->n_verts = n_verts;
    m->n_cells = n_cells;
    m->n_faces = t.n_faces;
    m->n_edges = t.n_edges;
    hexfc_status st = HEXFC_OK;
    auto A = [&](hexfc_status s2) { if (st == HEXFC_OK) st = s2; };
    A(dalloc(&m->verts, 3 * (size_t)n_verts));
    A(dalloc(&m->cells, 8 * (size_t)n_cells));
    A(dalloc(&m->cell_edges, 12 * (size_t)n_cells));
    A(dalloc(&m->cell_imp, (size_t)n_cells));
    A(dalloc(&m->vkey, (size_t)n_verts));
    A(dalloc(&m->ekey, (size_t)t.n_edges));
    A(dalloc(&m->vimp, (size_t)n_verts));
    A(dalloc(&m->eattr, (size_t)t.n_edges));
    A(dalloc(&m->elevel, (size_t)t.n_edges));
    A(dalloc(&m->fverts, (size_t)t.n_faces));
    A(dalloc(&m->fedges, (size_t)t.n_faces));
    A(dalloc(&m->fstat, (size_t)t.n_faces));
    A(dalloc(&m->fbound, (size_t)t.n_faces));
    if (st != HEXFC_OK) {
        free_mesh(m);
        return st;
    }
    cudaError_t e = cudaSuccess;
    auto H2D = [&](void* d, const void* h, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice);
    };
    H2D(m->verts, verts, sizeof(float) * 3 * (size_t)n_verts);
    H2D(m->cells, cells, sizeof(int32_t) * 8 * (size_t)n_cells);
    H2D(m->cell_edges, t.cell_edges.data(), sizeof(int32_t) * t.cell_edges.size());
    H2D(m->elevel, t.elevel.data(), t.elevel.size());
    H2D(m->fverts, t.fverts.data(), sizeof(int32_t) * t.fverts.size());
    H2D(m->fedges, t.fedges.data(), sizeof(int32_t) * t.fedges.size());
    H2D(m->fbound, t.fbound.data(), t.fbound.size());
    if (cell_scalar) H2D(m->cell_imp, cell_scalar, sizeof(float) * (size_t)n_cells);
    if (e == cudaSuccess && !cell_scalar) e = launch_cell_quality(*m, HEXFC_METRIC_IMPORTANCE, m->cell_imp, 0);
    if (e == cudaSuccess) e = launch_importance(*m, true, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        note_cuda(e);
        free_mesh(m);
        return HEXFC_ERR_CUDA;
    }
    const int dev = ctx->device;
    try {
        ctx->meshes.emplace_back(m, [dev](DevMesh* p) {
            DeviceGuard g2(dev);
            free_mesh(p);
        });
    } catch (...) {
        free_mesh(m);
        return HEXFC_ERR_OOM;
    }
    *mesh_id_out = (int32_t)(ctx->meshes.size() - 1);
    return HEXFC_OK;
}

hexfc_status hexfc_render_batch(hexfc_ctx* ctx, int32_t n, const hexfc_batch_item* items,
                                hexfc_frame_stats* stats, hexfc_status* item_status, void* stream)
{
    if (!ctx || n < 0 || (n > 0 && !items)) return HEXFC_ERR_ARG;
    std::vector<CamParams> cams((size_t)n);
    std::vector<double> zrefs((size_t)n, 1.0);
    for (int32_t i = 0; i < n; ++i) {
        const hexfc_batch_item& it = items[i];
        if (!it.out_rgba || !valid_lens(&it.lens) || !valid_style(&it.style)) return HEXFC_ERR_ARG;
        if (!valid_view(&it.view, cams[(size_t)i], zrefs[(size_t)i])) return HEXFC_ERR_ARG;
        if (!get_mesh(ctx, it.mesh)) return HEXFC_ERR_STATE;
    }
    if (n == 0) return HEXFC_OK;
    DeviceGuard g(ctx->device);
    const cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->origin) {
        CK(cudaStreamCreateWithFlags(&ctx->origin, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));
    }
    while ((int32_t)ctx->batch.size() < n) {
        std::unique_ptr<hexfc_ctx::BatchSlot> b(new (std::nothrow) hexfc_ctx::BatchSlot());
        if (!b) return HEXFC_ERR_OOM;
        CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
        ctx->batch.push_back(std::move(b));
    }
    std::vector<FrameJob> jobs((size_t)n);
    std::vector<hexfc_status> res((size_t)n, HEXFC_OK);
    std::vector<int> live;
    hexfc_status st;
    for (int32_t i = 0; i < n; ++i) {
        const hexfc_batch_item& it = items[i];
        FrameJob& j = jobs[(size_t)i];
        j.fb = &ctx->batch[(size_t)i]->fb;
        j.m = get_mesh(ctx, it.mesh);
        j.cam = cams[(size_t)i];
        j.sp = make_shade_params(it.lens, it.style, zrefs[(size_t)i], j.cam.ortho);
        j.lod = it.style.lod;
        j.delta = it.style.delta;
        j.W = it.view.width;
        j.H = it.view.height;
        j.tiles_x = (j.W + kTileW - 1) / kTileW;
        j.tiles_y = (j.H + kTileH - 1) / kTileH;
        j.n_tiles = (int64_t)j.tiles_x * j.tiles_y;
        j.n_pix = j.n_tiles * kTilePix;
        j.reverse = ctx->reverse_bins;
        j.buckets = ctx->depth_buckets;
        j.window = ctx->window;
        j.budget = ctx->budget;
        j.out = it.out_rgba;
        j.win = OutWin{0, 0, j.W, j.H};   // whole frames
        j.sil_alpha = it.style.sil_alpha;
        j.sil_threshold = it.style.sil_threshold;
        j.frame_w = j.W;
        j.frame_h = j.H;
        if ((st = job_alloc(j)) != HEXFC_OK) return st;
        live.push_back(i);
    }
    // the batch starts after the caller's earlier work on its stream
    CK(cudaEventRecord(ctx->ev_out, s));
    CK(cudaStreamWaitEvent(ctx->origin, ctx->ev_out, 0));
    auto none = [](int, cudaStream_t) -> hexfc_status { return HEXFC_OK; };
    auto no_mid = [](cudaStream_t) -> hexfc_status { return HEXFC_OK; };
    if ((st = batch_graph(
             ctx, 0, live, [&](int i, cudaStream_t si) { return job_phase1(jobs[(size_t)i], si); }, no_mid, none,
             false)) != HEXFC_OK)
        return st;
    CK(cudaStreamSynchronize(ctx->origin));
    for (int i : live)
        if ((st = job_read1(jobs[(size_t)i])) != HEXFC_OK) return st;
    // the count of every frame in one launch (per group of kBatchLaunchMax frames)
    auto count_all = [&](cudaStream_t o) -> hexfc_status {
        CountBatch b;
        return batched(
            b, live,
            [&](CountBatch& cb, int i) {
                const FrameJob& j = jobs[(size_t)i];
                cb.it[cb.n] = count_item(j);
                cb.tile_begin[cb.n + 1] = cb.tile_begin[cb.n] + (uint32_t)j.n_tiles;
                ++cb.n;
            },
            [&](CountBatch& cb) { return launch_count_batch(cb, o); });
    };
    const bool one = ctx->batch_launch;
    if (one && (st = batch_graph(
                    ctx, 1, live, [&](int i, cudaStream_t si) { return job_phase2_bins(jobs[(size_t)i], si); },
                    count_all, [&](int i, cudaStream_t si) { return job_phase2_scan(jobs[(size_t)i], si); }, true)) !=
                   HEXFC_OK)
        return st;
    if (!one && (st = batch_graph(
                     ctx, 1, live, [&](int i, cudaStream_t si) { return job_phase2(jobs[(size_t)i], si); }, no_mid,
                     none, false)) != HEXFC_OK)
        return st;
    CK(cudaStreamSynchronize(ctx->origin));
    std::vector<int> draw, draw_sil, draw_plain;
    for (int i : live) {
        res[(size_t)i] = job_read2(jobs[(size_t)i], ctx->batch[(size_t)i]->stream);
        if (res[(size_t)i] != HEXFC_OK) continue;
        draw.push_back(i);
        (jobs[(size_t)i].sil_alpha > 0.f ? draw_sil : draw_plain).push_back(i);
    }
    // the fill of every frame in one launch (one per fill variant), then the
    // main resolve pass of every frame in one launch
    auto fill_composite_all = [&](cudaStream_t o) -> hexfc_status {
        hexfc_status r = HEXFC_OK;
        for (int variant = 0; variant < 2 && r == HEXFC_OK; ++variant) {
            FillBatch b;
            r = batched(
                b, variant ? draw_sil : draw_plain,
                [&](FillBatch& fbt, int i) {
                    const FrameJob& j = jobs[(size_t)i];
                    fbt.it[fbt.n] = fill_item(j);
                    fbt.tile_begin[fbt.n + 1] = fbt.tile_begin[fbt.n] + (uint32_t)j.n_tiles;
                    ++fbt.n;
                },
                [&](FillBatch& fbt) { return launch_fill_batch(fbt, variant == 1, o); });
        }
        if (r != HEXFC_OK) return r;
        CompositeBatch cb;
        return batched(
            cb, draw,
            [&](CompositeBatch& c, int i) {
                const FrameJob& j = jobs[(size_t)i];
                c.it[c.n] = composite_item(j);
                c.tile_begin[c.n + 1] = c.tile_begin[c.n] + (uint32_t)j.n_tiles;
                ++c.n;
            },
            [&](CompositeBatch& c) { return launch_composite_batch(c, ctx->window, o); });
    };
    auto tail = [&](int i, cudaStream_t si) -> hexfc_status {   // short lists past the window, long lists, silhouettes
        FrameJob& j = jobs[(size_t)i];
        CK(launch_composite_tail(*j.fb, j.sp, j.tiles_x, j.out, j.n_long, j.win, si));
        hexfc_status r = job_silhouette(j, j.out, si);
        j.launches += 3 + (j.n_long > 0 ? 1 : 0);
        j.fs.kernel_launches = j.launches;
        return r;
    };
    if (one && !draw.empty() &&
        (st = batch_graph(
             ctx, 2, draw, [&](int i, cudaStream_t si) { return job_sil_clear(jobs[(size_t)i], si); },
             fill_composite_all, tail, true)) != HEXFC_OK)
        return st;
    if (!one && !draw.empty() &&
        (st = batch_graph(
             ctx, 2, draw, [&](int i, cudaStream_t si) { return job_phase3(jobs[(size_t)i], si); }, no_mid, none,
             false)) != HEXFC_OK)
        return st;
    // the caller's stream continues after the batch
    CK(cudaEventRecord(ctx->ev_out, ctx->origin));
    CK(cudaStreamWaitEvent(s, ctx->ev_out, 0));
    hexfc_status first = HEXFC_OK;
    for (int32_t i = 0; i < n; ++i) {
        if (stats) stats[i] = jobs[(size_t)i].fs;
        if (item_status) item_status[i] = res[(size_t)i];
        if (first == HEXFC_OK) first = res[(size_t)i];
    }
    return first;
}

hexfc_status hexfc_capacity_set_weights(hexfc_ctx* ctx, const float* w, int64_t n)
{
    if (!ctx || !w || n != kCapParams) return HEXFC_ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(w[i])) return HEXFC_ERR_ARG;
    DeviceGuard g(ctx->device);
    CapNet& c = ctx->cap;
    hexfc_status st;
    if ((st = cap_alloc(c)) != HEXFC_OK) return st;
    CK(cudaMemcpy(c.w, w, sizeof(float) * kCapParams, cudaMemcpyHostToDevice));
    CK(cudaMemset(c.m, 0, sizeof(float) * kCapParams));
    CK(cudaMemset(c.v, 0, sizeof(float) * kCapParams));
    CK(launch_cap_to_half(c, 0));
    CK(cudaDeviceSynchronize());
    c.step = 0;
    c.ready = true;
    return HEXFC_OK;
}

hexfc_status hexfc_capacity_reset(hexfc_ctx* ctx, uint64_t seed)
{
    if (!ctx) return HEXFC_ERR_ARG;
    std::vector<float> w((size_t)kCapParams, 0.f);
    NormalStream rs{seed};
    const int oW1 = 0, oB1 = kCapHid * kCapIn, oW2 = oB1 + kCapHid, oB2 = oW2 + kCapHid * kCapHid;
    const int oW3 = oB2 + kCapHid, oB3 = oW3 + kCapHid;
    for (int i = oW1; i < oB1; ++i) w[(size_t)i] = (float)(rs.next() * std::sqrt(2.0 / kCapIn));
    for (int i = oW2; i < oB2; ++i) w[(size_t)i] = (float)(rs.next() * std::sqrt(2.0 / kCapHid));
    for (int i = oW3; i < oB3; ++i) w[(size_t)i] = (float)(rs.next() * std::sqrt(1.0 / kCapHid));
    w[(size_t)oB3] = 5.f;   // log(1 + count) of a few hundred fragments
    return hexfc_capacity_set_weights(ctx, w.data(), kCapParams);
}

hexfc_status hexfc_capacity_get_weights(hexfc_ctx* ctx, float* w, int64_t n)
{
    if (!ctx || !w || n != kCapParams) return HEXFC_ERR_ARG;
    if (!ctx->cap.ready) return HEXFC_ERR_STATE;
    DeviceGuard g(ctx->device);
    CK(cudaMemcpy(w, ctx->cap.w, sizeof(float) * kCapParams, cudaMemcpyDeviceToHost));
    return HEXFC_OK;
}

hexfc_status hexfc_capacity_grad(hexfc_ctx* ctx, const float* x, const uint32_t* counts, int64_t n, float* grad,
                                 float* loss)
{
    if (!ctx || !x || !counts || n < 1 || !grad) return HEXFC_ERR_ARG;
    if (!ctx->cap.ready) return HEXFC_ERR_STATE;
    DeviceGuard g(ctx->device);
    CapNet& c = ctx->cap;
    hexfc_status st;
    if ((st = cap_train_buffers(c, n)) != HEXFC_OK) return st;
    CK(cudaMemcpy(c.x, x, sizeof(float) * 4 * (size_t)n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.t, counts, sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice));
    CK(launch_cap_grad(c, c.x, c.t, n, 0));
    CK(cudaMemcpy(grad, c.grad, sizeof(float) * kCapParams, cudaMemcpyDeviceToHost));
    if (loss) CK(cudaMemcpy(loss, c.grad + kCapParams, sizeof(float), cudaMemcpyDeviceToHost));
    return HEXFC_OK;
}

hexfc_status hexfc_capacity_train(hexfc_ctx* ctx, int32_t steps, float lr, float* loss, void* stream)
{
    if (!ctx || steps < 0 || !(lr > 0.f)) return HEXFC_ERR_ARG;
    if (!ctx->cap.ready || ctx->feat_tiles == 0) return HEXFC_ERR_STATE;
    DeviceGuard g(ctx->device);
    CapNet& c = ctx->cap;
    const cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = ctx->feat_tiles;
    hexfc_status st;
    if ((st = cap_train_buffers(c, n)) != HEXFC_OK) return st;
    for (int32_t k = 0; k < steps; ++k) {
        CK(launch_cap_grad(c, ctx->fb.cap_x, ctx->fb.tile_frag, n, s));
        CK(launch_cap_adam(c, lr, s));
    }
    if (loss) {
        if (steps == 0) CK(launch_cap_grad(c, ctx->fb.cap_x, ctx->fb.tile_frag, n, s));
        CK(cudaMemcpyAsync(loss, c.grad + kCapParams, sizeof(float), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return HEXFC_OK;
}

hexfc_status hexfc_frame_memory(const hexfc_ctx* ctx, uint64_t* bytes)
{
    if (!ctx || !bytes) return HEXFC_ERR_ARG;
    uint64_t b = frame_bytes(ctx->fb, ctx->fb.frag_cap);
    b += (uint64_t)ctx->d_out_cap * sizeof(float);
    for (const auto& bs : ctx->batch) {
        const FrameBufs& g = bs->fb;
        b += (uint64_t)g.v_cap * (sizeof(int4) + sizeof(float)) +
             (uint64_t)g.f_cap * (sizeof(FaceFrame) + 2 * sizeof(uint32_t)) +
             (uint64_t)g.t_cap * (9 * sizeof(uint32_t) + sizeof(uint64_t) + sizeof(uint32_t)) +
             (uint64_t)(2 * g.bin_cap + g.mask_cap) * sizeof(uint32_t) + (uint64_t)g.seg_cap * sizeof(uint64_t) +
             (uint64_t)g.p_cap * (3 * sizeof(uint32_t) + sizeof(uint64_t)) +
             (uint64_t)g.part_cap * (sizeof(uint64_t) + sizeof(uint32_t)) +
             (uint64_t)g.frag_cap * (sizeof(uint64_t) + sizeof(float4));
    }
    *bytes = b;
    return HEXFC_OK;
}

hexfc_status hexfc_trim(hexfc_ctx* ctx)
{
    if (!ctx) return HEXFC_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (ctx->pend.active) {
        const hexfc_status st = finish_pending(ctx);
        if (st != HEXFC_OK) return st;
    }
    uint64_t* pinned = ctx->fb.h_scal;
    ctx->fb.h_scal = nullptr;   // the pinned mirror is small: keep it
    free_frame(ctx->fb);
    ctx->fb.h_scal = pinned;
    for (auto& bs : ctx->batch) {
        uint64_t* hp = bs->fb.h_scal;
        bs->fb.h_scal = nullptr;
        free_frame(bs->fb);
        bs->fb.h_scal = hp;
    }
    dfree(ctx->d_out);
    ctx->d_out_cap = 0;
    ctx->have_frame = false;
    return HEXFC_OK;
}

hexfc_status hexfc_share_mesh(hexfc_ctx* dst, const hexfc_ctx* src, int32_t mesh, int32_t* mesh_id_out)
{
    if (!dst || !src || !mesh_id_out || dst->device != src->device) return HEXFC_ERR_ARG;
    if (mesh < 0 || mesh >= (int32_t)src->meshes.size()) return HEXFC_ERR_STATE;
    try {
        dst->meshes.push_back(src->meshes[(size_t)mesh]);
    } catch (...) {
        return HEXFC_ERR_OOM;
    }
    *mesh_id_out = (int32_t)(dst->meshes.size() - 1);
    return HEXFC_OK;
}

hexfc_status hexfc_cell_quality(hexfc_ctx* ctx, int32_t mesh, int32_t metric, float* out, void* stream)
{
    if (!ctx || !out || metric < 0 || metric > 2) return HEXFC_ERR_ARG;
    DevMesh* m = get_mesh(ctx, mesh);
    if (!m) return HEXFC_ERR_STATE;
    DeviceGuard g(ctx->device);
    CK(launch_cell_quality(*m, metric, out, (cudaStream_t)stream));
    return HEXFC_OK;
}

hexfc_status hexfc_set_cell_importance(hexfc_ctx* ctx, int32_t mesh, const float* cell_importance, void* stream)
{
    if (!ctx || !cell_importance) return HEXFC_ERR_ARG;
    DevMesh* m = get_mesh(ctx, mesh);
    if (!m) return HEXFC_ERR_STATE;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(m->cell_imp, cell_importance, sizeof(float) * (size_t)m->n_cells, cudaMemcpyDeviceToDevice, s));
    CK(launch_importance(*m, false, s));   // positions unchanged since the upload
    return HEXFC_OK;
}

hexfc_status hexfc_mesh_info(hexfc_ctx* ctx, int32_t mesh, int64_t* n_faces, int64_t* n_edges)
{
    DevMesh* m = get_mesh(ctx, mesh);
    if (!m) return ctx ? HEXFC_ERR_STATE : HEXFC_ERR_ARG;
    if (n_faces) *n_faces = m->n_faces;
    if (n_edges) *n_edges = m->n_edges;
    return HEXFC_OK;
}

hexfc_status hexfc_set_view(hexfc_ctx* ctx, const hexfc_view* v)
{
    if (!ctx || !v) return HEXFC_ERR_ARG;
    CamParams c{};
    double zref = 1.0;
    if (!valid_view(v, c, zref)) return HEXFC_ERR_ARG;
    ctx->view = *v;
    ctx->cam = c;
    ctx->zref = zref;
    ctx->have_view = true;
    ctx->sub_x0 = ctx->sub_y0 = ctx->sub_w = ctx->sub_h = 0;   // the whole frame
    return HEXFC_OK;
}

hexfc_status hexfc_set_subrect(hexfc_ctx* ctx, int32_t x0, int32_t y0, int32_t w, int32_t h)
{
    if (!ctx) return HEXFC_ERR_ARG;
    if (!ctx->have_view) return HEXFC_ERR_STATE;
    const hexfc_view& v = ctx->view;
    if (w == 0 && h == 0 && x0 == 0 && y0 == 0) {
        ctx->sub_x0 = ctx->sub_y0 = ctx->sub_w = ctx->sub_h = 0;
    } else {
        if (x0 < 0 || y0 < 0 || w < 1 || h < 1 || (int64_t)x0 + w > v.width || (int64_t)y0 + h > v.height)
            return HEXFC_ERR_ARG;
        ctx->sub_x0 = x0;
        ctx->sub_y0 = y0;
        ctx->sub_w = w;
        ctx->sub_h = h;
    }
    // drawn: the rectangle and an apron of one pixel inside the frame. The face
    // stage clamps triangle boxes to it (its tiles), like every later stage:
    // W, H are its own, the projection keeps the frame's centre
    if (ctx->sub_w == 0) {
        ctx->cam.ox = ctx->cam.oy = 0;
        ctx->cam.W = v.width;
        ctx->cam.H = v.height;
    } else {
        const int x0a = std::max(0, x0 - 1), y0a = std::max(0, y0 - 1);
        const int x1a = std::min(v.width, x0 + w + 1), y1a = std::min(v.height, y0 + h + 1);
        ctx->cam.ox = x0a;
        ctx->cam.oy = y0a;
        ctx->cam.W = x1a - x0a;
        ctx->cam.H = y1a - y0a;
    }
    return HEXFC_OK;
}

hexfc_status hexfc_set_lens(hexfc_ctx* ctx, const hexfc_lens* l)
{
    if (!ctx || !l || !valid_lens(l)) return HEXFC_ERR_ARG;
    ctx->lens = *l;
    return HEXFC_OK;
}

hexfc_status hexfc_set_style(hexfc_ctx* ctx, const hexfc_style* s)
{
    if (!ctx || !s || !valid_style(s)) return HEXFC_ERR_ARG;
    ctx->style = *s;
    return HEXFC_OK;
}

hexfc_status hexfc_render(hexfc_ctx* ctx, int32_t mesh, float* out_rgba, hexfc_frame_stats* stats, void* stream)
{
    if (!ctx || !out_rgba) return HEXFC_ERR_ARG;
    DevMesh* m = get_mesh(ctx, mesh);
    if (!m || !ctx->have_view) return HEXFC_ERR_STATE;
    DeviceGuard g(ctx->device);
    if (ctx->predicted) return render_frame_predicted(ctx, m, out_rgba, stats, (cudaStream_t)stream);
    return render_frame(ctx, m, out_rgba, stats, (cudaStream_t)stream);
}

hexfc_status hexfc_render_host(hexfc_ctx* ctx, int32_t mesh, float* out_rgba_host, hexfc_frame_stats* stats,
                               void* stream)
{
    if (!ctx || !out_rgba_host) return HEXFC_ERR_ARG;
    DevMesh* m = get_mesh(ctx, mesh);
    if (!m || !ctx->have_view) return HEXFC_ERR_STATE;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = sizeof(float) * 4 * (size_t)draw_w(ctx) * (size_t)draw_h(ctx);
    // A page-locked buffer of this device, 16-byte aligned, is written by the
    // resolve kernels through its device mapping: the image crosses to the
    // host while they run rather than in a copy after them.
    float* d_out = nullptr;
    cudaPointerAttributes pa{};
    const cudaError_t pe = cudaPointerGetAttributes(&pa, out_rgba_host);
    if (pe != cudaSuccess) (void)cudaGetLastError();   // not a pointer CUDA knows: the copy path
    else if (pa.type == cudaMemoryTypeHost && pa.device == ctx->device && pa.devicePointer != nullptr &&
             ((uintptr_t)pa.devicePointer & 15u) == 0)
        d_out = static_cast<float*>(pa.devicePointer);
    const bool direct = d_out != nullptr;
    hexfc_status st = HEXFC_OK;
    if (!direct) {
        st = ensure(&ctx->d_out, &ctx->d_out_cap, (int64_t)(bytes / sizeof(float)));
        if (st != HEXFC_OK) return st;
        d_out = ctx->d_out;
    }
    st = ctx->predicted ? render_frame_predicted(ctx, m, d_out, stats, s) : render_frame(ctx, m, d_out, stats, s);
    if (st == HEXFC_OK && ctx->pend.active) {   // this call waits anyway: verify the frame now
        st = finish_pending(ctx);
        if (stats) *stats = ctx->completed;
    }
    if (st == HEXFC_OK) {
        // the image (unless written in place) and this frame's device error bits
        FrameBufs& fb = ctx->fb;
        cudaError_t e = direct ? cudaSuccess
                               : cudaMemcpyAsync(out_rgba_host, d_out, bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(fb.h_scal + 5, fb.scal + 5, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            note_cuda(e);
            st = HEXFC_ERR_CUDA;
        } else if (fb.h_scal[5] != 0) {
            st = device_error_status(fb.h_scal[5]);
            CK(cudaMemsetAsync(fb.scal + 5, 0, sizeof(uint64_t), s));
            CK(cudaStreamSynchronize(s));
        }
    }
    return st;
}

hexfc_status hexfc_debug_pixels(hexfc_ctx* ctx, const int32_t* px, const int32_t* py, int64_t n, uint32_t* counts,
                                uint64_t* keys, float* rgba, uint64_t cap)
{
    if (!ctx || !px || !py || !counts || n < 0) return HEXFC_ERR_ARG;
    if (!ctx->have_frame) return HEXFC_ERR_STATE;
    if (ctx->pend.active) {
        DeviceGuard g0(ctx->device);
        const hexfc_status st0 = finish_pending(ctx);
        if (st0 != HEXFC_OK) return st0;
    }
    const OutWin win = ctx->last_win;   // pixels of the output image, placed in the drawn rectangle
    for (int64_t i = 0; i < n; ++i)
        if (px[i] < 0 || py[i] < 0 || px[i] >= win.w || py[i] >= win.h) return HEXFC_ERR_ARG;
    if (n == 0) return HEXFC_OK;
    std::vector<int32_t> qx((size_t)n), qy((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        qx[(size_t)i] = px[i] + win.x0;
        qy[(size_t)i] = py[i] + win.y0;
    }
    px = qx.data();
    py = qy.data();
    DeviceGuard g(ctx->device);
    FrameBufs& fb = ctx->fb;
    int32_t *d_px = nullptr, *d_py = nullptr;
    uint32_t* d_cnt = nullptr;
    uint64_t* d_off = nullptr;
    uint64_t* d_keys = nullptr;
    float4* d_rgba = nullptr;
    hexfc_status st = HEXFC_OK;
    auto cleanup = [&]() {
        dfree(d_px); dfree(d_py); dfree(d_cnt); dfree(d_off); dfree(d_keys); dfree(d_rgba);
    };
    if ((st = dalloc(&d_px, (size_t)n)) != HEXFC_OK || (st = dalloc(&d_py, (size_t)n)) != HEXFC_OK ||
        (st = dalloc(&d_cnt, (size_t)n)) != HEXFC_OK || (st = dalloc(&d_off, (size_t)n)) != HEXFC_OK) {
        cleanup();
        return st;
    }
    cudaError_t e = cudaMemcpy(d_px, px, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_py, py, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_debug_gather(fb, d_px, d_py, n, nullptr, ctx->last_tiles_x, ctx->last_W, ctx->last_H, nullptr,
                                nullptr, d_cnt, 0);
    if (e == cudaSuccess) e = cudaMemcpy(counts, d_cnt, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        note_cuda(e);
        cleanup();
        return HEXFC_ERR_CUDA;
    }
    std::vector<uint64_t> hoff((size_t)n);
    uint64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        hoff[(size_t)i] = total;
        total += counts[i];
    }
    if (!keys && !rgba) {
        cleanup();
        return HEXFC_OK;
    }
    if (total > cap) {
        cleanup();
        return HEXFC_ERR_OVERFLOW;
    }
    if ((st = dalloc(&d_keys, (size_t)total)) != HEXFC_OK || (st = dalloc(&d_rgba, (size_t)total)) != HEXFC_OK) {
        cleanup();
        return st;
    }
    e = cudaMemcpy(d_off, hoff.data(), sizeof(uint64_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_debug_gather(fb, d_px, d_py, n, d_off, ctx->last_tiles_x, ctx->last_W, ctx->last_H, d_keys, d_rgba,
                                nullptr, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && keys) e = cudaMemcpy(keys, d_keys, sizeof(uint64_t) * total, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && rgba) e = cudaMemcpy(rgba, d_rgba, sizeof(float4) * total, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && fb.scal) {
        uint64_t errflag = 0;
        e = cudaMemcpy(&errflag, fb.scal + 5, sizeof(uint64_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && errflag) st = device_error_status(errflag);
    }
    cleanup();
    if (e != cudaSuccess) {
        note_cuda(e);
        return HEXFC_ERR_CUDA;
    }
    return st;
}

hexfc_status hexfc_set_option(hexfc_ctx* ctx, int32_t option, int64_t value)
{
    if (!ctx) return HEXFC_ERR_ARG;
    switch (option) {
    case HEXFC_OPT_REVERSE_BIN_ORDER: ctx->reverse_bins = value != 0; return HEXFC_OK;
    case HEXFC_OPT_STAGE_TIMING: ctx->timing = value != 0; return HEXFC_OK;
    case HEXFC_OPT_DEPTH_BUCKETS:
        if (value != 0 && (value < 256 || value > 4096 || (value & (value - 1)) != 0)) return HEXFC_ERR_ARG;
        ctx->depth_buckets = (int)value;
        return HEXFC_OK;
    case HEXFC_OPT_COMPOSITE_WINDOW:
        if (value != 2 && value != 4 && value != 8) return HEXFC_ERR_ARG;
        ctx->window = (int)value;
        return HEXFC_OK;
    case HEXFC_OPT_PREDICTED_CAPACITY:
        if (value < 0 || value > 3) return HEXFC_ERR_ARG;
        ctx->predicted = (int)value;
        return HEXFC_OK;
    case HEXFC_OPT_FRAG_BUDGET:
        if (value < 0) return HEXFC_ERR_ARG;
        ctx->budget = (uint64_t)value;
        return HEXFC_OK;
    case HEXFC_OPT_BATCH_LAUNCH:
        if (value != 0 && value != 1) return HEXFC_ERR_ARG;
        ctx->batch_launch = value != 0;
        return HEXFC_OK;
    case HEXFC_OPT_DEBUG_ERROR_BITS:
        if (value < 0 || value > 7) return HEXFC_ERR_ARG;
        ctx->inject_bits = (uint64_t)value;
        return HEXFC_OK;
    default: return HEXFC_ERR_ARG;
    }
}

hexfc_status hexfc_finish(hexfc_ctx* ctx, hexfc_frame_stats* stats)
{
    if (!ctx) return HEXFC_ERR_ARG;
    DeviceGuard g(ctx->device);
    hexfc_status st = finish_pending(ctx);
    if (stats) *stats = ctx->completed;
    return st;
}

hexfc_status hexfc_completed_stats(const hexfc_ctx* ctx, uint64_t frame, hexfc_frame_stats* stats)
{
    if (!ctx || !stats) return HEXFC_ERR_ARG;
    if (frame == 0) {
        *stats = ctx->completed;
        return HEXFC_OK;
    }
    const hexfc_frame_stats& h = ctx->history[frame % 16];
    if (h.frame != frame) return HEXFC_ERR_STATE;   // not verified yet, or no longer kept
    *stats = h;
    return HEXFC_OK;
}

hexfc_status hexfc_stage_times(hexfc_ctx* ctx, double* ms, uint64_t* frames, int32_t reset)
{
    if (!ctx || !ms || !frames) return HEXFC_ERR_ARG;
    DeviceGuard g(ctx->device);
    collect_set(ctx, ctx->ev_cur ^ 1);
    collect_set(ctx, ctx->ev_cur);
    for (int k = 0; k < HEXFC_N_STAGES; ++k) ms[k] = ctx->stage_ms[k];
    *frames = ctx->timed_frames;
    if (reset) {
        for (double& v : ctx->stage_ms) v = 0.0;
        ctx->timed_frames = 0;
    }
    return HEXFC_OK;
}

int32_t hexfc_last_cuda_error(void) { return t_last_cuda; }

void hexfc_raster_tile(int32_t* width, int32_t* height)
{
    if (width) *width = kTileW;
    if (height) *height = kTileH;
}

const char* hexfc_cuda_error_name(int32_t code) { return cudaGetErrorName((cudaError_t)code); }

const char* hexfc_status_string(hexfc_status s)
{
    switch (s) {
    case HEXFC_OK: return "ok";
    case HEXFC_ERR_ARG: return "invalid argument";
    case HEXFC_ERR_OOM: return "out of memory or fragment budget exceeded";
    case HEXFC_ERR_OVERFLOW: return "per-pixel list or output capacity exceeded";
    case HEXFC_ERR_CUDA: return "CUDA error";
    case HEXFC_ERR_TIMEOUT: return "device wait timed out";
    case HEXFC_ERR_CHECK: return "device-side consistency check failed";
    case HEXFC_ERR_MESH: return "malformed mesh";
    case HEXFC_ERR_STATE: return "call out of order";
    default: return "unknown status";
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Rendering without any allocation (no counterpart in the paper).
//
// Every per-frame buffer of hexfc_render_noalloc lives in one fixed device
// array of HEXFC_NOALLOC_SCRATCH_BYTES, defined here at file scope. Each GPU
// that loads this library holds it until the process exits. In host code the
// array's name is only a host-side stand-in, never a device address, so the
// first call on a device (with that device current) looks the address up with
// cudaGetSymbolAddress and remembers it for that device.

static __device__ __align__(256) unsigned char g_noalloc_scratch[HEXFC_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch on the current device; nullptr on
// failure. Looked up on every call (a table lookup in the runtime; nothing is
// allocated), so that concurrent first calls from several host threads need no
// lock and a context created after cudaDeviceReset gets the new address. The
// first lookup on a device loads this file's module there, which creates the
// array: that first call should come before any stream capture.
void* noalloc_scratch()
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Bump carving of the scratch array in 256-byte aligned pieces.
struct Arena {
    unsigned char* base;
    size_t used, cap;
    template <typename T>
    T* take(size_t n)
    {
        size_t off = (used + 255) & ~(size_t)255;
        size_t bytes = (n == 0 ? 1 : n) * sizeof(T);
        if (off > cap || bytes > cap - off) return nullptr;
        used = off + bytes;
        return reinterpret_cast<T*>(base + off);
    }
};

hexfc_status render_frame_noalloc(hexfc_ctx* ctx, DevMesh* m, float* out, hexfc_frame_stats* stats, cudaStream_t s)
{
    unsigned char* scratch = static_cast<unsigned char*>(noalloc_scratch());
    if (!scratch) return HEXFC_ERR_CUDA;
    const int W = ctx->cam.W, H = ctx->cam.H;   // the drawn rectangle (with its apron)
    const OutWin win = output_window(ctx);
    const bool sil = ctx->style.sil_alpha > 0.f;
    const int tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (H + kTileH - 1) / kTileH;
    const int64_t n_tiles = (int64_t)tiles_x * tiles_y;
    const int64_t n_pix = n_tiles * kTilePix;
    const int64_t nparts = scan_partials_needed(std::max<int64_t>(n_pix, n_tiles)) + 1;
    Arena a{scratch, 0, (size_t)HEXFC_NOALLOC_SCRATCH_BYTES};
    FrameBufs fb;
    // the device scalars first, at the same place in every call: slot 5, the
    // device error word, outlives the call (see below)
    fb.scal = a.take<uint64_t>(kScal);
    fb.vproj = a.take<int4>((size_t)m->n_verts);
    fb.ved = a.take<float>((size_t)m->n_verts);
    fb.fframe = a.take<FaceFrame>((size_t)m->n_faces);
    fb.tzsum = a.take<uint32_t>(2 * (size_t)m->n_faces);
    fb.tile_cnt = a.take<uint32_t>((size_t)n_tiles + 1);
    fb.tile_off = a.take<uint64_t>((size_t)n_tiles + 1);
    fb.tile_cur = a.take<uint32_t>((size_t)n_tiles + 1);
    fb.tile_order = a.take<uint32_t>((size_t)n_tiles + 1);
    fb.tile_frag = a.take<uint32_t>((size_t)n_tiles + 1);
    fb.tile_zr = a.take<float>((size_t)n_tiles + 1);
    fb.cnt = a.take<uint32_t>((size_t)n_pix + 1);
    fb.off = a.take<uint64_t>((size_t)n_pix + 1);
    fb.long_q = a.take<uint32_t>((size_t)n_pix + 1);
    fb.fix_q = a.take<uint32_t>((size_t)n_pix + 1);
    fb.zsil = sil ? a.take<uint32_t>((size_t)n_pix) : nullptr;
    fb.part = a.take<uint64_t>(2 * (size_t)nparts);
    fb.part_max = a.take<uint32_t>(2 * (size_t)nparts);
    if (!fb.vproj || !fb.ved || !fb.fframe || !fb.tzsum || !fb.tile_cnt ||
        !fb.tile_off || !fb.tile_cur || !fb.tile_order || !fb.tile_frag || !fb.tile_zr || !fb.cnt || !fb.off || !fb.long_q || !fb.fix_q || (sil && !fb.zsil) || !fb.part || !fb.part_max ||
        !fb.scal)
        return HEXFC_ERR_OVERFLOW;
    // the array keeps the previous call's contents: clear what must start at zero
    CK(cudaMemsetAsync(fb.tile_cnt, 0, sizeof(uint32_t) * (size_t)n_tiles, s));
    CK(cudaMemsetAsync(fb.tile_cur, 0, sizeof(uint32_t) * (size_t)n_tiles, s));
    // all device scalars but the error word (slot 5): the fill and the composite
    // of the previous call on this device may have set bits there after that
    // call returned, and they are reported below, by this call (the array starts
    // zeroed when the module is loaded)
    CK(cudaMemsetAsync(fb.scal, 0, sizeof(uint64_t) * 5, s));
    CK(cudaMemsetAsync(fb.scal + 6, 0, sizeof(uint64_t) * (kScal - 6), s));
    CK(launch_vertex_setup(*m, ctx->cam, fb, s));
    CK(launch_face_setup(*m, ctx->cam, ctx->style.lod, ctx->style.delta, fb, tiles_x, tiles_y, s));
    CK(scan_u32_to_u64(fb.tile_cnt, fb.tile_off, n_tiles, fb.part, fb.part_max, fb.scal + 8, 0xFFFFFFFFu, s,
                       (uint32_t)kChunk));
    uint64_t h[16] = {};  // pageable host copy of the totals (no pinned allocation)
    CK(cudaMemcpyAsync(h + 8, fb.scal + 8, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t n_bins = h[8];
    fb.bins = a.take<uint32_t>((size_t)n_bins);
    fb.bins_tmp = a.take<uint32_t>((size_t)n_bins);
    fb.masks = a.take<uint32_t>((size_t)n_bins * (kTilePix / kChunk));
    fb.seg = a.take<uint64_t>((size_t)(n_bins / kChunk) * (kTilePix / 32));
    hexfc_frame_stats fs{};
    fs.bin_entries = n_bins;
    fs.width = (uint32_t)win.w;
    fs.height = (uint32_t)win.h;
    if (!fb.bins || !fb.bins_tmp || !fb.masks || !fb.seg) {
        if (stats) *stats = fs;
        return HEXFC_ERR_OVERFLOW;
    }
    CK(cudaMemsetAsync(fb.bins, 0xFF, sizeof(uint32_t) * (size_t)n_bins, s));   // padding slots = kPadBin
    CK(launch_bin_fill(*m, fb, tiles_x, W, H, ctx->reverse_bins, s));
    CK(launch_bin_sort(*m, fb, tiles_x, tiles_y, ctx->depth_buckets, s));
    CK(launch_tile_order(fb, n_tiles, s));
    CK(launch_count(*m, fb, tiles_x, tiles_y, W, H, false, s));
    CK(scan_u32_to_u64(fb.cnt, fb.off, n_pix, fb.part, fb.part_max, fb.scal, (uint32_t)kWarpSortMax, s));
    CK(cudaMemcpyAsync(h, fb.scal, 6 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h[5] != 0) {   // this call's count pass, or the previous call's fill or composite
        CK(cudaMemsetAsync(fb.scal + 5, 0, sizeof(uint64_t), s));
        CK(cudaStreamSynchronize(s));
        if (stats) *stats = fs;
        return device_error_status(h[5]);
    }
    const uint64_t total = h[0];
    const uint32_t n_long = (uint32_t)h[2];
    fs.fragments = total;
    fs.max_list = (uint32_t)h[1];
    fs.long_lists = n_long;
    fs.kernel_launches = 15 + (n_long > 0 ? 1u : 0u) + (sil ? 2u : 0u);
    if (stats) *stats = fs;
    if (fs.max_list > HEXFC_MAX_LIST) return HEXFC_ERR_OVERFLOW;
    fb.key = a.take<uint64_t>((size_t)total);
    fb.rgba = a.take<float4>((size_t)total);
    if (!fb.key || !fb.rgba) return HEXFC_ERR_OVERFLOW;
    fb.frag_cap = (int64_t)total;
    ShadeParams sp = make_shade(ctx);
    if (sil) CK(cudaMemsetAsync(fb.zsil, 0xFF, sizeof(uint32_t) * (size_t)n_pix, s));
    CK(launch_fill(*m, fb, sp, tiles_x, tiles_y, W, H, false, sil, s));
    CK(launch_composite(fb, sp, tiles_x, tiles_y, W, H, out, n_long, ctx->window, win, s));
    if (sil)
        CK(launch_silhouette(fb, tiles_x, ctx->cam.ox, ctx->cam.oy, ctx->view.width, ctx->view.height,
                             ctx->style.sil_alpha, ctx->style.sil_threshold, out, win, s));
    return inject_error_bits(ctx, fb.scal, s);
}

}  // namespace

extern "C" hexfc_status hexfc_render_noalloc(hexfc_ctx* ctx, int32_t mesh, float* out_rgba,
                                             hexfc_frame_stats* stats, void* stream)
{
    if (!ctx || !out_rgba) return HEXFC_ERR_ARG;
    DevMesh* m = get_mesh(ctx, mesh);
    if (!m || !ctx->have_view) return HEXFC_ERR_STATE;
    DeviceGuard g(ctx->device);
    if (ctx->pend.active) {
        const hexfc_status st = finish_pending(ctx);
        if (st != HEXFC_OK) return st;
    }
    return render_frame_noalloc(ctx, m, out_rgba, stats, (cudaStream_t)stream);
}

// Fill pass of the renderer.
//
//   k_fill          per tile: every covered sample (from the count pass's
//                   masks) gets its exact depth, is shaded with Eqs. 1-4 and
//                   written into its warp's region of the fragment arrays.
//                   With capacities chosen before the frame, k_fill lays
//                   out each tile's lists in the tile's region itself (no
//                   pixel scan, no host wait between count and fill).
//
// Each face is drawn as two triangles (Section "Method Overview"; Section "GPU
// Implementation"), all covered samples are kept (per-pixel fragment lists,
// Section "GPU Implementation"), and the fragment shader computes focus from
// the lens, the edge distance to the four face edges ignoring invisible ones,
// and Eqs. 1-4 (Section "Focus+Context").
#include "count_tiles.cuh"
#include "shade.cuh"

namespace hexfc {
namespace {

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------ fill + shade

// Both records of a face as the producer stages them in shared memory: the
// 64 bytes of FaceFrame, the 64 bytes of FaceStatic, and 16 bytes of padding
// that make the stride 9 x 16 bytes. Each lane copies and reads its own
// record 16 bytes at a time; with an odd stride in 16-byte units the lanes of
// each quarter warp touch different banks (a 128-byte stride put all 32
// lanes on the same four banks).
struct RawFace {
    int4 X, Y;      // FaceFrame
    uint4 Z;
    float4 ed;
    float4 imp;     // FaceStatic
    float4 px, py, pz;
    int4 pad;
};
static_assert(sizeof(FaceFrame) == 64 && sizeof(FaceStatic) == 64, "face records of 4 x 16 bytes");
static_assert(sizeof(RawFace) == 144, "record stride of 9 x 16 bytes");

// Producer lane: fetch the records of face f into shared memory.
__device__ __forceinline__ void rec_fetch(RawFace& r, const FaceFrame* __restrict__ fframe,
                                          const FaceStatic* __restrict__ fstat, uint32_t f)
{
    const int4* a = reinterpret_cast<const int4*>(fframe + f);
    const int4* b = reinterpret_cast<const int4*>(fstat + f);
    int4* dst = reinterpret_cast<int4*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cp_async16(dst + k, a + k);
        cp_async16(dst + 4 + k, b + k);
    }
}

// Producer lane j: the shading and depth inputs of triangle t (coverage setup
// already in c) into its record.
__device__ __forceinline__ void stage_shade(const RawFace& r, uint32_t f2t, const TriGeom& t, const ShadeParams& sp,
                                            const CovSoA& c, ShadeRec& R, int j)
{
    const int32_t FX[4] = {r.X.x, r.X.y, r.X.z, r.X.w}, FY[4] = {r.Y.x, r.Y.y, r.Y.z, r.Y.w};
    float il[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int k1 = (k + 1) & 3;
        const int32_t ex = FX[k1] - FX[k], ey = FY[k1] - FY[k];
        const float l2 = u64_to_f32((uint64_t)((int64_t)ex * ex + (int64_t)ey * ey));
        il[k] = l2 > 0.f ? 1.f / l2 : 0.f;
    }
    // |coordinate| <= 2^22: exact in float
    R.fx = make_float4((float)FX[0], (float)FX[1], (float)FX[2], (float)FX[3]);
    R.fy = make_float4((float)FY[0], (float)FY[1], (float)FY[2], (float)FY[3]);
    R.il = make_float4(il[0], il[1], il[2], il[3]);
    const uint32_t zz[4] = {r.Z.x & kZ24, r.Z.y & kZ24, r.Z.z & kZ24, r.Z.w & kZ24};
    const float ee[4] = {r.ed.x, r.ed.y, r.ed.z, r.ed.w}, ii[4] = {r.imp.x, r.imp.y, r.imp.z, r.imp.w};
    const float xx[4] = {r.px.x, r.px.y, r.px.z, r.px.w}, yy[4] = {r.py.x, r.py.y, r.py.z, r.py.w};
    const float ww[4] = {r.pz.x, r.pz.y, r.pz.z, r.pz.w};
    const bool ortho = sp.ortho != 0;
    uint32_t z[3];
    float q[3], a[3], P[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int cc = t.vi[k];
        // select corner cc without dynamic register indexing
        z[k] = cc == 0 ? zz[0] : cc == 1 ? zz[1] : cc == 2 ? zz[2] : zz[3];
        q[k] = ortho ? 1.f : 1.f / (cc == 0 ? ee[0] : cc == 1 ? ee[1] : cc == 2 ? ee[2] : ee[3]);
        a[k] = (cc == 0 ? ii[0] : cc == 1 ? ii[1] : cc == 2 ? ii[2] : ii[3]) * q[k];
        // offset from the sphere lens centre (unused by the screen lens)
        P[k][0] = ((cc == 0 ? xx[0] : cc == 1 ? xx[1] : cc == 2 ? xx[2] : xx[3]) - sp.lens_c[0]) * q[k];
        P[k][1] = ((cc == 0 ? yy[0] : cc == 1 ? yy[1] : cc == 2 ? yy[2] : yy[3]) - sp.lens_c[1]) * q[k];
        P[k][2] = ((cc == 0 ? ww[0] : cc == 1 ? ww[1] : cc == 2 ? ww[2] : ww[3]) - sp.lens_c[2]) * q[k];
    }
    R.qa = make_float4(q[0], q[1] - q[0], q[2] - q[0], a[0]);
    R.ap = make_float4(a[1] - a[0], a[2] - a[0], P[0][0], P[0][1]);
    R.pp = make_float4(P[0][2], P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]);
    R.pq = make_float4(P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2], 0.f);
    R.zm = make_uint4(z[0], z[1], z[2], face_edge_flags(r.Z) | (face_boundary(r.Z) << 8));
    // the edge functions of vertices 1 and 2 moved from the box origin to the
    // tile's first sample (low words: exact modulo 2^32, and at a covered
    // sample of a small triangle the value itself lies in [0, area]); depth
    // differences below 2^24 in magnitude: exact in float
    const int bx = c.box[j];
    const uint32_t ox = (uint32_t)box_lx0(bx) << 8, oy = (uint32_t)box_ly0(bx) << 8;
    const uint32_t w1 = (uint32_t)c.e0[1][j] - (uint32_t)c.dx[1][j] * oy + (uint32_t)c.dy[1][j] * ox;
    const uint32_t w2 = (uint32_t)c.e0[2][j] - (uint32_t)c.dx[2][j] * oy + (uint32_t)c.dy[2][j] * ox;
    R.wd = make_uint4(w1, w2, __float_as_uint((float)(int32_t)(z[1] - z[0])), __float_as_uint((float)(int32_t)(z[2] - z[0])));
    R.ev = make_int4(c.dx[1][j], c.dy[1][j], c.dx[2][j], c.dy[2][j]);
    R.hd = make_uint4((uint32_t)c.box[j], f2t, t.area < (1ll << 26) ? (uint32_t)t.area : 0u,
                      __float_as_uint(1.f / u64_to_f32((uint64_t)t.area)));
}

// A ring slot: the coverage setup and the shading inputs of one chunk.
struct FillSlot {
    CovSoA c;
    ShadeRec sh[kChunk];
    int64_t area[kChunk];   // twice the area (16.8 squared)
};

// Warp queues of covered samples: entry = j | pixel << 5 | ring slot << 13 | counted << 16.
constexpr int kWQ = 256;               // entries per consumer warp (a power of two)
constexpr int kWQWin = kWQ - 32;       // entries queued per window: fewer than 32 leftovers + a window fit
constexpr uint32_t kCounted = 1u << 16;  // the count pass sized the sample's list for it
constexpr unsigned long long kErrPool = 16ull;   // error bit: no room for a tile's lists (chosen capacities)
static_assert(kRing <= 8, "three bits of ring slot");

constexpr size_t kRawOff = (kRing * sizeof(FillSlot) + 127) & ~(size_t)127;   // face records: 128-aligned

__host__ __device__ constexpr size_t fill_smem_bytes()
{
    return kRawOff + 2 * kChunk * sizeof(RawFace) + (size_t)kConsumerWarps * kWQ * sizeof(uint32_t);
}

// The fill pipeline of one tile block: s_base / s_len hold the offsets and
// lengths of the tile's 256 lists, the ring barriers are initialised, and
// `smem` is the dynamic shared memory (fill_smem_bytes()).
template <bool kSil>
__device__ __forceinline__ void fill_tile(unsigned char* smem, const uint64_t* s_base, const uint32_t* s_len,
                                          uint64_t* s_full, uint64_t* s_empty,
                                          const uint32_t* __restrict__ bins, const uint32_t* __restrict__ masks,
                                          const FaceFrame* __restrict__ fframe,
                                          const FaceStatic* __restrict__ fstat, uint64_t beg, uint32_t n_chunks,
                                          int px0, int py0, int W, int H, const ShadeParams& sp,
                                          uint64_t* __restrict__ key, float4* __restrict__ rgba,
                                          uint64_t* __restrict__ seg, unsigned long long* __restrict__ err,
                                          uint32_t* __restrict__ zsil_t)
{
    FillSlot* s_ring = reinterpret_cast<FillSlot*>(smem);                                    // [kRing]
    RawFace* s_raw = reinterpret_cast<RawFace*>(smem + kRawOff);                            // [2][kChunk]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == kConsumerWarps) {  // producer
        uint32_t f2t_c = n_chunks > 0 ? bins[beg + lane] : kPadBin;
        uint32_t f2t_n = n_chunks > 1 ? bins[beg + kChunk + lane] : kPadBin;
        if (f2t_c != kPadBin) rec_fetch(s_raw[lane], fframe, fstat, f2t_c >> 1);
        cp_async_commit();
        for (uint32_t c = 0; c < n_chunks; ++c) {
            const int s = c % kRing;
            uint32_t f2t_nn = kPadBin;
            if (c + 1 < n_chunks) {
                if (f2t_n != kPadBin) rec_fetch(s_raw[((c + 1) & 1) * kChunk + lane], fframe, fstat, f2t_n >> 1);
                if (c + 2 < n_chunks) f2t_nn = bins[beg + (uint64_t)(c + 2) * kChunk + lane];
            }
            cp_async_commit();
            cp_async_wait<1>();   // this lane's copies of chunk c have landed
            if (!mbar_wait(&s_empty[s], ((c / kRing) & 1) ^ 1)) {
                if (lane == 0) atomicOr(err, kErrWait);
                break;
            }
            FillSlot& S = s_ring[s];
            if (f2t_c != kPadBin) {
                const RawFace& r = s_raw[(c & 1) * kChunk + lane];
                TriGeom t;
                stage_cov(r.X, r.Y, f2t_c, W, H, px0, py0, S.c, lane, t);
                if (S.c.box[lane] != 0) {
                    stage_shade(r, f2t_c, t, sp, S.c, S.sh[lane], lane);
                    S.area[lane] = t.area;
                }
            } else {
                S.c.box[lane] = 0;
            }
            mbar_arrive(&s_full[s]);
            f2t_c = f2t_n;
            f2t_n = f2t_nn;
        }
        cp_async_wait<0>();
        return;
    }
    // consumers: warp w owns pixels 32w .. 32w + 31 and a private queue; each
    // warp goes through the chunks on its own (no block barrier), so warps
    // may be up to kRing chunks apart
    const int p = threadIdx.x;
    uint32_t* s_q = reinterpret_cast<uint32_t*>(s_raw + 2 * kChunk) + warp * kWQ;   // [kWQ]
    uint32_t k_run = 0;
    bool bad = false, stalled = false;
    // The warp's 32 lists are one region of the fragment arrays, from the
    // offset of its first pixel; the region holds them chunk-major (fragment
    // e of the warp's queue at region start + e), so every shading round
    // writes 32 consecutive records.
    const uint64_t w_beg = s_base[warp * 32];
    const uint32_t w_len = __reduce_add_sync(0xffffffffu, s_len[p]);
    // Queue positions are absolute counts (modulo kWQ): entries [head, tail) are
    // queued. Only whole rounds of 32 entries are shaded; the rest waits for
    // the next chunk unless it would keep an older chunk's slot (then it is
    // shaded as a partial round), so at most the newest chunk's slot is held.
    uint32_t head = 0, tail = 0, released = 0;
    auto shade_entry = [&](uint32_t qe, uint32_t e) {
        if (!(qe & kCounted) || e >= w_len) return;
        const int j = (int)(qe & 31u);
        const uint32_t pl = (qe >> 5) & 255u;
        const FillSlot& S = s_ring[(qe >> 13) & 7u];
        const int lx = (int)(pl % kTileW), ly = (int)(pl / kTileW);
        const ShadeRec& R = S.sh[j];
        const uint4 hd = R.hd, zm = R.zm, wd = R.wd;
        const int4 ev = R.ev;
        // exact weights of vertices 1 and 2 (edge functions opposite them)
        const uint32_t sx8 = (uint32_t)lx << 8, sy8 = (uint32_t)ly << 8;
        const float ia = __uint_as_float(hd.w);
        const float dz1 = __uint_as_float(wd.z), dz2 = __uint_as_float(wd.w);
        float lam1, lam2;
        uint32_t z;
        if (hd.z != 0) {   // 0 <= l <= area < 2^26: the weights in 32-bit arithmetic (exact mod 2^32)
            const uint32_t l1 = wd.x + (uint32_t)ev.x * sy8 - (uint32_t)ev.y * sx8;
            const uint32_t l2 = wd.y + (uint32_t)ev.z * sy8 - (uint32_t)ev.w * sx8;
            lam1 = (float)l1 * ia;
            lam2 = (float)l2 * ia;
            z = sample_depth_small(zm.x, zm.y, zm.z, l1, l2, hd.z, lam1, lam2, dz1, dz2, bad);
        } else {
            const int64_t area = S.area[j];
            const int bx = (int)hd.x;
            const int32_t sxr = (lx - box_lx0(bx)) << 8, syr = (ly - box_ly0(bx)) << 8;
            const int64_t l1 = S.c.e0[1][j] + (int64_t)ev.x * syr - (int64_t)ev.y * sxr;
            const int64_t l2 = S.c.e0[2][j] + (int64_t)ev.z * syr - (int64_t)ev.w * sxr;
            lam1 = u64_to_f32((uint64_t)l1) * ia;
            lam2 = u64_to_f32((uint64_t)l2) * ia;
            z = sample_depth_lam(zm.x, zm.y, zm.z, l1, l2, area, lam1, lam2, dz1, dz2, bad);
        }
        const float4 col = shade_fragment(R, zm.w, lam1, lam2, px0 + lx, py0 + ly, sp);
        const uint64_t o = w_beg + e;
        key[o] = ((uint64_t)z << 32) | (uint64_t)hd.y;
        rgba[o] = col;
        // the boundary surface's depth image (silhouettes): nearest boundary fragment
        if constexpr (kSil) {
            if (zm.w & 0x100u) atomicMin(zsil_t + pl, z);
        }
    };
    // masks of the next two chunks are in flight while this one is shaded
    const uint32_t* mp = masks + (beg / kChunk) * kTilePix + p;             // this pixel's mask of chunk 0
    uint64_t* sgp = seg + (beg / kChunk) * kConsumerWarps + warp;           // this group's run of chunk 0
    uint32_t mk_a = n_chunks > 0 ? mp[0] : 0u;
    uint32_t mk_b = n_chunks > 1 ? mp[kTilePix] : 0u;
    for (uint32_t c = 0; c < n_chunks; ++c) {
        const int s = c % kRing;
        const uint32_t mk = mk_a;
        mk_a = mk_b;
        if (c + 2 < n_chunks) mk_b = mp[(size_t)(c + 2) * kTilePix];
        // every entry of the chunks before c - 1 (and of c - 1 if nothing is
        // left over) has been shaded by the whole warp: release their slots
        __syncwarp();
        const uint32_t rel_to = head == tail ? c : c - 1;
        if (lane == 0)
            for (uint32_t r = released; r < rel_to; ++r) mbar_arrive(&s_empty[r % kRing]);
        released = max(released, rel_to);
        if (!__all_sync(0xffffffffu, mbar_wait(&s_full[s], (c / kRing) & 1))) {
            if (lane == 0) atomicOr(err, kErrWait);
            stalled = true;
            break;
        }
        // warp exclusive scan of the hit counts
        const uint32_t h = __popc(mk);
        uint32_t incl = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const bool fits = k_run + h <= s_len[p];   // the count pass sized this list
        bad = bad || !fits;
        const uint32_t chunk_start = tail;
        if (lane == 0) sgp[(size_t)c * kConsumerWarps] = w_beg + chunk_start;
        const uint32_t tag = ((uint32_t)p << 5) | ((uint32_t)s << 13) | (fits ? kCounted : 0u);
        for (uint32_t w0 = 0; w0 < total; w0 += kWQWin) {
            uint32_t m2 = mk, r = incl - h;
            if (total <= (uint32_t)kWQWin) {   // one window: every entry is queued
                uint32_t pos = tail + r;
                while (m2) {
                    s_q[pos++ & (kWQ - 1)] = (__ffs(m2) - 1) | tag;
                    m2 &= m2 - 1;
                }
            } else {
                while (m2) {
                    const uint32_t j = __ffs(m2) - 1;
                    m2 &= m2 - 1;
                    if (r >= w0 && r < w0 + kWQWin) s_q[(tail + r - w0) & (kWQ - 1)] = j | tag;
                    ++r;
                }
            }
            __syncwarp();   // the window's entries are queued
            tail += min((uint32_t)kWQWin, total - w0);
            const uint32_t rounds = (tail - head) / 32;
            for (uint32_t i = 0; i < rounds; ++i) {
                const uint32_t e = head + i * 32 + lane;
                shade_entry(s_q[e & (kWQ - 1)], e);
            }
            head += rounds * 32;
            __syncwarp();   // shaded entries are read before the next window overwrites them
        }
        if (head < chunk_start) {   // leftovers of an older chunk: shade them all now
            if (lane < tail - head) shade_entry(s_q[(head + lane) & (kWQ - 1)], head + lane);
            head = tail;
        }
        k_run += h;
    }
    // the last leftovers (the producer is done; no slot is released any more)
    if (!stalled && lane < tail - head) shade_entry(s_q[(head + lane) & (kWQ - 1)], head + lane);
    if (bad) atomicOr(err, 1ull);
}

// Per tile: the coverage masks of the count pass give, chunk by chunk, each
// pixel's covered triangles; each consumer warp compacts its 32 pixels'
// covered samples into its queue (pixel-major, in list order) and shades it
// 32 samples at a time, so that every lane has work, writing the fragments in
// queue order into the warp's region (the 32 lists the count pass sized):
// chunk by chunk, pixel by pixel within a chunk. The producer fetches the face
// records of chunk c+1 with cp.async while it sets up chunk c. Three blocks
// per SM leave 72 registers a thread: a sample's inputs arrive as eleven
// 16-byte vectors, more values live at once than at four blocks (56
// registers), where they spill.
template <bool kSil>
__global__ void __launch_bounds__(kPipeThreads, 3) k_fill(const uint64_t* __restrict__ tile_off,
                                                          const uint32_t* __restrict__ bins,
                                                          uint32_t* __restrict__ masks,
                                                          const FaceFrame* __restrict__ fframe,
                                                          const FaceStatic* __restrict__ fstat,
                                                          const uint32_t* __restrict__ order, int tiles_x, int W,
                                                          int H, ShadeParams sp, const uint64_t* __restrict__ off,
                                                          uint32_t* __restrict__ cnt,
                                                          uint64_t* __restrict__ key, float4* __restrict__ rgba,
                                                          uint64_t* __restrict__ seg,
                                                          unsigned long long* __restrict__ err,
                                                          const uint64_t* __restrict__ cap_off,
                                                          const uint32_t* __restrict__ tile_frag, int n_tiles,
                                                          uint64_t frag_cap, unsigned long long* __restrict__ scal,
                                                          uint32_t* __restrict__ zsil)
{
    extern __shared__ __align__(128) unsigned char fill_smem[];
    __shared__ uint64_t s_base[kTilePix];
    __shared__ uint32_t s_len[kTilePix];
    __shared__ uint32_t s_wsum[kConsumerWarps];
    __shared__ uint64_t s_tile_base;
    __shared__ __align__(8) uint64_t s_full[kRing], s_empty[kRing];
    const int tile = (int)order[blockIdx.x];
    const int px0 = (tile % tiles_x) * kTileW, py0 = (tile / tiles_x) * kTileH;
    const uint64_t beg = tile_off[tile], end = tile_off[tile + 1];  // multiples of kChunk
    const uint32_t n_chunks = (uint32_t)((end - beg) / kChunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)tile * kTilePix + threadIdx.x;
    if (!cap_off) {   // offsets from the pixel scan
        if (threadIdx.x < kTilePix) {
            s_base[threadIdx.x] = off[q];
            s_len[threadIdx.x] = cnt[q];
        }
    } else if (threadIdx.x == 0) {
        // capacities chosen before the frame: the tile's lists are laid out in its
        // region [cap_off[t], cap_off[t+1]), or in the pool after all regions
        // (scal[14] records taken, scal[6] tiles) if they do not fit (the tile's
        // exact total is the count pass's); with no room left there the tile is
        // not drawn (error bit kErrPool)
        const uint64_t total = tile_frag[tile];
        const uint64_t region = cap_off[tile];
        uint64_t b = region;
        if (region + total > cap_off[tile + 1] || region + total > frag_cap) {
            const uint64_t p = atomicAdd(&scal[14], (unsigned long long)total);
            atomicAdd(&scal[6], 1ull);
            b = cap_off[n_tiles] + p;
            if (b + total > frag_cap) {
                atomicOr(err, kErrPool);
                b = ~0ull;
            }
        }
        s_tile_base = b;
    }
    pipe_init(s_full, s_empty);   // (its block barrier publishes s_tile_base, s_base, s_len)
    if (cap_off) {
        if (s_tile_base == ~0ull) {   // no room: the frame is drawn again exactly
            // the resolve must find no fragment here: clear the tile's masks and counts
            uint32_t* mt = masks + (beg / kChunk) * kTilePix;
            for (uint32_t i = threadIdx.x; i < n_chunks * kTilePix; i += blockDim.x) mt[i] = 0u;
            if (threadIdx.x < kTilePix) cnt[q] = 0u;
            return;
        }
        if (threadIdx.x < kTilePix) {
            // the consumers lay out the tile's lists (a scan of the counts over the
            // 256 pixels, consumer warps only: named barrier 1) while the producer
            // starts on the first chunks
            const uint32_t n = cnt[q];
            uint32_t incl = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_wsum[warp] = incl;
            asm volatile("bar.sync 1, %0;" ::"n"(kTilePix) : "memory");
            uint32_t pre = 0;
            for (int w = 0; w < warp; ++w) pre += s_wsum[w];
            s_base[threadIdx.x] = s_tile_base + pre + incl - n;
            s_len[threadIdx.x] = n;
            __syncwarp();
        }
    }
    fill_tile<kSil>(fill_smem, s_base, s_len, s_full, s_empty, bins, masks, fframe, fstat, beg, n_chunks, px0, py0,
                    W, H, sp, key, rgba, seg, err, kSil ? zsil + (int64_t)tile * kTilePix : nullptr);
}

// The fill of several frames in one grid (a batch; offsets from each frame's
// pixel scan).
template <bool kSil>
__global__ void __launch_bounds__(kPipeThreads, 3) k_fill_batch(const __grid_constant__ FillBatch b)
{
    extern __shared__ __align__(128) unsigned char fill_smem[];
    __shared__ uint64_t s_base[kTilePix];
    __shared__ uint32_t s_len[kTilePix];
    __shared__ __align__(8) uint64_t s_full[kRing], s_empty[kRing];
    __shared__ FillItem s_it;   // the frame's pointers and constants, read from shared memory
    const int i = batch_item(b.tile_begin, b.n, blockIdx.x);
    const int tile = (int)b.it[i].order[blockIdx.x - b.tile_begin[i]];
    if (threadIdx.x == 0) s_it = b.it[i];
    __syncthreads();
    const FillItem& it = s_it;
    const int px0 = (tile % it.tiles_x) * kTileW, py0 = (tile / it.tiles_x) * kTileH;
    const uint64_t beg = it.tile_off[tile], end = it.tile_off[tile + 1];
    const uint32_t n_chunks = (uint32_t)((end - beg) / kChunk);
    const int64_t q = (int64_t)tile * kTilePix + threadIdx.x;
    if (threadIdx.x < kTilePix) {
        s_base[threadIdx.x] = it.off[q];
        s_len[threadIdx.x] = it.cnt[q];
    }
    pipe_init(s_full, s_empty);
    fill_tile<kSil>(fill_smem, s_base, s_len, s_full, s_empty, it.bins, it.masks, it.fframe, it.fstat, beg, n_chunks,
                    px0, py0, it.W, it.H, it.sp, it.key, it.rgba, it.seg, it.err,
                    kSil ? it.zsil + (int64_t)tile * kTilePix : nullptr);
}

// Capacities from the previous frame's exact tile counts: prev * (1 + margin)
// + pad; or, given a uniform count (> 0), that count for every tile instead.
__global__ void k_capacity_from_previous(const uint32_t* __restrict__ prev, int64_t n_tiles, float margin,
                                         uint32_t pad, uint32_t uniform, uint32_t* __restrict__ cap)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const float c = uniform ? (float)uniform : (float)prev[t];
    cap[t] = (uint32_t)fminf(c * (1.f + margin) + (float)pad, 4.0e9f);
}

}  // namespace

cudaError_t prepare_fill_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_fill<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fill_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fill<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fill_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fill_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fill_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fill_smem_bytes());
    return e;
}

cudaError_t launch_fill_batch(const FillBatch& b, bool sil, cudaStream_t s)
{
    if (b.n == 0 || b.tile_begin[b.n] == 0) return cudaSuccess;
    if (sil) k_fill_batch<true><<<b.tile_begin[b.n], kPipeThreads, fill_smem_bytes(), s>>>(b);
    else k_fill_batch<false><<<b.tile_begin[b.n], kPipeThreads, fill_smem_bytes(), s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_capacity_from_previous(FrameBufs& fb, int64_t n_tiles, float margin, uint32_t pad, uint32_t uniform,
                                          cudaStream_t s)
{
    k_capacity_from_previous<<<grid_for(n_tiles, 256), 256, 0, s>>>(fb.tile_frag, n_tiles, margin, pad, uniform,
                                                                     fb.tile_cap);
    return cudaGetLastError();
}

cudaError_t launch_fill(const DevMesh& m, FrameBufs& fb, const ShadeParams& sp, int tiles_x, int tiles_y, int W,
                        int H, bool regions, bool sil, cudaStream_t s)
{
    const size_t smem = fill_smem_bytes();
    auto go = [&](auto kernel) {   // with silhouettes, the variant that records the boundary depths
        kernel<<<(unsigned)(tiles_x * tiles_y), kPipeThreads, smem, s>>>(
            fb.tile_off, fb.bins, fb.masks, fb.fframe, m.fstat, fb.tile_order, tiles_x, W, H, sp, fb.off, fb.cnt,
            fb.key, fb.rgba, fb.seg, reinterpret_cast<unsigned long long*>(fb.scal + 5),
            regions ? fb.cap_off : nullptr, fb.tile_frag, tiles_x * tiles_y, (uint64_t)fb.frag_cap,
            reinterpret_cast<unsigned long long*>(fb.scal), sil ? fb.zsil : nullptr);
    };
    if (sil) go(k_fill<true>);
    else go(k_fill<false>);
    return cudaGetLastError();
}

}  // namespace hexfc

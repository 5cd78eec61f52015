// New-view rendering at the views' own resolution (out_w = W, out_h = H), the
// interactive case of Section 3.6, with the on-demand decode shared between
// views.
//
// Every new camera (u, v) inside grid cell (i0, j0) blends the same four
// neighbour views (i0, j0), (i0+1, j0), (i0, j0+1), (i0+1, j0+1).  One CTA owns
// one cell and one 64 x 16 output tile: it collects the requested views that
// fall in its cell, decodes from the compressed stream only the blocks of the
// four neighbours that those views sample for this tile, and renders the tile
// of every such view.  At native size the ray of output pixel x lands at
// x + d (i - u) in neighbour i, a shift that is constant over the tile, so
// each neighbour contributes a fixed 2 x 2 stencil with four fixed weights.
//
// Phases per CTA (views handled in groups whose shifted windows fit shared
// memory):
//  1. collect the cell's views; per neighbour k the union of their integer
//     shifts fixes a padded window of the tile, and its clamp to the image a
//     source rectangle;
//  2. one thread per (block location, channel) walks the location's record
//     once, in BFS order, and tables the payload offset and header of every
//     node the four neighbours need (their leaves and ancestors);
//  3. one thread per (block location, neighbour) adds the top RKV block and
//     the neighbour's ancestors' residuals for the three channels, converts
//     to RGB and writes the window cells whose clamped position is that pixel
//     (which replicates the image edge as clamp-to-edge sampling does);
//  4. per view, each thread blends one column of 4 pixels, sliding a 2 x 2
//     stencil down the window (lanes read consecutive words, no bank
//     conflicts), and writes with streaming stores.
#include <cuda_runtime.h>

#include <algorithm>

#include "warp_decode.cuh"

namespace rlfc {
namespace {

constexpr int kTW = 64, kTH = 16;       // output tile
constexpr int kThreads = 256;           // one column of kRows pixels per thread
constexpr int kRows = kTH * kTW / kThreads;
constexpr int kListCap = 1024;          // views collected per pass
constexpr int kGroupCap = 64;           // views whose parameters are cached per group
constexpr int kMaxNeed = 4 * kMaxLevels;
constexpr uint32_t kSmemBytes = 64 * 1024;        // decoding on demand: windows + node table
// Decoding first: the windows alone, four CTAs per SM (dynamic + static shared
// memory of four CTAs within the SM's 228 KB)
constexpr uint32_t kSmemDecoded = 48 * 1024;
constexpr int kListCapDecoded = 1024;
constexpr int kGroupCapDecoded = 32;
// Batches of at least this many cameras decode the neighbour views they need
// first (one pass over every record, the needed views only, then a cheap
// blend per camera); smaller ones decode block by block inside the render
// kernel.  Measured on 17 x 17 views of 1024^2: 4 cameras take 0.51 ms the
// first way and 1.0 ms the second; 1 camera 0.37 against 0.27 ms.  Under a
// serving load of many small calls on several streams, decoding first for
// two or three cameras (a full-GPU pass over every record each time)
// saturated the GPU at 5000 requests/s, so the switch sits at four.
constexpr uint32_t kDecodeFirstViews = 4;

__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

struct Args {
    StreamView sv;
    const float *uv;
    const float *disp;
    float *out;
    uint8_t *out8;             // when set, 8-bit RGB goes here instead of out
    const uint32_t *decoded;   // packed RGB views [slot][H][W] decoded for this call, or null
    const uint32_t *slot_of;   // with decoded views: the slot of each view
    uint32_t U, V, W, H, n;
    uint32_t tiles_x, cells_u;
    uint32_t n_tiles;           // tiles per view
    const uint32_t *cell_list;  // the grid cells that hold cameras, *cell_count of them
    const uint32_t *cell_count;
    uint32_t need_max;   // distinct nodes four views can need: 4 (L - 1)
};

struct Shift {
    int ox, oy;       // integer part of the shift
    float fx, fy;     // fractional part
};

__device__ __forceinline__ void camera_axis(float u, uint32_t G, int &i0, float &f)
{
    u = fminf(fmaxf(u, 0.0f), (float)(G - 1));
    if (G == 1) {
        i0 = 0;
        f = 0.0f;
        return;
    }
    i0 = min((int)floorf(u), (int)G - 2);
    f = u - (float)i0;
}

// Cell of view r, its four blend weights and per-neighbour shifts.
__device__ __forceinline__ void view_params(const Args &a, uint32_t r, int &ci, int &cj, float w[4], Shift sh[4])
{
    const float u = fminf(fmaxf(a.uv[2 * r], 0.0f), (float)(a.U - 1));
    const float v = fminf(fmaxf(a.uv[2 * r + 1], 0.0f), (float)(a.V - 1));
    const float d = a.disp[r];
    float fu, fv;
    camera_axis(u, a.U, ci, fu);
    camera_axis(v, a.V, cj, fv);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int ia = k & 1, jb = k >> 1;
        const int i = a.U == 1 ? 0 : ci + ia, j = a.V == 1 ? 0 : cj + jb;
        w[k] = (ia ? fu : 1.0f - fu) * (jb ? fv : 1.0f - fv);
        // a shift beyond twice the image size samples only the clamped edge
        // either way; bounding it keeps the integer pixel arithmetic in range
        const float lim = 2.0f * (float)max(a.W, a.H) + 4.0f;
        const float sx = fminf(fmaxf(d * ((float)i - u), -lim), lim);
        const float sy = fminf(fmaxf(d * ((float)j - v), -lim), lim);
        const float flx = floorf(sx), fly = floorf(sy);
        sh[k].ox = (int)flx;
        sh[k].oy = (int)fly;
        sh[k].fx = sx - flx;
        sh[k].fy = sy - fly;
    }
}

__device__ __forceinline__ uint32_t cell_of(const Args &a, uint32_t r)
{
    const float u = fminf(fmaxf(a.uv[2 * r], 0.0f), (float)(a.U - 1));
    const float v = fminf(fmaxf(a.uv[2 * r + 1], 0.0f), (float)(a.V - 1));
    int ci = 0, cj = 0;
    float f;
    camera_axis(u, a.U, ci, f);
    camera_axis(v, a.V, cj, f);
    return (uint32_t)cj * a.cells_u + (uint32_t)ci;
}

struct Window {
    int wx0, wy0, WX, WY;     // padded window: global pixel origin and size
    int FW;                   // row stride of the window (WX + 1)
    int cx0, cy0, cx1, cy1;   // the window clamped to the image
    int oxmin, oymin;
    uint32_t f_off;           // offset (in 32-bit words) into shared memory
};

// Per view of the current group: the four neighbours' stencil weights (blend
// weight / 255 times the bilinear weights; all zero for an unused neighbour)
// and integer shifts.
struct __align__(16) ViewP {
    float w[4][4];            // [k][00, 10, 01, 11]
    int base[4];              // sample (0, 0) of the view's 2 x 2 stencil in window k
    int16_t ox[4], oy[4];
    uint32_t used;            // bit k: neighbour k has a non-zero weight
};

extern __shared__ __align__(16) uint32_t g_dyn[];

// Shared-memory words of one neighbour's window (two words per pixel) for a
// tile of tw x th pixels with the given shift spreads.
__host__ __device__ __forceinline__ uint32_t window_words(int tw, int th, int sx, int sy)
{
    return 2u * (uint32_t)(tw + 2 + sx) * (uint32_t)(th + 1 + sy);
}

// A window pixel, two words that unpack to floats with one shift or mask
// each (win_r, win_g, win_b): R and G as bf16 halves, B as a float; 8-bit
// values are exact in both.
__device__ __forceinline__ uint2 rgb_window(uint32_t rgb24)
{
    // bf16: R in the low half, G in the high half of one word; B as a full
    // float (8-bit integers have no bits below the top 16)
    const uint32_t r = __float_as_uint((float)(rgb24 & 255u)) >> 16;
    const uint32_t g = __float_as_uint((float)((rgb24 >> 8) & 255u));
    const uint32_t b = __float_as_uint((float)((rgb24 >> 16) & 255u));
    return make_uint2(g | r, b);
}
__device__ __forceinline__ float win_r(uint2 p) { return __uint_as_float(__byte_perm(p.x, 0u, 0x1044)); }   // p.x << 16
__device__ __forceinline__ float win_g(uint2 p) { return __uint_as_float(p.x & 0xFFFF0000u); }
__device__ __forceinline__ float win_b(uint2 p) { return __uint_as_float(p.y); }

// One out-of-line copy of the block decoder keeps the kernel's code small
// enough for the instruction cache.
__device__ __noinline__ void decode_block_values(const uint32_t *rec, uint32_t pos, uint32_t mode, int32_t mn,
                                                 int32_t scale, int32_t acc[kVals])
{
    int32_t u[kVals];
    bise_decode16(rec, pos, mode, u);
#pragma unroll
    for (int v = 0; v < kVals; v++)
        acc[v] += (mn + u[v]) * scale;
}


template <bool kDecoded>
__global__ void __launch_bounds__(kThreads, kDecoded ? 4 : 3) render_native_kernel(const Args a)
{
    constexpr int kLC = kDecoded ? kListCapDecoded : kListCap;
    constexpr int kGC = kDecoded ? kGroupCapDecoded : kGroupCap;
    constexpr uint32_t kSmem = kDecoded ? kSmemDecoded : kSmemBytes;
    __shared__ uint32_t s_mode[kNumModes];
    __shared__ uint16_t s_list[kLC];
    __shared__ ViewP s_vp[kGC];
    __shared__ int s_count, s_gend;
    __shared__ int s_oxmin[4], s_oxmax[4], s_oymin[4], s_oymax[4], s_used[4];
    __shared__ Window s_win[4];
    __shared__ uint32_t s_need_pos[kMaxNeed];
    __shared__ int s_slot_need[4][kMaxLevels];
    __shared__ int s_nneed;
    __shared__ uint32_t s_top[4];
    __shared__ int s_rect[4];          // union block rectangle bx0, by0, nbx, nby
    __shared__ uint32_t s_ent_off;     // word offset of the node table

    const int tid = threadIdx.x;
    if (tid < kNumModes)
        s_mode[tid] = c_modes[tid];
    // with a cell list the CTAs are persistent over (occupied cell, tile)
    // items, cell-major so that neighbouring CTAs read the same neighbour
    // views; otherwise a CTA is the one item (cell blockIdx.y, tile
    // blockIdx.x)
    const bool listed = a.cell_list != nullptr;
    const uint32_t n_items = listed ? *a.cell_count * a.n_tiles : 1u;
    for (uint32_t item = listed ? blockIdx.x : 0u; item < n_items; item += gridDim.x) {
    const uint32_t cell = listed ? a.cell_list[item / a.n_tiles] : blockIdx.y;
    const uint32_t tile = listed ? item % a.n_tiles : blockIdx.x;
    const int ci = (int)(cell % a.cells_u), cj = (int)(cell / a.cells_u);
    const int tx0 = (int)(tile % a.tiles_x) * kTW, ty0 = (int)(tile / a.tiles_x) * kTH;
    const int tw = min(kTW, (int)a.W - tx0), th = min(kTH, (int)a.H - ty0);
    int nview[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int i = a.U == 1 ? 0 : ci + (k & 1), j = a.V == 1 ? 0 : cj + (k >> 1);
        nview[k] = j * (int)a.U + i;
    }

    for (uint32_t base = 0; base < a.n; base += kLC) {
        // ---- phase 1: the views of this cell among [base, base + kLC)
        if (tid == 0)
            s_count = 0;
        __syncthreads();
        const uint32_t lim = min(a.n, base + kLC);
        for (uint32_t r = base + tid; r < lim; r += kThreads)
            if (cell_of(a, r) == cell)
                s_list[atomicAdd(&s_count, 1)] = (uint16_t)r;
        __syncthreads();
        const int count = s_count;
        for (int g0 = 0; g0 < count;) {
            // ---- per-view parameters of the next group, in parallel
            const int gcap = min(kGC, count - g0);
            if (tid < 4) {
                s_oxmin[tid] = s_oymin[tid] = INT_MAX;
                s_oxmax[tid] = s_oymax[tid] = INT_MIN;
                s_used[tid] = 0;
            }
            __syncthreads();
            if (tid < gcap) {
                int c1, c2;
                float w[4];
                Shift sh[4];
                view_params(a, s_list[g0 + tid], c1, c2, w, sh);
                ViewP &vp = s_vp[tid];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float wk = w[k] * (1.0f / 255.0f);
                    vp.w[k][0] = wk * (1.0f - sh[k].fx) * (1.0f - sh[k].fy);
                    vp.w[k][1] = wk * sh[k].fx * (1.0f - sh[k].fy);
                    vp.w[k][2] = wk * (1.0f - sh[k].fx) * sh[k].fy;
                    vp.w[k][3] = wk * sh[k].fx * sh[k].fy;
                    vp.ox[k] = (int16_t)sh[k].ox;
                    vp.oy[k] = (int16_t)sh[k].oy;
                    if (k == 0)
                        vp.used = 0;
                    if (w[k] != 0.0f)
                        vp.used |= 1u << k;
                }
            }
            if (tid < kGC) {
                // group extents per neighbour: warp reductions, one atomic per warp
                const bool mine = tid < gcap;
                const ViewP &vp = s_vp[mine ? tid : 0];
                for (int k = 0; k < 4; k++) {
                    const int lo_x = __reduce_min_sync(kFullMask, mine ? (int)vp.ox[k] : INT_MAX);
                    const int hi_x = __reduce_max_sync(kFullMask, mine ? (int)vp.ox[k] : INT_MIN);
                    const int lo_y = __reduce_min_sync(kFullMask, mine ? (int)vp.oy[k] : INT_MAX);
                    const int hi_y = __reduce_max_sync(kFullMask, mine ? (int)vp.oy[k] : INT_MIN);
                    const unsigned used = __reduce_or_sync(kFullMask, mine ? (vp.used >> k) & 1u : 0u);
                    if ((tid & 31) == 0 && (tid < gcap)) {
                        atomicMin(&s_oxmin[k], lo_x);
                        atomicMax(&s_oxmax[k], hi_x);
                        atomicMin(&s_oymin[k], lo_y);
                        atomicMax(&s_oymax[k], hi_y);
                        if (used)
                            atomicOr(&s_used[k], 1);
                    }
                }
            }
            __syncthreads();
            if (tid == 0) {
                // exact shared-memory words of the windows plus the node table
                auto fits = [&](const int *oxl, const int *oxh, const int *oyl, const int *oyh, const int *used) {
                    uint32_t words = 0;
                    int bx0 = INT_MAX, by0 = INT_MAX, bx1 = INT_MIN, by1 = INT_MIN;
                    for (int k = 0; k < 4; k++) {
                        words += window_words(tw, kTH, oxh[k] - oxl[k], oyh[k] - oyl[k]);
                        if (!used[k])
                            continue;
                        bx0 = min(bx0, min(max(tx0 + oxl[k], 0), (int)a.W - 1) / kBlock);
                        bx1 = max(bx1, min(max(tx0 + tw + oxh[k], 0), (int)a.W - 1) / kBlock);
                        by0 = min(by0, min(max(ty0 + oyl[k], 0), (int)a.H - 1) / kBlock);
                        by1 = max(by1, min(max(ty0 + th + oyh[k], 0), (int)a.H - 1) / kBlock);
                    }
                    words = (words + 3) & ~3u;
                    if (!kDecoded)
                        words += (uint32_t)((bx1 - bx0 + 1) * (by1 - by0 + 1) * 3 * 2) * a.need_max;
                    return words * 4 <= kSmem;
                };
                int ge = g0 + gcap;
                if (!fits(s_oxmin, s_oxmax, s_oymin, s_oymax, s_used)) {
                    // rare (a large disparity spread): the longest prefix that fits
                    int oxl[4], oxh[4], oyl[4], oyh[4], used[4];
                    for (int k = 0; k < 4; k++) {
                        oxl[k] = oyl[k] = INT_MAX;
                        oxh[k] = oyh[k] = INT_MIN;
                        used[k] = 0;
                    }
                    ge = g0;
                    while (ge < g0 + gcap) {
                        const ViewP &vp = s_vp[ge - g0];
                        int nl[4], nh[4], ml[4], mh[4], nu[4];
                        for (int k = 0; k < 4; k++) {
                            nl[k] = min(oxl[k], (int)vp.ox[k]);
                            nh[k] = max(oxh[k], (int)vp.ox[k]);
                            ml[k] = min(oyl[k], (int)vp.oy[k]);
                            mh[k] = max(oyh[k], (int)vp.oy[k]);
                            nu[k] = used[k] | (vp.w[k][0] != 0.0f || vp.w[k][1] != 0.0f || vp.w[k][2] != 0.0f ||
                                               vp.w[k][3] != 0.0f);
                        }
                        if (ge > g0 && !fits(nl, nh, ml, mh, nu))
                            break;
                        for (int k = 0; k < 4; k++) {
                            oxl[k] = nl[k];
                            oxh[k] = nh[k];
                            oyl[k] = ml[k];
                            oyh[k] = mh[k];
                            used[k] = nu[k];
                        }
                        ge++;
                    }
                    for (int k = 0; k < 4; k++) {
                        s_oxmin[k] = oxl[k];
                        s_oxmax[k] = oxh[k];
                        s_oymin[k] = oyl[k];
                        s_oymax[k] = oyh[k];
                        s_used[k] = used[k];
                    }
                }
                s_gend = ge;
                uint32_t off = 0;
                int bx0 = INT_MAX, by0 = INT_MAX, bx1 = INT_MIN, by1 = INT_MIN;
                for (int k = 0; k < 4; k++) {
                    Window &wn = s_win[k];
                    wn.oxmin = s_oxmin[k];
                    wn.oymin = s_oymin[k];
                    wn.wx0 = tx0 + s_oxmin[k];
                    wn.wy0 = ty0 + s_oymin[k];
                    wn.WX = tw + 1 + s_oxmax[k] - s_oxmin[k];
                    // full tile height even for a partial tile: the rows past
                    // the image repeat its last row, and the blend loop then
                    // reads every row it steps through without a bounds test
                    wn.WY = kTH + 1 + s_oymax[k] - s_oymin[k];
                    wn.FW = wn.WX + 1;
                    wn.cx0 = min(max(wn.wx0, 0), (int)a.W - 1);
                    wn.cx1 = min(max(wn.wx0 + wn.WX - 1, 0), (int)a.W - 1);
                    wn.cy0 = min(max(wn.wy0, 0), (int)a.H - 1);
                    wn.cy1 = min(max(wn.wy0 + wn.WY - 1, 0), (int)a.H - 1);
                    wn.f_off = off;
                    off += 2u * (uint32_t)(wn.FW * wn.WY);
                    if (s_used[k]) {
                        bx0 = min(bx0, wn.cx0 / kBlock);
                        by0 = min(by0, wn.cy0 / kBlock);
                        bx1 = max(bx1, wn.cx1 / kBlock);
                        by1 = max(by1, wn.cy1 / kBlock);
                    }
                }
                s_rect[0] = bx0;
                s_rect[1] = by0;
                s_rect[2] = bx1 - bx0 + 1;
                s_rect[3] = by1 - by0 + 1;
                s_ent_off = (off + 3) & ~3u;
                // BFS positions the used neighbours need, ascending (only
                // when decoding here)
                int nn = 0;
                for (int k = 0; k < 4 && !kDecoded; k++) {
                    const uint32_t *anc = a.sv.view_anc + nview[k] * kMaxLevels;
                    s_top[k] = anc[a.sv.L - 1];
                    if (!s_used[k])
                        continue;
                    for (uint32_t l = 0; l + 1 < a.sv.L; l++) {
                        const uint32_t p = anc[l];
                        int e = 0;
                        while (e < nn && s_need_pos[e] != p)
                            e++;
                        if (e == nn)
                            s_need_pos[nn++] = p;
                    }
                }
                for (int x = 1; x < nn; x++)   // insertion sort by position
                    for (int y = x; y > 0 && s_need_pos[y - 1] > s_need_pos[y]; y--) {
                        const uint32_t tp = s_need_pos[y];
                        s_need_pos[y] = s_need_pos[y - 1];
                        s_need_pos[y - 1] = tp;
                    }
                for (int k = 0; k < 4 && !kDecoded; k++) {
                    const uint32_t *anc = a.sv.view_anc + nview[k] * kMaxLevels;
                    for (uint32_t l = 0; l + 1 < a.sv.L; l++) {
                        int e = -1;
                        if (s_used[k])
                            for (e = 0; s_need_pos[e] != anc[l]; e++) {
                            }
                        s_slot_need[k][l] = e;
                    }
                }
                s_nneed = nn;
            }
            __syncthreads();
            const int ge = s_gend;
            if (tid < ge - g0) {
                ViewP &vp = s_vp[tid];
                for (int k = 0; k < 4; k++)
                    vp.base[k] = (vp.oy[k] - s_win[k].oymin) * s_win[k].FW + (vp.ox[k] - s_win[k].oxmin);
            }
            const int nbx = s_rect[2], nloc_r = nbx * s_rect[3];
            const int nn = s_nneed;
            // node table entry (2 words) of needed node e at union location li, channel c:
            // [0] payload offset (bits 0..21) | mode << 22 | shift << 27 | present << 31
            // [1] the block minimum (sign-extended)
            uint32_t *ent = g_dyn + s_ent_off;

            if constexpr (kDecoded) {
                // ---- phase 2 (decoded views): copy the windows, clamped to the image
                const int lane = tid & 31, warp = tid >> 5;
                int rows = 0;
                for (int k = 0; k < 4; k++)
                    rows += s_used[k] ? s_win[k].WY : 0;
                // two rows per step (rows rr and rr + 8): both rows' loads are
                // issued before either row is converted
                auto locate = [&](int rr, int &k, int &r) {
                    k = 0;
                    r = rr;
                    while (!s_used[k] || r >= s_win[k].WY) {
                        r -= s_used[k] ? s_win[k].WY : 0;
                        k++;
                    }
                };
                for (int rr = warp; rr < rows; rr += 2 * (kThreads / 32)) {
                    const int rb = rr + kThreads / 32;
                    const bool has_b = rb < rows;
                    int ka, ra, kb = 0, r_b = 0;
                    locate(rr, ka, ra);
                    if (has_b)
                        locate(rb, kb, r_b);
                    const Window &wa = s_win[ka];
                    const Window &wb = s_win[kb];
                    const uint32_t *sa = a.decoded + ((size_t)a.slot_of[nview[ka]] * a.H + min(max(wa.wy0 + ra, 0), (int)a.H - 1)) * a.W;
                    const uint32_t *sb = a.decoded + ((size_t)a.slot_of[nview[kb]] * a.H + min(max(wb.wy0 + r_b, 0), (int)a.H - 1)) * a.W;
                    uint32_t va0, va1, va2, vb0 = 0u, vb1 = 0u, vb2 = 0u;
                    va0 = lane < wa.WX ? __ldg(sa + min(max(wa.wx0 + lane, 0), (int)a.W - 1)) : 0u;
                    va1 = lane + 32 < wa.WX ? __ldg(sa + min(max(wa.wx0 + lane + 32, 0), (int)a.W - 1)) : 0u;
                    va2 = lane + 64 < wa.WX ? __ldg(sa + min(max(wa.wx0 + lane + 64, 0), (int)a.W - 1)) : 0u;
                    if (has_b) {
                        vb0 = lane < wb.WX ? __ldg(sb + min(max(wb.wx0 + lane, 0), (int)a.W - 1)) : 0u;
                        vb1 = lane + 32 < wb.WX ? __ldg(sb + min(max(wb.wx0 + lane + 32, 0), (int)a.W - 1)) : 0u;
                        vb2 = lane + 64 < wb.WX ? __ldg(sb + min(max(wb.wx0 + lane + 64, 0), (int)a.W - 1)) : 0u;
                    }
                    uint2 *da = reinterpret_cast<uint2 *>(g_dyn + wa.f_off) + ra * wa.FW;
                    if (lane < wa.WX)
                        da[lane] = rgb_window(va0);
                    if (lane + 32 < wa.WX)
                        da[lane + 32] = rgb_window(va1);
                    if (lane + 64 < wa.WX)
                        da[lane + 64] = rgb_window(va2);
                    for (int cc = 96 + lane; cc < wa.WX; cc += 32)   // spreads wider than 96 pixels
                        da[cc] = rgb_window(__ldg(sa + min(max(wa.wx0 + cc, 0), (int)a.W - 1)));
                    if (has_b) {
                        uint2 *db = reinterpret_cast<uint2 *>(g_dyn + wb.f_off) + r_b * wb.FW;
                        if (lane < wb.WX)
                            db[lane] = rgb_window(vb0);
                        if (lane + 32 < wb.WX)
                            db[lane + 32] = rgb_window(vb1);
                        if (lane + 64 < wb.WX)
                            db[lane + 64] = rgb_window(vb2);
                        for (int cc = 96 + lane; cc < wb.WX; cc += 32)
                            db[cc] = rgb_window(__ldg(sb + min(max(wb.wx0 + cc, 0), (int)a.W - 1)));
                    }
                }
                __syncthreads();
            } else {
            // ---- phase 2a: one walk per (location, channel)
            for (int task = tid; task < nloc_r * 3; task += kThreads) {
                const int c = task % 3, li = task / 3;
                const int bx = s_rect[0] + li % nbx, by = s_rect[1] + li / nbx;
                const uint32_t loc = (uint32_t)by * a.sv.nlx + (uint32_t)bx;
                const uint32_t *rec = a.sv.records + a.sv.offsets[3 * loc + c];
                uint32_t *my = ent + (size_t)(li * 3 + c) * 2 * nn;
                uint32_t P = 0;
                for (uint32_t m = 0; m < a.sv.MW; m++)
                    P += __popc(rec[m]);
                const uint32_t hdr0 = 32 * a.sv.MW;
                uint32_t rank = 0, off = hdr0 + kHdrBits * P, cur = 0;
                for (int e = 0; e < nn; e++) {
                    const uint32_t p = s_need_pos[e];
                    uint32_t rp = rank;
                    for (uint32_t m = cur >> 5; m <= (p >> 5); m++) {
                        uint32_t word = rec[m];
                        if (m == (cur >> 5))
                            word &= ~((1u << (cur & 31u)) - 1u);
                        if (m == (p >> 5))
                            word &= (1u << (p & 31u)) - 1u;
                        rp += __popc(word);
                    }
                    for (uint32_t h = rank; h < rp; h++) {
                        const uint32_t mh = get_bits(rec, hdr0 + kHdrBits * h, 5);
#ifdef RLFC_DEBUG
                        off += mh < (uint32_t)kNumModes ? mode_bits(s_mode[mh]) : 0u;
#else
                        off += mode_bits(s_mode[mh]);
#endif
                    }
                    rank = rp;
                    cur = p + 1;
                    if ((rec[p >> 5] >> (p & 31u)) & 1u) {
                        const BlockHeader hd = unpack_header(get_bits(rec, hdr0 + kHdrBits * rank, kHdrBits));
#ifdef RLFC_DEBUG
                        const uint32_t rec_bits = 32u * (a.sv.offsets[3 * loc + c + 1] - a.sv.offsets[3 * loc + c]);
                        const uint32_t pay = hd.mode < (uint32_t)kNumModes ? mode_bits(s_mode[hd.mode]) : 0u;
                        const bool ok = RLFC_DBG_BLOCK_OK(a.sv.dbg, hd.mode, hdr0 + kHdrBits * (rank + 1),
                                                          hdr0 + kHdrBits * P, off, pay, rec_bits);
#else
                        constexpr bool ok = true;
                        const uint32_t pay = mode_bits(s_mode[hd.mode]);
#endif
                        // a block that fails the checks of a debug build is left out
                        my[2 * e] = ok ? (off | (hd.mode << 22) | (hd.shift << 27) | 0x80000000u) : 0u;
                        my[2 * e + 1] = (uint32_t)hd.min;
                        off += pay;
                        rank++;
                    } else {
                        my[2 * e] = 0u;
                    }
                }
            }
            __syncthreads();

            // ---- phase 2b: per (location, neighbour): top RKV + ancestors'
            // residuals for the three channels, RGB, into the window (pixels on
            // the image edge also fill the window cells beyond it)
            for (int task = tid; task < nloc_r * 4; task += kThreads) {
                const int k = task & 3, li = task >> 2;
                if (!s_used[k])
                    continue;
                const Window &wn = s_win[k];
                const int bx = s_rect[0] + li % nbx, by = s_rect[1] + li / nbx;
                if (bx * kBlock + kBlock - 1 < wn.cx0 || bx * kBlock > wn.cx1 ||
                    by * kBlock + kBlock - 1 < wn.cy0 || by * kBlock > wn.cy1)
                    continue;
                const uint32_t loc = (uint32_t)by * a.sv.nlx + (uint32_t)bx;
                uint32_t pk[3][kVals / 2];   // finished channels as int16 pairs
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    int32_t acc[kVals];
                    const uint4 *tp = reinterpret_cast<const uint4 *>(
                        a.sv.top + ((size_t)s_top[k] * a.sv.nloc + loc) * 48 + c * 16);
                    const uint4 t0 = tp[0], t1 = tp[1];
                    const uint32_t t32[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
                    for (int v = 0; v < kVals; v++)
                        acc[v] = (int32_t)(int16_t)(t32[v >> 1] >> (16 * (v & 1)));
                    const uint32_t *rec = a.sv.records + a.sv.offsets[3 * loc + c];
                    const uint32_t *my = ent + (size_t)(li * 3 + c) * 2 * nn;
                    for (uint32_t l = 0; l + 1 < a.sv.L; l++) {
                        const int e = s_slot_need[k][l];
                        const uint32_t w0 = my[2 * e];
                        if (!(w0 >> 31))
                            continue;
                        decode_block_values(rec, w0 & 0x3FFFFFu, s_mode[(w0 >> 22) & 31u], (int32_t)my[2 * e + 1],
                                            1 << (a.sv.q + ((w0 >> 27) & 3u)), acc);
                    }
#pragma unroll
                    for (int v = 0; v < kVals; v += 2)
                        pk[c][v >> 1] = ((uint32_t)acc[v] & 0xFFFFu) | ((uint32_t)acc[v + 1] << 16);
                }
                uint2 *f = reinterpret_cast<uint2 *>(g_dyn + wn.f_off);
#pragma unroll
                for (int v = 0; v < kVals; v++) {
                    const int px = bx * kBlock + (v & 3), py = by * kBlock + (v >> 2);
                    if (px < wn.cx0 || px > wn.cx1 || py < wn.cy0 || py > wn.cy1)
                        continue;
                    const int sh16 = 16 * (v & 1);
                    const uint2 rgb = rgb_window(ycocg_to_rgb24((int16_t)(pk[0][v >> 1] >> sh16),
                                                              (int16_t)(pk[1][v >> 1] >> sh16),
                                                              (int16_t)(pk[2][v >> 1] >> sh16)));
                    // window columns whose clamped x is px (more than one on the image edge)
                    const int xa = (px == 0 ? wn.wx0 : px) - wn.wx0, xb = (px == (int)a.W - 1 ? wn.wx0 + wn.WX - 1 : px) - wn.wx0;
                    const int ya = (py == 0 ? wn.wy0 : py) - wn.wy0, yb = (py == (int)a.H - 1 ? wn.wy0 + wn.WY - 1 : py) - wn.wy0;
                    for (int yy = max(ya, 0); yy <= min(yb, wn.WY - 1); yy++)
                        for (int xx = max(xa, 0); xx <= min(xb, wn.WX - 1); xx++)
                            f[yy * wn.FW + xx] = rgb;
                }
            }
            __syncthreads();

            }
            // ---- phase 4: blend and store, view by view; thread = one column
            // of kRows rows, sliding the 2 x 2 stencil down the window
            const int col = tid % kTW, r0 = (tid / kTW) * kRows;
            const bool active = col < tw && r0 < th;
            int win_fw[4];
            const uint2 *win_at[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                win_fw[k] = s_win[k].FW;
                win_at[k] = reinterpret_cast<const uint2 *>(g_dyn + s_win[k].f_off) + r0 * win_fw[k] + col;
            }
            for (int q = g0; q < ge; q++) {
                if (!active)
                    continue;
                const ViewP &vp = s_vp[q - g0];
                // R and G accumulate as a pair (one paired FMA per tap), B on
                // its own; the taps are added in the order 00, 10, 01, 11
                float2 acc_rg[kRows];
                float acc_b[kRows];
#pragma unroll
                for (int rr = 0; rr < kRows; rr++) {
                    acc_rg[rr] = make_float2(0.0f, 0.0f);
                    acc_b[rr] = 0.0f;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (!((vp.used >> k) & 1u))
                        continue;
                    const float4 wk = *reinterpret_cast<const float4 *>(vp.w[k]);
                    const float2 w00 = make_float2(wk.x, wk.x), w10 = make_float2(wk.y, wk.y);
                    const float2 w01 = make_float2(wk.z, wk.z), w11 = make_float2(wk.w, wk.w);
                    const int fw = win_fw[k];
                    const uint2 *f = win_at[k] + vp.base[k];
                    float2 a0, a1;
                    float a0b, a1b;
                    {
                        const uint2 p0 = f[0], p1 = f[1];
                        a0 = make_float2(win_r(p0), win_g(p0));
                        a1 = make_float2(win_r(p1), win_g(p1));
                        a0b = win_b(p0);
                        a1b = win_b(p1);
                    }
#pragma unroll
                    for (int rr = 0; rr < kRows; rr++) {
                        f += fw;
                        const uint2 p0 = f[0], p1 = f[1];
                        const float2 b0 = make_float2(win_r(p0), win_g(p0)), b1 = make_float2(win_r(p1), win_g(p1));
                        const float b0b = win_b(p0), b1b = win_b(p1);
                        acc_rg[rr] = __ffma2_rn(w11, b1, __ffma2_rn(w01, b0, __ffma2_rn(w10, a1, __ffma2_rn(w00, a0, acc_rg[rr]))));
                        acc_b[rr] = fmaf(w11.x, b1b, fmaf(w01.x, b0b, fmaf(w10.x, a1b, fmaf(w00.x, a0b, acc_b[rr]))));
                        a0 = b0;
                        a1 = b1;
                        a0b = b0b;
                        a1b = b1b;
                    }
                }
                float acc[kRows][3];
#pragma unroll
                for (int rr = 0; rr < kRows; rr++) {
                    acc[rr][0] = acc_rg[rr].x;
                    acc[rr][1] = acc_rg[rr].y;
                    acc[rr][2] = acc_b[rr];
                }
                const uint32_t r = s_list[q];
#pragma unroll
                for (int rr = 0; rr < kRows; rr++) {
                    if (r0 + rr >= th)
                        break;
                    const size_t px = ((size_t)r * a.H + (ty0 + r0 + rr)) * a.W + (tx0 + col);
                    if (a.out8) {
                        uint8_t *o = a.out8 + px * 3;
                        o[0] = to_u8(acc[rr][0]);
                        o[1] = to_u8(acc[rr][1]);
                        o[2] = to_u8(acc[rr][2]);
                    } else {
                        float *o = a.out + px * 3;
                        // evict-first: the outputs stream through L2 without pushing out the stream
                        __stcs(o, acc[rr][0]);
                        __stcs(o + 1, acc[rr][1]);
                        __stcs(o + 2, acc[rr][2]);
                    }
                }
            }
            g0 = ge;
            __syncthreads();
        }
    }
    __syncthreads();   // the next item reuses the shared memory
    }
}

// Lists the grid cells that hold at least one camera (each once; the
// order does not matter).  One CTA: a bitmask of the cells in shared memory
// (at most 65535 cells, 2048 words), then the set bits appended to the list.
constexpr int kListThreads = 1024;
constexpr uint32_t kMaxCellWords = 2048;

__global__ void __launch_bounds__(kListThreads) list_cells_kernel(const Args a, uint32_t n_cells, uint32_t *list,
                                                                  uint32_t *count)
{
    __shared__ uint32_t mask[kMaxCellWords];
    __shared__ uint32_t total;
    const uint32_t words = (n_cells + 31) / 32;
    for (uint32_t w = threadIdx.x; w < words; w += kListThreads)
        mask[w] = 0u;
    if (threadIdx.x == 0)
        total = 0u;
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < a.n; r += kListThreads) {
        const uint32_t cell = cell_of(a, r);
        atomicOr(&mask[cell >> 5], 1u << (cell & 31));
    }
    __syncthreads();
    for (uint32_t w = threadIdx.x; w < words; w += kListThreads) {
        uint32_t bits = mask[w];
        uint32_t at = atomicAdd(&total, (uint32_t)__popc(bits));
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            list[at++] = w * 32 + (uint32_t)b;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        *count = total;
}

// Numbers the marked views 0, 1, ... in view order (one CTA; at most 16383
// views, 16 per thread): slot_of[v] for a marked view v.
__global__ void __launch_bounds__(kListThreads) assign_slots_kernel(const uint8_t *needed, uint32_t n_views,
                                                                    uint32_t *slot_of)
{
    __shared__ uint32_t s_warp[kListThreads / 32];
    const uint32_t per = (n_views + kListThreads - 1) / kListThreads;
    const uint32_t v0 = threadIdx.x * per, v1 = min(n_views, v0 + per);
    uint32_t cnt = 0;
    for (uint32_t v = v0; v < v1; v++)
        cnt += needed[v] != 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = cnt;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d)
            incl += y;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, d);
            if (lane >= d)
                w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t at = incl - cnt + (warp ? s_warp[warp - 1] : 0u);
    for (uint32_t v = v0; v < v1; v++)
        if (needed[v])
            slot_of[v] = at++;
}

// Marks the neighbour views that each camera blends with a non-zero weight.
__global__ void mark_needed_kernel(const Args a, uint8_t *needed)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n)
        return;
    int ci, cj;
    float w[4];
    Shift sh[4];
    view_params(a, r, ci, cj, w, sh);
    for (int k = 0; k < 4; k++) {
        const int i = a.U == 1 ? 0 : ci + (k & 1), j = a.V == 1 ? 0 : cj + (k >> 1);
        if (w[k] != 0.0f)
            needed[j * (int)a.U + i] = 1;
    }
}

}  // namespace

// Native-size rendering of n views; returns RLFC_E_UNSUPPORTED when the
// geometry is not native (the general kernels handle it).
int launch_render_native(const rlfc_stream *s, const float *d_uv, const float *d_disp, uint32_t n, float *d_out,
                         cudaStream_t st, uint8_t *d_out8)
{
    Args a;
    a.sv.records = s->d_records;
    a.sv.offsets = s->d_offsets;
    a.sv.top = s->d_top;
    a.sv.view_anc = s->d_view_anc;
    a.sv.n_views = s->tab.n_views;
    a.sv.nloc = s->info.nloc_x * s->info.nloc_y;
    a.sv.nlx = s->info.nloc_x;
    a.sv.L = s->tab.L;
    a.sv.q = s->info.q;
    a.sv.MW = s->MW;
    a.sv.dbg = s->d_debug;
    a.uv = d_uv;
    a.disp = d_disp;
    a.out = d_out;
    a.out8 = d_out8;
    a.U = s->info.U;
    a.V = s->info.V;
    a.W = s->info.W;
    a.H = s->info.H;
    a.n = n;
    a.tiles_x = (a.W + kTW - 1) / kTW;
    const uint32_t tiles_y = (a.H + kTH - 1) / kTH;
    a.cells_u = a.U > 1 ? a.U - 1 : 1;
    const uint32_t cells_v = a.V > 1 ? a.V - 1 : 1;
    const uint32_t n_cells = a.cells_u * cells_v;
    if ((uint64_t)a.tiles_x * tiles_y >= (1u << 31) || n_cells > 65535)
        return RLFC_E_UNSUPPORTED;
    a.n_tiles = a.tiles_x * tiles_y;
    // a single view (no shift spread) needs four windows of the full tile,
    // and, decoding on demand, the node table of its footprint
    a.need_max = 4 * (a.sv.L - 1);
    const uint32_t win1 = 4 * 4 * window_words(kTW, kTH, 0, 0);
    const uint32_t single = win1 + 4 * ((kTW + 7) / kBlock + 1) * ((kTH + 7) / kBlock + 1) * 3 * 2 * a.need_max;
    cudaError_t e;

    // Batches of many views decode the views they need once into a transient
    // packed-RGB buffer (stream-ordered allocation, freed on the same stream),
    // one slot per needed view: a camera needs at most four views, so
    // min(views, 4n) slots suffice.  Small batches decode block by block
    // inside the render kernel.
    a.decoded = nullptr;
    a.slot_of = nullptr;
    void *scratch = nullptr;
    const size_t view_words = (size_t)a.W * a.H;
    const size_t mask_bytes = (a.sv.n_views + 255) / 256 * 256;
    const size_t slot_bytes = (4ull * a.sv.n_views + 255) / 256 * 256;
    const size_t n_slots = std::min<size_t>(a.sv.n_views, 4ull * n);
    bool first = n >= kDecodeFirstViews && win1 <= kSmemDecoded;
    if (first && cudaMallocAsync(&scratch, mask_bytes + slot_bytes + 4 * view_words * n_slots, st) != cudaSuccess) {
        cudaGetLastError();   // a failed stream-ordered allocation only selects the other path
        first = false;
    }
    if (!first && single > kSmemBytes)
        return RLFC_E_UNSUPPORTED;
    auto kern = first ? render_native_kernel<true> : render_native_kernel<false>;
    const uint32_t smem = first ? kSmemDecoded : kSmemBytes;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem)) != cudaSuccess) {
        if (scratch)
            cudaFreeAsync(scratch, st);
        return cuda_fail(e, "render_native: launch configuration");
    }
    dim3 grid(a.n_tiles, n_cells);
    uint32_t *cells = nullptr;
    a.cell_list = nullptr;
    a.cell_count = nullptr;
    int rc = RLFC_OK;
    const uint32_t resident = (uint32_t)std::max(sms, 1) * (uint32_t)std::max(per_sm, 1);
    if (n < 2 * n_cells && (uint64_t)a.n_tiles * n_cells >= 8ull * resident) {
        // few cameras for a large grid: most of its CTAs would find an empty
        // cell, so list the occupied cells and run persistent CTAs over their
        // tiles only (list and count in stream-ordered scratch)
        grid = dim3(resident);
        if ((e = cudaMallocAsync(&cells, 4ull * (n_cells + 1), st)) != cudaSuccess) {
            rc = cuda_fail(e, "render_native: cell list");
        } else {
            a.cell_list = cells;
            a.cell_count = cells + n_cells;
            { rlfc::TraceScope trace_("list_cells_kernel", st); list_cells_kernel<<<1, kListThreads, 0, st>>>(a, n_cells, cells, cells + n_cells); }
        }
    }
    if (rc == RLFC_OK && first) {
        uint8_t *needed = static_cast<uint8_t *>(scratch);
        uint32_t *slot_of = reinterpret_cast<uint32_t *>(needed + mask_bytes);
        uint32_t *decoded = reinterpret_cast<uint32_t *>(needed + mask_bytes + slot_bytes);
        if ((e = cudaMemsetAsync(needed, 0, mask_bytes, st)) != cudaSuccess)
            rc = cuda_fail(e, "render: clearing the view mask");
        if (rc == RLFC_OK) {
            { rlfc::TraceScope trace_("mark_needed_kernel", st); mark_needed_kernel<<<(n + 255) / 256, 256, 0, st>>>(a, needed); }
            { rlfc::TraceScope trace_("assign_slots_kernel", st); assign_slots_kernel<<<1, kListThreads, 0, st>>>(needed, a.sv.n_views, slot_of); }
            rc = launch_decode_packed(s, decoded, needed, slot_of, (uint32_t)n_slots, st);
        }
        a.decoded = decoded;
        a.slot_of = slot_of;
    }
    if (rc == RLFC_OK) {
        { rlfc::TraceScope trace_("render_native_kernel", st); kern<<<grid, kThreads, smem, st>>>(a); }
        if ((e = cudaGetLastError()) != cudaSuccess)
            rc = cuda_fail(e, "render_native launch");
    }
    if (scratch)
        cudaFreeAsync(scratch, st);
    if (cells)
        cudaFreeAsync(cells, st);
    return rc;
}

}  // namespace rlfc

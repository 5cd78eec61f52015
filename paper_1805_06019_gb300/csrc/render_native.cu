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
//     once, in BFS order, decoding only the four neighbours' leaf blocks and
//     their ancestors, and accumulates top RKV + residuals (YCoCg-R, int16)
//     into the source rectangles;
//  3. the windows are filled with packed RGB from the source rectangles,
//     which replicates the image edge exactly as clamp-to-edge sampling does;
//  4. per view, each thread blends 4 horizontally adjacent pixels from 2 x 5
//     window samples per neighbour and writes them with three 16-byte
//     streaming stores.
#include <cuda_runtime.h>

#include <algorithm>

#include "warp_decode.cuh"

namespace rlfc {
namespace {

constexpr int kTW = 64, kTH = 16;       // output tile
constexpr int kThreads = 256;           // 4 pixels per thread
constexpr int kListCap = 1024;          // views collected per pass
constexpr int kMaxNeed = 4 * kMaxLevels;
constexpr uint32_t kSmemBytes = 64 * 1024;

__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

struct Args {
    StreamView sv;
    const float *uv;
    const float *disp;
    float *out;
    uint32_t U, V, W, H, n;
    uint32_t tiles_x, cells_u;
    uint32_t out_aligned16;
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
    int wx0, wy0, WX, WY;     // padded window (global pixel origin, size)
    int FW;                   // row stride of the window: WX + 3, so that a
                              // 5-sample read of a ragged last group stays in the row
    int sx0, sy0, SW, SH;     // source rectangle: the window clamped to the image
    int oxmin, oymin;
    uint32_t f_off, s_off;    // offsets (in 32-bit words) into shared memory
};

extern __shared__ __align__(16) uint32_t g_dyn[];

__global__ void __launch_bounds__(kThreads) render_native_kernel(const Args a)
{
    __shared__ uint32_t s_mode[kNumModes];
    __shared__ uint32_t s_list[kListCap];
    __shared__ int s_count, s_gstart, s_gend;
    __shared__ int s_oxmin[4], s_oxmax[4], s_oymin[4], s_oymax[4], s_used[4];
    __shared__ Window s_win[4];
    __shared__ uint32_t s_need_pos[kMaxNeed], s_need_slots[kMaxNeed];
    __shared__ int s_nneed;
    __shared__ uint32_t s_top[4];
    __shared__ int s_rect[4];   // union block rectangle bx0, by0, nbx, nby

    const int tid = threadIdx.x;
    const uint32_t cell = blockIdx.y;
    const int ci = (int)(cell % a.cells_u), cj = (int)(cell / a.cells_u);
    const int tx0 = (int)(blockIdx.x % a.tiles_x) * kTW, ty0 = (int)(blockIdx.x / a.tiles_x) * kTH;
    const int tw = min(kTW, (int)a.W - tx0), th = min(kTH, (int)a.H - ty0);
    if (tid < kNumModes)
        s_mode[tid] = c_modes[tid];
    // the four neighbour views of this cell
    int nview[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int i = a.U == 1 ? 0 : ci + (k & 1), j = a.V == 1 ? 0 : cj + (k >> 1);
        nview[k] = j * (int)a.U + i;
    }

    for (uint32_t base = 0; base < a.n; base += kListCap) {
        // ---- phase 1: the views of this cell among [base, base + kListCap)
        if (tid == 0)
            s_count = 0;
        __syncthreads();
        const uint32_t lim = min(a.n, base + kListCap);
        for (uint32_t r = base + tid; r < lim; r += kThreads)
            if (cell_of(a, r) == cell)
                s_list[atomicAdd(&s_count, 1)] = r;
        __syncthreads();
        const int count = s_count;
        if (count == 0)
            continue;
        // groups of views whose windows fit shared memory
        for (int g0 = 0; g0 < count;) {
            if (tid == 0) {
                // grow the group while the four windows fit
                int oxl[4], oxh[4], oyl[4], oyh[4];
                for (int k = 0; k < 4; k++) {
                    oxl[k] = oyl[k] = INT_MAX;
                    oxh[k] = oyh[k] = INT_MIN;
                }
                int g1 = g0;
                while (g1 < count) {
                    int c1, c2;
                    float w[4];
                    Shift sh[4];
                    view_params(a, s_list[g1], c1, c2, w, sh);
                    uint32_t words = 0;
                    int nl[4], nh[4], ml[4], mh[4];
                    for (int k = 0; k < 4; k++) {
                        nl[k] = min(oxl[k], sh[k].ox);
                        nh[k] = max(oxh[k], sh[k].ox);
                        ml[k] = min(oyl[k], sh[k].oy);
                        mh[k] = max(oyh[k], sh[k].oy);
                        const uint32_t wx = (uint32_t)(tw + 1 + nh[k] - nl[k]), wy = (uint32_t)(th + 1 + mh[k] - ml[k]);
                        words += (wx + 3) * wy + (3 * wx * wy + 1) / 2 + 8;
                    }
                    if (words * 4 > kSmemBytes && g1 > g0)
                        break;
                    for (int k = 0; k < 4; k++) {
                        oxl[k] = nl[k];
                        oxh[k] = nh[k];
                        oyl[k] = ml[k];
                        oyh[k] = mh[k];
                    }
                    g1++;
                }
                s_gstart = g0;
                s_gend = g1;
                for (int k = 0; k < 4; k++) {
                    s_oxmin[k] = oxl[k];
                    s_oxmax[k] = oxh[k];
                    s_oymin[k] = oyl[k];
                    s_oymax[k] = oyh[k];
                    s_used[k] = 0;
                }
            }
            __syncthreads();
            const int gs = s_gstart, ge = s_gend;
            // neighbours with a non-zero weight for some view of the group
            for (int q = gs + tid; q < ge; q += kThreads) {
                int c1, c2;
                float w[4];
                Shift sh[4];
                view_params(a, s_list[q], c1, c2, w, sh);
                for (int k = 0; k < 4; k++)
                    if (w[k] != 0.0f)
                        s_used[k] = 1;
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t off = 0;
                int bx0 = INT_MAX, by0 = INT_MAX, bx1 = INT_MIN, by1 = INT_MIN;
                for (int k = 0; k < 4; k++) {
                    Window &wn = s_win[k];
                    wn.oxmin = s_oxmin[k];
                    wn.oymin = s_oymin[k];
                    wn.wx0 = tx0 + s_oxmin[k];
                    wn.wy0 = ty0 + s_oymin[k];
                    wn.WX = tw + 1 + s_oxmax[k] - s_oxmin[k];
                    wn.WY = th + 1 + s_oymax[k] - s_oymin[k];
                    wn.FW = wn.WX + 3;
                    wn.sx0 = min(max(wn.wx0, 0), (int)a.W - 1);
                    wn.sy0 = min(max(wn.wy0, 0), (int)a.H - 1);
                    const int sx1 = min(max(wn.wx0 + wn.WX - 1, 0), (int)a.W - 1);
                    const int sy1 = min(max(wn.wy0 + wn.WY - 1, 0), (int)a.H - 1);
                    wn.SW = sx1 - wn.sx0 + 1;
                    wn.SH = sy1 - wn.sy0 + 1;
                    wn.f_off = off;
                    off += (uint32_t)(wn.FW * wn.WY);
                    wn.s_off = off;
                    off += (uint32_t)(3 * wn.SW * wn.SH + 1) / 2;
                    off = (off + 3) & ~3u;
                    if (s_used[k]) {
                        bx0 = min(bx0, wn.sx0 / kBlock);
                        by0 = min(by0, wn.sy0 / kBlock);
                        bx1 = max(bx1, sx1 / kBlock);
                        by1 = max(by1, sy1 / kBlock);
                    }
                }
                s_rect[0] = bx0;
                s_rect[1] = by0;
                s_rect[2] = bx1 - bx0 + 1;
                s_rect[3] = by1 - by0 + 1;
                // BFS positions the four neighbours need, ascending, with the
                // neighbours each one serves
                int nn = 0;
                for (int k = 0; k < 4; k++) {
                    if (!s_used[k])
                        continue;
                    const uint32_t *anc = a.sv.view_anc + nview[k] * kMaxLevels;
                    s_top[k] = anc[a.sv.L - 1];
                    for (uint32_t l = 0; l + 1 < a.sv.L; l++) {
                        const uint32_t p = anc[l];
                        int e = 0;
                        while (e < nn && s_need_pos[e] != p)
                            e++;
                        if (e == nn) {
                            s_need_pos[nn] = p;
                            s_need_slots[nn] = 0;
                            nn++;
                        }
                        s_need_slots[e] |= 1u << k;
                    }
                }
                for (int x = 1; x < nn; x++)   // insertion sort by position
                    for (int y = x; y > 0 && s_need_pos[y - 1] > s_need_pos[y]; y--) {
                        const uint32_t tp = s_need_pos[y], ts = s_need_slots[y];
                        s_need_pos[y] = s_need_pos[y - 1];
                        s_need_slots[y] = s_need_slots[y - 1];
                        s_need_pos[y - 1] = tp;
                        s_need_slots[y - 1] = ts;
                    }
                s_nneed = nn;
            }
            __syncthreads();

            // ---- phase 2: one record walk per (block location, channel)
            const int nbx = s_rect[2], ntask = nbx * s_rect[3] * 3;
            for (int task = tid; task < ntask; task += kThreads) {
                const int c = task % 3, li = task / 3;
                const int bx = s_rect[0] + li % nbx, by = s_rect[1] + li / nbx;
                const uint32_t loc = (uint32_t)by * a.sv.nlx + (uint32_t)bx;
                // which neighbours' source rectangles this block overlaps
                uint32_t touch = 0;
                for (int k = 0; k < 4; k++) {
                    const Window &wn = s_win[k];
                    if (s_used[k] && bx * kBlock + kBlock - 1 >= wn.sx0 && bx * kBlock <= wn.sx0 + wn.SW - 1 &&
                        by * kBlock + kBlock - 1 >= wn.sy0 && by * kBlock <= wn.sy0 + wn.SH - 1)
                        touch |= 1u << k;
                }
                if (!touch)
                    continue;
                // top RKV values first
                for (int k = 0; k < 4; k++) {
                    if (!((touch >> k) & 1u))
                        continue;
                    const Window &wn = s_win[k];
                    int16_t *src = reinterpret_cast<int16_t *>(g_dyn + wn.s_off) + c * wn.SW * wn.SH;
                    const int16_t *tp = a.sv.top + ((size_t)s_top[k] * a.sv.nloc + loc) * 48 + c * 16;
#pragma unroll
                    for (int v = 0; v < kVals; v++) {
                        const int px = bx * kBlock + (v & 3) - wn.sx0, py = by * kBlock + (v >> 2) - wn.sy0;
                        if (px >= 0 && px < wn.SW && py >= 0 && py < wn.SH)
                            src[py * wn.SW + px] = tp[v];
                    }
                }
                const uint32_t *rec = a.sv.records + a.sv.offsets[3 * loc + c];
                uint32_t P = 0;
                for (uint32_t m = 0; m < a.sv.MW; m++)
                    P += __popc(rec[m]);
                const uint32_t hdr0 = 32 * a.sv.MW;
                uint32_t rank = 0, off = hdr0 + kHdrBits * P, cur = 0;
                const int nn = s_nneed;
                for (int e = 0; e < nn; e++) {
                    const uint32_t p = s_need_pos[e];
                    const uint32_t use = s_need_slots[e] & touch;
                    // stored blocks in [cur, p): skip their payloads
                    uint32_t rp = rank;
                    for (uint32_t m = cur >> 5; m <= (p >> 5); m++) {
                        uint32_t word = rec[m];
                        if (m == (cur >> 5))
                            word &= ~((1u << (cur & 31u)) - 1u);
                        if (m == (p >> 5))
                            word &= (1u << (p & 31u)) - 1u;
                        rp += __popc(word);
                    }
                    for (uint32_t h = rank; h < rp; h++)
                        off += mode_bits(s_mode[get_bits(rec, hdr0 + kHdrBits * h, 5)]);
                    rank = rp;
                    cur = p + 1;
                    if (!((rec[p >> 5] >> (p & 31u)) & 1u))
                        continue;
                    const BlockHeader hd = unpack_header(get_bits(rec, hdr0 + kHdrBits * rank, kHdrBits));
                    const uint32_t m = s_mode[hd.mode];
                    if (use) {
                        int32_t u[kVals];
                        bise_decode16(rec, off, m, u);
                        const int32_t scale = 1 << (a.sv.q + hd.shift);
                        for (int k = 0; k < 4; k++) {
                            if (!((use >> k) & 1u))
                                continue;
                            const Window &wn = s_win[k];
                            int16_t *src = reinterpret_cast<int16_t *>(g_dyn + wn.s_off) + c * wn.SW * wn.SH;
#pragma unroll
                            for (int v = 0; v < kVals; v++) {
                                const int px = bx * kBlock + (v & 3) - wn.sx0, py = by * kBlock + (v >> 2) - wn.sy0;
                                if (px >= 0 && px < wn.SW && py >= 0 && py < wn.SH)
                                    src[py * wn.SW + px] = (int16_t)(src[py * wn.SW + px] + (hd.min + u[v]) * scale);
                            }
                        }
                    }
                    off += mode_bits(m);
                    rank++;
                }
            }
            __syncthreads();

            // ---- phase 3: padded windows of packed RGB (edge replicated)
            for (int k = 0; k < 4; k++) {
                if (!s_used[k])
                    continue;
                const Window &wn = s_win[k];
                const int16_t *src = reinterpret_cast<const int16_t *>(g_dyn + wn.s_off);
                const int plane = wn.SW * wn.SH;
                uint32_t *f = g_dyn + wn.f_off;
                for (int i = tid; i < wn.WX * wn.WY; i += kThreads) {
                    const int r = i / wn.WX, cc = i - r * wn.WX;
                    const int gx = min(max(wn.wx0 + cc, 0), (int)a.W - 1) - wn.sx0;
                    const int gy = min(max(wn.wy0 + r, 0), (int)a.H - 1) - wn.sy0;
                    const int at = gy * wn.SW + gx;
                    f[r * wn.FW + cc] = ycocg_to_rgb24(src[at], src[plane + at], src[2 * plane + at]);
                }
            }
            __syncthreads();

            // ---- phase 4: blend and store, view by view
            const int row = tid / (kTW / 4), col = (tid % (kTW / 4)) * 4;
            for (int q = gs; q < ge; q++) {
                const uint32_t r = s_list[q];
                int c1, c2;
                float w[4];
                Shift sh[4];
                view_params(a, r, c1, c2, w, sh);
                if (row >= th || col >= tw)
                    continue;
                float acc[4][3];
#pragma unroll
                for (int p = 0; p < 4; p++)
                    acc[p][0] = acc[p][1] = acc[p][2] = 0.0f;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (w[k] == 0.0f)
                        continue;
                    const Window &wn = s_win[k];
                    const float wk = w[k] * (1.0f / 255.0f);
                    const float w00 = wk * (1.0f - sh[k].fx) * (1.0f - sh[k].fy), w10 = wk * sh[k].fx * (1.0f - sh[k].fy);
                    const float w01 = wk * (1.0f - sh[k].fx) * sh[k].fy, w11 = wk * sh[k].fx * sh[k].fy;
                    const uint32_t *f0 = g_dyn + wn.f_off + (row + sh[k].oy - wn.oymin) * wn.FW + (col + sh[k].ox - wn.oxmin);
                    const uint32_t *f1 = f0 + wn.FW;
                    uint32_t A[5], Bv[5];
#pragma unroll
                    for (int x = 0; x < 5; x++) {
                        A[x] = f0[x];
                        Bv[x] = f1[x];
                    }
#pragma unroll
                    for (int ch = 0; ch < 3; ch++) {
                        float a5[5], b5[5];
#pragma unroll
                        for (int x = 0; x < 5; x++) {
                            a5[x] = (float)((A[x] >> (8 * ch)) & 255u);
                            b5[x] = (float)((Bv[x] >> (8 * ch)) & 255u);
                        }
#pragma unroll
                        for (int p = 0; p < 4; p++)
                            acc[p][ch] += w00 * a5[p] + w10 * a5[p + 1] + w01 * b5[p] + w11 * b5[p + 1];
                    }
                }
                const int y = ty0 + row, x = tx0 + col;
                float *o = a.out + (((size_t)r * a.H + y) * a.W + x) * 3;
                if (a.out_aligned16 && col + 4 <= tw) {
                    float4 *o4 = reinterpret_cast<float4 *>(o);
                    __stcs(o4 + 0, make_float4(acc[0][0], acc[0][1], acc[0][2], acc[1][0]));
                    __stcs(o4 + 1, make_float4(acc[1][1], acc[1][2], acc[2][0], acc[2][1]));
                    __stcs(o4 + 2, make_float4(acc[2][2], acc[3][0], acc[3][1], acc[3][2]));
                } else {
                    for (int p = 0; p < 4 && col + p < tw; p++) {
                        o[3 * p] = acc[p][0];
                        o[3 * p + 1] = acc[p][1];
                        o[3 * p + 2] = acc[p][2];
                    }
                }
            }
            g0 = ge;
            __syncthreads();
        }
    }
}

}  // namespace

// Native-size rendering of n views; returns RLFC_E_UNSUPPORTED when the
// geometry is not native (the general kernels handle it).
int launch_render_native(const rlfc_stream *s, const float *d_uv, const float *d_disp, uint32_t n, float *d_out,
                         cudaStream_t st)
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
    a.uv = d_uv;
    a.disp = d_disp;
    a.out = d_out;
    a.U = s->info.U;
    a.V = s->info.V;
    a.W = s->info.W;
    a.H = s->info.H;
    a.n = n;
    a.tiles_x = (a.W + kTW - 1) / kTW;
    const uint32_t tiles_y = (a.H + kTH - 1) / kTH;
    a.cells_u = a.U > 1 ? a.U - 1 : 1;
    const uint32_t cells_v = a.V > 1 ? a.V - 1 : 1;
    a.out_aligned16 = ((uintptr_t)d_out & 15u) == 0 && (a.W % 4) == 0;
    // a single view needs windows of (64+1) x (16+1) pixels per neighbour
    const uint32_t single = 4 * ((kTW + 4) * (kTH + 1) + (3 * (kTW + 1) * (kTH + 1) + 1) / 2 + 8) * 4;
    if (single > kSmemBytes || (uint64_t)a.tiles_x * tiles_y >= (1u << 31) || a.cells_u * cells_v > 65535)
        return RLFC_E_UNSUPPORTED;
    cudaError_t e = cudaFuncSetAttribute(render_native_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess)
        return cuda_fail(e, "render_native: shared memory attribute");
    dim3 grid(a.tiles_x * tiles_y, a.cells_u * cells_v);
    render_native_kernel<<<grid, kThreads, kSmemBytes, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "render_native launch");
    return RLFC_OK;
}

}  // namespace rlfc

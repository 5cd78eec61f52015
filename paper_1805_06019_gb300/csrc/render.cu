// New-view rendering (Section 3.6): quadrilinear interpolation of the light
// field, decoding the needed blocks on demand from the compressed stream.
//
// Ray geometry (the dynamically reparameterised focal plane the paper cites):
// the camera sits at continuous (u, v) on the grid, clamped to it; output
// pixel (x, y) follows s = (x + 0.5) W / out_w - 0.5, t = (y + 0.5) H / out_h
// - 0.5; in neighbour view (i, j) it lands at (s + d (i - u), t + d (j - v)),
// sampled bilinearly with clamp-to-edge; the neighbours i0 = min(floor(u),
// U - 2), i1 = i0 + 1 are blended with weights 1 - fu, fu, and the same in v.
//
// Tiled kernel: one CTA renders a 32 x 8 tile of one view.  Since s, t are
// monotone in x, y, the tile's samples in neighbour view k fall inside the
// block rectangle spanned by its corner rays; the warps decode those blocks
// (warp-cooperative random access) into shared memory, then every thread
// blends its 16 samples in fp32 and writes its RGB triple.
// Fallback kernel (footprints too large for shared memory, i.e. heavy
// downscaling): each thread decodes the pixels it samples one by one.
#include <cuda_runtime.h>

#include <algorithm>

#include "warp_decode.cuh"

namespace rlfc {
namespace {

constexpr int kTX = 32, kTY = 8, kThreads = kTX * kTY;
constexpr uint32_t kFootprintBudget = 96 * 1024;

__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

struct Args {
    StreamView sv;
    const float *uv;
    const float *disp;
    float *out;
    uint8_t *out8;      // when set, 8-bit RGB goes here instead of out
    uint32_t U, V, W, H, out_w, out_h;
    uint32_t tiles_x;
    uint32_t max_fp_blocks;  // per neighbour view
};

struct Camera {
    int view[4];
    float w[4];
    float shift_x[4], shift_y[4];
};

__device__ __forceinline__ void axis(float u, uint32_t G, int &i0, int &i1, float &f)
{
    u = fminf(fmaxf(u, 0.0f), (float)(G - 1));
    if (G == 1) {
        i0 = i1 = 0;
        f = 0.0f;
        return;
    }
    i0 = min((int)floorf(u), (int)G - 2);
    i1 = i0 + 1;
    f = u - (float)i0;
}

__device__ __forceinline__ Camera make_camera(const Args &a, uint32_t n)
{
    Camera cam;
    const float u = fminf(fmaxf(a.uv[2 * n], 0.0f), (float)(a.U - 1));
    const float v = fminf(fmaxf(a.uv[2 * n + 1], 0.0f), (float)(a.V - 1));
    const float d = a.disp[n];
    int i0, i1, j0, j1;
    float fu, fv;
    axis(u, a.U, i0, i1, fu);
    axis(v, a.V, j0, j1, fv);
    const int iv[2] = {i0, i1}, jv[2] = {j0, j1};
    const float wu[2] = {1.0f - fu, fu}, wv[2] = {1.0f - fv, fv};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int ia = k & 1, jb = k >> 1;
        cam.view[k] = jv[jb] * (int)a.U + iv[ia];
        cam.w[k] = wu[ia] * wv[jb];
        // a shift beyond twice the image size samples only the clamped edge
        // either way; bounding it keeps the integer pixel arithmetic in range
        const float lim = 2.0f * (float)max(a.W, a.H) + 4.0f;
        cam.shift_x[k] = fminf(fmaxf(d * ((float)iv[ia] - u), -lim), lim);
        cam.shift_y[k] = fminf(fmaxf(d * ((float)jv[jb] - v), -lim), lim);
    }
    return cam;
}

__device__ __forceinline__ float ray_s(uint32_t x, uint32_t W, uint32_t out_w)
{
    return ((float)x + 0.5f) * (float)W / (float)out_w - 0.5f;
}

// bilinear weights and clamped pixel indices along one axis
__device__ __forceinline__ void taps(float xs, uint32_t W, int &xa, int &xb, float &fx)
{
    const float x0 = floorf(xs);
    fx = xs - x0;
    const int xi = (int)x0;
    xa = min(max(xi, 0), (int)W - 1);
    xb = min(max(xi + 1, 0), (int)W - 1);
}

__device__ __forceinline__ float chan(uint32_t rgb, int c) { return (float)((rgb >> (8 * c)) & 255u); }

extern __shared__ __align__(16) unsigned char g_smem[];

__global__ void __launch_bounds__(kThreads) render_tiled_kernel(const Args a)
{
    __shared__ uint32_t s_mode[kNumModes];
    __shared__ int s_rect[4][4];   // per neighbour: block x0, y0, nbx, nby
    uint32_t *s_fp = reinterpret_cast<uint32_t *>(g_smem);   // [4][max_fp_blocks][16] packed RGB
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = blockIdx.y;
    const uint32_t tx0 = (blockIdx.x % a.tiles_x) * kTX, ty0 = (blockIdx.x / a.tiles_x) * kTY;
    const uint32_t tx1 = min(tx0 + kTX, a.out_w) - 1, ty1 = min(ty0 + kTY, a.out_h) - 1;
    const Camera cam = make_camera(a, n);
    if (tid < kNumModes)
        s_mode[tid] = c_modes[tid];
    if (tid < 4) {
        const int k = tid;
        int xa, xb, ya, yb;
        float f;
        taps(ray_s(tx0, a.W, a.out_w) + cam.shift_x[k], a.W, xa, xb, f);
        const int px_lo = xa;
        taps(ray_s(tx1, a.W, a.out_w) + cam.shift_x[k], a.W, xa, xb, f);
        const int px_hi = xb;
        taps(ray_s(ty0, a.H, a.out_h) + cam.shift_y[k], a.H, ya, yb, f);
        const int py_lo = ya;
        taps(ray_s(ty1, a.H, a.out_h) + cam.shift_y[k], a.H, ya, yb, f);
        const int py_hi = yb;
        s_rect[k][0] = px_lo / kBlock;
        s_rect[k][1] = py_lo / kBlock;
        s_rect[k][2] = px_hi / kBlock - px_lo / kBlock + 1;
        s_rect[k][3] = py_hi / kBlock - py_lo / kBlock + 1;
        if (cam.w[k] == 0.0f)
            s_rect[k][2] = s_rect[k][3] = 0;   // a zero weight contributes nothing
    }
    __syncthreads();
    // on-demand decode of the footprint blocks, one block per warp step
    uint32_t total = 0, count[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        count[k] = (uint32_t)(s_rect[k][2] * s_rect[k][3]);
        total += count[k];
    }
    for (uint32_t item = warp; item < total; item += kThreads / 32) {
        uint32_t k = 0, r = item;
        while (r >= count[k]) {
            r -= count[k];
            k++;
        }
        const uint32_t nbx = (uint32_t)s_rect[k][2];
        const uint32_t bx = s_rect[k][0] + r % nbx, by = s_rect[k][1] + r / nbx;
        const uint32_t rgb = warp_decode_block(a.sv, s_mode, (uint32_t)cam.view[k], by * a.sv.nlx + bx, lane);
        if (lane < 16)
            s_fp[((size_t)k * a.max_fp_blocks + r) * 16 + lane] = rgb;
    }
    __syncthreads();
    const uint32_t x = tx0 + (tid % kTX), y = ty0 + (tid / kTX);
    if (x >= a.out_w || y >= a.out_h)
        return;
    const float s = ray_s(x, a.W, a.out_w), t = ray_s(y, a.H, a.out_h);
    float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (cam.w[k] == 0.0f)
            continue;
        int xa, xb, ya, yb;
        float fx, fy;
        taps(s + cam.shift_x[k], a.W, xa, xb, fx);
        taps(t + cam.shift_y[k], a.H, ya, yb, fy);
        const uint32_t *fp = s_fp + (size_t)k * a.max_fp_blocks * 16;
        const int bx0 = s_rect[k][0], by0 = s_rect[k][1], nbx = s_rect[k][2];
        auto px = [&](int xx, int yy) -> uint32_t {
            const int blk = (yy / kBlock - by0) * nbx + (xx / kBlock - bx0);
            return fp[blk * 16 + (yy % kBlock) * kBlock + (xx % kBlock)];
        };
        const uint32_t p00 = px(xa, ya), p10 = px(xb, ya), p01 = px(xa, yb), p11 = px(xb, yb);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float top = (1.0f - fx) * chan(p00, c) + fx * chan(p10, c);
            const float bot = (1.0f - fx) * chan(p01, c) + fx * chan(p11, c);
            acc[c] += cam.w[k] * (((1.0f - fy) * top + fy * bot) / 255.0f);
        }
    }
    store_rgb(a.out, a.out8, ((size_t)n * a.out_h + y) * a.out_w + x, acc[0], acc[1], acc[2]);
}

// One pixel of one view, decoded by a single thread: walk the record of each
// channel to the view's ancestors and extract the one value needed.
__device__ uint32_t thread_decode_pixel(const StreamView &sv, const uint32_t *s_mode, uint32_t view,
                                        uint32_t x, uint32_t y)
{
    const uint32_t loc = (y / kBlock) * sv.nlx + x / kBlock;
    const uint32_t v = (y % kBlock) * kBlock + x % kBlock;
    const uint32_t *anc = sv.view_anc + view * kMaxLevels;
    int32_t ycc[3];
    for (int c = 0; c < 3; c++) {
        const uint32_t *rec = sv.records + sv.offsets[3 * loc + c];
        int32_t acc = sv.top[((size_t)anc[sv.L - 1] * sv.nloc + loc) * 48 + c * 16 + v];
        uint32_t P = 0;
        for (uint32_t m = 0; m < sv.MW; m++)
            P += __popc(rec[m]);
        const uint32_t hdr0 = 32 * sv.MW;
        for (uint32_t l = 0; l + 1 < sv.L; l++) {
            const uint32_t p = anc[l];
            if (!((rec[p >> 5] >> (p & 31u)) & 1u))
                continue;
            uint32_t rank = 0;
            for (uint32_t m = 0; m < (p >> 5); m++)
                rank += __popc(rec[m]);
            rank += __popc(rec[p >> 5] & ((1u << (p & 31u)) - 1u));
            uint32_t off = hdr0 + kHdrBits * P;
            for (uint32_t h = 0; h < rank; h++)
                off += mode_bits(s_mode[get_bits(rec, hdr0 + kHdrBits * h, 5)]);
            const BlockHeader hd = unpack_header(get_bits(rec, hdr0 + kHdrBits * rank, kHdrBits));
            const uint32_t u = bise_value(rec, off, s_mode[hd.mode], v);
            acc += (hd.min + (int32_t)u) * (1 << (sv.q + hd.shift));
        }
        ycc[c] = acc;
    }
    return ycocg_to_rgb24(ycc[0], ycc[1], ycc[2]);
}

__global__ void __launch_bounds__(256) render_direct_kernel(const Args a)
{
    __shared__ uint32_t s_mode[kNumModes];
    if (threadIdx.x < kNumModes)
        s_mode[threadIdx.x] = c_modes[threadIdx.x];
    __syncthreads();
    const uint32_t n = blockIdx.y;
    const uint32_t pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= a.out_w * a.out_h)
        return;
    const uint32_t x = pix % a.out_w, y = pix / a.out_w;
    const Camera cam = make_camera(a, n);
    const float s = ray_s(x, a.W, a.out_w), t = ray_s(y, a.H, a.out_h);
    float acc[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < 4; k++) {
        if (cam.w[k] == 0.0f)
            continue;
        int xa, xb, ya, yb;
        float fx, fy;
        taps(s + cam.shift_x[k], a.W, xa, xb, fx);
        taps(t + cam.shift_y[k], a.H, ya, yb, fy);
        const uint32_t vw = (uint32_t)cam.view[k];
        const uint32_t p00 = thread_decode_pixel(a.sv, s_mode, vw, xa, ya);
        const uint32_t p10 = thread_decode_pixel(a.sv, s_mode, vw, xb, ya);
        const uint32_t p01 = thread_decode_pixel(a.sv, s_mode, vw, xa, yb);
        const uint32_t p11 = thread_decode_pixel(a.sv, s_mode, vw, xb, yb);
        for (int c = 0; c < 3; c++) {
            const float top = (1.0f - fx) * chan(p00, c) + fx * chan(p10, c);
            const float bot = (1.0f - fx) * chan(p01, c) + fx * chan(p11, c);
            acc[c] += cam.w[k] * (((1.0f - fy) * top + fy * bot) / 255.0f);
        }
    }
    store_rgb(a.out, a.out8, ((size_t)n * a.out_h + y) * a.out_w + x, acc[0], acc[1], acc[2]);
}

}  // namespace

int launch_render(const rlfc_stream *s, const float *d_uv, const float *d_disp, uint32_t out_w,
                  uint32_t out_h, uint32_t n, float *d_out, cudaStream_t st, uint8_t *d_out8)
{
    if (out_w == s->info.W && out_h == s->info.H) {
        const int rc = launch_render_native(s, d_uv, d_disp, n, d_out, st, d_out8);
        if (rc != RLFC_E_UNSUPPORTED)
            return rc;
    }
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
    a.out_w = out_w;
    a.out_h = out_h;
    a.tiles_x = (out_w + kTX - 1) / kTX;
    const uint32_t tiles_y = (out_h + kTY - 1) / kTY;
    // footprint of a tile in one view: the sample span of kTX (kTY) rays plus
    // the bilinear neighbour, in whole blocks (plus one for misalignment and
    // one for float rounding of the corner rays)
    const double span_x = (kTX - 1) * (double)a.W / out_w + 2.0;
    const double span_y = (kTY - 1) * (double)a.H / out_h + 2.0;
    const uint64_t bx = (uint64_t)(span_x / kBlock) + 3, by = (uint64_t)(span_y / kBlock) + 3;
    const uint64_t fp_blocks = std::min<uint64_t>(bx, s->info.nloc_x) * std::min<uint64_t>(by, s->info.nloc_y);
    const uint64_t smem = 4 * fp_blocks * 16 * sizeof(uint32_t);
    cudaError_t e;
    if (smem <= kFootprintBudget && (uint64_t)a.tiles_x * tiles_y < (1ull << 31)) {
        a.max_fp_blocks = (uint32_t)fp_blocks;
        e = cudaFuncSetAttribute(render_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return cuda_fail(e, "render: shared memory attribute");
        dim3 grid(a.tiles_x * tiles_y, n);
        { rlfc::TraceScope trace_("render_tiled_kernel", st); render_tiled_kernel<<<grid, kThreads, smem, st>>>(a); }
    } else {
        a.max_fp_blocks = 0;
        const uint64_t pix = (uint64_t)out_w * out_h;
        if (pix >= (1ull << 31)) {
            set_error("output view too large");
            return RLFC_E_RANGE;
        }
        dim3 grid((uint32_t)((pix + 255) / 256), n);
        { rlfc::TraceScope trace_("render_direct_kernel", st); render_direct_kernel<<<grid, 256, 0, st>>>(a); }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "render launch");
    return RLFC_OK;
}

}  // namespace rlfc

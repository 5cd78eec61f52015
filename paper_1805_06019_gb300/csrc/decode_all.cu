// Full light-field decode: Algorithm 2 for every (view, block location).
//
// One CTA owns a strip of kStrip consecutive block locations of one block row.
// The strip's records are contiguous in the stream (location-major, then
// Y / Co / Cg), so they are staged into shared memory with coalesced 16-byte
// loads, together with the strip's top-RKV blocks.  Three walker warps (one per
// channel, lane = location) then walk their record once in BFS order:
// internal nodes (levels >= 1) are reconstructed into shared memory as
// parent + residual, leaves (the views) are reconstructed the same way in
// batches of kLeafBatch, converted from YCoCg-R to RGB by all four warps and
// written as whole 384-byte image rows.  Every SRV block of the strip is thus
// decoded exactly once and every output byte written once.
//
// A second instantiation writes one packed RGB word per pixel (r | g << 8 |
// b << 16, 512-byte rows) and decodes only the views a per-view mask asks for;
// the renderer uses it to decode, from the compressed stream, just the views a
// batch of new cameras samples.
#include <cuda_runtime.h>

#include <algorithm>

#include "rlfc_device.cuh"
#include "rlfc_internal.h"

namespace rlfc {
namespace {

constexpr int kStrip = 32;       // block locations per CTA
constexpr int kThreads = 128;
constexpr int kLeafBatch = 8;
constexpr uint32_t kSmemBudget = 200 * 1024;

__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

struct Args {
    const uint32_t *records;
    const uint32_t *offsets;
    const int16_t *top;
    const uint32_t *node_info;
    uint8_t *out;          // RGB bytes, or packed RGB words (packed instantiation)
    const uint8_t *needed; // packed instantiation: per-view mask (nonzero = decode), may be null
    uint32_t S, n_int, n_top, L, q, MW;
    uint32_t nlx, nloc, W, H;
    uint32_t out_aligned16; // output base is 16-byte aligned
    uint32_t node_words;   // S rounded up to 4
    uint32_t stage_words;  // capacity of the record staging area (multiple of 4)
};

// Decode SRV node p of a record into v (zeros when the node has no block).
__device__ __forceinline__ void decode_node(const uint32_t *rec, uint32_t p, uint32_t &hdr_pos,
                                            uint32_t &pay_pos, const uint32_t *s_mode, uint32_t q,
                                            int32_t v[kVals])
{
    if ((rec[p >> 5] >> (p & 31u)) & 1u) {
        const BlockHeader h = unpack_header(get_bits(rec, hdr_pos, kHdrBits));
        hdr_pos += kHdrBits;
        const uint32_t m = s_mode[h.mode];
        int32_t u[kVals];
        bise_decode16(rec, pay_pos, m, u);
        pay_pos += mode_bits(m);
        const int32_t scale = 1 << (q + h.shift);
#pragma unroll
        for (int k = 0; k < kVals; k++)
            v[k] = (h.min + u[k]) * scale;
    } else {
#pragma unroll
        for (int k = 0; k < kVals; k++)
            v[k] = 0;
    }
}

// Step past SRV node p of a record without decoding it.
__device__ __forceinline__ void skip_node(const uint32_t *rec, uint32_t p, uint32_t &hdr_pos, uint32_t &pay_pos,
                                          const uint32_t *s_mode)
{
    if ((rec[p >> 5] >> (p & 31u)) & 1u) {
        pay_pos += mode_bits(s_mode[get_bits(rec, hdr_pos, 5)]);
        hdr_pos += kHdrBits;
    }
}

extern __shared__ __align__(16) unsigned char g_smem[];

template <bool kPacked>
__global__ void __launch_bounds__(kThreads) decode_all_kernel(const Args a)
{
    constexpr uint32_t kRowBytes = kPacked ? kStrip * 16 : kStrip * 12;
    __shared__ uint32_t s_mode[kNumModes];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bx0 = blockIdx.x * kStrip, by = blockIdx.y;
    const uint32_t nl = min((uint32_t)kStrip, a.nlx - bx0);
    const uint32_t b0 = by * a.nlx + bx0;

    uint32_t *s_node = reinterpret_cast<uint32_t *>(g_smem);
    int16_t *s_top = reinterpret_cast<int16_t *>(s_node + a.node_words);       // [n_top][48][kStrip]
    int16_t *s_int = s_top + (size_t)a.n_top * 48 * kStrip;                     // [n_int][48][kStrip]
    int16_t *s_leaf = s_int + (size_t)a.n_int * 48 * kStrip;                    // [batch][48][kStrip]
    uint8_t *s_rgb = reinterpret_cast<uint8_t *>(s_leaf + kLeafBatch * 48 * kStrip);  // [batch*4][kRowBytes]
    uint32_t *s_words = reinterpret_cast<uint32_t *>(s_rgb + kLeafBatch * 4 * kStrip * 16);

    if (tid < kNumModes)
        s_mode[tid] = c_modes[tid];
    for (uint32_t i = tid; i < a.S; i += kThreads)
        s_node[i] = a.node_info[i];
    for (uint32_t i = tid; i < a.n_top * nl * 48; i += kThreads) {
        const uint32_t t = i / (nl * 48), r = i - t * nl * 48, loc = r / 48, cv = r - loc * 48;
        s_top[(t * 48 + cv) * kStrip + loc] = a.top[((size_t)t * a.nloc + b0 + loc) * 48 + cv];
    }
    const uint32_t w_begin = a.offsets[3 * b0], w_end = a.offsets[3 * (b0 + nl)];
    const uint32_t base = w_begin & ~3u;
    const uint32_t n16 = (w_end + 2 - base + 3) / 4;
    const bool staged = n16 * 4 <= a.stage_words;
    if (staged) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.records) + base / 4;
        uint4 *dst = reinterpret_cast<uint4 *>(s_words);
        for (uint32_t i = tid; i < n16; i += kThreads)
            dst[i] = src[i];
    }
    __syncthreads();

    const bool walker = warp < 3 && (uint32_t)lane < nl;
    const uint32_t c = warp;
    const uint32_t *rec = nullptr;
    uint32_t hdr_pos = 0, pay_pos = 0;
    if (walker) {
        const uint32_t w0 = a.offsets[3 * (b0 + lane) + c];
        rec = staged ? s_words + (w0 - base) : a.records + w0;
        uint32_t P = 0;
        for (uint32_t m = 0; m < a.MW; m++)
            P += __popc(rec[m]);
        hdr_pos = 32 * a.MW;
        pay_pos = hdr_pos + kHdrBits * P;
    }

    // levels >= 1 first (BFS order lists them before the views)
    if (walker) {
        for (uint32_t p = 0; p < a.n_int; p++) {
            int32_t v[kVals];
            decode_node(rec, p, hdr_pos, pay_pos, s_mode, a.q, v);
            const uint32_t info = s_node[p];
            const uint32_t par = node_parent(info);
            const int16_t *src = (node_level(info) + 2 == a.L ? s_top : s_int) + (par * 48 + c * 16) * kStrip;
            int16_t *dst = s_int + (p * 48 + c * 16) * kStrip;
#pragma unroll
            for (int k = 0; k < kVals; k++)
                dst[k * kStrip + lane] = (int16_t)(src[k * kStrip + lane] + v[k]);
        }
    }

    const bool fast_rows = a.out_aligned16 && (a.W % (kPacked ? 4 : 16) == 0) && nl == kStrip && bx0 * 4 + kStrip * 4 <= a.W;
    for (uint32_t p0 = a.n_int; p0 < a.S; p0 += kLeafBatch) {
        const uint32_t nb = min((uint32_t)kLeafBatch, a.S - p0);
        if (walker) {
            for (uint32_t j = 0; j < nb; j++) {
                const uint32_t p = p0 + j;
                const uint32_t info = s_node[p];
                if (kPacked && a.needed && !a.needed[node_view(info)]) {
                    skip_node(rec, p, hdr_pos, pay_pos, s_mode);
                    continue;
                }
                int32_t v[kVals];
                decode_node(rec, p, hdr_pos, pay_pos, s_mode, a.q, v);
                const uint32_t par = node_parent(info);
                const int16_t *src = (node_level(info) + 2 == a.L ? s_top : s_int) + (par * 48 + c * 16) * kStrip;
                int16_t *dst = s_leaf + (j * 48 + c * 16) * kStrip;
#pragma unroll
                for (int k = 0; k < kVals; k++)
                    dst[k * kStrip + lane] = (int16_t)(src[k * kStrip + lane] + v[k]);
            }
        }
        __syncthreads();
        // YCoCg-R -> RGB, one (leaf, pixel row) per warp iteration, lane = location
        for (uint32_t job = warp; job < nb * 4; job += kThreads / 32) {
            const uint32_t j = job >> 2, row = job & 3;
            const uint32_t view = node_view(s_node[p0 + j]);
            if (kPacked && a.needed && !a.needed[view])
                continue;
            uint8_t *srow = s_rgb + job * kRowBytes;
            if ((uint32_t)lane < nl) {
                uint32_t px[4];
#pragma unroll
                for (int x = 0; x < 4; x++) {
                    const uint32_t k = row * 4 + x;
                    const int16_t *lv = s_leaf + j * 48 * kStrip;
                    px[x] = ycocg_to_rgb24(lv[k * kStrip + lane], lv[(16 + k) * kStrip + lane],
                                           lv[(32 + k) * kStrip + lane]);
                }
                if (kPacked) {
                    reinterpret_cast<uint4 *>(srow)[lane] = make_uint4(px[0], px[1], px[2], px[3]);
                } else {
                    uint32_t *w = reinterpret_cast<uint32_t *>(srow + lane * 12);
                    w[0] = px[0] | (px[1] << 24);
                    w[1] = (px[1] >> 8) | (px[2] << 16);
                    w[2] = (px[2] >> 16) | (px[3] << 8);
                }
            }
            __syncwarp();
            const uint32_t y = by * 4 + row, x0 = bx0 * 4;
            if (y < a.H && x0 < a.W) {
                if (kPacked) {
                    uint32_t *dst = reinterpret_cast<uint32_t *>(a.out) + ((size_t)view * a.H + y) * a.W + x0;
                    const uint32_t *src = reinterpret_cast<const uint32_t *>(srow);
                    if (fast_rows) {
                        reinterpret_cast<uint4 *>(dst)[lane] = reinterpret_cast<const uint4 *>(src)[lane];
                    } else {
                        const uint32_t npx = min(nl * 4, a.W - x0);
                        for (uint32_t b = lane; b < npx; b += 32)
                            dst[b] = src[b];
                    }
                } else {
                    uint8_t *dst = a.out + (((size_t)view * a.H + y) * a.W + x0) * 3;
                    if (fast_rows) {
                        if (lane < kStrip * 12 / 16)
                            reinterpret_cast<uint4 *>(dst)[lane] = reinterpret_cast<const uint4 *>(srow)[lane];
                    } else {
                        const uint32_t nbytes = min(nl * 4, a.W - x0) * 3;
                        for (uint32_t b = lane; b < nbytes; b += 32)
                            dst[b] = srow[b];
                    }
                }
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

}  // namespace

namespace {

template <bool kPacked>
int launch_decode(const rlfc_stream *s, uint8_t *d_out, const uint8_t *needed, cudaStream_t st)
{
    const Tables &t = s->tab;
    Args a;
    a.records = s->d_records;
    a.offsets = s->d_offsets;
    a.top = s->d_top;
    a.node_info = s->d_node_info;
    a.out = d_out;
    a.needed = needed;
    a.S = t.S;
    a.n_int = t.n_int;
    a.n_top = t.n_top;
    a.L = t.L;
    a.q = s->info.q;
    a.MW = s->MW;
    a.nlx = s->info.nloc_x;
    a.nloc = s->info.nloc_x * s->info.nloc_y;
    a.W = s->info.W;
    a.H = s->info.H;
    a.out_aligned16 = ((uintptr_t)d_out & 15u) == 0;
    a.node_words = (t.S + 3) & ~3u;
    const size_t fixed = 4ull * a.node_words + 2ull * (t.n_top + t.n_int + kLeafBatch) * 48 * kStrip +
                         (size_t)kLeafBatch * 4 * kStrip * 16;
    if (fixed + 1024 > kSmemBudget) {
        set_error("tree too large for the decode-all kernel's shared memory");
        return RLFC_E_UNSUPPORTED;
    }
    // stage whole strips when they fit (the largest strip plus alignment slack)
    const size_t want = (size_t)s->max_strip_words + 8;
    const size_t room = (kSmemBudget - fixed) / 16 * 4;
    a.stage_words = (uint32_t)std::min(room, (want + 3) & ~size_t(3));
    const size_t smem = fixed + 4ull * a.stage_words;
    cudaError_t e = cudaFuncSetAttribute(decode_all_kernel<kPacked>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "decode_all: shared memory attribute");
    dim3 grid((a.nlx + kStrip - 1) / kStrip, s->info.nloc_y);
    decode_all_kernel<kPacked><<<grid, kThreads, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "decode_all launch");
    return RLFC_OK;
}

}  // namespace

int launch_decode_all(const rlfc_stream *s, uint8_t *d_out, cudaStream_t st)
{
    return launch_decode<false>(s, d_out, nullptr, st);
}

int launch_decode_packed(const rlfc_stream *s, uint32_t *d_out, const uint8_t *needed, cudaStream_t st)
{
    return launch_decode<true>(s, reinterpret_cast<uint8_t *>(d_out), needed, st);
}

}  // namespace rlfc

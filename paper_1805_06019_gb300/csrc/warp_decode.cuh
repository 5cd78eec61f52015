// Warp-cooperative random-access decode of one block (Algorithm 2,
// DecompressLFIBlock) for any (view, location): used by the request decoder
// and by the renderer's on-demand decode.
//
// For each channel the warp reads the record's presence mask, turns the
// ancestors' BFS positions into ranks with popcounts and a warp scan, sums the
// closed-form payload lengths of the stored blocks in front of each ancestor
// (32 headers per step, one per lane, then a warp scan), and extracts the
// ancestors' BISE values lane-per-value: lanes 0..15 and 16..31 take one tree
// level each, so a three-level tree decodes both SRV levels in one pass.
#pragma once

#include "rlfc_device.cuh"
#include "rlfc_internal.h"

namespace rlfc {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

struct StreamView {
    const uint32_t *records;
    const uint32_t *offsets;
    const int16_t *top;
    const uint32_t *view_anc;
    uint32_t n_views, nloc, nlx, L, q, MW;
    uint32_t *dbg = nullptr;   // debug builds: the stream's flag word (rlfc_debug_flags)
};

__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t x, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, x, d);
        if (lane >= d)
            x += y;
    }
    return x;
}

// Value v (0..15) of a BISE block at bit `pos` in (packed) mode m.
__device__ __forceinline__ uint32_t bise_value(const uint32_t *rec, uint32_t pos, uint32_t m, uint32_t v)
{
    const uint32_t b = mode_b(m), kind = mode_kind(m);
    uint32_t digit = 0, D = 0;
    if (kind == 1) {
        const uint32_t g = v / 5, e = v - 5 * g;
        uint32_t t = get_bits(rec, pos + 8 * g, g < 3 ? 8u : 2u);
        for (uint32_t i = 0; i < e; i++)
            t /= 3u;
        digit = t % 3u;
        D = 26;
    } else if (kind == 2) {
        const uint32_t g = v / 3, e = v - 3 * g;
        uint32_t t = get_bits(rec, pos + 7 * g, g < 5 ? 7u : 3u);
        for (uint32_t i = 0; i < e; i++)
            t /= 5u;
        digit = t % 5u;
        D = 38;
    }
    return (digit << b) | get_bits(rec, pos + D + v * b, b);
}

// Decode block `loc` of `view` (both in range) cooperatively; lanes 0..15 get
// pixel `lane` of the block as packed RGB (r | g << 8 | b << 16).  All 32 lanes
// must call it with the same arguments.
__device__ __forceinline__ uint32_t warp_decode_block(const StreamView &sv, const uint32_t *s_mode,
                                                      uint32_t view, uint32_t loc, int lane)
{
    const uint32_t anc_l = lane < (int)sv.L ? sv.view_anc[view * kMaxLevels + lane] : 0u;
    const uint32_t top_idx = __shfl_sync(kFullMask, anc_l, sv.L - 1);
    const uint32_t v = lane & 15;
    int32_t ycc[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const uint32_t *rec = sv.records + sv.offsets[3 * loc + c];
        int32_t acc = lane < 16 ? sv.top[((size_t)top_idx * sv.nloc + loc) * 48 + c * 16 + v] : 0;
        // lane l < L-1 tracks the ancestor at level l: is it stored, and its rank
        uint32_t total = 0, my_rank = 0, my_present = 0;
        const uint32_t my_pos = anc_l;
        for (uint32_t w0 = 0; w0 < sv.MW; w0 += 32) {
            const uint32_t wi = w0 + lane;
            const uint32_t word = wi < sv.MW ? rec[wi] : 0u;
            const uint32_t cnt = __popc(word);
            const uint32_t incl = warp_inclusive_scan(cnt, lane);
            const int src = (int)(my_pos >> 5) - (int)w0;
            const uint32_t src_c = (uint32_t)min(max(src, 0), 31);
            const uint32_t src_word = __shfl_sync(kFullMask, word, src_c);
            const uint32_t src_excl = __shfl_sync(kFullMask, incl - cnt, src_c);
            if (src >= 0 && src < 32) {
                const uint32_t bit = my_pos & 31u;
                my_present = (src_word >> bit) & 1u;
                my_rank = total + src_excl + __popc(src_word & ((1u << bit) - 1u));
            }
            total += __shfl_sync(kFullMask, incl, 31);
        }
        // payload offset of each tracked ancestor: the lengths of the stored
        // blocks in front of it, 32 headers per step
        const uint32_t hdr0 = 32 * sv.MW;
        const uint32_t pay0 = hdr0 + kHdrBits * total;
        uint32_t max_rank = 0;
        for (uint32_t l = 0; l + 1 < sv.L; l++)
            max_rank = max(max_rank, __shfl_sync(kFullMask, my_present ? my_rank : 0u, l));
        uint32_t my_off = pay0, run = 0;
        for (uint32_t h0 = 0; h0 < max_rank; h0 += 32) {
            const uint32_t hi = h0 + lane;
            const uint32_t len = hi < total ? mode_bits(s_mode[get_bits(sv.records + sv.offsets[3 * loc + c],
                                                                        hdr0 + kHdrBits * hi, 5)])
                                            : 0u;
            const uint32_t incl = warp_inclusive_scan(len, lane);
            const int src = (int)my_rank - (int)h0;   // prefix of the first `src` headers of this step
            const uint32_t pre = __shfl_sync(kFullMask, incl, (uint32_t)min(max(src - 1, 0), 31));
            if (src > 0 && src <= 32)
                my_off = pay0 + run + pre;
            run += __shfl_sync(kFullMask, incl, 31);
        }
        // lane-per-value extraction, two SRV levels per pass
        for (uint32_t l0 = 0; l0 + 1 < sv.L; l0 += 2) {
            const uint32_t l = l0 + (uint32_t)(lane >> 4);
            const bool in_tree = l + 1 < sv.L;
            const uint32_t src_lane = in_tree ? l : 0u;
            const uint32_t present = __shfl_sync(kFullMask, my_present, src_lane);
            const uint32_t rank = __shfl_sync(kFullMask, my_rank, src_lane);
            const uint32_t off = __shfl_sync(kFullMask, my_off, src_lane);
            int32_t val = 0;
            if (in_tree && present) {
                const BlockHeader h = unpack_header(get_bits(rec, hdr0 + kHdrBits * rank, kHdrBits));
#ifdef RLFC_DEBUG
                const uint32_t rec_bits = 32u * (sv.offsets[3 * loc + c + 1] - sv.offsets[3 * loc + c]);
                const bool ok = RLFC_DBG_BLOCK_OK(sv.dbg, h.mode, hdr0 + kHdrBits * (rank + 1), pay0, off,
                                                  h.mode < (uint32_t)kNumModes ? mode_bits(s_mode[h.mode]) : 0u,
                                                  rec_bits);
#else
                constexpr bool ok = true;
#endif
                if (ok) {
                    const uint32_t u = bise_value(rec, off, s_mode[h.mode], v);
                    val = (h.min + (int32_t)u) * (1 << (sv.q + h.shift));
                }
            }
            val += __shfl_down_sync(kFullMask, val, 16);
            acc += val;
        }
        ycc[c] = acc;
    }
    return ycocg_to_rgb24(ycc[0], ycc[1], ycc[2]);
}

}  // namespace rlfc

// Device-side building blocks of the RLFC decoder (paper Section 3.3-3.5,
// Algorithm 2) for sm_103a.  Integer work only: bit extraction with funnel
// shifts, trit/quint digit splitting, residual accumulation and the inverse
// YCoCg-R of Section 4.
#pragma once

#include <cstdint>

namespace rlfc {

constexpr int kNumModes = 28;
constexpr int kBlock = 4;          // block side handled by the kernels
constexpr int kVals = 16;          // values per channel block (kBlock^2)
constexpr int kHdrBits = 18;       // block header: mode 5 | shift 2 | min 11

// Mode k -> packed (payload bits for 16 values) | b << 8 | kind << 12,
// kind 0 = plain bits, 1 = trits (N = 3*2^b), 2 = quints (N = 5*2^b).
// The ranges ascend: 1 2 3 4 5 6 8 10 12 16 20 24 ... 640 768 1024.
__host__ __device__ constexpr uint32_t pack_mode(uint32_t kind, uint32_t b)
{
    return (16u * b + (kind == 1 ? 26u : (kind == 2 ? 38u : 0u))) | (b << 8) | (kind << 12);
}

#define RLFC_MODE_TABLE_INIT                                                          \
    {pack_mode(0, 0),  pack_mode(0, 1), pack_mode(1, 0), pack_mode(0, 2),             \
     pack_mode(2, 0),  pack_mode(1, 1), pack_mode(0, 3), pack_mode(2, 1),             \
     pack_mode(1, 2),  pack_mode(0, 4), pack_mode(2, 2), pack_mode(1, 3),             \
     pack_mode(0, 5),  pack_mode(2, 3), pack_mode(1, 4), pack_mode(0, 6),             \
     pack_mode(2, 4),  pack_mode(1, 5), pack_mode(0, 7), pack_mode(2, 5),             \
     pack_mode(1, 6),  pack_mode(0, 8), pack_mode(2, 6), pack_mode(1, 7),             \
     pack_mode(0, 9),  pack_mode(2, 7), pack_mode(1, 8), pack_mode(0, 10)}

__device__ __forceinline__ uint32_t mode_bits(uint32_t m) { return m & 0xFFu; }
__device__ __forceinline__ uint32_t mode_b(uint32_t m) { return (m >> 8) & 0xFu; }
__device__ __forceinline__ uint32_t mode_kind(uint32_t m) { return m >> 12; }

// Bounds checks of debug builds (compiled with RLFC_DEBUG).  Before a stored
// block is decoded, the decoders (full, per-request, binned and the
// renderer's on-demand decode) check it against its record: the mode index
// is one of the 28, the 18-bit header lies in the record's header area, and
// the payload lies inside the record.  A failed check sets its bit in the
// stream's flag word (rlfc_debug_flags) and the block is treated as absent,
// so nothing is read outside the record and the kernel never traps.  Release
// builds compile the checks away (the macro is `true`).
constexpr uint32_t kDbgMode = 1u;      // mode index >= 28
constexpr uint32_t kDbgHeader = 2u;    // header past the record's header area
constexpr uint32_t kDbgPayload = 4u;   // payload past the end of the record
constexpr uint32_t kDbgOutput = 8u;    // an output index out of range
#ifdef RLFC_DEBUG
// hdr_end: the bit after the block's header; hdr_area: the bit after the
// record's last header; pos, pay_bits: the payload; rec_bits: the record's
// length in bits.  `pay_bits` is read only for a valid mode.
__device__ __forceinline__ bool dbg_block_ok(uint32_t *flags, uint32_t mode, uint32_t hdr_end, uint32_t hdr_area,
                                             uint32_t pos, uint32_t pay_bits, uint32_t rec_bits)
{
    uint32_t bad = 0;
    if (mode >= (uint32_t)kNumModes)
        bad |= kDbgMode;
    if (hdr_end > hdr_area || hdr_area > rec_bits)
        bad |= kDbgHeader;
    if (mode < (uint32_t)kNumModes && (uint64_t)pos + pay_bits > rec_bits)
        bad |= kDbgPayload;
    if (bad && flags)
        atomicOr(flags, bad);
    return bad == 0;
}
__device__ __forceinline__ bool dbg_index_ok(uint32_t *flags, uint64_t i, uint64_t n)
{
    if (i < n)
        return true;
    if (flags)
        atomicOr(flags, kDbgOutput);
    return false;
}
#define RLFC_DBG_BLOCK_OK(...) ::rlfc::dbg_block_ok(__VA_ARGS__)
#define RLFC_DBG_INDEX_OK(...) ::rlfc::dbg_index_ok(__VA_ARGS__)
#else
#define RLFC_DBG_BLOCK_OK(...) true
#define RLFC_DBG_INDEX_OK(...) true
#endif

// Bits [pos, pos + width) of a little-endian word array, width <= 32.  Reads
// words pos/32 and pos/32 + 1, so buffers carry one word of padding.
__device__ __forceinline__ uint32_t get_bits(const uint32_t *w, uint32_t pos, uint32_t width)
{
    const uint32_t i = pos >> 5;
    const uint32_t v = __funnelshift_r(w[i], w[i + 1], pos & 31u);
    return width >= 32u ? v : (v & ((1u << width) - 1u));
}

// Sequential reader over a bit string: a 64-bit window refilled one word at a
// time, so a block payload (at most 160 bits) costs at most six word loads.
struct BitReader {
    const uint32_t *w;
    uint64_t acc;
    uint32_t avail;
    uint32_t next;

    __device__ __forceinline__ BitReader(const uint32_t *words, uint32_t pos)
    {
        w = words;
        const uint32_t i = pos >> 5, sh = pos & 31u;
        acc = ((uint64_t)w[i] | ((uint64_t)w[i + 1] << 32)) >> sh;
        avail = 64u - sh;
        next = i + 2;
    }
    __device__ __forceinline__ uint32_t take(uint32_t width)  // width <= 32
    {
        if (avail < width) {
            acc |= (uint64_t)w[next++] << avail;
            avail += 32u;
        }
        const uint32_t v = (uint32_t)acc & (width >= 32u ? 0xFFFFFFFFu : ((1u << width) - 1u));
        acc >>= width;
        avail -= width;
        return v;
    }
};

// BISE payload of one 16-value block starting at bit `pos` -> u[0..15].
// Layout (stream format v1): trit blocks hold four digit words (three groups
// of five values in 8 bits, the last value in 2 bits), quint blocks six (five
// groups of three in 7 bits, the last value in 3 bits), then the sixteen
// b-bit low parts.
__device__ __forceinline__ void bise_decode16(const uint32_t *rec, uint32_t pos, uint32_t mode,
                                              int32_t u[kVals])
{
    const uint32_t b = mode_b(mode), kind = mode_kind(mode);
    BitReader br(rec, pos);
    uint32_t digits[kVals];
#pragma unroll
    for (int v = 0; v < kVals; v++)
        digits[v] = 0;
    if (kind == 1) {
#pragma unroll
        for (int g = 0; g < 4; g++) {
            uint32_t t = br.take(g < 3 ? 8u : 2u);
#pragma unroll
            for (int e = 0; e < 5; e++) {
                const int v = 5 * g + e;
                if (v < kVals) {
                    digits[v] = t % 3u;
                    t /= 3u;
                }
            }
        }
    } else if (kind == 2) {
#pragma unroll
        for (int g = 0; g < 6; g++) {
            uint32_t t = br.take(g < 5 ? 7u : 3u);
#pragma unroll
            for (int e = 0; e < 3; e++) {
                const int v = 3 * g + e;
                if (v < kVals) {
                    digits[v] = t % 5u;
                    t /= 5u;
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < kVals; v++)
        u[v] = (int32_t)((digits[v] << b) | br.take(b));
}

// Block header fields.
struct BlockHeader {
    uint32_t mode;   // index 0..27
    uint32_t shift;  // per-block extra shift
    int32_t min;     // 11-bit two's complement
};

__device__ __forceinline__ BlockHeader unpack_header(uint32_t h)
{
    BlockHeader r;
    r.mode = h & 31u;
    r.shift = (h >> 5) & 3u;
    r.min = ((int32_t)(h << 14)) >> 21;   // bits 7..17, sign-extended
    return r;
}

__device__ __forceinline__ int clamp255(int v) { return min(max(v, 0), 255); }

// Inverse YCoCg-R (Section 4), then clamp to 8 bits.
__device__ __forceinline__ uint32_t ycocg_to_rgb24(int y, int co, int cg)
{
    const int t = y - (cg >> 1);
    const int g = cg + t;
    const int b = t - (co >> 1);
    const int r = b + co;
    return (uint32_t)clamp255(r) | ((uint32_t)clamp255(g) << 8) | ((uint32_t)clamp255(b) << 16);
}

// 8-bit output of a rendered value: floor(clamp(v, 0, 1) * 255 + 0.5), the
// product and the sum each rounded on their own (never fused), so the result
// equals that of the same float operations anywhere else.
__device__ __forceinline__ uint8_t to_u8(float v)
{
    // __saturatef clamps to [0, 1] (NaN to 0); the argument of the
    // round-down conversion is at least 0.5, so it is the floor
    return (uint8_t)__float2uint_rd(__fadd_rn(__fmul_rn(__saturatef(v), 255.0f), 0.5f));
}

// Store a rendered RGB pixel (pixel index px) as floats, or as 8 bits when
// out8 is set.
__device__ __forceinline__ void store_rgb(float *out, uint8_t *out8, size_t px, float r, float g, float b)
{
    if (out8) {
        out8[px * 3] = to_u8(r);
        out8[px * 3 + 1] = to_u8(g);
        out8[px * 3 + 2] = to_u8(b);
    } else {
        out[px * 3] = r;
        out[px * 3 + 1] = g;
        out[px * 3 + 2] = b;
    }
}

}  // namespace rlfc

// Full light-field decode: Algorithm 2 for every (view, block location).
//
// One CTA owns a strip of kNL consecutive block locations of one block row.
// Its 3 * kNL records (location-major, then Y / Co / Cg) are contiguous in the
// stream; they are copied into shared memory when they fit the CTA's staging
// budget and read from the stream otherwise.  Phases:
//  1. parse (one warp per location): the warp stores its three records'
//     presence masks, the stored-block count in front of each mask word, and
//     the payload bit offset of every stored block (closed-form lengths of
//     the 18-bit headers, warp scan);
//  2. internal nodes (levels >= 1, first in BFS order), by the same warp,
//     level by level from the top: reconstruction = parent reconstruction
//     (or top RKV) + the decoded residual where a block is stored; then the
//     location's rows of every parent of a view are converted to RGB once;
//     one barrier, then
//  3. the views, one unit of 16 BFS positions at a time per warp (each warp
//     takes the next unit from a shared counter and never waits for the
//     others):
//     a. every block of the unit is written as its parent's RGB, the exact
//        result for every block without a stored residual (most of them);
//     b. then, for runs of locations whose stored blocks fit the warp's
//        kWSlots decode slots: the three channel masks give the items (a
//        view whose block has at least one stored channel) and the slots
//        (record, rank), their positions following from popcounts and one
//        warp scan; every slot is decoded by one lane (a mode-generic BISE
//        decoder: the payload is aligned once, digits come from base-3 /
//        base-5 tables, low parts from the slot's own words used as a column
//        of the aligned bits); every item adds its residual rows to the
//        parent rows, applies the inverse YCoCg-R two pixels per instruction
//        and overwrites its parent copy.
// Reconstructions are 16-bit values plus a bias of 2^14, two to a word (the
// loader refuses streams whose values could leave that range).  Every stored
// block of the strip is decoded once.
//
// A second instantiation writes one packed RGB word per pixel (r | g << 8 |
// b << 16) and decodes only the views a per-view mask asks for, into the
// output slots a table gives; the renderer uses it to decode, from the
// compressed stream, just the views a batch of new cameras samples.
#include <cuda_runtime.h>

#include <algorithm>

#include "warp_decode.cuh"

namespace rlfc {
namespace {

constexpr int kNL = (int)kDecodeStrip;          // block locations per CTA
constexpr int kRecs = 3 * kNL;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kUnit = 16;                        // BFS positions per unit of view work (half a mask word)
constexpr int kWSlots = 64;                      // decode slots per warp (one view of a unit always fits)
constexpr int kZeroSlot = kWSlots;               // a slot of zero residuals, for channels without a stored block
constexpr int kWItems = kNL * kUnit;             // items per warp at most (every block of a unit)
constexpr int kCols = 6;                         // column words of the generic decoder
constexpr uint32_t kSmemBudget = 200 * 1024;
constexpr size_t kCtaSmemTarget = 72 * 1024;     // three CTAs per SM: staging fills up to this
constexpr uint32_t kNodeSmemMax = 4096;          // node tables up to this size are cached per CTA

static_assert(kNL == 8, "the location and group splits below assume eight locations per strip");
static_assert(kCols <= 8, "the decoder's columns live in the slot's eight words");
static_assert(3 * kUnit <= kWSlots, "one location of a unit must fit the warp's slots");
static_assert(kNL == kWarps, "one warp per location of the strip in phases 1 and 2");
static_assert(kUnit == 16, "a unit must lie inside one 32-bit mask word");

// Reconstructions and residuals are held as 16-bit values plus a bias of
// 2^14, two to a word: then parent + residual is one 32-bit add for two
// values (no carry crosses a half while every value stays in
// [-2^14, 2^14)), and the inverse YCoCg-R runs on two pixels per
// instruction.
constexpr uint32_t kB2 = 0x40004000u;     // the bias in both halves (a zero pair)
constexpr uint32_t kHalfB2 = 0x20002000u;

// Decoder tables, built at compile time: the 28 modes (payload bits | b << 8
// | kind << 12, four unused entries), and the digits of t in base 3 (t <
// 256, five digits) and in base 5 (t < 128, three digits), three bits per
// digit.
struct DecodeTables {
    uint32_t mode[32];
    uint16_t dig[256 + 128];
    // per (kind - 1, block row): where the row's four digits sit.  Word 0:
    // bit offset of digit group A | of group B << 8 | first digit of the row
    // in group A << 16 | digits of the row in group A << 20; word 1: width
    // mask of group A | of group B << 8
    uint32_t row[2][4][2];
};

constexpr DecodeTables make_tables()
{
    DecodeTables t{};
    constexpr uint32_t modes[kNumModes] = RLFC_MODE_TABLE_INIT;
    for (int k = 0; k < 32; k++)
        t.mode[k] = k < kNumModes ? modes[k] : 0u;
    for (uint32_t i = 0; i < 256 + 128; i++) {
        const uint32_t base = i < 256 ? 3u : 5u, n = i < 256 ? 5u : 3u;
        uint32_t x = i < 256 ? i : i - 256, e = 0;
        for (uint32_t k = 0; k < n; k++) {
            e |= (x % base) << (3 * k);
            x /= base;
        }
        t.dig[i] = (uint16_t)e;
    }
    // trits: groups of five digits in 8 bits (the last, value 15, in 2 bits);
    // quints: groups of three in 7 bits (the last, value 15, in 3 bits)
    for (uint32_t kind = 1; kind <= 2; kind++) {
        const uint32_t per = kind == 1 ? 5u : 3u, gw = kind == 1 ? 8u : 7u, ng = kind == 1 ? 4u : 6u;
        const uint32_t last_w = kind == 1 ? 3u : 7u;
        for (uint32_t rr = 0; rr < 4; rr++) {
            const uint32_t v0 = 4 * rr, gA = v0 / per, eA = v0 % per;
            const uint32_t nA = (per - eA) < 4u ? (per - eA) : 4u, gB = gA + 1;
            const uint32_t mA = gA + 1 == ng ? last_w : (1u << gw) - 1u;
            const uint32_t mB = gB + 1 == ng ? last_w : (gB < ng ? (1u << gw) - 1u : 0u);
            t.row[kind - 1][rr][0] = (gw * gA) | ((gw * gB) << 8) | (eA << 16) | (nA << 20);
            t.row[kind - 1][rr][1] = mA | (mB << 8);
        }
    }
    return t;
}

__device__ const DecodeTables g_tables = make_tables();

struct Args {
    const uint32_t *records;
    const uint32_t *offsets;
    const int16_t *top;
    const uint32_t *node_info;
    uint8_t *out;            // RGB bytes, or packed RGB words (packed instantiation)
    const uint8_t *needed;   // packed instantiation: per-view mask (nonzero = decode), may be null
    const uint32_t *slot_of; // packed instantiation with a mask: output slot of each needed view
    uint32_t S, n_int, n_top, L, q, MW;
    uint32_t par_base;       // BFS position (or top index) of the first parent of a view
    uint32_t n_par;          // parents of views
    uint32_t nlx, nloc, W, H;
    uint32_t vec16;          // 16-byte stores of 4-location groups are aligned (RGB: W % 16 == 0; packed: W % 4 == 0)
    uint32_t vec4;           // 4-byte stores of one location's row are aligned (W % 4 == 0)
    uint32_t vec8;           // RGB: 8-byte stores at even locations are aligned (W % 8 == 0)
    uint32_t sec32;          // every strip row starts on a 32-byte boundary (RGB: W % 32 == 0; packed: W % 8 == 0)
    uint32_t pmax;           // largest number of stored blocks in one record
    uint32_t n_units;        // ceil(S / kUnit)
    uint32_t node_smem;      // the node table is cached in shared memory
    uint32_t stage_words;    // shared-memory words for the strip's records (0: read them from the stream)
    uint32_t lvl_begin[kMaxLevels];  // first BFS position of each internal level, top level first; [L-2] = n_int
};

template <bool kPacked>
__host__ __device__ constexpr uint32_t row_words() { return kPacked ? 4u : 3u; }

struct Smem {
    uint32_t *slots;   // [warp][kWSlots + 1][8]  decoded blocks, biased pairs; slot kZeroSlot is zero
    uint32_t *cols;    // [warp][kCols][32]  the generic decoder's columns, one per lane
    uint32_t *top;     // [n_top][kNL][24]  biased pairs
    uint32_t *inter;   // [n_int][kNL][24]  internal reconstructions, biased pairs
    uint32_t *mask;    // [kRecs][MW]
    uint32_t *mpre;    // [kRecs][MW]  stored blocks in front of each mask word
    uint32_t *need;    // [MW]  views to decode (bit per BFS position)
    uint32_t *node;    // [S]  node table (when cached)
    uint32_t *sent;    // [warp][kWSlots]  record | rank << 8
    uint32_t *items;   // [warp][kWItems]  p | l << 14 | stored channels << 18 | first slot << 21
    uint32_t *prgb;    // [n_par][4][kNL][row_words]  parent rows converted to RGB
    void *off;         // [kRecs][pmax]  payload bit offset of each stored block (OffT)
    uint32_t *stage;   // [stage_words]  the strip's records, from a 16-byte boundary
};

extern __shared__ __align__(16) unsigned char g_smem[];

__host__ __device__ inline size_t r16(size_t b) { return (b + 15) & ~size_t(15); }

// Shared-memory layout; the same function sizes it on the host (base null).
template <bool kPacked>
__host__ __device__ inline size_t layout(unsigned char *base, const Args &a, size_t off_size, Smem *m)
{
    size_t at = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base ? base + at : nullptr;
        at += r16(bytes);
        return p;
    };
    Smem s;
    s.slots = reinterpret_cast<uint32_t *>(take(32ull * (kWSlots + 1) * kWarps));
    s.cols = reinterpret_cast<uint32_t *>(take(4ull * kCols * 32 * kWarps));
    s.top = reinterpret_cast<uint32_t *>(take(96ull * a.n_top * kNL));
    s.inter = reinterpret_cast<uint32_t *>(take(96ull * a.n_int * kNL));
    s.mask = reinterpret_cast<uint32_t *>(take(4ull * kRecs * a.MW));
    s.mpre = reinterpret_cast<uint32_t *>(take(4ull * kRecs * a.MW));
    s.need = reinterpret_cast<uint32_t *>(take(4ull * a.MW));
    s.node = reinterpret_cast<uint32_t *>(take(a.node_smem ? 4ull * a.S : 0));
    s.sent = reinterpret_cast<uint32_t *>(take(4ull * kWSlots * kWarps));
    s.items = reinterpret_cast<uint32_t *>(take(4ull * kWItems * kWarps));
    s.prgb = reinterpret_cast<uint32_t *>(take(16ull * row_words<kPacked>() * a.n_par * kNL));
    s.off = take(off_size * kRecs * a.pmax);
    s.stage = reinterpret_cast<uint32_t *>(take(4ull * a.stage_words));
    if (m)
        *m = s;
    return at;
}

// ---- one BISE block, any mode ---------------------------------------------
//
// The payload (at most 160 bits) is aligned to its first bit once, into
// seven words.  The digit words of a trit or quint block sit at fixed
// positions: their digits come from s_dig (base-3 digits of t < 256 at bits
// 3e, then base-5 digits of t < 128) and are gathered into one 64-bit word,
// digit v at bits 3v.  The low parts, at D + v * b for a b known only at run
// time, are read from a column of the aligned bits in shared memory (word k
// at col[k * 32]: one word per lane per row, no bank conflicts).
// The 16 values come out dequantised and biased, two to a word.
__device__ __forceinline__ void decode_block_generic(const uint32_t *rec, uint32_t pos, uint32_t hdr, uint32_t q,
                                                     const uint32_t *s_mode, const uint16_t *s_dig, uint32_t *col,
                                                     uint32_t out[8])
{
    const uint32_t mp = s_mode[hdr & 31u];
    const uint32_t b = mode_b(mp), kind = mode_kind(mp);
    const uint32_t scale = 1u << (q + ((hdr >> 5) & 3u));
    const int32_t mn = ((int32_t)(hdr << 14)) >> 21;   // header bits 7..17, sign-extended
    const uint32_t base = (uint32_t)mn * scale + 0x4000u;
    const uint32_t *w = rec + (pos >> 5);
    const uint32_t sh = pos & 31u;
    uint32_t A[7];
    {
        uint32_t raw[8];
#pragma unroll
        for (int k = 0; k < 8; k++)
            raw[k] = w[k];
#pragma unroll
        for (int k = 0; k < 7; k++)
            A[k] = __funnelshift_r(raw[k], raw[k + 1], sh);
    }
    uint64_t dw = 0;
    uint32_t Lw[kCols];
    if (kind == 1) {
        // trits: three 8-bit digit words and a 2-bit one (value 15), then the low parts at bit 26
        uint32_t t3 = (A[0] >> 24) & 3u;
        t3 = t3 == 3u ? 0u : t3;
        dw = (uint64_t)s_dig[A[0] & 0xFFu] | ((uint64_t)s_dig[(A[0] >> 8) & 0xFFu] << 15) |
             ((uint64_t)s_dig[(A[0] >> 16) & 0xFFu] << 30) | ((uint64_t)t3 << 45);
#pragma unroll
        for (int k = 0; k < kCols; k++)
            Lw[k] = __funnelshift_r(A[k], A[k + 1], 26);
    } else if (kind == 2) {
        // quints: five 7-bit digit words and a 3-bit one (value 15), then the low parts at bit 38
        uint32_t t5 = (A[1] >> 3) & 7u;
        t5 = t5 >= 5u ? t5 - 5u : t5;
        dw = (uint64_t)s_dig[256u + (A[0] & 0x7Fu)] | ((uint64_t)s_dig[256u + ((A[0] >> 7) & 0x7Fu)] << 9) |
             ((uint64_t)s_dig[256u + ((A[0] >> 14) & 0x7Fu)] << 18) |
             ((uint64_t)s_dig[256u + ((A[0] >> 21) & 0x7Fu)] << 27) |
             ((uint64_t)s_dig[256u + (__funnelshift_r(A[0], A[1], 28) & 0x7Fu)] << 36) | ((uint64_t)t5 << 45);
#pragma unroll
        for (int k = 0; k < kCols - 1; k++)
            Lw[k] = __funnelshift_r(A[k + 1], A[k + 2], 6);
        Lw[kCols - 1] = A[6] >> 6;
    } else {
#pragma unroll
        for (int k = 0; k < kCols; k++)
            Lw[k] = A[k];
    }
#pragma unroll
    for (int k = 0; k < kCols; k++)
        col[k * 32] = Lw[k];
    const uint32_t lmask = (1u << b) - 1u;
    const uint32_t sb = scale << b;
    uint32_t u[kVals];
    uint32_t p = 0;
#pragma unroll
    for (int v = 0; v < kVals; v++) {
        const uint32_t k = p >> 5;
        const uint32_t lo = __funnelshift_r(col[k * 32], col[(k + 1) * 32], p) & lmask;
        const uint32_t d = (uint32_t)(dw >> (3 * v)) & 7u;
        u[v] = d * sb + lo * scale + base;
        p += b;
    }
#pragma unroll
    for (int j = 0; j < 8; j++)
        out[j] = __byte_perm(u[2 * j], u[2 * j + 1], 0x5410);
}

// ---- one block row of a BISE block, any mode ---------------------------------
//
// Four lanes decode one block, lane `rr` its row: values 4rr .. 4rr + 3.
// Their digits lie in at most two consecutive digit groups (A, B) at offsets
// the row table gives; the table lookups return all digits of a group three
// bits apart, and the row's four digits are gathered into one word, digit i
// at bits 3i.  Their low parts lie in one 64-bit window of the payload.  The
// four values come out dequantised and biased, two to a word.  (A last digit
// group that holds one value reads its table's first digit, t mod 3 or t mod
// 5: the same value the stream's shorter last group encodes.)
__device__ __forceinline__ void decode_row_generic(const uint32_t *rec, uint32_t pos, uint32_t hdr, uint32_t q,
                                                   uint32_t rr, const uint32_t *s_mode, const uint16_t *s_dig,
                                                   const uint32_t *s_row, uint32_t &o0, uint32_t &o1)
{
    const uint32_t mp = s_mode[hdr & 31u];
    const uint32_t b = mode_b(mp), kind = mode_kind(mp);
    const uint32_t scale = 1u << (q + ((hdr >> 5) & 3u));
    const int32_t mn = ((int32_t)(hdr << 14)) >> 21;   // header bits 7..17, sign-extended
    const uint32_t base = (uint32_t)mn * scale + 0x4000u;
    uint32_t dg = 0;   // digit i of the row at bits 3i
    uint32_t D = 0;    // digit bits in front of the low parts
    if (kind != 0) {
        const uint32_t *w = rec + (pos >> 5);
        const uint32_t x0 = w[0], x1 = w[1], x2 = w[2];
        const uint64_t win = (uint64_t)__funnelshift_r(x0, x1, pos) | ((uint64_t)__funnelshift_r(x1, x2, pos) << 32);
        const uint32_t r0 = s_row[((kind - 1) * 4 + rr) * 2], r1 = s_row[((kind - 1) * 4 + rr) * 2 + 1];
        const uint32_t tA = (uint32_t)(win >> (r0 & 0xFFu)) & (r1 & 0xFFu);
        const uint32_t tB = (uint32_t)(win >> ((r0 >> 8) & 0xFFu)) & (r1 >> 8);
        const uint32_t toff = kind == 1 ? 0u : 256u;
        const uint32_t dA = s_dig[toff + tA], dB = s_dig[toff + tB];
        dg = (dA >> (3 * ((r0 >> 16) & 15u))) | (dB << (3 * (r0 >> 20)));
        D = kind == 1 ? 26u : 38u;
    }
    const uint32_t lp = pos + D + 4 * rr * b;   // the row's first low part
    const uint32_t *w = rec + (lp >> 5);
    const uint32_t y0 = w[0], y1 = w[1], y2 = w[2];
    const uint32_t lo32 = __funnelshift_r(y0, y1, lp), hi32 = __funnelshift_r(y1, y2, lp);
    const uint32_t lmask = (1u << b) - 1u, sb = scale << b;
    uint32_t u[4];
#pragma unroll
    for (uint32_t i = 0; i < 4; i++) {
        const uint32_t low = __funnelshift_r(lo32, hi32, i * b) & lmask;   // i * b <= 30
        u[i] = ((dg >> (3 * i)) & 7u) * sb + low * scale + base;
    }
    o0 = __byte_perm(u[0], u[1], 0x5410);
    o1 = __byte_perm(u[2], u[3], 0x5410);
}

__device__ __forceinline__ uint32_t clamp_biased_u8(uint32_t x)
{
    // each biased half into [2^14, 2^14 + 255]: its low byte is then the value
    uint32_t r;
    asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(0x40004000u));
    asm("min.u16x2 %0, %0, %1;" : "+r"(r) : "r"(0x40FF40FFu));
    return r;
}

// Inverse YCoCg-R (Section 4) of two pixels held as biased halves; returns
// R, G and B clamped to 8 bits in the low byte of each half.
__device__ __forceinline__ void ycocg_pair_to_rgb(uint32_t y, uint32_t co, uint32_t cg, uint32_t &r, uint32_t &g,
                                                  uint32_t &b)
{
    // (v + 2^14) >> 1 = floor(v / 2) + 2^13 in each half
    const uint32_t hcg = (cg >> 1) & 0x7FFF7FFFu, hco = (co >> 1) & 0x7FFF7FFFu;
    const uint32_t t = y - hcg + kHalfB2;   // y - floor(cg / 2)
    g = clamp_biased_u8(cg + t - kB2);
    const uint32_t bb = t - hco + kHalfB2;  // t - floor(co / 2)
    r = clamp_biased_u8(bb + co - kB2);
    b = clamp_biased_u8(bb);
}

// One block row (four pixels) from its biased Y, Co, Cg pairs: 12 RGB bytes
// in w[0..2] (R0 G0 B0 R1 | G1 B1 R2 G2 | B2 R3 G3 B3) or four packed words.
template <bool kPacked>
__device__ __forceinline__ void row_to_rgb(const uint2 y, const uint2 co, const uint2 cg, uint32_t w[4])
{
    uint32_t r01, g01, b01, r23, g23, b23;
    ycocg_pair_to_rgb(y.x, co.x, cg.x, r01, g01, b01);
    ycocg_pair_to_rgb(y.y, co.y, cg.y, r23, g23, b23);
    const uint32_t t01 = __byte_perm(r01, g01, 0x6240);   // R0 G0 R1 G1
    const uint32_t t23 = __byte_perm(r23, g23, 0x6240);   // R2 G2 R3 G3
    if (kPacked) {
        w[0] = __byte_perm(t01, b01, 0x0410) & 0xFFFFFFu;
        w[1] = __byte_perm(t01, b01, 0x0632) & 0xFFFFFFu;
        w[2] = __byte_perm(t23, b23, 0x0410) & 0xFFFFFFu;
        w[3] = __byte_perm(t23, b23, 0x0632) & 0xFFFFFFu;
    } else {
        w[0] = __byte_perm(t01, b01, 0x2410);
        w[1] = __byte_perm(__byte_perm(t01, b01, 0x0063), t23, 0x5410);
        w[2] = __byte_perm(b23, t23, 0x2760);
        w[3] = 0;
    }
}

// Store one location's block row (four pixels from column x) at dst, the
// output address of pixel x of that row.
template <bool kPacked>
__device__ __forceinline__ void store_row(const Args &a, uint8_t *dst, uint32_t x, const uint32_t w[4])
{
    const bool whole = x + 4 <= a.W;
    if (kPacked) {
        uint32_t *d = reinterpret_cast<uint32_t *>(dst);
        if (whole && a.vec16) {
            *reinterpret_cast<uint4 *>(d) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            for (uint32_t k = 0; k < 4 && x + k < a.W; k++)
                d[k] = w[k];
        }
    } else {
        if (whole && a.vec8) {
            // 12 bytes in two stores: 8 + 4 at an even location, 4 + 8 at an odd one
            const bool even = ((x >> 2) & 1u) == 0;
            *reinterpret_cast<uint2 *>(dst + (even ? 0 : 4)) = even ? make_uint2(w[0], w[1]) : make_uint2(w[1], w[2]);
            *reinterpret_cast<uint32_t *>(dst + (even ? 8 : 0)) = even ? w[2] : w[0];
        } else if (whole && a.vec4) {
            uint32_t *d = reinterpret_cast<uint32_t *>(dst);
            d[0] = w[0];
            d[1] = w[1];
            d[2] = w[2];
        } else {
            for (uint32_t k = 0; k < 12 && x + k / 3 < a.W; k++)
                dst[k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
        }
    }
}

// Address of pixel (x, y) of output view slot ov.
template <bool kPacked>
__device__ __forceinline__ uint8_t *out_px(const Args &a, uint32_t ov, uint32_t y, uint32_t x)
{
    return a.out + (((size_t)ov * a.H + y) * a.W + x) * (kPacked ? 4u : 3u);
}

template <bool kPacked, typename OffT>
__global__ void __launch_bounds__(kThreads, 3) decode_all_kernel(const Args a)
{
    __shared__ uint32_t s_mode[32];
    __shared__ uint16_t s_dig[256 + 128];
    __shared__ uint32_t s_row[16];
    __shared__ uint32_t s_roff[kRecs];
    __shared__ uint32_t s_unit;   // next unit of view work
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bx0 = blockIdx.x * kNL, by = blockIdx.y;
    const uint32_t nl = min((uint32_t)kNL, a.nlx - bx0);
    const uint32_t b0 = by * a.nlx + bx0;
    Smem m;
    layout<kPacked>(g_smem, a, sizeof(OffT), &m);
    OffT *m_off = reinterpret_cast<OffT *>(m.off);
    constexpr uint32_t RW = row_words<kPacked>();
    const uint32_t *nodes = a.node_smem ? m.node : a.node_info;

    // ---- set-up: tables, the strip's records and top-RKV blocks, zero reconstructions
    if (tid < 32)
        s_mode[tid] = g_tables.mode[tid];
    if (tid < (256 + 128) / 2)
        reinterpret_cast<uint32_t *>(s_dig)[tid] = reinterpret_cast<const uint32_t *>(g_tables.dig)[tid];
    if (tid < 16)
        s_row[tid] = (&g_tables.row[0][0][0])[tid];
    if (tid == 0)
        s_unit = 0;
    // the strip's records are contiguous in the stream: stage them (from a
    // 16-byte boundary, plus the eight words the decoder may read past a
    // payload; the stream ends in zero padding) when they fit
    const uint32_t w_lo = __ldg(a.offsets + 3 * b0) & ~3u;
    const uint32_t n4 = (__ldg(a.offsets + 3 * (b0 + nl)) + 8 - w_lo + 3) / 4;
    const bool staged = 4 * n4 <= a.stage_words;
    if (staged) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.records + w_lo);
        uint4 *dst = reinterpret_cast<uint4 *>(m.stage);
        for (uint32_t i = tid; i < n4; i += kThreads)
            dst[i] = __ldg(src + i);
    }
    const uint32_t *rb = staged ? m.stage : a.records;   // records base: smem copy or stream
    if (tid < kRecs)
        s_roff[tid] = tid < 3 * (int)nl ? __ldg(a.offsets + 3 * b0 + tid) - (staged ? w_lo : 0u) : 0u;
    {
        const uint32_t *tg = reinterpret_cast<const uint32_t *>(a.top);
        for (uint32_t i = tid; i < a.n_top * kNL * 24; i += kThreads) {
            const uint32_t t = i / (kNL * 24), rest = i - t * (kNL * 24), loc = rest / 24, wi = rest - loc * 24;
            m.top[i] = loc < nl ? (__ldg(tg + ((size_t)t * a.nloc + b0 + loc) * 24 + wi) ^ 0x80008000u) - kB2 : kB2;
        }
    }
    uint32_t *wslots = m.slots + warp * (8 * (kWSlots + 1));   // this warp's slots
    uint32_t *wcol = m.cols + warp * (kCols * 32) + lane;      // this lane's decoder column
    uint32_t *wsent = m.sent + warp * kWSlots;
    uint32_t *witems = m.items + warp * kWItems;
    if (lane < 8)
        wslots[kZeroSlot * 8 + lane] = kB2;   // the warp's zero slot
    if (a.node_smem)
        for (uint32_t i = tid; i < a.S; i += kThreads)
            m.node[i] = __ldg(a.node_info + i);
    __syncthreads();
    // the views to decode, one bit per BFS position (internal positions 0)
    for (uint32_t w0 = warp * 32; w0 < a.MW * 32; w0 += kWarps * 32) {
        const uint32_t p = w0 + lane;
        bool need = p >= a.n_int && p < a.S;
        if (need && kPacked && a.needed)
            need = __ldg(a.needed + node_view(nodes[p])) != 0;
        const unsigned bal = __ballot_sync(kFullMask, need);
        if (lane == 0)
            m.need[w0 >> 5] = bal;
    }

    // ---- phases 1 and 2, one warp per location l of the strip (no CTA-wide
    // step until the views): parse the location's three records, reconstruct
    // its internal nodes level by level, convert its view parents to RGB
    const uint32_t hdr0 = 32 * a.MW;
    const uint32_t l = warp;
    if (l < nl) {
        // 1. per record: mask words, stored blocks in front of each, payload offsets
        for (uint32_t c = 0; c < 3; c++) {
            const uint32_t r = 3 * l + c;
            uint32_t *mk = m.mask + r * a.MW;
            uint32_t *mp = m.mpre + r * a.MW;
            const uint32_t *rec = rb + s_roff[r];
            uint32_t P = 0;
            for (uint32_t w0 = 0; w0 < a.MW; w0 += 32) {
                const uint32_t word = w0 + lane < a.MW ? rec[w0 + lane] : 0u;
                const uint32_t cnt = (uint32_t)__popc(word);
                const uint32_t incl = warp_inclusive_scan(cnt, lane);
                if (w0 + lane < a.MW) {
                    mk[w0 + lane] = word;
                    mp[w0 + lane] = P + incl - cnt;
                }
                P += __shfl_sync(kFullMask, incl, 31);
            }
            uint32_t run = hdr0 + kHdrBits * P;
            for (uint32_t h0 = 0; h0 < P; h0 += 32) {
                const uint32_t h = h0 + lane;
                uint32_t len = 0;
                if (h < P) {
                    const uint32_t bp = hdr0 + kHdrBits * h;
                    len = mode_bits(s_mode[__funnelshift_r(rec[bp >> 5], rec[(bp >> 5) + 1], bp) & 31u]);
                }
                const uint32_t incl = warp_inclusive_scan(len, lane);
                if (h < P)
                    m_off[r * a.pmax + h] = (OffT)(run + incl - len);
                run += __shfl_sync(kFullMask, incl, 31);
            }
        }
        __syncwarp();
        // 2. internal nodes, level by level from the top: reconstruction =
        // parent reconstruction (top RKV or a node of the level above) +
        // the decoded residual where a block is stored.  Per chunk of 32
        // (node, channel) pairs: the stored ones are decoded into the warp's
        // slots, four lanes per block, then one lane per pair adds.
        for (uint32_t lv = 0; lv + 2 < a.L; lv++) {
            const uint32_t g0 = a.lvl_begin[lv], g1 = a.lvl_begin[lv + 1];
            const uint32_t *src = lv == 0 ? m.top : m.inter;
            for (uint32_t q0 = 0; q0 < (g1 - g0) * 3; q0 += 32) {
                const uint32_t q = q0 + lane;
                const bool valid = q < (g1 - g0) * 3;
                const uint32_t p = g0 + q / 3, c = q - 3 * (q / 3), r = 3 * l + c;
                uint32_t word = 0;
                if (valid)
                    word = m.mask[r * a.MW + (p >> 5)];
                const bool stored = valid && ((word >> (p & 31u)) & 1u);
                const unsigned bal = __ballot_sync(kFullMask, stored);
                const uint32_t my_slot = __popc(bal & ((1u << lane) - 1u));
                if (stored)
                    wsent[my_slot] = r | ((m.mpre[r * a.MW + (p >> 5)] + __popc(word & ((1u << (p & 31u)) - 1u))) << 8);
                __syncwarp();
                const uint32_t n_st = __popc(bal);
                for (uint32_t t0 = 0; t0 < n_st; t0 += 8) {
                    const uint32_t t = t0 + (lane >> 2), rr = lane & 3u;
                    if (t < n_st) {
                        const uint32_t e = wsent[t], rs = e & 255u, rank = e >> 8;
                        const uint32_t *rec = rb + s_roff[rs];
                        const uint32_t bp = hdr0 + kHdrBits * rank;
                        const uint32_t hdr = __funnelshift_r(rec[bp >> 5], rec[(bp >> 5) + 1], bp) & 0x3FFFFu;
                        uint32_t o0, o1;
                        decode_row_generic(rec, m_off[rs * a.pmax + rank], hdr, a.q, rr, s_mode, s_dig, s_row, o0, o1);
                        *reinterpret_cast<uint2 *>(wslots + t * 8 + 2 * rr) = make_uint2(o0, o1);
                    }
                }
                __syncwarp();
                if (valid) {
                    const uint32_t sl = stored ? my_slot : (uint32_t)kZeroSlot;
                    const uint4 *ps = reinterpret_cast<const uint4 *>(src + (node_parent(nodes[p]) * kNL + l) * 24 + c * 8);
                    uint4 *pd = reinterpret_cast<uint4 *>(m.inter + (p * kNL + l) * 24 + c * 8);
                    const uint4 s0 = ps[0], s1 = ps[1];
                    const uint4 v0 = *reinterpret_cast<const uint4 *>(wslots + sl * 8);
                    const uint4 v1 = *reinterpret_cast<const uint4 *>(wslots + sl * 8 + 4);
                    pd[0] = make_uint4(s0.x + v0.x - kB2, s0.y + v0.y - kB2, s0.z + v0.z - kB2, s0.w + v0.w - kB2);
                    pd[1] = make_uint4(s1.x + v1.x - kB2, s1.y + v1.y - kB2, s1.z + v1.z - kB2, s1.w + v1.w - kB2);
                }
                __syncwarp();
            }
        }
        // 3. the location's block rows of every parent of a view, as RGB
        const uint32_t *src = a.L == 2 ? m.top : m.inter;
        for (uint32_t q = lane; q < a.n_par * 4; q += 32) {
            const uint32_t n = q >> 2, rr = q & 3u;
            const uint32_t *sl = src + ((a.par_base + n) * kNL + l) * 24 + rr * 2;
            uint32_t w[4];
            row_to_rgb<kPacked>(*reinterpret_cast<const uint2 *>(sl), *reinterpret_cast<const uint2 *>(sl + 8),
                                *reinterpret_cast<const uint2 *>(sl + 16), w);
            uint32_t *d = m.prgb + ((n * 4 + rr) * kNL + l) * RW;
#pragma unroll
            for (uint32_t k = 0; k < RW; k++)
                d[k] = w[k];
        }
    } else {
        // locations past the end of the row: nothing stored
        for (uint32_t c = 0; c < 3; c++)
            for (uint32_t w = lane; w < a.MW; w += 32) {
                m.mask[(3 * l + c) * a.MW + w] = 0;
                m.mpre[(3 * l + c) * a.MW + w] = 0;
            }
    }
    __syncthreads();

    // ---- phase 3: the views, one unit of kUnit positions at a time per warp
    const uint32_t *par_slab = a.L == 2 ? m.top : m.inter;
    const size_t row_bytes = (size_t)a.W * (kPacked ? 4u : 3u);
    const uint32_t u_first = a.n_int / kUnit;
    const uint32_t nrows = min(4u, a.H - by * 4);
    const bool pairs = a.sec32 && nl == (uint32_t)kNL;   // whole 32-byte-aligned strip rows
    for (;;) {
        uint32_t u = 0;
        if (lane == 0)
            u = atomicAdd(&s_unit, 1u);
        u = __shfl_sync(kFullMask, u, 0) + u_first;
        if (u >= a.n_units)
            break;
        const uint32_t w = u >> 1, ub = 16u * (u & 1u);   // the unit is bits [ub, ub + 16) of mask word w
        const uint32_t P0 = max(u * kUnit, a.n_int), P1 = min(u * kUnit + kUnit, a.S);
        const uint32_t lo = P0 - w * 32, hi = P1 - w * 32;
        const uint32_t sel = (hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u) & m.need[w];
        // (a) copies: lane = (position, group of four locations), four block
        // rows each: the parent's RGB rows, the exact result for every block
        // without a stored residual
        {
            const uint32_t bit = ub + ((uint32_t)lane >> 1), g = lane & 1u, l0 = 4u * g;
            const bool act = ((sel >> bit) & 1u) && l0 < nl;
            const uint32_t info = act ? nodes[w * 32 + bit] : 0u;
            const uint32_t ov = act ? (a.slot_of ? __ldg(a.slot_of + node_view(info)) : node_view(info)) : 0u;
            const uint32_t *src = m.prgb + (act ? ((node_parent(info) - a.par_base) * 4 * kNL + l0) * RW : 0u);
            if (pairs) {
                // the two lanes of a view swap chunks so that every store
                // instruction writes whole 32-byte sectors (lane 0 the even
                // 16-byte chunks of the row, lane 1 the odd ones)
                uint8_t *dst = out_px<kPacked>(a, ov, by * 4, bx0 * 4);
#pragma unroll
                for (uint32_t rr = 0; rr < 4; rr++) {
                    if (rr < nrows) {
                        const uint4 *s4 = reinterpret_cast<const uint4 *>(src + rr * kNL * RW);
                        uint4 *d4 = reinterpret_cast<uint4 *>(dst + rr * row_bytes);
                        if (kPacked) {
                            const uint4 c0 = s4[0], c1 = s4[1], c2 = s4[2], c3 = s4[3];
                            const uint4 t0 = g ? c0 : c1, t1 = g ? c2 : c3;
                            uint4 r0, r1;
                            r0.x = __shfl_xor_sync(kFullMask, t0.x, 1); r0.y = __shfl_xor_sync(kFullMask, t0.y, 1);
                            r0.z = __shfl_xor_sync(kFullMask, t0.z, 1); r0.w = __shfl_xor_sync(kFullMask, t0.w, 1);
                            r1.x = __shfl_xor_sync(kFullMask, t1.x, 1); r1.y = __shfl_xor_sync(kFullMask, t1.y, 1);
                            r1.z = __shfl_xor_sync(kFullMask, t1.z, 1); r1.w = __shfl_xor_sync(kFullMask, t1.w, 1);
                            if (act) {
                                d4[0 + g] = g ? r0 : c0;
                                d4[2 + g] = g ? r1 : c2;
                                d4[4 + g] = g ? c1 : r0;
                                d4[6 + g] = g ? c3 : r1;
                            }
                        } else {
                            const uint4 c0 = s4[0], c1 = s4[1], c2 = s4[2];
                            uint4 x1;
                            x1.x = __shfl_xor_sync(kFullMask, c1.x, 1); x1.y = __shfl_xor_sync(kFullMask, c1.y, 1);
                            x1.z = __shfl_xor_sync(kFullMask, c1.z, 1); x1.w = __shfl_xor_sync(kFullMask, c1.w, 1);
                            if (act) {
                                d4[0 + g] = g ? x1 : c0;
                                d4[2 + g] = g ? c0 : c2;
                                d4[4 + g] = g ? c2 : x1;
                            }
                        }
                    }
                }
            } else if (act) {
                const uint32_t x = (bx0 + l0) * 4;
                uint8_t *dst = out_px<kPacked>(a, ov, by * 4, x);
                const bool fast = a.vec16 && l0 + 4 <= nl && x + 16 <= a.W;
                for (uint32_t rr = 0; rr < nrows; rr++) {
                    if (fast) {
                        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
                        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll
                        for (uint32_t kk = 0; kk < RW; kk++)
                            d4[kk] = s4[kk];
                    } else {
                        for (uint32_t l = l0; l < min(l0 + 4, nl); l++) {
                            uint32_t wv[4];
#pragma unroll
                            for (uint32_t kk = 0; kk < RW; kk++)
                                wv[kk] = src[(l - l0) * RW + kk];
                            store_row<kPacked>(a, dst + (l - l0) * 4 * (kPacked ? 4u : 3u), (bx0 + l) * 4, wv);
                        }
                    }
                    src += kNL * RW;
                    dst += row_bytes;
                }
            }
        }
        // lanes 0..kNL-1 hold location `lane`'s three channel masks: full
        // (ranks) and restricted to the unit's views to decode
        uint32_t f0 = 0, f1 = 0, f2 = 0;
        if (lane < kNL) {
            f0 = m.mask[(3 * lane) * a.MW + w];
            f1 = m.mask[(3 * lane + 1) * a.MW + w];
            f2 = m.mask[(3 * lane + 2) * a.MW + w];
        }
        const uint32_t ns_l = (uint32_t)(__popc(f0 & sel) + __popc(f1 & sel) + __popc(f2 & sel));
        const uint32_t ni_l = (uint32_t)__popc((f0 | f1 | f2) & sel);
        // (b) runs of locations [l0, l1) whose stored blocks fit the warp's slots
        for (uint32_t l0 = 0; l0 < kNL;) {
            const bool in0 = (uint32_t)lane >= l0 && lane < kNL;
            const uint32_t run = warp_inclusive_scan(in0 ? ns_l : 0u, lane);
            const unsigned fit = __ballot_sync(kFullMask, in0 && run <= (uint32_t)kWSlots);
            const uint32_t l1 = max(l0 + 1, 32u - (uint32_t)__clz(fit));
            const bool in = (uint32_t)lane >= l0 && (uint32_t)lane < l1;
            const uint32_t cnt = in ? (ni_l | (ns_l << 16)) : 0u;
            const uint32_t incl = warp_inclusive_scan(cnt, lane);
            const uint32_t excl = incl - cnt;
            const uint32_t totals = __shfl_sync(kFullMask, incl, 31);
            const uint32_t n_items = totals & 0xFFFFu, n_slots = totals >> 16;
            // items are numbered view-major (a view's locations in order), so
            // that lanes of the conversion below write neighbouring blocks of
            // one output row together; slots stay location-major.  Lane v < 16:
            // the run's locations holding an item of view ub + v, and the
            // items of the views before it.
            uint32_t vrow = 0;
            for (uint32_t l = l0; l < l1; l++) {
                const uint32_t al = __shfl_sync(kFullMask, (f0 | f1 | f2) & sel, l);
                vrow |= ((al >> ((ub + lane) & 31u)) & 1u) << l;
            }
            vrow = lane < kUnit ? vrow : 0u;
            const uint32_t vcnt = (uint32_t)__popc(vrow);
            const uint32_t vbase = warp_inclusive_scan(vcnt, lane) - vcnt;
            // items and slots: lane = (location, position) pairs of the run
            for (uint32_t q0 = 0; q0 < (l1 - l0) * kUnit; q0 += 32) {
                const uint32_t q = q0 + lane;
                const uint32_t l = min(l0 + (q >> 4), (uint32_t)kNL - 1u), bit = ub + (q & 15u);
                const uint32_t g0 = __shfl_sync(kFullMask, f0, l), g1 = __shfl_sync(kFullMask, f1, l),
                               g2 = __shfl_sync(kFullMask, f2, l), eb = __shfl_sync(kFullMask, excl, l);
                const uint32_t vb = __shfl_sync(kFullMask, vbase, q & 15u), vr = __shfl_sync(kFullMask, vrow, q & 15u);
                const bool valid = q < (l1 - l0) * kUnit;
                const uint32_t m0 = valid ? g0 & sel : 0u, m1 = valid ? g1 & sel : 0u, m2 = valid ? g2 & sel : 0u;
                const uint32_t st3 = ((m0 >> bit) & 1u) | (((m1 >> bit) & 1u) << 1) | (((m2 >> bit) & 1u) << 2);
                if (st3) {
                    const uint32_t lt = (1u << bit) - 1u;
                    const uint32_t item = vb + __popc(vr & ((1u << l) - 1u));
                    uint32_t slot = (eb >> 16) + __popc(m0 & lt) + __popc(m1 & lt) + __popc(m2 & lt);
                    witems[item] = (w * 32 + bit) | (l << 14) | (st3 << 18) | (slot << 21);
                    if (st3 & 1u)
                        wsent[slot++] = (3 * l) | ((m.mpre[(3 * l) * a.MW + w] + __popc(g0 & lt)) << 8);
                    if (st3 & 2u)
                        wsent[slot++] = (3 * l + 1) | ((m.mpre[(3 * l + 1) * a.MW + w] + __popc(g1 & lt)) << 8);
                    if (st3 & 4u)
                        wsent[slot] = (3 * l + 2) | ((m.mpre[(3 * l + 2) * a.MW + w] + __popc(g2 & lt)) << 8);
                }
            }
            __syncwarp();
            // decode every slot of the run, one lane each
            for (uint32_t t = lane; t < n_slots; t += 32) {
                const uint32_t e = wsent[t];
                const uint32_t r = e & 255u, rank = e >> 8;
                const uint32_t *rec = rb + s_roff[r];
                const uint32_t bp = hdr0 + kHdrBits * rank;
                const uint32_t hdr = __funnelshift_r(rec[bp >> 5], rec[(bp >> 5) + 1], bp) & 0x3FFFFu;
                uint32_t v[8];
                decode_block_generic(rec, m_off[r * a.pmax + rank], hdr, a.q, s_mode, s_dig, wcol, v);
                uint4 *d = reinterpret_cast<uint4 *>(wslots + t * 8);
                d[0] = make_uint4(v[0], v[1], v[2], v[3]);
                d[1] = make_uint4(v[4], v[5], v[6], v[7]);
            }
            __syncwarp();
            // items: parent + residual -> RGB, one lane per item, four block rows each
            for (uint32_t i = lane; i < n_items; i += 32) {
                const uint32_t it = witems[i];
                const uint32_t p = it & 0x3FFFu, l = (it >> 14) & 15u, st3 = (it >> 18) & 7u, s0 = it >> 21;
                const uint32_t info = nodes[p];
                const uint32_t *ps = par_slab + (node_parent(info) * kNL + l) * 24;
                // slot of each channel's residual, or the zero slot
                const uint32_t *ry = wslots + 8 * ((st3 & 1u) ? s0 : (uint32_t)kZeroSlot);
                const uint32_t *rco = wslots + 8 * ((st3 & 2u) ? s0 + (st3 & 1u) : (uint32_t)kZeroSlot);
                const uint32_t *rcg = wslots + 8 * ((st3 & 4u) ? s0 + __popc(st3 & 3u) : (uint32_t)kZeroSlot);
                const uint32_t ov = a.slot_of ? __ldg(a.slot_of + node_view(info)) : node_view(info);
                const uint32_t x = (bx0 + l) * 4;
                uint8_t *dst = out_px<kPacked>(a, ov, by * 4, x);
#pragma unroll
                for (uint32_t rr = 0; rr < 4; rr++) {
                    if (rr < nrows) {
                        const uint32_t j = 2 * rr;
                        const uint2 py = *reinterpret_cast<const uint2 *>(ps + j);
                        const uint2 pco = *reinterpret_cast<const uint2 *>(ps + 8 + j);
                        const uint2 pcg = *reinterpret_cast<const uint2 *>(ps + 16 + j);
                        const uint2 vy = *reinterpret_cast<const uint2 *>(ry + j);
                        const uint2 vco = *reinterpret_cast<const uint2 *>(rco + j);
                        const uint2 vcg = *reinterpret_cast<const uint2 *>(rcg + j);
                        uint32_t wv[4];
                        row_to_rgb<kPacked>(make_uint2(py.x + vy.x - kB2, py.y + vy.y - kB2),
                                            make_uint2(pco.x + vco.x - kB2, pco.y + vco.y - kB2),
                                            make_uint2(pcg.x + vcg.x - kB2, pcg.y + vcg.y - kB2), wv);
                        store_row<kPacked>(a, dst + rr * row_bytes, x, wv);
                    }
                }
            }
            __syncwarp();
            l0 = l1;
        }
    }
}

template <bool kPacked>
int launch_decode(const rlfc_stream *s, uint8_t *d_out, const uint8_t *needed, const uint32_t *slot_of, cudaStream_t st)
{
    const Tables &t = s->tab;
    Args a;
    a.records = s->d_records;
    a.offsets = s->d_offsets;
    a.top = s->d_top;
    a.node_info = s->d_node_info;
    a.out = d_out;
    a.needed = needed;
    a.slot_of = slot_of;
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
    // parents of views: the level-1 nodes (the last internal positions) or the tops
    if (t.L == 2) {
        a.par_base = 0;
        a.n_par = t.n_top;
    } else {
        uint32_t n1 = 0;
        for (uint32_t p = 0; p < t.n_int; p++)
            n1 += node_level(t.node_info[p]) == 1;
        a.par_base = t.n_int - n1;
        a.n_par = n1;
    }
    if (kPacked) {
        a.vec16 = ((uintptr_t)d_out & 15u) == 0 && (a.W & 3u) == 0;
        a.vec4 = a.vec16;
        a.vec8 = 0;
        a.sec32 = ((uintptr_t)d_out & 31u) == 0 && (a.W & 7u) == 0;
    } else {
        a.vec16 = ((uintptr_t)d_out & 15u) == 0 && (a.W & 15u) == 0;
        a.vec4 = ((uintptr_t)d_out & 3u) == 0 && (a.W & 3u) == 0;
        a.vec8 = ((uintptr_t)d_out & 7u) == 0 && (a.W & 7u) == 0;
        a.sec32 = ((uintptr_t)d_out & 31u) == 0 && (a.W & 31u) == 0;
    }
    a.pmax = std::max<uint32_t>(s->max_present, 1);
    a.n_units = (t.S + kUnit - 1) / kUnit;
    a.node_smem = t.S <= kNodeSmemMax;
    // internal levels in BFS order: L-2 first, down to 1
    for (uint32_t k = 0; k < (uint32_t)kMaxLevels; k++)
        a.lvl_begin[k] = t.n_int;
    for (uint32_t lv = 0; lv + 2 < t.L; lv++) {
        const uint32_t level = t.L - 2 - lv;
        uint32_t p = 0;
        while (p < t.n_int && node_level(t.node_info[p]) != level)
            p++;
        a.lvl_begin[lv] = p;
    }
    // payload offsets are bit positions inside one record: 16 bits suffice
    // unless a record reaches 2^16 bits
    const bool off16 = (uint64_t)s->max_record_words * 32 < 65536;
    const size_t off_size = off16 ? 2 : 4;
    // staging for the largest strip's records (16-byte boundary, decoder
    // slack), within what keeps three CTAs per SM; strips whose records do
    // not fit read them from the stream
    a.stage_words = 0;
    const size_t base = layout<kPacked>(nullptr, a, off_size, nullptr);
    const size_t room = base < kCtaSmemTarget ? (kCtaSmemTarget - base) / 4 : 0;
    a.stage_words = (uint32_t)std::min<size_t>((size_t)((s->max_strip_words + 8 + 3 + 3) & ~3u), room & ~size_t(3));
    const size_t smem = layout<kPacked>(nullptr, a, off_size, nullptr);
    if (smem > kSmemBudget || a.S >= 16384) {
        set_error("tree too large for the decode-all kernel's shared memory");
        return RLFC_E_UNSUPPORTED;
    }
    auto kern = off16 ? decode_all_kernel<kPacked, uint16_t> : decode_all_kernel<kPacked, uint32_t>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "decode_all: shared memory attribute");
    dim3 grid((a.nlx + kNL - 1) / kNL, s->info.nloc_y);
    { rlfc::TraceScope trace_((kPacked ? "decode_all_kernel<packed>" : "decode_all_kernel"), st); kern<<<grid, kThreads, smem, st>>>(a); }
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "decode_all launch");
    return RLFC_OK;
}

}  // namespace

int launch_decode_all(const rlfc_stream *s, uint8_t *d_out, cudaStream_t st)
{
    return launch_decode<false>(s, d_out, nullptr, nullptr, st);
}

int launch_decode_packed(const rlfc_stream *s, uint32_t *d_out, const uint8_t *needed, const uint32_t *slot_of,
                         cudaStream_t st)
{
    return launch_decode<true>(s, reinterpret_cast<uint8_t *>(d_out), needed, slot_of, st);
}

}  // namespace rlfc
